"""The GPU path on the paper's validation cases at the paper's sizes (Sec.
3.1), where the FP64 oracle is too slow to follow: the physics pins of the
oracle (closed forms and the paper's statements) applied to the CUDA results
directly, in FP32 and in the 16-bit storage forms."""
import numpy as np
import pytest

from paper_2101_06769_gb300 import Domain
from paper_2101_06769_gb300.lbmp import BF16_SHIFTED, FP16_SHIFTED, FP32

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("r", [25, 35, 45])
@pytest.mark.parametrize("sigma", [1e-3, 1e-1])
def test_laplace_law_paper_grid(r, sigma):
    """Sec. 3.1: static drop on 256^2, density ratio 20, nu = 0.1, W = 5 (reading
    A19): the converged pressure jump follows Delta P = sigma / r within 5 %
    (measured 0.953-0.955 sigma / r for r = 25-45; the largest drop needs
    about 16000 steps to converge)."""
    d = Domain(2, (256, 256, 1), (1, 1, 1), rho_ratio=20.0, nu_ratio=1.0, nu_h=0.1, mobility=0.02, width=5.0,
               sigma=sigma)
    d.init("drop_static", [float(r), 1.0, 0.0], seed=1)
    d.step(20000)
    ob = d.observables()
    assert ob.health == 0
    assert abs(ob.laplace_dp / (sigma / r) - 1) < 0.05, ob.laplace_dp / (sigma / r)


@pytest.mark.parametrize("storage", [FP32, FP16_SHIFTED, BF16_SHIFTED])
def test_laplace_law_3d(storage):
    """3-D static drop, W = 5 as in the paper's Laplace test: Delta P = 2 sigma / R
    within 5 % in every storage form (64^3, R = 12; measured 0.968, and
    0.956-0.961 for R = 16-24 on 96^3; an under-resolved W = 4 interface gives
    0.93 instead, a property of the discretised model the oracle shares)."""
    sigma, R = 1e-3, 12.0
    d = Domain(3, (64, 64, 64), (1, 1, 1), rho_ratio=20.0, nu_ratio=1.0, nu_h=0.1, mobility=0.02, width=5.0,
               sigma=sigma, storage=storage)
    d.init("drop_static", [R, 1.0, 0.0], seed=1)
    d.step(4000)
    ob = d.observables()
    assert ob.health == 0 and abs(ob.mass_drift_rel) < 1e-6
    assert abs(ob.laplace_dp / (2 * sigma / R) - 1) < 0.05, ob.laplace_dp / (2 * sigma / R)


def test_spurious_currents_density_ratio_1000_paper_grid():
    """Sec. 3.1: density ratio 1000, sigma = 1e-3: spurious currents of order
    1e-6 (bound 1e-5) on the 256^2 grid."""
    d = Domain(2, (256, 256, 1), (1, 1, 1), rho_ratio=1000.0, nu_ratio=1.0, nu_h=0.1, mobility=0.02, width=5.0,
               sigma=1e-3)
    d.init("drop_static", [45.0, 1.0, 0.0], seed=1)
    d.step(8000)
    ob = d.observables()
    assert ob.health == 0
    assert ob.max_u < 1e-5, ob.max_u


@pytest.mark.parametrize("D,dims", [(2, (128, 128, 1)), (3, (64, 64, 64))])
def test_shear_wave_viscosity(D, dims):
    """Single-phase shear wave: the amplitude decays as exp(-nu k^2 t) with the
    viscosity of reading A7 (within 1 %)."""
    nu = 0.02
    d = Domain(D, dims, (1, 1, 1), rho_ratio=3.0, nu_ratio=1.0, nu_h=nu, mobility=0.02, width=4.0, sigma=0.0)
    d.init("shear_wave", [1e-3, 0.0], seed=1)
    d.step(50)
    e0 = d.observables().kinetic_energy
    T = 2000
    d.step(T)
    e1 = d.observables().kinetic_energy
    k = 2 * np.pi / dims[1]
    nu_meas = -np.log(e1 / e0) / (2 * k * k * T)  # energy decays at twice the amplitude rate
    assert abs(nu_meas / nu - 1) < 0.01, nu_meas


def spread(case, times, slice3d=False):
    """r_K/D (paper_2101_06769_gb300.observe) of a shipped droplet-impact
    case at the given t/T after contact, with the run's health and drift."""
    from paper_2101_06769_gb300 import cases, observe
    c = cases.load(case)
    wl = cases.as_workload(c)
    d = cases.make_domain(c)
    D, sheet, U0 = wl["args"][0], wl["args"][1], wl["args"][2]
    T, t0 = D / U0, observe.contact_time(wl["phys"]["width"], U0)
    nx, ny = wl["dims"][0], wl["dims"][1]
    done, out = 0, []
    for tt in times:
        n = int(round(t0 + tt * T))
        d.step(n - done)
        done = n
        phi = d.get_state()[2]
        plane = phi[:, ny // 2, :] if slice3d else phi[0]
        ob = d.observables()
        if wl["periodic"][0] == 2:  # half domain, the axis on the symmetry face
            r = observe.spreading_radius_half(plane, sheet)
        else:
            r = observe.spreading_radius(plane, sheet, nx // 2)
        out.append((r / D, ob.health, ob.mass_drift_rel))
    d.close()
    return out


# t/T at which r_K is compared with the paper's line, and the lower bound of
# r_K / (1.1 sqrt(t/T)): the neck on the first row above the film is measured
# until the ejected lamella reaches that row (after t/T = 0.2 for the two
# Re = 1000 impacts, 0.5 for Re = 200)
SPLASH = {"splash2d_k56": ((0.25, 0.5), 0.78, 3.0), "splash2d_k83": ((0.15, 0.2), 0.78, 3.0),
          "splash2d_k264": ((0.15, 0.2), 0.78, 3.0), "splash3d": ((0.1, 0.2), 0.5, 4.0)}


@pytest.mark.parametrize("case,slice3d", [("splash2d_k56", False), ("splash2d_k83", False), ("splash2d_k264", False),
                                          ("splash3d", True)])
def test_droplet_splash_spreading_radius(case, slice3d):
    """Sec. 3.4: after impact the neck radius grows like sqrt(t) at first; the
    paper plots r_K/D = 1.1 sqrt(t/T).  The three 2-D impacts (K = 55.7,
    83.4, 263.8; D = 100, W = 5, M = 0.1; half domains with the paper's
    symmetry boundaries) run finite to t/T = 3 and their measured neck
    radius stays within 22 % of that line while the row measurement holds
    (measured 0.81 / 0.84 at t/T = 0.25 / 0.5 for K = 55.7, 0.82 / 0.81 at
    0.15 / 0.2 for K = 83.4 and 263.8); the reduced-size 3-D
    impact (D = 64, W = 4, M = 0.1) grows monotonically at 0.5-1.0 of the
    line at t/T = 0.1, 0.2 (measured 0.60 / 0.78) and runs finite to t/T = 4.
    Every run keeps its mass."""
    (t1, t2), low, t_end = SPLASH[case]
    rows = spread(case, [t1, t2, t_end], slice3d)
    assert all(h == 0 and abs(drift) <= 1e-6 for _, h, drift in rows)
    radii = [r for r, _, _ in rows[:2]]
    assert radii[1] > radii[0], radii
    for tt, r in zip((t1, t2), radii):
        ratio = r / (1.1 * np.sqrt(tt))
        assert low <= ratio <= (1.0 if slice3d else 1.2), (case, tt, r, ratio)


def test_reduced_phase_lattice_physics():
    """The D3Q7 / D2Q5 phase field (first-order equilibrium and correction
    term, Sec. 2.2) on the paper's checks: the Laplace law of the 256^2 drop
    (r = 45, 20000 steps) and of the 64^3 drop (R = 12, 4000 steps) within
    5 % (measured 0.955 and 0.971 of sigma/r and 2 sigma/R, against 0.953 and
    0.968 on the full lattice), spurious currents below 5e-5 (measured 9.6e-6
    and 2.0e-5: a few times the full lattice's 1.2e-6 and 3.0e-6, the
    reduced lattice being less isotropic), and the reduced 3-D RT tips
    within 0.1 cells of the full-lattice run over five time units
    (measured 0.051)."""
    from paper_2101_06769_gb300.lbmp import FLAG_PHASE_REDUCED
    from test_gpu_storage import EVEN
    red = FLAG_PHASE_REDUCED
    d = Domain(2, (256, 256, 1), (1, 1, 1), rho_ratio=20.0, nu_ratio=1.0, nu_h=0.1, mobility=0.02, width=5.0,
               sigma=1e-3, flags=red)
    d.init("drop_static", [45.0, 1.0, 0.0], seed=1)
    d.step(20000)
    ob = d.observables()
    assert ob.health == 0 and abs(ob.laplace_dp / (1e-3 / 45) - 1) < 0.05 and ob.max_u < 5e-5
    d = Domain(3, (64, 64, 64), (1, 1, 1), rho_ratio=20.0, nu_ratio=1.0, nu_h=0.1, mobility=0.02, width=5.0,
               sigma=1e-3, flags=red)
    d.init("drop_static", [12.0, 1.0, 0.0], seed=1)
    d.step(4000)
    ob = d.observables()
    assert ob.health == 0 and abs(ob.laplace_dp / (2e-3 / 12) - 1) < 0.05 and ob.max_u < 5e-5
    c = EVEN["rt3d"]
    T = int(round(c["phys"]["L_ref"] / 0.04))
    tips = []
    for flags in (0, red):
        phys = dict(c["phys"])
        phys["flags"] = flags
        d = Domain(c["D"], c["dims"], c["periodic"], **phys)
        d.init(c["case"], c["args"], seed=c["seed"])
        rec = []
        for _ in range(5):
            d.step(T)
            ob = d.observables()
            assert ob.health == 0 and abs(ob.mass_drift_rel) <= 1e-6
            rec.append((ob.tip_spike, ob.tip_bubble))
        tips.append(np.array(rec))
    assert np.abs(tips[0] - tips[1]).max() <= 0.1
