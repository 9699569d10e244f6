"""Pins of the oracle's observables and initial states against closed forms
and geometry, independent of the oracle's own formulas:

* kinetic energy 1/2 sum rho |u|^2 of flows whose velocity and density are
  known exactly (a uniform flow at a density other than one, a shear wave
  whose sum of sin^2 over a period is N/2);
* max |u| of the same flows (the speed, not its square; the largest, not an
  average);
* the interpolated phi = 1/2 crossings of the spike and bubble columns on
  synthetic columns with a linear crossing, where linear interpolation is
  exact (and on the Rayleigh-Taylor start, whose crossings sit on lattice
  points);
* the drop-on-sheet start: the phi = 1/2 surface passes through the drop's
  top, side and bottom points (centre sheet + D/2 + 2W above the floor,
  radius D/2) and the sheet surface far from the drop, the gap between the
  drop and the sheet holds light fluid, the profile's slope at the surface
  obeys the equilibrium relation dphi/dn = 4 phi (1 - phi)/W of Sec. 2.1,
  and the drop falls at U0 while the fluid far from it is at rest;
* the Rayleigh-Taylor start: the interface heights of the cosine
  perturbation on three columns, and the hydrostatic pressure, whose
  difference over a column equals minus the integral of (rho - rho_bar) g
  (composite Simpson rule on the lattice densities).
"""
import numpy as np
import pytest

import oracle as O


def _sum_sin2(n):
    """sum_{y=0}^{n-1} sin^2(2 pi y / n) = n / 2 for n >= 3"""
    return n / 2.0


def test_kinetic_energy_closed_forms():
    # uniform flow, phi = 0.3 at density ratio 10: rho = rho_l + (rho_h - rho_l) phi
    o = O.Oracle(3, (6, 5, 4), (1, 1, 1), rho_ratio=10.0, nu_h=0.05, sigma=1e-3, width=4.0)
    u0 = np.array([0.012, -0.007, 0.004])
    o.init("uniform", [0.3, 0.01, *u0])
    rho = 0.1 + 0.9 * 0.3
    ob = o.observables()
    want = 0.5 * rho * float(u0 @ u0) * o.N
    assert abs(ob.kinetic_energy / want - 1.0) < 1e-12
    # shear wave u_x = U sin(2 pi y / ny) at phi = 1 (rho = rho_h = 1)
    U = 0.02
    o = O.Oracle(3, (4, 12, 3), (1, 1, 1), nu_h=0.05, width=4.0)
    o.init("shear_wave", [U, 0.0])
    ob = o.observables()
    want = 0.5 * U ** 2 * (4 * 3) * _sum_sin2(12)
    assert abs(ob.kinetic_energy / want - 1.0) < 1e-12


def test_max_speed_closed_forms():
    o = O.Oracle(2, (7, 5, 1), (1, 1, 1), rho_ratio=3.0, nu_h=0.05, sigma=1e-3, width=4.0)
    o.init("uniform", [0.6, 0.0, 0.03, -0.04, 0.0])
    assert abs(o.observables().max_u - 0.05) < 1e-14
    # the shear wave reaches U at y = ny/4 (ny divisible by 4)
    o = O.Oracle(3, (4, 16, 3), (1, 1, 1), nu_h=0.05, width=4.0)
    o.init("shear_wave", [0.03, 0.0])
    assert abs(o.observables().max_u - 0.03) < 1e-14


def _set_columns(o, spike_col, bubble_col, fill):
    """a state at rest whose phi is `fill` everywhere except on the spike
    column (x = nx/2, y = ny/2) and the bubble column (origin)"""
    D = o.D
    nx, ny, nz = o.dims
    phi = np.full((nz, ny, nx), fill)
    if D == 3:
        phi[:, ny // 2, nx // 2] = spike_col
        phi[:, 0, 0] = bubble_col
    else:
        phi[0, :, nx // 2] = spike_col
        phi[0, :, 0] = bubble_col
    _, w = O.lattice(D)
    g = w[:, None, None, None] * phi[None]
    f = np.zeros((o.Q,) + phi.shape)
    o.set_state(f, g)


@pytest.mark.parametrize("D", [2, 3])
def test_tip_interpolation_exact_on_linear_columns(D):
    nv = 48
    dims = (8, nv, 1) if D == 2 else (8, 6, nv)
    per = (1, 0, 1) if D == 2 else (1, 1, 0)
    o = O.Oracle(D, dims, per, rho_ratio=3.0, nu_h=0.05, sigma=1e-3, width=5.0)
    k = np.arange(nv, dtype=float)
    t_spike, t_bubble, slope = 17.3, 31.65, 1.0 / 7.0
    # heavy (phi = 1) on top on both columns, linear through the crossing
    spike = np.clip(0.5 + slope * (k - t_spike), 0.0, 1.0)
    bubble = np.clip(0.5 + slope * (k - t_bubble), 0.0, 1.0)
    _set_columns(o, spike, bubble, fill=1.0)
    ob = o.observables()
    assert abs(ob.tip_spike - t_spike) < 1e-12
    assert abs(ob.tip_bubble - t_bubble) < 1e-12


@pytest.mark.parametrize("D", [2, 3])
def test_rt_start_interface_and_tips(D):
    h0, amp = 20.0, 2.0
    if D == 3:
        dims, per = (16, 12, 40), (1, 1, 0)
    else:
        dims, per = (16, 40, 1), (1, 0, 1)
    o = O.Oracle(D, dims, per, atwood=0.5, nu_ratio=1.0, Re=256.0, g_accel=2.5e-5, L_ref=16.0, width=5.0)
    o.init("rt", [h0, amp, 0.0])
    _, _, phi = o.get_state()
    nx, ny = dims[0], dims[1]
    amp_n = amp * (2 if D == 3 else 1)  # the cosines of x and y add in 3-D

    def col(x, y):
        return phi[:, y, x] if D == 3 else phi[0, :, x]

    # interface (phi = 1/2) at h0 + amp cos(2 pi x/nx) [+ amp cos(2 pi y/ny)]
    assert abs(col(0, 0)[int(h0 + amp_n)] - 0.5) < 1e-12                # both cosines +1
    assert abs(col(nx // 2, 0)[int(h0 + (0 if D == 3 else -amp))] - 0.5) < 1e-12
    if D == 3:
        assert abs(col(nx // 2, ny // 2)[int(h0 - amp_n)] - 0.5) < 1e-12  # both cosines -1
    assert col(0, 0)[-1] > 0.99 and col(0, 0)[0] < 0.01  # heavy fluid on top
    ob = o.observables()
    assert abs(ob.tip_bubble - (h0 + amp_n)) < 1e-12
    assert abs(ob.tip_spike - (h0 - amp_n)) < 1e-12


def test_rt_hydrostatic_start():
    """dp/dz = -(rho - rho_bar) g: the pressure difference along a column
    equals minus the integral of (rho - rho_bar) g over it."""
    W, g, h0 = 8.0, 1e-4, 30.0
    o = O.Oracle(3, (8, 6, 60), (1, 1, 0), atwood=0.5, nu_ratio=1.0, Re=256.0, g_accel=g, L_ref=8.0, width=W)
    o.init("rt", [h0, 0.0, 0.0, 1.0])
    d = o.derived()
    rho, _, _ = o.fields()
    f, _, _ = o.get_state()
    p = f.sum(axis=0)  # the pressure the start sets: P = sum f' (u = 0, sum of f'_eq = w p + rho cs2 (Gamma - w))
    rho_bar = 0.5 * (d.rho_h + d.rho_l)
    colr, colp = rho[:, 2, 3], p[:, 2, 3]
    for z1, z2 in ((10, 50), (22, 38), (30, 46)):
        zz = np.arange(z1, z2 + 1)
        f = -(colr[zz] - rho_bar) * g
        simpson = (f[0] + f[-1] + 4 * f[1:-1:2].sum() + 2 * f[2:-1:2].sum()) / 3.0
        dp = colp[z2] - colp[z1]
        assert abs(dp - simpson) <= 1e-3 * abs(simpson) + 1e-15, (z1, z2, dp, simpson)
    # p vanishes on the interface and is the same on every column of a flat start
    assert abs(colp[int(h0)]) < 1e-15
    assert np.abs(p - p[:, :1, :1]).max() < 1e-15


def test_drop_sheet_start_geometry():
    Dd, sheet, W, U0 = 16.0, 4.0, 4.0, 0.05
    n = 48
    o = O.Oracle(3, (n, n, 40), (1, 1, 0), rho_ratio=1000.0, nu_ratio=15.0, We=8000.0, Re=1000.0, U0=U0,
                 L_ref=Dd, width=W)
    o.init("drop_sheet", [Dd, sheet, U0, 0.0])
    _, _, phi = o.get_state()
    c = n // 2
    zc = int(sheet + Dd / 2 + 2 * W)  # 20: two interface widths of light fluid between drop and sheet
    R = int(Dd / 2)
    # the phi = 1/2 surface: drop top, side, bottom, and the sheet far from the drop
    for (x, y, z) in ((c, c, zc + R), (c + R, c, zc), (c, c - R, zc), (c, c, zc - R), (0, 0, int(sheet))):
        assert abs(phi[z, y, x] - 0.5) < 1e-12, (x, y, z, phi[z, y, x])
    assert phi[zc, c, c] > 0.99 and phi[1, 0, 0] > 0.95          # inside the drop and the sheet
    assert phi[zc - R - int(W), c, c] < 0.02                       # the gap is light fluid
    assert phi[39, 0, 0] < 1e-6 and phi[zc, 0, 0] < 1e-6
    # slope at the drop's top surface against dphi/dn = 4 phi (1 - phi)/W
    # (central difference over two cells: within 10 % for W = 4)
    col = phi[:, c, c]
    slope = 0.5 * (col[zc + R - 1] - col[zc + R + 1])
    assert abs(slope / (4 * 0.5 * 0.5 / W) - 1.0) < 0.1
    # the drop falls at U0, the fluid far from it is at rest (the velocity
    # observable adds the half force F/(2 rho): surface tension at the
    # interfaces leaves horizontal speeds far below U0)
    _, _, u = o.fields()
    assert abs(u[2, zc, c, c] / -U0 - 1.0) < 1e-3
    assert np.abs(u[:2]).max() < 1e-4 * U0
    assert abs(u[2, 30, 0, 0]) < 1e-6 * U0
