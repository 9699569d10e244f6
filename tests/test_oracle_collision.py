"""Pins of one-cell collision identities and whole-step invariants of the
oracle (Sec. 2.2 and 2.3).

Closed-form identities per cell, exact for the second-order Hermite
equilibrium on D2Q9 / D3Q27:
    sum_a Xi_a          = cs2 u . grad(rho)
    sum_a c_a Xi_a      = cs2 F
    sum f'* - sum f'    = sum Xi
    sum c f'* - sum c f'= cs2 F
    sum g* = sum g when phi = sum g,  sum c g* = (1-1/tau) sum c g + phi u/tau + lambda cs2 n X
and with every relaxation rate equal to one the post-collision state is the
product-form equilibrium whatever the pre-collision populations were.
"""
import numpy as np
import pytest

import oracle as O

CS2 = 1.0 / 3.0


def make(D, **kw):
    dims = (4, 4, 1) if D == 2 else (4, 4, 4)
    p = dict(rho_ratio=20.0, nu_ratio=3.0, nu_h=0.05, mobility=0.02, width=5.0, sigma=1e-2,
             g_accel=1e-4)
    p.update(kw)
    return O.Oracle(D, dims, (1, 1, 1), **p)


def random_cell(D, rng):
    c, w = O.lattice(D)
    phi = rng.uniform(0.05, 0.95)
    f = w * rng.uniform(-0.02, 0.02, len(w)) + w * 0.01
    g = w * phi * (1 + rng.uniform(-0.1, 0.1, len(w)))
    grad = rng.uniform(-0.2, 0.2, 3)
    if D == 2:
        grad[2] = 0.0
    lap = rng.uniform(-0.1, 0.1)
    return c, w, f, g, phi, grad, lap


@pytest.mark.parametrize("D", [2, 3])
@pytest.mark.parametrize("seed", range(4))
def test_moment_identities(D, seed):
    rng = np.random.default_rng(seed)
    o = make(D)
    d = o.derived()
    c, w, f, g, phi, grad, lap = random_cell(D, rng)
    fo, go, diag = o.collide_cell(f, g, phi, grad, lap)
    rho, u, ph, theta, omega, F = diag[0], diag[1:4], diag[4], diag[5], diag[6], diag[7:10]
    sumXi, sumcXi = diag[10], diag[11:14]
    gradrho = (d.rho_h - d.rho_l) * grad
    assert abs(rho - (d.rho_l + (d.rho_h - d.rho_l) * phi)) < 1e-15
    assert abs(sumXi - CS2 * u @ gradrho) < 1e-15
    assert np.abs(sumcXi - CS2 * F).max() < 1e-15
    assert abs((fo.sum() - f.sum()) - sumXi) < 1e-15
    dJ = (c * fo[:, None]).sum(0) - (c * f[:, None]).sum(0)
    assert np.abs(dJ - CS2 * F).max() < 1e-15
    # u = J/(rho cs2) + F/(2 rho)
    J = (c * f[:, None]).sum(0)
    assert np.abs(u - (J / (rho * CS2) + F / (2 * rho))).max() < 1e-15
    # F = mu grad(phi) + F_b, mu = 2 beta phi(phi-1)(2phi-1) - kappa lap
    mu = 2 * d.beta * phi * (phi - 1) * (2 * phi - 1) - d.kappa * lap
    Fb = np.zeros(3)
    Fb[D - 1] = -(rho - 0.5 * (d.rho_h + d.rho_l)) * d.g_accel
    assert np.abs(F - (mu * grad + Fb)).max() < 1e-15
    # omega from the interpolated kinematic viscosity
    nu = d.nu_h + (d.nu_l - d.nu_h) * (1 - phi)
    assert abs(omega - 1.0 / (nu / CS2 + 0.5)) < 1e-14


@pytest.mark.parametrize("D", [2, 3])
def test_phase_field_collision_moments(D):
    rng = np.random.default_rng(3)
    o = make(D)
    d = o.derived()
    c, w, f, g, phi, grad, lap = random_cell(D, rng)
    phi = g.sum()
    fo, go, diag = o.collide_cell(f, g, phi, grad, lap)
    u = diag[1:4]
    assert abs(go.sum() - g.sum()) < 1e-15
    n = grad / np.linalg.norm(grad)
    X = 4 * phi * (1 - phi) / d.W
    tau = d.tau_phi
    expect = (1 - 1 / tau) * (c * g[:, None]).sum(0) + phi * u / tau + d.lambda_phi * CS2 * n * X
    assert np.abs((c * go[:, None]).sum(0) - expect).max() < 1e-15


def product_equilibrium(D, u):
    c, _ = O.lattice(D)
    out = np.ones(len(c))
    for i in range(D):
        ui = u[i]
        e = {-1: 0.5 * (ui * ui - ui + CS2), 0: 1.0 - ui * ui - CS2, 1: 0.5 * (ui * ui + ui + CS2)}
        out = out * np.array([e[int(v)] for v in c[:, i]])
    return out


@pytest.mark.parametrize("D", [2, 3])
def test_unit_rates_give_product_equilibrium(D):
    """With Xi = 0 (no gradients, no force) and every rate 1 the collision maps
    any f' to rho cs2 (E(u) + w(theta-1)), E the product-form equilibrium."""
    rng = np.random.default_rng(21)
    o = make(D, sigma=0.0, g_accel=0.0)
    o.set_rates(shear=1.0)
    c, w, f, g, phi, _, _ = random_cell(D, rng)
    fo, go, diag = o.collide_cell(f, g, phi, np.zeros(3), 0.0)
    rho, u, theta = diag[0], diag[1:4], diag[5]
    assert abs(theta - f.sum() / (rho * CS2)) < 1e-14
    expect = rho * CS2 * (product_equilibrium(D, u) + w * (theta - 1))
    assert np.abs(fo - expect).max() < 1e-15


@pytest.mark.parametrize("D", [2, 3])
def test_shear_rate_on_second_order_only(D):
    """Post-collision second-order central moments of h: off-diagonal scaled by
    (1-omega), deviatoric scaled by (1-omega), trace set to D cs2 (rate 1)."""
    rng = np.random.default_rng(8)
    o = make(D, sigma=0.0, g_accel=0.0)
    c, w, f, g, phi, _, _ = random_cell(D, rng)
    fo, go, diag = o.collide_cell(f, g, phi, np.zeros(3), 0.0)
    rho, u, theta, om = diag[0], diag[1:4], diag[5], diag[6]
    h_in = f / (rho * CS2) - w * (theta - 1)
    h_out = fo / (rho * CS2) - w * (theta - 1)
    def k2(h):
        cc = c - u
        return np.einsum("a,ai,aj->ij", h, cc, cc)[:D, :D]
    kin, kout = k2(h_in), k2(h_out)
    off = ~np.eye(D, dtype=bool)
    assert np.abs(kout[off] - (1 - om) * kin[off]).max() < 1e-15
    tr_in = np.trace(kin)
    assert abs(np.trace(kout) - D * CS2) < 1e-15
    dev_in = np.diag(kin) - tr_in / D
    dev_out = np.diag(kout) - np.trace(kout) / D
    assert np.abs(dev_out - (1 - om) * dev_in).max() < 1e-15


@pytest.mark.parametrize("D", [2, 3])
@pytest.mark.parametrize("phi0", [0.0, 1.0, 0.3])
def test_rest_state_invariant(D, phi0):
    dims = (8, 6, 1) if D == 2 else (6, 5, 4)
    o = O.Oracle(D, dims, (1, 1, 1), rho_ratio=20.0, nu_ratio=2.0, nu_h=0.05, mobility=0.02,
                 width=5.0, sigma=1e-3)
    o.init("uniform", [phi0, 0.01, 0.0, 0.0, 0.0])
    f0, g0, p0 = o.get_state()
    o.step(10)
    f1, g1, p1 = o.get_state()
    assert np.abs(f1 - f0).max() < 1e-14
    assert np.abs(g1 - g0).max() < 1e-14
    assert np.abs(p1 - phi0).max() < 1e-14


@pytest.mark.parametrize("D,dims,periodic,steps", [
    (2, (64, 64, 1), (1, 0, 1), 1000),
    (2, (32, 32, 1), (1, 1, 1), 1000),
    (3, (16, 16, 32), (1, 1, 0), 150),
])
def test_mass_conservation(D, dims, periodic, steps):
    o = O.Oracle(D, dims, periodic, atwood=0.5, nu_ratio=1.0, nu_h=0.01, g_accel=1e-4,
                 mobility=0.02, width=5.0, sigma=1e-3)
    nv = dims[D - 1]
    o.init("rt", [nv / 2, nv / 20, 1e-3], seed=3)
    m0 = o.observables().mass
    o.step(steps)
    ob = o.observables()
    assert ob.health == 0
    assert abs(ob.mass - m0) / m0 < 1e-12


def test_step_matches_cellwise_collision_and_push():
    """One whole step equals collide_cell at every cell followed by a push with
    periodic wrap and half-way bounce-back (Sec. 2.2/2.3, reading A17)."""
    D, dims = 2, (6, 5, 1)
    o = O.Oracle(D, dims, (1, 0, 1), rho_ratio=5.0, nu_ratio=2.0, nu_h=0.05, mobility=0.02,
                 width=3.0, sigma=1e-2, g_accel=1e-4)
    o.init("rt", [2.0, 0.5, 1e-2], seed=9)
    f, g, phi = o.get_state()
    grad, lap = o.fd(phi)
    c, w = O.lattice(D)
    fn = np.full_like(f, np.nan)
    gn = np.full_like(g, np.nan)
    nx, ny = dims[0], dims[1]
    for y in range(ny):
        for x in range(nx):
            fo, go, _ = o.collide_cell(f[:, 0, y, x], g[:, 0, y, x], phi[0, y, x], grad[0, y, x],
                                       lap[0, y, x])
            for a in range(9):
                xx, yy = (x + c[a, 0]) % nx, y + c[a, 1]
                if 0 <= yy < ny:
                    fn[a, 0, yy, xx] = fo[a]
                    gn[a, 0, yy, xx] = go[a]
                else:
                    fn[8 - a, 0, y, x] = fo[a]
                    gn[8 - a, 0, y, x] = go[a]
    o.step(1)
    f1, g1, phi1 = o.get_state()
    assert not np.isnan(fn).any()
    assert np.abs(f1 - fn).max() < 1e-15
    assert np.abs(g1 - gn).max() < 1e-15
    assert np.abs(phi1 - gn.sum(0)).max() < 1e-15
