"""Pins of the oracle's LBMO_FLAG_DIVU alternative to reading A6: the
w cs2 rho div(u) term of Xi (Sec. 2.3) kept, with div(u) the isotropic
difference of the previous step's velocity (reading V1).

What fixes each check:
  - the divergence stencil is exact on linear velocity fields, and at a
    half-way wall with the no-slip ghost (minus the wall cell's velocity) a
    uniform wall-normal velocity U gives the closed form -U at the top wall
    and +U at the bottom wall;
  - the term is isotropic (proportional to w), so it adds cs2 rho div(u) to
    the zeroth moment of the update and nothing to the first, and leaves g
    alone;
  - one step equals the cell-wise collision with div(u) of the stored
    previous velocity followed by the push, over two steps (before the first
    step the previous velocity is the current one);
  - a fluid at rest stays at rest.
"""
import numpy as np
import pytest

import oracle as O

CS2 = 1.0 / 3.0
DIVU = O.FLAG_DIVU


@pytest.mark.parametrize("D", [2, 3])
def test_divergence_exact_on_linear_fields(D):
    dims = (12, 12, 12) if D == 3 else (12, 12, 1)
    o = O.Oracle(D, dims, (1, 1, 1), rho_ratio=2.0, nu_ratio=1.0, nu_h=0.05, mobility=0.02, width=4.0,
                 sigma=0.0, flags=DIVU)
    z, y, x = np.meshgrid(*[np.arange(n, dtype=float) for n in dims[::-1]], indexing="ij")
    coef = np.array([[0.3, -0.2, 0.1], [0.05, -0.4, 0.2], [0.15, 0.25, 0.7]])
    u = np.zeros((3,) + x.shape)
    for k in range(D):
        u[k] = coef[k, 0] * x + coef[k, 1] * y + (coef[k, 2] * z if D == 3 else 0.0) + 0.01 * (k + 1)
    div = o.divu(u)
    want = sum(coef[k, k] for k in range(D))
    inner = (slice(1, -1),) * 3 if D == 3 else (0, slice(1, -1), slice(1, -1))
    assert np.abs(div[inner] - want).max() < 1e-13


@pytest.mark.parametrize("D", [2, 3])
def test_divergence_wall_ghost_closed_form(D):
    dims = (6, 6, 8) if D == 3 else (6, 8, 1)
    per = (1, 1, 0) if D == 3 else (1, 0, 1)
    o = O.Oracle(D, dims, per, rho_ratio=2.0, nu_ratio=1.0, nu_h=0.05, mobility=0.02, width=4.0, sigma=0.0,
                 flags=DIVU)
    U = 0.03
    u = np.zeros((3,) + o.shape[1:])
    u[D - 1] = U
    div = o.divu(u)
    v = D - 1  # vertical axis index in (x, y, z) order
    ax = {3: 0, 2: 1}[D]  # the vertical axis in the [z][y][x] array
    top = np.take(div, -1, axis=ax)
    bot = np.take(div, 0, axis=ax)
    mid = np.take(div, np.arange(1, dims[v] - 1), axis=ax)
    assert np.abs(top + U).max() < 1e-15 and np.abs(bot - U).max() < 1e-15
    assert np.abs(mid).max() < 1e-15


def random_cell(D, rng):
    c, w = O.lattice(D)
    u = rng.uniform(-0.05, 0.05, 3)
    if D == 2:
        u[2] = 0
    cu = c @ u
    G = w * (1 + cu / CS2 + (cu * cu - CS2 * u @ u) / (2 * CS2 * CS2))
    f = 0.6 * CS2 * (G - w) + w * 1e-3 + rng.normal(0, 1e-5, len(c))
    g = G * rng.uniform(0.3, 0.7)
    grad = rng.normal(0, 0.05, 3)
    if D == 2:
        grad[2] = 0
    return c, w, f, g, g.sum(), grad, rng.normal(0, 0.01)


@pytest.mark.parametrize("D", [2, 3])
def test_divergence_term_moments(D):
    rng = np.random.default_rng(5)
    dims = (4, 4, 4) if D == 3 else (4, 4, 1)
    kw = dict(rho_ratio=5.0, nu_ratio=2.0, nu_h=0.05, mobility=0.02, width=4.0, sigma=1e-2, g_accel=1e-4)
    o = O.Oracle(D, dims, (1, 1, 1), flags=DIVU, **kw)
    o0 = O.Oracle(D, dims, (1, 1, 1), **kw)
    for _ in range(5):
        c, w, f, g, phi, grad, lap = random_cell(D, rng)
        div = rng.normal(0, 1e-3)
        fo, go, diag = o.collide_cell(f, g, phi, grad, lap, divu=div)
        fo0, go0, diag0 = o0.collide_cell(f, g, phi, grad, lap)
        rho, u, F = diag[0], diag[1:4], diag[7:10]
        d = o.derived()
        gradrho = (d.rho_h - d.rho_l) * grad
        assert abs((fo.sum() - f.sum()) - (CS2 * u @ gradrho + CS2 * rho * div)) < 1e-15
        assert np.abs(c.T @ (fo - f) - CS2 * F).max() < 1e-16
        # the term is w cs2 rho div(u): half through theta, half through Xi/2
        assert np.abs((fo - fo0) - w * CS2 * rho * div).max() < 1e-16
        assert np.array_equal(go, go0)
        # without the flag the argument is ignored (reading A6)
        assert np.array_equal(o0.collide_cell(f, g, phi, grad, lap, divu=div)[0], fo0)


def test_divergence_step_matches_cellwise():
    D, dims = 2, (6, 5, 1)
    o = O.Oracle(D, dims, (1, 0, 1), rho_ratio=5.0, nu_ratio=2.0, nu_h=0.05, mobility=0.02,
                 width=3.0, sigma=1e-2, g_accel=1e-4, flags=DIVU)
    o.init("rt", [2.0, 0.5, 1e-2], seed=9)
    c, _ = O.lattice(D)
    nx, ny = dims[0], dims[1]
    f, g, phi = o.get_state()
    uprev = None
    for step in range(2):
        grad, lap = o.fd(phi)
        if uprev is None:  # before the first step the previous velocity is the current one
            uprev = np.zeros((3, 1, ny, nx))
            for y in range(ny):
                for x in range(nx):
                    uprev[:, 0, y, x] = o.collide_cell(f[:, 0, y, x], g[:, 0, y, x], phi[0, y, x], grad[0, y, x],
                                                       lap[0, y, x])[2][1:4]
        div = o.divu(uprev)
        fn = np.full_like(f, np.nan)
        gn = np.full_like(g, np.nan)
        unew = np.zeros_like(uprev)
        for y in range(ny):
            for x in range(nx):
                fo, go, diag = o.collide_cell(f[:, 0, y, x], g[:, 0, y, x], phi[0, y, x], grad[0, y, x],
                                              lap[0, y, x], divu=div[0, y, x])
                unew[:, 0, y, x] = diag[1:4]
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
        assert np.abs(f1 - fn).max() < 1e-15 and np.abs(g1 - gn).max() < 1e-15
        f, g, phi, uprev = f1, g1, phi1, unew


def test_divergence_rest_state():
    o = O.Oracle(3, (8, 8, 8), (1, 1, 0), rho_ratio=3.0, nu_ratio=1.0, nu_h=0.05, mobility=0.02, width=4.0,
                 sigma=0.0, flags=DIVU)
    # bulk heavy phase (phi = 1: no sharpening flux) with walls in z
    o.init("uniform", [1.0, 1e-3, 0.0, 0.0, 0.0])
    f0, g0, _ = o.get_state()
    o.step(20)
    f1, g1, _ = o.get_state()
    assert np.abs(f1 - f0).max() < 1e-14 and np.abs(g1 - g0).max() < 1e-14
