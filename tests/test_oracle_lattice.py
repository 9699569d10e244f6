"""Pins of the oracle's lattice, finite differences, parameter closure and
random generator against values fixed by the mathematics or printed in the
paper (Sec. 2.2 isotropic differences, Sec. 3 parameter relations)."""
import itertools
import os

import numpy as np
import pytest

import oracle as O

CS2 = 1.0 / 3.0
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("D", [2, 3])
def test_lattice_isotropy(D):
    c, w = O.lattice(D)
    Q = 9 if D == 2 else 27
    assert c.shape == (Q, 3) and np.all(np.abs(c) <= 1)
    # exchange-format ordering a = (cx+1) + 3(cy+1) + 9(cz+1), opposite = Q-1-a
    for a in range(Q):
        assert a == (c[a, 0] + 1) + 3 * (c[a, 1] + 1) + (9 * (c[a, 2] + 1) if D == 3 else 0)
        assert np.all(c[Q - 1 - a] == -c[a])
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.abs((w[:, None] * c).sum(0)).max() < 1e-15
    M2 = np.einsum("a,ai,aj->ij", w, c, c)
    assert np.abs(M2[:D, :D] - CS2 * np.eye(D)).max() < 1e-15
    M3 = np.einsum("a,ai,aj,ak->ijk", w, c, c, c)
    assert np.abs(M3).max() < 1e-15
    M4 = np.einsum("a,ai,aj,ak,al->ijkl", w, c, c, c, c)
    d = np.eye(3)
    iso = CS2 ** 2 * (np.einsum("ij,kl->ijkl", d, d) + np.einsum("ik,jl->ijkl", d, d)
                      + np.einsum("il,jk->ijkl", d, d))
    sl = (slice(0, D),) * 4
    assert np.abs(M4[sl] - iso[sl]).max() < 1e-15


def test_lattice_weights_values():
    _, w2 = O.lattice(2)
    assert sorted(set(np.round(w2 * 36).astype(int))) == [1, 4, 16]  # 1/36, 1/9, 4/9
    _, w3 = O.lattice(3)
    assert sorted(set(np.round(w3 * 216).astype(int))) == [1, 4, 16, 64]  # 1/216 .. 8/27


def _fd_oracle(D, dims, periodic=(1, 1, 1)):
    return O.Oracle(D, dims, periodic, rho_ratio=1.0, nu_ratio=1.0, nu_h=0.1,
                    mobility=0.02, width=4.0, sigma=0.0)


@pytest.mark.parametrize("D", [2, 3])
def test_fd_exact_on_polynomials(D):
    dims = (12, 10, 1) if D == 2 else (8, 9, 10)
    o = _fd_oracle(D, dims)
    nz, ny, nx = o.shape[1:]
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    lin = 0.3 * x - 0.7 * y + (1.1 * z if D == 3 else 0.0) + 2.0
    grad, lap = o.fd(lin)
    inner = (slice(1, -1) if D == 3 else slice(None), slice(1, -1), slice(1, -1))
    assert np.abs(grad[inner][..., 0] - 0.3).max() < 1e-13
    assert np.abs(grad[inner][..., 1] + 0.7).max() < 1e-13
    if D == 3:
        assert np.abs(grad[inner][..., 2] - 1.1).max() < 1e-13
    assert np.abs(lap[inner]).max() < 1e-13
    quad = 0.5 * x ** 2 + 0.25 * y ** 2 + (0.125 * z ** 2 if D == 3 else 0.0) + 0.1 * x * y
    grad, lap = o.fd(quad)
    expect = 1.0 + 0.5 + (0.25 if D == 3 else 0.0)
    assert np.abs(lap[inner] - expect).max() < 1e-12
    assert np.abs(grad[inner][..., 0] - (x + 0.1 * y)[inner]).max() < 1e-12


@pytest.mark.parametrize("D", [2, 3])
def test_fd_fourier_symbol(D):
    """For phi = cos(k.x) on a periodic box the tensor-product stencils have
    the closed-form symbols grad_x: -sin(kx) prod_{d!=x}(2+cos kd)/3 * sin-part,
    lap: 6 [prod_d (2 + cos kd)/3 - 1]."""
    dims = (16, 8, 1) if D == 2 else (16, 8, 4)
    o = _fd_oracle(D, dims)
    nz, ny, nx = o.shape[1:]
    k = np.array([2 * np.pi / nx, 2 * 2 * np.pi / ny, (2 * np.pi / nz) if D == 3 else 0.0])
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    arg = k[0] * x + k[1] * y + k[2] * z
    grad, lap = o.fd(np.cos(arg))
    fac = [(2.0 + np.cos(k[i])) / 3.0 for i in range(D)]
    for i in range(D):
        other = np.prod([fac[j] for j in range(D) if j != i])
        assert np.abs(grad[..., i] - (-np.sin(k[i]) * other * np.sin(arg))).max() < 1e-13
    assert np.abs(lap - 6.0 * (np.prod(fac) - 1.0) * np.cos(arg)).max() < 1e-13


def _golden_params():
    rows = []
    with open(os.path.join(GOLDEN, "paper_parameters.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append(line.split("|")[0].split())
    return rows


def test_paper_parameter_relations():
    rows = _golden_params()
    assert len(rows) == 6
    for r in rows:
        kv = dict(t.split("=") for t in r if "=" in t)
        vals = [t for t in r[1:] if "=" not in t]
        expected, tol = float(vals[0]), float(vals[1])
        if r[0] == "nu":
            d = O.derive(2, Re=float(kv["Re"]), g_accel=float(kv["g"]), L_ref=float(kv["L"]),
                         rho_ratio=3.0)
            assert abs(d.nu_h - expected) <= tol, r
        else:
            d = O.derive(2, We=float(kv["We"]), Re=float(kv["Re"]), U0=0.05, L_ref=100.0,
                         rho_ratio=1000.0, nu_ratio=15.0)
            assert abs(d.K_impact - expected) <= tol, r


def test_derived_closure():
    # beta = 12 sigma/W, kappa = 3 sigma W/2 (Sec. 2.1); tau_phi = M/cs2 + 1/2 (Sec. 2.2)
    d = O.derive(3, rho_ratio=1000.0, nu_ratio=15.0, We=8000.0, Re=1000.0, U0=0.05, L_ref=64.0,
                 width=4.0, mobility=0.02)
    assert abs(d.sigma - 64 * 0.05 ** 2 / 8000) < 1e-18
    assert abs(d.beta - 12 * d.sigma / 4.0) < 1e-18
    assert abs(d.kappa - 1.5 * d.sigma * 4.0) < 1e-18
    assert abs(d.tau_phi - 0.56) < 1e-15
    assert abs(d.lambda_phi - (1 - 1 / 1.12)) < 1e-15
    assert abs(d.nu_h - 0.0032) < 1e-15 and abs(d.nu_l - 0.048) < 1e-15
    assert abs(d.rho_l - 1e-3) < 1e-18
    # Atwood number overrides the ratio: At = 0.5 -> rho_h/rho_l = 3
    d = O.derive(2, atwood=0.5, Re=256, g_accel=2.5e-5, L_ref=64)
    assert abs(d.rho_l - 1 / 3) < 1e-15 and abs(d.nu_h - 0.01) < 1e-15


def test_splitmix64_published_outputs():
    with open(os.path.join(GOLDEN, "splitmix64.txt")) as fh:
        lines = [l.split() for l in fh if l.strip() and not l.startswith("#")]
    seed = int(lines[0][1])
    expect = [int(l[0]) for l in lines[1:]]
    assert [O.splitmix64(seed, i) for i in range(len(expect))] == expect


def test_invalid_parameters_rejected():
    with pytest.raises(ValueError):
        O.derive(2, rho_ratio=-1.0, nu_h=0.1)
    with pytest.raises(ValueError):
        O.derive(2, rho_ratio=2.0, nu_h=0.1, width=0.0)
    with pytest.raises(ValueError):
        O.derive(2, rho_ratio=2.0)  # no viscosity information
