"""Pins of the oracle's symmetry axis (the symmetry boundary of the 2-D
splash, Sec. 3.4; reading A28: half-way specular reflection, the phi ghost
equal to the boundary cell).

A periodic domain of width 2L whose state is mirror-symmetric about a cell
face stays symmetric (every rule of the method commutes with the reflection),
so each of its halves evolves exactly like a domain of width L with symmetry
faces at both ends: the full domain is symmetric about the face x = L - 1/2
and, by periodicity, about x = -1/2.  The half domain must reproduce the
right half of the full one to rounding, in both population sets and phi,
for both phase lattices; a wrong reflection (bounce-back, the wrong mirrored
direction, a ghost from the far side) leaves differences of the order of
the populations themselves."""
import numpy as np
import pytest

import oracle

L, NY = 12, 20
PHYS = dict(rho_ratio=100.0, nu_ratio=5.0, We=200.0, Re=200.0, U0=0.05, L_ref=8.0, mobility=0.05, width=3.0)


def _pair(flags=0, steps=40):
    phys = dict(PHYS, flags=flags)
    full = oracle.Oracle(2, (2 * L, NY, 1), (1, 0, 1), **phys)
    half = oracle.Oracle(2, (L, NY, 1), (2, 0, 1), **phys)
    # drop of diameter 8 on a sheet 3 cells deep, no noise, axis on a face
    full.init("drop_sheet", [8.0, 3.0, 0.05, 0.0, L - 0.5], seed=1)
    half.init("drop_sheet", [8.0, 3.0, 0.05, 0.0, -0.5], seed=1)
    full.step(steps)
    half.step(steps)
    return full, half


@pytest.mark.parametrize("flags", [0, oracle.FLAG_PHASE_REDUCED])
def test_half_domain_equals_half_of_the_symmetric_full_domain(flags):
    full, half = _pair(flags)
    ff, gf, pf = full.get_state()
    fh, gh, ph = half.get_state()
    # [a][y][x] arrays: the half domain is columns L .. 2L-1 of the full one
    for a_full, a_half in ((ff, fh), (gf, gh), (pf, ph)):
        right = a_full[..., L:]
        scale = np.abs(right).max()
        assert np.abs(a_half - right).max() <= 1e-11 * scale
    # and the full state is itself symmetric: the left half mirrored
    mir = pf[..., :L][..., ::-1]
    assert np.abs(mir - pf[..., L:]).max() <= 1e-11
    assert abs(pf.sum() - 2 * ph.sum()) <= 1e-10 * pf.sum()
    full.close()
    half.close()


def test_symmetry_axis_conserves_mass_exactly():
    half = oracle.Oracle(2, (L, NY, 1), (2, 0, 1), **PHYS)
    half.init("drop_sheet", [8.0, 3.0, 0.05, 1e-3, -0.5], seed=4)
    m0 = half.get_state()[2].sum()
    half.step(150)
    m1 = half.get_state()[2].sum()
    assert abs(m1 - m0) <= 1e-12 * m0
    half.close()


def test_rest_state_is_unchanged_by_symmetry_faces():
    """A uniform rest state is its own mirror image: every reflected
    population equals the one it replaces."""
    o = oracle.Oracle(2, (7, 9, 1), (2, 1, 1), **dict(PHYS, rho_ratio=3.0))
    o.init("uniform", [0.7, 0.01, 0.0, 0.0, 0.0])
    f0, g0, _ = o.get_state()
    o.step(5)
    f1, g1, _ = o.get_state()
    assert np.abs(f1 - f0).max() <= 1e-15 and np.abs(g1 - g0).max() <= 1e-15
    o.close()


def test_symmetry_axis_rejected_where_undefined():
    with pytest.raises(Exception):
        oracle.Oracle(2, (8, 8, 1), (1, 2, 1), **PHYS)  # the vertical axis
    with pytest.raises(Exception):
        oracle.Oracle(2, (8, 8, 1), (2, 0, 1), **dict(PHYS, flags=oracle.FLAG_DIVU))
