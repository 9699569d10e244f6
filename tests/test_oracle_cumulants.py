"""Pins of the oracle's moment and cumulant machinery (Sec. 2.3).

The paper prints the central-moment -> cumulant relations with two garbled
terms in the sixth order (reading A9).  They are pinned here against the
general moment-cumulant formula of probability theory,
    kappa(X_1..X_n) = sum over set partitions pi of (|pi|-1)! (-1)^(|pi|-1)
                      prod_{B in pi} E[prod_{i in B} X_i],
evaluated by brute force from the populations themselves, so that a wrong
coefficient, a wrong index or a wrong sign in any relation fails.
"""
import math

import numpy as np
import pytest

import oracle as O

CS2 = 1.0 / 3.0


def set_partitions(items):
    if not items:
        yield []
        return
    first, rest = items[0], items[1:]
    for p in set_partitions(rest):
        yield [[first]] + p
        for i in range(len(p)):
            yield p[:i] + [[first] + p[i]] + p[i + 1:]


def brute_cumulant(h, c, expo):
    """joint cumulant of the lattice velocity components, distribution h (sum 1)"""
    axes = [0] * expo[0] + [1] * expo[1] + [2] * expo[2]
    n = len(axes)

    def moment(block):
        v = np.ones(len(h))
        for i in block:
            v = v * c[:, axes[i]]
        return float((v * h).sum())

    tot = 0.0
    for p in set_partitions(list(range(n))):
        k = len(p)
        term = math.factorial(k - 1) * (-1) ** (k - 1)
        for B in p:
            term *= moment(B)
        tot += term
    return tot


def random_h(D, rng, amp=0.3):
    c, w = O.lattice(D)
    h = w * (1.0 + amp * rng.uniform(-1, 1, len(w)))
    h /= h.sum()
    u = (c * h[:, None]).sum(0)
    return c, w, h, u


def exponents(D):
    cm = 2 if D == 3 else 0
    return [(a, b, cc) for cc in range(cm + 1) for b in range(3) for a in range(3)]


@pytest.mark.parametrize("D", [2, 3])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_forward_cumulants_match_partition_formula(D, seed):
    rng = np.random.default_rng(seed)
    c, w, h, u = random_h(D, rng)
    kap = O.central_moments(D, h, u)
    K = O.cumulants_forward(D, kap)
    for (a, b, cc) in exponents(D):
        n = a + b + cc
        idx = a + 3 * b + 9 * cc
        if n < 2:
            continue
        ref = brute_cumulant(h, c.astype(float), (a, b, cc))
        assert abs(K[idx] - ref) < 1e-13, ((a, b, cc), K[idx], ref)


@pytest.mark.parametrize("D", [2, 3])
def test_central_moments_direct_definition(D):
    rng = np.random.default_rng(5)
    c, w, h, u = random_h(D, rng)
    u = u + 0.05  # any shift: definition sum (c-u)^a (c-u)^b (c-u)^c h
    kap = O.central_moments(D, h, u)
    for (a, b, cc) in exponents(D):
        ref = ((c[:, 0] - u[0]) ** a * (c[:, 1] - u[1]) ** b * (c[:, 2] - u[2]) ** cc * h).sum()
        assert abs(kap[a + 3 * b + 9 * cc] - ref) < 1e-15
    assert abs(kap[0] - 1.0) < 1e-15


@pytest.mark.parametrize("D", [2, 3])
def test_inverse_of_forward_is_identity(D):
    rng = np.random.default_rng(7)
    _, _, h, u = random_h(D, rng, amp=0.6)
    kap = O.central_moments(D, h, u)
    back = O.cumulants_inverse(D, O.cumulants_forward(D, kap))
    assert np.abs(back - kap).max() < 1e-14
    K = rng.normal(size=27) * 0.1
    if D == 2:
        K[9:] = 0.0
    assert np.abs(O.cumulants_forward(D, O.cumulants_inverse(D, K)) - K).max() < 1e-14


@pytest.mark.parametrize("D", [2, 3])
def test_kron_inverse_round_trip(D):
    rng = np.random.default_rng(11)
    _, _, h, u = random_h(D, rng, amp=0.6)
    u = u + np.array([0.03, -0.02, 0.01 if D == 3 else 0.0])
    back = O.kron_inverse(D, O.central_moments(D, h, u), u)
    assert np.abs(back[:len(h)] - h).max() < 1e-15


def product_equilibrium(D, u):
    """per-axis populations ((u^2-u+cs2)/2, 1-u^2-cs2, (u^2+u+cs2)/2), tensorised"""
    c, _ = O.lattice(D)
    out = np.ones(len(c))
    for i in range(D):
        ui = u[i]
        e = {-1: 0.5 * (ui * ui - ui + CS2), 0: 1.0 - ui * ui - CS2, 1: 0.5 * (ui * ui + ui + CS2)}
        out = out * np.array([e[int(v)] for v in c[:, i]])
    return out


@pytest.mark.parametrize("D", [2, 3])
def test_equilibrium_cumulants(D):
    u = np.array([0.04, -0.07, 0.02 if D == 3 else 0.0])
    h = product_equilibrium(D, u)
    assert abs(h.sum() - 1) < 1e-15
    K = O.cumulants_forward(D, O.central_moments(D, h, u))
    for (a, b, cc) in exponents(D):
        idx = a + 3 * b + 9 * cc
        n = a + b + cc
        if n >= 3 or (n == 2 and 1 in (a, b, cc)):
            assert abs(K[idx]) < 1e-15, (a, b, cc)
        elif n == 2:
            assert abs(K[idx] - CS2) < 1e-15
    # the product form is exactly the distribution whose cumulants are (1, u, cs2 I, 0...)
    Kp = np.zeros(27)
    Kp[0] = 1.0
    for i, e in enumerate([(2, 0, 0), (0, 2, 0), (0, 0, 2)][:D]):
        Kp[e[0] + 3 * e[1] + 9 * e[2]] = CS2
    back = O.kron_inverse(D, O.cumulants_inverse(D, Kp), u)
    assert np.abs(back[:len(h)] - h).max() < 1e-15


def test_sixth_order_printed_sign_fails():
    """The relation as printed (cubic group subtracted) gives K_x2y2z2 = -4 cs^6
    for the rest equilibrium; the corrected one gives 0 (reading A9)."""
    h = product_equilibrium(3, np.zeros(3))
    kap = O.central_moments(3, h, np.zeros(3))
    K = O.cumulants_forward(3, kap)
    assert abs(K[26]) < 1e-16
    cub = 2 * CS2 ** 3
    printed = K[26] - 2 * cub
    assert abs(printed + 4 * CS2 ** 3) < 1e-15
