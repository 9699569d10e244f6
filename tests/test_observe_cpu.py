"""Host-side spreading-radius measurement (Sec. 3.4) on synthetic phi fields
whose neck radius is known by construction."""
import math

import numpy as np

from paper_2101_06769_gb300 import observe


def field(nx, ny, sheet_h, r_neck, axis, W=4.0, drop=True):
    """Film below sheet_h joined to a liquid column |x - axis| < r_neck that
    reaches 8 cells above the film; tanh profiles of width W."""
    y, x = np.mgrid[0:ny, 0:nx].astype(float)
    dx = np.abs((x - axis + nx / 2) % nx - nx / 2)
    d_film = sheet_h - y
    d_col = np.minimum(r_neck - dx, sheet_h + 8 - y) if drop else -np.inf * np.ones_like(x)
    return 0.5 * (1 + np.tanh(2 * np.maximum(d_film, d_col) / W))


def test_known_neck_radius():
    for r in (3.0, 7.5, 20.25, 41.0):
        for axis in (100, 3):  # the second wraps around x
            phi = field(200, 60, 20.0, r, axis)
            got = observe.spreading_radius(phi, 20.0, axis)
            assert abs(got - r) < 0.05, (r, axis, got)


def test_no_contact_is_nan():
    phi = field(200, 60, 20.0, 10.0, 100, drop=False)
    assert math.isnan(observe.spreading_radius(phi, 20.0, 100))


def test_asymmetric_neck_averages_sides():
    phi = np.minimum(field(200, 60, 20.0, 10.0, 100), 1.0)
    y, x = np.mgrid[0:60, 0:200]
    # widen the right side by moving its edge 4 cells outward
    right = field(200, 60, 20.0, 14.0, 100)
    phi = np.where(x > 100, right, phi)
    assert abs(observe.spreading_radius(phi, 20.0, 100) - 12.0) < 0.05


def test_contact_time():
    assert observe.contact_time(4.0, 0.05) == 160.0


def test_known_neck_radius_half_domain():
    """The half domain of a symmetric impact: the axis on the face before
    column 0, so a neck of radius r crosses phi = 1/2 at x = r - 1/2."""
    for r in (3.0, 7.5, 20.25, 41.0):
        full = field(400, 60, 20.0, r, 199.5)  # axis on the face between columns 199 and 200
        half = full[:, 200:]
        got = observe.spreading_radius_half(half, 20.0)
        assert abs(got - r) < 0.05, (r, got)
    assert math.isnan(observe.spreading_radius_half(field(400, 60, 20.0, 5.0, 199.5, drop=False)[:, 200:], 20.0))
