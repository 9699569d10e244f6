"""Host-side measurements on a domain's phi field that the paper reports
for its droplet-impact cases (Sec. 3.4) and that are not per-step
observables of the C ABI.

Spreading radius r_K.  After a drop touches a liquid film the two merge
through a neck that widens as sqrt(t) at first (the scaling the paper shows
as r_K/D = 1.1 sqrt(t/T), T = D/U0, after Josserand & Zaleski).  Reading
taken here: r_K is the horizontal distance from the drop's axis to where
phi crosses 1/2 on the first row of cells above the undisturbed film surface
(the film's phi = 1/2 level is at sheet_h, so that row holds gas, phi < 1/2,
everywhere but in the neck), following the liquid outward from the axis; the
crossing is interpolated linearly between cell centres.  Before contact the
row is gas at the axis and r_K is NaN.  t counts from the geometric contact
time 2W/U0 (the drop's phi = 1/2 surface starts 2W above the film's and
falls at U0).
"""
import math

import numpy as np


def spreading_radius(phi_xy, sheet_h, axis_x):
    """r_K of a 2-D phi field phi_xy[y][x] (x periodic), film surface at
    height sheet_h, drop axis at column axis_x (an integer).  Returns the
    mean of the left and right radii, or NaN before contact."""
    phi_xy = np.asarray(phi_xy, dtype=np.float64)
    ny, nx = phi_xy.shape
    row = phi_xy[int(math.floor(sheet_h)) + 1]
    if row[axis_x % nx] < 0.5:
        return float("nan")
    radii = []
    for step in (1, -1):
        prev = row[axis_x % nx]
        r = float("nan")
        for k in range(1, nx // 2 + 1):
            cur = row[(axis_x + step * k) % nx]
            if cur < 0.5:
                r = (k - 1) + (prev - 0.5) / (prev - cur)
                break
            prev = cur
        radii.append(r)
    return 0.5 * (radii[0] + radii[1])


def spreading_radius_half(phi_xy, sheet_h):
    """r_K of the half domain of a symmetric impact: phi_xy[y][x] with the
    drop's axis on the symmetry face x = -1/2 before column 0 (reading A28),
    film surface at height sheet_h.  Column k's centre lies k + 1/2 from the
    axis.  Returns NaN before contact."""
    phi_xy = np.asarray(phi_xy, dtype=np.float64)
    ny, nx = phi_xy.shape
    row = phi_xy[int(math.floor(sheet_h)) + 1]
    if row[0] < 0.5:
        return float("nan")
    for k in range(1, nx):
        if row[k] < 0.5:
            return (k - 0.5) + (row[k - 1] - 0.5) / (row[k - 1] - row[k])
    return float("nan")


def contact_time(width, U0):
    """Steps from the initial state to the geometric contact of the drop with
    the film: the drop's phi = 1/2 surface starts 2W above the film's."""
    return 2.0 * width / U0
