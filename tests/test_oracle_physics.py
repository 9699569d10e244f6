"""Pins of the oracle against closed-form physics the paper's model must
reproduce (Sec. 2.1 targets, Sec. 3.1 Laplace law and spurious currents).
Sizes are kept small so the whole CPU suite runs in about a minute."""
import numpy as np
import pytest
from scipy.integrate import cumulative_trapezoid
from scipy.optimize import curve_fit

import oracle as O


@pytest.mark.parametrize("D,dims", [(2, (4, 64, 1)), (3, (4, 64, 4))])
@pytest.mark.parametrize("nu", [0.02, 0.1])
def test_shear_wave_decay(D, dims, nu):
    """u_x = U sin(2 pi y/L) decays as exp(-nu k^2 t) with nu = cs2 (1/omega - 1/2)."""
    o = O.Oracle(D, dims, (1, 1, 1), rho_ratio=3.0, nu_ratio=1.0, nu_h=nu, mobility=0.02,
                 width=5.0)
    o.init("shear_wave", [1e-4, 0.0])
    o.step(100)
    a0 = np.abs(o.fields()[2][0]).max()
    T = 500
    o.step(T)
    a1 = np.abs(o.fields()[2][0]).max()
    k = 2 * np.pi / 64
    nu_meas = -np.log(a1 / a0) / (k * k * T)
    assert abs(nu_meas / nu - 1) < 0.01


@pytest.mark.parametrize("D,dims", [(2, (64, 2, 1)), (3, (64, 2, 2))])
def test_flat_interface_tanh_profile(D, dims):
    """The conservative Allen-Cahn equation (Sec. 2.1) has the steady profile
    phi = (1 + tanh(2 d / W))/2; with the wrong source sign or the wrong
    discrete factor (readings A3, A4) the width is off by a large factor."""
    W = 5.0
    o = O.Oracle(D, dims, (1, 1, 1), rho_ratio=3.0, nu_ratio=1.0, nu_h=0.05, mobility=0.02,
                 width=W, sigma=0.0)
    o.init("flat", [16.3, 47.8, 0.0])
    o.step(4000)
    line = o.get_state()[2][0, 0, :]
    x = np.arange(64.0)

    def model(x, x0, x1, w):
        return 0.5 * (1 + np.tanh(2 * np.minimum(x - x0, x1 - x) / w))

    popt, _ = curve_fit(model, x, line, p0=[16, 48, 5])
    assert abs(popt[2] / W - 1) < 0.02
    assert abs(popt[0] - 16.3) < 0.01 and abs(popt[1] - 47.8) < 0.01
    assert np.abs(model(x, popt[0], popt[1], W) - line).max() < 5e-3


@pytest.mark.parametrize("R,sigma", [(12, 1e-3), (16, 1e-3), (16, 1e-1)])
def test_laplace_law_2d(R, sigma):
    """Static drop, density ratio 20, nu = 0.1 (Sec. 3.1): Delta P = sigma / r."""
    o = O.Oracle(2, (64, 64, 1), (1, 1, 1), rho_ratio=20.0, nu_ratio=1.0, nu_h=0.1,
                 mobility=0.02, width=5.0, sigma=sigma)
    o.init("drop_static", [R, 0.0, 0.0])
    o.step(4000)
    ob = o.observables()
    assert ob.laplace_dp > 0
    assert abs(ob.laplace_dp / (sigma / R) - 1) < 0.05


def test_laplace_law_3d():
    """3-D static drop: Delta P = 2 sigma / R."""
    R, sigma = 7.0, 1e-3
    o = O.Oracle(3, (24, 24, 24), (1, 1, 1), rho_ratio=20.0, nu_ratio=1.0, nu_h=0.1,
                 mobility=0.02, width=4.0, sigma=sigma)
    o.init("drop_static", [R, 0.0, 0.0])
    o.step(1000)
    ob = o.observables()
    assert abs(ob.laplace_dp / (2 * sigma / R) - 1) < 0.05


def test_spurious_currents_density_ratio_1000():
    """Sec. 3.1: at density ratio 1000 and sigma = 1e-3 the spurious currents
    are of order 1e-6."""
    o = O.Oracle(2, (64, 64, 1), (1, 1, 1), rho_ratio=1000.0, nu_ratio=1.0, nu_h=0.1,
                 mobility=0.02, width=5.0, sigma=1e-3)
    o.init("drop_static", [16, 0.0, 0.0])
    o.step(3000)
    ob = o.observables()
    assert ob.health == 0
    assert ob.max_u < 1e-5
    assert abs(ob.laplace_dp / (1e-3 / 16) - 1) < 0.06


def _poiseuille(H, rho_ratio, flags, steps, G=1e-7):
    o = O.Oracle(2, (4, H, 1), (1, 0, 1), rho_ratio=rho_ratio, nu_ratio=10.0, nu_h=0.05,
                 mobility=0.02, width=4.0, sigma=0.0, force_x=G,
                 flags=O.FLAG_UNIFORM_FORCE | flags)
    o.init("poiseuille", [0.0])
    o.step(steps)
    ux = o.fields()[2][0, 0, :, 0]
    d = o.derived()
    h = H / 2
    y = np.arange(H) - (H - 1) / 2
    # sharp-interface closed form (walls at y = +-h, fluid a below, b above)
    ea, eb = d.rho_h * d.nu_h, d.rho_l * d.nu_l
    S = (G * h / 2) * (ea - eb) / (ea + eb)
    B = G * h * h / (2 * ea) + S * h / ea
    sharp = np.where(y < 0, -G * y ** 2 / (2 * ea) + S / ea * y + B,
                     -G * y ** 2 / (2 * eb) + S / eb * y + B)
    # the same 1-D momentum balance d/dy(eta du/dy) = -G integrated with the
    # diffuse profile eta(phi(y)), phi = (1 + tanh(-2y/W))/2
    s = np.linspace(-h, h, 200001)
    ph = 0.5 * (1 + np.tanh(-2 * s / d.W))
    if flags & O.FLAG_DYNAMIC_VISC:
        eta = d.rho_l * d.nu_l + (d.rho_h * d.nu_h - d.rho_l * d.nu_l) * ph
    else:
        eta = (d.rho_l + (d.rho_h - d.rho_l) * ph) * (d.nu_h + (d.nu_l - d.nu_h) * (1 - ph))
    I1 = cumulative_trapezoid(1 / eta, s, initial=0)
    I2 = cumulative_trapezoid(s / eta, s, initial=0)
    us = (G * I2[-1] / I1[-1]) * I1 - G * I2
    smeared = np.interp(y, s, us)
    err = lambda ref: np.linalg.norm(ux - ref) / np.linalg.norm(ref)
    return err(sharp), err(smeared)


def test_layered_poiseuille_kinematic():
    e_sharp, e_smeared = _poiseuille(64, 1.0, 0, 60000)
    assert e_smeared < 5e-3
    assert e_sharp < 0.10


def test_layered_poiseuille_dynamic_viscosity_flag():
    e_sharp, e_smeared = _poiseuille(64, 3.0, O.FLAG_DYNAMIC_VISC, 60000)
    assert e_smeared < 0.02
    assert e_sharp < 0.03


def test_rayleigh_taylor_soft():
    """2-D RT at At = 0.5 (Sec. 3.2 set-up, 64 x 256): the spike falls, the
    bubble rises, mass is conserved to round-off."""
    o = O.Oracle(2, (64, 256, 1), (1, 0, 1), atwood=0.5, nu_ratio=1.0, Re=256, g_accel=2.5e-5,
                 L_ref=64, mobility=0.02, width=5.0)
    o.init("rt", [128, 6.4, 0.0])
    ob0 = o.observables()
    o.step(1500)
    ob = o.observables()
    assert ob.tip_spike < ob0.tip_spike - 1.0
    assert ob.tip_bubble > ob0.tip_bubble + 1.0
    assert abs(ob.mass / ob0.mass - 1) < 1e-12
