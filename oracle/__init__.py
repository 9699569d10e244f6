"""ctypes wrapper of the FP64 CPU oracle (liblbmo).

TEST INFRASTRUCTURE ONLY.  The oracle is a plain, slow, literal FP64
implementation of the coupled conservative Allen-Cahn / pressure-based
cumulant lattice Boltzmann step of Hosseini, Safari & Thevenin (arXiv
2101.06769, Sec. 2).  Only tests/, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import it; the CUDA library never does.

Arrays use the exchange format both implementations agree on:
direction a = (cx+1) + 3(cy+1) + 9(cz+1), layout [a][z][y][x].  With
FLAG_PHASE_REDUCED the phase field g lives on the rest and face directions
only (D3Q7 / D2Q5), in the same relative order.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

CASE = {"rt": 0, "drop_static": 1, "flat": 2, "poiseuille": 3, "drop_sheet": 4,
        "shear_wave": 5, "uniform": 6}
FLAG_WE_LIGHT = 1 << 0
FLAG_DYNAMIC_VISC = 1 << 1
FLAG_UNIFORM_FORCE = 1 << 2
FLAG_PHASE_REDUCED = 1 << 3
FLAG_DIVU = 1 << 4


class Phys(C.Structure):
    _fields_ = [(n, C.c_double) for n in
                ("rho_ratio", "nu_ratio", "We", "Re", "atwood", "mobility", "width",
                 "g_accel", "U0", "L_ref", "sigma", "nu_h", "force_x")] + [("flags", C.c_uint)]


class Derived(C.Structure):
    _fields_ = [(n, C.c_double) for n in
                ("rho_h", "rho_l", "nu_h", "nu_l", "sigma", "beta", "kappa", "M", "W",
                 "tau_phi", "lambda_phi", "g_accel", "U_ref", "force_x", "K_impact")]


class Obs(C.Structure):
    _fields_ = [(n, C.c_double) for n in
                ("mass", "kinetic_energy", "max_u", "p_in", "p_out", "laplace_dp",
                 "tip_spike", "tip_bubble")] + [("step", C.c_long), ("health", C.c_int)]


_lib = None
_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def lib():
    global _lib
    if _lib is None:
        # LBMO_LIBRARY: a separately built copy (the mutation test builds
        # oracles with a planted mistake to show that the pins catch it)
        path = os.environ.get("LBMO_LIBRARY") or _build.build()
        L = C.CDLL(path)
        L.lbmo_create.restype = C.c_void_p
        L.lbmo_create.argtypes = [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(Phys)]
        L.lbmo_destroy.argtypes = [C.c_void_p]
        L.lbmo_last_error.restype = C.c_char_p
        L.lbmo_derive.argtypes = [C.c_int, C.POINTER(Phys), C.POINTER(Derived)]
        L.lbmo_get_derived.argtypes = [C.c_void_p, C.POINTER(Derived)]
        L.lbmo_set_rates.argtypes = [C.c_void_p] + [C.c_double] * 6
        L.lbmo_init.argtypes = [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.c_int, C.c_ulonglong]
        L.lbmo_step.argtypes = [C.c_void_p, C.c_long]
        L.lbmo_get_state.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.lbmo_set_state.argtypes = [C.c_void_p, _dp, _dp]
        L.lbmo_observables.argtypes = [C.c_void_p, C.POINTER(Obs)]
        L.lbmo_fields.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.lbmo_set_threads.argtypes = [C.c_int]
        L.lbmo_get_threads.restype = C.c_int
        L.lbmo_lattice.argtypes = [C.c_int, C.POINTER(C.c_int), C.c_void_p, C.c_void_p]
        L.lbmo_fd.argtypes = [C.c_void_p, _dp, _dp, _dp]
        L.lbmo_central_moments.argtypes = [C.c_int, _dp, _dp, _dp]
        L.lbmo_cumulants_forward.argtypes = [C.c_int, _dp, _dp]
        L.lbmo_cumulants_inverse.argtypes = [C.c_int, _dp, _dp]
        L.lbmo_kron_inverse.argtypes = [C.c_int, _dp, _dp, _dp]
        L.lbmo_collide_cell.argtypes = [C.c_void_p, _dp, _dp, C.c_double, _dp, C.c_double,
                                        _dp, _dp, C.c_void_p]
        L.lbmo_collide_cell_prev.argtypes = [C.c_void_p, _dp, _dp, C.c_double, _dp, C.c_double,
                                             C.c_void_p, _dp, _dp, C.c_void_p]
        L.lbmo_phase_lattice.argtypes = [C.c_int, C.c_int, C.POINTER(C.c_int), C.c_void_p, C.c_void_p,
                                         C.POINTER(C.c_double)]
        L.lbmo_collide_cell_ex.argtypes = [C.c_void_p, _dp, _dp, C.c_double, _dp, C.c_double,
                                           C.c_void_p, C.c_double, _dp, _dp, C.c_void_p]
        L.lbmo_divu.argtypes = [C.c_void_p, _dp, _dp]
        L.lbmo_phase_q.argtypes = [C.c_void_p]
        L.lbmo_phase_q.restype = C.c_int
        L.lbmo_splitmix64.restype = C.c_ulonglong
        L.lbmo_splitmix64.argtypes = [C.c_ulonglong, C.c_ulonglong]
        _lib = L
    return _lib


def make_phys(**kw) -> Phys:
    p = Phys(rho_ratio=1.0, nu_ratio=1.0, We=0.0, Re=0.0, atwood=0.0, mobility=0.02,
             width=5.0, g_accel=0.0, U0=0.0, L_ref=0.0, sigma=-1.0, nu_h=-1.0, force_x=0.0,
             flags=0)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def derive(D: int, **kw) -> Derived:
    d = Derived()
    if lib().lbmo_derive(D, C.byref(make_phys(**kw)), C.byref(d)) != 0:
        raise ValueError(lib().lbmo_last_error().decode())
    return d


def lattice(D: int):
    Q = C.c_int()
    c = np.zeros((27, 3), dtype=np.int32)
    w = np.zeros(27)
    lib().lbmo_lattice(D, C.byref(Q), c.ctypes.data, w.ctypes.data)
    return c[:Q.value].copy(), w[:Q.value].copy()


def phase_lattice(D: int, reduced: bool):
    """(c, w, cs2) of the phase-field lattice: the flow lattice, or D3Q7 / D2Q5."""
    Q = C.c_int()
    cs2 = C.c_double()
    c = np.zeros((27, 3), dtype=np.int32)
    w = np.zeros(27)
    lib().lbmo_phase_lattice(D, int(bool(reduced)), C.byref(Q), c.ctypes.data, w.ctypes.data, C.byref(cs2))
    return c[:Q.value].copy(), w[:Q.value].copy(), cs2.value


def splitmix64(seed: int, counter: int) -> int:
    return int(lib().lbmo_splitmix64(seed, counter))


def central_moments(D, h, u):
    out = np.zeros(27)
    lib().lbmo_central_moments(D, np.ascontiguousarray(h, dtype=np.float64),
                               np.ascontiguousarray(u, dtype=np.float64), out)
    return out


def cumulants_forward(D, k):
    out = np.zeros(27)
    lib().lbmo_cumulants_forward(D, np.ascontiguousarray(k, dtype=np.float64), out)
    return out


def cumulants_inverse(D, K):
    out = np.zeros(27)
    lib().lbmo_cumulants_inverse(D, np.ascontiguousarray(K, dtype=np.float64), out)
    return out


def kron_inverse(D, k, u):
    out = np.zeros(27)
    lib().lbmo_kron_inverse(D, np.ascontiguousarray(k, dtype=np.float64),
                            np.ascontiguousarray(u, dtype=np.float64), out)
    return out


class Oracle:
    """One FP64 CPU domain.  dims = (nx, ny, nz); nz = 1 for D = 2."""

    def __init__(self, D, dims, periodic=(1, 1, 1), **phys):
        self.D = D
        self.dims = tuple(int(v) for v in dims)
        self.Q = 27 if D == 3 else 9
        self.N = self.dims[0] * self.dims[1] * self.dims[2]
        d = (C.c_int * 3)(*self.dims)
        p = (C.c_int * 3)(*[int(v) for v in periodic])
        self._h = lib().lbmo_create(D, d, p, C.byref(make_phys(**phys)))
        if not self._h:
            raise ValueError(lib().lbmo_last_error().decode())
        self.Qg = int(lib().lbmo_phase_q(self._h))

    def close(self):
        if self._h:
            lib().lbmo_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def shape(self):
        nx, ny, nz = self.dims
        return (self.Q, nz, ny, nx)

    def derived(self) -> Derived:
        d = Derived()
        lib().lbmo_get_derived(self._h, C.byref(d))
        return d

    def set_rates(self, shear=-1.0, bulk=1.0, r3=1.0, r4=1.0, r5=1.0, r6=1.0):
        lib().lbmo_set_rates(self._h, shear, bulk, r3, r4, r5, r6)

    def init(self, case, args, seed=0):
        cid = CASE[case] if isinstance(case, str) else int(case)
        a = (C.c_double * max(1, len(args)))(*args)
        if lib().lbmo_init(self._h, cid, a, len(args), seed) != 0:
            raise ValueError(lib().lbmo_last_error().decode())

    def step(self, n=1):
        lib().lbmo_step(self._h, int(n))

    @property
    def gshape(self):
        return (self.Qg,) + self.shape[1:]

    def get_state(self):
        f = np.zeros(self.shape)
        g = np.zeros(self.gshape)
        phi = np.zeros(self.shape[1:])
        lib().lbmo_get_state(self._h, f.ctypes.data, g.ctypes.data, phi.ctypes.data)
        return f, g, phi

    def set_state(self, f, g):
        lib().lbmo_set_state(self._h, np.ascontiguousarray(f, dtype=np.float64).ravel(),
                             np.ascontiguousarray(g, dtype=np.float64).ravel())

    def observables(self) -> Obs:
        o = Obs()
        lib().lbmo_observables(self._h, C.byref(o))
        return o

    def fields(self):
        rho = np.zeros(self.shape[1:])
        p = np.zeros(self.shape[1:])
        u = np.zeros((self.D,) + self.shape[1:])
        lib().lbmo_fields(self._h, rho.ctypes.data, p.ctypes.data, u.ctypes.data)
        return rho, p, u

    def fd(self, field):
        field = np.ascontiguousarray(field, dtype=np.float64)
        grad = np.zeros(self.shape[1:] + (3,))
        lap = np.zeros(self.shape[1:])
        lib().lbmo_fd(self._h, field.ravel(), grad.ravel(), lap.ravel())
        return grad, lap

    def collide_cell(self, f, g, phi, grad, lap, phiu_prev=None, divu=0.0):
        """One cell's collision; phiu_prev: the previous step's phi u (reduced
        phase lattice; None = no time derivative); divu: div(u) for the
        w cs2 rho div(u) term (FLAG_DIVU).  diag[14:17] = phi u."""
        fo = np.zeros(self.Q)
        go = np.zeros(self.Qg)
        diag = np.zeros(17)
        prev = None if phiu_prev is None else np.ascontiguousarray(phiu_prev, dtype=np.float64)
        lib().lbmo_collide_cell_ex(self._h, np.ascontiguousarray(f, dtype=np.float64),
                                   np.ascontiguousarray(g, dtype=np.float64), float(phi),
                                   np.ascontiguousarray(grad, dtype=np.float64), float(lap),
                                   None if prev is None else prev.ctypes.data, float(divu), fo, go,
                                   diag.ctypes.data)
        return fo, go, diag

    def divu(self, u):
        """div(u) of a velocity field u[k][z][y][x] (k < 3) by the isotropic
        difference, no-slip ghosts across walls"""
        u3 = np.zeros((3,) + self.shape[1:])
        u3[:len(u)] = u
        out = np.zeros(self.shape[1:])
        lib().lbmo_divu(self._h, np.ascontiguousarray(u3).ravel(), out.ravel())
        return out


def set_threads(n: int):
    lib().lbmo_set_threads(int(n))


def get_threads() -> int:
    return int(lib().lbmo_get_threads())
