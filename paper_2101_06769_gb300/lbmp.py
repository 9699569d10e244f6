"""ctypes binding of the C ABI in include/lbmp.h (argument marshalling only).

Every step of the multiphase update runs in the CUDA library
``_build/liblbmp.so``; this module converts Python arguments to the C
structures and back.  There is no CPU fallback: if the library is missing or
no GPU is present the calls raise.
"""
import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblbmp.so")

D2Q9, D3Q27 = 0, 1
FP32, FP16_SHIFTED, BF16_SHIFTED = 0, 1, 2
CASE = {"rt": 0, "drop_static": 1, "flat": 2, "poiseuille": 3, "drop_sheet": 4, "shear_wave": 5,
        "uniform": 6}
FLAG_WE_LIGHT, FLAG_DYNAMIC_VISC, FLAG_UNIFORM_FORCE, FLAG_PHASE_REDUCED, FLAG_DIVU, FLAG_AA = 1, 2, 4, 8, 16, 32
OPT_KERNEL, OPT_CHUNK, OPT_CTAS_PER_SM, OPT_WAIT_LIMIT_NS, OPT_TEST_STALL, OPT_TILE = 0, 1, 2, 3, 4, 5
OPT_TEST_POISON = 6
ERRORS = {0: "OK", -1: "INVALID_ARG", -2: "NOMEM", -3: "CUDA", -4: "TIMEOUT", -5: "UNSTABLE",
          -6: "UNSUPPORTED"}

# every entry point declared in include/lbmp.h
EXPORTS = ("lbmp_create", "lbmp_create_ex", "lbmp_destroy", "lbmp_last_error", "lbmp_get_derived", "lbmp_init",
           "lbmp_step", "lbmp_sync", "lbmp_observables", "lbmp_get_state", "lbmp_set_state",
           "lbmp_state_bytes", "lbmp_upload", "lbmp_download", "lbmp_set_option", "lbmp_mass_noalloc",
           "lbmp_batch_create", "lbmp_batch_destroy", "lbmp_batch_add", "lbmp_batch_remove",
           "lbmp_batch_step", "lbmp_batch_members", "lbmp_autotune", "lbmp_device_name",
           "lbmp_batch_autotune", "lbmp_create_slab", "lbmp_slab_layout", "lbmp_pack_planes",
           "lbmp_unpack_planes")


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("periodic", C.c_int * 3)]


class Params(C.Structure):
    _fields_ = [(n, C.c_double) for n in
                ("rho_ratio", "nu_ratio", "We", "Re", "atwood", "mobility", "width", "g_accel",
                 "U0", "L_ref", "sigma", "nu_h", "force_x")] + [("storage", C.c_int),
                                                                ("flags", C.c_uint)]


class Derived(C.Structure):
    _fields_ = [(n, C.c_double) for n in
                ("rho_h", "rho_l", "nu_h", "nu_l", "sigma", "beta", "kappa", "M", "W", "tau_phi",
                 "lambda_phi", "g_accel", "U_ref", "force_x")]


class Obs(C.Structure):
    _fields_ = [(n, C.c_double) for n in
                ("mass", "mass_drift_rel", "kinetic_energy", "max_u", "p_in", "p_out", "laplace_dp",
                 "tip_spike", "tip_bubble")] + [("step", C.c_long), ("health", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# lbmp_allocator: caller-supplied device memory (include/lbmp.h)
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class Allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", C.c_void_p)]


def make_allocator(alloc, free):
    """An lbmp_allocator from two Python callables: alloc(nbytes, stream)
    returns a device address (int) or 0, free(ptr, nbytes, stream).  Keep the
    returned structure alive as long as any handle created with it."""
    def _alloc(nbytes, stream, ctx):
        try:
            return int(alloc(int(nbytes), int(stream or 0))) or None
        except Exception:
            return None

    def _free(ptr, nbytes, stream, ctx):
        free(int(ptr), int(nbytes), int(stream or 0))

    return Allocator(ALLOC_FN(_alloc), FREE_FN(_free), None)


def torch_allocator(device=None):
    """lbmp_allocator backed by torch's CUDA caching allocator: the library's
    device arrays then count in torch.cuda.memory_allocated() and reuse the
    cache of the calling process."""
    import torch
    dev = torch.cuda.current_device() if device is None else int(device)
    return make_allocator(lambda n, s: torch.cuda.caching_allocator_alloc(n, dev, s),
                          lambda p, n, s: torch.cuda.caching_allocator_delete(p))


class TuneEntry(C.Structure):
    _fields_ = [("chunk", C.c_int), ("ctas_per_sm", C.c_int), ("ms", C.c_double), ("tile", C.c_int)]


class LbmpError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def load(path=None):
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or os.environ.get("LBMP_LIBRARY") or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    L = C.CDLL(path)
    vp = C.c_void_p
    L.lbmp_create.argtypes = [C.POINTER(Grid), C.c_int, C.POINTER(Params), vp, C.POINTER(vp)]
    L.lbmp_create_ex.argtypes = [C.POINTER(Grid), C.c_int, C.POINTER(Params), vp, C.POINTER(Allocator),
                                 C.POINTER(vp)]
    L.lbmp_create_slab.argtypes = [C.POINTER(Grid), C.c_int, C.c_int, C.c_int, C.POINTER(Params), vp,
                                   C.POINTER(Allocator), C.POINTER(vp)]
    L.lbmp_slab_layout.argtypes = [vp, C.POINTER(C.c_int)]
    L.lbmp_pack_planes.argtypes = [vp, C.POINTER(C.c_int), C.c_int, vp]
    L.lbmp_unpack_planes.argtypes = [vp, C.POINTER(C.c_int), C.c_int, vp]
    L.lbmp_destroy.argtypes = [vp]
    L.lbmp_last_error.restype = C.c_char_p
    L.lbmp_get_derived.argtypes = [vp, C.POINTER(Derived)]
    L.lbmp_init.argtypes = [vp, C.c_int, C.POINTER(C.c_double), C.c_int, C.c_ulonglong]
    L.lbmp_step.argtypes = [vp, C.c_long]
    L.lbmp_sync.argtypes = [vp]
    L.lbmp_observables.argtypes = [vp, C.POINTER(Obs)]
    L.lbmp_get_state.argtypes = [vp, vp, vp, vp]
    L.lbmp_set_state.argtypes = [vp, vp, vp]
    L.lbmp_state_bytes.restype = C.c_size_t
    L.lbmp_state_bytes.argtypes = [vp]
    L.lbmp_upload.argtypes = [vp, vp, C.c_size_t]
    L.lbmp_download.argtypes = [vp, vp, C.c_size_t]
    L.lbmp_set_option.argtypes = [vp, C.c_int, C.c_long]
    L.lbmp_mass_noalloc.argtypes = [vp, C.c_longlong, C.POINTER(C.c_double), vp]
    L.lbmp_batch_create.argtypes = [C.c_size_t, vp, C.POINTER(vp)]
    L.lbmp_batch_destroy.argtypes = [vp]
    L.lbmp_batch_add.argtypes = [vp, vp, C.c_long]
    L.lbmp_batch_remove.argtypes = [vp, vp]
    L.lbmp_batch_step.argtypes = [vp, C.c_long, C.POINTER(C.c_int)]
    L.lbmp_batch_members.argtypes = [vp, C.POINTER(vp), C.POINTER(C.c_long), C.c_int]
    L.lbmp_autotune.argtypes = [vp, C.c_int, C.POINTER(TuneEntry), C.c_int, C.POINTER(C.c_int)]
    L.lbmp_device_name.argtypes = [C.c_char_p, C.c_int]
    L.lbmp_batch_autotune.argtypes = [vp, C.c_int, C.POINTER(TuneEntry), C.c_int, C.POINTER(C.c_int)]
    _lib = L
    return L


def _check(rc):
    if rc != 0:
        raise LbmpError(rc, load().lbmp_last_error().decode())
    return rc


def make_params(**kw):
    p = Params(rho_ratio=1.0, nu_ratio=1.0, We=0.0, Re=0.0, atwood=0.0, mobility=0.02, width=5.0,
               g_accel=0.0, U0=0.0, L_ref=0.0, sigma=-1.0, nu_h=-1.0, force_x=0.0, storage=FP32,
               flags=0)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


class Domain:
    """One simulation domain on the current CUDA device.

    dims = (nx, ny, nz) with nz = 1 for D = 2; periodic = (px, py, pz).
    ``stream`` is a raw cudaStream_t handle (int) or None for the default stream.
    """

    def __init__(self, D, dims, periodic=(1, 1, 1), stream=None, allocator=None, **params):
        """allocator: None (cudaMalloc), "torch" (torch's caching allocator)
        or an Allocator structure (make_allocator)."""
        L = load()
        self.D = D
        self.periodic = tuple(int(v) for v in periodic)
        self.storage = int(params.get("storage", FP32))
        self.dims = tuple(int(v) for v in dims)
        self.Q = 27 if D == 3 else 9
        # phase-field populations: 2D+1 on the reduced phase lattice (D3Q7 / D2Q5)
        self.Qg = 2 * D + 1 if int(params.get("flags", 0)) & FLAG_PHASE_REDUCED else self.Q
        self.N = self.dims[0] * self.dims[1] * self.dims[2]
        g = Grid(self.dims[0], self.dims[1], self.dims[2], (C.c_int * 3)(*[int(v) for v in periodic]))
        h = C.c_void_p()
        if isinstance(allocator, str):
            if allocator != "torch":
                raise ValueError(f"unknown allocator {allocator!r}")
            allocator = torch_allocator()
        self._allocator = allocator  # the callbacks must outlive the handle
        lat = D3Q27 if D == 3 else D2Q9
        st = C.c_void_p(stream) if stream else None
        if allocator is None:
            _check(L.lbmp_create(C.byref(g), lat, C.byref(make_params(**params)), st, C.byref(h)))
        else:
            _check(L.lbmp_create_ex(C.byref(g), lat, C.byref(make_params(**params)), st, C.byref(allocator),
                                    C.byref(h)))
        self._h = h

    @property
    def handle(self):
        return self._h

    @property
    def shape(self):
        nx, ny, nz = self.dims
        return (self.Q, nz, ny, nx)

    @property
    def gshape(self):
        return (self.Qg,) + self.shape[1:]

    def close(self):
        if getattr(self, "_h", None):
            load().lbmp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def derived(self):
        d = Derived()
        _check(load().lbmp_get_derived(self._h, C.byref(d)))
        return d

    def set_kernel(self, k):
        _check(load().lbmp_set_option(self._h, OPT_KERNEL, int(k)))

    def set_option(self, option, value):
        _check(load().lbmp_set_option(self._h, int(option), int(value)))

    def autotune(self, reps=5, cache=True):
        """Pick the fused kernel's launch shape (lbmp_autotune).  With
        cache=True the choice is stored per (device, lattice, storage, grid,
        boundaries) in a JSON file (LBMP_TUNE_CACHE, default
        ~/.cache/lbmp/tune.json) and reused without trials.  Returns
        (chunk, ctas_per_sm, trials) with trials a list of
        (chunk, ctas, ms, tile); the chosen tile is applied as LBMP_OPT_TILE."""
        from . import tune
        return tune.autotune(self, reps=reps, cache=cache)

    def init(self, case, args, seed=0):
        cid = CASE[case] if isinstance(case, str) else int(case)
        a = (C.c_double * max(1, len(args)))(*args)
        _check(load().lbmp_init(self._h, cid, a, len(args), int(seed)))

    def step(self, n=1):
        _check(load().lbmp_step(self._h, int(n)))

    def sync(self):
        _check(load().lbmp_sync(self._h))

    def observables(self):
        o = Obs()
        rc = load().lbmp_observables(self._h, C.byref(o))
        if rc not in (0, -5):
            _check(rc)
        return o

    def get_state(self):
        f = np.empty(self.shape)
        g = np.empty(self.gshape)
        phi = np.empty(self.shape[1:])
        _check(load().lbmp_get_state(self._h, f.ctypes.data, g.ctypes.data, phi.ctypes.data))
        return f, g, phi

    def get_phi(self):
        """phi alone in the exchange format (lbmp_get_state with f and g NULL)"""
        phi = np.empty(self.shape[1:])
        _check(load().lbmp_get_state(self._h, None, None, phi.ctypes.data))
        return phi

    def set_state(self, f, g):
        f = np.ascontiguousarray(f, dtype=np.float64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        assert f.size == self.Q * self.N and g.size == self.Qg * self.N
        _check(load().lbmp_set_state(self._h, f.ctypes.data, g.ctypes.data))

    def state_bytes(self):
        return int(load().lbmp_state_bytes(self._h))

    def upload(self, host_ptr, nbytes):
        _check(load().lbmp_upload(self._h, C.c_void_p(host_ptr), nbytes))

    def download(self, host_ptr, nbytes):
        _check(load().lbmp_download(self._h, C.c_void_p(host_ptr), nbytes))


class Batch:
    """Domains advanced together by one persistent kernel per step (see
    lbmp_batch_* in include/lbmp.h).  Members stay owned by the caller."""

    def __init__(self, hbm_budget=0, stream=None):
        h = C.c_void_p()
        _check(load().lbmp_batch_create(int(hbm_budget), C.c_void_p(stream) if stream else None, C.byref(h)))
        self._h = h
        self._members = {}

    def close(self):
        if getattr(self, "_h", None):
            load().lbmp_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add(self, dom, steps):
        rc = load().lbmp_batch_add(self._h, dom.handle, int(steps))
        _check(rc)
        self._members[dom.handle.value] = dom

    def try_add(self, dom, steps):
        """False (instead of raising) when the domain does not fit the budget"""
        rc = load().lbmp_batch_add(self._h, dom.handle, int(steps))
        if rc == -2:
            return False
        _check(rc)
        self._members[dom.handle.value] = dom
        return True

    def remove(self, dom):
        _check(load().lbmp_batch_remove(self._h, dom.handle))
        self._members.pop(dom.handle.value, None)

    def step(self, n):
        fin = C.c_int(0)
        _check(load().lbmp_batch_step(self._h, int(n), C.byref(fin)))
        return fin.value

    def members(self):
        n = load().lbmp_batch_members(self._h, None, None, 0)
        if n < 0:
            _check(n)
        hs = (C.c_void_p * max(1, n))()
        left = (C.c_long * max(1, n))()
        load().lbmp_batch_members(self._h, hs, left, n)
        return [(self._members.get(hs[k]), int(left[k])) for k in range(n)]

    def autotune(self, reps=3):
        """Pick the batch kernels' tile shape and planes per work item for the
        current members (lbmp_batch_autotune); returns the best trial
        (chunk, ms, tile) and the list of trials."""
        table = (TuneEntry * 64)()
        n = C.c_int(0)
        _check(load().lbmp_batch_autotune(self._h, int(reps), table, 64, C.byref(n)))
        trials = [(table[k].chunk, table[k].ms, table[k].tile) for k in range(min(n.value, 64))]
        best = min(trials, key=lambda t: t[1]) if trials else None
        return best, trials
