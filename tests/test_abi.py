"""CPU checks of the C-ABI library: it builds for sm_103a, loads, exports every
entry point include/lbmp.h declares, and the ctypes structures of the binding
match the C layout (offsets checked by compiling a probe against the header)."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import pytest

import paper_2101_06769_gb300 as P
from paper_2101_06769_gb300 import build as lib_build
from paper_2101_06769_gb300 import lbmp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbmp.h")


def header_functions():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"LBMP_API\s+[\w\s\*]*?\b(lbmp_\w+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    lib_build.build()
    return lbmp.load()


def test_exports_every_declared_symbol(lib):
    declared = header_functions()
    assert len(declared) >= 14
    assert sorted(P.EXPORTS) == declared
    out = subprocess.run(["nm", "-D", "--defined-only", lbmp.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r" T (lbmp_\w+)", out))
    for name in declared:
        assert name in exported, name
        assert hasattr(lib, name)
    # nothing else leaks out of the library
    assert exported == set(declared)


def test_struct_layout_matches_header():
    probe = r"""
#include <stdio.h>
#include <stddef.h>
#include "lbmp.h"
#define O(T, f) printf(#T "." #f " %zu\n", offsetof(T, f))
int main(void) {
  printf("lbmp_grid %zu\nlbmp_params %zu\nlbmp_obs %zu\nlbmp_derived %zu\nlbmp_tune_entry %zu\n",
         sizeof(lbmp_grid), sizeof(lbmp_params), sizeof(lbmp_obs), sizeof(lbmp_derived),
         sizeof(lbmp_tune_entry));
  O(lbmp_tune_entry, ms); O(lbmp_tune_entry, tile);
  O(lbmp_grid, periodic); O(lbmp_params, force_x); O(lbmp_params, storage); O(lbmp_params, flags);
  O(lbmp_obs, tip_bubble); O(lbmp_obs, step); O(lbmp_obs, health); O(lbmp_derived, force_x);
  printf("lbmp_allocator %zu\n", sizeof(lbmp_allocator));
  O(lbmp_allocator, alloc); O(lbmp_allocator, free); O(lbmp_allocator, ctx);
  return 0;
}
"""
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "probe.c")
        exe = os.path.join(d, "probe")
        open(src, "w").write(probe)
        subprocess.run(["gcc", "-std=c11", "-I", os.path.dirname(HEADER), src, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout
    vals = dict(line.rsplit(" ", 1) for line in out.strip().splitlines())
    assert int(vals["lbmp_grid"]) == C.sizeof(lbmp.Grid)
    assert int(vals["lbmp_params"]) == C.sizeof(lbmp.Params)
    assert int(vals["lbmp_obs"]) == C.sizeof(lbmp.Obs)
    assert int(vals["lbmp_derived"]) == C.sizeof(lbmp.Derived)
    assert int(vals["lbmp_grid.periodic"]) == lbmp.Grid.periodic.offset
    assert int(vals["lbmp_params.force_x"]) == lbmp.Params.force_x.offset
    assert int(vals["lbmp_params.storage"]) == lbmp.Params.storage.offset
    assert int(vals["lbmp_params.flags"]) == lbmp.Params.flags.offset
    assert int(vals["lbmp_obs.tip_bubble"]) == lbmp.Obs.tip_bubble.offset
    assert int(vals["lbmp_obs.step"]) == lbmp.Obs.step.offset
    assert int(vals["lbmp_obs.health"]) == lbmp.Obs.health.offset
    assert int(vals["lbmp_derived.force_x"]) == lbmp.Derived.force_x.offset
    assert int(vals["lbmp_tune_entry"]) == C.sizeof(lbmp.TuneEntry)
    assert int(vals["lbmp_tune_entry.ms"]) == lbmp.TuneEntry.ms.offset
    assert int(vals["lbmp_tune_entry.tile"]) == lbmp.TuneEntry.tile.offset
    assert int(vals["lbmp_allocator"]) == C.sizeof(lbmp.Allocator)
    for f in ("alloc", "free", "ctx"):
        assert int(vals["lbmp_allocator." + f]) == getattr(lbmp.Allocator, f).offset


def test_invalid_arguments_rejected_without_device_work(lib):
    """Validation happens before any CUDA call, so it is testable on a host
    without a GPU: bad grids and parameters return INVALID_ARG."""
    h = C.c_void_p()
    p = lbmp.make_params(rho_ratio=3.0, nu_h=0.1)
    bad = [
        (lbmp.Grid(0, 4, 4, (C.c_int * 3)(1, 1, 0)), lbmp.D3Q27, p),
        (lbmp.Grid(4, 4, 2, (C.c_int * 3)(1, 1, 1)), lbmp.D2Q9, p),
        (lbmp.Grid(4, 4, 4, (C.c_int * 3)(0, 1, 1)), lbmp.D3Q27, p),
        (lbmp.Grid(4, 4, 4, (C.c_int * 3)(1, 1, 1)), lbmp.D3Q27, lbmp.make_params(rho_ratio=-1.0, nu_h=0.1)),
        (lbmp.Grid(4, 4, 4, (C.c_int * 3)(1, 1, 1)), lbmp.D3Q27, lbmp.make_params(rho_ratio=2.0)),
        (lbmp.Grid(4, 4, 4, (C.c_int * 3)(1, 1, 1)), lbmp.D3Q27,
         lbmp.make_params(rho_ratio=2.0, nu_h=0.1, width=0.0)),
        (lbmp.Grid(4, 4, 4, (C.c_int * 3)(1, 1, 1)), 7, p),
    ]
    for g, lat, prm in bad:
        rc = lib.lbmp_create(C.byref(g), lat, C.byref(prm), None, C.byref(h))
        assert rc == -1, (rc, lib.lbmp_last_error())
        assert not h.value
    assert lib.lbmp_step(None, 1) == -1
    assert b"null" in lib.lbmp_last_error()


def test_size_flag_and_form_limits_rejected_without_device_work(lib):
    """More limits checked before any CUDA call: more than 2^31-1 cells, 16-bit
    storage with an odd nx, unknown flag bits (INVALID_ARG); the reduced phase
    lattice or the divergence term with 16-bit storage, the two flags
    together, in-place AA storage outside D3Q27 FP32 with the full phase
    lattice, and FP32 two-set domains of 2^30 cells, whose arrays their
    kernels could not address by 32-bit byte offsets (UNSUPPORTED)."""
    h = C.c_void_p()
    per = (C.c_int * 3)(1, 1, 0)
    ok = dict(rho_ratio=3.0, nu_h=0.1)
    cases = [
        (lbmp.Grid(2048, 2048, 1024, per), lbmp.make_params(**ok), -1),
        (lbmp.Grid(37, 8, 8, per), lbmp.make_params(storage=lbmp.FP16_SHIFTED, **ok), -1),
        (lbmp.Grid(8, 8, 8, per), lbmp.make_params(flags=1 << 6, **ok), -1),
        (lbmp.Grid(8, 8, 8, per), lbmp.make_params(flags=lbmp.FLAG_AA, storage=lbmp.FP16_SHIFTED, **ok), -6),
        (lbmp.Grid(8, 8, 8, per), lbmp.make_params(flags=lbmp.FLAG_AA | lbmp.FLAG_PHASE_REDUCED, **ok), -6),
        (lbmp.Grid(8, 8, 8, per), lbmp.make_params(flags=lbmp.FLAG_AA | lbmp.FLAG_DIVU, **ok), -6),
        (lbmp.Grid(8, 8, 8, per), lbmp.make_params(flags=lbmp.FLAG_PHASE_REDUCED, storage=lbmp.FP16_SHIFTED, **ok), -6),
        (lbmp.Grid(8, 8, 8, per), lbmp.make_params(flags=lbmp.FLAG_DIVU, storage=lbmp.BF16_SHIFTED, **ok), -6),
        (lbmp.Grid(8, 8, 8, per), lbmp.make_params(flags=lbmp.FLAG_DIVU | lbmp.FLAG_PHASE_REDUCED, **ok), -6),
        (lbmp.Grid(1024, 1024, 1024, per), lbmp.make_params(**ok), -6),
        (lbmp.Grid(1024, 1024, 1024, per), lbmp.make_params(flags=lbmp.FLAG_PHASE_REDUCED, **ok), -6),
    ]
    for g, prm, want in cases:
        rc = lib.lbmp_create(C.byref(g), lbmp.D3Q27, C.byref(prm), None, C.byref(h))
        assert rc == want, (rc, lib.lbmp_last_error())
        assert not h.value
    per2 = (C.c_int * 3)(1, 0, 1)
    for prm in (lbmp.make_params(**ok), lbmp.make_params(flags=lbmp.FLAG_PHASE_REDUCED, **ok)):
        rc = lib.lbmp_create(C.byref(lbmp.Grid(32768, 32768, 1, per2)), lbmp.D2Q9, C.byref(prm), None, C.byref(h))
        assert rc == -6, (rc, lib.lbmp_last_error())
        assert not h.value


def test_symmetry_axis_limits_rejected_without_device_work(lib):
    """A symmetry axis (periodic = 2) is the x axis of a D2Q9 FP32 domain
    without the divergence term: elsewhere creation fails before any CUDA
    call (INVALID_ARG for the axis, UNSUPPORTED for the form)."""
    h = C.c_void_p()
    ok = dict(rho_ratio=3.0, nu_ratio=1.0, nu_h=0.05)
    cases = [
        (lbmp.Grid(8, 8, 8, (C.c_int * 3)(2, 1, 0)), lbmp.D3Q27, lbmp.make_params(**ok), -1),
        (lbmp.Grid(8, 8, 1, (C.c_int * 3)(1, 2, 1)), lbmp.D2Q9, lbmp.make_params(**ok), -1),
        (lbmp.Grid(8, 8, 1, (C.c_int * 3)(2, 0, 1)), lbmp.D2Q9, lbmp.make_params(storage=lbmp.FP16_SHIFTED, **ok), -6),
        (lbmp.Grid(8, 8, 1, (C.c_int * 3)(2, 0, 1)), lbmp.D2Q9, lbmp.make_params(flags=lbmp.FLAG_DIVU, **ok), -6),
    ]
    for g, lat, prm, want in cases:
        rc = lib.lbmp_create(C.byref(g), lat, C.byref(prm), None, C.byref(h))
        assert rc == want, (rc, lib.lbmp_last_error())
        assert not h.value
