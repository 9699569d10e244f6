"""Launch-shape tuning cache over lbmp_autotune (host logic only: the trials
run in the CUDA library).

The cache maps a key (device name, lattice, phase lattice, storage, grid,
boundaries) to the
chosen (chunk, ctas_per_sm).  It is a JSON file, LBMP_TUNE_CACHE or
~/.cache/lbmp/tune.json, written atomically (temporary file + rename).
"""
import ctypes as C
import json
import os

from .lbmp import OPT_CHUNK, OPT_CTAS_PER_SM, OPT_TILE, TuneEntry, _check, load


def cache_path():
    return os.environ.get("LBMP_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "lbmp",
                                                              "tune.json")


def device_name():
    buf = C.create_string_buffer(256)
    _check(load().lbmp_device_name(buf, 256))
    return buf.value.decode()


def key_of(dom, device):
    parts = [device, f"D{dom.D}"]
    if dom.Qg != dom.Q:  # the reduced phase lattice runs its own kernel
        parts.append(f"g{dom.Qg}")
    return "|".join(parts + [f"storage{dom.storage}", "x".join(map(str, dom.dims)),
                             "p" + "".join(map(str, dom.periodic))])


def read_cache(path):
    try:
        with open(path) as fh:
            data = json.load(fh)
        return data if isinstance(data, dict) else {}
    except (OSError, ValueError):
        return {}


def write_cache(path, data):
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = f"{path}.{os.getpid()}.tmp"
    with open(tmp, "w") as fh:
        json.dump(data, fh, indent=1, sort_keys=True)
    os.replace(tmp, path)


def apply(dom, chunk, ctas, tile=0):
    L = load()
    _check(L.lbmp_set_option(dom.handle, OPT_CHUNK, int(chunk)))
    _check(L.lbmp_set_option(dom.handle, OPT_CTAS_PER_SM, int(ctas)))
    _check(L.lbmp_set_option(dom.handle, OPT_TILE, int(tile)))


def autotune(dom, reps=5, cache=True):
    path = cache_path()
    key = key_of(dom, device_name()) if cache else None
    if cache:
        hit = read_cache(path).get(key)
        if hit:
            apply(dom, hit["chunk"], hit["ctas_per_sm"], hit.get("tile", 0))
            return hit["chunk"], hit["ctas_per_sm"], []
    table = (TuneEntry * 256)()
    n = C.c_int(0)
    _check(load().lbmp_autotune(dom.handle, int(reps), table, 256, C.byref(n)))
    trials = [(table[k].chunk, table[k].ctas_per_sm, table[k].ms, table[k].tile) for k in range(min(n.value, 256))]
    if not trials:
        return 0, 0, []
    best = min(trials, key=lambda t: t[2])
    if cache:
        data = read_cache(path)
        data[key] = {"chunk": best[0], "ctas_per_sm": best[1], "ms": best[2], "tile": best[3]}
        write_cache(path, data)
    return best[0], best[1], trials
