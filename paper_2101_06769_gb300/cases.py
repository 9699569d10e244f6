"""JSON case files: a problem statement (lattice, grid, boundaries, the
physical parameters of lbmp_params, the initial condition) that maps onto
lbmp_create and lbmp_init.  The benchmark workloads ship as cases/*.json.

    {"name": ..., "desc": ..., "lattice": "D3Q27" | "D2Q9",
     "grid": [nx, ny, nz], "periodic": [px, py, pz],
     "params": {<lbmp_params field>: value, ...},
     "init": {"case": <LBMP_CASE name>, "args": [...], "seed": int}}
"""
import json
import os

from .lbmp import CASE, Domain, Params

CASE_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cases")
PARAM_FIELDS = {name for name, _ in Params._fields_}


def load(name_or_path):
    """A case by file path, or by the name of a shipped case."""
    path = name_or_path
    if not os.path.exists(path):
        path = os.path.join(CASE_DIR, name_or_path + ".json")
    with open(path) as fh:
        case = json.load(fh)
    validate(case)
    return case


def shipped():
    return sorted(f[:-5] for f in os.listdir(CASE_DIR) if f.endswith(".json"))


def validate(case):
    for key in ("lattice", "grid", "periodic", "params", "init"):
        if key not in case:
            raise ValueError(f"case lacks '{key}'")
    if case["lattice"] not in ("D3Q27", "D2Q9"):
        raise ValueError("lattice must be D3Q27 or D2Q9")
    if len(case["grid"]) != 3 or len(case["periodic"]) != 3:
        raise ValueError("grid and periodic take three entries")
    unknown = set(case["params"]) - PARAM_FIELDS
    if unknown:
        raise ValueError(f"unknown parameters: {sorted(unknown)}")
    if case["init"].get("case") not in CASE:
        raise ValueError("unknown initial condition")


def as_workload(case):
    """The case in the form the benchmark uses (D, dims, periodic, phys, ...)."""
    return dict(desc=case.get("desc", case.get("name", "")), D=3 if case["lattice"] == "D3Q27" else 2,
                dims=tuple(case["grid"]), periodic=tuple(case["periodic"]), phys=dict(case["params"]),
                case=case["init"]["case"], args=list(case["init"]["args"]), seed=int(case["init"].get("seed", 0)))


def make_domain(case, stream=None, **overrides):
    """Create and initialise the domain of a case (overrides: lbmp_params fields)."""
    wl = as_workload(case)
    phys = dict(wl["phys"])
    phys.update(overrides)
    d = Domain(wl["D"], wl["dims"], wl["periodic"], stream=stream, **phys)
    d.init(wl["case"], wl["args"], seed=wl["seed"])
    return d
