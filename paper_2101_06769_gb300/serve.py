"""Continuous-batching request loop over the batch form of the library.

A request is one simulation: a Rayleigh-Taylor or droplet-on-sheet case (the
paper's Sec. 3.2-3.4 set-ups) of a given size, lattice, parameter set and
step count.  Requests arrive over time (a seeded Poisson process); the loop
admits every arrived request whose device state fits the free HBM (minus a
reserve), adds it to one lbmp batch, advances the batch a round of steps at a
time (one persistent kernel per lattice type per step, replayed as a CUDA
graph), and retires requests as their steps run out: their observables are
read back, their memory freed, and the freed memory admits waiting requests
before the next round.  After every `health_every` rounds the observables of
every running request are read; a request whose state has become
non-finite or unstable (library health word set) is evicted as failed at
once, its memory freed, and the others continue.  Work of requests that
arrive while others are running overlaps on the device.

Every arithmetic step runs in the CUDA library; this module only schedules.
"""
import math
import time
from dataclasses import dataclass, field

import numpy as np

from .lbmp import Batch, Domain, LbmpError


@dataclass
class Request:
    rid: int
    kind: str            # "rt" or "drop_sheet"
    D: int               # 2 or 3
    dims: tuple
    periodic: tuple
    phys: dict
    args: list
    steps: int
    seed: int
    storage: int = 0              # lbmp_storage of the domain (16-bit forms for D3Q27 only)
    arrival: float = 0.0          # seconds after the start of the run
    admitted: float = float("nan")
    done: float = float("nan")
    status: str = "queued"        # queued, running, done, failed
    obs: dict = field(default_factory=dict)

    @property
    def cells(self):
        return self.dims[0] * self.dims[1] * self.dims[2]

    def state_bytes(self):
        q = 27 if self.D == 3 else 9
        if self.storage == 0:
            return 4 * 4 * q * self.cells  # two population sets, two families, FP32
        return 4 * (4 + 2 * (q - 1)) * self.cells  # FP32 reference + 16-bit codes per set

    def latency(self):
        return self.done - self.arrival


def make_request(rid, rng, D, side, kind, steps, We, Re, rho_ratio, storage=0):
    """A request of the serving stream: the drop-on-sheet or RT set-up of the
    paper at a given size and non-dimensional parameter set (lattice units:
    U0 = 0.05, W = 5, M = 0.1 for the drop, the reading of the paper's
    impacts; sqrt(g L) = 0.04, W = 4, M = 0.02 for RT).  storage applies to
    D3Q27 requests (D2Q9 requests stay FP32)."""
    if D == 3:
        dims = (side, side, side)
    else:
        dims = (side, side, 1)
    periodic = (1, 1, 0) if D == 3 else (1, 0, 1)
    nv = dims[D - 1]
    if kind == "rt":
        L = float(side)
        g = 0.04 ** 2 / L
        phys = dict(rho_ratio=rho_ratio, nu_ratio=1.0, Re=Re, g_accel=g, L_ref=L, mobility=0.02, width=4.0,
                    We=We, U0=0.0)
        # surface tension from We with U* as the velocity scale
        phys["sigma"] = L * 0.04 ** 2 / We
        args = [nv / 2.0, 0.05 * side, 1e-4, 1.0]
    else:
        Dd = max(8.0, side / 4.0)
        phys = dict(rho_ratio=rho_ratio, nu_ratio=15.0, We=We, Re=Re, U0=0.05, L_ref=Dd, mobility=0.1,
                    width=5.0)
        args = [Dd, 0.2 * Dd, 0.05, 1e-4]
    st = storage if D == 3 else 0
    phys["storage"] = st
    return Request(rid=rid, kind=kind, D=D, dims=dims, periodic=periodic, phys=phys, args=args, steps=int(steps),
                   seed=int(rng.integers(1, 2 ** 31)), storage=st)


def request_stream(n, seed=7, sides2=(64, 128, 256, 512), sides3=(64, 96, 128, 192, 256),
                   steps_range=(2000, 20000), rate=None, storage=0):
    """Seeded stream of n requests: type RT or drop-on-sheet (p = 1/2), 2-D or
    3-D (p = 1/2) with the side drawn uniformly from sides2 / sides3, We
    log-uniform in [10, 8000], Re uniform in [100, 1000], density ratio
    log-uniform in [3, 1000], steps uniform in steps_range; Poisson arrivals
    of the given rate (requests per second; None = all at t = 0)."""
    rng = np.random.default_rng(seed)
    reqs = []
    t = 0.0
    for k in range(n):
        kind = "rt" if rng.random() < 0.5 else "drop_sheet"
        D = 3 if rng.random() < 0.5 else 2
        side = int(rng.choice(sides3 if D == 3 else sides2))
        We = float(math.exp(rng.uniform(math.log(10.0), math.log(8000.0))))
        Re = float(rng.uniform(100.0, 1000.0))
        rr = float(math.exp(rng.uniform(math.log(3.0), math.log(1000.0))))
        steps = int(rng.integers(steps_range[0], steps_range[1] + 1))
        r = make_request(k, rng, D, side, kind, steps, We, Re, rr, storage=storage)
        if rate:
            t += float(rng.exponential(1.0 / rate))
        r.arrival = t
        reqs.append(r)
    return reqs


class Server:
    """Admission by free HBM (and an optional cap on the summed state of the
    running requests, state_budget), one batch, rounds of `round_steps` steps."""

    def __init__(self, stream=None, hbm_reserve=2 << 30, round_steps=64, free_hbm=None, domain_factory=None,
                 batch=None, state_budget=None, health_every=1):
        self.stream = stream
        self.health_every = health_every  # rounds between health checks of the running requests (0: never)
        self.reserve = hbm_reserve
        self.state_budget = state_budget
        self.round_steps = round_steps
        self._free_hbm = free_hbm  # callable -> free bytes (None: torch.cuda.mem_get_info)
        self._domain = domain_factory or Domain
        self.batch = batch if batch is not None else Batch(stream=stream)
        self.running = {}  # rid -> (request, domain)

    def free_hbm(self):
        if self._free_hbm is not None:
            return self._free_hbm()
        import torch
        return torch.cuda.mem_get_info()[0]

    def _admit(self, r, now):
        d = self._domain(r.D, r.dims, r.periodic, stream=self.stream, **r.phys)
        d.init(r.kind, r.args, seed=r.seed)
        self.batch.add(d, r.steps)
        r.admitted = now
        r.status = "running"
        self.running[r.rid] = (r, d)

    def _retire(self, now):
        done = []
        for (dom, left) in self.batch.members():
            if left == 0:
                done.append(dom)
        by_handle = {d.handle.value: (r, d) for (r, d) in self.running.values()}
        for dom in done:
            r, d = by_handle[dom.handle.value]
            self.batch.remove(d)
            ob = d.observables()
            r.obs = ob.as_dict()
            r.status = "done" if ob.health == 0 else "failed"
            r.done = now
            del self.running[r.rid]
            d.close()

    def _evict_unhealthy(self, now):
        """Evict every running request whose health word is set (non-finite
        state or a speed beyond the stable range) before it uses more of
        the batch's kernel time."""
        for rid, (r, d) in list(self.running.items()):
            ob = d.observables()
            if ob.health == 0:
                continue
            self.batch.remove(d)
            r.obs = ob.as_dict()
            r.status = "failed"
            r.done = now
            del self.running[rid]
            d.close()

    def run(self, requests, clock=time.perf_counter, max_wall=None):
        """Serve the requests; returns a summary dict."""
        pending = sorted(requests, key=lambda r: r.arrival)
        t0 = clock()
        k = 0
        cell_updates = 0
        rounds = 0
        while k < len(pending) or self.running:
            now = clock() - t0
            if max_wall is not None and now > max_wall:
                break
            # continuous admission: every arrived request that fits
            while k < len(pending) and pending[k].arrival <= now:
                r = pending[k]
                over = (self.state_budget is not None and
                        self.resident_bytes() + r.state_bytes() > self.state_budget)
                if over or r.state_bytes() + self.reserve > self.free_hbm():
                    if self.running:
                        break  # wait for memory to be freed
                    r.status = "failed"  # does not fit even on an idle device
                    r.done = now
                    k += 1
                    continue
                try:
                    self._admit(r, now)
                except LbmpError:
                    r.status = "failed"
                    r.done = now
                k += 1
            if not self.running:
                if k < len(pending):
                    time.sleep(max(0.0, min(0.05, pending[k].arrival - now)))
                continue
            before = {rid: left for rid, left in ((self._rid(d), l) for d, l in self.batch.members())}
            self.batch.step(self.round_steps)
            after = {self._rid(d): l for d, l in self.batch.members()}
            for rid, l0 in before.items():
                cell_updates += (l0 - after.get(rid, 0)) * self.running[rid][0].cells
            self._retire(clock() - t0)
            rounds += 1
            if self.health_every and rounds % self.health_every == 0:
                self._evict_unhealthy(clock() - t0)
        wall = clock() - t0
        done = [r for r in pending if r.status == "done"]
        lat = np.array([r.latency() for r in done]) if done else np.array([float("nan")])
        return {"requests": len(pending), "done": len(done),
                "failed": sum(r.status == "failed" for r in pending),
                "unserved": sum(r.status in ("queued", "running") for r in pending),
                "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                "wall_s": wall, "mlups": cell_updates / wall / 1e6 if wall > 0 else 0.0,
                "cell_updates": cell_updates}

    def resident_bytes(self):
        return sum(r.state_bytes() for r, _ in self.running.values())

    def _rid(self, dom):
        for rid, (r, d) in self.running.items():
            if d.handle.value == dom.handle.value:
                return rid
        return None

    def close(self):
        for r, d in list(self.running.values()):
            try:
                self.batch.remove(d)
            except LbmpError:
                pass
            d.close()
        self.running.clear()
        self.batch.close()
