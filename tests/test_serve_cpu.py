"""Scheduling logic of the serving loop, on the CPU with a fake backend: the
fake domains and batch stand in for the library (no GPU work), so admission
by free memory, continuous admission, retirement, eviction of a failed
request and the latency accounting are checked on the host."""
import numpy as np

from paper_2101_06769_gb300 import serve


class FakeObs:
    def __init__(self, step, health):
        self.step, self.health = step, health

    def as_dict(self):
        return {"step": self.step, "health": self.health}


class FakeHandle:
    _next = 1

    def __init__(self):
        self.value = FakeHandle._next
        FakeHandle._next += 1


class FakeDomain:
    live_bytes = 0
    poison = set()  # seeds whose runs go non-finite

    def __init__(self, D, dims, periodic, stream=None, **phys):
        self.D, self.dims = D, dims
        self.bytes = 4 * 4 * (27 if D == 3 else 9) * dims[0] * dims[1] * dims[2]
        FakeDomain.live_bytes += self.bytes
        self.handle = FakeHandle()
        self.step_count, self.seed = 0, None

    def init(self, case, args, seed=0):
        self.seed = seed

    def observables(self):
        return FakeObs(self.step_count, 1 if self.seed in FakeDomain.poison else 0)

    def close(self):
        FakeDomain.live_bytes -= self.bytes


class FakeBatch:
    def __init__(self):
        self.m = {}
        self.max_concurrent = 0

    def add(self, d, steps):
        self.m[d.handle.value] = [d, steps]
        self.max_concurrent = max(self.max_concurrent, len(self.m))

    def remove(self, d):
        del self.m[d.handle.value]

    def step(self, n):
        fin = 0
        for v in self.m.values():
            k = min(n, v[1])
            v[0].step_count += k
            v[1] -= k
            fin += v[1] == 0 and k > 0
        return fin

    def members(self):
        return [(v[0], v[1]) for v in self.m.values()]


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 0.01  # every look at the clock advances it
        return self.t


def small_stream(n, rate=None, seed=3):
    return serve.request_stream(n, seed=seed, sides2=(32, 64), sides3=(16, 24), steps_range=(50, 300), rate=rate)


def run(reqs, budget, reserve=0):
    batch = FakeBatch()
    srv = serve.Server(hbm_reserve=reserve, round_steps=32, domain_factory=FakeDomain, batch=batch,
                       free_hbm=lambda: budget - FakeDomain.live_bytes)
    out = srv.run(reqs, clock=FakeClock())
    return out, batch


def test_every_request_served_within_memory():
    reqs = small_stream(20)
    biggest = max(r.state_bytes() for r in reqs)
    out, batch = run(reqs, budget=3 * biggest)
    assert out["done"] == 20 and out["failed"] == 0 and out["unserved"] == 0
    assert 1 < batch.max_concurrent < 20  # memory limited the batch, several ran together
    assert FakeDomain.live_bytes == 0
    for r in reqs:
        assert r.obs["step"] == r.steps
        assert r.admitted >= r.arrival and r.done > r.admitted


def test_continuous_admission_with_poisson_arrivals():
    reqs = small_stream(16, rate=5.0, seed=9)
    out, batch = run(reqs, budget=1 << 40)
    assert out["done"] == 16
    lat = [r.latency() for r in reqs]
    assert out["p50_s"] == np.percentile(lat, 50) and out["p99_s"] == np.percentile(lat, 99)
    # later arrivals were admitted while earlier requests were still running
    assert batch.max_concurrent >= 2


def test_failed_request_is_evicted_and_others_continue():
    reqs = small_stream(10, seed=4)
    FakeDomain.poison = {reqs[3].seed}
    try:
        out, _ = run(reqs, budget=1 << 40)
    finally:
        FakeDomain.poison = set()
    assert out["failed"] == 1 and out["done"] == 9
    assert reqs[3].status == "failed"


def test_unhealthy_request_is_evicted_before_its_steps_run_out():
    """The health of every running request is read after each round: a
    request that blows up is removed at once (its memory freed, its batch
    time given back), not when its step count runs out."""
    reqs = [r for r in small_stream(12, seed=4) if r.steps > 3 * 32]
    bad = reqs[0]
    FakeDomain.poison = {bad.seed}
    try:
        out, batch = run(reqs, budget=1 << 40)
    finally:
        FakeDomain.poison = set()
    assert bad.status == "failed" and out["failed"] == 1 and out["done"] == len(reqs) - 1
    assert bad.obs["step"] == 32  # evicted after its first round of 32 steps
    assert FakeDomain.live_bytes == 0


def test_stream_distribution():
    reqs = serve.request_stream(256, seed=7)
    kinds = {r.kind for r in reqs}
    assert kinds == {"rt", "drop_sheet"}
    assert {r.D for r in reqs} == {2, 3}
    assert all(2000 <= r.steps <= 20000 for r in reqs)
    ratios = [r.phys["rho_ratio"] for r in reqs]
    assert 3.0 <= min(ratios) and max(ratios) <= 1000.0


def test_state_budget_limits_residency_and_16bit_doubles_it():
    """With a cap on the summed state of running requests, 16-bit storage
    (224 instead of 432 bytes per D3Q27 cell) lets more requests run at once
    (up to 1.93x; discrete request sizes pack less tightly); every request is
    still served."""
    conc = {}
    for storage in (0, 1):
        reqs = [r for r in serve.request_stream(24, seed=5, sides2=(32,), sides3=(16, 24), steps_range=(50, 300),
                                                storage=storage) if r.D == 3]
        cap = 3 * max(serve.request_stream(24, seed=5, sides2=(32,), sides3=(16, 24),
                                           steps_range=(50, 300))[k].state_bytes() for k in range(24))
        batch = FakeBatch()
        srv = serve.Server(hbm_reserve=0, round_steps=32, domain_factory=FakeDomain, batch=batch,
                           free_hbm=lambda: 1 << 40, state_budget=cap)
        out = srv.run(reqs, clock=FakeClock())
        assert out["done"] == len(reqs) and out["failed"] == 0
        conc[storage] = batch.max_concurrent
    assert conc[1] >= 1.5 * conc[0]


def test_request_state_bytes_by_storage():
    reqs = serve.request_stream(16, seed=2, sides2=(32,), sides3=(16,), steps_range=(50, 60), storage=1)
    for r in reqs:
        q = 27 if r.D == 3 else 9
        if r.D == 3:
            assert r.storage == 1 and r.phys["storage"] == 1
            assert r.state_bytes() == 4 * (4 + 2 * 26) * r.cells
        else:
            assert r.storage == 0 and r.phys["storage"] == 0
            assert r.state_bytes() == 16 * q * r.cells
