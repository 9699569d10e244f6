"""The z-slab exchange on the CPU: its plan (which populations cross a face,
from which planes, into which ghost slots), the neighbour and face pairing,
the periodic seam and the walls, and the torch.distributed transport on two
gloo ranks.  The slabs run a stand-in step with the library kernel's data
dependencies (numpy, FP64): pull streaming of two population sets with
half-way bounce-back at walls, phi summed from the pulled g on the planes
around each updated plane (mirrored beyond a wall), and a local update that
uses the pulled values and the isotropic stencil of phi.  The slabs must
reproduce the undivided domain bitwise."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2101_06769_gb300 import slab as S

C = np.array([[(a % 3) - 1, ((a // 3) % 3) - 1, (a // 9) - 1] for a in range(27)])
W1 = {0: 2.0 / 3.0, 1: 1.0 / 6.0, -1: 1.0 / 6.0}
W = np.array([W1[cx] * W1[cy] * W1[cz] for cx, cy, cz in C])


class FakeBackend:
    """A slab (or, with z0 = 0 and z1 = nz on a walled axis, the undivided
    domain) run by the stand-in step; message buffers are numpy arrays."""

    def __init__(self, dims, periodic, z0, z1, whole=False):
        self.nx, self.ny, self.nz = dims
        per = bool(periodic[2])
        if whole:
            glo = ghi = 0
        else:
            glo = 0 if (z0 == 0 and not per) else 2
            ghi = 0 if (z1 == self.nz and not per) else 2
        self.wall_lo = (not per) and z0 == 0 and glo == 0
        self.wall_hi = (not per) and z1 == self.nz and ghi == 0
        self.per_local = whole and per  # the undivided periodic domain wraps; slabs never pull across their ends
        self.nzl = (z1 - z0) + glo + ghi
        self.layout = (z0, z1, glo, ghi, self.nzl)
        self.zb, self.ze, self.zoff = glo, glo + (z1 - z0), z0 - glo
        self.sets = [np.zeros((2, 27, self.nzl, self.ny, self.nx)) for _ in range(2)]
        self.parity = 0

    def buffer(self, n):
        return np.zeros(n)

    def init(self, case, args, seed):
        rng = np.random.default_rng(seed)
        full = rng.standard_normal((2, 27, self.nz, self.ny, self.nx)) * 0.01 + W[None, :, None, None, None]
        zg = (np.arange(self.nzl) + self.zoff) % self.nz
        self.sets[0][...] = full[:, :, zg]
        self.parity = 0

    def _pulled(self, A, z):
        """pulled values of the 27 directions at local plane z: [a][y][x]"""
        out = np.empty((27, self.ny, self.nx))
        for a in range(27):
            cx, cy, cz = C[a]
            zs = z - cz
            if zs < 0 or zs >= self.nzl:
                if (zs < 0 and self.wall_lo) or (zs >= self.nzl and self.wall_hi):
                    out[a] = A[26 - a, z]  # half-way bounce-back
                    continue
                assert self.per_local, "a slab pulled across its local end"
                zs %= self.nzl
            out[a] = np.roll(np.roll(A[a, zs], cy, axis=0), cx, axis=1)
        return out

    def step(self):
        cur = self.sets[self.parity]
        new = self.sets[1 - self.parity]
        Fa, Ga = cur[0], cur[1]
        phi = {}
        for z in range(self.zb - 1, self.ze + 1):
            zz = z
            if z < 0:
                zz = 0 if self.wall_lo else z % self.nzl
            if z >= self.nzl:
                zz = self.nzl - 1 if self.wall_hi else z % self.nzl
            if zz != z and not self.per_local:
                phi[z] = None  # mirrored: filled below
                continue
            phi[z] = self._pulled(Ga, zz).sum(axis=0)
        for z in list(phi):
            if phi[z] is None:
                phi[z] = phi[0] if z < 0 else phi[self.nzl - 1]
        for z in range(self.zb, self.ze):
            pf, pg = self._pulled(Fa, z), self._pulled(Ga, z)
            lap = np.zeros((self.ny, self.nx))
            gz = np.zeros((self.ny, self.nx))
            for a in range(27):
                cx, cy, cz = C[a]
                nb = np.roll(np.roll(phi[z + cz], -cy, axis=0), -cx, axis=1)
                lap = lap + W[a] * (nb - phi[z])
                gz = gz + W[a] * cz * nb
            mean = pf.mean(axis=0)
            new[0, :, z] = pf + 0.05 * (mean[None] - pf) + 1e-3 * W[:, None, None] * lap[None] + 1e-3 * C[:, 2, None, None] * gz[None]
            new[1, :, z] = pg + 0.1 * (phi[z][None] * W[:, None, None] - pg)
        self.parity = 1 - self.parity

    def pack(self, plan, buf):
        cur = self.sets[self.parity]
        n = self.nx * self.ny
        for k, (s, a, z) in enumerate(plan):
            buf[k * n:(k + 1) * n] = cur[s, a, z].ravel()

    def unpack(self, plan, buf):
        cur = self.sets[self.parity]
        n = self.nx * self.ny
        for k, (s, a, z) in enumerate(plan):
            cur[s, a, z] = buf[k * n:(k + 1) * n].reshape(self.ny, self.nx)

    def sync(self):
        pass

    def own(self):
        cur = self.sets[self.parity]
        return cur[:, :, self.zb:self.ze]

    def close(self):
        pass


def whole_run(dims, periodic, steps, seed):
    b = FakeBackend(dims, periodic, 0, dims[2], whole=True)
    b.init(None, None, seed)
    for _ in range(steps):
        b.step()
    return b.own()


def make_slabs(dims, periodic, world, seed, transport=None):
    slabs = []
    for r in range(world):
        z0, z1 = S.split(dims[2], world, r)
        sd = S.SlabDomain(dims, periodic, r, world, transport=transport,
                          backend=FakeBackend(dims, periodic, z0, z1))
        sd.init(None, None, seed)
        slabs.append(sd)
    return slabs


@pytest.mark.parametrize("periodic_z,world", [(0, 2), (1, 2), (0, 3), (1, 3), (1, 4)])
def test_local_slabs_equal_the_whole_domain(periodic_z, world):
    dims, steps, seed = (5, 4, 13), 6, 11
    periodic = (1, 1, periodic_z)
    want = whole_run(dims, periodic, steps, seed)
    slabs = make_slabs(dims, periodic, world, seed)
    S.local_step(slabs, steps)
    got = np.concatenate([s.backend.own() for s in slabs], axis=2)
    assert np.array_equal(got, want)


def test_plan_covers_exactly_what_the_step_reads_across_a_face():
    """Dropping any block of the plan changes the result: each of the four
    blocks (f' across, g across, g level, g across from the second plane)
    is needed."""
    dims, steps, seed, periodic = (4, 4, 10), 3, 5, (1, 1, 0)
    want = whole_run(dims, periodic, steps, seed)
    for drop in range(4):
        send, recv = S.send_plan, S.recv_plan
        try:
            S.send_plan = lambda f, zb, ze: [e for k, e in enumerate(send(f, zb, ze)) if k // 9 != drop]
            S.recv_plan = lambda f, zb, ze: [e for k, e in enumerate(recv(f, zb, ze)) if k // 9 != drop]
            slabs = make_slabs(dims, periodic, 2, seed)
            S.local_step(slabs, steps)
        finally:
            S.send_plan, S.recv_plan = send, recv
        got = np.concatenate([s.backend.own() for s in slabs], axis=2)
        assert not np.array_equal(got, want), drop


def test_split_and_neighbours():
    assert [S.split(10, 3, r) for r in range(3)] == [(0, 4), (4, 7), (7, 10)]
    assert S.neighbours(0, 3, False) == (None, 1) and S.neighbours(2, 3, False) == (1, None)
    assert S.neighbours(0, 3, True) == (2, 1) and S.neighbours(2, 3, True) == (1, 0)
    assert S.neighbours(0, 2, True) == (1, 1)
    for f in (0, 1):
        assert len(S.send_plan(f, 2, 6)) == S.PLANES_PER_FACE == len(S.recv_plan(f, 2, 6))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, ws, port, periodic_z, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        dims, steps, seed = (5, 4, 12), 5, 23
        periodic = (1, 1, periodic_z)
        z0, z1 = S.split(dims[2], ws, rank)
        sd = S.SlabDomain(dims, periodic, rank, ws, transport=S.DistTransport(dist),
                          backend=FakeBackend(dims, periodic, z0, z1))
        sd.init(None, None, seed)
        sd.step(steps)
        out[rank] = sd.backend.own().copy()
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("periodic_z", [0, 1])
def test_two_gloo_ranks_equal_the_whole_domain(periodic_z):
    ws = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank, args=(ws, port, periodic_z, out), nprocs=ws, start_method="spawn", join=True)
    dims, steps, seed = (5, 4, 12), 5, 23
    want = whole_run(dims, (1, 1, periodic_z), steps, seed)
    got = np.concatenate([out[0], out[1]], axis=2)
    assert np.array_equal(got, want)
