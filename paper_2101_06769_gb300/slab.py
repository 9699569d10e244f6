"""Z-slab decomposition of one D3Q27 domain over several GPUs (one rank per
GPU), on top of the library's slab handles (include/lbmp.h, lbmp_create_slab).

Each rank holds the global planes [z0, z1) of the domain and, on every face
that borders another slab, two ghost planes.  The step is pull streaming: a
cell at plane z reads the post-collision populations that the previous step
left at z - c.  So after every step the populations that cross a face must be
copied from the neighbour's boundary planes into this slab's ghost planes:

* the slab's first own plane zb pulls its upward-moving populations (c_z =
  +1) of f' and g from the ghost plane zb - 1;
* phi on the ghost plane zb - 1 (the isotropic stencil of plane zb needs it)
  is formed from the g that plane zb - 1 pulls: its level populations (c_z =
  0) from zb - 1 itself, its upward-moving ones from zb - 2, its
  downward-moving ones from zb (an own plane);

and the same, mirrored, above the slab.  A face's message is therefore four
blocks of nine planes: f' moving across the face and g moving across it from
the boundary plane, g level on the boundary plane, and g moving across it
from the plane behind (36 planes of nx ny floats; `send_plan` / `recv_plan`
below, the one place where this plan is written down).  Faces on the
domain's walls keep the wall and exchange nothing.  With the ghosts refilled
every step the slabs reproduce the undivided domain bitwise.

The transport moves the messages: `DistTransport` over torch.distributed
(NCCL send/recv between GPUs, or gloo with host staging), `local_step` for
several slabs in one process (device copies).  Mass, kinetic energy and
max |u| are reduced across ranks; the Laplace probes and RT tips are left to
the caller (a slab returns NaN for them).
"""
import ctypes as C

import numpy as np

from .lbmp import D3Q27, Grid, Obs, _check, load, make_params

# canonical directions a = (cx+1) + 3(cy+1) + 9(cz+1), grouped by c_z
DOWN = tuple(range(0, 9))     # c_z = -1
LEVEL = tuple(range(9, 18))   # c_z = 0
UP = tuple(range(18, 27))     # c_z = +1
F_SET, G_SET = 0, 1
PLANES_PER_FACE = 36


def split(nz, world, rank):
    """planes [z0, z1) of `rank` when nz planes are split as evenly as possible"""
    base, extra = divmod(nz, world)
    z0 = rank * base + min(rank, extra)
    return z0, z0 + base + (1 if rank < extra else 0)


def neighbours(rank, world, periodic_z):
    """ranks of the slabs below and above (None where the domain's wall is)"""
    lower = rank - 1 if rank > 0 else (world - 1 if periodic_z else None)
    upper = rank + 1 if rank < world - 1 else (0 if periodic_z else None)
    return lower, upper


def send_plan(face, zb, ze):
    """(set, direction, local plane) of the populations that leave through
    face 0 (below plane zb) or 1 (above plane ze - 1), in message order"""
    if face == 0:
        z1, z2, across = zb, zb + 1, DOWN
    else:
        z1, z2, across = ze - 1, ze - 2, UP
    return ([(F_SET, a, z1) for a in across] + [(G_SET, a, z1) for a in across] +
            [(G_SET, a, z1) for a in LEVEL] + [(G_SET, a, z2) for a in across])


def recv_plan(face, zb, ze):
    """the ghost slots that the neighbour's message through this face fills,
    in the order of that message (its send_plan of the opposite face)"""
    if face == 0:
        z1, z2, across = zb - 1, zb - 2, UP
    else:
        z1, z2, across = ze, ze + 1, DOWN
    return ([(F_SET, a, z1) for a in across] + [(G_SET, a, z1) for a in across] +
            [(G_SET, a, z1) for a in LEVEL] + [(G_SET, a, z2) for a in across])


def _plan_array(plan):
    flat = np.asarray(plan, dtype=np.int32).ravel()
    return flat, flat.ctypes.data_as(C.POINTER(C.c_int))


class LibBackend:
    """A slab handle of the CUDA library; message buffers are device tensors."""

    def __init__(self, dims, periodic, z0, z1, stream=None, allocator=None, **phys):
        import torch
        self.torch = torch
        L = load()
        g = Grid(dims[0], dims[1], dims[2], (C.c_int * 3)(*[int(v) for v in periodic]))
        h = C.c_void_p()
        self._allocator = allocator
        _check(L.lbmp_create_slab(C.byref(g), int(z0), int(z1), D3Q27, C.byref(make_params(**phys)),
                                  C.c_void_p(stream) if stream else None,
                                  C.byref(allocator) if allocator is not None else None, C.byref(h)))
        self.h = h
        self.stream = stream
        self.nxy = dims[0] * dims[1]
        lay = (C.c_int * 5)()
        _check(L.lbmp_slab_layout(h, lay))
        self.layout = tuple(lay)
        self.nz_local = lay[4]
        self.N = self.nxy * self.nz_local

    def buffer(self, nfloats):
        return self.torch.empty(nfloats, dtype=self.torch.float32, device="cuda")

    def init(self, case, args, seed):
        from .lbmp import CASE
        cid = CASE[case] if isinstance(case, str) else int(case)
        a = (C.c_double * max(1, len(args)))(*args)
        _check(load().lbmp_init(self.h, cid, a, len(args), int(seed)))

    def step(self):
        _check(load().lbmp_step(self.h, 1))

    def pack(self, plan, buf):
        flat, ptr = _plan_array(plan)
        _check(load().lbmp_pack_planes(self.h, ptr, len(plan), C.c_void_p(buf.data_ptr())))

    def unpack(self, plan, buf):
        flat, ptr = _plan_array(plan)
        _check(load().lbmp_unpack_planes(self.h, ptr, len(plan), C.c_void_p(buf.data_ptr())))

    def sync(self):
        _check(load().lbmp_sync(self.h))

    def get_state(self):
        nx = self.nxy  # flattened planes: [a][z][xy]
        f = np.zeros((27, self.nz_local, nx))
        g = np.zeros((27, self.nz_local, nx))
        _check(load().lbmp_get_state(self.h, f.ctypes.data, g.ctypes.data, None))
        return f, g

    def observables(self):
        o = Obs()
        rc = load().lbmp_observables(self.h, C.byref(o))
        if rc not in (0, -5):
            _check(rc)
        return o

    def close(self):
        if self.h:
            load().lbmp_destroy(self.h)
            self.h = None


class SlabDomain:
    """Rank `rank` of `world` slabs of a D3Q27 domain of `dims` cells
    (periodic x and y; z periodic or walled).  `backend` is LibBackend (the
    default) or any object with the same methods."""

    def __init__(self, dims, periodic, rank, world, transport=None, backend=None, **kw):
        self.dims = tuple(int(v) for v in dims)
        self.rank, self.world = rank, world
        self.z0, self.z1 = split(self.dims[2], world, rank)
        self.lower, self.upper = neighbours(rank, world, bool(periodic[2]))
        self.peer = {0: self.lower, 1: self.upper}
        self.backend = backend if backend is not None else LibBackend(self.dims, periodic, self.z0, self.z1, **kw)
        z0, z1, glo, ghi, _ = self.backend.layout
        assert (z0, z1) == (self.z0, self.z1)
        self.zb, self.ze = glo, glo + (z1 - z0)
        self.faces = [f for f in (0, 1) if self.peer[f] is not None]
        n = PLANES_PER_FACE * self.dims[0] * self.dims[1]
        self.send = {f: self.backend.buffer(n) for f in self.faces}
        self.recv = {f: self.backend.buffer(n) for f in self.faces}
        self.splan = {f: send_plan(f, self.zb, self.ze) for f in self.faces}
        self.rplan = {f: recv_plan(f, self.zb, self.ze) for f in self.faces}
        self.transport = transport

    def init(self, case, args, seed=0):
        self.backend.init(case, args, seed)

    def advance(self):
        self.backend.step()

    def pack(self):
        for f in self.faces:
            self.backend.pack(self.splan[f], self.send[f])
        self.backend.sync()

    def unpack(self):
        for f in self.faces:
            self.backend.unpack(self.rplan[f], self.recv[f])

    def step(self, n=1):
        """n coupled steps with the ghost exchange after each (all ranks call it)"""
        for _ in range(n):
            self.advance()
            self.pack()
            self.transport.exchange(self)
            self.unpack()

    def own_state(self):
        """f', g of the slab's own planes ([a][z][y][x], global planes z0..z1)"""
        f, g = self.backend.get_state()
        nx, ny = self.dims[0], self.dims[1]
        sl = slice(self.zb, self.ze)
        return (f[:, sl].reshape(27, -1, ny, nx), g[:, sl].reshape(27, -1, ny, nx))

    def observables(self):
        """mass, kinetic energy, max |u| and health: of the whole domain when
        the slab has a transport (reduced across ranks), else of this slab's
        own planes"""
        o = self.backend.observables()
        vals = np.array([o.mass, o.kinetic_energy, o.max_u, float(o.health)])
        if self.transport is not None:
            vals = self.transport.reduce(vals)
        return {"mass": vals[0], "kinetic_energy": vals[1], "max_u": vals[2], "health": int(vals[3])}

    def close(self):
        self.backend.close()


class DistTransport:
    """Moves the face messages with torch.distributed point-to-point calls.
    Messages are posted with sends in face order (0, 1) and receives in face
    order (1, 0), so that with two slabs on a periodic axis (both neighbours
    are the same rank) the k-th message of one rank to the other is the k-th
    that the other receives from it, as NCCL matches them.  With the gloo
    backend the device buffers are staged through host memory."""

    def __init__(self, dist):
        self.dist = dist
        self.host = dist.get_backend() == "gloo"

    def exchange(self, slab):
        import torch
        d = self.dist

        def tensor(b):  # host arrays travel as tensors sharing their memory
            return torch.from_numpy(b) if isinstance(b, np.ndarray) else b

        sbuf = {f: tensor(b) for f, b in slab.send.items()}
        rbuf = {f: tensor(b) for f, b in slab.recv.items()}
        send = {f: (b.cpu() if self.host and b.is_cuda else b) for f, b in sbuf.items()}
        recv = {f: (torch.empty_like(b, device="cpu") if self.host and b.is_cuda else b) for f, b in rbuf.items()}
        ops = [d.P2POp(d.isend, send[f], slab.peer[f], tag=f) for f in (0, 1) if f in send]
        ops += [d.P2POp(d.irecv, recv[f], slab.peer[f], tag=1 - f) for f in (1, 0) if f in recv]
        for r in d.batch_isend_irecv(ops):
            r.wait()
        for f, b in rbuf.items():
            if recv[f] is not b:
                b.copy_(recv[f])

    def reduce(self, vals):
        import torch
        t = torch.tensor(vals[:2], dtype=torch.float64)
        m = torch.tensor(vals[2:], dtype=torch.float64)
        if self.dist.get_backend() == "nccl":
            t, m = t.cuda(), m.cuda()
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM)
        self.dist.all_reduce(m, op=self.dist.ReduceOp.MAX)
        return np.concatenate([t.cpu().numpy(), m.cpu().numpy()])


def local_step(slabs, n=1):
    """Advance slabs of one domain that live in this process (for instance
    on one GPU) n steps: every slab steps, packs, the messages are copied
    to the neighbours' receive buffers, every slab unpacks."""
    for _ in range(n):
        for s in slabs:
            s.advance()
        for s in slabs:
            s.pack()
        for s in slabs:
            for f in s.faces:
                # the message through face f lands on the neighbour's opposite face
                slabs[s.peer[f]].recv[1 - f][...] = s.send[f]
        for s in slabs:
            s.unpack()
