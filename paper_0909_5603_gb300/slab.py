"""Domain decomposition of one boosted-frame run along z.

Sec. 3.2 of Vay et al. notes that running in the boosted frame changes nothing in how an
already parallel PIC code is parallelised; the split used here is the usual spatial one,
along the boosted axis z (the long axis of a boosted grid, so the planes exchanged are
few).  Rank r owns the z planes [k0, k1) of the whole grid and runs them as a context of
its own, extended by `ghost` planes on each face that another slab owns.  Those faces
are absorbing without a damping layer (`absorb_faces`), so nothing wraps or reflects
there; a face of the whole grid keeps its own boundary.  One step of the whole grid is,
on every slab:

1. the particle phase (gather, push, deposit) of the slab's particles;
2. the J exchange: each ghost plane of J holds the part of a neighbour's current that this
   slab's particles deposited; it is added into the owner's plane, then every ghost
   plane of J is overwritten with its owner's now complete value;
3. the filter and Maxwell phases, on the extended slab;
4. the E/B exchange: every ghost plane of E and B is overwritten with its owner's value;
5. every `migrate_every` steps, particles that left the owned planes move to the slab
   that owns their cell.

Why that is the whole grid's step, to rounding order.  At the start of a step E and B
are exact on every local plane.  A particle moves less than one cell per step, so with
m = migrate_every it sits at most m - 1 planes beyond its slab's owned planes at the
start of a step and m at its end, and its gather and deposit windows (shape order <= 2)
reach 3 planes beyond that: inside the ghosts when ghost >= m + 3.  After step 2, J is
exact on every local plane.  Each filter pass reads one plane beyond the last and so
spoils one more plane at each face (zero is read beyond a face).  The first half-step
of B spoils one plane at the top (forward difference) and, under the low-dispersion
solver, one at the bottom (its transverse average); E spoils one more at the bottom
(backward difference); the second half of B one more at each face.  With p filter
passes the planes max(4, p + 1) or more from a face are exact, so
ghost = max(4, p + 1, m + 3) keeps every owned plane exact, and step 4 restores the
ghosts.  Only the order of the sums in J differs from the unsplit step (a ghost plane's partial
sum is added to the owner's own).  The particles' order within a tile also changes
when a slab's set is laid out again; in FP32 the block scale of the deposit depends on
which particles share a chunk, so FP32 results agree with the unsplit run to FP32
rounding, FP64 ones to FP64 rounding.

The exchange is staged through host memory with the C-ABI calls pic_get_planes_n,
pic_put_planes_n (all components of an exchange in one call), pic_extract_particles and
pic_add_particles; a transport moves the
host arrays between slabs: `InProcess` (every slab in this process, e.g. several
contexts on one GPU) or `Distributed` (one slab per rank over a torch.distributed
process group; gloo moves host tensors).  Moving particles reads the slab's particles
out and lays them out again on the device, with their cells (not the particles) copied
to the host for the order, O(particles) device work per call: migrate_every > 1 spreads
that over several steps at the price of deeper ghosts.
"""
from __future__ import annotations

import io
import pickle
from dataclasses import dataclass

import numpy as np

from . import (PIC_ABSORBING, PIC_BX, PIC_BY, PIC_BZ, PIC_EX, PIC_EY, PIC_EZ, PIC_JX, PIC_JY, PIC_JZ,
               PIC_PERIODIC, PIC_PHASE_FILTER, PIC_PHASE_MAXWELL, PIC_PHASE_PARTICLES, Simulation)

J_COMPS = (PIC_JX, PIC_JY, PIC_JZ)
EB_COMPS = (PIC_EX, PIC_EY, PIC_EZ, PIC_BX, PIC_BY, PIC_BZ)
BELOW, ABOVE = 0, 1


def ghost_planes(filter_passes: int, migrate_every: int = 1) -> int:
    """Ghost planes per inner face that keep the owned planes exact for a step."""
    return max(4, int(filter_passes) + 1, int(migrate_every) + 3)


@dataclass(frozen=True)
class Slab:
    """Rank `rank` owns planes [k0, k1) of the whole grid; its local plane 0 is plane `lo`
    of the whole grid (negative, or the planes past the end, only when z is periodic:
    they wrap), and it has `nz` local planes.  `below` / `above`: the ranks owning the
    planes just under k0 / from k1 on (None at a face of the whole grid)."""
    rank: int
    k0: int
    k1: int
    lo: int
    nz: int
    ghost: int
    below: int | None
    above: int | None

    @property
    def own_lo(self) -> int:
        return self.k0 - self.lo

    @property
    def own_hi(self) -> int:
        return self.k1 - self.lo

    def neighbours(self):
        """(side, rank) of each face that has a neighbour."""
        return [(side, r) for side, r in ((BELOW, self.below), (ABOVE, self.above)) if r is not None]

    def ghost_range(self, side):
        """Local planes of the ghosts on `side`."""
        return (0, self.ghost) if side == BELOW else (self.own_hi, self.own_hi + self.ghost)

    def edge_range(self, side):
        """Local owned planes that are the ghosts of the neighbour on `side`."""
        return (self.own_lo, self.own_lo + self.ghost) if side == BELOW else (self.own_hi - self.ghost, self.own_hi)

    def absorb_faces(self, whole_faces: int = 0x3F) -> int:
        """The slab's damping-layer faces: the whole grid's on x and y; on z only the
        faces that are the whole grid's own."""
        f = whole_faces & 0x0F
        if self.below is None:
            f |= whole_faces & 0x10
        if self.above is None:
            f |= whole_faces & 0x20
        return f


def plan(nz: int, nranks: int, z_periodic: bool, ghost: int = 4) -> list[Slab]:
    """Splits nz planes into nranks slabs of near-equal width (the first nz % nranks one
    plane wider).  Each slab owns at least `ghost` planes, so its ghosts belong to its
    immediate neighbours only."""
    if nranks < 1:
        raise ValueError("nranks must be >= 1")
    if nranks == 1:
        return [Slab(0, 0, nz, 0, nz, 0, None, None)]
    base, extra = divmod(nz, nranks)
    if base < ghost:
        raise ValueError(f"{nz} planes over {nranks} slabs: each must own at least {ghost} planes")
    out, k0 = [], 0
    for r in range(nranks):
        k1 = k0 + base + (1 if r < extra else 0)
        below = (r - 1) % nranks if (r > 0 or z_periodic) else None
        above = (r + 1) % nranks if (r < nranks - 1 or z_periodic) else None
        lo = k0 - ghost if below is not None else k0
        hi = k1 + ghost if above is not None else k1
        out.append(Slab(r, k0, k1, lo, hi - lo, ghost, below, above))
        k0 = k1
    return out


# ---- transports ----------------------------------------------------------------------
class InProcess:
    """Every slab lives in this process: messages are handed over directly."""

    def exchange(self, outbox):
        """outbox: {(src, dst, side): payload}, side the face of src it leaves by.
        Returns {dst: [(src, side, payload), ...]} in the order given."""
        inbox = {}
        for (src, dst, side), payload in outbox.items():
            inbox.setdefault(dst, []).append((src, side, payload))
        return inbox


class Distributed:
    """One slab per rank over a torch.distributed process group whose backend moves
    host (CPU) tensors, e.g. gloo.  Every exchange sends one message across each face
    that has a neighbour and receives one the same way, so sends and receives pair up;
    the tag is the face the message leaves by."""

    def __init__(self, slab: Slab, group=None):
        self.slab = slab
        self.group = group

    @staticmethod
    def _pack(payload):
        buf = io.BytesIO()
        pickle.dump(payload, buf, protocol=pickle.HIGHEST_PROTOCOL)
        return np.frombuffer(buf.getbuffer(), dtype=np.uint8).copy()

    def exchange(self, outbox):
        import torch
        import torch.distributed as dist

        s = self.slab
        sends, recvs = [], []
        for (src, dst, side), payload in outbox.items():
            assert src == s.rank
            data = torch.from_numpy(self._pack(payload))
            sends.append((dst, side, data))
        # sizes first, then the bytes
        size_out = [torch.tensor([d.numel()], dtype=torch.int64) for _, _, d in sends]
        expect = [(r, 1 - side) for side, r in s.neighbours()]  # a neighbour below sent up
        size_in = [torch.zeros(1, dtype=torch.int64) for _ in expect]
        ops = [dist.P2POp(dist.isend, t, dst, self.group, tag=side) for t, (dst, side, _) in zip(size_out, sends)]
        ops += [dist.P2POp(dist.irecv, t, src, self.group, tag=tag) for t, (src, tag) in zip(size_in, expect)]
        for req in dist.batch_isend_irecv(ops):
            req.wait()
        bufs = [torch.empty(int(t.item()), dtype=torch.uint8) for t in size_in]
        ops = [dist.P2POp(dist.isend, d, dst, self.group, tag=2 + side) for dst, side, d in sends]
        ops += [dist.P2POp(dist.irecv, b, src, self.group, tag=2 + tag) for b, (src, tag) in zip(bufs, expect)]
        for req in dist.batch_isend_irecv(ops):
            req.wait()
        inbox = {s.rank: []}
        for b, (src, tag) in zip(bufs, expect):
            inbox[s.rank].append((src, tag, pickle.loads(b.numpy().tobytes())))
        return inbox


# ---- the shard interface and its GPU form ---------------------------------------------
class GpuShard:
    """A slab run by the CUDA library (a Simulation of the slab's extended grid)."""

    def __init__(self, sim: Simulation):
        self.sim = sim
        self.plane_launches = 0  # pack / unpack launches of the plane calls (one per component)

    def particle_phase(self):
        self.sim.run_phases(PIC_PHASE_PARTICLES)

    def field_phases(self):
        self.sim.run_phases(PIC_PHASE_FILTER | PIC_PHASE_MAXWELL)

    def get_planes(self, comps, k0, nk):
        """Planes of several components, (len(comps), nk, n1, n0), in one call."""
        self.plane_launches += len(comps)
        return self.sim.get_planes_n(comps, k0, nk)

    def put_planes(self, comps, k0, values, add):
        self.plane_launches += len(comps)
        self.sim.put_planes_n(comps, k0, values, add=add)

    def extract(self, k_lo, k_hi):
        return self.sim.extract_particles(k_lo, k_hi)

    def add(self, p):
        if p["cell"].size:
            self.sim.add_particles(p["cell"], p["off"], p["u"], p["w"], p["id"] if p["id"].size else None)


# ---- the step -------------------------------------------------------------------------
class SlabRun:
    """Steps the slabs of `shards` ({rank: shard}, the ones in this process) of the split
    `slabs` (every rank's Slab) through `transport`.  nx, ny: the x-y grid."""

    def __init__(self, slabs: list[Slab], shards: dict, transport, nx: int, ny: int, migrate_every: int = 1):
        if migrate_every < 1:
            raise ValueError("migrate_every must be >= 1")
        for s in slabs:
            if len(slabs) > 1 and s.ghost < migrate_every + 3:
                raise ValueError(f"slab {s.rank}: {s.ghost} ghost planes, {migrate_every} steps between "
                                 f"migrations need {migrate_every + 3}")
        self.slabs = slabs
        self.shards = shards
        self.transport = transport
        self.plane = nx * ny
        self.nx, self.ny = nx, ny
        self.migrate_every = migrate_every
        self.steps = 0

    def _swap(self, make, take):
        outbox = {}
        for r in self.shards:
            s = self.slabs[r]
            for side, dst in s.neighbours():
                outbox[(r, dst, side)] = make(s, side)
        inbox = self.transport.exchange(outbox)
        for r in self.shards:
            for src, side, payload in inbox.get(r, []):
                # the message left src by `side`, so it reaches r by the other face
                take(self.slabs[r], 1 - side, payload)

    def _exchange_j(self):
        def make_partial(s, side):
            a, b = s.ghost_range(side)
            return self.shards[s.rank].get_planes(J_COMPS, a, b - a)

        def add_partial(s, face, arr):
            a, _ = s.edge_range(face)
            self.shards[s.rank].put_planes(J_COMPS, a, arr, True)

        self._swap(make_partial, add_partial)
        self._refresh(J_COMPS)

    def _refresh(self, comps):
        def make_edge(s, side):
            a, b = s.edge_range(side)
            return self.shards[s.rank].get_planes(comps, a, b - a)

        def put_ghost(s, face, arr):
            a, _ = s.ghost_range(face)
            self.shards[s.rank].put_planes(comps, a, arr, False)

        self._swap(make_edge, put_ghost)

    def _migrate(self):
        leaving = {}
        for r, sh in self.shards.items():
            s = self.slabs[r]
            leaving[r] = sh.extract(s.own_lo, s.own_hi)

        def make(s, side):
            p = leaving[s.rank]
            k = p["cell"] // self.plane
            sel = k < s.own_lo if side == BELOW else k >= s.own_hi
            # plane relative to the ghost region it sits in
            rel = k[sel] - (0 if side == BELOW else s.own_hi)
            return dict(rel=rel.astype(np.int32), xy=(p["cell"][sel] % self.plane).astype(np.int32), off=p["off"][sel],
                        u=p["u"][sel], w=p["w"][sel], id=p["id"][sel] if p["id"].size else np.zeros(0, np.int32))

        def take(s, face, m):
            a, _ = s.edge_range(face)
            k = a + m["rel"]
            cell = (m["xy"] + self.plane * k).astype(np.int32)
            self.shards[s.rank].add(dict(cell=cell, off=m["off"], u=m["u"], w=m["w"], id=m["id"]))

        for r in self.shards:
            s = self.slabs[r]
            p = leaving[r]
            k = p["cell"] // self.plane
            stray = ((k < s.own_lo) & (s.below is None)) | ((k >= s.own_hi) & (s.above is None))
            if np.any(stray):
                raise RuntimeError(f"slab {r}: particles outside its planes with no neighbour there")
        self._swap(make, take)

    def step(self, n: int = 1):
        for _ in range(n):
            for sh in self.shards.values():
                sh.particle_phase()
            self._exchange_j()
            for sh in self.shards.values():
                sh.field_phases()
            self._refresh(EB_COMPS)
            self.steps += 1
            if self.steps % self.migrate_every == 0:
                self._migrate()

    # -- read-out of the whole grid's owned planes (for checks)
    def owned_field(self, rank, comp):
        s = self.slabs[rank]
        return self.shards[rank].get_planes((comp,), s.own_lo, s.k1 - s.k0)[0]


# ---- the GPU split of a whole-grid context ----------------------------------------------
def split_gpu(whole: Simulation, slabs: list[Slab], ranks, **create) -> dict:
    """Slab contexts for `ranks` cut from the loaded context `whole` (its fields, its
    particles by owned plane, its ion background, step count and phase counter).
    `create` holds the Simulation keywords of the whole context (dx, dt, gamma_boost,
    order, precision, pusher, filter_passes, solver, tile, absorb_cells, ...); `bc` and
    `absorb_faces` are the whole grid's."""
    nx, ny, nzw = whole.n
    bc = tuple(create.pop("bc"))
    faces = create.pop("absorb_faces", 0x3F)
    dx, dt = create.pop("dx"), create.pop("dt")
    zper = bc[2] == PIC_PERIODIC
    fields = {c: whole.get_field(c) for c in EB_COMPS}
    parts = whole.get_particles()
    kz = parts["cell"] // (nx * ny)
    out = {}
    for r in ranks:
        s = slabs[r]
        sim = Simulation(3, (nx, ny, s.nz), (bc[0], bc[1], PIC_ABSORBING), dx, dt,
                         absorb_faces=s.absorb_faces(faces), **create)
        sel = (kz >= s.k0) & (kz < s.k1)
        cell = (parts["cell"][sel] - (s.lo * nx * ny)).astype(np.int32)
        sim.load_particles(cell, parts["off"][sel], parts["u"][sel], parts["w"][sel],
                           parts["id"][sel] if parts["id"].size else None)
        sim.adopt_slab(whole, s.lo, s.own_lo, s.own_hi)
        planes = np.arange(s.lo, s.lo + s.nz)
        if zper:
            planes %= nzw
        for c in EB_COMPS:
            sim.put_planes(c, 0, fields[c][planes], add=False)
        out[r] = sim
    return out
