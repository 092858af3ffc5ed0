"""The z-slab split of one run (paper_0909_5603_gb300.slab) on the CPU, driven with FP64
oracle instances as the slabs.

The planner and the exchange schedule are the library's; each slab is an oracle Sim of
its extended grid (z absorbing there, no damping layer), behind the same five operations
the GPU slab offers.  After every step the owned planes of every slab, and every
particle, must equal the unsplit oracle run to 1e-12: in-process with 2 and 3 slabs
(periodic and absorbing z, Yee and the low-dispersion solver, 3 filter passes,
order-2 shape) and on two gloo ranks exchanging through torch.distributed.
"""
import json
import os
import socket

import numpy as np
import pytest

import oracle
import synth
from paper_0909_5603_gb300 import slab as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N = (8, 8, 32)
DX, DT = (1.0, 1.0, 1.0), 0.45


# ---- the planner -------------------------------------------------------------------------
def test_plan_absorbing_three_slabs():
    p = S.plan(30, 3, z_periodic=False, ghost=4)
    assert [(s.k0, s.k1) for s in p] == [(0, 10), (10, 20), (20, 30)]
    assert [(s.lo, s.nz) for s in p] == [(0, 14), (6, 18), (16, 14)]
    assert [(s.below, s.above) for s in p] == [(None, 1), (0, 2), (1, None)]
    assert [(s.own_lo, s.own_hi) for s in p] == [(0, 10), (4, 14), (4, 14)]
    assert [s.absorb_faces() for s in p] == [0x1F, 0x0F, 0x2F]
    assert p[1].ghost_range(S.BELOW) == (0, 4) and p[1].ghost_range(S.ABOVE) == (14, 18)
    assert p[1].edge_range(S.BELOW) == (4, 8) and p[1].edge_range(S.ABOVE) == (10, 14)


def test_plan_periodic_wraps_and_uneven_widths():
    p = S.plan(11, 2, z_periodic=True, ghost=4)
    assert [(s.k0, s.k1) for s in p] == [(0, 6), (6, 11)]
    assert [(s.below, s.above) for s in p] == [(1, 1), (0, 0)]
    assert p[0].lo == -4 and p[0].nz == 14 and p[1].lo == 2 and p[1].nz == 13
    assert all(s.absorb_faces() == 0x0F for s in p)


def test_plan_rejects_slabs_thinner_than_the_ghosts_and_single_slab_is_whole():
    with pytest.raises(ValueError):
        S.plan(12, 4, z_periodic=False, ghost=4)
    (only,) = S.plan(12, 1, z_periodic=True)
    assert (only.k0, only.k1, only.lo, only.nz, only.below, only.above) == (0, 12, 0, 12, None, None)
    assert S.ghost_planes(3) == 4 and S.ghost_planes(6) == 7 and S.ghost_planes(3, 8) == 11
    with pytest.raises(ValueError):
        S.SlabRun(S.plan(32, 2, True, ghost=4), {}, S.InProcess(), 8, 8, migrate_every=2)


# ---- oracle slabs ---------------------------------------------------------------------------
class OracleShard:
    """An oracle Sim of a slab's extended grid behind the slab operations."""

    def __init__(self, sim):
        self.sim = sim

    def particle_phase(self):
        self.sim.particle_phase()

    def field_phases(self):
        self.sim.filter()
        self.sim.maxwell()

    def get_planes(self, comps, k0, nk):
        return np.stack([self.sim.get_field(c)[k0:k0 + nk].copy() for c in comps])

    def put_planes(self, comps, k0, values, add):
        for c, v in zip(comps, values):
            f = self.sim.get_field(c)
            f[k0:k0 + v.shape[0]] = f[k0:k0 + v.shape[0]] + v if add else v
            self.sim.set_field(c, f)

    def extract(self, k_lo, k_hi):
        p = self.sim.get_particles()
        k = p["cell"] // (self.sim.n[0] * self.sim.n[1])
        go = (k < k_lo) | (k >= k_hi)
        self.sim.set_particles(*(p[key][~go] for key in ("cell", "off", "u", "w", "id")))
        return {key: v[go] for key, v in p.items()}

    def add(self, q):
        if q["cell"].size == 0:
            return
        p = self.sim.get_particles()
        self.sim.set_particles(*(np.concatenate([p[key], q[key]]) for key in ("cell", "off", "u", "w", "id")))


def problem(z_bc, seed=3):
    """Random particles (|u| ~ 0.5: several cross a slab face each step) and smooth
    fields on the whole grid."""
    parts = synth.random_particles(N, 3, 6000, 0.5, seed=seed)
    fields = synth.smooth_fields(N, 3, 0.05, seed=seed + 1)
    return parts, fields


def make_oracle(n, z_bc, solver, fields=None, parts=None):
    sim = oracle.Sim(3, n, (oracle.PERIODIC, oracle.PERIODIC, z_bc), DX, DT, order=2, filter_passes=3,
                     tile=(8, 8, 8), absorb_cells=0, solver=solver)
    if fields is not None:
        for c in range(6):
            sim.set_field(c, fields[c])
    if parts is not None:
        sim.set_particles(parts["cell"], parts["off"], parts["u"], parts["w"], parts["id"])
    return sim


def oracle_slab(s, z_periodic, solver, parts, fields):
    """The slab of rank s.rank cut from the whole grid's initial state."""
    nx, ny, nz = N
    sim = make_oracle((nx, ny, s.nz), oracle.ABSORBING, solver)
    planes = np.arange(s.lo, s.lo + s.nz) % nz if z_periodic else np.arange(s.lo, s.lo + s.nz)
    for c in range(6):
        sim.set_field(c, fields[c][planes])
    k = parts["cell"] // (nx * ny)
    sel = (k >= s.k0) & (k < s.k1)
    cell = parts["cell"][sel] - s.lo * nx * ny
    sim.set_particles(cell.astype(np.int32), parts["off"][sel], parts["u"][sel], parts["w"][sel], parts["id"][sel])
    return OracleShard(sim)


def whole_state(z_bc, solver, steps, parts, fields):
    w = make_oracle(N, z_bc, solver, fields, parts)
    w.step(steps)
    return {c: w.get_field(c) for c in range(9)}, w.get_particles()


def check_against_whole(slabs, owned, particles, whole_fields, whole_parts):
    """owned: {rank: {comp: planes}}, particles: {rank: dict with global cells}."""
    for c in range(9):
        got = np.concatenate([owned[s.rank][c] for s in slabs])
        ref = whole_fields[c]
        scale = max(np.abs(ref).max(), 1e-300)
        assert np.abs(got - ref).max() <= 1e-12 * scale, (c, np.abs(got - ref).max() / scale)
    cell = np.concatenate([particles[s.rank]["cell"] for s in slabs])
    ids = np.concatenate([particles[s.rank]["id"] for s in slabs])
    off = np.concatenate([particles[s.rank]["off"] for s in slabs])
    u = np.concatenate([particles[s.rank]["u"] for s in slabs])
    order = np.argsort(ids)
    ref = np.argsort(whole_parts["id"])
    assert np.array_equal(ids[order], whole_parts["id"][ref])
    assert np.array_equal(cell[order], whole_parts["cell"][ref])
    assert np.abs(off[order] - whole_parts["off"][ref]).max() <= 1e-12
    assert np.abs(u[order] - whole_parts["u"][ref]).max() <= 1e-12 * np.abs(whole_parts["u"]).max()


def slab_particles(s, shard):
    p = shard.sim.get_particles()
    p = dict(p)
    p["cell"] = p["cell"] + s.lo * N[0] * N[1]
    if s.lo < 0 or s.lo + s.nz > N[2]:
        p["cell"] = p["cell"] % (N[0] * N[1] * N[2])
    return p


@pytest.mark.parametrize("nslabs,migrate_every", [(2, 1), (3, 1), (2, 3)])
@pytest.mark.parametrize("z_bc", [oracle.PERIODIC, oracle.ABSORBING], ids=["z-periodic", "z-absorbing"])
@pytest.mark.parametrize("solver", [oracle.SOLVER_YEE, oracle.SOLVER_CK], ids=["yee", "ck"])
def test_oracle_slabs_in_process_equal_the_whole_run(nslabs, migrate_every, z_bc, solver):
    """migrate_every 3: particles stay up to 3 planes outside their slab (6 ghost planes)
    and move every third step; the last of the 12 steps is a migration step."""
    oracle.build()
    steps = 12
    parts, fields = problem(z_bc)
    zper = z_bc == oracle.PERIODIC
    slabs = S.plan(N[2], nslabs, zper, ghost=S.ghost_planes(3, migrate_every))
    shards = {s.rank: oracle_slab(s, zper, solver, parts, fields) for s in slabs}
    run = S.SlabRun(slabs, shards, S.InProcess(), N[0], N[1], migrate_every=migrate_every)
    run.step(steps)
    owned = {s.rank: {c: run.owned_field(s.rank, c) for c in range(9)} for s in slabs}
    particles = {s.rank: slab_particles(s, shards[s.rank]) for s in slabs}
    moved = sum(p["cell"].size for p in particles.values())
    assert moved > 5000  # few particles leave (absorbing z) in 12 steps
    check_against_whole(slabs, owned, particles, *whole_state(z_bc, solver, steps, parts, fields))


# ---- two gloo ranks ----------------------------------------------------------------------------
def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out, z_bc, steps):
    import sys

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch.distributed as dist

    from paper_0909_5603_gb300 import slab as SS

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        zper = z_bc == oracle.PERIODIC
        parts, fields = problem(z_bc)
        slabs = SS.plan(N[2], world, zper, ghost=SS.ghost_planes(3))
        me = slabs[rank]
        shard = oracle_slab(me, zper, oracle.SOLVER_YEE, parts, fields)
        run = SS.SlabRun(slabs, {rank: shard}, SS.Distributed(me), N[0], N[1])
        run.step(steps)
        owned = {c: run.owned_field(rank, c).tolist() for c in range(9)}
        p = slab_particles(me, shard)
        with open(os.path.join(out, f"slab{rank}.json"), "w") as f:
            json.dump({"owned": owned, "particles": {k: v.tolist() for k, v in p.items()}}, f)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("z_bc", [oracle.PERIODIC, oracle.ABSORBING], ids=["z-periodic", "z-absorbing"])
def test_oracle_slabs_on_two_gloo_ranks_equal_the_whole_run(tmp_path, z_bc):
    import torch.multiprocessing as mp

    oracle.build()
    steps = 10
    mp.spawn(_rank_main, args=(2, free_port(), str(tmp_path), z_bc, steps), nprocs=2, join=True)
    slabs = S.plan(N[2], 2, z_bc == oracle.PERIODIC, ghost=S.ghost_planes(3))
    owned, particles = {}, {}
    for s in slabs:
        d = json.load(open(tmp_path / f"slab{s.rank}.json"))
        owned[s.rank] = {int(c): np.array(v) for c, v in d["owned"].items()}
        particles[s.rank] = {k: np.array(v) for k, v in d["particles"].items()}
    parts, fields = problem(z_bc)
    check_against_whole(slabs, owned, particles, *whole_state(z_bc, oracle.SOLVER_YEE, steps, parts, fields))
