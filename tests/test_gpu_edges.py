"""Degenerate and boundary cases of the particle phase on the GPU against the oracle
(FP64: cells, ids and order bit-exact, the rest within 1e-12):

* offsets at 0 and at the largest value below 1, moves that end exactly on a cell face,
  and corner wraps through every periodic face at once (+x+y+z out of the last cell,
  -x-y-z out of the first);
* particles leaving an absorbing box through edges and corners (two or three faces in
  the same step), with zero-weight and zero-momentum particles among them;
* 20,000 particles crowded into one cell next to a tile corner (one tile's population
  spans 20 chunks and spills into its neighbours);
* FP32: an offset whose update rounds to exactly 1 lands in the next cell at offset 0.
"""
import numpy as np
import pytest

import oracle
import paper_0909_5603_gb300 as pic

pytestmark = pytest.mark.gpu

FP32, FP64 = pic.PIC_PREC_FP32, pic.PIC_PREC_FP64
JS = [pic.PIC_JX, pic.PIC_JY, pic.PIC_JZ]


@pytest.fixture(scope="module", autouse=True)
def built():
    pic.build()
    oracle.build()


def relinf(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300))


def pair(n, bc, dt, order, prec=FP64):
    g = pic.Simulation(3, n, bc, (1.0, 1.0, 1.0), dt, order=order, precision=prec, tile=(8, 8, 8))
    o = oracle.Sim(3, n, bc, (1.0, 1.0, 1.0), dt, order=order, tile=(8, 8, 8))
    return g, o


def smooth(n, amp, seed):
    rng = np.random.default_rng(seed)
    z, y, x = np.meshgrid(*[np.arange(m) for m in (n[2], n[1], n[0])], indexing="ij")
    out = []
    for _ in range(6):
        k = rng.integers(1, 3, size=3)
        ph = rng.uniform(0, 2 * np.pi)
        out.append(amp * np.cos(2 * np.pi * (k[0] * x / n[0] + k[1] * y / n[1] + k[2] * z / n[2]) + ph))
    return out


def load(g, o, cell, off, u, w):
    ids = np.arange(cell.size, dtype=np.int32)
    g.load_particles(cell, off, u, w, ids)
    o.set_particles(cell, off, u, w, ids)


def compare(g, o):
    pg, po = g.get_particles(), o.get_particles()
    assert np.array_equal(pg["id"], po["id"]) and np.array_equal(pg["cell"], po["cell"])
    for k in ("off", "u", "w"):
        if po[k].size:
            assert relinf(pg[k], po[k]) <= 1e-12, k
    for c in JS:
        jo = o.get_field(c)
        if np.abs(jo).max() > 0:
            assert relinf(g.get_field(c), jo) <= 1e-12, c
    assert g.diagnostics()["n_lost"] == o.diagnostics()["n_lost"]


def cell_of(n, i, j, k):
    return i + n[0] * (j + n[1] * k)


@pytest.mark.parametrize("order", [1, 2])
def test_faces_offsets_and_corner_wraps_periodic(order):
    """No fields, so the moves are those of the loaded momenta."""
    n = (24, 24, 24)
    dt = 0.5
    g, o = pair(n, (0, 0, 0), dt, order)
    below = np.nextafter(1.0, 0.0)
    v = 0.5  # dt v / dx = 0.25 exactly (u = v gamma with gamma = 1 / sqrt(1 - v^2))
    uq = v / np.sqrt(1 - v * v)
    cells, offs, us = [], [], []
    for (i, j, k), off, u in [
        ((23, 23, 23), (below, below, below), (uq, uq, uq)),        # out through the +x+y+z corner
        ((0, 0, 0), (0.0, 0.0, 0.0), (-uq, -uq, -uq)),               # out through the -x-y-z corner
        ((7, 7, 7), (0.75, 0.75, 0.75), (uq, 0.0, 0.0)),             # ends on (or next to) the x face
        ((8, 8, 8), (0.25, 0.5, 0.0), (-uq, 0.0, 0.0)),              # ends at (or next to) offset 0
        ((3, 12, 23), (0.5, below, below), (0.0, uq, uq)),           # +y+z edge wrap
        ((23, 0, 4), (below, 0.0, 0.5), (uq, -uq, 0.0)),             # +x-y edge wrap
        ((5, 5, 5), (0.5, 0.5, 0.5), (0.0, 0.0, 0.0)),               # at rest
    ]:
        cells.append(cell_of(n, i, j, k))
        offs.append(off)
        us.append(u)
    cell = np.array(cells, np.int32)
    load(g, o, cell, np.array(offs), np.array(us), np.array([1.0, 0.5, 2.0, 1.0, 0.0, 1.0, 1.0]))
    for _ in range(3):
        g.run_phases(pic.PIC_PHASE_PARTICLES)
        o.particle_phase()
        compare(g, o)


@pytest.mark.parametrize("order", [1, 2])
def test_absorbing_edges_and_corners(order):
    n = (16, 16, 24)
    g, o = pair(n, (1, 1, 1), 0.5, order)
    rng = np.random.default_rng(5)
    uq = 0.9 / np.sqrt(1 - 0.81)  # v = 0.9: 0.45 cells a step
    cells, offs, us = [], [], []
    for (i, j, k) in [(0, 0, 0), (15, 15, 23), (0, 15, 0), (15, 0, 23), (0, 7, 23), (8, 15, 0)]:
        for _ in range(40):
            d = [(-1 if c == 0 else 1) * uq * rng.uniform(0.6, 1.0) for c in (i, j, k)]
            d = [d[0] if i in (0, 15) else 0.0, d[1] if j in (0, 15) else 0.0, d[2] if k in (0, 23) else 0.0]
            cells.append(cell_of(n, i, j, k))
            offs.append(rng.uniform(0.0, 1.0, 3))
            us.append(d)
    w = rng.uniform(0.5, 1.5, len(cells))
    w[::7] = 0.0  # zero-weight particles move and leave like the others
    load(g, o, np.array(cells, np.int32), np.array(offs), np.array(us), w)
    for _ in range(4):
        g.run_phases(pic.PIC_PHASE_PARTICLES)
        o.particle_phase()
        compare(g, o)
    assert o.diagnostics()["n_lost"] > 100


def test_crowded_cell_at_a_tile_corner():
    n = (24, 24, 24)
    g, o = pair(n, (0, 0, 0), 0.45, 2)
    rng = np.random.default_rng(9)
    m = 20000
    cell = np.full(m, cell_of(n, 7, 7, 7), np.int32)  # the corner cell of tile (0, 0, 0)
    off = rng.uniform(0.0, 1.0, (m, 3))
    u = rng.normal(0.0, 0.6, (m, 3))
    load(g, o, cell, off, u, np.full(m, 1.0 / m))
    for c, f in zip([pic.PIC_EX, pic.PIC_EY, pic.PIC_EZ, pic.PIC_BX, pic.PIC_BY, pic.PIC_BZ], smooth(n, 0.02, 4)):
        g.set_field(c, f)
        o.set_field(c, f)
    for _ in range(3):
        g.run_phases(pic.PIC_PHASE_PARTICLES)
        o.particle_phase()
        compare(g, o)
    # the crowd has spread over the eight tiles that meet at the corner
    c = g.get_particles()["cell"]
    i, j, k = c % n[0], (c // n[0]) % n[1], c // (n[0] * n[1])
    assert len(set(zip(i // 8, j // 8, k // 8))) == 8


def test_fp32_offset_rounding_to_one_moves_to_next_cell():
    """x = 1 - 2^-24 (the largest FP32 below 1) plus a displacement of 4e-8 cells (more than
    half of the 5.96e-8 spacing below 1) rounds to 1 in FP32: the particle is in the next
    cell at offset 0.  One just under half the spacing (2e-8) stays."""
    n = (24, 8, 8)
    g = pic.Simulation(3, n, (0, 0, 0), (1.0, 1.0, 1.0), 0.5, order=1, precision=FP32, tile=(8, 8, 8))
    below = float(np.nextafter(np.float32(1.0), np.float32(0.0)))
    c0 = cell_of(n, 3, 2, 2)
    g.load_particles(np.array([c0, c0], np.int32), np.array([[below, 0.5, 0.5], [below, 0.5, 0.25]]),
                     np.array([[8e-8, 0.0, 0.0], [4e-8, 0.0, 0.0]]), np.ones(2), np.array([0, 1], np.int32))
    g.run_phases(pic.PIC_PHASE_PARTICLES)
    p = g.get_particles()
    by_id = {int(i): (int(c), o) for i, c, o in zip(p["id"], p["cell"], p["off"])}
    assert by_id[0][0] == cell_of(n, 4, 2, 2) and by_id[0][1][0] == 0.0
    assert by_id[1][0] == c0 and by_id[1][1][0] == below
