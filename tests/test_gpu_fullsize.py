"""The boosted laser-wakefield stage at its full size -- 128 x 128 x 1024 cells,
33,554,432 particles, in the launch configuration the benchmark times (FP32 storage with
the FP64 gamma solve, order-2 shape, 3-pass filter, 8 x 8 x 8 tiles, absorbing faces) --
checked on sampled outputs the oracle computes one particle at a time, and by properties
that hold at any size:

* 4096 sampled particles: the oracle's gather (from the GPU's own fields) and Vay push
  give each particle's new momentum to FP32 round-off, and its move the new position.
* The particle array stays a sorted-by-tile permutation: ids unique, a subset of the
  previous ids, the missing ones exactly the particles that left through a face.
* Charge conservation: div E - F rho (F the current filter) keeps its value through full
  steps (1e-6 of the plasma's charge density) away from the absorbing layers.
"""
import numpy as np
import pytest

import oracle
import paper_0909_5603_gb300 as pic
import synth

pytestmark = pytest.mark.gpu

N = (128, 128, 1024)
GB = 13.0


@pytest.fixture(scope="module")
def stage():
    pic.build()
    oracle.build()
    w = synth.lwfa_stage(N, GB, 2)
    sim = pic.Simulation(3, w["n"], (1, 1, 1), w["dx"], w["dt"], gamma_boost=GB, order=2,
                         precision=pic.PIC_PREC_FP32, filter_passes=3, tile=(8, 8, 8))
    sim.load_lab_frame(laser=w["laser"], plasma=w["plasma"])
    assert sim.num_particles() == 2 * N[0] * N[1] * N[2]
    sim.step(2)
    return sim, w


def tile_of(cell, n, ts=(8, 8, 8)):
    i = cell % n[0]
    j = (cell // n[0]) % n[1]
    k = cell // (n[0] * n[1])
    nt = [(n[a] + ts[a] - 1) // ts[a] for a in range(3)]
    return (i // ts[0]) + nt[0] * ((j // ts[1]) + nt[1] * (k // ts[2]))


def test_sampled_particles_match_oracle_push(stage):
    sim, w = stage
    comps = [pic.PIC_EX, pic.PIC_EY, pic.PIC_EZ, pic.PIC_BX, pic.PIC_BY, pic.PIC_BZ]
    o = oracle.Sim(3, N, (1, 1, 1), w["dx"], w["dt"], order=2, tile=(8, 8, 8))
    for c in comps:
        o.set_field(c, sim.get_field(c))
    p0 = sim.get_particles()
    lost0 = sim.diagnostics()["n_lost"]
    sim.run_phases(pic.PIC_PHASE_PARTICLES)  # the fields stay as read
    p1 = sim.get_particles()
    lost1 = sim.diagnostics()["n_lost"]

    # permutation properties, bit-exact
    t1 = tile_of(p1["cell"], N)
    assert np.all(np.diff(t1) >= 0)
    ids0, ids1 = np.sort(p0["id"]), np.sort(p1["id"])
    assert np.all(np.diff(ids1) > 0)
    assert np.all(np.isin(ids1, ids0))
    assert ids0.size - ids1.size == lost1 - lost0

    # 4096 sampled particles, one by one through the oracle
    rng = np.random.default_rng(17)
    pick = rng.choice(p0["id"].size, 4096, replace=False)
    order1 = np.argsort(p1["id"])
    dx = np.array(w["dx"])
    checked = 0
    worst_u, worst_x = 0.0, 0.0
    for p in pick:
        pid = p0["id"][p]
        q = np.searchsorted(p1["id"][order1], pid)
        if q >= order1.size or p1["id"][order1[q]] != pid:
            continue  # left the box
        q = order1[q]
        E, Bf = o.gather(int(p0["cell"][p]), p0["off"][p])
        u = oracle.push_vay(p0["u"][p], E, Bf, -1.0, w["dt"])
        scale = np.abs(p0["u"][p]).max() + 1e-3
        worst_u = max(worst_u, float(np.abs(p1["u"][q] - u).max() / scale))
        # the move: x_new = x_old + dt u / gamma / dx, in cells
        c0, c1 = int(p0["cell"][p]), int(p1["cell"][q])
        cc0 = np.array([c0 % N[0], (c0 // N[0]) % N[1], c0 // (N[0] * N[1])])
        cc1 = np.array([c1 % N[0], (c1 // N[0]) % N[1], c1 // (N[0] * N[1])])
        g = np.sqrt(1.0 + np.dot(u, u))
        x_orc = cc0 + p0["off"][p] + w["dt"] * u / g / dx
        worst_x = max(worst_x, float(np.abs(cc1 + p1["off"][q] - x_orc).max()))
        checked += 1
    print(f"checked {checked}, worst momentum error {worst_u:.2e} (relative), worst position {worst_x:.2e} cells")
    assert checked > 4000
    assert worst_u < 1e-6
    assert worst_x < 1e-5


def filtered(rho, passes=3):
    """The current filter's 1-2-1 passes along x, y and z applied to rho (wrapping: only
    the interior is used)."""
    f = rho.copy()
    for _ in range(passes):
        for ax in (2, 1, 0):
            f = 0.25 * np.roll(f, 1, ax) + 0.5 * f + 0.25 * np.roll(f, -1, ax)
    return f


def test_charge_conservation_full_size(stage):
    """The filter is a convolution, which commutes with the differences: E advanced with
    the filtered current keeps div E - F rho constant, F the same three 1-2-1 passes on
    the nodes.  Checked on the nodes away from the absorbing layers (16 cells, damped
    fields, outflow) and the filter's reach, in units of the plasma's charge density
    gamma_b n0 (the net density, ions included, is nearly zero)."""
    sim, w = stage
    r0 = sim.get_field(pic.PIC_DIVE) - filtered(sim.get_field(pic.PIC_RHO))
    sim.step(3)
    r1 = sim.get_field(pic.PIC_DIVE) - filtered(sim.get_field(pic.PIC_RHO))
    inner = (slice(18, N[2] - 18), slice(18, N[1] - 18), slice(18, N[0] - 18))
    scale = GB * w["plasma"][0]
    err = float(np.abs(r1[inner] - r0[inner]).max() / scale)
    print(f"div E - rho change after 3 steps: {err:.2e} of gamma_b n0")
    assert err < 1e-6
