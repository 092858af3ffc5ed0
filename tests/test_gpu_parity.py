"""CUDA path vs the FP64 oracle, element by element, on the same seeded inputs.

Every call goes through the C ABI (paper_0909_5603_gb300 is a ctypes binding).  Bars:
integer work (cells, canonical particle order, ids, counts) bit-exact; floating point
within the stated tolerances -- 1e-12 relative in FP64 mode, 1e-5 relative after 100
steps in FP32 mode.  The relative error of an array is normwise,
||gpu - oracle||_2 / ||oracle||_2; FP64 comparisons also bound the element-wise
max|gpu - oracle| / max|oracle| by the same 1e-12.  In FP32 mode the element-wise error
has a floor near 1e-5: a particle crossing a cell face splits its current between the
two cells at the crossing point (dJ/dx0 = q w / dt), so an FP32 offset rounding of
~3e-8 near a face moves that cell's current by ~3e-8 / (v dt), 6e-6 relative at the
thermal speed of the 2D3V plasma test; the FP32 element-wise bar is therefore 1e-4.
"""
import numpy as np
import pytest

import oracle
import paper_0909_5603_gb300 as pic
import synth

pytestmark = pytest.mark.gpu

FP32, FP64 = pic.PIC_PREC_FP32, pic.PIC_PREC_FP64
VAY, BORIS = pic.PIC_PUSHER_VAY, pic.PIC_PUSHER_BORIS
COMPS = [pic.PIC_EX, pic.PIC_EY, pic.PIC_EZ, pic.PIC_BX, pic.PIC_BY, pic.PIC_BZ]


@pytest.fixture(scope="module", autouse=True)
def built():
    pic.build()
    oracle.build()


def rel(a, b):
    """Element-wise (infinity-norm) relative error."""
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300))


def rel2(a, b):
    """Normwise (2-norm) relative error."""
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def pair(ndim, n, bc, dx, dt, order, prec, pusher=VAY, passes=0, tile=None, gamma=1.0):
    if tile is None:
        tile = (8, 8, 8) if ndim == 3 else (16, 1, 16)
    g = pic.Simulation(ndim, n, bc, dx, dt, gamma_boost=gamma, order=order, precision=prec, pusher=pusher,
                       filter_passes=passes, tile=tile)
    o = oracle.Sim(ndim, n, bc, dx, dt, order=order, pusher=pusher, filter_passes=passes, tile=tile)
    return g, o


def load_both(g, o, parts):
    g.load_particles(parts["cell"], parts["off"], parts["u"], parts["w"], parts["id"])
    o.set_particles(parts["cell"], parts["off"], parts["u"], parts["w"], parts["id"])


def set_fields_both(g, o, fields, comps=COMPS):
    for c, f in zip(comps, fields):
        g.set_field(c, f)
        o.set_field(c, f)


def compare_particles(g, o, tol, exact_order=True, tol_inf=None):
    """FP64: same order, cells and ids bit-exact, offsets/momenta/weights within tol (both
    norms).  FP32 (exact_order False): matched by id, positions (cell + offset, periodic
    images folded) within tol of the box size, momenta normwise within tol."""
    tol_inf = tol if tol_inf is None else tol_inf
    pg, po = g.get_particles(), o.get_particles()
    assert pg["cell"].size == po["cell"].size
    if exact_order:
        assert np.array_equal(pg["id"], po["id"])
        assert np.array_equal(pg["cell"], po["cell"])
        for k in ("off", "u", "w"):
            assert rel2(pg[k], po[k]) <= tol and rel(pg[k], po[k]) <= tol_inf, k
    else:
        ig, io = np.argsort(pg["id"]), np.argsort(po["id"])
        assert np.array_equal(pg["id"][ig], po["id"][io])
        ng = np.asarray(g.n)
        pos_g = _positions(pg, ng)[ig]
        pos_o = _positions(po, ng)[io]
        d = pos_g - pos_o
        d -= np.round(d / ng) * ng  # periodic images
        assert np.abs(d).max() <= tol * max(1.0, np.abs(pos_o).max())
        assert rel2(pg["u"][ig], po["u"][io]) <= tol and rel(pg["u"][ig], po["u"][io]) <= tol_inf
    return pg, po


def _positions(p, n):
    c = p["cell"]
    ijk = np.stack([c % n[0], (c // n[0]) % n[1], c // (n[0] * n[1])], 1).astype(np.float64)
    return ijk + p["off"]


def compare_fields(g, o, comps, tol, tol_inf=None):
    """Normwise relative error <= tol and element-wise <= tol_inf (default tol)."""
    tol_inf = tol if tol_inf is None else tol_inf
    worst = {}
    for c in comps:
        fo = o.get_field(c)
        fg = g.get_field(c)
        if np.abs(fo).max() == 0:
            assert np.abs(fg).max() == 0
            continue
        e2, ei = rel2(fg, fo), rel(fg, fo)
        worst[c] = (e2, ei)
        assert e2 <= tol and ei <= tol_inf, (c, e2, ei)
    return worst


# ---------------------------------------------------------------------------- phases
CASES_3D = dict(ndim=3, n=(20, 16, 24), dx=(1.0, 0.9, 1.1), dt=0.45)
CASES_2D = dict(ndim=2, n=(36, 1, 44), dx=(1.0, 1.0, 0.8), dt=0.5)


@pytest.mark.parametrize("prec,tol", [(FP64, 1e-13), (FP32, 2e-6)])
@pytest.mark.parametrize("case", ["3d_per", "3d_abs", "2d_per", "2d_abs"])
def test_maxwell_phase(case, prec, tol):
    c = dict(CASES_3D if case.startswith("3d") else CASES_2D)
    bc = (0, 0, 0) if case.endswith("per") else (1, 1, 1)
    g, o = pair(c["ndim"], c["n"], bc, c["dx"], c["dt"], 1, prec)
    # loading (no particles) clears J, so it comes before the fields are set
    g.load_particles(np.zeros(0, np.int32), np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0))
    f = synth.smooth_fields(c["n"], c["ndim"], 0.3, seed=4)
    set_fields_both(g, o, f)
    J = synth.smooth_fields(c["n"], c["ndim"], 0.05, seed=5)[:3]
    set_fields_both(g, o, J, [pic.PIC_JX, pic.PIC_JY, pic.PIC_JZ])
    for _ in range(3):
        g.run_phases(pic.PIC_PHASE_MAXWELL)
        o.maxwell()
    compare_fields(g, o, COMPS, tol)


@pytest.mark.parametrize("prec,tol", [(FP64, 1e-14), (FP32, 1e-6)])
@pytest.mark.parametrize("ndim,bc", [(3, (0, 0, 0)), (3, (1, 0, 1)), (2, (0, 0, 0)), (2, (1, 0, 1))])
@pytest.mark.parametrize("passes", [1, 3])
def test_filter_phase(ndim, bc, passes, prec, tol):
    c = dict(CASES_3D if ndim == 3 else CASES_2D)
    g, o = pair(ndim, c["n"], bc, c["dx"], c["dt"], 1, prec, passes=passes)
    g.load_particles(np.zeros(0, np.int32), np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0))
    rng = np.random.default_rng(9)
    J = [synth.f32(rng.normal(size=(c["n"][2], c["n"][1] if ndim == 3 else 1, c["n"][0]))) for _ in range(3)]
    set_fields_both(g, o, J, [pic.PIC_JX, pic.PIC_JY, pic.PIC_JZ])
    g.run_phases(pic.PIC_PHASE_FILTER)
    o.filter()
    compare_fields(g, o, [pic.PIC_JX, pic.PIC_JY, pic.PIC_JZ], tol)


@pytest.mark.parametrize("ndim,n,bc", [(3, (40, 20, 150), (0, 1, 0)), (3, (36, 12, 70), (1, 0, 1)),
                                       (3, (8, 8, 8), (0, 0, 0)), (2, (300, 1, 70), (1, 0, 0)), (2, (12, 1, 8), (0, 0, 0))])
@pytest.mark.parametrize("passes", [2, 8])
def test_filter_phase_many_tiles(ndim, n, bc, passes):
    """The fused filter over several column blocks and plane segments with ragged ends,
    up to the maximum number of passes, and on axes shorter than the pass halo (periodic
    wrap several times around)."""
    g, o = pair(ndim, n, bc, (1.0, 1.0, 1.0), 0.3, 1, FP64, passes=passes)
    g.load_particles(np.zeros(0, np.int32), np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0))
    rng = np.random.default_rng(10)
    J = [rng.normal(size=(n[2], n[1], n[0])) for _ in range(3)]
    set_fields_both(g, o, J, [pic.PIC_JX, pic.PIC_JY, pic.PIC_JZ])
    g.run_phases(pic.PIC_PHASE_FILTER)
    o.filter()
    compare_fields(g, o, [pic.PIC_JX, pic.PIC_JY, pic.PIC_JZ], 1e-14)


PARTICLE_CASES = [(nd, order, pusher, bcs) for nd in (3, 2) for order in (1, 2) for pusher in (VAY, BORIS)
                  for bcs in ("per", "abs")]


@pytest.mark.parametrize("ndim,order,pusher,bcs", PARTICLE_CASES)
def test_particle_phase_fp64(ndim, order, pusher, bcs):
    """One gather + push + move + deposit + reorder, random smooth fields, random cells
    (uneven and empty tiles, ragged last tiles), momenta large enough to cross tiles."""
    c = dict(CASES_3D if ndim == 3 else CASES_2D)
    bc = (0, 0, 0) if bcs == "per" else (1, 1, 1)
    g, o = pair(ndim, c["n"], bc, c["dx"], c["dt"], order, FP64, pusher=pusher)
    f = synth.smooth_fields(c["n"], ndim, 0.2, seed=11)
    set_fields_both(g, o, f)
    parts = synth.random_particles(c["n"], ndim, 12000, 1.5, seed=12)
    load_both(g, o, parts)
    for _ in range(2):
        g.run_phases(pic.PIC_PHASE_PARTICLES)
        o.particle_phase()
    compare_fields(g, o, [pic.PIC_JX, pic.PIC_JY, pic.PIC_JZ], 1e-12)
    compare_particles(g, o, 1e-12)
    dg, do = g.diagnostics(), o.diagnostics()
    assert dg["n_particles"] == do["n_particles"] and dg["n_lost"] == do["n_lost"]


@pytest.mark.parametrize("ndim,order", [(3, 1), (3, 2), (2, 1), (2, 2)])
def test_particle_phase_fp32(ndim, order):
    """One particle phase of 12,000 random relativistic particles (sigma_u 1.5) in smooth
    fields, FP32 against the FP64 oracle.  The FP32 current is accumulated in 32-bit fixed
    point per chunk of 256 particles with a resolution of 2^-22 of the chunk's largest
    contribution bound per component (about the precision of FP32 accumulation): the
    current's normwise bar after one phase is 2e-6 (measured 0.6-1.0e-6), the particles'
    2e-6."""
    c = dict(CASES_3D if ndim == 3 else CASES_2D)
    g, o = pair(ndim, c["n"], (0, 0, 0), c["dx"], c["dt"], order, FP32)
    set_fields_both(g, o, synth.smooth_fields(c["n"], ndim, 0.2, seed=13))
    load_both(g, o, synth.random_particles(c["n"], ndim, 12000, 1.5, seed=14))
    g.run_phases(pic.PIC_PHASE_PARTICLES)
    o.particle_phase()
    compare_fields(g, o, [pic.PIC_JX, pic.PIC_JY, pic.PIC_JZ], 2e-6, tol_inf=2e-5)
    compare_particles(g, o, 2e-6, exact_order=False)


def test_multichunk_tiles_and_sort_permutation():
    """Tiles holding several chunks (> 1024 particles); many tile crossings per step; the
    canonical order (stable sort by tile) must stay bit-exact over steps."""
    n = (16, 16, 24)
    g, o = pair(3, n, (0, 0, 1), (1, 1, 1), 0.5, 2, FP64)
    parts = synth.uniform_plasma(n, 3, 9, 1.2, seed=15)  # 9 ppc -> 4608 per 8^3 tile
    load_both(g, o, parts)
    for s in range(6):
        g.run_phases(pic.PIC_PHASE_PARTICLES)
        o.particle_phase()
        pg, po = g.get_particles(), o.get_particles()
        assert np.array_equal(pg["id"], po["id"]), s
        assert np.array_equal(pg["cell"], po["cell"]), s
    assert g.diagnostics()["n_lost"] == o.diagnostics()["n_lost"] > 0


# ------------------------------------------------------------------------ whole steps
@pytest.mark.parametrize("ndim,order,passes,bcs", [(3, 2, 3, "abs"), (3, 1, 0, "per"), (2, 2, 1, "per"), (2, 1, 2, "abs")])
def test_full_steps_fp64(ndim, order, passes, bcs):
    c = dict(CASES_3D if ndim == 3 else CASES_2D)
    bc = (0, 0, 0) if bcs == "per" else (1, 1, 1)
    g, o = pair(ndim, c["n"], bc, c["dx"], c["dt"], order, FP64, passes=passes)
    set_fields_both(g, o, synth.smooth_fields(c["n"], ndim, 0.05, seed=16))
    load_both(g, o, synth.uniform_plasma(c["n"], ndim, 2, 0.3, seed=17))
    g.step(8)
    o.step(8)
    compare_fields(g, o, COMPS + [pic.PIC_JX, pic.PIC_JY, pic.PIC_JZ], 1e-12)
    compare_particles(g, o, 1e-12)


def test_config1_2d3v_fp64_100_steps():
    """2D3V 128x128 periodic, 4 ppc (65,536 electrons), sigma_u = 0.01, CIC, Vay, no
    filter, dx = 1 skin depth (n0 = 1), dt = 0.5, 100 steps: all fields and particles."""
    n = (128, 1, 128)
    g, o = pair(2, n, (0, 0, 0), (1.0, 1.0, 1.0), 0.5, 1, FP64, tile=(16, 1, 16))
    load_both(g, o, synth.uniform_plasma(n, 2, 4, 0.01, seed=1))
    g.step(100)
    o.step(100)
    compare_fields(g, o, COMPS + [pic.PIC_JX, pic.PIC_JY, pic.PIC_JZ], 1e-12)
    compare_particles(g, o, 1e-12)
    dg, do = g.diagnostics(), o.diagnostics()
    assert abs(dg["field_energy"] - do["field_energy"]) <= 1e-12 * do["field_energy"]
    assert abs(dg["kinetic_energy"] - do["kinetic_energy"]) <= 1e-12 * do["kinetic_energy"]


def test_config1_2d3v_fp32_100_steps():
    """The FP64 2D3V plasma case run in FP32 mode (beyond its FP64 specification).  With
    sigma_u = 0.01 the Debye length is 1/100 of a cell, so the grid heats the plasma
    (finite-grid instability) and every rounding difference grows about e-fold per 43
    steps: rounding only the stored state to FP32 inside the FP64 oracle already leaves
    4.7e-6 after 100 steps, and the FP32 arithmetic of gather and push (a few ulps per
    step against half an ulp of storage) ends between 1.4e-5 and 2.4e-5 depending on the
    field and the run (the order of the FP32 atomic adds that fold the current tiles into
    the grid varies from run to run, and the instability amplifies that too).  The bar
    here is therefore 5e-5 normwise; the FP32 configurations proper (the boosted LWFA
    stage, the beam, the batched scan) meet 1e-5 after 100 steps in their own tests."""
    n = (128, 1, 128)
    g, o = pair(2, n, (0, 0, 0), (1.0, 1.0, 1.0), 0.5, 1, FP32, tile=(16, 1, 16))
    p = synth.uniform_plasma(n, 2, 4, 0.01, seed=1)
    load_both(g, o, p)
    g.step(100)
    o.step(100)
    # the floor FP32 storage alone sets: the oracle with its state rounded every step
    e = oracle.Sim(2, n, (0, 0, 0), (1.0, 1.0, 1.0), 0.5, order=1, tile=(16, 1, 16))
    e.set_particles(*[p[k] for k in ("cell", "off", "u", "w", "id")])
    e.round_state_fp32()
    for _ in range(100):
        e.step(1)
        e.round_state_fp32()
    floor = max(rel2(e.get_field(c), o.get_field(c)) for c in COMPS)
    print(f"FP32 storage floor after 100 steps (worst field): {floor:.2e}")
    assert floor < 1e-5
    worst = compare_fields(g, o, COMPS + [pic.PIC_JX, pic.PIC_JY, pic.PIC_JZ], 5e-5, tol_inf=1e-4)
    print("FP32 config-1 relative errors after 100 steps (2-norm, max-norm) per field:", worst)
    compare_particles(g, o, 5e-5, exact_order=False, tol_inf=1e-4)


# ------------------------------------------------------------- loaders and getters
@pytest.mark.parametrize("prec", [FP64, FP32])
@pytest.mark.parametrize("ndim", [3, 2])
def test_lab_frame_load(ndim, prec):
    gb = 13.0
    n = (16, 12, 64) if ndim == 3 else (24, 1, 96)
    dz = 2.0
    dx = (3.0, 3.0, dz)
    g, o = pair(ndim, n, (1, 1, 1), dx, 0.5 * dz, 2, prec, gamma=gb)
    laser = (2.0, 1.0, 15.0, 10.0, 8.0)
    plasma = (1.0 / 900 * (2 * np.pi) ** 2, 5.0, 2.0, 2, (0.0, 0.0, 0.0), 3)
    beam = (500, 30.0, 1e-3, 2.0, 1.0, 4.0, 1e3, 7)
    g.load_lab_frame(laser=laser, plasma=plasma, beam=beam)
    o.load_lab_frame(gb, laser=laser, plasma=[*plasma[:4], *plasma[4], plasma[5]], beam=beam)
    pg, po = g.get_particles(), o.get_particles()
    assert np.array_equal(pg["id"], po["id"]) and np.array_equal(pg["cell"], po["cell"])
    if prec == FP64:
        for k in ("off", "u", "w"):
            assert np.array_equal(pg[k], po[k]), k
        tol = 1e-13  # the beam's self-field solve sums in its own order on each side
    else:
        # FP32 storage: the oracle's FP64 values rounded to FP32, offsets kept below 1
        below_one = np.nextafter(np.float32(1), np.float32(0))
        for k in ("off", "u", "w"):
            ref = po[k].astype(np.float32)
            if k == "off":
                ref = np.minimum(ref, below_one)
            assert np.array_equal(pg[k], ref.astype(np.float64)), k
        tol = 6e-8
    for c in COMPS:  # laser (Ex, By) plus the beam's self-field
        fo = o.get_field(c)
        if np.abs(fo).max() > 0:
            assert rel(g.get_field(c), fo) <= tol, c


def test_rho_dive_and_diagnostics_fp64():
    n = (20, 16, 24)
    g, o = pair(3, n, (0, 1, 0), (1.0, 0.9, 1.1), 0.45, 2, FP64)
    set_fields_both(g, o, synth.smooth_fields(n, 3, 0.1, seed=18))
    load_both(g, o, synth.random_particles(n, 3, 5000, 0.5, seed=19))
    g.step(2)
    o.step(2)
    assert rel(g.get_field(pic.PIC_RHO), o.rho()) <= 1e-12
    assert rel(g.get_field(pic.PIC_DIVE), o.div_e()) <= 1e-12
    dg, do = g.diagnostics(), o.diagnostics()
    for k in ("field_energy", "kinetic_energy", "total_charge"):
        assert abs(dg[k] - do[k]) <= 1e-12 * abs(do[k]), k
    assert dg["n_particles"] == do["n_particles"] and dg["step"] == do["step"] == 2


def test_get_fields_and_gauss_residual():
    n = (20, 16, 24)
    g, o = pair(3, n, (0, 1, 0), (1.0, 0.9, 1.1), 0.45, 2, FP64)
    set_fields_both(g, o, synth.smooth_fields(n, 3, 0.1, seed=28))
    load_both(g, o, synth.random_particles(n, 3, 5000, 0.5, seed=29))
    g.step(2)
    o.step(2)
    comps = [pic.PIC_EX, pic.PIC_BZ, pic.PIC_JY, pic.PIC_RHO]
    many = g.get_fields(comps)
    for i, c in enumerate(comps[:3]):  # stored components: the same values
        assert np.array_equal(many[i], g.get_field(c)), c
    # rho is deposited anew by each call, with FP64 atomics in no fixed order
    assert rel(many[3], g.get_field(pic.PIC_RHO)) <= 1e-13
    r = o.div_e() - o.rho()
    m, rms = g.gauss_residual()
    assert abs(m - np.abs(r).max()) <= 1e-12 * np.abs(r).max()
    assert abs(rms - np.sqrt(np.mean(r * r))) <= 1e-12 * np.sqrt(np.mean(r * r))


@pytest.mark.parametrize("order", [1, 2])
def test_gauss_law_on_gpu(order):
    """Esirkepov + Yee on the GPU keep div E - rho constant to round-off (FP64)."""
    n = (24, 16, 16)
    g = pic.Simulation(3, n, (0, 0, 0), (1, 1, 1), 0.5, order=order, precision=FP64)
    parts = synth.uniform_plasma(n, 3, 2, 0.3, seed=20)
    g.load_particles(parts["cell"], parts["off"], parts["u"], parts["w"], parts["id"])
    r0 = g.get_field(pic.PIC_DIVE) - g.get_field(pic.PIC_RHO)
    g.step(10)
    r1 = g.get_field(pic.PIC_DIVE) - g.get_field(pic.PIC_RHO)
    assert np.abs(r1 - r0).max() < 1e-11
    assert g.diagnostics()["field_energy"] > 0


def test_batch_matches_oracle_per_instance():
    """Instances of different sizes and densities advanced in one launch per phase."""
    sims, orcs = [], []
    for i, (nx, nz, ppc) in enumerate([(32, 48, 2), (64, 32, 5), (48, 48, 1)]):
        n = (nx, 1, nz)
        g, o = pair(2, n, (0, 0, 1), (1.0, 1.0, 1.0), 0.5, 1 + i % 2, FP64, passes=i)
        set_fields_both(g, o, synth.smooth_fields(n, 2, 0.05, seed=30 + i))
        load_both(g, o, synth.uniform_plasma(n, 2, ppc, 0.2, seed=40 + i))
        sims.append(g)
        orcs.append(o)
    # shape orders differ: one batch per order
    b1 = pic.Batch([sims[0], sims[2]])
    b2 = pic.Batch([sims[1]])
    for _ in range(6):
        b1.step(1)
        b2.step(1)
    for o in orcs:
        o.step(6)
    for g, o in zip(sims, orcs):
        compare_fields(g, o, COMPS, 1e-12)
        compare_particles(g, o, 1e-12)


def test_errors_surface_as_status():
    g = pic.Simulation(3, (16, 16, 16), (0, 0, 0), (1, 1, 1), 0.5)
    with pytest.raises(pic.PicError) as e:
        g.step(1)
    assert e.value.status == pic.PIC_ERR_STATE
    with pytest.raises(pic.PicError) as e:
        g.load_particles(np.array([0], np.int32), np.array([[1.5, 0.0, 0.0]]), np.zeros((1, 3)), np.ones(1))
    assert e.value.status == pic.PIC_ERR_ARG
    with pytest.raises(pic.PicError) as e:
        g.load_particles(np.array([0], np.int32), np.array([[0.5, 0.0, 0.0]]), np.array([[np.nan, 0, 0]]), np.ones(1))
    assert e.value.status == pic.PIC_ERR_NAN


@pytest.mark.parametrize("ndim", [3, 2])
def test_phases_one_call_each_equal_the_oracle_step(ndim):
    """The three phases run as three pic_run_phases calls (particles, filter, Yee) make
    the oracle's step: the Yee call reads the current the filter call left (FP64, 1e-12)."""
    c = dict(CASES_3D if ndim == 3 else CASES_2D)
    bc = (0, 0, 0)
    g, o = pair(ndim, c["n"], bc, c["dx"], c["dt"], 2, FP64, passes=2)
    parts = synth.random_particles(c["n"], ndim, 6000, 0.2, seed=91)
    load_both(g, o, parts)
    set_fields_both(g, o, synth.smooth_fields(c["n"], ndim, 0.2, seed=92))
    for _ in range(3):
        g.run_phases(pic.PIC_PHASE_PARTICLES)
        g.run_phases(pic.PIC_PHASE_FILTER)
        g.run_phases(pic.PIC_PHASE_MAXWELL)
        o.step(1)
    compare_fields(g, o, COMPS + [pic.PIC_JX, pic.PIC_JY, pic.PIC_JZ], 1e-12)
