"""The z-slab split of one run on the GPU: the whole grid's context cut into 2 or 3 slab
contexts on the same device (paper_0909_5603_gb300.slab.split_gpu), stepped with the
in-process exchange, against the unsplit run.

* Random particles under smooth fields, x-y periodic, z periodic or absorbing (no damping
  layer), order 2, 3 filter passes, Yee and the low-dispersion solver, FP64: every owned
  plane of E, B, J and every particle equal the unsplit GPU run and the FP64 oracle to
  1e-12 after 12 steps.
* The boosted laser-wakefield stage (16 x 16 x 96, gamma_b 13, lab-frame plasma with its
  ion background streaming through the slab faces, absorbing box with its damping layer)
  in FP64 against the unsplit GPU run to 1e-12 and in FP32 within 1e-5 normwise, 40 steps.
"""
import numpy as np
import pytest

import oracle
import paper_0909_5603_gb300 as pic
import synth
from paper_0909_5603_gb300 import slab as S

pytestmark = pytest.mark.gpu

FP32, FP64 = pic.PIC_PREC_FP32, pic.PIC_PREC_FP64
COMPS = list(range(9))


def run_split(whole_kw, load, nslabs, steps, n):
    """Returns the owned planes of every component (stacked along z) and the particles
    (global cells) of the split run, and the whole context after the same steps."""
    whole = pic.Simulation(3, n, **{k: v for k, v in whole_kw.items()})
    load(whole)
    bc = whole_kw["bc"]
    slabs = S.plan(n[2], nslabs, bc[2] == pic.PIC_PERIODIC, ghost=S.ghost_planes(whole_kw.get("filter_passes", 0)))
    kw = dict(whole_kw)
    sims = S.split_gpu(whole, slabs, range(nslabs), **kw)
    run = S.SlabRun(slabs, {r: S.GpuShard(s) for r, s in sims.items()}, S.InProcess(), n[0], n[1])
    run.step(steps)
    owned = {c: np.concatenate([run.owned_field(s.rank, c) for s in slabs]) for c in COMPS}
    parts = []
    for s in slabs:
        p = sims[s.rank].get_particles()
        cell = p["cell"].astype(np.int64) + s.lo * n[0] * n[1]
        if s.lo < 0 or s.lo + s.nz > n[2]:
            cell %= n[0] * n[1] * n[2]
        parts.append(dict(p, cell=cell))
    merged = {k: np.concatenate([p[k] for p in parts]) for k in parts[0]}
    whole.step(steps)
    return owned, merged, whole


def by_id(p):
    o = np.argsort(p["id"], kind="stable")
    return {k: v[o] for k, v in p.items()}


def relinf(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300))


def rel2(a, b):
    return float(np.linalg.norm(np.ravel(a - b)) / max(np.linalg.norm(np.ravel(b)), 1e-300))


@pytest.mark.parametrize("nslabs", [2, 3])
@pytest.mark.parametrize("zbc", [pic.PIC_PERIODIC, pic.PIC_ABSORBING], ids=["z-periodic", "z-absorbing"])
@pytest.mark.parametrize("solver", [pic.PIC_SOLVER_YEE, pic.PIC_SOLVER_CK], ids=["yee", "ck"])
def test_slabs_fp64_equal_whole_gpu_run_and_oracle(nslabs, zbc, solver):
    pic.build()
    oracle.build()
    n, steps = (16, 8, 48), 12
    parts = synth.random_particles(n, 3, 20000, 0.5, seed=21)
    fields = synth.smooth_fields(n, 3, 0.05, seed=22)

    def load(sim):
        sim.load_particles(parts["cell"], parts["off"], parts["u"], parts["w"], parts["id"])
        for c in range(6):
            sim.set_field(c, fields[c])

    kw = dict(bc=(pic.PIC_PERIODIC, pic.PIC_PERIODIC, zbc), dx=(1.0, 1.0, 1.0), dt=0.45, order=2,
              precision=FP64, filter_passes=3, absorb_cells=0, solver=solver, tile=(8, 8, 8))
    owned, sp, whole = run_split(kw, load, nslabs, steps, n)
    o = oracle.Sim(3, n, kw["bc"], (1.0, 1.0, 1.0), 0.45, order=2, filter_passes=3, tile=(8, 8, 8),
                   absorb_cells=0, solver=solver)
    for c in range(6):
        o.set_field(c, fields[c])
    o.set_particles(parts["cell"], parts["off"], parts["u"], parts["w"], parts["id"])
    o.step(steps)
    errs = {}
    for c in COMPS:
        errs[f"{c} vs whole"] = relinf(owned[c], whole.get_field(c))
        errs[f"{c} vs oracle"] = relinf(owned[c], o.get_field(c))
    a, w, r = by_id(sp), by_id(whole.get_particles()), by_id(o.get_particles())
    assert np.array_equal(a["id"], w["id"]) and np.array_equal(a["id"], r["id"])
    assert np.array_equal(a["cell"], w["cell"]) and np.array_equal(a["cell"], r["cell"])
    errs["u vs oracle"] = relinf(a["u"], r["u"])
    errs["off vs oracle"] = float(np.abs(a["off"] - r["off"]).max())
    print(f"{nslabs} slabs zbc {zbc} solver {solver}: max " + f"{max(errs.values()):.2e}")
    for k, v in errs.items():
        assert v <= 1e-12, (k, v)


@pytest.mark.parametrize("prec", [FP64, FP32], ids=["fp64", "fp32"])
def test_slabs_lwfa_with_ions_equal_whole_gpu_run(prec):
    pic.build()
    gb = 13.0
    w = synth.lwfa_stage((16, 16, 96), gb, 2, seed=11)
    kw = dict(bc=(1, 1, 1), dx=w["dx"], dt=w["dt"], gamma_boost=gb, order=2, precision=prec, filter_passes=3,
              tile=(8, 8, 8), track_ids=True)

    def load(sim):
        sim.load_lab_frame(laser=w["laser"], plasma=w["plasma"])

    owned, sp, whole = run_split(kw, load, 2, 40, w["n"])
    a, b = by_id(sp), by_id(whole.get_particles())
    errs = {}
    if prec == FP64:
        assert np.array_equal(a["id"], b["id"]) and np.array_equal(a["cell"], b["cell"])
        for c in COMPS:
            errs[c] = relinf(owned[c], whole.get_field(c))
        errs["u"] = relinf(a["u"], b["u"])
        tol = 1e-12
    else:
        common, ia, ib = np.intersect1d(a["id"], b["id"], return_indices=True)
        assert max(a["id"].size, b["id"].size) - common.size <= 4
        for name, cs in (("E", COMPS[0:3]), ("B", COMPS[3:6]), ("J", COMPS[6:9])):
            errs[name] = rel2(np.stack([owned[c] for c in cs]), np.stack([whole.get_field(c) for c in cs]))
        errs["u"] = rel2(a["u"][ia], b["u"][ib])
        tol = 1e-5
    print(f"LWFA 16x16x96 gamma_b 13, 2 slabs vs whole, prec {prec}: " + " ".join(f"{k} {v:.2e}" for k, v in errs.items()))
    for k, v in errs.items():
        assert v <= tol, (k, v)


@pytest.mark.parametrize("prec", [FP64, FP32], ids=["fp64", "fp32"])
def test_extract_then_add_back_continues_the_run(prec):
    """pic_extract_particles takes out exactly the particles outside the planes asked for
    (their values bit for bit, in canonical order) and pic_add_particles puts them back:
    the run then continues as if nothing had happened (FP64 within 1e-12; FP32 bit for
    bit on particles and fields is not expected, the tiles' summation order changes, so
    within 1e-6)."""
    pic.build()
    n = (16, 16, 40)
    parts = synth.random_particles(n, 3, 30000, 0.3, seed=31)
    fields = synth.smooth_fields(n, 3, 0.05, seed=32)

    def make():
        s = pic.Simulation(3, n, (0, 0, 1), (1.0, 1.0, 1.0), 0.45, order=2, precision=prec, filter_passes=2,
                           absorb_cells=4)
        s.load_particles(parts["cell"], parts["off"], parts["u"], parts["w"], parts["id"])
        for c in range(6):
            s.set_field(c, fields[c])
        return s

    a, b = make(), make()
    a.step(3)
    b.step(3)
    before = by_id(b.get_particles())
    out = b.extract_particles(10, 30)
    k = out["cell"] // (n[0] * n[1])
    assert out["cell"].size > 1000 and np.all((k < 10) | (k >= 30))
    rest = b.get_particles()
    kr = rest["cell"] // (n[0] * n[1])
    assert np.all((kr >= 10) & (kr < 30))
    assert out["cell"].size + rest["cell"].size == before["cell"].size
    got = by_id({key: np.concatenate([out[key], rest[key]]) for key in out})
    for key in ("cell", "id", "off", "u", "w"):
        assert np.array_equal(got[key], before[key]), key
    b.add_particles(out["cell"], out["off"], out["u"], out["w"], out["id"])
    assert np.array_equal(by_id(b.get_particles())["u"], before["u"])
    a.step(5)
    b.step(5)
    tol = 1e-12 if prec == FP64 else 1e-6
    for c in COMPS:
        assert relinf(b.get_field(c), a.get_field(c)) <= tol, c
    pa, pb = by_id(a.get_particles()), by_id(b.get_particles())
    assert np.array_equal(pa["id"], pb["id"]) and np.array_equal(pa["cell"], pb["cell"])
    assert relinf(pb["u"], pa["u"]) <= tol
