"""The batched 2D3V boosted-frame scan: independent instances of uneven grid and particle
counts advanced together (one launch per phase over all instances, replayed from one
CUDA graph).

Instances follow the scan recipe (tests/synth.py scan_instance: gamma_b in [1, 50],
n/n_c in [1e-4, 1e-2], 1-16 electrons per cell, laser pulse, periodic box with the ions'
background), shrunk to grids the oracle steps in seconds.  FP32 batched against the FP64
oracle per instance after 100 steps: E, B and J (each as a vector field) and the momenta
within 1e-5 normwise, or within 8x of the FP32-storage floor where the grid is numerically
unstable; FP64 batched against the same instances stepped one by one, within 1e-12.
"""
import numpy as np
import pytest

import oracle
import paper_0909_5603_gb300 as pic
import synth

pytestmark = pytest.mark.gpu

FP32, FP64 = pic.PIC_PREC_FP32, pic.PIC_PREC_FP64
FIELDS = [pic.PIC_EX, pic.PIC_EY, pic.PIC_EZ, pic.PIC_BX, pic.PIC_BY, pic.PIC_BZ, pic.PIC_JX, pic.PIC_JY,
          pic.PIC_JZ]


@pytest.fixture(scope="module", autouse=True)
def built():
    pic.build()
    oracle.build()


def rel2(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def small_instance(i, n_side):
    """Scan instance i with its grid replaced by n_side x n_side (same spacing, step,
    boost, density, particles per cell up to 8)."""
    d = synth.scan_instance(i)
    d["n"] = (n_side, 1, n_side)
    ppc = min(d["ppc"], 8)
    pl = list(d["plasma"])
    pl[3] = ppc
    d["plasma"] = tuple(pl)
    lz = n_side * d["dx"][2]
    doppler = d["gamma_boost"] * (1 + np.sqrt(1 - 1 / d["gamma_boost"] ** 2))
    la = list(d["laser"])
    la[2] = 0.25 * n_side * d["dx"][0]
    la[4] = 0.5 * lz / doppler
    d["laser"] = tuple(la)
    return d


def make_gpu(d, prec):
    s = pic.Simulation(2, d["n"], (0, 0, 0), d["dx"], d["dt"], gamma_boost=d["gamma_boost"], order=2, precision=prec,
                       filter_passes=3, tile=(16, 1, 16))
    s.load_lab_frame(laser=d["laser"], plasma=d["plasma"])
    return s


def make_oracle(d):
    o = oracle.Sim(2, d["n"], (0, 0, 0), d["dx"], d["dt"], order=2, filter_passes=3, tile=(16, 1, 16))
    pl = d["plasma"]
    o.load_lab_frame(d["gamma_boost"], laser=d["laser"], plasma=[*pl[:4], *pl[4], pl[5]])
    return o


CASES = [(0, 32), (1, 48), (2, 64), (3, 32), (4, 48)]


def errors(a, b):
    """Normwise relative differences of E, B, J (each as a vector field) and u."""
    errs = {}
    for name, comps in (("E", FIELDS[0:3]), ("B", FIELDS[3:6]), ("J", FIELDS[6:9])):
        errs[name] = rel2(np.stack([a.get_field(c) for c in comps]), np.stack([b.get_field(c) for c in comps]))
    pa, pb = a.get_particles(), b.get_particles()
    assert np.array_equal(np.sort(pa["id"]), np.sort(pb["id"]))
    ia, ib = np.argsort(pa["id"]), np.argsort(pb["id"])
    errs["u"] = rel2(pa["u"][ia], pb["u"][ib])
    return errs


def test_scan_batch_fp32_against_oracle():
    """After 100 steps each instance is within 1e-5 of the FP64 oracle (normwise, per field
    and for the momenta).  The one exception is a reading: an instance whose coarse
    boosted grid is numerically unstable (max |E| grown more than 3x above the laser's
    amplitude; the paper's Sec. 2 instability) amplifies every rounding difference, and
    there a field may exceed 1e-5 if it stays within 8x of the floor that FP32 storage
    alone sets: the FP64 oracle with its state rounded to FP32 after every step.  The
    instances and fields that use the exception are printed."""
    ds = [small_instance(i, n) for i, n in CASES]
    sims = [make_gpu(d, FP32) for d in ds]
    batch = pic.Batch(sims)
    batch.step(100)
    batch.synchronize()
    rows = []
    for d, g in zip(ds, sims):
        o = make_oracle(d)
        o.step(100)
        e = make_oracle(d)
        e.round_state_fp32()
        for _ in range(100):
            e.step(1)
            e.round_state_fp32()
        gpu, floor = errors(g, o), errors(e, o)
        growth = max(np.abs(o.get_field(c)).max() for c in FIELDS[:3]) / (2 * np.pi / (
            d["gamma_boost"] * (1 + np.sqrt(1 - 1 / d["gamma_boost"] ** 2))))
        print(f"gamma_b {d['gamma_boost']:.1f} n {d['n'][0]} ppc {d['plasma'][3]} max|E|/laser {growth:.1f}: "
              + " ".join(f"{k} {v:.1e} (floor {floor[k]:.1e})" for k, v in gpu.items()))
        rows.append((d, gpu, floor, growth))
    over = []
    for d, gpu, floor, growth in rows:
        for k, v in gpu.items():
            if v <= 1e-5:
                continue
            over.append(f"gamma_b {d['gamma_boost']:.1f} n {d['n'][0]} {k} {v:.2e} floor {floor[k]:.2e} "
                        f"growth {growth:.1f}")
            assert growth > 3.0 and v <= 8 * floor[k], over[-1]
    print("above 1e-5 (unstable instances, within 8x the FP32 storage floor):", over or "none")


def test_scan_batch_fp64_equals_instances_stepped_alone():
    ds = [small_instance(i, n) for i, n in CASES]
    alone = [make_gpu(d, FP64) for d in ds]
    together = [make_gpu(d, FP64) for d in ds]
    for s in alone:
        s.step(20)
    batch = pic.Batch(together)
    batch.step(20)
    batch.synchronize()
    for a, b in zip(alone, together):
        for c in FIELDS:
            fa, fb = a.get_field(c), b.get_field(c)
            assert np.abs(fa - fb).max() <= 1e-12 * max(np.abs(fa).max(), 1e-300), c
        pa, pb = a.get_particles(), b.get_particles()
        assert np.array_equal(pa["id"], pb["id"]) and np.array_equal(pa["cell"], pb["cell"])
        assert np.abs(pa["u"] - pb["u"]).max() <= 1e-12 * np.abs(pa["u"]).max()
