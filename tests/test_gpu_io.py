"""Particle input and output in the storage precision on the GPU.

* pic_get_particles_stored: an FP32 context's particles as floats, which widened are
  exactly what pic_get_particles returns (FP64 contexts: the same doubles); into
  caller-provided page-locked arrays, reused across calls.
* pic_load_particles_stored: FP32 values loaded as they are give the bit pattern of the
  same values loaded through the FP64 entry, and the two runs stay together (an FP32 run
  is not bit-reproducible: the tiles add their current to the global grid in no fixed
  order, so after steps within 1e-5); invalid floats (an offset of 1, a non-finite
  momentum) are refused like invalid doubles.
"""
import numpy as np
import pytest

import paper_0909_5603_gb300 as pic
import synth

pytestmark = pytest.mark.gpu

FP32, FP64 = pic.PIC_PREC_FP32, pic.PIC_PREC_FP64
N = (16, 16, 40)
KEYS = ("cell", "off", "u", "w", "id")


@pytest.fixture(scope="module", autouse=True)
def built():
    pic.build()


def make(prec, track_ids=True):
    return pic.Simulation(3, N, (0, 0, 1), (1.0, 1.0, 1.0), 0.45, order=2, precision=prec, filter_passes=2,
                          absorb_cells=4, track_ids=track_ids)


def problem(seed=41):
    return synth.random_particles(N, 3, 30000, 0.3, seed=seed), synth.smooth_fields(N, 3, 0.05, seed=seed + 1)


def below_one_f32(off):
    """off rounded to FP32 the way the device stores it (round to nearest, an offset that
    rounds to 1 kept just below it)."""
    return np.minimum(off.astype(np.float32), np.nextafter(np.float32(1), np.float32(0)))


@pytest.mark.parametrize("prec", [FP32, FP64], ids=["fp32", "fp64"])
def test_stored_readout_is_the_widened_readout(prec):
    import torch

    parts, fields = problem()
    s = make(prec)
    s.load_particles(parts["cell"], parts["off"], parts["u"], parts["w"], parts["id"])
    for c in range(6):
        s.set_field(c, fields[c])
    s.step(4)
    wide = s.get_particles()
    st = s.get_particles(stored=True)
    vt = np.float32 if prec == FP32 else np.float64
    n = wide["cell"].size
    assert n > 20000
    for k in ("off", "u", "w"):
        assert st[k].dtype == vt
        assert np.array_equal(st[k].astype(np.float64), wide[k]), k
    for k in ("cell", "id"):
        assert np.array_equal(st[k], wide[k]), k
    # page-locked output arrays with room to spare, filled in place and reused
    room = n + 1000
    out = {"cell": torch.empty(room, dtype=torch.int32).pin_memory().numpy(),
           "off": torch.empty(3 * room, dtype=torch.float32 if prec == FP32 else torch.float64).pin_memory().numpy(),
           "u": torch.empty((room, 3), dtype=torch.float32 if prec == FP32 else torch.float64).pin_memory().numpy(),
           "w": torch.empty(room, dtype=torch.float32 if prec == FP32 else torch.float64).pin_memory().numpy()}
    for _ in range(2):
        got = s.get_particles(stored=True, out=out)
        for k in ("cell", "off", "u", "w"):
            assert np.shares_memory(got[k], out[k]), k
            assert got[k].shape == st[k].shape
            assert np.array_equal(got[k], st[k]), k
        assert np.array_equal(got["id"], st["id"])  # not in out: allocated
        s.step(1)
        st = s.get_particles(stored=True)
        n = st["cell"].size
    with pytest.raises(ValueError):
        s.get_particles(stored=True, out={"w": np.empty(room, np.float16)})
    with pytest.raises(ValueError):
        s.get_particles(out={"cell": np.empty(3, np.int32)})


def test_stored_load_steps_like_the_fp64_load():
    parts, fields = problem(seed=43)
    off32, u32, w32 = below_one_f32(parts["off"]), parts["u"].astype(np.float32), parts["w"].astype(np.float32)
    a, b = make(FP32), make(FP32)
    a.load_particles(parts["cell"], off32.astype(np.float64), u32.astype(np.float64), w32.astype(np.float64),
                     parts["id"])
    b.load_particles(parts["cell"], off32, u32, w32, parts["id"])
    for s in (a, b):
        for c in range(6):
            s.set_field(c, fields[c])
    pa, pb = a.get_particles(stored=True), b.get_particles(stored=True)
    for k in KEYS:
        assert np.array_equal(pa[k], pb[k]), k
    for c in range(6):
        assert np.array_equal(a.get_field(c), b.get_field(c)), c
    a.step(6)
    b.step(6)
    for c in range(9):
        fa, fb = a.get_field(c), b.get_field(c)
        assert np.linalg.norm(fa - fb) <= 1e-5 * np.linalg.norm(fa), c
    pa, pb = a.get_particles(), b.get_particles()
    ia, ib = np.argsort(pa["id"]), np.argsort(pb["id"])
    assert np.array_equal(pa["id"][ia], pb["id"][ib])
    du = pa["u"][ia] - pb["u"][ib]
    assert np.linalg.norm(du) <= 1e-5 * np.linalg.norm(pa["u"])


def test_stored_load_refuses_invalid_floats():
    parts, _ = problem(seed=47)
    s = make(FP32, track_ids=False)
    off32, u32, w32 = below_one_f32(parts["off"]), parts["u"].astype(np.float32), parts["w"].astype(np.float32)
    bad = off32.copy()
    bad[1234, 2] = np.float32(1.0)
    with pytest.raises(pic.PicError) as e:
        s.load_particles(parts["cell"], bad, u32, w32)
    assert e.value.status == pic.PIC_ERR_ARG and "1234" in str(e.value)
    bad = u32.copy()
    bad[777, 0] = np.float32(np.inf)
    with pytest.raises(pic.PicError) as e:
        s.load_particles(parts["cell"], off32, bad, w32)
    assert e.value.status == pic.PIC_ERR_NAN and "777" in str(e.value)
    s.load_particles(parts["cell"], off32, u32, w32)
    assert s.num_particles() == parts["cell"].size
