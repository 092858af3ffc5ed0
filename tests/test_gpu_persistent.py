"""The persistent batched step (pic_batch_set_persistent): a batch's steps as one launch
whose CTAs pull (step, phase, instance, item) work items, each waiting only for its own
instance's previous phase, with bounded waits.

* Against the per-phase launches of the same batch (CUDA graph): the batched 2D3V scan
  instances (uneven grids, 1-8 electrons per cell, lab-frame plasma with ions, laser,
  periodic box) and a 3D batch with absorbing and periodic boxes, FP32, 20 steps: every
  field (normwise) and the momenta within 1e-5, the particle counts equal.  Both runs are
  FP32 with the current tiles folded into the grid by atomic adds in no fixed order, so
  the two agree to FP32 rounding, not bit for bit.
* The timeout: an instance whose J set-up waits for an item that never runs (test_stall)
  ends the launch with PIC_ERR_TIMEOUT after the configured number of polls, and the
  device stays usable.
* What the persistent step refuses (FP64 members, the low-dispersion solver), and the
  online choice between the two launch forms (pic_batch_autotune).
"""
import numpy as np
import pytest

import paper_0909_5603_gb300 as pic
import synth

pytestmark = pytest.mark.gpu

FP32, FP64 = pic.PIC_PREC_FP32, pic.PIC_PREC_FP64
FIELDS = [pic.PIC_EX, pic.PIC_EY, pic.PIC_EZ, pic.PIC_BX, pic.PIC_BY, pic.PIC_BZ, pic.PIC_JX, pic.PIC_JY,
          pic.PIC_JZ]


@pytest.fixture(scope="module", autouse=True)
def built():
    pic.build()


def rel2(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def scan_members(count, prec=FP32, solver=pic.PIC_SOLVER_YEE):
    sims = []
    for i in range(count):
        d = synth.scan_instance(i)
        side = (48, 64, 96, 40, 80, 56)[i % 6]  # uneven, ragged against the 16 x 16 tiles
        d["n"] = (side, 1, side + 16 * (i % 3))
        pl = list(d["plasma"])
        pl[3] = min(pl[3], 8)
        lz = d["n"][2] * d["dx"][2]
        doppler = d["gamma_boost"] * (1 + np.sqrt(1 - 1 / d["gamma_boost"] ** 2))
        la = list(d["laser"])
        la[2] = 0.25 * d["n"][0] * d["dx"][0]
        la[4] = 0.5 * lz / doppler
        d["laser"] = tuple(la)
        s = pic.Simulation(2, d["n"], (0, 0, 0), d["dx"], d["dt"], gamma_boost=d["gamma_boost"], order=2,
                           precision=prec, filter_passes=3, tile=(16, 1, 16), solver=solver)
        s.load_lab_frame(laser=d["laser"], plasma=tuple(pl))
        sims.append(s)
    return sims


def members_3d():
    sims = []
    for i, (n, bc, order) in enumerate([((24, 16, 40), (0, 0, 0), 2), ((32, 24, 48), (1, 1, 1), 2),
                                         ((20, 20, 36), (0, 1, 0), 2)]):
        parts = synth.random_particles(n, 3, 30000 + 5000 * i, 0.4, seed=40 + i)
        fields = synth.smooth_fields(n, 3, 0.05, seed=50 + i)
        s = pic.Simulation(3, n, bc, (1.0, 1.0, 1.0), 0.45, order=order, precision=FP32, filter_passes=2,
                           tile=(8, 8, 8), absorb_cells=4)
        s.load_particles(parts["cell"], parts["off"], parts["u"], parts["w"], parts["id"])
        for c in range(6):
            s.set_field(c, fields[c])
        sims.append(s)
    return sims


def compare(a_sims, b_sims, tol):
    worst = 0.0
    for a, b in zip(a_sims, b_sims):
        assert a.num_particles() == b.num_particles()
        for c in FIELDS:
            fb = b.get_field(c)
            if np.abs(fb).max() == 0:
                assert np.abs(a.get_field(c)).max() == 0
                continue
            e = rel2(a.get_field(c), fb)
            worst = max(worst, e)
            assert e <= tol, (c, e)
        pa, pb = a.get_particles(), b.get_particles()
        common, ia, ib = np.intersect1d(pa["id"], pb["id"], return_indices=True)
        e = rel2(pa["u"][ia], pb["u"][ib])
        worst = max(worst, e)
        assert e <= tol
    return worst


@pytest.mark.parametrize("kind", ["scan_2d", "boxes_3d"])
def test_persistent_batch_matches_per_phase_launches(kind):
    make = (lambda: scan_members(12)) if kind == "scan_2d" else members_3d
    ref, per = make(), make()
    bref, bper = pic.Batch(ref), pic.Batch(per)
    bper.set_persistent(True)
    bref.step(20)
    bper.step(20)  # one launch
    bref.synchronize()
    bper.synchronize()
    worst = compare(per, ref, 1e-5)
    print(f"{kind}: persistent vs per-phase launches after 20 steps, worst normwise {worst:.2e}")
    # step() again in two calls: the counters restart per launch
    bref.step(3)
    bper.step(1)
    bper.step(2)
    bref.synchronize()
    bper.synchronize()
    compare(per, ref, 1e-5)


def test_persistent_wait_times_out_and_device_stays_usable():
    sims = scan_members(6)
    b = pic.Batch(sims)
    b.set_persistent(True, spin_limit=2000, test_stall=3)
    b.step(2)
    with pytest.raises(pic.PicError) as e:
        b.synchronize()
    assert e.value.status == pic.PIC_ERR_TIMEOUT
    # a fresh batch on the same device steps normally afterwards
    again = scan_members(3)
    b2 = pic.Batch(again)
    b2.set_persistent(True)
    b2.step(2)
    b2.synchronize()


def test_persistent_refuses_what_it_does_not_run():
    b = pic.Batch(scan_members(2, prec=FP64))
    with pytest.raises(pic.PicError) as e:
        b.set_persistent(True)
    assert e.value.status == pic.PIC_ERR_UNSUPPORTED
    b2 = pic.Batch(scan_members(2, solver=pic.PIC_SOLVER_CK))
    with pytest.raises(pic.PicError) as e:
        b2.set_persistent(True)
    assert e.value.status == pic.PIC_ERR_UNSUPPORTED


def test_batch_autotune_times_both_forms_and_keeps_the_faster():
    b = pic.Batch(scan_members(8))
    chosen, ms_graph, ms_persistent = b.autotune(2)
    print(f"batch autotune: graph {ms_graph:.3f} ms/step, persistent {ms_persistent:.3f} ms/step, "
          f"persistent chosen: {chosen}")
    assert ms_graph > 0 and ms_persistent > 0
    assert chosen == (ms_persistent < ms_graph)
    b.step(2)
    b.synchronize()
    # a batch the persistent step does not run: only the graph is timed
    b64 = pic.Batch(scan_members(2, prec=FP64))
    chosen, ms_graph, ms_persistent = b64.autotune(1)
    assert not chosen and ms_graph > 0 and ms_persistent == -1.0
