"""pic_autotune: times every candidate tile on the workload and returns the fastest; the
chosen tile must be one of the candidates and give the same physics (FP64, to 1e-12)."""
import numpy as np
import pytest

import paper_0909_5603_gb300 as pic
import synth

pytestmark = pytest.mark.gpu

CAND_2D = {(16, 1, 16), (32, 1, 8), (8, 1, 32), (32, 1, 16), (16, 1, 32), (32, 1, 32), (64, 1, 8)}
CAND_3D = {(8, 8, 8), (16, 8, 8), (8, 8, 16), (8, 16, 8), (16, 16, 4), (16, 8, 4), (8, 8, 4), (4, 8, 8),
           (16, 16, 8), (32, 8, 4)}


def test_autotune_2d_scan_instance():
    d = synth.scan_instance(2)
    n = (128, 1, 128)
    tile, ms = pic.autotune(2, n, (0, 0, 0), d["dx"], d["dt"], d["gamma_boost"], order=2, filter_passes=3,
                            laser=d["laser"], plasma=d["plasma"], steps=3)
    assert tuple(tile) in CAND_2D and ms > 0
    # the tile changes the schedule, not the result
    runs = []
    for t in (tile, (16, 1, 16)):
        s = pic.Simulation(2, n, (0, 0, 0), d["dx"], d["dt"], gamma_boost=d["gamma_boost"], order=2,
                           precision=pic.PIC_PREC_FP64, filter_passes=3, tile=t)
        s.load_lab_frame(laser=d["laser"], plasma=d["plasma"])
        s.step(5)
        runs.append((s.get_field(pic.PIC_EX), s.get_field(pic.PIC_JZ)))
    for a, b in zip(*runs):
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


def test_autotune_3d_lwfa_slab():
    w = synth.lwfa_stage((64, 64, 64), 13.0, 2)
    tile, ms = pic.autotune(3, w["n"], (1, 1, 1), w["dx"], w["dt"], 13.0, order=2, filter_passes=3,
                            laser=w["laser"], plasma=w["plasma"], steps=2)
    assert tuple(tile) in CAND_3D and ms > 0
