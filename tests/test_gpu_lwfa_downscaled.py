"""The boosted laser-wakefield stage's precision sweep on a downscaled copy against the FP64
oracle: the recipe of the 256 x 256 x 2048 sweep (tests/synth.py lwfa_stage: cell size,
a0 = 2 laser, plasma at n/n_c = 1/900 with its ion background, order-2 shape, 3-pass
filter, Vay, absorbing box) on 64 x 64 x 512 cells with 4 electrons per cell (8,388,608
particles), gamma_b in {2, 5, 13, 30, 100}, 100 steps.

The oracle's results are stored summaries (tests/golden/lwfa_64x64x512_gb<gamma>.json,
written by tests/golden/make_lwfa_64x64x512.py, which calls only the oracle): the wake
field E_z and the laser field E_x along the axis and the plane-by-plane rms of E_z at
steps 50 and 100, and the field and kinetic energies every 10 steps.  Both GPU precisions
run the same seeded load; the errors per boost are printed (the precision report).

Bars.  The all-FP64 GPU path within 1e-9 of the oracle on every summary (measured on
GB300: fields 1e-15 to 1.4e-12, the energy sums 1e-12 to 1e-10, which add the particles
and cells in another order).  The FP32 path (FP32 storage, FP64 gamma solve where sigma
can cancel) within 1e-5 where the boosted grid is stable (gamma_b 2, 5: measured at most
1.9e-6).  Where the Sec. 2 instability grows the field (field energy at step 100 more
than 3x its step-10 value: x97 at gamma_b 13, x340 at 30, x470 at 100) every rounding
difference grows with it, and the bar is 1e-4 (measured at most 5.6e-5, E_z on the axis
at gamma_b 30, step 50; 2.5e-6 at gamma_b 13).
"""
import json
import os

import numpy as np
import pytest

import paper_0909_5603_gb300 as pic
import synth

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
GAMMAS = [2.0, 5.0, 13.0, 30.0, 100.0]
FP32, FP64 = pic.PIC_PREC_FP32, pic.PIC_PREC_FP64


def rel2(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def golden(gb):
    with open(os.path.join(HERE, "golden", f"lwfa_64x64x512_gb{gb:g}.json")) as f:
        return json.load(f)


@pytest.mark.parametrize("gb", GAMMAS)
@pytest.mark.parametrize("prec", [FP64, FP32], ids=["fp64", "fp32"])
def test_lwfa_64x64x512_against_oracle(prec, gb):
    pic.build()
    gold = golden(gb)
    n = tuple(gold["grid"])
    w = synth.lwfa_stage(n, gb, gold["ppc"], seed=gold["seed"])
    assert np.allclose(w["dx"], gold["dx"]) and w["dt"] == gold["dt"]
    g = pic.Simulation(3, n, (1, 1, 1), w["dx"], w["dt"], gamma_boost=gb, order=2, precision=prec, filter_passes=3,
                       tile=(8, 8, 8), track_ids=False)
    g.load_lab_frame(laser=w["laser"], plasma=w["plasma"])
    assert g.num_particles() == gold["particles_loaded"]
    ax = gold["axis"]
    errs, done = {}, 0
    diag = {d["step"]: d for d in gold["diagnostics"]}
    for step in sorted(set(diag) | {int(k) for k in gold["checkpoints"]}):
        g.step(step - done)
        done = step
        if step in diag:
            d = g.diagnostics()
            for k in ("field_energy", "kinetic_energy"):
                e = abs(d[k] - diag[step][k]) / max(abs(diag[step][k]), 1e-300)
                errs[k] = max(errs.get(k, 0.0), e)
        if str(step) in gold["checkpoints"]:
            ck = gold["checkpoints"][str(step)]
            ez, ex = g.get_field(pic.PIC_EZ), g.get_field(pic.PIC_EX)
            errs[f"Ez_axis@{step}"] = rel2(ez[:, ax[1], ax[0]], ck["ez_axis"])
            errs[f"Ex_axis@{step}"] = rel2(ex[:, ax[1], ax[0]], ck["ex_axis"])
            errs[f"Ez_planes@{step}"] = rel2(np.sqrt((ez ** 2).mean(axis=(1, 2))), ck["ez_plane_rms"])
    growth = diag[100]["field_energy"] / diag[10]["field_energy"]
    print(f"gamma_b {gb:g} {'FP64' if prec == FP64 else 'FP32'} vs oracle (64x64x512, 4 ppc), field energy "
          f"x{growth:.2f} from step 10 to 100: " + " ".join(f"{k} {v:.2e}" for k, v in errs.items()))
    bar = 1e-9 if prec == FP64 else (1e-5 if growth <= 3.0 else 1e-4)
    for k, v in errs.items():
        assert v <= bar, (k, v, bar)
