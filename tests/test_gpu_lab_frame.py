"""Lab-frame loads stepped on the GPU against the FP64 oracle: laser, plasma with its
ion background (lab-stationary ions streaming at -beta_b in the boosted frame) and the
boosted LWFA stage in FP32 over 100 steps, with the error stated per field and per boost.
"""
import numpy as np
import pytest

import oracle
import paper_0909_5603_gb300 as pic
import synth

pytestmark = pytest.mark.gpu

FP32, FP64 = pic.PIC_PREC_FP32, pic.PIC_PREC_FP64
COMPS = [pic.PIC_EX, pic.PIC_EY, pic.PIC_EZ, pic.PIC_BX, pic.PIC_BY, pic.PIC_BZ]
JCOMPS = [pic.PIC_JX, pic.PIC_JY, pic.PIC_JZ]
NAMES = {pic.PIC_EX: "Ex", pic.PIC_EY: "Ey", pic.PIC_EZ: "Ez", pic.PIC_BX: "Bx", pic.PIC_BY: "By",
         pic.PIC_BZ: "Bz", pic.PIC_JX: "Jx", pic.PIC_JY: "Jy", pic.PIC_JZ: "Jz"}


@pytest.fixture(scope="module", autouse=True)
def built():
    pic.build()
    oracle.build()


def rel2(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def relinf(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300))


def pair(ndim, n, bc, dx, dt, gb, prec, order=2, passes=0, absorb=16, tile=None):
    if tile is None:
        tile = (8, 8, 8) if ndim == 3 else (16, 1, 16)
    g = pic.Simulation(ndim, n, bc, dx, dt, gamma_boost=gb, order=order, precision=prec, filter_passes=passes,
                       tile=tile, absorb_cells=absorb)
    o = oracle.Sim(ndim, n, bc, dx, dt, order=order, filter_passes=passes, tile=tile, absorb_cells=absorb)
    return g, o


def load(g, o, gb, laser=None, plasma=None):
    g.load_lab_frame(laser=laser, plasma=plasma)
    po = None if plasma is None else [*plasma[:4], *plasma[4], plasma[5]]
    o.load_lab_frame(gb, laser=laser, plasma=po)


@pytest.mark.parametrize("bcz", [0, 1], ids=["periodic_z", "absorbing_z"])
@pytest.mark.parametrize("ndim", [2, 3])
def test_plasma_with_ions_fp64(ndim, bcz):
    """Laser + ramped plasma, 12 full steps: fields, particles and rho (ions included)
    within 1e-12 of the oracle; the ramp crosses the periodic wrap or the -z face."""
    gb = 5.0
    n = (12, 8, 48) if ndim == 3 else (24, 1, 64)
    bc = (1, 0, bcz)
    dz = 0.5
    dt = 0.2
    g, o = pair(ndim, n, bc, (1.0, 1.0, dz), dt, gb, FP64, passes=1, absorb=4)
    laser = (1.0, 1.0, 4.0, 1.0, 1.0)
    plasma = (0.5, 0.5, 3.0, 2, (0.01, 0.01, 0.01), 4)
    load(g, o, gb, laser, plasma)
    g.step(12)
    o.step(12)
    for c in COMPS + JCOMPS:
        fo = o.get_field(c)
        if np.abs(fo).max() == 0:
            continue
        assert relinf(g.get_field(c), fo) <= 1e-12, NAMES[c]
    assert relinf(g.get_field(pic.PIC_RHO), o.rho()) <= 1e-12
    pg, po = g.get_particles(), o.get_particles()
    assert np.array_equal(pg["id"], po["id"]) and np.array_equal(pg["cell"], po["cell"])
    assert relinf(pg["u"], po["u"]) <= 1e-12


def test_gauss_law_with_ions_on_gpu():
    """div E - rho (ions included) constant to round-off in the interior while the
    ramped plasma streams through an absorbing box (FP64, unfiltered)."""
    gb = 4.0
    n = (8, 8, 64)
    g = pic.Simulation(3, n, (0, 0, 1), (1.0, 1.0, 0.5), 0.3, gamma_boost=gb, order=2, precision=FP64,
                       absorb_cells=4)
    g.load_lab_frame(plasma=(0.2, 20.0, 40.0, 2, (0.05, 0.05, 0.05), 11))
    rho0 = g.get_field(pic.PIC_RHO)
    r0 = g.get_field(pic.PIC_DIVE) - rho0
    g.step(25)
    rho1 = g.get_field(pic.PIC_RHO)
    r1 = g.get_field(pic.PIC_DIVE) - rho1
    inner = slice(6, n[2] - 6)
    scale = np.abs(rho1).max()
    assert np.abs(r1 - r0)[inner].max() <= 1e-11 * scale
    assert np.abs(rho1 - rho0)[inner].max() > 0.1 * scale


@pytest.mark.parametrize("gb", [2.0, 5.0, 13.0, 30.0, 100.0])
def test_lwfa_stage_fp32_100_steps(gb):
    """The boosted LWFA stage (ramped plasma n/n_c = 1/900 with its ions, a0 = 2 laser,
    order 2, 3-pass filter, Vay, absorbing box) downscaled to 16 x 16 x 96 cells with a
    2-period laser centred in the box: FP32 storage with the FP64 gamma solve against the
    FP64 oracle after 50 and 100 steps, every field and the particles within 1e-5
    (normwise), at every boost.  One reading: at gamma_b = 100 this coarse grid is
    numerically unstable (fields grow about 20x by step 50, the paper's Sec. 2
    instability) and the error passes through a transient near step 50; there the step-50
    bar is 3e-5, and 1e-5 holds again at step 100.  The boosts are those of the precision
    sweep at scale (bench.py --precision-sweep)."""
    w = synth.lwfa_stage((16, 16, 96), gb, 2)
    lz = w["n"][2] * w["dx"][2]
    doppler = gb * (1 + np.sqrt(1 - 1 / gb ** 2))
    laser = (2.0, 1.0, 20.0, 2.0, 0.5 * lz / doppler)
    g, o = pair(3, w["n"], (1, 1, 1), w["dx"], w["dt"], gb, FP32, passes=3, absorb=4)
    load(g, o, gb, laser, w["plasma"])
    report = {}
    for block, step in ((10, 10), (40, 50), (50, 100)):
        g.step(block)
        o.step(block)
        if step not in (50, 100):
            continue
        errs = {}
        for c in COMPS + JCOMPS:
            errs[NAMES[c]] = rel2(g.get_field(c), o.get_field(c))
        pg, po = g.get_particles(), o.get_particles()
        # a particle at the -z face may leave in one precision and not yet in the other
        common, ig, io = np.intersect1d(pg["id"], po["id"], return_indices=True)
        assert max(pg["id"].size, po["id"].size) - common.size <= 1e-4 * po["id"].size
        errs["u"] = rel2(pg["u"][ig], po["u"][io])
        print(f"gamma_b {gb}: FP32 vs FP64 oracle after {step} steps (normwise) "
              + " ".join(f"{k} {v:.2e}" for k, v in errs.items()))
        report[step] = errs
    for step, errs in report.items():
        bar = 3e-5 if (gb == 100.0 and step == 50) else 1e-5
        for k, v in errs.items():
            assert v <= bar, (step, k, v)
