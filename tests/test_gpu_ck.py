"""The low-dispersion field solver on the GPU (pic_options.solver = PIC_SOLVER_CK) against
the oracle, at time steps beyond the Yee Courant limit, and its dispersion-free axis wave."""
import math

import numpy as np
import pytest

import oracle
import paper_0909_5603_gb300 as pic
import synth

pytestmark = pytest.mark.gpu

FP32, FP64 = pic.PIC_PREC_FP32, pic.PIC_PREC_FP64
CK = pic.PIC_SOLVER_CK
COMPS = [pic.PIC_EX, pic.PIC_EY, pic.PIC_EZ, pic.PIC_BX, pic.PIC_BY, pic.PIC_BZ]


@pytest.fixture(scope="module", autouse=True)
def built():
    pic.build()
    oracle.build()


def relinf(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300))


CASES = [(3, (20, 16, 24), (0, 0, 0), (1.0, 0.9, 1.1)), (3, (20, 16, 24), (1, 0, 1), (1.0, 0.9, 1.1)),
         (2, (36, 1, 44), (0, 0, 0), (1.0, 1.0, 0.8)), (2, (36, 1, 44), (1, 0, 1), (1.0, 1.0, 0.8))]


@pytest.mark.parametrize("prec,tol", [(FP64, 1e-13), (FP32, 2e-6)])
@pytest.mark.parametrize("ndim,n,bc,dx", CASES)
def test_ck_maxwell_phase(ndim, n, bc, dx, prec, tol):
    dt = 0.95 * min(dx[a] for a in (0, 1, 2) if ndim == 3 or a != 1)  # beyond the Yee limit
    g = pic.Simulation(ndim, n, bc, dx, dt, order=1, precision=prec, solver=CK, absorb_cells=4)
    o = oracle.Sim(ndim, n, bc, dx, dt, order=1, solver=oracle.SOLVER_CK, absorb_cells=4,
                   tile=(8, 8, 8) if ndim == 3 else (16, 1, 16))
    g.load_particles(np.zeros(0, np.int32), np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0))
    for c, f in zip(COMPS, synth.smooth_fields(n, ndim, 1.0, seed=71, modes=4)):
        g.set_field(c, f)
        o.set_field(c, f)
    for _ in range(6):
        g.run_phases(pic.PIC_PHASE_MAXWELL)
        o.maxwell()
    for c in COMPS:
        fo = o.get_field(c)
        if np.abs(fo).max() > 0:
            assert relinf(g.get_field(c), fo) <= tol, c


def test_ck_full_steps_with_plasma_fp64():
    gb = 5.0
    n = (12, 8, 48)
    dz = 0.5
    dt = 0.9 * dz
    g = pic.Simulation(3, n, (1, 0, 1), (1.0, 1.0, dz), dt, gamma_boost=gb, order=2, precision=FP64,
                       filter_passes=1, absorb_cells=4, solver=CK)
    o = oracle.Sim(3, n, (1, 0, 1), (1.0, 1.0, dz), dt, order=2, filter_passes=1, absorb_cells=4,
                   solver=oracle.SOLVER_CK)
    laser = (1.0, 1.0, 4.0, 1.0, 1.0)
    plasma = (0.5, 0.5, 3.0, 2, (0.01, 0.01, 0.01), 4)
    g.load_lab_frame(laser=laser, plasma=plasma)
    o.load_lab_frame(gb, laser=laser, plasma=[*plasma[:4], *plasma[4], plasma[5]])
    g.step(10)
    o.step(10)
    for c in COMPS:
        assert relinf(g.get_field(c), o.get_field(c)) <= 1e-12, c
    pg, po = g.get_particles(), o.get_particles()
    assert np.array_equal(pg["cell"], po["cell"])
    assert relinf(pg["u"], po["u"]) <= 1e-12


def test_ck_axis_wave_dispersion_free_on_gpu():
    dx = (1.5, 1.3, 1.0)
    n = (8, 8, 24)
    g = pic.Simulation(3, n, (0, 0, 0), dx, dx[2], order=1, precision=FP64, solver=CK)
    g.load_particles(np.zeros(0, np.int32), np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0))
    k = 2 * math.pi * 5 / (n[2] * dx[2])
    z = np.broadcast_to(np.arange(n[2])[:, None, None] * dx[2], (n[2], n[1], n[0]))
    g.set_field(pic.PIC_EX, np.cos(k * z))
    steps = 37
    for _ in range(steps):
        g.run_phases(pic.PIC_PHASE_MAXWELL)
    assert np.abs(g.get_field(pic.PIC_EX) - np.cos(k * z) * math.cos(k * dx[2] * steps)).max() < 1e-12
