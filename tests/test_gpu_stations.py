"""Lab-frame stations on the GPU against the oracle's station records (FP64 to 1e-12,
FP32 to 1e-5), and the lab pulse's history recovered at a lab station."""
import math

import numpy as np
import pytest

import oracle
import paper_0909_5603_gb300 as pic

pytestmark = pytest.mark.gpu

FP32, FP64 = pic.PIC_PREC_FP32, pic.PIC_PREC_FP64


@pytest.fixture(scope="module", autouse=True)
def built():
    pic.build()
    oracle.build()


@pytest.mark.parametrize("prec,tol", [(FP64, 1e-12), (FP32, 1e-5)])
@pytest.mark.parametrize("ndim,bcz", [(3, 1), (2, 0)])
def test_station_histories_match_oracle(ndim, bcz, prec, tol):
    gb = 5.0
    n = (12, 8, 48) if ndim == 3 else (24, 1, 64)
    dz, dt = 0.5, 0.2
    bc = (1, 0, bcz)
    laser = (1.0, 1.0, 4.0, 1.0, 1.0)
    plasma = (0.5, 0.5, 3.0, 2, (0.01, 0.01, 0.01), 4)
    g = pic.Simulation(ndim, n, bc, (1.0, 1.0, dz), dt, gamma_boost=gb, order=2, precision=prec, filter_passes=1,
                       absorb_cells=4)
    o = oracle.Sim(ndim, n, bc, (1.0, 1.0, dz), dt, order=2, filter_passes=1, absorb_cells=4,
                   tile=(8, 8, 8) if ndim == 3 else (16, 1, 16))
    z_lab = [40.0, 60.0, 90.0, 1e4]  # the last never enters the box
    g.set_stations(z_lab, 64)
    g.load_lab_frame(laser=laser, plasma=plasma)
    o.load_lab_frame(gb, laser=laser, plasma=[*plasma[:4], *plasma[4], plasma[5]])
    ref = {i: [] for i in range(len(z_lab))}
    for step in range(25):
        for i, z in enumerate(z_lab):
            r = o.station_record(gb, z)
            if r is not None:
                ref[i].append(r)
        g.step(1)
        o.step(1)
    for i, z in enumerate(z_lab):
        r = o.station_record(gb, z)
        if r is not None:
            ref[i].append(r)
    for i in range(len(z_lab)):
        t, f = g.station(i)
        assert len(t) == len(ref[i]), (i, len(t), len(ref[i]))
        if not ref[i]:
            continue
        t_ref = np.array([r[0] for r in ref[i]])
        f_ref = np.stack([r[1] for r in ref[i]])
        assert np.abs(t - t_ref).max() <= 1e-12 * np.abs(t_ref).max()
        scale = np.abs(f_ref).max()
        err = np.linalg.norm(f - f_ref) / np.linalg.norm(f_ref) if prec == FP32 else np.abs(f - f_ref).max() / scale
        assert err <= tol, (i, err)
    assert sum(len(v) for v in ref.values()) > 20


def test_lab_pulse_history_at_a_gpu_station():
    gb = 4.0
    b = math.sqrt(1 - 1 / gb ** 2)
    dz = gb * (1 + b) / 32.0
    dt = 0.5 * dz
    a0, L, zc = 0.5, 1.5, 5.0
    g = pic.Simulation(2, (16, 1, 512), (0, 0, 1), (1.0, 1.0, dz), dt, gamma_boost=gb, order=1, precision=FP32,
                       absorb_cells=8)
    Z = 320.0
    g.set_stations([Z], 400)
    g.load_lab_frame(laser=(a0, 1.0, 1e6, L, zc))
    g.step(300)
    t, f = g.station(0)
    assert t.min() < Z - zc - 2 * L and t.max() > Z - zc + 2 * L
    xi = Z - zc - t
    k0 = 2 * math.pi
    expect = a0 * k0 * np.exp(-(xi / L) ** 2) * np.cos(k0 * xi)
    assert np.abs(f[:, 0, 0, 0] - expect).max() < 0.05 * a0 * k0
    assert np.abs(f[:, 4, 0, 0] - f[:, 0, 0, 0]).max() < 0.05 * a0 * k0
