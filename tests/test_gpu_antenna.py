"""The laser antenna on a lab-fixed plane (Sec. 2 of Vay et al.) on the GPU against the
oracle, under the Yee and the low-dispersion (CK) field solvers: the moving
total-field/scattered-field boundary in 2D3V (fields only) and in 3D with a lab-frame
plasma and full steps, FP64 within 1e-12 and FP32 within 1e-5 (normwise); a plane wave
crosses the moving boundary without reflection on the GPU too (zero behind the plane,
the loaded free pulse ahead of it; under CK at dt = 0.9 dz); an antenna set in mid-run; a
batch member with an antenna steps as alone; the setter's argument checks."""
import math

import numpy as np
import pytest

import oracle
import paper_0909_5603_gb300 as pic

pytestmark = pytest.mark.gpu

FP32, FP64 = pic.PIC_PREC_FP32, pic.PIC_PREC_FP64
FIELDS = [pic.PIC_EX, pic.PIC_EY, pic.PIC_EZ, pic.PIC_BX, pic.PIC_BY, pic.PIC_BZ]
GB = 4.0
B = math.sqrt(1 - 1 / GB ** 2)
D = GB * (1 + B)


@pytest.fixture(scope="module", autouse=True)
def built():
    pic.build()
    oracle.build()


def rel2(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def relinf(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300))


YEE, CK = pic.PIC_SOLVER_YEE, pic.PIC_SOLVER_CK


def empty_pair(n, dz, dt, prec, tile=(16, 1, 16), bc=(0, 0, 1), solver=YEE):
    g = pic.Simulation(2, n, bc, (1.0, 1.0, dz), dt, gamma_boost=GB, order=1, precision=prec,
                       absorb_cells=8, tile=tile, solver=solver)
    o = oracle.Sim(2, n, bc, (1.0, 1.0, dz), dt, order=1, absorb_cells=8, tile=tile, solver=solver)
    none = (np.zeros(0, np.int32), np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0))
    g.load_particles(*none)
    o.set_particles(*none)
    return g, o


# 16 boosted wavelengths at 32 cells; the pulse starts 7.6 wavelengths in, the plane at 14
N2D = (16, 1, 512)
DZ2D = D / 32
LASER2D = (0.5, 1.0, 6.0, 1.5, 7.6)
ZLAB2D = 14 * GB * D


@pytest.mark.parametrize("solver", [YEE, CK], ids=["yee", "ck"])
@pytest.mark.parametrize("prec,tol", [(FP64, 1e-12), (FP32, 1e-5)])
def test_antenna_fields_match_oracle_2d(prec, tol, solver):
    dt = 0.5 * DZ2D if solver == YEE else 0.9 * DZ2D
    g, o = empty_pair(N2D, DZ2D, dt, prec, solver=solver)
    g.set_antenna(LASER2D, ZLAB2D)
    o.set_antenna(GB, LASER2D, ZLAB2D)
    for chunk in (1, 149, 150):
        for _ in range(chunk):
            g.run_phases(pic.PIC_PHASE_MAXWELL)
            o.maxwell()
        for c in FIELDS:
            fo = o.get_field(c)
            if np.abs(fo).max() == 0:
                assert np.abs(g.get_field(c)).max() == 0, c
                continue
            err = relinf(g.get_field(c), fo) if prec == FP64 else rel2(g.get_field(c), fo)
            assert err <= tol, (chunk, c, err)


@pytest.mark.parametrize("solver,cfl", [(YEE, 0.5), (CK, 0.9)], ids=["yee", "ck"])
def test_plane_wave_without_reflection_on_gpu(solver, cfl):
    """Transversely uniform pulse (waist 1e9): behind the plane the field stays zero, ahead
    of it it equals the same lab pulse loaded whole and propagated (FP64), at dt = cfl dz
    (under the low-dispersion solver above the Yee scheme's Courant limit)."""
    laser = (0.5, 1.0, 1e9, 1.5, 7.6)
    n = (8, 1, 768)
    dt = cfl * DZ2D
    a, _ = empty_pair(n, DZ2D, dt, FP64, tile=(8, 1, 16), solver=solver)
    a.set_antenna(laser, ZLAB2D)
    f = pic.Simulation(2, n, (0, 0, 1), (1.0, 1.0, DZ2D), dt, gamma_boost=GB, order=1, precision=FP64,
                       absorb_cells=8, tile=(8, 1, 16), solver=solver)
    f.load_lab_frame(laser=laser)
    steps = int(450 * 0.5 / cfl)
    for _ in range(steps):
        a.run_phases(pic.PIC_PHASE_MAXWELL)
        f.run_phases(pic.PIC_PHASE_MAXWELL)
    zp = (ZLAB2D / GB - B * steps * dt) / DZ2D
    k = np.arange(n[2])
    amp = np.abs(f.get_field(pic.PIC_EX)).max()
    for c, half in ((pic.PIC_EX, 0.0), (pic.PIC_BY, 0.5)):
        fa, ff = a.get_field(c)[:, 0, 0], f.get_field(c)[:, 0, 0]
        pos = k + half
        assert np.abs(fa[pos <= zp]).max() < 1e-12 * amp, c
        assert np.abs(fa[pos > zp] - ff[pos > zp]).max() < 1e-10 * amp, c


N3D = (12, 12, 96)
DZ3D = D / 16
LASER3D = (1.0, 1.0, 4.0, 0.5, 2.5)
ZLAB3D = 4 * GB * D
PLASMA = (0.05, 0.5, 3.0, 2, (0.01, 0.01, 0.01), 4)


def pair3d(prec, solver=YEE):
    dt = 0.5 * DZ3D if solver == YEE else 0.9 * DZ3D
    g = pic.Simulation(3, N3D, (1, 1, 1), (1.0, 1.0, DZ3D), dt, gamma_boost=GB, order=2, precision=prec,
                       filter_passes=1, absorb_cells=4, solver=solver)
    o = oracle.Sim(3, N3D, (1, 1, 1), (1.0, 1.0, DZ3D), dt, order=2, filter_passes=1, absorb_cells=4,
                   tile=(8, 8, 8), solver=solver)
    g.load_lab_frame(plasma=PLASMA)
    o.load_lab_frame(GB, plasma=[*PLASMA[:4], *PLASMA[4], PLASMA[5]])
    g.set_antenna(LASER3D, ZLAB3D)
    o.set_antenna(GB, LASER3D, ZLAB3D)
    return g, o


@pytest.mark.parametrize("solver", [YEE, CK], ids=["yee", "ck"])
@pytest.mark.parametrize("prec,tol", [(FP64, 1e-12), (FP32, 1e-5)])
def test_antenna_with_plasma_full_steps_3d(prec, tol, solver):
    g, o = pair3d(prec, solver)
    g.step(40)
    o.step(40)
    for c in FIELDS + [pic.PIC_JX, pic.PIC_JY, pic.PIC_JZ]:
        fo = o.get_field(c)
        err = relinf(g.get_field(c), fo) if prec == FP64 else rel2(g.get_field(c), fo)
        assert err <= tol, (c, err)
    pg, po = g.get_particles(), o.get_particles()
    if prec == FP64:
        assert np.array_equal(pg["cell"], po["cell"])
        assert relinf(pg["u"], po["u"]) <= tol
    else:
        common, ig, io = np.intersect1d(pg["id"], po["id"], return_indices=True)
        assert max(pg["id"].size, po["id"].size) - common.size <= 2
        assert rel2(pg["u"][ig], po["u"][io]) <= tol
    # the laser has been emitted into the plasma: a transverse field well above the wake's
    assert np.abs(o.get_field(pic.PIC_EX)).max() > 0.02


def test_antenna_set_in_mid_run_fp64():
    g, o = empty_pair(N2D, DZ2D, 0.5 * DZ2D, FP64)
    for _ in range(37):
        g.run_phases(pic.PIC_PHASE_MAXWELL)
        o.maxwell()
    g.set_antenna(LASER2D, ZLAB2D)
    o.set_antenna(GB, LASER2D, ZLAB2D)
    for _ in range(120):
        g.run_phases(pic.PIC_PHASE_MAXWELL)
        o.maxwell()
    for c in (pic.PIC_EX, pic.PIC_BY, pic.PIC_EZ, pic.PIC_BZ):
        assert relinf(g.get_field(c), o.get_field(c)) <= 1e-12, c


def test_batch_member_with_antenna_steps_as_alone():
    alone, _ = pair3d(FP64)
    member, _ = pair3d(FP64)
    other, _ = pair3d(FP64)
    other.set_antenna(None)
    alone.step(12)
    batch = pic.Batch([member, other])
    batch.step(12)
    batch.synchronize()
    for c in FIELDS:
        fa, fb = alone.get_field(c), member.get_field(c)
        assert np.abs(fa - fb).max() <= 1e-12 * max(np.abs(fa).max(), 1e-300), c
    assert np.abs(alone.get_field(pic.PIC_EX) - other.get_field(pic.PIC_EX)).max() > 0


def test_set_antenna_argument_checks():
    per = pic.Simulation(2, (16, 1, 64), (1, 0, 0), (1.0, 1.0, 0.5), 0.2, gamma_boost=2.0)
    per.load_particles(np.zeros(0, np.int32), np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0))
    with pytest.raises(pic.PicError):
        per.set_antenna(LASER2D, 10.0)  # periodic z
    ck = pic.Simulation(2, (16, 1, 64), (1, 0, 1), (1.0, 1.0, 0.5), 0.2, gamma_boost=2.0,
                        solver=pic.PIC_SOLVER_CK)
    ck.load_particles(np.zeros(0, np.int32), np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0))
    ck.set_antenna(LASER2D, 10.0)  # the low-dispersion solver takes an antenna too
    fresh = pic.Simulation(2, (16, 1, 64), (1, 0, 1), (1.0, 1.0, 0.5), 0.2, gamma_boost=2.0)
    with pytest.raises(pic.PicError):
        fresh.set_antenna(LASER2D, 10.0)  # nothing loaded
    fresh.load_particles(np.zeros(0, np.int32), np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0))
    with pytest.raises(pic.PicError):
        fresh.set_antenna((0.5, -1.0, 6.0, 1.5, 7.6), 10.0)  # negative wavelength
    fresh.set_antenna(LASER2D, 10.0)
    fresh.set_antenna(None)
