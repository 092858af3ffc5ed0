"""The GPU pushers inside the fused particle kernel against closed forms, at the single-
particle level of the rigid-beam test (Sec. 2 of Vay et al.: Boris's inexact E + v x B
cancellation at large gamma, cured by the Vay pusher).

Particles sit in a periodic box with uniform fields set on every Yee component; only the
particle phase runs (gather + push + move + deposit), so the deposit never feeds back.
FP32 storage with the FP64 gamma solve unless stated.
"""
import math

import numpy as np
import pytest

import paper_0909_5603_gb300 as pic

pytestmark = pytest.mark.gpu

FP32, FP64 = pic.PIC_PREC_FP32, pic.PIC_PREC_FP64


def box(prec, pusher, dt=0.5, n=(16, 16, 16)):
    s = pic.Simulation(3, n, (0, 0, 0), (1.0, 1.0, 1.0), dt, order=2, precision=prec, pusher=pusher)
    return s


def uniform(s, E, B):
    shape = (s.n[2], s.n[1], s.n[0])
    for c, v in zip((pic.PIC_EX, pic.PIC_EY, pic.PIC_EZ, pic.PIC_BX, pic.PIC_BY, pic.PIC_BZ), list(E) + list(B)):
        s.set_field(c, np.full(shape, float(v)))


def load(s, u):
    u = np.asarray(u, np.float64)
    npart = u.shape[0]
    cell = (np.arange(npart) * 37 % (s.ncell)).astype(np.int32)
    off = np.full((npart, 3), 0.5)
    w = np.full(npart, 1e-9)  # negligible current
    s.load_particles(cell, off, u, w, np.arange(npart, dtype=np.int32))


def momenta(s):
    p = s.get_particles()
    return p["u"][np.argsort(p["id"])]


@pytest.mark.parametrize("prec,tol", [(FP32, 2e-7), (FP64, 1e-14)])
def test_force_free_vay_vs_boris_up_to_gamma_1e4(prec, tol):
    """E = -v x B: Vay leaves u unchanged at every gamma (to the storage precision; here
    tau^2 << gamma'^2, so FP32 mode forms sigma in FP32); Boris leaves the kick
    h^3 B^3 beta^2 / gamma^2."""
    gammas = np.array([10.0, 100.0, 1e3, 1e4])
    uz = np.sqrt(gammas ** 2 - 1)
    beta = uz / gammas
    Bm = 0.7
    res = {}
    for pusher in (pic.PIC_PUSHER_VAY, pic.PIC_PUSHER_BORIS):
        kicks = []
        for g, u, b in zip(gammas, uz, beta):
            s = box(prec, pusher)
            uniform(s, (b * Bm, 0.0, 0.0), (0.0, Bm, 0.0))  # E = -v x B for v = b z
            load(s, [[0.0, 0.0, u]])
            s.run_phases(pic.PIC_PHASE_PARTICLES)
            un = momenta(s)[0]
            kicks.append(un - np.array([0.0, 0.0, u]))
        res[pusher] = np.array(kicks)
    vay, bor = res[pic.PIC_PUSHER_VAY], res[pic.PIC_PUSHER_BORIS]
    assert np.all(np.abs(vay).max(axis=1) <= tol * uz)
    h = 0.5 * (-1.0) * 0.5
    expect = h ** 3 * Bm ** 3 * beta ** 2 / gammas ** 2
    if prec == FP64:
        assert np.all(np.abs(bor[:, 0] - expect) <= 0.02 * np.abs(expect))
    else:  # FP32 resolves the Boris kick at gamma 10 (5e-5); above, it drops below an ulp of u
        assert abs(bor[0, 0] - expect[0]) <= 0.05 * abs(expect[0])


@pytest.mark.parametrize("pusher", [pic.PIC_PUSHER_VAY, pic.PIC_PUSHER_BORIS])
def test_uniform_B_rotation_angle(pusher):
    B = np.array([0.0, 0.0, 1.1])
    u0 = np.array([[0.8, 0.0, 0.3], [5.0, 0.0, -2.0], [40.0, 0.0, 10.0]])
    s = box(FP32, pusher, dt=0.4)
    uniform(s, (0, 0, 0), B)
    load(s, u0)
    nsteps = 25
    for _ in range(nsteps):
        s.run_phases(pic.PIC_PHASE_PARTICLES)
    u = momenta(s)
    for k in range(3):
        g = math.sqrt(1 + u0[k] @ u0[k])
        t = 0.5 * 0.4 * 1.1 / g
        theta = nsteps * 2 * math.atan(t)
        ang0 = math.atan2(u0[k, 1], u0[k, 0])
        ang = math.atan2(u[k, 1], u[k, 0])
        # electrons (q < 0) rotate counter-clockwise about +B
        assert abs(math.remainder(ang - ang0 - theta, 2 * math.pi)) < 2e-5
        assert abs(np.linalg.norm(u[k, :2]) - np.linalg.norm(u0[k, :2])) < 2e-6 * np.linalg.norm(u0[k])
        assert abs(u[k, 2] - u0[k, 2]) < 2e-6 * np.linalg.norm(u0[k])


@pytest.mark.parametrize("pusher", [pic.PIC_PUSHER_VAY, pic.PIC_PUSHER_BORIS])
def test_uniform_E_acceleration(pusher):
    """u parallel to E: u grows by q E dt per step exactly (FP32 rounding only)."""
    E = 0.05
    u0 = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 50.0], [0.0, 0.0, 5000.0]])
    s = box(FP32, pusher)
    uniform(s, (0, 0, E), (0, 0, 0))
    load(s, u0)
    for _ in range(10):
        s.run_phases(pic.PIC_PHASE_PARTICLES)
    u = momenta(s)
    expect = u0[:, 2] + 10 * (-1.0) * E * 0.5
    assert np.all(np.abs(u[:, 2] - expect) <= 1e-6 * np.maximum(1.0, np.abs(expect)))


def test_exb_drift_gpu():
    """Average velocity over whole relativistic gyro-periods equals E x B / B^2."""
    E = np.array([0.05, 0.0, 0.0])
    B = np.array([0.0, 0.0, 1.0])
    vd = np.cross(E, B) / (B @ B)
    gd = 1 / math.sqrt(1 - vd @ vd)
    dt = 0.05
    nsteps = int(round(2 * 2 * math.pi * gd ** 3 / dt))
    s = pic.Simulation(3, (16, 16, 16), (0, 0, 0), (1.0, 1.0, 1.0), dt, order=1, precision=FP64)
    uniform(s, E, B)
    load(s, [[0.0, 0.0, 0.0]])
    p0 = s.get_particles()
    for _ in range(nsteps):
        s.run_phases(pic.PIC_PHASE_PARTICLES)
    p1 = s.get_particles()
    n = 16
    def pos(p):
        c = p["cell"][0]
        return np.array([c % n, (c // n) % n, c // (n * n)]) + p["off"][0]
    d = pos(p1) - pos(p0)
    d -= np.round(d / n) * n
    vmean = d / (nsteps * dt)
    assert np.linalg.norm(vmean - vd) < 5e-3 * np.linalg.norm(vd)


def test_vay_cancelling_sigma_fp32_matches_fp64_solve():
    """sigma = gamma'^2 - tau^2 cancels when |h B| ~ gamma': FP32 mode takes the FP64
    difference there (one warp vote: any particle with tau^2 >= gamma'^2 / 4).  A warp of
    particles around tau^2 = gamma'^2 (ratios 0.25 .. 4) in a uniform strong B: one push
    in FP32 storage against the FP64 Vay push of the same FP32 inputs (the oracle's),
    within 2e-6 of |u| (a 90-degree rotation per step, a few dozen FP32 operations)."""
    import oracle
    oracle.build()
    Bm = 400.0  # tau = h B = -100 at dt = 0.5, q/m = -1
    ratios = np.geomspace(0.25, 4.0, 32)
    uz = np.float32(100.0 * np.sqrt(ratios)).astype(np.float64)  # gamma'^2 ~ uz^2 vs tau^2 = 1e4
    u0 = np.stack([np.zeros_like(uz), 0.3 * uz, uz], axis=1).astype(np.float32).astype(np.float64)
    s = box(FP32, pic.PIC_PUSHER_VAY)
    uniform(s, (0.0, 0.0, 0.0), (Bm, 0.0, 0.0))
    load(s, u0)
    s.run_phases(pic.PIC_PHASE_PARTICLES)
    got = momenta(s)
    for k in range(len(uz)):
        ref = np.array(oracle.push_vay(u0[k].copy(), np.zeros(3), np.array([Bm, 0.0, 0.0]), -1.0, 0.5))
        assert np.abs(got[k] - ref).max() <= 2e-6 * np.linalg.norm(ref), (k, got[k], ref)
