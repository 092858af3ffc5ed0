"""Pins of the oracle's pushers and shape factors against closed forms.

Vay and Boris pushers: Sec. 2 of Vay et al. (arXiv:0909.5603) and its references
VayPOP08 / BorisICNSP.  Each test fixes a result that a dropped term, a wrong sign or a
swapped operand in the oracle would break.
"""
import math

import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("order", [1, 2])
def test_shape_partition_of_unity_and_first_moment(order):
    rng = np.random.default_rng(0)
    for x in rng.uniform(-5, 5, 200):
        nodes = np.arange(math.floor(x) - 3, math.floor(x) + 4)
        s = np.array([oracle.shape(order, x - i) for i in nodes])
        assert abs(s.sum() - 1.0) < 1e-15
        assert abs((s * nodes).sum() - x) < 1e-13
        # discrete second moment: f (1 - f) for the linear spline (f = x - floor x),
        # the constant 1/4 for the quadratic one
        f = x - math.floor(x)
        var = f * (1 - f) if order == 1 else 0.25
        assert abs((s * (nodes - x) ** 2).sum() - var) < 1e-13


def test_shape_values():
    assert oracle.shape(1, 0.0) == 1.0 and oracle.shape(1, 1.0) == 0.0 and oracle.shape(1, -0.5) == 0.5
    assert oracle.shape(2, 0.0) == 0.75
    assert oracle.shape(2, 0.5) == 0.5 and oracle.shape(2, -0.5) == 0.5
    assert oracle.shape(2, 1.5) == 0.0 and oracle.shape(2, 1.0) == 0.125


@pytest.mark.parametrize("push", [oracle.push_vay, oracle.push_boris])
def test_uniform_B_rotation(push):
    """Pure magnetic field: |u| and u_par conserved, u_perp rotates by 2 atan(|t|) per step
    with t = (q dt / 2m) B / gamma (exact for both schemes)."""
    B = np.array([0.3, -0.2, 1.1])
    bhat = B / np.linalg.norm(B)
    u0 = np.array([2.0, 1.0, -0.5])
    qm, dt = -1.0, 0.37
    gamma = math.sqrt(1 + u0 @ u0)
    t = abs(0.5 * qm * dt) * np.linalg.norm(B) / gamma
    theta = 2 * math.atan(t)
    u = u0.copy()
    upar0 = u0 @ bhat
    e1 = u0 - upar0 * bhat
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(bhat, e1)
    nsteps = 57
    for _ in range(nsteps):
        u = push(u, np.zeros(3), B, qm, dt)
    assert abs(np.linalg.norm(u) - np.linalg.norm(u0)) < 1e-13
    assert abs(u @ bhat - upar0) < 1e-13
    uperp = u - (u @ bhat) * bhat
    ang = math.atan2(uperp @ e2, uperp @ e1)
    # electrons (q < 0) rotate positively about B
    expect = math.remainder(nsteps * theta, 2 * math.pi)
    assert abs(math.remainder(ang - expect, 2 * math.pi)) < 1e-11


@pytest.mark.parametrize("push", [oracle.push_vay, oracle.push_boris])
def test_uniform_E_parallel(push):
    """u parallel to E, B = 0: u^{n+1/2} = u^{n-1/2} + q E dt exactly."""
    E = np.array([0.0, 0.0, 0.25])
    u = np.array([0.0, 0.0, 3.0])
    qm, dt = -1.0, 0.5
    for n in range(1, 41):
        u = push(u, E, np.zeros(3), qm, dt)
        assert abs(u[2] - (3.0 + qm * E[2] * dt * n)) < 1e-13
        assert u[0] == 0.0 and u[1] == 0.0


@pytest.mark.parametrize("gamma", [10.0, 100.0, 1e3, 1e4])
def test_force_free_E_equals_minus_v_cross_B(gamma):
    """E = -v x B: the Lorentz force vanishes.  Vay keeps u unchanged to round-off at any
    gamma.  Boris rotates with gamma^- = sqrt(gamma^2 + (hE)^2) instead of gamma, so it
    leaves a transverse kick whose leading order is h^3 B^3 beta^2 / gamma^2
    (h = q dt / 2m; angle mismatch 2 atan(hB/gamma) - 2 atan(hB/gamma^-)) -- Sec. 2."""
    uz = math.sqrt(gamma ** 2 - 1)
    beta = uz / gamma
    u = np.array([0.0, 0.0, uz])
    Bm = 0.7
    B = np.array([0.0, Bm, 0.0])
    E = -np.cross(u / gamma, B)
    qm, dt = -1.0, 0.5
    h = 0.5 * qm * dt
    uv = oracle.push_vay(u, E, B, qm, dt)
    ub = oracle.push_boris(u, E, B, qm, dt)
    assert np.linalg.norm(uv - u) <= 4e-16 * uz
    kick = h ** 3 * Bm ** 3 * beta ** 2 / gamma ** 2
    assert abs(ub[0] - kick) < 0.02 * abs(kick)


def test_boris_beam_error_grows_with_gamma():
    """Self-field of a beam of fixed rest-frame density: E_r = gamma E0, B_theta = beta E_r.
    The true transverse kick is q E_r dt / gamma^2; Boris's relative error grows as
    gamma^2 while Vay's stays at the level of its O(dt^2) truncation (Sec. 2)."""
    E0, qm, dt = 0.07, -1.0, 0.5
    rel_b, rel_v = [], []
    for gamma in [10.0, 100.0, 1e3]:
        uz = math.sqrt(gamma ** 2 - 1)
        beta = uz / gamma
        u = np.array([0.0, 0.0, uz])
        E = np.array([gamma * E0, 0.0, 0.0])
        B = np.array([0.0, beta * gamma * E0, 0.0])
        true = qm * gamma * E0 * dt / gamma ** 2
        rel_b.append(abs(oracle.push_boris(u, E, B, qm, dt)[0] - true) / abs(true))
        rel_v.append(abs(oracle.push_vay(u, E, B, qm, dt)[0] - true) / abs(true))
    assert rel_b[0] > 1e-4
    for a, b in zip(rel_b, rel_b[1:]):
        assert 50.0 < b / a < 200.0  # ~ gamma^2
    assert max(rel_v) < 1e-6


def test_exb_drift():
    """Crossed fields |E| < |B|, particle starting at rest: averaged over whole gyro-periods
    the velocity is the drift v_d = E x B / B^2.  Relativistically the lab-frame period is
    T = 2 pi gamma_d^3 m / (|q| B), gamma_d = 1 / sqrt(1 - v_d^2) (the orbit is a circle at
    speed v_d in the drift frame, where B' = B / gamma_d, seen time-dilated)."""
    E = np.array([0.05, 0.0, 0.0])
    B = np.array([0.0, 0.0, 1.0])
    vd = np.cross(E, B) / (B @ B)
    gd = 1.0 / math.sqrt(1.0 - vd @ vd)
    T = 2 * math.pi * gd ** 3
    qm, dt = -1.0, 0.01
    for push in (oracle.push_vay, oracle.push_boris):
        u = np.zeros(3)
        vsum = np.zeros(3)
        nsteps = int(round(10 * T / dt))
        for _ in range(nsteps):
            u = push(u, E, B, qm, dt)
            vsum += u / math.sqrt(1 + u @ u)
        vmean = vsum / nsteps
        assert np.linalg.norm(vmean - vd) < 5e-4 * np.linalg.norm(vd)


def test_uniform_E_trajectory_closed_form():
    """Relativistic acceleration in uniform E from rest: with leapfrog positions the
    displacement converges to (sqrt(1 + (qEt)^2) - 1)/(qE) at O(dt^2)."""
    qE = -0.2 * -1.0  # q = -1, E = -0.2 along z -> force +0.2
    T = 20.0
    errs = []
    for dt in (0.1, 0.05):
        u = np.zeros(3)
        # start at u^{-1/2} = -qE dt/2 so that u^{n+1/2} is time-centred
        u[2] = -qE * dt / 2
        z = 0.0
        n = int(round(T / dt))
        for _ in range(n):
            u = oracle.push_vay(u, np.array([0, 0, -0.2]), np.zeros(3), -1.0, dt)
            z += dt * u[2] / math.sqrt(1 + u @ u)
        exact = (math.sqrt(1 + (qE * T) ** 2) - 1) / qE
        errs.append(abs(z - exact))
    assert errs[0] < 1e-2 and errs[1] < errs[0] / 3.0  # second order


def test_splitmix64_known_answer():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_seed0.txt")
    gamma = 0x9E3779B97F4A7C15
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    for k, val in rows:
        k = int(k)
        ctr = ((k - 1) * gamma) % (1 << 64)
        assert oracle.splitmix64(0, 0, ctr) == int(val, 16)


def test_uniform_and_normal_moments():
    u = np.array([oracle.uniform(7, 2, i) for i in range(20000)])
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.01 and abs(u.var() - 1 / 12) < 0.003
    g = np.array([oracle.normal(7, 3, i) for i in range(20000)])
    assert abs(g.mean()) < 0.03 and abs(g.std() - 1.0) < 0.02
