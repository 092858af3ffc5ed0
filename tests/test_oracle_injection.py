"""Pins of the oracle's beam injection through a lab-fixed plane (Sec. 2 of Vay et al.:
the beam enters the boosted frame through a transverse plane fixed in the laboratory and
drifting in the boosted frame; the part still upstream is carried by frozen, drifting
macro-particles).

Every expectation below comes from laboratory-frame kinematics and the Lorentz
transformation, not from the freezing rule itself:

* A test particle drifting freely in the lab until it crosses the plane z_lab, then
  accelerated by a uniform longitudinal field (E_z is the same in both frames): in the
  boosted frame its momentum stays exactly constant until the boosted time of the lab
  crossing event, t'_c = gamma_b (t_c - beta_b z_lab), and then grows by q E dt per step.
  The first active step is the first n with n dt >= t'_c.
* The same with a uniform transverse lab field E_x (boosted: E'_x and B'_y): the record
  transformed back to the lab matches the lab solution u_x = q E_x (t - t_c),
  u_z = const, to the activation step's half-step uncertainty.
* A lab-frame beam loaded with the plane: the number of frozen particles at step n is
  the number whose lab crossing event has t'_c > n dt, computed from the beam's lab
  draws (ballistic lab motion from t = 0); frozen particles keep their momenta bit for
  bit; plasma particles are never frozen.
* Frozen particles still deposit their current: div E - rho stays at its initial value.
* Only particles with id >= first_id are frozen.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import EX, EZ, BY


def beta(g):
    return math.sqrt(1 - 1 / g ** 2)


def lab_to_boosted(gb, t, z, u):
    """Event (t, z) and momentum u = (ux, uy, uz) of the lab frame, seen from the frame
    moving at +beta_b along z."""
    b = beta(gb)
    g = math.sqrt(1 + sum(v * v for v in u))
    return gb * (t - b * z), gb * (z - b * t), (u[0], u[1], gb * (u[2] - b * g))


def boosted_to_lab(gb, tp, zp, up):
    b = beta(gb)
    gp = math.sqrt(1 + sum(v * v for v in up))
    return gb * (tp + b * zp), gb * (zp + b * tp), (up[0], up[1], gb * (up[2] + b * gp))


def one_particle(gb, zp0, u_lab, fields, z_lab, steps, dt=0.1, dz=0.25, first_id=0):
    """A zero-weight particle at boosted z'(0) = zp0 with lab momentum u_lab in uniform
    boosted fields; returns the per-step (t'_n, z'_n, u'^{n-1/2}) history."""
    n = (4, 1, 256)
    s = oracle.Sim(2, n, (0, 0, 0), (1.0, 1.0, dz), dt, order=1, tile=(4, 1, 16))
    for c, v in fields.items():
        s.set_field(c, np.full((n[2], n[1], n[0]), v))
    _, _, up = lab_to_boosted(gb, 0.0, 0.0, u_lab)
    k = int(zp0 // dz)
    s.set_particles(np.array([2 + n[0] * k], np.int32), np.array([[0.5, 0.0, zp0 / dz - k]]), np.array([up]),
                    np.zeros(1))
    s.set_injection(gb, z_lab, first_id)
    hist = []
    for step in range(steps):
        s.step(1)
        p = s.get_particles()
        z = (p["cell"][0] // n[0] + p["off"][0, 2]) * dz
        hist.append(((step + 1) * dt, z, p["u"][0].copy()))
    return hist, up


def lab_crossing(gb, zp0, u_lab, z_lab):
    """Lab crossing of the plane by the lab worldline through the boosted event (0, zp0)."""
    b = beta(gb)
    t_e, z_e = gb * b * zp0, gb * zp0  # the event (t' = 0, z' = zp0) in the lab
    g = math.sqrt(1 + sum(v * v for v in u_lab))
    t_c = t_e + (z_lab - z_e) / (u_lab[2] / g)
    return t_c, gb * (t_c - b * z_lab)


def test_longitudinal_field_acts_from_the_lab_crossing_on():
    gb, E0, dt = 4.0, 0.05, 0.1
    u_lab = (0.0, 0.0, math.sqrt(10.0 ** 2 - 1))
    zp0, z_lab = 10.0, 80.0  # the plane starts at z' = 20 and moves to -z
    q = -1.0
    steps = 150
    hist, up0 = one_particle(gb, zp0, u_lab, {EZ: E0}, z_lab, steps, dt=dt)
    _, tpc = lab_crossing(gb, zp0, u_lab, z_lab)
    assert 3.0 < tpc < 0.8 * steps * dt
    n_a = math.ceil(tpc / dt)  # first step with t^n >= t'_c
    for i, (_, _, u) in enumerate(hist):  # hist[i]: after phase i (pushed at t^i = i dt)
        active = max(0, i + 1 - n_a)
        assert abs(u[2] - (up0[2] + q * E0 * dt * active)) < 1e-12 * (1 + abs(up0[2]))
        assert u[0] == 0.0 and u[1] == 0.0
    # the final momentum against the continuous boosted solution (u^{N-1/2})
    u_end = up0[2] + q * E0 * ((steps - 0.5) * dt - tpc)
    assert abs(hist[-1][2][2] - u_end) <= 0.5 * abs(q * E0) * dt + 1e-12
    # without the plane the particle would have gained q E0 t'_c more: far outside that
    assert abs(q * E0) * tpc > 10 * abs(q * E0) * dt


def test_frozen_particle_drifts_at_its_own_velocity():
    gb, dt = 4.0, 0.1
    u_lab = (0.0, 0.0, math.sqrt(10.0 ** 2 - 1))
    hist, up0 = one_particle(gb, 10.0, u_lab, {EZ: 0.05, EX: 0.02, BY: -0.03}, 80.0, 30, dt=dt)
    vz = up0[2] / math.sqrt(1 + up0[2] ** 2)
    for i, (t, z, u) in enumerate(hist):
        assert np.array_equal(u, np.array(up0))  # t'_c > 3: still frozen after 30 steps
        assert abs(z - (10.0 + vz * t)) < 1e-12


def test_transverse_lab_field_matches_lab_solution():
    gb, E1, dt = 4.0, 0.02, 0.05
    b = beta(gb)
    q = -1.0
    Ep, Bp = oracle.boost_fields(gb, [E1, 0.0, 0.0], [0.0, 0.0, 0.0])
    assert abs(Ep[0] - gb * E1) < 1e-15 and abs(Bp[1] + gb * b * E1) < 1e-15
    u_lab = (0.0, 0.0, math.sqrt(10.0 ** 2 - 1))
    zp0, z_lab, steps = 10.0, 80.0, 300
    hist, up0 = one_particle(gb, zp0, u_lab, {EX: Ep[0], BY: Bp[1]}, z_lab, steps, dt=dt)
    t_c, tpc = lab_crossing(gb, zp0, u_lab, z_lab)
    # u^{N-1/2} at t' = (N - 1/2) dt, position halfway between z'^{N-1} and z'^N
    tp = (steps - 0.5) * dt
    zp = 0.5 * (hist[-1][1] + hist[-2][1])
    t, _, u = boosted_to_lab(gb, tp, zp, tuple(hist[-1][2]))
    ux_lab = q * E1 * (t - t_c)
    assert abs(ux_lab) > 0.1  # a real transverse kick
    # activation within half a boosted step of t'_c: |du'_x/dt'| <= |q| gamma_b E1 (1 + b)
    tol = 0.5 * dt * abs(q) * gb * E1 * (1 + b) + 1e-3 * abs(ux_lab)
    assert abs(u[0] - ux_lab) < tol
    assert abs(u[2] - u_lab[2]) < 1e-3 * u_lab[2]
    # the same run without the plane is far from the lab solution
    s_free, _ = one_particle(gb, zp0, u_lab, {EX: Ep[0], BY: Bp[1]}, -1e9, steps, dt=dt)
    t2, _, u2 = boosted_to_lab(gb, tp, 0.5 * (s_free[-1][1] + s_free[-2][1]), tuple(s_free[-1][2]))
    assert abs(u2[0] - q * E1 * (t2 - t_c)) > 20 * tol


def beam_case(plasma, periodic=False):
    gb = 4.0
    n = (8, 8, 64)
    dz, dt = 0.5, 0.2
    bc = (0, 0, 0) if periodic else (1, 1, 1)
    s = oracle.Sim(3, n, bc, (1.0, 1.0, dz), dt, order=2, tile=(8, 8, 8), absorb_cells=4)
    beam = [400, 20.0, 0.01, 1.0, 0.3, 2.0, 1e-3, 5]
    s.load_lab_frame(gb, plasma=plasma, beam=beam)
    z_lab = 72.0  # at z' = 18 when t' = 0
    s.set_injection(gb, z_lab)
    return s, gb, beam, z_lab, dt, dz


def lab_crossings(gb, beam, z_lab):
    """t'_c of every beam particle from its lab draws (ballistic lab motion from t = 0)."""
    nb, gam, spread, _, sz, z0, _, seed = beam
    g0 = math.sqrt(gam * gam - 1)
    b = beta(gb)
    out = []
    for i in range(nb):
        z = z0 + sz * oracle.normal(seed, 14, i)
        u = [spread * g0 * oracle.normal(seed, 16, i), spread * g0 * oracle.normal(seed, 18, i),
             g0 + spread * g0 * oracle.normal(seed, 20, i)]
        g = math.sqrt(1 + sum(v * v for v in u))
        t_c = (z_lab - z) / (u[2] / g)
        out.append(gb * (t_c - b * z_lab))
    return np.array(out)


@pytest.mark.parametrize("with_plasma", [False, True])
def test_frozen_count_follows_lab_crossings(with_plasma):
    ppc = 1
    plasma = [1e-3, -1e9, 0.0, ppc, 0.0, 0.0, 0.0, 3] if with_plasma else None
    s, gb, beam, z_lab, dt, dz = beam_case(plasma)
    first = 8 * 8 * 64 * ppc if with_plasma else 0  # every plasma sample has weight
    tpc = lab_crossings(gb, beam, z_lab)
    p0 = s.get_particles()
    ids = p0["id"][p0["id"] >= first] - first
    assert len(ids) > 300  # most of the beam is in the box
    u0 = {int(i): u.copy() for i, u in zip(p0["id"], p0["u"])}
    seen_frozen = seen_active = 0
    for step in range(40):
        expect = int(np.sum(tpc[ids] > step * dt))
        assert s.num_frozen() == expect, step
        seen_frozen += expect > 0
        seen_active += expect < len(ids)
        s.step(1)
        p = s.get_particles()
        ids = p["id"][p["id"] >= first] - first  # absorbing faces may remove some
        # particles frozen through this step kept their momenta exactly
        for i, u in zip(p["id"], p["u"]):
            if i >= first and tpc[i - first] > step * dt:
                assert np.array_equal(u, u0[int(i)])
    assert seen_frozen > 10 and seen_active > 10


def test_gauss_law_holds_with_frozen_particles():
    plasma = [1e-3, -1e9, 0.0, 1, 0.01, 0.01, 0.01, 3]
    s, gb, beam, z_lab, dt, dz = beam_case(plasma, periodic=True)
    r0 = s.div_e() - s.rho()
    assert s.num_frozen() > 50
    scale = np.abs(s.rho()).max()
    for _ in range(20):
        s.step(1)
        assert np.abs(s.div_e() - s.rho() - r0).max() < 1e-11 * scale
    assert s.num_frozen() < 50  # the plane has passed most of the beam meanwhile


def test_only_ids_from_first_id_are_frozen():
    n = (4, 1, 64)
    s = oracle.Sim(2, n, (0, 0, 0), (1.0, 1.0, 0.5), 0.1, tile=(4, 1, 16))
    s.set_field(EZ, np.full((n[2], n[1], n[0]), 0.1))
    cell = np.array([1 + 4 * 10, 1 + 4 * 10], np.int32)
    off = np.array([[0.5, 0, 0.5], [0.5, 0, 0.5]])
    u = np.array([[0.0, 0.0, 1.0], [0.0, 0.0, 1.0]])
    s.set_particles(cell, off, u, np.zeros(2), ids=np.array([3, 4]))
    s.set_injection(2.0, 50.0, first_id=4)  # plane at z' = 25, both upstream
    assert s.num_frozen() == 1
    s.step(1)
    p = s.get_particles()
    by_id = {int(i): uu for i, uu in zip(p["id"], p["u"])}
    assert by_id[4][2] == 1.0
    assert abs(by_id[3][2] - (1.0 - 0.1 * 0.1)) < 1e-15
    s.set_injection(2.0, 50.0, enable=False)
    assert s.num_frozen() == 0
