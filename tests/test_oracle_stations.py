"""Pins of the oracle's lab-frame stations (Sec. 2 of Vay et al.: results are recorded at
planes immobile in the laboratory frame, interpolating between the boosted grid's planes,
and transformed back to the laboratory frame).

* Uniform boosted fields: the record is their inverse Lorentz transform -- boosting it
  forward again with the (separately pinned) field transform gives the fields back.
* A field linear in z: the record samples it at the plane's boosted position; the event
  (record time, station position) boosted forward with the pinned event transform lands
  on (t', z') of the sample.
* Physics: a lab laser pulse loaded into the boosted frame, propagated, and recorded at a
  lab station reproduces the lab-frame pulse's time history at that plane.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import EX, EY, EZ, BX, BY, BZ


def beta(g):
    return math.sqrt(1 - 1 / g ** 2)


def test_station_of_uniform_fields_is_their_inverse_boost():
    gb = 7.0
    n = (4, 3, 32)
    s = oracle.Sim(3, n, (0, 0, 0), (1.0, 1.0, 0.5), 0.2, tile=(4, 3, 8))
    rng = np.random.default_rng(51)
    Ep, Bp = rng.normal(size=3), rng.normal(size=3)
    for c, v in zip((EX, EY, EZ, BX, BY, BZ), list(Ep) + list(Bp)):
        s.set_field(c, np.full((n[2], n[1], n[0]), v))
    rec = s.station_record(gb, 5.0 * gb)  # z' = 5 at t' = 0
    assert rec is not None
    t_lab, f = rec
    lab = f[:, 0, 0].copy()
    assert np.allclose(f, lab[:, None, None], rtol=0, atol=0)
    E2, B2 = oracle.boost_fields(gb, lab[:3], lab[3:])
    assert np.allclose(E2, Ep, rtol=1e-13, atol=1e-13) and np.allclose(B2, Bp, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("steps", [0, 7])
def test_station_samples_the_plane_at_its_boosted_position_and_time(steps):
    gb, dz, dt = 3.0, 0.5, 0.2
    n = (2, 2, 64)
    s = oracle.Sim(3, n, (1, 1, 1), (1.0, 1.0, dz), dt, tile=(2, 2, 8))
    s.step(steps)  # empty box: only the step count moves
    a, b_, c, d = 0.3, 0.7, -0.2, 1.1
    z_ex = np.arange(n[2]) * dz          # Ex, Ey, Bz sit on z nodes
    z_by = (np.arange(n[2]) + 0.5) * dz  # Ez, Bx, By sit half a cell up
    s.set_field(EX, np.broadcast_to((a + b_ * z_ex)[:, None, None], (n[2], n[1], n[0])).copy())
    s.set_field(BY, np.broadcast_to((c + d * z_by)[:, None, None], (n[2], n[1], n[0])).copy())
    z_lab = 20.0
    rec = s.station_record(gb, z_lab)
    assert rec is not None
    t_lab, f = rec
    # the lab event (t_lab, z_lab) seen from the boosted frame
    ev, _ = oracle.boost_event(gb, [t_lab, 0.0, 0.0, z_lab], [0.0, 0.0, 0.0])
    assert abs(ev[0] - steps * dt) < 1e-12 and 0 < ev[3] < n[2] * dz
    zp = ev[3]
    b = beta(gb)
    ex, by = a + b_ * zp, c + d * zp  # linear fields: the interpolation is exact
    assert np.allclose(f[0], gb * (ex + b * by), rtol=1e-12)
    assert np.allclose(f[4], gb * (by + b * ex), rtol=1e-12)
    assert np.all(f[[1, 2, 3, 5]] == 0)
    # outside the box: no record
    assert s.station_record(gb, -5.0) is None


def test_lab_pulse_history_at_a_station():
    """A plane-wave lab pulse (a0, lambda0 = 1, 1/e length L) centred at z_c at t = 0 has,
    at the lab plane Z, E_x(t) = a0 k0 exp(-((Z - z_c - t) / L)^2) cos(k0 (Z - z_c - t)).
    Loaded into a gamma_b = 4 frame, propagated by the Yee scheme at 32 cells per boosted
    wavelength and recorded at Z, the history matches it to the scheme's dispersion."""
    gb = 4.0
    b = beta(gb)
    doppler = gb * (1 + b)
    dz = doppler / 32.0
    dt = 0.5 * dz
    n = (8, 1, 512)
    a0, L, zc = 0.5, 1.5, 5.0
    s = oracle.Sim(2, n, (0, 0, 1), (1.0, 1.0, dz), dt, tile=(8, 1, 16), absorb_cells=8)
    s.load_lab_frame(gb, laser=[a0, 1.0, 1e6, L, zc])
    # the boosted t' = 0 slice holds lab time b z at lab position z: a station at Z first
    # records at t = b Z, so Z is chosen where the pulse arrives later, Z - z_c > b Z + 2L
    Z = 320.0
    times, ex, by = [], [], []
    for _ in range(300):
        rec = s.station_record(gb, Z)
        if rec is not None:
            times.append(rec[0])
            ex.append(rec[1][0, 0, 0])
            by.append(rec[1][4, 0, 0])
        s.step(1)
    t = np.array(times)
    assert t.min() < Z - zc - 2 * L and t.max() > Z - zc + 2 * L
    xi = Z - zc - t
    k0 = 2 * math.pi
    expect = a0 * k0 * np.exp(-(xi / L) ** 2) * np.cos(k0 * xi)
    amp = a0 * k0
    assert np.abs(np.array(ex) - expect).max() < 0.05 * amp
    # a forward wave: B_y = E_x in the lab frame too
    assert np.abs(np.array(by) - np.array(ex)).max() < 0.05 * amp
