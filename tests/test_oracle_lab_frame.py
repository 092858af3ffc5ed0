"""Pins of the oracle's lab -> boosted-frame input transform (Sec. 2 of Vay et al.):
Lorentz invariants, boost composition, the Doppler-shifted laser against the lab-frame
pulse transformed event by event, plasma density/drift and beam worldlines."""
import math

import numpy as np
import pytest

import oracle
from oracle import EX, BY


def beta(g):
    return math.sqrt(1 - 1 / g ** 2)


@pytest.mark.parametrize("gb", [1.5, 13.0, 100.0])
def test_field_invariants_and_doppler(gb):
    rng = np.random.default_rng(1)
    for _ in range(20):
        E, B = rng.normal(size=3), rng.normal(size=3)
        Ep, Bp = oracle.boost_fields(gb, E, B)
        assert abs(Ep @ Bp - E @ B) < 1e-10 * gb ** 2
        assert abs((Ep @ Ep - Bp @ Bp) - (E @ E - B @ B)) < 1e-10 * gb ** 2
    # a +z plane wave Ex = By = 1 is red-shifted by 1 / (gamma (1 + beta))
    Ep, Bp = oracle.boost_fields(gb, [1, 0, 0], [0, 1, 0])
    D = 1 / (gb * (1 + beta(gb)))
    assert abs(Ep[0] - D) < 1e-12 and abs(Bp[1] - D) < 1e-12


def test_boost_composition_adds_rapidities():
    g1, g2 = 3.0, 7.0
    eta = math.acosh(g1) + math.acosh(g2)
    g3 = math.cosh(eta)
    rng = np.random.default_rng(2)
    for _ in range(10):
        tx, u = rng.normal(size=4), rng.normal(size=3)
        a, ua = oracle.boost_event(g1, tx, u)
        b, ub = oracle.boost_event(g2, a, ua)
        c, uc = oracle.boost_event(g3, tx, u)
        assert np.abs(b - c).max() < 1e-10 and np.abs(ub - uc).max() < 1e-10
        # interval and mass shell
        assert abs((tx[0] ** 2 - tx[1:] @ tx[1:]) - (c[0] ** 2 - c[1:] @ c[1:])) < 1e-9
        g = math.sqrt(1 + u @ u)
        gp = math.sqrt(1 + uc @ uc)
        assert abs(gp - g3 * (g - beta(g3) * u[2])) < 1e-9
        E, B = rng.normal(size=3), rng.normal(size=3)
        Ea, Ba = oracle.boost_fields(g1, E, B)
        Eb, Bb = oracle.boost_fields(g2, Ea, Ba)
        Ec, Bc = oracle.boost_fields(g3, E, B)
        assert np.abs(Eb - Ec).max() < 1e-10 and np.abs(Bb - Bc).max() < 1e-10


@pytest.mark.parametrize("gb", [1.0, 4.0, 13.0])
def test_laser_is_lab_pulse_transformed(gb):
    """Boosted-frame laser at t' = 0 equals the lab pulse Ex = By = f(z - t - z_c) evaluated
    at the lab event of each grid point and transformed with the field boost."""
    lam0, a0, w0, tau, zc = 1.0, 2.0, 6.0, 3.0, 2.0
    D = gb * (1 + beta(gb))
    nz = 64
    dz = D * lam0 / 8
    s = oracle.Sim(2, (16, 1, nz), (1, 0, 1), (1.0, 1.0, dz), 0.5 * dz, order=2, tile=(8, 1, 8))
    s.load_lab_frame(gb, laser=[a0, lam0, w0, tau, zc])
    Ex = s.get_field(EX)[:, 0, :]
    By = s.get_field(BY)[:, 0, :]
    k0 = 2 * math.pi / lam0
    b = beta(gb)
    for kk in range(nz):
        for i in (3, 8, 12):
            x = (i + 0.5) * 1.0 - 8.0
            for zp, got, comp in (((kk) * dz, Ex[kk, i], 0), ((kk + 0.5) * dz, By[kk, i], 1)):
                t, z = gb * b * zp, gb * zp  # lab event of (t' = 0, z')
                xi = z - t - zc
                f = a0 * k0 * math.exp(-x * x / w0 ** 2) * math.exp(-(xi / tau) ** 2) * math.cos(k0 * xi)
                Ep, Bp = oracle.boost_fields(gb, [f, 0, 0], [0, f, 0])
                expect = Ep[0] if comp == 0 else Bp[1]
                assert abs(got - expect) < 1e-11 * a0 * k0


@pytest.mark.parametrize("gb", [1.0, 13.0])
def test_plasma_density_drift_and_charge(gb):
    """Cold lab plasma at rest -> drifting at -beta with density gamma n0; the number of
    physical electrons equals n0 times the lab volume (charge invariance)."""
    n0, ppc = 0.04, 2
    n = (8, 6, 32)
    dx = (2.0, 2.0, 1.5)
    s = oracle.Sim(3, n, (1, 1, 1), dx, 0.5, order=2, tile=(4, 3, 8))
    zs, ramp = 0.0, 0.0
    s.load_lab_frame(gb, plasma=[n0, zs, ramp, ppc, 0, 0, 0, 9])
    p = s.get_particles()
    assert p["cell"].size == ppc * 8 * 6 * 32
    assert np.allclose(p["u"][:, 2], -gb * beta(gb), rtol=0, atol=1e-12)
    assert np.all(p["u"][:, :2] == 0)
    Vlab = (8 * dx[0]) * (6 * dx[1]) * (32 * dx[2] * gb)
    assert abs(p["w"].sum() - n0 * Vlab) < 1e-9 * n0 * Vlab
    # offsets are the seeded uniforms of streams 0..2
    cell, c0 = p["cell"], p["cell"][0]
    first = np.where(cell == c0)[0]
    ctr = c0 * ppc
    assert abs(p["off"][first[0], 0] - oracle.uniform(9, 0, ctr)) < 1e-15


def test_plasma_ramp():
    n0, ppc, gb = 1.0, 1, 2.0
    s = oracle.Sim(2, (4, 1, 40), (1, 0, 1), (1.0, 1.0, 1.0), 0.5, order=1, tile=(4, 1, 8))
    zs, ramp = 20.0, 30.0  # lab: starts at 20, full density from 50 (boosted: 10 .. 25)
    s.load_lab_frame(gb, plasma=[n0, zs, ramp, ppc, 0, 0, 0, 3])
    p = s.get_particles()
    zp = (p["cell"] // 4 + p["off"][:, 2])
    zlab = gb * zp
    prof = np.clip((zlab - zs) / ramp, 0, 1)
    assert np.all(zlab >= zs)
    assert np.allclose(p["w"], gb * n0 * prof / ppc, rtol=1e-13, atol=0)


def test_beam_worldlines():
    """Each beam particle loaded at t' = 0 lies on the boosted worldline through its
    sampled lab event: x'_event = x'_0 + v' t'_event."""
    gb = 5.0
    n = (16, 16, 64)
    dx = (1.0, 1.0, 1.0)
    s = oracle.Sim(3, n, (1, 1, 1), dx, 0.5, order=2, tile=(8, 8, 8))
    # a beam near c at lab z0 sits near z' = gamma_b (1 + beta_b) z0 at t' = 0 and is
    # stretched by the same factor
    nb, gam, spread, sr, sz, z0, seed = 400, 50.0, 1e-2, 1.5, 0.3, 3.2, 4
    s.load_lab_frame(gb, beam=[nb, gam, spread, sr, sz, z0, 1.0, seed])
    p = s.get_particles()
    assert 0.95 * nb <= p["cell"].size <= nb
    D = gb * (1 + beta(gb))
    zc = (p["cell"] // 256 + p["off"][:, 2]).mean()
    assert abs(zc - D * z0) < 0.05 * D * z0
    ids = p["id"]
    pos0 = np.stack([(p["cell"] % 16) + p["off"][:, 0], (p["cell"] // 16 % 16) + p["off"][:, 1],
                     (p["cell"] // 256) + p["off"][:, 2]], 1)
    for q in range(p["cell"].size):
        i = int(ids[q])
        g0 = math.sqrt(gam ** 2 - 1)
        tx = [0.0, 8.0 + sr * oracle.normal(seed, 10, i), 8.0 + sr * oracle.normal(seed, 12, i),
              z0 + sz * oracle.normal(seed, 14, i)]
        u = [spread * g0 * oracle.normal(seed, 16, i), spread * g0 * oracle.normal(seed, 18, i),
             g0 + spread * g0 * oracle.normal(seed, 20, i)]
        txp, up = oracle.boost_event(gb, tx, u)
        assert np.abs(up - p["u"][q]).max() < 1e-12 * np.abs(up).max()
        gp = math.sqrt(1 + up @ up)
        for a in range(3):
            assert abs(txp[1 + a] - (pos0[q, a] + up[a] / gp * txp[0])) < 1e-9
