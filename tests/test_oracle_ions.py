"""Pins of the oracle's ion background for lab-frame plasma loads (Sec. 2 of Vay et al.:
the plasma is at rest in the lab frame, so in the boosted frame its ions form a rigid,
gamma_b-contracted charge density streaming at -beta_b).

The checks tie the ion term to quantities computed elsewhere: the ion density seen on the
grid equals the contracted lab profile translated by -beta_b t' (closed form on every
node whose dual cell lies in one linear piece of the profile); the ions' current cancels
the mean current that the Esirkepov deposit gets from the independently boosted
electrons, so a cold neutral plasma streams without driving the k = 0 mode of E_z; and
div E - rho, ions included, stays constant to round-off while the ramp moves through the
grid (the ions' current and charge obey the discrete continuity equation).
"""
import math

import numpy as np

import oracle
from oracle import JZ, EZ


def beta(g):
    return math.sqrt(1 - 1 / g ** 2)


def electrons_only(s, like):
    """A copy of `s`'s particles in a fresh simulation without the ion background."""
    p = s.get_particles()
    like.set_particles(p["cell"], p["off"], p["u"], p["w"], p["id"])
    return like


def test_ion_density_is_contracted_lab_profile_moving_at_minus_beta():
    gb, n0, zs, ramp = 5.0, 0.3, 100.0, 60.0  # boosted: ramp from z' = 20 to z' = 32
    n, dz, dt = (4, 1, 200), 0.5, 0.25
    mk = lambda: oracle.Sim(2, n, (0, 0, 1), (1.0, 1.0, dz), dt, order=1, tile=(4, 1, 8))
    s = mk()
    s.load_lab_frame(gb, plasma=[n0, zs, ramp, 1, 0, 0, 0, 5])
    b = beta(gb)
    z = np.arange(n[2]) * dz
    for steps in (0, 9, 40):
        s.step(steps)
        t = s.diagnostics()["step"] * dt
        rho_i = (s.rho() - electrons_only(s, mk()).rho())[:, 0, 0]  # same in every x column
        # lab profile at the lab position of each node's dual-cell ends
        lo = gb * (z - dz / 2 + b * t)
        hi = gb * (z + dz / 2 + b * t)
        mid = gb * (z + b * t)
        in_box = (z - dz / 2 + b * t >= 0) & (z + dz / 2 + b * t <= n[2] * dz)
        ramp_nodes = in_box & (lo >= zs) & (hi <= zs + ramp)
        plateau = in_box & (lo >= zs + ramp)
        empty = (hi <= zs) | (z + dz / 2 + b * t <= 0) | (z - dz / 2 + b * t >= n[2] * dz)
        assert ramp_nodes.sum() > 10 and plateau.sum() > 10 and empty.sum() >= 1
        expect_ramp = gb * n0 * (mid - zs) / ramp  # midpoint value of a linear profile
        assert np.allclose(rho_i[ramp_nodes], expect_ramp[ramp_nodes], rtol=1e-12, atol=0)
        assert np.allclose(rho_i[plateau], gb * n0, rtol=1e-12, atol=0)
        assert np.all(rho_i[empty] == 0)


def test_ion_current_cancels_the_electrons_mean_current():
    """Cold uniform plasma, periodic box: sum over the grid of Jz (electrons + ions) is
    zero to round-off, so the box-mean E_z stays zero; the same electrons without their
    ions drive it at dE/dt = -<J_e>."""
    gb, n0, ppc = 13.0, 0.05, 2
    n, dx, dt = (6, 1, 48), (1.5, 1.0, 0.4), 0.3
    mk = lambda: oracle.Sim(2, n, (0, 0, 0), dx, dt, order=2, tile=(6, 1, 8))
    s = mk()
    s.load_lab_frame(gb, plasma=[n0, -1e9, 0.0, ppc, 0, 0, 0, 8])
    e = electrons_only(s, mk())
    s.particle_phase()
    e.particle_phase()
    je, jt = e.get_field(JZ).sum(), s.get_field(JZ).sum()
    expect_je = n[0] * n[2] * gb * n0 * beta(gb)  # -q n' v summed over cells, q = -1, v = -beta
    assert abs(je - expect_je) <= 1e-12 * expect_je
    assert abs(jt) <= 1e-12 * je
    s.maxwell()
    e.maxwell()
    for _ in range(10):
        s.step(1)
        e.step(1)
    steps = 11
    print("mean Ez with / without ions", s.get_field(EZ).mean(), e.get_field(EZ).mean())
    # later steps: only the noise fields change the mean electron velocity (by ~1e-5 here)
    assert abs(s.get_field(EZ).mean()) <= 1e-4 * abs(e.get_field(EZ).mean())
    # without ions the k = 0 mode follows dE/dt = -<J> (it feeds back on the electrons
    # only through a uniform field, which decelerates them: 10 % bound)
    assert abs(e.get_field(EZ).mean() + steps * dt * expect_je / (n[0] * n[2])) <= 0.1 * steps * dt * expect_je / (n[0] * n[2])


def test_gauss_law_with_moving_ions():
    """div E - rho (ions included) constant to round-off away from the absorbing layers
    while the ramp streams through the grid, thermal electrons, unfiltered current."""
    gb, n0, zs, ramp = 4.0, 0.2, 20.0, 40.0
    n, dx, dt = (8, 6, 64), (1.0, 1.0, 0.5), 0.3
    s = oracle.Sim(3, n, (0, 0, 1), dx, dt, order=2, tile=(4, 3, 8), absorb_cells=4)
    s.load_lab_frame(gb, plasma=[n0, zs, ramp, 2, 0.05, 0.05, 0.05, 11])
    rho0 = s.rho()
    r0 = s.div_e() - rho0
    s.step(25)
    rho1 = s.rho()
    r1 = s.div_e() - rho1
    inner = slice(6, n[2] - 6)
    scale = np.abs(rho1).max()
    print("Gauss residual drift", np.abs(r1 - r0)[inner].max() / scale)
    assert np.abs(r1 - r0)[inner].max() <= 1e-12 * scale
    # the ramp moved by beta t = 14.5 cells: the charge on the inner nodes changed
    assert np.abs(rho1 - rho0)[inner].max() > 0.1 * scale
    assert s.diagnostics()["field_energy"] > 0
