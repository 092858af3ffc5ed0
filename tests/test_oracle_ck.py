"""Pins of the oracle's low-dispersion field solver (Sec. 2 of Vay et al. cures the
boosted-frame instability partly with low-dispersion solvers, citing Karkkainen et al.):
Faraday differences averaged over their transverse neighbours (7/12, 1/12, 1/48).

* Standing waves E_pol = cos(k.x), k normal to pol: E^N = cos(N w dt) E^0 exactly with
  sin^2(w dt/2)/dt^2 = sum_a S_a sin^2(k_a dx_a/2)/dx_a^2,
  S_a = 7/12 + (cos th_b + cos th_c)/6 + cos th_b cos th_c/12 (th = k dx), in 3D and 2D3V,
  for several k (the relation differs from Yee's by the factors S_a).
* The one-step propagator of a small periodic grid has no eigenvalue off the unit circle
  and no defective eigenvalue at 1 (every mode keeps its Faraday coupling), so random
  fields stay bounded.
* A wave along a grid axis at dt equal to that axis's cell size travels without
  dispersion: w = |k| exactly, the continuum value.
* Bounded at dt = 0.99 min(dx) on cubic cells, where the Yee scheme (limit dx / sqrt 3)
  blows up.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import EX, EY, EZ, BX, BY, BZ, SOLVER_CK, SOLVER_YEE

STAG = {EX: (0.5, 0, 0), EY: (0, 0.5, 0), EZ: (0, 0, 0.5)}


def coords(n, stag):
    z, y, x = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    return x + stag[0], y + stag[1], z + stag[2]


def ck_mode(ndim, pol, n, dx, dt, m, steps):
    s = oracle.Sim(ndim, n, (0, 0, 0), dx, dt, solver=SOLVER_CK)
    active = [0, 1, 2] if ndim == 3 else [0, 2]
    axes = [a for a in active if a != pol]
    k = [2 * math.pi * m[a] / (s.n[a] * dx[a]) if a in axes else 0.0 for a in range(3)]
    x, y, z = coords(s.n, STAG[pol])
    pos = [x * dx[0], y * dx[1], z * dx[2]]
    phase = sum(k[a] * pos[a] for a in axes)
    s.set_field(pol, np.cos(phase))
    for _ in range(steps):
        s.maxwell()
    rhs = 0.0
    for a in active:
        cb, cc = [math.cos(k[b] * dx[b]) for b in range(3) if b != a]
        S = 7 / 12 + (cb + cc) / 6 + cb * cc / 12  # an invariant axis has cos 0 = 1
        rhs += S * (math.sin(k[a] * dx[a] / 2) / dx[a]) ** 2
    w = 2 / dt * math.asin(dt * math.sqrt(rhs))
    return s.get_field(pol), np.cos(phase) * math.cos(w * dt * steps), s


@pytest.mark.parametrize("m", [(2, 3, 4), (1, 4, 2), (5, 1, 1)])
@pytest.mark.parametrize("pol", [EX, EY, EZ])
def test_ck_dispersion_relation_3d(pol, m):
    got, exact, s = ck_mode(3, pol, (12, 10, 14), (1.0, 0.9, 1.2), 0.8, m, 40)
    assert np.abs(got - exact).max() < 1e-12
    assert np.abs(s.div_e()).max() < 1e-12


@pytest.mark.parametrize("pol", [EX, EY, EZ])
def test_ck_dispersion_relation_2d(pol):
    got, exact, _ = ck_mode(2, pol, (16, 1, 12), (1.0, 1.0, 0.8), 0.7, (3, 0, 2), 60)
    assert np.abs(got - exact).max() < 1e-12


def test_ck_axis_wave_is_dispersion_free_at_dt_equal_dz():
    """E_x = cos(k z), k = 2 pi m / Lz on a grid with dz the smallest cell: at dt = dz the
    standing wave oscillates at the continuum frequency w = k."""
    dx = (1.5, 1.3, 1.0)
    n = (4, 4, 24)
    s = oracle.Sim(3, n, (0, 0, 0), dx, dx[2], solver=SOLVER_CK)
    k = 2 * math.pi * 5 / (n[2] * dx[2])
    _, _, z = coords(n, STAG[EX])
    s.set_field(EX, np.cos(k * z * dx[2]))
    steps = 37
    for _ in range(steps):
        s.maxwell()
    assert np.abs(s.get_field(EX) - np.cos(k * z * dx[2]) * math.cos(k * dx[2] * steps)).max() < 1e-12


def test_ck_propagator_spectrum_on_unit_circle():
    """One Maxwell step as a matrix on a 4^3 periodic grid (all 6 x 64 unit states):
    every eigenvalue has modulus 1 to round-off at dt = 0.99 dx.  Averaging weights that
    vanish at some wavevector (1-2-1 products, zero at two Nyquist indices) leave those
    modes' B static while E grows linearly: a defective eigenvalue 1."""
    n, N = (4, 4, 4), 64
    P = np.zeros((6 * N, 6 * N))
    for col in range(6 * N):
        s = oracle.Sim(3, n, (0, 0, 0), (1.0, 1.0, 1.0), 0.99, solver=SOLVER_CK)
        v = np.zeros(6 * N)
        v[col] = 1.0
        for c in range(6):
            s.set_field(c, v[c * N:(c + 1) * N].reshape(4, 4, 4))
        s.maxwell()
        P[:, col] = np.concatenate([s.get_field(c).ravel() for c in range(6)])
    ev = np.linalg.eigvals(P)
    assert np.abs(np.abs(ev) - 1).max() < 1e-10
    # 100 steps of the propagator stay bounded (no Jordan block)
    assert np.abs(np.linalg.matrix_power(P, 100)).max() < 10


def test_ck_stable_where_yee_is_not():
    n = (10, 10, 10)
    rng = np.random.default_rng(61)
    init = [rng.normal(size=(10, 10, 10)) for _ in range(6)]
    energies = {}
    for solver in (SOLVER_CK, SOLVER_YEE):
        s = oracle.Sim(3, n, (0, 0, 0), (1.0, 1.0, 1.0), 0.99, solver=solver)
        for c, f in zip((EX, EY, EZ, BX, BY, BZ), init):
            s.set_field(c, f)
        e0 = s.diagnostics()["field_energy"]
        for _ in range(200):
            s.maxwell()
        energies[solver] = s.diagnostics()["field_energy"] / e0
    # near the Courant limit (E^2 + B^2) at whole steps oscillates (the leapfrog's
    # conserved energy pairs B at the half steps): bounded, not constant
    assert energies[SOLVER_CK] < 30.0
    assert not np.isfinite(energies[SOLVER_YEE]) or energies[SOLVER_YEE] > 1e6
