"""Pins of the oracle's beam self-field (the field a relativistic beam carries, whose
effect on the beam itself is the case of Sec. 2 of Vay et al.).

* The eigen-expansion solve equals a dense direct solve of the same discrete system
  (second differences, phi = 0 beyond an absorbing face, wrap on a periodic axis) for
  mixed boundaries, in 3D and 2D3V.
* Lorentz covariance, exactly on the grid: a charge at rest solved on a grid of spacing
  dz0, and the same charge moving at gamma, contracted (rho = gamma rho0 on the grid of
  spacing dz0 / gamma), give E_perp = gamma E0_perp, E_z = E0_z and B = beta z x E.  This
  fixes where gamma enters (a 1/gamma^2 on d/dz and on E_z).
* Gauss's law div E = rho on every node not on the first layer of an absorbing axis.
* Loading a beam adds the self-field of its deposited charge for its velocity.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import EX, EY, EZ, BX, BY, BZ


def second_difference(n, periodic, dx):
    D = np.zeros((n, n))
    for i in range(n):
        D[i, i] = -2.0
        for j in (i - 1, i + 1):
            if 0 <= j < n:
                D[i, j] += 1.0
            elif periodic:
                D[i, j % n] += 1.0
    return D / dx ** 2


def dense_fields(n, bc, dx, rho, gamma, beta, ndim=3):
    """Direct solve of the discrete system, then E and B on the Yee grid."""
    n0, n1, n2 = n
    I = [np.eye(m) for m in n]
    L = [second_difference(n[a], bc[a] == 0, dx[a]) for a in range(3)]
    if ndim == 2:
        L[1] = np.zeros((1, 1))
    # unknowns ordered x fastest: kron(z, y, x)
    A = (np.kron(I[2], np.kron(I[1], L[0])) + np.kron(I[2], np.kron(L[1], I[0]))
         + np.kron(L[2], np.kron(I[1], I[0])) / gamma ** 2)
    phi = np.linalg.solve(A, -rho.ravel()).reshape(n2, n1, n0)

    def shifted(f, axis_xyz):
        ax = 2 - axis_xyz  # array axes are (z, y, x)
        out = np.roll(f, -1, axis=ax)
        if bc[axis_xyz] == 1:
            idx = [slice(None)] * 3
            idx[ax] = -1
            out[tuple(idx)] = 0.0
        return out

    Ex = -(shifted(phi, 0) - phi) / dx[0]
    Ey = -(shifted(phi, 1) - phi) / dx[1] if ndim == 3 else np.zeros_like(phi)
    Ez = -(shifted(phi, 2) - phi) / (dx[2] * gamma ** 2)
    # E at z + 1: wrap, or zero beyond an absorbing face
    Ex1, Ey1 = shifted(Ex, 2), shifted(Ey, 2)
    Bx = -beta * 0.5 * (Ey + Ey1)
    By = beta * 0.5 * (Ex + Ex1)
    return Ex, Ey, Ez, Bx, By


def fields_of(s):
    return [s.get_field(c) for c in (EX, EY, EZ, BX, BY, BZ)]


@pytest.mark.parametrize("ndim,n,bc", [(3, (5, 4, 7), (1, 0, 1)), (3, (4, 6, 5), (0, 1, 0)),
                                       (3, (4, 3, 5), (0, 0, 0)), (2, (6, 1, 8), (1, 0, 0))])
def test_self_field_equals_dense_solve(ndim, n, bc):
    rng = np.random.default_rng(31)
    dx = (0.7, 1.1, 0.9)
    gamma = 3.0
    beta = math.sqrt(1 - 1 / gamma ** 2)
    rho = rng.normal(size=(n[2], n[1], n[0]))
    if all(b == 0 for b in bc):
        rho -= rho.mean()  # all periodic: the mean is dropped
    s = oracle.Sim(ndim, n, bc, dx, 0.1, order=1, tile=(n[0], n[1], n[2]))
    s.beam_self_field(rho, gamma, beta)
    Ex, Ey, Ez, Bx, By, Bz = fields_of(s)
    ref = dense_fields(n, bc, dx, rho, gamma, beta, ndim)
    scale = max(np.abs(r).max() for r in ref)
    for got, want in zip((Ex, Ey, Ez, Bx, By), ref):
        assert np.abs(got - want).max() <= 1e-12 * scale
    assert np.all(Bz == 0)


def test_self_field_is_lorentz_covariant_on_the_grid():
    n, bc = (6, 5, 12), (1, 1, 1)
    rng = np.random.default_rng(32)
    rho0 = rng.random((n[2], n[1], n[0]))
    dz0 = 0.8
    rest = oracle.Sim(3, n, bc, (1.0, 1.0, dz0), 0.1, order=1, tile=(6, 5, 12))
    rest.beam_self_field(rho0, 1.0, 0.0)
    E0x, E0y, E0z, B0x, B0y, _ = fields_of(rest)
    assert np.all(B0x == 0) and np.all(B0y == 0)
    for gamma in (2.0, 50.0):
        beta = math.sqrt(1 - 1 / gamma ** 2)
        mov = oracle.Sim(3, n, bc, (1.0, 1.0, dz0 / gamma), 0.1, order=1, tile=(6, 5, 12))
        mov.beam_self_field(gamma * rho0, gamma, beta)
        Ex, Ey, Ez, Bx, By, _ = fields_of(mov)
        sc = gamma * max(np.abs(E0x).max(), np.abs(E0y).max())
        assert np.abs(Ex - gamma * E0x).max() <= 1e-12 * sc
        assert np.abs(Ey - gamma * E0y).max() <= 1e-12 * sc
        assert np.abs(Ez - E0z).max() <= 1e-12 * sc
        # B = beta z x E at B's half-integer z (E averaged over the two z nodes)
        ex1 = np.concatenate([Ex[1:], np.zeros_like(Ex[:1])], axis=0)
        ey1 = np.concatenate([Ey[1:], np.zeros_like(Ey[:1])], axis=0)
        assert np.abs(By - beta * 0.5 * (Ex + ex1)).max() <= 1e-12 * sc
        assert np.abs(Bx + beta * 0.5 * (Ey + ey1)).max() <= 1e-12 * sc


def test_self_field_satisfies_gauss_law():
    n, bc = (8, 6, 10), (1, 0, 1)
    rng = np.random.default_rng(33)
    rho = rng.normal(size=(n[2], n[1], n[0]))
    s = oracle.Sim(3, n, bc, (1.0, 0.8, 1.2), 0.1, order=2, tile=(8, 6, 10))
    s.beam_self_field(rho, 7.0, math.sqrt(1 - 1 / 49.0))
    div = s.div_e()
    interior = (slice(1, None), slice(None), slice(1, None))  # first layer of absorbing x, z
    assert np.abs(div - rho)[interior].max() <= 1e-12 * np.abs(rho).max()


@pytest.mark.parametrize("gamma_boost", [1.0, 3.0])
def test_beam_load_adds_its_self_field(gamma_boost):
    """The loader adds the self-field of the loaded beam's charge for the centroid
    velocity in the simulation frame (rapidities subtract: gamma' = cosh(eta - eta_b))."""
    n = (8, 8, 24)
    gamma = 20.0
    eta = math.acosh(gamma) - math.acosh(gamma_boost)
    # lab lengths at lab t = 0 map to boosted lengths at t' = 0 times gb (1 + beta' beta_b)
    stretch = gamma_boost * (1 + math.tanh(eta) * math.sqrt(1 - 1 / gamma_boost ** 2))
    beam = (3000, gamma, 1e-3, 1.5, 3.0 / stretch, 12.0 / stretch, 50.0, 5)
    s = oracle.Sim(3, n, (1, 1, 1), (1.0, 1.0, 1.0), 0.5, order=2, tile=(8, 8, 8))
    s.load_lab_frame(gamma_boost, beam=beam)
    ref = oracle.Sim(3, n, (1, 1, 1), (1.0, 1.0, 1.0), 0.5, order=2, tile=(8, 8, 8))
    p = s.get_particles()
    assert p["id"].size > 2500
    ref.set_particles(p["cell"], p["off"], p["u"], p["w"], p["id"])
    gp = math.cosh(eta)
    ref.beam_self_field(ref.rho(), gp, math.sqrt(1 - 1 / gp ** 2))
    for got, want in zip(fields_of(s), fields_of(ref)):
        assert np.abs(got - want).max() <= 1e-13 * max(np.abs(want).max(), 1e-300)
    # a relativistic beam: the radial field is gamma^2 times the longitudinal one at most
    Ex, _, Ez, _, By, _ = fields_of(s)
    assert np.abs(Ex).max() > 10 * np.abs(Ez).max()
    assert np.abs(By).max() == pytest.approx(np.abs(Ex).max(), rel=0.05)
