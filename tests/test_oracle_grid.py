"""Pins of the oracle's grid operations: gather, Esirkepov deposit, binomial filter, Yee
FDTD, absorbing layer, canonical sort and the whole step's Gauss-law invariant.

Each check is a closed form, an invariant or a brute-force recount -- never the oracle
compared with a retyped copy of itself.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import EX, EY, EZ, BX, BY, BZ, JX, JY, JZ

STAG = {EX: (0.5, 0, 0), EY: (0, 0.5, 0), EZ: (0, 0, 0.5),
        BX: (0, 0.5, 0.5), BY: (0.5, 0, 0.5), BZ: (0.5, 0.5, 0)}


def grid_coords(n, stag):
    k, j, i = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    return i + stag[0], j + stag[1], k + stag[2]


def make(ndim, n, bc=(0, 0, 0), dx=(1.0, 1.0, 1.0), dt=0.4, **kw):
    return oracle.Sim(ndim, n, bc, dx, dt, **kw)


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("ndim", [2, 3])
def test_gather_reproduces_linear_fields(order, ndim):
    """Both B-splines reproduce linear functions exactly, so a linear field sampled at each
    component's own staggered position gathers to its value at the particle; a wrong
    stagger or axis would shift it by half a slope."""
    n = (12, 10, 14) if ndim == 3 else (12, 1, 14)
    s = make(ndim, n, order=order)
    coef = {c: np.array([0.3 + c, -0.7 + 0.1 * c, 0.45 - 0.2 * c]) for c in STAG}
    for c, st in STAG.items():
        x, y, z = grid_coords(s.n, st)
        if ndim == 2:
            y = np.zeros_like(y)
        s.set_field(c, 1.0 + coef[c][0] * x + coef[c][1] * y + coef[c][2] * z)
    rng = np.random.default_rng(3)
    for _ in range(30):
        c3 = [rng.integers(3, s.n[0] - 3), rng.integers(3, s.n[1] - 3) if ndim == 3 else 0,
              rng.integers(3, s.n[2] - 3)]
        off = rng.random(3)
        if ndim == 2:
            off[1] = 0.0
        cell = c3[0] + s.n[0] * (c3[1] + s.n[1] * c3[2])
        E, B = s.gather(cell, off)
        pos = np.array(c3) + off
        for c in STAG:
            expect = 1.0 + coef[c] @ pos
            got = E[c] if c < 3 else B[c - 3]
            assert abs(got - expect) < 1e-12


def test_gather_quadratic_second_moment():
    """Order 2 reproduces x^2 up to the spline's constant second moment 1/4 per axis."""
    s = make(3, (10, 10, 10), order=2)
    x, y, z = grid_coords(s.n, STAG[EX])
    s.set_field(EX, x ** 2)
    c3 = [4, 5, 6]
    off = np.array([0.3, 0.8, 0.1])
    E, _ = s.gather(c3[0] + 10 * (c3[1] + 10 * c3[2]), off)
    assert abs(E[0] - ((4.3) ** 2 + 0.25)) < 1e-12


def _one_particle_deposit(ndim, order, u, cell3, off, n=(10, 10, 10), dx=(1.0, 0.8, 1.3), dt=0.35, w=0.7):
    s = make(ndim, n, dx=dx, dt=dt, order=order)
    nn = s.n
    cell = cell3[0] + nn[0] * (cell3[1] + nn[1] * cell3[2])
    s.set_particles(np.array([cell]), np.array([off]), np.array([u]), np.array([w]))
    rho0 = s.rho()
    s.particle_phase()
    rho1 = s.rho()
    J = [s.get_field(c) for c in (JX, JY, JZ)]
    return s, rho0, rho1, J


def _div(J, dx, ndim):
    d = np.zeros_like(J[0])
    axes = [0, 1, 2] if ndim == 3 else [0, 2]
    for a in axes:
        arr = J[a]
        npax = 2 - a  # arrays are [z, y, x]
        d += (arr - np.roll(arr, 1, axis=npax)) / dx[a]
    return d


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("ndim", [2, 3])
def test_esirkepov_discrete_continuity(order, ndim):
    """Charge conservation: (rho^{n+1} - rho^n)/dt + div J^{n+1/2} = 0 to round-off, for
    random single particles, including cell and periodic-boundary crossings."""
    rng = np.random.default_rng(11 + order + ndim)
    dx, dt = (1.0, 0.8, 1.3), 0.35
    for trial in range(25):
        u = rng.normal(0, 3.0, 3)
        cell3 = [int(rng.integers(0, 10)), int(rng.integers(0, 10)) if ndim == 3 else 0, int(rng.integers(0, 10))]
        if trial < 4:  # force boundary crossings
            cell3 = [9 if trial % 2 else 0, cell3[1], 0 if trial % 2 else 9]
            u = np.array([8.0 if trial % 2 else -8.0, 0.3, -8.0 if trial % 2 else 8.0])
        off = rng.random(3)
        if ndim == 2:
            off[1] = 0
        s, r0, r1, J = _one_particle_deposit(ndim, order, u, cell3, off, dx=dx, dt=dt)
        resid = (r1 - r0) / dt + _div(J, dx, ndim)
        assert np.abs(resid).max() < 1e-13 * max(1.0, np.abs(r0).max() / dt)
        # total charge is conserved by construction
        assert abs(r1.sum() - r0.sum()) < 1e-13


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("ndim", [2, 3])
def test_esirkepov_total_current(order, ndim):
    """sum J dV = q w (x^{n+1} - x^n) / dt per axis (the first moment of the deposit); in
    2D3V the out-of-plane current sums to q w v_y."""
    rng = np.random.default_rng(5)
    dx, dt, w = (1.0, 0.8, 1.3), 0.35, 0.7
    for _ in range(10):
        u = rng.normal(0, 2.0, 3)
        cell3 = [4, 4 if ndim == 3 else 0, 5]
        off = rng.random(3)
        if ndim == 2:
            off[1] = 0
        s, r0, r1, J = _one_particle_deposit(ndim, order, u, cell3, off, dx=dx, dt=dt, w=w)
        g = math.sqrt(1 + u @ u)  # zero fields -> u unchanged
        dV = dx[0] * dx[1] * dx[2]
        for a in range(3):
            if ndim == 2 and a == 1:
                expect = -1.0 * w * u[1] / g
            else:
                expect = -1.0 * w * u[a] / g  # q = -1; displacement/dt = v
            assert abs(J[a].sum() * dV - expect) < 1e-13 * max(1, abs(expect)) + 1e-15


def test_esirkepov_2d_out_of_plane_static():
    """2D3V particle moving only along y (out of plane): J_y = q w v_y S(x) S(z) / dV."""
    s, r0, r1, J = _one_particle_deposit(2, 2, np.array([0.0, 1.5, 0.0]), [4, 0, 5], np.array([0.3, 0.0, 0.6]),
                                         dx=(1.0, 1.0, 1.0), dt=0.4, w=0.7)
    v = 1.5 / math.sqrt(1 + 1.5 ** 2)
    # rho0 = q w S(x) S(z) / dV, so J_y = v_y rho0 when the in-plane shapes do not change
    assert np.abs(J[1] - v * r0).max() < 1e-14
    assert np.abs(J[0]).max() == 0.0 and np.abs(J[2]).max() == 0.0


@pytest.mark.parametrize("passes", [1, 3])
def test_filter_gain_on_sinusoid(passes):
    """1-2-1 on cos(k x) gives cos^2(k dx / 2) cos(k x); N passes over all axes multiply."""
    n = (16, 12, 20)
    s = make(3, n, filter_passes=passes)
    m = (3, 2, 5)
    k = [2 * math.pi * m[a] / n[a] for a in range(3)]
    for c in (JX, JY, JZ):
        x, y, z = grid_coords(s.n, (0, 0, 0))
        s.set_field(c, np.cos(k[0] * x + k[1] * y + k[2] * z + 0.3 * c))
    s.filter()
    gain = np.prod([math.cos(k[a] / 2) ** (2 * passes) for a in range(3)])
    for c in (JX, JY, JZ):
        x, y, z = grid_coords(s.n, (0, 0, 0))
        assert np.abs(s.get_field(c) - gain * np.cos(k[0] * x + k[1] * y + k[2] * z + 0.3 * c)).max() < 1e-13


def test_filter_binomial_impulse_absorbing():
    """On a zero-padded (absorbing) line, N passes of 1-2-1 turn an impulse into the
    binomial row C(2N, j) / 4^N; the sum is preserved while the spread stays inside."""
    passes = 3
    s = make(2, (21, 1, 17), bc=(1, 0, 1), filter_passes=passes)
    J = np.zeros((17, 1, 21))
    J[8, 0, 10] = 1.0
    s.set_field(JZ, J)
    s.filter()
    out = s.get_field(JZ)[:, 0, :]
    row = np.array([math.comb(2 * passes, j) for j in range(2 * passes + 1)]) / 4.0 ** passes
    expect = np.zeros((17, 21))
    expect[8 - passes:8 + passes + 1, 10 - passes:10 + passes + 1] = np.outer(row, row)
    assert np.abs(out - expect).max() < 1e-15


@pytest.mark.parametrize("bcx", [0, 1])
def test_filter_passes_at_the_faces(bcx):
    """Each pass is the 1-2-1 matrix of the axis: tridiagonal with nothing beyond an
    absorbing face (what leaves does not come back in the next pass), circulant on a
    periodic axis.  Random currents next to the faces after three passes equal the cube of
    that matrix applied along x and along z (the axes commute), to round-off."""
    passes = 3
    nx, nz = 12, 10
    s = make(2, (nx, 1, nz), bc=(bcx, 0, 1), filter_passes=passes)
    rng = np.random.default_rng(11)
    J = np.zeros((nz, 1, nx))
    J[:, 0, :2] = rng.normal(size=(nz, 2))
    J[:, 0, -2:] = rng.normal(size=(nz, 2))
    J[:2, 0, :] += rng.normal(size=(2, nx))
    s.set_field(JY, J)
    s.filter()

    def matrix(n, periodic):
        A = 0.5 * np.eye(n) + 0.25 * np.eye(n, k=1) + 0.25 * np.eye(n, k=-1)
        if periodic:
            A[0, -1] = A[-1, 0] = 0.25
        return A

    Ax = np.linalg.matrix_power(matrix(nx, bcx == 0), passes)
    Az = np.linalg.matrix_power(matrix(nz, False), passes)
    expect = Az @ J[:, 0, :] @ Ax.T
    assert np.abs(s.get_field(JY)[:, 0, :] - expect).max() < 1e-14
    # a plausible mistake, the (2N+1)-tap binomial applied once and cut at the faces,
    # differs near an absorbing face (what left in one pass would come back in the next)
    row = np.array([math.comb(2 * passes, j) for j in range(2 * passes + 1)]) / 4.0 ** passes
    once = sum(row[m + passes] * np.eye(nz, k=m) for m in range(-passes, passes + 1))
    assert np.abs(once - Az).max() > 1e-2


def _yee_mode(ndim, pol, n, dx, dt, m, steps):
    s = make(ndim, n, dx=dx, dt=dt)
    axes = [a for a in range(3) if a != pol and (ndim == 3 or a != 1)]
    k = [2 * math.pi * m[a] / (s.n[a] * dx[a]) if a in axes else 0.0 for a in range(3)]
    x, y, z = grid_coords(s.n, STAG[pol])
    pos = [x * dx[0], y * dx[1], z * dx[2]]
    phase = sum(k[a] * pos[a] for a in axes)
    s.set_field(pol, np.cos(phase))
    for _ in range(steps):
        s.maxwell()
    Kt2 = sum((2 / dx[a] * math.sin(k[a] * dx[a] / 2)) ** 2 for a in axes)
    w = 2 / dt * math.asin(dt * math.sqrt(Kt2) / 2)
    return s.get_field(pol), np.cos(phase) * math.cos(w * dt * steps), s


@pytest.mark.parametrize("pol", [EX, EY, EZ])
def test_yee_numerical_dispersion_3d(pol):
    """Vacuum standing wave E_pol = cos(k.x) with k normal to pol: Yee leapfrog gives
    E^N = cos(N w dt) E^0 exactly, with sin(w dt/2) = dt sqrt(sum_a (sin(k_a dx_a/2)/dx_a)^2)."""
    got, exact, s = _yee_mode(3, pol, (12, 10, 14), (1.0, 0.9, 1.2), 0.5, (2, 3, 4), 40)
    assert np.abs(got - exact).max() < 1e-12
    # no charge appears: div E stays zero
    assert np.abs(s.div_e()).max() < 1e-12


@pytest.mark.parametrize("pol", [EX, EY, EZ])
def test_yee_numerical_dispersion_2d(pol):
    got, exact, _ = _yee_mode(2, pol, (16, 1, 12), (1.0, 1.0, 0.8), 0.45, (3, 0, 2), 60)
    assert np.abs(got - exact).max() < 1e-12


def test_yee_keeps_div_b_zero():
    """Faraday's update adds the discrete curl of E to B, whose divergence (forward
    differences at the cell centres, where Bx, By, Bz meet) is zero identically: from random
    E and B = 0 on a periodic box, div B stays at round-off after 20 full steps while B
    grows to order one.  A wrong difference direction or stagger in any curl component
    breaks it."""
    n = (10, 12, 14)
    dx = (1.0, 0.9, 1.1)
    s = make(3, n, dx=dx, dt=0.3)
    rng = np.random.default_rng(21)
    for c in (EX, EY, EZ):
        s.set_field(c, rng.normal(size=(n[2], n[1], n[0])))
    for _ in range(20):
        s.maxwell()
    bx, by, bz = s.get_field(BX), s.get_field(BY), s.get_field(BZ)
    div = ((np.roll(bx, -1, 2) - bx) / dx[0] + (np.roll(by, -1, 1) - by) / dx[1] +
           (np.roll(bz, -1, 0) - bz) / dx[2])
    scale = max(np.abs(b).max() for b in (bx, by, bz))
    assert scale > 0.1
    assert np.abs(div).max() < 1e-13 * scale


def test_absorbing_layer_profile():
    """A uniform E (curl-free) in an absorbing box: one Maxwell step multiplies E by the
    damping profile prod_a (1 - 0.1 (d_a/L)^2) exactly, d_a the depth into the layer."""
    n, L = (20, 1, 24), 6
    s = make(2, n, bc=(1, 0, 1), absorb_cells=L, absorb_strength=0.1)
    s.set_field(EY, np.ones((24, 1, 20)))  # Ey is out of plane: its curl is only in B
    # Ey uniform -> dBx/dt = dEy/dz = 0 inside, but at the faces the zero outside makes a
    # jump; check the profile on interior cells away from the faces (i, k in [1, n-2])
    s.maxwell()
    out = s.get_field(EY)[:, 0, :]
    for k in range(1, 23):
        for i in range(1, 19):
            di = max(0, L - i, i - (20 - 1 - L))
            dk = max(0, L - k, k - (24 - 1 - L))
            f = (1 - 0.1 * (di / L) ** 2) * (1 - 0.1 * (dk / L) ** 2)
            assert abs(out[k, i] - f) < 1e-15


def test_sort_is_stable_by_tile():
    """Canonical order = stable sort by tile id (z slowest); recount by brute force."""
    rng = np.random.default_rng(2)
    n, tile = (24, 16, 20), (8, 4, 5)
    s = make(3, n, tile=tile)
    npart = 3000
    cell = rng.integers(0, 24 * 16 * 20, npart).astype(np.int32)
    ids = np.arange(npart, dtype=np.int32)
    s.set_particles(cell, rng.random((npart, 3)), np.zeros((npart, 3)), np.ones(npart), ids)
    p = s.get_particles()
    ci, cj, ck = cell % 24, (cell // 24) % 16, cell // (24 * 16)
    key = (ci // 8) + 3 * ((cj // 4) + 4 * (ck // 5))
    order = sorted(range(npart), key=lambda q: (key[q], q))
    assert np.array_equal(p["id"], ids[order])
    assert np.array_equal(p["cell"], cell[order])


def test_absorbing_particle_removal():
    s = make(3, (12, 12, 12), bc=(1, 1, 1), dt=0.5)
    cells = np.array([0, 5 + 12 * (5 + 12 * 5)], np.int32)
    s.set_particles(cells, np.array([[0.1, 0.5, 0.5], [0.5, 0.5, 0.5]]),
                    np.array([[-5.0, 0, 0], [0.1, 0, 0]]), np.ones(2))
    s.particle_phase()
    d = s.diagnostics()
    assert d["n_particles"] == 1 and d["n_lost"] == 1


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("ndim", [2, 3])
def test_gauss_law_residual_constant(order, ndim):
    """Esirkepov deposit + Yee: div E - rho is constant in time to round-off (periodic,
    unfiltered), a whole-loop pin of the deposit/field coupling and of their signs."""
    rng = np.random.default_rng(21)
    n = (16, 12, 16) if ndim == 3 else (24, 1, 20)
    s = make(ndim, n, dx=(1.0, 1.0, 1.0), dt=0.45 if ndim == 3 else 0.6, order=order, tile=(8, 4, 8))
    nc = s.n[0] * s.n[1] * s.n[2]
    ppc = 2
    cell = np.repeat(np.arange(nc), ppc).astype(np.int32)
    off = rng.random((cell.size, 3))
    if ndim == 2:
        off[:, 1] = 0
    u = rng.normal(0, 0.3, (cell.size, 3))
    s.set_particles(cell, off, u, np.full(cell.size, 1.0 / ppc))
    r0 = s.div_e() - s.rho()
    s.step(12)
    r1 = s.div_e() - s.rho()
    assert np.abs(r1 - r0).max() < 1e-12
    # the field energy grew from zero: the coupling did something
    assert s.diagnostics()["field_energy"] > 1e-6


@pytest.mark.parametrize("passes", [1, 3])
def test_gauss_law_with_filter_conserves_filtered_charge(passes):
    """With the current filtered, E changes by -dt div(F J) = -dt F div J (the binomial
    filter is a convolution, which commutes with the differences on a periodic grid), so
    div E - F rho is what stays constant, F the same 1-2-1 passes on the nodes; div E - rho
    does not."""
    rng = np.random.default_rng(22)
    n = (16, 12, 16)
    s2 = oracle.Sim(3, n, (0, 0, 0), (1.0, 1.0, 1.0), 0.45, order=2, filter_passes=passes, tile=(8, 4, 8))
    nc = n[0] * n[1] * n[2]
    cell = np.repeat(np.arange(nc), 2).astype(np.int32)
    off = rng.random((cell.size, 3))
    u = rng.normal(0, 0.3, (cell.size, 3))
    s2.set_particles(cell, off, u, np.full(cell.size, 0.5))

    def F(rho):
        f = rho.copy()
        for _ in range(passes):
            for ax in (2, 1, 0):
                f = 0.25 * np.roll(f, 1, ax) + 0.5 * f + 0.25 * np.roll(f, -1, ax)
        return f

    r0, q0 = s2.div_e() - F(s2.rho()), s2.div_e() - s2.rho()
    s2.step(12)
    r1, q1 = s2.div_e() - F(s2.rho()), s2.div_e() - s2.rho()
    assert np.abs(r1 - r0).max() < 1e-12
    assert np.abs(q1 - q0).max() > 1e-3


def test_diagnostics_closed_forms():
    s = make(3, (8, 8, 8), dx=(1.0, 0.5, 2.0))
    s.set_field(EY, np.full((8, 8, 8), 0.3))
    s.set_field(BZ, np.full((8, 8, 8), -0.2))
    u = np.array([[0.0, 0.0, 3.0], [1.0, 2.0, 2.0]])
    s.set_particles(np.array([0, 7], np.int32), np.full((2, 3), 0.5), u, np.array([2.0, 0.5]))
    d = s.diagnostics()
    V = 512 * 1.0
    assert abs(d["field_energy"] - 0.5 * (0.09 + 0.04) * V) < 1e-12
    assert abs(d["kinetic_energy"] - 2.5 * (math.sqrt(10) - 1)) < 1e-12  # both have gamma = sqrt(10)
    assert d["total_charge"] == -2.5 and d["n_particles"] == 2


def test_round_state_fp32_matches_float32_storage():
    """The FP32-storage helper rounds each stored value as a float32 cast does and keeps
    offsets below 1."""
    s = make(3, (4, 4, 4), dx=(1.0, 1.0, 1.0))
    rng = np.random.default_rng(41)
    cell = np.arange(3, dtype=np.int32)
    off = np.array([[0.1, 0.2, 0.3], [1 - 2 ** -30, 0.5, 0.25], [0.123456789123, 0.999999999, 0.0]])
    u = rng.normal(size=(3, 3)) * 1e3
    w = rng.random(3)
    s.set_particles(cell, off, u, w)
    f = rng.normal(size=(4, 4, 4))
    s.set_field(oracle.EX, f)
    s.round_state_fp32()
    p = s.get_particles()
    below = np.float64(np.nextafter(np.float32(1), np.float32(0)))
    ref_off = np.minimum(off.astype(np.float32).astype(np.float64), below)
    assert np.array_equal(p["off"], ref_off) and p["off"][1, 0] == below
    assert np.array_equal(p["u"], u.astype(np.float32).astype(np.float64))
    assert np.array_equal(p["w"], w.astype(np.float32).astype(np.float64))
    assert np.array_equal(s.get_field(oracle.EX), f.astype(np.float32).astype(np.float64))
