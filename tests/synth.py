"""Seeded synthetic inputs shared by the CUDA-path tests, the oracle tests and the smoke
check.  Holds no arithmetic of the PIC method: only random particle and field arrays in
the layout of include/pic.h (values chosen exactly representable in FP32, so an FP32
store of them is lossless).
"""
import numpy as np


def f32(a):
    return np.asarray(a, np.float32).astype(np.float64)


def uniform_plasma(n, ndim, ppc, sigma_u, seed, weight=None, drift=(0.0, 0.0, 0.0)):
    """ppc particles per cell at uniform random in-cell offsets, Gaussian momenta
    (sigma_u per component, plus a drift), equal weights (default 1/ppc)."""
    rng = np.random.default_rng(seed)
    n = list(n)
    if ndim == 2:
        n[1] = 1
    ncell = n[0] * n[1] * n[2]
    cell = np.repeat(np.arange(ncell, dtype=np.int32), ppc)
    npart = cell.size
    off = f32(rng.random((npart, 3), dtype=np.float32))
    if ndim == 2:
        off[:, 1] = 0.0
    u = f32(rng.normal(0.0, sigma_u, (npart, 3)) + np.asarray(drift))
    w = np.full(npart, (1.0 / ppc) if weight is None else weight)
    return dict(cell=cell, off=off, u=u, w=f32(w), id=np.arange(npart, dtype=np.int32))


def random_particles(n, ndim, npart, sigma_u, seed):
    """npart particles in random cells (uneven tile populations, empty tiles possible)."""
    rng = np.random.default_rng(seed)
    n = list(n)
    if ndim == 2:
        n[1] = 1
    ncell = n[0] * n[1] * n[2]
    cell = rng.integers(0, ncell, npart).astype(np.int32)
    off = f32(rng.random((npart, 3), dtype=np.float32))
    if ndim == 2:
        off[:, 1] = 0.0
    u = f32(rng.normal(0.0, sigma_u, (npart, 3)))
    w = f32(rng.uniform(0.5, 1.5, npart))
    return dict(cell=cell, off=off, u=u, w=w, id=np.arange(npart, dtype=np.int32))


def smooth_fields(n, ndim, amp, seed, modes=3):
    """Six smooth periodic random fields (sums of a few Fourier modes), (n2, n1, n0) each."""
    rng = np.random.default_rng(seed)
    n = list(n)
    if ndim == 2:
        n[1] = 1
    k, j, i = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    out = []
    for _ in range(6):
        f = np.zeros(i.shape)
        for _m in range(modes):
            m = rng.integers(0, 3, 3)
            ph = rng.uniform(0, 2 * np.pi)
            f += rng.normal() * np.cos(2 * np.pi * (m[0] * i / n[0] + m[1] * j / n[1] + m[2] * k / n[2]) + ph)
        out.append(f32(amp * f))
    return out


def lwfa_stage(n=(128, 128, 1024), gamma_boost=13.0, ppc=2, seed=3, lambda0=1.0):
    """Lab-frame inputs of the boosted laser-wakefield stage (normalised units, c = 1):
    plasma at n/n_c = 1/900 behind a linear up-ramp two boosted cells long (in lab length,
    2 dz gamma_b), Gaussian laser a0 = 2, waist 20 lambda0, 10 periods long, centred two
    durations ahead of the plasma.  The boosted grid resolves the Doppler-stretched laser
    wavelength gamma_b (1 + beta_b) lambda0 with 16 cells; transverse cells are 2 lambda0
    (10 across the waist); dt = dz / 2, capped at 0.9 of the 3D Yee Courant limit (the cap
    binds from gamma_b ~ 25 on, where dz outgrows the transverse cells).  Returns the grid
    and the tuples that Simulation.load_lab_frame takes."""
    b = np.sqrt(1.0 - 1.0 / gamma_boost ** 2)
    dz = gamma_boost * (1.0 + b) * lambda0 / 16.0
    dx = 2.0 * lambda0
    k0 = 2.0 * np.pi / lambda0
    n_c = k0 * k0  # critical density for q = m = eps0 = c = 1
    duration = 10.0 * lambda0
    laser = (2.0, lambda0, 20.0 * lambda0, duration, 2.0 * duration)
    plasma = (n_c / 900.0, 0.0, 2.0 * dz * gamma_boost, ppc, (0.0, 0.0, 0.0), seed)
    courant = 1.0 / np.sqrt(2.0 / dx ** 2 + 1.0 / dz ** 2)
    dt = min(0.5 * dz, 0.9 * courant)
    return dict(n=tuple(n), dx=(dx, dx, dz), dt=dt, gamma_boost=gamma_boost, laser=laser, plasma=plasma)


def scan_instance(i, seed_base=5000, tile=16):
    """Instance i of the batched 2D3V boosted-frame scan (seeded with seed_base + i):
    N x N cells with log2 N uniform in [6, 9] (N rounded to a multiple of the tile),
    1-16 electrons per cell, gamma_b uniform in [1, 50], n/n_c uniform in [1e-4, 1e-2];
    a cold plasma filling the periodic box with its ions and an a0 = 1 laser pulse two
    wavelengths long in the middle; cells and step as in lwfa_stage (dz = lambda' / 16,
    dx = 2 lambda0, dt = dz / 2 capped at 0.9 of the 2D Courant limit)."""
    rng = np.random.default_rng(seed_base + i)
    n_side = int(max(tile, round(2.0 ** rng.uniform(6.0, 9.0) / tile) * tile))
    ppc = int(rng.integers(1, 17))
    gb = float(rng.uniform(1.0, 50.0))
    dens = float(rng.uniform(1e-4, 1e-2))
    b = np.sqrt(1.0 - 1.0 / gb ** 2)
    doppler = gb * (1.0 + b)
    dz = doppler / 16.0
    dx = 2.0
    dt = min(0.5 * dz, 0.9 / np.sqrt(1.0 / dx ** 2 + 1.0 / dz ** 2))
    n_c = (2.0 * np.pi) ** 2
    lz = n_side * dz
    laser = (1.0, 1.0, 0.25 * n_side * dx, 2.0, 0.5 * lz / doppler)
    plasma = (dens * n_c, -1e9, 0.0, ppc, (0.0, 0.0, 0.0), seed_base + i)
    return dict(n=(n_side, 1, n_side), dx=(dx, 1.0, dz), dt=dt, gamma_boost=gb, laser=laser, plasma=plasma,
                ppc=ppc)
