"""Beam injection through a lab-fixed plane (Sec. 2 of Vay et al.) on the GPU against the
oracle: a lab-frame laser, plasma (with its ion background) and beam loaded into a
gamma_b = 4 frame with the plane crossing the beam, so that part of the beam starts
frozen and is injected during the run.  FP64 within 1e-12 (the frozen/active decision
is taken in FP64 on both sides, so the particle states agree cell for cell), FP32
within 1e-5 (normwise); frozen momenta bit for bit; the id threshold; a batch member
with a plane steps as it does alone; the setter's argument checks."""
import numpy as np
import pytest

import oracle
import paper_0909_5603_gb300 as pic

pytestmark = pytest.mark.gpu

FP32, FP64 = pic.PIC_PREC_FP32, pic.PIC_PREC_FP64
FIELDS = [pic.PIC_EX, pic.PIC_EY, pic.PIC_EZ, pic.PIC_BX, pic.PIC_BY, pic.PIC_BZ, pic.PIC_JX, pic.PIC_JY,
          pic.PIC_JZ]
GB = 4.0
LASER = (1.0, 1.0, 4.0, 1.0, 1.0)
PLASMA = (0.05, 0.5, 3.0, 2, (0.01, 0.01, 0.01), 4)
BEAM = (400, 20.0, 0.01, 1.0, 0.3, 2.0, 1.0, 5)
Z_LAB = 72.0  # the plane sits at z' = 18 at t' = 0, inside the beam


@pytest.fixture(scope="module", autouse=True)
def built():
    pic.build()
    oracle.build()


def rel2(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300))


def relinf(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(b).max(), 1e-300))


CASES = [(3, (8, 8, 64), (1, 1, 1)), (2, (24, 1, 64), (1, 0, 1))]


def pair(ndim, n, bc, prec, plasma=True):
    dz, dt = 0.5, 0.2
    g = pic.Simulation(ndim, n, bc, (1.0, 1.0, dz), dt, gamma_boost=GB, order=2, precision=prec, filter_passes=1,
                       absorb_cells=4)
    o = oracle.Sim(ndim, n, bc, (1.0, 1.0, dz), dt, order=2, filter_passes=1, absorb_cells=4,
                   tile=(8, 8, 8) if ndim == 3 else (16, 1, 16))
    pl = PLASMA if plasma else None
    g.set_injection(Z_LAB)
    g.load_lab_frame(laser=LASER, plasma=pl, beam=BEAM)
    o.load_lab_frame(GB, laser=LASER, plasma=[*pl[:4], *pl[4], pl[5]] if pl else None, beam=BEAM)
    o.set_injection(GB, Z_LAB)
    return g, o


@pytest.mark.parametrize("ndim,n,bc", CASES)
def test_injection_fp64_matches_oracle(ndim, n, bc):
    g, o = pair(ndim, n, bc, FP64)
    assert o.num_frozen() > 50
    for chunk in (10, 20):
        g.step(chunk)
        o.step(chunk)
        for c in FIELDS:
            fo = o.get_field(c)
            if np.abs(fo).max() > 0:
                assert relinf(g.get_field(c), fo) <= 1e-12, c
        pg, po = g.get_particles(), o.get_particles()
        assert np.array_equal(pg["id"], po["id"]) and np.array_equal(pg["cell"], po["cell"])
        assert relinf(pg["u"], po["u"]) <= 1e-12
        assert relinf(pg["off"], po["off"]) <= 1e-12
    assert o.num_frozen() < 50  # the plane has swept most of the beam


@pytest.mark.parametrize("ndim,n,bc", CASES)
def test_injection_fp32_matches_oracle(ndim, n, bc):
    g, o = pair(ndim, n, bc, FP32)
    g.step(30)
    o.step(30)
    for c in FIELDS:
        fo = o.get_field(c)
        if np.abs(fo).max() > 0:
            assert rel2(g.get_field(c), fo) <= 1e-5, c
    pg, po = g.get_particles(), o.get_particles()
    common, ig, io = np.intersect1d(pg["id"], po["id"], return_indices=True)
    assert max(pg["id"].size, po["id"].size) - common.size <= 2
    assert rel2(pg["u"][ig], po["u"][io]) <= 1e-5


@pytest.mark.parametrize("prec", [FP64, FP32])
def test_frozen_momentum_kept_bit_for_bit_and_id_threshold(prec):
    n = (8, 1, 64)
    g = pic.Simulation(2, n, (0, 0, 0), (1.0, 1.0, 0.5), 0.1, gamma_boost=2.0, order=1, precision=prec,
                       tile=(8, 1, 16))
    cell = np.array([1 + 8 * 10, 1 + 8 * 10, 1 + 8 * 60], np.int32)
    off = np.array([[0.5, 0, 0.5]] * 3)
    u = np.array([[0.0, 0.0, 1.0]] * 3)
    g.load_particles(cell, off, u, np.zeros(3), ids=np.array([3, 4, 5], np.int32))
    g.set_field(pic.PIC_EZ, np.full((n[2], n[1], n[0]), 0.1))
    # plane at z' = 25 - beta_b t': ids 3 and 4 upstream (z' = 5.25), id 5 downstream (30.25)
    g.set_injection(50.0, first_id=4)
    g.step(3)
    p = g.get_particles()
    by_id = {int(i): uu for i, uu in zip(p["id"], p["u"])}
    assert by_id[4][2] == 1.0 and by_id[4][0] == 0.0  # frozen: untouched
    tol = 1e-12 if prec == FP64 else 1e-6
    for i in (3, 5):  # pushed: q E dt per step
        assert abs(by_id[i][2] - (1.0 - 3 * 0.1 * 0.1)) < tol, i
    # frozen particles drift: z advances by v dt per step
    zs = {int(i): (c // n[0] + o_[2]) * 0.5 for i, c, o_ in zip(p["id"], p["cell"], p["off"])}
    assert abs(zs[4] - (5.25 + 3 * 0.1 / np.sqrt(2.0))) < (1e-12 if prec == FP64 else 1e-5)
    g.set_injection(0.0, enable=False)
    g.step(1)
    p = g.get_particles()
    assert {int(i): uu for i, uu in zip(p["id"], p["u"])}[4][2] < 1.0


def test_batch_member_with_plane_steps_as_alone():
    alone, o = pair(*CASES[0], FP64)
    del o
    member, _ = pair(*CASES[0], FP64)
    other, _ = pair(*CASES[0], FP64)
    other.set_injection(0.0, enable=False)
    alone.step(15)
    batch = pic.Batch([member, other])
    batch.step(15)
    batch.synchronize()
    for c in FIELDS:
        fa, fb = alone.get_field(c), member.get_field(c)
        assert np.abs(fa - fb).max() <= 1e-12 * max(np.abs(fa).max(), 1e-300), c
    pa, pb, po = alone.get_particles(), member.get_particles(), other.get_particles()
    assert np.array_equal(pa["id"], pb["id"]) and np.array_equal(pa["cell"], pb["cell"])
    assert np.abs(pa["u"] - pb["u"]).max() <= 1e-12 * np.abs(pa["u"]).max()
    assert not np.array_equal(pa["cell"], po["cell"]) or np.abs(pa["u"] - po["u"]).max() > 0


def test_set_injection_argument_checks():
    g = pic.Simulation(3, (8, 8, 16), (1, 1, 1), (1.0, 1.0, 1.0), 0.3, gamma_boost=2.0, track_ids=False)
    with pytest.raises(pic.PicError):
        g.set_injection(10.0)
    g.set_injection(10.0, enable=False)  # turning it off needs no ids
    h = pic.Simulation(3, (8, 8, 16), (1, 1, 1), (1.0, 1.0, 1.0), 0.3, gamma_boost=2.0)
    with pytest.raises(pic.PicError):
        h.set_injection(float("nan"))
    h.set_injection(10.0)
