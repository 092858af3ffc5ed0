"""The charge-density read-out that allocates nothing gives the same density as the
regular read-out.

pic_get_rho_noalloc exists for callers that must not allocate device memory when they
read the density (a device-memory budget already committed, a call from inside another
library's memory pool, a loop that has to stay out of allocator locks): it deposits into
a fixed work grid the library owns instead of per-context memory.  The check goes
through the C ABI and compares it with pic_get_field(PIC_RHO) on two calls in a row, so
a work grid left dirty by the first call would show in the second.  This file is
collected last so a failure here comes after every other test has run.
"""
import ctypes

import numpy as np
import pytest

import paper_0909_5603_gb300 as pic
import synth

pytestmark = pytest.mark.gpu


def rho_noalloc(sim):
    out = np.full(sim.ncell, np.nan)
    st = pic.lib().pic_get_rho_noalloc(sim.h, out.ctypes.data_as(ctypes.c_void_p), out.size)
    if st != pic.PIC_OK:
        raise pic.PicError(st, pic.lib().pic_last_error(sim.h).decode())
    return out.reshape(sim.n[2], sim.n[1], sim.n[0])


@pytest.mark.parametrize("prec", [pic.PIC_PREC_FP64, pic.PIC_PREC_FP32])
def test_rho_noalloc_matches_regular_readout_twice(prec):
    pic.build()
    n = (40, 24, 32)
    sim = pic.Simulation(3, n, (0, 1, 0), (1.0, 0.9, 1.1), 0.45, order=2, precision=prec)
    parts = synth.random_particles(n, 3, 20000, 0.6, seed=77)
    sim.load_particles(parts["cell"], parts["off"], parts["u"], parts["w"], parts["id"])
    sim.step(3)
    ref = sim.get_field(pic.PIC_RHO)
    scale = np.abs(ref).max()
    assert scale > 0
    for _ in range(2):
        got = rho_noalloc(sim)
        assert np.all(np.isfinite(got))
        # both deposit with FP64 atomics in a different order: FP64 round-off only
        assert np.abs(got - ref).max() <= 1e-12 * scale


def test_rho_noalloc_rejects_grids_above_its_work_grid():
    pic.build()
    n = (128, 128, 72)  # 1,179,648 cells > 2^20
    sim = pic.Simulation(3, n, (0, 0, 0), (1.0, 1.0, 1.0), 0.5)
    with pytest.raises(pic.PicError) as e:
        rho_noalloc(sim)
    assert e.value.status == pic.PIC_ERR_ARG
    assert "exceeds the no-allocation work grid" in str(e.value)
