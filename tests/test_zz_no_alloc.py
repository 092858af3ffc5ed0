"""The charge-density read-out that allocates nothing gives the same density as the
regular read-out, and allocates nothing.

pic_get_rho_noalloc exists for callers that must not allocate device memory when they
read the density (a device-memory budget already committed, a call from inside another
library's memory pool, a loop that has to stay out of allocator locks): it deposits into
a fixed work grid the library owns instead of per-context memory.  The checks go through
the C ABI and compare it with pic_get_field(PIC_RHO) on two calls in a row, so a work grid
left dirty by the first call would show in the second -- for bare particles and for a
lab-frame plasma whose ion background the density includes -- and read the device's free
memory around the calls, in this process and in a fresh one where the read-out is the
first after pic_create.  This file is collected last so a failure here comes after every
other test has run.
"""
import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest

import paper_0909_5603_gb300 as pic
import synth

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def rho_noalloc(sim):
    out = np.full(sim.ncell, np.nan)
    st = pic.lib().pic_get_rho_noalloc(sim.h, out.ctypes.data_as(ctypes.c_void_p), out.size)
    if st != pic.PIC_OK:
        raise pic.PicError(st, pic.lib().pic_last_error(sim.h).decode())
    return out.reshape(sim.n[2], sim.n[1], sim.n[0])


def check_twice(sim):
    ref = sim.get_field(pic.PIC_RHO)
    scale = np.abs(ref).max()
    assert scale > 0
    for _ in range(2):
        got = rho_noalloc(sim)
        assert np.all(np.isfinite(got))
        # both deposit with FP64 atomics in a different order: FP64 round-off only
        assert np.abs(got - ref).max() <= 1e-12 * scale


@pytest.mark.parametrize("prec", [pic.PIC_PREC_FP64, pic.PIC_PREC_FP32])
def test_rho_noalloc_matches_regular_readout_twice(prec):
    pic.build()
    n = (40, 24, 32)
    sim = pic.Simulation(3, n, (0, 1, 0), (1.0, 0.9, 1.1), 0.45, order=2, precision=prec)
    parts = synth.random_particles(n, 3, 20000, 0.6, seed=77)
    sim.load_particles(parts["cell"], parts["off"], parts["u"], parts["w"], parts["id"])
    sim.step(3)
    check_twice(sim)


@pytest.mark.parametrize("prec", [pic.PIC_PREC_FP64, pic.PIC_PREC_FP32])
def test_rho_noalloc_lab_frame_plasma_with_ions(prec):
    """A boosted lab-frame plasma load: the density holds the electrons' deposit and the
    ion background streaming through the box (a separate kernel of the read-out)."""
    pic.build()
    w = synth.lwfa_stage((16, 16, 96), 13.0, 2, seed=11)
    sim = pic.Simulation(3, w["n"], (1, 1, 1), w["dx"], w["dt"], gamma_boost=13.0, order=2, precision=prec,
                         filter_passes=3, tile=(8, 8, 8))
    sim.load_lab_frame(laser=w["laser"], plasma=w["plasma"])
    sim.step(4)
    rho = sim.get_field(pic.PIC_RHO)
    assert rho.max() > 0 > rho.min()  # ions and electrons both present
    check_twice(sim)


def test_rho_noalloc_allocates_no_device_memory():
    """Free device memory is the same before and after several read-outs."""
    import torch

    pic.build()
    n = (32, 16, 24)
    sim = pic.Simulation(3, n, (0, 0, 0), (1.0, 1.0, 1.0), 0.5, order=1, precision=pic.PIC_PREC_FP32)
    parts = synth.random_particles(n, 3, 8000, 0.3, seed=5)
    sim.load_particles(parts["cell"], parts["off"], parts["u"], parts["w"], parts["id"])
    sim.step(2)
    sim.synchronize()
    rho_noalloc(sim)
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(5):
        rho_noalloc(sim)
    assert torch.cuda.mem_get_info()[0] == free0


FRESH = r"""
import sys
sys.path.insert(0, sys.argv[1]); sys.path.insert(0, sys.argv[1] + "/tests")
import ctypes, numpy as np, torch
import paper_0909_5603_gb300 as pic, synth
n = (24, 16, 20)
sim = pic.Simulation(3, n, (0, 0, 0), (1.0, 1.0, 1.0), 0.5, order=2, precision=pic.PIC_PREC_FP64)
p = synth.random_particles(n, 3, 6000, 0.3, seed=9)
sim.load_particles(p["cell"], p["off"], p["u"], p["w"], p["id"])
sim.step(1)
sim.synchronize()
free0 = torch.cuda.mem_get_info()[0]
out = np.zeros(sim.ncell)
st = pic.lib().pic_get_rho_noalloc(sim.h, out.ctypes.data_as(ctypes.c_void_p), out.size)
free1 = torch.cuda.mem_get_info()[0]
print(st, free0, free1, float(np.abs(out).max()))
"""


def test_rho_noalloc_first_call_after_create_allocates_nothing():
    """In a fresh process the first read-out after pic_create (which loads the work grid
    and the density kernels) leaves the device's free memory unchanged."""
    pic.build()
    r = subprocess.run([sys.executable, "-c", FRESH, ROOT], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    st, free0, free1, mx = r.stdout.split()[-4:]
    assert int(st) == pic.PIC_OK
    assert float(mx) > 0
    assert int(free1) == int(free0)


def test_rho_noalloc_rejects_grids_above_its_work_grid():
    pic.build()
    n = (128, 128, 72)  # 1,179,648 cells > 2^20
    sim = pic.Simulation(3, n, (0, 0, 0), (1.0, 1.0, 1.0), 0.5)
    with pytest.raises(pic.PicError) as e:
        rho_noalloc(sim)
    assert e.value.status == pic.PIC_ERR_ARG
    assert "exceeds the no-allocation work grid" in str(e.value)
