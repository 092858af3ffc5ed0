"""FP64 CPU oracle of the boosted-frame explicit EM-PIC step (ctypes wrapper).

TEST INFRASTRUCTURE ONLY.  Imported by the test suite, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py``; never by the product path.  It shares no code
with the CUDA library (``paper_0909_5603_gb300``) and imports nothing from it.

The arithmetic lives in ``pic_oracle.c`` (plain C, FP64, ``-ffp-contract=off``); each
function there cites the passage of Vay et al. (arXiv:0909.5603, Sec. 2) or the named
published method it restates.  This module only marshals arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBDIR = os.path.join(_HERE, "lib")
_LIB = os.path.join(_LIBDIR, "libpic_oracle.so")
_SRC = [os.path.join(_HERE, "pic_oracle.c")]
_HDR = [os.path.join(_HERE, "pic_oracle.h")]

EX, EY, EZ, BX, BY, BZ, JX, JY, JZ = range(9)
PERIODIC, ABSORBING = 0, 1
VAY, BORIS = 0, 1
SOLVER_YEE, SOLVER_CK = 0, 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, so host arithmetic matches on
    x86-64 and aarch64)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    newest = max(os.path.getmtime(p) for p in _SRC + _HDR)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= newest:
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", tmp] + _SRC + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None

_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_I3 = ctypes.c_int * 3
_D3 = ctypes.c_double * 3


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        vp = ctypes.c_void_p
        L.orc_shape.restype = ctypes.c_double
        L.orc_shape.argtypes = [ctypes.c_int, ctypes.c_double]
        for name in ("orc_push_vay", "orc_push_boris"):
            getattr(L, name).restype = None
            getattr(L, name).argtypes = [_f64p, _f64p, _f64p, ctypes.c_double, ctypes.c_double]
        L.orc_boost_fields.restype = None
        L.orc_boost_fields.argtypes = [ctypes.c_double, _f64p, _f64p, _f64p, _f64p]
        L.orc_boost_event.restype = None
        L.orc_boost_event.argtypes = [ctypes.c_double, _f64p, _f64p, _f64p, _f64p]
        L.orc_splitmix64.restype = ctypes.c_uint64
        L.orc_splitmix64.argtypes = [ctypes.c_uint64] * 3
        L.orc_uniform.restype = ctypes.c_double
        L.orc_uniform.argtypes = [ctypes.c_uint64] * 3
        L.orc_normal.restype = ctypes.c_double
        L.orc_normal.argtypes = [ctypes.c_uint64] * 3
        L.orc_create.restype = vp
        L.orc_create.argtypes = [ctypes.c_int, _I3, _I3, _D3, ctypes.c_double, ctypes.c_int,
                                 ctypes.c_int, ctypes.c_int, _I3, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_int, ctypes.c_double]
        L.orc_destroy.restype = None
        L.orc_destroy.argtypes = [vp]
        L.orc_set_field.restype = None
        L.orc_set_field.argtypes = [vp, ctypes.c_int, _f64p]
        L.orc_get_field.restype = None
        L.orc_get_field.argtypes = [vp, ctypes.c_int, _f64p]
        L.orc_set_particles.restype = ctypes.c_int
        L.orc_set_particles.argtypes = [vp, ctypes.c_int64, _i32p, _f64p, _f64p, _f64p, _i32p]
        L.orc_num_particles.restype = ctypes.c_int64
        L.orc_num_particles.argtypes = [vp]
        L.orc_get_particles.restype = None
        L.orc_get_particles.argtypes = [vp, _i32p, _f64p, _f64p, _f64p, _i32p]
        for name in ("orc_sort", "orc_particle_phase", "orc_filter", "orc_maxwell"):
            getattr(L, name).restype = None
            getattr(L, name).argtypes = [vp]
        L.orc_gather.restype = None
        L.orc_gather.argtypes = [vp, ctypes.c_int32, _f64p, _f64p, _f64p]
        L.orc_step.restype = None
        L.orc_step.argtypes = [vp, ctypes.c_int]
        L.orc_rho.restype = None
        L.orc_rho.argtypes = [vp, _f64p]
        L.orc_div_e.restype = None
        L.orc_div_e.argtypes = [vp, _f64p]
        L.orc_diagnostics.restype = None
        L.orc_diagnostics.argtypes = [vp, _f64p]
        L.orc_load_lab_frame.restype = ctypes.c_int
        L.orc_load_lab_frame.argtypes = [vp, ctypes.c_double, vp, vp, vp]
        L.orc_beam_self_field.restype = ctypes.c_int
        L.orc_beam_self_field.argtypes = [vp, _f64p, ctypes.c_double, ctypes.c_double]
        L.orc_set_solver.restype = None
        L.orc_set_solver.argtypes = [vp, ctypes.c_int]
        L.orc_station_record.restype = ctypes.c_int
        L.orc_station_record.argtypes = [vp, ctypes.c_double, ctypes.c_double, _f64p, _f64p]
        L.orc_round_state_fp32.restype = None
        L.orc_round_state_fp32.argtypes = [vp]
        L.orc_set_injection.restype = None
        L.orc_set_injection.argtypes = [vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int32]
        L.orc_num_frozen.restype = ctypes.c_int64
        L.orc_num_frozen.argtypes = [vp]
        L.orc_set_antenna.restype = None
        L.orc_set_antenna.argtypes = [vp, ctypes.c_int, ctypes.c_double, vp, ctypes.c_double]
        L.orc_ion_integral.restype = ctypes.c_double
        L.orc_ion_integral.argtypes = [vp, ctypes.c_double, ctypes.c_double]
        _lib = L
    return _lib


def shape(order: int, x: float) -> float:
    return lib().orc_shape(order, float(x))


def push_vay(u, E, B, q_over_m, dt):
    """One Vay push; returns u^{n+1/2} (Sec. 2, VayPOP08)."""
    u = np.array(u, dtype=np.float64)
    lib().orc_push_vay(u, np.asarray(E, np.float64), np.asarray(B, np.float64), q_over_m, dt)
    return u


def push_boris(u, E, B, q_over_m, dt):
    """One Boris push; returns u^{n+1/2} (Sec. 2, BorisICNSP)."""
    u = np.array(u, dtype=np.float64)
    lib().orc_push_boris(u, np.asarray(E, np.float64), np.asarray(B, np.float64), q_over_m, dt)
    return u


def boost_fields(gamma_b, E, B):
    Ep = np.zeros(3)
    Bp = np.zeros(3)
    lib().orc_boost_fields(gamma_b, np.asarray(E, np.float64), np.asarray(B, np.float64), Ep, Bp)
    return Ep, Bp


def boost_event(gamma_b, tx, u):
    txp = np.zeros(4)
    up = np.zeros(3)
    lib().orc_boost_event(gamma_b, np.asarray(tx, np.float64), np.asarray(u, np.float64), txp, up)
    return txp, up


def splitmix64(seed, stream, counter):
    return lib().orc_splitmix64(seed, stream, counter)


def uniform(seed, stream, counter):
    return lib().orc_uniform(seed, stream, counter)


def normal(seed, stream, counter):
    return lib().orc_normal(seed, stream, counter)


class Sim:
    """One FP64 CPU simulation instance (same conventions as the CUDA library)."""

    def __init__(self, ndim, n, bc, dx, dt, order=1, pusher=VAY, filter_passes=0,
                 tile=(8, 8, 8), q=-1.0, m=1.0, absorb_cells=16, absorb_strength=0.1, solver=0):
        n = list(n)
        if ndim == 2:
            n[1] = 1
        self.ndim = ndim
        self.n = tuple(int(v) for v in n)
        self.ncell = self.n[0] * self.n[1] * self.n[2]
        self._h = lib().orc_create(ndim, _I3(*self.n), _I3(*bc), _D3(*dx), dt, order, pusher,
                                   filter_passes, _I3(*tile), q, m, absorb_cells, absorb_strength)
        if solver:
            lib().orc_set_solver(self._h, int(solver))

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.orc_destroy(self._h)
            self._h = None

    def set_field(self, comp, arr):
        a = np.ascontiguousarray(np.asarray(arr, dtype=np.float64).reshape(-1))
        assert a.size == self.ncell
        lib().orc_set_field(self._h, comp, a)

    def get_field(self, comp):
        out = np.zeros(self.ncell)
        lib().orc_get_field(self._h, comp, out)
        return out.reshape(self.n[2], self.n[1], self.n[0])

    def set_particles(self, cell, off, u, w, ids=None):
        cell = np.ascontiguousarray(cell, dtype=np.int32)
        np_ = cell.size
        off = np.ascontiguousarray(np.asarray(off, np.float64).reshape(np_, 3))
        u = np.ascontiguousarray(np.asarray(u, np.float64).reshape(np_, 3))
        w = np.ascontiguousarray(w, dtype=np.float64)
        ids = np.ascontiguousarray(np.arange(np_) if ids is None else ids, dtype=np.int32)
        rc = lib().orc_set_particles(self._h, np_, cell, off, u, w, ids)
        if rc != 0:
            raise ValueError(f"orc_set_particles rejected the input ({rc})")

    def num_particles(self):
        return int(lib().orc_num_particles(self._h))

    def get_particles(self):
        n = self.num_particles()
        cell = np.zeros(n, np.int32)
        off = np.zeros((n, 3))
        u = np.zeros((n, 3))
        w = np.zeros(n)
        ids = np.zeros(n, np.int32)
        lib().orc_get_particles(self._h, cell, off, u, w, ids)
        return dict(cell=cell, off=off, u=u, w=w, id=ids)

    def gather(self, cell, off):
        E = np.zeros(3)
        B = np.zeros(3)
        lib().orc_gather(self._h, int(cell), np.asarray(off, np.float64), E, B)
        return E, B

    def sort(self):
        lib().orc_sort(self._h)

    def particle_phase(self):
        lib().orc_particle_phase(self._h)

    def filter(self):
        lib().orc_filter(self._h)

    def maxwell(self):
        lib().orc_maxwell(self._h)

    def step(self, n=1):
        lib().orc_step(self._h, n)

    def rho(self):
        out = np.zeros(self.ncell)
        lib().orc_rho(self._h, out)
        return out.reshape(self.n[2], self.n[1], self.n[0])

    def beam_self_field(self, rho, gamma, beta):
        """Adds the self-field of node charge density rho (n2, n1, n0) moving at beta z."""
        r = np.ascontiguousarray(np.asarray(rho, np.float64).ravel())
        lib().orc_beam_self_field(self._h, r, float(gamma), float(beta))

    def station_record(self, gamma_b, z_lab):
        """Lab-frame station at z_lab now: (t_lab, fields (6, n2=1.., n1, n0)) or None."""
        out = np.zeros(6 * self.n[0] * self.n[1])
        t = np.zeros(1)
        if not lib().orc_station_record(self._h, float(gamma_b), float(z_lab), out, t):
            return None
        return float(t[0]), out.reshape(6, self.n[1], self.n[0])

    def set_injection(self, gamma_b, z_lab, first_id=-1, enable=True):
        """Beam injection through the lab plane z_lab: beam particles (id >= first_id, or
        the last lab-frame load's beam) upstream of it are frozen."""
        lib().orc_set_injection(self._h, int(bool(enable)), float(gamma_b), float(z_lab), int(first_id))

    def set_antenna(self, gamma_b, laser, z_lab, enable=True):
        """Laser antenna on the lab plane z_lab: laser = (a0, lambda0, waist, duration,
        z_center) of the lab pulse it emits forward (None or enable=False: off)."""
        if laser is None or not enable:
            lib().orc_set_antenna(self._h, 0, float(gamma_b), None, 0.0)
            return
        a = (ctypes.c_double * 5)(*[float(v) for v in laser])
        lib().orc_set_antenna(self._h, 1, float(gamma_b), ctypes.cast(a, ctypes.c_void_p), float(z_lab))

    def num_frozen(self):
        return int(lib().orc_num_frozen(self._h))

    def round_state_fp32(self):
        """Rounds the stored state to FP32 (the storage of an FP32 implementation)."""
        lib().orc_round_state_fp32(self._h)

    def ion_integral(self, a, b):
        """Ion-background charge between box coordinates a < b at t' = 0 (per unit area)."""
        return lib().orc_ion_integral(self._h, float(a), float(b))

    def div_e(self):
        out = np.zeros(self.ncell)
        lib().orc_div_e(self._h, out)
        return out.reshape(self.n[2], self.n[1], self.n[0])

    def diagnostics(self):
        out = np.zeros(8)
        lib().orc_diagnostics(self._h, out)
        return dict(field_energy=out[0], kinetic_energy=out[1], total_charge=out[2],
                    n_particles=int(out[3]), n_lost=int(out[4]), step=int(out[5]))

    def load_lab_frame(self, gamma_b, laser=None, plasma=None, beam=None):
        def arr(x, k):
            if x is None:
                return None, None
            a = (ctypes.c_double * k)(*[float(v) for v in x])
            return a, ctypes.cast(a, ctypes.c_void_p)
        la, lp = arr(laser, 5)
        pa, pp = arr(plasma, 8)
        ba, bp = arr(beam, 8)
        return lib().orc_load_lab_frame(self._h, gamma_b, lp, pp, bp)
