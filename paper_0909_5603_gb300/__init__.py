"""GB300 (sm_103a) boosted-frame explicit electromagnetic PIC step -- Python binding.

A thin ctypes layer over the C ABI in ``include/pic.h`` (``lib/libpic.so``): the
functions keep the C names (``pic_create``, ``pic_step`` ...) and only marshal
arguments.  Every step of the method runs in the library's CUDA kernels; PyTorch only
supplies device memory (through the allocator hooks of ``pic_options``) and the CUDA
stream.  There is no CPU fallback: without the built library every call raises.

The method is the one of Vay et al., "Speeding up simulations of relativistic systems
using an optimal boosted frame" (arXiv:0909.5603, Sec. 2): lab-frame inputs transformed
to a Lorentz-boosted frame, then field gather, Vay pusher, charge-conserving current
deposit, binomial filtering and the Yee Maxwell update in that frame.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libpic.so")

PIC_OK, PIC_ERR_ARG, PIC_ERR_CFL, PIC_ERR_CUDA, PIC_ERR_OOM, PIC_ERR_STATE = 0, 1, 2, 3, 4, 5
PIC_ERR_PARTICLE_SPEED, PIC_ERR_TIMEOUT, PIC_ERR_NAN, PIC_ERR_UNSUPPORTED, PIC_ERR_INTERNAL = 6, 7, 8, 9, 10
PIC_PERIODIC, PIC_ABSORBING = 0, 1
PIC_PREC_FP32, PIC_PREC_FP64 = 0, 1
PIC_PUSHER_VAY, PIC_PUSHER_BORIS = 0, 1
PIC_SOLVER_YEE, PIC_SOLVER_CK = 0, 1
PIC_EX, PIC_EY, PIC_EZ, PIC_BX, PIC_BY, PIC_BZ, PIC_JX, PIC_JY, PIC_JZ, PIC_RHO, PIC_DIVE = range(11)
PIC_PHASE_PARTICLES, PIC_PHASE_FILTER, PIC_PHASE_MAXWELL, PIC_PHASE_ALL = 1, 2, 4, 7

EXPORTED = ["pic_default_options", "pic_create", "pic_destroy", "pic_last_error", "pic_load_lab_frame",
            "pic_load_particles", "pic_set_field", "pic_step", "pic_run_phases", "pic_get_field",
            "pic_num_particles", "pic_get_particles", "pic_get_diagnostics", "pic_set_profiling",
            "pic_get_timings", "pic_synchronize", "pic_batch_create", "pic_get_rho_noalloc", "pic_autotune",
            "pic_set_stations", "pic_get_station", "pic_set_injection", "pic_set_laser_antenna",
            "pic_get_fields", "pic_get_gauss_residual", "pic_get_planes", "pic_put_planes",
            "pic_extract_particles", "pic_add_particles", "pic_adopt_slab", "pic_batch_set_persistent",
            "pic_batch_autotune", "pic_get_planes_n", "pic_put_planes_n", "pic_load_particles_stored",
            "pic_get_particles_stored"]
PIC_NOALLOC_RHO_MAX_CELLS = 1 << 20


class PicError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"pic status {status}: {msg}")
        self.status = status


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class pic_grid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("n", ctypes.c_int * 3), ("bc", ctypes.c_int * 3)]


class pic_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("pusher", ctypes.c_int), ("filter_passes", ctypes.c_int),
                ("tile", ctypes.c_int * 3), ("threads", ctypes.c_int), ("absorb_cells", ctypes.c_int),
                ("absorb_strength", ctypes.c_double), ("charge", ctypes.c_double), ("mass", ctypes.c_double),
                ("track_ids", ctypes.c_int), ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_user", ctypes.c_void_p),
                ("stream", ctypes.c_void_p), ("device", ctypes.c_int), ("solver", ctypes.c_int),
                ("absorb_faces", ctypes.c_int)]


class pic_diag(ctypes.Structure):
    _fields_ = [("step", ctypes.c_int64), ("t", ctypes.c_double), ("field_energy", ctypes.c_double),
                ("kinetic_energy", ctypes.c_double), ("total_charge", ctypes.c_double),
                ("n_particles", ctypes.c_int64), ("n_lost", ctypes.c_int64), ("error_flags", ctypes.c_int32)]


class pic_timings(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_int64), ("ms_particles", ctypes.c_double), ("ms_scan", ctypes.c_double),
                ("ms_filter", ctypes.c_double), ("ms_maxwell", ctypes.c_double), ("ms_other", ctypes.c_double),
                ("launches", ctypes.c_int64)]


class pic_laser_lab(ctypes.Structure):
    _fields_ = [("a0", ctypes.c_double), ("lambda0", ctypes.c_double), ("waist", ctypes.c_double),
                ("duration", ctypes.c_double), ("z_center", ctypes.c_double)]


class pic_plasma_lab(ctypes.Structure):
    _fields_ = [("n0", ctypes.c_double), ("z_start", ctypes.c_double), ("ramp_len", ctypes.c_double),
                ("ppc", ctypes.c_int), ("u_th", ctypes.c_double * 3), ("seed", ctypes.c_uint64)]


class pic_beam_lab(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("gamma", ctypes.c_double), ("rel_spread", ctypes.c_double),
                ("sigma_r", ctypes.c_double), ("sigma_z", ctypes.c_double), ("z0", ctypes.c_double),
                ("total_weight", ctypes.c_double), ("seed", ctypes.c_uint64)]


_lib = None


def build(force: bool = False) -> str:
    from . import native_build
    return native_build.build(force=force)


def lib():
    """The loaded library; raises when it has not been built (there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: run paper_0909_5603_gb300.build() first")
        L = ctypes.CDLL(LIB_PATH)
        P = ctypes.POINTER
        vp = ctypes.c_void_p
        st = ctypes.c_int
        L.pic_default_options.restype = None
        L.pic_default_options.argtypes = [P(pic_options)]
        L.pic_create.restype = st
        L.pic_create.argtypes = [P(pic_grid), P(ctypes.c_double), ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                 P(pic_options), P(vp)]
        L.pic_destroy.restype = None
        L.pic_destroy.argtypes = [vp]
        L.pic_last_error.restype = ctypes.c_char_p
        L.pic_last_error.argtypes = [vp]
        L.pic_load_lab_frame.restype = st
        L.pic_load_lab_frame.argtypes = [vp, P(pic_laser_lab), P(pic_plasma_lab), P(pic_beam_lab)]
        L.pic_load_particles.restype = st
        L.pic_load_particles.argtypes = [vp, ctypes.c_int64, vp, vp, vp, vp, vp]
        L.pic_set_field.restype = st
        L.pic_set_field.argtypes = [vp, ctypes.c_int, vp, ctypes.c_size_t]
        L.pic_step.restype = st
        L.pic_step.argtypes = [vp, ctypes.c_int]
        L.pic_run_phases.restype = st
        L.pic_run_phases.argtypes = [vp, ctypes.c_int]
        L.pic_get_field.restype = st
        L.pic_get_field.argtypes = [vp, ctypes.c_int, vp, ctypes.c_size_t]
        L.pic_num_particles.restype = st
        L.pic_num_particles.argtypes = [vp, P(ctypes.c_int64)]
        L.pic_get_particles.restype = st
        L.pic_get_particles.argtypes = [vp, vp, vp, vp, vp, vp, ctypes.c_int64, P(ctypes.c_int64)]
        L.pic_get_particles_stored.restype = st
        L.pic_get_particles_stored.argtypes = [vp, vp, vp, vp, vp, vp, ctypes.c_int64, P(ctypes.c_int64)]
        L.pic_load_particles_stored.restype = st
        L.pic_load_particles_stored.argtypes = [vp, ctypes.c_int64, vp, vp, vp, vp, vp]
        L.pic_get_diagnostics.restype = st
        L.pic_get_diagnostics.argtypes = [vp, P(pic_diag)]
        L.pic_set_profiling.restype = st
        L.pic_set_profiling.argtypes = [vp, ctypes.c_int, ctypes.c_int]
        L.pic_get_timings.restype = st
        L.pic_get_timings.argtypes = [vp, P(pic_timings)]
        L.pic_synchronize.restype = st
        L.pic_synchronize.argtypes = [vp]
        L.pic_batch_create.restype = st
        L.pic_batch_create.argtypes = [ctypes.c_int, P(vp), P(vp)]
        L.pic_get_rho_noalloc.restype = st
        L.pic_get_rho_noalloc.argtypes = [vp, vp, ctypes.c_size_t]
        L.pic_set_stations.restype = st
        L.pic_set_stations.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int]
        L.pic_get_station.restype = st
        L.pic_get_station.argtypes = [vp, ctypes.c_int, P(ctypes.c_int), vp, ctypes.c_size_t, vp, ctypes.c_size_t]
        L.pic_get_fields.restype = st
        L.pic_get_fields.argtypes = [vp, vp, ctypes.c_int, vp, ctypes.c_size_t]
        L.pic_get_gauss_residual.restype = st
        L.pic_get_gauss_residual.argtypes = [vp, P(ctypes.c_double), P(ctypes.c_double)]
        L.pic_set_laser_antenna.restype = st
        L.pic_set_laser_antenna.argtypes = [vp, P(pic_laser_lab), ctypes.c_double]
        L.pic_set_injection.restype = st
        L.pic_set_injection.argtypes = [vp, ctypes.c_int, ctypes.c_double, ctypes.c_int32]
        L.pic_get_planes.restype = st
        L.pic_get_planes.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, ctypes.c_size_t]
        L.pic_put_planes.restype = st
        L.pic_put_planes.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, ctypes.c_size_t, ctypes.c_int]
        L.pic_extract_particles.restype = st
        L.pic_extract_particles.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, vp, ctypes.c_int64,
                                            P(ctypes.c_int64)]
        L.pic_add_particles.restype = st
        L.pic_add_particles.argtypes = [vp, ctypes.c_int64, vp, vp, vp, vp, vp]
        L.pic_batch_autotune.restype = st
        L.pic_batch_autotune.argtypes = [vp, ctypes.c_int, P(ctypes.c_int), P(ctypes.c_double), P(ctypes.c_double)]
        L.pic_batch_set_persistent.restype = st
        L.pic_batch_set_persistent.argtypes = [vp, ctypes.c_int, ctypes.c_int64, ctypes.c_int]
        L.pic_get_planes_n.restype = st
        L.pic_get_planes_n.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, ctypes.c_size_t]
        L.pic_put_planes_n.restype = st
        L.pic_put_planes_n.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, ctypes.c_size_t, ctypes.c_int]
        L.pic_adopt_slab.restype = st
        L.pic_adopt_slab.argtypes = [vp, vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
        L.pic_autotune.restype = st
        L.pic_autotune.argtypes = [P(pic_grid), P(ctypes.c_double), ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                   P(pic_options), P(pic_laser_lab), P(pic_plasma_lab), P(pic_beam_lab), ctypes.c_int,
                                   P(pic_options), P(ctypes.c_double)]
        _lib = L
    return _lib


def _check(status, handle=None):
    if status != PIC_OK:
        msg = lib().pic_last_error(handle)
        raise PicError(status, msg.decode() if msg else "")


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


# ---- thin wrappers with the C names -------------------------------------------------
def pic_default_options():
    o = pic_options()
    lib().pic_default_options(ctypes.byref(o))
    return o


def pic_create(grid, dx, dt, gamma_boost, shape_order, opt=None):
    h = ctypes.c_void_p()
    d = (ctypes.c_double * 3)(*dx)
    _check(lib().pic_create(ctypes.byref(grid), d, dt, gamma_boost, shape_order,
                            ctypes.byref(opt) if opt is not None else None, ctypes.byref(h)))
    return h


def pic_destroy(h):
    lib().pic_destroy(h)


def pic_step(h, n=1):
    _check(lib().pic_step(h, n), h)


def pic_run_phases(h, mask):
    _check(lib().pic_run_phases(h, mask), h)


def pic_synchronize(h):
    _check(lib().pic_synchronize(h), h)


def pic_batch_create(handles):
    arr = (ctypes.c_void_p * len(handles))(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    out = ctypes.c_void_p()
    _check(lib().pic_batch_create(len(handles), arr, ctypes.byref(out)))
    return out


# ---- convenience object ---------------------------------------------------------------
def _lab_structs(laser, plasma, beam):
    """Tuples (as in Simulation.load_lab_frame) -> the pic.h structs (or None)."""
    la = pic_laser_lab(*laser) if laser is not None else None
    if plasma is not None:
        n0, zs, ramp, ppc, uth, seed = plasma
        pl = pic_plasma_lab(n0, zs, ramp, int(ppc), (ctypes.c_double * 3)(*uth), int(seed))
    else:
        pl = None
    if beam is not None:
        nb, gam, spread, sr, sz, z0, tw, seed = beam
        be = pic_beam_lab(int(nb), gam, spread, sr, sz, z0, tw, int(seed))
    else:
        be = None
    return la, pl, be


def autotune(ndim, n, bc, dx, dt, gamma_boost=1.0, order=1, precision=PIC_PREC_FP32, pusher=PIC_PUSHER_VAY,
             filter_passes=0, laser=None, plasma=None, beam=None, steps=5, track_ids=False):
    """pic_autotune: the fastest particle tile for this workload.  Returns (tile, ms per
    step of the winner)."""
    opt = pic_default_options()
    opt.precision = precision
    opt.pusher = pusher
    opt.filter_passes = filter_passes
    opt.track_ids = 1 if track_ids else 0
    n = list(n)
    if ndim == 2:
        n[1] = 1
    grid = pic_grid(ndim, (ctypes.c_int * 3)(*[int(v) for v in n]), (ctypes.c_int * 3)(*bc))
    d = (ctypes.c_double * 3)(*dx)
    la, pl, be = _lab_structs(laser, plasma, beam)
    best = pic_options()
    ms = ctypes.c_double(0.0)
    st = lib().pic_autotune(ctypes.byref(grid), d, dt, gamma_boost, order, ctypes.byref(opt),
                            ctypes.byref(la) if la else None, ctypes.byref(pl) if pl else None,
                            ctypes.byref(be) if be else None, int(steps), ctypes.byref(best), ctypes.byref(ms))
    _check(st)
    return tuple(best.tile), ms.value


class Simulation:
    """One boosted-frame PIC instance (a pic_ctx) with torch-provided device memory.

    Arrays exchanged with the host follow pic.h: fields are returned as (n2, n1, n0)
    numpy arrays (x fastest), particles as dicts of numpy arrays in canonical order.
    """

    def __init__(self, ndim, n, bc, dx, dt, gamma_boost=1.0, order=1, precision=PIC_PREC_FP32,
                 pusher=PIC_PUSHER_VAY, filter_passes=0, tile=(0, 0, 0), absorb_cells=16,
                 absorb_strength=0.1, charge=-1.0, mass=1.0, track_ids=True, stream=None, device=None,
                 use_torch_allocator=True, solver=PIC_SOLVER_YEE, absorb_faces=0x3F):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required: the PIC step runs only in the sm_103a kernels")
        lib()
        self._torch = torch
        n = list(n)
        if ndim == 2:
            n[1] = 1
        self.ndim = ndim
        self.n = tuple(int(v) for v in n)
        self.ncell = self.n[0] * self.n[1] * self.n[2]
        self.precision = int(precision)
        self.device = torch.cuda.current_device() if device is None else int(device)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        opt = pic_default_options()
        opt.precision = precision
        opt.pusher = pusher
        opt.filter_passes = filter_passes
        for a in range(3):
            opt.tile[a] = int(tile[a])
        opt.absorb_cells = absorb_cells
        opt.absorb_strength = absorb_strength
        opt.charge = charge
        opt.mass = mass
        opt.track_ids = 1 if track_ids else 0
        opt.solver = solver
        opt.absorb_faces = int(absorb_faces)
        opt.stream = self.stream.cuda_stream
        opt.device = self.device
        self._live = {}
        if use_torch_allocator:
            dev, strm = self.device, self.stream

            def _alloc(nbytes, user):
                try:
                    return torch.cuda.caching_allocator_alloc(nbytes, device=dev, stream=strm)
                except Exception:  # reported to the library as NULL -> PIC_ERR_OOM
                    return None

            def _free(ptr, user):
                torch.cuda.caching_allocator_delete(ptr)

            self._alloc_cb = ALLOC_FN(_alloc)
            self._free_cb = FREE_FN(_free)
            opt.alloc = self._alloc_cb
            opt.free = self._free_cb
        grid = pic_grid(ndim, (ctypes.c_int * 3)(*self.n), (ctypes.c_int * 3)(*bc))
        self.h = pic_create(grid, dx, dt, gamma_boost, order, opt)

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib().pic_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- loading
    @property
    def stored_dtype(self):
        """numpy type of the particle values as the device stores them."""
        return np.float32 if self.precision == PIC_PREC_FP32 else np.float64

    def load_particles(self, cell, off, u, w, ids=None):
        """Replaces the particles.  float32 off, u and w on an FP32 context go in as they
        are (pic_load_particles_stored: no FP64 copy, half the bytes); anything else is
        taken as FP64 (pic_load_particles)."""
        cell = np.ascontiguousarray(cell, dtype=np.int32)
        npart = cell.size
        ids = None if ids is None else np.ascontiguousarray(ids, dtype=np.int32)
        arrs = [np.asarray(a) for a in (off, u, w)]
        if self.precision == PIC_PREC_FP32 and all(a.dtype == np.float32 for a in arrs):
            off, u, w = (np.ascontiguousarray(a) for a in arrs)
            if off.size != 3 * npart or u.size != 3 * npart or w.size != npart:
                raise ValueError("off and u need 3 values per particle, w one")
            _check(lib().pic_load_particles_stored(self.h, npart, _ptr(cell), _ptr(off), _ptr(u), _ptr(w), _ptr(ids)),
                   self.h)
            return
        off = np.ascontiguousarray(np.asarray(off, np.float64).reshape(npart, 3))
        u = np.ascontiguousarray(np.asarray(u, np.float64).reshape(npart, 3))
        w = np.ascontiguousarray(w, dtype=np.float64)
        _check(lib().pic_load_particles(self.h, npart, _ptr(cell), _ptr(off), _ptr(u), _ptr(w), _ptr(ids)), self.h)

    def load_lab_frame(self, laser=None, plasma=None, beam=None):
        la, pl, be = _lab_structs(laser, plasma, beam)
        _check(lib().pic_load_lab_frame(self.h, ctypes.byref(la) if la else None, ctypes.byref(pl) if pl else None,
                                        ctypes.byref(be) if be else None), self.h)

    def set_stations(self, z_lab, max_records):
        """pic_set_stations: lab-frame stations at the planes z_lab."""
        z = np.ascontiguousarray(z_lab, dtype=np.float64)
        self._stations = z.size
        _check(lib().pic_set_stations(self.h, z.size, _ptr(z), int(max_records)), self.h)

    def get_fields(self, comps):
        """pic_get_fields: several components as one (ncomp, n2, n1, n0) array."""
        c = np.ascontiguousarray(comps, dtype=np.int32)
        out = np.empty((c.size, self.n[2], self.n[1], self.n[0]))
        _check(lib().pic_get_fields(self.h, _ptr(c), c.size, _ptr(out), out.size), self.h)
        return out

    def gauss_residual(self):
        """pic_get_gauss_residual: (max |div E - rho|, rms)."""
        m, r = ctypes.c_double(), ctypes.c_double()
        _check(lib().pic_get_gauss_residual(self.h, ctypes.byref(m), ctypes.byref(r)), self.h)
        return m.value, r.value

    def set_antenna(self, laser, z_lab=0.0):
        """pic_set_laser_antenna: the lab pulse laser = (a0, lambda0, waist, duration,
        z_center) emitted forward through the lab plane z_lab (None: remove it)."""
        la = _lab_structs(laser, None, None)[0] if laser is not None else None
        _check(lib().pic_set_laser_antenna(self.h, ctypes.byref(la) if la else None, float(z_lab)), self.h)

    def set_injection(self, z_lab, first_id=-1, enable=True):
        """pic_set_injection: beam particles (id >= first_id; -1: the last lab-frame load's
        beam) upstream of the lab plane z_lab are frozen."""
        _check(lib().pic_set_injection(self.h, int(bool(enable)), float(z_lab), int(first_id)), self.h)

    def station(self, i):
        """History of station i: (t_lab (n,), fields (n, 6, n1, n0)) in the lab frame."""
        n = ctypes.c_int(0)
        _check(lib().pic_get_station(self.h, i, ctypes.byref(n), None, 0, None, 0), self.h)
        t = np.zeros(n.value)
        f = np.zeros((n.value, 6, self.n[1], self.n[0]))
        _check(lib().pic_get_station(self.h, i, ctypes.byref(n), _ptr(t), t.size, _ptr(f), f.size), self.h)
        return t, f

    def set_field(self, comp, arr):
        a = np.ascontiguousarray(np.asarray(arr, dtype=np.float64).reshape(-1))
        _check(lib().pic_set_field(self.h, comp, _ptr(a), a.size), self.h)

    # -- stepping
    def step(self, n=1):
        _check(lib().pic_step(self.h, n), self.h)

    def run_phases(self, mask):
        _check(lib().pic_run_phases(self.h, mask), self.h)

    def synchronize(self):
        _check(lib().pic_synchronize(self.h), self.h)

    # -- getters
    def get_field(self, comp):
        out = np.empty(self.ncell)
        _check(lib().pic_get_field(self.h, comp, _ptr(out), out.size), self.h)
        return out.reshape(self.n[2], self.n[1], self.n[0])

    def num_particles(self):
        v = ctypes.c_int64()
        _check(lib().pic_num_particles(self.h, ctypes.byref(v)), self.h)
        return int(v.value)

    def get_particles(self, stored=False, out=None):
        """The live particles in canonical order: dict of cell (n,), off (n, 3), u (n, 3), w
        (n,), id (n,).  stored: values in the storage precision (float32 for an FP32
        context; pic_get_particles_stored), else FP64.  out: a dict of such arrays with room
        for at least n particles (any of the five keys; e.g. page-locked buffers reused
        across calls), filled in place and returned cut to n."""
        n = self.num_particles()
        vt = self.stored_dtype if stored else np.float64
        shapes = dict(cell=((n,), np.int32), off=((n, 3), vt), u=((n, 3), vt), w=((n,), vt), id=((n,), np.int32))
        arrs = {}
        for k, (shape, dt) in shapes.items():
            if out is None or k not in out:
                arrs[k] = np.empty(shape, dt)
                continue
            a = out[k]
            per = int(np.prod(shape[1:])) if len(shape) > 1 else 1
            if a.dtype != dt or not a.flags.c_contiguous or a.size < n * per:
                raise ValueError(f"out[{k!r}] must be a C-contiguous {np.dtype(dt).name} array of >= {n * per} values")
            arrs[k] = a.reshape(-1)[:n * per].reshape(shape)
        got = ctypes.c_int64()
        fn = lib().pic_get_particles_stored if stored else lib().pic_get_particles
        _check(fn(self.h, *(_ptr(arrs[k]) for k in ("cell", "off", "u", "w", "id")), n, ctypes.byref(got)), self.h)
        return arrs

    # -- z-slab exchange
    def get_planes(self, comp, k0, nk):
        out = np.empty((nk, self.n[1], self.n[0]))
        _check(lib().pic_get_planes(self.h, comp, int(k0), int(nk), _ptr(out), out.size), self.h)
        return out

    def put_planes(self, comp, k0, values, add=False):
        v = np.ascontiguousarray(np.asarray(values, np.float64).reshape(-1, self.n[1], self.n[0]))
        _check(lib().pic_put_planes(self.h, comp, int(k0), v.shape[0], _ptr(v), v.size, 1 if add else 0), self.h)

    def get_planes_n(self, comps, k0, nk):
        """Planes k0 .. k0 + nk - 1 of several components, (len(comps), nk, n1, n0)."""
        cs = np.ascontiguousarray(comps, dtype=np.int32)
        out = np.empty((cs.size, nk, self.n[1], self.n[0]))
        _check(lib().pic_get_planes_n(self.h, _ptr(cs), cs.size, int(k0), int(nk), _ptr(out), out.size), self.h)
        return out

    def put_planes_n(self, comps, k0, values, add=False):
        cs = np.ascontiguousarray(comps, dtype=np.int32)
        v = np.ascontiguousarray(np.asarray(values, np.float64).reshape(cs.size, -1, self.n[1], self.n[0]))
        _check(lib().pic_put_planes_n(self.h, _ptr(cs), cs.size, int(k0), v.shape[1], _ptr(v), v.size, 1 if add else 0),
               self.h)

    def extract_particles(self, k_lo, k_hi):
        """Removes and returns the particles whose z cell index is outside [k_lo, k_hi)."""
        cap = self.num_particles()
        cell = np.empty(cap, np.int32)
        off = np.empty((cap, 3))
        u = np.empty((cap, 3))
        w = np.empty(cap)
        ids = np.empty(cap, np.int32)
        got = ctypes.c_int64()
        _check(lib().pic_extract_particles(self.h, int(k_lo), int(k_hi), _ptr(cell), _ptr(off), _ptr(u), _ptr(w),
                                           _ptr(ids), cap, ctypes.byref(got)), self.h)
        m = int(got.value)
        return dict(cell=cell[:m], off=off[:m], u=u[:m], w=w[:m], id=ids[:m])

    def add_particles(self, cell, off, u, w, ids=None):
        cell = np.ascontiguousarray(cell, dtype=np.int32)
        npart = cell.size
        off = np.ascontiguousarray(np.asarray(off, np.float64).reshape(npart, 3))
        u = np.ascontiguousarray(np.asarray(u, np.float64).reshape(npart, 3))
        w = np.ascontiguousarray(w, dtype=np.float64)
        idp = None if ids is None else np.ascontiguousarray(ids, dtype=np.int32)
        _check(lib().pic_add_particles(self.h, npart, _ptr(cell), _ptr(off), _ptr(u), _ptr(w),
                                       None if idp is None else _ptr(idp)), self.h)

    def adopt_slab(self, whole, k_origin, k_lo, k_hi):
        """Continue the run of `whole` as its z slab starting at plane k_origin and owning
        local planes k_lo .. k_hi - 1."""
        _check(lib().pic_adopt_slab(self.h, whole.h, int(k_origin), int(k_lo), int(k_hi)), self.h)

    def diagnostics(self):
        d = pic_diag()
        _check(lib().pic_get_diagnostics(self.h, ctypes.byref(d)), self.h)
        return {k: getattr(d, k) for k, _ in pic_diag._fields_}

    def set_profiling(self, on, reset=False):
        _check(lib().pic_set_profiling(self.h, 1 if on else 0, 1 if reset else 0), self.h)

    def timings(self):
        t = pic_timings()
        _check(lib().pic_get_timings(self.h, ctypes.byref(t)), self.h)
        return {k: getattr(t, k) for k, _ in pic_timings._fields_}


class Batch:
    """Several Simulations advanced together, one launch per phase (pic_batch_create)."""

    def __init__(self, sims):
        self.sims = list(sims)
        self.h = pic_batch_create([s.h for s in self.sims])

    def step(self, n=1):
        _check(lib().pic_step(self.h, n), self.h)

    def autotune(self, steps=3):
        """pic_batch_autotune: times both launch forms on real steps and keeps the faster.
        Returns (persistent chosen, ms per step graph, ms per step persistent)."""
        pers, mg, mp = ctypes.c_int(), ctypes.c_double(), ctypes.c_double()
        _check(lib().pic_batch_autotune(self.h, int(steps), ctypes.byref(pers), ctypes.byref(mg), ctypes.byref(mp)),
               self.h)
        return bool(pers.value), mg.value, mp.value

    def set_persistent(self, on=True, spin_limit=0, test_stall=-1):
        """pic_batch_set_persistent: each step() call as one persistent launch."""
        _check(lib().pic_batch_set_persistent(self.h, 1 if on else 0, int(spin_limit), int(test_stall)), self.h)

    def synchronize(self):
        _check(lib().pic_synchronize(self.h), self.h)

    def set_profiling(self, on, reset=False):
        _check(lib().pic_set_profiling(self.h, 1 if on else 0, 1 if reset else 0), self.h)

    def timings(self):
        t = pic_timings()
        _check(lib().pic_get_timings(self.h, ctypes.byref(t)), self.h)
        return {k: getattr(t, k) for k, _ in pic_timings._fields_}

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib().pic_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
