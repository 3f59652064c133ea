"""Thin ctypes binding of the gbfdtd C ABI (include/fdtd.h).

Every `fdtd_*` function here has the C function's name and arguments; it only marshals
arguments and turns a non-OK status into `FdtdError`.  All arithmetic runs in the CUDA
kernels of libgbfdtd.so: there is no CPU fallback, and a missing library is an error.

`Context` is argument marshalling for the common case: it turns a workload `Scene` plus
torch device tensors into the C descriptors, and keeps those tensors alive (the library
borrows them).
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Optional, Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libgbfdtd.so")

FDTD_OK, FDTD_EINVAL, FDTD_ECFL, FDTD_ETENSOR, FDTD_ENOMEM, FDTD_ECUDA, FDTD_ESTATE, FDTD_ENONFINITE, \
    FDTD_ETIMEOUT = range(9)
STATUS_NAMES = ["FDTD_OK", "FDTD_EINVAL", "FDTD_ECFL", "FDTD_ETENSOR", "FDTD_ENOMEM", "FDTD_ECUDA",
                "FDTD_ESTATE", "FDTD_ENONFINITE", "FDTD_ETIMEOUT"]
FDTD_F32, FDTD_F64 = 0, 1
FDTD_LORENTZ, FDTD_DRUDE = 0, 1
FDTD_CODEC_NATIVE, FDTD_CODEC_BF16 = 0, 1
LAUNCH_MODES = 5   # FDTD_LAUNCH_MODES: entries of the autotuner's array, indexed by mode
MODES = (0, 4)     # the launch modes: per-half-step tile launches over all domains, per-cell launches
KERNEL_CLASSES = ["e_update", "h_update", "source", "dft", "step", "adj_e", "adj_h", "unused"]


class fdtd_grid(C.Structure):
    _fields_ = [("nx", C.c_int32), ("ny", C.c_int32), ("nz", C.c_int32), ("dx", C.c_double),
                ("courant", C.c_double), ("dt", C.c_double), ("dtype", C.c_int32)]


class fdtd_cpml(C.Structure):
    _fields_ = [("cells", C.c_int32 * 6), ("m", C.c_double), ("kappa_max", C.c_double),
                ("alpha_max", C.c_double), ("sigma_max", C.c_double)]


class fdtd_pole(C.Structure):
    _fields_ = [("kind", C.c_int32), ("delta_eps", C.c_double), ("omega_dt", C.c_double),
                ("gamma_dt", C.c_double)]


class fdtd_material(C.Structure):
    _fields_ = [("inv_eps", C.c_void_p * 3), ("n_poles", C.c_int32), ("poles", C.POINTER(fdtd_pole)),
                ("pole_mask", C.c_void_p)]


class FdtdError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{where}: {name}: {msg}")


_lib = None
_lock = threading.Lock()
_i32p = C.POINTER(C.c_int32)
_i64p = C.POINTER(C.c_int64)
_vp = C.c_void_p
_ctx = C.c_void_p

# name -> argtypes (all return fdtd_status unless listed in _RESTYPE)
_SIGS = {
    "fdtd_create": [C.c_int32, C.POINTER(fdtd_grid), C.POINTER(fdtd_cpml), C.POINTER(fdtd_material), _vp,
                    C.POINTER(_ctx)],
    "fdtd_create_streamed": [C.POINTER(fdtd_grid), C.POINTER(fdtd_cpml), C.POINTER(fdtd_material), C.c_int32,
                             C.c_int32, _vp, C.POINTER(_ctx)],
    "fdtd_destroy": [_ctx],
    "fdtd_run_schedule": [_ctx, C.POINTER(C.c_int32), C.c_int32, C.c_int32, C.POINTER(C.c_int32)],
    "fdtd_set_pole_grad": [_ctx, C.c_int32, C.c_int32],
    "fdtd_pole_grad": [_ctx, C.c_int32, C.POINTER(C.c_double)],
    "fdtd_last_error": [_ctx],
    "fdtd_version": [],
    "fdtd_set_material": [_ctx, C.c_int32, C.POINTER(fdtd_material)],
    "fdtd_set_periodic": [_ctx, C.c_int32, _i32p],
    "fdtd_set_bloch": [_ctx, C.c_int32, C.POINTER(C.c_double)],
    "fdtd_set_tensor": [_ctx, C.c_int32, C.POINTER(C.c_void_p)],
    "fdtd_dft_flux": [_ctx, C.c_int32, C.POINTER(C.c_double), C.c_int32],
    "fdtd_step_backward": [_ctx, C.c_int32],
    "fdtd_record_interface": [_ctx, C.c_int32],
    "fdtd_stream_checkpoints": [_ctx, C.c_int32],
    "fdtd_add_source": [_ctx, C.c_int32, C.c_int32, _i32p, _i32p, C.POINTER(C.c_double), C.c_int32, _i32p],
    "fdtd_add_dft_monitor": [_ctx, C.c_int32, _i32p, _i32p, C.c_uint32, C.c_int32, C.POINTER(C.c_double),
                             _i32p],
    "fdtd_dft_size": [_ctx, C.c_int32, _i64p],
    "fdtd_dft_read": [_ctx, C.c_int32, _vp, C.c_size_t, C.c_int32],
    "fdtd_dft_reset": [_ctx],
    "fdtd_dft_enable": [_ctx, C.c_int32],
    "fdtd_enable_energy": [_ctx, C.c_int32],
    "fdtd_energy_read": [_ctx, C.c_int32, C.POINTER(C.c_double), C.c_int32],
    "fdtd_step_forward": [_ctx, C.c_int32],
    "fdtd_step_count": [_ctx, _i64p],
    "fdtd_set_launch_mode": [_ctx, C.c_int32],
    "fdtd_get_launch_mode": [_ctx, _i32p],
    "fdtd_autotune": [_ctx, C.c_int32, C.POINTER(C.c_double)],
    "fdtd_reset": [_ctx],
    "fdtd_part_count": [_ctx, C.c_int32, _i32p],
    "fdtd_part_size": [_ctx, C.c_int32, C.c_int32, _i64p],
    "fdtd_get_part": [_ctx, C.c_int32, C.c_int32, C.c_int32, _vp],
    "fdtd_set_part": [_ctx, C.c_int32, C.c_int32, C.c_int32, _vp],
    "fdtd_ade_box": [_ctx, C.c_int32, _i32p, _i32p],
    "fdtd_set_step_count": [_ctx, C.c_int64],
    "fdtd_state_save": [_ctx, C.c_int32, C.c_int32],
    "fdtd_state_restore": [_ctx, C.c_int32],
    "fdtd_snapshot_bytes": [_ctx, C.c_int32, _i64p],
    "fdtd_snapshots_free": [_ctx],
    "fdtd_set_design": [_ctx, C.c_int32, _i32p, _i32p, _vp],
    "fdtd_set_adjoint_source": [_ctx, C.c_int32, _vp],
    "fdtd_adjoint_begin": [_ctx],
    "fdtd_step_adjoint": [_ctx, C.c_int32],
    "fdtd_adjoint_step_count": [_ctx, _i64p],
    "fdtd_set_adjoint_step_count": [_ctx, C.c_int64],
    "fdtd_check_finite": [_ctx],
    "fdtd_synchronize": [_ctx, C.c_int32],
    "fdtd_time_half_steps": [_ctx, C.c_int32, C.c_int32, C.POINTER(C.c_double)],
    "fdtd_measure_fp64_rate": [_vp, C.POINTER(C.c_double), C.POINTER(C.c_double)],
    "fdtd_launch_count": [_ctx, _i64p],
    "fdtd_count_nonfinite_noalloc": [_vp, C.c_int64, C.c_int32, _vp, _i64p],
    "fdtd_profile_begin": [_ctx, C.c_int32],
    "fdtd_profile_end": [_ctx, C.POINTER(C.c_double), _i64p],
}
_RESTYPE = {"fdtd_last_error": C.c_char_p, "fdtd_version": C.c_char_p}


def declared_functions():
    return sorted(_SIGS)


def load(path: Optional[str] = None):
    """Loads libgbfdtd.so (built by __graft_entry__.build() / paper_2609_30039_gb300.build)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"libgbfdtd.so not found at {p}: build it first (python -c "
                               "'import __graft_entry__ as g; g.build()'); there is no CPU fallback")
        lib = C.CDLL(p)
        for name, args in _SIGS.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = _RESTYPE.get(name, C.c_int)
        _lib = lib
        return lib


def _check(st, name, ctx=None):
    if st != FDTD_OK:
        msg = _lib.fdtd_last_error(ctx).decode() if _lib is not None else ""
        raise FdtdError(int(st), name, msg)


def _i3(v):
    return (C.c_int32 * 3)(*[int(x) for x in v])


# ------------------------------------------------------------------ C functions, same names
def fdtd_version() -> str:
    return load().fdtd_version().decode()


def fdtd_last_error(ctx) -> str:
    return load().fdtd_last_error(ctx).decode()


def fdtd_create(grids, cpmls, materials, stream=0):
    lib = load()
    n = len(grids)
    ga = (fdtd_grid * n)(*grids)
    ca = (fdtd_cpml * n)(*cpmls)
    ma = (fdtd_material * n)(*materials)
    out = _ctx()
    st = lib.fdtd_create(n, ga, ca, ma, _vp(stream), C.byref(out))
    _check(st, "fdtd_create", None)
    return out


def fdtd_create_streamed(grid, cpml, material, slab, halo, stream=0):
    """Host-streamed context of one domain (Sec. 4.2): state in pinned host memory, stepped in
    z-slabs of `slab` planes with `halo` halo planes (batches of at most `halo` steps)."""
    out = _ctx()
    st = load().fdtd_create_streamed(C.byref(grid), C.byref(cpml), C.byref(material), int(slab), int(halo),
                                     _vp(stream), C.byref(out))
    _check(st, "fdtd_create_streamed", None)
    return out


def fdtd_set_pole_grad(ctx, domain, enabled):
    _check(load().fdtd_set_pole_grad(ctx, int(domain), int(bool(enabled))), "fdtd_set_pole_grad", ctx)


MAX_POLES = 16


def fdtd_pole_grad(ctx, domain, n_poles):
    """d J / d(delta_eps, omega_dt, gamma_dt) of each pole of a domain, shape (n_poles, 3).  The
    library writes 3 values per pole of the domain, so the buffer holds the largest pole count."""
    if not 0 <= int(n_poles) <= MAX_POLES:
        raise ValueError("n_poles must be in [0, 16]")
    out = np.zeros(3 * MAX_POLES)
    _check(load().fdtd_pole_grad(ctx, int(domain), out.ctypes.data_as(C.POINTER(C.c_double))), "fdtd_pole_grad", ctx)
    return out[: 3 * int(n_poles)].reshape(int(n_poles), 3)


FDTD_ACT_SAVE, FDTD_ACT_RESTORE, FDTD_ACT_ADVANCE, FDTD_ACT_ADJOINT, FDTD_ACT_STOP = 0, 1, 2, 3, 4


def fdtd_run_schedule(ctx, actions, start, codec):
    """Runs the (kind, arg) int32 rows actions[start:] natively until a STOP or the end; returns
    the index of the next action to run."""
    a = np.ascontiguousarray(actions, dtype=np.int32).reshape(-1, 2)
    n = a.shape[0] - int(start)
    if n <= 0:
        return int(start)
    done = C.c_int32(0)
    ptr = a[int(start):].ctypes.data_as(C.POINTER(C.c_int32))
    st = load().fdtd_run_schedule(ctx, ptr, n, int(codec), C.byref(done))
    _check(st, "fdtd_run_schedule", ctx)
    return int(start) + done.value


def fdtd_destroy(ctx):
    _check(load().fdtd_destroy(ctx), "fdtd_destroy", ctx)


def _wrap_simple(name):
    def f(ctx, *args):
        st = getattr(load(), name)(ctx, *args)
        _check(st, name, ctx)
    f.__name__ = name
    return f


fdtd_dft_reset = _wrap_simple("fdtd_dft_reset")
fdtd_dft_enable = _wrap_simple("fdtd_dft_enable")
fdtd_enable_energy = _wrap_simple("fdtd_enable_energy")
fdtd_step_forward = _wrap_simple("fdtd_step_forward")
fdtd_set_launch_mode = _wrap_simple("fdtd_set_launch_mode")


def fdtd_get_launch_mode(ctx):
    v = C.c_int32()
    _check(load().fdtd_get_launch_mode(ctx, C.byref(v)), "fdtd_get_launch_mode", ctx)
    return int(v.value)


def fdtd_autotune(ctx, n_steps):
    """Times launch modes 0 and 4 on the live state, keeps the faster; returns ms per mode index
    (-1 for the mode numbers that are not available)."""
    ms = (C.c_double * LAUNCH_MODES)()
    _check(load().fdtd_autotune(ctx, int(n_steps), ms), "fdtd_autotune", ctx)
    return [float(v) for v in ms]
fdtd_reset = _wrap_simple("fdtd_reset")
fdtd_set_step_count = _wrap_simple("fdtd_set_step_count")
fdtd_state_save = _wrap_simple("fdtd_state_save")
fdtd_state_restore = _wrap_simple("fdtd_state_restore")
fdtd_snapshots_free = _wrap_simple("fdtd_snapshots_free")
fdtd_adjoint_begin = _wrap_simple("fdtd_adjoint_begin")
fdtd_step_adjoint = _wrap_simple("fdtd_step_adjoint")
fdtd_set_adjoint_step_count = _wrap_simple("fdtd_set_adjoint_step_count")
fdtd_check_finite = _wrap_simple("fdtd_check_finite")
fdtd_synchronize = _wrap_simple("fdtd_synchronize")


def fdtd_measure_fp64_rate(stream=0):
    """(FP64 FMA instructions per second, best run in ms) measured on the current device."""
    r, ms = C.c_double(), C.c_double()
    _check(load().fdtd_measure_fp64_rate(stream, C.byref(r), C.byref(ms)), "fdtd_measure_fp64_rate")
    return r.value, ms.value


def fdtd_time_half_steps(ctx, which, n_launches=32):
    """Milliseconds per launch of the E (0), H (1), DFT-of-E (2), transposed E (3) or transposed H (4)
    kernels, back to back in a graph."""
    ms = C.c_double()
    _check(load().fdtd_time_half_steps(ctx, int(which), int(n_launches), C.byref(ms)), "fdtd_time_half_steps", ctx)
    return ms.value


def _get_i64(name, ctx, *args):
    v = C.c_int64()
    st = getattr(load(), name)(ctx, *args, C.byref(v))
    _check(st, name, ctx)
    return int(v.value)


fdtd_profile_begin = _wrap_simple("fdtd_profile_begin")


def fdtd_count_nonfinite_noalloc(data_ptr, n, dtype, stream=0):
    """NaN/Inf count of n values at a device pointer; allocates no device memory (see fdtd.h)."""
    cnt = C.c_int64()
    st = load().fdtd_count_nonfinite_noalloc(_vp(data_ptr), int(n), int(dtype), _vp(stream), C.byref(cnt))
    _check(st, "fdtd_count_nonfinite_noalloc", None)
    return int(cnt.value)


def fdtd_profile_end(ctx):
    """Returns {kernel class: (summed device ms, timed launches)}."""
    n = len(KERNEL_CLASSES)
    ms = (C.c_double * n)()
    cnt = (C.c_int64 * n)()
    _check(load().fdtd_profile_end(ctx, ms, cnt), "fdtd_profile_end", ctx)
    return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(KERNEL_CLASSES)}


def fdtd_step_count(ctx):
    return _get_i64("fdtd_step_count", ctx)


def fdtd_adjoint_step_count(ctx):
    return _get_i64("fdtd_adjoint_step_count", ctx)


def fdtd_launch_count(ctx):
    return _get_i64("fdtd_launch_count", ctx)


def fdtd_dft_size(ctx, monitor_id):
    return _get_i64("fdtd_dft_size", ctx, int(monitor_id))


def fdtd_part_size(ctx, domain, part):
    return _get_i64("fdtd_part_size", ctx, int(domain), int(part))


def fdtd_snapshot_bytes(ctx, codec):
    return _get_i64("fdtd_snapshot_bytes", ctx, int(codec))


def fdtd_part_count(ctx, domain):
    v = C.c_int32()
    _check(load().fdtd_part_count(ctx, int(domain), C.byref(v)), "fdtd_part_count", ctx)
    return int(v.value)


def fdtd_dft_flux(ctx, monitor, n_freq):
    """Net +z Poynting flux per frequency through a two-plane monitor (numpy array)."""
    out = np.zeros(max(int(n_freq), 1), dtype=np.float64)
    _check(load().fdtd_dft_flux(ctx, int(monitor), out.ctypes.data_as(C.POINTER(C.c_double)), int(n_freq)),
           "fdtd_dft_flux", ctx)
    return out[: int(n_freq)]


fdtd_step_backward = _wrap_simple("fdtd_step_backward")
fdtd_record_interface = _wrap_simple("fdtd_record_interface")
fdtd_stream_checkpoints = _wrap_simple("fdtd_stream_checkpoints")


def fdtd_set_periodic(ctx, domain, periodic):
    arr = (C.c_int32 * 3)(*[int(v) for v in periodic])
    _check(load().fdtd_set_periodic(ctx, int(domain), arr), "fdtd_set_periodic", ctx)


def fdtd_set_bloch(ctx, domain, phase):
    ph = (C.c_double * 2)(float(phase[0]), float(phase[1]))
    _check(load().fdtd_set_bloch(ctx, int(domain), ph), "fdtd_set_bloch", ctx)


def fdtd_set_tensor(ctx, domain, components):
    """components: six arrays (device tensors or host arrays of the context's dtype, contiguous) of
    eps^-1 xx, yy, zz, xy, xz, yz at the nodes, or None to return to the diagonal eps^-1."""
    if components is None:
        _check(load().fdtd_set_tensor(ctx, int(domain), None), "fdtd_set_tensor", ctx)
        return
    ptrs = (C.c_void_p * 6)(*[int(t.data_ptr()) if hasattr(t, "data_ptr") else int(t.ctypes.data) for t in components])
    _check(load().fdtd_set_tensor(ctx, int(domain), ptrs), "fdtd_set_tensor", ctx)


def fdtd_set_material(ctx, domain, material):
    _check(load().fdtd_set_material(ctx, int(domain), C.byref(material)), "fdtd_set_material", ctx)


def fdtd_add_source(ctx, domain, component, lo, hi, waveform):
    w = np.ascontiguousarray(waveform, dtype=np.float64)
    sid = C.c_int32()
    st = load().fdtd_add_source(ctx, int(domain), int(component), _i3(lo), _i3(hi),
                                w.ctypes.data_as(C.POINTER(C.c_double)), int(w.size), C.byref(sid))
    _check(st, "fdtd_add_source", ctx)
    return int(sid.value)


def fdtd_add_dft_monitor(ctx, domain, lo, hi, component_mask, omega_dt):
    om = np.ascontiguousarray(omega_dt, dtype=np.float64)
    mid = C.c_int32()
    st = load().fdtd_add_dft_monitor(ctx, int(domain), _i3(lo), _i3(hi), int(component_mask), int(om.size),
                                     om.ctypes.data_as(C.POINTER(C.c_double)), C.byref(mid))
    _check(st, "fdtd_add_dft_monitor", ctx)
    return int(mid.value)


def fdtd_dft_read(ctx, monitor_id, dst_ptr, nbytes, dst_on_device):
    _check(load().fdtd_dft_read(ctx, int(monitor_id), _vp(dst_ptr), C.c_size_t(nbytes), int(dst_on_device)),
           "fdtd_dft_read", ctx)


def fdtd_energy_read(ctx, domain, n):
    out = np.zeros(int(n), dtype=np.float64)
    _check(load().fdtd_energy_read(ctx, int(domain), out.ctypes.data_as(C.POINTER(C.c_double)), int(n)),
           "fdtd_energy_read", ctx)
    return out


def fdtd_get_part(ctx, domain, which, part, dst_ptr):
    _check(load().fdtd_get_part(ctx, int(domain), int(which), int(part), _vp(dst_ptr)), "fdtd_get_part", ctx)


def fdtd_set_part(ctx, domain, which, part, src_ptr):
    _check(load().fdtd_set_part(ctx, int(domain), int(which), int(part), _vp(src_ptr)), "fdtd_set_part", ctx)


def fdtd_ade_box(ctx, domain):
    lo, hi = (C.c_int32 * 3)(), (C.c_int32 * 3)()
    _check(load().fdtd_ade_box(ctx, int(domain), lo, hi), "fdtd_ade_box", ctx)
    return tuple(lo), tuple(hi)


def fdtd_set_design(ctx, domain, lo, hi, grad_ptr):
    _check(load().fdtd_set_design(ctx, int(domain), _i3(lo) if lo is not None else None,
                                  _i3(hi) if hi is not None else None, _vp(grad_ptr) if grad_ptr else None),
           "fdtd_set_design", ctx)


def fdtd_set_adjoint_source(ctx, monitor_id, cot_ptr):
    _check(load().fdtd_set_adjoint_source(ctx, int(monitor_id), _vp(cot_ptr) if cot_ptr else None),
           "fdtd_set_adjoint_source", ctx)


# ------------------------------------------------------------------ marshalling helper
class Context:
    """Owns one fdtd_ctx built from workload Scenes (one per domain) and the torch tensors the
    library borrows (inv_eps, pole masks, gradient buffers, adjoint sources)."""

    def __init__(self, scenes, dtype: str = "f32", device: str = "cuda:0", stream=None, streamed=None):
        """streamed: None (state in device memory) or (slab, halo) for a host-streamed context of
        one domain (Sec. 4.2), whose materials are then kept in pinned host memory."""
        import torch
        self.torch = torch
        if not isinstance(scenes, (list, tuple)):
            scenes = [scenes]
        self.scenes = list(scenes)
        self.streamed = tuple(int(v) for v in streamed) if streamed is not None else None
        if self.streamed is not None and len(self.scenes) != 1:
            raise ValueError("a host-streamed context holds one domain")
        self.tdtype = torch.float32 if dtype == "f32" else torch.float64
        self.npdtype = np.float32 if dtype == "f32" else np.float64
        self.code = FDTD_F32 if dtype == "f32" else FDTD_F64
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._keep = []
        grids, cpmls, mats = [], [], []
        self.inv_eps = []
        self.masks = []
        for sc in self.scenes:
            nx, ny, nz = sc.shape
            grids.append(fdtd_grid(nx, ny, nz, 1.0, sc.courant, 0.0, self.code))
            cp = fdtd_cpml()
            for f in range(6):
                cp.cells[f] = int(sc.cpml[f])
            cp.m, cp.kappa_max, cp.alpha_max, cp.sigma_max = sc.cpml_m, sc.kappa_max, sc.alpha_max, sc.sigma_max
            cpmls.append(cp)
            ie = self._material_tensors(sc)
            self.inv_eps.append(ie)
            mats.append(self._material_struct(sc, ie))
        if self.streamed is not None:
            self.ctx = fdtd_create_streamed(grids[0], cpmls[0], mats[0], self.streamed[0], self.streamed[1],
                                            stream=self.stream.cuda_stream)
        else:
            self.ctx = fdtd_create(grids, cpmls, mats, stream=self.stream.cuda_stream)
        self.monitors = []
        self.sources = []
        for d, sc in enumerate(self.scenes):
            if any(sc.periodic):
                fdtd_set_periodic(self.ctx, d, sc.periodic)
            if getattr(sc, "tensor", None) is not None:
                t = torch.from_numpy(np.ascontiguousarray(sc.tensor, dtype=self.npdtype)).to(self.device)
                fdtd_set_tensor(self.ctx, d, [t[q] for q in range(6)])
            for s in sc.sources:
                self.sources.append(fdtd_add_source(self.ctx, d, s.comp, s.lo, s.hi, s.wave))
            for m in sc.monitors:
                mask = 0
                for c in m.comps:
                    mask |= 1 << int(c)
                mid = fdtd_add_dft_monitor(self.ctx, d, m.lo, m.hi, mask, m.omegas)
                ext = tuple(int(h) - int(lo) for lo, h in zip(m.lo, m.hi))
                self.monitors.append((mid, (len(m.comps), len(m.omegas), ext[2], ext[1], ext[0]), d))
            if sc.energy:
                fdtd_enable_energy(self.ctx, sc.n_steps + 8)

    def _place(self, t):
        """Material arrays live on the device, or in pinned host memory for a streamed context."""
        return t.pin_memory() if self.streamed is not None else t.to(self.device)

    def _material_tensors(self, sc):
        torch = self.torch
        arrs = sc.inv_eps3()
        if arrs[0] is arrs[1] and arrs[1] is arrs[2]:
            t = self._place(torch.from_numpy(np.ascontiguousarray(arrs[0], dtype=self.npdtype)))
            return [t, t, t]
        return [self._place(torch.from_numpy(np.ascontiguousarray(a, dtype=self.npdtype))) for a in arrs]

    def _material_struct(self, sc, ie, mask_tensor=None):
        torch = self.torch
        m = fdtd_material()
        for a in range(3):
            m.inv_eps[a] = ie[a].data_ptr()
        npole = len(sc.poles) if sc.pole_mask is not None else 0
        m.n_poles = npole
        if npole:
            arr = (fdtd_pole * npole)(*[fdtd_pole(int(k), float(de), float(w), float(g)) for k, de, w, g in sc.poles])
            self._keep.append(arr)
            m.poles = C.cast(arr, C.POINTER(fdtd_pole))
            mk = mask_tensor if mask_tensor is not None else self._place(torch.from_numpy(
                np.ascontiguousarray(sc.pole_mask, dtype=np.uint8)))
            self.masks.append(mk)
            m.pole_mask = mk.data_ptr()
        else:
            m.poles = None
            m.pole_mask = None
        return m

    def set_inv_eps(self, domain, ie_tensors):
        """Rebinds domain's eps^-1 to the given device tensors (kept alive here)."""
        sc = self.scenes[domain]
        ie = [t.contiguous() for t in ie_tensors]
        if self.streamed is not None:
            pinned = {}
            for t in ie:   # the same tensor three times stays one (isotropic) array
                if id(t) not in pinned:
                    pinned[id(t)] = t if t.is_pinned() else t.cpu().pin_memory()
            ie = [pinned[id(t)] for t in ie]
        self.inv_eps[domain] = ie
        mk = None
        if sc.pole_mask is not None and len(sc.poles):
            mk = self.masks[min(domain, len(self.masks) - 1)]
        fdtd_set_material(self.ctx, domain, self._material_struct(sc, ie, mk))

    # -- stepping and outputs ----------------------------------------------------------------
    def step(self, n):
        fdtd_step_forward(self.ctx, int(n))

    @property
    def step_count(self):
        return fdtd_step_count(self.ctx)

    def dft(self, k=0):
        """Spectra of the k-th monitor as a complex128 device tensor (ncomp, nf, bz, by, bx)."""
        torch = self.torch
        mid, shape, _ = self.monitors[k]
        n = fdtd_dft_size(self.ctx, mid)
        out = torch.empty(2 * n, dtype=torch.float64, device=self.device)
        fdtd_dft_read(self.ctx, mid, out.data_ptr(), out.numel() * 8, 1)
        return torch.view_as_complex(out.view(n, 2)).view(shape)

    def energy(self, domain=0, n=None):
        n = self.step_count if n is None else n
        return fdtd_energy_read(self.ctx, domain, n)

    def part(self, domain, part, which=0):
        torch = self.torch
        n = fdtd_part_size(self.ctx, domain, part)
        out = torch.empty(n, dtype=self.tdtype, device=self.device)
        if n:
            fdtd_get_part(self.ctx, domain, which, part, out.data_ptr())
        return out

    def set_part(self, domain, part, tensor, which=0):
        t = tensor.to(self.device, self.tdtype).contiguous()
        if t.numel() != fdtd_part_size(self.ctx, domain, part):
            raise ValueError("size mismatch")
        if t.numel():
            fdtd_set_part(self.ctx, domain, which, part, t.data_ptr())
        self.torch.cuda.current_stream(self.device).synchronize() if self.stream is None else self.stream.synchronize()

    def field(self, domain, comp, which=0):
        nx, ny, nz = self.scenes[domain].shape
        return self.part(domain, comp, which).view(nz, ny, nx)

    def part_count(self, domain=0):
        return fdtd_part_count(self.ctx, domain)

    def launches(self):
        return fdtd_launch_count(self.ctx)

    def synchronize(self, timeout_ms: int = 600000):
        """Waits at most timeout_ms for the context's work (FdtdError with FDTD_ETIMEOUT if it has
        not finished; the work goes on and the context stays usable; a CUDA error the stream reports
        poisons the context: FDTD_ECUDA)."""
        fdtd_synchronize(self.ctx, int(timeout_ms))

    def close(self):
        if getattr(self, "ctx", None):
            fdtd_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
