"""ctypes binding of the C ABI declared in include/mg.h.

Argument marshalling only: every function forwards to the entry point of the
same name in libgbmg.so (built by ``paper_1104_1703_gb300.build``).  Arrays
may be torch tensors (CUDA tensors are passed as device pointers) or numpy
arrays (host pointers), indexed [k, j, i] with x fastest.  There is no CPU
path: if the CUDA library cannot be built or loaded, ``lib()`` raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

MG_OK, MG_ERR_INVALID_ARG, MG_ERR_CUDA, MG_ERR_OOM, MG_ERR_EMPTY_DOMAIN = 0, 1, 2, 3, 4
MG_ERR_NOT_CONVERGED, MG_ERR_DIVERGED, MG_ERR_INTERNAL = 5, 6, 7
MG_MEM_HOST, MG_MEM_DEVICE = 0, 1
MG_FIELD_PHI, MG_FIELD_RHS, MG_FIELD_MASKSUM, MG_FIELD_INVDIAG = 0, 1, 2, 3
MG_HIST_MAX = 256

_vp = ctypes.c_void_p
_i = ctypes.c_int
_d = ctypes.c_double


class MGOptions(ctypes.Structure):
    _fields_ = [("n_pre", _i), ("n_post", _i), ("n_cycles", _i), ("coarse_sweeps", _i), ("hold_solves", _i),
                ("eta", _d), ("order", _i), ("use_graphs", _i), ("precision", _i), ("inner_cycles", _i),
                ("coarse_cluster", _i), ("smoother_pass", _i), ("fp64_sum", _i), ("fine_segments", _i),
                ("coarse_matrix", _i)]


class MGSolveInfo(ctypes.Structure):
    _fields_ = [("cycles", _i), ("order_used", _i), ("switched", _i), ("status", _i),
                ("cell_updates", ctypes.c_longlong), ("r_zero", _d),
                ("r_init", _d), ("r_final", _d), ("rel", _d), ("hist", _d * (MG_HIST_MAX + 1))]


class MGBatchTuning(ctypes.Structure):
    _fields_ = [("threads", _i), ("persistent_ctas", _i), ("bottom_slots", _i), ("n_pre", _i), ("n_post", _i),
                ("ms_per_cycle", _d), ("chunk", _i)]


MG_TUNE_SCHEDULE = 1


class MGError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s (status %d)" % (message, status))
        self.status = status
        self.message = message


# name -> (restype, argtypes); the exported symbols of include/mg.h
SIGNATURES = {
    "mg_default_options": (None, [_vp]),
    "mg_create_hierarchy": (_i, [_vp, _i, _i, _i, _i, _d, _vp, _vp, _vp]),
    "mg_update_mask": (_i, [_vp, _vp, _i]),
    "mg_destroy_hierarchy": (_i, [_vp]),
    "mg_set_rhs": (_i, [_vp, _vp, _i]),
    "mg_set_dirichlet": (_i, [_vp, _vp, _vp, _vp, _i]),
    "mg_set_dirichlet_from_coarse": (_i, [_vp, _vp, _i, _i, _i, _i, _i, _i, _i]),
    "mg_set_solution": (_i, [_vp, _vp, _i]),
    "mg_get_solution": (_i, [_vp, _vp, _i]),
    "mg_vcycle": (_i, [_vp, _vp]),
    "mg_solve": (_i, [_vp, _d, _i, _vp]),
    "mg_residual_norm": (_i, [_vp, _vp, _vp]),
    "mg_get_smoother_pass": (_i, [_vp, _vp]),
    "mg_get_hold": (_i, [_vp, _vp]),
    "mg_set_hold": (_i, [_vp, _i]),
    "mg_last_error": (ctypes.c_char_p, [_vp]),
    "mg_status_string": (ctypes.c_char_p, [_i]),
    "mg_num_levels": (_i, [_vp, _vp, _vp, _vp]),
    "mg_level_info": (_i, [_vp, _i, _vp, _vp, _vp]),
    "mg_level_get": (_i, [_vp, _i, _i, _vp, _i]),
    "mg_level_set": (_i, [_vp, _i, _i, _vp, _i]),
    "mg_level_smooth": (_i, [_vp, _i, _i, _i]),
    "mg_level_restrict": (_i, [_vp, _i, _i]),
    "mg_level_prolong": (_i, [_vp, _i, _i]),
    "mg_residual_norm_noalloc": (_i, [_vp, _vp, _vp, _vp, _vp, _vp, _i, _i, _i, _d, _vp, _vp]),
    "mg_launch_count": (ctypes.c_ulonglong, []),
    "mg_probe_fp64_rate": (_i, [_i, _vp]),
    "mg_checked_build": (_i, []),
    "mg_debug_fail_alloc": (None, [_i]),
    "mg_debug_stall_pass": (None, [_i]),
    "mg_timing_enable": (_i, [_vp, _i]),
    "mg_timing_read": (_i, [_vp, _vp, _vp]),
    "mg_batch_create": (_i, [_i, _vp, _i, _vp, _vp, _vp, _vp, _vp]),
    "mg_batch_destroy": (_i, [_vp]),
    "mg_batch_patch": (_i, [_vp, _i, _vp]),
    "mg_batch_vcycle": (_i, [_vp, _vp]),
    "mg_batch_solve": (_i, [_vp, _d, _i, _vp]),
    "mg_batch_get_tuning": (_i, [_vp, _vp]),
    "mg_batch_set_tuning": (_i, [_vp, _vp]),
    "mg_batch_autotune": (_i, [_vp, _i, _d, _i, _i, _vp]),
    "mg_batch_launches_per_cycle": (_i, [_vp, _vp]),
    "mg_batch_last_error": (ctypes.c_char_p, [_vp]),
    "mg_unet_create": (_i, [_i, _i, _i, _i, _i, _vp, _vp]),
    "mg_unet_destroy": (_i, [_vp]),
    "mg_unet_num_params": (_i, [_vp, _vp]),
    "mg_unet_set_params": (_i, [_vp, _vp, _i]),
    "mg_unet_get_params": (_i, [_vp, _vp, _i]),
    "mg_unet_forward": (_i, [_vp, _vp, _i, _vp, _i]),
    "mg_unet_features": (_i, [_vp, _vp, _vp, _vp, _vp, _vp, _d, _vp, _i, _vp]),
    "mg_unet_predict": (_i, [_vp, _vp, _vp, _vp, _vp, _vp, _d, _vp]),
    "mg_unet_train_patch": (_i, [_vp, _vp, _vp, _vp, _vp, _vp, _d, _vp, _d, _vp]),
    "mg_faces_from_coarse": (_i, [_vp, _vp, _i, _i, _i, _i, _i, _i, _i, _vp, _vp, _vp]),
    "mg_generate_blob_patch": (_i, [ctypes.c_ulonglong, _i, _i, _i, _d, _vp, _vp, _vp, _vp, _vp]),
    "mg_unet_backward": (_i, [_vp, _vp, _i]),
    "mg_unet_get_grads": (_i, [_vp, _vp, _i]),
    "mg_unet_adam_step": (_i, [_vp, _d, _d, _d, _d]),
    "mg_unet_train_step": (_i, [_vp, _vp, _vp, _i, _d, _vp]),
    "mg_unet_layer_info": (_i, [_vp, _i, _vp]),
    "mg_unet_layer_output": (_i, [_vp, _i, _vp, _i]),
    "mg_unet_layer_grad": (_i, [_vp, _i, _vp, _i]),
    "mg_unet_last_error": (ctypes.c_char_p, [_vp]),
}

_LIB = None
_LOCK = threading.Lock()


def lib() -> ctypes.CDLL:
    """Loads libgbmg.so, building it first if it is missing or stale.  With
    MG_CHECKED=1 in the environment it loads the bounds-checked build
    libgbmg_checked.so instead (a debugging aid: every list-driven kernel
    checks its entries, see mg_checked_build in mg.h)."""
    global _LIB
    with _LOCK:
        if _LIB is None:
            path = _build.build(checked=os.environ.get("MG_CHECKED") == "1")
            L = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _LIB = L
    return _LIB


def _check(st, h=None):
    if st != MG_OK:
        raise MGError(st, mg_last_error(h))


def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _in(a, dtype, shape, name):
    """(pointer, where, keepalive) for an input array."""
    if _is_torch(a):
        import torch
        tdt = {np.float64: torch.float64, np.int8: torch.int8, np.int32: torch.int32}[dtype]
        if a.dtype != tdt or not a.is_contiguous() or tuple(a.shape) != tuple(shape):
            raise ValueError("%s: expected a contiguous %s tensor of shape %s" % (name, tdt, shape))
        return _vp(a.data_ptr()), (MG_MEM_DEVICE if a.is_cuda else MG_MEM_HOST), a
    arr = np.ascontiguousarray(a, dtype=dtype)
    if arr.shape != tuple(shape):
        raise ValueError("%s: expected shape %s, got %s" % (name, tuple(shape), arr.shape))
    return arr.ctypes.data_as(_vp), MG_MEM_HOST, arr


def _out(a, dtype, shape, name):
    if a is None:
        a = np.zeros(shape, dtype=dtype)
    if _is_torch(a):
        return _in(a, dtype, shape, name)[:2] + (a,)
    if not (isinstance(a, np.ndarray) and a.dtype == dtype and a.flags.c_contiguous and a.shape == tuple(shape)):
        raise ValueError("%s: expected a contiguous %s array of shape %s" % (name, np.dtype(dtype), shape))
    return a.ctypes.data_as(_vp), MG_MEM_HOST, a


def _default_stream():
    try:
        import torch
        if torch.cuda.is_available() and torch.cuda.is_initialized():
            s = torch.cuda.current_stream().cuda_stream
            return _vp(s) if s else None
    except Exception:
        pass
    return None


# --------------------------------------------------------------------------
# Entry points (same names as the C ABI)
# --------------------------------------------------------------------------

def mg_default_options() -> MGOptions:
    o = MGOptions()
    lib().mg_default_options(ctypes.byref(o))
    return o


def mg_last_error(h=None) -> str:
    return lib().mg_last_error(h).decode()


def mg_status_string(st) -> str:
    return lib().mg_status_string(st).decode()


def mg_create_hierarchy(mask, h, options=None, stream="auto"):
    """Returns an opaque handle; dims are taken from mask.shape = (nz, ny, nx)."""
    nz, ny, nx = mask.shape
    p, where, keep = _in(mask, np.int8, (nz, ny, nx), "mask")
    if stream == "auto":
        stream = _default_stream()
    out = _vp()
    st = lib().mg_create_hierarchy(p, where, nx, ny, nz, float(h),
                                   ctypes.byref(options) if options is not None else None, stream, ctypes.byref(out))
    _check(st)
    return out


def mg_destroy_hierarchy(h):
    _check(lib().mg_destroy_hierarchy(h))


def mg_update_mask(h, mask):
    p, where, keep = _in(mask, np.int8, mask.shape, "mask")
    _check(lib().mg_update_mask(h, p, where), h)


def mg_set_rhs(h, rho):
    p, where, keep = _in(rho, np.float64, rho.shape, "rho")
    _check(lib().mg_set_rhs(h, p, where), h)


def mg_set_dirichlet(h, bx=None, by=None, bz=None):
    ptrs, keeps, wheres = [], [], set()
    for name, a in (("bx", bx), ("by", by), ("bz", bz)):
        if a is None:
            ptrs.append(None)
            continue
        p, where, keep = _in(a, np.float64, a.shape, name)
        ptrs.append(p)
        keeps.append(keep)
        wheres.add(where)
    if len(wheres) > 1:
        raise ValueError("face arrays must all be host or all be device arrays")
    where = wheres.pop() if wheres else MG_MEM_HOST
    _check(lib().mg_set_dirichlet(h, ptrs[0], ptrs[1], ptrs[2], where), h)


def mg_set_dirichlet_from_coarse(h, phi_c, origin):
    cz, cy, cx = phi_c.shape
    p, where, keep = _in(phi_c, np.float64, (cz, cy, cx), "phi_c")
    _check(lib().mg_set_dirichlet_from_coarse(h, p, where, cx, cy, cz, int(origin[0]), int(origin[1]),
                                              int(origin[2])), h)


def mg_set_solution(h, phi=None):
    if phi is None:
        _check(lib().mg_set_solution(h, None, MG_MEM_HOST), h)
        return
    p, where, keep = _in(phi, np.float64, phi.shape, "phi")
    _check(lib().mg_set_solution(h, p, where), h)


def mg_get_solution(h, shape, out=None):
    p, where, keep = _out(out, np.float64, shape, "out")
    _check(lib().mg_get_solution(h, p, where), h)
    return keep


def mg_vcycle(h, want_rel=True):
    rel = _d()
    _check(lib().mg_vcycle(h, ctypes.byref(rel) if want_rel else None), h)
    return rel.value if want_rel else None


def mg_solve(h, tol, max_cycles=100, raise_on_failure=False):
    """Returns (status, info dict); raises MGError for argument and CUDA
    errors, and for NOT_CONVERGED / DIVERGED only if raise_on_failure."""
    info = MGSolveInfo()
    st = lib().mg_solve(h, float(tol), int(max_cycles), ctypes.byref(info))
    if st not in (MG_OK, MG_ERR_NOT_CONVERGED, MG_ERR_DIVERGED) or (raise_on_failure and st != MG_OK):
        _check(st, h)
    n = min(info.cycles, MG_HIST_MAX)
    return st, {"cycles": info.cycles, "order": info.order_used, "switched": info.switched,
                "cell_updates": info.cell_updates,
                "r_zero": info.r_zero, "r_init": info.r_init, "r_final": info.r_final, "rel": info.rel,
                "hist": np.array(info.hist[: n + 1])}


def mg_residual_norm(h):
    r, r0 = _d(), _d()
    _check(lib().mg_residual_norm(h, ctypes.byref(r), ctypes.byref(r0)), h)
    return r.value, r0.value


def mg_get_smoother_pass(h) -> bool:
    v = _i()
    _check(lib().mg_get_smoother_pass(h, ctypes.byref(v)), h)
    return bool(v.value)


def mg_get_hold(h):
    v = _i()
    _check(lib().mg_get_hold(h, ctypes.byref(v)), h)
    return v.value


def mg_set_hold(h, hold):
    _check(lib().mg_set_hold(h, int(hold)), h)


def mg_num_levels(h):
    n, d2, d1 = _i(), _i(), _i()
    _check(lib().mg_num_levels(h, ctypes.byref(n), ctypes.byref(d2), ctypes.byref(d1)), h)
    return n.value, d2.value, d1.value


def mg_level_info(h, level):
    dims = (_i * 3)()
    a2, a1 = ctypes.c_longlong(), ctypes.c_longlong()
    _check(lib().mg_level_info(h, level, dims, ctypes.byref(a2), ctypes.byref(a1)), h)
    return (dims[2], dims[1], dims[0]), a2.value, a1.value


def mg_level_get(h, level, field, out=None):
    shape = mg_level_info(h, level)[0]
    dtype = np.int32 if field == MG_FIELD_MASKSUM else np.float64
    p, where, keep = _out(out, dtype, shape, "out")
    _check(lib().mg_level_get(h, level, field, p, where), h)
    return keep


def mg_level_set(h, level, field, arr):
    shape = mg_level_info(h, level)[0]
    p, where, keep = _in(arr, np.float64, shape, "arr")
    _check(lib().mg_level_set(h, level, field, p, where), h)


def mg_level_smooth(h, level, order, sweeps):
    _check(lib().mg_level_smooth(h, level, order, sweeps), h)


def mg_level_restrict(h, level, order):
    _check(lib().mg_level_restrict(h, level, order), h)


def mg_level_prolong(h, level, order):
    _check(lib().mg_level_prolong(h, level, order), h)


def mg_residual_norm_noalloc(mask, phi, rho, h, norm_out, bx=None, by=None, bz=None, stream=None):
    """Enqueues ||Laplacian(Phi) - rho|| of the fine level into norm_out (a
    one-element float64 CUDA tensor) from CUDA tensors, allocating nothing."""
    nz, ny, nx = mask.shape
    args = []
    for name, a, dt, shape in (("mask", mask, np.int8, (nz, ny, nx)), ("phi", phi, np.float64, (nz, ny, nx)),
                               ("rho", rho, np.float64, (nz, ny, nx)), ("bx", bx, np.float64, (nz, ny, nx + 1)),
                               ("by", by, np.float64, (nz, ny + 1, nx)), ("bz", bz, np.float64, (nz + 1, ny, nx))):
        if a is None:
            args.append(None)
            continue
        p, where, keep = _in(a, dt, shape, name)
        if where != MG_MEM_DEVICE:
            raise ValueError("%s must be a CUDA tensor" % name)
        args.append(p)
    p_out, where, keep = _in(norm_out, np.float64, (1,), "norm_out")
    if where != MG_MEM_DEVICE:
        raise ValueError("norm_out must be a CUDA tensor")
    _check(lib().mg_residual_norm_noalloc(args[0], args[1], args[2], args[3], args[4], args[5], nx, ny, nz,
                                          float(h), p_out, stream))


def mg_launch_count() -> int:
    return int(lib().mg_launch_count())


def mg_probe_fp64_rate(iters=4096) -> float:
    v = _d()
    _check(lib().mg_probe_fp64_rate(int(iters), ctypes.byref(v)))
    return v.value


def mg_checked_build() -> bool:
    return bool(lib().mg_checked_build())


def mg_debug_fail_alloc(nth: int):
    lib().mg_debug_fail_alloc(int(nth))


def mg_debug_stall_pass(on: bool):
    lib().mg_debug_stall_pass(1 if on else 0)


def mg_timing_enable(h, enable=True):
    _check(lib().mg_timing_enable(h, 1 if enable else 0), h)


def mg_timing_read(h):
    n, ms = ctypes.c_longlong(), _d()
    _check(lib().mg_timing_read(h, ctypes.byref(n), ctypes.byref(ms)), h)
    return n.value, ms.value


class Hierarchy:
    """Owns one handle; methods forward to the functions above."""

    def faces_from_coarse(self, phi_c, origin, bx, by, bz):
        mg_faces_from_coarse(self.handle, phi_c, origin, bx, by, bz)

    def __init__(self, mask, h, options=None, stream="auto", **opts):
        if options is None and opts:
            options = mg_default_options()
            for k, v in opts.items():
                setattr(options, k, v)
        self.shape = tuple(mask.shape)
        self.h = float(h)
        self.handle = mg_create_hierarchy(mask, h, options, stream)

    def close(self):
        if self.handle:
            mg_destroy_hierarchy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_rhs(self, rho):
        mg_set_rhs(self.handle, rho)

    def set_dirichlet(self, bx=None, by=None, bz=None):
        mg_set_dirichlet(self.handle, bx, by, bz)

    def set_dirichlet_from_coarse(self, phi_c, origin):
        mg_set_dirichlet_from_coarse(self.handle, phi_c, origin)

    def set_solution(self, phi=None):
        mg_set_solution(self.handle, phi)

    def get_solution(self, out=None):
        return mg_get_solution(self.handle, self.shape, out)

    def update_mask(self, mask):
        mg_update_mask(self.handle, mask)

    def vcycle(self, want_rel=True):
        return mg_vcycle(self.handle, want_rel)

    def solve(self, tol, max_cycles=100):
        return mg_solve(self.handle, tol, max_cycles)

    def residual_norm(self):
        return mg_residual_norm(self.handle)

    @property
    def smoother_pass(self):
        return mg_get_smoother_pass(self.handle)

    @property
    def hold(self):
        return mg_get_hold(self.handle)

    @hold.setter
    def hold(self, v):
        mg_set_hold(self.handle, v)

    def levels(self):
        return mg_num_levels(self.handle)

    def level_info(self, level):
        return mg_level_info(self.handle, level)

    def level_get(self, level, field, out=None):
        return mg_level_get(self.handle, level, field, out)

    def level_set(self, level, field, arr):
        mg_level_set(self.handle, level, field, arr)

    def smooth(self, level, order, sweeps):
        mg_level_smooth(self.handle, level, order, sweeps)

    def restrict_to(self, level, order):
        mg_level_restrict(self.handle, level, order)

    def prolong_from(self, level, order):
        mg_level_prolong(self.handle, level, order)


# --------------------------------------------------------------------------
# Batched solve of many patches
# --------------------------------------------------------------------------

def mg_batch_last_error(b=None) -> str:
    return lib().mg_batch_last_error(b).decode()


def _check_batch(st, b=None):
    if st != MG_OK:
        raise MGError(st, mg_batch_last_error(b))


def _info_dict(info):
    n = min(info.cycles, MG_HIST_MAX)
    return {"cycles": info.cycles, "order": info.order_used, "switched": info.switched, "status": info.status,
            "cell_updates": info.cell_updates, "r_zero": info.r_zero, "r_init": info.r_init,
            "r_final": info.r_final, "rel": info.rel, "hist": np.array(info.hist[: n + 1])}


def mg_batch_create(masks, hs, options=None, stream="auto"):
    """masks: a sequence of (nz, ny, nx) int8 arrays or tensors, all on the
    host or all on the device; hs: one cell size per patch."""
    n = len(masks)
    if n < 1 or len(hs) != n:
        raise ValueError("need one h per mask and at least one patch")
    ptrs = (_vp * n)()
    dims = (_i * (3 * n))()
    harr = (_d * n)(*[float(h) for h in hs])
    keep, where = [], None
    for p, m in enumerate(masks):
        nz, ny, nx = m.shape
        ptr, w, k = _in(m, np.int8, (nz, ny, nx), "mask %d" % p)
        if where is not None and w != where:
            raise ValueError("masks must all be host arrays or all device tensors")
        where = w
        ptrs[p] = ptr
        dims[3 * p], dims[3 * p + 1], dims[3 * p + 2] = nx, ny, nz
        keep.append(k)
    if stream == "auto":
        stream = _default_stream()
    out = _vp()
    st = lib().mg_batch_create(n, ptrs, where, dims, harr, ctypes.byref(options) if options is not None else None,
                               stream, ctypes.byref(out))
    _check_batch(st)
    return out


def mg_batch_destroy(b):
    _check_batch(lib().mg_batch_destroy(b))


def mg_batch_patch(b, p):
    out = _vp()
    _check_batch(lib().mg_batch_patch(b, int(p), ctypes.byref(out)), b)
    return out


def mg_batch_vcycle(b, n, want_rel=True):
    rel = (_d * n)()
    _check_batch(lib().mg_batch_vcycle(b, rel if want_rel else None), b)
    return np.array(rel[:]) if want_rel else None


def mg_batch_solve(b, n, tol, max_cycles=100):
    """Returns (status, list of per-patch info dicts); raises MGError for
    argument and CUDA errors."""
    infos = (MGSolveInfo * n)()
    st = lib().mg_batch_solve(b, float(tol), int(max_cycles), infos)
    if st not in (MG_OK, MG_ERR_NOT_CONVERGED, MG_ERR_DIVERGED):
        _check_batch(st, b)
    return st, [_info_dict(infos[p]) for p in range(n)]


def mg_batch_get_tuning(b):
    t = MGBatchTuning()
    _check_batch(lib().mg_batch_get_tuning(b, ctypes.byref(t)), b)
    return t


def mg_batch_set_tuning(b, t):
    _check_batch(lib().mg_batch_set_tuning(b, ctypes.byref(t)), b)


def mg_batch_autotune(b, reps=5, tol=1e-8, max_cycles=100, flags=0):
    t = MGBatchTuning()
    _check_batch(lib().mg_batch_autotune(b, int(reps), float(tol), int(max_cycles), int(flags), ctypes.byref(t)), b)
    return t


def mg_batch_launches_per_cycle(b):
    v = ctypes.c_longlong()
    _check_batch(lib().mg_batch_launches_per_cycle(b, ctypes.byref(v)), b)
    return v.value


class _Patch(Hierarchy):
    """A patch of a Batch: the batch owns the handle."""

    def __init__(self, batch, p, shape, h):
        self._batch = batch
        self.shape = tuple(shape)
        self.h = float(h)
        self.handle = mg_batch_patch(batch.handle, p)

    def close(self):
        self.handle = None


class Batch:
    """Owns one batch handle; patch(p) gives the hierarchy of patch p."""

    def __init__(self, masks, hs, options=None, stream="auto", **opts):
        if options is None and opts:
            options = mg_default_options()
            for k, v in opts.items():
                setattr(options, k, v)
        self.n = len(masks)
        self.handle = mg_batch_create(masks, hs, options, stream)
        self._patches = [_Patch(self, p, masks[p].shape, hs[p]) for p in range(self.n)]

    def patch(self, p):
        return self._patches[p]

    def close(self):
        if self.handle:
            for q in self._patches:
                q.close()
            mg_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def vcycle(self, want_rel=True):
        return mg_batch_vcycle(self.handle, self.n, want_rel)

    def solve(self, tol, max_cycles=100):
        return mg_batch_solve(self.handle, self.n, tol, max_cycles)

    @property
    def tuning(self):
        return mg_batch_get_tuning(self.handle)

    @tuning.setter
    def tuning(self, t):
        mg_batch_set_tuning(self.handle, t)

    def autotune(self, reps=5, tol=1e-8, max_cycles=100, flags=0):
        return mg_batch_autotune(self.handle, reps, tol, max_cycles, flags)

    def launches_per_cycle(self):
        return mg_batch_launches_per_cycle(self.handle)


# --------------------------------------------------------------------------
# Learned initial guess (3D U-Net)
# --------------------------------------------------------------------------

def mg_unet_last_error(n=None) -> str:
    return lib().mg_unet_last_error(n).decode()


def _check_unet(st, n=None):
    if st != MG_OK:
        raise MGError(st, mg_unet_last_error(n))


def _in_f32(a, shape, name):
    if _is_torch(a):
        import torch
        if a.dtype != torch.float32 or not a.is_contiguous() or tuple(a.shape) != tuple(shape):
            raise ValueError("%s: expected a contiguous float32 tensor of shape %s" % (name, shape))
        return _vp(a.data_ptr()), (MG_MEM_DEVICE if a.is_cuda else MG_MEM_HOST), a
    arr = np.ascontiguousarray(a, dtype=np.float32)
    if arr.shape != tuple(shape):
        raise ValueError("%s: expected shape %s, got %s" % (name, tuple(shape), arr.shape))
    return arr.ctypes.data_as(_vp), MG_MEM_HOST, arr


class UNet:
    """Owns one network handle (the C ABI's mg_unet_*)."""

    def __init__(self, levels, base, shape, stream="auto"):
        nz, ny, nx = shape
        self.shape = tuple(shape)
        if stream == "auto":
            stream = _default_stream()
        out = _vp()
        _check_unet(lib().mg_unet_create(int(levels), int(base), nx, ny, nz, stream, ctypes.byref(out)))
        self.handle = out

    def close(self):
        if self.handle:
            lib().mg_unet_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def num_params(self):
        v = ctypes.c_longlong()
        _check_unet(lib().mg_unet_num_params(self.handle, ctypes.byref(v)), self.handle)
        return v.value

    def set_params(self, flat):
        arr = np.ascontiguousarray(flat, dtype=np.float64)
        if arr.size != self.num_params():
            raise ValueError("expected %d parameters" % self.num_params())
        _check_unet(lib().mg_unet_set_params(self.handle, arr.ctypes.data_as(_vp), MG_MEM_HOST), self.handle)

    def get_params(self):
        out = np.zeros(self.num_params())
        _check_unet(lib().mg_unet_get_params(self.handle, out.ctypes.data_as(_vp), MG_MEM_HOST), self.handle)
        return out

    def forward(self, x, out=None):
        p, where, keep = _in_f32(x, (3,) + self.shape, "x")
        if out is None:
            out = np.zeros(self.shape, dtype=np.float32)
        po, wo, keep_o = _in_f32(out, self.shape, "pred")
        _check_unet(lib().mg_unet_forward(self.handle, p, where, po, wo), self.handle)
        return out

    def backward(self, g_pred):
        p, where, keep = _in_f32(g_pred, self.shape, "g_pred")
        _check_unet(lib().mg_unet_backward(self.handle, p, where), self.handle)

    def get_grads(self):
        out = np.zeros(self.num_params())
        _check_unet(lib().mg_unet_get_grads(self.handle, out.ctypes.data_as(_vp), MG_MEM_HOST), self.handle)
        return out

    def adam_step(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        _check_unet(lib().mg_unet_adam_step(self.handle, float(lr), float(beta1), float(beta2), float(eps)),
                    self.handle)

    def train_step(self, x, y, lr=1e-3):
        px, wx, kx = _in_f32(x, (3,) + self.shape, "x")
        py, wy, ky = _in_f32(y, self.shape, "y")
        if wx != wy:
            raise ValueError("x and y must both be host arrays or both CUDA tensors")
        loss = _d()
        _check_unet(lib().mg_unet_train_step(self.handle, px, py, wx, float(lr), ctypes.byref(loss)), self.handle)
        return loss.value

    @staticmethod
    def _dev(a, name):
        if a is None:
            return None
        if not (_is_torch(a) and a.is_cuda and a.is_contiguous()):
            raise ValueError("%s must be a contiguous CUDA tensor" % name)
        return _vp(a.data_ptr())

    def features(self, mask, rho, faces, h):
        """(x [3][nz][ny][nx] float32 numpy, scale s) of a patch given as CUDA
        tensors (faces a (bx, by, bz) tuple, entries may be None)."""
        x = np.zeros((3,) + self.shape, dtype=np.float32)
        s = _d()
        bx, by, bz = faces
        _check_unet(lib().mg_unet_features(self.handle, self._dev(mask, "mask"), self._dev(rho, "rho"),
                                           self._dev(bx, "bx"), self._dev(by, "by"), self._dev(bz, "bz"), float(h),
                                           x.ctypes.data_as(_vp), MG_MEM_HOST, ctypes.byref(s)), self.handle)
        return x, s.value

    def predict(self, mask, rho, faces, h, phi_out):
        """Writes the learned guess into phi_out (a float64 CUDA tensor)."""
        bx, by, bz = faces
        _check_unet(lib().mg_unet_predict(self.handle, self._dev(mask, "mask"), self._dev(rho, "rho"),
                                          self._dev(bx, "bx"), self._dev(by, "by"), self._dev(bz, "bz"), float(h),
                                          self._dev(phi_out, "phi")), self.handle)
        return phi_out

    def train_patch(self, mask, rho, faces, h, phi, lr=1e-3):
        bx, by, bz = faces
        loss = _d()
        _check_unet(lib().mg_unet_train_patch(self.handle, self._dev(mask, "mask"), self._dev(rho, "rho"),
                                              self._dev(bx, "bx"), self._dev(by, "by"), self._dev(bz, "bz"), float(h),
                                              self._dev(phi, "phi"), float(lr), ctypes.byref(loss)), self.handle)
        return loss.value

    def layer_grad(self, layer):
        dims = (_i * 4)()
        _check_unet(lib().mg_unet_layer_info(self.handle, int(layer), dims), self.handle)
        out = np.zeros(tuple(dims[:4]), dtype=np.float32)
        _check_unet(lib().mg_unet_layer_grad(self.handle, int(layer), out.ctypes.data_as(_vp), MG_MEM_HOST),
                    self.handle)
        return out

    def layer_output(self, layer):
        dims = (_i * 4)()
        _check_unet(lib().mg_unet_layer_info(self.handle, int(layer), dims), self.handle)
        out = np.zeros(tuple(dims[:4]), dtype=np.float32)
        _check_unet(lib().mg_unet_layer_output(self.handle, int(layer), out.ctypes.data_as(_vp), MG_MEM_HOST),
                    self.handle)
        return out


def mg_faces_from_coarse(h, phi_c, origin, bx, by, bz):
    """Writes the interpolated Dirichlet values of hierarchy h's boundary
    faces into the CUDA tensors bx, by, bz."""
    cz, cy, cx = phi_c.shape
    p, where, keep = _in(phi_c, np.float64, (cz, cy, cx), "phi_c")
    for name, a in (("bx", bx), ("by", by), ("bz", bz)):
        if not (_is_torch(a) and a.is_cuda and a.is_contiguous() and a.dtype == __import__("torch").float64):
            raise ValueError("%s must be a contiguous float64 CUDA tensor" % name)
    _check(lib().mg_faces_from_coarse(h, p, where, cx, cy, cz, int(origin[0]), int(origin[1]), int(origin[2]),
                                      _vp(bx.data_ptr()), _vp(by.data_ptr()), _vp(bz.data_ptr())), h)


def mg_generate_blob_patch(seed, shape, scratch, mask, rho, phi_c, corr_cells=8.0, stream=None):
    """Fills the CUDA tensors mask (int8), rho (float64) and phi_c (float64,
    the coarse grid) with the synthetic patch of `seed`; scratch is a float32
    CUDA tensor of at least 2 V + 8 corr_cells + 2 elements."""
    nz, ny, nx = shape
    if stream is None:
        stream = _default_stream()
    st = lib().mg_generate_blob_patch(int(seed) & 0xFFFFFFFFFFFFFFFF, nx, ny, nz, float(corr_cells),
                                      _vp(scratch.data_ptr()), _vp(mask.data_ptr()), _vp(rho.data_ptr()),
                                      _vp(phi_c.data_ptr()), stream)
    _check(st)
