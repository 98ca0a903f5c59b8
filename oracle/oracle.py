"""ctypes access to the plain FP64 CPU oracle in ``mg_oracle.c``.

TEST INFRASTRUCTURE ONLY.  The oracle restates Guillet & Teyssier,
arXiv:1104.1703 (Sections 2-4, Figs. 3 and 5) as straight CPU loops.  Only
the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module.  The CUDA library never imports it and
shares no code with it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# MG_ORACLE_SRC / MG_ORACLE_BUILD let the mutation tests load a copy of the
# source with one planted mistake; nothing else sets them.
_SRC = os.environ.get("MG_ORACLE_SRC") or os.path.join(_HERE, "mg_oracle.c")
_BUILD = os.environ.get("MG_ORACLE_BUILD") or os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_LOCK = threading.Lock()
_LIB = None

_i32 = ctypes.c_int
_i64 = ctypes.c_int64
_dbl = ctypes.c_double
_vp = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FMA contraction, OpenMP if the
    compiler has it).  Returns the path of the shared library."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    base = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c99", _SRC, "-lm"]
    tmp = _SO + ".tmp%d" % os.getpid()
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:] + ["-o", tmp], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + ["-o", tmp], check=True, capture_output=True)
    os.replace(tmp, _SO)
    return _SO


def lib() -> ctypes.CDLL:
    global _LIB
    with _LOCK:
        if _LIB is None:
            L = ctypes.CDLL(build())
            L.orc_theta.restype = _dbl
            L.orc_theta.argtypes = [_dbl, _dbl]
            L.orc_ghost.restype = _dbl
            L.orc_ghost.argtypes = [_dbl, _dbl, _dbl]
            L.orc_is_active.restype = _i32
            L.orc_is_active.argtypes = [_i64, _i32, _i32]
            L.orc_num_threads.restype = _i32
            L.orc_laplacian.argtypes = [_i32, _i32, _i32, _i32, _vp, _i32, _dbl, _vp, _vp, _vp, _vp, _vp]
            L.orc_residual.argtypes = [_i32, _i32, _i32, _i32, _vp, _i32, _dbl, _vp, _vp, _vp, _vp, _vp, _vp]
            L.orc_gs_sweeps.argtypes = [_i32, _i32, _i32, _i32, _vp, _i32, _dbl, _vp, _vp, _vp, _vp, _vp, _i32]
            L.orc_mask_restrict.restype = ctypes.c_long
            L.orc_mask_restrict.argtypes = [_i32, _i32, _i32, _i32, _vp, _vp]
            L.orc_restrict.argtypes = [_i32, _i32, _i32, _vp, _vp]
            L.orc_prolong_add.argtypes = [_i32, _i32, _i32, _vp, _i32, _i32, _i32, _i32, _vp, _i32, _vp]
            L.orc_dirichlet_from_coarse.restype = _i32
            L.orc_dirichlet_from_coarse.argtypes = [_i32, _i32, _i32, _vp, _vp, _i32, _i32, _i32,
                                                    _i32, _i32, _i32, _vp, _vp, _vp]
            L.orc_create.restype = _vp
            L.orc_create.argtypes = [_vp, _i32, _i32, _i32, _dbl]
            L.orc_destroy.argtypes = [_vp]
            L.orc_num_levels.restype = _i32
            L.orc_num_levels.argtypes = [_vp]
            L.orc_deepest.restype = _i32
            L.orc_deepest.argtypes = [_vp, _i32]
            L.orc_level_active.restype = ctypes.c_long
            L.orc_level_active.argtypes = [_vp, _i32, _i32]
            L.orc_level_dims.argtypes = [_vp, _i32, _vp]
            L.orc_get_hold.restype = _i32
            L.orc_get_hold.argtypes = [_vp]
            L.orc_set_hold.argtypes = [_vp, _i32]
            L.orc_level_ptr.restype = _vp
            L.orc_level_ptr.argtypes = [_vp, _i32, _i32]
            L.orc_set_rhs.argtypes = [_vp, _vp]
            L.orc_set_faces.argtypes = [_vp, _vp, _vp, _vp]
            L.orc_set_phi.argtypes = [_vp, _vp]
            L.orc_get_phi.argtypes = [_vp, _vp]
            L.orc_level_smooth.argtypes = [_vp, _i32, _i32, _i32]
            L.orc_level_residual.restype = _dbl
            L.orc_level_residual.argtypes = [_vp, _i32, _i32]
            L.orc_level_restrict.argtypes = [_vp, _i32, _i32]
            L.orc_level_prolong.argtypes = [_vp, _i32, _i32]
            L.orc_vcycle.argtypes = [_vp, _i32, _i32, _i32, _i32, _i32]
            L.orc_residual_norm.restype = _dbl
            L.orc_residual_norm.argtypes = [_vp]
            L.orc_residual_norm_zero.restype = _dbl
            L.orc_residual_norm_zero.argtypes = [_vp]
            L.orc_solve.restype = _i32
            L.orc_solve.argtypes = [_vp, _i32, _i32, _i32, _i32, _i32, _i32, _dbl, _dbl, _i32, _vp, _vp]
            _LIB = L
    return _LIB


def _p(a):
    return None if a is None else a.ctypes.data_as(_vp)


def _c(a, dtype):
    return None if a is None else np.ascontiguousarray(a, dtype=dtype)


def num_threads() -> int:
    return lib().orc_num_threads()


# --------------------------------------------------------------------------
# Pointwise formulas (Section 3, Fig. 5)
# --------------------------------------------------------------------------

def theta(m_i: float, m_j: float) -> float:
    return lib().orc_theta(m_i, m_j)


def ghost(phi_i: float, phi_b: float, th: float) -> float:
    return lib().orc_ghost(phi_i, phi_b, th)


def is_active(S: int, level: int, order: int) -> bool:
    return bool(lib().orc_is_active(S, level, order))


# --------------------------------------------------------------------------
# Operators on caller arrays; arrays are indexed [k, j, i] (x fastest)
# --------------------------------------------------------------------------

def _faces(bx, by, bz):
    return _c(bx, np.float64), _c(by, np.float64), _c(bz, np.float64)


def laplacian(S, level, order, hl, phi, bx=None, by=None, bz=None):
    S = _c(S, np.int64)
    phi = _c(phi, np.float64)
    nz, ny, nx = S.shape
    bx, by, bz = _faces(bx, by, bz)
    out = np.zeros_like(phi)
    lib().orc_laplacian(nx, ny, nz, level, _p(S), order, hl, _p(phi), _p(bx), _p(by), _p(bz), _p(out))
    return out


def residual(S, level, order, hl, phi, rho, bx=None, by=None, bz=None):
    S = _c(S, np.int64)
    phi = _c(phi, np.float64)
    rho = _c(rho, np.float64)
    nz, ny, nx = S.shape
    bx, by, bz = _faces(bx, by, bz)
    out = np.zeros_like(phi)
    lib().orc_residual(nx, ny, nz, level, _p(S), order, hl, _p(phi), _p(rho), _p(bx), _p(by), _p(bz), _p(out))
    return out


def gs_sweeps(S, level, order, hl, phi, rho, sweeps=1, bx=None, by=None, bz=None):
    S = _c(S, np.int64)
    phi = np.array(phi, dtype=np.float64, copy=True, order="C")
    rho = _c(rho, np.float64)
    nz, ny, nx = S.shape
    bx, by, bz = _faces(bx, by, bz)
    lib().orc_gs_sweeps(nx, ny, nz, level, _p(S), order, hl, _p(phi), _p(rho), _p(bx), _p(by), _p(bz), sweeps)
    return phi


def mask_restrict(S, level):
    S = _c(S, np.int64)
    nz, ny, nx = S.shape
    Sc = np.zeros(((nz + 1) // 2, (ny + 1) // 2, (nx + 1) // 2), dtype=np.int64)
    lib().orc_mask_restrict(nx, ny, nz, level, _p(S), _p(Sc))
    return Sc


def restrict(r):
    r = _c(r, np.float64)
    nz, ny, nx = r.shape
    rc = np.zeros(((nz + 1) // 2, (ny + 1) // 2, (nx + 1) // 2))
    lib().orc_restrict(nx, ny, nz, _p(r), _p(rc))
    return rc


def prolong_add(ec, Sf, level_f, order, phi):
    ec = _c(ec, np.float64)
    Sf = _c(Sf, np.int64)
    phi = np.array(phi, dtype=np.float64, copy=True, order="C")
    cz, cy, cx = ec.shape
    nz, ny, nx = Sf.shape
    lib().orc_prolong_add(cx, cy, cz, _p(ec), nx, ny, nz, level_f, _p(Sf), order, _p(phi))
    return phi


def dirichlet_from_coarse(mask, phi_c, origin):
    """Face values (bx, by, bz) trilinearly interpolated from a coarse AMR
    solution at spacing 2h whose cell (0,0,0) has its lower corner at
    ``origin`` (fine-cell units).  Raises ValueError if a needed face lies
    outside the coarse cell centres."""
    mask = _c(mask, np.int8)
    pc = _c(phi_c, np.float64)
    nz, ny, nx = mask.shape
    cz, cy, cx = pc.shape
    bx = np.zeros((nz, ny, nx + 1))
    by = np.zeros((nz, ny + 1, nx))
    bz = np.zeros((nz + 1, ny, nx))
    st = lib().orc_dirichlet_from_coarse(nx, ny, nz, _p(mask), _p(pc), cx, cy, cz, int(origin[0]),
                                         int(origin[1]), int(origin[2]), _p(bx), _p(by), _p(bz))
    if st != 0:
        raise ValueError("coarse grid does not cover every boundary face")
    return bx, by, bz


# --------------------------------------------------------------------------
# Whole-hierarchy object
# --------------------------------------------------------------------------

class Hierarchy:
    """The oracle's multigrid hierarchy for one fine level (Section 2)."""

    def __init__(self, mask, h):
        mask = _c(mask, np.int8)
        self.shape = mask.shape
        nz, ny, nx = mask.shape
        self._mask = mask
        self._h = lib().orc_create(_p(mask), nx, ny, nz, float(h))
        if not self._h:
            raise ValueError("empty domain or invalid arguments")
        self.h = float(h)

    def close(self):
        if self._h:
            lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def num_levels(self):
        return lib().orc_num_levels(self._h)

    def deepest(self, order):
        return lib().orc_deepest(self._h, order)

    def level_active(self, level, order):
        return lib().orc_level_active(self._h, level, order)

    def level_shape(self, level):
        d = np.zeros(3, dtype=np.int32)
        lib().orc_level_dims(self._h, level, _p(d))
        return (int(d[2]), int(d[1]), int(d[0]))

    @property
    def hold(self):
        return lib().orc_get_hold(self._h)

    @hold.setter
    def hold(self, v):
        lib().orc_set_hold(self._h, int(v))

    def _view(self, level, field):
        shape = self.level_shape(level)
        n = shape[0] * shape[1] * shape[2]
        ptr = lib().orc_level_ptr(self._h, level, field)
        ct = ctypes.c_int64 if field == 0 else ctypes.c_double
        buf = (ct * n).from_address(ptr)
        return np.ctypeslib.as_array(buf).reshape(shape)

    def S(self, level):
        return self._view(level, 0).copy()

    def phi(self, level=0):
        return self._view(level, 1).copy()

    def rhs(self, level=0):
        return self._view(level, 2).copy()

    def res(self, level=0):
        return self._view(level, 3).copy()

    def set_level_phi(self, level, arr):
        self._view(level, 1)[...] = arr

    def set_level_rhs(self, level, arr):
        self._view(level, 2)[...] = arr

    def set_rhs(self, rho):
        rho = _c(rho, np.float64)
        lib().orc_set_rhs(self._h, _p(rho))

    def set_faces(self, bx=None, by=None, bz=None):
        bx, by, bz = _faces(bx, by, bz)
        lib().orc_set_faces(self._h, _p(bx), _p(by), _p(bz))

    def set_phi(self, phi=None):
        phi = _c(phi, np.float64)
        lib().orc_set_phi(self._h, _p(phi))

    def get_phi(self):
        out = np.zeros(self.shape)
        lib().orc_get_phi(self._h, _p(out))
        return out

    def smooth(self, level, order, sweeps):
        lib().orc_level_smooth(self._h, level, order, sweeps)

    def level_residual(self, level, order):
        return lib().orc_level_residual(self._h, level, order)

    def restrict_to(self, level, order):
        lib().orc_level_restrict(self._h, level, order)

    def prolong_from(self, level, order):
        lib().orc_level_prolong(self._h, level, order)

    def vcycle(self, order=2, n_pre=2, n_post=2, n_cycles=1, coarse_sweeps=50):
        lib().orc_vcycle(self._h, order, n_pre, n_post, n_cycles, coarse_sweeps)

    def residual_norm(self):
        return lib().orc_residual_norm(self._h)

    def residual_norm_zero(self):
        return lib().orc_residual_norm_zero(self._h)

    def solve(self, tol, max_cycles=100, order=0, n_pre=2, n_post=2, n_cycles=1, coarse_sweeps=50,
              hold_solves=10, eta=0.5):
        """Returns (status, info dict).  status 0 converged, 1 not converged,
        2 non-finite residual."""
        info = np.zeros(6)
        hist = np.zeros(max_cycles + 1)
        st = lib().orc_solve(self._h, order, n_pre, n_post, n_cycles, coarse_sweeps, hold_solves, eta,
                             tol, max_cycles, _p(info), _p(hist))
        cyc = int(info[0])
        return st, {"cycles": cyc, "order": int(info[1]), "switched": int(info[2]), "r_zero": info[3],
                    "r_final": info[4], "rel": info[5], "hist": hist[: cyc + 1].copy()}
