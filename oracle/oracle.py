"""ctypes binding of the CPU FP64 oracle (plain C, in this folder).

TEST INFRASTRUCTURE ONLY: the slow, plain reference implementation of the
third-order gas-kinetic scheme with CLS reconstruction that the CUDA library
is checked against.  Only the test-suite, the smoke check and the CPU-baseline
leg of the benchmark may import this module.  It shares no code with the CUDA
library and never imports it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SOURCES = ["or_geom_cls.c", "or_linsolve.c", "or_kinetic.c", "or_scheme.c", "or_limiter.c"]
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (C11, -O2, no FMA contraction, OpenMP over
    faces; OMP_NUM_THREADS=1 gives the single-threaded oracle)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    hdr = os.path.join(_HERE, "or_internal.h")
    if not force and os.path.exists(_LIB_PATH):
        t = os.path.getmtime(_LIB_PATH)
        if all(os.path.getmtime(s) <= t for s in srcs + [hdr]):
            return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=gnu11", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-fopenmp", "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True, cwd=_HERE)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(C.Structure):
    _fields_ = [("gamma", C.c_double), ("cfl", C.c_double), ("mu", C.c_double), ("cls_w", C.c_double),
                ("gmres_m", C.c_int), ("gmres_maxit", C.c_int), ("gmres_rtol", C.c_double),
                ("tau2_exact", C.c_int), ("slope0_mode", C.c_int), ("limiter", C.c_int), ("second_order", C.c_int),
                ("prandtl", C.c_double), ("limit_char", C.c_int), ("cls_global", C.c_int),
                ("cls_M", C.c_int)]


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        P, D, I64, I32, I = C.c_void_p, C.c_double, C.c_int64, C.c_int32, C.c_int
        lib.or_mesh_new.restype = P
        lib.or_mesh_new.argtypes = [P, I64, P, I64, P, P, I64, P, C.POINTER(Params), C.POINTER(I)]
        lib.or_mesh_free.argtypes = [P]
        lib.or_char_basis.argtypes = [P, C.c_double, C.c_double, C.c_double, P, P]
        lib.or_char_basis.restype = None
        lib.or_mesh_ndof.restype = I64
        lib.or_mesh_ndof.argtypes = [P]
        lib.or_cell_geometry.argtypes = [P, P]
        lib.or_face_geometry.argtypes = [P, P]
        lib.or_rcm_perm.argtypes = [P, P]
        lib.or_cls_matrix.restype = I64
        lib.or_cls_matrix.argtypes = [P, P, P, P, P]
        lib.or_cls_rhs.argtypes = [P, P, P]
        lib.or_cls_solve.restype = I
        lib.or_cls_solve.argtypes = [P, P, P, I, P, P]
        lib.or_cls_dense.restype = I
        lib.or_cls_dense.argtypes = [P, P, P]
        lib.or_eval_cell.argtypes = [P, P, P, I, D, D, P]
        lib.or_face_flux.restype = I
        lib.or_face_flux.argtypes = [P, P, P, D, P]
        lib.or_face_flux_subset.restype = I
        lib.or_face_flux_subset.argtypes = [P, P, P, D, P, I64, P]
        lib.or_update.argtypes = [P, P, P]
        lib.or_cfl_dt.restype = D
        lib.or_cfl_dt.argtypes = [P, P]
        lib.or_step.restype = I
        lib.or_step.argtypes = [P, P, D, P, P, P]
        lib.or_point_flux.restype = I
        lib.or_point_flux.argtypes = [P, P, D, C.POINTER(Params), P, P]
        lib.or_state_slopes.restype = I
        lib.or_state_slopes.argtypes = [P, D, P]
        lib.or_interface_w0.restype = I
        lib.or_interface_w0.argtypes = [P, P, D, I, P]
        lib.or_moment_abz.restype = D
        lib.or_moment_abz.argtypes = [D, D, D, D, I, I, I, I]
        lib.or_time_integrals.argtypes = [D, D, I, P]
        lib.or_gauss_legendre.argtypes = [I, P, P]
        lib.or_params_default.argtypes = [C.POINTER(Params)]
        lib.or_ghost_rows.restype = None
        lib.or_ghost_rows.argtypes = [I, P, D, D, D, P, P]
        lib.or_limit.restype = I
        lib.or_limit.argtypes = [P, P, P, P, P]
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def params(**kw) -> Params:
    lib = _load()
    p = Params()
    lib.or_params_default(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


@dataclass
class StepInfo:
    dt: float
    iters: np.ndarray
    relres: np.ndarray
    status: int


class OracleMesh:
    """One mesh with its CLS system, RCM order and ILU(0) factors."""

    def __init__(self, mesh, **prm):
        self._lib = _load()
        self.prm = params(**prm)
        self.nodes = np.ascontiguousarray(mesh.nodes, dtype=np.float64)
        self.tris = np.ascontiguousarray(mesh.tris, dtype=np.int32)
        self.faces = np.ascontiguousarray(mesh.faces, dtype=np.int32)
        self.shift = np.ascontiguousarray(mesh.face_shift, dtype=np.float64)
        self.bc = np.ascontiguousarray(mesh.bc_state, dtype=np.float64)
        self.T = int(self.tris.shape[0])
        self.F = int(self.faces.shape[0])
        err = C.c_int(0)
        h = self._lib.or_mesh_new(_ptr(self.nodes), self.nodes.shape[0], _ptr(self.tris), self.T,
                                  _ptr(self.faces), _ptr(self.shift), self.F, _ptr(self.bc),
                                  C.byref(self.prm), C.byref(err))
        if not h:
            raise RuntimeError(f"oracle mesh construction failed ({err.value})")
        self._h = C.c_void_p(h)
        self.ndof = int(self._lib.or_mesh_ndof(self._h))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.or_mesh_free(h)
            self._h = None

    # geometry -----------------------------------------------------------
    def cell_geometry(self) -> dict:
        out = np.zeros((self.T, 10))
        self._lib.or_cell_geometry(self._h, _ptr(out))
        keys = ["area", "cx", "cy", "crad", "h", "inrad", "mxx", "mxy", "myy", "k"]
        return {k: out[:, i].copy() for i, k in enumerate(keys)}

    def face_geometry(self) -> dict:
        out = np.zeros((self.F, 7))
        self._lib.or_face_geometry(self._h, _ptr(out))
        return {"nx": out[:, 0].copy(), "ny": out[:, 1].copy(), "len": out[:, 2].copy(),
                "gauss": out[:, 3:7].reshape(self.F, 2, 2).copy()}

    def rcm_perm(self) -> np.ndarray:
        p = np.zeros(self.T, dtype=np.int32)
        self._lib.or_rcm_perm(self._h, _ptr(p))
        return p

    # CLS ---------------------------------------------------------------
    def cls_matrix(self):
        nnz = int(self._lib.or_cls_matrix(self._h, None, None, None, None))
        rp = np.zeros(self.ndof + 1, dtype=np.int32)
        col = np.zeros(nnz, dtype=np.int32)
        val = np.zeros(nnz)
        off = np.zeros(self.T, dtype=np.int32)
        self._lib.or_cls_matrix(self._h, _ptr(rp), _ptr(col), _ptr(val), _ptr(off))
        return rp, col, val, off

    def cls_rhs(self, w: np.ndarray) -> np.ndarray:
        w = np.ascontiguousarray(w, dtype=np.float64)
        out = np.zeros((4, self.ndof))
        self._lib.or_cls_rhs(self._h, _ptr(w), _ptr(out))
        return out

    def cls_solve(self, w: np.ndarray, warm: bool = False):
        w = np.ascontiguousarray(w, dtype=np.float64)
        coef = np.zeros((4, 5, self.T))
        it = np.zeros(4, dtype=np.int32)
        rr = np.zeros(4)
        bad = self._lib.or_cls_solve(self._h, _ptr(w), _ptr(coef), int(warm), _ptr(it), _ptr(rr))
        return coef, it, rr, int(bad)

    def cls_dense(self, w: np.ndarray) -> np.ndarray:
        w = np.ascontiguousarray(w, dtype=np.float64)
        coef = np.zeros((4, 5, self.T))
        if self._lib.or_cls_dense(self._h, _ptr(w), _ptr(coef)) != 0:
            raise RuntimeError("dense CLS solve failed")
        return coef

    def eval_cell(self, w, coef, cell: int, x: float, y: float) -> np.ndarray:
        w = np.ascontiguousarray(w, dtype=np.float64)
        coef = np.ascontiguousarray(coef, dtype=np.float64)
        out = np.zeros((6, 4))
        self._lib.or_eval_cell(self._h, _ptr(w), _ptr(coef), int(cell), float(x), float(y), _ptr(out))
        return out

    # scheme ------------------------------------------------------------
    def limit(self, w, coef):
        """Detector + DWBAP limiter: (limited coefficients, flags)."""
        w = np.ascontiguousarray(w, dtype=np.float64)
        coef = np.ascontiguousarray(coef, dtype=np.float64)
        out = np.zeros_like(coef)
        flag = np.zeros(self.T, dtype=np.int32)
        self._lib.or_limit(self._h, _ptr(w), _ptr(coef), _ptr(out), _ptr(flag))
        return out, flag

    def cfl_dt(self, w) -> float:
        w = np.ascontiguousarray(w, dtype=np.float64)
        return float(self._lib.or_cfl_dt(self._h, _ptr(w)))

    def face_flux(self, w, coef, dt: float) -> np.ndarray:
        w = np.ascontiguousarray(w, dtype=np.float64)
        coef = np.ascontiguousarray(coef, dtype=np.float64)
        out = np.zeros((4, self.F))
        bad = self._lib.or_face_flux(self._h, _ptr(w), _ptr(coef), float(dt), _ptr(out))
        if bad:
            raise FloatingPointError(f"{bad} Gauss points with a non-physical state")
        return out

    def face_flux_subset(self, w, coef, dt: float, ids) -> np.ndarray:
        w = np.ascontiguousarray(w, dtype=np.float64)
        coef = np.ascontiguousarray(coef, dtype=np.float64)
        ids = np.ascontiguousarray(ids, dtype=np.int64)
        out = np.zeros((4, ids.shape[0]))
        bad = self._lib.or_face_flux_subset(self._h, _ptr(w), _ptr(coef), float(dt), _ptr(ids), ids.shape[0],
                                            _ptr(out))
        if bad:
            raise FloatingPointError(f"{bad} Gauss points with a non-physical state")
        return out

    def update(self, w, flux) -> np.ndarray:
        w2 = np.array(w, dtype=np.float64, order="C", copy=True)
        flux = np.ascontiguousarray(flux, dtype=np.float64)
        self._lib.or_update(self._h, _ptr(w2), _ptr(flux))
        return w2

    def step(self, w: np.ndarray, dt: float = 0.0):
        """Advance w (4, T) in place by one step; returns StepInfo."""
        assert w.flags.c_contiguous and w.dtype == np.float64
        dto = C.c_double(0.0)
        it = np.zeros(4, dtype=np.int32)
        rr = np.zeros(4)
        st = self._lib.or_step(self._h, _ptr(w), float(dt), C.byref(dto), _ptr(it), _ptr(rr))
        return StepInfo(dto.value, it, rr, int(st))


# kinetic unit functions ------------------------------------------------------

def point_flux(wl: np.ndarray, wr: np.ndarray, dt: float, **prm):
    """Time-integrated flux at one Gauss point, face frame, unit face length.
    wl, wr: (6, 4) rows value, d/dn, d/dt, d2/dn2, d2/dndt, d2/dt2."""
    lib = _load()
    p = params(**prm)
    wl = np.ascontiguousarray(wl, dtype=np.float64)
    wr = np.ascontiguousarray(wr, dtype=np.float64)
    f = np.zeros(4)
    aux = np.zeros(16)
    st = lib.or_point_flux(_ptr(wl), _ptr(wr), float(dt), C.byref(p), _ptr(f), _ptr(aux))
    return f, aux, int(st)


def ghost_rows(tag: int, bc, nx: float, ny: float, wl: np.ndarray, gamma: float = 1.4) -> np.ndarray:
    """Ghost right state (6, 4) of a boundary face with tag `tag` and boundary
    data bc (4,) from the left state wl (6, 4), both in the face frame."""
    lib = _load()
    bc = np.ascontiguousarray(bc, dtype=np.float64)
    wl = np.ascontiguousarray(wl, dtype=np.float64)
    wr = np.zeros((6, 4))
    lib.or_ghost_rows(int(tag), _ptr(bc), float(nx), float(ny), float(gamma), _ptr(wl), _ptr(wr))
    return wr


def char_basis(W, gamma: float = 1.4, nx: float = 1.0, ny: float = 0.0):
    """(R, L) eigenvectors of the Euler flux Jacobian along (nx, ny) at W (4,)."""
    lib = _load()
    W = np.ascontiguousarray(W, dtype=np.float64)
    R = np.zeros(16)
    L = np.zeros(16)
    lib.or_char_basis(_ptr(W), float(gamma), float(nx), float(ny), _ptr(R), _ptr(L))
    return R.reshape(4, 4), L.reshape(4, 4)


def state_slopes(w: np.ndarray, gamma: float = 1.4) -> np.ndarray:
    """Slopes (9, 4): a1 a2 A a11 a12 a22 A1 A2 At of one state (6, 4), full space."""
    lib = _load()
    w = np.ascontiguousarray(w, dtype=np.float64)
    out = np.zeros((9, 4))
    if lib.or_state_slopes(_ptr(w), float(gamma), _ptr(out)) != 0:
        raise RuntimeError("polynomial degree overflow")
    return out


def interface_w0(wl: np.ndarray, wr: np.ndarray, gamma: float = 1.4, mode: int = 0) -> np.ndarray:
    """Interface equilibrium W0 (6, 4) of one Gauss point from the face-frame
    states wl, wr (6, 4); mode = slope0_mode (0 mean, 1 kinetic weighting)."""
    lib = _load()
    wl = np.ascontiguousarray(wl, dtype=np.float64)
    wr = np.ascontiguousarray(wr, dtype=np.float64)
    out = np.zeros((6, 4))
    st = lib.or_interface_w0(_ptr(wl), _ptr(wr), float(gamma), int(mode), _ptr(out))
    if st != 0:
        raise RuntimeError("non-physical state" if st == 1 else "polynomial degree overflow")
    return out


def moment(U: float, V: float, lam: float, K: float, half: int, a: int, b: int, z: int) -> float:
    return float(_load().or_moment_abz(U, V, lam, K, half, a, b, z))


def time_integrals(dt: float, tau: float, tau2_exact: int = 0) -> np.ndarray:
    out = np.zeros(9)
    _load().or_time_integrals(float(dt), float(tau), int(tau2_exact), _ptr(out))
    return out


def gauss_legendre(n: int):
    x = np.zeros(n)
    w = np.zeros(n)
    _load().or_gauss_legendre(int(n), _ptr(x), _ptr(w))
    return x, w
