"""ctypes binding of libgks.so (C ABI in include/gks.h).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of the library.  Device arrays are torch tensors (float64, CUDA,
contiguous); the current torch stream is passed to the library.  If the
library has not been built, loading fails with an error: there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgks.so")

GKS_OK, GKS_EINVAL, GKS_ENOMEM, GKS_ECUDA, GKS_ENOCONV, GKS_ENONPHYS, GKS_ETIMEOUT, GKS_EUNSUPPORTED = range(8)
STATUS_NAMES = ["GKS_OK", "GKS_EINVAL", "GKS_ENOMEM", "GKS_ECUDA", "GKS_ENOCONV", "GKS_ENONPHYS", "GKS_ETIMEOUT",
                "GKS_EUNSUPPORTED"]
PC_ILU_EXACT, PC_ILU_SWEEP, PC_BJACOBI, PC_ILU_LEVELS = 0, 1, 2, 3
FP64, MIXED = 0, 1

EXPORTED = ["gks_config_default", "gks_mesh_create", "gks_mesh_destroy", "gks_mesh_get_stats", "gks_cfl_dt",
            "gks_cls_reconstruct", "gks_reset_warm_start", "gks_flux", "gks_step", "gks_run", "gks_point_flux",
            "gks_profile_begin", "gks_profile_end", "gks_launch_count", "gks_cfl_dt_noalloc", "gks_batch_create",
            "gks_batch_run", "gks_limit", "gks_autotune", "gks_last_error", "gks_probe_fma", "gks_probe_read",
            "gks_probe_copy", "gks_probe_df", "gks_probe_wait"]
DF_OPS = {"split": 0, "exp": 1, "expm1": 2, "erfcx": 3, "sqrt": 4, "div": 5, "mul": 6, "add": 7, "recip": 8}
PROF_FLUX, PROF_SPMV, PROF_ILU, PROF_ORTH, PROF_UPDATE, PROF_RESID, PROF_CORR, PROF_CTL = range(8)
PROF_CLASSES = 8


class GksError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")


class Config(C.Structure):
    _fields_ = [("gamma", C.c_double), ("cfl", C.c_double), ("mu", C.c_double), ("cls_w", C.c_double),
                ("gmres_m", C.c_int32), ("gmres_maxit", C.c_int32), ("gmres_rtol", C.c_double),
                ("precision", C.c_int32), ("precond", C.c_int32), ("ilu_sweeps", C.c_int32),
                ("tau2_exact", C.c_int32), ("limiter", C.c_int32),
                ("basis_fp32", C.c_int32), ("warm_extrap", C.c_int32), ("second_order", C.c_int32),
                ("no_graphs", C.c_int32), ("limit_char", C.c_int32),
                ("inner_rtol", C.c_double), ("prandtl", C.c_double), ("slope0_mode", C.c_int32),
                ("ilu_fp16", C.c_int32), ("cls_global", C.c_int32), ("cls_M", C.c_int32),
                ("ilu_sweeps_bwd", C.c_int32), ("ilu_fuse_first", C.c_int32),
                ("flux_split", C.c_int32), ("ilu_sweep_pairs", C.c_int32), ("spmv_dots", C.c_int32),
                ("flux_lead", C.c_int32), ("flux_shape", C.c_int32), ("reserved", C.c_int32)]


class SolveInfo(C.Structure):
    _fields_ = [("iters", C.c_int32 * 4), ("relres", C.c_double * 4), ("converged", C.c_int32)]


class StepInfo(C.Structure):
    _fields_ = [("dt", C.c_double), ("iters", C.c_int32 * 4), ("relres", C.c_double * 4), ("status", C.c_int32)]


class RunInfo(C.Structure):
    _fields_ = [("steps", C.c_int64), ("t", C.c_double), ("last_dt", C.c_double), ("gmres_iters", C.c_int64),
                ("steady_res", C.c_double), ("status", C.c_int32)]


class TuneResult(C.Structure):
    _fields_ = [("ilu_sweeps", C.c_int32), ("warm_extrap", C.c_int32), ("inner_rtol", C.c_double),
                ("ms_per_step", C.c_double), ("ms_per_step_before", C.c_double), ("n_candidates", C.c_int32),
                ("n_failed", C.c_int32), ("ilu_sweeps_bwd", C.c_int32), ("gmres_m", C.c_int32),
                ("flux_variant", C.c_int32)]


class Profile(C.Structure):
    _fields_ = [("n", C.c_int64 * PROF_CLASSES), ("ms", C.c_double * PROF_CLASSES), ("arnoldi", C.c_int64),
                ("arnoldi_jsum", C.c_int64),
                ("precond", C.c_int64), ("residuals", C.c_int64)]


class MeshStats(C.Structure):
    _fields_ = [("n_tri", C.c_int64), ("n_face", C.c_int64), ("n_boundary_face", C.c_int64), ("n_k1", C.c_int64),
                ("nnzb", C.c_int64), ("levels_lower", C.c_int32), ("levels_upper", C.c_int32),
                ("rcm_bandwidth", C.c_int64), ("device_bytes", C.c_int64), ("n_case", C.c_int32)]


class CaseDesc(C.Structure):
    _fields_ = [("nodes", C.c_void_p), ("n_nodes", C.c_int64), ("tris", C.c_void_p), ("n_tri", C.c_int64),
                ("faces", C.c_void_p), ("face_shift", C.c_void_p), ("n_face", C.c_int64), ("bc_state", C.c_void_p)]


class BatchInfo(C.Structure):
    _fields_ = [("steps", C.c_int64), ("gmres_iters", C.c_int64), ("n_failed", C.c_int32), ("n_finished", C.c_int32)]


_lib = None


def load():
    """Load libgks.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_1802_00704_gb300.build.build() "
                          "(there is no CPU fallback)")
    lib = C.CDLL(LIB_PATH)
    P, D, I64, I32 = C.c_void_p, C.c_double, C.c_int64, C.c_int32
    st = C.c_int
    lib.gks_config_default.argtypes = [C.POINTER(Config)]
    lib.gks_config_default.restype = None
    lib.gks_mesh_create.argtypes = [P, I64, P, I64, P, P, I64, P, C.POINTER(Config), C.POINTER(P)]
    lib.gks_mesh_create.restype = st
    lib.gks_batch_create.argtypes = [P, I32, C.POINTER(Config), C.POINTER(P)]
    lib.gks_batch_create.restype = st
    lib.gks_batch_run.argtypes = [P, P, P, I64, P, P, C.POINTER(BatchInfo), P]
    lib.gks_batch_run.restype = st
    lib.gks_mesh_destroy.argtypes = [P]
    lib.gks_mesh_destroy.restype = st
    lib.gks_mesh_get_stats.argtypes = [P, C.POINTER(MeshStats)]
    lib.gks_mesh_get_stats.restype = st
    lib.gks_cfl_dt.argtypes = [P, P, C.POINTER(D), P]
    lib.gks_cfl_dt.restype = st
    lib.gks_cfl_dt_noalloc.argtypes = [P, P, P, P]
    lib.gks_cfl_dt_noalloc.restype = st
    lib.gks_cls_reconstruct.argtypes = [P, P, P, C.POINTER(SolveInfo), P]
    lib.gks_cls_reconstruct.restype = st
    lib.gks_reset_warm_start.argtypes = [P]
    lib.gks_reset_warm_start.restype = st
    lib.gks_flux.argtypes = [P, P, P, D, P, P]
    lib.gks_flux.restype = st
    lib.gks_autotune.argtypes = [P, P, I32, C.POINTER(TuneResult), P]
    lib.gks_autotune.restype = st
    lib.gks_limit.argtypes = [P, P, P, P, P, P]
    lib.gks_limit.restype = st
    lib.gks_step.argtypes = [P, P, C.POINTER(D), C.POINTER(StepInfo), P]
    lib.gks_step.restype = st
    lib.gks_run.argtypes = [P, P, D, I64, D, C.POINTER(RunInfo), P]
    lib.gks_run.restype = st
    lib.gks_point_flux.argtypes = [I64, P, P, D, C.POINTER(Config), P, P]
    lib.gks_point_flux.restype = st
    lib.gks_profile_begin.argtypes = [P, I32]
    lib.gks_profile_begin.restype = st
    lib.gks_profile_end.argtypes = [P, C.POINTER(Profile)]
    lib.gks_profile_end.restype = st
    lib.gks_launch_count.argtypes = []
    lib.gks_launch_count.restype = I64
    lib.gks_probe_fma.argtypes = [I32, I32, I32, P, P, C.POINTER(D)]
    lib.gks_probe_fma.restype = st
    lib.gks_probe_read.argtypes = [P, I64, P, P]
    lib.gks_probe_read.restype = st
    lib.gks_probe_copy.argtypes = [P, P, I64, P]
    lib.gks_probe_copy.restype = st
    lib.gks_probe_df.argtypes = [I32, I64, P, P, P, P]
    lib.gks_probe_df.restype = st
    lib.gks_probe_wait.argtypes = [I64, I32, C.POINTER(I32), C.POINTER(I64), P]
    lib.gks_probe_wait.restype = st
    lib.gks_last_error.argtypes = []
    lib.gks_last_error.restype = C.c_char_p
    _lib = lib
    return lib


def last_error() -> str:
    return load().gks_last_error().decode()


def _check(status: int, where: str, ok=(GKS_OK,)):
    if status not in ok:
        raise GksError(status, where, last_error())
    return status


def config(**kw) -> Config:
    c = Config()
    load().gks_config_default(C.byref(c))
    for k, v in kw.items():
        if not hasattr(c, k):
            raise AttributeError(f"gks_config has no field {k}")
        setattr(c, k, v)
    return c


def _dev(t, shape=None):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"expected shape {shape}, got {tuple(t.shape)}")
    return C.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _mesh_arrays(mesh):
    return (np.ascontiguousarray(mesh.nodes, dtype=np.float64), np.ascontiguousarray(mesh.tris, dtype=np.int32),
            np.ascontiguousarray(mesh.faces, dtype=np.int32), np.ascontiguousarray(mesh.face_shift, dtype=np.float64),
            np.ascontiguousarray(mesh.bc_state, dtype=np.float64))


class GksMesh:
    """A handle: geometry, CLS operator, ILU(0) factors and work buffers in HBM.
    GksMesh(mesh) holds one mesh; GksMesh.batch([mesh, ...]) holds independent
    cases that advance together (state arrays concatenate the cases' cells)."""

    def __init__(self, mesh, **cfg):
        self._lib = load()
        self.cfg = config(**cfg)
        nodes, tris, faces, shift, bc = _mesh_arrays(mesh)
        self.T, self.F = int(tris.shape[0]), int(faces.shape[0])
        self.case_tri = [self.T]
        h = C.c_void_p()
        p = lambda a: a.ctypes.data_as(C.c_void_p)
        _check(self._lib.gks_mesh_create(p(nodes), nodes.shape[0], p(tris), self.T, p(faces), p(shift), self.F,
                                         p(bc), C.byref(self.cfg), C.byref(h)), "gks_mesh_create")
        self._h = h

    @classmethod
    def batch(cls, meshes, **cfg):
        self = cls.__new__(cls)
        self._lib = load()
        self.cfg = config(**cfg)
        keep = [_mesh_arrays(m) for m in meshes]
        descs = (CaseDesc * len(keep))()
        p = lambda a: a.ctypes.data_as(C.c_void_p)
        for q, (nodes, tris, faces, shift, bc) in enumerate(keep):
            descs[q] = CaseDesc(p(nodes), nodes.shape[0], p(tris), tris.shape[0], p(faces), p(shift), faces.shape[0],
                                p(bc))
        self.case_tri = [int(k[1].shape[0]) for k in keep]
        self.T = sum(self.case_tri)
        self.F = sum(int(k[2].shape[0]) for k in keep)
        h = C.c_void_p()
        _check(self._lib.gks_batch_create(descs, len(keep), C.byref(self.cfg), C.byref(h)), "gks_batch_create")
        self._h = h
        return self

    def batch_run(self, w, t_final=None, max_steps: int = 1, stream=None) -> dict:
        n = len(self.case_tri)
        tf = None if t_final is None else np.ascontiguousarray(t_final, dtype=np.float64)
        tr = np.zeros(n)
        cs = np.zeros(n, dtype=np.int32)
        info = BatchInfo()
        p = lambda a: a.ctypes.data_as(C.c_void_p)
        _check(self._lib.gks_batch_run(self._h, _dev(w, (4, self.T)), p(tf) if tf is not None else None,
                                       int(max_steps), p(tr), p(cs), C.byref(info), _stream(stream)),
               "gks_batch_run")
        return {"t": tr, "status": cs, "steps": info.steps, "gmres_iters": info.gmres_iters,
                "n_failed": info.n_failed, "n_finished": info.n_finished}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.gks_mesh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def stats(self) -> dict:
        s = MeshStats()
        _check(self._lib.gks_mesh_get_stats(self._h, C.byref(s)), "gks_mesh_get_stats")
        return {k: getattr(s, k) for k, _ in MeshStats._fields_}

    def cfl_dt(self, w, stream=None) -> float:
        dt = C.c_double(0.0)
        _check(self._lib.gks_cfl_dt(self._h, _dev(w, (4, self.T)), C.byref(dt), _stream(stream)), "gks_cfl_dt")
        return dt.value

    def cfl_dt_noalloc(self, w, dt_dev, stream=None):
        """CFL step into the device scalar dt_dev (1-element float64 CUDA tensor);
        allocates nothing, does not synchronise."""
        _check(self._lib.gks_cfl_dt_noalloc(self._h, _dev(w, (4, self.T)), _dev(dt_dev, (1,)), _stream(stream)),
               "gks_cfl_dt_noalloc")
        return dt_dev

    def cls_reconstruct(self, w, coef=None, stream=None, check=True):
        import torch
        if coef is None:
            coef = torch.empty((4, 5, self.T), dtype=torch.float64, device=w.device)
        info = SolveInfo()
        st = self._lib.gks_cls_reconstruct(self._h, _dev(w, (4, self.T)), _dev(coef, (4, 5, self.T)),
                                           C.byref(info), _stream(stream))
        if check:
            _check(st, "gks_cls_reconstruct")
        return coef, {"iters": list(info.iters), "relres": list(info.relres), "converged": info.converged,
                      "status": st}

    def reset_warm_start(self):
        _check(self._lib.gks_reset_warm_start(self._h), "gks_reset_warm_start")

    def flux(self, w, coef, dt: float, out=None, stream=None, check=True):
        import torch
        if out is None:
            out = torch.empty((4, self.F), dtype=torch.float64, device=w.device)
        st = self._lib.gks_flux(self._h, _dev(w, (4, self.T)), _dev(coef, (4, 5, self.T)), float(dt),
                                _dev(out, (4, self.F)), _stream(stream))
        if check:
            _check(st, "gks_flux")
        return out, st

    def autotune(self, w, trial_steps: int = 3, stream=None) -> dict:
        """Pick ilu_sweeps, ilu_sweeps_bwd, warm_extrap, (mixed) inner_rtol, then the
        GMRES restart length, then (double-FP32 flux) its launch shape, by timing
        trial steps from the state w (not modified); the handle keeps the fastest."""
        r = TuneResult()
        _check(self._lib.gks_autotune(self._h, _dev(w, (4, self.T)), int(trial_steps), C.byref(r), _stream(stream)),
               "gks_autotune")
        self.cfg.ilu_sweeps, self.cfg.warm_extrap, self.cfg.inner_rtol = r.ilu_sweeps, r.warm_extrap, r.inner_rtol
        self.cfg.ilu_sweeps_bwd = r.ilu_sweeps_bwd
        self.cfg.gmres_m = r.gmres_m
        self.cfg.flux_shape = r.flux_variant
        return {k: getattr(r, k) for k, _ in TuneResult._fields_}

    def limit(self, w, coef, out=None, flags=None, stream=None):
        """Shock detector and DWBAP limiter on coef (mesh created with limiter=1);
        returns (limited coefficients, flags: 0 untouched, 1 limited, 2 reset)."""
        import torch
        if out is None:
            out = torch.empty((4, 5, self.T), dtype=torch.float64, device=w.device)
        if flags is None:
            flags = torch.empty(self.T, dtype=torch.int32, device=w.device)
        if not (flags.is_cuda and flags.dtype == torch.int32 and flags.is_contiguous() and flags.numel() == self.T):
            raise TypeError("flags: expected a contiguous int32 CUDA tensor of n_tri elements")
        _check(self._lib.gks_limit(self._h, _dev(w, (4, self.T)), _dev(coef, (4, 5, self.T)),
                                   _dev(out, (4, 5, self.T)), C.c_void_p(flags.data_ptr()), _stream(stream)),
               "gks_limit")
        return out, flags

    def step(self, w, dt: float = 0.0, stream=None, check=True) -> dict:
        info = StepInfo()
        d = C.c_double(dt)
        st = self._lib.gks_step(self._h, _dev(w, (4, self.T)), C.byref(d), C.byref(info), _stream(stream))
        if check:
            _check(st, "gks_step")
        return {"dt": d.value, "iters": list(info.iters), "relres": list(info.relres), "status": st}

    def step_async(self, w, dt_ptr, info_ptr, stream_ptr) -> int:
        """Raw call for timing loops: pointers already marshalled."""
        return self._lib.gks_step(self._h, w, dt_ptr, info_ptr, stream_ptr)

    def profile_begin(self, classes) -> None:
        mask = 0
        for c in classes:
            mask |= 1 << c
        _check(self._lib.gks_profile_begin(self._h, mask), "gks_profile_begin")

    def profile_end(self) -> dict:
        p = Profile()
        _check(self._lib.gks_profile_end(self._h, C.byref(p)), "gks_profile_end")
        return {"n": list(p.n), "ms": list(p.ms), "arnoldi": p.arnoldi, "arnoldi_jsum": p.arnoldi_jsum,
                "precond": p.precond, "residuals": p.residuals}

    def run(self, w, t_final: float = 0.0, max_steps: int = 1, steady_tol: float = 0.0, stream=None,
            check=True) -> dict:
        info = RunInfo()
        st = self._lib.gks_run(self._h, _dev(w, (4, self.T)), float(t_final), int(max_steps), float(steady_tol),
                               C.byref(info), _stream(stream))
        if check:
            _check(st, "gks_run")
        return {k: getattr(info, k) for k, _ in RunInfo._fields_}


def launch_count() -> int:
    """Kernel launches issued by the library in this process."""
    return int(load().gks_launch_count())


def point_flux(wl, wr, dt: float, out=None, stream=None, **cfg):
    """Gauss-point fluxes for n face-frame state pairs wl, wr (n, 6, 4) -> (n, 4)."""
    import torch
    n = int(wl.shape[0])
    if out is None:
        out = torch.empty((n, 4), dtype=torch.float64, device=wl.device)
    c = config(**cfg)
    _check(load().gks_point_flux(n, _dev(wl, (n, 6, 4)), _dev(wr, (n, 6, 4)), float(dt), C.byref(c),
                                 _dev(out, (n, 4)), _stream(stream)), "gks_point_flux")
    return out


def probe_fma(fp64: bool, sink, blocks_per_sm: int = 8, iters: int = 4096, stream=None) -> float:
    """Launch the FMA-chain probe on the stream; returns the launch's flops.
    sink: float64 CUDA tensor of at least blocks_per_sm x (SM count) entries."""
    fl = C.c_double(0.0)
    _check(load().gks_probe_fma(int(bool(fp64)), int(blocks_per_sm), int(iters), _dev(sink), _stream(stream),
                                C.byref(fl)), "gks_probe_fma")
    return fl.value


def probe_read(buf, sink, stream=None) -> int:
    """Launch the streaming-read probe over a CUDA tensor; returns the bytes read."""
    nbytes = buf.numel() * buf.element_size()
    _check(load().gks_probe_read(C.c_void_p(buf.data_ptr()), nbytes, _dev(sink), _stream(stream)),
           "gks_probe_read")
    return nbytes


def probe_copy(src, dst, stream=None) -> int:
    """Launch the copy probe src -> dst (CUDA tensors of the same size); returns bytes read + written."""
    nbytes = src.numel() * src.element_size()
    if dst.numel() * dst.element_size() != nbytes:
        raise ValueError("probe_copy: sizes differ")
    _check(load().gks_probe_copy(C.c_void_p(src.data_ptr()), C.c_void_p(dst.data_ptr()), nbytes, _stream(stream)),
           "gks_probe_copy")
    return 2 * nbytes


def probe_df(op: str, x, y=None, stream=None):
    """Apply a double-FP32 operation of the mixed flux elementwise to the float64
    CUDA tensor x (and y); returns a (n, 2) float64 tensor (see gks_probe_df)."""
    import torch
    out = torch.empty((x.numel(), 2), dtype=torch.float64, device=x.device)
    _check(load().gks_probe_df(DF_OPS[op], x.numel(), _dev(x), _dev(y) if y is not None else None, _dev(out),
                               _stream(stream)), "gks_probe_df")
    return out


def probe_wait(limit_ns: int, set_flag: bool, stream=None) -> tuple:
    """The solver's bounded device wait on its own (see gks_probe_wait):
    (timed_out, waited_ns)."""
    to, ns = C.c_int32(0), C.c_int64(0)
    _check(load().gks_probe_wait(int(limit_ns), int(bool(set_flag)), C.byref(to), C.byref(ns), _stream(stream)),
           "gks_probe_wait")
    return bool(to.value), int(ns.value)
