"""Thin ctypes binding of libmfsolve.so (include/mfsolve.h).

Argument marshalling only: every step of analysis, factorization, solve and
refinement runs in the C/CUDA library.  Device arrays are torch CUDA tensors
(PyTorch supplies device memory and streams); host arrays are numpy.  The
library must be present: importing this module raises if it is not, and no
step falls back to a CPU implementation.

Multi-right-hand-side vectors are passed as contiguous ``(nrhs, n_dof)``
tensors, i.e. the column-major ``n_dof x nrhs`` layout of the C ABI.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmfsolve.so")

MF_OK, MF_EINVAL, MF_ENOMEM, MF_ECUDA, MF_EZERO_PIVOT, MF_ENOCONV, MF_ETIMEOUT, MF_ENOTSUP = 0, -1, -2, -3, -4, -5, -6, -7
MF_ETOOLARGE = -8
MF_NOALLOC_MAX_ENTRIES = 1 << 20
MF_F64, MF_F32, MF_TF32, MF_TF32_BF16 = 0, 1, 2, 3
PRECISIONS = {"f64": MF_F64, "f32": MF_F32, "tf32": MF_TF32, "tf32_bf16": MF_TF32_BF16}
MF_FUSED_BUCKETS = 9
FUSED_BOUNDS = (16, 32, 48, 64, 96, 128, 160, 192, 224)


class mf_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("pivot_tol", ctypes.c_double), ("pivot_fail", ctypes.c_int),
                ("small_front_max", ctypes.c_int), ("panel_width", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("max_nrhs", ctypes.c_int), ("subtree_levels", ctypes.c_int), ("sweep_kernel", ctypes.c_int),
                ("subtree_solve_levels", ctypes.c_int),
                ("tc_min_cb", ctypes.c_int),
                ("super_panel", ctypes.c_int), ("fused_threads", ctypes.c_int * MF_FUSED_BUCKETS),
                ("lookahead", ctypes.c_int), ("bf16_min_cb", ctypes.c_int), ("bf16_passes", ctypes.c_int),
                ("foata_classes", ctypes.c_int), ("symmetric", ctypes.c_int), ("refine_cg", ctypes.c_int),
                ("panel_trsm", ctypes.c_int), ("tc_direct", ctypes.c_int),
                ("root_f64", ctypes.c_int)]

    def as_dict(self) -> dict:
        return {f: (list(getattr(self, f)) if f == "fused_threads" else getattr(self, f)) for f, _ in self._fields_}


class mf_mesh_desc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n_nodes", ctypes.c_int64), ("n_elem", ctypes.c_int64),
                ("nodes_per_elem", ctypes.c_int), ("elem_nodes", ctypes.c_void_p),
                ("elem_centroid", ctypes.c_void_p), ("grid_dims", ctypes.c_void_p)]


class mf_info(ctypes.Structure):
    _fields_ = [("n_dof", ctypes.c_int64), ("n_elem", ctypes.c_int64), ("n_front", ctypes.c_int64),
                ("n_meshes", ctypes.c_int64), ("n_classes", ctypes.c_int32), ("max_m", ctypes.c_int32),
                ("max_k", ctypes.c_int32), ("root_m", ctypes.c_int32), ("sum_k", ctypes.c_int64),
                ("nnz_lu", ctypes.c_int64), ("sum_cb", ctypes.c_int64), ("factor_flops", ctypes.c_double),
                ("solve_flops", ctypes.c_double)]


class mf_status_info(ctypes.Structure):
    _fields_ = [("n_perturbed", ctypes.c_int64), ("first_front", ctypes.c_int32), ("first_pivot", ctypes.c_int32),
                ("nonfinite", ctypes.c_int32), ("timeout", ctypes.c_int32)]


class mf_refine_info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("backward_error", ctypes.c_double), ("rel_residual", ctypes.c_double)]


class mf_trace_rec(ctypes.Structure):
    _fields_ = [("family", ctypes.c_int), ("kind", ctypes.c_int), ("cls", ctypes.c_int), ("tasks", ctypes.c_int),
                ("ms", ctypes.c_double), ("bytes", ctypes.c_double), ("flops", ctypes.c_double)]


TRACE_KINDS = {0: "fused", 1: "assemble", 2: "panel_diag", 3: "gemm", 4: "inv_diag", 5: "subtree", 6: "gemm_tc",
               7: "fused_grp", 8: "tc_pack", 9: "foata", 13: "sym_r", 14: "sym_mirror", 15: "panel_trsm", 16: "gemm_tcd",
               100: "fwd_class", 101: "bwd_class", 102: "subtree_fwd", 103: "subtree_bwd", 104: "fwd_sweep",
               105: "bwd_sweep", 199: "other"}


class mf_tune_info(ctypes.Structure):
    _fields_ = [("ms_default", ctypes.c_double), ("ms_best", ctypes.c_double), ("candidates", ctypes.c_int),
                ("from_cache", ctypes.c_int)]


# every symbol include/mfsolve.h declares
EXPORTS = ["mf_default_options", "mf_strerror", "mf_analyze_mesh", "mf_analyze_batch", "mf_analyze_csr",
           "mf_analysis_info",
           "mf_analysis_export", "mf_factors_create", "mf_factor", "mf_solve", "mf_solve_adjoint", "mf_refine_solve",
           "mf_refine_solve_adjoint", "mf_residual", "mf_element_grad", "mf_element_outer", "mf_status",
           "mf_factors_export_front",
           "mf_free_factors", "mf_free_analysis", "mf_profile_enable", "mf_profile_read", "mf_residual_noalloc",
           "mf_autotune", "mf_profile_trace", "mf_test_fail_alloc", "mf_test_bounded_wait"]
PROFILE_FAMILIES = ["fused", "assemble", "panel", "trailing_gemm", "schur_gemm", "forward", "backward", "residual",
                    "other", "inverse"]


class MFError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {_lib.mf_strerror(code).decode()} ({code})")


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libmfsolve.so not built ({LIB_PATH}); run python -m paper_2306_08994_b300.build")
    L = ctypes.CDLL(LIB_PATH)
    P, I, I64, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
    sig = {
        "mf_default_options": ([P], None), "mf_strerror": ([I], ctypes.c_char_p),
        "mf_analyze_mesh": ([P, P, P], I), "mf_analyze_batch": ([P, I, P, P], I),
        "mf_analyze_csr": ([I64, P, P, P, P], I),
        "mf_analysis_info": ([P, P], I), "mf_analysis_export": ([P, P, P, P, P, P, P], I),
        "mf_factors_create": ([P, P, P], I), "mf_factor": ([P, P, P], I),
        "mf_solve": ([P, P, I, P], I), "mf_solve_adjoint": ([P, P, I, P], I),
        "mf_refine_solve": ([P, P, P, P, I, D, I, P, P], I), "mf_residual": ([P, P, P, P, P, I, P], I),
        "mf_refine_solve_adjoint": ([P, P, P, P, I, D, I, P, P], I),
        "mf_element_grad": ([P, P, P, P, P, P], I), "mf_element_outer": ([P, P, P, I, P, P], I),
        "mf_status": ([P, P], I), "mf_factors_export_front": ([P, ctypes.c_int32, P, P], I),
        "mf_free_factors": ([P], None), "mf_free_analysis": ([P], None),
        "mf_profile_enable": ([P, I], I), "mf_profile_read": ([P, P, P, P, P], I),
        "mf_residual_noalloc": ([I64, I64, I, P, P, P, P, P, I, P], I),
        "mf_autotune": ([P, P, P, P, I, ctypes.c_char_p, P, P, P], I),
        "mf_profile_trace": ([P, P, I, P], I),
        "mf_test_fail_alloc": ([I64], None), "mf_test_bounded_wait": ([P, D, P], I),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    return L


_lib = _load()


def lib():
    return _lib


def _check(rc: int, what: str):
    if rc != MF_OK:
        raise MFError(rc, what)


def default_options(**kw) -> mf_options:
    o = mf_options()
    _lib.mf_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = PRECISIONS[v]
        if k == "fused_threads":
            v = (ctypes.c_int * MF_FUSED_BUCKETS)(*v)
        setattr(o, k, v)
    return o


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _dptr(t) -> int:
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _stream(stream) -> Optional[int]:
    import torch
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Mesh:
    """Host description of one mesh: element->node table plus the geometry the tree is cut from."""

    def __init__(self, elem_nodes: np.ndarray, n_nodes: int, dim: int, grid_dims: Optional[Sequence[int]] = None,
                 centroids: Optional[np.ndarray] = None):
        self.elem_nodes = np.ascontiguousarray(elem_nodes, dtype=np.int64)
        self.n_nodes, self.dim = int(n_nodes), int(dim)
        self.grid_dims = None if grid_dims is None else np.ascontiguousarray(
            list(grid_dims) + [1] * (3 - len(grid_dims)), dtype=np.int32)
        self.centroids = None if centroids is None else np.ascontiguousarray(centroids, dtype=np.float64)
        if self.grid_dims is None and self.centroids is None:
            raise ValueError("need grid_dims or centroids")

    def desc(self) -> mf_mesh_desc:
        d = mf_mesh_desc()
        d.dim, d.n_nodes = self.dim, self.n_nodes
        d.n_elem, d.nodes_per_elem = self.elem_nodes.shape
        d.elem_nodes = _ptr(self.elem_nodes)
        d.elem_centroid = _ptr(self.centroids) if self.centroids is not None else None
        d.grid_dims = _ptr(self.grid_dims) if self.grid_dims is not None else None
        return d


class Analysis:
    """mf_analyze_mesh / mf_analyze_batch: tree, pivot sets, fronts, Foata classes."""

    def __init__(self, meshes, options: Optional[mf_options] = None):
        if isinstance(meshes, Mesh):
            meshes = [meshes]
        self.meshes = list(meshes)
        self.options = options or default_options()
        descs = (mf_mesh_desc * len(self.meshes))(*[m.desc() for m in self.meshes])
        h = ctypes.c_void_p()
        _check(_lib.mf_analyze_batch(descs, len(self.meshes), ctypes.byref(self.options), ctypes.byref(h)),
               "mf_analyze_batch")
        self._h = h
        self._load_info()
        self.npe = int(self.meshes[0].elem_nodes.shape[1])

    @classmethod
    def from_csr(cls, n: int, rowptr: np.ndarray, col: np.ndarray, options: Optional[mf_options] = None):
        """mf_analyze_csr: analysis of a general sparse matrix from its CSR pattern (host arrays).
        The numeric calls on its factors take the CSR values (device, rowptr[n] doubles)."""
        self = cls.__new__(cls)
        self.meshes = []
        self.options = options or default_options()
        rp = np.ascontiguousarray(rowptr, dtype=np.int64)
        cl = np.ascontiguousarray(col, dtype=np.int32)
        h = ctypes.c_void_p()
        _check(_lib.mf_analyze_csr(int(n), _ptr(rp), _ptr(cl), ctypes.byref(self.options), ctypes.byref(h)),
               "mf_analyze_csr")
        self._h = h
        self._load_info()
        self.npe = None  # no mesh elements: the element-gradient calls are not available
        self.nnz = int(rp[-1])
        return self

    def _load_info(self):
        i = mf_info()
        _check(_lib.mf_analysis_info(self._h, ctypes.byref(i)), "mf_analysis_info")
        self.info = {f: getattr(i, f) for f, _ in mf_info._fields_}
        self.n_dof = int(i.n_dof)
        self.n_front = int(i.n_front)
        self.n_elem = int(i.n_elem)

    def export(self) -> dict:
        n = self.n_front
        parent, cls, m, k = (np.empty(n, np.int32) for _ in range(4))
        ptr = np.empty(n + 1, np.int64)
        _check(_lib.mf_analysis_export(self._h, _ptr(parent), _ptr(cls), _ptr(m), _ptr(k), _ptr(ptr), None),
               "mf_analysis_export")
        dofs = np.empty(int(ptr[-1]), np.int32)
        _check(_lib.mf_analysis_export(self._h, None, None, None, None, None, _ptr(dofs)), "mf_analysis_export")
        return {"parent": parent, "cls": cls, "m": m, "k": k, "dof_ptr": ptr, "dofs": dofs}

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _lib.mf_free_analysis(h)
            self._h = None


class Factors:
    """Device factor storage for one analysis (mf_factors_create) and the numeric calls on it."""

    def __init__(self, analysis: Analysis, options: Optional[mf_options] = None):
        self.analysis = analysis
        self.options = options or analysis.options
        h = ctypes.c_void_p()
        _check(_lib.mf_factors_create(analysis._h, ctypes.byref(self.options), ctypes.byref(h)), "mf_factors_create")
        self._h = h
        self.n_dof = analysis.n_dof

    @property
    def precision(self) -> str:
        """Front arithmetic of these factors: "f64", "f32" or "tf32"."""
        return {v: k for k, v in PRECISIONS.items()}[self.options.precision]

    def factor(self, values, stream=None):
        _check(_lib.mf_factor(self._h, _dptr(values), _stream(stream)), "mf_factor")

    def solve(self, rhs, stream=None, adjoint: bool = False):
        """In place: rhs (n_dof,) or (nrhs, n_dof) float64 CUDA tensor -> solution."""
        nrhs = 1 if rhs.dim() == 1 else int(rhs.shape[0])
        assert rhs.numel() == nrhs * self.n_dof
        f = _lib.mf_solve_adjoint if adjoint else _lib.mf_solve
        _check(f(self._h, _dptr(rhs), nrhs, _stream(stream)), "mf_solve_adjoint" if adjoint else "mf_solve")
        return rhs

    def refine_solve(self, values, b, x, tol: float = 1e-14, maxit: int = 10, stream=None, check: bool = True,
                     adjoint: bool = False):
        nrhs = 1 if b.dim() == 1 else int(b.shape[0])
        info = mf_refine_info()
        fn = _lib.mf_refine_solve_adjoint if adjoint else _lib.mf_refine_solve
        rc = fn(self._h, _dptr(values), _dptr(b), _dptr(x), nrhs, float(tol), int(maxit), ctypes.byref(info),
                _stream(stream))
        if check and rc not in (MF_OK, MF_ENOCONV):
            _check(rc, "mf_refine_solve_adjoint" if adjoint else "mf_refine_solve")
        return {"rc": rc, "iterations": info.iterations, "backward_error": info.backward_error,
                "rel_residual": info.rel_residual}

    def residual(self, values, x, b, r, stream=None):
        nrhs = 1 if b.dim() == 1 else int(b.shape[0])
        _check(_lib.mf_residual(self._h, _dptr(values), _dptr(x), _dptr(b), _dptr(r), nrhs, _stream(stream)),
               "mf_residual")
        return r

    def element_grad(self, dvalues, lam, x, g, stream=None):
        _check(_lib.mf_element_grad(self._h, _dptr(dvalues), _dptr(lam), _dptr(x), _dptr(g), _stream(stream)),
               "mf_element_grad")
        return g

    def element_outer(self, lam, x, gK, stream=None):
        nrhs = 1 if x.dim() == 1 else int(x.shape[0])
        _check(_lib.mf_element_outer(self._h, _dptr(lam), _dptr(x), nrhs, _dptr(gK), _stream(stream)),
               "mf_element_outer")
        return gK

    def status(self) -> dict:
        st = mf_status_info()
        rc = _lib.mf_status(self._h, ctypes.byref(st))
        out = {f: getattr(st, f) for f, _ in mf_status_info._fields_}
        out["rc"] = rc
        return out

    def profile(self, enable: bool = True):
        _check(_lib.mf_profile_enable(self._h, int(enable)), "mf_profile_enable")

    def profile_read(self) -> dict:
        """Per kernel family since the last read: ms (event-timed, only while profiling is
        enabled), kernel launches, algorithmic bytes and flops."""
        n = len(PROFILE_FAMILIES)
        ms, by, fl = np.zeros(n), np.zeros(n), np.zeros(n)
        ln = np.zeros(n, np.int64)
        _check(_lib.mf_profile_read(self._h, _ptr(ms), _ptr(ln), _ptr(by), _ptr(fl)), "mf_profile_read")
        return {fam: {"ms": float(ms[i]), "launches": int(ln[i]), "bytes": float(by[i]), "flops": float(fl[i])}
                for i, fam in enumerate(PROFILE_FAMILIES)}

    def trace(self) -> list:
        """Per-launch records of the profiled region (call before profile_read)."""
        n = ctypes.c_int(0)
        _check(_lib.mf_profile_trace(self._h, None, 0, ctypes.byref(n)), "mf_profile_trace")
        recs = (mf_trace_rec * max(n.value, 1))()
        _check(_lib.mf_profile_trace(self._h, recs, n.value, ctypes.byref(n)), "mf_profile_trace")
        return [{"family": PROFILE_FAMILIES[r.family], "kind": TRACE_KINDS.get(r.kind, str(r.kind)), "cls": r.cls,
                 "tasks": r.tasks, "ms": r.ms, "bytes": r.bytes, "flops": r.flops} for r in recs[:n.value]]

    def export_front(self, front: int):
        ex = self.analysis.export()
        m, k = int(ex["m"][front]), int(ex["k"][front])
        L = np.empty(m * k)
        U = np.empty(m * k)
        _check(_lib.mf_factors_export_front(self._h, int(front), _ptr(L), _ptr(U)), "mf_factors_export_front")
        return L.reshape(k, m).T.copy(), U.reshape(m, k).T.copy()

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            _lib.mf_free_factors(h)
            self._h = None


def autotune(analysis: Analysis, values, b, base: Optional[mf_options] = None, reps: int = 3,
             cache_path: Optional[str] = None, stream=None):
    """mf_autotune: (tuned options, info dict).  values/b are CUDA tensors (element
    matrices; one right-hand side of n_dof values, not modified)."""
    best = mf_options()
    info = mf_tune_info()
    base = base if base is not None else analysis.options
    path = cache_path.encode() if cache_path else None
    _check(_lib.mf_autotune(analysis._h, _dptr(values), _dptr(b), ctypes.byref(base), int(reps), path,
                            ctypes.byref(best), ctypes.byref(info), _stream(stream)), "mf_autotune")
    return best, {f: getattr(info, f) for f, _ in mf_tune_info._fields_}
