"""ORACLE -- test infrastructure only (plain FP64 CPU multifrontal solver).

Python face of ``orc.c`` over ctypes.  Only the tests, the smoke check and the
benchmark's CPU-baseline leg may import this package; the product library
(paper_2306_08994_b300) never does, and this package never imports it.

Functions follow the paper (arXiv 2306.08994): elimination tree from element
fronts (Sec. 2.4, Table 3), pivots = dofs whose every element lies in the
front (Table 2), pivots-first reordering (Sec. 3.2), extend-add + partial LU
with the division / multiplication / subtraction tasks (Sec. 3, Table 2),
solution by forward/backward substitution (`get_solution`, Table 2).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "orc.c")
_LIB = os.path.join(_HERE, "liborc.so")

ORC_EZERO_PIVOT = -4


def build(force: bool = False) -> str:
    """Compile orc.c with gcc (OpenMP, no FP contraction) into liborc.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-o", _LIB, _SRC, "-lm"]
        subprocess.check_call(cmd)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i32, i64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        L.orc_tree_bisection.argtypes = [P, P, P, P]
        L.orc_tree_bisection.restype = ctypes.c_int
        L.orc_tree_pairing.argtypes = [P, P, P, P]
        L.orc_tree_pairing.restype = ctypes.c_int
        L.orc_create.argtypes = [i32, i32, i32, P, i32, P, P, P]
        L.orc_create.restype = P
        L.orc_free.argtypes = [P]
        L.orc_info.argtypes = [P, P]
        L.orc_fronts.argtypes = [P, P, P, P, P, P, P]
        L.orc_factor.argtypes = [P, P, f64, ctypes.c_int, ctypes.c_int]
        L.orc_factor.restype = i64
        L.orc_get_factor.argtypes = [P, i32, P, P]
        L.orc_get_factor.restype = ctypes.c_int
        L.orc_solve.argtypes = [P, P, ctypes.c_int]
        L.orc_solve.restype = ctypes.c_int
        L.orc_solve_adjoint.argtypes = [P, P, ctypes.c_int]
        L.orc_solve_adjoint.restype = ctypes.c_int
        L.orc_residual_dd.argtypes = [i32, i32, i32, P, P, P, P, P, ctypes.c_int]
        L.orc_solve_refined.argtypes = [P, P, P, P, ctypes.c_int, ctypes.c_int]
        L.orc_solve_refined.restype = ctypes.c_int
        L.orc_element_grad.argtypes = [i32, i32, P, P, P, P, P]
        L.orc_max_threads.restype = ctypes.c_int
        L.orc_sum_m.argtypes = [P]
        L.orc_sum_m.restype = i64
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


@dataclass
class Tree:
    """Elimination tree in postorder: parent (-1 root), child (n,2; -1 none), leaf_elem (-1 internal)."""
    parent: np.ndarray
    child: np.ndarray
    leaf_elem: np.ndarray

    @property
    def n(self) -> int:
        return int(self.parent.size)


def tree_bisection(nel) -> Tree:
    """Recursive longest-axis floor bisection of the element box (ties: x, y, z)."""
    nel3 = np.array(list(nel) + [1] * (3 - len(nel)), dtype=np.int32)
    ne = int(np.prod(nel3))
    par = np.empty(2 * ne - 1, np.int32)
    ch = np.empty(2 * (2 * ne - 1), np.int32)
    le = np.empty(2 * ne - 1, np.int32)
    n = lib().orc_tree_bisection(_p(nel3), _p(par), _p(ch), _p(le))
    assert n == 2 * ne - 1
    return Tree(par, ch.reshape(-1, 2), le)


def tree_pairing(nel) -> Tree:
    """The paper's Table 3 rule: Morton-sorted element fronts joined pairwise, odd one carried up."""
    nel3 = np.array(list(nel) + [1] * (3 - len(nel)), dtype=np.int32)
    ne = int(np.prod(nel3))
    par = np.empty(2 * ne - 1, np.int32)
    ch = np.empty(2 * (2 * ne - 1), np.int32)
    le = np.empty(2 * ne - 1, np.int32)
    n = lib().orc_tree_pairing(_p(nel3), _p(par), _p(ch), _p(le))
    assert n == 2 * ne - 1
    return Tree(par, ch.reshape(-1, 2), le)


class OracleSolver:
    """Plain FP64 multifrontal solver on one mesh (symbolic at construction)."""

    def __init__(self, n_dof: int, elem_nodes: np.ndarray, tree: Tree):
        self._lib = lib()
        self.en = np.ascontiguousarray(elem_nodes, dtype=np.int64)
        self.n_dof, self.n_elem, self.npe = int(n_dof), int(self.en.shape[0]), int(self.en.shape[1])
        self.tree = tree
        self._h = self._lib.orc_create(self.n_dof, self.n_elem, self.npe, _p(self.en), tree.n,
                                       _p(np.ascontiguousarray(tree.parent, np.int32)),
                                       _p(np.ascontiguousarray(tree.child, np.int32)),
                                       _p(np.ascontiguousarray(tree.leaf_elem, np.int32)))
        info = np.zeros(8, np.int64)
        self._lib.orc_info(self._h, _p(info))
        (self.n_front, self.n_classes, self.max_m, self.sum_k, self.nnz_lu, self.sum_cb,
         self.flops, self.max_k) = [int(v) for v in info]
        self.m = np.empty(self.n_front, np.int32)
        self.k = np.empty(self.n_front, np.int32)
        self.height = np.empty(self.n_front, np.int32)
        self.parent = np.empty(self.n_front, np.int32)
        self.dof_ptr = np.empty(self.n_front + 1, np.int64)
        self.dofs = np.empty(int(self._lib.orc_sum_m(self._h)), np.int32)
        self._lib.orc_fronts(self._h, _p(self.m), _p(self.k), _p(self.height), _p(self.parent),
                             _p(self.dof_ptr), _p(self.dofs))

    def front_dofs(self, v: int) -> np.ndarray:
        return self.dofs[self.dof_ptr[v]: self.dof_ptr[v + 1]]

    def factor(self, Ke_colmajor: np.ndarray, tau: float = 0.0, fail_small: bool = False, nthreads: int = 1) -> int:
        """Numeric factorization; returns #perturbed pivots (or ORC_EZERO_PIVOT)."""
        self._Ke = np.ascontiguousarray(Ke_colmajor, dtype=np.float64)
        assert self._Ke.size == self.n_elem * self.npe * self.npe
        return int(self._lib.orc_factor(self._h, _p(self._Ke), float(tau), int(fail_small), int(nthreads)))

    def factor_of(self, v: int):
        """(L, U) of front v: L is m x k (pivot columns), U is k x m (pivot rows)."""
        m, k = int(self.m[v]), int(self.k[v])
        Lb = np.empty(m * k)
        Ub = np.empty(m * k)
        rc = self._lib.orc_get_factor(self._h, int(v), _p(Lb), _p(Ub))
        assert rc == 0
        return Lb.reshape(k, m).T.copy(), Ub.reshape(m, k).T.copy()

    def solve(self, b: np.ndarray, adjoint: bool = False) -> np.ndarray:
        x = np.asfortranarray(np.array(b, dtype=np.float64, copy=True).reshape(self.n_dof, -1))
        f = self._lib.orc_solve_adjoint if adjoint else self._lib.orc_solve
        rc = f(self._h, _p(x), int(x.shape[1]))
        assert rc == 0
        return x.reshape(np.shape(b))

    def solve_refined(self, b: np.ndarray, maxit: int = 10):
        """Solve, then refine with a double-double residual; returns (x, steps)."""
        bb = np.asfortranarray(np.array(b, dtype=np.float64).reshape(self.n_dof, -1))
        x = np.empty_like(bb, order="F")
        it = self._lib.orc_solve_refined(self._h, _p(self._Ke), _p(bb), _p(x), int(bb.shape[1]), int(maxit))
        return x.reshape(np.shape(b)), int(it)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_free(h)
            self._h = None


def residual_dd(elem_nodes, Ke_colmajor, x, b) -> np.ndarray:
    """r = b - A x with double-double accumulation (A given element by element)."""
    en = np.ascontiguousarray(elem_nodes, dtype=np.int64)
    n = int(np.shape(b)[0])
    xx = np.asfortranarray(np.asarray(x, np.float64).reshape(n, -1))
    bb = np.asfortranarray(np.asarray(b, np.float64).reshape(n, -1))
    r = np.empty_like(bb, order="F")
    K = np.ascontiguousarray(Ke_colmajor, np.float64)
    lib().orc_residual_dd(n, en.shape[0], en.shape[1], _p(en), _p(K), _p(xx), _p(bb), _p(r), int(bb.shape[1]))
    return r.reshape(np.shape(b))


def element_grad(elem_nodes, dK_colmajor, lam, x) -> np.ndarray:
    """g_e = -lambda_e^T dK_e x_e."""
    en = np.ascontiguousarray(elem_nodes, dtype=np.int64)
    g = np.empty(en.shape[0])
    K = np.ascontiguousarray(dK_colmajor, np.float64)
    lib().orc_element_grad(en.shape[0], en.shape[1], _p(en), _p(K), _p(np.ascontiguousarray(lam, np.float64)),
                           _p(np.ascontiguousarray(x, np.float64)), _p(g))
    return g


def max_threads() -> int:
    return int(lib().orc_max_threads())
