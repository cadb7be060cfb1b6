"""mf_analyze_csr on the GPU: factor + (refined) solve of matrices given only by CSR, through the C
ABI, against LAPACK's dense solve.

Cases: FEM matrices whose dofs were renumbered by a random permutation (so nothing of the mesh
survives), a random sparse SPD matrix that comes from no mesh, and an unsymmetric convection
matrix for the adjoint solve.  Tolerances as for the mesh path: normwise backward error <= 1e-12
for refined solves, solution within 1e-10 of LAPACK's (relative 2-norm) after refinement to the
FP64 floor.
"""
import numpy as np
import pytest
import torch

import fem_inputs as F
import paper_2306_08994_b300 as M
from test_csr import _permuted_csr, _random_spd

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _factors(A, prec, **opt):
    an = M.Analysis.from_csr(A.shape[0], A.indptr, A.indices, M.default_options(precision=prec, **opt))
    f = M.Factors(an)
    vals = torch.tensor(A.data, device=DEV)
    return an, f, vals


def _eta(A, x, b):
    r = b - A @ x
    return np.abs(r).max() / (abs(A).sum(axis=1).max() * np.abs(x).max() + np.abs(b).max())


CASES = {
    "q3_16_hetero_permuted": lambda: _permuted_csr(F.diffusion_2d(16, 3, seed=51), 7)[0],
    "q1_40_permuted": lambda: _permuted_csr(F.poisson_2d_q1(40), 8)[0],
    "q1_3d_10_permuted": lambda: _permuted_csr(F.diffusion_3d_q1(10, seed=52), 9)[0],
    "l2_q3_10_permuted": lambda: _permuted_csr(F.l2_projection(10, 3), 10)[0],
    "random_spd_3000": lambda: _random_spd(3000, seed=53),
}


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec,opt", [("f64", {}), ("f32", {}), ("tf32", {"tc_min_cb": 16, "small_front_max": 32})])
def test_csr_solution_matches_lapack(case, prec, opt):
    A = CASES[case]()
    n = A.shape[0]
    rng = np.random.default_rng(3)
    b = rng.uniform(-1, 1, n)
    x_ref = np.linalg.solve(A.toarray(), b)
    an, f, vals = _factors(A, prec, **opt)
    f.factor(vals)
    assert f.status()["rc"] == 0
    bt = torch.tensor(b, device=DEV)
    if prec == "f64":
        x = bt.clone()
        f.solve(x)
        assert _eta(A, x.cpu().numpy(), b) <= 1e-14
    x = torch.empty_like(bt)
    info = f.refine_solve(vals, bt, x, tol=1e-15, maxit=30)
    xg = x.cpu().numpy()
    assert info["backward_error"] <= 1e-12 and _eta(A, xg, b) <= 1e-12, info
    err = np.linalg.norm(xg - x_ref) / np.linalg.norm(x_ref)
    assert err <= 1e-10, (case, prec, err, info)
    # residual through the CSR values
    r = torch.empty_like(bt)
    f.residual(vals, x, bt, r)
    r_ref = b - A @ xg
    assert np.abs(r.cpu().numpy() - r_ref).max() <= 1e-13 * (abs(A).sum(axis=1).max() * np.abs(xg).max())


def test_csr_adjoint_solve_of_an_unsymmetric_matrix():
    import scipy.sparse as sp
    pr = F.convection_2d_q1(8)
    A, _ = _permuted_csr(pr, 12)
    n = A.shape[0]
    b = np.random.default_rng(4).uniform(-1, 1, n)
    an, f, vals = _factors(A, "f64")
    f.factor(vals)
    bt = torch.tensor(b, device=DEV)
    x = bt.clone()
    f.solve(x, adjoint=True)
    xr = np.linalg.solve(A.toarray().T, b)
    assert np.linalg.norm(x.cpu().numpy() - xr) <= 1e-12 * np.linalg.norm(xr)
    x = torch.empty_like(bt)
    info = f.refine_solve(vals, bt, x, tol=1e-15, maxit=20, adjoint=True)
    assert info["backward_error"] <= 1e-14
    assert np.linalg.norm(x.cpu().numpy() - xr) <= 1e-12 * np.linalg.norm(xr)


def test_csr_element_gradients_are_not_supported():
    A = CASES["q1_40_permuted"]()
    an, f, vals = _factors(A, "f64")
    v = torch.zeros(A.shape[0], dtype=torch.float64, device=DEV)
    from paper_2306_08994_b300 import mfsolve as B
    with pytest.raises(B.MFError):
        f.element_grad(vals, v, v, v)
