"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (derived from the arithmetic):
  * FP64 factors: |L - L_oracle| <= 1e-11 * max|front| per front (two FP64
    eliminations of the same front differing only in summation order);
  * solutions: ||x - x_oracle||_2 / ||x_oracle||_2 <= 1e-10 (the stated bar),
    x_oracle refined with a double-double residual;
  * refined paths (FP64 and FP32 fronts): normwise backward error
    ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf) <= 1e-12.
Refinement in these tests stops at a backward error of 1e-15: the forward
error of a refined solution is about cond * eta, and with cond near 1e4 on the
larger heterogeneous cases a stop at 1e-14 can leave it just above the 1e-10
solution bar although the next correction would bring it to ~1e-13.
"""
import numpy as np
import pytest
import torch

import fem_inputs as F
import oracle as O
import paper_2306_08994_b300 as M

pytestmark = pytest.mark.gpu

DEV = "cuda"


def _setup(pr, prec="f64", **opt):
    pm = pr.mesh
    a = M.Analysis(M.Mesh(pm.elem_nodes, pm.n_nodes, pm.dim, grid_dims=pm.nel),
                   M.default_options(precision=prec, **opt))
    f = M.Factors(a)
    vals = torch.tensor(F.to_colmajor(pr.Ke), device=DEV)
    return a, f, vals


def _oracle(pr):
    pm = pr.mesh
    s = O.OracleSolver(pm.n_nodes, pm.elem_nodes, O.tree_bisection(pm.nel))
    assert s.factor(F.to_colmajor(pr.Ke)) == 0
    return s


def _backward_error_host(pr, x, b):
    """eta = ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf) with the oracle's
    double-double residual and the assembled ||A||_inf (host, independent of the GPU)."""
    import scipy.sparse as sp
    r = O.residual_dd(pr.mesh.elem_nodes, F.to_colmajor(pr.Ke), x, b)
    rp, cp, vp = F.assemble_csr(pr.mesh, pr.Ke)
    A = sp.csr_matrix((vp, cp, rp))
    an = np.abs(A).sum(axis=1).max()
    x2 = np.asarray(x).reshape(pr.mesh.n_nodes, -1)
    b2 = np.asarray(b).reshape(pr.mesh.n_nodes, -1)
    r2 = np.asarray(r).reshape(pr.mesh.n_nodes, -1)
    out = 0.0
    for j in range(x2.shape[1]):
        num = np.abs(r2[:, j]).max()
        den = an * np.abs(x2[:, j]).max() + np.abs(b2[:, j]).max()
        out = max(out, num / den if den > 0 else (0.0 if num == 0 else np.inf))
    return out


CASES = {
    "q1_16": (lambda: F.poisson_2d_q1(16), {}),
    "q3_12_large_path": (lambda: F.diffusion_2d(12, 3, seed=31), {"small_front_max": 16}),
    "q3_10_mixed_buckets": (lambda: F.diffusion_2d(10, 3, seed=32), {"small_front_max": 48}),
    "q1_3d_6_large_path": (lambda: F.diffusion_3d_q1(6, seed=33), {"small_front_max": 24}),
    "q1_1x1": (lambda: F.poisson_2d_q1(1), {}),
    "q3_12_no_subtree": (lambda: F.diffusion_2d(12, 3, seed=34), {"subtree_levels": -1, "small_front_max": 32}),
    "q1_9_subtree3_unbalanced": (lambda: F.poisson_2d_q1(9), {"subtree_levels": 3}),
    "q1_3d_5_subtree": (lambda: F.diffusion_3d_q1(5, seed=35), {"subtree_levels": 4, "small_front_max": 24}),
    "q3_12_solve_subtree_only": (lambda: F.diffusion_2d(12, 3, seed=37), {"subtree_solve_levels": 5}),
    "q1_20_solve_subtree8": (lambda: F.poisson_2d_q1(20), {"subtree_solve_levels": 8, "small_front_max": 32}),
    # large-front partial LU with one-panel lookahead (default when the super-panel is one panel:
    # FP64 always, FP32 with super_panel = 64); the root (73 pivots) spans 3 FP64 / 2 FP32 panels
    "q3_24_lookahead": (lambda: F.diffusion_2d(24, 3, seed=38), {"small_front_max": 16, "super_panel": 64}),
    "q3_24_no_lookahead": (lambda: F.diffusion_2d(24, 3, seed=38), {"small_front_max": 16, "super_panel": 64,
                                                                    "lookahead": -1}),
    # the paper's own model problem: L2-projection mass matrices (no boundary condition), p = 1, 2, 3
    "l2_q1_32": (lambda: F.l2_projection(32, 1), {}),
    "l2_q2_16_large_path": (lambda: F.l2_projection(16, 2), {"small_front_max": 16}),
    "l2_q3_12": (lambda: F.l2_projection(12, 3), {"small_front_max": 48}),
}


@pytest.mark.parametrize("case", list(CASES))
def test_f64_factors_match_oracle_front_by_front(case):
    mk, opt = CASES[case]
    pr = mk()
    a, f, vals = _setup(pr, "f64", **opt)
    f.factor(vals)
    st = f.status()
    assert st["rc"] == 0 and st["n_perturbed"] == 0
    _check_factors(f, _oracle(pr), case)


def _check_factors(f, s, tag, stride=1):
    """Front by front: the library numbers fronts class by class (stable in the
    oracle's postorder), so sorting the oracle's fronts by height pairs them up."""
    order = np.lexsort((np.arange(s.n_front), s.height))
    for g in range(0, len(order), stride):
        Lg, Ug = f.export_front(g)
        Lo, Uo = s.factor_of(order[g])
        k = Lo.shape[1]
        if k == 0:
            continue
        sc = max(np.abs(Lo).max(), np.abs(Uo).max(), 1.0)
        low = np.tril(np.ones((Lo.shape[0], k), bool))
        up = np.triu(np.ones((k, Uo.shape[1]), bool), 1)
        assert np.abs(Lg - Lo)[low].max() <= 1e-11 * sc, (tag, g)
        if up.any():
            assert np.abs(Ug - Uo)[up].max() <= 1e-11 * sc, (tag, g)


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_solution_matches_oracle(case, prec):
    mk, opt = CASES[case]
    pr = mk()
    a, f, vals = _setup(pr, prec, **opt)
    f.factor(vals)
    s = _oracle(pr)
    b = np.ascontiguousarray(pr.b.T)  # (nrhs, n)
    xo, _ = s.solve_refined(pr.b)
    bt = torch.tensor(b, device=DEV)
    x = torch.empty_like(bt)
    info = f.refine_solve(vals, bt, x, tol=1e-15, maxit=30)
    xg = x.cpu().numpy().T
    assert info["backward_error"] <= 1e-12, info
    assert _backward_error_host(pr, xg, pr.b) <= 1e-12
    err = np.linalg.norm(xg - xo) / np.linalg.norm(xo)
    assert err <= 1e-10, (case, prec, err, info)
    if prec == "f64":
        # the plain FP64 solve (no refinement) also meets the solution bar
        x1 = bt.clone()
        f.solve(x1)
        e1 = np.linalg.norm(x1.cpu().numpy().T - xo) / np.linalg.norm(xo)
        assert e1 <= 1e-10, e1


@pytest.mark.parametrize("n", [40, 56, 96])
def test_tensor_core_schur_path(n):
    """MF_TF32: Schur updates of large fronts on tcgen05 (3-pass TF32).  Factors agree
    with the FP32 SIMT path to within the FP32 path's own distance from FP64, and the
    refined solution meets the same bars.  tc_min_cb = 32 sends contribution blocks
    from 32 up (partial 128 x 256 tiles, several tiles per front at n = 96) through
    the tensor-core kernels."""
    pr = F.diffusion_2d(n, 3, seed=36)
    factors = {}
    for prec in ("f64", "f32", "tf32"):
        a, f, vals = _setup(pr, prec, small_front_max=64, tc_min_cb=32)
        if prec == "tf32":
            f.profile(True)
        f.factor(vals)
        if prec == "tf32":
            kinds = {r["kind"] for r in f.trace()}
            f.profile_read()
            f.profile(False)
            assert kinds & {"gemm_tc", "gemm_tcd"}, kinds
        assert f.status()["rc"] == 0
        g = a.n_front - 2  # a front just below the root: its front matrix came through Schur updates
        factors[prec] = f.export_front(g)[0]
        if prec == "tf32":
            s = _oracle(pr)
            xo, _ = s.solve_refined(pr.b)
            bt = torch.tensor(np.ascontiguousarray(pr.b.T), device=DEV)
            x = torch.empty_like(bt)
            info = f.refine_solve(vals, bt, x, tol=1e-15, maxit=40)
            xg = x.cpu().numpy().T
            assert info["backward_error"] <= 1e-12, info
            assert np.linalg.norm(xg - xo) / np.linalg.norm(xo) <= 1e-10
    d32 = np.abs(factors["f32"] - factors["f64"]).max()
    dtc = np.abs(factors["tf32"] - factors["f64"]).max()
    assert dtc <= 10 * d32 + 1e-12, (dtc, d32)


@pytest.mark.parametrize("prec,panels", [("f64", 1), ("f32", 1), ("f64", 3), ("f32", 3)])
def test_lookahead_factors_match_plain_panel_order(prec, panels):
    """One-panel lookahead (the next pivot block takes its pending update inside the
    pivot-block kernel, on a second stream, while the trailing update or the Crout strips
    run) against the plain panel order: the same factors up to rounding, front by front,
    on the top fronts of a 48 x 48 Q3 mesh (root: 145 pivots, 3 FP32 / 5 FP64 panels).
    Super-panels of 1 panel (the update is one panel deep) and of 3 panels (up to 3 panels
    deep, staged in several slices)."""
    pr = F.diffusion_2d(48, 3, seed=39)
    nb = 64 if prec == "f32" else 32
    out = {}
    for la in (0, -1):
        a, f, vals = _setup(pr, prec, small_front_max=16, super_panel=panels * nb, lookahead=la)
        f.factor(vals)
        assert f.status()["rc"] == 0
        out[la] = [f.export_front(g) for g in range(a.n_front - 7, a.n_front)]
    tol = 1e-12 if prec == "f64" else 2e-4
    for (L0, U0), (L1, U1) in zip(out[0], out[-1]):
        sc = max(np.abs(L1).max(), np.abs(U1).max(), 1.0)
        assert np.abs(L0 - L1).max() <= tol * sc
        assert np.abs(U0 - U1).max() <= tol * sc


def test_adjoint_solve_on_unsymmetric_matrix():
    pr = F.convection_2d_q1(9)
    a, f, vals = _setup(pr, "f64", small_front_max=8)
    f.factor(vals)
    s = _oracle(pr)
    g = np.ascontiguousarray(pr.b[:, 0])
    lo = s.solve(g, adjoint=True)
    xo = s.solve(g)
    t = torch.tensor(g, device=DEV)
    lam = t.clone()
    f.solve(lam, adjoint=True)
    x = t.clone()
    f.solve(x)
    assert np.linalg.norm(lam.cpu().numpy() - lo) <= 1e-12 * np.linalg.norm(lo)
    assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-12 * np.linalg.norm(xo)
    assert np.linalg.norm(lo - xo) > 1e-3 * np.linalg.norm(xo)  # really unsymmetric


@pytest.mark.parametrize("prec", ["f32", "tf32"])
def test_adjoint_refinement_unsymmetric(prec):
    """mf_refine_solve_adjoint: FP32-family factors of an unsymmetric (convection) matrix and
    the adjoint system A^T x = g refined in FP64 (residual with the transposed element
    matrices): the oracle's adjoint solution to 1e-10, and the backward error of A^T
    recomputed on the host from the assembled matrix <= 1e-12."""
    import scipy.sparse as sp
    pr = F.convection_2d_q1(9)
    a, f, vals = _setup(pr, prec, small_front_max=8)
    f.factor(vals)
    s = _oracle(pr)
    g = np.ascontiguousarray(pr.b[:, 0])
    lo = s.solve(g, adjoint=True)
    gt = torch.tensor(g, device=DEV)
    lam = torch.empty_like(gt)
    info = f.refine_solve(vals, gt, lam, tol=1e-15, maxit=40, adjoint=True)
    assert info["backward_error"] <= 1e-12, info
    lh = lam.cpu().numpy()
    assert np.linalg.norm(lh - lo) <= 1e-10 * np.linalg.norm(lo)
    rp, cp, vp = F.assemble_csr(pr.mesh, pr.Ke)
    A = sp.csr_matrix((vp, cp, rp))
    r = g - A.T @ lh
    eta = np.abs(r).max() / (abs(A.T).sum(axis=1).max() * np.abs(lh).max() + np.abs(g).max())
    assert eta <= 1e-12, eta
    # the forward refinement on the same factors solves the other system
    x = torch.empty_like(gt)
    f.refine_solve(vals, gt, x, tol=1e-15, maxit=40)
    assert np.linalg.norm(x.cpu().numpy() - lh) > 1e-3 * np.linalg.norm(lh)


def test_element_gradient_matches_oracle_and_autograd():
    pr = F.adjoint_problem(n=24, n_fd=8)
    a, f, vals = _setup(pr, "f64")
    ut = pr.extra["u_target"]
    b = torch.tensor(pr.b[:, 0], device=DEV)
    K = vals.clone().requires_grad_(True)
    x = M.MFSolve.apply(K, b, f, 0.0)
    J = 0.5 * torch.sum((x - torch.tensor(ut, device=DEV)) ** 2)
    J.backward()
    s = _oracle(pr)
    xo = s.solve(pr.b[:, 0])
    lo = s.solve(xo - ut, adjoint=True)
    go = O.element_grad(pr.mesh.elem_nodes, F.to_colmajor(pr.extra["dK"]), lo, xo)
    # dJ/dK_e = -lambda_e x_e^T ; chain to theta through dK_e/dtheta_e
    gK = K.grad.cpu().numpy().reshape(pr.mesh.n_elem, -1)
    g_chain = (gK * F.to_colmajor(pr.extra["dK"]).reshape(pr.mesh.n_elem, -1)).sum(axis=1)
    assert np.abs(g_chain - go).max() <= 1e-10 * np.abs(go).max()
    lam = torch.tensor(lo, device=DEV)
    g = torch.empty(pr.mesh.n_elem, dtype=torch.float64, device=DEV)
    f.element_grad(torch.tensor(F.to_colmajor(pr.extra["dK"]), device=DEV), lam,
                   torch.tensor(xo, device=DEV), g)
    assert np.abs(g.cpu().numpy() - go).max() <= 1e-12 * np.abs(go).max()


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_static_pivot_check_on_singular_matrix(prec):
    pm = F.structured_mesh((4, 4), 1)
    Ke = F.element_matrices(pm, dirichlet=False)  # pure Neumann: singular
    pr = F.Problem("neumann", pm, Ke, np.zeros((pm.n_nodes, 1)))
    a, f, vals = _setup(pr, prec, pivot_tol=1e-6)
    f.factor(vals)
    st = f.status()
    assert st["rc"] == 0 and st["n_perturbed"] >= 1 and st["first_front"] == a.n_front - 1
    a2, f2, vals2 = _setup(pr, prec, pivot_tol=1e-6, pivot_fail=1)
    f2.factor(vals2)
    assert f2.status()["rc"] == M.mfsolve.MF_EZERO_PIVOT


def test_batched_meshes_with_four_rhs():
    sizes = [5, 9, 4, 12]
    probs = F.batched_poisson(sizes, nrhs=4, seed=77)
    meshes = [M.Mesh(p.mesh.elem_nodes, p.mesh.n_nodes, 2, grid_dims=p.mesh.nel) for p in probs]
    for prec in ("f64", "f32"):
        a = M.Analysis(meshes, M.default_options(precision=prec, small_front_max=24))
        f = M.Factors(a)
        vals = torch.tensor(np.concatenate([F.to_colmajor(p.Ke) for p in probs]), device=DEV)
        f.factor(vals)
        b = np.concatenate([p.b for p in probs], axis=0)  # (N, 4)
        bt = torch.tensor(np.ascontiguousarray(b.T), device=DEV)
        x = torch.empty_like(bt)
        info = f.refine_solve(vals, bt, x, tol=1e-15, maxit=30)
        assert info["backward_error"] <= 1e-12
        xg = x.cpu().numpy().T
        off = 0
        for p in probs:
            xo, _ = _oracle(p).solve_refined(p.b)
            n = p.mesh.n_nodes
            assert np.linalg.norm(xg[off:off + n] - xo) <= 1e-10 * np.linalg.norm(xo)
            off += n


@pytest.mark.parametrize("sym", [0, 1])
@pytest.mark.parametrize("case", ["q3_24", "q1_3d_8"])
def test_one_and_four_rhs_substitutions_agree(case, sym):
    """One FP32 factorization, then unrefined solves with one right-hand side (lane groups of
    4-16 lanes with up to 4 rows per lane, row loads batched in the CTA kernels) and with four
    (one row per lane, per-coefficient loops): the scaled copies of b give the scaled solution up
    to FP32 rounding, and the single solve has an FP32-level backward error (host double-double
    residual, Sec. 2.1 eq. Linear_system)."""
    pr = {"q3_24": lambda: F.diffusion_2d(24, 3, seed=91), "q1_3d_8": lambda: F.diffusion_3d_q1(8, seed=92)}[case]()
    a, f, vals = _setup(pr, "f32", symmetric=sym)
    f.factor(vals)
    b = pr.b[:, 0]
    y1 = torch.tensor(b, device=DEV)
    f.solve(y1)
    scales = [1.0, 2.0, -1.0, 0.5]
    y4 = torch.tensor(np.stack([s_ * b for s_ in scales]), device=DEV)
    f.solve(y4)
    y1 = y1.cpu().numpy()
    y4 = y4.cpu().numpy()
    top = np.abs(y1).max()
    for c, s_ in enumerate(scales):
        assert np.abs(y4[c] / s_ - y1).max() <= 1e-4 * top, (c, np.abs(y4[c] / s_ - y1).max() / top)
    assert _backward_error_host(pr, y1, b) <= 1e-5


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_graph_replay_equals_direct_launches(prec):
    """use_graph: factor, solve and refinement replayed from captured CUDA graphs on a
    user stream give bitwise the same results as direct launches."""
    pr = F.diffusion_2d(20, 3, seed=42)
    outs = []
    for graph in (0, 1):
        a, f, vals = _setup(pr, prec, use_graph=graph, small_front_max=32)
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            b = torch.tensor(pr.b[:, 0], device=DEV)
            res = []
            for rep in range(3):  # capture, then replays
                f.factor(vals, stream=stream)
                x = torch.empty_like(b)
                info = f.refine_solve(vals, b, x, tol=1e-15, maxit=30, stream=stream)
                y = b.clone()
                f.solve(y, stream=stream)
                stream.synchronize()
                res.append((x.cpu().numpy(), y.cpu().numpy(), info["iterations"]))
        for r in res[1:]:
            assert np.array_equal(r[0], res[0][0]) and np.array_equal(r[1], res[0][1])
        outs.append(res[0])
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])
    assert outs[0][2] == outs[1][2]


def test_repeat_factor_is_bitwise_deterministic():
    pr = F.diffusion_2d(16, 3, seed=41)
    a, f, vals = _setup(pr, "f32", small_front_max=64)
    b = torch.tensor(pr.b[:, 0], device=DEV)
    outs = []
    for _ in range(2):
        f.factor(vals)
        x = b.clone()
        f.solve(x)
        outs.append(x.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("threads", [32, 64, 128, 256])
def test_fused_threads_per_bucket_keep_parity(threads):
    """Every thread count the autotuner may pick for a fused size bucket gives FP64
    factors equal to the oracle's (front by front) and the same refined solution."""
    pr = F.diffusion_2d(14, 3, seed=43)
    a, f, vals = _setup(pr, "f64", small_front_max=160, fused_threads=[threads] * M.mfsolve.MF_FUSED_BUCKETS)
    f.factor(vals)
    assert f.status()["rc"] == 0
    s = _oracle(pr)
    _check_factors(f, s, threads, stride=3)
    b = torch.tensor(pr.b[:, 0], device=DEV)
    x = torch.empty_like(b)
    info = f.refine_solve(vals, b, x, tol=1e-15, maxit=30)
    xo, _ = s.solve_refined(pr.b)
    assert info["backward_error"] <= 1e-12
    assert np.linalg.norm(x.cpu().numpy() - xo[:, 0]) <= 1e-10 * np.linalg.norm(xo[:, 0])


def test_autotune_returns_a_correct_plan_and_caches_it(tmp_path):
    pr = F.diffusion_2d(24, 3, seed=44)
    pm = pr.mesh
    a = M.Analysis(M.Mesh(pm.elem_nodes, pm.n_nodes, pm.dim, grid_dims=pm.nel), M.default_options(precision="f32"))
    vals = torch.tensor(F.to_colmajor(pr.Ke), device=DEV)
    b = torch.tensor(pr.b[:, 0], device=DEV)
    b0 = b.clone()
    cache = str(tmp_path / "plans.jsonl")
    best, info = M.mfsolve.autotune(a, vals, b, reps=2, cache_path=cache)
    assert torch.equal(b, b0)
    assert info["from_cache"] == 0 and info["candidates"] >= 8
    assert 0 < info["ms_best"] <= info["ms_default"]
    assert best.precision in (M.mfsolve.MF_F32, M.mfsolve.MF_TF32)
    assert all(t in (0, 32, 64, 128, 256) for t in best.fused_threads)
    best2, info2 = M.mfsolve.autotune(a, vals, b, reps=2, cache_path=cache)
    assert info2["from_cache"] == 1 and best2.as_dict() == best.as_dict()
    with open(cache) as fh:
        assert len(fh.read().strip().splitlines()) == 1
    f = M.Factors(a, best)
    f.factor(vals)
    x = torch.empty_like(b)
    info3 = f.refine_solve(vals, b, x, tol=1e-15, maxit=30)
    xo, _ = _oracle(pr).solve_refined(pr.b)
    assert info3["backward_error"] <= 1e-12
    assert np.linalg.norm(x.cpu().numpy() - xo[:, 0]) <= 1e-10 * np.linalg.norm(xo[:, 0])


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_persistent_sweep_matches_per_class_launches(prec):
    """sweep_kernel (one cooperative launch per substitution sweep, grid barriers between
    classes) gives the per-class path's solution, forward and transposed, 1 and 4 RHS."""
    pr = F.diffusion_2d(40, 3, seed=45)
    outs = {}
    for sw in (0, 100):  # per-class launches; every class above the subtrees in the sweep
        a, f, vals = _setup(pr, prec, sweep_kernel=sw, small_front_max=48)
        f.factor(vals)
        b4 = torch.tensor(np.random.default_rng(7).uniform(-1, 1, (4, pr.mesh.n_nodes)), device=DEV)
        res = []
        for adj in (False, True):
            y = b4.clone()
            f.solve(y, adjoint=adj)
            y1 = b4[0].clone()
            f.solve(y1, adjoint=adj)
            res.append((y.cpu().numpy(), y1.cpu().numpy()))
        outs[sw] = res
    # the 1-RHS kernels divide by the pivot, the 4-RHS ones multiply by its reciprocal: the two
    # agree to rounding (FP32 fronts: a few units of 1e-7 after amplification by the condition);
    # the per-class path's small fronts (pivot-bounded lane groups, backward by group sums) and the
    # sweep's bodies also order their sums differently, which shows at the same FP32 level
    tol_rhs = 1e-9 if prec == "f64" else 1e-5
    for (ya, y1a), (yb, y1b) in zip(outs[0], outs[100]):
        assert np.linalg.norm(ya - yb) <= tol_rhs * np.linalg.norm(ya)
        assert np.linalg.norm(y1a - y1b) <= tol_rhs * np.linalg.norm(y1a)
        assert np.linalg.norm(y1b - yb[0]) <= tol_rhs * np.linalg.norm(y1b)


FP32_CASES = {
    "q1_32": (lambda: F.poisson_2d_q1(32), {"small_front_max": 32}),
    "q3_16_hetero": (lambda: F.diffusion_2d(16, 3, seed=41), {"small_front_max": 48}),
    "q3_24_large_path": (lambda: F.diffusion_2d(24, 3, seed=42), {"small_front_max": 16, "super_panel": 64}),
    "q1_3d_8": (lambda: F.diffusion_3d_q1(8, seed=43), {"small_front_max": 24}),
    # larger fronts: contribution blocks of up to 361 rows, pivot blocks of up to 289
    "q3_96_large_fronts": (lambda: F.diffusion_2d(96, 3, seed=44), {"small_front_max": 16, "super_panel": 64}),
}


@pytest.mark.parametrize("case", list(FP32_CASES))
@pytest.mark.parametrize("prec", ["f32", "tf32"])
def test_fp32_family_factors_match_oracle_front_by_front(case, prec):
    """FP32 and split-TF32 fronts against the oracle's FP64 factors, front by front.

    Tolerance from the arithmetic: an entry of front f is the result of at most K_f updates,
    K_f = the pivots eliminated in f's subtree (every pivot below f can reach it once through the
    extend-add chain, and f's own pivots once each); each update adds a product of entries no
    larger than the front's scale and is rounded once in FP32 (unit roundoff u = 2^-24) or, with
    three split-TF32 products, carries a product error of about 2^-21 (the dropped lo x lo term
    and the TF32 truncation of the lo parts).  So |L - L_oracle| <= 4 K_f u_eff max|front| with
    u_eff = 2^-24 (f32) or 2^-21 (tf32), the factor 4 covering the division by the pivot and the
    rounding of the assembled inputs."""
    mk, opt = FP32_CASES[case]
    pr = mk()
    if prec == "tf32":
        opt = dict(opt, tc_min_cb=16)
    a, f, vals = _setup(pr, prec, **opt)
    f.factor(vals)
    st = f.status()
    assert st["rc"] == 0 and st["n_perturbed"] == 0
    _check_fp32_family_factors(f, _oracle(pr), prec, case)


@pytest.mark.parametrize("case", ["q3_96_large_fronts", "q3_24_large_path"])
def test_symmetric_mode_fp32_factors_match_oracle_front_by_front(case):
    """Option symmetric with FP32 fronts and SIMT products (the Schur updates only on and below
    the diagonal, then mirrored): the exported L and U against the
    oracle's FP64 LU factors front by front, within the FP32 bound of the general test above."""
    mk, opt = FP32_CASES[case]
    pr = mk()
    a, f, vals = _setup(pr, "f32", symmetric=1, **opt)
    f.factor(vals)
    st = f.status()
    assert st["rc"] == 0 and st["n_perturbed"] == 0
    _check_fp32_family_factors(f, _oracle(pr), "f32", case)


def _check_fp32_family_factors(f, s, prec, case):
    ksub = np.asarray(s.k, dtype=np.int64).copy()
    for v in range(s.n_front):  # postorder: children before parents
        if s.parent[v] >= 0:
            ksub[s.parent[v]] += ksub[v]
    u_eff = 2.0 ** -24 if prec == "f32" else 2.0 ** -21
    order = np.lexsort((np.arange(s.n_front), s.height))
    worst = 0.0
    for g in range(len(order)):
        v = order[g]
        Lo, Uo = s.factor_of(v)
        k = Lo.shape[1]
        if k == 0:
            continue
        Lg, Ug = f.export_front(g)
        sc = max(np.abs(Lo).max(), np.abs(Uo).max(), 1.0)
        tol = 4.0 * ksub[v] * u_eff * sc
        low = np.tril(np.ones((Lo.shape[0], k), bool))
        up = np.triu(np.ones((k, Uo.shape[1]), bool), 1)
        eL = np.abs(Lg - Lo)[low].max()
        eU = np.abs(Ug - Uo)[up].max() if up.any() else 0.0
        worst = max(worst, max(eL, eU) / tol)
        assert eL <= tol and eU <= tol, (case, prec, g, eL, eU, tol)
    print(f"{case} {prec}: worst error / bound = {worst:.3f}")


@pytest.mark.parametrize("case,root_f64", [("q3_24_large_path", 1), ("q3_24_large_path", 3), ("q1_3d_8", 2)])
def test_fp64_root_pivot_blocks_factors_and_solution(case, root_f64):
    """FP32 fronts whose top `root_f64` classes factor and invert their pivot blocks in FP64
    (option root_f64): front by front within the FP32 bound of
    test_fp32_family_factors_match_oracle_front_by_front, and the refined solution within 1e-10."""
    mk, opt = FP32_CASES[case]
    pr = mk()
    a, f, vals = _setup(pr, "f32", root_f64=root_f64, **opt)
    f.factor(vals)
    assert f.status()["rc"] == 0
    s = _oracle(pr)
    ksub = np.asarray(s.k, dtype=np.int64).copy()
    for v in range(s.n_front):
        if s.parent[v] >= 0:
            ksub[s.parent[v]] += ksub[v]
    order = np.lexsort((np.arange(s.n_front), s.height))
    top = s.n_classes - root_f64
    checked = 0
    for g in range(len(order)):
        v = order[g]
        if s.height[v] - 1 < top:
            continue
        Lo, Uo = s.factor_of(v)
        k = Lo.shape[1]
        if k == 0:
            continue
        Lg, Ug = f.export_front(g)
        sc = max(np.abs(Lo).max(), np.abs(Uo).max(), 1.0)
        tol = 4.0 * ksub[v] * 2.0 ** -24 * sc
        low = np.tril(np.ones((Lo.shape[0], k), bool))
        up = np.triu(np.ones((k, Uo.shape[1]), bool), 1)
        assert np.abs(Lg - Lo)[low].max() <= tol, (g, root_f64)
        if up.any():
            assert np.abs(Ug - Uo)[up].max() <= tol, (g, root_f64)
        checked += 1
    assert checked >= 1
    b = torch.tensor(np.ascontiguousarray(pr.b.T), device=DEV)
    x = torch.empty_like(b)
    info = f.refine_solve(vals, b, x, tol=1e-15, maxit=30)
    xo, _ = s.solve_refined(pr.b)
    err = np.linalg.norm(x.cpu().numpy().T - xo) / np.linalg.norm(xo)
    assert info["backward_error"] <= 1e-12 and err <= 1e-10, (info, err)


@pytest.mark.parametrize("passes", [1, 3])
def test_bf16_schur_products_refine_to_the_fp64_bar(passes):
    """MF_TF32_BF16 with every Schur update on BF16 tensor-core products (bf16_min_cb and tc_min_cb
    small), on the L2-projection mass matrix, whose condition number is bounded independently of h
    (so even a single BF16 pass, about 2^-9 per product, leaves the refinement contracting):
    (a) front by front within 4 K_f u_eff max|front| of the oracle with u_eff = 2^-8 (one pass) or
    2^-16 (three split passes: the dropped lo x lo term); (b) the refined solution meets the
    1e-12 backward-error and 1e-10 solution bars."""
    pr = F.l2_projection(24, 3)
    a, f, vals = _setup(pr, "tf32_bf16", bf16_passes=passes, bf16_min_cb=16, tc_min_cb=16, small_front_max=16)
    f.factor(vals)
    assert f.status()["rc"] == 0
    s = _oracle(pr)
    ksub = np.asarray(s.k, dtype=np.int64).copy()
    for v in range(s.n_front):
        if s.parent[v] >= 0:
            ksub[s.parent[v]] += ksub[v]
    u_eff = 2.0 ** -8 if passes == 1 else 2.0 ** -16
    order = np.lexsort((np.arange(s.n_front), s.height))
    for g in range(len(order)):
        v = order[g]
        Lo, Uo = s.factor_of(v)
        k = Lo.shape[1]
        if k == 0:
            continue
        Lg, Ug = f.export_front(g)
        sc = max(np.abs(Lo).max(), np.abs(Uo).max())
        tol = 4.0 * ksub[v] * u_eff * sc
        low = np.tril(np.ones((Lo.shape[0], k), bool))
        assert np.abs(Lg - Lo)[low].max() <= tol, (g, passes)
    b = torch.tensor(np.ascontiguousarray(pr.b.T), device=DEV)
    x = torch.empty_like(b)
    info = f.refine_solve(vals, b, x, tol=1e-15, maxit=40)
    xo, _ = s.solve_refined(pr.b)
    err = np.linalg.norm(x.cpu().numpy().T - xo) / np.linalg.norm(xo)
    assert info["backward_error"] <= 1e-12 and err <= 1e-10, (passes, info, err)


FOATA_CASES = {
    "q1_16_all": (lambda: F.poisson_2d_q1(16), 99, {}),
    "q3_6_all": (lambda: F.diffusion_2d(6, 3, seed=61), 99, {}),
    "q1_3d_4_all": (lambda: F.diffusion_3d_q1(4, seed=62), 99, {}),
    "q3_16_bottom4": (lambda: F.diffusion_2d(16, 3, seed=63), 4, {"small_front_max": 48}),
    "l2_q2_12_bottom3": (lambda: F.l2_projection(12, 2), 3, {"small_front_max": 16}),
}


@pytest.mark.parametrize("case", list(FOATA_CASES))
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_scalar_task_foata_executor(case, prec):
    """The bottom classes run as the paper's scalar-task Foata classes (per pivot step one launch of
    assertion, division, multiplication and subtraction tasks over every front of the class):
    FP64 factors front by front within 1e-11 of the oracle (the same tasks in the same order per
    entry as the oracle's Table 2 loop, up to the reciprocal-free division); FP32 factors within the
    FP32 bound of test_fp32_family_factors_match_oracle_front_by_front; refined solutions within
    1e-10."""
    mk, ncls, opt = FOATA_CASES[case]
    pr = mk()
    a, f, vals = _setup(pr, prec, foata_classes=ncls, **opt)
    f.factor(vals)
    st = f.status()
    assert st["rc"] == 0 and st["n_perturbed"] == 0
    s = _oracle(pr)
    if prec == "f64":
        _check_factors(f, s, case)
    else:
        ksub = np.asarray(s.k, dtype=np.int64).copy()
        for v in range(s.n_front):
            if s.parent[v] >= 0:
                ksub[s.parent[v]] += ksub[v]
        order = np.lexsort((np.arange(s.n_front), s.height))
        for g in range(len(order)):
            v = order[g]
            Lo, Uo = s.factor_of(v)
            k = Lo.shape[1]
            if k == 0:
                continue
            Lg, Ug = f.export_front(g)
            tol = 4.0 * ksub[v] * 2.0 ** -24 * max(np.abs(Lo).max(), np.abs(Uo).max(), 1.0)
            low = np.tril(np.ones((Lo.shape[0], k), bool))
            assert np.abs(Lg - Lo)[low].max() <= tol, (case, g)
    b = torch.tensor(np.ascontiguousarray(pr.b.T), device=DEV)
    x = torch.empty_like(b)
    info = f.refine_solve(vals, b, x, tol=1e-15, maxit=30)
    xo, _ = s.solve_refined(pr.b)
    err = np.linalg.norm(x.cpu().numpy().T - xo) / np.linalg.norm(xo)
    assert info["backward_error"] <= 1e-12 and err <= 1e-10, (case, prec, info, err)


def test_scalar_task_foata_executor_static_pivot_check():
    """A singular (pure Neumann) Q1 Laplacian through the Foata executor: the assertion tasks replace
    the zero pivot and count it, as the fused kernels do."""
    mesh = F.structured_mesh((4, 4), 1)
    Ke = F.element_matrices(mesh, dirichlet=False)
    pr = F.Problem("neumann", mesh, Ke, np.ones((mesh.n_nodes, 1)))
    a, f, vals = _setup(pr, "f64", foata_classes=99, pivot_tol=1e-6)
    f.factor(vals)
    st = f.status()
    assert st["rc"] == 0 and st["n_perturbed"] >= 1 and st["first_front"] == a.n_front - 1
    a2, f2, vals2 = _setup(pr, "f64", foata_classes=99, pivot_tol=1e-6, pivot_fail=1)
    f2.factor(vals2)
    assert f2.status()["rc"] == M.mfsolve.MF_EZERO_PIVOT


SYM_CASES = {
    "q3_12_large_path": (lambda: F.diffusion_2d(12, 3, seed=71), {"small_front_max": 16}),
    "q3_24_super_panel": (lambda: F.diffusion_2d(24, 3, seed=72), {"small_front_max": 16, "super_panel": 128}),
    "q1_3d_6_large_path": (lambda: F.diffusion_3d_q1(6, seed=73), {"small_front_max": 24}),
    "l2_q3_10": (lambda: F.l2_projection(10, 3), {"small_front_max": 32}),
}


@pytest.mark.parametrize("case", list(SYM_CASES))
def test_symmetric_mode_f64_factors_match_oracle(case):
    """Option symmetric on SPD matrices: beyond the pivot blocks the large fronts factor only L and
    take U12 = D^-1 L21^T; the exported L and U still equal the oracle's LU factors front by front
    within 1e-11 (U = D^-1 L^T holds exactly for a symmetric A), and solves, adjoint solves and
    refined solves match the oracle."""
    mk, opt = SYM_CASES[case]
    pr = mk()
    a, f, vals = _setup(pr, "f64", symmetric=1, **opt)
    f.factor(vals)
    assert f.status()["rc"] == 0
    s = _oracle(pr)
    _check_factors(f, s, case)
    xo = s.solve(pr.b)
    for adjoint in (False, True):
        x = torch.tensor(np.ascontiguousarray(pr.b.T), device=DEV)
        f.solve(x, adjoint=adjoint)
        assert np.linalg.norm(x.cpu().numpy().T - xo) <= 1e-10 * np.linalg.norm(xo), (case, adjoint)
    b = torch.tensor(np.ascontiguousarray(pr.b.T), device=DEV)
    x = torch.empty_like(b)
    info = f.refine_solve(vals, b, x, tol=1e-15, maxit=20)
    xr, _ = s.solve_refined(pr.b)
    assert info["backward_error"] <= 1e-14
    assert np.linalg.norm(x.cpu().numpy().T - xr) <= 1e-10 * np.linalg.norm(xr)


@pytest.mark.parametrize("case", ["q3_24_super_panel", "q1_3d_6_large_path"])
@pytest.mark.parametrize("prec,extra", [("f32", {}), ("tf32", {"tc_min_cb": 16})])
def test_symmetric_mode_fp32_family_refined_solution(case, prec, extra):
    mk, opt = SYM_CASES[case]
    pr = mk()
    a, f, vals = _setup(pr, prec, symmetric=1, **opt, **extra)
    f.factor(vals)
    assert f.status()["rc"] == 0
    s = _oracle(pr)
    b = torch.tensor(np.ascontiguousarray(pr.b.T), device=DEV)
    x = torch.empty_like(b)
    info = f.refine_solve(vals, b, x, tol=1e-15, maxit=30)
    xr, _ = s.solve_refined(pr.b)
    err = np.linalg.norm(x.cpu().numpy().T - xr) / np.linalg.norm(xr)
    assert info["backward_error"] <= 1e-12 and err <= 1e-10, (info, err)


@pytest.mark.parametrize("case", ["q3_24_super_panel", "q1_3d_6_large_path", "l2_q3_10"])
@pytest.mark.parametrize("prec", ["f32", "tf32"])
def test_conjugate_gradient_refinement(case, prec):
    """Option refine_cg with symmetric factors: FP64 preconditioned conjugate gradients (M^-1 =
    L^-T D L^-1 from the FP32-family factors).  It reaches the 1e-12 backward-error bar (recomputed
    on the host from the true residual) with no more preconditioner applications than stationary
    refinement, and to the FP64 floor the solution matches the oracle to 1e-10."""
    mk, opt = SYM_CASES[case]
    pr = mk()
    extra = {"tc_min_cb": 16} if prec == "tf32" else {}
    a, f, vals = _setup(pr, prec, symmetric=1, refine_cg=1, **opt, **extra)
    a2, f2, _ = _setup(pr, prec, symmetric=1, refine_cg=0, **opt, **extra)
    f.factor(vals)
    f2.factor(vals)
    b = torch.tensor(np.ascontiguousarray(pr.b.T), device=DEV)
    x = torch.empty_like(b)
    x2 = torch.empty_like(b)
    i_cg = f.refine_solve(vals, b, x, tol=1e-12, maxit=30)
    i_st = f2.refine_solve(vals, b, x2, tol=1e-12, maxit=30)
    assert i_cg["rc"] == 0 and i_cg["backward_error"] <= 1e-12
    assert _backward_error_host(pr, x.cpu().numpy().T, pr.b) <= 1e-12
    assert i_cg["iterations"] <= i_st["iterations"], (i_cg, i_st)
    info = f.refine_solve(vals, b, x, tol=1e-15, maxit=30)
    s = _oracle(pr)
    xr, _ = s.solve_refined(pr.b)
    err = np.linalg.norm(x.cpu().numpy().T - xr) / np.linalg.norm(xr)
    assert info["backward_error"] <= 1e-15 and err <= 1e-10, (info, err)


@pytest.mark.parametrize("prec", ["f32", "tf32"])
@pytest.mark.parametrize("maxit", [30, 1])
@pytest.mark.parametrize("method", ["cg", "stationary", "adjoint"])
def test_device_side_refinement_loop_matches_host_loop(prec, maxit, method):
    """With graph replay on a created stream the refinement iterations run inside one graph (a
    while-conditional node whose body is one iteration and the stop test computed on the device):
    CG, stationary refinement, and stationary refinement of the adjoint system.  On the default
    stream (no graphs) the host drives the same steps.  Iteration count, backward error, the
    iterate itself (bit for bit: the same kernels in the same order) and the per-family launch
    accounting (plus one stop-test kernel per loop test) agree, on a converging run and on one
    stopped by the iteration limit; a second call replays the cached loop graph."""
    mk, opt = SYM_CASES["q3_24_super_panel"]
    pr = mk()
    extra = {"tc_min_cb": 16} if prec == "tf32" else {}
    a, f, vals = _setup(pr, prec, symmetric=1, refine_cg=1 if method != "stationary" else 0, use_graph=1, **opt,
                        **extra)
    f.factor(vals)
    torch.cuda.synchronize()
    adj = method == "adjoint"
    b = torch.tensor(np.ascontiguousarray(pr.b.T), device=DEV)
    x_h = torch.empty_like(b)
    f.profile_read()
    i_h = f.refine_solve(vals, b, x_h, tol=1e-12, maxit=maxit, adjoint=adj)
    torch.cuda.synchronize()
    l_h = {k: v["launches"] for k, v in f.profile_read().items()}
    st = torch.cuda.Stream()
    outs = []
    for rep in range(2):
        x_d = torch.empty_like(b)
        with torch.cuda.stream(st):
            i_d = f.refine_solve(vals, b, x_d, tol=1e-12, maxit=maxit, stream=st, adjoint=adj)
        st.synchronize()
        outs.append((i_d, x_d, {k: v["launches"] for k, v in f.profile_read().items()}))
    for i_d, x_d, l_d in outs:
        assert i_d["rc"] == i_h["rc"] and i_d["iterations"] == i_h["iterations"], (i_d, i_h)
        assert i_d["backward_error"] == i_h["backward_error"], (i_d, i_h)
        assert torch.equal(x_d, x_h)
        # stop tests on the device: one per iteration, plus the one after the first solve for the
        # stationary loop (counted with the "other" family)
        tests = i_d["iterations"] + (0 if method == "cg" else 1)
        l_d = dict(l_d, other=l_d["other"] - tests)
        assert l_d == l_h, (l_d, l_h)
    if maxit == 1:
        assert i_h["iterations"] == 1
    else:
        assert i_h["rc"] == 0 and i_h["backward_error"] <= 1e-12


@pytest.mark.parametrize("case", ["q3_24_lookahead", "q3_12_large_path", "q1_3d_6_large_path"])
@pytest.mark.parametrize("sym", [0, 1])
def test_panel_triangular_solves_factors_match_oracle(case, sym):
    """Option panel_trsm: each pivot block's panel finished by triangular solves against the factored
    block instead of products with its inverses; FP64 factors front by front within 1e-11."""
    mk, opt = CASES[case] if case in CASES else SYM_CASES[case]
    pr = mk()
    a, f, vals = _setup(pr, "f64", panel_trsm=1, symmetric=sym, **opt)
    f.factor(vals)
    assert f.status()["rc"] == 0
    _check_factors(f, _oracle(pr), case)


@pytest.mark.parametrize("case", ["q3_24_large_path", "q1_3d_8"])
@pytest.mark.parametrize("tc_direct", [0, 1])
def test_tensor_core_operand_paths_front_by_front(case, tc_direct):
    """3xTF32 tensor-core products through the separate pack pass (tc_direct 0, the default) and with
    the operands split inside the product kernel (tc_direct 1): every front within the split-TF32
    bound of test_fp32_family_factors_match_oracle_front_by_front, on the same inputs."""
    mk, opt = FP32_CASES[case]
    pr = mk()
    a, f, vals = _setup(pr, "tf32", tc_min_cb=16, tc_direct=tc_direct, **opt)
    f.factor(vals)
    assert f.status()["rc"] == 0
    s = _oracle(pr)
    ksub = np.asarray(s.k, dtype=np.int64).copy()
    for v in range(s.n_front):
        if s.parent[v] >= 0:
            ksub[s.parent[v]] += ksub[v]
    order = np.lexsort((np.arange(s.n_front), s.height))
    for g in range(len(order)):
        v = order[g]
        Lo, Uo = s.factor_of(v)
        k = Lo.shape[1]
        if k == 0:
            continue
        Lg, Ug = f.export_front(g)
        tol = 4.0 * ksub[v] * 2.0 ** -21 * max(np.abs(Lo).max(), np.abs(Uo).max(), 1.0)
        low = np.tril(np.ones((Lo.shape[0], k), bool))
        up = np.triu(np.ones((k, Uo.shape[1]), bool), 1)
        assert np.abs(Lg - Lo)[low].max() <= tol, (case, tc_direct, g)
        if up.any():
            assert np.abs(Ug - Uo)[up].max() <= tol, (case, tc_direct, g)

