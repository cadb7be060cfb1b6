"""Pins for the FP64 CPU oracle against facts fixed by mathematics and the paper.

Each test checks the oracle against something other than itself: LAPACK
(dense solve, Cholesky), exact rational arithmetic, closed forms, brute force
on tiny meshes, and invariants the paper states (Foata classes, Sec. 3.3).
"""
import itertools
from fractions import Fraction

import numpy as np
import pytest

import fem_inputs as F
import oracle as O


def _solver(mesh, tree=None):
    tree = tree or O.tree_bisection(mesh.nel)
    return O.OracleSolver(mesh.n_nodes, mesh.elem_nodes, tree)


# ----------------------------------------------------------------- inputs
def test_q1_element_stiffness_closed_form():
    # textbook bilinear square stiffness, lexicographic local order (0,0),(1,0),(0,1),(1,1)
    K = F.reference_stiffness(2, 1)
    ref = np.array([[4, -1, -1, -2], [-1, 4, -2, -1], [-1, -2, 4, -1], [-2, -1, -1, 4]]) / 6.0
    assert np.allclose(K, ref, atol=1e-15)
    gold = np.loadtxt(__file__.replace("test_oracle.py", "golden/q1_square_stiffness.txt"))
    assert np.allclose(K, gold, atol=1e-15)


@pytest.mark.parametrize("dim,p", [(2, 1), (2, 3), (3, 1)])
def test_stiffness_kills_constants(dim, p):
    K = F.reference_stiffness(dim, p)
    assert np.abs(K.sum(axis=1)).max() < 1e-13
    assert np.allclose(K, K.T)


# ------------------------------------------------------------------ trees
@pytest.mark.parametrize("nel", [(2, 2), (8, 8), (16, 16), (4, 4, 4), (8, 8, 8)])
def test_bisection_equals_paper_pairing_on_power_of_two_grids(nel):
    a = O.tree_bisection(nel)
    b = O.tree_pairing(nel)
    assert np.array_equal(a.parent, b.parent)
    assert np.array_equal(a.child, b.child)
    assert np.array_equal(a.leaf_elem, b.leaf_elem)


@pytest.mark.parametrize("nel", [(3, 3), (5, 7)])
def test_pairing_carries_odd_front(nel):
    t = O.tree_pairing(nel)
    ne = int(np.prod(nel))
    assert t.n == 2 * ne - 1
    assert sorted(t.leaf_elem[t.leaf_elem >= 0].tolist()) == list(range(ne))
    # every internal node has exactly two children (the odd front is not wrapped)
    internal = t.leaf_elem < 0
    assert np.all(t.child[internal] >= 0)


# --------------------------------------------------------------- symbolic
def _subtree_elems(tree):
    out = [None] * tree.n
    for v in range(tree.n):
        if tree.leaf_elem[v] >= 0:
            out[v] = {int(tree.leaf_elem[v])}
        else:
            out[v] = set().union(*[out[c] for c in tree.child[v] if c >= 0])
    return out


@pytest.mark.parametrize("nel,p,rule", [((4, 4), 1, "bisect"), ((5, 5), 1, "bisect"), ((3, 3), 3, "bisect"),
                                         ((3, 3, 3), 1, "bisect"), ((5, 5), 1, "pair"), ((3, 3), 2, "pair")])
def test_symbolic_matches_brute_force(nel, p, rule):
    mesh = F.structured_mesh(nel, p)
    tree = O.tree_bisection(nel) if rule == "bisect" else O.tree_pairing(nel)
    s = _solver(mesh, tree)
    sub = _subtree_elems(tree)
    elems_of = [set() for _ in range(mesh.n_nodes)]
    for e, nodes in enumerate(mesh.elem_nodes):
        for d in nodes:
            elems_of[d].add(e)
    # pivot front of a dof: smallest subtree containing all its elements
    elim = []
    for d in range(mesh.n_nodes):
        cands = [v for v in range(tree.n) if elems_of[d] <= sub[v]]
        elim.append(min(cands, key=lambda v: len(sub[v])))
    for v in range(tree.n):
        fd = s.front_dofs(v)
        k = int(s.k[v])
        piv = sorted(d for d in range(mesh.n_nodes) if elim[d] == v)
        assert fd[:k].tolist() == piv
        touching = {int(d) for e in sub[v] for d in mesh.elem_nodes[e]}
        cbset = sorted(d for d in touching if elim[d] != v and not (sub[elim[d]] < sub[v]))
        assert fd[k:].tolist() == cbset
    assert int(s.k.sum()) == mesh.n_nodes


@pytest.mark.parametrize("n,p", [(16, 1), (32, 3), (8, 3)])
def test_root_is_the_full_separator_line_2d(n, p):
    mesh = F.structured_mesh((n, n), p)
    s = _solver(mesh)
    assert int(s.m[-1]) == p * n + 1 == int(s.k[-1])
    assert s.n_classes == int(np.log2(n * n)) + 1
    assert s.n_front == 2 * n * n - 1


def test_root_is_the_full_separator_plane_3d():
    mesh = F.structured_mesh((8, 8, 8), 1)
    s = _solver(mesh)
    assert int(s.m[-1]) == 81 and s.n_classes == 10


def test_symbolic_counts_golden():
    """Sizes of the 16x16 Q1 case, written by tests/golden/make_golden.py from the oracle."""
    gold = dict(np.loadtxt(__file__.replace("test_oracle.py", "golden/symbolic_poisson2d_q1_16.txt"),
                           dtype=str, delimiter="="))
    s = _solver(F.structured_mesh((16, 16), 1))
    assert s.n_front == int(gold["n_front"]) and s.n_classes == int(gold["n_classes"])
    assert s.max_m == int(gold["max_m"]) and s.nnz_lu == int(gold["nnz_lu"])
    assert s.sum_cb == int(gold["sum_cb"]) and s.flops == int(gold["flops"])


# ------------------------------------------------------------------ Foata
@pytest.mark.parametrize("nel,rule", [((8, 8), "bisect"), ((5, 5), "bisect"), ((4, 4, 4), "bisect"),
                                      ((7, 7), "pair"), ((3, 3, 3), "pair")])
def test_foata_classes_are_the_brute_force_layering(nel, rule):
    tree = O.tree_bisection(nel) if rule == "bisect" else O.tree_pairing(nel)
    # brute force: repeatedly peel every front whose children are all done
    done = np.zeros(tree.n, bool)
    layer = np.zeros(tree.n, int)
    c = 0
    while not done.all():
        c += 1
        ready = [v for v in range(tree.n) if not done[v] and all(done[ch] for ch in tree.child[v] if ch >= 0)]
        for v in ready:
            layer[v] = c
        done[ready] = True
    s = _solver(F.structured_mesh(nel, 1), tree)
    assert np.array_equal(layer, s.height)
    assert s.n_classes == layer.max()
    anc = [set() for _ in range(tree.n)]
    for v in range(tree.n - 1, -1, -1):
        if tree.parent[v] >= 0:
            anc[v] = anc[tree.parent[v]] | {int(tree.parent[v])}
    for cl in range(1, s.n_classes + 1):
        members = np.nonzero(s.height == cl)[0]
        for a, b in itertools.combinations(members, 2):
            assert a not in anc[b] and b not in anc[a]
        if cl > 1:
            for v in members:
                assert any(s.height[ch] == cl - 1 for ch in tree.child[v] if ch >= 0)


@pytest.mark.parametrize("nel", [(2, 2), (3, 3)])
def test_front_classes_coarsen_the_scalar_task_dag(nel):
    """Sec. 3.3 defines Foata classes over the scalar tasks of Table 2 (T1: divide an entry of
    the pivot row; T2/T3: update a trailing entry) and the extend-add of a child's block into
    its parent; the build schedules whole fronts by height instead.  On tiny Q1 meshes the
    scalar task DAG is built from the data each task reads and writes (program order inside a
    front, extend-add after the child's last write), and the front-level classes are checked to
    be a valid coarsening of it: every dependency between tasks of different fronts goes from a
    lower class to a higher one, no dependency path joins two fronts of the same class, and the
    task-level Foata layering needs at least as many layers as there are front classes."""
    mesh = F.structured_mesh(nel, 1)
    tree = O.tree_bisection(mesh.nel)
    s = _solver(mesh, tree)
    tasks = []        # (front, label)
    preds = []        # list of predecessor task ids
    last_write = {}   # (front, i, j) -> task id of the last write of that entry
    def add(front, label, reads, writes):
        tid = len(tasks)
        tasks.append((front, label))
        preds.append(sorted({last_write[e] for e in reads + writes if e in last_write}))
        for e in writes:
            last_write[e] = tid
        return tid
    for v in range(s.n_front):  # fronts in postorder: children first
        m, k = int(s.m[v]), int(s.k[v])
        for c in tree.child[v]:
            if c < 0:
                continue
            cd = s.front_dofs(c)
            kc = int(s.k[c])
            pos = {int(d): q for q, d in enumerate(s.front_dofs(v))}
            for a in range(kc, int(s.m[c])):
                for b in range(kc, int(s.m[c])):
                    add(v, "extend-add", [(c, a, b)], [(v, pos[int(cd[a])], pos[int(cd[b])])])
        for p in range(k):
            for j in range(p + 1, m):
                add(v, "T1", [(v, p, p), (v, p, j)], [(v, p, j)])
            for i in range(p + 1, m):
                for j in range(p + 1, m):
                    add(v, "T23", [(v, i, j), (v, i, p), (v, p, j)], [(v, i, j)])
    n = len(tasks)
    layer = np.zeros(n, int)
    for t in range(n):  # ids are a topological order
        layer[t] = 1 + max((layer[q] for q in preds[t]), default=0)
    front = np.array([f for f, _ in tasks])
    h = np.asarray(s.height)
    for t in range(n):
        for q in preds[t]:
            if front[q] != front[t]:
                assert h[front[q]] < h[front[t]], (tasks[q], tasks[t])
    # no path between two different fronts of one class: reachable fronts per task (bitsets)
    reach = [0] * n
    for t in range(n):
        r = 1 << int(front[t])
        for q in preds[t]:
            r |= reach[q]
        reach[t] = r
    for t in range(n):
        for f2 in range(s.n_front):
            if f2 != front[t] and (reach[t] >> f2) & 1:
                assert h[f2] < h[front[t]], (tasks[t], f2)
    assert layer.max() >= s.n_classes


# ------------------------------------------------- work counts (orc_info)
def test_work_counts_of_a_hand_worked_two_element_mesh():
    """2x1 Q1 mesh, 6 nodes numbered x fastest: element 0 = {0,1,3,4}, element 1 = {1,2,4,5}.
    By hand: each leaf eliminates its two private nodes (k = 2, m = 4: pivot 0 costs 3 divisions
    + 2*3^2 mult/sub = 21, pivot 1 costs 2 + 2*2^2 = 10, so 31) and passes the shared pair {1, 4}
    up; the root has m = k = 2 (pivot 0: 1 + 2*1 = 3, pivot 1: 0).  Flops 31 + 31 + 3 = 65.
    nnz(L+U): a leaf stores 4*2 + 2*2 = 12 entries, the root 2*2 = 4, so 28; CB entries 4 + 4."""
    en = np.array([[0, 1, 3, 4], [1, 2, 4, 5]], dtype=np.int64)
    s = O.OracleSolver(6, en, O.tree_bisection((2, 1)))
    assert s.n_front == 3 and s.n_classes == 2
    assert s.flops == 65 and s.nnz_lu == 28 and s.sum_cb == 8 and s.max_m == 4 and s.max_k == 2


@pytest.mark.parametrize("p", [1, 2, 3])
def test_work_counts_of_one_dense_element_closed_form(p):
    """One element = one front factored completely (m = k = (p+1)^2): divisions
    sum_{q<m} (m-q-1) = m(m-1)/2, multiplications and subtractions 2 sum_{q<m} (m-q-1)^2
    = (m-1)m(2m-1)/3, nnz(L+U) = m^2, no contribution block."""
    s = _solver(F.structured_mesh((1, 1), p))
    m = (p + 1) ** 2
    assert s.n_front == 1 and int(s.k[0]) == m
    assert s.flops == m * (m - 1) // 2 + (m - 1) * m * (2 * m - 1) // 3
    assert s.nnz_lu == m * m and s.sum_cb == 0


@pytest.mark.parametrize("nel,p", [((4, 4), 1), ((3, 3), 3), ((3, 3, 3), 1), ((5, 5), 2)])
def test_work_counts_by_task_enumeration(nel, p):
    """orc_info's flop count equals the number of Table 2 tasks the fronts perform, enumerated one
    by one (a division per entry right of each pivot in its row, a multiplication and a
    subtraction per trailing entry), and nnz(L+U) equals the number of front positions a pivot row
    or column covers (counted on a boolean mask of each front)."""
    s = _solver(F.structured_mesh(nel, p))
    t1 = t23 = nnz = 0
    for v in range(s.n_front):
        m, k = int(s.m[v]), int(s.k[v])
        for q in range(k):
            t1 += len(range(q + 1, m))
            t23 += len(range(q + 1, m)) ** 2
        mask = np.zeros((m, m), bool)
        mask[:k, :] = True
        mask[:, :k] = True
        nnz += int(mask.sum())
    assert s.flops == t1 + 2 * t23
    assert s.nnz_lu == nnz


@pytest.mark.parametrize("mk", [lambda: F.poisson_2d_q1(6), lambda: F.diffusion_2d(2, 3, seed=7)])
def test_front_blocks_cover_every_nonzero_of_the_dense_factors(mk):
    """The fronts' pivot rows and columns (the nnz(L+U) positions) contain every nonzero of the
    dense L and U of P A P^T computed by LAPACK, so nnz_lu bounds the true factor count from above;
    it is tight up to the structural zeros a dense front keeps."""
    pr = mk()
    mesh = pr.mesh
    s = _solver(mesh)
    n = mesh.n_nodes
    perm = np.concatenate([s.front_dofs(v)[: s.k[v]] for v in range(s.n_front)])
    pos = np.empty(n, int)
    pos[perm] = np.arange(n)
    covered = np.zeros((n, n), bool)
    for v in range(s.n_front):
        fd = pos[s.front_dofs(v)]
        k = int(s.k[v])
        covered[np.ix_(fd, fd[:k])] = True      # L: pivot columns
        covered[np.ix_(fd[:k], fd)] = True      # U: pivot rows
    assert int(covered.sum()) == s.nnz_lu       # fronts' pivot blocks never overlap
    A = F.assemble_dense(mesh, pr.Ke)[np.ix_(perm, perm)]
    C = np.linalg.cholesky(A)
    nzL = np.abs(C) > 1e-14 * np.abs(C).max()
    full = nzL | nzL.T
    assert not (full & ~covered).any()
    assert int(full.sum()) <= s.nnz_lu


# --------------------------------------------------------------- factors
def _global_factors(s, n):
    perm = np.concatenate([s.front_dofs(v)[: s.k[v]] for v in range(s.n_front)])
    pos = np.empty(n, int)
    pos[perm] = np.arange(n)
    L = np.zeros((n, n))
    U = np.eye(n)
    for v in range(s.n_front):
        Lv, Uv = s.factor_of(v)
        fd = s.front_dofs(v)
        k = int(s.k[v])
        for p in range(k):
            L[pos[fd[p:]], pos[fd[p]]] = Lv[p:, p]
            U[pos[fd[p]], pos[fd[p + 1:]]] = Uv[p, p + 1:]
    return perm, L, U


@pytest.mark.parametrize("mk", [lambda: F.poisson_2d_q1(8), lambda: F.diffusion_2d(3, 3, seed=7),
                                lambda: F.diffusion_3d_q1(3, seed=5)])
def test_factors_equal_dense_cholesky_derived_lu(mk):
    pr = mk()
    mesh = pr.mesh
    s = _solver(mesh)
    assert s.factor(F.to_colmajor(pr.Ke)) == 0
    A = F.assemble_dense(mesh, pr.Ke)
    perm, L, U = _global_factors(s, mesh.n_nodes)
    Ap = A[np.ix_(perm, perm)]
    # SPD: A_p = C C^T (LAPACK) -> the unique L (non-unit) U (unit) pair is
    # L = C diag(C), U = diag(C)^-1 C^T
    C = np.linalg.cholesky(Ap)
    d = np.diag(C)
    Lref = C * d[None, :]
    Uref = (C / d[None, :]).T
    sc = np.abs(Ap).max()
    assert np.abs(L - Lref).max() <= 1e-13 * sc
    assert np.abs(U - Uref).max() <= 1e-13
    assert np.abs(np.triu(L, 1)).max() == 0 and np.abs(np.tril(U, -1)).max() == 0


def test_factors_reproduce_unsymmetric_matrix():
    pr = F.convection_2d_q1(4)
    s = _solver(pr.mesh)
    assert s.factor(F.to_colmajor(pr.Ke)) == 0
    A = F.assemble_dense(pr.mesh, pr.Ke)
    assert np.abs(A - A.T).max() > 1e-3
    perm, L, U = _global_factors(s, pr.mesh.n_nodes)
    Ap = A[np.ix_(perm, perm)]
    assert np.abs(L @ U - Ap).max() <= 1e-14 * np.abs(Ap).max()


# ------------------------------------------------------------------ solve
@pytest.mark.parametrize("mk", [lambda: F.poisson_2d_q1(8), lambda: F.diffusion_2d(4, 3, seed=3),
                                lambda: F.diffusion_3d_q1(4, seed=5), lambda: F.convection_2d_q1(5)])
def test_solve_matches_dense_lapack(mk):
    pr = mk()
    s = _solver(pr.mesh)
    s.factor(F.to_colmajor(pr.Ke))
    A = F.assemble_dense(pr.mesh, pr.Ke)
    x = s.solve(pr.b)
    xr = np.linalg.solve(A, pr.b)
    assert np.abs(x - xr).max() <= 1e-12 * np.abs(xr).max()
    xa = s.solve(pr.b, adjoint=True)
    xar = np.linalg.solve(A.T, pr.b)
    assert np.abs(xa - xar).max() <= 1e-12 * np.abs(xar).max()


def test_adjoint_solve_equals_solve_for_symmetric():
    pr = F.poisson_2d_q1(16)
    s = _solver(pr.mesh)
    s.factor(F.to_colmajor(pr.Ke))
    x = s.solve(pr.b)
    xa = s.solve(pr.b, adjoint=True)
    assert np.abs(x - xa).max() <= 1e-13 * np.abs(x).max()


def test_residual_small_at_16():
    pr = F.poisson_2d_q1(16)
    s = _solver(pr.mesh)
    K = F.to_colmajor(pr.Ke)
    s.factor(K)
    x = s.solve(pr.b)
    r = O.residual_dd(pr.mesh.elem_nodes, K, x, pr.b)
    assert np.linalg.norm(r) / np.linalg.norm(pr.b) <= 1e-14


def test_manufactured_solution_converges_second_order():
    errs = []
    for n in (16, 32, 64):
        pr = F.poisson_2d_q1(n)
        s = _solver(pr.mesh)
        s.factor(F.to_colmajor(pr.Ke))
        x = s.solve(pr.b[:, 0])
        errs.append(np.abs(x - F.manufactured_u(pr.mesh.node_coords)).max())
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.6 <= r1 <= 4.4 and 3.6 <= r2 <= 4.4, errs


# --------------------------------------------------- exact arithmetic pins
def _integer_problem(n=4, seed=0):
    rng = np.random.default_rng(seed)
    mesh = F.structured_mesh((n, n), 1)
    Ke = np.round(F.element_matrices(mesh, dirichlet=False) * 6.0)  # integer Q1 stiffness
    # add an integer diagonal shift per element so the matrix is nonsingular
    Ke[:, np.arange(4), np.arange(4)] += rng.integers(1, 4, (mesh.n_elem, 4))
    return mesh, Ke


def test_residual_dd_is_exact_on_integers():
    mesh, Ke = _integer_problem(6)
    rng = np.random.default_rng(1)
    x = rng.integers(-1000, 1000, mesh.n_nodes).astype(np.float64) + 0.5
    b = rng.integers(-10 ** 6, 10 ** 6, mesh.n_nodes).astype(np.float64)
    A = F.assemble_dense(mesh, Ke).astype(np.int64)
    exact = (2 * b.astype(np.int64) - A @ (2 * x).astype(np.int64)) / 2.0
    r = O.residual_dd(mesh.elem_nodes, F.to_colmajor(Ke), x, b)
    assert np.array_equal(r, exact)


def test_refined_solution_is_correctly_rounded_against_rationals():
    mesh, Ke = _integer_problem(3, seed=2)
    n = mesh.n_nodes
    A = F.assemble_dense(mesh, Ke).astype(np.int64)
    rng = np.random.default_rng(3)
    b = rng.integers(-50, 50, n)
    # exact rational Gaussian elimination
    M = [[Fraction(int(A[i, j])) for j in range(n)] + [Fraction(int(b[i]))] for i in range(n)]
    for c in range(n):
        piv = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[piv] = M[piv], M[c]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c] / M[c][c]
                M[r] = [a - f * bb for a, bb in zip(M[r], M[c])]
    xex = np.array([float(M[i][n] / M[i][i]) for i in range(n)])
    s = _solver(mesh)
    s.factor(F.to_colmajor(Ke))
    x, it = s.solve_refined(b.astype(np.float64))
    ulps = np.abs(x - xex) / np.spacing(np.abs(xex))
    assert ulps.max() <= 2, ulps.max()


# -------------------------------------------------------------- pivoting
def test_static_pivot_check_on_singular_neumann_matrix():
    mesh = F.structured_mesh((4, 4), 1)
    Ke = F.element_matrices(mesh, dirichlet=False)  # pure Neumann: constants in the kernel
    s = _solver(mesh)
    n = s.factor(F.to_colmajor(Ke), tau=1e-8)
    assert n >= 1
    assert s.factor(F.to_colmajor(Ke), tau=1e-8, fail_small=True) == O.ORC_EZERO_PIVOT
    # a regular matrix never trips the same threshold
    pr = F.poisson_2d_q1(4)
    assert _solver(pr.mesh).factor(F.to_colmajor(pr.Ke), tau=1e-8, fail_small=True) == 0


# -------------------------------------------------------------- gradient
def test_element_gradient_matches_central_differences():
    pr = F.adjoint_problem(n=6, n_fd=6)
    mesh, ut, theta = pr.mesh, pr.extra["u_target"], pr.extra["theta"]

    def J(th):
        Ke = F.element_matrices(mesh, np.exp(th))
        s = _solver(mesh)
        s.factor(F.to_colmajor(Ke))
        x = s.solve(pr.b[:, 0])
        return 0.5 * np.sum((x - ut) ** 2), s, x

    J0, s, x = J(theta)
    lam = s.solve(x - ut, adjoint=True)
    g = O.element_grad(mesh.elem_nodes, F.to_colmajor(pr.extra["dK"]), lam, x)
    h = 1e-5
    for e in pr.extra["fd_elems"]:
        tp, tm = theta.copy(), theta.copy()
        tp[e] += h
        tm[e] -= h
        fd = (J(tp)[0] - J(tm)[0]) / (2 * h)
        assert abs(fd - g[e]) <= 1e-6 * max(abs(fd), 1e-12) + 1e-11, (e, fd, g[e])


def test_openmp_class_parallel_factor_is_bitwise_serial():
    pr = F.diffusion_2d(16, 3, seed=11)
    K = F.to_colmajor(pr.Ke)
    s1 = _solver(pr.mesh)
    s1.factor(K, nthreads=1)
    s2 = _solver(pr.mesh)
    s2.factor(K, nthreads=4)
    assert np.array_equal(s1.solve(pr.b), s2.solve(pr.b))


# ------------------------------------------------- L2-projection workload
def test_q1_element_mass_closed_form():
    """Bilinear unit-square mass matrix, lexicographic local order: (1/36)[[4,2,2,1],...]."""
    M = F.reference_mass(2, 1)
    ref = np.array([[4, 2, 2, 1], [2, 4, 1, 2], [2, 1, 4, 2], [1, 2, 2, 4]]) / 36.0
    assert np.allclose(M, ref, atol=1e-16)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_mass_entries_sum_to_the_area(p):
    """Partition of unity: sum_ab int phi_a phi_b = int 1 over the unit square = 1 (any order)."""
    assert abs(F.reference_mass(2, p).sum() - 1.0) < 1e-14
    pr = F.l2_projection(5, p)
    A = F.assemble_dense(pr.mesh, pr.Ke)
    assert abs(A.sum() - 1.0) < 1e-13
    assert np.allclose(A, A.T) and np.linalg.eigvalsh(A).min() > 0


@pytest.mark.parametrize("p", [1, 2, 3])
def test_l2_projection_reproduces_the_discrete_space(p):
    """The L2 projection onto Qp is the identity on Qp: projecting f = x^p y^(p-1) + x y (a member
    of Qp) with the oracle returns f at every node up to rounding."""
    f = lambda x, y, z=None: x ** p * y ** (p - 1) + x * y
    pr = F.l2_projection(6, p, f)
    s = _solver(pr.mesh)
    assert s.factor(F.to_colmajor(pr.Ke)) == 0
    u, _ = s.solve_refined(pr.b)
    c = pr.mesh.node_coords
    assert np.abs(u[:, 0] - f(c[:, 0], c[:, 1])).max() <= 1e-12


def _l2_error(pr, u, f):
    """||u_h - f||_L2 over the unit square, element by element with (p+3)^2 Gauss points."""
    m = pr.mesh
    t, w = F.gauss_legendre_01(m.p + 3)
    V, _ = F.lagrange_1d(m.p, t)
    phi = np.einsum("aq,br->barq", V, V).reshape((m.p + 1) ** 2, -1)   # x-fastest local, x-fastest points
    qx, qy = np.meshgrid(t, t, indexing="xy")
    wq = np.outer(w, w).ravel()
    org = m.node_coords[m.elem_nodes[:, 0]]
    X = org[:, 0:1] + m.h * qx.ravel()[None, :]
    Y = org[:, 1:2] + m.h * qy.ravel()[None, :]
    uq = u[m.elem_nodes] @ phi
    return float(np.sqrt(((uq - f(X, Y)) ** 2 * wq[None, :]).sum() * m.h ** 2))


@pytest.mark.parametrize("p", [1, 2, 3])
def test_l2_projection_converges_at_order_p_plus_1(p):
    """For a smooth f the L2-projection error ||u_h - f||_L2 (quadrature of degree 2p+5 per
    element) falls like h^(p+1): halving h divides it by about 2^(p+1)."""
    errs = []
    for n in (4, 8, 16):
        pr = F.l2_projection(n, p)
        s = _solver(pr.mesh)
        assert s.factor(F.to_colmajor(pr.Ke)) == 0
        u, _ = s.solve_refined(pr.b)
        errs.append(_l2_error(pr, u[:, 0], F.l2_field))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    lo, hi = 0.8 * 2 ** (p + 1), 1.25 * 2 ** (p + 1)
    assert lo <= r2 <= hi and r1 >= 0.6 * 2 ** (p + 1), (errs, r1, r2)
