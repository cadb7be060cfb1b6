"""Seeded synthetic finite-element inputs shared by the oracle and the CUDA path.

This module only *produces inputs*: structured meshes, element stiffness
matrices (with Dirichlet rows/columns already folded in), right-hand sides and
per-element coefficients.  It contains none of the multifrontal method's
arithmetic (no elimination tree, no factorization, no solve), so both the
oracle and the product path can draw their inputs from it without sharing any
of the method.

The paper's benchmark system is an SPD finite-element matrix (Sec. 2.1, Eq.
"Linear_system"); each front at the bottom of the elimination tree is one
element matrix (Sec. 2.4, step 1).  The stand-in workloads here are Poisson /
heterogeneous-diffusion stiffness matrices on structured quad/hex grids with
Lagrange elements of order p = 1 or 3, the p-range the paper measures (Sec. 4).

Conventions
-----------
* Nodes are numbered lexicographically, x fastest: node (ix, iy[, iz]) has id
  ix + NX*(iy + NY*iz) with NX = p*nx + 1 etc.
* Element-local nodes are tensor-product lexicographic, x fastest, on the
  equispaced points t_a = a/p of the element.
* ``Ke[e, a, b]`` is row a, column b of element e's matrix.  The C ABI wants
  each element matrix column-major; :func:`to_colmajor` does that transpose.
* Dirichlet nodes (domain boundary): the element rows and columns of such a
  node are zeroed and its diagonal set to 1/mult(node), mult = number of
  elements touching the node, so the assembled row is the identity row.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, List, Optional

import numpy as np

SEED_BASE = 20230615


# --------------------------------------------------------------------------- mesh
@dataclass
class StructuredMesh:
    dim: int
    nel: tuple            # elements per axis (nx, ny[, nz])
    p: int                # Lagrange order
    elem_nodes: np.ndarray  # (n_elem, npe) int64
    node_coords: np.ndarray  # (n_nodes, dim) float64
    boundary: np.ndarray  # (n_nodes,) bool, on the domain boundary
    mult: np.ndarray      # (n_nodes,) int32, elements touching each node
    h: float

    @property
    def n_elem(self) -> int:
        return int(self.elem_nodes.shape[0])

    @property
    def npe(self) -> int:
        return int(self.elem_nodes.shape[1])

    @property
    def n_nodes(self) -> int:
        return int(self.node_coords.shape[0])

    @property
    def grid_dims(self) -> np.ndarray:
        return np.array(list(self.nel) + [1] * (3 - self.dim), dtype=np.int32)

    def elem_centroids(self) -> np.ndarray:
        return self.node_coords[self.elem_nodes].mean(axis=1)


def structured_mesh(nel, p: int = 1) -> StructuredMesh:
    """Unit square/cube split into nx*ny(*nz) equal elements of order p."""
    nel = tuple(int(n) for n in nel)
    dim = len(nel)
    assert dim in (2, 3) and p >= 1
    if dim == 3:
        assert nel[0] == nel[1] == nel[2], "cubes only"
    else:
        assert nel[0] == nel[1], "squares only (h equal on both axes)"
    h = 1.0 / nel[0]
    NN = [p * n + 1 for n in nel]
    n_nodes = int(np.prod(NN))
    # node coordinates
    axes = [np.arange(N) * (h / p) for N in NN]
    if dim == 2:
        X, Y = np.meshgrid(axes[0], axes[1], indexing="xy")  # shape (NY, NX)
        coords = np.stack([X.ravel(), Y.ravel()], axis=1)
        idx = np.arange(n_nodes).reshape(NN[1], NN[0])
        bnd = np.zeros((NN[1], NN[0]), bool)
        bnd[0, :] = bnd[-1, :] = bnd[:, 0] = bnd[:, -1] = True
        ex, ey = np.meshgrid(np.arange(nel[0]), np.arange(nel[1]), indexing="xy")
        ex, ey = ex.ravel(), ey.ravel()   # element id = ex + nx*ey
        la, lb = np.meshgrid(np.arange(p + 1), np.arange(p + 1), indexing="xy")
        la, lb = la.ravel(), lb.ravel()   # local id = a + (p+1)*b
        en = idx[(p * ey)[:, None] + lb[None, :], (p * ex)[:, None] + la[None, :]]
    else:
        Z, Y, X = np.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
        coords = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
        idx = np.arange(n_nodes).reshape(NN[2], NN[1], NN[0])
        bnd = np.zeros((NN[2], NN[1], NN[0]), bool)
        bnd[0], bnd[-1] = True, True
        bnd[:, 0], bnd[:, -1] = True, True
        bnd[:, :, 0], bnd[:, :, -1] = True, True
        ez, ey, ex = np.meshgrid(np.arange(nel[2]), np.arange(nel[1]), np.arange(nel[0]), indexing="ij")
        ex, ey, ez = ex.ravel(), ey.ravel(), ez.ravel()
        lc, lb, la = np.meshgrid(np.arange(p + 1), np.arange(p + 1), np.arange(p + 1), indexing="ij")
        la, lb, lc = la.ravel(), lb.ravel(), lc.ravel()
        en = idx[(p * ez)[:, None] + lc[None, :], (p * ey)[:, None] + lb[None, :], (p * ex)[:, None] + la[None, :]]
    en = np.ascontiguousarray(en, dtype=np.int64)
    mult = np.bincount(en.ravel(), minlength=n_nodes).astype(np.int32)
    return StructuredMesh(dim, nel, p, en, coords, bnd.ravel().copy(), mult, h)


# ------------------------------------------------------------- reference element
def gauss_legendre_01(n: int):
    """n-point Gauss-Legendre rule on [0, 1]."""
    t, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (t + 1.0), 0.5 * w


def lagrange_1d(p: int, t: np.ndarray):
    """Values and derivatives of the p+1 equispaced Lagrange polynomials on [0,1].

    Returns (V, D) with V[a, q] = l_a(t_q), D[a, q] = l_a'(t_q)."""
    nodes = np.arange(p + 1) / p
    t = np.asarray(t, dtype=np.float64)
    V = np.ones((p + 1, t.size))
    D = np.zeros((p + 1, t.size))
    for a in range(p + 1):
        others = [c for c in range(p + 1) if c != a]
        denom = np.prod([nodes[a] - nodes[c] for c in others])
        num = np.ones(t.size)
        for c in others:
            num = num * (t - nodes[c])
        V[a] = num / denom
        d = np.zeros(t.size)
        for skip in others:
            term = np.ones(t.size)
            for c in others:
                if c != skip:
                    term = term * (t - nodes[c])
            d = d + term
        D[a] = d / denom
    return V, D


def reference_1d(p: int):
    """1D stiffness S_ab = int l_a' l_b' and mass M_ab = int l_a l_b on [0,1],
    with p+1 Gauss points (exact for these polynomial degrees)."""
    t, w = gauss_legendre_01(p + 1)
    V, D = lagrange_1d(p, t)
    S = (D * w) @ D.T
    M = (V * w) @ V.T
    return S, M


def reference_stiffness(dim: int, p: int) -> np.ndarray:
    """Laplace stiffness of the unit reference square/cube, x-fastest ordering."""
    S, M = reference_1d(p)
    if dim == 2:
        return np.kron(M, S) + np.kron(S, M)
    return np.kron(np.kron(M, M), S) + np.kron(np.kron(M, S), M) + np.kron(np.kron(S, M), M)


def reference_mass(dim: int, p: int) -> np.ndarray:
    _, M = reference_1d(p)
    return np.kron(M, M) if dim == 2 else np.kron(np.kron(M, M), M)


# ---------------------------------------------------------------- element data
def element_matrices(mesh: StructuredMesh, coef: Optional[np.ndarray] = None,
                     dirichlet: bool = True, kind: str = "stiffness") -> np.ndarray:
    """Element matrices Ke[e] = coef[e] * h^(d-2) * K_ref, Dirichlet folded in.

    ``kind='mass'`` gives the L2-projection mass matrix h^d * M_ref (Sec. 2.1)."""
    ne, npe = mesh.n_elem, mesh.npe
    if kind == "stiffness":
        ref = reference_stiffness(mesh.dim, mesh.p) * mesh.h ** (mesh.dim - 2)
    elif kind == "mass":
        ref = reference_mass(mesh.dim, mesh.p) * mesh.h ** mesh.dim
    else:
        raise ValueError(kind)
    c = np.ones(ne) if coef is None else np.asarray(coef, np.float64)
    Ke = c[:, None, None] * ref[None, :, :]
    if dirichlet:
        dmask = mesh.boundary[mesh.elem_nodes]              # (ne, npe)
        keep = (~dmask).astype(np.float64)
        Ke *= keep[:, :, None]
        Ke *= keep[:, None, :]
        ar = np.arange(npe)
        Ke[:, ar, ar] += dmask / mesh.mult[mesh.elem_nodes]
    return Ke


def load_vector(mesh: StructuredMesh, f: Callable, g_dirichlet: Optional[np.ndarray] = None,
                dirichlet: bool = True) -> np.ndarray:
    """Assembled b_i = int f phi_i with (p+2)^d Gauss points; Dirichlet entries = g (0 default),
    or left as assembled when ``dirichlet`` is False."""
    nq = mesh.p + 2
    t, w = gauss_legendre_01(nq)
    V, _ = lagrange_1d(mesh.p, t)                  # (p+1, nq)
    h, d = mesh.h, mesh.dim
    origin = mesh.node_coords[mesh.elem_nodes[:, 0]]   # (ne, d): lower corner
    if d == 2:
        qx, qy = np.meshgrid(t, t, indexing="xy")
        qx, qy = qx.ravel(), qy.ravel()
        wq = np.outer(w, w).ravel()                 # [iy, ix] -> iy*nq+ix, matches x-fastest
        phi = np.einsum("aq,br->barq", V, V).reshape((mesh.p + 1) ** 2, nq * nq)
        X = origin[:, 0:1] + h * qx[None, :]
        Y = origin[:, 1:2] + h * qy[None, :]
        fq = f(X, Y)
    else:
        qz, qy, qx = np.meshgrid(t, t, t, indexing="ij")
        qx, qy, qz = qx.ravel(), qy.ravel(), qz.ravel()
        wq = np.einsum("i,j,k->ijk", w, w, w).ravel()
        phi = np.einsum("aq,br,cs->cbasrq", V, V, V).reshape((mesh.p + 1) ** 3, nq ** 3)
        X = origin[:, 0:1] + h * qx[None, :]
        Y = origin[:, 1:2] + h * qy[None, :]
        Z = origin[:, 2:3] + h * qz[None, :]
        fq = f(X, Y, Z)
    be = (fq * wq[None, :]) @ phi.T * h ** d          # (ne, npe)
    b = np.bincount(mesh.elem_nodes.ravel(), weights=be.ravel(), minlength=mesh.n_nodes)
    if dirichlet:
        b[mesh.boundary] = 0.0 if g_dirichlet is None else g_dirichlet[mesh.boundary]
    return b


def manufactured_f(x, y, z=None):
    """f = 2 pi^2 sin(pi x) sin(pi y), so that -Laplace u = f for u = sin(pi x) sin(pi y)."""
    return 2.0 * np.pi ** 2 * np.sin(np.pi * x) * np.sin(np.pi * y)


def manufactured_u(coords: np.ndarray) -> np.ndarray:
    return np.sin(np.pi * coords[:, 0]) * np.sin(np.pi * coords[:, 1])


def to_colmajor(Ke: np.ndarray) -> np.ndarray:
    """(n_elem, npe, npe) row/col -> flat per-element column-major float64 array."""
    return np.ascontiguousarray(np.transpose(Ke, (0, 2, 1))).reshape(-1)


def assemble_dense(mesh: StructuredMesh, Ke: np.ndarray) -> np.ndarray:
    """Dense global matrix (tiny meshes only; used by tests as a cross-check)."""
    N = mesh.n_nodes
    A = np.zeros((N, N))
    en = mesh.elem_nodes
    for e in range(mesh.n_elem):
        A[np.ix_(en[e], en[e])] += Ke[e]
    return A


def assemble_csr(mesh: StructuredMesh, Ke: np.ndarray):
    """Global matrix in CSR (rowptr int64, col int32, val float64), sorted columns."""
    import scipy.sparse as sp
    en = mesh.elem_nodes
    npe = mesh.npe
    rows = np.repeat(en, npe, axis=1).ravel()
    cols = np.tile(en, (1, npe)).ravel()
    A = sp.coo_matrix((Ke.reshape(-1), (rows, cols)), shape=(mesh.n_nodes, mesh.n_nodes)).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    return A.indptr.astype(np.int64), A.indices.astype(np.int32), A.data.astype(np.float64)


# ------------------------------------------------------------------ workloads
@dataclass
class Problem:
    """One linear system A x = b, given element by element."""
    name: str
    mesh: StructuredMesh
    Ke: np.ndarray                    # (n_elem, npe, npe)
    b: np.ndarray                     # (n_nodes, nrhs) float64
    coef: Optional[np.ndarray] = None  # per-element coefficient (k_e)
    extra: dict = field(default_factory=dict)

    @property
    def nrhs(self) -> int:
        return int(self.b.shape[1])


def poisson_2d_q1(n: int = 16, seed: int = SEED_BASE + 1) -> Problem:
    """2D Poisson, n x n Q1, k = 1; RHS 0: manufactured load, RHS 1: U[-1,1] per node."""
    rng = np.random.default_rng(seed)
    mesh = structured_mesh((n, n), 1)
    Ke = element_matrices(mesh)
    b0 = load_vector(mesh, manufactured_f)
    b1 = rng.uniform(-1.0, 1.0, mesh.n_nodes)
    return Problem(f"poisson2d_q1_{n}", mesh, Ke, np.stack([b0, b1], axis=1))


def diffusion_2d(n: int, p: int, seed: int, decades: float = 2.0, rhs: str = "manufactured") -> Problem:
    """2D heterogeneous diffusion, k_e = 10^U(-decades, decades) per element."""
    rng = np.random.default_rng(seed)
    mesh = structured_mesh((n, n), p)
    coef = 10.0 ** rng.uniform(-decades, decades, mesh.n_elem)
    Ke = element_matrices(mesh, coef)
    if rhs == "manufactured":
        b = load_vector(mesh, manufactured_f)[:, None]
    else:
        b = rng.uniform(-1.0, 1.0, (mesh.n_nodes, 1))
    return Problem(f"diffusion2d_q{p}_{n}", mesh, Ke, b, coef)


def diffusion_3d_q1(n: int, seed: int, decades: float = 1.0) -> Problem:
    """3D Poisson-type diffusion on n^3 Q1 hexahedra, k_e = 10^U(-1,1), f = 1."""
    rng = np.random.default_rng(seed)
    mesh = structured_mesh((n, n, n), 1)
    coef = 10.0 ** rng.uniform(-decades, decades, mesh.n_elem)
    Ke = element_matrices(mesh, coef)
    b = load_vector(mesh, lambda x, y, z: np.ones_like(x))[:, None]
    return Problem(f"diffusion3d_q1_{n}", mesh, Ke, b, coef)


def l2_field(x, y, z=None):
    """Smooth field projected by the L2-projection workload: exp(x) sin(3 x + 2 y) + x y^2."""
    return np.exp(x) * np.sin(3.0 * x + 2.0 * y) + x * y * y


# sizes of the L2-projection workload, one per order, each near the paper's largest system (3e5 dofs)
L2_SIZES = {1: 512, 2: 256, 3: 180}


def l2_projection(n: int, p: int, f: Callable = l2_field) -> Problem:
    """The paper's model problem (Sec. 2.1): the L2 projection of f onto the Qp space of an n x n
    mesh of the unit square, M u = b with the mass matrix M_ij = int phi_i phi_j (SPD, no boundary
    condition: every node is an unknown) and b_i = int f phi_i."""
    mesh = structured_mesh((n, n), p)
    Ke = element_matrices(mesh, dirichlet=False, kind="mass")
    b = load_vector(mesh, f, dirichlet=False)[:, None]
    return Problem(f"l2proj_q{p}_{n}", mesh, Ke, b)


def batched_poisson_sizes(count: int = 256, lo: int = 32, hi: int = 256, seed: int = SEED_BASE + 3) -> np.ndarray:
    """Mesh sizes n ~ U{lo..hi} for the batch of independent square Q1 meshes."""
    rng = np.random.default_rng(seed)
    return rng.integers(lo, hi + 1, count)


def batched_poisson(sizes, nrhs: int = 4, seed: int = SEED_BASE + 3) -> List[Problem]:
    """Independent 2D Q1 Poisson meshes, k = 1, each with nrhs U[-1,1] right-hand sides."""
    rng = np.random.default_rng(seed + 1000)
    out = []
    for n in sizes:
        mesh = structured_mesh((int(n), int(n)), 1)
        Ke = element_matrices(mesh)
        b = rng.uniform(-1.0, 1.0, (mesh.n_nodes, nrhs))
        out.append(Problem(f"poisson2d_q1_{int(n)}", mesh, Ke, b))
    return out


def adjoint_problem(n: int = 1024, seed: int = SEED_BASE + 5, n_fd: int = 32) -> Problem:
    """2D Q1 diffusion with theta_e ~ N(0,1), k_e = exp(theta_e); loss J = 1/2 |u - u_target|^2.

    u_target = 0.5 sin(2 pi x) cos(pi y) + a seeded sum of 8 smooth Gaussian bumps;
    ``extra['fd_elems']`` holds the n_fd elements for the finite-difference check."""
    rng = np.random.default_rng(seed)
    mesh = structured_mesh((n, n), 1)
    theta = rng.normal(0.0, 1.0, mesh.n_elem)
    coef = np.exp(theta)
    Ke = element_matrices(mesh, coef)
    b = load_vector(mesh, manufactured_f)[:, None]
    x, y = mesh.node_coords[:, 0], mesh.node_coords[:, 1]
    ut = 0.5 * np.sin(2 * np.pi * x) * np.cos(np.pi * y)
    for _ in range(8):
        cx, cy = rng.uniform(0.1, 0.9, 2)
        s = rng.uniform(0.05, 0.2)
        a = rng.uniform(-0.3, 0.3)
        ut = ut + a * np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / (2 * s * s))
    fd = rng.choice(mesh.n_elem, n_fd, replace=False)
    dK = element_matrices(mesh, coef, dirichlet=False)
    keep = (~mesh.boundary[mesh.elem_nodes]).astype(np.float64)
    dK *= keep[:, :, None]
    dK *= keep[:, None, :]
    return Problem(f"adjoint2d_q1_{n}", mesh, Ke, b, coef,
                   extra={"theta": theta, "u_target": ut, "fd_elems": np.sort(fd), "dK": dK})


def convection_2d_q1(n: int = 4, beta=(1.0, 0.5), seed: int = SEED_BASE + 9) -> Problem:
    """Small unsymmetric system: Poisson Q1 plus a Galerkin convection term beta . grad u.

    Used to exercise the transposed (adjoint) solve on a matrix with A != A^T."""
    rng = np.random.default_rng(seed)
    mesh = structured_mesh((n, n), 1)
    t, w = gauss_legendre_01(2)
    V, D = lagrange_1d(1, t)
    # C_ab = int phi_a (beta . grad phi_b) on the unit element, x-fastest local order
    C = np.zeros((4, 4))
    for qy in range(2):
        for qx in range(2):
            wt = w[qx] * w[qy]
            for a in range(4):
                ax, ay = a % 2, a // 2
                pa = V[ax, qx] * V[ay, qy]
                for bb in range(4):
                    bx, by = bb % 2, bb // 2
                    gx = D[bx, qx] * V[by, qy] / mesh.h
                    gy = V[bx, qx] * D[by, qy] / mesh.h
                    C[a, bb] += wt * pa * (beta[0] * gx + beta[1] * gy) * mesh.h ** 2
    Ke = element_matrices(mesh, dirichlet=False) + C[None]
    dmask = mesh.boundary[mesh.elem_nodes]
    keep = (~dmask).astype(np.float64)
    Ke *= keep[:, :, None]
    Ke *= keep[:, None, :]
    ar = np.arange(4)
    Ke[:, ar, ar] += dmask / mesh.mult[mesh.elem_nodes]
    b = rng.uniform(-1.0, 1.0, (mesh.n_nodes, 1))
    return Problem(f"convection2d_q1_{n}", mesh, Ke, b)
