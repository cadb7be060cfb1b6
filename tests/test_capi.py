"""C ABI checks that need no GPU: the library loads and exports every symbol
include/mfsolve.h declares; the host analysis agrees with the oracle's
independent symbolic code; bad input returns error codes."""
import ctypes
import os
import re

import numpy as np
import pytest

import fem_inputs as F
import oracle as O
import paper_2306_08994_b300 as M
from paper_2306_08994_b300 import mfsolve as B

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "mfsolve.h")


def _declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mf_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported():
    names = _declared_functions()
    assert len(names) >= 18
    lib = ctypes.CDLL(B.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(B.EXPORTS) == names


def test_strerror_and_defaults():
    lib = B.lib()
    assert lib.mf_strerror(0) == b"ok"
    assert b"pivot" in lib.mf_strerror(-4)
    o = B.default_options()
    assert o.precision == B.MF_F64 and o.max_nrhs == 4


def _mesh(pm):
    return M.Mesh(pm.elem_nodes, pm.n_nodes, pm.dim, grid_dims=pm.nel)


def _oracle_in_class_order(pm):
    s = O.OracleSolver(pm.n_nodes, pm.elem_nodes, O.tree_bisection(pm.nel))
    order = np.lexsort((np.arange(s.n_front), s.height))  # class-major, postorder inside a class
    return s, order


@pytest.mark.parametrize("nel,p", [((16, 16), 1), ((6, 6), 3), ((5, 5), 1), ((4, 4, 4), 1), ((7, 7), 2)])
def test_analysis_matches_oracle_symbolic(nel, p):
    pm = F.structured_mesh(nel, p)
    a = M.Analysis(_mesh(pm))
    ex = a.export()
    s, order = _oracle_in_class_order(pm)
    assert a.n_front == s.n_front
    assert np.array_equal(ex["m"], s.m[order]) and np.array_equal(ex["k"], s.k[order])
    assert np.array_equal(ex["cls"] + 1, s.height[order])
    newid = np.empty(s.n_front, np.int64)
    newid[order] = np.arange(s.n_front)
    par = np.where(s.parent[order] >= 0, newid[np.maximum(s.parent[order], 0)], -1)
    assert np.array_equal(ex["parent"], par)
    for g, v in enumerate(order):
        assert np.array_equal(ex["dofs"][ex["dof_ptr"][g]:ex["dof_ptr"][g + 1]], s.front_dofs(v))
    i = a.info
    assert i["nnz_lu"] == s.nnz_lu and i["sum_cb"] == s.sum_cb and i["n_classes"] == s.n_classes
    assert i["factor_flops"] == s.flops and i["sum_k"] == pm.n_nodes


@pytest.mark.parametrize("name", ["diffusion2d_q3_512", "diffusion3d_q1_64", "poisson2d_q1_1024"])
def test_analysis_full_size_matches_golden(name):
    gold = dict(np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", f"symbolic_{name}.txt"), dtype=str,
                           delimiter="="))
    nel, p = {"diffusion2d_q3_512": ((512, 512), 3), "diffusion3d_q1_64": ((64, 64, 64), 1),
              "poisson2d_q1_1024": ((1024, 1024), 1)}[name]
    pm = F.structured_mesh(nel, p)
    i = M.Analysis(_mesh(pm)).info
    assert i["n_front"] == int(gold["n_front"]) and i["n_classes"] == int(gold["n_classes"])
    assert i["max_m"] == int(gold["max_m"]) and i["root_m"] == int(gold["root_m"])
    assert i["nnz_lu"] == int(gold["nnz_lu"]) and i["sum_cb"] == int(gold["sum_cb"])
    assert i["factor_flops"] == float(gold["flops"])


def test_batch_analysis_is_a_forest_with_aligned_classes():
    meshes = [F.structured_mesh((n, n), 1) for n in (4, 7, 5)]
    a = M.Analysis([_mesh(pm) for pm in meshes])
    ex = a.export()
    assert a.n_dof == sum(pm.n_nodes for pm in meshes)
    assert (ex["parent"] < 0).sum() == 3
    singles = [M.Analysis(_mesh(pm)).export() for pm in meshes]
    for c in range(ex["cls"].max() + 1):
        assert (ex["cls"] == c).sum() == sum((s["cls"] == c).sum() for s in singles)
    assert ex["k"].sum() == a.n_dof


def test_centroid_bisection_equals_box_bisection_on_power_of_two_grid():
    pm = F.structured_mesh((8, 8), 1)
    a1 = M.Analysis(_mesh(pm)).export()
    a2 = M.Analysis(M.Mesh(pm.elem_nodes, pm.n_nodes, 2, centroids=pm.elem_centroids())).export()
    for key in ("m", "k", "cls", "parent", "dofs"):
        assert np.array_equal(a1[key], a2[key])


def test_bad_inputs_return_error_codes():
    lib = B.lib()
    h = ctypes.c_void_p()
    assert lib.mf_analyze_mesh(None, None, ctypes.byref(h)) == B.MF_EINVAL
    pm = F.structured_mesh((4, 4), 1)
    bad = pm.elem_nodes.copy()
    bad[0, 0] = pm.n_nodes + 5
    with pytest.raises(M.MFError) as e:
        M.Analysis(M.Mesh(bad, pm.n_nodes, 2, grid_dims=pm.nel))
    assert e.value.code == B.MF_EINVAL
    with pytest.raises(M.MFError):
        M.Analysis(M.Mesh(pm.elem_nodes, pm.n_nodes, 2, grid_dims=(3, 4)))
    assert lib.mf_analysis_info(None, None) == B.MF_EINVAL
    assert lib.mf_factor(None, None, None) == B.MF_EINVAL
    assert lib.mf_solve(None, None, 1, None) == B.MF_EINVAL
    assert lib.mf_status(None, None) == B.MF_EINVAL
