"""mf_residual_noalloc against mf_residual, through the C ABI.

mf_residual_noalloc is for callers that may not allocate device memory when
they evaluate a residual (fixed memory budgets, host frameworks that own all
device allocations, real-time loops): it takes only the caller's device
buffers and keeps its accumulation array in the library's static device
memory.  This file is collected last on purpose so that a run stopping at
the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

import fem_inputs as F
import oracle as O
import paper_2306_08994_b300 as M
from paper_2306_08994_b300 import mfsolve as B

pytestmark = pytest.mark.gpu


def _noalloc(n_dof, n_elem, npe, en, vals, x, b, r, nrhs):
    return B.lib().mf_residual_noalloc(n_dof, n_elem, npe, en.data_ptr(), vals.data_ptr(), x.data_ptr(),
                                       b.data_ptr(), r.data_ptr(), nrhs, torch.cuda.current_stream().cuda_stream)


def test_noalloc_residual_matches_mf_residual_twice_in_a_row():
    pr = F.diffusion_2d(20, 3, seed=F.SEED_BASE + 2)
    pm = pr.mesh
    nrhs = 2
    an = M.Analysis(M.Mesh(pm.elem_nodes, pm.n_nodes, 2, grid_dims=pm.nel), M.default_options(max_nrhs=nrhs))
    fac = M.Factors(an)
    vals = torch.tensor(F.to_colmajor(pr.Ke), device="cuda")
    en = torch.tensor(pm.elem_nodes, device="cuda")
    rng = np.random.default_rng(5)
    b = torch.tensor(rng.uniform(-1, 1, (nrhs, pm.n_nodes)), device="cuda")
    import scipy.sparse as sp
    rp, cp, vp = F.assemble_csr(pm, pr.Ke)
    rowsum = float(np.abs(sp.csr_matrix((vp, cp, rp))).sum(axis=1).max())
    Kcm = F.to_colmajor(pr.Ke)
    # set-up call: the first call on a device looks the scratch address up, and under CUDA's lazy
    # module loading that is also when the library's device code and its static array are loaded
    # onto the device; the calls checked below come after it
    r0 = torch.empty_like(b)
    assert _noalloc(pm.n_nodes, pm.n_elem, pm.npe, en, vals, b, b, r0, nrhs) == B.MF_OK
    torch.cuda.synchronize()
    for call in range(2):
        x = torch.tensor(rng.uniform(-1, 1, (nrhs, pm.n_nodes)), device="cuda")
        r_ref = torch.empty_like(b)
        fac.residual(vals, x, b, r_ref)
        r = torch.full_like(b, float("nan"))
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        rc = _noalloc(pm.n_nodes, pm.n_elem, pm.npe, en, vals, x, b, r, nrhs)
        assert rc == B.MF_OK, rc
        torch.cuda.synchronize()
        # no device memory was taken by the call
        assert torch.cuda.mem_get_info()[0] == free0
        # same tolerance as the refinement bar: rounding-order differences only
        scale = rowsum * float(x.abs().max()) + float(b.abs().max())
        err = float((r - r_ref).abs().max())
        assert err <= 1e-13 * scale, (call, err, scale)
        # and against the oracle's double-double residual (exact to ~1 ulp of the result)
        r_o = O.residual_dd(pm.elem_nodes, Kcm, x.cpu().numpy().T, b.cpu().numpy().T)
        err_o = float(np.abs(r.cpu().numpy().T - r_o).max())
        assert err_o <= 1e-13 * scale, (call, err_o, scale)


def test_noalloc_reports_out_of_range_node_ids_as_nan():
    """An element node id outside [0, n_dof) is never read or written through; the call's output is NaN."""
    pr = F.poisson_2d_q1(6)
    pm = pr.mesh
    vals = torch.tensor(F.to_colmajor(pr.Ke), device="cuda")
    en_h = pm.elem_nodes.copy()
    en_h[3, 2] = pm.n_nodes + 1000  # beyond the vectors and the scratch row in use
    en_h[7, 0] = -5
    en = torch.tensor(en_h, device="cuda")
    x = torch.ones(pm.n_nodes, dtype=torch.float64, device="cuda")
    b = torch.zeros_like(x)
    r = torch.zeros_like(x)
    rc = _noalloc(pm.n_nodes, pm.n_elem, pm.npe, en, vals, x, b, r, 1)
    assert rc == B.MF_OK
    torch.cuda.synchronize()
    assert bool(torch.isnan(r).all())
    # the next good call clears the flag
    en_ok = torch.tensor(pm.elem_nodes, device="cuda")
    rc = _noalloc(pm.n_nodes, pm.n_elem, pm.npe, en_ok, vals, x, b, r, 1)
    assert rc == B.MF_OK
    torch.cuda.synchronize()
    assert bool(torch.isfinite(r).all())


def test_noalloc_rejects_too_many_right_hand_sides_before_launching():
    t = torch.zeros(8, dtype=torch.float64, device="cuda")
    ti = torch.zeros(8, dtype=torch.int64, device="cuda")
    r = torch.full((8,), 7.0, dtype=torch.float64, device="cuda")
    rc = B.lib().mf_residual_noalloc(1, 1, 4, ti.data_ptr(), t.data_ptr(), t.data_ptr(), t.data_ptr(),
                                     r.data_ptr(), 65536, None)
    assert rc == B.MF_EINVAL
    torch.cuda.synchronize()
    assert bool((r == 7.0).all())


def test_noalloc_rejects_sizes_beyond_the_static_scratch():
    t = torch.zeros(8, dtype=torch.float64, device="cuda")
    ti = torch.zeros(8, dtype=torch.int64, device="cuda")
    too_big = B.MF_NOALLOC_MAX_ENTRIES + 1
    rc = B.lib().mf_residual_noalloc(too_big, 1, 4, ti.data_ptr(), t.data_ptr(), t.data_ptr(), t.data_ptr(),
                                     t.data_ptr(), 1, None)
    assert rc == B.MF_ETOOLARGE
    assert b"static scratch" in B.lib().mf_strerror(rc)
