"""Error paths driven from the host, through the C ABI, without faulting the GPU.

* Every device allocation of mf_factors_create is made to fail in turn
  (mf_test_fail_alloc): the call returns MF_ENOMEM, releases what it had
  allocated, and a later create on the same analysis succeeds.
* A bounded device wait that nothing releases (mf_test_bounded_wait: one CTA
  at the substitution sweep's grid barrier, waiting for a CTA that is never
  launched) gives up after its limit; mf_status returns MF_ETIMEOUT, and the
  handle factors and solves correctly afterwards.
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


def _problem():
    pr = F.diffusion_2d(10, 3, seed=F.SEED_BASE + 2)
    pm = pr.mesh
    return pr, M.Mesh(pm.elem_nodes, pm.n_nodes, 2, grid_dims=pm.nel)


@pytest.mark.parametrize("prec", ["f64", "tf32"])
def test_every_allocation_failure_of_factors_create_returns_enomem(prec):
    pr, mesh = _problem()
    an = M.Analysis(mesh, M.default_options(precision=prec, small_front_max=32, tc_min_cb=16))
    L = B.lib()
    opts = an.options
    # warm-up create/free so the context's lazy allocations are not counted below
    M.Factors(an, opts)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failed = 0
    try:
        for n in range(500):
            L.mf_test_fail_alloc(n)
            h = ctypes.c_void_p()
            rc = L.mf_factors_create(an._h, ctypes.byref(opts), ctypes.byref(h))
            if rc == B.MF_OK:
                L.mf_free_factors(h)
                break
            assert rc == B.MF_ENOMEM, (n, rc)
            assert not h.value
            failed += 1
        else:
            pytest.fail("mf_factors_create never succeeded")
    finally:
        L.mf_test_fail_alloc(-1)
    assert failed >= 20  # arenas, maps, plan lists, work vectors: every one was made to fail
    torch.cuda.synchronize()
    # nothing leaked: what the failed calls allocated was released
    assert abs(torch.cuda.mem_get_info()[0] - free0) <= (4 << 20)
    # and the library still works
    f = M.Factors(an, opts)
    vals = torch.tensor(F.to_colmajor(pr.Ke), device="cuda")
    b = torch.tensor(pr.b[:, 0], device="cuda")
    x = torch.empty_like(b)
    f.factor(vals)
    info = f.refine_solve(vals, b, x, tol=1e-14, maxit=20)
    assert info["backward_error"] <= 1e-14


def test_bounded_wait_times_out_and_the_handle_stays_usable():
    pr = F.poisson_2d_q1(16)
    pm = pr.mesh
    mesh = M.Mesh(pm.elem_nodes, pm.n_nodes, 2, grid_dims=pm.nel)
    an = M.Analysis(mesh, M.default_options(precision="f64", small_front_max=32))
    f = M.Factors(an)
    vals = torch.tensor(F.to_colmajor(pr.Ke), device="cuda")
    b = torch.tensor(pr.b[:, 0], device="cuda")
    f.factor(vals)
    assert f.status()["rc"] == B.MF_OK
    stream = torch.cuda.current_stream().cuda_stream
    assert B.lib().mf_test_bounded_wait(f._h, 20.0, stream) == B.MF_OK
    st = f.status()  # synchronises: the wait has given up by now
    assert st["rc"] == B.MF_ETIMEOUT and st["timeout"] == 1
    assert B.lib().mf_test_bounded_wait(f._h, 0.0, stream) == B.MF_EINVAL
    # the context and the handle are intact: factor again (clears the status) and solve
    f.factor(vals)
    x = b.clone()
    f.solve(x)
    assert f.status()["rc"] == B.MF_OK
    s = O.OracleSolver(pm.n_nodes, pm.elem_nodes, O.tree_bisection(pm.nel))
    s.factor(F.to_colmajor(pr.Ke))
    xo = s.solve(pr.b[:, 0])
    assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-10 * np.linalg.norm(xo)
