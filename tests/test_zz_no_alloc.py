"""amg_residual_noalloc: the residual entry point that allocates nothing.

It serves callers that cannot allocate device memory when they call: code
whose device memory comes only from its own pool (a framework or real-time
loop), or a process whose memory budget is fully committed.  Its output is
checked against the existing entry point amg_solve, whose info.final_relres
is ||b - A x|| / ||b||, on two calls in a row (the shared scratch must be
reusable).  This file is collected last so a failure here cannot hide the
other tests.
"""
import ctypes as C

import numpy as np
import pytest

import amg_inputs as gen

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amg():
    from paper_1512_04629_gb300 import build

    build.build()
    import paper_1512_04629_gb300 as m

    return m


def _call(amg, h, b, x, r, nrm):
    lib = amg.lib()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    ptr = lambda t: C.c_void_p(t.data_ptr())
    return lib.amg_residual_noalloc(h.handle, ptr(b), ptr(x), ptr(r), ptr(nrm), stream)


def test_residual_noalloc_matches_solve_on_two_calls(amg):
    A = gen.poisson3d_7pt(30)  # n = 27,000: several scratch blocks and a ragged last one
    h = amg.Hierarchy.setup(A, gamma=[0.0, 0.1])
    b = torch.from_numpy(gen.rhs_uniform(A.n, 1)).cuda()
    x, info = h.solve(b, tol=1e-8)
    assert info.status == 0
    r = torch.full_like(b, np.nan)
    nrm = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
    r0 = torch.full_like(b, np.nan)
    nb = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
    zero = torch.zeros_like(b)
    for _ in range(2):
        assert _call(amg, h, b, zero, r0, nb) == 0
        assert _call(amg, h, b, x, r, nrm) == 0
        torch.cuda.synchronize()
        bnorm = float(nb.item())
        assert torch.equal(r0, b)  # b - A 0 = b exactly
        assert abs(bnorm - float(torch.linalg.norm(b))) <= 1e-12 * bnorm
        # the existing entry point reported ||b - A x|| / ||b|| for the same x
        assert abs(float(nrm.item()) / bnorm - info.final_relres) <= 1e-12
        # r is the residual vector: its norm is rnorm
        assert abs(float(torch.linalg.norm(r)) - float(nrm.item())) <= 1e-12 * bnorm
    first = (r.clone(), nrm.clone())
    assert _call(amg, h, b, x, r, nrm) == 0
    torch.cuda.synchronize()
    assert torch.equal(r, first[0]) and torch.equal(nrm, first[1])


def test_residual_noalloc_rejects_host_pointers(amg):
    A = gen.poisson2d_5pt(16)
    h = amg.Hierarchy.setup(A)
    lib = amg.lib()
    bh = np.ones(A.n)
    xh = np.zeros(A.n)
    rh = np.zeros(A.n)
    nh = np.zeros(1)
    st = lib.amg_residual_noalloc(h.handle, bh.ctypes.data_as(C.c_void_p), xh.ctypes.data_as(C.c_void_p),
                                  rh.ctypes.data_as(C.c_void_p), nh.ctypes.data_as(C.c_void_p), None)
    assert st == 1
    assert b"device memory of the hierarchy's device" in lib.amg_last_error()

