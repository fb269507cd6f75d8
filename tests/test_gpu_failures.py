"""Failure paths exercised from the host: no GPU fault, trap or hang.

* Out of memory: amg_debug_fail_allocation makes one chosen device
  allocation fail on the host, before CUDA is asked.  Setup is swept over
  every allocation it makes; the solve paths that allocate (GMRES basis,
  batched workspace, Algorithm 5's checkpoint) and the server's staging and
  admission are hit too.  Each failure must surface as AMG_ERR_OOM (or, in
  the server, as a fallback that still gives the right answer), release what
  was allocated, and leave the library usable: the next call's results are
  bit-identical to a run that never failed.
* Server wait limit: a limit of 1 ms runs out on an ordinary batch
  iteration (several ms on a 2M-row problem), so every request ends with
  AMG_TIMEOUT, later submits are refused with AMG_TIMEOUT, and a new server
  works normally.
"""
import gc
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


@pytest.fixture(autouse=True)
def _disarm(amg):
    yield
    amg.debug_fail_allocation(-1)


def test_setup_survives_every_injected_allocation_failure(amg):
    A = gen.poisson2d_5pt(40)
    b = gen.rhs_uniform(A.n, 1)
    gam = [0.0, 0.1]
    x_ref, i_ref = amg.Hierarchy.setup(A, gamma=gam).solve(b, tol=1e-8)
    gc.collect()  # hierarchies that earlier tests left in reference cycles are freed now, not mid-sweep
    torch.cuda.synchronize()
    base = amg.device_bytes()
    failures = 0
    for k in range(5000):
        amg.debug_fail_allocation(k)
        try:
            h = amg.Hierarchy.setup(A, gamma=gam)
        except amg.AmgError as e:
            assert e.status == amg.ERR_OOM, str(e)
            assert "injected" in str(e)
            failures += 1
            torch.cuda.synchronize()
            assert amg.device_bytes() == base, k  # nothing held after the failure
            continue
        amg.debug_fail_allocation(-1)
        break
    else:
        pytest.fail("setup never completed")
    assert failures >= 20  # the sweep reached deep into the setup
    x, info = h.solve(b, tol=1e-8)
    assert info.status == 0 and info.iterations == i_ref.iterations
    np.testing.assert_array_equal(x, x_ref)


@pytest.mark.parametrize("path", ["gmres", "batch", "adaptive"])
def test_solve_paths_report_oom_and_recover(amg, path):
    A = gen.poisson3d_7pt(20)
    b = gen.rhs_uniform(A.n, 2)
    kw = dict(krylov=amg.KRYLOV_GMRES) if path == "gmres" else {}
    gam = [0.0, 1.0] if path == "adaptive" else [0.0, 0.1]

    def run(h):
        if path == "batch":
            B = np.stack([b, gen.rhs_uniform(A.n, 3)], axis=1)
            X, infos = h.solve_batch(B, tol=1e-8)
            return X, infos[0]
        return h.solve(b, tol=1e-8, adaptive=(path == "adaptive"))

    x_ref, i_ref = run(amg.Hierarchy.setup(A, gamma=gam, **kw))
    h = amg.Hierarchy.setup(A, gamma=gam, **kw)
    failures = 0
    for k in range(200):
        amg.debug_fail_allocation(k)
        try:
            x, info = run(h)
        except amg.AmgError as e:
            assert e.status == amg.ERR_OOM, str(e)
            failures += 1
            if path == "adaptive":  # the failed solve may have reintroduced entries: start over
                h.sparsify(gam)
            continue
        amg.debug_fail_allocation(-1)
        break
    assert failures >= 1
    assert info.status == 0 and info.iterations == i_ref.iterations
    np.testing.assert_array_equal(x, x_ref)


def test_server_injected_failures_fall_back_and_keep_results(amg):
    """A failed staging allocation sends the request through host memory; a
    failed batch-workspace allocation re-queues the admitted requests until
    memory is there.  Results are the same bits as without failures."""
    A = gen.poisson3d_7pt(16)
    h = amg.Hierarchy.setup(A, gamma=[0.0, 0.1], precision=1)
    bs = [gen.rhs_uniform(A.n, 40 + i) for i in range(6)]
    srv = amg.Server(max_batch=8)
    hid = srv.register(h)
    ref = [srv.wait(srv.submit(hid, b), hid)[1] for b in bs]
    srv.close()
    for k in range(0, 12):
        srv = amg.Server(max_batch=8)
        hid = srv.register(h)
        amg.debug_fail_allocation(k)
        tickets = [srv.submit(hid, b) for b in bs]
        for t, want in zip(tickets, ref):
            st, x, info = srv.wait(t, hid)
            assert st == 0, (k, info.status)
            np.testing.assert_array_equal(x, want)
        srv.close()
        amg.debug_fail_allocation(-1)


def test_server_wait_limit_times_out_every_request(amg):
    A = gen.poisson3d_7pt(128)
    h = amg.Hierarchy.setup(A, gamma=[0.0, 0.1], precision=1)
    bs = [gen.rhs_uniform(A.n, 60 + i) for i in range(4)]
    srv = amg.Server(max_batch=32, wait_limit_ms=1)
    hid = srv.register(h)
    tickets = [srv.submit(hid, b) for b in bs]
    for t in tickets:
        st, _, info = srv.wait(t, hid, timeout_ms=60000)
        assert st == amg.TIMEOUT and info.status == amg.TIMEOUT
        assert b"wait limit" in amg.lib().amg_last_error()
    st, _ = srv.try_submit(hid, bs[0])
    assert st == amg.TIMEOUT
    srv.close()
    # the library and the hierarchy stay usable
    srv = amg.Server(max_batch=32)
    hid = srv.register(h)
    st, x, info = srv.wait(srv.submit(hid, bs[0]), hid)
    assert st == 0 and info.final_relres <= 1e-8
    srv.close()
