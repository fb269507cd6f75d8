"""Multi-right-hand-side solves, the serving loop and save/load on the GPU."""
import os
import time

import numpy as np
import pytest

import amg_inputs as gen
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def amg():
    from paper_1512_04629_gb300 import build

    build.build()
    import paper_1512_04629_gb300 as m

    return m


@pytest.mark.parametrize("k", [1, 5, 8, 13, 32, 64])
@pytest.mark.parametrize("prec", [0, 1])
def test_solve_batch_columns(amg, k, prec):
    A = gen.poisson3d_7pt(17)
    h = amg.Hierarchy.setup(A, gamma=[0.0, 0.1], precision=prec)
    ref = oracle.Hierarchy(A)
    ref.sparsify([0.0, 0.1])
    B = np.stack([gen.rhs_uniform(A.n, 100 + c) for c in range(k)], axis=1)
    if k > 3:
        B[:, 3] = 0.0  # an empty column converges at once
    X, infos = h.solve_batch(B, tol=1e-8)
    S = A.to_scipy()
    for c in range(k):
        if not B[:, c].any():
            assert infos[c].iterations == 0 and not X[:, c].any()
            continue
        assert infos[c].status == 0, infos[c].as_dict()
        r = B[:, c] - S @ X[:, c]
        assert np.linalg.norm(r) <= 1e-8 * np.linalg.norm(B[:, c]) * (1 + 1e-6)
        xr, ir = ref.pcg(B[:, c], tol=1e-8)
        assert abs(infos[c].iterations - ir.iterations) <= (1 if prec == 0 else 3)
        assert np.linalg.norm(X[:, c] - xr) <= 1e-6 * np.linalg.norm(xr)


def test_solve_batch_device_buffers(amg):
    A = gen.fv7_lognormal(14, seed=3)
    h = amg.Hierarchy.setup(A, gamma=[0.0, 0.1], precision=1)
    B = torch.from_numpy(np.stack([gen.rhs_uniform(A.n, c) for c in range(8)], axis=1)).cuda()
    X, infos = h.solve_batch(B, tol=1e-8)
    Xh = X.cpu().numpy()
    S = A.to_scipy()
    for c in range(8):
        b = B[:, c].cpu().numpy()
        assert np.linalg.norm(b - S @ Xh[:, c]) <= 1e-8 * np.linalg.norm(b) * (1 + 1e-6)


def test_column_result_independent_of_batch(amg):
    """A right-hand side gives bit-identical x whichever column it occupies
    and whatever the other columns hold."""
    A = gen.poisson3d_7pt(15)
    h = amg.Hierarchy.setup(A, gamma=[0.0, 0.1], precision=1)
    b = gen.rhs_uniform(A.n, 7)
    B1 = np.zeros((A.n, 32))
    B1[:, 0] = b
    B2 = np.stack([gen.rhs_uniform(A.n, 200 + c) for c in range(32)], axis=1)
    B2[:, 21] = b
    X1, i1 = h.solve_batch(B1)
    X2, i2 = h.solve_batch(B2)
    assert i1[0].iterations == i2[21].iterations
    np.testing.assert_array_equal(X1[:, 0], X2[:, 21])


def test_save_load_roundtrip(amg, tmp_path):
    A = gen.poisson3d_7pt(16)
    h = amg.Hierarchy.setup(A, gamma=[0.0, 0.1])
    p = str(tmp_path / "h.amgh")
    h.save(p)
    g = amg.Hierarchy.load(p)
    assert g.num_levels == h.num_levels
    for l in range(h.num_levels):
        for which in ["A", "Ahat"]:
            a, b = h.export(l, which), g.export(l, which)
            np.testing.assert_array_equal(a.col, b.col)
            np.testing.assert_array_equal(a.val, b.val)
        assert g.level_stats(l)["gamma"] == h.level_stats(l)["gamma"]
    b = gen.rhs_uniform(A.n, 3)
    x1, i1 = h.solve(b)
    x2, i2 = g.solve(b)
    assert i1.iterations == i2.iterations
    np.testing.assert_allclose(x1, x2, rtol=1e-13, atol=1e-13)
    with open(p, "r+b") as f:
        f.truncate(100)
    with pytest.raises(amg.AmgError):
        amg.Hierarchy.load(p)


def _hier(amg, kind, N):
    A = gen.generate(kind, N)
    return A, amg.Hierarchy.setup(A, gamma=[0.0, 0.1], precision=1)


def test_server_results_alone_and_in_the_mix(amg):
    A1, h1 = _hier(amg, "2d5", 40)
    A2, h2 = _hier(amg, "3d7", 14)
    srv = amg.Server(max_batch=8)
    id1, id2 = srv.register(h1), srv.register(h2)
    b = gen.rhs_uniform(A1.n, 42)
    t = srv.submit(id1, b)
    st, x_alone, info_alone = srv.wait(t, id1)
    assert st == 0 and info_alone.final_relres <= 1e-8
    tickets = []
    for r in range(30):
        hid, A = (id1, A1) if r % 2 == 0 else (id2, A2)
        tickets.append((srv.submit(hid, gen.rhs_uniform(A.n, 1000 + r)), hid, A, r))
        if r == 11:
            tickets.append((srv.submit(id1, b), id1, A1, -1))
    for t, hid, A, r in tickets:
        st, x, info = srv.wait(t, hid)
        assert st == 0, info.as_dict()
        bb = b if r < 0 else gen.rhs_uniform(A.n, 1000 + r)
        assert np.linalg.norm(bb - A.to_scipy() @ x) <= 1e-8 * np.linalg.norm(bb) * (1 + 1e-6)
        if r < 0:
            np.testing.assert_array_equal(x, x_alone)
            assert info.iterations == info_alone.iterations
    srv.close()


def test_server_memory_budget_queues_instead_of_failing(amg):
    A1, h1 = _hier(amg, "2d5", 48)
    A2, h2 = _hier(amg, "2d5", 50)
    # room for about one batch workspace at a time
    one = 8 * A2.n * 8 * 4 * 2 + 7 * 8 * A2.n * 8
    srv = amg.Server(max_batch=8, hbm_budget=int(one * 1.3))
    ids = [srv.register(h1), srv.register(h2)]
    ts = [(srv.submit(ids[r % 2], gen.rhs_uniform((A1 if r % 2 == 0 else A2).n, r)), r) for r in range(12)]
    for t, r in ts:
        st, x, info = srv.wait(t, ids[r % 2])
        assert st == 0
    srv.close()


def test_server_rejects_and_times_out(amg):
    A, h = _hier(amg, "3d7", 20)
    srv = amg.Server(max_batch=8, max_queue=2)
    hid = srv.register(h)
    sts = [srv.try_submit(hid, gen.rhs_uniform(A.n, r))[0] for r in range(50)]
    assert 8 in sts  # AMG_REJECTED once the queue is full
    st, t = srv.try_submit(hid, gen.rhs_uniform(A.n, 999))
    while st == 8:
        time.sleep(0.01)
        st, t = srv.try_submit(hid, gen.rhs_uniform(A.n, 999))
    st0, _, _ = srv.wait(t, hid, timeout_ms=0)
    assert st0 in (0, 7)  # 7 = AMG_TIMEOUT while the request is still running
    st, x, info = srv.wait(t, hid, timeout_ms=60000)
    assert st == 0
    with pytest.raises(amg.AmgError):
        srv.submit(hid, np.full(A.n, np.nan))
    with pytest.raises(amg.AmgError):
        srv.submit(57, gen.rhs_uniform(A.n, 1))
    srv.close()


def _serve(amg, hs, reqs, **opts):
    """Submit every (hierarchy index, b) of `reqs`, then wait them in order."""
    srv = amg.Server(max_batch=8, **opts)
    ids = [srv.register(h) for h in hs]
    ts = [srv.submit(ids[i], b) for i, b in reqs]
    out = [srv.wait(t, ids[i]) for t, (i, _) in zip(ts, reqs)]
    srv.close()
    return out


@pytest.mark.parametrize("stage", ["tight", "none"])
def test_server_staging_paths_agree(amg, stage):
    """Requests staged on the device (submit uploads, wait downloads) and
    through the worker's host buffer give the same bits; a staging budget
    that holds only a few vectors mixes the two paths."""
    A1, h1 = _hier(amg, "2d5", 40)
    A2, h2 = _hier(amg, "3d7", 14)
    reqs = [(r % 2, gen.rhs_uniform((A1 if r % 2 == 0 else A2).n, 500 + r)) for r in range(24)]
    ref = _serve(amg, [h1, h2], reqs)
    budget = 3 * 8 * max(A1.n, A2.n) if stage == "tight" else -1
    got = _serve(amg, [h1, h2], reqs, stage_budget=budget)
    for (st0, x0, i0), (st1, x1, i1), (i, b) in zip(ref, got, reqs):
        assert st0 == 0 and st1 == 0
        np.testing.assert_array_equal(x1, x0)
        assert i1.iterations == i0.iterations and i1.final_relres == i0.final_relres
        A = A1 if i == 0 else A2
        assert np.linalg.norm(b - A.to_scipy() @ x1) <= 1e-8 * np.linalg.norm(b) * (1 + 1e-6)


def test_server_submit_copies_b_and_close_frees_unwaited(amg):
    A, h = _hier(amg, "2d5", 40)
    srv = amg.Server(max_batch=8)
    hid = srv.register(h)
    b = gen.rhs_uniform(A.n, 7)
    keep = b.copy()
    t = srv.submit(hid, b)
    b[:] = np.nan  # the caller's buffer is free once submit returns
    st, x, info = srv.wait(t, hid)
    assert st == 0
    assert np.linalg.norm(keep - A.to_scipy() @ x) <= 1e-8 * np.linalg.norm(keep) * (1 + 1e-6)
    for r in range(12):  # results never waited for are freed by close
        srv.submit(hid, gen.rhs_uniform(A.n, 60 + r))
    srv.close()
    srv2 = amg.Server(max_batch=8, stage_budget=1 << 20)
    hid2 = srv2.register(h)
    st, x2, _ = srv2.wait(srv2.submit(hid2, keep), hid2)
    assert st == 0
    np.testing.assert_array_equal(x2, x)
    srv2.close()
    with pytest.raises(amg.AmgError):
        amg.Server(stage_budget=-2)
