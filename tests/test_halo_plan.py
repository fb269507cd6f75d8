"""The host-side halo plan of a row-partitioned operator (amg_halo_plan; no
GPU), checked against ghost sets computed independently with numpy, and used
for a real distributed product: 2 and 3 gloo ranks on CPU each hold their row
block, receive their ghost values from the owners by point-to-point messages
as the plan prescribes, multiply, and allreduce a dot product -- the paper's
parallel SpMV (Section 2) -- against the global product."""
import os
import socket

import numpy as np
import pytest
import scipy.sparse as sp

import amg_inputs as gen


@pytest.fixture(scope="module")
def amg():
    from paper_1512_04629_gb300 import build

    build.build()
    import paper_1512_04629_gb300 as m

    return m


def _rand_csr(nrows, ncols, density, seed):
    rng = np.random.default_rng(seed)
    M = sp.random(nrows, ncols, density=density, random_state=rng, format="csr")
    M.data[:] = rng.uniform(-1, 1, M.nnz)
    M.sort_indices()
    return M


def _bounds(n, parts, rng=None):
    if rng is None:
        return np.array([p * n // parts for p in range(parts + 1)], dtype=np.int64)
    cuts = np.sort(rng.integers(0, n + 1, parts - 1))
    return np.concatenate([[0], cuts, [n]]).astype(np.int64)


def _reference(M, row0, col0):
    """Ghost sets straight from the definition: block p's ghosts are the
    columns its rows touch outside [col0[p], col0[p+1])."""
    parts = len(row0) - 1
    owner = np.searchsorted(col0, np.arange(M.shape[1]), side="right") - 1
    ghosts, recv = [], np.zeros((parts, parts), dtype=np.int64)
    for p in range(parts):
        cols = M[row0[p]:row0[p + 1]].indices
        g = np.unique(cols[(cols < col0[p]) | (cols >= col0[p + 1])])
        ghosts.append(g)
        for q in owner[g]:
            recv[p, q] += 1
    return ghosts, recv


@pytest.mark.parametrize("case", range(8))
def test_plan_matches_definition(amg, case):
    rng = np.random.default_rng(case)
    nrows, ncols = int(rng.integers(1, 300)), int(rng.integers(1, 300))
    if case % 2 == 0:
        ncols = nrows  # square operators, as A_l
    parts = int(rng.integers(1, 9))
    M = _rand_csr(nrows, ncols, 0.05, case)
    row0, col0 = _bounds(nrows, parts, rng), _bounds(ncols, parts, rng)  # empty blocks included
    cext, goff, gcol, recv = amg.halo_plan(M.indptr, M.indices, ncols, row0, col0)
    ghosts, rrecv = _reference(M, row0, col0)
    np.testing.assert_array_equal(recv, rrecv)
    for p in range(parts):
        np.testing.assert_array_equal(gcol[goff[p]:goff[p + 1]], ghosts[p])
        nloc = col0[p + 1] - col0[p]
        for i in range(row0[p], row0[p + 1]):
            for q in range(M.indptr[i], M.indptr[i + 1]):
                j, c = M.indices[q], cext[q]
                if col0[p] <= j < col0[p + 1]:
                    assert c == j - col0[p]
                else:
                    assert c >= nloc and gcol[goff[p] + c - nloc] == j
    assert np.all(np.diag(recv) == 0)  # a block owns what it does not receive


def test_plan_of_poisson_blocks(amg):
    """2D 5-point Poisson on an N x N grid cut into row blocks of whole grid
    lines: each inner block receives one grid line from each neighbour."""
    N, parts = 24, 4
    A = gen.poisson2d_5pt(N).to_scipy()
    row0 = np.arange(parts + 1, dtype=np.int64) * (N * N // parts)
    _, _, _, recv = amg.halo_plan(A.indptr, A.indices, A.shape[1], row0, row0)
    want = np.zeros((parts, parts), dtype=np.int64)
    for p in range(parts - 1):
        want[p, p + 1] = want[p + 1, p] = N
    np.testing.assert_array_equal(recv, want)


@pytest.mark.parametrize("bad", ["row_end", "col_end", "decreasing", "parts"])
def test_plan_rejects_inconsistent_bounds(amg, bad):
    A = gen.poisson2d_5pt(8).to_scipy()
    n = A.shape[0]
    row0 = np.array([0, 30, n], dtype=np.int64)
    col0 = row0.copy()
    if bad == "row_end":
        row0[-1] = n - 1
    elif bad == "col_end":
        col0[-1] = n + 1
    elif bad == "decreasing":
        row0[1] = n + 5
    if bad == "parts":
        row0 = np.zeros(66, dtype=np.int64)
        row0[-1] = n
        col0 = row0.copy()
    with pytest.raises(amg.AmgError) as e:
        amg.halo_plan(A.indptr, A.indices, n, row0, col0)
    assert e.value.status == amg.ERR_INVALID


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist

    from paper_1512_04629_gb300 import amg as lib

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # every rank knows the operator's shape and the partition; it keeps only
    # its own rows and its own slice of x
    A = gen.fv7_lognormal(12, seed=3).to_scipy()
    n = A.shape[0]
    row0 = np.array([p * n // world for p in range(world + 1)], dtype=np.int64)
    cext, goff, gcol, recv = lib.halo_plan(A.indptr, A.indices, n, row0, row0)
    x = gen.rhs_uniform(n, 9)
    lo, hi = row0[rank], row0[rank + 1]
    x_own = x[lo:hi].copy()
    # messages: block q sends block p the values of p's ghosts that q owns
    reqs = []
    for q in range(world):
        if q == rank:
            continue
        g_q = gcol[goff[q]:goff[q + 1]]
        mine = g_q[(g_q >= lo) & (g_q < hi)]
        if len(mine):
            reqs.append(dist.isend(torch.from_numpy(x_own[mine - lo].copy()), dst=q))
    ghosts = np.zeros(goff[rank + 1] - goff[rank])
    g_me = gcol[goff[rank]:goff[rank + 1]]
    for q in range(world):
        k = recv[rank, q]
        if q == rank or k == 0:
            continue
        buf = torch.zeros(int(k), dtype=torch.float64)
        dist.recv(buf, src=q)
        sel = (g_me >= row0[q]) & (g_me < row0[q + 1])
        ghosts[sel] = buf.numpy()
    for r in reqs:
        r.wait()
    # local product over owned columns and ghosts, in stored order
    nloc = hi - lo
    y = np.zeros(nloc)
    for i in range(lo, hi):
        s = 0.0
        for p in range(A.indptr[i], A.indptr[i + 1]):
            c = cext[p]
            s += A.data[p] * (x_own[c] if c < nloc else ghosts[c - nloc])
        y[i - lo] = s
    # allreduce of the partial dot product x . A x
    d = torch.tensor([float(x_own @ y)], dtype=torch.float64)
    dist.all_reduce(d)
    out[rank] = (y, float(d.item()), int(recv[rank].sum()))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_distributed_spmv_with_the_plan(amg, world):
    import torch.multiprocessing as mp

    port = _free_port()
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    A = gen.fv7_lognormal(12, seed=3).to_scipy()
    x = gen.rhs_uniform(A.shape[0], 9)
    y = A @ x
    got = np.concatenate([res[r][0] for r in range(world)])
    np.testing.assert_allclose(got, y, rtol=1e-14, atol=1e-14 * np.abs(y).max())
    for r in range(world):
        assert abs(res[r][1] - x @ y) <= 1e-12 * abs(x @ y)
    assert all(res[r][2] > 0 for r in range(world))  # every block received ghosts
