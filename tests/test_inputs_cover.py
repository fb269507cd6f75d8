"""The hub-graph input covers what its parity cases are there for.

The setup's sparse products sort their rows by product count into bins: up
to 128 products (register sorts and small tables), 129..512, 513..4096 and
more than 4096.  Rows of more than 128 products are first accumulated in a
hash table sized for 128 distinct columns; a row with more goes on to its
bin's larger table.  This checks, on the oracle's own hierarchy and with
plain scipy products, that ``amg_inputs.hub_graphs`` has, in A_0 P_0 or in
P_0^T (A_0 P_0), rows in each of the three upper bins with more than 128
distinct columns, and rows of more than 4096 products with 128 or fewer --
so that the GPU parity cases on it run every fallback.
"""
import numpy as np

import amg_inputs as gen
import oracle


def _sp(M):
    import scipy.sparse as sp

    return sp.csr_matrix((M.val, M.col, M.rowptr), shape=(M.nrows, M.ncols))


def _products(X, Y):
    lens = np.diff(Y.indptr)
    out = np.zeros(X.shape[0], dtype=np.int64)
    rows = np.repeat(np.arange(X.shape[0]), np.diff(X.indptr))
    np.add.at(out, rows, lens[X.indices])
    return out


def test_hub_graphs_cover_every_table_fallback():
    A = gen.hub_graphs()
    h = oracle.Hierarchy(A)
    A0, P0 = _sp(h.matrix(0, "A")), _sp(h.matrix(0, "P"))
    AP = A0 @ P0
    prods, distinct = [], []
    for X, Y in ((A0, P0), (P0.T.tocsr(), AP)):
        prods.append(_products(X, Y))
        distinct.append(np.diff((X @ Y).tocsr().indptr))
    p, d = np.concatenate(prods), np.concatenate(distinct)
    for lo, hi in ((128, 512), (512, 4096), (4096, None)):
        in_bin = (p > lo) & ((p <= hi) if hi else True)
        assert (in_bin & (d > 128)).any(), (lo, hi)
    assert ((p > 4096) & (d <= 128)).any()
