"""Pins of the CPU oracle against facts outside the oracle itself.

Every check here compares the oracle with a closed form, a textbook special
case, dense brute force on tiny inputs, the paper's Example 1, or a published
test vector -- never with a retyped copy of the oracle's own formula.
"""
import json
import os
from fractions import Fraction as Fr

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import amg_inputs as gen
import oracle
from conftest import GOLDEN


# ---------------------------------------------------------------------------
# helpers (test-only inputs)
# ---------------------------------------------------------------------------
def csr_from_dense(M):
    S = sp.csr_matrix(M)
    S.sort_indices()
    return S


def pattern(M):
    """Dense boolean structural pattern (stored entries, zeros included)."""
    S = M.to_scipy() if hasattr(M, "to_scipy") else M
    out = np.zeros(S.shape, dtype=bool)
    rows = np.repeat(np.arange(S.shape[0]), np.diff(S.indptr))
    out[rows, S.indices] = True
    return out


def laplace1d(n):
    return csr_from_dense(2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1))


def aniso2d(N, eps):
    """5-point stencil with -1 couplings in x and -eps in y (diag 2 + 2 eps)."""
    Ix = sp.identity(N)
    T = sp.diags([-1.0, 2.0, -1.0], [-1, 0, 1], shape=(N, N))
    A = sp.kron(Ix, T) + eps * sp.kron(T, Ix)
    A = sp.csr_matrix(A)
    A.sort_indices()
    return A


# ---------------------------------------------------------------------------
# generators: closed-form spectra (SpMV and assembly pins)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("N", [5, 9, 12])
def test_poisson2d_eigenvalues(N):
    A = gen.poisson2d_5pt(N).to_scipy().toarray()
    k = np.arange(1, N + 1)
    s = 4 * np.sin(k * np.pi / (2 * (N + 1))) ** 2
    lam = np.sort((s[:, None] + s[None, :]).ravel())
    np.testing.assert_allclose(np.linalg.eigvalsh(A), lam, rtol=0, atol=1e-12)


@pytest.mark.parametrize("N", [4, 6])
def test_poisson3d_eigenvalues(N):
    A = gen.poisson3d_7pt(N).to_scipy().toarray()
    k = np.arange(1, N + 1)
    s = 4 * np.sin(k * np.pi / (2 * (N + 1))) ** 2
    lam = np.sort((s[:, None, None] + s[None, :, None] + s[None, None, :]).ravel())
    np.testing.assert_allclose(np.linalg.eigvalsh(A), lam, rtol=0, atol=1e-12)


def test_generators_structure():
    for A in [gen.poisson2d_5pt(7), gen.poisson3d_7pt(5), gen.poisson3d_27pt(4),
              gen.fv7_lognormal(5, seed=3), gen.q1_laplace3d(4), gen.hub_graphs()]:
        S = A.to_scipy()
        assert abs(S - S.T).max() < 1e-15
        for i in range(A.n):
            cols = A.col[A.rowptr[i]:A.rowptr[i + 1]]
            assert np.all(np.diff(cols) > 0) and i in cols
        rs = np.asarray(S.sum(axis=1)).ravel()
        assert rs.min() > -1e-12 * abs(S).max()
    # nnz formulas of the 2D / 3D stencils
    N = 11
    assert gen.poisson2d_5pt(N).nnz == 5 * N * N - 4 * N
    assert gen.poisson3d_7pt(N).nnz == 7 * N ** 3 - 6 * N ** 2
    assert gen.poisson3d_27pt(4).nnz == (3 * 4 - 2) ** 3
    # hub graphs: 2 (50*100 + 130*140) bipartite, 2 (2*39*40 + 320) and
    # 2 (2*23*24 + 192) grid and hub off-diagonals, plus the diagonal
    assert gen.hub_graphs().nnz == 2 * (5000 + 18200 + 3120 + 320 + 1104 + 192) + 2598


def test_spmv_matches_dense():
    A = gen.fv7_lognormal(6, seed=3)
    x = gen.rhs_uniform(A.n, 5)
    np.testing.assert_allclose(oracle.spmv(A, x), A.to_scipy().toarray() @ x, rtol=1e-14, atol=1e-12)


def test_splitmix64_published_vectors():
    ref = json.load(open(os.path.join(GOLDEN, "splitmix64_vectors.json")))
    G = 0x9E3779B97F4A7C15
    keys = np.array([(t * G) % 2 ** 64 for t in range(3)], dtype=np.uint64)
    got = [format(int(v), "016x") for v in gen.splitmix64(keys)]
    assert got == ref["seed0_outputs_hex"]
    # the oracle's own SplitMix64 (PMIS weights): key t*G with seed 0, level 0
    for t, h in enumerate(ref["seed0_outputs_hex"]):
        key = (t * G) % 2 ** 64
        u = oracle.uniform_weight(key, 0, 0)
        assert u == (int(h, 16) >> 11) * 2.0 ** -53


# ---------------------------------------------------------------------------
# strength of connection
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("eps,expect_y", [(0.1, False), (0.2499, False), (0.25, True), (0.5, True)])
def test_strength_anisotropic(eps, expect_y):
    """Classical rule: y-couplings (-eps) are strong iff eps >= theta * 1."""
    N = 6
    A = aniso2d(N, eps)
    s = oracle.strength(A, 0.25)
    for i in range(A.shape[0]):
        for p in range(A.indptr[i], A.indptr[i + 1]):
            j = A.indices[p]
            if j == i:
                assert s[p] == 0
            elif abs(j - i) == 1:
                assert s[p] == 1
            else:
                assert s[p] == int(expect_y)


def test_strength_positive_and_weak_rows():
    M = np.array([[4.0, 1.0, -2.0, -0.4],
                  [1.0, 3.0, 0.5, 0.0],
                  [-2.0, 0.5, 5.0, -1.0],
                  [-0.4, 0.0, -1.0, 2.0]])
    A = csr_from_dense(M)
    s = oracle.strength(A, 0.25)
    got = {(i, A.indices[p]) for i in range(4) for p in range(A.indptr[i], A.indptr[i + 1]) if s[p]}
    # row 0: max neg 2 -> threshold 0.5: -2 strong, -0.4 weak, +1 never
    # row 1: no negative coupling -> nothing strong
    # row 2: max neg 2 -> 0.5: -2 and -1 strong
    # row 3: max neg 1 -> 0.25: -0.4 and -1 strong
    assert got == {(0, 2), (2, 0), (2, 3), (3, 0), (3, 2)}


# ---------------------------------------------------------------------------
# PMIS: equals the sequential greedy by decreasing (w, i)
# ---------------------------------------------------------------------------
def greedy_reference(A, strong, weights):
    """Independent formulation: visit points by decreasing (w_i, i); a point that
    is not initially F becomes C unless a C point already chosen lies in S_i."""
    n = A.shape[0]
    S = [set() for _ in range(n)]
    ST_count = np.zeros(n, dtype=int)
    for i in range(n):
        for p in range(A.indptr[i], A.indptr[i + 1]):
            if strong[p]:
                S[i].add(A.indices[p])
                ST_count[A.indices[p]] += 1
    w = ST_count + weights
    order = sorted(range(n), key=lambda i: (w[i], i), reverse=True)
    cf = np.zeros(n, dtype=np.int8)
    for i in order:
        if ST_count[i] == 0:
            cf[i] = -1
        elif any(cf[c] == 1 for c in S[i]):
            cf[i] = -1
        else:
            cf[i] = 1
    return cf


@pytest.mark.parametrize("case", ["2d", "3d", "aniso", "fv", "random"])
def test_pmis_equals_greedy(case):
    rng = np.random.default_rng(7)
    if case == "2d":
        A = gen.poisson2d_5pt(12).to_scipy()
    elif case == "3d":
        A = gen.poisson3d_7pt(6).to_scipy()
    elif case == "aniso":
        A = aniso2d(10, 0.1)
    elif case == "fv":
        A = gen.fv7_lognormal(6, seed=3).to_scipy()
    else:
        n = 80
        M = np.zeros((n, n))
        for _ in range(250):
            i, j = rng.integers(0, n, 2)
            if i != j:
                v = -rng.uniform(0.05, 1.0)
                M[i, j] = M[j, i] = v
        M += np.diag(-M.sum(axis=1) + 0.1)
        A = csr_from_dense(M)
    A.sort_indices()
    for seed, level in [(0, 0), (12345, 3)]:
        s = oracle.strength(A, 0.25)
        cf = oracle.pmis(A, s, seed, level)
        u = np.array([oracle.uniform_weight(seed, level, i) for i in range(A.shape[0])])
        assert np.array_equal(cf, greedy_reference(A, s, u))
        assert set(np.unique(cf)) <= {-1, 1}


def test_pmis_f_points_depend_on_c():
    A = gen.poisson3d_7pt(8).to_scipy()
    s = oracle.strength(A, 0.25)
    cf = oracle.pmis(A, s, 0, 0)
    for i in range(A.shape[0]):
        if cf[i] == -1:
            nbrs = [A.indices[p] for p in range(A.indptr[i], A.indptr[i + 1]) if s[p]]
            assert any(cf[j] == 1 for j in nbrs)
    assert 0 < (cf == 1).sum() < A.shape[0]


# ---------------------------------------------------------------------------
# direct interpolation
# ---------------------------------------------------------------------------
def test_direct_interp_1d_textbook():
    """1D Laplacian: an F point between two C points interpolates linearly
    (1/2, 1/2); with one C neighbour and one F neighbour it copies (weight 1);
    a boundary F point next to a C point gets 1/2."""
    n = 9
    A = laplace1d(n)
    s = oracle.strength(A, 0.25)
    cf = np.array([-1, 1, -1, 1, -1, -1, 1, -1, 1], dtype=np.int8)
    P = oracle.direct_interp(A, s, cf).todense()
    cidx = np.cumsum(cf == 1) - 1
    expect = np.zeros((n, 4))
    for i in range(n):
        if cf[i] == 1:
            expect[i, cidx[i]] = 1.0
    expect[0, 0] = 0.5
    expect[2, 0] = expect[2, 1] = 0.5
    expect[4, 1] = 1.0
    expect[5, 2] = 1.0
    expect[7, 2] = expect[7, 3] = 0.5
    np.testing.assert_array_equal(P, expect)


@pytest.mark.parametrize("which", ["2d", "3d", "fv"])
def test_direct_interp_preserves_constants(which):
    A = {"2d": lambda: gen.poisson2d_5pt(10), "3d": lambda: gen.poisson3d_7pt(6),
         "fv": lambda: gen.fv7_lognormal(6, seed=3)}[which]().to_scipy()
    s = oracle.strength(A, 0.25)
    cf = oracle.pmis(A, s, 0, 0)
    P = oracle.direct_interp(A, s, cf).to_scipy()
    ones = P @ np.ones(P.shape[1])
    rs = np.asarray(A.sum(axis=1)).ravel()
    for i in range(A.shape[0]):
        if cf[i] == 1:
            assert ones[i] == 1.0 and P.indptr[i + 1] - P.indptr[i] == 1
        elif abs(rs[i]) <= 1e-12 * A[i, i] and P.indptr[i + 1] > P.indptr[i]:
            assert abs(ones[i] - 1.0) <= 1e-14
        else:
            assert ones[i] <= 1.0 + 1e-14
    assert P.shape[1] == (cf == 1).sum()


# A 6 x 6 SPD (strictly diagonally dominant) matrix with positive couplings.
# Points 1, 2, 3 are C (coarse columns 0, 1, 2); 0, 4, 5 are F.
_POS6 = [
    [Fr(5), Fr(-2), Fr(-1), Fr(1, 2), Fr(-1), Fr(1, 4)],
    [Fr(-2), Fr(6), Fr(0), Fr(-1), Fr(0), Fr(0)],
    [Fr(-1), Fr(0), Fr(4), Fr(0), Fr(-1), Fr(0)],
    [Fr(1, 2), Fr(-1), Fr(0), Fr(3), Fr(0), Fr(-1)],
    [Fr(-1), Fr(0), Fr(-1), Fr(0), Fr(4), Fr(1, 2)],
    [Fr(1, 4), Fr(0), Fr(0), Fr(-1), Fr(1, 2), Fr(3)],
]
_POS6_CF = np.array([-1, 1, 1, 1, -1, -1], dtype=np.int8)


def _pos6():
    D = np.array([[float(v) for v in row] for row in _POS6])
    S = sp.csr_matrix(D)
    S.sort_indices()
    return S


def _assert_weights(P, expect):
    """P (oracle) against exact fractions, to a couple of ulps."""
    Pd = P.todense()
    want = np.zeros(Pd.shape)
    for (i, j), w in expect.items():
        want[i, j] = float(w)
    assert np.array_equal(Pd != 0, want != 0), (Pd, want)
    np.testing.assert_allclose(Pd, want, rtol=4e-16, atol=0)


def test_direct_interp_positive_couplings_lumped_to_diagonal():
    """Direct interpolation (Section 2; Stueben's sign split) when the F row
    has positive off-diagonals but no strong positive C neighbour -- the case
    every hierarchy meets, since the classical strength rule never marks a
    positive coupling strong.  The positive sum then joins the diagonal:
    row 0: alpha = (-2 - 1 - 1) / (-2 - 1) = 4/3, a_00 -> 5 + 1/2 + 1/4 = 23/4,
           w = -alpha a_0j / (23/4): 32/69 (C 1), 16/69 (C 2);
    row 4: alpha = -2 / -1 = 2, a_44 -> 4 + 1/2 = 9/2, w_42 = 4/9;
    row 5: alpha = 1, a_55 -> 3 + 3/4 = 15/4, w_53 = 4/15.
    A dropped fallback (a_ii unchanged) gives 8/15, 1/2 and 1/3 instead."""
    A = _pos6()
    s = oracle.strength(A, 0.25)
    # the strength rule marks exactly the negative couplings above theta
    dense_s = np.zeros((6, 6), dtype=bool)
    rows = np.repeat(np.arange(6), np.diff(A.indptr))
    dense_s[rows, A.indices] = s.astype(bool)
    assert not dense_s[A.toarray() > 0].any()
    assert dense_s[0, 1] and dense_s[0, 2] and dense_s[0, 4] and not dense_s[0, 3]
    P = oracle.direct_interp(A, s, _POS6_CF)
    _assert_weights(P, {(0, 0): Fr(32, 69), (0, 1): Fr(16, 69), (1, 0): 1, (2, 1): 1, (3, 2): 1,
                        (4, 1): Fr(4, 9), (5, 2): Fr(4, 15)})
    # closed form: with the positive sum lumped, sum_j w_ij = -sum a_ik^- / (a_ii + sum a_ik^+)
    rowsum = P.todense().sum(axis=1)
    np.testing.assert_allclose(rowsum[[0, 4, 5]], [16 / 23, 4 / 9, 4 / 15], rtol=4e-16)


def test_direct_interp_positive_couplings_beta_branch():
    """The beta branch of direct interpolation, reached when a strong
    positive C neighbour exists (here a_03 = +1/2 is marked strong by hand;
    orc_direct_interp takes any strength flags):
    alpha = (-4) / (-3) = 4/3, beta = (1/2 + 1/4) / (1/2) = 3/2, a_00 = 5,
    w_01 = 8/15, w_02 = 4/15, w_03 = -beta a_03 / a_00 = -3/20.
    Closed form: the weights then sum to -sum_{k != i} a_ik / a_ii
    = 1 - 7/4 / 5 = 13/20.  A beta over all positive couplings (rather than
    the C ones) would give 1 and w_03 = -1/10."""
    A = _pos6()
    s = oracle.strength(A, 0.25).copy()
    p03 = A.indptr[0] + int(np.where(A.indices[A.indptr[0]:A.indptr[1]] == 3)[0][0])
    s[p03] = 1
    P = oracle.direct_interp(A, s, _POS6_CF)
    _assert_weights(P, {(0, 0): Fr(8, 15), (0, 1): Fr(4, 15), (0, 2): Fr(-3, 20), (1, 0): 1, (2, 1): 1,
                        (3, 2): 1, (4, 1): Fr(4, 9), (5, 2): Fr(4, 15)})
    assert abs(P.todense()[0].sum() - 13 / 20) <= 4e-16


# ---------------------------------------------------------------------------
# Galerkin product
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("which", ["2d8", "2d16", "3d6", "fv5"])
def test_galerkin_matches_dense(which):
    A = {"2d8": lambda: gen.poisson2d_5pt(8), "2d16": lambda: gen.poisson2d_5pt(16),
         "3d6": lambda: gen.poisson3d_7pt(6), "fv5": lambda: gen.fv7_lognormal(5, seed=3)}[which]()
    h = oracle.Hierarchy(A, max_size=10, max_levels=3)
    for l in range(h.num_levels - 1):
        Al = h.matrix(l, "A").todense()
        P = h.matrix(l, "P").todense()
        Ac = h.matrix(l + 1, "A").todense()
        ref = P.T @ Al @ P
        scale = np.abs(ref).max()
        np.testing.assert_allclose(Ac, ref, rtol=0, atol=1e-14 * scale)
        np.testing.assert_allclose(Ac, Ac.T, rtol=0, atol=1e-14 * scale)
        # row sums of A_c equal P^T (A P 1)
        np.testing.assert_allclose(Ac.sum(axis=1), P.T @ (Al @ (P @ np.ones(P.shape[1]))),
                                   rtol=0, atol=1e-13 * scale)
        # structural pattern: every product creates an entry
        pp = pattern(h.matrix(l, "P")).astype(int)
        patt = (pp.T @ pattern(h.matrix(l, "A")).astype(int) @ pp) > 0
        assert np.array_equal(pattern(h.matrix(l + 1, "A")), patt)


def test_spgemm_rectangular_dense():
    rng = np.random.default_rng(3)
    Ad = rng.standard_normal((9, 7)) * (rng.random((9, 7)) < 0.3)
    Bd = rng.standard_normal((7, 5)) * (rng.random((7, 5)) < 0.4)
    C = oracle.spgemm(csr_from_dense(Ad), csr_from_dense(Bd))
    np.testing.assert_allclose(C.todense(), Ad @ Bd, rtol=1e-15, atol=1e-15)
    np.testing.assert_array_equal(oracle.transpose(csr_from_dense(Ad)).todense(), Ad.T)


def test_table1_density_growth():
    """Table 1 shape: nnz per row rises on the coarse levels of a 3D 7-point
    Poisson hierarchy before the last level."""
    t1 = json.load(open(os.path.join(GOLDEN, "table1_hierarchy.json")))
    dens_paper = [lv["nnz"] / lv["n"] for lv in t1["levels"]]
    assert max(dens_paper) > 5 * dens_paper[0]
    h = oracle.Hierarchy(gen.poisson3d_7pt(40))
    dens = [nnz / n for (n, nnz, _) in h.level_sizes()]
    assert abs(dens[0] - 7 * (1 - 6 / 7 / 40)) < 1e-9
    assert max(dens[1:]) > 3 * dens[0]
    assert dens[1] > dens[0] and dens[2] > dens[1]


# ---------------------------------------------------------------------------
# minimal pattern M and sparsify (Algorithm 3 / 3b)
# ---------------------------------------------------------------------------
def _level_pair(A, l=0, max_levels=4):
    h = oracle.Hierarchy(A, max_size=20, max_levels=max_levels)
    return h


def test_minimal_pattern_brute_force():
    A = gen.poisson3d_7pt(7)
    h = _level_pair(A)
    for l in range(h.num_levels - 1):
        Al = h.matrix(l, "A").todense()
        P = h.matrix(l, "P").todense()
        cf = h.cf(l)
        Phat = np.zeros_like(P)
        Phat[np.where(cf == 1)[0], np.arange(P.shape[1])] = 1.0
        pa = pattern(h.matrix(l, "A")).astype(int)
        pp = pattern(h.matrix(l, "P")).astype(int)
        ph = (Phat > 0).astype(int)
        M = ((ph.T @ pa @ pp) + (pp.T @ pa @ ph)) > 0
        Acs = h.matrix(l + 1, "A").to_scipy()
        inM = h.inM(l + 1)
        rows = np.repeat(np.arange(Acs.shape[0]), np.diff(Acs.indptr))
        assert np.array_equal(inM.astype(bool), M[rows, Acs.indices])
        # M lies inside the Galerkin pattern
        assert M.sum() == inM.sum()


def _dense_sparsify_reference(Ac, inM, gamma):
    """Brute force over a dense copy: N from the drop test and M, mirrored;
    dropped entries summed into the diagonal."""
    D = Ac.toarray()
    n = D.shape[0]
    stored = np.zeros_like(D, dtype=bool)
    rows = np.repeat(np.arange(n), np.diff(Ac.indptr))
    stored[rows, Ac.indices] = True
    Mset = np.zeros_like(stored)
    Mset[rows, Ac.indices] = inM.astype(bool)
    off = stored & ~np.eye(n, dtype=bool)
    rowmax = np.where(off, np.abs(D), 0).max(axis=1)
    passes = off & (Mset | (np.abs(D) >= gamma * rowmax[:, None]))
    N = passes | passes.T
    keep = N | np.eye(n, dtype=bool)
    keep &= stored
    H = np.where(keep, D, 0.0)
    dropped = np.where(stored & ~keep, D, 0.0)
    H[np.arange(n), np.arange(n)] += dropped.sum(axis=1)
    return H, keep[rows, Ac.indices]


@pytest.mark.parametrize("gamma", [0.0, 0.01, 0.1, 0.5, 1.0])
def test_sparsify_against_dense(gamma):
    h = _level_pair(gen.poisson3d_7pt(8))
    for l in range(1, h.num_levels):
        Ac = h.matrix(l, "A").to_scipy()
        inM = h.inM(l)
        H, keep = oracle.sparsify_diag(Ac, inM, gamma)
        Href, keep_ref = _dense_sparsify_reference(Ac, inM, gamma)
        np.testing.assert_array_equal(keep, keep_ref.astype(np.uint8))
        scale = np.abs(Href).max()
        np.testing.assert_allclose(H.todense(), Href, rtol=0, atol=1e-14 * scale)
        if gamma == 0.0:
            assert keep.all()
            np.testing.assert_array_equal(H.todense(), Ac.toarray())


def test_sparsify_gamma_one_keeps_only_M_and_row_maxima():
    """gamma = 1: only M, the row maxima and their mirrors survive (Section 2.1
    uses 1.0 as 'everything outside M')."""
    h = _level_pair(gen.poisson3d_7pt(8))
    for l in range(1, h.num_levels):
        Ac = h.matrix(l, "A").to_scipy()
        D = Ac.toarray()
        inM = h.inM(l)
        _, keep = oracle.sparsify_diag(Ac, inM, 1.0)
        n = D.shape[0]
        allowed = np.zeros_like(D, dtype=bool)
        rows = np.repeat(np.arange(n), np.diff(Ac.indptr))
        allowed[rows[inM == 1], Ac.indices[inM == 1]] = True
        offd = D - np.diag(np.diag(D))
        stored = np.zeros_like(allowed)
        stored[rows, Ac.indices] = True
        rmax = np.where(stored & ~np.eye(n, dtype=bool), np.abs(offd), 0).max(axis=1)
        allowed |= stored & (np.abs(offd) == rmax[:, None]) & (rmax[:, None] > 0)
        allowed |= allowed.T
        allowed |= np.eye(n, dtype=bool)
        assert np.array_equal(keep.astype(bool), allowed[rows, Ac.indices])


@pytest.mark.parametrize("gamma", [0.01, 0.1, 1.0])
def test_theorem1_spd_and_rowsums(gamma):
    """Theorem 1 and its Remark: diagonal lumping keeps symmetry, row sums and
    (semi-)definiteness; with a strictly dominant row the result is PD."""
    h = _level_pair(gen.poisson3d_7pt(10), max_levels=5)
    for l in range(1, h.num_levels):
        Ac = h.matrix(l, "A").to_scipy()
        H, keep = oracle.sparsify_diag(Ac, h.inM(l), gamma)
        Hd = H.todense()
        Ad = Ac.toarray()
        scale = np.abs(Ad).max()
        np.testing.assert_allclose(Hd, Hd.T, rtol=0, atol=1e-14 * scale)
        np.testing.assert_allclose(Hd.sum(axis=1), Ad.sum(axis=1), rtol=0, atol=1e-13 * scale)
        # N symmetric: kept pattern symmetric
        Kp = (np.abs(Hd) > 0) | np.eye(Hd.shape[0], dtype=bool)
        assert np.array_equal(Kp, Kp.T)
        lam_min = np.linalg.eigvalsh(Hd).min()
        dd_in = np.all(2 * np.abs(np.diag(Ad)) >= np.abs(Ad).sum(axis=1) - 1e-12 * scale)
        if dd_in:
            assert lam_min > -1e-12 * scale
            assert np.all(2 * np.abs(np.diag(Hd)) >= np.abs(Hd).sum(axis=1) - 1e-12 * scale)
        strict = np.any(2 * np.abs(np.diag(Ad)) > np.abs(Ad).sum(axis=1) + 1e-9 * scale)
        if dd_in and strict:
            assert lam_min > 0


def test_sparsify_ismax_guard():
    """gamma > 1 with a zero-row-sum row: its largest entries are kept, mirrored."""
    M = np.array([[3.0, -2.0, -1.0, 0.0],
                  [-2.0, 4.0, -1.0, -1.0],
                  [-1.0, -1.0, 3.0, -1.0],
                  [0.0, -1.0, -1.0, 2.5]])
    Ac = csr_from_dense(M)
    inM = np.zeros(Ac.nnz, dtype=np.uint8)
    H, keep = oracle.sparsify_diag(Ac, inM, 2.0)
    Hd = H.todense()
    # rows 0,1,2 have zero sums -> keep their maxima (0,1),(1,0) [row 1 max 2],
    # row 2 ties at 1 -> (2,0),(2,1),(2,3) and mirrors; row 3 (sum 0.5) lumps all
    kept = {(i, j) for i in range(4) for j in range(4) if i != j and Hd[i, j] != 0}
    assert kept == {(0, 1), (1, 0), (2, 0), (0, 2), (2, 1), (1, 2), (2, 3), (3, 2)}
    np.testing.assert_allclose(Hd.sum(axis=1), M.sum(axis=1), atol=1e-15)


def test_reintroduce_to_zero_restores_galerkin():
    A = gen.poisson3d_7pt(10)
    h = oracle.Hierarchy(A, max_size=20)
    L = h.num_levels
    h.sparsify([0.0] + [1.0] * (L - 1))
    assert any(h.matrix(l, "Ahat").nnz < h.matrix(l, "A").nnz for l in range(1, L))
    for _ in range(10 * L):
        cnt, _ = h.reintroduce(s=1)
        if cnt == 0:
            break
    for l in range(L):
        assert h.gamma(l) == 0.0
        np.testing.assert_array_equal(h.matrix(l, "Ahat").val, h.matrix(l, "A").val)
        assert h.keep(l).all()


# ---------------------------------------------------------------------------
# Algorithm 5 drop-tolerance schedule: Example 1 exactly
# ---------------------------------------------------------------------------
def test_example1_gamma_schedule():
    ex = json.load(open(os.path.join(GOLDEN, "example1_gamma_schedule.json")))
    seq = ex["sequence"]
    g = np.array([0.0] * ex["levels_offset"] + seq[0])  # level 0 is never sparsified
    for want in seq[1:]:
        g, changed = oracle.gamma_schedule(g, ex["s"], ex["gamma_min"])
        np.testing.assert_allclose(g[ex["levels_offset"]:], want, rtol=1e-12, atol=0)
        assert changed.sum() == ex["s"]
    g0 = np.zeros(5)
    g1, ch = oracle.gamma_schedule(g0, 2, 0.01)
    assert not ch.any() and not g1.any()


# ---------------------------------------------------------------------------
# V-cycle and PCG
# ---------------------------------------------------------------------------
def test_cholesky_matches_library():
    A = gen.poisson2d_5pt(6).to_scipy().toarray()
    L = oracle.cholesky(A)
    np.testing.assert_allclose(np.tril(L), np.linalg.cholesky(A), rtol=1e-13, atol=1e-14)
    b = gen.rhs_uniform(A.shape[0], 2)
    np.testing.assert_allclose(oracle.chol_solve(L, b), sla.solve(A, b), rtol=1e-12)


def test_single_level_is_exact_solve():
    A = gen.poisson2d_5pt(8)
    h = oracle.Hierarchy(A, max_size=1000)
    assert h.num_levels == 1
    b = gen.rhs_uniform(A.n, 0)
    np.testing.assert_allclose(h.vcycle(b), sla.solve(A.to_scipy().toarray(), b), rtol=1e-12)
    x, info = h.pcg(b)
    assert info.iterations == 1 and info.status == 0


def _dense_two_grid(Ad, P, Acoarse_hat, Ahat0, b):
    """Two-level V(1,1) written densely: x = D^-1 b; coarse correction; post-relax."""
    d = np.abs(Ahat0).sum(axis=1)
    x = b / d
    r = b - Ahat0 @ x
    xc = np.linalg.solve(Acoarse_hat, P.T @ r)
    x = x + P @ xc
    return x + (b - Ahat0 @ x) / d


def test_two_level_vcycle_dense():
    A = gen.poisson2d_5pt(10)
    h = oracle.Hierarchy(A, max_size=40, max_levels=2)
    assert h.num_levels == 2
    h.sparsify([0.0, 0.1])
    b = gen.rhs_uniform(A.n, 3)
    ref = _dense_two_grid(A.to_scipy().toarray(), h.matrix(0, "P").todense(),
                          h.matrix(1, "Ahat").todense(), A.to_scipy().toarray(), b)
    np.testing.assert_allclose(h.vcycle(b), ref, rtol=1e-12, atol=1e-13)


@pytest.mark.parametrize("gamma", [0.0, 0.1, 1.0])
def test_vcycle_symmetric_linear_and_contracting(gamma):
    A = gen.poisson3d_7pt(9)
    h = oracle.Hierarchy(A, max_size=30)
    h.sparsify([0.0, gamma])
    n = A.n
    y = gen.rhs_uniform(n, 11)
    z = gen.rhs_uniform(n, 12)
    My, Mz = h.vcycle(y), h.vcycle(z)
    assert abs(y @ Mz - z @ My) <= 1e-12 * abs(y @ My)
    np.testing.assert_allclose(h.vcycle(2 * y - 3 * z), 2 * My - 3 * Mz, rtol=1e-12, atol=1e-12)
    # M is positive definite (PCG needs it; Theorem 1 keeps each Ahat_l SPD)
    for seed in range(14, 18):
        v = gen.rhs_uniform(n, seed)
        assert v @ h.vcycle(v) > 0
    if gamma == 0.0:
        # Galerkin: the error propagation I - M A contracts (power iteration)
        S = A.to_scipy()
        e = gen.rhs_uniform(n, 13)
        for _ in range(30):
            e = e - h.vcycle(S @ e)
            nrm = np.linalg.norm(e)
            e /= nrm
        assert nrm < 1.0


def test_pcg_solution_matches_direct():
    A = gen.poisson2d_5pt(64)
    b = gen.rhs_uniform(A.n, 0)
    h = oracle.Hierarchy(A)
    x, info = h.pcg(b, tol=1e-8)
    assert info.status == 0 and info.final_relres <= 1e-8
    S = A.to_scipy().tocsc()
    xs = spla.spsolve(S, b)
    lam = np.linalg.eigvalsh(A.to_scipy().toarray())
    kappa = lam[-1] / lam[0]
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) <= kappa * 1e-8
    assert 0 < info.conv_factor < 1


def test_pcg_zero_rhs():
    A = gen.poisson2d_5pt(16)
    h = oracle.Hierarchy(A)
    x, info = h.pcg(np.zeros(A.n))
    assert info.iterations == 0 and not x.any()


def test_adaptive_recovers_and_is_noop_for_galerkin():
    A = gen.poisson3d_7pt(24)
    b = gen.rhs_uniform(A.n, 1)
    h = oracle.Hierarchy(A)
    xg, ig = h.pcg(b)
    h2 = oracle.Hierarchy(A)
    xa, ia = h2.adaptive_solve(b, rho_max=0.5)
    assert ia.resets == 0 and ia.iterations == ig.iterations
    h3 = oracle.Hierarchy(A)
    h3.sparsify([0.0, 1.0])
    x1, i1 = h3.pcg(b)
    h4 = oracle.Hierarchy(A)
    h4.sparsify([0.0, 1.0])
    x4, i4 = h4.adaptive_solve(b, rho_max=0.2, s=1)
    assert i4.status == 0 and i4.final_relres <= 1e-8
    assert i4.resets >= 1
    assert h4.gamma(1) < 1.0


# ---------------------------------------------------------------------------
# Algorithm 5's control, restated with dense linear algebra
# ---------------------------------------------------------------------------
def _shifted_poisson2d(N, sigma):
    """2D 5-point Poisson with sigma taken off the diagonal: symmetric with a
    positive diagonal, indefinite once sigma passes the smallest eigenvalue
    -- the input on which CG's residual really grows."""
    A = gen.poisson2d_5pt(N)
    A.val = A.val.copy()
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    A.val[A.col == rows] -= sigma
    return A


def _vcycle_operator(A, gammas, max_size):
    """The V-cycle of the oracle hierarchy sparsified with `gammas`, as a
    dense matrix (the cycle is linear in its right-hand side)."""
    h = oracle.Hierarchy(A, max_size=max_size)
    h.sparsify(gammas)
    M = np.empty((A.n, A.n))
    for j in range(A.n):
        e = np.zeros(A.n)
        e[j] = 1.0
        M[:, j] = h.vcycle(e)
    return M, h.num_levels


def _alg5_dense(A, b, gammas, k, s, rho_max, divf, max_size, tol=1e-8, max_it=300, gamma_min=0.01):
    """Algorithm 5 (Section 6) from its steps: PCG is run k steps at a time;
    after each window the true residual gives the factor
    (||r_end|| / ||r_start||)^(1/k); above rho_max (or on a breakdown, or a
    growth beyond divf) the finest levels with gamma > 0 get gamma / 10
    (0 below gamma_min) on s levels and PCG restarts -- from the window's
    starting x when the residual grew.  Returns (x, status, windows, its,
    resets) with windows = [(steps, action, factor)]."""
    Ad = A.to_scipy().toarray()
    _, L = _vcycle_operator(A, [0.0], max_size)
    g = [0.0] + [gammas[min(l, len(gammas) - 1)] for l in range(1, L)]
    M, _ = _vcycle_operator(A, g, max_size)
    bn = np.linalg.norm(b)
    x = np.zeros(A.n)

    def start(x):
        r = b - Ad @ x
        z = M @ r
        return r, z.copy(), r @ z

    r, p, rho = start(x)
    rstart, total, resets, windows, status = bn, 0, 0, [], oracle.NOT_CONVERGED
    while total < max_it:
        xs = x.copy()
        steps, taken, conv, brk = min(k, max_it - total), 0, False, False
        conv = np.linalg.norm(r) <= tol * bn
        while not conv and taken < steps:
            q = Ad @ p
            pq = p @ q
            taken += 1
            if not (pq > 0 and rho > 0):
                brk = True
                break
            a = rho / pq
            x = x + a * p
            r = r - a * q
            if np.linalg.norm(r) <= tol * bn:
                t = b - Ad @ x
                if np.linalg.norm(t) <= tol * bn:
                    conv = True
                    break
                r = t
            z = M @ r
            rho_new = r @ z
            p = z + (rho_new / rho) * p
            rho = rho_new
        total += taken
        rend = np.linalg.norm(b - Ad @ x)
        factor = (rend / rstart) ** (1.0 / taken) if taken else 1.0
        if conv or rend <= tol * bn:
            windows.append((taken, "converged", factor))
            status = oracle.OK
            break
        growing = divf > 0 and not (rend <= divf * rstart)
        action = "continue"
        if factor > rho_max or brk or growing:
            lstart = next((l for l in range(1, L) if g[l] > 0), None)
            changed = 0
            if lstart is not None:
                for l in range(lstart, min(lstart + s, L)):
                    g[l] = g[l] / 10 if g[l] / 10 >= gamma_min * (1 - 1e-12) else 0.0
                    changed += 1
            back = not (rend <= rstart)
            if changed == 0 and brk:
                windows.append((taken, "breakdown_back" if back else "breakdown_stop", factor))
                x = xs if back else x
                status = oracle.BREAKDOWN
                break
            if changed == 0 and growing:
                windows.append((taken, "diverged", factor))
                x, status = xs, oracle.DIVERGED
                break
            if changed:
                resets += 1
                M, _ = _vcycle_operator(A, g, max_size)
                action = "restart_back" if back else "restart_here"
                if back:
                    x, rend = xs, rstart
                r, p, rho = start(x)
            else:
                action = "nothing_left"
        windows.append((taken, action, factor))
        rstart = rend
    return x, status, windows, total, resets


_ALG5_CASES = {
    # SPD: restarts from the current x, windows that go on, nothing left
    "q27_restarts": (lambda: gen.poisson3d_27pt(7), [0.0, 1.0], 1, 1, 0.1, 1e3, 20),
    "aniso_slow": (lambda: gen.rotated_aniso_q1(20), [0.0, 0.1, 1.0], 3, 1, 0.3, 1e3, 20),
    "aniso_s2": (lambda: gen.rotated_aniso_q1(20), [0.0, 0.1, 1.0], 2, 2, 0.5, 1e3, 20),
    # indefinite: restarts from the window's start, final breakdowns
    "shift_back": (lambda: _shifted_poisson2d(16, 0.2), [0.0, 1.0], 1, 1, 0.5, 0.0, 20),
    "shift_breakdown_back": (lambda: _shifted_poisson2d(24, 0.2), [0.0, 0.0], 2, 1, 0.5, 0.0, 20),
    "shift_restarts_back": (lambda: _shifted_poisson2d(24, 0.2), [0.0, 1.0], 2, 1, 0.5, 0.0, 20),
    # growth with nothing left to reintroduce: diverged
    "shift_diverged": (lambda: _shifted_poisson2d(16, 0.065), [0.0, 0.0], 1, 1, 0.5, 1.0, 20),
}


@pytest.mark.parametrize("case", sorted(_ALG5_CASES))
def test_adaptive_trace_matches_dense_restatement(case):
    """The oracle's Algorithm 5 against the dense restatement above, window by
    window: the steps of each window, the action taken (continue, restart
    from the current or the window's x, nothing left, converged, breakdown,
    diverged), the window factor, and the final x, iterations and resets."""
    make, gam, k, s, rho_max, divf, ms = _ALG5_CASES[case]
    A = make()
    b = gen.rhs_uniform(A.n, 1)
    h = oracle.Hierarchy(A, max_size=ms)
    h.sparsify(gam)
    x, info, tr = h.adaptive_solve(b, max_it=300, k=k, s=s, rho_max=rho_max, div_factor=divf, trace=True)
    xd, status, windows, its, resets = _alg5_dense(A, b, gam, k, s, rho_max, divf, ms)
    assert [(t["steps"], t["action"]) for t in tr] == [(w[0], w[1]) for w in windows]
    np.testing.assert_allclose([t["factor"] for t in tr], [w[2] for w in windows], rtol=1e-8)
    assert (info.status, info.iterations, info.resets) == (status, its, resets)
    assert np.linalg.norm(x - xd) <= 1e-8 * max(np.linalg.norm(xd), 1e-300)
    # every window's factor is its residual ratio per step
    for t in tr:
        if t["steps"]:
            assert abs(t["factor"] - (t["rend"] / t["rstart"]) ** (1 / t["steps"])) <= 1e-14 * t["factor"]


def test_adaptive_cases_cover_every_branch():
    seen = set()
    for case in _ALG5_CASES.values():
        make, gam, k, s, rho_max, divf, ms = case
        A = make()
        h = oracle.Hierarchy(A, max_size=ms)
        h.sparsify(gam)
        _, _, tr = h.adaptive_solve(gen.rhs_uniform(A.n, 1), max_it=300, k=k, s=s, rho_max=rho_max,
                                    div_factor=divf, trace=True)
        seen |= {t["action"] for t in tr}
    assert seen == set(oracle.WIN_ACTIONS), set(oracle.WIN_ACTIONS) - seen


@pytest.mark.parametrize("N,sigma,k", [(16, 0.065, 1), (20, 0.045, 2), (20, 0.05, 1)])
def test_pcg_divergence_stops_at_the_window_start(N, sigma, k):
    """PCG's divergence test (windows of k steps; the recurrence residual at a
    window's end against its start; growth beyond the factor -- 1 here --
    stops the run with x at the window's start), against plain dense CG."""
    A = _shifted_poisson2d(N, sigma)
    b = gen.rhs_uniform(A.n, 1)
    h = oracle.Hierarchy(A, max_size=20)
    x, info = h.pcg(b, max_it=300, k=k, div_factor=1.0)
    M, _ = _vcycle_operator(A, [0.0], 20)
    Ad = A.to_scipy().toarray()
    xd = np.zeros(A.n)
    r = b.copy()
    z = M @ r
    p, rho = z.copy(), r @ z
    xs, rws, its = xd.copy(), np.linalg.norm(r), 0
    while True:
        if its % k == 0:
            xs = xd.copy()
        q = Ad @ p
        assert p @ q > 0 and rho > 0, "the case must diverge before it breaks down"
        a = rho / (p @ q)
        xd, r = xd + a * p, r - a * q
        its += 1
        if its % k == 0:
            if np.linalg.norm(r) > rws:
                break
            rws = np.linalg.norm(r)
        z = M @ r
        rho_new = r @ z
        p, rho = z + (rho_new / rho) * p, rho_new
    assert info.status == oracle.DIVERGED and info.iterations == its
    np.testing.assert_allclose(x, xs, rtol=1e-10, atol=1e-12 * np.linalg.norm(xs))
    assert its > k  # it stops after more than one window
    # the default factor (1e3) never fires on an SPD problem
    A2 = gen.poisson2d_5pt(N)
    x2, i2 = oracle.Hierarchy(A2, max_size=20).pcg(gen.rhs_uniform(A2.n, 1))
    assert i2.status == oracle.OK


# ---------------------------------------------------------------------------
# Hybrid Galerkin (Algorithm 4, hybrid line): M from the sparsified Ahat_{l-1}
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("gamma", [0.1, 1.0])
def test_hybrid_minimal_pattern_brute_force(gamma):
    A = gen.poisson3d_7pt(9)
    h = oracle.Hierarchy(A, max_size=20)
    h.sparsify([0.0, gamma], method=1)
    ref = oracle.Hierarchy(A, max_size=20)
    for l in range(1, h.num_levels):
        Ah_prev = h.matrix(l - 1, "Ahat")
        P = h.matrix(l - 1, "P").todense()
        cf = h.cf(l - 1)
        Phat = np.zeros_like(P)
        Phat[np.where(cf == 1)[0], np.arange(P.shape[1])] = 1.0
        pa = pattern(Ah_prev).astype(int)
        pp = pattern(h.matrix(l - 1, "P")).astype(int)
        ph = (Phat > 0).astype(int)
        M = ((ph.T @ pa @ pp) + (pp.T @ pa @ ph)) > 0
        Ac = h.matrix(l, "A").to_scipy()
        rows = np.repeat(np.arange(Ac.shape[0]), np.diff(Ac.indptr))
        inM_h = M[rows, Ac.indices].astype(np.uint8)
        # the kept pattern is what sparsify gives with that M (dense reference)
        _, keep_ref = _dense_sparsify_reference(Ac, inM_h, gamma)
        np.testing.assert_array_equal(h.keep(l), keep_ref.astype(np.uint8))
        # Hybrid M is inside Sparse Galerkin's M (Ahat_{l-1} has fewer edges)
        assert np.all(inM_h <= ref.inM(l))
    # level 1 is identical for both methods (Ahat_0 = A_0)
    hs = oracle.Hierarchy(A, max_size=20)
    hs.sparsify([0.0, gamma], method=0)
    np.testing.assert_array_equal(h.keep(1), hs.keep(1))


@pytest.mark.parametrize("gamma", [0.1, 1.0])
def test_hybrid_keeps_theorem1_and_solves(gamma):
    """Row sums and symmetry always; semi-definiteness where Theorem 1's
    diagonal-dominance hypothesis holds (coarse Galerkin operators need not
    be diagonally dominant, and aggressive Hybrid dropping can then make
    Ahat_l indefinite)."""
    A = gen.poisson3d_7pt(12)
    h = oracle.Hierarchy(A, max_size=30)
    h.sparsify([0.0, gamma], method=1)
    for l in range(1, h.num_levels):
        Hd = h.matrix(l, "Ahat").todense()
        Ad = h.matrix(l, "A").todense()
        scale = np.abs(Ad).max()
        np.testing.assert_allclose(Hd.sum(axis=1), Ad.sum(axis=1), atol=1e-13 * scale)
        np.testing.assert_allclose(Hd, Hd.T, atol=1e-14 * scale)
        if np.all(2 * np.abs(np.diag(Ad)) >= np.abs(Ad).sum(axis=1) - 1e-12 * scale):
            assert np.linalg.eigvalsh(Hd).min() > -1e-12 * scale
    if gamma <= 0.1:
        b = gen.rhs_uniform(A.n, 4)
        x, info = h.pcg(b)
        assert info.status == 0 and info.final_relres <= 1e-8


# ---------------------------------------------------------------------------
# Algorithm 3's own loop: full lumping to strong neighbours
# ---------------------------------------------------------------------------
def test_full_lumping_hand_example():
    """Worked by hand (gamma = 0.5, theta = 0.25, M empty).

    Row maxima 2, 2, 1, 2: only a_03 = a_30 = -0.5 fail the drop test, so N is
    every other entry plus the diagonal.  Strength rows (theta 0.25): row 0 ->
    {1, 3}, row 3 -> {0, 1, 2}.
    Drop (0,3): W = {k : S_3k != 0, (0,k) in N} = {0, 1}, weights |a_30| = 0.5
    and |a_31| = 2 -> alpha = 0.2, 0.8; t = -0.1, -0.4.  k = 0 adds t twice to
    a_00 and subtracts it once (net -0.1); k = 1 adds -0.4 to a_01 and a_10
    and +0.4 to a_11.
    Drop (3,0): W = {k : S_0k != 0, (3,k) in N} = {1, 3}, weights 2 and 0.5
    -> t = -0.4 (k = 1: a_31, a_13 -= 0.4, a_11 += 0.4) and t = -0.1 (k = 3:
    net -0.1 on a_33).
    """
    A = np.array([[4.0, -2.0, 0.0, -0.5],
                  [-2.0, 6.0, -1.0, -2.0],
                  [0.0, -1.0, 3.0, -1.0],
                  [-0.5, -2.0, -1.0, 4.0]])
    want = np.array([[3.9, -2.4, 0.0, 0.0],
                     [-2.4, 6.8, -1.0, -2.4],
                     [0.0, -1.0, 3.0, -1.0],
                     [0.0, -2.4, -1.0, 3.9]])
    Ac = csr_from_dense(A)
    H, keep = oracle.sparsify_full(Ac, np.zeros(Ac.nnz, np.uint8), 0.5, 0.25)
    np.testing.assert_allclose(H.todense(), want, rtol=0, atol=1e-15)
    assert H.nnz == Ac.nnz - 2 and keep.sum() == Ac.nnz - 2


def test_full_lumping_empty_w_goes_to_diagonal():
    """Worked by hand: a_02 = a_20 = -0.1 are dropped (gamma 0.5); row 2's only
    strong neighbour is 3, which row 0 does not hold, and row 0's only strong
    neighbour is 1, which row 2 does not hold, so both W are empty and each
    value goes to its own row's diagonal (4 -> 3.9)."""
    A = np.array([[4.0, -3.0, -0.1, 0.0],
                  [-3.0, 5.0, 0.0, 0.0],
                  [-0.1, 0.0, 4.0, -3.0],
                  [0.0, 0.0, -3.0, 5.0]])
    want = np.array([[3.9, -3.0, 0.0, 0.0],
                     [-3.0, 5.0, 0.0, 0.0],
                     [0.0, 0.0, 3.9, -3.0],
                     [0.0, 0.0, -3.0, 5.0]])
    Ac = csr_from_dense(A)
    H, _ = oracle.sparsify_full(Ac, np.zeros(Ac.nnz, np.uint8), 0.5, 0.25)
    np.testing.assert_allclose(H.todense(), want, rtol=0, atol=1e-15)


def _dense_full_lumping(Ac, inM, gamma, theta):
    """Brute force on a dense copy: Ahat = A on N, then for each dropped
    (i, j) in row-major order the rank-3 symmetric update
    t (e_i e_k^T + e_k e_i^T - e_k e_k^T) for every k in W, t = alpha a_ij."""
    D = Ac.toarray()
    n = D.shape[0]
    rows = np.repeat(np.arange(n), np.diff(Ac.indptr))
    stored = np.zeros_like(D, dtype=bool)
    stored[rows, Ac.indices] = True
    _, keep = _dense_sparsify_reference(Ac, inM, gamma)
    N = np.zeros_like(stored)
    N[rows, Ac.indices] = keep
    # classical strength on negative couplings (an independent dense form)
    off = stored & ~np.eye(n, dtype=bool)
    neg = np.where(off, -D, -np.inf)
    m = neg.max(axis=1)
    S = off & (m[:, None] > 0) & (-D >= theta * m[:, None])
    H = np.where(N, D, 0.0)
    for i in range(n):
        for j in range(n):
            if not stored[i, j] or N[i, j]:
                continue
            a = D[i, j]
            W = [k for k in range(n) if S[j, k] and N[i, k]]
            den = sum(abs(D[j, k]) for k in W)
            if not den > 0:
                H[i, i] += a
                continue
            for k in W:
                t = abs(D[j, k]) / den * a
                U = np.zeros((n, n))
                U[i, k] += t
                U[k, i] += t
                U[k, k] -= t
                H += U
    return H, N[rows, Ac.indices]


@pytest.mark.parametrize("gamma", [0.0, 0.1, 0.5, 1.0])
def test_full_lumping_against_dense(gamma):
    h = _level_pair(gen.poisson3d_7pt(8))
    for l in range(1, h.num_levels):
        Ac = h.matrix(l, "A").to_scipy()
        H, keep = oracle.sparsify_full(Ac, h.inM(l), gamma, 0.25)
        Href, keep_ref = _dense_full_lumping(Ac, h.inM(l), gamma, 0.25)
        np.testing.assert_array_equal(keep, keep_ref.astype(np.uint8))
        scale = np.abs(Href).max()
        np.testing.assert_allclose(H.todense(), Href, rtol=0, atol=1e-13 * scale)
        if gamma == 0.0:
            np.testing.assert_array_equal(H.todense(), Ac.toarray())


@pytest.mark.parametrize("gamma", [0.1, 1.0])
def test_full_lumping_symmetry_rowsums_and_pattern(gamma):
    """Each update is symmetric with zero row sums: Ahat stays symmetric with
    the row sums of A_c; it keeps exactly N (no guard); off-diagonal values
    change where diagonal lumping would leave them."""
    h = _level_pair(gen.poisson3d_7pt(10), max_levels=5)
    changed_offdiag = False
    for l in range(1, h.num_levels):
        Ac = h.matrix(l, "A").to_scipy()
        Hf, kf = oracle.sparsify_full(Ac, h.inM(l), gamma, 0.25)
        Hd, kd = oracle.sparsify_diag(Ac, h.inM(l), gamma)
        np.testing.assert_array_equal(kf, kd)
        F, Ad = Hf.todense(), Ac.toarray()
        scale = np.abs(Ad).max()
        np.testing.assert_allclose(F, F.T, rtol=0, atol=1e-14 * scale)
        np.testing.assert_allclose(F.sum(axis=1), Ad.sum(axis=1), rtol=0, atol=1e-13 * scale)
        G = Hd.todense()
        offd = ~np.eye(F.shape[0], dtype=bool)
        changed_offdiag |= bool(np.any(np.abs(F - G)[offd] > 1e-12 * scale))
    assert changed_offdiag


def test_full_lumping_hierarchy_and_reintroduction():
    """Through the hierarchy (Sparse and Hybrid): reintroduction down to gamma
    = 0 restores the Galerkin operators exactly."""
    A = gen.poisson3d_7pt(10)
    for method in (0, 1):
        h = oracle.Hierarchy(A, max_size=20)
        L = h.num_levels
        h.sparsify([0.0] + [1.0] * (L - 1), method=method, lump=1)
        for l in range(1, L):
            Ac = h.matrix(l, "A").to_scipy()
            if method == 0:
                Hf, _ = oracle.sparsify_full(Ac, h.inM(l), 1.0, 0.25)
                np.testing.assert_array_equal(h.matrix(l, "Ahat").val, Hf.val)
        for _ in range(10 * L):
            cnt, _ = h.reintroduce(s=1)
            if cnt == 0:
                break
        for l in range(L):
            np.testing.assert_array_equal(h.matrix(l, "Ahat").val, h.matrix(l, "A").val)


# ---------------------------------------------------------------------------
# LU with partial pivoting (coarsest-level fallback) and GMRES
# ---------------------------------------------------------------------------
def test_lu_matches_library():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((9, 9))
    LU, piv = oracle.lu(A)
    lu_ref, piv_ref = sla.lu_factor(A)
    np.testing.assert_array_equal(piv, piv_ref)
    np.testing.assert_allclose(LU, lu_ref, rtol=1e-12, atol=1e-13)
    b = rng.standard_normal(9)
    np.testing.assert_allclose(oracle.lu_solve(LU, piv, b), sla.solve(A, b), rtol=1e-11)


def test_indefinite_coarsest_uses_lu():
    """A one-level hierarchy of a symmetric indefinite matrix: Cholesky fails,
    the pivoted LU solves it exactly."""
    rng = np.random.default_rng(6)
    Q, _ = np.linalg.qr(rng.standard_normal((8, 8)))
    A = Q @ np.diag([3.0, 2.0, 1.5, 1.0, -0.5, 2.5, -1.0, 4.0]) @ Q.T
    A = 0.5 * (A + A.T)
    h = oracle.Hierarchy(csr_from_dense(A), max_size=100)
    assert h.num_levels == 1
    b = rng.standard_normal(8)
    np.testing.assert_allclose(h.vcycle(b), sla.solve(A, b), rtol=1e-11, atol=1e-12)


def _krylov_minimiser(Aop, r0, k):
    """argmin over u in K_k(Aop, r0) of ||r0 - Aop u|| (orthonormal basis by QR)."""
    K = np.empty((r0.size, k))
    v = r0.copy()
    for c in range(k):
        K[:, c] = v
        v = Aop @ v
    Q, _ = np.linalg.qr(K)
    y, *_ = np.linalg.lstsq(Aop @ Q, r0, rcond=None)
    return Q @ y


def _nonsym(n, seed):
    rng = np.random.default_rng(seed)
    return np.eye(n) * 4 + rng.standard_normal((n, n)) * 0.6


@pytest.mark.parametrize("k", [1, 2, 3, 5])
def test_gmres_iterate_is_krylov_minimiser(k):
    A = _nonsym(12, 1)
    b = np.random.default_rng(2).standard_normal(12)
    x, info = oracle.gmres_plain(csr_from_dense(A), b, tol=0.0, max_it=k, restart=30)
    assert info.iterations == k
    np.testing.assert_allclose(x, _krylov_minimiser(A, b, k), rtol=1e-10, atol=1e-12)


def test_gmres_restart_is_two_minimisations():
    A = _nonsym(12, 3)
    b = np.random.default_rng(4).standard_normal(12)
    x, _ = oracle.gmres_plain(csr_from_dense(A), b, tol=0.0, max_it=5, restart=3)
    x3 = _krylov_minimiser(A, b, 3)
    x5 = x3 + _krylov_minimiser(A, b - A @ x3, 2)
    np.testing.assert_allclose(x, x5, rtol=1e-10, atol=1e-12)


def test_gmres_exact_within_n_steps():
    A = _nonsym(10, 7)
    b = np.random.default_rng(8).standard_normal(10)
    x, info = oracle.gmres_plain(csr_from_dense(A), b, tol=1e-12, max_it=50, restart=10)
    assert info.status == 0 and info.iterations <= 10
    np.testing.assert_allclose(x, sla.solve(A, b), rtol=1e-10)


def test_gmres_preconditioned_minimiser():
    """Right preconditioning: x_k = M u_k, u_k minimising ||b - A M u|| over
    K_k(A M, b), with M the (linear) V-cycle assembled column by column."""
    A = gen.poisson2d_5pt(9)
    h = oracle.Hierarchy(A, max_size=20)
    assert h.num_levels >= 2
    h.sparsify([0.0, 0.5])
    n = A.n
    Ad = A.to_scipy().toarray()
    M = np.column_stack([h.vcycle(e) for e in np.eye(n)])
    b = gen.rhs_uniform(n, 9)
    for k in (1, 2, 4):
        x, _ = h.gmres(b, tol=0.0, max_it=k, restart=30)
        u = _krylov_minimiser(Ad @ M, b, k)
        np.testing.assert_allclose(x, M @ u, rtol=1e-9, atol=1e-11)


def test_gmres_single_level_converges_in_one_step():
    A = gen.poisson2d_5pt(8)
    h = oracle.Hierarchy(A, max_size=1000)
    b = gen.rhs_uniform(A.n, 0)
    x, info = h.gmres(b)
    assert info.iterations == 1 and info.status == 0
    np.testing.assert_allclose(x, sla.solve(A.to_scipy().toarray(), b), rtol=1e-11)


def test_gmres_solves_full_lumping_hierarchy():
    A = gen.poisson3d_7pt(16)
    b = gen.rhs_uniform(A.n, 1)
    h = oracle.Hierarchy(A)
    xg, ig = h.gmres(b, tol=1e-8)
    assert ig.status == 0 and ig.final_relres <= 1e-8
    xp, ip = h.pcg(b, tol=1e-8)
    S = A.to_scipy().tocsc()
    xs = spla.spsolve(S, b)
    assert np.linalg.norm(xg - xs) <= 1e-5 * np.linalg.norm(xs)
    h.sparsify([0.0, 0.1, 1.0], lump=1)
    x, info = h.gmres(b, tol=1e-8)
    assert info.status == 0 and info.final_relres <= 1e-8
    h2 = oracle.Hierarchy(A)
    h2.sparsify([0.0, 1.0], lump=1)
    x2, i2 = h2.adaptive_gmres(b, tol=1e-8, rho_max=0.2)
    assert i2.status == 0 and i2.final_relres <= 1e-8


def test_gmres_zero_rhs():
    A = gen.poisson2d_5pt(8)
    h = oracle.Hierarchy(A)
    x, info = h.gmres(np.zeros(A.n))
    assert info.iterations == 0 and not x.any()


# ---------------------------------------------------------------------------
# rotated anisotropic Q1 generator (the paper's second test problem)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("theta,eps", [(np.pi / 8, 1e-3), (0.0, 0.01), (np.pi / 3, 0.2), (0.7, 1.0)])
def test_rotated_aniso_q1_consistency(theta, eps):
    """Q1 on a uniform grid reproduces -div(K grad u) exactly at interior
    nodes for polynomials of degree <= 2 (grid units): the stencil sums to 0,
    annihilates x and y, and maps x^2, y^2, xy to -2 K11, -2 K22, -2 K12."""
    N = 9
    A = gen.rotated_aniso_q1(N, theta=theta, eps=eps).to_scipy().toarray()
    c, s = np.cos(theta), np.sin(theta)
    K11, K22, K12 = c * c + eps * s * s, s * s + eps * c * c, c * s * (1 - eps)
    yy, xx = np.divmod(np.arange(N * N), N)
    row = 4 * N + 4  # centre node: all 9 neighbours interior
    for u, want in ((np.ones(N * N), 0.0), (xx * 1.0, 0.0), (yy * 1.0, 0.0),
                    (xx ** 2.0, -2 * K11), (yy ** 2.0, -2 * K22), (xx * yy * 1.0, -2 * K12)):
        assert A[row] @ u == pytest.approx(want, abs=1e-12)
    np.testing.assert_allclose(A, A.T, atol=1e-15)
    assert np.linalg.eigvalsh(A).min() > 0


def test_rotated_aniso_q1_isotropic_is_q1_laplacian():
    """eps = 1: K = I for every rotation; the textbook Q1 stencil 8/3, -1/3."""
    A = gen.rotated_aniso_q1(5, theta=0.3, eps=1.0).to_scipy().toarray()
    st = A[12].reshape(5, 5)[1:4, 1:4]
    want = np.full((3, 3), -1.0 / 3.0)
    want[1, 1] = 8.0 / 3.0
    np.testing.assert_allclose(st, want, atol=1e-15)


# ---------------------------------------------------------------------------
# non-Galerkin (Algorithm 1 with the in-loop sparsify)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("lump", [0, 1])
def test_nongalerkin_levels_built_from_sparsified_operators(lump):
    """Level by level, from the oracle's own building blocks (each pinned
    above): strength, PMIS and interpolation of the *sparsified* A_l, the
    Galerkin product, M from A_l, then the dense sparsify reference."""
    A = gen.poisson3d_7pt(10)
    g = [0.0, 0.5, 1.0]
    h = oracle.Hierarchy(A, max_size=20, nongalerkin=g, lump=lump)
    assert h.num_levels >= 3
    Al = A.to_scipy()
    for l in range(h.num_levels - 1):
        np.testing.assert_array_equal(h.matrix(l, "A").todense(), Al.toarray())
        S = oracle.strength(Al)
        cf = oracle.pmis(Al, S, seed=0, level=l)
        np.testing.assert_array_equal(h.cf(l), cf)
        Pm = oracle.direct_interp(Al, S, cf)
        P = Pm.todense()
        Ac = csr_from_dense(P.T @ Al.toarray() @ P)
        Gal = h.matrix(l + 1, "A")
        # M of the coarse operator from the current A_l (dense brute force
        # over the stored patterns: edges are structural)
        pa = pattern(Al).astype(int)
        pp = pattern(Pm).astype(int)
        ph = np.zeros_like(pp)
        ph[np.where(cf == 1)[0], np.arange(P.shape[1])] = 1
        Mset = ((ph.T @ pa @ pp) + (pp.T @ pa @ ph)) > 0
        AP = oracle.spgemm(Al, Pm)
        Ac_or = oracle.spgemm(oracle.transpose(Pm), AP).to_scipy()
        rows = np.repeat(np.arange(Ac_or.shape[0]), np.diff(Ac_or.indptr))
        inM = Mset[rows, Ac_or.indices].astype(np.uint8)
        gam = g[min(l + 1, len(g) - 1)]
        if lump:
            Href, _ = _dense_full_lumping(Ac_or, inM, gam, 0.25)
        else:
            Href, _ = _dense_sparsify_reference(Ac_or, inM, gam)
        scale = np.abs(Href).max()
        np.testing.assert_allclose(Gal.todense(), Href, rtol=0, atol=1e-12 * scale)
        assert Gal.nnz < Ac.nnz  # thinned, so not the Galerkin product any more
        Al = Gal.to_scipy()


def test_nongalerkin_gamma_zero_is_galerkin_and_refuses_alg5():
    A = gen.poisson3d_7pt(12)
    h0 = oracle.Hierarchy(A, max_size=20)
    h1 = oracle.Hierarchy(A, max_size=20, nongalerkin=[0.0])
    assert h0.num_levels == h1.num_levels
    for l in range(h0.num_levels):
        np.testing.assert_array_equal(h0.matrix(l, "A").val, h1.matrix(l, "A").val)
    h2 = oracle.Hierarchy(A, max_size=20, nongalerkin=[0.0, 1.0], lump=1)
    with pytest.raises(RuntimeError):
        h2.sparsify([0.0, 0.1])
    with pytest.raises(RuntimeError):
        h2.reintroduce(1)


def test_nongalerkin_negative_diagonal_is_a_breakdown():
    """12^3 Poisson, gamma 1 from level 1 with diagonal lumping: rebuilding
    level 2 from the pinned building blocks (strength, PMIS with level index
    1, direct interpolation, Galerkin product, M, dense-pinned 3b sparsify)
    on the thinned level 1 gives a non-positive diagonal entry, and the
    non-Galerkin setup reports that as a breakdown."""
    A = gen.poisson3d_7pt(12)
    with pytest.raises(RuntimeError, match="status 6"):
        oracle.Hierarchy(A, nongalerkin=[0.0, 1.0], lump=0)
    h1 = oracle.Hierarchy(A, max_levels=2, nongalerkin=[0.0, 1.0], lump=0)
    A1 = h1.matrix(1, "A")
    assert (A1.to_scipy().diagonal() > 0).all()
    S = oracle.strength(A1)
    cf = oracle.pmis(A1, S, seed=0, level=1)
    P = oracle.direct_interp(A1, S, cf)
    AP = oracle.spgemm(A1, P)
    Ac = oracle.spgemm(oracle.transpose(P), AP)
    inM = oracle.minimal_pattern(Ac, AP, cf)
    H, _ = oracle.sparsify_diag(Ac, inM, 1.0)
    assert H.to_scipy().diagonal().min() <= 0.0


def test_nongalerkin_full_lumping_rescues_aggressive_dropping():
    """The paper's motivating example (Section 2.1, Figures 1-2): gamma = 1
    from the first coarse level on removes essential entries.  With diagonal
    lumping the non-Galerkin setup breaks down here (a thinned diagonal
    crosses zero); Algorithm 3's lumping to strong neighbours keeps every
    operator's row sums and symmetry and converges."""
    A = gen.poisson3d_7pt(16)
    b = gen.rhs_uniform(A.n, 1)
    with pytest.raises(RuntimeError, match="status 6"):  # a thinned diagonal crosses zero
        oracle.Hierarchy(A, nongalerkin=[0.0, 1.0], lump=0)
    hf = oracle.Hierarchy(A, nongalerkin=[0.0, 1.0], lump=1)
    _, ifl = hf.pcg(b)
    assert ifl.status == 0 and ifl.final_relres <= 1e-8
    for l in range(1, hf.num_levels):
        H = hf.matrix(l, "A").todense()
        np.testing.assert_allclose(H, H.T, atol=1e-13 * np.abs(H).max())


# ---------------------------------------------------------------------------
# l1 smoother diagonal d_i = sum_j |a_ij| (the relaxation weight of the
# l1-Jacobi smoother on every level)
# ---------------------------------------------------------------------------
def test_l1_diag_closed_form_on_2d_poisson():
    N = 7
    d = oracle.l1_diag(gen.poisson2d_5pt(N)).reshape(N, N)
    # 4 on the diagonal plus one per neighbour inside the grid (Dirichlet boundary)
    expect = np.full((N, N), 8.0)
    expect[0, :] -= 1
    expect[-1, :] -= 1
    expect[:, 0] -= 1
    expect[:, -1] -= 1
    assert np.array_equal(d, expect)
    assert d[0, 0] == 6.0 and d[0, 3] == 7.0 and d[3, 3] == 8.0


def test_l1_diag_of_zero_row_sum_m_matrix_is_twice_the_diagonal():
    # graph Laplacian of a path with weights: every row sums to zero, off-diagonals negative
    w = np.array([1.5, 0.25, 2.0, 3.0])
    n = len(w) + 1
    L = np.zeros((n, n))
    for k, wk in enumerate(w):
        L[k, k] += wk
        L[k + 1, k + 1] += wk
        L[k, k + 1] -= wk
        L[k + 1, k] -= wk
    A = sp.csr_matrix(L)
    d = oracle.l1_diag(A)
    assert np.array_equal(d, 2.0 * np.diag(L))


def test_l1_diag_counts_positive_couplings_by_absolute_value():
    # row 0: 5 -2 +3  -> 10;  row 1: -2 4 0 -> 6;  row 2: +3 0 9 -> 12
    A = sp.csr_matrix(np.array([[5.0, -2.0, 3.0], [-2.0, 4.0, 0.0], [3.0, 0.0, 9.0]]))
    assert np.array_equal(oracle.l1_diag(A), [10.0, 6.0, 12.0])


def test_openmp_timing_build_matches_sequential_oracle():
    """The all-core timing build of the oracle (the same source with the
    solve phase's row loops split over threads) solves like the sequential
    parity build: same iterations, x within 1e-12 (only dot products sum in
    another order).  Sized above the loops' threading threshold."""
    A = gen.poisson3d_7pt(40)
    b = gen.rhs_uniform(A.n, 1)
    out = []
    for omp in (False, True):
        h = oracle.Hierarchy(A, omp=omp)
        h.sparsify([0.0, 0.1])
        out.append(h.pcg(b) + (h.level_sizes(),))
    (x0, i0, s0), (x1, i1, s1) = out
    assert s0 == s1 and i0.status == i1.status == 0
    assert abs(i0.iterations - i1.iterations) <= 1
    assert np.linalg.norm(x1 - x0) <= 1e-12 * np.linalg.norm(x0)
