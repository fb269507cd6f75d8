"""GPU path vs the CPU oracle for full lumping to strong neighbours
(Algorithm 3's own loop) and for the restarted GMRES outer solver.

Kept-entry masks are bit-exact; the lumped values are accumulated in the
oracle's update order, so Ahat_l matches to 1e-12 relative (expected
identical).  GMRES orthogonalises by classical Gram-Schmidt run twice where
the oracle uses modified Gram-Schmidt: the iterates agree to rounding, the
iteration counts within one, the solutions to the solver tolerance.
"""
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


def _same_csr(got, ref, rtol=1e-12, what=""):
    assert got.nrows == ref.nrows and got.ncols == ref.ncols, what
    np.testing.assert_array_equal(got.rowptr, ref.rowptr, err_msg=what + " rowptr")
    np.testing.assert_array_equal(got.col, ref.col, err_msg=what + " col")
    scale = max(np.abs(ref.val).max() if ref.nnz else 1.0, 1e-300)
    np.testing.assert_allclose(got.val, ref.val, rtol=0, atol=rtol * scale, err_msg=what + " val")


CASES = {
    "2d5_64": lambda: gen.poisson2d_5pt(64),
    "3d7_20": lambda: gen.poisson3d_7pt(20),
    "3d27_11": lambda: gen.poisson3d_27pt(11),
    "fv7_15": lambda: gen.fv7_lognormal(15, seed=3),
}


@pytest.mark.parametrize("method", [0, 1])
@pytest.mark.parametrize("gamma", [0.01, 0.1, 1.0])
@pytest.mark.parametrize("case", list(CASES))
def test_full_lumping_matches_oracle(amg, case, gamma, method):
    A = CASES[case]()
    ref = oracle.Hierarchy(A)
    ref.sparsify([0.0, gamma], method=method, lump=1)
    h = amg.Hierarchy.setup(A, gamma=[0.0, gamma], method=method, lump=amg.LUMP_STRONG)
    assert h.num_levels == ref.num_levels
    for l in range(1, h.num_levels):
        np.testing.assert_array_equal(h.level_array(l, "keep"), ref.keep(l), err_msg=f"keep_{l}")
        _same_csr(h.export(l, "Ahat"), ref.matrix(l, "Ahat"), what=f"Ahat_{l}")
        np.testing.assert_allclose(h.level_array(l, "l1"), ref.l1(l), rtol=1e-14)


def test_full_lumping_values_bit_exact(amg):
    """The gather adds every update in the sequential loop's order."""
    A = gen.poisson3d_27pt(12)
    ref = oracle.Hierarchy(A)
    ref.sparsify([0.0, 0.5], lump=1)
    h = amg.Hierarchy.setup(A, gamma=[0.0, 0.5], lump=amg.LUMP_STRONG)
    for l in range(1, h.num_levels):
        np.testing.assert_array_equal(h.export(l, "Ahat").val, ref.matrix(l, "Ahat").val)


def test_full_lumping_reintroduction_matches_oracle(amg):
    A = gen.poisson3d_7pt(20)
    ref = oracle.Hierarchy(A)
    ref.sparsify([0.0, 1.0], lump=1)
    h = amg.Hierarchy.setup(A, gamma=[0.0, 1.0], lump=amg.LUMP_STRONG)
    for _ in range(20):
        c1 = h.reintroduce(1)
        c2, _ = ref.reintroduce(1)
        assert c1 == c2
        for l in range(1, h.num_levels):
            np.testing.assert_array_equal(h.level_array(l, "keep"), ref.keep(l))
            _same_csr(h.export(l, "Ahat"), ref.matrix(l, "Ahat"), what=f"Ahat_{l}")
        if c1 == 0:
            break
    for l in range(h.num_levels):
        np.testing.assert_array_equal(h.export(l, "Ahat").val, h.export(l, "A").val)


def test_full_lumping_on_assembled_hierarchy(amg):
    """Assembled from the oracle's Galerkin operators: S comes from the
    options' theta, as in a setup."""
    A = gen.poisson3d_7pt(22)
    ref = oracle.Hierarchy(A)
    L = ref.num_levels
    h = amg.Hierarchy.assemble([ref.matrix(l, "A") for l in range(L)],
                               [ref.matrix(l, "P") for l in range(L - 1)],
                               [ref.cf(l) for l in range(L - 1)],
                               [None] + [ref.inM(l) for l in range(1, L)],
                               gamma=[0.0, 0.1, 1.0], lump=amg.LUMP_STRONG)
    ref.sparsify([0.0, 0.1, 1.0], lump=1)
    for l in range(1, L):
        np.testing.assert_array_equal(h.level_array(l, "keep"), ref.keep(l))
        _same_csr(h.export(l, "Ahat"), ref.matrix(l, "Ahat"), what=f"Ahat_{l}")


@pytest.mark.parametrize("use_graph", [1, 0])
@pytest.mark.parametrize("case,gamma,lump", [("2d5_64", 0.0, 0), ("3d7_20", 0.1, 1), ("3d7_20", 1.0, 1),
                                             ("fv7_15", 0.1, 1), ("3d27_11", 0.1, 0), ("3d7_20", 1.0, 0)])
def test_gmres_matches_oracle(amg, case, gamma, lump, use_graph):
    A = CASES[case]()
    b = gen.rhs_uniform(A.n, 1)
    ref = oracle.Hierarchy(A)
    ref.sparsify([0.0, gamma], lump=lump)
    xr, ir = ref.gmres(b, tol=1e-8, restart=30)
    h = amg.Hierarchy.setup(A, gamma=[0.0, gamma], lump=lump, krylov=amg.KRYLOV_GMRES, restart=30,
                            use_graph=use_graph)
    for on_dev in (False, True):
        bb = torch.from_numpy(b).cuda() if on_dev else b
        x, info = h.solve(bb, tol=1e-8)
        x = x.cpu().numpy() if on_dev else x
        assert ir.status == 0
        assert info.status == 0 and info.final_relres <= 1e-8
        assert abs(info.iterations - ir.iterations) <= 1, (info.iterations, ir.iterations)
        resid = b - A.to_scipy() @ x
        assert np.linalg.norm(resid) <= 1e-8 * np.linalg.norm(b) * (1 + 1e-6)
        assert np.linalg.norm(x - xr) <= 1e-6 * np.linalg.norm(xr)


@pytest.mark.parametrize("restart", [1, 3, 7])
def test_gmres_restarts_match_oracle(amg, restart):
    A = gen.poisson3d_7pt(16)
    b = gen.rhs_uniform(A.n, 2)
    ref = oracle.Hierarchy(A)
    ref.sparsify([0.0, 0.1], lump=1)
    xr, ir = ref.gmres(b, tol=1e-8, restart=restart, max_it=200)
    h = amg.Hierarchy.setup(A, gamma=[0.0, 0.1], lump=amg.LUMP_STRONG, krylov=amg.KRYLOV_GMRES,
                            restart=restart)
    x, info = h.solve(b, tol=1e-8, max_it=200)
    assert info.status == ir.status == 0
    assert abs(info.iterations - ir.iterations) <= 1, (info.iterations, ir.iterations)
    assert np.linalg.norm(x - xr) <= 1e-6 * np.linalg.norm(xr)


def test_gmres_iterates_match_oracle_step_by_step(amg):
    """After k steps without the stop test (a tolerance no residual reaches)
    both sides hold the same Krylov minimiser, to rounding."""
    A = gen.poisson3d_7pt(17)
    b = gen.rhs_uniform(A.n, 3)
    ref = oracle.Hierarchy(A)
    ref.sparsify([0.0, 0.5], lump=1)
    h = amg.Hierarchy.setup(A, gamma=[0.0, 0.5], lump=amg.LUMP_STRONG, krylov=amg.KRYLOV_GMRES)
    for k in (1, 2, 5, 9):
        xr, _ = ref.gmres(b, tol=1e-300, max_it=k)
        x, info = h.solve(b, tol=1e-300, max_it=k)
        assert info.iterations == k
        np.testing.assert_allclose(x, xr, rtol=0, atol=1e-10 * np.abs(xr).max())


@pytest.mark.parametrize("use_graph", [1, 0])
def test_adaptive_gmres_matches_oracle(amg, use_graph):
    A = gen.poisson3d_7pt(24)
    b = gen.rhs_uniform(A.n, 1)
    ref = oracle.Hierarchy(A)
    ref.sparsify([0.0, 1.0], lump=1)
    xr, ir = ref.adaptive_gmres(b, rho_max=0.2, s=1, k=3)
    h = amg.Hierarchy.setup(A, gamma=[0.0, 1.0], lump=amg.LUMP_STRONG, krylov=amg.KRYLOV_GMRES,
                            rho_max=0.2, s_levels=1, k_check=3, use_graph=use_graph)
    x, info = h.solve(b, tol=1e-8, adaptive=True)
    assert ir.status == 0 and info.status == 0 and info.final_relres <= 1e-8
    assert info.resets == ir.resets
    assert abs(info.iterations - ir.iterations) <= 1
    for l in range(h.num_levels):
        assert h.level_stats(l)["gamma"] == pytest.approx(ref.gamma(l), rel=1e-12)


def test_gmres_single_level_and_zero_rhs(amg):
    A = gen.poisson2d_5pt(8)
    h = amg.Hierarchy.setup(A, max_size=1000, krylov=amg.KRYLOV_GMRES)
    b = gen.rhs_uniform(A.n, 0)
    x, info = h.solve(b)
    assert info.status == 0 and info.iterations == 1
    x0, i0 = h.solve(np.zeros(A.n))
    assert i0.iterations == 0 and not x0.any()


@pytest.mark.parametrize("prec", [1, 2])
def test_gmres_mixed_precision_cycle(amg, prec):
    """FP32 / BF16 cycles: flexible GMRES reaches the FP64 tolerance."""
    A = gen.poisson3d_7pt(20)
    b = gen.rhs_uniform(A.n, 4)
    h = amg.Hierarchy.setup(A, gamma=[0.0, 0.1], lump=amg.LUMP_STRONG, krylov=amg.KRYLOV_GMRES, precision=prec)
    x, info = h.solve(b, tol=1e-8)
    assert info.status == 0 and info.final_relres <= 1e-8


def test_indefinite_coarsest_uses_pivoting(amg):
    """A one-level hierarchy of a symmetric indefinite matrix with a positive
    diagonal (tridiagonal 1, 0.8: eigenvalues 1 + 1.6 cos(k pi / 41)): the
    Cholesky factorization fails, the coarse solve falls back to Gauss-Jordan
    with pivoting and is exact."""
    import scipy.sparse as sp
    n = 40
    S = sp.diags([0.8, 1.0, 0.8], [-1, 0, 1], shape=(n, n), format="csr")
    S.sort_indices()
    M = S.toarray()
    assert np.linalg.eigvalsh(M).min() < 0
    h = amg.Hierarchy.setup(S, max_size=1000, krylov=amg.KRYLOV_GMRES)
    b = np.random.default_rng(6).standard_normal(n)
    x, info = h.solve(b, tol=1e-10)
    assert info.status == 0 and info.iterations == 1
    np.testing.assert_allclose(x, np.linalg.solve(M, b), rtol=1e-9, atol=1e-10)


def test_full_size_full_lumping_levels_match_oracle(amg):
    """64^3 7-point Poisson, full lumping with gamma 1 on the coarse levels:
    masks and values of every level equal the oracle's."""
    A = gen.poisson3d_7pt(64)
    ref = oracle.Hierarchy(A)
    ref.sparsify([0.0, 1.0], lump=1)
    h = amg.Hierarchy.setup(A, gamma=[0.0, 1.0], lump=amg.LUMP_STRONG)
    for l in range(1, h.num_levels):
        np.testing.assert_array_equal(h.level_array(l, "keep"), ref.keep(l))
        np.testing.assert_array_equal(h.export(l, "Ahat").val, ref.matrix(l, "Ahat").val)


# ---------------------------------------------------------------------------
# non-Galerkin (Algorithm 1 with the in-loop sparsify)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("lump", [0, 1])
@pytest.mark.parametrize("case,gamma", [("3d7_20", [0.0, 0.5, 1.0]), ("fv7_15", [0.0, 0.1]),
                                        ("3d27_11", [0.0, 0.0, 1.0]), ("2d5_64", [0.0, 1.0])])
def test_nongalerkin_matches_oracle(amg, case, gamma, lump):
    """Every level -- operators, C/F splits, P -- bit-identical: the thinned
    operator feeds the next level's strength, PMIS, interpolation and RAP."""
    A = CASES[case]()
    ref = oracle.Hierarchy(A, nongalerkin=gamma, lump=lump)
    h = amg.Hierarchy.setup(A, gamma=gamma, method=amg.METHOD_NONGALERKIN, lump=lump)
    assert h.num_levels == ref.num_levels
    for l in range(h.num_levels):
        _same_csr(h.export(l, "A"), ref.matrix(l, "A"), what=f"A_{l}")
        np.testing.assert_array_equal(h.export(l, "A").val, ref.matrix(l, "A").val)
        _same_csr(h.export(l, "Ahat"), ref.matrix(l, "A"), what=f"Ahat_{l}")
        if l + 1 < h.num_levels:
            np.testing.assert_array_equal(h.level_array(l, "cf"), ref.cf(l), err_msg=f"cf_{l}")
            _same_csr(h.export(l, "P"), ref.matrix(l, "P"), what=f"P_{l}")
        np.testing.assert_allclose(h.level_array(l, "l1"), ref.l1(l), rtol=1e-14)
    b = gen.rhs_uniform(A.n, 1)
    xr, ir = ref.gmres(b, tol=1e-8)
    h2 = amg.Hierarchy.setup(A, gamma=gamma, method=amg.METHOD_NONGALERKIN, lump=lump, krylov=amg.KRYLOV_GMRES)
    x, info = h2.solve(b, tol=1e-8)
    assert ir.status == 0 and info.status == 0 and info.final_relres <= 1e-8
    assert abs(info.iterations - ir.iterations) <= 1, (info.iterations, ir.iterations)


def test_nongalerkin_breakdown_matches_oracle(amg):
    """12^3 Poisson, gamma 1 from level 1, diagonal lumping: level 2's thinned
    operator has a negative diagonal entry; both sides stop the setup with a
    breakdown.  Full lumping of the same case sets up and solves."""
    A = gen.poisson3d_7pt(12)
    with pytest.raises(RuntimeError, match="status 6"):
        oracle.Hierarchy(A, nongalerkin=[0.0, 1.0], lump=0)
    with pytest.raises(amg.AmgError) as e:
        amg.Hierarchy.setup(A, gamma=[0.0, 1.0], method=amg.METHOD_NONGALERKIN)
    assert e.value.status == amg.BREAKDOWN
    h = amg.Hierarchy.setup(A, gamma=[0.0, 1.0], method=amg.METHOD_NONGALERKIN, lump=amg.LUMP_STRONG,
                            krylov=amg.KRYLOV_GMRES)
    _, info = h.solve(gen.rhs_uniform(A.n, 0))
    assert info.status == 0


def test_nongalerkin_refuses_retained_operator_calls(amg, tmp_path):
    A = gen.poisson3d_7pt(12)
    h = amg.Hierarchy.setup(A, gamma=[0.0, 0.1], method=amg.METHOD_NONGALERKIN)
    for call in (lambda: h.sparsify([0.0, 0.1]), lambda: h.reintroduce(1),
                 lambda: h.solve(gen.rhs_uniform(A.n, 0), adaptive=True),
                 lambda: h.save(str(tmp_path / "h.bin"))):
        with pytest.raises(amg.AmgError) as e:
            call()
        assert e.value.status == 1
