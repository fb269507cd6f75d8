"""GPU parity on the paper's second workload and on the larger configurations.

* The rotated anisotropic Q1 problem (Section 5, second test problem: theta =
  pi/8, eps = 1e-3): half of its fine-level off-diagonals are positive, which
  is where the strength rule's sign handling and direct interpolation's
  positive-coupling branch decide the hierarchy.  Every setup array is
  compared with the oracle's (integer work bit for bit, FP64 values to
  1e-12), then the GMRES solve (iterations within one, x within 1e-6).
* Mixed precision (FP32 cycle, BF16 values on levels >= 2, FP64 outer
  flexible CG) on 27-point Poisson grids whose levels >= 2 hold thousands of
  rows, against the FP64 oracle solution.
* A batched multi-right-hand-side solve shaped like the lognormal
  finite-volume workload (FP32 cycle, gamma = 0.1), columns against the
  oracle's single solves.
* At the full 27-point 192^3 size the oracle is too slow for a test, so the
  reduced-precision solves are checked there by properties that hold at any
  size: the FP64 true residual (recomputed on the host) and the distance to
  the GPU's own FP64 solve, whose parity the smaller cases establish.
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


_ANISO = {}


def _aniso(N):
    if N not in _ANISO:
        _ANISO[N] = gen.rotated_aniso_q1(N)
    return _ANISO[N]


@pytest.mark.parametrize("N,method,lump", [(96, 0, 0), (96, 1, 0), (96, 0, 1), (96, 1, 1), (512, 0, 0),
                                           (512, 1, 1)])
def test_rotated_aniso_hierarchy_matches_oracle(amg, N, method, lump):
    A = _aniso(N)
    S = A.to_scipy()
    assert (S.data > 0).sum() > 0.3 * (S.nnz - A.n)  # many positive couplings
    gam = [0.0, 0.1, 1.0]
    ref = oracle.Hierarchy(A)
    ref.sparsify(gam, method=method, lump=lump)
    h = amg.Hierarchy.setup(A, gamma=gam, method=method, lump=lump)
    assert h.num_levels == ref.num_levels
    for l in range(h.num_levels):
        _same_csr(h.export(l, "A"), ref.matrix(l, "A"), what=f"A_{l}")
        if l + 1 < h.num_levels:
            np.testing.assert_array_equal(h.level_array(l, "strong"), ref.strong(l), err_msg=f"S_{l}")
            np.testing.assert_array_equal(h.level_array(l, "cf"), ref.cf(l), err_msg=f"cf_{l}")
            _same_csr(h.export(l, "P"), ref.matrix(l, "P"), what=f"P_{l}")
            _same_csr(h.export(l, "R"), ref.matrix(l, "R"), what=f"R_{l}")
        if l > 0:
            np.testing.assert_array_equal(h.level_array(l, "inM"), ref.inM(l), err_msg=f"M_{l}")
            np.testing.assert_array_equal(h.level_array(l, "keep"), ref.keep(l), err_msg=f"keep_{l}")
        _same_csr(h.export(l, "Ahat"), ref.matrix(l, "Ahat"), what=f"Ahat_{l}")
        np.testing.assert_allclose(h.level_array(l, "l1"), ref.l1(l), rtol=1e-14, atol=0)


@pytest.mark.parametrize("N", [96, 512])
@pytest.mark.parametrize("method,lump", [(0, 0), (1, 1)])
def test_rotated_aniso_gmres_matches_oracle(amg, N, method, lump):
    A = _aniso(N)
    b = gen.rhs_uniform(A.n, 1)
    gam = [0.0, 0.1, 1.0]
    ref = oracle.Hierarchy(A)
    ref.sparsify(gam, method=method, lump=lump)
    xr, ir = ref.gmres(b, tol=1e-8, restart=30, max_it=1000)
    assert ir.status == 0
    h = amg.Hierarchy.setup(A, gamma=gam, method=method, lump=lump, krylov=amg.KRYLOV_GMRES, restart=30)
    x, info = h.solve(b, tol=1e-8, max_it=1000)
    assert info.status == 0 and info.final_relres <= 1e-8
    assert abs(info.iterations - ir.iterations) <= 1, (info.iterations, ir.iterations)
    resid = b - A.to_scipy() @ x
    assert np.linalg.norm(resid) <= 1e-8 * np.linalg.norm(b) * (1 + 1e-6)
    assert np.linalg.norm(x - xr) <= 1e-6 * np.linalg.norm(xr)


def test_rotated_aniso_adaptive_gmres_matches_oracle(amg):
    A = _aniso(96)
    b = gen.rhs_uniform(A.n, 1)
    ref = oracle.Hierarchy(A)
    ref.sparsify([0.0, 1.0])
    xr, ir = ref.adaptive_gmres(b, tol=1e-8, restart=30, max_it=1000, k=3, s=1, rho_max=0.5)
    h = amg.Hierarchy.setup(A, gamma=[0.0, 1.0], krylov=amg.KRYLOV_GMRES, restart=30, k_check=3,
                            s_levels=1, rho_max=0.5)
    x, info = h.solve(b, tol=1e-8, max_it=1000, adaptive=True)
    assert info.status == ir.status == 0
    assert info.resets == ir.resets
    assert abs(info.iterations - ir.iterations) <= 1
    assert np.linalg.norm(x - xr) <= 1e-6 * np.linalg.norm(xr)
    for l in range(h.num_levels):
        assert h.level_stats(l)["gamma"] == pytest.approx(ref.gamma(l), rel=1e-12)


_Q27 = {}


def _q27(N):
    if N not in _Q27:
        A = gen.poisson3d_27pt(N)
        b = gen.rhs_uniform(A.n, 1)
        _Q27[N] = (A, b, {})
    return _Q27[N]


def _q27_oracle(N, gamma):
    A, b, cache = _q27(N)
    if gamma not in cache:
        ref = oracle.Hierarchy(A)
        ref.sparsify([0.0, gamma])
        cache[gamma] = ref.pcg(b, tol=1e-8) + (ref.level_sizes(),)
    return cache[gamma]


@pytest.mark.parametrize("N", [64, 96])
@pytest.mark.parametrize("prec", [1, 2])
@pytest.mark.parametrize("gamma", [0.0, 0.1])
def test_mixed_precision_at_scale_matches_fp64_oracle(amg, N, prec, gamma):
    """FP32 cycle (prec 1) and FP32 cycle with BF16 values on levels >= 2
    (prec 2), FP64 outer flexible CG, on grids whose level 2 has thousands of
    rows: the FP64 relative residual reaches 1e-8 and x is within 1e-6 of the
    FP64 oracle solution."""
    A, b, _ = _q27(N)
    xr, ir, sizes = _q27_oracle(N, gamma)
    assert ir.status == 0 and sizes[2][0] >= 3000
    h = amg.Hierarchy.setup(A, gamma=[0.0, gamma], precision=prec)
    vb = [h.level_stats(l)["value_bytes"] for l in range(h.num_levels)]
    assert vb[:2] == [4, 4] and all(v == (2 if prec == 2 else 4) for v in vb[2:])
    x, info = h.solve(b, tol=1e-8)
    assert info.status == 0 and info.final_relres <= 1e-8
    resid = b - A.to_scipy() @ x
    assert np.linalg.norm(resid) <= 1e-8 * np.linalg.norm(b) * (1 + 1e-6)
    assert np.linalg.norm(x - xr) <= 1e-6 * np.linalg.norm(xr)
    assert abs(info.iterations - ir.iterations) <= 3, (info.iterations, ir.iterations)


def test_batched_lognormal_at_scale_matches_oracle(amg):
    """The batched finite-volume workload's shape (lognormal coefficients,
    sigma = 2; gamma = 0.1; FP32 cycle, FP64 outer CG) at 64^3 with k = 8
    right-hand sides: every column reaches 1e-8 in FP64, and sampled columns
    match the oracle's single solves."""
    A = gen.fv7_lognormal(64, seed=3)
    k = 8
    B = np.stack([gen.rhs_uniform(A.n, 300 + c) for c in range(k)], axis=1)
    h = amg.Hierarchy.setup(A, gamma=[0.0, 0.1], precision=1)
    X, infos = h.solve_batch(torch.from_numpy(B).cuda(), tol=1e-8)
    X = X.cpu().numpy()
    S = A.to_scipy()
    for c in range(k):
        assert infos[c].status == 0, infos[c].as_dict()
        assert np.linalg.norm(B[:, c] - S @ X[:, c]) <= 1e-8 * np.linalg.norm(B[:, c]) * (1 + 1e-6)
    ref = oracle.Hierarchy(A)
    ref.sparsify([0.0, 0.1])
    for c in (0, 5):
        xr, ir = ref.pcg(B[:, c], tol=1e-8)
        assert abs(infos[c].iterations - ir.iterations) <= 3
        assert np.linalg.norm(X[:, c] - xr) <= 1e-6 * np.linalg.norm(xr)


def test_mixed_precision_full_size_27pt_192(amg):
    """The 27-point 192^3 workload (7.1 M rows, 189 M entries), gamma = 0.1:
    FP64, FP32 and FP32 + BF16 cycles all reach the FP64 relative residual
    1e-8 (recomputed on the host in FP64) and the reduced-precision solutions
    lie within 1e-6 of the FP64 one."""
    A = gen.poisson3d_27pt(192)
    b = gen.rhs_uniform(A.n, 1)
    S = A.to_scipy()
    bn = np.linalg.norm(b)
    xs = {}
    for prec in (0, 1, 2):
        h = amg.Hierarchy.setup(A, gamma=[0.0, 0.1], precision=prec)
        x, info = h.solve(torch.from_numpy(b).cuda(), tol=1e-8)
        x = x.cpu().numpy()
        assert info.status == 0 and info.final_relres <= 1e-8
        assert np.linalg.norm(b - S @ x) <= 1e-8 * bn * (1 + 1e-6)
        xs[prec] = x
        del h
        torch.cuda.empty_cache()
    for prec in (1, 2):
        assert np.linalg.norm(xs[prec] - xs[0]) <= 1e-6 * np.linalg.norm(xs[0])
