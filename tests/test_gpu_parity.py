"""GPU path vs the CPU oracle, through the C ABI (libamg.so).

Integer work (strength flags, C/F split, kept-entry masks, patterns, per-level
sizes) must match bit for bit.  FP64 setup values (P, Galerkin A_l, Ahat_l)
must match to 1e-12 relative (the kernels accumulate in the oracle's order,
so they are in fact expected to be identical).  Solutions must reach the
1e-8 relative residual and match the oracle's iteration count within one.
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
    "2d5_37": lambda: gen.poisson2d_5pt(37),
    "3d7_20": lambda: gen.poisson3d_7pt(20),
    "3d27_11": lambda: gen.poisson3d_27pt(11),
    "fv7_15": lambda: gen.fv7_lognormal(15, seed=3),
    # rows of 129..18201 products, some with more than 128 distinct columns:
    # every fallback of the capped hash table (tests/test_inputs_cover.py)
    "hubs": gen.hub_graphs,
}


@pytest.mark.parametrize("case", list(CASES))
def test_setup_end_to_end_matches_oracle(amg, case):
    A = CASES[case]()
    ref = oracle.Hierarchy(A)
    h = amg.Hierarchy.setup(A)
    assert h.num_levels == ref.num_levels
    for l in range(h.num_levels):
        _same_csr(h.export(l, "A"), ref.matrix(l, "A"), what=f"A_{l}")
        if l + 1 < h.num_levels:
            np.testing.assert_array_equal(h.level_array(l, "strong"), ref.strong(l), err_msg=f"S_{l}")
            np.testing.assert_array_equal(h.level_array(l, "cf"), ref.cf(l), err_msg=f"cf_{l}")
            _same_csr(h.export(l, "P"), ref.matrix(l, "P"), what=f"P_{l}")
            _same_csr(h.export(l, "R"), ref.matrix(l, "R"), what=f"R_{l}")
        if l > 0:
            np.testing.assert_array_equal(h.level_array(l, "inM"), ref.inM(l), err_msg=f"inM_{l}")
        np.testing.assert_allclose(h.level_array(l, "l1"), ref.l1(l), rtol=1e-14)


def test_full_size_bench_workload_matches_oracle(amg):
    """The bench workload at its full size (3D 7-point 128^3, Sparse Galerkin
    gamma = 0.1, FP64, the same entry points and launch configuration the
    bench times): every level of the GPU hierarchy -- strength, C/F split, P,
    R, Galerkin A_l, M, kept entries, sparsified operators, l1 diagonals -- is
    identical to the oracle's, and the PCG solve matches it (iterations within
    one, solution within the stopping tolerance)."""
    import torch

    A = gen.poisson3d_7pt(128)
    b = gen.rhs_uniform(A.n, 1)
    ref = oracle.Hierarchy(A)
    ref.sparsify([0.0, 0.1])
    rp, ci, va = (torch.from_numpy(a).cuda() for a in (A.rowptr, A.col, A.val))
    h = amg.Hierarchy.setup(amg.amg.csr_struct(rp, ci, va), gamma=[0.0, 0.1])
    assert h.num_levels == ref.num_levels == 7
    for l in range(h.num_levels):
        _same_csr(h.export(l, "A"), ref.matrix(l, "A"), rtol=0.0, what=f"A_{l}")
        _same_csr(h.export(l, "Ahat"), ref.matrix(l, "Ahat"), rtol=0.0, what=f"Ahat_{l}")
        if l + 1 < h.num_levels:
            np.testing.assert_array_equal(h.level_array(l, "strong"), ref.strong(l), err_msg=f"S_{l}")
            np.testing.assert_array_equal(h.level_array(l, "cf"), ref.cf(l), err_msg=f"cf_{l}")
            _same_csr(h.export(l, "P"), ref.matrix(l, "P"), rtol=0.0, what=f"P_{l}")
        if l > 0:
            np.testing.assert_array_equal(h.level_array(l, "inM"), ref.inM(l), err_msg=f"inM_{l}")
            np.testing.assert_array_equal(h.level_array(l, "keep"), ref.keep(l), err_msg=f"keep_{l}")
        np.testing.assert_allclose(h.level_array(l, "l1"), ref.l1(l), rtol=1e-14, err_msg=f"l1_{l}")
    bd = torch.from_numpy(b).cuda()
    x, info = h.solve(bd, tol=1e-8)
    xr, ir = ref.pcg(b, tol=1e-8)
    assert info.status == 0 and info.final_relres <= 1e-8
    assert abs(info.iterations - ir.iterations) <= 1
    x = x.cpu().numpy()
    assert np.linalg.norm(x - xr) <= 1e-6 * np.linalg.norm(xr)


@pytest.mark.parametrize("case", ["3d27_11", "hubs"])
def test_setup_two_pass_spgemm_matches_oracle(amg, monkeypatch, case):
    """The counting (two-pass) SpGEMM, used when product bounds do not fit in
    memory, gives the same hierarchy."""
    monkeypatch.setenv("AMG_SPGEMM_TWO_PASS", "1")
    A = CASES[case]()
    ref = oracle.Hierarchy(A)
    h = amg.Hierarchy.setup(A)
    assert h.num_levels == ref.num_levels
    for l in range(h.num_levels):
        _same_csr(h.export(l, "A"), ref.matrix(l, "A"), rtol=0.0, what=f"A_{l}")
        if l + 1 < h.num_levels:
            _same_csr(h.export(l, "P"), ref.matrix(l, "P"), rtol=0.0, what=f"P_{l}")


@pytest.mark.parametrize("gamma", [0.01, 0.1, 1.0])
@pytest.mark.parametrize("case", ["2d5_64", "3d7_20", "fv7_15", "hubs"])
def test_sparsify_end_to_end_matches_oracle(amg, case, gamma):
    A = CASES[case]()
    ref = oracle.Hierarchy(A)
    ref.sparsify([0.0, gamma])
    h = amg.Hierarchy.setup(A, gamma=[0.0, gamma])
    for l in range(1, h.num_levels):
        np.testing.assert_array_equal(h.level_array(l, "keep"), ref.keep(l), err_msg=f"keep_{l}")
        _same_csr(h.export(l, "Ahat"), ref.matrix(l, "Ahat"), what=f"Ahat_{l}")
        np.testing.assert_allclose(h.level_array(l, "l1"), ref.l1(l), rtol=1e-14)
    # re-sparsify in place and reintroduce back to Galerkin
    h.sparsify([0.0, 1.0])
    ref.sparsify([0.0, 1.0])
    for l in range(1, h.num_levels):
        np.testing.assert_array_equal(h.level_array(l, "keep"), ref.keep(l))
    for _ in range(20):
        c1 = h.reintroduce(1)
        c2, _ = ref.reintroduce(1)
        assert c1 == c2
        for l in range(1, h.num_levels):
            np.testing.assert_array_equal(h.level_array(l, "keep"), ref.keep(l))
        if c1 == 0:
            break
    for l in range(h.num_levels):
        np.testing.assert_array_equal(h.export(l, "Ahat").val, h.export(l, "A").val)


@pytest.mark.parametrize("gamma", [0.1, 1.0])
@pytest.mark.parametrize("case", ["3d7_20", "fv7_15", "3d27_11"])
def test_hybrid_end_to_end_matches_oracle(amg, case, gamma):
    """Hybrid Galerkin: M from the sparsified level above; masks bit-exact,
    also along an Algorithm 5 schedule."""
    A = CASES[case]()
    ref = oracle.Hierarchy(A)
    ref.sparsify([0.0, gamma], method=1)
    h = amg.Hierarchy.setup(A, gamma=[0.0, gamma], method=amg.METHOD_HYBRID)
    for l in range(1, h.num_levels):
        np.testing.assert_array_equal(h.level_array(l, "keep"), ref.keep(l), err_msg=f"keep_{l}")
        _same_csr(h.export(l, "Ahat"), ref.matrix(l, "Ahat"), what=f"Ahat_{l}")
    for _ in range(6):
        c1 = h.reintroduce(1)
        c2, _ = ref.reintroduce(1)
        assert c1 == c2
        for l in range(1, h.num_levels):
            np.testing.assert_array_equal(h.level_array(l, "keep"), ref.keep(l))
    if gamma <= 0.1:
        b = gen.rhs_uniform(A.n, 1)
        x, info = h.solve(b)
        xr, ir = ref.pcg(b)
        assert info.status == 0 and abs(info.iterations - ir.iterations) <= 1


def test_per_level_on_oracle_matrices(amg):
    """Given the oracle's own A_l, the GPU's strength/PMIS/interpolation/RAP
    reproduce the oracle's level l (PMIS seeded with the level index)."""
    A = gen.poisson3d_7pt(22)
    ref = oracle.Hierarchy(A)
    for l in range(ref.num_levels - 1):
        Al = ref.matrix(l, "A")
        h = amg.Hierarchy.setup(Al, max_levels=2, max_size=1, level_offset=l)
        assert h.num_levels == 2
        np.testing.assert_array_equal(h.level_array(0, "cf"), ref.cf(l))
        _same_csr(h.export(0, "P"), ref.matrix(l, "P"), what=f"P_{l}")
        _same_csr(h.export(1, "A"), ref.matrix(l + 1, "A"), what=f"A_{l + 1}")
        np.testing.assert_array_equal(h.level_array(1, "inM"), ref.inM(l + 1))


def _assemble_oracle(amg, ref, gamma=None, **opts):
    L = ref.num_levels
    As = [ref.matrix(l, "A") for l in range(L)]
    Ps = [ref.matrix(l, "P") for l in range(L - 1)]
    cfs = [ref.cf(l) for l in range(L - 1)]
    inMs = [None] + [ref.inM(l) for l in range(1, L)]
    return amg.Hierarchy.assemble(As, Ps, cfs, inMs, gamma=gamma, **opts)


@pytest.mark.parametrize("gamma", [0.0, 0.1, 1.0])
def test_sparsify_on_oracle_galerkin(amg, gamma):
    """Kept-entry pattern is bit-exact when given the oracle's Galerkin A_l."""
    A = gen.poisson3d_7pt(24)
    ref = oracle.Hierarchy(A)
    h = _assemble_oracle(amg, ref, gamma=[0.0, gamma])
    ref.sparsify([0.0, gamma])
    for l in range(1, ref.num_levels):
        np.testing.assert_array_equal(h.level_array(l, "keep"), ref.keep(l))
        _same_csr(h.export(l, "Ahat"), ref.matrix(l, "Ahat"), what=f"Ahat_{l}")
        st = h.level_stats(l)
        assert st["nnz_operator"] == ref.matrix(l, "Ahat").nnz


@pytest.mark.parametrize("variant", [-1, 1, 2, 3, 4, 5, 6, 7, 8, 9])
@pytest.mark.parametrize("gamma", [0.0, 0.1])
def test_vcycle_matches_oracle(amg, variant, gamma):
    A = gen.poisson3d_7pt(23)  # n = 12167: ragged against 32-row slices and 256-thread blocks
    ref = oracle.Hierarchy(A)
    ref.sparsify([0.0, gamma])
    h = _assemble_oracle(amg, ref, gamma=[0.0, gamma], spmv_variant=variant)
    for seed in (5, 6):
        r = gen.rhs_uniform(A.n, seed)
        z = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        h.precond_apply(torch.from_numpy(r).cuda(), z)
        zr = ref.vcycle(r)
        np.testing.assert_allclose(z.cpu().numpy(), zr, rtol=1e-12, atol=1e-12 * np.abs(zr).max())


@pytest.mark.parametrize("relax,transfer", [(8, 8), (9, 9), (8, 9), (9, 8), (6, 8), (6, 9), (2, 9)])
@pytest.mark.parametrize("case", ["3d7_23", "3d27_13", "fv7_18"])
def test_vcycle_sell_lanes_matches_oracle(amg, relax, transfer, case):
    """SELL-16 / SELL-8 (two or four lanes per row, rows summed in another
    order than sequentially) for the relaxation and, forced, for the transfers
    P and R, on sizes ragged against every slice height."""
    A = {"3d7_23": lambda: gen.poisson3d_7pt(23), "3d27_13": lambda: gen.poisson3d_27pt(13),
         "fv7_18": lambda: gen.fv7_lognormal(18, seed=3)}[case]()
    ref = oracle.Hierarchy(A)
    ref.sparsify([0.0, 0.1])
    h = _assemble_oracle(amg, ref, gamma=[0.0, 0.1], spmv_variant=relax, transfer_variant=transfer)
    for l in range(h.num_levels - 1):
        st = h.level_stats(l)
        assert (st["spmv_variant"], st["spmv_variant_p"], st["spmv_variant_r"]) == (relax, transfer, transfer)
    for seed in (5, 6):
        r = gen.rhs_uniform(A.n, seed)
        z = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        h.precond_apply(torch.from_numpy(r).cuda(), z)
        zr = ref.vcycle(r)
        np.testing.assert_allclose(z.cpu().numpy(), zr, rtol=1e-12, atol=1e-12 * np.abs(zr).max())
    # the FP32 / BF16 instantiations of the same kernels, inside flexible CG
    b = gen.rhs_uniform(A.n, 1)
    xr, ir = ref.pcg(b, tol=1e-8)
    for prec in (1, 2):
        h2 = amg.Hierarchy.setup(A, gamma=[0.0, 0.1], precision=prec, spmv_variant=relax, transfer_variant=transfer)
        x, info = h2.solve(b, tol=1e-8)
        assert info.status == 0 and info.final_relres <= 1e-8
        assert np.linalg.norm(x - xr) <= 1e-6 * np.linalg.norm(xr)
    for seed in (5, 6):
        r = gen.rhs_uniform(A.n, seed)
        z = torch.zeros(A.n, dtype=torch.float64, device="cuda")
        h.precond_apply(torch.from_numpy(r).cuda(), z)
        zr = ref.vcycle(r)
        np.testing.assert_allclose(z.cpu().numpy(), zr, rtol=1e-12, atol=1e-12 * np.abs(zr).max())


@pytest.mark.parametrize("use_graph", [1, 0])
@pytest.mark.parametrize("case,gamma", [("2d5_64", 0.0), ("3d7_20", 0.1), ("3d7_20", 1.0),
                                        ("fv7_15", 0.1), ("3d27_11", 0.1)])
def test_pcg_matches_oracle(amg, case, gamma, use_graph):
    A = CASES[case]()
    b = gen.rhs_uniform(A.n, 1)
    ref = oracle.Hierarchy(A)
    ref.sparsify([0.0, gamma])
    xr, ir = ref.pcg(b, tol=1e-8)
    h = amg.Hierarchy.setup(A, gamma=[0.0, gamma], use_graph=use_graph)
    for on_dev in (False, True):
        bb = torch.from_numpy(b).cuda() if on_dev else b
        x, info = h.solve(bb, tol=1e-8)
        x = x.cpu().numpy() if on_dev else x
        assert info.status == 0 and info.final_relres <= 1e-8
        assert abs(info.iterations - ir.iterations) <= 1, (info.iterations, ir.iterations)
        assert abs(info.conv_factor - ir.conv_factor) < 0.02
        resid = b - A.to_scipy() @ x
        assert np.linalg.norm(resid) <= 1e-8 * np.linalg.norm(b) * (1 + 1e-6)
        assert np.linalg.norm(x - xr) <= 1e-6 * np.linalg.norm(xr)


@pytest.mark.parametrize("use_graph", [1, 0])
def test_adaptive_matches_oracle(amg, use_graph):
    A = gen.poisson3d_7pt(24)
    b = gen.rhs_uniform(A.n, 1)
    ref = oracle.Hierarchy(A)
    ref.sparsify([0.0, 1.0])
    xr, ir = ref.adaptive_solve(b, rho_max=0.3, s=1, k=3)
    h = amg.Hierarchy.setup(A, gamma=[0.0, 1.0], rho_max=0.3, s_levels=1, k_check=3, use_graph=use_graph)
    x, info = h.solve(b, tol=1e-8, adaptive=True)
    assert info.status == 0 and info.final_relres <= 1e-8
    assert info.resets == ir.resets
    assert abs(info.iterations - ir.iterations) <= 1
    for l in range(h.num_levels):
        assert h.level_stats(l)["gamma"] == pytest.approx(ref.gamma(l), rel=1e-12)


def _shifted_poisson2d(N, sigma):
    """2D 5-point Poisson minus sigma on the diagonal: symmetric, positive
    diagonal, indefinite past the smallest eigenvalue (CG's residual grows)."""
    A = gen.poisson2d_5pt(N)
    A.val = A.val.copy()
    rows = np.repeat(np.arange(A.n), np.diff(A.rowptr))
    A.val[A.col == rows] -= sigma
    return A


@pytest.mark.parametrize("N,sigma,k", [(16, 0.065, 1), (20, 0.045, 2), (20, 0.05, 1)])
@pytest.mark.parametrize("use_graph", [1, 0])
def test_divergence_matches_oracle(amg, N, sigma, k, use_graph):
    """The divergence stop (a window whose residual grew by more than
    div_factor; forced here with div_factor = 1 on indefinite inputs): the
    same status and step count as the oracle, x at the window's start."""
    A = _shifted_poisson2d(N, sigma)
    b = gen.rhs_uniform(A.n, 1)
    ref = oracle.Hierarchy(A, max_size=20)
    xr, ir = ref.pcg(b, max_it=300, k=k, div_factor=1.0)
    assert ir.status == oracle.DIVERGED
    h = amg.Hierarchy.setup(A, max_size=20, k_check=k, div_factor=1.0, use_graph=use_graph)
    x, info = h.solve(b, tol=1e-8, max_it=300)
    assert info.status == amg.DIVERGED
    assert info.iterations == ir.iterations
    assert np.linalg.norm(x - xr) <= 1e-10 * np.linalg.norm(xr)
    # the default factor (1e3) lets the same solve run on (to convergence or a breakdown)
    h2 = amg.Hierarchy.setup(A, max_size=20, k_check=k, use_graph=use_graph)
    _, i2 = h2.solve(b, tol=1e-8, max_it=300)
    _, i2r = ref.pcg(b, max_it=300, k=k)
    assert i2.status == i2r.status != amg.DIVERGED


_ALG5_GPU = {
    # (matrix, gammas, k, s, rho_max, div_factor): indefinite inputs that reach
    # restarts from the window's start, breakdowns and divergence
    "shift_back": (lambda: _shifted_poisson2d(16, 0.2), [0.0, 1.0], 1, 1, 0.5, 0.0),
    "shift_breakdown_back": (lambda: _shifted_poisson2d(24, 0.2), [0.0, 0.0], 2, 1, 0.5, 0.0),
    "shift_restarts_back": (lambda: _shifted_poisson2d(24, 0.2), [0.0, 1.0], 2, 1, 0.5, 0.0),
    "shift_diverged": (lambda: _shifted_poisson2d(16, 0.065), [0.0, 0.0], 1, 1, 0.5, 1.0),
    "aniso_s2": (lambda: gen.rotated_aniso_q1(20), [0.0, 0.1, 1.0], 2, 2, 0.5, 1e3),
}


@pytest.mark.parametrize("case", sorted(_ALG5_GPU))
def test_adaptive_branches_match_oracle(amg, case):
    """Algorithm 5 on the GPU takes the oracle's branch at every window:
    same status, steps, resets and final x (restarts from the window's start,
    final breakdowns and divergence included)."""
    make, gam, k, s, rho_max, divf = _ALG5_GPU[case]
    A = make()
    b = gen.rhs_uniform(A.n, 1)
    ref = oracle.Hierarchy(A, max_size=20)
    ref.sparsify(gam)
    xr, ir, tr = ref.adaptive_solve(b, max_it=300, k=k, s=s, rho_max=rho_max, div_factor=divf, trace=True)
    h = amg.Hierarchy.setup(A, gamma=gam, max_size=20, k_check=k, s_levels=s, rho_max=rho_max, div_factor=divf)
    x, info = h.solve(b, tol=1e-8, max_it=300, adaptive=True)
    assert (info.status, info.iterations, info.resets) == (ir.status, ir.iterations, ir.resets), tr
    assert np.linalg.norm(x - xr) <= 1e-8 * np.linalg.norm(xr)
    for l in range(h.num_levels):
        assert h.level_stats(l)["gamma"] == pytest.approx(ref.gamma(l), rel=1e-12)


@pytest.mark.parametrize("permute", [False, True])
def test_sell_matches_sequential_csr(amg, permute):
    """SELL-32 (int16 column offsets, or int32 columns when a random symmetric
    permutation puts offsets beyond 32767) sums each row in the same order as
    the one-lane CSR kernel; only the dot products' grids differ, so the two
    PCG iterates agree to rounding."""
    import scipy.sparse as sp

    A = gen.poisson2d_5pt(200).to_scipy()
    if permute:
        perm = np.random.default_rng(7).permutation(A.shape[0])
        A = A[perm][:, perm].tocsr()
        A.sort_indices()
    b = gen.rhs_uniform(A.shape[0], 2)
    xs = []
    for variant in (amg.SPMV_SELL32, 7):
        h = amg.Hierarchy.setup(A, gamma=[0.0, 0.1], spmv_variant=variant)
        x, info = h.solve(b, tol=1e-8)
        assert info.status == 0
        xs.append((x, info.iterations))
    assert abs(xs[0][1] - xs[1][1]) <= 1
    assert np.linalg.norm(xs[0][0] - xs[1][0]) <= 1e-9 * np.linalg.norm(xs[1][0])


def test_reintroduce_equals_fresh_setup(amg):
    """Reintroducing entries level by level leaves the hierarchy a fresh setup
    with the resulting tolerances would build: the same operators and, to the
    bit, the same PCG iterate -- with the CUDA graph and without it."""
    A = gen.poisson3d_7pt(64)
    b = gen.rhs_uniform(A.n, 3)
    h = amg.Hierarchy.setup(A, gamma=[0.0, 1.0])
    for _ in range(5):
        assert h.reintroduce(1) == 1
        gam = [h.level_stats(l)["gamma"] for l in range(h.num_levels)]
        x1, i1 = h.solve(b, tol=1e-8)
        assert i1.status == 0
        for use_graph in (1, 0):
            hf = amg.Hierarchy.setup(A, gamma=[0.0] + gam[1:], use_graph=use_graph)
            for l in range(h.num_levels):
                _same_csr(h.export(l, "Ahat"), hf.export(l, "Ahat"), rtol=0.0, what=f"Ahat_{l}")
            x2, i2 = hf.solve(b, tol=1e-8)
            assert i2.iterations == i1.iterations
            np.testing.assert_array_equal(x1, x2)


def test_adaptive_large_converges(amg):
    """Algorithm 5 on the 128^3 benchmark problem from gamma = 1: every check
    that reintroduces entries lowers one level's tolerance, the solve
    converges and the iterate stays finite (a breakdown leaves x untouched
    and a restart falls back to the checkpoint)."""
    A = gen.poisson3d_7pt(128)
    b = gen.rhs_uniform(A.n, 1)
    h = amg.Hierarchy.setup(A, gamma=[0.0, 1.0])
    x, info = h.solve(b, tol=1e-8, adaptive=True)
    assert np.isfinite(x).all()
    assert info.status == 0 and info.final_relres <= 1e-8, info.as_dict()
    gam = [h.level_stats(l)["gamma"] for l in range(h.num_levels)]
    # each reset moved one level one step down the schedule 1 -> 0.1 -> 0.01 -> 0
    steps = sum({1.0: 0, 0.1: 1, 0.01: 2, 0.0: 3}[round(g, 12)] for g in gam[1:])
    assert steps == info.resets


@pytest.mark.parametrize("prec", [1, 2])
def test_mixed_precision_reaches_fp64_tolerance(amg, prec):
    A = gen.poisson3d_27pt(14)
    b = gen.rhs_uniform(A.n, 2)
    ref = oracle.Hierarchy(A)
    ref.sparsify([0.0, 0.1])
    xr, ir = ref.pcg(b, tol=1e-8)
    h = amg.Hierarchy.setup(A, gamma=[0.0, 0.1], precision=prec)
    x, info = h.solve(b, tol=1e-8)
    assert info.status == 0 and info.final_relres <= 1e-8
    assert info.iterations <= ir.iterations + 3
    assert np.linalg.norm(x - xr) <= 1e-6 * np.linalg.norm(xr)


def test_timing_counters(amg):
    """Per-kernel event timing accumulates launches and bytes on every level."""
    A = gen.poisson3d_7pt(20)
    h = amg.Hierarchy.setup(A, gamma=[0.0, 0.1])
    h.timing_enable(True)
    x, info = h.solve(gen.rhs_uniform(A.n, 1))
    assert info.status == 0
    for kind in (amg.K_PRE, amg.K_POST, amg.K_RESTRICT, amg.K_PROLONG):
        for l in range(h.num_levels - 1):
            n, ms, by = h.timing_get(kind, l)
            assert n == info.iterations and ms > 0 and by > 0
    n, ms, by = h.timing_get(amg.K_AP, 0)
    assert n == info.iterations
    h.timing_reset()
    assert h.timing_get(amg.K_PRE, 0)[0] == 0


def test_setup_phase_timing(amg):
    """setup_timing records every setup phase and changes nothing in the result."""
    A = gen.poisson3d_7pt(20)
    h0 = amg.Hierarchy.setup(A, gamma=[0.0, 0.1])
    h1 = amg.Hierarchy.setup(A, gamma=[0.0, 0.1], setup_timing=1)
    L = h1.num_levels
    assert L == h0.num_levels and L >= 3
    for kind in (8, 9, 10, 11, 12):
        for l in range(L - 1):
            n, ms, by = h1.timing_get(kind, l)
            assert n >= 1 and ms > 0 and by == 0, (kind, l)
    for l in range(1, L):
        assert h1.timing_get(13, l)[0] == 1
    for l in range(L):
        assert h1.timing_get(14, l)[0] >= 1
    assert h1.timing_get(15, L - 1)[0] == 1
    for l in range(L):
        for which in ("A", "Ahat"):
            _same_csr(h1.export(l, which), h0.export(l, which), rtol=0.0, what=f"{which}_{l}")
    # solve-phase timing stays off unless asked for
    h1.solve(gen.rhs_uniform(A.n, 1))
    assert h1.timing_get(amg.K_PRE, 0)[0] == 0


def test_single_level_and_zero_rhs(amg):
    A = gen.poisson2d_5pt(9)
    h = amg.Hierarchy.setup(A, max_size=1000)
    assert h.num_levels == 1
    b = gen.rhs_uniform(A.n, 0)
    x, info = h.solve(b)
    assert info.iterations == 1 and info.status == 0
    x, info = h.solve(np.zeros(A.n))
    assert info.iterations == 0 and not x.any()


def test_tiny_matrix(amg):
    import scipy.sparse as sp

    A = sp.csr_matrix(np.array([[2.0]]))
    h = amg.Hierarchy.setup(A)
    x, info = h.solve(np.array([3.0]))
    assert info.status == 0 and abs(x[0] - 1.5) < 1e-14
    # 2 x 2 SPD with both couplings: one level (below max_size), direct solve
    A2 = sp.csr_matrix(np.array([[4.0, -1.0], [-1.0, 3.0]]))
    h2 = amg.Hierarchy.setup(A2)
    x2, info2 = h2.solve(np.array([1.0, 2.0]))
    np.testing.assert_allclose(x2, np.linalg.solve(A2.toarray(), [1.0, 2.0]), rtol=1e-13)
    # an empty matrix is rejected, not set up
    E = amg.amg.csr_struct(np.zeros(1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    with pytest.raises(amg.AmgError) as e:
        amg.Hierarchy.setup(E)
    assert e.value.status == 1


def test_invalid_device_structures_rejected(amg):
    """Row pointers and indices that would lead a kernel outside its arrays
    are reported as AMG_ERR_INVALID by the kernels' own range checks."""
    import copy

    import torch

    A = gen.poisson2d_5pt(12)
    rp, ci, va = (torch.from_numpy(np.array(a)).cuda() for a in (A.rowptr, A.col, A.val))

    def expect_invalid_dev(rp_, ci_, va_):
        M = amg.amg.csr_struct(rp_, ci_, va_)
        with pytest.raises(amg.AmgError) as e:
            amg.Hierarchy.setup(M)
        assert e.value.status == 1

    bad_rp = rp.clone()
    bad_rp[5] = bad_rp[7] + 3  # row 4 ends past row 5's end: pointers out of order
    expect_invalid_dev(bad_rp, ci, va)
    bad_rp = rp.clone()
    bad_rp[3] = -4
    expect_invalid_dev(bad_rp, ci, va)
    bad_ci = ci.clone()
    bad_ci[10] = A.n + 1000
    expect_invalid_dev(rp, bad_ci, va)
    bad_ci = ci.clone()
    bad_ci[10] = -7
    expect_invalid_dev(rp, bad_ci, va)
    # still usable afterwards
    h = amg.Hierarchy.setup(amg.amg.csr_struct(rp, ci, va))
    assert h.solve(gen.rhs_uniform(A.n, 0))[1].status == 0

    # caller-given interpolation with a column outside [0, n_{l+1})
    ref = oracle.Hierarchy(gen.poisson3d_7pt(12))
    L = ref.num_levels
    As = [ref.matrix(l, "A") for l in range(L)]
    Ps = [copy.deepcopy(ref.matrix(l, "P")) for l in range(L - 1)]
    cfs = [ref.cf(l) for l in range(L - 1)]
    inMs = [None] + [ref.inM(l) for l in range(1, L)]
    Ps[0].col[3] = As[1].nrows + 5
    with pytest.raises(amg.AmgError) as e:
        amg.Hierarchy.assemble(As, Ps, cfs, inMs)
    assert e.value.status == 1
    # C/F markers whose C count differs from the coarse size (hybrid pattern path)
    Ps = [ref.matrix(l, "P") for l in range(L - 1)]
    cfs = [np.array(c, copy=True) for c in cfs]
    assert L >= 3
    cfs[1][np.flatnonzero(cfs[1] == -1)[0]] = 1  # the hybrid pattern of level 2 numbers level 1's C points
    with pytest.raises(amg.AmgError) as e:
        amg.Hierarchy.assemble(As, Ps, cfs, inMs, gamma=[0.0, 0.1], method=1)
    assert e.value.status == 1


def test_invalid_inputs_rejected(amg):
    import scipy.sparse as sp

    good = gen.poisson2d_5pt(6).to_scipy()

    def expect_invalid(M, **kw):
        with pytest.raises(amg.AmgError) as e:
            amg.Hierarchy.setup(M, **kw)
        assert e.value.status == 1

    bad = good.copy()
    bad.data[bad.indptr[3]] = np.nan
    expect_invalid(bad)
    d = good.toarray()
    d[4, 4] = -1.0
    expect_invalid(sp.csr_matrix(d))
    d = good.toarray()
    d[0, 5] = -0.5  # breaks pattern symmetry
    expect_invalid(sp.csr_matrix(d))
    d = good.toarray()
    d[2, 2] = 0.0
    m = sp.csr_matrix(d)
    m.eliminate_zeros()
    expect_invalid(m)  # missing diagonal
    unsorted = good.copy()
    r0 = slice(unsorted.indptr[7], unsorted.indptr[8])
    unsorted.indices[r0] = unsorted.indices[r0][::-1].copy()
    unsorted.data[r0] = unsorted.data[r0][::-1].copy()
    expect_invalid(unsorted)
    expect_invalid(good, gamma=[0.5, 0.1])  # gamma_0 must be 0
    # non-finite right-hand sides, host and device, single and batched
    import torch

    h = amg.Hierarchy.setup(good)
    bad_b = np.ones(good.shape[0])
    bad_b[5] = np.inf
    for rhs in (bad_b, torch.from_numpy(bad_b).cuda()):
        with pytest.raises(amg.AmgError) as e:
            h.solve(rhs)
        assert e.value.status == 1
    B = np.ones((good.shape[0], 3))
    B[7, 1] = np.nan
    with pytest.raises(amg.AmgError) as e:
        h.solve_batch(B)
    assert e.value.status == 1
    x, info = h.solve(np.ones(good.shape[0]))  # still usable
    assert info.status == 0
    expect_invalid(sp.csr_matrix(np.ones((2, 3))))
