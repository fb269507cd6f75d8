"""Row-partitioned execution (amg_partition) on one GPU.

Every level is split into blocks of rows, each operator gets its halo plan,
and every product first gathers each block's ghost values (the exchange a
distributed run performs by messages), then multiplies owned columns and
ghosts.  Rows keep their stored order, so a partitioned solve must equal,
bit for bit, the unpartitioned solve whose kernels run one lane per row --
and the oracle within the usual tolerances.  The communication statistics
are checked against ghost sets computed with numpy from the exported
operators and block boundaries.
"""
import numpy as np
import pytest

import amg_inputs as gen
import oracle

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

ONE_LANE = dict(spmv_variant=7, transfer_variant=7)  # AMG_SPMV_CSR1 everywhere


@pytest.fixture(scope="module")
def amg():
    from paper_1512_04629_gb300 import build

    build.build()
    import paper_1512_04629_gb300 as m

    return m


CASES = {
    "3d7_24": lambda: gen.poisson3d_7pt(24),
    "2d5_61": lambda: gen.poisson2d_5pt(61),
    "fv7_17": lambda: gen.fv7_lognormal(17, seed=3),
    "aniso_40": lambda: gen.rotated_aniso_q1(40),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("parts", [2, 3, 8, 64])
def test_partitioned_solve_is_bit_identical(amg, case, parts):
    A = CASES[case]()
    b = gen.rhs_uniform(A.n, 1)
    gam = [0.0, 0.1]
    ref = amg.Hierarchy.setup(A, gamma=gam, **ONE_LANE)
    h = amg.Hierarchy.setup(A, gamma=gam, **ONE_LANE)
    h.partition(parts)
    for seed in (5, 6):
        r = torch.from_numpy(gen.rhs_uniform(A.n, seed)).cuda()
        z0, z1 = torch.zeros_like(r), torch.zeros_like(r)
        ref.precond_apply(r, z0)
        h.precond_apply(r, z1)
        assert torch.equal(z0, z1)
    x0, i0 = ref.solve(b, tol=1e-8)
    x1, i1 = h.solve(b, tol=1e-8)
    assert i1.status == 0 and i1.iterations == i0.iterations
    np.testing.assert_array_equal(x1, x0)
    # and against the oracle
    o = oracle.Hierarchy(A)
    o.sparsify(gam)
    r = gen.rhs_uniform(A.n, 5)
    z = torch.zeros(A.n, dtype=torch.float64, device="cuda")
    h.precond_apply(torch.from_numpy(r).cuda(), z)
    zr = o.vcycle(r)
    np.testing.assert_allclose(z.cpu().numpy(), zr, rtol=1e-12, atol=1e-12 * np.abs(zr).max())
    xr, ir = o.pcg(b, tol=1e-8)
    assert abs(i1.iterations - ir.iterations) <= 1
    assert np.linalg.norm(x1 - xr) <= 1e-6 * np.linalg.norm(xr)
    # removing the split gives the unpartitioned solve back
    h.partition(1)
    x2, i2 = h.solve(b, tol=1e-8)
    np.testing.assert_array_equal(x2, x0)


def _ghost_counts(M, row0, col0):
    parts = len(row0) - 1
    owner = np.searchsorted(col0, np.arange(M.shape[1]), side="right") - 1
    msgs = vals = 0
    per = []
    for p in range(parts):
        cols = M[row0[p]:row0[p + 1]].indices
        g = np.unique(cols[(cols < col0[p]) | (cols >= col0[p + 1])])
        q = np.unique(owner[g])
        msgs += len(q)
        vals += len(g)
        per.append((len(q), len(g)))
    return msgs, vals, per


@pytest.mark.parametrize("gamma", [0.0, 0.1, 1.0])
def test_comm_stats_match_ghost_sets(amg, gamma):
    A = gen.poisson3d_7pt(32)
    h = amg.Hierarchy.setup(A, gamma=[0.0, gamma])
    parts = 8
    h.partition(parts)
    L = h.num_levels
    for l in range(L):
        row0 = h.partition_rows(l)
        assert row0[0] == 0 and row0[-1] == h.level_stats(l)["n"] and np.all(np.diff(row0) >= 0)
        st = h.comm_stats(l)
        assert st["parts"] == parts
        Ah = h.export(l, "Ahat").to_scipy()
        Ag = h.export(l, "A").to_scipy()
        m, v, per = _ghost_counts(Ah, row0, row0)
        assert (st["messages"], st["halo_values"]) == (m, v)
        assert st["max_messages"] == max(a for a, _ in per) and st["max_halo"] == max(b for _, b in per)
        assert (st["messages_galerkin"], st["halo_galerkin"]) == _ghost_counts(Ag, row0, row0)[:2]
        if l + 1 < L:
            c0 = h.partition_rows(l + 1)
            # a block keeps the C points of its own rows
            cf = h.level_array(l, "cf")
            for p in range(parts):
                assert (cf[row0[p]:row0[p + 1]] == 1).sum() == c0[p + 1] - c0[p]
            P = h.export(l, "P").to_scipy()
            R = h.export(l, "R").to_scipy()
            assert (st["messages_p"], st["halo_p"]) == _ghost_counts(P, row0, c0)[:2]
            assert (st["messages_r"], st["halo_r"]) == _ghost_counts(R, c0, row0)[:2]
        if gamma == 0.0:
            assert (st["messages"], st["halo_values"]) == (st["messages_galerkin"], st["halo_galerkin"])


def test_sparsification_cuts_coarse_communication(amg):
    """The paper's point (Sections 3-4): dropping weak coarse entries removes
    ghost values and messages on the coarse levels."""
    A = gen.poisson3d_7pt(48)
    tot = {}
    for g in (0.0, 0.1, 1.0):
        h = amg.Hierarchy.setup(A, gamma=[0.0, g])
        h.partition(16)
        st = [h.comm_stats(l) for l in range(1, h.num_levels)]
        tot[g] = (sum(s["messages"] for s in st), sum(s["halo_values"] for s in st))
        for s in st:
            assert s["messages"] <= s["messages_galerkin"] and s["halo_values"] <= s["halo_galerkin"]
    assert tot[0.1][1] < tot[0.0][1] and tot[1.0][1] < tot[0.1][1]
    assert tot[1.0][0] < tot[0.0][0]


@pytest.mark.parametrize("what", ["adaptive", "gmres", "graph_off"])
def test_partitioned_paths_match_unpartitioned(amg, what):
    A = gen.poisson3d_7pt(20)
    b = gen.rhs_uniform(A.n, 2)
    kw = dict(ONE_LANE)
    if what == "gmres":
        kw["krylov"] = amg.KRYLOV_GMRES
    if what == "graph_off":
        kw["use_graph"] = 0
    gam = [0.0, 1.0] if what == "adaptive" else [0.0, 0.1]
    ref = amg.Hierarchy.setup(A, gamma=gam, rho_max=0.3, **kw)
    h = amg.Hierarchy.setup(A, gamma=gam, rho_max=0.3, **kw)
    h.partition(4)
    x0, i0 = ref.solve(b, tol=1e-8, adaptive=(what == "adaptive"))
    x1, i1 = h.solve(b, tol=1e-8, adaptive=(what == "adaptive"))
    assert (i1.status, i1.iterations, i1.resets) == (i0.status, i0.iterations, i0.resets)
    np.testing.assert_array_equal(x1, x0)
    if what == "adaptive":
        assert i1.resets >= 1  # reintroduction re-planned the changed levels
        for l in range(1, h.num_levels):
            Ah = h.export(l, "Ahat").to_scipy()
            row0 = h.partition_rows(l)
            assert (h.comm_stats(l)["halo_values"]) == _ghost_counts(Ah, row0, row0)[1]


def test_partition_rejects_reduced_precision_and_bad_counts(amg):
    A = gen.poisson2d_5pt(20)
    h = amg.Hierarchy.setup(A, precision=1)
    with pytest.raises(amg.AmgError) as e:
        h.partition(2)
    assert e.value.status == amg.ERR_INVALID
    h = amg.Hierarchy.setup(A)
    for bad in (0, 65):
        with pytest.raises(amg.AmgError):
            h.partition(bad)
    x, info = h.solve(gen.rhs_uniform(A.n, 1), tol=1e-8)  # still usable, unpartitioned
    assert info.status == 0
