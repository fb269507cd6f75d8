"""Setups issued from several host threads at once.

Every amg_setup runs its own setup pipeline: a second host thread and two
more streams beside the coarsening.  Several such setups at the same time,
on the caller's current (shared) stream or on streams of their own, must
each give the hierarchy a lone setup gives -- the same bits on every level
(operators, interpolation, sparsified operators) and the same solve.
"""
import threading

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


CASES = [
    lambda: gen.poisson3d_7pt(28),
    lambda: gen.poisson3d_27pt(16),
    lambda: gen.fv7_lognormal(20, seed=4),
    lambda: gen.poisson2d_5pt(96),
]


def _snapshot(h):
    out = []
    for l in range(h.num_levels):
        for what in ("A", "Ahat") + (("P", "R") if l + 1 < h.num_levels else ()):
            M = h.export(l, what)
            out.append((l, what, M.rowptr.copy(), M.col.copy(), M.val.copy()))
    return out


def _same(a, b):
    assert len(a) == len(b)
    for (l, w, r0, c0, v0), (_, _, r1, c1, v1) in zip(a, b):
        assert np.array_equal(r0, r1) and np.array_equal(c0, c1), (l, w)
        assert np.array_equal(v0, v1), (l, w)


@pytest.mark.parametrize("own_streams", [False, True])
def test_concurrent_setups_equal_lone_setups(amg, own_streams):
    mats = [c() for c in CASES]
    gam = [0.0, 0.1]
    ref = []
    for A in mats:
        h = amg.Hierarchy.setup(A, gamma=gam)
        x, info = h.solve(gen.rhs_uniform(A.n, 1), tol=1e-8)
        ref.append((_snapshot(h), x, info.iterations))
        del h
    for _ in range(2):
        results = [None] * len(mats)
        errors = []

        def work(k):
            try:
                if own_streams:
                    s = torch.cuda.Stream()
                    with torch.cuda.stream(s):
                        h = amg.Hierarchy.setup(mats[k], gamma=gam, stream=s.cuda_stream)
                        s.synchronize()
                else:
                    h = amg.Hierarchy.setup(mats[k], gamma=gam)
                results[k] = h
            except Exception as e:  # reported below, in the main thread
                errors.append((k, e))

        threads = [threading.Thread(target=work, args=(k,)) for k in range(len(mats))]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
        assert not errors, errors
        torch.cuda.synchronize()
        for k, h in enumerate(results):
            snap, x_ref, its = ref[k]
            _same(_snapshot(h), snap)
            x, info = h.solve(gen.rhs_uniform(mats[k].n, 1), tol=1e-8)
            assert info.status == 0 and info.iterations == its
            np.testing.assert_array_equal(x, x_ref)
