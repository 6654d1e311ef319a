"""The plain FP64 path on the 3D 6^3 workload, every orbit in full, against the
oracle: 4 von Mises(kappa = 1) orbits (seeds 1-4) and the cold orbit hidden
by a random gauge (seed 5), 10^5 starts each, omega = 1.7, eps = 1e-24, dense
first-region test.

The plain path repeats the oracle's operations in its order (Section III's
relaxation, Eq. 3, the canonical copy of Section II), so it must give the
oracle's results start by start (status, sweep count, F, copy) and the same
distinct-copy table: count, order, F, canonical angles, first start,
multiplicity, lambda_2 and region flag of every copy.
"""
import numpy as np
import pytest

import oracle
import orbit_inputs as oi
from gpu_helpers import assert_copies_equal, assert_starts_equal, oracle_pool, run_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("which", [0, 1, 2, 3, 4])
def test_config2_plain_full_copy_set(which):
    import paper_1403_0555_b300 as gb
    w = oi.workload_3d_6cubed()
    o = w.orbits[which]
    d, L, n = o.d, o.L, w.n_starts
    gs, gc, st = run_gpu(d, L, o.phi, o.orbit_id, n, omega=w.omega, eps=w.eps, precision=gb.GC_FP64,
                         check_every=1, fp_mode=gb.GC_FP_DENSE)
    assert st["n_starts"] == n and st["n_dedup_failed"] == 0
    with oracle_pool() as pool:
        relaxed, cp = oracle.enumerate_copies(d, L, o.phi, 1, o.orbit_id, n, w.omega, w.eps,
                                              lam_map=lambda f, it: pool.map(f, it, chunksize=256))
    _, th = oracle.canonical(relaxed.g)
    F_or = oracle.functional(d, L, o.phi, th)
    print(f"\n{o.name}: {cp.F.size} distinct copies of {n} starts, {int((relaxed.status == 1).sum())} converged, "
          f"region IN/MARGINAL/OUT {[(cp.region == r).sum() for r in (1, 2, 0)]}, n_distinct_F8 {cp.n_distinct_F8}")
    assert_starts_equal(gs, relaxed, cp, F_or, gpu_copies=gc)
    assert_copies_equal(gc, cp, theta_tol=1e-9, f_tol=1e-12, lam_tol=1e-10)
    assert st["n_distinct"] == cp.F.size
    assert st["n_distinct_F8"] == cp.n_distinct_F8
