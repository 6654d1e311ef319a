"""The enumerator's paper-style statistics against the values the paper
prints (Table I: distinct minima per orbit; Table III: global-minimum
F/(dV)), over random uniform orbits at omega = 1 as in the paper, through the
library's mixed path.  Tolerance: 3.5 standard errors of the difference of two
sample means (the paper's 100 orbits, ours)."""
import json
import math
import os

import pytest

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")


@pytest.mark.parametrize("d,N", [(2, 2), (2, 4), (3, 2), (4, 2)])
def test_tables_I_and_III_on_the_gpu(d, N):
    from paper_1403_0555_b300.analysis import table_statistics
    g = json.load(open(GOLDEN))
    t1 = next(r for r in g["table_I"]["rows"] if r["d"] == d and r["N"] == N)
    t3 = next(r for r in g["table_III"]["rows"] if r["d"] == d and r["N"] == N)
    n_orbits = 100
    st = table_statistics(d, N, n_orbits, 1 << 20, omega=1.0, curve=True)
    m1, s1 = st["minima_F8"]
    se1 = math.sqrt(t1["std"] ** 2 / t1["orbits"] + s1 ** 2 / n_orbits)
    assert abs(m1 - t1["avg_minima"]) < 3.5 * se1, (st, t1)
    m3, s3 = st["global_min_F_per_link"]
    se3 = math.sqrt(t3["std"] ** 2 / t3["orbits"] + s3 ** 2 / n_orbits)
    assert abs(m3 - t3["avg_Fmin"]) < 3.5 * se3, (st, t3)
    # the discovery curve is non-decreasing and ends at the per-orbit copy count
    c = st["curve_mean"]
    assert all(b >= a for a, b in zip(c, c[1:]))
    assert abs(c[-1] - st["copies"][0]) < 1e-9
    assert st["converged_fraction"][0] > 0.999


def test_section_iv_distributions_match_the_oracle():
    """The 2D 4^2 parity workload (uniform orbit, seed 1, 10^4 starts, plain
    FP64 path): the sample-weighted histogram of F/(dV) at the resolution of
    Fig. 5, the relative deviations from the global minimum (Fig. 8) and the
    F-quantised minima count equal the oracle's."""
    import numpy as np
    import oracle
    import orbit_inputs as oi
    import paper_1403_0555_b300 as gb
    from paper_1403_0555_b300 import analysis as an
    w = oi.workload_2d_4x4()
    o = w.orbits[0]
    d, L, n = o.d, o.L, w.n_starts
    V = L ** d
    _, ref = oracle.enumerate_copies(d, L, o.phi, 1, o.orbit_id, n, w.omega, w.eps)
    h = gb.gc_create_orbit(d, L, o.phi, o.orbit_id)
    try:
        gb.gc_enumerate_copies(h, n, w.omega, w.eps, gb.gc_options_default(precision=gb.GC_FP64, check_every=1))
        st = gb.gc_orbit_stats(h)
        c = gb.gc_fetch_copies(h, V)
    finally:
        gb.gc_destroy_orbit(h)
    bo, co = an.minima_histogram(ref.F / (d * V), ref.count)
    bg, cg = an.minima_histogram(c["F"] / (d * V), c["count"])
    assert np.array_equal(bo, bg) and np.array_equal(co, cg)
    r = an.histogram_ratio(bg, cg, bo, co)
    assert np.all(r["ratio"] == 1.0) and len(r["only_a"]) == 0 and len(r["only_b"]) == 0
    assert np.allclose(an.relative_deviation(c["F"]), an.relative_deviation(ref.F), rtol=0, atol=1e-12)
    assert st["n_distinct_F8"] == ref.n_distinct_F8


def test_section_iv_histogram_ratio_of_two_sample_sizes():
    """Fig. 5 on a small case: 2D 6^2, uniform orbits, 2^12 against 2^16 starts,
    mixed path.  The longer run's first 2^12 starts are the shorter run, so
    every bin of the short run is a bin of the long one, no bin count falls,
    the ratio of all entries is 16, and well-filled bins sit near it."""
    import numpy as np
    import orbit_inputs as oi
    import paper_1403_0555_b300 as gb
    from paper_1403_0555_b300 import analysis as an
    d, L = 2, 6
    V = L ** d
    for seed in (1, 2):
        phi = oi.uniform_orbit(d, L, seed)
        hist = {}
        for n in (1 << 12, 1 << 16):
            h = gb.gc_create_orbit(d, L, phi, seed)
            try:
                gb.gc_enumerate_copies(h, n, 1.0, 1e-24, gb.gc_options_default(precision=gb.GC_MIXED))
                st = gb.gc_orbit_stats(h)
                c = gb.gc_fetch_copies(h, V)
            finally:
                gb.gc_destroy_orbit(h)
            assert st["n_converged"] == n
            hist[n] = an.minima_histogram(c["F"] / (d * V), c["count"])
        (bl, cl), (bs, cs) = hist[1 << 16], hist[1 << 12]
        r = an.histogram_ratio(bl, cl, bs, cs)
        assert len(r["only_b"]) == 0                       # no bin of the short run is missing
        assert np.all(r["ratio"] >= 1.0)
        assert cl.sum() / cs.sum() == 16.0
        c_short = cs[np.searchsorted(bs, r["bins"])]
        full = c_short >= 200
        # ratio = 1 + X / c with X the long run's other 15 x 2^12 samples in the
        # bin: relative spreads 1/sqrt(15 c) and 1/sqrt(c), so within 6 sigma
        sig = 15.0 * np.sqrt(1.0 / (15.0 * c_short[full]) + 1.0 / c_short[full])
        assert np.all(np.abs(r["ratio"][full] - 16.0) <= 6.0 * sig)
        # relative deviations are non-negative and vanish at the global minimum
        rd = an.relative_deviation(np.unique(np.floor(c["F"] / (d * V) * 1e8)) * 1e-8)
        assert rd.min() == 0.0 and np.all(rd >= 0)
