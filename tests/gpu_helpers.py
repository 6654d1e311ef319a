"""Shared helpers of the GPU tests: run the library and the oracle on one input."""
import numpy as np

import oracle


def run_gpu(d, L, phi, orbit_id, n, omega=1.7, eps=1e-24, calls=None, **opts):
    import paper_1403_0555_b300 as gb
    opts.setdefault("keep_per_start", 1)
    opt = gb.gc_options_default(**opts)
    h = gb.gc_create_orbit(d, L, phi, orbit_id)
    try:
        for m in (calls or [n]):
            gb.gc_enumerate_copies(h, m, omega, eps, opt)
        last = (calls or [n])[-1]
        starts = gb.gc_fetch_starts(h, n - last, last) if opt.keep_per_start else None
        copies = gb.gc_fetch_copies(h, L ** d)
        stats = gb.gc_orbit_stats(h)
    finally:
        gb.gc_destroy_orbit(h)
    return starts, copies, stats


def wrap(a):
    return np.angle(np.exp(1j * np.asarray(a)))


def assert_copies_equal(gpu, orc, theta_tol=1e-9, f_tol=1e-12, lam_tol=None):
    """Distinct-copy sets equal: count, order, F, first_start, multiplicity, angles."""
    n = len(orc.F)
    assert gpu["n_distinct"] == n
    assert np.array_equal(gpu["first_start"].astype(np.int64), orc.first_start)
    assert np.array_equal(gpu["count"].astype(np.int64), orc.count)
    assert np.all(np.abs(gpu["F"] - orc.F) <= f_tol * np.maximum(1.0, np.abs(orc.F)))
    if n:
        assert np.max(np.abs(wrap(gpu["theta"] - orc.theta))) <= theta_tol
    if lam_tol is not None:
        assert np.all(np.abs(gpu["lambda2"] - orc.lambda2) <= lam_tol)
        assert np.array_equal(gpu["region"], orc.region)


def assert_starts_equal(gs, relaxed, orc_copies, F_or, f_tol=1e-12):
    assert np.array_equal(gs["status"], relaxed.status.astype(np.int32))
    assert np.array_equal(gs["sweeps"], relaxed.sweeps)
    conv = relaxed.status == oracle.CONVERGED
    assert np.all(np.abs(gs["F"][conv] - F_or[conv]) <= f_tol * np.maximum(1.0, np.abs(F_or[conv])))
    assert np.array_equal(gs["copy_idx"], orc_copies.copy_of_start)
