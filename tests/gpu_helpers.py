"""Shared helpers of the GPU tests: run the library and the oracle on one input."""
import os

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
    """Distinct-copy sets equal: count, F, first_start, multiplicity, angles
    (and lambda_2 / region with lam_tol), copy by copy.  Copies are matched by
    their first start, which is unique per copy.  Both tables are sorted by
    (F, first_start); where two copies' F agree to rounding (symmetric images
    of one minimum), the rounding of F decides their order, so the order is
    checked only to be non-decreasing in F within f_tol."""
    n = len(orc.F)
    assert gpu["n_distinct"] == n
    pg = np.argsort(gpu["first_start"].astype(np.int64), kind="stable")
    po = np.argsort(orc.first_start, kind="stable")
    assert np.array_equal(gpu["first_start"].astype(np.int64)[pg], orc.first_start[po])
    assert np.array_equal(gpu["count"].astype(np.int64)[pg], orc.count[po])
    Fg, Fo = gpu["F"][pg], orc.F[po]
    assert np.all(np.abs(Fg - Fo) <= f_tol * np.maximum(1.0, np.abs(Fo)))
    assert np.all(np.diff(gpu["F"]) >= -f_tol * np.maximum(1.0, np.abs(gpu["F"][1:])))
    if n:
        assert np.max(np.abs(wrap(gpu["theta"][pg] - orc.theta[po]))) <= theta_tol
    if lam_tol is not None:
        assert np.all(np.abs(gpu["lambda2"][pg] - orc.lambda2[po]) <= lam_tol)
        assert np.array_equal(gpu["region"][pg], orc.region[po])


def assert_starts_equal(gs, relaxed, orc_copies, F_or, f_tol=1e-12, gpu_copies=None):
    """Per start: status, sweeps, F, and the copy it reached (the same copy:
    identified by the copy's first start when gpu_copies is given, else by
    position in the sorted table)."""
    assert np.array_equal(gs["status"], relaxed.status.astype(np.int32))
    assert np.array_equal(gs["sweeps"], relaxed.sweeps)
    conv = relaxed.status == oracle.CONVERGED
    assert np.all(np.abs(gs["F"][conv] - F_or[conv]) <= f_tol * np.maximum(1.0, np.abs(F_or[conv])))
    if gpu_copies is None:
        assert np.array_equal(gs["copy_idx"], orc_copies.copy_of_start)
        return
    assert np.array_equal(gs["copy_idx"] >= 0, orc_copies.copy_of_start >= 0)
    ok = orc_copies.copy_of_start >= 0
    assert np.array_equal(gpu_copies["first_start"].astype(np.int64)[gs["copy_idx"][ok]],
                          orc_copies.first_start[orc_copies.copy_of_start[ok]])


class oracle_pool:
    """Process pool for the oracle's per-copy work (spawned, so it is safe
    after CUDA has been initialised in this process), one BLAS thread per
    worker so the workers do not oversubscribe the host cores."""

    def __init__(self, processes=None):
        self.processes = processes or min(16, os.cpu_count() or 1)

    def __enter__(self):
        import multiprocessing as mp
        keys = ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")
        old = {k: os.environ.get(k) for k in keys}
        for k in keys:
            os.environ[k] = "1"
        try:
            self.pool = mp.get_context("spawn").Pool(self.processes)
        finally:
            for k, v in old.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        return self.pool

    def __exit__(self, *exc):
        self.pool.terminate()
        self.pool.join()
        return False
