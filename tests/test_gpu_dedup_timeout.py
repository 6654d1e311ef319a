"""A device-side bounded wait that runs out: the copy table's lock wait.

With every bucket lock of the table held (gc_test_dedup_locks) and a budget of
a few dozen tries, the starts of a call whose copies are not in the table yet
cannot insert them.  Their waits end after the budget, the kernel marks them
GC_START_DEDUP_FAILED and returns, and the call reports GC_ETIMEDOUT; nothing
waits without limit.  Every other start (its copy was found in the first call,
a lock-free search) has exactly the result of an undisturbed run, and once the
locks are freed the orbit enumerates normally.  Plain FP64 path: start by start
identical to the undisturbed run.
"""
import numpy as np
import pytest

import orbit_inputs as oi
from gpu_helpers import wrap

pytestmark = pytest.mark.gpu


def test_lock_wait_runs_out_marks_starts_and_reports_timeout():
    import paper_1403_0555_b300 as gb
    d, L = 2, 6
    phi = oi.uniform_orbit(d, L, 1)
    n1, n2, n3 = 300, 2000, 200
    opt = gb.gc_options_default(precision=gb.GC_FP64, check_every=1, keep_per_start=1, fp_mode=gb.GC_FP_NONE)
    # undisturbed run, the same three calls
    ref = gb.gc_create_orbit(d, L, phi, 1, n1 + n2 + n3)
    try:
        gb.gc_enumerate_copies(ref, n1, 1.7, 1e-24, opt)
        gb.gc_enumerate_copies(ref, n2, 1.7, 1e-24, opt)
        rs = gb.gc_fetch_starts(ref, n1, n2)
        rc = gb.gc_fetch_copies(ref, L ** d)
    finally:
        gb.gc_destroy_orbit(ref)
    h = gb.gc_create_orbit(d, L, phi, 1, n1 + n2 + n3)
    try:
        gb.gc_enumerate_copies(h, n1, 1.7, 1e-24, opt)
        n_before = gb.gc_orbit_stats(h)["n_distinct"]
        gb.gc_test_dedup_locks(h, True, 32)
        with pytest.raises(gb.GribovError) as e:
            gb.gc_enumerate_copies(h, n2, 1.7, 1e-24, opt)
        assert e.value.code == gb.GC_ETIMEDOUT
        s = gb.gc_fetch_starts(h, n1, n2)
        st = gb.gc_orbit_stats(h)
        c = gb.gc_fetch_copies(h, L ** d)
        # a start fails exactly when its copy was first reached in the second call
        first_of_start = rc["first_start"][rs["copy_idx"]].astype(np.int64)
        new_copy = first_of_start >= n1
        failed = s["status"] == gb.GC_START_DEDUP_FAILED
        print(f"\n{int(failed.sum())} of {n2} starts reached copies not in the table; "
              f"{n_before} copies before, {c['n_distinct']} after")
        assert failed.sum() > 0 and (~failed).sum() > 0
        assert np.array_equal(failed, new_copy)
        assert st["n_dedup_failed"] == int(failed.sum())
        assert c["n_distinct"] == n_before
        assert np.all(s["copy_idx"][failed] == -1)
        ok = ~failed
        assert np.array_equal(s["status"][ok], rs["status"][ok])
        assert np.array_equal(s["sweeps"], rs["sweeps"])          # the relaxation itself is untouched
        assert np.array_equal(s["F"], rs["F"])
        th = c["theta"][s["copy_idx"][ok]]
        th_ref = rc["theta"][rs["copy_idx"][ok]]
        assert np.max(np.abs(wrap(th - th_ref))) <= 1e-12
        # the locks freed and the default budget back: the orbit enumerates normally
        gb.gc_test_dedup_locks(h, False, 0)
        gb.gc_enumerate_copies(h, n3, 1.7, 1e-24, opt)
        s3 = gb.gc_fetch_starts(h, n1 + n2, n3)
        assert np.all(s3["status"] == gb.GC_START_CONVERGED)
        assert gb.gc_orbit_stats(h)["n_dedup_failed"] == int(failed.sum())
    finally:
        gb.gc_destroy_orbit(h)


def test_lock_hook_arguments():
    import paper_1403_0555_b300 as gb
    h = gb.gc_create_orbit(2, 4, oi.uniform_orbit(2, 4, 1), 1)
    try:
        with pytest.raises(gb.GribovError) as e:
            gb.gc_test_dedup_locks(h, True, -1)
        assert e.value.code == gb.GC_EINVAL
    finally:
        gb.gc_destroy_orbit(h)
