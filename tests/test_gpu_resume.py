"""Checkpoint / resume (gc_load_copies).  A run broken after n1 starts, its
fetched copies and quantised minima restored into a new orbit and continued
for n2 starts, gives what the run continued without the break gives: the same
copy set, F, counts, first starts, lambda_2 and region flags, the same
quantised minima, and the angles to rounding (the restored configurations
are rebuilt from them)."""
import numpy as np
import pytest

import orbit_inputs as oi
from gpu_helpers import wrap

pytestmark = pytest.mark.gpu

# (d, L, kappa (None: a uniform orbit), seed, precision, n1, n2, fp_mode): orbits
# with many copies, so that the starts after the break find new ones
CASES = [
    (2, 6, None, 3, 0, 1500, 3000, 2),
    (3, 4, None, 5, 1, 2000, 4000, 1),
    (4, 4, 0.5, 1, 1, 4096, 4096, 1),
    (2, 64, 1.0, 1, 0, 48, 48, 1),        # beyond shared memory: hyperplane sweeps, slab Lanczos
]


def _orbit(d, L, kappa, seed):
    if kappa is None:
        return oi.uniform_orbit(d, L, seed), seed
    return oi.von_mises_orbit(d, L, kappa, seed), seed


def _by_first(c):
    p = np.argsort(c["first_start"].astype(np.int64), kind="stable")
    return {k: (v[p] if isinstance(v, np.ndarray) and len(v) == len(p) else v) for k, v in c.items()}


@pytest.mark.parametrize("d,L,kappa,seed,precision,n1,n2,fp_mode", CASES)
def test_resume_equals_unbroken_run(d, L, kappa, seed, precision, n1, n2, fp_mode):
    import paper_1403_0555_b300 as gb
    V = L ** d
    phi, oid = _orbit(d, L, kappa, seed)
    opt = gb.gc_options_default(precision=precision, check_every=4 if precision else 1, fp_mode=fp_mode)

    h = gb.gc_create_orbit(d, L, phi, oid)
    gb.gc_enumerate_copies(h, n1, 1.7, 1e-24, opt)
    gb.gc_enumerate_copies(h, n2, 1.7, 1e-24, opt)
    ref, ref_m = gb.gc_fetch_copies(h, V), gb.gc_fetch_minima_f8(h)
    gb.gc_destroy_orbit(h)

    h = gb.gc_create_orbit(d, L, phi, oid)
    gb.gc_enumerate_copies(h, n1, 1.7, 1e-24, opt)
    ckpt, ckpt_m = gb.gc_fetch_copies(h, V), gb.gc_fetch_minima_f8(h)
    gb.gc_destroy_orbit(h)

    h = gb.gc_create_orbit(d, L, phi, oid)
    gb.gc_load_copies(h, ckpt, ckpt_m, n1)
    assert gb.gc_orbit_stats(h)["n_distinct"] == ckpt["n_distinct"]
    gb.gc_enumerate_copies(h, n2, 1.7, 1e-24, opt)
    got, got_m = gb.gc_fetch_copies(h, V), gb.gc_fetch_minima_f8(h)
    st = gb.gc_orbit_stats(h)
    gb.gc_destroy_orbit(h)

    assert ckpt["n_distinct"] < ref["n_distinct"]          # the second part found new copies
    assert got["n_distinct"] == ref["n_distinct"]
    a, b = _by_first(got), _by_first(ref)
    for k in ("first_start", "count", "region", "F"):
        assert np.array_equal(a[k], b[k]), k
    assert np.array_equal(a["lambda2"], b["lambda2"], equal_nan=True)
    assert np.max(np.abs(wrap(a["theta"] - b["theta"]))) <= 1e-15
    assert np.array_equal(got["F"], ref["F"])                # the fetch order too
    assert got_m["n_minima"] == ref_m["n_minima"] == st["n_distinct_F8"]
    assert np.array_equal(got_m["F_norm"], ref_m["F_norm"])
    assert np.array_equal(got_m["count"], ref_m["count"])
    assert st["n_starts"] == n2


def test_resume_refuses_a_used_orbit_and_bad_records():
    import paper_1403_0555_b300 as gb
    d, L = 2, 4
    phi, oid = _orbit(d, L, None, 1)           # the uniform 2D 4x4 parity orbit
    opt = gb.gc_options_default(precision=0, check_every=1)
    h = gb.gc_create_orbit(d, L, phi, oid)
    gb.gc_enumerate_copies(h, 500, 1.7, 1e-24, opt)
    ckpt, ckpt_m = gb.gc_fetch_copies(h, L ** d), gb.gc_fetch_minima_f8(h)
    with pytest.raises(gb.GribovError) as e:
        gb.gc_load_copies(h, ckpt, ckpt_m, 500)               # the orbit has run starts
    assert e.value.code == gb.GC_ESTATE
    gb.gc_destroy_orbit(h)
    h = gb.gc_create_orbit(d, L, phi, oid)
    with pytest.raises(gb.GribovError) as e:                  # next_start not above every first start
        gb.gc_load_copies(h, ckpt, ckpt_m, int(ckpt["first_start"].max()))
    assert e.value.code == gb.GC_EINVAL
    gb.gc_load_copies(h, ckpt, ckpt_m, 500)                   # the refused calls left it fresh
    with pytest.raises(gb.GribovError) as e:                  # a second restore: the table is not empty
        gb.gc_load_copies(h, ckpt, ckpt_m, 500)
    assert e.value.code == gb.GC_ESTATE
    gb.gc_destroy_orbit(h)
