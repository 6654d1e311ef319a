"""Lattices beyond shared memory: the sweeps stream each start's lattice in
hyperplanes from global memory (bulk copies).  The plain path stays bit-exact
to the oracle start by start; the mixed path (FP32 sweeps, then FP64 sweeps)
agrees with it; the first-region fast path flags what the weights decide."""
import numpy as np
import pytest

import oracle
import orbit_inputs as oi
from gpu_helpers import wrap

pytestmark = pytest.mark.gpu


def _plain(gb, d, L, phi, oid, n, omega=1.7, eps=1e-24, **kw):
    h = gb.gc_create_orbit(d, L, phi, oid)
    try:
        gb.gc_enumerate_copies(h, n, omega, eps, gb.gc_options_default(keep_per_start=1, **kw))
        return gb.gc_orbit_stats(h), gb.gc_fetch_starts(h, 0, n), gb.gc_fetch_copies(h, L ** d)
    finally:
        gb.gc_destroy_orbit(h)


@pytest.mark.parametrize("d,L,n", [(2, 64, 24), (3, 16, 12), (2, 128, 6)])
def test_hyperplane_plain_path_is_bit_exact_to_the_oracle(d, L, n):
    """2D 64^2 and 3D 16^3 (links beyond shared memory) and 2D 128^2 (beyond
    the shared-memory kernels' 4096 sites): status and sweep counts equal the
    oracle's, F within 1e-12, each start's canonical copy within 1e-9 rad."""
    import paper_1403_0555_b300 as gb
    V = L ** d
    phi = oi.von_mises_orbit(d, L, 1.0, 7)
    st, s, c = _plain(gb, d, L, phi, 7, n, precision=gb.GC_FP64, check_every=1)
    rel = oracle.relax_starts(d, L, phi, 1, 7, 0, n, 1.7, 1e-24)
    assert np.array_equal(s["status"], rel.status.astype(np.int32))
    assert np.array_equal(s["sweeps"], rel.sweeps)
    conv = rel.status == oracle.CONVERGED
    assert conv.all()
    _, th = oracle.canonical(rel.g)
    F = oracle.functional(d, L, phi, th)
    assert np.all(np.abs(s["F"] - F) <= 1e-12 * np.maximum(1.0, np.abs(F)))
    for k in range(n):
        ci = s["copy_idx"][k]
        assert ci >= 0
        assert np.max(np.abs(wrap(c["theta"][ci] - th[k]))) <= 1e-9 or c["first_start"][ci] < k
    assert np.all(np.abs(c["theta"][:, V - 1]) <= 1e-15)
    assert st["n_distinct"] == c["n_distinct"] > 0


def test_hyperplane_mixed_path_agrees_with_the_plain_path():
    """4D 8^4 (FP32 hyperplane sweeps, then FP64 ones): every start converges to
    the FP64 tolerance and reaches the plain path's minimum in at least 90 % of
    the starts (the FP32 phase may settle a start near a basin boundary
    elsewhere; 8^4 landscapes hold many close minima)."""
    import paper_1403_0555_b300 as gb
    d, L, n = 4, 8, 32
    phi = oi.von_mises_orbit(d, L, 1.0, 3)
    st_p, s_p, c_p = _plain(gb, d, L, phi, 3, n, precision=gb.GC_FP64, check_every=1)
    st_m, s_m, c_m = _plain(gb, d, L, phi, 3, n, precision=gb.GC_MIXED, check_every=4)
    assert st_m["n_converged"] == n and st_p["n_converged"] == n
    assert st_m["sweeps_fp32"] > 0 and st_m["site_updates_fp64"] > 0
    same = 0
    for k in range(n):
        ta, tb = c_p["theta"][s_p["copy_idx"][k]], c_m["theta"][s_m["copy_idx"][k]]
        if np.max(np.abs(wrap(ta - tb))) <= 1e-6:
            same += 1
            assert abs(s_p["F"][k] - s_m["F"][k]) <= 1e-10 * s_p["F"][k]
    assert same >= 0.9 * n, same


def test_hyperplane_first_region_fast_path():
    """Region flags of the fast path: IN exactly when every weight
    cos(phi^theta) is positive (the oracle's weights of each copy), else
    untested; lambda_2 is not computed on this path."""
    import paper_1403_0555_b300 as gb
    d, L, n = 2, 64, 16
    phi = oi.von_mises_orbit(d, L, 3.0, 11)
    st, s, c = _plain(gb, d, L, phi, 11, n, precision=gb.GC_FP64, check_every=1)
    for k in range(c["n_distinct"]):
        w = oracle.fp_weights(d, L, phi, c["theta"][k])
        assert c["region"][k] == (1 if np.all(w > 0) else -1)
        assert np.isnan(c["lambda2"][k])
