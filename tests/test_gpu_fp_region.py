"""The first-region test (Section I: minimal Landau gauge, the Faddeev-Popov
operator non-negative off its constant zero mode) of every distinct copy
against the oracle's dense eigensolve.

4D 4^4, the bench's lattice and precision (FP32 sweeps + FP64 polish), on the
kappa = 0.5 orbit (the one with the most copies) and the kappa = 0.93 orbit,
2^14 starts each.  For every copy: lambda_2 and the region flag of
GC_FP_LANCZOS (FP64 Lanczos, the bench's test) and of GC_FP_AUTO (FP32 Lanczos
screen, FP64 Lanczos below 1e-3) against numpy's eigvalsh of the dense
operator (oracle.lambda2).  The copy tables of the modes are the same: the
test changes no relaxation.
"""
import numpy as np
import pytest

import oracle
import orbit_inputs as oi
from gpu_helpers import oracle_pool, run_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("j", [0, 2])
def test_every_copy_region_and_lambda2_against_dense(j):
    import paper_1403_0555_b300 as gb
    d, L, n = 4, 4, 1 << 14
    o = oi.workload_4d_4to4(n).orbits[j]
    runs = {}
    for mode in (gb.GC_FP_LANCZOS, gb.GC_FP_AUTO):
        _, c, st = run_gpu(d, L, o.phi, o.orbit_id, n, precision=gb.GC_MIXED, check_every=4,
                           fp_mode=mode, keep_per_start=0)
        runs[mode] = (c, st)
    c_l, st_l = runs[gb.GC_FP_LANCZOS]
    c_a, st_a = runs[gb.GC_FP_AUTO]
    assert c_l["n_distinct"] == c_a["n_distinct"] > 100
    assert np.array_equal(c_l["first_start"], c_a["first_start"])
    assert st_l["fp_tests_fp64"] == st_l["fp_tests"] == c_l["n_distinct"]     # FP64 for every copy
    with oracle_pool() as pool:
        lam = np.array(pool.map(oracle.lambda2_of_copy,
                                [(d, L, o.phi, th) for th in c_l["theta"]], chunksize=64))
    reg = np.array([oracle.region_flag(x, 1e-9) for x in lam], dtype=np.int32)
    rel_l = np.abs(c_l["lambda2"] - lam) / np.maximum(np.abs(lam), 1e-3)
    rel_a = np.abs(c_a["lambda2"] - lam) / np.maximum(np.abs(lam), 1e-3)
    print(f"\norbit {j}: {len(lam)} copies, IN/MARGINAL/OUT {np.bincount(reg, minlength=3)[[1, 2, 0]]}, "
          f"min lambda_2 {lam.min():.3e}; LANCZOS max rel err {rel_l.max():.2e}; AUTO max rel err "
          f"{rel_a.max():.2e}, > 1e-3 on {int((rel_a > 1e-3).sum())} copies")
    # FP64 Lanczos: the flag of every copy, and lambda_2 to 1e-9 relative
    assert np.array_equal(c_l["region"], reg)
    assert rel_l.max() <= 1e-9
    # FP32 screen: the same flag for every copy (the screen only accepts
    # copies whose FP32 Ritz value is above 1e-3; the rest are FP64)
    assert np.array_equal(c_a["region"], reg)
    # a Ritz value never lies below the smallest eigenvalue (to rounding)
    assert np.all(c_l["lambda2"] >= lam - 1e-12 * np.maximum(1.0, np.abs(lam)))


@pytest.mark.parametrize("d,L,kappa", [(3, 6, 1.0), (2, 16, 1.0), (4, 3, 0.5)])
def test_lanczos_mode_other_lattices_against_dense(d, L, kappa):
    """The Lanczos mode on lattices outside the 4^4 line layout (the generic
    kernel: FP32 Ritz seed then FP64 Lanczos, vectors in shared memory): the
    flag of every copy equals the dense eigensolve's, lambda_2 within 1e-9
    relative, and never below the smallest eigenvalue."""
    import paper_1403_0555_b300 as gb
    n = 1 << 12
    phi = oi.von_mises_orbit(d, L, kappa, 3)
    _, c, st = run_gpu(d, L, phi, 3, n, precision=gb.GC_MIXED, check_every=4,
                       fp_mode=gb.GC_FP_LANCZOS, keep_per_start=0)
    assert c["n_distinct"] > 10
    assert st["fp_tests_fp64"] == st["fp_tests"] == c["n_distinct"]
    assert 0 < st["lanczos_steps_fp64"] < st["lanczos_steps"]
    with oracle_pool() as pool:
        lam = np.array(pool.map(oracle.lambda2_of_copy,
                                [(d, L, phi, th) for th in c["theta"]], chunksize=16))
    reg = np.array([oracle.region_flag(x, 1e-9) for x in lam], dtype=np.int32)
    rel = np.abs(c["lambda2"] - lam) / np.maximum(np.abs(lam), 1e-3)
    print(f"\n{d}D L={L}: {len(lam)} copies, IN/MARGINAL/OUT {np.bincount(reg, minlength=3)[[1, 2, 0]]}, "
          f"max rel err {rel.max():.2e}, FP64 steps per copy {st['lanczos_steps_fp64'] / st['fp_tests']:.2f}")
    assert np.array_equal(c["region"], reg)
    assert rel.max() <= 1e-9
    assert np.all(c["lambda2"] >= lam - 1e-12 * np.maximum(1.0, np.abs(lam)))
