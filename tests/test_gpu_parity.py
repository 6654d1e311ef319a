"""Parity of the CUDA path (through the C ABI) with the oracle, start by start.

Plain FP64 path: the sweeps use explicitly rounded IEEE operations in the
oracle's order, so every start follows the oracle's trajectory exactly; the
tests demand identical statuses, sweep counts, copy sets, multiplicities and
first starts, F within 1e-12 (relative, absolute below 1) and lambda_2 (dense
mode) within 1e-9.  The canonical angles are within 2e-15 rad: the
configurations are the oracle's to rounding (the canonical product's), so
the fetch's angle (table reduction and arcsine series) is held to the
oracle's arctangent at a few units in the last place.
"""
import math

import numpy as np
import pytest

import oracle
import orbit_inputs as oi
from gpu_helpers import assert_copies_equal, assert_starts_equal, run_gpu, wrap

pytestmark = pytest.mark.gpu


def _oracle_F(d, L, phi, relaxed):
    _, th = oracle.canonical(relaxed.g)
    return oracle.functional(d, L, phi, th)


def test_2d_4x4_uniform_full_parity():
    """2D 4x4, uniform orbit seed 1, 10^4 starts, omega 1.7, eps 1e-24, FP64, dense FP test."""
    w = oi.workload_2d_4x4()
    o = w.orbits[0]
    gs, gc_, st = run_gpu(o.d, o.L, o.phi, o.orbit_id, w.n_starts, w.omega, w.eps,
                          fp_mode=2, check_every=1)
    relaxed, cp = oracle.enumerate_copies(o.d, o.L, o.phi, 1, o.orbit_id, w.n_starts, w.omega, w.eps)
    assert_starts_equal(gs, relaxed, cp, _oracle_F(o.d, o.L, o.phi, relaxed))
    assert_copies_equal(gc_, cp, theta_tol=2e-15, lam_tol=1e-9)
    assert st["n_distinct_F8"] == cp.n_distinct_F8
    assert st["n_converged"] == int((relaxed.status == 1).sum())
    assert st["n_in"] == int((cp.region == oracle.REGION_IN).sum())


SMALL = [(1, 5), (1, 6), (2, 2), (2, 3), (2, 5), (3, 3), (3, 4), (4, 2), (4, 3)]


@pytest.mark.parametrize("d,L", SMALL)
@pytest.mark.parametrize("omega,check_every", [(1.0, 1), (1.7, 3)])
def test_small_lattices_parity(d, L, omega, check_every):
    """Ragged start counts, odd L (3 colours), L = 2 double links, d = 1..4."""
    phi = oi.von_mises_orbit(d, L, 0.8, 100 * d + L)
    n = 1037
    gs, gc_, st = run_gpu(d, L, phi, 7, n, omega, 1e-24, fp_mode=2, check_every=check_every)
    relaxed, cp = oracle.enumerate_copies(d, L, phi, 1, 7, n, omega, 1e-24, check_every=check_every)
    assert_starts_equal(gs, relaxed, cp, _oracle_F(d, L, phi, relaxed))
    assert_copies_equal(gc_, cp, theta_tol=2e-15, lam_tol=1e-9)
    assert st["n_distinct_F8"] == cp.n_distinct_F8


def test_sweep_cap_gives_not_converged():
    d, L = 3, 4
    phi = oi.uniform_orbit(d, L, 3)
    gs, gc_, st = run_gpu(d, L, phi, 2, 500, 1.7, 1e-24, max_sweeps=12, check_every=4, fp_mode=2)
    relaxed, cp = oracle.enumerate_copies(d, L, phi, 1, 2, 500, 1.7, 1e-24, check_every=4,
                                          max_sweeps=12)
    assert (relaxed.status == oracle.NOT_CONVERGED).sum() > 0
    assert_starts_equal(gs, relaxed, cp, _oracle_F(d, L, phi, relaxed))
    assert_copies_equal(gc_, cp, lam_tol=1e-9)
    assert st["n_not_converged"] == int((relaxed.status == 2).sum())


def test_calls_accumulate_like_one_call():
    d, L = 2, 6
    phi = oi.uniform_orbit(d, L, 5)
    _, one, _ = run_gpu(d, L, phi, 3, 3000, keep_per_start=0, fp_mode=2)
    _, three, _ = run_gpu(d, L, phi, 3, 3000, calls=[1000, 1500, 500], keep_per_start=0, fp_mode=2)
    for k in ("F", "first_start", "count", "lambda2", "region"):
        assert np.array_equal(one[k], three[k]), k
    assert np.array_equal(one["theta"], three["theta"])


def test_small_batches_match_large_batch():
    d, L = 3, 4
    phi = oi.von_mises_orbit(d, L, 1.0, 9)
    _, a, _ = run_gpu(d, L, phi, 4, 2500, keep_per_start=0, fp_mode=2)
    _, b, _ = run_gpu(d, L, phi, 4, 2500, keep_per_start=0, fp_mode=2, batch_starts=333)
    for k in ("F", "first_start", "count", "region"):
        assert np.array_equal(a[k], b[k]), k


def test_cold_orbit_plane_waves():
    """Gauge-hidden cold orbit 2D 6x6: every found plane wave matches the closed form."""
    d, L = 2, 6
    phi = oi.trivial_gauge_orbit(d, L, 5)
    _, cp, _ = run_gpu(d, L, phi, 5, 4000, keep_per_start=0, fp_mode=2)
    assert cp["F"][0] < 1e-12            # the global minimum F = 0
    links = oracle.link_angles_gauged(d, L, phi, cp["theta"])
    spread = np.abs(wrap(links - links[:, :1, :])).max(axis=(1, 2))
    waves = cp["F"][spread < 1e-9]
    pred = {round(L ** d * sum(1 - math.cos(2 * math.pi * k / L) for k in ks), 9)
            for ks in [(a, b) for a in (0, 1, 5) for b in (0, 1, 5)]}
    for f in waves:
        assert round(f, 9) in pred


def test_fp_modes_agree():
    d, L = 3, 4
    phi = oi.von_mises_orbit(d, L, 0.7, 12)
    _, dense, _ = run_gpu(d, L, phi, 1, 1500, keep_per_start=0, fp_mode=2)
    _, lanc, _ = run_gpu(d, L, phi, 1, 1500, keep_per_start=0, fp_mode=1)
    _, auto, st = run_gpu(d, L, phi, 1, 1500, keep_per_start=0, fp_mode=0)
    assert np.array_equal(dense["region"], lanc["region"])
    assert np.array_equal(dense["region"], auto["region"])
    assert np.max(np.abs(dense["lambda2"] - lanc["lambda2"])) < 1e-8
    assert np.max(np.abs(dense["lambda2"] - auto["lambda2"])) < 1e-4
    assert st["fp_tests"] == auto["n_distinct"]


def test_invalid_arguments_and_empty_call():
    import paper_1403_0555_b300 as gb
    phi = oi.uniform_orbit(2, 4, 1)
    h = gb.gc_create_orbit(2, 4, phi, 1)
    try:
        gb.gc_enumerate_copies(h, 0, 1.7, 1e-24)
        assert gb.gc_fetch_copies(h, 16)["n_distinct"] == 0
        for omega, eps in ((0.0, 1e-24), (2.0, 1e-24), (1.7, 0.0), (1.7, -1.0)):
            with pytest.raises(gb.GribovError) as e:
                gb.gc_enumerate_copies(h, 10, omega, eps)
            assert e.value.code == gb.GC_EINVAL
        with pytest.raises(gb.GribovError) as e:
            gb.gc_fetch_starts(h, 0, 1)
        assert e.value.code == gb.GC_ESTATE
        gb.gc_enumerate_copies(h, 100, 1.7, 1e-24)
        part = gb.gc_fetch_copies(h, 16, capacity=1)
        full = gb.gc_fetch_copies(h, 16)
        assert part["F"].shape == (1,) and part["F"][0] == full["F"][0]
    finally:
        gb.gc_destroy_orbit(h)
