"""Mixed-precision path (FP32 sweeps + FP64 Newton polish) against the plain FP64
path and the oracle.

The mixed path is not bitwise equal to the plain one (its FP32 trajectory
rounds differently), so it is held to: (a) every converged copy satisfies the
FP64 stopping rule when re-checked by the oracle's own divergence; (b) F of each
copy matches Eq. 3 evaluated by the oracle; (c) start by start it reaches the
same canonical copy as the plain path on at least 99.9% of starts (the measured
rate is printed); (d) its distinct-copy set restricted to copies found by both
paths is identical.
"""
import numpy as np
import pytest

import oracle
import orbit_inputs as oi
from gpu_helpers import run_gpu, wrap

pytestmark = pytest.mark.gpu


def _g_from_theta(theta):
    return np.stack([np.cos(theta), np.sin(theta)], axis=-1)


@pytest.mark.parametrize("d,L,kappa,n,variant", [(4, 4, 1.0, 4096, 0), (4, 4, 1.0, 4096, 1),
                                                 (3, 8, 1.0, 2048, 0), (3, 6, 1.0, 4096, 0),
                                                 (2, 8, 0.5, 4096, 0), (4, 3, 1.0, 2048, 0),
                                                 (3, 5, 1.0, 2048, 0)])
def test_mixed_agrees_with_plain(d, L, kappa, n, variant):
    """variant 0: the line-owner FP32 kernel where it exists (4^4, 8^3); 1: generic teams."""
    phi = oi.von_mises_orbit(d, L, kappa, 40 + d * 10 + L)
    ps, pc, _ = run_gpu(d, L, phi, 3, n, check_every=1, fp_mode=0)
    ms, mc, mst = run_gpu(d, L, phi, 3, n, check_every=4, fp_mode=0, precision=1,
                          relax_variant=variant)
    assert (ps["status"] == 1).all() and (ms["status"] == 1).all()
    # (a) FP64 stopping rule, re-checked by the oracle on the fetched angles
    div = np.stack([oracle.divergence(d, L, phi, _g_from_theta(t)) for t in mc["theta"][:512]])
    assert np.max(div ** 2) < 1e-22
    # (b) F of every copy against Eq. 3 evaluated by the oracle
    F_or = oracle.functional(d, L, phi, mc["theta"])
    assert np.max(np.abs(F_or - mc["F"]) / np.maximum(1.0, F_or)) < 1e-12
    # (c) start by start: same canonical copy
    th_p = pc["theta"][ps["copy_idx"]]
    th_m = mc["theta"][ms["copy_idx"]]
    same = np.max(np.abs(wrap(th_p - th_m)), axis=1) < 1e-6
    print(f"\nmixed vs plain agreement {d}D L={L} variant {variant}: {same.mean():.5f} of {n} starts; "
          f"newton steps/start {mst['newton_steps'] / n:.2f}, fallbacks {mst['polish_fallbacks']}")
    assert same.mean() >= 0.999
    # (d) copies found by both paths are the same configurations
    for i in np.flatnonzero(same)[:200]:
        assert abs(pc["F"][ps["copy_idx"][i]] - mc["F"][ms["copy_idx"][i]]) < 1e-10


def test_mixed_sampled_against_oracle():
    """Sampled starts of a 4^4 orbit: the oracle's FP64 relaxation of the same
    start index reaches the copy the mixed path reports for it."""
    d, L = 4, 4
    w = oi.workload_4d_4to4(1 << 14)
    o = w.orbits[3]
    ms, mc, _ = run_gpu(d, L, o.phi, o.orbit_id, 1 << 14, check_every=4, fp_mode=0, precision=1)
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(1 << 14, 48, replace=False))
    rel = oracle.relax_indices(d, L, o.phi, 1, o.orbit_id, idx)
    _, th = oracle.canonical(rel.g)
    th_m = mc["theta"][ms["copy_idx"][idx]]
    same = np.max(np.abs(wrap(th - th_m)), axis=1) < 1e-6
    assert same.sum() >= len(idx) - 1       # 99.9 % agreement: a miss in 48 is rare
    F_or = oracle.functional(d, L, o.phi, th)
    assert np.all(np.abs(F_or[same] - ms["F"][idx][same]) < 1e-10 * np.maximum(1, F_or[same]))


def test_hard_start_through_the_cg_redo_matches_oracle():
    """A start whose Faddeev-Popov operator is nearly singular at its minimum
    (4D 5^4, lambda_2 ~ 1e-4; the oracle's FP64 relaxation needs ~5e4 sweeps):
    the main polish hands it on, the conjugate-gradient instance finishes it,
    and it lands on the oracle's copy."""
    d, L = 4, 5
    phi = oi.von_mises_orbit(d, L, 1.0, 3)
    ms, mc, st = run_gpu(d, L, phi, 3, 8, check_every=4, fp_mode=0, precision=1)
    assert st["polish_redo_starts"] >= 1
    assert ms["status"][2] == oracle.CONVERGED
    rel = oracle.relax_indices(d, L, phi, 1, 3, [2])
    assert rel.status[0] == oracle.CONVERGED
    _, th = oracle.canonical(rel.g)
    th_m = mc["theta"][ms["copy_idx"][2]]
    assert np.max(np.abs(wrap(th[0] - th_m))) < 1e-6
    lam = oracle.lambda2(d, L, oracle.fp_weights(d, L, phi, th[0]))
    assert 0 < lam < 1e-3


def test_mixed_agrees_with_plain_on_the_bench_orbits():
    """The bench's eight 4^4 orbits (kappa 0.5 .. 2.0), 2^16 starts each: the
    mixed path (FP32 sweeps to 1e-10, FP64 polish) reaches the plain FP64
    path's canonical copy on at least 99.9 % of the starts of every orbit."""
    d, L, n = 4, 4, 1 << 16
    w = oi.workload_4d_4to4(n)
    tot = agree = 0
    for j, o in enumerate(w.orbits):
        ps, pc, _ = run_gpu(d, L, o.phi, o.orbit_id, n, check_every=1, fp_mode=3)
        ms, mc, _ = run_gpu(d, L, o.phi, o.orbit_id, n, check_every=4, fp_mode=3, precision=1)
        assert (ps["status"] == 1).all() and (ms["status"] == 1).all()
        th_p = pc["theta"][ps["copy_idx"]]
        th_m = mc["theta"][ms["copy_idx"]]
        same = np.max(np.abs(wrap(th_p - th_m)), axis=1) < 1e-6
        print(f"\norbit {j}: mixed vs plain {same.mean():.6f} ({n - int(same.sum())} of {n} differ)")
        assert same.mean() >= 0.999
        tot += n
        agree += int(same.sum())
    print(f"all orbits: {agree / tot:.6f}")
