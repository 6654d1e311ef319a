"""Lattices beyond shared memory: the sweeps stream each start's lattice in
hyperplanes from global memory (bulk copies).  The plain path stays bit-exact
to the oracle start by start; the mixed path (FP32 sweeps, then the inexact
Newton polish, FP64 sweeps for what it leaves) agrees with it; the
first-region fast path flags what the weights decide."""
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


@pytest.mark.parametrize("variant", ["cluster", "cta"])
@pytest.mark.parametrize("d,L,n", [(2, 64, 24), (3, 16, 12), (2, 128, 6)])
def test_hyperplane_plain_path_is_bit_exact_to_the_oracle(d, L, n, variant):
    """2D 64^2 and 3D 16^3 (links beyond shared memory) and 2D 128^2 (beyond
    the shared-memory kernels' 4096 sites), fewer starts than SMs: each start
    on a cluster of CTAs that split its planes ("cluster", the default for
    few starts) or on one CTA ("cta").  Status and sweep counts equal the
    oracle's, F within 1e-12, each start's canonical copy within 1e-9 rad."""
    import paper_1403_0555_b300 as gb
    V = L ** d
    phi = oi.von_mises_orbit(d, L, 1.0, 7)
    rv = gb.GC_RELAX_AUTO if variant == "cluster" else gb.GC_RELAX_GENERIC
    st, s, c = _plain(gb, d, L, phi, 7, n, precision=gb.GC_FP64, check_every=1, relax_variant=rv)
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


def _agree(c_a, s_a, c_b, s_b, n):
    same = 0
    for k in range(n):
        ta, tb = c_a["theta"][s_a["copy_idx"][k]], c_b["theta"][s_b["copy_idx"][k]]
        if np.max(np.abs(wrap(ta - tb))) <= 1e-6:
            same += 1
            assert abs(s_a["F"][k] - s_b["F"][k]) <= 1e-10 * s_a["F"][k]
    return same


@pytest.mark.parametrize("d,L,seed,n", [(3, 16, 3, 1024), (4, 8, 3, 1024), (2, 64, 3, 512), (4, 16, 1, 512)])
def test_hyperplane_mixed_path_agrees_with_the_plain_path(d, L, seed, n):
    """Lattices beyond shared memory, von Mises kappa = 1: the mixed path (the
    plain path's first FP64 sweeps, FP32 sweeps, Newton steps with an FP32 SOR
    inner solve, FP64 sweeps for what Newton leaves) converges every start to
    the FP64 tolerance, the oracle's divergence of the copies is below it, and
    start by start the copy is the plain path's on at least 99.9 % of the
    starts (the whole sample at 512 starts)."""
    import paper_1403_0555_b300 as gb
    phi = oi.von_mises_orbit(d, L, 1.0, seed)
    st_p, s_p, c_p = _plain(gb, d, L, phi, seed, n, precision=gb.GC_FP64, check_every=1)
    st_m, s_m, c_m = _plain(gb, d, L, phi, seed, n, precision=gb.GC_MIXED, check_every=4)
    assert st_m["n_converged"] == n and st_p["n_converged"] == n
    assert st_m["sweeps_fp32"] > 0 and st_m["newton_steps"] > 0 and st_m["newton_inner_sweeps"] > 0
    assert st_m["polish_fallbacks"] <= n // 8
    for k in range(0, c_m["n_distinct"], max(1, c_m["n_distinct"] // 16)):
        t = c_m["theta"][k]
        dv = oracle.divergence(d, L, phi, np.stack([np.cos(t), np.sin(t)], axis=-1))
        assert np.max(dv ** 2) < 2e-24
    same = _agree(c_p, s_p, c_m, s_m, n)
    print(f"\n{d}D L={L}: mixed vs plain {same} of {n} starts")
    assert same >= 0.999 * n, same


def test_hyperplane_newton_fallback_to_fp64_sweeps():
    """3D 16^3 mixed path with no Newton steps allowed: every start goes on to
    the FP64 hyperplane sweeps, converges, and ends at the minimum the Newton
    polish reaches from the same FP32 state (both finish the same basin)."""
    import paper_1403_0555_b300 as gb
    d, L, n = 3, 16, 24
    phi = oi.von_mises_orbit(d, L, 1.0, 5)
    st_n, s_n, c_n = _plain(gb, d, L, phi, 5, n, precision=gb.GC_MIXED, check_every=4)
    st_f, s_f, c_f = _plain(gb, d, L, phi, 5, n, precision=gb.GC_MIXED, check_every=4, newton_max=0)
    assert st_n["n_converged"] == n and st_f["n_converged"] == n
    assert st_f["polish_fallbacks"] == n and st_f["newton_steps"] == 0 and st_f["site_updates_fp64"] > 0
    assert st_n["newton_steps"] >= n
    assert np.array_equal(s_n["sweeps"] <= s_f["sweeps"], np.ones(n, bool))
    assert _agree(c_n, s_n, c_f, s_f, n) >= n - 1


@pytest.mark.parametrize("d,L", [(3, 16), (2, 64)])
def test_hyperplane_cluster_and_cta_forms_agree_bitwise(d, L):
    """Mixed path with 8 starts, so that every start gets a cluster in the
    FP32 sweeps, the Newton polish and the FP64 sweeps (3D 16^3: streamed
    hyperplanes; 2D 64^2: the FP32 sweeps with the lattice in the cluster's
    distributed shared memory, 4 planes per CTA): the cluster forms split each
    pass by planes but keep every site's arithmetic and the maxima, so they
    equal the one-CTA form bit for bit (statuses, sweep and Newton counts, F,
    every copy's angles)."""
    import paper_1403_0555_b300 as gb
    n = 8
    phi = oi.von_mises_orbit(d, L, 1.0, 9)
    st_c, s_c, c_c = _plain(gb, d, L, phi, 9, n, precision=gb.GC_MIXED, check_every=4,
                            relax_variant=gb.GC_RELAX_AUTO)
    st_g, s_g, c_g = _plain(gb, d, L, phi, 9, n, precision=gb.GC_MIXED, check_every=4,
                            relax_variant=gb.GC_RELAX_GENERIC)
    assert st_c["n_converged"] == n
    for k in ("n_converged", "n_distinct", "sweeps_fp32", "newton_steps", "newton_inner_sweeps",
              "polish_fallbacks", "fp64_residual_passes", "site_updates_fp64"):
        assert st_c[k] == st_g[k], k
    for k in ("status", "sweeps", "F", "copy_idx"):
        assert np.array_equal(s_c[k], s_g[k]), k
    assert np.array_equal(c_c["theta"], c_g["theta"]) and np.array_equal(c_c["F"], c_g["F"])


@pytest.mark.parametrize("mode", ["lanczos", "auto"])
def test_hyperplane_first_region_lanczos_matches_the_oracle(mode):
    """2D 64^2 (4096 sites, von Mises kappa = 1), plain path: lambda_2 of each
    copy by the large-lattice Lanczos (vectors in global memory) against the
    oracle's dense eigensolve of the same copy.  FP64 Lanczos (`lanczos`): a
    Ritz value, so at or above lambda_2 and within 1e-4 relative of it; the
    FP32 screen (`auto`: it decides copies above 1e-4 and hands the rest to
    FP64) within 1e-4; region flags equal."""
    import paper_1403_0555_b300 as gb
    d, L, n = 2, 64, 6
    phi = oi.von_mises_orbit(d, L, 1.0, 11)
    fm, tol = (gb.GC_FP_LANCZOS, 1e-6) if mode == "lanczos" else (gb.GC_FP_AUTO, 1e-4)
    st, s, c = _plain(gb, d, L, phi, 11, n, precision=gb.GC_FP64, check_every=1, fp_mode=fm)
    assert c["n_distinct"] > 0 and st["fp_tests"] == c["n_distinct"]
    if mode == "lanczos":
        assert st["fp_tests_fp64"] == c["n_distinct"]
    for k in range(min(3, c["n_distinct"])):
        lam = oracle.lambda2(d, L, oracle.fp_weights(d, L, phi, c["theta"][k]))
        if mode == "lanczos":
            assert -1e-12 <= c["lambda2"][k] - lam <= 1e-4 * abs(lam) + 1e-12, (k, c["lambda2"][k], lam)
        else:
            assert abs(c["lambda2"][k] - lam) <= tol * max(1.0, abs(lam)), (k, c["lambda2"][k], lam)
        assert c["region"][k] == oracle.region_flag(lam, 1e-9)


def test_hyperplane_requests_served_alongside_others():
    """Serving: two large-lattice requests (2D 64^2 and 3D 16^3, mixed path)
    admitted while a small 4^4 request runs give the same copies, statistics
    and region flags as when run alone (every stage is per start or per copy,
    with no dependence on what shares the GPU)."""
    import paper_1403_0555_b300 as gb
    opt = gb.gc_options_default(precision=gb.GC_MIXED, check_every=4)
    reqs = [(4, 4, 20000), (2, 64, 12), (3, 16, 10)]
    srv = gb.gc_server_create(3, 0, opt)
    try:
        tickets = []
        for i, (d, L, n) in enumerate(reqs):
            phi = oi.von_mises_orbit(d, L, 1.0, 70 + i)
            tickets.append((gb.gc_server_submit(srv, d, L, phi, 70 + i, n), d, L, n, phi, i))
        for t, d, L, n, phi, i in tickets:
            status, latency, orb = gb.gc_server_wait(srv, t, 300.0)
            assert status == gb.GC_OK and orb is not None and latency > 0
            mixed = gb.gc_fetch_copies(orb, L ** d)
            mst = gb.gc_orbit_stats(orb)
            gb.gc_destroy_orbit(orb)
            h = gb.gc_create_orbit(d, L, phi, 70 + i)
            try:
                gb.gc_enumerate_copies(h, n, 1.7, 1e-24, opt)
                alone, ast = gb.gc_fetch_copies(h, L ** d), gb.gc_orbit_stats(h)
            finally:
                gb.gc_destroy_orbit(h)
            assert mixed["n_distinct"] == alone["n_distinct"] > 0
            for k in ("F", "first_start", "count", "region", "lambda2", "theta"):
                assert np.array_equal(mixed[k], alone[k]), (d, L, k)
            for k in ("n_converged", "newton_steps", "newton_inner_sweeps", "sweeps_fp32"):
                assert mst[k] == ast[k], (d, L, k)
    finally:
        gb.gc_server_destroy(srv)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_hyperplane_batches_give_the_single_batch_result(precision):
    """2D 64^2, 20 starts split into device batches of 7 (three batches, the
    last ragged) against one batch: every stage works per start or per copy,
    so statuses, sweeps, F and the copy table (first starts, counts, angles,
    region flags) are identical."""
    import paper_1403_0555_b300 as gb
    d, L, n = 2, 64, 20
    phi = oi.von_mises_orbit(d, L, 1.0, 13)
    prec = gb.GC_FP64 if precision == "fp64" else gb.GC_MIXED
    ce = 1 if precision == "fp64" else 4
    st_1, s_1, c_1 = _plain(gb, d, L, phi, 13, n, precision=prec, check_every=ce)
    st_b, s_b, c_b = _plain(gb, d, L, phi, 13, n, precision=prec, check_every=ce, batch_starts=7)
    for k in ("status", "sweeps", "F", "copy_idx"):
        assert np.array_equal(s_1[k], s_b[k]), k
    assert c_1["n_distinct"] == c_b["n_distinct"] > 0
    for k in ("F", "first_start", "count", "theta", "region"):
        assert np.array_equal(c_1[k], c_b[k]), k
    for k in ("n_converged", "sweeps_fp32", "site_updates_fp64", "newton_steps"):
        assert st_1[k] == st_b[k], k


@pytest.mark.parametrize("use_graph", [0, 1])
def test_hyperplane_orbit_in_a_batch(use_graph):
    """A 4^4 orbit and a 2D 64^2 orbit (the hyperplane path) in one
    gc_enumerate_batch call, plainly and captured as one CUDA graph (every
    buffer and launch query of the hyperplane path is set up before the
    capture): each orbit's copies equal its single call."""
    import torch
    import paper_1403_0555_b300 as gb
    side = torch.cuda.Stream()
    specs = [(4, 4, 4000, 1), (2, 64, 12, 2)]
    opt = gb.gc_options_default(precision=gb.GC_MIXED, check_every=4, stream=side, use_graph=use_graph)
    hs = [gb.gc_create_orbit(d, L, oi.von_mises_orbit(d, L, 1.0, sd), sd, n) for d, L, n, sd in specs]
    try:
        with torch.cuda.stream(side):
            gb.gc_enumerate_batch(hs, [n for _, _, n, _ in specs], 1.7, 1e-24, opt)
        side.synchronize()
        got = [gb.gc_fetch_copies(h, L ** d) for h, (d, L, _, _) in zip(hs, specs)]
    finally:
        for h in hs:
            gb.gc_destroy_orbit(h)
    for (d, L, n, sd), c in zip(specs, got):
        h = gb.gc_create_orbit(d, L, oi.von_mises_orbit(d, L, 1.0, sd), sd)
        try:
            gb.gc_enumerate_copies(h, n, 1.7, 1e-24, gb.gc_options_default(precision=gb.GC_MIXED, check_every=4))
            ref = gb.gc_fetch_copies(h, L ** d)
        finally:
            gb.gc_destroy_orbit(h)
        assert c["n_distinct"] == ref["n_distinct"] > 0
        for k in ("F", "theta", "first_start", "count", "region", "lambda2"):
            assert np.array_equal(c[k], ref[k]), (d, L, k)


@pytest.mark.parametrize("d,L", [(3, 17), (4, 18), (1, 5000), (2, 300)])
def test_lattices_neither_path_takes_are_refused(d, L):
    """Beyond shared memory only even L, d >= 2 and V <= 65 536 are taken:
    3D 17^3 (odd L), 4D 18^4 (V = 104 976), 1D of 5000 sites and 2D 300^2
    (V = 90 000) are GC_EINVAL at gc_create_orbit, with nothing allocated."""
    import paper_1403_0555_b300 as gb
    phi = np.zeros((L ** d, d))
    with pytest.raises(gb.GribovError) as e:
        gb.gc_create_orbit(d, L, phi, 1)
    assert e.value.code == gb.GC_EINVAL


def test_hyperplane_f8_minima():
    """The paper's count (F/(dV) quantised at 1e-8, with the starts reaching
    each) on 2D 64^2, plain path: equal to the oracle's, in the configuration
    mode and in the F-only mode (which keeps no configurations)."""
    import paper_1403_0555_b300 as gb
    d, L, n = 2, 64, 12
    phi = oi.von_mises_orbit(d, L, 1.0, 17)
    rel = oracle.relax_starts(d, L, phi, 1, 17, 0, n, 1.7, 1e-24)
    _, th = oracle.canonical(rel.g)
    conv = rel.status == oracle.CONVERGED
    F = oracle.functional(d, L, phi, th)
    keys, counts = np.unique(np.floor(oracle.f_norm(F[conv], d, L) * 1e8).astype(np.int64), return_counts=True)
    for mode in (gb.GC_DEDUP_CONFIG, gb.GC_DEDUP_F8):
        h = gb.gc_create_orbit(d, L, phi, 17)
        try:
            gb.gc_enumerate_copies(h, n, 1.7, 1e-24, gb.gc_options_default(precision=gb.GC_FP64, check_every=1,
                                                                          dedup_mode=mode))
            m, st = gb.gc_fetch_minima_f8(h), gb.gc_orbit_stats(h)
        finally:
            gb.gc_destroy_orbit(h)
        assert np.array_equal(np.round(m["F_norm"] * 1e8).astype(np.int64), keys)
        assert np.array_equal(m["count"].astype(np.int64), counts)
        assert (st["n_distinct"] == 0) == (mode == gb.GC_DEDUP_F8)
