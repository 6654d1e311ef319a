"""Batches of orbits of uneven size: one call (optionally one captured CUDA graph)
gives every orbit exactly the result of its own gc_enumerate_copies call."""
import numpy as np
import pytest

import orbit_inputs as oi

pytestmark = pytest.mark.gpu

SHAPES = [(2, 4), (2, 6), (3, 4), (3, 5), (4, 3), (4, 4)]


def _orbits():
    return [(d, L, oi.von_mises_orbit(d, L, 1.0, 10 * d + L), 100 + 10 * d + L) for d, L in SHAPES]


def _fetch_all(gb, h, V):
    c = gb.gc_fetch_copies(h, V)
    s = gb.gc_orbit_stats(h)
    return c, s


def _single(gb, orbits, n, opt):
    out = []
    for d, L, phi, oid in orbits:
        h = gb.gc_create_orbit(d, L, phi, oid)
        gb.gc_enumerate_copies(h, n, 1.7, 1e-24, opt)
        out.append(_fetch_all(gb, h, L ** d))
        gb.gc_destroy_orbit(h)
    return out


def _batch(gb, orbits, n, opt, calls=1):
    hs = [gb.gc_create_orbit(d, L, phi, oid) for d, L, phi, oid in orbits]
    for _ in range(calls):
        gb.gc_enumerate_batch(hs, [n // calls] * len(hs), 1.7, 1e-24, opt)
    out = [_fetch_all(gb, h, L ** d) for h, (d, L, _, _) in zip(hs, orbits)]
    for h in hs:
        gb.gc_destroy_orbit(h)
    return out


def _same(a, b):
    for (ca, sa), (cb, sb) in zip(a, b):
        assert ca["n_distinct"] == cb["n_distinct"]
        for k in ("F", "first_start", "count", "region", "lambda2", "theta"):
            assert np.array_equal(ca[k], cb[k]), k
        for k in ("n_converged", "n_not_converged", "n_distinct_F8", "sweeps_fp32", "sweeps_fp64"):
            assert sa[k] == sb[k], k


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_equals_single_calls(precision):
    import paper_1403_0555_b300 as gb
    orbits = _orbits()
    opt = gb.gc_options_default(precision=precision, check_every=4 if precision else 1)
    _same(_single(gb, orbits, 3000, opt), _batch(gb, orbits, 3000, opt))


def test_batch_in_one_cuda_graph_and_async():
    import torch
    import paper_1403_0555_b300 as gb
    orbits = _orbits()
    side = torch.cuda.Stream()
    ref = _single(gb, orbits, 2000, gb.gc_options_default(precision=1, check_every=4))
    with torch.cuda.stream(side):
        opt = gb.gc_options_default(precision=1, check_every=4, use_graph=1, stream=side)
        _same(ref, _batch(gb, orbits, 2000, opt))
        opt = gb.gc_options_default(precision=1, check_every=4, stream=side)
        opt.async_ = 1
        _same(ref, _batch(gb, orbits, 2000, opt, calls=2))


def test_autotune_is_result_neutral():
    import paper_1403_0555_b300 as gb
    orbits = _orbits()[-2:]
    opt = gb.gc_options_default(precision=1, check_every=4)
    ref = _single(gb, orbits, 2000, opt)
    h = gb.gc_create_orbit(*orbits[0][:3], orbits[0][3])
    t = gb.gc_autotune(h, 1)
    gb.gc_destroy_orbit(h)
    assert t["r_warps"] in (2, 4, 8) and t["p_warps"] in (2, 4, 8, 16) and t["f_warps"] in (1, 2, 4)
    opt.autotune = 1
    _same(ref, _batch(gb, orbits, 2000, opt))


def test_autotune_mode2_equals_fixed_depth():
    """Mode 2 also tunes the sweep-unroll depth; its results are exactly those of
    an untuned run with that check_every (launch shapes are result-neutral)."""
    import paper_1403_0555_b300 as gb
    orbits = _orbits()[-2:]
    h = gb.gc_create_orbit(*orbits[1][:3], orbits[1][3])
    t = gb.gc_autotune(h, 1, mode=2)
    gb.gc_destroy_orbit(h)
    assert t["check_every"] in (2, 4, 8)
    tuned = gb.gc_options_default(precision=1, check_every=4)
    tuned.autotune = 2
    fixed = gb.gc_options_default(precision=1, check_every=t["check_every"])
    d, L, phi, oid = orbits[1]
    _same(_single(gb, [orbits[1]], 3000, fixed), _batch(gb, [orbits[1]], 3000, tuned))


def test_async_fetch_pipelined_equals_sync_fetch():
    """Batches in flight as the bench's end-to-end leg runs them: batch k + 1 is
    launched (asynchronously, on the next of three streams) before batch k's
    copies are fetched asynchronously into pinned host arrays, and
    gc_fetch_wait completes them a batch later.  Every array equals the
    synchronous fetch's."""
    import torch
    import paper_1403_0555_b300 as gb
    orbits = _orbits()
    ref = _single(gb, orbits, 2000, gb.gc_options_default(precision=1, check_every=4))
    streams = [torch.cuda.Stream() for _ in range(3)]

    def pinned_set(V, cap):
        p = lambda shape, dt: torch.empty(shape, dtype=dt, pin_memory=True).numpy()
        return {"F": p((cap,), torch.float64), "theta": p((cap, V), torch.float64),
                "first_start": p((cap,), torch.int64).view(np.uint64),
                "count": p((cap,), torch.int64).view(np.uint64),
                "lambda2": p((cap,), torch.float64), "region": p((cap,), torch.int32)}

    def launch(k):
        with torch.cuda.stream(streams[k % 3]):
            opt = gb.gc_options_default(precision=1, check_every=4, stream=streams[k % 3])
            opt.async_ = 1
            hs = [gb.gc_create_orbit(d, L, phi, oid) for d, L, phi, oid in orbits]
            gb.gc_enumerate_batch(hs, [2000] * len(hs), 1.7, 1e-24, opt)
        return hs

    def fetch(hs):
        return [gb.gc_fetch_copies_async(h, L ** d, out=pinned_set(L ** d, 4000))
                for h, (d, L, _, _) in zip(hs, orbits)]

    def finish(pending):
        hs, fetched = pending
        for h in hs:
            gb.gc_fetch_wait(h)
        out = [(c, gb.gc_orbit_stats(h)) for h, c in zip(hs, fetched)]
        for h in hs:
            gb.gc_destroy_orbit(h)
        return out

    n = 4
    results, prev, older = [], launch(0), None
    for k in range(1, n + 1):
        hs = launch(k) if k < n else None
        if older is not None:
            results.append(finish(older))
        older, prev = (prev, fetch(prev)), hs
    results.append(finish(older))
    assert len(results) == n
    for r in results:
        _same(ref, r)


@pytest.mark.parametrize("capacity,theta", [(7, True), (None, False)])
def test_async_fetch_partial_and_without_angles(capacity, theta):
    """A fetch of the first `capacity` copies, or of every copy without the
    angles, gives asynchronously (pinned arrays, completed by gc_fetch_wait)
    exactly what the synchronous fetch gives."""
    import torch
    import paper_1403_0555_b300 as gb
    d, L, phi, oid = _orbits()[3]
    V = L ** d
    h = gb.gc_create_orbit(d, L, phi, oid)
    gb.gc_enumerate_copies(h, 3000, 1.7, 1e-24, gb.gc_options_default(precision=1, check_every=4))
    ref = gb.gc_fetch_copies(h, V, capacity, theta=theta)
    m = len(ref["F"])
    assert m == (min(capacity, ref["n_distinct"]) if capacity else ref["n_distinct"]) and m > 0
    p = lambda shape, dt: torch.empty(shape, dtype=dt, pin_memory=True).numpy()
    out = {"F": p((m,), torch.float64), "theta": p((m, V), torch.float64) if theta else None,
           "first_start": p((m,), torch.int64).view(np.uint64), "count": p((m,), torch.int64).view(np.uint64),
           "lambda2": p((m,), torch.float64), "region": p((m,), torch.int32)}
    got = gb.gc_fetch_copies_async(h, V, capacity, theta=theta, out=out)
    gb.gc_fetch_wait(h)
    assert got["n_distinct"] == ref["n_distinct"]
    for k in ("F", "first_start", "count", "region", "lambda2") + (("theta",) if theta else ()):
        assert np.array_equal(got[k], ref[k], equal_nan=True), k
    gb.gc_destroy_orbit(h)
