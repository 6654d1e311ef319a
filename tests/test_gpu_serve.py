"""Serving with continuous batching: requests admitted while others run give the
same result as when run alone; admission and waits are bounded."""
import time

import numpy as np
import pytest

import orbit_inputs as oi
from gpu_helpers import run_gpu

pytestmark = pytest.mark.gpu

MIX = [(2, 4, 3000), (2, 8, 5000), (3, 4, 4000), (3, 5, 2000), (4, 3, 3000), (4, 4, 6000),
       (3, 6, 2000), (2, 6, 8000), (4, 4, 2000), (2, 12, 1000), (3, 8, 2000), (4, 5, 1000)]


def test_each_result_same_alone_and_in_the_mix():
    import paper_1403_0555_b300 as gb
    opt = gb.gc_options_default(precision=1, check_every=4)
    srv = gb.gc_server_create(4, 0, opt)
    tickets = []
    rng = np.random.default_rng(3)
    try:
        for i, (d, L, n) in enumerate(MIX):
            phi = oi.von_mises_orbit(d, L, 1.0, 50 + i)
            tickets.append((gb.gc_server_submit(srv, d, L, phi, 50 + i, n), d, L, n, phi, i))
            time.sleep(rng.exponential(0.002))         # arrivals while others run
        lat = []
        for t, d, L, n, phi, i in tickets:
            status, latency, orb = gb.gc_server_wait(srv, t, 120.0)
            assert status == gb.GC_OK and orb is not None
            lat.append(latency)
            mixed = gb.gc_fetch_copies(orb, L ** d)
            mst = gb.gc_orbit_stats(orb)
            gb.gc_destroy_orbit(orb)
            _, alone, ast = run_gpu(d, L, phi, 50 + i, n, keep_per_start=0, precision=1, check_every=4)
            assert mixed["n_distinct"] == alone["n_distinct"]
            for k in ("F", "first_start", "count", "region", "lambda2", "theta"):
                assert np.array_equal(mixed[k], alone[k]), (d, L, k)
            assert mst["n_converged"] == ast["n_converged"]
        assert all(x > 0 for x in lat)
    finally:
        gb.gc_server_destroy(srv)


def test_budget_and_bounded_wait():
    import paper_1403_0555_b300 as gb
    srv = gb.gc_server_create(2, 2 << 30, gb.gc_options_default(precision=1, check_every=4))
    try:
        big = oi.von_mises_orbit(4, 6, 1.0, 1)
        with pytest.raises(gb.GribovError) as e:
            gb.gc_server_submit(srv, 4, 6, big, 1, 1_000_000)
        assert e.value.code == gb.GC_ENOMEM
        phi = oi.von_mises_orbit(4, 4, 1.0, 2)
        t = gb.gc_server_submit(srv, 4, 4, phi, 2, 200_000)
        with pytest.raises(gb.GribovError) as e:
            gb.gc_server_wait(srv, t, 1e-5)
        assert e.value.code == gb.GC_ETIMEDOUT
        status, latency, orb = gb.gc_server_wait(srv, t, 120.0)
        assert status == gb.GC_OK and latency > 0
        assert gb.gc_orbit_stats(orb)["n_converged"] == 200_000
        gb.gc_destroy_orbit(orb)
        with pytest.raises(gb.GribovError):
            gb.gc_server_wait(srv, t, 1.0)          # ticket retired
    finally:
        gb.gc_server_destroy(srv)


def test_concurrent_shapes_of_one_dimension_all_succeed():
    """Workers launch the same kernels for different lattice sizes at once (one
    kernel, different shared-memory footprints): every request must succeed."""
    import paper_1403_0555_b300 as gb
    srv = gb.gc_server_create(8, 0, gb.gc_options_default(precision=1, check_every=4))
    tickets = []
    try:
        for i in range(48):
            L = (3, 4, 5, 6)[i % 4]
            phi = oi.von_mises_orbit(4, L, 1.0, 200 + i)
            tickets.append(gb.gc_server_submit(srv, 4, L, phi, 200 + i, 600 + 97 * i))
        for t in tickets:
            status, latency, orb = gb.gc_server_wait(srv, t, 120.0)
            assert status == gb.GC_OK and orb is not None
            st = gb.gc_orbit_stats(orb)
            assert st["n_converged"] + st["n_not_converged"] == st["n_starts"]
            gb.gc_destroy_orbit(orb)
    finally:
        gb.gc_server_destroy(srv)


def test_device_loop_admits_by_budget_and_times_out_when_idle():
    """The request loop runs on the GPU: with an arena for about one and a half
    requests, admissions wait for regions to come back (never more bytes in use
    than the budget, some requests waiting), every request completes with the
    result it has alone, every region comes back; after about 0.2 s without
    work the loop's launch ends with GC_ETIMEDOUT, and the next request starts
    it again."""
    import paper_1403_0555_b300 as gb
    d, L, n = 4, 4, 40_000
    opt = gb.gc_options_default(precision=1, check_every=4)
    phi = oi.von_mises_orbit(d, L, 1.0, 7)
    # the estimate of one request: the smallest budget that takes it (bisection in MiB)
    def takes(mib):
        srv = gb.gc_server_create(1, mib << 20, opt)
        try:
            gb.gc_server_submit(srv, d, L, phi, 7, n)
            return True
        except gb.GribovError as e:
            assert e.code == gb.GC_ENOMEM
            return False
        finally:
            gb.gc_server_destroy(srv)
    lo, hi = 1, 4096
    assert takes(hi) and not takes(lo)
    while hi - lo > 1:
        mid = (lo + hi) // 2
        lo, hi = (lo, mid) if takes(mid) else (mid, hi)
    est = hi << 20
    srv = gb.gc_server_create(4, est * 3 // 2, opt)
    try:
        tickets = [(gb.gc_server_submit(srv, d, L, oi.von_mises_orbit(d, L, 1.0, 30 + i), 30 + i, n), i)
                   for i in range(6)]
        seen_waiting = 0
        for _ in range(200):
            s = gb.gc_server_state(srv)
            assert s["bytes_in_use"] <= s["budget_bytes"]
            seen_waiting = max(seen_waiting, s["waiting"])
            if s["admitted"] == len(tickets):
                break
            time.sleep(0.005)
        assert seen_waiting >= 1
        for t, i in tickets:
            status, latency, orb = gb.gc_server_wait(srv, t, 120.0)
            assert status == gb.GC_OK and orb is not None
            served = gb.gc_fetch_copies(orb, L ** d)
            gb.gc_destroy_orbit(orb)
            _, alone, _ = run_gpu(d, L, oi.von_mises_orbit(d, L, 1.0, 30 + i), 30 + i, n, keep_per_start=0,
                                  precision=1, check_every=4)
            for k in ("F", "first_start", "count", "region", "lambda2", "theta"):
                assert np.array_equal(served[k], alone[k]), k
        time.sleep(0.2)
        s = gb.gc_server_state(srv)
        assert s["admitted"] == 6 and s["released"] == 6 and s["bytes_in_use"] == 0 and s["waiting"] == 0
        time.sleep(0.6)                                   # idle: the loop's launch ends
        s = gb.gc_server_state(srv)
        assert s["loop_running"] == 0 and s["loop_status"] == gb.GC_ETIMEDOUT
        launches = s["loop_launches"]
        t = gb.gc_server_submit(srv, d, L, oi.von_mises_orbit(d, L, 1.0, 40), 40, 5000)
        status, latency, orb = gb.gc_server_wait(srv, t, 120.0, keep_orbit=False)
        assert status == gb.GC_OK
        s = gb.gc_server_state(srv)
        assert s["loop_launches"] == launches + 1 and s["admitted"] == 7
    finally:
        gb.gc_server_destroy(srv)
