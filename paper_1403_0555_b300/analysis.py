"""Paper-style statistics on the enumerator's output (Section IV).

All enumeration runs through the library; these helpers only count and
average what gc_fetch_copies / gc_orbit_stats return.

* discovery_curve: distinct copies found within the first n starts, for the
  powers of two the paper samples at (Figs. 1-3).  A copy's first start is
  the lowest start index that reaches it, so the count for n starts is the
  number of copies whose first start is below n.
* table_statistics: over random orbits at beta = 0 (link angles uniform), the
  number of distinct minima per orbit (Table I; counted as the paper does,
  by the functional quantised at 1e-8, and by configuration identity) and the
  global-minimum functional F/(dV) (Table III), with standard deviations.
"""
from __future__ import annotations

import math

import numpy as np


def discovery_curve(first_start: np.ndarray, n_starts: int) -> tuple[np.ndarray, np.ndarray]:
    """(n, distinct copies within the first n starts) for n = 1, 2, 4, ..., n_starts."""
    fs = np.sort(np.asarray(first_start, dtype=np.int64))
    ns = [1 << k for k in range(int(math.log2(max(1, n_starts))) + 1)]
    if ns[-1] != n_starts:
        ns.append(n_starts)
    ns = np.asarray(ns, dtype=np.int64)
    return ns, np.searchsorted(fs, ns, side="left")


def table_statistics(d: int, N: int, n_orbits: int, n_starts: int, omega: float = 1.0,
                     precision: int | None = None, seed0: int = 1, check_every: int = 4,
                     curve: bool = False) -> dict:
    """Enumerate n_orbits uniform orbits of N^d with n_starts starts each.

    Orbit j uses link angles from seed seed0 + j (orbit id = seed).  Returns
    the means and standard deviations across orbits of the paper-style count
    of distinct minima (n_distinct_F8), of distinct canonical copies, and of
    the global minimum of F/(dV); with `curve`, the discovery curve averaged
    over the orbits.
    """
    import orbit_inputs as oi
    import paper_1403_0555_b300 as gb

    if precision is None:
        precision = gb.GC_MIXED
    V = N ** d
    opt = gb.gc_options_default(precision=precision, check_every=check_every)
    f8, nd, fmin, nconv, curves = [], [], [], [], []
    for j in range(n_orbits):
        seed = seed0 + j
        h = gb.gc_create_orbit(d, N, oi.uniform_orbit(d, N, seed), seed)
        try:
            gb.gc_enumerate_copies(h, n_starts, omega, 1e-24, opt)
            st = gb.gc_orbit_stats(h)
            c = gb.gc_fetch_copies(h, V, theta=False)
        finally:
            gb.gc_destroy_orbit(h)
        f8.append(st["n_distinct_F8"])
        nd.append(st["n_distinct"])
        nconv.append(st["n_converged"] / n_starts)
        fmin.append(float(c["F"].min()) / (d * V) if c["n_distinct"] else float("nan"))
        if curve:
            curves.append(discovery_curve(c["first_start"], n_starts)[1])

    def ms(x):
        x = np.asarray(x, dtype=float)
        return float(x.mean()), float(x.std(ddof=1)) if len(x) > 1 else 0.0

    out = {"d": d, "N": N, "orbits": n_orbits, "starts_per_orbit": n_starts, "omega": omega,
           "minima_F8": ms(f8), "copies": ms(nd), "global_min_F_per_link": ms(fmin),
           "converged_fraction": ms(nconv)}
    if curve:
        out["curve_n"] = discovery_curve(np.zeros(0), n_starts)[0].tolist()
        out["curve_mean"] = np.mean(np.asarray(curves, dtype=float), axis=0).tolist()
    return out
