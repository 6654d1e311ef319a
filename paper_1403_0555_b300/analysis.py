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
* minima_histogram, histogram_ratio, normalised_distribution: the binned
  distribution of the functional at the minima (Section IV: Fig. 5 compares
  two sample sizes bin by bin at resolution 1e-4, Fig. 7 shows the normalised
  distribution over all orbits and samples).
* relative_deviation, relative_deviation_stats: (F_i - F_g)/F_g of the local
  minima against the orbit's global minimum, averaged over orbits (Fig. 8).
* fit_count_growth: the fit of Eq. 6, h(N) = a exp(b N^c), to the number of
  minima per lattice size (Fig. 4, Table II).
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


def orbit_runs(d: int, N: int, n_orbits: int, n_starts: int, omega: float = 1.0,
               precision: int | None = None, seed0: int = 1, check_every: int = 4):
    """Enumerate n_orbits uniform orbits of N^d with n_starts starts each and
    yield (stats, copies) per orbit.  Orbit j uses link angles from seed
    seed0 + j (orbit id = seed)."""
    import orbit_inputs as oi
    import paper_1403_0555_b300 as gb

    if precision is None:
        precision = gb.GC_MIXED
    V = N ** d
    opt = gb.gc_options_default(precision=precision, check_every=check_every)
    for j in range(n_orbits):
        seed = seed0 + j
        h = gb.gc_create_orbit(d, N, oi.uniform_orbit(d, N, seed), seed)
        try:
            gb.gc_enumerate_copies(h, n_starts, omega, 1e-24, opt)
            st = gb.gc_orbit_stats(h)
            c = gb.gc_fetch_copies(h, V, theta=False)
        finally:
            gb.gc_destroy_orbit(h)
        yield st, c


def _mean_std(x):
    x = np.asarray(x, dtype=float)
    return float(x.mean()), float(x.std(ddof=1)) if len(x) > 1 else 0.0


def table_statistics(d: int, N: int, n_orbits: int, n_starts: int, omega: float = 1.0,
                     precision: int | None = None, seed0: int = 1, check_every: int = 4,
                     curve: bool = False) -> dict:
    """Enumerate n_orbits uniform orbits of N^d with n_starts starts each.

    Returns the means and standard deviations across orbits of the paper-style
    count of distinct minima (n_distinct_F8), of distinct canonical copies, and
    of the global minimum of F/(dV); with `curve`, the discovery curve averaged
    over the orbits.
    """
    V = N ** d
    f8, nd, fmin, nconv, curves = [], [], [], [], []
    for st, c in orbit_runs(d, N, n_orbits, n_starts, omega, precision, seed0, check_every):
        f8.append(st["n_distinct_F8"])
        nd.append(st["n_distinct"])
        nconv.append(st["n_converged"] / n_starts)
        fmin.append(float(c["F"].min()) / (d * V) if c["n_distinct"] else float("nan"))
        if curve:
            curves.append(discovery_curve(c["first_start"], n_starts)[1])
    out = {"d": d, "N": N, "orbits": n_orbits, "starts_per_orbit": n_starts, "omega": omega,
           "minima_F8": _mean_std(f8), "copies": _mean_std(nd), "global_min_F_per_link": _mean_std(fmin),
           "converged_fraction": _mean_std(nconv)}
    if curve:
        out["curve_n"] = discovery_curve(np.zeros(0), n_starts)[0].tolist()
        out["curve_mean"] = np.mean(np.asarray(curves, dtype=float), axis=0).tolist()
    return out


def section_iv_statistics(d: int, N: int, n_orbits: int, n_starts: int, omega: float = 1.0,
                          precision: int | None = None, seed0: int = 1, check_every: int = 4,
                          width: float = 1e-3) -> dict:
    """Section IV over n_orbits uniform orbits of N^d: the global minimum of
    F/(dV) per orbit (Table III, Fig. 6), the relative deviation of the
    minima from it (Fig. 8; minima counted as the paper does, by F/(dV)
    quantised at 1e-8), over the distinct minima and over the samples, and
    the normalised distribution of F/(dV) over all orbits and samples (Fig. 7)
    as bin left edges and density at `width`."""
    V = N ** d
    fmin, minima, mcount, Fs, ws = [], [], [], [], []
    for st, c in orbit_runs(d, N, n_orbits, n_starts, omega, precision, seed0, check_every):
        Fn = c["F"] / (d * V)
        fmin.append(float(Fn.min()))
        keys, inv = np.unique(np.floor(Fn * 1e8), return_inverse=True)
        minima.append(keys * 1e-8)
        mcount.append(np.bincount(inv, weights=c["count"].astype(np.float64)))
        Fs.append(Fn)
        ws.append(c["count"])
    rel = relative_deviation_stats(minima)
    rel_s = relative_deviation_stats(minima, mcount)
    edges, dens = normalised_distribution(Fs, ws, width)
    return {"d": d, "N": N, "orbits": n_orbits, "starts_per_orbit": n_starts, "omega": omega,
            "global_min_F_per_link": _mean_std(fmin),
            "relative_deviation": {"mean": rel["mean"], "std": rel["std"]},
            "relative_deviation_samples": {"mean": rel_s["mean"], "std": rel_s["std"]},
            "distribution": {"width": width, "left_edges": edges.tolist(), "density": dens.tolist()}}


def compare_sample_sizes(d: int, N: int, n_orbits: int, n_small: int, n_large: int,
                         omega: float = 1.0, precision: int | None = None, seed0: int = 1,
                         check_every: int = 4, width: float = 1e-4) -> dict:
    """Fig. 5: the same orbits enumerated with n_small and n_large starts; the
    sample-weighted histograms of F/(dV) over all orbits at resolution `width`,
    bin by bin.  Reports the expected ratio n_large / n_small, the median
    ratio over the bins of the lower, middle and upper third of the F range,
    and the bins the small run left empty."""
    V = N ** d
    runs = {}
    for n in (n_small, n_large):
        Fs, ws = [], []
        for _, c in orbit_runs(d, N, n_orbits, n, omega, precision, seed0, check_every):
            Fs.append(c["F"] / (d * V))
            ws.append(c["count"])
        runs[n] = minima_histogram(np.concatenate(Fs), np.concatenate(ws), width)
    (bl, cl), (bs, cs) = runs[n_large], runs[n_small]
    r = histogram_ratio(bl, cl, bs, cs)
    lo, hi = bl.min(), bl.max()
    thirds = {}
    for name, (a, b) in {"low": (lo, lo + (hi - lo) / 3), "mid": (lo + (hi - lo) / 3, lo + 2 * (hi - lo) / 3),
                         "high": (lo + 2 * (hi - lo) / 3, hi + 1)}.items():
        m = (r["bins"] >= a) & (r["bins"] < b)
        thirds[name] = {"bins": int(m.sum()), "median_ratio": float(np.median(r["ratio"][m])) if m.any() else None}
    return {"d": d, "N": N, "orbits": n_orbits, "n_small": n_small, "n_large": n_large,
            "expected_ratio": n_large / n_small, "bins_both": int(len(r["bins"])), "ratio_by_third": thirds,
            "bins_only_large": int(len(r["only_a"])), "samples_in_bins_only_large": float(r["only_a_counts"].sum()),
            "only_large_lowest_F_per_link": float(r["only_a"].min() * width) if len(r["only_a"]) else None,
            "bins_only_small": int(len(r["only_b"]))}


# ---------------------------------------------------------------------------
# Section IV: distribution of the functional at the minima, and Eq. 6
# ---------------------------------------------------------------------------
def minima_histogram(F_norm, weights=None, width: float = 1e-4) -> tuple[np.ndarray, np.ndarray]:
    """(bin index j, count) over the occupied bins; bin j holds F_norm in
    [j width, (j + 1) width).  With `weights` (each copy's number of converged
    starts) the entries count samples, as in Fig. 5, where the bins of two runs
    differ by their ratio of samples; without, distinct minima."""
    F_norm = np.asarray(F_norm, dtype=np.float64)
    j = np.floor(F_norm / width).astype(np.int64)
    w = np.ones(len(j)) if weights is None else np.asarray(weights, dtype=np.float64)
    bins, inv = np.unique(j, return_inverse=True)
    return bins, np.bincount(inv, weights=w, minlength=len(bins))


def histogram_ratio(bins_a, counts_a, bins_b, counts_b) -> dict:
    """Fig. 5: for the bins occupied in both runs, counts_a / counts_b; and the
    bins occupied in run a only (run b's bin empty, the ratio undefined) with
    run a's counts.  Run b's bins that run a lacks are listed too."""
    bins_a, bins_b = np.asarray(bins_a), np.asarray(bins_b)
    both, ia, ib = np.intersect1d(bins_a, bins_b, return_indices=True)
    only_a = np.setdiff1d(bins_a, bins_b)
    only_b = np.setdiff1d(bins_b, bins_a)
    return {"bins": both, "ratio": np.asarray(counts_a)[ia] / np.asarray(counts_b)[ib],
            "only_a": only_a, "only_a_counts": np.asarray(counts_a)[np.searchsorted(bins_a, only_a)],
            "only_b": only_b}


def normalised_distribution(F_norm_per_orbit, weights_per_orbit=None, width: float = 1e-2):
    """Fig. 7: the distribution of F_norm over all orbits and samples (entries
    weighted by their sample counts when given), as a density: bin left edges
    and values integrating to 1."""
    F = np.concatenate([np.asarray(f, dtype=np.float64) for f in F_norm_per_orbit])
    w = None if weights_per_orbit is None else np.concatenate(
        [np.asarray(x, dtype=np.float64) for x in weights_per_orbit])
    bins, counts = minima_histogram(F, w, width)
    return bins * width, counts / (counts.sum() * width)


def relative_deviation(F) -> np.ndarray:
    """(F_i - F_g)/F_g for the minima F_i of one orbit, F_g their minimum (Fig. 8)."""
    F = np.asarray(F, dtype=np.float64)
    Fg = F.min()
    return (F - Fg) / Fg


def relative_deviation_stats(F_per_orbit, weights_per_orbit=None) -> dict:
    """Fig. 8: per orbit the mean and standard deviation of the relative
    deviation over its distinct minima, then their averages over the orbits.
    With weights (each minimum's number of starts) the per-orbit moments are
    taken over the samples instead."""
    means, stds = [], []
    for j, F in enumerate(F_per_orbit):
        r = relative_deviation(F)
        if weights_per_orbit is None:
            means.append(r.mean())
            stds.append(r.std(ddof=1) if len(r) > 1 else 0.0)
        else:
            w = np.asarray(weights_per_orbit[j], dtype=np.float64)
            m = float(np.sum(w * r) / w.sum())
            means.append(m)
            stds.append(float(np.sqrt(np.sum(w * (r - m) ** 2) / w.sum())))
    return {"mean": float(np.mean(means)), "std": float(np.mean(stds)), "orbits": len(means),
            "mean_per_orbit": [float(m) for m in means]}


def fit_count_growth(N, counts, sigma=None, a: float | None = None) -> dict:
    """Eq. 6, h(N) = a exp(b N^c), fitted to the number of minima per lattice
    size by least squares, weighted by `sigma` when given (the spread of the
    counts over orbits).  With `a` given it is held fixed (the paper fixes
    a = 1 for d = 4).  As many points as free parameters give the exact
    solution, without uncertainties; otherwise the uncertainties are the
    square roots of the covariance's diagonal."""
    import warnings
    from scipy.optimize import OptimizeWarning, curve_fit

    N = np.asarray(N, dtype=np.float64)
    y = np.asarray(counts, dtype=np.float64)
    # starting point: log h = log a + b N^c through the two outer points, c = 2
    c0 = 2.0
    b0 = (np.log(y[-1]) - np.log(y[0])) / (N[-1] ** c0 - N[0] ** c0)
    la0 = np.log(y[0]) - b0 * N[0] ** c0
    with warnings.catch_warnings():
        warnings.simplefilter("ignore", OptimizeWarning)
        if a is None:
            # first in log space (well conditioned), then in counts
            p, _ = curve_fit(lambda x, la, b, c: la + b * x ** c, N, np.log(y), p0=(la0, b0, c0), maxfev=20000)
            p, cov = curve_fit(lambda x, aa, b, c: aa * np.exp(b * x ** c), N, y, p0=(np.exp(p[0]), p[1], p[2]),
                               sigma=sigma, absolute_sigma=sigma is not None, maxfev=20000)
            names, vals = ("a", "b", "c"), p
        else:
            p, _ = curve_fit(lambda x, b, c: np.log(a) + b * x ** c, N, np.log(y), p0=(b0, c0), maxfev=20000)
            p, cov = curve_fit(lambda x, b, c: a * np.exp(b * x ** c), N, y, p0=p,
                               sigma=sigma, absolute_sigma=sigma is not None, maxfev=20000)
            names, vals = ("b", "c"), p
    out = {"a": float(a) if a is not None else None}
    exact = len(N) <= len(names)
    err = np.sqrt(np.diag(cov)) if not exact and np.all(np.isfinite(cov)) else [None] * len(names)
    for k, v, e in zip(names, vals, err):
        out[k] = float(v)
        out[k + "_err"] = None if e is None else float(e)
    return out
