"""Host-side statistics on enumerator output (Section IV): the binned
distribution of the functional at the minima (Figs. 5, 7), the relative
deviation from the global minimum (Fig. 8) and the fit of Eq. 6 (Table II).

Pins: the fit of Eq. 6 to the paper's own Table I reproduces its Table II;
synthetic counts drawn from Eq. 6 give their parameters back; histograms,
ratios and deviations on hand-made inputs with known answers.
"""
import json
import os

import numpy as np
import pytest

from paper_1403_0555_b300 import analysis as an

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")


def _table(d):
    g = json.load(open(GOLDEN))
    rows = [r for r in g["table_I_all"]["rows"] if r["d"] == d]
    fit = next(r for r in g["table_II"]["rows"] if r["d"] == d)
    return rows, fit


def test_eq6_fit_to_table_I_reproduces_table_II_d2():
    """d = 2: five lattice sizes, weighted by the spread over orbits; every
    parameter within one printed uncertainty of Table II."""
    rows, fit = _table(2)
    r = an.fit_count_growth([x["N"] for x in rows], [x["avg_minima"] for x in rows],
                            sigma=[x["std"] for x in rows])
    for k in ("a", "b", "c"):
        assert abs(r[k] - fit[k]) <= fit[k + "_err"], (k, r[k], fit[k])


def test_eq6_fit_to_table_I_reproduces_table_II_d3_exact():
    """d = 3: three sizes fix the three parameters; Table II prints them to
    three digits."""
    rows, fit = _table(3)
    r = an.fit_count_growth([x["N"] for x in rows], [x["avg_minima"] for x in rows])
    assert r["a_err"] is None
    for k in ("a", "b", "c"):
        assert abs(r[k] - fit[k]) <= 0.002 * fit[k] + 5e-4, (k, r[k], fit[k])


def test_eq6_fit_to_table_I_reproduces_table_II_d4_fixed_a():
    """d = 4: a = 1 fixed, two sizes fix b and c; Table II's values follow from
    Table I's rounded averages to within 3 %."""
    rows, fit = _table(4)
    r = an.fit_count_growth([x["N"] for x in rows], [x["avg_minima"] for x in rows], a=1.0)
    assert r["a"] == 1.0
    for k in ("b", "c"):
        assert abs(r[k] - fit[k]) <= 0.03 * fit[k], (k, r[k], fit[k])


@pytest.mark.parametrize("a,b,c", [(0.5, 0.2, 1.8), (2.0, 0.05, 2.6), (1.0, 0.3, 1.2)])
def test_eq6_fit_recovers_synthetic_parameters(a, b, c):
    N = np.array([2, 3, 4, 5, 6, 7], dtype=float)
    y = a * np.exp(b * N ** c)
    r = an.fit_count_growth(N, y, sigma=0.01 * y)
    assert r["a"] == pytest.approx(a, rel=1e-5)
    assert r["b"] == pytest.approx(b, rel=1e-5)
    assert r["c"] == pytest.approx(c, rel=1e-5)


def test_minima_histogram_bins_and_weights():
    F = np.array([0.20001, 0.20009, 0.20011, 0.5, 0.49999])
    bins, counts = an.minima_histogram(F)
    # 1e-4 bins: [0.2000, 0.2001) holds two, [0.2001, 0.2002) one, 0.49999 and 0.5 apart
    assert list(bins) == [2000, 2001, 4999, 5000]
    assert list(counts) == [2, 1, 1, 1]
    bins, counts = an.minima_histogram(F, weights=[3, 4, 5, 6, 7])
    assert list(counts) == [7, 5, 7, 6]
    assert counts.sum() == 25


def test_histogram_ratio_and_bins_of_one_run_only():
    ba, ca = np.array([1, 2, 3, 7]), np.array([64.0, 128.0, 32.0, 5.0])
    bb, cb = np.array([1, 2, 3, 9]), np.array([1.0, 2.0, 0.5, 1.0])
    r = an.histogram_ratio(ba, ca, bb, cb)
    assert list(r["bins"]) == [1, 2, 3]
    assert np.all(r["ratio"] == 64.0)
    assert list(r["only_a"]) == [7] and list(r["only_a_counts"]) == [5.0]
    assert list(r["only_b"]) == [9]


def test_normalised_distribution_integrates_to_one():
    rng = np.random.default_rng(4)
    F = [rng.uniform(0.2, 0.4, 500), rng.uniform(0.25, 0.45, 300)]
    w = [rng.integers(1, 9, 500), rng.integers(1, 9, 300)]
    edges, dens = an.normalised_distribution(F, w, width=0.01)
    assert np.sum(dens) * 0.01 == pytest.approx(1.0, rel=1e-12)
    assert edges.min() >= 0.19 and edges.max() < 0.45


def test_relative_deviation_and_orbit_averages():
    r = an.relative_deviation([0.25, 0.3, 0.5])
    assert r == pytest.approx([0.0, 0.2, 1.0])
    s = an.relative_deviation_stats([[0.25, 0.3, 0.5], [0.4, 0.4 * 1.1]])
    m1, m2 = np.mean([0.0, 0.2, 1.0]), np.mean([0.0, 0.1])
    assert s["mean"] == pytest.approx((m1 + m2) / 2)
    assert s["std"] == pytest.approx((np.std([0.0, 0.2, 1.0], ddof=1) + np.std([0.0, 0.1], ddof=1)) / 2)
    # a single minimum deviates by nothing
    assert an.relative_deviation_stats([[0.3]])["mean"] == 0.0
    # over samples: minima 0.25 (3 starts) and 0.5 (1 start): deviations 0, 1
    w = an.relative_deviation_stats([[0.25, 0.5]], [[3, 1]])
    assert w["mean"] == pytest.approx(0.25)
    assert w["std"] == pytest.approx(np.sqrt(0.75 * 0.25 ** 2 + 0.25 * 0.75 ** 2))
