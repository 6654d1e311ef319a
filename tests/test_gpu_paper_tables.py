"""The enumerator's paper-style statistics against the values the paper
prints (Table I: distinct minima per orbit; Table III: global-minimum
F/(dV)), over random uniform orbits at omega = 1 as in the paper, through the
library's mixed path.  Tolerance: 3.5 standard errors of the difference of two
sample means (the paper's 100 orbits, ours)."""
import json
import math
import os

import pytest

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")


@pytest.mark.parametrize("d,N", [(2, 2), (2, 4), (3, 2), (4, 2)])
def test_tables_I_and_III_on_the_gpu(d, N):
    from paper_1403_0555_b300.analysis import table_statistics
    g = json.load(open(GOLDEN))
    t1 = next(r for r in g["table_I"]["rows"] if r["d"] == d and r["N"] == N)
    t3 = next(r for r in g["table_III"]["rows"] if r["d"] == d and r["N"] == N)
    n_orbits = 100
    st = table_statistics(d, N, n_orbits, 1 << 20, omega=1.0, curve=True)
    m1, s1 = st["minima_F8"]
    se1 = math.sqrt(t1["std"] ** 2 / t1["orbits"] + s1 ** 2 / n_orbits)
    assert abs(m1 - t1["avg_minima"]) < 3.5 * se1, (st, t1)
    m3, s3 = st["global_min_F_per_link"]
    se3 = math.sqrt(t3["std"] ** 2 / t3["orbits"] + s3 ** 2 / n_orbits)
    assert abs(m3 - t3["avg_Fmin"]) < 3.5 * se3, (st, t3)
    # the discovery curve is non-decreasing and ends at the per-orbit copy count
    c = st["curve_mean"]
    assert all(b >= a for a, b in zip(c, c[1:]))
    assert abs(c[-1] - st["copies"][0]) < 1e-9
    assert st["converged_fraction"][0] > 0.999
