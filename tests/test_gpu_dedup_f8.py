"""The paper's count of minima (Section III: minima told apart by F/(dV)
quantised at 1e-8) as fetched from the library, and the F-only dedup mode,
which keeps that set without the configuration table."""
import numpy as np
import pytest

import oracle
import orbit_inputs as oi

pytestmark = pytest.mark.gpu


def _run(gb, d, L, phi, orbit_id, n, omega, eps, **opt):
    h = gb.gc_create_orbit(d, L, phi, orbit_id)
    try:
        gb.gc_enumerate_copies(h, n, omega, eps, gb.gc_options_default(**opt))
        return gb.gc_orbit_stats(h), gb.gc_fetch_minima_f8(h), gb.gc_fetch_copies(h, L ** d, theta=False)
    finally:
        gb.gc_destroy_orbit(h)


def test_minima_f8_equal_the_oracle_on_the_parity_workload():
    """2D 4^2, uniform orbit from seed 1, 10^4 starts, plain FP64 path (bit-exact
    start by start): the quantised minima and their start counts equal the
    oracle's, in both dedup modes."""
    import paper_1403_0555_b300 as gb
    w = oi.workload_2d_4x4()
    o = w.orbits[0]
    d, L, n = o.d, o.L, w.n_starts
    rel = oracle.relax_starts(d, L, o.phi, 1, o.orbit_id, 0, n, w.omega, w.eps)
    _, theta = oracle.canonical(rel.g)
    F = oracle.functional(d, L, o.phi, theta)
    conv = rel.status == oracle.CONVERGED
    keys, counts = np.unique(np.floor(oracle.f_norm(F[conv], d, L) * 1e8).astype(np.int64), return_counts=True)
    for mode in (gb.GC_DEDUP_CONFIG, gb.GC_DEDUP_F8):
        st, m, c = _run(gb, d, L, o.phi, o.orbit_id, n, w.omega, w.eps,
                        precision=gb.GC_FP64, check_every=1, dedup_mode=mode)
        assert m["n_minima"] == st["n_distinct_F8"] == len(keys)
        assert np.array_equal(np.round(m["F_norm"] * 1e8).astype(np.int64), keys)
        assert np.array_equal(m["count"].astype(np.int64), counts)
        assert int(m["count"].sum()) == st["n_converged"] == int(conv.sum())
        if mode == gb.GC_DEDUP_F8:
            assert st["n_distinct"] == 0 and c["n_distinct"] == 0
        else:
            assert st["n_distinct"] > 0


def test_f8_mode_keeps_the_same_set_on_the_mixed_path():
    """4D 4^4 von Mises orbit, 2^16 starts, mixed path: the F-only mode leaves
    relaxation and polish unchanged, so its quantised minima and counts equal
    those kept beside the configuration table; it makes no copies and runs no
    first-region test."""
    import paper_1403_0555_b300 as gb
    d, L, n = 4, 4, 1 << 16
    phi = oi.von_mises_orbit(d, L, 0.5, 3)
    st_c, m_c, _ = _run(gb, d, L, phi, 3, n, 1.7, 1e-24, precision=gb.GC_MIXED, check_every=4)
    st_f, m_f, c_f = _run(gb, d, L, phi, 3, n, 1.7, 1e-24, precision=gb.GC_MIXED, check_every=4,
                          dedup_mode=gb.GC_DEDUP_F8)
    assert st_f["n_converged"] == st_c["n_converged"]
    assert m_f["n_minima"] == m_c["n_minima"] == st_c["n_distinct_F8"]
    assert np.array_equal(m_f["F_norm"], m_c["F_norm"]) and np.array_equal(m_f["count"], m_c["count"])
    assert np.all(np.diff(m_f["F_norm"]) > 0)
    assert st_f["n_distinct"] == 0 and c_f["n_distinct"] == 0 and st_f["fp_tests"] == 0
    # every configuration copy's F falls in one of the quantised minima
    _, _, c_c = _run(gb, d, L, phi, 3, 1 << 12, 1.7, 1e-24, precision=gb.GC_MIXED, check_every=4)
    k = np.floor(c_c["F"] / (d * L ** d) * 1e8) * 1e-8
    assert np.all(np.isin(np.round(k * 1e8), np.round(m_c["F_norm"] * 1e8)))


def test_dedup_mode_is_validated():
    import paper_1403_0555_b300 as gb
    h = gb.gc_create_orbit(2, 4, oi.uniform_orbit(2, 4, 1), 1)
    try:
        with pytest.raises(gb.GribovError):
            gb.gc_enumerate_copies(h, 16, 1.7, 1e-24, gb.gc_options_default(dedup_mode=7))
    finally:
        gb.gc_destroy_orbit(h)
