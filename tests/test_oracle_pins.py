"""Pins of the oracle to facts fixed by the paper and by the mathematics.

Each test checks the oracle against something other than itself: numpy's
independent Philox, closed forms (1D periodic chain, constant-field plane
waves, Laplacian spectra), gauge invariance, brute-force enumeration of every
stationary point of a 2x2 lattice with the Morse-theory sum of Eq. 2, and the
orbit statistics printed in Tables I and III.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import orbit_inputs as oi

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")


# ----------------------------------------------------------------------------
# random starts
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("key", [(0, 0), (1, 2), (2**63 + 5, 12345)])
def test_philox_matches_numpy(key):
    # numpy.random.Philox is an independent Philox4x64-10; it advances its
    # counter before producing a block, so its block at counter c is ours at c+1.
    for c in (0, 1, 7, 2**40):
        bg = np.random.Philox(key=np.array(key, dtype=np.uint64),
                              counter=np.array([c, 0, 0, 0], dtype=np.uint64))
        ref = bg.random_raw(4)
        mine = oracle.philox4x64_10([c + 1, 0, 0, 0], key)
        assert (mine == ref).all()


def test_start_is_uniform_on_circle():
    from scipy import stats
    V = 64
    g = np.concatenate([oracle.random_start(V, 3, 9, s) for s in range(200)])
    assert np.allclose(np.hypot(g[:, 0], g[:, 1]), 1.0, atol=2e-16)
    ang = (np.arctan2(g[:, 1], g[:, 0]) + math.pi) / (2 * math.pi)
    assert stats.kstest(ang, "uniform").pvalue > 1e-3
    # counter-based: a start depends only on (seed, orbit, start index)
    assert np.array_equal(oracle.random_start(V, 3, 9, 17), oracle.random_start(V, 3, 9, 17))
    assert not np.array_equal(oracle.random_start(V, 3, 9, 17), oracle.random_start(V, 3, 10, 17))


# ----------------------------------------------------------------------------
# local update and residual
# ----------------------------------------------------------------------------

def _random_state(V, seed):
    t = np.random.default_rng(seed).uniform(-math.pi, math.pi, V)
    return np.stack([np.cos(t), np.sin(t)], axis=1), t


@pytest.mark.parametrize("d,L", [(1, 5), (2, 4), (2, 5), (3, 3), (4, 2)])
def test_divergence_is_minus_gradient(d, L):
    # div_x = sum_mu [sin(phi^theta_{x,mu}) - sin(phi^theta_{x-mu,mu})] from the angles,
    # and equals -dF/dtheta_x by central finite differences of Eq. 3.
    phi = oi.uniform_orbit(d, L, 11)
    g, t = _random_state(L ** d, 12)
    div = oracle.divergence(d, L, phi, g)
    V = L ** d
    coords = oi.site_coords(d, L)
    ref = np.zeros(V)
    for x in range(V):
        for mu in range(d):
            c = coords[x].copy(); c[mu] = (c[mu] + 1) % L
            xp = int((c * L ** np.arange(d)).sum())
            c = coords[x].copy(); c[mu] = (c[mu] - 1) % L
            xm = int((c * L ** np.arange(d)).sum())
            ref[x] += math.sin(phi[x, mu] + t[xp] - t[x]) - math.sin(phi[xm, mu] + t[x] - t[xm])
    assert np.max(np.abs(div - ref)) < 1e-13

    def F_of(tt):
        tot = 0.0
        for x in range(V):
            for mu in range(d):
                c = coords[x].copy(); c[mu] = (c[mu] + 1) % L
                xp = int((c * L ** np.arange(d)).sum())
                tot += 1 - math.cos(phi[x, mu] + tt[xp] - tt[x])
        return tot
    h = 1e-6
    for x in range(min(V, 6)):
        tp = t.copy(); tp[x] += h
        tm = t.copy(); tm[x] -= h
        assert abs(-(F_of(tp) - F_of(tm)) / (2 * h) - div[x]) < 1e-7


@pytest.mark.parametrize("d,L", [(2, 4), (2, 5), (3, 4), (4, 3)])
def test_plain_sweep_reaches_local_optimum_on_last_colour(d, L):
    # At omega = 1 the update sets theta_x = arg S_x (Eq. 4/5).  After a full
    # sweep nothing adjacent to the last colour moves again, so every site of
    # that colour has zero divergence.
    phi = oi.uniform_orbit(d, L, 5)
    g, _ = _random_state(L ** d, 6)
    g1 = oracle.sweeps(d, L, phi, 1.0, 1, g)
    col, nc = oracle.colors(d, L)
    div = oracle.divergence(d, L, phi, g1)
    assert np.max(np.abs(div[col == nc - 1])) < 1e-13
    assert np.max(np.abs(div[col == 0])) > 1e-3   # earlier colours are not at rest


@pytest.mark.parametrize("omega", [1.0, 1.3, 1.7, 1.95])
@pytest.mark.parametrize("d,L", [(2, 6), (3, 3), (4, 4)])
def test_sweeps_never_increase_functional(d, L, omega):
    # Each site move lowers its local part of Eq. 3 (the overrelaxed point lies
    # strictly closer in angle to arg S_x than the old one for 0 < omega < 2).
    phi = oi.von_mises_orbit(d, L, 0.7, 21)
    g, _ = _random_state(L ** d, 22)
    F_prev = oracle.functional(d, L, phi, np.arctan2(g[:, 1], g[:, 0]))
    for _ in range(25):
        g = oracle.sweeps(d, L, phi, omega, 1, g)
        F = oracle.functional(d, L, phi, np.arctan2(g[:, 1], g[:, 0]))
        assert F <= F_prev + 1e-12
        F_prev = F


def test_colouring_is_proper():
    for d in (1, 2, 3, 4):
        for L in (2, 3, 4, 5, 6, 7):
            if L ** d > 3000:
                continue
            col, nc = oracle.colors(d, L)
            assert nc == (2 if L % 2 == 0 else 3)
            for mu in range(d):
                nb = oi.shifted_index(d, L, mu, +1)
                assert np.all(col != col[nb])


# ----------------------------------------------------------------------------
# closed forms
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("L,Phi", [(3, 0.4), (5, -1.1), (7, 2.0), (8, 0.3), (6, 3.0)])
def test_1d_closed_form(L, Phi):
    # d = 1, periodic chain: div = 0 forces sin(phi^theta) constant along the
    # ring; a weighted cycle Laplacian is PSD on 1^perp only when all weights
    # are positive (one negative weight gives sum 1/w > 0 for L >= 3 only if ...
    # the mixed a / pi-a solutions are saddles).  So the first-region copies
    # are exactly phi^theta_x = wrap((Phi + 2 pi k)/L) for all x with
    # cos((Phi + 2 pi k)/L) > 0, with F = L (1 - cos(.)).
    rng = np.random.default_rng(L)
    phi = rng.uniform(-math.pi, math.pi, (L, 1))
    phi[-1, 0] += Phi - phi[:, 0].sum()
    phi = oi.wrap(phi)
    pred_all, pred_robust = [], []
    for k in range(L):
        a = (Phi + 2 * math.pi * k) / L
        if math.cos(a) > 0:
            pred_all.append(L * (1 - math.cos(a)))
            if math.cos(a) > 0.15:       # copies near the margin have tiny basins
                pred_robust.append(L * (1 - math.cos(a)))
    pred_all = np.array(pred_all)
    relaxed, cp = oracle.enumerate_copies(1, L, phi, seed=1, orbit_id=L, n_starts=4000,
                                          omega=1.7)
    assert (relaxed.status == oracle.CONVERGED).all()
    found = cp.F[cp.region == oracle.REGION_IN]
    assert (cp.region == oracle.REGION_IN).all()
    for f in found:                      # found is a subset of the closed form
        assert np.min(np.abs(pred_all - f)) < 1e-12
    for p in pred_robust:                # and contains every well-separated copy
        assert np.min(np.abs(found - p)) < 1e-12
    # the paper's count (F/(dV) quantised at 1e-8) of the closed-form copies
    # that were found equals the pipeline's count
    x_found = np.array([1 - math.cos((Phi + 2 * math.pi * k) / L) for k in range(L)
                        if math.cos((Phi + 2 * math.pi * k) / L) > 0
                        and np.min(np.abs(found - L * (1 - math.cos((Phi + 2 * math.pi * k) / L)))) < 1e-12])
    assert cp.n_distinct_F8 == len(np.unique(np.floor(x_found * 1e8)))
    # every copy has all gauge-fixed link angles equal
    ang = oracle.link_angles_gauged(1, L, phi, cp.theta)[..., 0]
    spread = np.abs(np.angle(np.exp(1j * (ang - ang[:, :1]))))
    assert spread.max() < 1e-9
    assert (cp.lambda2 > 0).all()


def test_plane_waves_of_constant_field_are_found():
    # phi_{x,mu} = alpha_mu: theta_x = sum_mu 2 pi k_mu x_mu / L is stationary with
    # phi^theta_mu = alpha_mu + 2 pi k_mu / L; it lies in the first region iff
    # every cos > 0 (positive constant weights), with
    # F = V sum_mu (1 - cos(alpha_mu + 2 pi k_mu / L)).  High-F waves have tiny
    # basins, so only the low ones must be found; every plane wave that is
    # found must match the closed form.
    import itertools
    d, L = 2, 6
    alpha = np.array([0.3, -0.2])
    phi = oi.constant_orbit(d, L, alpha)
    pred = []
    for k in itertools.product(range(L), repeat=d):
        a = alpha + 2 * math.pi * np.array(k) / L
        if np.all(np.cos(a) > 0):
            pred.append(L ** d * np.sum(1 - np.cos(a)))
    pred = np.sort(pred)
    _, cp = oracle.enumerate_copies(d, L, phi, seed=2, orbit_id=3, n_starts=20000)
    F_in = cp.F[cp.region == oracle.REGION_IN]
    for p in pred[:3]:
        assert np.min(np.abs(F_in - p)) < 1e-10
    links = oracle.link_angles_gauged(d, L, phi, cp.theta)
    spread = np.abs(np.angle(np.exp(1j * (links - links[:, :1, :])))).max(axis=(1, 2))
    waves = cp.F[spread < 1e-9]
    assert len(waves) >= 3
    for f in waves:
        assert np.min(np.abs(pred - f)) < 1e-10
    assert abs(cp.F[0] - pred[0]) < 1e-10  # the global minimum is the k = 0 wave


@pytest.mark.parametrize("d,L", [(2, 5), (3, 4), (2, 6)])
def test_fp_operator_spectrum_closed_form(d, L):
    # Constant weights w_mu: M is diagonal in Fourier space with eigenvalues
    # sum_mu w_mu (2 - 2 cos(2 pi p_mu / L)).
    import itertools
    w_mu = np.linspace(0.3, 0.9, d)
    w = np.tile(w_mu, (L ** d, 1))
    M = oracle.fp_operator(d, L, w)
    ev = np.sort(np.linalg.eigvalsh(M))
    ref = np.sort([np.sum(w_mu * (2 - 2 * np.cos(2 * math.pi * np.array(p) / L)))
                   for p in itertools.product(range(L), repeat=d)])
    assert np.max(np.abs(ev - ref)) < 1e-12
    assert abs(oracle.lambda2(d, L, w) - ref[1]) < 1e-12
    # cold orbit at theta = const: lambda_2 = 2 - 2 cos(2 pi / L)
    assert abs(oracle.lambda2(d, L, np.ones((L ** d, d))) - (2 - 2 * math.cos(2 * math.pi / L))) < 1e-12


def _jacobi_eigs(A, sweeps=60):
    A = A.copy()
    n = A.shape[0]
    for _ in range(sweeps):
        # off-diagonal norm from the entries themselves (sum A^2 - sum diag^2
        # cancels to rounding noise long before the rotations have converged)
        off = np.sqrt(2.0 * np.sum(np.triu(A, 1) ** 2))
        if off < 1e-14:
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                if abs(A[p, q]) < 1e-300:
                    continue
                th = 0.5 * math.atan2(2 * A[p, q], A[q, q] - A[p, p])
                c, s = math.cos(th), math.sin(th)
                J = np.eye(n)
                J[p, p] = c; J[q, q] = c; J[p, q] = s; J[q, p] = -s
                A = J.T @ A @ J
    return np.sort(np.diag(A))


def test_fp_operator_invariants_and_sign_certificate():
    from scipy.linalg import ldl
    d, L = 2, 4
    phi = oi.uniform_orbit(d, L, 1)
    rng = np.random.default_rng(0)
    for trial in range(6):
        theta = rng.uniform(-math.pi, math.pi, L ** d)
        w = oracle.fp_weights(d, L, phi, theta)
        M = oracle.fp_operator(d, L, w)
        assert np.allclose(M, M.T)
        assert np.max(np.abs(M @ np.ones(L ** d))) < 1e-13
        assert abs(np.trace(M) - 2 * w.sum()) < 1e-12
        ev_j = _jacobi_eigs(M)
        assert np.max(np.abs(ev_j - np.linalg.eigvalsh(M))) < 1e-10
        lam2 = oracle.lambda2(d, L, w)
        # Sylvester: inertia of the grounded matrix (last site removed) equals
        # the spectrum's sign pattern on the complement of the constant mode.
        _, D, _ = ldl(M[:-1, :-1])
        n_neg = int(np.sum(np.linalg.eigvalsh(D) < 0))
        assert (n_neg == 0) == (lam2 > 0)


# ----------------------------------------------------------------------------
# gauge covariance
# ----------------------------------------------------------------------------

def test_gauge_covariance():
    d, L = 3, 4
    V = L ** d
    phi = oi.von_mises_orbit(d, L, 1.0, 4)
    chi = np.random.default_rng(8).uniform(-math.pi, math.pi, V)
    phi_chi = oi.gauge_transform(phi, d, L, chi)
    g0 = np.stack([oracle.random_start(V, 1, 1, s) for s in range(40)])
    # transformed start: g_x exp(-i chi_x) gives the same phi^theta on phi^chi
    z = (g0[..., 0] + 1j * g0[..., 1]) * np.exp(-1j * chi)
    g0_chi = np.stack([z.real, z.imag], axis=-1)
    ra = oracle.relax_given(d, L, phi, g0)
    rb = oracle.relax_given(d, L, phi_chi, g0_chi)
    ta = np.arctan2(ra.g[..., 1], ra.g[..., 0])
    tb = np.arctan2(rb.g[..., 1], rb.g[..., 0])
    la = oracle.link_angles_gauged(d, L, phi, ta)
    lb = oracle.link_angles_gauged(d, L, phi_chi, tb)
    diff = np.abs(np.angle(np.exp(1j * (la - lb)))).max(axis=(1, 2))
    assert np.mean(diff < 1e-9) >= 0.9
    # plaquettes of phi^theta equal those of phi (mod 2 pi)
    def plaq(p):
        out = []
        for mu in range(d):
            for nu in range(mu + 1, d):
                xm = oi.shifted_index(d, L, mu, 1)
                xn = oi.shifted_index(d, L, nu, 1)
                out.append(p[..., mu] + p[..., xm, nu] - p[..., xn, mu] - p[..., nu])
        return np.stack(out, -1)
    dp = np.angle(np.exp(1j * (plaq(la) - plaq(phi)[None])))
    assert np.abs(dp).max() < 1e-12


# ----------------------------------------------------------------------------
# brute force 2x2 with the Morse sum (Eq. 2)
# ----------------------------------------------------------------------------

def _brute_force_2x2(phi):
    """All stationary points of Eq. 3 on a 2x2 lattice with theta_3 = 0.

    Links (a -> b, phi): the 8 links of the 2x2 torus.  Damped Newton from a
    regular grid of the three free angles.
    """
    d, L = 2, 2
    links = []
    for x in range(4):
        for mu in range(d):
            b = int(oi.shifted_index(d, L, mu, +1)[x])
            links.append((x, b, phi[x, mu]))
    n = 16
    g = (np.arange(n) + 0.5) / n * 2 * math.pi - math.pi
    T = np.array(np.meshgrid(g, g, g, indexing="ij")).reshape(3, -1).T
    T = np.concatenate([T, np.zeros((T.shape[0], 1))], axis=1)

    def grad_hess(T):
        G = np.zeros_like(T)
        H = np.zeros((T.shape[0], 4, 4))
        for a, b, p in links:
            psi = p + T[:, b] - T[:, a]
            s, c = np.sin(psi), np.cos(psi)
            G[:, b] += s; G[:, a] -= s
            H[:, a, a] += c; H[:, b, b] += c; H[:, a, b] -= c; H[:, b, a] -= c
        return G[:, :3], H[:, :3, :3]

    for _ in range(80):
        G, H = grad_hess(T)
        step = np.linalg.solve(H + 1e-14 * np.eye(3), G[..., None])[..., 0]
        nrm = np.linalg.norm(step, axis=1, keepdims=True)
        step = np.where(nrm > 0.5, step * 0.5 / np.maximum(nrm, 1e-300), step)
        T[:, :3] -= step
    G, H = grad_hess(T)
    ok = np.linalg.norm(G, axis=1) < 1e-12
    pts = []
    for t, h in zip(T[ok], H[ok]):
        t = np.angle(np.exp(1j * t))
        if any(np.max(np.abs(np.angle(np.exp(1j * (t - q[0]))))) < 1e-7 for q in pts):
            continue
        ev = np.linalg.eigvalsh(h)
        pts.append((t, int(np.sum(ev < 0)), float(np.min(np.abs(ev)))))
    return pts


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
def test_brute_force_2x2_and_morse_sum(seed):
    d, L = 2, 2
    phi = oi.uniform_orbit(d, L, seed)
    pts = _brute_force_2x2(phi)
    assert all(p[2] > 1e-6 for p in pts)            # non-degenerate
    # Eq. 2: sum of sign det M_FP over all copies = chi(T^3) = 0
    assert sum((-1) ** p[1] for p in pts) == 0
    minima = [p[0] for p in pts if p[1] == 0]
    relaxed, cp = oracle.enumerate_copies(d, L, phi, seed=5, orbit_id=seed, n_starts=3000)
    assert (relaxed.status == oracle.CONVERGED).all()
    assert len(cp.F) == len(minima)
    for t in minima:
        assert min(np.max(np.abs(np.angle(np.exp(1j * (t - th))))) for th in cp.theta) < 1e-8
    assert (cp.region == oracle.REGION_IN).all()


# ----------------------------------------------------------------------------
# dedup
# ----------------------------------------------------------------------------

def test_dedup_identity_and_representatives():
    d, L = 2, 3
    V = L ** d
    rng = np.random.default_rng(0)
    base = [rng.uniform(-math.pi, math.pi, V) for _ in range(3)]
    for b in base:
        b[-1] = 0.0
    # starts 0..8: copies of base 2, 0, 1, 0, 2, 2 (+ jitter below delta) and two beyond delta
    which = [2, 0, 1, 0, 2, 2]
    theta = [base[w] + rng.normal(0, 1e-8, V) * (np.arange(V) < V - 1) for w in which]
    far = base[0].copy(); far[0] += 3e-6
    theta += [far, far + 1e-9]
    theta = np.array(theta)
    # copies of one stationary point share F up to second order in the jitter
    Fb = [1.5, 2.5, 3.5]
    F = np.array([Fb[w] + 1e-13 * i for i, w in enumerate(which)] + [1.5, 1.5])
    starts = np.array([10, 11, 12, 13, 14, 15, 16, 17])
    rep_of, reps = oracle.dedup(d, L, theta, F, starts, np.ones(8, bool), delta=1e-6)
    assert len(reps) == 4
    assert rep_of[0] == rep_of[4] == rep_of[5]
    assert rep_of[1] == rep_of[3]
    assert rep_of[6] == rep_of[7] != rep_of[1]
    assert [starts[r] for r in reps] == [10, 11, 12, 16]


# ----------------------------------------------------------------------------
# statistics printed in the paper (plain relaxation, as the paper ran it)
# ----------------------------------------------------------------------------

def _golden():
    with open(GOLDEN) as f:
        return json.load(f)


def _orbit_stats(d, L, n_orbits, n_starts):
    fmin, nmin = [], []
    for o in range(n_orbits):
        phi = oi.uniform_orbit(d, L, 10_000 + o)
        _, cp = oracle.enumerate_copies(d, L, phi, seed=1, orbit_id=o, n_starts=n_starts,
                                        omega=1.0, eps=1e-24)
        inr = cp.region == oracle.REGION_IN
        fmin.append(oracle.f_norm(cp.F[inr].min(), d, L))
        nmin.append(int(inr.sum()))
    return np.array(fmin), np.array(nmin)


@pytest.mark.parametrize("d,N,n_orbits,n_starts", [(2, 2, 300, 256), (2, 4, 200, 1024),
                                                   (3, 2, 200, 1024), (4, 2, 200, 2048)])
def test_tables_I_and_III_statistics(d, N, n_orbits, n_starts):
    g = _golden()
    t3 = next(r for r in g["table_III"]["rows"] if r["d"] == d and r["N"] == N)
    t1 = next(r for r in g["table_I"]["rows"] if r["d"] == d and r["N"] == N)
    fmin, nmin = _orbit_stats(d, N, n_orbits, n_starts)
    # difference of two sample means: standard error sqrt(s^2/100 + s^2/M)
    se3 = t3["std"] * math.sqrt(1 / t3["orbits"] + 1 / n_orbits)
    assert abs(fmin.mean() - t3["avg_Fmin"]) < 3.5 * se3, (fmin.mean(), t3)
    se1 = t1["std"] * math.sqrt(1 / t1["orbits"] + 1 / n_orbits)
    assert abs(nmin.mean() - t1["avg_minima"]) < 3.5 * se1, (nmin.mean(), t1)


def test_n_distinct_f8_quantisation():
    """The paper's distinct-minima count: x = F/(dV) mapped to floor(x * 1e8)
    (Section III).  The cases are built so that a wrong normalisation (by V
    or by d alone), rounding instead of the floor, or a count of raw F values
    each gives a different answer."""
    d, L = 2, 4                        # dV = 32 links
    dV = d * L ** d
    # two minima in one 1e-8 bin (floor), next-bin neighbour, and a value on a
    # bin's lower edge: bins 12345678, 12345678, 12345679 and 25000000
    x = np.array([0.1234567810, 0.1234567890, 0.1234567900000004, 0.25])
    assert oracle.n_distinct_f8(x * dV, d, L) == 3
    # rounding to nearest would split the first two (12345678 / 12345679)
    assert len(np.unique(np.round(x * 1e8))) == 3 and len(np.unique(np.round(x[:2] * 1e8))) == 2
    assert oracle.n_distinct_f8(x[:2] * dV, d, L) == 1
    # normalised by V alone the pair 0.3 / 0.300000005 would fall into two bins
    y = np.array([0.3, 0.300000005]) * dV
    assert oracle.n_distinct_f8(y, d, L) == 1
    assert len(np.unique(np.floor(y / L ** d * 1e8))) == 2
    # raw F values are all distinct; the quantised count merges them
    assert oracle.n_distinct_f8(np.array([1.0, 1.0 + 1e-9, 1.0 + 2e-9]) , d, L) == 1
    # the ends of [0, 1] map to 0 and 1e8
    assert oracle.n_distinct_f8(np.array([0.0, dV * 1.0]), d, L) == 2
    assert oracle.n_distinct_f8(np.zeros(0), d, L) == 0
