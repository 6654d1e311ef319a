"""Oracle for the Gribov-copy enumeration -- TEST INFRASTRUCTURE ONLY.

Plain FP64 CPU restatement of the method of Mehta & Schroeck (arXiv:1403.0555)
for compact U(1) lattice Landau gauge.  Only ``tests/``, ``__graft_entry__.smoke``
and ``bench.py``'s CPU-baseline leg may import this package; the library path
never does.  It shares no code with the CUDA path (the seeded input generators
live in ``orbit_inputs``, which holds none of the method's arithmetic).

Pieces and the passages they follow:
  * relaxation sweeps, residual, random starts: C core ``gribov_oracle.c``
    (Section III, Eqs. 4-5; Philox generator named in Section III);
  * canonical copy: the global gauge freedom is removed by setting the angle of
    the last site (N,...,N) to zero (Section II, U(1) paragraph);
  * functional: Eq. 3, evaluated from angles with cos();
  * Faddeev-Popov operator: Hessian of Eq. 3 in the gauge angles (Section I,
    "Landau gauge on the lattice"); for U(1) a lattice Laplacian with link
    weights cos(phi^theta); first Gribov region = its spectrum on the complement
    of the constant mode is non-negative (Section I, minimal Landau gauge);
  * paper-style distinct count: minima normalised to [0,1], mapped to integers
    in [0, 1e8] and counted distinct (Section III, quantisation paragraph).

Readings where the paper is silent are listed in the repository's design
notes; the two that shape this file: F_norm = F/(d V) and configuration
identity max_x |wrap(theta'_A - theta'_B)| <= delta for deduplication.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass

import numpy as np

from . import build as _build

_LIB = None

CONVERGED = 1
NOT_CONVERGED = 2

REGION_OUT = 0       # lambda_2 < -tau: a saddle, outside the first Gribov region
REGION_IN = 1        # lambda_2 > tau
REGION_MARGINAL = 2  # |lambda_2| <= tau


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        p_u64 = ctypes.POINTER(ctypes.c_uint64)
        p_d = ctypes.POINTER(ctypes.c_double)
        p_i8 = ctypes.POINTER(ctypes.c_int8)
        p_i32 = ctypes.POINTER(ctypes.c_int32)
        L.or_philox4x64_10.argtypes = [p_u64, p_u64, p_u64]
        L.or_random_start.argtypes = [ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64,
                                      ctypes.c_uint64, p_d]
        L.or_divergence.argtypes = [ctypes.c_int, ctypes.c_int, p_d, p_d, p_d]
        L.or_sweeps.argtypes = [ctypes.c_int, ctypes.c_int, p_d, ctypes.c_double,
                                ctypes.c_int, p_d]
        L.or_colors.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
        L.or_relax_given.argtypes = [ctypes.c_int, ctypes.c_int, p_d, ctypes.c_int64,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_int, p_d, p_i8, p_i32, p_d]
        L.or_enumerate.argtypes = [ctypes.c_int, ctypes.c_int, p_d, ctypes.c_uint64,
                                   ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64,
                                   ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                   ctypes.c_int, ctypes.c_int, p_d, p_i8, p_i32, p_d]
        L.or_enumerate_indices.argtypes = [ctypes.c_int, ctypes.c_int, p_d, ctypes.c_uint64,
                                           ctypes.c_uint64, p_u64, ctypes.c_int64,
                                           ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                           ctypes.c_int, ctypes.c_int, p_d, p_i8, p_i32, p_d]
        L.or_max_threads.restype = ctypes.c_int
        _LIB = L
    return _LIB


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _phi(phi, d, L):
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    assert phi.shape == (L ** d, d), phi.shape
    return phi


def max_threads() -> int:
    return int(lib().or_max_threads())


# ----------------------------------------------------------------------------
# random starts (Section III: Philox)
# ----------------------------------------------------------------------------

def philox4x64_10(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().or_philox4x64_10(_ptr(c, ctypes.c_uint64), _ptr(k, ctypes.c_uint64),
                           _ptr(out, ctypes.c_uint64))
    return out


def random_start(V: int, seed: int, orbit_id: int, start: int) -> np.ndarray:
    """(V, 2) unit complex numbers (cos theta_x, sin theta_x) of one start."""
    g = np.zeros((V, 2))
    lib().or_random_start(V, seed, orbit_id, start, _ptr(g, ctypes.c_double))
    return g


# ----------------------------------------------------------------------------
# relaxation (Section III)
# ----------------------------------------------------------------------------

def colors(d: int, L: int):
    out = np.zeros(L ** d, dtype=np.int32)
    nc = lib().or_colors(d, L, _ptr(out, ctypes.c_int))
    return out, nc


def divergence(d, L, phi, g) -> np.ndarray:
    """Im[conj(g_x) S_x] per site (minus the gradient of Eq. 3)."""
    phi = _phi(phi, d, L)
    g = np.ascontiguousarray(g, dtype=np.float64)
    out = np.zeros(L ** d)
    lib().or_divergence(d, L, _ptr(phi, ctypes.c_double), _ptr(g, ctypes.c_double),
                        _ptr(out, ctypes.c_double))
    return out


def sweeps(d, L, phi, omega, n, g) -> np.ndarray:
    phi = _phi(phi, d, L)
    g = np.array(g, dtype=np.float64, copy=True, order="C")
    lib().or_sweeps(d, L, _ptr(phi, ctypes.c_double), omega, n, _ptr(g, ctypes.c_double))
    return g


@dataclass
class Relaxed:
    g: np.ndarray        # (n, V, 2) final states
    status: np.ndarray   # (n,) CONVERGED / NOT_CONVERGED
    sweeps: np.ndarray   # (n,) sweeps performed
    resid: np.ndarray    # (n,) last residual


def relax_given(d, L, phi, g0, omega=1.7, eps=1e-24, check_every=1, max_sweeps=100_000,
                nthreads=0) -> Relaxed:
    phi = _phi(phi, d, L)
    g = np.array(g0, dtype=np.float64, copy=True, order="C").reshape(-1, L ** d, 2)
    n = g.shape[0]
    st = np.zeros(n, np.int8)
    sw = np.zeros(n, np.int32)
    rs = np.zeros(n)
    lib().or_relax_given(d, L, _ptr(phi, ctypes.c_double), n, omega, eps, check_every,
                         max_sweeps, nthreads, _ptr(g, ctypes.c_double),
                         _ptr(st, ctypes.c_int8), _ptr(sw, ctypes.c_int32),
                         _ptr(rs, ctypes.c_double))
    return Relaxed(g, st, sw, rs)


def relax_starts(d, L, phi, seed, orbit_id, start0, n, omega=1.7, eps=1e-24, check_every=1,
                 max_sweeps=100_000, nthreads=0) -> Relaxed:
    phi = _phi(phi, d, L)
    V = L ** d
    g = np.zeros((n, V, 2))
    st = np.zeros(n, np.int8)
    sw = np.zeros(n, np.int32)
    rs = np.zeros(n)
    lib().or_enumerate(d, L, _ptr(phi, ctypes.c_double), seed, orbit_id, start0, n, omega,
                       eps, check_every, max_sweeps, nthreads, _ptr(g, ctypes.c_double),
                       _ptr(st, ctypes.c_int8), _ptr(sw, ctypes.c_int32),
                       _ptr(rs, ctypes.c_double))
    return Relaxed(g, st, sw, rs)


def relax_indices(d, L, phi, seed, orbit_id, starts, omega=1.7, eps=1e-24, check_every=1,
                  max_sweeps=100_000, nthreads=0) -> Relaxed:
    phi = _phi(phi, d, L)
    idx = np.ascontiguousarray(starts, dtype=np.uint64)
    n = idx.shape[0]
    V = L ** d
    g = np.zeros((n, V, 2))
    st = np.zeros(n, np.int8)
    sw = np.zeros(n, np.int32)
    rs = np.zeros(n)
    lib().or_enumerate_indices(d, L, _ptr(phi, ctypes.c_double), seed, orbit_id,
                               _ptr(idx, ctypes.c_uint64), n, omega, eps, check_every,
                               max_sweeps, nthreads, _ptr(g, ctypes.c_double),
                               _ptr(st, ctypes.c_int8), _ptr(sw, ctypes.c_int32),
                               _ptr(rs, ctypes.c_double))
    return Relaxed(g, st, sw, rs)


# ----------------------------------------------------------------------------
# canonical copy, functional (Eq. 3)
# ----------------------------------------------------------------------------

def canonical(g: np.ndarray):
    """Fix the global gauge: theta' = theta - theta_{V-1} (site (N,...,N) set to 0).

    g: (..., V, 2).  Returns (g' as complex (..., V), theta' (..., V)).
    """
    z = g[..., 0] + 1j * g[..., 1]
    zp = z * np.conj(z[..., -1:])
    return zp, np.angle(zp)


def _shift(d, L, mu, step):
    V = L ** d
    idx = np.arange(V)
    coord = (idx // (L ** mu)) % L
    return idx + (((coord + step) % L) - coord) * (L ** mu)


def link_angles_gauged(d, L, phi, theta) -> np.ndarray:
    """phi^theta_{x,mu} = phi_{x,mu} + theta_{x+mu} - theta_x, shape (..., V, d)."""
    theta = np.asarray(theta)
    cols = [phi[:, mu] + theta[..., _shift(d, L, mu, +1)] - theta for mu in range(d)]
    return np.stack(cols, axis=-1)


def functional(d, L, phi, theta) -> np.ndarray:
    """Eq. 3: F = sum_{x,mu} (1 - cos(phi^theta_{x,mu}))."""
    return np.sum(1.0 - np.cos(link_angles_gauged(d, L, phi, theta)), axis=(-1, -2))


def f_norm(F, d, L):
    """The paper's minimum value x in [0, 1]: F divided by the number of links."""
    return np.asarray(F) / (d * L ** d)


def n_distinct_f8(F, d, L) -> int:
    """The paper's count of distinct minima (Section III, quantisation
    paragraph): each minimum x = F/(dV) in [0, 1] is mapped to the integer
    floor(x * 1e8) in [0, 1e8] (floor: the paper does not name the rounding),
    and the distinct integers are counted."""
    q = np.floor(f_norm(F, d, L) * 1e8).astype(np.int64)
    return int(np.unique(q).size)


# ----------------------------------------------------------------------------
# Faddeev-Popov operator: Hessian of Eq. 3 in the gauge angles
# ----------------------------------------------------------------------------

def fp_weights(d, L, phi, theta) -> np.ndarray:
    """w_{x,mu} = cos(phi^theta_{x,mu}), the second derivative of each term of Eq. 3."""
    return np.cos(link_angles_gauged(d, L, phi, theta))


def fp_operator(d, L, w) -> np.ndarray:
    """Dense M = sum_links w_l (e_a - e_b)(e_a - e_b)^T for link l from a=x to b=x+mu."""
    V = L ** d
    M = np.zeros((V, V))
    x = np.arange(V)
    for mu in range(d):
        y = _shift(d, L, mu, +1)
        for a, b, wl in zip(x, y, w[:, mu]):
            M[a, a] += wl
            M[b, b] += wl
            M[a, b] -= wl
            M[b, a] -= wl
    return M


def lambda2(d, L, w) -> float:
    """Smallest eigenvalue of M on the complement of the constant mode.

    The constant vector is an exact zero mode; adding (alpha/V) 1 1^T with
    alpha = 4d + 1 > lambda_max(M) (Gershgorin, |w| <= 1) moves it above the
    rest of the spectrum, so the smallest eigenvalue of the sum is lambda_2.
    """
    V = L ** d
    M = fp_operator(d, L, w)
    alpha = 4.0 * d + 1.0
    return float(np.linalg.eigvalsh(M + (alpha / V) * np.ones((V, V)))[0])


def region_flag(lam2: float, tau: float) -> int:
    if lam2 > tau:
        return REGION_IN
    if lam2 < -tau:
        return REGION_OUT
    return REGION_MARGINAL


# ----------------------------------------------------------------------------
# deduplication and the full pipeline
# ----------------------------------------------------------------------------

def same_copy(theta_a, theta_b, delta) -> bool:
    return float(np.max(np.abs(np.angle(np.exp(1j * (theta_a - theta_b)))))) <= delta


@dataclass
class Copies:
    F: np.ndarray            # (m,) functional of each distinct copy
    theta: np.ndarray        # (m, V) canonical angles, theta'_{V-1} = 0
    first_start: np.ndarray  # (m,) lowest start index reaching the copy
    count: np.ndarray        # (m,) number of starts reaching it
    lambda2: np.ndarray      # (m,)
    region: np.ndarray       # (m,)
    copy_of_start: np.ndarray  # (n,) index into the sorted copy list, -1 if not converged
    n_distinct_F8: int         # paper-style count of distinct quantised minima


def dedup(d, L, theta, F, start_ids, converged, delta=1e-6):
    """Group converged starts into distinct copies (configuration identity).

    Two canonical copies are the same iff max_x |wrap(theta'_A - theta'_B)| <= delta.
    Copies of one stationary point differ in F by at most 2 d V delta^2 (F is
    stationary there and its Hessian is bounded by 4d), so candidates are
    looked up among copies with |F - F_c| <= tolF only.
    Returns (rep_index_per_start, list of representative start positions).
    """
    V = L ** d
    tolF = 2.0 * d * V * delta * delta + 1e-9
    buckets: dict[int, list[int]] = {}
    reps: list[int] = []          # position (into the arrays) of each copy's representative
    rep_of = np.full(len(F), -1, dtype=np.int64)
    order = np.argsort(start_ids, kind="stable")
    for i in order:
        if not converged[i]:
            continue
        k = int(math.floor(F[i] / tolF))
        hit = -1
        for kk in (k - 1, k, k + 1):
            for c in buckets.get(kk, ()):
                if abs(F[reps[c]] - F[i]) <= tolF and same_copy(theta[reps[c]], theta[i], delta):
                    hit = c
                    break
            if hit >= 0:
                break
        if hit < 0:
            hit = len(reps)
            reps.append(i)
            buckets.setdefault(k, []).append(hit)
        rep_of[i] = hit
    return rep_of, reps


def lambda2_of_copy(args) -> float:
    """lambda_2 of one canonical copy, args = (d, L, phi, theta)."""
    d, L, phi, theta = args
    return lambda2(d, L, fp_weights(d, L, phi, theta))


def enumerate_copies(d, L, phi, seed, orbit_id, n_starts, omega=1.7, eps=1e-24,
                     check_every=1, max_sweeps=100_000, delta=1e-6, tau=1e-9,
                     start0=0, nthreads=0, relaxed: Relaxed | None = None, lam_map=map):
    """Whole pipeline on random starts start0 .. start0+n_starts-1.

    Returns (Relaxed, Copies) with copies sorted by (F, first_start).
    lam_map maps lambda2_of_copy over the distinct copies (e.g. a process
    pool's map for large tables; the values do not depend on it).
    """
    phi = _phi(phi, d, L)
    if relaxed is None:
        relaxed = relax_starts(d, L, phi, seed, orbit_id, start0, n_starts, omega, eps,
                               check_every, max_sweeps, nthreads)
    _, theta = canonical(relaxed.g)
    F = functional(d, L, phi, theta)
    conv = relaxed.status == CONVERGED
    starts = np.arange(start0, start0 + n_starts, dtype=np.int64)
    rep_of, reps = dedup(d, L, theta, F, starts, conv, delta)
    m = len(reps)
    cF = np.array([F[r] for r in reps]) if m else np.zeros(0)
    cth = np.array([theta[r] for r in reps]) if m else np.zeros((0, L ** d))
    cfirst = np.array([starts[r] for r in reps], dtype=np.int64)
    ccount = np.bincount(rep_of[rep_of >= 0], minlength=m).astype(np.int64)
    lam = np.array(list(lam_map(lambda2_of_copy, [(d, L, phi, t) for t in cth]))) if m else np.zeros(0)
    reg = np.array([region_flag(v, tau) for v in lam], dtype=np.int32)
    order = np.lexsort((cfirst, cF)) if m else np.zeros(0, np.int64)
    inv = np.empty(m, np.int64)
    inv[order] = np.arange(m)
    copy_of = np.full(len(rep_of), -1, np.int64)
    copy_of[rep_of >= 0] = inv[rep_of[rep_of >= 0]]
    if m == 0:
        lam = np.zeros(0)
        reg = np.zeros(0, np.int32)
    copies = Copies(cF[order], cth[order], cfirst[order], ccount[order], lam[order],
                    reg[order], copy_of, n_distinct_f8(F[conv], d, L))
    return relaxed, copies
