"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds no arithmetic of the enumeration method (no sweep, residual,
functional, dedup or Faddeev-Popov test).  It only builds link-angle arrays for
gauge orbits and request streams, from numpy's seeded generators.

Lattice conventions (used everywhere in this repository):
  * Lambda = Z_L^d with periodic boundaries, V = L**d sites;
  * site index idx(x) = sum_mu x_mu * L**mu  (x_0 runs fastest);
  * link (x, mu) stored at ``phi[idx(x), mu]`` -- an array of shape (V, d);
  * angles are wrapped to [-pi, pi).

Orbits are random at strong coupling (beta = 0): link angles drawn independently
of any action (Section II, "Lattice Landau gauge for compact U(1)" paragraph).
The von Mises variants give finite-coupling-like structure for the
multi-orbit workloads; the trivial (cold) orbit is phi = 0, optionally hidden
by a random gauge transformation.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

TWO_PI = 2.0 * math.pi


def wrap(a):
    """Wrap angles to [-pi, pi)."""
    return np.mod(np.asarray(a, dtype=np.float64) + math.pi, TWO_PI) - math.pi


def volume(d: int, L: int) -> int:
    return int(L) ** int(d)


def site_coords(d: int, L: int) -> np.ndarray:
    """(V, d) integer coordinates of every site, x_0 fastest."""
    V = volume(d, L)
    idx = np.arange(V)
    return np.stack([(idx // (L ** mu)) % L for mu in range(d)], axis=1)


def shifted_index(d: int, L: int, mu: int, step: int) -> np.ndarray:
    """idx(x + step*e_mu) for every site x (periodic)."""
    c = site_coords(d, L).copy()
    c[:, mu] = (c[:, mu] + step) % L
    return (c * (L ** np.arange(d))).sum(axis=1)


# ----------------------------------------------------------------------------
# orbit generators
# ----------------------------------------------------------------------------

def uniform_orbit(d: int, L: int, seed: int) -> np.ndarray:
    """Hot orbit: link angles i.i.d. uniform on [-pi, pi)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-math.pi, math.pi, (volume(d, L), d))


def von_mises_orbit(d: int, L: int, kappa: float, seed: int) -> np.ndarray:
    """Link angles i.i.d. von Mises(0, kappa), wrapped to [-pi, pi)."""
    rng = np.random.default_rng(seed)
    return wrap(rng.vonmises(0.0, kappa, (volume(d, L), d)))


def constant_orbit(d: int, L: int, alpha) -> np.ndarray:
    """phi_{x,mu} = alpha_mu on every site (alpha = 0 is the cold orbit)."""
    alpha = np.broadcast_to(np.asarray(alpha, dtype=np.float64), (d,))
    return np.tile(wrap(alpha), (volume(d, L), 1))


def gauge_transform(phi: np.ndarray, d: int, L: int, chi: np.ndarray) -> np.ndarray:
    """phi^chi_{x,mu} = wrap(phi_{x,mu} + chi_{x+mu} - chi_x) (Eq. 3 convention).

    Used only to build inputs (a cold orbit hidden by a random gauge, or a
    transformed copy of an orbit for covariance checks).
    """
    out = np.empty_like(phi)
    for mu in range(d):
        out[:, mu] = phi[:, mu] + chi[shifted_index(d, L, mu, +1)] - chi
    return wrap(out)


def trivial_gauge_orbit(d: int, L: int, seed: int) -> np.ndarray:
    """Cold orbit phi = 0 after a random gauge transformation chi ~ U[-pi, pi)."""
    chi = np.random.default_rng(seed).uniform(-math.pi, math.pi, volume(d, L))
    return gauge_transform(np.zeros((volume(d, L), d)), d, L, chi)


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------

@dataclass
class Orbit:
    name: str
    d: int
    L: int
    phi: np.ndarray
    orbit_id: int


@dataclass
class Workload:
    name: str
    orbits: list
    n_starts: int
    omega: float = 1.7
    eps: float = 1e-24
    extra: dict = field(default_factory=dict)


def workload_2d_4x4() -> Workload:
    """2D 4x4, one uniform orbit from seed 1, 10^4 starts (parity workload)."""
    return Workload("2d_L4_uniform", [Orbit("u1", 2, 4, uniform_orbit(2, 4, 1), 1)], 10_000)


def workload_3d_6cubed() -> Workload:
    """3D 6^3: 4 von Mises(kappa=1) orbits (seeds 1-4) + gauge-hidden cold orbit."""
    orbits = [Orbit(f"vm{s}", 3, 6, von_mises_orbit(3, 6, 1.0, s), s) for s in (1, 2, 3, 4)]
    orbits.append(Orbit("cold", 3, 6, trivial_gauge_orbit(3, 6, 5), 5))
    return Workload("3d_L6_vonmises+cold", orbits, 100_000)


def kappa_grid_4d():
    return [0.5 + 1.5 * j / 7.0 for j in range(8)]


def workload_4d_4to4(n_starts: int = 1 << 20) -> Workload:
    """4D 4^4: 8 von Mises orbits with kappa_j = 0.5 + 1.5 j/7, seeds 1-8."""
    orbits = [Orbit(f"vm_k{k:.3f}", 4, 4, von_mises_orbit(4, 4, k, j + 1), j + 1)
              for j, k in enumerate(kappa_grid_4d())]
    return Workload("4d_L4_vonmises_x8", orbits, n_starts,
                    extra={"eps32": 1e-10})


UNEVEN_SIZES = {2: (4, 6, 8, 12, 16), 3: (4, 5, 6, 8), 4: (3, 4, 5, 6)}


def uneven_starts(d: int, L: int, site_updates: float = 1e9, sweeps: float = 100.0) -> int:
    """Starts per orbit so that a size's two orbits do about `site_updates`
    site updates at `sweeps` sweeps per start (a multiple of 256)."""
    n = site_updates / (2.0 * volume(d, L) * sweeps)
    return max(256, int(round(n / 256.0)) * 256)


def workload_uneven(scale: float = 1.0, mean_sweeps: dict | None = None) -> Workload:
    """Uneven batch: every (d, L) of UNEVEN_SIZES, two von Mises(1.0) orbits each,
    start counts in extra["n_starts"] (times `scale`): about 1e9 site updates
    per size, from `mean_sweeps[(d, L)]` (sweeps per start measured on a
    pilot) where given, else at 100 sweeps per start."""
    orbits, n = [], []
    for d, Ls in UNEVEN_SIZES.items():
        for L in Ls:
            sw = (mean_sweeps or {}).get((d, L), 100.0)
            for s in (1, 2):
                orbits.append(Orbit(f"d{d}L{L}s{s}", d, L, von_mises_orbit(d, L, 1.0, s),
                                    1000 * d + 10 * L + s))
                n.append(max(256, int(uneven_starts(d, L, sweeps=sw) * scale) // 256 * 256))
    return Workload("uneven_batch", orbits, 0, extra={"n_starts": n})


@dataclass
class Request:
    rid: int
    arrival_s: float
    d: int
    L: int
    seed: int
    n_starts: int
    phi: np.ndarray


def request_stream(n_requests: int, rate_hz: float = 200.0, seed: int = 7,
                   n_min: int = 1_000, n_max: int = 1_000_000):
    """Poisson arrivals of enumeration requests of mixed dimension and size.

    dim uniform in {2,3,4}; L uniform from the uneven-batch lists; orbit von
    Mises(1.0) with a per-request seed; n_starts log-uniform in [n_min, n_max].
    """
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for rid in range(n_requests):
        t += rng.exponential(1.0 / rate_hz)
        d = int(rng.choice([2, 3, 4]))
        L = int(rng.choice(UNEVEN_SIZES[d]))
        oseed = int(rng.integers(1, 2**31 - 1))
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        out.append(Request(rid, t, d, L, oseed, n, von_mises_orbit(d, L, 1.0, oseed)))
    return out
