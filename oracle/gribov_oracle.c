/*
 * Oracle for the Gribov-copy enumeration -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow FP64 CPU restatement of the relaxation method of
 * "Enumerating Copies in the First Gribov Region on the Lattice in up to four
 * Dimensions" (Mehta & Schroeck, arXiv:1403.0555), for compact U(1):
 *
 *   functional      F(theta) = sum_{x,mu} (1 - cos(phi_{x,mu} + theta_{x+mu} - theta_x))   (Eq. 3)
 *   local update    maximise Re[g_x K_x] at one site, i.e. theta_x = arg S_x   (Eq. 4, Eq. 5)
 *   checkerboard    all sites of one colour updated independently            (Section III)
 *   starts          uniform random gauge angles from the Philox generator    (Section III)
 *   stopping        largest squared lattice divergence below eps             (Section III)
 *
 * Only tests/, the package's smoke check and bench.py's CPU baseline may load
 * this file's library.  It shares no code with the CUDA path.
 *
 * Conventions: V = L^d sites, idx(x) = sum_mu x_mu L^mu (x_0 fastest), link
 * (x,mu) at index idx(x)*d + mu; complex numbers are stored as (re, im) pairs.
 * g_x = exp(i theta_x), u_{x,mu} = exp(i phi_{x,mu}).  With these,
 *   S_x = sum_mu [ u_{x,mu} g_{x+mu} + conj(u_{x-mu,mu}) g_{x-mu} ]
 * and the terms of Eq. 3 that involve theta_x sum to Re[conj(g_x) S_x], so the
 * local optimum of Eq. 4 is g_x = S_x/|S_x| (Section III).  The lattice
 * divergence (minus the gradient of Eq. 3 in theta_x) is Im[conj(g_x) S_x].
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -fPIC -shared (no FMA contraction,
 * so every product and sum below is one IEEE-rounded operation).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw: "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11).  Multipliers and Weyl key increments are the   */
/* published 4x64 constants.                                                  */
/* ------------------------------------------------------------------------ */
static const uint64_t PHILOX_M0 = 0xD2E7470EE14C6C93ULL;
static const uint64_t PHILOX_M1 = 0xCA5A826395121157ULL;
static const uint64_t PHILOX_W0 = 0x9E3779B97F4A7C15ULL;
static const uint64_t PHILOX_W1 = 0xBB67AE8584CAA73BULL;

static void mul128(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo) {
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void or_philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4]) {
    uint64_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint64_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += PHILOX_W0; k1 += PHILOX_W1; }
        uint64_t hi0, lo0, hi1, lo1;
        mul128(PHILOX_M0, c0, &hi0, &lo0);
        mul128(PHILOX_M1, c2, &hi1, &lo1);
        uint64_t n0 = hi1 ^ c1 ^ k0;
        uint64_t n1 = lo1;
        uint64_t n2 = hi0 ^ c3 ^ k1;
        uint64_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* A uniform point on the unit circle for site `site` of start `start`.
 * Counter (start, site, attempt, 0), key (seed, orbit_id).  Each Philox block
 * gives two candidate points in [-1,1)^2 (53-bit uniforms); the first with
 * 0 < x^2+y^2 <= 1 is accepted and scaled onto the circle, which makes its
 * angle uniform on the circle without any trigonometric call. */
void or_start_site(uint64_t seed, uint64_t orbit_id, uint64_t start, uint64_t site, double *gxy) {
    const uint64_t key[2] = {seed, orbit_id};
    for (uint64_t attempt = 0;; ++attempt) {
        const uint64_t ctr[4] = {start, site, attempt, 0};
        uint64_t w[4];
        or_philox4x64_10(ctr, key, w);
        for (int k = 0; k < 2; ++k) {
            double x = 2.0 * ((double)(w[2 * k] >> 11) * 0x1.0p-53) - 1.0;
            double y = 2.0 * ((double)(w[2 * k + 1] >> 11) * 0x1.0p-53) - 1.0;
            double n2 = x * x + y * y;
            if (n2 > 0.0 && n2 <= 1.0) {
                double r = 1.0 / sqrt(n2);
                gxy[0] = x * r;
                gxy[1] = y * r;
                return;
            }
        }
    }
}

void or_random_start(int V, uint64_t seed, uint64_t orbit_id, uint64_t start, double *g) {
    for (int x = 0; x < V; ++x) or_start_site(seed, orbit_id, start, (uint64_t)x, g + 2 * x);
}

/* ------------------------------------------------------------------------ */
/* lattice geometry                                                           */
/* ------------------------------------------------------------------------ */
typedef struct {
    int d, L, V, ncolor;
    int *fwd;   /* fwd[x*d+mu] = idx(x + e_mu) */
    int *bwd;   /* bwd[x*d+mu] = idx(x - e_mu) */
    int *color; /* checkerboard colour of each site */
} lattice;

/* Colouring: L even -> parity of sum_mu x_mu (two colours, Section III).
 * L odd (not in the paper) -> sum_mu c(x_mu) mod 3 with c(j) = j mod 2 for
 * j < L-1 and c(L-1) = 2, a proper 3-colouring of the odd periodic lattice. */
static int lat_init(lattice *lat, int d, int L) {
    lat->d = d; lat->L = L;
    int V = 1;
    for (int mu = 0; mu < d; ++mu) V *= L;
    lat->V = V;
    lat->ncolor = (L % 2 == 0) ? 2 : 3;
    lat->fwd = (int *)malloc(sizeof(int) * (size_t)V * d);
    lat->bwd = (int *)malloc(sizeof(int) * (size_t)V * d);
    lat->color = (int *)malloc(sizeof(int) * (size_t)V);
    if (!lat->fwd || !lat->bwd || !lat->color) return -1;
    for (int x = 0; x < V; ++x) {
        int rem = x, stride = 1, csum = 0;
        for (int mu = 0; mu < d; ++mu) {
            int xm = rem % L;
            rem /= L;
            int up = (xm + 1) % L, dn = (xm + L - 1) % L;
            lat->fwd[x * d + mu] = x + (up - xm) * stride;
            lat->bwd[x * d + mu] = x + (dn - xm) * stride;
            stride *= L;
            if (L % 2 == 0) csum += xm;
            else csum += (xm == L - 1) ? 2 : (xm % 2);
        }
        lat->color[x] = csum % lat->ncolor;
    }
    return 0;
}

static void lat_free(lattice *lat) {
    free(lat->fwd); free(lat->bwd); free(lat->color);
}

/* u_{x,mu} = (cos phi, sin phi) from libm */
static double *links_from_angles(const lattice *lat, const double *phi) {
    size_t n = (size_t)lat->V * lat->d;
    double *u = (double *)malloc(sizeof(double) * 2 * n);
    if (!u) return NULL;
    for (size_t l = 0; l < n; ++l) { u[2 * l] = cos(phi[l]); u[2 * l + 1] = sin(phi[l]); }
    return u;
}

/* S_x = sum_mu [ u_{x,mu} g_{x+mu} + conj(u_{x-mu,mu}) g_{x-mu} ], accumulated
 * in the order mu = 0..d-1, forward term before backward term. */
static void staple_sum(const lattice *lat, const double *u, const double *g, int x,
                       double *Sx_out, double *Sy_out) {
    const int d = lat->d;
    double Sx = 0.0, Sy = 0.0;
    for (int mu = 0; mu < d; ++mu) {
        int xp = lat->fwd[x * d + mu];
        int xm = lat->bwd[x * d + mu];
        double ax = u[2 * (x * d + mu)], ay = u[2 * (x * d + mu) + 1];
        double gx = g[2 * xp], gy = g[2 * xp + 1];
        double tx = ax * gx - ay * gy;           /* u * g */
        double ty = ax * gy + ay * gx;
        Sx = Sx + tx;
        Sy = Sy + ty;
        double bx = u[2 * (xm * d + mu)], by = u[2 * (xm * d + mu) + 1];
        double hx = g[2 * xm], hy = g[2 * xm + 1];
        tx = bx * hx + by * hy;                  /* conj(u) * g */
        ty = bx * hy - by * hx;
        Sx = Sx + tx;
        Sy = Sy + ty;
    }
    *Sx_out = Sx;
    *Sy_out = Sy;
}

/* One checkerboard sweep with overrelaxation parameter omega:
 *   g_hat = S_x/|S_x|,  g_x <- normalise((1-omega) g_x + omega g_hat).
 * omega = 1 is the paper's plain relaxation (theta_x = arg S_x).  A site with
 * S_x = 0 is left unchanged. */
static void sweep(const lattice *lat, const double *u, double omega, double *g) {
    const double om1 = 1.0 - omega;
    for (int c = 0; c < lat->ncolor; ++c) {
        for (int x = 0; x < lat->V; ++x) {
            if (lat->color[x] != c) continue;
            double Sx, Sy;
            staple_sum(lat, u, g, x, &Sx, &Sy);
            double n2 = Sx * Sx + Sy * Sy;
            if (!(n2 > 0.0)) continue;
            double r = 1.0 / sqrt(n2);
            double hx = Sx * r, hy = Sy * r;
            double vx = om1 * g[2 * x] + omega * hx;
            double vy = om1 * g[2 * x + 1] + omega * hy;
            double m2 = vx * vx + vy * vy;
            if (m2 > 0.0) {
                double q = 1.0 / sqrt(m2);
                g[2 * x] = vx * q;
                g[2 * x + 1] = vy * q;
            } else {
                g[2 * x] = hx;
                g[2 * x + 1] = hy;
            }
        }
    }
}

/* Landau residual: max_x (Im[conj(g_x) S_x])^2 on the current state. */
static double residual(const lattice *lat, const double *u, const double *g) {
    double r = 0.0;
    for (int x = 0; x < lat->V; ++x) {
        double Sx, Sy;
        staple_sum(lat, u, g, x, &Sx, &Sy);
        double dv = g[2 * x] * Sy - g[2 * x + 1] * Sx;
        double d2 = dv * dv;
        if (d2 > r) r = d2;
    }
    return r;
}

enum { OR_CONVERGED = 1, OR_NOT_CONVERGED = 2 };

/* Relax one start in place.  A residual check follows every check_every-th
 * sweep; the start stops at the first check with residual < eps. */
static int relax(const lattice *lat, const double *u, double omega, double eps,
                 int check_every, int max_sweeps, double *g, int *sweeps_out, double *resid_out) {
    int s = 0;
    double r = INFINITY;
    while (s < max_sweeps) {
        sweep(lat, u, omega, g);
        ++s;
        if (s % check_every == 0) {
            r = residual(lat, u, g);
            if (r < eps) { *sweeps_out = s; *resid_out = r; return OR_CONVERGED; }
        }
    }
    *sweeps_out = s;
    *resid_out = residual(lat, u, g);
    return OR_NOT_CONVERGED;
}

/* ------------------------------------------------------------------------ */
/* exported entry points                                                      */
/* ------------------------------------------------------------------------ */

/* Per-site lattice divergence Im[conj(g_x) S_x] for a given state. */
int or_divergence(int d, int L, const double *phi, const double *g, double *div_out) {
    lattice lat;
    if (lat_init(&lat, d, L)) return -1;
    double *u = links_from_angles(&lat, phi);
    if (!u) { lat_free(&lat); return -1; }
    for (int x = 0; x < lat.V; ++x) {
        double Sx, Sy;
        staple_sum(&lat, u, g, x, &Sx, &Sy);
        div_out[x] = g[2 * x] * Sy - g[2 * x + 1] * Sx;
    }
    free(u); lat_free(&lat);
    return 0;
}

/* Apply n_sweeps sweeps to g (no convergence test). */
int or_sweeps(int d, int L, const double *phi, double omega, int n_sweeps, double *g) {
    lattice lat;
    if (lat_init(&lat, d, L)) return -1;
    double *u = links_from_angles(&lat, phi);
    if (!u) { lat_free(&lat); return -1; }
    for (int s = 0; s < n_sweeps; ++s) sweep(&lat, u, omega, g);
    free(u); lat_free(&lat);
    return 0;
}

/* Checkerboard colour of every site. */
int or_colors(int d, int L, int *color_out) {
    lattice lat;
    if (lat_init(&lat, d, L)) return -1;
    memcpy(color_out, lat.color, sizeof(int) * (size_t)lat.V);
    int nc = lat.ncolor;
    lat_free(&lat);
    return nc;
}

/* Relax `n` given starts (g: n x 2V, in place). */
int or_relax_given(int d, int L, const double *phi, int64_t n, double omega, double eps,
                   int check_every, int max_sweeps, int nthreads, double *g,
                   int8_t *status, int32_t *sweeps, double *resid) {
    lattice lat;
    if (lat_init(&lat, d, L)) return -1;
    double *u = links_from_angles(&lat, phi);
    if (!u) { lat_free(&lat); return -1; }
    const int V = lat.V;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t i = 0; i < n; ++i) {
        int sw; double r;
        status[i] = (int8_t)relax(&lat, u, omega, eps, check_every, max_sweeps,
                                  g + (size_t)i * 2 * V, &sw, &r);
        sweeps[i] = sw;
        resid[i] = r;
    }
    free(u); lat_free(&lat);
    return 0;
}

/* Random starts start0 .. start0+n-1 of an orbit, relaxed (g_out: n x 2V). */
int or_enumerate(int d, int L, const double *phi, uint64_t seed, uint64_t orbit_id,
                 uint64_t start0, int64_t n, double omega, double eps, int check_every,
                 int max_sweeps, int nthreads, double *g_out, int8_t *status,
                 int32_t *sweeps, double *resid) {
    lattice lat;
    if (lat_init(&lat, d, L)) return -1;
    double *u = links_from_angles(&lat, phi);
    if (!u) { lat_free(&lat); return -1; }
    const int V = lat.V;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16)
#endif
    for (int64_t i = 0; i < n; ++i) {
        double *g = g_out + (size_t)i * 2 * V;
        or_random_start(V, seed, orbit_id, start0 + (uint64_t)i, g);
        int sw; double r;
        status[i] = (int8_t)relax(&lat, u, omega, eps, check_every, max_sweeps, g, &sw, &r);
        sweeps[i] = sw;
        resid[i] = r;
    }
    free(u); lat_free(&lat);
    return 0;
}

/* Same as or_enumerate for an explicit list of start indices. */
int or_enumerate_indices(int d, int L, const double *phi, uint64_t seed, uint64_t orbit_id,
                         const uint64_t *starts, int64_t n, double omega, double eps,
                         int check_every, int max_sweeps, int nthreads, double *g_out,
                         int8_t *status, int32_t *sweeps, double *resid) {
    lattice lat;
    if (lat_init(&lat, d, L)) return -1;
    double *u = links_from_angles(&lat, phi);
    if (!u) { lat_free(&lat); return -1; }
    const int V = lat.V;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
#endif
    for (int64_t i = 0; i < n; ++i) {
        double *g = g_out + (size_t)i * 2 * V;
        or_random_start(V, seed, orbit_id, starts[i], g);
        int sw; double r;
        status[i] = (int8_t)relax(&lat, u, omega, eps, check_every, max_sweeps, g, &sw, &r);
        sweeps[i] = sw;
        resid[i] = r;
    }
    free(u); lat_free(&lat);
    return 0;
}

int or_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
