// First-Gribov-region test on the Faddeev-Popov operator of each new distinct
// copy.  For compact U(1) the operator is the Hessian of Eq. 3 in the gauge
// angles: the lattice Laplacian with link weights w = cos(phi^theta),
//   (M v)_x = sum_mu [ w_{x,mu} (v_x - v_{x+mu}) + w_{x-mu,mu} (v_x - v_{x-mu}) ].
// The constant vector is an exact zero mode (the global phase); the copy is in
// the first Gribov region when the rest of the spectrum is non-negative, i.e.
// lambda_2 = min spec(M | 1^perp) >= 0 (minimal Landau gauge, Section I).
//
// Lanczos on M restricted to 1^perp (every vector is projected off the mean),
// one warp per copy, vectors in shared memory; the smallest eigenvalue of the
// Lanczos tridiagonal is located by warp-parallel Sturm multisection.
// Two kernels: fp_screen_kernel (FP32, small footprint, high occupancy) and
// fp_test_kernel (FP64).  Modes:
//   kFpAuto     -- FP32 Lanczos screen; copies with lambda_2 clearly above 0
//                  are accepted, the rest go to a second list that the FP64
//                  kernel decides by FP64 Lanczos;
//   kFpLanczos  -- FP64 Lanczos for every copy, started from the FP64
//                  Rayleigh-Ritz vector of the two lowest Ritz vectors of an
//                  FP32 Lanczos run (lanczos32_ritz, rayleigh_ritz2_64,
//                  lanczos64_seeded; fp_test_pairs_kernel on 4^4);
//   kFpDense    -- FP64 Lanczos with full reorthogonalisation run to
//                  dimension V-1 (the whole spectrum; a dense-solver grade
//                  lambda_2), basis vectors in a global scratch slot per warp;
//   kFpNone     -- skip.
#pragma once
#include "gc_common.cuh"

namespace gc {

enum { kFpAuto = 0, kFpLanczos = 1, kFpDense = 2, kFpNone = 3 };
enum { kRegionOut = 0, kRegionIn = 1, kRegionMarginal = 2 };

struct FpArgs {
  Geom geom;
  const double2* cfg;          // pool configurations
  const float2* links32;
  const unsigned long long* first_start;  // seeds each copy's Lanczos start vector
  const double2* links64;
  const unsigned int* list;    // entries to test
  const unsigned int* n_list;  // device count
  unsigned int* redo;          // screen: entries left to the FP64 test
  unsigned int* n_redo;
  double* lambda2;
  int* region;
  int mode, kmax32, kmax64, count_tests;
  int extra32;                 // Lanczos mode: FP32 steps after the FP32 Ritz values stall
  double tau, margin32, tol32, tol64;
  double* scratch;             // dense mode: one (V x V) slot per warp of the grid
  uint64_t seed;
  unsigned long long* stats;   // [13] tests, [14] FP64 decisions, [15] Lanczos steps (FP32 and FP64),
                               // [24] FP64 Lanczos steps
};

// Shared memory: the site-order neighbour table (uint4 per site, per mu the
// packed pair (x + mu) | (x - mu) << 16), then per warp the link weights
// [mu][x], the Lanczos vectors and the tridiagonal, in arithmetic R.
//   FP32 (screen): three vectors; alpha and beta^2.
//   FP64: four vector slots (three Lanczos vectors and the diagonal of M) that
//   the FP32 seed phase of the Lanczos mode uses first for its weights and
//   five vectors; a tail with alpha, beta^2 and a third array (dense mode:
//   projection coefficients), or the seed phase's eight FP32 arrays of
//   kmax32_of(kmax) + 2 entries.
__host__ __device__ inline int kmax32_of(int kmax) { return kmax < 160 ? kmax : 160; }

template <typename R>
struct FpSmem {
  size_t nbr, warp0, per_warp, total;
  __host__ __device__ static size_t align16s(size_t b) { return (b + 15) & ~size_t(15); }
  __host__ __device__ static size_t max2(size_t a, size_t b) { return a > b ? a : b; }
  // FP64 vector region: 4 slots of V doubles, or the seed phase's layout
  __host__ __device__ static size_t slot(int V) { return align16s((size_t)V * sizeof(R)); }
  __host__ __device__ static size_t seed_w32(int V, int d) { return align16s((size_t)V * d * 4); }
  __host__ __device__ static size_t seed_vec(int V) { return align16s((size_t)V * 4); }
  __host__ __device__ static size_t vec_bytes(int V, int d) {
    return sizeof(R) == 8 ? max2(4 * slot(V), seed_w32(V, d) + 5 * seed_vec(V)) : 3 * slot(V);
  }
  __host__ __device__ static size_t tri(int kmax) { return align16s((size_t)(kmax + 2) * sizeof(R)); }
  __host__ __device__ static size_t tri32(int kmax) { return align16s((size_t)(kmax32_of(kmax) + 2) * 4); }
  __host__ __device__ static size_t tail_bytes(int kmax) {
    return sizeof(R) == 8 ? max2(3 * tri(kmax), 8 * tri32(kmax)) : 3 * tri(kmax);
  }
  __host__ __device__ static size_t warp_bytes(int V, int d, int kmax) {
    return align16s((size_t)V * d * sizeof(R)) + vec_bytes(V, d) + tail_bytes(kmax);
  }
  __host__ __device__ FpSmem(int V, int d, int kmax, int warps) {
    nbr = 0;
    warp0 = align16s((size_t)V * sizeof(uint4));
    per_warp = warp_bytes(V, d, kmax);
    total = warp0 + (size_t)warps * per_warp;
  }
};

__device__ __forceinline__ float sturm_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double sturm_div(double a, double b) { return a / b; }

// number of eigenvalues of the k x k tridiagonal (alpha, beta2 = squared
// off-diagonal, beta2[i] couples rows i-1 and i) below x: the negative pivots
// of the LDL^T factorisation of T - x (Sylvester's law of inertia).  Only the
// pivots' signs matter, so FP32 takes the fast divide.
template <typename S>
__device__ inline int sturm_count(const S* alpha, const S* beta2, int k, S x) {
  const S tiny = sizeof(S) == 4 ? (S)-1e-30f : (S)-1e-300;
  int cnt = 0;
  S q = alpha[0] - x;
  if (q == (S)0) q = tiny;
  cnt += q < (S)0;
  for (int i = 1; i < k; ++i) {
    q = (alpha[i] - x) - sturm_div(beta2[i], q);
    if (q == (S)0) q = tiny;
    cnt += q < (S)0;
  }
  return cnt;
}

template <typename S>
__device__ __forceinline__ S tri_rel() { return sizeof(S) == 4 ? (S)2e-7 : (S)1e-15; }

// smallest eigenvalue of the tridiagonal, given a bracket lo <= lambda_min <= hi,
// by 32-way multisection, entirely in the arithmetic of the Lanczos vectors
// (kth > 1: the kth smallest, given lo below it and hi above it)
template <typename S>
__device__ inline S tri_min(const S* alpha, const S* beta2, int k, S lo, S hi, int lane, S rel = tri_rel<S>(),
                            int kth = 1) {
  for (int round = 0; round < 14; ++round) {
    const S scale = fabs(lo) > (S)1 ? fabs(lo) : (S)1;
    if (hi - lo <= rel * scale) break;
    const S step = (hi - lo) / (S)33;
    const S x = lo + step * (S)(lane + 1);
    const bool below = sturm_count<S>(alpha, beta2, k, x) >= kth;  // lambda_kth < x
    const unsigned m = __ballot_sync(0xffffffffu, below);
    const int first = m ? __ffs(m) - 1 : 32;                      // first point above lambda_min
    const S nlo = lo + step * (S)first;
    const S nhi = first == 32 ? hi : lo + step * (S)(first + 1);
    lo = nlo; hi = nhi;
  }
  return (S)0.5 * (lo + hi);
}

// (M v)_x with weights stored [mu][x]
template <int DD, typename R>
__device__ __forceinline__ R matvec_site(const R* w, const R* v, const uint4 nb, int x, int V) {
  const R vx = v[x];
  R acc = 0;
#pragma unroll
  for (int mu = 0; mu < DD; ++mu) {
    const unsigned wd = nb_word(nb, mu);
    const int xp = wd & 0xffffu, xm = wd >> 16;
    acc = fma(w[mu * V + x], vx - v[xp], acc);
    acc = fma(w[mu * V + xm], vx - v[xm], acc);
  }
  return acc;
}

template <typename R>
__device__ __forceinline__ R warp_sum(R v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Lanczos estimate of lambda_2 in arithmetic R: vectors, dot products and the
// tridiagonal (alpha, beta^2) all in R.  REORTH keeps every basis vector in Q
// (global scratch, FP64) and reorthogonalises against all of them.
template <typename R, bool REORTH, int DD>
__device__ R lanczos_min(const R* w, R* vprev, R* vcur, R* z, R* alpha, R* beta, double* h,
                         double* Q, int kmax, double tol, const uint4* nbr, int V, int lane,
                         uint64_t seed, unsigned long long entry, int* steps) {
  // random start vector orthogonal to the constant mode
  R s = 0;
  for (int x = lane; x < V; x += 32) {
    const U64x4 r = philox4x64_10(entry, (uint64_t)x, 0, 1, seed, 0x4C414E43ULL);
    const R v = (R)(unsigned)(r.v[0] >> 40) * (R)0x1.0p-24 - (R)0.5;
    vcur[x] = v;
    vprev[x] = 0;
    s += v;
  }
  s = warp_sum(s) / (R)V;
  R nn = 0;
  for (int x = lane; x < V; x += 32) { const R v = vcur[x] - s; vcur[x] = v; nn += v * v; }
  const R inv0 = (R)1 / sqrt(warp_sum(nn));
  for (int x = lane; x < V; x += 32) vcur[x] *= inv0;
  __syncwarp();
  const R bound = (R)(4 * DD + 1);
  R b = 0;
  R theta = bound, theta_prev = bound, theta_pp = bound;   // bound = no estimate yet
  int stalls = 0;
  int j = 0;
  for (; j < kmax; ++j) {
    if (REORTH) {
      for (int x = lane; x < V; x += 32) Q[(size_t)j * V + x] = (double)vcur[x];
    }
    R a = 0;
    for (int x = lane; x < V; x += 32) {
      const R mv = matvec_site<DD>(w, vcur, nbr[x], x, V) - b * vprev[x];
      z[x] = mv;
      a += mv * vcur[x];
    }
    a = warp_sum(a);
    R m = 0;
    for (int x = lane; x < V; x += 32) { const R v = z[x] - a * vcur[x]; z[x] = v; m += v; }
    if (REORTH) {
      __syncwarp();
      for (int pass = 0; pass < 2; ++pass) {
        for (int i = 0; i <= j; ++i) {
          double p = 0.0;
          for (int x = lane; x < V; x += 32) p += Q[(size_t)i * V + x] * (double)z[x];
          p = warp_sum(p);
          if (lane == 0) h[i] = p;
        }
        __syncwarp();
        for (int x = lane; x < V; x += 32) {
          double acc = (double)z[x];
          for (int i = 0; i <= j; ++i) acc -= h[i] * Q[(size_t)i * V + x];
          z[x] = (R)acc;
        }
        __syncwarp();
      }
      m = 0;
      for (int x = lane; x < V; x += 32) m += z[x];
    }
    // mean and norm of z in one reduction: |z - m|^2 = sum z^2 - V m^2
    R zz = 0;
    for (int x = lane; x < V; x += 32) { const R v = z[x]; zz += v * v; }
    for (int o = 16; o > 0; o >>= 1) {
      m += __shfl_xor_sync(0xffffffffu, m, o);
      zz += __shfl_xor_sync(0xffffffffu, zz, o);
    }
    m /= (R)V;
    const R bn = sqrt(fmax(zz - (R)V * m * m, (R)0));
    for (int x = lane; x < V; x += 32) z[x] -= m;
    if (lane == 0) { alpha[j] = a; beta[j + 1] = bn * bn; }
    __syncwarp();
    const bool last = (j + 1 == kmax) || bn < (R)1e-12;
    if (last || (!REORTH && (j + 1) % 8 == 0 && j + 1 >= 16)) {
      // bracket: Cauchy interlacing gives lambda_min(T_k) <= lambda_min(T_{k-8})
      // (the previous estimate, to within its bracket); below, a step of four
      // times the last decrease, checked by one Sturm count
      R lo = -bound, hi = bound;
      if (theta_prev < bound) {
        const R slack = (R)2 * tri_rel<R>() * fmax(fabs(theta_prev), (R)1);
        hi = theta_prev + slack;
        if (theta_pp < bound) {
          const R l = theta_prev - (R)4 * fmax(theta_pp - theta_prev, slack);
          if (sturm_count<R>(alpha, beta, j + 1, l) == 0) lo = l;
        }
      }
      theta = tri_min<R>(alpha, beta, j + 1, lo, hi, lane);
      if (last) { ++j; break; }
      // stop when the value holds over two checks in a row (16 steps): one
      // stall can be a plateau above lambda_2 that later steps leave
      if (fabs(theta - theta_prev) <= (R)tol * fmax(fabs(theta), (R)1e-3)) {
        if (++stalls == 2) { ++j; break; }
      } else {
        stalls = 0;
      }
      theta_pp = theta_prev;
      theta_prev = theta;
    }
    const R ib = (R)1 / bn;   // beta[] holds squares; bn is the norm itself
    for (int x = lane; x < V; x += 32) { vprev[x] = vcur[x]; vcur[x] = z[x] * ib; }
    b = bn;
    __syncwarp();
  }
  *steps += j;
  return theta;
}

// ---------------------------------------------------------------------------
// FP64 helpers of the Lanczos mode.  On this part an FP64 instruction costs
// the SM about 64 FP32 ones, so:
//   * M v = D v - sum_mu [w_{x,mu} v_{x+mu} + w_{x-mu,mu} v_{x-mu}], with the
//     diagonal D and the negated weights stored once per copy: 2d + 1 FMAs per
//     site, and the whole Lanczos step (recurrence, alpha, mean, norm, next
//     vector) in 15 FP64 operations per site;
//   * the mean and the squared norm of the new vector share one warp
//     reduction that adds each level once (warp_sum2);
//   * lambda_min of the FP64 tridiagonal by tri_min64 (division-free Sturm
//     counts, Newton steps from below), warm-started just below the previous
//     value (Cauchy interlacing bounds the new one by it); on this part an
//     FP64 instruction costs the pipe the same with one active lane as with
//     32, so each round uses all 32 lanes (32 points);
//   * the normalisation's 1/sqrt in FP64 from the FP32 unit's estimate and
//     two Newton steps (rsqrt64), and comparisons on the integer pipe.
// ---------------------------------------------------------------------------

struct SturmPoint { int cnt; double p, dp; };

__device__ __forceinline__ int dexp_of(double v) {
  return (int)(((unsigned)__double2hiint(v) >> 20) & 0x7ffu) - 1023;
}
__device__ __forceinline__ unsigned dsign(double v) { return (unsigned)__double2hiint(v) >> 31; }
__device__ __forceinline__ bool dzero(double v) {
  return ((((unsigned)__double2hiint(v)) & 0x7fffffffu) | (unsigned)__double2loint(v)) == 0u;
}

// Sturm count and Newton quotient at x for the k x k tridiagonal (alpha,
// beta2 = squared off-diagonal, beta2[i] couples rows i-1 and i), without
// divisions: the leading minors' characteristic polynomials p_0 = 1,
// p_1 = alpha_0 - x, p_{i+1} = (alpha_i - x) p_i - beta2_i p_{i-1}, and their
// derivatives.  The number of sign changes along p_0 .. p_k is the number of
// eigenvalues below x (a p_i that is exactly 0 takes the sign opposite to
// p_{i-1}, the LDL^T convention of sturm_count).  Every 16 steps the pair is
// rescaled by a power of two once it leaves [2^-400, 2^400]; signs and p/p'
// do not change.
__device__ inline SturmPoint sturm_point64(const double* alpha, const double* beta2, int k, double x) {
  double pm = 1.0, dpm = 0.0;
  double p = alpha[0] - x, dp = -1.0;
  unsigned sp = 0u;
  unsigned s = dzero(p) ? 1u : dsign(p);
  int cnt = s != sp;
  sp = s;
  for (int i = 1; i < k; ++i) {
    const double e = alpha[i] - x;
    const double b2 = beta2[i];
    const double pn = fma(e, p, -b2 * pm);
    const double dpn = fma(e, dp, fma(-b2, dpm, -p));
    pm = p; dpm = dp; p = pn; dp = dpn;
    s = dzero(p) ? (sp ^ 1u) : dsign(p);
    cnt += s != sp;
    sp = s;
    if ((i & 15) == 0) {
      const int ea = dexp_of(p), eb = dexp_of(pm);
      const int ex = ea > eb ? ea : eb;
      if (ex > 400 || ex < -400) {
        const double sc = __hiloint2double((1023 - ex) << 20, 0);
        p *= sc; pm *= sc; dp *= sc; dpm *= sc;
      }
    }
  }
  SturmPoint r;
  r.cnt = cnt; r.p = p; r.dp = dp;
  return r;
}

// lambda_min of the tridiagonal to FP64 accuracy from a bracket
// lo < lambda_min <= hi; *ok = false when the counts at the bracket's ends
// contradict it.  Each round spreads the warp's 32 points over [lo, hi] --
// evenly in the first round, geometrically towards lo (ratio 0.35) in the
// later ones -- keeps the last point below lambda_min (count 0) and takes a
// Newton step from it.  Below the smallest root of a polynomial with real
// roots, Newton's iterates increase and stay below the root, so the step
// gives the new lower end; the next point up gives the upper end.
// With near_hi there is one round only, its points crowding towards hi (at
// hi - (hi - lo) 0.35^l): the warm start of a later check, whose root lies a
// little below the previous check's value hi.  If the root is delta below hi,
// the last point under it is within 1.9 delta of it, and the Newton step from
// there is off by O(delta^2 / gap): negligible once the values stall.
__device__ inline double tri_min64(const double* alpha, const double* beta2, int k, double lo, double hi,
                                   int lane, bool* ok, bool near_hi = false) {
  *ok = true;
  for (int round = 0; round < (near_hi ? 1 : 8); ++round) {
    double x;
    if (lane == 0) x = lo;
    else if (lane == 31) x = hi;
    else if (round == 0 && near_hi) x = fma(lo - hi, f2d_bits(exp2f((float)lane * -1.51457317f)), hi);
    else if (round == 0) x = fma(hi - lo, (double)lane * (1.0 / 31.0), lo);
    else x = fma(hi - lo, f2d_bits(exp2f((float)(31 - lane) * -1.51457317f)), lo);
    const SturmPoint r = sturm_point64(alpha, beta2, k, x);
    const unsigned m = __ballot_sync(0xffffffffu, r.cnt == 0);
    if (!(m & 1u)) {            // lambda_min <= lo
      if (round == 0) *ok = false;
      return lo;                // later rounds: the Newton iterate met lambda_min to rounding
    }
    const int f = __ffs(~m);    // first point at or above lambda_min (1-based), 0: none
    if (f == 0) { *ok = false; return hi; }
    const int ls = f - 2;
    const double xl = __shfl_sync(0xffffffffu, x, ls);
    const double pl = __shfl_sync(0xffffffffu, r.p, ls);
    const double dl = __shfl_sync(0xffffffffu, r.dp, ls);
    const double xh = __shfl_sync(0xffffffffu, x, ls + 1);
    double xn = xl - pl / dl;
    if (!(xn >= xl && xn < xh)) xn = xl;
    lo = xn;
    hi = xh;
    if (round >= 1 && hi - lo <= 1e-13 * fmax(fabs(lo), 1e-3)) break;
  }
  return lo;
}

// 1/sqrt(x) for x > 0 in FP64: the special-function unit's FP32 estimate
// (relative error < 2^-22) refined by two Newton steps y <- y (3 - x y^2) / 2,
// each squaring the error (2^-44, then below FP64 rounding)
__device__ __forceinline__ double rsqrt64(double x) {
  double y = f2d_bits(rsqrt_sfu(d2f_bits(x)));
  const double hx = 0.5 * x;
  double e = fma(-hx * y, y, 0.5);
  y = fma(y, e, y);
  e = fma(-hx * y, y, 0.5);
  return fma(y, e, y);
}
// ordering of non-negative doubles by their bit patterns (integer pipe)
__device__ __forceinline__ bool dbelow(double a, double b) {
  return __double_as_longlong(a) < __double_as_longlong(b);
}

// sums of a and b over the warp: the first level exchanges the half each lane
// does not keep, so every level adds once
__device__ __forceinline__ void warp_sum2(double& a, double& b, int lane) {
  const bool up = (lane & 16) != 0;
  double keep = up ? b : a;
  const double send = up ? a : b;
  keep += __shfl_xor_sync(0xffffffffu, send, 16);
  for (int o = 8; o > 0; o >>= 1) keep += __shfl_xor_sync(0xffffffffu, keep, o);
  a = __shfl_sync(0xffffffffu, keep, 0);
  b = __shfl_sync(0xffffffffu, keep, 16);
}

// ---------------------------------------------------------------------------
// FP64 Lanczos seeded by an FP32 Ritz vector (the Lanczos mode's test).
// The FP64 pipe is the scarce unit, so the Lanczos process first runs in FP32
// (lanczos32_ritz): from the random start until its Ritz values stall, plus
// `extra` steps; the eigenvector s of the FP32 tridiagonal T_k for its
// smallest eigenvalue comes from two inverse iterations, and a second pass
// regenerates the Lanczos vectors q_j from the recorded recurrence
// coefficients and sums y = sum_j s_j q_j.  The FP64 Lanczos process then
// starts from y (lanczos64_seeded): its first Rayleigh quotient already holds
// lambda_2 to roughly the square of the FP32 Ritz vector's error, and a few
// FP64 steps take it to FP64 accuracy.  The result is the smallest Ritz value
// of the FP64 tridiagonal; only the start vector differs from a random one.
// ---------------------------------------------------------------------------

// the random start (Philox draws, projected off the constant mode,
// normalised), shared by both FP32 passes so they start from the same bits
__device__ __forceinline__ void ritz_start(float* v, float* vprev, int V, int lane, uint64_t seed,
                                           unsigned long long entry) {
  float s = 0.f;
  for (int x = lane; x < V; x += 32) {
    const U64x4 r = philox4x64_10(entry, (uint64_t)x, 0, 1, seed, 0x4C414E43ULL);
    const float v0 = (float)(unsigned)(r.v[0] >> 40) * 0x1.0p-24f - 0.5f;
    v[x] = v0;
    vprev[x] = 0.f;
    s += v0;
  }
  s = warp_sum(s) / (float)V;
  float nn = 0.f;
  for (int x = lane; x < V; x += 32) { const float t = v[x] - s; v[x] = t; nn = fmaf(t, t, nn); }
  const float inv0 = 1.f / sqrtf(warp_sum(nn));
  for (int x = lane; x < V; x += 32) v[x] *= inv0;
  __syncwarp();
}

// M q_j - b q_{j-1} at site x with explicit FMAs: both passes round alike
template <int DD>
__device__ __forceinline__ float ritz_mv(const float* w, const float* vcur, const float* vprev, const uint4 nb,
                                         int x, int V, float b) {
  return fmaf(-b, vprev[x], matvec_site<DD, float>(w, vcur, nb, x, V));
}

// the FP32 tridiagonal and the recurrence record of the first pass
struct Ritz32 {
  float* al;    // alpha_j
  float* be2;   // beta_j^2 (beta2[i] couples rows i-1 and i)
  float* mm;    // mean removed from step j's new direction
  float* bn;    // beta_j
  float* s;     // eigenvector of T_k for its smallest eigenvalue
  float* s2;    //                      for its second smallest
  float* pd;    // LDL^T pivots of T_k - sigma (reciprocals)
  float* pl;    // LDL^T multipliers
};

// x <- (T_k - sigma)^-1 x on the LDL^T factors (reciprocal pivots pd,
// multipliers pl), scaled to a largest entry of 1
__device__ __forceinline__ void ldl_solve32(const float* pd, const float* pl, int k, float* x) {
  float u = x[0];
  for (int i = 1; i < k; ++i) { u = fmaf(-pl[i], u, x[i]); x[i] = u; }
  float xn = u * pd[k - 1];
  x[k - 1] = xn;
  float big = fabsf(xn);
  for (int i = k - 2; i >= 0; --i) {
    xn = fmaf(-pl[i + 1], xn, x[i] * pd[i]);
    x[i] = xn;
    big = fmaxf(big, fabsf(xn));
  }
  const float sc = big > 0.f ? __fdividef(1.f, big) : 1.f;
  for (int i = 0; i < k; ++i) x[i] *= sc;
}

// Eigenvectors of the k x k tridiagonal (alpha, beta) for its smallest
// eigenvalue theta (s) and the next one up (s2), by inverse iteration with the
// shift sigma just below theta on the LDL^T factors of T_k - sigma (a zero
// pivot replaced by a tiny one): two iterations for s; two for s2, each
// after removing its component along s, so s2 converges to the eigenvector
// whose eigenvalue is the next closest to sigma at the rate
// (theta_2 - sigma) / (theta_3 - sigma), fastest when theta_2 is near theta.
// Both scaled to a largest entry of 1.  One lane runs it.
__device__ inline void ritz_coeffs32(const float* al, const float* bn, int k, float theta, float* pd,
                                           float* pl, float* s, float* s2) {
  const float sigma = theta - 2.f * tri_rel<float>() * fmaxf(fabsf(theta), 1.f);
  float dd = al[0] - sigma;
  if (fabsf(dd) < 1e-30f) dd = 1e-30f;
  float rd = __fdividef(1.f, dd);
  pd[0] = rd;
  for (int i = 1; i < k; ++i) {
    const float l = bn[i] * rd;
    dd = (al[i] - sigma) - l * bn[i];
    if (fabsf(dd) < 1e-30f) dd = 1e-30f;
    rd = __fdividef(1.f, dd);
    pl[i] = l;
    pd[i] = rd;
  }
  for (int i = 0; i < k; ++i) { s[i] = 1.f; s2[i] = (i & 1) ? -1.f : 1.f; }
  // s: two solves; s2: (project off s, solve) twice, then project off s
#pragma unroll 1
  for (int it = 0; it < 4; ++it) {
    float* x = it < 2 ? s : s2;
    if (it >= 2) {
      float p = 0.f, ss = 0.f;
      for (int i = 0; i < k; ++i) { p = fmaf(s[i], s2[i], p); ss = fmaf(s[i], s[i], ss); }
      p = __fdividef(p, ss);
      for (int i = 0; i < k; ++i) s2[i] = fmaf(-p, s[i], s2[i]);
    }
    ldl_solve32(pd, pl, k, x);
  }
  float p = 0.f, ss = 0.f;
  for (int i = 0; i < k; ++i) { p = fmaf(s[i], s2[i], p); ss = fmaf(s[i], s[i], ss); }
  p = __fdividef(p, ss);
  for (int i = 0; i < k; ++i) s2[i] = fmaf(-p, s[i], s2[i]);
}

// FP32 Ritz values resolve lambda only to ~ eps32 ||T|| absolute (the Sturm
// counts' backward error), so the stall test of the FP32 phase takes
// tol32 |theta| with that floor
__device__ __forceinline__ bool ritz32_stalled(float theta, float prev, double tol32) {
  return fabsf(theta - prev) <= fmaxf((float)tol32 * fabsf(theta), 2e-6f);
}

// The FP32 phase checks its smallest Ritz value at step 48 and every 16
// steps after; one stall between two checks ends it (16 extra steps later).
// Each check is a Sturm multisection over the whole tridiagonal, so checks
// are kept few: the Ritz vector that matters needs the extra steps anyway.
__device__ __forceinline__ bool ritz32_check_due(int steps) {
  return steps >= 48 && ((steps - 48) & 15) == 0;
}

// Returns the smallest FP32 Ritz value; y and y2 receive the (unnormalised)
// Ritz vectors of the smallest and second smallest Ritz values (y2 zero when
// T_k has one row).  w: weights [mu][x] (positive); q, qp, z: work vectors.
template <int DD>
__device__ float lanczos32_ritz(const float* w, float* q, float* qp, float* z, float* y, float* y2,
                                const Ritz32 R, int kmax, double tol32, int extra, const uint4* nbr, int V,
                                int lane, uint64_t seed, unsigned long long entry, int* steps) {
  ritz_start(q, qp, V, lane, seed, entry);
  const float bound = (float)(4 * DD + 1);
  float b = 0.f, theta = bound, theta_prev = bound, theta_pp = bound;
  int kend = kmax, j = 0;
  bool settled = false;
  for (; j < kend; ++j) {
    float a = 0.f;
    for (int x = lane; x < V; x += 32) {
      const float mv = ritz_mv<DD>(w, q, qp, nbr[x], x, V, b);
      z[x] = mv;
      a = fmaf(mv, q[x], a);
    }
    a = warp_sum(a);
    float m = 0.f, zz = 0.f;
    for (int x = lane; x < V; x += 32) {
      const float v = fmaf(-a, q[x], z[x]);
      z[x] = v;
      m += v;
      zz = fmaf(v, v, zz);
    }
    for (int o = 16; o > 0; o >>= 1) {
      m += __shfl_xor_sync(0xffffffffu, m, o);
      zz += __shfl_xor_sync(0xffffffffu, zz, o);
    }
    m /= (float)V;
    const float bn = sqrtf(fmaxf(zz - (float)V * m * m, 0.f));
    if (lane == 0) { R.al[j] = a; R.be2[j + 1] = bn * bn; R.mm[j] = m; R.bn[j + 1] = bn; }
    __syncwarp();
    const bool last = (j + 1 == kend) || bn < 1e-12f;
    if (last || (!settled && ritz32_check_due(j + 1))) {
      float lo = -bound, hi = bound;
      if (theta_prev < bound) {
        const float slack = 2.f * tri_rel<float>() * fmaxf(fabsf(theta_prev), 1.f);
        hi = theta_prev + slack;
        if (theta_pp < bound) {
          const float l = theta_prev - 4.f * fmaxf(theta_pp - theta_prev, slack);
          if (sturm_count<float>(R.al, R.be2, j + 1, l) == 0) lo = l;
        }
      }
      // the stall test needs 1e-6; the final value (the inverse iteration's
      // shift) the full FP32 resolution
      theta = tri_min<float>(R.al, R.be2, j + 1, lo, hi, lane, last ? tri_rel<float>() : 1e-6f);
      if (last) { ++j; break; }
      // one stall over 16 steps, then `extra` steps more
      if (ritz32_stalled(theta, theta_prev, tol32)) {
        settled = true;
        kend = j + 1 + extra < kmax ? j + 1 + extra : kmax;
      }
      theta_pp = theta_prev;
      theta_prev = theta;
    }
    const float ib = 1.f / bn;
    for (int x = lane; x < V; x += 32) { qp[x] = q[x]; q[x] = (z[x] - m) * ib; }
    b = bn;
    __syncwarp();
  }
  const int k = j;
  *steps += k;
  if (lane == 0) ritz_coeffs32(R.al, R.bn, k, theta, R.pd, R.pl, R.s, R.s2);
  __syncwarp();
  // second pass: the same vectors again, summed with the Ritz coefficients
  ritz_start(q, qp, V, lane, seed, entry);
  const float s0 = R.s[0], t0 = R.s2[0];
  for (int x = lane; x < V; x += 32) { y[x] = s0 * q[x]; y2[x] = t0 * q[x]; }
  b = 0.f;
  for (int i = 0; i + 1 < k; ++i) {
    const float a = R.al[i], m = R.mm[i], bn = R.bn[i + 1];
    const float ib = 1.f / bn;
    for (int x = lane; x < V; x += 32) z[x] = (fmaf(-a, q[x], ritz_mv<DD>(w, q, qp, nbr[x], x, V, b)) - m) * ib;
    __syncwarp();
    const float si = R.s[i + 1], ti = R.s2[i + 1];
    for (int x = lane; x < V; x += 32) {
      qp[x] = q[x];
      q[x] = z[x];
      y[x] = fmaf(si, z[x], y[x]);
      y2[x] = fmaf(ti, z[x], y2[x]);
    }
    b = bn;
    __syncwarp();
  }
  return theta;
}

// The smallest eigenpair of the symmetric 2 x 2 matrix [[a, b], [b, c]]:
// (cs, sn) with the eigenvector cs e1 + sn e2, by the Jacobi rotation that
// diagonalises it.
__device__ inline void rr2_rotation(double a, double b, double c, double* cs, double* sn) {
  if (b == 0.0) {
    *cs = a <= c ? 1.0 : 0.0;
    *sn = a <= c ? 0.0 : 1.0;
    return;
  }
  const double zeta = (c - a) / (2.0 * b);
  const double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(fma(zeta, zeta, 1.0)));
  const double co = 1.0 / sqrt(fma(t, t, 1.0)), si = t * co;
  // eigenvalues a - t b (vector (co, -si)) and c + t b (vector (si, co))
  if (a - t * b <= c + t * b) { *cs = co; *sn = -si; } else { *cs = si; *sn = co; }
}

// out = M v (weights negated [mu][x], diagonal Dg), all in shared memory
template <int DD>
__device__ __forceinline__ void mv64(const double* nw, const double* Dg, const double* v, double* out,
                                     const uint4* nbr, int V, int lane) {
  for (int x = lane; x < V; x += 32) {
    const uint4 nb = nbr[x];
    double yv = Dg[x] * v[x];
#pragma unroll
    for (int mu = 0; mu < DD; ++mu) {
      const unsigned wd = nb_word(nb, mu);
      const int xp = wd & 0xffffu, xm = wd >> 16;
      yv = fma(nw[mu * V + x], v[xp], yv);
      yv = fma(nw[mu * V + xm], v[xm], yv);
    }
    out[x] = yv;
  }
  __syncwarp();
}

// FP64 Rayleigh-Ritz on span{e1, e2}: e1 in va (normalised, off the constant
// mode), y2 in vb (off the constant mode); vc is scratch.  Leaves in va the
// unit vector of the span with the smallest Rayleigh quotient.  Near-equal
// lambda_2 and lambda_3 leave a component of the lambda_3 eigenvector in the
// FP32 Ritz vector that Lanczos steps remove slowly; the second Ritz vector
// removes most of it at once.
template <int DD>
__device__ void rayleigh_ritz2_64(const double* nw, const double* Dg, double* va, double* vb, double* vc,
                                  const uint4* nbr, int V, int lane) {
  double p = 0.0, q2 = 0.0;
  for (int x = lane; x < V; x += 32) { p = fma(va[x], vb[x], p); q2 = fma(vb[x], vb[x], q2); }
  warp_sum2(p, q2, lane);
  const double r2 = fma(-p, p, q2);   // |vb - (va . vb) va|^2
  if (!(r2 > 1e-12 * q2)) return;     // vb (nearly) along va: no second direction
  const double ir = rsqrt64(r2);
  for (int x = lane; x < V; x += 32) vb[x] = fma(-p, va[x], vb[x]) * ir;
  __syncwarp();
  mv64<DD>(nw, Dg, va, vc, nbr, V, lane);
  double a11 = 0.0, a12 = 0.0;
  for (int x = lane; x < V; x += 32) { a11 = fma(va[x], vc[x], a11); a12 = fma(vb[x], vc[x], a12); }
  warp_sum2(a11, a12, lane);
  mv64<DD>(nw, Dg, vb, vc, nbr, V, lane);
  double a22 = 0.0;
  for (int x = lane; x < V; x += 32) a22 = fma(vb[x], vc[x], a22);
  a22 = warp_sum(a22);
  double cs, sn;
  rr2_rotation(a11, a12, a22, &cs, &sn);
  for (int x = lane; x < V; x += 32) va[x] = fma(cs, va[x], sn * vb[x]);
  __syncwarp();
}

// FP64 Lanczos from the start vector in va (normalised, orthogonal to the
// constant mode).  Each step takes 15 FP64 ops per site; lambda_min of the FP64
// tridiagonal is taken after every step (T_1 is the seed's Rayleigh quotient;
// later ones by tri_min64 warm-started just below the previous value, whose
// window the last decrease sets), and the run stops when two successive
// values agree to tol64 twice in a row.  theta32 (the FP32 Ritz value) seeds
// the bracket when the warm start misses.
template <int DD>
__device__ double lanczos64_seeded(const double* nw, const double* Dg, double* va, double* vb, double* vc,
                                   double* a64, double* b64, int kmax, double tol64, float theta32,
                                   const uint4* nbr, int V, int lane, int* steps) {
  double* vcur = va;
  double* vprev = vb;
  double* z = vc;
  for (int x = lane; x < V; x += 32) vprev[x] = 0.0;
  __syncwarp();
  const double invV = 1.0 / (double)V;
  const double bound = (double)(4 * DD + 1);
  double t64 = bound, d64 = 0.0, b = 0.0;
  int stalls = 0, j = 0;
  for (; j < kmax; ++j) {
    double a = 0.0;
    const double mb = -b;
    for (int x = lane; x < V; x += 32) {
      const uint4 nb = nbr[x];
      const double vx = vcur[x];
      double yv = fma(Dg[x], vx, mb * vprev[x]);
#pragma unroll
      for (int mu = 0; mu < DD; ++mu) {
        const unsigned wd = nb_word(nb, mu);
        const int xp = wd & 0xffffu, xm = wd >> 16;
        yv = fma(nw[mu * V + x], vcur[xp], yv);
        yv = fma(nw[mu * V + xm], vcur[xm], yv);
      }
      z[x] = yv;
      a = fma(yv, vx, a);
    }
    a = warp_sum(a);
    double m = 0.0, zz = 0.0;
    for (int x = lane; x < V; x += 32) {
      const double v = fma(-a, vcur[x], z[x]);
      z[x] = v;
      m += v;
      zz = fma(v, v, zz);
    }
    warp_sum2(m, zz, lane);
    m *= invV;
    double bn2 = fma(-(double)V * m, m, zz);   // |z - m|^2
    if (__double_as_longlong(bn2) < 0) bn2 = 0.0;
    if (lane == 0) { a64[j] = a; b64[j + 1] = bn2; }
    __syncwarp();
    const bool last = (j + 1 == kmax) || dbelow(bn2, 1e-24);
    double t;
    if (j == 0) {
      t = a;
    } else {
      // brackets tried in turn (one call site, so the multisection is
      // compiled once): the warm window below the last value, a window around
      // the FP32 Ritz value, then the Gershgorin interval
      bool ok = false, near = true;
      double lo = t64 - fmax(8.0 * d64, 4e-5 * fmax(fabs(t64), 1e-3));
      double hi = t64 + 1e-14 * fmax(fabs(t64), 1.0);
#pragma unroll 1
      for (int attempt = 0;; ++attempt) {
        t = tri_min64(a64, b64, j + 1, lo, hi, lane, &ok, near);
        if (ok || attempt == 2) break;
        near = false;
        if (attempt == 0) {
          const double c = f2d_bits(theta32);
          const double del = 2e-5 * fmax(1.0, fabs(c));
          lo = fmin(c, t64) - del;
          hi = t64 + del;
        } else {
          lo = -bound;
          hi = bound;
        }
      }
    }
    const bool stall = j > 0 && fabs(t - t64) <= tol64 * fmax(fabs(t), 1e-3);
    d64 = j > 0 ? fmax(t64 - t, 0.0) : 0.0;
    t64 = t;
    if (last) { ++j; break; }
    if (stall) {
      if (++stalls == 2) { ++j; break; }
    } else {
      stalls = 0;
    }
    const double ib = rsqrt64(bn2);
    const double mib = -m * ib;
    for (int x = lane; x < V; x += 32) z[x] = fma(z[x], ib, mib);
    b = bn2 * ib;
    double* tt = vprev;
    vprev = vcur;
    vcur = z;
    z = tt;
    __syncwarp();
  }
  *steps += j;
  return t64;
}

__device__ inline void build_site_neighbours(const Geom& G, uint4* nbr) {
  for (int x = threadIdx.x; x < G.V; x += blockDim.x) {
    unsigned w[4] = {0u, 0u, 0u, 0u};
    for (int mu = 0; mu < G.d; ++mu)
      w[mu] = (unsigned)neighbor(x, mu, +1, G.L) | ((unsigned)neighbor(x, mu, -1, G.L) << 16);
    nbr[x] = make_uint4(w[0], w[1], w[2], w[3]);
  }
  __syncthreads();
}

__device__ __forceinline__ int region_of(double lam, double tau) {
  return lam > tau ? kRegionIn : (lam < -tau ? kRegionOut : kRegionMarginal);
}

// FP32 screen (auto mode): a copy whose FP32 lambda_2 is above margin32 is in
// the first region; every other copy goes to the redo list for FP64.
template <int DD>
__global__ void __launch_bounds__(256) fp_screen_kernel(const FpArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Geom G = a.geom;
  const int V = G.V;
  const int warps = blockDim.x >> 5;
  const int kmax = a.kmax32;
  const unsigned n = *a.n_list;
  if ((unsigned long long)blockIdx.x * warps >= n) return;   // no copy for this CTA (uniform)
  const FpSmem<float> lay(V, DD, kmax, warps);
  uint4* nbr = reinterpret_cast<uint4*>(smem + lay.nbr);
  build_site_neighbours(G, nbr);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned char* base = smem + lay.warp0 + (size_t)warp * lay.per_warp;
  float* w32 = reinterpret_cast<float*>(base);
  const size_t vstride = FpSmem<float>::align16s((size_t)V * 4);
  unsigned char* vb = base + FpSmem<float>::align16s((size_t)V * DD * 4);
  float* alpha = reinterpret_cast<float*>(vb + 3 * vstride);
  float* beta = alpha + FpSmem<float>::align16s((size_t)(kmax + 2) * 4) / 4;

  const long long gwarp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  unsigned long long c_tests = 0;
  int steps = 0;
  for (long long li = gwarp; li < (long long)n; li += nwarps) {
    const unsigned e = a.list[li];
    const double2* g = a.cfg + (size_t)e * V;
    // the start vector depends on the copy (its lowest start index), not on
    // where the copy sits in the pool, so results do not depend on insertion order
    const unsigned long long key = __ldcg(a.first_start + e);
    float2* g32 = reinterpret_cast<float2*>(vb);   // scratch until the Lanczos vectors start
    for (int x = lane; x < V; x += 32) {
      const double2 gx = __ldcg(g + x);
      g32[x] = make_float2(d2f_bits(gx.x), d2f_bits(gx.y));
    }
    __syncwarp();
    for (int x = lane; x < V; x += 32) {
      const float2 gx = g32[x];
      const uint4 nb = nbr[x];
#pragma unroll
      for (int mu = 0; mu < DD; ++mu) {
        const float2 hx = g32[nb_word(nb, mu) & 0xffffu];
        const float2 uu = a.links32[x * DD + mu];
        const float tx = fmaf(uu.x, hx.x, -uu.y * hx.y), ty = fmaf(uu.x, hx.y, uu.y * hx.x);
        w32[mu * V + x] = fmaf(gx.x, tx, gx.y * ty);   // cos(phi^theta_{x,mu})
      }
    }
    __syncwarp();
    const int k = V - 1 < kmax ? V - 1 : kmax;
    const float lam = lanczos_min<float, false, DD>(
        w32, reinterpret_cast<float*>(vb), reinterpret_cast<float*>(vb + vstride),
        reinterpret_cast<float*>(vb + 2 * vstride), alpha, beta, nullptr, nullptr, k, a.tol32, nbr,
        V, lane, a.seed, key, &steps);
    if (lane == 0) {
      if (lam > (float)a.margin32) {
        a.lambda2[e] = (double)lam;
        a.region[e] = region_of((double)lam, a.tau);
      } else {
        a.redo[atomicAdd(a.n_redo, 1u)] = e;
      }
    }
    ++c_tests;
    __syncwarp();
  }
  if (lane == 0 && c_tests) {
    atomicAdd(&a.stats[13], c_tests);
    atomicAdd(&a.stats[15], (unsigned long long)steps);
  }
}

// FP64 test: Lanczos (kFpLanczos) or full reorthogonalisation to dimension
// V - 1 (kFpDense); kFpNone marks every copy untested.
template <int DD>
__global__ void __launch_bounds__(128, 4) fp_test_kernel(const FpArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Geom G = a.geom;
  const int V = G.V;
  const int warps = blockDim.x >> 5;
  const int kmax = a.kmax64;
  const unsigned n = *a.n_list;
  if ((unsigned long long)blockIdx.x * warps >= n) return;   // no copy for this CTA (uniform)
  const FpSmem<double> lay(V, DD, kmax, warps);
  uint4* nbr = reinterpret_cast<uint4*>(smem + lay.nbr);
  build_site_neighbours(G, nbr);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned char* base = smem + lay.warp0 + (size_t)warp * lay.per_warp;
  double* w64 = reinterpret_cast<double*>(base);
  unsigned char* vb = base + FpSmem<double>::align16s((size_t)V * DD * 8);
  const size_t vstride = FpSmem<double>::slot(V);
  unsigned char* tail = vb + FpSmem<double>::vec_bytes(V, DD);
  double* alpha = reinterpret_cast<double*>(tail);
  double* beta = alpha + FpSmem<double>::tri(kmax) / 8;
  double* h = beta + FpSmem<double>::tri(kmax) / 8;

  const long long gwarp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  double* Q = a.mode == kFpDense ? a.scratch + (size_t)gwarp * V * V : nullptr;
  unsigned long long c_tests = 0, c64 = 0;
  int steps = 0, steps64 = 0;
  for (long long li = gwarp; li < (long long)n; li += nwarps) {
    const unsigned e = a.list[li];
    const double2* g = a.cfg + (size_t)e * V;
    const unsigned long long key = __ldcg(a.first_start + e);
    double lam;
    if (a.mode == kFpNone) {
      lam = __longlong_as_double(0x7ff8000000000000LL);
    } else {
      const bool dense = a.mode == kFpDense;
      const double sgn = dense ? 1.0 : -1.0;   // Lanczos mode keeps the weights negated
      for (int x = lane; x < V; x += 32) {
        const double2 gx = __ldcg(g + x);
        const uint4 nb = nbr[x];
#pragma unroll
        for (int mu = 0; mu < DD; ++mu) {
          const double2 hx = __ldcg(g + (nb_word(nb, mu) & 0xffffu));
          const double2 uu = a.links64[x * DD + mu];
          const double tx = fma(uu.x, hx.x, -uu.y * hx.y), ty = fma(uu.x, hx.y, uu.y * hx.x);
          w64[mu * V + x] = sgn * fma(gx.x, tx, gx.y * ty);
        }
      }
      __syncwarp();
      const int k = V - 1 < kmax ? V - 1 : kmax;
      double* v0 = reinterpret_cast<double*>(vb);
      double* v1 = reinterpret_cast<double*>(vb + vstride);
      double* v2 = reinterpret_cast<double*>(vb + 2 * vstride);
      double* v3 = reinterpret_cast<double*>(vb + 3 * vstride);
      if (dense) {
        int sd = 0;
        lam = lanczos_min<double, true, DD>(w64, v0, v1, v2, alpha, beta, h, Q, k, 0.0, nbr, V, lane,
                                            a.seed, key, &sd);
        steps += sd;
        steps64 += sd;
      } else {
        // FP32 seed: the weights' FP32 image (positive) and five FP32 vectors
        // in the vector region, the FP32 tridiagonal in the tail
        float* w32 = reinterpret_cast<float*>(vb);
        float* q32 = reinterpret_cast<float*>(vb + FpSmem<double>::seed_w32(V, DD));
        float* qp32 = q32 + FpSmem<double>::seed_vec(V) / 4;
        float* z32 = qp32 + FpSmem<double>::seed_vec(V) / 4;
        float* y32 = z32 + FpSmem<double>::seed_vec(V) / 4;
        float* y2_32 = y32 + FpSmem<double>::seed_vec(V) / 4;
        for (int i = lane; i < V * DD; i += 32) w32[i] = -d2f_near(w64[i]);
        __syncwarp();
        const size_t t32 = FpSmem<double>::tri32(kmax) / 4;
        float* f = reinterpret_cast<float*>(tail);
        const Ritz32 R{f, f + t32, f + 2 * t32, f + 3 * t32, f + 4 * t32, f + 5 * t32, f + 6 * t32, f + 7 * t32};
        const int k32 = kmax32_of(k);
        const float th32 = lanczos32_ritz<DD>(w32, q32, qp32, z32, y32, y2_32, R, k32, a.tol32, a.extra32, nbr,
                                              V, lane, a.seed, key, &steps);
        // the two Ritz vectors in FP64 (into slots 0 and 1, which they do not
        // overlap), off the constant mode; the first normalised
        double sm = 0.0, sm2 = 0.0;
        for (int x = lane; x < V; x += 32) {
          const double t = f2d_bits(y32[x]), t2 = f2d_bits(y2_32[x]);
          v0[x] = t; v1[x] = t2;
          sm += t; sm2 += t2;
        }
        warp_sum2(sm, sm2, lane);
        sm /= (double)V;
        sm2 /= (double)V;
        double nn = 0.0;
        for (int x = lane; x < V; x += 32) {
          const double t = v0[x] - sm;
          v0[x] = t;
          v1[x] -= sm2;
          nn = fma(t, t, nn);
        }
        const double inv = rsqrt64(warp_sum(nn));
        for (int x = lane; x < V; x += 32) v0[x] *= inv;
        __syncwarp();
        // the diagonal of M: D_x = sum_mu (w_{x,mu} + w_{x-mu,mu})
        for (int x = lane; x < V; x += 32) {
          const uint4 nb = nbr[x];
          double dsum = 0.0;
#pragma unroll
          for (int mu = 0; mu < DD; ++mu) dsum -= w64[mu * V + x] + w64[mu * V + (nb_word(nb, mu) >> 16)];
          v3[x] = dsum;
        }
        __syncwarp();
        rayleigh_ritz2_64<DD>(w64, v3, v0, v1, v2, nbr, V, lane);
        int s64 = 0;
        lam = lanczos64_seeded<DD>(w64, v3, v0, v1, v2, alpha, beta, k, a.tol64, th32, nbr, V, lane, &s64);
        steps += s64;
        steps64 += s64;
      }
      ++c64;
    }
    if (lane == 0) {
      a.lambda2[e] = lam;
      a.region[e] = a.mode == kFpNone ? -1 : region_of(lam, a.tau);
    }
    ++c_tests;
    __syncwarp();
  }
  if (lane == 0 && c_tests) {
    if (a.count_tests) atomicAdd(&a.stats[13], c_tests);
    atomicAdd(&a.stats[14], c64);
    atomicAdd(&a.stats[15], (unsigned long long)steps);
    atomicAdd(&a.stats[24], (unsigned long long)steps64);
  }
}

}  // namespace gc
