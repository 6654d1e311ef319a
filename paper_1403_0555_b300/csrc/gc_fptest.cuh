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
//   kFpLanczos  -- FP64 Lanczos for every copy;
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
  double tau, margin32, tol32, tol64;
  double* scratch;             // dense mode: one (V x V) slot per warp of the grid
  uint64_t seed;
  unsigned long long* stats;   // [13] tests, [14] FP64 decisions, [15] Lanczos steps
};

// Shared memory: the site-order neighbour table (uint4 per site, per mu the
// packed pair (x + mu) | (x - mu) << 16), then per warp the link weights
// [mu][x], three Lanczos vectors and the tridiagonal (alpha, beta^2 and, for
// full reorthogonalisation, the projection coefficients), in arithmetic R.
template <typename R>
struct FpSmem {
  size_t nbr, warp0, per_warp, total;
  __host__ __device__ static size_t align16s(size_t b) { return (b + 15) & ~size_t(15); }
  __host__ __device__ static size_t warp_bytes(int V, int d, int kmax) {
    return align16s((size_t)V * d * sizeof(R)) + 3 * align16s((size_t)V * sizeof(R)) +
           3 * align16s((size_t)(kmax + 2) * sizeof(R));
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
template <typename S>
__device__ inline S tri_min(const S* alpha, const S* beta2, int k, S lo, S hi, int lane) {
  const S rel = tri_rel<S>();
  for (int round = 0; round < 14; ++round) {
    const S scale = fabs(lo) > (S)1 ? fabs(lo) : (S)1;
    if (hi - lo <= rel * scale) break;
    const S step = (hi - lo) / (S)33;
    const S x = lo + step * (S)(lane + 1);
    const bool below = sturm_count<S>(alpha, beta2, k, x) >= 1;  // lambda_min < x
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
      if (fabs(theta - theta_prev) <= (R)tol * fmax(fabs(theta), (R)1e-3)) { ++j; break; }
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
__global__ void __launch_bounds__(128) fp_test_kernel(const FpArgs a) {
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
  const size_t vstride = FpSmem<double>::align16s((size_t)V * 8);
  double* alpha = reinterpret_cast<double*>(vb + 3 * vstride);
  double* beta = alpha + FpSmem<double>::align16s((size_t)(kmax + 2) * 8) / 8;
  double* h = beta + FpSmem<double>::align16s((size_t)(kmax + 2) * 8) / 8;

  const long long gwarp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  double* Q = a.mode == kFpDense ? a.scratch + (size_t)gwarp * V * V : nullptr;
  unsigned long long c_tests = 0, c64 = 0;
  int steps = 0;
  for (long long li = gwarp; li < (long long)n; li += nwarps) {
    const unsigned e = a.list[li];
    const double2* g = a.cfg + (size_t)e * V;
    const unsigned long long key = __ldcg(a.first_start + e);
    double lam;
    if (a.mode == kFpNone) {
      lam = __longlong_as_double(0x7ff8000000000000LL);
    } else {
      for (int x = lane; x < V; x += 32) {
        const double2 gx = __ldcg(g + x);
        const uint4 nb = nbr[x];
#pragma unroll
        for (int mu = 0; mu < DD; ++mu) {
          const double2 hx = __ldcg(g + (nb_word(nb, mu) & 0xffffu));
          const double2 uu = a.links64[x * DD + mu];
          const double tx = fma(uu.x, hx.x, -uu.y * hx.y), ty = fma(uu.x, hx.y, uu.y * hx.x);
          w64[mu * V + x] = fma(gx.x, tx, gx.y * ty);
        }
      }
      __syncwarp();
      const int k = V - 1 < kmax ? V - 1 : kmax;
      double* v0 = reinterpret_cast<double*>(vb);
      double* v1 = reinterpret_cast<double*>(vb + vstride);
      double* v2 = reinterpret_cast<double*>(vb + 2 * vstride);
      lam = a.mode == kFpDense
                ? lanczos_min<double, true, DD>(w64, v0, v1, v2, alpha, beta, h, Q, k, 0.0, nbr, V,
                                                lane, a.seed, key, &steps)
                : lanczos_min<double, false, DD>(w64, v0, v1, v2, alpha, beta, h, nullptr, k,
                                                 a.tol64, nbr, V, lane, a.seed, key, &steps);
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
  }
}

}  // namespace gc
