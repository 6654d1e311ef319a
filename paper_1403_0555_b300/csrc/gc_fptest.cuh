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
// Modes:
//   kFpAuto     -- FP32 Lanczos screen; copies with lambda_2 clearly above 0
//                  are accepted, the rest are decided by FP64 Lanczos;
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
  double* lambda2;
  int* region;
  int mode, kmax32, kmax64;
  double tau, margin32, tol32, tol64;
  double* scratch;             // dense mode: one (V x V) slot per warp of the grid
  uint64_t seed;
  unsigned long long* stats;   // [13] tests, [14] FP64 decisions, [15] Lanczos steps
};

struct FpSmem {
  size_t nbr, warp0, per_warp, total;
  // per warp: w64[V d], w32[V d], three FP64 vectors (aliased as FP32), alpha, beta, h
  __host__ __device__ static size_t warp_bytes(int V, int d, int kmax) {
    return align16s((size_t)V * d * 8) + align16s((size_t)V * d * 4) + 3 * align16s((size_t)V * 8) +
           3 * align16s((size_t)(kmax + 2) * 8);
  }
  __host__ __device__ static size_t align16s(size_t b) { return (b + 15) & ~size_t(15); }
  __host__ __device__ FpSmem(int V, int d, int kmax, int warps) {
    nbr = 0;
    warp0 = align16s((size_t)V * 2 * d * sizeof(uint16_t));
    per_warp = warp_bytes(V, d, kmax);
    total = warp0 + (size_t)warps * per_warp;
  }
};

__device__ __forceinline__ double warp_sum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// number of eigenvalues of the k x k tridiagonal (alpha, beta[1..k-1]) below x
template <typename S>
__device__ inline int sturm_count(const S* alpha, const S* beta, int k, S x) {
  const S tiny = sizeof(S) == 4 ? (S)-1e-30f : (S)-1e-300;
  int cnt = 0;
  S q = alpha[0] - x;
  if (q == (S)0) q = tiny;
  cnt += q < (S)0;
  for (int i = 1; i < k; ++i) {
    const S bb = beta[i];
    q = (alpha[i] - x) - bb * bb / q;
    if (q == (S)0) q = tiny;
    cnt += q < (S)0;
  }
  return cnt;
}

// smallest eigenvalue of the tridiagonal, by 32-way multisection on [lo, hi],
// entirely in the arithmetic of the Lanczos vectors
template <typename S>
__device__ inline S tri_min(const S* alpha, const S* beta, int k, S lo, S hi, int lane) {
  const S rel = sizeof(S) == 4 ? (S)2e-7 : (S)1e-15;
  for (int round = 0; round < 14; ++round) {
    const S step = (hi - lo) / (S)33;
    const S x = lo + step * (S)(lane + 1);
    const bool below = sturm_count<S>(alpha, beta, k, x) >= 1;  // lambda_min < x
    const unsigned m = __ballot_sync(0xffffffffu, below);
    const int first = m ? __ffs(m) - 1 : 32;                    // first point above lambda_min
    const S nlo = lo + step * (S)first;
    const S nhi = first == 32 ? hi : lo + step * (S)(first + 1);
    lo = nlo; hi = nhi;
    const S scale = fabs(lo) > (S)1 ? fabs(lo) : (S)1;
    if (hi - lo <= rel * scale) break;
  }
  return (S)0.5 * (lo + hi);
}

// (M v)_x with weights stored [mu][x]
template <typename R>
__device__ __forceinline__ R matvec_site(const R* w, const R* v, const uint16_t* nb, int x, int d, int V) {
  const R vx = v[x];
  R acc = 0;
  for (int mu = 0; mu < d; ++mu) {
    const int xp = nb[2 * mu], xm = nb[2 * mu + 1];
    acc += w[mu * V + x] * (vx - v[xp]) + w[mu * V + xm] * (vx - v[xm]);
  }
  return acc;
}

template <typename R>
__device__ __forceinline__ R warp_sum(R v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Lanczos estimate of lambda_2 in arithmetic R (vector work and dot products
// stay in R; only the tridiagonal is kept in FP64).  REORTH keeps every basis
// vector in Q (global scratch) and reorthogonalises against all of them.
template <typename R, bool REORTH>
__device__ double lanczos_min(const R* w, R* vprev, R* vcur, R* z, R* alpha, R* beta,
                              double* h, double* Q, int kmax, double tol, const uint16_t* nbr, int V,
                              int d, int lane, uint64_t seed, unsigned long long entry, int* steps) {
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
  const R bound = (R)(4 * d + 1);
  R b = 0;
  R theta = bound, theta_prev = (R)1e30;
  int j = 0;
  for (; j < kmax; ++j) {
    if (REORTH) {
      for (int x = lane; x < V; x += 32) Q[(size_t)j * V + x] = (double)vcur[x];
    }
    R a = 0;
    for (int x = lane; x < V; x += 32) {
      const R mv = matvec_site(w, vcur, nbr + x * 2 * d, x, d, V) - b * vprev[x];
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
    m = warp_sum(m) / (R)V;
    R bn = 0;
    for (int x = lane; x < V; x += 32) { const R v = z[x] - m; z[x] = v; bn += v * v; }
    bn = sqrt(warp_sum(bn));
    if (lane == 0) { alpha[j] = a; beta[j + 1] = bn; }
    __syncwarp();
    const bool last = (j + 1 == kmax) || bn < (R)1e-12;
    if (last || (!REORTH && (j + 1) % 8 == 0 && j + 1 >= 16)) {
      theta = tri_min<R>(alpha, beta, j + 1, -bound, bound, lane);
      if (last) { ++j; break; }
      if (fabs(theta - theta_prev) <= (R)tol * fmax(fabs(theta), (R)1e-3)) { ++j; break; }
      theta_prev = theta;
    }
    const R ib = (R)1 / bn;
    for (int x = lane; x < V; x += 32) { vprev[x] = vcur[x]; vcur[x] = z[x] * ib; }
    b = bn;
    __syncwarp();
  }
  *steps += j;
  return (double)theta;
}

__global__ void __launch_bounds__(128) fp_test_kernel(const FpArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Geom G = a.geom;
  const int V = G.V, d = G.d;
  const int warps = blockDim.x >> 5;
  const int kmax = a.mode == kFpDense ? a.kmax64 : (a.kmax64 > a.kmax32 ? a.kmax64 : a.kmax32);
  const FpSmem lay(V, d, kmax, warps);
  uint16_t* nbr = reinterpret_cast<uint16_t*>(smem + lay.nbr);
  uint16_t csite_dummy[1];
  (void)csite_dummy;
  for (int x = threadIdx.x; x < V; x += blockDim.x)
    for (int mu = 0; mu < d; ++mu) {
      nbr[x * 2 * d + 2 * mu] = (uint16_t)neighbor(x, mu, +1, G.L);
      nbr[x * 2 * d + 2 * mu + 1] = (uint16_t)neighbor(x, mu, -1, G.L);
    }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned char* base = smem + lay.warp0 + (size_t)warp * lay.per_warp;
  double* w64 = reinterpret_cast<double*>(base);
  float* w32 = reinterpret_cast<float*>(base + FpSmem::align16s((size_t)V * d * 8));
  unsigned char* vb = reinterpret_cast<unsigned char*>(w32) + FpSmem::align16s((size_t)V * d * 4);
  const size_t vstride = FpSmem::align16s((size_t)V * 8);
  double* alpha = reinterpret_cast<double*>(vb + 3 * vstride);
  double* beta = alpha + FpSmem::align16s((size_t)(kmax + 2) * 8) / 8;
  double* h = beta + FpSmem::align16s((size_t)(kmax + 2) * 8) / 8;

  const long long gwarp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  double* Q = a.mode == kFpDense ? a.scratch + (size_t)gwarp * V * V : nullptr;
  const unsigned n = *a.n_list;
  unsigned long long c_tests = 0, c64 = 0;
  int steps = 0;
  for (long long li = gwarp; li < (long long)n; li += nwarps) {
    const unsigned e = a.list[li];
    const double2* g = a.cfg + (size_t)e * V;
    // the start vector depends on the copy (its lowest start index), not on
    // where the copy sits in the pool, so results do not depend on insertion order
    const unsigned long long key = __ldcg(a.first_start + e);
    float2* g32 = reinterpret_cast<float2*>(vb);   // scratch until the Lanczos vectors start
    for (int x = lane; x < V; x += 32) {
      const double2 gx = g[x];
      g32[x] = make_float2(d2f_bits(gx.x), d2f_bits(gx.y));
    }
    __syncwarp();
    for (int x = lane; x < V; x += 32) {
      const float2 gx = g32[x];
      for (int mu = 0; mu < d; ++mu) {
        const float2 hx = g32[nbr[x * 2 * d + 2 * mu]];
        const float2 uu = a.links32[x * d + mu];
        const float tx = fmaf(uu.x, hx.x, -uu.y * hx.y), ty = fmaf(uu.x, hx.y, uu.y * hx.x);
        w32[mu * V + x] = fmaf(gx.x, tx, gx.y * ty);   // cos(phi^theta_{x,mu})
      }
    }
    __syncwarp();
    // FP64 weights, only when an FP64 Lanczos will run
    auto weights64 = [&]() {
      for (int x = lane; x < V; x += 32) {
        const double2 gx = g[x];
        for (int mu = 0; mu < d; ++mu) {
          const double2 hx = g[nbr[x * 2 * d + 2 * mu]];
          const double2 uu = a.links64[x * d + mu];
          const double tx = fma(uu.x, hx.x, -uu.y * hx.y), ty = fma(uu.x, hx.y, uu.y * hx.x);
          w64[mu * V + x] = fma(gx.x, tx, gx.y * ty);
        }
      }
      __syncwarp();
    };
    double lam;
    if (a.mode == kFpNone) {
      lam = __longlong_as_double(0x7ff8000000000000LL);
    } else if (a.mode == kFpDense) {
      const int k = V - 1 < a.kmax64 ? V - 1 : a.kmax64;
      weights64();
      lam = lanczos_min<double, true>(w64, (double*)vb, (double*)(vb + vstride), (double*)(vb + 2 * vstride),
                                      alpha, beta, h, Q, k, 0.0, nbr, V, d, lane, a.seed, key, &steps);
      ++c64;
    } else {
      bool decided = false;
      lam = 0.0;
      if (a.mode == kFpAuto) {
        const int k = V - 1 < a.kmax32 ? V - 1 : a.kmax32;
        lam = lanczos_min<float, false>(w32, (float*)vb, (float*)(vb + vstride), (float*)(vb + 2 * vstride),
                                        (float*)alpha, (float*)beta, h, nullptr, k, a.tol32, nbr, V, d,
                                        lane, a.seed, key, &steps);
        decided = lam > a.margin32;
      }
      if (!decided) {
        const int k = V - 1 < a.kmax64 ? V - 1 : a.kmax64;
        weights64();
        lam = lanczos_min<double, false>(w64, (double*)vb, (double*)(vb + vstride), (double*)(vb + 2 * vstride),
                                         alpha, beta, h, nullptr, k, a.tol64, nbr, V, d, lane, a.seed, key, &steps);
        ++c64;
      }
    }
    if (lane == 0) {
      a.lambda2[e] = lam;
      a.region[e] = a.mode == kFpNone ? -1 : (lam > a.tau ? kRegionIn : (lam < -a.tau ? kRegionOut : kRegionMarginal));
    }
    ++c_tests;
    __syncwarp();
  }
  if (lane == 0 && c_tests) {
    atomicAdd(&a.stats[13], c_tests);
    atomicAdd(&a.stats[14], c64);
    atomicAdd(&a.stats[15], (unsigned long long)steps);
  }
}

}  // namespace gc
