// Shared device helpers of the Gribov-copy enumerator (sm_103a).
//
// Lattice conventions: V = L^d sites, idx(x) = sum_mu x_mu L^mu (x_0 fastest),
// link (x, mu) at idx(x)*d + mu, complex numbers as (re, im) pairs.
// g_x = exp(i theta_x) is the gauge transformation, u_{x,mu} = exp(i phi_{x,mu})
// the link (compact U(1), Eq. 3).  S_x = sum_mu [u_{x,mu} g_{x+mu} +
// conj(u_{x-mu,mu}) g_{x-mu}] collects every term of Eq. 3 that involves
// theta_x: they sum to Re[conj(g_x) S_x], so the local optimum of Eq. 4 is
// g_x = S_x / |S_x|, and Im[conj(g_x) S_x] is the lattice divergence (minus the
// gradient of Eq. 3).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace gc {

constexpr int kMaxDim = 4;
constexpr int kMaxSites = 4096;   // per lattice in shared memory; neighbour tables use uint16
constexpr int kMaxSlabSites = 1 << 16;   // per lattice streamed in hyperplanes (gc_slab.cuh)

// ---------------------------------------------------------------------------
// Philox4x64-10 counter-based generator (Salmon et al., SC'11): the generator
// the paper names for its random starts (Section III).
// ---------------------------------------------------------------------------
struct U64x4 { uint64_t v[4]; };

__device__ __forceinline__ U64x4 philox4x64_10(uint64_t c0, uint64_t c1, uint64_t c2,
                                               uint64_t c3, uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
  const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += W0; k1 += W1; }
    const uint64_t lo0 = M0 * c0, hi0 = __umul64hi(M0, c0);
    const uint64_t lo1 = M1 * c2, hi1 = __umul64hi(M1, c2);
    const uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
  }
  U64x4 o; o.v[0] = c0; o.v[1] = c1; o.v[2] = c2; o.v[3] = c3;
  return o;
}

// Uniform point on the unit circle for (start, site): counter (start, site,
// attempt, 0), key (seed, orbit_id).  Each block yields two candidate points
// in [-1,1)^2 from 53-bit uniforms; the first with 0 < r^2 <= 1 is scaled onto
// the circle.  Every operation is an explicitly rounded IEEE step so the
// result does not depend on FMA contraction.
__device__ __forceinline__ double2 random_unit(uint64_t seed, uint64_t orbit_id,
                                               uint64_t start, uint64_t site) {
  for (uint64_t attempt = 0;; ++attempt) {
    const U64x4 w = philox4x64_10(start, site, attempt, 0, seed, orbit_id);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const double x = __dsub_rn(__dmul_rn(2.0, __dmul_rn((double)(w.v[2 * k] >> 11), 0x1.0p-53)), 1.0);
      const double y = __dsub_rn(__dmul_rn(2.0, __dmul_rn((double)(w.v[2 * k + 1] >> 11), 0x1.0p-53)), 1.0);
      const double n2 = __dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y));
      if (n2 > 0.0 && n2 <= 1.0) {
        const double r = __drcp_rn(__dsqrt_rn(n2));
        return make_double2(__dmul_rn(x, r), __dmul_rn(y, r));
      }
    }
  }
}

// 1/sqrt(x) by the special-function unit's approximation, subnormals flushed
// (PTX rsqrt.approx.ftz.f32).  Every caller passes a normal x
// (at least 1e-30).
__device__ __forceinline__ float rsqrt_sfu(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// The same construction in FP32 (bulk phase of the mixed path): the candidate
// points are the top 24 bits of the same Philox words, so a start is the FP64
// start to FP32 precision (an acceptance decision can differ only when
// x^2 + y^2 lies within FP32 rounding of 1).  No FP64 instruction is used.
__device__ __forceinline__ float2 random_unit32(uint64_t seed, uint64_t orbit_id, uint64_t start,
                                                uint64_t site) {
  for (uint64_t attempt = 0; attempt < 64; ++attempt) {
    const U64x4 w = philox4x64_10(start, site, attempt, 0, seed, orbit_id);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const float x = fmaf((float)(unsigned)(w.v[2 * k] >> 40), 0x1.0p-23f, -1.0f);
      const float y = fmaf((float)(unsigned)(w.v[2 * k + 1] >> 40), 0x1.0p-23f, -1.0f);
      const float n2 = fmaf(x, x, y * y);
      if (n2 > 0.f && n2 <= 1.f) {
        const float r = rsqrtf(n2);
        return make_float2(x * r, y * r);
      }
    }
  }
  return make_float2(1.f, 0.f);  // unreachable in practice (p = 0.046^64)
}

// ---------------------------------------------------------------------------
// lattice geometry, computed once per CTA into shared memory
// ---------------------------------------------------------------------------
struct Geom {
  int d, L, V, ncolor;
  int color_off[4];     // first position of each colour (+ end)
  int pos_last;         // position of site V-1 (the site whose angle is fixed to 0)
};

__host__ __device__ inline int ipow(int b, int e) { int r = 1; for (int i = 0; i < e; ++i) r *= b; return r; }

// Colour: L even -> parity of sum x_mu; L odd -> sum_mu c(x_mu) mod 3 with
// c(j) = j mod 2 (j < L-1) and c(L-1) = 2 (a proper colouring of odd tori).
__host__ __device__ inline int site_color(int x, int d, int L) {
  int s = 0;
  for (int mu = 0; mu < d; ++mu) {
    const int xm = x % L; x /= L;
    s += (L % 2 == 0) ? xm : ((xm == L - 1) ? 2 : (xm & 1));
  }
  return s % ((L % 2 == 0) ? 2 : 3);
}

__host__ __device__ inline int neighbor(int x, int mu, int step, int L) {
  const int stride = ipow(L, mu);
  const int xm = (x / stride) % L;
  const int xn = (xm + step + L) % L;
  return x + (xn - xm) * stride;
}

// nbr[x*2d + 2mu] = x+mu, nbr[x*2d + 2mu + 1] = x-mu; csite = sites sorted by colour.
__device__ inline void build_geometry(const Geom& g, uint16_t* nbr, uint16_t* csite) {
  const int V = g.V, d = g.d, L = g.L;
  for (int x = threadIdx.x; x < V; x += blockDim.x) {
    for (int mu = 0; mu < d; ++mu) {
      nbr[x * 2 * d + 2 * mu] = (uint16_t)neighbor(x, mu, +1, L);
      nbr[x * 2 * d + 2 * mu + 1] = (uint16_t)neighbor(x, mu, -1, L);
    }
  }
  // colour lists: ordered by site index within a colour (order is irrelevant
  // for the result: sites of one colour never neighbour each other)
  if (threadIdx.x < 32) {
    for (int c = 0; c < g.ncolor; ++c) {
      int base = g.color_off[c];
      for (int x0 = 0; x0 < V; x0 += 32) {
        const int x = x0 + (int)threadIdx.x;
        const bool mine = x < V && site_color(x, d, L) == c;
        const unsigned m = __ballot_sync(0xffffffffu, mine);
        if (mine) csite[base + __popc(m & ((1u << threadIdx.x) - 1u))] = (uint16_t)x;
        base += __popc(m);
      }
    }
  }
}

// Colour-major geometry.  Position p enumerates the sites of colour 0, then
// colour 1 (then 2), each colour in increasing site order, so the sites one
// colour phase updates are contiguous and their neighbours (the other
// colours) sit at nearly contiguous positions: shared-memory accesses of a
// warp stay (almost) free of bank conflicts.
//   site[p]: site index at position p (site 0 is at position 0)
//   nbp[p] : word mu (of 4) = pos(x + e_mu) | pos(x - e_mu) << 16
// pos (V entries) is scratch for the construction.  Must be called by every
// thread of the block; ends with __syncthreads().
__device__ inline void build_colour_geometry(const Geom& G, uint16_t* site, uint4* nbp, uint16_t* pos) {
  const int V = G.V, d = G.d, L = G.L;
  if (threadIdx.x < 32) {
    for (int c = 0; c < G.ncolor; ++c) {
      int base = G.color_off[c];
      for (int x0 = 0; x0 < V; x0 += 32) {
        const int x = x0 + (int)threadIdx.x;
        const bool mine = x < V && site_color(x, d, L) == c;
        const unsigned m = __ballot_sync(0xffffffffu, mine);
        if (mine) {
          const int p = base + __popc(m & ((1u << threadIdx.x) - 1u));
          site[p] = (uint16_t)x;
          pos[x] = (uint16_t)p;
        }
        base += __popc(m);
      }
    }
  }
  __syncthreads();
  for (int p = threadIdx.x; p < V; p += blockDim.x) {
    const int x = site[p];
    unsigned w[4] = {0u, 0u, 0u, 0u};
    for (int mu = 0; mu < d; ++mu)
      w[mu] = (unsigned)pos[neighbor(x, mu, +1, L)] | ((unsigned)pos[neighbor(x, mu, -1, L)] << 16);
    nbp[p] = make_uint4(w[0], w[1], w[2], w[3]);
  }
  __syncthreads();
}

__device__ __forceinline__ unsigned nb_word(const uint4& nb, int mu) {
  return mu == 0 ? nb.x : (mu == 1 ? nb.y : (mu == 2 ? nb.z : nb.w));
}

// ---------------------------------------------------------------------------
// team helpers: a team is T consecutive lanes of one warp (T a power of 2)
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ R team_max(R v, int T, unsigned mask) {
  for (int o = T >> 1; o > 0; o >>= 1) { const R w = __shfl_xor_sync(mask, v, o); v = v > w ? v : w; }
  return v;
}
template <typename R>
__device__ __forceinline__ R team_sum(R v, int T, unsigned mask) {
  for (int o = T >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o);
  return v;
}

__device__ __forceinline__ unsigned team_mask(int T, int team_in_warp) {
  return T == 32 ? 0xffffffffu : (((1u << T) - 1u) << (team_in_warp * T));
}

// ---------------------------------------------------------------------------
// float <-> double by bit manipulation on the integer pipe.  On this part the
// FP64 pipe, which also executes the F2F conversion instructions, is the
// scarce unit (about 1/64 of the FP32 rate); these helpers keep conversions
// off it.  f2d is exact for normal floats and zero (subnormals become 0);
// d2f truncates toward zero (|error| < 1 ulp of float, |x| < 2^-126 -> 0).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned hi = e ? ((u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7fffffu) >> 3))
                        : (u & 0x80000000u);
  const unsigned lo = e ? (u << 29) : 0u;
  return __hiloint2double((int)hi, (int)lo);
}
__device__ __forceinline__ float d2f_bits(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const int e = (int)((hi >> 20) & 0x7ffu) - 896;
  const unsigned sign = hi & 0x80000000u;
  if (e <= 0) return __uint_as_float(sign);
  if (e >= 255) return __uint_as_float(sign | 0x7f800000u);
  return __uint_as_float(sign | ((unsigned)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
}
// the same to nearest (ties away from zero): half an FP32 unit in the last
// place added to the magnitude's bit pattern before truncation
__device__ __forceinline__ float d2f_near(double x) {
  return d2f_bits(__longlong_as_double(__double_as_longlong(x) + 0x10000000LL));
}
// max of two non-negative doubles by their bit patterns (integer compare)
__device__ __forceinline__ double dmax_pos(double a, double b) {
  return __double_as_longlong(a) > __double_as_longlong(b) ? a : b;
}
__device__ __forceinline__ bool dless_pos(double a, double b) {
  return __double_as_longlong(a) < __double_as_longlong(b);
}

// 64-bit mixer (splitmix64 finaliser) for hash-table bucket indices.
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

}  // namespace gc
