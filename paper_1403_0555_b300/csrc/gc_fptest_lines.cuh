// FP32 first-region screen for lattices whose lines of each parity fill one
// warp (4^4): one warp per copy, lane h owns the h-th line (along axis 0) of
// each parity, as in polish_pairs_kernel.  The lane keeps its 2L sites' link
// weights (forward, and backward off axis 0) and its entries of the Lanczos
// vectors in registers; axis-0 neighbours are its own sites, the others'
// entries of the current vector come from a [x_0][parity][h] shared copy.  A
// matrix-vector product then reads 2(D-1) shared words per site.  The Lanczos
// recurrence, its convergence test (Sturm multisection on the tridiagonal,
// brackets from Cauchy interlacing), the margin and the redo list are those of
// fp_screen_kernel; sums run in a different order, so Ritz values agree to
// rounding.
#pragma once
#include "gc_fptest.cuh"
#include "gc_relax.cuh"

namespace gc {

template <int D, int L>
struct FpPairSmem {
  using LG = LineGeom<D, L>;
  static constexpr size_t links = 0;                                    // float2 [L][D][2][NLH]
  static constexpr size_t warp0 = (size_t)LG::V * D * sizeof(float2);
  // per warp: the copy's FP32 configuration (float2 [L][2][NLH]), reused for
  // the Lanczos vector (float), then alpha and beta^2
  __host__ __device__ static size_t per_warp(int kmax) { return (size_t)LG::V * 8 + 2 * ((((size_t)kmax + 2) * 4 + 15) & ~size_t(15)); }
  __host__ __device__ static size_t bytes(int warps, int kmax) { return warp0 + (size_t)warps * per_warp(kmax); }
};

template <int D, int L>
__global__ void __launch_bounds__(256, 2) fp_screen_pairs_kernel(const FpArgs a) {
  using LG = LineGeom<D, L>;
  using SM = FpPairSmem<D, L>;
  constexpr int NLH = LG::NLH, V = LG::V;
  static_assert(NLH == 32, "one warp holds one line of each parity per lane");
  constexpr int SG = 2 * NLH * 8;   // bytes from x0 to x0 + 1 of a line: configuration, links
  constexpr int SV = 2 * NLH * 4;   //                                     Lanczos vector
  extern __shared__ __align__(16) unsigned char smem[];
  const int warps = blockDim.x >> 5;
  const unsigned n = *a.n_list;
  if ((unsigned long long)blockIdx.x * warps >= n) return;   // no copy for this CTA (uniform)
  const int kmax = a.kmax32;
  const int h = threadIdx.x & 31, warp = threadIdx.x >> 5;

  // FP32 links into shared memory, [x0][mu][parity][h]
  for (int e = threadIdx.x; e < 2 * NLH * L * D; e += blockDim.x) {
    const int lq = e % (2 * NLH), rest = e / (2 * NLH), mu = rest % D, k = rest / D;
    const int ql = lq / NLH, hl = lq % NLH;
    const int ll = line_of<D, L>(ql, hl);
    reinterpret_cast<float2*>(smem + SM::links)[((k * D + mu) * 2 + ql) * NLH + hl] =
        a.links32[(size_t)(k + L * ll) * D + mu];
  }
  __syncthreads();

  unsigned char* wbase = smem + SM::warp0 + (size_t)warp * SM::per_warp(kmax);
  const unsigned s_g = (unsigned)__cvta_generic_to_shared(wbase);   // configuration, then vector
  const unsigned s_u = (unsigned)__cvta_generic_to_shared(smem + SM::links);
  float* alpha = reinterpret_cast<float*>(wbase + (size_t)V * 8);
  float* beta = alpha + ((((size_t)kmax + 2) * 4 + 15) & ~size_t(15)) / 4;
  // per parity P: the line, and the neighbour lines' element indices along mu >= 1
  int line[2];
  unsigned ep[2][D], em[2][D];
#pragma unroll
  for (int P = 0; P < 2; ++P) {
    const int l = line_of<D, L>(P, h);
    line[P] = l;
    int t = l, stride = 1;
    ep[P][0] = em[P][0] = 0;
#pragma unroll
    for (int mu = 1; mu < D; ++mu) {
      const int c = t % L;
      t /= L;
      const int lp = l + (((c + 1) % L) - c) * stride;
      const int lm = l + (((c + L - 1) % L) - c) * stride;
      ep[P][mu] = (1 - P) * NLH + half_of<D, L>(lp);
      em[P][mu] = (1 - P) * NLH + half_of<D, L>(lm);
      stride *= L;
    }
  }
  auto warp_sum = [](float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
  };

  const long long gwarp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  unsigned long long c_tests = 0;
  int steps = 0;
  float wf[2][L][D], wb[2][L][D], v[2][L], vp[2][L];
  for (long long li = gwarp; li < (long long)n; li += nwarps) {
    const unsigned e = a.list[li];
    const double2* g = a.cfg + (size_t)e * V;
    const unsigned long long key = __ldcg(a.first_start + e);
    // the copy's configuration in FP32, [x0][parity][h]
    static_for<2>([&](auto PC) {
      constexpr int P = decltype(PC)::value;
      static_for<L>([&](auto KC) {
        constexpr int K = decltype(KC)::value;
        const double2 gx = __ldcg(g + K + L * line[P]);
        sts_f2<K * SG>(s_g + 8u * (P * NLH + h), make_float2(d2f_bits(gx.x), d2f_bits(gx.y)));
      });
    });
    __syncwarp();
    // link weights cos(phi^theta): forward w_{x,mu}, and w_{x-mu,mu} for mu >= 1
    static_for<2>([&](auto PC) {
      constexpr int P = decltype(PC)::value;
      const unsigned go = s_g + 8u * (P * NLH + h), uo = s_u + 8u * (P * NLH + h);
      static_for<L>([&](auto KC) {
        constexpr int K = decltype(KC)::value;
        const float2 gx = lds_f2<K * SG>(go);
        static_for<D>([&](auto MC) {
          constexpr int mu = decltype(MC)::value;
          const float2 A = lds_f2<(K * D + mu) * SG>(uo);
          float2 H;
          if constexpr (mu == 0) H = lds_f2<((K + 1) % L) * SG>(go);
          else H = lds_f2<K * SG>(s_g + 8u * ep[P][mu]);
          const float tx = fmaf(A.x, H.x, -A.y * H.y), ty = fmaf(A.x, H.y, A.y * H.x);
          wf[P][K][mu] = fmaf(gx.x, tx, gx.y * ty);
          if constexpr (mu > 0) {
            const float2 B = lds_f2<(K * D + mu) * SG>(s_u + 8u * em[P][mu]);
            const float2 Gm = lds_f2<K * SG>(s_g + 8u * em[P][mu]);
            const float sx = fmaf(B.x, gx.x, -B.y * gx.y), sy = fmaf(B.x, gx.y, B.y * gx.x);
            wb[P][K][mu] = fmaf(Gm.x, sx, Gm.y * sy);
          }
        });
      });
    });
    __syncwarp();   // the configuration's shared copy is now free for the vector
    // random start vector orthogonal to the constant mode (as in lanczos_min),
    // drawn in a loop through the lane's own shared slots (compact code)
#pragma unroll 1
    for (int i = 0; i < 2 * L; ++i) {
      const int P = i / L, K = i % L;
      const U64x4 r = philox4x64_10(key, (uint64_t)(K + L * line[P ? 1 : 0]), 0, 1, a.seed, 0x4C414E43ULL);
      sts_f1<0>(s_g + 4u * (P * NLH + h) + (unsigned)K * SV, (float)(unsigned)(r.v[0] >> 40) * 0x1.0p-24f - 0.5f);
    }
    float s = 0.f;
    static_for<2>([&](auto PC) {
      constexpr int P = decltype(PC)::value;
      static_for<L>([&](auto KC) {
        constexpr int K = decltype(KC)::value;
        v[P][K] = lds_f1<K * SV>(s_g + 4u * (P * NLH + h));
        vp[P][K] = 0.f;
        s += v[P][K];
      });
    });
    s = warp_sum(s) / (float)V;
    float nn = 0.f;
    static_for<2>([&](auto PC) {
      static_for<L>([&](auto KC) {
        constexpr int P = decltype(PC)::value, K = decltype(KC)::value;
        v[P][K] -= s;
        nn += v[P][K] * v[P][K];
      });
    });
    const float inv0 = 1.f / sqrtf(warp_sum(nn));
    static_for<2>([&](auto PC) {
      constexpr int P = decltype(PC)::value;
      static_for<L>([&](auto KC) {
        constexpr int K = decltype(KC)::value;
        v[P][K] *= inv0;
        sts_f1<K * SV>(s_g + 4u * (P * NLH + h), v[P][K]);
      });
    });
    __syncwarp();
    const float bound = (float)(4 * D + 1);
    float bprev = 0.f, theta = bound, theta_prev = bound, theta_pp = bound;
    const int kk = V - 1 < kmax ? V - 1 : kmax;
    int stalls = 0;
    int j = 0;
    for (; j < kk; ++j) {
      // z = M v - b v_prev, alpha = z . v
      float z[2][L], av = 0.f;
      static_for<2>([&](auto PC) {
        constexpr int P = decltype(PC)::value;
        static_for<L>([&](auto KC) {
          constexpr int K = decltype(KC)::value;
          const float vx = v[P][K];
          float acc = 0.f;
          static_for<D>([&](auto MC) {
            constexpr int mu = decltype(MC)::value;
            if constexpr (mu == 0) {
              acc = fmaf(wf[P][K][0], vx - v[P][(K + 1) % L], acc);
              acc = fmaf(wf[P][(K + L - 1) % L][0], vx - v[P][(K + L - 1) % L], acc);
            } else {
              acc = fmaf(wf[P][K][mu], vx - lds_f1<K * SV>(s_g + 4u * ep[P][mu]), acc);
              acc = fmaf(wb[P][K][mu], vx - lds_f1<K * SV>(s_g + 4u * em[P][mu]), acc);
            }
          });
          z[P][K] = acc - bprev * vp[P][K];
          av += z[P][K] * vx;
        });
      });
      const float al = warp_sum(av);
      float m = 0.f, zz = 0.f;
      static_for<2>([&](auto PC) {
        static_for<L>([&](auto KC) {
          constexpr int P = decltype(PC)::value, K = decltype(KC)::value;
          z[P][K] -= al * v[P][K];
          m += z[P][K];
          zz += z[P][K] * z[P][K];
        });
      });
      for (int o = 16; o > 0; o >>= 1) {
        m += __shfl_xor_sync(0xffffffffu, m, o);
        zz += __shfl_xor_sync(0xffffffffu, zz, o);
      }
      m /= (float)V;
      const float bn = sqrtf(fmaxf(zz - (float)V * m * m, 0.f));
      if (h == 0) { alpha[j] = al; beta[j + 1] = bn * bn; }
      __syncwarp();
      const bool last = (j + 1 == kk) || bn < 1e-12f;
      if (last || ((j + 1) % 8 == 0 && j + 1 >= 16)) {
        float lo = -bound, hi = bound;
        if (theta_prev < bound) {
          const float slack = 2.f * tri_rel<float>() * fmaxf(fabsf(theta_prev), 1.f);
          hi = theta_prev + slack;
          if (theta_pp < bound) {
            const float l = theta_prev - 4.f * fmaxf(theta_pp - theta_prev, slack);
            if (sturm_count<float>(alpha, beta, j + 1, l) == 0) lo = l;
          }
        }
        theta = tri_min<float>(alpha, beta, j + 1, lo, hi, h);
        if (last) { ++j; break; }
        // two checks in a row (16 steps), as in lanczos_min
        if (fabsf(theta - theta_prev) <= (float)a.tol32 * fmaxf(fabsf(theta), 1e-3f)) {
          if (++stalls == 2) { ++j; break; }
        } else {
          stalls = 0;
        }
        theta_pp = theta_prev;
        theta_prev = theta;
      }
      const float ib = 1.f / bn;
      static_for<2>([&](auto PC) {
        constexpr int P = decltype(PC)::value;
        static_for<L>([&](auto KC) {
          constexpr int K = decltype(KC)::value;
          vp[P][K] = v[P][K];
          v[P][K] = (z[P][K] - m) * ib;
          sts_f1<K * SV>(s_g + 4u * (P * NLH + h), v[P][K]);
        });
      });
      bprev = bn;
      __syncwarp();
    }
    steps += j;
    if (h == 0) {
      if (theta > (float)a.margin32) {
        a.lambda2[e] = (double)theta;
        a.region[e] = region_of((double)theta, a.tau);
      } else {
        a.redo[atomicAdd(a.n_redo, 1u)] = e;
      }
    }
    ++c_tests;
    __syncwarp();
  }
  if (h == 0 && c_tests) {
    atomicAdd(&a.stats[13], c_tests);
    atomicAdd(&a.stats[15], (unsigned long long)steps);
  }
}

// ---------------------------------------------------------------------------
// The Lanczos mode's first-region test on the same layout (4^4): an FP64
// Lanczos process seeded by an FP32 Ritz vector, as lanczos32_ritz +
// lanczos64_seeded do for any lattice, with the FP32 work in registers.
//   The copy's FP64 weights cos(phi^theta) (negated, forward links) are formed
//   first, from the FP64 configuration and links in global memory, into a
//   shared [x_0][mu][parity][h] table; lane h rounds its 2L sites' weights
//   (forward, and backward off axis 0) to FP32 registers.
//   FP32 seed: the lane keeps its entries of the Lanczos vectors in registers
//   (axis-0 neighbours are its own sites, the others come from a
//   [x_0][parity][h] shared copy of the vector).  Pass 1 runs the recurrence
//   from the random start until its Ritz values stall, then `extra32` steps
//   more, recording alpha, beta and the mean each step removes; two inverse
//   iterations give the eigenvector s of T_k for its smallest eigenvalue; pass
//   2 runs the same loop body from the recorded coefficients (same operations,
//   same bits) and sums y = sum_j s_j q_j.
//   FP64: the diagonal of M and the Lanczos vectors in registers, the
//   weights from the shared table; the process starts from y.
// Shared memory per warp: the FP64 weight table, then either the FP32 phase
// (vector copy, tridiagonal record) or, in the same bytes, the FP64 phase
// (vector copy, alpha and beta^2 of at most kMax64 steps).
// ---------------------------------------------------------------------------
template <int D, int L>
struct FpTestPairSmem {
  using LG = LineGeom<D, L>;
  static constexpr int kMax64 = 128;   // cap on the FP64 steps that follow the seed
  static constexpr int kMax32 = 150;   // cap on the FP32 steps of the seed
  static constexpr size_t warp0 = 0;
  __host__ __device__ static size_t a16(size_t b) { return (b + 15) & ~size_t(15); }
  __host__ __device__ static int k32(int kmax32) { return kmax32 < kMax32 ? kmax32 : kMax32; }
  __host__ __device__ static size_t tri32(int kmax32) { return a16(((size_t)k32(kmax32) + 2) * 4); }
  __host__ __device__ static size_t tri64(int kmax64) { return a16(((size_t)kmax64 + 2) * 8); }
  static constexpr size_t table = (size_t)LG::V * D * 8;
  __host__ __device__ static size_t per_warp(int kmax32, int kmax64) {
    const size_t p32 = (size_t)LG::V * 4 + 8 * tri32(kmax32);
    const size_t p64 = (size_t)LG::V * 8 + 2 * tri64(kmax64);
    return table + (p32 > p64 ? p32 : p64);
  }
  __host__ __device__ static size_t bytes(int warps, int kmax32, int kmax64) {
    return warp0 + (size_t)warps * per_warp(kmax32, kmax64);
  }
};

template <int OFF>
__device__ __forceinline__ double lds_d1(unsigned base) {
  double v;
  asm volatile("ld.shared.f64 %0, [%1+%2];" : "=d"(v) : "r"(base), "n"(OFF));
  return v;
}
template <int OFF>
__device__ __forceinline__ void sts_d1(unsigned base, double v) {
  asm volatile("st.shared.f64 [%0+%1], %2;" ::"r"(base), "n"(OFF), "d"(v) : "memory");
}

template <int D, int L>
__global__ void __launch_bounds__(384, 1) fp_test_pairs_kernel(const FpArgs a) {
  using LG = LineGeom<D, L>;
  using SM = FpTestPairSmem<D, L>;
  constexpr int NLH = LG::NLH, V = LG::V;
  static_assert(NLH == 32, "one warp holds one line of each parity per lane");
  constexpr int SG = 2 * NLH * 8;   // bytes from x0 to x0 + 1: FP64 vector
  constexpr int SV = 2 * NLH * 4;   //                          FP32 vector
  constexpr int SW = 2 * NLH * 8;   // bytes from (x0, mu) to the next pair of the FP64 weights
  extern __shared__ __align__(16) unsigned char smem[];
  const int warps = blockDim.x >> 5;
  const unsigned n = *a.n_list;
  if ((unsigned long long)blockIdx.x * warps >= n) return;   // no copy for this CTA (uniform)
  const int kmax32 = SM::k32(a.kmax32);
  const int kmax64 = a.kmax64 < SM::kMax64 ? a.kmax64 : SM::kMax64;
  const int h = threadIdx.x & 31, warp = threadIdx.x >> 5;

  unsigned char* wbase = smem + SM::warp0 + (size_t)warp * SM::per_warp(kmax32, kmax64);
  const unsigned s_w = (unsigned)__cvta_generic_to_shared(wbase);   // FP64 weight table
  const unsigned s_v = s_w + (unsigned)SM::table;                    // FP32, then FP64, vector copy
  float* f = reinterpret_cast<float*>(wbase + SM::table + (size_t)V * 4);
  const size_t t32 = SM::tri32(kmax32) / 4;
  const Ritz32 R{f, f + t32, f + 2 * t32, f + 3 * t32, f + 4 * t32, f + 5 * t32, f + 6 * t32, f + 7 * t32};
  // the second Ritz vector's sums, float2 [x0][h], in the bytes of R.pd and
  // R.pl once the inverse iterations are done
  const unsigned s_y2 = (unsigned)__cvta_generic_to_shared(R.pd) + 8u * h;
  double* a64 = reinterpret_cast<double*>(wbase + SM::table + (size_t)V * 8);
  double* b64 = a64 + SM::tri64(kmax64) / 8;
  // per parity P: the line, and the neighbour lines' element indices along mu >= 1
  int line[2];
  unsigned ep[2][D], em[2][D];
#pragma unroll
  for (int P = 0; P < 2; ++P) {
    const int l = line_of<D, L>(P, h);
    line[P] = l;
    int t = l, stride = 1;
    ep[P][0] = em[P][0] = 0;
#pragma unroll
    for (int mu = 1; mu < D; ++mu) {
      const int c = t % L;
      t /= L;
      const int lp = l + (((c + 1) % L) - c) * stride;
      const int lm = l + (((c + L - 1) % L) - c) * stride;
      ep[P][mu] = (1 - P) * NLH + half_of<D, L>(lp);
      em[P][mu] = (1 - P) * NLH + half_of<D, L>(lm);
      stride *= L;
    }
  }
  auto warp_sumf = [](float v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
  };

  const long long gwarp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  unsigned long long c_tests = 0;
  int steps = 0, steps64 = 0;
  // FP32 state as packed pairs: .x the lane's parity-0 site, .y its parity-1
  // site with the same x_0 (one f32x2 instruction serves both)
  float2 wf[L][D], wb[L][D], v[L], vp[L], y[L];

  for (long long li = gwarp; li < (long long)n; li += nwarps) {
    const unsigned e = a.list[li];
    const double2* g = a.cfg + (size_t)e * V;
    const unsigned long long key = __ldcg(a.first_start + e);
    // ---- FP64 weights (negated, forward links) into the shared table ----
#pragma unroll 1
    for (int i = 0; i < 2 * L * D; ++i) {
      const int P = i / (L * D), K = (i / D) % L, mu = i % D;
      const int l = line[P];
      int ln = l;   // the line of x + mu (axis 0 stays on the line)
      if (mu > 0) {
        int st = 1;
        for (int m = 1; m < mu; ++m) st *= L;
        const int c = (l / st) % L;
        ln = l + (((c + 1) % L) - c) * st;
      }
      const int x = K + L * l;
      const int xn = mu == 0 ? ((K + 1) % L) + L * l : K + L * ln;
      const double2 gx = __ldcg(g + x), hx = __ldcg(g + xn);
      const double2 uu = a.links64[x * D + mu];
      const double tx = fma(uu.x, hx.x, -uu.y * hx.y), ty = fma(uu.x, hx.y, uu.y * hx.x);
      const unsigned at = s_w + 8u * (unsigned)(P * NLH + h) + (unsigned)((K * D + mu) * SW);
      asm volatile("st.shared.f64 [%0], %1;" ::"r"(at), "d"(-fma(gx.x, tx, gx.y * ty)) : "memory");
    }
    __syncwarp();
    // the lane's FP32 weights: the FP64 ones rounded (positive), on the integer pipe
    static_for<L>([&](auto KC) {
      constexpr int K = decltype(KC)::value;
      static_for<D>([&](auto MC) {
        constexpr int mu = decltype(MC)::value;
        wf[K][mu] = make_float2(-d2f_near(lds_d1<(K * D + mu) * SW>(s_w + 8u * h)),
                                -d2f_near(lds_d1<(K * D + mu) * SW>(s_w + 8u * (NLH + h))));
        if constexpr (mu > 0)
          wb[K][mu] = make_float2(-d2f_near(lds_d1<(K * D + mu) * SW>(s_w + 8u * em[0][mu])),
                                  -d2f_near(lds_d1<(K * D + mu) * SW>(s_w + 8u * em[1][mu])));
      });
    });

    // ---- FP32 seed: pass 0 records the recurrence, pass 1 replays it into y ----
    // the random start vector (Philox draws, off the constant mode,
    // normalised); pass 0 keeps it in y for pass 1
#pragma unroll 1
    for (int i = 0; i < 2 * L; ++i) {
      const int P = i / L, K = i % L;
      const U64x4 r = philox4x64_10(key, (uint64_t)(K + L * line[P ? 1 : 0]), 0, 1, a.seed, 0x4C414E43ULL);
      sts_f1<0>(s_v + 4u * (P * NLH + h) + (unsigned)K * SV, (float)(unsigned)(r.v[0] >> 40) * 0x1.0p-24f - 0.5f);
    }
    __syncwarp();
    {
      float sm = 0.f;
      static_for<L>([&](auto KC) {
        constexpr int K = decltype(KC)::value;
        y[K] = make_float2(lds_f1<K * SV>(s_v + 4u * h), lds_f1<K * SV>(s_v + 4u * (NLH + h)));
        sm += y[K].x + y[K].y;
      });
      sm = warp_sumf(sm) / (float)V;
      float nn = 0.f;
      static_for<L>([&](auto KC) {
        constexpr int K = decltype(KC)::value;
        y[K] = fsub2(y[K], bcast2(sm));
        nn = fmaf(y[K].x, y[K].x, fmaf(y[K].y, y[K].y, nn));
      });
      const float inv0 = 1.f / sqrtf(warp_sumf(nn));
      static_for<L>([&](auto KC) { constexpr int K = decltype(KC)::value; y[K] = __fmul2_rn(y[K], bcast2(inv0)); });
    }
    const float bound = (float)(4 * D + 1);
    float theta = bound;
    const int kk = V - 1 < kmax32 ? V - 1 : kmax32;
    int k = kk;
#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {
      const float s0 = pass ? R.s[0] : 0.f, t0 = pass ? R.s2[0] : 0.f;
      static_for<L>([&](auto KC) {
        constexpr int K = decltype(KC)::value;
        v[K] = y[K];
        vp[K] = make_float2(0.f, 0.f);
        if (pass) {
          y[K] = __fmul2_rn(bcast2(s0), v[K]);
          sts_f2<K * 256>(s_y2, __fmul2_rn(bcast2(t0), v[K]));
        }
        sts_f1<K * SV>(s_v + 4u * h, v[K].x);
        sts_f1<K * SV>(s_v + 4u * (NLH + h), v[K].y);
      });
      __syncwarp();
      float theta_prev = bound, theta_pp = bound, b = 0.f;
      int kend = pass ? k - 1 : kk, j = 0;
      bool settled = false;
      for (; j < kend; ++j) {
        // z = M q_j - b q_{j-1} (and its product with q_j for alpha)
        float2 z[L], av = make_float2(0.f, 0.f);
        static_for<L>([&](auto KC) {
          constexpr int K = decltype(KC)::value;
          const float2 vx = v[K];
          float2 acc = __fmul2_rn(wf[K][0], fsub2(vx, v[(K + 1) % L]));
          acc = __ffma2_rn(wf[(K + L - 1) % L][0], fsub2(vx, v[(K + L - 1) % L]), acc);
          static_for<D - 1>([&](auto MC) {
            constexpr int mu = decltype(MC)::value + 1;
            const float2 np = make_float2(lds_f1<K * SV>(s_v + 4u * ep[0][mu]), lds_f1<K * SV>(s_v + 4u * ep[1][mu]));
            const float2 nm = make_float2(lds_f1<K * SV>(s_v + 4u * em[0][mu]), lds_f1<K * SV>(s_v + 4u * em[1][mu]));
            acc = __ffma2_rn(wf[K][mu], fsub2(vx, np), acc);
            acc = __ffma2_rn(wb[K][mu], fsub2(vx, nm), acc);
          });
          z[K] = __ffma2_rn(bcast2(-b), vp[K], acc);
          av = __ffma2_rn(z[K], vx, av);
        });
        float al, m, bn;
        if (pass == 0) {
          al = warp_sumf(av.x + av.y);
        } else {
          al = R.al[j];
        }
        float2 m2 = make_float2(0.f, 0.f), zz2 = make_float2(0.f, 0.f);
        static_for<L>([&](auto KC) {
          constexpr int K = decltype(KC)::value;
          z[K] = __ffma2_rn(bcast2(-al), v[K], z[K]);
          m2 = __fadd2_rn(m2, z[K]);
          zz2 = __ffma2_rn(z[K], z[K], zz2);
        });
        if (pass == 0) {
          m = m2.x + m2.y;
          float zz = zz2.x + zz2.y;
          for (int o = 16; o > 0; o >>= 1) {
            m += __shfl_xor_sync(0xffffffffu, m, o);
            zz += __shfl_xor_sync(0xffffffffu, zz, o);
          }
          m /= (float)V;
          bn = sqrtf(fmaxf(zz - (float)V * m * m, 0.f));
          if (h == 0) { R.al[j] = al; R.be2[j + 1] = bn * bn; R.mm[j] = m; R.bn[j + 1] = bn; }
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
            // the stall test needs 1e-6; the final value (the inverse
            // iteration's shift) the full FP32 resolution
            theta = tri_min<float>(R.al, R.be2, j + 1, lo, hi, h, last ? tri_rel<float>() : 1e-6f);
            if (last) { ++j; break; }
            // one stall over 16 steps, then extra32 steps more
            if (ritz32_stalled(theta, theta_prev, a.tol32)) {
              settled = true;
              kend = j + 1 + a.extra32 < kk ? j + 1 + a.extra32 : kk;
            }
            theta_pp = theta_prev;
            theta_prev = theta;
          }
        } else {
          m = R.mm[j];
          bn = R.bn[j + 1];
          __syncwarp();   // every lane has read the shared copy of q_j
        }
        const float2 ib = bcast2(1.f / bn), mm = bcast2(m);
        const float2 si = bcast2(pass ? R.s[j + 1] : 0.f), ti = bcast2(pass ? R.s2[j + 1] : 0.f);
        static_for<L>([&](auto KC) {
          constexpr int K = decltype(KC)::value;
          vp[K] = v[K];
          v[K] = __fmul2_rn(fsub2(z[K], mm), ib);
          if (pass) {
            y[K] = __ffma2_rn(si, v[K], y[K]);
            sts_f2<K * 256>(s_y2, __ffma2_rn(ti, v[K], lds_f2<K * 256>(s_y2)));
          }
          sts_f1<K * SV>(s_v + 4u * h, v[K].x);
          sts_f1<K * SV>(s_v + 4u * (NLH + h), v[K].y);
        });
        b = bn;
        __syncwarp();
      }
      if (pass == 0) {
        k = j;
        steps += k;
        // eigenvectors of T_k for its two smallest eigenvalues (lane 0)
        if (h == 0) ritz_coeffs32(R.al, R.bn, k, theta, R.pd, R.pl, R.s, R.s2);
        __syncwarp();
      }
    }
    __syncwarp();   // the FP32 record shares bytes with the FP64 vector and tridiagonal

    // ---- FP64: the diagonal of M, and the seed y off the constant mode, normalised ----
    double Dg[2][L], vd[2][L], vpd[2][L];
    double ysum = 0.0;
    static_for<2>([&](auto PC) {
      constexpr int P = decltype(PC)::value;
      const unsigned wo = s_w + 8u * (P * NLH + h);
      static_for<L>([&](auto KC) {
        constexpr int K = decltype(KC)::value;
        double dsum = 0.0;
        static_for<D>([&](auto MC) {
          constexpr int mu = decltype(MC)::value;
          const double wfo = lds_d1<(K * D + mu) * SW>(wo);
          double wbk;
          if constexpr (mu == 0) wbk = lds_d1<(((K + L - 1) % L) * D) * SW>(wo);
          else wbk = lds_d1<(K * D + mu) * SW>(s_w + 8u * em[P][mu]);
          dsum -= wfo + wbk;
        });
        Dg[P][K] = dsum;
        vd[P][K] = f2d_bits(P == 0 ? y[K].x : y[K].y);
        ysum += vd[P][K];
      });
    });
    ysum = warp_sum(ysum) / (double)V;
    double nn = 0.0;
    static_for<2>([&](auto PC) {
      static_for<L>([&](auto KC) {
        constexpr int P = decltype(PC)::value, K = decltype(KC)::value;
        vd[P][K] -= ysum;
        nn = fma(vd[P][K], vd[P][K], nn);
      });
    });
    {
      const double inv = rsqrt64(warp_sum(nn));
      static_for<2>([&](auto PC) {
        static_for<L>([&](auto KC) {
          constexpr int P = decltype(PC)::value, K = decltype(KC)::value;
          vd[P][K] *= inv;
        });
      });
    }
    // FP64 Rayleigh-Ritz on span{y, y2} (as rayleigh_ritz2_64): y2 off the
    // constant mode and off y, then the 2 x 2 projection of M
    {
      double s2m = 0.0;
      static_for<L>([&](auto KC) {
        constexpr int K = decltype(KC)::value;
        const float2 t = lds_f2<K * 256>(s_y2);
        vpd[0][K] = f2d_bits(t.x);
        vpd[1][K] = f2d_bits(t.y);
        s2m += vpd[0][K] + vpd[1][K];
      });
      s2m = warp_sum(s2m) / (double)V;
      double pr = 0.0, q2 = 0.0;
      static_for<2>([&](auto PC) {
        static_for<L>([&](auto KC) {
          constexpr int P = decltype(PC)::value, K = decltype(KC)::value;
          vpd[P][K] -= s2m;
          pr = fma(vd[P][K], vpd[P][K], pr);
          q2 = fma(vpd[P][K], vpd[P][K], q2);
        });
      });
      warp_sum2(pr, q2, h);
      const double r2 = fma(-pr, pr, q2);
      if (r2 > 1e-12 * q2) {
        const double ir = rsqrt64(r2);
        static_for<2>([&](auto PC) {
          static_for<L>([&](auto KC) {
            constexpr int P = decltype(PC)::value, K = decltype(KC)::value;
            vpd[P][K] = fma(-pr, vd[P][K], vpd[P][K]) * ir;
          });
        });
        double a11 = 0.0, a12 = 0.0, a22 = 0.0;
#pragma unroll 1
        for (int t = 0; t < 2; ++t) {
          double sr[2][L];
          static_for<2>([&](auto PC) {
            static_for<L>([&](auto KC) {
              constexpr int P = decltype(PC)::value, K = decltype(KC)::value;
              sr[P][K] = t ? vpd[P][K] : vd[P][K];
              sts_d1<K * SG>(s_v + 8u * (P * NLH + h), sr[P][K]);
            });
          });
          __syncwarp();
          double d1 = 0.0, d2 = 0.0;
          static_for<2>([&](auto PC) {
            constexpr int P = decltype(PC)::value;
            const unsigned wo = s_w + 8u * (P * NLH + h);
            static_for<L>([&](auto KC) {
              constexpr int K = decltype(KC)::value;
              double yv = Dg[P][K] * sr[P][K];
              static_for<D>([&](auto MC) {
                constexpr int mu = decltype(MC)::value;
                if constexpr (mu == 0) {
                  yv = fma(lds_d1<(K * D) * SW>(wo), sr[P][(K + 1) % L], yv);
                  yv = fma(lds_d1<(((K + L - 1) % L) * D) * SW>(wo), sr[P][(K + L - 1) % L], yv);
                } else {
                  yv = fma(lds_d1<(K * D + mu) * SW>(wo), lds_d1<K * SG>(s_v + 8u * ep[P][mu]), yv);
                  yv = fma(lds_d1<(K * D + mu) * SW>(s_w + 8u * em[P][mu]), lds_d1<K * SG>(s_v + 8u * em[P][mu]), yv);
                }
              });
              d1 = fma(vd[P][K], yv, d1);
              d2 = fma(vpd[P][K], yv, d2);
            });
          });
          warp_sum2(d1, d2, h);
          if (t == 0) { a11 = d1; a12 = d2; } else { a22 = d2; }
          __syncwarp();
        }
        double cs, sn;
        rr2_rotation(a11, a12, a22, &cs, &sn);
        static_for<2>([&](auto PC) {
          static_for<L>([&](auto KC) {
            constexpr int P = decltype(PC)::value, K = decltype(KC)::value;
            vd[P][K] = fma(cs, vd[P][K], sn * vpd[P][K]);
          });
        });
      }
      static_for<2>([&](auto PC) {
        static_for<L>([&](auto KC) {
          constexpr int P = decltype(PC)::value, K = decltype(KC)::value;
          vpd[P][K] = 0.0;
          sts_d1<K * SG>(s_v + 8u * (P * NLH + h), vd[P][K]);
        });
      });
    }
    __syncwarp();
    // ---- FP64 Lanczos from the seed (the step and stopping rule of lanczos64_seeded) ----
    const double invV = 1.0 / (double)V;
    const double dbound = (double)(4 * D + 1);
    double t64 = dbound, d64 = 0.0, b = 0.0;
    int st64 = 0, j64 = 0;
    const int kk64 = V - 1 < kmax64 ? V - 1 : kmax64;
    for (; j64 < kk64; ++j64) {
      double z[2][L], av = 0.0;
      const double mb = -b;
      static_for<2>([&](auto PC) {
        constexpr int P = decltype(PC)::value;
        const unsigned wo = s_w + 8u * (P * NLH + h);
        static_for<L>([&](auto KC) {
          constexpr int K = decltype(KC)::value;
          const double vx = vd[P][K];
          double yv = fma(Dg[P][K], vx, mb * vpd[P][K]);
          static_for<D>([&](auto MC) {
            constexpr int mu = decltype(MC)::value;
            if constexpr (mu == 0) {
              yv = fma(lds_d1<(K * D) * SW>(wo), vd[P][(K + 1) % L], yv);
              yv = fma(lds_d1<(((K + L - 1) % L) * D) * SW>(wo), vd[P][(K + L - 1) % L], yv);
            } else {
              yv = fma(lds_d1<(K * D + mu) * SW>(wo), lds_d1<K * SG>(s_v + 8u * ep[P][mu]), yv);
              yv = fma(lds_d1<(K * D + mu) * SW>(s_w + 8u * em[P][mu]), lds_d1<K * SG>(s_v + 8u * em[P][mu]), yv);
            }
          });
          z[P][K] = yv;
          av = fma(yv, vx, av);
        });
      });
      av = warp_sum(av);
      double m = 0.0, zz = 0.0;
      static_for<2>([&](auto PC) {
        static_for<L>([&](auto KC) {
          constexpr int P = decltype(PC)::value, K = decltype(KC)::value;
          z[P][K] = fma(-av, vd[P][K], z[P][K]);
          m += z[P][K];
          zz = fma(z[P][K], z[P][K], zz);
        });
      });
      warp_sum2(m, zz, h);
      m *= invV;
      double bn2 = fma(-(double)V * m, m, zz);   // |z - m|^2
      if (__double_as_longlong(bn2) < 0) bn2 = 0.0;
      if (h == 0) { a64[j64] = av; b64[j64 + 1] = bn2; }
      __syncwarp();
      const bool last = (j64 + 1 == kk64) || dbelow(bn2, 1e-24);
      double t;
      if (j64 == 0) {
        t = av;
      } else {
        // brackets tried in turn (one call site, so the multisection is
        // compiled once): the warm window below the last value, a window
        // around the FP32 Ritz value, then the Gershgorin interval
        bool ok = false, near = true;
        double lo = t64 - fmax(8.0 * d64, 4e-5 * fmax(fabs(t64), 1e-3));
        double hi = t64 + 1e-14 * fmax(fabs(t64), 1.0);
#pragma unroll 1
        for (int attempt = 0;; ++attempt) {
          t = tri_min64(a64, b64, j64 + 1, lo, hi, h, &ok, near);
          if (ok || attempt == 2) break;
          near = false;
          if (attempt == 0) {
            const double c = f2d_bits(theta);
            const double del = 2e-5 * fmax(1.0, fabs(c));
            lo = fmin(c, t64) - del;
            hi = t64 + del;
          } else {
            lo = -dbound;
            hi = dbound;
          }
        }
      }
      const bool stall = j64 > 0 && fabs(t - t64) <= a.tol64 * fmax(fabs(t), 1e-3);
      d64 = j64 > 0 ? fmax(t64 - t, 0.0) : 0.0;
      t64 = t;
      if (last) { ++j64; break; }
      if (stall) {
        if (++st64 == 2) { ++j64; break; }
      } else {
        st64 = 0;
      }
      const double ib = rsqrt64(bn2);
      const double mib = -m * ib;
      static_for<2>([&](auto PC) {
        static_for<L>([&](auto KC) {
          constexpr int P = decltype(PC)::value, K = decltype(KC)::value;
          vpd[P][K] = vd[P][K];
          vd[P][K] = fma(z[P][K], ib, mib);
          sts_d1<K * SG>(s_v + 8u * (P * NLH + h), vd[P][K]);
        });
      });
      b = bn2 * ib;
      __syncwarp();
    }
    steps += j64;
    steps64 += j64;
    if (h == 0) {
      a.lambda2[e] = t64;
      a.region[e] = region_of(t64, a.tau);
    }
    ++c_tests;
    __syncwarp();
  }
  if (h == 0 && c_tests) {
    if (a.count_tests) atomicAdd(&a.stats[13], c_tests);
    atomicAdd(&a.stats[14], c_tests);
    atomicAdd(&a.stats[15], (unsigned long long)steps);
    atomicAdd(&a.stats[24], (unsigned long long)steps64);
  }
}

}  // namespace gc
