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

}  // namespace gc
