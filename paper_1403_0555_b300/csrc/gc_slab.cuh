// Lattices beyond shared memory: each start's state lives in global memory and
// one CTA streams it through shared memory in hyperplanes (slabs) of constant
// x_{d-1}, moved by the bulk-copy (TMA) engine.
//
// A colour phase walks the planes z = 0 .. L-1 with a ring of three plane
// buffers (z-1, z, z+1): the colour-c sites of plane z read their neighbours
// along axes 0 .. d-2 from plane z's buffer and along axis d-1 from the
// neighbouring planes' buffers; plane z is then written back with one bulk
// store.  Sites of one colour never read each other, so within a phase the
// planes are independent: the ring can reload plane 0 at the end of the walk
// (it is needed as plane L-1's upper neighbour) in whichever of its two
// versions, because the colour that phase reads is unchanged.  A phase ends
// when its stores are complete; the next phase's loads then see them.
//
// Per sweep and start the state is read twice and written once (one load and
// one store of every plane per colour phase, each store holding the whole
// plane); the links are shared by every start of the orbit and stay in L2.  So
// with many starts in flight the sweeps are bound by HBM bandwidth.
//
// The residual is a separate read-only walk every check_every sweeps (the
// state after the sweep), so the checked state is the state kept.  The FP64
// site update is the oracle's operation for operation, hence the plain path is
// bit-exact to it start by start; the FP32 update is the FP32 bulk kernel's.
//
// Every wait on a bulk copy is bounded: when one runs out the kernel sets
// err[3], lets the copies in flight finish (bounded again) and returns.
#pragma once
#include "gc_relax.cuh"

namespace gc {

struct SlabArgs {
  int d, L, V, P;                  // P = V / L sites per plane
  const void* links;               // double2 or float2 [x*d + mu], site order
  void* state;                     // n * V elements (site order), this batch
  long long n;                     // starts in this batch
  uint64_t seed, orbit_id, start0;
  int init;                        // 1: generate the random start; 0: continue from state
  unsigned long long* work_ctr;
  double omega, om1, eps;          // FP64 update
  float omega32, om1_32, eps32;    // FP32 update
  int check_every, max_sweeps;
  int8_t* status;
  int32_t* sweeps;                 // init: set; continue: add
  double* resid;
  unsigned long long* stats;
  int s_sweeps, s_updates, s_conv, s_nconv;   // stats slots (-1: none)
  int* err;                        // [3] a bulk-copy wait ran out
};

// -- bulk copies and barriers (PTX) ------------------------------------------
__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
               "selp.u32 %0, 1, 0, p;\n\t}"
               : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
  return ok != 0;
}
// bounded: true when the phase completed
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
  for (long long i = 0; i < (1LL << 24); ++i)
    if (mbar_try(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void bulk_load(unsigned dst, const void* src, unsigned bytes, unsigned bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}
__device__ __forceinline__ void bulk_store(void* dst, unsigned src, unsigned bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;"
               ::"l"(dst), "r"(src), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_read_1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// -- the site update in each precision ----------------------------------------
template <class E> struct SlabOps;
template <> struct SlabOps<double2> {
  using R = double;
  // S in the order mu = 0..d-1, forward term then backward term (the oracle's)
  static __device__ __forceinline__ void acc_fwd(double2& S, double2 u, double2 h) {
    const double2 t = Exact64::mul(u, h);
    S.x = __dadd_rn(S.x, t.x); S.y = __dadd_rn(S.y, t.y);
  }
  static __device__ __forceinline__ void acc_bwd(double2& S, double2 u, double2 h) {
    const double2 t = Exact64::cmul(u, h);
    S.x = __dadd_rn(S.x, t.x); S.y = __dadd_rn(S.y, t.y);
  }
  static __device__ __forceinline__ double2 zero() { return make_double2(0.0, 0.0); }
  static __device__ __forceinline__ double2 move(double2 gx, double2 S, const SlabArgs& a) {
    const double n2 = __dadd_rn(__dmul_rn(S.x, S.x), __dmul_rn(S.y, S.y));
    if (!(n2 > 0.0)) return gx;
    const double r = __drcp_rn(__dsqrt_rn(n2));
    const double hx = __dmul_rn(S.x, r), hy = __dmul_rn(S.y, r);
    const double vx = __dadd_rn(__dmul_rn(a.om1, gx.x), __dmul_rn(a.omega, hx));
    const double vy = __dadd_rn(__dmul_rn(a.om1, gx.y), __dmul_rn(a.omega, hy));
    const double m2 = __dadd_rn(__dmul_rn(vx, vx), __dmul_rn(vy, vy));
    if (!(m2 > 0.0)) return make_double2(hx, hy);
    const double q = __drcp_rn(__dsqrt_rn(m2));
    return make_double2(__dmul_rn(vx, q), __dmul_rn(vy, q));
  }
  static __device__ __forceinline__ double div2(double2 gx, double2 S) {
    const double dv = __dsub_rn(__dmul_rn(gx.x, S.y), __dmul_rn(gx.y, S.x));
    return __dmul_rn(dv, dv);
  }
  static __device__ __forceinline__ double eps(const SlabArgs& a) { return a.eps; }
  static __device__ __forceinline__ double2 start(const SlabArgs& a, long long idx, int x) {
    return random_unit(a.seed, a.orbit_id, a.start0 + (uint64_t)idx, (uint64_t)x);
  }
};
template <> struct SlabOps<float2> {
  using R = float;
  static __device__ __forceinline__ void acc_fwd(float2& S, float2 u, float2 h) {
    S.x = fmaf(u.x, h.x, S.x); S.x = fmaf(-u.y, h.y, S.x);
    S.y = fmaf(u.x, h.y, S.y); S.y = fmaf(u.y, h.x, S.y);
  }
  static __device__ __forceinline__ void acc_bwd(float2& S, float2 u, float2 h) {
    S.x = fmaf(u.x, h.x, S.x); S.x = fmaf(u.y, h.y, S.x);
    S.y = fmaf(u.x, h.y, S.y); S.y = fmaf(-u.y, h.x, S.y);
  }
  static __device__ __forceinline__ float2 zero() { return make_float2(0.f, 0.f); }
  static __device__ __forceinline__ float2 move(float2 gx, float2 S, const SlabArgs& a) {
    const float n2 = fmaf(S.x, S.x, S.y * S.y);
    if (!(n2 > 1e-30f)) return gx;   // a vanishing staple leaves the site as it is
    const float r = rsqrt_sfu(n2) * a.omega32;
    const float vx = fmaf(S.x, r, a.om1_32 * gx.x), vy = fmaf(S.y, r, a.om1_32 * gx.y);
    const float m2 = fmaf(vx, vx, vy * vy);
    if (!(m2 > 1e-30f)) return gx;
    const float q = rsqrt_sfu(m2);
    return make_float2(vx * q, vy * q);
  }
  static __device__ __forceinline__ float div2(float2 gx, float2 S) {
    const float dv = fmaf(gx.x, S.y, -gx.y * S.x);
    return dv * dv;
  }
  static __device__ __forceinline__ float eps(const SlabArgs& a) { return a.eps32; }
  static __device__ __forceinline__ float2 start(const SlabArgs& a, long long idx, int x) {
    return random_unit32(a.seed, a.orbit_id, a.start0 + (uint64_t)idx, (uint64_t)x);
  }
};

// shared memory: 3 barriers and scratch in the first 512 bytes, then the ring
__host__ __device__ inline size_t slab_smem_bytes(int P, int elem) { return 512 + 3 * (size_t)P * elem; }

template <class E, int D>
__global__ void __launch_bounds__(512) relax_slab_kernel(const SlabArgs a) {
  using Ops = SlabOps<E>;
  using R = typename Ops::R;
  extern __shared__ __align__(16) unsigned char smem[];
  const int L = a.L, V = a.V, P = a.P, tid = threadIdx.x, nt = blockDim.x;
  const unsigned PB = (unsigned)(P * sizeof(E));
  const unsigned sbase = (unsigned)__cvta_generic_to_shared(smem);
  const unsigned bar0 = sbase;                           // 3 x 8 bytes
  long long* tidx = reinterpret_cast<long long*>(smem + 32);
  int* abort_flag = reinterpret_cast<int*>(smem + 40);
  R* red = reinterpret_cast<R*>(smem + 64);              // per-warp partials (<= 16 warps)
  E* ring = reinterpret_cast<E*>(smem + 512);
  const unsigned ring_s = sbase + 512;
  const E* links = static_cast<const E*>(a.links);
  const int H = L / 2;                                   // colour sites per row

  if (tid == 0) {
    for (int k = 0; k < 3; ++k) mbar_init(bar0 + 8u * k, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  unsigned parity = 0;                                   // bit k: next phase parity of barrier k
  unsigned long long my_sweeps = 0, my_conv = 0, my_nconv = 0;

  // load k of a walk (plane (k - 1) mod L into slot k mod 3); thread 0 only
  auto issue = [&](const E* st, int k) {
    const int slot = k % 3, z = (k - 1 + L) % L;
    mbar_expect(bar0 + 8u * slot, PB);
    bulk_load(ring_s + (unsigned)slot * PB, st + (size_t)z * P, PB, bar0 + 8u * slot);
  };
  // every thread waits for load k; false when the wait ran out
  auto await = [&](int k) -> bool {
    const int slot = k % 3;
    const bool ok = mbar_wait(bar0 + 8u * slot, (parity >> slot) & 1u);
    parity ^= 1u << slot;
    return ok;
  };
  auto fail = [&]() {
    if (tid == 0) { atomicExch(&a.err[3], 1); *abort_flag = 1; }
  };
  // the staple of in-plane site j of plane z (buffers: prev, cur, next)
  auto staple = [&](const E* prev, const E* cur, const E* next, int z, int j, int x0, int rowbase) -> E {
    E S = Ops::zero();
    const int x = z * P + j;
    int stride = 1;
#pragma unroll
    for (int mu = 0; mu < D; ++mu) {
      E hp, hm;
      int xm;
      if (mu == 0) {
        const int jp = rowbase + (x0 + 1 == L ? 0 : x0 + 1), jm = rowbase + (x0 == 0 ? L - 1 : x0 - 1);
        hp = cur[jp]; hm = cur[jm];
        xm = z * P + jm;
      } else if (mu < D - 1) {
        const int c = (j / stride) % L;
        const int jp = j + (c + 1 == L ? -(L - 1) * stride : stride);
        const int jm = j + (c == 0 ? (L - 1) * stride : -stride);
        hp = cur[jp]; hm = cur[jm];
        xm = z * P + jm;
      } else {
        hp = next[j]; hm = prev[j];
        xm = (z == 0 ? L - 1 : z - 1) * P + j;
      }
      Ops::acc_fwd(S, __ldg(links + (size_t)x * D + mu), hp);
      Ops::acc_bwd(S, __ldg(links + (size_t)xm * D + mu), hm);
      stride *= L;
    }
    return S;
  };
  // in-plane coordinates of the h-th colour-c site of plane z
  auto site_of = [&](int h, int c, int z, int& j, int& x0, int& rowbase) {
    const int row = h / H, k = h - row * H;
    int rs = 0, t = row;
#pragma unroll
    for (int mu = 1; mu < D - 1; ++mu) { rs += t % L; t /= L; }
    x0 = 2 * k + ((c + z + rs) & 1);
    rowbase = row * L;
    j = rowbase + x0;
  };
  // one colour phase over the whole lattice; false when a wait ran out
  auto phase = [&](E* st, int c) -> bool {
    if (tid == 0) { issue(st, 0); issue(st, 1); issue(st, 2); }
    bool ok = await(0);
    ok = await(1) && ok;
    ok = !__syncthreads_or(!ok);   // the same on every thread before the walk's barriers
    for (int z = 0; z < L && ok; ++z) {
      ok = await(z + 2);
      if (__syncthreads_or(!ok)) { ok = false; break; }
      const E* prev = ring + (size_t)(z % 3) * P;
      E* cur = ring + (size_t)((z + 1) % 3) * P;
      const E* next = ring + (size_t)((z + 2) % 3) * P;
      for (int h = tid; h < P / 2; h += nt) {
        int j, x0, rowbase;
        site_of(h, c, z, j, x0, rowbase);
        cur[j] = Ops::move(cur[j], staple(prev, cur, next, z, j, x0, rowbase), a);
      }
      fence_async_smem();
      __syncthreads();
      if (tid == 0) {
        bulk_store(st + (size_t)z * P, ring_s + (unsigned)((z + 1) % 3) * PB, PB);
        if (z + 3 <= L + 1) {
          bulk_wait_read_1();   // the store of step z-1 (slot z mod 3) has read its buffer
          issue(st, z + 3);
        }
      }
    }
    if (tid == 0) bulk_wait_all();
    return !__syncthreads_or(!ok);
  };
  // max div^2 over the lattice (read-only walk); nan when a wait ran out
  auto residual = [&](const E* st, bool& ok) -> R {
    R r = 0;
    if (tid == 0) { issue(st, 0); issue(st, 1); issue(st, 2); }
    ok = await(0);
    ok = await(1) && ok;
    ok = !__syncthreads_or(!ok);
    for (int z = 0; z < L && ok; ++z) {
      ok = await(z + 2);
      if (__syncthreads_or(!ok)) { ok = false; break; }
      const E* prev = ring + (size_t)(z % 3) * P;
      const E* cur = ring + (size_t)((z + 1) % 3) * P;
      const E* next = ring + (size_t)((z + 2) % 3) * P;
      for (int j = tid; j < P; j += nt) {
        const int x0 = j % L, rowbase = j - x0;
        const R v = Ops::div2(cur[j], staple(prev, cur, next, z, j, x0, rowbase));
        r = v > r ? v : r;
      }
      __syncthreads();   // slot z mod 3 is free
      if (tid == 0 && z + 3 <= L + 1) issue(st, z + 3);
    }
    ok = !__syncthreads_or(!ok);
    for (int o = 16; o > 0; o >>= 1) {
      const R w = __shfl_xor_sync(0xffffffffu, r, o);
      r = w > r ? w : r;
    }
    if ((tid & 31) == 0) red[tid >> 5] = r;
    __syncthreads();
    r = 0;
    for (int w = 0; w < nt / 32; ++w) r = red[w] > r ? red[w] : r;
    __syncthreads();
    return r;
  };

  for (;;) {
    if (tid == 0) *tidx = (long long)atomicAdd(a.work_ctr, 1ULL);
    __syncthreads();
    const long long idx = *tidx;
    __syncthreads();
    if (idx >= a.n || *abort_flag) break;
    E* st = static_cast<E*>(a.state) + (size_t)idx * V;
    if (a.init) {
      for (int x = tid; x < V; x += nt) st[x] = Ops::start(a, idx, x);
      fence_async_global();   // generic writes, then bulk reads of them
      __syncthreads();
    }
    int sweeps = 0, until = a.check_every;
    bool ok = true, conv = false;
    R r = 0;
    for (;;) {
      if (!phase(st, 0) || !phase(st, 1)) { ok = false; break; }
      ++sweeps;
      if (--until == 0) {
        until = a.check_every;
        r = residual(st, ok);
        if (!ok) break;
        conv = r < Ops::eps(a);
        if (conv || sweeps >= a.max_sweeps) break;
      }
    }
    if (!ok) {
      // a wait ran out: flag it, give the loads still in flight a bounded
      // time to land in their buffers, and stop
      fail();
      for (int k = 0; k < 3; ++k) mbar_wait(bar0 + 8u * k, (parity >> k) & 1u);
      if (tid == 0) bulk_wait_all();
      __syncthreads();
      break;
    }
    if (tid == 0) {
      a.status[idx] = conv ? kConverged : kNotConverged;
      if (a.init) a.sweeps[idx] = sweeps; else a.sweeps[idx] += sweeps;
      if (sizeof(R) == 8) a.resid[idx] = (double)r;
      my_sweeps += sweeps;
      if (conv) ++my_conv; else ++my_nconv;
    }
  }
  if (tid == 0) {
    if (a.s_sweeps >= 0) atomicAdd(&a.stats[a.s_sweeps], my_sweeps);
    if (a.s_updates >= 0) atomicAdd(&a.stats[a.s_updates], my_sweeps * (unsigned long long)V);
    if (a.s_conv >= 0) atomicAdd(&a.stats[a.s_conv], my_conv);
    if (a.s_nconv >= 0) atomicAdd(&a.stats[a.s_nconv], my_nconv);
  }
}

// FP32 state -> FP64, renormalised (the mixed path's hand-over to the FP64 sweeps)
__global__ void slab_promote_kernel(const float2* s32, double2* s64, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double x = s32[i].x, y = s32[i].y;
    const double q = 1.0 / sqrt(x * x + y * y);
    s64[i] = make_double2(x * q, y * q);
  }
}

// One CTA per start: the functional (Eq. 3), the fingerprint cos(phi^theta)
// of link (site 0, mu 0) and, in place, the canonical copy g'_x = g_x conj(g_{V-1})
__global__ void __launch_bounds__(256) slab_final_kernel(double2* state, const double2* links, int d, int V,
                                                         int L, long long n, double* F, double* fprint) {
  __shared__ double red[32];
  for (long long i = blockIdx.x; i < n; i += gridDim.x) {
    double2* g = state + (size_t)i * V;
    double Fp = 0.0;
    for (int x = threadIdx.x; x < V; x += blockDim.x) {
      const double2 gx = g[x];
      int stride = 1;
      for (int mu = 0; mu < d; ++mu) {
        const int c = (x / stride) % L;
        const int xp = x + (c + 1 == L ? -(L - 1) * stride : stride);
        const double2 h = g[xp], u = links[(size_t)x * d + mu];
        const double tx = u.x * h.x - u.y * h.y, ty = u.x * h.y + u.y * h.x;
        const double w = gx.x * tx + gx.y * ty;   // Re[conj(g_x) u g_{x+mu}]
        Fp += 1.0 - w;
        if (x == 0 && mu == 0) fprint[i] = w;
        stride *= L;
      }
    }
    for (int o = 16; o > 0; o >>= 1) Fp += __shfl_xor_sync(0xffffffffu, Fp, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = Fp;
    const double2 gc = g[V - 1];
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
      F[i] = t;
    }
    for (int x = threadIdx.x; x < V; x += blockDim.x) {
      const double2 gx = g[x];
      g[x] = make_double2(gx.x * gc.x + gx.y * gc.y, gx.y * gc.x - gx.x * gc.y);
    }
    __syncthreads();
  }
}

// First-region fast path for the copies a batch created: all weights
// cos(phi^theta) > 0 make the Faddeev-Popov operator a weighted graph
// Laplacian with positive weights, so lambda_2 > 0 (region IN); otherwise the
// copy is left untested (-1).  lambda_2 itself is not computed (NaN).
__global__ void __launch_bounds__(256) slab_fp_fast_kernel(const double2* cfg, const double2* links, int d,
                                                           int V, int L, const unsigned* list,
                                                           const unsigned* n_list, double* lambda2,
                                                           int* region, unsigned long long* tests) {
  __shared__ int neg;
  const unsigned n = *n_list;
  for (unsigned i = blockIdx.x; i < n; i += gridDim.x) {
    const unsigned e = list[i];
    const double2* g = cfg + (size_t)e * V;
    if (threadIdx.x == 0) neg = 0;
    __syncthreads();
    int mine = 0;
    for (int x = threadIdx.x; x < V && !mine; x += blockDim.x) {
      const double2 gx = g[x];
      int stride = 1;
      for (int mu = 0; mu < d; ++mu) {
        const int c = (x / stride) % L;
        const int xp = x + (c + 1 == L ? -(L - 1) * stride : stride);
        const double2 h = g[xp], u = links[(size_t)x * d + mu];
        const double w = gx.x * (u.x * h.x - u.y * h.y) + gx.y * (u.x * h.y + u.y * h.x);
        if (!(w > 0.0)) mine = 1;
        stride *= L;
      }
    }
    if (mine) atomicOr(&neg, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
      region[e] = neg ? -1 : 1;
      lambda2[e] = __longlong_as_double(0x7ff8000000000000LL);
      atomicAdd(tests, 1ULL);
    }
    __syncthreads();
  }
}

}  // namespace gc
