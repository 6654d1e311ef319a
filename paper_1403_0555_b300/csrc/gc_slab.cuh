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
// plane); the links are shared by every start of the orbit and stay in L2.
// With the starts in flight beyond L2 the sweeps would be bound by HBM
// bandwidth; one start per cluster keeps few in flight, and L2 serves them.
//
// The residual is a separate read-only walk every check_every sweeps (the
// state after the sweep), so the checked state is the state kept.  The FP64
// site update is the oracle's operation for operation, hence the plain path is
// bit-exact to it start by start; the FP32 update is the FP32 bulk kernel's.
//
// Every wait on a bulk copy is bounded: when one runs out the kernel sets
// err[3], lets the copies in flight finish (bounded again) and returns.
//
// Also here, for the same lattices: the FP32 sweeps with the lattice held in a
// cluster's distributed shared memory (relax_dsmem_kernel), the inexact Newton
// polish of the mixed path (slab_newton_kernel), the functional and canonical
// copy (slab_final_kernel) and the first-region test by Lanczos with vectors
// in global memory (slab_fp_lanczos_kernel).
#pragma once
#include <cooperative_groups.h>
#include "gc_fptest.cuh"
#include "gc_relax.cuh"

namespace cg = cooperative_groups;

namespace gc {

struct SlabArgs {
  int d, L, V, P;                  // P = V / L sites per plane
  const void* links;               // double2 or float2 [x*d + mu], site order
  void* state;                     // n * V elements (site order), this batch
  long long n;                     // starts in this batch
  uint64_t seed, orbit_id, start0;
  int init;                        // 1: generate the random start; 0: continue from state
  unsigned long long* work_ctr;
  const unsigned* list;            // when set: only these batch entries, *n_list of them
  const unsigned* n_list;
  double omega, om1, eps;          // FP64 update
  float omega32, om1_32, eps32;    // FP32 update
  int check_every, max_sweeps;
  int8_t* status;
  int32_t* sweeps;                 // init: set; continue: add
  double* resid;
  float* rate;                     // when set: per start, the contraction of max |div| per sweep
                                   // over the last check interval (0: none seen)
  const float* omega_rate;         // when set (FP64 polish of hard starts): per start the
                                   // contraction its FP32 sweeps showed at omega32; the sweeps
                                   // then run at Young's parameter for it (young_omega)
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

// -- the three-plane ring ------------------------------------------------------
// A walk over n consecutive planes z0 .. z0+n-1 (mod L) of one start's array
// (plane z at base + z * Ps elements) with three shared-memory plane buffers:
// load k brings plane z0 + k - 1 (mod L) into slot k mod 3, so step t sees
// planes z-1, z and z+1 (z = z0 + t) in slots t, t+1 and t+2 (mod 3).
// Thread 0 issues; every thread awaits.
template <class E>
struct PlaneRing {
  E* ring;                 // 3 * Ps elements
  unsigned ring_s, bar0;   // shared-window addresses of the ring and of 3 barriers
  unsigned PB;             // bytes per plane (a multiple of 16)
  int L, Ps;
  unsigned parity;         // bit k: the next phase parity of barrier k

  __device__ void issue(const E* base, int z0, int k) {
    const int slot = k % 3, z = (z0 + k - 1 + L) % L;
    mbar_expect(bar0 + 8u * slot, PB);
    bulk_load(ring_s + (unsigned)slot * PB, base + (size_t)z * Ps, PB, bar0 + 8u * slot);
  }
  // false when the wait ran out
  __device__ bool await(int k) {
    const int slot = k % 3;
    const bool ok = mbar_wait(bar0 + 8u * slot, (parity >> slot) & 1u);
    parity ^= 1u << slot;
    return ok;
  }
  __device__ E* plane(int k) const { return ring + (size_t)(k % 3) * Ps; }
  __device__ unsigned plane_s(int k) const { return ring_s + (unsigned)(k % 3) * PB; }
  // after a failed walk: give the loads still in flight a bounded time to land
  __device__ void drain() {
    for (int k = 0; k < 3; ++k) mbar_wait(bar0 + 8u * k, (parity >> k) & 1u);
  }
};

// One walk: body(prev, cur, next, z) on every thread for z = z0 .. z0+n-1
// (n >= 1); with `store` each plane goes back to global memory after its body
// (so the walk updates the array in place: within a walk the body must only
// write sites that no other plane's body reads, e.g. one colour).  Returns the
// same value on every thread: false when a wait ran out.
template <class E, class Body>
__device__ __forceinline__ bool ring_walk(PlaneRing<E>& R, E* base, bool store, Body&& body, int z0, int n) {
  const int tid = threadIdx.x;
  if (tid == 0) { R.issue(base, z0, 0); R.issue(base, z0, 1); R.issue(base, z0, 2); }
  bool ok = R.await(0);
  ok = R.await(1) && ok;
  ok = !__syncthreads_or(!ok);   // the same on every thread before the walk's barriers
  for (int t = 0; t < n && ok; ++t) {
    const int z = z0 + t;
    ok = R.await(t + 2);
    if (__syncthreads_or(!ok)) { ok = false; break; }
    body(static_cast<const E*>(R.plane(t)), R.plane(t + 1), static_cast<const E*>(R.plane(t + 2)), z);
    if (store) fence_async_smem();
    __syncthreads();   // slot t mod 3 is free (read-only walk); plane z is complete (store)
    if (tid == 0) {
      if (store) {
        bulk_store(base + (size_t)z * R.Ps, R.plane_s(t + 1), R.PB);
        if (t + 3 <= n + 1) {
          bulk_wait_read_1();   // the store of step t-1 (slot t mod 3) has read its buffer
          R.issue(base, z0, t + 3);
        }
      } else if (t + 3 <= n + 1) {
        R.issue(base, z0, t + 3);
      }
    }
  }
  if (store && tid == 0) bulk_wait_all();
  return !__syncthreads_or(!ok);
}
template <class E, class Body>
__device__ __forceinline__ bool ring_walk(PlaneRing<E>& R, E* base, bool store, Body&& body) {
  return ring_walk(R, base, store, static_cast<Body&&>(body), 0, R.L);
}

// Overrelaxation parameter of one start's sweeps (both precisions' forms);
// `fast`: FP64 normalisation by rsqrt, for sweeps that need not follow the
// oracle's correctly rounded operations (the polish of hard starts)
struct SlabOmega {
  double om, om1;
  float om32, om1_32;
  bool fast;
};

// Young's relation for consistently ordered matrices (the red-black ordering
// of this stencil): SOR at parameter w < w_opt contracting by lam per sweep
// means a Jacobi radius mu^2 = (lam + w - 1)^2 / (lam w^2), and
// w_opt = 2 / (1 + sqrt(1 - mu^2)).  Returns w_opt plus a tenth of its
// distance to 2 (the rate degrades more slowly above w_opt than below), or w
// when lam says nothing (lam <= w - 1: w is at or above w_opt already).
__device__ __forceinline__ float young_omega(float lam, float w) {
  if (!(lam > w - 1.f && lam < 1.f)) return w;
  const float m2 = fminf((lam + w - 1.f) * (lam + w - 1.f) / (lam * w * w), 0.99999f);
  const float wopt = 2.f / (1.f + sqrtf(1.f - m2));
  return fminf(wopt + 0.1f * (2.f - wopt), 1.985f);
}

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
  static __device__ __forceinline__ double2 move(double2 gx, double2 S, const SlabOmega& a) {
    if (a.fast) {
      const double n2 = S.x * S.x + S.y * S.y;
      if (!(n2 > 0.0)) return gx;
      const double r = rsqrt(n2) * a.om;
      const double vx = fma(S.x, r, a.om1 * gx.x), vy = fma(S.y, r, a.om1 * gx.y);
      const double m2 = vx * vx + vy * vy;
      if (!(m2 > 0.0)) return gx;
      const double q = rsqrt(m2);
      return make_double2(vx * q, vy * q);
    }
    const double n2 = __dadd_rn(__dmul_rn(S.x, S.x), __dmul_rn(S.y, S.y));
    if (!(n2 > 0.0)) return gx;
    const double r = __drcp_rn(__dsqrt_rn(n2));
    const double hx = __dmul_rn(S.x, r), hy = __dmul_rn(S.y, r);
    const double vx = __dadd_rn(__dmul_rn(a.om1, gx.x), __dmul_rn(a.om, hx));
    const double vy = __dadd_rn(__dmul_rn(a.om1, gx.y), __dmul_rn(a.om, hy));
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
  static __device__ __forceinline__ float2 move(float2 gx, float2 S, const SlabOmega& a) {
    const float n2 = fmaf(S.x, S.x, S.y * S.y);
    if (!(n2 > 1e-30f)) return gx;   // a vanishing staple leaves the site as it is
    const float r = rsqrt_sfu(n2) * a.om32;
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

// In-plane coordinates of the h-th colour-c site of plane z (row = the
// coordinates 1 .. D-2, x0 = coordinate 0): j = in-plane index.
template <int D>
__device__ __forceinline__ void slab_site_of(int L, int h, int c, int z, int& j, int& x0, int& rowbase) {
  const int H = L / 2;
  const int row = h / H, k = h - row * H;
  int rs = 0, t = row;
#pragma unroll
  for (int mu = 1; mu < D - 1; ++mu) { rs += t % L; t /= L; }
  x0 = 2 * k + ((c + z + rs) & 1);
  rowbase = row * L;
  j = rowbase + x0;
}

// Neighbours of in-plane site j (coordinate 0 = x0, row start rowbase) along
// axis mu < D-1: in-plane indices jp (forward) and jm (backward).
template <int D>
__device__ __forceinline__ void slab_inplane_nb(int L, int mu, int j, int x0, int rowbase, int& jp, int& jm) {
  if (mu == 0) {
    jp = rowbase + (x0 + 1 == L ? 0 : x0 + 1);
    jm = rowbase + (x0 == 0 ? L - 1 : x0 - 1);
  } else {
    int stride = 1;
    for (int k = 0; k < mu; ++k) stride *= L;
    const int c = (j / stride) % L;
    jp = j + (c + 1 == L ? -(L - 1) * stride : stride);
    jm = j + (c == 0 ? (L - 1) * stride : -stride);
  }
}

// The sweeps.  CL = false: one CTA per start, starts pulled from a counter.
// CL = true: one start per thread-block cluster of C CTAs (the multi-CTA form
// for few or hard starts), CTA q walking planes [q L / C, (q+1) L / C): a
// colour phase reads only the other colour, so the CTAs' plane ranges are
// independent within a phase (a neighbour plane that another CTA is storing
// changes only in the bytes of the colour this CTA does not read); the CTAs
// meet at one cluster barrier per phase and per residual, which also carries
// their max div^2 and whether a wait ran out, so every CTA of a cluster takes
// the same decisions.
template <class E, int D, bool CL>
__global__ void __launch_bounds__(512) relax_slab_kernel(const SlabArgs a) {
  using Ops = SlabOps<E>;
  using R = typename Ops::R;
  extern __shared__ __align__(16) unsigned char smem[];
  const int L = a.L, V = a.V, P = a.P, tid = threadIdx.x, nt = blockDim.x;
  const unsigned sbase = (unsigned)__cvta_generic_to_shared(smem);
  long long* tidx = reinterpret_cast<long long*>(smem + 32);
  int* abort_flag = reinterpret_cast<int*>(smem + 40);
  R* red = reinterpret_cast<R*>(smem + 64);              // per-warp partials (<= 16 warps)
  double* cl_slots = reinterpret_cast<double*>(smem + 192);   // [2][16] cluster exchange (rank 0's)
  PlaneRing<E> ring{reinterpret_cast<E*>(smem + 512), sbase + 512, sbase, (unsigned)(P * sizeof(E)), L, P, 0u};
  const E* links = static_cast<const E*>(a.links);
  int C = 1, q = 0, cid = 0, ncl = 1;
  if constexpr (CL) {
    cg::cluster_group cl = cg::this_cluster();
    C = (int)cl.num_blocks();
    q = (int)cl.block_rank();
    cid = blockIdx.x / C;
    ncl = gridDim.x / C;
  }
  const int z0 = q * L / C, nz = (q + 1) * L / C - z0;   // this CTA's planes (nz may be 0)
  int round = 0;

  if (tid == 0) {
    for (int k = 0; k < 3; ++k) mbar_init(sbase + 8u * k, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if constexpr (CL) cg::this_cluster().sync();   // every CTA's barriers and slots exist
  unsigned long long my_sweeps = 0, my_conv = 0, my_nconv = 0;
  SlabOmega w{};   // this start's parameter

  // cluster-wide: max of r over the CTAs, ok = every CTA's ok (identity
  // without a cluster).  Double-buffered slots in rank 0: round k+2 writes
  // slot set k mod 2 only after every CTA passed barrier k+1, i.e. read round k.
  auto combine = [&](bool& ok, double r) -> double {
    if constexpr (!CL) {
      return r;
    } else {
      cg::cluster_group cl = cg::this_cluster();
      double* set = cl_slots + 16 * (round & 1);
      if (tid == 0) {
        fence_async_global();   // this CTA's completed bulk stores, before the release
        cl.map_shared_rank(set, 0)[q] = ok ? r : -1.0;
      }
      cl.sync();
      if (tid == 0) fence_async_global();   // then the next bulk loads
      const double* src = cl.map_shared_rank(set, 0);
      double m = 0.0;
      bool all = true;
      for (int k = 0; k < C; ++k) {
        const double v = src[k];
        if (v < 0.0) all = false; else m = fmax(m, v);
      }
      ok = all;
      ++round;
      return m;
    }
  };

  // the staple of in-plane site j of plane z (buffers: prev, cur, next)
  auto staple = [&](const E* prev, const E* cur, const E* next, int z, int j, int x0, int rowbase) -> E {
    E S = Ops::zero();
    const int x = z * P + j;
#pragma unroll
    for (int mu = 0; mu < D; ++mu) {
      E hp, hm;
      int xm;
      if (mu < D - 1) {
        int jp, jm;
        slab_inplane_nb<D>(L, mu, j, x0, rowbase, jp, jm);
        hp = cur[jp]; hm = cur[jm];
        xm = z * P + jm;
      } else {
        hp = next[j]; hm = prev[j];
        xm = (z == 0 ? L - 1 : z - 1) * P + j;
      }
      Ops::acc_fwd(S, __ldg(links + (size_t)x * D + mu), hp);
      Ops::acc_bwd(S, __ldg(links + (size_t)xm * D + mu), hm);
    }
    return S;
  };
  // one colour phase over this CTA's planes, then (cluster) the others';
  // false everywhere when a wait ran out anywhere
  auto phase = [&](E* st, int c) -> bool {
    bool ok = nz == 0 || ring_walk(ring, st, true, [&](const E* prev, E* cur, const E* next, int z) {
      for (int h = tid; h < P / 2; h += nt) {
        int j, x0, rowbase;
        slab_site_of<D>(L, h, c, z, j, x0, rowbase);
        cur[j] = Ops::move(cur[j], staple(prev, cur, next, z, j, x0, rowbase), w);
      }
    }, z0, nz);
    combine(ok, 0.0);
    return ok;
  };
  // max div^2 over the lattice (read-only walk)
  auto residual = [&](E* st, bool& ok) -> R {
    R r = 0;
    ok = nz == 0 || ring_walk(ring, st, false, [&](const E* prev, E* cur, const E* next, int z) {
      for (int j = tid; j < P; j += nt) {
        const int x0 = j % L, rowbase = j - x0;
        const R v = Ops::div2(cur[j], staple(prev, cur, next, z, j, x0, rowbase));
        r = v > r ? v : r;
      }
    }, z0, nz);
    for (int o = 16; o > 0; o >>= 1) {
      const R w = __shfl_xor_sync(0xffffffffu, r, o);
      r = w > r ? w : r;
    }
    if ((tid & 31) == 0) red[tid >> 5] = r;
    __syncthreads();
    r = 0;
    for (int w = 0; w < nt / 32; ++w) r = red[w] > r ? red[w] : r;
    __syncthreads();
    return (R)combine(ok, (double)r);
  };

  const long long n = a.list ? (long long)*a.n_list : a.n;
  for (long long i = cid;; i += ncl) {
    if constexpr (!CL) {
      if (tid == 0) *tidx = (long long)atomicAdd(a.work_ctr, 1ULL);
      __syncthreads();
      i = *tidx;
      __syncthreads();
      if (*abort_flag) break;
    }
    if (i >= n) break;
    const long long idx = a.list ? (long long)a.list[i] : i;
    E* st = static_cast<E*>(a.state) + (size_t)idx * V;
    bool ok = true;
    w = SlabOmega{a.omega, a.om1, a.omega32, a.om1_32, false};
    if (a.omega_rate) {   // the polish of hard starts: Young's parameter, rsqrt normalisation
      const float wy = young_omega(a.omega_rate[idx], a.omega32);
      w = SlabOmega{(double)wy, 1.0 - (double)wy, wy, 1.f - wy, true};
    }
    if (a.init) {
      for (int x = z0 * P + tid; x < (z0 + nz) * P; x += nt) st[x] = Ops::start(a, idx, x);
      fence_async_global();   // generic writes, then bulk reads of them
      __syncthreads();
      combine(ok, 0.0);       // (cluster) the neighbours' planes too
    }
    int sweeps = 0, until = a.check_every;
    bool conv = false;
    R r = 0, r_last = 0;
    for (;;) {
      if (!phase(st, 0) || !phase(st, 1)) { ok = false; break; }
      ++sweeps;
      if (--until == 0) {
        until = a.check_every;
        r_last = r;
        r = residual(st, ok);
        if (!ok) break;
        conv = r < Ops::eps(a);
        if (conv || sweeps >= a.max_sweeps) break;
      }
    }
    if (!ok) {
      // a wait ran out: flag it, let the loads still in flight land, and stop
      // (in a cluster every CTA gets here together)
      if (tid == 0) { atomicExch(&a.err[3], 1); *abort_flag = 1; }
      ring.drain();
      if (tid == 0) bulk_wait_all();
      __syncthreads();
      break;
    }
    if (tid == 0 && q == 0) {
      a.status[idx] = conv ? kConverged : kNotConverged;
      if (a.init) a.sweeps[idx] = sweeps; else a.sweeps[idx] += sweeps;
      if (sizeof(R) == 8) a.resid[idx] = (double)r;
      // the contraction of |div| per sweep over the last check interval
      if (a.rate) a.rate[idx] = (r_last > 0 && r < r_last) ? (float)pow((double)r / (double)r_last, 0.5 / a.check_every) : 0.f;
      my_sweeps += sweeps;
      if (conv) ++my_conv; else ++my_nconv;
    }
  }
  if (tid == 0 && q == 0) {
    if (a.s_sweeps >= 0) atomicAdd(&a.stats[a.s_sweeps], my_sweeps);
    if (a.s_updates >= 0) atomicAdd(&a.stats[a.s_updates], my_sweeps * (unsigned long long)V);
    if (a.s_conv >= 0) atomicAdd(&a.stats[a.s_conv], my_conv);
    if (a.s_nconv >= 0) atomicAdd(&a.stats[a.s_nconv], my_nconv);
  }
  if constexpr (CL) cg::this_cluster().sync();   // no CTA leaves while its slots may be read
}

// -- FP32 sweeps with the lattice in a cluster's distributed shared memory ----
// One start per cluster of C CTAs (2 C <= L), CTA q holding the state of its
// planes [q L / C, (q+1) L / C) in its shared memory while the start relaxes:
// no bulk copies and no ring, 8 B per site (64 KB per CTA for 4D 16^4 on 8
// CTAs, so three CTAs of 256 threads fit per SM).  A site's neighbours along
// axis d-1 across the CTA's first or last plane are read from the
// neighbouring CTAs' shared memory (distributed shared memory); the links,
// shared by every start of the orbit, come through the read-only path from
// L2, as in the streamed sweeps.  One cluster barrier per colour phase orders
// the phases.  Per site the operations are relax_slab_kernel's
// (SlabOps<float2>, same order), so the results are the same bit for bit.
// FP32 only.
__host__ __device__ inline size_t dsmem_smem_bytes(int d, int L, int P, int C) {
  const int nzmax = (L + C - 1) / C;
  return 1024 + (size_t)nzmax * P * 8;
}

template <int D>
__global__ void __launch_bounds__(1024, 1) relax_dsmem_kernel(const SlabArgs a) {
  using Ops = SlabOps<float2>;
  extern __shared__ __align__(16) unsigned char smem[];
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks(), q = (int)cl.block_rank();
  const int cid = blockIdx.x / C, ncl = gridDim.x / C;
  const int L = a.L, V = a.V, P = a.P, P2 = a.P / 2, tid = threadIdx.x, nt = blockDim.x;
  const int z0 = q * L / C, nz = (q + 1) * L / C - z0;            // >= 1 (C <= L)
  const int qp = (q + C - 1) % C, qn = (q + 1) % C;
  const int nz_prev = (qp + 1) * L / C - qp * L / C;
  float* red = reinterpret_cast<float*>(smem + 64);               // per-warp partials (<= 32 warps)
  double* cl_slots = reinterpret_cast<double*>(smem + 256);       // [2][16] exchange (rank 0's)
  float2* st = reinterpret_cast<float2*>(smem + 1024);            // [own planes][P] state
  // the planes next to this CTA's, in the neighbouring CTAs' shared memory
  const float2* st_prev = cl.map_shared_rank(st, qp) + (size_t)(nz_prev - 1) * P;   // plane z0 - 1
  const float2* st_next = cl.map_shared_rank(st, qn);                                // plane z0 + nz
  const float2* links = static_cast<const float2*>(a.links);
  int round = 0;
  unsigned long long my_sweeps = 0, my_conv = 0, my_nconv = 0;
  const SlabOmega w{a.omega, a.om1, a.omega32, a.om1_32, false};
  __syncthreads();
  cl.sync();

  // cluster-wide max of r (rank 0 holds double-buffered slots)
  auto cmax = [&](float r) -> float {
    for (int o = 16; o > 0; o >>= 1) r = fmaxf(r, __shfl_xor_sync(0xffffffffu, r, o));
    if ((tid & 31) == 0) red[tid >> 5] = r;
    __syncthreads();
    r = 0.f;
    for (int k = 0; k < nt / 32; ++k) r = fmaxf(r, red[k]);
    __syncthreads();
    double* set = cl_slots + 16 * (round & 1);
    if (tid == 0) cl.map_shared_rank(set, 0)[q] = (double)r;
    cl.sync();
    const double* src = cl.map_shared_rank(set, 0);
    double m = 0.0;
    for (int k = 0; k < C; ++k) m = fmax(m, src[k]);
    ++round;
    return (float)m;
  };
  // staple of site j (x0, rowbase) of own plane t
  auto staple = [&](int t, int j, int x0, int rowbase) -> float2 {
    const float2* cur = st + (size_t)t * P;
    const float2* prev = t > 0 ? cur - P : st_prev;
    const float2* next = t + 1 < nz ? cur + P : st_next;
    const float2* lkc = links + (size_t)(z0 + t) * P * D;                 // links of plane z
    const float2* lkm = links + (size_t)((z0 + t + L - 1) % L) * P * D;   // of plane z - 1
    float2 S = Ops::zero();
#pragma unroll
    for (int mu = 0; mu < D; ++mu) {
      float2 hp, hm, ub;
      if (mu < D - 1) {
        int jp, jm;
        slab_inplane_nb<D>(L, mu, j, x0, rowbase, jp, jm);
        hp = cur[jp]; hm = cur[jm];
        ub = __ldg(lkc + (size_t)jm * D + mu);
      } else {
        hp = next[j]; hm = prev[j];
        ub = __ldg(lkm + (size_t)j * D + mu);
      }
      Ops::acc_fwd(S, __ldg(lkc + (size_t)j * D + mu), hp);
      Ops::acc_bwd(S, ub, hm);
    }
    return S;
  };
  auto phase = [&](int c) {
    for (int t = 0; t < nz; ++t) {
      float2* cur = st + (size_t)t * P;
      for (int h = tid; h < P2; h += nt) {
        int j, x0, rowbase;
        slab_site_of<D>(L, h, c, z0 + t, j, x0, rowbase);
        cur[j] = Ops::move(cur[j], staple(t, j, x0, rowbase), w);
      }
    }
    cl.sync();   // this phase's updates, everywhere, before the next phase reads them
  };
  auto residual = [&]() -> float {
    float r = 0.f;
    for (int t = 0; t < nz; ++t)
      for (int j = tid; j < P; j += nt) {
        const int x0 = j % L, rowbase = j - x0;
        r = fmaxf(r, Ops::div2(st[(size_t)t * P + j], staple(t, j, x0, rowbase)));
      }
    return cmax(r);
  };

  const long long n = a.list ? (long long)*a.n_list : a.n;
  for (long long i = cid; i < n; i += ncl) {
    const long long idx = a.list ? (long long)a.list[i] : i;
    float2* out = static_cast<float2*>(a.state) + (size_t)idx * V + (size_t)z0 * P;
    for (int x = tid; x < nz * P; x += nt)
      st[x] = a.init ? Ops::start(a, idx, z0 * P + x) : out[x];
    cl.sync();
    int sweeps = 0, until = a.check_every;
    bool conv = false;
    float r = 0.f, r_last = 0.f;
    for (;;) {
      phase(0);
      phase(1);
      ++sweeps;
      if (--until == 0) {
        until = a.check_every;
        r_last = r;
        r = residual();
        conv = r < a.eps32;
        if (conv || sweeps >= a.max_sweeps) break;
      }
    }
    for (int x = tid; x < nz * P; x += nt) out[x] = st[x];
    if (tid == 0 && q == 0) {
      a.status[idx] = conv ? kConverged : kNotConverged;
      if (a.init) a.sweeps[idx] = sweeps; else a.sweeps[idx] += sweeps;
      if (a.rate) a.rate[idx] = (r_last > 0.f && r < r_last) ? (float)pow((double)r / (double)r_last, 0.5 / a.check_every) : 0.f;
      my_sweeps += sweeps;
      if (conv) ++my_conv; else ++my_nconv;
    }
    cl.sync();   // the neighbours are done reading this start's planes
  }
  if (tid == 0 && q == 0) {
    if (a.s_sweeps >= 0) atomicAdd(&a.stats[a.s_sweeps], my_sweeps);
    if (a.s_updates >= 0) atomicAdd(&a.stats[a.s_updates], my_sweeps * (unsigned long long)V);
    if (a.s_conv >= 0) atomicAdd(&a.stats[a.s_conv], my_conv);
    if (a.s_nconv >= 0) atomicAdd(&a.stats[a.s_nconv], my_nconv);
  }
  cl.sync();     // no CTA leaves while its shared memory may be read
}

// -- inexact Newton polish of the mixed path ----------------------------------
// The FP32 sweeps leave each start with max div^2 below eps32; Newton steps on
// the gauge angles then finish it (the Jacobian of div is the Faddeev-Popov
// operator M, the Hessian of the functional of Eq. 3):
//   1. FP64 pass: div_x = sum_mu [sin phi^theta_{x,mu} - sin phi^theta_{x-mu,mu}]
//      and the weights w = cos phi^theta from the FP64 state; stop when
//      max div^2 < eps; else store, as FP32, b_x = div_x / D_x and the
//      weights over D_x (D_x = the sum of the 2d weights at x), delta = 0;
//   2. FP32 checkerboard SOR on M delta = div, streamed through the plane
//      ring like the sweeps, until the corrections stall below lin_tol
//      max |b|;
//   3. FP64 pass: g_x <- g_x exp(i delta_x).
// The SOR parameter is set per start by young_omega: near the minimum the
// FP32 sweeps at parameter w are the linear SOR on M, so the contraction they
// showed gives M's Jacobi radius.  Large lattices have it close to 1, where a
// fixed parameter needs many times the sweeps of w_opt.  A step that does not lower max div^2 is halved (up
// to six times); a start without descent, or still above eps after
// newton_max steps, is listed for the FP64 sweeps (an indefinite M near a
// saddle, which relaxation leaves and Newton would not).  The inner solve of
// a step that cut max div^2 less than 4x gets 4x the sweep cap (up to 4x
// inner_max); a start gets `budget` inner sweeps in a launch, so a
// near-singular M holds one CTA for a bounded time: the host then runs the
// few such starts again on clusters (CL), and what is left on the FP64
// sweeps.
struct SlabNewtonArgs {
  int d, L, V, P, Ps;              // Ps: plane stride of delta (P rounded up to 4 floats)
  const double2* links;            // FP64 [x*d + mu], site order
  double2* state;                  // n * V, site order
  long long n;
  const unsigned* list;            // when set: only these batch entries, *n_list of them
  const unsigned* n_list;
  unsigned long long* work_ctr;
  double eps;
  int budget;                      // inner sweeps a start may take in this launch
  float omega_sweeps, lin_tol;     // the FP32 sweeps' parameter; inner stop
  const float* rate;               // per start: their contraction per sweep (0: none)
  int inner_max, newton_max;
  float* scratch;                  // per CTA: (1 + 2d) V coefficients, then L * Ps delta
  size_t scratch_floats;           // per CTA (a multiple of 4)
  int8_t* status;
  double* resid;
  unsigned* redo;                  // starts left to the FP64 sweeps
  unsigned* n_redo;
  unsigned long long* stats;       // [kNewton] steps, [kInner] sweeps, [kPass] FP64 passes, ...
  int s_steps, s_inner, s_pass, s_conv, s_redo;
  int* err;
};

__host__ __device__ inline size_t slab_newton_smem_bytes(int Ps) { return 1024 + 3 * (size_t)Ps * 4; }
__host__ __device__ inline size_t slab_newton_scratch_floats(int d, int V, int L, int Ps) {
  return (((size_t)(1 + 2 * d) * V + (size_t)L * Ps) + 3) / 4 * 4;
}

// CL = false: one start per CTA (scratch per CTA), starts from a counter.
// CL = true: one start per cluster (scratch per cluster), CTA q taking planes
// [q L / C, (q+1) L / C) in every pass; the CTAs meet at a cluster barrier
// after each FP64 pass and each SOR phase, which carries the maxima (max
// div^2 and max |b|, or the group's correction) and whether a wait ran out.
template <int D, bool CL>
__global__ void __launch_bounds__(1024, 1) slab_newton_kernel(const SlabNewtonArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int L = a.L, V = a.V, P = a.P, P2 = a.P / 2, Ps = a.Ps, tid = threadIdx.x, nt = blockDim.x;
  const unsigned sbase = (unsigned)__cvta_generic_to_shared(smem);
  long long* tidx = reinterpret_cast<long long*>(smem + 32);
  int* abort_flag = reinterpret_cast<int*>(smem + 40);
  double* redd = reinterpret_cast<double*>(smem + 64);     // per-warp partials (<= 32 warps)
  float* redf = reinterpret_cast<float*>(smem + 320);
  double* cl_slots = reinterpret_cast<double*>(smem + 512);  // [2][16][2] cluster exchange (rank 0's)
  PlaneRing<float> ring{reinterpret_cast<float*>(smem + 1024), sbase + 1024, sbase, (unsigned)(Ps * 4), L, Ps, 0u};
  int C = 1, q = 0, cid = 0, ncl = 1;
  if constexpr (CL) {
    cg::cluster_group cl = cg::this_cluster();
    C = (int)cl.num_blocks();
    q = (int)cl.block_rank();
    cid = blockIdx.x / C;
    ncl = gridDim.x / C;
  }
  const int z0 = q * L / C, nz = (q + 1) * L / C - z0;   // this CTA's planes (nz may be 0)
  const int x_beg = z0 * P, x_end = (z0 + nz) * P;
  float* coef = a.scratch + (size_t)(CL ? cid : blockIdx.x) * a.scratch_floats;   // [1 + 2D][V], colour-split
  float* dl = coef + (size_t)(1 + 2 * D) * V;                                       // [L][Ps], plane order
  int round = 0;

  if (tid == 0) {
    for (int k = 0; k < 3; ++k) mbar_init(sbase + 8u * k, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if constexpr (CL) cg::this_cluster().sync();
  unsigned long long my_steps = 0, my_inner = 0, my_pass = 0, my_conv = 0, my_redo = 0;

  // block maxima of r and f, then (cluster) over the CTAs; ok = every CTA's ok.
  // Double-buffered slots in rank 0 (as in the sweeps).
  auto reduce = [&](bool& ok, double& r, float& f) {
    for (int o = 16; o > 0; o >>= 1) {
      r = fmax(r, __shfl_xor_sync(0xffffffffu, r, o));
      f = fmaxf(f, __shfl_xor_sync(0xffffffffu, f, o));
    }
    if ((tid & 31) == 0) { redd[tid >> 5] = r; redf[tid >> 5] = f; }
    __syncthreads();
    r = 0.0; f = 0.f;
    for (int w = 0; w < nt / 32; ++w) { r = fmax(r, redd[w]); f = fmaxf(f, redf[w]); }
    __syncthreads();
    if constexpr (CL) {
      cg::cluster_group cl = cg::this_cluster();
      double* set = cl_slots + 32 * (round & 1);
      if (tid == 0) {
        fence_async_global();   // completed bulk stores and generic writes, before the release
        double* dst = cl.map_shared_rank(set, 0);
        dst[2 * q] = ok ? r : -1.0;
        dst[2 * q + 1] = (double)f;
      }
      cl.sync();
      if (tid == 0) fence_async_global();   // then the next bulk loads
      const double* src = cl.map_shared_rank(set, 0);
      double m = 0.0, mf = 0.0;
      bool all = true;
      for (int k = 0; k < C; ++k) {
        const double v = src[2 * k];
        if (v < 0.0) all = false; else m = fmax(m, v);
        mf = fmax(mf, src[2 * k + 1]);
      }
      ok = all;
      r = m;
      f = (float)mf;
      ++round;
    }
  };

  // 1. FP64 residual and the FP32 system of this CTA's planes; returns max
  // div^2 over the start, bmax = max |b|
  auto rhs = [&](const double2* g, float& bmax) -> double {
    double r = 0.0;
    float bm = 0.f;
    for (int x = x_beg + tid; x < x_end; x += nt) {
      int c[D];
      int t = x;
#pragma unroll
      for (int mu = 0; mu < D; ++mu) { c[mu] = t % L; t /= L; }
      const double2 gx = g[x];
      double dv = 0.0, Ds = 0.0, wf[D], wb[D];
      int stride = 1;
#pragma unroll
      for (int mu = 0; mu < D; ++mu) {
        const int xp = x + (c[mu] + 1 == L ? -(L - 1) * stride : stride);
        const int xm = x + (c[mu] == 0 ? (L - 1) * stride : -stride);
        const double2 uf = a.links[(size_t)x * D + mu], ub = a.links[(size_t)xm * D + mu];
        const double2 hp = g[xp], hm = g[xm];
        const double tfx = uf.x * hp.x - uf.y * hp.y, tfy = uf.x * hp.y + uf.y * hp.x;   // u h_+
        const double tbx = ub.x * hm.x + ub.y * hm.y, tby = ub.x * hm.y - ub.y * hm.x;   // conj(u') h_-
        wf[mu] = gx.x * tfx + gx.y * tfy;                 // cos phi^theta_{x,mu}
        wb[mu] = gx.x * tbx + gx.y * tby;                 // cos phi^theta_{x-mu,mu}
        dv += (gx.x * tfy - gx.y * tfx) + (gx.x * tby - gx.y * tbx);
        Ds += wf[mu] + wb[mu];
        stride *= L;
      }
      r = fmax(r, dv * dv);
      const int z = c[D - 1], j = x - z * P;
      int rs = 0;
#pragma unroll
      for (int mu = 1; mu < D - 1; ++mu) rs += c[mu];
      const size_t ci = (size_t)z * P + (size_t)((c[0] + rs + z) & 1) * P2 + (size_t)(j / L) * (L / 2) + c[0] / 2;
      if (Ds > 0.0) {
        const double inv = 1.0 / Ds;
        const float bb = (float)(dv * inv);
        coef[ci] = bb;
        bm = fmaxf(bm, fabsf(bb));
#pragma unroll
        for (int mu = 0; mu < D; ++mu) {
          coef[(size_t)(1 + mu) * V + ci] = (float)(wf[mu] * inv);
          coef[(size_t)(1 + D + mu) * V + ci] = (float)(wb[mu] * inv);
        }
      } else {   // no positive diagonal: the site stays (the step may then not contract)
        coef[ci] = 0.f;
#pragma unroll
        for (int mu = 0; mu < 2 * D; ++mu) coef[(size_t)(1 + mu) * V + ci] = 0.f;
      }
    }
    bool ok = true;
    reduce(ok, r, bm);
    bmax = bm;
    return r;
  };

  // 2. SOR sweeps from delta = 0 in groups of four, the correction of each
  // group's last sweep deciding (a correction 16 times the first group's
  // means M is not positive: stop); returns the sweeps, false in ok when a
  // wait ran out (the same on every CTA)
  auto sor = [&](float bmax, int cap, float om, bool& ok) -> int {
    for (int x = tid; x < nz * Ps; x += nt) dl[(size_t)z0 * Ps + x] = 0.f;
    fence_async_global();   // generic writes, then bulk reads of them
    __syncthreads();
    {
      double r0 = 0.0;
      float f0 = 0.f;
      reduce(ok, r0, f0);   // (cluster) the neighbours' zeros too
    }
    const float thr = a.lin_tol * bmax;
    int k = 0;
    float first = 0.f;
    while (k < cap) {
      float corr = 0.f;
      for (int kk = 0; kk < 4; ++kk, ++k) {
        const bool last = kk == 3;
        for (int c = 0; c < 2; ++c) {
          ok = nz == 0 || ring_walk(ring, dl, true, [&](const float* prev, float* cur, const float* next, int z) {
            const float* cp = coef + (size_t)z * P + (size_t)c * P2;
            for (int h = tid; h < P2; h += nt) {
              int j, x0, rowbase;
              slab_site_of<D>(L, h, c, z, j, x0, rowbase);
              float acc = cp[h];
#pragma unroll
              for (int mu = 0; mu < D; ++mu) {
                float dp, dm;
                if (mu < D - 1) {
                  int jp, jm;
                  slab_inplane_nb<D>(L, mu, j, x0, rowbase, jp, jm);
                  dp = cur[jp]; dm = cur[jm];
                } else {
                  dp = next[j]; dm = prev[j];
                }
                acc = fmaf(cp[(size_t)(1 + mu) * V + h], dp, acc);
                acc = fmaf(cp[(size_t)(1 + D + mu) * V + h], dm, acc);
              }
              const float old = cur[j], diff = acc - old;
              if (last) corr = fmaxf(corr, fabsf(diff));
              cur[j] = fmaf(om, diff, old);
            }
          }, z0, nz);
          if constexpr (CL) {
            double r0 = 0.0;
            float f0 = 0.f;
            reduce(ok, r0, f0);
          }
          if (!ok) return k;
        }
      }
      double dummy = 0.0;
      reduce(ok, dummy, corr);
      if (corr <= thr) break;
      if (first == 0.f) first = corr;
      else if (!(corr < 16.f * first)) break;
    }
    return k;
  };

  // 3. g_x <- g_x exp(i f delta_x) on this CTA's planes, renormalised (f < 0
  // takes part of a step back); then (cluster) every CTA's rotation is seen
  auto rotate = [&](double2* g, double f) {
    if (tid == 0) fence_async_global();   // the ring's stores, then generic reads of delta
    __syncthreads();
    for (int x = x_beg + tid; x < x_end; x += nt) {
      const int z = x / P, j = x - z * P;
      const double tf = f * (double)fminf(fmaxf(__ldcg(dl + (size_t)z * Ps + j), -0.2f), 0.2f);
      double sn, cs;
      sincos(tf, &sn, &cs);
      const double2 gx = g[x];
      const double nx = gx.x * cs - gx.y * sn, ny = gx.x * sn + gx.y * cs;
      const double qn = rsqrt(nx * nx + ny * ny);
      g[x] = make_double2(nx * qn, ny * qn);
    }
    __syncthreads();
    if constexpr (CL) {
      bool ok = true;
      double r0 = 0.0;
      float f0 = 0.f;
      reduce(ok, r0, f0);
    }
  };

  const long long n = a.list ? (long long)*a.n_list : a.n;
  for (long long i = cid;; i += ncl) {
    if constexpr (!CL) {
      if (tid == 0) *tidx = (long long)atomicAdd(a.work_ctr, 1ULL);
      __syncthreads();
      i = *tidx;
      __syncthreads();
      if (*abort_flag) break;
    }
    if (i >= n) break;
    const long long idx = a.list ? (long long)a.list[i] : i;
    double2* g = a.state + (size_t)idx * V;
    // this start's SOR parameter (Young)
    const float om = young_omega(a.rate ? a.rate[idx] : 0.f, a.omega_sweeps);
    bool ok = true, conv = false;
    int cap = a.inner_max, budget = a.budget;   // inner sweeps per solve, per start
    float bmax;
    double r = rhs(g, bmax);
    ++my_pass;
    for (int it = 0;; ++it) {
      if (r < a.eps) { conv = true; break; }
      if (it >= a.newton_max || budget <= 0) break;
      ++my_steps;
      const int k = sor(bmax, min(cap, budget), om, ok);
      my_inner += (unsigned long long)k;
      budget -= k;
      if (!ok) break;
      const double r0 = r;
      rotate(g, 1.0);
      r = rhs(g, bmax);
      ++my_pass;
      double f = 1.0;
      for (int h = 0; h < 6 && !(r < r0); ++h) {   // backtrack to half the step
        rotate(g, -0.5 * f);
        f *= 0.5;
        r = rhs(g, bmax);
        ++my_pass;
      }
      if (!(r < r0)) break;
      if (!(r < 0.25 * r0)) cap = min(4 * cap, 4 * a.inner_max);
    }
    if (!ok) {
      // (in a cluster every CTA gets here together)
      if (tid == 0) { atomicExch(&a.err[3], 1); *abort_flag = 1; }
      ring.drain();
      if (tid == 0) bulk_wait_all();
      __syncthreads();
      break;
    }
    if (tid == 0 && q == 0) {
      a.resid[idx] = r;
      if (conv) {
        a.status[idx] = kConverged;
        ++my_conv;
      } else {
        a.redo[atomicAdd(a.n_redo, 1u)] = (unsigned)idx;
        ++my_redo;
      }
    }
  }
  if (tid == 0 && q == 0) {
    atomicAdd(&a.stats[a.s_steps], my_steps);
    atomicAdd(&a.stats[a.s_inner], my_inner);
    atomicAdd(&a.stats[a.s_pass], my_pass);
    atomicAdd(&a.stats[a.s_conv], my_conv);
    if (a.s_redo >= 0) atomicAdd(&a.stats[a.s_redo], my_redo);
  }
  if constexpr (CL) cg::this_cluster().sync();   // no CTA leaves while its slots may be read
}

// FP32 state -> FP64, renormalised (the mixed path's hand-over to the FP64 sweeps)
// FP64 state -> FP32 state (round to nearest) for the FP32 phase that follows
// the FP64 head sweeps of the mixed path
__global__ void slab_demote_kernel(const double2* s64, float2* s32, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double2 v = s64[i];
    s32[i] = make_float2((float)v.x, (float)v.y);
  }
}

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

// -- first-region test beyond shared memory ----------------------------------
// Lanczos on the Faddeev-Popov operator M restricted to 1^perp (every vector
// projected off the mean), as on small lattices, with the copy's weights and
// the three Lanczos vectors in a global scratch slot per CTA (one copy per
// 1024-thread CTA at a time).  The smallest eigenvalue of the tridiagonal is
// located by the same Sturm multisection every 8 steps from step 16 on;
// Lanczos stops when it moves by less than tol relative.  R = float: the
// screen (a copy with lambda_2 above `margin` is IN, every other copy goes to
// the redo list); R = double: lambda_2 and the region (tau) of every listed
// copy.  Neighbours come from a per-site byte of wrap flags (bit 2 mu: x_mu =
// L - 1, bit 2 mu + 1: x_mu = 0), so the matvec takes no integer division.
struct SlabFpArgs {
  const double2* cfg;              // table configurations [entry][V]
  const unsigned long long* first_start;   // per entry: the lowest start reaching it
  const double2* links;            // FP64 [x*d + mu]
  int d, L, V;
  const unsigned* list;            // entries to test, *n_list of them
  const unsigned* n_list;
  unsigned* redo;                  // the screen's undecided entries
  unsigned* n_redo;
  double* lambda2;
  int* region;
  double tau, margin, tol;
  int kmax;
  uint64_t seed;
  unsigned char* scratch;          // per CTA: weights [d][V], vprev, vcur, z [V] (R), wrap [V]
  size_t scratch_bytes;            // per CTA (a multiple of 16)
  unsigned long long* stats;
  int s_tests, s_tests64, s_steps, s_steps64;
  int count_tests;                 // R = double: also count the copies as tests (no screen ran)
};

template <class R>
__host__ __device__ inline size_t slab_fp_scratch_bytes(int d, int V) {
  return (((size_t)(d + 3) * V * sizeof(R) + (size_t)V) + 15) / 16 * 16;
}
__host__ __device__ inline size_t slab_fp_smem_bytes(int kmax, int elem) {
  return 1152 + 2 * (((size_t)(kmax + 2) * elem + 15) / 16 * 16);
}

// CL = false: one copy per CTA.  CL = true: one copy per cluster, CTA q
// taking sites [q V / C, (q+1) V / C) in every pass (the vectors and weights
// stay in global memory, so the matvec reads the other CTAs' entries there);
// a cluster barrier follows every pass whose output other CTAs read, and the
// dot products are summed over the CTAs in rank order, the same on every CTA,
// so every CTA keeps the same tridiagonal and reaches the same decisions.
template <class R, int D, bool CL>
__global__ void __launch_bounds__(1024, 1) slab_fp_lanczos_kernel(const SlabFpArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int L = a.L, V = a.V, tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, wid = tid >> 5;
  const int kmax = a.kmax;
  R* red = reinterpret_cast<R*>(smem);                 // [2][32] per-warp partials (<= 512 B)
  R* bcast = reinterpret_cast<R*>(smem + 512);         // [2]
  double* cl_slots = reinterpret_cast<double*>(smem + 528);   // [2][16][2] (rank 0's), to 1040
  R* alpha = reinterpret_cast<R*>(smem + 1152);
  R* beta2 = alpha + ((size_t)(kmax + 2) * sizeof(R) + 15) / 16 * 16 / sizeof(R);
  int C = 1, q = 0, cid = blockIdx.x, ncl = gridDim.x;
  if constexpr (CL) {
    cg::cluster_group cl = cg::this_cluster();
    C = (int)cl.num_blocks();
    q = (int)cl.block_rank();
    cid = blockIdx.x / C;
    ncl = gridDim.x / C;
  }
  const int xb = (int)((long long)q * V / C), xe = (int)((long long)(q + 1) * V / C);   // this CTA's sites
  unsigned char* base = a.scratch + (size_t)cid * a.scratch_bytes;
  R* w = reinterpret_cast<R*>(base);                   // [D][V]
  R* vprev = w + (size_t)D * V;
  R* vcur = vprev + V;
  R* z = vcur + V;
  unsigned char* wrap = reinterpret_cast<unsigned char*>(z + V);
  int round = 0;
  int strides[D];
  {
    int st = 1;
#pragma unroll
    for (int mu = 0; mu < D; ++mu) { strides[mu] = st; st *= L; }
  }
  for (int x = xb + tid; x < xe; x += nt) {
    int t = x;
    unsigned f = 0;
#pragma unroll
    for (int mu = 0; mu < D; ++mu) {
      const int c = t % L;
      t /= L;
      if (c == L - 1) f |= 1u << (2 * mu);
      if (c == 0) f |= 2u << (2 * mu);
    }
    wrap[x] = (unsigned char)f;
  }
  __syncthreads();
  // the other CTAs' writes of the last pass are seen (identity without a cluster)
  auto csync = [&]() {
    if constexpr (CL) cg::this_cluster().sync(); else __syncthreads();
  };
  // sums of two values over the block, then (cluster) over the CTAs in rank
  // order; every thread of every CTA gets both
  auto sum2 = [&](R& p, R& r2) {
    for (int o = 16; o > 0; o >>= 1) {
      p += __shfl_xor_sync(0xffffffffu, p, o);
      r2 += __shfl_xor_sync(0xffffffffu, r2, o);
    }
    if (lane == 0) { red[wid] = p; red[32 + wid] = r2; }
    __syncthreads();
    p = 0; r2 = 0;
    for (int k = 0; k < nt / 32; ++k) { p += red[k]; r2 += red[32 + k]; }
    __syncthreads();
    if constexpr (CL) {
      cg::cluster_group cl = cg::this_cluster();
      double* set = cl_slots + 32 * (round & 1);
      if (tid == 0) {
        double* dst = cl.map_shared_rank(set, 0);
        dst[2 * q] = (double)p;
        dst[2 * q + 1] = (double)r2;
      }
      cl.sync();
      // warp 0 reads the C partials (one remote load per lane), lane 0 sums
      // them in rank order, and the block reads the result locally
      if (wid == 0) {
        const double* src = cl.map_shared_rank(set, 0);
        const double vp = lane < C ? src[2 * lane] : 0.0, vq = lane < C ? src[2 * lane + 1] : 0.0;
        R sp = 0, sq = 0;
        for (int k = 0; k < C; ++k) {
          sp += (R)__shfl_sync(0xffffffffu, vp, k);
          sq += (R)__shfl_sync(0xffffffffu, vq, k);
        }
        if (lane == 0) { bcast[0] = sp; bcast[1] = sq; }
      }
      __syncthreads();
      p = bcast[0];
      r2 = bcast[1];
      __syncthreads();
      ++round;
    }
  };
  auto nbr = [&](int x, unsigned f, int mu, int& xp, int& xm) {
    const int st = strides[mu];
    xp = x + ((f >> (2 * mu)) & 1u ? -(L - 1) * st : st);
    xm = x + ((f >> (2 * mu + 1)) & 1u ? (L - 1) * st : -st);
  };
  const unsigned n = *a.n_list;
  unsigned long long my_steps = 0, my_tests = 0;
  for (unsigned i = cid; i < n; i += ncl) {
    const unsigned e = a.list[i];
    const double2* g = a.cfg + (size_t)e * V;
    // weights cos(phi^theta_{x,mu}) = Re[conj(g_x) u_{x,mu} g_{x+mu}]
    for (int x = xb + tid; x < xe; x += nt) {
      const double2 gx = g[x];
      const unsigned f = wrap[x];
#pragma unroll
      for (int mu = 0; mu < D; ++mu) {
        int xp, xm;
        nbr(x, f, mu, xp, xm);
        const double2 h = g[xp], u = a.links[(size_t)x * D + mu];
        w[(size_t)mu * V + x] = (R)(gx.x * (u.x * h.x - u.y * h.y) + gx.y * (u.x * h.y + u.y * h.x));
      }
    }
    // random start vector orthogonal to the constant mode, keyed by the
    // copy's first start (not its table slot, which depends on the order of
    // insertion), so that a Ritz value short of convergence is reproducible
    const unsigned long long key = a.first_start[e];
    R s = 0, dummy = 0;
    for (int x = xb + tid; x < xe; x += nt) {
      const U64x4 r = philox4x64_10(key, (uint64_t)x, 0, 1, a.seed, 0x4C414E43ULL);
      const R v = (R)(unsigned)(r.v[0] >> 40) * (R)0x1.0p-24 - (R)0.5;
      vcur[x] = v;
      vprev[x] = 0;
      s += v;
    }
    sum2(s, dummy);
    s /= (R)V;
    R nn = 0;
    for (int x = xb + tid; x < xe; x += nt) { const R v = vcur[x] - s; vcur[x] = v; nn += v * v; }
    dummy = 0;
    sum2(nn, dummy);
    {
      const R inv0 = (R)1 / sqrt(nn);
      for (int x = xb + tid; x < xe; x += nt) vcur[x] *= inv0;
    }
    csync();   // the weights and the start vector, everywhere
    const R bound = (R)(4 * D + 1);
    R b = 0, theta = bound, theta_prev = bound, theta_pp = bound;
    // The current vector is (vr[x] - mb) * ibv: the previous step's raw z,
    // normalised where it is read, so that a step takes two passes over the
    // sites (the same values as storing it normalised in a third pass)
    R* vp = vprev;   // v_{j-1}, normalised
    R* vr = vcur;    // raw v_j
    R* zs = z;       // z_j
    R mb = 0, ibv = 1;
    int j = 0;
    for (; j < kmax; ++j) {
      R al = 0;
      for (int x = xb + tid; x < xe; x += nt) {
        const unsigned f = wrap[x];
        const R vx = (vr[x] - mb) * ibv;
        R acc = 0;
#pragma unroll
        for (int mu = 0; mu < D; ++mu) {
          int xp, xm;
          nbr(x, f, mu, xp, xm);
          acc = fma(w[(size_t)mu * V + x], vx - (vr[xp] - mb) * ibv, acc);
          acc = fma(w[(size_t)mu * V + xm], vx - (vr[xm] - mb) * ibv, acc);
        }
        const R mv = acc - b * vp[x];
        zs[x] = mv;
        al += mv * vx;
      }
      dummy = 0;
      sum2(al, dummy);   // (and every CTA's matvec is done before vr is rewritten)
      R m = 0, zz = 0;
      for (int x = xb + tid; x < xe; x += nt) {
        const R vx = (vr[x] - mb) * ibv;
        const R v = zs[x] - al * vx;
        zs[x] = v;
        vr[x] = vx;      // v_j normalised in place: the next step's v_{j-1}
        m += v;
        zz += v * v;
      }
      sum2(m, zz);       // (cluster) also orders this pass's writes before the next matvec
      m /= (R)V;
      const R bn = sqrt(fmax(zz - (R)V * m * m, (R)0));   // |z - m|
      if (tid == 0) { alpha[j] = al; beta2[j + 1] = bn * bn; }
      __syncthreads();
      const bool last = (j + 1 == kmax) || bn < (R)1e-12;
      if (last || ((j + 1) % 8 == 0 && j + 1 >= 16)) {
        if (wid == 0) {
          R lo = -bound, hi = bound;
          if (theta_prev < bound) {
            const R slack = (R)2 * tri_rel<R>() * fmax(fabs(theta_prev), (R)1);
            hi = theta_prev + slack;
            if (theta_pp < bound) {
              const R l = theta_prev - (R)4 * fmax(theta_pp - theta_prev, slack);
              if (sturm_count<R>(alpha, beta2, j + 1, l) == 0) lo = l;
            }
          }
          const R th = tri_min<R>(alpha, beta2, j + 1, lo, hi, lane);
          if (lane == 0) bcast[0] = th;
        }
        __syncthreads();
        theta = bcast[0];
        __syncthreads();
        if (last) { ++j; break; }
        if (fabs(theta - theta_prev) <= (R)a.tol * fmax(fabs(theta), (R)1e-3)) { ++j; break; }
        theta_pp = theta_prev;
        theta_prev = theta;
      }
      // v_{j-1} <- v_j, raw v_{j+1} <- z_j, scratch <- the old v_{j-1}
      R* t = vp;
      vp = vr;
      vr = zs;
      zs = t;
      mb = m;
      ibv = (R)1 / bn;
      b = bn;
    }
    my_steps += j;
    ++my_tests;
    if (tid == 0 && q == 0) {
      if (sizeof(R) == 4) {
        if (theta > (R)a.margin) {
          a.lambda2[e] = (double)theta;
          a.region[e] = kRegionIn;
        } else {
          a.redo[atomicAdd(a.n_redo, 1u)] = e;
        }
      } else {
        a.lambda2[e] = (double)theta;
        a.region[e] = region_of((double)theta, a.tau);
      }
    }
    csync();   // this copy's scratch is reused by the next
  }
  if (tid == 0 && q == 0) {
    atomicAdd(&a.stats[a.s_steps], my_steps);
    if (sizeof(R) == 4 || a.count_tests) atomicAdd(&a.stats[a.s_tests], my_tests);
    if (sizeof(R) == 8) atomicAdd(&a.stats[a.s_tests64], my_tests);
    if (sizeof(R) == 8) atomicAdd(&a.stats[a.s_steps64], my_steps);
  }
  if constexpr (CL) cg::this_cluster().sync();   // no CTA leaves while its slots may be read
}

}  // namespace gc
