// Relaxation kernels: random starts -> checkerboard (over)relaxation sweeps ->
// Landau residual -> canonical copy + functional (Section III, Eqs. 3-5).
//
// Work layout (one design for every d, L): a CTA holds the orbit's links and
// the lattice's colour-major neighbour table in shared memory once; every
// team of T lanes (T a power of two, T <= 32) relaxes one start whose gauge
// field g lives in the team's own shared-memory slot, indexed by colour
// position.  All teams of a warp sweep in lock step; a team whose start
// converged (checked every `check_every` sweeps) writes its result and pulls
// the next start index from a global counter, so heavy-tailed sweep counts
// never idle a whole CTA.
//
// Precision policies:
//   Exact64 -- FP64 with every product / sum an explicitly rounded IEEE step
//              (no FMA), in the same order as a plain serial restatement, so
//              a start's trajectory is a fixed function of its input;
//   Fast32  -- FP32 with FMA and the MUFU reciprocal square root (bulk phase
//              of the mixed-precision path).
#pragma once
#include "gc_common.cuh"

namespace gc {

enum : int8_t { kConverged = 1, kNotConverged = 2, kDedupFailed = 3 };

struct RelaxArgs {
  Geom geom;
  const double2* links64;        // V*d (cos phi, sin phi), site-major [x*d + mu]
  const float2* links32;         // same, rounded to FP32
  uint64_t seed, orbit_id;
  uint64_t start0;               // first start index of this batch
  long long n;                   // starts in this batch
  unsigned long long* work_ctr;  // next batch-relative start to hand out
  double omega, om1, eps;        // om1 = 1 - omega (rounded once, on the host)
  float omega32, om1_32, eps32;
  int check_every, max_sweeps;
  int team;                      // lanes per team
  int stat_base;                 // first of the 4 stats slots this phase adds to
  // per-start outputs (batch-relative index)
  int8_t* status;
  int32_t* sweeps;
  double* resid;
  double* F;
  double* fprint;                // cos(phi^theta) of link (site 0, mu 0)
  double2* config;               // n*V canonical g' (FP64) in site order, g'_{V-1} = 1
  float2* state32;               // n*V final FP32 state in colour-position order (mixed path)
  unsigned long long* stats;     // [base] sweeps, [base+1] site-updates, [base+2] converged,
                                 // [base+3] not converged
};

__host__ __device__ inline size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

// Shared-memory layout shared by host (launch size) and device:
// links [mu][p] | nbp [p] | site [p] | pos scratch | per-team slots.
struct Smem {
  size_t links, nbp, site, pos, team0, per_team, total;
  __host__ __device__ Smem(int V, int d, size_t link_bytes, size_t team_bytes, int teams) {
    links = 0;
    nbp = align16((size_t)V * d * link_bytes);
    site = nbp + (size_t)V * sizeof(uint4);
    pos = site + align16((size_t)V * sizeof(uint16_t));
    team0 = pos + align16((size_t)V * sizeof(uint16_t));
    per_team = align16(team_bytes);
    total = team0 + (size_t)teams * per_team;
  }
};

struct Exact64 {
  using R = double;
  using R2 = double2;
  static __device__ __forceinline__ const R2* links(const RelaxArgs& a) { return a.links64; }
  // a * b
  static __device__ __forceinline__ R2 mul(R2 a, R2 b) {
    return make_double2(__dsub_rn(__dmul_rn(a.x, b.x), __dmul_rn(a.y, b.y)),
                        __dadd_rn(__dmul_rn(a.x, b.y), __dmul_rn(a.y, b.x)));
  }
  // conj(a) * b
  static __device__ __forceinline__ R2 cmul(R2 a, R2 b) {
    return make_double2(__dadd_rn(__dmul_rn(a.x, b.x), __dmul_rn(a.y, b.y)),
                        __dsub_rn(__dmul_rn(a.x, b.y), __dmul_rn(a.y, b.x)));
  }
  // S in the fixed order mu = 0..d-1, forward term then backward term
  static __device__ __forceinline__ R2 staple(const R2* __restrict__ u, const R2* __restrict__ g,
                                              const uint4 nb, int p, int d, int V) {
    R2 S = make_double2(0.0, 0.0);
    for (int mu = 0; mu < d; ++mu) {
      const unsigned wd = nb_word(nb, mu);
      const int xp = wd & 0xffffu, xm = wd >> 16;
      const R2 t = mul(u[mu * V + p], g[xp]);
      S.x = __dadd_rn(S.x, t.x); S.y = __dadd_rn(S.y, t.y);
      const R2 s = cmul(u[mu * V + xm], g[xm]);
      S.x = __dadd_rn(S.x, s.x); S.y = __dadd_rn(S.y, s.y);
    }
    return S;
  }
  static __device__ __forceinline__ void update(R2* g, const R2* u, const uint4* nbp, int p, int d,
                                                int V, const RelaxArgs& a) {
    const R2 S = staple(u, g, nbp[p], p, d, V);
    const double n2 = __dadd_rn(__dmul_rn(S.x, S.x), __dmul_rn(S.y, S.y));
    if (!(n2 > 0.0)) return;
    const double r = __drcp_rn(__dsqrt_rn(n2));
    const double hx = __dmul_rn(S.x, r), hy = __dmul_rn(S.y, r);
    const R2 gx = g[p];
    const double vx = __dadd_rn(__dmul_rn(a.om1, gx.x), __dmul_rn(a.omega, hx));
    const double vy = __dadd_rn(__dmul_rn(a.om1, gx.y), __dmul_rn(a.omega, hy));
    const double m2 = __dadd_rn(__dmul_rn(vx, vx), __dmul_rn(vy, vy));
    if (m2 > 0.0) {
      const double q = __drcp_rn(__dsqrt_rn(m2));
      g[p] = make_double2(__dmul_rn(vx, q), __dmul_rn(vy, q));
    } else {
      g[p] = make_double2(hx, hy);
    }
  }
  static __device__ __forceinline__ R div2(const R2* g, const R2* u, const uint4* nbp, int p, int d,
                                           int V) {
    const R2 S = staple(u, g, nbp[p], p, d, V);
    const R2 gx = g[p];
    const double dv = __dsub_rn(__dmul_rn(gx.x, S.y), __dmul_rn(gx.y, S.x));
    return __dmul_rn(dv, dv);
  }
  static __device__ __forceinline__ R eps(const RelaxArgs& a) { return a.eps; }
  static __device__ __forceinline__ R2 start(uint64_t seed, uint64_t orb, uint64_t s, int x) {
    return random_unit(seed, orb, s, (uint64_t)x);
  }
};

struct Fast32 {
  using R = float;
  using R2 = float2;
  static __device__ __forceinline__ const R2* links(const RelaxArgs& a) { return a.links32; }
  static __device__ __forceinline__ R2 staple(const R2* __restrict__ u, const R2* __restrict__ g,
                                              const uint4 nb, int p, int d, int V) {
    float sx = 0.f, sy = 0.f;
    for (int mu = 0; mu < d; ++mu) {
      const unsigned wd = nb_word(nb, mu);
      const int xp = wd & 0xffffu, xm = wd >> 16;
      const R2 a = u[mu * V + p], h = g[xp];
      sx = fmaf(a.x, h.x, sx); sx = fmaf(-a.y, h.y, sx);
      sy = fmaf(a.x, h.y, sy); sy = fmaf(a.y, h.x, sy);
      const R2 b = u[mu * V + xm], k = g[xm];
      sx = fmaf(b.x, k.x, sx); sx = fmaf(b.y, k.y, sx);
      sy = fmaf(b.x, k.y, sy); sy = fmaf(-b.y, k.x, sy);
    }
    return make_float2(sx, sy);
  }
  static __device__ __forceinline__ void update(R2* g, const R2* u, const uint4* nbp, int p, int d,
                                                int V, const RelaxArgs& a) {
    const R2 S = staple(u, g, nbp[p], p, d, V);
    const float n2 = fmaf(S.x, S.x, S.y * S.y);
    if (!(n2 > 0.f)) return;
    const float r = rsqrtf(n2) * a.omega32;
    const R2 gx = g[p];
    const float vx = fmaf(S.x, r, a.om1_32 * gx.x);
    const float vy = fmaf(S.y, r, a.om1_32 * gx.y);
    const float m2 = fmaf(vx, vx, vy * vy);
    if (m2 > 0.f) {
      const float q = rsqrtf(m2);
      g[p] = make_float2(vx * q, vy * q);
    }
  }
  static __device__ __forceinline__ R div2(const R2* g, const R2* u, const uint4* nbp, int p, int d,
                                           int V) {
    const R2 S = staple(u, g, nbp[p], p, d, V);
    const R2 gx = g[p];
    const float dv = fmaf(gx.x, S.y, -gx.y * S.x);
    return dv * dv;
  }
  static __device__ __forceinline__ R eps(const RelaxArgs& a) { return a.eps32; }
  static __device__ __forceinline__ R2 start(uint64_t seed, uint64_t orb, uint64_t s, int x) {
    return random_unit32(seed, orb, s, (uint64_t)x);
  }
};

// Canonical copy (theta'_{V-1} = 0), functional Eq. 3 and fingerprint for an
// FP64 state in colour-position order; writes record i (config in site order).
__device__ inline void write_copy64(const double2* g, const double2* u, const uint4* nbp,
                                    const uint16_t* site, const Geom& G, int tl, int T,
                                    unsigned mask, long long i, double2* config, double* Fout,
                                    double* fprint) {
  const int V = G.V, d = G.d;
  const double2 gc = g[G.pos_last];
  double Fp = 0.0;
  for (int p = tl; p < V; p += T) {
    const double2 gx = g[p];
    // g'_x = g_x conj(g_{V-1})
    config[(size_t)i * V + site[p]] = make_double2(gx.x * gc.x + gx.y * gc.y, gx.y * gc.x - gx.x * gc.y);
    const uint4 nb = nbp[p];
    for (int mu = 0; mu < d; ++mu) {
      const double2 h = g[nb_word(nb, mu) & 0xffffu];
      const double2 a = u[mu * V + p];
      // Re[conj(g_x) u g_{x+mu}] = cos(phi^theta_{x,mu})
      const double tx = a.x * h.x - a.y * h.y, ty = a.x * h.y + a.y * h.x;
      const double w = gx.x * tx + gx.y * ty;
      Fp += 1.0 - w;
      if (p == 0 && mu == 0) fprint[i] = w;   // site 0 sits at position 0
    }
  }
  Fp = team_sum(Fp, T, mask);
  if (tl == 0) Fout[i] = Fp;
}

// load links [x*d + mu] (global) into shared [mu][p]
template <typename R2>
__device__ inline void load_links(R2* u, const R2* gl, const uint16_t* site, int V, int d) {
  for (int p = threadIdx.x; p < V; p += blockDim.x) {
    const int x = site[p];
    for (int mu = 0; mu < d; ++mu) u[mu * V + p] = gl[x * d + mu];
  }
}

template <class P>
__global__ void __launch_bounds__(256) relax_kernel(const RelaxArgs a) {
  using R = typename P::R;
  using R2 = typename P::R2;
  extern __shared__ __align__(16) unsigned char smem[];
  const Geom G = a.geom;
  const int V = G.V, d = G.d, T = a.team;
  const int teams_per_warp = 32 / T;
  const int warps = blockDim.x >> 5;
  const Smem lay(V, d, sizeof(R2), (size_t)V * sizeof(R2), warps * teams_per_warp);
  R2* u = reinterpret_cast<R2*>(smem + lay.links);
  uint4* nbp = reinterpret_cast<uint4*>(smem + lay.nbp);
  uint16_t* site = reinterpret_cast<uint16_t*>(smem + lay.site);
  build_colour_geometry(G, site, nbp, reinterpret_cast<uint16_t*>(smem + lay.pos));
  load_links(u, P::links(a), site, V, d);
  __syncthreads();

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int tw = lane / T, tl = lane & (T - 1);
  const unsigned tmask = team_mask(T, tw);
  R2* g = reinterpret_cast<R2*>(smem + lay.team0 + (size_t)(warp * teams_per_warp + tw) * lay.per_team);

  unsigned long long my_sweeps = 0, my_updates = 0, my_conv = 0, my_nconv = 0;

  // fetch the first start of every team
  long long idx = 0;
  if (tl == 0) idx = (long long)atomicAdd(a.work_ctr, 1ULL);
  idx = __shfl_sync(0xffffffffu, idx, tw * T);
  bool active = idx < a.n;
  if (active)
    for (int p = tl; p < V; p += T) g[p] = P::start(a.seed, a.orbit_id, a.start0 + idx, site[p]);
  int sweeps = 0;
  __syncwarp();

  unsigned step = 0;
  while (__any_sync(0xffffffffu, active)) {
    for (int c = 0; c < G.ncolor; ++c) {
      if (active) {
        const int beg = G.color_off[c], end = G.color_off[c + 1];
        for (int p = beg + tl; p < end; p += T) P::update(g, u, nbp, p, d, V, a);
      }
      __syncwarp();
    }
    ++step;
    if (active) ++sweeps;
    if (step % (unsigned)a.check_every == 0) {
      R r = 0;
      if (active)
        for (int p = tl; p < V; p += T) { const R v = P::div2(g, u, nbp, p, d, V); r = v > r ? v : r; }
      r = team_max(r, T, 0xffffffffu);  // xor offsets < T stay inside the team
      const bool done = active && (r < P::eps(a) || sweeps >= a.max_sweeps);
      if (done) {
        const bool conv = r < P::eps(a);
        if (tl == 0) {
          a.status[idx] = conv ? kConverged : kNotConverged;
          a.sweeps[idx] = sweeps;
          if constexpr (sizeof(R) == 8) a.resid[idx] = r;
          my_sweeps += sweeps;
          my_updates += (unsigned long long)sweeps * V;
          if (conv) ++my_conv; else ++my_nconv;
        }
        if constexpr (sizeof(R) == 8) {
          write_copy64(reinterpret_cast<const double2*>(g), reinterpret_cast<const double2*>(u), nbp,
                       site, G, tl, T, tmask, idx, a.config, a.F, a.fprint);
        } else {
          for (int p = tl; p < V; p += T) a.state32[(size_t)idx * V + p] = reinterpret_cast<const float2*>(g)[p];
        }
        __syncwarp(tmask);
        if (tl == 0) idx = (long long)atomicAdd(a.work_ctr, 1ULL);
        idx = __shfl_sync(tmask, idx, tw * T);
        active = idx < a.n;
        sweeps = 0;
        if (active)
          for (int p = tl; p < V; p += T) g[p] = P::start(a.seed, a.orbit_id, a.start0 + idx, site[p]);
      }
      __syncwarp();
    }
  }
  if (tl == 0 && (my_sweeps | my_conv | my_nconv)) {
    atomicAdd(&a.stats[a.stat_base + 0], my_sweeps);
    atomicAdd(&a.stats[a.stat_base + 1], my_updates);
    atomicAdd(&a.stats[a.stat_base + 2], my_conv);
    atomicAdd(&a.stats[a.stat_base + 3], my_nconv);
  }
}

// ---------------------------------------------------------------------------
// FP64 polish of FP32-relaxed starts (mixed path)
// ---------------------------------------------------------------------------
// Inexact Newton with FP32 inner solves (mixed-precision iterative refinement):
//   0. once: link weights w = cos(phi^theta) in FP32 from the FP32 state;
//   1. FP64: S_x and div_x = Im[conj(g_x) S_x]; stop if max div^2 < eps;
//   2. FP32: solve M delta = div (M = the Faddeev-Popov Laplacian with weights
//      w, the Hessian of Eq. 3) by checkerboard SOR until the correction
//      stalls below lin_tol;
//   3. FP64: g_x <- g_x exp(i delta_x)   (theta <- theta + delta).
// The residual and the state stay FP64; only the correction is FP32, so each
// Newton step shrinks the FP64 residual by the inner solve's relative accuracy
// (stale FP32 weights only make the steps inexact).  If Newton stalls (an
// indefinite M near a saddle), the start falls back to FP64 relaxation sweeps.
// FP64 work per site and Newton step: 8d DFMA for S, 3 for the divergence,
// 9 for the rotation; every float<->double move uses the integer pipe.
struct PolishArgs {
  Geom geom;
  const double2* links64;
  const float2* links32;
  long long n;
  unsigned long long* work_ctr;
  double omega, om1, eps;
  float omega_in, lin_tol;       // inner SOR parameter; stop when the SOR correction
                                 // max|t - delta| <= lin_tol max|b / D|
  int inner_max, newton_max, max_sweeps, check_every;
  int team;
  int8_t* status;                // in: FP32 phase outcome; out: final outcome
  int32_t* sweeps;               // in: FP32 sweeps; out: + FP64 fallback sweeps
  double* resid;
  const float2* state32;         // colour-position order
  double* F;
  double* fprint;
  double2* config;
  unsigned long long* stats;     // [4] newton steps, [5] fallbacks, [6] fp64 fallback site
                                 // updates, [7] fp64 residual passes, [8] / [9] final
                                 // converged / not converged, [20] inner FP32 SOR sweeps,
                                 // [21] FP32 relaxation site updates of the fallback
};

// per team: g (FP64), w (FP32, [mu][p]), b, delta, 1/D (FP32)
__host__ __device__ inline size_t polish_team_bytes(int V, int d) {
  return align16((size_t)V * sizeof(double2)) + align16((size_t)V * d * sizeof(float)) +
         3 * align16((size_t)V * sizeof(float));
}

// S_x with DFMA chains (4 per complex term)
__device__ __forceinline__ double2 staple_dfma(const double2* __restrict__ u,
                                               const double2* __restrict__ g, const uint4 nb, int p,
                                               int d, int V) {
  double sx = 0.0, sy = 0.0;
  for (int mu = 0; mu < d; ++mu) {
    const unsigned wd = nb_word(nb, mu);
    const int xp = wd & 0xffffu, xm = wd >> 16;
    const double2 a = u[mu * V + p], h = g[xp];
    sx = fma(a.x, h.x, sx); sx = fma(-a.y, h.y, sx);
    sy = fma(a.x, h.y, sy); sy = fma(a.y, h.x, sy);
    const double2 b = u[mu * V + xm], k = g[xm];
    sx = fma(b.x, k.x, sx); sx = fma(b.y, k.y, sx);
    sy = fma(b.x, k.y, sy); sy = fma(-b.y, k.x, sy);
  }
  return make_double2(sx, sy);
}

__global__ void __launch_bounds__(256) polish_kernel(const PolishArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Geom G = a.geom;
  const int V = G.V, d = G.d, T = a.team;
  const int teams_per_warp = 32 / T, warps = blockDim.x >> 5;
  const Smem lay(V, d, sizeof(double2), polish_team_bytes(V, d), warps * teams_per_warp);
  double2* u = reinterpret_cast<double2*>(smem + lay.links);
  uint4* nbp = reinterpret_cast<uint4*>(smem + lay.nbp);
  uint16_t* site = reinterpret_cast<uint16_t*>(smem + lay.site);
  build_colour_geometry(G, site, nbp, reinterpret_cast<uint16_t*>(smem + lay.pos));
  load_links(u, a.links64, site, V, d);
  __syncthreads();

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int tw = lane / T, tl = lane & (T - 1);
  const unsigned tmask = team_mask(T, tw);
  unsigned char* base = smem + lay.team0 + (size_t)(warp * teams_per_warp + tw) * lay.per_team;
  double2* g = reinterpret_cast<double2*>(base);
  float* w = reinterpret_cast<float*>(base + align16((size_t)V * sizeof(double2)));
  float* b = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(w) + align16((size_t)V * d * sizeof(float)));
  float* dl = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(b) + align16((size_t)V * sizeof(float)));
  float* Dinv = reinterpret_cast<float*>(reinterpret_cast<unsigned char*>(dl) + align16((size_t)V * sizeof(float)));

  unsigned long long c_newton = 0, c_fallback = 0, c_upd64 = 0, c_pass = 0, c_conv = 0, c_nconv = 0;
  unsigned long long c_inner = 0, c_upd32 = 0;
  // Teams are independent here (no lock step needed): each loops over starts.
  for (;;) {
    long long idx = 0;
    if (tl == 0) idx = (long long)atomicAdd(a.work_ctr, 1ULL);
    idx = __shfl_sync(tmask, idx, tw * T);
    if (idx >= a.n) break;
    const int8_t st32 = a.status[idx];
    const float2* s32 = a.state32 + (size_t)idx * V;
    // promote: exact float -> double, then renormalise with two Newton steps
    // for 1/sqrt (|g32| = 1 to FP32 precision)
    for (int p = tl; p < V; p += T) {
      const float2 gx = s32[p];
      const double px = f2d_bits(gx.x), py = f2d_bits(gx.y);
      const double n2 = fma(px, px, py * py);
      double q = fma(-0.5, n2, 1.5);
      q = q * fma(-0.5 * n2, q * q, 1.5);
      g[p] = make_double2(px * q, py * q);
    }
    __syncwarp(tmask);
    bool conv = false;
    double r = 0.0;
    int extra_sweeps = 0;
    int relax32_sweeps = 0;
    if (st32 == kConverged) {
      // up to two Newton rounds; between them, FP32 relaxation sweeps from the
      // current state (a descent method, cheap) move a start that Newton could
      // not finish (near-singular or indefinite Hessian) closer to its minimum
      for (int round = 0; round < 2 && !conv; ++round) {
        if (round == 1) {
          if (d < 2) break;  // the FP32 scratch lattice reuses w (V d floats >= 2V)
          ++c_fallback;
          float2* g32 = reinterpret_cast<float2*>(w);
          for (int p = tl; p < V; p += T) g32[p] = make_float2(d2f_bits(g[p].x), d2f_bits(g[p].y));
          __syncwarp(tmask);
          const float om = (float)a.omega, om1 = (float)a.om1;
          for (int sw = 0; sw < a.max_sweeps; ++sw) {
            for (int c = 0; c < G.ncolor; ++c) {
              const int beg = G.color_off[c], end = G.color_off[c + 1];
              for (int p = beg + tl; p < end; p += T) {
                const uint4 nb = nbp[p];
                float sx = 0.f, sy = 0.f;
                for (int mu = 0; mu < d; ++mu) {
                  const unsigned wd = nb_word(nb, mu);
                  const int xp = wd & 0xffffu, xm = wd >> 16;
                  const float2 aa = a.links32[site[p] * d + mu], h = g32[xp];
                  sx = fmaf(aa.x, h.x, sx); sx = fmaf(-aa.y, h.y, sx);
                  sy = fmaf(aa.x, h.y, sy); sy = fmaf(aa.y, h.x, sy);
                  const float2 bb = a.links32[site[xm] * d + mu], k = g32[xm];
                  sx = fmaf(bb.x, k.x, sx); sx = fmaf(bb.y, k.y, sx);
                  sy = fmaf(bb.x, k.y, sy); sy = fmaf(-bb.y, k.x, sy);
                }
                const float n2 = fmaf(sx, sx, sy * sy);
                if (!(n2 > 0.f)) continue;
                const float rr = rsqrtf(n2) * om;
                const float2 gx = g32[p];
                const float vx = fmaf(sx, rr, om1 * gx.x), vy = fmaf(sy, rr, om1 * gx.y);
                const float q = rsqrtf(fmaf(vx, vx, vy * vy));
                g32[p] = make_float2(vx * q, vy * q);
              }
              __syncwarp(tmask);
            }
            ++relax32_sweeps;
            if (sw % 16 == 15) {
              // FP32 residual; stop near the FP32 floor
              float r32 = 0.f;
              for (int p = tl; p < V; p += T) {
                const uint4 nb = nbp[p];
                float sx = 0.f, sy = 0.f;
                for (int mu = 0; mu < d; ++mu) {
                  const unsigned wd = nb_word(nb, mu);
                  const int xp = wd & 0xffffu, xm = wd >> 16;
                  const float2 aa = a.links32[site[p] * d + mu], h = g32[xp];
                  sx = fmaf(aa.x, h.x, sx); sx = fmaf(-aa.y, h.y, sx);
                  sy = fmaf(aa.x, h.y, sy); sy = fmaf(aa.y, h.x, sy);
                  const float2 bb = a.links32[site[xm] * d + mu], k = g32[xm];
                  sx = fmaf(bb.x, k.x, sx); sx = fmaf(bb.y, k.y, sx);
                  sy = fmaf(bb.x, k.y, sy); sy = fmaf(-bb.y, k.x, sy);
                }
                const float2 gx = g32[p];
                const float dv = fmaf(gx.x, sy, -gx.y * sx);
                r32 = fmaxf(r32, dv * dv);
              }
              r32 = team_max(r32, T, tmask);
              if (r32 < 1e-12f) break;
            }
          }
          for (int p = tl; p < V; p += T) {
            const float2 gx = g32[p];
            const double px = f2d_bits(gx.x), py = f2d_bits(gx.y);
            const double n2 = fma(px, px, py * py);
            double q = fma(-0.5, n2, 1.5);
            q = q * fma(-0.5 * n2, q * q, 1.5);
            g[p] = make_double2(px * q, py * q);
          }
          __syncwarp(tmask);
        }
        double r_prev = 1e300;
        int inner_cap = a.inner_max;
        for (int it = 0;; ++it) {
          // (1) FP64 divergence; the FP32 copy feeds the inner solve
          r = 0.0;
          for (int p = tl; p < V; p += T) {
            const double2 S = staple_dfma(u, g, nbp[p], p, d, V);
            const double2 gx = g[p];
            const double dv = fma(gx.x, S.y, -gx.y * S.x);
            b[p] = d2f_bits(dv);
            r = dmax_pos(r, dv * dv);
          }
          ++c_pass;
          for (int o = T >> 1; o > 0; o >>= 1) r = dmax_pos(r, __shfl_xor_sync(tmask, r, o));
          if (dless_pos(r, a.eps)) { conv = true; break; }
          if (it >= a.newton_max) break;
          if (!dless_pos(r, 0.25 * r_prev)) inner_cap = min(4 * inner_cap, 8192);  // poor step
          r_prev = r;
          ++c_newton;
          // (2) Jacobian (FP32 link weights of the current state) and 1/D
          for (int p = tl; p < V; p += T) {
            const double2 gx = g[p];
            const float gxx = d2f_bits(gx.x), gxy = d2f_bits(gx.y);
            const uint4 nb = nbp[p];
            for (int mu = 0; mu < d; ++mu) {
              const double2 hd = g[nb_word(nb, mu) & 0xffffu];
              const float hx = d2f_bits(hd.x), hy = d2f_bits(hd.y);
              const double2 ud = u[mu * V + p];
              const float ux = d2f_bits(ud.x), uy = d2f_bits(ud.y);
              const float tx = fmaf(ux, hx, -uy * hy), ty = fmaf(ux, hy, uy * hx);
              w[mu * V + p] = fmaf(gxx, tx, gxy * ty);
            }
            dl[p] = 0.f;
          }
          __syncwarp(tmask);
          float bd = 0.f;
          for (int p = tl; p < V; p += T) {
            const uint4 nb = nbp[p];
            float D = 0.f;
            for (int mu = 0; mu < d; ++mu) D += w[mu * V + p] + w[mu * V + (nb_word(nb, mu) >> 16)];
            const float di = D > 1e-6f ? __frcp_rn(D) : 0.f;
            Dinv[p] = di;
            bd = fmaxf(bd, fabsf(b[p] * di));
          }
          bd = team_max(bd, T, tmask);
          __syncwarp(tmask);
          // (3) FP32 SOR on M delta = div until the corrections stall
          const float om = a.omega_in, om1 = 1.f - a.omega_in;
          int k = 0;
          while (k < inner_cap) {
            float corr = 0.f;
            for (int kk = 0; kk < 8; ++kk, ++k) {
              for (int c = 0; c < G.ncolor; ++c) {
                const int beg = G.color_off[c], end = G.color_off[c + 1];
                for (int p = beg + tl; p < end; p += T) {
                  const uint4 nb = nbp[p];
                  float acc = b[p];
                  for (int mu = 0; mu < d; ++mu) {
                    const unsigned wd = nb_word(nb, mu);
                    const int xp = wd & 0xffffu, xm = wd >> 16;
                    acc = fmaf(w[mu * V + p], dl[xp], acc);
                    acc = fmaf(w[mu * V + xm], dl[xm], acc);
                  }
                  const float t = acc * Dinv[p], old = dl[p];
                  if (kk == 7) corr = fmaxf(corr, fabsf(t - old));
                  dl[p] = fmaf(om, t, om1 * old);
                }
                __syncwarp(tmask);
              }
            }
            corr = team_max(corr, T, tmask);
            if (corr <= a.lin_tol * bd) break;
          }
          c_inner += (unsigned long long)k;
          // (4) FP64 rotation g_x <- g_x exp(i delta_x), |delta| capped at 0.2
          for (int p = tl; p < V; p += T) {
            const float tf = fminf(fmaxf(dl[p], -0.2f), 0.2f);
            const double t = f2d_bits(tf);
            const double t2 = t * t;
            double c, sn;
            if (fabsf(tf) < 1e-3f) {
              c = fma(t2, fma(t2, 1.0 / 24.0, -0.5), 1.0);
              sn = t * fma(t2, -1.0 / 6.0, 1.0);
            } else {
              c = 1.0 - t2 * (0.5 - t2 * (1.0 / 24.0 - t2 * (1.0 / 720.0)));
              sn = t * (1.0 - t2 * (1.0 / 6.0 - t2 * (1.0 / 120.0 - t2 * (1.0 / 5040.0))));
              const double q2 = rsqrt(c * c + sn * sn);
              c *= q2; sn *= q2;
            }
            const double2 gx = g[p];
            g[p] = make_double2(fma(gx.x, c, -gx.y * sn), fma(gx.x, sn, gx.y * c));
          }
          __syncwarp(tmask);
        }
      }
      if (!conv) {
        // last resort: FP64 relaxation sweeps (descent method; slow on this part)
        const double om1 = a.om1, om = a.omega;
        while (extra_sweeps < a.max_sweeps) {
          for (int c = 0; c < G.ncolor; ++c) {
            const int beg = G.color_off[c], end = G.color_off[c + 1];
            for (int p = beg + tl; p < end; p += T) {
              const double2 S = staple_dfma(u, g, nbp[p], p, d, V);
              const double n2 = S.x * S.x + S.y * S.y;
              if (!(n2 > 0.0)) continue;
              const double rr = om * rsqrt(n2);
              const double2 gx = g[p];
              const double vx = fma(S.x, rr, om1 * gx.x), vy = fma(S.y, rr, om1 * gx.y);
              const double q2 = rsqrt(vx * vx + vy * vy);
              g[p] = make_double2(vx * q2, vy * q2);
            }
            __syncwarp(tmask);
          }
          ++extra_sweeps;
          if (extra_sweeps % a.check_every == 0) {
            r = 0.0;
            for (int p = tl; p < V; p += T) {
              const double2 S = staple_dfma(u, g, nbp[p], p, d, V);
              const double2 gx = g[p];
              const double dv = fma(gx.x, S.y, -gx.y * S.x);
              r = dmax_pos(r, dv * dv);
            }
            for (int o = T >> 1; o > 0; o >>= 1) r = dmax_pos(r, __shfl_xor_sync(tmask, r, o));
            if (dless_pos(r, a.eps)) { conv = true; break; }
          }
        }
        c_upd64 += (unsigned long long)extra_sweeps * V;
      }
    }
    c_upd32 += (unsigned long long)relax32_sweeps * V;
    if (tl == 0) {
      a.status[idx] = conv ? kConverged : kNotConverged;
      a.sweeps[idx] += extra_sweeps;
      a.resid[idx] = r;
      if (conv) ++c_conv; else ++c_nconv;
    }
    write_copy64(g, u, nbp, site, G, tl, T, tmask, idx, a.config, a.F, a.fprint);
    __syncwarp(tmask);
  }
  if (tl == 0) {
    atomicAdd(&a.stats[4], c_newton);
    atomicAdd(&a.stats[5], c_fallback);
    atomicAdd(&a.stats[6], c_upd64);
    atomicAdd(&a.stats[7], c_pass);
    atomicAdd(&a.stats[8], c_conv);
    atomicAdd(&a.stats[9], c_nconv);
    atomicAdd(&a.stats[20], c_inner);
    atomicAdd(&a.stats[21], c_upd32);
  }
}

}  // namespace gc
