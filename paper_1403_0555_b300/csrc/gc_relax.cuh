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
#include <type_traits>

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
    if (!(n2 > 1e-30f)) return;      // a vanishing staple leaves the site as it is
    const float r = rsqrt_sfu(n2) * a.omega32;
    const R2 gx = g[p];
    const float vx = fmaf(S.x, r, a.om1_32 * gx.x);
    const float vy = fmaf(S.y, r, a.om1_32 * gx.y);
    const float m2 = fmaf(vx, vx, vy * vy);
    if (m2 > 1e-30f) {
      const float q = rsqrt_sfu(m2);
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

template <class P, int DD>
__global__ void __launch_bounds__(256) relax_kernel(const RelaxArgs a) {
  using R = typename P::R;
  using R2 = typename P::R2;
  extern __shared__ __align__(16) unsigned char smem[];
  const Geom G = a.geom;
  constexpr int d = DD;
  const int V = G.V, T = a.team;
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
// Polish of FP32-relaxed starts (mixed path)
// ---------------------------------------------------------------------------
// Inexact Newton on the gauge angles.  The Jacobian is the Faddeev-Popov
// operator M, the Hessian of Eq. 3 (a lattice Laplacian with weights
// cos(phi^theta)):
//   1. div_x = Im[conj(g_x) S_x] in double-float arithmetic (about 48
//      significant bits, 1e-13 absolute for d = 4); stop below eps / 4;
//   2. FP32: weights w from the state's high parts, then checkerboard SOR on
//      M delta = div until the correction stalls below lin_tol;
//   3. double-float rotation g_x <- g_x exp(i delta_x), back to |g_x| = 1.
// One FP64 pass over the FP64 image of the final state then gives the
// residual that decides convergence (max_x div^2 < eps), the functional
// (Eq. 3), the fingerprint and the canonical copy together.  That pass is the
// only FP64 work of a typical start: on this part the FP64 pipe has about
// 1/64 of the FP32 rate.  Starts the double-float Newton cannot finish (a
// near-singular or indefinite M) get FP64 Newton rounds, FP32 relaxation
// sweeps and, last, FP64 relaxation sweeps, all out of line.  With a redo list
// the main launch hands such starts on instead (after at most four
// contracting Newton steps, or when the FP64 pass rejects them) and the CG
// instance (inner solves by conjugate gradients) reruns them from their FP32
// state.
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
  int u64_smem;                  // FP64 links also in shared memory (else read from links64)
  int8_t* status;                // in: FP32 phase outcome; out: final outcome
  int32_t* sweeps;               // in: FP32 sweeps; out: + FP64 fallback sweeps
  double* resid;
  const float2* state32;         // colour-position order
  double* F;
  double* fprint;
  double2* config;
  unsigned* redo;                // polish_pairs_kernel: starts left to polish_kernel
  unsigned long long* n_redo;
  const unsigned* list;          // polish_kernel: only these batch entries, when set
  const unsigned long long* n_list;
  unsigned long long* stats;     // [4] newton steps, [5] fallbacks, [6] fp64 relaxation site
                                 // updates, [7] fp64 residual passes, [8] / [9] final
                                 // converged / not converged, [20] inner FP32 SOR sweeps,
                                 // [21] FP32 relaxation site updates of the fallback,
                                 // [22] double-float residual passes, [23] starts rerun
                                 // from the redo list
};

// per team: g (16 B per site: double-float float4 or FP64 double2), w (FP32,
// [mu][p]), b, delta, 1/D (FP32) and, for conjugate-gradient inner solves, the
// search direction and M times it
__host__ __device__ inline size_t polish_team_bytes(int V, int d, bool cg = false) {
  return align16((size_t)V * sizeof(double2)) + align16((size_t)V * d * sizeof(float)) +
         (cg ? 5 : 3) * align16((size_t)V * sizeof(float));
}
// per CTA and link: the double-float copy [mu][p], preceded by the FP64 (cos, sin)
// [mu][p] when those fit too
__host__ __device__ inline size_t polish_link_bytes(bool u64_smem) {
  return sizeof(float4) + (u64_smem ? sizeof(double2) : 0);
}

// FP64 links of the polish: colour-major in shared memory, or site-major in
// global memory through the position -> site table (large lattices)
struct Links64 {
  const double2* cm;     // [mu][p] shared, or nullptr
  const double2* sm;     // [x d + mu] global
  const uint16_t* site;
  int V, d;
  __device__ __forceinline__ double2 operator()(int mu, int p) const {
    return cm ? cm[mu * V + p] : __ldg(sm + (size_t)site[p] * d + mu);
  }
};

// ---- double-float arithmetic -------------------------------------------------
// A value is the unevaluated sum hi + lo of two floats (Dekker 1971).  A site
// of a double-float state is the float4 (x_hi, y_hi, x_lo, y_lo).  two_sum is
// Knuth's error-free sum; an FMA gives the exact error of a product.  The _rn
// intrinsics keep the compiler from contracting or reassociating these steps.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// (sh, sl) += (ah + al)(bh + bl), the al * bl term dropped
__device__ __forceinline__ void df_mac(float ah, float al, float bh, float bl, float& sh,
                                       float& sl) {
  const float p = __fmul_rn(ah, bh);
  const float c = __fmaf_rn(ah, bl, __fmaf_rn(al, bh, __fmaf_rn(ah, bh, -p)));
  float s, t;
  two_sum(sh, p, s, t);
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(t, c));
}

// div_x = Im[conj(g_x) S_x] of a double-float state
template <int DD>
__device__ __forceinline__ float df_divergence(const float4* __restrict__ ud,
                                               const float4* __restrict__ gd, const uint4 nb,
                                               int p, int V) {
  float sxh = 0.f, sxl = 0.f, syh = 0.f, syl = 0.f;
#pragma unroll
  for (int mu = 0; mu < DD; ++mu) {
    const unsigned wd = nb_word(nb, mu);
    const int xp = wd & 0xffffu, xm = wd >> 16;
    const float4 a = ud[mu * V + p], h = gd[xp];      // u_{x,mu} g_{x+mu}
    df_mac(a.x, a.z, h.x, h.z, sxh, sxl);
    df_mac(-a.y, -a.w, h.y, h.w, sxh, sxl);
    df_mac(a.x, a.z, h.y, h.w, syh, syl);
    df_mac(a.y, a.w, h.x, h.z, syh, syl);
    const float4 b = ud[mu * V + xm], k = gd[xm];     // conj(u_{x-mu,mu}) g_{x-mu}
    df_mac(b.x, b.z, k.x, k.z, sxh, sxl);
    df_mac(b.y, b.w, k.y, k.w, sxh, sxl);
    df_mac(b.x, b.z, k.y, k.w, syh, syl);
    df_mac(-b.y, -b.w, k.x, k.z, syh, syl);
  }
  const float4 gx = gd[p];
  float dh = 0.f, dl = 0.f;
  df_mac(gx.x, gx.z, syh, syl, dh, dl);
  df_mac(-gx.y, -gx.w, sxh, sxl, dh, dl);
  return __fadd_rn(dh, dl);
}

// (x, y) / |(x, y)| for a double-float pair with |(x, y)|^2 = 1 + eta, |eta| < 1e-6
__device__ __forceinline__ float4 df_unit(float xh, float xl, float yh, float yl) {
  const float px = __fmul_rn(xh, xh), py = __fmul_rn(yh, yh);
  const float ex = __fmaf_rn(xh, xh, -px), ey = __fmaf_rn(yh, yh, -py);
  float s, e;
  two_sum(px, py, s, e);
  // s - 1 is exact for s in [0.5, 2]
  const float rest = __fadd_rn(__fadd_rn(ex, ey),
                               __fmaf_rn(2.f * xh, xl, __fmaf_rn(2.f * yh, yl, e)));
  const float eta = __fadd_rn(__fsub_rn(s, 1.f), rest);
  const float q = __fmul_rn(eta, __fmaf_rn(0.375f, eta, -0.5f));  // (1 + eta)^(-1/2) - 1
  float4 r;
  two_sum(xh, __fmaf_rn(xh, q, xl), r.x, r.z);
  two_sum(yh, __fmaf_rn(yh, q, yl), r.y, r.w);
  return r;
}

// g exp(i t) in double-float, back to |g| = 1 (|t| <= 0.2).  The FP32 factor's
// rounding (about 1e-7 of t) is removed by the next Newton round.
__device__ __forceinline__ float4 df_rotate(const float4 g, float t) {
  const float t2 = t * t;
  const float cm = t2 * fmaf(t2, fmaf(t2, -1.f / 720.f, 1.f / 24.f), -0.5f);  // cos t - 1
  const float sn = t * fmaf(t2, fmaf(t2, 1.f / 120.f, -1.f / 6.f), 1.f);      // sin t
  const float cx = fmaf(g.x, cm, -g.y * sn), cy = fmaf(g.x, sn, g.y * cm);
  float xh, xe, yh, ye;
  two_sum(g.x, cx, xh, xe);
  two_sum(g.y, cy, yh, ye);
  return df_unit(xh, __fadd_rn(g.z, xe), yh, __fadd_rn(g.w, ye));
}

// FP64 image of a double-float state, in place (the same 16 bytes per site)
__device__ __forceinline__ void df_to_fp64(unsigned char* slot, int tl, int T, int V) {
  const float4* gd = reinterpret_cast<const float4*>(slot);
  double2* g = reinterpret_cast<double2*>(slot);
  for (int p = tl; p < V; p += T) {
    const float4 v = gd[p];
    g[p] = make_double2(f2d_bits(v.x) + f2d_bits(v.z), f2d_bits(v.y) + f2d_bits(v.w));
  }
}

// One FP64 pass over an FP64 state in colour-position order: returns the
// team's max_x div(x)^2 and writes record i: the functional (Eq. 3) as
// d V - (1/2) sum_x Re(conj(g_x) S_x) (the staple S_x holds each link once
// forward and once backward, so the sum counts every cos(phi^theta) twice),
// the fingerprint cos(phi^theta) of link (site 0, mu 0) and the canonical
// copy g'_x = g_x conj(g_{V-1}) in site order.
template <int DD>
__device__ __forceinline__ double final_pass64(const Links64& u,
                                               const double2* __restrict__ g, const uint4* nbp,
                                               const uint16_t* site, const Geom& G, int tl, int T,
                                               unsigned mask, long long i, double2* config,
                                               double* Fout, double* fprint) {
  const int V = G.V;
  const double2 gc = g[G.pos_last];
  double r = 0.0, Fp = 0.0;
  for (int p = tl; p < V; p += T) {
    const uint4 nb = nbp[p];
    double sx = 0.0, sy = 0.0;
#pragma unroll
    for (int mu = 0; mu < DD; ++mu) {
      const unsigned wd = nb_word(nb, mu);
      const int xp = wd & 0xffffu, xm = wd >> 16;
      const double2 a = u(mu, p), h = g[xp];
      sx = fma(a.x, h.x, sx); sx = fma(-a.y, h.y, sx);
      sy = fma(a.x, h.y, sy); sy = fma(a.y, h.x, sy);
      const double2 b = u(mu, xm), k = g[xm];
      sx = fma(b.x, k.x, sx); sx = fma(b.y, k.y, sx);
      sy = fma(b.x, k.y, sy); sy = fma(-b.y, k.x, sy);
    }
    const double2 gx = g[p];
    const double dv = fma(gx.x, sy, -gx.y * sx);
    r = dmax_pos(r, dv * dv);
    Fp = fma(gx.x, sx, fma(gx.y, sy, Fp));
    config[(size_t)i * V + site[p]] =
        make_double2(fma(gx.x, gc.x, gx.y * gc.y), fma(gx.y, gc.x, -gx.x * gc.y));
    if (p == 0) {   // site 0 sits at position 0
      const double2 a = u(0, 0), h = g[nb.x & 0xffffu];
      const double tx = fma(a.x, h.x, -a.y * h.y), ty = fma(a.x, h.y, a.y * h.x);
      fprint[i] = fma(gx.x, tx, gx.y * ty);
    }
  }
  for (int o = T >> 1; o > 0; o >>= 1) r = dmax_pos(r, __shfl_xor_sync(mask, r, o));
  Fp = team_sum(Fp, T, mask);
  if (tl == 0) Fout[i] = fma(-0.5, Fp, (double)(DD * V));
  return r;
}

// S_x with DFMA chains (4 per complex term)
__device__ __forceinline__ double2 staple_dfma(const Links64& u, const double2* __restrict__ g,
                                               const uint4 nb, int p, int d) {
  double sx = 0.0, sy = 0.0;
  for (int mu = 0; mu < d; ++mu) {
    const unsigned wd = nb_word(nb, mu);
    const int xp = wd & 0xffffu, xm = wd >> 16;
    const double2 a = u(mu, p), h = g[xp];
    sx = fma(a.x, h.x, sx); sx = fma(-a.y, h.y, sx);
    sy = fma(a.x, h.y, sy); sy = fma(a.y, h.x, sy);
    const double2 b = u(mu, xm), k = g[xm];
    sx = fma(b.x, k.x, sx); sx = fma(b.y, k.y, sx);
    sy = fma(b.x, k.y, sy); sy = fma(-b.y, k.x, sy);
  }
  return make_double2(sx, sy);
}

// Per-team shared-memory views of the polish
struct PolishTeam {
  unsigned char* slot;   // g: double-float float4 or FP64 double2 per position
  float *w, *b, *dl, *Dinv;
  float *pv, *qv;        // conjugate-gradient vectors, or nullptr (SOR)
  int tl, T;
  unsigned mask;
};

// FP32 link weights w = cos(phi^theta) of the state given by (x, y) per
// position (high parts of a double-float state, or an FP32 state) and 1/D;
// returns max |b / D| over the team
template <class GET>
__device__ __forceinline__ float newton_weights(const PolishTeam& t, const float4* ud,
                                                const uint4* nbp, int d, int V, GET gxy) {
  for (int p = t.tl; p < V; p += t.T) {
    const float2 gx = gxy(p);
    const uint4 nb = nbp[p];
    for (int mu = 0; mu < d; ++mu) {
      const float2 h = gxy(nb_word(nb, mu) & 0xffffu);
      const float4 a = ud[mu * V + p];
      const float tx = fmaf(a.x, h.x, -a.y * h.y), ty = fmaf(a.x, h.y, a.y * h.x);
      t.w[mu * V + p] = fmaf(gx.x, tx, gx.y * ty);
    }
    t.dl[p] = 0.f;
  }
  __syncwarp(t.mask);
  float bd = 0.f;
  for (int p = t.tl; p < V; p += t.T) {
    const uint4 nb = nbp[p];
    float D = 0.f;
    for (int mu = 0; mu < d; ++mu) D += t.w[mu * V + p] + t.w[mu * V + (nb_word(nb, mu) >> 16)];
    const float di = D > 1e-6f ? __frcp_rn(D) : 0.f;
    t.Dinv[p] = di;
    bd = fmaxf(bd, fabsf(t.b[p] * di));
  }
  bd = team_max(bd, t.T, t.mask);
  __syncwarp(t.mask);
  return bd;
}

// Jacobi-preconditioned conjugate gradients on M delta = b, M = D - A the
// Faddeev-Popov operator with the weights w.  Iterations grow like the square
// root of M's condition number, where SOR at a fixed omega needs sweeps in
// proportion to it: the solver of the starts whose M is nearly singular.
// Stops when max |D^-1 r| <= lin_tol max |D^-1 b|, at the cap, or when M is not
// positive along a search direction (indefinite Hessian).  b is overwritten by
// the residual; delta (dl) starts at 0.  Returns the iterations.
__device__ __forceinline__ int newton_cg(const PolishTeam& t, const uint4* nbp, int d, int V,
                                         float lin_tol, float bd, int cap) {
  float rz = 0.f;
  for (int p = t.tl; p < V; p += t.T) {
    const float z = t.b[p] * t.Dinv[p];
    t.pv[p] = z;
    rz = fmaf(t.b[p], z, rz);
  }
  rz = team_sum(rz, t.T, t.mask);
  __syncwarp(t.mask);
  int k = 0;
  while (k < cap) {
    ++k;
    float pq = 0.f;
    for (int p = t.tl; p < V; p += t.T) {   // q = M p
      const uint4 nb = nbp[p];
      const float pp = t.pv[p];
      float q = 0.f;
      for (int mu = 0; mu < d; ++mu) {
        const unsigned wd = nb_word(nb, mu);
        const int xp = wd & 0xffffu, xm = wd >> 16;
        q = fmaf(t.w[mu * V + p], pp - t.pv[xp], q);
        q = fmaf(t.w[mu * V + xm], pp - t.pv[xm], q);
      }
      t.qv[p] = q;
      pq = fmaf(pp, q, pq);
    }
    pq = team_sum(pq, t.T, t.mask);
    if (!(pq > 0.f)) break;
    const float alpha = rz / pq;
    float rz1 = 0.f, zmax = 0.f;
    for (int p = t.tl; p < V; p += t.T) {
      t.dl[p] = fmaf(alpha, t.pv[p], t.dl[p]);
      const float r = fmaf(-alpha, t.qv[p], t.b[p]);
      t.b[p] = r;
      const float z = r * t.Dinv[p];
      rz1 = fmaf(r, z, rz1);
      zmax = fmaxf(zmax, fabsf(z));
    }
    rz1 = team_sum(rz1, t.T, t.mask);
    zmax = team_max(zmax, t.T, t.mask);
    if (zmax <= lin_tol * bd) break;
    const float beta = rz1 / rz;
    rz = rz1;
    __syncwarp(t.mask);
    for (int p = t.tl; p < V; p += t.T) t.pv[p] = fmaf(beta, t.pv[p], t.b[p] * t.Dinv[p]);
    __syncwarp(t.mask);
  }
  __syncwarp(t.mask);
  return k;
}

// FP32 checkerboard SOR on M delta = b until the corrections stall (CG in the
// CG instances); returns sweeps / iterations
template <bool CG>
__device__ __forceinline__ int newton_solve(const PolishTeam& t, const uint4* nbp, const Geom& G,
                                            int d, float om, float lin_tol, float bd, int cap) {
  const int V = G.V;
  if constexpr (CG) return newton_cg(t, nbp, d, V, lin_tol, bd, cap);
  const float om1 = 1.f - om;
  int k = 0;
  while (k < cap) {
    float corr = 0.f;
    for (int kk = 0; kk < 8; ++kk, ++k) {
      for (int c = 0; c < G.ncolor; ++c) {
        const int beg = G.color_off[c], end = G.color_off[c + 1];
        for (int p = beg + t.tl; p < end; p += t.T) {
          const uint4 nb = nbp[p];
          float acc = t.b[p];
          for (int mu = 0; mu < d; ++mu) {
            const unsigned wd = nb_word(nb, mu);
            const int xp = wd & 0xffffu, xm = wd >> 16;
            acc = fmaf(t.w[mu * V + p], t.dl[xp], acc);
            acc = fmaf(t.w[mu * V + xm], t.dl[xm], acc);
          }
          const float tt = acc * t.Dinv[p], old = t.dl[p];
          if (kk == 7) corr = fmaxf(corr, fabsf(tt - old));
          t.dl[p] = fmaf(om, tt, om1 * old);
        }
        __syncwarp(t.mask);
      }
    }
    corr = team_max(corr, t.T, t.mask);
    if (corr <= lin_tol * bd) break;
  }
  return k;
}

struct NewtonOut {
  double r;
  int steps, passes, inner;
  bool conv;
};

// Rare path: FP64 Newton rounds on an FP64 state (FP64 residual, FP32 inner
// solve, FP64 rotation).  Stops when max div^2 < eps, after newton_max steps,
// or when the residual rises (M not positive definite here).
template <int DD, bool CG>
__device__ __noinline__ NewtonOut fp64_newton(const PolishTeam t, const Links64 u,
                                              const float4* ud, const uint4* nbp, const Geom G,
                                              double eps, int newton_max, int inner_max,
                                              float om_in, float lin_tol) {
  constexpr int d = DD;
  const int V = G.V;
  double2* g = reinterpret_cast<double2*>(t.slot);
  NewtonOut o{0.0, 0, 0, 0, false};
  double r_prev = 1e300;
  int inner_cap = inner_max;
  for (int it = 0;; ++it) {
    double r = 0.0;
    for (int p = t.tl; p < V; p += t.T) {
      const double2 S = staple_dfma(u, g, nbp[p], p, d);
      const double2 gx = g[p];
      const double dv = fma(gx.x, S.y, -gx.y * S.x);
      t.b[p] = d2f_bits(dv);
      r = dmax_pos(r, dv * dv);
    }
    ++o.passes;
    for (int k = t.T >> 1; k > 0; k >>= 1) r = dmax_pos(r, __shfl_xor_sync(t.mask, r, k));
    o.r = r;
    if (dless_pos(r, eps)) { o.conv = true; break; }
    if (it >= newton_max) break;
    if (it > 0 && !dless_pos(r, r_prev)) break;
    if (!dless_pos(r, 0.25 * r_prev)) inner_cap = min(4 * inner_cap, 8192);
    r_prev = r;
    ++o.steps;
    const float bd = newton_weights(t, ud, nbp, d, V, [&](int q) {
      const double2 v = g[q];
      return make_float2(d2f_bits(v.x), d2f_bits(v.y));
    });
    o.inner += newton_solve<CG>(t, nbp, G, d, om_in, lin_tol, bd, inner_cap);
    for (int p = t.tl; p < V; p += t.T) {
      const float tf = fminf(fmaxf(t.dl[p], -0.2f), 0.2f);
      const double tt = f2d_bits(tf);
      const double t2 = tt * tt;
      double c = 1.0 - t2 * (0.5 - t2 * (1.0 / 24.0 - t2 * (1.0 / 720.0)));
      double sn = tt * (1.0 - t2 * (1.0 / 6.0 - t2 * (1.0 / 120.0 - t2 * (1.0 / 5040.0))));
      const double q2 = rsqrt(c * c + sn * sn);
      c *= q2; sn *= q2;
      const double2 gx = g[p];
      g[p] = make_double2(fma(gx.x, c, -gx.y * sn), fma(gx.x, sn, gx.y * c));
    }
    __syncwarp(t.mask);
  }
  return o;
}

// Rare path: FP32 relaxation sweeps from an FP64 state (a descent method: it
// moves a start that Newton could not finish, e.g. one near a saddle, towards
// its minimum).  The FP32 lattice lives in w (V d floats >= 2V for d >= 2).
// A fixed budget: the residual may rise for a while, so only the FP32 floor
// (max div^2 ~ 1e-11) ends it early.  Returns the sweeps done.
template <int DD>
__device__ __noinline__ int relax32_fallback(const PolishTeam t, const float4* ud,
                                             const uint4* nbp, const Geom G, float om, float om1,
                                             int cap) {
  constexpr int d = DD;
  const int V = G.V;
  const double2* g = reinterpret_cast<const double2*>(t.slot);
  float2* g32 = reinterpret_cast<float2*>(t.w);
  for (int p = t.tl; p < V; p += t.T) g32[p] = make_float2(d2f_bits(g[p].x), d2f_bits(g[p].y));
  __syncwarp(t.mask);
  auto staple32 = [&](int p) {
    const uint4 nb = nbp[p];
    float sx = 0.f, sy = 0.f;
    for (int mu = 0; mu < d; ++mu) {
      const unsigned wd = nb_word(nb, mu);
      const int xp = wd & 0xffffu, xm = wd >> 16;
      const float4 aa = ud[mu * V + p], bb = ud[mu * V + xm];
      const float2 h = g32[xp], k = g32[xm];
      sx = fmaf(aa.x, h.x, sx); sx = fmaf(-aa.y, h.y, sx);
      sy = fmaf(aa.x, h.y, sy); sy = fmaf(aa.y, h.x, sy);
      sx = fmaf(bb.x, k.x, sx); sx = fmaf(bb.y, k.y, sx);
      sy = fmaf(bb.x, k.y, sy); sy = fmaf(-bb.y, k.x, sy);
    }
    return make_float2(sx, sy);
  };
  int sweeps = 0;
  for (int sw = 0; sw < cap; ++sw) {
    for (int c = 0; c < G.ncolor; ++c) {
      const int beg = G.color_off[c], end = G.color_off[c + 1];
      for (int p = beg + t.tl; p < end; p += t.T) {
        const float2 S = staple32(p);
        const float n2 = fmaf(S.x, S.x, S.y * S.y);
        if (!(n2 > 1e-30f)) continue;
        const float rr = rsqrt_sfu(n2) * om;
        const float2 gx = g32[p];
        const float vx = fmaf(S.x, rr, om1 * gx.x), vy = fmaf(S.y, rr, om1 * gx.y);
        const float q = rsqrt_sfu(fmaxf(fmaf(vx, vx, vy * vy), 1e-30f));
        g32[p] = make_float2(vx * q, vy * q);
      }
      __syncwarp(t.mask);
    }
    ++sweeps;
    if (sw % 16 == 15) {
      float r32 = 0.f;
      for (int p = t.tl; p < V; p += t.T) {
        const float2 S = staple32(p), gx = g32[p];
        const float dv = fmaf(gx.x, S.y, -gx.y * S.x);
        r32 = fmaxf(r32, dv * dv);
      }
      r32 = team_max(r32, t.T, t.mask);
      if (r32 < 1e-11f) break;
    }
  }
  return sweeps;
}

struct RelaxOut {
  double r;
  int sweeps;
  bool conv;
};

// Last resort: FP64 relaxation sweeps on an FP64 state until max div^2 < eps
template <int DD>
__device__ __noinline__ RelaxOut relax64_last_resort(const PolishTeam t, const Links64 u,
                                                     const uint4* nbp, const Geom G, double om,
                                                     double om1, double eps, int max_sweeps,
                                                     int check_every) {
  constexpr int d = DD;
  const int V = G.V;
  double2* g = reinterpret_cast<double2*>(t.slot);
  RelaxOut o{0.0, 0, false};
  while (o.sweeps < max_sweeps) {
    for (int c = 0; c < G.ncolor; ++c) {
      const int beg = G.color_off[c], end = G.color_off[c + 1];
      for (int p = beg + t.tl; p < end; p += t.T) {
        const double2 S = staple_dfma(u, g, nbp[p], p, d);
        const double n2 = S.x * S.x + S.y * S.y;
        if (!(n2 > 0.0)) continue;
        const double rr = om * rsqrt(n2);
        const double2 gx = g[p];
        const double vx = fma(S.x, rr, om1 * gx.x), vy = fma(S.y, rr, om1 * gx.y);
        const double q2 = rsqrt(vx * vx + vy * vy);
        g[p] = make_double2(vx * q2, vy * q2);
      }
      __syncwarp(t.mask);
    }
    ++o.sweeps;
    if (o.sweeps % check_every == 0) {
      double r = 0.0;
      for (int p = t.tl; p < V; p += t.T) {
        const double2 S = staple_dfma(u, g, nbp[p], p, d);
        const double2 gx = g[p];
        const double dv = fma(gx.x, S.y, -gx.y * S.x);
        r = dmax_pos(r, dv * dv);
      }
      for (int k = t.T >> 1; k > 0; k >>= 1) r = dmax_pos(r, __shfl_xor_sync(t.mask, r, k));
      o.r = r;
      if (dless_pos(r, eps)) { o.conv = true; break; }
    }
  }
  return o;
}

template <int DD, bool CG>
__global__ void __launch_bounds__(512, 1) polish_kernel(const PolishArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const long long n_items = a.list ? (long long)*a.n_list : a.n;
  if (n_items == 0) return;   // uniform: an empty redo list
  if (a.list && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&a.stats[23], (unsigned long long)n_items);
  const Geom G = a.geom;
  constexpr int d = DD;
  const int V = G.V, T = a.team;
  const int teams_per_warp = 32 / T, warps = blockDim.x >> 5;
  const Smem lay(V, d, polish_link_bytes(a.u64_smem), polish_team_bytes(V, d, CG),
                 warps * teams_per_warp);
  double2* u64s = a.u64_smem ? reinterpret_cast<double2*>(smem + lay.links) : nullptr;
  float4* ud = reinterpret_cast<float4*>(smem + lay.links +
                                         (a.u64_smem ? (size_t)V * d * sizeof(double2) : 0));
  uint4* nbp = reinterpret_cast<uint4*>(smem + lay.nbp);
  uint16_t* site = reinterpret_cast<uint16_t*>(smem + lay.site);
  build_colour_geometry(G, site, nbp, reinterpret_cast<uint16_t*>(smem + lay.pos));
  if (u64s) load_links(u64s, a.links64, site, V, d);
  for (int k = threadIdx.x; k < V * d; k += blockDim.x) {   // double-float split, once per CTA
    const int mu = k / V, p = k - mu * V;
    const double2 v = a.links64[(size_t)site[p] * d + mu];
    const float xh = __double2float_rn(v.x), yh = __double2float_rn(v.y);
    ud[k] = make_float4(xh, yh, __double2float_rn(v.x - (double)xh),
                        __double2float_rn(v.y - (double)yh));
  }
  __syncthreads();
  const Links64 u{u64s, a.links64, site, V, d};

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int tw = lane / T, tl = lane & (T - 1);
  PolishTeam t;
  t.mask = team_mask(T, tw);
  t.tl = tl;
  t.T = T;
  t.slot = smem + lay.team0 + (size_t)(warp * teams_per_warp + tw) * lay.per_team;
  t.w = reinterpret_cast<float*>(t.slot + align16((size_t)V * sizeof(double2)));
  t.b = t.w + align16((size_t)V * d * sizeof(float)) / sizeof(float);
  t.dl = t.b + align16((size_t)V * sizeof(float)) / sizeof(float);
  t.Dinv = t.dl + align16((size_t)V * sizeof(float)) / sizeof(float);
  t.pv = CG ? t.Dinv + align16((size_t)V * sizeof(float)) / sizeof(float) : nullptr;
  t.qv = CG ? t.pv + align16((size_t)V * sizeof(float)) / sizeof(float) : nullptr;
  float4* gd = reinterpret_cast<float4*>(t.slot);
  const double2* g64 = reinterpret_cast<const double2*>(t.slot);
  // double-float Newton runs while eps / 4 is above its noise floor (|div| ~ 1e-13)
  const bool use_df = a.eps >= 1e-25;
  const float eps_df = (float)(0.25 * a.eps);
  // main launch with a redo list: starts Newton does not finish quickly go to
  // the CG instance instead of this kernel's escalating solves and fallbacks
  const bool handoff = !CG && a.redo != nullptr;

  unsigned long long c_newton = 0, c_fallback = 0, c_upd64 = 0, c_pass = 0, c_conv = 0,
                     c_nconv = 0, c_inner = 0, c_upd32 = 0, c_df = 0;
  for (;;) {
    long long idx = 0;
    if (tl == 0) idx = (long long)atomicAdd(a.work_ctr, 1ULL);
    idx = __shfl_sync(t.mask, idx, tw * T);
    if (idx >= n_items) break;
    if (a.list) idx = a.list[idx];
    const int8_t st32 = a.status[idx];
    const float2* s32 = a.state32 + (size_t)idx * V;
    for (int p = tl; p < V; p += T) {
      const float2 v = s32[p];
      gd[p] = df_unit(v.x, 0.f, v.y, 0.f);
    }
    __syncwarp(t.mask);
    bool conv = false, written = false, handed = false;
    double r = 0.0;
    int extra_sweeps = 0;
    if (st32 == kConverged) {
      for (int round = 0; round < 2 && !conv && !handed; ++round) {
        if (round == 1) {
          if (d < 2) break;
          ++c_fallback;
          const int cap32 = a.max_sweeps < 2048 ? a.max_sweeps : 2048;
          const int sw = relax32_fallback<DD>(t, ud, nbp, G, (float)a.omega, (float)a.om1, cap32);
          c_upd32 += (unsigned long long)sw * V;
          const float2* g32 = reinterpret_cast<const float2*>(t.w);
          for (int p = tl; p < V; p += T) {
            const float2 v = g32[p];
            gd[p] = df_unit(v.x, 0.f, v.y, 0.f);
          }
          __syncwarp(t.mask);
        }
        bool dconv = false;
        if (use_df) {
          float r_prev = 3.4e38f;
          int inner_cap = a.inner_max;
          for (int it = 0;; ++it) {
            // (1) double-float divergence; its FP32 rounding feeds the inner solve
            float rf = 0.f;
            for (int p = tl; p < V; p += T) {
              const float dv = df_divergence<DD>(ud, gd, nbp[p], p, V);
              t.b[p] = dv;
              rf = fmaxf(rf, dv * dv);
            }
            ++c_df;
            rf = team_max(rf, T, t.mask);
            if (rf < eps_df) { dconv = true; break; }
            if (it >= (handoff ? min(a.newton_max, 4) : a.newton_max)) break;
            if (it > 0 && !(rf < r_prev)) break;   // rising: M not positive definite here
            if (!(rf < 0.25f * r_prev)) {          // poor step
              if (handoff) break;
              inner_cap = min(4 * inner_cap, 8192);
            }
            r_prev = rf;
            ++c_newton;
            // (2) Jacobian weights from the high parts, (3) FP32 SOR solve
            const float bd = newton_weights(t, ud, nbp, d, V, [&](int q) {
              const float4 v = gd[q];
              return make_float2(v.x, v.y);
            });
            c_inner += (unsigned long long)newton_solve<CG>(t, nbp, G, d, a.omega_in, a.lin_tol, bd,
                                                        inner_cap);
            // (4) g_x <- g_x exp(i delta_x), |delta| capped at 0.2
            for (int p = tl; p < V; p += T)
              gd[p] = df_rotate(gd[p], fminf(fmaxf(t.dl[p], -0.2f), 0.2f));
            __syncwarp(t.mask);
          }
        }
        if (handoff && use_df && !dconv) { handed = true; break; }
        df_to_fp64(t.slot, tl, T, V);
        __syncwarp(t.mask);
        r = final_pass64<DD>(u, g64, nbp, site, G, tl, T, t.mask, idx, a.config, a.F, a.fprint);
        ++c_pass;
        written = true;
        conv = dless_pos(r, a.eps);
        if (!conv && handoff) { handed = true; break; }
        if (!conv) {
          const NewtonOut o = fp64_newton<DD, CG>(t, u, ud, nbp, G, a.eps, a.newton_max, a.inner_max,
                                              a.omega_in, a.lin_tol);
          c_newton += o.steps;
          c_pass += o.passes;
          c_inner += o.inner;
          r = o.r;
          conv = o.conv;
          if (o.steps) written = false;
        }
      }
      if (!conv && !handed) {
        const RelaxOut o = relax64_last_resort<DD>(t, u, nbp, G, a.omega, a.om1, a.eps,
                                                   a.max_sweeps, a.check_every);
        extra_sweeps = o.sweeps;
        c_upd64 += (unsigned long long)o.sweeps * V;
        if (o.sweeps >= a.check_every) r = o.r;
        conv = o.conv;
        if (o.sweeps) written = false;
      }
    } else {
      df_to_fp64(t.slot, tl, T, V);
      __syncwarp(t.mask);
    }
    if (handed) {   // left, with its FP32 state, to the CG instance
      if (tl == 0) a.redo[atomicAdd(a.n_redo, 1ULL)] = (unsigned)idx;
      __syncwarp(t.mask);
      continue;
    }
    if (!written)
      final_pass64<DD>(u, g64, nbp, site, G, tl, T, t.mask, idx, a.config, a.F, a.fprint);
    if (tl == 0) {
      a.status[idx] = conv ? kConverged : kNotConverged;
      a.sweeps[idx] += extra_sweeps;
      a.resid[idx] = r;
      if (conv) ++c_conv; else ++c_nconv;
    }
    __syncwarp(t.mask);
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
    atomicAdd(&a.stats[22], c_df);
  }
}


// ---------------------------------------------------------------------------
// FP32 bulk relaxation, line-owner kernel (even L; the lines of one parity
// fill whole warps: 4^4, 8^3, ...)
// ---------------------------------------------------------------------------
// A team of NL = L^(D-1) threads relaxes one start.  Thread (q, h) owns the
// h-th line along axis 0 among the lines of parity q = (x_1 + ... + x_{D-1})
// mod 2; both parities fill whole warps, so every branch on q is warp-uniform
// and all site loops unroll at compile time.  A thread keeps its line's gauge
// field and all the links touching it in registers: neighbours along axis 0
// never leave the thread, and neighbours along the other axes are read from
// the team's shared copy.  The two sites x_0 = k and k + L/2 of a line have
// the same colour (L/2 even) and are updated together: their values are held
// as packed pairs (re of both, im of both), so each FP32 step is one f32x2
// instruction, and they share one 16-byte slot of the shared copy, stored
// [slot k][parity][h] so that every quarter-warp access touches 8 distinct
// 16-byte words.  Per pair of site updates: 8D + 13 f32x2 ops, 4 MUFU,
// 2(D-1) 16-byte shared loads and 1 store (per site: 8D + 11 FP32 ops after
// the paired form's two extra exact subtractions are taken away).
//
// Residual (exact, at no extra sweep): for the last colour, div = Im[conj(g) S]
// is taken right after the update with the S of that update; for colour 0 it
// is taken in the next sweep's colour-0 phase from the S computed there,
// before that phase's new values are committed.  Together they are
// max_x div(x)^2 of the state after the checked sweep, which is the state kept
// when the check passes.
template <int D, int L>
struct LineGeom {
  static constexpr int NL = (D == 2) ? L : (D == 3 ? L * L : L * L * L);  // lines
  static constexpr int NLH = NL / 2;                                     // per parity
  static constexpr int V = NL * L;
  static_assert(L % 2 == 0, "line kernel needs even L");
  static_assert(NLH % 32 == 0, "each parity must fill whole warps");
};

// compile-time loop: f(integral_constant<int, i>) for i = 0..N-1
template <class F, int... Is>
__device__ __forceinline__ void static_for_impl(F&& f, std::integer_sequence<int, Is...>) {
  (f(std::integral_constant<int, Is>{}), ...);
}
template <int N, class F>
__device__ __forceinline__ void static_for(F&& f) {
  static_for_impl(f, std::make_integer_sequence<int, N>{});
}

// shared-memory float2 access at a 32-bit shared address plus a compile-time
// byte offset (one LDS/STS with an immediate, no address arithmetic)
template <int OFF>
__device__ __forceinline__ float2 lds_f2(unsigned base) {
  float2 v;
  asm volatile("ld.shared.v2.f32 {%0, %1}, [%2+%3];" : "=f"(v.x), "=f"(v.y) : "r"(base), "n"(OFF));
  return v;
}
template <int OFF>
__device__ __forceinline__ void sts_f2(unsigned base, float2 v) {
  asm volatile("st.shared.v2.f32 [%0+%1], {%2, %3};" ::"r"(base), "n"(OFF), "f"(v.x), "f"(v.y) : "memory");
}

template <int OFF>
__device__ __forceinline__ float4 lds_f4(unsigned base) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4+%5];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(base), "n"(OFF));
  return v;
}
template <int OFF>
__device__ __forceinline__ void sts_f4(unsigned base, float4 v) {
  asm volatile("st.shared.v4.f32 [%0+%1], {%2, %3, %4, %5};" ::"r"(base), "n"(OFF), "f"(v.x),
               "f"(v.y), "f"(v.z), "f"(v.w) : "memory");
}

// Two sites of one line, x_0 = k and x_0 = k + L/2, as packed FP32 pairs so
// that each arithmetic step on both is one f32x2 instruction:
// re = (Re z_k, Re z_{k+L/2}), im = (Im z_k, Im z_{k+L/2}).
struct SitePair {
  float2 re, im;
};
__device__ __forceinline__ float2 bcast2(float v) { return make_float2(v, v); }
__device__ __forceinline__ SitePair swapped(const SitePair& p) {
  return {make_float2(p.re.y, p.re.x), make_float2(p.im.y, p.im.x)};
}
__device__ __forceinline__ SitePair site_pair(float4 v) {
  return {make_float2(v.x, v.y), make_float2(v.z, v.w)};
}
__device__ __forceinline__ float4 packed(const SitePair& p) {
  return make_float4(p.re.x, p.re.y, p.im.x, p.im.y);
}

// A fresh random start for the L sites of one line, written to the team's
// shared copy in the paired layout: site x_0 = k sits in slot k mod (L/2)
// (byte address `dst` + slot * `slot_bytes`), real part at float k / (L/2),
// imaginary part at float 2 + k / (L/2).  Kept out of line: start generation
// is rare next to the sweeps, and inlining the Philox rounds per site would
// crowd the sweep loop out of the instruction cache.
__device__ __noinline__ void line_start32(uint64_t seed, uint64_t orbit_id, uint64_t start,
                                          int first_site, int L, unsigned dst, unsigned slot_bytes) {
  const int H = L / 2;
  for (int k = 0; k < L; ++k) {
    const float2 v = random_unit32(seed, orbit_id, start, (uint64_t)(first_site + k));
    const unsigned p = dst + (unsigned)(k % H) * slot_bytes + 4u * (unsigned)(k / H);
    asm volatile("st.shared.f32 [%0], %1;" ::"r"(p), "f"(v.x) : "memory");
    asm volatile("st.shared.f32 [%0+8], %1;" ::"r"(p), "f"(v.y) : "memory");
  }
}

// The same starts, drawn ahead by a kernel of their own into the batch's
// FP32 state buffer (site order), so that the sweep kernel, whose warps are
// few, loads them instead of running the Philox rounds itself.
__global__ void __launch_bounds__(256) start32_kernel(uint64_t seed, uint64_t orbit_id, uint64_t start0,
                                                      long long n, int V, float2* __restrict__ out) {
  // a block per start at a time, its threads over the start's sites
  for (long long i = blockIdx.x; i < n; i += gridDim.x)
    for (int x = threadIdx.x; x < V; x += blockDim.x)
      out[i * V + x] = random_unit32(seed, orbit_id, start0 + (uint64_t)i, (uint64_t)x);
}

// A line's L drawn sites (site order, from start32_kernel) into the team's
// shared copy in line_start32's paired layout
template <int L>
__device__ __forceinline__ void line_load32(const float2* __restrict__ src, unsigned dst, unsigned slot_bytes) {
  constexpr int H = L / 2;
  float2 v[L];
#pragma unroll
  for (int k = 0; k < L; ++k) v[k] = __ldcs(src + k);
#pragma unroll
  for (int k = 0; k < L; ++k) {
    const unsigned p = dst + (unsigned)(k % H) * slot_bytes + 4u * (unsigned)(k / H);
    asm volatile("st.shared.f32 [%0], %1;" ::"r"(p), "f"(v[k].x) : "memory");
    asm volatile("st.shared.f32 [%0+8], %1;" ::"r"(p), "f"(v[k].y) : "memory");
  }
}

__device__ __forceinline__ void team_bar(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

template <int D, int L>
__device__ __forceinline__ int line_parity(int l) {
  int s = 0, t = l;
  for (int mu = 1; mu < D; ++mu) { s += t % L; t /= L; }
  return s & 1;
}

// h-th line (in increasing line index) of parity q
template <int D, int L>
__device__ inline int line_of(int q, int h) {
  int k = -1;
  for (int l = 0; l < LineGeom<D, L>::NL; ++l)
    if (line_parity<D, L>(l) == q && ++k == h) return l;
  return 0;
}
// rank of line l among the lines of its parity
template <int D, int L>
__device__ inline int half_of(int l) {
  const int q = line_parity<D, L>(l);
  int k = 0;
  for (int m = 0; m < l; ++m) k += line_parity<D, L>(m) == q;
  return k;
}

// f32x2 subtraction (PTX sub.rn.f32x2), a - b per half
__device__ __forceinline__ float2 fsub2(float2 a, float2 b) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\t"
      "mov.b64 rb, {%4, %5};\n\t"
      "sub.rn.f32x2 rd, ra, rb;\n\t"
      "mov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return d;
}

template <int D, int L, int TEAMS>
__global__ void __launch_bounds__(LineGeom<D, L>::NL * TEAMS, 1) relax32_lines_kernel(const RelaxArgs a) {
  using LG = LineGeom<D, L>;
  constexpr int NL = LG::NL, NLH = LG::NLH, V = LG::V, NW = NL / 32, H = L / 2;
  static_assert(H % 2 == 0, "the paired sites x_0 = k and k + L/2 must share a colour");
  constexpr int SLOT = 2 * NLH * 16;          // bytes from slot k to slot k + 1 of a team's copy
  extern __shared__ __align__(16) unsigned char smem[];
  const int team = threadIdx.x / NL, tt = threadIdx.x % NL;
  const int q = tt / NLH, h = tt % NLH;      // q is uniform across each warp
  const int bar_id = 1 + team;
  float4* gs = reinterpret_cast<float4*>(smem) + (size_t)team * (V / 2);   // [slot][parity][h]
  float* red = reinterpret_cast<float*>(reinterpret_cast<float4*>(smem) + (size_t)TEAMS * (V / 2)) + team * 32;
  long long* tidx = reinterpret_cast<long long*>(red + 16);

  const int l = line_of<D, L>(q, h);
  int cl[D];                                  // cl[mu] = x_mu of the line, mu >= 1
  {
    int t = l;
    cl[0] = 0;
#pragma unroll
    for (int mu = 1; mu < D; ++mu) { cl[mu] = t % L; t /= L; }
  }
  // shared-memory offsets of the neighbour lines (opposite parity), +mu and -mu
  int nbp[D], nbm[D];
  nbp[0] = nbm[0] = 0;
  {
    int stride = 1;
#pragma unroll
    for (int mu = 1; mu < D; ++mu) {
      const int lp = l + (((cl[mu] + 1) % L) - cl[mu]) * stride;
      const int lm = l + (((cl[mu] + L - 1) % L) - cl[mu]) * stride;
      nbp[mu] = (1 - q) * NLH + half_of<D, L>(lp);
      nbm[mu] = (1 - q) * NLH + half_of<D, L>(lm);
      stride *= L;
    }
  }
  const int own = q * NLH + h;
  // per-thread 32-bit shared addresses of slot 0; slot k sits k*SLOT bytes further
  unsigned snb[D], snm[D];
  const unsigned sgs = (unsigned)__cvta_generic_to_shared(gs);
#pragma unroll
  for (int mu = 0; mu < D; ++mu) { snb[mu] = sgs + 16u * nbp[mu]; snm[mu] = sgs + 16u * nbm[mu]; }
  const unsigned sown = sgs + 16u * own;
  // links touching the line, in registers, paired like the sites:
  // af[k][mu] = u_{x,mu} and ab[k][mu] = u_{x-mu,mu} (mu >= 1) at x_0 = k, k + H;
  // the axis-0 backward links are af[k-1][0], and for slot 0 the links at
  // x_0 = L-1, H-1, which are af[H-1][0] with its halves exchanged
  SitePair af[H][D], ab[H][D];
#pragma unroll
  for (int k = 0; k < H; ++k) {
#pragma unroll
    for (int mu = 0; mu < D; ++mu) {
      const int x0 = k + L * l, x1 = x0 + H;
      const float2 u0 = a.links32[x0 * D + mu], u1 = a.links32[x1 * D + mu];
      af[k][mu] = {make_float2(u0.x, u1.x), make_float2(u0.y, u1.y)};
      if (mu > 0) {
        int s = 1;
#pragma unroll
        for (int m = 1; m < mu; ++m) s *= L;
        const int dm = (((cl[mu] + L - 1) % L) - cl[mu]) * (s * L);
        const float2 b0 = a.links32[(x0 + dm) * D + mu], b1 = a.links32[(x1 + dm) * D + mu];
        ab[k][mu] = {make_float2(b0.x, b1.x), make_float2(b0.y, b1.y)};
      } else {
        ab[k][0] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
      }
    }
  }
  // blend weights: the move (1 - omega) g + omega S/|S| scaled by 1/omega
  // (omega > 0; the renormalisation removes the scale)
  const float2 cg = bcast2(a.om1_32 / a.omega32), tiny = bcast2(1e-30f);

  SitePair g[H];
  unsigned my_sweeps = 0, my_conv = 0, my_nconv = 0;   // thread 0's, per kernel
  auto fetch = [&]() -> long long {
    if (tt == 0) *tidx = (long long)atomicAdd(a.work_ctr, 1ULL);
    team_bar(bar_id, NL);
    const long long v = *tidx;
    team_bar(bar_id, NL);
    return v;
  };
  // new start: generated into the team's shared copy; g is reloaded after the
  // caller's barrier by `reload`
  auto init = [&](long long idx) { line_start32(a.seed, a.orbit_id, a.start0 + idx, L * l, L, sown, SLOT); };
  auto reload = [&]() {
    static_for<H>([&](auto KC) { g[decltype(KC)::value] = site_pair(lds_f4<decltype(KC)::value * SLOT>(sown)); });
  };
  // staples of slot K (compile time): the axis-0 neighbours are the line's own
  // sites (slot K+1 and K-1, across the ends with halves exchanged), the others
  // come from the shared copy, one 16-byte load per neighbour line.
  //   forward  u h:       re = u.re h.re - u.im h.im, im = u.re h.im + u.im h.re
  //   backward conj(u) h: re = u.re h.re + u.im h.im, im = u.re h.im - u.im h.re
  // summed in six chains (three per direction), the subtracted products apart
  auto staple = [&](auto KC, float2& sx, float2& sy) {
    constexpr int K = decltype(KC)::value;
    SitePair gp;
    if constexpr (K + 1 < H) gp = g[K + 1]; else gp = swapped(g[0]);
    // backward axis-0 neighbour: slot K-1; for slot 0 the sites x_0 = L-1 and
    // H-1 (slot H-1 with its halves exchanged), where the products are taken
    // unexchanged and their halves exchanged afterwards
    constexpr int KB = (K >= 1) ? K - 1 : H - 1;
    const SitePair& gm = g[KB];
    const SitePair& ub = af[KB][0];
    const SitePair& uf = af[K][0];
    float2 xp = __fmul2_rn(uf.re, gp.re), xm = __fmul2_rn(uf.im, gp.im);
    float2 yp = __ffma2_rn(uf.im, gp.re, __fmul2_rn(uf.re, gp.im));
    float2 xb = __ffma2_rn(ub.im, gm.im, __fmul2_rn(ub.re, gm.re));
    float2 yb = __fmul2_rn(ub.re, gm.im), ym = __fmul2_rn(ub.im, gm.re);
    if constexpr (K == 0) {
      xb = make_float2(xb.y, xb.x);
      yb = make_float2(yb.y, yb.x);
      ym = make_float2(ym.y, ym.x);
    }
    static_for<D - 1>([&](auto MC) {
      constexpr int mu = decltype(MC)::value + 1;
      const SitePair hp = site_pair(lds_f4<K * SLOT>(snb[mu]));
      const SitePair hm = site_pair(lds_f4<K * SLOT>(snm[mu]));
      const SitePair& A = af[K][mu];
      const SitePair& B = ab[K][mu];
      xp = __ffma2_rn(A.re, hp.re, xp);
      xm = __ffma2_rn(A.im, hp.im, xm);
      yp = __ffma2_rn(A.re, hp.im, yp);
      yp = __ffma2_rn(A.im, hp.re, yp);
      xb = __ffma2_rn(B.re, hm.re, xb);
      xb = __ffma2_rn(B.im, hm.im, xb);
      yb = __ffma2_rn(B.re, hm.im, yb);
      ym = __ffma2_rn(B.im, hm.re, ym);
    });
    sx = __fadd2_rn(fsub2(xp, xm), xb);
    sy = fsub2(__fadd2_rn(yp, yb), ym);
  };
  // overrelaxed move of both sites: ((1 - omega)/omega) g + S/|S|, renormalised
  auto blend = [&](const SitePair& gx, float2 sx, float2 sy) -> SitePair {
    // S = 0 or v = 0 exactly has probability zero; the 1e-30 only keeps the
    // reciprocal square roots finite
    const float2 n2 = __ffma2_rn(sx, sx, __ffma2_rn(sy, sy, tiny));
    const float2 r = make_float2(rsqrt_sfu(n2.x), rsqrt_sfu(n2.y));
    const float2 vx = __ffma2_rn(sx, r, __fmul2_rn(cg, gx.re));
    const float2 vy = __ffma2_rn(sy, r, __fmul2_rn(cg, gx.im));
    const float2 m2 = __ffma2_rn(vx, vx, __ffma2_rn(vy, vy, tiny));
    const float2 qn = make_float2(rsqrt_sfu(m2.x), rsqrt_sfu(m2.y));
    return {__fmul2_rn(vx, qn), __fmul2_rn(vy, qn)};
  };
  // larger squared divergence Im[conj(v) S]^2 of the two sites
  auto div2 = [&](const SitePair& v, float2 sx, float2 sy) -> float {
    const float2 dv = fsub2(__fmul2_rn(v.re, sy), __fmul2_rn(v.im, sx));
    const float2 d2 = __fmul2_rn(dv, dv);
    return fmaxf(d2.x, d2.y);
  };
  auto commit = [&](auto QC, auto CC) {
    constexpr int Q = decltype(QC)::value, C = decltype(CC)::value;
    static_for<H / 2>([&](auto JC) {
      constexpr int K = 2 * decltype(JC)::value + ((C + Q) & 1);
      sts_f4<K * SLOT>(sown, packed(g[K]));
    });
  };
  // Colour c of a parity-Q line: slots K = (c + Q) mod 2, + 2, ...  All staples
  // and moves come before the phase's stores.  `before`: squared divergences
  // before the move (colour 0 of a pending check; the new values then stay in
  // registers, so that the shared copy still holds the checked state until the
  // check is decided), `after`: after it.
  auto phase = [&](auto QC, auto CC, bool before, bool after, bool store) -> float {
    constexpr int Q = decltype(QC)::value, C = decltype(CC)::value;
    float rr = 0.f;
    static_for<H / 2>([&](auto JC) {
      constexpr int K = 2 * decltype(JC)::value + ((C + Q) & 1);
      float2 sx, sy;
      staple(std::integral_constant<int, K>{}, sx, sy);
      if (before) rr = fmaxf(rr, div2(g[K], sx, sy));
      g[K] = blend(g[K], sx, sy);
      if (after) rr = fmaxf(rr, div2(g[K], sx, sy));
    });
    if (store) commit(QC, CC);
    return rr;
  };
  auto warp_max = [](float v) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
  };

  // the whole sweep loop is instantiated per parity (warp-uniform), so no
  // branch on q remains inside it
  auto run = [&](auto QC) {
    using C0 = std::integral_constant<int, 0>;
    using C1 = std::integral_constant<int, 1>;
    long long idx = fetch();
    bool live = idx < a.n;
    if (live) init(idx);
    team_bar(bar_id, NL);
    if (live) reload();
    int sweeps = 0;
    int until = a.check_every;         // countdown to the next checked sweep
    bool pending = false;              // a checked sweep waits for its colour-0 half
    float r1 = 0.f;
    while (live) {
      const float r0 = phase(QC, C0{}, pending, false, !pending);
      if (pending) {
        const float v = warp_max(fmaxf(r0, r1));
        if ((tt & 31) == 0) red[tt >> 5] = v;
        team_bar(bar_id, NL);
        float r = red[0];
#pragma unroll
        for (int w = 1; w < NW; ++w) r = fmaxf(r, red[w]);
        team_bar(bar_id, NL);
        pending = false;
        const bool conv = r < a.eps32;
        if (conv || sweeps >= a.max_sweeps) {
          // keep the checked state (the shared copy), in colour-position order
          // for the polish
          reload();
          static_for<L>([&](auto KC) {
            constexpr int k = decltype(KC)::value;
            const SitePair& p = g[k % H];
            const float2 v = (k < H) ? make_float2(p.re.x, p.im.x) : make_float2(p.re.y, p.im.y);
            const int x = k + L * l;
            const int colour = (k + q) & 1;
            a.state32[(size_t)idx * V + colour * (V / 2) + (x >> 1)] = v;
          });
          if (tt == 0) {
            a.status[idx] = conv ? kConverged : kNotConverged;
            a.sweeps[idx] = sweeps;
            my_sweeps += sweeps;
            if (conv) ++my_conv; else ++my_nconv;
          }
          idx = fetch();
          live = idx < a.n;
          if (live) init(idx);
          sweeps = 0;
          until = a.check_every;
          team_bar(bar_id, NL);
          if (live) reload();
          continue;
        }
        commit(QC, C0{});
      }
      team_bar(bar_id, NL);
      ++sweeps;
      const bool check = --until == 0;
      if (check) until = a.check_every;
      r1 = phase(QC, C1{}, false, check, true);
      pending = check;
      team_bar(bar_id, NL);
    }
  };
  if (q) run(std::integral_constant<int, 1>{}); else run(std::integral_constant<int, 0>{});
  if (tt == 0 && (my_sweeps | my_conv | my_nconv)) {
    atomicAdd(&a.stats[a.stat_base + 0], (unsigned long long)my_sweeps);
    atomicAdd(&a.stats[a.stat_base + 1], (unsigned long long)my_sweeps * V);
    atomicAdd(&a.stats[a.stat_base + 2], (unsigned long long)my_conv);
    atomicAdd(&a.stats[a.stat_base + 3], (unsigned long long)my_nconv);
  }
}

template <int D, int L, int TEAMS>
__host__ inline size_t relax32_lines_smem() {
  return (size_t)TEAMS * LineGeom<D, L>::V * sizeof(float2) + (size_t)TEAMS * 32 * sizeof(float);
}

// ---------------------------------------------------------------------------
// FP32 bulk relaxation on 4^4, one warp per start (two lines per lane)
// ---------------------------------------------------------------------------
// Lane j = a + 2 (x_2 + 4 x_3), a in {0, 1}, owns two lines along axis 0 at
// the same (x_2, x_3): E at x_1 = s + 2a with s = (x_2 + x_3) mod 2 (line
// parity x_1 + x_2 + x_3 even) and O at x_1 + 1.  Besides the axis-0
// neighbours, E's forward and O's backward axis-1 neighbours are the lane's
// own sites, so a site pair reads 5 neighbour lines from the warp's shared
// copy instead of 6.  Every other neighbour line of an E line is an O line of
// another lane and vice versa, so each such read is one uniform 16-byte load
// per lane, touching 8 distinct 16-byte words per quarter warp.  A colour
// phase moves E's slot c and O's slot 1 - c: two independent site pairs per
// lane, in the same paired f32x2 arithmetic as the line kernel.  The start
// never leaves the warp: phases end in __syncwarp, and the residual's maximum
// is a shuffle reduction.  Layout of a warp's copy: [slot k][E, O][lane].
template <int WARPS, int MINB>
__global__ void __launch_bounds__(32 * WARPS, MINB) relax32_sheet_kernel(const RelaxArgs a) {
  constexpr int D = 4, L = 4, H = 2, V = 256;
  constexpr int ROLE = 32 * 16;     // bytes from a slot's E part to its O part
  constexpr int SLOT = 2 * ROLE;    // bytes from slot 0 to slot 1
  extern __shared__ __align__(16) unsigned char smem[];
  const int warp = threadIdx.x >> 5, j = threadIdx.x & 31;
  const unsigned base = (unsigned)__cvta_generic_to_shared(smem) + (unsigned)warp * (2 * SLOT);
  const int x2 = (j >> 1) & 3, x3 = j >> 3;
  const int x1e = ((x2 + x3) & 1) + 2 * (j & 1);
  const int x1[2] = {x1e, (x1e + 1) & 3};
  // byte offset (within a warp's copy) of the lane owning line (y1, y2, y3)
  auto owner = [](int y1, int y2, int y3) -> unsigned {
    const int t = (y1 - ((y2 + y3) & 1) + 4) & 3;
    return 16u * (unsigned)((t >> 1) + 2 * (y2 + 4 * y3));
  };
  const unsigned own = base + 16u * j;
  const unsigned a1e = base + owner((x1e + 3) & 3, x2, x3);      // E's backward axis-1 line (an O line)
  const unsigned a1o = base + owner((x1e + 2) & 3, x2, x3);      // O's forward axis-1 line (an E line)
  unsigned ap[2][2], am[2][2];                                   // [line][mu - 2], +mu and -mu
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    ap[r][0] = base + owner(x1[r], (x2 + 1) & 3, x3);
    am[r][0] = base + owner(x1[r], (x2 + 3) & 3, x3);
    ap[r][1] = base + owner(x1[r], x2, (x3 + 1) & 3);
    am[r][1] = base + owner(x1[r], x2, (x3 + 3) & 3);
  }
  // links, paired like the sites (x_0 = k, k + 2): af[r][k][mu] = u_{x,mu},
  // ab[r][k][mu] = u_{x-mu,mu} for mu = 2, 3, and for E also mu = 1 (O's
  // backward axis-1 link is E's forward one, af[E][k][1])
  SitePair af[2][H][D], ab[2][H][D];
#pragma unroll
  for (int r = 0; r < 2; ++r) {
    const int l = x1[r] + L * (x2 + L * x3);
#pragma unroll
    for (int k = 0; k < H; ++k) {
      const int s0 = k + L * l, s1 = s0 + H;
#pragma unroll
      for (int mu = 0; mu < D; ++mu) {
        const float2 u0 = a.links32[s0 * D + mu], u1 = a.links32[s1 * D + mu];
        af[r][k][mu] = {make_float2(u0.x, u1.x), make_float2(u0.y, u1.y)};
        ab[r][k][mu] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        if (mu >= 2 || (mu == 1 && r == 0)) {
          const int c = mu == 1 ? x1[r] : (mu == 2 ? x2 : x3);
          const int stride = mu == 1 ? L : (mu == 2 ? L * L : L * L * L);
          const int dm = (((c + L - 1) % L) - c) * stride;
          const float2 b0 = a.links32[(s0 + dm) * D + mu], b1 = a.links32[(s1 + dm) * D + mu];
          ab[r][k][mu] = {make_float2(b0.x, b1.x), make_float2(b0.y, b1.y)};
        }
      }
    }
  }
  const float2 cg = bcast2(a.om1_32 / a.omega32), tiny = bcast2(1e-30f);

  SitePair g[2][H];
  unsigned my_sweeps = 0, my_conv = 0, my_nconv = 0;   // lane 0's, per kernel
  auto fetch = [&]() -> long long {
    unsigned long long v = 0;
    if (j == 0) v = atomicAdd(a.work_ctr, 1ULL);
    return (long long)__shfl_sync(0xffffffffu, v, 0);
  };
  // the start, drawn ahead by start32_kernel into this start's slice of the
  // FP32 state buffer (which receives the final state at the end)
  auto init = [&](long long idx) {
#pragma unroll
    for (int r = 0; r < 2; ++r)
      line_load32<L>(a.state32 + (size_t)idx * V + L * (x1[r] + L * (x2 + L * x3)), own + r * ROLE, SLOT);
  };
  auto reload = [&]() {
    static_for<2>([&](auto RC) {
      static_for<H>([&](auto KC) {
        constexpr int R = decltype(RC)::value, K = decltype(KC)::value;
        g[R][K] = site_pair(lds_f4<R * ROLE + K * SLOT>(own));
      });
    });
  };
  // forward term u h and backward term conj(u) h into the six chains
  auto fwd = [](const SitePair& u, const SitePair& h, float2& xp, float2& xm, float2& yp) {
    xp = __ffma2_rn(u.re, h.re, xp);
    xm = __ffma2_rn(u.im, h.im, xm);
    yp = __ffma2_rn(u.re, h.im, yp);
    yp = __ffma2_rn(u.im, h.re, yp);
  };
  auto bwd = [](const SitePair& u, const SitePair& h, float2& xb, float2& yb, float2& ym) {
    xb = __ffma2_rn(u.re, h.re, xb);
    xb = __ffma2_rn(u.im, h.im, xb);
    yb = __ffma2_rn(u.re, h.im, yb);
    ym = __ffma2_rn(u.im, h.re, ym);
  };
  // staples of slot K of line R (compile time)
  auto staple = [&](auto RC, auto KC, float2& sx, float2& sy) {
    constexpr int R = decltype(RC)::value, K = decltype(KC)::value, N = 1 - R;
    SitePair gp;
    if constexpr (K + 1 < H) gp = g[R][K + 1]; else gp = swapped(g[R][0]);
    constexpr int KB = (K >= 1) ? K - 1 : H - 1;
    const SitePair& gm = g[R][KB];
    const SitePair& ub = af[R][KB][0];
    const SitePair& uf = af[R][K][0];
    float2 xp = __fmul2_rn(uf.re, gp.re), xm = __fmul2_rn(uf.im, gp.im);
    float2 yp = __ffma2_rn(uf.im, gp.re, __fmul2_rn(uf.re, gp.im));
    float2 xb = __ffma2_rn(ub.im, gm.im, __fmul2_rn(ub.re, gm.re));
    float2 yb = __fmul2_rn(ub.re, gm.im), ym = __fmul2_rn(ub.im, gm.re);
    if constexpr (K == 0) {      // slot-0 backward axis-0 products were taken unexchanged
      xb = make_float2(xb.y, xb.x);
      yb = make_float2(yb.y, yb.x);
      ym = make_float2(ym.y, ym.x);
    }
    // neighbour lines of the other kind from the shared copy
    const SitePair h2p = site_pair(lds_f4<N * ROLE + K * SLOT>(ap[R][0]));
    const SitePair h2m = site_pair(lds_f4<N * ROLE + K * SLOT>(am[R][0]));
    const SitePair h3p = site_pair(lds_f4<N * ROLE + K * SLOT>(ap[R][1]));
    const SitePair h3m = site_pair(lds_f4<N * ROLE + K * SLOT>(am[R][1]));
    if constexpr (R == 0) {
      const SitePair h1m = site_pair(lds_f4<N * ROLE + K * SLOT>(a1e));
      fwd(af[0][K][1], g[1][K], xp, xm, yp);
      bwd(ab[0][K][1], h1m, xb, yb, ym);
    } else {
      const SitePair h1p = site_pair(lds_f4<N * ROLE + K * SLOT>(a1o));
      fwd(af[1][K][1], h1p, xp, xm, yp);
      bwd(af[0][K][1], g[0][K], xb, yb, ym);
    }
    fwd(af[R][K][2], h2p, xp, xm, yp);
    bwd(ab[R][K][2], h2m, xb, yb, ym);
    fwd(af[R][K][3], h3p, xp, xm, yp);
    bwd(ab[R][K][3], h3m, xb, yb, ym);
    sx = __fadd2_rn(fsub2(xp, xm), xb);
    sy = fsub2(__fadd2_rn(yp, yb), ym);
  };
  auto blend = [&](const SitePair& gx, float2 sx, float2 sy) -> SitePair {
    const float2 n2 = __ffma2_rn(sx, sx, __ffma2_rn(sy, sy, tiny));
    const float2 r = make_float2(rsqrt_sfu(n2.x), rsqrt_sfu(n2.y));
    const float2 vx = __ffma2_rn(sx, r, __fmul2_rn(cg, gx.re));
    const float2 vy = __ffma2_rn(sy, r, __fmul2_rn(cg, gx.im));
    const float2 m2 = __ffma2_rn(vx, vx, __ffma2_rn(vy, vy, tiny));
    const float2 qn = make_float2(rsqrt_sfu(m2.x), rsqrt_sfu(m2.y));
    return {__fmul2_rn(vx, qn), __fmul2_rn(vy, qn)};
  };
  auto div2 = [&](const SitePair& v, float2 sx, float2 sy) -> float {
    const float2 dv = fsub2(__fmul2_rn(v.re, sy), __fmul2_rn(v.im, sx));
    const float2 d2 = __fmul2_rn(dv, dv);
    return fmaxf(d2.x, d2.y);
  };
  // colour c: E's slot c and O's slot 1 - c.  `before`: squared divergences
  // before the move (colour 0 of a pending check), else after it (`after`).
  auto phase = [&](auto CC, bool before, bool after, bool store) -> float {
    constexpr int C = decltype(CC)::value;
    float rr = 0.f;
    float2 sx0, sy0, sx1, sy1;
    staple(std::integral_constant<int, 0>{}, std::integral_constant<int, C>{}, sx0, sy0);
    staple(std::integral_constant<int, 1>{}, std::integral_constant<int, 1 - C>{}, sx1, sy1);
    if (before) rr = fmaxf(div2(g[0][C], sx0, sy0), div2(g[1][1 - C], sx1, sy1));
    g[0][C] = blend(g[0][C], sx0, sy0);
    g[1][1 - C] = blend(g[1][1 - C], sx1, sy1);
    if (after) rr = fmaxf(div2(g[0][C], sx0, sy0), div2(g[1][1 - C], sx1, sy1));
    if (store) {
      sts_f4<C * SLOT>(own, packed(g[0][C]));
      sts_f4<ROLE + (1 - C) * SLOT>(own, packed(g[1][1 - C]));
    }
    return rr;
  };
  auto warp_max = [](float v) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
  };

  long long idx = fetch();
  bool live = idx < a.n;
  if (live) init(idx);
  __syncwarp();
  if (live) reload();
  int sweeps = 0, until = a.check_every;
  bool pending = false;
  float r1 = 0.f;
  while (live) {
    const float r0 = phase(std::integral_constant<int, 0>{}, pending, false, !pending);
    if (pending) {
      const float r = warp_max(fmaxf(r0, r1));
      pending = false;
      const bool conv = r < a.eps32;
      if (conv || sweeps >= a.max_sweeps) {
        // keep the checked state (the shared copy), in colour-position order
        reload();
        static_for<2>([&](auto RC) {
          constexpr int R = decltype(RC)::value;
          const int l = x1[R] + L * (x2 + L * x3);
          static_for<L>([&](auto KC) {
            constexpr int k = decltype(KC)::value;
            const SitePair& p = g[R][k % H];
            const float2 v = (k < H) ? make_float2(p.re.x, p.im.x) : make_float2(p.re.y, p.im.y);
            const int x = k + L * l;
            constexpr int colour = (k + R) & 1;
            a.state32[(size_t)idx * V + colour * (V / 2) + (x >> 1)] = v;
          });
        });
        if (j == 0) {
          a.status[idx] = conv ? kConverged : kNotConverged;
          a.sweeps[idx] = sweeps;
          my_sweeps += sweeps;
          if (conv) ++my_conv; else ++my_nconv;
        }
        idx = fetch();
        live = idx < a.n;
        __syncwarp();
        if (live) init(idx);
        __syncwarp();
        if (live) reload();
        sweeps = 0;
        until = a.check_every;
        continue;
      }
      sts_f4<0>(own, packed(g[0][0]));
      sts_f4<ROLE + SLOT>(own, packed(g[1][1]));
    }
    __syncwarp();
    ++sweeps;
    const bool check = --until == 0;
    if (check) until = a.check_every;
    r1 = phase(std::integral_constant<int, 1>{}, false, check, true);
    pending = check;
    __syncwarp();
  }
  if (j == 0 && (my_sweeps | my_conv | my_nconv)) {
    atomicAdd(&a.stats[a.stat_base + 0], (unsigned long long)my_sweeps);
    atomicAdd(&a.stats[a.stat_base + 1], (unsigned long long)my_sweeps * V);
    atomicAdd(&a.stats[a.stat_base + 2], (unsigned long long)my_conv);
    atomicAdd(&a.stats[a.stat_base + 3], (unsigned long long)my_nconv);
  }
}

template <int WARPS>
__host__ inline size_t relax32_sheet_smem() {
  return (size_t)WARPS * 256 * sizeof(float2);
}

// ---------------------------------------------------------------------------
// Polish for lattices whose lines of each parity fill one warp (4^4, 8^3 ...):
// one warp per start, lane h owns the h-th line of each parity
// ---------------------------------------------------------------------------
// The double-float Newton polish of polish_kernel, with every step's
// arithmetic in the same order.  During the inner solve lane h keeps, for the
// 2L sites of its two lines, the Newton weights (forward and, off axis 0,
// backward), the right-hand side, 1/D and the correction in registers, packed
// in pairs over the sites x_0 = k and k + L/2: axis-0 neighbours are the
// lane's own sites, the other neighbours' corrections are read from the team's
// paired shared copy [k][parity][h], so an inner SOR step on a site pair reads
// 2(D-1) 8-byte words and runs as f32x2 instructions, and the warp
// synchronises with __syncwarp only.  The residual, rotation and FP64 passes run as loops over the lane's
// sites on the shared state (compact code: the whole kernel stays in the
// instruction cache).  The links, double-float and FP64, sit in shared memory
// as [x_0][mu][parity][h].  A start this common path does not finish (FP32
// phase not converged, the double-float Newton stalls, or the FP64 pass
// rejects it) goes to a redo list that polish_kernel reruns from its FP32
// state.
template <int D, int L>
struct PolishPairSmem {
  using LG = LineGeom<D, L>;
  static constexpr size_t u_df = 0;                                         // float4 [L][D][2][NLH]
  static constexpr size_t u_64 = u_df + (size_t)LG::V * D * sizeof(float4);  // double2, same order
  static constexpr size_t team0 = u_64 + (size_t)LG::V * D * sizeof(double2);
  // per team: state [x0][parity][h] (16 B), corrections as pairs over x0 = k,
  // k + L/2 [k][parity][h] (8 B), divergence [x0][parity][h] (4 B)
  static constexpr size_t per_team = (size_t)LG::V * 24;
  static constexpr size_t bytes(int teams) { return team0 + (size_t)teams * per_team; }
};

template <int OFF>
__device__ __forceinline__ float lds_f1(unsigned base) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1+%2];" : "=f"(v) : "r"(base), "n"(OFF));
  return v;
}
template <int OFF>
__device__ __forceinline__ void sts_f1(unsigned base, float v) {
  asm volatile("st.shared.f32 [%0+%1], %2;" ::"r"(base), "n"(OFF), "f"(v) : "memory");
}
template <int OFF>
__device__ __forceinline__ double2 lds_d2(unsigned base) {
  double2 v;
  asm volatile("ld.shared.v2.f64 {%0, %1}, [%2+%3];" : "=d"(v.x), "=d"(v.y) : "r"(base), "n"(OFF));
  return v;
}
template <int OFF>
__device__ __forceinline__ void sts_d2(unsigned base, double2 v) {
  asm volatile("st.shared.v2.f64 [%0+%1], {%2, %3};" ::"r"(base), "n"(OFF), "d"(v.x), "d"(v.y) : "memory");
}

template <int D, int L, int TEAMS>
__global__ void __launch_bounds__(32 * TEAMS, 1) polish_pairs_kernel(const PolishArgs a) {
  using LG = LineGeom<D, L>;
  using SM = PolishPairSmem<D, L>;
  constexpr int NLH = LG::NLH, V = LG::V;
  static_assert(NLH == 32, "one warp holds one line of each parity per lane");
  constexpr int SS = 2 * NLH * 16;   // bytes from site x0 to x0 + 1 of a line: state, links
  constexpr int SD = 2 * NLH * 4;    //                                          divergence
  constexpr int SD2 = 2 * NLH * 8;   // bytes from slot k to k + 1 of the paired corrections
  extern __shared__ __align__(16) unsigned char smem[];
  const int h = threadIdx.x & 31, team = threadIdx.x >> 5;
  unsigned char* tb = smem + SM::team0 + (size_t)team * SM::per_team;

  // links into shared memory, [x0][mu][parity][h]
  for (int e = threadIdx.x; e < 2 * NLH * L * D; e += blockDim.x) {
    const int lq = e % (2 * NLH), rest = e / (2 * NLH), mu = rest % D, k = rest / D;
    const int ql = lq / NLH, hl = lq % NLH;
    const int ll = line_of<D, L>(ql, hl);
    const double2 v = a.links64[(size_t)(k + L * ll) * D + mu];
    const int i = ((k * D + mu) * 2 + ql) * NLH + hl;
    reinterpret_cast<double2*>(smem + SM::u_64)[i] = v;
    const float xh = __double2float_rn(v.x), yh = __double2float_rn(v.y);
    reinterpret_cast<float4*>(smem + SM::u_df)[i] =
        make_float4(xh, yh, __double2float_rn(v.x - (double)xh), __double2float_rn(v.y - (double)yh));
  }
  __syncthreads();

  const unsigned s_st = (unsigned)__cvta_generic_to_shared(tb);
  const unsigned s_dl = s_st + (unsigned)V * 16u;
  const unsigned s_dv = s_dl + (unsigned)V * 4u;
  const unsigned s_udf = (unsigned)__cvta_generic_to_shared(smem + SM::u_df);
  const unsigned s_u64 = (unsigned)__cvta_generic_to_shared(smem + SM::u_64);
  // per parity P: the line, and the correction addresses of its neighbour lines
  // (parity 1 - P) along mu >= 1; element e sits at e*16 past the state and
  // link bases, e*8 past the correction base and e*4 past the divergence base
  int line[2];
  unsigned dlp[2][D], dlm[2][D];
#pragma unroll
  for (int P = 0; P < 2; ++P) {
    const int l = line_of<D, L>(P, h);
    line[P] = l;
    int t = l, stride = 1;
    dlp[P][0] = dlm[P][0] = 0;
#pragma unroll
    for (int mu = 1; mu < D; ++mu) {
      const int c = t % L;
      t /= L;
      const int lp = l + (((c + 1) % L) - c) * stride;
      const int lm = l + (((c + L - 1) % L) - c) * stride;
      dlp[P][mu] = s_dl + 8u * ((1 - P) * NLH + half_of<D, L>(lp));
      dlm[P][mu] = s_dl + 8u * ((1 - P) * NLH + half_of<D, L>(lm));
      stride *= L;
    }
  }
  const bool use_df = a.eps >= 1e-25;
  const float eps_df = (float)(0.25 * a.eps);
  const float om = a.omega_in, om1 = 1.f - a.omega_in;
  // site V-1 (all coordinates L-1): x0 = L-1 of the last line, parity (D-1)(L-1)
  const unsigned st_last = s_st + 16u * ((L - 1) * 2 * NLH + (((D - 1) * (L - 1)) & 1) * NLH + NLH - 1);
  auto warp_max = [&](float v) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
  };
  // the lane's site i = P L + K: own element and the neighbour correction addresses
  auto own_el = [&](int P) { return (unsigned)(P * NLH + h); };
  auto nbp_dl = [&](int P, int mu) { return P ? dlp[1][mu] : dlp[0][mu]; };
  auto nbm_dl = [&](int P, int mu) { return P ? dlm[1][mu] : dlm[0][mu]; };

  // Inner-solve state of the lane's two lines in packed pairs over the sites
  // x0 = k and k + L/2 (slot k; one colour, see relax32_lines_kernel), so an
  // SOR step on both is one f32x2 instruction per term and one 8-byte shared
  // load per neighbour line: right-hand side, 1/D, correction, and the weights
  // w_{x,mu} (wf) and w_{x-mu,mu} for mu >= 1 (wb).  The axis-0 backward
  // weights of slot 0, w at x0 = L-1 and H-1, are wf[H-1][0] with its halves
  // exchanged (w0s).
  constexpr int H = L / 2;
  static_assert(H % 2 == 0, "paired sites x0 = k and k + L/2 must share a colour");
  float2 b2[2][H], Dv2[2][H], dl2[2][H], wf2[2][H][D], wb2[2][H][D], w0s[2];
  unsigned c_newton = 0, c_inner = 0, c_df = 0, c_pass = 0, c_conv = 0;   // lane 0's
  auto el = [](float2& v, int half) -> float& { return half ? v.y : v.x; };

  // Newton weights of the parity-P line from the high parts, 1/D, zero correction
  auto weights = [&](auto PC, float& bd) {
    constexpr int P = decltype(PC)::value;
    const unsigned e = P * NLH + h;
    const unsigned so = s_st + 16u * e, uo = s_udf + 16u * e, dlo = s_dl + 8u * e, dvo = s_dv + 4u * e;
    static_for<L>([&](auto KC) {
      constexpr int K = decltype(KC)::value, k = K % H, hf = K / H;
      el(b2[P][k], hf) = lds_f1<K * SD>(dvo);
      const float4 gv = lds_f4<K * SS>(so);
      static_for<D>([&](auto MC) {
        constexpr int mu = decltype(MC)::value;
        const float4 A = lds_f4<(K * D + mu) * SS>(uo);
        float4 H4;
        if constexpr (mu == 0) H4 = lds_f4<((K + 1) % L) * SS>(so);
        else H4 = lds_f4<K * SS>(s_st + 2u * (dlp[P][mu] - s_dl));
        const float tx = fmaf(A.x, H4.x, -A.y * H4.y), ty = fmaf(A.x, H4.y, A.y * H4.x);
        el(wf2[P][k][mu], hf) = fmaf(gv.x, tx, gv.y * ty);
        if constexpr (mu > 0) {   // w_{x-mu,mu} = Re[conj(g_{x-mu}) u_{x-mu,mu} g_x]
          const unsigned em16 = 2u * (dlm[P][mu] - s_dl);
          const float4 B = lds_f4<(K * D + mu) * SS>(s_udf + em16);
          const float4 G = lds_f4<K * SS>(s_st + em16);
          const float sx = fmaf(B.x, gv.x, -B.y * gv.y), sy = fmaf(B.x, gv.y, B.y * gv.x);
          el(wb2[P][k][mu], hf) = fmaf(G.x, sx, G.y * sy);
        }
      });
    });
    w0s[P] = make_float2(wf2[P][H - 1][0].y, wf2[P][H - 1][0].x);
    static_for<L>([&](auto KC) {
      constexpr int K = decltype(KC)::value, k = K % H, hf = K / H;
      constexpr int KM = (K + L - 1) % L;
      float Dd = 0.f;
      static_for<D>([&](auto MC) {
        constexpr int mu = decltype(MC)::value;
        if constexpr (mu == 0) Dd += el(wf2[P][k][0], hf) + el(wf2[P][KM % H][0], KM / H);
        else Dd += el(wf2[P][k][mu], hf) + el(wb2[P][k][mu], hf);
      });
      el(Dv2[P][k], hf) = Dd > 1e-6f ? __frcp_rn(Dd) : 0.f;
      bd = fmaxf(bd, fabsf(el(b2[P][k], hf) * el(Dv2[P][k], hf)));
    });
    static_for<H>([&](auto KC) {
      constexpr int k = decltype(KC)::value;
      dl2[P][k] = make_float2(0.f, 0.f);
      sts_f2<k * SD2>(dlo, dl2[P][k]);
    });
  };
  // one SOR step on slot k of the parity-P line (both sites, each in the order
  // of the scalar update: b, axis 0 forward, axis 0 backward, then per mu >= 1
  // forward and backward); returns max |t - old|
  auto sor = [&](auto PC, auto KC) -> float {
    constexpr int P = decltype(PC)::value, k = decltype(KC)::value;
    float2 fwd, bwd, wbk;
    if constexpr (k + 1 < H) fwd = dl2[P][k + 1]; else fwd = make_float2(dl2[P][0].y, dl2[P][0].x);
    if constexpr (k >= 1) { bwd = dl2[P][k - 1]; wbk = wf2[P][k - 1][0]; }
    else { bwd = make_float2(dl2[P][H - 1].y, dl2[P][H - 1].x); wbk = w0s[P]; }
    float2 acc = __ffma2_rn(wf2[P][k][0], fwd, b2[P][k]);
    acc = __ffma2_rn(wbk, bwd, acc);
    static_for<D - 1>([&](auto MC) {
      constexpr int mu = decltype(MC)::value + 1;
      acc = __ffma2_rn(wf2[P][k][mu], lds_f2<k * SD2>(dlp[P][mu]), acc);
      acc = __ffma2_rn(wb2[P][k][mu], lds_f2<k * SD2>(dlm[P][mu]), acc);
    });
    const float2 t = __fmul2_rn(acc, Dv2[P][k]), old = dl2[P][k];
    dl2[P][k] = __ffma2_rn(make_float2(om, om), t, __fmul2_rn(make_float2(om1, om1), old));
    sts_f2<k * SD2>(s_dl + 8u * (P * NLH + h), dl2[P][k]);
    return fmaxf(fabsf(t.x - old.x), fabsf(t.y - old.y));
  };
  // colour C (0 or 1) of both lines: slots k = C xor P, + 2, ...
  auto colour = [&](auto CC, bool last, float& corr) {
    constexpr int C = decltype(CC)::value;
    static_for<2>([&](auto PC) {
      constexpr int P = decltype(PC)::value;
      static_for<H / 2>([&](auto JC) {
        const float c = sor(PC, std::integral_constant<int, 2 * decltype(JC)::value + (C ^ P)>{});
        if (last) corr = fmaxf(corr, c);
      });
    });
    __syncwarp();
  };

  for (;;) {
    long long idx = 0;
    if (h == 0) idx = (long long)atomicAdd(a.work_ctr, 1ULL);
    idx = __shfl_sync(0xffffffffu, idx, 0);
    if (idx >= a.n) break;
    const int8_t st32 = a.status[idx];
#pragma unroll 1
    for (int i = 0; i < 2 * L; ++i) {   // promote the FP32 state
      const int P = i / L, K = i % L;
      const int x = K + L * (P ? line[1] : line[0]);
      const float2 v = a.state32[(size_t)idx * V + ((K + P) & 1) * (V / 2) + (x >> 1)];
      sts_f4<0>(s_st + 16u * own_el(P) + (unsigned)K * SS, df_unit(v.x, 0.f, v.y, 0.f));
    }
    __syncwarp();
    bool ok = false;
    // FP64 image in place (the last warp reduction ended every lane's
    // double-float reads), then one FP64 pass: residual, functional,
    // fingerprint, canonical copy; true if max div^2 < eps
    auto fp64_pass = [&]() -> bool {
        // FP64 image in place (the last reduction ended every lane's double-float
        // reads), then one FP64 pass: residual, functional, fingerprint, copy
#pragma unroll 1
        for (int i = 0; i < 2 * L; ++i) {
          const unsigned sa = s_st + 16u * own_el(i / L) + (unsigned)(i % L) * SS;
          const float4 v = lds_f4<0>(sa);
          sts_d2<0>(sa, make_double2(f2d_bits(v.x) + f2d_bits(v.z), f2d_bits(v.y) + f2d_bits(v.w)));
        }
        __syncwarp();
        double2 gc;
        asm volatile("ld.shared.v2.f64 {%0, %1}, [%2];" : "=d"(gc.x), "=d"(gc.y) : "r"(st_last));
        double r = 0.0, Fp = 0.0;
#pragma unroll 1
        for (int i = 0; i < 2 * L; ++i) {
          const int P = i / L, K = i % L;
          const unsigned e = own_el(P);
          const unsigned so = s_st + 16u * e, uo = s_u64 + 16u * e + (unsigned)(K * D) * SS;
          // the staple S_x = sum_mu [u_{x,mu} g_{x+mu} + conj(u_{x-mu,mu}) g_{x-mu}]
          double sx = 0.0, sy = 0.0;
#pragma unroll
          for (int mu = 0; mu < D; ++mu) {
            double2 A, H, B, G;
            if (mu == 0) {
              A = lds_d2<0>(uo);
              H = lds_d2<0>(so + (unsigned)((K + 1) % L) * SS);
              B = lds_d2<0>(s_u64 + 16u * e + (unsigned)(((K + L - 1) % L) * D) * SS);
              G = lds_d2<0>(so + (unsigned)((K + L - 1) % L) * SS);
            } else {
              const unsigned ep16 = 2u * (nbp_dl(P, mu) - s_dl), em16 = 2u * (nbm_dl(P, mu) - s_dl);
              A = lds_d2<0>(uo + (unsigned)mu * SS);
              H = lds_d2<0>(s_st + ep16 + (unsigned)K * SS);
              B = lds_d2<0>(s_u64 + em16 + (unsigned)(K * D + mu) * SS);
              G = lds_d2<0>(s_st + em16 + (unsigned)K * SS);
            }
            sx = fma(A.x, H.x, sx); sx = fma(-A.y, H.y, sx);
            sy = fma(A.x, H.y, sy); sy = fma(A.y, H.x, sy);
            sx = fma(B.x, G.x, sx); sx = fma(B.y, G.y, sx);
            sy = fma(B.x, G.y, sy); sy = fma(-B.y, G.x, sy);
          }
          const double2 gx = lds_d2<0>(so + (unsigned)K * SS);
          // divergence Im(conj(g_x) S_x); and Re(conj(g_x) S_x), whose sum
          // over the sites counts every link's cos(phi^theta) twice
          const double dv = fma(gx.x, sy, -gx.y * sx);
          r = dmax_pos(r, dv * dv);
          Fp = fma(gx.x, sx, fma(gx.y, sy, Fp));
          const int x = K + L * (P ? line[1] : line[0]);
          a.config[(size_t)idx * V + x] =
              make_double2(fma(gx.x, gc.x, gx.y * gc.y), fma(gx.y, gc.x, -gx.x * gc.y));
          if (x == 0) {   // site 0: cos(phi^theta) of its mu = 0 link
            const double2 A = lds_d2<0>(uo), H = lds_d2<0>(so + (unsigned)SS);
            const double tx = fma(A.x, H.x, -A.y * H.y), ty = fma(A.x, H.y, A.y * H.x);
            a.fprint[idx] = fma(gx.x, tx, gx.y * ty);
          }
        }
        ++c_pass;
        for (int o = 16; o > 0; o >>= 1) {
          r = dmax_pos(r, __shfl_xor_sync(0xffffffffu, r, o));
          Fp += __shfl_xor_sync(0xffffffffu, Fp, o);
        }
        const bool pass = dless_pos(r, a.eps);
        if (pass && h == 0) {
          a.F[idx] = fma(-0.5, Fp, (double)(D * V));   // Eq. 3: sum over links of 1 - cos(phi^theta)
          a.resid[idx] = r;
          a.status[idx] = kConverged;
          ++c_conv;
        }
        return pass;
    };
    // after a rejected FP64 pass: the FP64 image split back into double-float
    auto back_to_df = [&]() {
#pragma unroll 1
      for (int i = 0; i < 2 * L; ++i) {
        const unsigned sa = s_st + 16u * own_el(i / L) + (unsigned)(i % L) * SS;
        const double2 v = lds_d2<0>(sa);
        const float xh = __double2float_rn(v.x), yh = __double2float_rn(v.y);
        sts_f4<0>(sa, make_float4(xh, yh, __double2float_rn(v.x - (double)xh),
                                  __double2float_rn(v.y - (double)yh)));
      }
      __syncwarp();
    };
    if (st32 == kConverged && use_df) {
      float r_prev = 3.4e38f;
      const int inner_cap = a.inner_max;
      bool dconv = false, verify = false;
      for (int it = 0;; ++it) {
        if (verify) {   // the FP64 pass in place of the double-float check
          verify = false;
          if (fp64_pass()) { ok = true; break; }
          back_to_df();
        }
        // double-float divergence of the lane's sites (order of df_divergence)
        float rf = 0.f;
#pragma unroll 1
        for (int i = 0; i < 2 * L; ++i) {
          const int P = i / L, K = i % L;
          const unsigned e = own_el(P);
          const unsigned so = s_st + 16u * e, uo = s_udf + 16u * e + (unsigned)(K * D) * SS;
          float sxh = 0.f, sxl = 0.f, syh = 0.f, syl = 0.f;
#pragma unroll
          for (int mu = 0; mu < D; ++mu) {
            float4 A, H, B, G;
            if (mu == 0) {
              A = lds_f4<0>(uo);
              H = lds_f4<0>(so + (unsigned)((K + 1) % L) * SS);
              B = lds_f4<0>(s_udf + 16u * e + (unsigned)(((K + L - 1) % L) * D) * SS);
              G = lds_f4<0>(so + (unsigned)((K + L - 1) % L) * SS);
            } else {
              const unsigned ep16 = 2u * (nbp_dl(P, mu) - s_dl), em16 = 2u * (nbm_dl(P, mu) - s_dl);
              A = lds_f4<0>(uo + (unsigned)mu * SS);
              H = lds_f4<0>(s_st + ep16 + (unsigned)K * SS);
              B = lds_f4<0>(s_udf + em16 + (unsigned)(K * D + mu) * SS);
              G = lds_f4<0>(s_st + em16 + (unsigned)K * SS);
            }
            df_mac(A.x, A.z, H.x, H.z, sxh, sxl);
            df_mac(-A.y, -A.w, H.y, H.w, sxh, sxl);
            df_mac(A.x, A.z, H.y, H.w, syh, syl);
            df_mac(A.y, A.w, H.x, H.z, syh, syl);
            df_mac(B.x, B.z, G.x, G.z, sxh, sxl);
            df_mac(B.y, B.w, G.y, G.w, sxh, sxl);
            df_mac(B.x, B.z, G.y, G.w, syh, syl);
            df_mac(-B.y, -B.w, G.x, G.z, syh, syl);
          }
          const float4 gx = lds_f4<0>(so + (unsigned)K * SS);
          float dh = 0.f, dlo = 0.f;
          df_mac(gx.x, gx.z, syh, syl, dh, dlo);
          df_mac(-gx.y, -gx.w, sxh, sxl, dh, dlo);
          const float dv = __fadd_rn(dh, dlo);
          sts_f1<0>(s_dv + 4u * e + (unsigned)K * SD, dv);
          rf = fmaxf(rf, dv * dv);
        }
        ++c_df;
        rf = warp_max(rf);
        if (rf < eps_df) { dconv = true; break; }
        // a start Newton does not contract quickly (near-singular or
        // indefinite M) leaves this kernel at once, for polish_kernel's
        // escalating inner solves and fallbacks
        if (it >= (a.newton_max < 4 ? a.newton_max : 4)) break;
        if (it > 0 && !(rf < 0.25f * r_prev)) break;
        r_prev = rf;
        ++c_newton;
        float bd = 0.f;
        weights(std::integral_constant<int, 0>{}, bd);
        weights(std::integral_constant<int, 1>{}, bd);
        bd = warp_max(bd);   // also orders the zeroed corrections before the sweeps
        int k = 0;
        while (k < inner_cap) {
          float corr = 0.f;
          for (int kk = 0; kk < 8; ++kk, ++k) {
            colour(std::integral_constant<int, 0>{}, kk == 7, corr);
            colour(std::integral_constant<int, 1>{}, kk == 7, corr);
          }
          corr = warp_max(corr);
          if (corr <= a.lin_tol * bd) break;
        }
        c_inner += (unsigned)k;
#pragma unroll 1
        for (int i = 0; i < 2 * L; ++i) {   // g_x <- g_x exp(i delta_x), |delta| capped at 0.2
          const int P = i / L, K = i % L;
          const unsigned e = own_el(P);
          const unsigned sa = s_st + 16u * e + (unsigned)K * SS;
          const float t = lds_f1<0>(s_dl + 8u * e + (unsigned)(K % H) * SD2 + 4u * (unsigned)(K / H));
          sts_f4<0>(sa, df_rotate(lds_f4<0>(sa), fminf(fmaxf(t, -0.2f), 0.2f)));
        }
        __syncwarp();
        // a step taken from max div^2 < 1e-16 (the second, typically) lands
        // below eps: check that with the FP64 pass directly
        verify = r_prev < 1e-16f;
      }
      if (dconv) ok = fp64_pass();
    }
    if (!ok && h == 0) a.redo[atomicAdd(a.n_redo, 1ULL)] = (unsigned)idx;
    __syncwarp();
  }
  if (h == 0) {
    atomicAdd(&a.stats[4], (unsigned long long)c_newton);
    atomicAdd(&a.stats[7], (unsigned long long)c_pass);
    atomicAdd(&a.stats[8], (unsigned long long)c_conv);
    atomicAdd(&a.stats[20], (unsigned long long)c_inner);
    atomicAdd(&a.stats[22], (unsigned long long)c_df);
  }
}

}  // namespace gc
