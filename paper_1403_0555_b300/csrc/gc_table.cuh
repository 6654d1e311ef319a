// Device table of distinct canonical copies (deduplication after fixing the
// global phase) and the paper-style set of quantised minima.
//
// Identity: two canonical copies (theta'_{V-1} = 0) are the same iff
// max_x |g'_A(x) - g'_B(x)| <= delta (chord distance, = angle to O(delta^3)).
// Copies of one stationary point share F to far below the bucket width wF and
// share the fingerprint c0 = cos(phi^theta) of link (site 0, mu 0) to far
// below wT, so candidates live in the 3 x 3 neighbouring (F, c0) buckets.
//
// Three kernels per batch.  dedup_kernel (a warp per start) finds or inserts
// each converged start's copy and records it in copy_of; an insert holds the
// locks of its three F-neighbour buckets (taken in ascending lock index, so
// no cycle can form), so every entry it may read or change sits under a held
// lock and no copy is inserted twice.  count_kernel (a thread per start)
// then adds each start to its copy's count and first start, and to the
// paper-style F set, with the starts of a warp that share a copy (or an F
// key) grouped first, so a copy that most starts reach costs one atomic per
// warp instead of one per start.  fixup_kernel gives every copy created in
// the batch the configuration and F of its lowest start.  The outcome is
// independent of the interleaving: count = number of starts that reached the
// copy, first_start = the lowest of those start indices, and the
// representative configuration and F of that start.  Every lock wait is
// bounded; a start whose wait runs out is marked kDedupFailed and the call
// reports a timeout.
#pragma once
#include "gc_common.cuh"

namespace gc {

struct TableView {
  double2* cfg;            // cap * V
  double* F;
  long long* q;            // F bucket
  int* t;                  // fingerprint bucket
  unsigned long long* first_start;
  unsigned long long* rep_start;   // start whose configuration cfg holds
  unsigned long long* count;
  int* next;
  double* lambda2;
  int* region;             // -1 untested, 0 out, 1 in, 2 marginal
  int* head;               // nb buckets
  int* lock;               // nl locks
  unsigned int* n_entries;
  unsigned int* new_list;  // entries created by the current batch
  unsigned int* n_new;
  unsigned long long* f8;  // open-addressing set of floor(F_norm * 1e8)
  unsigned long long* f8n; // starts reaching each slot's key
  unsigned long long* n_f8;
  int* err;                // [0] lock timeout, [1] pool overflow, [2] F8 set full
  unsigned int cap;
  unsigned int nb_mask, nl_mask, f8_mask;
  double wF, wT, tolF, delta2, f8_links;  // f8_links = d V (F_norm = F / (d V))
  double inv_wF, inv_wT;   // 1 / wF, 1 / wT: bucket keys by multiplication
  int f8_only;             // GC_DEDUP_F8: the F set only, no configuration table
  long long lock_spins;    // tries before a lock wait gives up (kLockSpins by default)
};

constexpr unsigned long long kF8Empty = ~0ULL;
constexpr long long kLockSpins = 1LL << 22;

__device__ __forceinline__ unsigned bucket_of(const TableView& T, long long q, int t) {
  return (unsigned)(mix64((unsigned long long)q * 0x9E3779B97F4A7C15ULL + (unsigned)t) & T.nb_mask);
}
__device__ __forceinline__ unsigned lock_of(const TableView& T, long long q) {
  return (unsigned)(mix64((unsigned long long)q) & T.nl_mask);
}

__device__ inline bool acquire(int* lk, long long spins) {
  unsigned ns = 32;
  for (long long s = 0; s < spins; ++s) {
    if (atomicCAS(lk, 0, 1) == 0) { __threadfence(); return true; }
    __nanosleep(ns);
    if (ns < 1024) ns <<= 1;
  }
  return false;
}
__device__ inline void release(int* lk) {
  __threadfence();
  atomicExch(lk, 0);
}

// warp-wide configuration comparison (all 32 lanes): 128 sites a round, the
// loads of a round issued before any comparison so that one round costs one
// memory latency
__device__ inline bool same_copy(const double2* __restrict__ a, const double2* __restrict__ b, int V,
                                 double delta2, int lane) {
  for (int x0 = 0; x0 < V; x0 += 128) {
    double2 p[4], r[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int x = x0 + 32 * c + lane;
      if (x < V) { p[c] = __ldcg(a + x); r[c] = b[x]; }
    }
    // FP64 differences; their squares and the test against delta^2 in FP32
    // (a relative blur of 1e-7 on a threshold that copies of one stationary
    // point undercut, and distinct copies exceed, by many orders)
    bool ok = true;
    const float d2 = (float)delta2;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int x = x0 + 32 * c + lane;
      if (x < V) {
        const float dx = d2f_bits(p[c].x - r[c].x), dy = d2f_bits(p[c].y - r[c].y);
        ok = ok && fmaf(dx, dx, dy * dy) <= d2;
      }
    }
    if (!__all_sync(0xffffffffu, ok)) return false;
  }
  return true;
}

// Search the 3 x 3 (F, fingerprint) neighbourhood for a copy equal to `mine`:
// lanes 0-8 walk the nine bucket lists side by side, and each entry whose
// (F, fingerprint) buckets and F match is compared by the whole warp.
// Safe without locks: entries are only ever prepended, and a representative
// that is being replaced differs from its successor far below delta.
__device__ inline int table_search(const TableView& T, long long q, int t, double F,
                                   const double2* mine, int V, int lane) {
  const long long qq = q + lane / 3 - 1;
  const int tt = t + lane % 3 - 1;
  int e = lane < 9 ? __ldcg(T.head + bucket_of(T, qq, tt)) : -1;
  for (unsigned depth = 0; depth <= T.cap; ++depth) {
    const bool cand = e >= 0 && __ldcg(T.q + e) == qq && __ldcg(T.t + e) == tt &&
                      fabs(__ldcg(T.F + e) - F) <= T.tolF;
    unsigned m = __ballot_sync(0xffffffffu, cand);
    while (m) {
      const int src = __ffs(m) - 1;
      m &= m - 1;
      const int ce = __shfl_sync(0xffffffffu, e, src);
      if (same_copy(T.cfg + (size_t)ce * V, mine, V, T.delta2, lane)) return ce;
    }
    if (e >= 0) e = __ldcg(T.next + e);
    if (!__any_sync(0xffffffffu, e >= 0)) break;
  }
  return -1;
}

struct DedupArgs {
  TableView tab;
  int V;
  long long n;
  uint64_t start0;
  int8_t* status;
  const double* F;
  const double* fprint;
  const double2* config;     // n * V canonical copies of this batch
  int* copy_of;              // out: pool entry of each start (-1 none)
  unsigned long long* stats; // [10] new, [11] hits, [12] failures
};

__global__ void __launch_bounds__(256, 4) dedup_kernel(const DedupArgs a) {
  const TableView& T = a.tab;
  const int lane = threadIdx.x & 31;
  const long long warp0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const int V = a.V;
  unsigned long long c_new = 0, c_hit = 0, c_fail = 0;
  for (long long i = warp0; i < a.n; i += nwarps) {
    if (a.status[i] != kConverged) { if (lane == 0) a.copy_of[i] = -1; continue; }
    const double F = a.F[i];
    const long long q = (long long)floor(F * T.inv_wF);
    const int t = (int)floor((a.fprint[i] + 1.0) * T.inv_wT);
    const unsigned long long start = a.start0 + (unsigned long long)i;
    const double2* mine = a.config + (size_t)i * V;
    if (T.f8_only) { if (lane == 0) a.copy_of[i] = -1; continue; }   // uniform across the warp
    // Search; most starts land on a copy that is already in the table.  On a
    // miss, try once for the three F-neighbour locks (ascending, distinct,
    // non-blocking) and search again: under the locks that search decides
    // the insert; without them, after a backoff, a start waiting on a copy
    // another warp is inserting takes the hit path as soon as it is
    // published instead of queueing on the lock.  (One search call site.)
    unsigned l0 = lock_of(T, q - 1), l1 = lock_of(T, q), l2 = lock_of(T, q + 1);
    {
      unsigned tmp;
      if (l0 > l1) { tmp = l0; l0 = l1; l1 = tmp; }
      if (l1 > l2) { tmp = l1; l1 = l2; l2 = tmp; }
      if (l0 > l1) { tmp = l0; l0 = l1; l1 = tmp; }
    }
    int e = -1;
    bool locked = false, failed = false;
    long long tries = 0;
    unsigned ns = 64;
    for (;;) {
      e = table_search(T, q, t, F, mine, V, lane);
      if (e >= 0 || locked) break;
      int ok = 0;
      if (lane == 0) {
        ok = atomicCAS(&T.lock[l0], 0, 1) == 0;
        if (ok && l1 != l0 && atomicCAS(&T.lock[l1], 0, 1) != 0) { atomicExch(&T.lock[l0], 0); ok = 0; }
        if (ok && l2 != l1 && atomicCAS(&T.lock[l2], 0, 1) != 0) {
          if (l1 != l0) atomicExch(&T.lock[l1], 0);
          atomicExch(&T.lock[l0], 0);
          ok = 0;
        }
        if (ok) __threadfence();
      }
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (ok) { locked = true; __syncwarp(); continue; }
      if (++tries >= T.lock_spins) { failed = true; break; }
      __nanosleep(ns);
      if (ns < 2048) ns <<= 1;
    }
    if (failed) {
      if (lane == 0) { atomicExch(&T.err[0], 1); a.status[i] = kDedupFailed; a.copy_of[i] = -1; }
      ++c_fail;
      continue;
    }
    if (locked) {
      if (e < 0) {
        if (lane == 0) e = (int)atomicAdd(T.n_entries, 1u);
        e = __shfl_sync(0xffffffffu, e, 0);
        if ((unsigned)e >= T.cap) {
          if (lane == 0) { atomicExch(&T.err[1], 1); a.status[i] = kDedupFailed; }
          e = -2;
          ++c_fail;
        } else {
          for (int x = lane; x < V; x += 32) T.cfg[(size_t)e * V + x] = mine[x];
          if (lane == 0) {
            T.F[e] = F; T.q[e] = q; T.t[e] = t;
            T.first_start[e] = start; T.rep_start[e] = start; T.count[e] = 0ULL;
            T.lambda2[e] = __longlong_as_double(0x7ff8000000000000LL);
            T.region[e] = -1;
            // Lock-free prepend: two q values may hash to one list, and their
            // inserters hold different locks.  next[e] and the entry's data are
            // visible before e is published.
            const unsigned b = bucket_of(T, q, t);
            int old = __ldcg(T.head + b);
            for (int k = 0; k < (1 << 24); ++k) {
              T.next[e] = old;
              __threadfence();
              const int seen = atomicCAS(T.head + b, old, e);
              if (seen == old) break;
              old = seen;
            }
            T.new_list[atomicAdd(T.n_new, 1u)] = (unsigned)e;
          }
          ++c_new;
          e = -3 - e;   // marks "newly inserted" (decoded below)
        }
      }
    }
    if (e >= 0) ++c_hit;   // counted, with its first start, by count_kernel
    __syncwarp();
    if (locked && lane == 0) {
      if (l2 != l1) release(&T.lock[l2]);
      if (l1 != l0) release(&T.lock[l1]);
      release(&T.lock[l0]);
    }
    if (lane == 0) a.copy_of[i] = e >= 0 ? e : (e == -2 ? -1 : -3 - e);
    __syncwarp();
  }
  if (lane == 0 && (c_new | c_hit | c_fail)) {
    atomicAdd(&a.stats[10], c_new);
    atomicAdd(&a.stats[11], c_hit);
    atomicAdd(&a.stats[12], c_fail);
  }
}

struct CountArgs {
  TableView tab;
  long long n;
  uint64_t start0;
  const int8_t* status;
  const double* F;
  const int* copy_of;
};

// A thread per start (whole warps, start index increasing with the lane):
// starts of one warp that reached the same copy add their number to its
// count in one atomic, and the group's lowest start (its first lane) to its
// first start; likewise every start that converged (also one whose dedup
// failed) adds itself to the set of floor(F/(dV) 1e8) keys (Section III).
__global__ void __launch_bounds__(256) count_kernel(const CountArgs a) {
  const TableView& T = a.tab;
  const int lane = threadIdx.x & 31;
  const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long base = w0 * 32; base < a.n; base += nw * 32) {
    const long long i = base + lane;
    const bool in = i < a.n;
    const int8_t st = in ? a.status[i] : (int8_t)0;
    const int e = in ? a.copy_of[i] : -1;
    const unsigned me = __match_any_sync(0xffffffffu, e);
    if (e >= 0 && lane == __ffs(me) - 1) {
      atomicAdd(&T.count[e], (unsigned long long)__popc(me));
      atomicMin(&T.first_start[e], a.start0 + (unsigned long long)i);
    }
    const bool conv = st == kConverged || st == kDedupFailed;
    const unsigned long long k8 = conv ? (unsigned long long)floor((a.F[i] / T.f8_links) * 1e8) : kF8Empty;
    const unsigned m8 = __match_any_sync(0xffffffffu, k8);
    if (conv && lane == __ffs(m8) - 1) {
      unsigned slot = (unsigned)(mix64(k8) & T.f8_mask);
      bool placed = false;
      for (unsigned p = 0; p <= T.f8_mask; ++p) {
        const unsigned long long prev = atomicCAS(&T.f8[slot], kF8Empty, k8);
        if (prev == kF8Empty) { atomicAdd(T.n_f8, 1ULL); placed = true; break; }
        if (prev == k8) { placed = true; break; }
        slot = (slot + 1) & T.f8_mask;
      }
      if (placed) atomicAdd(&T.f8n[slot], (unsigned long long)__popc(m8));
      else atomicExch(&T.err[2], 1);
    }
  }
}

// A warp per copy created in this batch: if its lowest start is not the one
// whose configuration it holds, take that start's configuration and F.
__global__ void __launch_bounds__(256) fixup_kernel(const TableView T, int V, uint64_t start0,
                                                    const double* __restrict__ F,
                                                    const double2* __restrict__ config) {
  const int lane = threadIdx.x & 31;
  const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  const unsigned n = *T.n_new;
  for (long long j = w0; j < (long long)n; j += nw) {
    const unsigned e = T.new_list[j];
    const unsigned long long fs = T.first_start[e];
    if (fs == T.rep_start[e]) continue;   // uniform across the warp
    const size_t i = (size_t)(fs - start0);
    for (int x = lane; x < V; x += 32) T.cfg[(size_t)e * V + x] = __ldcg(config + i * V + x);
    if (lane == 0) { T.F[e] = F[i]; T.rep_start[e] = fs; }
  }
}

// Re-thread every pool entry into a (larger) bucket array after growth.
__global__ void relink_kernel(TableView T, unsigned n) {
  for (unsigned e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const unsigned b = bucket_of(T, T.q[e], T.t[e]);
    T.next[e] = atomicExch(&T.head[b], (int)e);
  }
}

// Restore (gc_load_copies): entry e of an empty table from the e-th fetched
// copy.  The canonical configuration is rebuilt from its angles, and the F
// and fingerprint buckets from F and the configuration: the fingerprint is
// cos(phi^theta) of link (site 0, mu 0), Re[conj(g_0) u_{0,0} g_1], which a
// global phase leaves unchanged.  Count, first start (also the
// representative's start), lambda_2 and region are the fetched ones.  A warp
// per copy; relink_kernel then links the entries into their buckets.
__global__ void restore_kernel(TableView T, unsigned n, int V, const double* __restrict__ theta,
                               const double* __restrict__ F, const unsigned long long* __restrict__ first,
                               const unsigned long long* __restrict__ count, const double* __restrict__ lam,
                               const int* __restrict__ region, const double2* __restrict__ links64) {
  const int lane = threadIdx.x & 31;
  const long long w0 = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long e = w0; e < (long long)n; e += nw) {
    for (int x = lane; x < V; x += 32) {
      double sn, cs;
      sincos(theta[(size_t)e * V + x], &sn, &cs);
      T.cfg[(size_t)e * V + x] = make_double2(cs, sn);
    }
    __syncwarp();
    if (lane == 0) {
      const double2 g0 = T.cfg[(size_t)e * V], g1 = T.cfg[(size_t)e * V + 1], u = links64[0];
      const double tx = fma(u.x, g1.x, -u.y * g1.y), ty = fma(u.x, g1.y, u.y * g1.x);
      const double w = fma(g0.x, tx, g0.y * ty);
      T.F[e] = F[e];
      T.q[e] = (long long)floor(F[e] * T.inv_wF);
      T.t[e] = (int)floor((w + 1.0) * T.inv_wT);
      T.first_start[e] = first[e];
      T.rep_start[e] = first[e];
      T.count[e] = count[e];
      T.lambda2[e] = lam[e];
      T.region[e] = region[e];
    }
    __syncwarp();
  }
}

__global__ void fill_int_kernel(int* p, int v, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) p[i] = v;
}
__global__ void fill_u64_kernel(unsigned long long* p, unsigned long long v, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) p[i] = v;
}

// theta'_x = arg g'_x for the first n entries (fetch)
// ---------------------------------------------------------------------------
// Fetch: distinct copies in (F, first start) order
// ---------------------------------------------------------------------------
// ascending order of doubles as unsigned 64-bit keys (negative values too)
__device__ __forceinline__ unsigned long long f64_order_key(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ULL);
}

__global__ void iota_kernel(unsigned* idx, unsigned n) {
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) idx[i] = i;
}

// keys of the second sort pass: F of the entries in first-start order
__global__ void f_keys_kernel(const double* __restrict__ F, const unsigned* __restrict__ idx,
                              unsigned long long* __restrict__ key, unsigned n) {
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    key[i] = f64_order_key(F[idx[i]]);
}

// per-copy records in sorted order
__global__ void gather_meta_kernel(const unsigned* __restrict__ order, unsigned k,
                                   const double* __restrict__ F, const unsigned long long* __restrict__ first,
                                   const unsigned long long* __restrict__ count,
                                   const double* __restrict__ lam, const int* __restrict__ region,
                                   double* oF, unsigned long long* ofirst, unsigned long long* ocount,
                                   double* olam, int* oregion) {
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < k; i += gridDim.x * blockDim.x) {
    const unsigned e = order[i];
    oF[i] = F[e]; ofirst[i] = first[e]; ocount[i] = count[e]; olam[i] = lam[e]; oregion[i] = region[e];
  }
}

// canonical angles theta'_x = arg g'_x of the copies in sorted order
// The canonical angles theta' = arg(c + i s) of the fetched copies, without a
// double-precision arctangent (9 FP64 operations per site; the FP64
// arctangent cost about 46).  Range reduction by angle subtraction: a rough FP32
// estimate of the angle picks the nearest t_j = 2 pi j / kAngleSteps,
// j in [-kAngleSteps/2, kAngleSteps/2]; rotating (c, s) back by t_j leaves
// x = s cos t_j - c sin t_j = sin(theta - t_j) with |theta - t_j| <= pi /
// kAngleSteps plus the estimate's error, and theta = t_j + arcsin x, the
// arcsine summed as its Maclaurin series x + x^3/6 + 3x^5/40 + 5x^7/112 +
// 35x^9/1152 (the first omitted term, 63x^11/2816, is below 1e-22 for
// |x| <= 0.0123).  |(c, s)| = 1 to rounding, so the arcsine of the rotated
// sine is the angle to within 1e-18.  The table holds t_j (the double
// nearest 2 pi j / kAngleSteps) and the cosine and sine of that double,
// computed on the host in extended precision.
constexpr int kAngleSteps = 256;
constexpr int kAngleTable = kAngleSteps + 1;   // [t_j | cos t_j | sin t_j], j + kAngleSteps/2

// A float within 2^-20 relative of a double in [-1, 1] from its high word
// (integer operations only: the exponent re-biased, 20 mantissa bits kept);
// magnitudes below 2^-126 give a signed zero.
__device__ __forceinline__ float rough_float(double v) {
  const unsigned hi = (unsigned)__double2hiint(v);
  const unsigned mag = hi & 0x7fffffffu;
  const unsigned bits = mag < (897u << 20) ? 0u : ((mag - (896u << 20)) << 3);
  return __uint_as_float(bits | (hi & 0x80000000u));
}

__global__ void gather_angles_kernel(const unsigned* __restrict__ order, unsigned k, int V,
                                     const double2* __restrict__ cfg, const double* __restrict__ table,
                                     double* __restrict__ theta) {
  __shared__ double tab[3 * kAngleTable];
  for (int i = threadIdx.x; i < 3 * kAngleTable; i += blockDim.x) tab[i] = table[i];
  __syncthreads();
  const float to_step = (float)kAngleSteps / 6.28318530717958647692f;
  // a block per copy at a time, its threads over the copy's sites
  for (unsigned c = blockIdx.x; c < k; c += gridDim.x) {
    const double2* __restrict__ src = cfg + (size_t)order[c] * V;
    double* __restrict__ dst = theta + (size_t)c * V;
    for (int x = threadIdx.x; x < V; x += blockDim.x) {
      const double2 z = src[x];
      const float est = atan2f(rough_float(z.y), rough_float(z.x));
      const int j = min(max(__float2int_rn(est * to_step), -kAngleSteps / 2), kAngleSteps / 2) + kAngleSteps / 2;
      const double tj = tab[j], cj = tab[kAngleTable + j], sj = tab[2 * kAngleTable + j];
      const double r = fma(z.y, cj, -(z.x * sj));
      const double r2 = r * r;
      double q = fma(r2, 35.0 / 1152.0, 5.0 / 112.0);
      q = fma(r2, q, 3.0 / 40.0);
      q = fma(r2, q, 1.0 / 6.0);
      dst[x] = tj + fma(r * r2, q, r);
    }
  }
}

}  // namespace gc
