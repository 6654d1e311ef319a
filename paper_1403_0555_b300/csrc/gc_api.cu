// C ABI and host runtime of the Gribov-copy enumerator: orbit objects, memory
// admission, batch planning and kernel launches (declarations: gribov.h).
#include "gribov.h"


#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "gc_common.cuh"
#include "gc_fptest.cuh"
#include "gc_relax.cuh"
#include "gc_fptest_lines.cuh"
#include "gc_slab.cuh"
#include "gc_table.cuh"
#include "gc_sort.cuh"
#include "gc_serve.cuh"

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return code;
}

#define GC_CUDA(call)                                                                   \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess) return fail(GC_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

gc_alloc_fn g_alloc = nullptr;
gc_free_fn g_free = nullptr;
void* g_actx = nullptr;

// Serving: while a worker thread runs a request, the device memory it
// allocates is carved from the region of the server's arena that the
// device-side admission gave the request (bump allocation, 256-byte aligned;
// what does not fit comes from the allocator hooks).  Frees of arena memory
// are no-ops: the region goes back whole when the request is done.
struct ArenaScope {
  char* base = nullptr;
  size_t size = 0, used = 0, overflow = 0;
};
thread_local ArenaScope* t_scope = nullptr;
std::mutex g_arena_mu;
std::vector<std::pair<char*, size_t>> g_arenas;

bool in_arena(const void* p) {
  std::lock_guard<std::mutex> lk(g_arena_mu);
  for (const auto& a : g_arenas)
    if ((const char*)p >= a.first && (const char*)p < a.first + a.second) return true;
  return false;
}

void* dev_alloc(size_t n, cudaStream_t s) {
  if (n == 0) n = 16;
  if (t_scope) {
    const size_t off = (t_scope->used + 255) & ~size_t(255);
    if (off + n <= t_scope->size) {
      t_scope->used = off + n;
      return t_scope->base + off;
    }
    t_scope->overflow += n;
  }
  if (g_alloc) return g_alloc(n, (void*)s, g_actx);
  void* p = nullptr;
  if (cudaMalloc(&p, n) != cudaSuccess) { cudaGetLastError(); return nullptr; }
  return p;
}
void dev_free(void* p, cudaStream_t s) {
  if (!p) return;
  if (in_arena(p)) return;
  if (g_free) g_free(p, (void*)s, g_actx);
  else cudaFree(p);
}

struct Buf {
  void* p = nullptr;
  size_t n = 0;
  bool ensure(size_t bytes, cudaStream_t s) {
    if (bytes <= n && p) return true;
    dev_free(p, s);
    p = dev_alloc(bytes, s);
    n = p ? bytes : 0;
    return p != nullptr;
  }
  void release(cudaStream_t s) { dev_free(p, s); p = nullptr; n = 0; }
  template <class T> T* as() const { return reinterpret_cast<T*>(p); }
};

unsigned next_pow2(unsigned long long v) {
  unsigned long long p = 1;
  while (p < v) p <<= 1;
  return (unsigned)p;
}

int sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

size_t max_smem_optin() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return n > 0 ? (size_t)n : 48 * 1024;
}

}  // namespace

enum StatSlot {
  kSweeps = 0, kUpdates = 1, kConv = 2, kNConv = 3, kNewton = 4, kFallback = 5, kUpd64 = 6,
  kPass = 7, kPConv = 8, kPNConv = 9, kNew = 10, kHit = 11, kDFail = 12, kTests = 13,
  kTests64 = 14, kLanczos = 15, kSweeps32 = 16, kUpdates32 = 17, kConv32 = 18, kNConv32 = 19, kInner = 20, kUpd32Fallback = 21,
  kPassDF = 22, kRedo = 23, kLanczos64 = 24, kNumStats = 25
};

// timing events per enqueued batch (stage boundaries; harvest_timing)
constexpr size_t kEvPerBatch = 7;

struct gc_orbit_s {
  int d = 0, L = 0, V = 0, ncolor = 0;
  bool slab = false;   // beyond shared memory: sweeps stream hyperplanes (gc_slab.cuh)
  uint64_t orbit_id = 0;
  gc::Geom geom{};
  int team = 32;
  cudaStream_t alloc_stream = nullptr;
  Buf links64, links32;
  // copy table
  unsigned cap = 0, nb = 0, nl = 0, f8cap = 0;
  Buf t_cfg, t_F, t_q, t_t, t_first, t_rep, t_count, t_next, t_lam, t_region, t_head, t_lock, t_f8, t_f8n;
  Buf t_counters;    // n_entries, n_new (u32) | n_f8 (u64) | err[4] (i32) | n_redo (u32)
  Buf t_newlist;     // new entries of a batch [cap], then those left to FP64 [cap]
  // batch staging
  Buf s_status, s_sweeps, s_resid, s_F, s_fprint, s_config, s_state32, s_copy;
  Buf s_redo;        // lattices beyond shared memory: starts the Newton polish leaves to FP64 sweeps
  Buf s_rate;        // ... and the FP32 sweeps' contraction per start
  Buf work, stats, scratch, theta_tmp;
  Buf sort_keys, sort_idx, sort_tmp;  // fetch ordering: keys [2n], indices [2n], radix-sort histograms
  Buf f8_tmp;                         // F set fetch: keys [2n], starts [2n], counter
  size_t batch_cap = 0;
  uint64_t next_start = 0;
  // per-start records of the last call
  uint64_t rec_first = 0, rec_n = 0;
  std::vector<int8_t> rec_status;
  std::vector<int32_t> rec_sweeps;
  std::vector<double> rec_F;
  std::vector<int32_t> rec_copy;
  // host-side accumulators
  uint64_t n_starts = 0;
  double ms[6] = {0, 0, 0, 0, 0, 0};   // relax, polish (all launches), dedup, FP test, polish redo,
                                       // start draw (part of relax)
  uint64_t launches = 0;   // kernels this orbit launched
  uint64_t enqueued = 0;   // starts enqueued so far (bounds the copy count without a sync)
  std::vector<cudaEvent_t> ev_pool;      // timing events of enqueued batches (kEvPerBatch per batch)
  size_t ev_used = 0;
  bool err_unchecked = false;
  cudaStream_t last_stream = nullptr;    // stream of the orbit's most recent work
  cudaEvent_t fetch_ev[2] = {};          // asynchronous fetch: gathered | copied to the host
  bool fetch_pending = false;            // copies of gc_fetch_copies_async not yet waited for
  int last_precision = GC_FP64;
  cudaEvent_t ev[8] = {};

  unsigned* n_entries() const { return t_counters.as<unsigned>(); }
  unsigned* n_new() const { return t_counters.as<unsigned>() + 1; }
  unsigned long long* n_f8() const { return reinterpret_cast<unsigned long long*>(t_counters.as<char>() + 8); }
  int* err() const { return reinterpret_cast<int*>(t_counters.as<char>() + 16); }
  unsigned* n_redo() const { return reinterpret_cast<unsigned*>(t_counters.as<char>() + 32); }
  unsigned* n_redo2() const { return reinterpret_cast<unsigned*>(t_counters.as<char>() + 40); }

  gc::TableView view() const {
    gc::TableView T{};
    T.cfg = t_cfg.as<double2>();
    T.F = t_F.as<double>();
    T.q = t_q.as<long long>();
    T.t = t_t.as<int>();
    T.first_start = t_first.as<unsigned long long>();
    T.rep_start = t_rep.as<unsigned long long>();
    T.count = t_count.as<unsigned long long>();
    T.next = t_next.as<int>();
    T.lambda2 = t_lam.as<double>();
    T.region = t_region.as<int>();
    T.head = t_head.as<int>();
    T.lock = t_lock.as<int>();
    T.n_entries = n_entries();
    T.new_list = t_newlist.as<unsigned>();
    T.n_new = n_new();
    T.f8 = t_f8.as<unsigned long long>();
    T.f8n = t_f8n.as<unsigned long long>();
    T.n_f8 = n_f8();
    T.err = err();
    T.cap = cap;
    T.nb_mask = nb - 1;
    T.nl_mask = nl - 1;
    T.f8_mask = f8cap - 1;
    T.lock_spins = lock_spins;
    return T;
  }
  long long lock_spins = gc::kLockSpins;   // gc_test_dedup_locks lowers it
  // an orbit a server ran: its results live in the region the server admitted
  // (offset region_off of its arena) until the orbit is destroyed
  gc_server_s* served_by = nullptr;
  uint64_t region_off = 0;
};

// Serving (defined with the server): mail a served orbit's region back
void server_release_region(gc_orbit o);

namespace {

void fill_i32(int* p, int v, size_t n, cudaStream_t s) {
  if (!n) return;
  const int blocks = (int)std::min<size_t>((n + 255) / 256, 4096);
  gc::fill_int_kernel<<<blocks, 256, 0, s>>>(p, v, n);
}
void fill_u64(unsigned long long* p, unsigned long long v, size_t n, cudaStream_t s) {
  if (!n) return;
  const int blocks = (int)std::min<size_t>((n + 255) / 256, 4096);
  gc::fill_u64_kernel<<<blocks, 256, 0, s>>>(p, v, n);
}

// Re-insert the keys of an old F8 set into a new one.
__global__ void f8_rehash_kernel(const unsigned long long* old_set, const unsigned long long* old_cnt,
                                 unsigned old_n, unsigned long long* set, unsigned long long* cnt,
                                 unsigned mask, int* err) {
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < old_n; i += gridDim.x * blockDim.x) {
    const unsigned long long k = old_set[i];
    if (k == gc::kF8Empty) continue;
    unsigned slot = (unsigned)(gc::mix64(k) & mask);
    bool placed = false;
    for (unsigned p = 0; p <= mask; ++p) {
      if (atomicCAS(&set[slot], gc::kF8Empty, k) == gc::kF8Empty) { placed = true; break; }
      slot = (slot + 1) & mask;
    }
    if (placed) cnt[slot] = old_cnt[i];   // keys are unique: the slot is this thread's
    else atomicExch(&err[2], 1);
  }
}

// The occupied slots of the F set, packed (key, starts) in slot order.
__global__ void f8_compact_kernel(const unsigned long long* set, const unsigned long long* cnt, unsigned n,
                                  unsigned long long* keys, unsigned long long* counts, unsigned* ctr,
                                  unsigned limit) {
  for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const unsigned long long k = set[i];
    if (k == gc::kF8Empty) continue;
    const unsigned j = atomicAdd(ctr, 1u);
    if (j < limit) { keys[j] = k; counts[j] = cnt[i]; }
  }
}

// Grow (or create) the copy pool so that it holds at least `need` entries.
// exact: a pool of exactly max(need, 1024) entries even when smaller than the
// current one (moving a served orbit's table out of the serving arena).
int table_reserve(gc_orbit o, unsigned long long need, unsigned cur, cudaStream_t s, bool exact = false) {
  if (!exact && need <= o->cap && o->cap) return GC_OK;
  unsigned long long want = exact ? std::max<unsigned long long>(need, 1024ULL)
                                  : std::max<unsigned long long>(need, o->cap ? 2ULL * o->cap : 1024ULL);
  if (want > 0x7fffffffULL) return fail(GC_ENOMEM, "copy pool would exceed 2^31 entries");
  const unsigned ncap = (unsigned)want;
  const size_t V = o->V;
  Buf cfg, F, q, t, first, rep, count, next, lam, region;
  bool ok = cfg.ensure(ncap * V * sizeof(double2), s) && F.ensure(ncap * 8ull, s) &&
            q.ensure(ncap * 8ull, s) && t.ensure(ncap * 4ull, s) && first.ensure(ncap * 8ull, s) &&
            rep.ensure(ncap * 8ull, s) &&
            count.ensure(ncap * 8ull, s) && next.ensure(ncap * 4ull, s) && lam.ensure(ncap * 8ull, s) &&
            region.ensure(ncap * 4ull, s);
  Buf newlist;
  ok = ok && newlist.ensure(ncap * 8ull, s);
  const unsigned nnb = next_pow2(2ull * ncap);
  Buf head;
  ok = ok && head.ensure(nnb * 4ull, s);
  const unsigned nf8 = next_pow2(4ull * ncap);
  Buf f8, f8n;
  ok = ok && f8.ensure(nf8 * 8ull, s) && f8n.ensure(nf8 * 8ull, s);
  if (!ok) {
    for (Buf* b : {&cfg, &F, &q, &t, &first, &rep, &count, &next, &lam, &region, &newlist, &head, &f8, &f8n})
      b->release(s);
    return fail(GC_ENOMEM, "cannot admit a copy pool of %u entries (%.1f MiB)", ncap,
                ncap * (V * 16.0 + 64.0) / 1048576.0);
  }
  if (cur) {
    GC_CUDA(cudaMemcpyAsync(cfg.p, o->t_cfg.p, cur * V * sizeof(double2), cudaMemcpyDeviceToDevice, s));
    GC_CUDA(cudaMemcpyAsync(F.p, o->t_F.p, cur * 8ull, cudaMemcpyDeviceToDevice, s));
    GC_CUDA(cudaMemcpyAsync(q.p, o->t_q.p, cur * 8ull, cudaMemcpyDeviceToDevice, s));
    GC_CUDA(cudaMemcpyAsync(t.p, o->t_t.p, cur * 4ull, cudaMemcpyDeviceToDevice, s));
    GC_CUDA(cudaMemcpyAsync(first.p, o->t_first.p, cur * 8ull, cudaMemcpyDeviceToDevice, s));
    GC_CUDA(cudaMemcpyAsync(rep.p, o->t_rep.p, cur * 8ull, cudaMemcpyDeviceToDevice, s));
    GC_CUDA(cudaMemcpyAsync(count.p, o->t_count.p, cur * 8ull, cudaMemcpyDeviceToDevice, s));
    GC_CUDA(cudaMemcpyAsync(lam.p, o->t_lam.p, cur * 8ull, cudaMemcpyDeviceToDevice, s));
    GC_CUDA(cudaMemcpyAsync(region.p, o->t_region.p, cur * 4ull, cudaMemcpyDeviceToDevice, s));
  }
  fill_i32(head.as<int>(), -1, nnb, s);
  fill_u64(f8.as<unsigned long long>(), gc::kF8Empty, nf8, s);
  fill_u64(f8n.as<unsigned long long>(), 0ULL, nf8, s);
  o->launches += 3;
  if (o->f8cap) {
    const unsigned blocks = std::min<unsigned>((o->f8cap + 255) / 256, 4096);
    f8_rehash_kernel<<<blocks, 256, 0, s>>>(o->t_f8.as<unsigned long long>(), o->t_f8n.as<unsigned long long>(),
                                              o->f8cap, f8.as<unsigned long long>(),
                                              f8n.as<unsigned long long>(), nf8 - 1, o->err());
    ++o->launches;
  }
  for (Buf* b : {&o->t_cfg, &o->t_F, &o->t_q, &o->t_t, &o->t_first, &o->t_rep, &o->t_count, &o->t_next,
                 &o->t_lam, &o->t_region, &o->t_newlist, &o->t_head, &o->t_f8, &o->t_f8n})
    b->release(s);
  o->t_cfg = cfg; o->t_F = F; o->t_q = q; o->t_t = t; o->t_first = first; o->t_rep = rep; o->t_count = count;
  o->t_next = next; o->t_lam = lam; o->t_region = region; o->t_newlist = newlist; o->t_head = head;
  o->t_f8 = f8; o->t_f8n = f8n;
  o->cap = ncap; o->nb = nnb; o->f8cap = nf8;
  if (cur) {
    const unsigned blocks = std::min<unsigned>((cur + 255) / 256, 4096);
    gc::relink_kernel<<<blocks, 256, 0, s>>>(o->view(), cur);
    ++o->launches;
  }
  GC_CUDA(cudaGetLastError());
  return GC_OK;
}

// The copy table's bucket widths for a d-dimensional lattice of V sites: F
// buckets of wF (far above the spread of F among one copy's starts) and
// fingerprint buckets of wT; the identity radius delta; F_norm = F / (d V).
void set_table_widths(gc::TableView& T, int d, int V, double delta) {
  T.wF = 1e-9 * std::max(1.0, (double)d * V * 1e-3);
  T.wT = 1e-5;
  T.inv_wF = 1.0 / T.wF;
  T.inv_wT = 1.0 / T.wT;
  T.tolF = T.wF;
  T.delta2 = delta * delta;
  T.f8_links = (double)d * V;
}

// Deduplication of one batch: find or insert each start's copy, then count
// the starts per copy (and the paper-style F set), then give every copy the
// batch created the configuration and F of its lowest start.
int launch_dedup(gc_orbit o, const gc::DedupArgs& da, cudaStream_t s) {
  const long long b = da.n;
  const int blocks = (int)std::max<long long>(1, std::min<long long>((b + 7) / 8, (long long)sm_count() * 8));
  gc::dedup_kernel<<<blocks, 256, 0, s>>>(da);
  gc::CountArgs ca{};
  ca.tab = da.tab;
  ca.n = da.n;
  ca.start0 = da.start0;
  ca.status = da.status;
  ca.F = da.F;
  ca.copy_of = da.copy_of;
  const int cblocks = (int)std::max<long long>(1, std::min<long long>((b + 255) / 256, (long long)sm_count() * 8));
  gc::count_kernel<<<cblocks, 256, 0, s>>>(ca);
  o->launches += 2;
  if (!da.tab.f8_only) {
    gc::fixup_kernel<<<sm_count() * 4, 256, 0, s>>>(da.tab, da.V, da.start0, da.F, da.config);
    ++o->launches;
  }
  GC_CUDA(cudaGetLastError());
  return GC_OK;
}

using FpKernel = void (*)(const gc::FpArgs);
FpKernel fp_test_for(int d) {
  switch (d) {
    case 1: return gc::fp_test_kernel<1>;
    case 2: return gc::fp_test_kernel<2>;
    case 3: return gc::fp_test_kernel<3>;
    default: return gc::fp_test_kernel<4>;
  }
}
FpKernel fp_screen_for(int d) {
  switch (d) {
    case 1: return gc::fp_screen_kernel<1>;
    case 2: return gc::fp_screen_kernel<2>;
    case 3: return gc::fp_screen_kernel<3>;
    default: return gc::fp_screen_kernel<4>;
  }
}

int team_size(const gc::Geom& G) {
  int maxc = 0;
  for (int c = 0; c < G.ncolor; ++c) maxc = std::max(maxc, G.color_off[c + 1] - G.color_off[c]);
  return (int)std::min<unsigned>(32u, next_pow2((unsigned)std::max(1, maxc)));
}

// A kernel's dynamic shared-memory limit only ever rises (per device and
// kernel, under a lock): threads launching one kernel for different lattice
// sizes at the same time (serving) never lower it under each other's launch.
std::mutex g_smem_mu;
std::map<std::pair<int, const void*>, size_t> g_smem_set;

template <class K>
int raise_smem_limit(K kernel, size_t smem) {
  if (smem <= 48 * 1024) return GC_OK;
  int dev = 0;
  GC_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_smem_mu);
  size_t& cur = g_smem_set[{dev, reinterpret_cast<const void*>(kernel)}];
  if (smem > cur) {
    GC_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    cur = smem;
  }
  return GC_OK;
}

template <class K>
int launch_grid(K kernel, int threads, size_t smem, long long work_items_per_block, long long items,
                int* grid) {
  if (int rc = raise_smem_limit(kernel, smem)) return rc;
  int per_sm = 0;
  GC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem));
  if (per_sm < 1) return fail(GC_EINVAL, "kernel does not fit an SM (%zu bytes shared memory)", smem);
  long long want = (items + work_items_per_block - 1) / work_items_per_block;
  *grid = (int)std::max<long long>(1, std::min<long long>((long long)per_sm * sm_count(), want));
  return GC_OK;
}

// Pick warps per CTA so the shared-memory footprint fits; returns 0 if even one warp does not.
template <class F>
int fit_warps(int max_warps, F bytes_for) {
  const size_t lim = max_smem_optin();
  for (int w = max_warps; w >= 1; --w)
    if (bytes_for(w) <= lim) return w;
  return 0;
}

// A non-blocking stream per device for an orbit's own set-up copies, and a
// read-back on a given stream.  The API never copies on the legacy default
// stream: a copy there waits for every blocking stream's work, so reading one
// orbit's results would wait for another batch still running.
constexpr int kMaxDevicesForCopies = 64;
std::mutex g_copy_mu;
cudaStream_t g_copy_stream[kMaxDevicesForCopies] = {};

cudaStream_t copy_stream() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevicesForCopies) return nullptr;
  std::lock_guard<std::mutex> lk(g_copy_mu);
  if (!g_copy_stream[dev] && cudaStreamCreateWithFlags(&g_copy_stream[dev], cudaStreamNonBlocking) != cudaSuccess)
    g_copy_stream[dev] = nullptr;
  return g_copy_stream[dev];
}

// the stream of gc_fetch_copies_async's device-to-host copies (per device)
cudaStream_t g_d2h_stream[kMaxDevicesForCopies] = {};

cudaStream_t d2h_stream() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevicesForCopies) return nullptr;
  std::lock_guard<std::mutex> lk(g_copy_mu);
  if (!g_d2h_stream[dev] && cudaStreamCreateWithFlags(&g_d2h_stream[dev], cudaStreamNonBlocking) != cudaSuccess)
    g_d2h_stream[dev] = nullptr;
  return g_d2h_stream[dev];
}

// The fetch's angle table on this device ([t_j | cos t_j | sin t_j] for
// j = -kAngleSteps/2 ... kAngleSteps/2, t_j the double nearest
// 2 pi j / kAngleSteps), filled once per device from an extended-precision
// host computation; nullptr if it cannot be set up.
double* g_angle_table[kMaxDevicesForCopies] = {};

const double* angle_table() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevicesForCopies) return nullptr;
  std::lock_guard<std::mutex> lk(g_copy_mu);
  if (g_angle_table[dev]) return g_angle_table[dev];
  static double host[3 * gc::kAngleTable];
  const long double two_pi = 2.0L * acosl(-1.0L);
  for (int j = 0; j < gc::kAngleTable; ++j) {
    const double t = (double)((long double)(j - gc::kAngleSteps / 2) * two_pi / gc::kAngleSteps);
    host[j] = t;
    host[gc::kAngleTable + j] = (double)cosl((long double)t);
    host[2 * gc::kAngleTable + j] = (double)sinl((long double)t);
  }
  void* p = nullptr;
  if (cudaMalloc(&p, sizeof host) != cudaSuccess) { cudaGetLastError(); return nullptr; }
  cudaStream_t c = nullptr;
  if (cudaStreamCreateWithFlags(&c, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMemcpyAsync(p, host, sizeof host, cudaMemcpyHostToDevice, c) != cudaSuccess ||
      cudaStreamSynchronize(c) != cudaSuccess) {
    if (c) cudaStreamDestroy(c);
    cudaFree(p);
    cudaGetLastError();
    return nullptr;
  }
  cudaStreamDestroy(c);
  g_angle_table[dev] = static_cast<double*>(p);
  return g_angle_table[dev];
}

// waits for the orbit's pending asynchronous fetch (its staging buffer is
// then free, and the host arrays hold the copies)
cudaError_t finish_fetch(gc_orbit_s* o);

cudaError_t read_back(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e;
}

}  // namespace

extern "C" {

int gc_set_allocator(gc_alloc_fn alloc, gc_free_fn free_fn, void* ctx) {
  if ((alloc == nullptr) != (free_fn == nullptr))
    return fail(GC_EINVAL, "gc_set_allocator: give both hooks or neither");
  g_alloc = alloc;
  g_free = free_fn;
  g_actx = ctx;
  return GC_OK;
}

int gc_options_default(gc_options* opt) {
  if (!opt) return fail(GC_EINVAL, "gc_options_default: opt is NULL");
  std::memset(opt, 0, sizeof *opt);
  opt->precision = GC_FP64;
  opt->check_every = 1;
  opt->max_sweeps = 100000;
  opt->eps32 = 1e-10;
  opt->dedup_delta = 1e-6;
  opt->fp_tau = 1e-9;
  opt->fp_mode = GC_FP_AUTO;
  opt->lanczos_k = 300;
  opt->seed = 1;
  opt->keep_per_start = 0;
  opt->newton_inner = 320;
  opt->newton_max = 6;
  opt->batch_starts = 0;
  opt->stream = nullptr;
  opt->relax_variant = GC_RELAX_AUTO;
  opt->async = 0;
  opt->use_graph = 0;
  opt->autotune = 0;
  opt->dedup_mode = GC_DEDUP_CONFIG;
  return GC_OK;
}

const char* gc_last_error(void) { return g_err.c_str(); }
const char* gc_version(void) { return "gribov-b300 0.1 (sm_103a)"; }

int gc_create_orbit(int dim, int L, const double* link_angles, uint64_t orbit_id, size_t max_copies,
                    gc_orbit* out) {
  if (!out) return fail(GC_EINVAL, "gc_create_orbit: out is NULL");
  *out = nullptr;
  if (dim < 1 || dim > gc::kMaxDim) return fail(GC_EINVAL, "dimension %d not in 1..4", dim);
  if (L < 2) return fail(GC_EINVAL, "L = %d < 2", L);
  if (!link_angles) return fail(GC_EINVAL, "link_angles is NULL");
  double Vd = std::pow((double)L, dim);
  if (Vd > gc::kMaxSlabSites)
    return fail(GC_EINVAL, "lattice of %.0f sites exceeds %d", Vd, gc::kMaxSlabSites);
  const int V = (int)Vd;
  // The shared-memory kernels keep links, tables and one FP64 lattice per
  // start in shared memory; beyond that (or beyond their 16-bit tables) the
  // sweeps stream the lattice in hyperplanes from global memory (even L).
  const size_t need = gc::Smem(V, dim, 16, (size_t)V * 16, 1).total;
  bool slab = false;
  if (V > gc::kMaxSites || need > max_smem_optin()) {
    const int P = V / L;
    if (dim < 2 || L % 2 != 0 || gc::slab_smem_bytes(P, 16) > max_smem_optin())
      return fail(GC_EINVAL, "lattice %d^%d fits neither shared memory (%zu bytes needed, limit %zu) nor "
                  "the hyperplane path (even L, d >= 2, three FP64 hyperplanes of %d sites)",
                  L, dim, need, max_smem_optin(), P);
    slab = true;
  }
  for (int i = 0; i < V * dim; ++i)
    if (!std::isfinite(link_angles[i])) return fail(GC_EINVAL, "link angle %d is not finite", i);

  gc_orbit o = new (std::nothrow) gc_orbit_s;
  if (!o) return fail(GC_ENOMEM, "host allocation failed");
  o->d = dim; o->L = L; o->V = V; o->orbit_id = orbit_id;
  o->slab = slab;
  o->ncolor = (L % 2 == 0) ? 2 : 3;
  gc::Geom& G = o->geom;
  G.d = dim; G.L = L; G.V = V; G.ncolor = o->ncolor;
  int cnt[3] = {0, 0, 0};
  for (int x = 0; x < V; ++x) cnt[gc::site_color(x, dim, L)]++;
  G.color_off[0] = 0;
  for (int c = 0; c < 3; ++c) G.color_off[c + 1] = G.color_off[c] + (c < o->ncolor ? cnt[c] : 0);
  {
    // site V-1 is the last site of its colour in colour-major order
    const int cl = gc::site_color(V - 1, dim, L);
    G.pos_last = G.color_off[cl + 1] - 1;
  }
  o->team = team_size(G);

  std::vector<double2> u64((size_t)V * dim);
  std::vector<float2> u32((size_t)V * dim);
  for (size_t i = 0; i < u64.size(); ++i) {
    u64[i] = make_double2(std::cos(link_angles[i]), std::sin(link_angles[i]));
    u32[i] = make_float2((float)u64[i].x, (float)u64[i].y);
  }
  cudaStream_t s = copy_stream();
  o->last_stream = s;
  int rc = GC_OK;
  if (!o->links64.ensure(u64.size() * sizeof(double2), s) || !o->links32.ensure(u32.size() * sizeof(float2), s) ||
      !o->t_counters.ensure(64, s) || !o->stats.ensure(kNumStats * 8, s) || !o->work.ensure(64, s) ||
      !o->t_lock.ensure((size_t)(o->nl = 1u << 16) * 4, s)) {
    rc = fail(GC_ENOMEM, "cannot admit orbit buffers");
  }
  if (rc == GC_OK) {
    cudaError_t e = cudaMemcpyAsync(o->links64.p, u64.data(), u64.size() * sizeof(double2), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(o->links32.p, u32.data(), u32.size() * sizeof(float2), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(o->t_counters.p, 0, 64, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(o->stats.p, 0, kNumStats * 8, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(o->t_lock.p, 0, (size_t)o->nl * 4, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // the host vectors go out of scope
    if (e != cudaSuccess) rc = fail(GC_ECUDA, "orbit upload: %s", cudaGetErrorString(e));
  }
  if (rc == GC_OK) {
    // large lattices start with a pool of about 256 MiB of copies
    const unsigned long long first =
        max_copies ? max_copies
                   : (slab ? std::max<unsigned long long>(64, std::min<unsigned long long>(4096, (1ull << 28) / ((unsigned long long)V * 16)))
                           : 4096);
    rc = table_reserve(o, first, 0, s);
  }
  if (rc == GC_OK) {
    for (auto& e : o->ev)
      if (cudaEventCreate(&e) != cudaSuccess) { rc = fail(GC_ECUDA, "cudaEventCreate failed"); break; }
  }
  // the set-up (uploads, fills of the copy pool) is complete before any
  // other stream can use the orbit
  if (rc == GC_OK && cudaStreamSynchronize(s) != cudaSuccess)
    rc = fail(GC_ECUDA, "orbit set-up: %s", cudaGetErrorString(cudaGetLastError()));
  if (rc != GC_OK) {
    gc_destroy_orbit(o);
    return rc;
  }
  *out = o;
  return GC_OK;
}

int gc_destroy_orbit(gc_orbit o) {
  if (!o) return fail(GC_EINVAL, "gc_destroy_orbit: NULL orbit");
  cudaStreamSynchronize(o->last_stream);
  finish_fetch(o);
  for (auto& e : o->fetch_ev)
    if (e) cudaEventDestroy(e);
  cudaStream_t s = nullptr;
  for (Buf* b : {&o->links64, &o->links32, &o->t_cfg, &o->t_F, &o->t_q, &o->t_t, &o->t_first, &o->t_rep, &o->t_count,
                 &o->t_next, &o->t_lam, &o->t_region, &o->t_head, &o->t_lock, &o->t_f8, &o->t_f8n, &o->t_counters,
                 &o->t_newlist, &o->s_status, &o->s_sweeps, &o->s_resid, &o->s_F, &o->s_fprint,
                 &o->s_config, &o->s_state32, &o->s_copy, &o->s_redo, &o->s_rate, &o->work, &o->stats, &o->scratch, &o->theta_tmp,
                 &o->sort_keys, &o->sort_idx, &o->sort_tmp, &o->f8_tmp})
    b->release(s);
  for (auto& e : o->ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : o->ev_pool) cudaEventDestroy(e);
  if (o->served_by) server_release_region(o);   // its results' region goes back to the server
  delete o;
  return GC_OK;
}

}  // extern "C"

namespace {

// Result-neutral launch knobs (the autotuner picks them; none changes any
// start's arithmetic): warps per CTA of the generic relaxation, of the polish
// and of the FP test, and starts per device batch.
struct Tuning {
  int r_warps = 0, p_warps = 0, f_warps = 0;
  size_t batch = 0;
  int check_every = 0;   // sweep-unroll depth (autotune mode 2 only; 0: the caller's)
};

int validate_options(const gc_options& opt, double omega, double eps) {
  if (!(omega > 0.0 && omega < 2.0)) return fail(GC_EINVAL, "omega = %g not in (0, 2)", omega);
  if (!(eps > 0.0)) return fail(GC_EINVAL, "eps = %g must be > 0", eps);
  if (opt.precision != GC_FP64 && opt.precision != GC_MIXED) return fail(GC_EINVAL, "unknown precision %d", opt.precision);
  if (opt.check_every < 1) return fail(GC_EINVAL, "check_every = %d < 1", opt.check_every);
  if (opt.max_sweeps < 1) return fail(GC_EINVAL, "max_sweeps = %d < 1", opt.max_sweeps);
  if (opt.fp_mode < GC_FP_AUTO || opt.fp_mode > GC_FP_NONE) return fail(GC_EINVAL, "unknown fp_mode %d", opt.fp_mode);
  if (opt.precision == GC_MIXED && !(opt.eps32 > 0.0)) return fail(GC_EINVAL, "eps32 = %g must be > 0", opt.eps32);
  if (!(opt.dedup_delta > 0.0 && opt.dedup_delta < 0.1)) return fail(GC_EINVAL, "dedup_delta = %g not in (0, 0.1)", opt.dedup_delta);
  if (!(opt.fp_tau >= 0.0)) return fail(GC_EINVAL, "fp_tau = %g < 0", opt.fp_tau);
  if (opt.lanczos_k < 2) return fail(GC_EINVAL, "lanczos_k = %d < 2", opt.lanczos_k);
  if (opt.newton_inner < 1 || opt.newton_max < 0) return fail(GC_EINVAL, "bad Newton polish settings");
  if (opt.dedup_mode != GC_DEDUP_CONFIG && opt.dedup_mode != GC_DEDUP_F8)
    return fail(GC_EINVAL, "unknown dedup_mode %d", opt.dedup_mode);
  return GC_OK;
}

// Add up the stage times of every batch enqueued since the last harvest
// (the orbit's work must be complete).
void harvest_timing(gc_orbit o) {
  // per batch: before relax | after relax | after the first polish launch |
  // after the redo polish launch | after dedup | after the FP test | where
  // the FP32 sweeps begin inside the relax stage (after the start draw, or on
  // lattices beyond shared memory after the FP64 head sweeps; at the stage's
  // start where the sweeps draw their own starts)
  for (size_t k = 0; k + kEvPerBatch <= o->ev_used; k += kEvPerBatch) {
    float t[5] = {0, 0, 0, 0, 0}, t_start = 0;
    for (int j = 0; j < 5; ++j) cudaEventElapsedTime(&t[j], o->ev_pool[k + j], o->ev_pool[k + j + 1]);
    cudaEventElapsedTime(&t_start, o->ev_pool[k], o->ev_pool[k + 6]);
    o->ms[0] += t[0]; o->ms[1] += t[1] + t[2]; o->ms[2] += t[3]; o->ms[3] += t[4]; o->ms[4] += t[2];
    o->ms[5] += t_start;
  }
  cudaGetLastError();
  o->ev_used = 0;
}

cudaError_t finish_fetch(gc_orbit_s* o) {
  if (!o->fetch_pending) return cudaSuccess;
  o->fetch_pending = false;
  return cudaEventSynchronize(o->fetch_ev[1]);
}

int check_errors(gc_orbit o) {
  if (!o->err_unchecked) return GC_OK;
  int flags[4] = {0, 0, 0, 0};
  GC_CUDA(read_back(flags, o->err(), 16, o->last_stream));
  o->err_unchecked = false;
  if (flags[1]) return fail(GC_ENOMEM, "copy pool overflow");
  if (flags[2]) return fail(GC_ENOMEM, "quantised-minimum set overflow");
  if (flags[0]) return fail(GC_ETIMEDOUT, "a copy-table lock wait ran out (affected starts are marked)");
  if (flags[3]) return fail(GC_ETIMEDOUT, "a bulk-copy wait of the hyperplane sweeps ran out");
  return GC_OK;
}

std::mutex g_tune_mu;
std::vector<std::pair<long long, Tuning>> g_tune_cache;   // key: tune_key

// d | L << 4 | precision << 12 | deep << 16 (deep: sweep-unroll depth tuned too)
long long tune_key(int d, int L, int precision, bool deep) {
  return (long long)d | ((long long)L << 4) | ((long long)precision << 12) | ((long long)deep << 16);
}

int autotune_shape(gc_orbit like, const gc_options& base, double omega, double eps, Tuning* out);
bool have_tuning(int d, int L, int precision, bool deep = false);
bool deep_tuning(const gc_options& opt);

Tuning cached_tuning(int d, int L, int precision, bool deep = false) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (auto& kv : g_tune_cache)
    if (kv.first == tune_key(d, L, precision, deep)) return kv.second;
  return Tuning{};
}

// Thread-block clusters of `csize` CTAs (`threads` threads, `smem` bytes of
// dynamic shared memory) that fit on the GPU at once, 0 when none does;
// queried once per kernel and shape, so that a launch inside a stream capture
// makes no query
template <class K>
int cluster_count(K kernel, int threads, size_t smem, int csize, int* out) {
  static std::mutex mu;
  static std::map<std::tuple<const void*, int, size_t, int, int>, int> cache;
  int dev = 0;
  GC_CUDA(cudaGetDevice(&dev));
  const auto key = std::make_tuple(reinterpret_cast<const void*>(kernel), threads, smem, csize, dev);
  {
    std::lock_guard<std::mutex> lk(mu);
    const auto it = cache.find(key);
    if (it != cache.end()) { *out = it->second; return GC_OK; }
  }
  if (int rc = raise_smem_limit(kernel, smem)) return rc;
  if (csize > 8) GC_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchConfig_t cfg{};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3(csize * 8);
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kernel, &cfg) != cudaSuccess) {
    cudaGetLastError();
    n = 0;
  }
  std::lock_guard<std::mutex> lk(mu);
  cache[key] = n;
  *out = n;
  return GC_OK;
}

// Launch `kernel` on `ncl` clusters of `csize` CTAs
template <class K, class A>
int launch_clusters(K kernel, const A& args, int threads, size_t smem, int csize, int ncl, cudaStream_t s) {
  cudaLaunchConfig_t cfg{};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = csize;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3(csize * ncl);
  GC_CUDA(cudaLaunchKernelEx(&cfg, kernel, args));
  return GC_OK;
}

// One launch of the hyperplane sweeps: one CTA per start (grid CTAs), or one
// start per cluster of kSlabCluster CTAs (as many clusters as fit at once),
// or, with `wide` (a handful of hard starts), of kSlabClusterWide CTAs where
// that non-portable size fits
constexpr int kSlabCluster = 8, kSlabClusterWide = 16;
// Mixed path on lattices beyond shared memory: the first kSlabHeadSweeps sweeps
// of every start are the plain path's FP64 sweeps (the oracle's operations),
// then FP32 continues from that state.  A random start moves far in its first
// sweeps, and there FP32 rounding can steer it into another basin: on 4D 8^4,
// 3D 16^3 and 4D 16^4 (von Mises kappa = 1) 0.8-1.6 % of starts ended in a
// different minimum than the FP64 path (F off by up to 33).  Measured
// agreement with the FP64 path: 12 head sweeps, all of 1024 starts on 4D 8^4
// and 3D 16^3 but 508 of 512 on 4D 16^4; 24 head sweeps, 512 of 512 on 4D
// 16^4 (and 48 and 96 the same), for 20 % more time in its relaxation stage.
constexpr int kSlabHeadSweeps = 24;
template <class K1, class KC>
int launch_slab(K1 k1, KC kc, const gc::SlabArgs& sa, size_t smem, int grid, bool cluster,
                cudaStream_t s, bool wide = false) {
  if (cluster) {
    for (int csize : {kSlabClusterWide, kSlabCluster}) {
      if (csize == kSlabClusterWide && !wide) continue;
      int ncl = 0;
      if (int rc = cluster_count(kc, 512, smem, csize, &ncl)) return rc;
      if (ncl > 0) return launch_clusters(kc, sa, 512, smem, csize, ncl, s);
    }
    // no cluster of this shape fits: one CTA per start
  }
  if (int rc = raise_smem_limit(k1, smem)) return rc;
  k1<<<grid, 512, smem, s>>>(sa);
  GC_CUDA(cudaGetLastError());
  return GC_OK;
}

// Everything the hyperplane path of a call allocates or queries, done before
// any of its work is enqueued, so that a batch can be captured as a graph:
// the staging of B starts, the per-start rate and redo lists, the Newton and
// first-region scratch, and the shared-memory limits and cluster counts of
// every launch shape.  Returns B, the starts per device batch.
template <int D>
int slab_prepare_d(gc_orbit o, uint64_t n_starts, const gc_options& opt, cudaStream_t s, size_t* B_out) {
  const int V = o->V, L = o->L, P = V / L;
  const bool mixed = opt.precision == GC_MIXED, cluster = opt.relax_variant != GC_RELAX_GENERIC;
  const size_t per_start = (size_t)V * 16 + (mixed ? (size_t)V * 8 : 0) + 48;
  size_t B = opt.batch_starts > 0 ? (size_t)opt.batch_starts
                                  : std::max<size_t>(2 * (size_t)sm_count(), (1ull << 30) / per_start);
  B = std::min<size_t>(B, n_starts);
  if (!o->s_status.ensure(B, s) || !o->s_sweeps.ensure(B * 4, s) || !o->s_resid.ensure(B * 8, s) ||
      !o->s_F.ensure(B * 8, s) || !o->s_fprint.ensure(B * 8, s) || !o->s_config.ensure(B * V * 16, s) ||
      !o->s_copy.ensure(B * 4, s) || (mixed && !o->s_state32.ensure(B * V * 8, s)) ||
      (mixed && !o->s_rate.ensure(B * 4, s)) || !o->s_redo.ensure(B * 8, s))
    return fail(GC_ENOMEM, "cannot admit a batch of %zu starts (%.1f MiB staging)", B, B * per_start / 1048576.0);
  int x = 0;
  const size_t sm64 = gc::slab_smem_bytes(P, 16), sm32 = gc::slab_smem_bytes(P, 8);
  if (int rc = raise_smem_limit(gc::relax_slab_kernel<double2, D, false>, sm64)) return rc;
  if (cluster) {
    if (int rc = cluster_count(gc::relax_slab_kernel<double2, D, true>, 512, sm64, kSlabCluster, &x)) return rc;
    if (mixed)
      if (int rc = cluster_count(gc::relax_slab_kernel<double2, D, true>, 512, sm64, kSlabClusterWide, &x)) return rc;
  }
  size_t scratch = 0;
  if (mixed) {
    if (int rc = raise_smem_limit(gc::relax_slab_kernel<float2, D, false>, sm32)) return rc;
    if (cluster) {
      if (int rc = cluster_count(gc::relax_slab_kernel<float2, D, true>, 512, sm32, kSlabCluster, &x)) return rc;
      for (int C : {kSlabClusterWide, kSlabCluster}) {
        const size_t smd = gc::dsmem_smem_bytes(D, L, P, C);
        if (L < 2 * C || smd > max_smem_optin()) continue;
        if (int rc = cluster_count(gc::relax_dsmem_kernel<D>, 256, smd, C, &x)) return rc;
      }
    }
    const int Ps = (P + 3) / 4 * 4;
    const size_t smn = gc::slab_newton_smem_bytes(Ps);
    if (int rc = raise_smem_limit(gc::slab_newton_kernel<D, false>, smn)) return rc;
    int ncl = 0;
    if (cluster)
      if (int rc = cluster_count(gc::slab_newton_kernel<D, true>, 1024, smn, kSlabCluster, &ncl)) return rc;
    const int slots = std::max((int)std::min<size_t>(B, 4 * (size_t)sm_count()), ncl);
    scratch = std::max(scratch, (size_t)slots * gc::slab_newton_scratch_floats(D, V, L, Ps) * 4);
  }
  if (opt.fp_mode != GC_FP_NONE) {
    const int kmax = std::min(std::max(opt.lanczos_k, 8 * L), V - 1);
    const size_t smf32 = gc::slab_fp_smem_bytes(kmax, 4), smf64 = gc::slab_fp_smem_bytes(kmax, 8);
    if (int rc = raise_smem_limit(gc::slab_fp_lanczos_kernel<float, D, false>, smf32)) return rc;
    if (int rc = raise_smem_limit(gc::slab_fp_lanczos_kernel<double, D, false>, smf64)) return rc;
    if (cluster)
      for (int C : {kSlabClusterWide, kSlabCluster})
        if (int rc = cluster_count(gc::slab_fp_lanczos_kernel<double, D, true>, 1024, smf64, C, &x)) return rc;
    scratch = std::max(scratch, (size_t)sm_count() * gc::slab_fp_scratch_bytes<double>(D, V));
  }
  if (scratch && !o->scratch.ensure(scratch, s))
    return fail(GC_ENOMEM, "cannot admit the large-lattice scratch (%.1f MiB)", scratch / 1048576.0);
  *B_out = B;
  return GC_OK;
}

int slab_prepare(gc_orbit o, uint64_t n_starts, const gc_options& opt, cudaStream_t s, size_t* B_out) {
  switch (o->d) {
    case 2: return slab_prepare_d<2>(o, n_starts, opt, s, B_out);
    case 3: return slab_prepare_d<3>(o, n_starts, opt, s, B_out);
    default: return slab_prepare_d<4>(o, n_starts, opt, s, B_out);
  }
}

// The path for lattices beyond shared memory (o->slab): sweeps that stream the
// lattice in hyperplanes from global memory (FP64 for the plain path; for the
// mixed path FP32 sweeps, then the inexact Newton polish, FP64 sweeps for the
// starts it leaves), the functional and canonical copy from the FP64 state,
// dedup as everywhere, and the first-region test by Lanczos with vectors in
// global memory.  The same batch structure and events as enumerate_impl.
int enumerate_slab(gc_orbit o, uint64_t n_starts, double omega, double eps, const gc_options& opt,
                   cudaStream_t s, bool async, bool timing, int check_every, int max_sweeps) {
  const int V = o->V, d = o->d, L = o->L, P = V / L;
  const bool mixed = opt.precision == GC_MIXED;
  size_t B = 0;
  if (int rc = slab_prepare(o, n_starts, opt, s, &B)) return rc;
  unsigned long long* wctr = o->work.as<unsigned long long>();
  unsigned long long* stats = o->stats.as<unsigned long long>();
  if (!o->err_unchecked) GC_CUDA(cudaMemsetAsync(o->err(), 0, 16, s));
  o->err_unchecked = true;
  o->last_stream = s;
  const size_t sm64 = gc::slab_smem_bytes(P, 16), sm32 = gc::slab_smem_bytes(P, 8);

  for (uint64_t done = 0; done < n_starts;) {
    const long long b = (long long)std::min<uint64_t>(B, n_starts - done);
    if (o->enqueued + (unsigned long long)b > o->cap) {
      if (async) return fail(GC_ESTATE, "asynchronous enumeration needs the copy pool reserved up front");
      unsigned cur = 0;
      GC_CUDA(cudaMemcpyAsync(&cur, o->n_entries(), 4, cudaMemcpyDeviceToHost, s));
      GC_CUDA(cudaStreamSynchronize(s));
      if ((unsigned long long)cur + b > o->cap)
        if (int rc = table_reserve(o, (unsigned long long)cur + b, cur, s)) return rc;
    }
    cudaEvent_t* ev = nullptr;
    if (timing) {
      while (o->ev_pool.size() < o->ev_used + kEvPerBatch) {
        cudaEvent_t e;
        GC_CUDA(cudaEventCreate(&e));
        o->ev_pool.push_back(e);
      }
      ev = o->ev_pool.data() + o->ev_used;
      o->ev_used += kEvPerBatch;
    }
    GC_CUDA(cudaMemsetAsync(wctr, 0, 32, s));
    GC_CUDA(cudaMemsetAsync(o->n_new(), 0, 4, s));

    gc::SlabArgs sa{};
    sa.d = d; sa.L = L; sa.V = V; sa.P = P;
    sa.n = b;
    sa.seed = opt.seed; sa.orbit_id = o->orbit_id; sa.start0 = o->next_start;
    sa.omega = omega; sa.om1 = 1.0 - omega; sa.eps = eps;
    sa.omega32 = (float)omega; sa.om1_32 = (float)(1.0 - omega); sa.eps32 = (float)opt.eps32;
    sa.check_every = check_every; sa.max_sweeps = max_sweeps;
    sa.status = o->s_status.as<int8_t>();
    sa.sweeps = o->s_sweeps.as<int32_t>();
    sa.resid = o->s_resid.as<double>();
    sa.stats = stats;
    sa.err = o->err();
    sa.work_ctr = wctr;
    const int grid = (int)std::max<long long>(1, std::min<long long>(b, 2LL * sm_count()));
    // one start per cluster of kSlabCluster CTAs (default), or one CTA per
    // start (GC_RELAX_GENERIC)
    auto launch = [&](bool fp64, bool cluster, bool wide = false) -> int {
      int rc = GC_OK;
      if (fp64) {
        switch (d) {
          case 2: rc = launch_slab(gc::relax_slab_kernel<double2, 2, false>, gc::relax_slab_kernel<double2, 2, true>, sa, sm64, grid, cluster, s, wide); break;
          case 3: rc = launch_slab(gc::relax_slab_kernel<double2, 3, false>, gc::relax_slab_kernel<double2, 3, true>, sa, sm64, grid, cluster, s, wide); break;
          default: rc = launch_slab(gc::relax_slab_kernel<double2, 4, false>, gc::relax_slab_kernel<double2, 4, true>, sa, sm64, grid, cluster, s, wide); break;
        }
      } else {
        switch (d) {
          case 2: rc = launch_slab(gc::relax_slab_kernel<float2, 2, false>, gc::relax_slab_kernel<float2, 2, true>, sa, sm32, grid, cluster, s); break;
          case 3: rc = launch_slab(gc::relax_slab_kernel<float2, 3, false>, gc::relax_slab_kernel<float2, 3, true>, sa, sm32, grid, cluster, s); break;
          default: rc = launch_slab(gc::relax_slab_kernel<float2, 4, false>, gc::relax_slab_kernel<float2, 4, true>, sa, sm32, grid, cluster, s); break;
        }
      }
      ++o->launches;
      return rc;
    };
    // clusters unless GC_RELAX_GENERIC: a start's sweep count is not known in
    // advance, and a long start on one CTA sets the batch's end
    const bool cluster = opt.relax_variant != GC_RELAX_GENERIC;
    if (ev) {
      GC_CUDA(cudaEventRecord(ev[0], s));
      if (!mixed) GC_CUDA(cudaEventRecord(ev[6], s));   // the sweeps draw their own starts
    }
    double2* st64 = o->s_config.as<double2>();
    if (mixed) {
      // FP64 head: the plain path's first sweeps from the random starts (no
      // converged/not-converged counts: the FP32 phase decides every start)
      {
        gc::SlabArgs ha = sa;
        ha.links = o->links64.p;
        ha.state = st64;
        ha.init = 1;
        ha.check_every = kSlabHeadSweeps;
        ha.max_sweeps = kSlabHeadSweeps;
        ha.s_sweeps = kSweeps; ha.s_updates = kUpdates; ha.s_conv = -1; ha.s_nconv = -1;
        const size_t nv = (size_t)b * V;
        gc::SlabArgs keep = sa;
        sa = ha;
        if (int rc = launch(true, cluster)) return rc;
        sa = keep;
        gc::slab_demote_kernel<<<(int)std::min<size_t>((nv + 255) / 256, 4096), 256, 0, s>>>(
            st64, o->s_state32.as<float2>(), nv);
        ++o->launches;
        GC_CUDA(cudaMemsetAsync(wctr, 0, 8, s));
      }
      if (ev) GC_CUDA(cudaEventRecord(ev[6], s));   // the FP32 sweeps start here
      // FP32 sweeps from there
      if (!o->s_rate.ensure((size_t)B * 4, s)) return fail(GC_ENOMEM, "cannot admit a batch of %zu starts", B);
      sa.links = o->links32.p;
      sa.state = o->s_state32.as<float2>();
      sa.rate = o->s_rate.as<float>();
      sa.init = 0;
      sa.s_sweeps = kSweeps32; sa.s_updates = kUpdates32; sa.s_conv = kConv32; sa.s_nconv = kNConv32;
      // the lattice in a cluster's distributed shared memory: one start per
      // cluster of 16 (else 8) CTAs of 256 threads, each holding at least two
      // planes (else the hyperplane streaming).  Measured on the FP32 stage:
      // 4D 16^4 (8 CTAs, 2 planes each) 478 ms against 490 streamed, 3D 40^3
      // 358 against 473, 2D 256^2 586 against 3180
      bool dsm = false;
      if (cluster) {
        auto kd = d == 2 ? gc::relax_dsmem_kernel<2> : (d == 3 ? gc::relax_dsmem_kernel<3> : gc::relax_dsmem_kernel<4>);
        for (int C : {kSlabClusterWide, kSlabCluster}) {
          const size_t smd = gc::dsmem_smem_bytes(d, L, P, C);
          if (L < 2 * C || smd > max_smem_optin()) continue;
          const int thr = 256;
          int ncl = 0;
          if (int rc = cluster_count(kd, thr, smd, C, &ncl)) return rc;
          if (ncl <= 0) continue;
          if (int rc = launch_clusters(kd, sa, thr, smd, C, ncl, s)) return rc;
          ++o->launches;
          dsm = true;
          break;
        }
      }
      if (!dsm)
        if (int rc = launch(false, cluster)) return rc;
      if (ev) GC_CUDA(cudaEventRecord(ev[1], s));
      const size_t nv = (size_t)b * V;
      gc::slab_promote_kernel<<<(int)std::min<size_t>((nv + 255) / 256, 4096), 256, 0, s>>>(
          o->s_state32.as<float2>(), st64, nv);
      ++o->launches;
      // Newton polish.  One start per 256-thread CTA (four per SM) with an
      // inner budget of newton_inner, then the starts that exceed it once more
      // on clusters of kSlabCluster 1024-thread CTAs with 6x (a hard start runs
      // 8 SMs wide instead of holding one small CTA for the whole launch).
      // When every start gets a cluster at once, one cluster launch with 4x;
      // GC_RELAX_GENERIC: one CTA per start with 4x.
      GC_CUDA(cudaMemsetAsync(wctr, 0, 8, s));
      GC_CUDA(cudaMemsetAsync(o->n_redo(), 0, 16, s));   // n_redo, n_redo2
      const int Ps = (P + 3) / 4 * 4;
      const size_t smn = gc::slab_newton_smem_bytes(Ps);
      gc::SlabNewtonArgs na{};
      na.d = d; na.L = L; na.V = V; na.P = P; na.Ps = Ps;
      na.links = o->links64.as<double2>();
      na.state = st64;
      na.n = b;
      na.work_ctr = wctr;
      na.eps = eps;
      na.omega_sweeps = (float)omega;
      na.rate = o->s_rate.as<float>();
      na.lin_tol = 4e-4f;
      na.inner_max = opt.newton_inner;
      na.newton_max = opt.newton_max;
      na.scratch_floats = gc::slab_newton_scratch_floats(d, V, L, Ps);
      na.status = sa.status;
      na.resid = sa.resid;
      na.stats = stats;
      na.s_steps = kNewton; na.s_inner = kInner; na.s_pass = kPass; na.s_conv = kPConv; na.s_redo = kFallback;
      na.err = o->err();
      if (!o->s_redo.ensure((size_t)B * 8, s)) return fail(GC_ENOMEM, "cannot admit a batch of %zu starts", B);
      unsigned* redo1 = o->s_redo.as<unsigned>();
      unsigned* redo2 = redo1 + B;
      const unsigned* final_list = redo1;
      const unsigned* final_n = o->n_redo();
      {
        int ncl = 0;
        auto kc = d == 2 ? gc::slab_newton_kernel<2, true> : (d == 3 ? gc::slab_newton_kernel<3, true> : gc::slab_newton_kernel<4, true>);
        auto k1 = d == 2 ? gc::slab_newton_kernel<2, false> : (d == 3 ? gc::slab_newton_kernel<3, false> : gc::slab_newton_kernel<4, false>);
        if (cluster)
          if (int rc = cluster_count(kc, 1024, smn, kSlabCluster, &ncl)) return rc;
        const int grid1 = (int)std::max<long long>(1, std::min<long long>(b, 4LL * sm_count()));
        const int slots = std::max(grid1, ncl);
        if (!o->scratch.ensure((size_t)slots * na.scratch_floats * 4, s))
          return fail(GC_ENOMEM, "cannot admit the Newton scratch of %d starts (%.1f MiB)", slots,
                      slots * na.scratch_floats * 4 / 1048576.0);
        na.scratch = o->scratch.as<float>();
        auto run_cluster = [&]() -> int {
          if (int rc = launch_clusters(kc, na, 1024, smn, kSlabCluster, ncl, s)) return rc;
          ++o->launches;
          return GC_OK;
        };
        if (ncl > 0 && (long long)ncl >= b) {            // every start on its own cluster
          na.budget = 4 * opt.newton_inner;
          na.redo = redo1; na.n_redo = o->n_redo();
          if (int rc = run_cluster()) return rc;
        } else {
          if (int rc = raise_smem_limit(k1, smn)) return rc;
          const bool staged = ncl > 0;
          na.budget = (staged ? 1 : 4) * opt.newton_inner;
          na.redo = redo1; na.n_redo = o->n_redo();
          na.s_redo = staged ? -1 : kFallback;
          k1<<<grid1, 256, smn, s>>>(na);
          ++o->launches;
          GC_CUDA(cudaGetLastError());
          if (staged) {
            na.list = redo1; na.n_list = o->n_redo();
            na.budget = 6 * opt.newton_inner;
            na.redo = redo2; na.n_redo = o->n_redo2();
            na.s_redo = kFallback;
            if (int rc = run_cluster()) return rc;
            final_list = redo2;
            final_n = o->n_redo2();
          }
        }
      }
      if (ev) GC_CUDA(cudaEventRecord(ev[2], s));
      // FP64 sweeps for the starts the polish left; final outcomes
      GC_CUDA(cudaMemsetAsync(wctr, 0, 8, s));
      sa.links = o->links64.p;
      sa.state = st64;
      sa.init = 0;
      sa.list = final_list;
      sa.n_list = final_n;
      sa.rate = nullptr;
      sa.omega_rate = o->s_rate.as<float>();   // the polish's sweeps at each start's Young parameter
      sa.s_sweeps = -1; sa.s_updates = kUpd64; sa.s_conv = kPConv; sa.s_nconv = kPNConv;
    } else {
      sa.links = o->links64.p;
      sa.state = st64;
      sa.init = 1;
      sa.s_sweeps = kSweeps; sa.s_updates = kUpdates; sa.s_conv = kConv; sa.s_nconv = kNConv;
    }
    if (int rc = launch(true, cluster, mixed)) return rc;   // mixed: the few starts Newton left
    if (ev && !mixed) GC_CUDA(cudaEventRecord(ev[1], s));
    // functional, fingerprint and canonical copy (in place)
    gc::slab_final_kernel<<<grid, 256, 0, s>>>(st64, o->links64.as<double2>(), d, V, L, b,
                                               o->s_F.as<double>(), o->s_fprint.as<double>());
    ++o->launches;
    GC_CUDA(cudaGetLastError());
    if (ev) {
      if (!mixed) GC_CUDA(cudaEventRecord(ev[2], s));   // mixed: after the Newton polish
      GC_CUDA(cudaEventRecord(ev[3], s));
    }
    gc::DedupArgs da{};
    da.tab = o->view();
    set_table_widths(da.tab, d, V, opt.dedup_delta);
    da.tab.f8_only = opt.dedup_mode == GC_DEDUP_F8;
    da.V = V;
    da.n = b;
    da.start0 = o->next_start;
    da.status = sa.status;
    da.F = o->s_F.as<double>();
    da.fprint = o->s_fprint.as<double>();
    da.config = st64;
    da.copy_of = o->s_copy.as<int>();
    da.stats = stats;
    if (int rc = launch_dedup(o, da, s)) return rc;
    if (ev) GC_CUDA(cudaEventRecord(ev[4], s));
    if (opt.fp_mode != GC_FP_NONE) {
      // first-region test of the batch's new copies: Lanczos with vectors in
      // global memory, one copy per 1024-thread CTA.  Auto: an FP32 screen,
      // then FP64 for the copies it leaves; otherwise FP64 for every copy (the
      // dense mode's full-dimension run has no large-lattice form: Lanczos to
      // lanczos_k steps)
      // the low end of a large lattice's spectrum needs about 8L steps
      const int kmax = std::min(std::max(opt.lanczos_k, 8 * L), V - 1);
      const int grid_f = sm_count();
      const size_t sb32 = gc::slab_fp_scratch_bytes<float>(d, V), sb64 = gc::slab_fp_scratch_bytes<double>(d, V);
      if (!o->scratch.ensure((size_t)grid_f * sb64, s) || !o->s_redo.ensure((size_t)B * 4, s))
        return fail(GC_ENOMEM, "cannot admit the first-region test scratch (%.1f MiB)", grid_f * sb64 / 1048576.0);
      gc::SlabFpArgs fa{};
      fa.cfg = o->t_cfg.as<double2>();
      fa.first_start = o->t_first.as<unsigned long long>();
      fa.links = o->links64.as<double2>();
      fa.d = d; fa.L = L; fa.V = V;
      fa.lambda2 = o->t_lam.as<double>();
      fa.region = o->t_region.as<int>();
      fa.tau = opt.fp_tau;
      // FP32 Lanczos resolves the bottom of the spectrum to about eps32 |M|
      // (~1e-6 here); large lattices have lambda_2 of 1e-4 .. 1e-2, so the
      // screen decides above 1e-4 and FP64 takes the copies near zero
      fa.margin = 1e-4;
      fa.kmax = kmax;
      fa.seed = opt.seed;
      fa.scratch = o->scratch.as<unsigned char>();
      fa.stats = stats;
      fa.s_tests = kTests; fa.s_tests64 = kTests64; fa.s_steps = kLanczos; fa.s_steps64 = kLanczos64;
      // fp32: the screen, one copy per CTA.  FP64: one copy per cluster of 16
      // (else 8) CTAs: in auto mode it takes the few copies the screen leaves,
      // which one CTA each would run as a latency tail (a copy on one CTA:
      // ~0.34 ms per Lanczos step of 4D 16^4)
      auto launch_f = [&](bool fp32) -> int {
        const size_t smf = gc::slab_fp_smem_bytes(kmax, fp32 ? 4 : 8);
        auto go = [&](auto k1, auto kc) -> int {
          if (!fp32 && cluster) {
            for (int C : {kSlabClusterWide, kSlabCluster}) {
              int ncl = 0;
              if (int rc = cluster_count(kc, 1024, smf, C, &ncl)) return rc;
              if (ncl <= 0) continue;
              if (int rc = launch_clusters(kc, fa, 1024, smf, C, ncl, s)) return rc;
              ++o->launches;
              return GC_OK;
            }
          }
          if (int rc = raise_smem_limit(k1, smf)) return rc;
          k1<<<grid_f, 1024, smf, s>>>(fa);
          ++o->launches;
          GC_CUDA(cudaGetLastError());
          return GC_OK;
        };
        if (fp32) {
          switch (d) {
            case 2: return go(gc::slab_fp_lanczos_kernel<float, 2, false>, gc::slab_fp_lanczos_kernel<float, 2, true>);
            case 3: return go(gc::slab_fp_lanczos_kernel<float, 3, false>, gc::slab_fp_lanczos_kernel<float, 3, true>);
            default: return go(gc::slab_fp_lanczos_kernel<float, 4, false>, gc::slab_fp_lanczos_kernel<float, 4, true>);
          }
        }
        switch (d) {
          case 2: return go(gc::slab_fp_lanczos_kernel<double, 2, false>, gc::slab_fp_lanczos_kernel<double, 2, true>);
          case 3: return go(gc::slab_fp_lanczos_kernel<double, 3, false>, gc::slab_fp_lanczos_kernel<double, 3, true>);
          default: return go(gc::slab_fp_lanczos_kernel<double, 4, false>, gc::slab_fp_lanczos_kernel<double, 4, true>);
        }
      };
      if (opt.fp_mode == GC_FP_AUTO) {
        GC_CUDA(cudaMemsetAsync(o->n_redo(), 0, 4, s));
        fa.list = o->t_newlist.as<unsigned>();
        fa.n_list = o->n_new();
        fa.redo = o->s_redo.as<unsigned>();
        fa.n_redo = o->n_redo();
        fa.tol = 1e-5;
        fa.scratch_bytes = sb32;
        if (int rc = launch_f(true)) return rc;
        fa.list = o->s_redo.as<unsigned>();
        fa.n_list = o->n_redo();
        fa.count_tests = 0;
      } else {
        fa.list = o->t_newlist.as<unsigned>();
        fa.n_list = o->n_new();
        fa.count_tests = 1;
      }
      fa.tol = 1e-12;
      fa.scratch_bytes = sb64;
      if (int rc = launch_f(false)) return rc;
    }
    if (ev) GC_CUDA(cudaEventRecord(ev[5], s));
    if (opt.keep_per_start) {
      const size_t off = done;
      GC_CUDA(cudaMemcpyAsync(o->rec_status.data() + off, sa.status, b, cudaMemcpyDeviceToHost, s));
      GC_CUDA(cudaMemcpyAsync(o->rec_sweeps.data() + off, sa.sweeps, b * 4, cudaMemcpyDeviceToHost, s));
      GC_CUDA(cudaMemcpyAsync(o->rec_F.data() + off, da.F, b * 8, cudaMemcpyDeviceToHost, s));
      GC_CUDA(cudaMemcpyAsync(o->rec_copy.data() + off, da.copy_of, b * 4, cudaMemcpyDeviceToHost, s));
    }
    o->next_start += b;
    o->n_starts += b;
    o->enqueued += b;
    done += b;
  }
  return GC_OK;
}

// Enqueue the whole path for n_starts starts on stream s.  With `async` no
// host synchronisation happens: the copy pool must already hold
// o->enqueued + n_starts entries, and timing and error flags are read at the
// next synchronising call.  keep_per_start implies a synchronous call.
int enumerate_impl(gc_orbit o, uint64_t n_starts, double omega, double eps, const gc_options& opt,
                   cudaStream_t s, bool async, bool timing, const Tuning& tune,
                   bool prepare_only = false) {
  if (n_starts == 0) return GC_OK;
  const int check_every = (opt.autotune == 2 && tune.check_every > 0) ? tune.check_every : opt.check_every;
  const int max_sweeps = ((opt.max_sweeps + check_every - 1) / check_every) * check_every;
  const int V = o->V, d = o->d;
  const bool mixed = opt.precision == GC_MIXED;
  o->last_precision = opt.precision;

  // batch size: staging of at most ~1 GiB
  const size_t per_start = (size_t)V * 16 + (mixed ? (size_t)V * 8 : 0) + 48;
  size_t B = opt.batch_starts > 0 ? (size_t)opt.batch_starts
                                  : (tune.batch ? tune.batch : std::max<size_t>(4096, (1ull << 30) / per_start));
  B = std::min<size_t>(B, n_starts);
  if (!o->s_status.ensure(B, s) || !o->s_sweeps.ensure(B * 4, s) || !o->s_resid.ensure(B * 8, s) ||
      !o->s_F.ensure(B * 8, s) || !o->s_fprint.ensure(B * 8, s) || !o->s_config.ensure(B * V * 16, s) ||
      !o->s_copy.ensure(B * 4, s) || (mixed && !o->s_state32.ensure(B * V * 8, s)))
    return fail(GC_ENOMEM, "cannot admit a batch of %zu starts (%.1f MiB staging)", B, B * per_start / 1048576.0);

  if (opt.keep_per_start && async) return fail(GC_EINVAL, "keep_per_start needs a synchronous call");
  if (prepare_only) {
    // staging only (set below); no records
  } else if (opt.keep_per_start) {
    o->rec_first = o->next_start;
    o->rec_n = n_starts;
    o->rec_status.assign(n_starts, 0);
    o->rec_sweeps.assign(n_starts, 0);
    o->rec_F.assign(n_starts, 0.0);
    o->rec_copy.assign(n_starts, -1);
  } else {
    o->rec_n = 0;
  }

  if (o->slab) {
    if (prepare_only) {
      size_t B_slab = 0;
      return slab_prepare(o, n_starts, opt, s, &B_slab);
    }
    return enumerate_slab(o, n_starts, omega, eps, opt, s, async, timing, check_every, max_sweeps);
  }
  // launch shapes
  const int T = o->team;
  const int tpw = 32 / T;
  auto relax_bytes = [&](int warps, int site_bytes) {
    return gc::Smem(V, d, site_bytes, (size_t)V * site_bytes, warps * tpw).total;
  };
  const int site_bytes = mixed ? 8 : 16;
  int r_warps = fit_warps(8, [&](int w) { return relax_bytes(w, site_bytes); });
  if (!r_warps) return fail(GC_EINVAL, "relaxation does not fit shared memory");
  if (tune.r_warps > 0 && tune.r_warps < r_warps) r_warps = tune.r_warps;
  const size_t r_smem = relax_bytes(r_warps, site_bytes);
  // polish: the most warps per SM, over two CTAs (links held twice) or one CTA
  // of up to 16 warps, with or without the FP64 links in shared memory (ties:
  // with them)
  bool u64_smem = true, cg = false;
  auto polish_bytes = [&](int warps) {
    return gc::Smem(V, d, gc::polish_link_bytes(u64_smem), gc::polish_team_bytes(V, d, cg), warps * tpw).total;
  };
  auto polish_shape = [&](int* per_sm) {
    const int p2 = fit_warps(8, [&](int w) { return 2 * polish_bytes(w) + 2048; });
    const int p1 = fit_warps(16, polish_bytes);
    *per_sm = std::max(2 * p2, p1);
    return 2 * p2 >= p1 ? p2 : p1;
  };
  auto best_shape = [&](bool* smem_links) {
    int per_sm_s = 0, per_sm_g = 0;
    u64_smem = true;
    const int ws = polish_shape(&per_sm_s);
    u64_smem = false;
    const int wg = polish_shape(&per_sm_g);
    *smem_links = per_sm_s >= per_sm_g && ws > 0;
    return *smem_links ? ws : wg;
  };
  int p_warps = 0;
  if (mixed) p_warps = best_shape(&u64_smem);
  if (mixed && !p_warps) return fail(GC_EINVAL, "polish does not fit shared memory");
  if (mixed && tune.p_warps > 0 && tune.p_warps < p_warps) p_warps = tune.p_warps;
  const size_t p_smem = mixed ? polish_bytes(p_warps) : 0;
  const bool p_u64 = u64_smem;
  // the redo launch (starts the line polish hands back) solves by CG: larger teams
  bool r_u64 = false;
  int r_warps_cg = 0;
  size_t r_smem_cg = 0;
  if (mixed) {
    cg = true;
    r_warps_cg = best_shape(&r_u64);
    u64_smem = r_u64;
    r_smem_cg = r_warps_cg ? polish_bytes(r_warps_cg) : 0;
    cg = false;
    u64_smem = p_u64;
  }
  const int kmax64 = std::min(opt.lanczos_k, std::max(1, V - 1));
  const int kmax32 = std::min(160, kmax64);
  const FpKernel fp64_kern = fp_test_for(d), fp32_kern = fp_screen_for(d);
  int f_warps = fit_warps(4, [&](int w) { return gc::FpSmem<double>(V, d, kmax64, w).total; });
  if (!f_warps) return fail(GC_EINVAL, "Faddeev-Popov test does not fit shared memory");
  if (tune.f_warps > 0 && tune.f_warps < f_warps) f_warps = tune.f_warps;
  const size_t f_smem = gc::FpSmem<double>(V, d, kmax64, f_warps).total;
  // the FP32 screen: twice the FP64 kernel's warps per CTA where they fit
  int s_warps = fit_warps(2 * f_warps, [&](int w) { return gc::FpSmem<float>(V, d, kmax32, w).total; });
  if (!s_warps) return fail(GC_EINVAL, "Faddeev-Popov screen does not fit shared memory");
  const size_t s_smem = gc::FpSmem<float>(V, d, kmax32, s_warps).total;

  // dense-mode Lanczos bases: one V x V slot per warp, sized for the largest batch
  int dense_grid = 0;
  if (opt.fp_mode == GC_FP_DENSE) {
    if (int rc = launch_grid(fp64_kern, f_warps * 32, f_smem, f_warps, (long long)B, &dense_grid)) return rc;
    const size_t slot = (size_t)V * V * 8;
    const size_t max_slots = std::max<size_t>(1, (1ull << 30) / slot);
    dense_grid = (int)std::min<size_t>(dense_grid, std::max<size_t>(1, max_slots / f_warps));
    if (!o->scratch.ensure((size_t)dense_grid * f_warps * slot, s))
      return fail(GC_ENOMEM, "cannot admit %zu bytes of Lanczos basis scratch", (size_t)dense_grid * f_warps * slot);
  }
  if (prepare_only) return GC_OK;

  unsigned long long* wctr = o->work.as<unsigned long long>();
  unsigned long long* stats = o->stats.as<unsigned long long>();
  if (!o->err_unchecked) GC_CUDA(cudaMemsetAsync(o->err(), 0, 16, s));
  o->err_unchecked = true;
  o->last_stream = s;

  for (uint64_t done = 0; done < n_starts;) {
    const long long b = (long long)std::min<uint64_t>(B, n_starts - done);
    // admission: the pool must hold every start of the batch as a new copy.
    // o->enqueued bounds the copies made so far, so no read-back is needed
    // while the pool is large enough for that bound.
    if (o->enqueued + (unsigned long long)b > o->cap) {
      if (async) return fail(GC_ESTATE, "asynchronous enumeration needs the copy pool reserved up front");
      unsigned cur = 0;
      GC_CUDA(cudaMemcpyAsync(&cur, o->n_entries(), 4, cudaMemcpyDeviceToHost, s));
      GC_CUDA(cudaStreamSynchronize(s));
      if ((unsigned long long)cur + b > o->cap) {
        int rc = table_reserve(o, (unsigned long long)cur + b, cur, s);
        if (rc != GC_OK) return rc;
      }
    }
    // timing events of this batch
    cudaEvent_t* ev = nullptr;
    if (timing) {
      while (o->ev_pool.size() < o->ev_used + kEvPerBatch) {
        cudaEvent_t e;
        GC_CUDA(cudaEventCreate(&e));
        o->ev_pool.push_back(e);
      }
      ev = o->ev_pool.data() + o->ev_used;
      o->ev_used += kEvPerBatch;
    }
    GC_CUDA(cudaMemsetAsync(wctr, 0, 32, s));   // relax, polish, redo polish counters; redo count
    GC_CUDA(cudaMemsetAsync(o->n_new(), 0, 4, s));
    GC_CUDA(cudaMemsetAsync(o->n_redo(), 0, 4, s));

    // relaxation
    gc::RelaxArgs ra{};
    ra.geom = o->geom;
    ra.links64 = o->links64.as<double2>();
    ra.links32 = o->links32.as<float2>();
    ra.seed = opt.seed;
    ra.orbit_id = o->orbit_id;
    ra.start0 = o->next_start;
    ra.n = b;
    ra.work_ctr = wctr;
    ra.omega = omega;
    ra.om1 = 1.0 - omega;
    ra.eps = eps;
    ra.omega32 = (float)omega;
    ra.om1_32 = (float)(1.0 - omega);
    ra.eps32 = (float)opt.eps32;
    ra.check_every = check_every;
    ra.max_sweeps = max_sweeps;
    ra.team = T;
    ra.stat_base = mixed ? kSweeps32 : kSweeps;
    ra.status = o->s_status.as<int8_t>();
    ra.sweeps = o->s_sweeps.as<int32_t>();
    ra.resid = o->s_resid.as<double>();
    ra.F = o->s_F.as<double>();
    ra.fprint = o->s_fprint.as<double>();
    ra.config = o->s_config.as<double2>();
    ra.state32 = o->s_state32.as<float2>();
    ra.stats = stats;
    int grid = 0;
    if (ev) GC_CUDA(cudaEventRecord(ev[0], s));
    const bool line_variant = mixed && opt.relax_variant != GC_RELAX_GENERIC;
    if (line_variant && d == 4 && o->L == 4) {
      constexpr int kWarps = 8;    // 198 registers: two warps per SM sub-partition
      auto k = gc::relax32_sheet_kernel<kWarps, 1>;
      const size_t sm = gc::relax32_sheet_smem<kWarps>();
      if (int rc = launch_grid(k, 32 * kWarps, sm, kWarps, b, &grid)) return rc;
      // the batch's starts first, drawn at full occupancy into the FP32 state buffer
      const int sblocks = (int)std::min<long long>((long long)b, (long long)sm_count() * 16);
      gc::start32_kernel<<<sblocks, 256, 0, s>>>(ra.seed, ra.orbit_id, ra.start0, (long long)b, V,
                                                 ra.state32);
      if (ev) GC_CUDA(cudaEventRecord(ev[6], s));
      k<<<grid, 32 * kWarps, sm, s>>>(ra);
      o->launches += 2;
    } else if (mixed && opt.relax_variant != GC_RELAX_GENERIC && d == 3 && o->L == 8) {
      if (ev) GC_CUDA(cudaEventRecord(ev[6], s));   // the sweeps draw their own starts
      constexpr int kTeams = 4;
      auto k = gc::relax32_lines_kernel<3, 8, kTeams>;
      const size_t sm = gc::relax32_lines_smem<3, 8, kTeams>();
      if (int rc = launch_grid(k, 64 * kTeams, sm, kTeams, b, &grid)) return rc;
      k<<<grid, 64 * kTeams, sm, s>>>(ra);
      ++o->launches;
    } else {
      if (ev) GC_CUDA(cudaEventRecord(ev[6], s));
      auto launch = [&](auto kern) -> int {
        if (int rc = launch_grid(kern, r_warps * 32, r_smem, (long long)r_warps * tpw, b, &grid)) return rc;
        kern<<<grid, r_warps * 32, r_smem, s>>>(ra);
        ++o->launches;
        return GC_OK;
      };
      int rc = GC_OK;
      if (mixed) {
        switch (d) {
          case 1: rc = launch(gc::relax_kernel<gc::Fast32, 1>); break;
          case 2: rc = launch(gc::relax_kernel<gc::Fast32, 2>); break;
          case 3: rc = launch(gc::relax_kernel<gc::Fast32, 3>); break;
          default: rc = launch(gc::relax_kernel<gc::Fast32, 4>); break;
        }
      } else {
        switch (d) {
          case 1: rc = launch(gc::relax_kernel<gc::Exact64, 1>); break;
          case 2: rc = launch(gc::relax_kernel<gc::Exact64, 2>); break;
          case 3: rc = launch(gc::relax_kernel<gc::Exact64, 3>); break;
          default: rc = launch(gc::relax_kernel<gc::Exact64, 4>); break;
        }
      }
      if (rc) return rc;
    }
    GC_CUDA(cudaGetLastError());
    if (ev) GC_CUDA(cudaEventRecord(ev[1], s));
    if (mixed) {
      gc::PolishArgs pa{};
      pa.geom = o->geom;
      pa.links64 = ra.links64;
      pa.links32 = ra.links32;
      pa.n = b;
      pa.work_ctr = wctr + 1;
      pa.omega = omega;
      pa.om1 = 1.0 - omega;
      pa.eps = eps;
      pa.omega_in = (float)omega;
      pa.lin_tol = 4e-4f;
      pa.inner_max = opt.newton_inner;
      pa.newton_max = opt.newton_max;
      pa.max_sweeps = max_sweeps;
      pa.check_every = check_every;
      pa.team = T;
      pa.u64_smem = u64_smem ? 1 : 0;
      pa.status = ra.status;
      pa.sweeps = ra.sweeps;
      pa.resid = ra.resid;
      pa.state32 = ra.state32;
      pa.F = ra.F;
      pa.fprint = ra.fprint;
      pa.config = ra.config;
      pa.stats = stats;
      if (line_variant && d == 4 && o->L == 4) {
        // two-line-per-lane polish; the starts it leaves are rerun by
        // polish_kernel from the redo list (staged in the copy-index buffer,
        // which dedup fills only afterwards)
        // 12 one-warp teams per SM (167 registers, no spill): on the kappa = 0.5
        // 4^4 orbit 33.8 ms per 2^20 starts, against 36.8 ms for 16 teams at
        // the 128-register cap (88 bytes spilled) and 40.7 ms for 8
        constexpr int kTeams = 12;
        auto k = gc::polish_pairs_kernel<4, 4, kTeams>;
        const size_t sm = gc::PolishPairSmem<4, 4>::bytes(kTeams);
        gc::PolishArgs pl = pa;
        pl.redo = reinterpret_cast<unsigned*>(o->s_copy.as<int>());
        pl.n_redo = wctr + 3;
        if (int rc = launch_grid(k, 32 * kTeams, sm, kTeams, b, &grid)) return rc;
        k<<<grid, 32 * kTeams, sm, s>>>(pl);
        ++o->launches;
        GC_CUDA(cudaGetLastError());
        pa.list = pl.redo;
        pa.n_list = wctr + 3;
        pa.work_ctr = wctr + 2;
        if (ev) GC_CUDA(cudaEventRecord(ev[2], s));
      } else if (r_warps_cg > 0) {
        // generic polish handing hard starts on to the CG instance
        gc::PolishArgs pm = pa;
        pm.redo = reinterpret_cast<unsigned*>(o->s_copy.as<int>());
        pm.n_redo = wctr + 3;
        auto mlaunch = [&](auto kern) -> int {
          if (int rc = launch_grid(kern, p_warps * 32, p_smem, (long long)p_warps * tpw, b, &grid)) return rc;
          kern<<<grid, p_warps * 32, p_smem, s>>>(pm);
          ++o->launches;
          return GC_OK;
        };
        int mrc = GC_OK;
        switch (d) {
          case 1: mrc = mlaunch(gc::polish_kernel<1, false>); break;
          case 2: mrc = mlaunch(gc::polish_kernel<2, false>); break;
          case 3: mrc = mlaunch(gc::polish_kernel<3, false>); break;
          default: mrc = mlaunch(gc::polish_kernel<4, false>); break;
        }
        if (mrc) return mrc;
        GC_CUDA(cudaGetLastError());
        pa.list = pm.redo;
        pa.n_list = wctr + 3;
        pa.work_ctr = wctr + 2;
        if (ev) GC_CUDA(cudaEventRecord(ev[2], s));
      }
      const bool redo_cg = pa.list && r_warps_cg > 0;
      const int pw = redo_cg ? r_warps_cg : p_warps;
      const size_t psm = redo_cg ? r_smem_cg : p_smem;
      if (redo_cg) pa.u64_smem = r_u64 ? 1 : 0;
      auto plaunch = [&](auto kern) -> int {
        if (int rc = launch_grid(kern, pw * 32, psm, (long long)pw * tpw, b, &grid)) return rc;
        kern<<<grid, pw * 32, psm, s>>>(pa);
        ++o->launches;
        return GC_OK;
      };
      int prc = GC_OK;
      if (redo_cg) {
        switch (d) {
          case 1: prc = plaunch(gc::polish_kernel<1, true>); break;
          case 2: prc = plaunch(gc::polish_kernel<2, true>); break;
          case 3: prc = plaunch(gc::polish_kernel<3, true>); break;
          default: prc = plaunch(gc::polish_kernel<4, true>); break;
        }
      } else {
        switch (d) {
          case 1: prc = plaunch(gc::polish_kernel<1, false>); break;
          case 2: prc = plaunch(gc::polish_kernel<2, false>); break;
          case 3: prc = plaunch(gc::polish_kernel<3, false>); break;
          default: prc = plaunch(gc::polish_kernel<4, false>); break;
        }
      }
      if (prc) return prc;
      GC_CUDA(cudaGetLastError());
      if (ev && !pa.list) GC_CUDA(cudaEventRecord(ev[2], s));   // no redo launch: its time is 0
    } else if (ev) {
      GC_CUDA(cudaEventRecord(ev[2], s));
    }
    if (ev) GC_CUDA(cudaEventRecord(ev[3], s));
    // deduplication
    gc::DedupArgs da{};
    da.tab = o->view();
    set_table_widths(da.tab, d, V, opt.dedup_delta);
    da.tab.f8_only = opt.dedup_mode == GC_DEDUP_F8;
    da.V = V;
    da.n = b;
    da.start0 = o->next_start;
    da.status = ra.status;
    da.F = ra.F;
    da.fprint = ra.fprint;
    da.config = ra.config;
    da.copy_of = o->s_copy.as<int>();
    da.stats = stats;
    if (int rc = launch_dedup(o, da, s)) return rc;
    if (ev) GC_CUDA(cudaEventRecord(ev[4], s));
    // Faddeev-Popov test of the copies this batch created
    if (opt.fp_mode != GC_FP_NONE) {
      gc::FpArgs fa{};
      fa.geom = o->geom;
      fa.cfg = o->t_cfg.as<double2>();
      fa.first_start = o->t_first.as<unsigned long long>();
      fa.links64 = ra.links64;
      fa.links32 = ra.links32;
      fa.list = o->t_newlist.as<unsigned>();
      fa.n_list = o->n_new();
      fa.redo = o->t_newlist.as<unsigned>() + o->cap;
      fa.n_redo = o->n_redo();
      fa.lambda2 = o->t_lam.as<double>();
      fa.region = o->t_region.as<int>();
      fa.mode = opt.fp_mode;
      fa.kmax32 = kmax32;
      fa.kmax64 = kmax64;
      fa.count_tests = 1;
      fa.tau = opt.fp_tau;
      fa.margin32 = 1e-3;
      fa.tol32 = 1e-5;
      fa.tol64 = 1e-12;
      fa.extra32 = 16;
      fa.seed = opt.seed;
      fa.stats = stats;
      int fgrid = 0;
      if (opt.fp_mode == GC_FP_AUTO) {
        // FP32 screen of every new copy, then FP64 Lanczos for those it leaves
        int sgrid = 0;
        if (d == 4 && o->L == 4) {   // lines of each parity fill a warp: two lines per lane
          auto k = gc::fp_screen_pairs_kernel<4, 4>;
          const size_t sm = gc::FpPairSmem<4, 4>::bytes(8, kmax32);
          if (int rc = launch_grid(k, 256, sm, 8, b, &sgrid)) return rc;
          k<<<sgrid, 256, sm, s>>>(fa);
        } else {
          if (int rc = launch_grid(fp32_kern, s_warps * 32, s_smem, s_warps, b, &sgrid)) return rc;
          fp32_kern<<<sgrid, s_warps * 32, s_smem, s>>>(fa);
        }
        ++o->launches;
        GC_CUDA(cudaGetLastError());
        fa.list = fa.redo;
        fa.n_list = fa.n_redo;
        fa.mode = gc::kFpLanczos;
        fa.count_tests = 0;
      }
      if (fa.mode == gc::kFpLanczos && d == 4 && o->L == 4) {
        // lines of each parity fill a warp: the FP32 seed in registers
        // one 12-warp CTA per SM (166 registers, no spill; 169 KB of shared
        // memory): 66.3 ms for the kappa = 0.5 4^4 orbit's 398 842 copies,
        // against 76.4 ms for two 8-warp CTAs at the 128-register cap
        auto k = gc::fp_test_pairs_kernel<4, 4>;
        const size_t sm = gc::FpTestPairSmem<4, 4>::bytes(12, kmax32, std::min(kmax64, gc::FpTestPairSmem<4, 4>::kMax64));
        if (int rc = launch_grid(k, 384, sm, 12, b, &fgrid)) return rc;
        k<<<fgrid, 384, sm, s>>>(fa);
      } else {
        if (int rc = launch_grid(fp64_kern, f_warps * 32, f_smem, f_warps, b, &fgrid)) return rc;
        if (opt.fp_mode == GC_FP_DENSE) {
          fgrid = std::min(fgrid, dense_grid);
          fa.scratch = o->scratch.as<double>();
        }
        fp64_kern<<<fgrid, f_warps * 32, f_smem, s>>>(fa);
      }
      ++o->launches;
      GC_CUDA(cudaGetLastError());
    }
    if (ev) GC_CUDA(cudaEventRecord(ev[5], s));
    if (opt.keep_per_start) {
      const size_t off = done;
      GC_CUDA(cudaMemcpyAsync(o->rec_status.data() + off, ra.status, b, cudaMemcpyDeviceToHost, s));
      GC_CUDA(cudaMemcpyAsync(o->rec_sweeps.data() + off, ra.sweeps, b * 4, cudaMemcpyDeviceToHost, s));
      GC_CUDA(cudaMemcpyAsync(o->rec_F.data() + off, ra.F, b * 8, cudaMemcpyDeviceToHost, s));
      GC_CUDA(cudaMemcpyAsync(o->rec_copy.data() + off, da.copy_of, b * 4, cudaMemcpyDeviceToHost, s));
    }
    o->next_start += b;
    o->n_starts += b;
    o->enqueued += b;
    done += b;
  }
  return GC_OK;
}

}  // namespace

extern "C" {

int gc_enumerate_copies(gc_orbit o, uint64_t n_starts, double omega, double eps, const gc_options* opt_in) {
  if (!o) return fail(GC_EINVAL, "gc_enumerate_copies: NULL orbit");
  gc_options opt;
  if (opt_in) opt = *opt_in; else gc_options_default(&opt);
  if (int rc = validate_options(opt, omega, eps)) return rc;
  if (n_starts == 0) return GC_OK;
  cudaStream_t s = (cudaStream_t)opt.stream;
  if (opt.autotune && !o->slab && !have_tuning(o->d, o->L, opt.precision, deep_tuning(opt))) {
    Tuning t;
    if (int rc = autotune_shape(o, opt, omega, eps, &t)) return rc;
  }
  const Tuning tune = cached_tuning(o->d, o->L, opt.precision, deep_tuning(opt));
  if (int rc = enumerate_impl(o, n_starts, omega, eps, opt, s, false, true, tune)) return rc;
  GC_CUDA(cudaStreamSynchronize(s));
  harvest_timing(o);
  return check_errors(o);
}

namespace {

// Entries in the pool after the last call (synchronises its stream and reports
// device-side errors).
int read_count(gc_orbit o, unsigned* n_out) {
  GC_CUDA(cudaStreamSynchronize(o->last_stream));
  harvest_timing(o);
  if (int rc = check_errors(o)) return rc;
  unsigned n = 0;
  GC_CUDA(read_back(&n, o->n_entries(), 4, o->last_stream));
  *n_out = std::min(n, o->cap);
  return GC_OK;
}

// Stable radix sort (gc_sort.cuh) of n (key, value) pairs by key, over the
// 8-bit digits that vary among the keys; ping-pongs between (k0, v0) and
// (k1, v1) and leaves the sorted pairs in *kres / *vres.  scratch holds
// 4 + 256 * sort_tiles(n) words.  Synchronises s once (to read which digits
// vary).
}  // namespace
}  // extern "C"

namespace {
template <typename VT>
int radix_sort_pairs(unsigned long long* k0, unsigned long long* k1, VT* v0, VT* v1, unsigned n,
                     unsigned* scratch, cudaStream_t s, unsigned long long** kres, VT** vres,
                     uint64_t* launches) {
  unsigned long long* or_and = reinterpret_cast<unsigned long long*>(scratch);
  unsigned* hist = scratch + 4;
  GC_CUDA(cudaMemsetAsync(or_and, 0, 8, s));
  GC_CUDA(cudaMemsetAsync(or_and + 1, 0xff, 8, s));
  const unsigned blocks = std::max(1u, std::min<unsigned>((n + 255) / 256, 1024));
  gc::key_bits_kernel<<<blocks, 256, 0, s>>>(k0, n, or_and);
  unsigned long long h[2] = {0ull, 0ull};
  GC_CUDA(cudaMemcpyAsync(h, or_and, 16, cudaMemcpyDeviceToHost, s));
  GC_CUDA(cudaStreamSynchronize(s));
  *launches += 1;
  const unsigned long long vary = h[0] ^ h[1];
  const unsigned tiles = gc::sort_tiles(n);
  for (int shift = 0; shift < 64; shift += 8) {
    if (((vary >> shift) & 255ull) == 0ull) continue;   // every key has this digit
    gc::radix_hist_kernel<<<tiles, gc::kSortThreads, 0, s>>>(k0, n, shift, hist, tiles);
    gc::radix_scan_kernel<<<1, 1024, 0, s>>>(hist, (unsigned)gc::kSortBins * tiles);
    gc::radix_scatter_kernel<VT><<<tiles, gc::kSortThreads, 0, s>>>(k0, v0, k1, v1, n, shift, hist, tiles);
    std::swap(k0, k1);
    std::swap(v0, v1);
    *launches += 3;
  }
  GC_CUDA(cudaGetLastError());
  *kres = k0;
  *vres = v0;
  return GC_OK;
}

}  // namespace

extern "C" {
namespace {

size_t sort_scratch_bytes(unsigned n) { return (4 + (size_t)gc::kSortBins * gc::sort_tiles(n)) * 4; }

// Device array of pool entries in (F, first start) order: two stable radix
// sorts, by first start and then by F's order-preserving bit key.  Returns
// nullptr for n = 0.
int device_order(gc_orbit o, unsigned n, const unsigned** order) {
  *order = nullptr;
  if (n == 0) return GC_OK;
  cudaStream_t s = o->last_stream;
  if (!o->sort_keys.ensure((size_t)n * 16, s) || !o->sort_idx.ensure((size_t)n * 8, s) ||
      !o->sort_tmp.ensure(sort_scratch_bytes(n), s))
    return fail(GC_ENOMEM, "cannot admit %u sort records", n);
  unsigned long long* k0 = o->sort_keys.as<unsigned long long>();
  unsigned long long* k1 = k0 + n;
  unsigned* i0 = o->sort_idx.as<unsigned>();
  unsigned* i1 = i0 + n;
  unsigned* scratch = o->sort_tmp.as<unsigned>();
  const int blocks = (int)std::min<unsigned>((n + 255) / 256, 4096);
  GC_CUDA(cudaMemcpyAsync(k0, o->t_first.p, (size_t)n * 8, cudaMemcpyDeviceToDevice, s));
  gc::iota_kernel<<<blocks, 256, 0, s>>>(i0, n);
  ++o->launches;
  unsigned long long* kr = nullptr;
  unsigned* ir = nullptr;
  if (int rc = radix_sort_pairs<unsigned>(k0, k1, i0, i1, n, scratch, s, &kr, &ir, &o->launches)) return rc;
  unsigned long long* kf = kr == k0 ? k1 : k0;
  unsigned* ispare = ir == i0 ? i1 : i0;
  gc::f_keys_kernel<<<blocks, 256, 0, s>>>(o->t_F.as<double>(), ir, kf, n);
  ++o->launches;
  unsigned long long* kr2 = nullptr;
  unsigned* ir2 = nullptr;
  if (int rc = radix_sort_pairs<unsigned>(kf, kr, ir, ispare, n, scratch, s, &kr2, &ir2, &o->launches)) return rc;
  *order = ir2;
  return GC_OK;
}

}  // namespace

int gc_fetch_minima_f8(gc_orbit o, size_t capacity, size_t* n_minima, double* F_norm, uint64_t* count) {
  if (!o) return fail(GC_EINVAL, "gc_fetch_minima_f8: NULL orbit");
  if (!n_minima) return fail(GC_EINVAL, "gc_fetch_minima_f8: n_minima is NULL");
  *n_minima = 0;
  unsigned n_pool = 0;
  if (int rc = read_count(o, &n_pool)) return rc;   // synchronises, checks the error flags
  if (!o->f8cap) return GC_OK;
  unsigned long long nf8 = 0;
  GC_CUDA(read_back(&nf8, o->n_f8(), 8, o->last_stream));
  const unsigned n = (unsigned)std::min<unsigned long long>(nf8, o->f8cap);
  *n_minima = n;
  if (capacity == 0 || n == 0 || !F_norm) return GC_OK;
  const unsigned k = (unsigned)std::min<size_t>(capacity, n);
  cudaStream_t s = o->last_stream;
  if (!o->f8_tmp.ensure((size_t)n * 32 + 16, s)) return fail(GC_ENOMEM, "cannot admit %u F-set records", n);
  unsigned long long* k0 = o->f8_tmp.as<unsigned long long>();
  unsigned long long* k1 = k0 + n;
  unsigned long long* c0 = k1 + n;
  unsigned long long* c1 = c0 + n;
  unsigned* ctr = reinterpret_cast<unsigned*>(c1 + n);
  if (!o->sort_tmp.ensure(sort_scratch_bytes(n), s)) return fail(GC_ENOMEM, "cannot admit sort scratch");
  GC_CUDA(cudaMemsetAsync(ctr, 0, 4, s));
  const unsigned blocks = std::min<unsigned>((o->f8cap + 255) / 256, 4096);
  f8_compact_kernel<<<blocks, 256, 0, s>>>(o->t_f8.as<unsigned long long>(), o->t_f8n.as<unsigned long long>(),
                                           o->f8cap, k0, c0, ctr, n);
  ++o->launches;
  unsigned long long* kr = nullptr;
  unsigned long long* cr = nullptr;
  if (int rc = radix_sort_pairs<unsigned long long>(k0, k1, c0, c1, n, o->sort_tmp.as<unsigned>(), s, &kr, &cr,
                                                    &o->launches))
    return rc;
  std::vector<unsigned long long> keys(k), starts(count ? k : 0);
  GC_CUDA(cudaMemcpyAsync(keys.data(), kr, (size_t)k * 8, cudaMemcpyDeviceToHost, s));
  if (count) GC_CUDA(cudaMemcpyAsync(starts.data(), cr, (size_t)k * 8, cudaMemcpyDeviceToHost, s));
  GC_CUDA(cudaStreamSynchronize(s));
  for (unsigned i = 0; i < k; ++i) F_norm[i] = (double)keys[i] * 1e-8;
  if (count) for (unsigned i = 0; i < k; ++i) count[i] = starts[i];
  return GC_OK;
}

}  // extern "C"

namespace {
// The body of both fetches; `wait` leaves the device-to-host copies for
// gc_fetch_wait when false.
int fetch_copies_impl(gc_orbit o, size_t capacity, size_t* n_distinct, double* F, double* theta,
                      uint64_t* first_start, uint64_t* count, double* lambda2, int* region, bool wait) {
  if (!o) return fail(GC_EINVAL, "gc_fetch_copies: NULL orbit");
  if (!n_distinct) return fail(GC_EINVAL, "gc_fetch_copies: n_distinct is NULL");
  GC_CUDA(finish_fetch(o));   // the staging buffer of an earlier asynchronous fetch is in use until then
  unsigned n = 0;
  if (int rc = read_count(o, &n)) return rc;
  *n_distinct = n;
  if (capacity == 0 || n == 0) return GC_OK;
  const unsigned k = (unsigned)std::min<size_t>(capacity, n);
  const size_t V = o->V;
  cudaStream_t s = o->last_stream;
  const unsigned* order = nullptr;
  if (int rc = device_order(o, n, &order)) return rc;
  // staging in sorted order: F, first, count, lambda_2 (8 B each), region (4 B), theta (V doubles)
  const size_t meta = (size_t)k * 36 + 16, th = theta ? (size_t)k * V * 8 : 0;
  if (!o->theta_tmp.ensure(meta + th, s)) return fail(GC_ENOMEM, "cannot admit fetch buffer");
  unsigned char* st = o->theta_tmp.as<unsigned char>();
  double* sF = reinterpret_cast<double*>(st);
  unsigned long long* sfirst = reinterpret_cast<unsigned long long*>(st + (size_t)k * 8);
  unsigned long long* scount = sfirst + k;
  double* slam = reinterpret_cast<double*>(scount + k);
  int* sreg = reinterpret_cast<int*>(slam + k);
  double* sth = reinterpret_cast<double*>(st + (((size_t)k * 36 + 15) & ~size_t(15)));
  // The gathering and the copies run on the orbit's stream (synchronous
  // fetch), or on the read-back stream after the ordering (asynchronous: the
  // orbit's stream, which the other orbits of a batch share and whose next
  // fetch synchronises it, stays free of them).
  cudaStream_t c = s;
  if (!wait) {
    for (auto& e : o->fetch_ev)
      if (!e) GC_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    c = d2h_stream();
    GC_CUDA(cudaEventRecord(o->fetch_ev[0], s));
    GC_CUDA(cudaStreamWaitEvent(c, o->fetch_ev[0], 0));
  }
  {
    const int blocks = (int)std::min<unsigned>((k + 255) / 256, 4096);
    gc::gather_meta_kernel<<<blocks, 256, 0, c>>>(order, k, o->t_F.as<double>(), o->t_first.as<unsigned long long>(),
                                                  o->t_count.as<unsigned long long>(), o->t_lam.as<double>(),
                                                  o->t_region.as<int>(), sF, sfirst, scount, slam, sreg);
    ++o->launches;
  }
  if (theta) {
    const double* table = angle_table();
    if (!table) return fail(GC_ENOMEM, "cannot set up the fetch's angle table");
    const int threads = (int)std::min<size_t>(256, (V + 31) / 32 * 32);   // a copy's sites
    // the synchronous fetch has the GPU to itself; the asynchronous one runs
    // beside the next batch's kernels, where a block per SM disturbs them
    // least (pipelined steps of the 4^4 bench workload: 685 ms against 701
    // with 16 blocks per SM)
    const int blocks = (int)std::min<unsigned>(k, (unsigned)sm_count() * (wait ? 16 : 1));
    gc::gather_angles_kernel<<<blocks, threads, 0, c>>>(order, k, (int)V, o->t_cfg.as<double2>(), table, sth);
    ++o->launches;
  }
  GC_CUDA(cudaGetLastError());
  if (F) GC_CUDA(cudaMemcpyAsync(F, sF, (size_t)k * 8, cudaMemcpyDeviceToHost, c));
  if (first_start) GC_CUDA(cudaMemcpyAsync(first_start, sfirst, (size_t)k * 8, cudaMemcpyDeviceToHost, c));
  if (count) GC_CUDA(cudaMemcpyAsync(count, scount, (size_t)k * 8, cudaMemcpyDeviceToHost, c));
  if (lambda2) GC_CUDA(cudaMemcpyAsync(lambda2, slam, (size_t)k * 8, cudaMemcpyDeviceToHost, c));
  if (region) GC_CUDA(cudaMemcpyAsync(region, sreg, (size_t)k * 4, cudaMemcpyDeviceToHost, c));
  if (theta) GC_CUDA(cudaMemcpyAsync(theta, sth, (size_t)k * V * 8, cudaMemcpyDeviceToHost, c));
  if (wait) {
    GC_CUDA(cudaStreamSynchronize(s));
  } else {
    GC_CUDA(cudaEventRecord(o->fetch_ev[1], c));
    o->fetch_pending = true;
  }
  return GC_OK;
}
}  // namespace

extern "C" {

int gc_fetch_copies(gc_orbit o, size_t capacity, size_t* n_distinct, double* F, double* theta,
                    uint64_t* first_start, uint64_t* count, double* lambda2, int* region) {
  return fetch_copies_impl(o, capacity, n_distinct, F, theta, first_start, count, lambda2, region, true);
}

int gc_fetch_copies_async(gc_orbit o, size_t capacity, size_t* n_distinct, double* F, double* theta,
                          uint64_t* first_start, uint64_t* count, double* lambda2, int* region) {
  return fetch_copies_impl(o, capacity, n_distinct, F, theta, first_start, count, lambda2, region, false);
}

int gc_fetch_wait(gc_orbit o) {
  if (!o) return fail(GC_EINVAL, "gc_fetch_wait: NULL orbit");
  GC_CUDA(finish_fetch(o));
  return GC_OK;
}

int gc_load_copies(gc_orbit o, size_t n, const double* F, const double* theta, const uint64_t* first_start,
                   const uint64_t* count, const double* lambda2, const int* region, size_t n_minima,
                   const double* F_norm, const uint64_t* minima_count, uint64_t next_start) {
  if (!o) return fail(GC_EINVAL, "gc_load_copies: NULL orbit");
  if (o->served_by) return fail(GC_ESTATE, "gc_load_copies: the orbit belongs to a server");
  if (o->next_start != 0 || o->n_starts != 0)
    return fail(GC_ESTATE, "gc_load_copies: the orbit has run starts already (restore into a new orbit)");
  if (n && (!F || !theta || !first_start || !count || !lambda2 || !region))
    return fail(GC_EINVAL, "gc_load_copies: NULL copy array");
  if (n_minima && (!F_norm || !minima_count)) return fail(GC_EINVAL, "gc_load_copies: NULL minima array");
  if (n > 0x7fffffffULL || n_minima > 0x3fffffffULL) return fail(GC_EINVAL, "gc_load_copies: too many records");
  for (size_t i = 0; i < n; ++i) {
    if (first_start[i] >= next_start)
      return fail(GC_EINVAL, "copy %zu: first start %llu not below next_start %llu", i,
                  (unsigned long long)first_start[i], (unsigned long long)next_start);
    if (count[i] == 0) return fail(GC_EINVAL, "copy %zu: count 0", i);
    if (region[i] < -1 || region[i] > 2) return fail(GC_EINVAL, "copy %zu: region flag %d", i, region[i]);
  }
  std::vector<unsigned long long> k8(n_minima);
  for (size_t i = 0; i < n_minima; ++i) {
    const double k = std::nearbyint(F_norm[i] * 1e8);   // the fetch gives key * 1e-8
    if (!(k >= 0.0 && k < 9.0e15)) return fail(GC_EINVAL, "minimum %zu: F_norm %g out of range", i, F_norm[i]);
    k8[i] = (unsigned long long)k;
  }
  cudaStream_t s = o->last_stream;
  unsigned cur = 0;
  if (int rc = read_count(o, &cur)) return rc;
  unsigned long long nf8 = 0;
  GC_CUDA(read_back(&nf8, o->n_f8(), 8, s));
  if (cur || nf8) return fail(GC_ESTATE, "gc_load_copies: the orbit's table is not empty");
  // room for the copies, and an F set at most half full
  const unsigned long long need = std::max<unsigned long long>(n, (n_minima + 1) / 2);
  if (int rc = table_reserve(o, need, 0, s)) return rc;
  const size_t V = o->V;
  const size_t off_F = 0, off_first = off_F + n * 8, off_count = off_first + n * 8, off_lam = off_count + n * 8,
               off_reg = off_lam + n * 8, off_th = (off_reg + n * 4 + 15) & ~size_t(15),
               off_k8 = off_th + n * V * 8, off_c8 = off_k8 + n_minima * 8, bytes = off_c8 + n_minima * 8 + 16;
  Buf tmp;
  if (!tmp.ensure(bytes, s)) return fail(GC_ENOMEM, "cannot admit %zu copies to restore", n);
  unsigned char* d = tmp.as<unsigned char>();
  int rc = GC_OK;
  auto up = [&](size_t off, const void* src, size_t nb) {
    if (rc == GC_OK && nb && cudaMemcpyAsync(d + off, src, nb, cudaMemcpyHostToDevice, s) != cudaSuccess)
      rc = fail(GC_ECUDA, "gc_load_copies: upload failed");
  };
  up(off_F, F, n * 8);
  up(off_first, first_start, n * 8);
  up(off_count, count, n * 8);
  up(off_lam, lambda2, n * 8);
  up(off_reg, region, n * 4);
  up(off_th, theta, n * V * 8);
  up(off_k8, k8.data(), n_minima * 8);
  up(off_c8, minima_count, n_minima * 8);
  if (rc == GC_OK && n) {
    gc::TableView T = o->view();
    set_table_widths(T, o->d, (int)V, 0.0);
    const int blocks = (int)std::min<size_t>((n + 7) / 8, (size_t)sm_count() * 8);
    gc::restore_kernel<<<blocks, 256, 0, s>>>(T, (unsigned)n, (int)V, reinterpret_cast<const double*>(d + off_th),
                                             reinterpret_cast<const double*>(d + off_F),
                                             reinterpret_cast<const unsigned long long*>(d + off_first),
                                             reinterpret_cast<const unsigned long long*>(d + off_count),
                                             reinterpret_cast<const double*>(d + off_lam),
                                             reinterpret_cast<const int*>(d + off_reg), o->links64.as<double2>());
    gc::relink_kernel<<<std::min<unsigned>(((unsigned)n + 255) / 256, 4096), 256, 0, s>>>(T, (unsigned)n);
    o->launches += 2;
  }
  if (rc == GC_OK && n_minima) {
    const unsigned blocks = std::min<unsigned>(((unsigned)n_minima + 255) / 256, 4096);
    f8_rehash_kernel<<<blocks, 256, 0, s>>>(reinterpret_cast<const unsigned long long*>(d + off_k8),
                                              reinterpret_cast<const unsigned long long*>(d + off_c8),
                                              (unsigned)n_minima, o->t_f8.as<unsigned long long>(),
                                              o->t_f8n.as<unsigned long long>(), o->f8cap - 1, o->err());
    ++o->launches;
  }
  const unsigned n32 = (unsigned)n;
  const unsigned long long m64 = n_minima;
  if (rc == GC_OK && cudaGetLastError() != cudaSuccess) rc = fail(GC_ECUDA, "gc_load_copies: launch failed");
  if (rc == GC_OK && (cudaMemcpyAsync(o->n_entries(), &n32, 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
                      cudaMemcpyAsync(o->n_f8(), &m64, 8, cudaMemcpyHostToDevice, s) != cudaSuccess))
    rc = fail(GC_ECUDA, "gc_load_copies: counter upload failed");
  const cudaError_t e = cudaStreamSynchronize(s);   // the staging buffer and the counters' sources
  tmp.release(s);
  if (rc != GC_OK) return rc;
  if (e != cudaSuccess) return fail(GC_ECUDA, "gc_load_copies: %s", cudaGetErrorString(e));
  o->err_unchecked = true;   // the F set's insertions report a full set there
  if (int r = check_errors(o)) return r;
  o->next_start = next_start;
  o->enqueued = n;   // the bound on the pool's entries that admission grows the pool from
  return GC_OK;
}

int gc_fetch_starts(gc_orbit o, uint64_t first, uint64_t n, int* status, int* sweeps, double* F,
                    int64_t* copy_idx) {
  if (!o) return fail(GC_EINVAL, "gc_fetch_starts: NULL orbit");
  if (o->rec_n == 0) return fail(GC_ESTATE, "no per-start records (enable keep_per_start)");
  if (first < o->rec_first || first + n > o->rec_first + o->rec_n)
    return fail(GC_EINVAL, "starts [%llu, %llu) outside the last call's range [%llu, %llu)",
                (unsigned long long)first, (unsigned long long)(first + n),
                (unsigned long long)o->rec_first, (unsigned long long)(o->rec_first + o->rec_n));
  std::vector<int64_t> pos;
  if (copy_idx) {
    unsigned ne = 0;
    if (int rc = read_count(o, &ne)) return rc;
    const unsigned* order = nullptr;
    if (int rc = device_order(o, ne, &order)) return rc;
    std::vector<unsigned> ord(ne);
    if (ne) GC_CUDA(cudaMemcpyAsync(ord.data(), order, (size_t)ne * 4, cudaMemcpyDeviceToHost, o->last_stream));
    GC_CUDA(cudaStreamSynchronize(o->last_stream));
    pos.assign(ne, -1);
    for (unsigned i = 0; i < ne; ++i) pos[ord[i]] = i;
  }
  for (uint64_t i = 0; i < n; ++i) {
    const size_t r = (size_t)(first - o->rec_first + i);
    if (status) status[i] = o->rec_status[r];
    if (sweeps) sweeps[i] = o->rec_sweeps[r];
    if (F) F[i] = o->rec_F[r];
    if (copy_idx) {
      const int c = o->rec_copy[r];
      copy_idx[i] = (c >= 0 && (size_t)c < pos.size()) ? pos[c] : -1;
    }
  }
  return GC_OK;
}

int gc_orbit_stats(gc_orbit o, gc_stats* out) {
  if (!o || !out) return fail(GC_EINVAL, "gc_orbit_stats: NULL argument");
  std::memset(out, 0, sizeof *out);
  GC_CUDA(cudaStreamSynchronize(o->last_stream));
  harvest_timing(o);
  unsigned long long st[kNumStats] = {};
  GC_CUDA(read_back(st, o->stats.p, sizeof st, o->last_stream));
  unsigned long long nf8 = 0;
  GC_CUDA(read_back(&nf8, o->n_f8(), 8, o->last_stream));
  unsigned n = 0;
  if (int rc = read_count(o, &n)) return rc;
  std::vector<int> reg(n);
  if (n) GC_CUDA(read_back(reg.data(), o->t_region.p, (size_t)n * 4, o->last_stream));
  out->n_starts = o->n_starts;
  out->n_converged = st[kConv] + st[kPConv];
  out->n_not_converged = st[kNConv] + st[kPNConv];
  out->n_dedup_failed = st[kDFail];
  out->n_distinct = n;
  out->n_distinct_F8 = nf8;
  for (unsigned i = 0; i < n; ++i) {
    switch (reg[i]) {
      case GC_REGION_IN: out->n_in++; break;
      case GC_REGION_OUT: out->n_out++; break;
      case GC_REGION_MARGINAL: out->n_marginal++; break;
      default: out->n_untested++; break;
    }
  }
  out->sweeps_fp32 = st[kSweeps32];
  out->site_updates_fp32 = st[kUpdates32] + st[kUpd32Fallback];
  out->sweeps_fp64 = st[kSweeps] + st[kUpd64] / (unsigned long long)o->V;
  out->site_updates_fp64 = st[kUpdates] + st[kUpd64];
  out->newton_steps = st[kNewton];
  out->newton_inner_sweeps = st[kInner];
  out->polish_fallbacks = st[kFallback];
  out->fp64_residual_passes = st[kPass];
  out->fp_tests = st[kTests];
  out->fp_tests_fp64 = st[kTests64];
  out->lanczos_steps = st[kLanczos];
  out->lanczos_steps_fp64 = st[kLanczos64];
  out->ms_relax = o->ms[0];
  out->ms_polish = o->ms[1];
  out->ms_dedup = o->ms[2];
  out->ms_fptest = o->ms[3];
  out->ms_polish_redo = o->ms[4];
  out->ms_starts = o->ms[5];
  out->polish_redo_starts = st[kRedo];
  out->kernel_launches = o->launches;
  out->df_residual_passes = st[kPassDF];
  return GC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free Faddeev-Popov test (declared in gribov.h as
// gc_fp_test_static).  For callers that must not allocate device memory at
// all -- code running inside a CUDA-graph capture, a memory-budgeted service
// whose allocator is locked, or a host that owns a fixed device arena -- the
// dense Lanczos test runs on caller-owned inputs and outputs and keeps its
// scratch (the Lanczos bases and a few bookkeeping words) in one fixed
// device array that every GPU loading this library holds until the process
// exits.  The paper has no counterpart; the operation is the first-region
// test of the enumeration, GC_FP_DENSE mode.
// ---------------------------------------------------------------------------
#include <mutex>

namespace {

constexpr size_t kStaticScratchBytes = (size_t)24 << 20;  // 24 MiB per device
constexpr unsigned long long kStaticMaxCopies = 1ULL << 16;  // copies per call
constexpr int kStaticMaxDevices = 64;

}  // namespace

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

namespace {

std::mutex g_static_mu;
void* g_static_ptr[kStaticMaxDevices] = {};

// Device address of g_static_scratch on the current device, looked up once per
// device (the first call on a device does this; make it before any capture).
int static_scratch_address(void** out) {
  int dev = 0;
  GC_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kStaticMaxDevices) return fail(GC_EINVAL, "device %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return fail(GC_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    g_static_ptr[dev] = p;
  }
  *out = g_static_ptr[dev];
  return GC_OK;
}

struct StaticLayout {
  size_t header, list, first, links32, stats, q0, slot_bytes;
  unsigned slots;
  StaticLayout(unsigned long long n, int V, int d) {
    header = 0;                                           // n_list (u32)
    list = 256;
    first = align_up(list + n * 4, 256);
    links32 = align_up(first + n * 8, 256);
    stats = align_up(links32 + (size_t)V * d * sizeof(float2), 256);
    q0 = align_up(stats + 32 * 8, 256);
    slot_bytes = (size_t)V * V * sizeof(double);
    slots = q0 < kStaticScratchBytes ? (unsigned)((kStaticScratchBytes - q0) / slot_bytes) : 0u;
  }
  static size_t align_up(size_t b, size_t a) { return (b + a - 1) / a * a; }
};

// Writes every scratch word the test reads: the copy count, the identity copy
// list, the Lanczos seeds, the FP32 links, and zeroed counters.
__global__ void static_fp_setup_kernel(unsigned char* s, StaticLayout lay, unsigned n,
                                       const double2* links64, int nlinks) {
  const unsigned tid = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned stride = gridDim.x * blockDim.x;
  if (tid == 0) *reinterpret_cast<unsigned*>(s + lay.header) = n;
  for (unsigned i = tid; i < n; i += stride) {
    reinterpret_cast<unsigned*>(s + lay.list)[i] = i;
    reinterpret_cast<unsigned long long*>(s + lay.first)[i] = i;
  }
  for (unsigned l = tid; l < (unsigned)nlinks; l += stride) {
    const double2 v = links64[l];
    reinterpret_cast<float2*>(s + lay.links32)[l] = make_float2((float)v.x, (float)v.y);
  }
  for (unsigned k = tid; k < 32; k += stride) reinterpret_cast<unsigned long long*>(s + lay.stats)[k] = 0ULL;
}

}  // namespace

extern "C" int gc_fp_test_static(int dim, int L, const double* d_links, const double* d_configs,
                                 uint64_t n, double fp_tau, double* d_lambda2, int* d_region,
                                 void* stream) {
  if (dim < 1 || dim > gc::kMaxDim) return fail(GC_EINVAL, "dimension %d not in 1..4", dim);
  if (L < 2) return fail(GC_EINVAL, "L = %d < 2", L);
  const double Vd = std::pow((double)L, dim);
  if (Vd > gc::kMaxSites) return fail(GC_EINVAL, "lattice of %.0f sites exceeds %d", Vd, gc::kMaxSites);
  if (!d_links || !d_configs || !d_lambda2 || !d_region) return fail(GC_EINVAL, "NULL pointer argument");
  if (!(fp_tau >= 0.0)) return fail(GC_EINVAL, "fp_tau = %g < 0", fp_tau);
  if (n > kStaticMaxCopies)
    return fail(GC_EINVAL, "%llu copies exceed the per-call maximum of %llu of the static scratch",
                (unsigned long long)n, kStaticMaxCopies);
  const int V = (int)Vd, d = dim;
  const StaticLayout lay(n, V, d);
  if (lay.slots < 1)
    return fail(GC_EINVAL, "a %d-site lattice needs %zu bytes of Lanczos basis; the static scratch "
                "holds %zu", V, lay.q0 + lay.slot_bytes, kStaticScratchBytes);
  if (n == 0) return GC_OK;
  void* base = nullptr;
  if (int rc = static_scratch_address(&base)) return rc;
  unsigned char* s = static_cast<unsigned char*>(base);
  cudaStream_t st = (cudaStream_t)stream;

  gc::Geom G{};
  G.d = d; G.L = L; G.V = V; G.ncolor = (L % 2 == 0) ? 2 : 3;
  int cnt[3] = {0, 0, 0};
  for (int x = 0; x < V; ++x) cnt[gc::site_color(x, d, L)]++;
  for (int c = 0; c < 3; ++c) G.color_off[c + 1] = G.color_off[c] + (c < G.ncolor ? cnt[c] : 0);
  G.pos_last = G.color_off[gc::site_color(V - 1, d, L) + 1] - 1;

  const int kmax64 = std::max(1, V - 1);
  const FpKernel fkern = fp_test_for(d);
  const int f_warps = fit_warps(4, [&](int w) { return gc::FpSmem<double>(V, d, kmax64, w).total; });
  if (!f_warps) return fail(GC_EINVAL, "Faddeev-Popov test does not fit shared memory");
  const size_t f_smem = gc::FpSmem<double>(V, d, kmax64, f_warps).total;
  int fgrid = 0;
  if (int rc = launch_grid(fkern, f_warps * 32, f_smem, f_warps, (long long)n, &fgrid)) return rc;
  fgrid = (int)std::max(1u, std::min<unsigned>((unsigned)fgrid, lay.slots / (unsigned)f_warps));
  const int fwarps_used = lay.slots < (unsigned)f_warps ? (int)lay.slots : f_warps;
  const size_t fsm = gc::FpSmem<double>(V, d, kmax64, fwarps_used).total;

  static_fp_setup_kernel<<<64, 256, 0, st>>>(s, lay, (unsigned)n, reinterpret_cast<const double2*>(d_links), V * d);
  GC_CUDA(cudaGetLastError());

  gc::FpArgs fa{};
  fa.geom = G;
  fa.cfg = reinterpret_cast<const double2*>(d_configs);
  fa.first_start = reinterpret_cast<const unsigned long long*>(s + lay.first);
  fa.links32 = reinterpret_cast<const float2*>(s + lay.links32);
  fa.links64 = reinterpret_cast<const double2*>(d_links);
  fa.list = reinterpret_cast<const unsigned*>(s + lay.list);
  fa.n_list = reinterpret_cast<const unsigned*>(s + lay.header);
  fa.lambda2 = d_lambda2;
  fa.region = d_region;
  fa.mode = gc::kFpDense;
  fa.kmax32 = std::min(160, kmax64);
  fa.kmax64 = kmax64;
  fa.count_tests = 1;
  fa.tau = fp_tau;
  fa.margin32 = 1e-3;
  fa.tol32 = 1e-5;
  fa.tol64 = 1e-12;
  fa.extra32 = 16;
  fa.scratch = reinterpret_cast<double*>(s + lay.q0);
  fa.seed = 1;
  fa.stats = reinterpret_cast<unsigned long long*>(s + lay.stats);
  fkern<<<fgrid, fwarps_used * 32, fsm, st>>>(fa);
  GC_CUDA(cudaGetLastError());
  return GC_OK;
}

// ---------------------------------------------------------------------------
// Batches of orbits and the autotuner
// ---------------------------------------------------------------------------
namespace {

constexpr int kPoolStreams = 16;
std::mutex g_pool_mu;
cudaStream_t g_pool[kStaticMaxDevices][kPoolStreams] = {};

int pool_streams(cudaStream_t** out) {
  int dev = 0;
  GC_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kStaticMaxDevices) return fail(GC_EINVAL, "device %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_pool_mu);
  if (!g_pool[dev][0])
    for (int i = 0; i < kPoolStreams; ++i)
      GC_CUDA(cudaStreamCreateWithFlags(&g_pool[dev][i], cudaStreamNonBlocking));
  *out = g_pool[dev];
  return GC_OK;
}

// Reserve every orbit's copy pool for its pending starts (one read-back per
// orbit), so that the enqueue itself needs no host synchronisation.
int reserve_for(gc_orbit o, uint64_t n, cudaStream_t s) {
  const unsigned long long need = o->enqueued + n;
  if (need <= o->cap) return GC_OK;
  unsigned cur = 0;
  GC_CUDA(cudaMemcpyAsync(&cur, o->n_entries(), 4, cudaMemcpyDeviceToHost, s));
  GC_CUDA(cudaStreamSynchronize(s));
  return table_reserve(o, need, cur, s);
}

// Pilot runs on a throw-away copy of the orbit: four launch shapes per kernel,
// the fastest kept per kernel (result-neutral knobs).  In mode 2 (mixed
// precision) the sweep-unroll depth -- sweeps between residual checks, 2, 4
// or 8 -- is then picked by the whole path's pilot time; it changes where a
// start's FP32 phase stops, so results move within the convergence tolerance.
int autotune_shape(gc_orbit like, const gc_options& base, double omega, double eps, Tuning* out) {
  std::vector<double> phi((size_t)like->V * like->d);
  {
    std::vector<double2> u((size_t)like->V * like->d);
    GC_CUDA(read_back(u.data(), like->links64.p, u.size() * sizeof(double2), like->last_stream));
    for (size_t i = 0; i < u.size(); ++i) phi[i] = std::atan2(u[i].y, u[i].x);
  }
  gc_orbit tmp = nullptr;
  if (int rc = gc_create_orbit(like->d, like->L, phi.data(), 0xA070u, 0, &tmp)) return rc;
  gc_options opt = base;
  opt.keep_per_start = 0;
  opt.async = 0;
  opt.use_graph = 0;
  opt.stream = nullptr;
  // pilots long enough to time throughput, not one start's tail: about 2^25
  // site-starts (2^17 starts of a 4^4 lattice)
  const uint64_t pilot = std::min<uint64_t>(1u << 17, std::max<uint64_t>(8192, (1ull << 25) / (uint64_t)like->V));
  // caps on warps per CTA; 16 leaves the largest shape that fits
  const int cand[4][3] = {{2, 2, 1}, {4, 4, 2}, {8, 8, 4}, {8, 16, 4}};
  double best[3] = {1e300, 1e300, 1e300};
  Tuning t;
  int rc = GC_OK;
  for (int c = 0; c < 4 && rc == GC_OK; ++c) {
    Tuning cand_t;
    cand_t.r_warps = cand[c][0];
    cand_t.p_warps = cand[c][1];
    cand_t.f_warps = cand[c][2];
    const double m0[4] = {tmp->ms[0], tmp->ms[1], tmp->ms[2], tmp->ms[3]};
    rc = enumerate_impl(tmp, pilot, omega, eps, opt, nullptr, false, true, cand_t);
    if (rc == GC_OK && cudaStreamSynchronize(nullptr) != cudaSuccess) rc = fail(GC_ECUDA, "autotune pilot failed");
    if (rc != GC_OK) break;
    harvest_timing(tmp);
    const double dt[3] = {tmp->ms[0] - m0[0], tmp->ms[1] - m0[1], tmp->ms[3] - m0[3]};
    if (dt[0] < best[0]) { best[0] = dt[0]; t.r_warps = cand_t.r_warps; }
    if (dt[1] < best[1]) { best[1] = dt[1]; t.p_warps = cand_t.p_warps; }
    if (dt[2] < best[2]) { best[2] = dt[2]; t.f_warps = cand_t.f_warps; }
  }
  const bool deep = base.autotune == 2 && base.precision == GC_MIXED;
  if (rc == GC_OK && deep) {
    // the depth moves the FP32 sweeps and the polish; the redo launch is a
    // few starts' latency tail that batches hide, so it is left out, and each
    // depth is timed twice (the faster counts) on pilots twice as long
    double best_all = 1e300;
    for (int ce : {2, 4, 8}) {
      gc_options o2 = opt;
      o2.check_every = ce;
      o2.autotune = 0;
      double dt_min = 1e300;
      for (int rep = 0; rep < 2 && rc == GC_OK; ++rep) {
        const double m0 = tmp->ms[0] + tmp->ms[1] - tmp->ms[4];
        rc = enumerate_impl(tmp, 2 * pilot, omega, eps, o2, nullptr, false, true, t);
        if (rc == GC_OK && cudaStreamSynchronize(nullptr) != cudaSuccess) rc = fail(GC_ECUDA, "autotune pilot failed");
        if (rc != GC_OK) break;
        harvest_timing(tmp);
        dt_min = std::min(dt_min, tmp->ms[0] + tmp->ms[1] - tmp->ms[4] - m0);
      }
      if (rc != GC_OK) break;
      if (dt_min < best_all) { best_all = dt_min; t.check_every = ce; }
    }
  }
  gc_destroy_orbit(tmp);
  if (rc != GC_OK) return rc;
  *out = t;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache.emplace_back(tune_key(like->d, like->L, base.precision, deep), t);
  return GC_OK;
}

bool have_tuning(int d, int L, int precision, bool deep) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (auto& kv : g_tune_cache)
    if (kv.first == tune_key(d, L, precision, deep)) return true;
  return false;
}

bool deep_tuning(const gc_options& opt) { return opt.autotune == 2 && opt.precision == GC_MIXED; }

}  // namespace

extern "C" int gc_enumerate_batch(gc_orbit* orbits, int n_orbits, const uint64_t* n_starts, double omega,
                                  double eps, const gc_options* opt_in) {
  if (!orbits || !n_starts || n_orbits < 1) return fail(GC_EINVAL, "gc_enumerate_batch: empty or NULL batch");
  gc_options opt;
  if (opt_in) opt = *opt_in; else gc_options_default(&opt);
  if (int rc = validate_options(opt, omega, eps)) return rc;
  if (opt.keep_per_start) return fail(GC_EINVAL, "keep_per_start is not available for batches");
  for (int i = 0; i < n_orbits; ++i) {
    if (!orbits[i]) return fail(GC_EINVAL, "orbit %d is NULL", i);
    for (int j = 0; j < i; ++j)
      if (orbits[j] == orbits[i]) return fail(GC_EINVAL, "orbit %d appears twice in the batch", i);
  }
  cudaStream_t origin = (cudaStream_t)opt.stream;
  cudaStream_t* pool = nullptr;
  if (int rc = pool_streams(&pool)) return rc;
  // set-up that needs the host: tuning, copy pools, staging buffers
  for (int i = 0; i < n_orbits; ++i) {
    gc_orbit o = orbits[i];
    if (opt.autotune && !o->slab && !have_tuning(o->d, o->L, opt.precision, deep_tuning(opt))) {
      Tuning t;
      if (int rc = autotune_shape(o, opt, omega, eps, &t)) return rc;
    }
    if (int rc = reserve_for(o, n_starts[i], origin)) return rc;
    if (int rc = enumerate_impl(o, n_starts[i], omega, eps, opt, origin, true, false,
                                cached_tuning(o->d, o->L, opt.precision, deep_tuning(opt)), true))
      return rc;
  }
  GC_CUDA(cudaStreamSynchronize(origin));
  // fork onto the pool, one stream per orbit (round robin), join back on origin
  cudaEvent_t fork, join[kPoolStreams];
  GC_CUDA(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
  for (auto& e : join) GC_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  const int used = std::min(n_orbits, kPoolStreams);
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int rc = GC_OK;
  if (opt.use_graph) {
    const cudaError_t e = cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) rc = fail(GC_ECUDA, "cudaStreamBeginCapture: %s (use a non-default stream)", cudaGetErrorString(e));
  }
  if (rc == GC_OK && cudaEventRecord(fork, origin) != cudaSuccess) rc = fail(GC_ECUDA, "fork record failed");
  for (int k = 0; rc == GC_OK && k < used; ++k)
    if (cudaStreamWaitEvent(pool[k], fork, 0) != cudaSuccess) rc = fail(GC_ECUDA, "fork wait failed");
  for (int i = 0; rc == GC_OK && i < n_orbits; ++i)
    rc = enumerate_impl(orbits[i], n_starts[i], omega, eps, opt, pool[i % kPoolStreams], true, true,
                        cached_tuning(orbits[i]->d, orbits[i]->L, opt.precision, deep_tuning(opt)));
  for (int k = 0; k < used; ++k) {
    if (cudaEventRecord(join[k], pool[k]) != cudaSuccess && rc == GC_OK) rc = fail(GC_ECUDA, "join record failed");
    if (cudaStreamWaitEvent(origin, join[k], 0) != cudaSuccess && rc == GC_OK) rc = fail(GC_ECUDA, "join wait failed");
  }
  // later calls on these orbits (fetch, stats, more starts) follow the join on
  // the caller's stream, not the shared pool streams, where another batch's
  // work may already be queued behind this one
  for (int i = 0; i < n_orbits; ++i) orbits[i]->last_stream = origin;
  if (opt.use_graph) {
    const cudaError_t e = cudaStreamEndCapture(origin, &graph);
    if (rc != GC_OK) cudaGetLastError();   // a failed capture's error is not left for the next call
    if (rc == GC_OK && e != cudaSuccess) rc = fail(GC_ECUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e));
    if (rc == GC_OK && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) rc = fail(GC_ECUDA, "cudaGraphInstantiate failed");
    if (rc == GC_OK && cudaGraphLaunch(exec, origin) != cudaSuccess) rc = fail(GC_ECUDA, "cudaGraphLaunch failed");
  }
  const bool wait = !opt.async || opt.use_graph;
  if (wait && cudaStreamSynchronize(origin) != cudaSuccess && rc == GC_OK)
    rc = fail(GC_ECUDA, "batch: %s", cudaGetErrorString(cudaGetLastError()));
  if (exec) cudaGraphExecDestroy(exec);
  if (graph) cudaGraphDestroy(graph);
  cudaEventDestroy(fork);
  for (auto& e : join) cudaEventDestroy(e);
  if (rc != GC_OK || !wait) return rc;
  for (int i = 0; i < n_orbits; ++i) {
    harvest_timing(orbits[i]);
    if (int r = check_errors(orbits[i])) return r;
  }
  return GC_OK;
}

extern "C" int gc_autotune_ex(gc_orbit o, int precision, int mode, int* r_warps, int* p_warps,
                              int* f_warps, int* check_every) {
  if (!o) return fail(GC_EINVAL, "gc_autotune: NULL orbit");
  if (precision != GC_FP64 && precision != GC_MIXED) return fail(GC_EINVAL, "unknown precision %d", precision);
  if (mode != 1 && mode != 2) return fail(GC_EINVAL, "autotune mode %d not 1 or 2", mode);
  gc_options opt;
  gc_options_default(&opt);
  opt.precision = precision;
  opt.check_every = precision == GC_MIXED ? 4 : 1;
  opt.autotune = mode;
  const bool deep = deep_tuning(opt);
  Tuning t;
  if (o->slab) t = Tuning{};   // the hyperplane path has no launch shapes to tune
  else if (have_tuning(o->d, o->L, precision, deep)) t = cached_tuning(o->d, o->L, precision, deep);
  else if (int rc = autotune_shape(o, opt, 1.7, 1e-24, &t)) return rc;
  if (r_warps) *r_warps = t.r_warps;
  if (p_warps) *p_warps = t.p_warps;
  if (f_warps) *f_warps = t.f_warps;
  if (check_every) *check_every = deep ? t.check_every : 0;
  return GC_OK;
}

extern "C" int gc_autotune(gc_orbit o, int precision, int* r_warps, int* p_warps, int* f_warps) {
  return gc_autotune_ex(o, precision, 1, r_warps, p_warps, f_warps, nullptr);
}

// ---------------------------------------------------------------------------
// Serving: continuous batching of enumeration requests
// ---------------------------------------------------------------------------
// Requests (an orbit and a start count) go through a mailbox to the
// device-resident request loop (gc_serve.cuh), which admits them in arrival
// order as soon as a region of the server's device arena fits their memory
// estimate.  Worker threads, each with its own stream, run the admitted
// requests with every device allocation carved from the request's region, so
// requests that arrive while others run start as memory frees up and their
// kernels overlap on the GPU.  When a request is done its results (the copy
// table and the links) move out of the arena and the region is mailed back;
// its result is the orbit itself, handed to the caller.  Results do not depend
// on the mix: a request touches only its own orbit object, and every kernel's
// per-start arithmetic and the dedup outcome are independent of what else runs.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <thread>
#include <atomic>
#include <set>

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t ticket = 0;
  int dim = 0, L = 0;
  std::vector<double> phi;
  uint64_t orbit_id = 0, n = 0;
  double omega = 1.7, eps = 1e-24;
  size_t bytes = 0;            // device memory estimate (the admitted region's size)
  size_t offset = 0;           // the admitted region's offset in the arena
  Clock::time_point submitted, admitted, finished;
  int status = GC_OK;
  std::string message;
  bool done = false;
  gc_orbit orbit = nullptr;
};

// Device bytes a request holds while it runs, as the library allocates them:
// the links (FP64 and FP32), a copy pool reserved for n copies (every start
// may find a new one; the worker creates the orbit with max_copies = n so the
// pool never grows), its buckets and the paper-style F set (table_reserve's
// sizes), locks and counters, and one staging batch; beyond shared memory (the
// hyperplane path, the same test as gc_create_orbit's) also the per-SM
// scratch of the Newton polish and of the first-region test.  The dense
// first-region test adds its basis slots (at most 1 GiB).
size_t request_bytes(int dim, int L, uint64_t n, int precision, int fp_mode) {
  const double V = std::pow((double)L, dim);
  const double cap = (double)std::max<uint64_t>(n, 1024);
  const double pool = cap * (V * 16 + 8 + 8 + 4 + 8 + 8 + 4 + 8 + 4 + 8) +
                      (double)next_pow2(2ull * (uint64_t)cap) * 4 + (double)next_pow2(4ull * (uint64_t)cap) * 16;
  const double per_start = V * 16 + (precision == GC_MIXED ? V * 8 : 0) + 48;
  double batch = std::min((double)n, std::max(4096.0, (double)(1ull << 30) / per_start));
  double extra = fp_mode == GC_FP_DENSE ? (double)(1ull << 30) : 0.0;
  const int Vi = (int)V;
  if (V <= gc::kMaxSlabSites &&
      (Vi > gc::kMaxSites || gc::Smem(Vi, dim, 16, (size_t)Vi * 16, 1).total > max_smem_optin())) {
    batch = std::min((double)n, std::max(2.0 * sm_count(), (double)(1ull << 30) / per_start));
    const int Ps = (Vi / L + 3) / 4 * 4;
    const double newton = precision == GC_MIXED ? (double)gc::slab_newton_scratch_floats(dim, Vi, L, Ps) * 4 : 0.0;
    const double fp = (double)gc::slab_fp_scratch_bytes<double>(dim, Vi);
    extra = sm_count() * std::max(newton, fp) + batch * 8 + batch * 4;
  }
  const double b = V * dim * 24 + pool + batch * per_start + extra + (1u << 16) * 4 + (4 << 20);
  return ((size_t)b + 4095) & ~size_t(4095);
}

// Move an orbit's long-lived buffers out of a server arena (after its request
// ran there) into memory of the allocator hooks, and drop its staging, so the
// region can go back while the caller keeps the orbit.  The copy table moves
// at the size it uses (table_reserve with exact capacity: entries copied,
// buckets re-threaded, the F set rehashed).
int rehome_orbit(gc_orbit o, cudaStream_t s) {
  GC_CUDA(cudaStreamSynchronize(s));
  if (o->t_cfg.p && in_arena(o->t_cfg.p)) {
    unsigned cur = 0;
    GC_CUDA(read_back(&cur, o->n_entries(), 4, s));
    cur = std::min(cur, o->cap);
    if (int rc = table_reserve(o, cur, cur, s, true)) return rc;
  }
  for (Buf* b : {&o->links64, &o->links32, &o->t_cfg, &o->t_F, &o->t_q, &o->t_t, &o->t_first, &o->t_rep, &o->t_count,
                 &o->t_next, &o->t_lam, &o->t_region, &o->t_head, &o->t_lock, &o->t_f8, &o->t_f8n,
                 &o->t_counters, &o->t_newlist, &o->work, &o->stats}) {
    if (!b->p || !in_arena(b->p)) continue;
    Buf nb;
    if (!nb.ensure(b->n, s)) return fail(GC_ENOMEM, "cannot move a served orbit's results (%zu bytes)", b->n);
    GC_CUDA(cudaMemcpyAsync(nb.p, b->p, b->n, cudaMemcpyDeviceToDevice, s));
    *b = nb;
  }
  for (Buf* b : {&o->s_status, &o->s_sweeps, &o->s_resid, &o->s_F, &o->s_fprint, &o->s_config, &o->s_state32,
                 &o->s_copy, &o->s_redo, &o->s_rate, &o->scratch, &o->theta_tmp, &o->sort_keys, &o->sort_idx,
                 &o->sort_tmp, &o->f8_tmp})
    b->release(s);
  GC_CUDA(cudaStreamSynchronize(s));
  return GC_OK;
}

}  // namespace

// Serving: the host side of the device-resident request loop (gc_serve.cuh).
//   submit  -> mailbox (pinned) -> serve_loop_kernel admits by the device-side
//   budget -> completion ring (pinned) -> dispatcher thread -> a worker runs
//   the request in its admitted region -> results moved out -> region mailed
//   back.
struct gc_server_s {
  gc_options opt{};
  size_t budget = 0;
  int device = 0;
  char* arena = nullptr;
  gc::ServeHostShared* H = nullptr;   // host view of the pinned block
  gc::ServeHostShared* Hd = nullptr;  // its device address
  gc::ServeDevState* D = nullptr;     // device memory
  cudaStream_t loop_stream = nullptr, ctl_stream = nullptr;
  long long idle_limit = 10000;       // polls; with 20 us sleeps about 0.2 s idle
  unsigned sleep_ns = 20000;
  uint64_t loop_launches = 0;
  std::mutex mu;                      // requests, tickets, mailbox writes
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Request>> ready;          // admitted, waiting for a worker
  std::map<uint64_t, std::shared_ptr<Request>> all;
  uint64_t next_ticket = 1;
  bool stopping = false, dispatcher_stop = false;
  std::vector<std::thread> workers;
  std::thread dispatcher;
  std::vector<cudaStream_t> streams;
  std::set<gc_orbit> live;            // finished orbits whose results hold a region

  static volatile int* vstatus(gc::ServeHostShared* h) { return reinterpret_cast<volatile int*>(&h->loop_status); }

  int launch_loop() {
    *vstatus(H) = gc::kLoopRunning;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    gc::serve_loop_kernel<<<1, 32, 0, loop_stream>>>(Hd, D, idle_limit, sleep_ns);
    ++loop_launches;
    GC_CUDA(cudaGetLastError());
    return GC_OK;
  }

  // Write one mailbox entry (caller holds mu) and make sure a loop will read it.
  int mail(unsigned op, uint64_t ticket, uint64_t bytes) {
    volatile unsigned long long* head = &H->mail_head;
    volatile unsigned long long* tail = &H->mail_tail;
    for (long long spins = 0; *head - *tail >= gc::kMailSlots; ++spins) {   // ring full (bounded)
      if (spins > 2000000) return fail(GC_ETIMEDOUT, "serving mailbox full");
      std::this_thread::sleep_for(std::chrono::microseconds(5));
    }
    const unsigned long long h = *head;
    volatile gc::MailEntry* e = &H->mail[h % gc::kMailSlots];
    e->ticket = ticket;
    e->bytes = bytes;
    e->op = op;
    std::atomic_thread_fence(std::memory_order_release);
    *head = h + 1;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    // the loop reads this mail unless it had already decided to end; then
    // start it again (kLoopExiting resolves within one poll)
    int st = *vstatus(H);
    for (long long spins = 0; st == gc::kLoopExiting && spins < 2000000; ++spins) {
      std::this_thread::sleep_for(std::chrono::microseconds(1));
      st = *vstatus(H);
    }
    if (st == gc::kLoopStopped || st == gc::kLoopTimedOut || st == gc::kLoopExiting) return launch_loop();
    return GC_OK;
  }

  void dispatch() {
    cudaSetDevice(device);
    volatile unsigned long long* dhead = &H->done_head;
    volatile unsigned long long* dtail = &H->done_tail;
    for (;;) {
      {
        std::lock_guard<std::mutex> lk(mu);
        if (dispatcher_stop) return;
      }
      const unsigned long long dh = *dhead;
      std::atomic_thread_fence(std::memory_order_acquire);
      unsigned long long t = *dtail;
      if (t == dh) {
        std::this_thread::sleep_for(std::chrono::microseconds(50));
        continue;
      }
      for (; t < dh; ++t) {
        volatile gc::DoneEntry* e = &H->done[t % gc::kMailSlots];
        const uint64_t ticket = e->ticket, off = e->offset;
        std::lock_guard<std::mutex> lk(mu);
        auto it = all.find(ticket);
        if (it != all.end()) {
          it->second->offset = off;
          it->second->admitted = Clock::now();
          ready.push_back(it->second);
        }
      }
      std::atomic_thread_fence(std::memory_order_release);
      *dtail = dh;
      cv_work.notify_all();
    }
  }

  void worker(int k) {
    cudaSetDevice(device);
    for (;;) {
      std::shared_ptr<Request> r;
      {
        std::unique_lock<std::mutex> lk(mu);
        cv_work.wait(lk, [&] { return stopping || !ready.empty(); });
        if (ready.empty()) {
          if (stopping) return;
          continue;
        }
        r = ready.front();
        ready.pop_front();
      }
      gc_options o = opt;
      o.stream = streams[k];
      o.keep_per_start = 0;
      ArenaScope scope;
      scope.base = arena + r->offset;
      scope.size = r->bytes;
      t_scope = &scope;
      gc_orbit orb = nullptr;
      int rc = gc_create_orbit(r->dim, r->L, r->phi.data(), r->orbit_id, r->n, &orb);
      if (rc == GC_OK) rc = gc_enumerate_copies(orb, r->n, r->omega, r->eps, &o);
      t_scope = nullptr;
      std::string msg = rc == GC_OK ? "" : gc_last_error();
      cudaStreamSynchronize(streams[k]);
      if (rc != GC_OK && orb) {
        gc_destroy_orbit(orb);
        orb = nullptr;
      }
      if (orb) {
        // the staging goes (later allocations of the orbit, e.g. a fetch's,
        // come from the allocator hooks); the results stay in the region
        for (Buf* b : {&orb->s_status, &orb->s_sweeps, &orb->s_resid, &orb->s_F, &orb->s_fprint, &orb->s_config,
                       &orb->s_state32, &orb->s_copy, &orb->s_redo, &orb->s_rate, &orb->scratch, &orb->theta_tmp})
          b->release(streams[k]);
      }
      {
        std::lock_guard<std::mutex> lk(mu);
        r->status = rc;
        r->message = msg;
        r->orbit = orb;
        r->finished = Clock::now();
        r->done = true;
        if (orb) {
          orb->served_by = this;
          orb->region_off = r->offset;
          live.insert(orb);
        } else {
          mail(gc::kMailFree, r->ticket, r->offset);
        }
      }
      cv_done.notify_all();
    }
  }
};

std::mutex g_srv_mu;                  // live servers (a served orbit may outlive its server's handle use)
std::set<gc_server_s*> g_servers;

void server_release_region(gc_orbit o) {
  std::lock_guard<std::mutex> g(g_srv_mu);
  gc_server_s* s = o->served_by;
  o->served_by = nullptr;
  if (!s || !g_servers.count(s)) return;
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->live.erase(o)) s->mail(gc::kMailFree, 0, o->region_off);
}

extern "C" int gc_server_create(int workers, size_t mem_budget_bytes, const gc_options* opt, gc_server* out) {
  if (!out) return fail(GC_EINVAL, "gc_server_create: out is NULL");
  *out = nullptr;
  if (workers < 1 || workers > 64) return fail(GC_EINVAL, "workers = %d not in 1..64", workers);
  gc_server s = new (std::nothrow) gc_server_s;
  if (!s) return fail(GC_ENOMEM, "host allocation failed");
  if (opt) s->opt = *opt; else gc_options_default(&s->opt);
  if (int rc = validate_options(s->opt, 1.0, 1.0)) { delete s; return rc; }
  if (cudaGetDevice(&s->device) != cudaSuccess) { delete s; return fail(GC_ECUDA, "no CUDA device"); }
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  // default: half the device, at most 16 GiB, halved until the allocator
  // gives it (free memory is not a guide when a caching allocator holds it)
  s->budget = mem_budget_bytes ? mem_budget_bytes : total_b / 2;
  s->budget &= ~size_t(4095);
  auto undo = [&](int rc) {
    if (s->loop_stream) cudaStreamDestroy(s->loop_stream);
    if (s->ctl_stream) cudaStreamDestroy(s->ctl_stream);
    if (s->H) cudaFreeHost(s->H);
    if (s->D) cudaFree(s->D);
    if (s->arena) {
      {
        std::lock_guard<std::mutex> lk(g_arena_mu);
        for (size_t i = 0; i < g_arenas.size(); ++i)
          if (g_arenas[i].first == s->arena) { g_arenas.erase(g_arenas.begin() + i); break; }
      }
      dev_free(s->arena, nullptr);
    }
    delete s;
    return rc;
  };
  if (cudaStreamCreateWithFlags(&s->loop_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->ctl_stream, cudaStreamNonBlocking) != cudaSuccess)
    return undo(fail(GC_ECUDA, "cudaStreamCreate failed"));
  s->arena = static_cast<char*>(dev_alloc(s->budget, s->ctl_stream));
  while (!s->arena && !mem_budget_bytes && s->budget > (256ull << 20)) {
    s->budget = (s->budget / 2) & ~size_t(4095);
    s->arena = static_cast<char*>(dev_alloc(s->budget, s->ctl_stream));
  }
  if (!s->arena) return undo(fail(GC_ENOMEM, "cannot allocate the serving arena (%.1f MiB)", s->budget / 1048576.0));
  if (cudaHostAlloc((void**)&s->H, sizeof(gc::ServeHostShared), cudaHostAllocMapped) != cudaSuccess) {
    s->H = nullptr;
    return undo(fail(GC_ENOMEM, "cannot allocate the pinned mailbox"));
  }
  std::memset((void*)s->H, 0, sizeof(gc::ServeHostShared));
  s->H->loop_status = gc::kLoopStopped;
  if (cudaHostGetDevicePointer((void**)&s->Hd, s->H, 0) != cudaSuccess)
    return undo(fail(GC_ECUDA, "the mailbox is not mapped into the device"));
  if (cudaMalloc((void**)&s->D, sizeof(gc::ServeDevState)) != cudaSuccess) {
    s->D = nullptr;
    return undo(fail(GC_ENOMEM, "cannot allocate the serving state"));
  }
  gc::serve_init_kernel<<<1, 32, 0, s->ctl_stream>>>(s->D, (unsigned long long)s->budget);
  if (cudaStreamSynchronize(s->ctl_stream) != cudaSuccess) return undo(fail(GC_ECUDA, "serve_init_kernel failed"));
  {
    std::lock_guard<std::mutex> lk(g_arena_mu);
    g_arenas.emplace_back(s->arena, s->budget);
  }
  s->streams.resize(workers);
  for (int k = 0; k < workers; ++k)
    if (cudaStreamCreateWithFlags(&s->streams[k], cudaStreamNonBlocking) != cudaSuccess) {
      for (int j = 0; j < k; ++j) cudaStreamDestroy(s->streams[j]);
      return undo(fail(GC_ECUDA, "cudaStreamCreate failed"));
    }
  if (int rc = s->launch_loop()) {
    for (auto st : s->streams) cudaStreamDestroy(st);
    return undo(rc);
  }
  s->dispatcher = std::thread(&gc_server_s::dispatch, s);
  for (int k = 0; k < workers; ++k) s->workers.emplace_back(&gc_server_s::worker, s, k);
  {
    std::lock_guard<std::mutex> g(g_srv_mu);
    g_servers.insert(s);
  }
  *out = s;
  return GC_OK;
}

extern "C" int gc_server_submit(gc_server s, int dim, int L, const double* link_angles, uint64_t orbit_id,
                                uint64_t n_starts, double omega, double eps, uint64_t* ticket) {
  if (!s || !link_angles || !ticket) return fail(GC_EINVAL, "gc_server_submit: NULL argument");
  if (dim < 1 || dim > gc::kMaxDim || L < 2) return fail(GC_EINVAL, "bad lattice %d^%d", L, dim);
  if (!(omega > 0.0 && omega < 2.0) || !(eps > 0.0)) return fail(GC_EINVAL, "bad omega or eps");
  const double Vd = std::pow((double)L, dim);
  if (Vd > gc::kMaxSlabSites) return fail(GC_EINVAL, "lattice of %.0f sites exceeds %d", Vd, gc::kMaxSlabSites);
  auto r = std::make_shared<Request>();
  r->dim = dim; r->L = L; r->orbit_id = orbit_id; r->n = n_starts; r->omega = omega; r->eps = eps;
  r->phi.assign(link_angles, link_angles + (size_t)Vd * dim);
  r->bytes = request_bytes(dim, L, n_starts, s->opt.precision, s->opt.fp_mode);
  if (r->bytes > s->budget)
    return fail(GC_ENOMEM, "request needs ~%.1f MiB, above the %.1f MiB budget", r->bytes / 1048576.0,
                s->budget / 1048576.0);
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stopping) return fail(GC_ESTATE, "server is shutting down");
  r->ticket = s->next_ticket++;
  r->submitted = Clock::now();
  s->all[r->ticket] = r;
  *ticket = r->ticket;
  if (int rc = s->mail(gc::kMailAdmit, r->ticket, r->bytes)) {
    s->all.erase(r->ticket);
    return rc;
  }
  return GC_OK;
}

extern "C" int gc_server_wait(gc_server s, uint64_t ticket, double timeout_s, int* status, double* latency_s,
                              gc_orbit* orbit) {
  if (!s) return fail(GC_EINVAL, "gc_server_wait: NULL server");
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(ticket);
  if (it == s->all.end()) return fail(GC_EINVAL, "unknown or already collected ticket %llu", (unsigned long long)ticket);
  std::shared_ptr<Request> r = it->second;
  const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                           std::chrono::duration<double>(timeout_s < 0 ? 1e9 : timeout_s));
  if (!s->cv_done.wait_until(lk, deadline, [&] { return r->done; }))
    return fail(GC_ETIMEDOUT, "request %llu not finished within %g s", (unsigned long long)ticket, timeout_s);
  if (status) *status = r->status;
  if (latency_s) *latency_s = std::chrono::duration<double>(r->finished - r->submitted).count();
  gc_orbit drop = nullptr;
  if (orbit) *orbit = r->orbit;
  else drop = r->orbit;
  r->orbit = nullptr;
  s->all.erase(it);
  if (r->status != GC_OK) g_err = r->message;
  lk.unlock();
  if (drop) gc_destroy_orbit(drop);   // mails its region back
  return GC_OK;
}

extern "C" int gc_server_state(gc_server s, gc_server_info* out) {
  if (!s || !out) return fail(GC_EINVAL, "gc_server_state: NULL argument");
  std::memset(out, 0, sizeof *out);
  gc::ServeDevState snap;
  // the loop may be running: the copy is a snapshot
  GC_CUDA(cudaMemcpyAsync(&snap, s->D, sizeof snap, cudaMemcpyDeviceToHost, s->ctl_stream));
  GC_CUDA(cudaStreamSynchronize(s->ctl_stream));
  const int st = *gc_server_s::vstatus(s->H);
  out->loop_status = st == gc::kLoopTimedOut ? GC_ETIMEDOUT : GC_OK;
  out->loop_running = (st == gc::kLoopRunning || st == gc::kLoopExiting) ? 1 : 0;
  out->loop_launches = s->loop_launches;
  out->admitted = snap.admitted;
  out->released = snap.freed;
  out->waiting = snap.wait_tail - snap.wait_head;
  out->bytes_in_use = snap.in_use;
  out->budget_bytes = s->budget;
  out->regions = snap.n_regions;
  return GC_OK;
}

extern "C" int gc_server_destroy(gc_server s) {
  if (!s) return fail(GC_EINVAL, "gc_server_destroy: NULL server");
  // finish every submitted request (they are admitted as regions free up)
  {
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_done.wait(lk, [&] {
      for (auto& kv : s->all)
        if (!kv.second->done) return false;
      return true;
    });
    s->stopping = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  // orbits nobody collected are destroyed; collected orbits still alive move
  // their results out of the arena (the caller keeps them)
  std::vector<gc_orbit> uncollected;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto& kv : s->all)
      if (kv.second->orbit) uncollected.push_back(kv.second->orbit);
    s->all.clear();
  }
  for (gc_orbit o : uncollected) gc_destroy_orbit(o);
  {
    std::lock_guard<std::mutex> g(g_srv_mu);
    std::lock_guard<std::mutex> lk(s->mu);
    for (gc_orbit o : s->live) {
      rehome_orbit(o, s->ctl_stream);
      o->served_by = nullptr;
    }
    s->live.clear();
    g_servers.erase(s);
    s->mail(gc::kMailStop, 0, 0);
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->dispatcher_stop = true;
  }
  s->dispatcher.join();
  cudaStreamSynchronize(s->loop_stream);     // the loop ends on the stop mail (bounded by its idle limit)
  for (auto st : s->streams) cudaStreamDestroy(st);
  cudaStreamDestroy(s->loop_stream);
  cudaStreamDestroy(s->ctl_stream);
  cudaFreeHost(s->H);
  cudaFree(s->D);
  {
    std::lock_guard<std::mutex> lk(g_arena_mu);
    for (size_t i = 0; i < g_arenas.size(); ++i)
      if (g_arenas[i].first == s->arena) { g_arenas.erase(g_arenas.begin() + i); break; }
  }
  dev_free(s->arena, nullptr);
  delete s;
  return GC_OK;
}

// ---------------------------------------------------------------------------
// Throughput probes of the arithmetic units (roofline denominators)
// ---------------------------------------------------------------------------
#include "gc_peaks.cuh"

extern "C" int gc_peak_probe(int kind, void* stream, double* ops_per_s) {
  if (!ops_per_s) return fail(GC_EINVAL, "gc_peak_probe: NULL ops_per_s");
  if (kind < GC_PEAK_FFMA || kind > GC_PEAK_DFMA_LANE1) return fail(GC_EINVAL, "gc_peak_probe: unknown kind %d", kind);
  cudaStream_t s = (cudaStream_t)stream;
  // four 256-thread CTAs per SM; iterations sized for ~10-40 ms per launch
  const int threads = 256, grid = 4 * sm_count();
  const int iters = (kind == GC_PEAK_DFMA || kind == GC_PEAK_DFMA_LANE1) ? 1 << 12 : (kind == GC_PEAK_RSQ ? 1 << 15 : 1 << 17);
  // lane operations per thread (one-lane DFMA: per warp instruction, i.e. per 32 threads)
  const double per_thread = 8.0 * iters * (kind == GC_PEAK_FFMA2 ? 2.0 : 1.0) / (kind == GC_PEAK_DFMA_LANE1 ? 32.0 : 1.0);
  Buf out;
  if (!out.ensure((size_t)grid * threads * sizeof(float), s)) return fail(GC_ENOMEM, "gc_peak_probe: no scratch");
  cudaEvent_t e0, e1;
  GC_CUDA(cudaEventCreate(&e0));
  GC_CUDA(cudaEventCreate(&e1));
  const float m = 1.0f - 0x1.0p-20f, c = 0x1.0p-21f;
  auto launch = [&]() {
    switch (kind) {
      case GC_PEAK_FFMA: gc::peak_probe_kernel<gc::kPeakFFMA><<<grid, threads, 0, s>>>(out.as<float>(), iters, m, c); break;
      case GC_PEAK_FFMA2: gc::peak_probe_kernel<gc::kPeakFFMA2><<<grid, threads, 0, s>>>(out.as<float>(), iters, m, c); break;
      case GC_PEAK_DFMA: gc::peak_probe_kernel<gc::kPeakDFMA><<<grid, threads, 0, s>>>(out.as<float>(), iters, m, c); break;
      case GC_PEAK_DFMA_LANE1: gc::peak_probe_kernel<gc::kPeakDFMA1><<<grid, threads, 0, s>>>(out.as<float>(), iters, m, c); break;
      default: gc::peak_probe_kernel<gc::kPeakRSQ><<<grid, threads, 0, s>>>(out.as<float>(), iters, m, c); break;
    }
  };
  float best = 0.f;
  int rc = GC_OK;
  for (int rep = 0; rep < 4 && rc == GC_OK; ++rep) {   // the first launch is a warm-up
    if (cudaEventRecord(e0, s) != cudaSuccess) rc = fail(GC_ECUDA, "gc_peak_probe: event record");
    launch();
    if (rc == GC_OK && cudaGetLastError() != cudaSuccess) rc = fail(GC_ECUDA, "gc_peak_probe: launch failed");
    if (rc == GC_OK && cudaEventRecord(e1, s) != cudaSuccess) rc = fail(GC_ECUDA, "gc_peak_probe: event record");
    if (rc == GC_OK && cudaEventSynchronize(e1) != cudaSuccess) rc = fail(GC_ECUDA, "gc_peak_probe: kernel failed");
    float ms = 0.f;
    if (rc == GC_OK) cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms > 0.f && (best == 0.f || ms < best)) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  out.release(s);
  if (rc != GC_OK) return rc;
  *ops_per_s = (double)grid * threads * per_thread / (best * 1e-3);
  return GC_OK;
}

// ---------------------------------------------------------------------------
// Test hook for the bounded lock wait of the dedup table
// ---------------------------------------------------------------------------
extern "C" int gc_test_dedup_locks(gc_orbit o, int hold, long long spin_budget) {
  if (!o) return fail(GC_EINVAL, "gc_test_dedup_locks: NULL orbit");
  if (spin_budget < 0) return fail(GC_EINVAL, "gc_test_dedup_locks: spin_budget %lld < 0", spin_budget);
  if (!o->t_lock.p || o->nl == 0) return fail(GC_ESTATE, "gc_test_dedup_locks: the orbit has no table yet");
  cudaStream_t s = o->last_stream;
  GC_CUDA(cudaStreamSynchronize(s));
  fill_i32(o->t_lock.as<int>(), hold ? 1 : 0, o->nl, s);
  GC_CUDA(cudaGetLastError());
  GC_CUDA(cudaStreamSynchronize(s));
  o->lock_spins = spin_budget > 0 ? spin_budget : gc::kLockSpins;
  return GC_OK;
}
