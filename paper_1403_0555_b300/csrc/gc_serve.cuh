// Device-resident request loop of the serving layer: admission of enumeration
// requests by a device-side memory budget (the paper has no serving layer).
//
// The host writes requests into a mailbox in pinned, device-mapped memory;
// one warp on the GPU runs serve_loop_kernel, which reads the mailbox, keeps
// the FIFO of waiting requests and the region table of the server's device
// arena in device memory, and admits the head request as soon as a free
// region of the arena fits its memory estimate (first fit; freed regions
// merge with their free neighbours).  Each admission is posted to a completion
// ring in pinned memory, from which the host's workers take the request and
// run its kernels with all of its device state carved from the admitted
// region.  When a request is done, the host mails the region back.
//
// Every wait is bounded: the loop sleeps between polls and exits after
// idle_limit polls without work (status GC_ETIMEDOUT), or on a stop message
// (status GC_OK) once no request is waiting; its state stays in device
// memory, so the host relaunches it when new mail comes.  A full completion
// ring makes the loop keep the admission for a later poll.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace gc {

constexpr unsigned kMailSlots = 4096;     // mailbox and completion ring entries
constexpr unsigned kMaxRegions = 2048;    // arena region table entries
constexpr unsigned kMaxWaiting = 4096;    // requests waiting for admission

enum : unsigned { kMailAdmit = 1, kMailFree = 2, kMailStop = 3 };
enum : int { kLoopRunning = 1, kLoopExiting = 2, kLoopStopped = 3, kLoopTimedOut = 4 };

struct MailEntry {
  unsigned long long ticket;
  unsigned long long bytes;     // admit: the estimate; free: the region's offset
  unsigned op, pad;
};
struct DoneEntry {
  unsigned long long ticket;
  unsigned long long offset;    // admitted region [offset, offset + bytes) of the arena
  unsigned long long bytes;
};

// pinned, device-mapped
struct ServeHostShared {
  unsigned long long mail_head;   // host: entries written
  unsigned long long mail_tail;   // device: entries consumed
  unsigned long long done_head;   // device: admissions posted
  unsigned long long done_tail;   // host: admissions taken
  int loop_status;                // kLoop*
  int pad;
  unsigned long long polls;       // device: polls of the last launch
  MailEntry mail[kMailSlots];
  DoneEntry done[kMailSlots];
};

// device memory, owned by the loop (kept across its launches)
struct ServeDevState {
  unsigned long long consumed;                   // mailbox entries read
  unsigned long long wait_head, wait_tail;       // FIFO of requests waiting for admission
  unsigned long long wait_ticket[kMaxWaiting];
  unsigned long long wait_bytes[kMaxWaiting];
  unsigned n_regions;                            // regions in offset order, covering the arena
  unsigned pad;
  unsigned long long reg_off[kMaxRegions];
  unsigned long long reg_size[kMaxRegions];
  int reg_used[kMaxRegions];
  unsigned long long in_use;                     // bytes of admitted regions
  unsigned long long admitted, freed, stops;
  int stop;
};

__device__ __forceinline__ unsigned long long ld_acquire_sys(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed_sys(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.sys.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned ld_relaxed_sys_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.sys.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_sys(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void st_release_sys_i32(int* p, int v) {
  asm volatile("st.release.sys.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed_sys(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.sys.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// first fit; returns the offset or ~0 when nothing fits
__device__ inline unsigned long long region_alloc(ServeDevState* S, unsigned long long bytes) {
  for (unsigned i = 0; i < S->n_regions; ++i) {
    if (S->reg_used[i] || S->reg_size[i] < bytes) continue;
    const unsigned long long off = S->reg_off[i];
    if (S->reg_size[i] > bytes && S->n_regions < kMaxRegions) {   // split off the rest
      for (unsigned k = S->n_regions; k > i + 1; --k) {
        S->reg_off[k] = S->reg_off[k - 1];
        S->reg_size[k] = S->reg_size[k - 1];
        S->reg_used[k] = S->reg_used[k - 1];
      }
      S->reg_off[i + 1] = off + bytes;
      S->reg_size[i + 1] = S->reg_size[i] - bytes;
      S->reg_used[i + 1] = 0;
      S->reg_size[i] = bytes;
      ++S->n_regions;
    }
    S->reg_used[i] = 1;
    S->in_use += S->reg_size[i];
    return off;
  }
  return ~0ULL;
}

__device__ inline void region_free(ServeDevState* S, unsigned long long off) {
  unsigned i = 0;
  while (i < S->n_regions && S->reg_off[i] != off) ++i;
  if (i == S->n_regions || !S->reg_used[i]) return;   // unknown or already free: ignore
  S->reg_used[i] = 0;
  S->in_use -= S->reg_size[i];
  // merge with a free right neighbour, then with a free left one
  auto remove = [&](unsigned k) {
    for (unsigned m = k; m + 1 < S->n_regions; ++m) {
      S->reg_off[m] = S->reg_off[m + 1];
      S->reg_size[m] = S->reg_size[m + 1];
      S->reg_used[m] = S->reg_used[m + 1];
    }
    --S->n_regions;
  };
  if (i + 1 < S->n_regions && !S->reg_used[i + 1]) {
    S->reg_size[i] += S->reg_size[i + 1];
    remove(i + 1);
  }
  if (i > 0 && !S->reg_used[i - 1]) {
    S->reg_size[i - 1] += S->reg_size[i];
    remove(i);
  }
}

// One thread.  sleep_ns between polls without work; idle_limit such polls in
// a row end the launch with kLoopTimedOut.
__global__ void serve_loop_kernel(ServeHostShared* H, ServeDevState* S, long long idle_limit, unsigned sleep_ns) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  st_release_sys_i32(&H->loop_status, kLoopRunning);
  long long idle = 0;
  unsigned long long polls = 0;
  for (;;) {
    ++polls;
    bool progress = false;
    // read the new mail
    const unsigned long long head = ld_acquire_sys(&H->mail_head);
    while (S->consumed < head) {
      const MailEntry* m = &H->mail[S->consumed % kMailSlots];
      const unsigned op = ld_relaxed_sys_u32(&m->op);
      const unsigned long long ticket = ld_relaxed_sys(&m->ticket);
      const unsigned long long bytes = ld_relaxed_sys(&m->bytes);
      if (op == kMailAdmit) {
        if (S->wait_tail - S->wait_head >= kMaxWaiting) break;   // FIFO full: read it later
        S->wait_ticket[S->wait_tail % kMaxWaiting] = ticket;
        S->wait_bytes[S->wait_tail % kMaxWaiting] = bytes;
        ++S->wait_tail;
      } else if (op == kMailFree) {
        region_free(S, bytes);
        ++S->freed;
      } else if (op == kMailStop) {
        S->stop = 1;
        ++S->stops;
      }
      ++S->consumed;
      progress = true;
    }
    st_release_sys(&H->mail_tail, S->consumed);
    // admit waiting requests in arrival order while the head fits
    while (S->wait_head < S->wait_tail) {
      const unsigned long long done_tail = ld_acquire_sys(&H->done_tail);
      const unsigned long long dh = ld_relaxed_sys(&H->done_head);
      if (dh - done_tail >= kMailSlots) break;                   // completion ring full
      const unsigned long long bytes = S->wait_bytes[S->wait_head % kMaxWaiting];
      const unsigned long long off = region_alloc(S, bytes);
      if (off == ~0ULL) break;                                   // wait for frees
      DoneEntry* e = &H->done[dh % kMailSlots];
      st_relaxed_sys(&e->ticket, S->wait_ticket[S->wait_head % kMaxWaiting]);
      st_relaxed_sys(&e->offset, off);
      st_relaxed_sys(&e->bytes, bytes);
      st_release_sys(&H->done_head, dh + 1);
      ++S->wait_head;
      ++S->admitted;
      progress = true;
    }
    if (S->stop && S->wait_head == S->wait_tail) {
      S->stop = 0;
      st_relaxed_sys(&H->polls, polls);
      st_release_sys_i32(&H->loop_status, kLoopStopped);
      return;
    }
    if (progress) {
      idle = 0;
    } else if (++idle > idle_limit) {
      // announce the exit, then look at the mailbox once more: mail written
      // before the host saw kLoopExiting is read here, mail written after it
      // makes the host launch the loop again
      st_release_sys_i32(&H->loop_status, kLoopExiting);
      __threadfence_system();
      if (ld_acquire_sys(&H->mail_head) != S->consumed) {
        st_release_sys_i32(&H->loop_status, kLoopRunning);
        idle = 0;
        continue;
      }
      st_relaxed_sys(&H->polls, polls);
      st_release_sys_i32(&H->loop_status, kLoopTimedOut);
      return;
    }
    __nanosleep(sleep_ns);
  }
}

__global__ void serve_init_kernel(ServeDevState* S, unsigned long long arena_bytes) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  S->consumed = 0;
  S->wait_head = S->wait_tail = 0;
  S->n_regions = 1;
  S->reg_off[0] = 0;
  S->reg_size[0] = arena_bytes;
  S->reg_used[0] = 0;
  S->in_use = 0;
  S->admitted = S->freed = S->stops = 0;
  S->stop = 0;
}

}  // namespace gc
