// device.cuh -- device helpers shared by the TSQR kernels (sm_103a).
//
// * 1-D bulk TMA copies (cp.async.bulk) between global and shared memory,
//   completed on an mbarrier; every wait is bounded and reports
//   TSQR_ERR_TIMEOUT through the status word instead of hanging.
// * The device status word (first error wins, never a trap).
// * Warp "transpose-reduce": reduces V values per lane across the 32 lanes of
//   a warp with about V adds per lane instead of 5 V.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/tsqr.h"

namespace tsqr {

// Wall-clock limit (ns, %globaltimer) on any wait for a bulk copy; a copy of
// at most a few hundred KB completes in microseconds, so expiry means a lost
// transaction and is reported as TSQR_ERR_TIMEOUT.
constexpr uint64_t kWaitLimitNs = 1000000000ull;

__device__ __forceinline__ uint64_t global_timer_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Thread-block clusters: this CTA's rank, the cluster-wide barrier (every
// thread of every CTA; release / acquire orders the shared::cluster
// accesses around it), and loads / stores of another CTA's shared memory.
__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_barrier() {
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}
// shared-memory address of the same variable in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t cluster_map(const void* p, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_cluster(uint32_t addr, double v) {
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(addr), "d"(v) : "memory");
}
__device__ __forceinline__ double ld_cluster(uint32_t addr) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(addr) : "memory");
  return v;
}

__device__ __forceinline__ void set_status(int32_t* status, int32_t code) {
  if (status) atomicCAS(status, 0, code);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// The same with a suspend-time hint: a thread whose phase is not complete
// sleeps (issuing nothing) until it completes or about `ns` elapse.
__device__ __forceinline__ bool mbar_try_wait_sleep(uint64_t* bar, uint32_t parity, uint32_t ns) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity), "r"(ns)
      : "memory");
  return done != 0;
}

// Bounded wait for phase `parity` of `bar`; false after kWaitLimitNs.  The
// polls sleep between checks, so waiting warps take no issue slots.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_timer_ns();
  while (true) {
    if (mbar_try_wait_sleep(bar, parity, 100000u)) return true;
    if (global_timer_ns() - t0 > kWaitLimitNs) return false;
  }
}

// global -> shared bulk copy of `bytes` (multiple of 16, both addresses 16-aligned)
__device__ __forceinline__ void bulk_g2s(void* dst_smem, const void* src_gmem, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst_smem)),
      "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// shared -> global bulk copy (bulk-group completion)
__device__ __forceinline__ void bulk_s2g(void* dst_gmem, const void* src_smem, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst_gmem),
               "r"(smem_u32(src_smem)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// the shared-memory sources of every committed bulk store have been read
// (the buffers may be overwritten; the global writes may still be in flight)
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// ... of all but the most recently committed one
__device__ __forceinline__ void bulk_wait_read_1() { asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory"); }
// generic-proxy writes to shared memory become visible to the async (bulk) proxy
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 4-byte asynchronous global -> shared copy (cp.async, through L1), and the
// wait for all of this thread's outstanding ones.
__device__ __forceinline__ void cp_async_4(void* dst_smem, const void* src_gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst_smem)), "l"(src_gmem) : "memory");
}
__device__ __forceinline__ void cp_async_8(void* dst_smem, const void* src_gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst_smem)), "l"(src_gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// Largest chunk per bulk copy (keeps each mbarrier transaction count small).
constexpr uint32_t kBulkChunk = 1u << 16;

// Load `count` elements of T from global `src` into shared `dst` using bulk
// copies for the 16-byte-aligned body and plain loads for the ragged tail.
// Must be called by the whole CTA; returns false (and sets the status) if the
// copy did not complete.  `bar` is an initialised mbarrier whose next phase
// has parity `parity`; the parity is advanced when the barrier was used.
template <class T>
__device__ bool cta_load_bulk(T* dst, const T* src, int64_t count, uint64_t* bar, uint32_t& parity,
                              int32_t* status) {
  const uint64_t bytes = static_cast<uint64_t>(count) * sizeof(T);
  const uint64_t body = bytes & ~static_cast<uint64_t>(15);
  const bool aligned = (reinterpret_cast<uintptr_t>(src) & 15) == 0;
  const uint64_t use = aligned ? body : 0;
  if (threadIdx.x == 0 && use > 0) {
    mbar_arrive_expect_tx(bar, static_cast<uint32_t>(use));
    for (uint64_t off = 0; off < use; off += kBulkChunk) {
      uint32_t len = static_cast<uint32_t>(use - off < kBulkChunk ? use - off : kBulkChunk);
      bulk_g2s(reinterpret_cast<char*>(dst) + off, reinterpret_cast<const char*>(src) + off, len, bar);
    }
  }
  for (int64_t e = static_cast<int64_t>(use / sizeof(T)) + threadIdx.x; e < count; e += blockDim.x)
    dst[e] = src[e];
  bool ok = true;
  if (use > 0) {
    ok = mbar_wait_bounded(bar, parity);
    parity ^= 1u;
  }
  if (!ok && threadIdx.x == 0) set_status(status, TSQR_ERR_TIMEOUT);
  // every thread has left the wait before the barrier can be re-armed, so a
  // later phase of the same parity is never mistaken for this one
  __syncthreads();
  return ok;
}

// Store `count` elements from shared `src` to global `dst` (bulk body + plain
// tail).  Whole CTA.  Before the call every thread that wrote `src` executes
// fence_proxy_async_smem() and then the CTA synchronises, so that the bulk
// copy (async proxy) sees the generic-proxy writes.
template <class T>
__device__ void cta_store_bulk(T* dst, const T* src, int64_t count) {
  const uint64_t bytes = static_cast<uint64_t>(count) * sizeof(T);
  const uint64_t body = bytes & ~static_cast<uint64_t>(15);
  const bool aligned = (reinterpret_cast<uintptr_t>(dst) & 15) == 0;
  const uint64_t use = aligned ? body : 0;
  if (threadIdx.x == 0 && use > 0) {
    for (uint64_t off = 0; off < use; off += kBulkChunk) {
      uint32_t len = static_cast<uint32_t>(use - off < kBulkChunk ? use - off : kBulkChunk);
      bulk_s2g(reinterpret_cast<char*>(dst) + off, reinterpret_cast<const char*>(src) + off, len);
    }
    bulk_commit();
  }
  for (int64_t e = static_cast<int64_t>(use / sizeof(T)) + threadIdx.x; e < count; e += blockDim.x)
    dst[e] = src[e];
  if (threadIdx.x == 0 && use > 0) bulk_wait_all();
}

template <class T>
__device__ __forceinline__ T shfl_xor(T v, int o) {
  return __shfl_xor_sync(0xffffffffu, v, o);
}

// Named CTA barrier `id` (1..15; 0 is __syncthreads) over `nthreads`
// threads (a multiple of 32): producers arrive without waiting, consumers
// wait until all `nthreads` have arrived.  Writes made by a producer before
// its arrive are visible to the consumers after their sync.
__device__ __forceinline__ void named_bar_arrive(int id, int nthreads) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
__device__ __forceinline__ void named_bar_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}
// Named barrier that also returns the AND of `pred` over its `nthreads`
// threads (a uniform decision after per-thread bounded waits).
__device__ __forceinline__ bool named_bar_and(int id, int nthreads, bool pred) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
      "bar.red.and.pred q, %2, %3, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"(static_cast<uint32_t>(pred)), "r"(id), "r"(nthreads)
      : "memory");
  return r != 0;
}

// Warp transpose-reduce.  On entry every lane holds s[0..V); on exit the sum
// over all 32 lanes of index i is written to dst[i] for every i < V by the
// lanes that own it (several lanes may write the same, identical value).
// Each halving step exchanges half of the remaining values with the partner
// lane; once one value is left the remaining offsets are plain butterflies.
// `limit` is the exclusive end of the indices owned by the current subtree:
// the padding slot of an odd-length half must not be written, because its
// index belongs to the sibling subtree.
template <int V, int O>
struct TransposeReduce {
  template <class T>
  static __device__ __forceinline__ void run(const T (&s)[V], int lane, int base, int limit, T* dst) {
    if constexpr (O == 0) {
#pragma unroll
      for (int i = 0; i < V; ++i)
        if (base + i < limit) dst[base + i] = s[i];
    } else if constexpr (V == 1) {
      T t[1] = {s[0] + shfl_xor(s[0], O)};
      TransposeReduce<1, O / 2>::run(t, lane, base, limit, dst);
    } else {
      constexpr int H = (V + 1) / 2;
      T t[H];
      const bool up = (lane & O) != 0;
#pragma unroll
      for (int i = 0; i < H; ++i) {
        T lo = s[i];
        T hi = (H + i < V) ? s[H + i] : T(0);
        T send = up ? lo : hi;
        T keep = up ? hi : lo;
        t[i] = keep + shfl_xor(send, O);
      }
      // one call with selected arguments: no divergent branch, so every
      // lane reaches the same shuffles
      const int nbase = up ? base + H : base;
      const int nlimit = up ? limit : ((base + H < limit) ? base + H : limit);
      TransposeReduce<H, O / 2>::run(t, lane, nbase, nlimit, dst);
    }
  }
};

}  // namespace tsqr
