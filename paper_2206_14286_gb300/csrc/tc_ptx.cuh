// tc_ptx.cuh -- inline-PTX wrappers for TMA, mbarrier and tcgen05 used by the
// tensor-core kernels, plus the bounded wait and its device-wide timeout flag.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace tpuknn {

// Set by a kernel whose bounded wait ran out; read and cleared by the host
// (tc_take_timeout). Each translation unit including this header has its own
// copy, so every tensor-core kernel file exports a reader.
static __device__ unsigned int g_tc_timeout = 0;
constexpr uint64_t kTimeoutNs = 2000000000ull;
// The limit of the pipeline waits (mbar_wait, mbar_wait_sleep); the host may
// lower it (knn_set_wait_limit_ns) to make a wait run out in a test. The
// drain waits after a give-up (mbar_drain) keep kTimeoutNs.
static __device__ unsigned long long g_tc_wait_limit_ns = kTimeoutNs;
// Limits below this (under the global timer's resolution) make a pipeline wait
// give up at its first check instead of comparing times.
constexpr uint64_t kImmediateNs = 1000;
// Suspend-time hint of one mbarrier.try_wait probe in the sleeping waits.
constexpr uint32_t kSuspendHintNs = 20000;

namespace {
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Non-suspending probe of the phase (the thread keeps polling, so it sees the
// completion within a few cycles instead of a suspend interval).
__device__ __forceinline__ bool mbar_test_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Potentially suspending probe: if the phase is not complete the thread may
// be suspended until it completes or about `hint_ns` pass (the hardware's
// time limit may be shorter), so a waiting warp issues almost nothing.
__device__ __forceinline__ bool mbar_try_wait_hint(uint32_t bar, uint32_t parity,
                                                   uint32_t hint_ns) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(hint_ns)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ uint64_t wait_limit_ns() {
  return *reinterpret_cast<volatile unsigned long long*>(&g_tc_wait_limit_ns);
}
// Bounded wait for the phase of `parity` to complete. Returns false when the
// limit runs out (the caller's CTA then aborts: this thread raises the CTA's
// abort flag and the device-wide timeout flag) or when another thread of the
// CTA has raised the abort flag. Each lane decides on its own: callers that
// need a warp-wide decision combine the lanes' results (warp_all).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag) {
  if (mbar_test_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  const uint64_t lim = wait_limit_ns();
  for (uint32_t n = 1;; ++n) {
    if (mbar_test_wait(bar, parity)) return true;
    if (n == 1 || (n & 1023) == 0) {
      if (*abort_flag) return false;
      if (lim < kImmediateNs || global_ns() - t0 > lim) {
        *abort_flag = 1;
        atomicExch(&g_tc_timeout, 1u);
        return false;
      }
    }
  }
}
// Bounded wait for roles with slack (producer, epilogue, ...): the warp
// waits suspended in mbarrier.try_wait (woken when the phase completes), so
// its polling does not take issue slots from the roles that work.
__device__ __forceinline__ bool mbar_wait_sleep(uint32_t bar, uint32_t parity,
                                                volatile int* abort_flag) {
  if (mbar_test_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  const uint64_t lim = wait_limit_ns();
  for (;;) {
    if (*abort_flag) return false;
    if (lim < kImmediateNs || global_ns() - t0 > lim) {
      *abort_flag = 1;
      atomicExch(&g_tc_timeout, 1u);
      return false;
    }
    if (mbar_try_wait_hint(bar, parity, kSuspendHintNs)) return true;
  }
}
// Wait used on the way out after a give-up: the copies and MMAs a CTA has
// already issued must finish before it releases its shared and tensor memory,
// so this wait ignores the abort flag. It is bounded by the fixed kTimeoutNs
// (a wait that runs out here records the timeout and returns).
__device__ __forceinline__ bool mbar_drain(uint32_t bar, uint32_t parity) {
  if (mbar_test_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (uint32_t n = 1;; ++n) {
    __nanosleep(64);
    if (mbar_test_wait(bar, parity)) return true;
    if ((n & 15) == 0 && global_ns() - t0 > kTimeoutNs) {
      atomicExch(&g_tc_timeout, 1u);
      return false;
    }
  }
}
// A decision every lane of the warp takes together (all 32 lanes call it):
// true only if it holds in every lane. After a wait, lanes that may have given
// up at different moments then leave (or stay) as one warp, as the warp-wide
// .sync.aligned instructions that follow require.
__device__ __forceinline__ bool warp_all(bool ok) { return __all_sync(0xffffffffu, ok) != 0; }
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar,
                                            int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, uint32_t bar,
                                            int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}
template <int DT>
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                       uint32_t idesc, uint32_t accum) {
  if (DT == KNN_BF16) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
  }
}
// Start loading 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
}
// Wait for this thread's outstanding TMEM loads; the registers are tied to the
// wait so no use of them can be scheduled before it.
__device__ __forceinline__ void tmem_wait(uint32_t (&r)[32]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                 "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                 "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]),
                 "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]),
                 "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]),
                 "+r"(r[30]), "+r"(r[31])
               :
               : "memory");
}

// Shared-memory matrix descriptor of a K-major operand laid out by TMA with
// the 128-byte swizzle: rows of 128 bytes, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3ffffu) >> 4);        // start address
  d |= (uint64_t)(16u >> 4) << 16;                // leading byte offset (unused here)
  d |= (uint64_t)(1024u >> 4) << 32;              // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                         // descriptor version
  d |= (uint64_t)2 << 61;                         // 128-byte swizzle
  return d;
}


// Shared-memory descriptor of a K-major operand without swizzle: core
// matrices of 8 rows x 16 bytes stored contiguously; lbo = byte distance
// between core matrices adjacent along K, sbo = between 8-row groups.
__device__ __forceinline__ uint64_t smem_desc_noswz(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3ffffu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3fffu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3fffu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
}  // namespace

// Host: set this translation unit's pipeline-wait limit on the current
// device (ns = 0: the default kTimeoutNs).
static inline bool tc_set_wait_limit_local(unsigned long long ns) {
  const unsigned long long v = ns ? ns : kTimeoutNs;
  if (cudaMemcpyToSymbol(g_tc_wait_limit_ns, &v, sizeof(v)) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return true;
}

// Host: read and clear this translation unit's timeout flag.
static inline bool tc_take_timeout_local() {
  unsigned int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_tc_timeout, sizeof(v)) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (v) {
    unsigned int z = 0;
    cudaMemcpyToSymbol(g_tc_timeout, &z, sizeof(z));
  }
  return v != 0;
}

}  // namespace tpuknn
