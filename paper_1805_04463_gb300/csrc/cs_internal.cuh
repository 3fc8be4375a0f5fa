// cs_internal.cuh -- shared internals of the causal-set CUDA library.
//
// Generator, workspace header, status handling, PTX wrappers (mbarrier, TMA)
// and double-double arithmetic used by the kernels behind include/cs.h.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "../../include/cs.h"

namespace cs {

// ----------------------------------------------------------------- limits
constexpr int64_t kMaxN = int64_t(1) << 22;      // largest set the ABI accepts
constexpr int kGridBits = 20;                    // one unit of length = 2^20 grid steps
constexpr int64_t kGrid = int64_t(1) << kGridBits;
constexpr int kMaxAttempts = 16384;              // 4D rejection attempts per element
constexpr unsigned long long kWaitLimitNs = 4000000000ull;  // bounded in-kernel waits: 4 s

// ------------------------------------------------------------- generator
// SplitMix64 (Steele, Lea & Flood 2014) in counter form: output number q of
// a generator started at state s is mix(s + (q + 1) * gamma).
constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Key of a stream: output `stream` of the generator started at `seed`.
__host__ __device__ __forceinline__ uint64_t stream_key(uint64_t seed, uint32_t stream) {
    return mix64(seed + (uint64_t(stream) + 1) * kGamma);
}

// Draw `slot` of element e in a stream with key sigma: output e*65536+slot.
__host__ __device__ __forceinline__ uint64_t draw_from(uint64_t sigma, uint64_t e, uint32_t slot) {
    return mix64(sigma + (e * 65536ull + slot + 1) * kGamma);
}

// --------------------------------------------------------- workspace head
// Every workspace starts with this 256-byte header.
struct WsHeader {
    int32_t status;                  // first in-kernel error (cs_status), 0 = none
    uint32_t pad0;
    unsigned long long counter;      // work-queue cursor for persistent kernels
    unsigned long long aux[30];
};
static_assert(sizeof(WsHeader) == 256, "workspace header is 256 bytes");

__device__ __forceinline__ void set_status(WsHeader* h, int code) {
    atomicCAS(&h->status, 0, code);
}

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Tracing: every C-ABI entry point that enqueues GPU work opens an NVTX range
// named after itself (header-only NVTX; a no-op unless a profiler attaches).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};
#define CS_TRACE(name) ::cs::NvtxRange cs_trace_range_(name)

// --------------------------------------------------------------- PTX glue
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory add without a return value at a shared-window address (a
// generic-address atomicAdd on dynamic shared memory compiles to a generic
// atomic).
__device__ __forceinline__ void red_shared_add(uint32_t saddr, uint32_t v) {
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(saddr), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long global_timer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// `count` arrivals at once.
__device__ __forceinline__ void mbar_arrive_cnt(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// `count` arrivals without ordering earlier memory accesses (no fence): for
// a signal whose precondition is an instruction that has already completed
// (a tcgen05.ld after its tcgen05.wait::ld), not a memory access.
__device__ __forceinline__ void mbar_arrive_relaxed_cnt(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.arrive.relaxed.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of an mbarrier with a time limit.  Returns false
// (and records CS_ETIMEOUT) if the phase did not complete in time.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, WsHeader* h,
                                                  unsigned long long limit_ns = kWaitLimitNs) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_timer_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_timer_ns() - t0 > limit_ns) {
            set_status(h, CS_ETIMEOUT);
            return false;
        }
    }
    return true;
}

// 2D tiled TMA load global -> shared, completion signalled on `bar`.
__device__ __forceinline__ void tma_load_2d(void* smem_dst, const CUtensorMap* map, int32_t x, int32_t y,
                                            uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(smem_dst)), "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Contiguous bulk copy global -> shared of `bytes` (a multiple of 16, both
// addresses 16-byte aligned), completion signalled on `bar`.
__device__ __forceinline__ void bulk_load(void* smem_dst, const void* gsrc, uint32_t bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_u32(smem_dst)), "l"(gsrc), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

// ------------------------------------------------ thread-block clusters
__device__ __forceinline__ uint32_t cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// All threads of every CTA of the cluster; orders the memory operations
// before it (local and remote shared memory, mbarrier arrivals) before those
// after it.
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// The shared::cluster address of the same shared-memory offset in CTA `rank`.
__device__ __forceinline__ uint32_t cluster_map(const void* p, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(smem_u32(p)), "r"(rank));
    return r;
}

__device__ __forceinline__ void st_cluster_s64(uint32_t caddr, int64_t v) {
    asm volatile("st.shared::cluster.s64 [%0], %1;" ::"r"(caddr), "l"(v) : "memory");
}

// `count` arrivals on an mbarrier anywhere in the cluster, release at
// cluster scope (orders this thread's earlier accesses before them).
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t caddr, uint32_t count) {
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0], %1;" ::"r"(caddr), "r"(count)
                 : "memory");
}

// The same arrivals without ordering earlier memory accesses (see
// mbar_arrive_relaxed_cnt).
__device__ __forceinline__ void mbar_arrive_cluster_relaxed(uint32_t caddr, uint32_t count) {
    asm volatile("mbarrier.arrive.relaxed.cluster.shared::cluster.b64 _, [%0], %1;" ::"r"(caddr), "r"(count)
                 : "memory");
}

// try_wait with acquire at cluster scope: for phases completed by arrivals
// of other CTAs whose earlier shared-memory writes must be visible.
__device__ __forceinline__ bool mbar_try_wait_cluster(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.b32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait like mbar_wait_bounded, but also give up early once another warp of
// the CTA has raised *abort (set after its own wait timed out).
// kCluster: acquire at cluster scope (phases completed by other CTAs).
template <bool kCluster = false>
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t* bar, uint32_t parity, WsHeader* h,
                                                   volatile int* abort) {
    auto ready = [&] { return kCluster ? mbar_try_wait_cluster(bar, parity) : mbar_try_wait(bar, parity); };
    if (ready()) return true;
    const unsigned long long t0 = global_timer_ns();
    for (uint32_t spin = 0;; ++spin) {
        if (ready()) return true;
        if ((spin & 63u) == 0u) {
            if (*abort) return false;
            if (global_timer_ns() - t0 > kWaitLimitNs) {
                set_status(h, CS_ETIMEOUT);
                *abort = 1;
                return false;
            }
        }
    }
}

// ---------------------------------------------------- tcgen05 (sm_100 family)
// Tensor memory allocation by one full warp; the base address is written to
// shared memory.  ncols is a power of two >= 32.
__device__ __forceinline__ void tmem_alloc(uint32_t* smem_dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(smem_dst)),
                 "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor for a K-major operand tile stored by TMA
// with a 128- or 64-byte swizzle: rows of `row_bytes` bytes, 8-row swizzle
// atoms stacked at a stride of 8 * row_bytes.  Fields: start address >> 4
// (bits 0-13), leading byte offset >> 4 (16-29, unused for swizzled K-major),
// stride byte offset >> 4 (32-45), descriptor version 1 (46-47), layout type
// (61-63): 2 = 128B swizzle, 4 = 64B swizzle.  The tile base must be aligned
// to the swizzle atom (1024 bytes covers both).
__device__ __forceinline__ uint64_t sdesc_k_swizzled(uint32_t saddr, uint32_t row_bytes) {
    uint64_t d = 0;
    d |= uint64_t((saddr & 0x3FFFFu) >> 4);
    d |= uint64_t(1) << 16;
    d |= uint64_t((8u * row_bytes) >> 4) << 32;
    d |= uint64_t(1) << 46;
    d |= uint64_t(row_bytes == 128 ? 2 : 4) << 61;
    return d;
}

// Instruction descriptor for kind::f8f6f4: D = F32 (bits 4-5 = 1), A = B =
// E4M3 (bits 7-9, 10-12 = 0), both K-major (bits 15, 16 = 0), N >> 3 in bits
// 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_f8_f32(int m, int n) {
    return (1u << 4) | (uint32_t(n >> 3) << 17) | (uint32_t(m >> 4) << 24);
}

// D[tmem] (+)= A[smem] * B[smem]^T, one CTA, kind::f8f6f4.
__device__ __forceinline__ void mma_f8f6f4(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                           uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Instruction descriptor for kind::mxf4 (block-scaled FP4): A = B = E2M1
// (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 in bits
// 17-22, scale factors UE8M0 (bit 23 = 1), M >> 4 in bits 24-28; both
// scale-factor data IDs (bits 4-5, 29-30) and the K size bit (31, dense K64)
// are 0.  D is always F32 for the block-scaled kinds.
__host__ __device__ constexpr uint32_t idesc_mxf4_f32(int m, int n) {
    return (1u << 7) | (1u << 10) | (uint32_t(n >> 3) << 17) | (1u << 23) | (uint32_t(m >> 4) << 24);
}

// D[tmem] (+)= (A[smem] x SFA[tmem]) * (B[smem] x SFB[tmem])^T, one CTA,
// kind::mxf4 with one UE8M0 scale per 32 K-elements (K64 per instruction).
__device__ __forceinline__ void mma_mxf4(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t sfa_tmem, uint32_t sfb_tmem, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %6, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::mxf4.block_scale.scale_vec::2X [%0], %1, %2, %3, [%4], [%5], p;\n\t}"
        ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(sfa_tmem), "r"(sfb_tmem), "r"(accumulate)
        : "memory");
}

// Each lane writes the value v into 32 consecutive 32-bit columns of its TMEM
// lane (the warp's lane quarter only).
__device__ __forceinline__ void tmem_st_32x32b_x32_fill(uint32_t taddr, uint32_t v) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
        "{%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, "
        "%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1};" ::"r"(taddr),
        "r"(v)
        : "memory");
}

__device__ __forceinline__ void tmem_st_wait() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// ------------------------------------------ CTA-pair (cta_group::2) forms
// A pair of CTAs of one cluster shares each MMA: one warp of EACH CTA runs
// the allocation (both get the same columns in their own SM's TMEM); one
// thread of the even CTA issues every MMA, which reads the A and B halves
// held at the same shared-memory address in both CTAs and writes rows
// 0-127 of D to the even CTA's TMEM, rows 128-255 to the odd CTA's.
__device__ __forceinline__ void tmem_alloc_pair(uint32_t* smem_dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(smem_dst)),
                 "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void tmem_relinquish_pair() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc_pair(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void mma_mxf4_pair(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                              uint32_t sfa_tmem, uint32_t sfb_tmem, uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %6, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::mxf4.block_scale.scale_vec::2X [%0], %1, %2, %3, [%4], [%5], p;\n\t}"
        ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(sfa_tmem), "r"(sfb_tmem), "r"(accumulate)
        : "memory");
}

// Arrive once on the mbarrier at `bar`'s offset in every CTA of `mask` when
// the pair's previously issued MMAs have completed.
__device__ __forceinline__ void mma_commit_pair_mc(uint64_t* bar, uint16_t mask) {
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            smem_u32(bar)),
        "h"(mask)
        : "memory");
}

// 2D tiled TMA load into this CTA's shared memory whose byte count is
// signalled on an mbarrier of either CTA of the pair (shared::cluster
// address `bar_cluster`).
__device__ __forceinline__ void tma_load_2d_pair(void* smem_dst, const CUtensorMap* map, int32_t x, int32_t y,
                                                 uint32_t bar_cluster) {
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3}], [%4];"
        ::"r"(smem_u32(smem_dst)), "l"(map), "r"(x), "r"(y), "r"(bar_cluster)
        : "memory");
}

// Arrive once on an mbarrier when all previously issued tcgen05 ops of this
// thread have completed.
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// Each lane reads 32 consecutive 32-bit columns of its TMEM lane.
__device__ __forceinline__ void tmem_ld_32x32b_x32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr)
        : "memory");
}

__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// ----------------------------------------------------- double-double FP64
// Error-free transformations (Knuth TwoSum; FMA-based TwoProduct) and the
// double-double operations built on them (Dekker 1971; Hida, Li & Bailey,
// "Algorithms for quad-double precision floating point arithmetic", 2001).
struct dd {
    double hi, lo;
};

__host__ __device__ __forceinline__ dd dd_two_sum(double a, double b) {
    double s = a + b;
    double bb = s - a;
    double e = (a - (s - bb)) + (b - bb);
    return {s, e};
}

__host__ __device__ __forceinline__ dd dd_quick_two_sum(double a, double b) {
    double s = a + b;
    double e = b - (s - a);
    return {s, e};
}

__host__ __device__ __forceinline__ dd dd_two_prod(double a, double b) {
    double p = a * b;
    double e = fma(a, b, -p);
    return {p, e};
}

__host__ __device__ __forceinline__ dd dd_from(double a) { return {a, 0.0}; }

__host__ __device__ __forceinline__ dd dd_add(dd x, dd y) {
    dd s = dd_two_sum(x.hi, y.hi);
    dd t = dd_two_sum(x.lo, y.lo);
    s.lo += t.hi;
    s = dd_quick_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return dd_quick_two_sum(s.hi, s.lo);
}

__host__ __device__ __forceinline__ dd dd_neg(dd x) { return {-x.hi, -x.lo}; }

__host__ __device__ __forceinline__ dd dd_sub(dd x, dd y) { return dd_add(x, dd_neg(y)); }

__host__ __device__ __forceinline__ dd dd_mul(dd x, dd y) {
    dd p = dd_two_prod(x.hi, y.hi);
    p.lo = fma(x.hi, y.lo, p.lo);
    p.lo = fma(x.lo, y.hi, p.lo);
    return dd_quick_two_sum(p.hi, p.lo);
}

__host__ __device__ __forceinline__ dd dd_mul_d(dd x, double b) {
    dd p = dd_two_prod(x.hi, b);
    p.lo = fma(x.lo, b, p.lo);
    return dd_quick_two_sum(p.hi, p.lo);
}

// An int64 as a double-double, exactly (|v| < 2^106).
__host__ __device__ __forceinline__ dd dd_from_i64(int64_t v) {
    double hi = static_cast<double>(v);
    double lo = static_cast<double>(v - static_cast<int64_t>(hi));
    return dd_quick_two_sum(hi, lo);
}

// x^k by binary powering (k >= 0).
__host__ __device__ inline dd dd_pow(dd x, int64_t k) {
    dd r = dd_from(1.0);
    while (k > 0) {
        if (k & 1) r = dd_mul(r, x);
        x = dd_mul(x, x);
        k >>= 1;
    }
    return r;
}

// Smearing functions with the (1-eps) denominators cleared, so that they are
// exact at eps = 1 (Section "The Benincasa-Dowker Action"):
//   f2(k) = q^(k-2) [q^2 - 2 k eps q + k(k-1)/2 eps^2],                 q = 1 - eps
//   f3(k) = q^(k-2) [q^2 - 27/8 k eps q + 9/8 k(k-1) eps^2]
//   f4(k) = q^(k-3) [q^3 - 9 k eps q^2 + 8 k(k-1) eps^2 q - 8 C(k,3) eps^3]
// (4/3 k(k-1)(k-2) = 8 C(k,3) is an integer).  qpow = q^(k - deg) for the
// general branch; the small-k branches expand the printed forms directly.
__host__ __device__ inline dd smear_poly(int dim, int64_t k, dd q, double eps) {
    const dd e = dd_from(eps);
    if (dim == 2) {
        if (k == 0) return dd_from(1.0);
        if (k == 1) return dd_sub(q, dd_mul_d(e, 2.0));              // (1-eps) - 2 eps
        dd a = dd_mul(q, q);
        dd b = dd_mul(dd_mul_d(e, 2.0 * static_cast<double>(k)), q);
        dd c = dd_mul(dd_mul(e, e), dd_from_i64(k * (k - 1) / 2));
        return dd_add(dd_sub(a, b), c);
    }
    if (dim == 3) {
        if (k == 0) return dd_from(1.0);
        if (k == 1) return dd_sub(q, dd_mul_d(e, 3.375));            // (1-eps) - 27/8 eps
        // 27 k / 8 and 9 k(k-1)/8 are exact doubles for k < 2^22
        dd a = dd_mul(q, q);
        dd b = dd_mul(dd_mul_d(e, 3.375 * static_cast<double>(k)), q);
        dd c = dd_mul(dd_mul(e, e), dd_from(2.25 * static_cast<double>(k * (k - 1) / 2)));
        return dd_add(dd_sub(a, b), c);
    }
    // dim == 4
    if (k == 0) return dd_from(1.0);
    if (k == 1) return dd_sub(q, dd_mul_d(e, 9.0));                  // (1-eps) - 9 eps
    if (k == 2) {                                                     // q^2 - 18 eps q + 16 eps^2
        dd a = dd_mul(q, q);
        dd b = dd_mul(dd_mul_d(e, 18.0), q);
        dd c = dd_mul_d(dd_mul(e, e), 16.0);
        return dd_add(dd_sub(a, b), c);
    }
    // k < 2^22, so k(k-1)/2 < 2^43 and each factor below is an exact double;
    // a two_prod of exact factors is the exact product.
    const int64_t t = k * (k - 1) / 2;
    const dd c3 = ((k - 2) % 3 == 0)
                      ? dd_two_prod(static_cast<double>(t), static_cast<double>((k - 2) / 3))
                      : dd_two_prod(static_cast<double>(t / 3), static_cast<double>(k - 2));  // C(k,3)
    dd q2 = dd_mul(q, q);
    dd a = dd_mul(q2, q);
    dd b = dd_mul(dd_mul_d(e, 9.0 * static_cast<double>(k)), q2);
    dd c = dd_mul(dd_mul(dd_mul(e, e), dd_two_prod(8.0 * static_cast<double>(k), static_cast<double>(k - 1))), q);
    dd d = dd_mul(dd_mul(dd_mul(e, e), e), dd_mul_d(c3, 8.0));
    return dd_sub(dd_add(dd_sub(a, b), c), d);
}

// Degree of the polynomial factor of f_d (the power of 1/(1-eps) pulled out).
__host__ __device__ __forceinline__ int64_t smear_deg(int dim) { return dim == 4 ? 3 : 2; }

// Exponent of q multiplying smear_poly for index k.
__host__ __device__ __forceinline__ int64_t smear_qexp(int dim, int64_t k) {
    const int64_t deg = smear_deg(dim);
    return k >= deg ? k - deg : 0;
}

}  // namespace cs
