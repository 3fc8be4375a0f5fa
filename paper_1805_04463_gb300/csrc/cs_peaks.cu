// cs_peaks.cu -- peak probes for the rooflines of the count kernels: the
// innermost operation of each count path, on every SM, with nothing around
// it.  The tensor probes issue the count kernels' own MMA shapes back to back
// from operands resident in shared memory (no TMA, no epilogue, one commit at
// the end); the POPC probe issues independent 32-bit population counts from
// registers.  The thesis has no counterpart: this is measurement
// infrastructure for the library's own kernels.
#include "cs_kernels.cuh"

namespace cs {

namespace {

constexpr int kProbeThreads = 128;     // four warps: one per TMEM lane quarter
constexpr int kProbeA = 128 * 128;     // A slab bytes (128 rows of a 128-byte swizzle row)
constexpr int kProbeB8 = 256 * 128;    // FP8: B slab of 256 rows
constexpr int kProbeB4 = 128 * 128;    // FP4 pair: this CTA's half of a 256-row B slab
// More than half of an SM's shared memory, so that every probe CTA has an SM
// (and its tensor core) to itself, as in the count kernels.
constexpr int kProbeSmem = 120 * 1024;
static_assert(kProbeA + kProbeB8 + 1024 <= kProbeSmem, "the FP8 operands fit");
constexpr int kProbeSmem8 = kProbeSmem;
constexpr int kProbeSmem4 = kProbeSmem;
constexpr unsigned long long kProbeWaitNs = 10000000000ull;  // 10 s
// At most 2^22 repetitions: a few seconds of work on any path, far inside
// the bounded wait, so the MMAs have always finished when TMEM is freed.
constexpr int64_t kProbeMaxReps = int64_t(1) << 22;

// 0/1 operand bytes in the given one's format, a fixed pattern.
__device__ __forceinline__ void fill_operands(uint8_t* smem, int bytes, uint32_t one_lo, uint32_t one_hi) {
    for (int t = threadIdx.x; t < bytes / 16; t += blockDim.x) {
        const uint32_t m = uint32_t(t) * 0x9E3779B1u;
        reinterpret_cast<uint4*>(smem)[t] =
            make_uint4(m & one_lo, (m >> 3) & one_hi, (m >> 7) & one_lo, (m >> 11) & one_hi);
    }
    fence_proxy_async();  // the tensor core reads shared memory through the async proxy
}

// FP8, one CTA per SM: `reps` x 4 MMAs of M128 N256 K32 into one accumulator.
__global__ void __launch_bounds__(kProbeThreads, 1) k_probe_f8(int64_t reps, WsHeader* hdr) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ uint64_t bar;
    __shared__ uint32_t tslot;
    const int warp = threadIdx.x >> 5;
    fill_operands(smem, kProbeA + kProbeB8, 0x38383838u, 0x38003800u);  // E4M3 1.0 = 0x38
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(&tslot, 256);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t d = tslot;
    if (threadIdx.x == 0) {
        const uint32_t a = smem_u32(smem);
        const uint64_t adesc = sdesc_k_swizzled(a, 128), bdesc = sdesc_k_swizzled(a + kProbeA, 128);
        constexpr uint32_t idesc = idesc_f8_f32(128, 256);
        for (int64_t r = 0; r < reps; ++r)
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
                mma_f8f6f4(d, adesc + uint64_t(2 * kk), bdesc + uint64_t(2 * kk), idesc, (r > 0 || kk > 0) ? 1u : 0u);
        mma_commit(&bar);
        mbar_wait_bounded(&bar, 0, hdr, kProbeWaitNs);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(d, 256);
    }
}

// FP4 on CTA pairs: `reps` x 4 block-scaled MMAs of M256 N256 K64 issued by
// rank 0 for the pair (each CTA holds half of A and half of B).
__global__ void __launch_bounds__(kProbeThreads, 1) k_probe_f4_pair(int64_t reps, WsHeader* hdr) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ uint64_t bar;
    __shared__ uint32_t tslot;
    const int warp = threadIdx.x >> 5;
    const bool leader = cluster_ctarank() == 0;
    fill_operands(smem, kProbeA + kProbeB4, 0x22222222u, 0x20202020u);  // E2M1 1.0 = nibble 0x2
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc_pair(&tslot, 512);
        tmem_relinquish_pair();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t d = tslot;
    // every scale factor 1 (UE8M0 0x7F): columns 256..287 of all 128 lanes
    tmem_st_32x32b_x32_fill(d + (uint32_t(32 * warp) << 16) + 256u, 0x7F7F7F7Fu);
    tmem_st_wait();
    tc_fence_before();
    __syncthreads();
    cluster_sync();
    tc_fence_after();
    if (threadIdx.x == 0 && leader) {
        const uint32_t a = smem_u32(smem);
        const uint64_t adesc = sdesc_k_swizzled(a, 128), bdesc = sdesc_k_swizzled(a + kProbeA, 128);
        constexpr uint32_t idesc = idesc_mxf4_f32(256, 256);
        for (int64_t r = 0; r < reps; ++r)
#pragma unroll
            for (int kk = 0; kk < 4; ++kk)
                mma_mxf4_pair(d, adesc + uint64_t(2 * kk), bdesc + uint64_t(2 * kk), idesc, d + 256u, d + 272u,
                              (r > 0 || kk > 0) ? 1u : 0u);
        mma_commit_pair_mc(&bar, 0x3);
    }
    if (threadIdx.x == 0) mbar_wait_bounded(&bar, 0, hdr, kProbeWaitNs);
    tc_fence_before();
    __syncthreads();
    cluster_sync();  // neither CTA frees the pair's TMEM while the MMAs may run
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc_pair(d, 512);
    }
}

// 32-bit population counts: eight independent chains per thread, each step
// an XOR, a POPC and an add (the ALU has four times the POPC rate).
__global__ void __launch_bounds__(256) k_probe_popc(int64_t reps, uint32_t* sink) {
    uint32_t x[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) x[k] = (threadIdx.x + 1u) * 0x9E3779B1u + uint32_t(k);
    for (int64_t r = 0; r < reps; ++r)
#pragma unroll
        for (int k = 0; k < 8; ++k) x[k] += uint32_t(__popc(x[k] ^ (0x5bd1e995u * uint32_t(k + 1))));
    uint32_t s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += x[k];
    if (s == 0x12345678u) sink[threadIdx.x & 31] = s;  // keeps the chains live
}

}  // namespace

}  // namespace cs

using namespace cs;

extern "C" int cs_peak_probe(int path, int64_t reps, void* workspace_dev, double* rate) {
    CS_TRACE("cs_peak_probe");
    if (path < CS_PATH_POPC || path > CS_PATH_MMA4 || reps < 1 || reps > kProbeMaxReps || !workspace_dev ||
        (reinterpret_cast<uintptr_t>(workspace_dev) % 256) != 0 || !rate)
        return CS_EINVAL;
    if (path != CS_PATH_POPC && !device_has_tcgen05()) return CS_EUNSUPPORTED;
    WsHeader* hdr = static_cast<WsHeader*>(workspace_dev);
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t err = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (err == cudaSuccess) err = cudaEventCreate(&e0);
    if (err == cudaSuccess) err = cudaEventCreate(&e1);
    if (err == cudaSuccess) err = cudaMemsetAsync(&hdr->status, 0, sizeof(int32_t), st);
    const int sms = device_sm_count();
    double ops = 0.0;
    if (err == cudaSuccess) err = cudaEventRecord(e0, st);
    if (err == cudaSuccess) {
        if (path == CS_PATH_POPC) {
            const int blocks = sms * 8;
            k_probe_popc<<<blocks, 256, 0, st>>>(reps, reinterpret_cast<uint32_t*>(hdr->aux));
            ops = double(blocks) * 256.0 * 8.0 * double(reps);
            err = cudaGetLastError();
        } else if (path == CS_PATH_MMA) {
            err = cudaFuncSetAttribute(k_probe_f8, cudaFuncAttributeMaxDynamicSharedMemorySize, kProbeSmem8);
            if (err == cudaSuccess) {
                k_probe_f8<<<sms, kProbeThreads, kProbeSmem8, st>>>(reps, hdr);
                err = cudaGetLastError();
            }
            ops = 2.0 * double(sms) * double(reps) * 4.0 * 128.0 * 256.0 * 32.0;
        } else {
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeClusterDimension;
            at[0].val.clusterDim.x = 2;
            at[0].val.clusterDim.y = 1;
            at[0].val.clusterDim.z = 1;
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(unsigned(sms / 2 * 2));
            cfg.blockDim = dim3(kProbeThreads);
            cfg.dynamicSmemBytes = kProbeSmem4;
            cfg.stream = st;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            int clusters = 0;
            err = cudaFuncSetAttribute(k_probe_f4_pair, cudaFuncAttributeMaxDynamicSharedMemorySize, kProbeSmem4);
            if (err == cudaSuccess) err = cudaOccupancyMaxActiveClusters(&clusters, k_probe_f4_pair, &cfg);
            if (err == cudaSuccess && clusters < 1) err = cudaErrorNotSupported;
            if (err == cudaSuccess) {
                // one pair per two SMs, all of them resident at once
                if (clusters > sms / 2) clusters = sms / 2;
                cfg.gridDim = dim3(unsigned(2 * clusters));
                err = cudaLaunchKernelEx(&cfg, k_probe_f4_pair, reps, hdr);
            }
            ops = 2.0 * double(clusters) * double(reps) * 4.0 * 256.0 * 256.0 * 64.0;
        }
    }
    if (err == cudaSuccess) err = cudaEventRecord(e1, st);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    int32_t status = 0;
    if (err == cudaSuccess)
        err = cudaMemcpy(&status, &hdr->status, sizeof(status), cudaMemcpyDeviceToHost);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (err != cudaSuccess) return CS_ECUDA;
    if (status != 0) return status;
    *rate = ops / (double(ms) * 1e-3);
    return CS_OK;
}
