// cs_sparse.cu -- degree vectors and sparse relation lists from the bitset
// (Section "Optimized GPU Linking Algorithm": the in- and out-degree vectors,
// and the relation list decoded into past and future sparse lists).
//
// The thesis's linking kernel emits a list of related pairs and reduces the
// degrees with shared-memory trees and atomics, then sorts the list to build
// the past and future lists.  Here the causal matrix is already a symmetric
// bitset with time-sorted labels, so both come from row scans: the future
// list of i is the set bits of row i above column i, the past list the set
// bits below it.  One warp owns a row: each lane loads one 64-bit word per
// step (coalesced) and popcounts give the degrees; for the lists, a warp
// scan of those popcounts places each word's columns, every lane writes its
// own word's columns into a shared-memory run in order, and the run leaves
// in coalesced stores.  The row offsets are an exclusive scan of the
// degrees (three small kernels).
#include "cs_kernels.cuh"

namespace cs {

namespace {

constexpr int kScanBlock = 1024;  // rows per block of the offset scan
constexpr int kScanThreads = 256;

struct SparseLayout {
    size_t deg, totals, total;
};

SparseLayout sparse_layout(int64_t n) {
    SparseLayout L;
    size_t off = sizeof(WsHeader);
    L.deg = off;
    off = align_up(off + size_t(n) * 8, 256);
    L.totals = off;
    off = align_up(off + size_t((n + kScanBlock - 1) / kScanBlock) * 8, 256);
    L.total = off;
    return L;
}

// Bits of word w of row i that lie after (future) or before (past) column i.
__device__ __forceinline__ uint64_t side_mask(int64_t i, int64_t w, bool future) {
    const int64_t wi = i >> 6;
    const int b = int(i & 63);
    if (future) {
        if (w > wi) return ~0ull;
        if (w < wi) return 0ull;
        return b == 63 ? 0ull : (~0ull << (b + 1));
    }
    if (w < wi) return ~0ull;
    if (w > wi) return 0ull;
    return b == 0 ? 0ull : ((1ull << b) - 1ull);
}

__device__ __forceinline__ int warp_sum(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(256) k_degrees(const uint64_t* __restrict__ bits, int64_t n, int64_t row_words,
                                                 int32_t* __restrict__ kin, int32_t* __restrict__ kout) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (n + 63) >> 6;
    const int64_t warps = int64_t(gridDim.x) * (blockDim.x >> 5);
    for (int64_t i = int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
        int past = 0, future = 0;
        for (int64_t w = lane; w < nw; w += 32) {
            const uint64_t x = __ldg(bits + i * row_words + w);
            past += __popcll(x & side_mask(i, w, false));
            future += __popcll(x & side_mask(i, w, true));
        }
        past = warp_sum(past);
        future = warp_sum(future);
        if (lane == 0) {
            if (kin) kin[i] = past;
            if (kout) kout[i] = future;
        }
    }
}

// Relations of each row on one side (the lengths of the sparse lists).
__global__ void __launch_bounds__(256) k_side_counts(const uint64_t* __restrict__ bits, int64_t n, int64_t row_words,
                                                     bool future, int64_t* __restrict__ deg) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = int64_t(gridDim.x) * (blockDim.x >> 5);
    for (int64_t i = int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
        const int64_t wi = i >> 6;
        const int64_t wlo = future ? wi : 0, whi = future ? (n + 63) >> 6 : wi + 1;
        int c = 0;
        for (int64_t w = wlo + lane; w < whi; w += 32)
            c += __popcll(__ldg(bits + i * row_words + w) & side_mask(i, w, future));
        c = warp_sum(c);
        if (lane == 0) deg[i] = c;
    }
}

// Exclusive scan of deg within blocks of kScanBlock rows; block sums to totals.
__global__ void __launch_bounds__(kScanThreads) k_scan_blocks(const int64_t* __restrict__ deg, int64_t n,
                                                              int64_t* __restrict__ out, int64_t* __restrict__ totals) {
    constexpr int kPer = kScanBlock / kScanThreads;
    __shared__ int64_t warp_tot[kScanThreads / 32];
    const int64_t base = int64_t(blockIdx.x) * kScanBlock + int64_t(threadIdx.x) * kPer;
    int64_t v[kPer], run = 0;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        v[k] = base + k < n ? deg[base + k] : 0;
        run += v[k];
    }
    // inclusive scan of the per-thread sums across the block
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t inc = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    int64_t before = 0;
    for (int w = 0; w < warp; ++w) before += warp_tot[w];
    int64_t pos = before + inc - run;  // exclusive prefix of this thread's first row
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        if (base + k < n) out[base + k] = pos;
        pos += v[k];
    }
    if (threadIdx.x == kScanThreads - 1) totals[blockIdx.x] = before + inc;
}

// Exclusive scan of the block totals (one block; at most 4096 of them).
__global__ void __launch_bounds__(kScanThreads) k_scan_totals(int64_t* __restrict__ totals, int64_t nb,
                                                              int64_t* __restrict__ grand) {
    __shared__ int64_t warp_tot[kScanThreads / 32];
    const int per = int((nb + kScanThreads - 1) / kScanThreads);
    const int64_t base = int64_t(threadIdx.x) * per;
    int64_t run = 0;
    for (int k = 0; k < per; ++k)
        if (base + k < nb) run += totals[base + k];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t inc = run;
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    int64_t before = 0;
    for (int w = 0; w < warp; ++w) before += warp_tot[w];
    int64_t pos = before + inc - run;
    for (int k = 0; k < per; ++k) {
        if (base + k < nb) {
            const int64_t t = totals[base + k];
            totals[base + k] = pos;
            pos += t;
        }
    }
    if (threadIdx.x == kScanThreads - 1) *grand = before + inc;
}

__global__ void k_scan_add(int64_t* __restrict__ out, int64_t n, const int64_t* __restrict__ totals) {
    for (int64_t r = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; r < n; r += int64_t(gridDim.x) * blockDim.x)
        out[r] += totals[r / kScanBlock];
}

// Column indices of each row's relations on one side, in increasing order,
// at cols[offsets[i] ..).  A row whose list would end past cols_capacity is
// skipped and CS_ENOMEM recorded.  The warp walks its row 32 words at a
// time, lane l owning word l: an inclusive warp scan of the words'
// popcounts gives each word's first place in the step's run, each lane
// writes its word's set columns (lowest bit first) into the warp's shared
// buffer there, and the warp copies the run out in coalesced stores.  (One
// lane per bit of each half-word in turn, with a popcount, a rank and a
// predicated store per half-word, held the integer pipe at three times the
// instructions per relation: 0.42 of the HBM rate at N = 2^17.)
constexpr int kColsWarps = 4;                      // warps per block
constexpr int kColsRun = 32 * 64 + 4;              // the most columns one step emits, and an alignment shift
__global__ void __launch_bounds__(kColsWarps * 32) k_side_columns(const uint64_t* __restrict__ bits, int64_t n,
                                                                   int64_t row_words, bool future,
                                                                   const int64_t* __restrict__ offsets,
                                                                   int32_t* __restrict__ cols,
                                                                   int64_t cols_capacity, WsHeader* hdr) {
    __shared__ __align__(16) int32_t stage[kColsWarps][kColsRun];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int32_t* run = stage[warp];
    const int64_t warps = int64_t(gridDim.x) * kColsWarps;
    for (int64_t i = int64_t(blockIdx.x) * kColsWarps + warp; i < n; i += warps) {
        const int64_t end = offsets[i + 1];
        if (end > cols_capacity || end < offsets[i]) {
            if (lane == 0) set_status(hdr, CS_ENOMEM);
            continue;
        }
        const int64_t wi = i >> 6;
        const int64_t wlo = future ? wi : 0, whi = future ? (n + 63) >> 6 : wi + 1;
        int64_t pos = offsets[i];
        const uint64_t* row = bits + i * row_words;
        uint64_t xn = wlo + lane < whi ? __ldg(row + wlo + lane) : 0ull;  // the next step's word, in flight
        for (int64_t w0 = wlo; w0 < whi; w0 += 32) {
            const int64_t w = w0 + lane;
            uint64_t x = w < whi ? xn & side_mask(i, w, future) : 0ull;
            xn = w + 32 < whi ? __ldg(row + w + 32) : 0ull;
            const int c = __popcll(x);
            int incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            // element k of the run goes to cols[pos + k] and to run[s0 + k],
            // s0 = that position's 4-byte slot in its 16-byte group, so the
            // run's 16-byte groups are the output's
            const int s0 = int((reinterpret_cast<uintptr_t>(cols + pos) >> 2) & 3);
            int at = s0 + incl - c;
            const int32_t base = int32_t(64 * w);  // n <= 2^22
            // lowest bit first, one 32-bit half at a time (cheaper steps than
            // 64-bit find-first and clear-lowest)
            for (uint32_t h = uint32_t(x); h; h &= h - 1u) run[at++] = base + (__ffs(int(h)) - 1);
            for (uint32_t h = uint32_t(x >> 32); h; h &= h - 1u) run[at++] = base + 31 + __ffs(int(h));
            __syncwarp();
            // a head up to the first 16-byte boundary, whole groups as
            // 16-byte stores, then a tail; positions at or past `end` are
            // skipped (only if the bitset changed since the offsets)
            const int h0 = (4 - s0) & 3;
            const int head = h0 < total ? h0 : total;
            const int groups = (total - head) >> 2;
            if (lane < head && pos + lane < end) cols[pos + lane] = run[s0 + lane];
            for (int g = lane; g < groups; g += 32) {
                const int k = head + 4 * g;
                const int4 v = *reinterpret_cast<const int4*>(run + s0 + k);
                if (pos + k + 3 < end) {
                    *reinterpret_cast<int4*>(cols + pos + k) = v;
                } else {
                    const int32_t e4[4] = {v.x, v.y, v.z, v.w};
                    for (int e = 0; e < 4; ++e)
                        if (pos + k + e < end) cols[pos + k + e] = e4[e];
                }
            }
            for (int k = head + 4 * groups + lane; k < total; k += 32)
                if (pos + k < end) cols[pos + k] = run[s0 + k];
            __syncwarp();
            pos += total;
        }
    }
}

int cols_grid(int64_t n) {
    int64_t g = (n + kColsWarps - 1) / kColsWarps;
    const int64_t cap = int64_t(device_sm_count()) * 32;
    return int(g < 1 ? 1 : (g > cap ? cap : g));
}

int row_grid(int64_t n) {
    int64_t g = (n + 7) / 8;  // 8 warps per block
    const int64_t cap = int64_t(device_sm_count()) * 16;
    return int(g < 1 ? 1 : (g > cap ? cap : g));
}

bool bits_ok(int64_t n, const uint64_t* bits, int64_t row_words) {
    return n >= 1 && n <= kMaxN && bits && (reinterpret_cast<uintptr_t>(bits) % 16) == 0 &&
           row_words >= cs_row_words(n) && row_words % 16 == 0;
}

}  // namespace

}  // namespace cs

using namespace cs;

extern "C" int cs_degrees(int64_t n, const uint64_t* bits_dev, int64_t row_words, int32_t* in_dev, int32_t* out_dev,
                          void* stream) {
    CS_TRACE("cs_degrees");
    if (!bits_ok(n, bits_dev, row_words) || (!in_dev && !out_dev)) return CS_EINVAL;
    k_degrees<<<row_grid(n), 256, 0, static_cast<cudaStream_t>(stream)>>>(bits_dev, n, row_words, in_dev, out_dev);
    return cudaGetLastError() == cudaSuccess ? CS_OK : CS_ECUDA;
}

extern "C" size_t cs_sparse_workspace_bytes(int64_t n) {
    if (n < 1 || n > kMaxN) return 0;
    return sparse_layout(n).total;
}

extern "C" int cs_sparse_offsets(int64_t n, const uint64_t* bits_dev, int64_t row_words, int direction,
                                 int64_t* offsets_dev, void* workspace_dev, size_t workspace_bytes, void* stream) {
    CS_TRACE("cs_sparse_offsets");
    if (!bits_ok(n, bits_dev, row_words) || (direction != 0 && direction != 1) || !offsets_dev ||
        (reinterpret_cast<uintptr_t>(offsets_dev) % 8) != 0 || !workspace_dev ||
        (reinterpret_cast<uintptr_t>(workspace_dev) % 256) != 0)
        return CS_EINVAL;
    const SparseLayout L = sparse_layout(n);
    if (workspace_bytes < L.total) return CS_ENOMEM;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint8_t* ws = static_cast<uint8_t*>(workspace_dev);
    int64_t* deg = reinterpret_cast<int64_t*>(ws + L.deg);
    int64_t* totals = reinterpret_cast<int64_t*>(ws + L.totals);
    const int64_t nb = (n + kScanBlock - 1) / kScanBlock;
    if (cudaMemsetAsync(&reinterpret_cast<WsHeader*>(ws)->status, 0, sizeof(int32_t), st) != cudaSuccess)
        return CS_ECUDA;
    k_side_counts<<<row_grid(n), 256, 0, st>>>(bits_dev, n, row_words, direction == 1, deg);
    k_scan_blocks<<<unsigned(nb), kScanThreads, 0, st>>>(deg, n, offsets_dev, totals);
    k_scan_totals<<<1, kScanThreads, 0, st>>>(totals, nb, offsets_dev + n);
    int64_t g = (n + 255) / 256;
    if (g > int64_t(device_sm_count()) * 8) g = int64_t(device_sm_count()) * 8;
    k_scan_add<<<unsigned(g), 256, 0, st>>>(offsets_dev, n, totals);
    return cudaGetLastError() == cudaSuccess ? CS_OK : CS_ECUDA;
}

extern "C" int cs_sparse_columns(int64_t n, const uint64_t* bits_dev, int64_t row_words, int direction,
                                 const int64_t* offsets_dev, int32_t* cols_dev, int64_t cols_capacity,
                                 void* workspace_dev, size_t workspace_bytes, void* stream) {
    CS_TRACE("cs_sparse_columns");
    if (!bits_ok(n, bits_dev, row_words) || (direction != 0 && direction != 1) || !offsets_dev ||
        (reinterpret_cast<uintptr_t>(offsets_dev) % 8) != 0 || cols_capacity < 0 || (cols_capacity > 0 && !cols_dev) ||
        !workspace_dev || (reinterpret_cast<uintptr_t>(workspace_dev) % 256) != 0 || workspace_bytes < sizeof(WsHeader))
        return CS_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    WsHeader* hdr = static_cast<WsHeader*>(workspace_dev);
    if (cudaMemsetAsync(&hdr->status, 0, sizeof(int32_t), st) != cudaSuccess) return CS_ECUDA;
    k_side_columns<<<cols_grid(n), kColsWarps * 32, 0, st>>>(bits_dev, n, row_words, direction == 1, offsets_dev, cols_dev,
                                               cols_capacity, hdr);
    return cudaGetLastError() == cudaSuccess ? CS_OK : CS_ECUDA;
}
