// cs_count_popc.cu -- interval abundances with AND + popcount tiles on the
// CUDA cores (Algorithm "Optimized Interval Abundance Measurement", Figure
// "Proper distance and the order intervals").
//
// For time-sorted labels, row i of the symmetric bitset holds the future of i
// in columns > i and row j the past of j in columns < j, so for i < j
//     |A_ij| = popcount( F_i & P_j ),  F_i = row_i restricted to columns > i,
//                                      P_j = row_j restricted to columns < j,
// which is (C.C)_ij for the strict upper triangle C.  The kernel computes it
// for a 128 x 128 tile of pairs (i-block, j-block), i-block <= j-block, with
// the K loop running over the 64-bit words between the two blocks only.
//
// Data movement: one thread issues 2D TMA copies (cp.async.bulk.tensor) of a
// 128-row x 16-word slab of the i-block rows and of the j-block rows per
// K-chunk into a 3-stage ring of 128B-swizzled shared-memory buffers, with an
// mbarrier per stage.  Each of the 256 threads owns an 8 x 8 block of pairs
// (rows ti + 16a, columns tj + 16b), reads its 16 words per K-word from shared
// memory conflict-free and accumulates popc(f & p) in registers.  Only the
// chunks that overlap the i-block or j-block columns apply the per-row masks
// (bits <= i cleared in F, bits >= j cleared in P).
//
// Epilogue: a pair counts iff i < j < n and bit j of row i is set; its count k
// goes to a 8192-bin shared-memory histogram (global 64-bit atomics above
// that).  The kernel is persistent: CTAs pull tiles from a queue ordered by
// decreasing K length (largest first), and flush their shared histogram once.
#include <atomic>

#include "cs_kernels.cuh"

namespace cs {

namespace {

constexpr int kBT = 128;                     // rows per i-block / j-block
constexpr int kKW = 16;                      // 64-bit words per K-chunk (128-byte rows)
constexpr int kStages = 3;
constexpr int kThreads = 256;
constexpr int kTileBytes = kBT * kKW * 8;    // 16 KiB
constexpr int kStageBytes = 2 * kTileBytes;  // F slab + P slab
constexpr int kHistBins = 8192;
// A tile adds at most 128 x 128 to a shared bin, so flushing every 65536
// tiles keeps the 32-bit bins below 2^30 whatever the order (a bin could
// otherwise wrap on sets of more than about 10^6 elements whose pairs
// nearly all share one interval size).
constexpr uint32_t kFlushTiles = 65536;
constexpr int kSmemBytes = kStages * kStageBytes + kHistBins * 4 + kStages * 8 + 64 + 1024;

// Byte offset of word w of row r inside a [128][16] uint64 slab written by TMA
// with CU_TENSOR_MAP_SWIZZLE_128B: the 16-byte chunk index is XORed with r % 8.
__device__ __forceinline__ uint32_t swz(int r, int w) {
    return uint32_t(r) * 128u + (uint32_t((w >> 1) ^ (r & 7)) << 4) + (uint32_t(w & 1) << 3);
}

// Keep bits b > x of a word (columns strictly after row i: x = i - col0).
__device__ __forceinline__ uint64_t mask_after(int64_t x) {
    if (x < 0) return ~0ull;
    if (x >= 63) return 0ull;
    return ~0ull << (x + 1);
}

// Keep bits b < y of a word (columns strictly before row j: y = j - col0).
__device__ __forceinline__ uint64_t mask_before(int64_t y) {
    if (y <= 0) return 0ull;
    if (y >= 64) return ~0ull;
    return (1ull << y) - 1ull;
}

// Tile t of the queue -> (bi, bj).  Bands d = bj - bi are served from the
// widest (d = nb-1, one tile) to the diagonal (d = 0, nb tiles); band
// m = nb - d holds m tiles and is preceded by m(m-1)/2 tiles.
__device__ __forceinline__ void decode_tile(int64_t t, int64_t nb, int64_t& bi, int64_t& bj) {
    int64_t m = int64_t((1.0 + sqrt(1.0 + 8.0 * double(t))) * 0.5);
    while (m * (m - 1) / 2 > t) --m;
    while (m * (m + 1) / 2 <= t) ++m;
    bi = t - m * (m - 1) / 2;
    bj = bi + (nb - m);
}

template <bool kMask>
__device__ __forceinline__ void popc_chunk(const uint8_t* __restrict__ F, const uint8_t* __restrict__ P,
                                           uint32_t (&acc)[8][8], int ti, int tj, int64_t I0, int64_t J0,
                                           int64_t col0) {
#pragma unroll 2
    for (int w = 0; w < kKW; ++w) {
        uint64_t f[8], p[8];
#pragma unroll
        for (int a = 0; a < 8; ++a) f[a] = *reinterpret_cast<const uint64_t*>(F + swz(ti + 16 * a, w));
#pragma unroll
        for (int b = 0; b < 8; ++b) p[b] = *reinterpret_cast<const uint64_t*>(P + swz(tj + 16 * b, w));
        if (kMask) {
            const int64_t c = col0 + 64 * w;
#pragma unroll
            for (int a = 0; a < 8; ++a) f[a] &= mask_after(I0 + ti + 16 * a - c);
#pragma unroll
            for (int b = 0; b < 8; ++b) p[b] &= mask_before(J0 + tj + 16 * b - c);
        }
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int b = 0; b < 8; ++b) acc[a][b] += uint32_t(__popcll(f[a] & p[b]));
    }
}

// One causal set as the kernel sees it.
struct PopcView {
    const CUtensorMap* map;
    const uint64_t* bits;
    int64_t n, row_words, nb;
    unsigned long long* hist;
    int64_t hist_len;
    const double* phi;  // d'Alembertian field (NULL = 1)
    double* layer;      // layer sums [kmax+1][n], or NULL
    int kmax;           // < 0: no layer sums
};

// Work source: a single set passed in kernel parameters.
struct PopcSingle {
    PopcView v;
    int64_t ntiles;
    __device__ __forceinline__ int64_t total() const { return ntiles; }
    __device__ __forceinline__ int set_of(int64_t t, int64_t& local) const {
        local = t;
        return 0;
    }
    __device__ __forceinline__ PopcView view(int) const { return v; }
};

// Work source: many sets from a device table, items ordered set by set.
struct PopcMulti {
    const PopcSetEntry* sets;
    int nsets;
    int64_t ntiles;
    uintptr_t hist_base;
    __device__ __forceinline__ int64_t total() const { return ntiles; }
    __device__ __forceinline__ int set_of(int64_t t, int64_t& local) const {
        int lo = 0, hi = nsets - 1;  // last set with item_begin <= t
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (sets[mid].item_begin <= t) lo = mid; else hi = mid - 1;
        }
        local = t - sets[lo].item_begin + sets[lo].item_offset;
        return lo;
    }
    __device__ __forceinline__ PopcView view(int s) const {
        const PopcSetEntry& e = sets[s];
        return PopcView{&e.map, e.bits, e.n, e.row_words, e.nb,
                        reinterpret_cast<unsigned long long*>(hist_base + uintptr_t(e.hist_off)),
                        e.n > 1 ? e.n - 1 : 1, e.phi, e.layer, int(e.kmax)};
    }
};

// Add the shared histogram to the set's global histogram and clear it.
__device__ __forceinline__ void flush_hist(uint32_t* shist, const PopcView& v) {
    __syncthreads();
    const int64_t hb = v.hist_len < kHistBins ? v.hist_len : kHistBins;
    for (int64_t k = threadIdx.x; k < hb; k += kThreads) {
        const uint32_t c = shist[k];
        if (c) {
            atomicAdd(&v.hist[k], (unsigned long long)c);
            shist[k] = 0u;
        }
    }
    __syncthreads();
}

template <class Src>
__device__ __forceinline__ void popc_body(const Src& src, WsHeader* hdr) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint32_t* shist = reinterpret_cast<uint32_t*>(smem + kStages * kStageBytes);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(shist + kHistBins);
    int64_t* s_tile = reinterpret_cast<int64_t*>(mbar + kStages);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int tj = (lane & 7) + 8 * (warp >> 2);
    const int ti = (lane >> 3) + 4 * (warp & 3);

    for (int k = tid; k < kHistBins; k += kThreads) shist[k] = 0u;
    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&mbar[s], 1);
        fence_mbar_init();
    }
    __syncthreads();

    int cur = -1;  // set whose counts sit in the shared histogram
    PopcView v{};
    uint32_t seq = 0;  // K-chunks consumed so far by this CTA: stage = seq % S, parity = (seq / S) & 1
    uint32_t since_flush = 0;  // tiles counted into the shared histogram since its last flush
    bool aborted = false;
    for (;;) {
        if (tid == 0) *s_tile = int64_t(atomicAdd(&hdr->counter, 1ull));
        __syncthreads();
        const int64_t t = *s_tile;
        __syncthreads();
        if (t >= src.total()) break;

        int64_t local;
        const int sidx = src.set_of(t, local);
        if (sidx != cur || since_flush == kFlushTiles) {
            if (cur >= 0) flush_hist(shist, v);
            cur = sidx;
            v = src.view(sidx);
            since_flush = 0;
        }
        ++since_flush;
        const int64_t hb = v.hist_len < kHistBins ? v.hist_len : kHistBins;
        int64_t bi, bj;
        decode_tile(local, v.nb, bi, bj);
        const int64_t I0 = bi * kBT, J0 = bj * kBT;
        const int64_t wbeg = ((I0 >> 6) / kKW) * kKW;
        int64_t wend = (J0 + kBT + 63) >> 6;
        if (wend > v.row_words) wend = v.row_words;
        const int nch = int((wend - wbeg + kKW - 1) / kKW);

        if (tid == 0) {
            for (int c = 0; c < nch && c < kStages; ++c) {
                const int s = int((seq + c) % kStages);
                uint8_t* dst = smem + s * kStageBytes;
                mbar_arrive_expect_tx(&mbar[s], kStageBytes);
                tma_load_2d(dst, v.map, int32_t(wbeg + int64_t(c) * kKW), int32_t(I0), &mbar[s]);
                tma_load_2d(dst + kTileBytes, v.map, int32_t(wbeg + int64_t(c) * kKW), int32_t(J0), &mbar[s]);
            }
        }

        uint32_t acc[8][8];
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int b = 0; b < 8; ++b) acc[a][b] = 0u;

        for (int c = 0; c < nch; ++c) {
            const uint32_t g = seq + uint32_t(c);
            const int s = int(g % kStages);
            const bool ok = mbar_wait_bounded(&mbar[s], (g / kStages) & 1u, hdr);
            if (ok) {
                const uint8_t* F = smem + s * kStageBytes;
                const uint8_t* P = F + kTileBytes;
                const int64_t wc = wbeg + int64_t(c) * kKW;
                const bool need_mask = (wc * 64 <= I0 + kBT - 1) || ((wc + kKW) * 64 - 1 >= J0);
                if (need_mask)
                    popc_chunk<true>(F, P, acc, ti, tj, I0, J0, wc * 64);
                else
                    popc_chunk<false>(F, P, acc, ti, tj, I0, J0, wc * 64);
            }
            if (__syncthreads_or(!ok)) {
                // A copy never landed: wait (bounded) for the ones still in
                // flight so no TMA writes into freed shared memory, then stop.
                if (tid == 0)
                    for (int c2 = c; c2 < nch && c2 < c + kStages; ++c2) {
                        const uint32_t g2 = seq + uint32_t(c2);
                        mbar_wait_bounded(&mbar[g2 % kStages], (g2 / kStages) & 1u, hdr);
                    }
                aborted = true;
                break;
            }
            if (tid == 0 && c + kStages < nch) {
                uint8_t* dst = smem + s * kStageBytes;
                const int64_t wn = wbeg + int64_t(c + kStages) * kKW;
                mbar_arrive_expect_tx(&mbar[s], kStageBytes);
                tma_load_2d(dst, v.map, int32_t(wn), int32_t(I0), &mbar[s]);
                tma_load_2d(dst + kTileBytes, v.map, int32_t(wn), int32_t(J0), &mbar[s]);
            }
        }
        if (aborted) break;
        seq += uint32_t(nch);

#pragma unroll
        for (int a = 0; a < 8; ++a) {
            const int64_t i = I0 + ti + 16 * a;
            if (i >= v.n) continue;
            const uint64_t* row = v.bits + i * v.row_words;
#pragma unroll
            for (int b = 0; b < 8; ++b) {
                const int64_t j = J0 + tj + 16 * b;
                if (j <= i || j >= v.n) continue;
                if ((__ldg(row + (j >> 6)) >> (j & 63)) & 1ull) {
                    const uint32_t k = acc[a][b];
                    if (int64_t(k) < hb)
                        red_shared_add(smem_u32(shist) + 4u * k, 1u);
                    else
                        atomicAdd(&v.hist[k], 1ull);
                    if (int(k) <= v.kmax)  // i is in L_{k+1}(j)
                        atomicAdd(&v.layer[int64_t(k) * v.n + j], v.phi ? __ldg(v.phi + i) : 1.0);
                }
            }
        }
    }
    if (cur >= 0) flush_hist(shist, v);
}

__global__ void __launch_bounds__(kThreads, 1)
    k_count_popc(const __grid_constant__ CUtensorMap tmap, const uint64_t* __restrict__ bits, int64_t n,
                 int64_t row_words, int64_t nb, int64_t ntiles, unsigned long long* __restrict__ hist,
                 int64_t hist_len, const double* phi, double* layer, int kmax, WsHeader* hdr) {
    const PopcSingle src{PopcView{&tmap, bits, n, row_words, nb, hist, hist_len, phi, layer, kmax}, ntiles};
    popc_body(src, hdr);
}

__global__ void __launch_bounds__(kThreads, 1)
    k_count_popc_multi(const PopcSetEntry* __restrict__ sets, int nsets, int64_t ntiles, uintptr_t hist_base,
                       WsHeader* hdr) {
    const PopcMulti src{sets, nsets, ntiles, hist_base};
    popc_body(src, hdr);
}

std::atomic<bool> g_attr_set[64];  // per device: the large-shared-memory attribute is set
std::atomic<bool> g_attr_multi_set[64];

}  // namespace

int64_t popc_tiles(int64_t n) {
    const int64_t nb = (n + kBT - 1) / kBT;
    return nb * (nb + 1) / 2;
}

void popc_fill_entry(PopcSetEntry* e, const uint64_t* bits, int64_t n, int64_t row_words) {
    e->kmax = -1;
    e->bits = bits;
    e->n = n;
    e->row_words = row_words;
    e->nb = (n + kBT - 1) / kBT;
}

CUresult popc_encode_map(CUtensorMap* map, const uint64_t* bits, int64_t n, int64_t row_words) {
    return encode_tensor_map_2d(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, const_cast<uint64_t*>(bits),
                                uint64_t(row_words), uint64_t(n), uint64_t(row_words) * 8, kKW, kBT,
                                CU_TENSOR_MAP_SWIZZLE_128B);
}

cudaError_t launch_count_popc_multi(const PopcSetEntry* sets_dev, int nsets, int64_t ntiles, uintptr_t hist_base,
                                    WsHeader* hdr, int max_ctas, cudaStream_t st) {
    cudaError_t err = cudaMemsetAsync(&hdr->counter, 0, sizeof(hdr->counter), st);
    if (err != cudaSuccess) return err;
    if (ntiles < 1) return cudaSuccess;
    int dev = 0;
    if ((err = cudaGetDevice(&dev)) != cudaSuccess) return err;
    if (dev >= 0 && dev < 64 && !g_attr_multi_set[dev]) {
        err = cudaFuncSetAttribute(k_count_popc_multi, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
        if (err != cudaSuccess) return err;
        g_attr_multi_set[dev] = true;
    }
    int64_t grid = max_ctas > 0 ? max_ctas : device_sm_count();
    if (grid > ntiles) grid = ntiles;
    k_count_popc_multi<<<unsigned(grid), kThreads, kSmemBytes, st>>>(sets_dev, nsets, ntiles, hist_base, hdr);
    return cudaGetLastError();
}

size_t popc_workspace_bytes(int64_t) { return sizeof(WsHeader); }

cudaError_t launch_count_popc(int64_t n, const uint64_t* bits, int64_t row_words, int64_t* hist,
                              void* workspace, cudaStream_t st, const double* phi, double* layer, int kmax) {
    WsHeader* hdr = static_cast<WsHeader*>(workspace);
    const int64_t hist_len = n > 1 ? n - 1 : 1;
    cudaError_t err = cudaMemsetAsync(hist, 0, size_t(hist_len) * 8, st);
    if (err != cudaSuccess) return err;
    if ((err = cudaMemsetAsync(&hdr->counter, 0, sizeof(hdr->counter), st)) != cudaSuccess) return err;
    if (n < 2) return cudaSuccess;

    CUtensorMap map;
    if (encode_tensor_map_2d(&map, CU_TENSOR_MAP_DATA_TYPE_UINT64, const_cast<uint64_t*>(bits), uint64_t(row_words),
                             uint64_t(n), uint64_t(row_words) * 8, kKW, kBT, CU_TENSOR_MAP_SWIZZLE_128B) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;

    int dev = 0;
    if ((err = cudaGetDevice(&dev)) != cudaSuccess) return err;
    if (dev >= 0 && dev < 64 && !g_attr_set[dev]) {
        err = cudaFuncSetAttribute(k_count_popc, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBytes);
        if (err != cudaSuccess) return err;
        g_attr_set[dev] = true;
    }
    const int64_t nb = (n + kBT - 1) / kBT;
    const int64_t ntiles = nb * (nb + 1) / 2;
    int64_t grid = device_sm_count();
    if (grid > ntiles) grid = ntiles;
    k_count_popc<<<unsigned(grid), kThreads, kSmemBytes, st>>>(
        map, bits, n, row_words, nb, ntiles, reinterpret_cast<unsigned long long*>(hist), hist_len, phi, layer, kmax,
        hdr);
    return cudaGetLastError();
}

}  // namespace cs
