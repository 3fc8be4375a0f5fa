// cs_sprinkle.cu -- sprinkling on the device (Section "Coordinate Generation",
// Appendix "Causal Set Sprinklings": 1+1, 2+1 and 3+1 Minkowski diamonds and
// the 1+1 de Sitter slab of Section "Spacetime Region Considered").
//
// Coordinates are drawn independently per element from the counter-based
// generator, then elements are sorted by time (Section "Pairwise
// Relations").  The sort is an exact ranking: every element gets
// rank = #{f : (key_f, f) < (key_e, e)}.  Keys are bucketed on their top 16
// bits (a counting pass, a scan, a fill), and each element compares itself
// only with its bucket -- O(n + 65536) work for the hashed / uniform keys used
// here, and the same ranks for any bucket fill order.
#include <atomic>
#include <cmath>
#include <mutex>
#include <vector>

#include "cs_kernels.cuh"
#include "cs_sprinkle.cuh"

namespace cs {

namespace {

constexpr int kMaxDevices = 64;

// Cumulative sec^2 mass of the slab up to the end of each eta cell, scaled to
// 2^53.  With unit = 2 pi / 2^20 and t0 = tan((G + 1/2) unit), cell g ends
// at x_g = (tan((g + 1/2) unit) + t0) / (2 t0) (the density sec^2(eta) /
// (2 tan eta_0) integrated from -eta_0); this exact expression, in double
// with the C library's tan, is part of the generator's definition, so the
// table is built on the host.
static __device__ uint64_t g_ds_thresholds[kDsTable];
std::atomic<const uint64_t*> g_ds_ptr[kMaxDevices];
std::mutex g_ds_mu;

std::vector<uint64_t> ds_thresholds_host() {
    std::vector<uint64_t> t(kDsTable);
    const double unit = 2.0 * 3.14159265358979323846 / 1048576.0;
    const double t0 = std::tan((double(kDsCells) + 0.5) * unit);
    for (int i = 0; i < kDsTable; ++i) {
        const double g = double(i - kDsCells);
        const double x = (std::tan((g + 0.5) * unit) + t0) / (2.0 * t0);
        t[i] = static_cast<uint64_t>(x * 9007199254740992.0);  // x * 2^53
    }
    return t;
}

__global__ void k_keys_ds_slab(int64_t n, uint64_t seed, const uint64_t* __restrict__ thr,
                               int32_t* __restrict__ raw, uint64_t* __restrict__ key) {
    const uint64_t s = stream_key(seed, kStreamDeSitter);
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x)
        key[e] = draw_ds_slab(s, e, thr, raw[e], raw[n + e]);
}

constexpr int kBucketBits = 16;
constexpr int kBuckets = 1 << kBucketBits;
constexpr int kThreads = 256;

__global__ void k_keys_2d_order(int64_t n, uint64_t seed, uint64_t* __restrict__ key_u,
                                uint64_t* __restrict__ key_v) {
    const uint64_t su = stream_key(seed, kStreamOrderU), sv = stream_key(seed, kStreamOrderV);
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x)
        draw_2d_order(su, sv, e, key_u[e], key_v[e]);
}

__global__ void k_keys_2d_diamond(int64_t n, uint64_t seed, int32_t* __restrict__ raw,
                                  uint64_t* __restrict__ key) {
    const uint64_t s = stream_key(seed, kStreamDiamond2);
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x)
        key[e] = draw_2d_diamond(s, e, raw[e], raw[n + e]);
}

__global__ void k_keys_2d_square(int64_t n, uint64_t seed, int32_t* __restrict__ raw, uint64_t* __restrict__ key) {
    const uint64_t s = stream_key(seed, kStreamSquare);
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x)
        key[e] = draw_2d_square(s, e, raw[e], raw[n + e]);
}

__global__ void k_keys_2d_cylinder(int64_t n, uint64_t seed, int32_t* __restrict__ raw,
                                   uint64_t* __restrict__ key) {
    const uint64_t s = stream_key(seed, kStreamCylinder);
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x)
        key[e] = draw_2d_cylinder(s, e, raw[e], raw[n + e]);
}

template <int D>
__global__ void k_keys_diamond(int64_t n, uint64_t seed, int32_t* __restrict__ raw, uint64_t* __restrict__ key,
                               WsHeader* hdr) {
    const uint64_t s = stream_key(seed, D == 4 ? kStreamDiamond4 : kStreamDiamond3);
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x) {
        int32_t c[4];
        if (!draw_diamond<D>(s, e, c, key[e])) set_status(hdr, CS_ERANGE);
#pragma unroll
        for (int k = 0; k < D; ++k) raw[k * n + e] = c[k];
    }
}

__global__ void k_bucket_count(int64_t n, const uint64_t* __restrict__ key, uint32_t* __restrict__ count) {
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x)
        atomicAdd(&count[key[e] >> (64 - kBucketBits)], 1u);
}

// Exclusive scan of the bucket counts (one block of 1024 threads, 64 buckets
// each); start[b] = first slot of bucket b, start[kBuckets] = n.  The counts
// are turned into fill cursors (= start) for k_bucket_fill.
__global__ void __launch_bounds__(1024) k_bucket_scan(uint32_t* __restrict__ count, uint32_t* __restrict__ start) {
    constexpr int per = kBuckets / 1024;
    __shared__ uint32_t part[1024];
    const int t = threadIdx.x;
    uint32_t local[per];
    uint32_t sum = 0;
#pragma unroll
    for (int k = 0; k < per; ++k) {
        local[k] = count[t * per + k];
        sum += local[k];
    }
    part[t] = sum;
    __syncthreads();
    for (int off = 1; off < 1024; off <<= 1) {  // Hillis-Steele inclusive scan
        uint32_t v = t >= off ? part[t - off] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    uint32_t run = part[t] - sum;
#pragma unroll
    for (int k = 0; k < per; ++k) {
        start[t * per + k] = run;
        count[t * per + k] = run;  // becomes the fill cursor
        run += local[k];
    }
    if (t == 1023) start[kBuckets] = run;
}

__global__ void k_bucket_fill(int64_t n, const uint64_t* __restrict__ key, uint32_t* __restrict__ cursor,
                              uint32_t* __restrict__ slot) {
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x) {
        const uint32_t pos = atomicAdd(&cursor[key[e] >> (64 - kBucketBits)], 1u);
        slot[pos] = uint32_t(e);
    }
}

__global__ void k_bucket_rank(int64_t n, const uint64_t* __restrict__ key, const uint32_t* __restrict__ start,
                              const uint32_t* __restrict__ slot, uint32_t* __restrict__ rank) {
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x) {
        const uint64_t ke = key[e];
        const uint32_t b = uint32_t(ke >> (64 - kBucketBits));
        uint32_t r = start[b];
        for (uint32_t p = start[b]; p < start[b + 1]; ++p) {
            const uint32_t f = slot[p];
            const uint64_t kf = key[f];
            r += (kf < ke) || (kf == ke && f < uint32_t(e));
        }
        rank[e] = r;
    }
}

__global__ void k_scatter_2d_order(int64_t n, const uint32_t* __restrict__ ru, const uint32_t* __restrict__ rv,
                                   int32_t* __restrict__ coords) {
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x) {
        const uint32_t r = ru[e];
        coords[r] = int32_t(r);
        coords[n + r] = int32_t(rv[e]);
    }
}

__global__ void k_scatter_raw(int64_t n, int dim, const uint32_t* __restrict__ rank, const int32_t* __restrict__ raw,
                              int32_t* __restrict__ coords) {
    for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x) {
        const uint32_t r = rank[e];
        for (int c = 0; c < dim; ++c) coords[c * n + r] = raw[c * n + e];
    }
}

struct SprinkleLayout {
    size_t key0, key1, raw, rank0, rank1, slot, count, start, total;
};

SprinkleLayout sprinkle_layout(int64_t n) {
    SprinkleLayout L;
    size_t off = sizeof(WsHeader);
    auto take = [&](size_t bytes) {
        size_t at = off;
        off = align_up(off + bytes, 256);
        return at;
    };
    const size_t un = size_t(n);
    L.key0 = take(un * 8);
    L.key1 = take(un * 8);
    L.raw = take(un * 16);
    L.rank0 = take(un * 4);
    L.rank1 = take(un * 4);
    L.slot = take(un * 4);
    L.count = take(size_t(kBuckets) * 4);
    L.start = take(size_t(kBuckets + 1) * 4);
    L.total = off;
    return L;
}

int grid_for(int64_t n) {
    int64_t b = (n + kThreads - 1) / kThreads;
    if (b < 1) b = 1;
    if (b > int64_t(device_sm_count()) * 16) b = int64_t(device_sm_count()) * 16;
    return int(b);
}

// Exact rank of each key with ties broken by index.
cudaError_t rank_keys(int64_t n, const uint64_t* key, uint32_t* rank, uint8_t* ws, const SprinkleLayout& L,
                      cudaStream_t st) {
    uint32_t* count = reinterpret_cast<uint32_t*>(ws + L.count);
    uint32_t* start = reinterpret_cast<uint32_t*>(ws + L.start);
    uint32_t* slot = reinterpret_cast<uint32_t*>(ws + L.slot);
    cudaError_t err = cudaMemsetAsync(count, 0, size_t(kBuckets) * 4, st);
    if (err != cudaSuccess) return err;
    const int g = grid_for(n);
    k_bucket_count<<<g, kThreads, 0, st>>>(n, key, count);
    k_bucket_scan<<<1, 1024, 0, st>>>(count, start);
    k_bucket_fill<<<g, kThreads, 0, st>>>(n, key, count, slot);
    k_bucket_rank<<<g, kThreads, 0, st>>>(n, key, start, slot, rank);
    return cudaGetLastError();
}

}  // namespace

const uint64_t* ds_table_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    if (const uint64_t* p = g_ds_ptr[dev].load(std::memory_order_acquire)) return p;
    // Upload under the lock; the pointer is published only after a
    // successful upload, so a failed first attempt (e.g. made during stream
    // capture, where the synchronous copy is not allowed) is retried by the
    // next call instead of disabling the kind for the process.
    std::lock_guard<std::mutex> lk(g_ds_mu);
    if (const uint64_t* p = g_ds_ptr[dev].load(std::memory_order_acquire)) return p;
    static const std::vector<uint64_t> host = ds_thresholds_host();
    void* p = nullptr;
    if (cudaMemcpyToSymbol(g_ds_thresholds, host.data(), host.size() * sizeof(uint64_t)) != cudaSuccess ||
        cudaGetSymbolAddress(&p, g_ds_thresholds) != cudaSuccess) {
        cudaGetLastError();  // not sticky: clear it for the caller's next call
        return nullptr;
    }
    g_ds_ptr[dev].store(static_cast<const uint64_t*>(p), std::memory_order_release);
    return static_cast<const uint64_t*>(p);
}

size_t sprinkle_workspace_bytes(int64_t n) { return sprinkle_layout(n).total; }

cudaError_t launch_sprinkle(int kind, int64_t n, uint64_t seed, int32_t* coords, void* workspace,
                            cudaStream_t st) {
    const SprinkleLayout L = sprinkle_layout(n);
    uint8_t* ws = static_cast<uint8_t*>(workspace);
    WsHeader* hdr = reinterpret_cast<WsHeader*>(ws);
    uint64_t* key0 = reinterpret_cast<uint64_t*>(ws + L.key0);
    uint64_t* key1 = reinterpret_cast<uint64_t*>(ws + L.key1);
    int32_t* raw = reinterpret_cast<int32_t*>(ws + L.raw);
    uint32_t* rank0 = reinterpret_cast<uint32_t*>(ws + L.rank0);
    uint32_t* rank1 = reinterpret_cast<uint32_t*>(ws + L.rank1);
    const int g = grid_for(n);
    cudaError_t err;
    if (kind == CS_2D_ORDER) {
        k_keys_2d_order<<<g, kThreads, 0, st>>>(n, seed, key0, key1);
        if ((err = rank_keys(n, key0, rank0, ws, L, st)) != cudaSuccess) return err;
        if ((err = rank_keys(n, key1, rank1, ws, L, st)) != cudaSuccess) return err;
        k_scatter_2d_order<<<g, kThreads, 0, st>>>(n, rank0, rank1, coords);
        return cudaGetLastError();
    }
    if (kind == CS_2D_DIAMOND) {
        k_keys_2d_diamond<<<g, kThreads, 0, st>>>(n, seed, raw, key0);
    } else if (kind == CS_2D_SQUARE) {
        k_keys_2d_square<<<g, kThreads, 0, st>>>(n, seed, raw, key0);
    } else if (kind == CS_2D_CYLINDER) {
        k_keys_2d_cylinder<<<g, kThreads, 0, st>>>(n, seed, raw, key0);
    } else if (kind == CS_2D_DS_SLAB) {
        const uint64_t* thr = ds_table_device();
        if (!thr) return cudaErrorInvalidValue;
        k_keys_ds_slab<<<g, kThreads, 0, st>>>(n, seed, thr, raw, key0);
    } else if (kind == CS_3D_DIAMOND) {
        k_keys_diamond<3><<<g, kThreads, 0, st>>>(n, seed, raw, key0, hdr);
    } else {
        k_keys_diamond<4><<<g, kThreads, 0, st>>>(n, seed, raw, key0, hdr);
    }
    if ((err = rank_keys(n, key0, rank0, ws, L, st)) != cudaSuccess) return err;
    k_scatter_raw<<<g, kThreads, 0, st>>>(n, cs_dim(kind), rank0, raw, coords);
    return cudaGetLastError();
}

}  // namespace cs
