// cs_api.cu -- the extern "C" entry points of include/cs.h: argument
// validation, workspace bookkeeping and dispatch to the kernels.
#include <cstring>
#include <atomic>
#include <mutex>

#include "cs_kernels.cuh"

namespace cs {

// The last CUDA error an entry point turned into CS_ECUDA, per host thread.
thread_local cudaError_t t_last_cuda = cudaSuccess;

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return CS_OK;
    t_last_cuda = e;
    return CS_ECUDA;
}

namespace {

inline bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }


inline int from_cuda(cudaError_t e) { return cuda_status(e); }

inline bool valid_n(int64_t n) { return n >= 1 && n <= kMaxN; }

const double kZero = 0.0;

// Every call that owns a workspace first clears its status word, so the word
// always reports the last call that used the workspace.
inline cudaError_t clear_status(void* ws, cudaStream_t st) {
    return cudaMemsetAsync(&static_cast<WsHeader*>(ws)->status, 0, sizeof(int32_t), st);
}

}  // namespace

// CS_PATH_AUTO table: entry e applies from size n_min[e] up to the next
// entry.  The default follows GB300 measurements of random 2D orders: the
// FP8 tensor path beats POPC from n = 1024 (0.032 vs 0.042 ms), the FP4 pair
// path beats FP8 from n = 4096 (0.038 vs 0.044 ms; 12.1 vs 27.3 ms at
// 65536, 89.5 vs 224 ms at 131072); the autotuner replaces it with
// thresholds measured on the running device.
constexpr int kMaxAuto = 16;
std::mutex g_auto_mu;
int64_t g_auto_n[kMaxAuto] = {0, 1024, 4096};
int g_auto_p[kMaxAuto] = {CS_PATH_POPC, CS_PATH_MMA, CS_PATH_MMA4};
int g_auto_count = 3;

// Tile choices.  Raster side per size bucket of the single-set tensor
// counts (default 8 everywhere: a GB300 sweep of 4..16 found 8 best or
// within 1% from n = 2^15 to 2^17); the path CS_PATH_AUTO plans for batches
// and count jobs (0 = the default: FP4 pairs where the device has tcgen05,
// 9.8 vs 11.3 ms for the 768-set ensemble on GB300); the longest run of
// consecutive items a CTA takes from a multi-set queue.
constexpr int kMaxTiles = 16;
int64_t g_tile_n[kMaxTiles] = {0};
int g_tile_r[kMaxTiles] = {kRasterDefault};
int g_tile_count = 1;
std::atomic<int> g_batch_path{CS_PATH_AUTO};
std::atomic<int> g_max_run{16};

int auto_raster(int64_t n) {
    std::lock_guard<std::mutex> lk(g_auto_mu);
    int r = kRasterDefault;
    for (int e = 0; e < g_tile_count; ++e)
        if (n >= g_tile_n[e]) r = g_tile_r[e];
    return r;
}

int batch_auto_path() {
    const int p = g_batch_path.load(std::memory_order_relaxed);
    if (p != CS_PATH_AUTO) return (p == CS_PATH_POPC || device_has_tcgen05()) ? p : CS_PATH_POPC;
    return device_has_tcgen05() ? CS_PATH_MMA4 : CS_PATH_POPC;
}

int batch_max_run() { return g_max_run.load(std::memory_order_relaxed); }

// Device memory AUTO may plan for: the caller's limit, or 90% of the
// device's memory when none is set.
std::atomic<size_t> g_auto_mem_limit{0};

size_t auto_memory_limit() {
    const size_t lim = g_auto_mem_limit.load(std::memory_order_relaxed);
    return lim ? lim : device_total_memory() / 10 * 9;
}

// Memory the AUTO limit leaves for a count workspace beside the set's bitset.
size_t auto_workspace_room(int64_t n) {
    const size_t lim = auto_memory_limit(), bits = cs_bitset_bytes(n);
    return lim > bits ? lim - bits : 0;
}

// The FP4 path's workspace: the whole set's operands when they fit beside the
// bitset within the AUTO limit, else the widest bands of supertile rows that
// do (at least bands of one panel).
size_t mma4_planned_bytes(int64_t n) {
    const int64_t g = mma4_band_panels(n, auto_workspace_room(n));
    return mma4_band_bytes(n, g < 1 ? 1 : g);
}

// Bands narrower than this many supertile rows (or the whole set, if it has
// fewer) make AUTO take the POPC path: each band is one launch and one
// expansion of its rows, and narrow bands would spend more on those than the
// tensor cores save.
constexpr int64_t kMinBandPanels = 32;

// A tensor path fits when the set's bitset and the path's workspace together
// stay within the AUTO memory limit (FP4: bands of kMinBandPanels rows at
// least).  The rule reads the device's capacity, not its free memory, so that
// the workspace query and the count call that follows it (after the caller
// allocated that workspace) resolve alike.
bool tensor_fits(int64_t n, int p) {
    if (p == CS_PATH_MMA) return cs_bitset_bytes(n) + mma_workspace_bytes(n) <= auto_memory_limit();
    const int64_t nsb = (n + 255) / 256;
    return mma4_band_panels(n, auto_workspace_room(n)) >= (nsb < kMinBandPanels ? nsb : kMinBandPanels);
}

int resolve_path(int64_t n, int path) {
    if (path != CS_PATH_AUTO) return path;
    int p = CS_PATH_POPC;
    {
        std::lock_guard<std::mutex> lk(g_auto_mu);
        for (int e = 0; e < g_auto_count; ++e)
            if (n >= g_auto_n[e]) p = g_auto_p[e];
    }
    if ((p == CS_PATH_MMA || p == CS_PATH_MMA4) && !device_has_tcgen05()) return CS_PATH_POPC;
    // Too large for the table's tensor path: the FP4 path's smaller
    // workspace, else the POPC path, which needs no operands.
    if (p == CS_PATH_MMA && !tensor_fits(n, CS_PATH_MMA)) p = CS_PATH_MMA4;
    if (p == CS_PATH_MMA4 && !tensor_fits(n, CS_PATH_MMA4)) p = CS_PATH_POPC;
    return p;
}

}  // namespace cs

using namespace cs;

extern "C" {

int cs_dim(int kind) {
    if (kind == CS_2D_ORDER || kind == CS_2D_DIAMOND || kind == CS_2D_DS_SLAB || kind == CS_2D_SQUARE ||
        kind == CS_2D_CYLINDER)
        return 2;
    if (kind == CS_3D_DIAMOND) return 3;
    if (kind == CS_4D_DIAMOND) return 4;
    return 0;
}

size_t cs_coords_bytes(int kind, int64_t n) {
    const int d = cs_dim(kind);
    if (d == 0 || n < 0) return 0;
    return size_t(n) * size_t(d) * 4;
}

int64_t cs_row_words(int64_t n) {
    if (n < 0) return 0;
    const int64_t w = (n + 63) / 64;
    return (w + 15) / 16 * 16;
}

size_t cs_bitset_bytes(int64_t n) { return n < 0 ? 0 : size_t(n) * size_t(cs_row_words(n)) * 8; }

int64_t cs_hist_len(int64_t n) { return n > 1 ? n - 1 : 1; }

size_t cs_sprinkle_workspace_bytes(int kind, int64_t n) {
    if (cs_dim(kind) == 0 || !valid_n(n)) return 0;
    return sprinkle_workspace_bytes(n);
}

int cs_sprinkle(int kind, int64_t n, uint64_t seed, int32_t* coords_dev, void* workspace_dev, size_t workspace_bytes,
                void* stream) {
    CS_TRACE("cs_sprinkle");
    if (cs_dim(kind) == 0 || !valid_n(n) || !coords_dev || !aligned(coords_dev, 4) || !workspace_dev ||
        !aligned(workspace_dev, 256))
        return CS_EINVAL;
    if (workspace_bytes < sprinkle_workspace_bytes(n)) return CS_ENOMEM;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = clear_status(workspace_dev, st);
    if (e == cudaSuccess) e = launch_sprinkle(kind, n, seed, coords_dev, workspace_dev, st);
    return from_cuda(e);
}

int cs_causal_matrix(int kind, int64_t n, const int32_t* coords_dev, uint64_t* bits_dev, int64_t row_words,
                     void* stream) {
    CS_TRACE("cs_causal_matrix");
    if (cs_dim(kind) == 0 || !valid_n(n) || !coords_dev || !bits_dev || !aligned(bits_dev, 16) ||
        row_words < cs_row_words(n) || row_words % 16 != 0)
        return CS_EINVAL;
    return from_cuda(launch_relate(kind, n, coords_dev, bits_dev, row_words, static_cast<cudaStream_t>(stream)));
}

int cs_set_auto_paths(const int64_t* n_min, const int* paths, int count) {
    if (!n_min || !paths || count < 1 || count > kMaxAuto || n_min[0] != 0) return CS_EINVAL;
    for (int e = 0; e < count; ++e) {
        if (paths[e] != CS_PATH_POPC && paths[e] != CS_PATH_MMA && paths[e] != CS_PATH_MMA4) return CS_EINVAL;
        if (e > 0 && n_min[e] <= n_min[e - 1]) return CS_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_auto_mu);
    for (int e = 0; e < count; ++e) {
        g_auto_n[e] = n_min[e];
        g_auto_p[e] = paths[e];
    }
    g_auto_count = count;
    return CS_OK;
}

int cs_set_auto_tiles(const int64_t* n_min, const int* raster, int count) {
    if (!n_min || !raster || count < 1 || count > kMaxTiles || n_min[0] != 0) return CS_EINVAL;
    for (int e = 0; e < count; ++e) {
        if (raster[e] < 1 || raster[e] > 32) return CS_EINVAL;
        if (e > 0 && n_min[e] <= n_min[e - 1]) return CS_EINVAL;
    }
    std::lock_guard<std::mutex> lk(g_auto_mu);
    for (int e = 0; e < count; ++e) {
        g_tile_n[e] = n_min[e];
        g_tile_r[e] = raster[e];
    }
    g_tile_count = count;
    return CS_OK;
}

int cs_get_auto_tiles(int64_t* n_min, int* raster, int capacity) {
    std::lock_guard<std::mutex> lk(g_auto_mu);
    if (!n_min || !raster || capacity < g_tile_count) return g_tile_count;
    for (int e = 0; e < g_tile_count; ++e) {
        n_min[e] = g_tile_n[e];
        raster[e] = g_tile_r[e];
    }
    return g_tile_count;
}

int cs_set_batch_tuning(int path, int max_run) {
    if (path < CS_PATH_AUTO || path > CS_PATH_MMA4 || max_run < 1 || max_run > 64) return CS_EINVAL;
    g_batch_path.store(path, std::memory_order_relaxed);
    g_max_run.store(max_run, std::memory_order_relaxed);
    return CS_OK;
}

int cs_get_batch_tuning(int* path, int* max_run) {
    if (!path || !max_run) return CS_EINVAL;
    *path = g_batch_path.load(std::memory_order_relaxed);
    *max_run = g_max_run.load(std::memory_order_relaxed);
    return CS_OK;
}

int cs_set_auto_memory_limit(size_t bytes) {
    g_auto_mem_limit.store(bytes, std::memory_order_relaxed);
    return CS_OK;
}

size_t cs_get_auto_memory_limit(void) { return auto_memory_limit(); }

int cs_get_auto_paths(int64_t* n_min, int* paths, int capacity) {
    std::lock_guard<std::mutex> lk(g_auto_mu);
    if (!n_min || !paths || capacity < g_auto_count) return g_auto_count;
    for (int e = 0; e < g_auto_count; ++e) {
        n_min[e] = g_auto_n[e];
        paths[e] = g_auto_p[e];
    }
    return g_auto_count;
}

int cs_resolved_path(int64_t n, int path) {
    if (!valid_n(n) || path < CS_PATH_AUTO || path > CS_PATH_MMA4) return -1;
    return resolve_path(n, path);
}

size_t cs_interval_abundance_workspace(int64_t n, int path) {
    if (!valid_n(n) || path < CS_PATH_AUTO || path > CS_PATH_MMA4) return 0;
    const int p = resolve_path(n, path);
    return p == CS_PATH_MMA ? mma_workspace_bytes(n) : p == CS_PATH_MMA4 ? mma4_planned_bytes(n)
                                                                          : popc_workspace_bytes(n);
}

int64_t cs_mma4_band_cover(int64_t n, int64_t panels, int raster, int64_t* counts_host) {
    if (!valid_n(n) || n > (int64_t(1) << 20) || panels < 1 || raster < 1 || raster > 32 || !counts_host) return -1;
    return mma4_band_cover(n, panels, raster, counts_host);
}

int64_t cs_mma4_band_panels(int64_t n, size_t workspace_bytes) {
    if (!valid_n(n)) return -1;
    return mma4_band_panels(n, workspace_bytes);
}

namespace {

// The least workspace a count runs with: the planned one, except on the FP4
// path, which takes narrower bands down to one panel.
size_t min_count_workspace(int64_t n, int path) {
    return resolve_path(n, path) == CS_PATH_MMA4 ? mma4_band_bytes(n, 1) : cs_interval_abundance_workspace(n, path);
}

// The count kernels of a resolved path.
cudaError_t launch_count(int p, int64_t n, const uint64_t* bits, int64_t row_words, int64_t* hist, void* ws,
                         size_t ws_bytes, cudaStream_t st, const double* phi = nullptr, double* layer = nullptr,
                         int kmax = -1) {
    if (p == CS_PATH_MMA) return launch_count_mma(n, bits, row_words, hist, ws, st, phi, layer, kmax);
    if (p == CS_PATH_MMA4) return launch_count_mma4(n, bits, row_words, hist, ws, ws_bytes, st, phi, layer, kmax);
    return launch_count_popc(n, bits, row_words, hist, ws, st, phi, layer, kmax);
}

}  // namespace

int cs_interval_abundance(int64_t n, const uint64_t* bits_dev, int64_t row_words, int64_t* hist_dev, int path,
                          void* workspace_dev, size_t workspace_bytes, void* stream) {
    CS_TRACE("cs_interval_abundance");
    if (!valid_n(n) || !bits_dev || !aligned(bits_dev, 128) || !hist_dev || !aligned(hist_dev, 8) ||
        row_words < cs_row_words(n) || row_words % 16 != 0 || !workspace_dev || !aligned(workspace_dev, 256) ||
        path < CS_PATH_AUTO || path > CS_PATH_MMA4)
        return CS_EINVAL;
    if (workspace_bytes < min_count_workspace(n, path)) return CS_ENOMEM;
    const int p = resolve_path(n, path);
    if ((p == CS_PATH_MMA || p == CS_PATH_MMA4) && !device_has_tcgen05()) return CS_EUNSUPPORTED;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (fault_injected(CS_FAULT_LAUNCH)) return CS_ECUDA;
    cudaError_t e = clear_status(workspace_dev, st);
    if (e == cudaSuccess) e = launch_count(p, n, bits_dev, row_words, hist_dev, workspace_dev, workspace_bytes, st);
    return from_cuda(e);
}

int cs_layer_sums(int64_t n, const uint64_t* bits_dev, int64_t row_words, int64_t* hist_dev, int path,
                  const double* phi_dev, int kmax, double* layer_dev, void* workspace_dev, size_t workspace_bytes,
                  void* stream) {
    CS_TRACE("cs_layer_sums");
    if (!valid_n(n) || !bits_dev || !aligned(bits_dev, 128) || !hist_dev || !aligned(hist_dev, 8) ||
        row_words < cs_row_words(n) || row_words % 16 != 0 || !workspace_dev || !aligned(workspace_dev, 256) ||
        path < CS_PATH_AUTO || path > CS_PATH_MMA4 || kmax < 0 || kmax > 15 || !layer_dev ||
        !aligned(layer_dev, 8) || (phi_dev && !aligned(phi_dev, 8)))
        return CS_EINVAL;
    if (workspace_bytes < min_count_workspace(n, path)) return CS_ENOMEM;
    const int p = resolve_path(n, path);
    if ((p == CS_PATH_MMA || p == CS_PATH_MMA4) && !device_has_tcgen05()) return CS_EUNSUPPORTED;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e = clear_status(workspace_dev, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(layer_dev, 0, size_t(kmax + 1) * size_t(n) * 8, st);
    if (e == cudaSuccess)
        e = launch_count(p, n, bits_dev, row_words, hist_dev, workspace_dev, workspace_bytes, st, phi_dev, layer_dev,
                         kmax);
    return from_cuda(e);
}

int cs_dalembertian(int dim, int64_t n, const double* phi_dev, const double* layer_dev, int kmax, double ell,
                    double* out_dev, void* stream) {
    CS_TRACE("cs_dalembertian");
    if (dim < 2 || dim > 4 || !valid_n(n) || !layer_dev || !out_dev || !(ell > 0.0) ||
        kmax < (dim == 4 ? 3 : 2))
        return CS_EINVAL;
    return from_cuda(launch_dalembertian(dim, n, phi_dev, layer_dev, ell, out_dev, static_cast<cudaStream_t>(stream)));
}

int cs_workspace_status(void* workspace_dev, void* stream) {
    if (!workspace_dev) return CS_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int32_t status = 0;
    if (cudaMemcpyAsync(&status, &static_cast<WsHeader*>(workspace_dev)->status, sizeof(status),
                        cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return CS_ECUDA;
    if (clear_status(workspace_dev, st) != cudaSuccess) return CS_ECUDA;
    return status;
}

int cs_action(int dim, int64_t n, const int64_t* hist_host, int64_t len, double eps, double* out,
              int64_t* bracket_out) {
    return action_host(dim, n, hist_host, len, eps, out, bracket_out);
}

size_t cs_action_workspace_bytes(void) { return action_workspace_bytes(); }

int cs_action_device(int dim, int64_t n, const int64_t* hist_dev, int64_t len, const double* eps_host, int n_eps,
                     double* out_dev, int64_t* bracket_dev, void* workspace_dev, size_t workspace_bytes,
                     void* stream) {
    CS_TRACE("cs_action_device");
    if (dim < 2 || dim > 4 || n < 0 || len < 1 || !hist_dev || !eps_host || n_eps < 1 || n_eps > 16 ||
        !out_dev || !workspace_dev || !aligned(workspace_dev, 256))
        return CS_EINVAL;
    for (int e = 0; e < n_eps; ++e)
        if (!(eps_host[e] <= 1.0)) return CS_EINVAL;
    if (workspace_bytes < action_workspace_bytes()) return CS_ENOMEM;
    return from_cuda(launch_action_device(dim, n, hist_dev, len, eps_host, n_eps, out_dev, bracket_dev,
                                          workspace_dev, static_cast<cudaStream_t>(stream)));
}

int cs_evaluate(int kind, int64_t n, uint64_t seed, const int32_t* coords_host, int path, const double* eps_host,
                int n_eps, int64_t* hist_host, double* actions_host, int64_t* bracket_host, void* stream) {
    CS_TRACE("cs_evaluate");
    const int dim = cs_dim(kind);
    if (dim == 0 || !valid_n(n) || n_eps < 0 || n_eps > 16 || (n_eps > 0 && (!eps_host || !actions_host)) ||
        path < CS_PATH_AUTO || path > CS_PATH_MMA4)
        return CS_EINVAL;
    for (int e = 0; e < n_eps; ++e)
        if (!(eps_host[e] <= 1.0)) return CS_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);

    // Keep freed blocks in the device's stream-ordered pool between calls.
    static std::atomic<bool> pool_set[64];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CS_ECUDA;
    if (dev >= 0 && dev < 64 && !pool_set[dev].load(std::memory_order_acquire)) {
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t keep = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);  // idempotent
        }
        pool_set[dev].store(true, std::memory_order_release);
    }

    const int64_t rw = cs_row_words(n);
    const int64_t hl = cs_hist_len(n);
    size_t ws_bytes = cs_interval_abundance_workspace(n, path);
    if (cs_sprinkle_workspace_bytes(kind, n) > ws_bytes) ws_bytes = cs_sprinkle_workspace_bytes(kind, n);
    if (action_workspace_bytes() > ws_bytes) ws_bytes = action_workspace_bytes();

    int32_t* coords = nullptr;
    uint64_t* bits = nullptr;
    int64_t* hist = nullptr;
    void* ws = nullptr;
    double* out = nullptr;  // [16] actions, then the bracket as int64
    int rc = CS_OK;
    auto alloc = [&](void** p, size_t b) {
        if (rc == CS_OK && (fault_injected(CS_FAULT_ALLOC) || cudaMallocAsync(p, b, st) != cudaSuccess))
            rc = CS_ENOMEM;
    };
    alloc(reinterpret_cast<void**>(&coords), cs_coords_bytes(kind, n));
    alloc(reinterpret_cast<void**>(&bits), cs_bitset_bytes(n));
    alloc(reinterpret_cast<void**>(&hist), size_t(hl) * 8);
    alloc(&ws, ws_bytes);
    alloc(reinterpret_cast<void**>(&out), 17 * 8);
    int64_t* bracket = reinterpret_cast<int64_t*>(out + 16);

    if (rc == CS_OK) {
        if (coords_host)
            rc = from_cuda(cudaMemcpyAsync(coords, coords_host, cs_coords_bytes(kind, n), cudaMemcpyHostToDevice, st));
        else
            rc = cs_sprinkle(kind, n, seed, coords, ws, ws_bytes, st);
    }
    int32_t status_sprinkle = 0;
    if (rc == CS_OK && !coords_host)
        rc = from_cuda(cudaMemcpyAsync(&status_sprinkle, &static_cast<WsHeader*>(ws)->status, sizeof(int32_t),
                                       cudaMemcpyDeviceToHost, st));
    if (rc == CS_OK) rc = cs_causal_matrix(kind, n, coords, bits, rw, st);
    if (rc == CS_OK) rc = cs_interval_abundance(n, bits, rw, hist, path, ws, ws_bytes, st);
    int32_t status = 0;
    if (rc == CS_OK)
        rc = from_cuda(cudaMemcpyAsync(&status, &static_cast<WsHeader*>(ws)->status, sizeof(status),
                                       cudaMemcpyDeviceToHost, st));
    if (rc == CS_OK && n_eps > 0) {
        rc = cs_action_device(dim, n, hist, hl, eps_host, n_eps, out, bracket, ws, ws_bytes, st);
        if (rc == CS_OK)
            rc = from_cuda(cudaMemcpyAsync(actions_host, out, size_t(n_eps) * 8, cudaMemcpyDeviceToHost, st));
    }
    if (rc == CS_OK && bracket_host) {
        if (n_eps == 0) rc = cs_action_device(dim, n, hist, hl, eps_host ? eps_host : &kZero, 1, out, bracket, ws,
                                              ws_bytes, st);
        if (rc == CS_OK) rc = from_cuda(cudaMemcpyAsync(bracket_host, bracket, 8, cudaMemcpyDeviceToHost, st));
    }
    if (rc == CS_OK && hist_host)
        rc = from_cuda(cudaMemcpyAsync(hist_host, hist, size_t(hl) * 8, cudaMemcpyDeviceToHost, st));
    if (coords) cudaFreeAsync(coords, st);
    if (bits) cudaFreeAsync(bits, st);
    if (hist) cudaFreeAsync(hist, st);
    if (ws) cudaFreeAsync(ws, st);
    if (out) cudaFreeAsync(out, st);
    if (cudaStreamSynchronize(st) != cudaSuccess && rc == CS_OK) rc = CS_ECUDA;
    // Freed blocks stay in the pool for the next call, except after a call
    // that took more than a quarter of the device: those go back at once, so
    // one very large evaluation does not hold its memory for the process.
    const size_t took = cs_coords_bytes(kind, n) + cs_bitset_bytes(n) + size_t(hl) * 8 + ws_bytes;
    if (took > device_total_memory() / 4) {
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) cudaMemPoolTrimTo(pool, 0);
    }
    if (rc == CS_OK && status_sprinkle != 0) rc = status_sprinkle;
    if (rc == CS_OK && status != 0) rc = status;
    return rc;
}

const char* cs_strerror(int status) {
    switch (status) {
        case CS_OK: return "ok";
        case CS_EINVAL: return "invalid argument";
        case CS_ENOMEM: return "workspace too small or out of memory";
        case CS_ECUDA: return "CUDA error";
        case CS_ETIMEOUT: return "bounded in-kernel wait timed out";
        case CS_EUNSUPPORTED: return "unsupported on this device";
        case CS_ERANGE: return "sampler exhausted its attempt budget";
        case CS_PENDING: return "pending: the polled work has not finished";
        default: return "unknown status";
    }
}

const char* cs_version(void) { return "causet-gb300 0.1 (sm_103a)"; }

const char* cs_last_cuda_error(void) {
    return t_last_cuda == cudaSuccess ? "no error" : cudaGetErrorString(t_last_cuda);
}

}  // extern "C"
