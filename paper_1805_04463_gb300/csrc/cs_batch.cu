// cs_batch.cu -- batched ensembles: many causal sets of different kinds and
// sizes evaluated by one fixed sequence of launches (memsets and kernels
// only, so the sequence can be captured into a CUDA graph and replayed).
//
// Pipeline per launch, every kernel covering all sets at once:
//   k_batch_keys    per element: random keys / raw coordinates (same draws as
//                   cs_sprinkle, so every set equals its single-set result);
//   k_batch_rank    one CTA per set: exact ranks of the keys by a bucket
//                   count in shared memory give the time order; scatter
//                   coordinates;
//   k_batch_relate  every relate chunk (32 words of a 64-row tile, from its
//                   diagonal word) of every bitset, one launch per geometry;
//   k_batch_mirror  the lower triangle of every bitset, the transpose of the
//                   upper one (the past rows);
//   count           the multi-set POPC kernel, or expand + multi-set tcgen05
//                   kernel: one persistent grid over the tiles of all sets,
//                   largest sets first (longest-processing-time order);
//   k_batch_action  one CTA per set: bracket and smeared sums.
// Ensembles of Poisson-sized sprinklings are the thesis's experimental unit
// (Section "Simulations and Scaling Evaluations": ten graphs per size; the
// appendix's sprinklings draw N from a Poisson distribution).
#include <algorithm>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "cs_action.cuh"
#include <atomic>

#include "cs_kernels.cuh"
#include "cs_relate.cuh"
#include "cs_sprinkle.cuh"

namespace cs {

namespace {

// Per set, device-resident.
struct BatchSet {
    int32_t kind, dim;
    int64_t n;
    uint64_t seed;
    int32_t* coords;
    uint64_t* bits;
    int64_t row_words;
    uint64_t* key0;
    uint64_t* key1;
    int32_t* raw;
    int64_t elem_begin;    // first element of this set in the concatenated element range
    int64_t rblock_begin;  // first relate block
    int64_t vwords;        // valid words per row = row tiles = ceil(n / 64)
    int64_t mblock_begin;  // first mirror block (lower part by symmetry)
    int64_t mir_side;      // mirror super-tiles per side
    int64_t hist_off;      // offset of this set's histogram in the batch histogram
    ConeTable* ctab;       // light-cone kinds: one column table per column tile (else null)
    int64_t tile_begin;    // first column tile of this set in the concatenated tile range
};

constexpr int kRankThreads = 1024;

__device__ __forceinline__ int find_set_elem(const BatchSet* sets, int nsets, int64_t idx) {
    int lo = 0, hi = nsets - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sets[mid].elem_begin <= idx) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(256) k_batch_keys(const BatchSet* __restrict__ sets, int nsets, int64_t total,
                                                    const uint64_t* __restrict__ ds_thr, WsHeader* hdr) {
    for (int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; idx < total;
         idx += int64_t(gridDim.x) * blockDim.x) {
        const BatchSet& b = sets[find_set_elem(sets, nsets, idx)];
        const int64_t e = idx - b.elem_begin;
        if (b.kind == CS_2D_ORDER) {
            draw_2d_order(stream_key(b.seed, kStreamOrderU), stream_key(b.seed, kStreamOrderV), e, b.key0[e],
                          b.key1[e]);
        } else if (b.kind == CS_2D_DIAMOND) {
            b.key0[e] = draw_2d_diamond(stream_key(b.seed, kStreamDiamond2), e, b.raw[e], b.raw[b.n + e]);
        } else if (b.kind == CS_2D_SQUARE) {
            b.key0[e] = draw_2d_square(stream_key(b.seed, kStreamSquare), e, b.raw[e], b.raw[b.n + e]);
        } else if (b.kind == CS_2D_CYLINDER) {
            b.key0[e] = draw_2d_cylinder(stream_key(b.seed, kStreamCylinder), e, b.raw[e], b.raw[b.n + e]);
        } else if (b.kind == CS_2D_DS_SLAB) {
            b.key0[e] = draw_ds_slab(stream_key(b.seed, kStreamDeSitter), e, ds_thr, b.raw[e], b.raw[b.n + e]);
        } else {
            int32_t c[4];
            const bool ok = b.kind == CS_3D_DIAMOND
                                ? draw_3d_diamond(stream_key(b.seed, kStreamDiamond3), e, c, b.key0[e])
                                : draw_4d_diamond(stream_key(b.seed, kStreamDiamond4), e, c, b.key0[e]);
            if (!ok) set_status(hdr, CS_ERANGE);
            for (int k = 0; k < b.dim; ++k) b.raw[k * b.n + e] = c[k];
        }
    }
}

// Exact ranks of a set's n keys (ties by index: the order "sorted by time,
// ties by generation index") in shared memory, O(n): count the keys into P
// buckets by their top log2(P) bits (P the power of two >= n; the keys are
// a time coordinate in the top bits, or random, so a bucket holds about
// one key and at most a few), an exclusive scan of the counts, fill the
// buckets, then rank each key within its bucket by comparison.  After the
// fill, cnt[b] is the end of bucket b and cnt[b - 1] its start.  (A bitonic
// sort of the (key, index) pairs, O(n log^2 n), took 0.38 ms for the
// 768-set ensemble.)  All kRankThreads threads; rank[e] receives the rank.
__device__ void rank_keys_smem(const uint64_t* __restrict__ src, int n, int lgP, uint64_t* sk, uint32_t* cnt,
                               uint32_t* slot, uint32_t* rank) {
    const int P = 1 << lgP, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int shift = 64 - lgP;
    for (int i = tid; i < n; i += kRankThreads) sk[i] = src[i];
    for (int i = tid; i < P; i += kRankThreads) cnt[i] = 0u;
    __syncthreads();
    for (int i = tid; i < n; i += kRankThreads) atomicAdd(&cnt[sk[i] >> shift], 1u);
    __syncthreads();
    // exclusive scan: each thread a run of P / kRankThreads buckets (P >= 1024
    // is ensured by the caller), warp and block offsets through shuffles
    const int per = P / kRankThreads;
    uint32_t run = 0;
    for (int k = 0; k < per; ++k) run += cnt[tid * per + k];
    uint32_t incl = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    __shared__ uint32_t wsum[kRankThreads / 32];
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < kRankThreads / 32 ? wsum[lane] : 0u, wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < kRankThreads / 32) wsum[lane] = wi - w;  // exclusive warp offsets
    }
    __syncthreads();
    uint32_t at = wsum[warp] + incl - run;
    for (int k = 0; k < per; ++k) {
        const uint32_t c = cnt[tid * per + k];
        cnt[tid * per + k] = at;  // start of the bucket, then its fill cursor
        at += c;
    }
    __syncthreads();
    for (int i = tid; i < n; i += kRankThreads) slot[atomicAdd(&cnt[sk[i] >> shift], 1u)] = uint32_t(i);
    __syncthreads();
    for (int i = tid; i < n; i += kRankThreads) {
        const uint64_t ke = sk[i];
        const uint32_t bk = uint32_t(ke >> shift);
        const uint32_t s0 = bk ? cnt[bk - 1] : 0u, s1 = cnt[bk];
        uint32_t r = s0;
        for (uint32_t q = s0; q < s1; ++q) {
            const uint32_t f = slot[q];
            const uint64_t kf = sk[f];
            r += (kf < ke) || (kf == ke && f < uint32_t(i));
        }
        rank[i] = r;
    }
    __syncthreads();
}

// One CTA per set: exact rank of each element (ties by index), then the
// time-sorted coordinates.  Shared memory: keys 8P, bucket cursors 4P,
// bucket slots 4P, ranks 4P (and the u ranks 4P of a 2D order): 24P bytes.
__global__ void __launch_bounds__(kRankThreads) k_batch_rank(const BatchSet* __restrict__ sets) {
    extern __shared__ uint8_t smem_raw[];
    const BatchSet& b = sets[blockIdx.x];
    const int n = int(b.n);
    int lgP = 10;  // at least kRankThreads buckets (the scan's runs)
    while ((1 << lgP) < n) ++lgP;
    const int P = 1 << lgP;
    uint64_t* sk = reinterpret_cast<uint64_t*>(smem_raw);
    uint32_t* cnt = reinterpret_cast<uint32_t*>(sk + P);
    uint32_t* slot = cnt + P;
    uint32_t* rank = slot + P;
    uint32_t* ru = rank + P;
    rank_keys_smem(b.key0, n, lgP, sk, cnt, slot, rank);
    if (b.kind == CS_2D_ORDER) {
        for (int e = threadIdx.x; e < n; e += kRankThreads) ru[e] = rank[e];  // u rank of element e
        __syncthreads();
        rank_keys_smem(b.key1, n, lgP, sk, cnt, slot, rank);
        for (int e = threadIdx.x; e < n; e += kRankThreads) {
            b.coords[ru[e]] = int32_t(ru[e]);
            b.coords[n + ru[e]] = int32_t(rank[e]);
        }
    } else {
        for (int e = threadIdx.x; e < n; e += kRankThreads) {
            const uint32_t p = rank[e];  // the time-sorted position of element e
            for (int c = 0; c < b.dim; ++c) b.coords[c * n + p] = b.raw[c * n + e];
        }
    }
}

// Column tables of the light-cone sets (after k_batch_rank has written the
// time-sorted coordinates), one warp per column tile of the concatenated
// tile range, the set read from a table built at create time.
__global__ void __launch_bounds__(256) k_batch_ctab(const BatchSet* __restrict__ sets,
                                                    const int32_t* __restrict__ tile_set, int64_t tiles) {
    const int64_t g = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;  // warp-uniform
    if (g >= tiles) return;
    const BatchSet& b = sets[tile_set[g]];
    if (b.ctab) build_cone_table(b.coords, b.n, g - b.tile_begin, b.kind == CS_2D_ORDER, b.ctab + (g - b.tile_begin));
}

// Relate chunks.  Row tile rb of a set with V valid words needs words
// [rb, V) (the words before it are mirrored); they are covered by
// ceil((V - rb) / 32) chunks of 32 words starting at the diagonal word, so
// no block holds words before its row tile or whole groups of padding.
// chunk_sum(x) = sum_{m=1..x} ceil(m / 32); the chunks of row tiles < rb
// number chunk_sum(V) - chunk_sum(V - rb).
__host__ __device__ __forceinline__ int64_t chunk_sum(int64_t x) {
    const int64_t a = x / kRelWordsPerBlock, b = x % kRelWordsPerBlock;
    return kRelWordsPerBlock * a * (a + 1) / 2 + b * (a + 1);
}

// Relation geometry of a kind.
__host__ __device__ __forceinline__ int batch_geom(int kind) {
    return kind == CS_4D_DIAMOND                               ? kGeom4
           : kind == CS_3D_DIAMOND                             ? kGeom3
           : (kind == CS_2D_DS_SLAB || kind == CS_2D_CYLINDER) ? kGeomDeSitter
                                                               : kGeomLightCone;
}

// Relate block `local` of a set: its row tile rb, first word w0 and, for a
// row tile's last chunk, the first padding word to zero (else -1).
__device__ __forceinline__ void decode_rblock(const BatchSet& b, int64_t local, int64_t& rb, int64_t& w0,
                                              int64_t& zero_from) {
    const int64_t V = b.vwords, total = chunk_sum(V);
    int64_t lo = 0, hi = V - 1;  // last row tile whose first chunk is at or before `local`
    while (lo < hi) {
        const int64_t mid = (lo + hi + 1) >> 1;
        if (total - chunk_sum(V - mid) <= local) lo = mid; else hi = mid - 1;
    }
    rb = lo;
    w0 = rb + (local - (total - chunk_sum(V - rb))) * kRelWordsPerBlock;
    zero_from = w0 + kRelWordsPerBlock >= V ? w0 + kRelWordsPerBlock : -1;
}

// One block per relate chunk of one set, the set read from a table built at
// create time, the (row tile, chunk) by a binary search over row tiles.  The
// last chunk of a row tile also zeroes the row's padding words.  One
// instance per geometry, each launched over that geometry's chunks only (a
// table groups the chunks by geometry), so that every geometry's code gets
// the registers it needs for itself.  Block x of a geometry's launch: relate block order[x] (the launch's slice
// of the blocks grouped by geometry), of set rblock_set[order[x]].
template <int G>
__global__ void __launch_bounds__(kRelThreads, 5) k_batch_relate(const BatchSet* __restrict__ sets,
                                                              const int32_t* __restrict__ rblock_set,
                                                              const int32_t* __restrict__ order) {
    __shared__ __align__(16) int32_t sc[kStageInts];
    const int64_t blk = order[blockIdx.x];
    const BatchSet& b = sets[rblock_set[blk]];
    if (batch_geom(b.kind) != G) return;  // never, by the order's construction
    int64_t rb, w0, zero_from;
    decode_rblock(b, blk - b.rblock_begin, rb, w0, zero_from);
    relate_block<G>(b.coords, b.n, b.bits, b.row_words, rb, w0, sc, G == kGeomLightCone && b.kind == CS_2D_ORDER,
                    zero_from);
}

// The light-cone kinds, from the column tables k_batch_rank built (one
// look-up per word instead of 64 cone tests).
__global__ void __launch_bounds__(kRelThreads, 4) k_batch_relate_cone(const BatchSet* __restrict__ sets,
                                                                   const int32_t* __restrict__ rblock_set,
                                                                   const int32_t* __restrict__ order,
                                                                   WsHeader* hdr) {
    extern __shared__ __align__(16) uint8_t smem_rel[];
    const int64_t blk = order[blockIdx.x];
    const BatchSet& b = sets[rblock_set[blk]];
    if (batch_geom(b.kind) != kGeomLightCone) return;  // never, by the order's construction
    int64_t rb, w0, zero_from;
    decode_rblock(b, blk - b.rblock_begin, rb, w0, zero_from);
    relate_block_tables(b.coords, b.n, b.bits, b.row_words, rb, w0, b.ctab, smem_rel, b.kind == CS_2D_ORDER,
                        zero_from, hdr);
}

// One block per mirror super-tile of one set (the lower part of its bitset
// as the transpose of the upper part), the set read from a table.
__global__ void __launch_bounds__(kRelThreads) k_batch_mirror(const BatchSet* __restrict__ sets,
                                                              const int32_t* __restrict__ mblock_set) {
    __shared__ uint64_t sm[kMirRows][kMirTiles + 1];
    const BatchSet& b = sets[mblock_set[blockIdx.x]];
    const int64_t local = int64_t(blockIdx.x) - b.mblock_begin;
    mirror_block(b.bits, b.n, b.row_words, local / b.mir_side, local % b.mir_side, sm);
}

// Smeared-sum coefficients f_d(k, eps) (Eqs. f2, f3, f4), one table per
// dimension present and eps, shared by every set of that dimension: a set's
// cutoff never exceeds that of the dimension's largest set (smear_cutoff
// grows with n), which sizes the table.  Dimension slot: d - 2.
constexpr int kDimSlots = 3;
struct CoefArgs {
    int64_t base[kDimSlots];              // first table entry of the slot
    int64_t stride[kDimSlots];            // entries per eps (the slot's largest n)
    int64_t kcap[kDimSlots][kMaxEps];     // entries computed per (slot, eps)
    int64_t seg[kDimSlots * kMaxEps + 1];  // prefix sums of kcap in (slot, eps) order
};

// The same launch finds each (set, eps) cutoff once (kends), after the
// table entries: a fixed-point iteration of about 1500 FP64 operations, too
// costly to repeat in every thread of the action kernel.
__global__ void __launch_bounds__(32) k_batch_coef(dd* __restrict__ coef, CoefArgs c, EpsArgs eps,
                                                    const BatchSet* __restrict__ sets, int nsets,
                                                    int64_t* __restrict__ kends) {
    const int64_t total = c.seg[kDimSlots * kMaxEps];
    const int64_t all = total + int64_t(nsets) * eps.n;
    for (int64_t t = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; t < all; t += int64_t(gridDim.x) * blockDim.x) {
        if (t >= total) {
            const int set = int((t - total) / eps.n), e = int((t - total) % eps.n);
            const double ep = eps.v[e];
            const BatchSet& b = sets[set];
            const int64_t len = b.n > 1 ? b.n - 1 : 1;
            const int64_t kc = is_local(ep) ? 0 : smear_cutoff(b.dim, ep, 0.5 * double(b.n) * double(b.n), len);
            const int64_t cap = c.kcap[b.dim - 2][e];
            kends[int64_t(set) * kMaxEps + e] = kc < cap ? kc : cap;  // never beyond the table
            continue;
        }
        int g = 0;
        while (c.seg[g + 1] <= t) ++g;  // at most 48 segments
        const int slot = g / kMaxEps, e = g % kMaxEps, dim = slot + 2;
        const int64_t k = t - c.seg[g];
        const double ep = eps.v[e];
        const dd q = dd_two_sum(1.0, -ep);
        coef[c.base[slot] + e * c.stride[slot] + k] =
            dd_mul(dd_pow(q, smear_qexp(dim, k)), smear_poly(dim, k, q, ep));
    }
}

// One CTA per (set, eps): the set's bracket (written by its eps-0 CTA) and
// one local or smeared action; the smeared sums take their coefficients from
// the shared table.  Each sum keeps the per-thread order and the reduction
// tree of the single-set action, so both give the same bits; a CTA per set
// walking its eps values one after another left the FP64 pipe waiting on
// the sums' dependency chains (0.29 ms for 768 sets and three smeared eps).
__global__ void __launch_bounds__(kActThreads) k_batch_action(const BatchSet* __restrict__ sets,
                                                              const int64_t* __restrict__ hist_base, EpsArgs eps,
                                                              const dd* __restrict__ coef, CoefArgs c,
                                                              const int64_t* __restrict__ kends,
                                                              double* __restrict__ actions,
                                                              int64_t* __restrict__ brackets) {
    __shared__ dd red[kActThreads];
    const int per = eps.n > 0 ? eps.n : 1;  // no eps: one CTA per set for the bracket
    const int set = blockIdx.x / per, e = blockIdx.x % per;
    const BatchSet& b = sets[set];
    const int dim = b.dim, slot = dim - 2;
    const int64_t n = b.n, len = n > 1 ? n - 1 : 1;
    const int64_t* hist = hist_base + b.hist_off;
    const int tid = threadIdx.x;
    int64_t h4[4] = {0, 0, 0, 0};
    for (int k = 0; k < 4 && k < len; ++k) h4[k] = hist[k];
    const int64_t br = bracket_of(dim, n, h4);
    if (tid == 0 && e == 0 && brackets) brackets[set] = br;
    if (e >= eps.n) return;
    const double ep = eps.v[e];
    if (is_local(ep)) {  // uniform across the CTA
        if (tid == 0 && actions) {
            const dd s = local_action(dim, br);
            actions[int64_t(set) * eps.n + e] = s.hi + s.lo;
        }
        return;
    }
    const int64_t kend = kends[int64_t(set) * kMaxEps + e];  // k_batch_coef's cutoff
    const dd* f = coef + c.base[slot] + e * c.stride[slot];
    dd sum = dd_from(0.0);
    for (int64_t k = tid; k < kend; k += kActThreads) {
        const int64_t hk = hist[k];
        if (hk != 0) sum = dd_add(sum, dd_mul(dd_from_i64(hk), f[k]));
    }
    red[tid] = sum;
    __syncthreads();
    for (int s = kActThreads / 2; s > 0; s >>= 1) {
        if (tid < s) red[tid] = dd_add(red[tid], red[tid + s]);
        __syncthreads();
    }
    if (tid == 0 && actions) {
        const dd s = smeared_action(dim, n, ep, red[0]);
        actions[int64_t(set) * eps.n + e] = s.hi + s.lo;
    }
}

std::atomic<bool> g_rank_attr[64];  // per device: the rank kernel's shared-memory attribute is set
std::atomic<bool> g_cone_attr[64];  // per device: the light-cone relate's shared-memory attribute is set

}  // namespace

}  // namespace cs

using namespace cs;

// Host-side plan of a batch (the device tables live in the workspace).
struct cs_batch {
    int nsets = 0;
    int path = CS_PATH_POPC;
    uint8_t* ws = nullptr;
    WsHeader* hdr = nullptr;
    BatchSet* sets_dev = nullptr;
    PopcSetEntry* popc_dev = nullptr;
    MmaSetEntry* mma_dev = nullptr;
    int64_t total_elems = 0, total_rblocks = 0, total_items = 0, total_chunks = 0, total_hist = 0;
    int32_t* rtab = nullptr;  // relate block -> set
    int32_t* rorder = nullptr;  // relate blocks grouped by geometry (each launch covers its own)
    int64_t geo_begin[8] = {0, 0, 0, 0, 0, 0, 0, 0}, geo_count[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int32_t* etab = nullptr;  // expansion chunk -> count-table entry
    int32_t* mtab = nullptr;  // mirror block -> set
    int64_t total_mblocks = 0;
    int64_t total_tiles = 0;  // column tiles of all sets (k_batch_ctab's warps)
    int32_t* ttab = nullptr;  // column tile -> set
    unsigned geoms = 0;  // bit G: some set relates with geometry G
    int max_pow2 = 1;
    const uint64_t* ds_thr = nullptr;  // de Sitter thresholds, when a set needs them
    dd* coef = nullptr;                 // smeared-sum coefficient tables
    int64_t* kends = nullptr;           // per (set, eps): smeared-sum cutoff [set * kMaxEps + e]
    int64_t nmax[kDimSlots] = {0, 0, 0};  // largest n per dimension slot (0: absent)
    int64_t coef_base[kDimSlots] = {0, 0, 0};
    // cs_batch_poll: each launch copies the status word here (pinned) and
    // records `done` after it.
    int32_t* status_host = nullptr;
    cudaEvent_t done = nullptr;
    ~cs_batch() {
        if (done) cudaEventDestroy(done);
        if (status_host) cudaFreeHost(status_host);
    }
};

namespace {

struct Layout {
    size_t sets, entries, rtab, rorder, etab, mtab, ttab, coef, kends, total;
    std::vector<size_t> coords, bits, key0, key1, raw, ctab, op0, op1;
};

bool batch_valid(const cs_set_desc* sets, int n_sets) {
    if (!sets || n_sets < 1 || n_sets > CS_BATCH_MAX_SETS) return false;
    for (int s = 0; s < n_sets; ++s)
        if (cs_dim(sets[s].kind) == 0 || sets[s].n < 1 || sets[s].n > CS_BATCH_MAX_N || sets[s].reserved != 0)
            return false;
    return true;
}

int batch_path(const cs_set_desc* sets, int n_sets, int path) {
    if (path != CS_PATH_AUTO) return path;
    return batch_auto_path();
}

bool tensor_path(int path) { return path == CS_PATH_MMA || path == CS_PATH_MMA4; }

Layout batch_layout(const cs_set_desc* sets, int n_sets, int path) {
    Layout L;
    size_t off = sizeof(WsHeader);
    auto take = [&](size_t bytes) {
        size_t at = off;
        off = align_up(off + bytes, 256);
        return at;
    };
    L.sets = take(sizeof(BatchSet) * size_t(n_sets));
    off = align_up(off, 128);
    L.entries = take((tensor_path(path) ? sizeof(MmaSetEntry) : sizeof(PopcSetEntry)) * size_t(n_sets));
    int64_t rblocks = 0, chunks = 0, mblocks = 0, tiles = 0;
    for (int s = 0; s < n_sets; ++s) {
        const int64_t n = sets[s].n;
        rblocks += chunk_sum((n + 63) / 64);
        tiles += (n + 63) / 64;
        const int64_t side = ((n + 63) / 64 + kMirTiles - 1) / kMirTiles;
        mblocks += side * side;
        if (tensor_path(path)) chunks += mma_expand_chunks(n);
    }
    L.rtab = take(size_t(rblocks) * 4);  // relate block -> set
    L.rorder = take(size_t(rblocks) * 4);  // relate blocks by geometry
    L.etab = take(size_t(chunks) * 4);   // expansion chunk -> set
    L.mtab = take(size_t(mblocks) * 4);  // mirror block -> set
    L.ttab = take(size_t(tiles) * 4);    // column tile -> set
    int64_t nmax[kDimSlots] = {0, 0, 0};
    for (int s = 0; s < n_sets; ++s) {
        int64_t& m = nmax[cs_dim(sets[s].kind) - 2];
        m = sets[s].n > m ? sets[s].n : m;
    }
    L.coef = take(size_t(nmax[0] + nmax[1] + nmax[2]) * kMaxEps * sizeof(dd));  // coefficient tables
    L.kends = take(size_t(n_sets) * kMaxEps * 8);                                 // smeared-sum cutoffs
    for (int s = 0; s < n_sets; ++s) {
        const int64_t n = sets[s].n;
        const int dim = cs_dim(sets[s].kind);
        L.coords.push_back(take(size_t(n) * dim * 4));
        L.bits.push_back(take(size_t(n) * size_t(cs_row_words(n)) * 8));
        L.key0.push_back(take(size_t(n) * 8));
        L.key1.push_back(take(size_t(n) * 8));
        L.raw.push_back(take(size_t(n) * 16));
        L.ctab.push_back(batch_geom(sets[s].kind) == kGeomLightCone ? take(size_t((n + 63) / 64) * sizeof(ConeTable))
                                                                    : 0);
        if (tensor_path(path)) {
            off = align_up(off, 1024);
            L.op0.push_back(take(mma_operand_bytes(n, path == CS_PATH_MMA4, 0)));
            off = align_up(off, 1024);
            L.op1.push_back(take(mma_operand_bytes(n, path == CS_PATH_MMA4, 1)));
        }
    }
    L.total = off;
    return L;
}

}  // namespace

extern "C" {

size_t cs_batch_workspace_bytes(const cs_set_desc* sets, int n_sets, int path) {
    if (!batch_valid(sets, n_sets) || path < CS_PATH_AUTO || path > CS_PATH_MMA4) return 0;
    return batch_layout(sets, n_sets, batch_path(sets, n_sets, path)).total;
}

int64_t cs_batch_hist_len(const cs_set_desc* sets, int n_sets) {
    if (!batch_valid(sets, n_sets)) return -1;
    int64_t t = 0;
    for (int s = 0; s < n_sets; ++s) t += cs_hist_len(sets[s].n);
    return t;
}

int cs_batch_create(const cs_set_desc* sets, int n_sets, int path, void* workspace_dev, size_t workspace_bytes,
                    cs_batch** out, void* stream) {
    CS_TRACE("cs_batch_create");
    if (!out) return CS_EINVAL;
    *out = nullptr;
    if (!batch_valid(sets, n_sets) || path < CS_PATH_AUTO || path > CS_PATH_MMA4 || !workspace_dev ||
        (reinterpret_cast<uintptr_t>(workspace_dev) % 1024) != 0)
        return CS_EINVAL;
    const int p = batch_path(sets, n_sets, path);
    if (tensor_path(p) && !device_has_tcgen05()) return CS_EUNSUPPORTED;
    const Layout L = batch_layout(sets, n_sets, p);
    if (workspace_bytes < L.total) return CS_ENOMEM;
    const uint64_t* ds_thr = nullptr;
    for (int s = 0; s < n_sets && !ds_thr; ++s)
        if (sets[s].kind == CS_2D_DS_SLAB && !(ds_thr = ds_table_device())) return CS_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint8_t* ws = static_cast<uint8_t*>(workspace_dev);

    std::vector<BatchSet> bs(static_cast<size_t>(n_sets));
    int64_t elem = 0, rblk = 0, mblk = 0, hoff = 0, tiles = 0;
    int max_pow2 = 1;
    for (int s = 0; s < n_sets; ++s) {
        BatchSet& b = bs[s];
        b.kind = sets[s].kind;
        b.dim = cs_dim(b.kind);
        b.n = sets[s].n;
        b.seed = sets[s].seed;
        b.coords = reinterpret_cast<int32_t*>(ws + L.coords[s]);
        b.bits = reinterpret_cast<uint64_t*>(ws + L.bits[s]);
        b.row_words = cs_row_words(b.n);
        b.key0 = reinterpret_cast<uint64_t*>(ws + L.key0[s]);
        b.key1 = reinterpret_cast<uint64_t*>(ws + L.key1[s]);
        b.raw = reinterpret_cast<int32_t*>(ws + L.raw[s]);
        b.ctab = L.ctab[s] ? reinterpret_cast<ConeTable*>(ws + L.ctab[s]) : nullptr;
        b.elem_begin = elem;
        elem += b.n;
        b.vwords = (b.n + 63) / 64;
        b.rblock_begin = rblk;
        rblk += chunk_sum(b.vwords);
        b.mir_side = ((b.n + 63) / 64 + kMirTiles - 1) / kMirTiles;
        b.mblock_begin = mblk;
        b.tile_begin = tiles;
        tiles += b.vwords;
        mblk += b.mir_side * b.mir_side;
        b.hist_off = hoff;
        hoff += cs_hist_len(b.n);
        while (max_pow2 < b.n) max_pow2 <<= 1;
    }
    // Count tables in decreasing set size (the largest sets' tiles go first).
    std::vector<int> order(static_cast<size_t>(n_sets));
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return bs[a].n > bs[b].n; });
    int64_t items = 0, chunks = 0;
    std::vector<int32_t> rtab(static_cast<size_t>(rblk)), etab, mtab(static_cast<size_t>(mblk)),
        ttab(static_cast<size_t>(tiles));
    for (int s = 0; s < n_sets; ++s)
        std::fill(ttab.begin() + bs[s].tile_begin, ttab.begin() + bs[s].tile_begin + bs[s].vwords, int32_t(s));
    for (int s = 0; s < n_sets; ++s)
        std::fill(mtab.begin() + bs[s].mblock_begin, mtab.begin() + bs[s].mblock_begin + bs[s].mir_side * bs[s].mir_side,
                  int32_t(s));
    for (int s = 0; s < n_sets; ++s)
        std::fill(rtab.begin() + bs[s].rblock_begin, rtab.begin() + bs[s].rblock_begin + chunk_sum(bs[s].vwords),
                  int32_t(s));
    // the relate blocks grouped by geometry, so that each geometry's launch
    // covers only its own blocks (blocks of the other geometries returning at
    // once had cost their dispatch)
    std::vector<int32_t> rorder;
    rorder.reserve(rtab.size());
    int64_t geo_begin[8], geo_count[8];
    for (int g = 0; g < 8; ++g) {
        geo_begin[g] = int64_t(rorder.size());
        for (int s = 0; s < n_sets; ++s)
            if (batch_geom(bs[s].kind) == g)
                for (int64_t k = 0; k < chunk_sum(bs[s].vwords); ++k) rorder.push_back(int32_t(bs[s].rblock_begin + k));
        geo_count[g] = int64_t(rorder.size()) - geo_begin[g];
    }
    std::vector<PopcSetEntry> pe;
    std::vector<MmaSetEntry> me;
    for (int r = 0; r < n_sets; ++r) {
        const BatchSet& b = bs[order[r]];
        if (tensor_path(p)) {
            // FP4 pairs count in supertiles, FP8 in 128-row tiles
            const bool fp4 = p == CS_PATH_MMA4;
            MmaSetEntry e;
            std::memset(static_cast<void*>(&e), 0, sizeof(e));
            if (mma_fill_entry(&e, b.bits, b.n, b.row_words, ws + L.op0[order[r]], ws + L.op1[order[r]], fp4) !=
                CUDA_SUCCESS)
                return CS_ECUDA;
            e.item_begin = items;
            e.item_offset = 0;
            items += fp4 ? mma4_units(b.n) : mma_items(b.n);
            e.hist_off = b.hist_off * 8;
            e.chunk_begin = chunks;
            chunks += mma_expand_chunks(b.n);
            etab.insert(etab.end(), size_t(mma_expand_chunks(b.n)), int32_t(r));  // entry r of the table
            me.push_back(e);
        } else {
            PopcSetEntry e;
            std::memset(static_cast<void*>(&e), 0, sizeof(e));
            popc_fill_entry(&e, b.bits, b.n, b.row_words);
            if (popc_encode_map(&e.map, b.bits, b.n, b.row_words) != CUDA_SUCCESS) return CS_ECUDA;
            e.item_begin = items;
            e.item_offset = 0;
            items += popc_tiles(b.n);
            e.hist_off = b.hist_off * 8;
            pe.push_back(e);
        }
    }
    cs_batch* h = new (std::nothrow) cs_batch;
    if (!h) return CS_ENOMEM;
    if (cudaHostAlloc(reinterpret_cast<void**>(&h->status_host), sizeof(int32_t), cudaHostAllocDefault) !=
            cudaSuccess ||
        cudaEventCreateWithFlags(&h->done, cudaEventDisableTiming) != cudaSuccess) {
        delete h;
        return CS_ECUDA;
    }
    *h->status_host = CS_OK;
    h->nsets = n_sets;
    h->path = p;
    h->ws = ws;
    h->hdr = reinterpret_cast<WsHeader*>(ws);
    h->sets_dev = reinterpret_cast<BatchSet*>(ws + L.sets);
    h->total_elems = elem;
    h->total_rblocks = rblk;
    for (int s = 0; s < n_sets; ++s) h->geoms |= 1u << batch_geom(sets[s].kind);
    h->total_items = items;
    h->total_chunks = chunks;
    h->rtab = reinterpret_cast<int32_t*>(ws + L.rtab);
    h->rorder = reinterpret_cast<int32_t*>(ws + L.rorder);
    for (int g = 0; g < 8; ++g) {
        h->geo_begin[g] = geo_begin[g];
        h->geo_count[g] = geo_count[g];
    }
    h->mtab = reinterpret_cast<int32_t*>(ws + L.mtab);
    h->total_mblocks = mblk;
    h->total_tiles = tiles;
    h->ttab = reinterpret_cast<int32_t*>(ws + L.ttab);
    h->etab = reinterpret_cast<int32_t*>(ws + L.etab);
    h->total_hist = hoff;
    h->max_pow2 = max_pow2;
    h->ds_thr = ds_thr;
    h->coef = reinterpret_cast<dd*>(ws + L.coef);
    h->kends = reinterpret_cast<int64_t*>(ws + L.kends);
    for (int s = 0; s < n_sets; ++s) {
        int64_t& m = h->nmax[bs[s].dim - 2];
        m = bs[s].n > m ? bs[s].n : m;
    }
    int64_t at = 0;
    for (int d = 0; d < kDimSlots; ++d) {
        h->coef_base[d] = at;
        at += h->nmax[d] * kMaxEps;
    }
    cudaError_t e = cudaMemcpyAsync(h->sets_dev, bs.data(), sizeof(BatchSet) * bs.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !rtab.empty())
        e = cudaMemcpyAsync(h->rtab, rtab.data(), rtab.size() * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !rorder.empty())
        e = cudaMemcpyAsync(h->rorder, rorder.data(), rorder.size() * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !mtab.empty())
        e = cudaMemcpyAsync(h->mtab, mtab.data(), mtab.size() * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !ttab.empty())
        e = cudaMemcpyAsync(h->ttab, ttab.data(), ttab.size() * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !etab.empty())
        e = cudaMemcpyAsync(h->etab, etab.data(), etab.size() * 4, cudaMemcpyHostToDevice, st);
    if (tensor_path(p)) {
        h->mma_dev = reinterpret_cast<MmaSetEntry*>(ws + L.entries);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h->mma_dev, me.data(), sizeof(MmaSetEntry) * me.size(), cudaMemcpyHostToDevice, st);
    } else {
        h->popc_dev = reinterpret_cast<PopcSetEntry*>(ws + L.entries);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h->popc_dev, pe.data(), sizeof(PopcSetEntry) * pe.size(), cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // the host tables go out of scope
    if (e != cudaSuccess) {
        delete h;
        return CS_ECUDA;
    }
    *out = h;
    return CS_OK;
}

int cs_batch_launch(const cs_batch* b, const double* eps_host, int n_eps, int64_t* hist_dev, double* actions_dev,
                    int64_t* brackets_dev, void* stream) {
    CS_TRACE("cs_batch_launch");
    if (!b || !hist_dev || n_eps < 0 || n_eps > kMaxEps || (n_eps > 0 && (!eps_host || !actions_dev)) ||
        (reinterpret_cast<uintptr_t>(hist_dev) % 8) != 0)
        return CS_EINVAL;
    EpsArgs a;
    a.n = n_eps;
    for (int e = 0; e < kMaxEps; ++e) {
        a.v[e] = e < n_eps ? eps_host[e] : 0.0;
        a.kend[e] = 0;  // per set, in the kernel
        if (e < n_eps && !(a.v[e] <= 1.0)) return CS_EINVAL;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t err = cudaMemsetAsync(&b->hdr->status, 0, sizeof(int32_t), st);
    if (err == cudaSuccess) err = cudaMemsetAsync(hist_dev, 0, size_t(b->total_hist) * 8, st);
    if (err != cudaSuccess) return CS_ECUDA;
    const int sms = device_sm_count();

    int64_t g = (b->total_elems + 255) / 256;
    if (g > int64_t(sms) * 16) g = int64_t(sms) * 16;
    k_batch_keys<<<unsigned(g), 256, 0, st>>>(b->sets_dev, b->nsets, b->total_elems, b->ds_thr, b->hdr);

    const size_t rank_smem = size_t(b->max_pow2 > kRankThreads ? b->max_pow2 : kRankThreads) * 24;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return CS_ECUDA;
    if (dev >= 0 && dev < 64 && !g_rank_attr[dev]) {
        if (cudaFuncSetAttribute(k_batch_rank, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(size_t(CS_BATCH_MAX_N) * 24)) != cudaSuccess)
            return CS_ECUDA;
        g_rank_attr[dev] = true;
    }
    if ((b->geoms & (1u << kGeomLightCone)) && dev >= 0 && dev < 64 && !g_cone_attr[dev]) {
        if (cudaFuncSetAttribute(k_batch_relate_cone, cudaFuncAttributeMaxDynamicSharedMemorySize, kConeTableSmem) !=
            cudaSuccess)
            return CS_ECUDA;
        g_cone_attr[dev] = true;
    }
    k_batch_rank<<<unsigned(b->nsets), kRankThreads, rank_smem, st>>>(b->sets_dev);
    if (b->geoms & (1u << kGeomLightCone))
        k_batch_ctab<<<unsigned((b->total_tiles * 32 + 255) / 256), 256, 0, st>>>(b->sets_dev, b->ttab,
                                                                                 b->total_tiles);

    if (b->total_rblocks > int64_t(0x7fffffff)) return CS_EINVAL;
    // one launch per geometry present, over that geometry's blocks only
    auto range = [&](int g) { return b->rorder + b->geo_begin[g]; };
    if (b->geo_count[kGeomLightCone])
        k_batch_relate_cone<<<unsigned(b->geo_count[kGeomLightCone]), kRelThreads, kConeTableSmem, st>>>(
            b->sets_dev, b->rtab, range(kGeomLightCone), b->hdr);
    if (b->geo_count[kGeom3])
        k_batch_relate<kGeom3><<<unsigned(b->geo_count[kGeom3]), kRelThreads, 0, st>>>(b->sets_dev, b->rtab,
                                                                                     range(kGeom3));
    if (b->geo_count[kGeom4])
        k_batch_relate<kGeom4><<<unsigned(b->geo_count[kGeom4]), kRelThreads, 0, st>>>(b->sets_dev, b->rtab,
                                                                                     range(kGeom4));
    if (b->geo_count[kGeomDeSitter])
        k_batch_relate<kGeomDeSitter><<<unsigned(b->geo_count[kGeomDeSitter]), kRelThreads, 0, st>>>(
            b->sets_dev, b->rtab, range(kGeomDeSitter));
    if (b->total_mblocks > int64_t(0x7fffffff)) return CS_EINVAL;
    k_batch_mirror<<<unsigned(b->total_mblocks), kRelThreads, 0, st>>>(b->sets_dev, b->mtab);
    if ((err = cudaGetLastError()) != cudaSuccess) return CS_ECUDA;

    if (b->path == CS_PATH_MMA) {
        if ((err = launch_expand_multi(b->mma_dev, b->etab, b->total_chunks, st)) != cudaSuccess) return CS_ECUDA;
        err = launch_count_mma_multi(b->mma_dev, b->nsets, b->total_items, reinterpret_cast<uintptr_t>(hist_dev),
                                     b->hdr, 0, st);
    } else if (b->path == CS_PATH_MMA4) {
        if ((err = launch_expand_multi(b->mma_dev, b->etab, b->total_chunks, st, true)) != cudaSuccess)
            return CS_ECUDA;
        err = launch_count_mma4_multi(b->mma_dev, b->nsets, b->total_items, reinterpret_cast<uintptr_t>(hist_dev),
                                      b->hdr, st);
    } else {
        err = launch_count_popc_multi(b->popc_dev, b->nsets, b->total_items, reinterpret_cast<uintptr_t>(hist_dev),
                                      b->hdr, 0, st);
    }
    if (err != cudaSuccess) return CS_ECUDA;
    if (n_eps > 0 || brackets_dev) {
        CoefArgs c;
        std::memset(static_cast<void*>(&c), 0, sizeof(c));
        int64_t at = 0;
        for (int d = 0; d < kDimSlots; ++d) {
            c.base[d] = b->coef_base[d];
            c.stride[d] = b->nmax[d];
            const int64_t nm = b->nmax[d], len = nm > 1 ? nm - 1 : 1;
            for (int e = 0; e < kMaxEps; ++e) {
                c.kcap[d][e] = (nm > 0 && e < n_eps && !is_local(a.v[e]))
                                   ? smear_cutoff(d + 2, a.v[e], 0.5 * double(nm) * double(nm), len)
                                   : 0;
                c.seg[d * kMaxEps + e] = at;
                at += c.kcap[d][e];
            }
        }
        c.seg[kDimSlots * kMaxEps] = at;
        if (at > 0) {
            // one warp per block: the FP64 work (table entries, then the
            // cutoffs) spreads over every SM's FP64 pipe
            int64_t g = (at + int64_t(b->nsets) * a.n + 31) / 32;
            if (g > int64_t(sms) * 16) g = int64_t(sms) * 16;
            k_batch_coef<<<unsigned(g), 32, 0, st>>>(b->coef, c, a, b->sets_dev, b->nsets, b->kends);
        }
        k_batch_action<<<unsigned(b->nsets * (a.n > 0 ? a.n : 1)), kActThreads, 0, st>>>(
            b->sets_dev, hist_dev, a, b->coef, c, b->kends, actions_dev, brackets_dev);
        if (cudaGetLastError() != cudaSuccess) return CS_ECUDA;
    }
    // For cs_batch_poll: the status word to the plan's pinned copy, then the
    // event (recorded as an external event node when the stream is captured).
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if ((err = cudaStreamIsCapturing(st, &cap)) != cudaSuccess) return cuda_status(err);
    if ((err = cudaMemcpyAsync(b->status_host, &b->hdr->status, sizeof(int32_t), cudaMemcpyDeviceToHost, st)) !=
        cudaSuccess)
        return cuda_status(err);
    err = cap == cudaStreamCaptureStatusActive ? cudaEventRecordWithFlags(b->done, st, cudaEventRecordExternal)
                                               : cudaEventRecord(b->done, st);
    return cuda_status(err);
}

int cs_batch_poll(const cs_batch* b) {
    if (!b) return CS_EINVAL;
    const cudaError_t q = cudaEventQuery(b->done);
    if (q == cudaErrorNotReady) {
        cudaGetLastError();  // not sticky; keep it from the caller's next check
        return CS_PENDING;
    }
    if (q != cudaSuccess) return CS_ECUDA;
    return *static_cast<volatile int32_t*>(b->status_host);
}

int cs_batch_path(const cs_batch* b) { return b ? b->path : -1; }

void cs_batch_destroy(cs_batch* b) { delete b; }

}  // extern "C"
