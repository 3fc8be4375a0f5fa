// cs_chains.cu -- longest chains and greedy maximal antichains on the bitset
// (Section "Set Partitions": Algorithms "Maximal Chain Length" and "Maximal
// Antichain").
//
// Longest chain.  The thesis recurses through the Alexandroff set, caching
// the distance of each element to the top.  On the GPU the same length comes
// from peeling: the set S (A_ij for a pair, every element for the whole set)
// loses all its minimal elements -- those with no predecessor left in S --
// once per round; the number of rounds is the number of elements of the
// longest chain in S.  A round is one warp per element of S testing
// P_k & S over the words before k, then one block clearing the removed bits.
//
// Greedy antichain.  Each round scores every candidate j by
// c_j = |A - J(j)| (one warp per candidate, popcounts of A & ~row_j), keeps
// the best with one 64-bit atomicMax on (c_j, -j) -- the largest c, the
// smallest label on ties, as in the algorithm's scan -- and one block
// removes J(k) from A and J(k) + {k} from the candidates.
//
// Both run all their rounds in one cooperative launch, the rounds separated
// by bounded grid barriers; where a cooperative launch is not available they
// fall back to batches of kBatch launches between host checks of the number
// of elements left (rounds after the last one find nothing to do).
#include "cs_kernels.cuh"

namespace cs {

namespace {

constexpr int kBatch = 32;

struct ChainState {
    unsigned long long best;  // antichain: packed (c, ~label) of the best candidate
    int32_t found;            // chain: this round removed something
    int32_t related;          // chain: i precedes j
    int64_t rounds;           // rounds that removed something
    int64_t left;             // elements left in S (chain) or candidates left (antichain)
    // persistent (cooperative) kernels: grid barrier and per-round-parity counters
    unsigned int bar_count, bar_gen;
    unsigned long long left2[2];
    unsigned long long best2[2];
    unsigned int rcount[2];   // antichain: candidates removed this round (list length)
};

struct ChainLayout {
    size_t state, s, m, over, rlist, total;
};

ChainLayout chain_layout(int64_t row_words) {
    ChainLayout L;
    size_t off = sizeof(WsHeader);
    L.state = off;
    off = align_up(off + sizeof(ChainState), 256);
    L.s = off;
    off = align_up(off + size_t(row_words) * 8, 256);
    L.m = off;
    off = align_up(off + size_t(row_words) * 8, 256);
    L.over = off;  // antichain: overlap |A & J(j)| of every candidate j
    off = align_up(off + size_t(row_words) * 64 * 4, 256);
    L.rlist = off;  // antichain: the candidates removed in a round
    off = align_up(off + size_t(row_words) * 64 * 4, 256);
    L.total = off;
    return L;
}

__device__ __forceinline__ bool bit_of(const uint64_t* row, int64_t k) { return (row[k >> 6] >> (k & 63)) & 1ull; }

// Bits of word w strictly between columns lo and hi (lo < col < hi).
__device__ __forceinline__ uint64_t between_mask(int64_t w, int64_t lo, int64_t hi) {
    const int64_t c0 = 64 * w;
    uint64_t m = ~0ull;
    if (lo + 1 > c0) m = lo + 1 - c0 >= 64 ? 0ull : m & (~0ull << (lo + 1 - c0));
    if (hi < c0 + 64) m = hi <= c0 ? 0ull : m & (~0ull >> (c0 + 64 - hi));
    return m;
}

__device__ __forceinline__ int warp_or(int v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v |= __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// S = A_ij (bits strictly between i and j set in both rows), or all of [0, n).
__global__ void k_chain_init(const uint64_t* __restrict__ bits, int64_t n, int64_t row_words, int64_t i, int64_t j,
                             uint64_t* __restrict__ S, uint64_t* __restrict__ M, ChainState* st) {
    const bool whole = i < 0;
    const int64_t lo = whole ? -1 : i, hi = whole ? n : j;
    for (int64_t w = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; w < row_words;
         w += int64_t(gridDim.x) * blockDim.x) {
        uint64_t x = between_mask(w, lo, hi);
        if (!whole) x &= __ldg(bits + i * row_words + w) & __ldg(bits + j * row_words + w);
        S[w] = x;
        M[w] = 0ull;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->found = 0;
        st->rounds = 0;
        st->related = whole ? 1 : int(bit_of(bits + i * row_words, j));
        st->left = 1;
    }
}

// One peeling round: the elements of S with no predecessor in S go to M.
__global__ void __launch_bounds__(256) k_chain_peel(const uint64_t* __restrict__ bits, int64_t row_words,
                                                    int64_t lo, int64_t hi, const uint64_t* __restrict__ S,
                                                    uint64_t* __restrict__ M, ChainState* st) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = int64_t(gridDim.x) * (blockDim.x >> 5);
    const int64_t wlo = lo < 0 ? 0 : lo >> 6;
    for (int64_t k = lo + 1 + int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); k < hi; k += warps) {
        if (!bit_of(S, k)) continue;  // warp-uniform
        const int64_t wk = k >> 6;
        int any = 0;
        for (int64_t w = wlo + lane; w <= wk && !any; w += 32) {
            uint64_t x = __ldg(bits + k * row_words + w) & S[w];
            if (w == wk) x &= (k & 63) ? ((1ull << (k & 63)) - 1ull) : 0ull;  // predecessors only
            any = x != 0ull;
        }
        if (!warp_or(any) && lane == 0) {
            atomicOr(reinterpret_cast<unsigned long long*>(M + wk), 1ull << (k & 63));
            st->found = 1;
        }
    }
}

// Close a round: S -= M, count it if it removed anything, count what is left.
__global__ void __launch_bounds__(1024) k_chain_apply(int64_t row_words, uint64_t* __restrict__ S,
                                                      uint64_t* __restrict__ M, ChainState* st) {
    __shared__ unsigned long long left;
    __shared__ int found;
    if (threadIdx.x == 0) {
        left = 0;
        found = st->found;
    }
    __syncthreads();
    unsigned long long mine = 0;
    for (int64_t w = threadIdx.x; w < row_words; w += blockDim.x) {
        const uint64_t x = S[w] & ~M[w];
        S[w] = x;
        M[w] = 0ull;
        mine += __popcll(x);
    }
    atomicAdd(&left, mine);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (found) st->rounds += 1;
        st->found = 0;
        st->left = int64_t(left);
    }
}

// Antichain start: X = elements unrelated to the seed, A = X + {seed}.
__global__ void k_anti_init(const uint64_t* __restrict__ bits, int64_t n, int64_t row_words, int64_t seed,
                            uint64_t* __restrict__ A, uint64_t* __restrict__ X, ChainState* st) {
    for (int64_t w = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; w < row_words;
         w += int64_t(gridDim.x) * blockDim.x) {
        uint64_t x = ~__ldg(bits + seed * row_words + w) & between_mask(w, -1, n);
        if (w == (seed >> 6)) x &= ~(1ull << (seed & 63));
        X[w] = x;
        A[w] = w == (seed >> 6) ? x | (1ull << (seed & 63)) : x;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        st->best = 0ull;
        st->left = 1;
    }
}

// Score every candidate j by |A - J(j)|; keep the best (largest, then first).
__global__ void __launch_bounds__(256) k_anti_score(const uint64_t* __restrict__ bits, int64_t n, int64_t row_words,
                                                    const uint64_t* __restrict__ A, const uint64_t* __restrict__ X,
                                                    ChainState* st) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (n + 63) >> 6;
    const int64_t warps = int64_t(gridDim.x) * (blockDim.x >> 5);
    for (int64_t k = int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5); k < n; k += warps) {
        if (!bit_of(X, k)) continue;  // warp-uniform
        int c = 0;
        for (int64_t w = lane; w < nw; w += 32) c += __popcll(A[w] & ~__ldg(bits + k * row_words + w));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane == 0)
            atomicMax(&st->best, (static_cast<unsigned long long>(c) << 32) | (0xFFFFFFFFull - uint64_t(k)));
    }
}

// Take the best candidate k: A -= J(k), X -= J(k) + {k}.
__global__ void __launch_bounds__(1024) k_anti_apply(const uint64_t* __restrict__ bits, int64_t row_words,
                                                     uint64_t* __restrict__ A, uint64_t* __restrict__ X,
                                                     ChainState* st) {
    __shared__ unsigned long long left;
    __shared__ unsigned long long best;
    if (threadIdx.x == 0) {
        left = 0;
        best = st->best;
    }
    __syncthreads();
    const bool take = best != 0ull;
    const int64_t k = int64_t(0xFFFFFFFFull - (best & 0xFFFFFFFFull));
    unsigned long long mine = 0;
    for (int64_t w = threadIdx.x; w < row_words; w += blockDim.x) {
        uint64_t x = X[w];
        if (take) {
            const uint64_t r = __ldg(bits + k * row_words + w);
            A[w] &= ~r;
            x &= ~r;
            if (w == (k >> 6)) x &= ~(1ull << (k & 63));
            X[w] = x;
        }
        mine += __popcll(x);
    }
    atomicAdd(&left, mine);
    __syncthreads();
    if (threadIdx.x == 0) {
        st->best = 0ull;
        st->left = int64_t(left);
    }
}

// Number of set bits of a bitset into st->rounds.
__global__ void __launch_bounds__(1024) k_count_bits(const uint64_t* __restrict__ A, int64_t row_words,
                                                     ChainState* st) {
    __shared__ unsigned long long total;
    if (threadIdx.x == 0) total = 0;
    __syncthreads();
    unsigned long long mine = 0;
    for (int64_t w = threadIdx.x; w < row_words; w += blockDim.x) mine += __popcll(A[w]);
    atomicAdd(&total, mine);
    __syncthreads();
    if (threadIdx.x == 0) st->rounds = int64_t(total);
}

// ------------------------------------------- persistent (cooperative) rounds
//
// With a cooperative launch every block is resident, so the rounds can run in
// one kernel separated by grid barriers instead of two launches per round.
// The barrier's wait is bounded: after 4 s it records CS_ETIMEOUT and the
// kernel returns (every later barrier of the other blocks then times out
// too), so a fault cannot hang the GPU.

__device__ bool grid_barrier(ChainState* st, unsigned int nblocks, WsHeader* hdr) {
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned int* gen = &st->bar_gen;
        const unsigned int g = *gen;
        __threadfence();
        if (atomicAdd(&st->bar_count, 1u) == nblocks - 1u) {
            st->bar_count = 0u;
            __threadfence();
            atomicAdd(&st->bar_gen, 1u);
        } else {
            const unsigned long long t0 = global_timer_ns();
            while (*gen == g) {
                if (global_timer_ns() - t0 > kWaitLimitNs) {
                    set_status(hdr, CS_ETIMEOUT);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

__device__ __forceinline__ unsigned long long block_sum_to(unsigned long long v, unsigned long long* dst) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(dst, v);
    return v;
}

// All peeling rounds: peel (as k_chain_peel), barrier, S -= M with the count
// of what is left, barrier, stop when nothing is left.  rounds = the number
// of rounds run (S is not empty at the start).
__global__ void __launch_bounds__(256) k_chain_persist(const uint64_t* __restrict__ bits, int64_t row_words,
                                                       int64_t lo, int64_t hi, int64_t max_rounds, uint64_t* S,
                                                       uint64_t* M, ChainState* st, WsHeader* hdr) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = int64_t(gridDim.x) * (blockDim.x >> 5);
    const int64_t gwarp = int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t gthread = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t nthreads = int64_t(gridDim.x) * blockDim.x;
    const int64_t wlo = lo < 0 ? 0 : lo >> 6;
    for (int64_t r = 0; r < max_rounds; ++r) {
        for (int64_t k = lo + 1 + gwarp; k < hi; k += warps) {
            if (!bit_of(S, k)) continue;  // warp-uniform
            const int64_t wk = k >> 6;
            int any = 0;
            for (int64_t w = wk - lane; w >= wlo && !any; w -= 32) {  // nearest predecessors first
                uint64_t x = __ldg(bits + k * row_words + w) & S[w];
                if (w == wk) x &= (k & 63) ? ((1ull << (k & 63)) - 1ull) : 0ull;
                any = x != 0ull;
            }
            if (!warp_or(any) && lane == 0) atomicOr(reinterpret_cast<unsigned long long*>(M + wk), 1ull << (k & 63));
        }
        if (!grid_barrier(st, gridDim.x, hdr)) return;
        unsigned long long mine = 0;
        for (int64_t w = gthread; w < row_words; w += nthreads) {
            const uint64_t x = S[w] & ~M[w];
            S[w] = x;
            M[w] = 0ull;
            mine += __popcll(x);
        }
        block_sum_to(mine, &st->left2[r & 1]);
        if (gthread == 0) st->left2[(r + 1) & 1] = 0ull;  // last read before the previous barrier
        if (!grid_barrier(st, gridDim.x, hdr)) return;
        if (*reinterpret_cast<volatile unsigned long long*>(&st->left2[r & 1]) == 0ull) {
            if (gthread == 0) st->rounds = r + 1;
            return;
        }
    }
}

// All greedy rounds, with incremental scores.  Maximising c_j = |A - J(j)|
// is minimising the overlap o_j = |A & J(j)|.  When k is taken, A loses
// R = A & J(k), which are exactly the candidates related to k (the members
// are unrelated to every candidate), so every remaining o_j drops by the
// number of R's elements related to j.  Per round: the smallest (o_j, j) by
// one 64-bit atomicMin, barrier; remove J(k) from A and J(k) + {k} from X
// and list R, barrier; stop if X is empty; subtract R's contributions from
// the o_j of the remaining candidates (a thread per column, the list read
// in step), barrier.  The overlaps are computed in full once, at the start.
__global__ void __launch_bounds__(256) k_anti_persist(const uint64_t* __restrict__ bits, int64_t n,
                                                      int64_t row_words, int64_t max_rounds, uint64_t* A,
                                                      uint64_t* X, int32_t* over, int32_t* rlist, ChainState* st,
                                                      WsHeader* hdr) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = (n + 63) >> 6;
    const int64_t warps = int64_t(gridDim.x) * (blockDim.x >> 5);
    const int64_t gwarp = int64_t(blockIdx.x) * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int64_t gthread = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t nthreads = int64_t(gridDim.x) * blockDim.x;
    for (int64_t k = gwarp; k < n; k += warps) {  // o_j for every candidate, once
        if (!bit_of(X, k)) continue;               // warp-uniform
        int c = 0;
        for (int64_t w = lane; w < nw; w += 32) c += __popcll(A[w] & __ldg(bits + k * row_words + w));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
        if (lane == 0) over[k] = c;
    }
    if (!grid_barrier(st, gridDim.x, hdr)) return;
    for (int64_t r = 0; r < max_rounds; ++r) {
        // the candidate with the smallest overlap, the smallest label on ties
        unsigned long long mine = ~0ull;
        for (int64_t j = gthread; j < n; j += nthreads)
            if (bit_of(X, j)) {
                const unsigned long long key = (static_cast<unsigned long long>(over[j]) << 32) | uint64_t(j);
                mine = key < mine ? key : mine;
            }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long y = __shfl_xor_sync(0xffffffffu, mine, o);
            mine = y < mine ? y : mine;
        }
        if (lane == 0 && mine != ~0ull) atomicMin(&st->best2[r & 1], mine);
        if (gthread == 0) {
            st->best2[(r + 1) & 1] = ~0ull;  // last read before the previous round's second barrier
            st->rcount[(r + 1) & 1] = 0u;
            st->left2[(r + 1) & 1] = 0ull;
        }
        if (!grid_barrier(st, gridDim.x, hdr)) return;
        const unsigned long long best = *reinterpret_cast<volatile unsigned long long*>(&st->best2[r & 1]);
        if (best == ~0ull) return;  // no candidates (every block sees the same value)
        const int64_t k = int64_t(best & 0xFFFFFFFFull);
        unsigned long long left = 0;
        for (int64_t w = gthread; w < row_words; w += nthreads) {
            const uint64_t rk = __ldg(bits + k * row_words + w);
            const uint64_t x = X[w];
            uint64_t removed = x & rk;
            uint64_t nx = x & ~rk;
            if (w == (k >> 6)) nx &= ~(1ull << (k & 63));
            X[w] = nx;
            A[w] &= ~rk;
            left += __popcll(nx);
            if (removed) {
                unsigned int pos = atomicAdd(&st->rcount[r & 1], unsigned(__popcll(removed)));
                for (; removed; removed &= removed - 1ull)
                    rlist[pos++] = int32_t(64 * w + __ffsll(static_cast<long long>(removed)) - 1);
            }
        }
        block_sum_to(left, &st->left2[r & 1]);
        if (!grid_barrier(st, gridDim.x, hdr)) return;
        if (*reinterpret_cast<volatile unsigned long long*>(&st->left2[r & 1]) == 0ull) return;
        const unsigned int nr = *reinterpret_cast<volatile unsigned int*>(&st->rcount[r & 1]);
        for (int64_t j = gthread; j < n; j += nthreads) {
            if (!bit_of(X, j)) continue;
            int d = 0;
            for (unsigned int t = 0; t < nr; ++t)
                d += int((__ldg(bits + int64_t(rlist[t]) * row_words + (j >> 6)) >> (j & 63)) & 1ull);
            over[j] -= d;
        }
        if (!grid_barrier(st, gridDim.x, hdr)) return;
    }
}

// Blocks of a cooperative launch of `kernel` (all resident), capped by the work.
int coop_grid(const void* kernel, int64_t warps_of_work) {
    int dev = 0, coop = 0, per_sm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, 0) != cudaSuccess || per_sm < 1)
        return 0;
    int64_t g = int64_t(per_sm) * device_sm_count();
    const int64_t need = (warps_of_work + 7) / 8;
    if (g > need) g = need;
    return int(g < 1 ? 1 : g);
}

int warp_grid(int64_t rows) {
    int64_t g = (rows + 7) / 8;
    const int64_t cap = int64_t(device_sm_count()) * 16;
    return int(g < 1 ? 1 : (g > cap ? cap : g));
}

bool chain_args_ok(int64_t n, const uint64_t* bits, int64_t row_words, void* ws) {
    return n >= 1 && n <= kMaxN && bits && (reinterpret_cast<uintptr_t>(bits) % 16) == 0 &&
           row_words >= cs_row_words(n) && row_words % 16 == 0 && ws && (reinterpret_cast<uintptr_t>(ws) % 256) == 0;
}

cudaError_t read_state(const ChainState* dev, ChainState* host, cudaStream_t st) {
    cudaError_t e = cudaMemcpyAsync(host, dev, sizeof(ChainState), cudaMemcpyDeviceToHost, st);
    return e == cudaSuccess ? cudaStreamSynchronize(st) : e;
}

}  // namespace

}  // namespace cs

using namespace cs;

extern "C" size_t cs_chain_workspace_bytes(int64_t n) {
    if (n < 1 || n > kMaxN) return 0;
    return chain_layout(cs_row_words(n)).total;
}

extern "C" int cs_longest_chain(int64_t n, const uint64_t* bits_dev, int64_t row_words, int64_t i, int64_t j,
                                int64_t* length, void* workspace_dev, size_t workspace_bytes, void* stream) {
    CS_TRACE("cs_longest_chain");
    if (!chain_args_ok(n, bits_dev, row_words, workspace_dev) || !length) return CS_EINVAL;
    const bool whole = i < 0 && j < 0;
    if (!whole && (i < 0 || j < 0 || i >= n || j >= n)) return CS_EINVAL;
    const ChainLayout L = chain_layout(row_words);
    if (workspace_bytes < L.total) return CS_ENOMEM;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint8_t* ws = static_cast<uint8_t*>(workspace_dev);
    ChainState* sd = reinterpret_cast<ChainState*>(ws + L.state);
    uint64_t* S = reinterpret_cast<uint64_t*>(ws + L.s);
    uint64_t* M = reinterpret_cast<uint64_t*>(ws + L.m);
    if (!whole && j <= i) {
        *length = -1;
        return CS_OK;
    }
    const int64_t lo = whole ? -1 : i, hi = whole ? n : j;
    int64_t g = (row_words + 255) / 256;
    k_chain_init<<<unsigned(g < 1 ? 1 : g), 256, 0, st>>>(bits_dev, n, row_words, whole ? -1 : i, j, S, M, sd);
    ChainState h{};
    // one cooperative launch for all rounds when the device allows it
    const int cg = coop_grid(reinterpret_cast<const void*>(k_chain_persist), hi - lo - 1);
    if (cg > 0) {
        k_count_bits<<<1, 1024, 0, st>>>(S, row_words, sd);  // |S| at the start into rounds
        if (cudaGetLastError() != cudaSuccess || read_state(sd, &h, st) != cudaSuccess) return CS_ECUDA;
        if (!h.related) {
            *length = -1;
            return CS_OK;
        }
        if (h.rounds == 0) {  // empty interval: a link, or an empty set
            *length = whole ? 0 : 1;
            return CS_OK;
        }
        WsHeader* hdr = reinterpret_cast<WsHeader*>(ws);
        if (cudaMemsetAsync(&sd->bar_count, 0, sizeof(unsigned int) * 2 + sizeof(unsigned long long) * 4, st) !=
                cudaSuccess ||
            cudaMemsetAsync(&sd->rounds, 0xFF, sizeof(int64_t), st) != cudaSuccess ||  // -1 until the last round
            cudaMemsetAsync(&hdr->status, 0, sizeof(int32_t), st) != cudaSuccess)
            return CS_ECUDA;
        int64_t max_rounds = n + 1;
        void* args[] = {const_cast<uint64_t**>(&bits_dev), &row_words, const_cast<int64_t*>(&lo),
                        const_cast<int64_t*>(&hi), &max_rounds, &S, &M, &sd, &hdr};
        if (cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k_chain_persist), dim3(unsigned(cg)), dim3(256),
                                        args, 0, st) == cudaSuccess) {
            int32_t status = 0;
            if (read_state(sd, &h, st) != cudaSuccess ||
                cudaMemcpy(&status, &hdr->status, sizeof(status), cudaMemcpyDeviceToHost) != cudaSuccess)
                return CS_ECUDA;
            if (status != 0) return status;
            if (h.rounds < 0) return CS_ERANGE;  // cannot happen for a transitive relation
            *length = whole ? h.rounds : h.rounds + 1;
            return CS_OK;
        }
        cudaGetLastError();  // not launched: clear and take the multi-launch path
        k_chain_init<<<unsigned(g < 1 ? 1 : g), 256, 0, st>>>(bits_dev, n, row_words, whole ? -1 : i, j, S, M, sd);
    }
    for (int64_t done = 0; done <= n; done += kBatch) {  // at most n + 1 rounds remove anything
        for (int r = 0; r < kBatch; ++r) {
            k_chain_peel<<<warp_grid(hi - lo - 1), 256, 0, st>>>(bits_dev, row_words, lo, hi, S, M, sd);
            k_chain_apply<<<1, 1024, 0, st>>>(row_words, S, M, sd);
        }
        if (cudaGetLastError() != cudaSuccess || read_state(sd, &h, st) != cudaSuccess) return CS_ECUDA;
        if (h.left == 0 || !h.related) break;
    }
    if (h.left != 0 && h.related) return CS_ERANGE;  // cannot happen for a transitive relation
    *length = whole ? h.rounds : (h.related ? h.rounds + 1 : -1);
    return CS_OK;
}

extern "C" int cs_greedy_antichain(int64_t n, const uint64_t* bits_dev, int64_t row_words, int64_t seed,
                                   uint64_t* members_dev, int64_t* size, void* workspace_dev, size_t workspace_bytes,
                                   void* stream) {
    CS_TRACE("cs_greedy_antichain");
    if (!chain_args_ok(n, bits_dev, row_words, workspace_dev) || seed < 0 || seed >= n || !members_dev ||
        (reinterpret_cast<uintptr_t>(members_dev) % 8) != 0 || !size)
        return CS_EINVAL;
    const ChainLayout L = chain_layout(row_words);
    if (workspace_bytes < L.total) return CS_ENOMEM;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    uint8_t* ws = static_cast<uint8_t*>(workspace_dev);
    ChainState* sd = reinterpret_cast<ChainState*>(ws + L.state);
    uint64_t* X = reinterpret_cast<uint64_t*>(ws + L.s);
    int64_t g = (row_words + 255) / 256;
    k_anti_init<<<unsigned(g < 1 ? 1 : g), 256, 0, st>>>(bits_dev, n, row_words, seed, members_dev, X, sd);
    ChainState h{};
    const int cg = coop_grid(reinterpret_cast<const void*>(k_anti_persist), n);
    bool done = false;
    if (cg > 0) {
        WsHeader* hdr = reinterpret_cast<WsHeader*>(ws);
        int32_t* over = reinterpret_cast<int32_t*>(ws + L.over);
        int32_t* rlist = reinterpret_cast<int32_t*>(ws + L.rlist);
        if (cudaMemsetAsync(&sd->bar_count, 0, sizeof(unsigned int) * 2 + sizeof(unsigned long long) * 2, st) !=
                cudaSuccess ||
            cudaMemsetAsync(&sd->best2[0], 0xFF, sizeof(unsigned long long), st) != cudaSuccess ||  // no best yet
            cudaMemsetAsync(&sd->rcount[0], 0, sizeof(unsigned int) * 2, st) != cudaSuccess ||
            cudaMemsetAsync(&hdr->status, 0, sizeof(int32_t), st) != cudaSuccess)
            return CS_ECUDA;
        int64_t max_rounds = n + 1;
        void* args[] = {const_cast<uint64_t**>(&bits_dev), &n, &row_words, &max_rounds, &members_dev, &X,
                        &over, &rlist, &sd, &hdr};
        if (cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k_anti_persist), dim3(unsigned(cg)), dim3(256),
                                        args, 0, st) == cudaSuccess) {
            int32_t status = 0;
            if (cudaStreamSynchronize(st) != cudaSuccess ||
                cudaMemcpy(&status, &hdr->status, sizeof(status), cudaMemcpyDeviceToHost) != cudaSuccess)
                return CS_ECUDA;
            if (status != 0) return status;
            done = true;
        } else {
            cudaGetLastError();
            k_anti_init<<<unsigned(g < 1 ? 1 : g), 256, 0, st>>>(bits_dev, n, row_words, seed, members_dev, X, sd);
        }
    }
    for (int64_t rounds = 0; !done && rounds <= n; rounds += kBatch) {  // multi-launch path
        for (int r = 0; r < kBatch; ++r) {
            k_anti_score<<<warp_grid(n), 256, 0, st>>>(bits_dev, n, row_words, members_dev, X, sd);
            k_anti_apply<<<1, 1024, 0, st>>>(bits_dev, row_words, members_dev, X, sd);
        }
        if (cudaGetLastError() != cudaSuccess || read_state(sd, &h, st) != cudaSuccess) return CS_ECUDA;
        if (h.left == 0) done = true;
    }
    if (!done) return CS_ERANGE;
    k_count_bits<<<1, 1024, 0, st>>>(members_dev, row_words, sd);
    if (cudaGetLastError() != cudaSuccess || read_state(sd, &h, st) != cudaSuccess) return CS_ECUDA;
    *size = h.rounds;
    return CS_OK;
}

