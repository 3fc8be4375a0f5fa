// cs_relate.cu -- the causal matrix as row bitsets (Section "Data Structures
// for Totally Ordered Sets": the symmetrised matrix P + P^T, one bitset per
// row; Section "Lorentzian Geometry": related iff Delta s^2 < 0).
//
// A block owns 2048 columns (32 words) and 64 rows.  Column coordinates are
// staged once in shared memory; each warp walks its rows, and for every word
// its 32 lanes test 64 columns and fold the answers into the word with two
// __ballot_sync.  Lane w keeps word w, so a row's 32 words leave in one
// coalesced 256-byte store.  The tests are symmetric (du*dv > 0 in 2D,
// dt^2 - |dx|^2 > 0 in 4D, exact in int64), so no branch on i < j is needed.
#include "cs_kernels.cuh"

namespace cs {

namespace {

constexpr int kColsPerBlock = 2048;
constexpr int kWordsPerBlock = kColsPerBlock / 64;
constexpr int kRowsPerBlock = 64;
constexpr int kThreads = 256;

template <int DIM>
__device__ __forceinline__ bool related(const int32_t (&ci)[DIM], const int32_t (*sc)[kColsPerBlock], int col) {
    if constexpr (DIM == 2) {
        const int64_t du = int64_t(sc[0][col]) - ci[0];
        const int64_t dv = int64_t(sc[1][col]) - ci[1];
        return du * dv > 0;
    } else {
        const int64_t dt = int64_t(sc[0][col]) - ci[0];
        const int64_t dx = int64_t(sc[1][col]) - ci[1];
        const int64_t dy = int64_t(sc[2][col]) - ci[2];
        const int64_t dz = int64_t(sc[3][col]) - ci[3];
        return dt * dt - (dx * dx + dy * dy + dz * dz) > 0;
    }
}

template <int DIM>
__global__ void __launch_bounds__(kThreads) k_relate(const int32_t* __restrict__ coords, int64_t n,
                                                     uint64_t* __restrict__ bits, int64_t row_words) {
    __shared__ int32_t sc[DIM][kColsPerBlock];
    const int64_t w0 = int64_t(blockIdx.y) * kWordsPerBlock;
    const int64_t c0 = w0 * 64;
    for (int t = threadIdx.x; t < kColsPerBlock; t += kThreads) {
        const int64_t c = c0 + t;
#pragma unroll
        for (int d = 0; d < DIM; ++d) sc[d][t] = c < n ? coords[d * n + c] : 0;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t r0 = int64_t(blockIdx.x) * kRowsPerBlock;
    const int64_t r1 = r0 + kRowsPerBlock < n ? r0 + kRowsPerBlock : n;
    for (int64_t i = r0 + warp; i < r1; i += kThreads / 32) {
        int32_t ci[DIM];
#pragma unroll
        for (int d = 0; d < DIM; ++d) ci[d] = coords[d * n + i];
        uint64_t mine = 0;
#pragma unroll 4
        for (int w = 0; w < kWordsPerBlock; ++w) {
            const int col = w * 64 + lane;
            const bool b0 = c0 + col < n && related<DIM>(ci, sc, col);
            const bool b1 = c0 + col + 32 < n && related<DIM>(ci, sc, col + 32);
            const uint32_t lo = __ballot_sync(0xffffffffu, b0);
            const uint32_t hi = __ballot_sync(0xffffffffu, b1);
            if (lane == w) mine = (uint64_t(hi) << 32) | lo;
        }
        if (w0 + lane < row_words) bits[i * row_words + w0 + lane] = mine;
    }
}

}  // namespace

cudaError_t launch_relate(int kind, int64_t n, const int32_t* coords, uint64_t* bits, int64_t row_words,
                          cudaStream_t st) {
    dim3 grid(unsigned((n + kRowsPerBlock - 1) / kRowsPerBlock),
              unsigned((row_words + kWordsPerBlock - 1) / kWordsPerBlock));
    if (kind == CS_4D_DIAMOND)
        k_relate<4><<<grid, kThreads, 0, st>>>(coords, n, bits, row_words);
    else
        k_relate<2><<<grid, kThreads, 0, st>>>(coords, n, bits, row_words);
    return cudaGetLastError();
}

}  // namespace cs
