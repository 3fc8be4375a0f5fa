// cs_relate.cu -- the causal matrix as row bitsets (Section "Data Structures
// for Totally Ordered Sets": the symmetrised matrix P + P^T, one bitset per
// row; Section "Lorentzian Geometry": related iff Delta s^2 < 0).
//
// A block owns 2048 columns (32 words) and 64 rows (relate_block): column
// coordinates are staged once in shared memory, each warp folds 64 tests per
// word into a uint64 with two __ballot_sync, and a row's 32 words leave in
// one coalesced 256-byte store.  The tests are symmetric and exact in int64,
// so no branch on i < j is needed.
#include "cs_kernels.cuh"
#include "cs_relate.cuh"

namespace cs {

namespace {

template <int G>
__global__ void __launch_bounds__(kRelThreads) k_relate(const int32_t* __restrict__ coords, int64_t n,
                                                        uint64_t* __restrict__ bits, int64_t row_words, bool order2d) {
    __shared__ int32_t sc[geom_dim(G)][kRelColsPerBlock];
    relate_block<G>(coords, n, bits, row_words, blockIdx.x, blockIdx.y, sc, order2d);
}

}  // namespace

cudaError_t launch_relate(int kind, int64_t n, const int32_t* coords, uint64_t* bits, int64_t row_words,
                          cudaStream_t st) {
    dim3 grid(unsigned((n + kRelRowsPerBlock - 1) / kRelRowsPerBlock),
              unsigned((row_words + kRelWordsPerBlock - 1) / kRelWordsPerBlock));
    if (kind == CS_4D_DIAMOND)
        k_relate<kGeom4><<<grid, kRelThreads, 0, st>>>(coords, n, bits, row_words, false);
    else if (kind == CS_3D_DIAMOND)
        k_relate<kGeom3><<<grid, kRelThreads, 0, st>>>(coords, n, bits, row_words, false);
    else if (kind == CS_2D_DS_SLAB)
        k_relate<kGeomDeSitter><<<grid, kRelThreads, 0, st>>>(coords, n, bits, row_words, false);
    else
        k_relate<kGeomLightCone><<<grid, kRelThreads, 0, st>>>(coords, n, bits, row_words, kind == CS_2D_ORDER);
    return cudaGetLastError();
}

}  // namespace cs
