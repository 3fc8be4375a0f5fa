// cs_relate.cu -- the causal matrix as row bitsets (Section "Data Structures
// for Totally Ordered Sets": the symmetrised matrix P + P^T, one bitset per
// row; Section "Lorentzian Geometry": related iff Delta s^2 < 0).
//
// A block owns 2048 columns (32 words) and 64 rows (relate_block): column
// coordinates are staged once in shared memory, and each lane owns one
// 64-column word of a row.  For the words wholly after the row (labels are
// in time order, so only the future cone can hold there) the lane builds
// the word from the sign bits of integer multiply-adds (light cone) or of
// an FP32 filter with an exact int64 recompute near the cone (2+1, 3+1),
// funnel-shifting one sign per column into the word; the row's own word,
// which holds the diagonal, takes the full symmetric test by two
// __ballot_sync.  A row's words leave in coalesced stores.  64 x 64 tiles
// wholly below the diagonal are not tested: k_mirror fills them as bit
// transposes of the tiles above (the relation is symmetric), which halves
// the tests.
#include "cs_kernels.cuh"
#include "cs_relate.cuh"

namespace cs {

namespace {

template <int G>
__global__ void __launch_bounds__(kRelThreads) k_relate(const int32_t* __restrict__ coords, int64_t n,
                                                        uint64_t* __restrict__ bits, int64_t row_words, bool order2d) {
    // the light-cone kinds stage (u, v) transposed: 64 x 33 int2 and a 1; the
    // filtered 2+1 and 3+1 tests one float4 per column
    constexpr int kInts = G == kGeomLightCone                ? kConeInts
                          : (G == kGeom3 || G == kGeom4)     ? kStageInts
                                                             : geom_dim(G) * kRelColsPerBlock;
    __shared__ __align__(16) int32_t sc[kInts];
    relate_block<G>(coords, n, bits, row_words, blockIdx.x, int64_t(blockIdx.y) * kRelWordsPerBlock, sc, order2d);
}

__global__ void __launch_bounds__(kRelThreads, 4) k_mirror(uint64_t* __restrict__ bits, int64_t n, int64_t row_words) {
    __shared__ uint64_t sm[kMirRows][kMirTiles + 1];
    mirror_block(bits, n, row_words, blockIdx.x, blockIdx.y, sm);
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
    else if (kind == CS_2D_DS_SLAB || kind == CS_2D_CYLINDER)
        k_relate<kGeomDeSitter><<<grid, kRelThreads, 0, st>>>(coords, n, bits, row_words, false);
    else
        k_relate<kGeomLightCone><<<grid, kRelThreads, 0, st>>>(coords, n, bits, row_words, kind == CS_2D_ORDER);
    const int64_t st8 = ((n + 63) / 64 + kMirTiles - 1) / kMirTiles;  // super-tiles per side
    if (st8 > 0) k_mirror<<<dim3(unsigned(st8), unsigned(st8)), kRelThreads, 0, st>>>(bits, n, row_words);
    return cudaGetLastError();
}

}  // namespace cs
