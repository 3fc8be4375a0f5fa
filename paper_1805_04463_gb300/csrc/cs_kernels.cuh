// cs_kernels.cuh -- launchers shared between the translation units of the library.
#pragma once

#include "cs_internal.cuh"

namespace cs {

// cs_sprinkle.cu
size_t sprinkle_workspace_bytes(int64_t n);
// Device copy of the de Sitter slab's cumulative eta thresholds (uploaded
// once per device, synchronously, on first use); nullptr on failure, and a
// failed upload is tried again on the next call.
const uint64_t* ds_table_device();
cudaError_t launch_sprinkle(int kind, int64_t n, uint64_t seed, int32_t* coords, void* workspace,
                            cudaStream_t st);

// cs_relate.cu
cudaError_t launch_relate(int kind, int64_t n, const int32_t* coords, uint64_t* bits, int64_t row_words,
                          cudaStream_t st);

// cs_count_popc.cu
// One set of a multi-set POPC count: its TMA map, bitset, size, tile range and
// histogram offset.  128-byte aligned like the embedded tensor map.
struct alignas(128) PopcSetEntry {
    CUtensorMap map;
    const uint64_t* bits;
    int64_t n, row_words, nb;
    int64_t item_begin;   // first tile of this set in the concatenated tile list
    int64_t item_offset;  // tile index (within the set) of that first tile
    int64_t hist_off;     // byte offset of this set's histogram from the launch's histogram base
    const double* phi;    // d'Alembertian layer sums: field (NULL = 1),
    double* layer;        //   sums [kmax+1][n],
    int64_t kmax;         //   highest layer (< 0: none)
};
size_t popc_workspace_bytes(int64_t n);
int64_t popc_tiles(int64_t n);
void popc_fill_entry(PopcSetEntry* e, const uint64_t* bits, int64_t n, int64_t row_words);
CUresult popc_encode_map(CUtensorMap* map, const uint64_t* bits, int64_t n, int64_t row_words);
cudaError_t launch_count_popc_multi(const PopcSetEntry* sets_dev, int nsets, int64_t ntiles, uintptr_t hist_base,
                                    WsHeader* hdr, int max_ctas, cudaStream_t st);
cudaError_t launch_count_popc(int64_t n, const uint64_t* bits, int64_t row_words, int64_t* hist,
                              void* workspace, cudaStream_t st, const double* phi = nullptr, double* layer = nullptr,
                              int kmax = -1);

// cs_count_mma.cu
// TMA maps of one set's operands.  FP8 (CS_PATH_MMA): U and L, the masked
// future and past rows.  FP4 pairs (CS_PATH_MMA4): E, every row of the
// symmetric matrix unmasked, and the masked diagonal blocks DU (each row's own
// 256-column block, columns after the row) and DL (columns before it).
constexpr int kMapU = 0, kMapL = 1;
constexpr int kMapE = 0, kMapDU = 1, kMapDL = 2;
struct MmaMaps {
    CUtensorMap m[3];
};
// One set of a multi-set tensor-core count: TMA maps of its operands,
// bitset, sizes, item range, histogram offset, and where its operands live.
struct alignas(128) MmaSetEntry {
    MmaMaps maps;
    const uint64_t* bits;
    int64_t n, row_words, nsb, kblocks;
    int64_t item_begin;   // first item of this set in the concatenated item list
    int64_t item_offset;  // item index (within the set) of that first item
    int64_t hist_off;     // byte offset of this set's histogram from the launch's histogram base
    uint8_t* op0;         // FP8: U; FP4: E
    uint8_t* op1;         // FP8: L; FP4: DU, then DL at mma4_dl_offset(n)
    int64_t kpad;
    int64_t chunk_begin;  // first expansion chunk of this set (multi-set expansion)
    const double* phi;   // d'Alembertian layer sums: field (NULL = 1),
    double* layer;       //   sums [kmax+1][n],
    int64_t kmax;        //   highest layer (< 0: none)
};
// Packed FP4 (E2M1) 0/1 operands.  Bits 0..7 of x -> 8 nibbles of 0x0 / 0x2
// (bit b -> nibble b): three shift-and-mask steps move bit groups of 4, 2
// and 1 apart (no carries), then the shift by one turns each 1 into 0x2 = 1.0
// in E2M1.  Element k of a row sits in byte k/2, low nibble for even k; A
// and B use the same packing, so every product pairs the same columns
// whatever nibble order the MMA reads.
__device__ __forceinline__ uint32_t spread8_e2m1(uint32_t x) {
    x &= 0xFFu;
    x = (x | (x << 12)) & 0x000F000Fu;
    x = (x | (x << 6)) & 0x03030303u;
    x = (x | (x << 3)) & 0x11111111u;
    return x << 1;
}

// 32 bits of a bitset row -> 16 operand bytes.
__device__ __forceinline__ uint4 spread32_e2m1(uint32_t b) {
    return make_uint4(spread8_e2m1(b), spread8_e2m1(b >> 8), spread8_e2m1(b >> 16), spread8_e2m1(b >> 24));
}

// fp4 selects the packed-FP4 operand format of the pair path (CS_PATH_MMA4):
// K padded to 256 elements, two per byte; its work unit is a 256 x 256
// supertile (mma4_units per set) instead of a 128 x 256 tile (mma_items).
// Work items of a set: slots of 128 x 256 tiles (FP8) or units of 256 x 256
// supertiles (FP4 pairs) in raster blocks of side `raster`.  The multi-set
// counts use kRasterDefault; the single-set counts auto_raster(n).
constexpr int kRasterDefault = 8;
size_t mma_workspace_bytes(int64_t n);
int64_t mma_items(int64_t n, int raster = kRasterDefault);
int64_t mma4_units(int64_t n, int raster = kRasterDefault);
int64_t mma_kpad(int64_t n, bool fp4 = false);
// Bytes of a set's first (U, or E) and second (L, or DU and DL) operand buffer.
size_t mma_operand_bytes(int64_t n, bool fp4, int which);
// DL within the second FP4 buffer: after n DU rows of 128 bytes, 1024-byte aligned.
__host__ __device__ inline int64_t mma4_dl_offset(int64_t n) { return (n * 128 + 1023) / 1024 * 1024; }
// Fill sizes, operand pointers and TMA maps of an entry (item_begin, hist_off,
// chunk_begin are the caller's).  op0, op1: 1024-byte aligned.
CUresult mma_fill_entry(MmaSetEntry* e, const uint64_t* bits, int64_t n, int64_t row_words, uint8_t* op0,
                        uint8_t* op1, bool fp4 = false);
// uses bits, n, row_words, kpad, op0, op1
cudaError_t launch_expand_single(const MmaSetEntry* e, cudaStream_t st, bool fp4 = false);
// Expansion of many sets: chunk c of the concatenated chunk range belongs to
// set chunk_set[c] (a table the caller builds; mma_expand_chunks(n) chunks per
// set, numbered from the set's chunk_begin).
int64_t mma_expand_chunks(int64_t n);
cudaError_t launch_expand_multi(const MmaSetEntry* sets_dev, const int32_t* chunk_set, int64_t total_chunks,
                                cudaStream_t st, bool fp4 = false);
cudaError_t launch_count_mma_multi(const MmaSetEntry* sets_dev, int nsets, int64_t nitems, uintptr_t hist_base,
                                   WsHeader* hdr, int max_ctas, cudaStream_t st);
// The FP4 pair path over many sets: entries filled with fp4 = true, their
// item_begin / item_offset counted in supertiles, nunits supertiles in all.
cudaError_t launch_count_mma4_multi(const MmaSetEntry* sets_dev, int nsets, int64_t nunits, uintptr_t hist_base,
                                    WsHeader* hdr, cudaStream_t st);
cudaError_t launch_count_mma(int64_t n, const uint64_t* bits, int64_t row_words, int64_t* hist,
                             void* workspace, cudaStream_t st, const double* phi = nullptr, double* layer = nullptr,
                             int kmax = -1);
// The single-set count on packed FP4 operands (kind::mxf4, unit scales).
// mma4_workspace_bytes: the whole set's operands.  mma4_band_panels: the
// supertile rows per group when the operands go through a band buffer of
// `bytes` (nsb = (n + 255) / 256 when the whole set fits, 0 when not even a
// band of one panel does); mma4_band_bytes: the workspace of bands of g
// panels (the whole set's for g >= nsb).  The count takes the widest bands
// its workspace holds.
size_t mma4_workspace_bytes(int64_t n);
int64_t mma4_band_panels(int64_t n, size_t bytes);
size_t mma4_band_bytes(int64_t n, int64_t g);
// Host check of the band plan: counts[si * nsb + sj] (nsb^2 entries, zeroed
// here) = how many work items of all band launches of bands of g panels and
// raster side `raster` decode to supertile (si, sj); returns the item count.
int64_t mma4_band_cover(int64_t n, int64_t g, int raster, int64_t* counts);
cudaError_t launch_count_mma4(int64_t n, const uint64_t* bits, int64_t row_words, int64_t* hist,
                              void* workspace, size_t ws_bytes, cudaStream_t st, const double* phi = nullptr,
                              double* layer = nullptr, int kmax = -1);

// CS_OK for cudaSuccess; otherwise CS_ECUDA, remembering the error for
// cs_last_cuda_error (per host thread).
int cuda_status(cudaError_t e);

// Path chosen for CS_PATH_AUTO at size n.
int resolve_path(int64_t n, int path);
// Tile choices (cs_set_auto_tiles, cs_set_batch_tuning): the raster side of
// a single-set tensor count of size n; the path CS_PATH_AUTO plans for
// batches and count jobs; the longest run of consecutive work items a CTA
// takes from the queue of a multi-set count.
int auto_raster(int64_t n);
int batch_auto_path();
int batch_max_run();

// cs_action.cu
int action_host(int dim, int64_t n, const int64_t* hist, int64_t len, double eps, double* out,
                int64_t* bracket);
size_t action_workspace_bytes();
cudaError_t launch_action_device(int dim, int64_t n, const int64_t* hist, int64_t len, const double* eps,
                                 int n_eps, double* out, int64_t* bracket, void* workspace, cudaStream_t st);

cudaError_t launch_dalembertian(int dim, int64_t n, const double* phi, const double* layer, double ell, double* out,
                                cudaStream_t st);

// cs_selftest.cu: host fault injection (cs_inject_fault).  True when the
// step `where` (a CS_FAULT_* bit) must fail this time.
bool fault_injected(int where);

// Device properties cached per device.
int device_sm_count();
bool device_has_tcgen05();
size_t device_total_memory();  // bytes of device memory (0 if unknown)

// cuTensorMapEncodeTiled, resolved once through the runtime's driver entry point.
CUresult encode_tensor_map_2d(CUtensorMap* map, CUtensorMapDataType type, void* base, uint64_t dim0,
                              uint64_t dim1, uint64_t stride1_bytes, uint32_t box0, uint32_t box1,
                              CUtensorMapSwizzle swizzle);

}  // namespace cs
