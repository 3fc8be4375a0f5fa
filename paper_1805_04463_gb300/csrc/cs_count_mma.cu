// cs_count_mma.cu -- interval abundances as an exact dense contraction on the
// tcgen05 tensor cores (Figure "Proper distance and the order intervals": the
// interval of a related pair is the inner product of rows i and j between
// columns i and j, i.e. (C.C)_ij for the strict upper triangle C).
//
// Operands (FP8 path).  The symmetric bitset is expanded once into two
// K-major byte matrices of 0/1 values in FP8 E4M3 (1.0 = 0x38):
//   U[i][k] = 1 iff k > i and i, k related   (row i = future of i, F_i)
//   L[j][k] = 1 iff k < j and j, k related   (row j = past of j,  P_j)
// so M = U . L^T holds |A_ij| = sum_k U_ik L_jk with no masking at all: the
// zeros of U (k <= i) and L (k >= j) restrict k to i < k < j.  Products are 0
// or 1 and every partial sum is an integer below 2^24, so FP32 accumulation
// is exact.  The FP4 pair path needs the masks only in the two K-blocks that
// hold the supertile's own bands, so it keeps one unmasked matrix E of the
// symmetric relation plus the masked diagonal blocks DU and DL (below, at
// the FP4 expansion): half the operand memory.
//
// Kernel.  A persistent grid (one CTA per SM) walks 128 x 256 output tiles
// (128 i-rows, 256 j-rows, i-block at or before the j-block), rasterised in
// 8 x 8 blocks of 256 x 256 supertiles served widest band first from one
// global queue, so the CTAs running at any moment share operand panels in
// L2.  Warp roles:
//   warp 0      queue and TMA producer: takes the next item, hands its index
//               to the other roles through a 4-slot shared ring, and loads a
//               128-row A slab and a 256-row B slab of 128 K-bytes per stage
//               (128B swizzle) into a 4-stage shared-memory ring;
//   warp 1      TMEM allocator and MMA issuer: 4 x tcgen05.mma (M128 N256 K32)
//               per stage into one of two TMEM accumulators (2 x 256 columns);
//   warps 2..17 epilogue: tcgen05.ld of the finished accumulator (one TMEM
//               lane = one row i per thread; four warps per lane quarter, each
//               taking a quarter of the 256 columns), mask by i < j < n and C_ij
//               from the bitset, bucket k into a shared-memory histogram
//               (global atomics above 8192), then release the accumulator.
// The K loop of a tile runs only over the K-blocks between the i-block and the
// end of the j-block.  C.C is never written to memory.
#include <atomic>
#include <cstring>
#include <vector>

#include "cs_kernels.cuh"

namespace cs {

namespace {

constexpr int kBM = 128;                 // i rows per tile (TMEM lanes)
constexpr int kBN = 256;                 // j rows per tile (accumulator columns)
constexpr int kBK = 128;                 // K bytes per stage and operand row = one swizzle row (128 or 64)
constexpr int kUK = 32;                  // K bytes per tcgen05.mma (K32 FP8 or K64 packed FP4)
constexpr int kABytes = kBM * kBK;       // 16 KiB
constexpr int kBBytes = kBN * kBK;       // 32 KiB
constexpr int kStageBytes = kABytes + kBBytes;
// A tile adds at most 128 x 256 to a CTA's shared bin; flushing every 32768
// tiles keeps the 32-bit bins below 2^30 whatever the order.
constexpr int64_t kFlushTiles = 32768;
constexpr int kEpiWarps = 16;            // four epilogue warps per TMEM lane quarter
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr int kSchedWarp = 2 + kEpiWarps;  // the scheduler: finds, decodes and publishes the items
constexpr int kThreads = 64 + kEpiThreads + 32;
// Registers per thread of the count kernels, set explicitly (__maxnreg__):
// the warps of a CTA spread over the SM's four register-file quarters of
// 16384 registers, so the fullest quarter (ceil(19 / 4) = 5 warps) must hold
// 5 x 32 x kMaxRegs; 104 registers would not launch.
constexpr int kMaxRegs = 96;
static_assert((kThreads / 32 + 3) / 4 * 32 * kMaxRegs <= 16384, "the fullest register-file quarter fits");
constexpr int kEpiChunks = (kBN / 32) / (kEpiWarps / 4);  // 32-column chunks per epilogue warp
static_assert(kEpiWarps % 4 == 0 && (kBN / 32) % (kEpiWarps / 4) == 0, "epilogue warps split the columns evenly");
constexpr int kTmemCols = 512;           // two 256-column FP32 accumulators, or one and the FP4 scales
constexpr uint32_t kIdesc = idesc_f8_f32(kBM, kBN);
constexpr uint32_t kIdesc4 = idesc_mxf4_f32(kBM, kBN);
constexpr uint32_t kSfCol = 256;         // FP4: scale factors of A at this TMEM column, of B 16 further
constexpr uint32_t kScaleOne = 0x7F7F7F7Fu;  // four UE8M0 scale factors 2^0 = 1
constexpr int kRing = 4;                 // items in flight between the roles
constexpr int kBarrierBytes = 512;       // mbarriers, item ring, TMEM address, abort flag
constexpr uint8_t kOne = 0x38;           // 1.0 in FP8 E4M3

// Operand formats.  A stage holds one 128-byte swizzle row of K per operand
// row in both; they differ in how many K elements those bytes carry.
//   FmtF8: kind::f8f6f4, one E4M3 byte per element, two TMEM accumulators
//          (the epilogue of one tile overlaps the MMAs of the next).
//   FmtF4: kind::mxf4 (block-scaled), two E2M1 nibbles per byte (1.0 = 0x2)
//          with every scale factor 1, so products are again 0 or 1; one
//          accumulator, because the scale factors take TMEM columns too --
//          the epilogue copies it to registers and releases it at once.
// kLayers: the kernel may add d'Alembertian layer sums (kmax >= 0);
// kSmallSet: it has the branch-free epilogue for sets whose histogram fits
// in shared memory.  The FP4 kernel holds 64 accumulator values per thread
// and needs every register for them, so it comes in two builds: counts only
// (the large sets it is for) and counts with layer sums.
// kPair: a CTA pair (a cluster of two) runs each 256 x 256 supertile as one
// 2-SM MMA (tcgen05 cta_group::2, M = 256): CTA r loads A rows 128r.. and B
// rows 128r.. of the supertile into its own shared memory, rank 0 issues
// the MMAs, which read both CTAs' halves, and each CTA's TMEM receives its
// 128 accumulator rows.  A stage then costs each SM 32 KiB (16 of A, 16 of
// B) for the multiply-adds that take 48 KiB on one SM: the single-SM
// kernels are bound by shared-memory traffic per MAC (TMA writes plus
// tensor-core reads), and six stages fit instead of four.  Both halves run
// the same K range, which wastes nothing when K-blocks hold 256 elements.
// kStages and kHistBins split the shared memory between the operand ring
// and the privatised histogram (bins at or above kHistBins go to global
// atomics).  Both stay at their largest joint size: a seventh FP4 stage with
// 256 shared bins (96% of the counts of a 2^17 order then global atomics,
// against 52% with 8192 bins) made the count 24% slower at n = 2^17 and
// 2.9x slower at 2^15, the L2 atomics competing with the operand loads
// (the multi-set form below, whose tiles are short, takes five stages).
struct FmtF8 {
    static constexpr int kKE = kBK;      // K elements per stage
    static constexpr int kAcc = 2;
    static constexpr bool kLayers = true, kSmallSet = true, kPair = false;
    static constexpr int kStages = 4, kHistBins = 8192;
};
struct FmtF4 {
    static constexpr int kKE = 2 * kBK;
    static constexpr int kAcc = 1;
    static constexpr bool kLayers = false, kSmallSet = false, kPair = true;
    static constexpr int kStages = 6, kHistBins = 8192;
};
struct FmtF4Layers : FmtF4 {
    static constexpr bool kLayers = true;
};
// The multi-set form: its sets are small (a batch holds n <= 8192, a count
// job any n), so it keeps the branch-free histogram of the FP8 kernel for
// sets whose histogram fits in shared memory.  Its tiles hold few K-blocks
// (4-6 at n = 4096), and five stages suit them best: a 768-set batch of
// n ~ 2048-4096 replayed in 8.43 ms with 5, 8.45 with 4, 8.59 with 6,
// 8.80 with 3 and 9.27 with 2.
struct FmtF4Multi : FmtF4 {
    static constexpr bool kSmallSet = true;
    static constexpr int kStages = 5;
};
// Bytes of one operand stage in each CTA, and the dynamic shared memory of
// a kernel on format Fmt (the base is rounded up to 1024 inside).
template <class Fmt>
constexpr int stage_bytes() { return kABytes + (Fmt::kPair ? kBN / 2 : kBN) * kBK; }
template <class Fmt>
constexpr int smem_bytes() { return Fmt::kStages * stage_bytes<Fmt>() + Fmt::kHistBins * 4 + kBarrierBytes + 1024; }
static_assert(smem_bytes<FmtF8>() <= 232448 && smem_bytes<FmtF4>() <= 232448 && smem_bytes<FmtF4Multi>() <= 232448,
              "227 KiB of shared memory per CTA");
constexpr CUtensorMapSwizzle kSwizzle = kBK == 128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B;
static_assert(kBK == 128 || kBK == 64, "one 128- or 64-byte swizzle row per stage");
static_assert(kStageBytes % 1024 == 0 && kABytes % 1024 == 0, "stage buffers stay swizzle-atom aligned");

// Items.  Pairs are covered by 256 x 256 supertiles (si <= sj), each split
// into two 128-row halves (one MMA tile each).  Supertiles are grouped into
// R x R raster blocks; blocks are served from the widest band
// (longest K) to the diagonal, and the 2 * R^2 slots of a block are
// consecutive item indices.  CTAs that run at the same time therefore share
// A panels (same si) and B panels (same sj) through L2 instead of each
// streaming its own operands from HBM.  Slots with si > sj, or beyond n,
// decode to nothing: the producer skips them, and hands the other roles
// only the valid items, already decoded (pack_item).
// The raster side R is a runtime parameter of the single-set counts (the
// autotuner may choose it per size); the multi-set counts (batches, count
// jobs) keep kRasterDefault, so a set's item list is fixed for them.

struct Item {
    int64_t I0, J0;
    int64_t kb0, kb1;  // K-blocks [kb0, kb1)
};

// Slot t of a set's item list -> supertile (si, sj) and its 128-row half;
// false for a slot that holds no work.
__host__ __device__ __forceinline__ bool decode_slot(int64_t t, int64_t nsb, int64_t n, int64_t R, int64_t& si, int64_t& sj,
                                            int64_t& half) {
    const int64_t spb = 2 * R * R;  // slots per raster block
    const int64_t blk = t / spb, slot = t - blk * spb;
    const int64_t nbg = (nsb + R - 1) / R;
    int64_t m = int64_t((1.0f + sqrtf(1.0f + 8.0f * float(blk))) * 0.5f);  // corrected below
    while (m * (m - 1) / 2 > blk) --m;
    while (m * (m + 1) / 2 <= blk) ++m;
    const int64_t gi = blk - m * (m - 1) / 2;
    const int64_t gj = gi + (nbg - m);
    si = gi * R + slot / (2 * R);
    const int64_t rem = slot % (2 * R);
    sj = gj * R + rem / 2;
    half = rem & 1;
    return si <= sj && sj < nsb && si * 256 + half * kBM < n;
}

// A band of the FP4 pair count, for sets whose full operand matrix does not
// fit the workspace: the supertiles with si in panels [i0, i0 + ni) and sj in
// [j0, j0 + nj) -- a triangle when the two ranges are the same (diag), else
// a rectangle wholly above the diagonal -- whose E rows sit in a band buffer
// (row I of the set at band row I - erow_i as an A row, J - erow_j as a B
// row).  The whole set is the one band {0, 0, nsb, nsb, 0, 0, 1}.
struct MmaBand {
    int64_t i0, j0, ni, nj;
    int64_t erow_i, erow_j;
    int diag;
};

// Slot t of a band's item list -> supertile (si, sj) of the set and its half.
// The rectangle is rasterised like the triangle: R x R blocks, row by row.
__host__ __device__ __forceinline__ bool decode_band(int64_t t, const MmaBand& b, int64_t n, int64_t R, int64_t& si,
                                            int64_t& sj, int64_t& half) {
    if (b.diag) {
        if (!decode_slot(t, b.ni, n - b.i0 * 256, R, si, sj, half)) return false;
        si += b.i0;
        sj += b.i0;
        return true;
    }
    const int64_t spb = 2 * R * R;
    const int64_t blk = t / spb, slot = t - blk * spb;
    const int64_t nbj = (b.nj + R - 1) / R;
    const int64_t gi = blk / nbj, gj = blk - gi * nbj;
    si = gi * R + slot / (2 * R);
    const int64_t rem = slot % (2 * R);
    sj = gj * R + rem / 2;
    half = rem & 1;
    if (si >= b.ni || sj >= b.nj) return false;
    si += b.i0;
    sj += b.j0;
    return si * 256 + half * kBM < n;
}

// Ring entry of a valid item: set index << 33 | half << 32 | si << 16 | sj
// (nsb <= 2^14 for n <= 2^22); -1 = no more items.
__device__ __forceinline__ int64_t pack_item(int sidx, int64_t si, int64_t sj, int64_t half) {
    return (int64_t(sidx) << 33) | (half << 32) | (si << 16) | sj;
}

__device__ __forceinline__ int item_set(int64_t e) { return int(e >> 33); }

template <int KE>
__device__ __forceinline__ Item unpack_item(int64_t e, int64_t kblocks) {
    Item it;
    it.I0 = ((e >> 16) & 0xFFFF) * 256 + ((e >> 32) & 1) * kBM;
    it.J0 = (e & 0xFFFF) * kBN;
    it.kb0 = it.I0 / KE;
    const int64_t end = (it.J0 + kBN + KE - 1) / KE;
    it.kb1 = end < kblocks ? end : kblocks;
    return it;
}

// Bits 0..3 of x -> 4 bytes of 0x00 / 0x38 (bit b -> byte b).  The product
// x + (x << 7) + (x << 14) + (x << 21) has its four copies in the disjoint
// bit ranges 0-3, 7-10, 14-17, 21-24 (no carries), and copy b puts bit b at
// bit 8b; the mask keeps those four bits.
__device__ __forceinline__ uint32_t spread4(uint32_t x) {
    return (((x & 0xFu) * 0x00204081u) & 0x01010101u) * kOne;
}

// 16 bits of a bitset row -> 16 operand bytes.
__device__ __forceinline__ uint4 spread16(uint32_t b) {
    return make_uint4(spread4(b), spread4(b >> 4), spread4(b >> 8), spread4(b >> 12));
}

// The parts of the operands any tile reads (decode_slot): row i of U is an A
// row of the tile starting at I0 = 128 * floor(i / 128), whose K range starts
// at I0; row j of L is a B row of the tile starting at J0 = 256 * floor(j /
// 256), whose K range ends at J0 + 256.  In 16-column pieces: U row i from
// piece u_first_piece(i), L row j below piece l_end_piece(j).  Nothing reads
// the rest, so the expansion leaves it unwritten (half of the 2 n^2 bytes).
__device__ __forceinline__ int64_t u_first_piece(int64_t i) { return (i / kBM) * (kBM / 16); }
__device__ __forceinline__ int64_t l_end_piece(int64_t j) { return (j / kBN + 1) * (kBN / 16); }

// Row i of U (the columns after i) and of L (the columns before i), each
// only where a tile reads it, in 16-column pieces handed out to thread t of
// a team of `size`: consecutive threads load consecutive 32-bit halves of
// the row's words and store consecutive 16-byte pieces.
__device__ __forceinline__ void expand_row(const uint64_t* __restrict__ bits, int64_t row_words, int64_t kpad,
                                           uint8_t* __restrict__ U, uint8_t* __restrict__ L, int64_t i, int t,
                                           int size) {
    const int ppr = int(kpad / 16);
    const uint32_t* brow = reinterpret_cast<const uint32_t*>(bits + i * row_words);
    uint4* urow = reinterpret_cast<uint4*>(U + i * kpad);
    uint4* lrow = reinterpret_cast<uint4*>(L + i * kpad);
    const int ii = int(i);  // n < 2^31
    auto piece = [&](int c) { return (__ldg(brow + (c >> 1)) >> (16 * (c & 1))) & 0xFFFFu; };
    for (int c = int(u_first_piece(i)) + t; c < ppr; c += size) {
        const int d = ii - 16 * c;  // column i relative to the piece's first column
        const uint32_t keep = d < 0 ? 0xFFFFu : (d >= 15 ? 0u : (0xFFFFu << (d + 1)) & 0xFFFFu);
        urow[c] = spread16(piece(c) & keep);
    }
    const int le = int(l_end_piece(i)) < ppr ? int(l_end_piece(i)) : ppr;
    for (int c = t; c < le; c += size) {
        const int d = ii - 16 * c;
        const uint32_t keep = d >= 16 ? 0xFFFFu : (d <= 0 ? 0u : (1u << d) - 1u);
        lrow[c] = spread16(piece(c) & keep);
    }
}

// U and L rows [r0, r1) of one set from the symmetric bitset.  Long rows (at
// least 4 pieces per thread of the block): the block sweeps each row;
// shorter rows: one warp per row.
__device__ __forceinline__ void expand_rows(const uint64_t* __restrict__ bits, int64_t row_words, int64_t kpad,
                                            uint8_t* __restrict__ U, uint8_t* __restrict__ L, int64_t r0,
                                            int64_t r1) {
    if (kpad / 16 >= 4 * int64_t(blockDim.x)) {
        for (int64_t i = r0; i < r1; ++i) expand_row(bits, row_words, kpad, U, L, i, threadIdx.x, blockDim.x);
        return;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int64_t i = r0 + warp; i < r1; i += nw) expand_row(bits, row_words, kpad, U, L, i, lane, 32);
}

constexpr int kExpandRows = 16;  // rows per block step

__global__ void __launch_bounds__(256) k_expand_f8(const uint64_t* __restrict__ bits, int64_t n, int64_t row_words,
                                                   int64_t kpad, uint8_t* __restrict__ U, uint8_t* __restrict__ L) {
    for (int64_t r0 = int64_t(blockIdx.x) * kExpandRows; r0 < n; r0 += int64_t(gridDim.x) * kExpandRows)
        expand_rows(bits, row_words, kpad, U, L, r0, r0 + kExpandRows < n ? r0 + kExpandRows : n);
}

// The same over many sets: one block per chunk of kExpandRows rows of one
// set, the set read from the caller's chunk table (no search).
__global__ void __launch_bounds__(256) k_expand_f8_multi(const MmaSetEntry* __restrict__ sets,
                                                         const int32_t* __restrict__ chunk_set) {
    const MmaSetEntry& e = sets[chunk_set[blockIdx.x]];
    const int64_t r0 = (int64_t(blockIdx.x) - e.chunk_begin) * kExpandRows;
    expand_rows(e.bits, e.row_words, e.kpad, e.op0, e.op1, r0, r0 + kExpandRows < e.n ? r0 + kExpandRows : e.n);
}

// ------------------------------------------------ packed FP4 operands
// (spread32_e2m1: cs_kernels.cuh)

// The FP4 operands.  A K-block holds 256 columns, the width of a supertile
// band, so for the supertile of bands (sI, sJ), sI <= sJ, every K-block kb
// strictly between the bands has sI*256 + 255 < k < sJ*256 for all its
// columns k: there i < k < j holds for every pair of the supertile, and both
// operands can be unmasked rows of the symmetric matrix, E[r][k] = C_rk.
// Only the two bands' own blocks need masks: kb = sI reads DU (row i, own
// block, columns k > i) for A, kb = sJ reads DL (row j, own block, columns
// k < j) for B; a diagonal supertile (sI = sJ) reads both.  E's own blocks
// are therefore never read and not written.  One operand matrix of n^2 / 2
// bytes plus 256 bytes per row, where U and L took twice that.
// Pieces of 32 columns (one 32-bit half of a bitset word, 16 operand bytes).
__device__ __forceinline__ int64_t own_first_piece(int64_t i) { return (i / 256) * 8; }

// Row i of E, pieces [p0, p1) of it (E row bytes kpad / 2), into erow, and,
// when D is not NULL, row i of DU and DL (rows of 128 bytes, DL starting
// dl_off bytes after DU); pieces handed out to thread t of a team of `size`.
__device__ __forceinline__ void expand_row_f4(const uint64_t* __restrict__ bits, int64_t row_words, uint4* erow,
                                              int p0, int p1, uint8_t* __restrict__ D, int64_t dl_off, int64_t i,
                                              int t, int size) {
    const uint32_t* brow = reinterpret_cast<const uint32_t*>(bits + i * row_words);
    const int own = int(own_first_piece(i));
    // four pieces per step, their loads issued together (memory-level
    // parallelism: one load, spread and store at a time left the expansion
    // latency-bound)
    for (int c0 = p0 + t; c0 < p1; c0 += 4 * size) {
        uint32_t w[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int c = c0 + k * size;
            w[k] = c < p1 ? __ldg(brow + c) : 0u;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int c = c0 + k * size;
            if (c < p1 && unsigned(c - own) >= 8u) erow[c] = spread32_e2m1(w[k]);
        }
    }
    if (D == nullptr) return;
    uint4* du = reinterpret_cast<uint4*>(D + i * 128);
    uint4* dl = reinterpret_cast<uint4*>(D + dl_off + i * 128);
    const int ii = int(i);  // n < 2^31
    for (int p = t; p < 16; p += size) {
        const int c = own + (p & 7);
        const int d = ii - 32 * c;  // column i relative to the piece's first column
        const uint32_t w = __ldg(brow + c);
        if (p < 8)
            du[p] = spread32_e2m1(w & (d < 0 ? ~0u : (d >= 31 ? 0u : (~0u << (d + 1)))));
        else
            dl[p - 8] = spread32_e2m1(w & (d >= 32 ? ~0u : (d <= 0 ? 0u : (1u << d) - 1u)));
    }
}

// FP4 operand rows [r0, r1) of one set: row i of E at E + (i - ebase) rows,
// its pieces [p0, p1); DU and DL too unless D is NULL.  The block sweeps each
// long row, one warp takes each short one.
__device__ __forceinline__ void expand_rows_f4(const uint64_t* __restrict__ bits, int64_t row_words, int64_t kpad,
                                               uint8_t* __restrict__ E, int64_t ebase, int p0, int p1,
                                               uint8_t* __restrict__ D, int64_t dl_off, int64_t r0, int64_t r1) {
    auto erow = [&](int64_t i) { return reinterpret_cast<uint4*>(E + (i - ebase) * (kpad / 2)); };
    if (p1 - p0 >= 4 * int(blockDim.x)) {
        for (int64_t i = r0; i < r1; ++i)
            expand_row_f4(bits, row_words, erow(i), p0, p1, D, dl_off, i, threadIdx.x, blockDim.x);
        return;
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int64_t i = r0 + warp; i < r1; i += nw)
        expand_row_f4(bits, row_words, erow(i), p0, p1, D, dl_off, i, lane, 32);
}

__global__ void __launch_bounds__(256) k_expand_f4(const uint64_t* __restrict__ bits, int64_t n, int64_t row_words,
                                                   int64_t kpad, uint8_t* __restrict__ E, uint8_t* __restrict__ D,
                                                   int64_t dl_off) {
    const int ppr = int(kpad / 32);
    for (int64_t r0 = int64_t(blockIdx.x) * kExpandRows; r0 < n; r0 += int64_t(gridDim.x) * kExpandRows)
        expand_rows_f4(bits, row_words, kpad, E, 0, 0, ppr, D, dl_off, r0, r0 + kExpandRows < n ? r0 + kExpandRows : n);
}

// Rows [r_begin, r_end) of a band: E row i at band row e_row0 + (i - r_begin),
// 32-column pieces [p0, p1); DU and DL too unless D is NULL.
__global__ void __launch_bounds__(256) k_expand_f4_band(const uint64_t* __restrict__ bits, int64_t row_words,
                                                        int64_t kpad, uint8_t* __restrict__ E, int64_t r_begin,
                                                        int64_t r_end, int64_t e_row0, int p0, int p1,
                                                        uint8_t* __restrict__ D, int64_t dl_off) {
    for (int64_t r0 = r_begin + int64_t(blockIdx.x) * kExpandRows; r0 < r_end;
         r0 += int64_t(gridDim.x) * kExpandRows)
        expand_rows_f4(bits, row_words, kpad, E, r_begin - e_row0, p0, p1, D, dl_off, r0,
                       r0 + kExpandRows < r_end ? r0 + kExpandRows : r_end);
}

// The same over many sets, one block per chunk of kExpandRows rows.
__global__ void __launch_bounds__(256) k_expand_f4_multi(const MmaSetEntry* __restrict__ sets,
                                                         const int32_t* __restrict__ chunk_set) {
    const MmaSetEntry& e = sets[chunk_set[blockIdx.x]];
    const int64_t r0 = (int64_t(blockIdx.x) - e.chunk_begin) * kExpandRows;
    expand_rows_f4(e.bits, e.row_words, e.kpad, e.op0, 0, 0, int(e.kpad / 32), e.op1, mma4_dl_offset(e.n), r0,
                   r0 + kExpandRows < e.n ? r0 + kExpandRows : e.n);
}

int expand_grid(int64_t rows) {
    int64_t g = int64_t(device_sm_count()) * 16;
    const int64_t steps = (rows + kExpandRows - 1) / kExpandRows;
    if (g > steps) g = steps;
    return int(g < 1 ? 1 : g);
}

// One causal set as the kernel sees it.
struct MmaView {
    const CUtensorMap* map;  // the set's operand maps (kMapU / kMapL, or kMapE / kMapDU / kMapDL)
    const uint64_t* bits;
    int64_t n, row_words, nsb, kblocks;
    unsigned long long* hist;
    int64_t hist_len;
    const double* phi;  // d'Alembertian field (NULL = 1)
    double* layer;      // layer sums [kmax+1][n], or NULL
    int kmax;           // < 0: no layer sums
    int raster;         // raster block side of the item order
    MmaBand band;       // the supertiles this launch counts (the whole set, or one band)
};

// Work source: a single set passed in kernel parameters.  The queue hands out
// one item at a time, so the CTAs running at any moment stay on consecutive,
// raster-local items.
struct MmaSingle {
    MmaView v;
    int64_t nitems;
    __device__ __forceinline__ int64_t total() const { return nitems; }
    __device__ __forceinline__ int64_t chunk() const { return 1; }
    __device__ __forceinline__ int set_of(int64_t t, int64_t& local, int) const {
        local = t;
        return 0;
    }
    __device__ __forceinline__ MmaView view(int) const { return v; }
};

// Work source: many sets from a device table, items ordered set by set.  The
// queue hands out runs of `run` consecutive items (up to 16, at least 8 runs
// per CTA), so a small set is spread over few CTAs and each CTA flushes its
// shared histogram into few sets, while a short launch still fills the GPU.
struct MmaMulti {
    const MmaSetEntry* sets;
    int nsets;
    int64_t nitems;
    uintptr_t hist_base;
    int64_t run;
    __device__ __forceinline__ int64_t total() const { return nitems; }
    __device__ __forceinline__ int64_t chunk() const { return run; }
    // The set holding item t: the hint (the previous item's set) or the next
    // set when t is still there, else a binary search.
    __device__ __forceinline__ int set_of(int64_t t, int64_t& local, int hint) const {
        int lo = -1;
        if (hint >= 0 && sets[hint].item_begin <= t) {
            if (hint + 1 == nsets || t < sets[hint + 1].item_begin)
                lo = hint;
            else if (hint + 2 == nsets || t < sets[hint + 2].item_begin)
                lo = hint + 1;
        }
        if (lo < 0) {
            int a = 0, b = nsets - 1;  // last set with item_begin <= t
            while (a < b) {
                const int mid = (a + b + 1) >> 1;
                if (sets[mid].item_begin <= t) a = mid; else b = mid - 1;
            }
            lo = a;
        }
        local = t - sets[lo].item_begin + sets[lo].item_offset;
        return lo;
    }
    __device__ __forceinline__ MmaView view(int s) const {
        const MmaSetEntry& e = sets[s];
        return MmaView{e.maps.m, e.bits, e.n, e.row_words, e.nsb, e.kblocks,
                       reinterpret_cast<unsigned long long*>(hist_base + uintptr_t(e.hist_off)),
                       e.n > 1 ? e.n - 1 : 1, e.phi, e.layer, int(e.kmax), kRasterDefault,
                       MmaBand{0, 0, e.nsb, e.nsb, 0, 0, 1}};
    }
};

// Barrier over the epilogue threads only, built on an mbarrier so that
// its wait is bounded and gives up once the CTA has aborted.
__device__ __forceinline__ bool epilogue_sync(uint64_t* ebar, uint32_t& phase, WsHeader* hdr, volatile int* abort) {
    mbar_arrive(ebar);
    const bool ok = mbar_wait_or_abort(ebar, phase, hdr, abort);
    phase ^= 1u;
    return ok;
}

// Epilogue threads add the shared histogram (its first `bins` bins) to the
// set's histogram and clear it.  Returns false if the CTA aborted.
__device__ __forceinline__ bool epilogue_flush(uint32_t* shist, int64_t bins, const MmaView& v, int etid,
                                               uint64_t* ebar, uint32_t& phase, WsHeader* hdr, volatile int* abort) {
    if (!epilogue_sync(ebar, phase, hdr, abort)) return false;
    const int64_t hb = v.hist_len < bins ? v.hist_len : bins;
    for (int64_t k = etid; k < hb; k += kEpiThreads) {
        const uint32_t c = shist[k];
        if (c) {
            atomicAdd(&v.hist[k], (unsigned long long)c);
            shist[k] = 0u;
        }
    }
    return epilogue_sync(ebar, phase, hdr, abort);
}

template <class Fmt, class Src>
__device__ __forceinline__ void mma_body(const Src& src, WsHeader* hdr) {
    constexpr bool kF4 = Fmt::kAcc == 1;
    constexpr bool kPair = Fmt::kPair;
    constexpr int kCl = kPair ? 2 : 1;                        // CTAs per cluster
    constexpr int kNS = Fmt::kStages;
    constexpr int kBRows = kPair ? kBN / 2 : kBN;             // B rows each CTA holds per stage
    constexpr int kSB = kABytes + kBRows * kBK;               // stage bytes per CTA
    constexpr int kMmaM = kPair ? 2 * kBM : kBM;
    constexpr int kHistBins = Fmt::kHistBins;
    static_assert(kSB == stage_bytes<Fmt>(), "stage layout");
    static_assert(kSB % 1024 == 0, "stage buffers stay swizzle-atom aligned");
    static_assert(!kPair || Fmt::kKE == kBN, "a pair's K-block is one supertile band (E, DU, DL operands)");
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint32_t* shist = reinterpret_cast<uint32_t*>(smem + kNS * kSB);
    uint64_t* full = reinterpret_cast<uint64_t*>(shist + kHistBins);
    uint64_t* empty = full + kNS;
    uint64_t* tfull = empty + kNS;
    uint64_t* tempty = tfull + 2;
    uint64_t* ebar = tempty + 2;
    uint64_t* ifull = ebar + 1;         // item ring: slot published by the producer
    uint64_t* iempty = ifull + kRing;   // item ring: slot read by its consumers
    uint64_t* done = iempty + kRing;    // the MMA thread's last commit: every MMA it issued has completed
    volatile int64_t* ring = reinterpret_cast<volatile int64_t*>(done + 1);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(const_cast<int64_t*>(ring) + kRing);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    static_assert((2 * kNS + 6 + 2 * kRing) * 8 + kRing * 8 + 8 <= kBarrierBytes, "barriers fit their area");

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t total = src.total();
    const uint32_t crank = kPair ? cluster_ctarank() : 0u;
    const bool leader = crank == 0;

    for (int k = tid; k < kHistBins; k += kThreads) shist[k] = 0u;
    if (tid == 0) {
        for (int s = 0; s < kNS; ++s) {
            mbar_init(&full[s], 1);   // pair: rank 0's receives both CTAs' bytes
            mbar_init(&empty[s], 1);  // the MMA commit (pair: rank 0's, multicast to both)
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], kCl * kEpiThreads);  // pair: both CTAs' epilogues, on rank 0
        }
        mbar_init(ebar, kEpiThreads);
        mbar_init(done, 1);
        // iempty counts every consumer of an entry: the producer, MMA thread
        // and epilogue; in a pair, rank 0's counts both CTAs' producers and
        // epilogues and rank 0's MMA thread (rank 1's own iempty is unused).
        for (int r = 0; r < kRing; ++r) {
            mbar_init(&ifull[r], 1);
            mbar_init(&iempty[r], kPair ? 2 * (1 + kEpiThreads) + 1 : 2 + kEpiThreads);
        }
        *abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        if constexpr (kPair) {
            tmem_alloc_pair(tmem_slot, kTmemCols);
            tmem_relinquish_pair();
        } else {
            tmem_alloc(tmem_slot, kTmemCols);
            tmem_relinquish();
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;
    if constexpr (kF4) {
        // Every scale factor the MMAs may read (A at kSfCol, B at kSfCol + 16,
        // all 128 lanes, 32 columns) is 1; one warp per TMEM lane quarter.
        if (warp >= 2 && warp < 6) {
            tmem_st_32x32b_x32_fill(tmem_base + (uint32_t(32 * (warp & 3)) << 16) + kSfCol, kScaleOne);
            tmem_st_wait();
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    }
    // The peer's barriers and TMEM are ready before anyone signals them.
    if constexpr (kPair) cluster_sync();

    // Item ring.  The scheduler (warp kSchedWarp; in a pair, rank 0's)
    // publishes each item to the producer, MMA and epilogue threads (in a
    // pair to both CTAs: its own slot and, through the cluster window, rank
    // 1's), and every consumer of either CTA releases the slot on rank 0's
    // iempty.  Running ahead of the producer by up to kRing items, it keeps
    // the search for work, its global queue atomic and the publication off
    // the path between one tile's last load and the next tile's first
    // (measured there: about 3500 SM cycles per tile when the producer did
    // both, and the MMAs then waited 1.2-1.8 us for each tile's first
    // K-block).  A ring entry is a decoded item
    // (pack_item): the unit the queue hands out is a slot (one CTA) or a
    // supertile slot (a pair, which runs it as slot 2 * unit, its upper
    // half), and the producer skips the units that hold no work.
    const uint32_t iempty0 = kPair ? cluster_map(iempty, 0) : 0u;
    const uint32_t tempty0 = kPair ? cluster_map(tempty, 0) : 0u;
    auto ring_wait = [&](uint32_t slot, uint32_t use) {
        return mbar_wait_or_abort<kPair>(&ifull[slot], use, hdr, abort_flag);
    };
    auto ring_release = [&](uint32_t slot) {
        if (kPair && !leader)
            mbar_arrive_cluster(iempty0 + 8u * slot, 1u);
        else
            mbar_arrive(&iempty[slot]);
    };
    // This CTA's first A row and B row within an item.
    const int64_t row_off = kPair ? int64_t(crank) * kBM : 0;

    if (warp == 0 && lane == 0) {
        // ---------------------------------------------------- TMA producer
        // Takes each item from the ring and streams its K-blocks into the
        // stages (a pair: each CTA its own rows).
        uint32_t s = 0, ph = 0, issued = 0;
        bool ok = true;
        int cur = -1;
        MmaView v{};
        for (uint32_t q = 0; ok; ++q) {
            const uint32_t slot = q % kRing, use = (q / kRing) & 1u;
            if (!ring_wait(slot, use)) { ok = false; break; }
            const int64_t e = ring[slot];
            ring_release(slot);
            if (e < 0) break;
            const int sidx = item_set(e);
            if (sidx != cur) {
                cur = sidx;
                v = src.view(sidx);
            }
            const Item it = unpack_item<Fmt::kKE>(e, v.kblocks);
            for (int64_t kb = it.kb0; kb < it.kb1; ++kb) {
                if (!mbar_wait_or_abort(&empty[s], ph ^ 1u, hdr, abort_flag)) { ok = false; break; }
                uint8_t* a = smem + s * kSB;
                if constexpr (kPair) {
                    // Both CTAs' bytes land on rank 0's full barrier.  A
                    // K-block holds one band: the i-band's own block comes
                    // from DU, the j-band's from DL, every other from E.
                    const uint32_t fb = cluster_map(&full[s], 0);
                    if (leader) mbar_arrive_expect_tx(&full[s], 2 * kSB);
                    const bool a_own = kb == it.I0 / kBN, b_own = kb == it.J0 / kBN;
                    tma_load_2d_pair(a, &v.map[a_own ? kMapDU : kMapE], a_own ? 0 : int32_t(kb * kBK),
                                     int32_t(it.I0 + row_off - (a_own ? 0 : v.band.erow_i)), fb);
                    tma_load_2d_pair(a + kABytes, &v.map[b_own ? kMapDL : kMapE], b_own ? 0 : int32_t(kb * kBK),
                                     int32_t(it.J0 + row_off - (b_own ? 0 : v.band.erow_j)), fb);
                } else {
                    mbar_arrive_expect_tx(&full[s], kSB);
                    tma_load_2d(a, &v.map[kMapU], int32_t(kb * kBK), int32_t(it.I0), &full[s]);
                    tma_load_2d(a + kABytes, &v.map[kMapL], int32_t(kb * kBK), int32_t(it.J0), &full[s]);
                }
                ++issued;
                if (++s == kNS) { s = 0; ph ^= 1u; }
            }
        }
        if (!ok && (!kPair || leader)) {
            // Let the copies still in flight land before shared memory goes away.
            for (uint32_t q = 0; q < kNS && q < issued; ++q) {
                const uint32_t g = issued - 1 - q;
                mbar_wait_bounded(&full[g % kNS], (g / kNS) & 1u, hdr);
            }
        }
        if constexpr (kPair) {
            // Each stage is released by the pair's MMA commit, which lands in
            // both CTAs; wait for the last ones (their data has landed by
            // then), so that nothing is still on its way to this CTA when it
            // leaves (shorter limit once aborted).
            for (int k = 0; k < kNS; ++k) {
                mbar_wait_bounded(&empty[s], ph ^ 1u, hdr, ok ? kWaitLimitNs : kWaitLimitNs / 40);
                if (++s == kNS) { s = 0; ph ^= 1u; }
            }
        }
    } else if (warp == kSchedWarp && lane == 0 && leader) {
        // ---------------------------------------------------- scheduler
        // Pulls units from the global queue (consecutive indices are
        // raster-local, so the CTAs running at any moment share operand
        // panels in L2), skips the units that hold no work, and publishes
        // the others decoded.
        int cur = -1;
        MmaView v{};
        int64_t next = 0, end = 0;  // the current run of units from the queue
        const int64_t units = total / kCl;
        for (uint32_t q = 0;; ++q) {
            const uint32_t slot = q % kRing, use = (q / kRing) & 1u;
            if (!mbar_wait_or_abort<kPair>(&iempty[slot], use ^ 1u, hdr, abort_flag)) break;
            int64_t e = -1;
            for (;;) {
                if (next >= end) {
                    next = int64_t(atomicAdd(&hdr->counter, 1ull)) * src.chunk();
                    end = next + src.chunk();
                }
                const int64_t t = next++;
                if (t >= units) break;
                int64_t lu, si, sj, half;
                const int sidx = src.set_of(t, lu, cur);
                if (sidx != cur) {
                    cur = sidx;
                    v = src.view(sidx);
                }
                if (decode_band(lu * kCl, v.band, v.n, v.raster, si, sj, half)) {
                    e = pack_item(sidx, si, sj, half);
                    break;
                }
            }
            ring[slot] = e;
            mbar_arrive(&ifull[slot]);
            if constexpr (kPair) {
                st_cluster_s64(cluster_map(const_cast<int64_t*>(&ring[slot]), 1), e);
                mbar_arrive_cluster(cluster_map(&ifull[slot], 1), 1u);
            }
            if (e < 0) break;
        }
    } else if (warp == 1 && lane == 0 && leader) {
        // ---------------------------------------------------- MMA issuer
        // (a pair: rank 0's, for both CTAs)
        uint32_t s = 0, ph = 0;
        int64_t local_count = 0;
        bool ok = true;
        int cur = -1;
        MmaView v{};
        for (uint32_t q = 0; ok; ++q) {
            const uint32_t slot = q % kRing, use = (q / kRing) & 1u;
            if (!ring_wait(slot, use)) break;
            const int64_t e = ring[slot];
            ring_release(slot);
            if (e < 0) break;
            const int sidx = item_set(e);
            if (sidx != cur) {
                cur = sidx;
                v = src.view(sidx);
            }
            const Item it = unpack_item<Fmt::kKE>(e, v.kblocks);
            const uint32_t buf = uint32_t(local_count % Fmt::kAcc), bu = uint32_t((local_count / Fmt::kAcc) & 1);
            ++local_count;
            if (!mbar_wait_or_abort<kPair>(&tempty[buf], bu ^ 1u, hdr, abort_flag)) break;
            tc_fence_after();
            const uint32_t d = tmem_base + buf * kBN;
            for (int64_t kb = it.kb0; kb < it.kb1; ++kb) {
                if (!mbar_wait_or_abort<kPair>(&full[s], ph, hdr, abort_flag)) { ok = false; break; }
                tc_fence_after();
                const uint32_t a = smem_u32(smem + s * kSB);
                const uint64_t adesc = sdesc_k_swizzled(a, kBK), bdesc = sdesc_k_swizzled(a + kABytes, kBK);
#pragma unroll
                for (int kk = 0; kk < kBK / kUK; ++kk) {
                    const uint32_t acc = (kb > it.kb0 || kk > 0) ? 1u : 0u;
                    const uint64_t ad = adesc + uint64_t((kk * kUK) >> 4), bd = bdesc + uint64_t((kk * kUK) >> 4);
                    if constexpr (kPair)
                        mma_mxf4_pair(d, ad, bd, idesc_mxf4_f32(kMmaM, kBN), tmem_base + kSfCol,
                                      tmem_base + kSfCol + 16, acc);
                    else if constexpr (kF4)
                        mma_mxf4(d, ad, bd, kIdesc4, tmem_base + kSfCol, tmem_base + kSfCol + 16, acc);
                    else
                        mma_f8f6f4(d, ad, bd, kIdesc, acc);
                }
                if constexpr (kPair)
                    mma_commit_pair_mc(&empty[s], 0x3);  // the stage is free in both CTAs
                else
                    mma_commit(&empty[s]);
                if (++s == kNS) { s = 0; ph ^= 1u; }
            }
            if (ok) {
                if constexpr (kPair)
                    mma_commit_pair_mc(&tfull[buf], 0x3);
                else
                    mma_commit(&tfull[buf]);
            }
        }
        // Also after an abort: nothing this thread issued may still run when
        // the CTA (or pair) frees its TMEM.
        if constexpr (kPair)
            mma_commit_pair_mc(done, 0x1);
        else
            mma_commit(done);
        mbar_wait_bounded(done, 0, hdr, kWaitLimitNs / 40);
    } else if (warp >= 2 && warp < 2 + kEpiWarps) {
        // ---------------------------------------------------- epilogue
        const int q = warp & 3;            // TMEM lane quarter this warp may access
        const int c0 = ((warp - 2) >> 2) * kEpiChunks;  // first of its 32-column chunks
        const int etid = tid - 64;
        const uint32_t shist_s = smem_u32(shist);
        int64_t local_count = 0;
        int64_t since_flush = 0;  // tiles counted into the shared histogram since its last flush
        int cur = -1;
        uint32_t ephase = 0;
        bool ok = true;
        MmaView v{};
        // Release the accumulator to the MMA issuer (a pair: rank 0's), one
        // arrival of 32 per warp once all its lanes' TMEM reads are done.
        // The accumulator's only users here are this warp's tcgen05.ld,
        // complete once tcgen05.wait::ld returned, so the arrival orders no
        // memory access and needs no fence (a release at cluster scope would
        // wait for the bitset word's global load still in flight).
        auto acc_release = [&](uint32_t buf) {
            tc_fence_before();
            if constexpr (kPair) {
                __syncwarp();
                if (lane == 0) {
                    if (leader)
                        mbar_arrive_relaxed_cnt(&tempty[buf], 32u);
                    else
                        mbar_arrive_cluster_relaxed(tempty0 + 8u * buf, 32u);
                }
            } else {
                mbar_arrive_relaxed_cnt(&tempty[buf], 1u);
            }
        };
        // Release an item-ring slot, likewise one arrival of 32 per warp in a pair.
        // The slot's only use before the arrival is the read of its entry e;
        // the arrival count is computed from e (entries are >= 0 or -1, so
        // the added term is always 0), which keeps the arrival behind the
        // read without a fence -- a release at cluster scope waited for the
        // previous tile's shared-memory histogram atomics (measured: 3% of
        // the 768-set batch).
        auto epi_ring_release = [&](uint32_t slot, int64_t e) {
            const uint32_t dep = e == -2 ? 1u : 0u;
            if constexpr (kPair) {
                __syncwarp();
                if (lane == 0) {
                    if (leader)
                        mbar_arrive_relaxed_cnt(&iempty[slot], 32u + dep);
                    else
                        mbar_arrive_cluster_relaxed(iempty0 + 8u * slot, 32u + dep);
                }
            } else {
                mbar_arrive_relaxed_cnt(&iempty[slot], 1u + dep);
            }
        };
        for (uint32_t qi = 0; ok; ++qi) {
            const uint32_t slot = qi % kRing, ru = (qi / kRing) & 1u;
            if (!ring_wait(slot, ru)) { ok = false; break; }
            const int64_t e = ring[slot];
            epi_ring_release(slot, e);
            if (e < 0) break;
            const int sidx = item_set(e);
            if (sidx != cur || since_flush == kFlushTiles) {
                if (cur >= 0 && !epilogue_flush(shist, kHistBins, v, etid, ebar, ephase, hdr, abort_flag)) { ok = false; break; }
                cur = sidx;
                v = src.view(sidx);
                since_flush = 0;
            }
            const Item it = unpack_item<Fmt::kKE>(e, v.kblocks);
            ++since_flush;
            const int64_t hb = v.hist_len < kHistBins ? v.hist_len : kHistBins;
            const uint32_t buf = uint32_t(local_count % Fmt::kAcc), use = uint32_t((local_count / Fmt::kAcc) & 1);
            ++local_count;
            const int64_t i = it.I0 + row_off + 32 * q + lane;
            // the C_ij word of this warp's 64 columns, loaded before the wait
            // for the accumulator so that its latency hides behind the MMAs
            static_assert(kEpiChunks == 2, "one bitset word per epilogue warp");
            const int64_t word0 = (it.J0 + 32 * c0) >> 6;
            const uint64_t cw = (i < v.n && word0 < v.row_words) ? __ldg(v.bits + i * v.row_words + word0) : 0ull;
            if (!mbar_wait_or_abort<kPair>(&tfull[buf], use, hdr, abort_flag)) { ok = false; break; }
            tc_fence_after();
            // Every count of this set lands in the shared histogram and there
            // are no layer sums: the common case, kept branch-free.
            const bool simple = v.kmax < 0 && v.hist_len <= kHistBins;
            // Histogram the 32 counts r of chunk c (columns J0 + 32c ..); index
            // arithmetic in 32 bits (n <= 2^22).
            const int ii = int(i), nn = int(v.n), hb32 = int(hb);
            auto chunk = [&](int c, const uint32_t (&r)[32]) {
                // pairs to count among these 32 j: C_ij, i < j < n
                const int jb = int(it.J0) + 32 * c;
                uint32_t m = uint32_t(cw >> (32 * (c & 1)));
                const int lo = ii - jb + 1;  // first u with j > i
                m &= lo <= 0 ? ~0u : (lo >= 32 ? 0u : (~0u << lo));
                const int hi = nn - jb;      // u < hi keeps j < n
                m &= hi >= 32 ? ~0u : (hi <= 0 ? 0u : ((1u << hi) - 1u));
                if (m == 0u) return;
                // counts are integers below 2^23: adding 2^23 puts k in the
                // low mantissa bits, exactly
                if (Fmt::kSmallSet && simple) {
#pragma unroll
                    for (int u = 0; u < 32; ++u)
                        if ((m >> u) & 1u)
                            red_shared_add(shist_s + 4u * (__float_as_uint(__uint_as_float(r[u]) + 8388608.0f) - 0x4B000000u), 1u);
                    return;
                }
                if constexpr (Fmt::kLayers) {
                    if (v.kmax >= 0) {
#pragma unroll
                        for (int u = 0; u < 32; ++u) {
                            if ((m >> u) & 1u) {
                                const int k = int(__float_as_uint(__uint_as_float(r[u]) + 8388608.0f) - 0x4B000000u);
                                if (k < hb32)
                                    red_shared_add(shist_s + 4u * uint32_t(k), 1u);
                                else
                                    atomicAdd(&v.hist[k], 1ull);
                                if (k <= v.kmax)  // i is in L_{k+1}(j)
                                    atomicAdd(&v.layer[int64_t(k) * nn + jb + u], v.phi ? __ldg(v.phi + i) : 1.0);
                            }
                        }
                        return;
                    }
                }
#pragma unroll
                for (int u = 0; u < 32; ++u) {
                    if ((m >> u) & 1u) {
                        const int k = int(__float_as_uint(__uint_as_float(r[u]) + 8388608.0f) - 0x4B000000u);
                        if (k < hb32)
                            red_shared_add(shist_s + 4u * uint32_t(k), 1u);
                        else
                            atomicAdd(&v.hist[k], 1ull);
                    }
                }
            };
            if constexpr (kF4) {
                // The single accumulator goes to registers and is released
                // before the histogram work, so the next tile's MMAs start at once.
                uint32_t r0[32], r1[32];
                tmem_ld_32x32b_x32(tmem_base + (uint32_t(32 * q) << 16) + uint32_t(32 * c0), r0);
                tmem_ld_32x32b_x32(tmem_base + (uint32_t(32 * q) << 16) + uint32_t(32 * (c0 + 1)), r1);
                tmem_ld_wait();
                acc_release(buf);
                chunk(c0, r0);
                chunk(c0 + 1, r1);
            } else {
#pragma unroll 1
                for (int c = c0; c < c0 + kEpiChunks; ++c) {
                    uint32_t r[32];
                    tmem_ld_32x32b_x32(tmem_base + (uint32_t(32 * q) << 16) + buf * kBN + uint32_t(32 * c), r);
                    tmem_ld_wait();
                    chunk(c, r);
                }
                acc_release(buf);
            }
        }
        if (ok && cur >= 0) epilogue_flush(shist, kHistBins, v, etid, ebar, ephase, hdr, abort_flag);
    }
    __syncthreads();
    // No CTA of a pair leaves (or frees the pair's TMEM) while the other
    // may still signal it or its MMAs may still run.
    if constexpr (kPair) cluster_sync();
    if (warp == 1) {
        tc_fence_after();
        if constexpr (kPair)
            tmem_dealloc_pair(tmem_base, kTmemCols);
        else
            tmem_dealloc(tmem_base, kTmemCols);
    }
}

__global__ void __maxnreg__(kMaxRegs)
    k_count_mma(const __grid_constant__ MmaMaps maps, const uint64_t* __restrict__ bits, int64_t n,
                int64_t row_words, int64_t nsb, int64_t nitems, int64_t kblocks,
                unsigned long long* __restrict__ hist, int64_t hist_len, const double* phi, double* layer, int kmax,
                int raster, MmaBand band, WsHeader* hdr) {
    const MmaSingle src{MmaView{maps.m, bits, n, row_words, nsb, kblocks, hist, hist_len, phi, layer, kmax, raster,
                                band},
                        nitems};
    mma_body<FmtF8>(src, hdr);
}

// The same count on packed FP4 operands (kind::mxf4): counts only, and
// counts with layer sums.
template <class Fmt>
__global__ void __maxnreg__(kMaxRegs)
    k_count_mma4(const __grid_constant__ MmaMaps maps, const uint64_t* __restrict__ bits, int64_t n,
                 int64_t row_words, int64_t nsb, int64_t nitems, int64_t kblocks,
                 unsigned long long* __restrict__ hist, int64_t hist_len, const double* phi, double* layer, int kmax,
                 int raster, MmaBand band, WsHeader* hdr) {
    const MmaSingle src{MmaView{maps.m, bits, n, row_words, nsb, kblocks, hist, hist_len, phi, layer, kmax, raster,
                                band},
                        nitems};
    mma_body<Fmt>(src, hdr);
}

__global__ void __maxnreg__(kMaxRegs)
    k_count_mma_multi(const MmaSetEntry* __restrict__ sets, int nsets, int64_t nitems, uintptr_t hist_base,
                      int64_t run, WsHeader* hdr) {
    const MmaMulti src{sets, nsets, nitems, hist_base, run};
    mma_body<FmtF8>(src, hdr);
}

// Many sets on the FP4 pair path.  The table's item_begin / item_offset and
// `run` count supertiles (the pair's unit of work); nitems is twice the
// number of supertiles.
__global__ void __maxnreg__(kMaxRegs)
    k_count_mma4_multi(const MmaSetEntry* __restrict__ sets, int nsets, int64_t nitems, uintptr_t hist_base,
                       int64_t run, WsHeader* hdr) {
    const MmaMulti src{sets, nsets, nitems, hist_base, run};
    mma_body<FmtF4Multi>(src, hdr);
}

std::atomic<bool> g_attr_set[64];  // per device: the large-shared-memory attribute is set
std::atomic<bool> g_attr_multi_set[64];
std::atomic<bool> g_attr4_set[64];
std::atomic<bool> g_attr4l_set[64];
std::atomic<int> g_clusters4[64];   // per device: CTA pairs of the FP4 kernels resident at once (0 = not queried)
std::atomic<int> g_clusters4l[64];
std::atomic<bool> g_attr4m_set[64];
std::atomic<int> g_clusters4m[64];

// Launch configuration of a persistent grid of CTA pairs: as many clusters
// of two as fit at once (queried once per device and kernel), at most
// `units` of them.
template <class K>
cudaError_t pair_config(K kernel, int smem, std::atomic<bool>* attr, std::atomic<int>* cached, int64_t units,
                        cudaStream_t st, cudaLaunchAttribute* at, cudaLaunchConfig_t* cfg, int* pairs) {
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr[dev]) {
        if ((err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) != cudaSuccess)
            return err;
        attr[dev] = true;
    }
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 2;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    *cfg = cudaLaunchConfig_t{};
    cfg->gridDim = dim3(unsigned(device_sm_count() / 2 * 2));
    cfg->blockDim = dim3(kThreads);
    cfg->dynamicSmemBytes = smem;
    cfg->stream = st;
    cfg->attrs = at;
    cfg->numAttrs = 1;
    int clusters = cached[dev];
    if (clusters == 0) {
        if ((err = cudaOccupancyMaxActiveClusters(&clusters, kernel, cfg)) != cudaSuccess) return err;
        if (clusters < 1) return cudaErrorNotSupported;
        cached[dev] = clusters;
    }
    *pairs = int(clusters < units ? clusters : units);
    cfg->gridDim = dim3(unsigned(2 * *pairs));
    return cudaSuccess;
}

// Workspace: header, then the two operand buffers: FP8 U and L, each n rows
// of kpad bytes; FP4 E (n rows of kpad / 2 bytes) and the diagonal blocks
// (DU, then DL at mma4_dl_offset(n), n rows of 128 bytes each).
struct MmaLayout {
    int64_t kpad, row;  // K elements per row, bytes per row of U, L or E
    size_t op0, op1, total;
};

size_t operand_bytes(int64_t n, int64_t kpad, bool fp4, int which) {
    if (!fp4) return size_t(n) * size_t(kpad);
    return which == 0 ? size_t(n) * size_t(kpad / 2) : size_t(mma4_dl_offset(n)) + size_t(n) * 128;
}

MmaLayout mma_layout(int64_t n, bool fp4) {
    MmaLayout m;
    const int64_t ke = fp4 ? FmtF4::kKE : FmtF8::kKE;
    m.kpad = (n + ke - 1) / ke * ke;
    m.row = fp4 ? m.kpad / 2 : m.kpad;
    m.op0 = 1024;  // after the 256-byte header, 1024-byte aligned
    m.op1 = align_up(m.op0 + operand_bytes(n, m.kpad, fp4, 0), 1024);
    m.total = align_up(m.op1 + operand_bytes(n, m.kpad, fp4, 1), 256);
    return m;
}

// The FP4 layout when the set's E does not fit: header, a band buffer of
// 2 g panels of 256 E rows (two groups of g supertile rows), then DU and DL
// for every row.
MmaLayout mma4_band_layout(int64_t n, int64_t g) {
    MmaLayout m;
    m.kpad = (n + FmtF4::kKE - 1) / FmtF4::kKE * FmtF4::kKE;
    m.row = m.kpad / 2;
    m.op0 = 1024;
    m.op1 = align_up(m.op0 + size_t(2 * g * 256) * size_t(m.row), 1024);
    m.total = align_up(m.op1 + operand_bytes(n, m.kpad, true, 1), 256);
    return m;
}

// TMA maps of one set's operands (128B swizzle; boxes of one 128-byte
// K-stage).  FP8: U (box 128 rows, the A slab) and L (box 256 rows, the B
// slab).  FP4 pairs: each CTA of a pair loads 128 rows of A and of B, so E,
// DU and DL all take 128-row boxes.
// E (FP4): `rows` rows of kpad / 2 bytes (the rows of the set, or of a band
// buffer up to its last row of the set: the map reads zeros past them).
CUresult encode_e_map(CUtensorMap* map, int64_t kpad, uint8_t* op0, int64_t rows) {
    const uint64_t row = uint64_t(kpad / 2);
    return encode_tensor_map_2d(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, op0, row, uint64_t(rows), row, kBK, kBM,
                                kSwizzle);
}

CUresult encode_operand_maps(MmaMaps* maps, int64_t n, int64_t kpad, bool fp4, uint8_t* op0, uint8_t* op1) {
    const uint64_t row = uint64_t(fp4 ? kpad / 2 : kpad);
    CUresult r = fp4 ? encode_e_map(&maps->m[kMapE], kpad, op0, n)
                     : encode_tensor_map_2d(&maps->m[kMapU], CU_TENSOR_MAP_DATA_TYPE_UINT8, op0, row, uint64_t(n),
                                            row, kBK, kBM, kSwizzle);
    if (r != CUDA_SUCCESS) return r;
    if (!fp4) {
        std::memset(static_cast<void*>(&maps->m[2]), 0, sizeof(CUtensorMap));
        return encode_tensor_map_2d(&maps->m[kMapL], CU_TENSOR_MAP_DATA_TYPE_UINT8, op1, row, uint64_t(n), row, kBK,
                                    kBN, kSwizzle);
    }
    static_assert(kBK == 128, "a DU / DL row is one 128-byte K-stage");
    if ((r = encode_tensor_map_2d(&maps->m[kMapDU], CU_TENSOR_MAP_DATA_TYPE_UINT8, op1, 128, uint64_t(n), 128, kBK,
                                  kBN / 2, kSwizzle)) != CUDA_SUCCESS)
        return r;
    return encode_tensor_map_2d(&maps->m[kMapDL], CU_TENSOR_MAP_DATA_TYPE_UINT8, op1 + mma4_dl_offset(n), 128,
                                uint64_t(n), 128, kBK, kBN / 2, kSwizzle);
}

}  // namespace

size_t mma_workspace_bytes(int64_t n) { return mma_layout(n, false).total; }

size_t mma4_workspace_bytes(int64_t n) { return mma_layout(n, true).total; }

int64_t mma4_band_panels(int64_t n, size_t bytes) {
    if (n < 1) return 0;
    const int64_t nsb = (n + 255) / 256;
    if (mma_layout(n, true).total <= bytes) return nsb;
    const MmaLayout one = mma4_band_layout(n, 1);
    if (one.total > bytes) return 0;
    int64_t g = 1 + int64_t((bytes - one.total) / (size_t(2 * 256) * size_t(one.row)));
    while (g > 1 && mma4_band_layout(n, g).total > bytes) --g;
    return g < nsb ? g : nsb;
}

size_t mma4_band_bytes(int64_t n, int64_t g) {
    const int64_t nsb = (n + 255) / 256;
    return g >= nsb ? mma_layout(n, true).total : mma4_band_layout(n, g < 1 ? 1 : g).total;
}

int64_t mma_kpad(int64_t n, bool fp4) {
    const int64_t ke = fp4 ? FmtF4::kKE : FmtF8::kKE;
    return (n + ke - 1) / ke * ke;
}

size_t mma_operand_bytes(int64_t n, bool fp4, int which) { return operand_bytes(n, mma_kpad(n, fp4), fp4, which); }

int64_t mma4_units(int64_t n, int raster) { return mma_items(n, raster) / 2; }

int64_t mma_items(int64_t n, int raster) {
    const int64_t nsb = (n + 255) / 256;
    const int64_t R = raster;
    const int64_t nbg = (nsb + R - 1) / R;
    return 2 * R * R * nbg * (nbg + 1) / 2;
}

CUresult mma_fill_entry(MmaSetEntry* e, const uint64_t* bits, int64_t n, int64_t row_words, uint8_t* op0,
                        uint8_t* op1, bool fp4) {
    e->kmax = -1;
    e->bits = bits;
    e->n = n;
    e->row_words = row_words;
    e->nsb = (n + 255) / 256;
    e->kpad = mma_kpad(n, fp4);
    const int64_t row = fp4 ? e->kpad / 2 : e->kpad;  // operand row bytes
    e->kblocks = row / kBK;
    e->op0 = op0;
    e->op1 = op1;
    return encode_operand_maps(&e->maps, n, e->kpad, fp4, op0, op1);
}

cudaError_t launch_expand_single(const MmaSetEntry* e, cudaStream_t st, bool fp4) {
    if (e->n < 1) return cudaSuccess;
    if (fp4)
        k_expand_f4<<<unsigned(expand_grid(e->n)), 256, 0, st>>>(e->bits, e->n, e->row_words, e->kpad, e->op0, e->op1,
                                                                 mma4_dl_offset(e->n));
    else
        k_expand_f8<<<unsigned(expand_grid(e->n)), 256, 0, st>>>(e->bits, e->n, e->row_words, e->kpad, e->op0,
                                                                 e->op1);
    return cudaGetLastError();
}

int64_t mma_expand_chunks(int64_t n) { return (n + kExpandRows - 1) / kExpandRows; }

cudaError_t launch_expand_multi(const MmaSetEntry* sets_dev, const int32_t* chunk_set, int64_t total_chunks,
                                cudaStream_t st, bool fp4) {
    if (total_chunks < 1) return cudaSuccess;
    if (total_chunks > int64_t(0x7fffffff)) return cudaErrorInvalidValue;
    if (fp4)
        k_expand_f4_multi<<<unsigned(total_chunks), 256, 0, st>>>(sets_dev, chunk_set);
    else
        k_expand_f8_multi<<<unsigned(total_chunks), 256, 0, st>>>(sets_dev, chunk_set);
    return cudaGetLastError();
}

cudaError_t launch_count_mma4_multi(const MmaSetEntry* sets_dev, int nsets, int64_t nunits, uintptr_t hist_base,
                                    WsHeader* hdr, cudaStream_t st) {
    if (nunits < 1) return cudaSuccess;
    cudaError_t err = cudaMemsetAsync(&hdr->counter, 0, sizeof(hdr->counter), st);
    if (err != cudaSuccess) return err;
    cudaLaunchAttribute at[1];
    cudaLaunchConfig_t cfg;
    int pairs = 0;
    if ((err = pair_config(k_count_mma4_multi, smem_bytes<FmtF4Multi>(), g_attr4m_set, g_clusters4m, nunits, st, at,
                           &cfg, &pairs)) != cudaSuccess)
        return err;
    // runs of up to max_run consecutive supertiles, at least 8 runs per pair
    const int64_t cap = batch_max_run();
    int64_t run = nunits / (int64_t(pairs) * 8);
    run = run < 1 ? 1 : (run > cap ? cap : run);
    return cudaLaunchKernelEx(&cfg, k_count_mma4_multi, sets_dev, nsets, 2 * nunits, hist_base, run, hdr);
}

cudaError_t launch_count_mma_multi(const MmaSetEntry* sets_dev, int nsets, int64_t nitems, uintptr_t hist_base,
                                   WsHeader* hdr, int max_ctas, cudaStream_t st) {
    if (nitems < 1) return cudaSuccess;
    cudaError_t err = cudaMemsetAsync(&hdr->counter, 0, sizeof(hdr->counter), st);
    if (err != cudaSuccess) return err;
    int dev = 0;
    if ((err = cudaGetDevice(&dev)) != cudaSuccess) return err;
    if (dev >= 0 && dev < 64 && !g_attr_multi_set[dev]) {
        err = cudaFuncSetAttribute(k_count_mma_multi, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   smem_bytes<FmtF8>());
        if (err != cudaSuccess) return err;
        g_attr_multi_set[dev] = true;
    }
    int64_t grid = max_ctas > 0 ? max_ctas : device_sm_count();
    if (grid > nitems) grid = nitems;
    const int64_t cap = batch_max_run();
    int64_t run = nitems / (grid * 8);
    run = run < 1 ? 1 : (run > cap ? cap : run);
    k_count_mma_multi<<<unsigned(grid), kThreads, smem_bytes<FmtF8>(), st>>>(sets_dev, nsets, nitems, hist_base, run,
                                                                            hdr);
    return cudaGetLastError();
}

namespace {

// Items of a band: the triangle's raster blocks, or the rectangle's.
int64_t band_items(const MmaBand& b, int raster) {
    const int64_t R = raster;
    const int64_t nbi = (b.ni + R - 1) / R, nbj = (b.nj + R - 1) / R;
    return 2 * R * R * (b.diag ? nbi * (nbi + 1) / 2 : nbi * nbj);
}

// The bands of a set counted in groups of g panels, in launch order: for
// each group a the triangle (a, a), then the rectangles (a, b), b > a; the
// whole set as one band when g >= nsb.  The E rows of the triangle's group
// sit in band rows [0, 256 g), those of a rectangle's second group in
// [256 g, 512 g).
std::vector<MmaBand> mma4_bands(int64_t n, int64_t g) {
    const int64_t nsb = (n + 255) / 256;
    std::vector<MmaBand> out;
    if (g >= nsb) {
        out.push_back(MmaBand{0, 0, nsb, nsb, 0, 0, 1});
        return out;
    }
    const int64_t m = (nsb + g - 1) / g;
    for (int64_t a = 0; a < m; ++a) {
        const int64_t a0 = a * g, ga = nsb - a0 < g ? nsb - a0 : g;
        out.push_back(MmaBand{a0, a0, ga, ga, a0 * 256, a0 * 256, 1});
        for (int64_t b = a + 1; b < m; ++b) {
            const int64_t b0 = b * g, gb = nsb - b0 < g ? nsb - b0 : g;
            out.push_back(MmaBand{a0, b0, ga, gb, a0 * 256, b0 * 256 - g * 256, 0});
        }
    }
    return out;
}

template <bool kFp4>
cudaError_t launch_count_tensor(int64_t n, const uint64_t* bits, int64_t row_words, int64_t* hist, void* workspace,
                                size_t ws_bytes, cudaStream_t st, const double* phi, double* layer, int kmax) {
    WsHeader* hdr = static_cast<WsHeader*>(workspace);
    const int64_t hist_len = n > 1 ? n - 1 : 1;
    cudaError_t err = cudaMemsetAsync(hist, 0, size_t(hist_len) * 8, st);
    if (err != cudaSuccess) return err;
    if ((err = cudaMemsetAsync(&hdr->counter, 0, sizeof(hdr->counter), st)) != cudaSuccess) return err;
    if (n < 2) return cudaSuccess;
    const int64_t nsb = (n + 255) / 256;
    // FP4: the whole E when it fits the workspace, else bands of g panels
    const int64_t g = kFp4 ? mma4_band_panels(n, ws_bytes) : nsb;
    if (g < 1) return cudaErrorMemoryAllocation;
    const bool banded = g < nsb;
    const MmaLayout lay = banded ? mma4_band_layout(n, g) : mma_layout(n, kFp4);
    uint8_t* op0 = static_cast<uint8_t*>(workspace) + lay.op0;
    uint8_t* op1 = static_cast<uint8_t*>(workspace) + lay.op1;

    auto kernel = !kFp4 ? k_count_mma : kmax >= 0 ? k_count_mma4<FmtF4Layers> : k_count_mma4<FmtF4>;
    std::atomic<bool>* attr = !kFp4 ? g_attr_set : kmax >= 0 ? g_attr4l_set : g_attr4_set;
    int dev = 0;
    if ((err = cudaGetDevice(&dev)) != cudaSuccess) return err;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    constexpr int kSmem = kFp4 ? smem_bytes<FmtF4>() : smem_bytes<FmtF8>();
    static_assert(smem_bytes<FmtF4Layers>() == smem_bytes<FmtF4>(), "one shared-memory size per format family");
    if (!attr[dev]) {
        err = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
        if (err != cudaSuccess) return err;
        attr[dev] = true;
    }
    const int raster = auto_raster(n);
    const int64_t kblocks = lay.row / kBK;
    unsigned long long* h = reinterpret_cast<unsigned long long*>(hist);

    if constexpr (!kFp4) {
        k_expand_f8<<<unsigned(expand_grid(n)), 256, 0, st>>>(bits, n, row_words, lay.kpad, op0, op1);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
        MmaMaps maps;
        if (encode_operand_maps(&maps, n, lay.kpad, false, op0, op1) != CUDA_SUCCESS) return cudaErrorInvalidValue;
        const int64_t nitems = mma_items(n, raster);
        int64_t grid = device_sm_count();
        if (grid > nitems) grid = nitems;
        kernel<<<unsigned(grid), kThreads, kSmem, st>>>(maps, bits, n, row_words, nsb, nitems, kblocks, h, hist_len,
                                                        phi, layer, kmax, raster, MmaBand{0, 0, nsb, nsb, 0, 0, 1},
                                                        hdr);
        return cudaGetLastError();
    } else {
        // One persistent pair grid per band; its queue counter restarts at 0.
        auto count_band = [&](const MmaMaps& maps, const MmaBand& band, bool reset) -> cudaError_t {
            const int64_t nitems = band_items(band, raster);
            cudaError_t e = reset ? cudaMemsetAsync(&hdr->counter, 0, sizeof(hdr->counter), st) : cudaSuccess;
            if (e != cudaSuccess) return e;
            cudaLaunchAttribute at[1];
            cudaLaunchConfig_t cfg;
            int pairs = 0;
            if ((e = pair_config(kernel, kSmem, attr, kmax >= 0 ? g_clusters4l : g_clusters4, nitems / 2, st, at,
                                 &cfg, &pairs)) != cudaSuccess)
                return e;
            return cudaLaunchKernelEx(&cfg, kernel, maps, bits, n, row_words, nsb, nitems, kblocks, h, hist_len, phi,
                                      layer, kmax, raster, band, hdr);
        };
        if (!banded) {
            k_expand_f4<<<unsigned(expand_grid(n)), 256, 0, st>>>(bits, n, row_words, lay.kpad, op0, op1,
                                                                  mma4_dl_offset(n));
            if ((err = cudaGetLastError()) != cudaSuccess) return err;
            MmaMaps maps;
            if (encode_operand_maps(&maps, n, lay.kpad, true, op0, op1) != CUDA_SUCCESS) return cudaErrorInvalidValue;
            return count_band(maps, MmaBand{0, 0, nsb, nsb, 0, 0, 1}, false);
        }
        // Bands.  Supertile rows fall into groups of g panels; for each group
        // a, its E rows (the A rows of every band (a, b), and the B rows of
        // the triangle (a, a)) take band rows [0, 256 g), from column 256 g a
        // on; for each later group b, its rows take band rows [256 g, 512 g),
        // columns 256 g a up to the end of group b (the K range of the bands
        // (a, b)).  DU and DL hold every row, written once.  Each band's E map
        // ends at the last band row that holds a row of the set, so the
        // rows past n read as zeros, as in the whole-set map.
        const int ppr = int(lay.kpad / 32);
        const int64_t dl_off = mma4_dl_offset(n);
        k_expand_f4_band<<<unsigned(expand_grid(n)), 256, 0, st>>>(bits, row_words, lay.kpad, op0, 0, n, 0, 0, 0,
                                                                   op1, dl_off);
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
        MmaMaps maps;
        if (encode_operand_maps(&maps, n, lay.kpad, true, op0, op1) != CUDA_SUCCESS) return cudaErrorInvalidValue;
        bool first = true;
        for (const MmaBand& band : mma4_bands(n, g)) {
            // the rows this band brings into the buffer: a triangle's group
            // (the A rows of its group's later bands too), or a rectangle's
            // second group, over the columns from the first group's start
            const int64_t p0 = band.diag ? band.i0 : band.j0, np = band.diag ? band.ni : band.nj;
            const int64_t r0 = p0 * 256, r1 = (p0 + np) * 256 < n ? (p0 + np) * 256 : n;
            const int c1 = band.diag ? ppr : (int((p0 + np) * 8) < ppr ? int((p0 + np) * 8) : ppr);
            const int64_t e0 = band.diag ? 0 : g * 256;  // first band row written
            k_expand_f4_band<<<unsigned(expand_grid(r1 - r0)), 256, 0, st>>>(
                bits, row_words, lay.kpad, op0, r0, r1, e0, int(band.i0 * 8), c1, nullptr, 0);
            if ((err = cudaGetLastError()) != cudaSuccess) return err;
            if (encode_e_map(&maps.m[kMapE], lay.kpad, op0, e0 + (r1 - r0)) != CUDA_SUCCESS)
                return cudaErrorInvalidValue;
            if ((err = count_band(maps, band, !first)) != cudaSuccess) return err;
            first = false;
        }
        return cudaSuccess;
    }
}

}  // namespace

int64_t mma4_band_cover(int64_t n, int64_t g, int raster, int64_t* counts) {
    const int64_t nsb = (n + 255) / 256;
    std::memset(counts, 0, size_t(nsb) * size_t(nsb) * sizeof(int64_t));
    int64_t items = 0;
    for (const MmaBand& band : mma4_bands(n, g)) {
        const int64_t slots = band_items(band, raster);
        for (int64_t t = 0; t < slots; t += 2) {  // a pair's unit u is slot 2 u
            int64_t si, sj, half;
            if (!decode_band(t, band, n, raster, si, sj, half)) continue;
            ++counts[si * nsb + sj];
            ++items;
        }
    }
    return items;
}

cudaError_t launch_count_mma(int64_t n, const uint64_t* bits, int64_t row_words, int64_t* hist, void* workspace,
                             cudaStream_t st, const double* phi, double* layer, int kmax) {
    return launch_count_tensor<false>(n, bits, row_words, hist, workspace, mma_workspace_bytes(n), st, phi, layer,
                                      kmax);
}

cudaError_t launch_count_mma4(int64_t n, const uint64_t* bits, int64_t row_words, int64_t* hist, void* workspace,
                              size_t ws_bytes, cudaStream_t st, const double* phi, double* layer, int kmax) {
    return launch_count_tensor<true>(n, bits, row_words, hist, workspace, ws_bytes, st, phi, layer, kmax);
}

}  // namespace cs
