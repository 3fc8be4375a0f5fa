// cs_relate.cuh -- one block of the causal-matrix build (2048 columns x 64
// rows), shared by the single-set and batched relate kernels.
#pragma once

#include "cs_internal.cuh"

namespace cs {

constexpr int kRelColsPerBlock = 2048;
constexpr int kRelWordsPerBlock = kRelColsPerBlock / 64;
constexpr int kRelRowsPerBlock = 64;
constexpr int kRelThreads = 256;

// Geometries of the relation test; the number of coordinates is geom_dim(G).
constexpr int kGeomLightCone = 2, kGeom3 = 3, kGeom4 = 4, kGeomDeSitter = 5;
constexpr int geom_dim(int g) { return g == kGeomDeSitter ? 2 : g; }

// Symmetric timelike test between row element ci and staged column `col`:
// du * dv > 0 (1+1, light-cone coordinates), dt^2 - |dx|^2 > 0 (2+1, 3+1)
// exact in int64, or, on a circle (the de Sitter slab's conformal grid, Eq.
// ds_metric, and the 1+1 cylinder), the angular separation below the
// (conformal-)time separation.
template <int G>
__device__ __forceinline__ bool rel_related(const int32_t (&ci)[geom_dim(G)], const int32_t (*sc)[kRelColsPerBlock],
                                            int col) {
    if constexpr (G == kGeomDeSitter) {
        // |eta| < 2^30 (slab: < 2^29, cylinder: < 2^31 / pi), so de fits
        // int32; theta differences wrap modulo 2^32, one full turn.
        const int32_t de = sc[0][col] - ci[0];
        const uint32_t d = uint32_t(sc[1][col]) - uint32_t(ci[1]);
        const uint32_t circ = min(d, 0u - d);
        return circ < uint32_t(abs(de));
    } else if constexpr (G == kGeomLightCone) {
        // du * dv > 0 as a sign test (|du|, |dv| < 2^31 fit int32)
        const int32_t du = sc[0][col] - ci[0];
        const int32_t dv = sc[1][col] - ci[1];
        return (du ^ dv) >= 0 && du != 0 && dv != 0;
    } else {
        // |coordinates| < 2^29: differences fit int32 and each square is one
        // widening multiply-add into the int64 sum (< 2^62, exact)
        const int32_t dt = sc[0][col] - ci[0];
        int64_t s2 = int64_t(dt) * dt;
#pragma unroll
        for (int d = 1; d < G; ++d) {
            const int32_t dx = sc[d][col] - ci[d];
            s2 -= int64_t(dx) * dx;
        }
        return s2 > 0;
    }
}

// FP32 filter for the 2+1 and 3+1 tests.  With every coordinate in
// [-kFilterRange, kFilterRange] = [-2^20, 2^20] the coordinates and their
// differences (|d| <= 2^21) are exact in FP32, every partial result of
// dt^2 - dx^2 - ... is below 2^44 in magnitude, so each of the (at most
// five) roundings is at most 2^20 and the FP32 value lies within
// kFilterSlack = 2^23 of the exact one: above it the pair is related, below
// its negative it is not, and only in between the exact int64 test runs.
constexpr int32_t kFilterRange = 1 << 20;
constexpr float kFilterSlack = 8388608.0f;  // 2^23

// s2 = dt^2 - dx^2 - dy^2 (- dz^2) in FP32 between a row (rc) and a staged
// column x = (t, x, y, z), z = 0 in 2+1; the same chain of roundings
// everywhere, so that every test of a pair decides alike.
template <int DIM>
__device__ __forceinline__ float filter_s2(const float (&rc)[4], float4 x) {
    const float dt = x.x - rc[0];
    float s2 = dt * dt;
    const float dx = x.y - rc[1];
    s2 = fmaf(-dx, dx, s2);
    const float dy = x.z - rc[2];
    s2 = fmaf(-dy, dy, s2);
    if constexpr (DIM == 4) {
        const float dz = x.w - rc[3];
        s2 = fmaf(-dz, dz, s2);
    }
    return s2;
}

// The lane-per-word form's chain: 2^23 - s2 = 2^23 - dt^2 + dx^2 + dy^2
// (+ dz^2), each square added by one fused multiply-add.  Every partial
// result is below 2^44 in magnitude, so each of the (at most four) roundings
// is at most 2^20 and the value lies within 2^22 of the exact one: negative
// means s2 > 2^23 - 2^22 > 0 (related), above 2^24 means s2 < 0, and only
// [0, 2^24] needs the exact test.
template <int DIM>
__device__ __forceinline__ float filter_offset(const float (&rc)[4], float4 x) {
    const float dt = x.x - rc[0];
    float s = fmaf(-dt, dt, kFilterSlack);
    const float dx = x.y - rc[1];
    s = fmaf(dx, dx, s);
    const float dy = x.z - rc[2];
    s = fmaf(dy, dy, s);
    if constexpr (DIM == 4) {
        const float dz = x.w - rc[3];
        s = fmaf(dz, dz, s);
    }
    return s;
}
// Bits of the float 2^24: a value in [+0, 2^24] has bits at most this as an
// unsigned integer, and every negative value (sign bit set) has more.
constexpr uint32_t kBandBits = 0x4B800000u;

// The exact int64 test on the same (integral) coordinates.
template <int DIM>
__device__ __forceinline__ bool exact_related(const float (&rc)[4], float4 x) {
    const int32_t dt = int32_t(x.x) - int32_t(rc[0]), dx = int32_t(x.y) - int32_t(rc[1]),
                  dy = int32_t(x.z) - int32_t(rc[2]), dz = int32_t(x.w) - int32_t(rc[3]);
    int64_t e2 = int64_t(dt) * dt - int64_t(dx) * dx - int64_t(dy) * dy;
    if constexpr (DIM == 4) e2 -= int64_t(dz) * dz;
    return e2 > 0;
}

// The filtered test: the FP32 sign outside the band, the exact one inside.
template <int DIM>
__device__ __forceinline__ bool rel_filtered(const float (&rc)[4], float4 x) {
    const float s2 = filter_s2<DIM>(rc, x);
    if (s2 > kFilterSlack) return true;
    if (s2 < -kFilterSlack) return false;
    return exact_related<DIM>(rc, x);
}

// Light-cone kinds.  Labels are in time order, so in a word wholly after
// the row tile only the future cone can hold (u_j > u_i and v_j > v_i); for
// a random 2D order labelled by u the u test is implied by j > i and only v
// is compared (USE_U = false).  Each lane owns one word (64 columns) of the
// block and tests its columns one by one, for four rows at a time, with no
// ballots.  Coordinates lie in [0, 2^31), so x_j - x_i - 1 fits int32 and is
// non-negative iff x_j > x_i: a test is one or two integer multiply-adds
// (x_j * 1 + ~x_i, on the FMA pipe, the multiplier a runtime 1 so that the
// compiler keeps the multiply-add), an OR of the two with u, and a funnel
// shift that appends the sign bit to the half-word's accumulator; the
// accumulated sign bits are the complement of the relation bits.  The
// compare-and-OR form it replaces kept the integer ALU pipe saturated.
// The column coordinates are staged transposed, st[c][w] = column 64 w + c
// (row pitch kConePitch: the lanes' reads of one offset c hit consecutive
// banks); columns at or beyond n are staged as 0, which no cone test
// passes.  The row tile's own word (lane ws) takes the full symmetric test
// by ballots; words before the row tile are left to mirror_block.
constexpr int kConePitch = kRelWordsPerBlock + 1;  // staged words per column offset
constexpr int kConeRows = 4;                        // rows a lane tests together
constexpr int kStageInts = 4 * kRelColsPerBlock;    // staging ints any geometry needs
constexpr int kConeOne = 2 * 64 * kConePitch;       // after the (u, v) staging: a runtime 1 (the multiplier)
constexpr int kConeInts = kConeOne + 1;             // staging ints of the light-cone kinds
static_assert(kStageInts >= kConeInts, "the transposed (u, v) staging and the 1 fit");

// x * one + y as a multiply-add (one is 1 at run time).
__device__ __forceinline__ int32_t cone_mad(int32_t x, int32_t one, int32_t y) {
    int32_t d;
    asm("mad.lo.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(x), "r"(one), "r"(y));
    return d;
}

// Lane `lane` stores word w0 + lane of row i (words before the row tile are
// mirror_block's), and, when zero_from >= 0, zeroes word zero_from + lane
// (padding words past the last chunk of a row, fewer than 32).
__device__ __forceinline__ void store_row_words(uint64_t* __restrict__ bits, int64_t i, int64_t row_words, int64_t w0,
                                                int lane, int wbeg, uint64_t word, int64_t zero_from) {
    if (lane >= wbeg && w0 + lane < row_words) bits[i * row_words + w0 + lane] = word;
    if (zero_from >= 0 && zero_from + lane < row_words) bits[i * row_words + zero_from + lane] = 0ull;
}

// The lane layout of the lane-per-word forms: W words from w0 (a power of
// two, at most 32, the fewest covering the chunk's valid words), lane l
// testing word l % W for the rows of row group l / W.  A chunk at the end of
// a row with few valid words then keeps its lanes busy on more rows instead
// of on words past the row's end.
__device__ __forceinline__ int lane_words(int64_t valid) {
    int W = 1;
    while (W < valid && W < kRelWordsPerBlock) W <<= 1;
    return W;
}

// Per row of the block, all lanes of a warp: the row tile's own word when
// ws >= 0 (own(i, k): the relation of row i with column offset k of word ws,
// folded by two ballots) and the zero padding words [z0, z1) of the row.
template <class Own>
__device__ __forceinline__ void own_words_and_padding(uint64_t* __restrict__ bits, int64_t row_words, int64_t w0,
                                                      int64_t r0, int64_t r1, int ws, int64_t z0, int64_t z1,
                                                      Own own) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int kWarps = kRelThreads / 32;
    if (ws < 0 && z0 >= z1) return;
    for (int64_t i = r0 + warp; i < r1; i += kWarps) {
        if (ws >= 0) {
            const bool b0 = own(i, lane), b1 = own(i, lane + 32);
            const uint64_t d = (uint64_t(__ballot_sync(0xffffffffu, b1)) << 32) | __ballot_sync(0xffffffffu, b0);
            if (lane == 0) bits[i * row_words + w0 + ws] = d;
        }
        for (int64_t w = z0 + lane; w < z1; w += 32) bits[i * row_words + w] = 0ull;
    }
}

template <bool USE_U>
__device__ __forceinline__ void relate_rows_cone(const int32_t* __restrict__ coords, int64_t n,
                                                 uint64_t* __restrict__ bits, int64_t row_words, int64_t w0,
                                                 int64_t c0, int64_t r0, int64_t r1, int ws,
                                                 const int32_t* __restrict__ st, int64_t zero_from) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int kWarps = kRelThreads / 32;
    const int2* st2 = reinterpret_cast<const int2*>(st);  // USE_U: (u, v) pairs
    const int wbeg = ws > 0 ? ws : 0;
    const int32_t one = st[kConeOne];
    for (int64_t ib = r0 + int64_t(warp) * kConeRows; ib < r1; ib += int64_t(kWarps) * kConeRows) {
        int32_t ru[kConeRows], rv[kConeRows], nu[kConeRows], nv[kConeRows];
        uint32_t lo[kConeRows], hi[kConeRows];
#pragma unroll
        for (int r = 0; r < kConeRows; ++r) {
            const int64_t i = ib + r;
            ru[r] = i < r1 ? coords[i] : INT32_MAX;  // a missing row passes no test
            rv[r] = i < r1 ? coords[n + i] : INT32_MAX;
            nu[r] = ~ru[r];  // -x_i - 1
            nv[r] = ~rv[r];
            lo[r] = hi[r] = 0u;
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {  // the word's low and high halves
            // highest column first: after 32 shifts column 32 h is bit 0
#pragma unroll 8
            for (int c = 32 * h + 31; c >= 32 * h; --c) {
                int32_t xu = 0, xv;
                if constexpr (USE_U) {
                    const int2 x = st2[c * kConePitch + lane];
                    xu = x.x;
                    xv = x.y;
                } else {
                    xv = st[c * kConePitch + lane];
                }
#pragma unroll
                for (int r = 0; r < kConeRows; ++r) {
                    // sign bit set iff the column is not in the future cone
                    const int32_t d = USE_U ? (cone_mad(xu, one, nu[r]) | cone_mad(xv, one, nv[r]))
                                            : cone_mad(xv, one, nv[r]);
                    if (h == 0) lo[r] = __funnelshift_l(uint32_t(d), lo[r], 1);
                    else hi[r] = __funnelshift_l(uint32_t(d), hi[r], 1);
                }
            }
        }
#pragma unroll
        for (int r = 0; r < kConeRows; ++r) {
            const int64_t i = ib + r;
            if (i >= r1) break;  // warp-uniform
            uint64_t word = ~((uint64_t(hi[r]) << 32) | lo[r]);
            if (ws >= 0) {  // the row tile's own word: full test (warp-uniform)
                bool b[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int k = lane + 32 * h;  // column offset in the word
                    const int64_t j = c0 + int64_t(ws) * 64 + k;
                    if constexpr (USE_U) {
                        const int2 x = st2[k * kConePitch + ws];
                        const int32_t du = x.x - ru[r], dv = x.y - rv[r];
                        b[h] = j < n && (du ^ dv) >= 0 && du != 0 && dv != 0;
                    } else {  // u increases with the label
                        const int32_t xv = st[k * kConePitch + ws];
                        b[h] = j < n && (j > i ? xv > rv[r] : (j < i && xv < rv[r]));
                    }
                }
                const uint64_t d = (uint64_t(__ballot_sync(0xffffffffu, b[1])) << 32) | __ballot_sync(0xffffffffu, b[0]);
                if (lane == ws) word = d;
            }
            store_row_words(bits, i, row_words, w0, lane, wbeg, word, zero_from);
        }
    }
}

// 2+1 and 3+1 with the FP32 filter, laid out like the light-cone kinds: each
// lane owns one word and tests its 64 columns one by one against two rows
// held in registers.  The columns are staged as float4 (t, x, y, z; z = 0 in
// 2+1) at st4[c * 32 + (w ^ (c & 7))] for column 64 w + c of the block: one
// 16-byte load per column and lane, conflict-free for the lanes' loads of
// one offset c and for the staging stores of consecutive columns.  A test is
// filter_offset's chain, a funnel shift of its sign (set: related) into the
// half-word's accumulator and an unsigned minimum of its bits; a word whose
// minimum shows a value in [0, 2^24] (near the light cone, about one word in
// a thousand) is recomputed exactly by its lane.  Columns at or beyond n are
// staged 10^9 units away in space (far outside the cone and the band) and
// masked off.  The row tile's own word (lane ws, which holds the diagonal)
// takes the filtered test by ballots; words before the row tile are left to
// mirror_block.
constexpr int kFiltRows = 2;  // rows a lane tests together (the 48-register budget of the batched kernel)

template <int DIM>
__device__ __forceinline__ void relate_rows_filtered(const int32_t* __restrict__ coords, int64_t n,
                                                     uint64_t* __restrict__ bits, int64_t row_words, int64_t w0,
                                                     int64_t c0, int64_t r0, int64_t r1, int ws, int W,
                                                     const float4* __restrict__ st4) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int kWarps = kRelThreads / 32;
    const int wbeg = ws > 0 ? ws : 0;
    const int wl = lane & (W - 1);                                   // this lane's word
    const int64_t pass = int64_t(kFiltRows) * (kRelWordsPerBlock / W);  // rows of one warp pass
    const int64_t g0 = int64_t(lane / W) * kFiltRows;                 // this lane's first row in a pass
    // with W = 32 a pass's rows are the same in every lane, and the row
    // tile's own word is folded by ballots right here; narrower layouts
    // leave it to own_words_and_padding
    const bool inline_own = W == kRelWordsPerBlock && ws >= 0;
    const bool keep = wl >= wbeg && (wl != ws || inline_own) && w0 + wl < row_words;
    const int64_t cw = c0 + 64 * int64_t(wl);  // this lane's first column
    const uint64_t valid = cw >= n ? 0ull : (n - cw >= 64 ? ~0ull : (~0ull >> (64 - (n - cw))));
    for (int64_t ib = r0 + int64_t(warp) * pass; ib < r1; ib += int64_t(kWarps) * pass) {
        float rc[kFiltRows][4];
        uint32_t lo[kFiltRows], hi[kFiltRows];
        uint32_t band[kFiltRows];  // unsigned minimum of the chain's bits
#pragma unroll
        for (int r = 0; r < kFiltRows; ++r) {
            const int64_t i = ib + g0 + r;
#pragma unroll
            for (int d = 0; d < 4; ++d) rc[r][d] = (d < DIM && i < r1) ? float(coords[d * n + i]) : 0.0f;
            lo[r] = hi[r] = 0u;
            band[r] = ~0u;
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            // highest column first: after 32 shifts column 32 h is bit 0
#pragma unroll 4
            for (int c = 32 * h + 31; c >= 32 * h; --c) {
                const float4 x = st4[c * 32 + (wl ^ (c & 7))];
#pragma unroll
                for (int r = 0; r < kFiltRows; ++r) {
                    const uint32_t sb = __float_as_uint(filter_offset<DIM>(rc[r], x));
                    if (h == 0) lo[r] = __funnelshift_l(sb, lo[r], 1);
                    else hi[r] = __funnelshift_l(sb, hi[r], 1);
                    band[r] = min(band[r], sb);
                }
            }
        }
#pragma unroll
        for (int r = 0; r < kFiltRows; ++r) {
            const int64_t i = ib + g0 + r;
            uint64_t word = ((uint64_t(hi[r]) << 32) | lo[r]) & valid;
            if (keep && i < r1 && wl != ws && band[r] <= kBandBits) {  // near the light cone: the word exactly
                word = 0ull;
                for (int c = 0; c < 64 && cw + c < n; ++c)
                    if (rel_filtered<DIM>(rc[r], st4[c * 32 + (wl ^ (c & 7))])) word |= 1ull << c;
            }
            if (inline_own) {
                if (i >= r1) break;  // warp-uniform (g0 = 0)
                bool b[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int k = lane + 32 * h;  // column offset in the word
                    b[h] = c0 + int64_t(ws) * 64 + k < n && rel_filtered<DIM>(rc[r], st4[k * 32 + (ws ^ (k & 7))]);
                }
                const uint64_t d = (uint64_t(__ballot_sync(0xffffffffu, b[1])) << 32) | __ballot_sync(0xffffffffu, b[0]);
                if (lane == ws) word = d;
            }
            if (keep && i < r1) bits[i * row_words + w0 + wl] = word;
        }
    }
}

// Rows [rb*64, rb*64+64) x words [w0, w0+32) of the bitset, less the
// words wholly before the row tile (word < rb): the relation is symmetric,
// so mirror_block fills those as transposes.  Column coordinates are staged
// in shared memory `sc` (kStageInts ints, 16-byte aligned).  The light-cone
// kinds test one cone per word (relate_rows_cone); order2d: the set is a
// random 2D order whose coords[0] (u) increases strictly with the label,
// which also drops the u test there.  The other geometries stage sc[d][col]
// and each warp folds 64 tests per word into a uint64 with two
// __ballot_sync, lane w keeps word w, and a row's words leave in one
// coalesced store.  zero_from >= 0: the block also zeroes each row's words
// [zero_from, row_words) (padding past a row's last chunk).  Must be called
// by all 256 threads.
template <int G>
__device__ __forceinline__ void relate_block(const int32_t* __restrict__ coords, int64_t n,
                                             uint64_t* __restrict__ bits, int64_t row_words, int64_t rb, int64_t w0,
                                             int32_t* sc, bool order2d = false, int64_t zero_from = -1) {
    constexpr int DIM = geom_dim(G);
    const int64_t c0 = w0 * 64;
    if (w0 + kRelWordsPerBlock <= rb) return;  // wholly below the diagonal
    // first word of the block at or after the row tile (< 0: all of them)
    const int ws = rb - w0 < 0 ? -1 : int(rb - w0);
    const int wbeg = ws > 0 ? ws : 0;
    const int64_t r0 = rb * kRelRowsPerBlock;
    const int64_t r1 = r0 + kRelRowsPerBlock < n ? r0 + kRelRowsPerBlock : n;
    // The filtered 3+1 and 2+1 form tests W = lane_words(valid words) words
    // from w0 and zeroes the row's words [w0 + W, z1) past them: the rest of
    // the block's 32, and, at a row's last chunk (zero_from >= 0), the
    // padding to row_words.  (The light-cone test, at a few instructions,
    // gained less from narrow blocks than their fixed costs took, and keeps
    // all 32 lanes on words.)
    const int64_t z1 = zero_from >= 0 ? row_words : (w0 + kRelWordsPerBlock < row_words ? w0 + kRelWordsPerBlock
                                                                                          : row_words);
    auto pad_from = [&](int W) { return w0 + W < z1 ? w0 + W : z1; };
    if constexpr (G == kGeomLightCone) {  // time order: one cone per word, see above
        // transposed staging, word w of the block at row offset c: column 64 w + c
        for (int t = threadIdx.x + 64 * wbeg; t < kRelColsPerBlock; t += kRelThreads) {
            const int64_t col = c0 + t;
            const int at = (t & 63) * kConePitch + (t >> 6);
            if (order2d) {
                sc[at] = col < n ? coords[n + col] : 0;
            } else {
                reinterpret_cast<int2*>(sc)[at] =
                    col < n ? make_int2(coords[col], coords[n + col]) : make_int2(0, 0);
            }
        }
        if (threadIdx.x == 0) sc[kConeOne] = 1;
        __syncthreads();
        if (order2d) relate_rows_cone<false>(coords, n, bits, row_words, w0, c0, r0, r1, ws, sc, zero_from);
        else relate_rows_cone<true>(coords, n, bits, row_words, w0, c0, r0, r1, ws, sc, zero_from);
    } else {
        auto sd = reinterpret_cast<int32_t(*)[kRelColsPerBlock]>(sc);
        // 2+1 and 3+1: when the block's columns and rows all lie within
        // kFilterRange the columns are staged as floats for the FP32 filter.
        constexpr bool kFilter = G == kGeom3 || G == kGeom4;
        constexpr int kPer = kRelColsPerBlock / kRelThreads;  // staged columns per thread
        int32_t v[kPer][DIM];
        int out = 0;
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const int t = threadIdx.x + q * kRelThreads;
            const int64_t c = c0 + t;
#pragma unroll
            for (int d = 0; d < DIM; ++d) {
                v[q][d] = (t >= 64 * wbeg && c < n) ? coords[d * n + c] : 0;
                out |= v[q][d] < -kFilterRange || v[q][d] > kFilterRange;
            }
        }
        if (kFilter && threadIdx.x < r1 - r0) {
#pragma unroll
            for (int d = 0; d < DIM; ++d) {
                const int32_t x = coords[d * n + r0 + threadIdx.x];
                out |= x < -kFilterRange || x > kFilterRange;
            }
        }
        const bool fast = kFilter && !__syncthreads_or(out);
        if constexpr (kFilter) {
            if (fast) {
                float4* st4 = reinterpret_cast<float4*>(sc);
#pragma unroll
                for (int q = 0; q < kPer; ++q) {
                    const int t = threadIdx.x + q * kRelThreads;
                    if (t < 64 * wbeg) continue;
                    const int c = t & 63, w = t >> 6;
                    float f[4] = {0.0f, 1e9f, 0.0f, 0.0f};  // a column at or beyond n: far away in space
                    if (c0 + t < n) {
#pragma unroll
                        for (int d = 0; d < 4; ++d) f[d] = d < DIM ? float(v[q][d < DIM ? d : 0]) : 0.0f;
                    }
                    st4[c * 32 + (w ^ (c & 7))] = make_float4(f[0], f[1], f[2], f[3]);
                }
                __syncthreads();
                // the row tile's own word (it holds the diagonal): the filtered test
                auto own = [&](int64_t i, int k) {
                    if (c0 + int64_t(ws) * 64 + k >= n) return false;
                    float rc[4];
#pragma unroll
                    for (int d = 0; d < 4; ++d) rc[d] = d < DIM ? float(coords[d * n + i]) : 0.0f;
                    return rel_filtered<DIM>(rc, st4[k * 32 + (ws ^ (k & 7))]);
                };
                const int W = lane_words((n + 63) / 64 - w0);
                relate_rows_filtered<DIM>(coords, n, bits, row_words, w0, c0, r0, r1, ws, W, st4);
                own_words_and_padding(bits, row_words, w0, r0, r1, W == kRelWordsPerBlock ? -1 : ws, pad_from(W), z1,
                                      own);
                return;
            }
        }
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const int t = threadIdx.x + q * kRelThreads;
            if (t < 64 * wbeg) continue;
#pragma unroll
            for (int d = 0; d < DIM; ++d) sd[d][t] = v[q][d];
        }
        __syncthreads();
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int64_t i = r0 + warp; i < r1; i += kRelThreads / 32) {
            int32_t ci[DIM];
#pragma unroll
            for (int d = 0; d < DIM; ++d) ci[d] = coords[d * n + i];
            uint64_t mine = 0;
#pragma unroll 4
            for (int w = wbeg; w < kRelWordsPerBlock; ++w) {
                const int col = w * 64 + lane;
                const bool b0 = c0 + col < n && rel_related<G>(ci, sd, col);
                const bool b1 = c0 + col + 32 < n && rel_related<G>(ci, sd, col + 32);
                const uint32_t lo = __ballot_sync(0xffffffffu, b0);
                const uint32_t hi = __ballot_sync(0xffffffffu, b1);
                if (lane == w) mine = (uint64_t(hi) << 32) | lo;
            }
            store_row_words(bits, i, row_words, w0, lane, wbeg, mine, zero_from);
        }
    }
}

// ------------------------------------------------ light-cone column tables
//
// In the light-cone kinds a row i and a column tile C wholly after i's row
// tile relate exactly where u_j > u_i and v_j > v_i (the future cone; labels
// are in time order).  Sorting the tile's 64 values of one coordinate turns
// "the columns whose value exceeds y" into a suffix of the sorted order, so
// with the suffix masks precomputed the whole 64-bit word is
//   above_u[#{p : us[p] <= u_i}] & above_v[#{p : vs[p] <= v_i}],
// two binary searches of six steps instead of 64 tests (for a random 2D
// order, whose u increases with the label, the v term alone).  Columns at or
// beyond n hold -1, which exceeds no coordinate (all lie in [0, 2^31)).
struct alignas(16) ConeTable {
    int32_t xs[2][64];      // u and v of the tile's columns, each sorted ascending
    uint64_t above[2][66];  // above[x][m], m <= 64: the columns at sorted positions >= m of coordinate x
    uint32_t pad[4];        // 1584 bytes: consecutive tables start at different 16-byte offsets of
};                          // a 128-byte line, so the lanes' bucket loads spread over the banks
static_assert(sizeof(ConeTable) == 1584, "cone table layout");

// Table of column tile C, one full warp.  The 64 keys (value + 1) << 6 |
// column, two per lane (element lane + 32 h), go through a bitonic network
// (partners at distance 32 inside the lane, the others by shuffles); after
// it element e is the e-th smallest, and a suffix OR over the elements gives
// the masks.  order2d: only the v table (its u is the label order).
__device__ __forceinline__ void build_cone_table(const int32_t* __restrict__ coords, int64_t n, int64_t C,
                                                 bool order2d, ConeTable* __restrict__ t) {
    const int lane = threadIdx.x & 31;
    for (int x = order2d ? 1 : 0; x < 2; ++x) {
        uint64_t k[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t col = 64 * C + lane + 32 * h;
            const int32_t v = col < n ? coords[x * n + col] : -1;
            k[h] = (uint64_t(uint32_t(v + 1)) << 6) | uint64_t(lane + 32 * h);
        }
#pragma unroll
        for (int size = 2; size <= 64; size <<= 1) {
#pragma unroll
            for (int j = size >> 1; j > 0; j >>= 1) {
                if (j == 32) {  // size 64: ascending, partner e + 32 in the same lane
                    const uint64_t lo = k[0] < k[1] ? k[0] : k[1], hi = k[0] < k[1] ? k[1] : k[0];
                    k[0] = lo;
                    k[1] = hi;
                } else {
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int e = lane + 32 * h;
                        const uint64_t p = __shfl_xor_sync(0xffffffffu, k[h], j);
                        const bool keep_min = ((e & j) == 0) == ((e & size) == 0);
                        k[h] = keep_min ? (k[h] < p ? k[h] : p) : (k[h] < p ? p : k[h]);
                    }
                }
            }
        }
        t->xs[x][lane] = int32_t(uint32_t(k[0] >> 6)) - 1;
        t->xs[x][lane + 32] = int32_t(uint32_t(k[1] >> 6)) - 1;
        uint64_t s0 = 1ull << (k[0] & 63), s1 = 1ull << (k[1] & 63);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t a = __shfl_down_sync(0xffffffffu, s0, o), b = __shfl_down_sync(0xffffffffu, s1, o);
            if (lane + o < 32) {
                s0 |= a;
                s1 |= b;
            }
        }
        s0 |= __shfl_sync(0xffffffffu, s1, 0);  // every element of the upper half follows the lower half
        t->above[x][lane] = s0;
        t->above[x][lane + 32] = s1;
        if (lane == 0) t->above[x][64] = 0ull;
    }
}

// #{m < 7 : s[m] <= y} for ascending s, by binary lifting with selects
// (steps of 4, 2, 1): three compares instead of seven.
__device__ __forceinline__ int cone_lift7(int32_t s0, int32_t s1, int32_t s2, int32_t s3, int32_t s4, int32_t s5,
                                          int32_t s6, int32_t y) {
    const bool a = s3 <= y;
    const bool b = (a ? s5 : s1) <= y;
    const bool d = (a ? (b ? s6 : s4) : (b ? s2 : s0)) <= y;
    return (a ? 4 : 0) + (b ? 2 : 0) + (d ? 1 : 0);
}

// #{p : xs[p] <= y} over 64 ascending values, and the mask of the columns
// above y.  s[m] = xs[8 m + 7] (m < 7) are the bucket splitters, kept in
// registers: they give the buckets wholly at or below y, then the one
// 32-byte bucket that may straddle y is loaded and counted the same way.
__device__ __forceinline__ uint64_t cone_above(const int32_t* __restrict__ xs, const uint64_t* __restrict__ above,
                                               const int32_t (&s)[7], int32_t y) {
    const int c1 = cone_lift7(s[0], s[1], s[2], s[3], s[4], s[5], s[6], y);
    const int4 a = reinterpret_cast<const int4*>(xs)[2 * c1], b = reinterpret_cast<const int4*>(xs)[2 * c1 + 1];
    const int c = 8 * c1 + cone_lift7(a.x, a.y, a.z, a.w, b.x, b.y, b.z, y) + (b.w <= y ? 1 : 0);
    return above[c];
}

// Bytes of dynamic shared memory of relate_block_tables: 32 tables, the own
// tile's columns, the copy's mbarrier.
constexpr int kConeTableSmem = kRelWordsPerBlock * int(sizeof(ConeTable)) + 128 * 4 + 16;

// Rows [64 rb, 64 rb + 64) x words [w0, w0 + 32) (w0 >= rb) of a light-cone
// set from its column tables (tables[C] for column tile C): the row tile's
// own word rb by the exact symmetric test folded with ballots, every word
// after it by the table look-ups, words at or past the last valid one zeroed
// (and, with zero_from >= 0, the row's words [zero_from, row_words)).  The
// block's tables arrive by one bulk copy.  smem: kConeTableSmem bytes,
// 16-byte aligned.  All 256 threads.  Returns false (status recorded) if the
// copy did not complete in time.
__device__ __forceinline__ bool relate_block_tables(const int32_t* __restrict__ coords, int64_t n,
                                                    uint64_t* __restrict__ bits, int64_t row_words, int64_t rb,
                                                    int64_t w0, const ConeTable* __restrict__ tables, uint8_t* smem,
                                                    bool order2d, int64_t zero_from, WsHeader* hdr) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int kWarps = kRelThreads / 32;
    ConeTable* st = reinterpret_cast<ConeTable*>(smem);
    // u, v of the row tile's elements: the rows here, and the columns of the own word
    int32_t* own = reinterpret_cast<int32_t*>(smem + kRelWordsPerBlock * sizeof(ConeTable));
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + kRelWordsPerBlock * sizeof(ConeTable) + 128 * 4);
    const int64_t V = (n + 63) >> 6;
    const int64_t r0 = rb * 64, r1 = r0 + 64 < n ? r0 + 64 : n;
    const int64_t wt = w0 > rb ? w0 : rb + 1;                                      // first table word
    const int64_t we = w0 + kRelWordsPerBlock < V ? w0 + kRelWordsPerBlock : V;  // end of the valid words
    const int nt = wt < we ? int(we - wt) : 0;
    const bool has_own = rb >= w0;  // then rb == w0: chunks start at the diagonal word
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t bytes = uint32_t(nt) * uint32_t(sizeof(ConeTable));
        mbar_arrive_expect_tx(bar, bytes);
        if (bytes) bulk_load(st, tables + wt, bytes, bar);
    }
    if (threadIdx.x < 128) {
        const int64_t e = r0 + (threadIdx.x & 63);
        own[threadIdx.x] = e < n ? coords[(threadIdx.x >> 6) * n + e] : 0;
    }
    __syncthreads();
    if (has_own) {
        for (int64_t i = r0 + warp; i < r1; i += kWarps) {
            const int32_t ui = own[i - r0], vi = own[64 + (i - r0)];
            bool b[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int k = lane + 32 * h;
                const int64_t j = r0 + k;
                const int32_t du = own[k] - ui, dv = own[64 + k] - vi;
                b[h] = j < n && (order2d ? (j > i ? dv > 0 : (j < i && dv < 0))
                                         : ((du ^ dv) >= 0 && du != 0 && dv != 0));
            }
            const uint64_t d = (uint64_t(__ballot_sync(0xffffffffu, b[1])) << 32) | __ballot_sync(0xffffffffu, b[0]);
            if (lane == 0) bits[i * row_words + rb] = d;
        }
    }
    if (!mbar_wait_bounded(bar, 0, hdr)) {
        mbar_wait_bounded(bar, 0, hdr);  // the copy may still be writing: wait once more before leaving
        return false;
    }
    // lane l: word w0 + l of each of the warp's rows, 32 consecutive words per row and warp
    const int64_t w = w0 + lane;
    const bool tab = w >= wt && w < we;
    if (tab || (w >= V && w < row_words)) {
        const ConeTable& T = st[tab ? int(w - wt) : 0];
        int32_t su[7], sv[7];
#pragma unroll
        for (int m = 0; m < 7; ++m) {
            sv[m] = tab ? T.xs[1][8 * m + 7] : 0;
            su[m] = tab && !order2d ? T.xs[0][8 * m + 7] : 0;
        }
#pragma unroll 2
        for (int64_t i = r0 + warp; i < r1; i += kWarps) {
            uint64_t word = 0ull;
            if (tab) {
                word = cone_above(T.xs[1], T.above[1], sv, own[64 + (i - r0)]);
                if (!order2d) word &= cone_above(T.xs[0], T.above[0], su, own[i - r0]);
            }
            bits[i * row_words + w] = word;
        }
    }
    if (zero_from >= 0)
        for (int64_t i = r0 + warp; i < r1; i += kWarps)
            for (int64_t z = zero_from + lane; z < row_words; z += 32) bits[i * row_words + z] = 0ull;
    return true;
}

// ------------------------------------------------ the lower part by symmetry
//
// A 64 x 64 tile wholly below the diagonal (row tile A, word B < A) is the
// transpose of tile (B, A) above it.  mirror_block fills one super-tile of
// 512 output rows x 8 output words (8 x 8 tiles): the 512 source rows x 8
// source words land in shared memory with 64-byte reads, each warp
// transposes its output row tile's 8 tiles in registers (six butterfly
// stages, five of them across lanes) and writes its row tile's words
// below the diagonal back through shared memory, 64 contiguous bytes per
// output row off the diagonal super-tiles, four lanes to a row.
constexpr int kMirTiles = 8;                    // tiles per super-tile side
constexpr int kMirRows = 64 * kMirTiles;        // 512 source / output rows

// Transposes of bit tiles held one row per lane (bit c = column c).  Stage
// j of the recursive block swap exchanges, between lanes l and l ^ j, the
// j-bit groups that lie off the diagonal: the lane with (l & j) == 0 keeps
// its low groups and takes its partner's low groups into its high ones, the
// other keeps its high groups and takes its partner's high groups into its
// low ones.  Per lane constants make every stage lane-uniform: for j = 16
// and 8 a byte permute of the lane's word and its partner's; for j = 4, 2, 1
// each lane sends its word rotated toward its partner's positions (right by
// j, or by 32 - j, i.e. left by j) and masked to the groups the partner
// takes, and keeps (own & mask) | received.
struct Tr32 {
    uint32_t s16, s8;       // byte-permute selectors
    uint32_t r[3], m[3];    // rotations and kept masks for j = 4, 2, 1
};
__device__ __forceinline__ Tr32 tr32_consts(int lane) {
    Tr32 c;
    c.s16 = (lane & 16) ? 0x3276u : 0x5410u;  // high: partner's bytes 2,3 then own 2,3; low: own 0,1 then partner's 0,1
    c.s8 = (lane & 8) ? 0x3715u : 0x6240u;    // high: p1 v1 p3 v3; low: v0 p0 v2 p2
    const uint32_t mk[3] = {0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        const int j = 4 >> s;
        const bool high = (lane & j) != 0;
        c.r[s] = high ? uint32_t(32 - j) : uint32_t(j);
        c.m[s] = high ? ~mk[s] : mk[s];
    }
    return c;
}
__device__ __forceinline__ uint32_t transpose32(uint32_t v, const Tr32& c) {
    v = __byte_perm(v, __shfl_xor_sync(0xffffffffu, v, 16), c.s16);
    v = __byte_perm(v, __shfl_xor_sync(0xffffffffu, v, 8), c.s8);
#pragma unroll
    for (int s = 0; s < 3; ++s)
        v = (v & c.m[s]) | __shfl_xor_sync(0xffffffffu, __funnelshift_r(v, v, c.r[s]) & c.m[s], 4 >> s);
    return v;
}

// Transpose the 64 x 64 bit tile whose rows l and l + 32 lane l holds: the
// stage j = 32 inside the lane (x's high half with y's low half), then the
// four 32 x 32 quarters independently.
__device__ __forceinline__ void transpose64(uint64_t& x, uint64_t& y, const Tr32& c) {
    const uint64_t t = ((x >> 32) ^ y) & 0x00000000FFFFFFFFull;
    y ^= t;
    x ^= t << 32;
    x = uint64_t(transpose32(uint32_t(x), c)) | (uint64_t(transpose32(uint32_t(x >> 32), c)) << 32);
    y = uint64_t(transpose32(uint32_t(y), c)) | (uint64_t(transpose32(uint32_t(y >> 32), c)) << 32);
}

// Super-tile (A8, B8): output rows [512 A8, 512 A8 + 512), output words
// [8 B8, 8 B8 + 8).  sm: 512 x 9 words of shared memory.  All 256 threads.
__device__ __forceinline__ void mirror_block(uint64_t* __restrict__ bits, int64_t n, int64_t row_words, int64_t A8,
                                             int64_t B8, uint64_t (*sm)[kMirTiles + 1]) {
    const int64_t tiles = (n + 63) >> 6;  // row tiles = valid words
    const int64_t A0 = A8 * kMirTiles, B0 = B8 * kMirTiles;
    // anything to do here? (uniform: some tile with B < A < tiles)
    if (A0 >= tiles || B0 >= (A0 + kMirTiles - 1 < tiles ? A0 + kMirTiles - 1 : tiles - 1)) return;
    // source rows 64 B0 .. + 512, source words A0 .. A0 + 8, as 16-byte word
    // pairs (A0 is even and rows are 16-word multiples), every load of a
    // thread issued before the first shared-memory store: with one load in
    // flight per thread the kernel waited on memory latency at a quarter of
    // the HBM rate.  The second word of a pair at the last valid word is a
    // padding word of the row (loaded, then replaced by 0).
    constexpr int kPairs = kMirRows * kMirTiles / 2, kPerThread = kPairs / kRelThreads;
    static_assert(kPairs % kRelThreads == 0 && kMirTiles % 2 == 0, "word pairs split evenly over the block");
    ulonglong2 v[kPerThread];
#pragma unroll
    for (int s = 0; s < kPerThread; ++s) {
        const int t = threadIdx.x + s * kRelThreads;
        const int64_t row = 64 * B0 + t / (kMirTiles / 2), word = A0 + 2 * (t % (kMirTiles / 2));
        v[s] = (row < n && word < tiles) ? __ldg(reinterpret_cast<const ulonglong2*>(bits + row * row_words + word))
                                         : make_ulonglong2(0ull, 0ull);
    }
#pragma unroll
    for (int s = 0; s < kPerThread; ++s) {
        const int t = threadIdx.x + s * kRelThreads;
        const int r = t / (kMirTiles / 2), w = 2 * (t % (kMirTiles / 2));
        sm[r][w] = v[s].x;
        sm[r][w + 1] = A0 + w + 1 < tiles ? v[s].y : 0ull;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t A = A0 + warp;  // this warp's output row tile
    const bool active = A < tiles && B0 < A;  // warp-uniform
    uint64_t ox[kMirTiles], oy[kMirTiles];
    if (active) {
        const Tr32 tc = tr32_consts(lane);
#pragma unroll
        for (int qb = 0; qb < kMirTiles; ++qb) {
            uint64_t x = sm[64 * qb + lane][warp], y = sm[64 * qb + lane + 32][warp];
            transpose64(x, y, tc);
            ox[qb] = x;
            oy[qb] = y;
        }
    }
    __syncthreads();  // every warp has read its column of the source words
    if (active) {
        // The warp's 64 output rows go through its own 64 rows of shared
        // memory, then out with four lanes per row (16 bytes each): every
        // row's 64 bytes leave as two whole 32-byte sectors.  Words B0 + w
        // < A only (all inside the row: B < A < tiles).
        uint64_t (*out)[kMirTiles + 1] = sm + 64 * warp;
#pragma unroll
        for (int qb = 0; qb < kMirTiles; ++qb) {
            out[lane][qb] = ox[qb];
            out[lane + 32][qb] = oy[qb];
        }
        __syncwarp();
        const int w = 2 * (lane & 3);  // this lane's word pair
        static_assert(kMirTiles == 8, "four lanes cover a row's eight words");
#pragma unroll
        for (int s = 0; s < 8; ++s) {
            const int r = 8 * s + (lane >> 2);
            const int64_t row = 64 * A + r;
            if (row < n && B0 + w < A) {
                uint64_t* dst = bits + row * row_words + B0 + w;
                if (B0 + w + 1 < A)
                    *reinterpret_cast<ulonglong2*>(dst) = make_ulonglong2(out[r][w], out[r][w + 1]);
                else
                    *dst = out[r][w];
            }
        }
    }
}

}  // namespace cs
