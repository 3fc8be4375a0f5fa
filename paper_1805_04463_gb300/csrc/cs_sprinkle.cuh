// cs_sprinkle.cuh -- per-element draws of the sprinklers (Appendix "Causal Set
// Sprinklings"), shared by the single-set and batched sprinkle kernels.
#pragma once

#include "cs_internal.cuh"

namespace cs {

// Stream numbers of the generator specification.
constexpr uint32_t kStreamOrderU = 0, kStreamOrderV = 1, kStreamDiamond2 = 2, kStreamDiamond4 = 3,
                   kStreamDiamond3 = 4, kStreamDeSitter = 5, kStreamSquare = 6, kStreamCylinder = 7;

// de Sitter slab: eta is drawn in coarse cells -kDsCells .. kDsCells of
// 2 pi / 2^20 rad (eta_0 = 0.5 rad), then uniformly among the kDsSub fine
// units (2 pi / 2^32 rad) of the cell; theta is a uint32, a full turn 2^32.
constexpr int kDsCells = 83443;
constexpr int kDsTable = 2 * kDsCells + 1;
constexpr int kDsSub = 4096;

// Random 2D order: the two 64-bit keys whose ranks are u and v.
__device__ __forceinline__ void draw_2d_order(uint64_t su, uint64_t sv, int64_t e, uint64_t& ku, uint64_t& kv) {
    ku = draw_from(su, uint64_t(e), 0);
    kv = draw_from(sv, uint64_t(e), 0);
}

// 2D diamond: u, v on the 2^31 grid (grid-null pairs, du = 0 or dv = 0, are
// then negligible); sort key (u + v) in the top 32 bits.
__device__ __forceinline__ uint64_t draw_2d_diamond(uint64_t s, int64_t e, int32_t& u, int32_t& v) {
    const uint32_t uu = uint32_t(draw_from(s, uint64_t(e), 0) >> 33);
    const uint32_t vv = uint32_t(draw_from(s, uint64_t(e), 1) >> 33);
    u = int32_t(uu);
    v = int32_t(vv);
    return uint64_t(uu + vv) << 32;
}

// D-dimensional diamond of height 1 (D = 3: 2+1, D = 4: 3+1): rejection
// sampling in the box t in [0, 2^20), spatial coordinates in [-2^19, 2^19),
// accepting |x|^2 < min(t, 2^20-t)^2; attempt a uses slots D*a .. D*a+D-1.
// Sort key t in the top 20 bits.  Returns false if no attempt was accepted.
template <int D>
__device__ __forceinline__ bool draw_diamond(uint64_t s, int64_t e, int32_t (&c)[4], uint64_t& key) {
    const int64_t half = kGrid / 2;
    for (int a = 0; a < kMaxAttempts; ++a) {
        int64_t q[D];
#pragma unroll
        for (int k = 0; k < D; ++k) q[k] = int64_t(draw_from(s, uint64_t(e), uint32_t(D * a + k)) >> (64 - kGridBits));
        int64_t r2 = 0;
#pragma unroll
        for (int k = 1; k < D; ++k) {
            q[k] -= half;
            r2 += q[k] * q[k];
        }
        const int64_t t = q[0];
        const int64_t h = t < kGrid - t ? t : kGrid - t;
        if (r2 < h * h) {
#pragma unroll
            for (int k = 0; k < 4; ++k) c[k] = k < D ? int32_t(q[k < D ? k : 0]) : 0;
            key = uint64_t(t) << (64 - kGridBits);
            return true;
        }
    }
    c[0] = c[1] = c[2] = c[3] = 0;
    key = 0;
    return false;
}

__device__ __forceinline__ bool draw_4d_diamond(uint64_t s, int64_t e, int32_t (&c)[4], uint64_t& key) {
    return draw_diamond<4>(s, e, c, key);
}

__device__ __forceinline__ bool draw_3d_diamond(uint64_t s, int64_t e, int32_t (&c)[4], uint64_t& key) {
    return draw_diamond<3>(s, e, c, key);
}

// 1+1 de Sitter slab (spherical foliation, Eq. ds_metric): theta uniform on
// 2^32 fine units; the coarse eta cell is the inverse CDF of the sec^2 mass,
// found by a binary search of the 53-bit uniform U against the cumulative
// thresholds `thr` (thr[g + kDsCells] for cell g, the last one 2^53), and eta
// is uniform among the cell's fine units.  Sort key: eta + 2^31 in the top
// 32 bits.
__device__ __forceinline__ uint64_t draw_ds_slab(uint64_t s, int64_t e, const uint64_t* __restrict__ thr,
                                                 int32_t& eta, int32_t& theta) {
    theta = int32_t(uint32_t(draw_from(s, uint64_t(e), 0) >> 32));
    const uint64_t u = draw_from(s, uint64_t(e), 1) >> 11;
    int lo = 0, hi = kDsTable - 1;  // smallest index with u < thr[index]
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (u < thr[mid]) hi = mid; else lo = mid + 1;
    }
    const int32_t off = int32_t(draw_from(s, uint64_t(e), 2) >> 52);
    eta = (lo - kDsCells) * kDsSub - kDsSub / 2 + off;
    return uint64_t(uint32_t(eta) ^ 0x80000000u) << 32;
}

// 1+1 square t in [-1/2, 1/2), x in [-1/2, 1/2) on a grid of 2^30 per unit,
// stored in light-cone coordinates u = t + x + 2^30, v = t - x + 2^30 (both
// in [0, 2^31), so the diamond's light-cone test applies); sort key
// u + v = 2 t + 2^31 in the top 32 bits.
__device__ __forceinline__ uint64_t draw_2d_square(uint64_t s, int64_t e, int32_t& u, int32_t& v) {
    const int32_t t = int32_t(draw_from(s, uint64_t(e), 0) >> 34) - (1 << 29);
    const int32_t x = int32_t(draw_from(s, uint64_t(e), 1) >> 34) - (1 << 29);
    u = t + x + (1 << 30);
    v = t - x + (1 << 30);
    return uint64_t(uint32_t(u) + uint32_t(v)) << 32;
}

// 1+1 cylinder: theta uniform on 2^32 fine units (a full turn), t uniform on
// [-T, T) fine units with T = floor(2^31 / pi), one radian (t0 = 1), by a
// 32 x 32-bit multiply of a uniform word by 2T.  Sort key: t + 2^31 in the
// top 32 bits.
constexpr uint32_t kCylinderT = 683565275u;
__device__ __forceinline__ uint64_t draw_2d_cylinder(uint64_t s, int64_t e, int32_t& t, int32_t& theta) {
    theta = int32_t(uint32_t(draw_from(s, uint64_t(e), 0) >> 32));
    const uint64_t r = draw_from(s, uint64_t(e), 1) >> 32;
    t = int32_t(int64_t((r * uint64_t(2u * kCylinderT)) >> 32) - int64_t(kCylinderT));
    return uint64_t(uint32_t(t) ^ 0x80000000u) << 32;
}

}  // namespace cs
