/*
 * oracle.c -- CPU oracle for causal-set interval abundances and the
 * Benincasa-Dowker (BD) action.
 *
 * TEST INFRASTRUCTURE ONLY.  This is the plain, slow, obviously-correct
 * restatement of what the CUDA path computes.  Only the test suite, the
 * package smoke check and the benchmark's CPU-baseline / reference leg may
 * load it.  It shares no code, header, table or helper with the CUDA library
 * (paper_1805_04463_gb300/csrc) and the library never loads it.
 *
 * Source: W. J. Cunningham, "High Performance Algorithms for Quantum Gravity
 * and Cosmology" (arXiv:1805.04463).  Each function cites the section,
 * equation or algorithm it follows.  Where the thesis is silent (random
 * number generator, tie-breaking, grid quantisation) the generator
 * specification below is this project's own reading and is implemented
 * independently on both sides.
 *
 * Generator specification (shared *definition*, separate implementations):
 *   SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): state += 0x9E3779B97F4A7C15,
 *   output = mix(state) with the published two-multiply finaliser.  Output
 *   number n (0-based) of a generator started at state s is therefore
 *   mix(s + (n+1)*gamma).  A draw for (seed, stream, element e, slot q) is
 *   output (e*65536 + q) of the generator started at sigma, where sigma is
 *   output `stream` of the generator started at `seed`.  Grid value of a
 *   draw = draw >> 44 (20 bits, one unit of length = 2^20 grid steps).
 *
 * Parity pins live in tests/test_oracle_*.py; every function here is pinned
 * by at least one check that does not re-run this file's own formulae.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#if defined(__aarch64__)
typedef long double q128; /* binary128 on AArch64 Linux */
#elif defined(__x86_64__)
typedef __float128 q128;  /* binary128 via libgcc soft-float */
#else
#error "oracle needs a binary128 type"
#endif

#define OR_GAMMA 0x9E3779B97F4A7C15ULL
#define OR_GRID  (1LL << 20)
#define OR_HALF  (1LL << 19)
#define OR_MAX_ATTEMPTS 16384

enum { OR_2D_ORDER = 0, OR_2D_DIAMOND = 1, OR_4D_DIAMOND = 2, OR_3D_DIAMOND = 3, OR_2D_DS_SLAB = 4,
       OR_2D_SQUARE = 5, OR_2D_CYLINDER = 6 };

/* de Sitter slab: eta is drawn in coarse cells of 2 pi / 2^20 rad, the cells
 * -OR_DS_G .. OR_DS_G, i.e. |eta| <= (OR_DS_G + 1/2) coarse units, and
 * OR_DS_G = round(0.5 rad / coarse unit) sets eta_0 = 0.5.  Stored
 * coordinates use the fine unit 2 pi / 2^32 rad (OR_DS_SUB fine units per
 * coarse cell). */
#define OR_DS_G 83443
#define OR_DS_SUB 4096
enum { OR_OK = 0, OR_EINVAL = -1, OR_ENOMEM = -2, OR_ERANGE = -6 };

/* ------------------------------------------------------------------ PRNG */

static uint64_t or_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* SplitMix64 next(): advance then mix (Steele, Lea & Flood 2014). */
uint64_t oracle_splitmix64_next(uint64_t *state)
{
    *state += OR_GAMMA;
    return or_mix(*state);
}

/* Output number n of SplitMix64 started at state s: n+1 advances, then mix. */
static uint64_t or_output_at(uint64_t s, uint64_t n)
{
    uint64_t st = s;
    st += n * OR_GAMMA; /* n advances without output */
    return oracle_splitmix64_next(&st);
}

uint64_t oracle_draw(uint64_t seed, uint32_t stream, uint64_t elem, uint32_t slot)
{
    uint64_t sigma = or_output_at(seed, (uint64_t)stream);
    return or_output_at(sigma, elem * 65536ULL + (uint64_t)slot);
}

int oracle_dim(int kind)
{
    if (kind == OR_2D_ORDER || kind == OR_2D_DIAMOND || kind == OR_2D_DS_SLAB || kind == OR_2D_SQUARE ||
        kind == OR_2D_CYLINDER)
        return 2;
    if (kind == OR_3D_DIAMOND) return 3;
    if (kind == OR_4D_DIAMOND) return 4;
    return 0;
}

/* ------------------------------------------------------------ sprinkling */

typedef struct { int64_t key; int64_t idx; } or_pair;

static int or_cmp_pair(const void *a, const void *b)
{
    const or_pair *x = (const or_pair *)a, *y = (const or_pair *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->idx != y->idx) return x->idx < y->idx ? -1 : 1;
    return 0;
}

typedef struct { uint64_t key; int64_t idx; } or_upair;

static int or_cmp_upair(const void *a, const void *b)
{
    const or_upair *x = (const or_upair *)a, *y = (const or_upair *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->idx != y->idx) return x->idx < y->idx ? -1 : 1;
    return 0;
}

/*
 * Cumulative sec^2 mass of the de Sitter slab up to the end of eta cell g,
 * scaled to 2^53 (see kind 4 below).  The expression and its evaluation order
 * are part of the generator specification, so that any implementation using
 * the same libm tan reaches the same integers.
 */
uint64_t oracle_ds_threshold(int64_t g)
{
    double unit = 2.0 * M_PI / 1048576.0;
    double t0 = tan(((double)OR_DS_G + 0.5) * unit);
    double x = (tan(((double)g + 0.5) * unit) + t0) / (2.0 * t0);
    return (uint64_t)(x * 9007199254740992.0);
}

/*
 * Sprinkle n elements and write them, labelled in time order, as
 * structure-of-arrays int32 coordinates: coords[c*n + label].
 *
 * kind 0, random 2D order: u and v are two independent uniform random
 *   permutations (ranks of 64-bit keys from streams 0 and 1, ties broken by
 *   element index); elements are relabelled by u, so coords[0] = 0..n-1.
 *   A 2D order is the 1+1 Minkowski diamond in light-cone coordinates
 *   (Appendix "Causal Set Sprinklings", 1+1 Dimensional Diamond) with only
 *   the order of u and v kept.
 * kind 1, 2D diamond: u, v uniform on the grid [0, 2^31) (same appendix
 *   entry, u* = U u0 with u0 = 1; u, v = draw >> 33), time t = u + v.  The
 *   grid is fine enough that grid-null pairs (du = 0 or dv = 0, unrelated)
 *   are negligible: about N^2 / 2^31 of them, against N^2 / 2^20 on a 2^20
 *   grid, which at N = 2^17 would remove ~10^4 near-null links.
 * kind 2, 4D diamond of height 1: rejection sampling (allowed by the
 *   appendix's general method) in the box t in [0, 2^20),
 *   x, y, z in [-2^19, 2^19): accept iff x^2+y^2+z^2 < min(t, 2^20-t)^2.
 *   Attempt a of element e uses slots 4a..4a+3 of stream 3.
 * kind 3, 3D (2+1) diamond of height 1: the same rejection method in the box
 *   t in [0, 2^20), x, y in [-2^19, 2^19): accept iff
 *   x^2+y^2 < min(t, 2^20-t)^2 (Appendix "Causal Set Sprinklings", 2+1
 *   Dimensional Diamond, volume pi/(3 sqrt 2) u0^3 = pi/12 for height 1).
 *   Attempt a of element e uses slots 3a..3a+2 of stream 4.
 * kind 4, 1+1 de Sitter slab in the spherical foliation (Section "Spacetime
 *   Region Considered", Eq. ds_metric; Appendix "Causal Set Sprinklings", de
 *   Sitter 1+1 Dimensional Slab) with eta_0 = 0.5 and pseudo-radius 1:
 *   theta uniform, eta with density sec^2(eta) / (2 tan eta_0), both on the
 *   grid of 2 pi / 2^32 rad (the fine unit).  theta = draw(stream 5, slot 0)
 *   >> 32, a full turn being 2^32 (stored as the int32 bit pattern).  eta
 *   first picks a coarse cell of 4096 fine units by the inverse CDF of the
 *   cell masses: coarse cell g (|g| <= G = 83443) covers [(g - 1/2),
 *   (g + 1/2)] coarse units, and with t0 = tan((G + 1/2) coarse unit) the
 *   cumulative mass up to the end of cell g is
 *   x_g = (tan((g + 1/2) coarse unit) + t0) / (2 t0) (exactly 1 for g = G);
 *   g = the smallest cell with U < floor(x_g 2^53), U = draw(stream 5,
 *   slot 1) >> 11.  Within the cell eta is uniform on the fine grid:
 *   eta = 4096 g - 2048 + (draw(stream 5, slot 2) >> 52).  (sec^2 varies by
 *   less than 1e-5 across one cell.)  Coordinates: coords[0] = eta,
 *   coords[1] = theta, both in fine units.
 * kind 5, 1+1 square (Appendix "Causal Set Sprinklings", 1+1 Dimensional
 *   Square) with t0 = x0 = 1/2: t and x uniform on the grid of 2^30 per unit
 *   length, t = (draw(stream 6, slot 0) >> 34) - 2^29 and
 *   x = (draw(stream 6, slot 1) >> 34) - 2^29, stored in light-cone
 *   coordinates shifted to be non-negative: coords[0] = u = t + x + 2^30,
 *   coords[1] = v = t - x + 2^30 (so ds^2 = -du dv).  Time t.
 * kind 6, 1+1 cylinder (same appendix, 1+1 Dimensional Cylinder) with
 *   t0 = 1 and a circle of circumference 2 pi: theta uniform, a full turn
 *   being 2^32 fine units, theta = draw(stream 7, slot 0) >> 32 (stored as
 *   the int32 bit pattern); t uniform on [-T, T) in the same units,
 *   T = floor(2^31 / pi) = 683565275 (one radian, so t0 = 1),
 *   t = ((draw(stream 7, slot 1) >> 32) * 2T >> 32) - T.  Coordinates:
 *   coords[0] = t, coords[1] = theta.
 * Elements are sorted by time with ties broken by generation index
 * (Section "Pairwise Relations": elements are sorted by their time
 * coordinate before relations are identified).
 */
int oracle_sprinkle(int kind, int64_t n, uint64_t seed, int32_t *coords)
{
    if (n < 0 || !coords) return OR_EINVAL;
    if (n == 0) return OR_OK;
    if (kind == OR_2D_ORDER) {
        or_upair *ku = malloc((size_t)n * sizeof *ku);
        or_upair *kv = malloc((size_t)n * sizeof *kv);
        int64_t *vrank = malloc((size_t)n * sizeof *vrank);
        if (!ku || !kv || !vrank) { free(ku); free(kv); free(vrank); return OR_ENOMEM; }
        for (int64_t e = 0; e < n; e++) {
            ku[e].key = oracle_draw(seed, 0, (uint64_t)e, 0); ku[e].idx = e;
            kv[e].key = oracle_draw(seed, 1, (uint64_t)e, 0); kv[e].idx = e;
        }
        qsort(ku, (size_t)n, sizeof *ku, or_cmp_upair);
        qsort(kv, (size_t)n, sizeof *kv, or_cmp_upair);
        for (int64_t r = 0; r < n; r++) vrank[kv[r].idx] = r;
        for (int64_t r = 0; r < n; r++) {
            coords[r] = (int32_t)r;
            coords[n + r] = (int32_t)vrank[ku[r].idx];
        }
        free(ku); free(kv); free(vrank);
        return OR_OK;
    }
    if (kind == OR_2D_DIAMOND) {
        int32_t *u = malloc((size_t)n * 4), *v = malloc((size_t)n * 4);
        or_pair *t = malloc((size_t)n * sizeof *t);
        if (!u || !v || !t) { free(u); free(v); free(t); return OR_ENOMEM; }
        for (int64_t e = 0; e < n; e++) {
            u[e] = (int32_t)(oracle_draw(seed, 2, (uint64_t)e, 0) >> 33);
            v[e] = (int32_t)(oracle_draw(seed, 2, (uint64_t)e, 1) >> 33);
            t[e].key = (int64_t)u[e] + v[e];
            t[e].idx = e;
        }
        qsort(t, (size_t)n, sizeof *t, or_cmp_pair);
        for (int64_t r = 0; r < n; r++) {
            coords[r] = u[t[r].idx];
            coords[n + r] = v[t[r].idx];
        }
        free(u); free(v); free(t);
        return OR_OK;
    }
    if (kind == OR_2D_DS_SLAB) {
        int32_t *eta = malloc((size_t)n * 4), *th = malloc((size_t)n * 4);
        or_pair *t = malloc((size_t)n * sizeof *t);
        if (!eta || !th || !t) { free(eta); free(th); free(t); return OR_ENOMEM; }
        for (int64_t e = 0; e < n; e++) {
            th[e] = (int32_t)(uint32_t)(oracle_draw(seed, 5, (uint64_t)e, 0) >> 32);
            uint64_t u = oracle_draw(seed, 5, (uint64_t)e, 1) >> 11;
            int64_t lo = -OR_DS_G, hi = OR_DS_G; /* answer in [lo, hi] */
            while (lo < hi) {
                int64_t mid = lo + (hi - lo) / 2;
                if (u < oracle_ds_threshold(mid)) hi = mid; else lo = mid + 1;
            }
            int64_t off = (int64_t)(oracle_draw(seed, 5, (uint64_t)e, 2) >> 52);
            eta[e] = (int32_t)(lo * OR_DS_SUB - OR_DS_SUB / 2 + off);
            t[e].key = eta[e];
            t[e].idx = e;
        }
        qsort(t, (size_t)n, sizeof *t, or_cmp_pair);
        for (int64_t r = 0; r < n; r++) {
            coords[r] = eta[t[r].idx];
            coords[n + r] = th[t[r].idx];
        }
        free(eta); free(th); free(t);
        return OR_OK;
    }
    if (kind == OR_2D_SQUARE || kind == OR_2D_CYLINDER) {
        int32_t *c0 = malloc((size_t)n * 4), *c1 = malloc((size_t)n * 4);
        or_pair *t = malloc((size_t)n * sizeof *t);
        if (!c0 || !c1 || !t) { free(c0); free(c1); free(t); return OR_ENOMEM; }
        for (int64_t e = 0; e < n; e++) {
            if (kind == OR_2D_SQUARE) {
                int64_t tt = (int64_t)(oracle_draw(seed, 6, (uint64_t)e, 0) >> 34) - (1LL << 29);
                int64_t xx = (int64_t)(oracle_draw(seed, 6, (uint64_t)e, 1) >> 34) - (1LL << 29);
                c0[e] = (int32_t)(tt + xx + (1LL << 30));
                c1[e] = (int32_t)(tt - xx + (1LL << 30));
                t[e].key = tt;
            } else {
                const uint64_t T = 683565275ULL;
                c1[e] = (int32_t)(uint32_t)(oracle_draw(seed, 7, (uint64_t)e, 0) >> 32);
                uint64_t r = oracle_draw(seed, 7, (uint64_t)e, 1) >> 32;
                c0[e] = (int32_t)((int64_t)((r * (2 * T)) >> 32) - (int64_t)T);
                t[e].key = c0[e];
            }
            t[e].idx = e;
        }
        qsort(t, (size_t)n, sizeof *t, or_cmp_pair);
        for (int64_t r = 0; r < n; r++) {
            coords[r] = c0[t[r].idx];
            coords[n + r] = c1[t[r].idx];
        }
        free(c0); free(c1); free(t);
        return OR_OK;
    }
    if (kind == OR_4D_DIAMOND || kind == OR_3D_DIAMOND) {
        const int d = oracle_dim(kind);
        const uint32_t stream = kind == OR_4D_DIAMOND ? 3 : 4;
        int32_t *x = malloc((size_t)n * (size_t)d * sizeof *x);
        or_pair *t = malloc((size_t)n * sizeof *t);
        if (!x || !t) { free(x); free(t); return OR_ENOMEM; }
        int bad = 0;
        for (int64_t e = 0; e < n && !bad; e++) {
            int found = 0;
            for (int a = 0; a < OR_MAX_ATTEMPTS && !found; a++) {
                int64_t c[4] = {0, 0, 0, 0}, r2 = 0;
                for (int q = 0; q < d; q++)
                    c[q] = (int64_t)(oracle_draw(seed, stream, (uint64_t)e, (uint32_t)(d * a + q)) >> 44);
                int64_t tt = c[0];
                for (int q = 1; q < d; q++) {
                    c[q] -= OR_HALF;
                    r2 += c[q] * c[q];
                }
                int64_t h = tt < OR_GRID - tt ? tt : OR_GRID - tt;
                if (r2 < h * h) {
                    for (int q = 0; q < d; q++) x[(int64_t)d * e + q] = (int32_t)c[q];
                    found = 1;
                }
            }
            if (!found) bad = 1;
            t[e].key = x[(int64_t)d * e];
            t[e].idx = e;
        }
        if (bad) { free(x); free(t); return OR_ERANGE; }
        qsort(t, (size_t)n, sizeof *t, or_cmp_pair);
        for (int64_t r = 0; r < n; r++)
            for (int q = 0; q < d; q++) coords[(int64_t)q * n + r] = x[(int64_t)d * t[r].idx + q];
        free(x); free(t);
        return OR_OK;
    }
    return OR_EINVAL;
}

/* --------------------------------------------------------------- relation */

/*
 * a precedes b: timelike (Delta s^2 < 0, strictly) and future-directed
 * (Section "Lorentzian Geometry"; the 1+1 diamond interval is ds^2 = -2 du dv).
 */
int oracle_precedes(int kind, int64_t n, const int32_t *coords, int64_t a, int64_t b)
{
    if (kind == OR_2D_DS_SLAB || kind == OR_2D_CYLINDER) {
        /* timelike iff the angular separation on the circle is below the
         * (conformal-)time separation: pi - |pi - |dtheta|| < |deta|, with a
         * full turn of 2^32 fine units */
        int64_t deta = (int64_t)coords[b] - coords[a];
        int64_t ta = (int64_t)(uint32_t)coords[n + a], tb = (int64_t)(uint32_t)coords[n + b];
        int64_t dth = tb > ta ? tb - ta : ta - tb;
        int64_t circ = dth < (1LL << 32) - dth ? dth : (1LL << 32) - dth;
        return deta > 0 && circ < deta;
    }
    if (kind == OR_2D_SQUARE) {
        /* dt > |dx| with 2 dt = du + dv and 2 dx = du - dv */
        int64_t du = (int64_t)coords[b] - coords[a];
        int64_t dv = (int64_t)coords[n + b] - coords[n + a];
        int64_t dt2 = du + dv, dx2 = du - dv;
        return dt2 > 0 && dt2 > (dx2 < 0 ? -dx2 : dx2);
    }
    if (kind == OR_2D_ORDER || kind == OR_2D_DIAMOND) {
        int64_t du = (int64_t)coords[b] - coords[a];
        int64_t dv = (int64_t)coords[n + b] - coords[n + a];
        return du > 0 && dv > 0;
    }
    int d = oracle_dim(kind);
    int64_t dt = (int64_t)coords[b] - coords[a], r2 = 0;
    for (int q = 1; q < d; q++) {
        int64_t dx = (int64_t)coords[q * n + b] - coords[q * n + a];
        r2 += dx * dx;
    }
    return dt > 0 && dt * dt - r2 > 0;
}

/* Row words of the bitset: ceil(n/64) rounded up to a multiple of 16. */
int64_t oracle_row_words(int64_t n)
{
    int64_t w = (n + 63) / 64;
    return (w + 15) / 16 * 16;
}

/*
 * Symmetrised causal matrix P + P^T as one bitset per row (Section "Data
 * Structures for Totally Ordered Sets"): bit j of row i is 1 iff i and j
 * are related either way.  Column j lives in word j/64, bit j%64.  All
 * padding bits and words are zero.
 */
int oracle_causal_matrix(int kind, int64_t n, const int32_t *coords, uint64_t *bits, int64_t row_words)
{
    if (n < 0 || row_words * 64 < n) return OR_EINVAL;
    memset(bits, 0, (size_t)n * (size_t)row_words * 8);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; i++) {
        uint64_t *row = bits + i * row_words;
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            if (oracle_precedes(kind, n, coords, i, j) || oracle_precedes(kind, n, coords, j, i))
                row[j >> 6] |= 1ULL << (j & 63);
        }
    }
    return OR_OK;
}

/* ------------------------------------------------------ interval counting */

static int or_bit(const uint64_t *row, int64_t j)
{
    return (int)((row[j >> 6] >> (j & 63)) & 1ULL);
}

/*
 * popcount(x & y) restricted to bit columns [lo, hi): the partial inner
 * product of two bitsets (Algorithms "Vectorized Partial Intersection" and
 * "Vectorized Inner Product", restated with a portable popcount).
 */
static int64_t or_partial_inner_product(const uint64_t *x, const uint64_t *y, int64_t lo, int64_t hi)
{
    if (hi <= lo) return 0;
    int64_t wlo = lo >> 6, whi = (hi - 1) >> 6, c = 0;
    for (int64_t w = wlo; w <= whi; w++) {
        uint64_t m = ~0ULL;
        if (w == wlo) m &= ~0ULL << (lo & 63);
        if (w == whi) m &= ~0ULL >> (63 - ((hi - 1) & 63));
        c += __builtin_popcountll(x[w] & y[w] & m);
    }
    return c;
}

/*
 * |A_ij| for one pair i < j, or -1 if i does not precede j.  For time-sorted
 * labels the elements between i and j in the order lie in columns i+1..j-1,
 * where row i holds the future of i and row j the past of j (Figure
 * "Proper distance and the order intervals"; Section "Partially Ordered Sets").
 */
int64_t oracle_interval_size(int64_t n, const uint64_t *bits, int64_t row_words, int64_t i, int64_t j)
{
    if (i < 0 || j >= n || i >= j) return -1;
    const uint64_t *ri = bits + i * row_words, *rj = bits + j * row_words;
    if (!or_bit(ri, j)) return -1;
    return or_partial_inner_product(ri, rj, i + 1, j);
}

/*
 * Interval abundances from the bitset (Algorithm "Optimized Interval
 * Abundance Measurement"): for every related pair i < j the partial inner
 * product of rows i and j gives m = |A_ij|; each thread keeps its own
 * abundance array and the arrays are summed at the end (Section "Parallel
 * Action Algorithm").  hist[k] counts pairs with |A_ij| = k, i.e. hist[k] is
 * the thesis's n_{k+1}; hist has len = max(n-1, 1) entries.
 *
 * Only rows i = row_begin, row_begin + row_step, ... < row_end are visited
 * (all rows: 0, n, 1), which lets a caller evaluate a bounded sample.
 * threads <= 0 uses the OpenMP default.  Returns the number of threads used.
 */
int oracle_interval_abundance_rows(int64_t n, const uint64_t *bits, int64_t row_words,
                                   int64_t row_begin, int64_t row_end, int64_t row_step,
                                   int64_t *hist, int64_t len, int threads)
{
    if (n < 0 || len < (n > 1 ? n - 1 : 1) || row_step < 1) return OR_EINVAL;
    memset(hist, 0, (size_t)len * 8);
    if (n < 2) return 1;
    int T = 1;
#ifdef _OPENMP
    T = threads > 0 ? threads : omp_get_max_threads();
#endif
    int64_t *local = calloc((size_t)T * (size_t)len, 8);
    if (!local) return OR_ENOMEM;
    if (row_end > n) row_end = n;
#pragma omp parallel for schedule(dynamic, 1) num_threads(T)
    for (int64_t i = row_begin; i < row_end; i += row_step) {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        int64_t *h = local + (int64_t)t * len;
        const uint64_t *ri = bits + i * row_words;
        for (int64_t j = i + 1; j < n; j++) {
            if (!or_bit(ri, j)) continue;
            int64_t m = or_partial_inner_product(ri, bits + j * row_words, i + 1, j);
            h[m]++;
        }
    }
    for (int t = 0; t < T; t++)
        for (int64_t k = 0; k < len; k++) hist[k] += local[(int64_t)t * len + k];
    free(local);
    return T;
}

int oracle_interval_abundance(int64_t n, const uint64_t *bits, int64_t row_words,
                              int64_t *hist, int64_t len, int threads)
{
    return oracle_interval_abundance_rows(n, bits, row_words, 0, n, 1, hist, len, threads);
}

/*
 * Brute force (Algorithm "Naive Interval Abundance Measurement"), with the
 * relation evaluated from the coordinates instead of a stored matrix: for
 * every related pair count the k with i < k < j, i precedes k and k precedes j.
 * O(n^3); meant for n <= a few hundred.
 */
int oracle_interval_abundance_naive(int kind, int64_t n, const int32_t *coords, int64_t *hist, int64_t len)
{
    if (n < 0 || len < (n > 1 ? n - 1 : 1)) return OR_EINVAL;
    memset(hist, 0, (size_t)len * 8);
    for (int64_t i = 0; i + 1 < n; i++)
        for (int64_t j = i + 1; j < n; j++) {
            if (!oracle_precedes(kind, n, coords, i, j)) continue;
            int64_t x = 0;
            for (int64_t k = i + 1; k < j; k++)
                if (oracle_precedes(kind, n, coords, i, k) && oracle_precedes(kind, n, coords, k, j)) x++;
            hist[x]++;
        }
    return OR_OK;
}

/*
 * 2D orders only, a structurally different count: with labels sorted by u,
 * |A_ij| = #{i < k < j : v_i < v_k < v_j}.  For each i a Fenwick tree over v
 * holds the v_k (k > i, v_k > v_i) seen so far; a prefix query gives the
 * count for each later j.  O(n^2 log n), no bitsets.  Rows are sampled as in
 * oracle_interval_abundance_rows.
 */
int oracle_interval_abundance_dominance2d(int64_t n, const int32_t *v, int64_t row_begin, int64_t row_end,
                                          int64_t row_step, int64_t *hist, int64_t len)
{
    if (n < 0 || len < (n > 1 ? n - 1 : 1) || row_step < 1) return OR_EINVAL;
    memset(hist, 0, (size_t)len * 8);
    if (row_end > n) row_end = n;
    int T = 1;
#ifdef _OPENMP
    T = omp_get_max_threads();
#endif
    int64_t *local = calloc((size_t)T * (size_t)len, 8);
    int32_t *fen = calloc((size_t)T * (size_t)(n + 1), 4);
    if (!local || !fen) { free(local); free(fen); return OR_ENOMEM; }
#pragma omp parallel for schedule(dynamic, 1) num_threads(T)
    for (int64_t i = row_begin; i < row_end; i += row_step) {
        int t = 0;
#ifdef _OPENMP
        t = omp_get_thread_num();
#endif
        int32_t *f = fen + (int64_t)t * (n + 1);
        memset(f, 0, (size_t)(n + 1) * 4);
        for (int64_t j = i + 1; j < n; j++) {
            if (v[j] <= v[i]) continue;
            int64_t c = 0; /* number of inserted values < v[j] */
            for (int64_t p = v[j]; p > 0; p -= p & -p) c += f[p];
            local[(int64_t)t * len + c]++;
            for (int64_t p = (int64_t)v[j] + 1; p <= n; p += p & -p) f[p]++;
        }
    }
    for (int t = 0; t < T; t++)
        for (int64_t k = 0; k < len; k++) hist[k] += local[(int64_t)t * len + k];
    free(local); free(fen);
    return OR_OK;
}

/*
 * 2D orders only: number of links (covering pairs, the transitive
 * reduction).  j > i is a link from i iff v_j > v_i and v_j is below every
 * v_k (i < k < j) that is above v_i: a running minimum, O(n^2), using
 * neither bitsets nor interval counts.
 */
int64_t oracle_links_2d(int64_t n, const int32_t *v)
{
    int64_t links = 0;
#pragma omp parallel for reduction(+ : links) schedule(dynamic, 16)
    for (int64_t i = 0; i < n; i++) {
        int64_t lo = INT64_MAX; /* min v_k above v_i seen so far */
        for (int64_t j = i + 1; j < n; j++) {
            if (v[j] <= v[i]) continue;
            if (v[j] < lo) { links++; lo = v[j]; }
        }
    }
    return links;
}

/* ----------------------------------------------------------------- action */

static q128 or_qsqrt(q128 x)
{
    if (x <= 0) return 0;
    q128 y = (q128)__builtin_sqrt((double)x);
    for (int it = 0; it < 3; it++) y = y - (y * y - x) / (2 * y);
    return y;
}

/*
 * Benincasa-Dowker action from the abundances (Section "The Benincasa-Dowker
 * Action").  With hist[k] = n_{k+1}:
 *   local 1+1 (Eq. s2d_local):  S = 2 (N - 2 n1 + 4 n2 - 2 n3)
 *   local 2+1 (Eq. s3d_local):  S = c3 (N - n1 + 27/8 n2 - 9/4 n3),
 *                               c3 = (pi/(3 sqrt 2))^(2/3) / Gamma(5/3), l/l_p = 1
 *   local 3+1 (Eq. s4d_local):  S = 4/sqrt(6) (N - n1 + 9 n2 - 16 n3 + 8 n4),
 *                               with (l/l_p)^2 = 1
 *   smeared 1+1 (Eq. s2d_smeared): S = 2 eps [N - 2 eps sum_m n_m f2(m-1, eps)]
 *   smeared 2+1:                   S = c3 eps^(2/3) [N - eps sum_m n_m f3(m-1, eps)]
 *   smeared 3+1 (Eq. s4d_smeared): S = 4 sqrt(eps/6) [N - eps sum_m n_m f4(m-1, eps)]
 * with f2, f3 and f4 evaluated as printed (divisions by 1-eps) in binary128
 * and (1-eps)^m built by repeated multiplication.  eps <= 0 or eps == 1
 * selects the local action.  bracket receives the exact integer in
 * parentheses of the local form (2+1: eight times it, 8N - 8n1 + 27n2 - 18n3,
 * so that it stays an integer).  out receives S rounded to double.  The 2+1
 * constant c3 and eps^(2/3) come from libm in double (relative error near
 * 1e-16, a constant factor on an otherwise binary128 result).
 */
int oracle_action(int dim, int64_t n, const int64_t *hist, int64_t len, double eps, double *out,
                  int64_t *bracket)
{
    if ((dim < 2 || dim > 4) || n < 0 || len < 0 || eps > 1.0 || eps != eps) return OR_EINVAL;
    int64_t h[4] = {0, 0, 0, 0};
    for (int k = 0; k < 4 && k < len; k++) h[k] = hist[k];
    int64_t b = dim == 2 ? n - 2 * h[0] + 4 * h[1] - 2 * h[2]
              : dim == 3 ? 8 * n - 8 * h[0] + 27 * h[1] - 18 * h[2]
                         : n - h[0] + 9 * h[1] - 16 * h[2] + 8 * h[3];
    if (bracket) *bracket = b;
    q128 c3 = (q128)(pow(M_PI / (3.0 * sqrt(2.0)), 2.0 / 3.0) / tgamma(5.0 / 3.0));
    if (eps <= 0.0 || eps == 1.0) {
        q128 s = dim == 2 ? (q128)2 * (q128)b
               : dim == 3 ? c3 * (q128)b / 8
                          : (q128)4 / or_qsqrt((q128)6) * (q128)b;
        if (out) *out = (double)s;
        return OR_OK;
    }
    q128 e = (q128)eps, one_m = (q128)1 - e, p = 1, sum = 0;
    for (int64_t k = 0; k < len; k++) { /* k = m - 1 */
        q128 m = (q128)k, f;
        if (dim == 2) {
            f = p * ((q128)1 - 2 * m * e / one_m + m * (m - 1) * e * e / (2 * one_m * one_m));
        } else if (dim == 3) {
            f = p * ((q128)1 - 27 * m * e / (8 * one_m) + 9 * m * (m - 1) * e * e / (8 * one_m * one_m));
        } else {
            f = p * ((q128)1 - 9 * m * e / one_m + 8 * m * (m - 1) * e * e / (one_m * one_m)
                     - 4 * m * (m - 1) * (m - 2) * e * e * e / (3 * one_m * one_m * one_m));
        }
        sum += (q128)hist[k] * f;
        p *= one_m;
    }
    q128 s = dim == 2 ? 2 * e * ((q128)n - 2 * e * sum)
           : dim == 3 ? c3 * (q128)pow(eps, 2.0 / 3.0) * ((q128)n - e * sum)
                      : 4 * or_qsqrt(e / 6) * ((q128)n - e * sum);
    if (out) *out = (double)s;
    return OR_OK;
}

/* --------------------------------------------- degrees and sparse lists */

/*
 * In- and out-degree vectors (Section "Optimized GPU Linking Algorithm",
 * Algorithm "Write Operations for Degrees"): with time-sorted labels,
 * kin[j] = #{i < j : i precedes j} (past relations of j) and
 * kout[i] = #{j > i : i precedes j} (future relations of i), read bit by
 * bit from the symmetric bitset.
 */
int oracle_degrees(int64_t n, const uint64_t *bits, int64_t row_words, int32_t *kin, int32_t *kout)
{
    if (n < 0 || !bits || !kin || !kout) return OR_EINVAL;
    for (int64_t i = 0; i < n; i++) {
        int64_t past = 0, future = 0;
        const uint64_t *row = bits + i * row_words;
        for (int64_t j = 0; j < n; j++) {
            if (!or_bit(row, j)) continue;
            if (j < i) past++; else if (j > i) future++;
        }
        kin[i] = (int32_t)past;
        kout[i] = (int32_t)future;
    }
    return OR_OK;
}

/*
 * The past (direction 0) or future (direction 1) sparse relation lists in
 * compressed-row form (Section "GPU Linking Algorithm": the relation list is
 * decoded into past and future sparse lists): row i owns
 * cols[offsets[i] .. offsets[i+1]), the labels related to i before
 * (direction 0) or after (direction 1) it, in increasing order.  offsets
 * has n+1 entries; cols may be NULL to get the offsets alone.  cols_capacity
 * is the room in cols; returns OR_ENOMEM if the lists do not fit.
 */
int oracle_sparse_relations(int64_t n, const uint64_t *bits, int64_t row_words, int direction, int64_t *offsets,
                            int32_t *cols, int64_t cols_capacity)
{
    if (n < 0 || !bits || !offsets || (direction != 0 && direction != 1)) return OR_EINVAL;
    int64_t pos = 0;
    for (int64_t i = 0; i < n; i++) {
        offsets[i] = pos;
        const uint64_t *row = bits + i * row_words;
        int64_t lo = direction ? i + 1 : 0, hi = direction ? n : i;
        for (int64_t j = lo; j < hi; j++) {
            if (!or_bit(row, j)) continue;
            if (cols) {
                if (pos >= cols_capacity) return OR_ENOMEM;
                cols[pos] = (int32_t)j;
            }
            pos++;
        }
    }
    offsets[n] = pos;
    return OR_OK;
}

/* ------------------------------------------------- chains and antichains */

/*
 * Longest chain (Section "Set Partitions", Algorithm "Maximal Chain
 * Length"), written as its definition: with time-sorted labels the longest
 * path from i to k, in relations, is d(k) = 1 + max d(m) over m in
 * {i} + A_ij preceding k (d(i) = 0), filled in label order.  Returns d(j)
 * for a related pair i < j and -1 if i does not precede j.  With i = j = -1
 * returns the height of the whole set: the number of elements of its longest
 * chain (0 for n = 0).
 */
int64_t oracle_longest_chain(int64_t n, const uint64_t *bits, int64_t row_words, int64_t i, int64_t j)
{
    if (n < 0 || !bits) return -2;
    int64_t *d = malloc((size_t)(n > 0 ? n : 1) * sizeof *d);
    if (!d) return -2;
    int64_t best = 0;
    if (i < 0 && j < 0) {
        for (int64_t k = 0; k < n; k++) {
            int64_t dk = 1;
            for (int64_t m = 0; m < k; m++)
                if (or_bit(bits + k * row_words, m) && d[m] + 1 > dk) dk = d[m] + 1;
            d[k] = dk;
            if (dk > best) best = dk;
        }
        free(d);
        return best;
    }
    if (i < 0 || j <= i || j >= n || !or_bit(bits + i * row_words, j)) {
        free(d);
        return -1;
    }
    const uint64_t *ri = bits + i * row_words, *rj = bits + j * row_words;
    d[i] = 0;
    for (int64_t k = i + 1; k <= j; k++) {
        d[k] = -1;
        if (k < j && !(or_bit(ri, k) && or_bit(rj, k))) continue; /* k not in A_ij */
        int64_t dk = 1;                                          /* from i directly */
        for (int64_t m = i + 1; m < k; m++)
            if (d[m] >= 0 && or_bit(bits + k * row_words, m) && d[m] + 1 > dk) dk = d[m] + 1;
        d[k] = dk;
    }
    best = d[j];
    free(d);
    return best;
}

/*
 * Greedy maximal antichain (Section "Set Partitions", Algorithm "Maximal
 * Antichain"): candidates X = the elements unrelated to the seed, the
 * antichain A = X + {seed}; while X is not empty, take the candidate k that
 * leaves the most elements in A when its relations J(k) are removed
 * (c = |A - J(k)|, the first such k in label order on ties), then remove
 * J(k) from A and J(k) + {k} from X.  out (row_words words) receives A as a
 * bitset; returns |A|, or -1 for a bad seed.
 */
int64_t oracle_greedy_antichain(int64_t n, const uint64_t *bits, int64_t row_words, int64_t seed, uint64_t *out)
{
    if (n < 1 || !bits || !out || seed < 0 || seed >= n) return -1;
    uint64_t *X = calloc((size_t)row_words, 8);
    if (!X) return -2;
    const uint64_t *rs = bits + seed * row_words;
    memset(out, 0, (size_t)row_words * 8);
    for (int64_t k = 0; k < n; k++)
        if (k != seed && !or_bit(rs, k)) X[k >> 6] |= 1ULL << (k & 63);
    for (int64_t w = 0; w < row_words; w++) out[w] = X[w];
    out[seed >> 6] |= 1ULL << (seed & 63);
    for (;;) {
        int64_t bestk = -1, bestc = -1;
        for (int64_t k = 0; k < n; k++) {
            if (!((X[k >> 6] >> (k & 63)) & 1ULL)) continue;
            const uint64_t *rk = bits + k * row_words;
            int64_t c = 0;
            for (int64_t w = 0; w < row_words; w++) c += __builtin_popcountll(out[w] & ~rk[w]);
            if (c > bestc) { bestc = c; bestk = k; }
        }
        if (bestk < 0) break;
        const uint64_t *rk = bits + bestk * row_words;
        for (int64_t w = 0; w < row_words; w++) {
            out[w] &= ~rk[w];
            X[w] &= ~rk[w];
        }
        X[bestk >> 6] &= ~(1ULL << (bestk & 63));
    }
    int64_t size = 0;
    for (int64_t w = 0; w < row_words; w++) size += __builtin_popcountll(out[w]);
    free(X);
    return size;
}

/* ------------------------------------------------- discrete d'Alembertian */

/*
 * Layer sums of the discrete d'Alembertian (Section "The Benincasa-Dowker
 * Action", Eqs. b2d_local, b4d_local): for every element j and m = 0..kmax,
 * out[m*n + j] = sum of phi(i) over the elements i preceding j with
 * |A_ij| = m, i.e. over the inclusive order interval L_{m+1}(j) (Eq. IOIs).
 * phi == NULL means phi = 1.  Sums are carried in binary128.
 */
int oracle_layer_sums(int64_t n, const uint64_t *bits, int64_t row_words, const double *phi, int kmax,
                      double *out)
{
    if (n < 0 || kmax < 0 || !out) return OR_EINVAL;
    q128 *acc = calloc((size_t)(kmax + 1) * (size_t)(n > 0 ? n : 1), sizeof *acc);
    if (!acc) return OR_ENOMEM;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t j = 0; j < n; j++) {
        const uint64_t *rj = bits + j * row_words;
        for (int64_t i = 0; i < j; i++) {
            if (!or_bit(rj, i)) continue; /* i precedes j (time order) */
            int64_t m = or_partial_inner_product(bits + i * row_words, rj, i + 1, j);
            if (m <= kmax) acc[m * n + j] += phi ? (q128)phi[i] : (q128)1;
        }
    }
    for (int64_t k = 0; k < (int64_t)(kmax + 1) * n; k++) out[k] = (double)acc[k];
    free(acc);
    return OR_OK;
}

/*
 * B phi(j) from the layer sums S_m(j) (m = |A_ij|), Eqs. b2d_local,
 * b3d_local and b4d_local with discreteness scale ell:
 *   1+1: (2/ell^2) [-phi(j) + 2 (S_0 - 2 S_1 + S_2)]
 *   2+1: (c3/ell^2) [-phi(j) + S_0 - 27/8 S_1 + 9/4 S_2],
 *        c3 = (pi/(3 sqrt 2))^(2/3) / Gamma(5/3)
 *   3+1: (4/(ell^2 sqrt 6)) [-phi(j) + S_0 - 9 S_1 + 16 S_2 - 8 S_3]
 * layers holds kmax+1 >= 3 (1+1, 2+1) or >= 4 (3+1) rows of n values;
 * phi == NULL means phi = 1.
 */
int oracle_dalembertian(int dim, int64_t n, const double *phi, const double *layers, int kmax, double ell,
                        double *out)
{
    if ((dim < 2 || dim > 4) || n < 0 || !layers || !out || !(ell > 0)) return OR_EINVAL;
    if (kmax < (dim == 4 ? 3 : 2)) return OR_EINVAL;
    q128 c3 = (q128)(pow(M_PI / (3.0 * sqrt(2.0)), 2.0 / 3.0) / tgamma(5.0 / 3.0));
    q128 l2 = (q128)ell * (q128)ell;
    for (int64_t j = 0; j < n; j++) {
        q128 p = phi ? (q128)phi[j] : (q128)1;
        q128 s0 = layers[j], s1 = layers[n + j], s2 = layers[2 * n + j];
        q128 b;
        if (dim == 2) {
            b = (q128)2 / l2 * (-p + 2 * (s0 - 2 * s1 + s2));
        } else if (dim == 3) {
            b = c3 / l2 * (-p + s0 - (q128)27 / 8 * s1 + (q128)9 / 4 * s2);
        } else {
            q128 s3 = layers[3 * n + j];
            b = (q128)4 / (l2 * or_qsqrt((q128)6)) * (-p + s0 - 9 * s1 + 16 * s2 - 8 * s3);
        }
        out[j] = (double)b;
    }
    return OR_OK;
}
