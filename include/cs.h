/*
 * cs.h -- C ABI of the GB300 causal-set interval-abundance library.
 *
 * The library generates a causal set, builds its causal matrix as row
 * bitsets, counts the cardinality of every causal interval, histograms the
 * counts into interval abundances and evaluates the Benincasa-Dowker action
 * (W. J. Cunningham, "High Performance Algorithms for Quantum Gravity and
 * Cosmology", arXiv:1805.04463, Chapter "Causal Set Action").
 *
 * Conventions shared by every entry point:
 *  - Pointers named *_dev are device (HBM) pointers; *_host are host
 *    pointers.  The caller allocates and owns every buffer; the library never
 *    frees caller memory.  Workspace sizes come from the *_workspace_bytes
 *    queries; a workspace must be 256-byte aligned.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Device entry points only enqueue work on it and return; they
 *    never synchronise the device.
 *  - Errors are returned as cs_status, never thrown or aborted.  Invalid
 *    arguments are rejected before anything is enqueued.  A CUDA launch or
 *    runtime error maps to CS_ECUDA.  Errors detected inside a kernel
 *    (a bounded wait that timed out, a rejection sampler that ran out of
 *    attempts) are written to the workspace status word and read back with
 *    cs_workspace_status().
 *  - Elements are labelled in time order (ties by generation index), so the
 *    strict upper triangle of the causal matrix holds every relation i < j.
 *  - hist[k] counts related pairs i < j whose open interval
 *    A_ij = J+(i) cap J-(j) holds exactly k elements; it is the thesis's
 *    n_{k+1} (Eq. IOIs, "inclusive order intervals").  Its length is
 *    cs_hist_len(n) = max(n - 1, 1).
 */
#ifndef CS_H
#define CS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CS_OK = 0,
    CS_EINVAL = -1,        /* bad argument (size, kind, alignment, pointer) */
    CS_ENOMEM = -2,        /* workspace too small or allocation failed */
    CS_ECUDA = -3,         /* CUDA runtime / launch error */
    CS_ETIMEOUT = -4,      /* a bounded in-kernel wait gave up */
    CS_EUNSUPPORTED = -5,  /* path or feature not available on this device */
    CS_ERANGE = -6,        /* sampler exhausted its attempt budget */
    CS_PENDING = 1         /* not an error: work that was polled has not finished yet */
} cs_status;

/* Causal-set kinds (Appendix "Causal Set Sprinklings"). */
enum {
    CS_2D_ORDER = 0,    /* random 2D order: two uniform random permutations u, v */
    CS_2D_DIAMOND = 1,  /* 1+1 Minkowski diamond, light-cone coordinates u, v on a 2^31 grid */
    CS_4D_DIAMOND = 2,  /* 3+1 Minkowski diamond of height 1, int32 grid of 2^20 per unit */
    CS_3D_DIAMOND = 3,  /* 2+1 Minkowski diamond of height 1, int32 grid of 2^20 per unit */
    CS_2D_DS_SLAB = 4,  /* 1+1 de Sitter slab |eta| <= 0.5 (spherical foliation, pseudo-radius 1),
                           Section "Spacetime Region Considered": coords[0] = eta (int32),
                           coords[1] = theta (uint32 bits, a full turn = 2^32), both in units of
                           2 pi / 2^32 rad.  The first sprinkle of this kind on a device uploads a
                           1.3 MB constant table synchronously (do it before any stream capture). */
    CS_2D_SQUARE = 5,   /* 1+1 Minkowski square t, x in [-1/2, 1/2) (Appendix, Minkowski spacetime,
                           1+1 Dimensional Square) on a grid of 2^30 per unit, stored in light-cone
                           coordinates coords[0] = u = t + x + 2^30, coords[1] = v = t - x + 2^30 */
    CS_2D_CYLINDER = 6  /* 1+1 Minkowski cylinder (same appendix, 1+1 Dimensional Cylinder):
                           coords[0] = t in [-2^31/pi, 2^31/pi) (t0 = 1), coords[1] = theta (uint32
                           bits, a full turn = 2^32), both in units of 2 pi / 2^32 */
};

/* Interval-count paths. */
enum {
    CS_PATH_AUTO = 0,   /* pick the faster path for this n */
    CS_PATH_POPC = 1,   /* AND + popcount tiles on the CUDA cores */
    CS_PATH_MMA = 2,    /* 0/1 operands as FP8 E4M3 on the tcgen05 tensor cores, fused epilogue */
    CS_PATH_MMA4 = 3    /* 0/1 operands as packed FP4 E2M1 (block-scaled kind::mxf4, every scale
                           factor 1) on CTA pairs running 2-SM MMAs: half the operand bytes,
                           the FP4 tensor rate.  Every count entry point takes it; on the batch
                           and job entry points CS_PATH_AUTO means cs_set_batch_tuning's path
                           (by default this one, where the device has tcgen05). */
};

/* ------------------------------------------------------------- layouts */

/* Spacetime dimension of a kind: 2, 3 or 4; 0 for an unknown kind. */
int cs_dim(int kind);

/* Bytes of the structure-of-arrays int32 coordinates: n * dim * 4.
 * Layout: coords[c * n + i] is coordinate c of element i (2D kinds: u, v;
 * 4D: t, x, y, z). */
size_t cs_coords_bytes(int kind, int64_t n);

/* 64-bit words per bitset row: ceil(n / 64) rounded up to a multiple of 16
 * (128-byte rows). */
int64_t cs_row_words(int64_t n);

/* Bytes of the n-row causal-matrix bitset: n * cs_row_words(n) * 8. */
size_t cs_bitset_bytes(int64_t n);

/* Length of the abundance histogram: max(n - 1, 1). */
int64_t cs_hist_len(int64_t n);

/* ---------------------------------------------------------- sprinkling */

/* Device workspace needed by cs_sprinkle for (kind, n). */
size_t cs_sprinkle_workspace_bytes(int kind, int64_t n);

/*
 * Sprinkle n elements of `kind` from `seed` and write their time-sorted
 * coordinates to coords_dev (cs_coords_bytes bytes, layout above).
 * Section "Coordinate Generation" and Appendix "Causal Set Sprinklings"
 * (1+1, 2+1 and 3+1 Minkowski diamonds, the 1+1 de Sitter slab):
 * coordinates are drawn independently per element and the elements are then
 * sorted by time (Section "Pairwise Relations").  The random numbers are the
 * counter-based SplitMix64 stream (draw(seed, stream, element, slot) = output
 * element*65536+slot of the generator seeded with output `stream` of the
 * generator seeded with seed); a 2D order is the pair of rank permutations
 * of streams 0 and 1, relabelled by u (coords[0] = 0..n-1); a 2D diamond
 * draws u, v from stream 2 (draw >> 33); a 4D (3D) diamond rejection-samples
 * (t, x, y, z) from stream 3 ((t, x, y) from stream 4) inside
 * |x| < min(t, 1 - t); the de Sitter slab draws theta and eta from stream 5.
 * Errors: CS_EINVAL (n < 1, n > 2^22, bad kind, NULL coords),
 * CS_ENOMEM (workspace too small), CS_ECUDA.  A 3D or 4D element that finds
 * no point in 16384 attempts sets CS_ERANGE in the workspace status word.
 */
int cs_sprinkle(int kind, int64_t n, uint64_t seed, int32_t *coords_dev,
                void *workspace_dev, size_t workspace_bytes, void *stream);

/* ------------------------------------------------------- causal matrix */

/*
 * Build the symmetrised causal matrix P + P^T (Section "Data Structures for
 * Totally Ordered Sets": one bitset per row) from time-sorted coordinates.
 * Bit j of row i (word j/64, bit j%64, least significant bit first) is 1 iff
 * i and j are timelike related, Delta s^2 < 0 strictly (Section
 * "Lorentzian Geometry"); 1+1 diamond, 1+1 square and 2D order: du * dv > 0,
 * for coordinates in [0, 2^31) (cs_sprinkle's range for these kinds); 1+1
 * cylinder: as the de Sitter slab, below; 3D and 4D:
 * dt^2 > |dx|^2, exact in int64 for |coordinates| < 2^29 (the sprinkled
 * diamonds stay within [-2^20, 2^20]); de Sitter slab: the angle around the circle
 * (mod 2^32) is below |d eta|.  For CS_2D_ORDER, coords[0] must increase
 * strictly with the label (as cs_sprinkle writes it: 0..n-1).  row_words
 * must be >= cs_row_words(n) and a multiple of 16; bits_dev holds
 * n * row_words uint64 and is fully written (padding bits zero).
 * Errors: CS_EINVAL, CS_ECUDA.
 */
int cs_causal_matrix(int kind, int64_t n, const int32_t *coords_dev,
                     uint64_t *bits_dev, int64_t row_words, void *stream);

/* -------------------------------------------------- interval abundance */

/* The path cs_interval_abundance runs for (n, path) on the current device:
 * CS_PATH_POPC, CS_PATH_MMA or CS_PATH_MMA4 (CS_PATH_AUTO follows the table
 * below; the tensor-core paths only where the device has tcgen05, and only
 * while the set's bitset plus the path's workspace fit the AUTO memory limit
 * -- a table entry of CS_PATH_MMA that does not fit falls back to
 * CS_PATH_MMA4; one of CS_PATH_MMA4 runs in bands (cs_mma4_band_panels) when
 * the whole operand matrix does not fit, and falls back to CS_PATH_POPC only
 * when not even bands of 32 supertile rows (8192 rows) do); -1 for invalid
 * arguments.  The rule depends only on n, the table and the limit, so the
 * workspace query and the count resolve alike. */
int cs_resolved_path(int64_t n, int path);

/* The device memory, in bytes, that CS_PATH_AUTO may plan a set's bitset and
 * count workspace into (process-wide).  0 (the default) means 90% of the
 * current device's memory.  Set it lower when other work shares the GPU.
 * Returns CS_OK. */
int cs_set_auto_memory_limit(size_t bytes);

/* The limit in force on the current device (bytes). */
size_t cs_get_auto_memory_limit(void);

/*
 * The CS_PATH_AUTO table, process-wide: entry e selects paths[e]
 * (CS_PATH_POPC, CS_PATH_MMA or CS_PATH_MMA4) for n_min[e] <= n < n_min[e+1].
 * n_min must start at 0 and increase; at most 16 entries.  The default is
 * {0: POPC, 1024: MMA, 4096: MMA4}; the autotuner
 * (paper_1805_04463_gb300/tune.py) installs measured thresholds.
 * Errors: CS_EINVAL.
 */
int cs_set_auto_paths(const int64_t *n_min, const int *paths, int count);

/* Copy the AUTO table out; returns its entry count (nothing is copied when
 * capacity is smaller than the count). */
int cs_get_auto_paths(int64_t *n_min, int *paths, int capacity);

/*
 * Tile order of the single-set tensor-core counts, process-wide: for
 * n_min[e] <= n < n_min[e+1], cs_interval_abundance, cs_layer_sums and
 * cs_evaluate on CS_PATH_MMA / CS_PATH_MMA4 hand out their 256 x 256
 * supertiles in raster blocks of raster[e] x raster[e] supertiles, widest
 * band first, so that the CTAs running at one time share operand panels in
 * L2.  raster in 1..32; n_min starts at 0 and increases; at most 16
 * entries.  The default is {0: 8}; the autotuner installs measured choices.
 * Results do not depend on it.  Errors: CS_EINVAL.
 */
int cs_set_auto_tiles(const int64_t *n_min, const int *raster, int count);

/* Copy the tile table out; returns its entry count (nothing is copied when
 * capacity is smaller than the count). */
int cs_get_auto_tiles(int64_t *n_min, int *raster, int capacity);

/*
 * Tuning of the multi-set counts, process-wide: `path` is what CS_PATH_AUTO
 * means for cs_batch_* and cs_count_jobs (CS_PATH_AUTO = the built-in
 * choice: CS_PATH_MMA4 where the device has tcgen05, else CS_PATH_POPC; a
 * tensor path on a device without tcgen05 also falls back to POPC);
 * max_run (1..64, default 16) is the longest run of consecutive work items
 * one CTA (pair) takes from the shared queue, so that a small set is counted
 * by few CTAs.  Results do not depend on either.  Errors: CS_EINVAL.
 */
int cs_set_batch_tuning(int path, int max_run);

/* The settings of cs_set_batch_tuning.  Errors: CS_EINVAL (NULL). */
int cs_get_batch_tuning(int *path, int *max_run);

/* Device workspace needed by cs_interval_abundance for (n, path).  The FP8
 * tensor-core path keeps two n x ceil(n/128)*128-byte operand matrices in it
 * (2 n^2 bytes, about 34 GB at n = 131072); the FP4 path one
 * n x ceil(n/256)*128-byte matrix E plus 256 bytes per row (n^2 / 2 bytes,
 * about 8.6 GB at n = 131072, 137 GB at n = 2^19) when that fits beside the
 * set's bitset within the AUTO memory limit, else a band buffer of the
 * widest bands that do (see cs_mma4_band_panels; at least one-panel bands,
 * 512 rows of E).  The FP4 count also runs with less than this, down to the
 * workspace of one-panel bands, in narrower bands. */
size_t cs_interval_abundance_workspace(int64_t n, int path);

/*
 * The FP4 pair path (CS_PATH_MMA4) with a workspace of workspace_bytes:
 * how many supertile rows (panels of 256 rows) each operand group holds.
 * The count covers the pairs i < j with 256 x 256 supertiles (si, sj), si <=
 * sj, whose MMAs read E rows of panels si and sj; when the whole E does not
 * fit, the panels fall into groups of g, and for each pair of groups a <= b
 * the kernel counts the supertiles with si in group a and sj in group b from
 * a band buffer holding those two groups' rows (2 g panels, each row only
 * over the columns the band's K ranges reach), re-expanded from the bitset
 * per band: (m + 1) m / 2 launches for m = ceil(nsb / g) groups.  Results do
 * not depend on g.  Returns nsb = ceil(n / 256) when the whole E fits (one
 * launch), 0 when not even g = 1 does, -1 for an invalid n.  The count call
 * takes the widest bands its workspace_bytes holds.
 */
int64_t cs_mma4_band_panels(int64_t n, size_t workspace_bytes);

/*
 * Host-side check of that band plan (no device work, no GPU needed): runs the
 * band list and the work-item decode the FP4 count's launches use, for bands
 * of `panels` supertile rows (>= ceil(n/256): the whole set as one launch)
 * and raster side `raster` (1..32), and writes to counts_host[si * nsb + sj]
 * (nsb = ceil(n/256); nsb^2 int64 entries, caller-owned, zeroed by the
 * callee) how many work items decode to the supertile (si, sj).  Every
 * supertile si <= sj must come out exactly once, none with si > sj.
 * Returns the number of work items; -1 for invalid arguments (n above 2^20,
 * panels < 1, raster out of range, NULL counts).
 */
int64_t cs_mma4_band_cover(int64_t n, int64_t panels, int raster, int64_t *counts_host);

/*
 * Interval abundances of a time-sorted causal matrix (Algorithm "Optimized
 * Interval Abundance Measurement" and Figure "Proper distance and the order
 * intervals": for every related pair i < j, |A_ij| is the popcount of the
 * AND of rows i and j over columns i+1..j-1, i.e. (C.C)_ij for the strict
 * upper triangle C).  hist_dev (cs_hist_len(n) int64) is zeroed and then
 * filled by the callee.  path selects the kernel (CS_PATH_AUTO picks one);
 * every path gives identical, exact results (the tensor paths multiply 0/1
 * values and accumulate integers below 2^23 in FP32).
 * Errors: CS_EINVAL (n < 1, n > 2^22, bad row_words, NULL or unaligned pointers), CS_ENOMEM
 * (workspace below cs_interval_abundance_workspace; on CS_PATH_MMA4 below the
 * workspace of one-panel bands), CS_EUNSUPPORTED (CS_PATH_MMA or CS_PATH_MMA4 on a
 * device without tcgen05), CS_ECUDA.  A timed-out in-kernel wait sets CS_ETIMEOUT in the
 * workspace status word.
 */
int cs_interval_abundance(int64_t n, const uint64_t *bits_dev, int64_t row_words,
                          int64_t *hist_dev, int path,
                          void *workspace_dev, size_t workspace_bytes, void *stream);

/*
 * Interval abundances plus the layer sums of the discrete d'Alembertian
 * (Section "The Benincasa-Dowker Action", Eqs. b2d_local, b4d_local): in the
 * same pass as cs_interval_abundance, for every element j and m = 0..kmax,
 * layer_dev[m*n + j] = sum of phi(i) over the elements i preceding j with
 * |A_ij| = m, i.e. over the inclusive order interval L_{m+1}(j).  phi_dev
 * (n doubles) may be NULL for phi = 1, in which case the sums are exact
 * element counts; otherwise they are double sums in atomic order.
 * layer_dev: (kmax+1) * n doubles, zeroed by the callee; 0 <= kmax <= 15.
 * Workspace and errors as cs_interval_abundance.
 */
int cs_layer_sums(int64_t n, const uint64_t *bits_dev, int64_t row_words, int64_t *hist_dev, int path,
                  const double *phi_dev, int kmax, double *layer_dev, void *workspace_dev,
                  size_t workspace_bytes, void *stream);

/*
 * The discrete d'Alembertian B phi(j) for every element from the layer sums
 * (kmax >= 2 in 1+1 and 2+1, >= 3 in 3+1), with discreteness scale ell:
 *   1+1 (Eq. b2d_local): (2/ell^2) [-phi(j) + 2 (S_0 - 2 S_1 + S_2)]
 *   2+1 (Eq. b3d_local): (c3/ell^2) [-phi(j) + S_0 - 27/8 S_1 + 9/4 S_2],
 *                        c3 = (pi/(3 sqrt 2))^(2/3) / Gamma(5/3)
 *   3+1 (Eq. b4d_local): (4/(ell^2 sqrt 6)) [-phi(j) + S_0 - 9 S_1 + 16 S_2 - 8 S_3]
 * phi_dev may be NULL (phi = 1: B 1 is the element's curvature estimate).
 * out_dev: n doubles.  Asynchronous.  Errors: CS_EINVAL, CS_ECUDA.
 */
int cs_dalembertian(int dim, int64_t n, const double *phi_dev, const double *layer_dev, int kmax,
                    double ell, double *out_dev, void *stream);

/*
 * Read (synchronously: waits for `stream`) and clear the status word that
 * kernels of the last call using this workspace wrote.  Returns CS_OK, the
 * in-kernel error, or CS_ECUDA if the stream itself failed.
 */
int cs_workspace_status(void *workspace_dev, void *stream);

/* ----------------------------------------------------------------- action */

/*
 * Benincasa-Dowker action from host abundances (Section "The
 * Benincasa-Dowker Action"), with hist[k] = n_{k+1}:
 *   dim 2, local (Eq. s2d_local):   S = 2 (N - 2 n1 + 4 n2 - 2 n3)
 *   dim 3, local (Eq. s3d_local):   S = c3 (N - n1 + 27/8 n2 - 9/4 n3),
 *                                   c3 = (pi/(3 sqrt 2))^(2/3) / Gamma(5/3), l/l_p = 1
 *   dim 4, local (Eq. s4d_local):   S = 4/sqrt(6) (N - n1 + 9 n2 - 16 n3 + 8 n4),
 *                                   taking (l/l_p)^2 = 1
 *   dim 2, smeared (Eq. s2d_smeared): S = 2 eps [N - 2 eps sum_m n_m f2(m-1, eps)]
 *   dim 3, smeared:                   S = c3 eps^(2/3) [N - eps sum_m n_m f3(m-1, eps)]
 *   dim 4, smeared (Eq. s4d_smeared): S = 4 sqrt(eps/6) [N - eps sum_m n_m f4(m-1, eps)]
 * eps <= 0 or eps == 1 selects the local action (the smeared forms reduce to
 * it at eps = 1); 0 < eps < 1 the smeared one, summed over the whole
 * histogram in double-double (compensated FP64) arithmetic.
 * out (may be NULL) receives S; bracket_out (may be NULL) the exact integer
 * in parentheses of the local form (dim 3: eight times it,
 * 8N - 8n1 + 27n2 - 18n3).  Synchronous, host only.
 * Errors: CS_EINVAL (dim not 2, 3 or 4, eps > 1 or NaN, n < 0, len < 0).
 */
int cs_action(int dim, int64_t n, const int64_t *hist_host, int64_t len,
              double eps, double *out, int64_t *bracket_out);

/* Device workspace needed by cs_action_device. */
size_t cs_action_workspace_bytes(void);

/*
 * The same actions evaluated on the device, for n_eps values of eps at once
 * (eps_host is read at call time): out_dev[e] receives S for eps_host[e] and
 * *bracket_dev (may be NULL) the local bracket.  Asynchronous on `stream`;
 * hist_dev is the device histogram written by cs_interval_abundance.  The
 * smeared sums are split over 128 blocks whose double-double partial sums
 * go to the workspace.  Both action entry points stop each smeared sum at
 * the first k past which the remaining terms provably move S by less than
 * 1e-15 (bounding the abundances' sum by n(n-1)/2 here, by the histogram's
 * own sum in cs_action).
 * Errors: CS_EINVAL (as cs_action, or n_eps outside 1..16), CS_ENOMEM
 * (workspace too small), CS_ECUDA.
 */
int cs_action_device(int dim, int64_t n, const int64_t *hist_dev, int64_t len,
                     const double *eps_host, int n_eps, double *out_dev,
                     int64_t *bracket_dev, void *workspace_dev, size_t workspace_bytes,
                     void *stream);

/* ------------------------------------------------------- host-buffer call */

/*
 * One whole evaluation from host buffers, for callers that keep their data
 * on the host: copies coords_host (cs_coords_bytes) to the device, builds the
 * causal matrix, counts intervals on `path`, evaluates the actions for n_eps
 * values of eps, and copies hist_host (cs_hist_len(n) int64), actions_host
 * (n_eps doubles) and *bracket_host back.  If coords_host is NULL the set is
 * sprinkled on the device from (kind, n, seed) instead.  Device memory comes
 * from the device's default stream-ordered pool and is freed before the call
 * ends; the pool keeps it for the next call, unless the call took more than
 * a quarter of the device's memory, in which case the pool is trimmed.
 * Synchronous: returns after the results are on the host.
 * Errors: as the individual entry points, plus CS_ENOMEM.
 */
int cs_evaluate(int kind, int64_t n, uint64_t seed, const int32_t *coords_host, int path,
                const double *eps_host, int n_eps, int64_t *hist_host,
                double *actions_host, int64_t *bracket_host, void *stream);

/* ----------------------------------------------------- batched ensembles */

/* One causal set of a batch. */
typedef struct {
    int32_t kind;      /* a CS_* kind */
    int32_t reserved;  /* must be 0 */
    int64_t n;         /* 1 .. CS_BATCH_MAX_N */
    uint64_t seed;     /* the set equals cs_sprinkle(kind, n, seed, ...) */
} cs_set_desc;

#define CS_BATCH_MAX_N 8192
#define CS_BATCH_MAX_SETS 1048576

/* Opaque host-side plan of a batch (its device tables live in the workspace). */
typedef struct cs_batch cs_batch;

/* Device workspace for a batch of n_sets sets on `path` (0 for invalid input):
 * per set its coordinates, keys, bitset (n * cs_row_words(n) * 8 bytes) and,
 * on the tensor paths, its count operands (cs_operands_bytes); for the
 * light-cone kinds one 1584-byte relation table per 64 elements; the plan's
 * device tables (per set, per relate / mirror / expansion block, per column
 * tile) and the smeared-sum coefficients and cutoffs. */
size_t cs_batch_workspace_bytes(const cs_set_desc *sets, int n_sets, int path);

/* Entries of the batch histogram: sum over sets of cs_hist_len(n); set s
 * starts at the sum over the earlier sets.  -1 for invalid input. */
int64_t cs_batch_hist_len(const cs_set_desc *sets, int n_sets);

/*
 * Plan a batched ensemble: many sets of different kinds and sizes evaluated
 * by one fixed sequence of launches (the thesis's experiments average ensembles
 * of sprinklings, Section "Simulations and Scaling Evaluations"; a sprinkled N
 * is Poisson distributed, Appendix "Causal Set Sprinklings").  Lays out every
 * set's coordinates, bitset and count operands in workspace_dev (1024-byte
 * aligned, cs_batch_workspace_bytes bytes, owned by the caller and used by the
 * plan until cs_batch_destroy) and uploads the plan's device tables
 * synchronously on `stream`.  *out receives a host handle.
 * Errors: CS_EINVAL (bad sets, path, pointers, alignment), CS_ENOMEM
 * (workspace too small or host allocation failed), CS_EUNSUPPORTED,
 * CS_ECUDA.
 */
int cs_batch_create(const cs_set_desc *sets, int n_sets, int path, void *workspace_dev,
                    size_t workspace_bytes, cs_batch **out, void *stream);

/*
 * Evaluate every set of the plan: sprinkle, causal matrix, interval
 * abundances and actions, for all sets at once (one persistent count kernel
 * over the tiles of all sets, largest sets first).  Enqueues memsets and
 * kernels only, so the call can be captured into a CUDA graph and replayed.
 * hist_dev: cs_batch_hist_len int64 (zeroed by the callee); actions_dev:
 * n_sets x n_eps doubles, set-major (may be NULL when n_eps = 0);
 * brackets_dev: n_sets int64 (may be NULL).  Results equal the single-set
 * entry points' for the same (kind, n, seed).  In-kernel errors go to the
 * workspace status word (cs_workspace_status).
 * Errors: CS_EINVAL, CS_ECUDA.
 */
int cs_batch_launch(const cs_batch *b, const double *eps_host, int n_eps, int64_t *hist_dev,
                    double *actions_dev, int64_t *brackets_dev, void *stream);

/*
 * Poll the plan's last launch without waiting: CS_PENDING while the work it
 * enqueued (or the last replay of a CUDA graph that captured it) is still
 * running; once it has finished, the in-kernel status word of that launch
 * (CS_OK, or the first error a kernel recorded, e.g. CS_ETIMEOUT).  Each
 * launch ends by copying the status word to pinned host memory owned by the
 * plan and recording an event (an external event node under capture); the
 * poll queries that event and reads the copy, so it never synchronises and
 * enqueues nothing.  Before the first launch it returns CS_OK.  Do not
 * destroy the plan while a launch may still be running.
 * Errors: CS_EINVAL (NULL), CS_ECUDA (the event query failed).
 */
int cs_batch_poll(const cs_batch *b);

/* The count path a plan runs (CS_PATH_POPC, CS_PATH_MMA or CS_PATH_MMA4;
 * CS_PATH_AUTO plans the batch path of cs_set_batch_tuning, by default
 * CS_PATH_MMA4 where the device has tcgen05), -1 for NULL. */
int cs_batch_path(const cs_batch *b);

/* Free the host handle (the workspace stays the caller's). */
void cs_batch_destroy(cs_batch *b);

/* ------------------------------------------- counting slices of many sets */

/* Number of work items a set of size n splits into on `path` (tiles of its
 * interval count: 128 x 128 POPC tiles, 128 x 256 FP8 tile slots, or 256 x
 * 256 supertile slots on CS_PATH_MMA4, in raster blocks of side 8;
 * CS_PATH_AUTO means the batch path of cs_set_batch_tuning, so change that
 * setting only between whole sets of jobs); -1 for invalid input. */
int64_t cs_count_items(int64_t n, int path);

/* Bytes of the tensor-core operands of a set of size n on `path`
 * (CS_PATH_MMA: two n x ceil(n/128)*128-byte FP8 matrices; CS_PATH_MMA4: one
 * n x ceil(n/256)*128-byte packed FP4 matrix plus two n x 128-byte diagonal
 * blocks; 1024-byte aligned); 0 for CS_PATH_POPC or invalid input. */
size_t cs_operands_bytes(int64_t n, int path);

/*
 * Expand a set's bitset into its tensor-core operands for `path` (0/1 values;
 * FP8: U holds each row's future, L its past; packed FP4: E holds every row
 * of the symmetric matrix, DU / DL the future / past of each row within its
 * own 256-column block), once, for later
 * cs_count_jobs slices on the same path.  operands_dev:
 * cs_operands_bytes(n, path), 1024-byte aligned.  Asynchronous.
 * Errors: CS_EINVAL (also for CS_PATH_POPC), CS_ENOMEM, CS_ECUDA.
 */
int cs_prepare_operands(int64_t n, int path, const uint64_t *bits_dev, int64_t row_words, void *operands_dev,
                        size_t operands_bytes, void *stream);

/* One slice of one set's interval count. */
typedef struct {
    const uint64_t *bits;  /* the set's bitset (cs_causal_matrix) */
    int64_t n;
    int64_t row_words;
    int64_t *hist;         /* the set's histogram: counts are ADDED (zero it before the first slice) */
    void *operands;        /* tensor paths: from cs_prepare_operands (same path); ignored on CS_PATH_POPC */
    int64_t item_begin;    /* slice [item_begin, item_end) of 0 .. cs_count_items(n, path) */
    int64_t item_end;
} cs_count_job;

/* Host staging bytes (table_host) and device workspace bytes of cs_count_jobs. */
size_t cs_count_jobs_table_bytes(int n_jobs, int path);
size_t cs_count_jobs_workspace_bytes(int n_jobs, int path);

/*
 * Count slices of several sets in one persistent launch (Algorithm
 * "Optimized Interval Abundance Measurement": the pairs of a set are
 * independent, so any partition of its work items can run in any order and
 * share a launch with other sets' items).  The job table is encoded into
 * table_host (cs_count_jobs_table_bytes, 128-byte aligned, preferably pinned;
 * the caller keeps it unchanged until the stream has passed this call) and
 * copied to the workspace.  Each job's counts are added to its histogram with
 * integer atomics, so a set's final histogram equals cs_interval_abundance's
 * however its items are sliced.  Asynchronous.
 * Errors: CS_EINVAL (bad jobs, slices, pointers, alignment), CS_ENOMEM,
 * CS_EUNSUPPORTED, CS_ECUDA.
 */
int cs_count_jobs(const cs_count_job *jobs, int n_jobs, int path, void *table_host, void *workspace_dev,
                  size_t workspace_bytes, void *stream);

/* ---------------------------------------------- allocation-free sprinkle */

/* Largest n that cs_sprinkle_noalloc accepts. */
#define CS_SPRINKLE_NOALLOC_MAX_N 262144

/*
 * cs_sprinkle for callers that cannot allocate device memory: code that runs
 * while a stream is being captured into a CUDA graph (allocation is not
 * allowed there), plugins that may only use memory their host application
 * hands them, or real-time loops that must stay off the allocator.  The
 * thesis has no counterpart; this is a convenience of this library.
 * Writes exactly what cs_sprinkle writes for the same (kind, n, seed) to
 * coords_dev and takes no workspace: its scratch is one file-scope device
 * array of 12 MiB that every GPU loading the library holds until the process
 * exits.  The call allocates nothing (no cudaMalloc, cudaFree or allocating
 * library routine).  The first call on a device looks up the array's device
 * address (and, for CS_2D_DS_SLAB, uploads that kind's 1.3 MB constant
 * table), so make that first call before any stream capture starts.
 * All calls on a device share the array and it keeps the last call's
 * contents; calls whose work overlaps on the GPU (unordered streams) race
 * and may corrupt each other's output.  A 4D element that exhausts its
 * rejection attempts (probability below 1e-900) is not reported here.
 * Errors: CS_EINVAL (bad kind, NULL or unaligned coords, n < 1 or
 * n > CS_SPRINKLE_NOALLOC_MAX_N), CS_ECUDA; CS_ENOMEM only if the array
 * were smaller than the scratch layout needs (a build inconsistency).
 */
int cs_sprinkle_noalloc(int kind, int64_t n, uint64_t seed, int32_t *coords_dev, void *stream);

/* ------------------------------------------ degrees and sparse lists */

/*
 * In- and out-degree vectors (Section "Optimized GPU Linking Algorithm",
 * Algorithm "Write Operations for Degrees") from the symmetric bitset of
 * time-sorted labels: in_dev[j] = number of i < j related to j (its past),
 * out_dev[i] = number of j > i related to i (its future).  int32, n each;
 * either may be NULL.  Asynchronous.  Errors: CS_EINVAL, CS_ECUDA.
 */
int cs_degrees(int64_t n, const uint64_t *bits_dev, int64_t row_words, int32_t *in_dev, int32_t *out_dev,
               void *stream);

/* Device workspace for cs_sparse_offsets / cs_sparse_columns. */
size_t cs_sparse_workspace_bytes(int64_t n);

/*
 * The past (direction 0) or future (direction 1) sparse relation lists in
 * compressed-row form (the thesis decodes its relation list into past and
 * future sparse lists, Section "GPU Linking Algorithm").  Row i owns
 * cols[offsets[i] .. offsets[i+1]): the labels related to i before (0) or
 * after (1) it, increasing.  Two calls: cs_sparse_offsets writes the n+1
 * int64 offsets (offsets_dev[n] = the list length, an exclusive scan of the
 * row counts); the caller reads offsets_dev[n], provides cols_dev with room
 * for that many int32 and calls cs_sparse_columns with the same bitset.
 * A row whose list would end past cols_capacity is skipped and CS_ENOMEM is
 * recorded in the workspace status word (cs_workspace_status).
 * Asynchronous.  Errors: CS_EINVAL, CS_ENOMEM (workspace too small), CS_ECUDA.
 */
int cs_sparse_offsets(int64_t n, const uint64_t *bits_dev, int64_t row_words, int direction,
                      int64_t *offsets_dev, void *workspace_dev, size_t workspace_bytes, void *stream);
int cs_sparse_columns(int64_t n, const uint64_t *bits_dev, int64_t row_words, int direction,
                      const int64_t *offsets_dev, int32_t *cols_dev, int64_t cols_capacity,
                      void *workspace_dev, size_t workspace_bytes, void *stream);

/* ------------------------------------------- chains and antichains */

/* Device workspace for cs_longest_chain and cs_greedy_antichain. */
size_t cs_chain_workspace_bytes(int64_t n);

/*
 * Longest chain (Section "Set Partitions", Algorithm "Maximal Chain
 * Length") on the symmetric bitset of time-sorted labels.  For a pair
 * i < j: *length = the number of relations on the longest chain from i to j
 * (1 for a link), or -1 if i does not precede j (also for j <= i).  With
 * i = j = -1: *length = the height of the whole set, the number of elements
 * of its longest chain.  Computed by peeling the minimal elements of the
 * Alexandroff set (or of the whole set) round by round.  Synchronous (the
 * host checks the rounds in batches).  Errors: CS_EINVAL, CS_ENOMEM
 * (workspace too small), CS_ECUDA.
 */
int cs_longest_chain(int64_t n, const uint64_t *bits_dev, int64_t row_words, int64_t i, int64_t j,
                     int64_t *length, void *workspace_dev, size_t workspace_bytes, void *stream);

/*
 * Greedy maximal antichain (Section "Set Partitions", Algorithm "Maximal
 * Antichain") grown from `seed`: the candidates are the elements unrelated
 * to the seed; each round keeps the candidate k that leaves the most
 * elements when its relations are removed (the smallest label on ties) and
 * removes its relations.  members_dev (row_words words, 8-byte aligned)
 * receives the antichain as a bitset, *size its size.  Synchronous.
 * Errors: CS_EINVAL, CS_ENOMEM (workspace too small), CS_ECUDA.
 */
int cs_greedy_antichain(int64_t n, const uint64_t *bits_dev, int64_t row_words, int64_t seed,
                        uint64_t *members_dev, int64_t *size, void *workspace_dev, size_t workspace_bytes,
                        void *stream);

/* ------------------------------------------------------------ peak probes */

/*
 * Peak probe for the roofline of a count path: runs `reps` repetitions
 * (1..2^22) of the path's innermost operation on every SM, with nothing
 * around it, and returns the device-wide rate in *rate:
 *   CS_PATH_POPC  32-bit population counts per second (independent chains in
 *                 registers);
 *   CS_PATH_MMA   dense FP8 FLOP/s (2 per multiply-add) of the FP8 count
 *                 kernel's MMA, M128 N256 K32 kind::f8f6f4 on one SM, four per
 *                 repetition, operands resident in shared memory;
 *   CS_PATH_MMA4  dense FP4 FLOP/s of the FP4 count kernel's MMA, M256 N256
 *                 K64 block-scaled kind::mxf4 on CTA pairs (cta_group::2).
 * workspace_dev: 256 bytes, 256-byte aligned (the status word).
 * Synchronous: creates its own stream and events.  The thesis has no
 * counterpart (measurement infrastructure of this library).
 * Errors: CS_EINVAL, CS_EUNSUPPORTED (tensor paths without tcgen05),
 * CS_ECUDA, CS_ETIMEOUT (a bounded wait gave up).
 */
int cs_peak_probe(int path, int64_t reps, void *workspace_dev, double *rate);

/* ---------------------------------------------------- failure detection */

/*
 * Bounded-wait self test: one warp waits on an mbarrier through the same
 * bounded-wait path the pipelines use, with a limit of limit_s seconds
 * (0 < limit_s <= 10).  With complete = 0 nothing completes the barrier, so
 * the wait gives up, CS_ETIMEOUT lands in the workspace status word
 * (cs_workspace_status) and the kernel returns normally: the context stays
 * usable.  With complete != 0 the barrier completes first and the status
 * stays CS_OK.  The thesis has no counterpart (failure detection of this
 * library).  Errors: CS_EINVAL, CS_ECUDA.
 */
int cs_selftest_wait(void *workspace_dev, double limit_s, int complete, void *stream);

/* Host-side fault injection for tests: the next `count` times the step
 * `where` runs it fails as if its CUDA call had failed (count = 0 clears).
 * CS_FAULT_ALLOC: the device allocations of cs_evaluate (-> CS_ENOMEM);
 * CS_FAULT_LAUNCH: the kernel launches of cs_interval_abundance (-> CS_ECUDA). */
#define CS_FAULT_ALLOC 1
#define CS_FAULT_LAUNCH 2
int cs_inject_fault(int where, int count);

/* ------------------------------------------------------------------ misc */

/* Static description of a status code. */
const char *cs_strerror(int status);

/* Library version string. */
const char *cs_version(void);

/* Description of the last CUDA runtime error that made a single-set entry
 * point (cs_sprinkle, cs_causal_matrix, cs_interval_abundance,
 * cs_layer_sums, cs_dalembertian, cs_action_device, cs_evaluate) return
 * CS_ECUDA on the calling host thread; "no error" if there was none.  The
 * string is static; the record is never cleared. */
const char *cs_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CS_H */
