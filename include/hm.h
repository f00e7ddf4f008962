/*
 * hm.h -- C ABI of the GB300 (sm_103a) graph-coloured H^1 peeling compressor.
 *
 * Problem statement (Levitt & Martinsson, Section 1): a user can apply an
 * N x N matrix A and its adjoint A^* to tall thin matrices, Y = A Omega and
 * Z = A^* Psi.  From such products with structured random test matrices the
 * library recovers an H^1 representation of A on a cluster tree of points:
 * low-rank factors U B V^T for every admissible block of levels 2..L
 * (Section 4.1, Algorithm 4.1) and dense neighbour blocks of the leaf level
 * (Section 4.1.3).
 *
 * Conventions shared by every entry point
 *  - Every call returns hm_status; no exception crosses the ABI.  On error the
 *    context keeps its last consistent state and hm_last_error() describes the
 *    failure; hm_destroy() is always safe.
 *  - Calls run in order: hm_tree_build -> (hm_color, hm_sample)* / hm_compress
 *    -> hm_apply, hm_relerr.  A call out of order returns HM_ESTATE.
 *  - Pointers named *_dev are device pointers, owned by the caller, read during
 *    the call only (inputs) or written before the call returns (outputs).
 *    Pointers named *_host are host pointers, likewise owned by the caller.
 *  - All device work is issued on the stream given to hm_create (a
 *    cudaStream_t passed as void*; NULL = the legacy default stream).  Calls
 *    that return sizes to the host (hm_tree_build, hm_color, hm_compress,
 *    hm_get_info, hm_export) synchronise that stream; the others do not.
 *    hm_compress also colours the levels on two more streams that the context
 *    creates (non-blocking, highest priority), from two host threads of its
 *    own, ahead of the level loop; all have finished when hm_compress returns.
 *  - The context owns every device buffer it allocates (tree, colourings,
 *    samples, factors); hm_destroy frees them.  Allocation is stream-ordered
 *    (cudaMallocAsync) from the device's default memory pool, whose release
 *    threshold hm_create raises to the maximum, so freed blocks stay cached in
 *    the process for the next call instead of returning to the driver.
 *  - Matrices at the boundary are column-major with leading dimension n and are
 *    indexed in the caller's ORIGINAL point order.
 */
#ifndef HM_H
#define HM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    HM_OK = 0,
    HM_EINVAL = 1,    /* invalid argument (null pointer, bad size, bad mode) */
    HM_ENOMEM = 2,    /* device or host allocation failed */
    HM_ESTATE = 3,    /* call made out of order */
    HM_ECUDA = 4,     /* a CUDA runtime call or kernel launch failed */
    HM_EOP = 5,       /* the user's black-box operator returned non-zero */
    HM_ETIMEOUT = 6,  /* a bounded device-side wait gave up */
    HM_ENOTSUP = 7    /* outside the implemented limits (e.g. > 1024 colours) */
} hm_status;

/* Arithmetic of the path.  Samples, factors and every subtraction from a
 * sample are stored and done in FP64 in all three modes. */
typedef enum {
    HM_FP64 = 0,             /* FP64 throughout */
    HM_MIXED_BF16X6 = 1,     /* black box (built-in kernel operator): FP32 kernel
                                evaluation, 3-piece BF16 split of both operands,
                                6 tcgen05 products, FP32 accumulation promoted to
                                double-float, FP64 output; peel, QR and core
                                solves FP64 */
    HM_MIXED_BF16X6_F32 = 2  /* the same black box; the products of the peel, the
                                pivoted QR factorisations, the core's Gram
                                products and least-squares solves in FP32 (the
                                samples they work on carry FP32-class rounding
                                from the black box already) */
} hm_precision;

/* Kernel functions of the built-in operator (A_ij = K(x_i, x_j)). */
enum {
    HM_K_LOG = 1,        /* log|x - y|, 0 where x == y        */
    HM_K_LAPLACE3D = 2,  /* 1 / (4 pi |x - y|), 0 where x == y */
    HM_K_INVR = 3,       /* 1 / |x - y|, 0 where x == y        */
    HM_K_EXP = 4         /* exp(-|x - y|)                       */
};

/* Kinds of black-box operator. */
enum {
    HM_OP_KERNEL = 0,    /* built-in: kernel function on the tree's points   */
    HM_OP_DENSE = 1,     /* built-in: stored dense n x n matrix (device)     */
    HM_OP_CALLBACK = 2   /* user routine, see hm_apply_fn                    */
};

#define HM_LEVEL_LEAF (-1)

typedef struct hm_ctx hm_ctx;

typedef struct {
    int d;                /* dimension of the points: 1, 2 or 3 */
    int leaf_size;        /* m: a box is split while it holds more than m points; the
                             default of hm_tree_build when its leaf_size is 0 */
    int uniform_depth;    /* 0: adaptive tree; > 0: split every box down to this level */
    int r;                /* columns per colour of the Gaussian test matrices (k + p), 1..64 */
    int oversample;       /* p: in tolerance mode k <= r - p (Section 2.5 suggests p = 10) */
    int rank;             /* default rank of hm_compress (used when its tol and rank are
                             both 0): > 0 fixed rank k (<= r), or the cap with tol */
    double tol;           /* default tolerance of hm_compress (same rule): > 0 keep pivots
                             with |R_jj| > tol |R_11| (at most r - p, and at most rank
                             when rank > 0 too) */
    int precision;        /* hm_precision */
    int keep_samples;     /* non-zero: keep every level's peeled samples for hm_export */
    uint64_t seed;        /* Philox4x32-10 key of all test matrices */
    int format;           /* HM_FORMAT_H1 (per-block bases, Section 4.1),
                             HM_FORMAT_UNIFORM_H1 (one column and one row basis per
                             box and level, Section 4.2) or HM_FORMAT_H2 (nested
                             bases, Section 4.3) */
} hm_config;

/* Formats of the compressed operator (hm_config.format). */
enum {
    HM_FORMAT_H1 = 0,          /* Algorithm 4.1: A_ab ~ U_ab B_ab V_ab^T, bases per pair */
    HM_FORMAT_UNIFORM_H1 = 1,  /* Section 4.2: A_ab ~ U_a B_ab V_b^T.  Stage 1 samples every
                                  box's interactions at once (box colouring, Gaussian test
                                  matrices) and keeps the whole r-column sample basis U_a;
                                  stage 2 fills the pair test matrices with the bases,
                                  Z(I_b) = A_ab^* U_a, and V_b = qr(sum over a of
                                  A_ab^* U_a M_a, k) with Gaussian k_a x r mixes M_a,
                                  B_ab = (A_ab^* U_a)^T V_b.  The truncation (rank or tol)
                                  applies to V.  QR and the mixing in FP64 in every mode */
    HM_FORMAT_H2 = 2           /* Section 4.3, Algorithm 4.2: as HM_FORMAT_UNIFORM_H1, but
                                  every basis is a truncated SVD of its sample augmented by
                                  the parent's far field, U_t(I_a) S_t (U_t^T Gamma_t) with
                                  a Gaussian Gamma_t of the parent's rows (the same on the
                                  row side), the stage-2 mixes are U_a^T Gamma'_a, and once
                                  a cut's bases exist the previous cut is nested: its short
                                  bases U~_t = U_a^T U_t (eq. nested_basis).  The operator
                                  keeps the long bases of the finest cut, the short bases,
                                  the cores and the leaf blocks; hm_apply runs the upward
                                  and downward passes of Algorithm 4.3.  SVD, nesting and
                                  mixing in FP64 in every mode.  hm_apply_noalloc and
                                  keep_samples are not supported (HM_ENOTSUP) */
};

/*
 * User black box (Section 1): Y = A X when trans == 0, Y = A^* X when trans == 1.
 * X_dev and Y_dev are device, column-major n x s (leading dimension n), in the
 * original point order; the routine must enqueue its work on `stream` (or
 * finish it before returning).  Return 0 on success; any other value makes the
 * library call fail with HM_EOP.
 */
typedef int (*hm_apply_fn)(void *user, int trans, const double *X_dev, double *Y_dev,
                           int64_t s, void *stream);

typedef struct {
    int kind;                 /* HM_OP_* */
    int kernel;               /* HM_K_* for HM_OP_KERNEL */
    const double *dense_dev;  /* HM_OP_DENSE: n x n column-major, original order */
    hm_apply_fn apply;        /* HM_OP_CALLBACK */
    void *user;               /* HM_OP_CALLBACK: passed back to apply */
} hm_op;

typedef struct {
    int64_t n;
    int L;                    /* depth of the tree */
    int n_boxes;              /* boxes over all levels */
    int colors[32];           /* chi_l per cut level (0 where none), index L+1 = leaf */
    int64_t pairs[32];        /* admissible pairs per cut level; index L+1 = neighbour pairs */
    int64_t vertices[32];     /* constraint sets per cut level; index L+1 = leaf */
    int64_t matvec_cols;      /* columns of Omega and Psi applied to A or A^* */
    int64_t factor_floats;    /* floats stored in U, B, V and the leaf blocks */
    int max_rank;             /* largest k over all blocks */
    double seconds_sample;    /* time in the black box during hm_compress */
    double seconds_total;     /* wall time of hm_compress */
    double seconds_phase[8];  /* device time per phase of hm_compress (CUDA events):
                                 0 colouring (host time the level loop waited for
                                 the colourings that run ahead of it), 1 test matrices, 2 black box (admissible
                                 levels), 3 peel, 4 bases and cores, 5 leaf black box,
                                 6 leaf peel and extraction, 7 the tensor-core
                                 contraction kernels alone (inside 2) */
    int64_t act_rows[32];     /* per cut level: sum over colours of the active rows
                                 (rows of Omega that are not zero); index L+1 = leaf */
    int64_t kernel_launches;  /* kernels this library launched during hm_compress */
    int64_t launches_total;   /* kernels this library launched since it was loaded */
    int64_t tc_kernel_evals;  /* kernel-matrix entries the tensor-core sampler evaluated
                                 during hm_compress: for every colour, its output rows
                                 (the rows of its sample tiles) x its active rows */
    int64_t device_allocs;    /* device allocations this library has made since it was
                                 loaded (all contexts; hm_apply_noalloc makes none) */
    int bb_tc_levels;         /* admissible levels of the last hm_compress whose black box
                                 ran on the tensor cores (split-BF16) */
    int bb_fp64_levels;       /* levels (admissible and leaf) whose black box ran in FP64:
                                 HM_FP64, a dense or callback operator, or, in a mixed
                                 mode, an r the tensor-core sampler does not take
                                 (r % 8 != 0 or r > 40).  The leaf level of a mixed mode
                                 with the kernel operator evaluates K in FP32 and sums
                                 in FP64, and counts in neither field */
    int leaf_size;            /* m of the current tree (hm_tree_build) */
    int rank;                 /* rank (or rank cap) of the last hm_compress; 0 = none */
    double tol;               /* tolerance of the last hm_compress; 0 = fixed rank */
    double seconds_peel_update; /* HM_MIXED_BF16X6: device time (CUDA events) of the
                                 double-float peel update kernels during hm_compress */
    int64_t peel_update_macs; /* their multiply-adds: sum over tile rows, live coarse
                                 pairs and columns of rows x k x columns */
    uint64_t pool_used_bytes; /* device memory in use in the device's default memory pool
                                 (all contexts of the process) when the info was read */
    uint64_t pool_peak_bytes; /* its high-water mark since the start of the last
                                 hm_compress (which resets it) */
} hm_info;

/*
 * Create a context for one compression job.  cfg is copied (Section 2.5 for r,
 * p, rank and tol; Section 3 for d, leaf_size, uniform_depth).  stream: a
 * cudaStream_t or NULL.  The device current at this call is the context's
 * device: every later call on the context runs on it (and restores the
 * caller's current device before returning).  *out receives the context,
 * owned by the caller until hm_destroy.  Errors: HM_EINVAL (null out or cfg;
 * d not 1..3; leaf_size < 0; r not 1..64; rank < 0 or > r; tol < 0 or NaN;
 * with tol > 0, p not in 0..r-1; unknown precision; uniform_depth not 0..21),
 * HM_ENOMEM.
 */
hm_status hm_create(hm_ctx **out, const hm_config *cfg, void *stream);

/* Free the context and everything it owns.  Safe on NULL and after errors. */
hm_status hm_destroy(hm_ctx *ctx);

/*
 * Section 3: cluster tree over n points (points_dev: device, n x d row-major
 * FP64, original order) with leaves of at most leaf_size points (the paper's
 * m; 0 = hm_config.leaf_size), and the neighbour and interaction lists of
 * every cut.  The points are copied into the context (permuted into Morton
 * order); a second call starts a new job on the same context.  Errors:
 * HM_EINVAL (null ctx or points, n < 1 or n > 2^30, leaf_size < 0, or both
 * leaf sizes 0), HM_ENOMEM, HM_ECUDA.
 */
hm_status hm_tree_build(hm_ctx *ctx, const double *points_dev, int64_t n, int leaf_size);

/*
 * Sections 4.1.2-4.1.3, Algorithm 2.3: build the constraint-incompatibility
 * graph of cut `level` (2..L, or HM_LEVEL_LEAF for the leaf neighbour pairs)
 * and colour it with DSatur.  *n_colors (host, may be NULL) receives chi.
 * Errors: HM_EINVAL (null ctx, level out of range), HM_ESTATE (no tree),
 * HM_ENOTSUP (more than 2^20 constraint sets or 1024 colours), HM_ENOMEM,
 * HM_ECUDA.
 */
hm_status hm_color(hm_ctx *ctx, int level, int *n_colors);

/*
 * Section 4.2 (uniform H^1, first stage): the incompatibility graph of the box
 * constraint sets of cut `level` (2..L) -- box alpha, with a non-empty
 * interaction list, asks for random rows on int(alpha) and zeros on
 * near(alpha); two boxes conflict when one's random boxes meet the other's
 * zero boxes -- coloured with DSatur (Algorithm 2.3, ties by degree then
 * id).  hm_compress does this itself in HM_FORMAT_UNIFORM_H1; the call exposes
 * the stage (and hm_export its result) for tests.  *n_colors (host, may be
 * NULL) receives chi.  Errors: HM_EINVAL (null ctx, level out of range),
 * HM_ESTATE (no tree), HM_ENOTSUP (more than 2^20 boxes or 1024 colours),
 * HM_ENOMEM, HM_ECUDA.
 */
hm_status hm_color_boxes(hm_ctx *ctx, int level, int *n_colors);

/*
 * Algorithm 4.1, sampling step of one level: draw the colour-masked Gaussian
 * test matrices Omega_l and Psi_l (identity blocks for HM_LEVEL_LEAF) and store
 * Y = A Omega_l and Z = A^* Psi_l (not yet peeled) in the context.
 * Requires hm_color(level) first.  In the two mixed-precision modes the
 * built-in kernel operator computes only the rows the method reads: for
 * every colour c, the rows I_alpha of its pairs (alpha, beta) (the sample
 * tiles, Section 4.1.2); the other rows of the stored samples are unspecified.
 */
hm_status hm_sample(hm_ctx *ctx, const hm_op *op, int level);
/* Errors of hm_sample: HM_EINVAL (null ctx or op, null callback or dense
 * matrix, level out of range), HM_ESTATE (no tree, or the level not coloured),
 * HM_EOP (the callback failed), HM_ETIMEOUT, HM_ENOMEM, HM_ECUDA. */

/*
 * Algorithm 4.1: the whole compression (colour, sample, peel, bases, cores for
 * levels 2..L, then the leaf blocks).  Truncation of qr(Y, k) (Section 2.4):
 *   tol > 0, rank == 0: k = #{|R_jj| > tol |R_11|}, at most r - p;
 *   tol > 0, rank > 0:  the same, at most min(r - p, rank);
 *   tol == 0, rank > 0: fixed rank k = rank (<= r);
 *   both 0:             hm_config's tol and rank, by the same rules.
 * k never exceeds min(|I_alpha|, |I_beta|).  Requires hm_tree_build; the
 * factors stay in the context for hm_apply / hm_relerr / hm_export.  Errors:
 * HM_EINVAL (null ctx or op, null callback or dense matrix, unknown kernel,
 * tol < 0 or NaN, rank < 0 or > r, no tolerance and no rank, or with tol > 0
 * p not in 0..r-1), HM_ESTATE (no tree), HM_EOP (the callback failed; the
 * context stays usable), HM_ETIMEOUT (a bounded wait of the tensor-core
 * sampler expired), HM_ENOTSUP (r x k or r x columns beyond shared memory),
 * HM_ENOMEM, HM_ECUDA.
 */
hm_status hm_compress(hm_ctx *ctx, const hm_op *op, double tol, int rank);

/*
 * Section 4.1.2 (level-truncated product over every level, plus the leaf
 * blocks): y = A~ x (trans = 0) or A~^* x (trans = 1) with the compressed
 * operator; x_dev, y_dev device, column-major n x nrhs (1 <= nrhs <= 64),
 * original order.  Asynchronous on the context's stream: y_dev is complete
 * when that stream reaches this point.  Every factor is read once per block
 * of 4 right-hand sides.  Errors: HM_EINVAL (null ctx or vectors, nrhs out of
 * range), HM_ESTATE (not compressed), HM_ENOMEM, HM_ECUDA.
 */
hm_status hm_apply(hm_ctx *ctx, const double *x_dev, double *y_dev, int64_t nrhs, int trans);

/*
 * Section 5: E = ||A~ - A|| / ||A|| by `iters` power iterations (20 in the
 * paper) on both operators from one Philox Gaussian start vector; *err (host)
 * receives E.  Errors: HM_EINVAL (null ctx, op or err, iters < 1), HM_ESTATE
 * (not compressed), HM_EOP, HM_ENOMEM, HM_ECUDA.
 */
hm_status hm_relerr(hm_ctx *ctx, const hm_op *op, int iters, double *err);

/*
 * Counters of the last hm_compress (Section 5's four quantities: time,
 * matvec columns, error inputs, storage) copied into *out (host).  Valid at
 * any stage (zeros before a compression).  Errors: HM_EINVAL (null ctx or out).
 */
hm_status hm_get_info(hm_ctx *ctx, hm_info *out);

/* Export selectors for hm_export (structure and numbers, for tests). */
enum {
    HM_X_PERM = 1,        /* int32[n]: original index of each sorted point */
    HM_X_LEVEL_BOXES = 2, /* int32[nb][8] of level `level`: start, end, a0, a1, a2, parent, leaf, gid */
    HM_X_CUT = 3,         /* int32[nc][2] of cut `level`: box level, index within level */
    HM_X_NEAR = 4,        /* int32: nc+1 CSR pointers then indices (cut `level`) */
    HM_X_INTER = 5,       /* int32: nc+1 CSR pointers then indices */
    HM_X_PAIR_VERTEX = 6, /* int32[n_pairs] (cut `level` or HM_LEVEL_LEAF) */
    HM_X_VERTEX_COLOR = 7,/* int32[n_vertices] */
    HM_X_VERTEX_BETA = 8, /* int32[n_vertices] */
    HM_X_GAUSS = 9,       /* double[2][n][r]: Omega-side then Psi-side G, sorted order */
    HM_X_SAMPLE_Y = 10,   /* double[chi][n][r']: colour-major, sorted order (r' = r or m_max);
                             rows outside the colour's tiles: see hm_sample */
    HM_X_SAMPLE_Z = 11,   /* double[chi][n][r] */
    HM_X_PAIR_RANKS = 12, /* int32[n_pairs][2]: k_U, k_V */
    HM_X_FACTORS = 13,    /* double: U arena, V arena, B arena concatenated */
    HM_X_FACTOR_OFFS = 14,/* int64[n_pairs][3]: offsets of U, V, B in their arenas */
    HM_X_LEAF_D = 15,     /* double: leaf blocks, row-major |I_a| x |I_b| per neighbour pair */
    HM_X_VERTEX_DEGREE = 16,/* int32[n_vertices] */
    HM_X_BOX_VERTEX_BOX = 17, /* int32[n_box_vertices]: cut entry of every vertex of the
                                 uniform H^1 box graph of cut `level` (hm_color_boxes) */
    HM_X_BOX_COLOR = 18,    /* int32[n_box_vertices]: its colour */
    HM_X_BOX_DEGREE = 19,   /* int32[n_box_vertices]: its degree */
    HM_X_H2_RANKS = 20,     /* int32[2][nc] of cut `level` (HM_FORMAT_H2): k of the column
                               basis of every entry, then of its row basis (0: none) */
    HM_X_H2_SIGMA = 21      /* double[nc][2][r]: S^in then S^out of every entry (the
                               first k valid) */
};

/*
 * Copy an exported array to host memory.  With host_buf == NULL only *bytes is
 * set to the size needed; otherwise *bytes must be at least that size.
 * Errors: HM_EINVAL (null ctx or bytes, unknown selector, level out of range,
 * buffer too small), HM_ESTATE (no tree, or the requested part not built, or
 * samples not kept: hm_config.keep_samples), HM_ECUDA.
 */
hm_status hm_export(hm_ctx *ctx, int what, int level, void *host_buf, size_t *bytes);

/*
 * hm_apply_noalloc: hm_apply without any device allocation.  (The paper has no
 * counterpart; this is a library convenience.)  For callers that cannot
 * allocate device memory when they apply the operator -- a serving loop whose
 * process has given all free device memory to another framework's caching
 * allocator, or a latency-critical loop that must not wait on cudaMalloc /
 * cudaFree or risk running out of memory mid-request.  Its scratch (permuted
 * vectors, per-pair intermediate products, offsets, level table) comes from one
 * array of HM_APPLY_NOALLOC_SCRATCH_BYTES inside the library, which every GPU
 * that loads the library holds until the process exits.  A request that needs
 * more returns HM_ENOTSUP (use hm_apply).  The first call on a device looks up
 * that array's address (cudaGetSymbolAddress) and caches it.  The offsets it
 * needs are computed by hm_compress; the call reads nothing back and is
 * asynchronous on the context's stream, like hm_apply.  All calls share the
 * array: calls that overlap on the GPU race.  Arguments, results and the other
 * errors are those of hm_apply.
 */
#define HM_APPLY_NOALLOC_SCRATCH_BYTES (64u << 20)
hm_status hm_apply_noalloc(hm_ctx *ctx, const double *x_dev, double *y_dev, int64_t nrhs, int trans);

/* Human-readable description of the last error on this context. */
const char *hm_last_error(const hm_ctx *ctx);

/* ---------------------------------------------------------------------------
 * Serving (a library service around Algorithm 4.1; the paper has no
 * counterpart).  A server admits compression jobs of differing size,
 * geometry and kernel as device memory and worker slots free up, keeps each
 * finished job's compressed operator resident, and serves matvecs with it.
 *  - Admission: jobs are taken in submission order; a job starts when a worker
 *    slot is free and its estimated peak footprint fits in the byte budget
 *    next to the reservations of the jobs already admitted.  When a job's
 *    compression ends, the samples and Gaussians are freed and its
 *    reservation shrinks to the bytes it keeps (factors, leaf blocks, tree
 *    and apply metadata), so queued jobs can start.
 *  - Concurrency: every job has its own CUDA stream and is compressed by one
 *    of the server's worker threads (hm_compress's colouring also runs ahead
 *    on its own streams), so the work of concurrent jobs overlaps on the GPU.
 *  - Results are those of the same job compressed alone with hm_compress on
 *    the same inputs.
 * The server uses the device current at hm_server_create.
 * ------------------------------------------------------------------------- */
typedef struct hm_server hm_server;

typedef struct {
    size_t hbm_budget;  /* bytes the admitted jobs may reserve; 0 = 85% of the free
                           device memory at hm_server_create */
    int slots;          /* jobs compressed at the same time (worker threads), 1..64 */
} hm_server_config;

typedef struct {
    hm_config cfg;              /* the job's configuration (see hm_create) */
    hm_op op;                   /* its black box; a dense matrix must stay valid and a
                                   callback callable until the job is done */
    const double *points_host;  /* n x d row-major FP64, original order; copied by
                                   hm_server_submit (the caller may free it after) */
    int64_t n;
    int leaf_size;              /* as hm_tree_build (0 = cfg.leaf_size) */
    double tol;                 /* as hm_compress (both 0 = cfg's) */
    int rank;
} hm_job_desc;

enum { HM_JOB_QUEUED = 0, HM_JOB_RUNNING = 1, HM_JOB_READY = 2, HM_JOB_FAILED = 3 };

typedef struct {
    int state;                  /* HM_JOB_* */
    hm_status status;           /* outcome of the compression (HM_OK when ready) */
    double t_submit, t_start, t_done;  /* seconds since the server was created */
    size_t reserved_bytes;      /* the job's current reservation */
    size_t estimate_bytes;      /* its estimated peak footprint (the reservation while
                                   it compresses) */
    hm_info info;               /* hm_get_info of the job after its compression */
} hm_job_stats;

typedef struct {
    int64_t submitted, completed, failed, released, queued, running;
    int max_running;            /* largest number of jobs compressed at the same time */
    size_t budget, reserved, max_reserved;
    double jobs_per_s;          /* completed jobs / (last completion - first submission) */
    double job_p50_s, job_p99_s;      /* submission -> compressed, over completed jobs */
    int64_t applies;
    double apply_p50_s, apply_p99_s;  /* hm_server_apply latency (host, end to end) */
} hm_server_info;

/* Create a server.  Errors: HM_EINVAL (null out or cfg, slots out of range),
 * HM_ENOMEM, HM_ECUDA (no device). */
hm_status hm_server_create(hm_server **out, const hm_server_config *cfg);

/* Queue a job; *job_id receives its id.  Returns at once.  Errors: HM_EINVAL
 * (null pointers, bad configuration or sizes), HM_ENOTSUP (the job's estimated
 * footprint exceeds the whole budget), HM_ENOMEM. */
hm_status hm_server_submit(hm_server *s, const hm_job_desc *job, int64_t *job_id);

/* Wait until the job is ready or failed (at most timeout_s seconds; < 0 waits
 * without limit); *stats (may be NULL) receives its record.  Returns the job's
 * status, HM_ETIMEOUT if it is still queued or running, or HM_EINVAL (unknown
 * or released id). */
hm_status hm_server_wait(hm_server *s, int64_t job_id, double timeout_s, hm_job_stats *stats);

/* y = A~ x (trans = 0) or A~^* x with a ready job's compressed operator, as
 * hm_apply (device pointers, column-major n x nrhs, original order), on the
 * job's stream; returns when y_dev is complete.  Calls on one job are
 * serialised.  Errors: HM_EINVAL (unknown id, bad vectors), HM_ESTATE (job not
 * ready), and those of hm_apply. */
hm_status hm_server_apply(hm_server *s, int64_t job_id, const double *x_dev, double *y_dev, int64_t nrhs,
                          int trans);

/* Free a job (ready or failed) and its reservation.  Errors: HM_EINVAL (unknown
 * id), HM_ESTATE (queued or running). */
hm_status hm_server_release(hm_server *s, int64_t job_id);

/* Counters and latency percentiles since hm_server_create.  Errors: HM_EINVAL. */
hm_status hm_server_get_info(hm_server *s, hm_server_info *out);

/* Stop the workers after the jobs already admitted, drop the queued ones and
 * free every job.  Safe on NULL. */
hm_status hm_server_destroy(hm_server *s);

#ifdef __cplusplus
}
#endif

#endif /* HM_H */
