/*
 * suppy.h -- C ABI of the GB300 (sm_103a) superiorized hyperslab-projection
 * library (libsuppy_gb300.so).
 *
 * The library solves the feasibility problem  l <= A x <= u,  lo <= x <= hi
 * (A sparse, CSR) with the simultaneous (Cimmino-type) or block-iterative
 * projection method, superiorized by nonascending subgradient perturbations of
 * an objective f (isotropic / anisotropic total variation, or a linear mean
 * dose).  Paper: arXiv 2606.27086, "GPU-accelerated superiorization on
 * constrained physical problems with SupPy".
 *
 *   hyperslab projection   Sec. 2.1.1, Eq. (2), taken two-sided:
 *                          P_i x = x + ((clamp(<a_i,x>, l_i, u_i) - <a_i,x>) / ||a_i||^2) a_i
 *   relaxation             Eq. (3): x + lambda (P x - x), lambda in (0, 2)
 *   simultaneous step      Sec. 2.1.1: x <- box(x + lambda sum_i w_i (P_i x - x)),
 *                          w_i = 1/m' over the m' nonzero rows
 *   block-iterative step   Sec. 2.1.1: the same step inside block B_t with
 *                          w_i = 1/|B_t|, blocks in order, box after each block
 *   box projection         Sec. 2.3.3 (BoxProjection after each iteration)
 *   proximity              Eq. (WeightedProximity): 1/2 sum_i w_i ||P_i x - x||^2, w_i = 1/m'
 *   superiorization        Algorithm 1; beta = gamma * alpha^l (Sec. 2.1.2),
 *                          v = -g_f / ||g_f||; trial accepted when f(z) <= f(y)
 *   stopping               Sec. 2.2.1 (P <= P*, relative change of P below dP*
 *                          for N consecutive iterations, N_max) and Sec. 2.2.3
 *                          (relative change of f below df*)
 *   objectives             Eq. (TV) with its Combettes/Penfold subgradient
 *                          (Sec. 2.3.1); anisotropic TV; f_Mean of Sec. 2.3.3;
 *                          the L1 / L2 perturbations of the seismic study
 *   adaptive step          beta = (f - f_ref)/||g_f|| of Nikazad et al. (Sec. 2.1.2)
 *   variance stopping      the CT study's variance of relative changes (Sec. 2.3.2)
 *   DROP, EL, EMR          the appendix table of used methods, in slab form
 *   split feasibility      Eq. (Split) and the CQ iteration after it, with the
 *                          dose-volume constraints of Sec. 2.3.3 as the sets Q_j
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every call returns a suppy_status.  Nothing aborts, traps or prints.  On
 *   failure suppy_last_error(ctx) (or suppy_last_error(NULL) when no context
 *   exists) returns a message; it stays valid until the next call on the same
 *   context / thread.
 * - Pointers flagged "on_device" are CUDA device pointers of the current
 *   device; otherwise they are host pointers (pageable or pinned).  Inputs are
 *   always copied: the caller keeps ownership and may free them after the call
 *   returns (suppy_update_bounds_async: after the next synchronizing call).
 *   Library device memory is owned by the context until suppy_destroy.
 * - All GPU work is enqueued on the context's stream (suppy_create /
 *   suppy_set_stream).  Calls that return host values (proximity, objective,
 *   get_x to host, run statistics, state) synchronize that stream.  A context
 *   is not thread-safe; separate contexts are independent.
 * - B right-hand sides (1 <= B <= 32) share one matrix.  Vectors over the
 *   unknowns are n x B row-major (element (j, b) at j*B + b); vectors over the
 *   constraints (l, u) are m x B row-major (i*B + b).  Per-RHS outputs are
 *   arrays of length B.
 * - Matrix indices are int32 and nnz must stay below 2^31 (SUPPY_EINVAL
 *   otherwise).  Column indices inside a row must be distinct.
 */
#ifndef SUPPY_GB300_H
#define SUPPY_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct suppy_ctx suppy_ctx;

typedef enum {
    SUPPY_OK = 0,
    SUPPY_EINVAL = -1,   /* bad argument, malformed CSR, NaN, l > u, ...         */
    SUPPY_ENOMEM = -2,   /* device or host allocation failed                     */
    SUPPY_ECUDA = -3,    /* a CUDA runtime call failed (message has the details) */
    SUPPY_ETIMEOUT = -4, /* a bounded device-side wait gave up                   */
    SUPPY_ESTATE = -5    /* call not valid in the context's state                */
} suppy_status;

/* Storage type of A's values on the device.  BF16/FP16 are rounded to nearest
 * even from the FP32 input; every accumulation stays FP32 (dot products,
 * corrections) or FP64 (row norms, proximity, objective, acceptance).
 * SUPPY_HALF_AUTO stores 16 bits in the format with the smaller rounding
 * error on this matrix: per entry the error bound is max(2^-11 |v|, 2^-25)
 * for FP16 (its unit roundoff, and half its subnormal spacing) and 2^-8 |v|
 * for BF16; FP16 is taken when no magnitude exceeds 65504 and its bounds,
 * summed in squares over the entries, are at most BF16's, else BF16.
 * suppy_info reports the choice. */
typedef enum { SUPPY_F32 = 0, SUPPY_BF16 = 1, SUPPY_F16 = 2, SUPPY_HALF_AUTO = 3 } suppy_dtype;

/* Feasibility-seeking operator T (Sec. 2.1.1). */
/* SUPPY_CIMMINO: simultaneous projections, w_i = 1/m' (Sec. 2.1.1).
 * SUPPY_BIP: block-iterative, w_i = 1/|B_t| inside block t, box after each block.
 * SUPPY_DROP: diagonally relaxed orthogonal projections (appendix Table of used
 *   methods, in slab form): x <- box(x + lambda Z sum_i (P_i x - x)) with unit
 *   row weights and Z = diag(1/s_j), s_j the stored nonzeros of column j in the
 *   rows with ||a_i|| > 0 (0 for an empty column).  The monitored proximity
 *   keeps the weights 1/m'. */
/* SUPPY_EL: extrapolated Landweber (appendix table of used methods), in slab
 *   form: x <- box(x + lambda t A^T D d), d_i = clamp(r_i, l_i, u_i) - r_i,
 *   D = diag(w_i/||a_i||^2), w_i = 1/m', t = d^T D d / ||A^T D d||^2.
 * SUPPY_EMR: Landweber with error-minimising relaxation (same table), slab
 *   form: x <- box(x + lambda t A^T M d), M = diag(w_i),
 *   t = ||A^T M d||^2 / ||M^(1/2) A A^T M d||^2 (one more pass over A).
 *   Both take the two-pass sweep; a zero correction leaves x unchanged. */
typedef enum {
    SUPPY_CIMMINO = 0,
    SUPPY_BIP = 1,
    SUPPY_DROP = 2,
    SUPPY_EL = 3,
    SUPPY_EMR = 4
} suppy_mode;

/* Objective of the perturbation phase. */
typedef enum {
    SUPPY_OBJ_NONE = 0,     /* feasibility-seeking only                              */
    SUPPY_OBJ_TV_ISO = 1,   /* Eq. (TV) on an img_h x img_w row-major image          */
    SUPPY_OBJ_TV_ANISO = 2, /* sum |x[i+1,j]-x[i,j]| + sum |x[i,j+1]-x[i,j]|         */
    SUPPY_OBJ_LINEAR = 3,   /* f = c.x, e.g. f_Mean = (1/N_S) sum_{i in S} (A_S x)_i */
    SUPPY_OBJ_L1 = 4,       /* f = ||x||_1, subgradient sign(x) (0 at 0)             */
    SUPPY_OBJ_L2 = 5        /* f = ||x||_2^2, gradient 2x (L1 / L2 perturbations of the
                             * seismic study, Sec. 2.3.1)                             */
} suppy_obj;

/* CSR matrix: row_ptr[m+1] (row_ptr[0] = 0, nondecreasing, row_ptr[m] = nnz),
 * col[nnz] in [0, n), val[nnz] finite.  Column order inside a row is free. */
typedef struct {
    int32_t m, n;
    int64_t nnz;
    const int32_t* row_ptr;
    const int32_t* col;
    const float* val;
    int32_t on_device; /* 1: the three arrays are device pointers */
} suppy_csr;

typedef struct {
    suppy_dtype a_dtype;
    suppy_mode mode;
    /* SUPPY_BIP: host array of m block ids in [0, nblocks).  Blocks are swept
     * in increasing id; rows keep their relative order inside a block. */
    const int32_t* block_of_row;
    int32_t nblocks;
    suppy_obj obj;
    int32_t img_h, img_w;     /* TV objectives: img_h * img_w == n; with other
                                 objectives optional (0, 0), the grid of the
                                 unknowns the tiled sweep cuts into tiles */
    /* SUPPY_OBJ_LINEAR: either c_lin (n floats, host) or obj_rows, an
     * objective matrix S whose column means c = S^T 1 / rows(S) are computed
     * on the device at create (f_Mean over the structure S). */
    const float* c_lin;
    const suppy_csr* obj_rows;
    int32_t nrhs;             /* B, 1..32 (0 is read as 1) */
    int64_t box_len;          /* 1: scalar box bounds; n: one bound per unknown */
    int32_t tune;             /* 1: time candidate strategies / launch shapes at create */
    /* Sweep strategy: 0 automatic; 1 one pass over A (row pass with the
     * correction scattered by L2 reductions, or staged in shared memory when
     * n*B*4 bytes fit); 2 two passes (row pass writing the coefficients, then a
     * column pass over a CSC copy of A gathering them -- no atomics, bitwise
     * reproducible, twice the matrix memory); 3 tiled one pass (one
     * right-hand side; Cimmino, BIP or DROP): the unknowns are split into one
     * tile per SM (image rectangles when img_h x img_w is given, column
     * ranges otherwise), each CTA keeps its tile's x and correction in shared
     * memory and streams its tile's segments of A -- runs of a row's entries
     * in the tile, with 16-bit tile-local indices -- once per sweep; the dot
     * products of a row are combined across tiles by L2 reductions, chunk by
     * chunk.  Strategy 3 gives SUPPY_EINVAL when the problem does not fit it
     * (a tile above 8192 unknowns, several right-hand sides, EL / EMR); with
     * tune set and strategy 0 it is one of the timed candidates. */
    int32_t strategy;
    /* Streaming of A through shared memory by bulk asynchronous copies (TMA)
     * for one right-hand side: 0 automatic (used when eligible), -1 off. */
    int32_t tma;
    /* Launch shape of the streaming passes, 0 = automatic (or measured when
     * tune is set): ring tile length in elements (a power of two, 256..4096),
     * ring stages (2..32, within the shared-memory budget) and lanes per item
     * (4, 8, 16 or 32).  Values outside these ranges give SUPPY_EINVAL; a shape
     * whose ring window cannot hold a warp's items leaves streaming off. */
    int32_t stream_tile, stream_stages, stream_lanes;
    /* Perturbation phase: 2 -- the whole phase on the whole GPU in one
     * cooperative launch (subgradient pass, passes evaluating up to eight
     * consecutive trial step sizes at once with the first accepted one
     * applied -- the same choice as the sequential trial loop -- and grid
     * barriers between passes; several right-hand sides one after the
     * other); 1 -- one thread-block cluster per right-hand side; 0 --
     * automatic: 2 for one right-hand side with n >= 65536, else 1. */
    int32_t perturb_path;
    /* Lane map of the streaming passes: 0 automatic (measured when tune is
     * set), 1 four consecutive elements per lane (16-byte ring reads),
     * 2 lane-interleaved elements (lane k of a group takes elements k, k + G,
     * k + 2G, ...: one gather instruction reads G consecutive elements of an
     * item).  Other values give SUPPY_EINVAL. */
    int32_t stream_map;
    /* Tiled sweep (strategy 3): warps of its dot-product phase (0 automatic
     * = 10, else 1..25; of the 32 warps of a CTA one streams A, one watches
     * the grid counters, four compute the correction coefficients and the
     * other 26 - tile_warps1 scatter the corrections).  Other values give
     * SUPPY_EINVAL. */
    int32_t tile_warps1;
    /* Tiled sweep: stream bytes per tile and chunk aimed at (0 automatic =
     * 16384; smaller values give more chunks) and a fixed ring (0 automatic =
     * up to 24 copies of 8 KB in the shared memory left; else 8 copies of
     * tile_ring_bytes / 8 bytes, a power of two in [256, 8192]). */
    int32_t tile_chunk_bytes, tile_ring_bytes;
    /* Tiled sweep: consecutive rows kept together when rows are dealt to
     * chunks (0 automatic = 1, else 1..1024): neighbouring rays share a slice
     * and read neighbouring columns at each step, while fewer rows per group
     * even out the tiles' shares of a chunk. */
    int32_t tile_group_rows;
    /* Lane map of the column pass of the two-pass sweep alone: 0 the same
     * as stream_map, else 1 or 2 as there (with stream_map and a fixed
     * stream shape, a configuration the tuner chose can be rebuilt without
     * timing, e.g. under a profiler).  Other values give SUPPY_EINVAL. */
    int32_t stream_col_map;
    /* Rows of A that run down the image (on an image grid img_h x img_w = n,
     * one right-hand side; a row that spans more image rows than columns)
     * handled in the column-major pixel numbering, where their consecutive
     * entries are neighbours.  One-pass sweep with L2-reduction scatter:
     * they add their corrections into a second, column-major accumulator
     * (fewer reduction requests), which the box step adds.  Two-pass sweep:
     * their stored indices are column-major (a second copy of the packed
     * indices, 4 bytes per stored entry) and their gathers read a
     * column-major copy of x made before each row pass.  The same sums in
     * another addition order.  2: the patch numbering for the one-pass
     * sweep.  The image, zero-padded to multiples of 8, is laid out in
     * patches: the rows closer to the horizontal use wide patches (128-byte
     * lines of 8 x 4 pixels made of 32-byte sectors of 4 x 2), the others
     * tall ones (lines of 4 x 8, sectors of 2 x 4).  Every row's indices are
     * stored as patch positions (a second copy of the packed indices, 4 bytes
     * per stored entry), its gathers read x from a copy in its layout (both
     * copies made at each sweep start -- in suppy_run by the whole-GPU
     * perturbation phase before the sweep -- and written by each block's box
     * step),
     * and its corrections go into an accumulator in the same layout, so that
     * a warp's gathers and reductions along a slanted ray touch fewer
     * sectors; the two-pass sweep takes 2 as 1.  0 automatic (the patch
     * numbering for the one-pass sweep when eligible, none for the two-pass
     * sweep; every form timed when tune is set), 1 on (SUPPY_EINVAL when
     * there is no image grid or several right-hand sides), -1 off.  Other
     * values give SUPPY_EINVAL. */
    int32_t scatter_transpose;
} suppy_opts;

/* Parameters of Algorithm 1 and of the stopping rule.  suppy_params_default
 * fills the paper's stopping defaults (P* = 1e-6, dP* = 1e-8, N = 5,
 * N_max = 500, df* = 1e-6), lambda = 1, gamma = 0.5, alpha = 0.99, n_red = 1,
 * max_trials = 100, check_every = 10, use_graphs = 1. */
typedef struct {
    double lambda;          /* relaxation, (0, 2)                                  */
    double gamma, alpha;    /* beta = gamma * alpha^l                              */
    int32_t n_red;          /* accepted reduction steps per perturbation phase     */
    int32_t max_trials;     /* trials per reduction step before the phase ends     */
    int32_t restart_every;  /* 0: no restarts; else l <- r after the r-th restart  */
    int32_t max_sweeps;     /* N_max                                               */
    int32_t check_every;    /* host polls the stop flags every this many sweeps    */
    double prox_abs;        /* P*                                                  */
    double prox_rel;        /* dP*                                                 */
    double obj_rel;         /* df*; <= 0 disables the objective criterion          */
    int32_t patience;       /* N                                                   */
    int32_t use_stopping;   /* 0: run exactly max_sweeps sweeps                    */
    int32_t use_graphs;     /* 1: suppy_run replays one captured iteration (CUDA graph) */
    /* > 0: the variance stopping rule of the CT study (Sec. 2.3.2): a right-hand
     * side stops after iteration k >= 2 once the sample variance of the
     * relative changes ||x^i - x^(i-1)|| / ||x^i||, i = 1..k, of its iterates
     * (since the last set_x / set_bounds / reset) is below variance_tol.  Applies
     * in suppy_run, whatever use_stopping says; 0 disables it. */
    double variance_tol;
    /* Step size of the perturbations: 0 the power law beta = gamma alpha^l;
     * 1 the adaptive step of Nikazad et al. (Sec. 2.1.2), beta = (f(y) -
     * f_ref)/||g|| when f(y) > f_ref and no step otherwise, with f_ref the
     * lowest objective value at the start of a perturbation phase so far (this
     * phase's included; reset by set_x / set_bounds); 2 the same with f_ref
     * fixed to the field below.  With 1 or 2 each reduction step takes this one
     * trial and keeps it when f(z) <= f(y); l and max_trials are not used. */
    int32_t adaptive;
    int32_t reserved;       /* 0                                                   */
    double f_ref;           /* the reference value when adaptive = 2 (finite)      */
} suppy_params;

typedef struct {
    int32_t sweeps;     /* sweeps applied to this right-hand side            */
    int32_t accepted;   /* accepted perturbation steps, total                */
    int32_t trials;     /* perturbation trials, total                        */
    int32_t stopped;    /* 1 when the stopping rule ended this RHS           */
    int64_t ell;        /* current power-law exponent l                      */
    double proximity;   /* monitored proximity of the last sweep             */
    double objective;   /* f(x^k) at the start of the last perturbation      */
} suppy_stats;

typedef struct {
    int32_t m, n, nrhs, m_kept;   /* m_kept = m' (rows with ||a_i|| > 0)     */
    int64_t nnz, nnz_csc;         /* nnz_csc: entries of the CSC copy (two passes) */
    int32_t nblocks;
    int32_t lanes_per_row;        /* launch shape chosen for the sweep       */
    int32_t elems_in_regs;        /* row elements a lane holds between dot and scatter */
    int32_t grid;                 /* CTAs of the sweep launch                */
    int32_t block;                /* threads per CTA of the sweep launch     */
    int32_t perturb_cluster;      /* CTAs per cluster of the perturbation    */
    int64_t device_bytes;         /* device memory held by the context       */
    int32_t strategy;             /* 1 one pass, 2 two passes, 3 tiled one pass */
    int32_t scatter;              /* one pass: 1 L2 reductions, 2 shared-memory staged */
    int32_t col_lanes;            /* two passes: lanes per column            */
    int32_t col_grid;             /* two passes: CTAs of the column pass     */
    int32_t tma;                  /* 1: the sweep streams A by bulk copies   */
    int32_t tile, stages;         /* streaming row pass: ring tile length (elements), stages */
    int32_t col_tile, col_stages; /* streaming column pass: the same       */
    int32_t map, col_map;         /* streaming lane maps (opts.stream_map: 1 or 2) */
    /* tiled sweep (strategy 3): tiles (= CTAs), chunks, warps of the dot
     * products, of the scatter and of the coefficients, ring bytes, bytes and
     * segments of the tile streams; zero for the other strategies */
    int32_t tiles, chunks, tile_warps1, tile_warps2, tile_coef_warps, tile_ring;
    int64_t tile_stream_bytes, tile_segments;
    /* rows handled column-major (opts.scatter_transpose); 0 when the sweep
     * does not use that form */
    int64_t transposed_rows;
    int32_t a_dtype;              /* storage type of A's values (HALF_AUTO resolved) */
    int32_t scatter_patch;        /* 1: the one-pass sweep uses the patch numbering */
} suppy_info;

/* Fill *p with the defaults listed above. */
void suppy_params_default(suppy_params* p);

/* Create a context: copy A, l, u and the box into library-owned device
 * memory, validate them, and run the setup step -- FP64 row norms
 * ||a_i||^2 (the denominator of Eq. (2)), weights w_i (1/m' or 1/|B_t|), the
 * zero-row drop (a row with ||a_i|| = 0 needs l_i <= 0 <= u_i, else
 * SUPPY_EINVAL), conversion of A's values to opts->a_dtype, the block
 * permutation and the launch partition.
 *   A        CSR of the constraint rows; A->on_device selects host/device for
 *            A, l, u, box_lo, box_hi and opts->c_lin alike.
 *   l, u     m x B, +-INFINITY allowed, no NaN, l <= u.
 *   box_lo, box_hi  opts->box_len values each (1 or n); -INF/+INF allowed.
 *   stream   cudaStream_t to enqueue on (NULL: the legacy default stream).
 * The initial point is x = box(0) for every right-hand side.  On success
 * *out receives the context; on failure *out is NULL and nothing is leaked. */
suppy_status suppy_create(const suppy_csr* A, const float* l, const float* u,
                          const float* box_lo, const float* box_hi, const suppy_opts* opts,
                          void* stream, suppy_ctx** out);

/* Release every resource of the context (NULL is a no-op).  Synchronizes the
 * context's stream first. */
void suppy_destroy(suppy_ctx* ctx);

/* Enqueue later work on another stream. */
suppy_status suppy_set_stream(suppy_ctx* ctx, void* stream);

/* Replace the slab bounds (m x B each, same rules as at create) -- e.g. a new
 * sinogram over the same geometry.  Resets iteration counters, exponents,
 * histories and stop flags, keeps x. */
suppy_status suppy_set_bounds(suppy_ctx* ctx, const float* l, const float* u, int32_t on_device);

/* Replace the slab bounds like suppy_set_bounds, but keep x and the iteration
 * state (exponent l, counters, histories, stop flags): Algorithm 1 continues
 * warm on the new bounds -- e.g. successive measurements of a slowly changing
 * object.  A rejected call (SUPPY_EINVAL) leaves the old bounds. */
suppy_status suppy_update_bounds(suppy_ctx* ctx, const float* l, const float* u, int32_t on_device);

/* suppy_update_bounds without its synchronization: the copies, checks and
 * the swap are enqueued on the context's stream and the call returns.  A
 * rejected set (NaN, l > u, a zero row whose slab excludes 0) is skipped on
 * the device, so the old bounds stay, and it is reported (SUPPY_EINVAL) by the
 * next call that synchronizes with the results: suppy_get_x into host memory
 * or suppy_run with statistics.  Host arrays must stay unchanged until then
 * (pinned host memory lets the copy overlap). */
suppy_status suppy_update_bounds_async(suppy_ctx* ctx, const float* l, const float* u,
                                       int32_t on_device);

/* Set x (n x B) and project it onto the box.  Resets iteration counters,
 * exponents, histories and stop flags. */
suppy_status suppy_set_x(suppy_ctx* ctx, const float* x, int32_t on_device);

/* Copy x (n x B) out.  A host copy synchronizes the stream. */
suppy_status suppy_get_x(suppy_ctx* ctx, float* x, int32_t on_device);

/* One perturbation phase of Algorithm 1 on every active right-hand side:
 * up to n_red accepted steps z = y - beta g/||g||, beta = gamma alpha^l, l
 * advanced at every trial, accepted when f(z) <= f(y) in FP64; the phase
 * ends early when ||g|| = 0 or max_trials trials in a row are rejected.
 * Restarts (Sec. 2.1.2) apply when the sweep count is a positive multiple
 * of restart_every.  accepted (host, B entries) may be NULL; when given the
 * call synchronizes and writes the accepted steps of this phase.
 * SUPPY_ESTATE when the context has no objective. */
suppy_status suppy_perturb(suppy_ctx* ctx, const suppy_params* p, int32_t* accepted);

/* Apply the feasibility-seeking operator T nsweeps times (no perturbation):
 * Cimmino -- x <- box(x + lambda sum_i w_i (P_i x - x)), by the strategy
 * chosen at create (one pass over A scattering the corrections, then the box
 * kernel; or a row pass writing the coefficients and a column pass over the
 * CSC copy applying the sum and the box); BIP -- the same per block, the box
 * after each block; DROP, EL and EMR -- their steps (suppy_mode).  With
 * dose-volume constraints (suppy_set_dvc) each sweep starts with the CQ step.
 * Each sweep records the monitored proximity (Cimmino: P at the sweep's input
 * point; BIP: the sum of each block's terms at that block's input point;
 * split problems: the target-space proximity) and advances the stopping rule
 * when p->use_stopping is set.  Asynchronous. */
suppy_status suppy_sweep(suppy_ctx* ctx, const suppy_params* p, int32_t nsweeps);

/* Eq. (WeightedProximity) at the current x, w_i = 1/m', FP64, deterministic:
 * out[b] for each right-hand side (host, B entries).  Synchronizes. */
suppy_status suppy_proximity(suppy_ctx* ctx, double* out);

/* f(x) at the current x, FP64, deterministic; out[b] (host, B entries).
 * Synchronizes.  SUPPY_ESTATE when the context has no objective. */
suppy_status suppy_objective(suppy_ctx* ctx, double* out);

/* Algorithm 1: repeat [perturbation phase (when an objective is set), one
 * sweep] until the stopping rule holds for every right-hand side or
 * max_sweeps sweeps ran.  Sweeps of a stopped right-hand side are skipped
 * on the device.  out (host, B entries) may be NULL.  Synchronizes at the
 * end and every check_every sweeps when use_stopping is set.  With out NULL
 * and use_stopping 0 the call only enqueues the iterations on the context's
 * stream and returns; a device-side wait that gave up is then reported
 * (SUPPY_ETIMEOUT) by the next call that synchronizes (suppy_get_x into host
 * memory, suppy_run with out, suppy_proximity, ...). */
suppy_status suppy_run(suppy_ctx* ctx, const suppy_params* p, suppy_stats* out);

/* Copy the per-sweep history of right-hand side rhs: prox[k] (monitored
 * proximity of sweep k) and obj[k] (f(x^k), NaN when no objective), up to cap
 * entries each; *count receives the number of recorded sweeps (which may
 * exceed cap).  Either array may be NULL.  Synchronizes. */
suppy_status suppy_history(suppy_ctx* ctx, int32_t rhs, double* prox, double* obj, int32_t cap,
                           int32_t* count);

/* Checkpoint: serialise x and the per-RHS iteration state (exponent l,
 * restart count, sweep count, stopping state) into buf.  With buf NULL, *len
 * receives the size needed.  Synchronizes. */
suppy_status suppy_get_state(suppy_ctx* ctx, void* buf, size_t* len);

/* Restore a checkpoint written by suppy_get_state for the same shapes. */
suppy_status suppy_set_state(suppy_ctx* ctx, const void* buf, size_t len);

/* Sizes and launch shapes of the context. */
suppy_status suppy_info_get(const suppy_ctx* ctx, suppy_info* out);

/* ---------------------------------------------------------------------------
 * Split feasibility with dose-volume constraints (Eq. (Split) and the CQ
 * iteration printed after it, Sec. 2.1.1; dose-volume constraints of
 * Sec. 2.3.3).  The hyperslabs of the context are the input-space sets C_k;
 * the dose-volume sets Q_j live in the dose space of the rows A_q. */
typedef enum { SUPPY_DVC_UPPER = 0, SUPPY_DVC_LOWER = 1 } suppy_dvc_kind;

typedef struct {
    int32_t kind;       /* SUPPY_DVC_UPPER: D_V <= d_ref, at most K = floor(V N) of
                           the structure's N voxels above d_ref; SUPPY_DVC_LOWER:
                           D_V >= d_ref, at least K = ceil(V N) voxels at or above
                           d_ref (V N is one double multiplication)              */
    int32_t structure;  /* index of the structure (row range of A_q)             */
    double volume;      /* V, the volume fraction, in [0, 1]                     */
    double d_ref;       /* reference dose, finite                                */
} suppy_dvc;

/* Attach the dose-volume sets of a split-feasibility problem.
 *
 * Aq: the dose rows (m_q x n, n the context's n) of the structures that carry
 * DVCs, grouped by structure: rows structure_ptr[s] .. structure_ptr[s+1]-1
 * (host array of nstruct + 1 entries, structure_ptr[0] = 0, nondecreasing,
 * structure_ptr[nstruct] = m_q) are structure s.  Values are kept in FP32
 * whatever the context's a_dtype.  dvc: ndvc constraints (host).  relax in
 * (0, 2) sets gamma = relax / L*, L* = sum_j w_j ||A_j||_F^2 with w_j = 1/ndvc
 * and A_j the rows of DVC j's structure (the Frobenius bound of the paper's
 * step-size rule).
 *
 * Afterwards every sweep (suppy_sweep, suppy_run, captured graphs) starts with
 * the CQ step x <- x + gamma sum_j w_j A_j^T (P_Qj(A_j x) - A_j x), where
 * P_Qj keeps (upper) or raises to d_ref (lower) the K highest doses of the
 * structure and lowers (upper) the other doses above d_ref to d_ref, equal
 * doses ranked by row; the feasibility sweep over the hyperslabs (P_C) and
 * the box follow.  The monitored proximity (history, stopping rule, stats)
 * becomes the target-space proximity 1/2 sum_j w_j ||P_Qj(A_j x) - A_j x||^2
 * at the CQ step's input point (Sec. 2.2.1: stopping on the target space).
 *
 * With several right-hand sides every one gets the same sets and its own CQ
 * step (each its own doses, projections and target-space proximity).
 * Copies its inputs (device inputs when Aq->on_device);
 * synchronizes; replaces an earlier set; ndvc = 0 removes the sets.
 * SUPPY_EINVAL for a malformed matrix (row_ptr, col range, NaN or
 * infinite values), bad structure ranges, kinds, structures, volumes or d_ref,
 * relax outside (0, 2), or zero rows in every constrained structure. */
suppy_status suppy_set_dvc(suppy_ctx* ctx, const suppy_csr* Aq, const int32_t* structure_ptr,
                           int32_t nstruct, const suppy_dvc* dvc, int32_t ndvc, double relax);

/* Doses d = A_q x at the current x (m_q x B floats, row-major like x: right-
 * hand side b's dose of row i at dose[i * B + b]; FP32 accumulation) into
 * host or device memory.  A host copy synchronizes.  SUPPY_ESTATE without
 * DVCs. */
suppy_status suppy_dvc_dose(suppy_ctx* ctx, float* dose, int32_t on_device);

/* Target-space proximity 1/2 sum_j w_j ||P_Qj(A_j x) - A_j x||^2 at the current
 * x (FP64, host; out receives B values, one per right-hand side).
 * Synchronizes.  SUPPY_ESTATE without DVCs. */
suppy_status suppy_dvc_proximity(suppy_ctx* ctx, double* out);

/* Kernel timing for measurement: when enabled, every launch of the kernels
 * below is bracketed by CUDA events on the context's stream.
 * suppy_kernel_time(kind) returns the summed event time (ms) and the launch
 * count since timing was enabled, and synchronizes.  kind: 0 the row pass
 * (the fused one-pass sweep, the row pass of the two-pass sweep, or the whole
 * tiled sweep); 1 the
 * box step (finalize kernel, or the column pass of the two-pass sweep); 2 the
 * perturbation phase; 3 the CQ step of a split problem (all its launches). */
suppy_status suppy_timing_enable(suppy_ctx* ctx, int32_t enable);
suppy_status suppy_kernel_time(suppy_ctx* ctx, int32_t kind, double* total_ms, int64_t* launches);

/* Budget of every bounded device-side wait of this context's kernels (ring
 * stages of the streamed passes, chunk counters of the tiled sweep, grid
 * barriers of the whole-GPU perturbation phase), in SM clock cycles; 0
 * restores the default (4e9 cycles, about two seconds).  A wait that runs out
 * makes its kernel stop and the next synchronizing call return SUPPY_ETIMEOUT,
 * after which the context's synchronisation words are reset and the context
 * stays usable.  A diagnostic knob (no paper counterpart): a short budget lets
 * a test exercise that path.  Negative values give SUPPY_EINVAL. */
suppy_status suppy_set_wait_limit(suppy_ctx* ctx, int64_t cycles);

/* One simultaneous sweep on caller-provided device buffers, allocating
 * nothing.  The paper has no counterpart: this is an integration entry point
 * for callers that cannot allocate device memory where they need a sweep
 * (an allocator that forbids cudaMalloc after start-up, a fixed memory pool
 * they own, or a loop that must not take the implicit synchronization of
 * cudaMalloc/cudaFree).  It computes, for the rows with ||a_i|| > 0,
 *   x <- clamp(x + lambda * weight * sum_i ((clamp(r_i, l_i, u_i) - r_i) / ||a_i||^2) a_i, lo, hi)
 * with r = A x (FP32) and ||a_i||^2 in FP64, and writes 1/2 weight sum_i
 * d_i^2 / ||a_i||^2 at the input point to *proximity (a device double; NULL
 * to skip).  weight = 1/m' gives the equal-weight step of suppy_sweep.
 * Bounds with a NaN or l_i > u_i, or a row with ||a_i|| = 0 whose slab
 * excludes 0, are found on the device (the call does not synchronize): x is
 * then left unchanged and *proximity is set to NaN.
 *   A            CSR with on_device = 1; l, u (m), box_lo, box_hi (box_len =
 *                1 or n) and x (n, updated in place) are device pointers.
 *   stream       cudaStream_t the kernels are enqueued on; asynchronous.
 * Its scratch (correction accumulator, per-CTA partials, a validity word) is
 * a static device array of 4 MiB + 16.25 KiB that every GPU loading the library holds
 * until exit; n above 1048576 is rejected with SUPPY_EINVAL.  Every call on a
 * device shares that array (each call clears what must start at zero), so
 * calls that can overlap on the GPU race.  The first call on a device looks
 * up the array's device address (cudaGetSymbolAddress): make that first
 * call before any stream capture.  Errors: SUPPY_EINVAL for bad arguments,
 * SUPPY_ECUDA for a failed lookup or launch; messages via
 * suppy_last_error(NULL). */
suppy_status suppy_sweep_static(const suppy_csr* A, const float* l, const float* u, float weight,
                                float lambda, const float* box_lo, const float* box_hi,
                                int64_t box_len, float* x, double* proximity, void* stream);

/* ---- Serving: continuous batching of many solves on one GPU --------------
 *
 * The paper runs one solve at a time; this runtime has no counterpart there.
 * A server holds registered matrices (CT geometries, seismic geometries,
 * radiotherapy plans) and serves requests -- one set of slab bounds l, u for
 * a registered matrix each -- through batched contexts: every context holds
 * one matrix resident and up to `slots` right-hand sides, each a request with
 * its own iterate, bounds, exponent l and stopping state on the device.  A
 * request waiting for its matrix takes a free slot as soon as one exists, or
 * a new context when the device-memory budget allows one; a finished request
 * leaves its slot at the next poll.  Contexts run on their own CUDA streams,
 * so the work of different matrices overlaps on the device.  Each request
 * runs Algorithm 1 with the matrix's parameters until the stopping rule holds
 * for it (p->use_stopping) or p->max_sweeps sweeps ran.  The result of a
 * request does not depend on the other requests in its context (every
 * right-hand side is computed independently).  Not thread-safe: one host
 * thread drives a server. */
typedef struct suppy_server suppy_server;

typedef struct {
    int64_t hbm_budget;      /* device bytes all contexts may hold; 0: 80% of the free memory */
    int32_t slots;           /* right-hand sides per context, 1..32 (0: 32)                   */
    int32_t check_every;     /* iterations enqueued per context between polls (0: 8)          */
} suppy_server_opts;

typedef struct {
    int32_t state;           /* 0 waiting, 1 running, 2 done                                   */
    int32_t sweeps, accepted, trials;
    double proximity;        /* monitored proximity of the last sweep                          */
    double objective;        /* f at the start of the last perturbation phase                  */
    double t_submit, t_start, t_done;   /* seconds on the server clock (suppy_server_clock)    */
} suppy_request_info;

/* Create a server.  Errors: SUPPY_EINVAL (bad options), SUPPY_ECUDA. */
suppy_status suppy_server_create(const suppy_server_opts* o, suppy_server** out);

/* Release every context and buffer of the server (NULL is a no-op). */
void suppy_server_destroy(suppy_server* srv);

/* Register a matrix with its box (o->box_len values each), context options
 * (value type, mode, blocks, objective; nrhs is the server's slot count) and
 * Algorithm 1 parameters.  Host arrays only (A->on_device = 0); they are
 * copied.  Nothing is put on the device until a request needs it. */
suppy_status suppy_server_add_matrix(suppy_server* srv, const suppy_csr* A, const float* box_lo,
                                     const float* box_hi, const suppy_opts* o,
                                     const suppy_params* p, int32_t* matrix_id);

/* Queue a request: slab bounds l, u (host, m values each, the matrix's row
 * order; same rules as suppy_create), copied.  *request_id identifies it. */
suppy_status suppy_server_submit(suppy_server* srv, int32_t matrix_id, const float* l,
                                 const float* u, int64_t* request_id);

/* One scheduling round, without blocking on the device: retire requests
 * whose contexts finished their last chunk (copying their x out), admit
 * waiting requests into free slots or new contexts, and enqueue the next
 * chunk of iterations on every idle context with running requests.
 * running / waiting (may be NULL) receive the counts after the round. */
suppy_status suppy_server_step(suppy_server* srv, int32_t* running, int32_t* waiting);

/* State of a request; x (host, n values, may be NULL) receives the solution
 * once the request is done.  SUPPY_EINVAL for an unknown id. */
suppy_status suppy_server_query(suppy_server* srv, int64_t request_id, suppy_request_info* info,
                                float* x);

/* Seconds since the server was created (monotonic clock). */
double suppy_server_clock(const suppy_server* srv);

/* Device bytes the server's contexts and buffers hold now. */
int64_t suppy_server_device_bytes(const suppy_server* srv);

/* Message of the last failed server call. */
const char* suppy_server_last_error(const suppy_server* srv);

/* Number of kernels the library launched on this context so far. */
int64_t suppy_launch_count(const suppy_ctx* ctx);

/* Message of the last failed call on ctx (ctx NULL: of this thread's last
 * failed call that had no context). */
const char* suppy_last_error(const suppy_ctx* ctx);

/* Library version string. */
const char* suppy_version(void);

#ifdef __cplusplus
}
#endif
#endif /* SUPPY_GB300_H */
