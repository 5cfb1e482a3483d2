// Shared declarations of the suppy GB300 library (device structs, launch
// entry points between translation units, small device helpers).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "suppy.h"

namespace suppy {

constexpr int kSweepThreads = 256;     // threads per CTA of the sweep kernels
constexpr int kFinalizeThreads = 256;
constexpr int kPerturbThreads = 512;   // threads per CTA of the perturbation cluster
constexpr int kMaxRhs = 32;
// Default budget of one bounded device-side wait: about two seconds of SM clock.
constexpr long long kDefaultWaitCycles = 4000000000LL;

// Per right-hand-side iteration state, resident on the device so that the
// perturbation, sweep and stopping logic never wait for the host.
struct RhsState {
    long long ell;          // power-law exponent l of beta = gamma * alpha^l
    int restarts;           // restarts applied so far
    int last_restart_k;     // sweep index of the last restart (-1: none)
    int k;                  // sweeps applied
    int stopped;            // stopping rule fired (or padding RHS)
    int calm;               // consecutive sweeps with small relative proximity change
    int accepted_total, trials_total;
    int accepted_last, trials_last;
    int has_prev_p, has_prev_f, f_valid;
    int pad0;
    double p_prev, f_prev, f_cur;
    double p_acc;           // running monitored proximity within a block-iterative sweep
    double last_prox;
    double w_s1, w_s2;      // variance rule: sums of the relative changes and their squares
    int w_n;                // relative changes recorded
    int has_ref;            // adaptive step: f_ref holds a phase-start objective
    double f_ref;           // adaptive step: lowest objective at a phase start so far
};

struct StopParams {
    double prox_abs, prox_rel, obj_rel;
    int patience;
    int use_stopping;
    int has_obj;
    int max_sweeps;         // > 0: a right-hand side also stops after this many sweeps
};

// One launch of the row pass over rows [part[0], part[ngroups]).
struct SweepArgs {
    const int2* rinfo;      // per row: {start, length}
    const int* col;         // column indices
    const void* val;        // values (float / bf16 / half)
    const float* l;         // m x B bounds (device row order)
    const float* u;
    const float* wr;        // w_i / ||a_i||^2 (0 for dropped rows)
    const float* x;         // n x B iterate (read only during the pass)
    float* delta;           // n x B correction accumulator (one-pass scatter)
    float* coef;            // m x B correction coefficients (two-pass) or null
    const float* coef_mul;  // per row multiplier of the coefficient (EMR) or null
    const float* prox_mul;  // per row multiplier of the proximity term or null
    const int* part;        // group boundaries (ngroups + 1 absolute row indices)
    double* pp;             // proximity partials: pp[cta * B + b]
    RhsState* st;
    float lam;
    int B;                  // right-hand sides in the device layout
    int n;                  // unknowns (shared-memory staging size)
    int check_stop;         // 1: skip the launch when right-hand side 0 has stopped (B = 1)
    int m;                  // rows (bounds checks of the checked build)
    long long nnz;          // entries (bounds checks of the checked build)
};

// Epilogue of a sweep (CTA 0 of the finalize / column pass): fixed-order
// reduction of the row-pass proximity partials, history, stopping rule.
struct EpiArgs {
    const double* pp;
    int npp;                // CTAs that wrote partials
    int B;
    double scale;           // factor applied to the partial sums (1/2 and block weight ratio)
    RhsState* st;
    double* prox_hist;      // [B][hist_cap]
    double* obj_hist;
    int hist_cap;
    int first_seg, last_seg;
    StopParams sp;
    const double* p_target;  // split problems: the monitored proximity (B = 1), else null
};

struct FinalizeArgs {
    float* x;
    float* delta;
    const float* zc;        // DROP column scaling 1/s_j (n) or null (1)
    const float* lo;
    const float* hi;
    long long nB;           // n * B elements
    int B;
    int box_len;            // 1 or n
    EpiArgs epi;
    // column-major second accumulator of the one-pass scatter (B = 1) or null
    float* deltaT;
    int imgW, imgH;
    // both accumulators in the patch numbering (patch_index) instead; when
    // xA / xB are set the new x is also written in the wide / tall patch
    // layout (the gathers of the next block's row pass)
    int patch, imgWp;
    float* xA;
    float* xB;
};

// Column pass of the two-pass sweep: x_j <- box(x_j + sum_i a_ij coef_i)
// over the columns [cpart[0], cpart[ngroups]) of one block's CSC.
struct ColArgs {
    const int2* cinfo;      // per column: {start, length}
    const int* ridx;        // device row index of each entry
    const void* cval;       // values (same storage type as the rows)
    const float* coef;      // m x B
    float* x;               // n x B
    const float* lo;
    const float* hi;
    const float* zc;        // DROP column scaling 1/s_j (n) or null (1)
    float* delta_out;       // EL / EMR: the column sums go here (n x B), x untouched
    int box_len;
    int B;
    const int* cpart;
    int n, m;               // columns / rows (checked build)
    long long nnz;
    EpiArgs epi;
};

// Arguments of the perturbation-phase kernels (cluster kernels and the
// whole-GPU cooperative kernel).
struct PerturbArgs {
    float* x;               // n x B
    float* g;               // n x B scratch for the subgradient
    const float* c32;       // linear objective (FP32) or null
    const double* c64;      // linear objective (FP64) or null
    int n, B, H, W, obj;
    double gamma, alpha;
    double log2_alpha;      // log2(alpha), for the trial step sizes
    int n_red, max_trials, restart_every;
    int adaptive;           // 0 power law, 1 adaptive (automatic f_ref), 2 adaptive (fixed f_ref)
    double f_ref;           // the fixed reference value (adaptive = 2)
    RhsState* st;
    int record_only;        // 1: compute f(x) into st->f_cur only (no step)
    double* part;           // whole-GPU kernel: per-CTA partials (two buffers)
    unsigned* ticket;       // whole-GPU kernel: grid barrier {arrivals, generation}
    int* err;               // whole-GPU kernel: error word (2: a barrier timed out)
    long long wait_cycles;  // whole-GPU kernel: budget of one barrier wait (SM clock cycles)
    // whole-GPU kernel, one right-hand side: when set, the phase also leaves
    // x in the wide / tall patch layouts (padded width pWp) for the one-pass
    // sweep that follows it
    float* pA;
    float* pB;
    int pWp;
};

// Threads per CTA of the whole-GPU reduction kernels (variance rule), of the
// whole-GPU perturbation kernel (one CTA per SM), and the trial points one of
// its passes evaluates.
constexpr int kWideThreads = 256;
constexpr int kPhaseThreads = 512;
constexpr int kWideTrials = 8;

struct ObjArgs {
    const float* x;
    const double* c64;
    int n, B, H, W, obj;
    double* partial;        // [cta][B]
};

// One launch of a TMA-fed streaming pass (stream.cu) over the items
// [cta_items[0], cta_items[grid]) of one block: rows of the CSR copy (row pass)
// or columns of the CSC copy (column pass), B = 1.  Items start at multiples
// of four elements and are zero-padded to a multiple of four.
constexpr int kStreamThreads = 768;
struct StreamArgs {
    const int2* info;       // per item {start, length}
    const int* idx;         // column (row pass) or row (column pass) indices
    const void* val;
    const int* cta_items;   // grid + 1 item boundaries
    int tile;               // ring stage length in elements (power of two)
    int stages;             // ring stages (2..32)
    int* err;               // set to 1 when a bounded wait gives up
    long long wait_cycles;  // budget of one bounded wait (SM clock cycles)
    // row pass
    const float* l;
    const float* u;
    const float* wr;
    const float* x;
    float* delta;
    float* coef;            // coefficients out (two-pass) or null
    const float* coef_mul;  // per row multiplier of the coefficient (EMR) or null
    const float* prox_mul;  // per row multiplier of the proximity term or null
    double* pp;
    RhsState* st;
    float lam;
    int check_stop;
    // column pass
    const float* coef_in;
    float* xw;
    const float* lo;
    const float* hi;
    const float* zc;        // DROP column scaling 1/s_j (n) or null (1)
    float* delta_out;       // EL / EMR: the column sums go here, x untouched
    int box_len;
    EpiArgs epi;
    unsigned* ticket;       // column pass of the last block: CTAs finished (the
                            // last one runs the sweep epilogue), or null
    // one-pass scatter on an H x W image: rows with rowT[i] set add into
    // deltaT at the column-major index (j mod W) * H + j / W (j / W by a
    // multiply-high with recipW = floor((2^64 - 1) / W) + 1).
    // In the two-pass row pass (SCAT 0) such rows' indices in idx are
    // column-major already, and their gathers read xT, the column-major copy
    // of x.
    const unsigned char* rowT;
    float* deltaT;
    const float* xT;
    unsigned long long recipW;
    int imgW, imgH;
    // patch numbering of the one-pass sweep (instead of row- and
    // column-major): idx holds every row's indices as patch_index(.., wide)
    // for rows without rowT and patch_index(.., tall) for rows with it; those
    // rows gather from xW (wide) and xT (tall), copies of x in the two patch
    // layouts, and add into delta and deltaT with the same indices.  imgWp =
    // W rounded up to a multiple of 8 (each layout holds ceil8(H) x imgWp).
    const float* xW;
    int patch, imgWp;
};

// Tiled one-pass sweep (tile.cu): one cooperative launch of P CTAs, CTA b
// owning tile b of the unknowns (x and the correction in shared memory) and
// streaming tile b's segments of A once per sweep.  A CTA is one warp for the
// bulk copies, one for the grid counters, W1 warps of dot products, NC warps
// of correction coefficients and W2 warps of the scatter and the box step.
constexpr int kTileMaxWarps = 32;
constexpr int kTileMaxStages = 64;
constexpr int kTileMaxChunks = 2048;
constexpr int kTileMaxCQ = 16;          // coefficient slots
constexpr int kTileQ = 32;              // chunks between the scatter and the newest data
struct TileArgs {
    const unsigned char* stream;   // every tile's byte stream
    const long long* base;         // P: start of tile b's stream (16-byte aligned)
    const int* coff;               // P x (K + 1): chunk byte offsets in the tile's stream
    const int* nsl;                // P x K: slices of tile b in chunk k
    const int4* rect;              // P: {first global column, rows, columns, local row stride}
    const int* chunk_blk;          // K: block of chunk k (chunks of a block are consecutive)
    const double* blk_scale;       // blocks: factor of the block's proximity terms
    int K;                         // chunks
    int W;                         // global column stride of a tile row (image width)
    int piece;                     // bytes per bulk copy (power of two)
    int stages;                    // ring stages of `piece` bytes
    int tile_cap;                  // words of the shared-memory x and Delta tiles
    int W1, NC, W2;                // warps of the dot products / coefficients / scatter
    int cq;                        // coefficient slots (chunks in flight between them)
    int cstride;                   // coefficients per slot (32 x most slices of a tile's chunk)
    const float* l;                // m bounds (device row order)
    const float* u;
    const float* wr;               // w_i / ||a_i||^2
    float* x;                      // n
    const float* lo;
    const float* hi;
    const float* zc;               // DROP column scaling or null
    int box_len;
    int m;
    float* r;                      // 2 x m: <a_i, x> accumulators of alternate sweeps
    unsigned* cnt;                 // K: phase-1 arrivals per chunk (zero between sweeps)
    unsigned* sync;                // {CTAs finished, epoch}
    double* pp;                    // P: proximity partials
    RhsState* st;
    int* err;                      // error word (3: a bounded wait gave up)
    long long wait_cycles;         // budget of one bounded wait
    float lam;
    EpiArgs epi;
};

// One slice of the tile streams (host plan -> device fill): up to 32
// segments of one tile and chunk, lanes longest first.
struct TileSliceRec {
    long long chunk_start;         // byte offset of the slice's chunk in the stream buffer
    int sidx;                      // table entry inside the chunk
    int off4;                      // slice offset inside the chunk, in 4-byte words
    int nl;                        // segments (lanes), 1..32
    int E;                         // entries
    int first;                     // first lane record
    int pad;
};
struct TileLaneRec {
    int row_flag;                  // device row; bit 31: the row's first segment
    int e0;                        // first entry in the packed row copy
    int len;                       // entries
};

struct TilePlanIn {
    int m, n, H, W;                // rows, unknowns, image rows and columns (H W = n)
    int P;                         // CTAs (tiles) wanted
    int vbytes;                    // bytes per stored value
    const int* perm;               // device row -> source row, or null
    const int* rp;                 // source row pointer (host)
    const int* col;                // source column indices (host)
    const int* row_start;          // device row -> first entry in the packed copy
    std::vector<int> seg_start;    // block row ranges (device order)
    long long chunk_target;        // stream bytes per CTA and chunk aimed at
    long long max_chunk;           // largest chunk of one tile the ring may hold
    int max_chunks;                // chunks the kernel's tables hold
    int max_slices;                // most slices of one tile in one chunk
    int max_seg;                   // longest segment (entries)
    int group_rows;                // consecutive rows kept together (slice neighbours)
    long long max_tile_words;      // shared-memory words of one tile
};

struct TilePlan {
    int P = 0, K = 0, tile_cap = 0, max_chunk = 0, max_slices = 0;
    long long bytes = 0, segments = 0;
    std::vector<long long> base;
    std::vector<int> coff, nsl, chunk_blk;
    std::vector<int4> rect;
    std::vector<int> tile_of;
    std::vector<unsigned short> local_of;
    std::vector<TileSliceRec> slices;
    std::vector<TileLaneRec> lanes;
};

bool plan_tiles(const TilePlanIn& in, TilePlan& out, std::string& why);
size_t tile_smem_bytes(int ring_bytes, int tile_cap, int K, int stages, int cq, int cstride);
int tile_blocks_per_sm(suppy_dtype dt, int threads, size_t smem);
cudaError_t launch_tile_sweep(const TileArgs& a, suppy_dtype dt, int grid, size_t smem,
                              cudaStream_t s);
cudaError_t launch_tile_fill(const TileSliceRec* slices, long long nslices, const TileLaneRec* lanes,
                             const void* val, suppy_dtype dt, const int* col,
                             const unsigned short* local_of, unsigned char* stream, cudaStream_t s);

// Extrapolated step of EL / EMR (sweep.cu): t_b from the sweep's reductions,
// then x <- box(x + lambda t_b delta), delta <- 0.
struct ExtArgs {
    float* x;
    float* delta;           // n x B column sums A^T (W d)
    const float* lo;
    const float* hi;
    int box_len;
    long long n;
    int B;
    RhsState* st;
    int method;             // SUPPY_EL or SUPPY_EMR
    const double* pp;       // row pass partials (sum w d^2 / ||a||^2), npp CTAs x B
    int npp;
    const double* qq;       // EMR: partials of sum w q^2 (q = A delta), nqq CTAs x B
    int nqq;
    double* part;           // grid x B x 1 partials of ||delta||^2
    unsigned* ticket;
    double* tstep;          // B step sizes
    float lam;
};

// --- launchers (defined in sweep.cu / stream.cu / perturb.cu / setup.cu) ----
size_t stream_smem_bytes(suppy_dtype dt, int tile, int stages);
int stream_stages_for(suppy_dtype dt, int tile);   // stages filling the shared-memory budget
int stream_max_item(int tile, int stages);          // longest item a ring window holds
int stream_blocks_per_sm(suppy_dtype dt, int tile, int stages);
// map: how a group's G lanes split an item -- 0 four consecutive elements per
// lane and 16-byte ring reads, 1 lane-interleaved elements (lane gl takes
// gl, gl + G, ...) and 4-byte ring reads
cudaError_t launch_rows_tma(const StreamArgs& a, suppy_dtype dt, int G, int scat, int map, int grid,
                            cudaStream_t s);
cudaError_t launch_cols_tma(const StreamArgs& a, suppy_dtype dt, int G, int map, int grid,
                            cudaStream_t s);
// scat: 0 no scatter (proximity / coefficient output), 1 global reductions,
// 2 shared-memory staged reductions (n * 4 bytes of shared memory)
cudaError_t launch_sweep(const SweepArgs& a, suppy_dtype dt, int G, int maxe, int scat, int grid,
                         cudaStream_t s);
cudaError_t launch_sweep_batched(const SweepArgs& a, suppy_dtype dt, int scat, int grid,
                                 cudaStream_t s);
int sweep_blocks_per_sm(suppy_dtype dt, int G, int maxe, int scat, int batchedB, int n);
cudaError_t launch_colpass(const ColArgs& a, suppy_dtype dt, int G, int grid, cudaStream_t s);
cudaError_t launch_epilogue(const EpiArgs& a, cudaStream_t s);
int colpass_blocks_per_sm(suppy_dtype dt, int G, int B);
cudaError_t launch_finalize(const FinalizeArgs& a, int grid, cudaStream_t s);
cudaError_t launch_patch_image(const float* x, float* xA, float* xB, int H, int W, int Wp, cudaStream_t s);
cudaError_t launch_patch_cols(const int2* rinfo, const unsigned char* rowT, int m, unsigned long long recipW,
                              int W, int Wp, int* col, cudaStream_t s);
cudaError_t launch_transpose_image(const float* x, float* xT, int H, int W, cudaStream_t s);
cudaError_t launch_transposed_cols(const int2* rinfo, const unsigned char* rowT, int m,
                                   unsigned long long recipW, int W, int H, int* col, cudaStream_t s);
cudaError_t launch_reduce_pp(const double* pp, int npp, int B, double scale, int accumulate,
                             double* out, cudaStream_t s);
cudaError_t launch_perturb(const PerturbArgs& a, int cluster, cudaStream_t s);
// The whole perturbation phase on the whole GPU: one cooperative launch of
// `grid` CTAs of kPhaseThreads threads, all resident (subgradient pass,
// kWideTrials trial evaluations per pass, update, grid barriers between).
cudaError_t launch_perturb_wide(const PerturbArgs& a, int grid, cudaStream_t s);
size_t wide_part_doubles(int grid);   // partials the whole-GPU kernel needs
int wide_phase_blocks_per_sm();       // its resident CTAs per SM
int choose_perturb_cluster(int n, int B);
int fit_perturb_cluster(int want, int obj, int n, int H, int W);
cudaError_t launch_objective(const ObjArgs& a, int grid, double* out, cudaStream_t s);
// Variance stopping rule after an iteration: relative change of every active
// right-hand side against xprev (then xprev <- x), running sums in the state,
// stop when the sample variance of the changes falls below tol.
cudaError_t launch_variance(float* x, float* xprev, long long n, int B, RhsState* st,
                            double* part, unsigned* ticket, double tol, int grid, cudaStream_t s);

cudaError_t launch_validate_csr(const int* row_ptr, const int* col, const float* val, int m,
                                int n, long long nnz, int* flags, cudaStream_t s,
                                double* err2 = nullptr);
cudaError_t launch_validate_vec(const float* v, long long len, int allow_inf, int* flags,
                                int bit, cudaStream_t s);
cudaError_t launch_validate_pair(const float* lo, const float* hi, long long len, int* flags,
                                 int bit, cudaStream_t s);
cudaError_t launch_pack(const int* row_ptr, const int* col, const float* val, const int* perm,
                        const int2* rinfo, int m, int* pcol, void* pval, suppy_dtype dt,
                        double* rho, cudaStream_t s);
cudaError_t launch_csc_fill(const int2* rinfo, int m, const void* pval, suppy_dtype dt,
                            const int* pos, int* ridx, void* cval, cudaStream_t s);
cudaError_t launch_count_kept(const double* rho, const int* seg_of_row, int m, int* kept,
                              cudaStream_t s);
cudaError_t launch_weights(const double* rho, const int* seg_of_row, const double* seg_w, int m,
                           float* wr, cudaStream_t s);
cudaError_t launch_zero_row_check(const double* rho, const float* l, const float* u, int m,
                                  int B, int* flags, cudaStream_t s);
cudaError_t launch_permute_bounds(const float* l_in, const float* u_in, const int* perm, int m,
                                  int B_in, int B, float* l, float* u, cudaStream_t s,
                                  const int* skip = nullptr, int nskip = 0);
cudaError_t launch_check_bounds(const double* rho, const float* l_in, const float* u_in,
                                const int* perm, int m, int B_in, int* flags, cudaStream_t s);
cudaError_t launch_reset_states(RhsState* st, int B, int B_user, cudaStream_t s);
cudaError_t launch_box_init(float* x, const float* lo, const float* hi, long long nB, int B,
                            int box_len, const float* x_in, int B_in, cudaStream_t s);
cudaError_t launch_unpad_x(const float* x, long long n, int B, int B_out, float* out,
                           cudaStream_t s);
cudaError_t launch_load_column(const float* l_in, const float* u_in, const int* perm, int m, int B,
                               int b, float* l, float* u, cudaStream_t s);
cudaError_t launch_reset_column(float* x, const float* lo, const float* hi, long long n, int B,
                                int b, int box_len, RhsState* st, float* xprev, cudaStream_t s);
cudaError_t launch_set_stopped(RhsState* st, int b, cudaStream_t s);
cudaError_t launch_extract_column(const float* x, long long n, int B, int b, float* out,
                                  cudaStream_t s);
// DROP: zc[j] = 1 / (stored nonzeros of column j in rows with ||a_i|| > 0), 0 if none.
cudaError_t launch_column_scaling(const int2* rinfo, const int* col, const void* val,
                                  suppy_dtype dt, const double* rho, int m, int n, int* counts,
                                  float* zc, cudaStream_t s);
cudaError_t launch_ext_step(const ExtArgs& a, int grid, cudaStream_t s);
cudaError_t launch_to_float(const double* v, int n, float* out, cudaStream_t s);
cudaError_t launch_colmean(const int* row_ptr, const int* col, const float* val, int m, int n,
                           double* c64, float* c32, double* work, int work_ctas,
                           cudaStream_t s);
cudaError_t launch_sumsq(const double* v, int n, double* out, cudaStream_t s);

// Split feasibility: one dose-volume constraint, in structure order.
// Doses are compared with d_ref through order-preserving keys of floats:
// d > d_ref iff key(d) > key_gt (key of the largest float <= d_ref), d >= d_ref
// iff key(d) >= key_ge (key of the smallest float >= d_ref).
struct DvcDesc {
    int kind;               // 0: upper (at most K above d_ref), 1: lower (at least K at or above)
    int K;                  // voxel count of the constraint
    int orig;               // position in the caller's list (proximity order)
    uint32_t key_gt, key_ge;
    float ref_hi, ref_lo;   // d_ref as float-float
    float wf;               // w as float
    double w;               // weight 1 / ndvc
    double d_ref;
};

struct DvcArgs {
    const int* rp;          // CSR of A_q: row_ptr (m_q + 1), col, val
    const int* col;
    const float* val;
    const int* cp;          // CSC of A_q: col_ptr (n + 1), row, val
    const int* crow;
    const float* cval;
    const int* sptr;        // structure row ranges (nstruct + 1)
    const int* sdvc;        // DVCs of structure s: dvc[sdvc[s] .. sdvc[s+1])
    const DvcDesc* dvc;
    const float* x;         // iterate read by the dose pass (element j at x[j * B])
    float* xw;              // iterate updated by the correction pass (the same layout)
    float* dose;            // m_q
    float* corr;            // m_q: sum_j w_j (P_Qj(d) - d)
    double* pd;             // per DVC (caller order) x cluster rank: chunk sums of the
                            // squared corrections
    double* target;         // their sum
    const RhsState* st;     // skip when right-hand side 0 has stopped, or null
    float gamma;
    int mq, n, nstruct, ndvc;
    int B;                  // stride of x: the context's right-hand sides (x is n x B);
                            // x, xw, st, pd and target point at the one being stepped
    long long nnz;          // entries of A_q
    size_t smem;            // dynamic shared memory of the projection (keys staged), or 0
};

constexpr int kDvcCluster = 8;                // CTAs (one cluster) per structure
constexpr size_t kDvcSmemMax = 192 * 1024;   // structures up to 8 x 49152 rows stage their keys
size_t dvc_project_smem(int max_rows);

cudaError_t launch_dvc_dose(const DvcArgs& a, cudaStream_t s);
cudaError_t launch_dvc_project(const DvcArgs& a, cudaStream_t s);   // + the proximity sum
cudaError_t launch_dvc_apply(const DvcArgs& a, cudaStream_t s);
// part: nstruct x 32 chunk sums (scratch), out: nstruct norms
cudaError_t launch_dvc_frob(const int* rp, const float* val, const int* sptr, int nstruct,
                            double* part, double* out, cudaStream_t s);

// Checked build (-DSUPPY_CHECKED): kernels verify indices and the alignment of
// vector accesses before issuing them; the first violation is recorded in a
// device word (kernel tag, index) and the access is skipped.
cudaError_t read_check_word(int* out3);   // {tag, index low, index high}; resets the word
cudaError_t read_check_word_perturb(int* out3);

// Set the message suppy_last_error(NULL) returns on this thread (api.cu).
void set_thread_error(const std::string& msg);

// Internal interface of a context for the serving runtime (api.cu, serve.cu).
int ctx_slots(const suppy_ctx* c);
int ctx_n(const suppy_ctx* c);
int ctx_m(const suppy_ctx* c);
cudaStream_t ctx_stream(const suppy_ctx* c);
size_t ctx_device_bytes(const suppy_ctx* c);
const char* ctx_error(const suppy_ctx* c);
void ctx_set_sweep_budget(suppy_ctx* c, int max_sweeps);
suppy_status ctx_slot_load(suppy_ctx* c, int b, const float* l, const float* u);
suppy_status ctx_slot_stop(suppy_ctx* c, int b);
suppy_status ctx_states_async(suppy_ctx* c, RhsState* host);
suppy_status ctx_slot_extract(suppy_ctx* c, int b, float* out);
suppy_status ctx_iterate(suppy_ctx* c, const suppy_params* p, int iters);

// --- device helpers ---------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Column-major index (j mod W) * H + j / W of the row-major pixel j of an
// H x W image.  j / W is the high word of j * recipW with recipW =
// floor((2^64 - 1) / W) + 1 = 2^64 / W + e, 0 <= e <= 1: the product over 2^64
// is j / W + j e / 2^64, and j e / 2^64 < 2^-32 <= 1/W never carries past the
// next integer because the fractional part of j / W is at most 1 - 1/W
// (j < 2^32, 2 <= W <= 2^32).
__device__ __forceinline__ int transposed_index(int j, unsigned long long recipW, int W, int H) {
    const int q = (int)__umul64hi((unsigned long long)(unsigned)j, recipW);
    return (j - q * W) * H + q;
}

// Patch numbering of pixel j = (y, x) of an H x W image for the one-pass
// scatter, over a zero-padded ceil8(H) x Wp grid (Wp = ceil8(W)).  Wide
// patches: 128-byte lines of 8 x 4 pixels (x by y), each made of four 32-byte
// sectors of 4 x 2 pixels; tall patches: lines of 4 x 8 pixels made of
// sectors of 2 x 4.  Lines and sectors are numbered row by row, pixels inside
// a sector row-major.  A ray's run of consecutive entries crosses fewer lines
// and sectors here than in a row- or column-major image whenever it is not
// axis-aligned: rays closer to the horizontal take the wide patches, the
// others the tall ones.  y = j / W as in transposed_index.
__device__ __forceinline__ int patch_pos(int y, int x, int Wp, bool tall) {
    if (!tall)
        return (((y >> 2) * (Wp >> 3) + (x >> 3)) << 5) | (((y >> 1) & 1) << 4) | (((x >> 2) & 1) << 3) |
               ((y & 1) << 2) | (x & 3);
    return (((y >> 3) * (Wp >> 2) + (x >> 2)) << 5) | (((y >> 2) & 1) << 4) | (((x >> 1) & 1) << 3) |
           ((y & 3) << 1) | (x & 1);
}
__device__ __forceinline__ int patch_index(int j, unsigned long long recipW, int W, int Wp, bool tall) {
    const int y = (int)__umul64hi((unsigned long long)(unsigned)j, recipW);
    return patch_pos(y, j - y * W, Wp, tall);
}

__device__ __forceinline__ float clampf(float v, float lo, float hi) {
    return fminf(fmaxf(v, lo), hi);
}

// Sweep epilogue, run by one CTA (warp w handles right-hand sides w, w + W,
// ... for W warps): the proximity partials of the pass summed in a fixed
// order, the monitored proximity and objective recorded, and the stopping
// rule of Sec. 2.2.1 / 2.2.3 applied.  The CTA that runs it must be the last
// reader of the stop flags in its launch.
__device__ __forceinline__ void sweep_epilogue(const EpiArgs& a) {
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int b = wid; b < a.B; b += blockDim.x / 32) {
        double s = 0.0;
        for (int c = lane; c < a.npp; c += 32) s += a.pp[(size_t)c * a.B + b];
        s = warp_sum(s);
        if (lane != 0) continue;
        RhsState& st = a.st[b];
        if (st.stopped) continue;
        if (a.first_seg) st.p_acc = 0.0;
        st.p_acc += a.scale * s;
        if (!a.last_seg) continue;
        const double p = a.p_target ? a.p_target[b] : st.p_acc;
        const int k = st.k;
        if (k < a.hist_cap) {
            a.prox_hist[(size_t)b * a.hist_cap + k] = p;
            a.obj_hist[(size_t)b * a.hist_cap + k] =
                st.f_valid ? st.f_cur : __longlong_as_double(0x7ff8000000000000LL);
        }
        // stopping rule (Sec. 2.2.1 and 2.2.3)
        if (st.has_prev_p && fabs(p - st.p_prev) / fmax(1.0, st.p_prev) < a.sp.prox_rel)
            st.calm += 1;
        else
            st.calm = 0;
        const bool feas = (p <= a.sp.prox_abs) || (st.calm >= a.sp.patience);
        bool objok = true;
        if (a.sp.has_obj && a.sp.obj_rel > 0.0 && st.f_valid) {
            objok = st.has_prev_f &&
                    fabs(st.f_cur - st.f_prev) / fmax(1.0, fabs(st.f_prev)) < a.sp.obj_rel;
        }
        st.p_prev = p;
        st.has_prev_p = 1;
        if (st.f_valid) {
            st.f_prev = st.f_cur;
            st.has_prev_f = 1;
        }
        st.f_valid = 0;
        st.last_prox = p;
        st.k = k + 1;
        if ((a.sp.use_stopping && feas && objok) || (a.sp.max_sweeps > 0 && k + 1 >= a.sp.max_sweeps))
            st.stopped = 1;
    }
}

}  // namespace suppy
