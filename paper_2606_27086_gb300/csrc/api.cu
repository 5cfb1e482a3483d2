// Host side of the C ABI declared in include/suppy.h: context lifetime, input
// validation, setup orchestration (device layout, weights, launch partition),
// the Algorithm 1 driver loop, checkpoints and measurement hooks.  All compute
// runs in the kernels of sweep.cu, perturb.cu and setup.cu.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "common.cuh"

using namespace suppy;

namespace {

thread_local std::string g_err;

// Longest ring tile of the streaming passes; the packed copies of A carry
// this much zeroed slack after the last item, since a pass reads whole tiles.
constexpr int kMaxTile = 4096;

// Lane maps of the streaming row and column passes when neither the caller
// nor the tuner chose one (0 quads per lane, 1 lane-interleaved).  Which map
// is faster depends on the matrix and the ring shape: tuned on CT 512x512,
// the column pass ran faster interleaved (202 against 213 us, 1024-element
// tiles) and the row pass with quads (217 against 249 us); on CT 384x384 at
// the default 4096-element tiles the interleaved column pass was slower
// (126 against 112 us).  Untuned contexts keep quads; the tuner tries both.
constexpr int kDefaultRowMap = 0;
constexpr int kDefaultColMap = 0;

// Stored length of an item: rows and columns start at multiples of four
// elements and are zero-padded to a multiple of four.
inline long long pad4(long long len) { return (len + 3) & ~3LL; }

}  // namespace

namespace suppy {
void set_thread_error(const std::string& msg) { g_err = msg; }
}  // namespace suppy

struct suppy_ctx {
    int dev = 0;
    cudaStream_t stream = nullptr;
    int m = 0, n = 0, B_user = 1, B = 1;
    long long nnz = 0;
    long long nnz_pad = 0;          // storage length of the row copy (rows padded to 4)
    suppy_dtype dt = SUPPY_F32;
    suppy_mode mode = SUPPY_CIMMINO;
    suppy_obj obj = SUPPY_OBJ_NONE;
    int H = 0, W = 0;
    int gH = 1, gW = 1;             // grid of the unknowns (image rows x columns, or 1 x n)
    int box_len = 1;
    int nseg = 1;
    std::vector<int> seg_start;     // device-order row ranges of the segments (blocks)
    std::vector<int> seg_kept;      // kept rows per segment
    int m_kept = 0;

    // device buffers
    int2* d_rinfo = nullptr;
    int* d_col = nullptr;
    void* d_val = nullptr;
    float* d_wr = nullptr;
    double* d_rho = nullptr;
    float* d_l = nullptr;
    float* d_u = nullptr;
    int* d_perm = nullptr;          // device row -> source row (null: identity)
    float* d_x = nullptr;
    float* d_delta = nullptr;
    // one-pass scatter on an image grid: rows added column-major (device row
    // order flags), their accumulator, and 2^64 / gW rounded up
    unsigned char* d_rowT = nullptr;
    float* d_deltaT = nullptr;
    int* d_colT = nullptr;          // the packed indices, those rows' column-major
    float* d_xT = nullptr;          // x column-major (the two-pass row pass gathers)
    unsigned long long recipW = 0;
    long long trows = 0;
    bool tr_on = false;             // the sweep uses them (chosen at create)
    bool tr_patch = false;          // the one-pass sweep numbers pixels by patches
    int* d_colP = nullptr;          // the packed indices, every row's in its patch layout
    float* d_xA = nullptr;          // x in the wide / tall patch layouts (the gathers)
    float* d_xB = nullptr;
    int gWp = 0;                    // image width rounded up to a multiple of 8
    size_t acc_len = 0;             // floats of d_delta and d_deltaT (padded grid when a grid is set)
    float* d_g = nullptr;
    float* d_lo = nullptr;
    float* d_hi = nullptr;
    float* d_zc = nullptr;          // DROP column scaling (null otherwise)
    // EL / EMR: ||a_i||^2 as FP32, zero bounds, q-pass partials, step sizes
    float* d_rhof = nullptr;
    float* d_zero = nullptr;
    double* d_qq = nullptr;
    double* d_xpart = nullptr;
    unsigned* d_xticket = nullptr;
    double* d_tstep = nullptr;
    int xgrid = 0;
    int qq_cap = 0;                 // CTAs the q-pass partials hold
    // variance stopping rule: previous iterate, partials, ticket
    float* d_xprev = nullptr;
    bool xprev_stale = true;
    double* d_vpart = nullptr;
    unsigned* d_vticket = nullptr;
    int vgrid = 0;
    double* d_pp = nullptr;
    RhsState* d_st = nullptr;
    double* d_prox_hist = nullptr;
    double* d_obj_hist = nullptr;
    int hist_cap = 0;
    double* d_c64 = nullptr;
    float* d_c32 = nullptr;
    double* d_out = nullptr;        // B doubles for proximity / objective results
    double* d_objpart = nullptr;
    int* d_part = nullptr;          // nseg x (groups + 1)
    double* h_out = nullptr;        // pinned B doubles
    int* h_err = nullptr;           // pinned copy of the streaming passes' error word
    int* h_bflags = nullptr;        // pinned copy of an enqueued bounds check (2 words)
    bool bounds_pending = false;    // h_bflags holds a check not yet reported
    int k_upper = 0;                // upper bound of the sweep counters (history sizing)
    float* d_stage_l = nullptr;     // persistent staging of host bounds (set_bounds)
    float* d_stage_u = nullptr;
    int* d_flags = nullptr;         // validation flags

    // two-pass layout: CSC copy of A per block, coefficients
    int2* d_cinfo = nullptr;        // nseg x n
    int* d_ridx = nullptr;
    void* d_cval = nullptr;
    float* d_coef = nullptr;        // m x B
    int* d_cpart = nullptr;         // nseg x (cgroups + 1)
    std::vector<long long> cpref;   // per segment column-work prefix (nseg x (n + 1))
    long long nnz_csc = 0;
    long long csc_len = 0;          // storage length of the CSC copy (columns padded to 4)

    // tiled one-pass sweep (strategy 3): tile streams, tables, accumulators
    unsigned char* d_tstream = nullptr;
    long long* d_tbase = nullptr;
    int* d_tcoff = nullptr;
    int* d_tnsl = nullptr;
    int4* d_trect = nullptr;
    int* d_tcblk = nullptr;
    double* d_tscale = nullptr;
    float* d_tr = nullptr;          // 2 x m
    unsigned* d_tcnt = nullptr;     // chunk counters
    unsigned* d_tsync = nullptr;    // {CTAs finished, epoch}
    double* d_tpp = nullptr;
    int tiP = 0, tiK = 0, ticap = 0, timaxchunk = 0;
    int tiW1 = 10, tiW2 = 16;             // warps of the dot products / scatter
    int tiNC = 4, ticq = 8, ticstride = 0; // coefficient warps, their slots, coefficients per slot
    int tipiece = 8192, tistages = 0;     // ring: bytes per copy, stages
    size_t tismem = 0;
    long long tibytes = 0;                // bytes of the tile streams
    long long tisegs = 0;                 // segments

    // launch shapes
    int strategy = 1;               // 1 one pass, 2 two passes, 3 tiled one pass
    int scat = 1;                   // one pass: 1 L2 reductions, 2 shared-memory staged
    int G = 32, maxe = 8;
    int grid_sweep = 0, groups = 0;             // largest row-pass launch
    int Gc = 32, grid_col = 0, cgroups = 0;     // largest column-pass launch
    std::vector<int> seg_grid, seg_cgrid;       // per block launch sizes
    std::vector<size_t> seg_part_off, seg_cpart_off;
    // TMA-fed streaming passes (B = 1): CTA item ranges per block
    bool use_tma = false;
    int tile = 4096, stages = 6;    // row pass ring: tile length, stages
    int ctile = 4096, cstages = 6;  // column pass ring
    int tG = 32, tGc = 32;          // lanes per item of the streaming row / column passes
    int tMap = 0, tMapc = 0;        // their lane maps (0 quads per lane, 1 lane-interleaved)
    int max_row = 0, max_col = 0;
    std::vector<int> seg_tgrid, seg_ctgrid;
    std::vector<size_t> seg_tpart_off, seg_ctpart_off;
    int* d_tpart = nullptr;
    int* d_ctpart = nullptr;
    int* d_err = nullptr;           // set by a kernel whose bounded wait gave up
    long long wait_cycles = kDefaultWaitCycles;   // budget of one bounded device wait
    unsigned* d_cticket = nullptr;  // streamed column pass: CTAs finished (fused epilogue)
    int grid_fin = 0;
    int grid_obj = 0;
    int perturb_cluster = 1;
    // serving: per right-hand side sweep budget and one-slot staging
    int slot_max_sweeps = 0;
    float* d_slot_l = nullptr;
    float* d_slot_u = nullptr;
    std::vector<unsigned char> zero_row;   // source order: ||a_i|| = 0
    // whole-GPU perturbation phase (one cooperative launch)
    bool wide = false;
    int wide_grid = 0;
    double* d_wpart = nullptr;
    unsigned* d_ticket = nullptr;   // grid barrier of the whole-GPU perturbation {count, generation}
    std::vector<long long> rpref;   // row-work prefix (m + 1)
    // split feasibility: dose rows A_q (CSR and CSC), structures, DVCs
    bool dvc_on = false;
    int mq = 0, nstruct = 0, ndvc = 0;
    float dvc_gamma = 0.f;
    size_t dvc_smem = 0;
    long long dvc_nnz = 0;
    int* d_qrp = nullptr;
    int* d_qcol = nullptr;
    float* d_qval = nullptr;
    int* d_qcp = nullptr;
    int* d_qrow = nullptr;
    float* d_qcval = nullptr;
    int* d_qsptr = nullptr;
    int* d_qsdvc = nullptr;
    DvcDesc* d_qdvc = nullptr;
    float* d_dose = nullptr;
    float* d_qcorr = nullptr;
    double* d_qpd = nullptr;
    double* d_target = nullptr;

    // measurement
    struct TimedLaunch {
        int kind;
        cudaEvent_t a, b;
    };
    bool timing = false;
    std::vector<TimedLaunch> evs;
    double timing_ms[4] = {0.0, 0.0, 0.0, 0.0};
    long long timing_n[4] = {0, 0, 0, 0};
    long long launches = 0;
    size_t dev_bytes = 0;                               // held now (allocs)
    std::vector<std::pair<void*, size_t>> allocs;      // library-owned device buffers

    // CUDA graph of one superiorized iteration (perturbation + sweep)
    cudaGraphExec_t graph = nullptr;
    std::vector<char> graph_key;
    long long graph_launches = 0;
    cudaStream_t cap_stream = nullptr;   // private stream used only while capturing

    std::string err;
};

namespace {

suppy_status fail(suppy_ctx* c, suppy_status s, const std::string& msg) {
    if (c) c->err = msg;
    else g_err = msg;
    return s;
}

// On failure the runtime's last-error slot is cleared so that a later,
// unrelated launch check does not report this error again.
#define CK(call)                                                                          \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess) {                                                          \
            cudaGetLastError();                                                           \
            return fail(c, SUPPY_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
        }                                                                                 \
    } while (0)

template <typename T>
suppy_status dalloc(suppy_ctx* c, T** p, size_t count) {
    size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, e == cudaErrorMemoryAllocation ? SUPPY_ENOMEM : SUPPY_ECUDA,
                    std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
    }
    c->allocs.emplace_back(q, bytes);
    c->dev_bytes += bytes;
    *p = static_cast<T*>(q);
    return SUPPY_OK;
}

void dfree(suppy_ctx* c, void* p) {
    if (!p) return;
    auto it = std::find_if(c->allocs.begin(), c->allocs.end(),
                           [p](const std::pair<void*, size_t>& a) { return a.first == p; });
    if (it != c->allocs.end()) {
        c->dev_bytes -= it->second;
        c->allocs.erase(it);
    }
    cudaFree(p);
}

// Copy a host vector into a new library-owned device buffer (enqueued).
template <typename T>
suppy_status upload(suppy_ctx* c, const std::vector<T>& v, T** out) {
    suppy_status s = dalloc(c, out, v.size());
    if (s != SUPPY_OK) return s;
    if (!v.empty())
        CK(cudaMemcpyAsync(*out, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, c->stream));
    return SUPPY_OK;
}

// Copy count elements from a host or device pointer into a new device buffer
// (returns src itself when it already lives on the device and own == false).
template <typename T>
suppy_status stage(suppy_ctx* c, const T* src, size_t count, int on_device, T** out,
                   std::vector<void*>& temps) {
    if (on_device) {
        *out = const_cast<T*>(src);
        return SUPPY_OK;
    }
    T* d = nullptr;
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(c, SUPPY_ENOMEM, std::string("cudaMalloc staging: ") + cudaGetErrorString(e));
    }
    d = static_cast<T*>(q);
    temps.push_back(q);
    if (count) CK(cudaMemcpyAsync(d, src, count * sizeof(T), cudaMemcpyHostToDevice, c->stream));
    *out = d;
    return SUPPY_OK;
}

struct TempGuard {
    std::vector<void*> v;
    cudaStream_t s = nullptr;
    ~TempGuard() {
        if (s) cudaStreamSynchronize(s);
        for (void* p : v) cudaFree(p);
    }
};

void note_launch(suppy_ctx* c, int k = 1) { c->launches += k; }

// nnz-balanced contiguous partition of rows [r0, r1) into ng groups; the work
// of a row is its padded length plus a fixed per-row cost.
void partition(const std::vector<long long>& pref, int r0, int r1, int ng, int* out) {
    const long long kRowCost = 16;
    auto work = [&](int r) { return pref[r] + kRowCost * r; };
    const long long w0 = work(r0), w1 = work(r1);
    out[0] = r0;
    int lo = r0;
    for (int g = 1; g < ng; ++g) {
        const long long target = w0 + (w1 - w0) * g / ng;
        int a = lo, b = r1;
        while (a < b) {
            const int mid = a + (b - a) / 2;
            if (work(mid) < target) a = mid + 1;
            else b = mid;
        }
        out[g] = a;
        lo = a;
    }
    out[ng] = r1;
}

// Fresh iteration state of every right-hand side (padding ones stopped),
// enqueued on the context's stream.
suppy_status reset_state(suppy_ctx* c) {
    c->k_upper = 0;
    c->xprev_stale = true;
    CK(launch_reset_states(c->d_st, c->B, c->B_user, c->stream));
    note_launch(c);
    return SUPPY_OK;
}

suppy_status ensure_hist(suppy_ctx* c, int need) {
    if (need <= c->hist_cap) return SUPPY_OK;
    int cap = std::max(need, std::max(1024, 2 * c->hist_cap));
    double *p = nullptr, *o = nullptr;
    suppy_status s;
    if ((s = dalloc(c, &p, (size_t)cap * c->B)) != SUPPY_OK) return s;
    if ((s = dalloc(c, &o, (size_t)cap * c->B)) != SUPPY_OK) return s;
    if (c->hist_cap > 0) {
        CK(cudaMemcpy2DAsync(p, cap * sizeof(double), c->d_prox_hist, c->hist_cap * sizeof(double),
                             c->hist_cap * sizeof(double), c->B, cudaMemcpyDeviceToDevice,
                             c->stream));
        CK(cudaMemcpy2DAsync(o, cap * sizeof(double), c->d_obj_hist, c->hist_cap * sizeof(double),
                             c->hist_cap * sizeof(double), c->B, cudaMemcpyDeviceToDevice,
                             c->stream));
        CK(cudaStreamSynchronize(c->stream));
        dfree(c, c->d_prox_hist);
        dfree(c, c->d_obj_hist);
    }
    c->d_prox_hist = p;
    c->d_obj_hist = o;
    c->hist_cap = cap;
    return SUPPY_OK;
}

suppy_status flush_timing(suppy_ctx* c) {
    if (c->evs.empty()) return SUPPY_OK;
    CK(cudaStreamSynchronize(c->stream));
    for (auto& t : c->evs) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, t.a, t.b));
        c->timing_ms[t.kind] += ms;
        c->timing_n[t.kind] += 1;
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    c->evs.clear();
    return SUPPY_OK;
}

// Bracket one launch with events when timing is enabled.
struct Timed {
    suppy_ctx* c;
    int kind;
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t begin() {
        if (!c->timing) return cudaSuccess;
        cudaError_t e = cudaEventCreate(&a);
        if (e == cudaSuccess) e = cudaEventCreate(&b);
        if (e == cudaSuccess) e = cudaEventRecord(a, c->stream);
        return e;
    }
    cudaError_t end() {
        if (!c->timing) return cudaSuccess;
        cudaError_t e = cudaEventRecord(b, c->stream);
        if (e == cudaSuccess) c->evs.push_back({kind, a, b});
        return e;
    }
};

StopParams stop_params(const suppy_ctx* c, const suppy_params* p) {
    StopParams sp;
    sp.prox_abs = p->prox_abs;
    sp.prox_rel = p->prox_rel;
    sp.obj_rel = p->obj_rel;
    sp.patience = p->patience;
    sp.use_stopping = p->use_stopping;
    sp.has_obj = c->obj != SUPPY_OBJ_NONE;
    sp.max_sweeps = c->slot_max_sweeps;
    return sp;
}

SweepArgs row_args(suppy_ctx* c, int t, float lam) {
    SweepArgs a;
    a.rinfo = c->d_rinfo;
    a.col = c->d_col;
    a.val = c->d_val;
    a.l = c->d_l;
    a.u = c->d_u;
    a.wr = c->d_wr;
    a.x = c->d_x;
    a.delta = c->d_delta;
    a.coef = nullptr;
    a.coef_mul = nullptr;
    a.prox_mul = nullptr;
    a.part = c->d_part + c->seg_part_off[t];
    a.pp = c->d_pp;
    a.st = c->d_st;
    a.lam = lam;
    a.B = c->B;
    a.n = c->n;
    a.check_stop = 1;
    a.m = c->m;
    a.nnz = c->nnz_pad;
    return a;
}

double seg_scale(const suppy_ctx* c, int t) {
    // DROP sweeps with unit row weights; the monitored proximity keeps 1/m'
    if (c->mode == SUPPY_DROP) return c->m_kept > 0 ? 0.5 / c->m_kept : 0.0;
    if (c->nseg == 1) return 0.5;
    return c->m_kept > 0 ? 0.5 * (double)c->seg_kept[t] / c->m_kept : 0.0;
}

EpiArgs epi_args(suppy_ctx* c, int t, const StopParams& sp) {
    EpiArgs e;
    e.pp = c->d_pp;
    e.npp = c->seg_grid[t];
    e.B = c->B;
    e.scale = seg_scale(c, t);
    e.st = c->d_st;
    e.prox_hist = c->d_prox_hist;
    e.obj_hist = c->d_obj_hist;
    e.hist_cap = c->hist_cap;
    e.first_seg = (t == 0);
    e.last_seg = (t == c->nseg - 1);
    e.sp = sp;
    e.p_target = c->dvc_on ? c->d_target : nullptr;
    return e;
}

// Row pass of block t: the fused one-pass sweep (scat 1/2) or the
// coefficient-writing row pass (scat 0).
suppy_status launch_rows(suppy_ctx* c, const SweepArgs& a, int scat, int t) {
    Timed tm{c, 0};
    CK(tm.begin());
    const int grid = c->seg_grid[t];
    if (c->B == 1) CK(launch_sweep(a, c->dt, c->G, c->maxe, scat, grid, c->stream));
    else CK(launch_sweep_batched(a, c->dt, scat, grid, c->stream));
    CK(tm.end());
    note_launch(c);
    return SUPPY_OK;
}

// Buffers of the EL / EMR step: ||a_i||^2 as FP32 and zero bounds (EMR's
// q-pass), the q-pass partials, the step's partials, ticket and step sizes.
suppy_status prepare_ext(suppy_ctx* c) {
    suppy_status s;
    int sms = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->dev));
    const long long nB = (long long)c->n * c->B;
    c->xgrid = (int)std::max<long long>(1, std::min<long long>(2LL * sms, (nB + 255) / 256));
    if ((s = dalloc(c, &c->d_xpart, (size_t)c->xgrid * c->B)) != SUPPY_OK) return s;
    if ((s = dalloc(c, &c->d_xticket, 1)) != SUPPY_OK) return s;
    if ((s = dalloc(c, &c->d_tstep, (size_t)c->B)) != SUPPY_OK) return s;
    CK(cudaMemsetAsync(c->d_xticket, 0, sizeof(unsigned), c->stream));
    if (c->mode == SUPPY_EMR) {
        // q-pass partials: one per CTA of any row-pass launch (at most 16 per SM)
        const int g = 16 * sms;
        c->qq_cap = g;
        if ((s = dalloc(c, &c->d_rhof, (size_t)std::max(c->m, 1))) != SUPPY_OK) return s;
        if ((s = dalloc(c, &c->d_zero, (size_t)std::max(c->m, 1) * c->B)) != SUPPY_OK) return s;
        if ((s = dalloc(c, &c->d_qq, (size_t)g * c->B)) != SUPPY_OK) return s;
        CK(cudaMemsetAsync(c->d_zero, 0, sizeof(float) * (size_t)std::max(c->m, 1) * c->B,
                           c->stream));
        if (c->m) CK(launch_to_float(c->d_rho, c->m, c->d_rhof, c->stream));
        note_launch(c);
    }
    CK(cudaStreamSynchronize(c->stream));
    return SUPPY_OK;
}

// EL / EMR after the column pass of block t (delta holds A^T(W d)): for EMR
// the row pass over q = A delta (zero bounds, so d = -q; the proximity
// machinery sums w_i q_i^2 with the multiplier ||a_i||^2), then the step.
suppy_status enqueue_ext_step(suppy_ctx* c, const suppy_params* p, int t, int npp) {
    int nqq = 0;
    if (c->mode == SUPPY_EMR) {
        // the launch writes one partial per CTA: check the buffer first
        nqq = c->use_tma ? c->seg_tgrid[t] : c->seg_grid[t];
        if (nqq > c->qq_cap) return fail(c, SUPPY_ECUDA, "q-pass launch exceeds its partials");
        if (c->use_tma) {
            StreamArgs q;
            std::memset(&q, 0, sizeof(q));
            q.info = c->d_rinfo;
            q.idx = c->d_col;
            q.val = c->d_val;
            q.cta_items = c->d_tpart + c->seg_tpart_off[t];
            q.tile = c->tile;
            q.stages = c->stages;
            q.err = c->d_err;
            q.wait_cycles = c->wait_cycles;
            q.l = c->d_zero;
            q.u = c->d_zero;
            q.wr = c->d_wr;
            q.x = c->d_delta;
            q.prox_mul = c->d_rhof;
            q.pp = c->d_qq;
            q.st = c->d_st;
            q.lam = 0.f;
            q.check_stop = 1;
            Timed tm{c, 0};
            CK(tm.begin());
            CK(launch_rows_tma(q, c->dt, c->tG, 0, c->tMap, c->seg_tgrid[t], c->stream));
            CK(tm.end());
        } else {
            SweepArgs q = row_args(c, t, 0.f);
            q.l = c->d_zero;
            q.u = c->d_zero;
            q.x = c->d_delta;
            q.prox_mul = c->d_rhof;
            q.pp = c->d_qq;
            Timed tm{c, 0};
            CK(tm.begin());
            if (c->B == 1) CK(launch_sweep(q, c->dt, c->G, c->maxe, 0, c->seg_grid[t], c->stream));
            else CK(launch_sweep_batched(q, c->dt, 0, c->seg_grid[t], c->stream));
            CK(tm.end());
        }
        note_launch(c);
    }
    ExtArgs e;
    e.x = c->d_x;
    e.delta = c->d_delta;
    e.lo = c->d_lo;
    e.hi = c->d_hi;
    e.box_len = c->box_len;
    e.n = c->n;
    e.B = c->B;
    e.st = c->d_st;
    e.method = (int)c->mode;
    e.pp = c->d_pp;
    e.npp = npp;
    e.qq = c->d_qq;
    e.nqq = nqq;
    e.part = c->d_xpart;
    e.ticket = c->d_xticket;
    e.tstep = c->d_tstep;
    e.lam = (float)p->lambda;
    Timed tm{c, 1};
    CK(tm.begin());
    CK(launch_ext_step(e, c->xgrid, c->stream));
    CK(tm.end());
    note_launch(c, 2);
    return SUPPY_OK;
}

// The CQ step's arguments for right-hand side b (x is n x B, one state, one
// set of projection partials and one target-space proximity per right-hand
// side).
DvcArgs dvc_args(suppy_ctx* c, bool check_stop, int b = 0) {
    DvcArgs a;
    a.rp = c->d_qrp;
    a.col = c->d_qcol;
    a.val = c->d_qval;
    a.cp = c->d_qcp;
    a.crow = c->d_qrow;
    a.cval = c->d_qcval;
    a.sptr = c->d_qsptr;
    a.sdvc = c->d_qsdvc;
    a.dvc = c->d_qdvc;
    a.x = c->d_x + b;
    a.xw = c->d_x + b;
    a.B = c->B;
    a.dose = c->d_dose;
    a.corr = c->d_qcorr;
    a.pd = c->d_qpd + (size_t)b * c->ndvc * kDvcCluster;
    a.target = c->d_target + b;
    a.st = check_stop ? c->d_st + b : nullptr;
    a.gamma = c->dvc_gamma;
    a.mq = c->mq;
    a.n = c->n;
    a.nstruct = c->nstruct;
    a.ndvc = c->ndvc;
    a.smem = c->dvc_smem;
    a.nnz = c->dvc_nnz;
    return a;
}

// The CQ step of a split problem: doses, projections onto the DVC sets and
// the target-space proximity, the correction x += gamma A_q^T corr.
suppy_status enqueue_cq_step(suppy_ctx* c) {
    Timed tm{c, 3};
    CK(tm.begin());
    // one right-hand side after the other: the dose and correction buffers
    // are shared, the stream orders the launches
    for (int b = 0; b < c->B_user; ++b) {
        const DvcArgs a = dvc_args(c, true, b);
        CK(launch_dvc_dose(a, c->stream));
        CK(launch_dvc_project(a, c->stream));
        CK(launch_dvc_apply(a, c->stream));
        note_launch(c, 4);
    }
    CK(tm.end());
    return SUPPY_OK;
}

// The tiled one-pass sweep: every block in one cooperative launch whose last
// CTA runs the epilogue (the proximity terms arrive scaled per block).
suppy_status enqueue_tile_sweep(suppy_ctx* c, const suppy_params* p, const StopParams& sp) {
    TileArgs a;
    std::memset(&a, 0, sizeof(a));
    a.stream = c->d_tstream;
    a.base = c->d_tbase;
    a.coff = c->d_tcoff;
    a.nsl = c->d_tnsl;
    a.rect = c->d_trect;
    a.chunk_blk = c->d_tcblk;
    a.blk_scale = c->d_tscale;
    a.K = c->tiK;
    a.W = c->gW;
    a.piece = c->tipiece;
    a.stages = c->tistages;
    a.tile_cap = c->ticap;
    a.W1 = c->tiW1;
    a.NC = c->tiNC;
    a.W2 = c->tiW2;
    a.cq = c->ticq;
    a.cstride = c->ticstride;
    a.l = c->d_l;
    a.u = c->d_u;
    a.wr = c->d_wr;
    a.x = c->d_x;
    a.lo = c->d_lo;
    a.hi = c->d_hi;
    a.zc = c->d_zc;
    a.box_len = c->box_len;
    a.m = c->m;
    a.r = c->d_tr;
    a.cnt = c->d_tcnt;
    a.sync = c->d_tsync;
    a.pp = c->d_tpp;
    a.st = c->d_st;
    a.err = c->d_err;
    a.wait_cycles = c->wait_cycles;
    a.lam = (float)p->lambda;
    EpiArgs e = epi_args(c, c->nseg - 1, sp);
    e.pp = c->d_tpp;
    e.npp = c->tiP;
    e.scale = 1.0;
    e.first_seg = 1;
    e.last_seg = 1;
    a.epi = e;
    {
        Timed tm{c, 0};
        CK(tm.begin());
        CK(launch_tile_sweep(a, c->dt, c->tiP, c->tismem, c->stream));
        CK(tm.end());
        note_launch(c);
    }
    c->k_upper += 1;
    if (c->evs.size() > 8192) return flush_timing(c);
    return SUPPY_OK;
}

// copies_fresh: the whole-GPU perturbation phase enqueued just before left
// the patch copies of x (a superiorized iteration), so the sweep need not
// make them.
suppy_status enqueue_sweep(suppy_ctx* c, const suppy_params* p, bool copies_fresh = false) {
    const StopParams sp = stop_params(c, p);
    suppy_status s;
    if (c->dvc_on && (s = enqueue_cq_step(c)) != SUPPY_OK) return s;
    if (c->strategy == 3) return enqueue_tile_sweep(c, p, sp);
    // EL / EMR: the row pass writes unrelaxed coefficients, the column pass
    // accumulates A^T(.) into delta, and the extrapolated step applies it
    const bool ext = (c->mode == SUPPY_EL || c->mode == SUPPY_EMR);
    const float lam_row = ext ? 1.f : (float)p->lambda;
    // one pass with the column-major accumulator (rows running down the image);
    // two passes with those rows read column-major (their indices and a copy
    // of x made before each block's row pass: x changes after every block)
    const bool tr_scatter = c->use_tma && c->strategy == 1 && c->scat == 1 && c->d_rowT && c->tr_on;
    const bool tr_gather = c->use_tma && c->strategy == 2 && c->d_colT && c->tr_on;
    // one pass in the patch numbering: patch indices, gathers from the patch
    // copies of x, both accumulators in patch layouts
    const bool patch = tr_scatter && c->tr_patch && c->d_colP;
    for (int t = 0; t < c->nseg; ++t) {
        SweepArgs a = row_args(c, t, lam_row);
        if (c->mode == SUPPY_EMR) a.coef_mul = c->d_rhof;
        const EpiArgs epi = epi_args(c, t, sp);
        if (c->use_tma) {
            StreamArgs sa;
            std::memset(&sa, 0, sizeof(sa));
            sa.info = c->d_rinfo;
            sa.idx = c->d_col;
            sa.val = c->d_val;
            sa.cta_items = c->d_tpart + c->seg_tpart_off[t];
            sa.tile = c->tile;
            sa.stages = c->stages;
            sa.err = c->d_err;
            sa.wait_cycles = c->wait_cycles;
            sa.l = c->d_l;
            sa.u = c->d_u;
            sa.wr = c->d_wr;
            sa.x = c->d_x;
            sa.delta = c->d_delta;
            sa.coef = (c->strategy == 2) ? c->d_coef : nullptr;
            sa.pp = c->d_pp;
            sa.st = c->d_st;
            sa.lam = lam_row;
            sa.coef_mul = (c->mode == SUPPY_EMR) ? c->d_rhof : nullptr;
            sa.check_stop = 1;
            if (tr_gather) {
                sa.idx = c->d_colT;
                sa.rowT = c->d_rowT;
                sa.xT = c->d_xT;
            }
            if (tr_scatter) {
                sa.rowT = c->d_rowT;
                sa.deltaT = c->d_deltaT;
                sa.recipW = c->recipW;
                sa.imgW = c->gW;
                sa.imgH = c->gH;
            }
            if (patch) {
                sa.idx = c->d_colP;
                sa.xW = c->d_xA;
                sa.xT = c->d_xB;
                sa.patch = 1;
                sa.imgWp = c->gWp;
            }
            EpiArgs e2 = epi;
            e2.npp = c->seg_tgrid[t];
            {
                // the row pass, after the column-major copy of x its steep
                // rows read (one timed bracket for both)
                Timed tm{c, 0};
                CK(tm.begin());
                if (tr_gather) {
                    CK(launch_transpose_image(c->d_x, c->d_xT, c->gH, c->gW, c->stream));
                    note_launch(c);
                }
                // the patch copies of x: at the sweep start (later blocks
                // find them written by the previous block's box step)
                // (a dose-volume CQ step before the row pass changes x)
                if (patch && t == 0 && !(copies_fresh && !c->dvc_on)) {
                    CK(launch_patch_image(c->d_x, c->d_xA, c->d_xB, c->gH, c->gW, c->gWp, c->stream));
                    note_launch(c);
                }
                CK(launch_rows_tma(sa, c->dt, c->tG, c->strategy == 2 ? 0 : 1, c->tMap, c->seg_tgrid[t],
                                   c->stream));
                CK(tm.end());
                note_launch(c);
            }
            if (c->strategy == 2) {
                StreamArgs ca;
                std::memset(&ca, 0, sizeof(ca));
                ca.info = c->d_cinfo + (size_t)t * c->n;
                ca.idx = c->d_ridx;
                ca.val = c->d_cval;
                ca.cta_items = c->d_ctpart + c->seg_ctpart_off[t];
                ca.tile = c->ctile;
                ca.stages = c->cstages;
                ca.err = c->d_err;
                ca.wait_cycles = c->wait_cycles;
                ca.coef_in = c->d_coef;
                ca.xw = c->d_x;
                ca.lo = c->d_lo;
                ca.hi = c->d_hi;
                ca.zc = c->d_zc;
                ca.delta_out = ext ? c->d_delta : nullptr;
                ca.box_len = c->box_len;
                ca.epi = e2;
                // without an extrapolated step the column pass's last CTA runs
                // the sweep epilogue (one launch fewer per sweep)
                const bool fuse_epi = !ext && e2.last_seg && c->d_cticket;
                ca.ticket = fuse_epi ? c->d_cticket : nullptr;
                {
                    Timed tm{c, 1};
                    CK(tm.begin());
                    CK(launch_cols_tma(ca, c->dt, c->tGc, c->tMapc, c->seg_ctgrid[t], c->stream));
                    CK(tm.end());
                    note_launch(c);
                }
                if (ext && (s = enqueue_ext_step(c, p, t, e2.npp)) != SUPPY_OK) return s;
                if (e2.last_seg && !fuse_epi) {
                    CK(launch_epilogue(e2, c->stream));
                    note_launch(c);
                }
            } else {
                FinalizeArgs f{};
                f.x = c->d_x;
                f.delta = c->d_delta;
                if (tr_scatter) {
                    f.deltaT = c->d_deltaT;
                    f.imgW = c->gW;
                    f.imgH = c->gH;
                }
                if (patch) {
                    f.patch = 1;
                    f.imgWp = c->gWp;
                    if (t + 1 < c->nseg) {
                        f.xA = c->d_xA;
                        f.xB = c->d_xB;
                    }
                }
                f.zc = c->d_zc;
                f.lo = c->d_lo;
                f.hi = c->d_hi;
                f.nB = (long long)c->n * c->B;
                f.B = c->B;
                f.box_len = c->box_len;
                f.epi = e2;
                Timed tm{c, 1};
                CK(tm.begin());
                CK(launch_finalize(f, c->grid_fin, c->stream));
                CK(tm.end());
                note_launch(c);
            }
        } else if (c->strategy == 2) {
            a.coef = c->d_coef;
            if ((s = launch_rows(c, a, 0, t)) != SUPPY_OK) return s;
            ColArgs ca;
            ca.cinfo = c->d_cinfo + (size_t)t * c->n;
            ca.ridx = c->d_ridx;
            ca.cval = c->d_cval;
            ca.coef = c->d_coef;
            ca.x = c->d_x;
            ca.lo = c->d_lo;
            ca.hi = c->d_hi;
            ca.zc = c->d_zc;
            ca.delta_out = ext ? c->d_delta : nullptr;
            ca.box_len = c->box_len;
            ca.B = c->B;
            ca.cpart = c->d_cpart + c->seg_cpart_off[t];
            ca.n = c->n;
            ca.m = c->m;
            ca.nnz = c->csc_len;
            ca.epi = epi;
            {
                Timed tm{c, 1};
                CK(tm.begin());
                CK(launch_colpass(ca, c->dt, c->Gc, c->seg_cgrid[t], c->stream));
                CK(tm.end());
                note_launch(c);
            }
            if (ext && (s = enqueue_ext_step(c, p, t, epi.npp)) != SUPPY_OK) return s;
            if (epi.last_seg) {
                CK(launch_epilogue(epi, c->stream));
                note_launch(c);
            }
        } else {
            if ((s = launch_rows(c, a, c->scat, t)) != SUPPY_OK) return s;
            FinalizeArgs f{};
            f.x = c->d_x;
            f.delta = c->d_delta;
            f.zc = c->d_zc;
            f.lo = c->d_lo;
            f.hi = c->d_hi;
            f.nB = (long long)c->n * c->B;
            f.B = c->B;
            f.box_len = c->box_len;
            f.epi = epi;
            Timed tm{c, 1};
            CK(tm.begin());
            CK(launch_finalize(f, c->grid_fin, c->stream));
            CK(tm.end());
            note_launch(c);
        }
    }
    c->k_upper += 1;
#ifdef SUPPY_CHECKED
    cudaStreamCaptureStatus capst = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(c->stream, &capst));
    if (capst == cudaStreamCaptureStatusNone) {
        CK(cudaStreamSynchronize(c->stream));
        int w[3];
        CK(read_check_word(w));
        if (w[0])
            return fail(c, SUPPY_EINVAL, "checked build: kernel check " + std::to_string(w[0]) +
                                             " failed at index " +
                                             std::to_string(((long long)w[2] << 32) | (unsigned)w[1]));
    }
#endif
    if (c->evs.size() > 8192) return flush_timing(c);
    return SUPPY_OK;
}

// copies: when not null, the phase also leaves x in the patch layouts of the
// one-pass sweep that follows it (whole-GPU phase, patch numbering), and
// *copies says whether it does.
suppy_status enqueue_perturb(suppy_ctx* c, const suppy_params* p, int record_only, bool* copies = nullptr) {
    PerturbArgs a;
    a.x = c->d_x;
    a.g = c->d_g;
    a.c32 = c->d_c32;
    a.c64 = c->d_c64;
    a.n = c->n;
    a.B = c->B;
    a.H = c->H;
    a.W = c->W;
    a.obj = (int)c->obj;
    a.gamma = p ? p->gamma : 0.0;
    a.alpha = p ? p->alpha : 0.0;
    a.log2_alpha = (p && p->alpha > 0.0) ? std::log2(p->alpha) : 0.0;
    a.n_red = p ? p->n_red : 0;
    a.max_trials = p ? p->max_trials : 0;
    a.restart_every = p ? p->restart_every : 0;
    a.adaptive = p ? p->adaptive : 0;
    a.f_ref = p ? p->f_ref : 0.0;
    a.st = c->d_st;
    a.record_only = record_only;
    a.part = c->d_wpart;
    a.ticket = c->d_ticket;
    a.err = c->d_err;
    a.wait_cycles = c->wait_cycles;
    a.pA = nullptr;
    a.pB = nullptr;
    a.pWp = 0;
    const bool patch_next = c->use_tma && c->strategy == 1 && c->scat == 1 && c->d_rowT && c->tr_on &&
                            c->tr_patch && c->d_colP && c->B == 1;
    if (copies) *copies = false;
    if (copies && patch_next && c->wide && !record_only) {
        a.pA = c->d_xA;
        a.pB = c->d_xB;
        a.pWp = c->gWp;
        *copies = true;
    }
    Timed tm{c, 2};
    CK(tm.begin());
    if (c->wide && !record_only) {
        CK(launch_perturb_wide(a, c->wide_grid, c->stream));
        note_launch(c);
    } else {
        CK(launch_perturb(a, c->perturb_cluster, c->stream));
        note_launch(c);
    }
    CK(tm.end());
#ifdef SUPPY_CHECKED
    cudaStreamCaptureStatus capst = cudaStreamCaptureStatusNone;
    CK(cudaStreamIsCapturing(c->stream, &capst));
    if (capst == cudaStreamCaptureStatusNone) {
        CK(cudaStreamSynchronize(c->stream));
        int w[3];
        CK(read_check_word_perturb(w));
        if (w[0])
            return fail(c, SUPPY_EINVAL, "checked build: perturbation check " + std::to_string(w[0]) +
                                             " failed at " + std::to_string(w[1]));
    }
#endif
    return SUPPY_OK;
}

// A streaming pass or the whole-GPU perturbation kernel whose bounded wait
// gave up leaves a nonzero error word; report (and clear) it at the next
// synchronizing call.
// The streaming passes' error word (sticky until read) travels to pinned
// host memory with the copies of a synchronizing call: enqueue the copy,
// synchronize once, then look.
suppy_status enqueue_err_copy(suppy_ctx* c) {
    if (c->d_err) CK(cudaMemcpyAsync(c->h_err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    return SUPPY_OK;
}

suppy_status reset_sync_words(suppy_ctx* c);

suppy_status err_after_sync(suppy_ctx* c) {
    if (c->bounds_pending) {
        // the checks of enqueued bounds updates (suppy_update_bounds_async)
        c->bounds_pending = false;
        const int f0 = c->h_bflags[0], f1 = c->h_bflags[1];
        if (f0 || f1) CK(cudaMemsetAsync(c->d_flags + 2, 0, 2 * sizeof(int), c->stream));
        if (f0) return fail(c, SUPPY_EINVAL, "an enqueued bounds update was rejected (l <= u and no NaN needed); the old bounds stay");
        if (f1) return fail(c, SUPPY_EINVAL, "an enqueued bounds update was rejected (a zero row needs l <= 0 <= u); the old bounds stay");
    }
    if (!c->d_err || !*c->h_err) return SUPPY_OK;
    *c->h_err = 0;
    CK(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
    suppy_status rs = reset_sync_words(c);
    if (rs != SUPPY_OK) return rs;
    return fail(c, SUPPY_ETIMEOUT, "a bounded device-side wait gave up (streaming pass, tiled sweep or whole-GPU perturbation barrier)");
}


suppy_status check_params(suppy_ctx* c, const suppy_params* p) {
    if (!p) return fail(c, SUPPY_EINVAL, "params is NULL");
    if (!(p->lambda > 0.0 && p->lambda < 2.0))
        return fail(c, SUPPY_EINVAL, "lambda must lie in (0, 2)");
    if (!(p->alpha > 0.0 && p->alpha <= 1.0) || !(p->gamma >= 0.0))
        return fail(c, SUPPY_EINVAL, "need gamma >= 0 and 0 < alpha <= 1");
    if (p->n_red < 0 || p->max_trials < 0 || p->max_sweeps < 0 || p->patience < 0 ||
        p->restart_every < 0)
        return fail(c, SUPPY_EINVAL, "negative count in params");
    if (p->adaptive < 0 || p->adaptive > 2)
        return fail(c, SUPPY_EINVAL, "adaptive must be 0, 1 or 2");
    if (p->adaptive == 2 && !std::isfinite(p->f_ref))
        return fail(c, SUPPY_EINVAL, "a fixed f_ref must be finite");
    return SUPPY_OK;
}

suppy_status read_flags(suppy_ctx* c, int* d_flags, int* h_flags, int count) {
    CK(cudaMemcpyAsync(h_flags, d_flags, sizeof(int) * count, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return SUPPY_OK;
}

// Launch shape of the row pass from the row-length mix: lanes per row and the
// row elements a lane keeps in registers between the dot product and the
// scatter (rows longer than G*maxe stream their tail twice).
void choose_row_shape(suppy_ctx* c, double mean_len, int max_len) {
    if (mean_len >= 192) c->G = 32;
    else if (mean_len >= 64) c->G = 16;
    else if (mean_len >= 20) c->G = 8;
    else c->G = 4;
    const int need = (max_len + c->G - 1) / c->G;
    if (c->strategy >= 2 || c->G == 4) c->maxe = 8;   // no scatter: registers only buffer loads
    else c->maxe = need <= 8 ? 8 : 16;
}

void choose_col_shape(suppy_ctx* c, double mean_col) {
    if (mean_col >= 128) c->Gc = 32;
    else if (mean_col >= 48) c->Gc = 16;
    else if (mean_col >= 12) c->Gc = 8;
    else c->Gc = 4;
}

// Work per group the launch aims for: enough rows (or columns) per group to
// amortize the group's start-up, capped by the resident grid.
constexpr long long kWorkPerGroup = 1024;

suppy_status build_row_partition(suppy_ctx* c) {
    int sms = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->dev));
    const int scat = (c->strategy == 2) ? 0 : c->scat;
    int bps = sweep_blocks_per_sm(c->dt, c->G, c->maxe, scat, c->B, c->n);
    if (bps <= 0) return fail(c, SUPPY_ECUDA, "no resident CTA for the chosen sweep shape");
    c->grid_sweep = sms * bps;
    const int gpc = (c->B > 1) ? kSweepThreads / 32 : kSweepThreads / c->G;
    c->groups = c->grid_sweep * gpc;
    c->seg_grid.assign(c->nseg, 0);
    c->seg_part_off.assign(c->nseg + 1, 0);
    for (int t = 0; t < c->nseg; ++t) {
        const long long work = c->rpref[c->seg_start[t + 1]] - c->rpref[c->seg_start[t]] +
                               16LL * (c->seg_start[t + 1] - c->seg_start[t]);
        long long g = (work + gpc * kWorkPerGroup - 1) / (gpc * kWorkPerGroup);
        // a shared-memory staged scatter flushes n values per CTA: fewer CTAs
        if (scat == 2) g = std::min<long long>(g, sms);
        c->seg_grid[t] = (int)std::max<long long>(1, std::min<long long>(g, c->grid_sweep));
        c->seg_part_off[t + 1] = c->seg_part_off[t] + (size_t)c->seg_grid[t] * gpc + 1;
    }
    std::vector<int> part(c->seg_part_off[c->nseg]);
    for (int t = 0; t < c->nseg; ++t)
        partition(c->rpref, c->seg_start[t], c->seg_start[t + 1], c->seg_grid[t] * gpc,
                  part.data() + c->seg_part_off[t]);
    if (c->d_part) dfree(c, c->d_part);
    c->d_part = nullptr;
    suppy_status s = dalloc(c, &c->d_part, part.size());
    if (s != SUPPY_OK) return s;
    CK(cudaMemcpyAsync(c->d_part, part.data(), part.size() * sizeof(int), cudaMemcpyHostToDevice,
                       c->stream));
    if (c->d_pp) dfree(c, c->d_pp);
    c->d_pp = nullptr;
    s = dalloc(c, &c->d_pp, (size_t)c->grid_sweep * c->B);
    if (s != SUPPY_OK) return s;
    long long vec4 = ((long long)c->n * c->B + 3) / 4;
    c->grid_fin = (int)std::min<long long>(std::max<long long>((vec4 + 255) / 256, 1), sms * 8LL);
    CK(cudaStreamSynchronize(c->stream));
    return SUPPY_OK;
}

suppy_status build_col_partition(suppy_ctx* c) {
    int sms = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->dev));
    int bps = colpass_blocks_per_sm(c->dt, c->Gc, c->B);
    if (bps <= 0) return fail(c, SUPPY_ECUDA, "no resident CTA for the column pass");
    c->grid_col = sms * bps;
    const int gpc = (c->B > 1) ? kSweepThreads / 32 : kSweepThreads / c->Gc;
    c->cgroups = c->grid_col * gpc;
    c->seg_cgrid.assign(c->nseg, 0);
    c->seg_cpart_off.assign(c->nseg + 1, 0);
    for (int t = 0; t < c->nseg; ++t) {
        const long long work = c->cpref[(size_t)t * (c->n + 1) + c->n];
        long long g = (work + gpc * kWorkPerGroup - 1) / (gpc * kWorkPerGroup);
        c->seg_cgrid[t] = (int)std::max<long long>(1, std::min<long long>(g, c->grid_col));
        c->seg_cpart_off[t + 1] = c->seg_cpart_off[t] + (size_t)c->seg_cgrid[t] * gpc + 1;
    }
    std::vector<int> part(c->seg_cpart_off[c->nseg]);
    std::vector<long long> pref(c->n + 1);
    for (int t = 0; t < c->nseg; ++t) {
        std::copy(c->cpref.begin() + (size_t)t * (c->n + 1),
                  c->cpref.begin() + (size_t)(t + 1) * (c->n + 1), pref.begin());
        partition(pref, 0, c->n, c->seg_cgrid[t] * gpc, part.data() + c->seg_cpart_off[t]);
    }
    if (c->d_cpart) dfree(c, c->d_cpart);
    c->d_cpart = nullptr;
    suppy_status s = dalloc(c, &c->d_cpart, part.size());
    if (s != SUPPY_OK) return s;
    CK(cudaMemcpyAsync(c->d_cpart, part.data(), part.size() * sizeof(int), cudaMemcpyHostToDevice,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return SUPPY_OK;
}

// Item ranges of the TMA-fed passes: per block, contiguous nnz-balanced item
// ranges, one per CTA, at least a few ring stages each.
void tma_partition(const std::vector<long long>& pref, int i0, int i1, int grid, int* out) {
    const long long w0 = pref[i0], w1 = pref[i1];
    out[0] = i0;
    int lo = i0;
    for (int g = 1; g < grid; ++g) {
        const long long target = w0 + (w1 - w0) * g / grid;
        int a = lo, b = i1;
        while (a < b) {
            const int mid = a + (b - a) / 2;
            if (pref[mid] < target) a = mid + 1;
            else b = mid;
        }
        out[g] = a;
        lo = a;
    }
    out[grid] = i1;
}

// The items one warp takes in a round (32/G of them) must fit the ring's
// window of S - 1 tiles.
bool group_fits(int G, int max_item, int tile, int stages) {
    return (long long)(32 / G) * max_item <= stream_max_item(tile, stages);
}

// Lanes per item of a streaming pass.  The items all consumer warps hold in
// one round must leave part of the ring to stream ahead of them; within that,
// narrow groups (several items per warp) keep more gathers in flight per lane.
// The budget (items of up to 90% of the ring in a round) matches the lane
// counts the tuner measured fastest on CT 384x384 and 512x512 (16 lanes where
// a budget of 45% gave 32).
int stream_group(double mean_len, int max_item, int tile, int stages) {
    const double budget = 0.9 * (double)stages * tile / (kStreamThreads / 32 - 1);
    int g = 4;
    while (g < 32 && ((32 / g) * mean_len > budget || !group_fits(g, max_item, tile, stages))) g *= 2;
    return g;
}

// Default ring and group shapes of the streaming passes: 4096-element tiles,
// as many stages as the shared-memory budget holds (6 for FP32 values, 9 for
// 16-bit values).
void default_tma_shape(suppy_ctx* c) {
    c->tile = c->ctile = kMaxTile;
    c->stages = c->cstages = stream_stages_for(c->dt, kMaxTile);
    c->tG = stream_group(c->m > 0 ? (double)c->nnz / c->m : 0.0, c->max_row, c->tile, c->stages);
    if (c->strategy == 2)
        c->tGc = stream_group((double)c->nnz / c->n / c->nseg, c->max_col, c->ctile, c->cstages);
}

// Caller-fixed shape (opts->stream_*), the same for both passes; zero fields
// keep the defaults.
void apply_stream_shape(suppy_ctx* c, int tile, int stages, int lanes) {
    if (tile) c->tile = c->ctile = tile;
    c->stages = c->cstages = stages ? stages : stream_stages_for(c->dt, c->tile);
    c->tG = lanes ? lanes
                  : stream_group(c->m > 0 ? (double)c->nnz / c->m : 0.0, c->max_row, c->tile, c->stages);
    if (c->strategy == 2)
        c->tGc = lanes ? lanes
                       : stream_group((double)c->nnz / c->n / c->nseg, c->max_col, c->ctile, c->cstages);
}

// Device row order inside each block: chunks of 32 consecutive rows are dealt
// out in a low-discrepancy order (chunk k takes source chunk k*S mod Q, S
// coprime to Q near Q/phi).  A simultaneous step does not depend on the row
// order, but the per-row cost of a pass does (how scattered the gathers of a
// row are): neighbouring rows of the input usually cost alike, so contiguous
// nnz-balanced CTA ranges of the input order can differ in time, while
// interleaved chunks give every CTA the same mix.  Rows inside a chunk keep
// their order, and with it the locality of their gathers.
void interleave_row_chunks(const std::vector<int>& seg_start, int m, std::vector<int>& perm,
                           std::vector<int>& seg_of_row) {
    constexpr int kChunk = 32, kMinChunks = 512;
    bool any = false;
    for (size_t t = 0; t + 1 < seg_start.size(); ++t)
        any |= (seg_start[t + 1] - seg_start[t]) >= kChunk * kMinChunks;
    if (!any) return;
    if (perm.empty()) {
        perm.resize(m);
        std::iota(perm.begin(), perm.end(), 0);
        seg_of_row.assign(m, 0);
    }
    std::vector<int> out(perm.size());
    for (size_t t = 0; t + 1 < seg_start.size(); ++t) {
        const int r0 = seg_start[t], r1 = seg_start[t + 1], len = r1 - r0;
        if (len < kChunk * kMinChunks) {
            std::copy(perm.begin() + r0, perm.begin() + r1, out.begin() + r0);
            continue;
        }
        const long long Q = (len + kChunk - 1) / kChunk;
        long long S = (long long)std::llround((double)Q * 0.6180339887498949);
        while (std::gcd(S, Q) != 1) ++S;
        int d = r0;
        for (long long k = 0; k < Q; ++k) {
            const long long q = (k * S) % Q;
            const int a = r0 + (int)(q * kChunk), b = std::min(r1, a + kChunk);
            for (int i = a; i < b; ++i) out[d++] = perm[i];
        }
    }
    perm.swap(out);
}

suppy_status build_tma_partitions(suppy_ctx* c) {
    int sms = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->dev));
    const int bps = stream_blocks_per_sm(c->dt, c->tile, c->stages);
    if (bps <= 0) return fail(c, SUPPY_ECUDA, "no resident CTA for the streaming passes");
    const long long per_cta_min = 4LL * c->tile;
    c->seg_tgrid.assign(c->nseg, 0);
    c->seg_tpart_off.assign(c->nseg + 1, 0);
    for (int t = 0; t < c->nseg; ++t) {
        const long long nz = c->rpref[c->seg_start[t + 1]] - c->rpref[c->seg_start[t]];
        const long long g = std::min<long long>((long long)sms * bps, (nz + per_cta_min - 1) / per_cta_min);
        c->seg_tgrid[t] = (int)std::max<long long>(1, g);
        c->seg_tpart_off[t + 1] = c->seg_tpart_off[t] + c->seg_tgrid[t] + 1;
    }
    std::vector<int> part(c->seg_tpart_off[c->nseg]);
    for (int t = 0; t < c->nseg; ++t)
        tma_partition(c->rpref, c->seg_start[t], c->seg_start[t + 1], c->seg_tgrid[t],
                      part.data() + c->seg_tpart_off[t]);
    if (c->d_tpart) dfree(c, c->d_tpart);
    c->d_tpart = nullptr;
    suppy_status s = dalloc(c, &c->d_tpart, part.size());
    if (s != SUPPY_OK) return s;
    CK(cudaMemcpyAsync(c->d_tpart, part.data(), part.size() * sizeof(int), cudaMemcpyHostToDevice,
                       c->stream));
    if (c->strategy == 2) {
        // columns: element prefix per block is the CSC offset (blocks are contiguous)
        c->seg_ctgrid.assign(c->nseg, 0);
        c->seg_ctpart_off.assign(c->nseg + 1, 0);
        std::vector<int2> cinfo((size_t)c->nseg * c->n);
        CK(cudaMemcpyAsync(cinfo.data(), c->d_cinfo, sizeof(int2) * cinfo.size(),
                           cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        std::vector<long long> pref(c->n + 1);
        std::vector<int> cpart;
        const int cbps = stream_blocks_per_sm(c->dt, c->ctile, c->cstages);
        if (cbps <= 0) return fail(c, SUPPY_ECUDA, "no resident CTA for the streaming column pass");
        const long long cper_cta_min = 4LL * c->ctile;
        for (int t = 0; t < c->nseg; ++t) {
            const int2* ci = cinfo.data() + (size_t)t * c->n;
            for (int j = 0; j < c->n; ++j) pref[j + 1] = pref[j] + pad4(ci[j].y);
            const long long nz = pref[c->n];
            const long long g = std::min<long long>((long long)sms * cbps, (nz + cper_cta_min - 1) / cper_cta_min);
            c->seg_ctgrid[t] = (int)std::max<long long>(1, g);
            c->seg_ctpart_off[t + 1] = c->seg_ctpart_off[t] + c->seg_ctgrid[t] + 1;
            const size_t base = cpart.size();
            cpart.resize(base + c->seg_ctgrid[t] + 1);
            tma_partition(pref, 0, c->n, c->seg_ctgrid[t], cpart.data() + base);
        }
        if (c->d_ctpart) dfree(c, c->d_ctpart);
        c->d_ctpart = nullptr;
        s = dalloc(c, &c->d_ctpart, cpart.size());
        if (s != SUPPY_OK) return s;
        CK(cudaMemcpyAsync(c->d_ctpart, cpart.data(), cpart.size() * sizeof(int),
                           cudaMemcpyHostToDevice, c->stream));
    }
    const int gmax = *std::max_element(c->seg_tgrid.begin(), c->seg_tgrid.end());
    if (gmax > c->grid_sweep) {
        if (c->d_pp) dfree(c, c->d_pp);
        c->d_pp = nullptr;
        c->grid_sweep = gmax;
        s = dalloc(c, &c->d_pp, (size_t)gmax * c->B);
        if (s != SUPPY_OK) return s;
    }
    CK(cudaStreamSynchronize(c->stream));
    return SUPPY_OK;
}

// CSC copy of the packed rows, one column range per block: a stable counting
// sort by column on the host (rows stay in device order inside a column) gives
// each CSR entry its CSC position; the device scatters rows and stored values.
suppy_status build_csc(suppy_ctx* c, const std::vector<int>& rp, const int* hcol,
                       const std::vector<int>& perm, const std::vector<int>& seg_of_row,
                       const std::vector<int2>& rinfo) {
    const int m = c->m, n = c->n, nseg = c->nseg;
    const size_t cells = (size_t)nseg * n;
    std::vector<long long> cnt(cells + 1, 0);
    for (int i = 0; i < m; ++i) {
        const int src = perm.empty() ? i : perm[i];
        const size_t base = (size_t)(seg_of_row.empty() ? 0 : seg_of_row[i]) * n;
        for (int e = rp[src]; e < rp[src + 1]; ++e) cnt[base + hcol[e]]++;
    }
    std::vector<int2> cinfo(cells);
    c->cpref.assign((size_t)nseg * (n + 1), 0);
    long long off = 0;
    long long real = 0;
    for (size_t k = 0; k < cells; ++k) {
        cinfo[k] = make_int2((int)off, (int)cnt[k]);
        const int t = (int)(k / n), j = (int)(k % n);
        long long* pr = c->cpref.data() + (size_t)t * (n + 1);
        pr[j + 1] = pr[j] + cnt[k] + 8;     // column work: entries plus a fixed cost
        real += cinfo[k].y;
        cnt[k] = off;                       // becomes the cursor
        off += pad4(cinfo[k].y);
    }
    if (off >= (1LL << 31) - kMaxTile - 16)
        return fail(c, SUPPY_EINVAL, "nnz (padded to four per column) must stay below 2^31");
    c->nnz_csc = real;
    c->csc_len = off;
    c->max_col = 0;
    for (size_t k = 0; k < cells; ++k) c->max_col = std::max(c->max_col, cinfo[k].y);
    std::vector<int> pos((size_t)std::max<long long>(c->nnz_pad, 1));
    for (int i = 0; i < m; ++i) {
        const int src = perm.empty() ? i : perm[i];
        const size_t base = (size_t)(seg_of_row.empty() ? 0 : seg_of_row[i]) * n;
        int d = rinfo[i].x;
        for (int e = rp[src]; e < rp[src + 1]; ++e, ++d) pos[d] = (int)(cnt[base + hcol[e]]++);
    }
    const size_t vsz = (c->dt == SUPPY_F32) ? 4 : 2;
    suppy_status s;
    if ((s = dalloc(c, &c->d_cinfo, cells)) != SUPPY_OK) return s;
    const size_t clen = (size_t)c->csc_len + kMaxTile + 16;
    if ((s = dalloc(c, &c->d_ridx, clen)) != SUPPY_OK) return s;
    {
        char* q = nullptr;
        if ((s = dalloc(c, &q, clen * vsz)) != SUPPY_OK) return s;
        c->d_cval = q;
    }
    // padding entries: index 0, value 0
    CK(cudaMemsetAsync(c->d_ridx, 0, sizeof(int) * clen, c->stream));
    CK(cudaMemsetAsync(c->d_cval, 0, vsz * clen, c->stream));
    if ((s = dalloc(c, &c->d_coef, (size_t)std::max(m, 1) * c->B)) != SUPPY_OK) return s;
    CK(cudaMemsetAsync(c->d_coef, 0, sizeof(float) * (size_t)std::max(m, 1) * c->B, c->stream));
    CK(cudaMemcpyAsync(c->d_cinfo, cinfo.data(), sizeof(int2) * cells, cudaMemcpyHostToDevice,
                       c->stream));
    int* d_pos = nullptr;
    CK(cudaMalloc(&d_pos, sizeof(int) * pos.size()));
    cudaError_t e = cudaMemcpyAsync(d_pos, pos.data(), sizeof(int) * pos.size(),
                                    cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = launch_csc_fill(c->d_rinfo, m, c->d_val, c->dt, d_pos, c->d_ridx, c->d_cval, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    cudaFree(d_pos);
    if (e != cudaSuccess)
        return fail(c, SUPPY_ECUDA, std::string("building the CSC copy: ") + cudaGetErrorString(e));
    note_launch(c);
    return SUPPY_OK;
}

void free_csc(suppy_ctx* c) {
    dfree(c, c->d_cinfo);
    dfree(c, c->d_ridx);
    dfree(c, c->d_cval);
    dfree(c, c->d_coef);
    dfree(c, c->d_cpart);
    c->d_cinfo = nullptr;
    c->d_ridx = nullptr;
    c->d_cval = nullptr;
    c->d_coef = nullptr;
    c->d_cpart = nullptr;
    c->nnz_csc = 0;
    c->csc_len = 0;
    c->cpref.clear();
    c->cpref.shrink_to_fit();
}

// Rows of A that run down the image (they span more image rows than image
// columns) scatter their corrections column-major, where their consecutive
// entries are neighbours: flags in device row order, the column-major
// accumulator, and the reciprocal of the image width for the index map.
suppy_status build_row_orientation(suppy_ctx* c, const std::vector<int>& rp, const int* hcol,
                                   const std::vector<int>& perm) {
    const int m = c->m, W = c->gW;
    c->recipW = ~0ULL / (unsigned long long)W + 1ULL;
    std::vector<unsigned char> flag(m, 0);
    long long nt = 0;
    for (int i = 0; i < m; ++i) {
        const int src = perm.empty() ? i : perm[i];
        int r0 = INT_MAX, r1 = -1, c0 = INT_MAX, c1 = -1;
        for (int k = rp[src]; k < rp[src + 1]; ++k) {
            const int r = hcol[k] / W, cc = hcol[k] - r * W;
            r0 = std::min(r0, r);
            r1 = std::max(r1, r);
            c0 = std::min(c0, cc);
            c1 = std::max(c1, cc);
        }
        if (r1 >= 0 && r1 - r0 > c1 - c0) {
            flag[i] = 1;
            ++nt;
        }
    }
    if (nt == 0) return SUPPY_OK;
    suppy_status s;
    if ((s = upload(c, flag, &c->d_rowT)) != SUPPY_OK) return s;
    // both accumulators cover the grid padded to multiples of 8 (the patch
    // numbering's lines); the padding is never added into
    c->gWp = (W + 7) & ~7;
    const size_t acc = std::max((size_t)c->n, (size_t)((c->gH + 7) & ~7) * (size_t)c->gWp);
    if (acc > c->acc_len) {
        dfree(c, c->d_delta);
        c->d_delta = nullptr;
        if ((s = dalloc(c, &c->d_delta, acc)) != SUPPY_OK) return s;
        CK(cudaMemsetAsync(c->d_delta, 0, sizeof(float) * acc, c->stream));
    }
    c->acc_len = acc;
    if ((s = dalloc(c, &c->d_deltaT, acc)) != SUPPY_OK) return s;
    CK(cudaMemsetAsync(c->d_deltaT, 0, sizeof(float) * acc, c->stream));
    c->trows = nt;
    CK(cudaStreamSynchronize(c->stream));   // the flags' host copy goes out of scope
    return SUPPY_OK;
}

// The two-pass row pass with the rows running down the image in the
// column-major numbering: a copy of the packed column indices with those
// rows' entries rewritten, and a column-major copy of x made before each row
// pass.
suppy_status build_col_transposed(suppy_ctx* c) {
    if (c->d_colT || !c->d_rowT) return SUPPY_OK;
    suppy_status s;
    const size_t rlen = (size_t)c->nnz_pad + kMaxTile + 16;
    if ((s = dalloc(c, &c->d_colT, rlen)) != SUPPY_OK) return s;
    if ((s = dalloc(c, &c->d_xT, (size_t)c->n)) != SUPPY_OK) return s;
    CK(cudaMemcpyAsync(c->d_colT, c->d_col, sizeof(int) * rlen, cudaMemcpyDeviceToDevice, c->stream));
    CK(launch_transposed_cols(c->d_rinfo, c->d_rowT, c->m, c->recipW, c->gW, c->gH, c->d_colT,
                              c->stream));
    note_launch(c);
    return SUPPY_OK;
}

// The one-pass sweep in the patch numbering: a copy of the packed column
// indices with every row's entries rewritten to its patch position (tall
// patches for the rows running down the image), and the two patch-layout
// copies of x its gathers read.
suppy_status build_col_patch(suppy_ctx* c) {
    if (c->d_colP || !c->d_rowT) return SUPPY_OK;
    suppy_status s;
    const size_t rlen = (size_t)c->nnz_pad + kMaxTile + 16;
    if ((s = dalloc(c, &c->d_colP, rlen)) != SUPPY_OK) return s;
    if ((s = dalloc(c, &c->d_xA, c->acc_len)) != SUPPY_OK) return s;
    if ((s = dalloc(c, &c->d_xB, c->acc_len)) != SUPPY_OK) return s;
    CK(cudaMemsetAsync(c->d_xA, 0, sizeof(float) * c->acc_len, c->stream));
    CK(cudaMemsetAsync(c->d_xB, 0, sizeof(float) * c->acc_len, c->stream));
    CK(cudaMemcpyAsync(c->d_colP, c->d_col, sizeof(int) * rlen, cudaMemcpyDeviceToDevice, c->stream));
    CK(launch_patch_cols(c->d_rinfo, c->d_rowT, c->m, c->recipW, c->gW, c->gWp, c->d_colP, c->stream));
    note_launch(c);
    return SUPPY_OK;
}

void free_col_patch(suppy_ctx* c) {
    dfree(c, c->d_colP);
    dfree(c, c->d_xA);
    dfree(c, c->d_xB);
    c->d_colP = nullptr;
    c->d_xA = nullptr;
    c->d_xB = nullptr;
}

void free_col_transposed(suppy_ctx* c) {
    dfree(c, c->d_colT);
    dfree(c, c->d_xT);
    c->d_colT = nullptr;
    c->d_xT = nullptr;
}

// Tiled one-pass sweep: plan the tiles and the chunked segment streams on the
// host (entries per column give nnz-balanced tiles; one CTA per SM), upload
// the tables, fill the streams on the device from the packed row copy, and
// size the ring to the shared memory left beside the tile's x and Delta.
void free_tile(suppy_ctx* c) {
    for (void* p : {(void*)c->d_tstream, (void*)c->d_tbase, (void*)c->d_tcoff, (void*)c->d_tnsl,
                    (void*)c->d_trect, (void*)c->d_tcblk, (void*)c->d_tscale, (void*)c->d_tr,
                    (void*)c->d_tcnt, (void*)c->d_tsync, (void*)c->d_tpp})
        if (p) dfree(c, p);
    c->d_tstream = nullptr;
    c->d_tbase = nullptr;
    c->d_tcoff = nullptr;
    c->d_tnsl = nullptr;
    c->d_trect = nullptr;
    c->d_tcblk = nullptr;
    c->d_tscale = nullptr;
    c->d_tr = nullptr;
    c->d_tcnt = nullptr;
    c->d_tsync = nullptr;
    c->d_tpp = nullptr;
    c->tiP = c->tiK = 0;
}

constexpr int kTileThreadsTotal = 1024;          // warps of a tiled-sweep CTA: 1 + W1 + W2
constexpr long long kTileMaxWords = 6144;        // unknowns of one tile (x and Delta in shared memory)
constexpr int kTileSmemMax = 227 * 1024;         // dynamic shared memory of one CTA
constexpr int kTileStaticSmem = 2048;            // the kernel's static shared memory, rounded up
constexpr int kTileGroupRows = 1;                // consecutive rows a chunk keeps together

// Why the tiled sweep cannot serve this context, or "" when it can.
std::string tile_ineligible(const suppy_ctx* c) {
    if (c->B != 1) return "the tiled sweep serves one right-hand side";
    if (c->mode != SUPPY_CIMMINO && c->mode != SUPPY_BIP && c->mode != SUPPY_DROP)
        return "the tiled sweep serves Cimmino, BIP and DROP sweeps";
    if (c->nnz == 0) return "the tiled sweep needs a nonempty matrix";
    return "";
}

suppy_status build_tile(suppy_ctx* c, const std::vector<int>& rp, const int* hcol,
                        const std::vector<int>& perm, const std::vector<int2>& rinfo,
                        int ring_req, int chunk_req, int group_req, bool* ok) {
    *ok = false;
    free_tile(c);
    int sms = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->dev));
    // ring: pieces of 8 KB, up to 24 of them (a caller-fixed ring is eight
    // pieces); the largest chunk of one tile is at most half the ring less a
    // piece, so two of them and a piece in flight fit
    int piece = 8192, want_stages = 24;
    if (ring_req) {
        piece = ring_req / 8;
        want_stages = 8;
    }
    const int vbytes = (c->dt == SUPPY_F32) ? 4 : 2;
    const long long max_chunk = (long long)(want_stages - 3) * piece / 2;
    TilePlanIn in;
    in.m = c->m;
    in.n = c->n;
    in.H = c->gH;
    in.W = c->gW;
    in.P = sms;
    in.vbytes = vbytes;
    in.perm = perm.empty() ? nullptr : perm.data();
    in.rp = rp.data();
    in.col = hcol;
    std::vector<int> rstart(c->m);
    for (int i = 0; i < c->m; ++i) rstart[i] = rinfo[i].x;
    in.row_start = rstart.data();
    in.seg_start = c->seg_start;
    in.max_chunk = max_chunk;
    in.chunk_target = chunk_req ? chunk_req : std::min<long long>(24 * 1024, in.max_chunk / 3);
    in.max_chunks = kTileMaxChunks;
    in.max_slices = 32;
    // a segment, its descriptor and padding fit well inside one chunk
    in.max_seg = (int)std::max<long long>(8, std::min<long long>(4096, (in.max_chunk / 4 - 32) / (vbytes + 2)));
    in.max_tile_words = kTileMaxWords;
    in.group_rows = group_req ? group_req : kTileGroupRows;
    TilePlan plan;
    std::string why;
    if (!plan_tiles(in, plan, why)) {
        c->err = why;
        return SUPPY_OK;   // not eligible: the caller keeps another strategy
    }
    // the ring takes the shared memory the tables and tiles leave
    const size_t fixed = tile_smem_bytes(0, plan.tile_cap, plan.K, kTileMaxStages, c->ticq,
                                         32 * plan.max_slices) + kTileStaticSmem;
    if (fixed >= (size_t)kTileSmemMax) {
        c->err = "tiled sweep: tiles and tables leave no room for the ring";
        return SUPPY_OK;
    }
    const int stages = std::min<int>(want_stages, (int)((kTileSmemMax - fixed) / piece));
    if (stages < 4 || (long long)(stages - 1) * piece < 2LL * plan.max_chunk) {
        c->err = "tiled sweep: the ring cannot hold two of the largest chunks";
        return SUPPY_OK;
    }
    c->tipiece = piece;
    c->tistages = stages;
    c->tiP = plan.P;
    c->tiK = plan.K;
    c->ticap = plan.tile_cap;
    c->timaxchunk = plan.max_chunk;
    c->tibytes = plan.bytes;
    c->tisegs = plan.segments;
    c->ticstride = 32 * std::max(1, plan.max_slices);
    c->tismem = tile_smem_bytes(c->tistages * c->tipiece, plan.tile_cap, plan.K, c->tistages,
                                c->ticq, c->ticstride);
    const int threads = 32 * (2 + c->tiW1 + c->tiNC + c->tiW2);
    if (tile_blocks_per_sm(c->dt, threads, c->tismem) < 1) {
        c->err = "tiled sweep: one CTA per SM is not resident";
        return SUPPY_OK;
    }
    suppy_status s;
    const int P = plan.P, K = plan.K;
    if ((s = dalloc(c, &c->d_tstream, (size_t)plan.bytes + 16)) != SUPPY_OK) return s;
    CK(cudaMemsetAsync(c->d_tstream, 0, (size_t)plan.bytes + 16, c->stream));
    if ((s = upload(c, plan.base, &c->d_tbase)) != SUPPY_OK) return s;
    if ((s = upload(c, plan.coff, &c->d_tcoff)) != SUPPY_OK) return s;
    if ((s = upload(c, plan.nsl, &c->d_tnsl)) != SUPPY_OK) return s;
    if ((s = upload(c, plan.rect, &c->d_trect)) != SUPPY_OK) return s;
    if ((s = upload(c, plan.chunk_blk, &c->d_tcblk)) != SUPPY_OK) return s;
    std::vector<double> scale(c->nseg);
    for (int t = 0; t < c->nseg; ++t) scale[t] = seg_scale(c, t);
    if ((s = upload(c, scale, &c->d_tscale)) != SUPPY_OK) return s;
    if ((s = dalloc(c, &c->d_tr, (size_t)2 * c->m)) != SUPPY_OK) return s;
    CK(cudaMemsetAsync(c->d_tr, 0, sizeof(float) * 2 * (size_t)c->m, c->stream));
    if ((s = dalloc(c, &c->d_tcnt, (size_t)K)) != SUPPY_OK) return s;
    CK(cudaMemsetAsync(c->d_tcnt, 0, sizeof(unsigned) * K, c->stream));
    if ((s = dalloc(c, &c->d_tsync, 2)) != SUPPY_OK) return s;
    CK(cudaMemsetAsync(c->d_tsync, 0, sizeof(unsigned) * 2, c->stream));
    if ((s = dalloc(c, &c->d_tpp, (size_t)P)) != SUPPY_OK) return s;
    // the streams: slice and lane records and the local column map, then the fill
    TileSliceRec* d_sl = nullptr;
    TileLaneRec* d_ln = nullptr;
    unsigned short* d_local = nullptr;
    if ((s = upload(c, plan.slices, &d_sl)) != SUPPY_OK) return s;
    if ((s = upload(c, plan.lanes, &d_ln)) != SUPPY_OK) return s;
    if ((s = upload(c, plan.local_of, &d_local)) != SUPPY_OK) return s;
    CK(launch_tile_fill(d_sl, (long long)plan.slices.size(), d_ln, c->d_val, c->dt, c->d_col, d_local,
                        c->d_tstream, c->stream));
    note_launch(c);
    CK(cudaStreamSynchronize(c->stream));
    dfree(c, d_sl);
    dfree(c, d_ln);
    dfree(c, d_local);
    *ok = true;
    c->err.clear();
    return SUPPY_OK;
}

// Clears the synchronisation words of the grid-wide kernels (tickets, chunk
// counters) after a bounded wait gave up: a CTA that left early may have left
// a count behind.
suppy_status reset_sync_words(suppy_ctx* c) {
    if (c->d_ticket) CK(cudaMemsetAsync(c->d_ticket, 0, 2 * sizeof(unsigned), c->stream));
    if (c->d_cticket) CK(cudaMemsetAsync(c->d_cticket, 0, sizeof(unsigned), c->stream));
    if (c->d_xticket) CK(cudaMemsetAsync(c->d_xticket, 0, sizeof(unsigned), c->stream));
    if (c->d_vticket) CK(cudaMemsetAsync(c->d_vticket, 0, sizeof(unsigned), c->stream));
    if (c->d_tcnt) CK(cudaMemsetAsync(c->d_tcnt, 0, sizeof(unsigned) * c->tiK, c->stream));
    if (c->d_tsync) CK(cudaMemsetAsync(c->d_tsync, 0, sizeof(unsigned), c->stream));
    return SUPPY_OK;
}

// Time nsweeps sweeps (after one untimed) of the current configuration on a
// scratch copy of the iterate and state (restored afterwards).
suppy_status time_config(suppy_ctx* c, float* ms_out, int nsweeps) {
    suppy_params p;
    suppy_params_default(&p);
    const size_t nB = (size_t)c->n * c->B;
    float* xs = nullptr;
    CK(cudaMalloc(&xs, sizeof(float) * nB));
    std::vector<RhsState> st(c->B);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMemcpyAsync(xs, c->d_x, sizeof(float) * nB, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(st.data(), c->d_st, sizeof(RhsState) * c->B, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    suppy_status s = SUPPY_OK;
    const bool was_timing = c->timing;
    c->timing = false;
    const int k_up = c->k_upper;
    if (e == cudaSuccess) s = enqueue_sweep(c, &p);
    if (e == cudaSuccess && s == SUPPY_OK) e = cudaEventRecord(e0, c->stream);
    for (int k = 0; k < nsweeps && e == cudaSuccess && s == SUPPY_OK; ++k) s = enqueue_sweep(c, &p);
    if (e == cudaSuccess && s == SUPPY_OK) e = cudaEventRecord(e1, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    float ms = 0.f;
    if (e == cudaSuccess && s == SUPPY_OK) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->d_x, xs, sizeof(float) * nB, cudaMemcpyDeviceToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->d_st, st.data(), sizeof(RhsState) * c->B, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess && c->d_delta)
        e = cudaMemsetAsync(c->d_delta, 0, sizeof(float) * std::max(nB, c->acc_len), c->stream);
    if (e == cudaSuccess && c->d_deltaT)
        e = cudaMemsetAsync(c->d_deltaT, 0, sizeof(float) * c->acc_len, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    c->timing = was_timing;
    c->k_upper = k_up;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(xs);
    if (s != SUPPY_OK) return s;
    if (e != cudaSuccess) return fail(c, SUPPY_ECUDA, std::string("tuning: ") + cudaGetErrorString(e));
    *ms_out = ms / 3.f;
    return SUPPY_OK;
}

// The TMA-fed passes serve one right-hand side with the L2-reduction scatter
// or the two-pass sweep, when every item fits in the ring's window.
bool tma_eligible(const suppy_ctx* c, int want) {
    if (want < 0) return false;                 // disabled by the caller
    if (c->B != 1) return false;
    if (c->strategy == 3) return false;         // the tiled sweep streams its own layout
    if (c->strategy == 1 && c->scat != 1) return false;
    if (c->max_row > stream_max_item(c->tile, c->stages)) return false;
    if (c->strategy == 2 && c->max_col > stream_max_item(c->ctile, c->cstages)) return false;
    return true;
}

// Measured choice of the streaming passes' shapes: every ring (tile length
// 1024 / 2048 / 4096 elements, the full shared-memory budget of stages or
// half of it), group width (4 .. 32 lanes per item) whose window holds a
// warp's round, and lane map (both, unless the caller fixed it) is timed on
// this matrix, first for the row pass, then for the column pass; the fastest
// stays.
suppy_status tune_tma(suppy_ctx* c, bool tune_map) {
    struct Shape {
        int G, tile, stages, map;
    };
    auto cands = [&](int max_item, int map_now) {
        std::vector<Shape> v;
        for (int tile : {1024, 2048, 4096}) {
            const int full = stream_stages_for(c->dt, tile);
            for (int st : {full, full / 2}) {
                if (st < 3 || stream_max_item(tile, st) < max_item) continue;
                for (int G : {4, 8, 16, 32})
                    if (group_fits(G, max_item, tile, st))
                        for (int map = tune_map ? 0 : map_now; map <= (tune_map ? 1 : map_now); ++map)
                            v.push_back({G, tile, st, map});
            }
        }
        return v;
    };
    suppy_status s;
    for (int pass = 0; pass < (c->strategy == 2 ? 2 : 1); ++pass) {
        const std::vector<Shape> v =
            cands(pass == 0 ? c->max_row : c->max_col, pass == 0 ? c->tMap : c->tMapc);
        Shape best{pass == 0 ? c->tG : c->tGc, pass == 0 ? c->tile : c->ctile,
                   pass == 0 ? c->stages : c->cstages, pass == 0 ? c->tMap : c->tMapc};
        float best_ms = 1e30f;
        std::vector<std::pair<float, Shape>> timed;
        for (const Shape& sh : v) {
            if (pass == 0) {
                c->tG = sh.G;
                c->tile = sh.tile;
                c->stages = sh.stages;
                c->tMap = sh.map;
            } else {
                c->tGc = sh.G;
                c->ctile = sh.tile;
                c->cstages = sh.stages;
                c->tMapc = sh.map;
            }
            if ((s = build_tma_partitions(c)) != SUPPY_OK) return s;
            float ms = 0.f;
            if ((s = time_config(c, &ms, 3)) != SUPPY_OK) return s;
            timed.push_back({ms, sh});
        }
        // the few fastest again, over more sweeps: three sweeps rank the
        // shapes, but neighbours within a few percent trade places from run
        // to run
        std::sort(timed.begin(), timed.end(),
                  [](const std::pair<float, Shape>& x, const std::pair<float, Shape>& y) {
                      return x.first < y.first;
                  });
        for (size_t k = 0; k < std::min<size_t>(timed.size(), 4); ++k) {
            const Shape& sh = timed[k].second;
            if (pass == 0) {
                c->tG = sh.G;
                c->tile = sh.tile;
                c->stages = sh.stages;
                c->tMap = sh.map;
            } else {
                c->tGc = sh.G;
                c->ctile = sh.tile;
                c->cstages = sh.stages;
                c->tMapc = sh.map;
            }
            if ((s = build_tma_partitions(c)) != SUPPY_OK) return s;
            float ms = 0.f;
            if ((s = time_config(c, &ms, 12)) != SUPPY_OK) return s;
            if (ms < best_ms) {
                best_ms = ms;
                best = sh;
            }
        }
        if (pass == 0) {
            c->tG = best.G;
            c->tile = best.tile;
            c->stages = best.stages;
            c->tMap = best.map;
        } else {
            c->tGc = best.G;
            c->ctile = best.tile;
            c->cstages = best.stages;
            c->tMapc = best.map;
        }
    }
    return build_tma_partitions(c);
}

suppy_status create_impl(const suppy_csr* A, const float* l, const float* u, const float* box_lo,
                         const float* box_hi, const suppy_opts* o, void* stream, suppy_ctx* c) {
    if (!A || !l || !u || !box_lo || !box_hi || !o)
        return fail(c, SUPPY_EINVAL, "NULL argument to suppy_create");
    if (A->m < 0 || A->n < 1 || A->nnz < 0 || !A->row_ptr || (A->nnz > 0 && (!A->col || !A->val)))
        return fail(c, SUPPY_EINVAL, "bad CSR shape or pointers");
    if (A->nnz >= (1LL << 31)) return fail(c, SUPPY_EINVAL, "nnz must be below 2^31");
    c->m = A->m;
    c->n = A->n;
    c->nnz = A->nnz;
    c->dt = o->a_dtype;
    if (c->dt != SUPPY_F32 && c->dt != SUPPY_BF16 && c->dt != SUPPY_F16 && c->dt != SUPPY_HALF_AUTO)
        return fail(c, SUPPY_EINVAL, "unknown a_dtype");
    c->mode = o->mode;
    if (c->mode != SUPPY_CIMMINO && c->mode != SUPPY_BIP && c->mode != SUPPY_DROP &&
        c->mode != SUPPY_EL && c->mode != SUPPY_EMR)
        return fail(c, SUPPY_EINVAL, "unknown mode");
    c->obj = o->obj;
    if ((int)c->obj < 0 || (int)c->obj > 5) return fail(c, SUPPY_EINVAL, "unknown objective");
    c->B_user = o->nrhs <= 0 ? 1 : o->nrhs;
    if (c->B_user > kMaxRhs) return fail(c, SUPPY_EINVAL, "nrhs must be at most 32");
    if (o->perturb_path < 0 || o->perturb_path > 2)
        return fail(c, SUPPY_EINVAL, "perturb_path must be 0, 1 or 2");
    {
        const int t = o->stream_tile, st = o->stream_stages, g = o->stream_lanes;
        if (t != 0 && (t < 256 || t > kMaxTile || (t & (t - 1))))
            return fail(c, SUPPY_EINVAL, "stream_tile must be 0 or a power of two in [256, 4096]");
        if (g != 0 && g != 4 && g != 8 && g != 16 && g != 32)
            return fail(c, SUPPY_EINVAL, "stream_lanes must be 0, 4, 8, 16 or 32");
        if (st != 0 && (st < 2 || st > stream_stages_for(o->a_dtype, t ? t : kMaxTile)))
            return fail(c, SUPPY_EINVAL, "stream_stages must be 0 or 2.. the shared-memory budget");
        if (o->stream_map < 0 || o->stream_map > 2)
            return fail(c, SUPPY_EINVAL, "stream_map must be 0, 1 or 2");
        if (o->stream_col_map < 0 || o->stream_col_map > 2)
            return fail(c, SUPPY_EINVAL, "stream_col_map must be 0, 1 or 2");
        if (o->scatter_transpose < -1 || o->scatter_transpose > 2)
            return fail(c, SUPPY_EINVAL, "scatter_transpose must be -1, 0, 1 or 2");
        if (o->tile_warps1 < 0 || o->tile_warps1 > 25)
            return fail(c, SUPPY_EINVAL, "tile_warps1 must lie in 0..25");
        const int rb = o->tile_ring_bytes;
        if (rb != 0 && (rb % 8 != 0 || (rb / 8) < 256 || (rb / 8) > 8192 || ((rb / 8) & (rb / 8 - 1))))
            return fail(c, SUPPY_EINVAL, "tile_ring_bytes must be 0 or 8 x a power of two in [256, 8192]");
        if (o->tile_chunk_bytes < 0) return fail(c, SUPPY_EINVAL, "tile_chunk_bytes must be >= 0");
        if (o->tile_group_rows < 0 || o->tile_group_rows > 1024)
            return fail(c, SUPPY_EINVAL, "tile_group_rows must lie in 0..1024");
    }
    c->B = 1;
    if (c->B_user > 1) {
        c->B = 4;
        while (c->B < c->B_user) c->B *= 2;
    }
    c->box_len = (int)o->box_len;
    if (o->box_len != 1 && o->box_len != (int64_t)A->n)
        return fail(c, SUPPY_EINVAL, "box_len must be 1 or n");
    if (c->obj == SUPPY_OBJ_TV_ISO || c->obj == SUPPY_OBJ_TV_ANISO) {
        if (o->img_h < 1 || o->img_w < 1 || (long long)o->img_h * o->img_w != A->n)
            return fail(c, SUPPY_EINVAL, "TV objectives need img_h * img_w == n");
        c->H = o->img_h;
        c->W = o->img_w;
    } else {
        c->H = 1;
        c->W = A->n;
    }
    // grid of the unknowns for the tiled sweep: the image when given (with
    // any objective), else one row of n
    if (o->img_h != 0 || o->img_w != 0) {
        if (o->img_h < 1 || o->img_w < 1 || (long long)o->img_h * o->img_w != A->n)
            return fail(c, SUPPY_EINVAL, "img_h * img_w must equal n when given");
        c->gH = o->img_h;
        c->gW = o->img_w;
    } else {
        c->gH = 1;
        c->gW = A->n;
    }
    if (c->obj == SUPPY_OBJ_LINEAR && !o->c_lin && !o->obj_rows)
        return fail(c, SUPPY_EINVAL, "linear objective needs c_lin or obj_rows");
    c->stream = static_cast<cudaStream_t>(stream);
    CK(cudaGetDevice(&c->dev));
    const int on_dev = A->on_device ? 1 : 0;
    const int m = c->m, n = c->n;

    // ---- host copy of row_ptr (partition, padding) and block structure
    std::vector<int> rp(m + 1);
    if (on_dev) {
        CK(cudaMemcpyAsync(rp.data(), A->row_ptr, sizeof(int) * (m + 1), cudaMemcpyDeviceToHost,
                           c->stream));
        CK(cudaStreamSynchronize(c->stream));
    } else {
        std::memcpy(rp.data(), A->row_ptr, sizeof(int) * (m + 1));
    }
    if (rp[0] != 0 || (long long)rp[m] != A->nnz)
        return fail(c, SUPPY_EINVAL, "row_ptr[0] must be 0 and row_ptr[m] must equal nnz");
    for (int i = 0; i < m; ++i)
        if (rp[i + 1] < rp[i]) return fail(c, SUPPY_EINVAL, "row_ptr must be nondecreasing");

    std::vector<int> perm;   // device row -> source row
    std::vector<int> seg_of_row;
    if (c->mode == SUPPY_BIP) {
        if (!o->block_of_row || o->nblocks < 1)
            return fail(c, SUPPY_EINVAL, "block-iterative mode needs block_of_row and nblocks >= 1");
        c->nseg = o->nblocks;
        std::vector<int> cnt(c->nseg + 1, 0);
        for (int i = 0; i < m; ++i) {
            const int t = o->block_of_row[i];
            if (t < 0 || t >= c->nseg) return fail(c, SUPPY_EINVAL, "block id out of range");
            cnt[t + 1]++;
        }
        for (int t = 0; t < c->nseg; ++t) cnt[t + 1] += cnt[t];
        c->seg_start.assign(cnt.begin(), cnt.end());
        perm.resize(m);
        seg_of_row.resize(m);
        std::vector<int> pos(cnt.begin(), cnt.end() - 1);
        for (int i = 0; i < m; ++i) {
            const int t = o->block_of_row[i];
            perm[pos[t]] = i;
            seg_of_row[pos[t]] = t;
            pos[t]++;
        }
    } else {
        c->nseg = 1;
        c->seg_start = {0, m};
    }
    interleave_row_chunks(c->seg_start, m, perm, seg_of_row);

    // row layout in device order (rows of a block contiguous)
    std::vector<int2> rinfo(m);
    c->rpref.assign(m + 1, 0);
    long long off = 0;
    int max_len = 0;
    for (int i = 0; i < m; ++i) {
        const int src = perm.empty() ? i : perm[i];
        const int len = rp[src + 1] - rp[src];
        rinfo[i] = make_int2((int)off, len);
        off += pad4(len);
        c->rpref[i + 1] = off;
        max_len = std::max(max_len, len);
    }
    if (off >= (1LL << 31) - kMaxTile - 16)
        return fail(c, SUPPY_EINVAL, "nnz (padded to four per row) must stay below 2^31");
    c->nnz_pad = off;

    TempGuard tg;
    tg.s = c->stream;
    int *s_rp = nullptr, *s_col = nullptr;
    float *s_val = nullptr, *s_l = nullptr, *s_u = nullptr, *s_lo = nullptr, *s_hi = nullptr;
    suppy_status s;
    const size_t mB = (size_t)m * c->B_user;
    if ((s = stage(c, A->row_ptr, (size_t)m + 1, on_dev, &s_rp, tg.v)) != SUPPY_OK) return s;
    if ((s = stage(c, A->col, (size_t)A->nnz, on_dev, &s_col, tg.v)) != SUPPY_OK) return s;
    if ((s = stage(c, A->val, (size_t)A->nnz, on_dev, &s_val, tg.v)) != SUPPY_OK) return s;
    if ((s = stage(c, l, mB, on_dev, &s_l, tg.v)) != SUPPY_OK) return s;
    if ((s = stage(c, u, mB, on_dev, &s_u, tg.v)) != SUPPY_OK) return s;
    if ((s = stage(c, box_lo, (size_t)c->box_len, on_dev, &s_lo, tg.v)) != SUPPY_OK) return s;
    if ((s = stage(c, box_hi, (size_t)c->box_len, on_dev, &s_hi, tg.v)) != SUPPY_OK) return s;

    // ---- validation on the device
    int* d_flags = nullptr;
    if ((s = dalloc(c, &d_flags, 8)) != SUPPY_OK) return s;
    CK(cudaMemsetAsync(d_flags, 0, 8 * sizeof(int), c->stream));
    // HALF_AUTO: the summed squared rounding-error bounds of FP16 and BF16
    double* d_err2 = nullptr;
    if (c->dt == SUPPY_HALF_AUTO) {
        if ((s = dalloc(c, &d_err2, 2)) != SUPPY_OK) return s;
        CK(cudaMemsetAsync(d_err2, 0, 2 * sizeof(double), c->stream));
    }
    CK(launch_validate_csr(s_rp, s_col, s_val, m, n, A->nnz, d_flags, c->stream, d_err2));
    CK(launch_validate_vec(s_l, (long long)mB, 1, d_flags + 1, 1, c->stream));
    CK(launch_validate_vec(s_u, (long long)mB, 1, d_flags + 1, 2, c->stream));
    CK(launch_validate_pair(s_l, s_u, (long long)mB, d_flags + 1, 4, c->stream));
    CK(launch_validate_vec(s_lo, c->box_len, 1, d_flags + 2, 1, c->stream));
    CK(launch_validate_vec(s_hi, c->box_len, 1, d_flags + 2, 2, c->stream));
    CK(launch_validate_pair(s_lo, s_hi, c->box_len, d_flags + 2, 4, c->stream));
    note_launch(c, 7);
    int hf[8];
    if ((s = read_flags(c, d_flags, hf, 3)) != SUPPY_OK) return s;
    if (hf[0] & 1) return fail(c, SUPPY_EINVAL, "row_ptr is not a valid CSR row pointer");
    if (hf[0] & 2) return fail(c, SUPPY_EINVAL, "column index outside [0, n)");
    if (hf[0] & 4) return fail(c, SUPPY_EINVAL, "matrix value is NaN or infinite");
    // 16 bits in the format whose rounding errors, summed in squares, are the
    // smaller one (FP16 only when no value overflows it)
    if (c->dt == SUPPY_HALF_AUTO) {
        double e2[2] = {0.0, 0.0};
        CK(cudaMemcpyAsync(e2, d_err2, sizeof(e2), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        dfree(c, d_err2);
        c->dt = (!(hf[0] & 8) && e2[0] <= e2[1]) ? SUPPY_F16 : SUPPY_BF16;
    }
    if (hf[1] & 3) return fail(c, SUPPY_EINVAL, "NaN in the slab bounds l or u");
    if (hf[1] & 4) return fail(c, SUPPY_EINVAL, "slab bounds need l <= u");
    if (hf[2] & 3) return fail(c, SUPPY_EINVAL, "NaN in the box bounds");
    if (hf[2] & 4) return fail(c, SUPPY_EINVAL, "box bounds need lo <= hi");

    // ---- packed matrix, row norms, weights
    const size_t vsz = (c->dt == SUPPY_F32) ? 4 : 2;
    if ((s = dalloc(c, &c->d_rinfo, (size_t)m)) != SUPPY_OK) return s;
    // slack of one ring stage: the streaming passes read whole stages
    const size_t rlen = (size_t)c->nnz_pad + kMaxTile + 16;
    if ((s = dalloc(c, &c->d_col, rlen)) != SUPPY_OK) return s;
    {
        char* q = nullptr;
        if ((s = dalloc(c, &q, rlen * vsz)) != SUPPY_OK) return s;
        c->d_val = q;
    }
    // padding entries: index 0, value 0
    CK(cudaMemsetAsync(c->d_col, 0, sizeof(int) * rlen, c->stream));
    CK(cudaMemsetAsync(c->d_val, 0, vsz * rlen, c->stream));
    if ((s = dalloc(c, &c->d_rho, (size_t)m)) != SUPPY_OK) return s;
    if ((s = dalloc(c, &c->d_wr, (size_t)m)) != SUPPY_OK) return s;
    if (m) CK(cudaMemcpyAsync(c->d_rinfo, rinfo.data(), sizeof(int2) * m, cudaMemcpyHostToDevice,
                              c->stream));
    int* d_perm_tmp = nullptr;
    int* d_seg = nullptr;
    if (!perm.empty()) {
        if ((s = dalloc(c, &c->d_perm, (size_t)m)) != SUPPY_OK) return s;
        CK(cudaMemcpyAsync(c->d_perm, perm.data(), sizeof(int) * m, cudaMemcpyHostToDevice,
                           c->stream));
        if ((s = stage(c, seg_of_row.data(), (size_t)m, 0, &d_seg, tg.v)) != SUPPY_OK) return s;
        d_perm_tmp = c->d_perm;
    }
    CK(launch_pack(s_rp, s_col, s_val, d_perm_tmp, c->d_rinfo, m, c->d_col, c->d_val, c->dt,
                   c->d_rho, c->stream));
    int* d_kept = nullptr;
    std::vector<int> zeros(c->nseg, 0);
    if ((s = stage(c, zeros.data(), zeros.size(), 0, &d_kept, tg.v)) != SUPPY_OK) return s;
    CK(launch_count_kept(c->d_rho, d_seg, m, d_kept, c->stream));
    c->seg_kept.assign(c->nseg, 0);
    CK(cudaMemcpyAsync(c->seg_kept.data(), d_kept, sizeof(int) * c->nseg, cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    note_launch(c, 2);
    c->m_kept = 0;
    for (int t = 0; t < c->nseg; ++t) c->m_kept += c->seg_kept[t];
    std::vector<double> segw(c->nseg, 0.0);
    for (int t = 0; t < c->nseg; ++t) {
        const int k = (c->mode == SUPPY_BIP) ? c->seg_kept[t] : c->m_kept;
        segw[t] = (c->mode == SUPPY_DROP) ? 1.0 : (k > 0 ? 1.0 / k : 0.0);
    }
    if (c->mode == SUPPY_DROP) {
        int* d_cnt = nullptr;
        if ((s = dalloc(c, &c->d_zc, (size_t)n)) != SUPPY_OK) return s;
        if ((s = dalloc(c, &d_cnt, (size_t)n)) != SUPPY_OK) return s;
        CK(launch_column_scaling(c->d_rinfo, c->d_col, c->d_val, c->dt, c->d_rho, m, n, d_cnt,
                                 c->d_zc, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        dfree(c, d_cnt);
        note_launch(c, 2);
    }
    double* d_segw = nullptr;
    if ((s = stage(c, segw.data(), segw.size(), 0, &d_segw, tg.v)) != SUPPY_OK) return s;
    CK(launch_weights(c->d_rho, d_seg, d_segw, m, c->d_wr, c->stream));

    // ---- bounds (device order, padded right-hand sides) and box
    if ((s = dalloc(c, &c->d_l, (size_t)m * c->B)) != SUPPY_OK) return s;
    if ((s = dalloc(c, &c->d_u, (size_t)m * c->B)) != SUPPY_OK) return s;
    CK(launch_permute_bounds(s_l, s_u, c->d_perm, m, c->B_user, c->B, c->d_l, c->d_u, c->stream));
    CK(cudaMemsetAsync(d_flags + 3, 0, sizeof(int), c->stream));
    CK(launch_zero_row_check(c->d_rho, c->d_l, c->d_u, m, c->B, d_flags + 3, c->stream));
    note_launch(c, 3);
    if ((s = read_flags(c, d_flags + 3, hf + 3, 1)) != SUPPY_OK) return s;
    if (hf[3]) return fail(c, SUPPY_EINVAL, "a zero row needs l <= 0 <= u");
    if ((s = dalloc(c, &c->d_lo, (size_t)c->box_len)) != SUPPY_OK) return s;
    if ((s = dalloc(c, &c->d_hi, (size_t)c->box_len)) != SUPPY_OK) return s;
    CK(cudaMemcpyAsync(c->d_lo, s_lo, sizeof(float) * c->box_len, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_hi, s_hi, sizeof(float) * c->box_len, cudaMemcpyDeviceToDevice, c->stream));

    // ---- iterate, correction, scratch, state
    const size_t nB = (size_t)n * c->B;
    if ((s = dalloc(c, &c->d_x, nB)) != SUPPY_OK) return s;
    if ((s = dalloc(c, &c->d_delta, nB)) != SUPPY_OK) return s;
    CK(cudaMemsetAsync(c->d_delta, 0, nB * sizeof(float), c->stream));
    c->acc_len = nB;
    CK(launch_box_init(c->d_x, c->d_lo, c->d_hi, (long long)nB, c->B, c->box_len, nullptr, 0,
                       c->stream));
    note_launch(c);
    int sms = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->dev));
    if (c->obj != SUPPY_OBJ_NONE) {
        if ((s = dalloc(c, &c->d_g, nB)) != SUPPY_OK) return s;
        // the whole-GPU phase pays off for one large image (a few fixed
        // microseconds of grid barriers and reductions against a single
        // cluster's per-pixel work); with two or more right-hand sides their
        // clusters already share the GPU, while the whole-GPU kernel takes
        // them one after the other, so the cluster path is faster; 2 forces
        // it, 1 disables it
        // (its pixel loops step an int index by the grid's thread count)
        const bool wide_fits = (long long)c->n + 2LL * sms * kPhaseThreads < (long long)INT_MAX;
        if (wide_fits && (o->perturb_path == 2 ||
                          (o->perturb_path == 0 && (long long)nB >= 65536 && c->B == 1))) {
            // a cooperative launch: every CTA must be resident at once
            const int per_sm = std::min(1, wide_phase_blocks_per_sm());
            if (per_sm < 1) return fail(c, SUPPY_ECUDA, "whole-GPU perturbation kernel cannot be resident");
            c->wide = true;
            c->wide_grid = (int)std::max<long long>(
                1, std::min<long long>((long long)per_sm * sms,
                                       ((long long)c->n + kPhaseThreads - 1) / kPhaseThreads));
            if ((s = dalloc(c, &c->d_wpart, wide_part_doubles(c->wide_grid))) != SUPPY_OK) return s;
            if ((s = dalloc(c, &c->d_ticket, 2)) != SUPPY_OK) return s;
            CK(cudaMemsetAsync(c->d_ticket, 0, 2 * sizeof(unsigned), c->stream));
        }
    }
    if ((s = dalloc(c, &c->d_st, (size_t)c->B)) != SUPPY_OK) return s;
    if ((s = dalloc(c, &c->d_out, (size_t)c->B)) != SUPPY_OK) return s;
    c->grid_obj = std::max(1, std::min(sms * 4, (n + 255) / 256));
    if ((s = dalloc(c, &c->d_objpart, (size_t)c->grid_obj * c->B)) != SUPPY_OK) return s;
    CK(cudaMallocHost(&c->h_out, sizeof(double) * kMaxRhs));
    CK(cudaMallocHost(&c->h_err, sizeof(int)));
    *c->h_err = 0;
    CK(cudaMallocHost(&c->h_bflags, 2 * sizeof(int)));
    c->h_bflags[0] = c->h_bflags[1] = 0;

    // ---- linear objective vector
    if (c->obj == SUPPY_OBJ_LINEAR) {
        if ((s = dalloc(c, &c->d_c64, (size_t)n)) != SUPPY_OK) return s;
        if ((s = dalloc(c, &c->d_c32, (size_t)n)) != SUPPY_OK) return s;
        if (o->obj_rows) {
            const suppy_csr* S = o->obj_rows;
            if (S->n != n || S->m < 1 || S->nnz < 0 || !S->row_ptr)
                return fail(c, SUPPY_EINVAL, "obj_rows must have n columns and at least one row");
            int *q_rp = nullptr, *q_col = nullptr;
            float* q_val = nullptr;
            const int sd = S->on_device ? 1 : 0;
            if ((s = stage(c, S->row_ptr, (size_t)S->m + 1, sd, &q_rp, tg.v)) != SUPPY_OK) return s;
            if ((s = stage(c, S->col, (size_t)S->nnz, sd, &q_col, tg.v)) != SUPPY_OK) return s;
            if ((s = stage(c, S->val, (size_t)S->nnz, sd, &q_val, tg.v)) != SUPPY_OK) return s;
            CK(cudaMemsetAsync(d_flags + 4, 0, sizeof(int), c->stream));
            CK(launch_validate_csr(q_rp, q_col, q_val, S->m, n, S->nnz, d_flags + 4, c->stream));
            if ((s = read_flags(c, d_flags + 4, hf + 4, 1)) != SUPPY_OK) return s;
            if (hf[4]) return fail(c, SUPPY_EINVAL, "obj_rows is not a valid CSR matrix");
            const int slices = std::max(1, std::min(512, S->m / 64));
            void* wq = nullptr;
            CK(cudaMalloc(&wq, sizeof(double) * (size_t)slices * n));
            tg.v.push_back(wq);
            double* work = static_cast<double*>(wq);
            CK(launch_colmean(q_rp, q_col, q_val, S->m, n, c->d_c64, c->d_c32, work, slices,
                              c->stream));
            note_launch(c, 3);
        } else {
            std::vector<float> hc(n);
            if (on_dev) {
                CK(cudaMemcpyAsync(hc.data(), o->c_lin, sizeof(float) * n, cudaMemcpyDeviceToHost,
                                   c->stream));
                CK(cudaStreamSynchronize(c->stream));
            } else {
                std::memcpy(hc.data(), o->c_lin, sizeof(float) * n);
            }
            std::vector<double> hd(hc.begin(), hc.end());
            for (double v : hd)
                if (!std::isfinite(v)) return fail(c, SUPPY_EINVAL, "c_lin must be finite");
            CK(cudaMemcpyAsync(c->d_c32, hc.data(), sizeof(float) * n, cudaMemcpyHostToDevice, c->stream));
            CK(cudaMemcpyAsync(c->d_c64, hd.data(), sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
            CK(cudaStreamSynchronize(c->stream));
        }
    }

    // ---- sweep strategy, launch shapes, partitions (K9 autotuner when tune)
    c->perturb_cluster = fit_perturb_cluster(choose_perturb_cluster(n, c->B), (int)c->obj, n, c->H, c->W);
    if ((s = ensure_hist(c, 1024)) != SUPPY_OK) return s;
    if ((s = reset_state(c)) != SUPPY_OK) return s;
    const double mean_len = m > 0 ? (double)A->nnz / m : 0.0;
    const double mean_col = (double)A->nnz / n / c->nseg;
    c->max_row = max_len;
    if ((s = dalloc(c, &c->d_err, 1)) != SUPPY_OK) return s;
    CK(cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream));
    if ((s = dalloc(c, &c->d_cticket, 1)) != SUPPY_OK) return s;
    CK(cudaMemsetAsync(c->d_cticket, 0, sizeof(unsigned), c->stream));
    const bool smem_ok = (c->B == 1) && (size_t)n * sizeof(float) <= 64 * 1024;
    // EL / EMR take the two-pass sweep (the column pass accumulates A^T(.));
    // their buffers exist before any timed candidate sweep
    const bool ext_mode = (c->mode == SUPPY_EL || c->mode == SUPPY_EMR);
    if (ext_mode && (s = prepare_ext(c)) != SUPPY_OK) return s;
    if (ext_mode && o->strategy == 3)
        return fail(c, SUPPY_EINVAL, "the tiled sweep serves Cimmino, BIP and DROP sweeps");
    const int want = ext_mode ? 2 : o->strategy;
    if (want < 0 || want > 3) return fail(c, SUPPY_EINVAL, "unknown strategy");
    const std::string tile_why = tile_ineligible(c);
    if (want == 3 && !tile_why.empty()) return fail(c, SUPPY_EINVAL, tile_why);
    const bool need_csc = (want == 2) || (want == 0 && (o->tune || !smem_ok));
    const bool tile_cand = tile_why.empty() && (want == 3 || (want == 0 && o->tune));
    // the one-pass scatter's column-major accumulator: one right-hand side
    // on an image grid, a strategy that may take the one-pass sweep
    const bool tr_grid = c->B == 1 && c->gH >= 2 && c->gW >= 2;
    if (o->scatter_transpose >= 1 && !tr_grid)
        return fail(c, SUPPY_EINVAL, "scatter_transpose needs an image grid and one right-hand side");
    if (o->scatter_transpose >= 1 && (long long)((c->gH + 7) & ~7) * ((c->gW + 7) & ~7) >= (1LL << 31))
        return fail(c, SUPPY_EINVAL, "scatter_transpose needs an image of fewer than 2^31 padded pixels");
    const bool tr_cand = tr_grid && o->scatter_transpose != -1 && !ext_mode && want != 3 &&
                         A->nnz > 0;
    std::vector<int> hcol_buf;
    const int* hcol = A->col;
    if ((need_csc || tile_cand || tr_cand) && on_dev) {
        hcol_buf.resize((size_t)std::max<long long>(A->nnz, 1));
        if (A->nnz)
            CK(cudaMemcpyAsync(hcol_buf.data(), A->col, sizeof(int) * A->nnz, cudaMemcpyDeviceToHost,
                               c->stream));
        CK(cudaStreamSynchronize(c->stream));
        hcol = hcol_buf.data();
    }
    if (need_csc) {
        if ((s = build_csc(c, rp, hcol, perm, seg_of_row, rinfo)) != SUPPY_OK) return s;
        choose_col_shape(c, mean_col);
        if ((s = build_col_partition(c)) != SUPPY_OK) return s;
    }
    bool tile_ok = false;
    if (tile_cand) {
        if (o->tile_warps1) {
            c->tiW1 = o->tile_warps1;
            c->tiW2 = kTileThreadsTotal / 32 - 2 - c->tiNC - c->tiW1;
        }
        if ((s = build_tile(c, rp, hcol, perm, rinfo, o->tile_ring_bytes, o->tile_chunk_bytes,
                            o->tile_group_rows, &tile_ok)) != SUPPY_OK)
            return s;
        if (want == 3 && !tile_ok) return fail(c, SUPPY_EINVAL, c->err);
    }
    if (tr_cand && (s = build_row_orientation(c, rp, hcol, perm)) != SUPPY_OK) return s;
    hcol_buf.clear();
    hcol_buf.shrink_to_fit();
    // tr: the one pass with L2 reductions takes the rows running down the
    // image column-major (1) or every row in the patch numbering (2)
    // (opts.scatter_transpose); untuned, it takes the patch numbering when
    // the grid allows it (on CT 512x512 its sweep measured 0.30 ms against
    // 0.42 ms column-major), and the tuner times every form
    struct Cand {
        int strategy, scat;
        int tr;   // 0 none, 1 column-major rows, 2 patch numbering (one pass)
    };
    const bool have_tr = c->d_rowT != nullptr;
    const int tr_one = !have_tr ? 0 : (o->scatter_transpose == 1 ? 1 : 2);
    std::vector<Cand> cands;
    if (want == 3) {
        cands.push_back({3, 0, 0});
    } else {
        if (want != 2) cands.push_back({1, smem_ok ? 2 : 1, smem_ok ? 0 : tr_one});
        if (want != 2 && !smem_ok && have_tr && o->tune && o->scatter_transpose == 0) {
            cands.push_back({1, 1, 0});
            cands.push_back({1, 1, 1});
        }
        if (want != 2 && smem_ok && o->tune) cands.push_back({1, 1, tr_one});
        if (need_csc) cands.push_back({2, 0, (o->scatter_transpose >= 1 && have_tr) ? 1 : 0});
        if (need_csc && have_tr && o->tune && o->scatter_transpose == 0) cands.push_back({2, 0, 1});
        if (tile_ok) cands.push_back({3, 0, 0});
    }
    Cand best = cands[0];
    if (want == 0 && !o->tune) best = smem_ok ? Cand{1, 2, 0} : Cand{2, 0, 0};
    const bool fixed_shape = o->stream_tile || o->stream_stages || o->stream_lanes;
    // Launch shape of a candidate: the register-fed sweep's row shape, then
    // (when the streamed passes serve it) their ring shapes and lane maps,
    // fixed by the caller, defaulted, or -- when tuning -- measured.
    struct Shapes {
        int tG, tile, stages, tMap, tGc, ctile, cstages, tMapc;
        bool use_tma;
    };
    auto set_up = [&](const Cand& cd, bool tune_streams) -> suppy_status {
        c->strategy = cd.strategy;
        c->scat = cd.scat;
        c->tr_on = cd.tr != 0;
        c->tr_patch = cd.tr == 2 && cd.strategy == 1;
        if (c->tr_patch) {
            suppy_status st2 = build_col_patch(c);
            if (st2 != SUPPY_OK) return st2;
        }
        if (cd.strategy == 2 && cd.tr) {
            suppy_status st2 = build_col_transposed(c);
            if (st2 != SUPPY_OK) return st2;
        }
        choose_row_shape(c, mean_len, max_len);
        suppy_status st;
        if ((st = build_row_partition(c)) != SUPPY_OK) return st;
        default_tma_shape(c);
        c->tMap = o->stream_map ? o->stream_map - 1 : kDefaultRowMap;
        c->tMapc = o->stream_col_map ? o->stream_col_map - 1
                                     : (o->stream_map ? o->stream_map - 1 : kDefaultColMap);
        if (fixed_shape) apply_stream_shape(c, o->stream_tile, o->stream_stages, o->stream_lanes);
        c->use_tma = tma_eligible(c, o->tma);
        if (fixed_shape && c->use_tma &&
            (!group_fits(c->tG, c->max_row, c->tile, c->stages) ||
             (c->strategy == 2 && !group_fits(c->tGc, c->max_col, c->ctile, c->cstages))))
            c->use_tma = false;
        if (c->use_tma) {
            if ((st = build_tma_partitions(c)) != SUPPY_OK) return st;
            if (tune_streams && !fixed_shape &&
                (st = tune_tma(c, o->stream_map == 0 && o->stream_col_map == 0)) != SUPPY_OK)
                return st;
        }
        return SUPPY_OK;
    };
    auto save = [&]() {
        return Shapes{c->tG, c->tile, c->stages, c->tMap, c->tGc, c->ctile, c->cstages, c->tMapc,
                      c->use_tma};
    };
    Shapes best_sh{};
    bool have_sh = false;
    if (o->tune && cands.size() > 1) {
        // every candidate strategy with its own streamed shapes tuned, so the
        // comparison is between the best form of each
        float best_ms = 1e30f;
        for (const Cand& cd : cands) {
            if ((s = set_up(cd, true)) != SUPPY_OK) return s;
            float ms = 0.f;
            if ((s = time_config(c, &ms, 12)) != SUPPY_OK) return s;
            if (ms < best_ms) {
                best_ms = ms;
                best = cd;
                best_sh = save();
                have_sh = true;
            }
        }
    }
    if (have_sh) {
        c->strategy = best.strategy;
        c->scat = best.scat;
        c->tr_on = best.tr != 0;
        c->tr_patch = best.tr == 2 && best.strategy == 1;
        choose_row_shape(c, mean_len, max_len);
        if ((s = build_row_partition(c)) != SUPPY_OK) return s;
        c->tG = best_sh.tG;
        c->tile = best_sh.tile;
        c->stages = best_sh.stages;
        c->tMap = best_sh.tMap;
        c->tGc = best_sh.tGc;
        c->ctile = best_sh.ctile;
        c->cstages = best_sh.cstages;
        c->tMapc = best_sh.tMapc;
        c->use_tma = best_sh.use_tma;
        if (c->use_tma && (s = build_tma_partitions(c)) != SUPPY_OK) return s;
    } else if ((s = set_up(best, o->tune != 0)) != SUPPY_OK) {
        return s;
    }
    if (c->strategy != 2 && c->d_cinfo) free_csc(c);
    if (!(c->strategy == 2 && c->tr_on) && c->d_colT) free_col_transposed(c);
    if (!(c->strategy == 1 && c->tr_patch) && c->d_colP) free_col_patch(c);
    if (c->strategy != 3 && c->d_tstream) free_tile(c);
    if ((s = reset_state(c)) != SUPPY_OK) return s;
    dfree(c, d_flags);
    CK(cudaStreamSynchronize(c->stream));
    CK(cudaGetLastError());
    return SUPPY_OK;
}

// Variance stopping rule: buffers on first use; the previous iterate starts
// as the current x whenever the state was reset.
suppy_status ensure_variance(suppy_ctx* c) {
    suppy_status s;
    const size_t nB = (size_t)c->n * c->B;
    if (!c->d_xprev) {
        int sms = 0;
        CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->dev));
        c->vgrid = (int)std::max<long long>(
            1, std::min<long long>(2LL * sms, ((long long)nB + kWideThreads - 1) / kWideThreads));
        if ((s = dalloc(c, &c->d_xprev, nB)) != SUPPY_OK) return s;
        if ((s = dalloc(c, &c->d_vpart, (size_t)c->vgrid * c->B * 2)) != SUPPY_OK) return s;
        if ((s = dalloc(c, &c->d_vticket, 1)) != SUPPY_OK) return s;
        CK(cudaMemsetAsync(c->d_vticket, 0, sizeof(unsigned), c->stream));
        c->xprev_stale = true;
    }
    if (c->xprev_stale) {
        CK(cudaMemcpyAsync(c->d_xprev, c->d_x, sizeof(float) * nB, cudaMemcpyDeviceToDevice,
                           c->stream));
        c->xprev_stale = false;
    }
    return SUPPY_OK;
}

suppy_status enqueue_variance(suppy_ctx* c, const suppy_params* p) {
    if (!(p->variance_tol > 0.0)) return SUPPY_OK;
    CK(launch_variance(c->d_x, c->d_xprev, c->n, c->B, c->d_st, c->d_vpart, c->d_vticket,
                       p->variance_tol, c->vgrid, c->stream));
    note_launch(c);
    return SUPPY_OK;
}

// Enqueue `iters` superiorized iterations.  With graphs, one iteration is
// captured once (per parameter set and buffer layout) and replayed; the
// captured kernels read every evolving quantity (iterate, state, counters)
// from device memory, so replays are exact.
suppy_status enqueue_iterations(suppy_ctx* c, const suppy_params* p, int iters) {
    suppy_status s;
    const bool use_graph = p->use_graphs && !c->timing;
    if (p->variance_tol > 0.0 && (s = ensure_variance(c)) != SUPPY_OK) return s;
    if (!use_graph) {
        for (int k = 0; k < iters; ++k) {
            bool fresh = false;
            if (c->obj != SUPPY_OBJ_NONE && (s = enqueue_perturb(c, p, 0, &fresh)) != SUPPY_OK) return s;
            if ((s = enqueue_sweep(c, p, fresh)) != SUPPY_OK) return s;
            if ((s = enqueue_variance(c, p)) != SUPPY_OK) return s;
        }
        return SUPPY_OK;
    }
    std::vector<char> key(sizeof(suppy_params) + sizeof(void*) + sizeof(int) * 2);
    std::memcpy(key.data(), p, sizeof(suppy_params));
    std::memcpy(key.data() + sizeof(suppy_params), &c->d_prox_hist, sizeof(void*));
    std::memcpy(key.data() + sizeof(suppy_params) + sizeof(void*), &c->hist_cap, sizeof(int));
    std::memcpy(key.data() + sizeof(suppy_params) + sizeof(void*) + sizeof(int), &c->strategy,
                sizeof(int));
    if (!c->graph || key != c->graph_key) {
        if (c->graph) {
            cudaGraphExecDestroy(c->graph);
            c->graph = nullptr;
        }
        const long long launches = c->launches;
        const int k_up = c->k_upper;
        // capture on a private stream (the caller's stream may be the legacy
        // default stream, which cannot be captured); the graph is then
        // launched on the caller's stream
        if (!c->cap_stream) CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
        CK(cudaStreamSynchronize(c->stream));
        cudaStream_t user = c->stream;
        c->stream = c->cap_stream;
        cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
            c->stream = user;
            cudaGetLastError();
            return fail(c, SUPPY_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        }
        s = SUPPY_OK;
        bool fresh = false;
        if (c->obj != SUPPY_OBJ_NONE) s = enqueue_perturb(c, p, 0, &fresh);
        if (s == SUPPY_OK) s = enqueue_sweep(c, p, fresh);
        if (s == SUPPY_OK) s = enqueue_variance(c, p);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(c->stream, &g);
        c->stream = user;
        if (s != SUPPY_OK) {
            if (g) cudaGraphDestroy(g);
            return s;
        }
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(c, SUPPY_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
        }
        e = cudaGraphInstantiate(&c->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            c->graph = nullptr;
            return fail(c, SUPPY_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
        }
        c->graph_launches = c->launches - launches;
        c->launches = launches;
        c->k_upper = k_up;
        c->graph_key = key;
    }
    for (int k = 0; k < iters; ++k) {
        CK(cudaGraphLaunch(c->graph, c->stream));
        c->launches += c->graph_launches;
        c->k_upper += 1;
    }
    return SUPPY_OK;
}

}  // namespace

// ---- internal interface of the serving runtime (serve.cu) -----------------
namespace suppy {

int ctx_slots(const suppy_ctx* c) { return c->B_user; }
int ctx_n(const suppy_ctx* c) { return c->n; }
int ctx_m(const suppy_ctx* c) { return c->m; }
cudaStream_t ctx_stream(const suppy_ctx* c) { return c->stream; }
size_t ctx_device_bytes(const suppy_ctx* c) { return c->dev_bytes; }
const char* ctx_error(const suppy_ctx* c) { return c->err.c_str(); }
void ctx_set_sweep_budget(suppy_ctx* c, int max_sweeps) { c->slot_max_sweeps = max_sweeps; }

// Load right-hand side b: bounds l, u (host, m values in the caller's row
// order) checked on the host, x[:, b] <- box(0), a fresh state.  Enqueued on
// the context's stream; nothing is synchronized.
suppy_status ctx_slot_load(suppy_ctx* c, int b, const float* l, const float* u) {
    if (b < 0 || b >= c->B_user) return fail(c, SUPPY_EINVAL, "slot out of range");
    const int m = c->m;
    suppy_status s;
    if (c->zero_row.empty() && m > 0) {
        std::vector<double> rho(m);
        std::vector<int> perm(m);
        CK(cudaMemcpyAsync(rho.data(), c->d_rho, sizeof(double) * m, cudaMemcpyDeviceToHost,
                           c->stream));
        if (c->d_perm)
            CK(cudaMemcpyAsync(perm.data(), c->d_perm, sizeof(int) * m, cudaMemcpyDeviceToHost,
                               c->stream));
        CK(cudaStreamSynchronize(c->stream));
        c->zero_row.assign(m, 0);
        for (int i = 0; i < m; ++i) c->zero_row[c->d_perm ? perm[i] : i] = rho[i] == 0.0;
    }
    for (int i = 0; i < m; ++i) {
        if (std::isnan(l[i]) || std::isnan(u[i]) || !(l[i] <= u[i]))
            return fail(c, SUPPY_EINVAL, "bounds need l <= u and no NaN");
        if (c->zero_row[i] && !(l[i] <= 0.f && 0.f <= u[i]))
            return fail(c, SUPPY_EINVAL, "a zero row needs l <= 0 <= u");
    }
    if (!c->d_slot_l) {
        if ((s = dalloc(c, &c->d_slot_l, (size_t)std::max(m, 1))) != SUPPY_OK) return s;
        if ((s = dalloc(c, &c->d_slot_u, (size_t)std::max(m, 1))) != SUPPY_OK) return s;
    }
    CK(cudaMemcpyAsync(c->d_slot_l, l, sizeof(float) * m, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_slot_u, u, sizeof(float) * m, cudaMemcpyHostToDevice, c->stream));
    CK(launch_load_column(c->d_slot_l, c->d_slot_u, c->d_perm, m, c->B, b, c->d_l, c->d_u,
                          c->stream));
    CK(launch_reset_column(c->d_x, c->d_lo, c->d_hi, c->n, c->B, b, c->box_len, c->d_st,
                           c->d_xprev, c->stream));
    note_launch(c, 2);
    return SUPPY_OK;
}

// Mark right-hand side b stopped (a free slot): every kernel skips it.
suppy_status ctx_slot_stop(suppy_ctx* c, int b) {
    if (b < 0 || b >= c->B) return fail(c, SUPPY_EINVAL, "slot out of range");
    CK(launch_set_stopped(c->d_st, b, c->stream));
    note_launch(c);
    return SUPPY_OK;
}

// Enqueue a copy of the per-RHS states (B_user entries) into host memory.
suppy_status ctx_states_async(suppy_ctx* c, RhsState* host) {
    CK(cudaMemcpyAsync(host, c->d_st, sizeof(RhsState) * c->B_user, cudaMemcpyDeviceToHost,
                       c->stream));
    return SUPPY_OK;
}

// Enqueue x[:, b] -> out (device, n floats).
suppy_status ctx_slot_extract(suppy_ctx* c, int b, float* out) {
    CK(launch_extract_column(c->d_x, c->n, c->B, b, out, c->stream));
    note_launch(c);
    return SUPPY_OK;
}

// Enqueue `iters` superiorized iterations of every active right-hand side.
suppy_status ctx_iterate(suppy_ctx* c, const suppy_params* p, int iters) {
    suppy_status s = check_params(c, p);
    if (s != SUPPY_OK) return s;
    // a served right-hand side never runs more than its sweep budget, so the
    // history stays that long however many requests pass through the slot
    const int need = c->slot_max_sweeps > 0 ? c->slot_max_sweeps : c->k_upper + iters;
    if ((s = ensure_hist(c, need)) != SUPPY_OK) return s;
    return enqueue_iterations(c, p, iters);
}

}  // namespace suppy

namespace {

void destroy_impl(suppy_ctx* c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    for (auto& t : c->evs) {
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    if (c->graph) cudaGraphExecDestroy(c->graph);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    for (auto& a : c->allocs) cudaFree(a.first);
    if (c->h_out) cudaFreeHost(c->h_out);
    if (c->h_err) cudaFreeHost(c->h_err);
    if (c->h_bflags) cudaFreeHost(c->h_bflags);
    delete c;
}

}  // namespace

extern "C" {

void suppy_params_default(suppy_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->lambda = 1.0;
    p->gamma = 0.5;
    p->alpha = 0.99;
    p->n_red = 1;
    p->max_trials = 100;
    p->restart_every = 0;
    p->max_sweeps = 500;
    p->check_every = 10;
    p->prox_abs = 1e-6;
    p->prox_rel = 1e-8;
    p->obj_rel = 1e-6;
    p->patience = 5;
    p->use_stopping = 0;
    p->use_graphs = 1;
}

suppy_status suppy_create(const suppy_csr* A, const float* l, const float* u,
                          const float* box_lo, const float* box_hi, const suppy_opts* opts,
                          void* stream, suppy_ctx** out) {
    if (!out) return fail(nullptr, SUPPY_EINVAL, "out is NULL");
    *out = nullptr;
    suppy_ctx* c = new (std::nothrow) suppy_ctx();
    if (!c) return fail(nullptr, SUPPY_ENOMEM, "host allocation failed");
    suppy_status s = create_impl(A, l, u, box_lo, box_hi, opts, stream, c);
    if (s != SUPPY_OK) {
        g_err = c->err;
        destroy_impl(c);
        return s;
    }
    *out = c;
    return SUPPY_OK;
}

void suppy_destroy(suppy_ctx* c) { destroy_impl(c); }

suppy_status suppy_set_stream(suppy_ctx* c, void* stream) {
    if (!c) return fail(nullptr, SUPPY_EINVAL, "ctx is NULL");
    CK(cudaStreamSynchronize(c->stream));
    c->stream = static_cast<cudaStream_t>(stream);
    return SUPPY_OK;
}

}  // extern "C"

namespace {

// New slab bounds, validated; the old ones stay when the call is rejected.
suppy_status load_bounds(suppy_ctx* c, const float* l, const float* u, int32_t on_device,
                         bool wait = true) {
    if (!c) return fail(nullptr, SUPPY_EINVAL, "ctx is NULL");
    if (!l || !u) return fail(c, SUPPY_EINVAL, "NULL bounds");
    const size_t mB = (size_t)c->m * c->B_user;
    suppy_status s;
    const float *s_l = l, *s_u = u;
    if (!on_device) {
        if (!c->d_stage_l) {
            if ((s = dalloc(c, &c->d_stage_l, mB)) != SUPPY_OK) return s;
            if ((s = dalloc(c, &c->d_stage_u, mB)) != SUPPY_OK) return s;
        }
        CK(cudaMemcpyAsync(c->d_stage_l, l, mB * sizeof(float), cudaMemcpyHostToDevice, c->stream));
        CK(cudaMemcpyAsync(c->d_stage_u, u, mB * sizeof(float), cudaMemcpyHostToDevice, c->stream));
        s_l = c->d_stage_l;
        s_u = c->d_stage_u;
    }
    // validation and the zero-row check read the new bounds in the caller's
    // row order; the permutation into the device layout is skipped on the
    // device when either failed, so a rejected call leaves the old bounds;
    // one synchronization reads both results
    if (!c->d_flags) {
        if ((s = dalloc(c, &c->d_flags, 4)) != SUPPY_OK) return s;
        CK(cudaMemsetAsync(c->d_flags, 0, 4 * sizeof(int), c->stream));
    }
    CK(cudaMemsetAsync(c->d_flags, 0, 2 * sizeof(int), c->stream));
    CK(launch_check_bounds(c->d_rho, s_l, s_u, c->d_perm, c->m, c->B_user, c->d_flags, c->stream));
    CK(launch_permute_bounds(s_l, s_u, c->d_perm, c->m, c->B_user, c->B, c->d_l, c->d_u, c->stream,
                             c->d_flags, 2));
    note_launch(c, 2);
    if (!wait) {
        // the sticky words collect every enqueued check until it is reported
        CK(cudaMemcpyAsync(c->h_bflags, c->d_flags + 2, 2 * sizeof(int), cudaMemcpyDeviceToHost,
                           c->stream));
        c->bounds_pending = true;
        return SUPPY_OK;
    }
    int hf[2] = {0, 0};
    if ((s = read_flags(c, c->d_flags, hf, 2)) != SUPPY_OK) return s;
    // earlier enqueued updates are reported first (their copy landed with
    // this synchronization); this check's own bits leave the sticky words
    const suppy_status pending = c->bounds_pending ? err_after_sync(c) : SUPPY_OK;
    CK(cudaMemsetAsync(c->d_flags + 2, 0, 2 * sizeof(int), c->stream));
    if (hf[0]) return fail(c, SUPPY_EINVAL, "bounds need l <= u and no NaN");
    if (hf[1]) return fail(c, SUPPY_EINVAL, "a zero row needs l <= 0 <= u");
    return pending;
}

}  // namespace

extern "C" {

suppy_status suppy_set_bounds(suppy_ctx* c, const float* l, const float* u, int32_t on_device) {
    suppy_status s = load_bounds(c, l, u, on_device);
    if (s != SUPPY_OK) return s;
    return reset_state(c);
}

suppy_status suppy_update_bounds(suppy_ctx* c, const float* l, const float* u, int32_t on_device) {
    return load_bounds(c, l, u, on_device);
}

suppy_status suppy_update_bounds_async(suppy_ctx* c, const float* l, const float* u,
                                       int32_t on_device) {
    return load_bounds(c, l, u, on_device, false);
}

}  // extern "C"

namespace {

// Order-preserving key of a float (the device's dose keys): larger value,
// larger key; -0 and +0 share a key.
uint32_t float_key(float f) {
    if (f == 0.0f) f = 0.0f;
    uint32_t b;
    std::memcpy(&b, &f, sizeof(b));
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

void free_dvc(suppy_ctx* c) {
    void* bufs[] = {c->d_qrp,   c->d_qcol,  c->d_qval, c->d_qcp,  c->d_qrow,
                    c->d_qcval, c->d_qsptr, c->d_qsdvc, c->d_qdvc, c->d_dose,
                    c->d_qcorr, c->d_qpd,   c->d_target};
    for (void* q : bufs) dfree(c, q);
    c->d_qrp = c->d_qcol = c->d_qcp = c->d_qrow = c->d_qsptr = c->d_qsdvc = nullptr;
    c->d_qval = c->d_qcval = c->d_dose = c->d_qcorr = nullptr;
    c->d_qdvc = nullptr;
    c->d_qpd = c->d_target = nullptr;
    c->dvc_on = false;
    c->dvc_smem = 0;
    c->mq = c->nstruct = c->ndvc = 0;
    c->dvc_gamma = 0.f;
}

template <typename T>
suppy_status to_host(suppy_ctx* c, const T* src, size_t count, int on_device, std::vector<T>& out) {
    out.resize(count);
    if (!count) return SUPPY_OK;
    if (!src) return fail(c, SUPPY_EINVAL, "a DVC matrix array is NULL");
    if (on_device) CK(cudaMemcpy(out.data(), src, count * sizeof(T), cudaMemcpyDeviceToHost));
    else std::memcpy(out.data(), src, count * sizeof(T));
    return SUPPY_OK;
}

suppy_status set_dvc_impl(suppy_ctx* c, const suppy_csr* A, const int32_t* sptr, int32_t nstruct,
                          const suppy_dvc* dvc, int32_t ndvc, double relax) {
    if (ndvc < 0) return fail(c, SUPPY_EINVAL, "ndvc must be >= 0");
    if (ndvc > 0) {
        if (!A || !sptr || !dvc) return fail(c, SUPPY_EINVAL, "Aq, structure_ptr and dvc must be given");
        if (A->n != c->n) return fail(c, SUPPY_EINVAL, "Aq must have the context's n columns");
        if (A->m < 1 || A->nnz < 0 || A->nnz >= (1LL << 31))
            return fail(c, SUPPY_EINVAL, "Aq needs m >= 1 rows and 0 <= nnz < 2^31");
        if (nstruct < 1) return fail(c, SUPPY_EINVAL, "nstruct must be >= 1");
        if (!(relax > 0.0 && relax < 2.0)) return fail(c, SUPPY_EINVAL, "relax must lie in (0, 2)");
    }
    const int mq = ndvc > 0 ? A->m : 0, n = c->n;
    std::vector<int> rp, col, st(nstruct > 0 && ndvc > 0 ? nstruct + 1 : 0);
    std::vector<float> val;
    std::vector<DvcDesc> desc;
    std::vector<int> sdvc;
    suppy_status s;
    if (ndvc > 0) {
        for (int k = 0; k <= nstruct; ++k) st[k] = sptr[k];
        if (st[0] != 0 || st[nstruct] != mq)
            return fail(c, SUPPY_EINVAL, "structure_ptr must start at 0 and end at m_q");
        for (int k = 0; k < nstruct; ++k)
            if (st[k + 1] < st[k]) return fail(c, SUPPY_EINVAL, "structure_ptr must be nondecreasing");
        if ((s = to_host(c, A->row_ptr, (size_t)mq + 1, A->on_device, rp)) != SUPPY_OK) return s;
        if (rp[0] != 0 || rp[mq] != A->nnz)
            return fail(c, SUPPY_EINVAL, "Aq row_ptr must start at 0 and end at nnz");
        for (int i = 0; i < mq; ++i)
            if (rp[i + 1] < rp[i]) return fail(c, SUPPY_EINVAL, "Aq row_ptr must be nondecreasing");
        if ((s = to_host(c, A->col, (size_t)A->nnz, A->on_device, col)) != SUPPY_OK) return s;
        if ((s = to_host(c, A->val, (size_t)A->nnz, A->on_device, val)) != SUPPY_OK) return s;
        for (long long e = 0; e < A->nnz; ++e) {
            if (col[e] < 0 || col[e] >= n) return fail(c, SUPPY_EINVAL, "Aq column index out of range");
            if (!std::isfinite(val[e])) return fail(c, SUPPY_EINVAL, "Aq values must be finite");
        }
        // DVCs grouped by structure, caller order kept inside a structure
        std::vector<int> order(ndvc);
        for (int j = 0; j < ndvc; ++j) {
            const suppy_dvc& q = dvc[j];
            if (q.kind != SUPPY_DVC_UPPER && q.kind != SUPPY_DVC_LOWER)
                return fail(c, SUPPY_EINVAL, "dvc kind must be SUPPY_DVC_UPPER or SUPPY_DVC_LOWER");
            if (q.structure < 0 || q.structure >= nstruct)
                return fail(c, SUPPY_EINVAL, "dvc structure out of range");
            if (!(q.volume >= 0.0 && q.volume <= 1.0))
                return fail(c, SUPPY_EINVAL, "dvc volume must lie in [0, 1]");
            if (!std::isfinite(q.d_ref)) return fail(c, SUPPY_EINVAL, "dvc d_ref must be finite");
            order[j] = j;
        }
        std::stable_sort(order.begin(), order.end(),
                         [&](int a, int b) { return dvc[a].structure < dvc[b].structure; });
        sdvc.assign(nstruct + 1, 0);
        for (int j = 0; j < ndvc; ++j) sdvc[dvc[j].structure + 1]++;
        for (int k = 0; k < nstruct; ++k) sdvc[k + 1] += sdvc[k];
        for (int j : order) {
            const suppy_dvc& q = dvc[j];
            const double N = (double)(st[q.structure + 1] - st[q.structure]);
            const double vN = q.volume * N;
            DvcDesc d;
            d.kind = q.kind;
            d.K = (int)(q.kind == SUPPY_DVC_UPPER ? std::floor(vN) : std::ceil(vN));
            d.orig = j;
            float lo_f = (float)q.d_ref, hi_f = (float)q.d_ref;
            if ((double)lo_f > q.d_ref) lo_f = std::nextafter(lo_f, -INFINITY);
            if ((double)hi_f < q.d_ref) hi_f = std::nextafter(hi_f, INFINITY);
            d.key_gt = float_key(lo_f);
            d.key_ge = float_key(hi_f);
            d.ref_hi = (float)q.d_ref;
            d.ref_lo = (float)(q.d_ref - (double)d.ref_hi);
            d.w = 1.0 / (double)ndvc;
            d.wf = (float)d.w;
            d.d_ref = q.d_ref;
            desc.push_back(d);
        }
    }
    // the old sets (if any) go; graphs captured with them too
    CK(cudaStreamSynchronize(c->stream));
    if (c->graph) {
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
        c->graph_key.clear();
    }
    free_dvc(c);
    if (ndvc == 0) return SUPPY_OK;

    // CSC copy (rows ascending inside a column)
    std::vector<int> cp(n + 1, 0), crow(A->nnz);
    std::vector<float> cval(A->nnz);
    for (long long e = 0; e < A->nnz; ++e) cp[col[e] + 1]++;
    for (int j = 0; j < n; ++j) cp[j + 1] += cp[j];
    {
        std::vector<int> cur(cp.begin(), cp.end() - 1);
        for (int i = 0; i < mq; ++i)
            for (int e = rp[i]; e < rp[i + 1]; ++e) {
                const int k = cur[col[e]]++;
                crow[k] = i;
                cval[k] = val[e];
            }
    }
    if ((s = upload(c, rp, &c->d_qrp)) != SUPPY_OK || (s = upload(c, col, &c->d_qcol)) != SUPPY_OK ||
        (s = upload(c, val, &c->d_qval)) != SUPPY_OK || (s = upload(c, cp, &c->d_qcp)) != SUPPY_OK ||
        (s = upload(c, crow, &c->d_qrow)) != SUPPY_OK || (s = upload(c, cval, &c->d_qcval)) != SUPPY_OK ||
        (s = upload(c, st, &c->d_qsptr)) != SUPPY_OK || (s = upload(c, sdvc, &c->d_qsdvc)) != SUPPY_OK ||
        (s = upload(c, desc, &c->d_qdvc)) != SUPPY_OK) {
        free_dvc(c);
        return s;
    }
    if ((s = dalloc(c, &c->d_dose, (size_t)mq)) != SUPPY_OK || (s = dalloc(c, &c->d_qcorr, (size_t)mq)) != SUPPY_OK ||
        (s = dalloc(c, &c->d_qpd, (size_t)ndvc * kDvcCluster * c->B)) != SUPPY_OK ||
        (s = dalloc(c, &c->d_target, (size_t)c->B)) != SUPPY_OK) {
        free_dvc(c);
        return s;
    }
    // step size: gamma = relax / sum_j w_j ||A_j||_F^2 (per-structure norms on the device)
    double* d_frob = nullptr;
    if ((s = dalloc(c, &d_frob, (size_t)nstruct * 33)) != SUPPY_OK) {
        free_dvc(c);
        return s;
    }
    cudaError_t fe = launch_dvc_frob(c->d_qrp, c->d_qval, c->d_qsptr, nstruct, d_frob + nstruct,
                                     d_frob, c->stream);
    note_launch(c, 2);
    std::vector<double> frob(nstruct);
    if (fe == cudaSuccess)
        fe = cudaMemcpyAsync(frob.data(), d_frob, sizeof(double) * nstruct, cudaMemcpyDeviceToHost,
                             c->stream);
    if (fe == cudaSuccess) fe = cudaMemsetAsync(c->d_target, 0, sizeof(double) * c->B, c->stream);
    if (fe == cudaSuccess) fe = cudaStreamSynchronize(c->stream);
    dfree(c, d_frob);
    if (fe != cudaSuccess) {
        free_dvc(c);
        cudaGetLastError();
        return fail(c, SUPPY_ECUDA, std::string("DVC norms: ") + cudaGetErrorString(fe));
    }
    double L = 0.0;
    for (int j = 0; j < ndvc; ++j) L += (1.0 / (double)ndvc) * frob[dvc[j].structure];
    if (!(L > 0.0)) {
        free_dvc(c);
        return fail(c, SUPPY_EINVAL, "the rows of the constrained structures are all zero");
    }
    c->mq = mq;
    c->nstruct = nstruct;
    c->ndvc = ndvc;
    c->dvc_gamma = (float)(relax / L);
    int max_rows = 0;
    for (int k = 0; k < nstruct; ++k) max_rows = std::max(max_rows, st[k + 1] - st[k]);
    c->dvc_smem = dvc_project_smem(max_rows);
    c->dvc_nnz = A->nnz;
    c->dvc_on = true;
    return SUPPY_OK;
}

}  // namespace

extern "C" {

suppy_status suppy_set_dvc(suppy_ctx* c, const suppy_csr* Aq, const int32_t* structure_ptr,
                           int32_t nstruct, const suppy_dvc* dvc, int32_t ndvc, double relax) {
    if (!c) return fail(nullptr, SUPPY_EINVAL, "ctx is NULL");
    return set_dvc_impl(c, Aq, structure_ptr, nstruct, dvc, ndvc, relax);
}

suppy_status suppy_dvc_dose(suppy_ctx* c, float* dose, int32_t on_device) {
    if (!c) return fail(nullptr, SUPPY_EINVAL, "ctx is NULL");
    if (!c->dvc_on) return fail(c, SUPPY_ESTATE, "no dose-volume constraints are set");
    if (!dose) return fail(c, SUPPY_EINVAL, "dose is NULL");
    // m_q x B, row-major like x: right-hand side b's doses at dose[i * B + b]
    const int Bu = c->B_user;
    for (int b = 0; b < Bu; ++b) {
        CK(launch_dvc_dose(dvc_args(c, false, b), c->stream));
        note_launch(c);
        CK(cudaMemcpy2DAsync(dose + b, sizeof(float) * Bu, c->d_dose, sizeof(float), sizeof(float),
                             (size_t)c->mq,
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                             c->stream));
    }
    if (!on_device) CK(cudaStreamSynchronize(c->stream));
    return SUPPY_OK;
}

suppy_status suppy_dvc_proximity(suppy_ctx* c, double* out) {
    if (!c) return fail(nullptr, SUPPY_EINVAL, "ctx is NULL");
    if (!c->dvc_on) return fail(c, SUPPY_ESTATE, "no dose-volume constraints are set");
    if (!out) return fail(c, SUPPY_EINVAL, "out is NULL");
    const int Bu = c->B_user;
    for (int b = 0; b < Bu; ++b) {
        const DvcArgs a = dvc_args(c, false, b);
        CK(launch_dvc_dose(a, c->stream));
        CK(launch_dvc_project(a, c->stream));
        note_launch(c, 3);
    }
    CK(cudaMemcpyAsync(c->h_out, c->d_target, sizeof(double) * Bu, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    for (int b = 0; b < Bu; ++b) out[b] = c->h_out[b];
    return SUPPY_OK;
}

suppy_status suppy_set_x(suppy_ctx* c, const float* x, int32_t on_device) {
    if (!c) return fail(nullptr, SUPPY_EINVAL, "ctx is NULL");
    if (!x) return fail(c, SUPPY_EINVAL, "x is NULL");
    TempGuard tg;
    tg.s = c->stream;
    float* s_x = nullptr;
    suppy_status s;
    if ((s = stage(c, x, (size_t)c->n * c->B_user, on_device, &s_x, tg.v)) != SUPPY_OK) return s;
    CK(launch_box_init(c->d_x, c->d_lo, c->d_hi, (long long)c->n * c->B, c->B, c->box_len, s_x,
                       c->B_user, c->stream));
    note_launch(c);
    return reset_state(c);
}

suppy_status suppy_get_x(suppy_ctx* c, float* x, int32_t on_device) {
    if (!c) return fail(nullptr, SUPPY_EINVAL, "ctx is NULL");
    if (!x) return fail(c, SUPPY_EINVAL, "x is NULL");
    const size_t cnt = (size_t)c->n * c->B_user;
    if (c->B == c->B_user) {
        CK(cudaMemcpyAsync(x, c->d_x, cnt * sizeof(float),
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
    } else {
        TempGuard tg;
        tg.s = c->stream;
        float* tmp = x;
        if (!on_device) {
            void* q = nullptr;
            CK(cudaMalloc(&q, cnt * sizeof(float)));
            tg.v.push_back(q);
            tmp = static_cast<float*>(q);
        }
        CK(launch_unpad_x(c->d_x, c->n, c->B, c->B_user, tmp, c->stream));
        note_launch(c);
        if (!on_device)
            CK(cudaMemcpyAsync(x, tmp, cnt * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    }
    if (on_device) return SUPPY_OK;
    suppy_status s = enqueue_err_copy(c);
    if (s != SUPPY_OK) return s;
    CK(cudaStreamSynchronize(c->stream));
    return err_after_sync(c);
}

suppy_status suppy_perturb(suppy_ctx* c, const suppy_params* p, int32_t* accepted) {
    if (!c) return fail(nullptr, SUPPY_EINVAL, "ctx is NULL");
    if (c->obj == SUPPY_OBJ_NONE) return fail(c, SUPPY_ESTATE, "the context has no objective");
    suppy_status s = check_params(c, p);
    if (s != SUPPY_OK) return s;
    if ((s = enqueue_perturb(c, p, 0)) != SUPPY_OK) return s;
    if (accepted) {
        std::vector<RhsState> st(c->B);
        CK(cudaMemcpyAsync(st.data(), c->d_st, sizeof(RhsState) * c->B, cudaMemcpyDeviceToHost,
                           c->stream));
        CK(cudaStreamSynchronize(c->stream));
        for (int b = 0; b < c->B_user; ++b) accepted[b] = st[b].stopped ? 0 : st[b].accepted_last;
    }
    return SUPPY_OK;
}

suppy_status suppy_sweep(suppy_ctx* c, const suppy_params* p, int32_t nsweeps) {
    if (!c) return fail(nullptr, SUPPY_EINVAL, "ctx is NULL");
    suppy_status s = check_params(c, p);
    if (s != SUPPY_OK) return s;
    if (nsweeps < 0) return fail(c, SUPPY_EINVAL, "nsweeps < 0");
    if ((s = ensure_hist(c, c->k_upper + nsweeps)) != SUPPY_OK) return s;
    for (int k = 0; k < nsweeps; ++k)
        if ((s = enqueue_sweep(c, p)) != SUPPY_OK) return s;
    return SUPPY_OK;
}

suppy_status suppy_proximity(suppy_ctx* c, double* out) {
    if (!c) return fail(nullptr, SUPPY_EINVAL, "ctx is NULL");
    if (!out) return fail(c, SUPPY_EINVAL, "out is NULL");
    for (int t = 0; t < c->nseg; ++t) {
        SweepArgs a = row_args(c, t, 0.f);
        a.check_stop = 0;
        if (c->B == 1) CK(launch_sweep(a, c->dt, c->G, c->maxe, 0, c->seg_grid[t], c->stream));
        else CK(launch_sweep_batched(a, c->dt, 0, c->seg_grid[t], c->stream));
        CK(launch_reduce_pp(c->d_pp, c->seg_grid[t], c->B, seg_scale(c, t), t > 0, c->d_out, c->stream));
        note_launch(c, 2);
    }
    CK(cudaMemcpyAsync(c->h_out, c->d_out, sizeof(double) * c->B, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    std::memcpy(out, c->h_out, sizeof(double) * c->B_user);
    return SUPPY_OK;
}

suppy_status suppy_objective(suppy_ctx* c, double* out) {
    if (!c) return fail(nullptr, SUPPY_EINVAL, "ctx is NULL");
    if (!out) return fail(c, SUPPY_EINVAL, "out is NULL");
    if (c->obj == SUPPY_OBJ_NONE) return fail(c, SUPPY_ESTATE, "the context has no objective");
    ObjArgs a;
    a.x = c->d_x;
    a.c64 = c->d_c64;
    a.n = c->n;
    a.B = c->B;
    a.H = c->H;
    a.W = c->W;
    a.obj = (int)c->obj;
    a.partial = c->d_objpart;
    CK(launch_objective(a, c->grid_obj, c->d_out, c->stream));
    note_launch(c, 2);
    CK(cudaMemcpyAsync(c->h_out, c->d_out, sizeof(double) * c->B, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    std::memcpy(out, c->h_out, sizeof(double) * c->B_user);
    return SUPPY_OK;
}

suppy_status suppy_run(suppy_ctx* c, const suppy_params* p, suppy_stats* out) {
    if (!c) return fail(nullptr, SUPPY_EINVAL, "ctx is NULL");
    suppy_status s = check_params(c, p);
    if (s != SUPPY_OK) return s;
    std::vector<RhsState> st(c->B);
    if ((s = ensure_hist(c, c->k_upper + p->max_sweeps)) != SUPPY_OK) return s;
    const int chunk = p->use_stopping ? std::max(1, p->check_every) : std::max(1, p->max_sweeps);
    int done = 0;
    while (done < p->max_sweeps) {
        const int todo = std::min(chunk, p->max_sweeps - done);
        if ((s = enqueue_iterations(c, p, todo)) != SUPPY_OK) return s;
        done += todo;
        if (p->use_stopping && done < p->max_sweeps) {
            CK(cudaMemcpyAsync(st.data(), c->d_st, sizeof(RhsState) * c->B, cudaMemcpyDeviceToHost,
                               c->stream));
            CK(cudaStreamSynchronize(c->stream));
            bool all = true;
            for (int b = 0; b < c->B_user; ++b) all = all && st[b].stopped;
            if (all) break;
        }
    }
    // the error word of the streaming passes and the statistics in one
    // synchronization; without statistics or the stopping rule the call only
    // enqueues, and the next synchronizing call reports the error word
    if ((s = enqueue_err_copy(c)) != SUPPY_OK) return s;
    if (!out && !p->use_stopping) return SUPPY_OK;
    if (out)
        CK(cudaMemcpyAsync(st.data(), c->d_st, sizeof(RhsState) * c->B, cudaMemcpyDeviceToHost,
                           c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if ((s = err_after_sync(c)) != SUPPY_OK) return s;
    if (out) {
        for (int b = 0; b < c->B_user; ++b) {
            out[b].sweeps = st[b].k;
            out[b].accepted = st[b].accepted_total;
            out[b].trials = st[b].trials_total;
            out[b].stopped = st[b].stopped;
            out[b].ell = st[b].ell;
            out[b].proximity = st[b].last_prox;
            out[b].objective = st[b].f_prev;
        }
    }
    return SUPPY_OK;
}

suppy_status suppy_history(suppy_ctx* c, int32_t rhs, double* prox, double* obj, int32_t cap,
                           int32_t* count) {
    if (!c) return fail(nullptr, SUPPY_EINVAL, "ctx is NULL");
    if (rhs < 0 || rhs >= c->B_user) return fail(c, SUPPY_EINVAL, "rhs out of range");
    RhsState st;
    CK(cudaMemcpyAsync(&st, c->d_st + rhs, sizeof(RhsState), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    const int k = std::min(st.k, c->hist_cap);
    const int cp = std::max(0, std::min(cap, k));
    if (prox && cp)
        CK(cudaMemcpyAsync(prox, c->d_prox_hist + (size_t)rhs * c->hist_cap, sizeof(double) * cp,
                           cudaMemcpyDeviceToHost, c->stream));
    if (obj && cp)
        CK(cudaMemcpyAsync(obj, c->d_obj_hist + (size_t)rhs * c->hist_cap, sizeof(double) * cp,
                           cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (count) *count = st.k;
    return SUPPY_OK;
}

namespace {
struct CkptHeader {
    uint64_t magic;
    int32_t version, n, m, B;
};
constexpr uint64_t kMagic = 0x5355505059434b31ULL;   // "SUPPYCK1"
}  // namespace

suppy_status suppy_get_state(suppy_ctx* c, void* buf, size_t* len) {
    if (!c) return fail(nullptr, SUPPY_EINVAL, "ctx is NULL");
    if (!len) return fail(c, SUPPY_EINVAL, "len is NULL");
    const size_t need = sizeof(CkptHeader) + sizeof(float) * (size_t)c->n * c->B +
                        sizeof(RhsState) * c->B;
    if (!buf) {
        *len = need;
        return SUPPY_OK;
    }
    if (*len < need) return fail(c, SUPPY_EINVAL, "checkpoint buffer too small");
    char* q = static_cast<char*>(buf);
    CkptHeader h{kMagic, 3, c->n, c->m, c->B};
    std::memcpy(q, &h, sizeof(h));
    CK(cudaMemcpyAsync(q + sizeof(h), c->d_x, sizeof(float) * (size_t)c->n * c->B,
                       cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(q + sizeof(h) + sizeof(float) * (size_t)c->n * c->B, c->d_st,
                       sizeof(RhsState) * c->B, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    *len = need;
    return SUPPY_OK;
}

suppy_status suppy_set_state(suppy_ctx* c, const void* buf, size_t len) {
    if (!c) return fail(nullptr, SUPPY_EINVAL, "ctx is NULL");
    if (!buf) return fail(c, SUPPY_EINVAL, "buf is NULL");
    const size_t need = sizeof(CkptHeader) + sizeof(float) * (size_t)c->n * c->B +
                        sizeof(RhsState) * c->B;
    if (len < need) return fail(c, SUPPY_EINVAL, "checkpoint too short");
    CkptHeader h;
    std::memcpy(&h, buf, sizeof(h));
    if (h.magic != kMagic || h.version != 3 || h.n != c->n || h.m != c->m || h.B != c->B)
        return fail(c, SUPPY_EINVAL, "checkpoint does not match this context");
    const char* q = static_cast<const char*>(buf);
    CK(cudaMemcpyAsync(c->d_x, q + sizeof(h), sizeof(float) * (size_t)c->n * c->B,
                       cudaMemcpyHostToDevice, c->stream));
    const RhsState* rs = reinterpret_cast<const RhsState*>(q + sizeof(h) + sizeof(float) * (size_t)c->n * c->B);
    std::vector<RhsState> st(rs, rs + c->B);
    c->k_upper = 0;
    c->xprev_stale = true;   // the variance rule continues from the restored iterate
    for (auto& r : st) c->k_upper = std::max(c->k_upper, r.k);
    CK(cudaMemcpyAsync(c->d_st, st.data(), sizeof(RhsState) * c->B, cudaMemcpyHostToDevice,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return SUPPY_OK;
}

suppy_status suppy_info_get(const suppy_ctx* cc, suppy_info* out) {
    suppy_ctx* c = const_cast<suppy_ctx*>(cc);
    if (!c) return fail(nullptr, SUPPY_EINVAL, "ctx is NULL");
    if (!out) return fail(c, SUPPY_EINVAL, "out is NULL");
    out->m = c->m;
    out->n = c->n;
    out->nrhs = c->B_user;
    out->m_kept = c->m_kept;
    out->nnz = c->nnz;
    out->nnz_csc = c->nnz_csc;
    out->nblocks = c->nseg;
    out->lanes_per_row = c->G;
    out->elems_in_regs = c->maxe;
    out->grid = c->seg_grid.empty() ? 0 : c->seg_grid[0];
    out->block = kSweepThreads;
    out->perturb_cluster = c->perturb_cluster;
    out->device_bytes = (int64_t)c->dev_bytes;
    out->strategy = c->strategy;
    out->scatter = c->strategy == 1 ? c->scat : 0;
    out->col_lanes = c->strategy == 2 ? c->Gc : 0;
    out->col_grid = (c->strategy == 2 && !c->seg_cgrid.empty()) ? c->seg_cgrid[0] : 0;
    out->tma = c->use_tma ? 1 : 0;
    out->tile = c->use_tma ? c->tile : 0;
    out->stages = c->use_tma ? c->stages : 0;
    out->col_tile = (c->use_tma && c->strategy == 2) ? c->ctile : 0;
    out->col_stages = (c->use_tma && c->strategy == 2) ? c->cstages : 0;
    out->tiles = c->strategy == 3 ? c->tiP : 0;
    out->chunks = c->strategy == 3 ? c->tiK : 0;
    out->tile_warps1 = c->strategy == 3 ? c->tiW1 : 0;
    out->tile_warps2 = c->strategy == 3 ? c->tiW2 : 0;
    out->tile_coef_warps = c->strategy == 3 ? c->tiNC : 0;
    out->tile_ring = c->strategy == 3 ? c->tistages * c->tipiece : 0;
    out->tile_stream_bytes = c->strategy == 3 ? c->tibytes : 0;
    out->tile_segments = c->strategy == 3 ? c->tisegs : 0;
    out->a_dtype = (int32_t)c->dt;
    out->transposed_rows = (((c->strategy == 1 && c->scat == 1 && c->d_rowT) ||
                             (c->strategy == 2 && c->d_colT)) && c->use_tma && c->tr_on) ? c->trows : 0;
    out->scatter_patch = (out->transposed_rows > 0 && c->strategy == 1 && c->tr_patch) ? 1 : 0;
    out->map = c->use_tma ? c->tMap + 1 : 0;
    out->col_map = (c->use_tma && c->strategy == 2) ? c->tMapc + 1 : 0;
    if (c->use_tma) {
        out->grid = c->seg_tgrid[0];
        out->block = kStreamThreads;
        out->lanes_per_row = c->tG;
        if (c->strategy == 2) {
            out->col_grid = c->seg_ctgrid[0];
            out->col_lanes = c->tGc;
        }
    }
    return SUPPY_OK;
}

suppy_status suppy_set_wait_limit(suppy_ctx* c, int64_t cycles) {
    if (!c) return fail(nullptr, SUPPY_EINVAL, "ctx is NULL");
    if (cycles < 0) return fail(c, SUPPY_EINVAL, "the wait limit must be >= 0");
    c->wait_cycles = cycles ? (long long)cycles : kDefaultWaitCycles;
    // a captured iteration holds the old budget in its launch arguments
    if (c->graph) {
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
        c->graph_key.clear();
    }
    return SUPPY_OK;
}

suppy_status suppy_timing_enable(suppy_ctx* c, int32_t enable) {
    if (!c) return fail(nullptr, SUPPY_EINVAL, "ctx is NULL");
    suppy_status s = flush_timing(c);
    if (s != SUPPY_OK) return s;
    c->timing = enable != 0;
    for (int k = 0; k < 4; ++k) {
        c->timing_ms[k] = 0.0;
        c->timing_n[k] = 0;
    }
    return SUPPY_OK;
}

suppy_status suppy_kernel_time(suppy_ctx* c, int32_t kind, double* total_ms, int64_t* launches) {
    if (!c) return fail(nullptr, SUPPY_EINVAL, "ctx is NULL");
    if (kind < 0 || kind > 3) return fail(c, SUPPY_EINVAL, "kernel kind must be 0, 1, 2 or 3");
    suppy_status s = flush_timing(c);
    if (s != SUPPY_OK) return s;
    if (total_ms) *total_ms = c->timing_ms[kind];
    if (launches) *launches = c->timing_n[kind];
    return SUPPY_OK;
}

int64_t suppy_launch_count(const suppy_ctx* c) { return c ? c->launches : 0; }

const char* suppy_last_error(const suppy_ctx* c) {
    return c ? c->err.c_str() : g_err.c_str();
}

const char* suppy_version(void) { return "suppy-gb300 0.1 (sm_103a)"; }

}  // extern "C"
