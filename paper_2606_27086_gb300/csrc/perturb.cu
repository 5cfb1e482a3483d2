// Perturbation phase of Algorithm 1 (nonascending subgradient steps with the
// power-law step size beta = gamma * alpha^l of Sec. 2.1.2) and the objective
// evaluations it needs: isotropic TV (Eq. (TV)) with the Combettes/Penfold
// subgradient, anisotropic TV, and the linear mean dose f = c.x (Sec. 2.3.3).
//
// One thread-block cluster owns one right-hand side.  Every trial needs a
// global decision f(z) <= f(y); the cluster makes it without the host: each
// CTA reduces its FP64 partial in a fixed order, the partials are exchanged
// through distributed shared memory after a hardware cluster barrier, and
// every CTA sums them in the same order -- so all CTAs take the same decision
// and the run is bitwise reproducible.  The trial loop is bounded by
// max_trials, so the kernel always ends.
#include <cooperative_groups.h>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace suppy {

#ifdef SUPPY_CHECKED
__device__ int g_check_p[3];
__device__ __noinline__ bool check_fail_p(int tag, long long idx) {
    if (atomicCAS(&g_check_p[0], 0, tag) == 0) {
        g_check_p[1] = (int)(idx & 0xffffffffLL);
        g_check_p[2] = (int)(idx >> 32);
    }
    return false;
}
#define PCHECKED(cond, tag, idx) ((cond) ? true : check_fail_p((tag), (long long)(idx)))
#else
#define PCHECKED(cond, tag, idx) true
#endif

cudaError_t read_check_word_perturb(int* out3) {
#ifdef SUPPY_CHECKED
    cudaError_t e = cudaMemcpyFromSymbol(out3, g_check_p, sizeof(int) * 3);
    if (e != cudaSuccess) return e;
    int z[3] = {0, 0, 0};
    return cudaMemcpyToSymbol(g_check_p, z, sizeof(int) * 3);
#else
    out3[0] = out3[1] = out3[2] = 0;
    return cudaSuccess;
#endif
}

namespace {

// Strided view of right-hand side b of an n x B row-major array.  Reads go
// through L2 only (ld.global.cg): other CTAs of the cluster rewrite these
// vectors between the passes of one launch, and L2 is the coherence point.
struct Vec {
    float* p;
    int B;
    __device__ __forceinline__ float operator()(int j) const { return __ldcg(p + (size_t)j * B); }
};

// z = y - s * g, the trial point, computed identically wherever it is used.
__device__ __forceinline__ float trial(float y, float g, float s) { return __fmaf_rn(-s, g, y); }

// Trial step beta / ||g|| with beta = gamma alpha^l (Sec. 2.1.2).  The
// exponent is split in FP64, alpha^l = 2^(l log2 alpha) = 2^k 2^f with k an
// integer and f in [0, 1), and the rest is FP32, so the relative error stays
// at a few FP32 ulps for any l.  (FP64 on GB300 costs tens of cycles per
// dependent operation; an FP64 pow() takes microseconds, on the critical
// path of every trial.)
__device__ __forceinline__ float trial_scale(double gamma, double log2_alpha, long long ell,
                                             float inv_gnorm) {
    const double e = (double)ell * log2_alpha;
    const double k = floor(e);
    const float f = (float)(e - k);
    return (float)gamma * ldexpf(exp2f(f), (int)k) * inv_gnorm;
}

// Adaptive step of Nikazad et al. (Sec. 2.1.2): the reference value of a
// phase that starts at f_start -- fixed, or the lowest phase-start objective
// so far, this one included -- and beta / ||g|| = (f - f_ref) / ||g||^2, the
// subgradient projection onto the level set of f's linearisation.
__device__ __forceinline__ double adaptive_ref(const PerturbArgs& a, const RhsState& st,
                                               double f_start) {
    if (a.adaptive == 2) return a.f_ref;
    return st.has_ref ? fmin(st.f_ref, f_start) : f_start;
}

__device__ __forceinline__ float adaptive_scale(double fy, double f_ref, double gg) {
    return fy > f_ref ? (float)((fy - f_ref) / gg) : 0.f;
}

// Objectives whose value is a sum of per-element terms (no stencil): the
// linear mean dose c.x, ||x||_1 and ||x||_2^2.
__device__ __forceinline__ bool elementwise(int obj) {
    return obj == SUPPY_OBJ_LINEAR || obj == SUPPY_OBJ_L1 || obj == SUPPY_OBJ_L2;
}

// Term and (sub)gradient of ||x||_1 (sign, 0 at 0) and ||x||_2^2 (2x).
__device__ __forceinline__ float norm_term(int obj, float v) {
    return obj == SUPPY_OBJ_L1 ? fabsf(v) : v * v;
}
__device__ __forceinline__ float norm_grad(int obj, float v) {
    if (obj == SUPPY_OBJ_L1) return (v > 0.f) ? 1.f : ((v < 0.f) ? -1.f : 0.f);
    return 2.f * v;
}

// Objective term owned by pixel p (FP64 result; TV terms are FP32 then widened).
template <class Y>
__device__ __forceinline__ double obj_term(int obj, int p, int H, int W, const double* c64,
                                           const Y& y) {
    if (obj == SUPPY_OBJ_LINEAR) return c64[p] * (double)y(p);
    if (obj == SUPPY_OBJ_L1 || obj == SUPPY_OBJ_L2) return (double)norm_term(obj, y(p));
    const int i = p / W, j = p - i * W;
    const float y0 = y(p);
    if (obj == SUPPY_OBJ_TV_ISO) {
        if (i < H - 1 && j < W - 1) {
            const float dx = y(p + W) - y0, dy = y(p + 1) - y0;
            return (double)sqrtf(dx * dx + dy * dy);
        }
        return 0.0;
    }
    float t = 0.f;   // anisotropic
    if (i < H - 1) t += fabsf(y(p + W) - y0);
    if (j < W - 1) t += fabsf(y(p + 1) - y0);
    return (double)t;
}

__device__ __forceinline__ float sgnf(float v) { return (v > 0.f) ? 1.f : ((v < 0.f) ? -1.f : 0.f); }

// Subgradient component at pixel p (gather form of the term-wise derivatives).
template <class Y>
__device__ __forceinline__ float subgrad(int obj, int p, int H, int W, const float* c32,
                                         const Y& y) {
    if (obj == SUPPY_OBJ_LINEAR) return c32[p];
    if (obj == SUPPY_OBJ_L1 || obj == SUPPY_OBJ_L2) return norm_grad(obj, y(p));
    const int i = p / W, j = p - i * W;
    const float y0 = y(p);
    float g = 0.f;
    if (obj == SUPPY_OBJ_TV_ISO) {
        // term (i, j): d/dX[i,j] = -(dx + dy) / phi
        if (i < H - 1 && j < W - 1) {
            const float dx = y(p + W) - y0, dy = y(p + 1) - y0;
            const float phi = sqrtf(dx * dx + dy * dy);
            if (phi > 0.f) g -= (dx + dy) / phi;
        }
        // term (i-1, j): d/dX[i,j] = dx' / phi'  (X[i,j] is its X[i'+1,j])
        if (i > 0 && j < W - 1) {
            const float ym = y(p - W);
            const float dx = y0 - ym, dy = y(p - W + 1) - ym;
            const float phi = sqrtf(dx * dx + dy * dy);
            if (phi > 0.f) g += dx / phi;
        }
        // term (i, j-1): d/dX[i,j] = dy'' / phi''  (X[i,j] is its X[i,j'+1])
        if (j > 0 && i < H - 1) {
            const float yl = y(p - 1);
            const float dx = y(p + W - 1) - yl, dy = y0 - yl;
            const float phi = sqrtf(dx * dx + dy * dy);
            if (phi > 0.f) g += dy / phi;
        }
        return g;
    }
    if (i < H - 1) g -= sgnf(y(p + W) - y0);
    if (i > 0) g += sgnf(y0 - y(p - W));
    if (j < W - 1) g -= sgnf(y(p + 1) - y0);
    if (j > 0) g += sgnf(y0 - y(p - 1));
    return g;
}

// Per-thread compensated FP32 sum (Kahan), handed to the CTA and cluster
// reductions as a float-float value.  FP64 arithmetic is scarce on GB300: one
// FP64 add per pixel and pass would cost more than the stencil itself.
struct KSum {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v) {
        const float y = v - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
};

// Float-float value hi + lo (about 44 significant bits): CTA-level sums of the
// per-thread compensated FP32 sums stay in FP32 arithmetic, and FP64 is used
// only for the grid-level sum of the CTA partials.
struct FF {
    float hi, lo;
};

__device__ __forceinline__ FF ff_add(FF a, FF b) {
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float e = (a.hi - (s - bb)) + (b.hi - bb) + (a.lo + b.lo);
    const float hi = s + e;
    return FF{hi, e - (hi - s)};
}

__device__ __forceinline__ FF ff_of(const KSum& k) { return FF{k.s, -k.c}; }

// An FP64 value as float-float (used for the FP64 per-element sums of the
// linear objective).
__device__ __forceinline__ FF ff_of(double v) {
    const float hi = (float)v;
    return FF{hi, (float)(v - (double)hi)};
}

// Deterministic cluster-wide sum of two values: float-float over the lanes
// and then the warps of each CTA (FP32 arithmetic), then one thread per CTA
// sums the cluster's CTA values in FP64 in rank order.  Every thread gets the
// same result, read from shared memory.  FP64 stays with one thread per CTA:
// it is scarce on GB300.
__device__ double2 cluster_sum2(FF a, FF b, FF* swf, double2* scta, double2* sres,
                                cg::cluster_group& cluster) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a = ff_add(a, FF{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)});
        b = ff_add(b, FF{__shfl_xor_sync(0xffffffffu, b.hi, o), __shfl_xor_sync(0xffffffffu, b.lo, o)});
    }
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        swf[2 * wid] = a;
        swf[2 * wid + 1] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        FF sa{0.f, 0.f}, sb{0.f, 0.f};
        for (int w = 0; w < kPerturbThreads / 32; ++w) {
            sa = ff_add(sa, swf[2 * w]);
            sb = ff_add(sb, swf[2 * w + 1]);
        }
        *scta = make_double2((double)sa.hi + (double)sa.lo, (double)sb.hi + (double)sb.lo);
    }
    cluster.sync();
    if (threadIdx.x == 0) {
        double2 t = make_double2(0.0, 0.0);
        const unsigned nr = cluster.num_blocks();
        for (unsigned r = 0; r < nr; ++r) {
            const double2 v = *cluster.map_shared_rank(scta, r);
            t.x += v.x;
            t.y += v.y;
        }
        *sres = t;
    }
    cluster.sync();   // every CTA has read scta; sres is visible to the CTA
    return *sres;
}

// Scalar decisions of a reduction step, taken by one thread after the
// subgradient pass and shared through shared memory: whether the step goes
// on, 1/||g|| and the adaptive step.
struct StepDecision {
    int go;
    float inv_gnorm, asc;
};

__device__ __forceinline__ StepDecision step_decision(const PerturbArgs& a, const RhsState& st,
                                                      double gg, double fy, double f_start) {
    StepDecision d{0, 0.f, 0.f};
    if (a.record_only || gg == 0.0) return d;
    d.inv_gnorm = 1.0f / sqrtf((float)gg);
    if (a.adaptive) {
        const double f_ref = adaptive_ref(a, st, f_start);
        if (!(fy > f_ref)) return d;
        d.asc = adaptive_scale(fy, f_ref, gg);
    }
    d.go = 1;
    return d;
}

// Where a perturbation phase starts: the restart rule (Sec. 2.1.2: l <- r at
// the r-th restart) applied to the exponent and the restart state.
struct PhaseStart {
    long long ell;
    int restarts, last_restart_k;
};

__device__ __forceinline__ PhaseStart phase_start(const PerturbArgs& a, int b) {
    const RhsState& st = a.st[b];
    PhaseStart ps;
    ps.ell = st.ell;
    ps.restarts = st.restarts;
    ps.last_restart_k = st.last_restart_k;
    const int k = st.k;
    if (!a.record_only && a.restart_every > 0 && k > 0 && k % a.restart_every == 0 &&
        ps.last_restart_k != k) {
        ps.restarts += 1;
        ps.ell = ps.restarts;
        ps.last_restart_k = k;
    }
    return ps;
}

// Bookkeeping at the end of a phase: f at its start, exponent, restart
// state, counts of this phase and in total.
__device__ __forceinline__ void phase_end(const PerturbArgs& a, RhsState& st, const PhaseStart& ps,
                                          long long ell, int accepted, int trials, double f_start) {
    st.f_cur = f_start;
    st.f_valid = 1;
    if (a.record_only) return;
    if (a.adaptive == 1) {
        st.f_ref = adaptive_ref(a, st, f_start);
        st.has_ref = 1;
    }
    st.ell = ell;
    st.restarts = ps.restarts;
    st.last_restart_k = ps.last_restart_k;
    st.accepted_last = accepted;
    st.trials_last = trials;
    st.accepted_total += accepted;
    st.trials_total += trials;
}

__global__ void __launch_bounds__(kPerturbThreads) k_perturb(const PerturbArgs a) {
    cg::cluster_group cluster = cg::this_cluster();
    __shared__ FF swf[2 * (kPerturbThreads / 32)];
    __shared__ double2 scta, sres;
    __shared__ StepDecision dec;
    __shared__ float sc_s;
    const int ncl = (int)cluster.num_blocks();
    const int b = blockIdx.x / ncl;             // right-hand side of this cluster
    RhsState& st = a.st[b];
    if (st.stopped) return;                     // uniform over the cluster
    const int rank = (int)cluster.block_rank();
    const int tid = rank * kPerturbThreads + threadIdx.x;
    const int nthr = ncl * kPerturbThreads;
    const int n = a.n, H = a.H, W = a.W, obj = a.obj;
    const bool lin = (obj == SUPPY_OBJ_LINEAR);
    Vec y{a.x + b, a.B};
    Vec g{a.g + b, a.B};

    const PhaseStart ps = phase_start(a, b);
    long long ell = ps.ell;
    int accepted = 0, trials = 0;
    double f_start = 0.0;   // thread 0 of each CTA
    bool have_f = false;
    for (int s = 0; s < (a.record_only ? 1 : a.n_red); ++s) {
        // pass G: subgradient, ||g||^2 and f(y) (the linear objective's terms
        // in FP64, the others compensated FP32)
        KSum kg, kf;
        double fl = 0.0;
        for (int p = tid; p < n; p += nthr) {
            const double t = obj_term(obj, p, H, W, a.c64, y);
            if (lin) fl += t;
            else kf.add((float)t);
            if (!a.record_only) {
                const float gp = subgrad(obj, p, H, W, a.c32, y);
                __stcg(g.p + (size_t)p * a.B, gp);
                kg.add(gp * gp);
            }
        }
        const double2 r = cluster_sum2(ff_of(kg), lin ? ff_of(fl) : ff_of(kf), swf, &scta, &sres,
                                       cluster);
        const double fy = r.y;
        if (threadIdx.x == 0) {
            if (!have_f) {
                f_start = fy;
                have_f = true;
            }
            dec = step_decision(a, st, r.x, fy, f_start);
        }
        __syncthreads();
        if (!dec.go) break;
        const float inv_gnorm = dec.inv_gnorm, asc = dec.asc;
        bool ok = false;
        const int jmax = a.adaptive ? 1 : a.max_trials;
        for (int j = 0; j < jmax; ++j) {
            if (threadIdx.x == 0)
                sc_s = a.adaptive ? asc : trial_scale(a.gamma, a.log2_alpha, ell, inv_gnorm);
            __syncthreads();
            const float sc = sc_s;
            if (!a.adaptive) ell += 1;
            trials += 1;
            Vec yy = y;
            Vec gv = g;
            auto z = [yy, gv, sc](int q) { return trial(yy(q), gv(q), sc); };
            KSum kz;
            double fzl = 0.0;
            for (int p = tid; p < n; p += nthr) {
                const double t = obj_term(obj, p, H, W, a.c64, z);
                if (lin) fzl += t;
                else kz.add((float)t);
            }
            const double fz =
                cluster_sum2(lin ? ff_of(fzl) : ff_of(kz), FF{0.f, 0.f}, swf, &scta, &sres, cluster).x;
            if (fz <= fy) {
                for (int p = tid; p < n; p += nthr) {
                    const size_t o = (size_t)p * a.B;
                    __stcg(y.p + o, trial(__ldcg(y.p + o), __ldcg(g.p + o), sc));
                }
                cluster.sync();
                accepted += 1;
                ok = true;
                break;
            }
        }
        if (!ok) break;
    }
    if (rank == 0 && threadIdx.x == 0) phase_end(a, st, ps, ell, accepted, trials, f_start);
}

// ------------------------------------------- shared-memory resident phase ----
// Same algorithm as k_perturb, with the right-hand side's iterate and
// subgradient held in the shared memory of the cluster for the whole phase:
// CTA r owns image rows [R_r, R_{r+1}) (TV) or elements [P_r, P_{r+1})
// (linear); the one halo row above and below a band is read from the
// neighbouring CTA's shared memory (distributed shared memory).  HBM / L2
// see one read and one write of x per phase.
struct Band {
    const float* own;
    const float* up;     // previous rank's band (DSMEM) or null
    const float* down;   // next rank's band (DSMEM) or null
    int r0, r1, up_r0, W;
    __device__ __forceinline__ float operator()(int i, int j) const {
        if (i >= r0 && i < r1) return own[(i - r0) * W + j];
        if (i < r0) return up[(i - up_r0) * W + j];
        return down[j];
    }
};

__device__ __forceinline__ int band_start(int r, int H, int cs) { return (int)((long long)H * r / cs); }

template <class Y>
__device__ __forceinline__ float tv_term(int obj, int i, int j, int H, int W, const Y& y) {
    const float y0 = y(i, j);
    if (obj == SUPPY_OBJ_TV_ISO) {
        if (i < H - 1 && j < W - 1) {
            const float dx = y(i + 1, j) - y0, dy = y(i, j + 1) - y0;
            return sqrtf(dx * dx + dy * dy);
        }
        return 0.f;
    }
    float t = 0.f;
    if (i < H - 1) t += fabsf(y(i + 1, j) - y0);
    if (j < W - 1) t += fabsf(y(i, j + 1) - y0);
    return t;
}

template <class Y>
__device__ __forceinline__ float tv_subgrad(int obj, int i, int j, int H, int W, const Y& y) {
    const float y0 = y(i, j);
    float g = 0.f;
    if (obj == SUPPY_OBJ_TV_ISO) {
        // each term contributes (its partial derivative) * 1/phi, phi = 0 -> 0
        if (i < H - 1 && j < W - 1) {
            const float dx = y(i + 1, j) - y0, dy = y(i, j + 1) - y0;
            const float q = dx * dx + dy * dy;
            if (q > 0.f) g -= (dx + dy) * rsqrtf(q);
        }
        if (i > 0 && j < W - 1) {
            const float ym = y(i - 1, j);
            const float dx = y0 - ym, dy = y(i - 1, j + 1) - ym;
            const float q = dx * dx + dy * dy;
            if (q > 0.f) g += dx * rsqrtf(q);
        }
        if (j > 0 && i < H - 1) {
            const float yl = y(i, j - 1);
            const float dx = y(i + 1, j - 1) - yl, dy = y0 - yl;
            const float q = dx * dx + dy * dy;
            if (q > 0.f) g += dy * rsqrtf(q);
        }
        return g;
    }
    if (i < H - 1) g -= sgnf(y(i + 1, j) - y0);
    if (i > 0) g += sgnf(y0 - y(i - 1, j));
    if (j < W - 1) g -= sgnf(y(i, j + 1) - y0);
    if (j > 0) g += sgnf(y0 - y(i, j - 1));
    return g;
}

// Row and column of element q of a strided loop over a row-major image (or
// band) of width W, advanced without a division per element: q grows by
// stride = si W + sj.
struct StrideWalk {
    int i, j, si, sj, W;
    __device__ StrideWalk(int q0, int stride, int w) : W(w) {
        i = q0 / w;
        j = q0 - i * w;
        si = stride / w;
        sj = stride - si * w;
    }
    __device__ __forceinline__ void next() {
        i += si;
        j += sj;
        if (j >= W) {
            j -= W;
            ++i;
        }
    }
};

__global__ void __launch_bounds__(kPerturbThreads) k_perturb_smem(const PerturbArgs a) {
    extern __shared__ float smem[];
    cg::cluster_group cluster = cg::this_cluster();
    __shared__ FF swf[2 * (kPerturbThreads / 32)];
    __shared__ double2 scta, sres;
    __shared__ StepDecision dec;
    __shared__ float sc_s;
    const int cs = (int)cluster.num_blocks();
    const int b = blockIdx.x / cs;
    RhsState& st = a.st[b];
    if (st.stopped) return;
    const PhaseStart ps = phase_start(a, b);
    const int rank = (int)cluster.block_rank();
    const bool lin = (a.obj == SUPPY_OBJ_LINEAR);
    const bool elem = elementwise(a.obj);
    const int H = elem ? a.n : a.H, W = elem ? 1 : a.W;   // element-wise: a column of n "rows"
    const int r0 = band_start(rank, H, cs), r1 = band_start(rank + 1, H, cs);
    int band = (r1 - r0) * W;
    const int maxband = ((H + cs - 1) / cs) * W;
    if (!PCHECKED(band >= 0 && band <= maxband && (elem || cs <= H), 401, rank)) band = 0;
    float* ys = smem;
    float* gs = smem + maxband;
    float* X = a.x + b;
    const int B = a.B;
    const int p0 = r0 * W;
    for (int q = threadIdx.x; q < band; q += kPerturbThreads) {
        ys[q] = X[(size_t)(p0 + q) * B];
        if (lin) gs[q] = a.c32[p0 + q];
    }
    cluster.sync();
    Band yb{ys, nullptr, nullptr, r0, r1, 0, W};
    Band gb{gs, nullptr, nullptr, r0, r1, 0, W};
    if (!elem) {
        if (rank > 0) {
            yb.up = cluster.map_shared_rank(ys, rank - 1);
            gb.up = cluster.map_shared_rank(gs, rank - 1);
            yb.up_r0 = gb.up_r0 = band_start(rank - 1, H, cs);
        }
        if (rank < cs - 1) {
            yb.down = cluster.map_shared_rank(ys, rank + 1);
            gb.down = cluster.map_shared_rank(gs, rank + 1);
        }
    }

    long long ell = ps.ell;
    int accepted = 0, trials = 0;
    double f_start = 0.0;   // thread 0 of each CTA
    bool have_f = false;
    for (int s = 0; s < (a.record_only ? 1 : a.n_red); ++s) {
        KSum kg, kf;
        double fl = 0.0;
        {
            StrideWalk px(threadIdx.x, kPerturbThreads, W);
            for (int q = threadIdx.x; q < band; q += kPerturbThreads, px.next()) {
                if (lin) {
                    const int p = p0 + q;
                    fl += a.c64[p] * (double)ys[q];
                    const float gp = gs[q];
                    kg.add(gp * gp);
                } else if (elem) {
                    kf.add(norm_term(a.obj, ys[q]));
                    if (!a.record_only) {
                        const float gp = norm_grad(a.obj, ys[q]);
                        gs[q] = gp;
                        kg.add(gp * gp);
                    }
                } else {
                    const int i = r0 + px.i, j = px.j;
                    kf.add(tv_term(a.obj, i, j, H, W, yb));
                    if (!a.record_only) {
                        const float gp = tv_subgrad(a.obj, i, j, H, W, yb);
                        gs[q] = gp;
                        kg.add(gp * gp);
                    }
                }
            }
        }
        const double2 r = cluster_sum2(ff_of(kg), lin ? ff_of(fl) : ff_of(kf), swf, &scta, &sres,
                                       cluster);
        const double fy = r.y;
        if (threadIdx.x == 0) {
            if (!have_f) {
                f_start = fy;
                have_f = true;
            }
            dec = step_decision(a, st, r.x, fy, f_start);
        }
        __syncthreads();
        if (!dec.go) break;
        const float inv_gnorm = dec.inv_gnorm, asc = dec.asc;
        bool ok = false;
        const int jmax = a.adaptive ? 1 : a.max_trials;
        for (int jt = 0; jt < jmax; ++jt) {
            if (threadIdx.x == 0)
                sc_s = a.adaptive ? asc : trial_scale(a.gamma, a.log2_alpha, ell, inv_gnorm);
            __syncthreads();
            const float sc = sc_s;
            if (!a.adaptive) ell += 1;
            trials += 1;
            FF fzp;
            if (lin) {
                double fzl = 0.0;
                for (int q = threadIdx.x; q < band; q += kPerturbThreads)
                    fzl += a.c64[p0 + q] * (double)trial(ys[q], gs[q], sc);
                fzp = ff_of(fzl);
            } else if (elem) {
                KSum kz;
                for (int q = threadIdx.x; q < band; q += kPerturbThreads)
                    kz.add(norm_term(a.obj, trial(ys[q], gs[q], sc)));
                fzp = ff_of(kz);
            } else {
                auto z = [&yb, &gb, sc](int i, int j) { return trial(yb(i, j), gb(i, j), sc); };
                KSum kz;
                StrideWalk px(threadIdx.x, kPerturbThreads, W);
                for (int q = threadIdx.x; q < band; q += kPerturbThreads, px.next())
                    kz.add(tv_term(a.obj, r0 + px.i, px.j, H, W, z));
                fzp = ff_of(kz);
            }
            const double fz = cluster_sum2(fzp, FF{0.f, 0.f}, swf, &scta, &sres, cluster).x;
            if (fz <= fy) {
                for (int q = threadIdx.x; q < band; q += kPerturbThreads)
                    ys[q] = trial(ys[q], gs[q], sc);
                cluster.sync();
                accepted += 1;
                ok = true;
                break;
            }
        }
        if (!ok) break;
    }
    if (!a.record_only) {
        for (int q = threadIdx.x; q < band; q += kPerturbThreads) X[(size_t)(p0 + q) * B] = ys[q];
    }
    if (rank == 0 && threadIdx.x == 0) phase_end(a, st, ps, ell, accepted, trials, f_start);
    // no CTA may leave while a neighbour can still read its shared memory
    cluster.sync();
}

// ------------------------------------------------ whole-GPU phase ----
// The perturbation phase of Algorithm 1 on the whole GPU, one right-hand side
// after the other, in a single cooperative launch (every CTA resident).  Each
// pass over the image -- the subgradient with ||g||^2 and f(y); f at up to
// kWideTrials consecutive trial points y - beta_j g/||g|| at once; the update
// y <- z_j -- takes a grid-stride share of the pixels per thread and ends in
// a grid barrier, inside which the last CTA to arrive sums the CTA partials
// in a fixed order; every CTA reads the same sums and takes the same
// decisions (the first j with f(z_j) <= f(y): exactly the trial the
// sequential loop accepts) without a further barrier.  y and g are read with plain coherent
// loads (other CTAs rewrite them between passes; the barrier's fences make
// those writes visible), never through the read-only path.  Element e of the
// n x B array is pixel e / B of right-hand side e % B.

// Last-CTA election: every CTA's partials are visible to the CTA that draws
// the last ticket; it resets the ticket for the next launch.
__device__ __forceinline__ bool last_cta(unsigned* ticket) {
    __shared__ bool is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = (atomicAdd(ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (is_last) __threadfence();
    return is_last;
}

// Fixed-order sum of part[c * stride + off] over the grid's CTAs by one warp.
__device__ __forceinline__ double warp_sum_parts(const double* part, int ncta, int stride,
                                                 int off) {
    const int lane = threadIdx.x & 31;
    double s = 0.0;
    for (int c = lane; c < ncta; c += 32) s += __ldcg(part + (size_t)c * stride + off);
    return warp_sum(s);
}

// Per-CTA sums of NV values per right-hand side, written as FP64 to
// part[(cta * B + b) * NV + v]: float-float sums over the lanes of each
// right-hand side, then over the warps in order.  sw holds 8 * NV * 32 values.
// Only the first nv values (uniform over the CTA) are reduced and written.
template <int NV, int NT = kWideThreads>
__device__ __forceinline__ void cta_partials(FF (&v)[NV], int B, FF* sw, double* part,
                                             int nv = NV) {
#pragma unroll
    for (int j = 0; j < NV; ++j)
        if (j < nv)
            for (int o = 16; o >= B && o > 0; o >>= 1) {
                const FF w{__shfl_xor_sync(0xffffffffu, v[j].hi, o),
                           __shfl_xor_sync(0xffffffffu, v[j].lo, o)};
                v[j] = ff_add(v[j], w);
            }
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane < B)
#pragma unroll
        for (int j = 0; j < NV; ++j)
            if (j < nv) sw[(wid * NV + j) * 32 + lane] = v[j];
    __syncthreads();
    for (int t = threadIdx.x; t < NV * B; t += NT) {
        const int b = t / NV, j = t - b * NV;
        if (j >= nv) continue;
        FF acc{0.f, 0.f};
        for (int w = 0; w < NT / 32; ++w) acc = ff_add(acc, sw[(w * NV + j) * 32 + b]);
        part[((size_t)blockIdx.x * B + b) * NV + j] = (double)acc.hi + (double)acc.lo;
    }
}

// The grid sums of the NV * B values, one warp per value, into res[b * NV + v]
// (shared memory).
template <int NV, int NT = kWideThreads>
__device__ __forceinline__ void grid_sums(const double* part, int B, double* res) {
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int t = wid; t < NV * B; t += NT / 32) {
        const double v = warp_sum_parts(part, gridDim.x, NV * B, t);
        if (lane == 0) res[t] = v;
    }
    __syncthreads();
}

// Grid barrier of a cooperative launch: bar[0] counts arrivals, bar[1] is the
// generation.  A CTA reads the generation before it arrives; the last to
// arrive first sums the NV CTA partials of the pass (one warp per value, a
// fixed order: the same FP64 sums whichever CTA arrives last) into gsum, then
// resets the count and advances the generation; the others wait, then read
// gsum into res (shared memory).  One CTA does the FP64 reduction: FP64 is
// scarce on GB300, and every CTA summing the partials itself took longer than
// the wait.  The wait is bounded: on timeout
// the CTA records error word 2 and every CTA leaves at its next barrier.  The
// budget is a launch argument (about two seconds of SM clock by default).
// The partials need no second buffer: they are read before the release, and
// written again only after it.
constexpr int kFirstTrials = 2;

template <int NV>
__device__ __forceinline__ bool grid_barrier(unsigned* bar, int* err, const double* part,
                                             double* gsum, double* res, long long limit) {
    __shared__ int st_s;   // bit 0: ok, bit 1: this CTA arrived last
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* gen = bar + 1;
        const unsigned g0 = *gen;
        __threadfence();
        int ok = 1, last = 0;
        if (atomicAdd(bar, 1u) == gridDim.x - 1) {
            last = 1;
            __threadfence();
        } else {
            const long long t0 = clock64();
            while (*gen == g0) {
                if (*(volatile int*)err || clock64() - t0 > limit) {
                    atomicExch(err, 2);
                    ok = 0;
                    break;
                }
                __nanosleep(32);
            }
            __threadfence();
        }
        st_s = ok | (last << 1);
    }
    __syncthreads();
    const int st = st_s;
    if (st & 2) {
        if constexpr (NV > 0) {
            grid_sums<NV, kPhaseThreads>(part, 1, res);
            if (threadIdx.x < NV) gsum[threadIdx.x] = res[threadIdx.x];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            __threadfence();
            atomicExch(bar, 0u);
            __threadfence();
            atomicAdd(bar + 1, 1u);
        }
    } else {
        if constexpr (NV > 0)
            if (threadIdx.x < NV) res[threadIdx.x] = __ldcg(gsum + threadIdx.x);
    }
    __syncthreads();
    return (st & 1) && *(volatile int*)err == 0;
}

// Image of one right-hand side read with plain (coherent, L1-cached) loads:
// other CTAs rewrite it between passes, and the grid barrier's fences make
// their writes visible to these loads, which the read-only path (ld.global.nc)
// would not guarantee.
struct CohImage {
    const float* y;   // element 0 of the right-hand side
    int B, W;
    __device__ __forceinline__ float operator()(int i, int j) const {
        return y[((size_t)i * W + j) * B];
    }
};

// The values a TV term of pixel (i, j) reads at every trial point z = y - s g:
// y and g at (i, j), (i + 1, j) and (i, j + 1), loaded once per pixel.
struct TvNbr {
    float y0, g0, yd, gd, yr, gr;
    bool down, right;
};

__device__ __forceinline__ TvNbr tv_nbr(int i, int j, int H, int W, const float* y, const float* g,
                                        int B) {
    const size_t p = (size_t)i * W + j;
    TvNbr t;
    t.down = i < H - 1;
    t.right = j < W - 1;
    t.y0 = y[p * B];
    t.g0 = g[p * B];
    t.yd = t.down ? y[(p + W) * B] : 0.f;
    t.gd = t.down ? g[(p + W) * B] : 0.f;
    t.yr = t.right ? y[(p + 1) * B] : 0.f;
    t.gr = t.right ? g[(p + 1) * B] : 0.f;
    return t;
}

// TV term at the trial point with step s (computed as in the cluster kernels).
__device__ __forceinline__ float tv_trial_term(int obj, const TvNbr& t, float s) {
    const float z0 = trial(t.y0, t.g0, s);
    if (obj == SUPPY_OBJ_TV_ISO) {
        if (t.down && t.right) {
            const float dx = trial(t.yd, t.gd, s) - z0;
            const float dy = trial(t.yr, t.gr, s) - z0;
            return sqrtf(dx * dx + dy * dy);
        }
        return 0.f;
    }
    float v = 0.f;
    if (t.down) v += fabsf(trial(t.yd, t.gd, s) - z0);
    if (t.right) v += fabsf(trial(t.yr, t.gr, s) - z0);
    return v;
}

__global__ void __launch_bounds__(kPhaseThreads, 1) k_wide_phase(const PerturbArgs a) {
    __shared__ FF sw[(kPhaseThreads / 32) * kWideTrials * 32];
    __shared__ double res[kWideTrials];
    __shared__ float sj_s[kWideTrials];
    __shared__ int dec_s[2];     // continue the step; the accepted trial (-1: none)
    __shared__ float dec_f[2];   // 1/||g||; the adaptive step
    const int B = a.B, n = a.n, H = a.H, W = a.W, obj = a.obj;
    const int tid = blockIdx.x * kPhaseThreads + threadIdx.x;
    const int stride = gridDim.x * kPhaseThreads;
    const bool lin = (obj == SUPPY_OBJ_LINEAR);
    const bool tv = !elementwise(obj);
    double* const part = a.part;
    double* const gsum = a.part + (size_t)gridDim.x * kWideTrials;
    for (int b = 0; b < B; ++b) {
        RhsState& st = a.st[b];
        if (st.stopped) continue;   // read by every CTA before the phase's first barrier
        const PhaseStart ps = phase_start(a, b);
        const bool has_ref = st.has_ref;
        const double st_ref = st.f_ref;
        long long ell = ps.ell;
        int accepted = 0, trials = 0;
        double f_start = 0.0;
        float* X = a.x + b;
        float* G = a.g + b;
        bool copied = false;   // the patch copies were written with the last update
        for (int s = 0; s < a.n_red; ++s) {
            // pass G: subgradient, ||g||^2 and f(y)
            KSum kg, kf;
            double fl = 0.0;
            StrideWalk px(tid, stride, tv ? W : 1);
            for (int p = tid; p < n; p += stride, px.next()) {
                float gp;
                if (lin) {
                    gp = a.c32[p];
                    fl += a.c64[p] * (double)X[(size_t)p * B];
                } else if (!tv) {
                    const float y0 = X[(size_t)p * B];
                    kf.add(norm_term(obj, y0));
                    gp = norm_grad(obj, y0);
                } else {
                    const CohImage yi{X, B, W};
                    kf.add(tv_term(obj, px.i, px.j, H, W, yi));
                    gp = tv_subgrad(obj, px.i, px.j, H, W, yi);
                }
                G[(size_t)p * B] = gp;
                kg.add(gp * gp);
            }
            {
                FF v[2] = {ff_of(kg), lin ? ff_of(fl) : ff_of(kf)};
                cta_partials<2, kPhaseThreads>(v, 1, sw, part);
            }
            if (!grid_barrier<2>(a.ticket, a.err, part, gsum, res, a.wait_cycles)) return;
            // the step's scalar decisions by one thread (FP64 is scarce on
            // GB300: not by every thread of the grid), shared through smem
            const double fy = res[1];
            if (threadIdx.x == 0) {
                const double gg = res[0];
                if (s == 0) f_start = fy;
                int go = gg != 0.0;
                float inv_gnorm = 0.f, asc = 0.f;
                if (go) {
                    inv_gnorm = 1.0f / sqrtf((float)gg);
                    if (a.adaptive) {
                        const double f_ref =
                            a.adaptive == 2 ? a.f_ref : (has_ref ? fmin(st_ref, f_start) : f_start);
                        if (!(fy > f_ref)) go = 0;
                        else asc = adaptive_scale(fy, f_ref, gg);
                    }
                }
                dec_s[0] = go;
                dec_f[0] = inv_gnorm;
                dec_f[1] = asc;
            }
            __syncthreads();
            if (!dec_s[0]) break;
            const float inv_gnorm = dec_f[0], asc = dec_f[1];
            const int jmax = a.adaptive ? 1 : a.max_trials;
            bool ok = false;
            for (int jt = 0; jt < jmax && !ok;) {
                // the first pass of a step tries kFirstTrials points (usually
                // the first is accepted once the exponent has settled), later
                // passes kWideTrials; the accepted trial is the same either way
                const int cnt = min(jt == 0 ? kFirstTrials : kWideTrials, jmax - jt);
                // the trial step sizes, one thread each
                if (threadIdx.x < kWideTrials)
                    sj_s[threadIdx.x] = a.adaptive
                                            ? asc
                                            : trial_scale(a.gamma, a.log2_alpha, ell + threadIdx.x,
                                                          inv_gnorm);
                __syncthreads();
                float sj[kWideTrials];
#pragma unroll
                for (int q = 0; q < kWideTrials; ++q) sj[q] = sj_s[q];
                // pass T: f at the cnt trial points (the slots past cnt are not read)
                KSum kz[kWideTrials];
                double fz[kWideTrials];
#pragma unroll
                for (int q = 0; q < kWideTrials; ++q) fz[q] = 0.0;
                StrideWalk px(tid, stride, tv ? W : 1);
                for (int p = tid; p < n; p += stride, px.next()) {
                    if (lin) {
                        const float y0 = X[(size_t)p * B], g0 = G[(size_t)p * B];
                        const double c = a.c64[p];
#pragma unroll
                        for (int q = 0; q < kWideTrials; ++q)
                            if (q < cnt) fz[q] += c * (double)trial(y0, g0, sj[q]);
                    } else if (!tv) {
                        const float y0 = X[(size_t)p * B], g0 = G[(size_t)p * B];
#pragma unroll
                        for (int q = 0; q < kWideTrials; ++q)
                            if (q < cnt) kz[q].add(norm_term(obj, trial(y0, g0, sj[q])));
                    } else {
                        const TvNbr t = tv_nbr(px.i, px.j, H, W, X, G, B);
#pragma unroll
                        for (int q = 0; q < kWideTrials; ++q)
                            if (q < cnt) kz[q].add(tv_trial_term(obj, t, sj[q]));
                    }
                }
                {
                    FF v[kWideTrials];
#pragma unroll
                    for (int q = 0; q < kWideTrials; ++q) v[q] = lin ? ff_of(fz[q]) : ff_of(kz[q]);
                    cta_partials<kWideTrials, kPhaseThreads>(v, 1, sw, part, cnt);
                }
                if (!grid_barrier<kWideTrials>(a.ticket, a.err, part, gsum, res, a.wait_cycles)) return;
                if (threadIdx.x == 0) {
                    int h = -1;
                    for (int q = 0; q < cnt; ++q)
                        if (res[q] <= fy) {
                            h = q;
                            break;
                        }
                    dec_s[1] = h;
                }
                __syncthreads();
                const int hit = dec_s[1];
                const int used = hit >= 0 ? hit + 1 : cnt;
                if (!a.adaptive) ell += used;
                trials += used;
                jt += used;
                if (hit >= 0) {
                    // pass U: y <- z_hit (and its patch copies, pixel by pixel)
                    const float sc = sj_s[hit];
                    if (a.pA) {
                        StrideWalk pw(tid, stride, W);
                        for (int p = tid; p < n; p += stride, pw.next()) {
                            const float v = trial(X[p], G[p], sc);
                            X[p] = v;
                            a.pA[patch_pos(pw.i, pw.j, a.pWp, false)] = v;
                            a.pB[patch_pos(pw.i, pw.j, a.pWp, true)] = v;
                        }
                        copied = true;
                    } else {
                        for (int p = tid; p < n; p += stride) {
                            const size_t o = (size_t)p * B;
                            X[o] = trial(X[o], G[o], sc);
                        }
                    }
                    accepted += 1;
                    ok = true;
                }
            }
            if (!ok) break;
            // the next reduction step reads the neighbours' new y
            if (s + 1 < a.n_red && !grid_barrier<0>(a.ticket, a.err, part, gsum, res, a.wait_cycles)) return;
        }
        if (a.pA && !copied) {
            // no step was taken: the copies of y as it stands (each thread its
            // own pixels, which no other thread writes in this launch)
            StrideWalk pw(tid, stride, W);
            for (int p = tid; p < n; p += stride, pw.next()) {
                const float v = X[p];
                a.pA[patch_pos(pw.i, pw.j, a.pWp, false)] = v;
                a.pB[patch_pos(pw.i, pw.j, a.pWp, true)] = v;
            }
        }
        if (blockIdx.x == 0 && threadIdx.x == 0) phase_end(a, st, ps, ell, accepted, trials, f_start);
    }
}

// ------------------------------------------------ variance stopping rule ----
// After an iteration: ||x - xprev||^2 and ||x||^2 per right-hand side
// (compensated FP32 per thread, float-float per CTA, FP64 over the grid),
// xprev <- x; the last CTA adds omega = ||x - xprev|| / ||x|| to the running
// sums of the state and stops a right-hand side once the sample variance of
// its omegas (k >= 2 of them) is below tol.
__global__ void __launch_bounds__(kWideThreads) k_variance(float* x, float* xprev, long long n,
                                                           int B, RhsState* st, double* part,
                                                           unsigned* ticket, double tol) {
    __shared__ FF sw[(kWideThreads / 32) * 2 * 32];
    __shared__ double res[2 * kMaxRhs];
    const long long nB = n * B;
    const long long tid = (long long)blockIdx.x * kWideThreads + threadIdx.x;
    const long long stride = (long long)gridDim.x * kWideThreads;
    const int b = (int)(tid & (B - 1));
    KSum kd, kx;
    if (!st[b].stopped)
        for (long long e = tid; e < nB; e += stride) {
            const float v = x[e], d = v - xprev[e];
            kd.add(d * d);
            kx.add(v * v);
            xprev[e] = v;
        }
    FF v[2] = {ff_of(kd), ff_of(kx)};
    cta_partials<2>(v, B, sw, part);
    if (!last_cta(ticket)) return;
    grid_sums<2>(part, B, res);
    if (threadIdx.x < B) {
        RhsState& s = st[threadIdx.x];
        if (!s.stopped) {
            const double D = res[2 * threadIdx.x], X = res[2 * threadIdx.x + 1];
            const double w = X > 0.0 ? sqrt(D / X) : 0.0;
            s.w_n += 1;
            s.w_s1 += w;
            s.w_s2 += w * w;
            if (s.w_n >= 2) {
                const double nn = (double)s.w_n;
                const double var = (s.w_s2 - s.w_s1 * s.w_s1 / nn) / (nn - 1.0);
                if (var < tol) s.stopped = 1;
            }
        }
    }
    if (threadIdx.x == 0) *ticket = 0u;
}

// Objective partials: CTA c writes f-partials of every right-hand side.
__global__ void __launch_bounds__(256) k_objective(const ObjArgs a) {
    __shared__ double sw[8];
    for (int b = 0; b < a.B; ++b) {
        Vec y{const_cast<float*>(a.x) + b, a.B};
        double f = 0.0;
        for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < a.n; p += gridDim.x * blockDim.x)
            f += obj_term(a.obj, p, a.H, a.W, a.c64, y);
        f = warp_sum(f);
        if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = f;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int w = 0; w < 8; ++w) s += sw[w];
            a.partial[(size_t)blockIdx.x * a.B + b] = s;
        }
        __syncthreads();
    }
}

}  // namespace

size_t perturb_smem_bytes(int obj, int n, int H, int W, int cs);

int choose_perturb_cluster(int n, int B) {
    // enough CTAs that each thread owns a handful of pixels; at most 16 (one GPC)
    int want = (n + kPerturbThreads * 8 - 1) / (kPerturbThreads * 8);
    int cs = 1;
    while (cs < want && cs < 16) cs <<= 1;
    (void)B;
    return cs;
}

int fit_perturb_cluster(int want, int obj, int n, int H, int W) {
    // largest power of two <= want for which a cluster can be resident
    for (int cs = want; cs >= 1; cs >>= 1) {
        const size_t smem = perturb_smem_bytes(obj, n, H, W, cs);
        auto kern = smem ? k_perturb_smem : k_perturb;
        cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (smem) cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(cs, 1, 1);
        cfg.blockDim = dim3(kPerturbThreads, 1, 1);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = cs;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int nc = 0;
        if (cudaOccupancyMaxActiveClusters(&nc, kern, &cfg) == cudaSuccess && nc > 0) return cs;
        cudaGetLastError();
    }
    return 1;
}

size_t perturb_smem_bytes(int obj, int n, int H, int W, int cs) {
    const bool elem = (obj == SUPPY_OBJ_LINEAR || obj == SUPPY_OBJ_L1 || obj == SUPPY_OBJ_L2);
    const long long rows = elem ? n : H, w = elem ? 1 : W;
    if (!elem && cs > H) return 0;
    const long long maxband = ((rows + cs - 1) / cs) * w;
    const size_t bytes = (size_t)(2 * maxband) * sizeof(float);
    return bytes <= 200 * 1024 ? bytes : 0;
}

cudaError_t launch_perturb(const PerturbArgs& a, int cluster, cudaStream_t s) {
    const size_t smem = perturb_smem_bytes(a.obj, a.n, a.H, a.W, cluster);
    auto kern = smem ? k_perturb_smem : k_perturb;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    if (smem) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(a.B * cluster, 1, 1);
    cfg.blockDim = dim3(kPerturbThreads, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, a);
}

// kWideTrials partials per CTA, then the kWideTrials grid sums
size_t wide_part_doubles(int grid) { return ((size_t)grid + 1) * kWideTrials; }

int wide_phase_blocks_per_sm() {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_wide_phase, kPhaseThreads, 0) !=
        cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nb;
}

cudaError_t launch_variance(float* x, float* xprev, long long n, int B, RhsState* st,
                            double* part, unsigned* ticket, double tol, int grid, cudaStream_t s) {
    k_variance<<<grid, kWideThreads, 0, s>>>(x, xprev, n, B, st, part, ticket, tol);
    return cudaGetLastError();
}

cudaError_t launch_perturb_wide(const PerturbArgs& a, int grid, cudaStream_t s) {
    if (!a.ticket || !a.err || !a.part || grid < 1) return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid, 1, 1);
    cfg.blockDim = dim3(kPhaseThreads, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_wide_phase, a);
}

cudaError_t launch_objective(const ObjArgs& a, int grid, double* out, cudaStream_t s) {
    k_objective<<<grid, 256, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_reduce_pp(a.partial, grid, a.B, 1.0, 0, out, s);
}

}  // namespace suppy
