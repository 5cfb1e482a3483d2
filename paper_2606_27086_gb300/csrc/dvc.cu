// Split feasibility with dose-volume constraints: the CQ step of Sec. 2.1.1
// (the iteration printed after Eq. (Split)) over the dose-volume sets of
// Sec. 2.3.3,
//
//     x <- x + gamma sum_j w_j A_j^T (P_Qj(A_j x) - A_j x),
//
// in four launches: the doses d = A_q x (warp per row), the projections onto
// the DVC sets (one CTA per structure: radix selection of the K-th highest
// dose, equal doses ranked by row), the fixed-order sum of the target-space
// proximity, and the correction gathered per column through the CSC copy of
// A_q (warp per column, deterministic).
//
// Sets (reading of the paper's wording): an upper DVC (D_V <= d_ref) lets at
// most K = floor(V N) of the structure's N voxels exceed d_ref, a lower DVC
// (D_V >= d_ref) demands at least K = ceil(V N) voxels at or above d_ref.  The
// Euclidean projection keeps (upper) or raises to d_ref (lower) the K highest
// doses and lowers (upper) every other dose above d_ref to d_ref.
#include "common.cuh"

namespace suppy {

namespace {

constexpr int kDoseThreads = 256;
constexpr int kProjectThreads = 1024;
constexpr int kApplyThreads = 256;

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Order-preserving key of a float dose: larger dose, larger key; -0 and +0
// map to the same key (they are equal doses).
__device__ __forceinline__ uint32_t dose_key(float f) {
    if (f == 0.0f) f = 0.0f;
    const uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// d_i = <a_i, x>: one warp per row, lanes strided over the row, warp tree.
__global__ void __launch_bounds__(kDoseThreads) k_dvc_dose(DvcArgs a) {
    if (a.st && a.st[0].stopped) return;
    const int warp = (blockIdx.x * kDoseThreads + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * kDoseThreads) >> 5;
    for (int i = warp; i < a.mq; i += nw) {
        const int e0 = a.rp[i], e1 = a.rp[i + 1];
        float s = 0.f;
        for (int e = e0 + lane; e < e1; e += 32) s = fmaf(__ldg(a.val + e), __ldg(a.x + a.col[e]), s);
        s = warp_sum_f(s);
        if (lane == 0) a.dose[i] = s;
    }
}

// CTA-wide sum of one int per thread (all threads get the result).
__device__ __forceinline__ int cta_count(int v, int* red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    __syncthreads();
    if (lane == 0) red[wid] = v;
    __syncthreads();
    int t = 0;
    for (int w = 0; w < kProjectThreads / 32; ++w) t += red[w];
    return t;
}

// One CTA per structure: for each DVC of the structure in the given order,
// decide the set's projection of the structure's doses and add
// w_j (P_Qj(d) - d) to the corrections; write 1/2 w_j ||P_Qj(d) - d||^2.
__global__ void __launch_bounds__(kProjectThreads) k_dvc_project(DvcArgs a) {
    if (a.st && a.st[0].stopped) return;
    const int s = blockIdx.x;
    const int r0 = a.sptr[s], r1 = a.sptr[s + 1];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    __shared__ int hist[256];
    __shared__ int red[kProjectThreads / 32];
    __shared__ uint32_t sh_prefix;
    __shared__ int sh_rank;
    __shared__ double dred[kProjectThreads / 32];

    for (int i = r0 + tid; i < r1; i += kProjectThreads) a.corr[i] = 0.f;

    for (int q = a.sdvc[s]; q < a.sdvc[s + 1]; ++q) {
        const DvcDesc dv = a.dvc[q];
        const bool upper = (dv.kind == 0);
        const int K = dv.K;
        // voxels already beyond d_ref (decided in FP64)
        int cnt = 0;
        for (int i = r0 + tid; i < r1; i += kProjectThreads) {
            const double d = (double)a.dose[i];
            cnt += upper ? (d > dv.d_ref) : (d >= dv.d_ref);
        }
        cnt = cta_count(cnt, red);
        const bool feasible = upper ? (cnt <= K) : (cnt >= K);
        if (feasible) {
            if (tid == 0) a.pd[dv.orig] = 0.0;
            __syncthreads();
            continue;
        }
        // K-th highest key by radix selection (8 bits a round, from the top);
        // afterwards `rank` is how many of the keys equal to the threshold
        // are kept (the lowest rows first).
        uint32_t thr = 0xffffffffu;
        int rank = 0;
        bool none_kept = (K == 0);
        if (!none_kept) {
            uint32_t prefix = 0, mask = 0;
            int kk = K;
            for (int shift = 24; shift >= 0; shift -= 8) {
                for (int b = tid; b < 256; b += kProjectThreads) hist[b] = 0;
                __syncthreads();
                for (int base = r0; base < r1; base += kProjectThreads) {
                    const int i = base + tid;
                    bool on = false;
                    uint32_t bin = 0;
                    if (i < r1) {
                        const uint32_t key = dose_key(a.dose[i]);
                        on = (key & mask) == prefix;
                        bin = (key >> shift) & 255u;
                    }
                    // warp-aggregated increments (many equal doses share a bin)
                    const unsigned act = __ballot_sync(0xffffffffu, on);
                    if (on) {
                        const unsigned peers = __match_any_sync(act, bin);
                        if ((int)(__ffs(peers) - 1) == lane) atomicAdd(&hist[bin], __popc(peers));
                    }
                }
                __syncthreads();
                if (tid == 0) {
                    int above = 0, b = 255;
                    for (; b > 0; --b) {
                        if (above + hist[b] >= kk) break;
                        above += hist[b];
                    }
                    sh_prefix = prefix | ((uint32_t)b << shift);
                    sh_rank = kk - above;
                }
                __syncthreads();
                prefix = sh_prefix;
                kk = sh_rank;
                mask |= 255u << shift;
                __syncthreads();
            }
            thr = prefix;
            rank = kk;
        }
        // apply in row order; a running count ranks the keys equal to thr
        double acc = 0.0;
        int eq_base = 0;
        for (int base = r0; base < r1; base += kProjectThreads) {
            const int i = base + tid;
            const bool in = i < r1;
            const float df = in ? a.dose[i] : 0.f;
            const uint32_t key = in ? dose_key(df) : 0u;
            const bool eq = in && !none_kept && key == thr;
            const unsigned bal = __ballot_sync(0xffffffffu, eq);
            if (lane == 0) red[wid] = __popc(bal);
            __syncthreads();
            int before = eq_base;
            for (int w = 0; w < wid; ++w) before += red[w];
            before += __popc(bal & ((1u << lane) - 1u));
            int tile_total = 0;
            for (int w = 0; w < kProjectThreads / 32; ++w) tile_total += red[w];
            __syncthreads();
            eq_base += tile_total;
            if (in) {
                const bool kept = !none_kept && (key > thr || (eq && before < rank));
                const double d = (double)df;
                double e = 0.0;
                if (upper) {
                    if (!kept && d > dv.d_ref) e = dv.d_ref - d;
                } else {
                    if (kept && d < dv.d_ref) e = dv.d_ref - d;
                }
                if (e != 0.0) {
                    a.corr[i] += (float)(dv.w * e);
                    acc += e * e;
                }
            }
        }
        // fixed-order CTA sum of the squared corrections
        acc = warp_sum(acc);
        if (lane == 0) dred[wid] = acc;
        __syncthreads();
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < kProjectThreads / 32; ++w) t += dred[w];
            a.pd[dv.orig] = 0.5 * dv.w * t;
        }
        __syncthreads();
    }
}

// Target-space proximity: the per-DVC terms summed in the caller's order.
__global__ void k_dvc_total(const double* pd, int ndvc, double* out, const RhsState* st) {
    if (st && st[0].stopped) return;
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int j = 0; j < ndvc; ++j) t += pd[j];
        out[0] = t;
    }
}

// x_j += gamma sum_i a_ij corr_i: one warp per column over the CSC copy.
__global__ void __launch_bounds__(kApplyThreads) k_dvc_apply(DvcArgs a) {
    if (a.st && a.st[0].stopped) return;
    const int warp = (blockIdx.x * kApplyThreads + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * kApplyThreads) >> 5;
    for (int j = warp; j < a.n; j += nw) {
        const int e0 = a.cp[j], e1 = a.cp[j + 1];
        float s = 0.f;
        for (int e = e0 + lane; e < e1; e += 32) s = fmaf(__ldg(a.cval + e), __ldg(a.corr + a.crow[e]), s);
        s = warp_sum_f(s);
        if (lane == 0 && e1 > e0) a.xw[j] = a.xw[j] + a.gamma * s;
    }
}

// ||A_s||_F^2 per structure (FP64, fixed order): one CTA per structure.
__global__ void __launch_bounds__(kDoseThreads) k_dvc_frob(const int* rp, const float* val,
                                                           const int* sptr, double* out) {
    const int s = blockIdx.x;
    const long long e0 = rp[sptr[s]], e1 = rp[sptr[s + 1]];
    double acc = 0.0;
    for (long long e = e0 + threadIdx.x; e < e1; e += kDoseThreads) {
        const double v = (double)val[e];
        acc += v * v;
    }
    acc = warp_sum(acc);
    __shared__ double sw[kDoseThreads / 32];
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kDoseThreads / 32; ++w) t += sw[w];
        out[s] = t;
    }
}

int grid_for(long long warps_needed, int threads) {
    long long g = (warps_needed * 32 + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > 152 * 16) g = 152 * 16;
    return (int)g;
}

}  // namespace

cudaError_t launch_dvc_dose(const DvcArgs& a, cudaStream_t s) {
    if (a.mq > 0) k_dvc_dose<<<grid_for(a.mq, kDoseThreads), kDoseThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_dvc_project(const DvcArgs& a, cudaStream_t s) {
    if (a.nstruct > 0) k_dvc_project<<<a.nstruct, kProjectThreads, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_dvc_total<<<1, 32, 0, s>>>(a.pd, a.ndvc, a.target, a.st);
    return cudaGetLastError();
}

cudaError_t launch_dvc_apply(const DvcArgs& a, cudaStream_t s) {
    if (a.n > 0) k_dvc_apply<<<grid_for(a.n, kApplyThreads), kApplyThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_dvc_frob(const int* rp, const float* val, const int* sptr, int nstruct,
                            double* out, cudaStream_t s) {
    if (nstruct > 0) k_dvc_frob<<<nstruct, kDoseThreads, 0, s>>>(rp, val, sptr, out);
    return cudaGetLastError();
}

}  // namespace suppy
