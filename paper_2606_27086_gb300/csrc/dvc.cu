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
#include <cooperative_groups.h>

#include <algorithm>

#include "common.cuh"

namespace suppy {

namespace cg = cooperative_groups;

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

// d_i = <a_i, x>: one warp per row, lanes strided over the row; each lane
// issues the loads of up to eight entries at once (one DRAM round trip per
// 256 entries of the row), then gathers x (L1-resident); fixed combination
// order, warp tree.
__global__ void __launch_bounds__(kDoseThreads) k_dvc_dose(DvcArgs a) {
    if (a.st && a.st[0].stopped) return;
    const int warp = (blockIdx.x * kDoseThreads + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int nw = (gridDim.x * kDoseThreads) >> 5;
    for (int i = warp; i < a.mq; i += nw) {
        const int e0 = a.rp[i], e1 = a.rp[i + 1];
        float s = 0.f;
        for (int b = e0; b < e1; b += 256) {
            int c[8];
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int e = b + u * 32 + lane;
                const bool ok = e < e1;
                c[u] = ok ? a.col[e] : 0;
                v[u] = ok ? __ldg(a.val + e) : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) s = fmaf(v[u], __ldg(a.x + (size_t)c[u] * a.B), s);
        }
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

// Float-float value hi + lo: the squared corrections are summed in FP32
// arithmetic with error-free transformations (FP64 throughput is far below
// FP32 on this part; FP64 appears only in the per-DVC total).
struct Ff {
    float hi, lo;
};

__device__ __forceinline__ Ff ff_add(Ff a, Ff b) {
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float e = (a.hi - (s - bb)) + (b.hi - bb) + (a.lo + b.lo);
    const float hi = s + e;
    return Ff{hi, e - (hi - s)};
}

// d_ref - d as float-float (d_ref = ref_hi + ref_lo)
__device__ __forceinline__ Ff ff_diff(float ref_hi, float ref_lo, float d) {
    const float s = ref_hi - d;
    const float bb = s - ref_hi;
    const float t = (ref_hi - (s - bb)) + (-d - bb);
    const float lo = t + ref_lo;
    const float hi = s + lo;
    return Ff{hi, lo - (hi - s)};
}

__device__ __forceinline__ Ff ff_sq(Ff e) {
    const float p = e.hi * e.hi;
    float q = fmaf(e.hi, e.hi, -p);
    q = fmaf(2.f * e.hi, e.lo, q);
    const float hi = p + q;
    return Ff{hi, q - (hi - p)};
}

__device__ __forceinline__ Ff warp_ff(Ff v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const Ff w{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
        v = ff_add(v, w);
    }
    return v;
}

__device__ __forceinline__ float key_dose(uint32_t k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// Radix selection digits: four bytes of the 32-bit key, from the top (wider
// digits make the cluster-wide histogram exchange cost more than the rounds
// they save).
constexpr int kBins = 256;
constexpr int kRounds = 4;
__device__ __forceinline__ int digit_shift(int r) { return 24 - 8 * r; }
__device__ __forceinline__ uint32_t digit_mask(int) { return 0xffu; }

// One thread-block cluster per structure (kDvcCluster CTAs, each a
// contiguous chunk of the structure's rows): for each DVC of the structure in
// the given order, decide the set's projection of the structure's doses, add
// w_j (P_Qj(d) - d) to the corrections and write this CTA's part of
// ||P_Qj(d) - d||^2.  Per DVC: the first pass counts the doses beyond d_ref
// and builds the histogram of the top digit; up to three more passes refine the
// K-th highest key; the apply pass moves the doses.  Histograms are combined
// over the cluster through distributed shared memory after a cluster barrier
// (fixed rank order); they are double-buffered by round, so a CTA never
// clears a histogram that a slower CTA may still be reading.  SMEM: the
// chunk's keys are staged in shared memory once; otherwise every pass
// re-reads the doses.
template <bool SMEM>
__global__ void __launch_bounds__(kProjectThreads) k_dvc_project(DvcArgs a) {
    if (a.st && a.st[0].stopped) return;          // uniform over the grid
    cg::cluster_group cl = cg::this_cluster();
    constexpr int CL = kDvcCluster;               // the launch's cluster size
    const int crank = (int)cl.block_rank();
    extern __shared__ uint32_t skey[];
    const int s = blockIdx.x / CL;
    const int r0 = a.sptr[s], N = a.sptr[s + 1] - r0;
    const int chunk = (N + CL - 1) / CL;
    const int c0 = min(N, crank * chunk), nloc = min(N, c0 + chunk) - c0;
    const int base_row = r0 + c0;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    __shared__ int hist[2][kBins];     // this CTA's histogram (double-buffered by round)
    __shared__ int ghist[kBins];       // the cluster's histogram
    __shared__ int red[kProjectThreads / 32];
    __shared__ Ff fred[kProjectThreads / 32];
    __shared__ uint32_t sh_prefix;
    __shared__ int sh_rank, sh_bin, sh_geq, sh_eqbase;
    __shared__ int slot_cnt[2];        // this CTA's count, double-buffered by DVC
    auto key_at = [&](int j) -> uint32_t {   // j in [0, nloc)
        if constexpr (SMEM) return skey[j];
        else return dose_key(a.dose[base_row + j]);
    };

    for (int j = tid; j < nloc; j += kProjectThreads) {
        a.corr[base_row + j] = 0.f;
        if constexpr (SMEM) skey[j] = dose_key(a.dose[base_row + j]);
    }
    int buf = 0;
    for (int q = a.sdvc[s], par = 0; q < a.sdvc[s + 1]; ++q, par ^= 1) {
        const DvcDesc dv = a.dvc[q];
        const bool upper = (dv.kind == 0);
        const int K = dv.K;
        const bool none_kept = (K == 0);
        uint32_t prefix = 0, mask = 0;
        int kk = K, eq_base = 0;
        bool feasible = false, need_order = false;
        for (int r = 0; r < kRounds; ++r, buf ^= 1) {
            const int shift = digit_shift(r);
            const uint32_t dm = digit_mask(r);
            int* h = hist[buf];
            for (int b = tid; b < kBins; b += kProjectThreads) h[b] = 0;
            __syncthreads();
            int cnt = 0;
            for (int base = 0; base < nloc; base += kProjectThreads) {
                const int j = base + tid;
                bool on = false;
                uint32_t bin = 0;
                if (j < nloc) {
                    const uint32_t key = key_at(j);
                    // first pass: also the doses beyond d_ref, compared with
                    // the FP64 d_ref exactly on keys (d > d_ref iff
                    // key > key_gt, d >= d_ref iff key >= key_ge)
                    if (r == 0) cnt += upper ? (key > dv.key_gt) : (key >= dv.key_ge);
                    on = (key & mask) == prefix;
                    bin = (key >> shift) & dm;
                }
                // warp-aggregated increments (many equal doses share a bin)
                const unsigned act = __ballot_sync(0xffffffffu, on);
                if (on) {
                    const unsigned peers = __match_any_sync(act, bin);
                    if ((int)(__ffs(peers) - 1) == lane) atomicAdd(&h[bin], __popc(peers));
                }
            }
            if (r == 0) {
                cnt = cta_count(cnt, red);
                if (tid == 0) slot_cnt[par] = cnt;
            }
            cl.sync();
            if (r == 0) {
                if (tid == 0) {
                    int v[CL];
#pragma unroll
                    for (int rr = 0; rr < CL; ++rr) v[rr] = *cl.map_shared_rank(slot_cnt + par, rr);
                    int t = 0;
#pragma unroll
                    for (int rr = 0; rr < CL; ++rr) t += v[rr];
                    sh_rank = t;
                }
                __syncthreads();
                const int total = sh_rank;
                feasible = upper ? (total <= K) : (total >= K);
                __syncthreads();
                if (feasible || none_kept) {
                    buf ^= 1;
                    break;
                }
            }
            for (int b = tid; b < kBins; b += kProjectThreads) {
                int v[CL];
#pragma unroll
                for (int rr = 0; rr < CL; ++rr) v[rr] = cl.map_shared_rank(h, rr)[b];
                int t = 0;
#pragma unroll
                for (int rr = 0; rr < CL; ++rr) t += v[rr];
                ghist[b] = t;
            }
            __syncthreads();
            if (wid == 0) {
                // bins from the top: lane L holds bins 255-8L .. 248-8L; the
                // lane whose range holds the kk-th highest key picks the bin
                // and the rank left inside it
                const int nb = (int)dm + 1, per = nb / 32;
                const int top = nb - 1 - per * lane;
                int tot = 0;
                for (int k = 0; k < per; ++k) tot += ghist[top - k];
                int incl = tot;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const int v = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += v;
                }
                const int excl = incl - tot;
                if (excl < kk && kk <= incl) {
                    int above = excl, k = 0;
                    for (; k < per - 1; ++k) {
                        if (above + ghist[top - k] >= kk) break;
                        above += ghist[top - k];
                    }
                    sh_prefix = prefix | ((uint32_t)(top - k) << shift);
                    sh_rank = kk - above;
                    sh_bin = top - k;
                    sh_geq = ghist[top - k];
                }
            }
            __syncthreads();
            prefix = sh_prefix;
            kk = sh_rank;
            mask |= dm << shift;
            if (r == kRounds - 1) {
                // all keys equal to the threshold are kept unless rank falls
                // short of their number; then the ones in the chunks of lower
                // rank come first (their counts: the last round's bin of
                // those CTAs)
                need_order = kk < sh_geq;
                if (need_order && tid < 32) {
                    const int v = (lane < crank) ? cl.map_shared_rank(h, lane)[sh_bin] : 0;
                    int t = v;
#pragma unroll
                    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
                    if (lane == 0) sh_eqbase = t;
                }
                __syncthreads();
                eq_base = sh_eqbase;
            }
        }
        Ff acc{0.f, 0.f};
        if (!feasible) {
            const uint32_t thr = none_kept ? 0xffffffffu : prefix;
            const int rank = kk;
            // apply in row order; a running count ranks the keys equal to thr
            for (int base = 0; base < nloc; base += kProjectThreads) {
                const int j = base + tid;
                const bool in = j < nloc;
                const uint32_t key = in ? key_at(j) : 0u;
                const bool eq = in && !none_kept && key == thr;
                int before = eq_base, tile_total = 0;
                if (need_order) {
                    const unsigned bal = __ballot_sync(0xffffffffu, eq);
                    __syncthreads();
                    if (lane == 0) red[wid] = __popc(bal);
                    __syncthreads();
                    for (int w = 0; w < kProjectThreads / 32; ++w) {
                        const int rr = red[w];
                        before += (w < wid) ? rr : 0;
                        tile_total += rr;
                    }
                    before += __popc(bal & ((1u << lane) - 1u));
                }
                eq_base += tile_total;
                if (in) {
                    const bool kept = !none_kept && (key > thr || (eq && (!need_order || before < rank)));
                    const bool moves = upper ? (!kept && key > dv.key_gt) : (kept && key < dv.key_ge);
                    if (moves) {
                        const Ff e = ff_diff(dv.ref_hi, dv.ref_lo, key_dose(key));
                        a.corr[base_row + j] += dv.wf * e.hi;
                        acc = ff_add(acc, ff_sq(e));
                    }
                }
            }
        }
        // this CTA's sum of the squared corrections (warp tree, warps in
        // order); the chunks are added in rank order by k_dvc_total
        acc = warp_ff(acc);
        __syncthreads();
        if (lane == 0) fred[wid] = acc;
        __syncthreads();
        if (wid == 0) {
            const Ff t = warp_ff(fred[lane]);
            if (lane == 0) a.pd[(size_t)dv.orig * CL + crank] = (double)t.hi + (double)t.lo;
        }
    }
    cl.sync();    // no CTA leaves while another may still read its shared memory
}

// Target-space proximity: 1/2 w_j times each DVC's chunk sums (chunks in rank
// order), the DVCs in the caller's order.
__global__ void k_dvc_total(const double* pd, int ndvc, double* out, const RhsState* st) {
    if (st && st[0].stopped) return;
    if (threadIdx.x == 0) {
        const double hw = 0.5 / (double)ndvc;
        double t = 0.0;
        for (int j = 0; j < ndvc; ++j) {
            double u = 0.0;
            for (int r = 0; r < kDvcCluster; ++r) u += pd[(size_t)j * kDvcCluster + r];
            t += hw * u;
        }
        out[0] = t;
    }
}

// x_j += gamma sum_i a_ij corr_i over the CSC copy: W warps per column (W
// chosen from the mean column length), lanes strided over the column; each
// lane issues the loads of up to eight entries at once, then gathers the
// corrections; per-warp sums added in warp order.
template <int W>
__global__ void __launch_bounds__(kApplyThreads) k_dvc_apply(DvcArgs a) {
    if (a.st && a.st[0].stopped) return;
    constexpr int kGroups = kApplyThreads / (32 * W);
    constexpr int kStep = 32 * W;
    __shared__ float part[kApplyThreads / 32];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = wid / W, wg = wid % W;
    for (int j0 = blockIdx.x * kGroups; j0 < a.n; j0 += gridDim.x * kGroups) {
        const int j = j0 + g;
        float sum = 0.f;
        int e1 = 0, e0 = 0;
        if (j < a.n) {
            e0 = a.cp[j];
            e1 = a.cp[j + 1];
            for (int b = e0 + wg * 32 + lane; b < e1; b += 8 * kStep) {
                int r[8];
                float v[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int e = b + u * kStep;
                    const bool ok = e < e1;
                    r[u] = ok ? a.crow[e] : 0;
                    v[u] = ok ? __ldg(a.cval + e) : 0.f;
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) sum = fmaf(v[u], a.corr[r[u]], sum);
            }
        }
        const float ws = warp_sum_f(sum);
        if (lane == 0) part[wid] = ws;
        __syncthreads();
        if (wg == 0 && lane == 0 && j < a.n && e1 > e0) {
            float t = 0.f;
#pragma unroll
            for (int w = 0; w < W; ++w) t += part[g * W + w];
            float* xj = a.xw + (size_t)j * a.B;
            *xj = *xj + a.gamma * t;
        }
        __syncthreads();
    }
}

// ||A_s||_F^2 per structure (FP64, fixed order): CTA (s, c) sums chunk c of
// structure s's entries, then one thread per structure adds the chunks in
// order.
constexpr int kFrobChunks = 32;
__global__ void __launch_bounds__(kDoseThreads) k_dvc_frob(const int* rp, const float* val,
                                                           const int* sptr, double* part) {
    const int s = blockIdx.x / kFrobChunks, c = blockIdx.x % kFrobChunks;
    const long long e0 = rp[sptr[s]], e1 = rp[sptr[s + 1]];
    const long long len = (e1 - e0 + kFrobChunks - 1) / kFrobChunks;
    const long long b0 = e0 + (long long)c * len, b1 = min(e1, b0 + len);
    double acc = 0.0;
    for (long long e = b0 + threadIdx.x; e < b1; e += kDoseThreads) {
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
        part[blockIdx.x] = t;
    }
}

__global__ void k_dvc_frob_sum(const double* part, int nstruct, double* out) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nstruct) return;
    double t = 0.0;
    for (int c = 0; c < kFrobChunks; ++c) t += part[(size_t)s * kFrobChunks + c];
    out[s] = t;
}

}  // namespace

cudaError_t launch_dvc_dose(const DvcArgs& a, cudaStream_t s) {
    const int grid = (int)std::min<long long>(((long long)a.mq * 32 + kDoseThreads - 1) / kDoseThreads,
                                              152LL * 64);
    if (a.mq > 0) k_dvc_dose<<<grid, kDoseThreads, 0, s>>>(a);
    return cudaGetLastError();
}

size_t dvc_project_smem(int max_rows) {
    const size_t b = (size_t)((max_rows + kDvcCluster - 1) / kDvcCluster) * sizeof(uint32_t);
    return b <= kDvcSmemMax ? b : 0;
}

cudaError_t launch_dvc_project(const DvcArgs& a, cudaStream_t s) {
    if (a.nstruct > 0) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(a.nstruct * kDvcCluster, 1, 1);
        cfg.blockDim = dim3(kProjectThreads, 1, 1);
        cfg.dynamicSmemBytes = a.smem;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = kDvcCluster;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cudaError_t e;
        if (a.smem > 0) {
            e = cudaFuncSetAttribute(k_dvc_project<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)a.smem);
            if (e == cudaSuccess) e = cudaLaunchKernelEx(&cfg, k_dvc_project<true>, a);
        } else {
            e = cudaLaunchKernelEx(&cfg, k_dvc_project<false>, a);
        }
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_dvc_total<<<1, 32, 0, s>>>(a.pd, a.ndvc, a.target, a.st);
    return cudaGetLastError();
}

cudaError_t launch_dvc_apply(const DvcArgs& a, cudaStream_t s) {
    if (a.n <= 0) return cudaSuccess;
    const long long mean = a.nnz / a.n;
    const int W = mean >= 1024 ? 8 : mean >= 512 ? 4 : mean >= 256 ? 2 : 1;
    const int groups = kApplyThreads / (32 * W);
    const int grid = (int)std::min<long long>((a.n + groups - 1) / groups, 152LL * 64);
    switch (W) {
        case 8: k_dvc_apply<8><<<grid, kApplyThreads, 0, s>>>(a); break;
        case 4: k_dvc_apply<4><<<grid, kApplyThreads, 0, s>>>(a); break;
        case 2: k_dvc_apply<2><<<grid, kApplyThreads, 0, s>>>(a); break;
        default: k_dvc_apply<1><<<grid, kApplyThreads, 0, s>>>(a); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_dvc_frob(const int* rp, const float* val, const int* sptr, int nstruct,
                            double* part, double* out, cudaStream_t s) {
    if (nstruct <= 0) return cudaSuccess;
    k_dvc_frob<<<nstruct * kFrobChunks, kDoseThreads, 0, s>>>(rp, val, sptr, part);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_dvc_frob_sum<<<(nstruct + 127) / 128, 128, 0, s>>>(part, nstruct, out);
    return cudaGetLastError();
}

}  // namespace suppy
