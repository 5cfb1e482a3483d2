// Fused one-pass CSR hyperslab sweep (the simultaneous projection step of
// Sec. 2.1.1 with the relaxation of Eq. (3)), its finalize step (box of
// Sec. 2.3.3) and the deterministic second-level proximity reduction
// (Eq. (WeightedProximity)).
//
// For every row i a group of G lanes streams a_i once from HBM with 128-bit
// loads (L1 bypass, L2 evict-first), forms r_i = <a_i, x> with an in-group
// shuffle reduction, computes d_i = clamp(r_i, l_i, u_i) - r_i and the
// correction coefficient lambda * w_i / ||a_i||^2 * d_i, and scatter-adds
// coef * a_i into delta with fire-and-forget L2 reductions -- reusing the row
// held in registers, so A crosses HBM once per sweep.  The proximity term
// w_i d_i^2 / ||a_i||^2 of the sweep's input point is accumulated in FP64 in a
// fixed order (per group, per CTA, then across CTAs in the finalize kernel).
#include "common.cuh"

namespace suppy {
namespace {

__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ int4 ld_stream_i4(const int* ptr, uint64_t pol) {
    int4 v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.s32 {%0,%1,%2,%3}, [%4], %5;"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
        : "l"(ptr), "l"(pol));
    return v;
}

template <typename VT>
struct ValLoad;

template <>
struct ValLoad<float> {
    static __device__ __forceinline__ float4 load4(const float* ptr, uint64_t pol) {
        float4 v;
        asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.f32 {%0,%1,%2,%3}, [%4], %5;"
            : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
            : "l"(ptr), "l"(pol));
        return v;
    }
};

template <>
struct ValLoad<__nv_bfloat16> {
    static __device__ __forceinline__ float4 load4(const __nv_bfloat16* ptr, uint64_t pol) {
        uint32_t a, b;
        asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.b32 {%0,%1}, [%2], %3;"
            : "=r"(a), "=r"(b)
            : "l"(ptr), "l"(pol));
        // bf16 -> fp32 is exact: the bf16 bits are the high half of the fp32
        return make_float4(__uint_as_float(a << 16), __uint_as_float(a & 0xffff0000u),
                           __uint_as_float(b << 16), __uint_as_float(b & 0xffff0000u));
    }
};

template <>
struct ValLoad<__half> {
    static __device__ __forceinline__ float4 load4(const __half* ptr, uint64_t pol) {
        uint32_t a, b;
        asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.b32 {%0,%1}, [%2], %3;"
            : "=r"(a), "=r"(b)
            : "l"(ptr), "l"(pol));
        __half2 ha = *reinterpret_cast<__half2*>(&a), hb = *reinterpret_cast<__half2*>(&b);
        float2 fa = __half22float2(ha), fb = __half22float2(hb);
        return make_float4(fa.x, fa.y, fb.x, fb.y);
    }
};

// Scalar value load through L1 (the batched kernel re-reads its row).
template <typename VT>
__device__ __forceinline__ float ld_val(const VT* p) {
    return __ldg(p);
}
template <>
__device__ __forceinline__ float ld_val<__nv_bfloat16>(const __nv_bfloat16* p) {
    return __bfloat162float(__ldg(p));
}
template <>
__device__ __forceinline__ float ld_val<__half>(const __half* p) {
    return __half2float(__ldg(p));
}

__device__ __forceinline__ void red_add_v4(float* p, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1,%2,%3,%4};" ::"l"(p), "f"(a), "f"(b), "f"(c),
                 "f"(d)
                 : "memory");
}

// ---------------------------------------------------------------- B = 1 ----
// G lanes per row (4..32), up to MAXCH chunks of 4*G elements held in
// registers between the dot product and the scatter; longer rows stream their
// remaining chunks twice (the second read hits L2).
template <typename VT, int G, int MAXCH>
__global__ void __launch_bounds__(kSweepThreads) k_sweep(const SweepArgs a) {
    if (a.check_stop && a.st[0].stopped) return;
    const int lane = threadIdx.x & (G - 1);
    const unsigned gmask =
        (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
    const int grp = (blockIdx.x * kSweepThreads + threadIdx.x) / G;
    const int rb = a.part[grp], re = a.part[grp + 1];
    const uint64_t pol = policy_evict_first();
    const VT* __restrict__ val = static_cast<const VT*>(a.val);
    const int* __restrict__ colp = a.col;
    const float* __restrict__ x = a.x;
    float* __restrict__ delta = a.delta;
    double prox = 0.0;

    for (int i = rb; i < re; ++i) {
        const int2 ri = a.rinfo[i];
        const int len = ri.y;
        if (len == 0) continue;
        const VT* vrow = val + ri.x;
        const int* crow = colp + ri.x;
        const int nch = (len + 4 * G - 1) / (4 * G);
        float4 v[MAXCH];
        int4 c[MAXCH];
#pragma unroll
        for (int k = 0; k < MAXCH; ++k) {
            const int e = k * 4 * G + 4 * lane;
            if (k < nch && e < len) {
                v[k] = ValLoad<VT>::load4(vrow + e, pol);
                c[k] = ld_stream_i4(crow + e, pol);
            } else {
                v[k] = make_float4(0.f, 0.f, 0.f, 0.f);
                c[k] = make_int4(0, 0, 0, 0);
            }
        }
        float dot = 0.f;
#pragma unroll
        for (int k = 0; k < MAXCH; ++k) {
            if (k < nch) {
                dot = fmaf(v[k].x, __ldg(x + c[k].x), dot);
                dot = fmaf(v[k].y, __ldg(x + c[k].y), dot);
                dot = fmaf(v[k].z, __ldg(x + c[k].z), dot);
                dot = fmaf(v[k].w, __ldg(x + c[k].w), dot);
            }
        }
        for (int k = MAXCH; k < nch; ++k) {
            const int e = k * 4 * G + 4 * lane;
            if (e < len) {
                const float4 vv = ValLoad<VT>::load4(vrow + e, pol);
                const int4 cc = ld_stream_i4(crow + e, pol);
                dot = fmaf(vv.x, __ldg(x + cc.x), dot);
                dot = fmaf(vv.y, __ldg(x + cc.y), dot);
                dot = fmaf(vv.z, __ldg(x + cc.z), dot);
                dot = fmaf(vv.w, __ldg(x + cc.w), dot);
            }
        }
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) dot += __shfl_xor_sync(gmask, dot, o);

        const float d = clampf(dot, a.l[i], a.u[i]) - dot;
        const float w = a.wr[i];
        if (lane == 0) prox += (double)d * (double)d * (double)w;
        const float coef = a.lam * w * d;
        if (a.scatter && coef != 0.f) {
#pragma unroll
            for (int k = 0; k < MAXCH; ++k) {
                const int e = k * 4 * G + 4 * lane;
                if (k < nch && e < len) {
                    atomicAdd(delta + c[k].x, coef * v[k].x);
                    if (e + 1 < len) atomicAdd(delta + c[k].y, coef * v[k].y);
                    if (e + 2 < len) atomicAdd(delta + c[k].z, coef * v[k].z);
                    if (e + 3 < len) atomicAdd(delta + c[k].w, coef * v[k].w);
                }
            }
            for (int k = MAXCH; k < nch; ++k) {
                const int e = k * 4 * G + 4 * lane;
                if (e < len) {
                    const float4 vv = ValLoad<VT>::load4(vrow + e, pol);
                    const int4 cc = ld_stream_i4(crow + e, pol);
                    atomicAdd(delta + cc.x, coef * vv.x);
                    if (e + 1 < len) atomicAdd(delta + cc.y, coef * vv.y);
                    if (e + 2 < len) atomicAdd(delta + cc.z, coef * vv.z);
                    if (e + 3 < len) atomicAdd(delta + cc.w, coef * vv.w);
                }
            }
        }
    }
    // deterministic CTA partial: warp tree, then warps in order
    prox = warp_sum(prox);
    __shared__ double sw[kSweepThreads / 32];
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = prox;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < kSweepThreads / 32; ++w) s += sw[w];
        a.pp[blockIdx.x] = s;
    }
}

// -------------------------------------------------------------- B = 4Q ----
// One warp per row; lane = e*Q + q handles element slot e (E = 32/Q slots per
// pass) and right-hand sides 4q..4q+3, so the Q lanes of one element gather
// the contiguous 4B floats X[col*B .. col*B+B) with 128-bit loads and scatter
// them back with 128-bit vector reductions.  The row is streamed from HBM for
// the dot products and re-read (L1/L2) for the scatter.
template <typename VT, int Q>
__global__ void __launch_bounds__(kSweepThreads) k_sweep_batched(const SweepArgs a) {
    constexpr int E = 32 / Q;
    constexpr int B = 4 * Q;
    const int lane = threadIdx.x & 31;
    const int q = lane % Q;
    const int e0 = lane / Q;
    const int warp = (blockIdx.x * kSweepThreads + threadIdx.x) >> 5;
    const int rb = a.part[warp], re = a.part[warp + 1];
    const VT* __restrict__ val = static_cast<const VT*>(a.val);
    const int* __restrict__ colp = a.col;
    const float* __restrict__ X = a.x;
    float* __restrict__ D = a.delta;
    bool live[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) live[t] = !a.st[4 * q + t].stopped;
    double prox[4] = {0.0, 0.0, 0.0, 0.0};

    for (int i = rb; i < re; ++i) {
        const int2 ri = a.rinfo[i];
        const int len = ri.y;
        if (len == 0) continue;
        const VT* vrow = val + ri.x;
        const int* crow = colp + ri.x;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int e = e0; e < len; e += E) {
            const float v = ld_val<VT>(vrow + e);
            const int c = __ldg(crow + e);
            const float4 xv = __ldg(reinterpret_cast<const float4*>(X + (size_t)c * B) + q);
            acc.x = fmaf(v, xv.x, acc.x);
            acc.y = fmaf(v, xv.y, acc.y);
            acc.z = fmaf(v, xv.z, acc.z);
            acc.w = fmaf(v, xv.w, acc.w);
        }
#pragma unroll
        for (int o = 16; o >= Q; o >>= 1) {
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
            acc.z += __shfl_xor_sync(0xffffffffu, acc.z, o);
            acc.w += __shfl_xor_sync(0xffffffffu, acc.w, o);
        }
        const float4 lv = __ldg(reinterpret_cast<const float4*>(a.l + (size_t)i * B) + q);
        const float4 uv = __ldg(reinterpret_cast<const float4*>(a.u + (size_t)i * B) + q);
        const float w = a.wr[i];
        float d[4];
        d[0] = clampf(acc.x, lv.x, uv.x) - acc.x;
        d[1] = clampf(acc.y, lv.y, uv.y) - acc.y;
        d[2] = clampf(acc.z, lv.z, uv.z) - acc.z;
        d[3] = clampf(acc.w, lv.w, uv.w) - acc.w;
        float cf[4];
        bool any = false;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            if (e0 == 0) prox[t] += (double)d[t] * (double)d[t] * (double)w;
            cf[t] = live[t] ? a.lam * w * d[t] : 0.f;
            any |= (cf[t] != 0.f);
        }
        if (a.scatter && any) {
            for (int e = e0; e < len; e += E) {
                const float v = ld_val<VT>(vrow + e);
                const int c = __ldg(crow + e);
                red_add_v4(D + (size_t)c * B + 4 * q, cf[0] * v, cf[1] * v, cf[2] * v,
                           cf[3] * v);
            }
        }
    }
    // per-CTA partial per right-hand side, fixed order
    __shared__ double sw[kSweepThreads / 32][B];
    const int wid = threadIdx.x >> 5;
    if (e0 == 0) {
#pragma unroll
        for (int t = 0; t < 4; ++t) sw[wid][4 * q + t] = prox[t];
    }
    __syncthreads();
    if (threadIdx.x < B) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < kSweepThreads / 32; ++w) s += sw[w][threadIdx.x];
        a.pp[(size_t)blockIdx.x * B + threadIdx.x] = s;
    }
}

// ------------------------------------------------------------- finalize ----
// x <- clamp(x + delta, lo, hi), delta <- 0 (n x B elements, 128-bit).  CTA 0
// also reduces the sweep's proximity partials in a fixed order, records the
// history and advances the stopping rule of each right-hand side.
__global__ void __launch_bounds__(kFinalizeThreads) k_finalize(const FinalizeArgs a) {
    const long long nv = a.nB >> 2;   // nB is a multiple of 4 (n*B, B in {1,4..32} padded)
    float4* x4 = reinterpret_cast<float4*>(a.x);
    float4* d4 = reinterpret_cast<float4*>(a.delta);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += stride) {
        float4 xv = x4[v];
        const float4 dv = d4[v];
        float lo[4], hi[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const long long idx = 4 * v + t;
            const long long j = (a.box_len == 1) ? 0 : idx / a.B;
            lo[t] = a.lo[j];
            hi[t] = a.hi[j];
        }
        xv.x = clampf(xv.x + dv.x, lo[0], hi[0]);
        xv.y = clampf(xv.y + dv.y, lo[1], hi[1]);
        xv.z = clampf(xv.z + dv.z, lo[2], hi[2]);
        xv.w = clampf(xv.w + dv.w, lo[3], hi[3]);
        x4[v] = xv;
        d4[v] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    // tail when n*B is not a multiple of 4 (B = 1 only)
    if (blockIdx.x == 0) {
        for (long long idx = 4 * nv + threadIdx.x; idx < a.nB; idx += blockDim.x) {
            const long long j = (a.box_len == 1) ? 0 : idx / a.B;
            a.x[idx] = clampf(a.x[idx] + a.delta[idx], a.lo[j], a.hi[j]);
            a.delta[idx] = 0.f;
        }
    }
    if (blockIdx.x != 0) return;
    // proximity partials: warp w handles right-hand sides w, w+8, ...
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int b = wid; b < a.B; b += kFinalizeThreads / 32) {
        double s = 0.0;
        for (int c = lane; c < a.npp; c += 32) s += a.pp[(size_t)c * a.B + b];
        s = warp_sum(s);
        if (lane != 0) continue;
        RhsState& st = a.st[b];
        if (st.stopped) continue;
        if (a.first_seg) st.p_acc = 0.0;
        st.p_acc += a.scale * s;
        if (!a.last_seg) continue;
        const double p = st.p_acc;
        const int k = st.k;
        if (k < a.hist_cap) {
            a.prox_hist[(size_t)b * a.hist_cap + k] = p;
            a.obj_hist[(size_t)b * a.hist_cap + k] = st.f_valid ? st.f_cur : __longlong_as_double(0x7ff8000000000000LL);
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
        if (a.sp.use_stopping && feas && objok) st.stopped = 1;
    }
}

// Sum partials pp[c*B + b] over c in a fixed order: out[b] (+)= scale * sum.
__global__ void k_reduce_pp(const double* pp, int npp, int B, double scale, int accumulate,
                            double* out) {
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int b = wid; b < B; b += blockDim.x / 32) {
        double s = 0.0;
        for (int c = lane; c < npp; c += 32) s += pp[(size_t)c * B + b];
        s = warp_sum(s);
        if (lane == 0) out[b] = (accumulate ? out[b] : 0.0) + scale * s;
    }
}

using SweepFn = void (*)(SweepArgs);

template <typename VT>
SweepFn pick_sweep(int G, int maxch) {
    if (G == 32 && maxch == 8) return k_sweep<VT, 32, 8>;
    if (G == 32 && maxch == 4) return k_sweep<VT, 32, 4>;
    if (G == 32 && maxch == 2) return k_sweep<VT, 32, 2>;
    if (G == 16 && maxch == 4) return k_sweep<VT, 16, 4>;
    if (G == 16 && maxch == 2) return k_sweep<VT, 16, 2>;
    if (G == 8 && maxch == 4) return k_sweep<VT, 8, 4>;
    if (G == 8 && maxch == 2) return k_sweep<VT, 8, 2>;
    if (G == 4 && maxch == 2) return k_sweep<VT, 4, 2>;
    return nullptr;
}

template <typename VT>
SweepFn pick_batched(int B) {
    switch (B) {
        case 4: return k_sweep_batched<VT, 1>;
        case 8: return k_sweep_batched<VT, 2>;
        case 16: return k_sweep_batched<VT, 4>;
        case 32: return k_sweep_batched<VT, 8>;
        default: return nullptr;
    }
}

}  // namespace

cudaError_t launch_sweep(const SweepArgs& a, suppy_dtype dt, int G, int maxch, int grid,
                         cudaStream_t s) {
    SweepFn f = nullptr;
    if (dt == SUPPY_F32) f = pick_sweep<float>(G, maxch);
    else if (dt == SUPPY_BF16) f = pick_sweep<__nv_bfloat16>(G, maxch);
    else f = pick_sweep<__half>(G, maxch);
    if (!f) return cudaErrorInvalidValue;
    f<<<grid, kSweepThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_sweep_batched(const SweepArgs& a, suppy_dtype dt, int /*G*/, int grid,
                                 cudaStream_t s) {
    SweepFn f = nullptr;
    if (dt == SUPPY_F32) f = pick_batched<float>(a.B);
    else if (dt == SUPPY_BF16) f = pick_batched<__nv_bfloat16>(a.B);
    else f = pick_batched<__half>(a.B);
    if (!f) return cudaErrorInvalidValue;
    f<<<grid, kSweepThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const FinalizeArgs& a, int grid, cudaStream_t s) {
    k_finalize<<<grid, kFinalizeThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_reduce_pp(const double* pp, int npp, int B, double scale, int accumulate,
                             double* out, cudaStream_t s) {
    k_reduce_pp<<<1, 256, 0, s>>>(pp, npp, B, scale, accumulate, out);
    return cudaGetLastError();
}

}  // namespace suppy

namespace suppy {

int sweep_blocks_per_sm(suppy_dtype dt, int G, int maxch, int batchedB) {
    SweepFn f = nullptr;
    if (batchedB > 1) {
        if (dt == SUPPY_F32) f = pick_batched<float>(batchedB);
        else if (dt == SUPPY_BF16) f = pick_batched<__nv_bfloat16>(batchedB);
        else f = pick_batched<__half>(batchedB);
    } else {
        if (dt == SUPPY_F32) f = pick_sweep<float>(G, maxch);
        else if (dt == SUPPY_BF16) f = pick_sweep<__nv_bfloat16>(G, maxch);
        else f = pick_sweep<__half>(G, maxch);
    }
    if (!f) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, kSweepThreads, 0) != cudaSuccess)
        return 0;
    return nb;
}

}  // namespace suppy
