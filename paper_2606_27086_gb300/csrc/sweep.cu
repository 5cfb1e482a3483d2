// Simultaneous hyperslab projection sweep (Sec. 2.1.1 with the relaxation of
// Eq. (3)) and its finalize step (box of Sec. 2.3.3), with the deterministic
// FP64 proximity of Eq. (WeightedProximity) fused in.
//
// Two strategies share the row pass:
//  * one-pass: a group of G lanes streams row a_i once from HBM (lane-strided,
//    fully coalesced loads, L1 bypass, L2 evict-first), keeps it in registers,
//    forms r_i = <a_i, x> with an in-group shuffle tree, computes
//    coef_i = lambda w_i (clamp(r_i, l_i, u_i) - r_i) / ||a_i||^2 and
//    scatter-adds coef_i * a_i into delta -- with global L2 reductions whose
//    lanes hit consecutive columns (address-coalesced), or staged in shared
//    memory when delta fits there -- then the finalize kernel applies the box;
//  * two-pass: the row pass writes coef_i only; a column pass streams the CSC
//    copy of A and computes x_j <- box(x_j + sum_i a_ij coef_i) with gathers
//    of coef from L2, no atomics at all (bitwise deterministic).
#include <algorithm>

#include "common.cuh"

namespace suppy {

#ifdef SUPPY_CHECKED
__device__ int g_check[3];
__device__ __noinline__ bool check_fail(int tag, long long idx) {
    if (atomicCAS(&g_check[0], 0, tag) == 0) {
        g_check[1] = (int)(idx & 0xffffffffLL);
        g_check[2] = (int)(idx >> 32);
    }
    return false;
}
#define CHECKED(cond, tag, idx) ((cond) ? true : check_fail((tag), (long long)(idx)))
#define ALIGNED16(p) ((((uintptr_t)(p)) & 15u) == 0)
#else
#define CHECKED(cond, tag, idx) true
#define ALIGNED16(p) true
#endif

cudaError_t read_check_word(int* out3) {
#ifdef SUPPY_CHECKED
    cudaError_t e = cudaMemcpyFromSymbol(out3, g_check, sizeof(int) * 3);
    if (e != cudaSuccess) return e;
    int z[3] = {0, 0, 0};
    return cudaMemcpyToSymbol(g_check, z, sizeof(int) * 3);
#else
    out3[0] = out3[1] = out3[2] = 0;
    return cudaSuccess;
#endif
}

namespace {

__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ int ld_stream_i(const int* ptr, uint64_t pol) {
    int v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(ptr), "l"(pol));
    return v;
}

template <typename VT>
__device__ __forceinline__ float ld_stream_v(const VT* ptr, uint64_t pol);
template <>
__device__ __forceinline__ float ld_stream_v<float>(const float* ptr, uint64_t pol) {
    float v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(ptr), "l"(pol));
    return v;
}
template <>
__device__ __forceinline__ float ld_stream_v<__nv_bfloat16>(const __nv_bfloat16* ptr, uint64_t pol) {
    unsigned short h;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.b16 %0, [%1], %2;" : "=h"(h) : "l"(ptr), "l"(pol));
    return __uint_as_float(((uint32_t)h) << 16);   // exact widening
}
template <>
__device__ __forceinline__ float ld_stream_v<__half>(const __half* ptr, uint64_t pol) {
    unsigned short h;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.b16 %0, [%1], %2;" : "=h"(h) : "l"(ptr), "l"(pol));
    return __half2float(__ushort_as_half(h));
}

__device__ __forceinline__ void red_add_v4(float* p, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1,%2,%3,%4};" ::"l"(p), "f"(a), "f"(b), "f"(c),
                 "f"(d)
                 : "memory");
}

template <int G>
__device__ __forceinline__ unsigned group_mask() {
    if constexpr (G == 32) return 0xffffffffu;
    else return ((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1));
}

// Per-CTA proximity partial: lane 0 of each group holds its sum; warp tree,
// then warps in order.
__device__ __forceinline__ void cta_partial(double prox, double* out) {
    prox = warp_sum(prox);
    __shared__ double sw[kSweepThreads / 32];
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = prox;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < kSweepThreads / 32; ++w) s += sw[w];
        *out = s;
    }
}

// ------------------------------------------------------ row pass, B = 1 ----
// Lane `lane` of a G-lane group owns elements lane, lane+G, lane+2G, ... of
// the row.  Loads are issued in batches (all values and indices of a batch
// first, then all gathers of x) so that each lane keeps many independent
// loads in flight.  The first MAXE*G elements stay in registers for the
// scatter; longer rows stream their tail in batches of 8 per lane, twice.
// SCAT: 0 none (coefficients / proximity only), 1 global, 2 shared memory.
template <typename VT, int G, int U>
__device__ __forceinline__ float dot_batch(const VT* vrow, const int* crow, int base, int len,
                                           int lane, const float* __restrict__ x, uint64_t pol) {
    float v[U];
    int c[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int e = base + u * G + lane;
        if (e < len) {
            v[u] = ld_stream_v<VT>(vrow + e, pol);
            c[u] = ld_stream_i(crow + e, pol);
        } else {
            v[u] = 0.f;
            c[u] = 0;
        }
    }
    float s = 0.f;
#pragma unroll
    for (int u = 0; u < U; ++u) s = fmaf(v[u], __ldg(x + c[u]), s);
    return s;
}

template <typename VT, int G, int U>
__device__ __forceinline__ void scatter_batch(const VT* vrow, const int* crow, int base, int len,
                                              int lane, float coef, float* delta, uint64_t pol) {
    float v[U];
    int c[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const int e = base + u * G + lane;
        if (e < len) {
            v[u] = ld_stream_v<VT>(vrow + e, pol);
            c[u] = ld_stream_i(crow + e, pol);
        }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
        if (base + u * G + lane < len) atomicAdd(delta + c[u], coef * v[u]);
}

template <typename VT, int G, int MAXE, int SCAT>
__global__ void __launch_bounds__(kSweepThreads, SCAT == 0 ? 6 : 2) k_sweep(const SweepArgs a) {
    extern __shared__ float s_delta[];
    if (a.check_stop && a.st[0].stopped) return;
    const int lane = threadIdx.x & (G - 1);
    const unsigned gmask = group_mask<G>();
    const int grp = (blockIdx.x * kSweepThreads + threadIdx.x) / G;
    int rb = a.part[grp], re = a.part[grp + 1];
    if (!CHECKED(rb >= 0 && rb <= re && re <= a.m, 1, grp)) re = rb;
    const uint64_t pol = policy_evict_first();
    const VT* __restrict__ val = static_cast<const VT*>(a.val);
    const int* __restrict__ colp = a.col;
    const float* __restrict__ x = a.x;
    float* __restrict__ delta = (SCAT == 2) ? s_delta : a.delta;
    if (SCAT == 2) {
        for (int j = threadIdx.x; j < a.n; j += kSweepThreads) s_delta[j] = 0.f;
        __syncthreads();
    }
    double prox = 0.0;
    constexpr int HOLD = (SCAT == 0) ? 0 : MAXE;   // elements per lane kept for the scatter
    constexpr int TB = (SCAT == 0) ? 8 : 4;        // tail batch per lane

    for (int i = rb; i < re; ++i) {
        const int2 ri = a.rinfo[i];
        const int len = ri.y;
        if (len == 0) continue;
        if (!CHECKED(ri.x >= 0 && (long long)ri.x + len <= a.nnz, 2, i)) continue;
        const VT* vrow = val + ri.x;
        const int* crow = colp + ri.x;
        const float li = __ldg(a.l + i), ui = __ldg(a.u + i), w = __ldg(a.wr + i);
        float v[HOLD > 0 ? HOLD : 1];
        int c[HOLD > 0 ? HOLD : 1];
        float dot = 0.f;
        if constexpr (HOLD > 0) {
#pragma unroll
            for (int k = 0; k < HOLD; ++k) {
                const int e = k * G + lane;
                if (e < len) {
                    v[k] = ld_stream_v<VT>(vrow + e, pol);
                    c[k] = ld_stream_i(crow + e, pol);
                } else {
                    v[k] = 0.f;
                    c[k] = 0;
                }
            }
#pragma unroll
            for (int k = 0; k < HOLD; ++k) dot = fmaf(v[k], __ldg(x + c[k]), dot);
        }
        for (int base = HOLD * G; base < len; base += TB * G)
            dot += dot_batch<VT, G, TB>(vrow, crow, base, len, lane, x, pol);
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) dot += __shfl_xor_sync(gmask, dot, o);

        const float d = clampf(dot, li, ui) - dot;
        const float wp = a.prox_mul ? w * __ldg(a.prox_mul + i) : w;
        if (lane == 0) prox += (double)d * (double)d * (double)wp;
        const float coef = a.lam * w * d * (a.coef_mul ? __ldg(a.coef_mul + i) : 1.f);
        if constexpr (SCAT == 0) {
            if (a.coef && lane == 0) a.coef[i] = coef;
        } else {
            if (coef != 0.f) {
#pragma unroll
                for (int k = 0; k < HOLD; ++k)
                    if (k * G + lane < len) atomicAdd(delta + c[k], coef * v[k]);
                for (int base = HOLD * G; base < len; base += TB * G)
                    scatter_batch<VT, G, TB>(vrow, crow, base, len, lane, coef, delta, pol);
            }
        }
    }
    if (SCAT == 2) {
        // flush the CTA's staged corrections with 128-bit reductions, skipping zeros
        __syncthreads();
        const int n4 = a.n >> 2;
        for (int q = threadIdx.x; q < n4; q += kSweepThreads) {
            const float4 d4 = reinterpret_cast<const float4*>(s_delta)[q];
            if (d4.x != 0.f || d4.y != 0.f || d4.z != 0.f || d4.w != 0.f)
                red_add_v4(a.delta + 4 * q, d4.x, d4.y, d4.z, d4.w);
        }
        for (int j = 4 * n4 + threadIdx.x; j < a.n; j += kSweepThreads)
            if (s_delta[j] != 0.f) atomicAdd(a.delta + j, s_delta[j]);
    }
    cta_partial(prox, a.pp + blockIdx.x);
}

// ------------------------------------------------------ row pass, B = 4Q ----
// One warp per row; lane = e*Q + q handles element slot e (E = 32/Q slots per
// pass) and right-hand sides 4q..4q+3: the Q lanes of one element gather the
// contiguous floats X[col*B .. col*B+B) with 128-bit loads and (one-pass)
// scatter them back with 128-bit vector reductions.  The row is streamed from
// HBM for the dot products and re-read through L1 for the scatter.  The
// coefficient-writing variant is held to 32 registers (eight CTAs an SM: more
// gathers in flight; measured 0.224 -> 0.178 ms on 16 seismic images); the
// scatter variant stays at five CTAs an SM (it spills under the tighter bound).
template <typename VT, int Q, int SCAT>
__global__ void __launch_bounds__(kSweepThreads, SCAT == 0 ? 8 : 5) k_sweep_batched(const SweepArgs a) {
    constexpr int E = 32 / Q;
    constexpr int B = 4 * Q;
    const int lane = threadIdx.x & 31;
    const int q = lane % Q;
    const int e0 = lane / Q;
    const int warp = (blockIdx.x * kSweepThreads + threadIdx.x) >> 5;
    int rb = a.part[warp], re = a.part[warp + 1];
    if (!CHECKED(rb >= 0 && rb <= re && re <= a.m, 101, warp)) re = rb;
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
        if (!CHECKED(ri.x >= 0 && (long long)ri.x + len <= a.nnz, 102, i)) continue;
        const VT* vrow = val + ri.x;
        const int* crow = colp + ri.x;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int e = e0; e < len; e += E) {
            const float v = (float)__ldg(vrow + e);
            int c = __ldg(crow + e);
            if (!CHECKED(c >= 0 && c < a.n && ALIGNED16(X + (size_t)c * B + 4 * q), 103,
                         (long long)i * 64 + e))
                c = 0;
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
        if (!CHECKED(ALIGNED16(a.l + (size_t)i * B + 4 * q) && ALIGNED16(a.u + (size_t)i * B + 4 * q),
                     104, i))
            continue;
        const float4 lv = __ldg(reinterpret_cast<const float4*>(a.l + (size_t)i * B) + q);
        const float4 uv = __ldg(reinterpret_cast<const float4*>(a.u + (size_t)i * B) + q);
        const float w = a.wr[i];
        const float wp = a.prox_mul ? w * a.prox_mul[i] : w;
        const float wc = a.coef_mul ? w * a.coef_mul[i] : w;
        float d[4];
        d[0] = clampf(acc.x, lv.x, uv.x) - acc.x;
        d[1] = clampf(acc.y, lv.y, uv.y) - acc.y;
        d[2] = clampf(acc.z, lv.z, uv.z) - acc.z;
        d[3] = clampf(acc.w, lv.w, uv.w) - acc.w;
        float cf[4];
        bool any = false;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            if (e0 == 0) prox[t] += (double)d[t] * (double)d[t] * (double)wp;
            cf[t] = live[t] ? a.lam * wc * d[t] : 0.f;
            any |= (cf[t] != 0.f);
        }
        if (SCAT == 0) {
            if (a.coef && e0 == 0)
                reinterpret_cast<float4*>(a.coef + (size_t)i * B)[q] =
                    make_float4(cf[0], cf[1], cf[2], cf[3]);
        } else if (any) {
            for (int e = e0; e < len; e += E) {
                const float v = (float)__ldg(vrow + e);
                const int c = __ldg(crow + e);
                if (!CHECKED(c >= 0 && c < a.n && ALIGNED16(D + (size_t)c * B + 4 * q), 105,
                             (long long)i * 64 + e))
                    continue;
                red_add_v4(D + (size_t)c * B + 4 * q, cf[0] * v, cf[1] * v, cf[2] * v, cf[3] * v);
            }
        }
    }
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

// ---------------------------------------------------------- column pass ----
// B = 1: a group of G lanes per column j streams its CSC entries and gathers
// coef from L2; lane 0 applies x_j <- clamp(x_j + sum, lo_j, hi_j).
template <typename VT, int G>
__global__ void __launch_bounds__(kSweepThreads) k_colpass(const ColArgs a) {
    // the row pass skipped a stopped system and left no coefficients; the flag
    // cannot change during this launch (the stopping rule runs in k_epilogue)
    if (a.epi.st[0].stopped) return;
    const int lane = threadIdx.x & (G - 1);
    const unsigned gmask = group_mask<G>();
    const int grp = (blockIdx.x * kSweepThreads + threadIdx.x) / G;
    int jb = a.cpart[grp], je = a.cpart[grp + 1];
    if (!CHECKED(jb >= 0 && jb <= je && je <= a.n, 301, grp)) je = jb;
    const uint64_t pol = policy_evict_first();
    const VT* __restrict__ val = static_cast<const VT*>(a.cval);
    const float* __restrict__ coef = a.coef;
    for (int j = jb; j < je; ++j) {
        const int2 ci = a.cinfo[j];
        if (!CHECKED(ci.x >= 0 && (long long)ci.x + ci.y <= a.nnz, 302, j)) continue;
        const VT* vcol = val + ci.x;
        const int* rcol = a.ridx + ci.x;
        float s = 0.f;
        for (int base = 0; base < ci.y; base += 8 * G)
            s += dot_batch<VT, G, 8>(vcol, rcol, base, ci.y, lane, coef, pol);
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(gmask, s, o);
        if (lane == 0) {   // an empty column still takes the box step
            const int bj = (a.box_len == 1) ? 0 : j;
            if (a.zc) s *= a.zc[j];
            if (a.delta_out) a.delta_out[j] = s;
            else a.x[j] = clampf(a.x[j] + s, a.lo[bj], a.hi[bj]);
        }
    }
    if (blockIdx.x == 0 && !a.epi.last_seg) sweep_epilogue(a.epi);
}

// B = 4Q: one warp per column; lane = e*Q + q gathers the 4 coefficients of
// right-hand sides 4q..4q+3 of row ridx[e] (contiguous 16 bytes).
template <typename VT, int Q>
__global__ void __launch_bounds__(kSweepThreads) k_colpass_batched(const ColArgs a) {
    constexpr int E = 32 / Q;
    constexpr int B = 4 * Q;
    const int lane = threadIdx.x & 31;
    const int q = lane % Q;
    const int e0 = lane / Q;
    const int warp = (blockIdx.x * kSweepThreads + threadIdx.x) >> 5;
    int jb = a.cpart[warp], je = a.cpart[warp + 1];
    if (!CHECKED(jb >= 0 && jb <= je && je <= a.n, 311, warp)) je = jb;
    const VT* __restrict__ val = static_cast<const VT*>(a.cval);
    for (int j = jb; j < je; ++j) {
        const int2 ci = a.cinfo[j];   // an empty column still takes the box step
        if (!CHECKED(ci.x >= 0 && (long long)ci.x + ci.y <= a.nnz, 312, j)) continue;
        const VT* vcol = val + ci.x;
        const int* rcol = a.ridx + ci.x;
        float4 s = make_float4(0.f, 0.f, 0.f, 0.f);
        auto load_el = [&](int e, float& v, int& r) {
            v = (float)__ldg(vcol + e);
            r = __ldg(rcol + e);
            if (!CHECKED(r >= 0 && r < a.m && ALIGNED16(a.coef + (size_t)r * B + 4 * q), 313,
                         (long long)j * 64 + e))
                r = 0;
        };
        auto fma4 = [&](float v, const float4& cv) {
            s.x = fmaf(v, cv.x, s.x);
            s.y = fmaf(v, cv.y, s.y);
            s.z = fmaf(v, cv.z, s.z);
            s.w = fmaf(v, cv.w, s.w);
        };
        int e = e0;
        // four elements a lane in flight: their loads, then their gathers
        for (; e + 3 * E < ci.y; e += 4 * E) {
            float v[4];
            int r[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) load_el(e + u * E, v[u], r[u]);
            float4 cv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                cv[u] = __ldg(reinterpret_cast<const float4*>(a.coef + (size_t)r[u] * B) + q);
#pragma unroll
            for (int u = 0; u < 4; ++u) fma4(v[u], cv[u]);
        }
        for (; e < ci.y; e += E) {
            float v;
            int r;
            load_el(e, v, r);
            fma4(v, __ldg(reinterpret_cast<const float4*>(a.coef + (size_t)r * B) + q));
        }
#pragma unroll
        for (int o = 16; o >= Q; o >>= 1) {
            s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
            s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
            s.z += __shfl_xor_sync(0xffffffffu, s.z, o);
            s.w += __shfl_xor_sync(0xffffffffu, s.w, o);
        }
        if (e0 == 0 && CHECKED(ALIGNED16(a.x + (size_t)j * B + 4 * q), 314, j)) {
            const int bj = (a.box_len == 1) ? 0 : j;
            const float lo = a.lo[bj], hi = a.hi[bj];
            if (a.zc) {
                const float z = a.zc[j];
                s.x *= z;
                s.y *= z;
                s.z *= z;
                s.w *= z;
            }
            if (a.delta_out) {
                reinterpret_cast<float4*>(a.delta_out + (size_t)j * B)[q] = s;
                continue;
            }
            float4* xp = reinterpret_cast<float4*>(a.x + (size_t)j * B) + q;
            float4 xv = *xp;
            xv.x = clampf(xv.x + s.x, lo, hi);
            xv.y = clampf(xv.y + s.y, lo, hi);
            xv.z = clampf(xv.z + s.z, lo, hi);
            xv.w = clampf(xv.w + s.w, lo, hi);
            *xp = xv;
        }
    }
    if (blockIdx.x == 0 && !a.epi.last_seg) sweep_epilogue(a.epi);
}

// Epilogue of the last block of a two-pass sweep (it may set the stop flag, so
// it runs after every column-pass CTA has read that flag).
__global__ void k_epilogue(const EpiArgs a) { sweep_epilogue(a); }

// ------------------------------------------------------------- finalize ----
// x <- clamp(x + delta, lo, hi), delta <- 0 (n x B elements, 128-bit); CTA 0
// also runs the sweep epilogue.
__global__ void __launch_bounds__(kFinalizeThreads) k_finalize(const FinalizeArgs a) {
    long long nv = a.nB >> 2;
    if (!CHECKED(ALIGNED16(a.x) && ALIGNED16(a.delta), 201, 0)) nv = 0;
    float4* x4 = reinterpret_cast<float4*>(a.x);
    float4* d4 = reinterpret_cast<float4*>(a.delta);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < nv; v += stride) {
        float4 xv = x4[v];
        float4 dv = d4[v];
        float lo[4], hi[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const long long idx = 4 * v + t;
            const long long j = (a.box_len == 1) ? 0 : idx / a.B;
            lo[t] = a.lo[j];
            hi[t] = a.hi[j];
        }
        if (a.zc) {
            dv.x *= a.zc[(4 * v) / a.B];
            dv.y *= a.zc[(4 * v + 1) / a.B];
            dv.z *= a.zc[(4 * v + 2) / a.B];
            dv.w *= a.zc[(4 * v + 3) / a.B];
        }
        xv.x = clampf(xv.x + dv.x, lo[0], hi[0]);
        xv.y = clampf(xv.y + dv.y, lo[1], hi[1]);
        xv.z = clampf(xv.z + dv.z, lo[2], hi[2]);
        xv.w = clampf(xv.w + dv.w, lo[3], hi[3]);
        x4[v] = xv;
        d4[v] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    if (blockIdx.x == 0) {
        for (long long idx = 4 * nv + threadIdx.x; idx < a.nB; idx += blockDim.x) {
            const long long j = (a.box_len == 1) ? 0 : idx / a.B;
            const float d = a.zc ? a.delta[idx] * a.zc[idx / a.B] : a.delta[idx];
            a.x[idx] = clampf(a.x[idx] + d, a.lo[j], a.hi[j]);
            a.delta[idx] = 0.f;
        }
        sweep_epilogue(a.epi);
    }
}

// The same box step with the one-pass scatter's column-major second
// accumulator (one right-hand side on an H x W image): x_j <- clamp(x_j +
// delta_j + deltaT_(c,r), lo, hi) for pixel j = (r, c), both accumulators
// cleared.  Tiles of 32 image rows x 8 columns, one pixel per thread: deltaT
// is read along its columns (32 consecutive floats), x and delta along the
// image rows (8), every load issued before any is used, and the transposed
// values pass through shared memory.
constexpr int kTrRows = 32, kTrCols = 8;
__global__ void __launch_bounds__(256) k_finalize_tr(const FinalizeArgs a) {
    __shared__ float t[kTrCols][kTrRows + 1];
    const int H = a.imgH, W = a.imgW;
    const int tw = (W + kTrCols - 1) / kTrCols;
    const long long ntiles = (long long)tw * ((H + kTrRows - 1) / kTrRows);
    // deltaT side: column c0 + ty, row r0 + tx; image side: row r0 + iy, column c0 + ix
    const int tx = threadIdx.x % kTrRows, ty = threadIdx.x / kTrRows;
    const int ix = threadIdx.x % kTrCols, iy = threadIdx.x / kTrCols;
    for (long long ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
        const int r0 = (int)(ti / tw) * kTrRows, c0 = (int)(ti % tw) * kTrCols;
        const int cT = c0 + ty, rT = r0 + tx;
        const int r = r0 + iy, c = c0 + ix;
        const bool inT = cT < W && rT < H, in = r < H && c < W;
        const long long jT = (long long)cT * H + rT, j = (long long)r * W + c;
        const float tv = inT ? a.deltaT[jT] : 0.f;
        const float dv = in ? a.delta[j] : 0.f;
        const float xv = in ? a.x[j] : 0.f;
        if (inT) a.deltaT[jT] = 0.f;
        if (in) a.delta[j] = 0.f;
        t[ty][tx] = tv;
        __syncthreads();
        if (in) {
            float d = dv + t[ix][iy];
            if (a.zc) d *= a.zc[j];
            const long long bj = (a.box_len == 1) ? 0 : j;
            a.x[j] = clampf(xv + d, a.lo[bj], a.hi[bj]);
        }
        __syncthreads();
    }
    if (blockIdx.x == 0) sweep_epilogue(a.epi);
}

// Patch blocks: one thread per 4 x 4 pixel block (x0 = 4 bx, y0 = 4 by) of
// the padded grid.  Such a block is exactly two 32-byte sectors of each patch
// layout: in the wide layout the sectors of rows y0, y0 + 1 and y0 + 2, y0 + 3
// (4 floats per row, at wa, wa + 4, wa + 16, wa + 20), in the tall layout
// those of columns x0, x0 + 1 and x0 + 2, x0 + 3 (2 floats per row, at tb and
// tb + 8), and four 16-byte rows of the row-major image when W is a multiple
// of 4.  Every access is a 16-byte vector and a warp's 32 blocks fill whole
// sectors; no shared memory, no barriers.  Positions as in patch_index.
struct PatchBlock {
    int x0, y0, wa, tb;
    __device__ PatchBlock(int blk, int Wp) {
        const int nbx = Wp >> 2;
        const int by = blk / nbx, bx = blk - by * nbx;
        x0 = bx << 2;
        y0 = by << 2;
        wa = ((by * (Wp >> 3) + (bx >> 1)) << 5) + ((bx & 1) << 3);
        tb = (((by >> 1) * (Wp >> 2) + bx) << 5) + ((by & 1) << 4);
    }
    // the block's rows r = 0..3 in the wide layout, and the tall layout's
    // float4 k = 0..3 (columns x0, x0 + 1 of rows 2k', 2k' + 1 for k = k',
    // columns x0 + 2, x0 + 3 for k = 2 + k')
    __device__ int wide(int r) const { return wa + ((r >> 1) << 4) + ((r & 1) << 2); }
    __device__ int tall(int k) const { return tb + (k << 2); }
};

__device__ __forceinline__ float4 ld4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float comp(const float4& v, int i) {
    return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}

// Row r of a 4 x 4 block from its two tall sectors (float4 t[0..3] as loaded
// at tall(0..3)): columns 0, 1 from t[r >> 1], columns 2, 3 from t[2 + (r >> 1)].
__device__ __forceinline__ float4 tall_row(const float4* t, int r) {
    const float4& a = t[r >> 1];
    const float4& b = t[2 + (r >> 1)];
    return (r & 1) ? make_float4(a.z, a.w, b.z, b.w) : make_float4(a.x, a.y, b.x, b.y);
}

// Rows r of a 4 x 4 block of the row-major H x W image (0 outside it):
// 16-byte loads when the block lies inside and W is a multiple of 4.
__device__ __forceinline__ void load_rows(const float* img, int H, int W, const PatchBlock& pb, bool vec,
                                          float4* row) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const int y = pb.y0 + r;
        if (vec) {
            row[r] = ld4(img + (size_t)y * W + pb.x0);
        } else {
            float v[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int x = pb.x0 + c;
                v[c] = (y < H && x < W) ? img[(size_t)y * W + x] : 0.f;
            }
            row[r] = make_float4(v[0], v[1], v[2], v[3]);
        }
    }
}

// Writes rows of the block to both patch layouts.
__device__ __forceinline__ void store_patches(float* xA, float* xB, const PatchBlock& pb, const float4* row) {
#pragma unroll
    for (int r = 0; r < 4; ++r) st4(xA + pb.wide(r), row[r]);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float4& a = row[2 * k];
        const float4& b = row[2 * k + 1];
        st4(xB + pb.tall(k), make_float4(a.x, a.y, b.x, b.y));       // columns 0, 1
        st4(xB + pb.tall(2 + k), make_float4(a.z, a.w, b.z, b.w));   // columns 2, 3
    }
}

// The same box step with both accumulators in the patch numbering
// (patch_index), both read and cleared per 4 x 4 block; with xA / xB set,
// the new x is also written in both patch layouts.  The sweep epilogue needs
// only the row pass's proximity partials and the right-hand-side state, which
// this kernel does not touch, so the last CTA runs it beside the others.
__global__ void __launch_bounds__(128) k_finalize_patch(const FinalizeArgs a) {
    if (blockIdx.x == gridDim.x - 1) {
        sweep_epilogue(a.epi);
        return;
    }
    const int H = a.imgH, W = a.imgW, Wp = a.imgWp;
    const int nblk = (Wp >> 2) * (((H + 7) & ~7) >> 2);
    const bool wvec = (W & 3) == 0;
    const int stride = (gridDim.x - 1) * blockDim.x;
    for (int blk = blockIdx.x * blockDim.x + threadIdx.x; blk < nblk; blk += stride) {
        const PatchBlock pb(blk, Wp);
        const bool vec = wvec && pb.x0 + 3 < W && pb.y0 + 3 < H;
        float4 dA[4], dB[4], xr[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) dA[r] = ld4(a.delta + pb.wide(r));
#pragma unroll
        for (int k = 0; k < 4; ++k) dB[k] = ld4(a.deltaT + pb.tall(k));
        load_rows(a.x, H, W, pb, vec, xr);
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int r = 0; r < 4; ++r) st4(a.delta + pb.wide(r), z4);
#pragma unroll
        for (int k = 0; k < 4; ++k) st4(a.deltaT + pb.tall(k), z4);
        float4 xn[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int y = pb.y0 + r;
            const float4 t = tall_row(dB, r);
            float o[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int x = pb.x0 + c;
                o[c] = 0.f;
                if (y < H && x < W) {
                    const size_t j = (size_t)y * W + x;
                    float d = comp(dA[r], c) + comp(t, c);
                    if (a.zc) d *= a.zc[j];
                    const size_t bj = (a.box_len == 1) ? 0 : j;
                    o[c] = clampf(comp(xr[r], c) + d, a.lo[bj], a.hi[bj]);
                    if (!vec) a.x[j] = o[c];
                }
            }
            xn[r] = make_float4(o[0], o[1], o[2], o[3]);
            if (vec) st4(a.x + (size_t)y * W + pb.x0, xn[r]);
        }
        if (a.xA) store_patches(a.xA, a.xB, pb, xn);
    }
}

// x (row-major H x W) copied into the wide and the tall patch layouts: the
// gathers of the one-pass row pass in the patch numbering.  Padding reads 0.
__global__ void __launch_bounds__(128) k_patch_image(const float* x, float* xA, float* xB, int H, int W,
                                                     int Wp) {
    const int nblk = (Wp >> 2) * (((H + 7) & ~7) >> 2);
    const bool wvec = (W & 3) == 0;
    for (int blk = blockIdx.x * blockDim.x + threadIdx.x; blk < nblk; blk += gridDim.x * blockDim.x) {
        const PatchBlock pb(blk, Wp);
        float4 xr[4];
        load_rows(x, H, W, pb, wvec && pb.x0 + 3 < W && pb.y0 + 3 < H, xr);
        store_patches(xA, xB, pb, xr);
    }
}

// The packed column indices of every row rewritten to its patch position,
// in place: tall patches for the rows marked in rowT, wide ones for the
// others (one warp per packed row; padding entries untouched).
__global__ void k_patch_cols(const int2* rinfo, const unsigned char* rowT, int m, unsigned long long recipW,
                             int W, int Wp, int* col) {
    const int lane = threadIdx.x & 31;
    const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
    for (long long i = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < m; i += nw) {
        const int2 ri = rinfo[i];
        const bool tall = rowT[i] != 0;
        for (int e = lane; e < ri.y; e += 32) col[ri.x + e] = patch_index(col[ri.x + e], recipW, W, Wp, tall);
    }
}

// xT <- x column-major (H x W image, one right-hand side): the copy that the
// two-pass row pass gathers from for the rows running down the image.  Tiles
// of 32 image rows x 8 columns as in k_finalize_tr, one pixel per thread.
__global__ void __launch_bounds__(256) k_transpose_image(const float* x, float* xT, int H, int W) {
    __shared__ float t[kTrCols][kTrRows + 1];
    const int tw = (W + kTrCols - 1) / kTrCols;
    const long long ntiles = (long long)tw * ((H + kTrRows - 1) / kTrRows);
    const int tx = threadIdx.x % kTrRows, ty = threadIdx.x / kTrRows;
    const int ix = threadIdx.x % kTrCols, iy = threadIdx.x / kTrCols;
    for (long long ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
        const int r0 = (int)(ti / tw) * kTrRows, c0 = (int)(ti % tw) * kTrCols;
        const int r = r0 + iy, c = c0 + ix;
        t[ix][iy] = (r < H && c < W) ? x[(long long)r * W + c] : 0.f;
        __syncthreads();
        const int cT = c0 + ty, rT = r0 + tx;
        if (cT < W && rT < H) xT[(long long)cT * H + rT] = t[ty][tx];
        __syncthreads();
    }
}

// The column indices of the rows marked in rowT rewritten to column-major
// pixel indices, in place (one warp per packed row; the rest untouched).
__global__ void k_transposed_cols(const int2* rinfo, const unsigned char* rowT, int m,
                                  unsigned long long recipW, int W, int H, int* col) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < m; i += warps) {
        if (!rowT[i]) continue;
        const int2 ri = rinfo[i];
        for (int e = lane; e < ri.y; e += 32) col[ri.x + e] = transposed_index(col[ri.x + e], recipW, W, H);
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
using ColFn = void (*)(ColArgs);

template <typename VT, int G, int MAXE>
SweepFn pick_scat(int scat) {
    if (scat == 0) return k_sweep<VT, G, MAXE, 0>;
    if (scat == 1) return k_sweep<VT, G, MAXE, 1>;
    return k_sweep<VT, G, MAXE, 2>;
}

template <typename VT>
SweepFn pick_sweep(int G, int maxe, int scat) {
    if (G == 32 && maxe == 16) return pick_scat<VT, 32, 16>(scat);
    if (G == 32 && maxe == 8) return pick_scat<VT, 32, 8>(scat);
    if (G == 16 && maxe == 16) return pick_scat<VT, 16, 16>(scat);
    if (G == 16 && maxe == 8) return pick_scat<VT, 16, 8>(scat);
    if (G == 8 && maxe == 16) return pick_scat<VT, 8, 16>(scat);
    if (G == 8 && maxe == 8) return pick_scat<VT, 8, 8>(scat);
    if (G == 4 && maxe == 8) return pick_scat<VT, 4, 8>(scat);
    return nullptr;
}

template <typename VT>
SweepFn pick_batched(int B, int scat) {
    const bool one = scat != 0;
    switch (B) {
        case 4: return one ? k_sweep_batched<VT, 1, 1> : k_sweep_batched<VT, 1, 0>;
        case 8: return one ? k_sweep_batched<VT, 2, 1> : k_sweep_batched<VT, 2, 0>;
        case 16: return one ? k_sweep_batched<VT, 4, 1> : k_sweep_batched<VT, 4, 0>;
        case 32: return one ? k_sweep_batched<VT, 8, 1> : k_sweep_batched<VT, 8, 0>;
        default: return nullptr;
    }
}

template <typename VT>
ColFn pick_col(int G, int B) {
    if (B > 1) {
        switch (B) {
            case 4: return k_colpass_batched<VT, 1>;
            case 8: return k_colpass_batched<VT, 2>;
            case 16: return k_colpass_batched<VT, 4>;
            case 32: return k_colpass_batched<VT, 8>;
            default: return nullptr;
        }
    }
    switch (G) {
        case 32: return k_colpass<VT, 32>;
        case 16: return k_colpass<VT, 16>;
        case 8: return k_colpass<VT, 8>;
        case 4: return k_colpass<VT, 4>;
        default: return nullptr;
    }
}

SweepFn sweep_fn(suppy_dtype dt, int G, int maxe, int scat, int B) {
    if (B > 1) {
        if (dt == SUPPY_F32) return pick_batched<float>(B, scat);
        if (dt == SUPPY_BF16) return pick_batched<__nv_bfloat16>(B, scat);
        return pick_batched<__half>(B, scat);
    }
    if (dt == SUPPY_F32) return pick_sweep<float>(G, maxe, scat);
    if (dt == SUPPY_BF16) return pick_sweep<__nv_bfloat16>(G, maxe, scat);
    return pick_sweep<__half>(G, maxe, scat);
}

ColFn col_fn(suppy_dtype dt, int G, int B) {
    if (dt == SUPPY_F32) return pick_col<float>(G, B);
    if (dt == SUPPY_BF16) return pick_col<__nv_bfloat16>(G, B);
    return pick_col<__half>(G, B);
}

// ------------------------------------------------ EL / EMR extrapolation ----
// k_ext_norm: ||delta_b||^2 per right-hand side (FP64 per thread, fixed-order
// sums over lanes, warps and CTAs); the last CTA to finish turns the sweep's
// reductions into the step t_b:
//   EL  t = sum_i w_i d_i^2 / ||a_i||^2 / ||delta||^2   (delta = A^T D d)
//   EMR t = ||delta||^2 / sum_i w_i q_i^2                (delta = A^T M d, q = A delta)
// and 0 when a denominator vanishes or the right-hand side has stopped.
__global__ void __launch_bounds__(256) k_ext_norm(const ExtArgs a) {
    __shared__ double sw[8][32];
    __shared__ bool is_last;
    const long long nB = a.n * a.B;
    const long long tid = (long long)blockIdx.x * 256 + threadIdx.x;
    const long long stride = (long long)gridDim.x * 256;
    const int B = a.B;
    double s = 0.0;
    for (long long e = tid; e < nB; e += stride) {
        const double d = (double)a.delta[e];
        s += d * d;
    }
    for (int o = 16; o >= B && o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane < B) sw[wid][lane] = s;
    __syncthreads();
    if (threadIdx.x < B) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += sw[w][threadIdx.x];
        a.part[(size_t)blockIdx.x * B + threadIdx.x] = t;
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) is_last = (atomicAdd(a.ticket, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    for (int b = wid; b < B; b += 8) {
        double d2 = 0.0, num = 0.0;
        for (int c = lane; c < (int)gridDim.x; c += 32) d2 += __ldcg(a.part + (size_t)c * B + b);
        const double* src = (a.method == SUPPY_EL) ? a.pp : a.qq;
        const int ns = (a.method == SUPPY_EL) ? a.npp : a.nqq;
        for (int c = lane; c < ns; c += 32) num += __ldcg(src + (size_t)c * B + b);
        d2 = warp_sum(d2);
        num = warp_sum(num);
        if (lane == 0) {
            double t = 0.0;
            if (!a.st[b].stopped) {
                if (a.method == SUPPY_EL && d2 > 0.0) t = num / d2;
                if (a.method == SUPPY_EMR && num > 0.0) t = d2 / num;
            }
            a.tstep[b] = t;
        }
    }
    if (threadIdx.x == 0) *a.ticket = 0u;
}

// x <- box(x + lambda t_b delta), delta <- 0 (the box also when t_b = 0: the
// perturbation may have left x outside it).
__global__ void __launch_bounds__(256) k_ext_apply(const ExtArgs a) {
    const long long nB = a.n * a.B;
    for (long long e = (long long)blockIdx.x * 256 + threadIdx.x; e < nB;
         e += (long long)gridDim.x * 256) {
        const int b = (int)(e % a.B);
        const long long j = e / a.B;
        const float t = a.lam * (float)a.tstep[b];
        const long long bj = (a.box_len == 1) ? 0 : j;
        const float d = a.delta[e];
        a.x[e] = clampf(a.x[e] + t * d, a.lo[bj], a.hi[bj]);
        a.delta[e] = 0.f;
    }
}

}  // namespace

cudaError_t launch_sweep(const SweepArgs& a, suppy_dtype dt, int G, int maxe, int scat, int grid,
                         cudaStream_t s) {
    SweepFn f = sweep_fn(dt, G, maxe, scat, 1);
    if (!f) return cudaErrorInvalidValue;
    size_t smem = 0;
    if (scat == 2) {
        smem = sizeof(float) * (size_t)a.n;
        cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    f<<<grid, kSweepThreads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_sweep_batched(const SweepArgs& a, suppy_dtype dt, int scat, int grid,
                                 cudaStream_t s) {
    SweepFn f = sweep_fn(dt, 32, 0, scat, a.B);
    if (!f) return cudaErrorInvalidValue;
    f<<<grid, kSweepThreads, 0, s>>>(a);
    return cudaGetLastError();
}

int sweep_blocks_per_sm(suppy_dtype dt, int G, int maxe, int scat, int B, int n) {
    SweepFn f = sweep_fn(dt, G, maxe, scat, B);
    if (!f) return 0;
    size_t smem = 0;
    if (scat == 2 && B == 1) {
        smem = sizeof(float) * (size_t)n;
        if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return 0;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, kSweepThreads, smem) != cudaSuccess)
        return 0;
    return nb;
}

cudaError_t launch_colpass(const ColArgs& a, suppy_dtype dt, int G, int grid, cudaStream_t s) {
    ColFn f = col_fn(dt, G, a.B);
    if (!f) return cudaErrorInvalidValue;
    f<<<grid, kSweepThreads, 0, s>>>(a);
    return cudaGetLastError();
}

int colpass_blocks_per_sm(suppy_dtype dt, int G, int B) {
    ColFn f = col_fn(dt, G, B);
    if (!f) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, kSweepThreads, 0) != cudaSuccess)
        return 0;
    return nb;
}

cudaError_t launch_epilogue(const EpiArgs& a, cudaStream_t s) {
    k_epilogue<<<1, kFinalizeThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const FinalizeArgs& a, int grid, cudaStream_t s) {
    if (a.deltaT && a.patch) {
        if (a.B != 1 || a.imgW < 1 || a.imgH < 1 || (long long)a.imgW * a.imgH != a.nB ||
            a.imgWp < a.imgW || (a.imgWp & 7) != 0)
            return cudaErrorInvalidValue;
        const long long blocks = (long long)(a.imgWp >> 2) * (((a.imgH + 7) & ~7) >> 2);
        // the pixel blocks' CTAs, then one for the epilogue
        k_finalize_patch<<<(int)std::min<long long>((blocks + 127) / 128, 152 * 16) + 1, 128, 0, s>>>(a);
        return cudaGetLastError();
    }
    if (a.deltaT) {
        if (a.B != 1 || a.imgW < 1 || a.imgH < 1 || (long long)a.imgW * a.imgH != a.nB)
            return cudaErrorInvalidValue;
        const long long tiles = (long long)((a.imgW + kTrCols - 1) / kTrCols) *
                                ((a.imgH + kTrRows - 1) / kTrRows);
        k_finalize_tr<<<(int)std::min<long long>(tiles, 4096), 256, 0, s>>>(a);
        return cudaGetLastError();
    }
    k_finalize<<<grid, kFinalizeThreads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_patch_image(const float* x, float* xA, float* xB, int H, int W, int Wp, cudaStream_t s) {
    if (H < 1 || W < 1 || Wp < W || (Wp & 7) != 0) return cudaErrorInvalidValue;
    const long long blocks = (long long)(Wp >> 2) * (((H + 7) & ~7) >> 2);
    k_patch_image<<<(int)std::min<long long>((blocks + 127) / 128, 152 * 16), 128, 0, s>>>(x, xA, xB, H, W,
                                                                                          Wp);
    return cudaGetLastError();
}

cudaError_t launch_patch_cols(const int2* rinfo, const unsigned char* rowT, int m, unsigned long long recipW,
                              int W, int Wp, int* col, cudaStream_t s) {
    if (m < 1) return cudaSuccess;
    if (W < 1 || Wp < W || (Wp & 7) != 0) return cudaErrorInvalidValue;
    const int grid = (int)std::min<long long>(((long long)m * 32 + 255) / 256, 152 * 16);
    k_patch_cols<<<grid, 256, 0, s>>>(rinfo, rowT, m, recipW, W, Wp, col);
    return cudaGetLastError();
}

cudaError_t launch_transpose_image(const float* x, float* xT, int H, int W, cudaStream_t s) {
    if (H < 1 || W < 1) return cudaErrorInvalidValue;
    const long long tiles = (long long)((W + kTrCols - 1) / kTrCols) * ((H + kTrRows - 1) / kTrRows);
    k_transpose_image<<<(int)std::min<long long>(tiles, 4096), 256, 0, s>>>(x, xT, H, W);
    return cudaGetLastError();
}

cudaError_t launch_transposed_cols(const int2* rinfo, const unsigned char* rowT, int m,
                                   unsigned long long recipW, int W, int H, int* col, cudaStream_t s) {
    if (m < 1) return cudaSuccess;
    const int grid = (int)std::min<long long>(((long long)m * 32 + 255) / 256, 152 * 16);
    k_transposed_cols<<<grid, 256, 0, s>>>(rinfo, rowT, m, recipW, W, H, col);
    return cudaGetLastError();
}

cudaError_t launch_reduce_pp(const double* pp, int npp, int B, double scale, int accumulate,
                             double* out, cudaStream_t s) {
    k_reduce_pp<<<1, 256, 0, s>>>(pp, npp, B, scale, accumulate, out);
    return cudaGetLastError();
}

cudaError_t launch_ext_step(const ExtArgs& a, int grid, cudaStream_t s) {
    k_ext_norm<<<grid, 256, 0, s>>>(a);
    k_ext_apply<<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace suppy
