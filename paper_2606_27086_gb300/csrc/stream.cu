// TMA-fed streaming passes of the simultaneous projection sweep (Sec. 2.1.1,
// Eq. (3)) for one right-hand side.
//
// Each CTA owns a contiguous, nnz-balanced range of items (rows of the CSR
// copy, or columns of the CSC copy of A), hence one contiguous slice of the
// index and value arrays.  One producer lane streams that slice into a
// four-stage shared-memory ring with 1-D bulk copies (cp.async.bulk, L2
// evict-first) tracked by mbarriers; twenty-three consumer warps, split into
// groups of G lanes (one group per item, G chosen from the item lengths), take
// the items round-robin and read them from the ring four elements per 16-byte
// access, so HBM streaming runs ahead of the gathers of x (or of the
// coefficients) instead of waiting behind them.  A consumer warp releases a
// stage once its items there are done; the producer refills a stage when all
// consumer warps released it.
//
//  * row pass: r_i = <a_i, x>, d_i = clamp(r_i, l_i, u_i) - r_i, the
//    proximity term (compensated FP32 per thread, FP64 across threads and
//    CTAs), and either coef_i = lambda w_i d_i / ||a_i||^2 written
//    out (two-pass) or coef_i * a_i scatter-added into delta by address-
//    coalesced L2 reductions (one-pass);
//  * column pass: x_j <- clamp(x_j + sum_i a_ij coef_i, lo_j, hi_j).
//
// Every mbarrier wait is bounded (about two seconds of SM clock); on timeout
// the CTA records an error word, stops, lets its copies in flight land and
// returns.
#include "common.cuh"

namespace suppy {
namespace {

constexpr int kStages = 6;
constexpr long long kWaitCycles = 4000000000LL;
constexpr uint32_t kSuspendNs = 2000;   // a waiting thread sleeps up to this long per try

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(kSuspendNs)
        : "memory");
    return ok != 0;
}

// Bounded wait for the completion of the phase with the given parity.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (*abort) return false;
        if (clock64() - t0 > kWaitCycles) return false;
    }
    return true;
}

__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                         uint64_t pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint "
        "[%0], [%1], %2, [%3], %4;" ::"r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar)), "l"(pol)
        : "memory");
}

template <typename VT>
__device__ __forceinline__ float to_f(VT v) { return (float)v; }

// Ring of the CTA's slice: element g of the slice (counted from the aligned
// start Ea) lies in tile g / T, held by stage (g / T) % kStages at offset
// g % T; groups of four elements starting at a multiple of four never straddle
// a tile and are 16-byte aligned in the ring.
template <typename VT>
struct Ring {
    const VT* val;
    const int* idx;
    int tshift;   // log2(T)
    __device__ __forceinline__ int pos(int g) const {
        const int k = g >> tshift;
        return ((k % kStages) << tshift) | (g & ((1 << tshift) - 1));
    }
};

template <typename VT>
struct Quad;
template <>
struct Quad<float> {
    static __device__ __forceinline__ float4 load(const float* p) {
        return *reinterpret_cast<const float4*>(p);
    }
};
template <>
struct Quad<__nv_bfloat16> {
    static __device__ __forceinline__ float4 load(const __nv_bfloat16* p) {
        const uint2 u = *reinterpret_cast<const uint2*>(p);
        return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u),
                           __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xffff0000u));
    }
};
template <>
struct Quad<__half> {
    static __device__ __forceinline__ float4 load(const __half* p) {
        const uint2 u = *reinterpret_cast<const uint2*>(p);
        const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&u.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&u.y));
        return make_float4(a.x, a.y, b.x, b.y);
    }
};

template <int G>
__device__ __forceinline__ unsigned gmask_of(int lane) {
    if constexpr (G == 32) return 0xffffffffu;
    else return ((1u << G) - 1u) << (lane & ~(G - 1));
}

// sum_e a_e * vec[idx_e] over the item's elements held in the ring, by the
// G lanes of one group reading four elements per 16-byte ring access.
template <typename VT, int G>
__device__ __forceinline__ float ring_dot(const Ring<VT>& r, int g0, int len, int gl,
                                          const float* __restrict__ vec) {
    constexpr int U = 4;
    const int q0 = g0 >> 2, q1 = (g0 + len + 3) >> 2;
    const int e_hi = g0 + len;
    float acc = 0.f;
    for (int qb = q0 + gl; qb < q1; qb += G * U) {
        float4 v[U];
        int4 c[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int q = qb + u * G;
            const int e = q << 2;
            if (q < q1) {
                const int pos = r.pos(e);
                v[u] = Quad<VT>::load(r.val + pos);
                c[u] = *reinterpret_cast<const int4*>(r.idx + pos);
                // mask the neighbours' elements that share the first / last quad
                if (e < g0 || e >= e_hi) { v[u].x = 0.f; c[u].x = 0; }
                if (e + 1 < g0 || e + 1 >= e_hi) { v[u].y = 0.f; c[u].y = 0; }
                if (e + 2 < g0 || e + 2 >= e_hi) { v[u].z = 0.f; c[u].z = 0; }
                if (e + 3 >= e_hi) { v[u].w = 0.f; c[u].w = 0; }
            } else {
                v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                c[u] = make_int4(0, 0, 0, 0);
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            acc = fmaf(v[u].x, __ldg(vec + c[u].x), acc);
            acc = fmaf(v[u].y, __ldg(vec + c[u].y), acc);
            acc = fmaf(v[u].z, __ldg(vec + c[u].z), acc);
            acc = fmaf(v[u].w, __ldg(vec + c[u].w), acc);
        }
    }
    return acc;
}

// Producer / consumer skeleton.  Consumer warps hold 32/G groups of G lanes;
// in each round the groups of a warp take consecutive items, so a warp's
// items cover a contiguous element range.  work(item, len, g0, ring, gl)
// returns the FP64 proximity contribution of the item (one lane), else 0;
// work.prefetch(next item or -1) loads the next round's per-item operands and
// work.advance() makes them current.
template <typename VT, int G, class Work>
__device__ double stream_items(const StreamArgs& a, Work& work) {
    extern __shared__ __align__(128) unsigned char smraw[];
    __shared__ volatile int abort_flag;
    const int T = a.tile;
    const int RING = kStages * T;
    VT* sval = reinterpret_cast<VT*>(smraw);
    int* sidx = reinterpret_cast<int*>(smraw + (size_t)RING * sizeof(VT));
    uint64_t* full = reinterpret_cast<uint64_t*>(sidx + RING);
    uint64_t* empty = full + kStages;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int NW = kStreamThreads / 32 - 1;
    constexpr int GPW = 32 / G;
    const int I0 = a.cta_items[blockIdx.x], I1 = a.cta_items[blockIdx.x + 1];
    double acc = 0.0;
    if (I0 >= I1) return 0.0;   // uniform over the CTA
    const long long E0 = a.info[I0].x;
    const long long E1 = (long long)a.info[I1 - 1].x + a.info[I1 - 1].y;
    const long long Ea = E0 & ~7LL;
    const int K = (int)((E1 - Ea + T - 1) / T);
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], NW);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const VT* gval = static_cast<const VT*>(a.val);
    if (warp == 0) {
        if (lane == 0) {
            const uint64_t pol = policy_evict_first();
            const uint32_t bytes_v = (uint32_t)(T * sizeof(VT)), bytes_i = (uint32_t)(T * 4);
            int issued = 0;
            for (int k = 0; k < K; ++k) {
                const int s = k % kStages;
                if (k >= kStages && !mbar_wait(&empty[s], ((k / kStages) - 1) & 1, &abort_flag)) {
                    abort_flag = 1;
                    atomicExch(a.err, 1);
                    break;
                }
                mbar_arrive_expect_tx(&full[s], bytes_v + bytes_i);
                bulk_g2s(sval + (size_t)s * T, gval + Ea + (long long)k * T, bytes_v, &full[s], pol);
                bulk_g2s(sidx + (size_t)s * T, a.idx + Ea + (long long)k * T, bytes_i, &full[s], pol);
                issued = k + 1;
            }
            if (abort_flag) {
                // let the copies in flight land before the CTA leaves
                volatile int never = 0;
                for (int k = (issued > kStages ? issued - kStages : 0); k < issued; ++k)
                    mbar_wait(&full[k % kStages], (k / kStages) & 1, &never);
            }
        }
    } else {
        const Ring<VT> ring{sval, sidx, 31 - __clz(T)};
        const int gw = lane / G, gl = lane % G;
        int next_rel = 0;
        bool ok = true;
        auto wait_tile = [&](int k) {
            return mbar_wait(&full[k % kStages], (k / kStages) & 1, &abort_flag);
        };
        auto release_upto = [&](int kend) {
            for (; ok && next_rel < kend; ++next_rel) {
                if (!__all_sync(0xffffffffu, wait_tile(next_rel))) {
                    ok = false;
                    break;
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty[next_rel % kStages]);
            }
        };
        constexpr int BIG = 0x7fffffff;
        // the next round's item descriptor is loaded while this round runs
        int base = I0 + (warp - 1) * GPW;
        int2 nxt = make_int2(0, 0);
        if (base + gw < I1) nxt = a.info[base + gw];
        for (; ok && base < I1; base += NW * GPW) {
            const int i = base + gw;
            const int2 inf = nxt;
            const int inext = i + NW * GPW;
            nxt = (inext < I1) ? a.info[inext] : make_int2(0, 0);
            work.prefetch(inext < I1 ? inext : -1);
            const int g0 = (int)((long long)inf.x - Ea);
            int kb = BIG, ke = -1;
            if (inf.y > 0) {
                kb = g0 / T;
                ke = (g0 + inf.y - 1) / T;
            }
            kb = __reduce_min_sync(0xffffffffu, kb);
            ke = __reduce_max_sync(0xffffffffu, ke);
            if (ke < 0) {
                work.advance();
                continue;   // no data needed by this warp in this round
            }
            release_upto(kb);
            for (int k = max(kb, next_rel); ok && k <= ke; ++k)
                ok = __all_sync(0xffffffffu, wait_tile(k));
            if (!ok) break;
            if (i < I1 && inf.y > 0) acc += work(i, inf.y, g0, ring, gl);
            work.advance();
        }
        if (ok) release_upto(K);
        if (!ok) {
            abort_flag = 1;
            if (lane == 0) atomicExch(a.err, 1);
        }
    }
    return acc;
}

__device__ __forceinline__ void cta_sum_to(double v, double* out) {
    v = warp_sum(v);
    __shared__ double sw[kStreamThreads / 32];
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < kStreamThreads / 32; ++w) s += sw[w];
        *out = s;
    }
}

// Row pass.  SCAT 0: coefficients written to a.coef (when set); 1: scatter.
template <typename VT, int G, int SCAT>
struct RowWork {
    const StreamArgs& a;
    float li = 0.f, ui = 0.f, w = 0.f;      // current round's bounds and weight
    float nl = 0.f, nu = 0.f, nw = 0.f;     // next round's
    // The group leader's proximity terms are summed in FP32 with Kahan
    // compensation (error independent of the term count) and widened to FP64
    // for the CTA and grid reductions: FP64 arithmetic is scarce on GB300 and
    // a warp-wide FP64 add per row would cost more than the row's gathers.
    float ps = 0.f, pc = 0.f;
    __device__ void kahan_add(float v) {
        const float y = v - pc;
        const float t = ps + y;
        pc = (t - ps) - y;
        ps = t;
    }
    __device__ double total() const { return (double)ps - (double)pc; }
    __device__ void prefetch(int i) {
        if (i >= 0) {
            nl = __ldg(a.l + i);
            nu = __ldg(a.u + i);
            nw = __ldg(a.wr + i);
        }
    }
    __device__ void advance() {
        li = nl;
        ui = nu;
        w = nw;
    }
    __device__ double operator()(int i, int len, int g0, const Ring<VT>& r, int gl) {
        const unsigned gm = gmask_of<G>(threadIdx.x & 31);
        float dot = ring_dot<VT, G>(r, g0, len, gl, a.x);
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) dot += __shfl_xor_sync(gm, dot, o);
        const float d = clampf(dot, li, ui) - dot;
        const float coef = a.lam * w * d;
        if (SCAT == 0) {
            if (a.coef && gl == 0) a.coef[i] = coef;
        } else if (coef != 0.f) {
            // lane-strided over the elements: consecutive lanes, consecutive columns
            for (int t = gl; t < len; t += G) {
                const int p = r.pos(g0 + t);
                atomicAdd(a.delta + r.idx[p], coef * to_f(r.val[p]));
            }
        }
        if (gl == 0) kahan_add(d * d * w);
        return 0.0;
    }
};

template <typename VT, int G, int SCAT>
__global__ void __launch_bounds__(kStreamThreads, 1) k_rows_tma(const StreamArgs a) {
    if (a.check_stop && a.st[0].stopped) return;
    RowWork<VT, G, SCAT> work{a};
    // the first round's operands
    {
        const int I0 = a.cta_items[blockIdx.x], I1 = a.cta_items[blockIdx.x + 1];
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const int i = I0 + (warp - 1) * (32 / G) + lane / G;
        work.prefetch(warp > 0 && i < I1 ? i : -1);
        work.advance();
    }
    stream_items<VT, G>(a, work);
    cta_sum_to(work.total(), a.pp + blockIdx.x);
}

// Column pass of the two-pass sweep (B = 1).
template <typename VT, int G>
struct ColWork {
    const StreamArgs& a;
    float xj = 0.f, lo = 0.f, hi = 0.f;
    float nx = 0.f, nlo = 0.f, nhi = 0.f;
    __device__ void prefetch(int j) {
        if (j >= 0) {
            const int bj = (a.box_len == 1) ? 0 : j;
            nx = a.xw[j];   // owned by this group alone during the pass
            nlo = __ldg(a.lo + bj);
            nhi = __ldg(a.hi + bj);
        }
    }
    __device__ void advance() {
        xj = nx;
        lo = nlo;
        hi = nhi;
    }
    __device__ double operator()(int j, int len, int g0, const Ring<VT>& r, int gl) {
        const unsigned gm = gmask_of<G>(threadIdx.x & 31);
        float s = ring_dot<VT, G>(r, g0, len, gl, a.coef_in);
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(gm, s, o);
        if (gl == 0) a.xw[j] = clampf(xj + s, lo, hi);
        return 0.0;
    }
};

template <typename VT, int G>
__global__ void __launch_bounds__(kStreamThreads, 1) k_cols_tma(const StreamArgs a) {
    if (a.epi.st[0].stopped) return;   // the row pass left no coefficients
    ColWork<VT, G> work{a};
    {
        const int I0 = a.cta_items[blockIdx.x], I1 = a.cta_items[blockIdx.x + 1];
        const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const int j = I0 + (warp - 1) * (32 / G) + lane / G;
        work.prefetch(warp > 0 && j < I1 ? j : -1);
        work.advance();
    }
    stream_items<VT, G>(a, work);
    __syncthreads();
    if (blockIdx.x == 0 && !a.epi.last_seg) {
        // CTA 0 also accumulates the row pass's proximity partials of this
        // block (never for the last block: the stop flag is set by a
        // separate launch)
        const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
        for (int b = wid; b < a.epi.B; b += kStreamThreads / 32) {
            double s = 0.0;
            for (int c = lane; c < a.epi.npp; c += 32) s += a.epi.pp[(size_t)c * a.epi.B + b];
            s = warp_sum(s);
            if (lane == 0 && !a.epi.st[b].stopped) {
                if (a.epi.first_seg) a.epi.st[b].p_acc = 0.0;
                a.epi.st[b].p_acc += a.epi.scale * s;
            }
        }
    }
}

using StreamFn = void (*)(StreamArgs);

template <typename VT>
StreamFn pick_rows(int G, int scat) {
    switch (G) {
        case 4: return scat ? k_rows_tma<VT, 4, 1> : k_rows_tma<VT, 4, 0>;
        case 8: return scat ? k_rows_tma<VT, 8, 1> : k_rows_tma<VT, 8, 0>;
        case 16: return scat ? k_rows_tma<VT, 16, 1> : k_rows_tma<VT, 16, 0>;
        default: return scat ? k_rows_tma<VT, 32, 1> : k_rows_tma<VT, 32, 0>;
    }
}

template <typename VT>
StreamFn pick_cols(int G) {
    switch (G) {
        case 4: return k_cols_tma<VT, 4>;
        case 8: return k_cols_tma<VT, 8>;
        case 16: return k_cols_tma<VT, 16>;
        default: return k_cols_tma<VT, 32>;
    }
}

StreamFn rows_fn(suppy_dtype dt, int G, int scat) {
    if (dt == SUPPY_F32) return pick_rows<float>(G, scat);
    if (dt == SUPPY_BF16) return pick_rows<__nv_bfloat16>(G, scat);
    return pick_rows<__half>(G, scat);
}

StreamFn cols_fn(suppy_dtype dt, int G) {
    if (dt == SUPPY_F32) return pick_cols<float>(G);
    if (dt == SUPPY_BF16) return pick_cols<__nv_bfloat16>(G);
    return pick_cols<__half>(G);
}

}  // namespace

size_t stream_smem_bytes(suppy_dtype dt, int tile) {
    const size_t vsz = (dt == SUPPY_F32) ? 4 : 2;
    return (size_t)kStages * tile * (vsz + 4) + 2 * kStages * sizeof(uint64_t);
}

int stream_max_item(int tile) { return (kStages - 1) * tile; }

static cudaError_t launch_stream(StreamFn f, const StreamArgs& a, suppy_dtype dt, int grid,
                                 cudaStream_t s) {
    const size_t smem = stream_smem_bytes(dt, a.tile);
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    f<<<grid, kStreamThreads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_rows_tma(const StreamArgs& a, suppy_dtype dt, int G, int scat, int grid,
                            cudaStream_t s) {
    return launch_stream(rows_fn(dt, G, scat), a, dt, grid, s);
}

cudaError_t launch_cols_tma(const StreamArgs& a, suppy_dtype dt, int G, int grid, cudaStream_t s) {
    return launch_stream(cols_fn(dt, G), a, dt, grid, s);
}

int stream_blocks_per_sm(suppy_dtype dt, int tile) {
    const size_t smem = stream_smem_bytes(dt, tile);
    StreamFn f = rows_fn(dt, 32, 1);
    if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, kStreamThreads, smem) != cudaSuccess)
        return 0;
    return nb;
}

}  // namespace suppy
