// TMA-fed streaming passes of the simultaneous projection sweep (Sec. 2.1.1,
// Eq. (3)) for one right-hand side.
//
// Each CTA owns a contiguous, nnz-balanced range of items (rows of the CSR
// copy, or columns of the CSC copy of A), hence one contiguous slice of the
// index and value arrays.  One producer lane streams that slice into a
// four-stage shared-memory ring with 1-D bulk copies (cp.async.bulk, L2
// evict-first) tracked by mbarriers; fifteen consumer warps take the items
// round-robin and read them from the ring, so HBM streaming runs ahead of the
// gathers of x (or of the coefficients) from L2 instead of waiting behind
// them.  A consumer releases a stage once every item it owns there is done;
// the producer refills a stage when all consumers released it.
//
//  * row pass: r_i = <a_i, x>, d_i = clamp(r_i, l_i, u_i) - r_i, the FP64
//    proximity term, and either coef_i = lambda w_i d_i / ||a_i||^2 written
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

constexpr int kStages = 4;
constexpr long long kWaitCycles = 4000000000LL;

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
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
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
// start Ea) lives at ring position g & mask.
template <typename VT>
struct Ring {
    const VT* val;
    const int* idx;
    long long ea;   // aligned slice start (global element index)
    int mask;
};

// Producer / consumer skeleton.  work(item, ring, lane) runs in a consumer
// warp for each of its items; returns the FP64 proximity contribution of the
// item (lane 0), zero elsewhere.
template <typename VT, class Work>
__device__ double stream_items(const StreamArgs& a, Work work) {
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
        const Ring<VT> ring{sval, sidx, Ea, RING - 1};
        int next_rel = 0;
        bool ok = true;
        auto wait_tile = [&](int k) { return mbar_wait(&full[k % kStages], (k / kStages) & 1, &abort_flag); };
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
        for (int i = I0 + (warp - 1); ok && i < I1; i += NW) {
            const int2 inf = a.info[i];
            if (inf.y == 0) continue;   // an empty item needs no data (and contributes nothing)
            const long long g0 = (long long)inf.x - Ea;
            const int k0 = (int)(g0 / T);
            const int k1 = (int)((g0 + (inf.y > 0 ? inf.y - 1 : 0)) / T);
            release_upto(k0);
            for (int k = max(k0, next_rel); ok && k <= k1; ++k)
                ok = __all_sync(0xffffffffu, wait_tile(k));
            if (!ok) break;
            acc += work(i, inf.y, g0, ring, lane);
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
template <typename VT, int SCAT>
__global__ void __launch_bounds__(kStreamThreads, 1) k_rows_tma(const StreamArgs a) {
    if (a.check_stop && a.st[0].stopped) return;
    const float* __restrict__ x = a.x;
    auto work = [&](int i, int len, long long g0, const Ring<VT>& r, int lane) -> double {
        constexpr int U = 8;
        float dot = 0.f;
        for (int t0 = lane; t0 < len; t0 += 32 * U) {
            float v[U];
            int c[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int t = t0 + 32 * u;
                const int p = (int)((g0 + t) & r.mask);
                v[u] = (t < len) ? to_f(r.val[p]) : 0.f;
                c[u] = (t < len) ? r.idx[p] : 0;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) dot = fmaf(v[u], __ldg(x + c[u]), dot);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
        const float d = clampf(dot, a.l[i], a.u[i]) - dot;
        const float w = a.wr[i];
        const float coef = a.lam * w * d;
        if (SCAT == 0) {
            if (a.coef && lane == 0) a.coef[i] = coef;
        } else if (coef != 0.f) {
            for (int t = lane; t < len; t += 32) {
                const int p = (int)((g0 + t) & r.mask);
                atomicAdd(a.delta + r.idx[p], coef * to_f(r.val[p]));
            }
        }
        return lane == 0 ? (double)d * (double)d * (double)w : 0.0;
    };
    const double prox = stream_items<VT>(a, work);
    cta_sum_to(prox, a.pp + blockIdx.x);
}

// Column pass of the two-pass sweep (B = 1).
template <typename VT>
__global__ void __launch_bounds__(kStreamThreads, 1) k_cols_tma(const StreamArgs a) {
    if (a.epi.st[0].stopped) return;   // the row pass left no coefficients
    const float* __restrict__ coef = a.coef_in;
    auto work = [&](int j, int len, long long g0, const Ring<VT>& r, int lane) -> double {
        constexpr int U = 8;
        float s = 0.f;
        for (int t0 = lane; t0 < len; t0 += 32 * U) {
            float v[U];
            int c[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int t = t0 + 32 * u;
                const int p = (int)((g0 + t) & r.mask);
                v[u] = (t < len) ? to_f(r.val[p]) : 0.f;
                c[u] = (t < len) ? r.idx[p] : 0;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) s = fmaf(v[u], __ldg(coef + c[u]), s);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0 && len > 0) {
            const int bj = (a.box_len == 1) ? 0 : j;
            a.xw[j] = clampf(a.xw[j] + s, a.lo[bj], a.hi[bj]);
        }
        return 0.0;
    };
    stream_items<VT>(a, work);
    __syncthreads();
    if (blockIdx.x == 0 && !a.epi.last_seg) {
        // CTA 0 also reduces the row pass's proximity partials (never the
        // last block: the stop flag is set by a separate launch)
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
StreamFn pick_rows(int scat) {
    return scat ? k_rows_tma<VT, 1> : k_rows_tma<VT, 0>;
}

StreamFn rows_fn(suppy_dtype dt, int scat) {
    if (dt == SUPPY_F32) return pick_rows<float>(scat);
    if (dt == SUPPY_BF16) return pick_rows<__nv_bfloat16>(scat);
    return pick_rows<__half>(scat);
}

StreamFn cols_fn(suppy_dtype dt) {
    if (dt == SUPPY_F32) return k_cols_tma<float>;
    if (dt == SUPPY_BF16) return k_cols_tma<__nv_bfloat16>;
    return k_cols_tma<__half>;
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

cudaError_t launch_rows_tma(const StreamArgs& a, suppy_dtype dt, int scat, int grid,
                            cudaStream_t s) {
    return launch_stream(rows_fn(dt, scat), a, dt, grid, s);
}

cudaError_t launch_cols_tma(const StreamArgs& a, suppy_dtype dt, int grid, cudaStream_t s) {
    return launch_stream(cols_fn(dt), a, dt, grid, s);
}

int stream_blocks_per_sm(suppy_dtype dt, int tile) {
    const size_t smem = stream_smem_bytes(dt, tile);
    StreamFn f = rows_fn(dt, 1);
    if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, kStreamThreads, smem) != cudaSuccess)
        return 0;
    return nb;
}

}  // namespace suppy
