// Tiled one-pass simultaneous projection sweep (Sec. 2.1.1, Eq. (3); the
// box projection after each sweep or block, Sec. 2.3.3), one right-hand side.
//
// The unknowns are split into P tiles (rectangles of the image for imaging
// problems, column ranges otherwise), one per CTA of one cooperative launch;
// a CTA keeps its tile's x and correction Delta in shared memory for the
// whole sweep.  Every row a_i is cut into segments, runs of its consecutive
// entries that fall in one tile, and each tile's segments are stored as one
// contiguous byte stream (values, then 16-bit tile-local column indices),
// grouped into chunks of consecutive rows.  A CTA streams its tile's bytes
// once per sweep into a shared-memory ring with bulk asynchronous copies, so
// A crosses HBM once; the gathers of x and the scatter into Delta never leave
// the SM.
//
// Per chunk k:
//   phase 1 (dot products): the partial <a_i, x> of every segment from the
//     tile's x, added to r_i (one FP32 L2 reduction per segment), then the
//     chunk's counter is raised (release);
//   phase 2 (corrections), once the counter says every CTA finished phase 1
//     of chunk k (acquire): c_i = lambda w_i (clamp(r_i, l_i, u_i) - r_i) / ||a_i||^2
//     from the complete r_i, and Delta_j += c_i a_ij for the segment's entries
//     (shared-memory compare-and-swap additions, several in flight per lane);
//     the proximity term of row i is added by the segment that holds the
//     row's first entry (FP64).
// Phase 1 runs ahead of phase 2 by as many chunks as the ring holds, so the
// cross-CTA dependency is a rolling one, not a grid barrier.  At the end of
// a block (the whole sweep for Cimmino and DROP) x_j <- box(x_j + z_j Delta_j)
// on the tile, and the next block's dot products use the new x.
//
// r_i lives in two buffers used on alternate sweeps (an epoch word): a sweep
// accumulates into one and clears the other.  The last CTA to finish runs the
// sweep epilogue (fixed-order proximity sum, stopping rule), resets the chunk
// counters and advances the epoch, so every launch finds the synchronisation
// words as it needs them, after a timeout too.  Every wait is bounded (the
// launch's cycle budget); on timeout the warp records the error word, stops
// working, and every CTA still reaches the end of the launch.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "common.cuh"
#include "tma.cuh"

namespace suppy {

#ifdef SUPPY_TILE_STATS
// Measurement build only: cycles per warp role, summed over the CTAs' warps
// (0/1 phase-1 waits / total, 2/3 coefficient waits / total, 4/5 scatter
// waits / total, 6/7 producer waits / total, 8/9 watcher idle polls / total).
__device__ unsigned long long g_tile_stats[16];
#define TSTAT_CLOCK() clock64()
#define TSTAT_ADD(k, v) atomicAdd(&g_tile_stats[k], (unsigned long long)(v))
#else
#define TSTAT_CLOCK() 0LL
#define TSTAT_ADD(k, v) ((void)0)
#endif

namespace {

constexpr long long kTileDrainCycles = 4000000000LL;

template <typename VT>
__device__ __forceinline__ float to_float(VT v);
template <>
__device__ __forceinline__ float to_float<float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_float<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <>
__device__ __forceinline__ float to_float<__half>(__half v) { return __half2float(v); }

__device__ __forceinline__ void red_add_gpu(float* p, float v) {
    asm volatile("red.relaxed.gpu.global.add.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}

__device__ __forceinline__ void red_release_add_gpu(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ float ld_relaxed_gpu(const float* p) {
    float v;
    asm volatile("ld.relaxed.gpu.global.f32 %0, [%1];" : "=f"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void named_sync(int id, int threads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

// Ring position of stream byte p, given the chunk's ring position rc and an
// offset within the chunk (both below the ring size).
__device__ __forceinline__ int wrap(int p, int ring) { return p >= ring ? p - ring : p; }

// Entries a lane adds to Delta per batch of the scatter.
constexpr int kCasBatch = 4;

// Delta_j += c a_ij for the entries e, e + G, ..., e + (kCasBatch - 1) G of a
// segment (those below len): FP32 additions into shared memory made atomic by
// compare-and-swap.  A lane reads its entries' current sums, issues all of its
// compare-and-swaps back to back, and retries only those another lane changed
// in between (rare: entries of one segment are distinct columns).  The
// library's float atomicAdd on shared memory is a compare-and-swap loop per
// element, whose round trips a lane would wait out one after another.
template <typename VT, int G>
__device__ __forceinline__ void scatter_batch(const unsigned char* ring, int RING, int vp, int ip,
                                              int e, int len, float c, float* dt) {
    int j[kCasBatch];
    float add[kCasBatch], old[kCasBatch];
#pragma unroll
    for (int u = 0; u < kCasBatch; ++u) {
        const int eu = e + u * G;
        j[u] = -1;
        add[u] = 0.f;
        if (eu < len) {
            add[u] = c * to_float(*reinterpret_cast<const VT*>(ring + wrap(vp + (int)sizeof(VT) * eu, RING)));
            j[u] = *reinterpret_cast<const unsigned short*>(ring + wrap(ip + 2 * eu, RING));
        }
    }
    volatile float* vd = dt;
#pragma unroll
    for (int u = 0; u < kCasBatch; ++u) old[u] = j[u] >= 0 ? vd[j[u]] : 0.f;
    unsigned pending = 0;
#pragma unroll
    for (int u = 0; u < kCasBatch; ++u) pending |= (j[u] >= 0 ? 1u : 0u) << u;
    while (pending) {
        unsigned prev[kCasBatch];
#pragma unroll
        for (int u = 0; u < kCasBatch; ++u)
            if (pending & (1u << u))
                prev[u] = atomicCAS(reinterpret_cast<unsigned*>(dt) + j[u], __float_as_uint(old[u]),
                                    __float_as_uint(old[u] + add[u]));
#pragma unroll
        for (int u = 0; u < kCasBatch; ++u)
            if (pending & (1u << u)) {
                if (prev[u] == __float_as_uint(old[u])) pending &= ~(1u << u);
                else old[u] = __uint_as_float(prev[u]);
            }
    }
}

__device__ __forceinline__ void st_release_cta(volatile int* p, int v) {
    asm volatile("st.release.cta.shared.u32 [%0], %1;" ::"r"(tma::smem_addr((const void*)p)), "r"(v)
                 : "memory");
}

__device__ __forceinline__ int ld_acquire_cta(const volatile int* p) {
    int v;
    asm volatile("ld.acquire.cta.shared.u32 %0, [%1];" : "=r"(v) : "r"(tma::smem_addr((const void*)p))
                 : "memory");
    return v;
}

__device__ __forceinline__ void red_add_u32_gpu(unsigned* p, unsigned v) {
    asm volatile("red.relaxed.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Bounded spin of every lane of a warp until cond() holds; false (for the
// whole warp) when the CTA aborted, the error word is set or `limit` cycles
// passed.
template <class Cond>
__device__ __forceinline__ bool warp_wait(Cond cond, volatile int* abort, const int* err,
                                          long long limit) {
    bool w = true;
    if (!cond()) {
        const long long t0 = clock64();
        while (!cond()) {
            if (*abort || *reinterpret_cast<const volatile int*>(err) || clock64() - t0 > limit) {
                w = false;
                break;
            }
            __nanosleep(32);
        }
    }
    return __all_sync(0xffffffffu, w);
}

// Warp roles of one CTA (tile b):
//   warp 0, lane 0   producer: streams the tile's bytes into the ring;
//   warp 0, lane 1   watcher: raises chunk k's grid counter once every
//                    phase-1 warp of the CTA finished it (one fence per batch
//                    of chunks), and publishes to the CTA how many chunks are
//                    complete on the whole grid;
//   W1 warps         phase 1: partial dot products, one FP32 L2 reduction per
//                    segment;
//   NC warps         coefficients: for grid-complete chunks (chunk k by warp
//                    k mod NC), c_i of every segment from the complete r_i,
//                    into a shared-memory slot of CQ, and the proximity terms;
//   W2 warps         scatter: Delta_j += c_i a_ij; the box step at the end of
//                    each block.
// Hand-offs inside the CTA are release / acquire operations on shared-memory
// words; across CTAs, relaxed reductions after one fence by the watcher and
// acquire loads of the counters.
template <typename VT, int G>
__global__ void __launch_bounds__(1024, 1) k_tile_sweep(const TileArgs a) {
    if (a.st[0].stopped) return;   // uniform over the grid: nothing is touched
    extern __shared__ __align__(128) unsigned char smraw[];
    __shared__ volatile int abort_flag;
    __shared__ volatile int xver;                     // blocks whose box step is done
    __shared__ volatile int gdone;                    // chunks complete on the grid
    __shared__ volatile int stage_piece[kTileMaxStages];
    __shared__ volatile int p1done[kTileMaxWarps];    // chunks phase-1 warp w finished
    __shared__ volatile int p2done[kTileMaxWarps];    // chunks scatter warp w finished
    __shared__ volatile int ctag[kTileMaxCQ];         // k + 1: slot holds chunk k's coefficients
    __shared__ double prox_w[kTileMaxWarps];
    __shared__ int last_s;
    const int RING = a.stages * a.piece;
    unsigned char* ring = smraw;
    float* xt = reinterpret_cast<float*>(smraw + RING);
    float* dt = xt + a.tile_cap;
    int* scoff = reinterpret_cast<int*>(dt + a.tile_cap);   // K + 1 chunk offsets
    int* snseg = scoff + (a.K + 1);                         // K segment counts
    int* sblk = snseg + a.K;                                // K blocks
    float* cbuf = reinterpret_cast<float*>(sblk + a.K);     // CQ x maxseg coefficients
    uint64_t* full = reinterpret_cast<uint64_t*>(
        (reinterpret_cast<uintptr_t>(cbuf + (size_t)a.cq * a.maxseg) + 15) & ~uintptr_t(15));
    const int b = blockIdx.x, tid = threadIdx.x;
    const int warp = tid >> 5, lane = tid & 31;
    const int W1 = a.W1, NC = a.NC, W2 = a.W2, CQ = a.cq;
    const unsigned epoch = *reinterpret_cast<volatile unsigned*>(a.sync + 1);
    float* r_cur = a.r + (size_t)(epoch & 1u) * a.m;
    float* r_next = a.r + (size_t)((epoch + 1u) & 1u) * a.m;
    const int4 rect = a.rect[b];   // {first global column, rows, columns, local row stride}
    const int ntile = rect.y * rect.w;

    // ---- prologue
    {
        // the other epoch's accumulators start the next sweep at zero
        const long long r0 = (long long)a.m * b / gridDim.x, r1 = (long long)a.m * (b + 1) / gridDim.x;
        for (long long i = r0 + tid; i < r1; i += blockDim.x) r_next[i] = 0.f;
        for (int j = tid; j < ntile; j += blockDim.x) {
            const int rr = j / rect.w, cc = j - rr * rect.w;
            float v = 0.f;
            if (cc < rect.z) v = a.x[rect.x + (long long)rr * a.W + cc];
            xt[j] = v;
            dt[j] = 0.f;
        }
        const int* gco = a.coff + (size_t)b * (a.K + 1);
        const int* gns = a.nseg + (size_t)b * a.K;
        for (int k = tid; k <= a.K; k += blockDim.x) scoff[k] = gco[k];
        for (int k = tid; k < a.K; k += blockDim.x) {
            snseg[k] = gns[k];
            sblk[k] = a.chunk_blk[k];
        }
        if (tid < kTileMaxWarps) {
            p1done[tid] = 0;
            p2done[tid] = 0;
            prox_w[tid] = 0.0;
        }
        if (tid < kTileMaxCQ) ctag[tid] = 0;
        if (tid < kTileMaxStages) stage_piece[tid] = -1;
        if (tid == 0) {
            for (int s = 0; s < a.stages; ++s) tma::mbar_init(&full[s], 1);
            abort_flag = 0;
            xver = 0;
            gdone = 0;
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
    }
    __syncthreads();

    const int ts = 31 - __clz(a.piece);
    const int len_stream = scoff[a.K];
    const long long limit = a.wait_cycles;
    auto give_up = [&](int code) {
        abort_flag = 1;
        atomicExch(a.err, code);
    };

    if (warp == 0) {
        if (lane == 0 && len_stream > 0) {
            // ---- producer: one lane streams the tile's bytes into the ring
            const unsigned char* src = a.stream + a.base[b];
            const uint64_t pol = tma::policy_evict_first();
            const int npieces = (len_stream + a.piece - 1) >> ts;
            int issued = 0;
            long long st_t0 = TSTAT_CLOCK(), st_w = 0;
            (void)st_t0;
            int rel_chunk = 0;   // chunks every scatter warp has finished (cached)
            for (int q = 0; q < npieces; ++q) {
                const int s = q % a.stages;
                if (q >= a.stages) {
                    // the stage's previous piece must be done with: every chunk
                    // overlapping it finished its scatter
                    const int need = (q - a.stages + 1) << ts;
                    if (scoff[rel_chunk] < need) {
                        const long long t0 = clock64();
                        st_w -= TSTAT_CLOCK();
                        bool ok = true;
                        while (true) {
                            int mn = 0x7fffffff;
                            for (int w = 0; w < W2; ++w) mn = min(mn, ld_acquire_cta(&p2done[w]));
                            rel_chunk = mn;
                            if (scoff[rel_chunk] >= need) break;
                            if (abort_flag || *reinterpret_cast<volatile int*>(a.err) ||
                                clock64() - t0 > limit) {
                                ok = false;
                                break;
                            }
                            __nanosleep(64);
                        }
                        st_w += TSTAT_CLOCK();
                        if (!ok) {
                            give_up(3);
                            break;
                        }
                    }
                }
                const int off = q << ts;
                const uint32_t bytes = (uint32_t)min(a.piece, len_stream - off);
                stage_piece[s] = q;
                tma::mbar_arrive_expect_tx(&full[s], bytes);
                tma::bulk_g2s(ring + ((size_t)s << ts), src + off, bytes, &full[s], pol);
                issued = q + 1;
            }
            TSTAT_ADD(6, st_w);
            TSTAT_ADD(7, TSTAT_CLOCK() - st_t0);
            // copies in flight land before the CTA may leave
            volatile int never = 0;
            for (int q = (issued > a.stages ? issued - a.stages : 0); q < issued; ++q)
                tma::mbar_wait(&full[q % a.stages], (q / a.stages) & 1, &never, kTileDrainCycles);
        } else if (lane == 1) {
            // ---- watcher
            int sig = 0, done = 0;
            long long t0 = clock64();
            const unsigned P = gridDim.x;
            long long st_t0 = TSTAT_CLOCK(), st_idle = 0;
            (void)st_t0;
            while (done < a.K) {
                bool prog = false;
                int m1 = a.K;
                for (int w = 0; w < W1; ++w) m1 = min(m1, ld_acquire_cta(&p1done[w]));
                if (m1 > sig) {
                    // the phase-1 warps' reductions (ordered before their
                    // release of p1done) reach the GPU before the counters
                    __threadfence();
                    for (int k = sig; k < m1; ++k) red_add_u32_gpu(a.cnt + k, 1u);
                    sig = m1;
                    prog = true;
                }
                while (done < sig && ld_acquire_gpu(a.cnt + done) >= P) {
                    ++done;
                    prog = true;
                }
                if (prog) {
                    st_release_cta(&gdone, done);
                    t0 = clock64();
                } else {
                    if (abort_flag || *reinterpret_cast<volatile int*>(a.err) || clock64() - t0 > limit) {
                        give_up(3);
                        break;
                    }
                    st_idle += 1;
                    __nanosleep(32);
                }
            }
            TSTAT_ADD(8, st_idle);
            TSTAT_ADD(9, TSTAT_CLOCK() - st_t0);
        }
    } else if (warp <= W1) {
        // ---- phase 1: partial dot products of the tile's segments
        const int w1 = warp - 1;
        constexpr int GPW = 32 / G;
        const int gi = lane / G, gl = lane % G;
        bool ok = true;
        int cur_blk = 0;
        long long st_t0 = TSTAT_CLOCK(), st_w = 0;
        (void)st_t0;
        for (int k = 0; k < a.K; ++k) {
            const int blk = sblk[k];
            st_w -= TSTAT_CLOCK();
            if (blk != cur_blk) {
                // the next block's dot products use x after the block's box step
                cur_blk = blk;
                if (ok) {
                    ok = warp_wait([&] { return ld_acquire_cta(&xver) >= blk; }, &abort_flag, a.err, limit);
                    if (!ok && lane == 0) give_up(3);
                }
            }
            const int c0 = scoff[k], c1 = scoff[k + 1];
            if (ok && c1 > c0) {
                for (int q = c0 >> ts; ok && q <= (c1 - 1) >> ts; ++q) {
                    const int s = q % a.stages;
                    ok = warp_wait([&] { return stage_piece[s] == q; }, &abort_flag, a.err, limit);
                    if (ok) ok = __all_sync(0xffffffffu, tma::mbar_wait(&full[s], (q / a.stages) & 1,
                                                                        &abort_flag, limit));
                }
                if (!ok && lane == 0) give_up(3);
            }
            st_w += TSTAT_CLOCK();
            if (ok && c1 > c0) {
                const int nseg = snseg[k];
                const int rc = c0 % RING;
                for (int base = w1 * GPW; base < nseg; base += W1 * GPW) {
                    const int sg = base + gi;
                    float dot = 0.f;
                    int row = -1;
                    if (sg < nseg) {
                        const uint2 d = *reinterpret_cast<const uint2*>(ring + wrap(rc + 8 * sg, RING));
                        row = (int)(d.x & 0x7fffffffu);
                        const int off = 4 * (int)(d.y & 0xffffu), len = (int)(d.y >> 16);
                        const int vp = wrap(rc + off, RING);
                        const int ip = wrap(vp + (int)sizeof(VT) * len, RING);
                        float d0 = 0.f, d1 = 0.f;
                        if (ip + 2 * len <= RING && vp + (int)sizeof(VT) * len <= RING) {
                            const VT* vv = reinterpret_cast<const VT*>(ring + vp);
                            const unsigned short* ii = reinterpret_cast<const unsigned short*>(ring + ip);
                            int e = gl;
                            for (; e + G < len; e += 2 * G) {
                                d0 = fmaf(to_float(vv[e]), xt[ii[e]], d0);
                                d1 = fmaf(to_float(vv[e + G]), xt[ii[e + G]], d1);
                            }
                            if (e < len) d0 = fmaf(to_float(vv[e]), xt[ii[e]], d0);
                        } else {
                            for (int e = gl; e < len; e += G) {
                                const float v = to_float(*reinterpret_cast<const VT*>(
                                    ring + wrap(vp + (int)sizeof(VT) * e, RING)));
                                const int j = *reinterpret_cast<const unsigned short*>(
                                    ring + wrap(ip + 2 * e, RING));
                                d0 = fmaf(v, xt[j], d0);
                            }
                        }
                        dot = d0 + d1;
                    }
#pragma unroll
                    for (int o = G / 2; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
                    // lane 0 issues the warp's reductions: its release of
                    // p1done then orders all of them
#pragma unroll
                    for (int g2 = 0; g2 < GPW; ++g2) {
                        const float pv = __shfl_sync(0xffffffffu, dot, g2 * G);
                        const int pr = __shfl_sync(0xffffffffu, row, g2 * G);
                        if (lane == 0 && pr >= 0) red_add_gpu(r_cur + pr, pv);
                    }
                }
            }
            __syncwarp();
            if (ok && lane == 0) st_release_cta(&p1done[w1], k + 1);
        }
        if (lane == 0) {
            TSTAT_ADD(0, st_w);
            TSTAT_ADD(1, TSTAT_CLOCK() - st_t0);
        }
    } else if (warp <= W1 + NC) {
        // ---- coefficients of grid-complete chunks
        const int wc = warp - 1 - W1;
        double pacc = 0.0;
        bool ok = true;
        long long st_t0 = TSTAT_CLOCK(), st_w = 0;
        (void)st_t0;
        for (int k = wc; k < a.K && ok; k += NC) {
            const int slot = k % CQ;
            st_w -= TSTAT_CLOCK();
            if (k >= CQ)
                ok = warp_wait([&] { return ld_acquire_cta(&p2done[lane < W2 ? lane : 0]) > k - CQ || lane >= W2; },
                               &abort_flag, a.err, limit);
            if (ok) ok = warp_wait([&] { return ld_acquire_cta(&gdone) > k; }, &abort_flag, a.err, limit);
            st_w += TSTAT_CLOCK();
            if (!ok) {
                if (lane == 0) give_up(3);
                break;
            }
            const int c0 = scoff[k], nseg = snseg[k];
            const int rc = c0 % RING;
            const double scale = a.blk_scale[sblk[k]];
            float* cb = cbuf + (size_t)slot * a.maxseg;
            for (int s0 = 0; s0 < nseg; s0 += 4 * 32) {
                uint2 d[4];
                float ri[4], li[4], ui[4], wi[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int sg = s0 + u * 32 + lane;
                    if (sg < nseg) {
                        d[u] = *reinterpret_cast<const uint2*>(ring + wrap(rc + 8 * sg, RING));
                        const int row = (int)(d[u].x & 0x7fffffffu);
                        ri[u] = ld_relaxed_gpu(r_cur + row);
                        li[u] = __ldg(a.l + row);
                        ui[u] = __ldg(a.u + row);
                        wi[u] = __ldg(a.wr + row);
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int sg = s0 + u * 32 + lane;
                    if (sg < nseg) {
                        const float dd = clampf(ri[u], li[u], ui[u]) - ri[u];
                        cb[sg] = a.lam * wi[u] * dd;
                        if (d[u].x & 0x80000000u) pacc += (double)dd * (double)dd * (double)wi[u] * scale;
                    }
                }
            }
            __syncwarp();
            if (lane == 0) st_release_cta(&ctag[slot], k + 1);
        }
        pacc = warp_sum(pacc);
        if (lane == 0) {
            prox_w[wc] = pacc;
            TSTAT_ADD(2, st_w);
            TSTAT_ADD(3, TSTAT_CLOCK() - st_t0);
        }
    } else {
        // ---- scatter into Delta, and the box step at the end of each block
        const int w2 = warp - 1 - W1 - NC;
        constexpr int GPW = 32 / G;
        const int gi = lane / G, gl = lane % G;
        const int t2 = tid - 32 * (1 + W1 + NC);   // 0 .. 32 W2 - 1
        bool ok = true;
        long long st_t0 = TSTAT_CLOCK(), st_w = 0;
        (void)st_t0;
        for (int k = 0; k < a.K; ++k) {
            const int blk = sblk[k];
            const int slot = k % CQ;
            st_w -= TSTAT_CLOCK();
            if (ok) {
                ok = warp_wait([&] { return ld_acquire_cta(&ctag[slot]) > k; }, &abort_flag, a.err, limit);
                if (!ok && lane == 0) give_up(3);
            }
            st_w += TSTAT_CLOCK();
            const int c0 = scoff[k], nseg = snseg[k];
            if (ok && nseg > 0) {
                const int rc = c0 % RING;
                const float* cb = cbuf + (size_t)slot * a.maxseg;
                for (int base = w2 * GPW; base < nseg; base += W2 * GPW) {
                    const int sg = base + gi;
                    if (sg < nseg) {
                        const float c = cb[sg];
                        if (c != 0.f) {
                            const uint2 d = *reinterpret_cast<const uint2*>(ring + wrap(rc + 8 * sg, RING));
                            const int off = 4 * (int)(d.y & 0xffffu), len = (int)(d.y >> 16);
                            const int vp = wrap(rc + off, RING);
                            const int ip = wrap(vp + (int)sizeof(VT) * len, RING);
                            for (int e = gl; e < len; e += kCasBatch * G)
                                scatter_batch<VT, G>(ring, RING, vp, ip, e, len, c, dt);
                        }
                    }
                }
            }
            __syncwarp();
            if (lane == 0) st_release_cta(&p2done[w2], k + 1);
            if (k + 1 == a.K || sblk[k + 1] != blk) {
                // end of the block: the box step on the tile (every scatter
                // warp has finished the block's chunks)
                named_sync(1, 32 * W2);
                const bool last = (k + 1 == a.K);
                for (int j = t2; j < ntile; j += 32 * W2) {
                    const int rr = j / rect.w, cc = j - rr * rect.w;
                    if (cc >= rect.z) continue;
                    const long long g = rect.x + (long long)rr * a.W + cc;
                    const int bj = (a.box_len == 1) ? 0 : (int)g;
                    float sv = dt[j];
                    if (a.zc) sv *= __ldg(a.zc + g);
                    const float v = clampf(xt[j] + sv, __ldg(a.lo + bj), __ldg(a.hi + bj));
                    xt[j] = v;
                    dt[j] = 0.f;
                    if (last) a.x[g] = v;
                }
                named_sync(1, 32 * W2);
                if (t2 == 0) st_release_cta(&xver, blk + 1);
            }
        }
        if (lane == 0) {
            TSTAT_ADD(4, st_w);
            TSTAT_ADD(5, TSTAT_CLOCK() - st_t0);
        }
    }
    __syncthreads();

    // ---- end: proximity partial, the last CTA runs the epilogue and resets
    if (tid == 0) {
        double sp = 0.0;
        for (int w = 0; w < NC; ++w) sp += prox_w[w];
        a.pp[b] = sp;
        __threadfence();
        last_s = (atomicAdd(a.sync, 1u) == gridDim.x - 1) ? 1 : 0;
    }
    __syncthreads();
    if (last_s) {
        __threadfence();
        sweep_epilogue(a.epi);
        for (int k = tid; k < a.K; k += blockDim.x) a.cnt[k] = 0u;
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            *reinterpret_cast<volatile unsigned*>(a.sync) = 0u;
            __threadfence();
            *reinterpret_cast<volatile unsigned*>(a.sync + 1) = epoch + 1u;
        }
    }
}

// Fill of the tile streams: one warp per segment writes its descriptor and
// copies its values and tile-local indices.
template <typename VT>
__global__ void k_tile_fill(const TileSegRec* segs, long long nsegs, const VT* val, const int* col,
                            const unsigned short* local_of, unsigned char* stream) {
    const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= nsegs) return;
    const TileSegRec r = segs[w];
    unsigned char* chunk = stream + r.chunk_start;
    if (lane == 0) {
        uint2 d;
        d.x = (unsigned)r.row_flag;
        d.y = (unsigned)r.off4 | ((unsigned)r.len << 16);
        *reinterpret_cast<uint2*>(chunk + 8LL * r.sidx) = d;
    }
    VT* dv = reinterpret_cast<VT*>(chunk + 4LL * r.off4);
    unsigned short* di = reinterpret_cast<unsigned short*>(chunk + 4LL * r.off4 + sizeof(VT) * r.len);
    for (int e = lane; e < r.len; e += 32) {
        dv[e] = val[r.e0 + e];
        di[e] = local_of[col[r.e0 + e]];
    }
}

using TileFn = void (*)(TileArgs);

template <typename VT>
TileFn tile_fn_g(int G) {
    switch (G) {
        case 8: return k_tile_sweep<VT, 8>;
        case 16: return k_tile_sweep<VT, 16>;
        default: return k_tile_sweep<VT, 32>;
    }
}

TileFn tile_fn(suppy_dtype dt, int G) {
    if (dt == SUPPY_F32) return tile_fn_g<float>(G);
    if (dt == SUPPY_BF16) return tile_fn_g<__nv_bfloat16>(G);
    return tile_fn_g<__half>(G);
}

}  // namespace

size_t tile_smem_bytes(int ring_bytes, int tile_cap, int K, int stages, int cq, int maxseg) {
    size_t b = (size_t)ring_bytes + 8 * (size_t)tile_cap + 4 * (3 * (size_t)K + 1) +
               4 * (size_t)cq * maxseg;
    b = (b + 15) & ~(size_t)15;
    return b + 8 * (size_t)stages;
}

int tile_blocks_per_sm(suppy_dtype dt, int G, int threads, size_t smem) {
    TileFn f = tile_fn(dt, G);
    if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, threads, smem) != cudaSuccess) return 0;
    return nb;
}

cudaError_t launch_tile_sweep(const TileArgs& a, suppy_dtype dt, int G, int grid, size_t smem,
                              cudaStream_t s) {
    if (a.W1 < 1 || a.W2 < 1 || a.NC < 1 || 1 + a.W1 + a.NC + a.W2 > kTileMaxWarps ||
        a.cq < a.NC || a.cq > kTileMaxCQ || a.stages < 2 ||
        a.stages > kTileMaxStages || a.piece < 256 || (a.piece & (a.piece - 1)) || grid < 1)
        return cudaErrorInvalidValue;
    TileFn f = tile_fn(dt, G);
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid, 1, 1);
    cfg.blockDim = dim3(32 * (1 + a.W1 + a.NC + a.W2), 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, f, a);
}

cudaError_t launch_tile_fill(const TileSegRec* segs, long long nsegs, const void* val,
                             suppy_dtype dt, const int* col, const unsigned short* local_of,
                             unsigned char* stream, cudaStream_t s) {
    if (nsegs <= 0) return cudaSuccess;
    const long long threads = nsegs * 32;
    const int block = 256;
    const long long grid = (threads + block - 1) / block;
    if (dt == SUPPY_F32)
        k_tile_fill<float><<<(unsigned)grid, block, 0, s>>>(segs, nsegs, static_cast<const float*>(val),
                                                           col, local_of, stream);
    else if (dt == SUPPY_BF16)
        k_tile_fill<__nv_bfloat16><<<(unsigned)grid, block, 0, s>>>(
            segs, nsegs, static_cast<const __nv_bfloat16*>(val), col, local_of, stream);
    else
        k_tile_fill<__half><<<(unsigned)grid, block, 0, s>>>(segs, nsegs, static_cast<const __half*>(val),
                                                            col, local_of, stream);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- host plan

namespace {

// Split [0, len) of a nonnegative weight sequence into `parts` consecutive
// nonempty ranges of about equal weight; bounds[0] = 0, bounds[parts] = len.
void balanced_cuts(const std::vector<double>& w, int parts, std::vector<int>& bounds) {
    const int len = (int)w.size();
    bounds.assign(parts + 1, 0);
    bounds[parts] = len;
    std::vector<double> pref(len + 1, 0.0);
    for (int i = 0; i < len; ++i) pref[i + 1] = pref[i] + w[i];
    const double tot = pref[len];
    int lo = 0;
    for (int p = 1; p < parts; ++p) {
        int cut;
        if (tot > 0.0) {
            const double target = tot * p / parts;
            cut = (int)(std::lower_bound(pref.begin(), pref.end(), target) - pref.begin());
        } else {
            cut = (int)((long long)len * p / parts);
        }
        // every range keeps at least one element
        cut = std::max(cut, lo + 1);
        cut = std::min(cut, len - (parts - p));
        bounds[p] = cut;
        lo = cut;
    }
}

}  // namespace

bool plan_tiles(const TilePlanIn& in, TilePlan& out, std::string& why) {
    const int n = in.n, H = in.H, W = in.W;
    if ((long long)H * W != n || H < 1 || W < 1) {
        why = "tile plan: H * W must equal n";
        return false;
    }
    const int vs = in.vbytes;
    // ---- column weights (entries per column)
    std::vector<double> colw(n, 0.0);
    for (int i = 0; i < in.m; ++i) {
        const int src = in.perm ? in.perm[i] : i;
        const int* cp = in.col + in.rp[src];
        const int len = in.rp[src + 1] - in.rp[src];
        for (int t = 0; t < len; ++t) colw[cp[t]] += 1.0;
    }
    // ---- tiles: R1 bands of image rows balanced by weight, each band cut
    // into column ranges balanced by its own weight
    int P = std::min<long long>(in.P, (long long)n) > 0 ? (int)std::min<long long>(in.P, n) : 1;
    int R1 = (int)std::lround(std::sqrt((double)P * H / W));
    R1 = std::max(1, std::min(R1, std::min(P, H)));
    std::vector<int> per_band(R1);
    for (int i = 0; i < R1; ++i) per_band[i] = P / R1 + (i < P % R1 ? 1 : 0);
    for (int i = 0; i < R1; ++i) per_band[i] = std::min(per_band[i], W);
    P = std::accumulate(per_band.begin(), per_band.end(), 0);
    std::vector<double> roww(H, 0.0);
    for (int i = 0; i < H; ++i)
        for (int j = 0; j < W; ++j) roww[i] += colw[(size_t)i * W + j];
    // band boundaries: cumulative weight in proportion to the band's tiles
    std::vector<int> band(R1 + 1, 0);
    {
        std::vector<double> pref(H + 1, 0.0);
        for (int i = 0; i < H; ++i) pref[i + 1] = pref[i] + roww[i];
        const double tot = pref[H];
        int acc = 0, lo = 0;
        band[R1] = H;
        for (int bi = 1; bi < R1; ++bi) {
            acc += per_band[bi - 1];
            int cut = tot > 0.0
                          ? (int)(std::lower_bound(pref.begin(), pref.end(), tot * acc / P) - pref.begin())
                          : (int)((long long)H * acc / P);
            cut = std::max(cut, lo + 1);
            cut = std::min(cut, H - (R1 - bi));
            band[bi] = cut;
            lo = cut;
        }
    }
    out.rect.clear();
    out.tile_of.assign(n, 0);
    out.local_of.assign(n, 0);
    out.tile_cap = 0;
    for (int bi = 0; bi < R1; ++bi) {
        const int i0 = band[bi], i1 = band[bi + 1];
        std::vector<double> cw(W, 0.0);
        for (int i = i0; i < i1; ++i)
            for (int j = 0; j < W; ++j) cw[j] += colw[(size_t)i * W + j];
        std::vector<int> cuts;
        balanced_cuts(cw, per_band[bi], cuts);
        for (int p = 0; p < per_band[bi]; ++p) {
            const int j0 = cuts[p], j1 = cuts[p + 1];
            const int th = i1 - i0, tw = j1 - j0;
            const int stride = tw | 1;   // odd: rays stepping by a row hit distinct banks
            const long long cap = (long long)th * stride;
            if (cap > in.max_tile_words) {
                why = "tile plan: a tile exceeds the shared-memory tile capacity";
                return false;
            }
            const int id = (int)out.rect.size();
            out.rect.push_back(make_int4(i0 * W + j0, th, tw, stride));
            out.tile_cap = std::max<int>(out.tile_cap, (int)cap);
            for (int i = i0; i < i1; ++i)
                for (int j = j0; j < j1; ++j) {
                    out.tile_of[(size_t)i * W + j] = id;
                    out.local_of[(size_t)i * W + j] = (unsigned short)((i - i0) * stride + (j - j0));
                }
        }
    }
    out.P = P;
    // ---- segments: runs of a row's consecutive entries in one tile
    struct Run {
        int tile, row, e0, len;
    };
    std::vector<Run> runs;
    runs.reserve((size_t)in.m * 8);
    std::vector<long long> row_bytes(in.m, 0);
    std::vector<int> row_run(in.m + 1, 0);
    for (int i = 0; i < in.m; ++i) {
        row_run[i] = (int)runs.size();
        const int src = in.perm ? in.perm[i] : i;
        const int* cp = in.col + in.rp[src];
        const int len = in.rp[src + 1] - in.rp[src];
        int t = 0;
        while (t < len) {
            const int tb = out.tile_of[cp[t]];
            int e = t + 1;
            while (e < len && e - t < in.max_seg && out.tile_of[cp[e]] == tb) ++e;
            runs.push_back(Run{tb, i, in.row_start[i] + t, e - t});
            row_bytes[i] += 8 + (((long long)(e - t) * (vs + 2) + 3) & ~3LL);
            t = e;
        }
    }
    row_run[in.m] = (int)runs.size();
    if (runs.size() >= (size_t)INT32_MAX) {
        why = "tile plan: too many segments";
        return false;
    }
    // ---- chunks: consecutive rows inside a block, about `target` stream
    // bytes per CTA each; halved while some tile's chunk exceeds max_chunk
    const int nblk = (int)in.seg_start.size() - 1;
    // rows of a block in a scattered order (a stride near len / golden ratio,
    // coprime to the block length): each chunk then holds rays of every
    // direction and position, so every tile gets about the same share of it
    std::vector<int> order(in.m);
    for (int t = 0; t < nblk; ++t) {
        const long long r0 = in.seg_start[t], len = in.seg_start[t + 1] - r0;
        long long S = std::max<long long>(1, std::llround((double)len * 0.6180339887498949));
        while (len > 1 && std::gcd(S, len) != 1) ++S;
        for (long long j = 0; j < len; ++j) order[r0 + j] = (int)(r0 + (j * S) % std::max<long long>(len, 1));
    }
    long long target = (long long)in.chunk_target * P;
    for (int attempt = 0; attempt < 12; ++attempt) {
        std::vector<int> ck;      // positions in `order` where the chunks start
        std::vector<int> cblk;
        for (int t = 0; t < nblk; ++t) {
            const int r0 = in.seg_start[t], r1 = in.seg_start[t + 1];
            long long acc = 0;
            int start = r0;
            for (int j = r0; j < r1; ++j) {
                acc += row_bytes[order[j]];
                if (acc >= target) {
                    ck.push_back(start);
                    cblk.push_back(t);
                    start = j + 1;
                    acc = 0;
                }
            }
            if (start < r1 || r0 == r1) {
                ck.push_back(start);
                cblk.push_back(t);
            }
        }
        const int K = (int)ck.size();
        ck.push_back(in.m);
        if (K > in.max_chunks) {
            why = "tile plan: more chunks than the kernel's tables hold";
            return false;
        }
        std::vector<int> nseg((size_t)P * K, 0);
        std::vector<long long> dbytes((size_t)P * K, 0);
        for (int k = 0; k < K; ++k)
            for (int j = ck[k]; j < ck[k + 1]; ++j) {
                const int i = order[j];
                for (int r = row_run[i]; r < row_run[i + 1]; ++r) {
                    const Run& u = runs[r];
                    nseg[(size_t)u.tile * K + k] += 1;
                    dbytes[(size_t)u.tile * K + k] += ((long long)u.len * (vs + 2) + 3) & ~3LL;
                }
            }
        long long worst = 0;
        int worst_nseg = 0;
        std::vector<long long> csize((size_t)P * K);
        for (size_t q = 0; q < csize.size(); ++q) {
            const long long desc = ((long long)nseg[q] * 8 + 15) & ~15LL;
            csize[q] = (desc + dbytes[q] + 15) & ~15LL;
            worst = std::max(worst, csize[q]);
            worst_nseg = std::max(worst_nseg, nseg[q]);
        }
        if (worst > in.max_chunk || worst_nseg > in.max_nseg) {
            target /= 2;
            if (target < 1024) break;
            continue;
        }
        // ---- offsets
        out.K = K;
        out.chunk_blk = cblk;
        out.nseg = nseg;
        out.coff.assign((size_t)P * (K + 1), 0);
        out.base.assign(P, 0);
        long long tot = 0;
        out.max_chunk = (int)worst;
        out.max_nseg = worst_nseg;
        for (int p = 0; p < P; ++p) {
            out.base[p] = tot;
            long long o = 0;
            for (int k = 0; k < K; ++k) {
                out.coff[(size_t)p * (K + 1) + k] = (int)o;
                o += csize[(size_t)p * K + k];
            }
            out.coff[(size_t)p * (K + 1) + K] = (int)o;
            if (o >= (1LL << 31) - 1) {
                why = "tile plan: a tile's stream exceeds 2 GB";
                return false;
            }
            tot += o;
        }
        out.bytes = tot;
        // ---- segment records in row order (descriptors first, then data)
        std::vector<int> sidx((size_t)P * K, 0);
        std::vector<long long> dpos((size_t)P * K);
        for (size_t q = 0; q < dpos.size(); ++q) dpos[q] = ((long long)nseg[q] * 8 + 15) & ~15LL;
        out.segs.resize(runs.size());
        for (int k = 0; k < K; ++k) {
            for (int j = ck[k]; j < ck[k + 1]; ++j) {
                const int i = order[j];
                for (int r = row_run[i]; r < row_run[i + 1]; ++r) {
                    const Run& u = runs[r];
                    const size_t q = (size_t)u.tile * K + k;
                    TileSegRec& s = out.segs[r];
                    s.chunk_start = out.base[u.tile] + out.coff[(size_t)u.tile * (K + 1) + k];
                    s.sidx = sidx[q]++;
                    s.off4 = (int)(dpos[q] >> 2);
                    s.row_flag = i | (r == row_run[i] ? (int)0x80000000u : 0);
                    s.e0 = u.e0;
                    s.len = u.len;
                    dpos[q] += ((long long)u.len * (vs + 2) + 3) & ~3LL;
                }
            }
        }
        return true;
    }
    why = "tile plan: no chunking keeps every tile's chunk within the ring";
    return false;
}

}  // namespace suppy

#ifdef SUPPY_TILE_STATS
extern "C" int suppy_tile_stats(unsigned long long* out16, int reset) {
    cudaError_t e = cudaMemcpyFromSymbol(out16, suppy::g_tile_stats, sizeof(unsigned long long) * 16);
    if (e != cudaSuccess || !reset) return (int)e;
    unsigned long long z[16] = {};
    return (int)cudaMemcpyToSymbol(suppy::g_tile_stats, z, sizeof(z));
}
#endif
