// Tiled one-pass simultaneous projection sweep (Sec. 2.1.1, Eq. (3); the
// box projection after each sweep or block, Sec. 2.3.3), one right-hand side.
//
// The unknowns are split into P tiles (rectangles of the image for imaging
// problems, column ranges otherwise), one per CTA of one cooperative launch;
// a CTA keeps its tile's x and correction Delta in shared memory for the
// whole sweep.  Every row a_i is cut into segments, runs of its consecutive
// entries that fall in one tile.  Each tile's segments form one contiguous
// byte stream, grouped into chunks of consecutive rows; inside a chunk, up to
// 32 segments (of neighbouring rows) form a slice, sorted by length, whose
// entries are stored step by step: first entry 0 of every segment, then entry
// 1 of those that have one, and so on (values, then 16-bit tile-local column
// indices).  A warp then takes a slice with one lane per segment, and at
// every step its active lanes read consecutive words.  A CTA streams its
// tile's bytes once per sweep into a shared-memory ring with bulk
// asynchronous copies, so A crosses HBM once; the gathers of x and the
// scatter into Delta never leave the SM.
//
// Per chunk k:
//   phase 1 (dot products): the partial <a_i, x> of every segment from the
//     tile's x, added to r_i (one FP32 L2 reduction per segment); once every
//     phase-1 warp of the CTA is done with the chunk, its grid counter is
//     raised;
//   coefficients, once the counter says every CTA finished phase 1 of chunk
//     k: c_i = lambda w_i (clamp(r_i, l_i, u_i) - r_i) / ||a_i||^2 from the
//     complete r_i (and the proximity term of row i, added by the segment
//     that holds the row's first entry, FP64);
//   scatter: Delta_j += c_i a_ij (shared-memory compare-and-swap additions).
// Phase 1 runs ahead of the scatter by as many chunks as the ring holds, so
// the cross-CTA dependency is a rolling one, not a grid barrier.  At the end
// of a block (the whole sweep for Cimmino and DROP) x_j <- box(x_j + z_j Delta_j)
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
// waits / total, 6/7 producer waits / total, 8/9 watcher idle polls / total),
// and per chunk of CTAs 0 and 1 the global time (ns) of six events: its last
// piece issued, phase 1 done, its counter raised, grid-complete seen,
// coefficients done, scatter done.
__device__ unsigned long long g_tile_stats[16];
__device__ unsigned long long g_tile_trace[2][kTileMaxChunks][6];
#define TSTAT_CLOCK() clock64()
#define TSTAT_ADD(k, v) atomicAdd(&g_tile_stats[k], (unsigned long long)(v))
__device__ __forceinline__ unsigned long long gtime() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}
#define TTRACE(k, ev) \
    do { if (blockIdx.x < 2 && (k) < kTileMaxChunks) g_tile_trace[blockIdx.x][k][ev] = gtime(); } while (0)
#else
#define TSTAT_CLOCK() 0LL
#define TSTAT_ADD(k, v) ((void)0)
#define TTRACE(k, ev) ((void)0)
#endif

namespace {

constexpr long long kTileDrainCycles = 4000000000LL;
constexpr unsigned kFull = 0xffffffffu;

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

__device__ __forceinline__ void red_add_u32_gpu(unsigned* p, unsigned v) {
    asm volatile("red.relaxed.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
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

__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

__device__ __forceinline__ void named_sync(int id, int threads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

// Ring position of a stream offset that lies less than one ring beyond the
// ring's end.
__device__ __forceinline__ int wrap(int p, int ring) { return p >= ring ? p - ring : p; }

// One try_wait with a suspend-time hint: the thread sleeps in hardware until
// the phase completes or about `ns` nanoseconds pass.
__device__ __forceinline__ bool mbar_try_wait_ns(uint64_t* bar, uint32_t parity, uint32_t ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(tma::smem_addr(bar)), "r"(parity), "r"(ns)
        : "memory");
    return ok != 0;
}

// Bounded wait of a whole warp for the phase of `bar` with the given parity:
// false for every lane when the CTA aborted, the error word is set or `limit`
// cycles passed.  The waiting threads sleep in hardware between tries.
__device__ __forceinline__ bool warp_bar_wait(uint64_t* bar, uint32_t parity, volatile int* abort,
                                              const int* err, long long limit) {
    bool w = true;
    if (!mbar_try_wait_ns(bar, parity, 1000)) {
        const long long t0 = clock64();
        while (!mbar_try_wait_ns(bar, parity, 1000)) {
            if (*abort || *reinterpret_cast<const volatile int*>(err) || clock64() - t0 > limit) {
                w = false;
                break;
            }
        }
    }
    return __all_sync(kFull, w);
}

// A slice in the ring, seen by one warp (lane j = the slice's j-th longest
// segment).  Layout from the slice start: nl rows (int32, bit 31 marks the
// segment holding the row's first entry), nl lengths (u16), padding to 4
// bytes, then E values and E column indices (u16), step by step.
struct Slice {
    int nl, E, L0;          // segments, entries, longest segment
    int row_pos, vpos, ipos;
    bool flat;              // the slice does not wrap around the ring end
};

template <typename VT>
__device__ __forceinline__ Slice slice_at(const unsigned char* ring, int RING, int rc, int s,
                                          int lane, int* row, int* len) {
    const uint2 d = *reinterpret_cast<const uint2*>(ring + wrap(rc + 8 * s, RING));
    Slice sl;
    sl.nl = (int)(d.y & 63u);
    sl.E = (int)(d.y >> 6);
    const int sp = wrap(rc + 4 * (int)d.x, RING);
    sl.row_pos = sp;
    const int lpos = wrap(sp + 4 * sl.nl, RING);
    sl.vpos = wrap(sp + ((6 * sl.nl + 3) & ~3), RING);
    sl.ipos = wrap(sl.vpos + (int)sizeof(VT) * sl.E, RING);
    sl.flat = (sp + ((6 * sl.nl + 3) & ~3) + ((int)sizeof(VT) + 2) * sl.E) <= RING;
    *row = -1;
    *len = 0;
    if (lane < sl.nl) {
        *row = *reinterpret_cast<const int*>(ring + wrap(sp + 4 * lane, RING));
        *len = *reinterpret_cast<const unsigned short*>(ring + wrap(lpos + 2 * lane, RING));
    }
    sl.L0 = __shfl_sync(kFull, *len, 0);
    return sl;
}

template <typename VT>
__device__ __forceinline__ float ring_val(const unsigned char* ring, int RING, const Slice& sl, int p) {
    return to_float(*reinterpret_cast<const VT*>(ring + wrap(sl.vpos + (int)sizeof(VT) * p, RING)));
}

__device__ __forceinline__ int ring_idx(const unsigned char* ring, int RING, const Slice& sl, int p) {
    return *reinterpret_cast<const unsigned short*>(ring + wrap(sl.ipos + 2 * p, RING));
}

// <a_i, x> over the lane's segment: at step e the lanes with len > e are
// lanes 0 .. n_e - 1, and their entries sit at positions base_e + lane.
template <typename VT>
__device__ __forceinline__ float slice_dot(const unsigned char* ring, int RING, const Slice& sl,
                                           int lane, int len, const float* xt) {
    float a0 = 0.f, a1 = 0.f;
    int base = 0;
    if (sl.flat) {
        const VT* vv = reinterpret_cast<const VT*>(ring + sl.vpos);
        const unsigned short* ii = reinterpret_cast<const unsigned short*>(ring + sl.ipos);
        int e = 0;
        for (; e + 3 < sl.L0; e += 4) {
            // four steps' loads in flight: positions from the counts of lanes
            // still active at each step
            const int n0 = __popc(__ballot_sync(kFull, e < len));
            const int n1 = __popc(__ballot_sync(kFull, e + 1 < len));
            const int n2 = __popc(__ballot_sync(kFull, e + 2 < len));
            const int n3 = __popc(__ballot_sync(kFull, e + 3 < len));
            const int p0 = base + lane, p1 = p0 + n0, p2 = p1 + n1, p3 = p2 + n2;
            float v[4] = {0.f, 0.f, 0.f, 0.f};
            int j[4] = {0, 0, 0, 0};
            if (e < len) { v[0] = to_float(vv[p0]); j[0] = ii[p0]; }
            if (e + 1 < len) { v[1] = to_float(vv[p1]); j[1] = ii[p1]; }
            if (e + 2 < len) { v[2] = to_float(vv[p2]); j[2] = ii[p2]; }
            if (e + 3 < len) { v[3] = to_float(vv[p3]); j[3] = ii[p3]; }
            a0 = fmaf(v[0], xt[j[0]], a0);
            a1 = fmaf(v[1], xt[j[1]], a1);
            a0 = fmaf(v[2], xt[j[2]], a0);
            a1 = fmaf(v[3], xt[j[3]], a1);
            base += n0 + n1 + n2 + n3;
        }
        for (; e < sl.L0; ++e) {
            const int n0 = __popc(__ballot_sync(kFull, e < len));
            if (e < len) a0 = fmaf(to_float(vv[base + lane]), xt[ii[base + lane]], a0);
            base += n0;
        }
    } else {
        for (int e = 0; e < sl.L0; ++e) {
            const bool c0 = e < len;
            const int n0 = __popc(__ballot_sync(kFull, c0));
            if (c0) a0 = fmaf(ring_val<VT>(ring, RING, sl, base + lane), xt[ring_idx(ring, RING, sl, base + lane)], a0);
            base += n0;
        }
    }
    return a0 + a1;
}

// Delta_j += c a_ij over the lane's segment (c = 0: the lane only counts its
// positions).  FP32 additions into shared memory made atomic by
// compare-and-swap: a lane reads the current sum, and retries only when
// another lane changed it in between (rare: a slice's segments are distinct
// rays, and its lanes' positions at one step are distinct columns).  Two steps
// are in flight per lane.
__device__ __forceinline__ void cas_add(float* dt, int j, float v, float old) {
    unsigned* p = reinterpret_cast<unsigned*>(dt) + j;
    unsigned prev = atomicCAS(p, __float_as_uint(old), __float_as_uint(old + v));
    while (prev != __float_as_uint(old)) {
        old = __uint_as_float(prev);
        prev = atomicCAS(p, prev, __float_as_uint(old + v));
    }
}

template <typename VT>
__device__ __forceinline__ void slice_scatter(const unsigned char* ring, int RING, const Slice& sl,
                                              int lane, int len, float c, float* dt) {
    volatile float* vd = dt;
    const int lact = (c != 0.f) ? len : 0;   // steps this lane adds
    int base = 0;
    if (sl.flat) {
        const VT* vv = reinterpret_cast<const VT*>(ring + sl.vpos);
        const unsigned short* ii = reinterpret_cast<const unsigned short*>(ring + sl.ipos);
        int e = 0;
        for (; e + 3 < sl.L0; e += 4) {
            const int n0 = __popc(__ballot_sync(kFull, e < len));
            const int n1 = __popc(__ballot_sync(kFull, e + 1 < len));
            const int n2 = __popc(__ballot_sync(kFull, e + 2 < len));
            const int n3 = __popc(__ballot_sync(kFull, e + 3 < len));
            const int p[4] = {base + lane, base + n0 + lane, base + n0 + n1 + lane,
                              base + n0 + n1 + n2 + lane};
            float v[4], o[4];
            int j[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                j[u] = 0;
                v[u] = 0.f;
                if (e + u < lact) {
                    j[u] = ii[p[u]];
                    v[u] = c * to_float(vv[p[u]]);
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) o[u] = (e + u < lact) ? vd[j[u]] : 0.f;
            // the four compare-and-swaps issued back to back; a lost race
            // retries with the value it found
            unsigned prev[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (e + u < lact)
                    prev[u] = atomicCAS(reinterpret_cast<unsigned*>(dt) + j[u], __float_as_uint(o[u]),
                                        __float_as_uint(o[u] + v[u]));
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (e + u < lact && prev[u] != __float_as_uint(o[u]))
                    cas_add(dt, j[u], v[u], __uint_as_float(prev[u]));
            base += n0 + n1 + n2 + n3;
        }
        for (; e < sl.L0; ++e) {
            const int n0 = __popc(__ballot_sync(kFull, e < len));
            if (e < lact) {
                const int j0 = ii[base + lane];
                cas_add(dt, j0, c * to_float(vv[base + lane]), vd[j0]);
            }
            base += n0;
        }
    } else {
        for (int e = 0; e < sl.L0; ++e) {
            const int n0 = __popc(__ballot_sync(kFull, e < len));
            if (e < lact) {
                const int j0 = ring_idx(ring, RING, sl, base + lane);
                cas_add(dt, j0, c * ring_val<VT>(ring, RING, sl, base + lane), vd[j0]);
            }
            base += n0;
        }
    }
}

// Warp roles of one CTA (tile b):
//   warp 0 (lane 0)  producer: streams the tile's bytes into the ring, at
//                    most kTileQ chunks ahead of the scatter;
//   warp 1           watcher: once every phase-1 warp of the CTA finished a
//                    chunk, one fence and a relaxed increment of the chunk's
//                    grid counter (several chunks share a fence); the lanes
//                    poll up to 32 counters at once and pass the chunks that
//                    are complete on the whole grid to the coefficient warps;
//   W1 warps         phase 1: partial dot products of slices, one FP32 L2
//                    reduction per segment;
//   NC warps         coefficients: for grid-complete chunks (chunk k by warp
//                    k mod NC), c_i of every segment from the complete r_i,
//                    into a shared-memory slot of CQ, and the proximity terms;
//   W2 warps         scatter: Delta_j += c_i a_ij; the box step at the end of
//                    each block.
// Every hand-off inside the CTA is an mbarrier of a ring of kTileQ slots
// (chunk k uses slot k mod kTileQ, phase parity (k / kTileQ) & 1): arrive
// releases and try_wait acquires at CTA scope, and a waiting warp sleeps in
// hardware instead of polling.  No role can run kTileQ chunks ahead of the
// scatter, so a slot's barrier never completes a phase its waiter has not
// seen yet.
template <typename VT>
__global__ void __launch_bounds__(1024, 1) k_tile_sweep(const TileArgs a) {
    if (a.st[0].stopped) return;   // uniform over the grid: nothing is touched
    extern __shared__ __align__(128) unsigned char smraw[];
    __shared__ volatile int abort_flag;
    __shared__ volatile int stage_piece[kTileMaxStages];
    __shared__ __align__(8) uint64_t bar_p1[kTileQ];   // W1 arrivals: phase 1 of chunk k done
    __shared__ __align__(8) uint64_t bar_g[kTileQ];    // 1 arrival: chunk k complete on the grid
    __shared__ __align__(8) uint64_t bar_c[kTileQ];    // 1 arrival: chunk k's coefficients in their slot
    __shared__ __align__(8) uint64_t bar_s[kTileQ];    // W2 arrivals: chunk k scattered
    __shared__ __align__(8) uint64_t bar_x;            // 1 arrival per block: its box step done
    __shared__ double prox_w[kTileMaxWarps];
    __shared__ int last_s;
    const int RING = a.stages * a.piece;
    unsigned char* ring = smraw;
    float* xt = reinterpret_cast<float*>(smraw + RING);
    float* dt = xt + a.tile_cap;
    int* scoff = reinterpret_cast<int*>(dt + a.tile_cap);   // K + 1 chunk offsets
    int* snsl = scoff + (a.K + 1);                          // K slice counts
    int* sblk = snsl + a.K;                                 // K blocks
    int* spref = sblk + a.K;                                // K + 1: slices before chunk k
    float* cbuf = reinterpret_cast<float*>(spref + a.K + 1);   // CQ x cstride coefficients
    uint64_t* full = reinterpret_cast<uint64_t*>(
        (reinterpret_cast<uintptr_t>(cbuf + (size_t)a.cq * a.cstride) + 15) & ~uintptr_t(15));
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
        const int* gns = a.nsl + (size_t)b * a.K;
        for (int k = tid; k <= a.K; k += blockDim.x) scoff[k] = gco[k];
        for (int k = tid; k < a.K; k += blockDim.x) {
            snsl[k] = gns[k];
            sblk[k] = a.chunk_blk[k];
        }
        if (tid == 0) {
            // a running slice index across the chunks: slice s of chunk k goes
            // to warp (spref[k] + s) mod W of a role, so every warp gets its
            // share of the slices however few a chunk holds
            int acc = 0;
            for (int k = 0; k < a.K; ++k) {
                spref[k] = acc;
                acc += gns[k];
            }
            spref[a.K] = acc;
        }
        if (tid < kTileMaxWarps) prox_w[tid] = 0.0;
        if (tid < kTileMaxStages) stage_piece[tid] = -1;
        if (tid == 0) {
            for (int s = 0; s < a.stages; ++s) tma::mbar_init(&full[s], 1);
            for (int q = 0; q < kTileQ; ++q) {
                tma::mbar_init(&bar_p1[q], W1);
                tma::mbar_init(&bar_g[q], 1);
                tma::mbar_init(&bar_c[q], 1);
                tma::mbar_init(&bar_s[q], W2);
            }
            tma::mbar_init(&bar_x, 1);
            abort_flag = 0;
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
        if (lane == 0) {
            // ---- producer
            long long st_t0 = TSTAT_CLOCK(), st_w = 0;
            (void)st_t0;
            const unsigned char* src = a.stream + a.base[b];
            const uint64_t pol = tma::policy_evict_first();
            const int npieces = (len_stream + a.piece - 1) >> ts;
            int issued = 0;
            int rel = 0;   // chunks whose scatter finished
            int jq = 0;    // chunk holding the last byte of the piece
#ifdef SUPPY_TILE_STATS
            int tr_k = 0;  // next chunk whose data is still to be issued
#endif
            bool ok = true;
            for (int q = 0; q < npieces && ok; ++q) {
                const int end = min((q + 1) << ts, len_stream);
                while (jq + 1 < a.K && scoff[jq + 1] < end) ++jq;
                // ring space (the stage's previous piece read by every role)
                // and at most kTileQ chunks between the scatter and the newest data
                const int need = (q >= a.stages) ? (q - a.stages + 1) << ts : 0;
                while (ok && (scoff[rel] < need || jq >= rel + kTileQ)) {
                    st_w -= TSTAT_CLOCK();
                    ok = tma::mbar_wait(&bar_s[rel % kTileQ], (rel / kTileQ) & 1, &abort_flag, limit);
                    st_w += TSTAT_CLOCK();
                    if (ok) ++rel;
                }
                if (!ok) {
                    give_up(3);
                    break;
                }
                const int s = q % a.stages;
                const uint32_t bytes = (uint32_t)(end - (q << ts));
#ifdef SUPPY_TILE_STATS
                while (tr_k < a.K && scoff[tr_k + 1] <= end) {
                    TTRACE(tr_k, 0);
                    ++tr_k;
                }
#endif
                stage_piece[s] = q;
                tma::mbar_arrive_expect_tx(&full[s], bytes);
                tma::bulk_g2s(ring + ((size_t)s << ts), src + (q << ts), bytes, &full[s], pol);
                issued = q + 1;
            }
            TSTAT_ADD(6, st_w);
            TSTAT_ADD(7, TSTAT_CLOCK() - st_t0);
            // copies in flight land before the CTA may leave
            volatile int never = 0;
            for (int q = (issued > a.stages ? issued - a.stages : 0); q < issued; ++q)
                tma::mbar_wait(&full[q % a.stages], (q / a.stages) & 1, &never, kTileDrainCycles);
        }
    } else if (warp == 1) {
        // ---- watcher
        long long st_t0 = TSTAT_CLOCK(), st_idle = 0;
        (void)st_t0;
        const unsigned P = gridDim.x;
        int sig = 0, done = 0;
        long long t0 = clock64();
        while (done < a.K) {
            bool prog = false;
            // local completions: the next chunks whose phase 1 is done here
            int nsig = sig;
            if (nsig < a.K) {
                bool got = true;
                if (lane == 0) got = mbar_try_wait_ns(&bar_p1[nsig % kTileQ], (nsig / kTileQ) & 1, 500);
                got = __shfl_sync(kFull, got, 0);
                if (got) {
                    ++nsig;
                    // more completed chunks share the fence
                    while (nsig < a.K && nsig < sig + 32) {
                        bool more = false;
                        if (lane == 0) more = mbar_try_wait_ns(&bar_p1[nsig % kTileQ], (nsig / kTileQ) & 1, 0);
                        if (!__shfl_sync(kFull, more, 0)) break;
                        ++nsig;
                    }
                }
            }
            if (nsig > sig) {
                if (lane < nsig - sig) TTRACE(sig + lane, 1);
                // the phase-1 warps' reductions, ordered before their
                // arrivals, reach the GPU before the counters move
                fence_acq_rel_gpu();
                if (lane < nsig - sig) red_add_u32_gpu(a.cnt + sig + lane, 1u);
                if (lane < nsig - sig) TTRACE(sig + lane, 2);
                sig = nsig;
                prog = true;
            }
            // grid completions: up to 32 counters at once
            if (done < sig) {
                const int j = done + lane;
                bool c = false;
                if (j < sig) c = ld_acquire_gpu(a.cnt + j) >= P;
                const unsigned m = __ballot_sync(kFull, c);
                const int nnew = (m == kFull) ? 32 : __ffs(~m) - 1;
                __syncwarp();
                if (nnew > 0) {
                    if (lane < nnew) TTRACE(done + lane, 3);
                    if (lane == 0)
                        for (int t = 0; t < nnew; ++t) tma::mbar_arrive(&bar_g[(done + t) % kTileQ]);
                    done += nnew;
                    prog = true;
                }
            }
            if (prog) {
                t0 = clock64();
            } else {
                st_idle += 1;
                if (abort_flag || *reinterpret_cast<volatile int*>(a.err) || clock64() - t0 > limit) {
                    if (lane == 0) give_up(3);
                    break;
                }
                if (sig >= a.K) __nanosleep(200);
            }
        }
        if (lane == 0) {
            TSTAT_ADD(8, st_idle);
            TSTAT_ADD(9, TSTAT_CLOCK() - st_t0);
        }
    } else if (warp <= 1 + W1) {
        // ---- phase 1: partial dot products of the tile's slices
        const int w1 = warp - 2;
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
                    ok = warp_bar_wait(&bar_x, (blk - 1) & 1, &abort_flag, a.err, limit);
                    if (!ok && lane == 0) give_up(3);
                }
            }
            const int c0 = scoff[k], c1 = scoff[k + 1];
            if (ok && c1 > c0) {
                for (int q = c0 >> ts; ok && q <= (c1 - 1) >> ts; ++q) {
                    const int s = q % a.stages;
                    bool w = true;
                    if (stage_piece[s] != q) {
                        const long long t0 = clock64();
                        int ns = 64;
                        while (stage_piece[s] != q) {
                            if (abort_flag || clock64() - t0 > limit) {
                                w = false;
                                break;
                            }
                            __nanosleep(ns);
                            ns = min(ns * 2, 1024);
                        }
                    }
                    if (w) w = tma::mbar_wait(&full[s], (q / a.stages) & 1, &abort_flag, limit);
                    ok = __all_sync(kFull, w);
                }
                if (!ok && lane == 0) give_up(3);
            }
            st_w += TSTAT_CLOCK();
            if (ok && c1 > c0) {
                const int nsl = snsl[k];
                const int rc = c0 % RING;
                for (int s = (w1 - spref[k] % W1 + W1) % W1; s < nsl; s += W1) {
                    int row, len;
                    const Slice sl = slice_at<VT>(ring, RING, rc, s, lane, &row, &len);
                    const float dot = slice_dot<VT>(ring, RING, sl, lane, len, xt);
                    if (lane < sl.nl) red_add_gpu(r_cur + (row & 0x7fffffff), dot);
                }
            }
            // every lane's reductions precede the warp's arrival
            __syncwarp();
            if (ok && lane == 0) tma::mbar_arrive(&bar_p1[k % kTileQ]);
        }
        if (lane == 0) {
            TSTAT_ADD(0, st_w);
            TSTAT_ADD(1, TSTAT_CLOCK() - st_t0);
        }
    } else if (warp <= 1 + W1 + NC) {
        // ---- coefficients of grid-complete chunks
        const int wc = warp - 2 - W1;
        double pacc = 0.0;
        bool ok = true;
        long long st_t0 = TSTAT_CLOCK(), st_w = 0;
        (void)st_t0;
        for (int k = wc; k < a.K && ok; k += NC) {
            const int slot = k % CQ;
            st_w -= TSTAT_CLOCK();
            // the slot's previous chunk is scattered, and chunk k is complete
            if (k >= CQ)
                ok = warp_bar_wait(&bar_s[(k - CQ) % kTileQ], ((k - CQ) / kTileQ) & 1, &abort_flag,
                                   a.err, limit);
            if (ok) ok = warp_bar_wait(&bar_g[k % kTileQ], (k / kTileQ) & 1, &abort_flag, a.err, limit);
            st_w += TSTAT_CLOCK();
            if (!ok) {
                if (lane == 0) give_up(3);
                break;
            }
            const int c0 = scoff[k], nsl = snsl[k];
            const int rc = c0 % RING;
            const double scale = a.blk_scale[sblk[k]];
            float* cb = cbuf + (size_t)slot * a.cstride;
            for (int s0 = 0; s0 < nsl; s0 += 4) {
                int row[4];
                bool has[4];
                float ri[4], li[4], ui[4], wi[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    has[u] = false;
                    row[u] = 0;
                    if (s0 + u < nsl) {
                        const uint2 d = *reinterpret_cast<const uint2*>(ring + wrap(rc + 8 * (s0 + u), RING));
                        const int nl = (int)(d.y & 63u);
                        const int sp = wrap(rc + 4 * (int)d.x, RING);
                        if (lane < nl) {
                            has[u] = true;
                            row[u] = *reinterpret_cast<const int*>(ring + wrap(sp + 4 * lane, RING));
                        }
                    }
                    if (has[u]) {
                        const int rw = row[u] & 0x7fffffff;
                        ri[u] = ld_relaxed_gpu(r_cur + rw);
                        li[u] = __ldg(a.l + rw);
                        ui[u] = __ldg(a.u + rw);
                        wi[u] = __ldg(a.wr + rw);
                    }
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (has[u]) {
                        const float dd = clampf(ri[u], li[u], ui[u]) - ri[u];
                        cb[(s0 + u) * 32 + lane] = a.lam * wi[u] * dd;
                        if (row[u] < 0) pacc += (double)dd * (double)dd * (double)wi[u] * scale;
                    }
                }
            }
            __syncwarp();
            if (lane == 0) {
                TTRACE(k, 4);
                tma::mbar_arrive(&bar_c[k % kTileQ]);
            }
        }
        pacc = warp_sum(pacc);
        if (lane == 0) {
            prox_w[wc] = pacc;
            TSTAT_ADD(2, st_w);
            TSTAT_ADD(3, TSTAT_CLOCK() - st_t0);
        }
    } else {
        // ---- scatter into Delta, and the box step at the end of each block
        const int w2 = warp - 2 - W1 - NC;
        const int t2 = tid - 32 * (2 + W1 + NC);   // 0 .. 32 W2 - 1
        bool ok = true;
        long long st_t0 = TSTAT_CLOCK(), st_w = 0;
        (void)st_t0;
        for (int k = 0; k < a.K; ++k) {
            const int blk = sblk[k];
            const int slot = k % CQ;
            st_w -= TSTAT_CLOCK();
            if (ok) {
                ok = warp_bar_wait(&bar_c[k % kTileQ], (k / kTileQ) & 1, &abort_flag, a.err, limit);
                if (!ok && lane == 0) give_up(3);
            }
            st_w += TSTAT_CLOCK();
            const int c0 = scoff[k], nsl = snsl[k];
            if (ok && nsl > 0) {
                const int rc = c0 % RING;
                const float* cb = cbuf + (size_t)slot * a.cstride;
                for (int s = (w2 - spref[k] % W2 + W2) % W2; s < nsl; s += W2) {
                    int row, len;
                    const Slice sl = slice_at<VT>(ring, RING, rc, s, lane, &row, &len);
                    const float c = (lane < sl.nl) ? cb[s * 32 + lane] : 0.f;
                    if (__any_sync(kFull, c != 0.f)) slice_scatter<VT>(ring, RING, sl, lane, len, c, dt);
                }
            }
            __syncwarp();
            if (lane == 0) {
                if (w2 == 0) TTRACE(k, 5);
                tma::mbar_arrive(&bar_s[k % kTileQ]);
            }
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
                if (t2 == 0 && !last) tma::mbar_arrive(&bar_x);
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

// Fill of the tile streams: one warp per slice writes the slice's table
// entry, its rows and lengths, and its values and tile-local indices step by
// step (lane j = the slice's j-th segment, longest first).
template <typename VT>
__global__ void k_tile_fill(const TileSliceRec* slices, long long nslices, const TileLaneRec* lanes,
                            const VT* val, const int* col, const unsigned short* local_of,
                            unsigned char* stream) {
    const long long w = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= nslices) return;
    const TileSliceRec r = slices[w];
    unsigned char* chunk = stream + r.chunk_start;
    if (lane == 0) {
        uint2 d;
        d.x = (unsigned)r.off4;
        d.y = (unsigned)r.nl | ((unsigned)r.E << 6);
        *reinterpret_cast<uint2*>(chunk + 8LL * r.sidx) = d;
    }
    unsigned char* sp = chunk + 4LL * r.off4;
    TileLaneRec ln = {0, 0, 0};
    if (lane < r.nl) {
        ln = lanes[r.first + lane];
        reinterpret_cast<int*>(sp)[lane] = ln.row_flag;
        reinterpret_cast<unsigned short*>(sp + 4 * r.nl)[lane] = (unsigned short)ln.len;
    }
    VT* dv = reinterpret_cast<VT*>(sp + ((6 * r.nl + 3) & ~3));
    unsigned short* di = reinterpret_cast<unsigned short*>(sp + ((6 * r.nl + 3) & ~3) + sizeof(VT) * r.E);
    const int L0 = __shfl_sync(kFull, ln.len, 0);
    int base = 0;
    for (int e = 0; e < L0; ++e) {
        const bool act = e < ln.len;
        const int n = __popc(__ballot_sync(kFull, act));
        if (act) {
            dv[base + lane] = val[ln.e0 + e];
            di[base + lane] = local_of[col[ln.e0 + e]];
        }
        base += n;
    }
}

using TileFn = void (*)(TileArgs);

TileFn tile_fn(suppy_dtype dt) {
    if (dt == SUPPY_F32) return k_tile_sweep<float>;
    if (dt == SUPPY_BF16) return k_tile_sweep<__nv_bfloat16>;
    return k_tile_sweep<__half>;
}

}  // namespace

size_t tile_smem_bytes(int ring_bytes, int tile_cap, int K, int stages, int cq, int cstride) {
    size_t b = (size_t)ring_bytes + 8 * (size_t)tile_cap + 4 * (4 * (size_t)K + 2) +
               4 * (size_t)cq * cstride;
    b = (b + 15) & ~(size_t)15;
    return b + 8 * (size_t)stages;
}

int tile_blocks_per_sm(suppy_dtype dt, int threads, size_t smem) {
    TileFn f = tile_fn(dt);
    if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, threads, smem) != cudaSuccess) return 0;
    return nb;
}

cudaError_t launch_tile_sweep(const TileArgs& a, suppy_dtype dt, int grid, size_t smem,
                              cudaStream_t s) {
    if (a.W1 < 1 || a.W2 < 1 || a.NC < 1 || 2 + a.W1 + a.NC + a.W2 > kTileMaxWarps ||
        a.cq < a.NC || a.cq > kTileMaxCQ || a.stages < 2 || a.stages > kTileMaxStages ||
        a.piece < 256 || (a.piece & (a.piece - 1)) || grid < 1)
        return cudaErrorInvalidValue;
    TileFn f = tile_fn(dt);
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid, 1, 1);
    cfg.blockDim = dim3(32 * (2 + a.W1 + a.NC + a.W2), 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, f, a);
}

cudaError_t launch_tile_fill(const TileSliceRec* slices, long long nslices, const TileLaneRec* lanes,
                             const void* val, suppy_dtype dt, const int* col,
                             const unsigned short* local_of, unsigned char* stream, cudaStream_t s) {
    if (nslices <= 0) return cudaSuccess;
    const int block = 256;
    const long long grid = (nslices * 32 + block - 1) / block;
    if (dt == SUPPY_F32)
        k_tile_fill<float><<<(unsigned)grid, block, 0, s>>>(slices, nslices, lanes,
                                                           static_cast<const float*>(val), col, local_of, stream);
    else if (dt == SUPPY_BF16)
        k_tile_fill<__nv_bfloat16><<<(unsigned)grid, block, 0, s>>>(
            slices, nslices, lanes, static_cast<const __nv_bfloat16*>(val), col, local_of, stream);
    else
        k_tile_fill<__half><<<(unsigned)grid, block, 0, s>>>(slices, nslices, lanes,
                                                            static_cast<const __half*>(val), col, local_of, stream);
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
        int tile, e0, len;
    };
    std::vector<Run> runs;
    runs.reserve((size_t)in.m * 8);
    std::vector<int> run_row;            // device row, bit 31 on the row's first run
    run_row.reserve((size_t)in.m * 8);
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
            runs.push_back(Run{tb, in.row_start[i] + t, e - t});
            run_row.push_back(t == 0 ? (int)((unsigned)i | 0x80000000u) : i);
            row_bytes[i] += 6 + (long long)(e - t) * (vs + 2);
            t = e;
        }
    }
    row_run[in.m] = (int)runs.size();
    if (runs.size() >= (size_t)INT32_MAX) {
        why = "tile plan: too many segments";
        return false;
    }
    // ---- row groups: group_rows consecutive rows of a block (neighbouring
    // rays of one direction for a ray-ordered matrix), the groups of a block in a
    // scattered order (a stride near ng / golden ratio, coprime to ng), so
    // that every chunk holds rays of every direction and position and every
    // tile gets about the same share of it
    const int kGroup = std::max(1, in.group_rows);
    const int nblk = (int)in.seg_start.size() - 1;
    std::vector<int> order(in.m);        // rows, group by group
    std::vector<int> gstart;             // positions in `order` where the groups start
    std::vector<int> gblk;
    {
        int pos = 0;
        for (int t = 0; t < nblk; ++t) {
            const int r0 = in.seg_start[t], r1 = in.seg_start[t + 1];
            const long long ng = (r1 - r0 + kGroup - 1) / kGroup;
            long long S = std::max<long long>(1, std::llround((double)ng * 0.6180339887498949));
            while (ng > 1 && std::gcd(S, ng) != 1) ++S;
            for (long long g = 0; g < ng; ++g) {
                const long long q = (g * S) % std::max<long long>(ng, 1);
                gstart.push_back(pos);
                gblk.push_back(t);
                for (int i = r0 + (int)q * kGroup; i < std::min(r1, r0 + (int)(q + 1) * kGroup); ++i)
                    order[pos++] = i;
            }
        }
        gstart.push_back(pos);
    }
    const int ngroups = (int)gblk.size();
    // ---- chunks: consecutive groups inside a block, about `target` stream
    // bytes per CTA each; halved while some tile's chunk exceeds max_chunk or
    // max_slices
    auto slice_bytes = [&](int nl, long long E) {
        return (((6LL * nl + 3) & ~3LL) + E * (vs + 2) + 15) & ~15LL;
    };
    // a slice stays well inside a chunk: at most a quarter of the largest
    // chunk (a slice of one segment may reach max_seg entries)
    const long long slice_cap = std::max<long long>(in.max_chunk / 4, slice_bytes(1, in.max_seg));
    long long target = (long long)in.chunk_target * P;
    for (int attempt = 0; attempt < 12; ++attempt) {
        std::vector<int> ck;      // group indices where the chunks start
        std::vector<int> cblk;
        {
            long long acc = 0;
            for (int g = 0; g < ngroups; ++g) {
                const bool new_blk = (g == 0) || gblk[g] != gblk[g - 1];
                if (new_blk || acc >= target) {
                    ck.push_back(g);
                    cblk.push_back(gblk[g]);
                    acc = 0;
                }
                for (int j = gstart[g]; j < gstart[g + 1]; ++j) acc += row_bytes[order[j]];
            }
            // blocks without rows still get a chunk (their box step)
            std::vector<char> seen(nblk, 0);
            for (int t : cblk) seen[t] = 1;
            std::vector<int> ck2, cb2;
            size_t p2 = 0;
            for (int t = 0; t < nblk; ++t) {
                if (!seen[t]) {
                    ck2.push_back(p2 < ck.size() ? ck[p2] : ngroups);
                    cb2.push_back(t);
                    continue;
                }
                while (p2 < ck.size() && cblk[p2] == t) {
                    ck2.push_back(ck[p2]);
                    cb2.push_back(t);
                    ++p2;
                }
            }
            ck.swap(ck2);
            cblk.swap(cb2);
        }
        const int K = (int)ck.size();
        ck.push_back(ngroups);
        if (K > in.max_chunks) {
            why = "tile plan: more chunks than the kernel's tables hold";
            return false;
        }
        // per (tile, chunk): the runs in group order, cut into slices of 32
        std::vector<int> nsl((size_t)P * K, 0);
        std::vector<long long> csize((size_t)P * K, 0);
        long long worst = 0;
        int worst_nsl = 0;
        std::vector<int> cnt(P, 0);
        std::vector<long long> ent(P, 0);
        for (int k = 0; k < K; ++k) {
            for (int p = 0; p < P; ++p) {
                cnt[p] = 0;
                ent[p] = 0;
            }
            std::vector<long long> body(P, 0);
            for (int g = ck[k]; g < ck[k + 1]; ++g)
                for (int j = gstart[g]; j < gstart[g + 1]; ++j) {
                    const int i = order[j];
                    for (int r = row_run[i]; r < row_run[i + 1]; ++r) {
                        const int p = runs[r].tile;
                        if (cnt[p] == 32 ||
                            (cnt[p] > 0 && slice_bytes(cnt[p] + 1, ent[p] + runs[r].len) > slice_cap)) {
                            body[p] += slice_bytes(cnt[p], ent[p]);
                            nsl[(size_t)p * K + k] += 1;
                            cnt[p] = 0;
                            ent[p] = 0;
                        }
                        cnt[p] += 1;
                        ent[p] += runs[r].len;
                    }
                }
            for (int p = 0; p < P; ++p) {
                if (cnt[p]) {
                    body[p] += slice_bytes(cnt[p], ent[p]);
                    nsl[(size_t)p * K + k] += 1;
                }
                const size_t q = (size_t)p * K + k;
                csize[q] = (((long long)nsl[q] * 8 + 15) & ~15LL) + body[p];
                worst = std::max(worst, csize[q]);
                worst_nsl = std::max(worst_nsl, nsl[q]);
            }
        }
        if (worst > in.max_chunk || worst_nsl > in.max_slices) {
            target /= 2;
            if (target < 1024) break;
            continue;
        }
        // ---- offsets
        out.K = K;
        out.chunk_blk = cblk;
        out.nsl = nsl;
        out.coff.assign((size_t)P * (K + 1), 0);
        out.base.assign(P, 0);
        out.max_chunk = (int)worst;
        out.max_slices = worst_nsl;
        long long tot = 0;
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
        // ---- slice and lane records (lanes of a slice longest first)
        out.slices.clear();
        out.lanes.clear();
        out.segments = (long long)runs.size();
        std::vector<std::vector<int>> pend((size_t)P);
        std::vector<long long> pend_ent(P, 0);
        std::vector<int> sidx(P, 0);
        std::vector<long long> dpos(P, 0);
        auto flush = [&](int p, int k) {
            std::vector<int>& v = pend[p];
            if (v.empty()) return;
            std::stable_sort(v.begin(), v.end(), [&](int x, int y) { return runs[x].len > runs[y].len; });
            TileSliceRec sr;
            sr.chunk_start = out.base[p] + out.coff[(size_t)p * (K + 1) + k];
            sr.sidx = sidx[p]++;
            sr.off4 = (int)(dpos[p] >> 2);
            sr.nl = (int)v.size();
            long long E = 0;
            for (int x : v) E += runs[x].len;
            sr.E = (int)E;
            sr.first = (int)out.lanes.size();
            sr.pad = 0;
            for (int x : v) {
                TileLaneRec lr;
                lr.row_flag = run_row[x];
                lr.e0 = runs[x].e0;
                lr.len = runs[x].len;
                out.lanes.push_back(lr);
            }
            dpos[p] += slice_bytes(sr.nl, E);
            out.slices.push_back(sr);
            v.clear();
            pend_ent[p] = 0;
        };
        for (int k = 0; k < K; ++k) {
            for (int p = 0; p < P; ++p) {
                sidx[p] = 0;
                dpos[p] = ((long long)nsl[(size_t)p * K + k] * 8 + 15) & ~15LL;
            }
            for (int g = ck[k]; g < ck[k + 1]; ++g)
                for (int j = gstart[g]; j < gstart[g + 1]; ++j) {
                    const int i = order[j];
                    for (int r = row_run[i]; r < row_run[i + 1]; ++r) {
                        const int p = runs[r].tile;
                        const int cntp = (int)pend[p].size();
                        if (cntp == 32 ||
                            (cntp > 0 && slice_bytes(cntp + 1, pend_ent[p] + runs[r].len) > slice_cap))
                            flush(p, k);
                        pend[p].push_back(r);
                        pend_ent[p] += runs[r].len;
                    }
                }
            for (int p = 0; p < P; ++p) flush(p, k);
        }
        return true;
    }
    why = "tile plan: no chunking keeps every tile's chunk within the ring";
    return false;
}

}  // namespace suppy

#ifdef SUPPY_TILE_STATS
extern "C" int suppy_tile_trace(unsigned long long* out) {
    return (int)cudaMemcpyFromSymbol(out, suppy::g_tile_trace, sizeof(unsigned long long) * 2 *
                                                                   suppy::kTileMaxChunks * 6);
}

extern "C" int suppy_tile_stats(unsigned long long* out16, int reset) {
    cudaError_t e = cudaMemcpyFromSymbol(out16, suppy::g_tile_stats, sizeof(unsigned long long) * 16);
    if (e != cudaSuccess || !reset) return (int)e;
    unsigned long long z[16] = {};
    return (int)cudaMemcpyToSymbol(suppy::g_tile_stats, z, sizeof(z));
}
#endif
