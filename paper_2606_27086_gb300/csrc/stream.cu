// TMA-fed streaming passes of the simultaneous projection sweep (Sec. 2.1.1,
// Eq. (3)) for one right-hand side.
//
// Each CTA owns a contiguous, nnz-balanced range of items (rows of the CSR
// copy, or columns of the CSC copy of A), hence one contiguous slice of the
// index and value arrays.  One producer lane streams that slice into an
// S-stage shared-memory ring of T-element tiles with 1-D bulk copies
// (cp.async.bulk, L2 evict-first) tracked by mbarriers; twenty-three consumer
// warps, split into groups of G lanes (one group per item), take batches of
// consecutive items in order from a shared counter and read them from the
// ring (four consecutive elements per lane and 16-byte access, or lane-
// interleaved elements), so HBM streaming runs ahead of the gathers of x (or
// of the coefficients) instead of waiting behind them.  A stage is refilled
// once every item element of its tile has been read (a group hands its
// elements back batch by batch as they reach registers, or, when it reads
// them again later, once the item is done).  G, T, S and the lane map are
// launch parameters (chosen per matrix, by measurement when the context is
// tuned).
//
// Items start at multiples of four elements and are zero-padded to a
// multiple of four (value 0, index 0), so a 16-byte ring access never holds
// two items' elements and the consumers need no per-element masking.
//
//  * row pass: r_i = <a_i, x>, d_i = clamp(r_i, l_i, u_i) - r_i, the
//    proximity term (compensated FP32 per thread, FP64 across threads and
//    CTAs), and either coef_i = lambda w_i d_i / ||a_i||^2 written
//    out (two-pass) or coef_i * a_i scatter-added into delta by address-
//    coalesced L2 reductions (one-pass);
//  * column pass: x_j <- clamp(x_j + sum_i a_ij coef_i, lo_j, hi_j).
//
// Every mbarrier wait is bounded (the launch's cycle budget, about two seconds
// of SM clock by default); on timeout the CTA records an error word, stops,
// lets its copies in flight land and returns.
#include <algorithm>

#include "common.cuh"
#include "tma.cuh"

namespace suppy {

#ifdef SUPPY_STREAM_STATS
// Measurement build only: cycle counters of the streaming skeleton (consumer
// waits for full tiles, releases, item work, rounds; producer waits for empty
// stages), summed over warps; slots 0-7 row pass, 8-15 column pass.
__device__ unsigned long long g_stream_stats[16];
#define SSTAT_CLOCK() clock64()
#define SSTAT_ADD(k, v) atomicAdd(&g_stream_stats[(k) + (a.coef_in ? 8 : 0)], (unsigned long long)(v))
#else
#define SSTAT_CLOCK() 0LL
#define SSTAT_ADD(k, v) ((void)0)
#endif

namespace {

constexpr int kMaxStages = 32;
// Copies already in flight always get this long to land before a CTA that gave
// up leaves (the launch's own wait budget may be shortened for diagnostics).
constexpr long long kDrainCycles = 4000000000LL;

using tma::bulk_g2s;
using tma::mbar_arrive;
using tma::mbar_arrive_expect_tx;
using tma::mbar_init;
using tma::policy_evict_first;

template <typename VT>
__device__ __forceinline__ float to_f(VT v) { return (float)v; }

// Ring of the CTA's slice: element g of the slice (counted from the aligned
// start Ea) lies in tile g / T, held by stage (g / T) % S at offset g % T;
// the stages are contiguous, so that position is g % (S T).  Groups of four
// elements starting at a multiple of four never straddle a tile and are
// 16-byte aligned in the ring.
template <typename VT>
struct Ring {
    const VT* val;
    const int* idx;
    int size;     // S * T elements
    __device__ __forceinline__ int pos(int g) const { return g % size; }
    __device__ __forceinline__ void step(int& p, int d) const {
        p += d;
        if (p >= size) p -= size;
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

// Hands ring space back: the padded elements [e0, e1) of the slice count
// toward their tiles, and the thread that completes a tile's count resets it
// and arrives on the stage's empty barrier, so the producer may refill it.
// Called by one lane of a group, after a __syncwarp over the group has
// ordered every lane's reads of those elements before it.
struct RingRelease {
    int* tile_done;
    uint64_t* empty;
    int S, ts, lo_r, hi_r;
    __device__ __forceinline__ void operator()(int e0, int e1) const {
        for (int k = e0 >> ts; k <= (e1 - 1) >> ts; ++k) {
            const int ov = min(e1, (k + 1) << ts) - max(e0, k << ts);
            const int s = k % S;
            const int target = min((k + 1) << ts, hi_r) - max(k << ts, lo_r);
            if (atomicAdd(&tile_done[s], ov) + ov == target) {
                tile_done[s] = 0;
                mbar_arrive(&empty[s]);
            }
        }
    }
};

// sum_e a_e * vec[idx_e] over the item's elements held in the ring, by the
// G lanes of one group reading four elements per 16-byte ring access.  The
// group walks the item in batches of 4G quads (uniform over the group):
// lane gl loads the quads qb + gl, qb + gl + G, qb + gl + 2G, qb + gl + 3G
// that exist (a missing quad gathers vec[0] with value 0), then issues their
// sixteen gathers together, so that a batch costs one gather latency.  With
// EARLY the group hands the batch's ring space back as soon as it sits in
// registers, while its gathers are in flight, so the producer can refill it
// meanwhile; without it each lane runs its own batches (the form that
// measured fastest for the row pass).
template <typename VT, int G, bool EARLY>
__device__ __forceinline__ float ring_dot(const Ring<VT>& r, int g0, int len, int gl,
                                          const float* __restrict__ vec, const RingRelease& rel) {
    const int nq = (len + 3) >> 2;
    float acc0 = 0.f, acc1 = 0.f;
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    const int4 zi = make_int4(0, 0, 0, 0);
    auto gather = [&](const int4& c) {
        return make_float4(__ldg(vec + c.x), __ldg(vec + c.y), __ldg(vec + c.z), __ldg(vec + c.w));
    };
    auto fma4 = [&](const float4& v, const float4& x) {
        acc0 = fmaf(v.x, x.x, acc0);
        acc1 = fmaf(v.y, x.y, acc1);
        acc0 = fmaf(v.z, x.z, acc0);
        acc1 = fmaf(v.w, x.w, acc1);
    };
    if constexpr (!EARLY) {
        // no hand-back per batch: each lane runs its own full batches, then
        // one batch of the one to three quads it has left
        int q = gl;
        int p = r.pos(g0 + 4 * gl);
        for (; q + 3 * G < nq; q += 4 * G) {
            float4 v[4];
            int4 c[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                v[k] = Quad<VT>::load(r.val + p);
                c[k] = *reinterpret_cast<const int4*>(r.idx + p);
                r.step(p, 4 * G);
            }
            float4 x[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) x[k] = gather(c[k]);
#pragma unroll
            for (int k = 0; k < 4; ++k) fma4(v[k], x[k]);
        }
        if (q < nq) {
            float4 v[3] = {z, z, z};
            int4 c[3] = {zi, zi, zi};
#pragma unroll
            for (int k = 0; k < 3; ++k)
                if (q + k * G < nq) {
                    v[k] = Quad<VT>::load(r.val + p);
                    c[k] = *reinterpret_cast<const int4*>(r.idx + p);
                    r.step(p, G * 4);
                }
            float4 x[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) x[k] = gather(c[k]);
#pragma unroll
            for (int k = 0; k < 3; ++k) fma4(v[k], x[k]);
        }
        return acc0 + acc1;
    } else {
        for (int qb = 0; qb < nq; qb += 4 * G) {
            float4 v[4];
            int4 c[4];
            if (qb + 4 * G <= nq) {
                int p = r.pos(g0 + 4 * (qb + gl));
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    v[k] = Quad<VT>::load(r.val + p);
                    c[k] = *reinterpret_cast<const int4*>(r.idx + p);
                    r.step(p, 4 * G);
                }
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int q = qb + gl + k * G;
                    if (q < nq) {
                        const int p = r.pos(g0 + 4 * q);
                        v[k] = Quad<VT>::load(r.val + p);
                        c[k] = *reinterpret_cast<const int4*>(r.idx + p);
                    } else {
                        v[k] = z;
                        c[k] = zi;
                    }
                }
            }
            // every lane's ring reads of the batch are done; the hand-back goes
            // after the gathers are issued, so its shared-memory atomics overlap
            // their latency instead of delaying them
            __syncwarp(gmask_of<G>(threadIdx.x & 31));
            float4 x[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) x[k] = gather(c[k]);
            if (gl == 0) rel(g0 + 4 * qb, g0 + 4 * min(qb + 4 * G, nq));
#pragma unroll
            for (int k = 0; k < 4; ++k) fma4(v[k], x[k]);
        }
        return acc0 + acc1;
    }
}

// Lane-interleaved form of ring_dot: lane gl takes the elements gl, gl + G,
// gl + 2G, ... of the item, U per batch (batches of U G elements, uniform
// over the group), with 4-byte ring reads.  One gather instruction of a group
// then reads G consecutive elements of the item (and the group beside it the
// same positions of the next item), which for the rows of a ray and the
// columns of neighbouring pixels lie in far fewer cache lines than the
// 4G-element spread of one quad-form instruction.  Masked-off positions are
// not read.  EARLY as in ring_dot (the last batch also hands back the padding).
template <typename VT, int G, int U, bool EARLY>
__device__ __forceinline__ float ring_dot_il(const Ring<VT>& r, int g0, int len, int gl,
                                             const float* __restrict__ vec, const RingRelease& rel) {
    float acc0 = 0.f, acc1 = 0.f;
    const int p0 = r.pos(g0);
    const int lenp = (len + 3) & ~3;
    const bool wraps = p0 + len > r.size;   // the item wraps around the end of the ring
    for (int e = 0; e < len; e += U * G) {
        int c[U];
        float av[U], xv[U];
        if (!wraps && e + U * G <= len) {
            const VT* v = r.val + p0 + e + gl;
            const int* ix = r.idx + p0 + e + gl;
#pragma unroll
            for (int t = 0; t < U; ++t) {
                c[t] = ix[t * G];
                av[t] = to_f(v[t * G]);
            }
        } else {
            // the item's last batch (or one that wraps around the ring's
            // end): slots four at a time, only while they hold elements
            int p = p0 + e + gl;
            if (p >= r.size) p -= r.size;
            for (int t0 = 0; t0 < U && e + t0 * G < len; t0 += 4) {   // uniform over the group
                int cc[4];
                float aa[4], xx[4];
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    const bool in = e + gl + (t0 + t) * G < len;
                    cc[t] = in ? r.idx[p] : 0;
                    aa[t] = in ? to_f(r.val[p]) : 0.f;
                    r.step(p, G);
                }
#pragma unroll
                for (int t = 0; t < 4; ++t) xx[t] = __ldg(vec + cc[t]);
                acc0 = fmaf(aa[0], xx[0], acc0);
                acc1 = fmaf(aa[1], xx[1], acc1);
                acc0 = fmaf(aa[2], xx[2], acc0);
                acc1 = fmaf(aa[3], xx[3], acc1);
            }
            if constexpr (EARLY) {
                __syncwarp(gmask_of<G>(threadIdx.x & 31));
                if (gl == 0) rel(g0 + e, g0 + (e + U * G >= len ? lenp : e + U * G));
            }
            continue;
        }
        if constexpr (EARLY) __syncwarp(gmask_of<G>(threadIdx.x & 31));
#pragma unroll
        for (int t = 0; t < U; ++t) xv[t] = __ldg(vec + c[t]);
        if constexpr (EARLY) {
            // after the gathers are issued (see ring_dot)
            if (gl == 0) rel(g0 + e, g0 + (e + U * G >= len ? lenp : e + U * G));
        }
#pragma unroll
        for (int t = 0; t < U; t += 2) {
            acc0 = fmaf(av[t], xv[t], acc0);
            acc1 = fmaf(av[t + 1], xv[t + 1], acc1);
        }
    }
    return acc0 + acc1;
}

// U: elements a lane holds per batch of the lane-interleaved form (the row
// pass keeps more per-item state live and takes fewer, spilling none).
template <typename VT, int G, int MAP, int U, bool EARLY>
__device__ __forceinline__ float item_dot(const Ring<VT>& r, int g0, int len, int gl,
                                          const float* __restrict__ vec, const RingRelease& rel) {
    if constexpr (MAP == 1) return ring_dot_il<VT, G, U, EARLY>(r, g0, len, gl, vec, rel);
    else return ring_dot<VT, G, EARLY>(r, g0, len, gl, vec, rel);
}

// Producer / consumer skeleton.  Consumer warps hold 32/G groups of G lanes.
// A warp takes the next 32/G consecutive items of the CTA's range from a
// shared counter (one group per item), so all warps move through the slice
// together and the ring holds only the items in work plus the prefetched
// tiles, however the item costs vary.  A stage is released when the padded
// elements of its tile that belong to finished items add up to all of the
// tile's item elements: the group that completes the count resets it and
// arrives on the stage's empty barrier.  work(item, len, g0, ring, gl)
// returns the FP64 proximity contribution of the item (one lane), else 0;
// work.prefetch(next item or -1) loads the next batch's per-item operands
// and work.advance() makes them current.  A warp takes its next batch before
// working on the current one, so those loads overlap the work.
template <typename VT, int G, class Work>
__device__ double stream_items(const StreamArgs& a, Work& work) {
    extern __shared__ __align__(128) unsigned char smraw[];
    __shared__ volatile int abort_flag;
    __shared__ int next_grab;                         // items handed out (from I0)
    __shared__ volatile int stage_tile[kMaxStages];   // tile issued into each stage
    __shared__ int tile_done[kMaxStages];             // finished item elements of it
    const int T = a.tile;
    const int S = a.stages;
    const int RING = S * T;
    const int ts = 31 - __clz(T);
    VT* sval = reinterpret_cast<VT*>(smraw);
    int* sidx = reinterpret_cast<int*>(smraw + (size_t)RING * sizeof(VT));
    uint64_t* full = reinterpret_cast<uint64_t*>(sidx + RING);
    uint64_t* empty = full + S;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int GPW = 32 / G;
    const int I0 = a.cta_items[blockIdx.x], I1 = a.cta_items[blockIdx.x + 1];
    double acc = 0.0;
    if (I0 >= I1) return 0.0;   // uniform over the CTA
    const long long E0 = a.info[I0].x;
    const int2 last = a.info[I1 - 1];
    const long long Ea = E0 & ~7LL;
    // the items' padded elements cover [lo_r, hi_r) of the slice, contiguously
    const int lo_r = (int)(E0 - Ea);
    const int hi_r = (int)((long long)last.x + ((last.y + 3) & ~3) - Ea);
    const int K = (hi_r + T - 1) >> ts;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
            stage_tile[s] = -1;
            tile_done[s] = 0;
        }
        next_grab = 0;
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
            long long st_t0 = SSTAT_CLOCK(), st_wait = 0;
            (void)st_t0;
            for (int k = 0, s = 0, ph = 0; k < K; ++k) {
                const long long tw = SSTAT_CLOCK();
                if (k >= S && !tma::mbar_wait(&empty[s], (ph - 1) & 1, &abort_flag, a.wait_cycles)) {
                    abort_flag = 1;
                    atomicExch(a.err, 1);
                    break;
                }
                st_wait += SSTAT_CLOCK() - tw;
                stage_tile[s] = k;
                mbar_arrive_expect_tx(&full[s], bytes_v + bytes_i);
                bulk_g2s(sval + (size_t)s * T, gval + Ea + (long long)k * T, bytes_v, &full[s], pol);
                bulk_g2s(sidx + (size_t)s * T, a.idx + Ea + (long long)k * T, bytes_i, &full[s], pol);
                issued = k + 1;
                if (++s == S) {
                    s = 0;
                    ++ph;
                }
            }
            SSTAT_ADD(6, st_wait);
            SSTAT_ADD(7, SSTAT_CLOCK() - st_t0);
            if (abort_flag) {
                // let the copies in flight land before the CTA leaves
                volatile int never = 0;
                for (int k = (issued > S ? issued - S : 0); k < issued; ++k)
                    tma::mbar_wait(&full[k % S], (k / S) & 1, &never, kDrainCycles);
            }
        }
    } else {
        const Ring<VT> ring{sval, sidx, RING};
        const int gw = lane / G, gl = lane % G;
        const int nitems = I1 - I0;
        bool ok = true;
        // tile k is in the ring once its stage holds it and the stage's
        // barrier completed the phase of that fill
        auto wait_tile = [&](int k) {
            const int s = k % S;
            if (stage_tile[s] != k) {
                const long long t0 = clock64();
                while (stage_tile[s] != k) {
                    if (abort_flag || clock64() - t0 > a.wait_cycles) return false;
                    __nanosleep(64);
                }
            }
            return tma::mbar_wait(&full[s], (k / S) & 1, &abort_flag, a.wait_cycles);
        };
        const RingRelease rel{tile_done, empty, S, ts, lo_r, hi_r};
        auto grab = [&]() {
            int b = 0;
            if (lane == 0) b = atomicAdd(&next_grab, GPW);
            return __shfl_sync(0xffffffffu, b, 0);
        };
        constexpr int BIG = 0x7fffffff;
        long long st_t0 = SSTAT_CLOCK(), st_full = 0, st_rel = 0, st_work = 0, st_rounds = 0;
        (void)st_t0;
        int nb = grab();
        int2 nxt = (nb + gw < nitems) ? a.info[I0 + nb + gw] : make_int2(0, 0);
        work.prefetch(nb + gw < nitems ? I0 + nb + gw : -1);
        while (ok && nb < nitems) {
            const bool valid = nb + gw < nitems;
            const int i = I0 + nb + gw;
            const int2 inf = nxt;
            work.advance();
            nb = grab();
            nxt = (nb + gw < nitems) ? a.info[I0 + nb + gw] : make_int2(0, 0);
            work.prefetch(nb + gw < nitems ? I0 + nb + gw : -1);
            const bool has = valid && inf.y > 0;
            if (valid && inf.y == 0 && gl == 0) work.empty(i);
            const int g0 = (int)((long long)inf.x - Ea);
            int kb = BIG, ke = -1;
            if (has) {
                kb = g0 >> ts;
                ke = (g0 + inf.y - 1) >> ts;
            }
            kb = __reduce_min_sync(0xffffffffu, kb);
            ke = __reduce_max_sync(0xffffffffu, ke);
            if (ke < 0) continue;   // only empty items in this batch
            const long long t2 = SSTAT_CLOCK();
            for (int k = kb; ok && k <= ke; ++k) ok = __all_sync(0xffffffffu, wait_tile(k));
            const long long t3 = SSTAT_CLOCK();
            if (!ok) break;
            if (has) acc += work(i, inf.y, g0, ring, gl, rel);
            __syncwarp();
            const long long t4 = SSTAT_CLOCK();
            // hand the group's padded elements back (a work that reads the
            // ring only once did so batch by batch)
            if (!Work::kEarly && has && gl == 0) rel(g0, g0 + ((inf.y + 3) & ~3));
            st_full += t3 - t2;
            st_work += t4 - t3;
            st_rel += SSTAT_CLOCK() - t4;
            st_rounds += 1;
        }
        if (lane == 0) {
            SSTAT_ADD(0, 1);
            SSTAT_ADD(1, st_full);
            SSTAT_ADD(2, st_rel);
            SSTAT_ADD(3, st_work);
            SSTAT_ADD(4, st_rounds);
            SSTAT_ADD(5, SSTAT_CLOCK() - st_t0);
        }
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
template <typename VT, int G, int SCAT, int MAP>
struct RowWork {
    // the scatter reads the item's ring elements a second time: they go back
    // only once the item is done; otherwise batch by batch, as they are read
    // (FP32 values: with 16-bit values the extra state spills and the BF16
    // row pass measured slower, 0.214 against 0.193 ms on CT 512x512)
    static constexpr bool kEarly = (SCAT == 0 && sizeof(VT) == 4);
    const StreamArgs& a;
    float li = 0.f, ui = 0.f, w = 0.f;      // current round's bounds and weight
    float nl = 0.f, nu = 0.f, nw = 0.f;     // next round's
    // the row multiplier of the coefficient (coef_mul) or of the proximity
    // term (prox_mul): a pass sets at most one of them
    float m = 1.f, nm = 1.f;
    // the row scatters into the column-major accumulator (a.rowT)
    bool tr = false, ntr = false;
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
            const float* mp = a.coef_mul ? a.coef_mul : a.prox_mul;
            if (mp) nm = __ldg(mp + i);
            if (a.rowT) ntr = __ldg(a.rowT + i) != 0;
        }
    }
    __device__ void advance() {
        li = nl;
        ui = nu;
        w = nw;
        m = nm;
        tr = ntr;
    }
    __device__ void empty(int) {}   // an empty row: no coefficient, no proximity term
    __device__ double operator()(int i, int len, int g0, const Ring<VT>& r, int gl,
                                 const RingRelease& rel) {
        const unsigned gm = gmask_of<G>(threadIdx.x & 31);
        // a row running down the image reads the column-major copy of x (its
        // stored indices are column-major then) in the two-pass row pass; in
        // the patch numbering every row reads the copy in its own layout
        const float* xs = (a.xT && tr) ? a.xT : (a.xW ? a.xW : a.x);
        float dot = item_dot<VT, G, MAP, 12, kEarly>(r, g0, len, gl, xs, rel);
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) dot += __shfl_xor_sync(gm, dot, o);
        const float d = clampf(dot, li, ui) - dot;
        const float coef = a.lam * w * d * (a.coef_mul ? m : 1.f);
        if (SCAT == 0) {
            if (a.coef && gl == 0) a.coef[i] = coef;
        } else if (coef != 0.f) {
            // lane-strided over the elements: consecutive lanes, consecutive
            // columns (column-major ones for a row running down the image, or
            // neighbouring pixels of one patch in the patch numbering)
            float* dst = tr ? a.deltaT : a.delta;
            // the accumulator position of column j: the stored index itself
            // (row-major, or a patch position in the patch numbering), or
            // the column-major position for a row running down the image
            const bool cm = SCAT == 1 && tr && !a.patch;
            auto at = [&](int j) {
                return dst + (cm ? transposed_index(j, a.recipW, a.imgW, a.imgH) : j);
            };
            const int p0 = r.pos(g0);
            if (p0 + len <= r.size) {
                // the item does not wrap around the ring's end: four
                // elements per lane at a time, plain offsets
                const VT* v = r.val + p0;
                const int* ix = r.idx + p0;
                int t = gl;
                for (; t + 3 * G < len; t += 4 * G) {
                    int c[4];
                    float av[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        c[u] = ix[t + u * G];
                        av[u] = to_f(v[t + u * G]);
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) atomicAdd(at(c[u]), coef * av[u]);
                }
                for (; t < len; t += G) atomicAdd(at(ix[t]), coef * to_f(v[t]));
            } else {
                int p = r.pos(g0 + gl);
                for (int t = gl; t < len; t += G) {
                    atomicAdd(at(r.idx[p]), coef * to_f(r.val[p]));
                    r.step(p, G);
                }
            }
        }
        if (gl == 0) kahan_add(d * d * w * (a.prox_mul ? m : 1.f));
        return 0.0;
    }
};

template <typename VT, int G, int SCAT, int MAP>
__global__ void __launch_bounds__(kStreamThreads, 1) k_rows_tma(const StreamArgs a) {
    if (a.check_stop && a.st[0].stopped) return;
    RowWork<VT, G, SCAT, MAP> work{a};
    stream_items<VT, G>(a, work);
    cta_sum_to(work.total(), a.pp + blockIdx.x);
}

// Column pass of the two-pass sweep (B = 1).
template <typename VT, int G, int MAP>
struct ColWork {
    static constexpr bool kEarly = true;
    const StreamArgs& a;
    float xj = 0.f, lo = 0.f, hi = 0.f, z = 1.f;
    float nx = 0.f, nlo = 0.f, nhi = 0.f, nz = 1.f;
    __device__ void prefetch(int j) {
        if (j >= 0) {
            const int bj = (a.box_len == 1) ? 0 : j;
            nx = a.xw[j];   // owned by this group alone during the pass
            nlo = __ldg(a.lo + bj);
            nhi = __ldg(a.hi + bj);
            if (a.zc) nz = __ldg(a.zc + j);
        }
    }
    __device__ void advance() {
        xj = nx;
        lo = nlo;
        hi = nhi;
        z = nz;
    }
    // an empty column: the box step alone (the perturbation may have left x_j
    // outside the box); in accumulate mode its sum is 0
    __device__ void empty(int j) {
        if (a.delta_out) a.delta_out[j] = 0.f;
        else a.xw[j] = clampf(xj, lo, hi);
    }
    __device__ double operator()(int j, int len, int g0, const Ring<VT>& r, int gl,
                                 const RingRelease& rel) {
        const unsigned gm = gmask_of<G>(threadIdx.x & 31);
        float s = item_dot<VT, G, MAP, sizeof(VT) == 4 ? 16 : 12, true>(r, g0, len, gl, a.coef_in, rel);
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) s += __shfl_xor_sync(gm, s, o);
        if (a.zc) s *= z;
        if (gl == 0) {
            if (a.delta_out) a.delta_out[j] = s;
            else a.xw[j] = clampf(xj + s, lo, hi);
        }
        return 0.0;
    }
};

template <typename VT, int G, int MAP>
__global__ void __launch_bounds__(kStreamThreads, 1) k_cols_tma(const StreamArgs a) {
    if (a.epi.st[0].stopped) return;   // the row pass left no coefficients
    ColWork<VT, G, MAP> work{a};
    stream_items<VT, G>(a, work);
    __syncthreads();
    if (a.epi.last_seg && a.ticket) {
        // the last CTA to finish runs the sweep epilogue: every CTA of the
        // launch has read the stop flag by then, so the flag it may set is
        // seen by the next launch only
        __shared__ bool last;
        __threadfence();
        if (threadIdx.x == 0) last = atomicAdd(a.ticket, 1u) == gridDim.x - 1;
        __syncthreads();
        if (last) {
            __threadfence();
            sweep_epilogue(a.epi);
            if (threadIdx.x == 0) *a.ticket = 0u;
        }
    } else if (blockIdx.x == 0 && !a.epi.last_seg) {
        // CTA 0 also accumulates the row pass's proximity partials of this
        // block (the last block's are summed by its epilogue)
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

template <typename VT, int MAP>
StreamFn pick_rows(int G, int scat) {
    switch (G) {
        case 4: return scat ? k_rows_tma<VT, 4, 1, MAP> : k_rows_tma<VT, 4, 0, MAP>;
        case 8: return scat ? k_rows_tma<VT, 8, 1, MAP> : k_rows_tma<VT, 8, 0, MAP>;
        case 16: return scat ? k_rows_tma<VT, 16, 1, MAP> : k_rows_tma<VT, 16, 0, MAP>;
        default: return scat ? k_rows_tma<VT, 32, 1, MAP> : k_rows_tma<VT, 32, 0, MAP>;
    }
}

template <typename VT, int MAP>
StreamFn pick_cols(int G) {
    switch (G) {
        case 4: return k_cols_tma<VT, 4, MAP>;
        case 8: return k_cols_tma<VT, 8, MAP>;
        case 16: return k_cols_tma<VT, 16, MAP>;
        default: return k_cols_tma<VT, 32, MAP>;
    }
}

template <typename VT>
StreamFn pick_rows_map(int G, int scat, int map) {
    return map ? pick_rows<VT, 1>(G, scat) : pick_rows<VT, 0>(G, scat);
}

template <typename VT>
StreamFn pick_cols_map(int G, int map) {
    return map ? pick_cols<VT, 1>(G) : pick_cols<VT, 0>(G);
}

StreamFn rows_fn(suppy_dtype dt, int G, int scat, int map) {
    if (dt == SUPPY_F32) return pick_rows_map<float>(G, scat, map);
    if (dt == SUPPY_BF16) return pick_rows_map<__nv_bfloat16>(G, scat, map);
    return pick_rows_map<__half>(G, scat, map);
}

StreamFn cols_fn(suppy_dtype dt, int G, int map) {
    if (dt == SUPPY_F32) return pick_cols_map<float>(G, map);
    if (dt == SUPPY_BF16) return pick_cols_map<__nv_bfloat16>(G, map);
    return pick_cols_map<__half>(G, map);
}

}  // namespace

size_t stream_smem_bytes(suppy_dtype dt, int tile, int stages) {
    const size_t vsz = (dt == SUPPY_F32) ? 4 : 2;
    return (size_t)stages * tile * (vsz + 4) + 2 * (size_t)stages * sizeof(uint64_t);
}

// Most stages of T elements that fit the dynamic shared-memory budget.
int stream_stages_for(suppy_dtype dt, int tile) {
    constexpr size_t kBudget = 220 * 1024;
    const size_t vsz = (dt == SUPPY_F32) ? 4 : 2;
    const size_t per = (size_t)tile * (vsz + 4) + 2 * sizeof(uint64_t);
    return (int)std::min<size_t>(kMaxStages, kBudget / per);
}

int stream_max_item(int tile, int stages) { return (stages - 1) * tile; }

#ifdef SUPPY_STREAM_STATS
cudaError_t stream_stats_read(unsigned long long* out16, int reset) {
    cudaError_t e = cudaMemcpyFromSymbol(out16, g_stream_stats, sizeof(unsigned long long) * 16);
    if (e != cudaSuccess || !reset) return e;
    unsigned long long z[16] = {};
    return cudaMemcpyToSymbol(g_stream_stats, z, sizeof(z));
}
#endif

static cudaError_t launch_stream(StreamFn f, const StreamArgs& a, suppy_dtype dt, int grid,
                                 cudaStream_t s) {
    if (a.stages < 2 || a.stages > kMaxStages || a.tile < 64 || (a.tile & (a.tile - 1)))
        return cudaErrorInvalidValue;
    const size_t smem = stream_smem_bytes(dt, a.tile, a.stages);
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    f<<<grid, kStreamThreads, smem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_rows_tma(const StreamArgs& a, suppy_dtype dt, int G, int scat, int map, int grid,
                            cudaStream_t s) {
    return launch_stream(rows_fn(dt, G, scat, map), a, dt, grid, s);
}

cudaError_t launch_cols_tma(const StreamArgs& a, suppy_dtype dt, int G, int map, int grid,
                            cudaStream_t s) {
    return launch_stream(cols_fn(dt, G, map), a, dt, grid, s);
}

int stream_blocks_per_sm(suppy_dtype dt, int tile, int stages) {
    const size_t smem = stream_smem_bytes(dt, tile, stages);
    StreamFn f = rows_fn(dt, 32, 1, 0);
    if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, kStreamThreads, smem) != cudaSuccess)
        return 0;
    return nb;
}

}  // namespace suppy

#ifdef SUPPY_STREAM_STATS
extern "C" int suppy_stream_stats(unsigned long long* out16, int reset) {
    return (int)suppy::stream_stats_read(out16, reset);
}
#endif
