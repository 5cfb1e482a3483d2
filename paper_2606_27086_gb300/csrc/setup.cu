// Setup kernels: input validation, packing A into the device layout
// (values converted to the storage dtype), FP64 row norms ||a_i||^2 (the
// denominator of Eq. (2)), kept-row counts and the weights w_i / ||a_i||^2 of
// the simultaneous or block-iterative step (Sec. 2.1.1), the zero-row check,
// bound permutation, the box projection of the initial point and the column
// means c = S^T 1 / rows(S) of the mean-dose objective (Sec. 2.3.3).
#include "common.cuh"

namespace suppy {
namespace {

// flags bits (kF16Over: a magnitude above FP16's largest finite value)
constexpr int kBadRowPtr = 1, kBadCol = 2, kBadVal = 4, kF16Over = 8;

// With err2 set, also the squared rounding-error bounds of storing the values
// in FP16 and in BF16, summed over the entries: err2[0] += max(2^-11 |v|,
// 2^-25)^2 (unit roundoff 2^-11 in the normal range, half the subnormal
// spacing below it), err2[1] += (2^-8 v)^2 (BF16 keeps FP32's range).
__global__ void k_validate_csr(const int* rp, const int* col, const float* val, int m, int n,
                               long long nnz, int* flags, double* err2) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (long long i = t0; i < m; i += stride) {
        const int a = rp[i], b = rp[i + 1];
        if (a > b || a < 0 || (long long)b > nnz) atomicOr(flags, kBadRowPtr);
    }
    if (t0 == 0 && (rp[0] != 0 || (long long)rp[m] != nnz)) atomicOr(flags, kBadRowPtr);
    double e16 = 0.0, ebf = 0.0;
    for (long long e = t0; e < nnz; e += stride) {
        const int c = col[e];
        if (c < 0 || c >= n) atomicOr(flags, kBadCol);
        const float v = fabsf(val[e]);
        if (!isfinite(v)) {
            atomicOr(flags, kBadVal);
        } else if (err2) {
            if (v > 65504.f) atomicOr(flags, kF16Over);
            const double a = fmax(0x1p-11 * (double)v, v != 0.f ? 0x1p-25 : 0.0);
            const double b = 0x1p-8 * (double)v;
            e16 += a * a;
            ebf += b * b;
        }
    }
    if (err2) {
        __shared__ double s16[8], sbf[8];
        e16 = warp_sum(e16);
        ebf = warp_sum(ebf);
        const int w = threadIdx.x >> 5;
        if ((threadIdx.x & 31) == 0) {
            s16[w] = e16;
            sbf[w] = ebf;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            double a = 0.0, b = 0.0;
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
                a += s16[k];
                b += sbf[k];
            }
            atomicAdd(err2, a);
            atomicAdd(err2 + 1, b);
        }
    }
}

__global__ void k_validate_vec(const float* v, long long len, int allow_inf, int* flags,
                               int bit) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < len;
         i += (long long)gridDim.x * blockDim.x) {
        const float f = v[i];
        if (isnan(f) || (!allow_inf && isinf(f))) atomicOr(flags, bit);
    }
}

__global__ void k_validate_pair(const float* lo, const float* hi, long long len, int* flags,
                                int bit) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < len;
         i += (long long)gridDim.x * blockDim.x) {
        if (!(lo[i] <= hi[i])) atomicOr(flags, bit);
    }
}

template <typename VT>
__device__ __forceinline__ VT to_store(float v);
template <>
__device__ __forceinline__ float to_store<float>(float v) { return v; }
template <>
__device__ __forceinline__ __nv_bfloat16 to_store<__nv_bfloat16>(float v) {
    return __float2bfloat16_rn(v);
}
template <>
__device__ __forceinline__ __half to_store<__half>(float v) { return __float2half_rn(v); }

template <typename VT>
__device__ __forceinline__ float from_store(VT v);
template <>
__device__ __forceinline__ float from_store<float>(float v) { return v; }
template <>
__device__ __forceinline__ float from_store<__nv_bfloat16>(__nv_bfloat16 v) {
    return __bfloat162float(v);
}
template <>
__device__ __forceinline__ float from_store<__half>(__half v) { return __half2float(v); }

// One warp per device row i (source row perm[i]): copy columns, convert
// values to the storage type, and accumulate the FP64 squared norm of the
// stored values.
template <typename VT>
__global__ void k_pack(const int* rp, const int* col, const float* val, const int* perm,
                       const int2* rinfo, int m, int* pcol, VT* pval, double* rho) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < m; i += warps) {
        const int src = perm ? perm[i] : i;
        const int a = rp[src], len = rp[src + 1] - a;
        const int2 ri = rinfo[i];
        double s = 0.0;
        for (int e = lane; e < len; e += 32) {
            const VT v = to_store<VT>(val[a + e]);
            pcol[ri.x + e] = col[a + e];
            pval[ri.x + e] = v;
            const double f = (double)from_store<VT>(v);
            s += f * f;
        }
        s = warp_sum(s);
        if (lane == 0) rho[i] = s;
    }
}

// CSC copy of the packed rows: entry e of device row i goes to position
// pos[e] (a stable counting sort by column computed on the host), carrying
// its row index and its stored value.
template <typename VT>
__global__ void k_csc_fill(const int2* rinfo, int m, const VT* pval, const int* pos, int* ridx,
                           VT* cval) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < m; i += warps) {
        const int2 ri = rinfo[i];
        for (int e = lane; e < ri.y; e += 32) {
            const int p = pos[ri.x + e];
            ridx[p] = i;
            cval[p] = pval[ri.x + e];
        }
    }
}

__global__ void k_count_kept(const double* rho, const int* seg, int m, int* kept) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
        if (rho[i] > 0.0) atomicAdd(kept + (seg ? seg[i] : 0), 1);
}

__global__ void k_weights(const double* rho, const int* seg, const double* seg_w, int m,
                          float* wr) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        const double r = rho[i];
        wr[i] = (r > 0.0) ? (float)(seg_w[seg ? seg[i] : 0] / r) : 0.f;
    }
}

__global__ void k_zero_row_check(const double* rho, const float* l, const float* u, int m,
                                 int B, int* flags) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        if (rho[i] > 0.0) continue;
        for (int b = 0; b < B; ++b) {
            const size_t o = (size_t)i * B + b;
            if (!(l[o] <= 0.f && u[o] >= 0.f)) atomicOr(flags, 1);
        }
    }
}

// Zero rows (||a_i|| = 0, device row i) against source-order bounds: the
// slab must contain 0.
// New slab bounds in one pass over the device rows: NaN or l > u anywhere
// sets bit 1 of flags[0]; a zero row whose slab excludes 0 sets flags[1].
// flags[2] and flags[3] receive the same bits and keep them across calls
// (the report of checks that were only enqueued).  (Each source row is the
// image of exactly one device row.)
__global__ void k_check_bounds(const double* rho, const float* l_in, const float* u_in,
                               const int* perm, int m, int B_in, int* flags) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        const int src = perm ? perm[i] : i;
        const bool zero = !(rho[i] > 0.0);
        for (int b = 0; b < B_in; ++b) {
            const size_t o = (size_t)src * B_in + b;
            const float lv = l_in[o], uv = u_in[o];
            if (isnan(lv) || isnan(uv) || !(lv <= uv)) {
                atomicOr(flags, 1);
                atomicOr(flags + 2, 1);
            }
            if (zero && !(lv <= 0.f && uv >= 0.f)) {
                atomicOr(flags + 1, 1);
                atomicOr(flags + 3, 1);
            }
        }
    }
}

__global__ void k_reset_states(RhsState* st, int B, int B_user) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) {
        RhsState r = {};
        r.last_restart_k = -1;
        r.stopped = (b >= B_user) ? 1 : 0;
        st[b] = r;
    }
}

// l[i*B + b] = l_in[perm[i]*B_in + b] for b < B_in; padding RHS get (-inf, inf).
// With `skip` set, nothing is written when any of skip[0..nskip) is nonzero
// (the bounds failed validation earlier on the same stream).
__global__ void k_permute_bounds(const float* l_in, const float* u_in, const int* perm, int m,
                                 int B_in, int B, float* l, float* u, const int* skip,
                                 int nskip) {
    for (int k = 0; skip && k < nskip; ++k)
        if (skip[k]) return;
    const long long tot = (long long)m * B;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < tot;
         t += (long long)gridDim.x * blockDim.x) {
        const int i = (int)(t / B), b = (int)(t - (long long)i * B);
        const int src = perm ? perm[i] : i;
        if (b < B_in) {
            l[t] = l_in[(size_t)src * B_in + b];
            u[t] = u_in[(size_t)src * B_in + b];
        } else {
            l[t] = -INFINITY;
            u[t] = INFINITY;
        }
    }
}

// x[j*B + b] = clamp(x_in[j*B_in + b] (or 0), lo, hi); padding RHS are 0-clamped.
__global__ void k_box_init(float* x, const float* lo, const float* hi, long long nB, int B,
                           int box_len, const float* x_in, int B_in) {
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < nB;
         t += (long long)gridDim.x * blockDim.x) {
        const long long j = t / B;
        const int b = (int)(t - j * B);
        const float v = (x_in && b < B_in) ? x_in[j * B_in + b] : 0.f;
        const long long bj = (box_len == 1) ? 0 : j;
        x[t] = clampf(v, lo[bj], hi[bj]);
    }
}

__global__ void k_unpad_x(const float* x, long long n, int B, int B_out, float* out) {
    const long long tot = n * B_out;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < tot;
         t += (long long)gridDim.x * blockDim.x) {
        const long long j = t / B_out;
        const int b = (int)(t - j * B_out);
        out[t] = x[j * B + b];
    }
}

// Column sums of S for column tiles held in shared memory: CTA (tile, slice)
// accumulates rows of its slice into a private FP64 tile, written to
// work[slice][col]; a second kernel sums the slices in order.
constexpr int kColTile = 4096;
__global__ void k_colsum_partial(const int* rp, const int* col, const float* val, int m, int n,
                                 int slices, double* work) {
    __shared__ double acc[kColTile];
    const int tile = blockIdx.x / slices, slice = blockIdx.x % slices;
    const int c0 = tile * kColTile;
    for (int t = threadIdx.x; t < kColTile; t += blockDim.x) acc[t] = 0.0;
    __syncthreads();
    const int r0 = (int)((long long)m * slice / slices);
    const int r1 = (int)((long long)m * (slice + 1) / slices);
    // one warp walks the slice's rows in order; the lanes of a row add
    // distinct columns, so every acc[c] receives its terms in row order
    if (threadIdx.x < 32) {
        for (int i = r0; i < r1; ++i) {
            for (int e = rp[i] + (int)threadIdx.x; e < rp[i + 1]; e += 32) {
                const int c = col[e] - c0;
                if (c >= 0 && c < kColTile) acc[c] += (double)val[e];
            }
            __syncwarp();
        }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < kColTile; t += blockDim.x) {
        const int c = c0 + t;
        if (c < n) work[(size_t)slice * n + c] = acc[t];
    }
}

__global__ void k_colsum_final(const double* work, int slices, int n, int m, double* c64,
                               float* c32) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int k = 0; k < slices; ++k) s += work[(size_t)k * n + c];
        s /= (double)m;
        c64[c] = s;
        c32[c] = (float)s;
    }
}

__global__ void k_sumsq(const double* v, int n, double* out) {
    __shared__ double sw[8];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += v[i] * v[i];
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < 8; ++w) t += sw[w];
        *out = t;
    }
}

inline int grid_for(long long work, int threads = 256) {
    long long g = (work + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > 152 * 8) g = 152 * 8;
    return (int)g;
}

}  // namespace

cudaError_t launch_validate_csr(const int* row_ptr, const int* col, const float* val, int m,
                                int n, long long nnz, int* flags, cudaStream_t s, double* err2) {
    k_validate_csr<<<grid_for(nnz > m ? nnz : m), 256, 0, s>>>(row_ptr, col, val, m, n, nnz,
                                                               flags, err2);
    return cudaGetLastError();
}

cudaError_t launch_validate_vec(const float* v, long long len, int allow_inf, int* flags,
                                int bit, cudaStream_t s) {
    k_validate_vec<<<grid_for(len), 256, 0, s>>>(v, len, allow_inf, flags, bit);
    return cudaGetLastError();
}

cudaError_t launch_validate_pair(const float* lo, const float* hi, long long len, int* flags,
                                 int bit, cudaStream_t s) {
    k_validate_pair<<<grid_for(len), 256, 0, s>>>(lo, hi, len, flags, bit);
    return cudaGetLastError();
}

cudaError_t launch_pack(const int* row_ptr, const int* col, const float* val, const int* perm,
                        const int2* rinfo, int m, int* pcol, void* pval, suppy_dtype dt,
                        double* rho, cudaStream_t s) {
    const int grid = grid_for((long long)m * 32);
    if (dt == SUPPY_F32)
        k_pack<float><<<grid, 256, 0, s>>>(row_ptr, col, val, perm, rinfo, m, pcol,
                                           static_cast<float*>(pval), rho);
    else if (dt == SUPPY_BF16)
        k_pack<__nv_bfloat16><<<grid, 256, 0, s>>>(row_ptr, col, val, perm, rinfo, m, pcol,
                                                   static_cast<__nv_bfloat16*>(pval), rho);
    else
        k_pack<__half><<<grid, 256, 0, s>>>(row_ptr, col, val, perm, rinfo, m, pcol,
                                            static_cast<__half*>(pval), rho);
    return cudaGetLastError();
}

cudaError_t launch_csc_fill(const int2* rinfo, int m, const void* pval, suppy_dtype dt,
                            const int* pos, int* ridx, void* cval, cudaStream_t s) {
    const int grid = grid_for((long long)m * 32);
    if (dt == SUPPY_F32)
        k_csc_fill<float><<<grid, 256, 0, s>>>(rinfo, m, static_cast<const float*>(pval), pos, ridx,
                                               static_cast<float*>(cval));
    else if (dt == SUPPY_BF16)
        k_csc_fill<__nv_bfloat16><<<grid, 256, 0, s>>>(
            rinfo, m, static_cast<const __nv_bfloat16*>(pval), pos, ridx,
            static_cast<__nv_bfloat16*>(cval));
    else
        k_csc_fill<__half><<<grid, 256, 0, s>>>(rinfo, m, static_cast<const __half*>(pval), pos,
                                                ridx, static_cast<__half*>(cval));
    return cudaGetLastError();
}

cudaError_t launch_count_kept(const double* rho, const int* seg, int m, int* kept,
                              cudaStream_t s) {
    k_count_kept<<<grid_for(m), 256, 0, s>>>(rho, seg, m, kept);
    return cudaGetLastError();
}

cudaError_t launch_weights(const double* rho, const int* seg, const double* seg_w, int m,
                           float* wr, cudaStream_t s) {
    k_weights<<<grid_for(m), 256, 0, s>>>(rho, seg, seg_w, m, wr);
    return cudaGetLastError();
}

cudaError_t launch_zero_row_check(const double* rho, const float* l, const float* u, int m,
                                  int B, int* flags, cudaStream_t s) {
    k_zero_row_check<<<grid_for(m), 256, 0, s>>>(rho, l, u, m, B, flags);
    return cudaGetLastError();
}

cudaError_t launch_permute_bounds(const float* l_in, const float* u_in, const int* perm, int m,
                                  int B_in, int B, float* l, float* u, cudaStream_t s,
                                  const int* skip, int nskip) {
    k_permute_bounds<<<grid_for((long long)m * B), 256, 0, s>>>(l_in, u_in, perm, m, B_in, B, l,
                                                                u, skip, nskip);
    return cudaGetLastError();
}

cudaError_t launch_check_bounds(const double* rho, const float* l_in, const float* u_in,
                                const int* perm, int m, int B_in, int* flags, cudaStream_t s) {
    k_check_bounds<<<grid_for(m), 256, 0, s>>>(rho, l_in, u_in, perm, m, B_in, flags);
    return cudaGetLastError();
}

cudaError_t launch_reset_states(RhsState* st, int B, int B_user, cudaStream_t s) {
    k_reset_states<<<1, 64, 0, s>>>(st, B, B_user);
    return cudaGetLastError();
}

cudaError_t launch_box_init(float* x, const float* lo, const float* hi, long long nB, int B,
                            int box_len, const float* x_in, int B_in, cudaStream_t s) {
    k_box_init<<<grid_for(nB), 256, 0, s>>>(x, lo, hi, nB, B, box_len, x_in, B_in);
    return cudaGetLastError();
}

cudaError_t launch_unpad_x(const float* x, long long n, int B, int B_out, float* out,
                           cudaStream_t s) {
    k_unpad_x<<<grid_for(n * B_out), 256, 0, s>>>(x, n, B, B_out, out);
    return cudaGetLastError();
}

// ---- one right-hand side (slot) of a batched context -------------------
// Column b of the device-order bounds from source-order l_in, u_in (m each).
__global__ void k_load_column(const float* l_in, const float* u_in, const int* perm, int m, int B,
                              int b, float* l, float* u) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        const int src = perm ? perm[i] : i;
        l[(size_t)i * B + b] = l_in[src];
        u[(size_t)i * B + b] = u_in[src];
    }
}

// x[:, b] <- box(0), and a fresh iteration state for right-hand side b.
__global__ void k_reset_column(float* x, const float* lo, const float* hi, long long n, int B,
                               int b, int box_len, RhsState* st, float* xprev) {
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (long long)gridDim.x * blockDim.x) {
        const long long bj = (box_len == 1) ? 0 : j;
        const float v = clampf(0.f, lo[bj], hi[bj]);
        x[j * B + b] = v;
        if (xprev) xprev[j * B + b] = v;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        RhsState r = {};
        r.last_restart_k = -1;
        st[b] = r;
    }
}

__global__ void k_set_stopped(RhsState* st, int b) { st[b].stopped = 1; }

// out[j] = x[j * B + b]
__global__ void k_extract_column(const float* x, long long n, int B, int b, float* out) {
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (long long)gridDim.x * blockDim.x)
        out[j] = x[j * B + b];
}

// DROP column counts: one warp per device row with ||a_i|| > 0 adds 1 to the
// count of every column it stores a nonzero in; zc = 1 / count.
template <typename VT>
__global__ void k_col_counts(const int2* rinfo, const int* col, const VT* val, const double* rho,
                             int m, int* counts) {
    const int lane = threadIdx.x & 31;
    const int warps = (gridDim.x * blockDim.x) >> 5;
    for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < m; i += warps) {
        if (!(rho[i] > 0.0)) continue;
        const int2 ri = rinfo[i];
        for (int e = lane; e < ri.y; e += 32)
            if ((float)val[ri.x + e] != 0.f) atomicAdd(counts + col[ri.x + e], 1);
    }
}

__global__ void k_inv_counts(const int* counts, int n, float* zc) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
        zc[j] = counts[j] > 0 ? 1.0f / (float)counts[j] : 0.f;
}

cudaError_t launch_column_scaling(const int2* rinfo, const int* col, const void* val,
                                  suppy_dtype dt, const double* rho, int m, int n, int* counts,
                                  float* zc, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(int) * (size_t)n, s);
    if (e != cudaSuccess) return e;
    const int grid = grid_for((long long)m * 32);
    if (dt == SUPPY_F32)
        k_col_counts<float><<<grid, 256, 0, s>>>(rinfo, col, static_cast<const float*>(val), rho, m,
                                                 counts);
    else if (dt == SUPPY_BF16)
        k_col_counts<__nv_bfloat16><<<grid, 256, 0, s>>>(
            rinfo, col, static_cast<const __nv_bfloat16*>(val), rho, m, counts);
    else
        k_col_counts<__half><<<grid, 256, 0, s>>>(rinfo, col, static_cast<const __half*>(val), rho,
                                                  m, counts);
    k_inv_counts<<<grid_for(n), 256, 0, s>>>(counts, n, zc);
    return cudaGetLastError();
}

__global__ void k_to_float(const double* v, int n, float* out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        out[i] = (float)v[i];
}

cudaError_t launch_to_float(const double* v, int n, float* out, cudaStream_t s) {
    k_to_float<<<grid_for(n), 256, 0, s>>>(v, n, out);
    return cudaGetLastError();
}

cudaError_t launch_load_column(const float* l_in, const float* u_in, const int* perm, int m, int B,
                               int b, float* l, float* u, cudaStream_t s) {
    k_load_column<<<grid_for(m), 256, 0, s>>>(l_in, u_in, perm, m, B, b, l, u);
    return cudaGetLastError();
}

cudaError_t launch_reset_column(float* x, const float* lo, const float* hi, long long n, int B,
                                int b, int box_len, RhsState* st, float* xprev, cudaStream_t s) {
    k_reset_column<<<grid_for(n), 256, 0, s>>>(x, lo, hi, n, B, b, box_len, st, xprev);
    return cudaGetLastError();
}

cudaError_t launch_set_stopped(RhsState* st, int b, cudaStream_t s) {
    k_set_stopped<<<1, 1, 0, s>>>(st, b);
    return cudaGetLastError();
}

cudaError_t launch_extract_column(const float* x, long long n, int B, int b, float* out,
                                  cudaStream_t s) {
    k_extract_column<<<grid_for(n), 256, 0, s>>>(x, n, B, b, out);
    return cudaGetLastError();
}

cudaError_t launch_colmean(const int* row_ptr, const int* col, const float* val, int m, int n,
                           double* c64, float* c32, double* work, int slices, cudaStream_t s) {
    const int tiles = (n + kColTile - 1) / kColTile;
    k_colsum_partial<<<tiles * slices, 256, 0, s>>>(row_ptr, col, val, m, n, slices, work);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_colsum_final<<<grid_for(n), 256, 0, s>>>(work, slices, n, m, c64, c32);
    return cudaGetLastError();
}

cudaError_t launch_sumsq(const double* v, int n, double* out, cudaStream_t s) {
    k_sumsq<<<1, 256, 0, s>>>(v, n, out);
    return cudaGetLastError();
}

}  // namespace suppy
