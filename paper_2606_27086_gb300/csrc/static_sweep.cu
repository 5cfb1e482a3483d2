// suppy_sweep_static: one simultaneous (Cimmino-type) hyperslab sweep on
// caller-provided device buffers that allocates nothing.
//
// Some callers cannot call cudaMalloc at the point where they want a sweep:
// code running under an allocator that forbids device allocations after
// start-up (a fixed memory budget, a real-time loop), code that owns all of
// its device memory through its own pool, or code that must not trigger the
// implicit synchronization a cudaMalloc/cudaFree can cause.  This entry point
// keeps its scratch (the correction accumulator, the per-CTA proximity
// partials and a validity word) in a file-scope device array of fixed size
// instead.  Since the bounds live on the device and the call only enqueues,
// invalid bounds are detected on the device: x is left unchanged and the
// proximity written is NaN.
//
// The scratch array is process-wide: every GPU that loads the library holds
// it until the process exits, and every call on a device shares it.  Calls
// that may overlap on the GPU (different streams, or the same scratch used
// from several host threads without ordering) race on it.
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "common.cuh"

namespace suppy {
namespace {

constexpr int kStaticMaxN = 1 << 20;        // largest n (unknowns) a call accepts
constexpr int kStaticMaxCtas = 2048;        // CTAs of the row kernel (partial slots)
constexpr int kStaticThreads = 256;
constexpr int kStaticDevices = 64;

// correction accumulator (kStaticMaxN floats), the CTA partials
// (kStaticMaxCtas doubles) and a validity word: 4 MiB + 16 KiB + 256 B
constexpr size_t kStaticFlagOffset = sizeof(float) * kStaticMaxN + sizeof(double) * kStaticMaxCtas;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticFlagOffset + 256];

std::mutex g_static_mu;
void* g_static_ptr[kStaticDevices] = {};

// messages go to the thread's context-free error slot (suppy_last_error(NULL))
suppy_status static_fail(suppy_status s, const std::string& msg) {
    set_thread_error(msg);
    return s;
}

// Device address of the scratch array on the current device, resolved once
// per device (cudaGetSymbolAddress with that device current).
suppy_status static_scratch(int dev, void** out) {
    if (dev < 0 || dev >= kStaticDevices) return static_fail(SUPPY_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return static_fail(SUPPY_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        }
        g_static_ptr[dev] = p;
    }
    *out = g_static_ptr[dev];
    return SUPPY_OK;
}

__global__ void k_static_zero(float* delta, int n, int* flag) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
        delta[j] = 0.f;
    if (blockIdx.x == 0 && threadIdx.x == 0) *flag = 0;
}

// One warp per row (grid-stride over rows): r = <a_i, x>, rho = ||a_i||^2 in
// FP64 (the library's row norms are FP64 everywhere: a row of tiny values
// whose squares underflow FP32 is still a constraint), d = clamp(r, l, u) - r;
// delta += lambda w d / rho * a_i; FP64 proximity partial 1/2 w d^2 / rho per
// CTA.  Bounds with a NaN or l > u, and a row with rho = 0 whose slab excludes
// 0, set the validity word (the finalize then leaves x alone).
__global__ void __launch_bounds__(kStaticThreads) k_static_rows(
    const int* rp, const int* col, const float* val, int m, const float* l, const float* u, float w,
    float lam, const float* x, float* delta, double* partial, int* flag) {
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (kStaticThreads / 32);
    double prox = 0.0;
    for (int i = (blockIdx.x * kStaticThreads + threadIdx.x) >> 5; i < m; i += warps) {
        const int a = rp[i], b = rp[i + 1];
        const float li = l[i], ui = u[i];
        float dot = 0.f;
        double rho = 0.0;
        for (int e = a + lane; e < b; e += 32) {
            const float v = val[e];
            dot = fmaf(v, __ldg(x + col[e]), dot);
            rho = fma((double)v, (double)v, rho);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            dot += __shfl_xor_sync(0xffffffffu, dot, o);
            rho += __shfl_xor_sync(0xffffffffu, rho, o);
        }
        const bool bad_bounds = isnan(li) || isnan(ui) || li > ui;
        if (rho == 0.0) {
            // an empty row carries no constraint, provided 0 lies in its slab
            if (lane == 0 && (bad_bounds || !(li <= 0.f && 0.f <= ui))) atomicOr(flag, 1);
            continue;
        }
        if (bad_bounds) {
            if (lane == 0) atomicOr(flag, 1);
            continue;
        }
        const float d = clampf(dot, li, ui) - dot;
        if (lane == 0) prox += 0.5 * (double)w * (double)d * (double)d / rho;
        const float coef = (float)((double)lam * (double)w * (double)d / rho);
        if (coef != 0.f)
            for (int e = a + lane; e < b; e += 32) atomicAdd(delta + col[e], coef * val[e]);
    }
    prox = warp_sum(prox);
    __shared__ double sw[kStaticThreads / 32];
    if (lane == 0) sw[threadIdx.x >> 5] = prox;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < kStaticThreads / 32; ++k) s += sw[k];
        partial[blockIdx.x] = s;
    }
}

// x <- clamp(x + delta, lo, hi); CTA 0 sums the partials in a fixed order.
// When the validity word is set, x stays as it was and the proximity is NaN.
__global__ void k_static_finalize(float* x, const float* delta, int n, const float* lo,
                                  const float* hi, int box_len, const double* partial, int np,
                                  double* prox_out, const int* flag) {
    if (*flag) {
        if (blockIdx.x == 0 && threadIdx.x == 0 && prox_out)
            *prox_out = __longlong_as_double(0x7ff8000000000000LL);
        return;
    }
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
        const int bj = (box_len == 1) ? 0 : j;
        x[j] = clampf(x[j] + delta[j], lo[bj], hi[bj]);
    }
    if (blockIdx.x == 0 && prox_out) {
        double s = 0.0;
        for (int c = threadIdx.x; c < np; c += blockDim.x) s += partial[c];
        s = warp_sum(s);
        __shared__ double sw[32];
        if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = s;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += sw[k];
            *prox_out = t;
        }
    }
}

}  // namespace
}  // namespace suppy

using namespace suppy;

extern "C" suppy_status suppy_sweep_static(const suppy_csr* A, const float* l, const float* u,
                                           float weight, float lambda, const float* box_lo,
                                           const float* box_hi, int64_t box_len, float* x,
                                           double* proximity, void* stream) {
    if (!A || !l || !u || !box_lo || !box_hi || !x)
        return static_fail(SUPPY_EINVAL, "NULL argument to suppy_sweep_static");
    if (!A->on_device) return static_fail(SUPPY_EINVAL, "suppy_sweep_static takes device arrays only");
    if (A->m < 0 || A->n < 1 || !A->row_ptr || (A->nnz > 0 && (!A->col || !A->val)))
        return static_fail(SUPPY_EINVAL, "bad CSR shape or pointers");
    if (A->n > kStaticMaxN)
        return static_fail(SUPPY_EINVAL, "suppy_sweep_static: n = " + std::to_string(A->n) +
                                             " exceeds the static scratch of " +
                                             std::to_string(kStaticMaxN) + " unknowns");
    if (box_len != 1 && box_len != (int64_t)A->n)
        return static_fail(SUPPY_EINVAL, "box_len must be 1 or n");
    if (!(lambda > 0.f && lambda < 2.f) || !(weight > 0.f) || !std::isfinite(weight))
        return static_fail(SUPPY_EINVAL, "need 0 < lambda < 2 and a finite weight > 0");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return static_fail(SUPPY_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    }
    void* base = nullptr;
    suppy_status s = static_scratch(dev, &base);
    if (s != SUPPY_OK) return s;
    float* delta = static_cast<float*>(base);
    double* partial = reinterpret_cast<double*>(static_cast<unsigned char*>(base) +
                                                sizeof(float) * (size_t)kStaticMaxN);
    int* flag = reinterpret_cast<int*>(static_cast<unsigned char*>(base) + kStaticFlagOffset);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int n = A->n, m = A->m;
    const int zgrid = std::min(1024, (n + kStaticThreads - 1) / kStaticThreads);
    const int rgrid = (int)std::max<long long>(
        1, std::min<long long>(kStaticMaxCtas, ((long long)m * 32 + kStaticThreads - 1) / kStaticThreads));
    k_static_zero<<<zgrid, kStaticThreads, 0, st>>>(delta, n, flag);
    k_static_rows<<<rgrid, kStaticThreads, 0, st>>>(A->row_ptr, A->col, A->val, m, l, u, weight,
                                                    lambda, x, delta, partial, flag);
    k_static_finalize<<<zgrid, kStaticThreads, 0, st>>>(x, delta, n, box_lo, box_hi, (int)box_len,
                                                       partial, rgrid, proximity, flag);
    e = cudaGetLastError();
    if (e != cudaSuccess) return static_fail(SUPPY_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
    return SUPPY_OK;
}
