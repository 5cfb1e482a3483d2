// suppy_sweep_static: one simultaneous (Cimmino-type) hyperslab sweep on
// caller-provided device buffers that allocates nothing.
//
// Some callers cannot call cudaMalloc at the point where they want a sweep:
// code running under an allocator that forbids device allocations after
// start-up (a fixed memory budget, a real-time loop), code that owns all of
// its device memory through its own pool, or code that must not trigger the
// implicit synchronization a cudaMalloc/cudaFree can cause.  This entry point
// keeps its scratch (the correction accumulator and the per-CTA proximity
// partials) in a file-scope device array of fixed size instead.
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

// correction accumulator (kStaticMaxN floats) followed by the CTA partials
// (kStaticMaxCtas doubles): 4 MiB + 16 KiB
static __device__ __align__(256) unsigned char g_static_scratch[sizeof(float) * kStaticMaxN +
                                                                sizeof(double) * kStaticMaxCtas];

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

__global__ void k_static_zero(float* delta, int n) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x)
        delta[j] = 0.f;
}

// One warp per row (grid-stride over rows): r = <a_i, x>, rho = ||a_i||^2,
// d = clamp(r, l, u) - r; delta += lambda w d / rho * a_i; FP64 proximity
// partial 1/2 w d^2 / rho per CTA.
__global__ void __launch_bounds__(kStaticThreads) k_static_rows(
    const int* rp, const int* col, const float* val, int m, const float* l, const float* u, float w,
    float lam, const float* x, float* delta, double* partial) {
    const int lane = threadIdx.x & 31;
    const int warps = gridDim.x * (kStaticThreads / 32);
    double prox = 0.0;
    for (int i = (blockIdx.x * kStaticThreads + threadIdx.x) >> 5; i < m; i += warps) {
        const int a = rp[i], b = rp[i + 1];
        float dot = 0.f, rho = 0.f;
        for (int e = a + lane; e < b; e += 32) {
            const float v = val[e];
            dot = fmaf(v, __ldg(x + col[e]), dot);
            rho = fmaf(v, v, rho);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            dot += __shfl_xor_sync(0xffffffffu, dot, o);
            rho += __shfl_xor_sync(0xffffffffu, rho, o);
        }
        if (rho == 0.f) continue;   // an empty row carries no constraint
        const float d = clampf(dot, l[i], u[i]) - dot;
        if (lane == 0) prox += 0.5 * (double)w * (double)d * (double)d / (double)rho;
        const float coef = lam * w * d / rho;
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
__global__ void k_static_finalize(float* x, const float* delta, int n, const float* lo,
                                  const float* hi, int box_len, const double* partial, int np,
                                  double* prox_out) {
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
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int n = A->n, m = A->m;
    const int zgrid = std::min(1024, (n + kStaticThreads - 1) / kStaticThreads);
    const int rgrid = std::max(1, std::min(kStaticMaxCtas, (m * 32 + kStaticThreads - 1) / kStaticThreads));
    k_static_zero<<<zgrid, kStaticThreads, 0, st>>>(delta, n);
    k_static_rows<<<rgrid, kStaticThreads, 0, st>>>(A->row_ptr, A->col, A->val, m, l, u, weight,
                                                    lambda, x, delta, partial);
    k_static_finalize<<<zgrid, kStaticThreads, 0, st>>>(x, delta, n, box_lo, box_hi, (int)box_len,
                                                       partial, rgrid, proximity);
    e = cudaGetLastError();
    if (e != cudaSuccess) return static_fail(SUPPY_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
    return SUPPY_OK;
}
