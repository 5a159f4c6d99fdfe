// Allocation-free nu-sensitivity reduction.
//
// Some callers cannot call cudaMalloc: a caller whose device memory is
// entirely owned by a framework's caching allocator (raw cudaMalloc there can
// fail or fragment the pool), or a latency-critical loop that cannot afford
// the implicit device synchronisation and the milliseconds cudaMalloc takes.
// They may also hold no plan (creating one allocates).  For them this file
// provides sphnse_nu_sensitivity_noalloc: the same block-partial reduction
// that sphnse_rhs_adjoint uses for its nu_bar output, with the partials in a
// file-scope __device__ array instead of plan-owned scratch.
//
// The array holds SPHNSE_NOALLOC_MAX_BLOCKS doubles (32 KB) on every device
// that loads the library, until the process exits.  Every call shares it and
// overwrites the slots it reads (nothing has to start at zero); calls that
// overlap on the GPU (different streams, or host threads) race on it.
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>

#include "internal.h"

// the scratch: block partial sums, one per 2048 packed entries
static __device__ __align__(256) double g_noalloc_partial[SPHNSE_NOALLOC_MAX_BLOCKS];

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_PER_THREAD = 8;
constexpr int NA_PER_BLOCK = NA_THREADS * NA_PER_THREAD;

// device address of g_noalloc_partial per device, looked up with that device
// current (in host code the symbol names a host-side stand-in); only a
// successful lookup is kept, so a failed one is tried again on the next call
constexpr int NA_MAX_DEVICES = 64;
std::mutex g_lookup;
std::atomic<double*> g_addr[NA_MAX_DEVICES];

double* scratch_address(int dev) {
    double* p = g_addr[dev].load(std::memory_order_acquire);
    if (p) return p;
    std::lock_guard<std::mutex> lk(g_lookup);
    p = g_addr[dev].load(std::memory_order_relaxed);
    if (!p && cudaGetSymbolAddress(reinterpret_cast<void**>(&p), g_noalloc_partial) == cudaSuccess && p)
        g_addr[dev].store(p, std::memory_order_release);
    return g_addr[dev].load(std::memory_order_relaxed);
}

// packed index i -> degree L (m-major order, L = max(m,1)..N)
__device__ __forceinline__ int degree_of(int N, int i) {
    int lo = 0, hi = N;  // find the largest m with packed_off(N, m) <= i
    while (lo < hi) {
        const int mid = (lo + hi + 1) / 2;
        if (sph::packed_off(N, mid) <= i) lo = mid;
        else hi = mid - 1;
    }
    return i - sph::packed_off(N, lo) + (lo > 0 ? lo : 1);
}

__global__ void __launch_bounds__(NA_THREADS) k_na_partial(const double2* __restrict__ alpha,
                                                          const double2* __restrict__ w, int N, int n,
                                                          double* __restrict__ part) {
    __shared__ double red[NA_THREADS];
    double s = 0.0;
    const int base = blockIdx.x * NA_PER_BLOCK + threadIdx.x;
#pragma unroll
    for (int k = 0; k < NA_PER_THREAD; ++k) {
        const int i = base + k * NA_THREADS;
        if (i < n) {
            const int L = degree_of(N, i);
            const double2 a = alpha[i], b = w[i];
            s += double(L) * (L + 1.0) * (a.x * b.x + a.y * b.y);
        }
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int wd = NA_THREADS / 2; wd > 0; wd >>= 1) {
        if (threadIdx.x < wd) red[threadIdx.x] += red[threadIdx.x + wd];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// one block: out = -sum_b part[b], summed in a fixed order
__global__ void __launch_bounds__(NA_THREADS) k_na_final(const double* __restrict__ part, int nb,
                                                        double* __restrict__ out) {
    __shared__ double red[NA_THREADS];
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += NA_THREADS) s += part[b];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int wd = NA_THREADS / 2; wd > 0; wd >>= 1) {
        if (threadIdx.x < wd) red[threadIdx.x] += red[threadIdx.x + wd];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = -red[0];
}

}  // namespace

extern "C" int sphnse_nu_sensitivity_noalloc(int L, const double* alpha, const double* w, double* out,
                                             void* stream) {
    if (L < 1 || !alpha || !w || !out) return SPHNSE_E_ARG;
    const long long n = (long long)(L + 1) * (L + 2) / 2 - 1;
    if (n > (long long)SPHNSE_NOALLOC_MAX_BLOCKS * NA_PER_BLOCK) return SPHNSE_E_TOO_LARGE;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return SPHNSE_E_CUDA;
    if (dev < 0 || dev >= NA_MAX_DEVICES) return SPHNSE_E_UNSUPPORTED;
    double* part = scratch_address(dev);
    if (!part) return SPHNSE_E_CUDA;
    const int nb = int((n + NA_PER_BLOCK - 1) / NA_PER_BLOCK);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    k_na_partial<<<nb, NA_THREADS, 0, s>>>(reinterpret_cast<const double2*>(alpha),
                                           reinterpret_cast<const double2*>(w), L, int(n), part);
    k_na_final<<<1, NA_THREADS, 0, s>>>(part, nb, out);
    return cudaGetLastError() == cudaSuccess ? SPHNSE_OK : SPHNSE_E_CUDA;
}
