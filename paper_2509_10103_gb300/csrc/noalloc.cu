// Energy of a spectral field without any device allocation.
//
// This is a variant of the library's inner-product reduction for callers that
// cannot call cudaMalloc at the point of use: for example code running where
// every byte of device memory has already been handed to another allocator (a
// framework's caching allocator or a fixed pool sized to the card), so a new
// cudaMalloc would fail; or a tight loop in which cudaMalloc/cudaFree are
// ruled out because they can synchronise the whole device and stall work on
// other streams.  Such callers cannot create a pnop_ctx either (creating one
// allocates operators and workspace), so this entry point needs no context:
// the caller passes the field, the radial weights and the sizes, and the
// reduction's scratch (per-block partial sums and the result slot) lives in a
// fixed array in device global memory that every GPU loading the library holds
// until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/pnop.h"

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 16;                       // values per thread per block
constexpr int kPerBlock = kThreads * kItems;     // 4096 complex values per block
constexpr int kMaxBlocks = (int)(PNOP_NOALLOC_MAX_VALUES / kPerBlock);
static_assert((long long)kMaxBlocks * kPerBlock == PNOP_NOALLOC_MAX_VALUES, "limit must be a whole number of blocks");
constexpr int kMaxDevices = 64;

// The scratch: kMaxBlocks partial sums followed by one result slot (32 KiB + 8 B).
static __device__ __align__(256) double g_energy_scratch[kMaxBlocks + 1];

// Device address of g_energy_scratch per device, resolved once per device.
std::mutex g_mutex;
double* g_scratch_ptr[kMaxDevices] = {};

// Per-block partial of sum_{c,j,m,k} W_j c_k |u|^2 over a fixed contiguous
// chunk of kPerBlock values (deterministic order: fixed chunks, fixed tree).
__global__ void k_energy_partial_noalloc(const double2* __restrict__ u, const double* __restrict__ W, int nr, int nm,
                                         int nk, long long n, double* __restrict__ scratch) {
    __shared__ double red[kThreads];
    const long long S = (long long)nr * nm * nk;
    const long long base = (long long)blockIdx.x * kPerBlock;
    double acc = 0.0;
    for (int it = 0; it < kItems; ++it) {
        const long long i = base + (long long)it * kThreads + threadIdx.x;
        if (i < n) {
            const long long e = i % S;
            const int k = (int)(e % nk);
            const int j = (int)(e / ((long long)nk * nm));
            const double2 v = u[i];
            acc += W[j] * (k == 0 ? 1.0 : 2.0) * (v.x * v.x + v.y * v.y);
        }
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = kThreads / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) scratch[blockIdx.x] = red[0];
}

// Sums the nb partials in a fixed order into the result slot, times scale.
__global__ void k_energy_final_noalloc(double* __restrict__ scratch, int nb, double scale) {
    __shared__ double red[1024];
    double acc = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) acc += scratch[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) scratch[kMaxBlocks] = red[0] * scale;
}

// Resolves (once per device, with that device current) the device address of
// the scratch array; host code may not use the symbol itself as an address.
// The address is cached for the life of the process: a cudaDeviceReset (or a
// reset of the primary context) unloads the module, after which the cached
// address is stale, so callers of this entry point must not reset the device.
int scratch_for_current_device(double** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PNOP_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_energy_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return PNOP_ERR_CUDA;
        }
        g_scratch_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_ptr[dev];
    return PNOP_OK;
}

}  // namespace

extern "C" int pnop_energy_noalloc(const void* u, const double* W, int nr, int M, int K, double Lz, double* E_out,
                                   void* cuda_stream) {
    if (!u || !W || !E_out || nr < 1 || M < 0 || K < 0 || !(Lz > 0)) return PNOP_ERR_INVALID_ARG;
    // 3 nr (2M+1) (K+1) <= max, checked one factor at a time so that no
    // product can overflow before the comparison
    const long long cap = PNOP_NOALLOC_MAX_VALUES;
    const long long f1 = 3LL * nr, f2 = 2LL * M + 1, f3 = (long long)K + 1;
    if (f1 > cap || f2 > cap / f1 || f3 > cap / (f1 * f2)) return PNOP_ERR_INVALID_ARG;
    const long long n = f1 * f2 * f3;
    double* scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc != PNOP_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const int nb = (int)((n + kPerBlock - 1) / kPerBlock);
    // The array keeps whatever the previous call left there.  Nothing needs
    // clearing: block b of the first kernel writes partial b for every b < nb,
    // the second kernel reads exactly those nb partials and writes the result
    // slot, and the copy below reads that slot after it in stream order.
    k_energy_partial_noalloc<<<nb, kThreads, 0, s>>>(static_cast<const double2*>(u), W, nr, 2 * M + 1, K + 1, n,
                                                     scratch);
    k_energy_final_noalloc<<<1, 1024, 0, s>>>(scratch, nb, 0.5 * 2.0 * M_PI * Lz);
    if (cudaGetLastError() != cudaSuccess) return PNOP_ERR_CUDA;
    if (cudaMemcpyAsync(E_out, scratch + kMaxBlocks, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return PNOP_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return PNOP_ERR_CUDA;
    return std::isfinite(*E_out) ? PNOP_OK : PNOP_ERR_NONFINITE;
}
