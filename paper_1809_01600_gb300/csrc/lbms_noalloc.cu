// Allocation-free variant of the residual reduction, for callers that cannot
// allocate device memory themselves: code running inside a CUDA graph being
// captured, a host framework whose memory pool owns every device allocation,
// or a real-time loop that must not call cudaMalloc (it synchronises the
// device).  The reduction needs scratch space (one FP64 partial per block and
// a completion counter); here that scratch is a fixed file-scope device array
// that every GPU loading this library holds until the process exits.
#include <climits>
#include <mutex>

#include "../../include/lbms.h"
#include "lbms_kernels.cuh"

namespace {

constexpr int kNoallocBlock = 256;
constexpr int kNoallocMaxBlocks = 512;   // grid cap: the scratch holds one partial slot per block
constexpr int kNoallocValues = 10;       // sums written per block (see lbms.h)
constexpr int64_t kNoallocMaxCells = INT_MAX;   // cells per species accepted (the kernel indexes in 64 bits)

// 512 blocks x 10 doubles (40 KiB) + the completion counter.
static __device__ __align__(256) double g_noalloc_partials[kNoallocMaxBlocks * kNoallocValues];
static __device__ __align__(256) unsigned int g_noalloc_counter;

// Residual sums over n caller-owned FP64 cells per species (species-major,
// row stride n): out[0..2] = sum (X - snap)^2, out[3..5] = sum X^2,
// out[6..8] = sum X, out[9] = count of non-finite X.  When update != 0 the
// snapshot takes X.  Grid-stride over a capped grid with a 64-bit index, so
// the stride never overflows whatever n the caller passes.
__global__ void __launch_bounds__(256) residual_kernel(const double* __restrict__ X, double* __restrict__ snap,
                                                       int64_t n, int update, double* __restrict__ partials,
                                                       unsigned int* __restrict__ counter, double* __restrict__ out) {
    double acc[10];
#pragma unroll
    for (int v = 0; v < 10; ++v) acc[v] = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            const double x = X[s * n + i];
            const double d = x - snap[s * n + i];
            acc[s] += d * d;
            acc[3 + s] += x * x;
            acc[6 + s] += x;
            if (!isfinite(x)) acc[9] += 1.0;
            if (update) snap[s * n + i] = x;
        }
    }
    lbms::reduce_to_out<10>(acc, partials, counter, out);
}

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
double* g_partials_ptr[kMaxDevices] = {};
unsigned int* g_counter_ptr[kMaxDevices] = {};

// In host code the array names are host-side stand-ins, not device addresses:
// the device addresses come from cudaGetSymbolAddress, looked up once per
// device with that device current.
cudaError_t scratch_for_current_device(double** partials, unsigned int** counter) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_partials_ptr[dev]) {
        void* p = nullptr;
        void* q = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess) return e;
        e = cudaGetSymbolAddress(&q, g_noalloc_counter);
        if (e != cudaSuccess) return e;
        g_partials_ptr[dev] = static_cast<double*>(p);
        g_counter_ptr[dev] = static_cast<unsigned int*>(q);
    }
    *partials = g_partials_ptr[dev];
    *counter = g_counter_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" lbms_status lbms_residual_sums_noalloc(const double* X, double* snapshot, int64_t n, int update,
                                                  double* out, void* stream) {
    if (!X || !snapshot || !out) return LBMS_EINVAL;
    if (n < 1 || n > kNoallocMaxCells) return LBMS_EINVAL;
    double* partials = nullptr;
    unsigned int* counter = nullptr;
    if (scratch_for_current_device(&partials, &counter) != cudaSuccess) return LBMS_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the counter must start at zero; the partials are written before they are read
    if (cudaMemsetAsync(counter, 0, sizeof(unsigned int), st) != cudaSuccess) return LBMS_ECUDA;
    const int64_t want = (n + kNoallocBlock - 1) / kNoallocBlock;
    const int blocks = (int)(want < kNoallocMaxBlocks ? want : kNoallocMaxBlocks);
    residual_kernel<<<blocks, kNoallocBlock, 0, st>>>(X, snapshot, n, update ? 1 : 0, partials, counter, out);
    return cudaGetLastError() == cudaSuccess ? LBMS_OK : LBMS_ECUDA;
}
