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

// 512 blocks x 10 doubles (40 KiB) + the completion counter.
static __device__ __align__(256) double g_noalloc_partials[kNoallocMaxBlocks * kNoallocValues];
static __device__ __align__(256) unsigned int g_noalloc_counter;

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
    if (n < 1 || n > (int64_t)INT_MAX) return LBMS_EINVAL;   // 32-bit cell index of the kernel
    double* partials = nullptr;
    unsigned int* counter = nullptr;
    if (scratch_for_current_device(&partials, &counter) != cudaSuccess) return LBMS_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the counter must start at zero; the partials are written before they are read
    if (cudaMemsetAsync(counter, 0, sizeof(unsigned int), st) != cudaSuccess) return LBMS_ECUDA;
    const int64_t want = (n + kNoallocBlock - 1) / kNoallocBlock;
    const int blocks = (int)(want < kNoallocMaxBlocks ? want : kNoallocMaxBlocks);
    lbms::residual_kernel<double><<<blocks, kNoallocBlock, 0, st>>>(X, snapshot, n, (int)n, update ? 1 : 0,
                                                                    partials, counter, out);
    return cudaGetLastError() == cudaSuccess ? LBMS_OK : LBMS_ECUDA;
}
