// Internal interface between the C ABI (lbms_capi.cu) and the kernel
// launchers (lbms_launch.cu).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace lbms {

constexpr int kRedSlots = 16;          // doubles per reduction result slot
constexpr int kRedResidual = 0;        // slot of the residual sums
constexpr int kRedBoundary = 1;        // slot of the boundary sums
constexpr int kRedMaxBlocks = 1216;    // 152 SMs x 8 resident blocks of 256 threads

struct DevBuffers {
    void* f[2] = {nullptr, nullptr};   // non-equilibrium populations h = f* - w X, [3][Q][S]
    void* X[2] = {nullptr, nullptr};   // mole fractions (double or double-float pairs), [3][S]
    double* snap = nullptr;            // residual snapshot, [3][S]
    int* nbr = nullptr;                // [S][nb_width]
    int* rows = nullptr;               // [3][nrows]: x = 0, x = 1, x = nx-1 cell per row (-1 if solid)
    double* red_partials = nullptr;    // [kRedMaxBlocks][kRedSlots]
    unsigned int* red_counter = nullptr;  // one per slot
    double* red_out = nullptr;         // [2][kRedSlots]
    void* fields = nullptr;            // [3 + 3 dim][S] of tau and u (lazy), FP64 or FP32
};

struct Launch {
    int dim = 2;
    int precision = 1;                 // 0 = FP64, 1 = FP32, 2 = FP16 populations / FP32 compute
    int64_t S = 0;                     // padded row stride (elements)
    int nf = 0;                        // fluid cells
    int nrows = 0;                     // ny * nz
    int cur = 0;                       // lattice holding the latest post-collision state
    DevBuffers b;
    double xin[3] = {0, 0, 0};
    double q[3] = {0, 0, 0};
    double D12 = 1, D13 = 1, D23 = 1;  // lattice binary diffusivities
    double stoich[3] = {-1, 1, 0};     // nu_i of the electrode reaction (Eq. 38)
    double tau_min = 1.0, tau_max = 5.0;
    int drift = 1;
    int sm_count = 152;
};

size_t pop_size(int precision);    // bytes per stored population
size_t x_size(int precision);      // bytes per stored mole fraction
size_t field_size(int precision);  // bytes per tau / u value of the fields kernel
int residual_blocks(const Launch& L);

cudaError_t launch_step(const Launch& L, cudaStream_t st);
cudaError_t launch_init(const Launch& L, cudaStream_t st);
cudaError_t launch_fields(const Launch& L, cudaStream_t st);
cudaError_t launch_residual(const Launch& L, int update, cudaStream_t st);
cudaError_t launch_boundary(const Launch& L, cudaStream_t st);

}  // namespace lbms
