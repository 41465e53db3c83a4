// Internal interface between the C ABI (lbms_capi.cu) and the kernel
// launchers (lbms_launch.cu).
#pragma once

#include <cstddef>
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

struct lbms_ctx;

namespace lbms {

constexpr int kCaseOutSlots = 16;      // doubles per case: residual sums (10) | boundary sums (6)

// Step-kernel variants the autotuner chooses from: (cells per block, minimum
// resident blocks per SM for the register budget, how neighbours are found,
// one thread per cell for all species instead of one per (cell, species)).
// Neighbours: kNbIndex32 reads a row of 32-bit fluid indices per cell,
// kNbOffset16 a row of 16-bit offsets, kNbRowMask decodes them from per-row
// fluid bitmasks and a 4-byte coordinate per cell (no per-link table).
enum { kNbIndex32 = 0, kNbOffset16 = 1, kNbRowMask = 2 };
constexpr int kStepVariants = 10;
constexpr int kVariantCells[kStepVariants] = {32, 32, 64, 32, 32, 64, 64, 32, 64, 32};
constexpr int kVariantMinBlocks[kStepVariants] = {8, 6, 4, 8, 6, 4, 8, 16, 8, 16};
constexpr int kVariantNb[kStepVariants] = {kNbIndex32,  kNbIndex32, kNbIndex32, kNbOffset16, kNbOffset16,
                                           kNbOffset16, kNbIndex32, kNbIndex32, kNbRowMask,  kNbRowMask};
constexpr int kVariantPerCell[kStepVariants] = {0, 0, 0, 0, 0, 0, 1, 1, 1, 1};

// Limits of the per-cell coordinate word of kNbRowMask (x | y << 11 | z << 21).
constexpr int kRowMaskMaxNx = 2048, kRowMaskMaxNy = 1024, kRowMaskMaxNz = 2048;

struct DevBuffers {
    void* f[2] = {nullptr, nullptr};   // non-equilibrium populations h = f* - w X, [3][Q][S]
    void* X[2] = {nullptr, nullptr};   // mole fractions (double or double-float blocks)
    double* snap = nullptr;            // residual snapshot, [3][S]
    int* nbr = nullptr;                // [S][nb_width]
    int16_t* nbr16 = nullptr;          // [S][nb16_width] offsets, when they all fit (else null)
    uint32_t* cell_code = nullptr;     // [S] x | y << 11 | z << 21 of each fluid cell (kNbRowMask; else null)
    uint4* rowtab = nullptr;           // per case [rows][words]: 64-bit fluid window + index (kNbRowMask)
    int* rows = nullptr;               // [3][total rows]: x = 0, x = 1, x = nx-1 cell of each row (-1 if solid)
    int2* case_rows = nullptr;         // [cases]: first row, row count
    void* cases = nullptr;             // [cases] CaseBC<XS> (inlet values, outlet flux, range)
    int* blk_case[kStepVariants] = {};  // step-kernel block -> case
    int2* segs = nullptr;              // [segments]: first cell, cell count (reduction segments)
    int2* case_segs = nullptr;         // [cases]: first segment, segment count
    int* seg_case = nullptr;           // [segments]: case of each segment
    double* partials = nullptr;        // [segments][10]
    double* extrap = nullptr;          // [3][S] X of the last extrapolation check (lazy)
    double* coef = nullptr;            // [cases] extrapolation factors
    double* rre_ring = nullptr;        // [order + 1][3][S] X snapshots of a reduced-rank extrapolation cycle (lazy)
    double* rre_partials = nullptr;    // [segments][order (order + 1) / 2] Gram partials (lazy)
    double* rre_out = nullptr;         // [cases][order (order + 1) / 2] Gram matrices (lazy)
    double* rre_coef = nullptr;        // [cases][order] coefficients of the differences (lazy)
    double* case_out = nullptr;        // [cases][10] residual sums, then [cases][6] boundary sums
    void* fields = nullptr;            // [3 + 3 dim][S] of tau and u (lazy), FP64 or FP32
};

struct Launch {
    int dim = 2;
    int precision = 1;                 // 0 = FP64, 1 = FP32, 2 = FP16 populations / FP32 compute
    int64_t S = 0;                     // padded row stride (elements), >= ncells
    int ncells = 0;                    // end of the last case's range (index space of the kernels)
    int n_cases = 1;
    int total_rows = 0;
    int n_segs = 0;
    int nblk[kStepVariants] = {};
    int variant = 0;                   // chosen step-kernel tile shape
    int cur = 0;                       // lattice holding the latest post-collision state
    DevBuffers b;
    double D12 = 1, D13 = 1, D23 = 1;  // lattice binary diffusivities
    double stoich[3] = {-1, 1, 0};     // nu_i of the electrode reaction (Eq. 38)
    double tau_min = 1.0, tau_max = 5.0;
    int drift = 1;
    int grad_forward = 0;              // Eq. 35 forward difference along x only
    int outlet_extrap = 0;             // extrapolated wet-node outlet (per-cell step kernel only)
    int sm_count = 152;
};

// Host image of one case's boundary data; the launcher converts it to the
// device CaseBC layout of the precision in use.
struct CaseHostBC {
    double xin[3];
    double q[3];
    int base;
    int nf;
    int nx, ny, nz;     // grid of the case
    int wpr;            // row-table entries per (y, z) row: ceil(nx / 32)
    int tab;            // first row-table entry of the case
};

size_t pop_size(int precision);    // bytes per stored population
size_t x_size(int precision);      // bytes per stored mole fraction
size_t field_size(int precision);  // bytes per tau / u value of the fields kernel
size_t case_bc_size(int precision);
void pack_case_bc(int precision, const CaseHostBC& h, void* dst);  // host-side CaseBC image

cudaError_t launch_step(const Launch& L, cudaStream_t st);
cudaError_t launch_step_variant(const Launch& L, int variant, cudaStream_t st);
// the same with the grad_forward / outlet_extrap options compiled in
cudaError_t launch_step_variant_literal(const Launch& L, int variant, cudaStream_t st);
cudaError_t launch_init(const Launch& L, int first, int count, cudaStream_t st);
cudaError_t launch_fields(const Launch& L, cudaStream_t st);
cudaError_t launch_case_residuals(const Launch& L, int update, cudaStream_t st);
cudaError_t launch_case_boundary(const Launch& L, cudaStream_t st);
// per-case sums of (X - E)^2 etc. into case_out[c * 10 + v], E unchanged
cudaError_t launch_case_extrap_norms(const Launch& L, cudaStream_t st);
cudaError_t launch_extrapolate(const Launch& L, cudaStream_t st);
// reduced-rank extrapolation of order M (2..6): snapshot into slot, Gram
// matrices of the M differences into rre_out, and the update from rre_coef
cudaError_t launch_rre_snapshot(const Launch& L, int slot, cudaStream_t st);
cudaError_t launch_rre_gram(const Launch& L, int order, cudaStream_t st);
cudaError_t launch_rre_apply(const Launch& L, int order, cudaStream_t st);
constexpr int kRreMaxOrder = 6;

// Neighbour tables of one case built on the device from its dense
// fluid-index map (index_of[cell] = index in the case or -1) and its fluid
// cell list; nbr16 may be null.  counts[0..1] accumulate the fluid links and
// the links that do not fit the 16-bit table.
cudaError_t launch_build_neighbours(int dim, const int64_t* fluid_cell, const int* index_of, int nf, int base, int nx,
                                    int ny, int nz, int periodic_x, int* nbr, int16_t* nbr16,
                                    unsigned long long* counts, cudaStream_t st);
cudaError_t launch_fill16(int16_t* p, int64_t n, int16_t v, cudaStream_t st);

// BF16 "TN" matrix product of the warm-start network on the tcgen05 tensor
// cores (lbms_umma.cu): P[z][M][N] = A[M][K chunk z] . B[N][K chunk z]^T,
// FP32.  Needs N a multiple of 64, (K / S) a multiple of 64, 16-byte aligned
// operands with row strides a multiple of 8 elements; M is free.  *err is
// raised if a wait in the kernel timed out.
cudaError_t umma_gemm_init();
bool umma_gemm_supported(const void* A, int lda, const void* B, int ldb, int M, int N, int K, int S);
cudaError_t umma_gemm_tn(const void* A, int lda, const void* B, int ldb, float* P, int M, int N, int K, int S,
                         unsigned int* err, cudaStream_t st);

// Tap table of the 3-D U-Net's convolutions on the tcgen05 kernel: per tap
// t = 9 (dz + 1) + 3 (dy + 1) + (dx + 1) a row offset in the zero-halo layout
// of the activations.  umma_conv_gemm: P[r][n] = sum_t sum_c x[r + off[t]][c]
// W[n][t C + c] over rows r of x [rows][C] (C = 64 per_tap), W [N][27 C].
// umma_wgrad_gemm: P[z][t C + c][n] = sum_{r in chunk z}
// xT[t % 3][c][r + off[t]] dzT[n][r] with xT[j] [C][rows], dzT [N][rows]
// (per_tap = C, a multiple of 64; N a multiple of 64; each off a multiple of
// 8).  Both read zeros outside their operands' extents.
struct ConvTaps {
    int per_tap = 1;
    int off[27] = {};
};
// Optional epilogue of umma_conv_gemm: instead of FP32 P, out[r][n] =
// BF16(relu(P[r][n] + bias[n])) on the interior rows of the zero-halo layout
// (volumes of X x Y x Z voxels in Xp x Yp x Zp rows, R rows in all) and 0 on
// every other row.
struct ConvEpilogue {
    const float* bias = nullptr;
    void* out = nullptr;          // BF16 [rows][N]
    int X = 0, Y = 0, Z = 0, Xp = 0, Yp = 0, Zp = 0;
    long long R = 0;
};
cudaError_t umma_conv_gemm(const void* x, int rows, int C, const void* W, int N, const ConvTaps& taps, float* P,
                           unsigned int* err, cudaStream_t st, const ConvEpilogue* ep = nullptr);
cudaError_t umma_wgrad_gemm(const void* dzT, int N, const void* const xT[3], int C, int rows, int S,
                            const ConvTaps& taps, float* P, unsigned int* err, cudaStream_t st);

// Read-only view of one case of a handle (for the warm-start network).
struct CaseView {
    int nx, ny, nz;
    int64_t N;                    // cells of the dense grid
    int nf;                       // fluid cells
    const int64_t* fluid_cell;    // dense index of each fluid cell (host)
    double x_in[3];
    double current;               // A/cm2
    bool periodic_x;
    bool has_bc;
};
// False if k is out of range.
bool case_view(const lbms_ctx* c, int k, CaseView* v);
// The initial profile of Section 4.1 for case k at its current boundary
// data, prof[s * nx + x]; false if it goes negative (or the box is periodic
// in x).
bool case_profile_1d(const lbms_ctx* c, int k, std::vector<double>& prof);

}  // namespace lbms
