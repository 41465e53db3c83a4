// Kernel instantiations and launch wrappers: D2Q9 / D3Q19 x
//   FP64   (X double,           h double)
//   FP32   (X double-float pair in FP32 words, h float)
//   FP16   (X double-float pair in FP32 words, h half, FP32 arithmetic)
#include <algorithm>

#include "lbms_internal.h"
#include "lbms_kernels.cuh"

namespace lbms {

namespace {

constexpr int kBlock = 256;
constexpr int kCells = 32;     // cells per block of the step kernel (3 threads per cell)

template <typename T>
MsConst<T> make_const(const Launch& L) {
    MsConst<T> c;
    const double Dl[3][3] = {{0.0, L.D12, L.D13}, {L.D12, 0.0, L.D23}, {L.D13, L.D23, 0.0}};
    c.i12 = T(1.0 / L.D12);
    c.i13 = T(1.0 / L.D13);
    c.i23 = T(1.0 / L.D23);
    for (int i = 0; i < 3; ++i) {
        // Eq. 24 with N_j / N_i = nu_j / nu_i: 1/D_i = sum_{j!=i} (X_j - X_i nu_j / nu_i) / D_ij
        c.reacting[i] = L.stoich[i] != 0.0 ? 1 : 0;
        double hs = 0.0, aii = 0.0;
        for (int j = 0; j < 3; ++j) {
            if (j == i) continue;
            c.a[i][j] = T(1.0 / Dl[i][j]);
            hs += 0.5 / Dl[i][j];
            if (c.reacting[i]) aii -= (L.stoich[j] / L.stoich[i]) / Dl[i][j];
        }
        c.a[i][i] = T(aii);
        c.h[i] = T(hs);
    }
    c.tau_min = T(L.tau_min);
    c.tau_max = T(L.tau_max);
    c.drift = L.drift;
    return c;
}

inline void to_x(double v, Xv<double>& out) { out.v = v; }
inline void to_x(double v, Xv<float>& out) {
    out.hi = (float)v;
    out.lo = (float)(v - (double)out.hi);
}

template <class Lat, typename XT, typename P>
cudaError_t step_t(const Launch& L, cudaStream_t st) {
    using T = typename Xv<XT>::T;
    StepParams<XT, P> p;
    p.hin = static_cast<const P*>(L.b.f[L.cur]);
    p.hout = static_cast<P*>(L.b.f[L.cur ^ 1]);
    p.xin = static_cast<const XT*>(L.b.X[L.cur]);
    p.xout = static_cast<XT*>(L.b.X[L.cur ^ 1]);
    p.nbr = L.b.nbr;
    p.S = L.S;
    p.nf = L.nf;
    for (int s = 0; s < 3; ++s) {
        to_x(L.xin[s], p.xbc[s]);
        p.qout[s] = T(L.q[s]);
    }
    p.c = make_const<T>(L);
    const int grid = (L.nf + kCells - 1) / kCells;
    step_kernel<Lat, XT, P, kCells><<<grid, 3 * kCells, 0, st>>>(p);
    return cudaGetLastError();
}

template <class Lat, typename XT, typename P>
cudaError_t init_t(const Launch& L, cudaStream_t st) {
    const int grid = (L.nf + kBlock - 1) / kBlock;
    init_kernel<Lat, XT, P><<<grid, kBlock, 0, st>>>(static_cast<P*>(L.b.f[L.cur]),
                                                     static_cast<const XT*>(L.b.X[L.cur]),
                                                     static_cast<XT*>(L.b.X[L.cur ^ 1]), L.b.snap, L.S, L.nf);
    return cudaGetLastError();
}

template <class Lat, typename XT, typename P>
cudaError_t fields_t(const Launch& L, cudaStream_t st) {
    using T = typename Xv<XT>::T;
    const int grid = (L.nf + kBlock - 1) / kBlock;
    T* base = static_cast<T*>(L.b.fields);
    fields_kernel<Lat, XT><<<grid, kBlock, 0, st>>>(static_cast<const XT*>(L.b.X[L.cur]),
                                                    static_cast<const XT*>(L.b.X[L.cur ^ 1]), L.b.nbr, L.S, L.nf,
                                                    make_const<T>(L), base, base + 3 * L.S);
    return cudaGetLastError();
}

template <typename XT>
cudaError_t residual_t(const Launch& L, int update, cudaStream_t st) {
    residual_kernel<XT><<<residual_blocks(L), kBlock, 0, st>>>(
        static_cast<const XT*>(L.b.X[L.cur]), L.b.snap, L.S, L.nf, update, L.b.red_partials,
        L.b.red_counter + kRedResidual, L.b.red_out + kRedResidual * kRedSlots);
    return cudaGetLastError();
}

template <class Lat, typename XT, typename P>
cudaError_t boundary_t(const Launch& L, cudaStream_t st) {
    const int blocks = std::max(1, std::min((L.nrows + kBlock - 1) / kBlock, kRedMaxBlocks / 2));
    boundary_kernel<Lat, XT, P><<<blocks, kBlock, 0, st>>>(
        static_cast<const P*>(L.b.f[L.cur]), static_cast<const XT*>(L.b.X[L.cur]), L.b.nbr, L.S, L.b.rows,
        L.b.rows + L.nrows, L.b.rows + 2 * L.nrows, L.nrows, L.b.red_partials + kRedMaxBlocks * kRedSlots / 2,
        L.b.red_counter + kRedBoundary, L.b.red_out + kRedBoundary * kRedSlots);
    return cudaGetLastError();
}

}  // namespace

size_t pop_size(int precision) { return precision == 0 ? sizeof(double) : (precision == 1 ? sizeof(float) : 2); }
size_t x_size(int precision) { return precision == 0 ? sizeof(double) : 2 * sizeof(float); }
size_t field_size(int precision) { return precision == 0 ? sizeof(double) : sizeof(float); }

int residual_blocks(const Launch& L) {
    const int want = (L.nf + kBlock - 1) / kBlock;
    return std::max(1, std::min(want, std::min(kRedMaxBlocks / 2, 4 * L.sm_count)));
}

#define LBMS_DISPATCH(FN, ...)                                                              \
    do {                                                                                    \
        if (L.dim == 2) {                                                                   \
            if (L.precision == 0) return FN<D2Q9, double, double>(__VA_ARGS__);             \
            if (L.precision == 1) return FN<D2Q9, float, float>(__VA_ARGS__);              \
            return FN<D2Q9, float, __half>(__VA_ARGS__);                                   \
        }                                                                                   \
        if (L.precision == 0) return FN<D3Q19, double, double>(__VA_ARGS__);                \
        if (L.precision == 1) return FN<D3Q19, float, float>(__VA_ARGS__);                 \
        return FN<D3Q19, float, __half>(__VA_ARGS__);                                      \
    } while (0)

cudaError_t launch_step(const Launch& L, cudaStream_t st) { LBMS_DISPATCH(step_t, L, st); }
cudaError_t launch_init(const Launch& L, cudaStream_t st) { LBMS_DISPATCH(init_t, L, st); }
cudaError_t launch_fields(const Launch& L, cudaStream_t st) { LBMS_DISPATCH(fields_t, L, st); }
cudaError_t launch_boundary(const Launch& L, cudaStream_t st) { LBMS_DISPATCH(boundary_t, L, st); }

cudaError_t launch_residual(const Launch& L, int update, cudaStream_t st) {
    return L.precision == 0 ? residual_t<double>(L, update, st) : residual_t<float>(L, update, st);
}

}  // namespace lbms
