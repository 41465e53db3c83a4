// Kernel instantiations and launch wrappers: D2Q9 / D3Q19 x
//   FP64   (X double,                          h double)
//   FP32   (X double-float pair in FP32 words, h float)
//   FP16   (X double-float pair in FP32 words, h half, FP32 arithmetic)
// and the step-kernel tile shapes of kVariantCells / kVariantMinBlocks.
#include <algorithm>
#include <cstring>

#include "lbms_internal.h"
#include "lbms_kernels.cuh"
#include "lbms_step_launch.cuh"

namespace lbms {

using launch_detail::make_const;

namespace {

constexpr int kBlock = 256;

inline void to_x(double v, Xv<double>& out) { out.v = v; }
inline void to_x(double v, Xv<float>& out) {
    out.hi = (float)v;
    out.lo = (float)(v - (double)out.hi);
}

template <typename XS>
void pack_t(const CaseHostBC& h, void* dst) {
    CaseBC<XS> c;
    std::memset(&c, 0, sizeof(c));
    for (int s = 0; s < 3; ++s) {
        to_x(h.xin[s], c.xbc[s]);
        c.qout[s] = typename Xv<XS>::T(h.q[s]);
    }
    c.base = h.base;
    c.nf = h.nf;
    c.nx = h.nx;
    c.ny = h.ny;
    c.nz = h.nz;
    c.wpr = h.wpr;
    c.tab = h.tab;
    std::memcpy(dst, &c, sizeof(c));
}

template <class Lat, typename XS, typename P>
cudaError_t init_t(const Launch& L, int first, int count, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    const int grid = (count + kBlock - 1) / kBlock;
    init_kernel<Lat, XS, P><<<grid, kBlock, 0, st>>>(static_cast<P*>(L.b.f[L.cur]),
                                                     static_cast<const XS*>(L.b.X[L.cur]),
                                                     static_cast<XS*>(L.b.X[L.cur ^ 1]), L.b.snap, L.S, first, count);
    return cudaGetLastError();
}

template <class Lat, typename XS, typename P>
cudaError_t fields_t(const Launch& L, cudaStream_t st) {
    using T = typename Xv<XS>::T;
    const int grid = (L.ncells + kBlock - 1) / kBlock;
    T* base = static_cast<T*>(L.b.fields);
    fields_kernel<Lat, XS><<<grid, kBlock, 0, st>>>(static_cast<const XS*>(L.b.X[L.cur]),
                                                    static_cast<const XS*>(L.b.X[L.cur ^ 1]), L.b.nbr, L.S,
                                                    L.ncells, make_const<T>(L), base, base + 3 * L.S);
    return cudaGetLastError();
}

template <typename XS>
cudaError_t residual_t(const Launch& L, int update, cudaStream_t st) {
    seg_residual_kernel<XS><<<L.n_segs, kSegThreads, 0, st>>>(static_cast<const XS*>(L.b.X[L.cur]), L.b.snap, L.S,
                                                              L.b.segs, update, L.b.partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // per-case sums land in case_out[c * 10 + v]
    seg_finalize_kernel<10><<<L.n_cases, kSegThreads, 0, st>>>(L.b.partials, L.b.case_segs, L.b.case_out);
    return cudaGetLastError();
}

template <typename XS>
cudaError_t extrap_norms_t(const Launch& L, cudaStream_t st) {
    seg_residual_kernel<XS><<<L.n_segs, kSegThreads, 0, st>>>(static_cast<const XS*>(L.b.X[L.cur]), L.b.extrap, L.S,
                                                              L.b.segs, 0, L.b.partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    seg_finalize_kernel<10><<<L.n_cases, kSegThreads, 0, st>>>(L.b.partials, L.b.case_segs, L.b.case_out);
    return cudaGetLastError();
}

template <typename XS>
cudaError_t extrapolate_t(const Launch& L, cudaStream_t st) {
    seg_extrapolate_kernel<XS><<<L.n_segs, kSegThreads, 0, st>>>(static_cast<XS*>(L.b.X[L.cur]),
                                                                 static_cast<XS*>(L.b.X[L.cur ^ 1]), L.b.extrap, L.S,
                                                                 L.b.segs, L.b.seg_case, L.b.coef);
    return cudaGetLastError();
}

template <class Lat, typename XS, typename P>
cudaError_t boundary_t(const Launch& L, cudaStream_t st) {
    // per-case sums land in case_out[n_cases * 10 + c * 6 + v]
    case_boundary_kernel<Lat, XS, P><<<L.n_cases, kSegThreads, 0, st>>>(
        static_cast<const P*>(L.b.f[L.cur]), static_cast<const XS*>(L.b.X[L.cur]), L.b.nbr, L.S, L.b.rows,
        L.b.rows + L.total_rows, L.b.rows + 2 * L.total_rows, L.b.case_rows,
        L.b.case_out + (int64_t)L.n_cases * 10);
    return cudaGetLastError();
}

}  // namespace

size_t pop_size(int precision) { return precision == 0 ? sizeof(double) : (precision == 1 ? sizeof(float) : 2); }
size_t x_size(int precision) { return precision == 0 ? sizeof(double) : 2 * sizeof(float); }
size_t field_size(int precision) { return precision == 0 ? sizeof(double) : sizeof(float); }
size_t case_bc_size(int precision) { return precision == 0 ? sizeof(CaseBC<double>) : sizeof(CaseBC<float>); }

void pack_case_bc(int precision, const CaseHostBC& h, void* dst) {
    if (precision == 0)
        pack_t<double>(h, dst);
    else
        pack_t<float>(h, dst);
}

#define LBMS_DISPATCH(FN, ...)                                                              \
    do {                                                                                    \
        if (L.dim == 2) {                                                                   \
            if (L.precision == 0) return FN<D2Q9, double, double>(__VA_ARGS__);             \
            if (L.precision == 1) return FN<D2Q9, float, float>(__VA_ARGS__);               \
            return FN<D2Q9, float, __half>(__VA_ARGS__);                                    \
        }                                                                                   \
        if (L.precision == 0) return FN<D3Q19, double, double>(__VA_ARGS__);                \
        if (L.precision == 1) return FN<D3Q19, float, float>(__VA_ARGS__);                  \
        return FN<D3Q19, float, __half>(__VA_ARGS__);                                       \
    } while (0)

cudaError_t launch_step_variant(const Launch& L, int variant, cudaStream_t st) {
    using launch_detail::step_t;
    if (L.grad_forward || L.outlet_extrap) return launch_step_variant_literal(L, variant, st);
    LBMS_STEP_DISPATCH(false);
}
cudaError_t launch_step(const Launch& L, cudaStream_t st) { return launch_step_variant(L, L.variant, st); }

cudaError_t launch_init(const Launch& L, int first, int count, cudaStream_t st) {
    LBMS_DISPATCH(init_t, L, first, count, st);
}
cudaError_t launch_fields(const Launch& L, cudaStream_t st) { LBMS_DISPATCH(fields_t, L, st); }
cudaError_t launch_case_boundary(const Launch& L, cudaStream_t st) { LBMS_DISPATCH(boundary_t, L, st); }

cudaError_t launch_case_extrap_norms(const Launch& L, cudaStream_t st) {
    return L.precision == 0 ? extrap_norms_t<double>(L, st) : extrap_norms_t<float>(L, st);
}

cudaError_t launch_extrapolate(const Launch& L, cudaStream_t st) {
    return L.precision == 0 ? extrapolate_t<double>(L, st) : extrapolate_t<float>(L, st);
}

cudaError_t launch_rre_snapshot(const Launch& L, int slot, cudaStream_t st) {
    if (L.precision == 0)
        seg_snapshot_kernel<double><<<L.n_segs, kSegThreads, 0, st>>>(static_cast<const double*>(L.b.X[L.cur]),
                                                                      L.b.rre_ring, L.S, L.b.segs, slot);
    else
        seg_snapshot_kernel<float><<<L.n_segs, kSegThreads, 0, st>>>(static_cast<const float*>(L.b.X[L.cur]),
                                                                     L.b.rre_ring, L.S, L.b.segs, slot);
    return cudaGetLastError();
}

namespace {
template <int M>
cudaError_t rre_gram_m(const Launch& L, cudaStream_t st) {
    constexpr int NV = M * (M + 1) / 2;
    seg_gram_kernel<M><<<L.n_segs, kSegThreads, 0, st>>>(L.b.rre_ring, L.S, L.b.segs, L.b.rre_partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    seg_finalize_kernel<NV><<<L.n_cases, kSegThreads, 0, st>>>(L.b.rre_partials, L.b.case_segs, L.b.rre_out);
    return cudaGetLastError();
}
template <int M>
cudaError_t rre_apply_m(const Launch& L, cudaStream_t st) {
    if (L.precision == 0)
        seg_rre_apply_kernel<double, M><<<L.n_segs, kSegThreads, 0, st>>>(
            static_cast<double*>(L.b.X[L.cur]), static_cast<double*>(L.b.X[L.cur ^ 1]), L.b.rre_ring, L.S, L.b.segs,
            L.b.seg_case, L.b.rre_coef);
    else
        seg_rre_apply_kernel<float, M><<<L.n_segs, kSegThreads, 0, st>>>(
            static_cast<float*>(L.b.X[L.cur]), static_cast<float*>(L.b.X[L.cur ^ 1]), L.b.rre_ring, L.S, L.b.segs,
            L.b.seg_case, L.b.rre_coef);
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_rre_gram(const Launch& L, int order, cudaStream_t st) {
    switch (order) {
        case 2: return rre_gram_m<2>(L, st);
        case 3: return rre_gram_m<3>(L, st);
        case 4: return rre_gram_m<4>(L, st);
        case 5: return rre_gram_m<5>(L, st);
        case 6: return rre_gram_m<6>(L, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_rre_apply(const Launch& L, int order, cudaStream_t st) {
    switch (order) {
        case 2: return rre_apply_m<2>(L, st);
        case 3: return rre_apply_m<3>(L, st);
        case 4: return rre_apply_m<4>(L, st);
        case 5: return rre_apply_m<5>(L, st);
        case 6: return rre_apply_m<6>(L, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_case_residuals(const Launch& L, int update, cudaStream_t st) {
    return L.precision == 0 ? residual_t<double>(L, update, st) : residual_t<float>(L, update, st);
}

}  // namespace lbms
