// Kernel instantiations and launch wrappers: D2Q9 / D3Q19 x
//   FP64   (X double,                          h double)
//   FP32   (X double-float pair in FP32 words, h float)
//   FP16   (X double-float pair in FP32 words, h half, FP32 arithmetic)
// and the step-kernel tile shapes of kVariantCells / kVariantMinBlocks.
#include <algorithm>
#include <cstring>

#include "lbms_internal.h"
#include "lbms_kernels.cuh"

namespace lbms {

namespace {

constexpr int kBlock = 256;

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
    std::memcpy(dst, &c, sizeof(c));
}

template <class Lat, typename XS, typename P, typename NBT, int W, int MB, bool PER_CELL = false>
cudaError_t step_w(const Launch& L, int variant, cudaStream_t st) {
    using T = typename Xv<XS>::T;
    StepParams<XS, P, NBT> p;
    p.hin = static_cast<const P*>(L.b.f[L.cur]);
    p.hout = static_cast<P*>(L.b.f[L.cur ^ 1]);
    p.xin = static_cast<const XS*>(L.b.X[L.cur]);
    p.xout = static_cast<XS*>(L.b.X[L.cur ^ 1]);
    if constexpr (sizeof(NBT) == 2)
        p.nbr = L.b.nbr16;
    else
        p.nbr = L.b.nbr;
    p.nbr32 = L.b.nbr;
    p.cases = static_cast<const CaseBC<XS>*>(L.b.cases);
    p.blk_case = L.b.blk_case[variant];
    p.S = L.S;
    // L2 prefetch distance: a fraction of a wave of resident blocks (per-cell kernel only)
    p.pf_dist = PER_CELL ? L.sm_count * MB * W / prefetch_wave_divisor<P>() : 0;
    p.c = make_const<T>(L);
    if constexpr (PER_CELL)
        step_kernel_cell<Lat, XS, P, NBT, W, MB><<<L.nblk[variant], W, 0, st>>>(p);
    else
        step_kernel<Lat, XS, P, NBT, W, MB><<<L.nblk[variant], 3 * W, 0, st>>>(p);
    return cudaGetLastError();
}

template <class Lat, typename XS, typename P>
cudaError_t step_t(const Launch& L, int variant, cudaStream_t st) {
    static_assert(kStepVariants == 8 && kVariantPerCell[6] && kVariantPerCell[7] && !kVariantPerCell[5],
                  "variant table");
    switch (variant) {
        case 0: return step_w<Lat, XS, P, int, kVariantCells[0], kVariantMinBlocks[0]>(L, 0, st);
        case 1: return step_w<Lat, XS, P, int, kVariantCells[1], kVariantMinBlocks[1]>(L, 1, st);
        case 2: return step_w<Lat, XS, P, int, kVariantCells[2], kVariantMinBlocks[2]>(L, 2, st);
        case 3: return step_w<Lat, XS, P, int16_t, kVariantCells[3], kVariantMinBlocks[3]>(L, 3, st);
        case 4: return step_w<Lat, XS, P, int16_t, kVariantCells[4], kVariantMinBlocks[4]>(L, 4, st);
        case 5: return step_w<Lat, XS, P, int16_t, kVariantCells[5], kVariantMinBlocks[5]>(L, 5, st);
        case 6: return step_w<Lat, XS, P, int, kVariantCells[6], kVariantMinBlocks[6], true>(L, 6, st);
        default: return step_w<Lat, XS, P, int, kVariantCells[7], kVariantMinBlocks[7], true>(L, 7, st);
    }
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
    LBMS_DISPATCH(step_t, L, variant, st);
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

cudaError_t launch_case_residuals(const Launch& L, int update, cudaStream_t st) {
    return L.precision == 0 ? residual_t<double>(L, update, st) : residual_t<float>(L, update, st);
}

}  // namespace lbms
