// Step-kernel launch templates shared by the two translation units that
// instantiate them: lbms_launch.cu (default readings, LIT = false) and
// lbms_launch_literal.cu (the grad_forward / outlet_extrap options,
// LIT = true), compiled in parallel.
#pragma once

#include "lbms_internal.h"
#include "lbms_kernels.cuh"

namespace lbms {
namespace launch_detail {

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
    c.grad_forward = L.grad_forward;
    c.outlet_extrap = L.outlet_extrap;
    return c;
}

template <class Lat, typename XS, typename P, typename NBT, int W, int MB, bool PER_CELL, bool LIT>
cudaError_t step_w(const Launch& L, int variant, cudaStream_t st) {
    using T = typename Xv<XS>::T;
    StepParams<XS, P, NBT> p;
    p.hin = static_cast<const P*>(L.b.f[L.cur]);
    p.hout = static_cast<P*>(L.b.f[L.cur ^ 1]);
    p.xin = static_cast<const XS*>(L.b.X[L.cur]);
    p.xout = static_cast<XS*>(L.b.X[L.cur ^ 1]);
    if constexpr (std::is_same<NBT, RowMaskNb>::value)
        p.nbr = nullptr;
    else if constexpr (sizeof(NBT) == 2)
        p.nbr = L.b.nbr16;
    else
        p.nbr = L.b.nbr;
    p.nbr32 = L.b.nbr;
    p.cell_code = L.b.cell_code;
    p.rowtab = L.b.rowtab;
    p.cases = static_cast<const CaseBC<XS>*>(L.b.cases);
    p.blk_case = L.b.blk_case[variant];
    p.S = L.S;
    // L2 prefetch distance: a fraction of a wave of resident blocks (per-cell kernel only)
    p.pf_dist = PER_CELL ? L.sm_count * MB * W / prefetch_wave_divisor<P>() : 0;
    p.c = make_const<T>(L);
    if constexpr (PER_CELL)
        step_kernel_cell<Lat, XS, P, NBT, W, MB, LIT><<<L.nblk[variant], W, 0, st>>>(p);
    else
        step_kernel<Lat, XS, P, NBT, W, MB, LIT><<<L.nblk[variant], 3 * W, 0, st>>>(p);
    return cudaGetLastError();
}

template <class Lat, typename XS, typename P, bool LIT>
cudaError_t step_t(const Launch& L, int variant, cudaStream_t st) {
    static_assert(kStepVariants == 10 && kVariantPerCell[6] && kVariantPerCell[7] && !kVariantPerCell[5] &&
                      kVariantNb[8] == kNbRowMask && kVariantNb[9] == kNbRowMask && kVariantPerCell[8] &&
                      kVariantPerCell[9],
                  "variant table");
    switch (variant) {
        case 0: return step_w<Lat, XS, P, int, kVariantCells[0], kVariantMinBlocks[0], false, LIT>(L, 0, st);
        case 1: return step_w<Lat, XS, P, int, kVariantCells[1], kVariantMinBlocks[1], false, LIT>(L, 1, st);
        case 2: return step_w<Lat, XS, P, int, kVariantCells[2], kVariantMinBlocks[2], false, LIT>(L, 2, st);
        case 3: return step_w<Lat, XS, P, int16_t, kVariantCells[3], kVariantMinBlocks[3], false, LIT>(L, 3, st);
        case 4: return step_w<Lat, XS, P, int16_t, kVariantCells[4], kVariantMinBlocks[4], false, LIT>(L, 4, st);
        case 5: return step_w<Lat, XS, P, int16_t, kVariantCells[5], kVariantMinBlocks[5], false, LIT>(L, 5, st);
        case 6: return step_w<Lat, XS, P, int, kVariantCells[6], kVariantMinBlocks[6], true, LIT>(L, 6, st);
        case 7: return step_w<Lat, XS, P, int, kVariantCells[7], kVariantMinBlocks[7], true, LIT>(L, 7, st);
        case 8: return step_w<Lat, XS, P, RowMaskNb, kVariantCells[8], kVariantMinBlocks[8], true, LIT>(L, 8, st);
        default: return step_w<Lat, XS, P, RowMaskNb, kVariantCells[9], kVariantMinBlocks[9], true, LIT>(L, 9, st);
    }
}

#define LBMS_STEP_DISPATCH(LIT)                                                            \
    do {                                                                                   \
        if (L.dim == 2) {                                                                  \
            if (L.precision == 0) return step_t<D2Q9, double, double, LIT>(L, variant, st); \
            if (L.precision == 1) return step_t<D2Q9, float, float, LIT>(L, variant, st);   \
            return step_t<D2Q9, float, __half, LIT>(L, variant, st);                       \
        }                                                                                  \
        if (L.precision == 0) return step_t<D3Q19, double, double, LIT>(L, variant, st);   \
        if (L.precision == 1) return step_t<D3Q19, float, float, LIT>(L, variant, st);     \
        return step_t<D3Q19, float, __half, LIT>(L, variant, st);                          \
    } while (0)

}  // namespace launch_detail
}  // namespace lbms
