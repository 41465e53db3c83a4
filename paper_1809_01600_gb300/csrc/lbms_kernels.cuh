// Device side of the solver: the fused collide + stream + Maxwell-Stefan
// step, the field recomputation, initialisation and the FP64 reductions.
//
// State (compact over the fluid cells, x-fastest order, padded row stride S,
// a multiple of 32 elements), two copies for pull streaming:
//   X[s][i]     mole fraction of species s after the step.  FP64, or a
//               double-float pair of FP32 words, hi in X[s][i] and lo in
//               X[3+s][i], whose sum carries ~48 significant bits, so that
//               per-step changes far below one FP32 ulp still accumulate (a
//               plain FP32 state freezes about ulp / (slowest decay rate)
//               away from the steady state).
//   h[s][k][i]  non-equilibrium part of the post-collision population,
//               h = f* - w_k X, in FP64, FP32 or FP16 (FP16 scaled by 2^14).
//   nbr[i][k-1] fluid index of the source cell x - e_k, or an NB_* code;
//               one row of nb_width() ints per cell, read with 16-byte loads.
//               Where every offset fits, a second table holds src - i in 16
//               bits (nb16_width() per row) and the autotuner may pick it.
// A pulled population is f_k(x) = w_k X(src) + h_k(src).  The step works on
// d_k = f_k(x) - w_k X_old(x) ~ w_k (X(src) - X_old(x)) + h_k(src): small
// numbers whose exchange terms w_k (X(src) - X(x)) are exactly antisymmetric
// between two cells, so streaming conserves every species without depending
// on how the weights round.  With the pair format the exchange terms use the
// hi words only (hi_src - hi_x is exact and antisymmetric); the lo word
// enters the cell's own accumulation, so the steady state is resolved to one
// FP32 ulp of X instead of freezing ulp / (decay rate) away from it.
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "lbms_lattice.cuh"

namespace lbms {

// Guards of the coupling (lattice units).
constexpr double kEpsX = 1.0e-12;      // guard of 1/X_i
constexpr double kMixDelta = 1.0e-12;  // guard of the mixture average
constexpr double kVMax = 0.1;          // bound on the drift velocity |v_i|
constexpr double kDBig = 1.0e30;       // an unbounded D_i (tau then sits at tau_max)

template <typename T>
struct MsConst {
    T i12, i13, i23;      // inverse lattice binary diffusivities 1/D*_ij
    T a[3][3];            // Eq. 24 with stoichiometric flux ratios: 1/D_i = sum_j a[i][j] X_j
    T h[3];               // mean inverse diffusivity seen by each species (mixture-value guard)
    int reacting[3];      // nu_i != 0 (Eq. 24 applies); 0: inert, mixture value
    T tau_min, tau_max;
    int drift;            // 1: drift velocity carries the Maxwell-Stefan flux tau does not
    int grad_forward;     // 1: Eq. 35 literally (forward difference along x only)
    int outlet_extrap;    // 1: outlet as an extrapolated wet node (Eq. 37 reading), per-cell kernel only
};

// One component of the lagged gradient (Eq. 35) from the differences to the
// +e_a and -e_a neighbours (pv, mv; 0 for a solid neighbour, the mirror about
// the half-way wall) and whether those neighbours are cells of the grid
// (hp, hm; false beyond the inlet and outlet columns).  Central differences
// on every axis, one-sided at x = 0 and x = nx-1; with `forward`, Eq. 35 as
// printed: the forward difference along x (backward at x = nx-1) and no
// y / z component.
template <typename T>
__device__ __forceinline__ T grad_component(bool hp, bool hm, T pv, T mv, int a, int forward) {
    if (forward) return a == 0 ? (hp ? pv : (hm ? -mv : T(0))) : T(0);
    return (hp && hm) ? T(0.5) * (pv - mv) : (hp ? pv : (hm ? -mv : T(0)));
}

// Neighbour row of cell i: nb[k] for k = 1..Q-1 (nb[0] is left to the caller).
template <class L>
__device__ __forceinline__ void load_neighbours(const int* __restrict__ nbr, int i, int (&nb)[L::Q]) {
    constexpr int NW = nb_width<L>();
    const int4* row = reinterpret_cast<const int4*>(nbr + (int64_t)i * NW);
#pragma unroll
    for (int j = 0; j < NW / 4; ++j) {
        const int4 v = __ldg(row + j);
        if (1 + 4 * j + 0 < L::Q) nb[1 + 4 * j + 0] = v.x;
        if (1 + 4 * j + 1 < L::Q) nb[1 + 4 * j + 1] = v.y;
        if (1 + 4 * j + 2 < L::Q) nb[1 + 4 * j + 2] = v.z;
        if (1 + 4 * j + 3 < L::Q) nb[1 + 4 * j + 3] = v.w;
    }
}

// Neighbours of a fluid cell from the per-row fluid bitmasks (kNbRowMask).
// code = x | y << 11 | z << 21 of the cell (all ones for the padding cells
// between cases, whose links are all solid).  Row-table entry (row, w) of a
// case: .x/.y = bits 0..31/32..63 of a window of fluid flags of the voxels
// x' = 32 w - 16 .. 32 w + 47 of that row (zero outside the grid), .z = the
// fluid index the first fluid voxel at or after x' = 32 w - 16 has (or would
// have).  Fluid cells are numbered in x-fastest order, so the index of a
// fluid voxel is .z plus the number of fluid voxels before it in the window.
// Link k pulls from (x, y, z) - e_k: one entry per source row gives the
// sources x - 1, x and x + 1 of that row.  y and z are periodic; x is not
// (beyond x = 0: inlet; beyond x = nx - 1: outlet).
template <class L>
__host__ __device__ constexpr bool row_used(int dy, int dz) {
    for (int k = 1; k < L::Q; ++k)
        if (-L::e(k, 1) == dy && -L::e(k, 2) == dz) return true;
    return false;
}

template <class L>
__device__ __forceinline__ void decode_neighbours(uint32_t code, const uint4* __restrict__ tab, int nx, int ny,
                                                  int nz, int wpr, int (&nb)[L::Q]) {
    if (code == 0xFFFFFFFFu) {
#pragma unroll
        for (int k = 1; k < L::Q; ++k) nb[k] = NB_SOLID;
        return;
    }
    const int x = (int)(code & 2047u);
    const int y = (int)((code >> 11) & 1023u);
    const int z = (int)(code >> 21);
    const int w = x >> 5;
    const int b = (x & 31) + 16;                       // bit of x in the window, 16..47
    const unsigned long long below = (1ull << b) - 1ull;
    const int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
    const int zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
    const int code_lo = x == 0 ? NB_INLET : NB_SOLID;        // source x - 1 not fluid
    const int code_hi = x == nx - 1 ? NB_OUTLET : NB_SOLID;  // source x + 1 not fluid
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz) {
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
            if (!row_used<L>(dy, dz)) continue;
            const int ys = dy == 0 ? y : (dy < 0 ? ym : yp);
            const int zs = dz == 0 ? z : (dz < 0 ? zm : zp);
            const uint4 e = __ldg(tab + (zs * ny + ys) * wpr + w);
            const unsigned long long win = ((unsigned long long)e.y << 32) | e.x;
            const int c = (int)e.z + __popcll(win & below);          // index x has (or would have)
            const unsigned bits = (unsigned)(win >> (b - 1)) & 7u;   // fluid flags of x - 1, x, x + 1
#pragma unroll
            for (int k = 1; k < L::Q; ++k) {
                if (-L::e(k, 1) != dy || -L::e(k, 2) != dz) continue;
                const int dx = -L::e(k, 0);
                if (dx < 0)
                    nb[k] = (bits & 1u) ? c - 1 : code_lo;
                else if (dx == 0)
                    nb[k] = (bits & 2u) ? c : NB_SOLID;
                else
                    nb[k] = (bits & 4u) ? c + (int)((bits >> 1) & 1u) : code_hi;
            }
        }
    }
}

// Output stores of the step kernel.
template <typename V>
__device__ __forceinline__ void step_store(V* ptr, V v) {
    *ptr = v;
}

// The same row from the 16-bit offset table (links marked NB16_FAR read the
// 32-bit table).
template <class L>
__device__ __forceinline__ void load_neighbours(const int16_t* __restrict__ nbr, const int* __restrict__ nbr32,
                                                int i, int (&nb)[L::Q]) {
    constexpr int NW = nb16_width<L>();
    const int4* row = reinterpret_cast<const int4*>(nbr + (int64_t)i * NW);
#pragma unroll
    for (int j = 0; j < NW / 8; ++j) {
        const int4 v = __ldg(row + j);
        const int w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int h = 0; h < 8; ++h) {
            const int k = 1 + 8 * j + h;
            if (k < L::Q) {
                const int d = (h & 1) ? (w[h >> 1] >> 16) : ((w[h >> 1] << 16) >> 16);
                nb[k] = d < NB16_MIN_OFFSET ? (NB16_SOLID - 1 - d) : i + d;
                if (d == NB16_FAR) nb[k] = __ldg(nbr32 + (int64_t)i * nb_width<L>() + (k - 1));
            }
        }
    }
}

// ------------------------------------------------------------------ storage
// Non-equilibrium populations: P = T, or __half holding h * 2^14.
constexpr float kHalfScale = 16384.0f;
constexpr float kHalfInvScale = 1.0f / 16384.0f;

// load / quant / dequant work in lattice units; raw / quant_raw /
// dequant_raw in storage units (lattice value times kStore).
template <typename T, typename P>
struct Pop {
    static constexpr float kStore = 1.0f;
    __device__ __forceinline__ static T load(const P* p) { return T(*p); }
    __device__ __forceinline__ static P quant(T v) { return P(v); }
    __device__ __forceinline__ static T dequant(P v) { return T(v); }
    __device__ __forceinline__ static T raw(const P* p) { return T(*p); }
    __device__ __forceinline__ static P quant_raw(T v) { return P(v); }
    __device__ __forceinline__ static T dequant_raw(P v) { return T(v); }
};
template <>
struct Pop<float, __half> {
    static constexpr float kStore = kHalfScale;
    __device__ __forceinline__ static float load(const __half* p) { return __half2float(*p) * kHalfInvScale; }
    __device__ __forceinline__ static __half quant(float v) { return __float2half_rn(v * kHalfScale); }
    __device__ __forceinline__ static float dequant(__half v) { return __half2float(v) * kHalfInvScale; }
    __device__ __forceinline__ static float raw(const __half* p) { return __half2float(*p); }
    __device__ __forceinline__ static __half quant_raw(float v) { return __float2half_rn(v); }
    __device__ __forceinline__ static float dequant_raw(__half v) { return __half2float(v); }
};

// Mole fractions.  Xv<double>: one FP64 value.  Xv<float>: a double-float
// pair whose hi word sits at X[s][i] and lo word at X[3+s][i].
template <typename XS>
struct Xv;
template <>
struct Xv<double> {
    using T = double;
    double v;
    __device__ __forceinline__ static Xv own(const double* xb, int64_t S, int s, int i) { return Xv{xb[s * S + i]}; }
    // with the species rows already located (hi = the FP64 row; lo unused)
    __device__ __forceinline__ static Xv own_rows(const double* hi, const double*, int i) { return Xv{hi[i]}; }
    __device__ __forceinline__ void store_rows(double* hi, double*, int i) const { step_store(hi + i, v); }
    // value of a neighbour as used by the exchange terms and the gradient
    __device__ __forceinline__ static T nb(const double* xb, int64_t S, int s, int j) { return xb[s * S + j]; }
    __device__ __forceinline__ T exch(T n) const { return n - v; }          // neighbour minus own
    __device__ __forceinline__ T minus(const Xv& b) const { return v - b.v; }  // full precision
    __device__ __forceinline__ T value() const { return v; }
    __device__ __forceinline__ double to_double() const { return v; }
    __device__ __forceinline__ Xv plus(T d) const { return Xv{v + d}; }
    __device__ __forceinline__ void store(double* xb, int64_t S, int s, int i) const { xb[s * S + i] = v; }
};
template <>
struct Xv<float> {
    using T = float;
    float hi, lo;
    __device__ __forceinline__ static Xv own(const float* xb, int64_t S, int s, int i) {
        return Xv{xb[s * S + i], xb[(3 + s) * S + i]};
    }
    __device__ __forceinline__ static Xv own_rows(const float* hi, const float* lo, int i) { return Xv{hi[i], lo[i]}; }
    __device__ __forceinline__ void store_rows(float* h, float* l, int i) const {
        step_store(h + i, hi);
        step_store(l + i, lo);
    }
    __device__ __forceinline__ static T nb(const float* xb, int64_t S, int s, int j) { return xb[s * S + j]; }
    // hi_n - hi is exact for neighbouring values and antisymmetric between two cells
    __device__ __forceinline__ T exch(T n) const { return n - hi; }
    __device__ __forceinline__ T minus(const Xv& b) const { return (hi - b.hi) + (lo - b.lo); }
    __device__ __forceinline__ T value() const { return hi + lo; }
    __device__ __forceinline__ double to_double() const { return (double)hi + (double)lo; }
    // (hi, lo) + d renormalised with Knuth's two-sum
    __device__ __forceinline__ Xv plus(float d) const {
        const float t = lo + d;
        const float s = hi + t;
        const float bb = s - hi;
        const float e = (hi - (s - bb)) + (t - bb);
        return Xv{s, e};
    }
    __device__ __forceinline__ void store(float* xb, int64_t S, int s, int i) const {
        xb[s * S + i] = hi;
        xb[(3 + s) * S + i] = lo;
    }
};

// Stores an FP64 value into the X format (double, or hi/lo FP32 words).
template <typename XS>
__device__ __forceinline__ void store_x(XS* xb, int64_t S, int s, int i, double v);
template <>
__device__ __forceinline__ void store_x<double>(double* xb, int64_t S, int s, int i, double v) {
    xb[s * S + i] = v;
}
template <>
__device__ __forceinline__ void store_x<float>(float* xb, int64_t S, int s, int i, double v) {
    const float hi = (float)v;
    xb[s * S + i] = hi;
    xb[(3 + s) * S + i] = (float)(v - (double)hi);
}

// Per-case data of a batch.  Every case owns the fluid-index range
// [base, base + nf), with base a multiple of kCaseAlign, so that no block of
// the step kernel spans two cases.
constexpr int kCaseAlign = 64;

template <typename XS>
struct CaseBC {
    Xv<XS> xbc[3];                    // inlet mole fractions (Eq. 36), in the X format
    typename Xv<XS>::T qout[3];       // outlet flux per node per step (Eq. 39)
    int base;                         // first fluid index of the case
    int nf;                           // fluid cells of the case
    int nx, ny, nz;                   // grid (for the row-bitmask neighbour decode)
    int wpr;                          // row-table entries per (y, z) row
    int tab;                          // first row-table entry of the case
};

template <typename XS, typename P, typename NBT>
struct StepParams {
    const P* __restrict__ hin;
    P* __restrict__ hout;
    const XS* __restrict__ xin;
    XS* __restrict__ xout;
    const NBT* __restrict__ nbr;
    const int* __restrict__ nbr32;      // the 32-bit table (for NB16_FAR links)
    const uint32_t* __restrict__ cell_code;   // coordinates of each cell (row-bitmask decode)
    const uint4* __restrict__ rowtab;         // row tables of all cases (row-bitmask decode)
    const CaseBC<XS>* __restrict__ cases;
    const int* __restrict__ blk_case;   // case of each block of W cells
    int64_t S;
    int pf_dist;                        // cells ahead to prefetch into L2 (0 = off)
    MsConst<typename Xv<XS>::T> c;
};

// -------------------------------------------------------------------------
// Maxwell-Stefan coupling of one cell (lattice units, c_s^2 = 1/3), for one
// species s at a time (the step kernel runs one thread per species):
//  B (Eq. 32, species 3 = reference n), J_1,2 = -B^-1 g (Eqs. 31, 33, 34,
//  Gamma = I), J_3 from the n-th row of Eq. 19; D_i from Eq. 24 with the
//  flux ratios of the electrode reaction (nu_j / nu_i), the mixture value
//  for the inert species; tau_i from Eq. 25 clamped; and the drift velocity
//  (velocity slot of Eq. 26) that makes the carried flux the Maxwell-Stefan
//  flux J_i.  FP32 divisions use the fast hardware reciprocal (2 ulp).
template <typename T>
struct Arith {
    __device__ __forceinline__ static T div(T a, T b) { return a / b; }
};
template <>
struct Arith<float> {
    __device__ __forceinline__ static float div(float a, float b) { return __fdividef(a, b); }
};

template <typename T, int DIM>
__device__ __forceinline__ void ms_flux(const T (&X)[3], const T (&g)[3][DIM], const MsConst<T>& c, int s,
                                        T (&J)[DIM]) {
    const T B11 = X[0] * c.i13 + X[1] * c.i12 + X[2] * c.i13;
    const T B12 = -X[0] * (c.i12 - c.i13);
    const T B21 = -X[1] * (c.i12 - c.i23);
    const T B22 = X[1] * c.i23 + X[0] * c.i12 + X[2] * c.i23;
    const T det = B11 * B22 - B12 * B21;
    const T idet = det > T(0) ? Arith<T>::div(T(1), det) : T(0);
    if (s == 0) {
#pragma unroll
        for (int d = 0; d < DIM; ++d) J[d] = -(B22 * g[0][d] - B12 * g[1][d]) * idet;
    } else if (s == 1) {
#pragma unroll
        for (int d = 0; d < DIM; ++d) J[d] = -(B11 * g[1][d] - B21 * g[0][d]) * idet;
    } else {
        const T d3 = X[0] * c.i13 + X[1] * c.i23;
        const T id3 = d3 > T(0) ? Arith<T>::div(T(1), d3) : T(0);
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            const T j1 = -(B22 * g[0][d] - B12 * g[1][d]) * idet;
            const T j2 = -(B11 * g[1][d] - B21 * g[0][d]) * idet;
            J[d] = (-g[2][d] + X[2] * (j1 * c.i13 + j2 * c.i23)) * id3;
        }
    }
}

// tau_s (Eqs. 24-25) and the drift velocity v_s of species s; also returns
// X_s / (X_s^2 + eps^2), the guarded 1/X_s used by the component velocity.
template <typename T, int DIM>
__device__ __forceinline__ void ms_relax(const T (&X)[3], const T (&gs)[DIM], const T (&J)[DIM], const MsConst<T>& c,
                                         int s, T& tau, T (&v)[DIM], T& xinv) {
    const T Xs = s == 0 ? X[0] : (s == 1 ? X[1] : X[2]);
    T D;
    if (c.reacting[s]) {
        const T inv = c.a[s][0] * X[0] + c.a[s][1] * X[1] + c.a[s][2] * X[2];
        D = inv > T(0) ? Arith<T>::div(T(1), inv) : T(kDBig);
    } else {
        // mixture value sum_{j!=s} X_j / sum_{j!=s} X_j / D_sj
        const T md = T(kMixDelta);
        const T num = (s == 0 ? X[1] + X[2] : (s == 1 ? X[0] + X[2] : X[0] + X[1])) + md;
        const T den = (s == 0 ? X[1] * c.i12 + X[2] * c.i13
                              : (s == 1 ? X[0] * c.i12 + X[2] * c.i23 : X[0] * c.i13 + X[1] * c.i23)) +
                      md * c.h[s];
        D = Arith<T>::div(num, den);
    }
    T t = D * T(3) + T(0.5);
    t = t < c.tau_min ? c.tau_min : (t > c.tau_max ? c.tau_max : t);
    tau = t;
    const T Dt = (t - T(0.5)) * T(1.0 / 3.0);
    xinv = Arith<T>::div(Xs, Xs * Xs + T(kEpsX * kEpsX));
    if (c.drift) {
        T vn2 = T(0);
#pragma unroll
        for (int d = 0; d < DIM; ++d) {
            v[d] = (J[d] + Dt * gs[d]) * xinv;
            vn2 += v[d] * v[d];
        }
        if (vn2 > T(kVMax * kVMax)) {
            const T sc = T(kVMax) * rsqrt(vn2);
#pragma unroll
            for (int d = 0; d < DIM; ++d) v[d] *= sc;
        }
    } else {
#pragma unroll
        for (int d = 0; d < DIM; ++d) v[d] = T(0);
    }
}

// -------------------------------------------------------------------------
// One time step for every fluid cell: pull-stream with bounce-back / inlet /
// outlet, moments, lagged gradient, Maxwell-Stefan coupling, BGK collision,
// store h and X.
//
// Thread mapping: a block covers W consecutive fluid cells with 3 W threads,
// one per (species, cell); warps are species-uniform, so every load and store
// of a warp walks consecutive cells of one species row.  The three threads of
// a cell meet once, through shared memory, to exchange X and its gradient for
// the coupling (which needs all species).  LIT = false compiles the default
// readings only (central gradient, flux outlet); LIT = true also honours the
// grad_forward / outlet_extrap options of MsConst.
template <class L, typename XS, typename P, typename NBT, int W, int MB, bool LIT>
__global__ void __launch_bounds__(3 * W, MB) step_kernel(const StepParams<XS, P, NBT> p) {
    using T = typename Xv<XS>::T;
    using XV = Xv<XS>;
    constexpr int Q = L::Q;
    constexpr int DIM = L::DIM;
    __shared__ T sX[3][W];
    __shared__ T sG[3][DIM][W];

    const int s = threadIdx.x / W;          // species of this thread
    const int c = threadIdx.x - s * W;      // cell slot in the block
    const int i = blockIdx.x * W + c;
    // Every thread of the grid runs, padding cells between cases included:
    // their neighbour rows hold only NB_SOLID and their state stays zero, no
    // real cell reads them, so no branch waits for the case lookup below.
    const CaseBC<XS>& cb = p.cases[__ldg(p.blk_case + blockIdx.x)];
    const int64_t S = p.S;
    const int S32 = (int)S;      // Q * S < 2^31 (checked at create): 32-bit offsets in a species block
    const P* hs = p.hin + (int64_t)s * Q * S;
    const XS* xhi = p.xin + (int64_t)s * S;         // X rows of this species (hi, lo)
    const XS* xlo = p.xin + (int64_t)(3 + s) * S;   // (lo row only read in the pair format)

    int nb[Q];
    T d[Q];          // f_k(x) - w_k X_old(x) after streaming
    XV xo, xn;
    T dX = T(0);
    {
        nb[0] = i;
        if constexpr (sizeof(NBT) == 2)
            load_neighbours<L>(p.nbr, p.nbr32, i, nb);
        else
            load_neighbours<L>(p.nbr, i, nb);
        xo = XV::own_rows(xhi, xlo, i);
        T dxs[Q];    // X(src) - X_old(x) for fluid sources, 0 otherwise
        constexpr T wx = T(weight_xplus<L>());
        const T qs = cb.qout[s];
        d[0] = Pop<T, P>::load(hs + i);
        dxs[0] = T(0);
        // Every link loads unconditionally (no branch between the gathers): a
        // fluid source gives h_k(src) and X(src); otherwise the cell's own
        // h_opp(k) (bounce-back and outlet) and its own X, whose difference is 0.
#pragma unroll
        for (int k = 1; k < Q; ++k) {
            const int src = nb[k];
            const bool fluid = src >= 0;
            const P* hp = hs + (fluid ? k * S32 + src : opp<L>(k) * S32 + i);
            const T hv = Pop<T, P>::load(hp);
            const T dx = xo.exch(xhi[fluid ? src : i]);
            T val = T(weight<L>(k)) * dx + hv;
            // only links entering from x = nx (e_x = -1) can carry the outlet flux
            if (L::e(k, 0) == -1) val -= (src == NB_OUTLET ? T(weight<L>(opp<L>(k))) / wx : T(0)) * qs;
            d[k] = val;
            dxs[k] = dx;
        }
        // inlet (Eq. 36): f_k = (w_k + w_opp) X_in - f_opp
        const XV xb = cb.xbc[s];
        const T din = xb.minus(xo);
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            if (L::e(k, 0) == 1) {
                const T inl = T(weight<L>(k) + weight<L>(opp<L>(k))) * din - d[opp<L>(k)];
                d[k] = nb[k] == NB_INLET ? inl : d[k];
            }
        }
        // lagged gradient (Eq. 35 as central differences) from the differences at hand
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            const int kp = 2 + 2 * a;   // source of -e_a: the cell at x + e_a
            const int km = 1 + 2 * a;   // source of +e_a: the cell at x - e_a
            const bool hp = nb[kp] >= NB_SOLID, hm = nb[km] >= NB_SOLID;
            const T pv = dxs[kp], mv = dxs[km];   // solid neighbour -> mirror (0)
            sG[s][a][c] = grad_component(hp, hm, pv, mv, a, LIT ? p.c.grad_forward : 0);
        }
#pragma unroll
        for (int k = 0; k < Q; ++k) dX += d[k];
        xn = xo.plus(dX);
        sX[s][c] = xn.value();
    }
    __syncthreads();

    T X[3], g[3][DIM];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        X[r] = sX[r][c];
#pragma unroll
        for (int a = 0; a < DIM; ++a) g[r][a] = sG[r][a][c];
    }
    T gs[DIM], J[DIM], vs[DIM], ts, xinv;
#pragma unroll
    for (int a = 0; a < DIM; ++a) gs[a] = s == 0 ? g[0][a] : (s == 1 ? g[1][a] : g[2][a]);
    ms_flux<T, DIM>(X, g, p.c, s, J);
    ms_relax<T, DIM>(X, gs, J, p.c, s, ts, vs, xinv);
    const T Xs = s == 0 ? X[0] : (s == 1 ? X[1] : X[2]);

    // BGK collision towards w X (1 + e.v / c_s^2); h* = f* - w X
    const T it = Arith<T>::div(T(1), ts);
    const T keep = T(1) - it;
    P* ho = p.hout + (int64_t)s * Q * S;
    T rest = T(0);
#pragma unroll
    for (int k = 1; k < Q; ++k) {
        T ev = T(0);
#pragma unroll
        for (int a = 0; a < DIM; ++a) ev += T(L::e(k, a)) * vs[a];
        const T w = T(weight<L>(k));
        const T hk = (d[k] - w * dX) * keep + T(3) * w * Xs * ev * it;
        const P q = Pop<T, P>::quant(hk);
        rest -= Pop<T, P>::dequant(q);
        step_store(ho + k * S32 + i, q);
    }
    // the rest population closes sum_k h_k = 0 (mass) on the stored values
    step_store(ho + i, Pop<T, P>::quant(rest));
    xn.store_rows(p.xout + (int64_t)s * S, p.xout + (int64_t)(3 + s) * S, i);
}

// L2 prefetch for the 32 cells starting at wb (a warp's cells a fraction of
// a wave of resident blocks ahead): their neighbour rows and, with 16-bit
// populations, their own populations and mole fractions.  The warp that
// steps those cells later finds its first, dependent loads in L2 instead of
// HBM.  Measured on the 256x128x128 anode: with FP16 populations the full
// prefetch an eighth of a wave ahead saves 8 %; with FP32 populations
// prefetching the populations costs up to 25 % (half a wave ahead) while the
// neighbour rows alone gain about 1 %, so FP32 / FP64 prefetch only those.
// Prefetches load nothing into registers and are issued only for addresses
// inside the buffers (wb + 32 <= S).
__device__ __forceinline__ void prefetch_l2(const void* a) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
}

template <typename P>
constexpr int prefetch_wave_divisor() {
    return sizeof(P) == 2 ? 8 : 4;
}

template <class L, typename XS, typename P, typename NBT>
__device__ __forceinline__ void prefetch_ahead(const StepParams<XS, P, NBT>& p, int64_t wb, int lane) {
    constexpr bool ROWMASK = std::is_same<NBT, RowMaskNb>::value;
    if (wb + 32 > p.S) return;
    constexpr int Q = L::Q;
    if constexpr (sizeof(P) == 2) {
        constexpr int XROWS = sizeof(XS) == 8 ? 3 : 6;    // FP64 X, or hi and lo rows
        constexpr int HB = 32 * (int)sizeof(P);            // bytes of one row segment
        constexpr int XB = 32 * (int)sizeof(XS);
        for (int r = lane; r < 3 * Q + XROWS; r += 32) {
            const char* a = r < 3 * Q ? reinterpret_cast<const char*>(p.hin + (int64_t)r * p.S + wb)
                                      : reinterpret_cast<const char*>(p.xin + (int64_t)(r - 3 * Q) * p.S + wb);
            const int nb = r < 3 * Q ? HB : XB;
            for (int o = 0; o < nb; o += 128) prefetch_l2(a + o);
        }
    }
    if constexpr (ROWMASK) {
        if (lane == 0) prefetch_l2(p.cell_code + wb);     // 32 coordinates: one 128-byte line
    } else {
        constexpr int NW = sizeof(NBT) == 2 ? nb16_width<L>() : nb_width<L>();
        constexpr int NBYTES = 32 * NW * (int)sizeof(NBT);
        const char* nbase = reinterpret_cast<const char*>(p.nbr + wb * NW);
        for (int o = lane * 128; o < NBYTES; o += 32 * 128) prefetch_l2(nbase + o);
    }
}

// Second half of a per-cell step, after the streamed populations of the
// cell are in sD (storage units, d_k = f_k - w_k X_old, column t of a
// [3][Q][W] array): boundary rules, gradient, Maxwell-Stefan coupling,
// collision and stores.  acc[s] holds sum_k d_k, dxa the X differences on the
// axis links.
template <class L, typename XS, typename P, typename NBT, int W, bool LIT>
__device__ __forceinline__ void cell_update(const StepParams<XS, P, NBT>& p, const CaseBC<XS>& cb, int t, int i,
                                            const int (&nb)[L::Q], const Xv<XS> (&xo)[3],
                                            typename Xv<XS>::T (&acc)[3],
                                            const typename Xv<XS>::T (&dxa)[3][2 * L::DIM],
                                            typename Xv<XS>::T (*sD)[L::Q][W]) {
    using T = typename Xv<XS>::T;
    using XV = Xv<XS>;
    constexpr int Q = L::Q;
    constexpr int DIM = L::DIM;
    constexpr T sc = T(Pop<T, P>::kStore);
    const int64_t S = p.S;
    const int S32 = (int)S;
    bool at_outlet = false;
#pragma unroll
    for (int k = 1; k < Q; ++k)
        if (L::e(k, 0) == -1) at_outlet = at_outlet || nb[k] == NB_OUTLET;

    T X[3], g[3][DIM], dXs[3];
    XV xn[3];
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        // Extrapolated outlet (Eq. 37 read as a wet node): X_out = X^{t-1}(x-1)
        // + dX, dX_s = sum_j (X_s q_j - X_j q_s) / D_sj (Eq. 19 over one
        // spacing at the outlet fluxes), with X at x - 1 (link 1 pulls from
        // there; the cell's own X where x - 1 is solid, whose difference is 0),
        // then the Eq. 36 rule on the links entering from beyond the outlet.
        if (LIT && p.c.outlet_extrap && at_outlet) {
            T Xn[3];
#pragma unroll
            for (int r = 0; r < 3; ++r) Xn[r] = xo[r].value() + dxa[r][0];
            const T q0 = cb.qout[0], q1 = cb.qout[1], q2 = cb.qout[2];
            T dX;
            if (s == 0)
                dX = (Xn[0] * q1 - Xn[1] * q0) * p.c.i12 + (Xn[0] * q2 - Xn[2] * q0) * p.c.i13;
            else if (s == 1)
                dX = (Xn[1] * q0 - Xn[0] * q1) * p.c.i12 + (Xn[1] * q2 - Xn[2] * q1) * p.c.i23;
            else
                dX = (Xn[2] * q0 - Xn[0] * q2) * p.c.i13 + (Xn[2] * q1 - Xn[1] * q2) * p.c.i23;
            const T xod = (dxa[s][0] + dX) * sc;   // (X_out - X_old(x)) in storage units
#pragma unroll
            for (int k = 1; k < Q; ++k) {
                if (L::e(k, 0) == -1 && nb[k] == NB_OUTLET) {
                    const T v = T(weight<L>(k) + weight<L>(opp<L>(k))) * xod - sD[s][opp<L>(k)][t];
                    acc[s] += v - sD[s][k][t];
                    sD[s][k][t] = v;
                }
            }
        }
        // inlet (Eq. 36): f_k = (w_k + w_opp) X_in - f_opp, replacing the gathered value
        const T din = cb.xbc[s].minus(xo[s]) * sc;
#pragma unroll
        for (int k = 1; k < Q; ++k) {
            if (L::e(k, 0) == 1 && nb[k] == NB_INLET) {
                const T inl = T(weight<L>(k) + weight<L>(opp<L>(k))) * din - sD[s][opp<L>(k)][t];
                acc[s] += inl - sD[s][k][t];
                sD[s][k][t] = inl;
            }
        }
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            const int kp = 2 + 2 * a, km = 1 + 2 * a;
            const bool hp = nb[kp] >= NB_SOLID, hm = nb[km] >= NB_SOLID;
            const T pv = dxa[s][kp - 1], mv = dxa[s][km - 1];
            g[s][a] = grad_component(hp, hm, pv, mv, a, LIT ? p.c.grad_forward : 0);
        }
        dXs[s] = acc[s];
        xn[s] = xo[s].plus(acc[s] * T(1.0 / sc));
        X[s] = xn[s].value();
    }

#pragma unroll
    for (int s = 0; s < 3; ++s) {
        T J[DIM], vs[DIM], ts, xinv;
        ms_flux<T, DIM>(X, g, p.c, s, J);
        ms_relax<T, DIM>(X, g[s], J, p.c, s, ts, vs, xinv);
        const T it = Arith<T>::div(T(1), ts);
        const T keep = T(1) - it;
        const T A = T(3) * sc * X[s] * it;
        P* ho = p.hout + (int64_t)s * Q * S;
        T rest = T(0);
#pragma unroll
        for (int k = 1; k < Q; ++k) {
            T ev = T(0);
#pragma unroll
            for (int a = 0; a < DIM; ++a) ev += T(L::e(k, a)) * vs[a];
            const T w = T(weight<L>(k));
            const T hk = (sD[s][k][t] - w * dXs[s]) * keep + (w * A) * ev;
            const P q = Pop<T, P>::quant_raw(hk);
            rest -= Pop<T, P>::dequant_raw(q);
            step_store(ho + k * S32 + i, q);
        }
        step_store(ho + i, Pop<T, P>::quant_raw(rest));
        xn[s].store_rows(p.xout + (int64_t)s * S, p.xout + (int64_t)(3 + s) * S, i);
    }
}

// -------------------------------------------------------------------------
// The same time step with one thread per fluid cell handling all three
// species: the neighbour decode and the address selection of every link are
// done once per cell instead of once per species thread.  The streamed
// populations d_k wait for the coupling in shared memory (each thread reads
// back only its own column, so no barrier), which keeps the register count
// low enough for a useful number of resident warps.  Everything from the
// gather to the store runs in storage units (h * kStore), so the FP16
// scaling costs one multiply per species instead of one per population.
template <class L, typename XS, typename P, typename NBT, int W, int MB, bool LIT>
__global__ void __launch_bounds__(W, MB) step_kernel_cell(const StepParams<XS, P, NBT> p) {
    using T = typename Xv<XS>::T;
    using XV = Xv<XS>;
    constexpr int Q = L::Q;
    constexpr int DIM = L::DIM;
    constexpr T sc = T(Pop<T, P>::kStore);
    __shared__ T sD[3][Q][W];
    const int t = threadIdx.x;
    const int i = blockIdx.x * W + t;
    const CaseBC<XS>& cb = p.cases[__ldg(p.blk_case + blockIdx.x)];
    const int64_t S = p.S;
    const int S32 = (int)S;
    if (p.pf_dist > 0) prefetch_ahead<L, XS, P, NBT>(p, i - (t & 31) + p.pf_dist, t & 31);
    const P* hs[3];
    const XS* xh[3];
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        hs[s] = p.hin + (int64_t)s * Q * S;
        xh[s] = p.xin + (int64_t)s * S;
    }

    int nb[Q];
    nb[0] = i;
    if constexpr (std::is_same<NBT, RowMaskNb>::value)
        decode_neighbours<L>(__ldg(p.cell_code + i), p.rowtab + cb.tab, cb.nx, cb.ny, cb.nz, cb.wpr, nb);
    else if constexpr (sizeof(NBT) == 2)
        load_neighbours<L>(p.nbr, p.nbr32, i, nb);
    else
        load_neighbours<L>(p.nbr, i, nb);

    XV xo[3];
    T acc[3], qs[3];
    T dxa[3][2 * DIM];   // X(src) - X_old(x) on the axis links 1 .. 2 DIM
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        xo[s] = XV::own_rows(xh[s], p.xin + (int64_t)(3 + s) * S, i);
        const T h0 = Pop<T, P>::raw(hs[s] + i);
        sD[s][0][t] = h0;
        acc[s] = h0;
        qs[s] = (LIT && p.c.outlet_extrap) ? T(0) : cb.qout[s] * sc;
    }
    constexpr T wx = T(weight_xplus<L>());
#pragma unroll
    for (int k = 1; k < Q; ++k) {
        const int src = nb[k];
        const bool fluid = src >= 0;
        const int hoff = fluid ? k * S32 + src : opp<L>(k) * S32 + i;
        const int xidx = fluid ? src : i;
        const bool out = L::e(k, 0) == -1 && src == NB_OUTLET;
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            const T dx = xo[s].exch(xh[s][xidx]);
            T val = T(weight<L>(k) * sc) * dx + Pop<T, P>::raw(hs[s] + hoff);
            if (L::e(k, 0) == -1) val -= out ? T(weight<L>(opp<L>(k))) / wx * qs[s] : T(0);
            sD[s][k][t] = val;
            acc[s] += val;
            if (k <= 2 * DIM) dxa[s][k - 1] = dx;
        }
    }

    cell_update<L, XS, P, NBT, W, LIT>(p, cb, t, i, nb, xo, acc, dxa, sD);
}

// -------------------------------------------------------------------------
// tau and the component velocity of the last step, recomputed from the
// stored fields (X of the step and of the step before).
template <class L, typename XS>
__global__ void fields_kernel(const XS* __restrict__ xcur, const XS* __restrict__ xprev,
                              const int* __restrict__ nbr, int64_t S, int nf, MsConst<typename Xv<XS>::T> c,
                              typename Xv<XS>::T* __restrict__ tau_out, typename Xv<XS>::T* __restrict__ u_out) {
    using T = typename Xv<XS>::T;
    using XV = Xv<XS>;
    constexpr int Q = L::Q;
    constexpr int DIM = L::DIM;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    int nb[Q];
    nb[0] = i;
#pragma unroll
    load_neighbours<L>(nbr, i, nb);
    T X[3], g[3][DIM];
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        X[s] = XV::own(xcur, S, s, i).value();
        const XV xo = XV::own(xprev, S, s, i);
#pragma unroll
        for (int a = 0; a < DIM; ++a) {
            const int cp = nb[2 + 2 * a], cm = nb[1 + 2 * a];
            const bool hp = cp >= NB_SOLID, hm = cm >= NB_SOLID;
            const T pv = cp >= 0 ? xo.exch(XV::nb(xprev, S, s, cp)) : T(0);
            const T mv = cm >= 0 ? xo.exch(XV::nb(xprev, S, s, cm)) : T(0);
            g[s][a] = grad_component(hp, hm, pv, mv, a, c.grad_forward);
        }
    }
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        T J[DIM], v[DIM], gs[DIM], tau, xinv;
#pragma unroll
        for (int a = 0; a < DIM; ++a) gs[a] = g[s][a];
        ms_flux<T, DIM>(X, g, c, s, J);
        ms_relax<T, DIM>(X, gs, J, c, s, tau, v, xinv);
        tau_out[s * S + i] = tau;
#pragma unroll
        for (int a = 0; a < DIM; ++a) u_out[(int64_t)(s * DIM + a) * S + i] = J[a] * xinv;
    }
}

// Equilibrium start (Eq. 29, f = w X) of cells [first, first + count): h = 0;
// the second X copy and the residual snapshot take X (already in x0).
template <class L, typename XS, typename P>
__global__ void init_kernel(P* __restrict__ h, const XS* __restrict__ x0, XS* __restrict__ x1,
                            double* __restrict__ snap, int64_t S, int first, int count) {
    using T = typename Xv<XS>::T;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= count) return;
    const int i = first + j;
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        const Xv<XS> v = Xv<XS>::own(x0, S, s, i);
        v.store(x1, S, s, i);
        snap[s * S + i] = v.to_double();
#pragma unroll
        for (int k = 0; k < L::Q; ++k) h[(int64_t)(s * L::Q + k) * S + i] = Pop<T, P>::quant(T(0));
    }
}

// -------------------------------------------------------------------------
// Deterministic FP64 block reduction: warp shuffles, one partial per block,
// and the last block to finish sums the partials in a fixed order.
template <int NV>
__device__ __forceinline__ void reduce_to_out(double (&acc)[NV], double* __restrict__ partials,
                                              unsigned int* __restrict__ counter, double* __restrict__ out) {
    __shared__ double sm[32][NV];
    __shared__ bool is_last;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        double a = acc[v];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if (lane == 0) sm[warp][v] = a;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            double a = lane < nwarps ? sm[lane][v] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
            if (lane == 0) partials[(int64_t)blockIdx.x * NV + v] = a;
        }
    }
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned int t = atomicAdd(counter, 1u);
        is_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();
    double b[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) b[v] = 0.0;
    for (int blk = threadIdx.x; blk < (int)gridDim.x; blk += blockDim.x) {
#pragma unroll
        for (int v = 0; v < NV; ++v) b[v] += __ldcg(partials + (int64_t)blk * NV + v);
    }
    __syncthreads();
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        double a = b[v];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if (lane == 0) sm[warp][v] = a;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            double a = lane < nwarps ? sm[lane][v] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
            if (lane == 0) out[v] = a;
        }
    }
    if (threadIdx.x == 0) *counter = 0u;
}

// -------------------------------------------------------------------------
// Per-case FP64 reductions of a batch, deterministic: a first kernel writes
// one partial per segment (a run of at most kSegCells cells of one case),
// a second sums each case's segments in order.
constexpr int kSegCells = 1024;
constexpr int kSegThreads = 256;

template <int NV>
__device__ __forceinline__ void block_sum(double (&acc)[NV], double* __restrict__ dst) {
    __shared__ double sm[kSegThreads / 32][NV];
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
        double a = acc[v];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
        if (lane == 0) sm[warp][v] = a;
    }
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            double a = lane < kSegThreads / 32 ? sm[lane][v] : 0.0;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) a += __shfl_down_sync(0xffffffffu, a, o);
            if (lane == 0) dst[v] = a;
        }
    }
}

// Residual partials of one segment (NV = 10: sum (X - snap)^2, sum X^2,
// sum X per species, count of non-finite X); the snapshot takes X when
// update != 0.
template <typename XS>
__global__ void __launch_bounds__(kSegThreads) seg_residual_kernel(const XS* __restrict__ X, double* __restrict__ snap,
                                                                   int64_t S, const int2* __restrict__ segs, int update,
                                                                   double* __restrict__ partials) {
    const int2 sg = segs[blockIdx.x];   // (first cell, cell count)
    double acc[10];
#pragma unroll
    for (int v = 0; v < 10; ++v) acc[v] = 0.0;
    for (int j = threadIdx.x; j < sg.y; j += kSegThreads) {
        const int i = sg.x + j;
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            const double x = Xv<XS>::own(X, S, s, i).to_double();
            const double d = x - snap[s * S + i];
            acc[s] += d * d;
            acc[3 + s] += x * x;
            acc[6 + s] += x;
            if (!isfinite(x)) acc[9] += 1.0;
            if (update) snap[s * S + i] = x;
        }
    }
    block_sum<10>(acc, partials + (int64_t)blockIdx.x * 10);
}

// Sums the partials of each case's segments [first, first + count) in order.
template <int NV>
__global__ void seg_finalize_kernel(const double* __restrict__ partials, const int2* __restrict__ case_segs,
                                    double* __restrict__ out) {
    const int2 r = case_segs[blockIdx.x];
    double acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = 0.0;
    for (int j = threadIdx.x; j < r.y; j += kSegThreads) {
#pragma unroll
        for (int v = 0; v < NV; ++v) acc[v] += partials[(int64_t)(r.x + j) * NV + v];
    }
    block_sum<NV>(acc, out + (int64_t)blockIdx.x * NV);
}

// Boundary sums of each case (one block per case, rows [first, first + count)
// of the concatenated row lists): out[0..2] = net flux toward +x through the
// plane between x = 0 and x = 1, carried by the post-collision populations
// w X + h of the last step; out[3..5] = sum of X over the outlet column.
template <class L, typename XS, typename P>
__global__ void __launch_bounds__(kSegThreads) case_boundary_kernel(
    const P* __restrict__ h, const XS* __restrict__ X, const int* __restrict__ nbr, int64_t S,
    const int* __restrict__ row_x0, const int* __restrict__ row_x1, const int* __restrict__ row_out,
    const int2* __restrict__ case_rows, double* __restrict__ out) {
    using T = typename Xv<XS>::T;
    constexpr int Q = L::Q;
    const int2 rr = case_rows[blockIdx.x];
    double acc[6];
#pragma unroll
    for (int v = 0; v < 6; ++v) acc[v] = 0.0;
    for (int j = threadIdx.x; j < rr.y; j += kSegThreads) {
        const int r = rr.x + j;
        const int i0 = row_x0[r];
        const int i1 = row_x1[r];
        const int io = row_out[r];
#pragma unroll
        for (int k = 1; k < Q; ++k) {
            const int ex = L::e(k, 0);
            const double w = weight<L>(k);
            if (ex == 1 && i0 >= 0) {
                // f*_k at x = 0 reaches x + e_k when that cell (the source of opp(k)) is fluid
                if (nbr[(int64_t)i0 * nb_width<L>() + opp<L>(k) - 1] >= 0) {
#pragma unroll
                    for (int s = 0; s < 3; ++s)
                        acc[s] += w * Xv<XS>::own(X, S, s, i0).to_double() +
                                  (double)Pop<T, P>::load(h + (int64_t)(s * Q + k) * S + i0);
                }
            } else if (ex == -1 && i1 >= 0) {
                if (nbr[(int64_t)i1 * nb_width<L>() + opp<L>(k) - 1] >= 0) {
#pragma unroll
                    for (int s = 0; s < 3; ++s)
                        acc[s] -= w * Xv<XS>::own(X, S, s, i1).to_double() +
                                  (double)Pop<T, P>::load(h + (int64_t)(s * Q + k) * S + i1);
                }
            }
        }
        if (io >= 0) {
#pragma unroll
            for (int s = 0; s < 3; ++s) acc[3 + s] += Xv<XS>::own(X, S, s, io).to_double();
        }
    }
    block_sum<6>(acc, out + (int64_t)blockIdx.x * 6);
}

// Extrapolation of the slowest decay mode for segment blockIdx.x of case
// seg_case[blockIdx.x]: with d = X - E (E = X of W steps ago) and
// c = coef[case], X += c d in both X copies (the step's and the lagged one);
// E takes the new X.  FP64 arithmetic, run once every W steps.
template <typename XS>
__global__ void __launch_bounds__(kSegThreads) seg_extrapolate_kernel(XS* __restrict__ X, XS* __restrict__ Xprev,
                                                                      double* __restrict__ E, int64_t S,
                                                                      const int2* __restrict__ segs,
                                                                      const int* __restrict__ seg_case,
                                                                      const double* __restrict__ coef) {
    const int2 sg = segs[blockIdx.x];
    const double c = coef[seg_case[blockIdx.x]];
    for (int j = threadIdx.x; j < sg.y; j += kSegThreads) {
        const int i = sg.x + j;
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            const double x = Xv<XS>::own(X, S, s, i).to_double();
            const double xp = Xv<XS>::own(Xprev, S, s, i).to_double();
            const double d = c * (x - E[s * S + i]);
            const double xn = x + d;
            store_x<XS>(X, S, s, i, xn);
            store_x<XS>(Xprev, S, s, i, xp + d);
            E[s * S + i] = xn;
        }
    }
}

// -------------------------------------------------------------------------
// Reduced-rank extrapolation (RRE; Mesina 1977, Eddy 1979, in the form of
// Sidi's vector extrapolation methods) over M + 1 snapshots x_0 .. x_M of X
// taken W steps apart, in FP64: with u_a = x_{a+1} - x_a, the limit is
// estimated as sum_j gamma_j x_j, where gamma minimises || sum_j gamma_j u_j ||
// subject to sum_j gamma_j = 1 (solved on the host from the Gram matrix of
// the u_a).  For an iteration whose error is a sum of at most M decaying
// modes the estimate is the fixed point.  Snapshot j of a cycle sits in slot j
// of `ring` ([slot][3][S] doubles).

// Snapshot of X into ring slot `slot`, per segment.
template <typename XS>
__global__ void __launch_bounds__(kSegThreads) seg_snapshot_kernel(const XS* __restrict__ X, double* __restrict__ ring,
                                                                   int64_t S, const int2* __restrict__ segs, int slot) {
    const int2 sg = segs[blockIdx.x];
    double* dst = ring + (int64_t)slot * 3 * S;
    for (int j = threadIdx.x; j < sg.y; j += kSegThreads) {
        const int i = sg.x + j;
#pragma unroll
        for (int s = 0; s < 3; ++s) dst[s * S + i] = Xv<XS>::own(X, S, s, i).to_double();
    }
}

// Partial Gram matrix of the differences u_a = x_{a+1} - x_a (a < M) over one
// segment: entries (a, b), a <= b, packed row by row (M (M + 1) / 2 values).
template <int M>
__global__ void __launch_bounds__(kSegThreads) seg_gram_kernel(const double* __restrict__ ring, int64_t S,
                                                               const int2* __restrict__ segs,
                                                               double* __restrict__ partials) {
    constexpr int NV = M * (M + 1) / 2;
    const int2 sg = segs[blockIdx.x];
    double acc[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) acc[v] = 0.0;
    for (int j = threadIdx.x; j < sg.y; j += kSegThreads) {
        const int i = sg.x + j;
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            double x[M + 1], u[M];
#pragma unroll
            for (int a = 0; a <= M; ++a) x[a] = ring[((int64_t)a * 3 + s) * S + i];
#pragma unroll
            for (int a = 0; a < M; ++a) u[a] = x[a + 1] - x[a];
            int v = 0;
#pragma unroll
            for (int a = 0; a < M; ++a)
#pragma unroll
                for (int b = a; b < M; ++b) acc[v++] += u[a] * u[b];
        }
    }
    block_sum<NV>(acc, partials + (int64_t)blockIdx.x * NV);
}

// X += sum_a c_a u_a with the case's coefficients coef[case * M + a], in both
// X copies (the step's and the lagged one); slot 0 also takes the new X.
template <typename XS, int M>
__global__ void __launch_bounds__(kSegThreads) seg_rre_apply_kernel(XS* __restrict__ X, XS* __restrict__ Xprev,
                                                                    double* __restrict__ ring, int64_t S,
                                                                    const int2* __restrict__ segs,
                                                                    const int* __restrict__ seg_case,
                                                                    const double* __restrict__ coef) {
    const int2 sg = segs[blockIdx.x];
    const double* c = coef + (int64_t)seg_case[blockIdx.x] * M;
    for (int j = threadIdx.x; j < sg.y; j += kSegThreads) {
        const int i = sg.x + j;
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            double d = 0.0;
#pragma unroll
            for (int a = 0; a < M; ++a)
                d += c[a] * (ring[((int64_t)(a + 1) * 3 + s) * S + i] - ring[((int64_t)a * 3 + s) * S + i]);
            const double x = Xv<XS>::own(X, S, s, i).to_double();
            const double xp = Xv<XS>::own(Xprev, S, s, i).to_double();
            const double xn = x + d;
            store_x<XS>(X, S, s, i, xn);
            store_x<XS>(Xprev, S, s, i, xp + d);
            ring[s * S + i] = xn;
        }
    }
}

}  // namespace lbms
