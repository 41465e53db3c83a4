// Device side of the solver: the fused collide + stream + Maxwell-Stefan
// step, the field recomputation, initialisation and the FP64 reductions.
//
// Storage (all compact over the fluid cells, x-fastest order, padded row
// stride S, a multiple of 32 elements):
//   f[s][k][i]   post-collision populations, two lattices (pull streaming),
//                stored shifted: f - w_k Xref_s (Xref = a fixed reference
//                composition), in FP64, FP32 or FP16 (FP16 scaled by 2^10)
//   X[s][i]      mole fractions of a step minus Xref, two buffers (this step /
//                previous), FP64 or FP32
//   nbr[k-1][i]  fluid index of the source cell x - e_k, or an NB_* code
// The shift is exact algebra (sum_k w_k = 1, w_k = w_opp(k)); it keeps the
// stored numbers near zero so that their rounding error scales with the
// departure from Xref rather than with X itself.
#pragma once

#include <cstdint>
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
};

// Population storage: P = T, or __half holding (f - w Xref) * 2^10.
constexpr float kHalfScale = 1024.0f;
constexpr float kHalfInvScale = 1.0f / 1024.0f;

template <typename T, typename P>
struct Pop {
    __device__ __forceinline__ static T load(const P* p) { return T(*p); }
    __device__ __forceinline__ static void store(P* p, T v) { *p = P(v); }
};
template <>
struct Pop<float, __half> {
    __device__ __forceinline__ static float load(const __half* p) { return __half2float(*p) * kHalfInvScale; }
    __device__ __forceinline__ static void store(__half* p, float v) { *p = __float2half_rn(v * kHalfScale); }
};

template <typename T, typename P>
struct StepParams {
    const P* __restrict__ fin;
    P* __restrict__ fout;
    const T* __restrict__ xprev;
    T* __restrict__ xnext;
    const int* __restrict__ nbr;
    int64_t S;
    int nf;
    T xref[3];      // shift of the stored populations and mole fractions
    T dxin[3];      // inlet mole fractions minus xref (Eq. 36)
    T qout[3];      // outlet flux per node per step (Eq. 39)
    MsConst<T> c;
};

// -------------------------------------------------------------------------
// Lagged gradient (Eq. 35 read as a central difference on every axis): the
// stored field of the previous step, a solid neighbour mirrored to the centre
// value, one-sided at the inlet/outlet nodes.
template <class L, typename T>
__device__ __forceinline__ void lagged_gradient(const T* __restrict__ xprev, int64_t S, int i,
                                                const int (&nb)[L::Q], T (&g)[3][L::DIM]) {
    T xc[3];
#pragma unroll
    for (int s = 0; s < 3; ++s) xc[s] = xprev[s * S + i];
#pragma unroll
    for (int d = 0; d < L::DIM; ++d) {
        const int cp = nb[2 + 2 * d];  // source of -e_d is the cell at x + e_d
        const int cm = nb[1 + 2 * d];  // source of +e_d is the cell at x - e_d
        const bool hp = cp >= NB_SOLID;
        const bool hm = cm >= NB_SOLID;
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            const T pv = cp >= 0 ? xprev[s * S + cp] : xc[s];
            const T mv = cm >= 0 ? xprev[s * S + cm] : xc[s];
            g[s][d] = (hp && hm) ? T(0.5) * (pv - mv) : (hp ? pv - xc[s] : (hm ? xc[s] - mv : T(0)));
        }
    }
}

// -------------------------------------------------------------------------
// Maxwell-Stefan coupling of one cell (lattice units, c_s^2 = 1/3):
//  B (Eq. 32, species 3 = reference n), J_1,2 = -B^-1 g (Eqs. 31, 33, 34,
//  Gamma = I), J_3 from the n-th row of Eq. 19; D_i from Eq. 24 with the
//  flux ratios of the electrode reaction (nu_j / nu_i), the mixture value
//  for the inert species; tau_i from Eq. 25 clamped; and the drift velocity
//  (velocity slot of Eq. 26) that makes the carried flux the Maxwell-Stefan
//  flux J_i.
template <typename T, int DIM>
__device__ __forceinline__ void ms_coupling(const T (&X)[3], const T (&g)[3][DIM], const MsConst<T>& c,
                                            T (&tau)[3], T (&v)[3][DIM], T (*u)[DIM]) {
    const T B11 = X[0] * c.i13 + X[1] * c.i12 + X[2] * c.i13;
    const T B12 = -X[0] * (c.i12 - c.i13);
    const T B21 = -X[1] * (c.i12 - c.i23);
    const T B22 = X[1] * c.i23 + X[0] * c.i12 + X[2] * c.i23;
    const T det = B11 * B22 - B12 * B21;
    const T idet = det > T(0) ? T(1) / det : T(0);
    const T d3 = X[0] * c.i13 + X[1] * c.i23;
    const T id3 = d3 > T(0) ? T(1) / d3 : T(0);

    T J[3][DIM];
#pragma unroll
    for (int d = 0; d < DIM; ++d) {
        J[0][d] = -(B22 * g[0][d] - B12 * g[1][d]) * idet;
        J[1][d] = -(B11 * g[1][d] - B21 * g[0][d]) * idet;
        J[2][d] = (-g[2][d] + X[2] * (J[0][d] * c.i13 + J[1][d] * c.i23)) * id3;
    }

    const T md = T(kMixDelta);
    const T ex2 = T(kEpsX * kEpsX);
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        T D;
        if (c.reacting[s]) {
            const T inv = c.a[s][0] * X[0] + c.a[s][1] * X[1] + c.a[s][2] * X[2];
            D = inv > T(0) ? T(1) / inv : T(kDBig);
        } else {
            // mixture value sum_{j!=s} X_j / sum_{j!=s} X_j / D_sj
            const T num = (X[0] + X[1] + X[2] - X[s]) + md;
            const T den = (s == 0 ? X[1] * c.i12 + X[2] * c.i13
                                  : (s == 1 ? X[0] * c.i12 + X[2] * c.i23 : X[0] * c.i13 + X[1] * c.i23)) +
                          md * c.h[s];
            D = num / den;
        }
        T t = D * T(3) + T(0.5);
        t = t < c.tau_min ? c.tau_min : (t > c.tau_max ? c.tau_max : t);
        tau[s] = t;
        const T Dt = (t - T(0.5)) * T(1.0 / 3.0);
        const T xinv = X[s] / (X[s] * X[s] + ex2);
        if (c.drift) {
            T vn2 = T(0);
#pragma unroll
            for (int d = 0; d < DIM; ++d) {
                v[s][d] = (J[s][d] + Dt * g[s][d]) * xinv;
                vn2 += v[s][d] * v[s][d];
            }
            if (vn2 > T(kVMax * kVMax)) {
                const T sc = T(kVMax) / sqrt(vn2);
#pragma unroll
                for (int d = 0; d < DIM; ++d) v[s][d] *= sc;
            }
        } else {
#pragma unroll
            for (int d = 0; d < DIM; ++d) v[s][d] = T(0);
        }
        if (u) {
#pragma unroll
            for (int d = 0; d < DIM; ++d) u[s][d] = J[s][d] * xinv;
        }
    }
}

// -------------------------------------------------------------------------
// One time step for every fluid cell (one thread per cell):
// pull-stream with bounce-back / inlet / outlet, moments, lagged gradient,
// coupling, BGK collision, store post-collision populations and X.
// All population arithmetic is on shifted values g_k = f_k - w_k Xref.
template <class L, typename T, typename P>
__global__ void __launch_bounds__(256) step_kernel(const StepParams<T, P> p) {
    constexpr int Q = L::Q;
    constexpr int DIM = L::DIM;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.nf) return;
    const int64_t S = p.S;

    int nb[Q];
    nb[0] = i;
#pragma unroll
    for (int k = 1; k < Q; ++k) nb[k] = __ldg(p.nbr + (int64_t)(k - 1) * S + i);

    // 1. stream (pull) with the boundary rules
    T f[3][Q];
    constexpr T wx = T(weight_xplus<L>());
#pragma unroll
    for (int s = 0; s < 3; ++s) {
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            const int src = nb[k];
            const P* row = p.fin + (int64_t)(s * Q + k) * S;
            const P* orow = p.fin + (int64_t)(s * Q + opp<L>(k)) * S;
            T val;
            if (src >= 0)
                val = Pop<T, P>::load(row + src);
            else if (src == NB_SOLID)
                val = Pop<T, P>::load(orow + i);
            else if (src == NB_OUTLET)
                val = Pop<T, P>::load(orow + i) - (T(weight<L>(opp<L>(k))) / wx) * p.qout[s];
            else
                val = T(0);
            f[s][k] = val;
        }
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            if (L::e(k, 0) == 1 && nb[k] == NB_INLET)
                f[s][k] = T(weight<L>(k) + weight<L>(opp<L>(k))) * p.dxin[s] - f[s][opp<L>(k)];
        }
    }

    // 2. moments (shifted: Xs = X - Xref)
    T Xs[3], X[3];
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        T acc = T(0);
#pragma unroll
        for (int k = 0; k < Q; ++k) acc += f[s][k];
        Xs[s] = acc;
        X[s] = p.xref[s] + acc;
    }

    // 3-6. lagged gradient and Maxwell-Stefan coupling
    T g[3][DIM];
    lagged_gradient<L, T>(p.xprev, S, i, nb, g);
    T tau[3], v[3][DIM];
    ms_coupling<T, DIM>(X, g, p.c, tau, v, nullptr);

    // 7. BGK collision towards w X (1 + e.v / c_s^2), shifted by w Xref, store
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        const T it = T(1) / tau[s];
#pragma unroll
        for (int k = 0; k < Q; ++k) {
            T ev = T(0);
#pragma unroll
            for (int d = 0; d < DIM; ++d) ev += T(L::e(k, d)) * v[s][d];
            const T w = T(weight<L>(k));
            const T geq = w * Xs[s] + T(3) * w * X[s] * ev;
            Pop<T, P>::store(p.fout + (int64_t)(s * Q + k) * S + i, f[s][k] - (f[s][k] - geq) * it);
        }
        p.xnext[s * S + i] = Xs[s];
    }
}

// -------------------------------------------------------------------------
// tau and the component velocity of the last step, recomputed from the
// stored fields (X of the step and of the step before).
template <class L, typename T>
__global__ void fields_kernel(const T* __restrict__ xcur, const T* __restrict__ xprev,
                              const int* __restrict__ nbr, int64_t S, int nf, MsConst<T> c, T xr0, T xr1, T xr2,
                              T* __restrict__ tau_out, T* __restrict__ u_out) {
    constexpr int Q = L::Q;
    constexpr int DIM = L::DIM;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    int nb[Q];
    nb[0] = i;
#pragma unroll
    for (int k = 1; k < Q; ++k) nb[k] = nbr[(int64_t)(k - 1) * S + i];
    const T xr[3] = {xr0, xr1, xr2};
    T X[3];
#pragma unroll
    for (int s = 0; s < 3; ++s) X[s] = xr[s] + xcur[s * S + i];
    T g[3][DIM];
    lagged_gradient<L, T>(xprev, S, i, nb, g);
    T tau[3], v[3][DIM], u[3][DIM];
    ms_coupling<T, DIM>(X, g, c, tau, v, u);
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        tau_out[s * S + i] = tau[s];
#pragma unroll
        for (int d = 0; d < DIM; ++d) u_out[(int64_t)(s * DIM + d) * S + i] = u[s][d];
    }
}

// f = w X (Eq. 29 equilibrium) in the current lattice, i.e. stored w (X - Xref);
// both X buffers and the residual snapshot take X - Xref (already in x0).
template <class L, typename T, typename P>
__global__ void init_kernel(P* __restrict__ f, const T* __restrict__ x0, T* __restrict__ x1, T* __restrict__ snap,
                            int64_t S, int nf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
#pragma unroll
    for (int s = 0; s < 3; ++s) {
        const T Xs = x0[s * S + i];
        x1[s * S + i] = Xs;
        snap[s * S + i] = Xs;
#pragma unroll
        for (int k = 0; k < L::Q; ++k) Pop<T, P>::store(f + (int64_t)(s * L::Q + k) * S + i, T(weight<L>(k)) * Xs);
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

// Residual sums over fluid cells in FP64 (X = Xref + stored value):
// out[0..2] = sum (X - snap)^2, out[3..5] = sum X^2, out[6..8] = sum X,
// out[9] = count of non-finite X.  When update != 0 the snapshot takes X.
// Grid-stride over a persistent grid.
template <typename T>
__global__ void __launch_bounds__(256) residual_kernel(const T* __restrict__ X, T* __restrict__ snap,
                                                       int64_t S, int nf, int update, double xr0, double xr1,
                                                       double xr2, double* __restrict__ partials,
                                                       unsigned int* __restrict__ counter, double* __restrict__ out) {
    const double xr[3] = {xr0, xr1, xr2};
    double acc[10];
#pragma unroll
    for (int v = 0; v < 10; ++v) acc[v] = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nf; i += gridDim.x * blockDim.x) {
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            const double xs = (double)X[s * S + i];
            const double d = xs - (double)snap[s * S + i];
            const double x = xr[s] + xs;
            acc[s] += d * d;
            acc[3 + s] += x * x;
            acc[6 + s] += x;
            if (!isfinite(x)) acc[9] += 1.0;
            if (update) snap[s * S + i] = X[s * S + i];
        }
    }
    reduce_to_out<10>(acc, partials, counter, out);
}

// Boundary sums in FP64 over the ny*nz rows: out[0..2] = net flux toward +x
// through the plane between x = 0 and x = 1 (post-collision populations of
// the last step), out[3..5] = sum of X over the outlet column.
template <class L, typename T, typename P>
__global__ void __launch_bounds__(256) boundary_kernel(const P* __restrict__ f, const T* __restrict__ X,
                                                       const int* __restrict__ nbr, int64_t S,
                                                       const int* __restrict__ row_x0, const int* __restrict__ row_x1,
                                                       const int* __restrict__ row_out, int nrows, double xr0,
                                                       double xr1, double xr2, double* __restrict__ partials,
                                                       unsigned int* __restrict__ counter, double* __restrict__ out) {
    constexpr int Q = L::Q;
    const double xr[3] = {xr0, xr1, xr2};
    double acc[6];
#pragma unroll
    for (int v = 0; v < 6; ++v) acc[v] = 0.0;
    for (int r = blockIdx.x * blockDim.x + threadIdx.x; r < nrows; r += gridDim.x * blockDim.x) {
        const int i0 = row_x0[r];
        const int i1 = row_x1[r];
        const int io = row_out[r];
#pragma unroll
        for (int k = 1; k < Q; ++k) {
            const int ex = L::e(k, 0);
            const double w = weight<L>(k);
            if (ex == 1 && i0 >= 0) {
                // f*_k at x = 0 reaches x + e_k when that cell (the source of opp(k)) is fluid
                if (nbr[(int64_t)(opp<L>(k) - 1) * S + i0] >= 0) {
#pragma unroll
                    for (int s = 0; s < 3; ++s)
                        acc[s] += (double)Pop<T, P>::load(f + (int64_t)(s * Q + k) * S + i0) + w * xr[s];
                }
            } else if (ex == -1 && i1 >= 0) {
                if (nbr[(int64_t)(opp<L>(k) - 1) * S + i1] >= 0) {
#pragma unroll
                    for (int s = 0; s < 3; ++s)
                        acc[s] -= (double)Pop<T, P>::load(f + (int64_t)(s * Q + k) * S + i1) + w * xr[s];
                }
            }
        }
        if (io >= 0) {
#pragma unroll
            for (int s = 0; s < 3; ++s) acc[3 + s] += xr[s] + (double)X[s * S + io];
        }
    }
    reduce_to_out<6>(acc, partials, counter, out);
}

}  // namespace lbms
