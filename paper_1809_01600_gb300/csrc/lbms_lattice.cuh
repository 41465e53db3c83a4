// Velocity sets of the solver, shared by host set-up and device kernels.
//
// D2Q9 is the set of Eq. 2 with the weights of Eq. 9; D3Q19 is the textbook
// 3-D set (rest 1/3, axis links 1/18, edge diagonals 1/36).  Both are stored
// in pairs: k and its opposite sit side by side (odd k, k + 1), and the axis
// links come first: k = 1 + 2d is +e_d, k = 2 + 2d is -e_d.
#pragma once

#include <cstdint>

#ifndef __CUDACC__
#define __host__
#define __device__
#endif

namespace lbms {

struct D2Q9 {
    static constexpr int Q = 9;
    static constexpr int DIM = 2;
    __host__ __device__ static constexpr int e(int k, int d) {
        constexpr int t[9][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0}, {0, -1, 0},
                                 {1, 1, 0},  {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}};
        return t[k][d];
    }
};

struct D3Q19 {
    static constexpr int Q = 19;
    static constexpr int DIM = 3;
    __host__ __device__ static constexpr int e(int k, int d) {
        constexpr int t[19][3] = {{0, 0, 0},   {1, 0, 0},   {-1, 0, 0},  {0, 1, 0},  {0, -1, 0},
                                  {0, 0, 1},   {0, 0, -1},  {1, 1, 0},   {-1, -1, 0}, {1, -1, 0},
                                  {-1, 1, 0},  {1, 0, 1},   {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                                  {0, 1, 1},   {0, -1, -1}, {0, 1, -1},  {0, -1, 1}};
        return t[k][d];
    }
};

template <class L>
__host__ __device__ constexpr int opp(int k) {
    return k == 0 ? 0 : ((k & 1) ? k + 1 : k - 1);
}

template <class L>
__host__ __device__ constexpr int norm2(int k) {
    return L::e(k, 0) * L::e(k, 0) + L::e(k, 1) * L::e(k, 1) + L::e(k, 2) * L::e(k, 2);
}

// Lattice weights: Eq. 9 for D2Q9, the standard D3Q19 weights.
template <class L>
__host__ __device__ constexpr double weight(int k) {
    return L::Q == 9 ? (norm2<L>(k) == 0 ? 4.0 / 9.0 : (norm2<L>(k) == 1 ? 1.0 / 9.0 : 1.0 / 36.0))
                     : (norm2<L>(k) == 0 ? 1.0 / 3.0 : (norm2<L>(k) == 1 ? 1.0 / 18.0 : 1.0 / 36.0));
}

// Sum of the weights of the links with e_x = +1 (1/6 for both sets).
template <class L>
__host__ __device__ constexpr double weight_xplus() {
    double s = 0.0;
    for (int k = 0; k < L::Q; ++k)
        if (L::e(k, 0) == 1) s += weight<L>(k);
    return s;
}

// Width (ints) of one cell's row of the neighbour table: the Q-1 links,
// padded to a multiple of 4 so that a row is read with 16-byte loads.
template <class L>
__host__ __device__ constexpr int nb_width() {
    return ((L::Q - 1) + 3) / 4 * 4;
}

// The compact table: 16-bit offsets src - i, rows padded to a multiple of 8
// entries (16-byte loads); the three lowest values stand for the NB_* codes
// and the fourth (NB16_FAR) sends the link to the 32-bit table (periodic
// wraps, whose offsets do not fit).
template <class L>
__host__ __device__ constexpr int nb16_width() {
    return ((L::Q - 1) + 7) / 8 * 8;
}
enum : int {
    NB16_SOLID = -32768,
    NB16_INLET = -32767,
    NB16_OUTLET = -32766,
    NB16_FAR = -32765,
    NB16_MIN_OFFSET = -32764,   // smallest offset a fluid source may have
    NB16_MAX_OFFSET = 32767
};

// Tag of the neighbour decode from per-row fluid bitmasks (no per-link table).
struct RowMaskNb {};

// Neighbour-table codes for a link whose source x - e_k is not a fluid cell.
enum : int {
    NB_SOLID = -1,   // half-way bounce-back
    NB_INLET = -2,   // beyond x = 0: Dirichlet inlet (Eq. 36)
    NB_OUTLET = -3   // beyond x = nx-1: reacting outlet flux (Eq. 39)
};

}  // namespace lbms
