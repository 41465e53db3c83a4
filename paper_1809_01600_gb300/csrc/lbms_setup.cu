// Set-up kernels: the neighbour tables of the step kernels, built on the
// device from each case's dense fluid-index map (the host only numbers the
// fluid cells).
#include <algorithm>

#include "lbms_internal.h"
#include "lbms_lattice.cuh"

namespace lbms {

namespace {

static_assert(NB_SOLID == -1, "the 32-bit table is cleared to NB_SOLID with a 0xFF byte fill");

// Row of fluid cell li of a case: the source x - e_k of every link k, as a
// fluid index of the batch's index space (base + index in the case) or an
// NB_* code (solid: bounce-back; beyond x = 0 / x = nx-1: inlet / outlet;
// y and z periodic, x too for a box periodic in x).  The 16-bit table gets
// src - i, or an NB16_* code, NB16_FAR where the offset does not fit.
// counts[0] += fluid links, counts[1] += links marked NB16_FAR.
template <class Lat>
__global__ void build_nbr_kernel(const int64_t* __restrict__ fluid_cell, const int* __restrict__ index_of, int nf,
                                 int base, int nx, int ny, int nz, int periodic_x, int* __restrict__ nbr,
                                 int16_t* __restrict__ nbr16, unsigned long long* __restrict__ counts) {
    constexpr int NW = nb_width<Lat>();
    constexpr int NW16 = nb16_width<Lat>();
    __shared__ unsigned long long s_links, s_far;
    if (threadIdx.x == 0) {
        s_links = 0;
        s_far = 0;
    }
    __syncthreads();
    const int li = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long links = 0, far = 0;
    if (li < nf) {
        const int64_t cell = fluid_cell[li];
        const int x = (int)(cell % nx);
        const int y = (int)((cell / nx) % ny);
        const int z = (int)(cell / ((int64_t)nx * ny));
        const int64_t i = (int64_t)base + li;
        for (int k = 1; k < Lat::Q; ++k) {
            int sx = x - Lat::e(k, 0);
            const int sy = ((y - Lat::e(k, 1)) % ny + ny) % ny;
            const int sz = ((z - Lat::e(k, 2)) % nz + nz) % nz;
            int code;
            if (!periodic_x && sx < 0) {
                code = NB_INLET;
            } else if (!periodic_x && sx >= nx) {
                code = NB_OUTLET;
            } else {
                sx = (sx % nx + nx) % nx;
                const int j = index_of[((int64_t)sz * ny + sy) * nx + sx];
                code = j >= 0 ? base + j : NB_SOLID;
            }
            nbr[i * NW + (k - 1)] = code;
            int c16;
            if (code >= 0) {
                ++links;
                const int64_t d = (int64_t)code - i;
                const bool fits = d >= NB16_MIN_OFFSET && d <= NB16_MAX_OFFSET;
                far += fits ? 0 : 1;
                c16 = fits ? (int)d : NB16_FAR;
            } else {
                c16 = code == NB_SOLID ? NB16_SOLID : (code == NB_INLET ? NB16_INLET : NB16_OUTLET);
            }
            if (nbr16) nbr16[i * NW16 + (k - 1)] = (int16_t)c16;
        }
    }
    if (links) atomicAdd(&s_links, links);
    if (far) atomicAdd(&s_far, far);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_links) atomicAdd(&counts[0], s_links);
        if (s_far) atomicAdd(&counts[1], s_far);
    }
}

__global__ void fill16_kernel(int16_t* __restrict__ p, int64_t n, int16_t v) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        p[e] = v;
}

}  // namespace

cudaError_t launch_build_neighbours(int dim, const int64_t* fluid_cell, const int* index_of, int nf, int base, int nx,
                                    int ny, int nz, int periodic_x, int* nbr, int16_t* nbr16,
                                    unsigned long long* counts, cudaStream_t st) {
    const int grid = (nf + 255) / 256;
    if (dim == 2)
        build_nbr_kernel<D2Q9><<<grid, 256, 0, st>>>(fluid_cell, index_of, nf, base, nx, ny, nz, periodic_x, nbr,
                                                     nbr16, counts);
    else
        build_nbr_kernel<D3Q19><<<grid, 256, 0, st>>>(fluid_cell, index_of, nf, base, nx, ny, nz, periodic_x, nbr,
                                                      nbr16, counts);
    return cudaGetLastError();
}

cudaError_t launch_fill16(int16_t* p, int64_t n, int16_t v, cudaStream_t st) {
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 152 * 16);
    fill16_kernel<<<(int)std::max<int64_t>(blocks, 1), 256, 0, st>>>(p, n, v);
    return cudaGetLastError();
}

}  // namespace lbms
