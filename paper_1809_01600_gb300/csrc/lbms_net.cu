// Learned warm start (declared in include/lbms_net.h): feature rows of an
// anode's fluid cells, a pointwise MLP with BF16 tensor-core matrix products
// (mma.sync m16n8k16, FP32 accumulation), its backward pass and Adam.
//
// Matrix products are all of one form, P = A . B^T with A [M][K] and B [N][K]
// both K-contiguous BF16 ("TN"), M and N multiples of 64, K a multiple of 32
// per split; the forward pass, the input gradients and the weight gradients
// get that form by keeping transposed copies of the weights and of the
// activations.  Every size is padded at allocation so that no tile crosses a
// buffer's end: the kernels need no bounds checks, and the host checks the
// divisibility before every launch.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/lbms.h"
#include "../../include/lbms_net.h"
#include "lbms_internal.h"

namespace {

using bf16 = __nv_bfloat16;

constexpr int kF = LBMS_NET_FEATURES;   // feature row width
constexpr int kFUsed = 16;              // features actually set
constexpr int kOutPad = 64;             // output layer rows (3 used)
constexpr int kOut = 3;
constexpr float kTargetScale = 100.0f;  // network output = 100 (X - X_profile)
constexpr int kMaxRows = 32768;         // rows per forward / training batch
constexpr int kTM = 64, kTN = 64, kTK = 32;

// ---------------------------------------------------------------- generator
// SplitMix64 (Steele, Lea, Flood 2014): a counter-based generator, one
// 64-bit output per key.
__host__ __device__ inline uint64_t splitmix64(uint64_t x) {
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}
inline double unit_double(uint64_t x) { return (double)(splitmix64(x) >> 11) * (1.0 / 9007199254740992.0); }

// ------------------------------------------------------------------- GEMM
__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
// Four 8x8 BF16 matrices from shared memory; lane l supplies the address of
// row (l % 8) of matrix l / 8.
__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void* smem) {
    const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(sa));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

// P[z][M][N] = sum over k in [z kchunk, (z+1) kchunk) of A[m][k] B[n][k].
// Block: 64 x 64 output tile, 4 warps of 32 x 32; K in steps of 32 staged in
// shared memory by cp.async, two stages (the next step loads while this one
// is multiplied); rows padded to 40 elements for conflict-free fragment
// reads.
__global__ void __launch_bounds__(128) gemm_tn_kernel(const bf16* __restrict__ A, int lda, const bf16* __restrict__ B,
                                                      int ldb, float* __restrict__ P, int M, int N, int kchunk) {
    __shared__ __align__(16) bf16 sA[2][kTM][kTK + 8];
    __shared__ __align__(16) bf16 sB[2][kTN][kTK + 8];
    const int m0 = blockIdx.y * kTM, n0 = blockIdx.x * kTN;
    const int k0 = blockIdx.z * kchunk;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int g = lane >> 2, t = lane & 3;
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.0f;

    // 64 rows x 32 elements = 256 chunks of 16 bytes per operand and stage
    auto stage = [&](int buf, int kk) {
        for (int c = threadIdx.x; c < kTM * kTK / 8; c += 128) {
            const int r = c >> 2, q = (c & 3) * 8;
            cp_async16(&sA[buf][r][q], A + (int64_t)(m0 + r) * lda + kk + q);
            cp_async16(&sB[buf][r][q], B + (int64_t)(n0 + r) * ldb + kk + q);
        }
        cp_async_commit();
    };
    const int nk = kchunk / kTK;
    stage(0, k0);
    for (int it = 0; it < nk; ++it) {
        const int buf = it & 1;
        if (it + 1 < nk) {
            stage(buf ^ 1, k0 + (it + 1) * kTK);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
#pragma unroll
        for (int ks = 0; ks < kTK; ks += 16) {
            // A fragments (16 x 16, rows m): matrices (rows 0-7 | 8-15) x (k 0-7 | 8-15);
            // B fragments of two n-blocks of 8: matrices (n 0-7, k 0-7), (n 0-7, k 8-15),
            // (n 8-15, k 0-7), (n 8-15, k 8-15), i.e. b[j][0], b[j][1], b[j+1][0], b[j+1][1]
            uint32_t a[2][4], b[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) ldsm_x4(a[i], &sA[buf][wm + i * 16 + (lane & 15)][ks + (lane >> 4) * 8]);
#pragma unroll
            for (int jj = 0; jj < 2; ++jj) {
                uint32_t r[4];
                ldsm_x4(r, &sB[buf][wn + jj * 16 + (lane & 7) + ((lane >> 4) << 3)][ks + ((lane >> 3) & 1) * 8]);
                b[2 * jj][0] = r[0];
                b[2 * jj][1] = r[1];
                b[2 * jj + 1][0] = r[2];
                b[2 * jj + 1][1] = r[3];
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], a[i], b[j]);
        }
        __syncthreads();   // the stage just read is refilled two steps later
    }
    float* Pz = P + (int64_t)blockIdx.z * M * N;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int r = m0 + wm + i * 16 + g;
            const int c = n0 + wn + j * 8 + 2 * t;
            *reinterpret_cast<float2*>(Pz + (int64_t)r * N + c) = make_float2(acc[i][j][0], acc[i][j][1]);
            *reinterpret_cast<float2*>(Pz + (int64_t)(r + 8) * N + c) = make_float2(acc[i][j][2], acc[i][j][3]);
        }
}

// ---------------------------------------------------------- elementwise
// Z = P + b (one row per thread block row); hidden layers store relu(Z) as
// BF16 [R][C], the output layer stores Z as FP32.
__global__ void bias_act_kernel(const float* __restrict__ P, const float* __restrict__ b, int R, int C, int relu,
                                bf16* __restrict__ act, float* __restrict__ Y) {
    const int64_t n = (int64_t)R * C;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const float z = P[e] + b[e % C];
        if (relu)
            act[e] = __float2bfloat16_rn(z > 0.0f ? z : 0.0f);
        else
            Y[e] = z;
    }
}

// out[c][r] = in[r][c]; R and C multiples of 32.
__global__ void transpose_kernel(const bf16* __restrict__ in, bf16* __restrict__ out, int R, int C) {
    __shared__ bf16 tile[32][33];
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    for (int y = threadIdx.y; y < 32; y += 8) tile[y][threadIdx.x] = in[(int64_t)(r0 + y) * C + c0 + threadIdx.x];
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += 8) out[(int64_t)(c0 + y) * R + r0 + threadIdx.x] = tile[threadIdx.x][y];
}

// Mean-square error over the 3 used outputs and its gradient dY (BF16,
// zero in the padded columns); bias gradient of the output layer and the
// loss summed with atomics.  One block of 256 threads per 64 rows.
__global__ void loss_grad_kernel(const float* __restrict__ Y, const float* __restrict__ T, int R,
                                 bf16* __restrict__ dY, float* __restrict__ gb, double* __restrict__ loss) {
    __shared__ float colsum[kOutPad];
    __shared__ double lsum[256];
    if (threadIdx.x < kOutPad) colsum[threadIdx.x] = 0.0f;
    __syncthreads();
    const float scale = 2.0f / (float)(R * kOut);
    double l = 0.0;
    const int r0 = blockIdx.x * 64;
    for (int e = threadIdx.x; e < 64 * kOutPad; e += 256) {
        const int r = r0 + e / kOutPad, c = e % kOutPad;
        float gval = 0.0f;
        if (c < kOut) {
            const float d = Y[(int64_t)r * kOutPad + c] - T[(int64_t)r * 4 + c];
            l += (double)d * d;
            gval = scale * d;
            atomicAdd(&colsum[c], gval);
        }
        dY[(int64_t)r * kOutPad + c] = __float2bfloat16_rn(gval);
    }
    lsum[threadIdx.x] = l;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) lsum[threadIdx.x] += lsum[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicAdd(loss, lsum[0] / (double)(R * kOut));
    if (threadIdx.x < kOut) atomicAdd(&gb[threadIdx.x], colsum[threadIdx.x]);
}

// dZ = dA * (layer input > 0) as BF16 [R][C]; bias gradient column sums.
// One block of 256 threads per 32 rows x C columns (C a multiple of 64).
__global__ void relu_back_kernel(const float* __restrict__ dA, const bf16* __restrict__ act, int R, int C,
                                 bf16* __restrict__ dZ, float* __restrict__ gb) {
    const int r0 = blockIdx.x * 32;
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        float s = 0.0f;
        for (int r = r0; r < r0 + 32; ++r) {
            const int64_t e = (int64_t)r * C + c;
            const float v = __bfloat162float(act[e]) > 0.0f ? dA[e] : 0.0f;
            dZ[e] = __float2bfloat16_rn(v);
            s += v;
        }
        atomicAdd(&gb[c], s);
    }
}

// G[e] = sum_z P[z][e]
__global__ void splitk_sum_kernel(const float* __restrict__ P, int S, int64_t n, float* __restrict__ G) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        float s = 0.0f;
        for (int z = 0; z < S; ++z) s += P[(int64_t)z * n + e];
        G[e] = s;
    }
}

// Adam on the weights of one layer [O][I] (and the refresh of the BF16 copy
// and its transpose), then on the biases [O].
__global__ void adam_kernel(float* __restrict__ W, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ G, int64_t n, float lr, float c1, float c2, int O, int I,
                            bf16* __restrict__ Wb, bf16* __restrict__ WbT) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const float gr = G[e];
        const float mm = 0.9f * m[e] + 0.1f * gr;
        const float vv = 0.999f * v[e] + 0.001f * gr * gr;
        m[e] = mm;
        v[e] = vv;
        const float w = W[e] - lr * (mm * c1) / (sqrtf(vv * c2) + 1e-8f);
        W[e] = w;
        if (Wb) {
            const int o = (int)(e / I), i = (int)(e % I);
            const bf16 wb = __float2bfloat16_rn(w);
            Wb[e] = wb;
            WbT[(int64_t)i * O + o] = wb;
        }
    }
}

// BF16 copy of the FP32 weights [O][I] and its transpose.
__global__ void cast_weights_kernel(const float* __restrict__ W, int O, int I, bf16* __restrict__ Wb,
                                    bf16* __restrict__ WbT) {
    const int64_t n = (int64_t)O * I;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int o = (int)(e / I), i = (int)(e % I);
        const bf16 wb = __float2bfloat16_rn(W[e]);
        Wb[e] = wb;
        WbT[(int64_t)i * O + o] = wb;
    }
}

// A training batch: row r takes training row splitmix64(key + r) mod n.
__global__ void sample_kernel(const bf16* __restrict__ feat, const float* __restrict__ targ, int64_t n, uint64_t key,
                              int R, bf16* __restrict__ X, float* __restrict__ T) {
    const int r = blockIdx.x;
    const int64_t src = (int64_t)(splitmix64(key + (uint64_t)r) % (uint64_t)n);
    for (int c = threadIdx.x; c < kF; c += blockDim.x) X[(int64_t)r * kF + c] = feat[src * kF + c];
    if (threadIdx.x < 4) T[(int64_t)r * 4 + threadIdx.x] = targ[src * 4 + threadIdx.x];
}

// ------------------------------------------------------------- features
// Sum of `in` over a window of half-width h along one axis of the dense
// grid [nz][ny][nx]: clamped at the ends of x, periodic in y and z.  With
// count != NULL the window sizes are accumulated too (x only).
__global__ void box_kernel(const float* __restrict__ in, float* __restrict__ out, int nx, int ny, int nz, int axis,
                           int h, const float* __restrict__ cnt_in, float* __restrict__ cnt_out) {
    const int64_t N = (int64_t)nx * ny * nz;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(e % nx);
        const int y = (int)((e / nx) % ny);
        const int z = (int)(e / ((int64_t)nx * ny));
        float s = 0.0f, c = 0.0f;
        for (int d = -h; d <= h; ++d) {
            int64_t j;
            if (axis == 0) {
                const int xx = x + d;
                if (xx < 0 || xx >= nx) continue;
                j = e + d;
            } else if (axis == 1) {
                const int yy = ((y + d) % ny + ny) % ny;
                j = e + (int64_t)(yy - y) * nx;
            } else {
                const int zz = ((z + d) % nz + nz) % nz;
                j = e + (int64_t)(zz - z) * nx * ny;
            }
            s += in[j];
            if (cnt_in) c += cnt_in[j];
        }
        out[e] = s;
        if (cnt_out) cnt_out[e] = c;
    }
}

// w[e] = w[e] / cnt[e]: window sum to fluid fraction.
__global__ void divide_kernel(float* __restrict__ w, const float* __restrict__ cnt, int64_t N) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < N; e += (int64_t)gridDim.x * blockDim.x)
        w[e] = cnt[e] > 0.0f ? w[e] / cnt[e] : 0.0f;
}

// Feature row of fluid cell j (dense index cell[j]), one thread per column:
//  0-2 profile X at x, 3 x / (nx - 1), 4-6 fluid fraction of the windows,
//  7 current / 2, 8-10 inlet X, 11 (x / (nx - 1)) current / 2,
//  12 cross-section porosity at x, 13 normalised cumulative resistance,
//  14 1 / (4 cross-section porosity), 15 one; 16-63 zero.
__global__ void assemble_kernel(const int64_t* __restrict__ cell, int nf, int nx, const float* __restrict__ xtab,
                                const float* __restrict__ w1, const float* __restrict__ w3,
                                const float* __restrict__ w7, float cur, float xi0, float xi1, float xi2,
                                bf16* __restrict__ out) {
    const int j = blockIdx.x * blockDim.y + threadIdx.y;
    if (j >= nf) return;
    const int64_t e = cell[j];
    const int x = (int)(e % nx);
    const float* tx = xtab + (int64_t)x * 8;
    const float xr = tx[3];
    float f = 0.0f;
    switch (threadIdx.x) {
        case 0: f = tx[0]; break;
        case 1: f = tx[1]; break;
        case 2: f = tx[2]; break;
        case 3: f = xr; break;
        case 4: f = w1[e]; break;
        case 5: f = w3[e]; break;
        case 6: f = w7[e]; break;
        case 7: f = 0.5f * cur; break;
        case 8: f = xi0; break;
        case 9: f = xi1; break;
        case 10: f = xi2; break;
        case 11: f = 0.5f * cur * xr; break;
        case 12: f = tx[4]; break;
        case 13: f = tx[5]; break;
        case 14: f = tx[6]; break;
        case 15: f = 1.0f; break;
        default: f = 0.0f;
    }
    out[(int64_t)j * kF + threadIdx.x] = __float2bfloat16_rn(f);
}

// X_s = profile_s(x) + Y[j][s] / 100, clamped at 1e-6 and renormalised;
// out [3][nf] in FP64.
__global__ void predict_post_kernel(const float* __restrict__ Y, const int64_t* __restrict__ cell, int j0, int rows,
                                    int nf, int nx, const float* __restrict__ xtab, double* __restrict__ out) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = j0 + r;
    if (r >= rows || j >= nf) return;
    const int x = (int)(cell[j] % nx);
    double X[3], s = 0.0;
    for (int q = 0; q < 3; ++q) {
        double v = (double)xtab[(int64_t)x * 8 + q] + (double)Y[(int64_t)r * kOutPad + q] / kTargetScale;
        v = v < 1e-6 ? 1e-6 : v;
        X[q] = v;
        s += v;
    }
    for (int q = 0; q < 3; ++q) out[(int64_t)q * nf + j] = X[q] / s;
}

}  // namespace

// ------------------------------------------------------------------ host
struct lbms_net {
    int width = 0, depth = 0, layers = 0;
    std::vector<int> in, out;               // padded sizes per layer
    std::vector<float*> W, b, mW, vW, mb, vb, gW, gb;
    std::vector<bf16*> Wb, WbT;
    std::vector<bf16*> act, actT;           // act[l] = input of layer l, [kMaxRows][in_l]
    bf16* dz[2] = {nullptr, nullptr};       // [kMaxRows][max width] ping-pong
    bf16* dzT = nullptr;                    // [max width][kMaxRows]
    float* P = nullptr;                     // GEMM partials
    size_t P_floats = 0;
    float* Y = nullptr;                     // [kMaxRows][kOutPad]
    float* T = nullptr;                     // [kMaxRows][4]
    double* loss = nullptr;
    bf16* feat = nullptr;                   // training rows [cap][kF]
    float* targ = nullptr;                  // [cap][4]
    int64_t n_rows = 0, cap = 0;
    int64_t step = 0;
    uint64_t seed = 0;
    unsigned int* gemm_err = nullptr;       // raised by the tensor-core GEMM on a timed-out wait
    int gemm_kind = LBMS_NET_GEMM_AUTO;
    int64_t tcgen05_calls = 0, mma_sync_calls = 0;
    std::vector<void*> allocs;
    std::string err;
};

namespace {

lbms_status nfail(lbms_net* n, lbms_status s, const char* fmt, ...) {
    if (n) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        std::vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        n->err = buf;
    }
    return s;
}

#define NCK(expr, what)                                                                               \
    do {                                                                                             \
        cudaError_t e_ = (expr);                                                                     \
        if (e_ != cudaSuccess) return nfail(n, LBMS_ECUDA, "%s: %s", what, cudaGetErrorString(e_)); \
    } while (0)

// Every request is recorded, failed ones as null, so that one scan of
// `allocs` finds a failure.
template <typename T>
T* nalloc(lbms_net* n, size_t count) {
    void* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) p = nullptr;
    n->allocs.push_back(p);
    return static_cast<T*>(p);
}

int grid_for(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 152 * 16); }

int64_t n_params(const lbms_net* n) {
    int64_t s = 0;
    for (int l = 0; l < n->layers; ++l) {
        const int o = l == n->layers - 1 ? kOut : n->out[l];
        s += (int64_t)o * n->in[l] + o;
    }
    return s;
}

// P[z] = A . B^T with the checks the kernel relies on.
// P = A . B^T on the fifth-generation tensor cores (tcgen05, lbms_umma.cu)
// whenever the shape allows it; otherwise, or when forced, the mma.sync
// kernel above.
lbms_status gemm(lbms_net* n, const bf16* A, int lda, const bf16* B, int ldb, int M, int N, int K, int S) {
    if ((size_t)S * M * N > n->P_floats)
        return nfail(n, LBMS_EINVAL, "internal GEMM shape %d x %d x %d (split %d) exceeds the partials", M, N, K, S);
    if (n->gemm_kind != LBMS_NET_GEMM_MMA_SYNC && lbms::umma_gemm_supported(A, lda, B, ldb, M, N, K, S) &&
        lbms::umma_gemm_init() == cudaSuccess) {
        NCK(lbms::umma_gemm_tn(A, lda, B, ldb, n->P, M, N, K, S, n->gemm_err, 0), "tensor-core gemm");
        ++n->tcgen05_calls;
        return LBMS_OK;
    }
    if (n->gemm_kind == LBMS_NET_GEMM_TCGEN05)
        return nfail(n, LBMS_EINVAL, "GEMM %d x %d x %d (split %d) is not supported by the tcgen05 kernel", M, N, K, S);
    if (M % kTM || N % kTN || K % (kTK * S) || lda % 8 || ldb % 8)
        return nfail(n, LBMS_EINVAL, "internal GEMM shape %d x %d x %d (split %d) not tileable", M, N, K, S);
    gemm_tn_kernel<<<dim3(N / kTN, M / kTM, S), 128>>>(A, lda, B, ldb, n->P, M, N, K / S);
    NCK(cudaGetLastError(), "gemm");
    ++n->mma_sync_calls;
    return LBMS_OK;
}

// Reads and clears the tensor-core GEMM's error flag (after the device work).
lbms_status check_gemm(lbms_net* n) {
    unsigned int f = 0;
    NCK(cudaMemcpy(&f, n->gemm_err, sizeof(f), cudaMemcpyDeviceToHost), "GEMM flag");
    if (!f) return LBMS_OK;
    NCK(cudaMemset(n->gemm_err, 0, sizeof(f)), "GEMM flag");
    return nfail(n, LBMS_ECUDA, "tensor-core GEMM: an mbarrier wait timed out (flag %u)", f);
}

lbms_status transpose(lbms_net* n, const bf16* in, bf16* out, int R, int C) {
    transpose_kernel<<<dim3(C / 32, R / 32), dim3(32, 8)>>>(in, out, R, C);
    NCK(cudaGetLastError(), "transpose");
    return LBMS_OK;
}

// Forward pass of R rows already in act[0]; with `train` the transposed
// activations are kept for the weight gradients.  Output in n->Y.
lbms_status forward(lbms_net* n, int R, bool train) {
    lbms_status st;
    for (int l = 0; l < n->layers; ++l) {
        const bool last = l == n->layers - 1;
        if (train) {
            st = transpose(n, n->act[l], n->actT[l], R, n->in[l]);
            if (st != LBMS_OK) return st;
        }
        st = gemm(n, n->act[l], n->in[l], n->Wb[l], n->in[l], R, n->out[l], n->in[l], 1);
        if (st != LBMS_OK) return st;
        bias_act_kernel<<<grid_for((int64_t)R * n->out[l]), 256>>>(n->P, n->b[l], R, n->out[l], last ? 0 : 1,
                                                                   last ? nullptr : n->act[l + 1],
                                                                   last ? n->Y : nullptr);
        NCK(cudaGetLastError(), "bias/activation");
    }
    return LBMS_OK;
}

// Backward pass and (lr > 0) Adam step for the R rows of the last forward
// pass with targets in n->T.  Gradients stay in gW / gb.
lbms_status backward_step(lbms_net* n, int R, double lr, double* loss) {
    lbms_status st;
    NCK(cudaMemset(n->loss, 0, sizeof(double)), "loss");
    for (int l = 0; l < n->layers; ++l) NCK(cudaMemset(n->gb[l], 0, n->out[l] * sizeof(float)), "bias grads");
    const int L = n->layers;
    loss_grad_kernel<<<R / 64, 256>>>(n->Y, n->T, R, n->dz[0], n->gb[L - 1], n->loss);
    NCK(cudaGetLastError(), "loss");
    int cur = 0;
    // split of the R-long reduction of the weight gradients: chunks of >= 512
    // rows, a divisor of R / 64 so that every chunk is whole 64-row steps (the
    // K step of the tcgen05 kernel; two of the mma.sync kernel's)
    int S = std::max(1, std::min(16, R / 512));
    while (S > 1 && (R / 64) % S) --S;
    for (int l = L - 1; l >= 0; --l) {
        const int O = n->out[l], I = n->in[l];
        // weight gradient: dZ^T [O][R] . act^T [I][R]
        st = transpose(n, n->dz[cur], n->dzT, R, O);
        if (st != LBMS_OK) return st;
        st = gemm(n, n->dzT, R, n->actT[l], R, O, I, R, S);
        if (st != LBMS_OK) return st;
        splitk_sum_kernel<<<grid_for((int64_t)O * I), 256>>>(n->P, S, (int64_t)O * I, n->gW[l]);
        NCK(cudaGetLastError(), "split-k sum");
        if (l > 0) {
            // input gradient: dZ [R][O] . W^T -> [R][I], then through the ReLU of layer l - 1
            st = gemm(n, n->dz[cur], O, n->WbT[l], O, R, I, O, 1);
            if (st != LBMS_OK) return st;
            relu_back_kernel<<<R / 32, 256>>>(n->P, n->act[l], R, I, n->dz[cur ^ 1], n->gb[l - 1]);
            NCK(cudaGetLastError(), "relu backward");
            cur ^= 1;
        }
    }
    if (lr > 0.0) {
        ++n->step;
        const float c1 = (float)(1.0 / (1.0 - std::pow(0.9, (double)n->step)));
        const float c2 = (float)(1.0 / (1.0 - std::pow(0.999, (double)n->step)));
        for (int l = 0; l < L; ++l) {
            const int64_t nw = (int64_t)n->out[l] * n->in[l];
            adam_kernel<<<grid_for(nw), 256>>>(n->W[l], n->mW[l], n->vW[l], n->gW[l], nw, (float)lr, c1, c2,
                                               n->out[l], n->in[l], n->Wb[l], n->WbT[l]);
            adam_kernel<<<grid_for(n->out[l]), 256>>>(n->b[l], n->mb[l], n->vb[l], n->gb[l], n->out[l], (float)lr,
                                                      c1, c2, n->out[l], 1, nullptr, nullptr);
            NCK(cudaGetLastError(), "adam");
        }
    }
    if (loss) NCK(cudaMemcpy(loss, n->loss, sizeof(double), cudaMemcpyDeviceToHost), "read loss");
    return LBMS_OK;
}

// Feature rows (device, [rows_pad][kF], zero padded) and the per-x table of
// one case; rows_pad = nf rounded up to 64.
struct CaseFeatures {
    bf16* rows = nullptr;
    float* xtab = nullptr;
    int64_t* cell = nullptr;
    int nf = 0, nx = 0, rows_pad = 0;
    std::vector<double> prof;
    std::vector<void*> tmp;
    ~CaseFeatures() {
        for (void* p : tmp) cudaFree(p);
    }
    template <typename T>
    T* alloc(size_t count) {   // failures are recorded as null (see nalloc)
        void* p = nullptr;
        if (cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) p = nullptr;
        tmp.push_back(p);
        return static_cast<T*>(p);
    }
};

lbms_status case_features(lbms_net* n, lbms_ctx* ctx, int k, CaseFeatures& F) {
    lbms::CaseView v;
    if (!lbms::case_view(ctx, k, &v)) return nfail(n, LBMS_EINVAL, "case index %d out of range", k);
    if (!v.has_bc) return nfail(n, LBMS_ESTATE, "case %d has no boundary data yet", k);
    if (v.periodic_x) return nfail(n, LBMS_EINVAL, "case %d is periodic in x (no inlet / outlet)", k);
    if (!lbms::case_profile_1d(ctx, k, F.prof))
        return nfail(n, LBMS_EDEPLETED, "the 1-D profile of case %d drives a mole fraction below zero", k);
    const int nx = v.nx, ny = v.ny, nz = v.nz;
    const int64_t N = v.N;
    F.nf = v.nf;
    F.nx = nx;
    F.rows_pad = (v.nf + 63) / 64 * 64;
    // host: dense fluid mask, per-x table (profile, x / (nx - 1), plane
    // porosity, normalised cumulative resistance, inverse porosity)
    std::vector<float> mask(N, 0.0f);
    for (int j = 0; j < v.nf; ++j) mask[v.fluid_cell[j]] = 1.0f;
    std::vector<double> phi(nx, 0.0);
    for (int64_t e = 0; e < N; ++e) phi[e % nx] += mask[e];
    for (int x = 0; x < nx; ++x) phi[x] = std::max(phi[x] / ((double)ny * nz), 1.0 / ((double)ny * nz));
    std::vector<double> res(nx, 0.0);
    for (int x = 1; x < nx; ++x) res[x] = res[x - 1] + 0.5 * (1.0 / phi[x - 1] + 1.0 / phi[x]);
    std::vector<float> xtab((size_t)nx * 8, 0.0f);
    for (int x = 0; x < nx; ++x) {
        for (int s = 0; s < 3; ++s) xtab[(size_t)x * 8 + s] = (float)F.prof[(size_t)s * nx + x];
        xtab[(size_t)x * 8 + 3] = (float)x / (float)(nx - 1);
        xtab[(size_t)x * 8 + 4] = (float)phi[x];
        xtab[(size_t)x * 8 + 5] = (float)(res[nx - 1] > 0 ? res[x] / res[nx - 1] : 0.0);
        xtab[(size_t)x * 8 + 6] = (float)(0.25 / phi[x]);
    }
    float* dmask = F.alloc<float>(N);
    float* ones = F.alloc<float>(N);
    float* t0 = F.alloc<float>(N);
    float* t1 = F.alloc<float>(N);
    float* c0 = F.alloc<float>(N);
    float* c1 = F.alloc<float>(N);
    float* w[3] = {F.alloc<float>(N), F.alloc<float>(N), F.alloc<float>(N)};
    float* cnt[3] = {F.alloc<float>(N), F.alloc<float>(N), F.alloc<float>(N)};
    F.xtab = F.alloc<float>(xtab.size());
    F.cell = F.alloc<int64_t>(v.nf);
    F.rows = F.alloc<bf16>((size_t)F.rows_pad * kF);
    for (void* p : F.tmp)
        if (!p) return nfail(n, LBMS_ENOMEM, "feature buffers");
    NCK(cudaMemcpy(dmask, mask.data(), N * sizeof(float), cudaMemcpyHostToDevice), "mask");
    std::vector<float> one(N, 1.0f);
    NCK(cudaMemcpy(ones, one.data(), N * sizeof(float), cudaMemcpyHostToDevice), "ones");
    NCK(cudaMemcpy(F.xtab, xtab.data(), xtab.size() * sizeof(float), cudaMemcpyHostToDevice), "x table");
    NCK(cudaMemcpy(F.cell, v.fluid_cell, v.nf * sizeof(int64_t), cudaMemcpyHostToDevice), "cells");
    NCK(cudaMemset(F.rows, 0, (size_t)F.rows_pad * kF * sizeof(bf16)), "rows");
    const int hw[3] = {1, 3, 7};
    const int g = grid_for(N);
    for (int q = 0; q < 3; ++q) {
        // window sums of the mask and of the window sizes (x clamped)
        box_kernel<<<g, 256>>>(dmask, t0, nx, ny, nz, 0, hw[q], ones, c0);
        box_kernel<<<g, 256>>>(t0, t1, nx, ny, nz, 1, hw[q], c0, c1);
        box_kernel<<<g, 256>>>(t1, w[q], nx, ny, nz, 2, nz > 1 ? hw[q] : 0, c1, cnt[q]);
        NCK(cudaGetLastError(), "box filter");
    }
    for (int q = 0; q < 3; ++q) divide_kernel<<<g, 256>>>(w[q], cnt[q], N);
    const dim3 blk(kF, 4);
    assemble_kernel<<<(v.nf + 3) / 4, blk>>>(F.cell, v.nf, nx, F.xtab, w[0], w[1], w[2], (float)v.current,
                                             (float)v.x_in[0], (float)v.x_in[1], (float)v.x_in[2], F.rows);
    NCK(cudaGetLastError(), "features");
    return LBMS_OK;
}

lbms_status grow(lbms_net* n, int64_t need) {
    if (need <= n->cap) return LBMS_OK;
    int64_t cap = std::max<int64_t>(need, 2 * n->cap);
    bf16* f = nullptr;
    float* t = nullptr;
    NCK(cudaMalloc(&f, (size_t)cap * kF * sizeof(bf16)), "training rows");
    if (cudaMalloc(&t, (size_t)cap * 4 * sizeof(float)) != cudaSuccess) {
        cudaFree(f);
        return nfail(n, LBMS_ENOMEM, "training targets");
    }
    if (n->n_rows) {
        NCK(cudaMemcpy(f, n->feat, (size_t)n->n_rows * kF * sizeof(bf16), cudaMemcpyDeviceToDevice), "grow");
        NCK(cudaMemcpy(t, n->targ, (size_t)n->n_rows * 4 * sizeof(float), cudaMemcpyDeviceToDevice), "grow");
    }
    cudaFree(n->feat);
    cudaFree(n->targ);
    n->feat = f;
    n->targ = t;
    n->cap = cap;
    return LBMS_OK;
}

lbms_status upload_rows(lbms_net* n, const uint16_t* features, int rows) {
    if (!features || rows < 64 || rows > kMaxRows || rows % 64)
        return nfail(n, LBMS_EINVAL, "rows must be a multiple of 64 in [64, %d]", kMaxRows);
    NCK(cudaMemcpy(n->act[0], features, (size_t)rows * kF * sizeof(bf16), cudaMemcpyHostToDevice), "features");
    return LBMS_OK;
}

}  // namespace

extern "C" {

lbms_status lbms_net_create(int width, int depth, uint64_t seed, lbms_net** out) {
    if (!out) return LBMS_EINVAL;
    *out = nullptr;
    if (width < 64 || width > 2048 || width % 64 || depth < 1 || depth > 8) return LBMS_EINVAL;
    lbms_net* n = new (std::nothrow) lbms_net;
    if (!n) return LBMS_ENOMEM;
    n->width = width;
    n->depth = depth;
    n->layers = depth + 1;
    n->seed = seed;
    for (int l = 0; l < n->layers; ++l) {
        n->in.push_back(l == 0 ? kF : width);
        n->out.push_back(l == n->layers - 1 ? kOutPad : width);
    }
    bool ok = true;
    size_t pmax = (size_t)kMaxRows * std::max(width, kF);
    for (int l = 0; l < n->layers; ++l) {
        const size_t nw = (size_t)n->out[l] * n->in[l];
        pmax = std::max(pmax, (size_t)16 * nw);
        n->W.push_back(nalloc<float>(n, nw));
        n->mW.push_back(nalloc<float>(n, nw));
        n->vW.push_back(nalloc<float>(n, nw));
        n->gW.push_back(nalloc<float>(n, nw));
        n->b.push_back(nalloc<float>(n, n->out[l]));
        n->mb.push_back(nalloc<float>(n, n->out[l]));
        n->vb.push_back(nalloc<float>(n, n->out[l]));
        n->gb.push_back(nalloc<float>(n, n->out[l]));
        n->Wb.push_back(nalloc<bf16>(n, nw));
        n->WbT.push_back(nalloc<bf16>(n, nw));
        n->act.push_back(nalloc<bf16>(n, (size_t)kMaxRows * n->in[l]));
        n->actT.push_back(nalloc<bf16>(n, (size_t)kMaxRows * n->in[l]));
    }
    const size_t wmax = std::max(width, kOutPad);
    n->dz[0] = nalloc<bf16>(n, (size_t)kMaxRows * wmax);
    n->dz[1] = nalloc<bf16>(n, (size_t)kMaxRows * wmax);
    n->dzT = nalloc<bf16>(n, (size_t)kMaxRows * wmax);
    n->P = nalloc<float>(n, pmax);
    n->P_floats = pmax;
    n->Y = nalloc<float>(n, (size_t)kMaxRows * kOutPad);
    n->T = nalloc<float>(n, (size_t)kMaxRows * 4);
    n->loss = nalloc<double>(n, 1);
    n->gemm_err = nalloc<unsigned int>(n, 1);
    for (void* p : n->allocs) ok = ok && p;
    if (!ok) {
        lbms_net_destroy(n);
        return LBMS_ENOMEM;
    }
    // He-uniform hidden layers, zero output layer and biases; moments zero
    for (int l = 0; l < n->layers; ++l) {
        const size_t nw = (size_t)n->out[l] * n->in[l];
        std::vector<float> w(nw, 0.0f);
        if (l < n->layers - 1) {
            const double a = std::sqrt(6.0 / (l == 0 ? kFUsed : n->in[l]));
            for (size_t e = 0; e < nw; ++e)
                w[e] = (float)(a * (2.0 * unit_double(seed * 0x100000001ull + (uint64_t)l * 0x1000000000ull + e) - 1.0));
        }
        if (cudaMemcpy(n->W[l], w.data(), nw * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) ok = false;
        cudaMemset(n->gemm_err, 0, sizeof(unsigned int));
        cudaMemset(n->mW[l], 0, nw * sizeof(float));
        cudaMemset(n->vW[l], 0, nw * sizeof(float));
        cudaMemset(n->gW[l], 0, nw * sizeof(float));
        cudaMemset(n->b[l], 0, n->out[l] * sizeof(float));
        cudaMemset(n->mb[l], 0, n->out[l] * sizeof(float));
        cudaMemset(n->vb[l], 0, n->out[l] * sizeof(float));
        cudaMemset(n->gb[l], 0, n->out[l] * sizeof(float));
        cast_weights_kernel<<<grid_for((int64_t)nw), 256>>>(n->W[l], n->out[l], n->in[l], n->Wb[l], n->WbT[l]);
    }
    for (int l = 0; l < n->layers; ++l)
        cudaMemset(n->act[l], 0, (size_t)kMaxRows * n->in[l] * sizeof(bf16));
    if (!ok || cudaDeviceSynchronize() != cudaSuccess) {
        lbms_net_destroy(n);
        return LBMS_ECUDA;
    }
    *out = n;
    return LBMS_OK;
}

void lbms_net_destroy(lbms_net* n) {
    if (!n) return;
    for (void* p : n->allocs) cudaFree(p);
    cudaFree(n->feat);
    cudaFree(n->targ);
    delete n;
}

const char* lbms_net_last_error(const lbms_net* n) { return n ? n->err.c_str() : ""; }

lbms_status lbms_net_info(const lbms_net* n, int64_t* np, int64_t* ns) {
    if (!n) return LBMS_EINVAL;
    if (np) *np = n_params(n);
    if (ns) *ns = n->n_rows;
    return LBMS_OK;
}

lbms_status lbms_net_features(lbms_net* n, lbms_ctx* ctx, int k, uint16_t* rows, int64_t n_rows) {
    if (!n || !ctx || !rows) return LBMS_EINVAL;
    lbms::CaseView v;
    if (!lbms::case_view(ctx, k, &v)) return nfail(n, LBMS_EINVAL, "case index %d out of range", k);
    if (n_rows != v.nf) return nfail(n, LBMS_EINVAL, "case %d has %d fluid cells, the buffer holds %lld rows", k, v.nf,
                                     (long long)n_rows);
    CaseFeatures F;
    lbms_status st = case_features(n, ctx, k, F);
    if (st != LBMS_OK) return st;
    NCK(cudaMemcpy(rows, F.rows, (size_t)v.nf * kF * sizeof(bf16), cudaMemcpyDeviceToHost), "feature rows");
    return LBMS_OK;
}

lbms_status lbms_net_add_sample(lbms_net* n, lbms_ctx* ctx, int k) {
    if (!n || !ctx) return LBMS_EINVAL;
    CaseFeatures F;
    lbms_status st = case_features(n, ctx, k, F);
    if (st != LBMS_OK) return st;
    lbms::CaseView v;
    lbms::case_view(ctx, k, &v);
    std::vector<double> X((size_t)3 * v.N);
    st = lbms_batch_get_fields(ctx, k, X.data(), nullptr, nullptr);
    if (st != LBMS_OK) return nfail(n, st, "reading the fields of case %d: %s", k, lbms_last_error(ctx));
    std::vector<float> t((size_t)v.nf * 4, 0.0f);
    for (int j = 0; j < v.nf; ++j) {
        const int64_t e = v.fluid_cell[j];
        const int x = (int)(e % v.nx);
        for (int s = 0; s < 3; ++s)
            t[(size_t)j * 4 + s] = (float)(kTargetScale * (X[(size_t)s * v.N + e] - F.prof[(size_t)s * v.nx + x]));
    }
    st = grow(n, n->n_rows + v.nf);
    if (st != LBMS_OK) return st;
    NCK(cudaMemcpy(n->feat + n->n_rows * kF, F.rows, (size_t)v.nf * kF * sizeof(bf16), cudaMemcpyDeviceToDevice),
        "append rows");
    NCK(cudaMemcpy(n->targ + n->n_rows * 4, t.data(), t.size() * sizeof(float), cudaMemcpyHostToDevice),
        "append targets");
    n->n_rows += v.nf;
    return LBMS_OK;
}

lbms_status lbms_net_train(lbms_net* n, int iters, int batch, double lr, double* last_loss) {
    if (!n) return LBMS_EINVAL;
    if (iters < 0 || batch < 64 || batch > kMaxRows || batch % 64 || !(lr > 0.0))
        return nfail(n, LBMS_EINVAL, "need iters >= 0, batch a multiple of 64 in [64, %d], lr > 0", kMaxRows);
    if (n->n_rows < 1) return nfail(n, LBMS_ESTATE, "no training rows (call lbms_net_add_sample first)");
    double tail = 0.0;
    int nt = 0;
    for (int it = 0; it < iters; ++it) {
        const double cw = 0.5 * (1.0 + std::cos(3.14159265358979323846 * (double)it / std::max(1, iters)));
        const double lr_it = lr / 20.0 + (lr - lr / 20.0) * cw;
        const uint64_t key = splitmix64(n->seed ^ 0xA5A5A5A5ull) + (uint64_t)n->step * (uint64_t)kMaxRows;
        sample_kernel<<<batch, 64>>>(n->feat, n->targ, n->n_rows, key, batch, n->act[0], n->T);
        NCK(cudaGetLastError(), "sample");
        lbms_status st = forward(n, batch, true);
        if (st != LBMS_OK) return st;
        const bool want = it >= iters - 10;
        double l = 0.0;
        st = backward_step(n, batch, lr_it, want ? &l : nullptr);
        if (st != LBMS_OK) return st;
        if (want) {
            tail += l;
            ++nt;
        }
    }
    NCK(cudaDeviceSynchronize(), "train");
    lbms_status gst = check_gemm(n);
    if (gst != LBMS_OK) return gst;
    if (last_loss) *last_loss = nt ? tail / nt : 0.0;
    return LBMS_OK;
}

lbms_status lbms_net_forward(lbms_net* n, const uint16_t* features, int rows, float* out) {
    if (!n || !out) return LBMS_EINVAL;
    lbms_status st = upload_rows(n, features, rows);
    if (st != LBMS_OK) return st;
    st = forward(n, rows, false);
    if (st != LBMS_OK) return st;
    std::vector<float> y((size_t)rows * kOutPad);
    NCK(cudaMemcpy(y.data(), n->Y, y.size() * sizeof(float), cudaMemcpyDeviceToHost), "read output");
    st = check_gemm(n);
    if (st != LBMS_OK) return st;
    for (int r = 0; r < rows; ++r)
        for (int s = 0; s < kOut; ++s) out[(size_t)r * kOut + s] = y[(size_t)r * kOutPad + s];
    return LBMS_OK;
}

lbms_status lbms_net_train_batch(lbms_net* n, const uint16_t* features, const float* targets, int rows, double lr,
                                 double* loss) {
    if (!n || !targets || !(lr >= 0.0)) return LBMS_EINVAL;
    lbms_status st = upload_rows(n, features, rows);
    if (st != LBMS_OK) return st;
    std::vector<float> t((size_t)rows * 4, 0.0f);
    for (int r = 0; r < rows; ++r)
        for (int s = 0; s < kOut; ++s) t[(size_t)r * 4 + s] = targets[(size_t)r * kOut + s];
    NCK(cudaMemcpy(n->T, t.data(), t.size() * sizeof(float), cudaMemcpyHostToDevice), "targets");
    st = forward(n, rows, true);
    if (st != LBMS_OK) return st;
    st = backward_step(n, rows, lr, loss);
    if (st != LBMS_OK) return st;
    NCK(cudaDeviceSynchronize(), "train batch");
    return check_gemm(n);
}

lbms_status lbms_net_set_gemm(lbms_net* n, int kind) {
    if (!n || (kind != LBMS_NET_GEMM_AUTO && kind != LBMS_NET_GEMM_TCGEN05 && kind != LBMS_NET_GEMM_MMA_SYNC))
        return LBMS_EINVAL;
    if (kind == LBMS_NET_GEMM_TCGEN05) {
        const cudaError_t e = lbms::umma_gemm_init();
        if (e != cudaSuccess) return nfail(n, LBMS_ECUDA, "tcgen05 GEMM unavailable: %s", cudaGetErrorString(e));
    }
    n->gemm_kind = kind;
    return LBMS_OK;
}

lbms_status lbms_net_gemm_calls(const lbms_net* n, int64_t* tcgen05, int64_t* mma_sync) {
    if (!n) return LBMS_EINVAL;
    if (tcgen05) *tcgen05 = n->tcgen05_calls;
    if (mma_sync) *mma_sync = n->mma_sync_calls;
    return LBMS_OK;
}

lbms_status lbms_net_get(const lbms_net* cn, int what, float* buf, int64_t count) {
    lbms_net* n = const_cast<lbms_net*>(cn);
    if (!n || !buf || (what != 0 && what != 1)) return LBMS_EINVAL;
    if (count < n_params(n)) return nfail(n, LBMS_EINVAL, "buffer holds %lld floats, need %lld", (long long)count,
                                          (long long)n_params(n));
    int64_t off = 0;
    for (int l = 0; l < n->layers; ++l) {
        const int o = l == n->layers - 1 ? kOut : n->out[l];
        const size_t nw = (size_t)o * n->in[l];   // the first o rows of [out][in]
        NCK(cudaMemcpy(buf + off, what ? n->gW[l] : n->W[l], nw * sizeof(float), cudaMemcpyDeviceToHost), "get");
        off += nw;
        NCK(cudaMemcpy(buf + off, what ? n->gb[l] : n->b[l], o * sizeof(float), cudaMemcpyDeviceToHost), "get");
        off += o;
    }
    return LBMS_OK;
}

lbms_status lbms_net_set(lbms_net* n, const float* buf, int64_t count) {
    if (!n || !buf) return LBMS_EINVAL;
    if (count < n_params(n)) return nfail(n, LBMS_EINVAL, "buffer holds %lld floats, need %lld", (long long)count,
                                          (long long)n_params(n));
    int64_t off = 0;
    for (int l = 0; l < n->layers; ++l) {
        const int o = l == n->layers - 1 ? kOut : n->out[l];
        const size_t nw = (size_t)o * n->in[l];
        NCK(cudaMemcpy(n->W[l], buf + off, nw * sizeof(float), cudaMemcpyHostToDevice), "set");
        off += nw;
        NCK(cudaMemcpy(n->b[l], buf + off, o * sizeof(float), cudaMemcpyHostToDevice), "set");
        off += o;
        cast_weights_kernel<<<grid_for((int64_t)n->out[l] * n->in[l]), 256>>>(n->W[l], n->out[l], n->in[l],
                                                                              n->Wb[l], n->WbT[l]);
        NCK(cudaGetLastError(), "cast");
    }
    NCK(cudaDeviceSynchronize(), "set");
    return LBMS_OK;
}

lbms_status lbms_net_warm_start(lbms_net* n, lbms_ctx* ctx, int k, double* Xout) {
    if (!n || !ctx) return LBMS_EINVAL;
    CaseFeatures F;
    lbms_status st = case_features(n, ctx, k, F);
    if (st != LBMS_OK) return st;
    lbms::CaseView v;
    lbms::case_view(ctx, k, &v);
    double* dX = F.alloc<double>((size_t)3 * v.nf);
    if (!dX) return nfail(n, LBMS_ENOMEM, "prediction buffer");
    for (int j0 = 0; j0 < F.rows_pad; j0 += kMaxRows) {
        const int rows = std::min(kMaxRows, F.rows_pad - j0);
        NCK(cudaMemcpy(n->act[0], F.rows + (size_t)j0 * kF, (size_t)rows * kF * sizeof(bf16),
                       cudaMemcpyDeviceToDevice),
            "rows");
        st = forward(n, rows, false);
        if (st != LBMS_OK) return st;
        predict_post_kernel<<<(rows + 255) / 256, 256>>>(n->Y, F.cell, j0, rows, v.nf, v.nx, F.xtab, dX);
        NCK(cudaGetLastError(), "prediction");
    }
    std::vector<double> c((size_t)3 * v.nf);
    NCK(cudaMemcpy(c.data(), dX, c.size() * sizeof(double), cudaMemcpyDeviceToHost), "read prediction");
    std::vector<double> X((size_t)3 * v.N, 0.0);
    for (int s = 0; s < 3; ++s)
        for (int j = 0; j < v.nf; ++j) X[(size_t)s * v.N + v.fluid_cell[j]] = c[(size_t)s * v.nf + j];
    st = lbms_batch_set_fields(ctx, k, X.data());
    if (st != LBMS_OK) return nfail(n, st, "restarting case %d: %s", k, lbms_last_error(ctx));
    if (Xout) std::copy(X.begin(), X.end(), Xout);
    return LBMS_OK;
}

}  // extern "C"

#include "lbms_unet.cuh"
