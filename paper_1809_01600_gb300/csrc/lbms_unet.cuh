// The convolutional warm start (declared in include/lbms_net.h): a 3-D U-Net
// over the anode's voxels, trained and run with this file's kernels and the
// tcgen05 kernels of lbms_umma.cu.  Included at the end of lbms_net.cu, whose
// feature builder, split-K sum, Adam and weight-cast kernels it shares.
//
// Layout.  Activations are channels-last BF16 rows [row][C] (C a multiple
// of 64, the real channels first, zeros after).  Each volume of X x Y x Z
// voxels is stored with a zero halo of one voxel per side, in Xp x Yp x Zp
// rows (Xp = X + 2 rounded up to a multiple of 8, Yp = Y + 2, Zp = Z + 2),
// volumes one after the other; the row count is padded to a multiple of 64 S
// (S chunks of the reductions over rows).  The neighbour of a voxel at tap
// (dz, dy, dx) is then off = (dz Yp + dy) Xp + dx rows away, so a 3x3x3
// convolution is an implicit GEMM on the tensor cores: the A tile of each
// tap is the activation matrix read at a shifted row (umma_conv_kernel,
// whose epilogue also adds the bias, applies ReLU and the zero halo and
// stores BF16).  Its input gradient is the same with the flipped weights
// and negated offsets, its weight gradient a product over rows against
// three shifted transposed copies of the input (load mode 2 of
// umma_gemm_kernel).  Every kernel that writes an activation writes all its
// rows, zeros outside the volumes, so the halo reads as zero padding
// whatever batch used the buffers before; an input gradient is masked the
// same way where its reader needs it (unet_backward says which).  The
// 2x2x2 transposed convolution of the decoder is one product whose 8 C
// columns go to the 8 children of each voxel; max pooling keeps the index
// of the first maximum.
namespace {

constexpr int kUInC = 64;      // stored input channels: the 16 feature columns, the fluid mask, zeros
constexpr int kUInReal = 17;
constexpr int kUOutC = 64;     // stored output channels of the 1x1 head (3 used)
constexpr int kULayers = 13;

// Layout of one resolution level of a batch (all row counts below 2^31).
struct Geo {
    int B = 0, X = 0, Y = 0, Z = 0;   // volumes; interior extents of one volume
    int Xp = 0, Yp = 0, Zp = 0;       // extents with the halo (Xp a multiple of 8)
    int64_t V = 0;                    // interior voxels of the batch
    int64_t R = 0;                    // rows of the layout, B Xp Yp Zp
    int64_t Rp = 0;                   // rows processed: R padded to a multiple of 64 S
    int S = 1;                        // chunks of the reductions over rows
};

// Interior coordinates of row r; false for halo and padding rows.
__device__ __forceinline__ bool row_voxel(const Geo& g, int64_t r, int& x, int& y, int& z, int& b) {
    if (r >= g.R) return false;
    unsigned q = (unsigned)r;
    x = (int)(q % (unsigned)g.Xp) - 1;
    q /= (unsigned)g.Xp;
    y = (int)(q % (unsigned)g.Yp) - 1;
    q /= (unsigned)g.Yp;
    z = (int)(q % (unsigned)g.Zp) - 1;
    b = (int)(q / (unsigned)g.Zp);
    return x >= 0 && x < g.X && y >= 0 && y < g.Y && z >= 0 && z < g.Z;
}

__device__ __forceinline__ int64_t voxel_row(const Geo& g, int b, int x, int y, int z) {
    return (((int64_t)b * g.Zp + z + 1) * g.Yp + y + 1) * g.Xp + x + 1;
}

// One warp per row: the global warp index and the warp count of the grid.
__device__ __forceinline__ int64_t warp_id() { return ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; }
__device__ __forceinline__ int64_t warp_count() { return ((int64_t)gridDim.x * blockDim.x) >> 5; }

// dst[r][c] = P[r][c] on interior rows, 0 elsewhere (FP32 gradients).
__global__ void mask_rows_kernel(const float* __restrict__ P, Geo g, int C, float* __restrict__ dst) {
    const int lane = threadIdx.x & 31;
    for (int64_t r = warp_id(); r < g.Rp; r += warp_count()) {
        int x, y, z, b;
        const bool in = row_voxel(g, r, x, y, z, b);
        for (int c = lane; c < C; c += 32) dst[r * C + c] = in ? P[r * C + c] : 0.0f;
    }
}

// 2x2x2 max pooling from level `hi` to level `lo` (C channels): every row
// of lo, the maximum of the 8 children and the child (dz 4 + dy 2 + dx) of
// the first maximum on interior rows, 0 elsewhere.
__global__ void pool_rows_kernel(const bf16* __restrict__ x, Geo hi, Geo lo, int C, bf16* __restrict__ y,
                                 uint8_t* __restrict__ arg) {
    const int lane = threadIdx.x & 31;
    for (int64_t r = warp_id(); r < lo.Rp; r += warp_count()) {
        int xl, yl, zl, b;
        const bool in = row_voxel(lo, r, xl, yl, zl, b);
        const int64_t c0 = in ? voxel_row(hi, b, 2 * xl, 2 * yl, 2 * zl) : 0;
        for (int c = lane; c < C; c += 32) {
            float best = 0.0f;
            int bi = 0;
            if (in) {
                best = -3.0e38f;
                for (int t = 0; t < 8; ++t) {
                    const int64_t w = c0 + ((int64_t)(t >> 2) * hi.Yp + ((t >> 1) & 1)) * hi.Xp + (t & 1);
                    const float v = __bfloat162float(x[w * C + c]);
                    if (v > best) {
                        best = v;
                        bi = t;
                    }
                }
            }
            y[r * C + c] = __float2bfloat16_rn(best);
            arg[r * C + c] = (uint8_t)bi;
        }
    }
}

// Gradient of the pooling: dx[r][c] += dp[parent][c] on the interior rows
// of hi that hold their parent's maximum.
__global__ void pool_back_rows_kernel(const float* __restrict__ dp, const uint8_t* __restrict__ arg, Geo hi, Geo lo,
                                      int C, float* __restrict__ dx) {
    const int lane = threadIdx.x & 31;
    for (int64_t r = warp_id(); r < hi.R; r += warp_count()) {
        int x, y, z, b;
        if (!row_voxel(hi, r, x, y, z, b)) continue;
        const int64_t p = voxel_row(lo, b, x >> 1, y >> 1, z >> 1);
        const int t = (z & 1) * 4 + (y & 1) * 2 + (x & 1);
        for (int c = lane; c < C; c += 32)
            if (arg[p * C + c] == t) dx[r * C + c] += dp[p * C + c];
    }
}

// Transposed 2x2x2 convolution, stride 2: every row of hi, y[r][c] =
// P[parent][t C + c] + b[c] with t the row's child index, on interior rows;
// 0 elsewhere.
__global__ void up_rows_kernel(const float* __restrict__ P, const float* __restrict__ bias, Geo lo, Geo hi, int C,
                               bf16* __restrict__ y) {
    const int lane = threadIdx.x & 31;
    for (int64_t r = warp_id(); r < hi.Rp; r += warp_count()) {
        int x, yy, z, b;
        const bool in = row_voxel(hi, r, x, yy, z, b);
        const int64_t p = in ? voxel_row(lo, b, x >> 1, yy >> 1, z >> 1) : 0;
        const int t = in ? (z & 1) * 4 + (yy & 1) * 2 + (x & 1) : 0;
        for (int c = lane; c < C; c += 32)
            y[r * C + c] = __float2bfloat16_rn(in ? P[p * 8 * C + t * C + c] + bias[c] : 0.0f);
    }
}

// Gradient of up_rows_kernel: every row of lo, G[r][t C + c] = dy[child t][c]
// (BF16) on interior rows, 0 elsewhere.
__global__ void upgather_rows_kernel(const float* __restrict__ dy, Geo lo, Geo hi, int C, bf16* __restrict__ G) {
    const int lane = threadIdx.x & 31;
    for (int64_t r = warp_id(); r < lo.Rp; r += warp_count()) {
        int xl, yl, zl, b;
        const bool in = row_voxel(lo, r, xl, yl, zl, b);
        const int64_t c0 = in ? voxel_row(hi, b, 2 * xl, 2 * yl, 2 * zl) : 0;
        for (int e = lane; e < 8 * C; e += 32) {
            float g = 0.0f;
            if (in) {
                const int t = e / C, c = e - t * C;
                g = dy[(c0 + ((int64_t)(t >> 2) * hi.Yp + ((t >> 1) & 1)) * hi.Xp + (t & 1)) * C + c];
            }
            G[r * 8 * C + e] = __float2bfloat16_rn(g);
        }
    }
}

// out[r] = (a[r][0:na], b[r][0:nb], zeros) with Co stored channels, R rows.
__global__ void concat_kernel(const bf16* __restrict__ a, int Ca, int na, const bf16* __restrict__ bsrc, int Cb, int nb,
                              int64_t R, int Co, bf16* __restrict__ out) {
    const int64_t n = R * Co;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / Co;
        const int c = (int)(e % Co);
        out[e] = c < na ? a[r * Ca + c] : c < na + nb ? bsrc[r * Cb + (c - na)] : __float2bfloat16_rn(0.0f);
    }
}

// The gradient of concat_kernel: da[r][c] = d[r][c] (c < na, else 0) and
// db[r][c] = d[r][na + c] (c < nb, else 0), with d stored Cd wide.
__global__ void split_kernel(const float* __restrict__ d, int Cd, int na, int nb, int Ca, int Cb, int64_t R,
                             float* __restrict__ da, float* __restrict__ db) {
    const int Cm = Ca > Cb ? Ca : Cb;
    const int64_t n = R * Cm;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / Cm;
        const int c = (int)(e % Cm);
        if (c < Ca) da[r * Ca + c] = c < na ? d[r * Cd + c] : 0.0f;
        if (c < Cb) db[r * Cb + c] = c < nb ? d[r * Cd + na + c] : 0.0f;
    }
}

// Column sums of a FP32 [R][C] added into acc (R a multiple of 32).
__global__ void colsum_kernel(const float* __restrict__ d, int64_t R, int C, float* __restrict__ acc) {
    const int64_t r0 = (int64_t)blockIdx.x * 32;
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        float s = 0.0f;
        for (int64_t r = r0; r < r0 + 32; ++r) s += d[r * C + c];
        atomicAdd(&acc[c], s);
    }
}

// ncopy transposed copies of in [R][C]: out[j][c][r] = in[r + j + shift0][c]
// (0 where that row is outside [0, R)); R and C multiples of 64.  A block of
// 256 threads reads 64 + ncopy - 1 rows x 64 channels once (16-byte loads)
// and writes the 64 x 64 tiles of every copy (16-byte stores, 8 threads per
// 128-byte output row).  The shared tile's rows are 33 words apart, so the
// 8 rows a warp reads at once fall in 2 ways of the banks.
__global__ void __launch_bounds__(256) transpose_copies_kernel(const bf16* __restrict__ in, bf16* __restrict__ out,
                                                               int64_t R, int C, int ncopy, int shift0) {
    __shared__ __align__(16) bf16 tile[66][66];
    const int64_t r0 = (int64_t)blockIdx.x * 64;
    const int c0 = blockIdx.y * 64;
    const int nrows = 64 + ncopy - 1;
    for (int e = threadIdx.x; e < nrows * 8; e += 256) {
        const int i = e >> 3, q = (e & 7) * 8;
        const int64_t rs = r0 + i + shift0;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (rs >= 0 && rs < R) v = *reinterpret_cast<const uint4*>(in + rs * C + c0 + q);
        uint32_t* d = reinterpret_cast<uint32_t*>(&tile[i][q]);
        d[0] = v.x;
        d[1] = v.y;
        d[2] = v.z;
        d[3] = v.w;
    }
    __syncthreads();
    for (int j = 0; j < ncopy; ++j) {
        bf16* o = out + (size_t)j * C * R;
        for (int e = threadIdx.x; e < 64 * 8; e += 256) {
            const int c = e >> 3, q = (e & 7) * 8;
            __align__(16) bf16 v[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = tile[q + k + j][c];
            *reinterpret_cast<uint4*>(o + (int64_t)(c0 + c) * R + r0 + q) = *reinterpret_cast<const uint4*>(v);
        }
    }
}

// dZ = dA * (act > 0) as BF16 [R][C] (C 64 or 128) and the column sums of
// dZ added into gb; a block of 256 threads per 64 rows.
__global__ void __launch_bounds__(256) relu_back_rows_kernel(const float* __restrict__ dA, const bf16* __restrict__ act,
                                                             int64_t R, int C, bf16* __restrict__ dZ,
                                                             float* __restrict__ gb) {
    __shared__ float part[256];
    const int64_t r0 = (int64_t)blockIdx.x * 64;
    const int c = threadIdx.x % C, g = threadIdx.x / C, ng = 256 / C;
    float s = 0.0f;
    for (int64_t r = r0 + g; r < r0 + 64 && r < R; r += ng) {
        const int64_t e = r * C + c;
        const float v = __bfloat162float(act[e]) > 0.0f ? dA[e] : 0.0f;
        dZ[e] = __float2bfloat16_rn(v);
        s += v;
    }
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x < C) {
        float t = 0.0f;
        for (int k = 0; k < ng; ++k) t += part[k * C + threadIdx.x];
        atomicAdd(&gb[threadIdx.x], t);
    }
}

// G[o][i] = sum_z P[z][i][o] (split-K partials of a transposed product).
__global__ void splitk_sum_t_kernel(const float* __restrict__ P, int S, int I, int O, float* __restrict__ G) {
    const int64_t n = (int64_t)O * I;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int o = (int)(e / I), i = (int)(e % I);
        float acc = 0.0f;
        for (int z = 0; z < S; ++z) acc += P[(int64_t)z * n + (int64_t)i * O + o];
        G[e] = acc;
    }
}

// BF16 copies of a 3x3x3 convolution's FP32 weights W [co_s][27 ci_s]
// (entry (co, tap ci_s + ci)): Wb, the same layout, and Wf [ci_s][27 co_s],
// the flipped weights of the input gradient, entry (ci, tap co_s + co).
__global__ void conv_cast_kernel(const float* __restrict__ W, int co_s, int ci_s, bf16* __restrict__ Wb,
                                 bf16* __restrict__ Wf) {
    const int K = 27 * ci_s;
    const int64_t n = (int64_t)co_s * K;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int co = (int)(e / K), k = (int)(e % K);
        const int tap = k / ci_s, ci = k - tap * ci_s;
        const bf16 wb = __float2bfloat16_rn(W[e]);
        Wb[e] = wb;
        Wf[(int64_t)ci * 27 * co_s + tap * co_s + co] = wb;
    }
}

// A batch given as FP32 [B][17][Z][Y][X] (channel 16 the fluid mask) into
// the interior rows of x0 [rows][64] (BF16) and the mask column of T [rows][4]
// (both cleared before); one warp per voxel.
__global__ void vol_in_kernel(const float* __restrict__ in, Geo g, bf16* __restrict__ x0, float* __restrict__ T) {
    const int lane = threadIdx.x & 31;
    const int64_t S = (int64_t)g.X * g.Y * g.Z;
    for (int64_t v = warp_id(); v < g.V; v += warp_count()) {
        const int b = (int)(v / S);
        const int64_t s = v - b * S;
        const int x = (int)(s % g.X), y = (int)((s / g.X) % g.Y), z = (int)(s / ((int64_t)g.X * g.Y));
        const int64_t r = voxel_row(g, b, x, y, z);
        for (int c = lane; c < kUInC; c += 32) {
            const float val = c < kUInReal ? in[((int64_t)b * kUInReal + c) * S + s] : 0.0f;
            x0[r * kUInC + c] = __float2bfloat16_rn(val);
            if (c == kUInReal - 1) T[r * 4 + 3] = val;
        }
    }
}

// Targets given as FP32 [B][3][Z][Y][X] into T[row][0:3] of the interior rows.
__global__ void vol_target_kernel(const float* __restrict__ t, Geo g, float* __restrict__ T) {
    const int64_t S = (int64_t)g.X * g.Y * g.Z;
    for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < g.V; v += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(v / S);
        const int64_t s = v - b * S;
        const int x = (int)(s % g.X), y = (int)((s / g.X) % g.Y), z = (int)(s / ((int64_t)g.X * g.Y));
        const int64_t r = voxel_row(g, b, x, y, z);
        for (int c = 0; c < 3; ++c) T[r * 4 + c] = t[((int64_t)b * 3 + c) * S + s];
    }
}

// Input rows of one case: vol[row[j]][c] = rows[j][c] (c < 16), the fluid
// mask in channel 16; every other row stays zero (cleared before).
__global__ void unet_inputs_kernel(const bf16* __restrict__ rows, const int64_t* __restrict__ row, int nf,
                                   bf16* __restrict__ vol) {
    const int64_t n = (int64_t)nf * kUInC;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e / kUInC), c = (int)(e % kUInC);
        bf16 val = __float2bfloat16_rn(0.0f);
        if (c < kFUsed) val = rows[(int64_t)j * kF + c];
        else if (c == kFUsed) val = __float2bfloat16_rn(1.0f);
        vol[row[j] * kUInC + c] = val;
    }
}

// Masked mean-square error of the head's output Y = P + b (3 used columns)
// against T [r][4] = (3 targets, fluid mask) over R rows (a multiple of 64),
// one block of 256 threads per 64 rows: dP (BF16, zero in the padded
// columns), the head's bias gradient and the loss, with inv_n = 1 / (3 x
// fluid voxels); Y[r][c] (c < 3) is kept for predictions.
__global__ void unet_loss_kernel(const float* __restrict__ P, const float* __restrict__ b, const float* __restrict__ T,
                                 int64_t R, float inv_n, bf16* __restrict__ dP, float* __restrict__ gb,
                                 double* __restrict__ loss, float* __restrict__ Y) {
    __shared__ float colsum[3];
    __shared__ double lsum[256];
    if (threadIdx.x < 3) colsum[threadIdx.x] = 0.0f;
    __syncthreads();
    double l = 0.0;
    const int64_t r0 = (int64_t)blockIdx.x * 64;
    for (int e = threadIdx.x; e < 64 * kUOutC; e += 256) {
        const int64_t r = r0 + e / kUOutC;
        const int c = e % kUOutC;
        float g = 0.0f;
        if (r < R && c < 3) {
            const float y = P[r * kUOutC + c] + b[c];
            if (Y) Y[r * 4 + c] = y;
            if (T) {
                const float d = (y - T[r * 4 + c]) * T[r * 4 + 3];
                l += (double)d * d;
                g = 2.0f * inv_n * d;
                atomicAdd(&colsum[c], g);
            }
        }
        if (r < R && dP) dP[r * kUOutC + c] = __float2bfloat16_rn(g);
    }
    lsum[threadIdx.x] = l;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) lsum[threadIdx.x] += lsum[threadIdx.x + s];
        __syncthreads();
    }
    if (T && threadIdx.x == 0) atomicAdd(loss, lsum[0] * (double)inv_n);
    if (T && threadIdx.x < 3) atomicAdd(&gb[threadIdx.x], colsum[threadIdx.x]);
}

// The prediction of one case from the head's output Y [r][4] at its row
// row[j]: X_s = profile_s(x) + Y[row][s] / 100, clamped at 1e-6 and
// renormalised; out [3][nf] FP64.  Xp: the padded x extent (x = row mod Xp - 1).
__global__ void unet_post_kernel(const float* __restrict__ Y, const int64_t* __restrict__ row, int nf, int Xp,
                                 const float* __restrict__ xtab, double* __restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nf) return;
    const int64_t r = row[j];
    const int x = (int)(r % Xp) - 1;
    double X[3], s = 0.0;
    for (int q = 0; q < 3; ++q) {
        double val = (double)xtab[(int64_t)x * 8 + q] + (double)Y[r * 4 + q] / kTargetScale;
        val = val < 1e-6 ? 1e-6 : val;
        X[q] = val;
        s += val;
    }
    for (int q = 0; q < 3; ++q) out[(int64_t)q * nf + j] = X[q] / s;
}

}  // namespace

// ------------------------------------------------------------------ host
struct lbms_unet {
    struct Layer {
        int kind = 3;            // 3: 3x3x3 conv + ReLU, 2: 2x2x2 transposed conv (stride 2), 1: 1x1 head
        int level = 0;           // resolution level of the output (0 full, 1 half, 2 quarter)
        int ci = 0, ci_s = 0, co = 0, co_s = 0;   // real / stored channels
        int rows = 0, K = 0;     // FP32 master weights W [rows][K]
        float *W = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;
        float *b = nullptr, *mb = nullptr, *vb = nullptr, *gb = nullptr;   // [co_s]
        bf16* Wb = nullptr;      // BF16 copy of W
        bf16* Wt = nullptr;      // kind 3: flipped weights [ci_s][27 co_s]; kinds 1, 2: transpose of Wb [K][rows]
    };
    int width = 0;
    Layer L[kULayers];           // e1a e1b e2a e2b e3a e3b u2 d2a d2b u1 d1a d1b head
    int64_t vcap = 0;            // interior voxels of one batch at most
    // activations and scratch, sized for the largest batch layout so far (grown on demand)
    int64_t cap[3] = {0, 0, 0};  // rows per level the buffers hold
    bf16 *x0 = nullptr, *e1a = nullptr, *e1 = nullptr, *u1 = nullptr, *c1 = nullptr, *d1a = nullptr, *d1 = nullptr;
    bf16 *p1 = nullptr, *e2a = nullptr, *e2 = nullptr, *u2 = nullptr, *c2 = nullptr, *d2a = nullptr, *d2 = nullptr;
    bf16 *p2 = nullptr, *e3a = nullptr, *e3 = nullptr;
    uint8_t *arg1 = nullptr, *arg2 = nullptr;
    bf16 *dz = nullptr, *dzT = nullptr, *G = nullptr, *aT = nullptr, *xT = nullptr;
    float *P = nullptr, *fa = nullptr, *fb = nullptr, *fc = nullptr, *fd = nullptr, *Y = nullptr, *T = nullptr;
    size_t P_floats = 0, g_elems = 0, xT_elems = 0, f_floats = 0;
    std::vector<void*> bufs;     // the grown buffers
    double* loss = nullptr;
    unsigned int* gemm_err = nullptr;
    struct Sample {
        int X = 0, Y = 0, Z = 0;                // interior extents (multiples of 4)
        int64_t rows = 0, nfluid = 0;           // rows of its layout; fluid voxels
        bf16* in = nullptr;                     // [rows][64]
        float* tg = nullptr;                    // [rows][4]: 100 (X - profile), fluid mask
    };
    std::vector<Sample> samples;
    int64_t step = 0, tcgen05_calls = 0;
    uint64_t seed = 0;
    std::vector<void*> allocs;   // weights and the small fixed buffers
    std::string msg;
    lbms_net feat;               // error messages of the shared feature builder (holds no device memory)
};

namespace {

lbms_status ufail(lbms_unet* u, lbms_status s, const char* fmt, ...) {
    if (u) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        std::vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        u->msg = buf;
    }
    return s;
}

#define UCK(expr, what)                                                                               \
    do {                                                                                             \
        cudaError_t e_ = (expr);                                                                     \
        if (e_ != cudaSuccess) return ufail(u, LBMS_ECUDA, "%s: %s", what, cudaGetErrorString(e_)); \
    } while (0)

#define UST(call)                     \
    do {                              \
        lbms_status s_ = (call);      \
        if (s_ != LBMS_OK) return s_; \
    } while (0)

template <typename T>
T* ualloc(lbms_unet* u, size_t count) {
    void* p = nullptr;
    if (cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) p = nullptr;
    u->allocs.push_back(p);
    return static_cast<T*>(p);
}

// The reductions over rows (weight gradients) are split in S chunks of at
// most kChunkRows (+ 63) rows, so that one CTA of the tensor-core GEMM
// streams a few MB and ends far inside the GEMM's bound on each wait.
constexpr int64_t kChunkRows = 16384;
constexpr int64_t kGemmMaxRows = 65535ll * 128;   // grid limit of the GEMM's row tiles

int64_t splits_for(int64_t R) { return std::max<int64_t>(1, (R + kChunkRows - 1) / kChunkRows); }
int64_t padded_rows(int64_t R) {
    const int64_t q = 64 * splits_for(R);
    return (R + q - 1) / q * q;
}

Geo make_geo(int B, int X, int Y, int Z) {
    Geo g;
    g.B = B;
    g.X = X;
    g.Y = Y;
    g.Z = Z;
    g.Xp = (X + 2 + 7) / 8 * 8;
    g.Yp = Y + 2;
    g.Zp = Z + 2;
    g.V = (int64_t)B * X * Y * Z;
    g.R = (int64_t)B * g.Xp * g.Yp * g.Zp;
    g.S = (int)splits_for(g.R);
    g.Rp = padded_rows(g.R);
    return g;
}

// The three levels of a batch of B volumes of X x Y x Z voxels.
struct Levels {
    Geo g[3];
};

Levels levels_of(int B, int X, int Y, int Z) {
    Levels v;
    for (int l = 0; l < 3; ++l) v.g[l] = make_geo(B, X >> l, Y >> l, Z >> l);
    return v;
}

bool levels_fit(const Levels& v) {
    for (const auto& g : v.g)
        if (g.Rp > kGemmMaxRows) return false;
    return true;
}

// Grows the activation and scratch buffers to hold the layout of `v`.
lbms_status ensure_buffers(lbms_unet* u, const Levels& v) {
    int64_t c[3];
    bool grow = false;
    for (int l = 0; l < 3; ++l) {
        c[l] = std::max(u->cap[l], v.g[l].Rp);
        grow = grow || c[l] > u->cap[l];
    }
    if (!grow) return LBMS_OK;
    UCK(cudaDeviceSynchronize(), "U-Net buffers");
    for (void* p : u->bufs) cudaFree(p);
    u->bufs.clear();
    for (int l = 0; l < 3; ++l) u->cap[l] = 0;
    const size_t c0 = c[0], c1 = c[1], c2 = c[2];
    const size_t s0 = splits_for(c0), s1 = splits_for(c1), s2 = splits_for(c2);
    u->g_elems = std::max({c0 * 64, c1 * 512, c2 * 512});
    u->xT_elems = 3 * std::max({c0 * 64, c1 * 128, c2 * 128});
    u->f_floats = std::max({c0 * 64, c1 * 128, c2 * 128});
    u->P_floats = std::max({c0 * 64, c1 * 512, c2 * 512, s0 * 64 * 1728, s1 * 64 * 3456, s2 * 128 * 3456,
                            s1 * 512 * 64, s2 * 512 * 128, s0 * 64 * 64});
    bool ok = true;
    auto get = [&](size_t bytes) {
        void* p = nullptr;
        if (ok && cudaMalloc(&p, std::max<size_t>(bytes, 16)) == cudaSuccess) {
            u->bufs.push_back(p);
            ok = cudaMemset(p, 0, std::max<size_t>(bytes, 16)) == cudaSuccess;
        } else {
            ok = false;
        }
        return p;
    };
    auto act = [&](size_t rows, int C) { return static_cast<bf16*>(get(rows * C * sizeof(bf16))); };
    u->x0 = act(c0, kUInC);
    u->e1a = act(c0, 64);
    u->e1 = act(c0, 64);
    u->u1 = act(c0, 64);
    u->c1 = act(c0, 64);
    u->d1a = act(c0, 64);
    u->d1 = act(c0, 64);
    u->p1 = act(c1, 64);
    u->e2a = act(c1, 64);
    u->e2 = act(c1, 64);
    u->u2 = act(c1, 64);
    u->c2 = act(c1, 128);
    u->d2a = act(c1, 64);
    u->d2 = act(c1, 64);
    u->p2 = act(c2, 64);
    u->e3a = act(c2, 128);
    u->e3 = act(c2, 128);
    u->arg1 = static_cast<uint8_t*>(get(c1 * 64));
    u->arg2 = static_cast<uint8_t*>(get(c2 * 64));
    u->dz = static_cast<bf16*>(get(u->g_elems * sizeof(bf16)));
    u->dzT = static_cast<bf16*>(get(u->g_elems * sizeof(bf16)));
    u->G = static_cast<bf16*>(get(u->g_elems * sizeof(bf16)));
    u->aT = static_cast<bf16*>(get(u->g_elems * sizeof(bf16)));
    u->xT = static_cast<bf16*>(get(u->xT_elems * sizeof(bf16)));
    u->P = static_cast<float*>(get(u->P_floats * sizeof(float)));
    u->fa = static_cast<float*>(get(u->f_floats * sizeof(float)));
    u->fb = static_cast<float*>(get(u->f_floats * sizeof(float)));
    u->fc = static_cast<float*>(get(u->f_floats * sizeof(float)));
    u->fd = static_cast<float*>(get(u->f_floats * sizeof(float)));
    u->Y = static_cast<float*>(get(c0 * 4 * sizeof(float)));
    u->T = static_cast<float*>(get(c0 * 4 * sizeof(float)));
    if (!ok) {
        for (void* p : u->bufs) cudaFree(p);
        u->bufs.clear();
        return ufail(u, LBMS_ENOMEM, "U-Net buffers for %lld rows", (long long)c0);
    }
    for (int l = 0; l < 3; ++l) u->cap[l] = c[l];
    return LBMS_OK;
}

// Blocks of 256 threads for one warp per row over R rows (grid-stride beyond 152 x 16 blocks).
int warp_grid(int64_t R) { return (int)std::max<int64_t>(1, std::min<int64_t>((R + 7) / 8, 152 * 16)); }

// Tap table of a 3x3x3 convolution on layout g: row offsets sign * off(t).
lbms::ConvTaps conv_taps(const Geo& g, int per_tap, int sign) {
    lbms::ConvTaps t;
    t.per_tap = per_tap;
    for (int k = 0; k < 27; ++k) {
        const int dx = k % 3 - 1, dy = (k / 3) % 3 - 1, dz = k / 9 - 1;
        t.off[k] = sign * ((dz * g.Yp + dy) * g.Xp + dx);
    }
    return t;
}

// Tap table of the weight gradient: the shift (dz Yp + dy) Xp of the copy dx + 1.
lbms::ConvTaps wgrad_taps(const Geo& g, int C) {
    lbms::ConvTaps t;
    t.per_tap = C;
    for (int k = 0; k < 27; ++k) {
        const int dy = (k / 3) % 3 - 1, dz = k / 9 - 1;
        t.off[k] = (dz * g.Yp + dy) * g.Xp;
    }
    return t;
}

// P[z] = A . B^T on the tcgen05 tensor cores (lbms_umma.cu), plain operands.
lbms_status ugemm(lbms_unet* u, const bf16* A, int64_t lda, const bf16* B, int64_t ldb, int64_t M, int N, int64_t K,
                  int S) {
    if ((size_t)S * M * N > u->P_floats || M > INT32_MAX || K > INT32_MAX || lda > INT32_MAX || ldb > INT32_MAX ||
        !lbms::umma_gemm_supported(A, (int)lda, B, (int)ldb, (int)M, N, (int)K, S))
        return ufail(u, LBMS_EINVAL, "U-Net product %lld x %d x %lld (split %d) not supported", (long long)M, N,
                     (long long)K, S);
    UCK(lbms::umma_gemm_tn(A, (int)lda, B, (int)ldb, u->P, (int)M, N, (int)K, S, u->gemm_err, 0), "tensor-core gemm");
    ++u->tcgen05_calls;
    return LBMS_OK;
}

// ncopy transposed copies out[j][c][r] = in[r + j + shift0][c] over R rows (zero outside).
lbms_status transpose_rows(lbms_unet* u, const bf16* in, bf16* out, int64_t R, int C, int ncopy, int shift0,
                           size_t cap) {
    if ((size_t)ncopy * R * C > cap || R % 64 || C % 64)
        return ufail(u, LBMS_EINVAL, "U-Net transpose %lld x %d not supported", (long long)R, C);
    transpose_copies_kernel<<<dim3((unsigned)(R / 64), C / 64), 256>>>(in, out, R, C, ncopy, shift0);
    UCK(cudaGetLastError(), "transpose");
    return LBMS_OK;
}

lbms_status mask_rows(lbms_unet* u, const Geo& g, int C, float* dst) {
    if ((size_t)g.Rp * C > u->f_floats) return ufail(u, LBMS_EINVAL, "U-Net gradient %lld x %d too large",
                                                      (long long)g.Rp, C);
    mask_rows_kernel<<<warp_grid(g.Rp), 256>>>(u->P, g, C, dst);
    UCK(cudaGetLastError(), "gradient rows");
    return LBMS_OK;
}

// ------------------------------------------------------ layer passes
// relu(conv3(x) + b) -> out (kind 3: implicit GEMM), or the 1x1 head's product (left in P, out unused)
lbms_status conv_fwd(lbms_unet* u, const lbms_unet::Layer& l, const bf16* x, const Geo& g, bf16* out) {
    if (l.kind == 3) {
        // bias, ReLU, the zero halo and the BF16 store happen in the GEMM's epilogue
        const lbms::ConvTaps tp = conv_taps(g, l.ci_s / 64, 1);
        lbms::ConvEpilogue ep;
        ep.bias = l.b;
        ep.out = out;
        ep.X = g.X;
        ep.Y = g.Y;
        ep.Z = g.Z;
        ep.Xp = g.Xp;
        ep.Yp = g.Yp;
        ep.Zp = g.Zp;
        ep.R = g.R;
        if (!out) return ufail(u, LBMS_EINVAL, "U-Net convolution without an output");
        UCK(lbms::umma_conv_gemm(x, (int)g.Rp, l.ci_s, l.Wb, l.co_s, tp, u->P, u->gemm_err, 0, &ep), "convolution");
        ++u->tcgen05_calls;
        return LBMS_OK;
    }
    return ugemm(u, x, l.ci_s, l.Wb, l.K, g.Rp, l.rows, l.K, 1);   // the 1x1 head: P [Rp][64]
}

// transposed 2x2x2 convolution of x [lo.Rp][ci_s] -> y [hi.Rp][co_s]
lbms_status up_fwd(lbms_unet* u, const lbms_unet::Layer& l, const bf16* x, const Geo& lo, const Geo& hi, bf16* y) {
    UST(ugemm(u, x, l.ci_s, l.Wb, l.K, lo.Rp, l.rows, l.K, 1));
    up_rows_kernel<<<warp_grid(hi.Rp), 256>>>(u->P, l.b, lo, hi, l.co_s, y);
    UCK(cudaGetLastError(), "up convolution");
    return LBMS_OK;
}

// Backward pass of a 3x3x3 convolution + ReLU from dA (the gradient of its
// output a; it may be u->P): weight and bias gradients and, with dx, the
// input gradient [Rp][ci_s]: masked to zero outside the volumes into dx, or
// left unmasked in u->P when dx is u->P (for a ReLU backward or a pooling
// gradient next, which read only what the zero halo of their activations
// lets through).
lbms_status conv_bwd(lbms_unet* u, const lbms_unet::Layer& l, const bf16* x, const bf16* a, const float* dA,
                     const Geo& g, float* dx) {
    relu_back_rows_kernel<<<(unsigned)(g.Rp / 64), 256>>>(dA, a, g.Rp, l.co_s, u->dz, l.gb);
    UCK(cudaGetLastError(), "relu backward");
    UST(transpose_rows(u, u->dz, u->dzT, g.Rp, l.co_s, 1, 0, u->g_elems));
    UST(transpose_rows(u, x, u->xT, g.Rp, l.ci_s, 3, -1, u->xT_elems));
    const void* xT[3];
    for (int j = 0; j < 3; ++j) xT[j] = u->xT + (size_t)j * l.ci_s * g.Rp;
    if ((size_t)g.S * l.co_s * l.K > u->P_floats) return ufail(u, LBMS_EINVAL, "U-Net weight gradient too large");
    const lbms::ConvTaps tw = wgrad_taps(g, l.ci_s);
    UCK(lbms::umma_wgrad_gemm(u->dzT, l.co_s, xT, l.ci_s, (int)g.Rp, g.S, tw, u->P, u->gemm_err, 0),
        "weight gradient");
    ++u->tcgen05_calls;
    splitk_sum_t_kernel<<<grid_for((int64_t)l.co_s * l.K), 256>>>(u->P, g.S, l.K, l.co_s, l.g);
    UCK(cudaGetLastError(), "split-k sum");
    if (!dx) return LBMS_OK;
    if ((size_t)g.Rp * l.ci_s > u->P_floats) return ufail(u, LBMS_EINVAL, "U-Net input gradient too large");
    const lbms::ConvTaps tn = conv_taps(g, l.co_s / 64, -1);
    UCK(lbms::umma_conv_gemm(u->dz, (int)g.Rp, l.co_s, l.Wt, l.ci_s, tn, u->P, u->gemm_err, 0), "input gradient");
    ++u->tcgen05_calls;
    return dx == u->P ? LBMS_OK : mask_rows(u, g, l.ci_s, dx);
}

// Backward pass of the transposed convolution from dy [hi.Rp][co_s]: weight
// and bias gradients and the gradient of its input [lo.Rp][ci_s].
lbms_status up_bwd(lbms_unet* u, const lbms_unet::Layer& l, const bf16* x, const float* dy, const Geo& lo,
                   const Geo& hi, float* dx) {
    colsum_kernel<<<(unsigned)(hi.Rp / 32), 128>>>(dy, hi.Rp, l.co_s, l.gb);
    UCK(cudaGetLastError(), "bias gradient");
    if ((size_t)lo.Rp * l.rows > u->g_elems) return ufail(u, LBMS_EINVAL, "U-Net gather too large");
    upgather_rows_kernel<<<warp_grid(lo.Rp), 256>>>(dy, lo, hi, l.co_s, u->G);
    UCK(cudaGetLastError(), "up gather");
    UST(transpose_rows(u, u->G, u->dzT, lo.Rp, l.rows, 1, 0, u->g_elems));
    UST(transpose_rows(u, x, u->aT, lo.Rp, l.ci_s, 1, 0, u->g_elems));
    UST(ugemm(u, u->dzT, lo.Rp, u->aT, lo.Rp, l.rows, l.ci_s, lo.Rp, lo.S));
    splitk_sum_kernel<<<grid_for((int64_t)l.rows * l.K), 256>>>(u->P, lo.S, (int64_t)l.rows * l.K, l.g);
    UCK(cudaGetLastError(), "split-k sum");
    UST(ugemm(u, u->G, l.rows, l.Wt, l.rows, lo.Rp, l.ci_s, l.rows, 1));
    return dx == u->P ? LBMS_OK : mask_rows(u, lo, l.ci_s, dx);
}

// ------------------------------------------------------ network passes
// Forward pass of a batch already in u->x0 (layout v.g[0]); the head's
// product (without its bias) is left in u->P [Rp][64].
lbms_status unet_forward(lbms_unet* u, const Levels& v) {
    const Geo &g0 = v.g[0], &g1 = v.g[1], &g2 = v.g[2];
    const int w = u->width;
    auto& L = u->L;
    UST(conv_fwd(u, L[0], u->x0, g0, u->e1a));
    UST(conv_fwd(u, L[1], u->e1a, g0, u->e1));
    pool_rows_kernel<<<warp_grid(g1.Rp), 256>>>(u->e1, g0, g1, 64, u->p1, u->arg1);
    UCK(cudaGetLastError(), "pool");
    UST(conv_fwd(u, L[2], u->p1, g1, u->e2a));
    UST(conv_fwd(u, L[3], u->e2a, g1, u->e2));
    pool_rows_kernel<<<warp_grid(g2.Rp), 256>>>(u->e2, g1, g2, 64, u->p2, u->arg2);
    UCK(cudaGetLastError(), "pool");
    UST(conv_fwd(u, L[4], u->p2, g2, u->e3a));
    UST(conv_fwd(u, L[5], u->e3a, g2, u->e3));
    UST(up_fwd(u, L[6], u->e3, g2, g1, u->u2));
    concat_kernel<<<grid_for(g1.Rp * 128), 256>>>(u->u2, 64, 2 * w, u->e2, 64, 2 * w, g1.Rp, 128, u->c2);
    UCK(cudaGetLastError(), "concat");
    UST(conv_fwd(u, L[7], u->c2, g1, u->d2a));
    UST(conv_fwd(u, L[8], u->d2a, g1, u->d2));
    UST(up_fwd(u, L[9], u->d2, g1, g0, u->u1));
    concat_kernel<<<grid_for(g0.Rp * 64), 256>>>(u->u1, 64, w, u->e1, 64, w, g0.Rp, 64, u->c1);
    UCK(cudaGetLastError(), "concat");
    UST(conv_fwd(u, L[10], u->c1, g0, u->d1a));
    UST(conv_fwd(u, L[11], u->d1a, g0, u->d1));
    return conv_fwd(u, L[12], u->d1, g0, nullptr);
}

// Loss against u->T (targets and mask) and the backward pass through every
// layer after unet_forward; gradients in each layer's g / gb.
lbms_status unet_backward(lbms_unet* u, const Levels& v, float inv_n) {
    const Geo &g0 = v.g[0], &g1 = v.g[1], &g2 = v.g[2];
    const int w = u->width;
    auto& L = u->L;
    UCK(cudaMemsetAsync(u->loss, 0, sizeof(double), 0), "loss");
    for (auto& l : L) UCK(cudaMemsetAsync(l.gb, 0, l.co_s * sizeof(float), 0), "bias gradients");
    // head: dP, its weight gradient dP^T . d1 and the gradient of d1
    const lbms_unet::Layer& h = L[12];
    unet_loss_kernel<<<(unsigned)(g0.Rp / 64), 256>>>(u->P, h.b, u->T, g0.Rp, inv_n, u->dz, h.gb, u->loss, u->Y);
    UCK(cudaGetLastError(), "loss");
    UST(transpose_rows(u, u->dz, u->dzT, g0.Rp, kUOutC, 1, 0, u->g_elems));
    UST(transpose_rows(u, u->d1, u->aT, g0.Rp, h.ci_s, 1, 0, u->g_elems));
    UST(ugemm(u, u->dzT, g0.Rp, u->aT, g0.Rp, h.rows, h.ci_s, g0.Rp, g0.S));
    splitk_sum_kernel<<<grid_for((int64_t)h.rows * h.K), 256>>>(u->P, g0.S, (int64_t)h.rows * h.K, h.g);
    UCK(cudaGetLastError(), "split-k sum");
    UST(ugemm(u, u->dz, kUOutC, h.Wt, h.rows, g0.Rp, h.ci_s, h.rows, 1));
    // Input gradients stay in P (unmasked) when a ReLU backward or a pooling
    // gradient reads them next; the two that feed a concatenation's split
    // are masked into fa / fb (the split's halves reach bias column sums).
    float* P = u->P;
    // decoder, level 0
    UST(conv_bwd(u, L[11], u->d1a, u->d1, P, g0, P));
    UST(conv_bwd(u, L[10], u->c1, u->d1a, P, g0, u->fa));
    split_kernel<<<grid_for(g0.Rp * 64), 256>>>(u->fa, 64, w, w, 64, 64, g0.Rp, u->fb, u->fc);
    UCK(cudaGetLastError(), "split");
    UST(up_bwd(u, L[9], u->d2, u->fb, g1, g0, P));
    // decoder, level 1
    UST(conv_bwd(u, L[8], u->d2a, u->d2, P, g1, P));
    UST(conv_bwd(u, L[7], u->c2, u->d2a, P, g1, u->fb));
    split_kernel<<<grid_for(g1.Rp * 64), 256>>>(u->fb, 128, 2 * w, 2 * w, 64, 64, g1.Rp, u->fa, u->fd);
    UCK(cudaGetLastError(), "split");
    UST(up_bwd(u, L[6], u->e3, u->fa, g2, g1, P));
    // bottom, level 2
    UST(conv_bwd(u, L[5], u->e3a, u->e3, P, g2, P));
    UST(conv_bwd(u, L[4], u->p2, u->e3a, P, g2, P));
    pool_back_rows_kernel<<<warp_grid(g1.R), 256>>>(P, u->arg2, g1, g2, 64, u->fd);
    UCK(cudaGetLastError(), "pool backward");
    // encoder, level 1
    UST(conv_bwd(u, L[3], u->e2a, u->e2, u->fd, g1, P));
    UST(conv_bwd(u, L[2], u->p1, u->e2a, P, g1, P));
    pool_back_rows_kernel<<<warp_grid(g0.R), 256>>>(P, u->arg1, g0, g1, 64, u->fc);
    UCK(cudaGetLastError(), "pool backward");
    // encoder, level 0
    UST(conv_bwd(u, L[1], u->e1a, u->e1, u->fc, g0, P));
    return conv_bwd(u, L[0], u->x0, u->e1a, P, g0, nullptr);
}

// The BF16 copies of one layer's weights from its FP32 master copy.
lbms_status cast_layer(lbms_unet* u, const lbms_unet::Layer& l) {
    if (l.kind == 3)
        conv_cast_kernel<<<grid_for((int64_t)l.rows * l.K), 256>>>(l.W, l.co_s, l.ci_s, l.Wb, l.Wt);
    else
        cast_weights_kernel<<<grid_for((int64_t)l.rows * l.K), 256>>>(l.W, l.rows, l.K, l.Wb, l.Wt);
    UCK(cudaGetLastError(), "weight cast");
    return LBMS_OK;
}

// One Adam step (betas 0.9 / 0.999, eps 1e-8) on every layer.
lbms_status unet_adam(lbms_unet* u, double lr) {
    ++u->step;
    const float c1 = (float)(1.0 / (1.0 - std::pow(0.9, (double)u->step)));
    const float c2 = (float)(1.0 / (1.0 - std::pow(0.999, (double)u->step)));
    for (const auto& l : u->L) {
        const int64_t nw = (int64_t)l.rows * l.K;
        adam_kernel<<<grid_for(nw), 256>>>(l.W, l.m, l.v, l.g, nw, (float)lr, c1, c2, l.rows, l.K, nullptr, nullptr);
        adam_kernel<<<grid_for(l.co_s), 256>>>(l.b, l.mb, l.vb, l.gb, l.co_s, (float)lr, c1, c2, l.co_s, 1, nullptr,
                                               nullptr);
        UCK(cudaGetLastError(), "adam");
        UST(cast_layer(u, l));
    }
    return LBMS_OK;
}

lbms_status unet_check_gemm(lbms_unet* u) {
    unsigned int f = 0;
    UCK(cudaMemcpy(&f, u->gemm_err, sizeof(f), cudaMemcpyDeviceToHost), "GEMM flag");
    if (!f) return LBMS_OK;
    UCK(cudaMemset(u->gemm_err, 0, sizeof(f)), "GEMM flag");
    return ufail(u, LBMS_ECUDA, "tensor-core GEMM: an mbarrier wait timed out (flag %u)", f);
}

int64_t unet_params(const lbms_unet* u) {
    int64_t s = 0;
    for (const auto& l : u->L) s += (int64_t)l.co * l.ci * (l.kind == 3 ? 27 : l.kind == 2 ? 8 : 1) + l.co;
    return s;
}

// Flat index in W of the real weight number e of a layer, in PyTorch's
// order: Conv3d [co][ci][kz][ky][kx], ConvTranspose3d [ci][co][kz][ky][kx].
size_t weight_slot(const lbms_unet::Layer& l, int64_t e) {
    if (l.kind == 3) {
        const int tap = (int)(e % 27), ci = (int)((e / 27) % l.ci), co = (int)(e / (27 * (int64_t)l.ci));
        return (size_t)co * l.K + (size_t)tap * l.ci_s + ci;
    }
    if (l.kind == 2) {
        const int t = (int)(e % 8), co = (int)((e / 8) % l.co), ci = (int)(e / (8 * (int64_t)l.co));
        return (size_t)(t * l.co_s + co) * l.K + ci;
    }
    const int ci = (int)(e % l.ci), co = (int)(e / l.ci);
    return (size_t)co * l.K + ci;
}

// A case on the network's grid: interior extents rounded up to multiples
// of 4 (the added voxels solid), each fluid cell's row in the layout of one volume.
struct CaseVolume {
    Geo g;
    std::vector<int64_t> row;
};

void case_volume(const lbms::CaseView& v, CaseVolume& cv) {
    cv.g = make_geo(1, (v.nx + 3) / 4 * 4, (v.ny + 3) / 4 * 4, (v.nz + 3) / 4 * 4);
    cv.row.resize(v.nf);
    for (int j = 0; j < v.nf; ++j) {
        const int64_t e = v.fluid_cell[j];
        const int x = (int)(e % v.nx), y = (int)((e / v.nx) % v.ny), z = (int)(e / ((int64_t)v.nx * v.ny));
        cv.row[j] = (((int64_t)z + 1) * cv.g.Yp + y + 1) * cv.g.Xp + x + 1;
    }
}

}  // namespace

extern "C" {

void lbms_unet_destroy(lbms_unet* u) {
    if (!u) return;
    cudaDeviceSynchronize();
    for (void* p : u->allocs) cudaFree(p);
    for (void* p : u->bufs) cudaFree(p);
    for (auto& s : u->samples) {
        cudaFree(s.in);
        cudaFree(s.tg);
    }
    delete u;
}

lbms_status lbms_unet_create(int width, int64_t max_voxels, uint64_t seed, lbms_unet** out) {
    if (!out) return LBMS_EINVAL;
    *out = nullptr;
    if (width < 4 || width > 32 || max_voxels < 64 || max_voxels > LBMS_UNET_MAX_VOXELS) return LBMS_EINVAL;
    lbms_unet* u = new (std::nothrow) lbms_unet;
    if (!u) return LBMS_ENOMEM;
    u->width = width;
    u->seed = seed;
    u->vcap = max_voxels;
    const int w = width;
    // kind, output level, real / stored input channels, real / stored output channels
    const int spec[kULayers][6] = {{3, 0, kUInReal, kUInC, w, 64}, {3, 0, w, 64, w, 64},
                                   {3, 1, w, 64, 2 * w, 64},       {3, 1, 2 * w, 64, 2 * w, 64},
                                   {3, 2, 2 * w, 64, 4 * w, 128},  {3, 2, 4 * w, 128, 4 * w, 128},
                                   {2, 1, 4 * w, 128, 2 * w, 64},  {3, 1, 4 * w, 128, 2 * w, 64},
                                   {3, 1, 2 * w, 64, 2 * w, 64},   {2, 0, 2 * w, 64, w, 64},
                                   {3, 0, 2 * w, 64, w, 64},       {3, 0, w, 64, w, 64},
                                   {1, 0, w, 64, 3, kUOutC}};
    for (int i = 0; i < kULayers; ++i) {
        auto& l = u->L[i];
        l.kind = spec[i][0];
        l.level = spec[i][1];
        l.ci = spec[i][2];
        l.ci_s = spec[i][3];
        l.co = spec[i][4];
        l.co_s = spec[i][5];
        l.rows = l.kind == 2 ? 8 * l.co_s : l.co_s;
        l.K = l.kind == 3 ? 27 * l.ci_s : l.ci_s;
        const size_t nw = (size_t)l.rows * l.K;
        l.W = ualloc<float>(u, nw);
        l.m = ualloc<float>(u, nw);
        l.v = ualloc<float>(u, nw);
        l.g = ualloc<float>(u, nw);
        l.b = ualloc<float>(u, l.co_s);
        l.mb = ualloc<float>(u, l.co_s);
        l.vb = ualloc<float>(u, l.co_s);
        l.gb = ualloc<float>(u, l.co_s);
        l.Wb = ualloc<bf16>(u, nw);
        l.Wt = ualloc<bf16>(u, l.kind == 3 ? (size_t)l.ci_s * 27 * l.co_s : nw);
    }
    u->loss = ualloc<double>(u, 1);
    u->gemm_err = ualloc<unsigned int>(u, 1);
    bool ok = true;
    for (void* p : u->allocs) ok = ok && p;
    if (!ok) {
        lbms_unet_destroy(u);
        return LBMS_ENOMEM;
    }
    ok = lbms::umma_gemm_init() == cudaSuccess;
    ok = ok && cudaMemset(u->gemm_err, 0, sizeof(unsigned int)) == cudaSuccess;
    // He-uniform weights on the real entries (fan-in 27 ci for the 3x3x3
    // convolutions, ci for the transposed ones), zero head, zero biases
    for (int i = 0; i < kULayers && ok; ++i) {
        auto& l = u->L[i];
        const size_t nw = (size_t)l.rows * l.K;
        std::vector<float> W(nw, 0.0f);
        if (l.kind != 1) {
            const int64_t taps = l.kind == 3 ? 27 : 8;
            const double a = std::sqrt(6.0 / (double)((l.kind == 3 ? 27 : 1) * l.ci));
            const int64_t n = (int64_t)l.co * l.ci * taps;
            for (int64_t e = 0; e < n; ++e)
                W[weight_slot(l, e)] =
                    (float)(a * (2.0 * unit_double(seed * 0x100000001ull + (uint64_t)(i + 1) * 0x1000000000ull + e) - 1.0));
        }
        ok = ok && cudaMemcpy(l.W, W.data(), nw * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess;
        for (float* p : {l.m, l.v, l.g}) ok = ok && cudaMemset(p, 0, nw * sizeof(float)) == cudaSuccess;
        for (float* p : {l.b, l.mb, l.vb, l.gb}) ok = ok && cudaMemset(p, 0, l.co_s * sizeof(float)) == cudaSuccess;
        ok = ok && cast_layer(u, l) == LBMS_OK;
    }
    if (!ok || cudaDeviceSynchronize() != cudaSuccess) {
        lbms_unet_destroy(u);
        return LBMS_ECUDA;
    }
    *out = u;
    return LBMS_OK;
}

const char* lbms_unet_last_error(const lbms_unet* u) { return u ? u->msg.c_str() : ""; }

lbms_status lbms_unet_info(const lbms_unet* u, int64_t* n_params, int64_t* n_samples) {
    if (!u) return LBMS_EINVAL;
    if (n_params) *n_params = unet_params(u);
    if (n_samples) *n_samples = (int64_t)u->samples.size();
    return LBMS_OK;
}

lbms_status lbms_unet_gemm_calls(const lbms_unet* u, int64_t* tcgen05_calls) {
    if (!u) return LBMS_EINVAL;
    if (tcgen05_calls) *tcgen05_calls = u->tcgen05_calls;
    return LBMS_OK;
}

lbms_status lbms_unet_add_sample(lbms_unet* u, lbms_ctx* ctx, int k) {
    if (!u || !ctx) return LBMS_EINVAL;
    CaseFeatures F;
    lbms_status st = case_features(&u->feat, ctx, k, F);
    if (st != LBMS_OK) return ufail(u, st, "%s", u->feat.err.c_str());
    lbms::CaseView v;
    lbms::case_view(ctx, k, &v);
    CaseVolume cv;
    case_volume(v, cv);
    if (cv.g.V > u->vcap || !levels_fit(levels_of(1, cv.g.X, cv.g.Y, cv.g.Z)))
        return ufail(u, LBMS_EINVAL, "case %d needs %lld voxels, the network was made for %lld", k, (long long)cv.g.V,
                     (long long)u->vcap);
    std::vector<double> X((size_t)3 * v.N);
    st = lbms_batch_get_fields(ctx, k, X.data(), nullptr, nullptr);
    if (st != LBMS_OK) return ufail(u, st, "reading the fields of case %d: %s", k, lbms_last_error(ctx));
    const int64_t R = cv.g.R;
    std::vector<float> t((size_t)R * 4, 0.0f);
    for (int j = 0; j < v.nf; ++j) {
        const int64_t e = v.fluid_cell[j];
        const int x = (int)(e % v.nx);
        float* r = &t[(size_t)cv.row[j] * 4];
        for (int s = 0; s < 3; ++s) r[s] = (float)(kTargetScale * (X[(size_t)s * v.N + e] - F.prof[(size_t)s * v.nx + x]));
        r[3] = 1.0f;
    }
    lbms_unet::Sample s;
    s.X = cv.g.X;
    s.Y = cv.g.Y;
    s.Z = cv.g.Z;
    s.rows = R;
    s.nfluid = v.nf;
    int64_t* prow = F.alloc<int64_t>(v.nf);
    if (!prow) return ufail(u, LBMS_ENOMEM, "cell rows");
    if (cudaMalloc(&s.in, (size_t)R * kUInC * sizeof(bf16)) != cudaSuccess) return ufail(u, LBMS_ENOMEM, "sample");
    if (cudaMalloc(&s.tg, (size_t)R * 4 * sizeof(float)) != cudaSuccess) {
        cudaFree(s.in);
        return ufail(u, LBMS_ENOMEM, "sample");
    }
    cudaError_t e = cudaMemcpy(prow, cv.row.data(), v.nf * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(s.in, 0, (size_t)R * kUInC * sizeof(bf16));
    if (e == cudaSuccess) {
        unet_inputs_kernel<<<grid_for((int64_t)v.nf * kUInC), 256>>>(F.rows, prow, v.nf, s.in);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(s.tg, t.data(), t.size() * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaFree(s.in);
        cudaFree(s.tg);
        return ufail(u, LBMS_ECUDA, "sample: %s", cudaGetErrorString(e));
    }
    u->samples.push_back(s);   // owned from here on (freed by destroy)
    return LBMS_OK;
}

lbms_status lbms_unet_add_volume(lbms_unet* u, const float* x, const float* t, int X, int Y, int Z) {
    if (!u || !x || !t) return LBMS_EINVAL;
    if (X < 4 || Y < 4 || Z < 4 || X % 4 || Y % 4 || Z % 4)
        return ufail(u, LBMS_EINVAL, "volume extents must be multiples of 4");
    const Geo g = make_geo(1, X, Y, Z);
    if (g.V > u->vcap || !levels_fit(levels_of(1, X, Y, Z)))
        return ufail(u, LBMS_EINVAL, "the volume holds %lld voxels, the network was made for %lld", (long long)g.V,
                     (long long)u->vcap);
    double nf = 0.0;
    for (int64_t s = 0; s < g.V; ++s) nf += x[(int64_t)(kUInReal - 1) * g.V + s];
    lbms_unet::Sample s;
    s.X = X;
    s.Y = Y;
    s.Z = Z;
    s.rows = g.R;
    s.nfluid = (int64_t)std::llround(nf);
    float* dev = nullptr;
    const size_t nin = (size_t)g.V * kUInReal, ntg = (size_t)g.V * 3;
    if (cudaMalloc(&dev, (nin + ntg) * sizeof(float)) != cudaSuccess) return ufail(u, LBMS_ENOMEM, "volume upload");
    cudaError_t e = cudaMalloc(&s.in, (size_t)g.R * kUInC * sizeof(bf16));
    if (e == cudaSuccess) e = cudaMalloc(&s.tg, (size_t)g.R * 4 * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(dev, x, nin * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dev + nin, t, ntg * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(s.in, 0, (size_t)g.R * kUInC * sizeof(bf16));
    if (e == cudaSuccess) e = cudaMemset(s.tg, 0, (size_t)g.R * 4 * sizeof(float));
    if (e == cudaSuccess) {
        vol_in_kernel<<<warp_grid(g.V), 256>>>(dev, g, s.in, s.tg);
        vol_target_kernel<<<grid_for(g.V), 256>>>(dev + nin, g, s.tg);
        e = cudaDeviceSynchronize();
    }
    cudaFree(dev);
    if (e != cudaSuccess) {
        cudaFree(s.in);
        cudaFree(s.tg);
        return ufail(u, LBMS_ECUDA, "volume upload: %s", cudaGetErrorString(e));
    }
    u->samples.push_back(s);
    return LBMS_OK;
}

lbms_status lbms_unet_train(lbms_unet* u, int iters, int max_batch, double lr, double* last_loss) {
    if (!u) return LBMS_EINVAL;
    if (iters < 0 || max_batch < 1 || !(lr > 0.0))
        return ufail(u, LBMS_EINVAL, "need iters >= 0, max_batch >= 1, lr > 0");
    if (u->samples.empty()) return ufail(u, LBMS_ESTATE, "no training volumes (call lbms_unet_add_sample first)");
    // groups of equal volume extents, in order of first appearance, and the batch size of each
    std::vector<std::vector<int>> groups;
    for (int i = 0; i < (int)u->samples.size(); ++i) {
        const auto& s = u->samples[i];
        bool placed = false;
        for (auto& g : groups) {
            const auto& f = u->samples[g[0]];
            if (f.X == s.X && f.Y == s.Y && f.Z == s.Z) {
                g.push_back(i);
                placed = true;
                break;
            }
        }
        if (!placed) groups.push_back({i});
    }
    std::vector<int> Bg(groups.size());
    for (size_t gi = 0; gi < groups.size(); ++gi) {
        const auto& s0 = u->samples[groups[gi][0]];
        const int64_t Vs = (int64_t)s0.X * s0.Y * s0.Z;
        int B = (int)std::min<int64_t>({(int64_t)max_batch, (int64_t)groups[gi].size(), u->vcap / Vs});
        while (B > 1 && !levels_fit(levels_of(B, s0.X, s0.Y, s0.Z))) --B;
        Bg[gi] = B;
        UST(ensure_buffers(u, levels_of(B, s0.X, s0.Y, s0.Z)));
    }
    double tail = 0.0;
    int nt = 0;
    for (int it = 0; it < iters; ++it) {
        const size_t gi = it % groups.size();
        const auto& g = groups[gi];
        const auto& s0 = u->samples[g[0]];
        const int B = Bg[gi];
        const Levels lv = levels_of(B, s0.X, s0.Y, s0.Z);
        const uint64_t key = splitmix64(u->seed ^ 0x5A5A5A5Aull) + (uint64_t)u->step * 64ull;
        int64_t nfl = 0;
        for (int i = 0; i < B; ++i) {
            const auto& s = u->samples[g[splitmix64(key + (uint64_t)i) % g.size()]];
            UCK(cudaMemcpyAsync(u->x0 + i * s.rows * kUInC, s.in, s.rows * kUInC * sizeof(bf16),
                                cudaMemcpyDeviceToDevice, 0),
                "batch");
            UCK(cudaMemcpyAsync(u->T + i * s.rows * 4, s.tg, s.rows * 4 * sizeof(float), cudaMemcpyDeviceToDevice, 0),
                "batch");
            nfl += s.nfluid;
        }
        const Geo& g0 = lv.g[0];
        UCK(cudaMemsetAsync(u->x0 + g0.R * kUInC, 0, (g0.Rp - g0.R) * kUInC * sizeof(bf16), 0), "batch");
        UCK(cudaMemsetAsync(u->T + g0.R * 4, 0, (g0.Rp - g0.R) * 4 * sizeof(float), 0), "batch");
        const double cw = 0.5 * (1.0 + std::cos(3.14159265358979323846 * (double)it / std::max(1, iters)));
        const double lr_it = lr / 20.0 + (lr - lr / 20.0) * cw;
        UST(unet_forward(u, lv));
        UST(unet_backward(u, lv, (float)(1.0 / (3.0 * (double)std::max<int64_t>(nfl, 1)))));
        UST(unet_adam(u, lr_it));
        if (it >= iters - 10) {
            double l = 0.0;
            UCK(cudaMemcpy(&l, u->loss, sizeof(double), cudaMemcpyDeviceToHost), "read loss");
            tail += l;
            ++nt;
        }
    }
    UCK(cudaDeviceSynchronize(), "train");
    UST(unet_check_gemm(u));
    if (last_loss) *last_loss = nt ? tail / nt : 0.0;
    return LBMS_OK;
}

lbms_status lbms_unet_warm_start(lbms_unet* u, lbms_ctx* ctx, int k, double* Xout) {
    if (!u || !ctx) return LBMS_EINVAL;
    CaseFeatures F;
    lbms_status st = case_features(&u->feat, ctx, k, F);
    if (st != LBMS_OK) return ufail(u, st, "%s", u->feat.err.c_str());
    lbms::CaseView v;
    lbms::case_view(ctx, k, &v);
    CaseVolume cv;
    case_volume(v, cv);
    const Levels lv = levels_of(1, cv.g.X, cv.g.Y, cv.g.Z);
    if (cv.g.V > u->vcap || !levels_fit(lv))
        return ufail(u, LBMS_EINVAL, "case %d needs %lld voxels, the network was made for %lld", k, (long long)cv.g.V,
                     (long long)u->vcap);
    UST(ensure_buffers(u, lv));
    int64_t* prow = F.alloc<int64_t>(v.nf);
    double* dX = F.alloc<double>((size_t)3 * v.nf);
    if (!prow || !dX) return ufail(u, LBMS_ENOMEM, "prediction buffers");
    const Geo& g0 = lv.g[0];
    UCK(cudaMemcpy(prow, cv.row.data(), v.nf * sizeof(int64_t), cudaMemcpyHostToDevice), "cells");
    UCK(cudaMemset(u->x0, 0, (size_t)g0.Rp * kUInC * sizeof(bf16)), "inputs");
    unet_inputs_kernel<<<grid_for((int64_t)v.nf * kUInC), 256>>>(F.rows, prow, v.nf, u->x0);
    UCK(cudaGetLastError(), "inputs");
    UST(unet_forward(u, lv));
    unet_loss_kernel<<<(unsigned)(g0.Rp / 64), 256>>>(u->P, u->L[kULayers - 1].b, nullptr, g0.Rp, 0.0f, nullptr,
                                                      nullptr, nullptr, u->Y);
    UCK(cudaGetLastError(), "head");
    unet_post_kernel<<<(v.nf + 255) / 256, 256>>>(u->Y, prow, v.nf, g0.Xp, F.xtab, dX);
    UCK(cudaGetLastError(), "prediction");
    std::vector<double> c((size_t)3 * v.nf);
    UCK(cudaMemcpy(c.data(), dX, c.size() * sizeof(double), cudaMemcpyDeviceToHost), "read prediction");
    UST(unet_check_gemm(u));
    std::vector<double> X((size_t)3 * v.N, 0.0);
    for (int s = 0; s < 3; ++s)
        for (int j = 0; j < v.nf; ++j) X[(size_t)s * v.N + v.fluid_cell[j]] = c[(size_t)s * v.nf + j];
    st = lbms_batch_set_fields(ctx, k, X.data());
    if (st != LBMS_OK) return ufail(u, st, "restarting case %d: %s", k, lbms_last_error(ctx));
    if (Xout) std::copy(X.begin(), X.end(), Xout);
    return LBMS_OK;
}

}  // extern "C"

namespace {

// Uploads a host batch FP32 [B][17][Z][Y][X] (and targets [B][3][Z][Y][X])
// into x0 and T in the layout of `lv`; nfluid receives the mask's sum.
lbms_status upload_batch(lbms_unet* u, const float* x, const float* t, int B, int X, int Y, int Z, Levels* lv,
                         double* nfluid) {
    if (!x || B < 1 || X < 4 || Y < 4 || Z < 4 || X % 4 || Y % 4 || Z % 4)
        return ufail(u, LBMS_EINVAL, "need B >= 1 volumes with extents multiples of 4");
    *lv = levels_of(B, X, Y, Z);
    const Geo& g0 = lv->g[0];
    if (g0.V > u->vcap || !levels_fit(*lv))
        return ufail(u, LBMS_EINVAL, "the batch holds %lld voxels, the network was made for %lld", (long long)g0.V,
                     (long long)u->vcap);
    UST(ensure_buffers(u, *lv));
    const int64_t S = (int64_t)X * Y * Z, V = g0.V;
    double nf = 0.0;
    for (int b = 0; b < B; ++b)
        for (int64_t s = 0; s < S; ++s) nf += x[((int64_t)b * kUInReal + kUInReal - 1) * S + s];
    if (nfluid) *nfluid = nf;
    float* dev = nullptr;
    const size_t nin = (size_t)V * kUInReal, ntg = t ? (size_t)V * 3 : 0;
    UCK(cudaMalloc(&dev, (nin + ntg) * sizeof(float)), "batch upload");
    lbms_status st = LBMS_OK;
    cudaError_t e = cudaMemcpy(dev, x, nin * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && t) e = cudaMemcpy(dev + nin, t, ntg * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(u->x0, 0, (size_t)g0.Rp * kUInC * sizeof(bf16));
    if (e == cudaSuccess) e = cudaMemset(u->T, 0, (size_t)g0.Rp * 4 * sizeof(float));
    if (e == cudaSuccess) {
        vol_in_kernel<<<warp_grid(V), 256>>>(dev, g0, u->x0, u->T);
        if (t) vol_target_kernel<<<grid_for(V), 256>>>(dev + nin, g0, u->T);
        e = cudaDeviceSynchronize();
    }
    if (e != cudaSuccess) st = ufail(u, LBMS_ECUDA, "batch upload: %s", cudaGetErrorString(e));
    cudaFree(dev);
    return st;
}

}  // namespace

extern "C" {

lbms_status lbms_unet_forward(lbms_unet* u, const float* x, int B, int X, int Y, int Z, float* y) {
    if (!u || !y) return LBMS_EINVAL;
    Levels lv;
    UST(upload_batch(u, x, nullptr, B, X, Y, Z, &lv, nullptr));
    UST(unet_forward(u, lv));
    const Geo& g0 = lv.g[0];
    unet_loss_kernel<<<(unsigned)(g0.Rp / 64), 256>>>(u->P, u->L[kULayers - 1].b, nullptr, g0.Rp, 0.0f, nullptr,
                                                      nullptr, nullptr, u->Y);
    UCK(cudaGetLastError(), "head");
    std::vector<float> h((size_t)g0.R * 4);
    UCK(cudaMemcpy(h.data(), u->Y, h.size() * sizeof(float), cudaMemcpyDeviceToHost), "read output");
    UST(unet_check_gemm(u));
    const int64_t S = (int64_t)X * Y * Z;
    for (int b = 0; b < B; ++b)
        for (int z = 0; z < Z; ++z)
            for (int yy = 0; yy < Y; ++yy)
                for (int xx = 0; xx < X; ++xx) {
                    const int64_t r = (((int64_t)b * g0.Zp + z + 1) * g0.Yp + yy + 1) * g0.Xp + xx + 1;
                    const int64_t s = ((int64_t)z * Y + yy) * X + xx;
                    for (int c = 0; c < 3; ++c) y[((int64_t)b * 3 + c) * S + s] = h[(size_t)r * 4 + c];
                }
    return LBMS_OK;
}

lbms_status lbms_unet_train_batch(lbms_unet* u, const float* x, const float* t, int B, int X, int Y, int Z, double lr,
                                  double* loss) {
    if (!u || !t || !(lr >= 0.0)) return LBMS_EINVAL;
    double nf = 0.0;
    Levels lv;
    UST(upload_batch(u, x, t, B, X, Y, Z, &lv, &nf));
    UST(unet_forward(u, lv));
    UST(unet_backward(u, lv, (float)(1.0 / (3.0 * std::max(nf, 1.0)))));
    if (lr > 0.0) UST(unet_adam(u, lr));
    if (loss) UCK(cudaMemcpy(loss, u->loss, sizeof(double), cudaMemcpyDeviceToHost), "read loss");
    UCK(cudaDeviceSynchronize(), "train batch");
    return unet_check_gemm(u);
}

lbms_status lbms_unet_get(const lbms_unet* cu, int what, float* buf, int64_t count) {
    lbms_unet* u = const_cast<lbms_unet*>(cu);
    if (!u || !buf || (what != 0 && what != 1)) return LBMS_EINVAL;
    if (count < unet_params(u))
        return ufail(u, LBMS_EINVAL, "buffer holds %lld floats, need %lld", (long long)count, (long long)unet_params(u));
    int64_t off = 0;
    for (const auto& l : u->L) {
        const size_t nw = (size_t)l.rows * l.K;
        std::vector<float> W(nw), b(l.co_s);
        UCK(cudaMemcpy(W.data(), what ? l.g : l.W, nw * sizeof(float), cudaMemcpyDeviceToHost), "get");
        UCK(cudaMemcpy(b.data(), what ? l.gb : l.b, l.co_s * sizeof(float), cudaMemcpyDeviceToHost), "get");
        const int64_t n = (int64_t)l.co * l.ci * (l.kind == 3 ? 27 : l.kind == 2 ? 8 : 1);
        for (int64_t e = 0; e < n; ++e) buf[off + e] = W[weight_slot(l, e)];
        off += n;
        for (int c = 0; c < l.co; ++c) buf[off + c] = b[c];
        off += l.co;
    }
    return LBMS_OK;
}

lbms_status lbms_unet_set(lbms_unet* u, const float* buf, int64_t count) {
    if (!u || !buf) return LBMS_EINVAL;
    if (count < unet_params(u))
        return ufail(u, LBMS_EINVAL, "buffer holds %lld floats, need %lld", (long long)count, (long long)unet_params(u));
    int64_t off = 0;
    for (const auto& l : u->L) {
        const size_t nw = (size_t)l.rows * l.K;
        std::vector<float> W(nw, 0.0f), b(l.co_s, 0.0f);
        const int64_t n = (int64_t)l.co * l.ci * (l.kind == 3 ? 27 : l.kind == 2 ? 8 : 1);
        for (int64_t e = 0; e < n; ++e) W[weight_slot(l, e)] = buf[off + e];
        off += n;
        for (int c = 0; c < l.co; ++c) b[c] = buf[off + c];
        off += l.co;
        UCK(cudaMemcpy(l.W, W.data(), nw * sizeof(float), cudaMemcpyHostToDevice), "set");
        UCK(cudaMemcpy(l.b, b.data(), l.co_s * sizeof(float), cudaMemcpyHostToDevice), "set");
        UST(cast_layer(u, l));
    }
    UCK(cudaDeviceSynchronize(), "set");
    return LBMS_OK;
}

}  // extern "C"
