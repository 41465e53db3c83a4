// The convolutional warm start (declared in include/lbms_net.h): a 3-D U-Net
// over the anode's voxels, trained and run with this file's kernels and the
// tcgen05 GEMM of lbms_umma.cu.  Included at the end of lbms_net.cu, whose
// feature builder, bias/ReLU, ReLU-backward, split-K sum and Adam kernels it
// shares.
//
// Activations are channels-last BF16, [voxel][C] with voxels in (volume, z,
// y, x) order and C stored as a multiple of 32 (the real channels first,
// zeros after); a level's voxel count is padded to a multiple of 64 with
// rows that hold no voxel (their gradients are zero by construction).  A
// 3x3x3 convolution with zero padding is an im2col into cols[v][tap * C + c]
// (taps z-major over {-1, 0, 1}^3, K padded to a multiple of 64) and one
// product P = cols . W^T.  Its backward pass is two more products: the
// weight gradient cols^T . dZ from an im2col written in transposed order,
// and the input gradient as a convolution of dZ with the flipped weights
// (an im2col at the reflected offsets).  The 2x2x2 transposed convolution
// of the decoder is one product whose 8 C columns scatter to the 8 children
// of each voxel; max pooling keeps the index of the maximum.
namespace {

constexpr int kUInC = 32;      // stored input channels: the 16 feature columns, the fluid mask, zeros
constexpr int kUInReal = 17;
constexpr int kUOutC = 64;     // stored output channels of the 1x1 head (3 used)
constexpr int kULayers = 13;

__device__ __forceinline__ void vox_coords(int64_t v, int X, int Y, int Z, int& x, int& y, int& z, int64_t& b) {
    x = (int)(v % X);
    y = (int)((v / X) % Y);
    z = (int)((v / ((int64_t)X * Y)) % Z);
    b = v / ((int64_t)X * Y * Z);
}

// cols[v][tap * C + c] = x[v + sign (dz, dy, dx)][c] for the Vr voxels
// (zero outside the volume), cols[v][k] = 0 for 27 C <= k < Kp and for the
// padding rows Vr <= v < Vp; C a multiple of 8, 16-byte chunks.  One warp
// per voxel (its coordinates found once), lanes over the row's chunks.
__global__ void im2col3_kernel(const bf16* __restrict__ x, int64_t Vr, int64_t Vp, int X, int Y, int Z, int C,
                               int Kp, int sign, bf16* __restrict__ cols) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int q8 = Kp / 8, live = 27 * C;
    for (int64_t v = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); v < Vp; v += nwarps) {
        int x0 = 0, y0 = 0, z0 = 0;
        int64_t b = 0;
        if (v < Vr) vox_coords(v, X, Y, Z, x0, y0, z0, b);
        const int64_t vbase = ((b * Z + z0) * Y + y0) * X + x0;
        uint4* row = reinterpret_cast<uint4*>(cols + v * Kp);
        for (int qi = lane; qi < q8; qi += 32) {
            const int q = qi * 8;
            uint4 val = make_uint4(0u, 0u, 0u, 0u);
            if (v < Vr && q < live) {
                const int tap = q / C, c = q - tap * C;
                const int dx = sign * (tap % 3 - 1), dy = sign * ((tap / 3) % 3 - 1), dz = sign * (tap / 9 - 1);
                const int xs = x0 + dx, ys = y0 + dy, zs = z0 + dz;
                if (xs >= 0 && xs < X && ys >= 0 && ys < Y && zs >= 0 && zs < Z)
                    val = *reinterpret_cast<const uint4*>(x + (vbase + ((int64_t)dz * Y + dy) * X + dx) * C + c);
            }
            row[qi] = val;
        }
    }
}

// The same columns in transposed order, colsT[k][v] (Vp a multiple of 32,
// C a multiple of 32 so that 32 consecutive k share one tap): per block 32
// voxels (coordinates found once, in shared memory) and every 32-wide k
// chunk in turn, each through a 32 x 32 tile; 32 x 8 threads.
__global__ void im2col3_t_kernel(const bf16* __restrict__ x, int64_t Vr, int64_t Vp, int X, int Y, int Z, int C,
                                 int Kp, bf16* __restrict__ colsT) {
    __shared__ bf16 tile[32][33];
    __shared__ int64_t s_base[32];
    __shared__ int s_xyz[32][3];
    const int64_t v0 = (int64_t)blockIdx.x * 32;
    const int tid = threadIdx.y * 32 + threadIdx.x;
    if (tid < 32) {
        const int64_t v = v0 + tid;
        int x0 = -8, y0 = -8, z0 = -8;     // far outside: every tap of a padding row reads zero
        int64_t b = 0;
        if (v < Vr) vox_coords(v, X, Y, Z, x0, y0, z0, b);
        s_base[tid] = ((b * Z + z0) * Y + y0) * X + x0;
        s_xyz[tid][0] = x0;
        s_xyz[tid][1] = y0;
        s_xyz[tid][2] = z0;
    }
    __syncthreads();
    const int live = 27 * C;
    for (int k0 = 0; k0 < Kp; k0 += 32) {
        const int tap = k0 < live ? k0 / C : 0, c0 = k0 < live ? k0 - tap * C : 0;
        const int dx = tap % 3 - 1, dy = (tap / 3) % 3 - 1, dz = tap / 9 - 1;
        const int64_t off = ((int64_t)dz * Y + dy) * X + dx;
        for (int r = threadIdx.y; r < 32; r += 8) {
            bf16 val = __float2bfloat16_rn(0.0f);
            const int xs = s_xyz[r][0] + dx, ys = s_xyz[r][1] + dy, zs = s_xyz[r][2] + dz;
            if (k0 < live && xs >= 0 && xs < X && ys >= 0 && ys < Y && zs >= 0 && zs < Z)
                val = x[(s_base[r] + off) * C + c0 + threadIdx.x];
            tile[r][threadIdx.x] = val;
        }
        __syncthreads();
        for (int r = threadIdx.y; r < 32; r += 8) colsT[(int64_t)(k0 + r) * Vp + v0 + threadIdx.x] = tile[threadIdx.x][r];
        __syncthreads();
    }
}

// out[c][r] = in[r][c]; R and C multiples of 32, rows on grid x (R may pass 2^21).
__global__ void utranspose_kernel(const bf16* __restrict__ in, bf16* __restrict__ out, int64_t R, int C) {
    __shared__ bf16 tile[32][33];
    const int64_t r0 = (int64_t)blockIdx.x * 32;
    const int c0 = blockIdx.y * 32;
    for (int y = threadIdx.y; y < 32; y += 8) tile[y][threadIdx.x] = in[(r0 + y) * C + c0 + threadIdx.x];
    __syncthreads();
    for (int y = threadIdx.y; y < 32; y += 8) out[(int64_t)(c0 + y) * R + r0 + threadIdx.x] = tile[threadIdx.x][y];
}

// BF16 copies of a 3x3x3 convolution's FP32 weights W [co_s][Kp] (entry
// (co, tap * ci_s + ci)): Wb, the same layout, and Wf [ci_s][Kq], the
// flipped weights of the input gradient, entry (ci, tap * co_s + co).
__global__ void conv_cast_kernel(const float* __restrict__ W, int co_s, int ci_s, int Kp, int Kq,
                                 bf16* __restrict__ Wb, bf16* __restrict__ Wf) {
    const int64_t n = (int64_t)co_s * Kp;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int co = (int)(e / Kp), k = (int)(e % Kp);
        const bf16 wb = __float2bfloat16_rn(W[e]);
        Wb[e] = wb;
        if (k < 27 * ci_s) {
            const int tap = k / ci_s, ci = k % ci_s;
            Wf[(int64_t)ci * Kq + tap * co_s + co] = wb;
        }
    }
}

// G[o][i] = sum_z P[z][i][o] (the split-K partials of a transposed product).
__global__ void splitk_sum_t_kernel(const float* __restrict__ P, int S, int I, int O, float* __restrict__ G) {
    const int64_t n = (int64_t)O * I;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int o = (int)(e / I), i = (int)(e % I);
        float s = 0.0f;
        for (int z = 0; z < S; ++z) s += P[(int64_t)z * n + (int64_t)i * O + o];
        G[e] = s;
    }
}

// 2x2x2 max pooling of [V][C] at (X, Y, Z) to half size (Vlow voxels);
// arg holds the child (dz * 4 + dy * 2 + dx) of the first maximum.
__global__ void pool_fwd_kernel(const bf16* __restrict__ x, int64_t Vlow, int X, int Y, int Z, int C,
                                bf16* __restrict__ y, uint8_t* __restrict__ arg) {
    const int Xl = X / 2, Yl = Y / 2, Zl = Z / 2;
    const int64_t n = Vlow * C;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = e / C;
        const int c = (int)(e % C);
        int xl, yl, zl;
        int64_t b;
        vox_coords(v, Xl, Yl, Zl, xl, yl, zl, b);
        float best = -3.0e38f;
        int bi = 0;
        for (int t = 0; t < 8; ++t) {
            const int64_t w = ((b * Z + 2 * zl + (t >> 2)) * Y + 2 * yl + ((t >> 1) & 1)) * X + 2 * xl + (t & 1);
            const float val = __bfloat162float(x[w * C + c]);
            if (val > best) {
                best = val;
                bi = t;
            }
        }
        y[e] = __float2bfloat16_rn(best);
        arg[e] = (uint8_t)bi;
    }
}

// dx[u][c] += dp[parent(u)][c] where u is the maximum's child (the V voxels
// of the finer level; its padding rows are left as they are).
__global__ void pool_bwd_kernel(const float* __restrict__ dp, const uint8_t* __restrict__ arg, int64_t V, int X, int Y,
                                int Z, int C, float* __restrict__ dx) {
    const int64_t n = V * C;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t u = e / C;
        const int c = (int)(e % C);
        int x0, y0, z0;
        int64_t b;
        vox_coords(u, X, Y, Z, x0, y0, z0, b);
        const int64_t p = ((b * (Z / 2) + z0 / 2) * (Y / 2) + y0 / 2) * (X / 2) + x0 / 2;
        const int t = (z0 & 1) * 4 + (y0 & 1) * 2 + (x0 & 1);
        if (arg[p * C + c] == t) dx[e] += dp[p * C + c];
    }
}

// Transposed 2x2x2 convolution, stride 2: y[child(v, t)][c] = P[v][t * C + c] + b[c]
// for the Vlow voxels of the coarser level.
__global__ void upscatter_kernel(const float* __restrict__ P, const float* __restrict__ bias, int64_t Vlow, int Xl,
                                 int Yl, int Zl, int C, bf16* __restrict__ y) {
    const int64_t n = Vlow * 8 * C;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = e / (8 * C);
        const int r = (int)(e % (8 * C));
        const int t = r / C, c = r % C;
        int xl, yl, zl;
        int64_t b;
        vox_coords(v, Xl, Yl, Zl, xl, yl, zl, b);
        const int64_t w = ((b * 2 * Zl + 2 * zl + (t >> 2)) * 2 * Yl + 2 * yl + ((t >> 1) & 1)) * 2 * Xl + 2 * xl + (t & 1);
        y[w * C + c] = __float2bfloat16_rn(P[e] + bias[c]);
    }
}

// G[v][t * C + c] = dy[child(v, t)][c] (BF16), the gradient of the scatter;
// zero in the padding rows Vlow <= v < Vlp.
__global__ void upgather_kernel(const float* __restrict__ dy, int64_t Vlow, int64_t Vlp, int Xl, int Yl, int Zl, int C,
                                bf16* __restrict__ G) {
    const int64_t n = Vlp * 8 * C;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = e / (8 * C);
        float g = 0.0f;
        if (v < Vlow) {
            const int r = (int)(e % (8 * C));
            const int t = r / C, c = r % C;
            int xl, yl, zl;
            int64_t b;
            vox_coords(v, Xl, Yl, Zl, xl, yl, zl, b);
            const int64_t w =
                ((b * 2 * Zl + 2 * zl + (t >> 2)) * 2 * Yl + 2 * yl + ((t >> 1) & 1)) * 2 * Xl + 2 * xl + (t & 1);
            g = dy[w * C + c];
        }
        G[e] = __float2bfloat16_rn(g);
    }
}

// out[v] = (a[v][0:na], b[v][0:nb], zeros) with Co stored channels.
__global__ void concat_kernel(const bf16* __restrict__ a, int Ca, int na, const bf16* __restrict__ bsrc, int Cb, int nb,
                              int64_t V, int Co, bf16* __restrict__ out) {
    const int64_t n = V * Co;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = e / Co;
        const int c = (int)(e % Co);
        out[e] = c < na ? a[v * Ca + c] : c < na + nb ? bsrc[v * Cb + (c - na)] : __float2bfloat16_rn(0.0f);
    }
}

// The gradient of concat_kernel: da[v][c] = d[v][c] (c < na, else 0) and
// db[v][c] = d[v][na + c] (c < nb, else 0), with d stored Cd wide.
__global__ void split_kernel(const float* __restrict__ d, int Cd, int na, int nb, int Ca, int Cb, int64_t V,
                             float* __restrict__ da, float* __restrict__ db) {
    const int Cm = Ca > Cb ? Ca : Cb;
    const int64_t n = V * Cm;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = e / Cm;
        const int c = (int)(e % Cm);
        if (c < Ca) da[v * Ca + c] = c < na ? d[v * Cd + c] : 0.0f;
        if (c < Cb) db[v * Cb + c] = c < nb ? d[v * Cd + na + c] : 0.0f;
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

// A batch given as FP32 [B][17][S] (S voxels a volume, channel 16 the fluid
// mask) into the input rows x0 [V][32] (BF16) and the mask column of T [V][4].
__global__ void vol_in_kernel(const float* __restrict__ in, int64_t V, int64_t S, bf16* __restrict__ x0,
                              float* __restrict__ T) {
    const int64_t n = V * kUInC;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = e / kUInC;
        const int c = (int)(e % kUInC);
        const int64_t b = v / S, s = v % S;
        const float val = c < kUInReal ? in[(b * kUInReal + c) * S + s] : 0.0f;
        x0[e] = __float2bfloat16_rn(val);
        if (c == kUInReal - 1) T[v * 4 + 3] = val;
    }
}

// Targets given as FP32 [B][3][S] into T[v][0:3].
__global__ void vol_target_kernel(const float* __restrict__ t, int64_t V, int64_t S, float* __restrict__ T) {
    const int64_t n = V * 3;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t v = e / 3;
        const int c = (int)(e % 3);
        T[v * 4 + c] = t[((v / S) * 3 + c) * S + v % S];
    }
}

// Input volume of one case: vol[cell[j]][c] = rows[j][c] (c < 16), the
// fluid mask in channel 16; solid voxels stay zero (cleared before).
__global__ void unet_inputs_kernel(const bf16* __restrict__ rows, const int64_t* __restrict__ cell, int nf,
                                   bf16* __restrict__ vol) {
    const int64_t n = (int64_t)nf * kUInC;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(e / kUInC), c = (int)(e % kUInC);
        bf16 val = __float2bfloat16_rn(0.0f);
        if (c < kFUsed) val = rows[(int64_t)j * kF + c];
        else if (c == kFUsed) val = __float2bfloat16_rn(1.0f);
        vol[cell[j] * kUInC + c] = val;
    }
}

// Masked mean-square error of the head's output Y = P + b (3 used columns)
// against T [v][4] = (3 targets, fluid mask), over the V (padded) rows,
// one block of 256 threads per 64 rows: dP (BF16, zero in the padded
// columns), the head's bias gradient and the loss, with inv_n = 1 / (3 x
// fluid voxels); Y[v][c] (c < 3) is kept for predictions.
__global__ void unet_loss_kernel(const float* __restrict__ P, const float* __restrict__ b, const float* __restrict__ T,
                                 int64_t V, float inv_n, bf16* __restrict__ dP, float* __restrict__ gb,
                                 double* __restrict__ loss, float* __restrict__ Y) {
    __shared__ float colsum[3];
    __shared__ double lsum[256];
    if (threadIdx.x < 3) colsum[threadIdx.x] = 0.0f;
    __syncthreads();
    double l = 0.0;
    const int64_t v0 = (int64_t)blockIdx.x * 64;
    for (int e = threadIdx.x; e < 64 * kUOutC; e += 256) {
        const int64_t v = v0 + e / kUOutC;
        const int c = e % kUOutC;
        float g = 0.0f;
        if (v < V && c < 3) {
            const float y = P[v * kUOutC + c] + b[c];
            if (Y) Y[v * 4 + c] = y;
            if (T) {
                const float d = (y - T[v * 4 + c]) * T[v * 4 + 3];
                l += (double)d * d;
                g = 2.0f * inv_n * d;
                atomicAdd(&colsum[c], g);
            }
        }
        if (v < V && dP) dP[v * kUOutC + c] = __float2bfloat16_rn(g);
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

// The prediction of one case from the head's output Y [v][4] at the padded
// voxel cell[j]: X_s = profile_s(x) + Y[cell][s] / 100, clamped at 1e-6 and
// renormalised; out [3][nf] FP64.  Xp is the padded volume's x extent.
__global__ void unet_post_kernel(const float* __restrict__ Y, const int64_t* __restrict__ cell, int nf, int Xp,
                                 const float* __restrict__ xtab, double* __restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nf) return;
    const int64_t v = cell[j];
    const int x = (int)(v % Xp);
    double X[3], s = 0.0;
    for (int q = 0; q < 3; ++q) {
        double val = (double)xtab[(int64_t)x * 8 + q] + (double)Y[v * 4 + q] / kTargetScale;
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
        int Kq = 0;              // kind 3: width of the flipped weights [ci_s][Kq]
        float *W = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;
        float *b = nullptr, *mb = nullptr, *vb = nullptr, *gb = nullptr;   // [co_s]
        bf16* Wb = nullptr;      // BF16 copy of W
        bf16* Wt = nullptr;      // kind 3: flipped weights [ci_s][Kq]; kinds 1, 2: transpose of Wb [K][rows]
    };
    int width = 0;
    Layer L[kULayers];       // e1a e1b e2a e2b e3a e3b u2 d2a d2b u1 d1a d1b head
    int64_t vcap = 0;              // voxels of one batch at most
    int64_t vmax[3] = {0, 0, 0};   // rows allocated per level (0: full resolution)
    bf16 *x0 = nullptr, *e1a = nullptr, *e1 = nullptr, *u1 = nullptr, *c1 = nullptr, *d1a = nullptr, *d1 = nullptr;
    bf16 *p1 = nullptr, *e2a = nullptr, *e2 = nullptr, *u2 = nullptr, *c2 = nullptr, *d2a = nullptr, *d2 = nullptr;
    bf16 *p2 = nullptr, *e3a = nullptr, *e3 = nullptr;
    uint8_t *arg1 = nullptr, *arg2 = nullptr;
    bf16* cols = nullptr;                       // im2col columns (either order)
    bf16 *dz = nullptr, *dzT = nullptr, *G = nullptr, *aT = nullptr;
    float* P = nullptr;                         // GEMM output / split-K partials
    float *fa = nullptr, *fb = nullptr, *fc = nullptr, *fd = nullptr;   // FP32 gradients of activations
    size_t P_floats = 0, cols_elems = 0, g_elems = 0, f_floats = 0;
    float *Y = nullptr, *T = nullptr;           // [vmax][4]
    double* loss = nullptr;
    unsigned int* gemm_err = nullptr;
    struct Sample {
        int X = 0, Y = 0, Z = 0;                // padded volume extents (multiples of 4)
        int64_t nfluid = 0;
        bf16* in = nullptr;                     // [X Y Z][32]
        float* tg = nullptr;                    // [X Y Z][4]: 100 (X - profile), fluid mask
    };
    std::vector<Sample> samples;
    int64_t step = 0, tcgen05_calls = 0;
    uint64_t seed = 0;
    std::vector<void*> allocs;
    std::string msg;
    lbms_net feat;           // error messages of the shared feature builder (holds no device memory)
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

int64_t round64(int64_t v) { return (v + 63) / 64 * 64; }
// Blocks of 256 threads for one warp per row over R rows (at most 152 x 16 blocks, grid-stride beyond).
int warp_grid(int64_t R) { return (int)std::min<int64_t>((R + 7) / 8, 152 * 16); }
int kp_of(int c_s) { return (27 * c_s + 63) / 64 * 64; }

// The weight gradients reduce over a level's voxels; that reduction is split
// in S chunks of at most kChunkRows (+ 63) rows, so that one CTA of the
// tensor-core GEMM streams a few MB and finishes far inside the GEMM's
// bound on each wait.  A level of V voxels is padded to Vp rows, a multiple
// of 64 S (whole 64-row K steps per chunk).
constexpr int64_t kChunkRows = 16384;

int64_t splits_for(int64_t V) { return std::max<int64_t>(1, (V + kChunkRows - 1) / kChunkRows); }
int64_t padded_rows(int64_t V) {
    const int64_t q = 64 * splits_for(V);
    return (V + q - 1) / q * q;
}
// Rows to allocate for a level that holds at most Vmax voxels (S grows with V).
int64_t rows_bound(int64_t Vmax) { return round64(Vmax + 64 * splits_for(Vmax)); }

struct Dims {
    int X = 0, Y = 0, Z = 0;   // extents of one volume
    int64_t V = 0, Vp = 0;     // voxels of the batch; rows, padded
    int S = 1;                 // chunks of the reduction over the rows
};

Dims level_dims(int B, int X, int Y, int Z, int level) {
    Dims d;
    d.X = X >> level;
    d.Y = Y >> level;
    d.Z = Z >> level;
    d.V = (int64_t)B * d.X * d.Y * d.Z;
    d.S = (int)splits_for(d.V);
    d.Vp = padded_rows(d.V);
    return d;
}

// P[z] = A . B^T on the tcgen05 tensor cores (lbms_umma.cu).
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

lbms_status utranspose(lbms_unet* u, const bf16* in, bf16* out, int64_t R, int C) {
    if ((size_t)R * C > u->g_elems) return ufail(u, LBMS_EINVAL, "U-Net transpose %lld x %d too large", (long long)R, C);
    utranspose_kernel<<<dim3((unsigned)(R / 32), C / 32), dim3(32, 8)>>>(in, out, R, C);
    UCK(cudaGetLastError(), "transpose");
    return LBMS_OK;
}

lbms_status copy_rows(lbms_unet* u, float* dst, int64_t Vp, int C) {
    if ((size_t)Vp * C > u->f_floats) return ufail(u, LBMS_EINVAL, "U-Net gradient %lld x %d too large", (long long)Vp, C);
    UCK(cudaMemcpyAsync(dst, u->P, (size_t)Vp * C * sizeof(float), cudaMemcpyDeviceToDevice, 0), "gradient copy");
    return LBMS_OK;
}

// ------------------------------------------------------ layer passes
// relu(conv(x) + b) -> out (kind 3, or the 1x1 head without ReLU / output)
lbms_status conv_fwd(lbms_unet* u, const lbms_unet::Layer& l, const bf16* x, const Dims& d, bf16* out) {
    if (l.kind == 3) {
        im2col3_kernel<<<warp_grid(d.Vp), 256>>>(x, d.V, d.Vp, d.X, d.Y, d.Z, l.ci_s, l.K, 1, u->cols);
        UCK(cudaGetLastError(), "im2col");
        UST(ugemm(u, u->cols, l.K, l.Wb, l.K, d.Vp, l.co_s, l.K, 1));
    } else {
        UST(ugemm(u, x, l.ci_s, l.Wb, l.K, d.Vp, l.rows, l.K, 1));
    }
    if (out) {
        bias_act_kernel<<<grid_for(d.Vp * l.co_s), 256>>>(u->P, l.b, (int)d.Vp, l.co_s, 1, out, nullptr);
        UCK(cudaGetLastError(), "bias relu");
    }
    return LBMS_OK;
}

// transposed 2x2x2 convolution of x [lo.Vp][ci_s] -> y [8 lo.V][co_s]
lbms_status up_fwd(lbms_unet* u, const lbms_unet::Layer& l, const bf16* x, const Dims& lo, bf16* y) {
    UST(ugemm(u, x, l.ci_s, l.Wb, l.K, lo.Vp, l.rows, l.K, 1));
    upscatter_kernel<<<grid_for(lo.V * l.rows), 256>>>(u->P, l.b, lo.V, lo.X, lo.Y, lo.Z, l.co_s, y);
    UCK(cudaGetLastError(), "up scatter");
    return LBMS_OK;
}

// Backward pass of a 3x3x3 convolution + ReLU: from dA (the gradient of its
// output a) the weight and bias gradients and, with dx, the input gradient
// [Vp][ci_s].
lbms_status conv_bwd(lbms_unet* u, const lbms_unet::Layer& l, const bf16* x, const bf16* a, const float* dA,
                     const Dims& d, float* dx) {
    relu_back_kernel<<<(unsigned)(d.Vp / 32), 256>>>(dA, a, (int)d.Vp, l.co_s, u->dz, l.gb);
    UCK(cudaGetLastError(), "relu backward");
    UST(utranspose(u, u->dz, u->dzT, d.Vp, l.co_s));
    if ((size_t)d.Vp * l.K > u->cols_elems) return ufail(u, LBMS_EINVAL, "U-Net columns too large");
    im2col3_t_kernel<<<(unsigned)(d.Vp / 32), dim3(32, 8)>>>(x, d.V, d.Vp, d.X, d.Y, d.Z, l.ci_s, l.K, u->cols);
    UCK(cudaGetLastError(), "im2col (transposed)");
    const int S = d.S;
    UST(ugemm(u, u->cols, d.Vp, u->dzT, d.Vp, l.K, l.co_s, d.Vp, S));
    splitk_sum_t_kernel<<<grid_for((int64_t)l.co_s * l.K), 256>>>(u->P, S, l.K, l.co_s, l.g);
    UCK(cudaGetLastError(), "split-k sum");
    if (!dx) return LBMS_OK;
    if ((size_t)d.Vp * l.Kq > u->cols_elems) return ufail(u, LBMS_EINVAL, "U-Net columns too large");
    im2col3_kernel<<<warp_grid(d.Vp), 256>>>(u->dz, d.V, d.Vp, d.X, d.Y, d.Z, l.co_s, l.Kq, -1, u->cols);
    UCK(cudaGetLastError(), "im2col (reflected)");
    UST(ugemm(u, u->cols, l.Kq, l.Wt, l.Kq, d.Vp, l.ci_s, l.Kq, 1));
    return copy_rows(u, dx, d.Vp, l.ci_s);
}

// Backward pass of the transposed convolution from dy [hi.Vp][co_s]: weight
// and bias gradients and the gradient of its input [lo.Vp][ci_s].
lbms_status up_bwd(lbms_unet* u, const lbms_unet::Layer& l, const bf16* x, const float* dy, const Dims& lo,
                   const Dims& hi, float* dx) {
    colsum_kernel<<<(unsigned)(hi.Vp / 32), 128>>>(dy, hi.Vp, l.co_s, l.gb);
    UCK(cudaGetLastError(), "bias gradient");
    if ((size_t)lo.Vp * l.rows > u->g_elems) return ufail(u, LBMS_EINVAL, "U-Net gather too large");
    upgather_kernel<<<grid_for(lo.Vp * l.rows), 256>>>(dy, lo.V, lo.Vp, lo.X, lo.Y, lo.Z, l.co_s, u->G);
    UCK(cudaGetLastError(), "up gather");
    UST(utranspose(u, u->G, u->dzT, lo.Vp, l.rows));
    UST(utranspose(u, x, u->aT, lo.Vp, l.ci_s));
    const int S = lo.S;
    UST(ugemm(u, u->dzT, lo.Vp, u->aT, lo.Vp, l.rows, l.ci_s, lo.Vp, S));
    splitk_sum_kernel<<<grid_for((int64_t)l.rows * l.K), 256>>>(u->P, S, (int64_t)l.rows * l.K, l.g);
    UCK(cudaGetLastError(), "split-k sum");
    UST(ugemm(u, u->G, l.rows, l.Wt, l.rows, lo.Vp, l.ci_s, l.rows, 1));
    return copy_rows(u, dx, lo.Vp, l.ci_s);
}

// ------------------------------------------------------ network passes
// Forward pass of B volumes of X x Y x Z voxels (multiples of 4) already in
// u->x0; the head's product (without its bias) is left in u->P [Vp][64].
lbms_status unet_forward(lbms_unet* u, int B, int X, int Y, int Z) {
    const Dims d0 = level_dims(B, X, Y, Z, 0), d1 = level_dims(B, X, Y, Z, 1), d2 = level_dims(B, X, Y, Z, 2);
    const int w = u->width;
    auto& L = u->L;
    UST(conv_fwd(u, L[0], u->x0, d0, u->e1a));
    UST(conv_fwd(u, L[1], u->e1a, d0, u->e1));
    pool_fwd_kernel<<<grid_for(d1.V * 64), 256>>>(u->e1, d1.V, X, Y, Z, 64, u->p1, u->arg1);
    UCK(cudaGetLastError(), "pool");
    UST(conv_fwd(u, L[2], u->p1, d1, u->e2a));
    UST(conv_fwd(u, L[3], u->e2a, d1, u->e2));
    pool_fwd_kernel<<<grid_for(d2.V * 64), 256>>>(u->e2, d2.V, d1.X, d1.Y, d1.Z, 64, u->p2, u->arg2);
    UCK(cudaGetLastError(), "pool");
    UST(conv_fwd(u, L[4], u->p2, d2, u->e3a));
    UST(conv_fwd(u, L[5], u->e3a, d2, u->e3));
    UST(up_fwd(u, L[6], u->e3, d2, u->u2));
    concat_kernel<<<grid_for(d1.Vp * 128), 256>>>(u->u2, 64, 2 * w, u->e2, 64, 2 * w, d1.Vp, 128, u->c2);
    UCK(cudaGetLastError(), "concat");
    UST(conv_fwd(u, L[7], u->c2, d1, u->d2a));
    UST(conv_fwd(u, L[8], u->d2a, d1, u->d2));
    UST(up_fwd(u, L[9], u->d2, d1, u->u1));
    concat_kernel<<<grid_for(d0.Vp * 64), 256>>>(u->u1, 64, w, u->e1, 64, w, d0.Vp, 64, u->c1);
    UCK(cudaGetLastError(), "concat");
    UST(conv_fwd(u, L[10], u->c1, d0, u->d1a));
    UST(conv_fwd(u, L[11], u->d1a, d0, u->d1));
    return conv_fwd(u, L[12], u->d1, d0, nullptr);
}

// Loss against u->T (targets and mask) and the backward pass through every
// layer after unet_forward; gradients in each layer's g / gb.
lbms_status unet_backward(lbms_unet* u, int B, int X, int Y, int Z, float inv_n) {
    const Dims d0 = level_dims(B, X, Y, Z, 0), d1 = level_dims(B, X, Y, Z, 1), d2 = level_dims(B, X, Y, Z, 2);
    const int w = u->width;
    auto& L = u->L;
    UCK(cudaMemsetAsync(u->loss, 0, sizeof(double), 0), "loss");
    for (auto& l : L) UCK(cudaMemsetAsync(l.gb, 0, l.co_s * sizeof(float), 0), "bias gradients");
    // head: dP, its weight gradient dP^T . d1 and the gradient of d1
    const lbms_unet::Layer& h = L[12];
    unet_loss_kernel<<<(unsigned)(d0.Vp / 64), 256>>>(u->P, h.b, u->T, d0.Vp, inv_n, u->dz, h.gb, u->loss, u->Y);
    UCK(cudaGetLastError(), "loss");
    UST(utranspose(u, u->dz, u->dzT, d0.Vp, kUOutC));
    UST(utranspose(u, u->d1, u->aT, d0.Vp, h.ci_s));
    const int S = d0.S;
    UST(ugemm(u, u->dzT, d0.Vp, u->aT, d0.Vp, h.rows, h.ci_s, d0.Vp, S));
    splitk_sum_kernel<<<grid_for((int64_t)h.rows * h.K), 256>>>(u->P, S, (int64_t)h.rows * h.K, h.g);
    UCK(cudaGetLastError(), "split-k sum");
    UST(ugemm(u, u->dz, kUOutC, h.Wt, h.rows, d0.Vp, h.ci_s, h.rows, 1));
    UST(copy_rows(u, u->fa, d0.Vp, h.ci_s));
    // decoder, level 0
    UST(conv_bwd(u, L[11], u->d1a, u->d1, u->fa, d0, u->fb));
    UST(conv_bwd(u, L[10], u->c1, u->d1a, u->fb, d0, u->fa));
    split_kernel<<<grid_for(d0.Vp * 64), 256>>>(u->fa, 64, w, w, 64, 64, d0.Vp, u->fb, u->fc);
    UCK(cudaGetLastError(), "split");
    UST(up_bwd(u, L[9], u->d2, u->fb, d1, d0, u->fd));
    // decoder, level 1
    UST(conv_bwd(u, L[8], u->d2a, u->d2, u->fd, d1, u->fa));
    UST(conv_bwd(u, L[7], u->c2, u->d2a, u->fa, d1, u->fb));
    split_kernel<<<grid_for(d1.Vp * 64), 256>>>(u->fb, 128, 2 * w, 2 * w, 64, 64, d1.Vp, u->fa, u->fd);
    UCK(cudaGetLastError(), "split");
    UST(up_bwd(u, L[6], u->e3, u->fa, d2, d1, u->fb));
    // bottom, level 2
    UST(conv_bwd(u, L[5], u->e3a, u->e3, u->fb, d2, u->fa));
    UST(conv_bwd(u, L[4], u->p2, u->e3a, u->fa, d2, u->fb));
    pool_bwd_kernel<<<grid_for(d1.V * 64), 256>>>(u->fb, u->arg2, d1.V, d1.X, d1.Y, d1.Z, 64, u->fd);
    UCK(cudaGetLastError(), "pool backward");
    // encoder, level 1
    UST(conv_bwd(u, L[3], u->e2a, u->e2, u->fd, d1, u->fa));
    UST(conv_bwd(u, L[2], u->p1, u->e2a, u->fa, d1, u->fb));
    pool_bwd_kernel<<<grid_for(d0.V * 64), 256>>>(u->fb, u->arg1, d0.V, d0.X, d0.Y, d0.Z, 64, u->fc);
    UCK(cudaGetLastError(), "pool backward");
    // encoder, level 0
    UST(conv_bwd(u, L[1], u->e1a, u->e1, u->fc, d0, u->fa));
    return conv_bwd(u, L[0], u->x0, u->e1a, u->fa, d0, nullptr);
}

// The BF16 copies of one layer's weights from its FP32 master copy.
lbms_status cast_layer(lbms_unet* u, const lbms_unet::Layer& l) {
    if (l.kind == 3)
        conv_cast_kernel<<<grid_for((int64_t)l.rows * l.K), 256>>>(l.W, l.co_s, l.ci_s, l.K, l.Kq, l.Wb, l.Wt);
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

// The volume of a case on the network's grid: extents rounded up to
// multiples of 4, each fluid cell's index in it.
struct CaseVolume {
    int X = 0, Y = 0, Z = 0;
    std::vector<int64_t> cell;
};

void case_volume(const lbms::CaseView& v, CaseVolume& cv) {
    cv.X = (v.nx + 3) / 4 * 4;
    cv.Y = (v.ny + 3) / 4 * 4;
    cv.Z = (v.nz + 3) / 4 * 4;
    cv.cell.resize(v.nf);
    for (int j = 0; j < v.nf; ++j) {
        const int64_t e = v.fluid_cell[j];
        const int64_t x = e % v.nx, y = (e / v.nx) % v.ny, z = e / ((int64_t)v.nx * v.ny);
        cv.cell[j] = (z * cv.Y + y) * cv.X + x;
    }
}

}  // namespace

extern "C" {

void lbms_unet_destroy(lbms_unet* u) {
    if (!u) return;
    for (void* p : u->allocs) cudaFree(p);
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
    const int w = width;
    // kind, output level, real / stored input channels, real / stored output channels
    const int spec[kULayers][6] = {{3, 0, kUInReal, kUInC, w, 64}, {3, 0, w, 64, w, 64},
                                   {3, 1, w, 64, 2 * w, 64},       {3, 1, 2 * w, 64, 2 * w, 64},
                                   {3, 2, 2 * w, 64, 4 * w, 128},  {3, 2, 4 * w, 128, 4 * w, 128},
                                   {2, 1, 4 * w, 128, 2 * w, 64},  {3, 1, 4 * w, 128, 2 * w, 64},
                                   {3, 1, 2 * w, 64, 2 * w, 64},   {2, 0, 2 * w, 64, w, 64},
                                   {3, 0, 2 * w, 64, w, 64},       {3, 0, w, 64, w, 64},
                                   {1, 0, w, 64, 3, kUOutC}};
    u->vcap = max_voxels;
    int64_t smax[3];
    for (int lev = 0; lev < 3; ++lev) {
        u->vmax[lev] = rows_bound(max_voxels >> (3 * lev));
        smax[lev] = splits_for(max_voxels >> (3 * lev));
    }
    size_t cols = 0, P = (size_t)u->vmax[0] * kUOutC, g = (size_t)u->vmax[0] * kUOutC, f = (size_t)u->vmax[0] * 64;
    for (int i = 0; i < kULayers; ++i) {
        auto& l = u->L[i];
        l.kind = spec[i][0];
        l.level = spec[i][1];
        l.ci = spec[i][2];
        l.ci_s = spec[i][3];
        l.co = spec[i][4];
        l.co_s = spec[i][5];
        const size_t vh = (size_t)u->vmax[l.level];
        if (l.kind == 3) {
            l.rows = l.co_s;
            l.K = kp_of(l.ci_s);
            l.Kq = kp_of(l.co_s);
            cols = std::max(cols, vh * std::max(l.K, l.Kq));
            P = std::max({P, vh * l.co_s, vh * l.ci_s, (size_t)smax[l.level] * l.K * l.co_s});
            g = std::max(g, vh * l.co_s);
            f = std::max({f, vh * l.co_s, vh * l.ci_s});
        } else if (l.kind == 2) {
            l.rows = 8 * l.co_s;
            l.K = l.ci_s;
            const size_t vl = (size_t)u->vmax[l.level + 1];
            P = std::max({P, vl * l.rows, vl * l.ci_s, (size_t)smax[l.level + 1] * l.rows * l.ci_s});
            g = std::max({g, vl * l.rows, vl * l.ci_s});
            f = std::max({f, vh * l.co_s, vl * l.ci_s});
        } else {
            l.rows = l.co_s;
            l.K = l.ci_s;
            P = std::max(P, (size_t)smax[0] * l.rows * l.K);
        }
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
        l.Wt = ualloc<bf16>(u, l.kind == 3 ? (size_t)l.ci_s * l.Kq : nw);
    }
    u->cols_elems = cols;
    u->P_floats = P;
    u->g_elems = g;
    u->f_floats = f;
    const size_t v0 = u->vmax[0], v1 = u->vmax[1], v2 = u->vmax[2];
    std::vector<std::pair<void*, size_t>> zero;   // activation buffers cleared once (no NaN in padding rows)
    auto act = [&](size_t n) {
        bf16* p = ualloc<bf16>(u, n);
        zero.emplace_back(p, n * sizeof(bf16));
        return p;
    };
    u->x0 = act(v0 * kUInC);
    u->e1a = act(v0 * 64);
    u->e1 = act(v0 * 64);
    u->u1 = act(v0 * 64);
    u->c1 = act(v0 * 64);
    u->d1a = act(v0 * 64);
    u->d1 = act(v0 * 64);
    u->p1 = act(v1 * 64);
    u->e2a = act(v1 * 64);
    u->e2 = act(v1 * 64);
    u->u2 = act(v1 * 64);
    u->c2 = act(v1 * 128);
    u->d2a = act(v1 * 64);
    u->d2 = act(v1 * 64);
    u->p2 = act(v2 * 64);
    u->e3a = act(v2 * 128);
    u->e3 = act(v2 * 128);
    u->arg1 = ualloc<uint8_t>(u, v1 * 64);
    u->arg2 = ualloc<uint8_t>(u, v2 * 64);
    u->cols = ualloc<bf16>(u, cols);
    u->dz = ualloc<bf16>(u, g);
    u->dzT = ualloc<bf16>(u, g);
    u->G = ualloc<bf16>(u, g);
    u->aT = ualloc<bf16>(u, g);
    u->P = ualloc<float>(u, P);
    u->fa = ualloc<float>(u, f);
    u->fb = ualloc<float>(u, f);
    u->fc = ualloc<float>(u, f);
    u->fd = ualloc<float>(u, f);
    u->Y = ualloc<float>(u, v0 * 4);
    u->T = ualloc<float>(u, v0 * 4);
    u->loss = ualloc<double>(u, 1);
    u->gemm_err = ualloc<unsigned int>(u, 1);
    bool ok = true;
    for (void* p : u->allocs) ok = ok && p;
    if (!ok) {
        lbms_unet_destroy(u);
        return LBMS_ENOMEM;
    }
    ok = lbms::umma_gemm_init() == cudaSuccess;
    for (auto& z : zero) ok = ok && cudaMemset(z.first, 0, z.second) == cudaSuccess;
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
        ok = ok && cudaMemset(l.Wt, 0, (l.kind == 3 ? (size_t)l.ci_s * l.Kq : nw) * sizeof(bf16)) == cudaSuccess;
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
    const int64_t Vs = (int64_t)cv.X * cv.Y * cv.Z;
    if (Vs > u->vcap)
        return ufail(u, LBMS_EINVAL, "case %d needs %lld voxels, the network was made for %lld", k, (long long)Vs,
                     (long long)u->vcap);
    std::vector<double> X((size_t)3 * v.N);
    st = lbms_batch_get_fields(ctx, k, X.data(), nullptr, nullptr);
    if (st != LBMS_OK) return ufail(u, st, "reading the fields of case %d: %s", k, lbms_last_error(ctx));
    std::vector<float> t((size_t)Vs * 4, 0.0f);
    for (int j = 0; j < v.nf; ++j) {
        const int64_t e = v.fluid_cell[j];
        const int x = (int)(e % v.nx);
        float* r = &t[(size_t)cv.cell[j] * 4];
        for (int s = 0; s < 3; ++s) r[s] = (float)(kTargetScale * (X[(size_t)s * v.N + e] - F.prof[(size_t)s * v.nx + x]));
        r[3] = 1.0f;
    }
    lbms_unet::Sample s;
    s.X = cv.X;
    s.Y = cv.Y;
    s.Z = cv.Z;
    s.nfluid = v.nf;
    int64_t* pcell = F.alloc<int64_t>(v.nf);
    if (!pcell) return ufail(u, LBMS_ENOMEM, "cell indices");
    if (cudaMalloc(&s.in, (size_t)Vs * kUInC * sizeof(bf16)) != cudaSuccess) return ufail(u, LBMS_ENOMEM, "sample");
    if (cudaMalloc(&s.tg, (size_t)Vs * 4 * sizeof(float)) != cudaSuccess) {
        cudaFree(s.in);
        return ufail(u, LBMS_ENOMEM, "sample");
    }
    cudaError_t e = cudaMemcpy(pcell, cv.cell.data(), v.nf * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(s.in, 0, (size_t)Vs * kUInC * sizeof(bf16));
    if (e == cudaSuccess) {
        unet_inputs_kernel<<<grid_for((int64_t)v.nf * kUInC), 256>>>(F.rows, pcell, v.nf, s.in);
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

lbms_status lbms_unet_train(lbms_unet* u, int iters, int max_batch, double lr, double* last_loss) {
    if (!u) return LBMS_EINVAL;
    if (iters < 0 || max_batch < 1 || !(lr > 0.0))
        return ufail(u, LBMS_EINVAL, "need iters >= 0, max_batch >= 1, lr > 0");
    if (u->samples.empty()) return ufail(u, LBMS_ESTATE, "no training volumes (call lbms_unet_add_sample first)");
    // groups of equal volume extents, in order of first appearance
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
    double tail = 0.0;
    int nt = 0;
    for (int it = 0; it < iters; ++it) {
        const auto& g = groups[it % groups.size()];
        const auto& s0 = u->samples[g[0]];
        const int64_t Vs = (int64_t)s0.X * s0.Y * s0.Z;
        const int B = (int)std::min<int64_t>({(int64_t)max_batch, (int64_t)g.size(), u->vcap / Vs});
        const uint64_t key = splitmix64(u->seed ^ 0x5A5A5A5Aull) + (uint64_t)u->step * 64ull;
        int64_t nfl = 0;
        for (int i = 0; i < B; ++i) {
            const auto& s = u->samples[g[splitmix64(key + (uint64_t)i) % g.size()]];
            UCK(cudaMemcpyAsync(u->x0 + i * Vs * kUInC, s.in, Vs * kUInC * sizeof(bf16), cudaMemcpyDeviceToDevice, 0),
                "batch");
            UCK(cudaMemcpyAsync(u->T + i * Vs * 4, s.tg, Vs * 4 * sizeof(float), cudaMemcpyDeviceToDevice, 0), "batch");
            nfl += s.nfluid;
        }
        const int64_t V = B * Vs;
        UCK(cudaMemsetAsync(u->T + V * 4, 0, (padded_rows(V) - V) * 4 * sizeof(float), 0), "batch");
        const double cw = 0.5 * (1.0 + std::cos(3.14159265358979323846 * (double)it / std::max(1, iters)));
        const double lr_it = lr / 20.0 + (lr - lr / 20.0) * cw;
        UST(unet_forward(u, B, s0.X, s0.Y, s0.Z));
        UST(unet_backward(u, B, s0.X, s0.Y, s0.Z, (float)(1.0 / (3.0 * (double)std::max<int64_t>(nfl, 1)))));
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
    const int64_t Vs = (int64_t)cv.X * cv.Y * cv.Z;
    if (Vs > u->vcap)
        return ufail(u, LBMS_EINVAL, "case %d needs %lld voxels, the network was made for %lld", k, (long long)Vs,
                     (long long)u->vcap);
    int64_t* pcell = F.alloc<int64_t>(v.nf);
    double* dX = F.alloc<double>((size_t)3 * v.nf);
    if (!pcell || !dX) return ufail(u, LBMS_ENOMEM, "prediction buffers");
    UCK(cudaMemcpy(pcell, cv.cell.data(), v.nf * sizeof(int64_t), cudaMemcpyHostToDevice), "cells");
    UCK(cudaMemset(u->x0, 0, (size_t)padded_rows(Vs) * kUInC * sizeof(bf16)), "inputs");
    unet_inputs_kernel<<<grid_for((int64_t)v.nf * kUInC), 256>>>(F.rows, pcell, v.nf, u->x0);
    UCK(cudaGetLastError(), "inputs");
    UST(unet_forward(u, 1, cv.X, cv.Y, cv.Z));
    const int64_t Vp = padded_rows(Vs);
    unet_loss_kernel<<<(unsigned)(Vp / 64), 256>>>(u->P, u->L[kULayers - 1].b, nullptr, Vp, 0.0f, nullptr, nullptr,
                                                   nullptr, u->Y);
    UCK(cudaGetLastError(), "head");
    unet_post_kernel<<<(v.nf + 255) / 256, 256>>>(u->Y, pcell, v.nf, cv.X, F.xtab, dX);
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

namespace {

// Uploads a host batch FP32 [B][17][X Y Z] (and targets [B][3][X Y Z]) into
// x0 and T; returns the number of fluid voxels (the mask channel's sum).
lbms_status upload_batch(lbms_unet* u, const float* x, const float* t, int B, int X, int Y, int Z, double* nfluid) {
    if (!x || B < 1 || X < 4 || Y < 4 || Z < 4 || X % 4 || Y % 4 || Z % 4)
        return ufail(u, LBMS_EINVAL, "need B >= 1 volumes with extents multiples of 4");
    const int64_t S = (int64_t)X * Y * Z, V = B * S;
    if (V > u->vcap)
        return ufail(u, LBMS_EINVAL, "the batch holds %lld voxels, the network was made for %lld", (long long)V,
                     (long long)u->vcap);
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
    if (e == cudaSuccess) e = cudaMemset(u->T, 0, (size_t)padded_rows(V) * 4 * sizeof(float));
    if (e == cudaSuccess) {
        vol_in_kernel<<<grid_for(V * kUInC), 256>>>(dev, V, S, u->x0, u->T);
        if (t) vol_target_kernel<<<grid_for(V * 3), 256>>>(dev + nin, V, S, u->T);
        e = cudaDeviceSynchronize();
    }
    if (e != cudaSuccess) st = ufail(u, LBMS_ECUDA, "batch upload: %s", cudaGetErrorString(e));
    cudaFree(dev);
    return st;
}

}  // namespace

lbms_status lbms_unet_forward(lbms_unet* u, const float* x, int B, int X, int Y, int Z, float* y) {
    if (!u || !y) return LBMS_EINVAL;
    UST(upload_batch(u, x, nullptr, B, X, Y, Z, nullptr));
    UST(unet_forward(u, B, X, Y, Z));
    const int64_t S = (int64_t)X * Y * Z, V = B * S, Vp = padded_rows(V);
    unet_loss_kernel<<<(unsigned)(Vp / 64), 256>>>(u->P, u->L[kULayers - 1].b, nullptr, Vp, 0.0f, nullptr, nullptr,
                                                   nullptr, u->Y);
    UCK(cudaGetLastError(), "head");
    std::vector<float> h((size_t)V * 4);
    UCK(cudaMemcpy(h.data(), u->Y, h.size() * sizeof(float), cudaMemcpyDeviceToHost), "read output");
    UST(unet_check_gemm(u));
    for (int64_t v = 0; v < V; ++v)
        for (int c = 0; c < 3; ++c) y[((v / S) * 3 + c) * S + v % S] = h[(size_t)v * 4 + c];
    return LBMS_OK;
}

lbms_status lbms_unet_train_batch(lbms_unet* u, const float* x, const float* t, int B, int X, int Y, int Z, double lr,
                                  double* loss) {
    if (!u || !t || !(lr >= 0.0)) return LBMS_EINVAL;
    double nf = 0.0;
    UST(upload_batch(u, x, t, B, X, Y, Z, &nf));
    UST(unet_forward(u, B, X, Y, Z));
    UST(unet_backward(u, B, X, Y, Z, (float)(1.0 / (3.0 * std::max(nf, 1.0)))));
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
