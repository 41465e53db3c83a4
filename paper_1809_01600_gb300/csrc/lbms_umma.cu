// BF16 matrix product of the warm-start network on the fifth-generation
// tensor cores: P[z][M][N] = sum_{k in chunk z} A[m][k] B[n][k] with A [M][K]
// and B [N][K] both K-contiguous ("TN"), FP32 accumulation.
//
// One CTA of 128 threads per 128 x 64 output tile and K chunk.  Operand
// tiles of 64 K-elements (one 128-byte swizzle span of BF16) are staged in
// shared memory by TMA (cp.async.bulk.tensor, 128-byte swizzle) through a
// four-stage ring of mbarriers; one thread issues tcgen05.mma (M = 128,
// N = 64, K = 16 per instruction) into a TMEM accumulator of 64 columns, and
// tcgen05.commit releases each stage when the products reading it are done.
// The four warps then read their 32 TMEM lanes (rows) with tcgen05.ld and
// store FP32.  Rows and K beyond the operands' extents are zero-filled by
// TMA, so M and K need no padding; N is a multiple of 64.
//
// The convolutions of the 3-D U-Net (lbms_unet.cuh) run on the same
// machinery.  Its activations are stored in a layout with a zero halo of one
// voxel per side, so that the neighbour of every interior voxel at tap
// t = (dz, dy, dx) lies a fixed number of rows off(t) away:
//  * implicit convolution (umma_conv_kernel below): K runs over 27 taps x C
//    channels; the A tile of tap t is the activation matrix [rows][C] read
//    at rows m0 + off(t) (TMA zero-fills rows outside it), one 130-row window
//    shared by the three taps of a (dz, dy) row; B the weights [N][27 C];
//  * weight gradient (load mode 2 of umma_gemm_kernel):
//    P[t C + c][n] = sum_r x[r + off(t)][c] dZ[r][n]
//    with B = dZ^T [N][rows]; the A tile's two 64-row halves come from three
//    transposed copies xT_j[c][r] = x[r + j - 1][c] (j = dx + 1) of the
//    input, each read at inner coordinate r + (dz Yp + dy) Xp, a multiple of
//    8 elements when the padded x extent Xp is (the 16-byte rule of tiled
//    TMA); rows of A past 27 C read as zero.
//
// Every mbarrier wait is bounded (about 2 s on the global timer): on a
// timeout the kernel raises *err, still waits (bounded) for the copies it
// issued, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "lbms_internal.h"

namespace lbms {
namespace {

constexpr int kUM = 128;                       // output rows per CTA (UMMA M)
constexpr int kUN = 64;                        // output columns per CTA (UMMA N)
constexpr int kUK = 64;                        // K per stage: 64 BF16 = one 128-byte swizzle row
constexpr int kStages = 4;
constexpr int kABytes = kUM * kUK * 2;         // 16 KiB
constexpr int kBBytes = kUN * kUK * 2;         // 8 KiB
constexpr int kStageBytes = kABytes + kBBytes;
constexpr int kTmemCols = 64;                  // FP32 accumulator: 128 lanes x 64 columns
constexpr size_t kSmemBytes = 1024 + (size_t)kStages * kStageBytes + 256;
constexpr uint64_t kWaitNs = 2000000000ull;    // bound of every mbarrier wait

// Instruction descriptor of tcgen05.mma kind::f16: D FP32 (bits 4-5 = 1),
// A and B BF16 (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0),
// N >> 3 in bits 17-22, M >> 4 in bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kUN >> 3) << 17) |
                            ((uint32_t)(kUM >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Waits for the completion of the phase of parity `par`; false after kWaitNs.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t par) {
    const uint32_t a = smem_u32(bar);
    const uint64_t t0 = global_ns();
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(a), "r"(par)
            : "memory");
        if (done) return true;
        if (global_ns() - t0 > kWaitNs) return false;
    }
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor of a K-major operand tile whose rows are
// 128 bytes (64 BF16) in the 128-byte swizzle written by TMA: start address
// >> 4 (bits 0-13), leading offset 16 B (unused with this swizzle, bits
// 16-29), 8-row groups 1024 B apart (bits 32-45), the fixed 0b001 of bits
// 46-48, swizzle mode 2 = 128 B (bits 61-63).  The tile base is 1024-byte
// aligned; the k-th 16-element slice starts 32 k bytes further.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
           ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

__device__ __forceinline__ void umma_f16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            tmem),
        "l"(ad), "l"(bd), "r"(kIdesc), "r"(accumulate));
}

__device__ __forceinline__ void umma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
        "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}

// Load modes of the kernel (see the head of the file).
constexpr int kModePlain = 0, kModeWgrad = 2;

template <int kMode>
__global__ void __launch_bounds__(128, 1) umma_gemm_kernel(const __grid_constant__ CUtensorMap mapA,
                                                           const __grid_constant__ CUtensorMap mapB,
                                                           const __grid_constant__ CUtensorMap mapB1,
                                                           const __grid_constant__ CUtensorMap mapB2,
                                                           float* __restrict__ P, int M, int N, int kchunk,
                                                           unsigned int* __restrict__ err, const __grid_constant__ ConvTaps taps) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint64_t* full = reinterpret_cast<uint64_t*>(base + (size_t)kStages * kStageBytes);
    uint64_t* empty = full + kStages;
    uint64_t* done = empty + kStages;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n0 = blockIdx.x * kUN, m0 = blockIdx.y * kUM, k0 = blockIdx.z * kchunk;
    const int nk = kchunk / kUK;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (threadIdx.x == 0) {
        bool ok = true;
        int issued = 0;                        // stages whose loads were issued
        // mode 2: each 64-row half h of the A tile is one tap's channel block:
        // its copy (by dx), its inner shift and its first channel
        const CUtensorMap* ma2[2] = {&mapA, &mapA};
        int shift2[2] = {0, 0}, c2[2] = {0, 0};
        if (kMode == kModeWgrad) {
            for (int h = 0; h < 2; ++h) {
                const int m = m0 + 64 * h, t = m / taps.per_tap;
                if (t < 27) {
                    ma2[h] = t % 3 == 0 ? &mapA : t % 3 == 1 ? &mapB1 : &mapB2;
                    shift2[h] = taps.off[t];
                    c2[h] = m - t * taps.per_tap;
                } else {
                    c2[h] = taps.per_tap;   // past the copy's rows: zero-filled
                }
            }
        }
        auto load = [&](int kt) {
            const int s = kt % kStages;
            uint8_t* sa = base + (size_t)s * kStageBytes;
            mbar_expect_tx(&full[s], kStageBytes);
            if (kMode == kModeWgrad) {
                tma_load_2d(sa, ma2[0], k0 + kt * kUK + shift2[0], c2[0], &full[s]);
                tma_load_2d(sa + kABytes / 2, ma2[1], k0 + kt * kUK + shift2[1], c2[1], &full[s]);
                tma_load_2d(sa + kABytes, &mapB, k0 + kt * kUK, n0, &full[s]);
            } else {
                tma_load_2d(sa, &mapA, k0 + kt * kUK, m0, &full[s]);
                tma_load_2d(sa + kABytes, &mapB, k0 + kt * kUK, n0, &full[s]);
            }
            ++issued;
        };
        for (int kt = 0; kt < nk && kt < kStages; ++kt) load(kt);
        int consumed = 0;
        for (int kt = 0; kt < nk; ++kt) {
            const int s = kt % kStages;
            const uint32_t ph = (uint32_t)(kt / kStages) & 1u;
            if (!mbar_wait(&full[s], ph)) {
                ok = false;
                break;
            }
            ++consumed;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t a = smem_u32(base + (size_t)s * kStageBytes);
            const uint32_t b = a + kABytes;
#pragma unroll
            for (int j = 0; j < kUK / 16; ++j)
                umma_f16(tmem, sw128_desc(a + 32 * j), sw128_desc(b + 32 * j), (kt | j) != 0 ? 1u : 0u);
            umma_commit(&empty[s]);
            if (kt + kStages < nk) {
                if (!mbar_wait(&empty[s], ph)) {
                    ok = false;
                    break;
                }
                load(kt + kStages);
            }
        }
        umma_commit(done);                     // arrives once every product issued above is complete
        if (!ok) {
            atomicOr(err, 1u);
            // copies still in flight land in their stages before the CTA exits
            for (int kt = consumed; kt < issued; ++kt) mbar_wait(&full[kt % kStages], (uint32_t)(kt / kStages) & 1u);
        }
    }
    __syncwarp();
    const bool got = mbar_wait(done, 0);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!got) {
        if (lane == 0) atomicOr(err, 2u);
    } else {
        // warp w holds TMEM lanes (rows) 32 w .. 32 w + 31: row m0 + 32 w + lane, 64 columns
        const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16);
        uint32_t v0[32], v1[32];
        tmem_ld32(taddr, v0);
        tmem_ld32(taddr + 32, v1);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int row = m0 + 32 * warp + lane;
        if (row < M) {
            float4* dst = reinterpret_cast<float4*>(P + (int64_t)blockIdx.z * M * N + (int64_t)row * N + n0);
#pragma unroll
            for (int q = 0; q < 8; ++q)
                dst[q] = make_float4(__uint_as_float(v0[4 * q]), __uint_as_float(v0[4 * q + 1]),
                                     __uint_as_float(v0[4 * q + 2]), __uint_as_float(v0[4 * q + 3]));
#pragma unroll
            for (int q = 0; q < 8; ++q)
                dst[8 + q] = make_float4(__uint_as_float(v1[4 * q]), __uint_as_float(v1[4 * q + 1]),
                                         __uint_as_float(v1[4 * q + 2]), __uint_as_float(v1[4 * q + 3]));
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// ---------------------------------------------------------------------------
// Implicit 3x3x3 convolution with the A tile shared by the three taps of a
// (dz, dy) row.  Those taps differ in dx only, so their A tiles are the same
// activation rows shifted by one: one TMA box of 130 rows (the window from
// the tap with the lowest offset) serves all three, each MMA reading it
// from row 0, 1 or 2.  The 128-byte swizzle is a function of the shared
// address bits, as TMA wrote it, so a descriptor whose start is s rows
// (128 s bytes) into the window reads those rows correctly with matrix base
// offset 0 (checked against a CPU implicit-GEMM reference; base offset
// (start >> 7) & 7 gives wrong products).  A stage holds the window and the
// three taps' 64 x 64 B tiles; K runs over 9 rows of taps x C / 64 channel
// blocks.
constexpr int kCRows = kUM + 2;                                   // window rows
constexpr int kCABytes = (kCRows * kUK * 2 + 1023) / 1024 * 1024;  // 17 KiB (1024-aligned B tiles follow)
constexpr int kCStageBytes = kCABytes + 3 * kBBytes;
constexpr int kCStages = 2;                                       // two CTAs fit on an SM
constexpr size_t kCSmemBytes = 1024 + (size_t)kCStages * kCStageBytes + 256;

__global__ void __launch_bounds__(128, 1) umma_conv_kernel(const __grid_constant__ CUtensorMap mapA,
                                                           const __grid_constant__ CUtensorMap mapB,
                                                           float* __restrict__ P, int M, int N, int cpt,
                                                           unsigned int* __restrict__ err,
                                                           const __grid_constant__ ConvTaps taps,
                                                           const __grid_constant__ ConvEpilogue ep) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t* base = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint64_t* full = reinterpret_cast<uint64_t*>(base + (size_t)kCStages * kCStageBytes);
    uint64_t* empty = full + kCStages;
    uint64_t* done = empty + kCStages;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n0 = blockIdx.x * kUN, m0 = blockIdx.y * kUM;
    const int nk = 9 * cpt;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kCStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;

    if (threadIdx.x == 0) {
        bool ok = true;
        int issued = 0;
        // the lowest of the three offsets of tap row g: the window's first row
        auto low = [&](int g) {
            const int a = taps.off[3 * g], b = taps.off[3 * g + 1], c = taps.off[3 * g + 2];
            return min(a, min(b, c));
        };
        auto load = [&](int kt) {
            const int s = kt % kCStages;
            const int g = kt / cpt, c = kt - g * cpt;
            uint8_t* sa = base + (size_t)s * kCStageBytes;
            mbar_expect_tx(&full[s], kCRows * kUK * 2 + 3 * kBBytes);
            tma_load_2d(sa, &mapA, c * kUK, m0 + low(g), &full[s]);
            for (int d = 0; d < 3; ++d)
                tma_load_2d(sa + kCABytes + d * kBBytes, &mapB, ((3 * g + d) * cpt + c) * kUK, n0, &full[s]);
            ++issued;
        };
        for (int kt = 0; kt < nk && kt < kCStages; ++kt) load(kt);
        int consumed = 0;
        for (int kt = 0; kt < nk; ++kt) {
            const int s = kt % kCStages;
            const uint32_t ph = (uint32_t)(kt / kCStages) & 1u;
            if (!mbar_wait(&full[s], ph)) {
                ok = false;
                break;
            }
            ++consumed;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int g = kt / cpt;
            const int lo = low(g);
            const uint32_t a = smem_u32(base + (size_t)s * kCStageBytes);
            for (int d = 0; d < 3; ++d) {
                const uint32_t arow = a + 128u * (uint32_t)(taps.off[3 * g + d] - lo);
                const uint32_t b = a + kCABytes + d * kBBytes;
#pragma unroll
                for (int j = 0; j < kUK / 16; ++j)
                    umma_f16(tmem, sw128_desc(arow + 32 * j), sw128_desc(b + 32 * j), (kt | d | j) != 0 ? 1u : 0u);
            }
            umma_commit(&empty[s]);
            if (kt + kCStages < nk) {
                if (!mbar_wait(&empty[s], ph)) {
                    ok = false;
                    break;
                }
                load(kt + kCStages);
            }
        }
        umma_commit(done);
        if (!ok) {
            atomicOr(err, 1u);
            for (int kt = consumed; kt < issued; ++kt) mbar_wait(&full[kt % kCStages], (uint32_t)(kt / kCStages) & 1u);
        }
    }
    __syncwarp();
    const bool got = mbar_wait(done, 0);
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (!got) {
        if (lane == 0) atomicOr(err, 2u);
    } else {
        const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16);
        uint32_t v0[32], v1[32];
        tmem_ld32(taddr, v0);
        tmem_ld32(taddr + 32, v1);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int row = m0 + 32 * warp + lane;
        if (row < M && ep.out) {
            // bias + ReLU + BF16 on interior rows of the zero-halo layout, 0 elsewhere
            bool in = row < ep.R;
            if (in) {
                unsigned q = (unsigned)row;
                const int x = (int)(q % (unsigned)ep.Xp) - 1;
                q /= (unsigned)ep.Xp;
                const int y = (int)(q % (unsigned)ep.Yp) - 1;
                q /= (unsigned)ep.Yp;
                const int z = (int)(q % (unsigned)ep.Zp) - 1;
                in = x >= 0 && x < ep.X && y >= 0 && y < ep.Y && z >= 0 && z < ep.Z;
            }
            const float* bias = ep.bias + n0;
            uint4* dst = reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(ep.out) + (int64_t)row * N + n0);
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                uint32_t w[4];
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const int c = 8 * q + 2 * h;
                    const uint32_t* v = c < 32 ? v0 : v1;
                    const int cc = c & 31;
                    const float a = in ? fmaxf(__uint_as_float(v[cc]) + bias[c], 0.0f) : 0.0f;
                    const float b = in ? fmaxf(__uint_as_float(v[cc + 1]) + bias[c + 1], 0.0f) : 0.0f;
                    const __nv_bfloat162 pr = __floats2bfloat162_rn(a, b);
                    w[h] = *reinterpret_cast<const uint32_t*>(&pr);
                }
                dst[q] = make_uint4(w[0], w[1], w[2], w[3]);
            }
        } else if (row < M) {
            float4* dst = reinterpret_cast<float4*>(P + (int64_t)row * N + n0);
#pragma unroll
            for (int q = 0; q < 8; ++q)
                dst[q] = make_float4(__uint_as_float(v0[4 * q]), __uint_as_float(v0[4 * q + 1]),
                                     __uint_as_float(v0[4 * q + 2]), __uint_as_float(v0[4 * q + 3]));
#pragma unroll
            for (int q = 0; q < 8; ++q)
                dst[8 + q] = make_float4(__uint_as_float(v1[4 * q]), __uint_as_float(v1[4 * q + 1]),
                                         __uint_as_float(v1[4 * q + 2]), __uint_as_float(v1[4 * q + 3]));
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_once;
cudaError_t g_init = cudaErrorNotReady;

void init_once() {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
        g_init = e != cudaSuccess ? e : cudaErrorNotSupported;
        return;
    }
    g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    g_init = cudaFuncSetAttribute(umma_gemm_kernel<kModePlain>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)kSmemBytes);
    if (g_init == cudaSuccess)
        g_init = cudaFuncSetAttribute(umma_gemm_kernel<kModeWgrad>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)kSmemBytes);
    if (g_init == cudaSuccess)
        g_init = cudaFuncSetAttribute(umma_conv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCSmemBytes);
}

// 2-D tensor map of a K-contiguous BF16 operand: inner extent K, `rows`
// rows `ld` elements apart, boxes of 64 x box_rows with the 128-byte swizzle;
// elements outside the extents read as zero.
bool make_map(CUtensorMap* map, const void* base, int K, int rows, int ld, int box_rows) {
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kUK, (cuuint32_t)box_rows};
    const cuuint32_t es[2] = {1, 1};
    return g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

cudaError_t umma_gemm_init() {
    std::call_once(g_once, init_once);
    return g_init;
}

bool umma_gemm_supported(const void* A, int lda, const void* B, int ldb, int M, int N, int K, int S) {
    if (M < 1 || N < kUN || N % kUN || K < 1 || S < 1 || K % S || (K / S) % kUK) return false;
    if (lda % 8 || ldb % 8 || lda < K || ldb < K) return false;
    if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) & 15u) return false;
    return (M + kUM - 1) / kUM <= 65535 && S <= 65535;
}

cudaError_t umma_gemm_tn(const void* A, int lda, const void* B, int ldb, float* P, int M, int N, int K, int S,
                         unsigned int* err, cudaStream_t st) {
    cudaError_t e = umma_gemm_init();
    if (e != cudaSuccess) return e;
    if (!umma_gemm_supported(A, lda, B, ldb, M, N, K, S)) return cudaErrorInvalidValue;
    CUtensorMap ma, mb;
    if (!make_map(&ma, A, K, M, lda, kUM) || !make_map(&mb, B, K, N, ldb, kUN)) return cudaErrorInvalidValue;
    const dim3 grid(N / kUN, (M + kUM - 1) / kUM, S);
    umma_gemm_kernel<kModePlain><<<grid, 128, kSmemBytes, st>>>(ma, mb, mb, mb, P, M, N, K / S, err, ConvTaps{});
    return cudaGetLastError();
}

cudaError_t umma_conv_gemm(const void* x, int rows, int C, const void* W, int N, const ConvTaps& taps, float* P,
                           unsigned int* err, cudaStream_t st, const ConvEpilogue* ep) {
    cudaError_t e = umma_gemm_init();
    if (e != cudaSuccess) return e;
    if (rows < 1 || C < kUK || C % kUK || N < kUN || N % kUN || taps.per_tap != C / kUK ||
        (rows + kUM - 1) / kUM > 65535 || ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(W)) & 15u))
        return cudaErrorInvalidValue;
    for (int g = 0; g < 9; ++g) {   // the three taps of a row lie in one window: offsets o, o + 1, o + 2
        const int a = taps.off[3 * g], b = taps.off[3 * g + 1], c = taps.off[3 * g + 2];
        const int lo = a < b ? (a < c ? a : c) : (b < c ? b : c);
        if (a - lo > 2 || b - lo > 2 || c - lo > 2 || a == b || b == c || a == c) return cudaErrorInvalidValue;
    }
    CUtensorMap ma, mb;
    if (!make_map(&ma, x, C, rows, C, kCRows) || !make_map(&mb, W, 27 * C, N, 27 * C, kUN))
        return cudaErrorInvalidValue;
    const dim3 grid(N / kUN, (rows + kUM - 1) / kUM, 1);
    if (ep && (!ep->bias || !ep->out || (reinterpret_cast<uintptr_t>(ep->out) & 15u) || ep->Xp < 1 || ep->Yp < 1 ||
               ep->Zp < 1))
        return cudaErrorInvalidValue;
    umma_conv_kernel<<<grid, 128, kCSmemBytes, st>>>(ma, mb, P, rows, N, C / kUK, err, taps,
                                                     ep ? *ep : ConvEpilogue{});
    return cudaGetLastError();
}

cudaError_t umma_wgrad_gemm(const void* dzT, int N, const void* const xT[3], int C, int rows, int S,
                            const ConvTaps& taps, float* P, unsigned int* err, cudaStream_t st) {
    cudaError_t e = umma_gemm_init();
    if (e != cudaSuccess) return e;
    uintptr_t al = reinterpret_cast<uintptr_t>(dzT);
    for (int j = 0; j < 3; ++j) al |= reinterpret_cast<uintptr_t>(xT[j]);
    bool ok = N >= kUN && N % kUN == 0 && C >= 64 && C % 64 == 0 && rows >= kUK && rows % 8 == 0 && S >= 1 &&
              rows % S == 0 && (rows / S) % kUK == 0 && taps.per_tap == C && S <= 65535 && !(al & 15u);
    for (int t = 0; t < 27 && ok; ++t) ok = taps.off[t] % 8 == 0;
    if (!ok) return cudaErrorInvalidValue;
    CUtensorMap ma[3], mb;
    for (int j = 0; j < 3; ++j)
        if (!make_map(&ma[j], xT[j], rows, C, rows, kUM / 2)) return cudaErrorInvalidValue;
    if (!make_map(&mb, dzT, rows, N, rows, kUN)) return cudaErrorInvalidValue;
    const int M = 27 * C;
    const dim3 grid(N / kUN, (M + kUM - 1) / kUM, S);
    umma_gemm_kernel<kModeWgrad><<<grid, 128, kSmemBytes, st>>>(ma[0], mb, ma[1], ma[2], P, M, N, rows / S, err,
                                                                taps);
    return cudaGetLastError();
}

}  // namespace lbms
