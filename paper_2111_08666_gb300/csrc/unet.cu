// Learned warm start: a U-Net that predicts the phase field of the next
// quasi-static equilibrium of a drainage step from (solid indicator,
// wettability xi, current phase field, pressure step), trained on LBM
// equilibria and used to initialise the next LBM relaxation.
//
// Network (levels L, base channels C0, C_l = C0 2^l), NHWC, BF16 storage of
// weights and activations, FP32 accumulation and FP32 master weights:
//   encoder l:  conv3x3 + ReLU, conv3x3 + ReLU = e_l; 2x2 average pooling
//   decoder l:  concat(e_l, nearest-upsample(d_{l+1})) (skip first),
//               conv3x3 + ReLU, conv3x3 + ReLU = d_l   (d_{L-1} = e_{L-1})
//   head:       1x1 conv C0 -> 1, tanh
// Loss: mean over the masked (fluid) pixels of (phi_hat - phi)^2; Adam.
//
// The three passes of every 3x3 convolution are implicit GEMMs on the
// tensor cores, BF16 x BF16 -> FP32:
//   forward  C[pixel][co] = sum_(tap,ci) X[pixel + d_tap][ci] W[co][tap][ci]
//   dgrad    C[pixel][ci] = sum_(tap,co) dZ[pixel - d_tap][co] W[co][tap][ci]
//   wgrad    C[co][ci]    = sum_pixel dZ[pixel][co] X[pixel + d_tap][ci]  (per tap)
// with operands gathered into shared memory by cp.async (zero fill at the
// image border; the decoder's concat and upsampling are folded into the
// gather).  All three run on tcgen05 with accumulators in tensor memory:
// for widths that are multiples of 128 as persistent row-tile kernels fed
// by tensor copies (conv_row_kernel, wgrad_row_kernel), else as a per-pixel
// gather kernel (forward, dgrad) and mma.sync m16n8k16 (wgrad).  Pooling,
// the head, the loss and Adam are elementwise kernels.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "async_copy.cuh"
#include "lbm.cuh"

using namespace mclbm;

namespace {

using bf16 = __nv_bfloat16;

// ---------------------------------------------------------------------------
// PTX helpers
// ---------------------------------------------------------------------------
// 16-byte copy global -> shared, or zeros when !valid (a plain shared store:
// the zero-fill form of cp.async was seen to move twice the bytes from L2)
__device__ __forceinline__ void cp_async16(void *dst, const void *src, bool valid) {
    if (valid)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
    else
        *reinterpret_cast<uint4 *>(dst) = make_uint4(0u, 0u, 0u, 0u);
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}
__device__ __forceinline__ void ldsm4t(uint32_t r[4], const void *p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}
// c += a (16x16, row) * b (16x8, col)
__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// 128-byte shared rows (64 BF16) of 8 chunks
__device__ __forceinline__ int sw128(int row, int chunk) { return row * 128 + ((chunk ^ (row & 7)) << 4); }

// ---------------------------------------------------------------------------
// Forward and data-gradient convolution: C[m][n] = sum_k A[m][k] B[n][k],
// m = pixel (b, y, x), k = (tap, channel), n = output channel.
// ---------------------------------------------------------------------------
struct ConvArgs {
    const bf16 *x0, *x1;  // gathered input: x0 [B][H][W][c0]; x1 [B][H/2][W/2][c1] upsampled,
    int c0, c1;           // or x1 [B][H][W][c1] when x1_full
    int x1_full;
    int B, H, W, M;       // M = B H W
    int sign;             // +1: taps read pixel + d; -1: pixel - d
    const bf16 *w;        // [N][9][c0 + c1]
    const bf16 *wp;       // w packed for the row kernel with N tile row_bn(N), or null
    int N;
    const float *bias;    // [N] or null
    bf16 *ybf;            // ReLU(C + bias) as BF16 [M][N], or null
    bf16 *yup;            // the same, nearest-upsampled to [B][2H][2W][N] (the next decoder's input), or null
    float *yf;            // C as FP32 [M][N], or null
    // concat data gradient (row kernel only; 0 = off): columns n < split_cs
    // go to yf as [M][split_cs], the others summed over each horizontal pixel
    // pair to yh [B][H][W/2][N - split_cs] (the first half of the
    // nearest-upsampling backward)
    int split_cs;
    float *yh;
    // data gradient into a ReLU layer: C masked by the forward activation
    // mask_h > 0 ([M][N]) as BF16 into ydz, or null
    const bf16 *mask_h;
    bf16 *ydz;
    int *err;             // set when a bounded wait gives up
};

// ---------------------------------------------------------------------------
// The same convolution on the 5th-generation tensor cores: a CTA of four
// warps owns 128 pixels x BN channels.  Per k-chunk of 32 (one tap, 32
// channels) every thread gathers one pixel row of A and (part of) the B rows
// with cp.async into shared memory in the K-major core-matrix layout (8 rows
// x 16 bytes per core matrix, no swizzle); one thread issues two
// tcgen05.mma (M = 128, N = BN, K = 16, BF16 x BF16 -> FP32) into a tensor-
// memory accumulator and commits them to the stage's mbarrier, so the next
// chunk's gather overlaps the MMAs (two stages).  The four warps then read
// their 32 accumulator lanes (pixels) with tcgen05.ld for the epilogue.
// ---------------------------------------------------------------------------
constexpr int TBM = 128, TBK = 32;

// shared-memory matrix descriptor: K-major, no swizzle; lbo = byte offset
// between core matrices adjacent in K, sbo = between 8-row groups
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3fffu) | (uint64_t)((lbo >> 4) & 0x3fffu) << 16 |
           (uint64_t)((sbo >> 4) & 0x3fffu) << 32 | (uint64_t)1 << 46;
}

// the same for the 64-byte-swizzled K-major layout (rows of 64 bytes, the
// 16-byte chunk c of a row stored at c ^ (address bits 7-8), as the tensor
// copy writes it): sbo between 8-row groups.  The swizzle follows the
// absolute shared-memory address, so a start moved by whole rows needs no
// base offset (measured: base offset 0 is exact for every row shift, the
// start's phase in that field is not)
__device__ __forceinline__ uint64_t umma_desc_sw64(uint32_t saddr, uint32_t sbo) {
    return (uint64_t)((saddr >> 4) & 0x3fffu) | (uint64_t)1 << 16 | (uint64_t)((sbo >> 4) & 0x3fffu) << 32 |
           (uint64_t)1 << 46 | (uint64_t)4 << 61;
}

// instruction descriptor: BF16 A and B (K-major), FP32 accumulator, M x N
__host__ __device__ constexpr uint32_t umma_idesc(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// epilogue of one pixel row and 16 accumulator columns n..n+15: FP32 C, or
// BF16 ReLU(C + bias) with bias = the 16 values for these columns (or null)
__device__ __forceinline__ void store_row16(const ConvArgs &a, size_t row, int n, const uint32_t r[16],
                                            const float *bias) {
    float v[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = __uint_as_float(r[k]);
    if (a.ydz) {
        const uint4 *hp = reinterpret_cast<const uint4 *>(a.mask_h + row * a.N + n);
        const uint4 h0 = hp[0], h1 = hp[1];
        const uint32_t hw[8] = {h0.x, h0.y, h0.z, h0.w, h1.x, h1.y, h1.z, h1.w};
        uint32_t o[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float2 hf = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&hw[k]));
            __nv_bfloat162 q = __floats2bfloat162_rn(hf.x > 0.f ? v[2 * k] : 0.f, hf.y > 0.f ? v[2 * k + 1] : 0.f);
            o[k] = *reinterpret_cast<uint32_t *>(&q);
        }
        uint4 *d = reinterpret_cast<uint4 *>(a.ydz + row * a.N + n);
        d[0] = make_uint4(o[0], o[1], o[2], o[3]);
        d[1] = make_uint4(o[4], o[5], o[6], o[7]);
    }
    if (a.yf && a.split_cs) {
        // n is the same in the whole warp and the split falls on a 16-column
        // boundary; lanes 2j, 2j + 1 hold pixels 2x, 2x + 1 of one row (row
        // tiles start at multiples of 128)
        if (n < a.split_cs) {
            float4 *d = reinterpret_cast<float4 *>(a.yf + row * a.split_cs + n);
#pragma unroll
            for (int k = 0; k < 4; ++k) d[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
        } else {
#pragma unroll
            for (int k = 0; k < 16; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], 1);
            if (!(row & 1)) {
                float4 *d = reinterpret_cast<float4 *>(a.yh + (row >> 1) * (size_t)(a.N - a.split_cs) +
                                                       (n - a.split_cs));
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    d[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
            }
        }
    } else if (a.yf) {
        float4 *d = reinterpret_cast<float4 *>(a.yf + row * a.N + n);
#pragma unroll
        for (int k = 0; k < 4; ++k) d[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
    }
    if (a.ybf) {
        __nv_bfloat162 h[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            float v0 = v[2 * k], v1 = v[2 * k + 1];
            if (bias) {
                v0 += bias[2 * k];
                v1 += bias[2 * k + 1];
            }
            h[k] = __floats2bfloat162_rn(fmaxf(v0, 0.f), fmaxf(v1, 0.f));
        }
        uint4 *d = reinterpret_cast<uint4 *>(a.ybf + row * a.N + n);
        d[0] = *reinterpret_cast<const uint4 *>(&h[0]);
        d[1] = *reinterpret_cast<const uint4 *>(&h[4]);
        if (a.yup) {
            const int x = (int)(row % a.W);
            const size_t t = row / a.W;
            const int y = (int)(t % a.H);
            const size_t b = t / a.H;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                uint4 *u = reinterpret_cast<uint4 *>(
                    a.yup + (((b * 2 * a.H + 2 * y + (k >> 1)) * 2 * a.W) + 2 * x + (k & 1)) * a.N + n);
                u[0] = *reinterpret_cast<const uint4 *>(&h[0]);
                u[1] = *reinterpret_cast<const uint4 *>(&h[4]);
            }
        }
    }
}

template <int BN>
__global__ void __launch_bounds__(128) conv_tc_kernel(const ConvArgs a) {
    constexpr int A_BYTES = TBM * TBK * 2, B_BYTES = BN * TBK * 2;
    constexpr int STAGE = A_BYTES + B_BYTES;
    constexpr uint32_t COLS = BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256;  // TMEM columns
    static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "UMMA N for M = 128");
    static_assert(TBK == 32, "four 16-byte pieces per row and chunk");
    extern __shared__ __align__(1024) unsigned char smem[];
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem + 2 * STAGE);  // [2]
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * TBM, n0 = blockIdx.y * BN;
    const int K0 = a.c0 + a.c1;
    const int kchunks = K0 / TBK;
    const int ksteps = 9 * kchunks;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    // A rows (pixels) this thread gathers: rows (tid >> 2) + 32 i, 16-byte
    // piece q = tid & 3 of each chunk, so that four neighbouring threads read
    // one pixel's 64 contiguous bytes
    const int q = tid & 3;
    int ax[4], ay[4], ab[4];
    bool am[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + (tid >> 2) + 32 * i;
        am[i] = m < a.M;
        const int mm = am[i] ? m : 0;
        ax[i] = mm % a.W;
        ay[i] = (mm / a.W) % a.H;
        ab[i] = mm / (a.W * a.H);
    }
    auto off = [](int row, int qq) { return ((row >> 3) * (TBK / 8) + qq) * 128 + (row & 7) * 16; };

    auto load = [&](int ks, int st) {
        unsigned char *As = smem + st * STAGE, *Bs = As + A_BYTES;
        const int tap = ks / kchunks, kc = ks - tap * kchunks;
        const int dy = (tap / 3 - 1) * a.sign, dx = (tap % 3 - 1) * a.sign;
        const int ci = kc * TBK + q * 8;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int yy = ay[i] + dy, xx = ax[i] + dx;
            const bool v = am[i] && yy >= 0 && yy < a.H && xx >= 0 && xx < a.W;
            const bf16 *src = a.x0;
            if (v) {
                if (ci < a.c0)
                    src = a.x0 + ((size_t)(ab[i] * a.H + yy) * a.W + xx) * a.c0 + ci;
                else if (a.x1_full)
                    src = a.x1 + ((size_t)(ab[i] * a.H + yy) * a.W + xx) * a.c1 + (ci - a.c0);
                else
                    src = a.x1 + ((size_t)(ab[i] * (a.H >> 1) + (yy >> 1)) * (a.W >> 1) + (xx >> 1)) * a.c1 +
                          (ci - a.c0);
            }
            cp_async16(As + off((tid >> 2) + 32 * i, q), src, v);
        }
#pragma unroll
        for (int n = tid >> 2; n < BN; n += 32) {
            const bool vb = n0 + n < a.N;
            const bf16 *src = vb ? a.w + ((size_t)(n0 + n) * 9 + tap) * K0 + ci : a.w;
            cp_async16(Bs + off(n, q), src, vb);
        }
        cp_async_commit();
    };

    bool bad = false;
    for (int ks = 0; ks < ksteps && !bad; ++ks) {
        const int st = ks & 1;
        if (ks >= 2) {
            // the MMAs of chunk ks - 2 have read stage st
            const bool ok = mbar_wait(&bar[st], ((ks - 2) >> 1) & 1, WAIT_LIMIT_NS);
            if (__syncthreads_or(!ok)) {
                bad = true;
                break;
            }
            tc_fence_after();
        }
        load(ks, st);
        cp_async_wait<0>();
        fence_proxy_async();  // the gathered tiles, for the tensor cores' (async) reads
        tc_fence_before();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t As = smem_u32(smem + st * STAGE), Bs = As + A_BYTES;
#pragma unroll
            for (int j = 0; j < TBK / 16; ++j) {
                const uint64_t ad = umma_desc(As + j * 256, 128, (TBK / 8) * 128);
                const uint64_t bd = umma_desc(Bs + j * 256, 128, (TBK / 8) * 128);
                const uint32_t acc = (ks > 0 || j > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(umma_idesc(TBM, BN)), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(&bar[st]))
                         : "memory");
        }
    }
    if (!bad && ksteps > 0) {
        const int last = ksteps - 1;
        const bool ok = mbar_wait(&bar[last & 1], (last >> 1) & 1, WAIT_LIMIT_NS);
        bad = __syncthreads_or(!ok);
    }
    tc_fence_after();
    if (bad) {
        if (tid == 0 && a.err) atomicExch(a.err, 1);
        // give in-flight MMAs a last, short chance before the memory is freed
        mbar_wait(&bar[0], 0, DRAIN_LIMIT_NS);
    } else {
        // epilogue: warp w reads accumulator lanes 32w..32w+31 (its pixels)
        const int row = m0 + warp * 32 + lane;
#pragma unroll 1
        for (int c = 0; c < BN; c += 16) {
            uint32_t r[16];
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                  "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                  "=r"(r[15])
                : "r"(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            const int n = n0 + c;
            if (row < a.M && n < a.N) store_row16(a, (size_t)row, n, r, a.bias ? a.bias + n : nullptr);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(COLS) : "memory");
    }
}

// ---------------------------------------------------------------------------
// Row-tile variant for images whose width is a multiple of 128, persistent
// and pipelined.  A tile is 128 consecutive pixels of one image row.  Per
// chunk of 32 input channels the tile needs the 3 x 130 halo of its row
// segment and the nine taps' weights.  The halo is stored pixel-major, 64
// bytes (32 channels) per pixel in the 64-byte-swizzled K-major layout of
// the tensor cores; the A operand of tap (dy, dx) is the same halo read
// through a descriptor whose start moves by dy rows and dx pixels (the
// descriptor's base offset carries the start's phase in the swizzle), so each
// input pixel crosses L2 -> shared memory about 3 x 130 / 128 times instead
// of nine.
//
// Copies: the halo of the directly read input comes by one tiled tensor load
// (box 32 channels x 130 pixels x 3 rows, swizzled, zero fill outside the
// image); the weights, pre-packed in global memory in exactly the shared
// layout (per N tile and chunk; K-major core matrices, no swizzle), by one
// bulk copy.  The upsampled input of a decoder concat comes as the coarse
// 2 x 66 pixels it needs (one tensor load) and is expanded into the halo by
// all threads (nearest upsampling is a gather the tensor copy cannot
// express).
//
// A CTA owns one N tile and walks its tiles as a sequence of jobs (tile,
// chunk) through a ring of S stages filled S - 1 jobs ahead.  When all
// chunks' weights fit they are loaded once per CTA and the stages carry
// halos only.  The accumulator is double-buffered in tensor memory: the
// epilogue of tile i - 1 runs while the MMAs of tile i execute.
// ---------------------------------------------------------------------------
constexpr int RW = 128, RHALO = RW + 2;
constexpr int RHALO_TX = 3 * RHALO * 64;  // halo of one chunk: 3 rows x 130 pixels x 64 bytes
constexpr int RA_BYTES = 25600;           // ... rounded up to 1024 (swizzled tensor-copy destination)
static_assert(RA_BYTES >= RHALO_TX && RA_BYTES % 1024 == 0, "halo area");

struct RowPlan {
    int wres;    // all chunks' weights resident (1) or streamed per job (0)
    int ux;      // the input has an upsampled part (stages carry its coarse staging)
    int stages;  // 2..4
    int smem;    // dynamic shared memory bytes
};

// coarse staging of an upsampled chunk: 2 rows x 66 pixels x 64 bytes,
// rounded up to 1024 (keeps the stages aligned)
constexpr int RU_TX = 2 * 66 * 64;
constexpr int RU_BYTES = 9216;
static_assert(RU_BYTES >= RU_TX && RU_BYTES % 1024 == 0, "staging area");

__host__ __device__ inline int row_weight_bytes(int BN, int kchunks) { return 9 * BN * 64 * kchunks; }
__host__ __device__ inline int row_stage_bytes(int BN, int wres, int ux) {
    return RA_BYTES + (ux ? RU_BYTES : 0) + (wres ? 0 : 9 * BN * 64);
}
__host__ __device__ inline int row_smem(int BN, int kchunks, int wres, int ux, int stages) {
    return (wres ? row_weight_bytes(BN, kchunks) : 0) + stages * row_stage_bytes(BN, wres, ux) + 256 + 4 * BN;
}

// N tile of the row kernel for N output channels (0: none)
__host__ __device__ inline int row_bn(int N) {
    if (N == 32 || N == 64) return N;
    if (N % 128 == 0) return 128;
    if (N % 96 == 0) return 96;
    if (N % 64 == 0) return 64;
    if (N % 32 == 0) return 32;
    return 0;
}

__device__ __forceinline__ void tma_load_4d(void *dst, const void *tmap, int c0, int c1, int c2, int c3,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}

// Roles (warp-specialized, mbarriers only in the steady state):
//   warp 0        producer: tensor/bulk copies of job j into stage j % S once
//                 the MMAs of job j - S have read that stage
//   warp 1        MMA issue: waits for job j's data (and expansion), for the
//                 accumulator buffer of tile i (its epilogue two tiles back),
//                 issues the 18 MMAs of the chunk and commits
//   warps 2-5     expansion of upsampled chunks into the halo (an arrival on
//                 expanded[st] for every job keeps the phases in step)
//   warps 6-9     epilogue: accumulator -> registers (tcgen05.ld), frees the
//                 buffer, bias + ReLU + stores (warp w reads lanes 32 (w % 4)..)
// bounded wait whose polls let the hardware suspend the thread until the
// phase completes (up to 0.1 ms a poll), so that waiting roles take no issue
// slots from the working ones
__device__ __forceinline__ bool mbar_test_sleep(uint64_t *bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity), "r"(100000u)
        : "memory");
    return done != 0;
}
__device__ __forceinline__ bool mbar_wait_sleep(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_test_sleep(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_test_sleep(bar, parity))
        if (global_ns() - t0 > limit_ns) return false;
    return true;
}

constexpr int ROW_THREADS = 320;
constexpr int ROW_EXP = 128;  // expansion threads

template <int BN>
__global__ void __launch_bounds__(ROW_THREADS, 1)
    conv_row_kernel(const ConvArgs a, const RowPlan plan, const bf16 *__restrict__ wp,
                    const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tmu) {
    constexpr uint32_t COLS = 2 * BN <= 64 ? 64 : 2 * BN <= 128 ? 128 : 256;  // two accumulators
    constexpr int WTILE = 9 * BN * 64;                                        // weights of one chunk
    static_assert(BN % 32 == 0 && BN >= 32 && BN <= 128, "UMMA N for M = 128");
    extern __shared__ __align__(1024) unsigned char smem[];
    if (smem_u32(smem) & 1023u) {  // the swizzled copies need 1024-byte-aligned stages
        if (threadIdx.x == 0 && a.err) atomicExch(a.err, 2);
        return;
    }
    const int K0 = a.c0 + a.c1;
    const int kchunks = K0 / 32;
    const int S = plan.stages, wres = plan.wres;
    const int WB = wres ? row_weight_bytes(BN, kchunks) : 0;
    const int STG = row_stage_bytes(BN, wres, plan.ux);
    unsigned char *wsm = smem;       // resident weights [kc][tap][core-matrix layout]
    unsigned char *stg = smem + WB;  // S stages: halo (+ coarse staging) (+ weights when streamed)
    uint64_t *full = reinterpret_cast<uint64_t *>(stg + S * STG);  // [4] copies landed
    uint64_t *done = full + 4;                                     // [4] MMAs have read the stage
    uint64_t *expd = full + 8;                                     // [4] halo complete (expansion)
    uint64_t *accf = full + 12;                                    // [2] accumulator complete
    uint64_t *acce = full + 14;                                    // [2] accumulator read out
    uint64_t *wfull = full + 16, *drain = full + 17;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(full + 18);
    int *flag = reinterpret_cast<int *>(full + 19);  // some role gave up waiting
    float *sbias = reinterpret_cast<float *>(full + 20);  // this N tile's biases [BN]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntn = a.N / BN;
    const int nt = blockIdx.x % ntn, n0 = nt * BN;
    const int tile0 = blockIdx.x / ntn, tstride = gridDim.x / ntn;
    const int segs = a.W / RW;
    const int ntiles = a.M / RW;
    const int my_tiles = tile0 < ntiles ? (ntiles - tile0 + tstride - 1) / tstride : 0;
    const int njobs = my_tiles * kchunks;
    const bf16 *wnt = wp + (size_t)nt * kchunks * (WTILE / 2);  // this N tile's packed weights

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int k = 0; k < 4; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&done[k], 1);
            mbar_init(&expd[k], ROW_EXP / 32);  // one arrival per expansion warp
        }
        for (int k = 0; k < 2; ++k) {
            mbar_init(&accf[k], 1);
            mbar_init(&acce[k], 4);
        }
        mbar_init(wfull, 1);
        mbar_init(drain, 1);
        *flag = 0;
        fence_mbar_init();
    }
    if (a.bias)
        for (int c = tid; c < BN; c += ROW_THREADS) sbias[c] = a.bias[n0 + c];
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    struct Where {
        int x0, y, b;
    };
    auto where = [&](int i) {
        const int t = tile0 + i * tstride;
        return Where{(t % segs) * RW, (t / segs) % a.H, t / (segs * a.H)};
    };
    auto give_up = [&]() {
        *(volatile int *)flag = 1;
        if (a.err) atomicExch(a.err, 1);
    };
    auto stopped = [&]() { return *(volatile int *)flag != 0; };

    if (warp == 0) {
        // ---------------- producer ----------------
        if (lane == 0) {
            if (wres && njobs > 0) {
                mbar_expect_tx(wfull, WB);
                bulk_g2s(wsm, wnt, WB, wfull);
            }
            int j = 0;
            for (; j < njobs && !stopped(); ++j) {
                const int st = j % S;
                if (j >= S && !mbar_wait_sleep(&done[st], ((j - S) / S) & 1, WAIT_LIMIT_NS)) {
                    give_up();
                    break;
                }
                const int i = j / kchunks, kc = j - i * kchunks;
                const Where w = where(i);
                unsigned char *As = stg + st * STG;
                const bool direct = kc * 32 < a.c0;
                mbar_expect_tx(&full[st], (direct || a.x1_full ? RHALO_TX : RU_TX) + (wres ? 0 : WTILE));
                if (direct)
                    tma_load_4d(As, &tmx, kc * 32, w.x0 - 1, w.y - 1, w.b, &full[st]);
                else if (a.x1_full)
                    tma_load_4d(As, &tmu, kc * 32 - a.c0, w.x0 - 1, w.y - 1, w.b, &full[st]);
                else
                    tma_load_4d(As + RA_BYTES, &tmu, kc * 32 - a.c0, (w.x0 >> 1) - 1, (w.y - 1) >> 1, w.b,
                                &full[st]);
                if (!wres)
                    bulk_g2s(As + RA_BYTES + (plan.ux ? RU_BYTES : 0), wnt + (size_t)kc * (WTILE / 2), WTILE,
                             &full[st]);
            }
            // copies in flight land before the CTA may end: the last S issued
            for (int jb = j - 1; jb >= 0 && jb >= j - S; --jb) mbar_wait_sleep(&full[jb % S], (jb / S) & 1, DRAIN_LIMIT_NS);
            if (wres && njobs > 0) mbar_wait_sleep(wfull, 0, DRAIN_LIMIT_NS);
        }
    } else if (warp == 1) {
        // ---------------- MMA issue ----------------
        if (lane == 0) {
            bool ok = !(wres && njobs > 0) || mbar_wait_sleep(wfull, 0, WAIT_LIMIT_NS);
            if (!ok) give_up();
            // this thread paces the tensor core: per job it only waits
            // (spinning, for the shortest hand-over), adds to two descriptors
            // and issues; stage, phase, tile and chunk advance incrementally
            uint32_t xpar = 0;  // bit st: parity of the upsampled-coarse jobs seen on stage st (expd phases)
            const uint64_t ad_stg = umma_desc_sw64(smem_u32(stg), 512);
            const uint64_t bd_w = wres ? umma_desc(smem_u32(wsm), 128, 512)
                                       : umma_desc(smem_u32(stg) + RA_BYTES + (plan.ux ? RU_BYTES : 0), 128, 512);
            // the taps' A offsets (64-byte pixels of the 130-wide halo; the data
            // gradient runs the taps mirrored)
            const int tap_dir = a.sign;
            int st = 0, i = 0, kc = 0;
            uint32_t ph = 0;
            for (int j = 0; ok && j < njobs && !stopped(); ++j) {
                ok = mbar_wait(&full[st], ph, WAIT_LIMIT_NS);
                if (ok && plan.ux && kc * 32 >= a.c0) {
                    ok = mbar_wait(&expd[st], (xpar >> st) & 1u, WAIT_LIMIT_NS);
                    xpar ^= 1u << st;
                }
                if (ok && kc == 0 && i >= 2) ok = mbar_wait(&acce[i & 1], ((i - 2) >> 1) & 1, WAIT_LIMIT_NS);
                if (!ok) {
                    give_up();
                    break;
                }
                tc_fence_after();
                // descriptors of the stage's operands; a start moved by b bytes
                // adds b / 16 to the address field (no carry: below 256 KB)
                const uint32_t d = tmem + (uint32_t)((i & 1) * BN);
                const uint64_t ad0 = ad_stg + (uint64_t)((st * STG) >> 4);
                const uint64_t bd0 = bd_w + (uint64_t)(((wres ? kc * WTILE : st * STG)) >> 4);
#pragma unroll
                for (int tap = 0; tap < 9; ++tap) {
                    const int dy = (tap / 3 - 1) * tap_dir, dx = (tap % 3 - 1) * tap_dir;
                    const int aoff = ((dy + 1) * RHALO + dx + 1) * 64;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const uint64_t ad = ad0 + (uint64_t)((aoff + h * 32) / 16);
                        const uint64_t bd = bd0 + (uint64_t)((tap * BN * 64 + h * 256) / 16);
                        const uint32_t accum = (kc > 0 || tap > 0 || h > 0) ? 1u : 0u;
                        asm volatile(
                            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
                            "l"(ad), "l"(bd), "r"(umma_idesc(RW, BN)), "r"(accum)
                            : "memory");
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(&done[st]))
                             : "memory");
                if (kc == kchunks - 1)
                    asm volatile(
                        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                            smem_u32(&accf[i & 1]))
                        : "memory");
                if (++st == S) {
                    st = 0;
                    ph ^= 1u;
                }
                if (++kc == kchunks) {
                    kc = 0;
                    ++i;
                }
            }
            // every MMA issued has completed before the tensor memory is freed
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(drain))
                         : "memory");
            if (!mbar_wait_sleep(drain, 0, WAIT_LIMIT_NS)) give_up();
        }
    } else if (warp < 6) {
        // ---------------- expansion (128 threads) ----------------
        // expands the jobs of an upsampled-coarse chunk; expd[st] completes once
        // per such job on stage st.  It follows done[st] for every job, so that
        // no parity wait here is ever two phases ahead (a wait for parity P
        // passes whenever the barrier is not in a phase of parity P)
        const int et = tid - 64, qq = et & 3;
        int st = 0, i = 0, kc = 0;  // advance incrementally, as in the MMA loop
        uint32_t ph = 0;
        for (int j = 0; plan.ux && j < njobs && !stopped(); ++j) {
            // the stage's previous job has been read by its MMAs
            if (j >= S && !mbar_wait_sleep(&done[st], ph ^ 1u, WAIT_LIMIT_NS)) {
                give_up();
                break;
            }
            if (kc * 32 >= a.c0) {
                // this job's coarse rows have landed
                if (!mbar_wait_sleep(&full[st], ph, WAIT_LIMIT_NS)) {
                    give_up();
                    break;
                }
                // nearest upsampling: halo pixel (r, p) takes coarse pixel
                // ((y + r - 1) >> 1, (x0 + p - 1) >> 1); relative to the staged
                // rows that is (cr(r), (p + 1) >> 1) since x0 is even.  Stages
                // are 1024-byte aligned, so the 64-byte swizzle of halo pixel
                // pix is (pix / 2) & 3
                const int y = where(i).y;
                unsigned char *As = stg + st * STG;
                const unsigned char *U = As + RA_BYTES;
                for (int r = 0; r < 3; ++r) {
                    const int cr = ((y + r - 1) >> 1) - ((y - 1) >> 1);
                    for (int p = et >> 2; p < RHALO; p += ROW_EXP / 4) {
                        const int pix = r * RHALO + p;
                        *reinterpret_cast<uint4 *>(As + pix * 64 + ((qq ^ ((pix >> 1) & 3)) << 4)) =
                            *reinterpret_cast<const uint4 *>(U + (cr * 66 + ((p + 1) >> 1)) * 64 + qq * 16);
                    }
                }
                fence_proxy_async();  // each thread's generic writes, for the tensor cores' reads
                __syncwarp();
                if (lane == 0) mbar_arrive(&expd[st]);
            }
            if (++st == S) {
                st = 0;
                ph ^= 1u;
            }
            if (++kc == kchunks) {
                kc = 0;
                ++i;
            }
        }
    } else {
        // ---------------- epilogue (128 threads) ----------------
        const int ew = warp & 3;  // accumulator lanes 32 ew .. 32 ew + 31
        for (int i = 0; i < my_tiles && !stopped(); ++i) {
            if (!mbar_wait_sleep(&accf[i & 1], (i >> 1) & 1, WAIT_LIMIT_NS)) {
                give_up();
                break;
            }
            tc_fence_after();
            const uint32_t acc = tmem + (uint32_t)((i & 1) * BN) + ((uint32_t)(ew * 32) << 16);
            const size_t row = (size_t)(tile0 + i * tstride) * RW + ew * 32 + lane;
#pragma unroll 1
            for (int c0 = 0; c0 < BN; c0 += 32) {
                uint32_t r[32];
#pragma unroll
                for (int c = 0; c < 32; c += 16) {
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
                        "%15}, [%16];"
                        : "=r"(r[c]), "=r"(r[c + 1]), "=r"(r[c + 2]), "=r"(r[c + 3]), "=r"(r[c + 4]), "=r"(r[c + 5]),
                          "=r"(r[c + 6]), "=r"(r[c + 7]), "=r"(r[c + 8]), "=r"(r[c + 9]), "=r"(r[c + 10]),
                          "=r"(r[c + 11]), "=r"(r[c + 12]), "=r"(r[c + 13]), "=r"(r[c + 14]), "=r"(r[c + 15])
                        : "r"(acc + (uint32_t)(c0 + c)));
                }
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (c0 + 32 >= BN) {
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&acce[i & 1]);  // the buffer may take tile i + 2
                }
                store_row16(a, row, n0 + c0, r, a.bias ? sbias + c0 : nullptr);
                store_row16(a, row, n0 + c0 + 16, r + 16, a.bias ? sbias + c0 + 16 : nullptr);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(COLS) : "memory");
    }
}

// ---------------------------------------------------------------------------
// Weight gradient on the tensor cores, per tap (widths that are multiples of
// 128 with the shared-tap kernel below switched off; it cross-checks that one):
//   dW[co][tap][ci] = sum_p dZ[p][co] X[p + d_tap][ci]
// a GEMM per tap with M = co (a tile of 128, rows past co zero), N = 32
// input channels, K = pixels.  Both operands stay pixel-major as the forward
// pass wrote them, read MN-major: dZ of one row tile (128 pixels x 128
// channels: two 64-channel boxes, 128-byte swizzle) and the same 3 x 130
// halo of X as the forward convolution (64-byte swizzle), whose K start
// moves by the tap's offset.  A CTA owns one (co tile, 32-channel chunk) and
// a strided set of row tiles; its nine accumulators (9 x 32 tensor-memory
// columns) sum over all of them and are added to dW with FP32 atomics at the
// end (split K across CTAs).  Roles as in the forward kernel: producer,
// MMA, expansion (coarse upsampled chunks), epilogue warps.
// ---------------------------------------------------------------------------
struct WgradRowArgs {
    const bf16 *dz;       // [B][H][W][co]
    int co;
    const bf16 *x0, *x1;  // the layer's input, as in ConvArgs (x1 coarse, upsampled)
    int c0, c1;
    int B, H, W, M;
    float *dw;            // [co][9][c0 + c1], accumulated into
    float *part;          // shared-tap kernel: per-CTA partial sums [grid][32][9][32]
    int *err;
};
constexpr int WG_A_ATOM = 128 * 128;  // 128 pixels x 64 channels x 2 bytes
constexpr int WG_A_BYTES = 2 * WG_A_ATOM;

__host__ __device__ inline int wg_stage_bytes(int ux) { return WG_A_BYTES + RA_BYTES + (ux ? RU_BYTES : 0); }

// MN-major shared-memory descriptor, swizzled (layout 2: 128-byte, 4: 64-byte):
// lbo = stride between MN atoms, sbo = stride between 8-row K groups
// (measured: these roles, base offset 0 for row-shifted starts)
__device__ __forceinline__ uint64_t umma_desc_mn(uint32_t saddr, uint32_t lbo, uint32_t sbo, uint32_t layout) {
    return (uint64_t)((saddr >> 4) & 0x3fffu) | (uint64_t)((lbo >> 4) & 0x3fffu) << 16 |
           (uint64_t)((sbo >> 4) & 0x3fffu) << 32 | (uint64_t)1 << 46 | (uint64_t)layout << 61;
}

__global__ void __launch_bounds__(ROW_THREADS, 1)
    wgrad_row_kernel(const WgradRowArgs a, const int S, const int ux, const __grid_constant__ CUtensorMap tdz,
                     const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tmu) {
    constexpr uint32_t COLS = 512;  // nine 32-column accumulators
    extern __shared__ __align__(1024) unsigned char smem[];
    if (smem_u32(smem) & 1023u) {
        if (threadIdx.x == 0 && a.err) atomicExch(a.err, 2);
        return;
    }
    const int K0 = a.c0 + a.c1;
    const int STG = wg_stage_bytes(ux);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + S * STG);
    uint64_t *done = full + 4, *expd = full + 8, *accf = full + 12, *drain = full + 13;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(full + 14);
    int *flag = reinterpret_cast<int *>(full + 15);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int mtiles = (a.co + 127) / 128, chunks = K0 / 32, combos = mtiles * chunks;
    const int combo = blockIdx.x % combos, mt = combo / chunks, cc = combo - mt * chunks;
    const int m0 = mt * 128;
    const int tile0 = blockIdx.x / combos, tstride = gridDim.x / combos;
    const int segs = a.W / RW, ntiles = a.M / RW;
    const int njobs = tile0 < ntiles ? (ntiles - tile0 + tstride - 1) / tstride : 0;
    const bool direct = cc * 32 < a.c0;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int k = 0; k < 4; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&done[k], 1);
            mbar_init(&expd[k], ROW_EXP);
        }
        mbar_init(accf, 1);
        mbar_init(drain, 1);
        *flag = 0;
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    struct Where {
        int x0, y, b;
    };
    auto where = [&](int i) {
        const int t = tile0 + i * tstride;
        return Where{(t % segs) * RW, (t / segs) % a.H, t / (segs * a.H)};
    };
    auto give_up = [&]() {
        *(volatile int *)flag = 1;
        if (a.err) atomicExch(a.err, 1);
    };
    auto stopped = [&]() { return *(volatile int *)flag != 0; };

    if (warp == 0) {
        // ---------------- producer ----------------
        if (lane == 0) {
            int j = 0;
            for (; j < njobs && !stopped(); ++j) {
                const int st = j % S;
                if (j >= S && !mbar_wait_sleep(&done[st], ((j - S) / S) & 1, WAIT_LIMIT_NS)) {
                    give_up();
                    break;
                }
                const Where w = where(j);
                unsigned char *As = smem + st * STG, *Hs = As + WG_A_BYTES;
                mbar_expect_tx(&full[st], 2 * (128 * 64 * 2) + (direct ? RHALO_TX : RU_TX));
                tma_load_4d(As, &tdz, m0, w.x0, w.y, w.b, &full[st]);
                tma_load_4d(As + WG_A_ATOM, &tdz, m0 + 64, w.x0, w.y, w.b, &full[st]);
                if (direct)
                    tma_load_4d(Hs, &tmx, cc * 32, w.x0 - 1, w.y - 1, w.b, &full[st]);
                else
                    tma_load_4d(Hs + RA_BYTES, &tmu, cc * 32 - a.c0, (w.x0 >> 1) - 1, (w.y - 1) >> 1, w.b,
                                &full[st]);
            }
            for (int jb = j - 1; jb >= 0 && jb >= j - S; --jb) mbar_wait(&full[jb % S], (jb / S) & 1, DRAIN_LIMIT_NS);
        }
    } else if (warp == 1) {
        // ---------------- MMA issue ----------------
        if (lane == 0) {
            constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
                                       ((32u >> 3) << 17) | ((128u >> 4) << 24);  // MN-major A and B
            bool ok = true;
            for (int j = 0; j < njobs && !stopped(); ++j) {
                const int st = j % S;
                ok = mbar_wait_sleep(&full[st], (j / S) & 1, WAIT_LIMIT_NS);
                if (ok && !direct) ok = mbar_wait_sleep(&expd[st], (j / S) & 1, WAIT_LIMIT_NS);
                if (!ok) {
                    give_up();
                    break;
                }
                tc_fence_after();
                const uint32_t As = smem_u32(smem + st * STG), Hs = As + WG_A_BYTES;
                // descriptors of the stage's operands; a start moved by b bytes
                // adds b / 16 to the address field (no carry: below 256 KB)
                const uint64_t ad0 = umma_desc_mn(As, WG_A_ATOM, 1024, 2);
                const uint64_t bd0 = umma_desc_mn(Hs, 16, 512, 4);
#pragma unroll
                for (int tap = 0; tap < 9; ++tap) {
                    const int sh = (tap / 3) * RHALO + tap % 3;  // (dy + 1) rows, dx + 1 pixels
#pragma unroll
                    for (int k = 0; k < RW / 16; ++k) {
                        const uint64_t ad = ad0 + (uint64_t)(k * 16 * 128 / 16);
                        const uint64_t bd = bd0 + (uint64_t)((sh + k * 16) * 64 / 16);
                        const uint32_t accum = (j > 0 || k > 0) ? 1u : 0u;
                        asm volatile(
                            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem + tap * 32),
                            "l"(ad), "l"(bd), "r"(idesc), "r"(accum)
                            : "memory");
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(&done[st]))
                             : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(accf))
                         : "memory");
        }
    } else if (warp < 6) {
        // ---------------- expansion of coarse upsampled chunks ----------------
        const int et = tid - 64, qq = et & 3;
        for (int j = 0; !direct && j < njobs && !stopped(); ++j) {
            const int st = j % S;
            if ((j >= S && !mbar_wait_sleep(&done[st], ((j - S) / S) & 1, WAIT_LIMIT_NS)) ||
                !mbar_wait_sleep(&full[st], (j / S) & 1, WAIT_LIMIT_NS)) {
                give_up();
                break;
            }
            const Where w = where(j);
            unsigned char *Hs = smem + st * STG + WG_A_BYTES;
            const unsigned char *U = Hs + RA_BYTES;
            const uint32_t hbase = smem_u32(Hs);
            for (int r = 0; r < 3; ++r) {
                const int cr = ((w.y + r - 1) >> 1) - ((w.y - 1) >> 1);
                for (int p = et >> 2; p < RHALO; p += ROW_EXP / 4) {
                    const int pix = r * RHALO + p;
                    const int sw = (int)(((hbase + pix * 64) >> 7) & 3u);
                    *reinterpret_cast<uint4 *>(Hs + pix * 64 + ((qq ^ sw) << 4)) =
                        *reinterpret_cast<const uint4 *>(U + (cr * 66 + ((p + 1) >> 1)) * 64 + qq * 16);
                }
            }
            fence_proxy_async();
            mbar_arrive(&expd[st]);
        }
    } else {
        // ---------------- epilogue: add the nine accumulators to dW ----------------
        if (njobs > 0 && mbar_wait_sleep(accf, 0, WAIT_LIMIT_NS) && !stopped()) {
            tc_fence_after();
            const int ew = warp & 3;
            const int row = m0 + ew * 32 + lane;  // output channel
            for (int tap = 0; tap < 9; ++tap) {
                uint32_t r[32];
#pragma unroll
                for (int c = 0; c < 32; c += 16) {
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
                        "%15}, [%16];"
                        : "=r"(r[c]), "=r"(r[c + 1]), "=r"(r[c + 2]), "=r"(r[c + 3]), "=r"(r[c + 4]), "=r"(r[c + 5]),
                          "=r"(r[c + 6]), "=r"(r[c + 7]), "=r"(r[c + 8]), "=r"(r[c + 9]), "=r"(r[c + 10]),
                          "=r"(r[c + 11]), "=r"(r[c + 12]), "=r"(r[c + 13]), "=r"(r[c + 14]), "=r"(r[c + 15])
                        : "r"(tmem + ((uint32_t)(ew * 32) << 16) + (uint32_t)(tap * 32 + c)));
                }
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (row < a.co) {
                    float *d = a.dw + ((size_t)row * 9 + tap) * K0 + cc * 32;
#pragma unroll
                    for (int c = 0; c < 32; ++c) atomicAdd(d + c, __uint_as_float(r[c]));
                }
            }
            tc_fence_before();
        } else if (njobs > 0 && !stopped()) {
            give_up();
        }
    }
    if (warp == 1 && lane == 0 && stopped()) {
        // one last commit tracks every MMA issued: a short wait before the
        // tensor memory is released
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(drain))
                     : "memory");
        mbar_wait(drain, 0, DRAIN_LIMIT_NS);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(COLS) : "memory");
    }
}

// ---------------------------------------------------------------------------
// Weight gradient with the nine taps sharing one MMA, per slice of 32 output
// channels.  With dZ rows y-1, y, y+1 of a row tile as the M atoms of A (64-byte
// swizzle, atom stride one row tile; the fourth atom's products are not
// used) and X row y with a one-pixel halo as B, read as three N atoms that
// start one pixel apart (atom stride 64 bytes), one M = 128, N = 96 product of
// K = 128 pixels gives
//   D[32 jy + co][32 jx + ci] = sum_x dZ[y - 1 + jy][x][co] X[y][x + jx - 1][ci],
// the contribution of X row y to the tap (dy, dx) = (1 - jy, jx - 1) of
//   dW[co][tap][ci] = sum_p dZ[p][co] X[p + d_tap][ci].
// Summed over all rows y of the image this is the whole gradient: rows of dZ
// outside the image are zero-filled by the tensor copy, and so are pixels of
// X outside it.  A CTA owns one (32-channel slice of dZ, 32-channel chunk of
// X) pair and a contiguous run of row tiles taken down each 128-pixel column
// strip, so consecutive tiles share two of their three dZ rows: the dZ rows
// live in a ring of R = S + 2 row slots (slots R and R + 1 repeat slots 0 and
// 1, so that any three consecutive rows are evenly spaced) and each tile
// loads one new dZ row and its X row.  Eight MMAs per tile, where the per-tap
// kernel above issues 72 of N = 32 (a quarter of them useful when the layer
// has 32 output channels), and half its copy traffic.
// ---------------------------------------------------------------------------
constexpr int WT_ROW = RW * 64;    // one dZ row tile: 128 pixels x 32 channels
constexpr int WT_B_BYTES = 9216;   // X row y, 130 pixels x 64 bytes (8320), rounded up to 1024
constexpr int WT_U_BYTES = 5120;   // one coarse row, 66 pixels x 64 bytes (4224), rounded up
constexpr int WT_MAX_STAGES = 8;
constexpr int WT_BAR_BYTES = 256;  // 3 x 8 + 2 barriers, the tensor-memory slot and the stop flag
constexpr int WT_MAX_CO = 256;     // the widest layer of the networks built here
constexpr int WT_PRODUCERS = 5;    // warps issuing the tensor copies: 0 and 6-9
static_assert(WT_PRODUCERS >= 1 && WT_PRODUCERS <= 5, "producer warps 0 and 6-9");
constexpr int WT_PART = 32 * 9 * 32;  // one CTA's partial sums: [co][tap][ci]
// shared memory of S stages: R + 2 ring slots, S X-row stages, barriers.  The
// fourth A atom of a window at slot R - 1 reads slot R + 2, the first X stage
__host__ __device__ inline int wt_stage_bytes(int ux) { return WT_B_BYTES + (ux ? WT_U_BYTES : 0); }
__host__ __device__ inline int wt_smem(int S, int ux) { return (S + 4) * WT_ROW + S * wt_stage_bytes(ux) + WT_BAR_BYTES; }

__global__ void __launch_bounds__(ROW_THREADS, 1)
    wgrad_tap_kernel(const WgradRowArgs a, const int S, const int ux, const __grid_constant__ CUtensorMap tdz,
                     const __grid_constant__ CUtensorMap tmx, const __grid_constant__ CUtensorMap tmu) {
    constexpr uint32_t COLS = 128;  // one 96-column accumulator
    extern __shared__ __align__(1024) unsigned char smem[];
    if (smem_u32(smem) & 1023u) {
        if (threadIdx.x == 0 && a.err) atomicExch(a.err, 2);
        return;
    }
    const int K0 = a.c0 + a.c1;
    const int R = S + 2, SB = wt_stage_bytes(ux);
    unsigned char *ring = smem, *stg = smem + (R + 2) * WT_ROW;
    uint64_t *full = reinterpret_cast<uint64_t *>(stg + S * SB);
    uint64_t *done = full + WT_MAX_STAGES, *expd = done + WT_MAX_STAGES, *accf = expd + WT_MAX_STAGES,
             *drain = accf + 1;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(drain + 1);
    int *flag = reinterpret_cast<int *>(drain + 2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int chunks = K0 / 32, combos = (a.co / 32) * chunks;
    const int combo = blockIdx.x % combos, mt = combo / chunks, cc = combo - mt * chunks;
    const int per = gridDim.x / combos, q = blockIdx.x / combos;
    const int segs = a.W / RW, ntiles = a.M / RW;  // tiles in (image, strip, row) order
    const int t_begin = (int)((long long)ntiles * q / per), t_end = (int)((long long)ntiles * (q + 1) / per);
    const int njobs = t_end - t_begin;
    const bool direct = cc * 32 < a.c0;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int k = 0; k < S; ++k) {
            mbar_init(&full[k], 1);
            mbar_init(&done[k], 1);
            mbar_init(&expd[k], ROW_EXP / 32);  // one arrival per expansion warp
        }
        mbar_init(accf, 1);
        mbar_init(drain, 1);
        *flag = 0;
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    struct Where {
        int x0, y, b;
    };
    auto where = [&](int j) {
        const int t = t_begin + j, strip = t / a.H;
        return Where{(strip % segs) * RW, t - strip * a.H, strip / segs};
    };
    // a tile starts a new window (three fresh dZ rows at slot 0) at the
    // start of the CTA's run and of each strip (row 0), else the window
    // moves down one slot of the ring
    auto give_up = [&]() {
        *(volatile int *)flag = 1;
        if (a.err) atomicExch(a.err, 1);
    };
    auto stopped = [&]() { return *(volatile int *)flag != 0; };

    // ---------------- producers ----------------
    // tile j's copies come from producer j % WT_PRODUCERS, lane 0 of warp 0
    // or of an epilogue warp (6..).  With the MMA loop this lean, one thread's
    // per-tile work (waits, bookkeeping, two or three copies) starts to pace
    // the pipeline: five producers measured 8 % faster than one
    const int prod = warp == 0 ? 0 : warp >= 6 && warp - 5 < WT_PRODUCERS ? warp - 5 : -1;
    if (prod >= 0 && lane == 0) {
        // row, strip, window, stage and phase advance tile by tile (as in the
        // MMA loop); only a producer's own tiles pay for their coordinates
        int last = -1, run = 0, ws = 0, st = 0;
        int yc = njobs > 0 ? where(0).y : 0, strip = (t_begin - yc) / a.H;
        uint32_t ph = 0;
        for (int j = 0; j < njobs && !stopped(); ++j) {
            if (j > 0) {
                ws = ++yc == a.H ? 0 : (ws + 1 == R ? 0 : ws + 1);
                if (yc == a.H) {
                    yc = 0;
                    ++strip;
                }
                if (++st == S) {
                    st = 0;
                    ph ^= 1u;
                }
            }
            const bool fresh = j == 0 || yc == 0;
            if (fresh) run = j;
            if (j % WT_PRODUCERS != prod) continue;
            const Where w{(strip % segs) * RW, yc, strip / segs};
            // the stage's X row, and the slot of the new dZ row: both were
            // last read by tile j - S (the ring holds S + 2 rows) or, early in
            // a run, by any tile of the run before (up to tile run - 1).  The
            // waits go in order up to the later of the two (a producer has
            // seen tile j - WT_PRODUCERS - S complete, so the previous phase
            // of each barrier waited on is complete and its parity
            // unambiguous: S >= WT_PRODUCERS)
            bool ok = j < S || mbar_wait_sleep(&done[st], ph ^ 1u, WAIT_LIMIT_NS);
            for (int k = j - S + 1 < 0 ? 0 : j - S + 1; ok && k < run; ++k)
                ok = mbar_wait_sleep(&done[k % S], (k / S) & 1, WAIT_LIMIT_NS);
            if (!ok) {
                give_up();
                break;
            }
            unsigned char *Bs = stg + st * SB;
            const int s_new = ws + 2 < R ? ws + 2 : ws + 2 - R;  // slot of row y + 1
            const int nrows = fresh ? 5 : (s_new < 2 ? 2 : 1);
            mbar_expect_tx(&full[st], nrows * WT_ROW + (direct ? RHALO * 64 : 66 * 64));
            if (fresh) {
                // rows y - 1, y, y + 1 into slots 0, 1, 2; rows y - 1 and y
                // again into slots R and R + 1
                for (int r = 0; r < 3; ++r)
                    tma_load_4d(ring + r * WT_ROW, &tdz, mt * 32, w.x0, w.y - 1 + r, w.b, &full[st]);
                for (int r = 0; r < 2; ++r)
                    tma_load_4d(ring + (R + r) * WT_ROW, &tdz, mt * 32, w.x0, w.y - 1 + r, w.b, &full[st]);
            } else {
                tma_load_4d(ring + s_new * WT_ROW, &tdz, mt * 32, w.x0, w.y + 1, w.b, &full[st]);
                if (s_new < 2)
                    tma_load_4d(ring + (R + s_new) * WT_ROW, &tdz, mt * 32, w.x0, w.y + 1, w.b, &full[st]);
            }
            if (direct)
                tma_load_4d(Bs, &tmx, cc * 32, w.x0 - 1, w.y, w.b, &full[st]);
            else
                tma_load_4d(Bs + WT_B_BYTES, &tmu, cc * 32 - a.c0, (w.x0 >> 1) - 1, w.y >> 1, w.b, &full[st]);
            last = j;
        }
        // after a stop, copies still in flight land before the CTA exits (a
        // normal run needs no drain: the MMA thread has waited for every
        // copy; nor could it wait here, as another producer may already have
        // reused the stage, putting the barrier a phase further on)
        for (int jb = last; stopped() && jb >= 0 && jb > last - S; jb -= WT_PRODUCERS)
            mbar_wait(&full[jb % S], (jb / S) & 1, DRAIN_LIMIT_NS);
    }
    __syncwarp();
    if (warp == 1) {
        // ---------------- MMA issue ----------------
        if (lane == 0) {
            constexpr uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
                                       ((96u >> 3) << 17) | ((128u >> 4) << 24);  // MN-major A and B
            // the issuing thread paces the tensor core: its per-tile work is
            // kept to the waits (spinning, for the shortest hand-over), two
            // descriptor adds and the MMAs (stage, phase, row and window
            // advance incrementally, no divisions)
            const uint64_t ad_ring = umma_desc_mn(smem_u32(ring), WT_ROW, 512, 4);
            const uint64_t bd_stg = umma_desc_mn(smem_u32(stg), 64, 512, 4);
            int st = 0, ws = 0, yc = njobs > 0 ? where(0).y : 0;
            uint32_t ph = 0, accum = 0;
            for (int j = 0; j < njobs && !stopped(); ++j) {
                if (j > 0) {
                    ws = ++yc == a.H ? 0 : (ws + 1 == R ? 0 : ws + 1);
                    if (yc == a.H) yc = 0;
                }
                bool ok = mbar_wait(&full[st], ph, WAIT_LIMIT_NS);
                if (ok && !direct) ok = mbar_wait(&expd[st], ph, WAIT_LIMIT_NS);
                if (!ok) {
                    give_up();
                    break;
                }
                tc_fence_after();
                // A: atoms one row slot apart from the window's first slot; B:
                // atoms one pixel apart.  Each K step of 16 pixels moves both
                // starts by 1024 bytes (64 in the address field: no carry
                // below 256 KB)
                const uint64_t ad0 = ad_ring + (uint64_t)((ws * WT_ROW) >> 4);
                const uint64_t bd0 = bd_stg + (uint64_t)((st * SB) >> 4);
#pragma unroll
                for (int k = 0; k < RW / 16; ++k) {
                    asm volatile(
                        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                        "l"(ad0 + (uint64_t)(k * 64)), "l"(bd0 + (uint64_t)(k * 64)), "r"(idesc), "r"(accum)
                        : "memory");
                    accum = 1u;
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(&done[st]))
                             : "memory");
                if (++st == S) {
                    st = 0;
                    ph ^= 1u;
                }
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(accf))
                         : "memory");
        }
    } else if (warp >= 2 && warp < 6) {
        // ---------------- expansion of the coarse upsampled row ----------------
        // a thread writes 16-byte chunk qq of pixels p = et / 4 + 32 i of the
        // fine row (stage bases are 1024-byte aligned, so the 64-byte swizzle
        // of pixel p is (p / 2) & 3); each thread fences its writes for the
        // tensor core, and one lane per warp arrives
        const int et = tid - 64, qq = et & 3;
        int st = 0;
        uint32_t ph = 0;
        for (int j = 0; !direct && j < njobs && !stopped(); ++j) {
            if ((j >= S && !mbar_wait_sleep(&done[st], ph ^ 1u, WAIT_LIMIT_NS)) ||
                !mbar_wait_sleep(&full[st], ph, WAIT_LIMIT_NS)) {
                give_up();
                break;
            }
            unsigned char *Bs = stg + st * SB;
            const unsigned char *U = Bs + WT_B_BYTES;
            for (int p = et >> 2; p < RHALO; p += ROW_EXP / 4)
                *reinterpret_cast<uint4 *>(Bs + p * 64 + ((qq ^ ((p >> 1) & 3)) << 4)) =
                    *reinterpret_cast<const uint4 *>(U + ((p + 1) >> 1) * 64 + qq * 16);
            fence_proxy_async();
            __syncwarp();
            if (lane == 0) mbar_arrive(&expd[st]);
            if (++st == S) {
                st = 0;
                ph ^= 1u;
            }
        }
    } else if (warp >= 6) {
        // ---------------- epilogue: the CTA's nine 32 x 32 blocks ----------------
        // stored as this CTA's partial sums (plain stores: every CTA finishing
        // at once with FP32 atomics on the same 36 KB of dW would serialise in
        // the L2); wgrad_reduce_kernel adds them up
        const int ew = warp & 3;  // accumulator lanes 32 ew..: dZ row y - 1 + ew, i.e. dy = 1 - ew
        float *part = a.part + (size_t)blockIdx.x * WT_PART;
        if (njobs == 0 && ew < 3) {
            for (int jx = 0; jx < 3; ++jx) {
                float4 *d = reinterpret_cast<float4 *>(part + ((size_t)lane * 9 + (2 - ew) * 3 + jx) * 32);
                for (int c = 0; c < 8; ++c) d[c] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        } else if (njobs > 0 && mbar_wait_sleep(accf, 0, WAIT_LIMIT_NS) && !stopped()) {
            tc_fence_after();
            if (ew < 3) {
                for (int jx = 0; jx < 3; ++jx) {
                    uint32_t r[32];
#pragma unroll
                    for (int c = 0; c < 32; c += 16) {
                        asm volatile(
                            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
                            "%14,%15}, [%16];"
                            : "=r"(r[c]), "=r"(r[c + 1]), "=r"(r[c + 2]), "=r"(r[c + 3]), "=r"(r[c + 4]),
                              "=r"(r[c + 5]), "=r"(r[c + 6]), "=r"(r[c + 7]), "=r"(r[c + 8]), "=r"(r[c + 9]),
                              "=r"(r[c + 10]), "=r"(r[c + 11]), "=r"(r[c + 12]), "=r"(r[c + 13]), "=r"(r[c + 14]),
                              "=r"(r[c + 15])
                            : "r"(tmem + ((uint32_t)(ew * 32) << 16) + (uint32_t)(jx * 32 + c)));
                    }
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    const int tap = (2 - ew) * 3 + jx;
                    float4 *d = reinterpret_cast<float4 *>(part + ((size_t)lane * 9 + tap) * 32);
#pragma unroll
                    for (int c = 0; c < 8; ++c)
                        d[c] = make_float4(__uint_as_float(r[4 * c]), __uint_as_float(r[4 * c + 1]),
                                           __uint_as_float(r[4 * c + 2]), __uint_as_float(r[4 * c + 3]));
                }
            }
            tc_fence_before();
        } else if (njobs > 0 && !stopped()) {
            give_up();
        }
    }
    if (warp == 1 && lane == 0 && stopped()) {
        // one last commit tracks every MMA issued: a short wait before the
        // tensor memory is released
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                         smem_u32(drain))
                     : "memory");
        mbar_wait(drain, 0, DRAIN_LIMIT_NS);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(COLS) : "memory");
    }
}

// dW += the shared-tap kernel's partial sums: CTA q * combos + combo holds
// [co][tap][ci] of the (32-channel slice of dZ, 32-channel chunk of X) pair
// combo.  Thread (element, split) sums the CTAs q = split, split + splits, ...
// of its pair and adds the sum to dW (dW starts at zero)
__global__ void wgrad_reduce_kernel(const float *part, int combos, int per, int chunks, int K0, float *dw) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)combos * WT_PART) return;
    const int combo = (int)(i / WT_PART), e = (int)(i - (long long)combo * WT_PART);
    const int split = blockIdx.y, splits = gridDim.y;
    float s0 = 0.f, s1 = 0.f;
    int q = split;
    for (; q + splits < per; q += 2 * splits) {
        s0 += part[((size_t)q * combos + combo) * WT_PART + e];
        s1 += part[((size_t)(q + splits) * combos + combo) * WT_PART + e];
    }
    if (q < per) s0 += part[((size_t)q * combos + combo) * WT_PART + e];
    const int co = e / (9 * 32), tap = (e / 32) % 9, ci = e % 32;
    const int mt = combo / chunks, cc = combo - mt * chunks;
    atomicAdd(dw + ((size_t)(mt * 32 + co) * 9 + tap) * K0 + cc * 32 + ci, s0 + s1);
}

// ---------------------------------------------------------------------------
// Weight gradient of one tap: dW[co][tap][ci] += sum_pixel dZ[p][co] X[p + d][ci]
// over a chunk of pixels per CTA (atomic FP32 accumulation of the chunks).
// ---------------------------------------------------------------------------
struct WgradArgs {
    const bf16 *dz;
    int co;
    const bf16 *x0, *x1;
    int c0, c1;
    int B, H, W, M;
    int chunk;
    float *dw;  // [co][9][c0 + c1]
};

__global__ void __launch_bounds__(256) wgrad_kernel(const WgradArgs a) {
    __shared__ __align__(128) unsigned char sA[2][32 * 128];  // [pixel][64 co]
    __shared__ __align__(128) unsigned char sB[2][32 * 128];  // [pixel][64 ci]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = warp & 1, wn = warp >> 1;  // 2 x 4 warps, warp tile 32 x 16
    const int tap = blockIdx.z % 9, part = blockIdx.z / 9;
    const int m0 = blockIdx.x * 64, n0 = blockIdx.y * 64;
    const int ci_all = a.c0 + a.c1;
    const int p_begin = part * a.chunk;
    const int p_end = min(a.M, p_begin + a.chunk);
    const int dy = tap / 3 - 1, dx = tap % 3 - 1;
    const int row = tid >> 3, ch = tid & 7;
    const bool a_col = m0 + ch * 8 < a.co;
    const int cin = n0 + ch * 8;
    const bool b_col = cin < ci_all;
    const int ksteps = (p_end - p_begin + 31) / 32;

    auto load = [&](int ks, int buf) {
        const int p = p_begin + ks * 32 + row;
        const bool pv = p < p_end;
        const bool va = pv && a_col;
        cp_async16(sA[buf] + sw128(row, ch), va ? a.dz + (size_t)p * a.co + m0 + ch * 8 : a.dz, va);
        bool vb = pv && b_col;
        const bf16 *src = a.x0;
        if (vb) {
            const int x = p % a.W, t = p / a.W, y = t % a.H, b = t / a.H;
            const int yy = y + dy, xx = x + dx;
            vb = yy >= 0 && yy < a.H && xx >= 0 && xx < a.W;
            if (vb) {
                if (cin < a.c0)
                    src = a.x0 + ((size_t)(b * a.H + yy) * a.W + xx) * a.c0 + cin;
                else
                    src = a.x1 + ((size_t)(b * (a.H >> 1) + (yy >> 1)) * (a.W >> 1) + (xx >> 1)) * a.c1 +
                          (cin - a.c0);
            }
        }
        cp_async16(sB[buf] + sw128(row, ch), src, vb);
        cp_async_commit();
    };

    float acc[2][2][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int k = 0; k < 4; ++k) acc[i][j][k] = 0.f;

    if (ksteps > 0) load(0, 0);
    for (int ks = 0; ks < ksteps; ++ks) {
        const int buf = ks & 1;
        if (ks + 1 < ksteps) {
            load(ks + 1, buf ^ 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        const int bi = lane >> 3, r = lane & 7;
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
            uint32_t af[2][4], bq[4];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
                ldsm4t(af[mt], sA[buf] + sw128(kk * 16 + (bi >> 1) * 8 + r, (wm * 32 + mt * 16 + (bi & 1) * 8) >> 3));
            ldsm4t(bq, sB[buf] + sw128(kk * 16 + (bi & 1) * 8 + r, (wn * 16 + (bi >> 1) * 8) >> 3));
#pragma unroll
            for (int mt = 0; mt < 2; ++mt) {
                mma_bf16(acc[mt][0], af[mt], bq[0], bq[1]);
                mma_bf16(acc[mt][1], af[mt], bq[2], bq[3]);
            }
        }
        __syncthreads();
    }

    const int g = lane >> 2, t4 = lane & 3;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int m = m0 + wm * 32 + mt * 16 + g + h * 8;
                const int n = n0 + wn * 16 + nt * 8 + 2 * t4;
                if (m >= a.co || n >= ci_all) continue;
                float *d = a.dw + ((size_t)m * 9 + tap) * ci_all + n;
                atomicAdd(d, acc[mt][nt][2 * h]);
                atomicAdd(d + 1, acc[mt][nt][2 * h + 1]);
            }
}

// ---------------------------------------------------------------------------
// Elementwise kernels
// ---------------------------------------------------------------------------
#define GRID_STRIDE(i, n) for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (n); \
                                i += (long long)gridDim.x * blockDim.x)

// network input: 4 FP32 channels per pixel -> BF16 padded to cpad channels;
// one thread per pixel and 8-channel piece
__global__ void pack_input_kernel(const float *x, bf16 *out, long long P, int cpad) {
    const int g = cpad / 8;
    GRID_STRIDE(i, P * g) {
        const long long p = i / g;
        uint4 o = make_uint4(0u, 0u, 0u, 0u);
        if (i - p * g == 0) {
            const float4 v = reinterpret_cast<const float4 *>(x)[p];
            __nv_bfloat162 lo = __floats2bfloat162_rn(v.x, v.y), hi = __floats2bfloat162_rn(v.z, v.w);
            o.x = *reinterpret_cast<uint32_t *>(&lo);
            o.y = *reinterpret_cast<uint32_t *>(&hi);
        }
        reinterpret_cast<uint4 *>(out)[i] = o;
    }
}

__device__ __forceinline__ float2 bf2_to_f2(uint32_t u) {
    return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u));
}

// 2x2 average pooling, NHWC BF16; one thread per output pixel and 8 channels
__global__ void pool_kernel(const bf16 *in, bf16 *out, int B, int H, int W, int C) {
    const int h2 = H / 2, w2 = W / 2, g = C / 8;
    GRID_STRIDE(i, (long long)B * h2 * w2 * g) {
        const int c8 = (int)(i % g);
        long long t = i / g;
        const int x = (int)(t % w2);
        t /= w2;
        const int y = (int)(t % h2);
        const int b = (int)(t / h2);
        const uint4 *src = reinterpret_cast<const uint4 *>(in);
        auto at = [&](int yy, int xx) { return src[(((long long)b * H + yy) * W + xx) * g + c8]; };
        const uint4 v00 = at(2 * y, 2 * x), v01 = at(2 * y, 2 * x + 1), v10 = at(2 * y + 1, 2 * x),
                    v11 = at(2 * y + 1, 2 * x + 1);
        const uint32_t *a = &v00.x, *b1 = &v01.x, *c = &v10.x, *d = &v11.x;
        uint4 o;
        uint32_t *op = &o.x;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float2 fa = bf2_to_f2(a[k]), fb = bf2_to_f2(b1[k]), fc = bf2_to_f2(c[k]), fd = bf2_to_f2(d[k]);
            __nv_bfloat162 r = __floats2bfloat162_rn(0.25f * (fa.x + fb.x + fc.x + fd.x),
                                                     0.25f * (fa.y + fb.y + fc.y + fd.y));
            op[k] = *reinterpret_cast<uint32_t *>(&r);
        }
        reinterpret_cast<uint4 *>(out)[i] = o;
    }
}

// head: phi = tanh(w . d + b) per pixel (C a multiple of 8)
__global__ void head_forward_kernel(const bf16 *d, const float *wb, int C, long long P, float *phi) {
    GRID_STRIDE(p, P) {
        float z = wb[C];
        const uint4 *row = reinterpret_cast<const uint4 *>(d + p * C);
        for (int c8 = 0; c8 < C / 8; ++c8) {
            const uint4 v = row[c8];
            const uint32_t *u = &v.x;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float2 f = bf2_to_f2(u[k]);
                z += f.x * wb[8 * c8 + 2 * k];
                z += f.y * wb[8 * c8 + 2 * k + 1];
            }
        }
        phi[p] = tanhf(z);
    }
}

// per-block partial sums of (mask, mask (phi - t)^2) for the loss (pass 1)
__global__ void loss_partial_kernel(const float *phi, const float *t, const float *mask, long long P,
                                    double *part) {
    __shared__ double s0[256], s1[256];
    double a = 0, b = 0;
    GRID_STRIDE(p, P) {
        const double m = mask[p];
        const double r = (double)phi[p] - (double)t[p];
        a += m;
        b += m * r * r;
    }
    s0[threadIdx.x] = a;
    s1[threadIdx.x] = b;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) {
            s0[threadIdx.x] += s0[threadIdx.x + s];
            s1[threadIdx.x] += s1[threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = s0[0];
        part[2 * blockIdx.x + 1] = s1[0];
    }
}

// pass 2: out[0] = number of masked pixels (at least 1), out[1] = loss
__global__ void loss_final_kernel(const double *part, int nblocks, double *out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double a = 0, b = 0;
    for (int k = 0; k < nblocks; ++k) {
        a += part[2 * k];
        b += part[2 * k + 1];
    }
    const double n = a > 1.0 ? a : 1.0;
    out[0] = n;
    out[1] = b / n;
}

// head backward: per pixel dz = d loss / d (w . d + b) = 2 mask (phi - t) (1 - phi^2) / n,
// the input gradient dd[p][c] = dz w[c], and the head's gradients
// gw[c] += sum_p dz d[p][c], gb += sum_p dz.  A thread owns 8 channels of a
// strided set of pixels (C / 8 threads share a pixel); the block reduces by
// channel in shared memory and adds to gwb
__global__ void head_backward_kernel(const float *phi, const float *t, const float *mask, const double *stat,
                                     const bf16 *d, const float *wb, int C, long long P, float *dd,
                                     float *gwb) {
    __shared__ float part[256 * 9];
    const float inv_n = (float)(1.0 / stat[0]);
    const int g8 = C / 8;
    const int lanes = blockDim.x / g8;
    const int grp = threadIdx.x % g8, sub = threadIdx.x / g8;
    float w[8], acc[9];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        w[k] = wb[grp * 8 + k];
        acc[k] = 0.f;
    }
    acc[8] = 0.f;
    if (sub < lanes)
        for (long long p = (long long)blockIdx.x * lanes + sub; p < P; p += (long long)gridDim.x * lanes) {
            const float f = phi[p];
            const float dz = 2.f * mask[p] * (f - t[p]) * inv_n * (1.f - f * f);
            const long long i = p * g8 + grp;
            const uint4 dv = reinterpret_cast<const uint4 *>(d)[i];
            const uint32_t *dp = &dv.x;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float2 df = bf2_to_f2(dp[k]);
                acc[2 * k] += dz * df.x;
                acc[2 * k + 1] += dz * df.y;
            }
            float4 *o = reinterpret_cast<float4 *>(dd) + 2 * i;
            o[0] = make_float4(dz * w[0], dz * w[1], dz * w[2], dz * w[3]);
            o[1] = make_float4(dz * w[4], dz * w[5], dz * w[6], dz * w[7]);
            if (grp == 0) acc[8] += dz;
        }
#pragma unroll
    for (int k = 0; k < 9; ++k) part[threadIdx.x * 9 + k] = acc[k];
    __syncthreads();
    for (int c = threadIdx.x; c <= C; c += blockDim.x) {
        float sum = 0.f;
        if (c < C)
            for (int l = 0; l < lanes; ++l) sum += part[(l * g8 + c / 8) * 9 + (c & 7)];
        else
            for (int l = 0; l < lanes; ++l) sum += part[(l * g8) * 9 + 8];
        atomicAdd(gwb + c, sum);
    }
}

// gb[c] += sum over pixels of dz[p][c] (BF16 [P][C]): a thread sums 8
// channels of a strided set of pixels, the block reduces by channel in
// shared memory and adds to gb
__global__ void bias_sum_kernel(const bf16 *dz, long long P, int C, float *gb) {
    __shared__ float part[256 * 8];
    const int g8 = C / 8;
    const int lanes = blockDim.x / g8;
    const int grp = threadIdx.x % g8, sub = threadIdx.x / g8;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (sub < lanes)
        for (long long p = (long long)blockIdx.x * lanes + sub; p < P; p += (long long)gridDim.x * lanes) {
            const uint4 v = reinterpret_cast<const uint4 *>(dz)[p * g8 + grp];
            const uint32_t *vp = &v.x;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float2 f = bf2_to_f2(vp[k]);
                acc[2 * k] += f.x;
                acc[2 * k + 1] += f.y;
            }
        }
#pragma unroll
    for (int k = 0; k < 8; ++k) part[threadIdx.x * 8 + k] = acc[k];
    __syncthreads();
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        float sum = 0.f;
        for (int l = 0; l < lanes; ++l) sum += part[(l * g8 + c / 8) * 8 + (c & 7)];
        atomicAdd(gb + c, sum);
    }
}

// dz = g where the forward activation h > 0, else 0 (BF16), and the bias
// gradient gb[c] += sum over pixels of that BF16 dz[p][c], in one pass: a
// thread owns 8 channels of a strided set of pixels, the block reduces by
// channel in shared memory and adds to gb.  With gc, the gradient that
// flows back through the 2 x 2 average pooling of this activation is added
// first: g[p] + gc[coarse pixel of p] / 4 (gc [B][H/2][W/2][C])
__global__ void relu_mask_bias_kernel(const float *g, const float *gc, int H, int W, const bf16 *h, bf16 *dz,
                                      long long P, int C, float *gb) {
    __shared__ float part[256 * 8];
    const int g8 = C / 8;
    const int lanes = blockDim.x / g8;  // pixels in flight per block
    const int grp = threadIdx.x % g8, sub = threadIdx.x / g8;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (sub < lanes)
        for (long long p = (long long)blockIdx.x * lanes + sub; p < P; p += (long long)gridDim.x * lanes) {
            const long long i = p * g8 + grp;  // 8-channel group index
            const float4 g0 = reinterpret_cast<const float4 *>(g)[2 * i], g1 = reinterpret_cast<const float4 *>(g)[2 * i + 1];
            const uint4 hv = reinterpret_cast<const uint4 *>(h)[i];
            const uint32_t *hp = &hv.x;
            float gv[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
            if (gc) {
                const int pi = (int)p, x = pi % W, r = pi / W, y = r % H, b = r / H;
                const long long ic = ((long long)(b * (H >> 1) + (y >> 1)) * (W >> 1) + (x >> 1)) * g8 + grp;
                const float4 c0 = reinterpret_cast<const float4 *>(gc)[2 * ic],
                             c1 = reinterpret_cast<const float4 *>(gc)[2 * ic + 1];
                gv[0] += 0.25f * c0.x;
                gv[1] += 0.25f * c0.y;
                gv[2] += 0.25f * c0.z;
                gv[3] += 0.25f * c0.w;
                gv[4] += 0.25f * c1.x;
                gv[5] += 0.25f * c1.y;
                gv[6] += 0.25f * c1.z;
                gv[7] += 0.25f * c1.w;
            }
            uint4 o;
            uint32_t *op = &o.x;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float2 hf = bf2_to_f2(hp[k]);
                __nv_bfloat162 r = __floats2bfloat162_rn(hf.x > 0.f ? gv[2 * k] : 0.f, hf.y > 0.f ? gv[2 * k + 1] : 0.f);
                op[k] = *reinterpret_cast<uint32_t *>(&r);
                const float2 rf = bf2_to_f2(op[k]);
                acc[2 * k] += rf.x;
                acc[2 * k + 1] += rf.y;
            }
            reinterpret_cast<uint4 *>(dz)[i] = o;
        }
#pragma unroll
    for (int k = 0; k < 8; ++k) part[threadIdx.x * 8 + k] = acc[k];
    __syncthreads();
    for (int c = threadIdx.x; c < C; c += blockDim.x) {
        float sum = 0.f;
        for (int l = 0; l < lanes; ++l) sum += part[(l * g8 + c / 8) * 8 + (c & 7)];
        atomicAdd(gb + c, sum);
    }
}

// gradient of concat(e, up(d)) from dcat [P][cs + cu]: de [P][cs] = the first
// cs channels (the skip connection's gradient; de has no other writer); dd
// (coarse [B][H/2][W/2][cu]) = the last cu channels summed over each 2 x 2
// block (nearest-upsampling backward); 4 channels a thread
__global__ void split_concat_kernel(const float *dcat, int cs, int cu, int B, int H, int W, float *de,
                                    float *dd) {
    const int ct = cs + cu;
    GRID_STRIDE(i, (long long)B * H * W * (cs / 4)) {
        const long long p = i / (cs / 4);
        const int c = (int)(i - p * (cs / 4)) * 4;
        *reinterpret_cast<float4 *>(de + p * cs + c) = *reinterpret_cast<const float4 *>(dcat + p * ct + c);
    }
    const int h2 = H / 2, w2 = W / 2;
    GRID_STRIDE(i, (long long)B * h2 * w2 * (cu / 4)) {
        const int c = (int)(i % (cu / 4)) * 4;
        long long t = i / (cu / 4);
        const int x = (int)(t % w2);
        t /= w2;
        const int y = (int)(t % h2);
        const int b = (int)(t / h2);
        float4 s4 = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int a = 0; a < 2; ++a)
            for (int e = 0; e < 2; ++e) {
                const float4 v = *reinterpret_cast<const float4 *>(
                    dcat + (((long long)b * H + 2 * y + a) * W + 2 * x + e) * ct + cs + c);
                s4.x += v.x;
                s4.y += v.y;
                s4.z += v.z;
                s4.w += v.w;
            }
        *reinterpret_cast<float4 *>(dd + (((long long)b * h2 + y) * w2 + x) * cu + c) = s4;
    }
}

// second half of the nearest-upsampling backward after a split epilogue:
// dd [B][H/2][W/2][cu] = dh [B][H][W/2][cu] summed over each vertical row
// pair (dh already holds the horizontal pair sums); 4 channels a thread
__global__ void pair_rows_kernel(const float *dh, int cu, int B, int H, int Wh, float *dd) {
    const int h2 = H / 2;
    GRID_STRIDE(i, (long long)B * h2 * Wh * (cu / 4)) {
        const int c = (int)(i % (cu / 4)) * 4;
        long long t = i / (cu / 4);
        const int x = (int)(t % Wh);
        t /= Wh;
        const int y = (int)(t % h2);
        const int b = (int)(t / h2);
        const float4 u = *reinterpret_cast<const float4 *>(dh + (((long long)b * H + 2 * y) * Wh + x) * cu + c);
        const float4 v = *reinterpret_cast<const float4 *>(dh + (((long long)b * H + 2 * y + 1) * Wh + x) * cu + c);
        *reinterpret_cast<float4 *>(dd + (((long long)b * h2 + y) * Wh + x) * cu + c) =
            make_float4(u.x + v.x, u.y + v.y, u.z + v.z, u.w + v.w);
    }
}

// index of element (n_all, tap, k_all) of BF16 weights [N][9][K0] in the row
// kernel's shared-memory image (per N tile of BN and chunk of 32 input channels,
// [tap][n / 8][k / 8][n % 8][k % 8]: the K-major core-matrix layout of the B
// operand; tiles and chunks in (N tile, chunk) order)
__device__ __forceinline__ long long row_pack_index(int n_all, int tap, int k_all, int K0, int BN) {
    const int nt = n_all / BN, n = n_all - nt * BN, kc = k_all / 32, k = k_all - kc * 32;
    return ((long long)(nt * (K0 / 32) + kc) * 9 + tap) * BN * 32 + ((n >> 3) * 4 + (k >> 3)) * 64 + (n & 7) * 8 +
           (k & 7);
}

// all four BF16 images of a layer's FP32 master weights w [co][3][3][ci] in
// one pass: wf [co][9][cpad] (forward), wt [cpad][9][co] (data gradient) and,
// where the row kernel takes the layer (bn_f, bn_t nonzero), the same two in
// its packed layout; zero in the padded channels
__global__ void weights_prep_kernel(const float *w, int co, int ci, int cpad, int bn_f, int bn_t, bf16 *wf,
                                    bf16 *wt, bf16 *wpf, bf16 *wpt) {
    GRID_STRIDE(i, (long long)co * 9 * cpad) {
        const int c = (int)(i % cpad);
        const long long t = i / cpad;
        const int tap = (int)(t % 9);
        const int o = (int)(t / 9);
        const bf16 h = __float2bfloat16_rn(c < ci ? w[((long long)o * 9 + tap) * ci + c] : 0.f);
        wf[i] = h;
        wt[((long long)c * 9 + tap) * co + o] = h;
        if (bn_f) wpf[row_pack_index(o, tap, c, cpad, bn_f)] = h;
        if (bn_t) wpt[row_pack_index(c, tap, o, co, bn_t)] = h;
    }
}

// padded weight gradient [co][9][cpad] -> flat [co][3][3][ci]
__global__ void grad_pack_kernel(const float *dw, int co, int ci, int cpad, float *g) {
    GRID_STRIDE(i, (long long)co * 9 * ci) {
        const int c = (int)(i % ci);
        const long long t = i / ci;
        g[i] = dw[t * cpad + c];
    }
}

// Adam (bias-corrected), in place on the FP32 master parameters
__global__ void adam_kernel(float *theta, const float *g, float *m, float *v, long long n, float lr, float b1,
                            float b2, float eps, float bc1, float bc2) {
    GRID_STRIDE(i, n) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        theta[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    }
}

int blocks_for(long long n, int per = 256) {
    long long b = (n + per - 1) / per;
    if (b > 65535LL * 16) b = 65535LL * 16;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

// ---------------------------------------------------------------------------
// The network object
// ---------------------------------------------------------------------------
constexpr int UNET_IN = 8;     // input channels of the parameter layout (4 used, 4 zero)
constexpr int UNET_PAD0 = 32;  // input channels on the device (multiple of the GEMM k-chunk)

struct UnetLayer {
    int co, ci, cpad, k;     // k = 3 (conv3x3) or 1 (head)
    long long off;           // offset of the weights in the flat parameter vector; bias follows
    bf16 *wf = nullptr, *wt = nullptr;
    bf16 *wpf = nullptr, *wpt = nullptr;  // wf, wt packed for the row kernel (N tile row_bn(N))
    float *dw = nullptr;     // [co][9][cpad]
};

struct mclbm_unet {
    int levels = 0, base = 0, max_b = 0, max_h = 0, max_w = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<UnetLayer> layers;  // parameter order
    long long nparam = 0;
    float *theta = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
    long long adam_t = 0;
    std::vector<bf16 *> a_in, e_ha, e_out, d_ha, d_out;  // per level
    std::vector<bf16 *> up;  // up[0]: d_1 (or e_1) upsampled to level 0, the finest decoder's input
    std::vector<float *> de;                              // per level
    float *phi = nullptr, *s1 = nullptr, *s2 = nullptr, *dd = nullptr;
    bf16 *z = nullptr, *z2 = nullptr;  // dz of a layer; z2 takes the next one's while z is read
    float *xin_f = nullptr, *t_f = nullptr, *mask_f = nullptr;  // staging of host inputs
    double *loss_part = nullptr, *loss_stat = nullptr;
    int *err = nullptr;  // device: set by a tensor-core kernel whose bounded wait gave up
    int max_ctas = 0;    // bound on the row-tile kernels' CTAs (0: one wave)
    int shared_taps = 1;  // weight gradients on the shared-tap kernel (else the per-tap one)
    float *wg_part = nullptr;  // the shared-tap kernel's per-CTA partial sums
    int wg_part_ctas = 0;
    std::vector<void *> allocs;
    int cur_b = 0, cur_h = 0, cur_w = 0;
};

namespace {

constexpr int LOSS_BLOCKS = 256;

int ch(const mclbm_unet &u, int l) { return u.base << l; }

int ualloc(mclbm_unet &u, void **p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes < 16 ? 16 : bytes);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(unet)");
    u.allocs.push_back(*p);
    return MCLBM_OK;
}

void unet_release(mclbm_unet *u) {
    if (!u) return;
    if (u->stream) cudaStreamSynchronize(u->stream);
    for (void *p : u->allocs) cudaFree(p);
    if (u->own_stream && u->stream) cudaStreamDestroy(u->stream);
    delete u;
}

template <int BN>
cudaError_t launch_tc(const mclbm_unet &u, ConvArgs a) {
    constexpr int bytes = 2 * (TBM * TBK * 2 + BN * TBK * 2) + 32;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(conv_tc_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const dim3 grid((a.M + TBM - 1) / TBM, (a.N + BN - 1) / BN);
    conv_tc_kernel<BN><<<grid, 128, bytes, u.stream>>>(a);
    count_launch();
    return cudaGetLastError();
}

constexpr int ROW_SMEM_MAX = 227 * 1024;   // opt-in dynamic shared memory per CTA
constexpr int ROW_SMEM_PAIR = 113 * 1024;  // per CTA when two share an SM

// stages and weight residency of the row kernel: two CTAs per SM where that
// leaves at least two stages, else one; weights resident where they fit
RowPlan row_plan(int BN, int kchunks, int ux) {
    for (int wres = 1; wres >= 0; --wres) {
        const int fixed = row_smem(BN, kchunks, wres, ux, 0);
        const int stg = row_stage_bytes(BN, wres, ux);
        for (int cap : {ROW_SMEM_PAIR, ROW_SMEM_MAX}) {
            int S = (cap - fixed) / stg;
            if (S > 4) S = 4;
            if (S >= 2) return RowPlan{wres, ux, S, row_smem(BN, kchunks, wres, ux, S)};
        }
    }
    return RowPlan{0, ux, 0, 0};
}

int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
            n = 1;
    }
    return n;
}

using EncodeTiledFn = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        cudaGetLastError();
    }
    return fn;
}

// tensor map of an NHWC BF16 tensor [B][H][W][C] read in boxes of box_c
// channels x bw pixels x bh rows x 1 image, zero fill outside
cudaError_t nhwc_map(const bf16 *base, int B, int H, int W, int C, int box_c, int bw, int bh,
                     CUtensorMapSwizzle sw, CUtensorMap *m) {
    EncodeTiledFn enc = encode_tiled();
    if (!enc) return cudaErrorNotSupported;
    const cuuint64_t dims[4] = {(cuuint64_t)C, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
    const cuuint64_t strides[3] = {(cuuint64_t)C * 2, (cuuint64_t)W * C * 2, (cuuint64_t)H * W * C * 2};
    const cuuint32_t box[4] = {(cuuint32_t)box_c, (cuuint32_t)bw, (cuuint32_t)bh, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<bf16 *>(base), dims, strides, box,
                           estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// the halo maps of a convolution input: x0 in swizzled boxes of 32 channels
// x 130 pixels x 3 rows; x1 likewise when at full resolution, else in plain
// boxes of 66 coarse pixels x 2 rows
cudaError_t halo_maps(const bf16 *x0, const bf16 *x1, int c0, int c1, int x1_full, int B, int H, int W,
                      CUtensorMap *tmx, CUtensorMap *tmu) {
    constexpr auto SW64 = CU_TENSOR_MAP_SWIZZLE_64B;
    cudaError_t e = nhwc_map(x0, B, H, W, c0, 32, RHALO, 3, SW64, tmx);
    if (e != cudaSuccess) return e;
    if (c1 == 0) return nhwc_map(x0, B, H, W, c0, 32, RHALO, 3, SW64, tmu);
    if (x1_full) return nhwc_map(x1, B, H, W, c1, 32, RHALO, 3, SW64, tmu);
    return nhwc_map(x1, B, H >> 1, W >> 1, c1, 32, 66, 2, CU_TENSOR_MAP_SWIZZLE_NONE, tmu);
}

template <int BN>
cudaError_t launch_row(const mclbm_unet &u, ConvArgs a) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e =
            cudaFuncSetAttribute(conv_row_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, ROW_SMEM_MAX);
        // all of the unified L1/shared memory as shared memory, so that two
        // CTAs fit where the plan allows
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(conv_row_kernel<BN>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const RowPlan plan = row_plan(BN, (a.c0 + a.c1) / 32, a.c1 > 0 && !a.x1_full ? 1 : 0);
    if (plan.stages < 2) return cudaErrorInvalidValue;
    // resident CTAs per SM: 228 KB of shared memory (1 KB reserved per CTA)
    // and 512 tensor-memory columns (the occupancy query was seen to answer
    // one where two fit; a CTA that does not fit merely starts later)
    constexpr int cols = 2 * BN <= 64 ? 64 : 2 * BN <= 128 ? 128 : 256;
    int per_sm = (228 * 1024) / (plan.smem + 1024);
    if (per_sm > 512 / cols) per_sm = 512 / cols;
    // and 64 K registers, allocated per warp in units of 256
    static int regs_per_cta = 0;
    if (!regs_per_cta) {
        cudaFuncAttributes fa;
        if (cudaFuncGetAttributes(&fa, conv_row_kernel<BN>) != cudaSuccess) return cudaErrorInvalidConfiguration;
        regs_per_cta = (ROW_THREADS / 32) * ((fa.numRegs * 32 + 255) / 256 * 256);
    }
    if (per_sm > 65536 / regs_per_cta) per_sm = 65536 / regs_per_cta;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const int ntn = a.N / BN;
    const long long items = (long long)(a.M / RW) * ntn;
    long long grid = (long long)per_sm * sm_count();
    if (u.max_ctas > 0 && grid > u.max_ctas) grid = u.max_ctas;
    if (grid > items) grid = items;
    grid -= grid % ntn;
    if (grid < ntn) grid = ntn;
    CUtensorMap tmx, tmu;
    cudaError_t e = halo_maps(a.x0, a.x1, a.c0, a.c1, a.x1_full, a.B, a.H, a.W, &tmx, &tmu);
    if (e != cudaSuccess) return e;
    conv_row_kernel<BN><<<(int)grid, ROW_THREADS, plan.smem, u.stream>>>(a, plan, a.wp, tmx, tmu);
    count_launch();
    return cudaGetLastError();
}

// forward and data-gradient convolutions on the tensor cores: the row-tile
// kernel where the width is a multiple of 128 and the N tile divides N,
// else the pixel-gather kernel (N tile = N up to 256, else 128)
cudaError_t launch_conv(const mclbm_unet &u, ConvArgs a) {
    a.err = u.err;
    if (a.c0 % TBK || (a.c0 + a.c1) % TBK || a.N % 16) return cudaErrorInvalidValue;
    if (a.W % RW == 0 && a.wp) {
        switch (row_bn(a.N)) {
            case 32: return launch_row<32>(u, a);
            case 64: return launch_row<64>(u, a);
            case 96: return launch_row<96>(u, a);
            case 128: return launch_row<128>(u, a);
            default: break;
        }
    }
    if (a.split_cs) return cudaErrorInvalidValue;  // the split epilogue is the row kernel's
    switch (a.N) {
        case 32: return launch_tc<32>(u, a);
        case 64: return launch_tc<64>(u, a);
        case 96: return launch_tc<96>(u, a);
        case 128: return launch_tc<128>(u, a);
        case 192: return launch_tc<192>(u, a);
        case 256: return launch_tc<256>(u, a);
        default: return a.N % 128 == 0 ? launch_tc<128>(u, a) : cudaErrorInvalidValue;
    }
}

// the weight gradient with the taps sharing one MMA (co a multiple of 32)
cudaError_t launch_wgrad_tap(const mclbm_unet &u, const WgradRowArgs &a, int ux) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(wgrad_tap_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             ROW_SMEM_MAX);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(wgrad_tap_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    int S = WT_MAX_STAGES;
    while (S > 2 && wt_smem(S, ux) > ROW_SMEM_MAX) --S;
    if (wt_smem(S, ux) > ROW_SMEM_MAX || S < WT_PRODUCERS) return cudaErrorInvalidConfiguration;
    const int smem = wt_smem(S, ux);
    constexpr auto SW64 = CU_TENSOR_MAP_SWIZZLE_64B;
    CUtensorMap tdz, tmx, tmu;
    cudaError_t e = nhwc_map(a.dz, a.B, a.H, a.W, a.co, 32, RW, 1, SW64, &tdz);
    if (e == cudaSuccess) e = nhwc_map(a.x0, a.B, a.H, a.W, a.c0, 32, RHALO, 1, SW64, &tmx);
    if (e == cudaSuccess)
        e = ux ? nhwc_map(a.x1, a.B, a.H >> 1, a.W >> 1, a.c1, 32, 66, 1, CU_TENSOR_MAP_SWIZZLE_NONE, &tmu)
               : nhwc_map(a.x0, a.B, a.H, a.W, a.c0, 32, RHALO, 1, SW64, &tmu);
    if (e != cudaSuccess) return e;
    const int combos = (a.co / 32) * ((a.c0 + a.c1) / 32);
    int grid = sm_count();
    if (u.max_ctas > 0 && grid > u.max_ctas) grid = u.max_ctas;
    if (grid > combos * (a.M / RW)) grid = combos * (a.M / RW);
    grid -= grid % combos;
    if (grid < combos) grid = combos;
    if (grid > u.wg_part_ctas) return cudaErrorInvalidConfiguration;
    WgradRowArgs b = a;
    b.part = u.wg_part;
    wgrad_tap_kernel<<<grid, ROW_THREADS, smem, u.stream>>>(b, S, ux, tdz, tmx, tmu);
    // enough threads for the GPU: the partials of each pair split over up to
    // 16 groups of CTAs
    const int per = grid / combos;
    const long long nel = (long long)combos * WT_PART;
    int splits = (int)((8LL * 152 * 256 + nel - 1) / nel);
    if (splits > 16) splits = 16;
    if (splits > per) splits = per;
    wgrad_reduce_kernel<<<dim3((unsigned)((nel + 255) / 256), (unsigned)splits), 256, 0, u.stream>>>(
        u.wg_part, combos, per, (a.c0 + a.c1) / 32, a.c0 + a.c1, a.dw);
    count_launch(2);
    return cudaGetLastError();
}

// the weight gradient on the tensor cores where the width is a multiple of
// 128 (row tiles), else on mma.sync
cudaError_t launch_wgrad_row(const mclbm_unet &u, const WgradArgs &w) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(wgrad_row_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             ROW_SMEM_MAX);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(wgrad_row_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                     (int)cudaSharedmemCarveoutMaxShared);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    WgradRowArgs a{};
    a.dz = w.dz;
    a.co = w.co;
    a.x0 = w.x0;
    a.x1 = w.x1;
    a.c0 = w.c0;
    a.c1 = w.c1;
    a.B = w.B;
    a.H = w.H;
    a.W = w.W;
    a.M = w.M;
    a.dw = w.dw;
    a.err = u.err;
    const int ux = w.c1 > 0 ? 1 : 0;
    if (u.shared_taps && w.co % 32 == 0 && w.co <= WT_MAX_CO) return launch_wgrad_tap(u, a, ux);
    int S = (ROW_SMEM_MAX - 256) / wg_stage_bytes(ux);
    if (S > 4) S = 4;
    if (S < 2) return cudaErrorInvalidConfiguration;
    const int smem = S * wg_stage_bytes(ux) + 256;
    CUtensorMap tdz, tmx, tmu;
    cudaError_t e = nhwc_map(w.dz, w.B, w.H, w.W, w.co, 64, RW, 1, CU_TENSOR_MAP_SWIZZLE_128B, &tdz);
    if (e == cudaSuccess) e = halo_maps(w.x0, w.x1, w.c0, w.c1, 0, w.B, w.H, w.W, &tmx, &tmu);
    if (e != cudaSuccess) return e;
    const int combos = ((w.co + 127) / 128) * ((w.c0 + w.c1) / 32);
    int grid = sm_count();
    if (u.max_ctas > 0 && grid > u.max_ctas) grid = u.max_ctas;
    if (grid > combos * (w.M / RW)) grid = combos * (w.M / RW);
    grid -= grid % combos;
    if (grid < combos) grid = combos;
    wgrad_row_kernel<<<grid, ROW_THREADS, smem, u.stream>>>(a, S, ux, tdz, tmx, tmu);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_wgrad(const mclbm_unet &u, WgradArgs a) {
    if (a.W % RW == 0 && a.c0 % 32 == 0 && a.c1 % 32 == 0) return launch_wgrad_row(u, a);
    a.chunk = 4096;
    const int parts = (a.M + a.chunk - 1) / a.chunk;
    const dim3 grid((a.co + 63) / 64, (a.c0 + a.c1 + 63) / 64, 9 * parts);
    wgrad_kernel<<<grid, 256, 0, u.stream>>>(a);
    count_launch();
    return cudaGetLastError();
}

// conv input description: x0 (c0 channels) and optionally the upsampled x1
struct In {
    const bf16 *x0, *x1;
    int c0, c1;
    int x1_full = 0;  // x1 at the resolution of x0 (an upsampled copy), else half
};

// forward of conv layer li on input `in` at (B, H, W): y = ReLU(conv + b)
cudaError_t conv_forward(const mclbm_unet &u, int li, In in, int B, int H, int W, bf16 *y, bf16 *yup = nullptr) {
    const UnetLayer &L = u.layers[li];
    ConvArgs a{};
    a.x0 = in.x0;
    a.x1 = in.x1;
    a.c0 = in.c0;
    a.c1 = in.c1;
    a.x1_full = in.x1_full;
    a.yup = yup;
    a.B = B;
    a.H = H;
    a.W = W;
    a.M = B * H * W;
    a.sign = 1;
    a.w = L.wf;
    a.wp = L.wpf;
    a.N = L.co;
    a.bias = u.theta + L.off + (long long)L.co * 9 * L.ci;
    a.ybf = y;
    a.yf = nullptr;
    return launch_conv(u, a);
}

// backward of conv layer li: dz (BF16 [P][co]) -> weight and bias gradients,
// and, if dx, the input gradient (FP32 [P][cpad])
// With split_cs (a decoder's concat input, row kernel only), the input
// gradient goes out split: the first split_cs channels to dx as [P][split_cs],
// the upsampled channels pair-summed along x to dh (see ConvArgs)
// With mask_h, the input gradient goes out masked by that forward
// activation, as BF16 into ydz (the next layer's dz)
cudaError_t conv_backward(mclbm_unet &u, int li, In in, int B, int H, int W, const bf16 *dz, float *dx,
                          int split_cs = 0, float *dh = nullptr, const bf16 *mask_h = nullptr,
                          bf16 *ydz = nullptr) {
    // the bias gradient comes with dz (mask_and_bias)
    UnetLayer &L = u.layers[li];
    const int M = B * H * W;
    cudaError_t e = cudaMemsetAsync(L.dw, 0, (size_t)L.co * 9 * L.cpad * sizeof(float), u.stream);
    if (e != cudaSuccess) return e;
    WgradArgs w{};
    w.dz = dz;
    w.co = L.co;
    w.x0 = in.x0;
    w.x1 = in.x1;
    w.c0 = in.c0;
    w.c1 = in.c1;
    w.B = B;
    w.H = H;
    w.W = W;
    w.M = M;
    w.dw = L.dw;
    if ((e = launch_wgrad(u, w)) != cudaSuccess) return e;
    float *gw = u.grad + L.off;
    grad_pack_kernel<<<blocks_for((long long)L.co * 9 * L.ci), 256, 0, u.stream>>>(L.dw, L.co, L.ci, L.cpad, gw);
    count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (!dx && !ydz) return cudaSuccess;
    ConvArgs a{};
    a.x0 = dz;
    a.x1 = nullptr;
    a.c0 = L.co;
    a.c1 = 0;
    a.B = B;
    a.H = H;
    a.W = W;
    a.M = M;
    a.sign = -1;
    a.w = L.wt;
    a.wp = L.wpt;
    a.N = L.cpad;
    a.bias = nullptr;
    a.ybf = nullptr;
    a.yf = dx;
    a.split_cs = split_cs;
    a.yh = dh;
    a.mask_h = mask_h;
    a.ydz = ydz;
    return launch_conv(u, a);
}

// layer li's bias gradient from its BF16 dz [P][C]
cudaError_t bias_grad(mclbm_unet &u, int li, const bf16 *dz, long long P, int C) {
    const UnetLayer &L = u.layers[li];
    float *gb = u.grad + L.off + (long long)L.co * 9 * L.ci;
    cudaError_t e = cudaMemsetAsync(gb, 0, C * sizeof(float), u.stream);
    if (e != cudaSuccess) return e;
    bias_sum_kernel<<<4 * sm_count(), 256, 0, u.stream>>>(dz, P, C, gb);
    count_launch();
    return cudaGetLastError();
}

cudaError_t refresh_weights(mclbm_unet &u) {
    for (auto &L : u.layers) {
        if (L.k != 3) continue;
        weights_prep_kernel<<<blocks_for((long long)L.co * 9 * L.cpad), 256, 0, u.stream>>>(
            u.theta + L.off, L.co, L.ci, L.cpad, row_bn(L.co), row_bn(L.cpad), L.wf, L.wt, L.wpf, L.wpt);
        count_launch();
    }
    return cudaGetLastError();
}

cudaError_t forward(mclbm_unet &u, int B, int H, int W) {
    const int Lv = u.levels;
    cudaError_t e = cudaSuccess;
    // encoder
    for (int l = 0; l < Lv && e == cudaSuccess; ++l) {
        const int h = H >> l, w = W >> l;
        if (l > 0) {
            pool_kernel<<<blocks_for((long long)B * h * w * (ch(u, l - 1) / 8)), 256, 0, u.stream>>>(
                u.e_out[l - 1], u.a_in[l], B, 2 * h, 2 * w, ch(u, l - 1));
            count_launch();
        }
        const In ina{u.a_in[l], nullptr, l == 0 ? UNET_PAD0 : ch(u, l - 1), 0};
        if ((e = conv_forward(u, 2 * l, ina, B, h, w, u.e_ha[l])) != cudaSuccess) break;
        const In inb{u.e_ha[l], nullptr, ch(u, l), 0};
        // the coarsest level writes its output upsampled too when the first
        // decoder is the finest level
        e = conv_forward(u, 2 * l + 1, inb, B, h, w, u.e_out[l], l == 1 && Lv == 2 ? u.up[0] : nullptr);
    }
    // decoder, coarse to fine
    int li = 2 * Lv;
    for (int l = Lv - 2; l >= 0 && e == cudaSuccess; --l, li += 2) {
        const int h = H >> l, w = W >> l;
        // concat(e_l, nearest-upsampled d_{l+1}).  At the finest level the
        // producer of d_1 also writes it upsampled (4x its output, but the
        // convolution then stages it like a direct input); coarser levels
        // expand the coarse rows in shared memory, where the extra writes
        // would cost more than they save
        const bf16 *coarse = l == Lv - 2 ? u.e_out[Lv - 1] : u.d_out[l + 1];
        const In ina = l == 0 ? In{u.e_out[0], u.up[0], ch(u, 0), ch(u, 1), 1}
                              : In{u.e_out[l], coarse, ch(u, l), ch(u, l + 1)};
        if ((e = conv_forward(u, li, ina, B, h, w, u.d_ha[l])) != cudaSuccess) break;
        const In inb{u.d_ha[l], nullptr, ch(u, l), 0};
        e = conv_forward(u, li + 1, inb, B, h, w, u.d_out[l], l == 1 ? u.up[0] : nullptr);
    }
    if (e != cudaSuccess) return e;
    const UnetLayer &hd = u.layers.back();
    const long long P = (long long)B * H * W;
    const bf16 *d0 = Lv > 1 ? u.d_out[0] : u.e_out[0];
    head_forward_kernel<<<blocks_for(P), 256, 0, u.stream>>>(d0, u.theta + hd.off, u.base, P, u.phi);
    count_launch();
    return cudaGetLastError();
}

// dz (u.z) = (g + gc / 4 upsampled, if gc) masked by the forward activation
// h > 0, and layer li's bias gradient from the same pass (images H x W)
cudaError_t mask_and_bias(mclbm_unet &u, int li, const float *g, const float *gc, int H, int W, const bf16 *h,
                          long long P, int C) {
    const UnetLayer &L = u.layers[li];
    float *gb = u.grad + L.off + (long long)L.co * 9 * L.ci;
    cudaError_t e = cudaMemsetAsync(gb, 0, C * sizeof(float), u.stream);
    if (e != cudaSuccess) return e;
    relu_mask_bias_kernel<<<4 * sm_count(), 256, 0, u.stream>>>(g, gc, H, W, h, u.z, P, C, gb);
    count_launch();
    return cudaGetLastError();
}

cudaError_t backward(mclbm_unet &u, int B, int H, int W) {
    const int Lv = u.levels;
    const long long P = (long long)B * H * W;
    const UnetLayer &hd = u.layers.back();
    cudaError_t e = cudaMemsetAsync(u.grad + hd.off, 0, (u.base + 1) * sizeof(float), u.stream);
    if (e != cudaSuccess) return e;
    const bf16 *d0 = Lv > 1 ? u.d_out[0] : u.e_out[0];
    head_backward_kernel<<<4 * sm_count(), 256, 0, u.stream>>>(u.phi, u.t_f, u.mask_f, u.loss_stat, d0,
                                                               u.theta + hd.off, u.base, P, u.dd, u.grad + hd.off);
    count_launch();
    // decoder, fine to coarse: the layer index of dec(l)a is 2L + 2 (L - 2 - l)
    for (int l = 0; l <= Lv - 2; ++l) {
        const int h = H >> l, w = W >> l;
        const long long Pl = (long long)B * h * w;
        const int cl = ch(u, l), cu = ch(u, l + 1);
        const int li = 2 * Lv + 2 * (Lv - 2 - l);
        if ((e = mask_and_bias(u, li + 1, u.dd, nullptr, h, w, u.d_out[l], Pl, cl)) != cudaSuccess) return e;
        // the data gradient of dec(l)b leaves masked by d_ha[l], as dec(l)a's dz
        if ((e = conv_backward(u, li + 1, In{u.d_ha[l], nullptr, cl, 0}, B, h, w, u.z, nullptr, 0, nullptr,
                               u.d_ha[l], u.z2)) != cudaSuccess)
            return e;
        if ((e = bias_grad(u, li, u.z2, Pl, cl)) != cudaSuccess) return e;
        const bf16 *coarse = l == Lv - 2 ? u.e_out[Lv - 1] : u.d_out[l + 1];
        const In in_a{u.e_out[l], coarse, cl, cu};
        if (w % RW == 0 && row_bn(u.layers[li].cpad)) {
            // the row kernel's epilogue writes the skip gradient to de[l] and
            // the pair sums along x to s1; the row pairs finish the
            // upsampling backward
            if ((e = conv_backward(u, li, in_a, B, h, w, u.z2, u.de[l], cl, u.s1)) != cudaSuccess) return e;
            pair_rows_kernel<<<blocks_for(Pl * cu / 16), 256, 0, u.stream>>>(u.s1, cu, B, h, w / 2, u.dd);
        } else {
            if ((e = conv_backward(u, li, in_a, B, h, w, u.z2, u.s1)) != cudaSuccess) return e;
            split_concat_kernel<<<blocks_for(Pl * cl / 4), 256, 0, u.stream>>>(u.s1, cl, cu, B, h, w, u.de[l],
                                                                                u.dd);
        }
        count_launch();
    }
    // encoder, coarse to fine
    for (int l = Lv - 1; l >= 0; --l) {
        const int h = H >> l, w = W >> l;
        const long long Pl = (long long)B * h * w;
        const int cl = ch(u, l);
        // the gradient reaching e_out[l]: at the coarsest level the decoder's
        // (dd: the upsampling backward of the last split, or the head's when
        // there is one level); below it the skip connection's (de[l]) plus
        // the gradient through the pooling into level l + 1 (in s1, from that
        // level's first convolution)
        const float *g_out = l == Lv - 1 ? u.dd : u.de[l];
        if ((e = mask_and_bias(u, 2 * l + 1, g_out, l < Lv - 1 ? u.s1 : nullptr, h, w, u.e_out[l], Pl, cl)) !=
            cudaSuccess)
            return e;
        // the data gradient of enc(l)b leaves masked by e_ha[l], as enc(l)a's dz
        if ((e = conv_backward(u, 2 * l + 1, In{u.e_ha[l], nullptr, cl, 0}, B, h, w, u.z, nullptr, 0, nullptr,
                               u.e_ha[l], u.z2)) != cudaSuccess)
            return e;
        if ((e = bias_grad(u, 2 * l, u.z2, Pl, cl)) != cudaSuccess) return e;
        const int cin = l == 0 ? UNET_PAD0 : ch(u, l - 1);
        if ((e = conv_backward(u, 2 * l, In{u.a_in[l], nullptr, cin, 0}, B, h, w, u.z2, l > 0 ? u.s1 : nullptr)) !=
            cudaSuccess)
            return e;
    }
    return cudaGetLastError();
}

bool dev_ptr(const void *p) {
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// copy a caller buffer (host or device) into a device staging buffer
cudaError_t stage_in(const mclbm_unet &u, float *dst, const float *src, size_t n) {
    return cudaMemcpyAsync(dst, src, n * sizeof(float), dev_ptr(src) ? cudaMemcpyDeviceToDevice
                                                                      : cudaMemcpyHostToDevice,
                           u.stream);
}
cudaError_t stage_out(const mclbm_unet &u, float *dst, const float *src, size_t n) {
    return cudaMemcpyAsync(dst, src, n * sizeof(float), dev_ptr(dst) ? cudaMemcpyDeviceToDevice
                                                                      : cudaMemcpyDeviceToHost,
                           u.stream);
}

int check_shape(const mclbm_unet *u, int B, int H, int W) {
    if (!u) return fail(MCLBM_ERR_ARG, "network is NULL");
    const int q = 1 << (u->levels - 1);
    if (B < 1 || H < q || W < q || B > u->max_b || H > u->max_h || W > u->max_w)
        return fail(MCLBM_ERR_ARG, "batch or image size outside the sizes the network was created for");
    if (H % q || W % q) return fail(MCLBM_ERR_ARG, "image sides must be multiples of 2^(levels-1)");
    if ((long long)B * H * W > (long long)u->max_b * u->max_h * u->max_w)
        return fail(MCLBM_ERR_ARG, "too many pixels");
    return MCLBM_OK;
}

// stage inputs, pack, forward (and the loss when targets are given)
int run_forward(mclbm_unet *u, int B, int H, int W, const float *x, const float *target, const float *mask) {
    const long long P = (long long)B * H * W;
    cudaError_t e = stage_in(*u, u->xin_f, x, (size_t)P * 4);
    if (e == cudaSuccess && target) e = stage_in(*u, u->t_f, target, (size_t)P);
    if (e == cudaSuccess && target) e = stage_in(*u, u->mask_f, mask, (size_t)P);
    if (e != cudaSuccess) return cuda_fail(e, "unet input copy");
    pack_input_kernel<<<blocks_for(P * (UNET_PAD0 / 8)), 256, 0, u->stream>>>(u->xin_f, u->a_in[0], P, UNET_PAD0);
    count_launch();
    if ((e = forward(*u, B, H, W)) != cudaSuccess) return cuda_fail(e, "unet forward");
    if (target) {
        loss_partial_kernel<<<LOSS_BLOCKS, 256, 0, u->stream>>>(u->phi, u->t_f, u->mask_f, P, u->loss_part);
        loss_final_kernel<<<1, 32, 0, u->stream>>>(u->loss_part, LOSS_BLOCKS, u->loss_stat);
        count_launch(2);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "unet loss");
    }
    return MCLBM_OK;
}

// after a synchronisation: report (and clear) a wait that gave up
int check_err(mclbm_unet *u) {
    int err = 0;
    cudaError_t e = cudaMemcpy(&err, u->err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "unet error word");
    if (err) {
        cudaMemset(u->err, 0, sizeof(int));
        if (err == 2) return fail(MCLBM_ERR_CUDA, "row-tile convolution: shared memory not 1024-byte aligned");
        return fail(MCLBM_ERR_TIMEOUT, "a tensor-core convolution timed out waiting for its copies or MMAs");
    }
    return MCLBM_OK;
}

int read_loss(mclbm_unet *u, double *loss) {
    double st[2] = {0, 0};
    cudaError_t e = cudaMemcpyAsync(st, u->loss_stat, sizeof(st), cudaMemcpyDeviceToHost, u->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(u->stream);
    if (e != cudaSuccess) return cuda_fail(e, "unet loss read-back");
    if (int rc = check_err(u)) return rc;
    if (loss) *loss = st[1];
    return MCLBM_OK;
}

}  // namespace

extern "C" {

int mclbm_unet_create(int levels, int base, int max_batch, int max_h, int max_w, void *cuda_stream,
                      mclbm_unet **out) {
    if (!out) return fail(MCLBM_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (levels < 1 || levels > 6) return fail(MCLBM_ERR_ARG, "levels must be 1..6");
    if (base < 32 || base % 32 || (base << (levels - 1)) > 1024)
        return fail(MCLBM_ERR_ARG, "base channels must be a multiple of 32 (and C0 2^(L-1) <= 1024)");
    if (base > 64) return fail(MCLBM_ERR_ARG, "base channels above 64 are not supported by the head");
    const int q = 1 << (levels - 1);
    if (max_batch < 1 || max_h < q || max_w < q || max_h % q || max_w % q)
        return fail(MCLBM_ERR_ARG, "maximum sizes must be positive multiples of 2^(levels-1)");
    if ((long long)max_batch * max_h * max_w > 0x7fffffffLL)
        return fail(MCLBM_ERR_ARG, "at most 2^31 - 1 pixels per batch (32-bit pixel indices)");
    mclbm_unet *u = new (std::nothrow) mclbm_unet;
    if (!u) return fail(MCLBM_ERR_NOMEM, "host allocation failed");
    u->levels = levels;
    u->base = base;
    u->max_b = max_batch;
    u->max_h = max_h;
    u->max_w = max_w;
    if (cuda_stream) {
        u->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
        cudaError_t e = cudaStreamCreateWithFlags(&u->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete u;
            return cuda_fail(e, "cudaStreamCreate");
        }
        u->own_stream = true;
    }
    // layers in parameter order
    long long off = 0;
    auto add = [&](int co, int ci, int k) {
        UnetLayer L;
        L.co = co;
        L.ci = ci;
        L.cpad = ci == UNET_IN ? UNET_PAD0 : ci;
        L.k = k;
        L.off = off;
        off += (long long)co * k * k * ci + co;
        u->layers.push_back(L);
    };
    for (int l = 0; l < levels; ++l) {
        add(base << l, l == 0 ? UNET_IN : base << (l - 1), 3);
        add(base << l, base << l, 3);
    }
    for (int l = levels - 2; l >= 0; --l) {
        add(base << l, (base << l) + (base << (l + 1)), 3);
        add(base << l, base << l, 3);
    }
    add(1, base, 1);
    u->nparam = off;
    const long long P = (long long)max_batch * max_h * max_w;
    int rc = MCLBM_OK;
    auto A = [&](void **p, size_t bytes) {
        if (rc == MCLBM_OK) rc = ualloc(*u, p, bytes);
    };
    A((void **)&u->theta, u->nparam * 4);
    A((void **)&u->grad, u->nparam * 4);
    A((void **)&u->m, u->nparam * 4);
    A((void **)&u->v, u->nparam * 4);
    for (auto &L : u->layers) {
        if (L.k != 3) continue;
        A((void **)&L.wf, (size_t)L.co * 9 * L.cpad * 2);
        A((void **)&L.wt, (size_t)L.co * 9 * L.cpad * 2);
        A((void **)&L.wpf, (size_t)L.co * 9 * L.cpad * 2);
        A((void **)&L.wpt, (size_t)L.co * 9 * L.cpad * 2);
        A((void **)&L.dw, (size_t)L.co * 9 * L.cpad * 4);
    }
    u->a_in.assign(levels, nullptr);
    u->e_ha.assign(levels, nullptr);
    u->e_out.assign(levels, nullptr);
    u->d_ha.assign(levels, nullptr);
    u->d_out.assign(levels, nullptr);
    u->up.assign(levels, nullptr);
    u->de.assign(levels, nullptr);
    for (int l = 0; l < levels; ++l) {
        const long long Pl = P >> (2 * l);
        const int cl = base << l;
        A((void **)&u->a_in[l], (size_t)Pl * (l == 0 ? UNET_PAD0 : base << (l - 1)) * 2);
        A((void **)&u->e_ha[l], (size_t)Pl * cl * 2);
        A((void **)&u->e_out[l], (size_t)Pl * cl * 2);
        A((void **)&u->de[l], (size_t)Pl * cl * 4);
        if (l < levels - 1) {
            A((void **)&u->d_ha[l], (size_t)Pl * cl * 2);
            A((void **)&u->d_out[l], (size_t)Pl * cl * 2);
            if (l == 0) A((void **)&u->up[l], (size_t)Pl * 2 * cl * 2);
        }
    }
    A((void **)&u->phi, P * 4);
    A((void **)&u->s1, (size_t)P * 3 * base * 4);
    A((void **)&u->s2, (size_t)P * UNET_PAD0 * 4 + (size_t)P * base * 4);
    A((void **)&u->dd, (size_t)P * base * 4);
    A((void **)&u->z, (size_t)P * base * 2);
    A((void **)&u->z2, (size_t)P * base * 2);
    A((void **)&u->xin_f, (size_t)P * 4 * 4);
    A((void **)&u->t_f, (size_t)P * 4);
    A((void **)&u->mask_f, (size_t)P * 4);
    A((void **)&u->loss_part, LOSS_BLOCKS * 2 * sizeof(double));
    A((void **)&u->loss_stat, 2 * sizeof(double));
    A((void **)&u->err, sizeof(int));
    // the shared-tap kernel's partial sums: one block per CTA, and a launch
    // has at least one CTA per (32-channel slice, 32-channel chunk) pair
    u->wg_part_ctas = sm_count();
    for (const auto &L : u->layers)
        if (L.k == 3 && L.co % 32 == 0 && L.co <= WT_MAX_CO)
            u->wg_part_ctas = std::max(u->wg_part_ctas, (L.co / 32) * (L.cpad / 32));
    A((void **)&u->wg_part, (size_t)u->wg_part_ctas * WT_PART * sizeof(float));
    if (rc == MCLBM_OK) {
        cudaError_t e = cudaMemsetAsync(u->theta, 0, u->nparam * 4, u->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(u->m, 0, u->nparam * 4, u->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(u->v, 0, u->nparam * 4, u->stream);
        if (e == cudaSuccess) e = cudaMemsetAsync(u->err, 0, sizeof(int), u->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(u->stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "unet initialisation");
    }
    if (rc != MCLBM_OK) {
        unet_release(u);
        return rc;
    }
    *out = u;
    return MCLBM_OK;
}

int mclbm_unet_destroy(mclbm_unet *u) {
    unet_release(u);
    return MCLBM_OK;
}

int mclbm_unet_param_count(const mclbm_unet *u, int64_t *n) {
    if (!u || !n) return fail(MCLBM_ERR_ARG, "NULL argument");
    *n = u->nparam;
    return MCLBM_OK;
}

int mclbm_unet_set_max_ctas(mclbm_unet *u, int n) {
    if (!u || n < 0) return fail(MCLBM_ERR_ARG, "NULL network or negative bound");
    u->max_ctas = n;
    return MCLBM_OK;
}

int mclbm_unet_set_shared_taps(mclbm_unet *u, int enable) {
    if (!u || (enable != 0 && enable != 1)) return fail(MCLBM_ERR_ARG, "NULL network or flag not 0/1");
    u->shared_taps = enable;
    return MCLBM_OK;
}

int mclbm_unet_set_params(mclbm_unet *u, const float *theta) {
    if (!u || !theta) return fail(MCLBM_ERR_ARG, "NULL argument");
    cudaError_t e = stage_in(*u, u->theta, theta, (size_t)u->nparam);
    if (e == cudaSuccess) e = cudaMemsetAsync(u->m, 0, u->nparam * 4, u->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(u->v, 0, u->nparam * 4, u->stream);
    if (e == cudaSuccess) e = refresh_weights(*u);
    if (e == cudaSuccess) e = cudaStreamSynchronize(u->stream);
    if (e != cudaSuccess) return cuda_fail(e, "unet parameters");
    u->adam_t = 0;
    return MCLBM_OK;
}

int mclbm_unet_get_params(mclbm_unet *u, float *theta) {
    if (!u || !theta) return fail(MCLBM_ERR_ARG, "NULL argument");
    cudaError_t e = stage_out(*u, theta, u->theta, (size_t)u->nparam);
    if (e == cudaSuccess) e = cudaStreamSynchronize(u->stream);
    if (e != cudaSuccess) return cuda_fail(e, "unet parameters");
    return MCLBM_OK;
}

int mclbm_unet_infer(mclbm_unet *u, int batch, int h, int w, const float *x, float *phi) {
    if (int rc = check_shape(u, batch, h, w)) return rc;
    if (!x || !phi) return fail(MCLBM_ERR_ARG, "NULL argument");
    if (int rc = run_forward(u, batch, h, w, x, nullptr, nullptr)) return rc;
    cudaError_t e = stage_out(*u, phi, u->phi, (size_t)batch * h * w);
    if (e == cudaSuccess) e = cudaStreamSynchronize(u->stream);
    if (e != cudaSuccess) return cuda_fail(e, "unet output");
    return check_err(u);
}

int mclbm_unet_gradient(mclbm_unet *u, int batch, int h, int w, const float *x, const float *target,
                        const float *mask, double *loss, float *grad) {
    if (int rc = check_shape(u, batch, h, w)) return rc;
    if (!x || !target || !mask) return fail(MCLBM_ERR_ARG, "NULL argument");
    if (int rc = run_forward(u, batch, h, w, x, target, mask)) return rc;
    cudaError_t e = backward(*u, batch, h, w);
    if (e != cudaSuccess) return cuda_fail(e, "unet backward");
    if (grad && (e = stage_out(*u, grad, u->grad, (size_t)u->nparam)) != cudaSuccess)
        return cuda_fail(e, "unet gradient copy");
    return read_loss(u, loss);
}

int mclbm_unet_train_step(mclbm_unet *u, int batch, int h, int w, const float *x, const float *target,
                          const float *mask, double lr, double *loss) {
    if (int rc = check_shape(u, batch, h, w)) return rc;
    if (!x || !target || !mask) return fail(MCLBM_ERR_ARG, "NULL argument");
    if (!(lr > 0) || !std::isfinite(lr)) return fail(MCLBM_ERR_ARG, "learning rate must be positive");
    if (int rc = run_forward(u, batch, h, w, x, target, mask)) return rc;
    cudaError_t e = backward(*u, batch, h, w);
    if (e != cudaSuccess) return cuda_fail(e, "unet backward");
    ++u->adam_t;
    const float b1 = 0.9f, b2 = 0.999f;
    const float bc1 = (float)(1.0 - std::pow(0.9, (double)u->adam_t));
    const float bc2 = (float)(1.0 - std::pow(0.999, (double)u->adam_t));
    adam_kernel<<<blocks_for(u->nparam), 256, 0, u->stream>>>(u->theta, u->grad, u->m, u->v, u->nparam, (float)lr,
                                                             b1, b2, 1e-8f, bc1, bc2);
    count_launch();
    if ((e = cudaGetLastError()) != cudaSuccess || (e = refresh_weights(*u)) != cudaSuccess)
        return cuda_fail(e, "unet update");
    return read_loss(u, loss);
}

}  // extern "C"
