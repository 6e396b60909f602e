// Level-set branch of DevelSet-Net (Sec. III-B): a 4-level convolutional
// encoder-decoder that maps the band-limited TSDF of a target to an initial level set
// for DSO, with its training step (MSE to the level set DSO converges to, Adam).
//
// Layers (width c): per encoder level two 3x3 convolutions (zero padding, bias, ReLU)
// of widths c, 2c, 4c, 8c with 2x2 average pooling between levels; per decoder level
// nearest 2x upsampling, concatenation [upsampled, encoder skip] and two 3x3
// convolutions; a 1x1 head added to the input (y = x + head). Tensors are NCHW;
// activations are stored in BF16, weights used in BF16 (FP32 master copy, updated by
// Adam), every sum accumulates in FP32; gradients are FP32 in memory (rounded to BF16
// where they enter a tensor-core convolution).
//
// Kernels: k_conv3_mma (on the tensor cores, warp-level BF16 MMA: the forward
// convolutions, and the input gradients as convolutions of the output gradients with
// the flipped, transposed weights); SIMT: k_conv3_wgrad (weight and bias gradients per
// spatial tile) + k_wgrad_reduce (fixed-order sum over tiles), k_relu_mask, pooling /
// upsampling and their adjoints, the head, the MSE and Adam. Every reduction runs in a
// fixed order: results are reproducible.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "conv_tc.cuh"
#include "tc_ptx.cuh"

struct devel_dsn;

namespace devel {
namespace {

using bf16 = __nv_bfloat16;
constexpr int kT = 16;      // output tile side
constexpr int kWC = 16;     // channels per block side (weight gradients)

__device__ __forceinline__ float ld(const bf16* p, size_t i) { return __bfloat162float(p[i]); }

// Forward 3x3 convolution on the tensor cores (warp-level BF16 MMA, FP32 accumulate):
// an implicit GEMM with M = 128 output pixels (4 rows x 32 columns), N = 64 output
// channels, K = 16 input channels x 9 taps per step. The input tile (6 x 34 pixels x 16
// channels, channel innermost, padded to 24 so ldmatrix rows hit distinct banks) and
// the step's weights Wm[cb][tap][co][16] are staged in shared memory; warp w computes
// row w % 4 (two 16-pixel fragments) for 32 channels (four 8-channel fragments).
constexpr int kMRows = 4, kMCols = 32, kMCo = 64, kMPad = 24;
__device__ __forceinline__ void ldsm_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}
__device__ __forceinline__ void mma_16816(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Shared memory of k_conv3_mma: two stages (input tile and weights) so that the global
// loads of channel block cb + 1 are in flight while block cb's MMAs run.
constexpr int kMTile = (kMRows + 2) * (kMCols + 2) * kMPad;  // bf16 elements
constexpr int kMW = 9 * kMCo * kMPad;
constexpr size_t kMSmem = 2 * (size_t)(kMTile + kMW) * sizeof(bf16);
constexpr int kMPairs = 16 * (kMRows + 2) * ((kMCols + 4) / 2);  // bf16 pairs of a tile (columns x0-2 .. x0+33)
constexpr int kMPairPT = (kMPairs + 255) / 256;
constexpr int kMWPT = (9 * kMCo * 2 + 255) / 256;                // uint4 of weights per thread

// Tin = bf16: the forward (bias, ReLU, bf16 output). Tin = float: the input gradient of a
// forward layer (the output gradient, rounded to bf16 on the way into shared memory,
// convolved with the flipped, transposed weights), FP32 output split along channels
// into YA (the first CYA) and YB, stored or added.
__device__ __forceinline__ uint32_t pair_bits(const bf16* p) { return *reinterpret_cast<const uint32_t*>(p); }
__device__ __forceinline__ uint32_t pair_bits(const float* p) {
    const float2 v = *reinterpret_cast<const float2*>(p);
    const __nv_bfloat162 b = __floats2bfloat162_rn(v.x, v.y);
    return *reinterpret_cast<const uint32_t*>(&b);
}
__device__ __forceinline__ unsigned short one_bits(const bf16* p) { return __bfloat16_as_ushort(*p); }
__device__ __forceinline__ unsigned short one_bits(const float* p) { return __bfloat16_as_ushort(__float2bfloat16_rn(*p)); }

template <typename Tin, bool kBf16Out>
__global__ void __launch_bounds__(256)
k_conv3_mma(const Tin* __restrict__ XA, int CA, const Tin* __restrict__ XB, int CB, const bf16* __restrict__ Wm,
            int Coutp, const float* __restrict__ bias, int relu, void* YA, int CYA, float* YB, int accumulate, int H,
            int Wd, int Cout) {
    extern __shared__ __align__(16) uint8_t msm[];
    bf16* patch_s = reinterpret_cast<bf16*>(msm);                  // [2][rows + 2][cols + 2][kMPad]
    bf16* w_s = patch_s + 2 * kMTile;                              // [2][9][kMCo][kMPad]
    const int tilesx = (Wd + kMCols - 1) / kMCols;
    const int x0 = (blockIdx.x % tilesx) * kMCols, y0 = (blockIdx.x / tilesx) * kMRows;
    const int co0 = blockIdx.y * kMCo, n = blockIdx.z;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = warp & 3, wn = warp >> 2;
    const int Cin = CA + CB, ncb = (Cin + 15) / 16;
    const size_t plane = (size_t)H * Wd;
    constexpr int kRowPairs = (kMCols + 4) / 2, kTilePairs = (kMRows + 2) * kRowPairs;
    uint32_t pv[kMPairPT];
    uint4 wv[kMWPT];
    auto pix = [&](int ci, int gy, int gx) -> unsigned short {
        if (ci >= Cin || gy < 0 || gy >= H || gx < 0 || gx >= Wd) return 0;
        const size_t off = (size_t)gy * Wd + gx;
        return one_bits(ci < CA ? XA + ((size_t)n * CA + ci) * plane + off
                                : XB + ((size_t)n * CB + (ci - CA)) * plane + off);
    };
    // global -> registers: the tile as bf16 pairs (columns x0-2+2p, x0-1+2p), and the weights
    auto load = [&](int cb) {
#pragma unroll
        for (int k = 0; k < kMPairPT; ++k) {
            const int i = threadIdx.x + k * 256;
            uint32_t v = 0;
            if (i < kMPairs) {
                const int c = i / kTilePairs, rp = i % kTilePairs, r = rp / kRowPairs, p = rp % kRowPairs;
                const int ci = cb * 16 + c, gy = y0 + r - 1, gx = x0 - 2 + 2 * p;
                if (ci < Cin && gy >= 0 && gy < H && gx >= 0 && gx + 1 < Wd) {
                    const size_t off = (size_t)gy * Wd + gx;
                    const Tin* src = ci < CA ? XA + ((size_t)n * CA + ci) * plane + off
                                             : XB + ((size_t)n * CB + (ci - CA)) * plane + off;
                    v = pair_bits(src);
                } else {
                    v = (uint32_t)pix(ci, gy, gx) | ((uint32_t)pix(ci, gy, gx + 1) << 16);
                }
            }
            pv[k] = v;
        }
        const uint4* wg = reinterpret_cast<const uint4*>(Wm + ((size_t)cb * 9 * Coutp + co0) * 16);
#pragma unroll
        for (int k = 0; k < kMWPT; ++k) {
            const int i = threadIdx.x + k * 256;
            if (i < 9 * kMCo * 2) {
                const int tap = i / (kMCo * 2), co = (i / 2) % kMCo, h = i & 1;
                wv[k] = wg[((size_t)tap * Coutp + co) * 2 + h];
            }
        }
    };
    // registers -> stage st of shared memory (tile channel innermost)
    auto store = [&](int st) {
        bf16* pt = patch_s + st * kMTile;
#pragma unroll
        for (int k = 0; k < kMPairPT; ++k) {
            const int i = threadIdx.x + k * 256;
            if (i < kMPairs) {
                const int c = i / kTilePairs, rp = i % kTilePairs, r = rp / kRowPairs, p = rp % kRowPairs;
                const int q0 = 2 * p - 1, q1 = 2 * p;  // tile columns of the pair (x0 - 1 is column 0)
                if (q0 >= 0) pt[(r * (kMCols + 2) + q0) * kMPad + c] = __ushort_as_bfloat16((unsigned short)(pv[k] & 0xffff));
                if (q1 < kMCols + 2)
                    pt[(r * (kMCols + 2) + q1) * kMPad + c] = __ushort_as_bfloat16((unsigned short)(pv[k] >> 16));
            }
        }
        bf16* wt = w_s + st * kMW;
#pragma unroll
        for (int k = 0; k < kMWPT; ++k) {
            const int i = threadIdx.x + k * 256;
            if (i < 9 * kMCo * 2) {
                const int tap = i / (kMCo * 2), co = (i / 2) % kMCo, h = i & 1;
                *reinterpret_cast<uint4*>(wt + (tap * kMCo + co) * kMPad + 8 * h) = wv[k];
            }
        }
    };
    float acc[2][4][4];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[a][b][e] = 0.f;
    load(0);
    store(0);
    __syncthreads();
    for (int cb = 0; cb < ncb; ++cb) {
        const int st = cb & 1;
        if (cb + 1 < ncb) load(cb + 1);  // in flight during this block's MMAs
        const bf16* pt = patch_s + st * kMTile;
        const bf16* wt = w_s + st * kMW;
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
            const int dy = tap / 3, dx = tap % 3;
            uint32_t a[2][4], b[4][2];
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) {
                const int mat = lane >> 3, r = lane & 7;
                const int m = (mat & 1) * 8 + r, koff = (mat >> 1) * 8;
                ldsm_x4(tc::smem_u32(pt + ((wm + dy) * (kMCols + 2) + 16 * mi + m + dx) * kMPad + koff), a[mi][0],
                        a[mi][1], a[mi][2], a[mi][3]);
            }
#pragma unroll
            for (int pp = 0; pp < 2; ++pp) {
                const int mat = lane >> 3, r = lane & 7;
                const int co = wn * 32 + 16 * pp + (mat >> 1) * 8 + r, koff = (mat & 1) * 8;
                ldsm_x4(tc::smem_u32(wt + (tap * kMCo + co) * kMPad + koff), b[2 * pp][0], b[2 * pp][1],
                        b[2 * pp + 1][0], b[2 * pp + 1][1]);
            }
#pragma unroll
            for (int mi = 0; mi < 2; ++mi)
#pragma unroll
                for (int nj = 0; nj < 4; ++nj) mma_16816(acc[mi][nj], a[mi], b[nj][0], b[nj][1]);
        }
        if (cb + 1 < ncb) store(st ^ 1);  // the other stage was last read before the previous barrier
        __syncthreads();
    }
    const int g = lane >> 2, cpair = 2 * (lane & 3);
    const int y = y0 + wm;
    if (y >= H) return;
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int nj = 0; nj < 4; ++nj)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int x = x0 + 16 * mi + g + (e >> 1) * 8;
                const int co = co0 + wn * 32 + 8 * nj + cpair + (e & 1);
                if (x >= Wd || co >= Cout) continue;
                const size_t off = (size_t)y * Wd + x;
                if (kBf16Out) {
                    float v = acc[mi][nj][e] + (bias ? bias[co] : 0.f);
                    if (relu) v = fmaxf(v, 0.f);
                    static_cast<bf16*>(YA)[((size_t)n * Cout + co) * plane + off] = __float2bfloat16_rn(v);
                } else {
                    const float v = acc[mi][nj][e];
                    float* dst = co < CYA ? static_cast<float*>(YA) + ((size_t)n * CYA + co) * plane + off
                                          : YB + ((size_t)n * (Cout - CYA) + (co - CYA)) * plane + off;
                    *dst = accumulate ? *dst + v : v;
                }
            }
}

// weights of a 3x3 layer for k_conv3_mma: Wm[cb][tap][co < Coutp][16] (zero past Cin / Cout);
// transposed: the layer seen from its output gradient (co <-> ci, taps mirrored), so the
// same kernel computes the input gradient
template <bool kT>
__global__ void k_prep_wm(const float* __restrict__ W, int CoutF, int CinF, int Coutp, bf16* __restrict__ Wm) {
    const int Cout = kT ? CinF : CoutF, Cin = kT ? CoutF : CinF;
    const int ncb = (Cin + 15) / 16;
    const size_t count = (size_t)ncb * 9 * Coutp * 16;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(i % 16);
        const size_t r = i / 16;
        const int co = (int)(r % Coutp), tap = (int)((r / Coutp) % 9), cb = (int)(r / ((size_t)Coutp * 9));
        const int ci = cb * 16 + j;
        float v = 0.f;
        if (co < Cout && ci < Cin)
            v = kT ? W[((size_t)ci * CinF + co) * 9 + (8 - tap)] : W[((size_t)co * Cin + ci) * 9 + tap];
        Wm[i] = __float2bfloat16_rn(v);
    }
}

// Per spatial tile: part[tile][co][ci][9] = sum_n sum_{tile px} dZ[n][co][p] X[n][ci][p + tap],
// and (blocks of the first input-channel group) bpart[tile][co] = sum_n sum_{tile px} dZ.
// A thread (co, ci) slides a 3 x 3 register window along each row of its tile: per
// pixel one dZ value and one new input column (4 shared-memory loads for 9 FMAs).
template <typename Tin>
__global__ void __launch_bounds__(256)
k_conv3_wgrad(const Tin* __restrict__ XA, int CA, const Tin* __restrict__ XB, int CB, const float* __restrict__ dZ,
              int Cout, int N, int H, int Wd, float* __restrict__ part, float* __restrict__ bpart) {
    __shared__ float dz[kWC][kT][kT];
    __shared__ float xp[kWC][kT + 2][kT + 2];
    const int tilesx = (Wd + kT - 1) / kT;
    const int tile = blockIdx.x;
    const int x0 = (tile % tilesx) * kT, y0 = (tile / tilesx) * kT;
    const int co0 = blockIdx.y * kWC, ci0 = blockIdx.z * kWC;
    const int col = threadIdx.x / kWC, cil = threadIdx.x % kWC;
    const int Cin = CA + CB;
    const size_t plane = (size_t)H * Wd;
    float acc[9], bsum = 0.f;
#pragma unroll
    for (int t = 0; t < 9; ++t) acc[t] = 0.f;
    constexpr int kDz = kWC * kT * kT, kXp = kWC * (kT + 2) * (kT + 2);
    for (int n = 0; n < N; ++n) {
#pragma unroll 8
        for (int k = 0; k < kDz / 256; ++k) {
            const int i = threadIdx.x + k * 256;
            const int c = i / (kT * kT), r = (i / kT) % kT, q = i % kT;
            const int o = co0 + c, gy = y0 + r, gx = x0 + q;
            (&dz[0][0][0])[i] = (o < Cout && gy < H && gx < Wd)
                                    ? dZ[((size_t)n * Cout + o) * plane + (size_t)gy * Wd + gx]
                                    : 0.f;
        }
#pragma unroll 8
        for (int k = 0; k < (kXp + 255) / 256; ++k) {
            const int i = threadIdx.x + k * 256;
            const int c = i / ((kT + 2) * (kT + 2)), r = (i / (kT + 2)) % (kT + 2), q = i % (kT + 2);
            const int ci = ci0 + c, gy = y0 + r - 1, gx = x0 + q - 1;
            float v = 0.f;
            if (i < kXp && ci < Cin && gy >= 0 && gy < H && gx >= 0 && gx < Wd) {
                const size_t off = (size_t)gy * Wd + gx;
                v = ci < CA ? ld(XA, ((size_t)n * CA + ci) * plane + off)
                            : ld(XB, ((size_t)n * CB + (ci - CA)) * plane + off);
            }
            if (i < kXp) (&xp[0][0][0])[i] = v;
        }
        __syncthreads();
        for (int r = 0; r < kT; ++r) {
            float w0[3], w1[3];
#pragma unroll
            for (int u = 0; u < 3; ++u) {
                w0[u] = xp[cil][r + u][0];
                w1[u] = xp[cil][r + u][1];
            }
#pragma unroll
            for (int q = 0; q < kT; ++q) {
                float w2[3];
#pragma unroll
                for (int u = 0; u < 3; ++u) w2[u] = xp[cil][r + u][q + 2];
                const float d = dz[col][r][q];
                bsum += d;
#pragma unroll
                for (int u = 0; u < 3; ++u) {
                    acc[3 * u + 0] = fmaf(d, w0[u], acc[3 * u + 0]);
                    acc[3 * u + 1] = fmaf(d, w1[u], acc[3 * u + 1]);
                    acc[3 * u + 2] = fmaf(d, w2[u], acc[3 * u + 2]);
                }
#pragma unroll
                for (int u = 0; u < 3; ++u) {
                    w0[u] = w1[u];
                    w1[u] = w2[u];
                }
            }
        }
        __syncthreads();
    }
    const int o = co0 + col, ci = ci0 + cil;
    if (o < Cout && ci < Cin) {
        float* dst = part + (((size_t)tile * Cout + o) * Cin + ci) * 9;
#pragma unroll
        for (int t = 0; t < 9; ++t) dst[t] = acc[t];
    }
    if (blockIdx.z == 0 && cil == 0 && o < Cout) bpart[(size_t)tile * Cout + o] = bsum;
}

// G[i] = sum over tiles of part[tile][i], in tile order
__global__ void k_wgrad_reduce(const float* __restrict__ part, int ntiles, size_t count, float* __restrict__ G) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    float s = 0.f;
    for (int t = 0; t < ntiles; ++t) s += part[(size_t)t * count + i];
    G[i] = s;
}

// fixed-order block sum of 256 values; valid in thread 0
__device__ __forceinline__ float block_sum256(float v, float* sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    float s = 0.f;
    if (threadIdx.x == 0)
        for (int i = 0; i < 8; ++i) s += sh[i];
    return s;
}

__global__ void k_relu_mask(float* __restrict__ dZ, const bf16* __restrict__ out, size_t count) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        if (!(__bfloat162float(out[i]) > 0.f)) dZ[i] = 0.f;
}

__global__ void k_avgpool(const bf16* __restrict__ X, int H, int Wd, size_t planes, bf16* __restrict__ Y) {
    const int h = H / 2, w = Wd / 2;
    const size_t count = planes * h * w;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        const size_t pl = i / ((size_t)h * w);
        const int r = (int)((i / w) % h), q = (int)(i % w);
        const bf16* p = X + pl * H * Wd + (size_t)(2 * r) * Wd + 2 * q;
        const float s = (__bfloat162float(p[0]) + __bfloat162float(p[1])) +
                        (__bfloat162float(p[Wd]) + __bfloat162float(p[Wd + 1]));
        Y[i] = __float2bfloat16_rn(0.25f * s);
    }
}

// The same pooling, four outputs of one row per thread from two 16-byte loads (8 inputs of
// each of its two input rows), the same sums in the same order; rows = planes * (H / 2),
// w = Wd / 2 a multiple of 4.
__global__ void k_avgpool4(const bf16* __restrict__ X, int w, size_t rows, bf16* __restrict__ Y) {
    const int wq = w >> 2;
    const size_t count = rows * wq;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        const size_t row = i / wq;
        const int q4 = (int)(i - row * wq);
        const bf16* p0 = X + (2 * row) * (size_t)(2 * w) + 8 * q4;
        const uint4 a = *reinterpret_cast<const uint4*>(p0);
        const uint4 b = *reinterpret_cast<const uint4*>(p0 + 2 * w);
        const bf16* ha = reinterpret_cast<const bf16*>(&a);
        const bf16* hb = reinterpret_cast<const bf16*>(&b);
        __align__(8) bf16 o[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float sum = (__bfloat162float(ha[2 * j]) + __bfloat162float(ha[2 * j + 1])) +
                              (__bfloat162float(hb[2 * j]) + __bfloat162float(hb[2 * j + 1]));
            o[j] = __float2bfloat16_rn(0.25f * sum);
        }
        *reinterpret_cast<uint2*>(Y + row * w + 4 * q4) = *reinterpret_cast<const uint2*>(o);
    }
}

// The first convolution (one input channel): Y[n][co] = ReLU(b[co] + sum_tap w[co][tap] X[n]
// shifted by the tap), zero padding, weights rounded to BF16 as on the tensor-core path,
// FP32 sums, BF16 output. A thread computes 8 consecutive pixels of one row for every
// output channel from its 3 x 10 input window (the tensor-core kernels would pad the one
// channel to 16). side % 8 == 0, Cout <= kC1Max.
constexpr int kC1Max = 64;
__global__ void __launch_bounds__(256) k_conv3_c1(const bf16* __restrict__ X, const float* __restrict__ W,
                                                 const float* __restrict__ bias, int Cout, int side, int nb,
                                                 bf16* __restrict__ Y) {
    __shared__ float ws[kC1Max * 9], bs[kC1Max];
    for (int i = threadIdx.x; i < Cout * 9; i += blockDim.x) ws[i] = __bfloat162float(__float2bfloat16_rn(W[i]));
    for (int i = threadIdx.x; i < Cout; i += blockDim.x) bs[i] = bias[i];
    __syncthreads();
    const size_t plane = (size_t)side * side;
    const int q8 = side / 8;
    const size_t count = (size_t)nb * side * q8;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        const size_t row = i / q8;                     // n * side + y
        const int x0 = 8 * (int)(i - row * q8);
        const size_t n = row / side;
        const int y = (int)(row - n * side);
        const bf16* Xn = X + n * plane;
        float win[3][10];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const int yy = y + r - 1;
            if (yy < 0 || yy >= side) {
#pragma unroll
                for (int j = 0; j < 10; ++j) win[r][j] = 0.f;
                continue;
            }
            const bf16* xr = Xn + (size_t)yy * side;
            const uint4 v = *reinterpret_cast<const uint4*>(xr + x0);
            const bf16* h = reinterpret_cast<const bf16*>(&v);
#pragma unroll
            for (int j = 0; j < 8; ++j) win[r][1 + j] = __bfloat162float(h[j]);
            win[r][0] = x0 > 0 ? __bfloat162float(xr[x0 - 1]) : 0.f;
            win[r][9] = x0 + 8 < side ? __bfloat162float(xr[x0 + 8]) : 0.f;
        }
        bf16* Yr = Y + n * Cout * plane + (size_t)y * side + x0;
        for (int co = 0; co < Cout; ++co) {
            float acc[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[j] = 0.f;
#pragma unroll
            for (int t = 0; t < 9; ++t) {
                const float wv = ws[co * 9 + t];
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[j] = fmaf(wv, win[t / 3][j + t % 3], acc[j]);
            }
            __align__(16) bf16 o[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) o[j] = __float2bfloat16_rn(fmaxf(acc[j] + bs[co], 0.f));
            *reinterpret_cast<uint4*>(Yr + co * plane) = *reinterpret_cast<const uint4*>(o);
        }
    }
}

// dX[2r+i][2q+j] (+)= dY[r][q] / 4
__global__ void k_avgpool_bwd(const float* __restrict__ dY, int H, int Wd, size_t planes, float* __restrict__ dX,
                              int accumulate) {
    const size_t count = planes * H * Wd;
    const int w = Wd / 2;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        const size_t pl = i / ((size_t)H * Wd);
        const int r = (int)((i / Wd) % H), q = (int)(i % Wd);
        const float v = 0.25f * dY[pl * (H / 2) * w + (size_t)(r / 2) * w + q / 2];
        dX[i] = accumulate ? dX[i] + v : v;
    }
}

__global__ void k_upsample(const bf16* __restrict__ X, int h, int w, size_t planes, bf16* __restrict__ Y) {
    const size_t count = planes * 4 * h * w;
    const int W2 = 2 * w;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        const size_t pl = i / ((size_t)4 * h * w);
        const int r = (int)((i / W2) % (2 * h)), q = (int)(i % W2);
        Y[i] = X[pl * h * w + (size_t)(r / 2) * w + q / 2];
    }
}

// The same copy, four source pixels of one row per thread (one 8-byte load) into 8 pixels
// of each of its two output rows (two 16-byte stores); rows = planes * h, w a multiple of 4.
__global__ void k_upsample4(const bf16* __restrict__ X, int w, size_t rows, bf16* __restrict__ Y) {
    const int wq = w >> 2;
    const size_t count = rows * wq;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        const size_t row = i / wq;
        const int q4 = (int)(i - row * wq);
        const uint2 v = *reinterpret_cast<const uint2*>(X + row * w + 4 * q4);
        const uint32_t p01 = v.x, p23 = v.y;  // bf16 pairs (x0, x1), (x2, x3)
        uint4 o;
        o.x = __byte_perm(p01, 0, 0x1010);     // x0 x0
        o.y = __byte_perm(p01, 0, 0x3232);     // x1 x1
        o.z = __byte_perm(p23, 0, 0x1010);     // x2 x2
        o.w = __byte_perm(p23, 0, 0x3232);     // x3 x3
        bf16* d = Y + (2 * row) * (size_t)(2 * w) + 8 * q4;
        *reinterpret_cast<uint4*>(d) = o;
        *reinterpret_cast<uint4*>(d + 2 * w) = o;
    }
}

// dX[r][q] = sum of the four dY values it was copied to
__global__ void k_upsample_bwd(const float* __restrict__ dY, int h, int w, size_t planes, float* __restrict__ dX) {
    const size_t count = planes * h * w;
    const int W2 = 2 * w;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        const size_t pl = i / ((size_t)h * w);
        const int r = (int)((i / w) % h), q = (int)(i % w);
        const float* p = dY + pl * 4 * h * w + (size_t)(2 * r) * W2 + 2 * q;
        dX[i] = (p[0] + p[1]) + (p[W2] + p[W2 + 1]);
    }
}

// y[n][p] = x[n][p] + b + sum_c w[c] d[n][c][p] (w rounded to BF16, the sum in channel order):
// eight pixels per thread (one 16-byte load per channel); plane a multiple of 8.
__global__ void k_head8(const float* __restrict__ x, const bf16* __restrict__ d, const float* __restrict__ w,
                        const float* __restrict__ b, int C, int N, size_t plane, float* __restrict__ y) {
    const size_t count = (size_t)N * plane / 8;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        const size_t e = 8 * i, n = e / plane, p = e - n * plane;
        float acc[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[j] = b[0];
        for (int c = 0; c < C; ++c) {
            const float wc = __bfloat162float(__float2bfloat16_rn(w[c]));
            const uint4 v = *reinterpret_cast<const uint4*>(d + (n * C + c) * plane + p);
            const bf16* h = reinterpret_cast<const bf16*>(&v);
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[j] = fmaf(wc, __bfloat162float(h[j]), acc[j]);
        }
        const float4 x0 = *reinterpret_cast<const float4*>(x + e), x1 = *reinterpret_cast<const float4*>(x + e + 4);
        *reinterpret_cast<float4*>(y + e) = make_float4(x0.x + acc[0], x0.y + acc[1], x0.z + acc[2], x0.w + acc[3]);
        *reinterpret_cast<float4*>(y + e + 4) = make_float4(x1.x + acc[4], x1.y + acc[5], x1.z + acc[6], x1.w + acc[7]);
    }
}

// dd[n][c][p] = w[c] dy[n][p]
__global__ void k_head_dgrad(const float* __restrict__ dy, const float* __restrict__ w, int C, int N, size_t plane,
                             float* __restrict__ dd) {
    const size_t count = (size_t)N * C * plane;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        const size_t p = i % plane, nc = i / plane, n = nc / C;
        const int c = (int)(nc % C);
        dd[i] = __bfloat162float(__float2bfloat16_rn(w[c])) * dy[n * plane + p];
    }
}

// Head gradients per slice of the pixels: part[split][c] = sum dy d[c] over the split's
// pixels (c < C), part[split][C] = sum dy; summed over the splits in order afterwards.
constexpr int kHeadSplits = 64;
__global__ void __launch_bounds__(256) k_head_wgrad(const float* __restrict__ dy, const bf16* __restrict__ d, int C,
                                                    int N, size_t plane, float* __restrict__ part) {
    __shared__ float sh[8];
    const int c = blockIdx.x, sp = blockIdx.y;
    const size_t total = (size_t)N * plane, i0 = total * sp / kHeadSplits, i1 = total * (sp + 1) / kHeadSplits;
    float s = 0.f;
    for (size_t i = i0 + threadIdx.x; i < i1; i += 256) {
        const float g = dy[i];
        const size_t n = i / plane, p = i % plane;
        s += c < C ? g * __bfloat162float(d[(n * C + c) * plane + p]) : g;
    }
    s = block_sum256(s, sh);
    if (threadIdx.x == 0) part[(size_t)sp * (C + 1) + c] = s;
}

// loss = mean (y - t)^2 (per-block FP32, exact fixed point across blocks), dy = 2 (y - t) / count
__global__ void __launch_bounds__(256) k_mse(const float* __restrict__ y, const float* __restrict__ t, size_t count,
                                             float* __restrict__ dy, long long* __restrict__ qpart, unsigned* counter,
                                             double* loss) {
    __shared__ float sh[8];
    __shared__ bool last;
    const float scale = 2.f / (float)count;
    float s = 0.f;
    for (size_t i = (size_t)blockIdx.x * 256 + threadIdx.x; i < count; i += (size_t)gridDim.x * 256) {
        const float d = y[i] - t[i];
        s = fmaf(d, d, s);
        dy[i] = scale * d;
    }
    s = block_sum256(s, sh);
    if (threadIdx.x == 0) {
        qpart[blockIdx.x] = to_q32(s);
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    long long q = 0;
    bool bad = false;
    for (unsigned i = 0; i < gridDim.x; ++i) {
        const long long v = __ldcg(qpart + i);
        bad |= v == kQBad;
        q += v;
    }
    *loss = bad ? __longlong_as_double(0x7ff8000000000000ll) : (double)q * (1.0 / 4294967296.0) / (double)count;
    *counter = 0u;
}

// modulation-branch loss: loss = mean (H_eps(y) - m)^2, dy = 2 (H_eps(y) - m) H_eps'(y) / count
// with H_eps(y) = 1/2 + atan(y / eps) / pi (exact fixed point across blocks)
__global__ void __launch_bounds__(256) k_ahf_mse(const float* __restrict__ y, const float* __restrict__ m, size_t count,
                                                 float eps, float* __restrict__ dy, long long* __restrict__ qpart,
                                                 unsigned* counter, double* loss) {
    __shared__ float sh[8];
    __shared__ bool last;
    const float scale = 2.f / (float)count, inv_eps = 1.f / eps;
    float s = 0.f;
    for (size_t i = (size_t)blockIdx.x * 256 + threadIdx.x; i < count; i += (size_t)gridDim.x * 256) {
        const float v = y[i];
        const float r = 0.5f + atanf(v * inv_eps) * 0.318309886f - m[i];
        s = fmaf(r, r, s);
        dy[i] = scale * r * (eps * 0.318309886f) / fmaf(v, v, eps * eps);
    }
    s = block_sum256(s, sh);
    if (threadIdx.x == 0) {
        qpart[blockIdx.x] = to_q32(s);
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    long long q = 0;
    bool bad = false;
    for (unsigned i = 0; i < gridDim.x; ++i) {
        const long long v = __ldcg(qpart + i);
        bad |= v == kQBad;
        q += v;
    }
    *loss = bad ? __longlong_as_double(0x7ff8000000000000ll) : (double)q * (1.0 / 4294967296.0) / (double)count;
    *counter = 0u;
}

__global__ void k_ahf_out(const float* __restrict__ y, size_t count, float eps, float* __restrict__ m) {
    const float inv_eps = 1.f / eps;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        m[i] = 0.5f + atanf(y[i] * inv_eps) * 0.318309886f;
}

__global__ void k_adam(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ M, float* __restrict__ V,
                       size_t count, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        const float g = G[i];
        const float m = b1 * M[i] + (1.f - b1) * g, v = b2 * V[i] + (1.f - b2) * g * g;
        M[i] = m;
        V[i] = v;
        P[i] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
    }
}

// x = clip(phi, -B, B) / B as FP32 (residual path) and BF16 (first convolution)
__global__ void k_band(const float* __restrict__ phi, size_t count, float B, float* __restrict__ x,
                       bf16* __restrict__ xb) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        const float v = fminf(fmaxf(phi[i], -B), B) / B;
        x[i] = v;
        if (xb) xb[i] = __float2bfloat16_rn(v);
    }
}

__global__ void k_scale(const float* __restrict__ y, size_t count, float s, float* __restrict__ out) {
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x)
        out[i] = s * y[i];
}

// coarse[b][I][J] = (sum of the f x f block of fine) * inv, inv = 1 / f^3; the block's
// rows in order, each left to right. Grid (coarse column blocks, coarse row I, images b in
// steps of gridDim.z): no index divisions.
__global__ void k_phi_down(const float* __restrict__ fine, int n, int f, int nb, float inv,
                           float* __restrict__ coarse) {
    const int m = n / f;
    const int J = blockIdx.x * blockDim.x + threadIdx.x, I = blockIdx.y;
    if (J >= m) return;
    for (int b = blockIdx.z; b < nb; b += gridDim.z) {
        const float* src = fine + (size_t)b * n * n + (size_t)I * f * n + (size_t)J * f;
        float s = 0.f;
        for (int u = 0; u < f; ++u)
            for (int v = 0; v < f; ++v) s += src[(size_t)u * n + v];
        coarse[((size_t)b * m + I) * m + J] = s * inv;
    }
}

// fine[b][p][q] = f * bilinear interpolation of coarse[b] at ((p + 1/2) / f - 1/2,
// (q + 1/2) / f - 1/2), coarse indices clamped to [0, m - 1]. Grid (blocks of 4 x 256
// fine columns, fine row p, images b in steps of gridDim.z); a thread writes four
// consecutive columns (one 16-byte store when n % 4 == 0).
__global__ void k_phi_up(const float* __restrict__ coarse, int n, int f, int nb, float* __restrict__ fine) {
    const int m = n / f;
    const float two_f = 2.f * (float)f, ff = (float)f;
    const int p = blockIdx.y, q0 = (blockIdx.x * blockDim.x + threadIdx.x) * 4;
    if (q0 >= n) return;
    const float yc = (float)(2 * p + 1 - f) / two_f;
    const float fy = floorf(yc), ty = yc - fy;
    const int i0 = (int)fy;
    const int ia = min(max(i0, 0), m - 1), ib = min(max(i0 + 1, 0), m - 1);
    for (int b = blockIdx.z; b < nb; b += gridDim.z) {
        const float* ca = coarse + ((size_t)b * m + ia) * m;
        const float* cb = coarse + ((size_t)b * m + ib) * m;
        float o[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int q = min(q0 + j, n - 1);
            const float xc = (float)(2 * q + 1 - f) / two_f;
            const float fx = floorf(xc), tx = xc - fx;
            const int j0 = (int)fx;
            const int ja = min(max(j0, 0), m - 1), jb = min(max(j0 + 1, 0), m - 1);
            const float top = (1.f - tx) * ca[ja] + tx * ca[jb];
            const float bot = (1.f - tx) * cb[ja] + tx * cb[jb];
            o[j] = ff * ((1.f - ty) * top + ty * bot);
        }
        float* out = fine + ((size_t)b * n + p) * n + q0;
        if ((n & 3) == 0) {
            *reinterpret_cast<float4*>(out) = make_float4(o[0], o[1], o[2], o[3]);
        } else {
            for (int j = 0; j < 4 && q0 + j < n; ++j) out[j] = o[j];
        }
    }
}

bool bad_ptr(const void* p) { return !p || (reinterpret_cast<uintptr_t>(p) & 15u); }

int grid1(size_t count) { return (int)std::max<size_t>(1, std::min<size_t>((count + 255) / 256, 152 * 16)); }

}  // namespace
}  // namespace devel

// ---------------------------------------------------------------------------
// The network object
// ---------------------------------------------------------------------------
struct devel_dsn {
    int S = 0, batch = 0, c = 0;
    struct Conv {
        int cin, cout, k;
        size_t w_off, b_off;  // into the flat parameter vector
        __nv_bfloat16* Wm = nullptr;   // tensor-core layout of the forward weights
        __nv_bfloat16* Wtm = nullptr;  // ... of the input-gradient (transposed, mirrored) weights
        int coutp = 0, cinp = 0;
        int side = 0;                  // plane side of the layer's output
        // tcgen05 forward path (conv_tc.cu), when the layer's shape allows it
        __nv_bfloat16* Wtc = nullptr;  // weights [ceil(Cin / 64)][9][Cout][64] (Cout = 32: [cb][dx][2 - dy])
        CUtensorMap mWtc;
    };
    std::vector<Conv> convs;
    size_t nparams = 0;
    float *P = nullptr, *G = nullptr, *M = nullptr, *V = nullptr;
    int t = 0;  // Adam steps taken
    // the tensor-core weight layouts (Wm, Wtm) no longer match P: rebuilt by the next pass
    // (set when the parameters change: init, set_params, every Adam step)
    bool wm_stale = true;
    // activations (bf16) and their gradients (fp32): index by name below
    struct Act {
        int C, side;
        __nv_bfloat16* a = nullptr;
        float* g = nullptr;
    };
    std::vector<Act> acts;
    float* x = nullptr;     // [batch][S][S] band-limited input (fp32)
    __nv_bfloat16* xb = nullptr;
    float* y = nullptr;     // network output
    float* dy = nullptr;
    float* part = nullptr;  // weight-gradient partials
    size_t part_count = 0;
    long long* qpart = nullptr;
    unsigned* counter = nullptr;
    double* loss = nullptr;
};

namespace devel {
namespace {

enum ActId { A0, S0, P1, A1, S1, P2, A2, S2, P3, A3, S3, U2, D2A, D2, U1, D1A, D1, U0, D0A, D0, NACT };

void free_dsn(devel_dsn* d) {
    if (!d) return;
    for (auto& cv : d->convs) {
        cudaFree(cv.Wm);
        cudaFree(cv.Wtm);
        if (cv.Wtc) cudaFree(cv.Wtc);
    }
    for (auto& a : d->acts) {
        cudaFree(a.a);
        cudaFree(a.g);
    }
    for (void* p : {(void*)d->P, (void*)d->G, (void*)d->M, (void*)d->V, (void*)d->x, (void*)d->xb, (void*)d->y,
                    (void*)d->dy, (void*)d->part, (void*)d->qpart, (void*)d->counter, (void*)d->loss})
        if (p) cudaFree(p);
    delete d;
}

int conv_fwd(devel_dsn* d, int ci, int nb, const __nv_bfloat16* XA, int CA, const __nv_bfloat16* XB, int CB, int side,
             __nv_bfloat16* Y, cudaStream_t s) {
    const auto& cv = d->convs[ci];
    if (cv.cin == 1 && CA == 1 && !XB && side % 8 == 0 && cv.cout <= kC1Max) {
        prof_begin(PK_DSN_CONV, s);
        k_conv3_c1<<<grid1((size_t)nb * side * side / 8), 256, 0, s>>>(XA, d->P + cv.w_off, d->P + cv.b_off, cv.cout,
                                                                       side, nb, Y);
        prof_end(PK_DSN_CONV, s);
        DEVEL_LAUNCH_CHECK("k_conv3_c1");
        return DEVEL_OK;
    }
    if (cv.Wtc && side == cv.side) {
        prof_begin(PK_DSN_CONV, s);
        const int rc = launch_conv3_tc(XA, CA, XB, CB, cv.mWtc, d->P + cv.b_off, Y, cv.cout, nb, side, s);
        prof_end(PK_DSN_CONV, s);
        return rc;
    }
    const int mtiles = ((side + kMCols - 1) / kMCols) * ((side + kMRows - 1) / kMRows);
    dim3 grid(mtiles, cv.coutp / kMCo, nb);
    prof_begin(PK_DSN_CONV, s);
    k_conv3_mma<__nv_bfloat16, true><<<grid, 256, kMSmem, s>>>(XA, CA, XB, CB, cv.Wm, cv.coutp, d->P + cv.b_off, 1, Y,
                                                               cv.cout, nullptr, 0, side, side, cv.cout);
    prof_end(PK_DSN_CONV, s);
    DEVEL_LAUNCH_CHECK("k_conv3_mma");
    return DEVEL_OK;
}

// backward of conv ci: dZ (= dY masked by the ReLU of Y, in place), weight and bias
// gradients, and (if dXA) the input gradient split into dXA / dXB (stored or added)
int conv_bwd(devel_dsn* d, int ci, int nb, const __nv_bfloat16* XA, int CA, const __nv_bfloat16* XB, int CB, int side,
             const __nv_bfloat16* Y, float* dY, float* dXA, float* dXB, int accumulate, cudaStream_t s) {
    const auto& cv = d->convs[ci];
    const size_t plane = (size_t)side * side;
    const size_t cnt = (size_t)nb * cv.cout * plane;
    k_relu_mask<<<grid1(cnt), 256, 0, s>>>(dY, Y, cnt);
    const int tiles = ((side + kT - 1) / kT) * ((side + kT - 1) / kT);
    dim3 gw(tiles, (cv.cout + kWC - 1) / kWC, (cv.cin + kWC - 1) / kWC);
    const size_t wc = (size_t)cv.cout * cv.cin * 9;
    float* bpart = d->part + (size_t)tiles * wc;
    k_conv3_wgrad<__nv_bfloat16><<<gw, 256, 0, s>>>(XA, CA, XB, CB, dY, cv.cout, nb, side, side, d->part, bpart);
    k_wgrad_reduce<<<(unsigned)((wc + 255) / 256), 256, 0, s>>>(d->part, tiles, wc, d->G + cv.w_off);
    k_wgrad_reduce<<<(unsigned)((cv.cout + 255) / 256), 256, 0, s>>>(bpart, tiles, (size_t)cv.cout,
                                                                     d->G + cv.b_off);
    if (dXA) {  // shared-memory attributes of both instances set at creation (mma_init_attrs)
        const int mtiles = ((side + kMCols - 1) / kMCols) * ((side + kMRows - 1) / kMRows);
        dim3 gd(mtiles, cv.cinp / kMCo, nb);
        k_conv3_mma<float, false><<<gd, 256, kMSmem, s>>>(dY, cv.cout, (const float*)nullptr, 0, cv.Wtm, cv.cinp,
                                                          nullptr, 0, dXA, CA, dXB, accumulate, side, side, cv.cin);
    }
    DEVEL_LAUNCH_CHECK("dsn conv backward");
    return DEVEL_OK;
}

// shared-memory opt-in of the warp-level MMA convolution (forward and input-gradient
// instances), once per device, at network creation: the input gradients need it even when
// every forward layer runs on the tensor-core kernel
int mma_init_attrs() {
    DEVEL_CUDA_TRY(cudaFuncSetAttribute(k_conv3_mma<__nv_bfloat16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)kMSmem));
    DEVEL_CUDA_TRY(cudaFuncSetAttribute(k_conv3_mma<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)kMSmem));
    return DEVEL_OK;
}

int prep_weights(devel_dsn* d, cudaStream_t s) {
    if (!d->wm_stale) return DEVEL_OK;
    prof_begin(PK_DSN_MISC, s);
    for (auto& cv : d->convs) {
        if (cv.k != 3) continue;
        if (cv.Wtc) {
            const int rc = launch_prep_wtc(d->P + cv.w_off, cv.cout, cv.cin, cv.Wtc, s);
            if (rc) return rc;
        }
        const size_t wm = (size_t)((cv.cin + 15) / 16) * 9 * cv.coutp * 16;
        k_prep_wm<false><<<grid1(wm), 256, 0, s>>>(d->P + cv.w_off, cv.cout, cv.cin, cv.coutp, cv.Wm);
        const size_t wt = (size_t)((cv.cout + 15) / 16) * 9 * cv.cinp * 16;
        k_prep_wm<true><<<grid1(wt), 256, 0, s>>>(d->P + cv.w_off, cv.cout, cv.cin, cv.cinp, cv.Wtm);
    }
    prof_end(PK_DSN_MISC, s);
    DEVEL_LAUNCH_CHECK("k_prep_wm");
    d->wm_stale = false;
    return DEVEL_OK;
}

int forward(devel_dsn* d, int nb, cudaStream_t s) {
    auto& A = d->acts;
    const int S = d->S, c = d->c;
    const int w[4] = {c, 2 * c, 4 * c, 8 * c};
    int rc = conv_fwd(d, 0, nb, d->xb, 1, nullptr, 0, S, A[A0].a, s);
    if (!rc) rc = conv_fwd(d, 1, nb, A[A0].a, w[0], nullptr, 0, S, A[S0].a, s);
    const int pin[3] = {S0, S1, S2}, pout[3] = {P1, P2, P3}, aa[3] = {A1, A2, A3}, ss[3] = {S1, S2, S3};
    for (int lv = 1; lv < 4 && !rc; ++lv) {
        const int side = S >> lv;
        const size_t planes = (size_t)nb * w[lv - 1];
        prof_begin(PK_DSN_MISC, s);
        if (side % 4 == 0)
            k_avgpool4<<<grid1(planes * side * side / 4), 256, 0, s>>>(A[pin[lv - 1]].a, side, planes * side,
                                                                     A[pout[lv - 1]].a);
        else
            k_avgpool<<<grid1(planes * side * side), 256, 0, s>>>(A[pin[lv - 1]].a, 2 * side, 2 * side, planes,
                                                                A[pout[lv - 1]].a);
        prof_end(PK_DSN_MISC, s);
        rc = conv_fwd(d, 2 * lv, nb, A[pout[lv - 1]].a, w[lv - 1], nullptr, 0, side, A[aa[lv - 1]].a, s);
        if (!rc) rc = conv_fwd(d, 2 * lv + 1, nb, A[aa[lv - 1]].a, w[lv], nullptr, 0, side, A[ss[lv - 1]].a, s);
    }
    // decoder: level lv takes up(previous) ++ skip(lv)
    const int up[3] = {U2, U1, U0}, da[3] = {D2A, D1A, D0A}, dd[3] = {D2, D1, D0}, skip[3] = {S2, S1, S0};
    int prev = S3;
    for (int j = 0; j < 3 && !rc; ++j) {
        const int lv = 2 - j, side = S >> lv;
        const size_t planes = (size_t)nb * w[lv + 1];
        prof_begin(PK_DSN_MISC, s);
        if ((side / 2) % 4 == 0)
            k_upsample4<<<grid1(planes * side * side / 16), 256, 0, s>>>(A[prev].a, side / 2, planes * (side / 2),
                                                                       A[up[j]].a);
        else
            k_upsample<<<grid1(planes * side * side), 256, 0, s>>>(A[prev].a, side / 2, side / 2, planes,
                                                                 A[up[j]].a);
        prof_end(PK_DSN_MISC, s);
        rc = conv_fwd(d, 8 + 2 * j, nb, A[up[j]].a, w[lv + 1], A[skip[j]].a, w[lv], side, A[da[j]].a, s);
        if (!rc) rc = conv_fwd(d, 9 + 2 * j, nb, A[da[j]].a, w[lv], nullptr, 0, side, A[dd[j]].a, s);
        prev = dd[j];
    }
    if (rc) return rc;
    const auto& h = d->convs[14];
    prof_begin(PK_DSN_MISC, s);
    k_head8<<<grid1((size_t)nb * S * S / 8), 256, 0, s>>>(d->x, A[D0].a, d->P + h.w_off, d->P + h.b_off, c, nb,
                                                          (size_t)S * S, d->y);
    prof_end(PK_DSN_MISC, s);
    DEVEL_LAUNCH_CHECK("dsn forward");
    return DEVEL_OK;
}

int backward(devel_dsn* d, int nb, cudaStream_t s) {
    auto& A = d->acts;
    const int S = d->S, c = d->c;
    const int w[4] = {c, 2 * c, 4 * c, 8 * c};
    const size_t plane0 = (size_t)S * S;
    const auto& h = d->convs[14];
    k_head_dgrad<<<grid1((size_t)nb * c * plane0), 256, 0, s>>>(d->dy, d->P + h.w_off, c, nb, plane0, A[D0].g);
    k_head_wgrad<<<dim3(c + 1, kHeadSplits), 256, 0, s>>>(d->dy, A[D0].a, c, nb, plane0, d->part);
    // weights then bias are contiguous in G
    k_wgrad_reduce<<<1, 256, 0, s>>>(d->part, kHeadSplits, (size_t)c + 1, d->G + h.w_off);
    const int up[3] = {U2, U1, U0}, da[3] = {D2A, D1A, D0A}, dd[3] = {D2, D1, D0}, skip[3] = {S2, S1, S0};
    const int prevs[3] = {S3, D2, D1};
    int rc = DEVEL_OK;
    for (int j = 2; j >= 0 && !rc; --j) {  // decoder levels, last first
        const int lv = 2 - j, side = S >> lv;
        rc = conv_bwd(d, 9 + 2 * j, nb, A[da[j]].a, w[lv], nullptr, 0, side, A[dd[j]].a, A[dd[j]].g, A[da[j]].g,
                      nullptr, 0, s);
        // the skip's gradient starts here (stored); the upsampled part goes to up[j]
        if (!rc)
            rc = conv_bwd(d, 8 + 2 * j, nb, A[up[j]].a, w[lv + 1], A[skip[j]].a, w[lv], side, A[da[j]].a, A[da[j]].g,
                          A[up[j]].g, A[skip[j]].g, 0, s);
        const size_t planes = (size_t)nb * w[lv + 1];
        k_upsample_bwd<<<grid1(planes * (side / 2) * (side / 2)), 256, 0, s>>>(A[up[j]].g, side / 2, side / 2, planes,
                                                                                A[prevs[j]].g);
    }
    // encoder, bottleneck first; the gradient of each level's output already holds the
    // skip contribution (levels 0-2) and gets the pooled path added
    const int aa[4] = {A0, A1, A2, A3}, ss[4] = {S0, S1, S2, S3}, pp[4] = {-1, P1, P2, P3};
    for (int lv = 3; lv >= 0 && !rc; --lv) {
        const int side = S >> lv;
        const __nv_bfloat16* in = lv == 0 ? d->xb : A[pp[lv]].a;
        const int cin = lv == 0 ? 1 : w[lv - 1];
        rc = conv_bwd(d, 2 * lv + 1, nb, A[aa[lv]].a, w[lv], nullptr, 0, side, A[ss[lv]].a, A[ss[lv]].g, A[aa[lv]].g,
                      nullptr, 0, s);
        if (!rc)
            rc = conv_bwd(d, 2 * lv, nb, in, cin, nullptr, 0, side, A[aa[lv]].a, A[aa[lv]].g,
                          lv == 0 ? nullptr : A[pp[lv]].g, nullptr, 0, s);
        if (!rc && lv > 0) {
            const size_t planes = (size_t)nb * w[lv - 1];
            k_avgpool_bwd<<<grid1(planes * 4 * side * side), 256, 0, s>>>(A[pp[lv]].g, 2 * side, 2 * side, planes,
                                                                          A[ss[lv - 1]].g, 1);
        }
    }
    DEVEL_LAUNCH_CHECK("dsn backward");
    return rc;
}

}  // namespace
}  // namespace devel

using namespace devel;

extern "C" {

int devel_dsn_create(int S, int batch, int width, devel_dsn** out) {
    if (!out) return set_error(DEVEL_EINVAL, "devel_dsn_create: out is NULL");
    *out = nullptr;
    if (S < 16 || S > 2048 || S % 16) return set_error(DEVEL_EINVAL, "devel_dsn_create: side %d not a multiple of 16 in [16, 2048]", S);
    if (batch < 1 || batch > 256) return set_error(DEVEL_EINVAL, "devel_dsn_create: batch %d outside [1, 256]", batch);
    if (width < 1 || width > 64) return set_error(DEVEL_EINVAL, "devel_dsn_create: width %d outside [1, 64]", width);
    devel_dsn* d = new devel_dsn;
    d->S = S;
    d->batch = batch;
    d->c = width;
    const int w[4] = {width, 2 * width, 4 * width, 8 * width};
    std::vector<std::array<int, 3>> L;
    int cin = 1;
    for (int lv = 0; lv < 4; ++lv) {
        L.push_back({cin, w[lv], 3});
        L.push_back({w[lv], w[lv], 3});
        cin = w[lv];
    }
    for (int lv = 2; lv >= 0; --lv) {
        L.push_back({w[lv + 1] + w[lv], w[lv], 3});
        L.push_back({w[lv], w[lv], 3});
    }
    L.push_back({w[0], 1, 1});
    size_t off = 0, maxpart = 0;
    cudaError_t e = cudaSuccess;
    for (auto& l : L) {
        devel_dsn::Conv cv{l[0], l[1], l[2], off, 0};
        off += (size_t)l[0] * l[1] * l[2] * l[2];
        cv.b_off = off;
        off += l[1];
        if (l[2] == 3 && e == cudaSuccess) {
            cv.coutp = (l[1] + kMCo - 1) / kMCo * kMCo;
            e = cudaMalloc(&cv.Wm, sizeof(__nv_bfloat16) * ((l[0] + 15) / 16) * 9 * cv.coutp * 16);
            cv.cinp = (l[0] + kMCo - 1) / kMCo * kMCo;
            if (e == cudaSuccess)
                e = cudaMalloc(&cv.Wtm, sizeof(__nv_bfloat16) * ((l[1] + 15) / 16) * 9 * cv.cinp * 16);
        }
        d->convs.push_back(cv);
    }
    d->nparams = off;
    // the plane side of each 3 x 3 layer (encoder levels 0-3, decoder levels 2, 1, 0) and,
    // where the tcgen05 kernel takes the layer, its weight layout and TMA map
    // (DEVEL_DSN_NO_TC=1 in the environment keeps every layer on the warp-level kernel)
    const char* no_tc = std::getenv("DEVEL_DSN_NO_TC");
    const bool use_tc = !(no_tc && no_tc[0] && no_tc[0] != '0');
    if (e == cudaSuccess && mma_init_attrs() != DEVEL_OK) e = cudaErrorUnknown;
    if (use_tc && e == cudaSuccess && conv3_tc_init_attrs() != DEVEL_OK) e = cudaErrorUnknown;
    for (size_t i = 0; i < d->convs.size() && e == cudaSuccess; ++i) {
        auto& cv = d->convs[i];
        if (cv.k != 3) continue;
        cv.side = i < 8 ? S >> (i / 2) : S >> (2 - (int)(i - 8) / 2);
        if (!use_tc || !conv3_tc_supported(cv.cin, cv.cout, cv.side)) continue;
        e = cudaMalloc(&cv.Wtc, sizeof(__nv_bfloat16) * conv3_tc_weight_elems(cv.cin, cv.cout));
        if (e == cudaSuccess && conv3_tc_make_map(&cv.mWtc, cv.Wtc, cv.cin, cv.cout) != DEVEL_OK) e = cudaErrorUnknown;
    }
    // activations: (channels, side) by id
    const int spec[NACT][2] = {{w[0], S},      {w[0], S},      {w[0], S / 2},  {w[1], S / 2}, {w[1], S / 2},
                               {w[1], S / 4},  {w[2], S / 4},  {w[2], S / 4},  {w[2], S / 8}, {w[3], S / 8},
                               {w[3], S / 8},  {w[3], S / 4},  {w[2], S / 4},  {w[2], S / 4}, {w[2], S / 2},
                               {w[1], S / 2},  {w[1], S / 2},  {w[1], S},      {w[0], S},     {w[0], S}};
    for (int i = 0; i < NACT; ++i) {
        devel_dsn::Act a{spec[i][0], spec[i][1]};
        const size_t cnt = (size_t)batch * a.C * a.side * a.side;
        if (e == cudaSuccess) e = cudaMalloc(&a.a, sizeof(__nv_bfloat16) * cnt);
        if (e == cudaSuccess) e = cudaMalloc(&a.g, sizeof(float) * cnt);
        d->acts.push_back(a);
    }
    // weight-gradient partials: spatial tiles x weights of the largest layer
    for (size_t i = 0; i < d->convs.size(); ++i) {
        const auto& cv = d->convs[i];
        if (cv.k != 3) continue;
        const int side = i < 8 ? S >> (i / 2) : S >> (2 - (int)(i - 8) / 2);
        const size_t tiles = (size_t)((side + kT - 1) / kT) * ((side + kT - 1) / kT);
        maxpart = std::max(maxpart, tiles * cv.cout * (cv.cin * 9 + 1));
    }
    maxpart = std::max(maxpart, (size_t)kHeadSplits * (width + 1));
    const size_t px = (size_t)batch * S * S;
    const int mse_blocks = grid1(px);
    if (e == cudaSuccess) e = cudaMalloc(&d->P, sizeof(float) * off);
    if (e == cudaSuccess) e = cudaMalloc(&d->G, sizeof(float) * off);
    if (e == cudaSuccess) e = cudaMalloc(&d->M, sizeof(float) * off);
    if (e == cudaSuccess) e = cudaMalloc(&d->V, sizeof(float) * off);
    if (e == cudaSuccess) e = cudaMalloc(&d->x, sizeof(float) * px);
    if (e == cudaSuccess) e = cudaMalloc(&d->xb, sizeof(__nv_bfloat16) * px);
    if (e == cudaSuccess) e = cudaMalloc(&d->y, sizeof(float) * px);
    if (e == cudaSuccess) e = cudaMalloc(&d->dy, sizeof(float) * px);
    if (e == cudaSuccess) e = cudaMalloc(&d->part, sizeof(float) * maxpart);
    if (e == cudaSuccess) e = cudaMalloc(&d->qpart, sizeof(long long) * mse_blocks);
    if (e == cudaSuccess) e = cudaMalloc(&d->counter, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc(&d->loss, sizeof(double));
    d->part_count = maxpart;
    if (e == cudaSuccess) e = cudaMemset(d->P, 0, sizeof(float) * off);
    if (e == cudaSuccess) e = cudaMemset(d->M, 0, sizeof(float) * off);
    if (e == cudaSuccess) e = cudaMemset(d->V, 0, sizeof(float) * off);
    if (e == cudaSuccess) e = cudaMemset(d->counter, 0, sizeof(unsigned));
    if (e != cudaSuccess) {
        free_dsn(d);
        return cuda_error(e, "devel_dsn_create");
    }
    *out = d;
    return DEVEL_OK;
}

int devel_dsn_destroy(devel_dsn* d) {
    if (!d) return DEVEL_OK;
    cudaDeviceSynchronize();
    free_dsn(d);
    return DEVEL_OK;
}

long long devel_dsn_param_count(const devel_dsn* d) { return d ? (long long)d->nparams : -1; }

int devel_dsn_set_params(devel_dsn* d, const float* host) {
    if (!d || !host) return set_error(DEVEL_EINVAL, "devel_dsn_set_params: NULL argument");
    DEVEL_CUDA_TRY(cudaMemcpy(d->P, host, sizeof(float) * d->nparams, cudaMemcpyHostToDevice));
    DEVEL_CUDA_TRY(cudaMemset(d->M, 0, sizeof(float) * d->nparams));
    DEVEL_CUDA_TRY(cudaMemset(d->V, 0, sizeof(float) * d->nparams));
    d->t = 0;
    d->wm_stale = true;
    return DEVEL_OK;
}

int devel_dsn_get_params(const devel_dsn* d, float* host) {
    if (!d || !host) return set_error(DEVEL_EINVAL, "devel_dsn_get_params: NULL argument");
    DEVEL_CUDA_TRY(cudaMemcpy(host, d->P, sizeof(float) * d->nparams, cudaMemcpyDeviceToHost));
    return DEVEL_OK;
}

int devel_dsn_init(devel_dsn* d, unsigned long long seed) {
    if (!d) return set_error(DEVEL_EINVAL, "devel_dsn_init: dsn is NULL");
    // He-normal weights from a splitmix64 stream and the Box-Muller transform, zero biases
    std::vector<float> h(d->nparams, 0.f);
    unsigned long long st = seed;
    auto next = [&]() {
        st += 0x9E3779B97F4A7C15ull;
        unsigned long long z = st;
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    auto uni = [&]() { return ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); };
    for (auto& cv : d->convs) {
        const size_t wc = (size_t)cv.cout * cv.cin * cv.k * cv.k;
        const double sd = std::sqrt(2.0 / (cv.cin * cv.k * cv.k));
        for (size_t i = 0; i < wc; ++i) {
            const double u1 = uni(), u2 = uni();
            h[cv.w_off + i] = (float)(sd * std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2));
        }
    }
    return devel_dsn_set_params(d, h.data());
}

int devel_dsn_forward(devel_dsn* d, int nb, const float* tsdf, float B, float* phi0, cudaStream_t s) {
    if (!d) return set_error(DEVEL_EINVAL, "devel_dsn_forward: dsn is NULL");
    if (nb < 1 || nb > d->batch) return set_error(DEVEL_EINVAL, "devel_dsn_forward: nb=%d outside [1, %d]", nb, d->batch);
    if (bad_ptr(tsdf) || bad_ptr(phi0))
        return set_error(DEVEL_EINVAL, "devel_dsn_forward: tsdf / phi0 NULL or not 16-byte aligned");
    if (!(B > 0.f)) return set_error(DEVEL_EINVAL, "devel_dsn_forward: band B must be > 0");
    const size_t px = (size_t)nb * d->S * d->S;
    int rc = prep_weights(d, s);
    if (rc) return rc;
    prof_begin(PK_DSN_MISC, s);
    k_band<<<grid1(px), 256, 0, s>>>(tsdf, px, B, d->x, d->xb);
    prof_end(PK_DSN_MISC, s);
    rc = forward(d, nb, s);
    if (rc) return rc;
    prof_begin(PK_DSN_MISC, s);
    k_scale<<<grid1(px), 256, 0, s>>>(d->y, px, B, phi0);
    prof_end(PK_DSN_MISC, s);
    DEVEL_LAUNCH_CHECK("devel_dsn_forward");
    return DEVEL_OK;
}

}  // extern "C"

namespace devel {
namespace {
// one training step; ahf_eps > 0: the modulation branch's loss against labels in
// `label` (0 / 1 maps), else the MSE against the band-limited level set `label`
int dsn_train(devel_dsn* d, int nb, const float* tsdf, const float* label, float B, float lr, float ahf_eps,
              double* loss_out, cudaStream_t s);
}  // namespace
}  // namespace devel

extern "C" {

int devel_dsn_train_step(devel_dsn* d, int nb, const float* tsdf, const float* phi_gt, float B, float lr,
                         double* loss_out, cudaStream_t s) {
    return dsn_train(d, nb, tsdf, phi_gt, B, lr, 0.f, loss_out, s);
}

int devel_dsn_train_step_ahf(devel_dsn* d, int nb, const float* tsdf, const float* m_gt, float B, float eps, float lr,
                             double* loss_out, cudaStream_t s) {
    if (!(eps > 0.f)) return set_error(DEVEL_EINVAL, "devel_dsn_train_step_ahf: eps must be > 0");
    return dsn_train(d, nb, tsdf, m_gt, B, lr, eps, loss_out, s);
}

int devel_dsn_forward_ahf(devel_dsn* d, int nb, const float* tsdf, float B, float eps, float* m_out, cudaStream_t s) {
    if (!d) return set_error(DEVEL_EINVAL, "devel_dsn_forward_ahf: dsn is NULL");
    if (nb < 1 || nb > d->batch)
        return set_error(DEVEL_EINVAL, "devel_dsn_forward_ahf: nb=%d outside [1, %d]", nb, d->batch);
    if (bad_ptr(tsdf) || bad_ptr(m_out))
        return set_error(DEVEL_EINVAL, "devel_dsn_forward_ahf: tsdf / m_out NULL or not 16-byte aligned");
    if (!(B > 0.f) || !(eps > 0.f)) return set_error(DEVEL_EINVAL, "devel_dsn_forward_ahf: band and eps must be > 0");
    const size_t px = (size_t)nb * d->S * d->S;
    int rc = prep_weights(d, s);
    if (rc) return rc;
    k_band<<<grid1(px), 256, 0, s>>>(tsdf, px, B, d->x, d->xb);
    rc = forward(d, nb, s);
    if (rc) return rc;
    k_ahf_out<<<grid1(px), 256, 0, s>>>(d->y, px, eps, m_out);
    DEVEL_LAUNCH_CHECK("devel_dsn_forward_ahf");
    return DEVEL_OK;
}

}  // extern "C"

namespace devel {
namespace {
int dsn_train(devel_dsn* d, int nb, const float* tsdf, const float* phi_gt, float B, float lr, float ahf_eps,
              double* loss_out, cudaStream_t s) {
    if (!d) return set_error(DEVEL_EINVAL, "devel_dsn_train_step: dsn is NULL");
    if (nb < 1 || nb > d->batch)
        return set_error(DEVEL_EINVAL, "devel_dsn_train_step: nb=%d outside [1, %d]", nb, d->batch);
    if (bad_ptr(tsdf) || bad_ptr(phi_gt))
        return set_error(DEVEL_EINVAL, "devel_dsn_train_step: tsdf / phi_gt NULL or not 16-byte aligned");
    if (!(B > 0.f) || !(lr >= 0.f)) return set_error(DEVEL_EINVAL, "devel_dsn_train_step: bad band or learning rate");
    const size_t px = (size_t)nb * d->S * d->S;
    int rc = prep_weights(d, s);
    if (rc) return rc;
    k_band<<<grid1(px), 256, 0, s>>>(tsdf, px, B, d->x, d->xb);
    rc = forward(d, nb, s);
    if (rc) return rc;
    const int mb = grid1(px);
    if (ahf_eps > 0.f) {
        k_ahf_mse<<<mb, 256, 0, s>>>(d->y, phi_gt, px, ahf_eps, d->dy, d->qpart, d->counter,
                                     loss_out ? loss_out : d->loss);
    } else {
        // labels band-limited into dy's buffer first, then the MSE overwrites it with dL/dy
        k_band<<<grid1(px), 256, 0, s>>>(phi_gt, px, B, d->dy, nullptr);
        k_mse<<<mb, 256, 0, s>>>(d->y, d->dy, px, d->dy, d->qpart, d->counter, loss_out ? loss_out : d->loss);
    }
    rc = backward(d, nb, s);
    if (rc) return rc;
    d->t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)d->t), c2 = 1.f - std::pow(b2, (float)d->t);
    k_adam<<<grid1(d->nparams), 256, 0, s>>>(d->P, d->G, d->M, d->V, d->nparams, lr, b1, b2, 1e-8f, c1, c2);
    d->wm_stale = true;
    DEVEL_LAUNCH_CHECK("devel_dsn_train_step");
    return DEVEL_OK;
}
}  // namespace
}  // namespace devel

extern "C" {

int devel_dsn_grads(const devel_dsn* d, float* host) {
    if (!d || !host) return set_error(DEVEL_EINVAL, "devel_dsn_grads: NULL argument");
    DEVEL_CUDA_TRY(cudaMemcpy(host, d->G, sizeof(float) * d->nparams, cudaMemcpyDeviceToHost));
    return DEVEL_OK;
}

}  // extern "C"

namespace devel {
namespace {
int resample_args(const char* where, int n, int f, int nb, const float* a, const float* b) {
    if (n < 1 || n > 16384 || f < 1 || n % f)
        return set_error(DEVEL_EINVAL, "%s: n=%d, f=%d (need 1 <= n <= 16384, f >= 1, n %% f == 0)", where, n, f);
    if (nb < 0) return set_error(DEVEL_EINVAL, "%s: nb=%d < 0", where, nb);
    if (nb > 0 && (bad_ptr(a) || bad_ptr(b)))
        return set_error(DEVEL_EINVAL, "%s: NULL or not 16-byte aligned argument", where);
    return DEVEL_OK;
}
}  // namespace
}  // namespace devel

extern "C" {

int devel_phi_downsample(int n, int f, int nb, const float* fine, float* coarse, cudaStream_t s) {
    const int rc = resample_args("devel_phi_downsample", n, f, nb, fine, coarse);
    if (rc || nb == 0) return rc;
    const int m = n / f;
    prof_begin(PK_RESAMPLE, s);
    k_phi_down<<<dim3((m + 255) / 256, m, std::min(nb, 65535)), 256, 0, s>>>(fine, n, f, nb,
                                                                             (float)(1.0 / ((double)f * f * f)), coarse);
    prof_end(PK_RESAMPLE, s);
    DEVEL_LAUNCH_CHECK("devel_phi_downsample");
    return DEVEL_OK;
}

int devel_phi_upsample(int n, int f, int nb, const float* coarse, float* fine, cudaStream_t s) {
    const int rc = resample_args("devel_phi_upsample", n, f, nb, coarse, fine);
    if (rc || nb == 0) return rc;
    prof_begin(PK_RESAMPLE, s);
    k_phi_up<<<dim3((n + 1023) / 1024, n, std::min(nb, 65535)), 256, 0, s>>>(coarse, n, f, nb, fine);
    prof_end(PK_RESAMPLE, s);
    DEVEL_LAUNCH_CHECK("devel_phi_upsample");
    return DEVEL_OK;
}

}  // extern "C"
