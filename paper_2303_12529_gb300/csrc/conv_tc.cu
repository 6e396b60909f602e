// Forward 3x3 convolution of the DSN level-set branch (Sec. III-B) on the tcgen05
// tensor cores: an implicit GEMM with the accumulators in TMEM.
//
//   D[p][co] = sum_{tap, ci} X[ci][y + dy - 1][x + dx - 1] W[co][ci][tap]      (zero padding)
//
// with M = 128 output pixels of one image row (x0 .. x0 + 127), N = Cout (32, 64 or 128),
// and K = 9 taps x Cin channels, 16 channels per MMA. A CTA computes TR (2, 2, 1 for
// N = 32, 64, 128) consecutive output rows of one 128-pixel segment; two CTAs share an SM.
//
// Operands:
//   A  the input rows y0 - 1 .. y0 + TR, transposed by the producer warps into
//      shared memory as "halo rows": per input row a 1024-byte-aligned block of 136
//      pixel rows (pixel x0 - 1 + p at row p), each 128 bytes = 64 channels, in the
//      128-byte-swizzled K-major layout (16-byte chunk c of row p at ((c ^ (p & 7)) << 4)).
//      Tap (dy, dx) of output row r reads the 128 rows dx .. dx + 127 of the halo block of
//      input row r + dy: a descriptor whose start is dx rows into the block. The swizzle
//      is a function of the shared-memory address (measured on this part: views starting
//      1, 2 or 7 rows into a 1024-byte pattern read exactly, with the descriptor's base
//      offset field left 0), so the shifted views need no copy.
//   B  the weights, prepared as Wtc[cb][tap][co][64] (bf16, channels of block cb,
//      zero past Cin), one [Cout x 64] box per (channel block, tap), by TMA into a ring.
//
// Warp roles (192 threads): warps 0-3 fill the halo rows (16-byte loads of 8 pixels along
// the NCHW planes of 8 channels, transposed in registers into one 16-byte chunk per pixel
// row) and, after the last MMA, drain TMEM (thread = output pixel) with the
// bias and ReLU into the NCHW bf16 output; warp 4 lane 0 loads the weights; warp 5
// lane 0 issues the MMAs. Every mbarrier wait is bounded; after a timeout the CTA stops
// issuing and writes NaN outputs (which the solve's non-finite checks report).
#include <cuda.h>
#include <cuda_bf16.h>

#include "common.cuh"
#include "conv_tc.cuh"
#include "tc.cuh"
#include "tc_ptx.cuh"

namespace devel {
namespace {

using bf16 = __nv_bfloat16;
using namespace tc;

constexpr int kHaloRows = 136;                      // pixel rows of one halo block (130 used)
constexpr uint32_t kHaloBytes = kHaloRows * 128;    // 17 KiB, a multiple of 1024

// Per output-channel count N: TR output rows per CTA and kBS weight slots, sized so that
// two CTAs share an SM (one's producer runs while the other's MMAs do). For N = 32 the nine
// taps' weights of a channel block all fit (TR = 2 leaves the room): a tap's MMAs take
// about a tenth of a TMA round trip, so a ring of a few slots left the MMA issuer waiting
// for weights (measured: 6.6 us of a 14 us CTA with TR = 3 and four slots).
template <int N>
struct CfgC {
    static constexpr int TR = N == 128 ? 1 : 2;
    static constexpr int kBS = N == 32 ? 9 : N == 64 ? 4 : 3;
    static constexpr uint32_t kA = (TR + 2) * kHaloBytes;   // the halo rows of one channel block
    static constexpr uint32_t kB = N * 128;                 // one (channel block, tap) weight box
    static constexpr uint32_t kCols = TR * N <= 32 ? 32 : TR * N <= 64 ? 64 : TR * N <= 128 ? 128 : 256;
    static constexpr size_t kSmem = 1024 + (size_t)kA + (size_t)kBS * kB + 256;
    static_assert(kSmem <= 113 * 1024, "two CTAs per SM");
};

// The MMAs of one (channel block, tap): TR output rows x KS 16-channel steps, unrolled
// (compile-time counts: a runtime-bounded issue loop measured about twice the cycles per
// MMA of a straight run of them).
template <int N, int TR, int KS>
__device__ __forceinline__ void conv_tap_mmas(uint32_t tmem, uint32_t stage, uint64_t bdesc, int dy, int dx,
                                              bool first) {
    constexpr uint32_t idesc = idesc_bf16(128, N);
    uint64_t adesc[TR];
#pragma unroll
    for (int r = 0; r < TR; ++r) adesc[r] = smem_desc_sw128(stage + (uint32_t)((r + dy) * kHaloBytes + dx * 128));
#pragma unroll
    for (int r = 0; r < TR; ++r)
#pragma unroll
        for (int kk = 0; kk < KS; ++kk) {
            const uint64_t adv = (uint64_t)(kk * 32) >> 4;
            mma_bf16(tmem + (uint32_t)(r * N), adesc[r] + adv, bdesc + adv, idesc, (first && kk == 0) ? 0u : 1u);
        }
}

template <int N>
__global__ void __launch_bounds__(192, 2)
k_conv3_tc(const bf16* __restrict__ XA, int CA, const bf16* __restrict__ XB, int CB,
           const __grid_constant__ CUtensorMap tmW, const float* __restrict__ bias, bf16* __restrict__ Y, int H,
           int Wd) {
    using CF = CfgC<N>;
    constexpr int TR = CF::TR, SA = 1, kBSlots = CF::kBS;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* sA = smem;                          // [SA][TR + 2][kHaloRows][128 B]
    uint8_t* sB = smem + SA * CF::kA;            // [kBSlots][N][128 B]
    uint64_t* a_full = reinterpret_cast<uint64_t*>(sB + kBSlots * CF::kB);
    uint64_t* a_empty = a_full + SA;
    uint64_t* b_full = a_empty + SA;
    uint64_t* b_empty = b_full + kBSlots;
    uint64_t* acc_full = b_empty + kBSlots;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_full + 1);
    volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int x0 = blockIdx.x * 128, y0 = blockIdx.y * TR, n = blockIdx.z;
    const int Cin = CA + CB, ncb = (Cin + 63) / 64;
    const size_t plane = (size_t)H * Wd;

    if (threadIdx.x == 0) {
        for (int s = 0; s < SA; ++s) {
            mbar_init(&a_full[s], 4);  // one arrival per producer warp
            mbar_init(&a_empty[s], 1);
        }
        for (int s = 0; s < kBSlots; ++s) {
            mbar_init(&b_full[s], 1);
            mbar_init(&b_empty[s], 1);
        }
        mbar_init(acc_full, 1);
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 5) tmem_alloc(tmem_slot, CF::kCols);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp < 4) {
        // ---------------- producer: halo rows of channel block cb into stage cb % SA
        const int t = threadIdx.x;  // pixel rows t and t + 128 (< 130)
        bool ok = true;
        for (int cb = 0; cb < ncb && ok; ++cb) {
            const int s = cb % SA;
            if (cb >= SA) {
                ok = mbar_wait_ab(&a_empty[s], ((cb / SA) - 1) & 1, nullptr, abort);
                ok = __all_sync(0xffffffffu, ok);
                if (!ok) break;
            }
            // tasks: (halo row, 8-pixel group, 8-channel group); a group of 8 aligned pixels
            // x0 - 8 + 8 g (g < 18) covers the halo columns x0 - 1 .. x0 + 128. Per task eight
            // 16-byte loads (eight channels, along the NCHW planes), an 8 x 8 transpose by
            // byte permutes, and one 16-byte store per halo pixel row.
            const int ci0 = cb * 64, ncg = min(64, Cin - ci0) / 8;
            uint8_t* stage = sA + s * CF::kA;
            const int ntask = (TR + 2) * 18 * ncg;
            // two tasks per round (t and t + 128): their sixteen loads are in flight together
            auto load = [&](int task, uint4 (&v)[8]) {
                const int cg = task % ncg, rest = task / ncg, g = rest % 18, hr = rest / 18;
                const int gy = y0 - 1 + hr, gx = x0 - 8 + 8 * g;
                const bool in = task < ntask && gy >= 0 && gy < H && gx >= 0 && gx + 8 <= Wd;
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    const int ci = ci0 + cg * 8 + c;
                    v[c] = make_uint4(0u, 0u, 0u, 0u);
                    if (in) {
                        const bf16* src = ci < CA ? XA + ((size_t)n * CA + ci) * plane
                                                  : XB + ((size_t)n * CB + (ci - CA)) * plane;
                        v[c] = __ldg(reinterpret_cast<const uint4*>(src + (size_t)gy * Wd + gx));
                    }
                }
            };
            auto store = [&](int task, const uint4 (&v)[8]) {
                const int cg = task % ncg, rest = task / ncg, g = rest % 18, hr = rest / 18;
                const int gx = x0 - 8 + 8 * g;
                uint8_t* blk = stage + hr * kHaloBytes;
#pragma unroll
                for (int j = 0; j < 8; ++j) {  // pixel gx + j: channels cg * 8 .. + 7
                    const int p = gx + j - (x0 - 1);
                    if (p < 0 || p >= 130) continue;
                    const uint32_t sel = (j & 1) ? 0x7632u : 0x5410u;
                    uint32_t o[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        const uint32_t* a = reinterpret_cast<const uint32_t*>(&v[2 * k]);
                        const uint32_t* b = reinterpret_cast<const uint32_t*>(&v[2 * k + 1]);
                        o[k] = __byte_perm(a[j >> 1], b[j >> 1], sel);
                    }
                    *reinterpret_cast<uint4*>(blk + p * 128 + ((cg ^ (p & 7)) << 4)) = make_uint4(o[0], o[1], o[2], o[3]);
                }
            };
            for (int task = t; task < ntask; task += 256) {
                uint4 va[8], vb[8];
                load(task, va);
                load(task + 128, vb);
                store(task, va);
                if (task + 128 < ntask) store(task + 128, vb);
            }
            fence_proxy_async_smem();  // generic-proxy stores -> visible to the tensor core
            __syncwarp();
            if (lane == 0) mbar_arrive(&a_full[s]);
        }
    } else if (warp == 4) {
        // ---------------- weights: one [N x 64] box per (channel block, tap)
        if (lane == 0) {
            int slot = 0;
            for (int cb = 0; cb < ncb; ++cb) {
                for (int tap = 0; tap < 9; ++tap, ++slot) {
                    const int sl = slot % kBSlots;
                    if (slot >= kBSlots && !mbar_wait_ab(&b_empty[sl], ((slot / kBSlots) - 1) & 1, nullptr, abort))
                        goto weights_done;
                    mbar_arrive_expect_tx(&b_full[sl], CF::kB);
                    tma_load_2d(&tmW, &b_full[sl], sB + sl * CF::kB, 0, (cb * 9 + tap) * N);
                }
            }
        weights_done:;
        }
    } else {
        // ---------------- MMA issuer
        if (lane == 0) {
            int slot = 0;
            bool ok = true;
            for (int cb = 0; cb < ncb && ok; ++cb) {
                const int s = cb % SA;
                if (!mbar_wait_ab(&a_full[s], (cb / SA) & 1, nullptr, abort)) {
                    ok = false;
                    break;
                }
                fence_after_sync();
                const int ksteps = min(64, Cin - cb * 64) / 16;
                const uint32_t stage = smem_u32(sA + s * CF::kA);
                for (int tap = 0; tap < 9 && ok; ++tap, ++slot) {
                    const int sl = slot % kBSlots, dy = tap / 3, dx = tap % 3;
                    if (!mbar_wait_ab(&b_full[sl], (slot / kBSlots) & 1, nullptr, abort)) {
                        ok = false;
                        break;
                    }
                    fence_after_sync();
                    const uint64_t bdesc = smem_desc_sw128(smem_u32(sB + sl * CF::kB));
                    const bool first = cb == 0 && tap == 0;
                    switch (ksteps) {
                        case 4: conv_tap_mmas<N, TR, 4>(tmem, stage, bdesc, dy, dx, first); break;
                        case 3: conv_tap_mmas<N, TR, 3>(tmem, stage, bdesc, dy, dx, first); break;
                        case 2: conv_tap_mmas<N, TR, 2>(tmem, stage, bdesc, dy, dx, first); break;
                        default: conv_tap_mmas<N, TR, 1>(tmem, stage, bdesc, dy, dx, first); break;
                    }
                    mma_commit(&b_empty[sl]);
                }
                mma_commit(&a_empty[s]);
            }
            mma_commit(acc_full);  // also after a failure: the MMAs in flight complete first
        }
    }
    __syncwarp();

    // ---------------- epilogue: TMEM lanes 32 w .. (pixels), columns r N + co
    if (warp < 4) {
        bool h = mbar_wait(acc_full, 0, nullptr);
        h = __all_sync(0xffffffffu, h) && !*abort;
        fence_after_sync();
        const int x = x0 + warp * 32 + lane;
        for (int r = 0; r < TR; ++r) {
            const int y = y0 + r;
            for (int c = 0; c < N; c += 32) {
                uint32_t v[32];
                if (h) {
                    tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(r * N + c), v);
                } else {
#pragma unroll
                    for (int j = 0; j < 32; ++j) v[j] = 0x7fc00000u;  // NaN: the result is unusable
                }
                if (x < Wd && y < H) {
                    bf16* dst = Y + ((size_t)n * N + c) * plane + (size_t)y * Wd + x;
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const float o = fmaxf(__uint_as_float(v[j]) + bias[c + j], 0.f);
                        dst[(size_t)j * plane] = __float2bfloat16_rn(h ? o : __uint_as_float(v[j]));
                    }
                }
            }
        }
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 5) {
        fence_after_sync();
        tmem_dealloc(tmem, CF::kCols);
    }
}

// Wtc[cb][tap][co][64] = bf16(W[co][ci = 64 cb + j][tap]), zero for ci >= Cin
__global__ void k_prep_wtc(const float* __restrict__ W, int Cout, int Cin, bf16* __restrict__ Wt) {
    const int ncb = (Cin + 63) / 64;
    const size_t count = (size_t)ncb * 9 * Cout * 64;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(i % 64);
        const size_t r = i / 64;
        const int co = (int)(r % Cout), tap = (int)((r / Cout) % 9), cb = (int)(r / ((size_t)Cout * 9));
        const int ci = cb * 64 + j;
        Wt[i] = __float2bfloat16_rn(ci < Cin ? W[((size_t)co * Cin + ci) * 9 + tap] : 0.f);
    }
}

template <int N>
cudaError_t set_attr_conv() {
    return cudaFuncSetAttribute(k_conv3_tc<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CfgC<N>::kSmem);
}

}  // namespace

bool conv3_tc_supported(int Cin, int Cout, int side) {
    return (Cout == 32 || Cout == 64 || Cout == 128) && Cin % 16 == 0 && Cin >= 16 && side >= 128;
}

size_t conv3_tc_weight_elems(int Cin, int Cout) { return (size_t)((Cin + 63) / 64) * 9 * Cout * 64; }

int conv3_tc_init_attrs() {
    cudaError_t e = set_attr_conv<32>();
    if (e == cudaSuccess) e = set_attr_conv<64>();
    if (e == cudaSuccess) e = set_attr_conv<128>();
    if (e != cudaSuccess) return cuda_error(e, "conv3_tc_init_attrs");
    return DEVEL_OK;
}

int conv3_tc_make_map(CUtensorMap* tm, const bf16* Wt, int Cin, int Cout) {
    const int rows = (Cin + 63) / 64 * 9 * Cout;
    return tc::make_map(tm, Wt, rows, 64, 64, Cout);
}

int launch_prep_wtc(const float* W, int Cout, int Cin, bf16* Wt, cudaStream_t s) {
    const size_t count = conv3_tc_weight_elems(Cin, Cout);
    k_prep_wtc<<<(unsigned)std::min<size_t>((count + 255) / 256, 152 * 16), 256, 0, s>>>(W, Cout, Cin, Wt);
    DEVEL_LAUNCH_CHECK("k_prep_wtc");
    return DEVEL_OK;
}

int launch_conv3_tc(const bf16* XA, int CA, const bf16* XB, int CB, const CUtensorMap& tmW, const float* bias,
                    bf16* Y, int Cout, int nb, int side, cudaStream_t s) {
    const int TR = Cout == 32 ? CfgC<32>::TR : Cout == 64 ? CfgC<64>::TR : CfgC<128>::TR;
    dim3 grid((side + 127) / 128, (side + TR - 1) / TR, nb);
    switch (Cout) {
        case 32:
            k_conv3_tc<32><<<grid, 192, CfgC<32>::kSmem, s>>>(XA, CA, XB, CB, tmW, bias, Y, side, side);
            break;
        case 64:
            k_conv3_tc<64><<<grid, 192, CfgC<64>::kSmem, s>>>(XA, CA, XB, CB, tmW, bias, Y, side, side);
            break;
        case 128:
            k_conv3_tc<128><<<grid, 192, CfgC<128>::kSmem, s>>>(XA, CA, XB, CB, tmW, bias, Y, side, side);
            break;
        default:
            return set_error(DEVEL_EINVAL, "conv3_tc: Cout %d unsupported", Cout);
    }
    DEVEL_LAUNCH_CHECK("k_conv3_tc");
    return DEVEL_OK;
}

}  // namespace devel
