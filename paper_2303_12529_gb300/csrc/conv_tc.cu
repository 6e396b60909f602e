// Forward 3x3 convolution of the DSN level-set branch (Sec. III-B) on the tcgen05
// tensor cores: an implicit GEMM with the accumulators in TMEM.
//
//   D[p][co] = sum_{tap, ci} X[ci][y + dy - 1][x + dx - 1] W[co][ci][tap]      (zero padding)
//
// with M = 128 output pixels of one image row (x0 .. x0 + 127), N = Cout (64 or 128), and
// K = 9 taps x Cin channels, 16 channels per MMA. A tile is TR consecutive output rows of
// one 128-pixel segment; a unit is one tile's 64-channel block. Two other forms share the
// kernel (CfgC): Cout = 32 stacks the three vertical taps of one dx along N (one N = 96
// product per halo row and dx, TR = 4), and Cout = 256 on 64^2 planes swaps the operands
// (weights as A, the 64 pixels of a row as N).
//
// Operands:
//   A  the input rows y0 - 1 .. y0 + TR of a unit as "halo rows": per input row a
//      1024-byte-aligned block of 136 pixel rows (pixel x0 - 1 + p at row p), each 128
//      bytes = 64 channels, in the 128-byte-swizzled K-major layout (16-byte chunk c of row
//      p at ((c ^ (p & 7)) << 4)). Tap (dy, dx) of output row r reads the 128 rows
//      dx .. dx + 127 of the block of input row r + dy: a descriptor whose start is dx rows
//      into the block. The swizzle is a function of the shared-memory address (measured on
//      this part: views starting 1, 2 or 7 rows into a 1024-byte pattern read exactly, with
//      the descriptor's base offset field left 0), so the shifted views need no copy.
//   B  the weights, prepared as Wtc[cb][tap][co][64] (bf16, channels of block cb, zero past
//      Cin; for Cout = 32 as [cb][dx][2 - dy][co][64]), by TMA in boxes of one (channel
//      block, tap) (96 rows for the stacked form): resident for the whole kernel when all
//      of a layer's boxes fit, else through a ring.
//
// The halo rows are built on chip: TMA copies the raw NCHW row segments (32 or 8 channel
// planes x 152 pixels from x0 - 8 per box; outside the image the copy fills zeros, which
// is the padding) into a ring of raw rows, and four warps transpose them with ldmatrix /
// stmatrix.trans. The kernel is persistent (one CTA per SM over a contiguous range of
// tiles), warp-specialised, with one mbarrier pair per halo row and per raw-row slot, so
// that the transposes of a unit's first halo rows overlap the MMAs still reading its
// predecessor's last ones, and with two TMEM accumulators, so that a tile's epilogue
// overlaps the next tile's MMAs. Every wait is bounded; after a timeout the CTA stops
// issuing and writes NaN outputs (which the solve's non-finite checks report).
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>

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
constexpr int kStgPx = 152;                         // pixels of a raw row box: x0 - 8 .. x0 + 143
constexpr uint32_t kStgBox = kStgPx * 8 * 2;        // one box: 8 planes x 152 pixels (19 x 128 B)
constexpr uint32_t kStgRow = 8 * kStgBox;           // the 64 channels of one raw row (19 KiB)
constexpr uint32_t kSmemMax = 232448;               // 227 KiB of dynamic shared memory per CTA

// Per output-channel count N: TR output rows per tile, HR = TR + 2 halo rows, RS raw-row
// slots, and as many weight granules (GT boxes each, at most 9 granules) as fit beside them
// in one CTA per SM.
//   N = 64, 128:     M = 128 pixels of one row (PX = 128), N = Cout; a granule is a tap
//                    row (the three boxes of one (channel block, dy));
//   N = 32 (ST):     the three vertical taps stacked along N: per halo row and dx one
//                    product of N = 96 (B = [W(dy 2); W(dy 1); W(dy 0)] of that dx) into
//                    TMEM columns 32 hr .. 32 hr + 95, so that every contribution to output
//                    row r lands at columns 32 (r + 2); TR = 4, accumulators zeroed by the
//                    epilogue; a granule is one (channel block, dx) box of 96 rows;
//   N = 256 (SW):    planes of side 64, operands swapped: A = the weights (M = 128 output
//                    channels, two halves), B = the halo rows (N = PX = 64 pixels); a
//                    granule is one tap's box of all 256 output channels.
template <int N>
struct CfgC {
    static constexpr bool SW = N == 256;
    static constexpr bool ST = N == 32;
    static constexpr int TR = ST ? 4 : 2;
    static constexpr int HR = TR + 2;
    static constexpr int RS = SW ? 2 : N == 64 ? 4 : 3;
    static constexpr int GT = SW || ST ? 1 : 3;       // boxes per weight granule
    static constexpr int GPU = ST ? 3 : 9 / GT;       // granules per unit
    static constexpr int kBoxPerCb = ST ? 3 : 9;      // weight boxes per channel block
    static constexpr int kBoxRows = ST ? 3 * N : N;   // rows of one weight box
    static constexpr int PX = SW ? 64 : 128;          // pixels of a tile row
    static constexpr uint32_t kA = HR * kHaloBytes;
    static constexpr uint32_t kStg = RS * kStgRow;
    static constexpr uint32_t kB = kBoxRows * 128;    // one weight box
    static constexpr uint32_t kFixed = 1024 + kA + kStg + 1024;  // alignment, halo, raw rows, barriers
    static constexpr int kFit = (int)((kSmemMax - kFixed) / (GT * kB));
    static constexpr int kRows = kFit > 9 ? 9 : kFit;  // weight granule slots
    static_assert(kFit >= 2, "weight ring too small");
    // TMEM columns of one accumulator
    static constexpr int kAcc = SW ? TR * (N / 128) * PX : ST ? N * (HR + 2) : TR * N;
    static_assert(2 * kAcc <= 512, "two accumulators in TMEM");
    static constexpr uint32_t kCols = 2 * kAcc <= 32 ? 32 : 2 * kAcc <= 64 ? 64 : 2 * kAcc <= 128 ? 128
                                    : 2 * kAcc <= 256 ? 256 : 512;
    static constexpr size_t kSmem = kFixed + (size_t)kRows * GT * kB;
    static_assert(kSmem <= kSmemMax, "shared memory");
};

// 8x8 b16 matrices between shared memory and registers. ldmatrix: lane 8 m + r gives the
// address of row r of matrix m, and thread t receives row t / 4, columns 2 (t % 4) .. + 1;
// stmatrix.trans stores the transpose (lane 8 m + j gives the address of the stored row j,
// which is column j of the fragment).
__device__ __forceinline__ void ldsm_x4(uint32_t a, uint32_t (&v)[4]) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]) : "r"(a) : "memory");
}
__device__ __forceinline__ void stsm_x4_trans(uint32_t a, const uint32_t (&v)[4]) {
    asm volatile("stmatrix.sync.aligned.m8n8.x4.trans.shared.b16 [%0], {%1, %2, %3, %4};"
                 ::"r"(a), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]) : "memory");
}
__device__ __forceinline__ void ldsm_x2(uint32_t a, uint32_t (&v)[2]) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0, %1}, [%2];" : "=r"(v[0]), "=r"(v[1]) : "r"(a)
                 : "memory");
}
__device__ __forceinline__ void stsm_x2_trans(uint32_t a, const uint32_t (&v)[2]) {
    asm volatile("stmatrix.sync.aligned.m8n8.x2.trans.shared.b16 [%0], {%1, %2};" ::"r"(a), "r"(v[0]), "r"(v[1])
                 : "memory");
}

// Shared-memory barriers of the kernel (one block; see k_conv3_tc for who arrives where)
struct ConvBars {
    uint64_t *st_full, *st_empty, *h_full, *h_empty, *t_full, *t_empty, *mma_done, *w_full, *w_empty;
};

// Tap row DY of one unit: waits for the halo rows it is the first to read (and, with a
// weight ring, for its three weight boxes), then 3 taps x TR output rows x KS 16-channel
// steps of MMAs with every descriptor a compile-time offset from two bases, then commits
// the halo rows it is the last to read (and its weight slot). Straight-line issue: a
// runtime loop, switch or branch between tcgen05.mma instructions measured ~60-250 extra
// cycles per MMA against ~46-64 for a straight run.
template <int N, int KS, bool RES, int DY>
__device__ __forceinline__ bool conv_tap_row(uint32_t acc, uint32_t halo, uint32_t wsm, int u, int cb, uint32_t accf,
                                             const ConvBars& b, volatile int* abort) {
    using CF = CfgC<N>;
    constexpr int TR = CF::TR, HR = CF::HR, R = CF::kRows;
    constexpr int r0 = DY == 0 ? 0 : TR + DY - 1, r1 = TR + DY;  // halo rows first read here
#pragma unroll
    for (int hr = r0; hr < r1; ++hr)
        if (!mbar_wait_ab(&b.h_full[hr], (uint32_t)u & 1u, nullptr, abort)) return false;
    int slot;
    if constexpr (RES) {
        slot = cb * 3 + DY;
    } else {
        const int g = u * 3 + DY;
        slot = g % R;
        if (!mbar_wait_ab(&b.w_full[slot], (uint32_t)(g / R) & 1u, nullptr, abort)) return false;
    }
    fence_after_sync();
    constexpr uint32_t idesc = idesc_bf16(128, N);
    const uint64_t a0 = smem_desc_sw128(halo), b0 = smem_desc_sw128(wsm + (uint32_t)slot * 3u * CF::kB);
#pragma unroll
    for (int dx = 0; dx < 3; ++dx)
#pragma unroll
        for (int r = 0; r < TR; ++r)
#pragma unroll
            for (int kk = 0; kk < KS; ++kk) {
                const uint64_t ad = a0 + (uint64_t)((((r + DY) * kHaloBytes + dx * 128) >> 4) + kk * 2);
                const uint64_t bd = b0 + (uint64_t)(((dx * CF::kB) >> 4) + kk * 2);
                mma_bf16(acc + (uint32_t)(r * N), ad, bd, idesc, (DY == 0 && dx == 0 && kk == 0) ? accf : 1u);
            }
    if constexpr (!RES) mma_commit(&b.w_empty[slot]);
    if constexpr (DY < 2) {
        mma_commit(&b.h_empty[DY]);
    } else {
#pragma unroll
        for (int hr = 2; hr < HR; ++hr) mma_commit(&b.h_empty[hr]);
    }
    return true;
}

// Tap row DY with swapped operands (N = 256 on planes of side 64): per tap, a wait for its
// weight box (a granule of one tap), then TR output rows x two 128-channel halves x KS
// steps: A = rows 128 h .. of the box, B = the halo view (64 pixel rows from dx), D =
// columns (r * 2 + h) * 64 of the accumulator (TMEM lane = output channel, column = pixel).
template <int N, int KS, bool RES, int DY>
__device__ __forceinline__ bool conv_tap_row_sw(uint32_t acc, uint32_t halo, uint32_t wsm, int u, int cb,
                                                uint32_t accf, const ConvBars& b, volatile int* abort) {
    using CF = CfgC<N>;
    constexpr int TR = CF::TR, HR = CF::HR, R = CF::kRows, NH = N / 128, PX = CF::PX;
    constexpr int r0 = DY == 0 ? 0 : TR + DY - 1, r1 = TR + DY;
#pragma unroll
    for (int hr = r0; hr < r1; ++hr)
        if (!mbar_wait_ab(&b.h_full[hr], (uint32_t)u & 1u, nullptr, abort)) return false;
    constexpr uint32_t idesc = idesc_bf16(128, PX);
    const uint64_t h0 = smem_desc_sw128(halo);
#pragma unroll
    for (int dx = 0; dx < 3; ++dx) {
        const int tap = DY * 3 + dx;
        int slot;
        if constexpr (RES) {
            slot = cb * 9 + tap;
        } else {
            const int g = u * 9 + tap;
            slot = g % R;
            if (!mbar_wait_ab(&b.w_full[slot], (uint32_t)(g / R) & 1u, nullptr, abort)) return false;
        }
        fence_after_sync();
        const uint64_t w0 = smem_desc_sw128(wsm + (uint32_t)slot * CF::kB);
#pragma unroll
        for (int r = 0; r < TR; ++r)
#pragma unroll
            for (int h = 0; h < NH; ++h)
#pragma unroll
                for (int kk = 0; kk < KS; ++kk) {
                    const uint64_t ad = w0 + (uint64_t)(((h * 128 * 128) >> 4) + kk * 2);
                    const uint64_t bd = h0 + (uint64_t)((((r + DY) * kHaloBytes + dx * 128) >> 4) + kk * 2);
                    mma_bf16(acc + (uint32_t)((r * NH + h) * PX), ad, bd, idesc,
                             (DY == 0 && dx == 0 && kk == 0) ? accf : 1u);
                }
        if constexpr (!RES) mma_commit(&b.w_empty[slot]);
    }
    if constexpr (DY < 2) {
        mma_commit(&b.h_empty[DY]);
    } else {
#pragma unroll
        for (int hr = 2; hr < HR; ++hr) mma_commit(&b.h_empty[hr]);
    }
    return true;
}

// One unit with the vertical taps stacked (N = 32): its three (channel block, dx) weight
// boxes first (resident: waited once before the first tile), then per halo row hr, once it
// is in, 3 dx x KS products of N = 96 into TMEM columns 32 hr .. (accumulating onto the
// zeroed accumulator), and the release of that halo row; the boxes are released at the end.
template <int N, int KS, bool RES>
__device__ __forceinline__ bool conv_unit_st(uint32_t acc, uint32_t halo, uint32_t wsm, int u, int cb,
                                             const ConvBars& b, volatile int* abort) {
    using CF = CfgC<N>;
    constexpr int HR = CF::HR, R = CF::kRows;
    // the unit's boxes are consecutive granules: slots s0, s0 + 1, s0 + 2 (mod R)
    const int g0 = RES ? cb * 3 : u * 3;
    const int s0 = RES ? g0 : g0 % R, s1 = RES ? g0 + 1 : (g0 + 1) % R, s2 = RES ? g0 + 2 : (g0 + 2) % R;
    if constexpr (!RES) {
        if (!mbar_wait_ab(&b.w_full[s0], (uint32_t)(g0 / R) & 1u, nullptr, abort) ||
            !mbar_wait_ab(&b.w_full[s1], (uint32_t)((g0 + 1) / R) & 1u, nullptr, abort) ||
            !mbar_wait_ab(&b.w_full[s2], (uint32_t)((g0 + 2) / R) & 1u, nullptr, abort))
            return false;
    }
    constexpr uint32_t idesc = idesc_bf16(128, 3 * N);
    const uint64_t a0 = smem_desc_sw128(halo);
    const uint64_t wd0 = smem_desc_sw128(wsm + (uint32_t)s0 * CF::kB), wd1 = smem_desc_sw128(wsm + (uint32_t)s1 * CF::kB),
                   wd2 = smem_desc_sw128(wsm + (uint32_t)s2 * CF::kB);
    // a runtime loop over the halo rows (each starts with a wait, a branch anyway); the 3 x KS
    // products of one row are one unrolled run
#pragma unroll 1
    for (int hr = 0; hr < HR; ++hr) {
        if (!mbar_wait_ab(&b.h_full[hr], (uint32_t)u & 1u, nullptr, abort)) return false;
        fence_after_sync();
#pragma unroll
        for (int dx = 0; dx < 3; ++dx)
#pragma unroll
            for (int kk = 0; kk < KS; ++kk) {
                const uint64_t ad = a0 + (uint64_t)(((hr * kHaloBytes + dx * 128) >> 4) + kk * 2);
                mma_bf16(acc + (uint32_t)(hr * N), ad, (dx == 0 ? wd0 : dx == 1 ? wd1 : wd2) + (uint64_t)(kk * 2), idesc, 1u);
            }
        mma_commit(&b.h_empty[hr]);
    }
    if constexpr (!RES) {
        mma_commit(&b.w_empty[s0]);
        mma_commit(&b.w_empty[s1]);
        mma_commit(&b.w_empty[s2]);
    }
    return true;
}

template <int N, int KS, bool RES>
__device__ __forceinline__ bool conv_unit(uint32_t acc, uint32_t halo, uint32_t wsm, int u, int cb, uint32_t accf,
                                          const ConvBars& b, volatile int* abort) {
    if constexpr (CfgC<N>::ST)
        return conv_unit_st<N, KS, RES>(acc, halo, wsm, u, cb, b, abort);
    else if constexpr (CfgC<N>::SW)
        return conv_tap_row_sw<N, KS, RES, 0>(acc, halo, wsm, u, cb, accf, b, abort) &&
               conv_tap_row_sw<N, KS, RES, 1>(acc, halo, wsm, u, cb, accf, b, abort) &&
               conv_tap_row_sw<N, KS, RES, 2>(acc, halo, wsm, u, cb, accf, b, abort);
    else
        return conv_tap_row<N, KS, RES, 0>(acc, halo, wsm, u, cb, accf, b, abort) &&
               conv_tap_row<N, KS, RES, 1>(acc, halo, wsm, u, cb, accf, b, abort) &&
               conv_tap_row<N, KS, RES, 2>(acc, halo, wsm, u, cb, accf, b, abort);
}

// The MMA issuer (one thread): tile i into TMEM accumulator i & 1, its channel blocks in
// order (the first overwrites the accumulator), then a commit to t_full. With resident
// weights every granule is waited for once, before the first tile.
template <int N, bool RES>
__device__ __forceinline__ void conv_mma_role(int T, int ncb, int Cin, uint32_t tmem, uint32_t halo, uint32_t wsm,
                                              const ConvBars& b, volatile int* abort) {
    bool ok = true;
    if constexpr (RES)
        for (int g = 0; g < CfgC<N>::GPU * ncb && ok; ++g) ok = mbar_wait_ab(&b.w_full[g], 0u, nullptr, abort);
    for (int i = 0; i < T && ok; ++i) {
        const int buf = i & 1;
        // the accumulator free: drained by the epilogue (and, stacked, zeroed: every tile waits,
        // the first two on the initial zeroing)
        const bool wait_acc = CfgC<N>::ST || i >= 2;
        const uint32_t par = CfgC<N>::ST ? (uint32_t)(i >> 1) & 1u : (uint32_t)((i >> 1) - 1) & 1u;
        if (wait_acc && !mbar_wait_ab(&b.t_empty[buf], par, nullptr, abort)) {
            ok = false;
            break;
        }
        fence_after_sync();
        const uint32_t acc = tmem + (uint32_t)(buf * CfgC<N>::kAcc);
        for (int cb = 0; cb < ncb && ok; ++cb) {
            const int u = i * ncb + cb;
            const uint32_t accf = cb == 0 ? 0u : 1u;
            switch (min(64, Cin - cb * 64) / 16) {
                case 4: ok = conv_unit<N, 4, RES>(acc, halo, wsm, u, cb, accf, b, abort); break;
                case 3: ok = conv_unit<N, 3, RES>(acc, halo, wsm, u, cb, accf, b, abort); break;
                case 2: ok = conv_unit<N, 2, RES>(acc, halo, wsm, u, cb, accf, b, abort); break;
                default: ok = conv_unit<N, 1, RES>(acc, halo, wsm, u, cb, accf, b, abort); break;
            }
        }
        if (ok) mma_commit(&b.t_full[buf]);
    }
    mma_commit(b.mma_done);  // also after a failure: the MMAs in flight complete before TMEM is freed
    mbar_wait(b.mma_done, 0, nullptr);
}

// Persistent, warp-specialised. CTA b takes the contiguous tiles [t0, t1) of the list
// (image n, row group, 128-pixel segment), n-major, and each tile's ceil(Cin / 64) channel
// blocks in order (units u = 0 .. U - 1); raw row k = HR u + hr is halo row hr of unit u.
// Roles (320 threads):
//   warp 8, lane 0   TMA, polling two queues: raw row k into slot k % RS once the
//                    transposers have emptied the slot, and the weights by tap row (the
//                    three boxes of one (channel block, dy)): all at the start when
//                    resident, else one tap row per (unit, dy) into a ring slot the MMAs
//                    have released;
//   warps 4-7        halo row hr of unit u from raw row k, once the MMAs of unit u - 1 have
//                    released that halo row (rows 0 and 1 after their taps dy = 0 and 1,
//                    the others after the last tap);
//   warp 9, lane 0   the MMAs of a tile into TMEM accumulator i & 1 (tile i), tap row dy as
//                    soon as halo rows dy .. dy + TR - 1 of the unit are in (conv_mma_role);
//   warps 0-3        a tile's epilogue (TMEM lane = pixel; bias, ReLU, bf16 NCHW stores)
//                    while the next tile's MMAs run.
template <int N>
__global__ void __launch_bounds__(320, 1)
k_conv3_tc(const __grid_constant__ CUtensorMap tmXA, const __grid_constant__ CUtensorMap tmXB, int CA, int CB,
           const __grid_constant__ CUtensorMap tmW, const float* __restrict__ bias, bf16* __restrict__ Y, int H,
           int Wd, int nb, int pb) {
    using CF = CfgC<N>;
    constexpr int TR = CF::TR, HR = CF::HR, RS = CF::RS, R = CF::kRows;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* sA = smem;                    // [HR][kHaloRows][128 B] halo rows
    uint8_t* sS = sA + CF::kA;             // [RS][8 channel groups][8 planes][152 px] raw rows
    uint8_t* misc = sS + CF::kStg;         // barriers, TMEM address, abort flag, dummy rows
    uint8_t* sB = misc + 1024;             // [R][GT taps][N][128 B] weight boxes
    uint64_t* st_full = reinterpret_cast<uint64_t*>(misc);  // [RS]
    uint64_t* st_empty = st_full + 4;      // [RS]
    uint64_t* h_full = st_full + 8;        // [HR]
    uint64_t* h_empty = st_full + 16;      // [HR]
    uint64_t* t_full = st_full + 24;       // [2]
    uint64_t* t_empty = st_full + 26;      // [2]
    uint64_t* mma_done = st_full + 28;
    uint64_t* w_full = st_full + 29;       // [R]
    uint64_t* w_empty = w_full + R;        // [R]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(w_empty + R);
    volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
    uint8_t* dummy = misc + 896;           // 8 x 16 B: stored matrix rows that fall outside a halo block
    static_assert(HR <= 8 && RS <= 4 && (29 + 2 * R) * 8 + 8 <= 896, "barrier block");

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int Cin = CA + CB, ncb = (Cin + 63) / 64;
    const bool resident = CF::GPU * ncb <= R;  // every weight box of the layer stays in shared memory
    const int segs = (Wd + CF::PX - 1) / CF::PX, rgroups = (H + TR - 1) / TR;
    const long long tiles = (long long)nb * rgroups * segs;
    const int t0 = (int)(tiles * blockIdx.x / gridDim.x), t1 = (int)(tiles * (blockIdx.x + 1) / gridDim.x);
    const int T = t1 - t0, U = T * ncb;
    const size_t plane = (size_t)H * Wd;
    auto tile_of = [&](int t, int& n, int& y0, int& x0) {
        x0 = (t % segs) * CF::PX;
        const int r = t / segs;
        y0 = (r % rgroups) * TR;
        n = r / rgroups;
    };

    if (threadIdx.x == 0) {
        for (int i = 0; i < RS; ++i) {
            mbar_init(&st_full[i], 1);
            mbar_init(&st_empty[i], 4);  // one arrival per transposing warp
        }
        for (int i = 0; i < HR; ++i) {
            mbar_init(&h_full[i], 4);
            mbar_init(&h_empty[i], 1);   // MMA commit
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&t_full[i], 1);
            mbar_init(&t_empty[i], 4);   // one arrival per epilogue warp
        }
        mbar_init(mma_done, 1);
        for (int i = 0; i < R; ++i) {
            mbar_init(&w_full[i], 1);
            mbar_init(&w_empty[i], 1);
        }
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 9) tmem_alloc(tmem_slot, CF::kCols);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    if (warp == 8) {
        // ---------------- TMA: raw rows and weight boxes
        if (lane == 0 && U > 0) {
            const int rows = U * HR, wtot = resident ? CF::GPU * ncb : CF::GPU * U;
            int k = 0, ws = 0;
            bool idle = false;
            unsigned long long t_idle = 0;
            while (k < rows || ws < wtot) {
                bool prog = false;
                if (k < rows && (k < RS || mbar_test_wait(&st_empty[k % RS], (uint32_t)((k / RS) - 1) & 1u))) {
                    const int u = k / HR, hr = k % HR, cb = u % ncb, ci0 = cb * 64, ncg = min(64, Cin - ci0) / 8;
                    int n, y0, x0;
                    tile_of(t0 + u / ncb, n, y0, x0);
                    uint8_t* dst = sS + (k % RS) * kStgRow;
                    mbar_arrive_expect_tx(&st_full[k % RS], (uint32_t)ncg * kStgBox);
                    for (int g = 0; g < ncg; g += pb / 8) {  // boxes of pb planes (8 or 32)
                        const int ci = ci0 + 8 * g;
                        if (ci < CA) tma_load_3d(&tmXA, &st_full[k % RS], dst + g * kStgBox, x0 - 8, y0 - 1 + hr, n * CA + ci);
                        else tma_load_3d(&tmXB, &st_full[k % RS], dst + g * kStgBox, x0 - 8, y0 - 1 + hr, n * CB + (ci - CA));
                    }
                    ++k;
                    prog = true;
                }
                if (ws < wtot && (resident || ws < R || mbar_test_wait(&w_empty[ws % R], (uint32_t)((ws / R) - 1) & 1u))) {
                    // granule ws: (channel block ws / GPU, granule ws % GPU) resident, else
                    // (unit ws / GPU, granule ws % GPU); its boxes are kBoxPerCb cb + GT granule + j
                    const int sl = resident ? ws : ws % R;
                    const int box =
                        resident ? CF::GT * ws : ((ws / CF::GPU) % ncb) * CF::kBoxPerCb + (ws % CF::GPU) * CF::GT;
                    mbar_arrive_expect_tx(&w_full[sl], CF::GT * CF::kB);
                    for (int j = 0; j < CF::GT; ++j)
                        tma_load_2d(&tmW, &w_full[sl], sB + (sl * CF::GT + j) * CF::kB, 0, (box + j) * CF::kBoxRows);
                    ++ws;
                    prog = true;
                }
                if (prog) {
                    idle = false;
                } else if (!idle) {
                    idle = true;
                    t_idle = globaltimer();
                } else if (*abort || globaltimer() - t_idle > kWaitNs) {
                    *abort = 1;
                    break;
                }
            }
            if (*abort) {  // the copies still in flight land before the CTA exits (bounded waits)
                for (int j = max(0, k - RS); j < k; ++j) mbar_wait(&st_full[j % RS], (uint32_t)(j / RS) & 1u, nullptr);
                for (int j = resident ? 0 : max(0, ws - R); j < ws; ++j)
                    mbar_wait(&w_full[resident ? j : j % R], resident ? 0u : (uint32_t)(j / R) & 1u, nullptr);
            }
        }
    } else if (warp >= 4 && warp < 8) {
        // ---------------- halo rows from raw rows: 8 planes x 8 pixels per matrix
        const int tw = warp - 4, m = lane >> 3, r = lane & 7;
        for (int k = 0; k < U * HR; ++k) {
            const int u = k / HR, hr = k % HR, cb = u % ncb, ncg = min(64, Cin - cb * 64) / 8;
            bool w = mbar_wait_ab(&st_full[k % RS], (uint32_t)(k / RS) & 1u, nullptr, abort);
            if (w && u > 0) w = mbar_wait_ab(&h_empty[hr], (uint32_t)(u - 1) & 1u, nullptr, abort);
            if (!__all_sync(0xffffffffu, w)) break;
            const uint8_t* raw = sS + (k % RS) * kStgRow;
            uint8_t* blk = sA + hr * kHaloBytes;
            // items (channel group g, part): parts 0-3 transpose pixel blocks 4 part + m
            // (x4), part 4 blocks 16 and 17 (x2); pixel block b holds pixels x0 - 8 + 8 b ..,
            // stored at halo row p = 8 b + j - 7 (rows outside 0 .. 135 go to the dummy rows)
            for (int it = tw; it < ncg * 5; it += 4) {
                const int part = it % 5, g = it / 5;
                const int b = part < 4 ? 4 * part + m : 16 + (m & 1);
                const uint32_t la = smem_u32(raw + g * kStgBox + r * (kStgPx * 2) + b * 16);
                const int p = 8 * b + r - 7;
                const uint32_t sa = (p >= 0 && p < kHaloRows)
                                        ? smem_u32(blk + p * 128 + (((uint32_t)g ^ (uint32_t)(p & 7)) << 4))
                                        : smem_u32(dummy + r * 16);
                if (part < 4) {
                    uint32_t v[4];
                    ldsm_x4(la, v);
                    stsm_x4_trans(sa, v);
                } else {
                    uint32_t v[2];
                    ldsm_x2(la, v);
                    stsm_x2_trans(sa, v);
                }
            }
            fence_proxy_async_smem();  // generic-proxy stores -> visible to the tensor core
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&h_full[hr]);
                mbar_arrive(&st_empty[k % RS]);
            }
        }
    } else if (warp == 9) {
        // ---------------- MMA issuer
        if (lane == 0) {
            const ConvBars bars{st_full, st_empty, h_full, h_empty, t_full, t_empty, mma_done, w_full, w_empty};
            if (resident) conv_mma_role<N, true>(T, ncb, Cin, tmem, smem_u32(sA), smem_u32(sB), bars, abort);
            else conv_mma_role<N, false>(T, ncb, Cin, tmem, smem_u32(sA), smem_u32(sB), bars, abort);
        }
    } else if constexpr (CF::SW) {
        // ---------------- epilogue, swapped operands: TMEM lanes 32 w .. (output channels of
        // half h), columns (r * 2 + h) * 64 .. (pixels): each thread writes its channel's
        // 64-pixel row (128 bytes) of output row y0 + r
        constexpr int NH = N / 128, PX = CF::PX;
        bool good = true;
        for (int i = 0; i < T; ++i) {
            const int buf = i & 1;
            if (good) {
                const bool w = mbar_wait_ab(&t_full[buf], (uint32_t)(i >> 1) & 1u, nullptr, abort);
                good = __all_sync(0xffffffffu, w);
            }
            fence_after_sync();
            int n, y0, x0;
            tile_of(t0 + i, n, y0, x0);
            for (int r = 0; r < TR; ++r) {
                const int y = y0 + r;
                for (int h = 0; h < NH; ++h) {
                    const int co = h * 128 + warp * 32 + lane;
                    static_assert(PX == 64, "two 32-column loads per row");
                    uint32_t v0[32], v1[32];  // pixels 0-31 and 32-63
                    if (good) {
                        const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(buf * CF::kAcc + (r * NH + h) * PX);
                        tmem_ld32(ta, v0);
                        tmem_ld32(ta + 32u, v1);
                    } else {
#pragma unroll
                        for (int j = 0; j < 32; ++j) v0[j] = v1[j] = 0x7fc00000u;  // NaN: the result is unusable
                    }
                    if (y < H) {
                        const float bv = bias[co];
                        uint4* dst = reinterpret_cast<uint4*>(Y + (((size_t)n * N + co) * H + y) * Wd + x0);
#pragma unroll
                        for (int q = 0; q < PX / 8; ++q) {
                            uint32_t pk[4];
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const int j = 8 * q + 2 * e;
                                const float a0 = __uint_as_float(j < 32 ? v0[j] : v1[j - 32]);
                                const float a1 = __uint_as_float(j < 32 ? v0[j + 1] : v1[j - 31]);
                                const __nv_bfloat162 hb = __floats2bfloat162_rn(good ? fmaxf(a0 + bv, 0.f) : a0,
                                                                                 good ? fmaxf(a1 + bv, 0.f) : a1);
                                pk[e] = *reinterpret_cast<const uint32_t*>(&hb);
                            }
                            dst[q] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                        }
                    }
                }
            }
            if (good) {
                fence_before_sync();
                __syncwarp();
                if (lane == 0) mbar_arrive(&t_empty[buf]);
            }
        }
    } else {
        // ---------------- epilogue: TMEM lanes 32 w .. (pixels), columns r N + co of accumulator
        // i & 1 (stacked: (r + 2) N + co, and the accumulator zeroed after the drain; both
        // zeroed before the first tile)
        const uint32_t tlane = tmem + ((uint32_t)(warp * 32) << 16);
        if constexpr (CF::ST) {
            for (int c = 0; c < 2 * CF::kAcc; c += 32) tmem_st32_zero(tlane + (uint32_t)c);
            tmem_wait_st();
            fence_before_sync();
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&t_empty[0]);
                mbar_arrive(&t_empty[1]);
            }
        }
        bool good = true;
        for (int i = 0; i < T; ++i) {
            const int buf = i & 1;
            if (good) {
                const bool w = mbar_wait_ab(&t_full[buf], (uint32_t)(i >> 1) & 1u, nullptr, abort);
                good = __all_sync(0xffffffffu, w);
            }
            fence_after_sync();
            int n, y0, x0;
            tile_of(t0 + i, n, y0, x0);
            const int x = x0 + warp * 32 + lane;
            for (int r = 0; r < TR; ++r) {
                const int y = y0 + r;
                for (int c = 0; c < N; c += 32) {
                    uint32_t v[32];
                    if (good) {
                        tmem_ld32(tlane + (uint32_t)(buf * CF::kAcc + (CF::ST ? r + 2 : r) * N + c), v);
                    } else {
#pragma unroll
                        for (int j = 0; j < 32; ++j) v[j] = 0x7fc00000u;  // NaN: the result is unusable
                    }
                    if (x < Wd && y < H) {
                        bf16* dst = Y + ((size_t)n * N + c) * plane + (size_t)y * Wd + x;
#pragma unroll
                        for (int j = 0; j < 32; ++j) {
                            const float o = fmaxf(__uint_as_float(v[j]) + bias[c + j], 0.f);
                            dst[(size_t)j * plane] = __float2bfloat16_rn(good ? o : __uint_as_float(v[j]));
                        }
                    }
                }
            }
            if (good) {
                if constexpr (CF::ST) {
                    for (int c = 0; c < CF::kAcc; c += 32) tmem_st32_zero(tlane + (uint32_t)(buf * CF::kAcc + c));
                    tmem_wait_st();
                }
                fence_before_sync();
                __syncwarp();
                if (lane == 0) mbar_arrive(&t_empty[buf]);
            }
        }
    }
    __syncwarp();
    fence_before_sync();
    __syncthreads();
    if (warp == 9) {
        fence_after_sync();
        tmem_dealloc(tmem, CF::kCols);
    }
}

// Wtc[cb][tap][co][64] = bf16(W[co][ci = 64 cb + j][tap]), zero for ci >= Cin; stacked
// (Cout = 32): Wtc[cb][dx][s][co][64] with the tap (dy = 2 - s, dx), so that the three
// vertical taps of one dx form one 96-row box
__global__ void k_prep_wtc(const float* __restrict__ W, int Cout, int Cin, int stacked, bf16* __restrict__ Wt) {
    const int ncb = (Cin + 63) / 64;
    const size_t count = (size_t)ncb * 9 * Cout * 64;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (size_t)gridDim.x * blockDim.x) {
        const int j = (int)(i % 64);
        const size_t r = i / 64;
        const int co = (int)(r % Cout), q = (int)((r / Cout) % 9), cb = (int)(r / ((size_t)Cout * 9));
        const int tap = stacked ? (2 - q % 3) * 3 + q / 3 : q;  // stacked: q = 3 dx + s
        const int ci = cb * 64 + j;
        Wt[i] = __float2bfloat16_rn(ci < Cin ? W[((size_t)co * Cin + ci) * 9 + tap] : 0.f);
    }
}

template <int N>
cudaError_t set_attr_conv() {
    return cudaFuncSetAttribute(k_conv3_tc<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CfgC<N>::kSmem);
}

// raw-row map over the NCHW planes of X[nb][C][side][side]: boxes of 152 pixels x 1 row x pb
// planes (a box of pb planes lands as pb / 8 consecutive 8-plane groups of a raw row)
int make_map_rows(CUtensorMap* tm, const bf16* X, int C, int nb, int side, int pb) {
    return tc::make_map_plain3(tm, X, (uint64_t)side, (uint64_t)side, (uint64_t)nb * C, (uint64_t)side * 2,
                               (uint64_t)side * side * 2, kStgPx, 1, (uint32_t)pb);
}

}  // namespace

bool conv3_tc_supported(int Cin, int Cout, int side) {
    const bool rows = (Cout == 32 || Cout == 64 || Cout == 128) && side >= 128 && side % 8 == 0;
    const bool swapped = Cout == 256 && side == CfgC<256>::PX;
    return (rows || swapped) && Cin % 16 == 0 && Cin >= 16;
}

size_t conv3_tc_weight_elems(int Cin, int Cout) { return (size_t)((Cin + 63) / 64) * 9 * Cout * 64; }

int conv3_tc_init_attrs() {
    cudaError_t e = set_attr_conv<32>();
    if (e == cudaSuccess) e = set_attr_conv<64>();
    if (e == cudaSuccess) e = set_attr_conv<128>();
    if (e == cudaSuccess) e = set_attr_conv<256>();
    if (e != cudaSuccess) return cuda_error(e, "conv3_tc_init_attrs");
    return DEVEL_OK;
}

int conv3_tc_make_map(CUtensorMap* tm, const bf16* Wt, int Cin, int Cout) {
    const int rows = (Cin + 63) / 64 * 9 * Cout;
    return tc::make_map(tm, Wt, rows, 64, 64, Cout == 32 ? CfgC<32>::kBoxRows : Cout);
}

int launch_prep_wtc(const float* W, int Cout, int Cin, bf16* Wt, cudaStream_t s) {
    const size_t count = conv3_tc_weight_elems(Cin, Cout);
    k_prep_wtc<<<(unsigned)std::min<size_t>((count + 255) / 256, 152 * 16), 256, 0, s>>>(W, Cout, Cin,
                                                                                          Cout == 32 ? 1 : 0, Wt);
    DEVEL_LAUNCH_CHECK("k_prep_wtc");
    return DEVEL_OK;
}

int launch_conv3_tc(const bf16* XA, int CA, const bf16* XB, int CB, const CUtensorMap& tmW, const float* bias,
                    bf16* Y, int Cout, int nb, int side, cudaStream_t s) {
    if (!conv3_tc_supported(CA + CB, Cout, side) || CA % 8 || CB % 8 || CA < 0 || CB < 0 || (CB > 0 && !XB) || nb < 1)
        return set_error(DEVEL_EINVAL, "conv3_tc: shape (CA %d, CB %d, Cout %d, side %d, nb %d) unsupported", CA, CB,
                         Cout, side, nb);
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        DEVEL_CUDA_TRY(cudaGetDevice(&dev));
        DEVEL_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    }
    // 32-plane boxes when no 32-channel group straddles the two sources or a channel block's
    // end (CA, CB multiples of 32; every channel block then holds 32 or 64 channels), else 8
    const int pb = CA % 32 == 0 && CB % 32 == 0 ? 32 : 8;
    CUtensorMap mA, mB;
    int rc = make_map_rows(&mA, XA, CA, nb, side, pb);
    if (rc == DEVEL_OK) rc = make_map_rows(&mB, CB > 0 ? XB : XA, CB > 0 ? CB : CA, nb, side, pb);
    if (rc != DEVEL_OK) return rc;
    const int px = Cout == 256 ? CfgC<256>::PX : CfgC<64>::PX;
    const int tr = Cout == 32 ? CfgC<32>::TR : CfgC<64>::TR;
    const long long tiles = (long long)nb * ((side + tr - 1) / tr) * ((side + px - 1) / px);
    const unsigned grid = (unsigned)std::min<long long>(tiles, sms);
    switch (Cout) {
        case 32:
            k_conv3_tc<32><<<grid, 320, CfgC<32>::kSmem, s>>>(mA, mB, CA, CB, tmW, bias, Y, side, side, nb, pb);
            break;
        case 64:
            k_conv3_tc<64><<<grid, 320, CfgC<64>::kSmem, s>>>(mA, mB, CA, CB, tmW, bias, Y, side, side, nb, pb);
            break;
        case 128:
            k_conv3_tc<128><<<grid, 320, CfgC<128>::kSmem, s>>>(mA, mB, CA, CB, tmW, bias, Y, side, side, nb, pb);
            break;
        default:
            k_conv3_tc<256><<<grid, 320, CfgC<256>::kSmem, s>>>(mA, mB, CA, CB, tmW, bias, Y, side, side, nb, pb);
            break;
    }
    DEVEL_LAUNCH_CHECK("k_conv3_tc");
    return DEVEL_OK;
}

}  // namespace devel
