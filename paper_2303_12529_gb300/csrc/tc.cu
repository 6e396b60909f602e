// Tensor-core (tcgen05) kernels of the truncated-DFT contractions, sm_103a: the
// n^2-sized work of the SOCS image of Sec. II-B (forward) and of its gradient, Eqs.
// (ilt_gradient), (pvb_gradient) (adjoint), both taken through the difference window.
//
// Operands are bf16 hi/lo pairs (x = hi + lo, hi = rn_bf16(x), lo = rn_bf16(x - hi));
// products are compensated, A B^T ~ A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T, with
// FP32 accumulation in TMEM (the A_lo term is skipped when A is exact in bf16, e.g.
// a 0/1 mask). UMMA M = 128, cta_group::1, K-major operands in 128-byte-swizzled
// shared memory fed by TMA.
//
//   k_tc_gemm    small NT GEMM, one 128 x BN tile per CTA, bf16 hi/lo output
//                (the expansion operand T = E Z);
//   k_tc_spec2   reduction of an image onto a window: both contractions in one CTA;
//   k_tc_expand  persistent expansion of a window onto the image.
//
// Every mbarrier wait is bounded (about one second of %globaltimer); a timeout sets
// *err = DEVEL_ETIMEOUT and the CTA stops issuing work, waits (bounded) for the
// copies it issued, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cfloat>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "tc.cuh"
#include "tc_ptx.cuh"

namespace devel {
namespace tc {
namespace {

// The compensated products of one 64-wide K slab, KS 16-deep steps, issued as one unrolled
// run (counts known at compile time: the issuing thread measured about twice the cycles per
// MMA when a runtime-bounded loop or a runtime branch sat between the MMAs).
//   ACC3: the three products into accumulators d, d + dstep, d + 2 dstep (summed later),
//         else all three into d;
//   ALO:  the A_lo B_hi product (skipped when A is exact in bf16);
//   first: the first slab of the accumulation (its first step overwrites).
template <int KS, bool ACC3, bool ALO>
__device__ __forceinline__ void slab_mmas(uint32_t d, uint32_t dstep, uint64_t dAhi, uint64_t dAlo, uint64_t dBhi,
                                          uint64_t dBlo, uint32_t idesc, bool first) {
#pragma unroll
    for (int kk = 0; kk < KS; ++kk) {
        const uint64_t adv = (uint64_t)(kk * 32) >> 4;  // 16 bf16 = 32 bytes along K
        const uint32_t acc = (first && kk == 0) ? 0u : 1u;
        if (ACC3) {
            mma_bf16(d, dAhi + adv, dBhi + adv, idesc, acc);
            mma_bf16(d + dstep, dAhi + adv, dBlo + adv, idesc, acc);
            if (ALO) mma_bf16(d + 2 * dstep, dAlo + adv, dBhi + adv, idesc, acc);
        } else {
            mma_bf16(d, dAhi + adv, dBhi + adv, idesc, acc);
            mma_bf16(d, dAhi + adv, dBlo + adv, idesc, 1u);
            if (ALO) mma_bf16(d, dAlo + adv, dBhi + adv, idesc, 1u);
        }
    }
}

// slab_mmas with the step count and the A_lo product chosen at run time (one branch per slab)
template <bool ACC3>
__device__ __forceinline__ void slab_mmas_rt(int ks, bool alo, uint32_t d, uint32_t dstep, uint64_t dAhi,
                                             uint64_t dAlo, uint64_t dBhi, uint64_t dBlo, uint32_t idesc,
                                             bool first) {
#define DEVEL_SLAB(k)                                                                               \
    if (ks == k) {                                                                                  \
        if (alo) slab_mmas<k, ACC3, true>(d, dstep, dAhi, dAlo, dBhi, dBlo, idesc, first);          \
        else slab_mmas<k, ACC3, false>(d, dstep, dAhi, dAlo, dBhi, dBlo, idesc, first);             \
        return;                                                                                     \
    }
    DEVEL_SLAB(4) DEVEL_SLAB(3) DEVEL_SLAB(2) DEVEL_SLAB(1)
#undef DEVEL_SLAB
}

template <int BN>
struct Cfg {
    static constexpr uint32_t kBBytes = BN * kBK * 2;
    static constexpr uint32_t kStage = 2 * kABytes + 2 * kBBytes;
    // two stages: the GEMM's contraction (a folded table's width, <= 128) is at most two
    // k-blocks deep, and two or more CTAs then fit on an SM
    static constexpr int kFit = (int)((227u * 1024u - 2048u) / kStage);
    static constexpr int kStages = kFit > 2 ? 2 : kFit;
    static_assert(kFit >= 2, "tile too wide for double buffering");
    static constexpr uint32_t kCols = BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256;
    static constexpr size_t kSmem = 1024 + (size_t)kStages * kStage + 256;
};

// One 128 x BN tile of D = A B^T per CTA, clip blockIdx.z of a batch (B: a 3-D map over the
// clips; D of clip z at ep.Chi / ep.Clo + z * ep.split_stride):
//   warp 0, one thread   TMA producer: 64-element K slabs of A_hi, A_lo, B_hi, B_lo
//                        into a STAGES ring;
//   warp 1, one thread   MMA issuer: 4 K-steps of 16 per slab, 3 MMAs each;
//   warps 0-3            epilogue: tcgen05.ld 32 lanes x 16 columns, scale, bf16 hi/lo
//                        split into ep.Chi / ep.Clo (row pitch ep.ldh).
template <int BN>
__global__ void __launch_bounds__(128, 1)
k_tc_gemm(const __grid_constant__ CUtensorMap tmAhi, const __grid_constant__ CUtensorMap tmAlo,
          const __grid_constant__ CUtensorMap tmBhi, const __grid_constant__ CUtensorMap tmBlo, int M, int N,
          int kb_total, int ksteps_last, int use_alo, const EpiArgs ep, int* err) {
    using CF = Cfg<BN>;
    constexpr int S = CF::kStages;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + S * CF::kStage);
    uint64_t* empty = full + S;
    uint64_t* accum = empty + S;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * BN, clip = blockIdx.z;
    const int kb0 = 0, nkb = kb_total;

    auto stage_ptr = [&](int s, int which) -> uint8_t* {
        // which: 0 A_hi, 1 A_lo, 2 B_hi, 3 B_lo
        uint8_t* base = smem + s * CF::kStage;
        return which < 2 ? base + which * kABytes : base + 2 * kABytes + (which - 2) * CF::kBBytes;
    };
    const uint32_t bytes = (use_alo ? 2 : 1) * kABytes + 2 * CF::kBBytes;
    pdl_trigger();
    int issued = 0;  // producer: slabs whose loads were issued
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(accum, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        // A (a DFT table, constant) of the first stages before the previous kernel has
        // finished; B (its output) after the wait
        const int npre = min(nkb, S);
        for (int i = 0; i < npre; ++i) {
            mbar_arrive_expect_tx(&full[i], bytes);
            tma_load_2d(&tmAhi, &full[i], stage_ptr(i, 0), (kb0 + i) * kBK, m0);
            if (use_alo) tma_load_2d(&tmAlo, &full[i], stage_ptr(i, 1), (kb0 + i) * kBK, m0);
        }
        pdl_wait();
        for (int i = 0; i < npre; ++i) {
            tma_load_3d(&tmBhi, &full[i], stage_ptr(i, 2), (kb0 + i) * kBK, n0, clip);
            tma_load_3d(&tmBlo, &full[i], stage_ptr(i, 3), (kb0 + i) * kBK, n0, clip);
        }
        issued = npre;
    }
    if (warp == 1) tmem_alloc(tmem_slot, CF::kCols);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    bool ok = true;
    if (warp == 0 && lane == 0 && nkb > 0) {
        for (int i = issued; i < nkb; ++i) {
            const int s = i % S;
            if (i >= S && !mbar_wait(&empty[s], ((i / S) - 1) & 1, err)) {
                ok = false;
                break;
            }
            mbar_arrive_expect_tx(&full[s], bytes);
            const int kc = (kb0 + i) * kBK;
            tma_load_2d(&tmAhi, &full[s], stage_ptr(s, 0), kc, m0);
            if (use_alo) tma_load_2d(&tmAlo, &full[s], stage_ptr(s, 1), kc, m0);
            tma_load_3d(&tmBhi, &full[s], stage_ptr(s, 2), kc, n0, clip);
            tma_load_3d(&tmBlo, &full[s], stage_ptr(s, 3), kc, n0, clip);
            ++issued;
        }
    } else if (warp == 1 && lane == 0 && nkb > 0) {
        constexpr uint32_t idesc = idesc_bf16(kBM, BN);
        for (int i = 0; i < nkb; ++i) {
            const int s = i % S;
            if (!mbar_wait(&full[s], (i / S) & 1, err)) {
                ok = false;
                break;
            }
            fence_after_sync();
            const int ksteps = (kb0 + i == kb_total - 1) ? ksteps_last : kBK / 16;
            const uint64_t dAhi = smem_desc_sw128(smem_u32(stage_ptr(s, 0)));
            const uint64_t dAlo = smem_desc_sw128(smem_u32(stage_ptr(s, 1)));
            const uint64_t dBhi = smem_desc_sw128(smem_u32(stage_ptr(s, 2)));
            const uint64_t dBlo = smem_desc_sw128(smem_u32(stage_ptr(s, 3)));
            slab_mmas_rt<false>(ksteps, use_alo != 0, tmem, 0u, dAhi, dAlo, dBhi, dBlo, idesc, i == 0);
            mma_commit(&empty[s]);
        }
        if (ok) mma_commit(accum);
    }
    __syncwarp();

    // ---- epilogue: warp w owns accumulator lanes 32w .. 32w + 31 (rows of the tile)
    bool have = nkb > 0;
    if (have) have = mbar_wait(accum, 0, err);
    have = __all_sync(0xffffffffu, have);  // tcgen05.ld below is warp-collective
    fence_after_sync();
    const int row = m0 + warp * 32 + lane;
    const float scale = ep.scale;
    for (int c = 0; c < BN; c += 16) {
        float v[16];
        if (have) {
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
        } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = 0.f;
        }
        const int col0 = n0 + c;
        if (row < M && col0 < N) {
            __nv_bfloat16* dh = ep.Chi + clip * ep.split_stride + (size_t)row * ep.ldh + col0;
            __nv_bfloat16* dl = ep.Clo + clip * ep.split_stride + (size_t)row * ep.ldh + col0;
            __align__(16) __nv_bfloat16 h[16], l[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const float x = v[j] * scale;
                h[j] = __float2bfloat16_rn(x);
                l[j] = __float2bfloat16_rn(x - __bfloat162float(h[j]));
            }
            if (col0 + 16 <= N && ((reinterpret_cast<uintptr_t>(dh) | reinterpret_cast<uintptr_t>(dl)) & 15u) == 0) {
                reinterpret_cast<uint4*>(dh)[0] = reinterpret_cast<const uint4*>(h)[0];
                reinterpret_cast<uint4*>(dh)[1] = reinterpret_cast<const uint4*>(h)[1];
                reinterpret_cast<uint4*>(dl)[0] = reinterpret_cast<const uint4*>(l)[0];
                reinterpret_cast<uint4*>(dl)[1] = reinterpret_cast<const uint4*>(l)[1];
            } else {
                for (int j = 0; j < 16 && col0 + j < N; ++j) {
                    dh[j] = h[j];
                    dl[j] = l[j];
                }
            }
        }
    }
    // a producer that stopped early waits (bounded) for the loads it issued
    if (warp == 0 && lane == 0 && !ok) {
        for (int i = max(0, issued - S); i < issued; ++i) mbar_wait(&full[i % S], (i / S) & 1, nullptr);
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        fence_after_sync();
        tmem_dealloc(tmem, CF::kCols);
    }
}

// ---------------------------------------------------------------------------
// Fused reduction onto a window: both contractions in one kernel
// ---------------------------------------------------------------------------
// The table is the folded one (BN = ldf rows: cos j for j = 0..r, sin j at row r + j).
// CTA (row tile m0 of 128 image rows y, K slice z of `split` columns x):
//   phase 1  D1[y][c] = sum_x X[y][x] basis[c][x]            (M = 128, N = BN)
//   phase 2  D1 is drained from TMEM, split to bf16 hi/lo and written transposed into shared
//            memory as a K-major operand B2[c2][y] (128-byte swizzle, as TMA would lay it out);
//            D2[c1][c2] = sum_y basis[c1][y] D1[y][c2]       (M = 128 >= BN, A2 by TMA)
//   store    the kw x kw block of D2 (cos / sin products at |frequencies| j1, j2) is staged
//            in shared memory and copied with coalesced rows to slice
//            blockIdx.y * gridDim.z + blockIdx.z of clip blockIdx.x's slices in G
//            ([clips][slices][kw][kc] floats, kc = round_up(kw, 16));
// k_spec_sum then adds the slices in slice order, forms the complex entries (+-j1, +-j2)
// and scales by 1/n^2.
// Every sum runs in a fixed order, so the result does not depend on timing. 8 warps: warps
// w and w + 4 share TMEM lanes 32 (w % 4).. and split the drains' 16-column chunks. Two
// CTAs fit on an SM (shared memory and TMEM), so one CTA's drains and second contraction
// overlap the other's loads.
template <int BN>
struct Cfg2 {
    static_assert(BN <= 128, "the folded table of a window fits one 128-row block");
    static constexpr uint32_t kB2 = BN * 128;                  // one k-block of B2 (bf16, 64 y)
    static constexpr uint32_t kStage = Cfg<BN>::kStage;
    // ring stages: as many as leave room for two CTAs per SM (at least 2, at most 4)
    static constexpr int kFit = (int)((110u * 1024u) / kStage);
    static constexpr int kStages = kFit < 2 ? 2 : kFit > 4 ? 4 : kFit;
    static constexpr uint32_t kPhase2 = 4 * kB2 + 4 * kABytes;  // B2 hi/lo, A2 hi/lo (2 k-blocks each)
    static constexpr uint32_t kRing = kStages * kStage;
    static constexpr uint32_t kArena = kRing > kPhase2 ? kRing : kPhase2;
    // one accumulator per compensation product (three independent MMA chains, summed by the
    // drains) while three fit in 256 TMEM columns, so that two CTAs share the SM's 512
    static constexpr int kAcc = 3 * BN <= 256 ? 3 : 1;
    static constexpr int kNeed = kAcc * BN;
    static constexpr uint32_t kCols = kNeed <= 32 ? 32 : kNeed <= 64 ? 64 : kNeed <= 128 ? 128 : kNeed <= 256 ? 256 : 512;
    static constexpr size_t kSmem = 1024 + (size_t)kArena + 512;
};

struct SpecOut {
    int kw;               // window side (kw <= BN)
    float* G;             // [slices][kw][round_up(kw, 16)] partial D2 blocks
};

template <int BN>
__global__ void __launch_bounds__(256, 2)
k_tc_spec2(const __grid_constant__ CUtensorMap tmAhi, const __grid_constant__ CUtensorMap tmAlo,
           const __grid_constant__ CUtensorMap tmBhi, const __grid_constant__ CUtensorMap tmBlo,
           const __grid_constant__ CUtensorMap tmChi, const __grid_constant__ CUtensorMap tmClo,
           int M, int kb_per_split, int kb_total, int use_alo, const SpecOut so, int* err) {
    using CF = Cfg<BN>;
    using C2 = Cfg2<BN>;
    constexpr int S = C2::kStages;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + C2::kArena);
    uint64_t* empty = full + S;
    uint64_t* accum = empty + S;
    uint64_t* a2full = accum + 1;
    uint64_t* acc2 = a2full + 1;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc2 + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * kBM;
    const int kb0 = blockIdx.z * kb_per_split;
    const int nkb = m0 < M ? max(0, min(kb_per_split, kb_total - kb0)) : 0;

    auto stage_ptr = [&](int s, int which) -> uint8_t* {
        uint8_t* base = smem + s * CF::kStage;
        return which < 2 ? base + which * kABytes : base + 2 * kABytes + (which - 2) * CF::kBBytes;
    };
    const uint32_t bytes1 = (use_alo ? 2 : 1) * kABytes + 2 * CF::kBBytes;
    pdl_trigger();
    const int clip = blockIdx.x;  // clip of a batch: the image maps are 3-D
    auto issue1 = [&](int i) {
        const int s = i % S;
        mbar_arrive_expect_tx(&full[s], bytes1);
        const int kc = (kb0 + i) * kBK;
        tma_load_3d(&tmAhi, &full[s], stage_ptr(s, 0), kc, m0, clip);
        if (use_alo) tma_load_3d(&tmAlo, &full[s], stage_ptr(s, 1), kc, m0, clip);
        tma_load_2d(&tmBhi, &full[s], stage_ptr(s, 2), kc, 0);
        tma_load_2d(&tmBlo, &full[s], stage_ptr(s, 3), kc, 0);
    };

    // thread 0 initialises the barriers and issues the first ring's copies before the
    // CTA-wide barrier (they need no wait)
    int issued = 0;
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(accum, 1);
        mbar_init(a2full, 1);
        mbar_init(acc2, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        // B (the DFT table, constant) of the first stages before the previous kernel has
        // finished; A (the image it wrote) after the wait
        const int npre = min(nkb, S);
        for (int i = 0; i < npre; ++i) {
            mbar_arrive_expect_tx(&full[i], bytes1);
            tma_load_2d(&tmBhi, &full[i], stage_ptr(i, 2), (kb0 + i) * kBK, 0);
            tma_load_2d(&tmBlo, &full[i], stage_ptr(i, 3), (kb0 + i) * kBK, 0);
        }
        pdl_wait();
        for (int i = 0; i < npre; ++i) {
            tma_load_3d(&tmAhi, &full[i], stage_ptr(i, 0), (kb0 + i) * kBK, m0, clip);
            if (use_alo) tma_load_3d(&tmAlo, &full[i], stage_ptr(i, 1), (kb0 + i) * kBK, m0, clip);
        }
        issued = npre;
    }
    if (warp == 1) tmem_alloc(tmem_slot, C2::kCols);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    // phase-2 buffers overlay the ring once phase 1 is complete
    uint8_t* B2hi = smem;                 // [2 k-blocks][BN rows][128 B]
    uint8_t* B2lo = smem + 2 * C2::kB2;
    uint8_t* A2 = smem + 4 * C2::kB2;     // [k-block][hi, lo][128 rows][128 B]
    auto a2_ptr = [&](int kb, int lo) -> uint8_t* { return A2 + (kb * 2 + lo) * kABytes; };
    constexpr uint32_t idesc = idesc_bf16(kBM, BN);

    // ---------------- phase 1 ----------------
    bool ok = true;
    if (warp == 0 && lane == 0 && nkb > 0) {
        for (int i = issued; i < nkb; ++i) {
            if (!mbar_wait(&empty[i % S], ((i / S) - 1) & 1, err)) {
                ok = false;
                break;
            }
            issue1(i);
            ++issued;
        }
    } else if (warp == 1 && lane == 0 && nkb > 0) {
        for (int i = 0; i < nkb; ++i) {
            const int s = i % S;
            if (!mbar_wait(&full[s], (i / S) & 1, err)) {
                ok = false;
                break;
            }
            fence_after_sync();
            const uint64_t dAhi = smem_desc_sw128(smem_u32(stage_ptr(s, 0)));
            const uint64_t dAlo = smem_desc_sw128(smem_u32(stage_ptr(s, 1)));
            const uint64_t dBhi = smem_desc_sw128(smem_u32(stage_ptr(s, 2)));
            const uint64_t dBlo = smem_desc_sw128(smem_u32(stage_ptr(s, 3)));
            if (use_alo) slab_mmas<kBK / 16, C2::kAcc == 3, true>(tmem, BN, dAhi, dAlo, dBhi, dBlo, idesc, i == 0);
            else slab_mmas<kBK / 16, C2::kAcc == 3, false>(tmem, BN, dAhi, dAlo, dBhi, dBlo, idesc, i == 0);
            mma_commit(&empty[s]);
        }
        if (ok) mma_commit(accum);
    }
    __syncwarp();
    bool have = nkb > 0 && ok;
    if (nkb > 0) have = mbar_wait(accum, 0, err);
    have = __syncthreads_and(have);  // phase 1 finished (or failed) for the whole CTA
    fence_after_sync();

    // ---------------- phase 2 ----------------
    if (have) {
        // A2 (the ring is idle now)
        if (warp == 0 && lane == 0) {
            mbar_arrive_expect_tx(a2full, 4 * kABytes);
            for (int kb = 0; kb < 2; ++kb) {
                tma_load_2d(&tmChi, a2full, a2_ptr(kb, 0), m0 + kb * kBK, 0);
                tma_load_2d(&tmClo, a2full, a2_ptr(kb, 1), m0 + kb * kBK, 0);
            }
        }
        // drain D1 (sum of the product accumulators): thread = row y of the tile, warp group
        // grp = 16-column chunks grp, grp + 2, ...; write B2[c][y] as bf16 hi/lo in the
        // 128-byte-swizzled K-major layout
        const int yl = (warp & 3) * 32 + lane, grp = warp >> 2;
        const uint32_t kbo = (uint32_t)(yl >> 6) * C2::kB2;
        const uint32_t chunk = (uint32_t)((yl & 63) >> 3), e2 = (uint32_t)(yl & 7) * 2;
        const uint32_t trow = tmem + ((uint32_t)((warp & 3) * 32) << 16);
        const int nacc = C2::kAcc == 3 ? (use_alo ? 3 : 2) : 1;
        auto put = [&](uint32_t c2, float x) {
            const uint32_t off = kbo + c2 * 128u + (((chunk ^ (c2 & 7u)) << 4) | e2);
            const __nv_bfloat16 h = __float2bfloat16_rn(x);
            *reinterpret_cast<__nv_bfloat16*>(B2hi + off) = h;
            *reinterpret_cast<__nv_bfloat16*>(B2lo + off) = __float2bfloat16_rn(x - __bfloat162float(h));
        };
#pragma unroll 1
        for (int c = 16 * grp; c < BN; c += 32) {
            float v[16];
            tmem_ld16(trow + (uint32_t)c, v);
            for (int a = 1; a < nacc; ++a) {
                float q[16];
                tmem_ld16(trow + (uint32_t)(a * BN + c), q);
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] += q[j];
            }
#pragma unroll
            for (int j = 0; j < 16; ++j) put((uint32_t)(c + j), v[j]);
        }
        // generic-proxy stores -> visible to the tensor core (async proxy); TMEM reads done
        fence_proxy_async_smem();
        fence_before_sync();
    }
    __syncthreads();
    fence_after_sync();
    if (have && warp == 1 && lane == 0) {
        // D2: the three products at TMEM columns 0, BN, 2 BN (or one accumulator)
        if (mbar_wait(a2full, 0, err)) {
            fence_after_sync();
#pragma unroll
            for (int kb = 0; kb < 2; ++kb)
                slab_mmas<kBK / 16, C2::kAcc == 3, true>(
                    tmem, BN, smem_desc_sw128(smem_u32(a2_ptr(kb, 0))), smem_desc_sw128(smem_u32(a2_ptr(kb, 1))),
                    smem_desc_sw128(smem_u32(B2hi + kb * C2::kB2)), smem_desc_sw128(smem_u32(B2lo + kb * C2::kB2)),
                    idesc, kb == 0);
            mma_commit(acc2);
        }
    }
    __syncwarp();
    // ---- epilogue. Every thread waits for the phase-2 MMAs (they read the shared memory
    // that D2 is drained into); D2 row c1 = the lane-row of this warp.
    bool h2 = have;
    if (h2) h2 = mbar_wait(acc2, 0, err);
    h2 = __syncthreads_and(h2);
    fence_after_sync();
    const int kw = so.kw;
    const int kc = (kw + 15) / 16 * 16;               // drained columns (16-column chunks)
    const int kDP = kc + 4;                           // row pitch in floats (16-byte rows)
    float* Dsm = reinterpret_cast<float*>(smem);     // [kw][kDP]
    float* Gs = so.G + ((size_t)(clip * gridDim.y + blockIdx.y) * gridDim.z + blockIdx.z) * kw * kc;
    if (h2 && (warp & 3) * 32 < kw) {  // warp-uniform: rows c1 >= kw are not needed
        const int c1 = (warp & 3) * 32 + lane;
        const uint32_t trow = tmem + ((uint32_t)((warp & 3) * 32) << 16);
#pragma unroll 1
        for (int c = 16 * (warp >> 2); c < kc; c += 32) {
            float v[16];
            tmem_ld16(trow + (uint32_t)c, v);
            for (int q = 1; q < C2::kAcc; ++q) {
                float w[16];
                tmem_ld16(trow + (uint32_t)(q * BN + c), w);
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] += w[j];
            }
            if (c1 < kw) {
                float4* d4 = reinterpret_cast<float4*>(Dsm + c1 * kDP + c);
#pragma unroll
                for (int j = 0; j < 4; ++j) d4[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
            }
        }
    }
    __syncthreads();
    // D2 rows to the slice: a warp per row, a lane per 16-byte column group (kc / 4 <= 32)
    for (int row = warp; row < kw; row += 8) {
        if (lane < kc / 4) {
            const float4 v = h2 ? *reinterpret_cast<const float4*>(Dsm + row * kDP + 4 * lane)
                                : make_float4(0.f, 0.f, 0.f, 0.f);
            reinterpret_cast<float4*>(Gs + (size_t)row * kc)[lane] = v;
        }
    }
    // a producer that stopped early waits (bounded) for the loads it issued
    if (warp == 0 && lane == 0 && !ok) {
        for (int i = max(0, issued - S); i < issued; ++i) mbar_wait(&full[i % S], (i / S) & 1, nullptr);
    }
    fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        fence_after_sync();
        tmem_dealloc(tmem, C2::kCols);
    }
}

// ---------------------------------------------------------------------------
// Persistent expansion GEMM: D = scale * A B^T over an n x n output
// ---------------------------------------------------------------------------
// A = [Re T | -Im T] rows (M x K, K = the window's ldk <= 64 KB), B = basis^T rows
// (N x K). Each CTA owns a contiguous range of 128 x BN output tiles (row-major
// tile order, so consecutive tiles share their A rows). Warp roles:
//   warp 4 (one thread)  TMA producer: the CTA's A rows (all K, kept resident while
//                        the tile row lasts) and the B slabs of every tile into an
//                        S-slot ring;
//   warp 5 (one thread)  MMA issuer into two TMEM accumulators (tile i in buffer i & 1),
//                        so the epilogue of one tile overlaps the MMAs of the next;
//   warps 0-3            epilogue: TMEM lanes 32w.. (tile rows), 32 columns at a time,
//                        scaled, staged in shared memory (128-byte swizzle) and written
//                        by TMA tensor stores (or plain stores when the output pitch is
//                        not 16-byte aligned); EPI_VEL also folds each tile's max |D|
//                        into its clip's word (ep.vbits), and the last CTA converts them.
// For a batch of clips the tiles run clip by clip (A and C are 3-D maps over the clips;
// B, the table, is shared).
template <int BN, int KB>
struct CfgX {
    static constexpr uint32_t kA = KB * 2 * kABytes;       // A hi/lo, all K
    static constexpr uint32_t kSlab = BN * kBK * 2;        // one 64-wide K slab of B (hi or lo)
    static constexpr uint32_t kSlot = 2 * kSlab;
    static constexpr uint32_t kStaging = 4 * 2 * 4096;     // 4 warps x 2 buffers x (32 rows x 128 B)
    static constexpr uint32_t kFixed = 1024 + kA + kStaging + 256;
    static constexpr int kFit = (int)((232448u - kFixed) / kSlot);
    static constexpr int kS = kFit > 8 ? 8 : kFit;
    static_assert(kFit >= 2, "expansion tile does not fit");
    // Accumulators per TMEM buffer: the three compensation products go to separate
    // accumulators when two buffers of three fit in TMEM, so that three independent MMA
    // chains interleave (a single accumulate chain of narrow MMAs is latency-bound);
    // they are summed in the epilogue.
    static constexpr int kAcc = 2 * 3 * BN <= 512 ? 3 : 1;
    static constexpr int kBuf = kAcc * BN;                 // TMEM columns of one buffer
    static constexpr uint32_t kCols = 2 * kBuf <= 32 ? 32 : 2 * kBuf <= 64 ? 64 : 2 * kBuf <= 128 ? 128
                                    : 2 * kBuf <= 256 ? 256 : 512;
    static constexpr size_t kSmem = kFixed + (size_t)kS * kSlot;
};

template <int BN, int KB, int EPI>
__global__ void __launch_bounds__(192, 1)
k_tc_expand(const __grid_constant__ CUtensorMap tmAhi, const __grid_constant__ CUtensorMap tmAlo,
            const __grid_constant__ CUtensorMap tmBhi, const __grid_constant__ CUtensorMap tmBlo,
            const __grid_constant__ CUtensorMap tmC, int use_tma_store, int M, int N, int ksteps_last,
            int tiles_m, int tiles_n, int tiles, const EpiArgs ep, int* err) {
    using CX = CfgX<BN, KB>;
    constexpr int S = CX::kS;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* sA = smem;
    uint8_t* sB = smem + CX::kA;
    uint8_t* sC = sB + S * CX::kSlot;
    uint64_t* a_full = reinterpret_cast<uint64_t*>(sC + CX::kStaging);
    uint64_t* a_empty = a_full + 1;
    uint64_t* b_full = a_empty + 1;
    uint64_t* b_empty = b_full + S;
    uint64_t* t_full = b_empty + S;
    uint64_t* t_empty = t_full + 2;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(t_empty + 2);
    volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t0 = (int)(((long long)blockIdx.x * tiles) / gridDim.x);
    const int t1 = (int)(((long long)(blockIdx.x + 1) * tiles) / gridDim.x);
    const bool producer = threadIdx.x == 128;  // warp 4, lane 0

    // Producer state. The producer initialises the barriers and issues the copies that
    // need no wait (the first A rows and up to S slabs) before the CTA-wide barrier.
    int p_t = t0, p_kb = 0, p_slab = 0, p_aload = 0, p_prev_m = -1;
    bool p_ok = true;
    auto produce = [&](bool prologue) {
        while (p_t < t1 && p_ok) {
            const int mt = p_t / tiles_n, nt = p_t - mt * tiles_n;
            if (p_kb == 0 && mt != p_prev_m) {
                if (p_aload > 0) {
                    if (prologue) return;
                    if (!mbar_wait_ab(a_empty, (p_aload - 1) & 1, err, abort)) {
                        p_ok = false;
                        return;
                    }
                }
                mbar_arrive_expect_tx(a_full, CX::kA);
                const int clip = mt / tiles_m, my = (mt - clip * tiles_m) * kBM;
                for (int kb = 0; kb < KB; ++kb) {
                    tma_load_3d(&tmAhi, a_full, sA + kb * 2 * kABytes, kb * kBK, my, clip);
                    tma_load_3d(&tmAlo, a_full, sA + kb * 2 * kABytes + kABytes, kb * kBK, my, clip);
                }
                ++p_aload;
                p_prev_m = mt;
            }
            const int sl = p_slab % S;
            if (p_slab >= S) {
                if (prologue) return;
                if (!mbar_wait_ab(&b_empty[sl], ((p_slab / S) - 1) & 1, err, abort)) {
                    p_ok = false;
                    return;
                }
            }
            mbar_arrive_expect_tx(&b_full[sl], CX::kSlot);
            tma_load_2d(&tmBhi, &b_full[sl], sB + sl * CX::kSlot, p_kb * kBK, nt * BN);
            tma_load_2d(&tmBlo, &b_full[sl], sB + sl * CX::kSlot + CX::kSlab, p_kb * kBK, nt * BN);
            ++p_slab;
            if (++p_kb == KB) {
                p_kb = 0;
                ++p_t;
            }
        }
    };

    pdl_trigger();
    if (producer) {
        mbar_init(a_full, 1);
        mbar_init(a_empty, 1);
        for (int i = 0; i < S; ++i) {
            mbar_init(&b_full[i], 1);
            mbar_init(&b_empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&t_full[i], 1);
            mbar_init(&t_empty[i], 4);  // one arrival per epilogue warp
        }
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        pdl_wait();  // the A operand is the previous kernel's output; outputs follow from it
        produce(true);
    }
    if (warp == 5) tmem_alloc(tmem_slot, CX::kCols);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;
    int mxi = 0;  // max |D| as a float bit pattern (EPI_VEL)

    if (warp == 4) {
        if (lane == 0) {
            produce(false);
            if (!p_ok || *abort) {  // wait (bounded) for the copies still in flight before the CTA exits
                if (p_aload > 0) mbar_wait(a_full, (p_aload - 1) & 1, nullptr);
                for (int i = max(0, p_slab - S); i < p_slab; ++i) mbar_wait(&b_full[i % S], (i / S) & 1, nullptr);
            }
        }
    } else if (warp == 5) {
        if (lane == 0) {
            constexpr uint32_t idesc = idesc_bf16(kBM, BN);
            int slab = 0, aload = 0, prev_m = -1, ti = 0;
            bool ok = true, pending = false;
            for (int t = t0; t < t1 && ok; ++t, ++ti) {
                const int mt = t / tiles_n;
                if (mt != prev_m) {
                    if (!mbar_wait_ab(a_full, aload & 1, err, abort)) {
                        ok = false;
                        break;
                    }
                    ++aload;
                    prev_m = mt;
                }
                const int buf = ti & 1;
                if (ti >= 2 && !mbar_wait_ab(&t_empty[buf], ((ti >> 1) - 1) & 1, err, abort)) {
                    ok = false;
                    break;
                }
                fence_after_sync();
                const uint32_t d = tmem + (uint32_t)(buf * CX::kBuf);
                for (int kb = 0; kb < KB; ++kb, ++slab) {
                    const int sl = slab % S;
                    if (!mbar_wait_ab(&b_full[sl], (slab / S) & 1, err, abort)) {
                        ok = false;
                        break;
                    }
                    fence_after_sync();
                    const int ksteps = kb == KB - 1 ? ksteps_last : kBK / 16;
                    const uint64_t dAhi = smem_desc_sw128(smem_u32(sA + kb * 2 * kABytes));
                    const uint64_t dAlo = smem_desc_sw128(smem_u32(sA + kb * 2 * kABytes + kABytes));
                    const uint64_t dBhi = smem_desc_sw128(smem_u32(sB + sl * CX::kSlot));
                    const uint64_t dBlo = smem_desc_sw128(smem_u32(sB + sl * CX::kSlot + CX::kSlab));
                    if (ksteps == kBK / 16)
                        slab_mmas<kBK / 16, CX::kAcc == 3, true>(d, BN, dAhi, dAlo, dBhi, dBlo, idesc, kb == 0);
                    else
                        slab_mmas_rt<CX::kAcc == 3>(ksteps, true, d, BN, dAhi, dAlo, dBhi, dBlo, idesc, kb == 0);
                    pending = true;
                    mma_commit(&b_empty[sl]);
                }
                if (!ok) break;
                mma_commit(&t_full[buf]);
                pending = false;
                if (t + 1 >= t1 || (t + 1) / tiles_n != mt) mma_commit(a_empty);
            }
            if (!ok && pending) {  // MMAs of an unfinished tile: let them complete before TMEM is freed
                uint64_t* b = &t_full[ti & 1];
                mma_commit(b);
                mbar_wait(b, (ti >> 1) & 1, nullptr);
            }
        }
    } else {
        // epilogue warps 0-3
        int ti = 0, chunk = 0;
        const float scale = ep.scale;
        for (int t = t0; t < t1; ++t, ++ti) {
            const int mg = t / tiles_n, nt = t - mg * tiles_n;   // global row tile: clip * tiles_m + mt
            const int clip = mg / tiles_m, mt = mg - clip * tiles_m;
            const int buf = ti & 1;
            bool h = mbar_wait_ab(&t_full[buf], (ti >> 1) & 1, err, abort);
            h = __all_sync(0xffffffffu, h);
            if (!h) break;
            fence_after_sync();
            const int row0 = mt * kBM + warp * 32;
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(buf * CX::kBuf);
            uint32_t r[BN];
            if constexpr (BN == 128) tmem_ld128(taddr, r);
            else tmem_ld64(taddr, r);
            if constexpr (CX::kAcc == 3) {  // (hi hi + hi lo) + lo hi
#pragma unroll
                for (int a = 1; a < 3; ++a) {
                    uint32_t q[BN];
                    if constexpr (BN == 128) tmem_ld128(taddr + (uint32_t)(a * BN), q);
                    else tmem_ld64(taddr + (uint32_t)(a * BN), q);
#pragma unroll
                    for (int j = 0; j < BN; ++j) r[j] = __float_as_uint(__uint_as_float(r[j]) + __uint_as_float(q[j]));
                }
            }
            // the accumulator is in registers: hand the TMEM buffer back to the MMA thread
            fence_before_sync();
            __syncwarp();
            if (lane == 0) mbar_arrive(&t_empty[buf]);
            const int row = row0 + lane;
#pragma unroll
            for (int c = 0; c < BN; c += 32, ++chunk) {
                float v[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[c + j]) * scale;
                const int col0 = nt * BN + c;
                if (EPI == EPI_VEL && row < M) {
                    // max |V| on the bit patterns: for non-negative floats the integer order is
                    // the float order, and a NaN (or inf) pattern exceeds every finite one, so
                    // a non-finite value survives into the CTA's partial (fmaxf would drop a NaN)
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        if (col0 + j < N) mxi = max(mxi, __float_as_int(fabsf(v[j])));
                }
                if (use_tma_store) {
                    uint8_t* stg = sC + (warp * 2 + (chunk & 1)) * 4096;
                    if (lane == 0) bulk_wait_read<1>();  // this buffer's previous store has been read
                    __syncwarp();
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        *reinterpret_cast<float4*>(stg + lane * 128 + ((j ^ (lane & 7)) << 4)) =
                            make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                    fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) {  // boxes entirely outside are not issued; every chunk commits a
                                      // (possibly empty) group, so the wait above always covers the
                                      // store that last read this buffer
                        if (row0 < M && col0 < N) tma_store_3d(&tmC, stg, col0, row0, clip);
                        bulk_commit();
                    }
                } else if (row < M) {
                    float* dst = ep.C + clip * ep.split_stride + (size_t)row * ep.ldc + col0;
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        if (col0 + j < N) dst[j] = v[j];
                }
            }
            if (EPI == EPI_VEL) {
                // the tile's max |V| into its clip's word (integer max of the bit patterns:
                // exact and order-independent)
                for (int o = 16; o > 0; o >>= 1) mxi = max(mxi, __shfl_down_sync(0xffffffffu, mxi, o));
                if (lane == 0) atomicMax(ep.vbits + clip, (unsigned)mxi);
                mxi = 0;
            }
        }
        if (use_tma_store && lane == 0) bulk_wait_all();
        if (EPI == EPI_VEL) __threadfence();  // the atomics above before this CTA's arrival
    }
    __syncwarp();
    fence_before_sync();
    __syncthreads();
    if (warp == 5) {
        fence_after_sync();
        tmem_dealloc(tmem, CX::kCols);
    }
    if (EPI == EPI_VEL) {
        // the last CTA to finish turns every clip's word into max |V| (FP64), flags a
        // non-finite value (an inf or NaN pattern is >= 0x7f800000) and clears the words
        __shared__ bool s_last;
        if (threadIdx.x == 0) {
            __threadfence();
            s_last = atomicAdd(ep.counter, 1u) == gridDim.x - 1u;
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            for (int c = threadIdx.x; c < ep.nclips; c += blockDim.x) {
                const unsigned b = atomicExch(ep.vbits + c, 0u);
                ep.vmax[c] = (double)__uint_as_float(b);
                if (b >= 0x7f800000u && ep.status) *ep.status = DEVEL_ENAN;
            }
            if (threadIdx.x == 0) *ep.counter = 0u;
        }
    }
}

// ---------------------------------------------------------------------------
// Sum of the reduction's slices and the complex spectrum. A lane owns one position
// (j1, j2) in [0, r]^2 of the folded block (block = 32 positions x kSumWarps warps; warp w
// adds slices w, w + kSumWarps, ... with up to four slices' loads issued before the adds,
// so 128 slices take one round of loads; then the warps' sums are added in warp order)
// and sums its four products over the slices:
//   CC = D2[j1][j2], CS = D2[j1][r + j2], SC = D2[r + j1][j2], SS = D2[r + j1][r + j2]
// (a sine at |frequency| 0 is absent). With the signs t1, t2 of (u1, u2) = (t1 j1, t2 j2),
//   out(u1, u2) = scale [(CC - t1 t2 SS) - i (t2 CS + t1 SC)],
// written for every sign pair (each sign flip taken only for j > 0).
// ---------------------------------------------------------------------------
constexpr int kSumWarps = 32;
__global__ void __launch_bounds__(32 * kSumWarps)
k_spec_sum(const float* __restrict__ G, int slices, int kw, int kc, float scale, float2* __restrict__ out) {
    __shared__ float4 part[kSumWarps][32];
    pdl_trigger();
    pdl_wait();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int r = (kw - 1) / 2, np = (r + 1) * (r + 1);
    const int p = blockIdx.x * 32 + lane;
    G += (size_t)blockIdx.y * slices * kw * kc;  // clip blockIdx.y of a batch
    out += (size_t)blockIdx.y * kw * kw;
    const int j1 = p / (r + 1), j2 = p - j1 * (r + 1);
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);  // CC, CS, SC, SS
    if (p < np) {
        const size_t E = (size_t)kw * kc;
        // offsets of the four products (a missing sine reads the cosine entry, weight 0)
        const size_t o_cc = (size_t)j1 * kc + j2;
        const size_t o_cs = j2 > 0 ? (size_t)j1 * kc + r + j2 : o_cc;
        const size_t o_sc = j1 > 0 ? (size_t)(r + j1) * kc + j2 : o_cc;
        const size_t o_ss = (j1 > 0 && j2 > 0) ? (size_t)(r + j1) * kc + r + j2 : o_cc;
        int sl = w;
        for (; sl + 3 * kSumWarps < slices; sl += 4 * kSumWarps) {
            float4 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const float* g = G + (size_t)(sl + u * kSumWarps) * E;
                v[u] = make_float4(__ldcg(g + o_cc), __ldcg(g + o_cs), __ldcg(g + o_sc), __ldcg(g + o_ss));
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                acc.x += v[u].x;
                acc.y += v[u].y;
                acc.z += v[u].z;
                acc.w += v[u].w;
            }
        }
        for (; sl < slices; sl += kSumWarps) {
            const float* g = G + (size_t)sl * E;
            acc.x += __ldcg(g + o_cc);
            acc.y += __ldcg(g + o_cs);
            acc.z += __ldcg(g + o_sc);
            acc.w += __ldcg(g + o_ss);
        }
    }
    part[w][lane] = acc;
    __syncthreads();
    if (w != 0 || p >= np) return;
    float4 t = part[0][lane];
    for (int i = 1; i < kSumWarps; ++i) {
        t.x += part[i][lane].x;
        t.y += part[i][lane].y;
        t.z += part[i][lane].z;
        t.w += part[i][lane].w;
    }
    const float cc = t.x, cs = j2 > 0 ? t.y : 0.f, sc = j1 > 0 ? t.z : 0.f, ss = (j1 > 0 && j2 > 0) ? t.w : 0.f;
    for (int q = 0; q < 4; ++q) {
        const int t1 = (q & 2) ? -1 : 1, t2 = (q & 1) ? -1 : 1;
        if ((t1 < 0 && j1 == 0) || (t2 < 0 && j2 == 0)) continue;
        const float f1 = (float)t1, f2 = (float)t2;
        out[(r + t1 * j1) * kw + (r + t2 * j2)] =
            make_float2((cc - f1 * f2 * ss) * scale, -(f2 * cs + f1 * sc) * scale);
    }
}

// ---------------------------------------------------------------------------
// Self-test of the bounded waits: one thread waits on an mbarrier that nothing
// arrives on; the wait gives up after its time limit and sets *err.
// ---------------------------------------------------------------------------
__global__ void k_wait_selftest(int* err) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_wait(&bar, 0, err);
}

// ---------------------------------------------------------------------------
// fp32 -> bf16 hi/lo splits
// ---------------------------------------------------------------------------
// One block row per image row (blockIdx.y), threads along the columns.
__global__ void k_split_rows(const float* __restrict__ X, int rows, int cols, int ldx, int ldo,
                             __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo) {
    const int r = blockIdx.y;
    const float* xr = X + (size_t)r * ldx;
    __nv_bfloat16* hr = hi + (size_t)r * ldo;
    __nv_bfloat16* lr = lo ? lo + (size_t)r * ldo : nullptr;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ldo; c += gridDim.x * blockDim.x) {
        const float x = c < cols ? xr[c] : 0.f;
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        hr[c] = h;
        if (lr) lr[c] = __float2bfloat16_rn(x - __bfloat162float(h));
    }
}

// 0/1 mask row -> bf16 row of pitch ldo, four pixels per thread (clip blockIdx.z of a
// batch: masks n^2 apart, outputs n ldo apart).
__global__ void k_mask_bf16(const unsigned char* __restrict__ M, int n, int ldo, __nv_bfloat16* __restrict__ hi) {
    const int r = blockIdx.y;
    const unsigned char* mr = M + (size_t)blockIdx.z * n * n + (size_t)r * n;
    __nv_bfloat16* hr = hi + (size_t)blockIdx.z * n * ldo + (size_t)r * ldo;
    const __nv_bfloat16 one = __float2bfloat16_rn(1.f), zero = __float2bfloat16_rn(0.f);
    const bool vec = (n & 3) == 0 && (ldo & 3) == 0;  // 4-byte mask loads, 8-byte bf16 stores
    for (int c = (blockIdx.x * blockDim.x + threadIdx.x) * 4; c < ldo; c += gridDim.x * blockDim.x * 4) {
        if (vec && c + 4 <= n) {
            const uchar4 m4 = *reinterpret_cast<const uchar4*>(mr + c);
            const unsigned short h1 = 0x3F80u;  // bf16 1.0
            const uint2 o = make_uint2((m4.x ? h1 : 0u) | ((m4.y ? h1 : 0u) << 16), (m4.z ? h1 : 0u) | ((m4.w ? h1 : 0u) << 16));
            *reinterpret_cast<uint2*>(hr + c) = o;
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (c + j < ldo) hr[c + j] = (c + j < n && mr[c + j]) ? one : zero;
        }
    }
}

template <int BN>
cudaError_t set_attr_bn() {
    return cudaFuncSetAttribute(k_tc_gemm<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Cfg<BN>::kSmem);
}

template <int BN>
int launch_gemm_bn(const Operands& op, int M, int N, int kb_total, int ksteps_last, int B, const EpiArgs& ep,
                   int* err, cudaStream_t s) {
    using CF = Cfg<BN>;
    dim3 grid((N + BN - 1) / BN, (M + kBM - 1) / kBM, B);
    cudaError_t e = launch_pdl(k_tc_gemm<BN>, grid, dim3(128), CF::kSmem, s, *op.Ahi, *op.Alo, *op.Bhi, *op.Blo, M, N,
                               kb_total, ksteps_last, op.use_alo, ep, err);
    if (e != cudaSuccess) return cuda_error(e, "k_tc_gemm");
    return DEVEL_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// 2-D bf16 tensor map over a row-major [rows][cols] array with row pitch ld
// elements; box = 64 columns x box_rows rows, 128-byte swizzle, zero fill.
int make_map(CUtensorMap* tm, const void* base, int rows, int cols, int ld, int box_rows) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return set_error(DEVEL_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    if ((reinterpret_cast<uintptr_t>(base) & 15u) || ((size_t)ld * 2) % 16 != 0 || box_rows > 256)
        return set_error(DEVEL_EINVAL, "tensor map: misaligned base/pitch or box too tall");
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(DEVEL_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return DEVEL_OK;
}

// 3-D bf16 tensor map over depth arrays [rows][cols] (row pitch ld elements), array d at
// base + d * dld elements: one array per clip of a batch; box = 64 columns x box_rows rows
// x 1 array, 128-byte swizzle, zero fill (rows past `rows` of an array read as zeros).
int make_map3(CUtensorMap* tm, const void* base, int depth, int rows, int cols, int ld, size_t dld, int box_rows) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return set_error(DEVEL_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    if ((reinterpret_cast<uintptr_t>(base) & 15u) || ((size_t)ld * 2) % 16 != 0 || (dld * 2) % 16 != 0 ||
        box_rows > 256 || depth < 1)
        return set_error(DEVEL_EINVAL, "tensor map: misaligned base/pitch or box too tall");
    cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)depth};
    cuuint64_t strides[2] = {(cuuint64_t)ld * 2, (cuuint64_t)dld * 2};
    cuuint32_t box[3] = {(cuuint32_t)kBK, (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(DEVEL_ECUDA, "cuTensorMapEncodeTiled (3-D) failed (%d)", (int)r);
    return DEVEL_OK;
}

// 3-D bf16 tensor map without swizzle: dims (d0 innermost, d1, d2), byte strides s1, s2 of
// dims 1 and 2, box (b0, b1, b2), zero fill (the raw boxes a kernel rearranges itself).
int make_map_plain3(CUtensorMap* tm, const void* base, uint64_t d0, uint64_t d1, uint64_t d2, uint64_t s1,
                    uint64_t s2, uint32_t b0, uint32_t b1, uint32_t b2) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return set_error(DEVEL_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    if ((reinterpret_cast<uintptr_t>(base) & 15u) || (s1 % 16) || (s2 % 16) || ((uint64_t)b0 * 2) % 16 ||
        b0 > 256 || b1 > 256 || b2 > 256)
        return set_error(DEVEL_EINVAL, "tensor map: misaligned base / strides or box");
    cuuint64_t dims[3] = {(cuuint64_t)d0, (cuuint64_t)d1, (cuuint64_t)d2};
    cuuint64_t strides[2] = {(cuuint64_t)s1, (cuuint64_t)s2};
    cuuint32_t box[3] = {b0, b1, b2};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(DEVEL_ECUDA, "cuTensorMapEncodeTiled (plain) failed (%d)", (int)r);
    return DEVEL_OK;
}

// fp32 output map over depth arrays [rows][cols] (pitch ld elements, a multiple of 4;
// array d at base + d * dld elements): boxes of 32 columns x 32 rows x 1 array, 128-byte
// swizzle (the epilogue's staging layout).
static int make_map_out(CUtensorMap* tm, const float* base, int depth, int rows, int cols, int ld, size_t dld) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return set_error(DEVEL_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)depth};
    cuuint64_t strides[2] = {(cuuint64_t)ld * 4, (cuuint64_t)dld * 4};
    cuuint32_t box[3] = {32, 32, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(DEVEL_ECUDA, "cuTensorMapEncodeTiled (output) failed (%d)", (int)r);
    return DEVEL_OK;
}

static int sm_count() {
    int dev = 0, c = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&c, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess)
        return 148;
    return c > 0 ? c : 148;
}

template <int BN, int KB, int EPI>
static int launch_expand_cfg(const Operands& op, int M, int N, int ksteps_last, int B, const EpiArgs& ep, int* err,
                             cudaStream_t s) {
    CUtensorMap tmC;
    const bool tma_store = (ep.ldc % 4) == 0 && (reinterpret_cast<uintptr_t>(ep.C) & 15u) == 0 &&
                           (ep.split_stride % 4) == 0;
    if (tma_store) {
        int rc = make_map_out(&tmC, ep.C, B, M, N, ep.ldc, B > 1 ? ep.split_stride : (size_t)M * ep.ldc);
        if (rc) return rc;
    } else {
        std::memset(&tmC, 0, sizeof(tmC));
    }
    const int tiles_m = (M + kBM - 1) / kBM, tiles_n = (N + BN - 1) / BN;
    const int tiles = B * tiles_m * tiles_n;
    const int grid = std::min(tiles, sm_count());
    EpiArgs e2 = ep;
    e2.nclips = B;
    cudaError_t e = launch_pdl(k_tc_expand<BN, KB, EPI>, dim3(grid), dim3(192), CfgX<BN, KB>::kSmem, s, *op.Ahi,
                               *op.Alo, *op.Bhi, *op.Blo, tmC, tma_store ? 1 : 0, M, N, ksteps_last, tiles_m, tiles_n,
                               tiles, e2, err);
    if (e != cudaSuccess) return cuda_error(e, "k_tc_expand");
    return DEVEL_OK;
}

int expand_grid(int M, int N, int BN) {
    const int tiles = ((M + kBM - 1) / kBM) * ((N + BN - 1) / BN);
    return std::min(tiles, sm_count());
}

int launch_expand(const Operands& op, int BN, int epi, int M, int N, int K, int B, const EpiArgs& ep, int* err,
                  cudaStream_t s) {
    const int KB = (K + kBK - 1) / kBK;
    if (K % 16 != 0 || KB < 1 || KB > 4 || (BN != 64 && BN != 128))
        return set_error(DEVEL_EINVAL, "tc expand: contraction length %d / tile width %d unsupported", K, BN);
    const int ksteps_last = (K - (KB - 1) * kBK) / 16;
    prof_begin(PK_TC_EXPAND, s);
    int rc = DEVEL_OK;
#define DEVEL_X_CASE(bn, kb)                                                                              \
    if (BN == bn && KB == kb)                                                                             \
        rc = epi == EPI_VEL ? launch_expand_cfg<bn, kb, EPI_VEL>(op, M, N, ksteps_last, B, ep, err, s)    \
                            : launch_expand_cfg<bn, kb, EPI_STORE>(op, M, N, ksteps_last, B, ep, err, s);
    DEVEL_X_CASE(64, 1) DEVEL_X_CASE(64, 2) DEVEL_X_CASE(64, 3) DEVEL_X_CASE(64, 4)
    DEVEL_X_CASE(128, 1) DEVEL_X_CASE(128, 2) DEVEL_X_CASE(128, 3) DEVEL_X_CASE(128, 4)
#undef DEVEL_X_CASE
    prof_end(PK_TC_EXPAND, s);
    return rc;
}

template <int BN, int KB>
static cudaError_t set_attr_expand() {
    cudaError_t e = cudaFuncSetAttribute(k_tc_expand<BN, KB, EPI_STORE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)CfgX<BN, KB>::kSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_tc_expand<BN, KB, EPI_VEL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)CfgX<BN, KB>::kSmem);
    return e;
}

int launch_gemm_split(const Operands& op, int BN, int prof_kind, int M, int N, int K, int B, const EpiArgs& ep,
                      int* err, cudaStream_t s) {
    if (K % 16 != 0) return set_error(DEVEL_EINVAL, "tc gemm: K=%d not a multiple of 16", K);
    const int kb_total = (K + kBK - 1) / kBK;
    const int ksteps_last = (K - (kb_total - 1) * kBK) / 16;
    prof_begin(prof_kind, s);
    int rc;
    switch (BN) {
#define DEVEL_TC_CASE(bn)                                                                            \
    case bn:                                                                                         \
        rc = launch_gemm_bn<bn>(op, M, N, kb_total, ksteps_last, B, ep, err, s);                      \
        break;
        DEVEL_TC_CASE(16) DEVEL_TC_CASE(32) DEVEL_TC_CASE(48) DEVEL_TC_CASE(64) DEVEL_TC_CASE(80)
        DEVEL_TC_CASE(96) DEVEL_TC_CASE(112) DEVEL_TC_CASE(128) DEVEL_TC_CASE(144) DEVEL_TC_CASE(160)
        DEVEL_TC_CASE(176) DEVEL_TC_CASE(192) DEVEL_TC_CASE(208) DEVEL_TC_CASE(224) DEVEL_TC_CASE(240)
        DEVEL_TC_CASE(256)
#undef DEVEL_TC_CASE
        default:
            rc = set_error(DEVEL_EINVAL, "tc gemm: unsupported tile width %d", BN);
    }
    prof_end(prof_kind, s);
    return rc;
}

template <int BN>
int launch_spec2_bn(const Operands& op, const CUtensorMap* Chi, const CUtensorMap* Clo, int M, int kb_per_split,
                    int kb_total, int splits, int B, SpecOut so, int* err, cudaStream_t s) {
    dim3 grid(B, (M + kBM - 1) / kBM, splits);
    cudaError_t e = launch_pdl(k_tc_spec2<BN>, grid, dim3(256), Cfg2<BN>::kSmem, s, *op.Ahi, *op.Alo, *op.Bhi,
                               *op.Blo, *Chi, *Clo, M, kb_per_split, kb_total, op.use_alo, so, err);
    if (e != cudaSuccess) return cuda_error(e, "k_tc_spec2");
    return DEVEL_OK;
}

template <int BN>
cudaError_t set_attr_spec2() {
    return cudaFuncSetAttribute(k_tc_spec2<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg2<BN>::kSmem);
}

int spectrum2_slices(int M, int K, int split) { return ((M + kBM - 1) / kBM) * ((K + split - 1) / split); }

int launch_spectrum2(const Operands& op, const CUtensorMap* Chi, const CUtensorMap* Clo, int BN, int kw, int n,
                     int M, int K, int split, int B, float* G, float2* out, int* err, cudaStream_t s) {
    if (K % kBK != 0 || split % kBK != 0 || split < kBK)
        return set_error(DEVEL_EINVAL, "tc spectrum: K=%d / split %d not multiples of %d", K, split, kBK);
    if (kw > BN) return set_error(DEVEL_EINVAL, "tc spectrum: window %d wider than the table's %d rows", kw, BN);
    const int kb_total = K / kBK, kb_per_split = split / kBK;
    const int splits = (kb_total + kb_per_split - 1) / kb_per_split;
    SpecOut so;
    so.kw = kw;
    so.G = G;
    prof_begin(PK_TC_SPECTRUM, s);
    int rc;
    switch (BN) {
#define DEVEL_SPEC2_CASE(bn)                                                                               \
    case bn:                                                                                               \
        rc = launch_spec2_bn<bn>(op, Chi, Clo, M, kb_per_split, kb_total, splits, B, so, err, s);          \
        break;
        DEVEL_SPEC2_CASE(16) DEVEL_SPEC2_CASE(32) DEVEL_SPEC2_CASE(48) DEVEL_SPEC2_CASE(64) DEVEL_SPEC2_CASE(80)
        DEVEL_SPEC2_CASE(96) DEVEL_SPEC2_CASE(112) DEVEL_SPEC2_CASE(128)
#undef DEVEL_SPEC2_CASE
        default:
            rc = set_error(DEVEL_EINVAL, "tc spectrum: unsupported window width %d", BN);
    }
    prof_end(PK_TC_SPECTRUM, s);
    if (rc) return rc;
    const int slices = spectrum2_slices(M, K, split), r = (kw - 1) / 2, np = (r + 1) * (r + 1);
    prof_begin(PK_SPECTRUM_REDUCE, s);
    cudaError_t e = launch_pdl(k_spec_sum, dim3((np + 31) / 32, B), dim3(32 * kSumWarps), 0, s, (const float*)G, slices,
                               kw, (kw + 15) / 16 * 16, 1.0f / ((float)n * (float)n), out);
    prof_end(PK_SPECTRUM_REDUCE, s);
    if (e != cudaSuccess) return cuda_error(e, "k_spec_sum");
    return DEVEL_OK;
}

int launch_wait_selftest(int* err, cudaStream_t s) {
    k_wait_selftest<<<1, 32, 0, s>>>(err);
    DEVEL_LAUNCH_CHECK("k_wait_selftest");
    return DEVEL_OK;
}

// Shared-memory opt-in of every kernel instantiation (call once per device,
// outside stream capture).
int init_attrs() {
    cudaError_t e = cudaSuccess;
#define DEVEL_TC_ATTR(bn) if (e == cudaSuccess) e = set_attr_bn<bn>();
    DEVEL_TC_ATTR(16) DEVEL_TC_ATTR(32) DEVEL_TC_ATTR(48) DEVEL_TC_ATTR(64) DEVEL_TC_ATTR(80) DEVEL_TC_ATTR(96)
    DEVEL_TC_ATTR(112) DEVEL_TC_ATTR(128) DEVEL_TC_ATTR(144) DEVEL_TC_ATTR(160) DEVEL_TC_ATTR(176)
    DEVEL_TC_ATTR(192) DEVEL_TC_ATTR(208) DEVEL_TC_ATTR(224) DEVEL_TC_ATTR(240) DEVEL_TC_ATTR(256)
#undef DEVEL_TC_ATTR
#define DEVEL_SPEC2_ATTR(bn) if (e == cudaSuccess) e = set_attr_spec2<bn>();
    DEVEL_SPEC2_ATTR(16) DEVEL_SPEC2_ATTR(32) DEVEL_SPEC2_ATTR(48) DEVEL_SPEC2_ATTR(64) DEVEL_SPEC2_ATTR(80)
    DEVEL_SPEC2_ATTR(96) DEVEL_SPEC2_ATTR(112) DEVEL_SPEC2_ATTR(128)
#undef DEVEL_SPEC2_ATTR
    if (e == cudaSuccess) e = set_attr_expand<64, 1>();
    if (e == cudaSuccess) e = set_attr_expand<64, 2>();
    if (e == cudaSuccess) e = set_attr_expand<64, 3>();
    if (e == cudaSuccess) e = set_attr_expand<64, 4>();
    if (e == cudaSuccess) e = set_attr_expand<128, 1>();
    if (e == cudaSuccess) e = set_attr_expand<128, 2>();
    if (e == cudaSuccess) e = set_attr_expand<128, 3>();
    if (e == cudaSuccess) e = set_attr_expand<128, 4>();
    if (e != cudaSuccess) return cuda_error(e, "tc::init_attrs");
    return DEVEL_OK;
}

int launch_split(const float* X, int rows, int cols, int ldx, int ldo, __nv_bfloat16* hi, __nv_bfloat16* lo,
                 cudaStream_t s) {
    prof_begin(PK_TC_SPLIT, s);
    k_split_rows<<<dim3((ldo + 255) / 256, rows), 256, 0, s>>>(X, rows, cols, ldx, ldo, hi, lo);
    prof_end(PK_TC_SPLIT, s);
    DEVEL_LAUNCH_CHECK("k_split_rows");
    return DEVEL_OK;
}

int launch_mask_bf16(const unsigned char* M, int n, int ldo, __nv_bfloat16* hi, cudaStream_t s, int B) {
    prof_begin(PK_TC_SPLIT, s);
    k_mask_bf16<<<dim3((ldo + 1023) / 1024, n, B), 256, 0, s>>>(M, n, ldo, hi);
    prof_end(PK_TC_SPLIT, s);
    DEVEL_LAUNCH_CHECK("k_mask_bf16");
    return DEVEL_OK;
}

}  // namespace tc
}  // namespace devel
