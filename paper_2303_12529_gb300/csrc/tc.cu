// Tensor-core (tcgen05) NT GEMM for the truncated-DFT contractions, sm_103a.
//
//   D[m][nn] = scale * sum_k A[m][k] B[nn][k]
//
// with A and B given as bf16 hi/lo pairs (x = hi + lo, hi = rn_bf16(x),
// lo = rn_bf16(x - hi)) and the compensated product
//   A B^T ~ A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T      (FP32 accumulate)
// (the A_lo term is skipped when A is exact in bf16, e.g. a 0/1 mask).
//
// One CTA computes a 128 x BN tile (UMMA M = 128, cta_group::1):
//   warp 0, one thread   TMA producer: 64-element K slabs of A_hi, A_lo,
//                        B_hi, B_lo (128-byte swizzle) into a STAGES ring;
//   warp 1, one thread   MMA issuer: 4 K-steps of 16 per slab, 2-3 MMAs each,
//                        accumulator in TMEM; tcgen05.commit frees a stage;
//   warps 0-3            epilogue: tcgen05.ld 32 lanes x 16 columns at a
//                        time, scale, store (and the per-CTA max |D|).
// Split-K runs over gridDim.z; every split writes its own slice of D.
// Every mbarrier wait is bounded (about one second of %globaltimer); a
// timeout sets *err = DEVEL_ETIMEOUT and the CTA stops issuing work, waits
// (bounded) for the copies it issued, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include <mutex>

#include "common.cuh"
#include "tc.cuh"

namespace devel {
namespace tc {
namespace {

constexpr int kBM = 128;
constexpr int kBK = 64;             // bf16 elements per 128-byte swizzle row
constexpr uint32_t kABytes = kBM * kBK * 2;
constexpr unsigned long long kWaitNs = 1000000000ull;  // bounded waits: 1 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n"
        "  .reg .pred p;\n"
        "  mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "  selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase with the given parity; false (and *err set) after ~1 s.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, int* err) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (globaltimer() - t0 > kWaitNs) {
            if (err) atomicExch(err, DEVEL_ETIMEOUT);
            return false;
        }
    }
}

__device__ __forceinline__ void tma_load_2d(const CUtensorMap* tm, uint64_t* bar, void* dst, int c0, int c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::
            "r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(tm)), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
        : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void fence_before_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row atoms of
// 1024 bytes (stride byte offset), start address >> 4 in bits [0, 14),
// descriptor version 1 in bits [46, 48), layout type 2 (SWIZZLE_128B) in [61, 64).
__device__ __forceinline__ uint64_t smem_desc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(16u >> 4) << 16;     // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024u >> 4) << 32;   // stride byte offset: next 8-row group
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction descriptor, kind::f16: D f32, A bf16, B bf16, both K-major, N >> 3, M >> 4.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n"
        "  .reg .pred p;\n"
        "  setp.ne.b32 p, %4, 0;\n"
        "  tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
        "}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <int BN>
struct Cfg {
    static constexpr uint32_t kBBytes = BN * kBK * 2;
    static constexpr uint32_t kStage = 2 * kABytes + 2 * kBBytes;
    // as many stages (2..4) as fit in 227 KB of shared memory with the alignment slack
    static constexpr int kFit = (int)((227u * 1024u - 2048u) / kStage);
    static constexpr int kStages = kFit > 4 ? 4 : kFit;
    static_assert(kFit >= 2, "tile too wide for double buffering");
    static constexpr uint32_t kCols = BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256;
    static constexpr size_t kSmem = 1024 + (size_t)kStages * kStage + 256;
};

template <int BN, int EPI>
__global__ void __launch_bounds__(128, 1)
k_tc_gemm(const __grid_constant__ CUtensorMap tmAhi, const __grid_constant__ CUtensorMap tmAlo,
          const __grid_constant__ CUtensorMap tmBhi, const __grid_constant__ CUtensorMap tmBlo, int M, int N,
          int kb_per_split, int kb_total, int ksteps_last, int use_alo, const EpiArgs ep, int* err) {
    using CF = Cfg<BN>;
    constexpr int S = CF::kStages;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + S * CF::kStage);
    uint64_t* empty = full + S;
    uint64_t* accum = empty + S;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum + 1);
    __shared__ float red[4];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * BN;
    const int kb0 = blockIdx.z * kb_per_split;
    const int nkb = max(0, min(kb_per_split, kb_total - kb0));

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(accum, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(tmem_slot, CF::kCols);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    auto stage_ptr = [&](int s, int which) -> uint8_t* {
        // which: 0 A_hi, 1 A_lo, 2 B_hi, 3 B_lo
        uint8_t* base = smem + s * CF::kStage;
        return which < 2 ? base + which * kABytes : base + 2 * kABytes + (which - 2) * CF::kBBytes;
    };

    int issued = 0;  // producer: slabs whose loads were issued
    bool ok = true;
    if (warp == 0 && lane == 0 && nkb > 0) {
        const uint32_t bytes = (use_alo ? 2 : 1) * kABytes + 2 * CF::kBBytes;
        for (int i = 0; i < nkb; ++i) {
            const int s = i % S;
            if (i >= S && !mbar_wait(&empty[s], ((i / S) - 1) & 1, err)) {
                ok = false;
                break;
            }
            mbar_arrive_expect_tx(&full[s], bytes);
            const int kc = (kb0 + i) * kBK;
            tma_load_2d(&tmAhi, &full[s], stage_ptr(s, 0), kc, m0);
            if (use_alo) tma_load_2d(&tmAlo, &full[s], stage_ptr(s, 1), kc, m0);
            tma_load_2d(&tmBhi, &full[s], stage_ptr(s, 2), kc, n0);
            tma_load_2d(&tmBlo, &full[s], stage_ptr(s, 3), kc, n0);
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
            for (int kk = 0; kk < ksteps; ++kk) {
                const uint64_t adv = (uint64_t)(kk * 32) >> 4;  // 16 bf16 = 32 bytes along K
                mma_bf16(tmem, dAhi + adv, dBhi + adv, idesc, (i > 0 || kk > 0) ? 1u : 0u);
                mma_bf16(tmem, dAhi + adv, dBlo + adv, idesc, 1u);
                if (use_alo) mma_bf16(tmem, dAlo + adv, dBhi + adv, idesc, 1u);
            }
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
    float mx = 0.f;
    const int row = m0 + warp * 32 + lane;
    float* Cz = ep.C ? ep.C + (size_t)blockIdx.z * ep.split_stride : nullptr;
    const float scale = ep.scale;
    for (int c = 0; c < BN; c += 16) {
        float v[16];
        if (have) {
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
        } else {
#pragma unroll
            for (int j = 0; j < 16; ++j) v[j] = 0.f;
        }
#pragma unroll
        for (int j = 0; j < 16; ++j) v[j] *= scale;
        const int col0 = n0 + c;
        if (row < M) {
            float* dst = Cz + (size_t)row * ep.ldc + col0;
            if (col0 + 16 <= N && ((reinterpret_cast<uintptr_t>(dst) & 15u) == 0)) {
#pragma unroll
                for (int j = 0; j < 16; j += 4) {
                    *reinterpret_cast<float4*>(dst + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                    if (EPI == EPI_VEL)
                        mx = fmaxf(mx, fmaxf(fmaxf(fabsf(v[j]), fabsf(v[j + 1])), fmaxf(fabsf(v[j + 2]), fabsf(v[j + 3]))));
                }
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    if (col0 + j < N) {
                        dst[j] = v[j];
                        if (EPI == EPI_VEL) mx = fmaxf(mx, fabsf(v[j]));
                    }
                }
            }
        }
    }
    if (EPI == EPI_VEL) {
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
        if (lane == 0) red[warp] = mx;
    }
    const int part = blockIdx.y * gridDim.x + blockIdx.x;
    // a producer that stopped early waits (bounded) for the loads it issued
    if (warp == 0 && lane == 0 && !ok) {
        for (int i = max(0, issued - S); i < issued; ++i) mbar_wait(&full[i % S], (i / S) & 1, nullptr);
    }
    fence_before_sync();
    __syncthreads();
    if (EPI == EPI_VEL && threadIdx.x == 0)
        ep.vpart[part] = fmaxf(fmaxf(red[0], red[1]), fmaxf(red[2], red[3]));
    if (warp == 1) {
        fence_after_sync();
        tmem_dealloc(tmem, CF::kCols);
    }
    if (EPI == EPI_VEL) vmax_last_block(ep.vpart, gridDim.x * gridDim.y, ep.counter, ep.vmax, ep.status);
}

// ---------------------------------------------------------------------------
// Fused reduction onto a window: both contractions in one kernel
// ---------------------------------------------------------------------------
// CTA (row tile m0 of 128 image rows y, K slice z of 256 columns x):
//   phase 1  D1[y][c] = sum_x X[y][x] basis[c][x]            (the mainloop above, M = 128, N = BN)
//   phase 2  D1 is drained from TMEM, split to bf16 hi/lo and written transposed into shared
//            memory as a K-major operand B2[c2][y] (128-byte swizzle, as TMA would lay it out);
//            D2[c1][c2] = sum_y basis[c1][y] D1[y][c2] for c1 in 128-row blocks (A2 by TMA)
//   out      D2 rows c1 < BN to Q + slice * BN^2, slice = m-tile * splits + z (BN = ldk)
// The slices are then summed (in slice order) and combined into the complex window spectrum.
template <int BN>
struct Cfg2 {
    static constexpr uint32_t kB2 = BN * 128;                 // one k-block of B2 (bf16, 64 y)
    static constexpr uint32_t kPhase2 = 4 * kB2 + 4 * kABytes; // B2 hi/lo x 2 k-blocks, A2 hi/lo x 2 k-blocks
    static constexpr uint32_t kRing = Cfg<BN>::kStages * Cfg<BN>::kStage;
    static constexpr uint32_t kArena = kRing > kPhase2 ? kRing : kPhase2;
    static constexpr int kMB = (BN + 127) / 128;               // 128-row blocks of c1
    static constexpr uint32_t kCols = kMB > 1 ? 512 : Cfg<BN>::kCols;
    static constexpr size_t kSmem = 1024 + (size_t)kArena + 512;
};

template <int BN>
__global__ void __launch_bounds__(128, 1)
k_tc_spec2(const __grid_constant__ CUtensorMap tmAhi, const __grid_constant__ CUtensorMap tmAlo,
           const __grid_constant__ CUtensorMap tmBhi, const __grid_constant__ CUtensorMap tmBlo,
           const __grid_constant__ CUtensorMap tmChi, const __grid_constant__ CUtensorMap tmClo,
           int kb_per_split, int kb_total, int use_alo, float* __restrict__ Q, int* err) {
    using CF = Cfg<BN>;
    using C2 = Cfg2<BN>;
    constexpr int S = CF::kStages;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint64_t* full = reinterpret_cast<uint64_t*>(smem + C2::kArena);
    uint64_t* empty = full + S;
    uint64_t* accum = empty + S;
    uint64_t* a2full = accum + 1;  // [2]
    uint64_t* acc2 = a2full + 2;   // [2]
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc2 + 2);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * kBM;
    const int kb0 = blockIdx.z * kb_per_split;
    const int nkb = max(0, min(kb_per_split, kb_total - kb0));

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(accum, 1);
        for (int i = 0; i < 2; ++i) {
            mbar_init(&a2full[i], 1);
            mbar_init(&acc2[i], 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(tmem_slot, C2::kCols);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = *tmem_slot;

    auto stage_ptr = [&](int s, int which) -> uint8_t* {
        uint8_t* base = smem + s * CF::kStage;
        return which < 2 ? base + which * kABytes : base + 2 * kABytes + (which - 2) * CF::kBBytes;
    };
    // phase-2 buffers overlay the ring once phase 1 is complete
    uint8_t* B2hi = smem;                 // [2 k-blocks][BN rows][128 B]
    uint8_t* B2lo = smem + 2 * C2::kB2;
    uint8_t* A2hi = smem + 4 * C2::kB2;   // [2 k-blocks][128 rows][128 B]
    uint8_t* A2lo = A2hi + 2 * kABytes;
    constexpr uint32_t idesc = idesc_bf16(kBM, BN);

    // ---------------- phase 1 ----------------
    int issued = 0;
    bool ok = true;
    if (warp == 0 && lane == 0 && nkb > 0) {
        const uint32_t bytes = (use_alo ? 2 : 1) * kABytes + 2 * CF::kBBytes;
        for (int i = 0; i < nkb; ++i) {
            const int s = i % S;
            if (i >= S && !mbar_wait(&empty[s], ((i / S) - 1) & 1, err)) {
                ok = false;
                break;
            }
            mbar_arrive_expect_tx(&full[s], bytes);
            const int kc = (kb0 + i) * kBK;
            tma_load_2d(&tmAhi, &full[s], stage_ptr(s, 0), kc, m0);
            if (use_alo) tma_load_2d(&tmAlo, &full[s], stage_ptr(s, 1), kc, m0);
            tma_load_2d(&tmBhi, &full[s], stage_ptr(s, 2), kc, 0);
            tma_load_2d(&tmBlo, &full[s], stage_ptr(s, 3), kc, 0);
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
            for (int kk = 0; kk < kBK / 16; ++kk) {
                const uint64_t adv = (uint64_t)(kk * 32) >> 4;
                mma_bf16(tmem, dAhi + adv, dBhi + adv, idesc, (i > 0 || kk > 0) ? 1u : 0u);
                mma_bf16(tmem, dAhi + adv, dBlo + adv, idesc, 1u);
                if (use_alo) mma_bf16(tmem, dAlo + adv, dBhi + adv, idesc, 1u);
            }
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
        // A2 of the first c1 block: TMA into its buffers (the ring is idle now)
        if (warp == 0 && lane == 0) {
            mbar_arrive_expect_tx(&a2full[0], 4 * kABytes);
            for (int kb = 0; kb < 2; ++kb) {
                tma_load_2d(&tmChi, &a2full[0], A2hi + kb * kABytes, m0 + kb * kBK, 0);
                tma_load_2d(&tmClo, &a2full[0], A2lo + kb * kABytes, m0 + kb * kBK, 0);
            }
        }
        // drain D1: thread = row y of the tile, 16 columns at a time; write B2[c][y] (bf16 hi/lo)
        const int yl = warp * 32 + lane;
        const uint32_t kbo = (uint32_t)(yl >> 6) * C2::kB2;
        const uint32_t chunk = (uint32_t)((yl & 63) >> 3), e2 = (uint32_t)(yl & 7) * 2;
        for (int c = 0; c < BN; c += 16) {
            float v[16];
            tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const uint32_t c2 = (uint32_t)(c + j);
                const uint32_t off = kbo + c2 * 128u + (((chunk ^ (c2 & 7u)) << 4) | e2);
                const __nv_bfloat16 h = __float2bfloat16_rn(v[j]);
                *reinterpret_cast<__nv_bfloat16*>(B2hi + off) = h;
                *reinterpret_cast<__nv_bfloat16*>(B2lo + off) = __float2bfloat16_rn(v[j] - __bfloat162float(h));
            }
        }
        // generic-proxy stores -> visible to the tensor core (async proxy); TMEM reads done
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        fence_before_sync();
    }
    __syncthreads();
    fence_after_sync();
    bool ok2 = have;
    if (have && warp == 1 && lane == 0) {
        for (int mb = 0; mb < C2::kMB && ok2; ++mb) {
            if (!mbar_wait(&a2full[mb], 0, err)) {
                ok2 = false;
                break;
            }
            fence_after_sync();
            const uint32_t d2 = tmem + (uint32_t)(mb * 256);
            for (int kb = 0; kb < 2; ++kb) {
                const uint64_t dAhi = smem_desc_sw128(smem_u32(A2hi + kb * kABytes));
                const uint64_t dAlo = smem_desc_sw128(smem_u32(A2lo + kb * kABytes));
                const uint64_t dBhi = smem_desc_sw128(smem_u32(B2hi + kb * C2::kB2));
                const uint64_t dBlo = smem_desc_sw128(smem_u32(B2lo + kb * C2::kB2));
                for (int kk = 0; kk < kBK / 16; ++kk) {
                    const uint64_t adv = (uint64_t)(kk * 32) >> 4;
                    mma_bf16(d2, dAhi + adv, dBhi + adv, idesc, (kb > 0 || kk > 0) ? 1u : 0u);
                    mma_bf16(d2, dAhi + adv, dBlo + adv, idesc, 1u);
                    mma_bf16(d2, dAlo + adv, dBhi + adv, idesc, 1u);
                }
            }
            mma_commit(&acc2[mb]);
        }
    }
    if (have && C2::kMB > 1 && warp == 0 && lane == 0) {
        // A2 of the second c1 block reuses the buffers once the first block's MMAs are done
        if (mbar_wait(&acc2[0], 0, err)) {
            mbar_arrive_expect_tx(&a2full[1], 4 * kABytes);
            for (int kb = 0; kb < 2; ++kb) {
                tma_load_2d(&tmChi, &a2full[1], A2hi + kb * kABytes, m0 + kb * kBK, kBM);
                tma_load_2d(&tmClo, &a2full[1], A2lo + kb * kABytes, m0 + kb * kBK, kBM);
            }
        }
    }
    __syncwarp();
    // epilogue: D2 row c1 = mb * 128 + lane-row of this warp; write the slice of Q
    const int slice = blockIdx.y * gridDim.z + blockIdx.z;
    float* Qs = Q + (size_t)slice * BN * BN;
    for (int mb = 0; mb < C2::kMB; ++mb) {
        bool h2 = have;
        if (h2) h2 = mbar_wait(&acc2[mb], 0, err);
        h2 = __all_sync(0xffffffffu, h2);
        fence_after_sync();
        const int c1 = mb * kBM + warp * 32 + lane;
        for (int c = 0; c < BN; c += 16) {
            float v[16];
            if (h2) {
                tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(mb * 256 + c), v);
            } else {
#pragma unroll
                for (int j = 0; j < 16; ++j) v[j] = 0.f;
            }
            if (c1 < BN) {  // BN == ldk: each row of the slice is 16-float aligned
                float4* q4 = reinterpret_cast<float4*>(Qs + (size_t)c1 * BN + c);
#pragma unroll
                for (int j = 0; j < 4; ++j) q4[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
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
        tmem_dealloc(tmem, C2::kCols);
    }
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

// 0/1 mask row -> bf16 row of pitch ldo, four pixels per thread.
__global__ void k_mask_bf16(const unsigned char* __restrict__ M, int n, int ldo, __nv_bfloat16* __restrict__ hi) {
    const int r = blockIdx.y;
    const unsigned char* mr = M + (size_t)r * n;
    __nv_bfloat16* hr = hi + (size_t)r * ldo;
    const __nv_bfloat16 one = __float2bfloat16_rn(1.f), zero = __float2bfloat16_rn(0.f);
    for (int c = (blockIdx.x * blockDim.x + threadIdx.x) * 4; c < ldo; c += gridDim.x * blockDim.x * 4) {
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (c + j < ldo) hr[c + j] = (c + j < n && mr[c + j]) ? one : zero;
    }
}

template <int BN, int EPI>
cudaError_t set_attr_bn() {
    return cudaFuncSetAttribute(k_tc_gemm<BN, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)Cfg<BN>::kSmem);
}

template <int BN, int EPI>
int launch_gemm_bn(const Operands& op, int M, int N, int kb_per_split, int kb_total, int ksteps_last, int splits,
                   const EpiArgs& ep, int* err, cudaStream_t s) {
    using CF = Cfg<BN>;
    dim3 grid((N + BN - 1) / BN, (M + kBM - 1) / kBM, splits);
    k_tc_gemm<BN, EPI><<<grid, 128, CF::kSmem, s>>>(*op.Ahi, *op.Alo, *op.Bhi, *op.Blo, M, N, kb_per_split,
                                                     kb_total, ksteps_last, op.use_alo, ep, err);
    DEVEL_LAUNCH_CHECK("k_tc_gemm");
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

int launch_gemm(const Operands& op, int BN, int epi, int prof_kind, int M, int N, int K, int k_per_split,
                const EpiArgs& ep, int* err, cudaStream_t s) {
    if (K % 16 != 0 || k_per_split % kBK != 0)
        return set_error(DEVEL_EINVAL, "tc gemm: K=%d / split %d not aligned", K, k_per_split);
    const int kb_total = (K + kBK - 1) / kBK;
    const int kb_per_split = k_per_split / kBK;
    const int splits = (kb_total + kb_per_split - 1) / kb_per_split;
    const int ksteps_last = (K - (kb_total - 1) * kBK) / 16;
    prof_begin(prof_kind, s);
    int rc;
#define DEVEL_TC_ARGS op, M, N, kb_per_split, kb_total, ksteps_last, splits, ep, err, s
    if (BN == 128 && epi == EPI_VEL) {
        rc = launch_gemm_bn<128, EPI_VEL>(DEVEL_TC_ARGS);
    } else if (epi == EPI_STORE) {
        switch (BN) {
#define DEVEL_TC_CASE(bn)                                         \
    case bn:                                                      \
        rc = launch_gemm_bn<bn, EPI_STORE>(DEVEL_TC_ARGS);        \
        break;
            DEVEL_TC_CASE(16) DEVEL_TC_CASE(32) DEVEL_TC_CASE(48) DEVEL_TC_CASE(64) DEVEL_TC_CASE(80)
            DEVEL_TC_CASE(96) DEVEL_TC_CASE(112) DEVEL_TC_CASE(128) DEVEL_TC_CASE(144) DEVEL_TC_CASE(160)
            DEVEL_TC_CASE(176) DEVEL_TC_CASE(192) DEVEL_TC_CASE(208) DEVEL_TC_CASE(224) DEVEL_TC_CASE(240)
            DEVEL_TC_CASE(256)
#undef DEVEL_TC_CASE
            default:
                rc = set_error(DEVEL_EINVAL, "tc gemm: unsupported tile width %d", BN);
        }
    } else {
        rc = set_error(DEVEL_EINVAL, "tc gemm: unsupported epilogue %d with tile width %d", epi, BN);
    }
#undef DEVEL_TC_ARGS
    prof_end(prof_kind, s);
    return rc;
}

template <int BN>
int launch_spec2_bn(const Operands& op, const CUtensorMap* Chi, const CUtensorMap* Clo, int M, int kb_per_split,
                    int kb_total, int splits, float* Q, int* err, cudaStream_t s) {
    dim3 grid(1, (M + kBM - 1) / kBM, splits);
    k_tc_spec2<BN><<<grid, 128, Cfg2<BN>::kSmem, s>>>(*op.Ahi, *op.Alo, *op.Bhi, *op.Blo, *Chi, *Clo, kb_per_split,
                                                      kb_total, op.use_alo, Q, err);
    DEVEL_LAUNCH_CHECK("k_tc_spec2");
    return DEVEL_OK;
}

template <int BN>
cudaError_t set_attr_spec2() {
    return cudaFuncSetAttribute(k_tc_spec2<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg2<BN>::kSmem);
}

int spectrum2_slices(int M, int K) { return ((M + kBM - 1) / kBM) * ((K + kTcSplitK - 1) / kTcSplitK); }

int launch_spectrum2(const Operands& op, const CUtensorMap* Chi, const CUtensorMap* Clo, int BN, int M, int K,
                     float* Q, int* err, cudaStream_t s) {
    if (K % kBK != 0) return set_error(DEVEL_EINVAL, "tc spectrum: K=%d not a multiple of %d", K, kBK);
    const int kb_total = K / kBK, kb_per_split = kTcSplitK / kBK;
    const int splits = (kb_total + kb_per_split - 1) / kb_per_split;
    prof_begin(PK_TC_SPECTRUM, s);
    int rc;
    switch (BN) {
#define DEVEL_SPEC2_CASE(bn)                                                                               \
    case bn:                                                                                               \
        rc = launch_spec2_bn<bn>(op, Chi, Clo, M, kb_per_split, kb_total, splits, Q, err, s);              \
        break;
        DEVEL_SPEC2_CASE(16) DEVEL_SPEC2_CASE(32) DEVEL_SPEC2_CASE(48) DEVEL_SPEC2_CASE(64) DEVEL_SPEC2_CASE(80)
        DEVEL_SPEC2_CASE(96) DEVEL_SPEC2_CASE(112) DEVEL_SPEC2_CASE(128) DEVEL_SPEC2_CASE(144)
        DEVEL_SPEC2_CASE(160) DEVEL_SPEC2_CASE(176) DEVEL_SPEC2_CASE(192) DEVEL_SPEC2_CASE(208)
        DEVEL_SPEC2_CASE(224) DEVEL_SPEC2_CASE(240) DEVEL_SPEC2_CASE(256)
#undef DEVEL_SPEC2_CASE
        default:
            rc = set_error(DEVEL_EINVAL, "tc spectrum: unsupported window width %d", BN);
    }
    prof_end(PK_TC_SPECTRUM, s);
    return rc;
}

// Shared-memory opt-in of every kernel instantiation (call once per device,
// outside stream capture).
int init_attrs() {
    cudaError_t e = set_attr_bn<128, EPI_VEL>();
#define DEVEL_TC_ATTR(bn) if (e == cudaSuccess) e = set_attr_bn<bn, EPI_STORE>();
    DEVEL_TC_ATTR(16) DEVEL_TC_ATTR(32) DEVEL_TC_ATTR(48) DEVEL_TC_ATTR(64) DEVEL_TC_ATTR(80) DEVEL_TC_ATTR(96)
    DEVEL_TC_ATTR(112) DEVEL_TC_ATTR(128) DEVEL_TC_ATTR(144) DEVEL_TC_ATTR(160) DEVEL_TC_ATTR(176)
    DEVEL_TC_ATTR(192) DEVEL_TC_ATTR(208) DEVEL_TC_ATTR(224) DEVEL_TC_ATTR(240) DEVEL_TC_ATTR(256)
#undef DEVEL_TC_ATTR
#define DEVEL_SPEC2_ATTR(bn) if (e == cudaSuccess) e = set_attr_spec2<bn>();
    DEVEL_SPEC2_ATTR(16) DEVEL_SPEC2_ATTR(32) DEVEL_SPEC2_ATTR(48) DEVEL_SPEC2_ATTR(64) DEVEL_SPEC2_ATTR(80)
    DEVEL_SPEC2_ATTR(96) DEVEL_SPEC2_ATTR(112) DEVEL_SPEC2_ATTR(128) DEVEL_SPEC2_ATTR(144) DEVEL_SPEC2_ATTR(160)
    DEVEL_SPEC2_ATTR(176) DEVEL_SPEC2_ATTR(192) DEVEL_SPEC2_ATTR(208) DEVEL_SPEC2_ATTR(224) DEVEL_SPEC2_ATTR(240)
    DEVEL_SPEC2_ATTR(256)
#undef DEVEL_SPEC2_ATTR
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

int launch_mask_bf16(const unsigned char* M, int n, int ldo, __nv_bfloat16* hi, cudaStream_t s) {
    prof_begin(PK_TC_SPLIT, s);
    k_mask_bf16<<<dim3((ldo + 1023) / 1024, n), 256, 0, s>>>(M, n, ldo, hi);
    prof_end(PK_TC_SPLIT, s);
    DEVEL_LAUNCH_CHECK("k_mask_bf16");
    return DEVEL_OK;
}

}  // namespace tc
}  // namespace devel
