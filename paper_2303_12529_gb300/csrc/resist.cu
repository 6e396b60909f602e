// Sigmoid resist, DSO loss, dL/dI and the binary printability metrics.
//
// Sec. III-A: Z = 1/(1 + exp(-sigma_z (I - I_th))), L_DSO = alpha L_ilt +
// beta L_pvb; process corners scale the image by the dose squared (Sec. II-C
// uses +/-2% dose). Sec. II-C: squared L2 = #{[I >= I_th] != Z_t}, PVBand =
// #{[d_in^2 I >= I_th] xor [d_out^2 I >= I_th]}.
//
// One HBM pass: read I and Z_t, write R (FP32, 9 B/px) or its bf16 hi/lo split
// (the operand of the adjoint's reduction, 9 B/px). Loss sums are FP32 within a
// block of 256 threads (in a fixed order) and exact fixed-point int64 across blocks,
// converted to FP64 once (the global loss reduction), so results are bitwise
// reproducible.
#include <algorithm>

#include "resist.cuh"

namespace devel {
namespace {

struct ResistOut {
    unsigned* counter;
    double alpha, beta;
    double* loss4;
    long long* cnt2;
    double* loss_hist;
    long long* l2_hist;
    long long* pvb_hist;
    int* status;
    // clip blockIdx.y of a batch: images (and targets) n^2 apart, bf16 outputs n ldr apart,
    // partials 3 / 2 x part_stride apart, counters 1 apart, history entries hist_stride apart
    int part_stride, hist_stride;
};

// The image is split into "logical blocks" of 256 threads, as many as fit on every SM
// at once (4 per SM for one image, 3 for two, whose registers allow no more), each over
// an equal contiguous share of the image and each writing one loss partial. A CTA runs
// LB logical blocks: LB = 1 (CTAs of 256 threads, for clips that share the GPU with
// other clips' kernels) or LB = blocks per SM (one CTA per SM, which gives every SM the
// same work when the clip runs alone). Every thread does the same work and every
// partial is the same sum in the same order either way, so the results are identical.
constexpr int kThreads = 256;
template <bool kDef>
__host__ __device__ constexpr int resist_blocks_per_sm() { return kDef ? 3 : 4; }
constexpr int kMaxParts = 1024;  // most blocks (loss partials) of a resist kernel

// Final sum of the per-block partials by all threads of the last CTA: thread t sums
// the fixed-point partials t, t + blockDim.x, ... (one round of loads), then warp
// shuffles and the first warp add the threads' sums, all in exact int64 arithmetic (the
// result depends neither on timing nor on the CTA shape); the totals are converted to
// FP64 once. Every thread of the CTA must call it.
__device__ void resist_final_block(const long long* __restrict__ qpart, const long long* __restrict__ lpart,
                                   int nparts, double alpha, double beta, double* loss4, long long* cnt2,
                                   double* loss_hist, long long* l2_hist, long long* pvb_hist, int* status) {
    __shared__ long long fq[5][32];
    __shared__ int fbad;
    long long v[5] = {0, 0, 0, 0, 0};
    bool bad = false;
    if (threadIdx.x == 0) fbad = 0;
#pragma unroll 4
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
        const long long va = __ldcg(qpart + i * 3 + 0), vb = __ldcg(qpart + i * 3 + 1),
                        vc = __ldcg(qpart + i * 3 + 2);
        bad |= (va == kQBad) | (vb == kQBad) | (vc == kQBad);
        v[0] += va;
        v[1] += vb;
        v[2] += vc;
        v[3] += __ldcg(lpart + i * 2 + 0);
        v[4] += __ldcg(lpart + i * 2 + 1);
    }
#pragma unroll
    for (int j = 0; j < 5; ++j)
        for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_down_sync(0xffffffffu, v[j], o);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
    __syncthreads();  // fbad initialised
    if (bad) fbad = 1;
    if (lane == 0)
        for (int j = 0; j < 5; ++j) fq[j][w] = v[j];
    __syncthreads();
    if (w != 0) return;
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        v[j] = lane < nw ? fq[j][lane] : 0;
        for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_down_sync(0xffffffffu, v[j], o);
    }
    if (lane != 0) return;
    const long long x = v[3], y = v[4];
    bad = fbad != 0;
    constexpr double kScale = 1.0 / 4294967296.0;  // 2^-32
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
    const double a = bad ? nan : (double)v[0] * kScale, b = bad ? nan : (double)v[1] * kScale,
                 c = bad ? nan : (double)v[2] * kScale;
    const double L = alpha * a + beta * (b + c);
    if (loss4) {
        loss4[0] = L;
        loss4[1] = a;
        loss4[2] = b;
        loss4[3] = c;
    }
    if (cnt2) {
        cnt2[0] = x;
        cnt2[1] = y;
    }
    if (loss_hist) *loss_hist = L;
    if (l2_hist) *l2_hist = x;
    if (pvb_hist) *pvb_hist = y;
    if (status && !isfinite(L)) *status = DEVEL_ENAN;
}

// Block b of the grid takes the b-th of gridDim.x equal contiguous ranges of the image
// (in groups of four adjacent pixels of one row when n % 4 == 0, else single pixels);
// thread t takes groups t, t + blockDim.x, ... of its block's range, two per step, and loads
// the next step's groups before computing the current ones (software pipelining), so
// the loads of a warp overlap its own arithmetic. kDef: two images (nominal focus In,
// defocused Id for the inner corner), dL/dIn and dL/dId out; else one image, dL/dI out.
// R outputs are FP32 images (Rn, Rd; may alias In, Id) or bf16 hi/lo operands with row
// pitch ldr.
constexpr int kStep = 2;  // groups per thread per step

template <bool kDef>
struct Px4 {
    float4 i, d;
    uchar4 z;
};

template <bool kDef>
__device__ __forceinline__ Px4<kDef> load4(const float* In, const float* Id, const unsigned char* Zt, long long g,
                                           long long g1) {
    Px4<kDef> v;
    if (g < g1) {
        v.i = __ldcs(reinterpret_cast<const float4*>(In) + g);
        if (kDef) v.d = __ldcs(reinterpret_cast<const float4*>(Id) + g);
        v.z = __ldcs(reinterpret_cast<const uchar4*>(Zt) + g);
    }
    return v;
}

// hi = rn_bf16(r), lo = rn_bf16(r - hi) for four values, two per packed conversion
__device__ __forceinline__ void split_store4(__nv_bfloat16* hi, __nv_bfloat16* lo, size_t q, const float (&r)[4]) {
    const __nv_bfloat162 h01 = __floats2bfloat162_rn(r[0], r[1]), h23 = __floats2bfloat162_rn(r[2], r[3]);
    const float2 f01 = __bfloat1622float2(h01), f23 = __bfloat1622float2(h23);
    const float2 d01 = __fadd2_rn(make_float2(r[0], r[1]), make_float2(-f01.x, -f01.y));
    const float2 d23 = __fadd2_rn(make_float2(r[2], r[3]), make_float2(-f23.x, -f23.y));
    const __nv_bfloat162 l01 = __floats2bfloat162_rn(d01.x, d01.y);
    const __nv_bfloat162 l23 = __floats2bfloat162_rn(d23.x, d23.y);
    *reinterpret_cast<uint2*>(hi + q) =
        make_uint2(*reinterpret_cast<const uint32_t*>(&h01), *reinterpret_cast<const uint32_t*>(&h23));
    *reinterpret_cast<uint2*>(lo + q) =
        make_uint2(*reinterpret_cast<const uint32_t*>(&l01), *reinterpret_cast<const uint32_t*>(&l23));
}

template <bool kDef, int LB>
__global__ void __launch_bounds__(kThreads * LB, resist_blocks_per_sm<kDef>() / LB)
k_resist(const float* In, const float* Id, const unsigned char* __restrict__ Zt, int n, ResistArgs p,
         float* Rn, float* Rd, __nv_bfloat16* __restrict__ Rnhi, __nv_bfloat16* __restrict__ Rnlo,
         __nv_bfloat16* __restrict__ Rdhi, __nv_bfloat16* __restrict__ Rdlo, int ldr,
         long long* __restrict__ qpart, long long* __restrict__ lpart, ResistOut out) {
    __shared__ float sf[3][32];
    __shared__ int si[2][32];
    pdl_trigger();
    pdl_wait();
    if (blockIdx.y) {
        const size_t c = blockIdx.y, np = (size_t)n * n;
        In += c * np;
        if (kDef) Id += c * np;
        Zt += c * np;
        if (Rn) Rn += c * np;
        if (kDef && Rd) Rd += c * np;
        if (Rnhi) {
            Rnhi += c * (size_t)n * ldr;
            Rnlo += c * (size_t)n * ldr;
        }
        if (kDef && Rdhi) {
            Rdhi += c * (size_t)n * ldr;
            Rdlo += c * (size_t)n * ldr;
        }
        qpart += c * 3 * (size_t)out.part_stride;
        lpart += c * 2 * (size_t)out.part_stride;
        out.counter += c;
        if (out.loss_hist) out.loss_hist += c * out.hist_stride;
        if (out.l2_hist) out.l2_hist += c * out.hist_stride;
        if (out.pvb_hist) out.pvb_hist += c * out.hist_stride;
    }
    LossAcc acc;
    float2 s2[3] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
    const long long npix = (long long)n * n;
    // logical block lb of nlb, thread tid of its 256
    const int nlb = gridDim.x * LB, lb = blockIdx.x * LB + threadIdx.x / kThreads, tid = threadIdx.x % kThreads;
    if ((n & 3) == 0 && (!Rnhi || (ldr & 3) == 0)) {
        const int nq = n >> 2;  // groups per row
        const long long G = npix >> 2;
        const long long g0 = G * lb / nlb, g1 = G * (lb + 1) / nlb;
        long long g = g0 + tid;
        // row / group-in-row of g, advanced incrementally (the step is kStep * 256 groups)
        int y = (int)(g / nq), xq = (int)(g - (long long)y * nq);
        Px4<kDef> cur[kStep];
#pragma unroll
        for (int k = 0; k < kStep; ++k) cur[k] = load4<kDef>(In, Id, Zt, g + (long long)k * kThreads, g1);
        while (g < g1) {
            Px4<kDef> nxt[kStep];
#pragma unroll
            for (int k = 0; k < kStep; ++k)
                nxt[k] = load4<kDef>(In, Id, Zt, g + (long long)(kStep + k) * kThreads, g1);
#pragma unroll
            for (int k = 0; k < kStep; ++k) {
                const long long gk = g + (long long)k * kThreads;
                if (gk < g1) {
                    const float iv[4] = {cur[k].i.x, cur[k].i.y, cur[k].i.z, cur[k].i.w};
                    const unsigned char zv[4] = {cur[k].z.x, cur[k].z.y, cur[k].z.z, cur[k].z.w};
                    float rn[4], rd[4];
                    if (kDef) {
                        const float dv[4] = {cur[k].d.x, cur[k].d.y, cur[k].d.z, cur[k].d.w};
#pragma unroll
                        for (int j = 0; j < 4; ++j) rn[j] = resist_px2(iv[j], dv[j], zv[j] != 0, p, acc, rd[j]);
                    } else {
                        const float2 r01 = resist_pair(make_float2(iv[0], iv[1]), zv[0] != 0, zv[1] != 0, p, acc, s2);
                        const float2 r23 = resist_pair(make_float2(iv[2], iv[3]), zv[2] != 0, zv[3] != 0, p, acc, s2);
                        rn[0] = r01.x;
                        rn[1] = r01.y;
                        rn[2] = r23.x;
                        rn[3] = r23.y;
                    }
                    if (Rn) {
                        reinterpret_cast<float4*>(Rn)[gk] = make_float4(rn[0], rn[1], rn[2], rn[3]);
                        if (kDef) reinterpret_cast<float4*>(Rd)[gk] = make_float4(rd[0], rd[1], rd[2], rd[3]);
                    }
                    if (Rnhi) {
                        int yk = y, xk = xq + k * kThreads;
                        while (xk >= nq) {
                            xk -= nq;
                            ++yk;
                        }
                        const size_t q = (size_t)yk * ldr + ((size_t)xk << 2);
                        split_store4(Rnhi, Rnlo, q, rn);
                        if (kDef) split_store4(Rdhi, Rdlo, q, rd);
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < kStep; ++k) cur[k] = nxt[k];
            g += (long long)kStep * kThreads;
            xq += kStep * kThreads;
            while (xq >= nq) {
                xq -= nq;
                ++y;
            }
        }
    } else {  // ragged sides: one pixel at a time
        const long long i0 = npix * lb / nlb, i1 = npix * (lb + 1) / nlb;
        for (long long i = i0 + tid; i < i1; i += kThreads) {
            float gD = 0.f;
            const float gN = kDef ? resist_px2(In[i], Id[i], Zt[i] != 0, p, acc, gD)
                                  : resist_px(In[i], Zt[i] != 0, p, acc);
            if (Rn) {
                Rn[i] = gN;
                if (kDef) Rd[i] = gD;
            }
            if (Rnhi) {
                const long long yy = i / n, q = yy * ldr + (i - yy * n);
                const __nv_bfloat16 hn = __float2bfloat16_rn(gN);
                Rnhi[q] = hn;
                Rnlo[q] = __float2bfloat16_rn(gN - __bfloat162float(hn));
                if (kDef) {
                    const __nv_bfloat16 hd = __float2bfloat16_rn(gD);
                    Rdhi[q] = hd;
                    Rdlo[q] = __float2bfloat16_rn(gD - __bfloat162float(hd));
                }
            }
        }
    }
    acc.s0 += s2[0].x + s2[0].y;  // the paired lanes of the four-pixel path (zero elsewhere)
    acc.s1 += s2[1].x + s2[1].y;
    acc.s2 += s2[2].x + s2[2].y;
    block_store_loss(acc, blockIdx.x * LB, qpart, lpart, sf, si);
    // the last block to finish sums all partials (fixed order) and resets the counter
    __shared__ bool last;
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(out.counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    resist_final_block(qpart, lpart, nlb, out.alpha, out.beta, out.loss4, out.cnt2, out.loss_hist,
                       out.l2_hist, out.pvb_hist, out.status);
    if (threadIdx.x == 0) *out.counter = 0u;
}

}  // namespace

// Blocks of the resist kernels (= loss partials, <= 1024): resist_blocks_per_sm per SM
// (the grid of the one-image kernel, which the two-image kernel's grid never exceeds;
// that one uses the first 3 per SM), fewer for small images (at least 4096 pixels per
// block).
static int sm_total() {
    static int sms = 0;
    if (!sms) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
            sms = v;
        else
            sms = 148;
    }
    return sms;
}
static int resist_grid(int n, int per_sm) {
    const long long want = ((long long)n * n + 4095) / 4096;
    return (int)std::max(1LL, std::min<long long>({want, (long long)per_sm * sm_total(), (long long)kMaxParts}));
}
int resist_parts(int n) { return resist_grid(n, resist_blocks_per_sm<false>()); }

template <bool kDef, typename... A>
static cudaError_t launch_resist_kernel(int n, int nparts, bool alone, int B, cudaStream_t s, A... args) {
    constexpr int per_sm = resist_blocks_per_sm<kDef>();
    const int nlb = std::min(nparts, resist_grid(n, per_sm));
    if (alone && B == 1 && nlb % per_sm == 0)
        return launch_pdl(k_resist<kDef, per_sm>, dim3(nlb / per_sm), dim3(kThreads * per_sm), 0, s, args...);
    return launch_pdl(k_resist<kDef, 1>, dim3(nlb, B), dim3(kThreads), 0, s, args...);
}

int launch_resist(int n, const float* I, const unsigned char* Zt, const devel_resist_params& p,
                  float* R, __nv_bfloat16* Rhi, __nv_bfloat16* Rlo, int ldr, long long* qpart,
                  long long* lpart, int nparts, double* loss4, long long* cnt2, double* loss_hist,
                  long long* l2_hist, long long* pvb_hist, int* status, unsigned* counter, cudaStream_t s,
                  bool alone, int B, int hist_stride) {
    ResistOut out{counter, (double)p.alpha, (double)p.beta, loss4, cnt2, loss_hist, l2_hist, pvb_hist, status,
                  nparts, hist_stride};
    prof_begin(PK_RESIST, s);
    cudaError_t e = launch_resist_kernel<false>(n, nparts, alone, B, s, I, (const float*)nullptr, Zt, n,
                                                make_resist_args(p), R, (float*)nullptr, Rhi, Rlo,
                                                (__nv_bfloat16*)nullptr, (__nv_bfloat16*)nullptr, ldr, qpart, lpart,
                                                out);
    prof_end(PK_RESIST, s);
    if (e != cudaSuccess) return cuda_error(e, "k_resist");
    return DEVEL_OK;
}

int launch_resist_defocus(int n, const float* In, const float* Id, const unsigned char* Zt,
                          const devel_resist_params& p, float* Rn, float* Rd, __nv_bfloat16* Rnhi,
                          __nv_bfloat16* Rnlo, __nv_bfloat16* Rdhi, __nv_bfloat16* Rdlo, int ldr, long long* qpart,
                          long long* lpart, int nparts, double* loss4, long long* cnt2, double* loss_hist,
                          long long* l2_hist, long long* pvb_hist, int* status, unsigned* counter, cudaStream_t s,
                          bool alone) {
    ResistOut out{counter, (double)p.alpha, (double)p.beta, loss4, cnt2, loss_hist, l2_hist, pvb_hist, status,
                  nparts, 0};
    prof_begin(PK_RESIST, s);
    cudaError_t e = launch_resist_kernel<true>(n, nparts, alone, 1, s, In, Id, Zt, n, make_resist_args(p), Rn, Rd,
                                               Rnhi, Rnlo, Rdhi, Rdlo, ldr, qpart, lpart, out);
    prof_end(PK_RESIST, s);
    if (e != cudaSuccess) return cuda_error(e, "k_resist_defocus");
    return DEVEL_OK;
}

}  // namespace devel
