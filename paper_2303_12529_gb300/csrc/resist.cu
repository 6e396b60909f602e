// Sigmoid resist, DSO loss, dL/dI and the binary printability metrics.
//
// Sec. III-A: Z = 1/(1 + exp(-sigma_z (I - I_th))), L_DSO = alpha L_ilt +
// beta L_pvb; process corners scale the image by the dose squared (Sec. II-C
// uses +/-2% dose). Sec. II-C: squared L2 = #{[I >= I_th] != Z_t}, PVBand =
// #{[d_in^2 I >= I_th] xor [d_out^2 I >= I_th]}.
//
// One HBM pass: read I and Z_t, write R (FP32, 9 B/px) or its bf16 hi/lo split
// (the operand of the adjoint's reduction, 9 B/px). Sums are FP32 within a block
// and FP64 across blocks (the global loss reduction), each in a fixed order, so
// results are bitwise reproducible.
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
};

// One block per SM (the grid is the SM count): a block of 1024 threads (768 for two
// images, whose registers allow no more), so that every SM gets the same share of the
// image; the block scheduler could otherwise stack several smaller blocks on some SMs
// and leave others idle.
template <bool kDef>
__host__ __device__ constexpr int resist_threads() { return kDef ? 768 : 1024; }
constexpr int kMaxParts = 512;  // most blocks (loss partials) of a resist kernel

// Final sum of the per-block partials by the first warp of the last block: lane l sums
// partials l, l + 32, ... in order, then a fixed shuffle tree; the result does not
// depend on timing. (One warp: the chain of dependent FP64 additions is ~10 long.)
__device__ void resist_final_warp(const double* __restrict__ dpart, const long long* __restrict__ lpart,
                                  int nparts, double alpha, double beta, double* loss4, long long* cnt2,
                                  double* loss_hist, long long* l2_hist, long long* pvb_hist, int* status) {
    const int lane = threadIdx.x;
    double a = 0, b = 0, c = 0;
    long long x = 0, y = 0;
#pragma unroll 4
    for (int i = lane; i < nparts; i += 32) {
        a += __ldcg(dpart + i * 3 + 0);
        b += __ldcg(dpart + i * 3 + 1);
        c += __ldcg(dpart + i * 3 + 2);
        x += __ldcg(lpart + i * 2 + 0);
        y += __ldcg(lpart + i * 2 + 1);
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
        c += __shfl_down_sync(0xffffffffu, c, o);
        x += __shfl_down_sync(0xffffffffu, x, o);
        y += __shfl_down_sync(0xffffffffu, y, o);
    }
    if (lane != 0) return;
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

__device__ __forceinline__ void split_store4(__nv_bfloat16* hi, __nv_bfloat16* lo, size_t q, const float (&r)[4]) {
    __nv_bfloat16 h[4], l[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        h[j] = __float2bfloat16_rn(r[j]);
        l[j] = __float2bfloat16_rn(r[j] - __bfloat162float(h[j]));
    }
    *reinterpret_cast<uint2*>(hi + q) = *reinterpret_cast<const uint2*>(h);
    *reinterpret_cast<uint2*>(lo + q) = *reinterpret_cast<const uint2*>(l);
}

template <bool kDef>
__global__ void __launch_bounds__(resist_threads<kDef>(), 1)
k_resist(const float* In, const float* Id, const unsigned char* __restrict__ Zt, int n, ResistArgs p,
         float* Rn, float* Rd, __nv_bfloat16* __restrict__ Rnhi, __nv_bfloat16* __restrict__ Rnlo,
         __nv_bfloat16* __restrict__ Rdhi, __nv_bfloat16* __restrict__ Rdlo, int ldr,
         double* __restrict__ dpart, long long* __restrict__ lpart, ResistOut out) {
    __shared__ float sf[3][32];
    __shared__ int si[2][32];
    constexpr int kThreads = resist_threads<kDef>();
    LossAcc acc;
    const long long npix = (long long)n * n;
    if ((n & 3) == 0 && (!Rnhi || (ldr & 3) == 0)) {
        const int nq = n >> 2;  // groups per row
        const long long G = npix >> 2;
        const long long g0 = G * blockIdx.x / gridDim.x, g1 = G * (blockIdx.x + 1) / gridDim.x;
        long long g = g0 + threadIdx.x;
        // row / group-in-row of g, advanced incrementally (the step is blockDim.x groups)
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
#pragma unroll
                        for (int j = 0; j < 4; ++j) rn[j] = resist_px(iv[j], zv[j] != 0, p, acc);
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
        const long long i0 = npix * blockIdx.x / gridDim.x, i1 = npix * (blockIdx.x + 1) / gridDim.x;
        for (long long i = i0 + threadIdx.x; i < i1; i += kThreads) {
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
    block_store_loss(acc, blockIdx.x, dpart, lpart, sf, si);
    // the last block to finish sums all partials (fixed order) and resets the counter
    __shared__ bool last;
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(out.counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last || threadIdx.x >= 32) return;
    __threadfence();
    resist_final_warp(dpart, lpart, gridDim.x, out.alpha, out.beta, out.loss4, out.cnt2, out.loss_hist,
                      out.l2_hist, out.pvb_hist, out.status);
    if (threadIdx.x == 0) *out.counter = 0u;
}

}  // namespace

// Blocks of the resist kernels (= loss partials, <= 512): one per SM, fewer for small
// images (at least 4096 pixels per block).
int resist_parts(int n) {
    static int sms = 0;
    if (!sms) {
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
            sms = v;
        else
            sms = 148;
    }
    const long long want = ((long long)n * n + 4095) / 4096;
    return (int)std::max(1LL, std::min<long long>({want, (long long)sms, (long long)kMaxParts}));
}

int launch_resist(int n, const float* I, const unsigned char* Zt, const devel_resist_params& p,
                  float* R, __nv_bfloat16* Rhi, __nv_bfloat16* Rlo, int ldr, double* dpart,
                  long long* lpart, int nparts, double* loss4, long long* cnt2, double* loss_hist,
                  long long* l2_hist, long long* pvb_hist, int* status, unsigned* counter, cudaStream_t s) {
    ResistOut out{counter, (double)p.alpha, (double)p.beta, loss4, cnt2, loss_hist, l2_hist, pvb_hist, status};
    prof_begin(PK_RESIST, s);
    k_resist<false><<<nparts, resist_threads<false>(), 0, s>>>(I, nullptr, Zt, n, make_resist_args(p), R, nullptr, Rhi, Rlo,
                                                nullptr, nullptr, ldr, dpart, lpart, out);
    prof_end(PK_RESIST, s);
    DEVEL_LAUNCH_CHECK("k_resist");
    return DEVEL_OK;
}

int launch_resist_defocus(int n, const float* In, const float* Id, const unsigned char* Zt,
                          const devel_resist_params& p, float* Rn, float* Rd, __nv_bfloat16* Rnhi,
                          __nv_bfloat16* Rnlo, __nv_bfloat16* Rdhi, __nv_bfloat16* Rdlo, int ldr, double* dpart,
                          long long* lpart, int nparts, double* loss4, long long* cnt2, double* loss_hist,
                          long long* l2_hist, long long* pvb_hist, int* status, unsigned* counter, cudaStream_t s) {
    ResistOut out{counter, (double)p.alpha, (double)p.beta, loss4, cnt2, loss_hist, l2_hist, pvb_hist, status};
    prof_begin(PK_RESIST, s);
    k_resist<true><<<nparts, resist_threads<true>(), 0, s>>>(In, Id, Zt, n, make_resist_args(p), Rn, Rd, Rnhi, Rnlo, Rdhi, Rdlo,
                                               ldr, dpart, lpart, out);
    prof_end(PK_RESIST, s);
    DEVEL_LAUNCH_CHECK("k_resist_defocus");
    return DEVEL_OK;
}

}  // namespace devel
