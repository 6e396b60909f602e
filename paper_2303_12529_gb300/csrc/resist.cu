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

constexpr int kThreads = 256;
constexpr int kMaxParts = 512;  // blocks of the resist kernel (rows split evenly when n % 512 == 0)

// Final sum of the per-block partials by one block (any multiple of 32 threads up to
// 1024): thread t sums partials t, t + blockDim, ... in order, then a fixed shuffle
// tree; the result does not depend on timing.
__device__ void resist_final_block(const double* __restrict__ dpart, const long long* __restrict__ lpart,
                                   int nparts, double alpha, double beta, double* loss4, long long* cnt2,
                                   double* loss_hist, long long* l2_hist, long long* pvb_hist, int* status) {
    __shared__ double fd[3][32];
    __shared__ long long fl[2][32];
    double a = 0, b = 0, c = 0;
    long long x = 0, y = 0;
#pragma unroll 2
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
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
    const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if ((threadIdx.x & 31) == 0) {
        fd[0][w] = a;
        fd[1][w] = b;
        fd[2][w] = c;
        fl[0][w] = x;
        fl[1][w] = y;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    a = b = c = 0;
    x = y = 0;
    for (int i = 0; i < nw; ++i) {
        a += fd[0][i];
        b += fd[1][i];
        c += fd[2][i];
        x += fl[0][i];
        y += fl[1][i];
    }
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

// Rows y = blockIdx.x, blockIdx.x + gridDim.x, ... taken two at a time; each thread
// takes kGrp groups of four adjacent pixels in both rows and issues all their loads
// before any arithmetic.
constexpr int kGrp = 2;
constexpr int kItems = 2 * kGrp;

__global__ void __launch_bounds__(kThreads)
k_resist(const float* __restrict__ I, const unsigned char* __restrict__ Zt, int n, ResistArgs p,
         float* __restrict__ R, __nv_bfloat16* __restrict__ Rhi, __nv_bfloat16* __restrict__ Rlo, int ldr,
         double* __restrict__ dpart, long long* __restrict__ lpart, ResistOut out) {
    __shared__ float sf[3][32];
    __shared__ int si[2][32];
    LossAcc acc;
    const bool vec = (n & 3) == 0;
    const int span = blockDim.x * 4;
    for (int y0 = blockIdx.x; y0 < n; y0 += 2 * gridDim.x) {
        for (int xg = threadIdx.x * 4; xg < n; xg += kGrp * span) {
            float iv[kItems][4];
            unsigned char zv[kItems][4];
            bool ok[kItems];
#pragma unroll
            for (int u = 0; u < kItems; ++u) {
                const int y = y0 + (u / kGrp) * gridDim.x;
                const int x0 = xg + (u % kGrp) * span;
                ok[u] = y < n && x0 < n;
                const size_t base = (size_t)y * n + x0;
                if (ok[u] && vec) {
                    const float4 f = *reinterpret_cast<const float4*>(I + base);
                    const uchar4 z = *reinterpret_cast<const uchar4*>(Zt + base);
                    iv[u][0] = f.x; iv[u][1] = f.y; iv[u][2] = f.z; iv[u][3] = f.w;
                    zv[u][0] = z.x; zv[u][1] = z.y; zv[u][2] = z.z; zv[u][3] = z.w;
                } else {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const bool in = ok[u] && x0 + j < n;
                        iv[u][j] = in ? I[base + j] : 0.f;
                        zv[u][j] = in ? Zt[base + j] : 0;
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < kItems; ++u) {
                if (!ok[u]) continue;
                const int y = y0 + (u / kGrp) * gridDim.x;
                const int x0 = xg + (u % kGrp) * span;
                const size_t base = (size_t)y * n + x0;
                float rv[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) rv[j] = (x0 + j < n) ? resist_px(iv[u][j], zv[u][j] != 0, p, acc) : 0.f;
                if (R) {
                    if (vec) {
                        *reinterpret_cast<float4*>(R + base) = make_float4(rv[0], rv[1], rv[2], rv[3]);
                    } else {
                        for (int j = 0; j < 4 && x0 + j < n; ++j) R[base + j] = rv[j];
                    }
                }
                if (Rhi) {
                    const size_t b2 = (size_t)y * ldr + x0;
                    __nv_bfloat16 h[4], l[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        h[j] = __float2bfloat16_rn(rv[j]);
                        l[j] = __float2bfloat16_rn(rv[j] - __bfloat162float(h[j]));
                    }
                    if (vec && (ldr & 3) == 0) {
                        *reinterpret_cast<uint2*>(Rhi + b2) = *reinterpret_cast<const uint2*>(h);
                        *reinterpret_cast<uint2*>(Rlo + b2) = *reinterpret_cast<const uint2*>(l);
                    } else {
                        for (int j = 0; j < 4 && x0 + j < n; ++j) {
                            Rhi[b2 + j] = h[j];
                            Rlo[b2 + j] = l[j];
                        }
                    }
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
    if (!last) return;
    __threadfence();
    resist_final_block(dpart, lpart, gridDim.x, out.alpha, out.beta, out.loss4, out.cnt2, out.loss_hist,
                       out.l2_hist, out.pvb_hist, out.status);
    if (threadIdx.x == 0) *out.counter = 0u;
}

// Two images (nominal focus In, defocused Id): one pixel per thread per pass, dL/dIn
// and dL/dId written as FP32 images (Rn, Rd; may alias In, Id) or as bf16 hi/lo
// operands (row pitch ldr); the same partial sums and last-block total as k_resist.
__global__ void __launch_bounds__(kThreads)
k_resist_defocus(const float* In, const float* Id, const unsigned char* __restrict__ Zt, int n, ResistArgs p,
                 float* Rn, float* Rd, __nv_bfloat16* __restrict__ Rnhi, __nv_bfloat16* __restrict__ Rnlo,
                 __nv_bfloat16* __restrict__ Rdhi, __nv_bfloat16* __restrict__ Rdlo, int ldr,
                 double* __restrict__ dpart, long long* __restrict__ lpart, ResistOut out) {
    __shared__ float sf[3][32];
    __shared__ int si[2][32];
    LossAcc acc;
    const size_t npix = (size_t)n * n, stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < npix; i += stride) {
        float gD;
        const float gN = resist_px2(In[i], Id[i], Zt[i] != 0, p, acc, gD);
        if (Rn) {
            Rn[i] = gN;
            Rd[i] = gD;
        }
        if (Rnhi) {
            const size_t y = i / (size_t)n, x = i - y * (size_t)n, q = y * ldr + x;
            const __nv_bfloat16 hn = __float2bfloat16_rn(gN), hd = __float2bfloat16_rn(gD);
            Rnhi[q] = hn;
            Rnlo[q] = __float2bfloat16_rn(gN - __bfloat162float(hn));
            Rdhi[q] = hd;
            Rdlo[q] = __float2bfloat16_rn(gD - __bfloat162float(hd));
        }
    }
    block_store_loss(acc, blockIdx.x, dpart, lpart, sf, si);
    __shared__ bool last;
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(out.counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    resist_final_block(dpart, lpart, gridDim.x, out.alpha, out.beta, out.loss4, out.cnt2, out.loss_hist,
                       out.l2_hist, out.pvb_hist, out.status);
    if (threadIdx.x == 0) *out.counter = 0u;
}

}  // namespace

int resist_parts(int n) { return n < kMaxParts ? n : kMaxParts; }  // <= 512 partials

int launch_resist(int n, const float* I, const unsigned char* Zt, const devel_resist_params& p,
                  float* R, __nv_bfloat16* Rhi, __nv_bfloat16* Rlo, int ldr, double* dpart,
                  long long* lpart, int nparts, double* loss4, long long* cnt2, double* loss_hist,
                  long long* l2_hist, long long* pvb_hist, int* status, unsigned* counter, cudaStream_t s) {
    ResistOut out{counter, (double)p.alpha, (double)p.beta, loss4, cnt2, loss_hist, l2_hist, pvb_hist, status};
    prof_begin(PK_RESIST, s);
    k_resist<<<nparts, kThreads, 0, s>>>(I, Zt, n, make_resist_args(p), R, Rhi, Rlo, ldr, dpart, lpart, out);
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
    k_resist_defocus<<<nparts, kThreads, 0, s>>>(In, Id, Zt, n, make_resist_args(p), Rn, Rd, Rnhi, Rnlo, Rdhi, Rdlo,
                                                 ldr, dpart, lpart, out);
    prof_end(PK_RESIST, s);
    DEVEL_LAUNCH_CHECK("k_resist_defocus");
    return DEVEL_OK;
}

}  // namespace devel
