// Sigmoid resist, DSO loss, dL/dI and the binary printability metrics.
//
// Sec. III-A: Z = 1/(1 + exp(-sigma_z (I - I_th))), L_DSO = alpha L_ilt +
// beta L_pvb; process corners scale the image by the dose squared (Sec. II-C
// uses +/-2% dose). Sec. II-C: squared L2 = #{[I >= I_th] != Z_t}, PVBand =
// #{[d_in^2 I >= I_th] xor [d_out^2 I >= I_th]}.
//
// The standalone kernel is one HBM pass (read I and Z_t, write R: 9 B/px);
// inside the solver the same per-pixel code runs in the epilogue of the
// forward expansion instead (resist.cuh). Sums are FP32 per thread, FP64 from
// the warp up, reduced per block in a fixed order and then over blocks in
// block order, so results are bitwise reproducible.
#include "resist.cuh"

namespace devel {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxParts = 1184;  // 8 x 148: bounded grid of the standalone kernel

// Rows y = blockIdx.x, blockIdx.x + gridDim.x, ...; each thread four adjacent
// pixels (float4 / uchar4 loads when the row is 16-byte aligned).
__global__ void __launch_bounds__(kThreads)
k_resist(const float* __restrict__ I, const unsigned char* __restrict__ Zt, int n, ResistArgs p,
         float* __restrict__ R, __nv_bfloat16* __restrict__ Rhi, __nv_bfloat16* __restrict__ Rlo, int ldr,
         double* __restrict__ dpart, long long* __restrict__ lpart) {
    __shared__ double sd[3][32];
    __shared__ long long sl[2][32];
    LossAcc acc;
    const bool vec = (n & 3) == 0;
    for (int y = blockIdx.x; y < n; y += gridDim.x) {
        const size_t base = (size_t)y * n;
        for (int x0 = threadIdx.x * 4; x0 < n; x0 += blockDim.x * 4) {
            float iv[4], rv[4];
            unsigned char zv[4];
            if (vec) {
                const float4 q = *reinterpret_cast<const float4*>(I + base + x0);
                const uchar4 z = *reinterpret_cast<const uchar4*>(Zt + base + x0);
                iv[0] = q.x; iv[1] = q.y; iv[2] = q.z; iv[3] = q.w;
                zv[0] = z.x; zv[1] = z.y; zv[2] = z.z; zv[3] = z.w;
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    iv[j] = x0 + j < n ? I[base + x0 + j] : 0.f;
                    zv[j] = x0 + j < n ? Zt[base + x0 + j] : 0;
                }
            }
#pragma unroll
            for (int j = 0; j < 4; ++j)
                rv[j] = (x0 + j < n) ? resist_px(iv[j], zv[j] != 0, p, acc) : 0.f;
            if (R) {
                if (vec) {
                    *reinterpret_cast<float4*>(R + base + x0) = make_float4(rv[0], rv[1], rv[2], rv[3]);
                } else {
                    for (int j = 0; j < 4 && x0 + j < n; ++j) R[base + x0 + j] = rv[j];
                }
            }
            if (Rhi) {
                const size_t b2 = (size_t)y * ldr + x0;
                for (int j = 0; j < 4 && x0 + j < n; ++j) {
                    const __nv_bfloat16 h = __float2bfloat16_rn(rv[j]);
                    Rhi[b2 + j] = h;
                    Rlo[b2 + j] = __float2bfloat16_rn(rv[j] - __bfloat162float(h));
                }
            }
        }
    }
    block_store_loss(acc, blockIdx.x, dpart, lpart, sd, sl);
}

// One block of 256 threads: thread t sums partials t, t+256, ... in order, then a
// fixed shuffle tree; the result does not depend on timing.
__global__ void __launch_bounds__(256)
k_resist_final(const double* __restrict__ dpart, const long long* __restrict__ lpart, int nparts,
               double alpha, double beta, double* loss4, long long* cnt2, double* loss_hist,
               long long* l2_hist, long long* pvb_hist, int* status) {
    __shared__ double sd[3][8];
    __shared__ long long sl[2][8];
    double a = 0, b = 0, c = 0;
    long long x = 0, y = 0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
        a += dpart[i * 3 + 0];
        b += dpart[i * 3 + 1];
        c += dpart[i * 3 + 2];
        x += lpart[i * 2 + 0];
        y += lpart[i * 2 + 1];
    }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
        c += __shfl_down_sync(0xffffffffu, c, o);
        x += __shfl_down_sync(0xffffffffu, x, o);
        y += __shfl_down_sync(0xffffffffu, y, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        sd[0][w] = a;
        sd[1][w] = b;
        sd[2][w] = c;
        sl[0][w] = x;
        sl[1][w] = y;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    a = b = c = 0;
    x = y = 0;
    for (int i = 0; i < 8; ++i) {
        a += sd[0][i];
        b += sd[1][i];
        c += sd[2][i];
        x += sl[0][i];
        y += sl[1][i];
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

}  // namespace

int resist_parts(int n) { return n < kMaxParts ? n : kMaxParts; }

int launch_resist_final(int nparts, const devel_resist_params& p, const double* dpart, const long long* lpart,
                        double* loss4, long long* cnt2, double* loss_hist, long long* l2_hist,
                        long long* pvb_hist, int* status, cudaStream_t s) {
    prof_begin(PK_RESIST_FINAL, s);
    k_resist_final<<<1, 256, 0, s>>>(dpart, lpart, nparts, (double)p.alpha, (double)p.beta, loss4, cnt2,
                                     loss_hist, l2_hist, pvb_hist, status);
    prof_end(PK_RESIST_FINAL, s);
    DEVEL_LAUNCH_CHECK("k_resist_final");
    return DEVEL_OK;
}

int launch_resist(int n, const float* I, const unsigned char* Zt, const devel_resist_params& p,
                  float* R, __nv_bfloat16* Rhi, __nv_bfloat16* Rlo, int ldr, double* dpart,
                  long long* lpart, int nparts, double* loss4, long long* cnt2, double* loss_hist,
                  long long* l2_hist, long long* pvb_hist, int* status, cudaStream_t s) {
    prof_begin(PK_RESIST, s);
    k_resist<<<nparts, kThreads, 0, s>>>(I, Zt, n, make_resist_args(p), R, Rhi, Rlo, ldr, dpart, lpart);
    prof_end(PK_RESIST, s);
    DEVEL_LAUNCH_CHECK("k_resist");
    return launch_resist_final(nparts, p, dpart, lpart, loss4, cnt2, loss_hist, l2_hist, pvb_hist, status, s);
}

}  // namespace devel
