// Sigmoid resist, DSO loss, dL/dI and the binary printability metrics.
//
// Sec. III-A: Z = 1/(1 + exp(-sigma_z (I - I_th))), L_DSO = alpha L_ilt +
// beta L_pvb; process corners scale the image by the dose squared (Sec. II-C
// uses +/-2% dose). Sec. II-C: squared L2 = #{[I >= I_th] != Z_t}, PVBand =
// #{[d_in^2 I >= I_th] xor [d_out^2 I >= I_th]}.
//
// The per-pixel work is one HBM pass (read I and Z_t, write R: 9 B/px). The
// sums are accumulated in FP64 per thread, reduced per block in a fixed
// order, and the per-block partials are summed in block order by a second
// kernel, so results are bitwise reproducible.
#include "common.cuh"

namespace devel {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxParts = 1184;  // 8 x 148: bounded grid of the reduction

struct ResistArgs {
    float sigma_z, I_th, alpha, beta, d2in, d2out;
};

__device__ __forceinline__ float sigmoidf(float t) { return 1.f / (1.f + expf(-t)); }

__global__ void __launch_bounds__(kThreads)
k_resist(const float* __restrict__ I, const unsigned char* __restrict__ Zt, size_t npix, ResistArgs p,
         float* __restrict__ R, double* __restrict__ dpart, long long* __restrict__ lpart) {
    __shared__ double sd[4][kThreads / 32];
    __shared__ long long sl[2][kThreads / 32];
    // per-thread partials in FP32 (a thread sums a handful of pixels), FP64 from
    // the warp level up: GB300 issues few FP64 operations per clock
    float f0 = 0.f, f1 = 0.f, f2 = 0.f;
    int l2 = 0, pvb = 0;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < npix; i += stride) {
        const float Iv = I[i];
        const float zt = Zt[i] ? 1.f : 0.f;
        const float In = Iv, Ii = p.d2in * Iv, Io = p.d2out * Iv;
        const float zn = sigmoidf(p.sigma_z * (In - p.I_th));
        const float zi = sigmoidf(p.sigma_z * (Ii - p.I_th));
        const float zo = sigmoidf(p.sigma_z * (Io - p.I_th));
        const float en = zn - zt, ei = zi - zt, eo = zo - zt;
        f0 = fmaf(en, en, f0);
        f1 = fmaf(ei, ei, f1);
        f2 = fmaf(eo, eo, f2);
        const float gn = p.alpha * 2.f * en * p.sigma_z * zn * (1.f - zn);
        const float gi = p.beta * 2.f * ei * p.sigma_z * zi * (1.f - zi) * p.d2in;
        const float go = p.beta * 2.f * eo * p.sigma_z * zo * (1.f - zo) * p.d2out;
        R[i] = gn + gi + go;
        const bool pn = In >= p.I_th;
        l2 += (pn != (Zt[i] != 0));
        pvb += ((Ii >= p.I_th) != (Io >= p.I_th));
    }
    double s0 = f0, s1 = f1, s2 = f2;
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_down_sync(0xffffffffu, s0, o);
        s1 += __shfl_down_sync(0xffffffffu, s1, o);
        s2 += __shfl_down_sync(0xffffffffu, s2, o);
        l2 += __shfl_down_sync(0xffffffffu, l2, o);
        pvb += __shfl_down_sync(0xffffffffu, pvb, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        sd[0][w] = s0;
        sd[1][w] = s1;
        sd[2][w] = s2;
        sl[0][w] = l2;
        sl[1][w] = pvb;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0, c = 0;
        long long x = 0, y = 0;
        for (int i = 0; i < kThreads / 32; ++i) {
            a += sd[0][i];
            b += sd[1][i];
            c += sd[2][i];
            x += sl[0][i];
            y += sl[1][i];
        }
        dpart[blockIdx.x * 3 + 0] = a;
        dpart[blockIdx.x * 3 + 1] = b;
        dpart[blockIdx.x * 3 + 2] = c;
        lpart[blockIdx.x * 2 + 0] = x;
        lpart[blockIdx.x * 2 + 1] = y;
    }
}

// One block of 256 threads: thread t sums partials t, t+256, ... in order, then a
// fixed shuffle tree; the result does not depend on timing.
__global__ void __launch_bounds__(256)
k_resist_final(const double* __restrict__ dpart, const long long* __restrict__ lpart,
               int nparts, double alpha, double beta, double* loss4,
               long long* cnt2, double* loss_hist, long long* l2_hist,
               long long* pvb_hist, int* status) {
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

int resist_parts(int n) {
    const size_t npix = (size_t)n * n;
    size_t blocks = (npix + (size_t)kThreads * 4 - 1) / ((size_t)kThreads * 4);
    if (blocks > (size_t)kMaxParts) blocks = kMaxParts;
    if (blocks < 1) blocks = 1;
    return (int)blocks;
}

int launch_resist(int n, const float* I, const unsigned char* Zt, const devel_resist_params& p,
                  float* R, double* dpart, long long* lpart, int nparts, double* loss4,
                  long long* cnt2, double* loss_hist, long long* l2_hist, long long* pvb_hist,
                  int* status, cudaStream_t s) {
    ResistArgs a;
    a.sigma_z = p.sigma_z;
    a.I_th = p.I_th;
    a.alpha = p.alpha;
    a.beta = p.beta;
    a.d2in = p.dose_in * p.dose_in;
    a.d2out = p.dose_out * p.dose_out;
    prof_begin(PK_RESIST, s);
    k_resist<<<nparts, kThreads, 0, s>>>(I, Zt, (size_t)n * n, a, R, dpart, lpart);
    prof_end(PK_RESIST, s);
    DEVEL_LAUNCH_CHECK("k_resist");
    prof_begin(PK_RESIST_FINAL, s);
    k_resist_final<<<1, 256, 0, s>>>(dpart, lpart, nparts, (double)p.alpha, (double)p.beta, loss4,
                                    cnt2, loss_hist, l2_hist, pvb_hist, status);
    prof_end(PK_RESIST_FINAL, s);
    DEVEL_LAUNCH_CHECK("k_resist_final");
    return DEVEL_OK;
}

}  // namespace devel
