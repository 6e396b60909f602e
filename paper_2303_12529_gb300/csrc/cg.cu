// Conjugate-gradient direction of the level-set velocity.
//
// Sec. III-C: DSO optimises with the conjugate-gradient method and sets the time step
// from max|v| (the CFL condition). The paper prints no CG update; the reading here is
// nonlinear CG on the velocity field with the Polak-Ribiere coefficient clipped at
// zero (PR+):
//   beta = max(0, <V, V - Vp> / <Vp, Vp>)   (0 when <Vp, Vp> = 0)
//   D    = V + beta D_prev                  (restart: D = V, beta = 0)
// and the level-set step then moves the front with D, normalised by max|D|.
//
//   k_cg_dots    one HBM pass over V and Vp: per-block FP32 sums of V.V, V.Vp, Vp.Vp
//                (fixed order), the last CTA adds the block sums (FP32, fixed order)
//                and writes beta;
//   k_cg_update  one pass: D = V + beta D, Vp = V, per-block max|D| (FP32 bit
//                patterns, so NaN/Inf reach the status word), the last CTA writes
//                max|D| as FP64.
// Pixels go four at a time (float4) when n*n % 4 == 0. Block b takes the b-th of
// gridDim.x equal contiguous ranges, so the partial sums depend only on n.
#include <algorithm>

#include "common.cuh"

namespace devel {
namespace {

constexpr int kCgThreads = 256;
constexpr int kCgMaxParts = 1024;

// V is read by both passes (kept in L2 by the first: plain loads; streamed by the
// second: evict-first); Vp and D once per pass
__device__ __forceinline__ float4 ld4(const float* p, long long g) {
    return reinterpret_cast<const float4*>(p)[g];
}
__device__ __forceinline__ float4 ld4_last(const float* p, long long g) {
    return __ldcs(reinterpret_cast<const float4*>(p) + g);
}

// FP32 dot products of one thread's pixels; vector path when npix % 4 == 0
__global__ void __launch_bounds__(kCgThreads)
k_cg_dots(const float* __restrict__ V, const float* __restrict__ Vp, long long npix, float* __restrict__ part,
          unsigned* counter, double* beta_out, float* beta_f, int* status) {
    pdl_trigger();
    pdl_wait();
    float vv = 0.f, vp = 0.f, pp = 0.f;
    const int b = blockIdx.x, nb = gridDim.x;
    if ((npix & 3) == 0) {
        const long long G = npix >> 2, g0 = G * b / nb, g1 = G * (b + 1) / nb;
        // two groups per step, both loaded before either is used
        long long g = g0 + threadIdx.x;
        for (; g + kCgThreads < g1; g += 2 * kCgThreads) {
            const float4 a = ld4(V, g), c = ld4(Vp, g), a2 = ld4(V, g + kCgThreads), c2 = ld4(Vp, g + kCgThreads);
            vv = fmaf(a.x, a.x, fmaf(a.y, a.y, fmaf(a.z, a.z, fmaf(a.w, a.w, vv))));
            vp = fmaf(a.x, c.x, fmaf(a.y, c.y, fmaf(a.z, c.z, fmaf(a.w, c.w, vp))));
            pp = fmaf(c.x, c.x, fmaf(c.y, c.y, fmaf(c.z, c.z, fmaf(c.w, c.w, pp))));
            vv = fmaf(a2.x, a2.x, fmaf(a2.y, a2.y, fmaf(a2.z, a2.z, fmaf(a2.w, a2.w, vv))));
            vp = fmaf(a2.x, c2.x, fmaf(a2.y, c2.y, fmaf(a2.z, c2.z, fmaf(a2.w, c2.w, vp))));
            pp = fmaf(c2.x, c2.x, fmaf(c2.y, c2.y, fmaf(c2.z, c2.z, fmaf(c2.w, c2.w, pp))));
        }
        if (g < g1) {
            const float4 a = ld4(V, g), c = ld4(Vp, g);
            vv = fmaf(a.x, a.x, fmaf(a.y, a.y, fmaf(a.z, a.z, fmaf(a.w, a.w, vv))));
            vp = fmaf(a.x, c.x, fmaf(a.y, c.y, fmaf(a.z, c.z, fmaf(a.w, c.w, vp))));
            pp = fmaf(c.x, c.x, fmaf(c.y, c.y, fmaf(c.z, c.z, fmaf(c.w, c.w, pp))));
        }
    } else {
        const long long i0 = npix * b / nb, i1 = npix * (b + 1) / nb;
        for (long long i = i0 + threadIdx.x; i < i1; i += kCgThreads) {
            const float a = V[i], c = Vp[i];
            vv = fmaf(a, a, vv);
            vp = fmaf(a, c, vp);
            pp = fmaf(c, c, pp);
        }
    }
    __shared__ float sf[3][kCgThreads / 32];
    for (int o = 16; o > 0; o >>= 1) {
        vv += __shfl_down_sync(0xffffffffu, vv, o);
        vp += __shfl_down_sync(0xffffffffu, vp, o);
        pp += __shfl_down_sync(0xffffffffu, pp, o);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        sf[0][w] = vv;
        sf[1][w] = vp;
        sf[2][w] = pp;
    }
    __syncthreads();
    __shared__ bool last;
    if (threadIdx.x == 0) {
        float a = 0.f, c = 0.f, d = 0.f;
        for (int i = 0; i < kCgThreads / 32; ++i) {
            a += sf[0][i];
            c += sf[1][i];
            d += sf[2][i];
        }
        part[b * 3 + 0] = a;
        part[b * 3 + 1] = c;
        part[b * 3 + 2] = d;
        __threadfence();
        last = atomicAdd(counter, 1u) == (unsigned)nb - 1u;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // the block partials summed in a fixed order: thread t takes t, t + 256, ..., then a
    // shuffle tree and the warps in order (FP32: the FP64 pipe of this part issues one
    // warp instruction per ~64 cycles, and beta needs no more than FP32 accuracy)
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
    for (int i = threadIdx.x; i < nb; i += kCgThreads) {
        s0 += __ldcg(part + i * 3 + 0);
        s1 += __ldcg(part + i * 3 + 1);
        s2 += __ldcg(part + i * 3 + 2);
    }
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_down_sync(0xffffffffu, s0, o);
        s1 += __shfl_down_sync(0xffffffffu, s1, o);
        s2 += __shfl_down_sync(0xffffffffu, s2, o);
    }
    if (lane == 0) {
        sf[0][w] = s0;
        sf[1][w] = s1;
        sf[2][w] = s2;
    }
    __syncthreads();
    if (threadIdx.x != 0) return;
    float a = 0.f, c = 0.f, d = 0.f;
    for (int i = 0; i < kCgThreads / 32; ++i) {
        a += sf[0][i];
        c += sf[1][i];
        d += sf[2][i];
    }
    float beta = 0.f;
    if (!isfinite(a) || !isfinite(c) || !isfinite(d)) {
        if (status) *status = DEVEL_ENAN;
    } else if (d > 0.f) {
        beta = fmaxf(0.f, (a - c) / d);
    }
    *beta_f = beta;
    if (beta_out) *beta_out = beta;
    *counter = 0u;
}

__device__ __forceinline__ int absbits(float x) { return (int)(__float_as_uint(x) & 0x7fffffffu); }

// D = V + beta D (beta_f NULL: restart, D = V), Vp = V, max|D|
__global__ void __launch_bounds__(kCgThreads)
k_cg_update(const float* __restrict__ V, float* __restrict__ Vp, float* __restrict__ D, long long npix,
            const float* __restrict__ beta_f, float* __restrict__ vpart, unsigned* counter, double* vmax,
            int* status) {
    pdl_trigger();
    pdl_wait();
    const float beta = beta_f ? *beta_f : 0.f;
    const int b = blockIdx.x, nb = gridDim.x;
    // max of |D| as the integer max of its bit pattern: a NaN (pattern above +Inf)
    // survives the max, where fmaxf would drop it
    int mx = 0;
    if ((npix & 3) == 0) {
        const long long G = npix >> 2, g0 = G * b / nb, g1 = G * (b + 1) / nb;
        for (long long g = g0 + threadIdx.x; g < g1; g += kCgThreads) {
            const float4 v = ld4_last(V, g);
            float4 d = make_float4(0.f, 0.f, 0.f, 0.f);
            if (beta_f) d = reinterpret_cast<const float4*>(D)[g];
            d.x = fmaf(beta, d.x, v.x);
            d.y = fmaf(beta, d.y, v.y);
            d.z = fmaf(beta, d.z, v.z);
            d.w = fmaf(beta, d.w, v.w);
            reinterpret_cast<float4*>(D)[g] = d;
            reinterpret_cast<float4*>(Vp)[g] = v;
            mx = max(max(mx, max(absbits(d.x), absbits(d.y))), max(absbits(d.z), absbits(d.w)));
        }
    } else {
        const long long i0 = npix * b / nb, i1 = npix * (b + 1) / nb;
        for (long long i = i0 + threadIdx.x; i < i1; i += kCgThreads) {
            const float v = V[i];
            const float d = beta_f ? fmaf(beta, D[i], v) : v;
            D[i] = d;
            Vp[i] = v;
            mx = max(mx, absbits(d));
        }
    }
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_down_sync(0xffffffffu, mx, o));
    __shared__ int sm[kCgThreads / 32];
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        int m = 0;
        for (int i = 0; i < kCgThreads / 32; ++i) m = max(m, sm[i]);
        vpart[b] = __int_as_float(m);
    }
    vmax_last_block(vpart, nb, counter, vmax, status);
}

}  // namespace

// Blocks of the CG passes (= partials): 4 per SM, at least 4096 pixels per block.
int cg_parts(int n) {
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
    return (int)std::max(1LL, std::min<long long>({want, 4LL * sms, (long long)kCgMaxParts}));
}

int launch_cg_direction(int n, const float* V, float* Vp, float* D, bool restart, float* part, float* vpart,
                        float* beta_f, double* beta_out, unsigned* counters, double* vmax, int* status,
                        cudaStream_t s) {
    const long long npix = (long long)n * n;
    const int nb = cg_parts(n);
    if (!restart) {
        prof_begin(PK_CG_DOTS, s);
        cudaError_t e = launch_pdl(k_cg_dots, dim3(nb), dim3(kCgThreads), 0, s, V, (const float*)Vp, npix, part,
                                   counters, beta_out, beta_f, status);
        prof_end(PK_CG_DOTS, s);
        if (e != cudaSuccess) return cuda_error(e, "k_cg_dots");
    } else if (beta_out) {
        DEVEL_CUDA_TRY(cudaMemsetAsync(beta_out, 0, sizeof(double), s));
    }
    prof_begin(PK_CG_UPDATE, s);
    cudaError_t e = launch_pdl(k_cg_update, dim3(nb), dim3(kCgThreads), 0, s, V, Vp, D, npix,
                               restart ? (const float*)nullptr : (const float*)beta_f, vpart, counters + 1, vmax,
                               status);
    prof_end(PK_CG_UPDATE, s);
    if (e != cudaSuccess) return cuda_error(e, "k_cg_update");
    return DEVEL_OK;
}

}  // namespace devel
