// Supervision of the curvature modulation m_theta (Sec. III-B, modulation branch).
//
//   k_mod_candidates  candidate maps m~_j = H(phi_gt + dh_j) for all j in one pass over
//                     phi_gt (Heaviside: 1 where phi_gt + dh_j >= 0, in FP32);
//   k_ahf_loss        L_m = sum (H_eps(phi_m) - m_gt)^2 with the approximated
//                     Heaviside H_eps(phi) = (1 + (2/pi) atan(phi/eps)) / 2, and
//                     dL_m/dphi_m = 2 (H_eps - m_gt) (eps/pi) / (eps^2 + phi^2).
// The label search itself (devel_modulation_search) runs the candidates as clips of one
// devel_ilt_solve, then
//   k_argmin_final    the index of the smallest final L_DSO (ties: the first; a
//                     non-finite loss never wins).
#include <algorithm>

#include "common.cuh"

namespace devel {
namespace {

constexpr int kModThreads = 256;

struct Shifts {
    float dh[DEVEL_MOD_MAX_CANDIDATES];
};

__global__ void __launch_bounds__(kModThreads)
k_mod_candidates(const float* __restrict__ phi, long long npix, int ncand, Shifts sh, float* __restrict__ m) {
    const long long stride = (long long)gridDim.x * kModThreads;
    if ((npix & 3) == 0) {
        const long long G = npix >> 2;
        for (long long g = (long long)blockIdx.x * kModThreads + threadIdx.x; g < G; g += stride) {
            const float4 p = reinterpret_cast<const float4*>(phi)[g];
            for (int j = 0; j < ncand; ++j) {
                const float d = sh.dh[j];
                reinterpret_cast<float4*>(m + (size_t)j * npix)[g] =
                    make_float4(p.x + d >= 0.f ? 1.f : 0.f, p.y + d >= 0.f ? 1.f : 0.f, p.z + d >= 0.f ? 1.f : 0.f,
                                p.w + d >= 0.f ? 1.f : 0.f);
            }
        }
    } else {
        for (long long i = (long long)blockIdx.x * kModThreads + threadIdx.x; i < npix; i += stride) {
            const float p = phi[i];
            for (int j = 0; j < ncand; ++j) m[(size_t)j * npix + i] = p + sh.dh[j] >= 0.f ? 1.f : 0.f;
        }
    }
}

// one pixel: residual r = H_eps(phi) - m and the gradient 2 r H_eps'(phi)
__device__ __forceinline__ float ahf_px(float phi, float m, float eps, float inv_eps, float& g) {
    const float h = 0.5f + atanf(phi * inv_eps) * 0.318309886f;  // 1/pi
    const float r = h - m;
    g = 2.f * r * (eps * 0.318309886f) / fmaf(phi, phi, eps * eps);
    return r;
}

// Block b sums its contiguous range in FP32 (fixed order), writes the block sum as
// fixed point; the last CTA adds the fixed-point partials exactly and writes FP64.
__global__ void __launch_bounds__(kModThreads)
k_ahf_loss(const float* __restrict__ phi, const float* __restrict__ mgt, long long npix, float eps,
           float* __restrict__ grad, long long* __restrict__ qpart, unsigned* counter, double* loss) {
    const int b = blockIdx.x, nb = gridDim.x;
    const float inv_eps = 1.f / eps;
    float s = 0.f;
    if ((npix & 3) == 0) {
        const long long G = npix >> 2, g0 = G * b / nb, g1 = G * (b + 1) / nb;
        for (long long g = g0 + threadIdx.x; g < g1; g += kModThreads) {
            const float4 p = reinterpret_cast<const float4*>(phi)[g], m = reinterpret_cast<const float4*>(mgt)[g];
            float4 d;
            const float r0 = ahf_px(p.x, m.x, eps, inv_eps, d.x), r1 = ahf_px(p.y, m.y, eps, inv_eps, d.y);
            const float r2 = ahf_px(p.z, m.z, eps, inv_eps, d.z), r3 = ahf_px(p.w, m.w, eps, inv_eps, d.w);
            s = fmaf(r0, r0, s);
            s = fmaf(r1, r1, s);
            s = fmaf(r2, r2, s);
            s = fmaf(r3, r3, s);
            if (grad) reinterpret_cast<float4*>(grad)[g] = d;
        }
    } else {
        const long long i0 = npix * b / nb, i1 = npix * (b + 1) / nb;
        for (long long i = i0 + threadIdx.x; i < i1; i += kModThreads) {
            float d;
            const float r = ahf_px(phi[i], mgt[i], eps, inv_eps, d);
            s = fmaf(r, r, s);
            if (grad) grad[i] = d;
        }
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    __shared__ float sw[kModThreads / 32];
    __shared__ bool last;
    if ((threadIdx.x & 31) == 0) sw[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int i = 0; i < kModThreads / 32; ++i) t += sw[i];
        qpart[b] = to_q32(t);
        __threadfence();
        last = atomicAdd(counter, 1u) == (unsigned)nb - 1u;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    long long q = 0;
    bool bad = false;
    for (int i = threadIdx.x; i < nb; i += kModThreads) {
        const long long v = __ldcg(qpart + i);
        bad |= v == kQBad;
        q += v;
    }
    for (int o = 16; o > 0; o >>= 1) q += __shfl_down_sync(0xffffffffu, q, o);
    bad = __syncthreads_or(bad);
    __shared__ long long sq[kModThreads / 32];
    if ((threadIdx.x & 31) == 0) sq[threadIdx.x >> 5] = q;
    __syncthreads();
    if (threadIdx.x != 0) return;
    long long t = 0;
    for (int i = 0; i < kModThreads / 32; ++i) t += sq[i];
    *loss = bad ? __longlong_as_double(0x7ff8000000000000ll) : (double)t * (1.0 / 4294967296.0);
    *counter = 0u;
}

// One warp: lane j reads candidates j, j + 32, ...; a candidate wins over another with a
// strictly smaller finite loss, or with an equal loss and a smaller index.
__global__ void k_argmin_final(const double* __restrict__ hist, int ncand, int ldh, int col, int* best) {
    const int lane = threadIdx.x;
    double v = 0.0;
    int i = -1;
    for (int j = lane; j < ncand; j += 32) {
        const double x = hist[(size_t)j * ldh + col];
        if (isfinite(x) && (i < 0 || x < v)) {
            v = x;
            i = j;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        const double v2 = __shfl_down_sync(0xffffffffu, v, o);
        const int i2 = __shfl_down_sync(0xffffffffu, i, o);
        if (i2 >= 0 && (i < 0 || v2 < v || (v2 == v && i2 < i))) {
            v = v2;
            i = i2;
        }
    }
    if (lane == 0) *best = i < 0 ? 0 : i;
}

}  // namespace

int launch_argmin_final(const double* hist, int ncand, int ldh, int col, int* best, cudaStream_t s) {
    k_argmin_final<<<1, 32, 0, s>>>(hist, ncand, ldh, col, best);
    DEVEL_LAUNCH_CHECK("k_argmin_final");
    return DEVEL_OK;
}

int launch_mod_candidates(int n, const float* phi, int ncand, const float* dh_host, float* m, cudaStream_t s) {
    Shifts sh{};
    for (int j = 0; j < ncand; ++j) sh.dh[j] = dh_host[j];
    const long long npix = (long long)n * n;
    const long long work = (npix & 3) == 0 ? npix >> 2 : npix;
    const int grid = (int)std::min<long long>((work + kModThreads - 1) / kModThreads, 4096);
    k_mod_candidates<<<grid, kModThreads, 0, s>>>(phi, npix, ncand, sh, m);
    DEVEL_LAUNCH_CHECK("k_mod_candidates");
    return DEVEL_OK;
}

int launch_ahf_loss(int n, const float* phi, const float* mgt, float eps, float* grad, long long* qpart, int nparts,
                    unsigned* counter, double* loss, cudaStream_t s) {
    const long long npix = (long long)n * n;
    const int grid = (int)std::max(1LL, std::min<long long>({(npix + 4095) / 4096, (long long)nparts}));
    k_ahf_loss<<<grid, kModThreads, 0, s>>>(phi, mgt, npix, eps, grad, qpart, counter, loss);
    DEVEL_LAUNCH_CHECK("k_ahf_loss");
    return DEVEL_OK;
}

}  // namespace devel
