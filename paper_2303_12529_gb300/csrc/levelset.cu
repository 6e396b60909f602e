// Level-set update of the DSO loop.
//
// Eq. (dso_evolution) with the descent sign (velocity V = +dL/dM), the
// central differences of Eq. (numerical-settings), the curvature term of
// Eq. (curva_numer), Godunov first-order upwinding for the transport term,
// and the mask of Eq. (phi2mask). One HBM pass: read phi and V (and m),
// write phi_out and the mask, 13 B/px (17 with m). The 3x3 neighbourhood
// comes from a shared-memory tile with a one-pixel halo; borders replicate
// the edge pixel (Neumann ghosts).
#include "common.cuh"

namespace devel {
namespace {

// Tile of 128 x 8 pixels per block of 32 x 8 threads, four adjacent pixels per
// thread; the (8 + 2) x (128 + 2) neighbourhood is staged in shared memory.
constexpr int kTX = 32, kTYS = 8, kPX = 4, kW = kTX * kPX;

__device__ __forceinline__ float step_px(float c, float xm, float xp, float ym, float yp, float xpyp, float xmyp,
                                         float xpym, float xmym, float v, float inv_vmax, float dt, float lam,
                                         float mm) {
    float out = c;
    if (inv_vmax > 0.f) {
        const float F = -dt * (v * inv_vmax);
        const float dmx = c - xm, dpx = xp - c, dmy = c - ym, dpy = yp - c;
        if (F > 0.f) {
            const float a = fmaxf(dmx, 0.f), b = fminf(dpx, 0.f), cc = fmaxf(dmy, 0.f), d = fminf(dpy, 0.f);
            out -= F * sqrtf(a * a + b * b + cc * cc + d * d);
        } else if (F < 0.f) {
            const float a = fminf(dmx, 0.f), b = fmaxf(dpx, 0.f), cc = fminf(dmy, 0.f), d = fmaxf(dpy, 0.f);
            out -= F * sqrtf(a * a + b * b + cc * cc + d * d);
        }
    }
    if (lam != 0.f) {
        const float px = 0.5f * (xp - xm), py = 0.5f * (yp - ym);
        const float pxx = xp + xm - 2.f * c, pyy = yp + ym - 2.f * c;
        const float pxy = 0.25f * ((xpyp - xmyp) - (xpym - xmym));
        const float den = px * px + py * py;
        float kc = 0.f;
        if (den >= 1e-12f) kc = __fdividef(pxx * py * py - 2.f * px * py * pxy + pyy * px * px, den);
        out += dt * lam * mm * kc;
    }
    return out;
}

__global__ void __launch_bounds__(kTX * kTYS)
k_levelset_step(const float* __restrict__ phi, const float* __restrict__ V,
                const double* __restrict__ vmax, const float* __restrict__ m, float dt, float lam,
                int n, float* __restrict__ phi_out, unsigned char* __restrict__ mask_out,
                __nv_bfloat16* __restrict__ mask_bf, int ldb) {
    __shared__ float t[kTYS + 2][kW + 2];
    __shared__ float s_inv;
    const int bx = blockIdx.x * kW, by = blockIdx.y * kTYS;
    const int tid = threadIdx.y * kTX + threadIdx.x;
    if (tid == 0) {
        // FP32 reciprocal of max|V| (0 when there is no transport); one per block
        const double vm = *vmax;
        s_inv = vm > 0.0 ? 1.0f / (float)vm : 0.f;
    }
    // stage the tile: all of a thread's loads are issued before its shared stores
    constexpr int kTile = (kTYS + 2) * (kW + 2);
    constexpr int kPer = (kTile + kTX * kTYS - 1) / (kTX * kTYS);
    float tv[kPer];
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
        const int i = tid + u * kTX * kTYS;
        const int ly = i / (kW + 2), lx = i - ly * (kW + 2);
        const int y = min(max(by + ly - 1, 0), n - 1);
        const int x = min(max(bx + lx - 1, 0), n - 1);
        tv[u] = i < kTile ? phi[(size_t)y * n + x] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
        const int i = tid + u * kTX * kTYS;
        if (i < kTile) (&t[0][0])[i] = tv[u];
    }
    __syncthreads();
    const int y = by + threadIdx.y;
    if (y >= n) return;
    const float inv = s_inv;
    const int ly = threadIdx.y + 1;
    const size_t prow = (size_t)y * n;
    // pixel j of this thread: x = bx + threadIdx.x + 32 j (consecutive lanes, consecutive
    // pixels: coalesced global access, conflict-free shared-memory reads)
    float vv[kPX], mv[kPX];
#pragma unroll
    for (int j = 0; j < kPX; ++j) {
        const int x = bx + threadIdx.x + kTX * j;
        vv[j] = x < n ? V[prow + x] : 0.f;
        mv[j] = (m && x < n) ? m[prow + x] : 1.f;
    }
#pragma unroll
    for (int j = 0; j < kPX; ++j) {
        const int lx0 = threadIdx.x + kTX * j;
        const int x = bx + lx0;
        if (x >= n) break;
        const int lx = lx0 + 1;
        const size_t p = prow + x;
        const float o = step_px(t[ly][lx], t[ly][lx - 1], t[ly][lx + 1], t[ly - 1][lx], t[ly + 1][lx],
                                t[ly + 1][lx + 1], t[ly + 1][lx - 1], t[ly - 1][lx + 1], t[ly - 1][lx - 1], vv[j], inv,
                                dt, lam, mv[j]);
        phi_out[p] = o;
        if (mask_out) mask_out[p] = o <= 0.f ? 1 : 0;
        if (mask_bf) mask_bf[(size_t)y * ldb + x] = __float2bfloat16_rn(o <= 0.f ? 1.f : 0.f);
    }
}

__global__ void k_mask_from_phi(const float* __restrict__ phi, size_t npix, unsigned char* __restrict__ M) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < npix; i += stride)
        M[i] = phi[i] <= 0.f ? 1 : 0;
}

__global__ void k_u8_to_f32(const unsigned char* __restrict__ M, size_t npix, float* __restrict__ out) {
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < npix; i += stride)
        out[i] = M[i] ? 1.f : 0.f;
}

int grid_for(size_t npix) {
    size_t b = (npix + 1023) / 1024;
    if (b > 4736) b = 4736;  // 32 x 148
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

int launch_levelset_step(int n, const float* phi, const float* V, const double* vmax,
                         const float* m, float dt, float lambda, float* phi_out,
                         unsigned char* mask_out, __nv_bfloat16* mask_bf, int ldb, cudaStream_t s) {
    dim3 grid((n + kW - 1) / kW, (n + kTYS - 1) / kTYS);
    prof_begin(PK_STEP, s);
    k_levelset_step<<<grid, dim3(kTX, kTYS), 0, s>>>(phi, V, vmax, m, dt, lambda, n, phi_out, mask_out, mask_bf,
                                                    ldb);
    prof_end(PK_STEP, s);
    DEVEL_LAUNCH_CHECK("k_levelset_step");
    return DEVEL_OK;
}

int launch_mask_from_phi(int n, const float* phi, unsigned char* M, cudaStream_t s) {
    const size_t npix = (size_t)n * n;
    prof_begin(PK_MASK, s);
    k_mask_from_phi<<<grid_for(npix), 256, 0, s>>>(phi, npix, M);
    prof_end(PK_MASK, s);
    DEVEL_LAUNCH_CHECK("k_mask_from_phi");
    return DEVEL_OK;
}

int launch_u8_to_f32(int n, const unsigned char* M, float* out, cudaStream_t s) {
    const size_t npix = (size_t)n * n;
    prof_begin(PK_U8F32, s);
    k_u8_to_f32<<<grid_for(npix), 256, 0, s>>>(M, npix, out);
    prof_end(PK_U8F32, s);
    DEVEL_LAUNCH_CHECK("k_u8_to_f32");
    return DEVEL_OK;
}

}  // namespace devel
