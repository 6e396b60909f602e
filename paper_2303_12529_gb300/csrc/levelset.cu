// Level-set update of the DSO loop.
//
// Eq. (dso_evolution) with the descent sign (velocity V = +dL/dM), the
// central differences of Eq. (numerical-settings), the curvature term of
// Eq. (curva_numer), Godunov first-order upwinding for the transport term,
// and the mask of Eq. (phi2mask). One HBM pass: read phi and V (and m),
// write phi_out and the mask, 13 B/px (17 with m; +2 with the bf16 mask of
// the tensor-core path). Borders replicate the edge pixel (Neumann ghosts).
#include "common.cuh"

namespace devel {
namespace {

// One thread per 4 adjacent pixels in each of kRows consecutive rows; its
// (kRows + 2) x 6 neighbourhood comes straight from global memory (rows
// y0-1 .. y0+kRows, columns x0-1 .. x0+4, borders replicated), each row loaded once
// for all the thread's outputs; overlapping reads between threads are served by
// L1. Vector loads and stores when the row is 16-byte aligned.
constexpr int kPX = 4;
constexpr int kRows = 2;

// sqrt by the SFU (relative error ~2^-22; phi tolerances are far looser)
__device__ __forceinline__ float sqrt_approx(float x) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

__device__ __forceinline__ float step_px(float c, float xm, float xp, float ym, float yp, float xpyp, float xmyp,
                                         float xpym, float xmym, float v, float inv_vmax, float dt, float lam,
                                         float mm) {
    float out = c;
    // Godunov upwind |grad phi| for the sign of F = -dt V / max|V| (one square root)
    const float F = -dt * (v * inv_vmax);
    const float dmx = c - xm, dpx = xp - c, dmy = c - ym, dpy = yp - c;
    const bool pos = F > 0.f;
    const float a = pos ? fmaxf(dmx, 0.f) : fminf(dmx, 0.f);
    const float b = pos ? fminf(dpx, 0.f) : fmaxf(dpx, 0.f);
    const float cc = pos ? fmaxf(dmy, 0.f) : fminf(dmy, 0.f);
    const float d = pos ? fminf(dpy, 0.f) : fmaxf(dpy, 0.f);
    out -= F * sqrt_approx(a * a + b * b + cc * cc + d * d);
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

__device__ __forceinline__ void load_row6(const float* __restrict__ r, int x0, int n, bool vec, float (&v)[kPX + 2]) {
    v[0] = r[max(x0 - 1, 0)];
    if (vec) {
        const float4 q = *reinterpret_cast<const float4*>(r + x0);
        v[1] = q.x; v[2] = q.y; v[3] = q.z; v[4] = q.w;
    } else {
#pragma unroll
        for (int j = 0; j < kPX; ++j) v[1 + j] = r[min(x0 + j, n - 1)];
    }
    v[kPX + 1] = r[min(x0 + kPX, n - 1)];
}

__global__ void __launch_bounds__(256)
k_levelset_step(const float* __restrict__ phi, const float* __restrict__ V,
                const double* __restrict__ vmax, const float* __restrict__ m, float dt, float lam,
                int n, float* __restrict__ phi_out, unsigned char* __restrict__ mask_out,
                __nv_bfloat16* __restrict__ mask_bf, int ldb) {
    const int y0 = blockIdx.y * kRows;
    const int x0 = (blockIdx.x * blockDim.x + threadIdx.x) * kPX;
    __shared__ float s_inv;
    pdl_trigger();
    pdl_wait();
    {  // clip blockIdx.z of a batch: its images n^2 apart, its bf16 mask n * ldb apart
        const size_t c = blockIdx.z, np = (size_t)n * n;
        phi += c * np;
        V += c * np;
        vmax += c;
        if (m) m += c * np;
        if (phi_out) phi_out += c * np;
        if (mask_out) mask_out += c * np;
        if (mask_bf) mask_bf += c * (size_t)n * ldb;
    }
    if (threadIdx.x == 0) {  // 1 / max|V| once per block (the FP64 pipe is narrow)
        const double vm = *vmax;
        s_inv = vm > 0.0 ? 1.0f / (float)vm : 0.f;  // F = 0 (no transport) when max|V| = 0
    }
    __syncthreads();
    if (x0 >= n) return;
    const float inv = s_inv;
    const bool vec = ((n & 3) == 0) && (x0 + kPX <= n);
    float rw[kRows + 2][kPX + 2];
#pragma unroll
    for (int r = 0; r < kRows + 2; ++r)
        load_row6(phi + (size_t)min(max(y0 - 1 + r, 0), n - 1) * n, x0, n, vec, rw[r]);
    float vv[kRows][kPX], mv[kRows][kPX];
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        const int y = min(y0 + r, n - 1);
        const size_t prow = (size_t)y * n;
        if (vec) {
            const float4 q = *reinterpret_cast<const float4*>(V + prow + x0);
            vv[r][0] = q.x; vv[r][1] = q.y; vv[r][2] = q.z; vv[r][3] = q.w;
            if (m) {
                const float4 w = *reinterpret_cast<const float4*>(m + prow + x0);
                mv[r][0] = w.x; mv[r][1] = w.y; mv[r][2] = w.z; mv[r][3] = w.w;
            } else {
                mv[r][0] = mv[r][1] = mv[r][2] = mv[r][3] = 1.f;
            }
        } else {
#pragma unroll
            for (int j = 0; j < kPX; ++j) {
                const bool in = x0 + j < n;
                vv[r][j] = in ? V[prow + x0 + j] : 0.f;
                mv[r][j] = (m && in) ? m[prow + x0 + j] : 1.f;
            }
        }
    }
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
        const int y = y0 + r;
        if (y >= n) break;
        const size_t prow = (size_t)y * n;
        const float(&rm)[kPX + 2] = rw[r];
        const float(&r0)[kPX + 2] = rw[r + 1];
        const float(&rp)[kPX + 2] = rw[r + 2];
        float o[kPX];
#pragma unroll
        for (int j = 0; j < kPX; ++j) {
            const int i = j + 1;
            o[j] = step_px(r0[i], r0[i - 1], r0[i + 1], rm[i], rp[i], rp[i + 1], rp[i - 1], rm[i + 1], rm[i - 1],
                           vv[r][j], inv, dt, lam, mv[r][j]);
        }
        if (vec) {
            if (phi_out) *reinterpret_cast<float4*>(phi_out + prow + x0) = make_float4(o[0], o[1], o[2], o[3]);
            if (mask_out)
                *reinterpret_cast<uchar4*>(mask_out + prow + x0) =
                    make_uchar4(o[0] <= 0.f, o[1] <= 0.f, o[2] <= 0.f, o[3] <= 0.f);
            if (mask_bf) {
                __nv_bfloat16 h[kPX];
#pragma unroll
                for (int j = 0; j < kPX; ++j) h[j] = __float2bfloat16_rn(o[j] <= 0.f ? 1.f : 0.f);
                *reinterpret_cast<uint2*>(mask_bf + (size_t)y * ldb + x0) = *reinterpret_cast<const uint2*>(h);
            }
        } else {
#pragma unroll
            for (int j = 0; j < kPX; ++j) {
                if (x0 + j < n) {
                    if (phi_out) phi_out[prow + x0 + j] = o[j];
                    if (mask_out) mask_out[prow + x0 + j] = o[j] <= 0.f ? 1 : 0;
                    if (mask_bf) mask_bf[(size_t)y * ldb + x0 + j] = __float2bfloat16_rn(o[j] <= 0.f ? 1.f : 0.f);
                }
            }
        }
    }
}

// ---------------------------------------------------------------------------
// WENO5 variant: the same update with fifth-order WENO one-sided derivatives
// (Hamilton-Jacobi WENO: three third-order ENO candidates on the one-sided
// differences, ideal weights 0.1 / 0.6 / 0.3 modulated by the smoothness
// indicators, eps = 1e-6 max v_k^2) in the Godunov flux. A block computes a
// 32 x 16 tile (two rows per thread) from a shared-memory copy with a 3-pixel
// halo (borders replicated).
// ---------------------------------------------------------------------------
constexpr int kWX = 32, kWY = 16, kWTh = 8, kWH = 3;
constexpr int kWTX = kWX + 2 * kWH, kWTY = kWY + 2 * kWH;

// WENO5 derivative from the one-sided differences v1..v5 (v3 nearest the node on the
// upwind side). The weights are invariant under v -> v / S (the smoothness
// indicators and eps scale as S^2), so they are computed on u = v / S with S the
// power of two at or below max|v| (an exact scaling; max|u| in [1, 2)): no overflow
// or underflow in FP32 where the differences are huge or tiny, and 0 where they all
// vanish. The normalised weights a_k / sum a_k with a_k = w_k / t_k^2 are formed as
// b_k / sum b_k with b_k = w_k prod_{l != k} t_l^2 (one division instead of four);
// with max|u| < 2 every t_k lies in [1e-6, 134], so the products stay in range.
__device__ __forceinline__ float weno5(float v1, float v2, float v3, float v4, float v5) {
    const float s = fmaxf(fmaxf(fmaxf(fabsf(v1), fabsf(v2)), fmaxf(fabsf(v3), fabsf(v4))), fabsf(v5));
    if (!(s > 0.f)) return 0.f;
    // S = 2^(E - 127) for the biased exponent E of s (E clamped to 253 so that 1/S is a
    // normal float; an infinite s still yields a non-finite result)
    const int eb = min(__float_as_int(s) & 0x7f800000, 253 << 23);
    const float S = __int_as_float(eb), r = __int_as_float((254 << 23) - eb);
    const float u1 = v1 * r, u2 = v2 * r, u3 = v3 * r, u4 = v4 * r, u5 = v5 * r;
    const float p1 = u1 * (1.f / 3.f) - u2 * (7.f / 6.f) + u3 * (11.f / 6.f);
    const float p2 = -u2 * (1.f / 6.f) + u3 * (5.f / 6.f) + u4 * (1.f / 3.f);
    const float p3 = u3 * (1.f / 3.f) + u4 * (5.f / 6.f) - u5 * (1.f / 6.f);
    const float a = u1 - 2.f * u2 + u3, b = u1 - 4.f * u2 + 3.f * u3;
    const float c = u2 - 2.f * u3 + u4, d = u2 - u4;
    const float e = u3 - 2.f * u4 + u5, f = 3.f * u3 - 4.f * u4 + u5;
    const float sr = s * r;
    const float eps = 1e-6f * sr * sr;
    const float t1 = (13.f / 12.f) * a * a + 0.25f * b * b + eps;
    const float t2 = (13.f / 12.f) * c * c + 0.25f * d * d + eps;
    const float t3 = (13.f / 12.f) * e * e + 0.25f * f * f + eps;
    const float q12 = t1 * t2, q13 = t1 * t3, q23 = t2 * t3;
    const float b1 = 0.1f * (q23 * q23), b2 = 0.6f * (q13 * q13), b3 = 0.3f * (q12 * q12);
    return S * __fdividef(b1 * p1 + b2 * p2 + b3 * p3, b1 + b2 + b3);
}

__device__ __forceinline__ float weno_px(const float (*t)[kWTX + 1], int cy, int cx, float F, float dt,
                                         float lam, float mm) {
    const float c = t[cy][cx];
    float out = c;
    if (F != 0.f) {
        float dx[6], dy[6];  // d(k) = phi(k) - phi(k - 1), k = -2 .. 3 relative to the node
#pragma unroll
        for (int k = -2; k <= 3; ++k) {
            dx[k + 2] = t[cy][cx + k] - t[cy][cx + k - 1];
            dy[k + 2] = t[cy + k][cx] - t[cy + k - 1][cx];
        }
        const float dmx = weno5(dx[0], dx[1], dx[2], dx[3], dx[4]);
        const float dpx = weno5(dx[5], dx[4], dx[3], dx[2], dx[1]);
        const float dmy = weno5(dy[0], dy[1], dy[2], dy[3], dy[4]);
        const float dpy = weno5(dy[5], dy[4], dy[3], dy[2], dy[1]);
        const bool pos = F > 0.f;
        const float a = pos ? fmaxf(dmx, 0.f) : fminf(dmx, 0.f);
        const float b = pos ? fminf(dpx, 0.f) : fmaxf(dpx, 0.f);
        const float cc = pos ? fmaxf(dmy, 0.f) : fminf(dmy, 0.f);
        const float d = pos ? fminf(dpy, 0.f) : fmaxf(dpy, 0.f);
        out -= F * sqrt_approx(a * a + b * b + cc * cc + d * d);
    }
    if (lam != 0.f) {
        const float xm = t[cy][cx - 1], xp = t[cy][cx + 1], ym = t[cy - 1][cx], yp = t[cy + 1][cx];
        const float px = 0.5f * (xp - xm), py = 0.5f * (yp - ym);
        const float pxx = xp + xm - 2.f * c, pyy = yp + ym - 2.f * c;
        const float pxy = 0.25f * ((t[cy + 1][cx + 1] - t[cy + 1][cx - 1]) - (t[cy - 1][cx + 1] - t[cy - 1][cx - 1]));
        const float den = px * px + py * py;
        float kc = 0.f;
        if (den >= 1e-12f) kc = __fdividef(pxx * py * py - 2.f * px * py * pxy + pyy * px * px, den);
        out += dt * lam * mm * kc;
    }
    return out;
}

__global__ void __launch_bounds__(kWX * kWTh)
k_levelset_step_weno(const float* __restrict__ phi, const float* __restrict__ V,
                     const double* __restrict__ vmax, const float* __restrict__ m, float dt, float lam,
                     int n, float* __restrict__ phi_out, unsigned char* __restrict__ mask_out,
                     __nv_bfloat16* __restrict__ mask_bf, int ldb) {
    __shared__ float t[kWTY][kWTX + 1];
    __shared__ float s_inv;
    pdl_trigger();
    pdl_wait();
    {  // clip blockIdx.z of a batch
        const size_t c = blockIdx.z, np = (size_t)n * n;
        phi += c * np;
        V += c * np;
        vmax += c;
        if (m) m += c * np;
        if (phi_out) phi_out += c * np;
        if (mask_out) mask_out += c * np;
        if (mask_bf) mask_bf += c * (size_t)n * ldb;
    }
    const int x0 = blockIdx.x * kWX, y0 = blockIdx.y * kWY;
    const int tid = threadIdx.y * kWX + threadIdx.x;
    if (tid == 0) {  // 1 / max|V| once per block (FP64 operand)
        const double vm = *vmax;
        s_inv = vm > 0.0 ? 1.0f / (float)vm : 0.f;
    }
    for (int i = tid; i < kWTX * kWTY; i += kWX * kWTh) {
        const int ty = i / kWTX, tx = i - ty * kWTX;
        const int gy = min(max(y0 + ty - kWH, 0), n - 1), gx = min(max(x0 + tx - kWH, 0), n - 1);
        t[ty][tx] = phi[(size_t)gy * n + gx];
    }
    __syncthreads();
    const float inv = s_inv;
    const int x = x0 + threadIdx.x;
    if (x >= n) return;
#pragma unroll
    for (int r = 0; r < kWY / kWTh; ++r) {
        const int ly = threadIdx.y + r * kWTh, y = y0 + ly;
        if (y >= n) break;
        const size_t p = (size_t)y * n + x;
        const float F = -dt * (V[p] * inv);
        const float out = weno_px(t, ly + kWH, threadIdx.x + kWH, F, dt, lam, m ? m[p] : 1.f);
        if (phi_out) phi_out[p] = out;
        if (mask_out) mask_out[p] = out <= 0.f ? 1 : 0;
        if (mask_bf) mask_bf[(size_t)y * ldb + x] = __float2bfloat16_rn(out <= 0.f ? 1.f : 0.f);
    }
}

// four pixels per thread and step (16-byte loads, 4-byte stores; the arrays are 16-byte
// aligned), then the npix % 4 tail
__global__ void k_mask_from_phi(const float* __restrict__ phi, size_t npix, unsigned char* __restrict__ M) {
    const size_t stride = (size_t)gridDim.x * blockDim.x, nq = npix / 4;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nq; i += stride) {
        const float4 v = reinterpret_cast<const float4*>(phi)[i];
        reinterpret_cast<uchar4*>(M)[i] = make_uchar4(v.x <= 0.f, v.y <= 0.f, v.z <= 0.f, v.w <= 0.f);
    }
    for (size_t i = 4 * nq + (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < npix; i += stride)
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
                         unsigned char* mask_out, __nv_bfloat16* mask_bf, int ldb, cudaStream_t s, int upwind,
                         int B) {
    if (upwind == DEVEL_UPWIND_WENO5) {
        prof_begin(PK_STEP, s);
        cudaError_t e = launch_pdl(k_levelset_step_weno, dim3((n + kWX - 1) / kWX, (n + kWY - 1) / kWY, B),
                                   dim3(kWX, kWTh), 0, s, phi, V, vmax, m, dt, lambda, n, phi_out, mask_out, mask_bf,
                                   ldb);
        prof_end(PK_STEP, s);
        if (e != cudaSuccess) return cuda_error(e, "k_levelset_step_weno");
        return DEVEL_OK;
    }
    dim3 grid((n + 256 * kPX - 1) / (256 * kPX), (n + kRows - 1) / kRows, B);
    prof_begin(PK_STEP, s);
    cudaError_t e = launch_pdl(k_levelset_step, grid, dim3(256), 0, s, phi, V, vmax, m, dt, lambda, n, phi_out,
                               mask_out, mask_bf, ldb);
    prof_end(PK_STEP, s);
    if (e != cudaSuccess) return cuda_error(e, "k_levelset_step");
    return DEVEL_OK;
}

int launch_mask_from_phi(int n, const float* phi, unsigned char* M, cudaStream_t s, int B) {
    const size_t npix = (size_t)n * n * B;
    prof_begin(PK_MASK, s);
    k_mask_from_phi<<<grid_for(npix / 4 + 1), 256, 0, s>>>(phi, npix, M);
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
