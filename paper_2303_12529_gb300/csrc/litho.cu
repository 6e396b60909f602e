// Truncated-DFT lithography kernels, FP32 on the CUDA cores.
//
// Every optical kernel's spectrum is confined to the k x k window W
// (Sec. II-B, SOCS). Then |A_j|^2 and R * A_j are confined to the
// (2k-1) x (2k-1) difference window W2 = W - W, and the forward image and
// the adjoint contract through those windows once, the sum over kernels
// being taken in the frequency domain:
//
//   mhat(a)  = n^-2 sum_p M(p) e^{-i 2pi a.p/n},            a in W
//   Y_j(a)   = sqrt(w_j) H_j(a) mhat(a)
//   Ihat(g)  = sum_j sum_{a - b = g} Y_j(a) conj(Y_j(b)),    g in W2
//   I(p)     = Re sum_g Ihat(g) e^{+i 2pi g.p/n}             (= sum_j w_j |A_j(p)|^2)
//
//   rhat(g)  = n^-2 sum_p R(p) e^{-i 2pi g.p/n},             g in W2
//   Shat(f)  = sum_j conj(sqrt(w_j) H_j(f)) sum_a Y_j(a) rhat(f - a),  f in W
//   V(q)     = 2 Re sum_f Shat(f) e^{+i 2pi f.q/n}           (= dL/dM, Eq. ilt_gradient)
//
// Each 2-D transform is separable: one contraction over image columns with
// a [2kw][n] cos/sin table, then one over rows.
#include <cstdio>

#include "common.cuh"

namespace devel {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a * conj(b)
    return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

// Fixed-order block reduction of a float2 (deterministic).
__device__ float2 block_sum2(float2 v, float2* sh) {
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_down_sync(0xffffffffu, v.x, o);
        v.y += __shfl_down_sync(0xffffffffu, v.y, o);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    float2 t = make_float2(0.f, 0.f);
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        t = lane < nw ? sh[lane] : make_float2(0.f, 0.f);
        for (int o = 16; o > 0; o >>= 1) {
            t.x += __shfl_down_sync(0xffffffffu, t.x, o);
            t.y += __shfl_down_sync(0xffffffffu, t.y, o);
        }
    }
    return t;  // valid in thread 0
}

template <typename T>
__device__ __forceinline__ float as_float(T v) { return static_cast<float>(v); }

// --------------------------------------------------------------------------
// spectrum: row block of TY rows -> partial window spectrum
// --------------------------------------------------------------------------
constexpr int kTY = 16;   // rows per block
constexpr int kXC = 32;   // columns per smem chunk
constexpr int kMaxOut = (kTY * 2 * (2 * kMaxWindow - 1) + kThreads - 1) / kThreads;

template <typename T>
__global__ void __launch_bounds__(kThreads)
k_spectrum_partial(const T* __restrict__ X, int n, const float* __restrict__ basis, int kw,
                   float2* __restrict__ part) {
    extern __shared__ float sm[];
    const int ncol = 2 * kw;
    float* Xs = sm;                        // [kTY][kXC]
    float* Bs = Xs + kTY * kXC;            // [ncol][kXC + 1]
    float* Ps = Bs + ncol * (kXC + 1);     // [kTY][ncol]
    const int tid = threadIdx.x;
    const int y0 = blockIdx.x * kTY;
    const int nout = kTY * ncol;

    float acc[kMaxOut];
#pragma unroll
    for (int j = 0; j < kMaxOut; ++j) acc[j] = 0.f;

    for (int x0 = 0; x0 < n; x0 += kXC) {
        for (int i = tid; i < kTY * kXC; i += kThreads) {
            const int ty = i / kXC, xx = i - ty * kXC;
            const int y = y0 + ty, x = x0 + xx;
            Xs[i] = (y < n && x < n) ? as_float(X[(size_t)y * n + x]) : 0.f;
        }
        for (int i = tid; i < ncol * kXC; i += kThreads) {
            const int c = i / kXC, xx = i - c * kXC;
            const int x = x0 + xx;
            Bs[c * (kXC + 1) + xx] = x < n ? basis[(size_t)c * n + x] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kMaxOut; ++j) {
            const int o = tid + j * kThreads;
            if (o < nout) {
                const int ty = o / ncol, c = o - ty * ncol;
                const float* xr = Xs + ty * kXC;
                const float* br = Bs + c * (kXC + 1);
                float a = acc[j];
#pragma unroll 8
                for (int xx = 0; xx < kXC; ++xx) a = fmaf(xr[xx], br[xx], a);
                acc[j] = a;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < kMaxOut; ++j) {
        const int o = tid + j * kThreads;
        if (o < nout) Ps[o] = acc[j];
    }
    __syncthreads();
    // P(y, b) = sum_x X e^{-i theta_b x} = Pc - i Ps  (Pc = sum X cos, Ps = sum X sin)
    // partial(a, b) = sum_y e^{-i theta_a y} P(y, b)
    for (int o = tid; o < kw * kw; o += kThreads) {
        const int a = o / kw, b = o - a * kw;
        float sr = 0.f, si = 0.f;
        for (int ty = 0; ty < kTY; ++ty) {
            const int y = y0 + ty;
            if (y >= n) break;
            const float ca = basis[(size_t)a * n + y];
            const float sa = basis[(size_t)(kw + a) * n + y];
            const float pc = Ps[ty * ncol + b];
            const float ps = Ps[ty * ncol + kw + b];
            sr = fmaf(ca, pc, fmaf(-sa, ps, sr));
            si = fmaf(-ca, ps, fmaf(-sa, pc, si));
        }
        part[(size_t)blockIdx.x * kw * kw + o] = make_float2(sr, si);
    }
}

__global__ void k_spectrum_reduce(const float2* __restrict__ part, int nblk, int nout, float scale,
                                  float2* __restrict__ out) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= nout) return;
    float2 s = make_float2(0.f, 0.f);
    for (int b = 0; b < nblk; ++b) {
        const float2 v = part[(size_t)b * nout + o];
        s.x += v.x;
        s.y += v.y;
    }
    out[o] = make_float2(s.x * scale, s.y * scale);
}

// --------------------------------------------------------------------------
// frequency-domain SOCS sums
// --------------------------------------------------------------------------
__global__ void k_socs_y(const float2* __restrict__ Hp, const float2* __restrict__ mhat, int K,
                         int kk, float2* __restrict__ Y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= K * kk) return;
    Y[i] = cmul(Hp[i], mhat[i % kk]);
}

// Ihat(g) = sum_j sum_{a in W, a - g in W} Y_j(a) conj(Y_j(a - g)); one block per g.
__global__ void __launch_bounds__(kThreads)
k_hopkins(const float2* __restrict__ Y, int K, int k, float2* __restrict__ Ihat) {
    __shared__ float2 sh[32];
    const int k2 = 2 * k - 1, r2 = k - 1;
    const int g = blockIdx.x;
    const int c1 = g / k2, c2 = g - c1 * k2;
    const int a1lo = max(0, c1 - r2), a1hi = min(k, c1 - r2 + k);
    const int a2lo = max(0, c2 - r2), a2hi = min(k, c2 - r2 + k);
    const int n1 = a1hi - a1lo, n2 = a2hi - a2lo;
    const int per = n1 * n2, total = K * per;
    const int kk = k * k;
    float2 acc = make_float2(0.f, 0.f);
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int j = t / per, rem = t - j * per;
        const int i1 = rem / n2, i2 = rem - i1 * n2;
        const int a1 = a1lo + i1, a2 = a2lo + i2;
        const int b1 = a1 - c1 + r2, b2 = a2 - c2 + r2;
        const float2 p = cmulc(Y[j * kk + a1 * k + a2], Y[j * kk + b1 * k + b2]);
        acc.x += p.x;
        acc.y += p.y;
    }
    const float2 s = block_sum2(acc, sh);
    if (threadIdx.x == 0) Ihat[g] = s;
}

// Shat(f) = sum_j conj(Hp_j(f)) sum_a Y_j(a) rhat(f - a); one block per f in W.
__global__ void __launch_bounds__(kThreads)
k_adjoint_window(const float2* __restrict__ Hp, const float2* __restrict__ Y,
                 const float2* __restrict__ rhat, int K, int k, float2* __restrict__ Shat) {
    __shared__ float2 sh[32];
    const int k2 = 2 * k - 1, r2 = k - 1, kk = k * k;
    const int f = blockIdx.x;
    const int f1 = f / k, f2 = f - f1 * k;
    float2 acc = make_float2(0.f, 0.f);
    for (int t = threadIdx.x; t < K * kk; t += blockDim.x) {
        const int j = t / kk, a = t - j * kk;
        const int a1 = a / k, a2 = a - a1 * k;
        const float2 u = cmul(Y[t], rhat[(f1 - a1 + r2) * k2 + (f2 - a2 + r2)]);
        const float2 p = cmulc(u, Hp[j * kk + f]);
        acc.x += p.x;
        acc.y += p.y;
    }
    const float2 s = block_sum2(acc, sh);
    if (threadIdx.x == 0) Shat[f] = s;
}

// --------------------------------------------------------------------------
// expansion: Acat = [Re T | -Im T], T(y, b) = sum_a e^{+i theta_a y} Z(a, b)
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads)
k_expand_T(const float2* __restrict__ Z, const float* __restrict__ basis, int n, int kw,
           float* __restrict__ Acat) {
    const int ly = threadIdx.x & 31, lb = threadIdx.x >> 5;  // 32 rows x 8 lanes over b
    const int y = blockIdx.x * 32 + ly;
    if (y >= n) return;
    for (int b = lb; b < kw; b += 8) {
        float tr = 0.f, ti = 0.f;
        for (int a = 0; a < kw; ++a) {
            const float ca = basis[(size_t)a * n + y];
            const float sa = basis[(size_t)(kw + a) * n + y];
            const float2 z = Z[a * kw + b];
            tr = fmaf(ca, z.x, fmaf(-sa, z.y, tr));
            ti = fmaf(ca, z.y, fmaf(sa, z.x, ti));
        }
        Acat[(size_t)y * 2 * kw + b] = tr;
        Acat[(size_t)y * 2 * kw + kw + b] = -ti;
    }
}

// out[y][x] = mult * sum_c Acat[y][c] B[c][x], B = basis [2kw][n]; optional block max |out|.
constexpr int kBM = 64, kBN = 64, kBK = 16;

__global__ void __launch_bounds__(kThreads)
k_expand_gemm(const float* __restrict__ A, const float* __restrict__ B, int n, int kc, float mult,
              float* __restrict__ out, float* __restrict__ vpart) {
    __shared__ float As[kBK][kBM + 4];
    __shared__ float Bs[kBK][kBN + 4];
    __shared__ float red[kThreads / 32];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int y0 = blockIdx.y * kBM, x0 = blockIdx.x * kBN;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

    for (int c0 = 0; c0 < kc; c0 += kBK) {
        for (int i = tid; i < kBK * kBM; i += kThreads) {
            const int m = i / kBK, kk = i - m * kBK;
            const int y = y0 + m, c = c0 + kk;
            As[kk][m] = (y < n && c < kc) ? A[(size_t)y * kc + c] : 0.f;
        }
        for (int i = tid; i < kBK * kBN; i += kThreads) {
            const int kk = i / kBN, xx = i - kk * kBN;
            const int x = x0 + xx, c = c0 + kk;
            Bs[kk][xx] = (x < n && c < kc) ? B[(size_t)c * n + x] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kBK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    float mx = 0.f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int y = y0 + ty + 16 * i;
        if (y >= n) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int x = x0 + tx + 16 * j;
            if (x >= n) continue;
            const float v = acc[i][j] * mult;
            out[(size_t)y * n + x] = v;
            mx = fmaxf(mx, fabsf(v));
        }
    }
    if (vpart) {
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
        if ((tid & 31) == 0) red[tid >> 5] = mx;
        __syncthreads();
        if (tid == 0) {
            float m = red[0];
            for (int w = 1; w < kThreads / 32; ++w) m = fmaxf(m, red[w]);
            vpart[blockIdx.y * gridDim.x + blockIdx.x] = m;
        }
    }
}

__global__ void k_vmax_final(const float* __restrict__ vpart, int nparts, double* vmax, int* status) {
    __shared__ float red[32];
    float m = 0.f;
    bool bad = false;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
        const float v = vpart[i];
        if (!(v == v) || isinf(v)) bad = true;  // NaN or Inf
        m = fmaxf(m, v);
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    bad = __syncthreads_or(bad);
    if (threadIdx.x == 0) {
        float r = red[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) r = fmaxf(r, red[w]);
        *vmax = (double)r;
        if (bad && status) *status = DEVEL_ENAN;
    }
}

template <typename T>
int spectrum_impl(const devel_optics* o, const T* X, const float* basis, int kw, float2* out,
                  float scale, cudaStream_t s) {
    const int n = o->n;
    const int nblk = (n + kTY - 1) / kTY;
    const size_t smem = sizeof(float) * (kTY * kXC + 2 * kw * (kXC + 1) + kTY * 2 * kw);
    static bool attr_set = false;
    if (!attr_set) {
        DEVEL_CUDA_TRY(cudaFuncSetAttribute(k_spectrum_partial<T>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024));
        attr_set = true;
    }
    prof_begin(PK_SPECTRUM, s);
    k_spectrum_partial<T><<<nblk, kThreads, smem, s>>>(X, n, basis, kw, o->ws.part);
    prof_end(PK_SPECTRUM, s);
    DEVEL_LAUNCH_CHECK("k_spectrum_partial");
    const int nout = kw * kw;
    prof_begin(PK_SPECTRUM_REDUCE, s);
    k_spectrum_reduce<<<(nout + 255) / 256, 256, 0, s>>>(o->ws.part, nblk, nout, scale, out);
    prof_end(PK_SPECTRUM_REDUCE, s);
    DEVEL_LAUNCH_CHECK("k_spectrum_reduce");
    return DEVEL_OK;
}

}  // namespace

int launch_spectrum_f32(const devel_optics* o, const float* X, const float* basis, int kw,
                        float2* out, float scale, cudaStream_t s) {
    return spectrum_impl<float>(o, X, basis, kw, out, scale, s);
}
int launch_spectrum_u8(const devel_optics* o, const unsigned char* X, const float* basis, int kw,
                       float2* out, float scale, cudaStream_t s) {
    return spectrum_impl<unsigned char>(o, X, basis, kw, out, scale, s);
}

int launch_socs_y(const devel_optics* o, cudaStream_t s) {
    const int kk = o->k * o->k;
    prof_begin(PK_SOCS_Y, s);
    k_socs_y<<<(o->K * kk + 255) / 256, 256, 0, s>>>(o->Hp, o->ws.mhat, o->K, kk, o->ws.Y);
    prof_end(PK_SOCS_Y, s);
    DEVEL_LAUNCH_CHECK("k_socs_y");
    return DEVEL_OK;
}

int launch_hopkins(const devel_optics* o, cudaStream_t s) {
    prof_begin(PK_HOPKINS, s);
    k_hopkins<<<o->k2 * o->k2, kThreads, 0, s>>>(o->ws.Y, o->K, o->k, o->ws.Ihat);
    prof_end(PK_HOPKINS, s);
    DEVEL_LAUNCH_CHECK("k_hopkins");
    return DEVEL_OK;
}

int launch_adjoint_window(const devel_optics* o, cudaStream_t s) {
    prof_begin(PK_ADJ_WINDOW, s);
    k_adjoint_window<<<o->k * o->k, kThreads, 0, s>>>(o->Hp, o->ws.Y, o->ws.rhat, o->K, o->k,
                                                      o->ws.Shat);
    prof_end(PK_ADJ_WINDOW, s);
    DEVEL_LAUNCH_CHECK("k_adjoint_window");
    return DEVEL_OK;
}

int launch_expand(const devel_optics* o, const float2* Z, const float* basis, int kw, float* out,
                  float mult, bool want_max, cudaStream_t s) {
    const int n = o->n;
    prof_begin(PK_EXPAND_T, s);
    k_expand_T<<<(n + 31) / 32, kThreads, 0, s>>>(Z, basis, n, kw, o->ws.Acat);
    prof_end(PK_EXPAND_T, s);
    DEVEL_LAUNCH_CHECK("k_expand_T");
    dim3 grid((n + kBN - 1) / kBN, (n + kBM - 1) / kBM);
    prof_begin(PK_EXPAND_GEMM, s);
    k_expand_gemm<<<grid, kThreads, 0, s>>>(o->ws.Acat, basis, n, 2 * kw, mult, out,
                                            want_max ? o->ws.vpart : nullptr);
    prof_end(PK_EXPAND_GEMM, s);
    DEVEL_LAUNCH_CHECK("k_expand_gemm");
    return DEVEL_OK;
}

int launch_vmax_final(const devel_optics* o, double* vmax, int* status, cudaStream_t s) {
    const int n = o->n;
    const int nparts = ((n + kBN - 1) / kBN) * ((n + kBM - 1) / kBM);
    prof_begin(PK_VMAX, s);
    k_vmax_final<<<1, 1024, 0, s>>>(o->ws.vpart, nparts, vmax, status);
    prof_end(PK_VMAX, s);
    DEVEL_LAUNCH_CHECK("k_vmax_final");
    return DEVEL_OK;
}

int expand_parts(int n) { return ((n + kBN - 1) / kBN) * ((n + kBM - 1) / kBM); }

}  // namespace devel
