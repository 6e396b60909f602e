// Truncated-DFT lithography, FP32 on the CUDA cores.
//
// Every optical kernel's spectrum is confined to the k x k window W
// (Sec. II-B, SOCS). Then |A_j|^2 and R * A_j are confined to the
// (2k-1) x (2k-1) difference window W2 = W - W, and the forward image and
// the adjoint contract through those windows once; the sum over the K
// kernels is carried by the rank-K transmission cross coefficient
// TCC_K(a, b) = sum_j w_j H_j(a) conj(H_j(b)) (Hopkins, Sec. II-B), formed
// once per optics handle:
//
//   mhat(a)  = n^-2 sum_p M(p) e^{-i 2pi a.p/n},             a in W
//   Ihat(g)  = sum_{a - b = g} TCC_K(a, b) mhat(a) conj(mhat(b)),  g in W2
//   I(p)     = Re sum_g Ihat(g) e^{+i 2pi g.p/n}              (= sum_j w_j |A_j(p)|^2)
//
//   rhat(g)  = n^-2 sum_p R(p) e^{-i 2pi g.p/n},              g in W2
//   Shat(f)  = sum_a conj(TCC_K(f, a)) mhat(a) rhat(f - a),   f in W
//   V(q)     = 2 Re sum_f Shat(f) e^{+i 2pi f.q/n}            (= dL/dM, Eq. ilt_gradient)
//
// The n^2-sized work is four separable contractions, all run by one
// register-tiled NT GEMM (C = A B^T, both operands K-major):
//   reduction onto a window of side kw:  P = X basis^T          (K = n, split-K)
//                                         Xhat = E* P           (per row block)
//   expansion from a window:             T = G Bmat^T           (K = 2kw)
//                                         out = T basisT^T      (K = 2kw)
// with basis[c][x] = cos / sin(2 pi (a - r) x / n) (c = a, kw + a) and
// basisT its transpose, zero-padded to ldk = round_up(2kw, 16) columns.
#include "common.cuh"
#include "tc.cuh"

namespace devel {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {  // a * conj(b)
    return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }

// Fixed-order block reduction of a float2 (deterministic); valid in thread 0.
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
    return t;
}

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(unsigned char v) { return v ? 1.f : 0.f; }

// --------------------------------------------------------------------------
// NT GEMM: C[m][nn] = scale * sum_k A[m][k] B[nn][k]
//   tile 128 x 64 x 16, 256 threads, 8 x 4 outputs per thread,
//   register prefetch of the next k-slab; split-K over gridDim.z.
// --------------------------------------------------------------------------
constexpr int gBM = 128, gBN = 64, gBK = 16;
enum { EPI_STORE = 0, EPI_VEL = 1 };

template <typename TA, int EPI>
__global__ void __launch_bounds__(kThreads)
k_gemm_nt(const TA* __restrict__ A, int lda, const float* __restrict__ B, int ldb, int M, int N,
          int K, int kchunk, float scale, float* __restrict__ C, int ldc, size_t split_stride,
          float* __restrict__ vpart) {
    __shared__ float As[gBK][gBM + 4];
    __shared__ float Bs[gBK][gBN + 4];
    __shared__ float red[kThreads / 32];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.y * gBM, n0 = blockIdx.x * gBN;
    const int kb = blockIdx.z * kchunk;
    const int ke = min(K, kb + kchunk);

    float acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

    float ra[8], rb[4];
    auto load = [&](int k0) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int e = tid + i * kThreads, r = e >> 4, kk = e & 15;
            const int m = m0 + r, k = k0 + kk;
            ra[i] = (m < M && k < ke) ? to_f(A[(size_t)m * lda + k]) : 0.f;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int e = tid + i * kThreads, r = e >> 4, kk = e & 15;
            const int nn = n0 + r, k = k0 + kk;
            rb[i] = (nn < N && k < ke) ? B[(size_t)nn * ldb + k] : 0.f;
        }
    };
    if (kb < ke) load(kb);
    for (int k0 = kb; k0 < ke; k0 += gBK) {
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int e = tid + i * kThreads;
            As[e & 15][e >> 4] = ra[i];
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int e = tid + i * kThreads;
            Bs[e & 15][e >> 4] = rb[i];
        }
        __syncthreads();
        if (k0 + gBK < ke) load(k0 + gBK);
#pragma unroll
        for (int kk = 0; kk < gBK; ++kk) {
            float a[8], b[4];
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    float* Cz = C + blockIdx.z * split_stride;
    float mx = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int m = m0 + ty + 16 * i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int nn = n0 + tx + 16 * j;
            if (nn >= N) continue;
            const float v = acc[i][j] * scale;
            Cz[(size_t)m * ldc + nn] = v;
            if (EPI == EPI_VEL) mx = fmaxf(mx, fabsf(v));
        }
    }
    if (EPI == EPI_VEL) {
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

// --------------------------------------------------------------------------
// reduction, second stage: row block of kTY rows, all kw x kw outputs
//   part[blk][a][b] = sum_{y in blk} e^{-i theta_a y} P(y, b),
//   P(y, b) = Pc - i Ps, Pc/Ps summed over the split-K slices in order.
// --------------------------------------------------------------------------
constexpr int kTY = 16;

__global__ void __launch_bounds__(kThreads)
k_spec_stage2(const float* __restrict__ Ppart, int nsplit, size_t sstride, int ldp, int n,
              const float* __restrict__ basis, int kw, float2* __restrict__ part) {
    extern __shared__ float sm[];
    float* Pc = sm;               // [kTY][kw]
    float* Ps = Pc + kTY * kw;    // [kTY][kw]
    float* Ca = Ps + kTY * kw;    // [kw][kTY]
    float* Sa = Ca + kw * kTY;    // [kw][kTY]
    const int y0 = blockIdx.x * kTY;
    const int rows = min(kTY, n - y0);
    for (int i = threadIdx.x; i < kTY * kw; i += blockDim.x) {
        const int ty = i / kw, b = i - ty * kw;
        float c = 0.f, s = 0.f;
        if (ty < rows) {
            const float* p = Ppart + (size_t)(y0 + ty) * ldp;
            for (int z = 0; z < nsplit; ++z) {
                c += p[z * sstride + b];
                s += p[z * sstride + kw + b];
            }
        }
        Pc[i] = c;
        Ps[i] = s;
    }
    for (int i = threadIdx.x; i < kw * kTY; i += blockDim.x) {
        const int a = i / kTY, ty = i - a * kTY;
        const bool ok = ty < rows;
        Ca[i] = ok ? basis[(size_t)a * n + y0 + ty] : 0.f;
        Sa[i] = ok ? basis[(size_t)(kw + a) * n + y0 + ty] : 0.f;
    }
    __syncthreads();
    // e^{-i ta y} (Pc - i Ps) = (ca Pc - sa Ps) - i (ca Ps + sa Pc)
    for (int o = threadIdx.x; o < kw * kw; o += blockDim.x) {
        const int a = o / kw, b = o - a * kw;
        float sr = 0.f, si = 0.f;
#pragma unroll 4
        for (int ty = 0; ty < kTY; ++ty) {
            const float ca = Ca[a * kTY + ty], sa = Sa[a * kTY + ty];
            const float pc = Pc[ty * kw + b], ps = Ps[ty * kw + b];
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
    for (int b = 0; b < nblk; ++b) s = cadd(s, part[(size_t)b * nout + o]);
    out[o] = make_float2(s.x * scale, s.y * scale);
}

// --------------------------------------------------------------------------
// frequency-domain sums with the rank-K TCC
// --------------------------------------------------------------------------
// Ihat(g) = sum_{a in rect(g)} Tdiff[off(g) + t] mhat(a) conj(mhat(a - g)), one block per g;
// rect(g) = {a in W : a - g in W}, t = row-major index within rect(g).
__global__ void __launch_bounds__(kThreads)
k_ihat_tcc(const float2* __restrict__ Tdiff, const int* __restrict__ goff,
           const float2* __restrict__ mhat, int k, float2* __restrict__ Ihat) {
    extern __shared__ float2 ms[];  // [k*k] mhat, then 32 for the reduction
    const int k2 = 2 * k - 1, r2 = k - 1, kk = k * k;
    for (int i = threadIdx.x; i < kk; i += blockDim.x) ms[i] = mhat[i];
    __syncthreads();
    const int g = blockIdx.x;
    const int c1 = g / k2, c2 = g - c1 * k2;
    const int a1lo = max(0, c1 - r2), a1hi = min(k, c1 - r2 + k);
    const int a2lo = max(0, c2 - r2), a2hi = min(k, c2 - r2 + k);
    const int n2 = a2hi - a2lo, total = (a1hi - a1lo) * n2;
    const float2* T = Tdiff + goff[g];
    float2 acc = make_float2(0.f, 0.f);
    for (int t = threadIdx.x; t < total; t += blockDim.x) {
        const int i1 = t / n2, i2 = t - i1 * n2;
        const int a1 = a1lo + i1, a2 = a2lo + i2;
        const int b1 = a1 - c1 + r2, b2 = a2 - c2 + r2;
        acc = cadd(acc, cmul(T[t], cmulc(ms[a1 * k + a2], ms[b1 * k + b2])));
    }
    const float2 s = block_sum2(acc, ms + kk);
    if (threadIdx.x == 0) Ihat[g] = s;
}

// Shat(f) = sum_{a in W} conj(TCC[f][a]) mhat(a) rhat(f - a), one block per f.
__global__ void __launch_bounds__(kThreads)
k_shat_tcc(const float2* __restrict__ TCC, const float2* __restrict__ mhat,
           const float2* __restrict__ rhat, int k, float2* __restrict__ Shat) {
    __shared__ float2 sh[32];
    const int k2 = 2 * k - 1, r2 = k - 1, kk = k * k;
    const int f = blockIdx.x, f1 = f / k, f2 = f - f1 * k;
    const float2* row = TCC + (size_t)f * kk;
    float2 acc = make_float2(0.f, 0.f);
    for (int a = threadIdx.x; a < kk; a += blockDim.x) {
        const int a1 = a / k, a2 = a - a1 * k;
        const float2 u = cmul(mhat[a], rhat[(f1 - a1 + r2) * k2 + (f2 - a2 + r2)]);
        acc = cadd(acc, cmulc(u, row[a]));
    }
    const float2 s = block_sum2(acc, sh);
    if (threadIdx.x == 0) Shat[f] = s;
}

// Bmat [ldk][ldk] such that T = G Bmat^T gives [Re T | -Im T] with
// T(y, b) = sum_a e^{+i theta_a y} Z(a, b) and G = [cos | sin] (basisT):
//   row b:      [ Zr(:, b) | -Zi(:, b) ]      row kw + b: [ -Zi(:, b) | -Zr(:, b) ]
__global__ void k_build_bmat(const float2* __restrict__ Z, int kw, int ldk, float* __restrict__ Bm) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ldk * ldk) return;
    const int cp = i / ldk, c = i - cp * ldk;
    float v = 0.f;
    if (cp < 2 * kw && c < 2 * kw) {
        const int b = cp < kw ? cp : cp - kw;
        const int a = c < kw ? c : c - kw;
        const float2 z = Z[a * kw + b];
        if (cp < kw) v = c < kw ? z.x : -z.y;
        else v = c < kw ? -z.y : -z.x;
    }
    Bm[i] = v;
}

__global__ void k_vmax_final(const float* __restrict__ vpart, int nparts, double* vmax, int* status) {
    __shared__ float red[32];
    float m = 0.f;
    bool bad = false;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
        const float v = vpart[i];
        if (!(v == v) || isinf(v)) bad = true;
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

constexpr int kTcSplitK = 256;  // K slice of one split of the tensor-core reduction

int tc_operand_f32(const devel_optics* o, const float* X, cudaStream_t s) {
    return tc::launch_split(X, o->n, o->n, o->n, o->ldn, o->Xhi, o->Xlo, s);
}
int tc_operand_f32(const devel_optics* o, const unsigned char* M, cudaStream_t s) {
    return tc::launch_mask_bf16(M, o->n, o->ldn, o->Xhi, s);
}

template <typename TA>
int spectrum_impl(const devel_optics* o, const TA* X, const Window& w, float2* out, cudaStream_t s) {
    const int n = o->n;
    const Workspace& ws = o->ws;
    const int nsplit = o->nsplit;
    const size_t sstride = (size_t)n * w.ldk;
    if (o->precision == DEVEL_PREC_BF16X3) {
        int rc = tc_operand_f32(o, X, s);
        if (rc) return rc;
        const TcWindow& tw = (&w == &o->W) ? o->tcW : o->tcW2;
        tc::Operands op{&o->m_X_hi, &o->m_X_lo, &tw.m_basis_hi, &tw.m_basis_lo, sizeof(TA) == 4 ? 1 : 0};
        rc = tc::launch_gemm(op, w.ldk, false, PK_TC_SPECTRUM, n, w.ldk, o->ldn, kTcSplitK, 1.0f, ws.Ppart,
                             w.ldk, sstride, nullptr, o->tc_err, s);
        if (rc) return rc;
    } else {
        const int kchunk = ((n + nsplit - 1) / nsplit + gBK - 1) / gBK * gBK;
        dim3 grid((w.ldk + gBN - 1) / gBN, (n + gBM - 1) / gBM, nsplit);
        prof_begin(PK_SPECTRUM, s);
        k_gemm_nt<TA, EPI_STORE><<<grid, kThreads, 0, s>>>(X, n, w.basis, n, n, w.ldk, n, kchunk, 1.0f,
                                                            ws.Ppart, w.ldk, sstride, nullptr);
        prof_end(PK_SPECTRUM, s);
        DEVEL_LAUNCH_CHECK("k_gemm_nt(spectrum)");
    }
    const int nblk = (n + kTY - 1) / kTY;
    const size_t smem = sizeof(float) * 4 * kTY * w.kw;
    prof_begin(PK_SPECTRUM_STAGE2, s);
    k_spec_stage2<<<nblk, kThreads, smem, s>>>(ws.Ppart, nsplit, sstride, w.ldk, n, w.basis, w.kw, ws.part);
    prof_end(PK_SPECTRUM_STAGE2, s);
    DEVEL_LAUNCH_CHECK("k_spec_stage2");
    const int nout = w.kw * w.kw;
    const float scale = 1.0f / ((float)n * (float)n);
    prof_begin(PK_SPECTRUM_REDUCE, s);
    k_spectrum_reduce<<<(nout + 255) / 256, 256, 0, s>>>(ws.part, nblk, nout, scale, out);
    prof_end(PK_SPECTRUM_REDUCE, s);
    DEVEL_LAUNCH_CHECK("k_spectrum_reduce");
    return DEVEL_OK;
}

}  // namespace

int spectrum_blocks(int n) { return (n + kTY - 1) / kTY; }

int launch_spectrum_f32(const devel_optics* o, const float* X, const Window& w, float2* out, cudaStream_t s) {
    return spectrum_impl<float>(o, X, w, out, s);
}
int launch_spectrum_u8(const devel_optics* o, const unsigned char* X, const Window& w, float2* out,
                       cudaStream_t s) {
    return spectrum_impl<unsigned char>(o, X, w, out, s);
}

int launch_ihat(const devel_optics* o, cudaStream_t s) {
    const int kk = o->k * o->k;
    prof_begin(PK_HOPKINS, s);
    k_ihat_tcc<<<o->k2 * o->k2, kThreads, sizeof(float2) * (kk + 32), s>>>(o->Tdiff, o->goff, o->ws.mhat,
                                                                           o->k, o->ws.Ihat);
    prof_end(PK_HOPKINS, s);
    DEVEL_LAUNCH_CHECK("k_ihat_tcc");
    return DEVEL_OK;
}

int launch_shat(const devel_optics* o, cudaStream_t s) {
    prof_begin(PK_ADJ_WINDOW, s);
    k_shat_tcc<<<o->k * o->k, kThreads, 0, s>>>(o->TCC, o->ws.mhat, o->ws.rhat, o->k, o->ws.Shat);
    prof_end(PK_ADJ_WINDOW, s);
    DEVEL_LAUNCH_CHECK("k_shat_tcc");
    return DEVEL_OK;
}

int launch_expand(const devel_optics* o, const float2* Z, const Window& w, float* out, float mult,
                  bool want_max, int* nparts, cudaStream_t s) {
    const int n = o->n;
    const Workspace& ws = o->ws;
    prof_begin(PK_EXPAND_T, s);
    k_build_bmat<<<(w.ldk * w.ldk + 255) / 256, 256, 0, s>>>(Z, w.kw, w.ldk, ws.Bmat);
    DEVEL_LAUNCH_CHECK("k_build_bmat");
    dim3 gT((w.ldk + gBN - 1) / gBN, (n + gBM - 1) / gBM, 1);
    k_gemm_nt<float, EPI_STORE><<<gT, kThreads, 0, s>>>(w.basisT, w.ldk, ws.Bmat, w.ldk, n, w.ldk, w.ldk,
                                                         w.ldk, 1.0f, ws.Acat, w.ldk, 0, nullptr);
    prof_end(PK_EXPAND_T, s);
    DEVEL_LAUNCH_CHECK("k_gemm_nt(T)");
    if (o->precision == DEVEL_PREC_BF16X3) {
        int rc = tc::launch_split(ws.Acat, n, w.ldk, w.ldk, w.ldk, o->Acat_hi, o->Acat_lo, s);
        if (rc) return rc;
        const TcWindow& tw = (&w == &o->W) ? o->tcW : o->tcW2;
        tc::Operands op{&tw.m_acat_hi, &tw.m_acat_lo, &tw.m_basisT_hi, &tw.m_basisT_lo, 1};
        const int kps = (w.ldk + 63) / 64 * 64;
        if (nparts) *nparts = ((n + 127) / 128) * ((n + 127) / 128);
        return tc::launch_gemm(op, 128, want_max, PK_TC_EXPAND, n, n, w.ldk, kps, mult, out, n, 0,
                               want_max ? ws.vpart : nullptr, o->tc_err, s);
    }
    if (nparts) *nparts = expand_parts(n);
    dim3 g((n + gBN - 1) / gBN, (n + gBM - 1) / gBM, 1);
    prof_begin(PK_EXPAND_GEMM, s);
    if (want_max)
        k_gemm_nt<float, EPI_VEL><<<g, kThreads, 0, s>>>(ws.Acat, w.ldk, w.basisT, w.ldk, n, n, w.ldk, w.ldk,
                                                          mult, out, n, 0, ws.vpart);
    else
        k_gemm_nt<float, EPI_STORE><<<g, kThreads, 0, s>>>(ws.Acat, w.ldk, w.basisT, w.ldk, n, n, w.ldk,
                                                            w.ldk, mult, out, n, 0, nullptr);
    prof_end(PK_EXPAND_GEMM, s);
    DEVEL_LAUNCH_CHECK("k_gemm_nt(expand)");
    return DEVEL_OK;
}

int expand_parts(int n) { return ((n + gBN - 1) / gBN) * ((n + gBM - 1) / gBM); }

int launch_vmax_final(const devel_optics* o, int nparts, double* vmax, int* status, cudaStream_t s) {
    prof_begin(PK_VMAX, s);
    k_vmax_final<<<1, 1024, 0, s>>>(o->ws.vpart, nparts, vmax, status);
    prof_end(PK_VMAX, s);
    DEVEL_LAUNCH_CHECK("k_vmax_final");
    return DEVEL_OK;
}

}  // namespace devel
