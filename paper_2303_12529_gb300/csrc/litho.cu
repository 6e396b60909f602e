// Truncated-DFT lithography through the difference window.
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
// Tables: basis[c][x] = cos / sin(2 pi (a - r) x / n) for c = a, kw + a,
// zero-padded to ldk = round_up(2 kw, 16) rows; basisT its transpose.
//
// Reduction of an n x n image X onto a window (two contractions):
//   1. P^T = basis X^T  (split-K over x; FP32 NT GEMM, or the tcgen05 GEMM
//      with a transposed store),  P^T[c][y] = sum_x basis[c][x] X[y][x]
//   2. Q = basis P      (split-K over y; FP32 NT GEMM summing the slices of 1)
//   3. Xhat(a,b) = n^-2 [(Q[a][b] - Q[kw+a][kw+b]) - i (Q[a][kw+b] + Q[kw+a][b])]
// Expansion of a window spectrum Z into an n x n image:
//   1. T(y, b) = sum_a e^{+i theta_a y} Z(a, b), stored as Acat = [Re T | -Im T]
//   2. out = Acat basisT^T   (FP32 NT GEMM or tcgen05), with a fused epilogue:
//      plain store, velocity (x2, max |.|) or the resist loss (dL/dI).
// The tensor-core path runs both on folded tables (one cosine row per |frequency| and
// one sine row per nonzero |frequency|, kw rows instead of 2 kw): the reduction's
// second contraction then yields cos / sin products at |u1|, |u2|, from which every
// entry (+-u1, +-u2) is formed with signs (real image: cos is even, sin odd), and the
// expansion's operand folds T at +-u2 into one cosine and one sine column.
#include <algorithm>
#include <cfloat>

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

__device__ __forceinline__ float2 warp_sum2(float2 v) {
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_down_sync(0xffffffffu, v.x, o);
        v.y += __shfl_down_sync(0xffffffffu, v.y, o);
    }
    return v;
}

// L2 prefetch of the 128-byte line holding p
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(unsigned char v) { return v ? 1.f : 0.f; }

// --------------------------------------------------------------------------
// FP32 GEMM: C[m][nn] = scale * sum_k A[m][k] B(k, nn), A K-major; B K-major
// (B[nn][k], BN_MAJOR = false) or N-major (B[k][nn], BN_MAJOR = true).
//   tile 128 x 64 x 16, 256 threads, 8 x 4 outputs per thread, register
//   prefetch of the next k-slab; split-K over gridDim.z.
// --------------------------------------------------------------------------
constexpr int gBM = 128, gBN = 64, gBK = 16;

template <typename TA, typename TB, int EPI, bool BN_MAJOR>
__global__ void __launch_bounds__(kThreads)
k_gemm_nt(const TA* __restrict__ A, int lda, const TB* __restrict__ B, int ldb, int M, int N, int K, int kchunk,
          EpiArgs ep) {
    __shared__ float As[gBK][gBM + 4];
    __shared__ float Bs[gBK][gBN + 4];
    __shared__ float red[kThreads / 32];
    pdl_trigger();
    pdl_wait();
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
            const int e = tid + i * kThreads;
            // K-major B: consecutive threads walk k; N-major B: consecutive threads walk nn
            const int r = BN_MAJOR ? (e & 63) : (e >> 4), kk = BN_MAJOR ? (e >> 6) : (e & 15);
            const int nn = n0 + r, k = k0 + kk;
            rb[i] = (nn < N && k < ke) ? to_f(BN_MAJOR ? B[(size_t)k * ldb + nn] : B[(size_t)nn * ldb + k]) : 0.f;
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
            if (BN_MAJOR) Bs[e >> 6][e & 63] = rb[i];
            else Bs[e & 15][e >> 4] = rb[i];
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
    float* Cz = ep.C + blockIdx.z * ep.split_stride;
    int mxi = 0;  // max |out| as a float bit pattern: a NaN or inf exceeds every finite value
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int m = m0 + ty + 16 * i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int nn = n0 + tx + 16 * j;
            if (nn >= N) continue;
            const float v = acc[i][j] * ep.scale;
            Cz[(size_t)m * ep.ldc + nn] = v;
            if (EPI == EPI_VEL) mxi = max(mxi, __float_as_int(fabsf(v)));
        }
    }
    const int part = blockIdx.y * gridDim.x + blockIdx.x;
    if (EPI == EPI_VEL) {
        for (int o = 16; o > 0; o >>= 1) mxi = max(mxi, __shfl_down_sync(0xffffffffu, mxi, o));
        if ((tid & 31) == 0) red[tid >> 5] = __int_as_float(mxi);
        __syncthreads();
        if (tid == 0) {
            int m = __float_as_int(red[0]);
            for (int w = 1; w < kThreads / 32; ++w) m = max(m, __float_as_int(red[w]));
            ep.vpart[part] = __int_as_float(m);
        }
        vmax_last_block(ep.vpart, gridDim.x * gridDim.y, ep.counter, ep.vmax, ep.status);
    }
}

// P = sum_z Ppart[z] over the split-K slices of stage 1, elementwise in slice order.
__global__ void k_sum_slices(const float* __restrict__ Ppart, int nz, size_t len, float* __restrict__ P) {
    pdl_trigger();
    pdl_wait();
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += stride) {
        float v = 0.f;
        for (int z = 0; z < nz; ++z) v += Ppart[z * len + i];
        P[i] = v;
    }
}

// Xhat(a, b) = scale [(Q[a][b] - Q[kw+a][kw+b]) - i (Q[a][kw+b] + Q[kw+a][b])], Q summed over
// nq partial slices. Block = (row a, 32 columns b); lane = column, warp w sums slices
// w, w + 16, ... (coalesced row reads, eight slices' loads in flight), then the 16 warp
// sums are added in warp order.
constexpr int kFinWarps = 16;
constexpr int kFinUnroll = 8;
__global__ void __launch_bounds__(32 * kFinWarps)
k_spec_final(const float* __restrict__ Q, int nq, int ldq, int kw, float scale, float2* __restrict__ out) {
    __shared__ float2 part[kFinWarps][32];
    pdl_trigger();
    pdl_wait();
    const int a = blockIdx.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int b = blockIdx.y * 32 + lane;
    float re = 0.f, im = 0.f;
    if (b < kw) {
        const size_t st = (size_t)ldq * ldq;
        const size_t o0 = (size_t)a * ldq + b, o1 = (size_t)(kw + a) * ldq + b;
        int z = w;
        for (; z + (kFinUnroll - 1) * kFinWarps < nq; z += kFinUnroll * kFinWarps) {
            float v[kFinUnroll][4];
#pragma unroll
            for (int u = 0; u < kFinUnroll; ++u) {
                const float* q = Q + (size_t)(z + u * kFinWarps) * st;
                v[u][0] = __ldcg(q + o0);
                v[u][1] = __ldcg(q + o1 + kw);
                v[u][2] = __ldcg(q + o0 + kw);
                v[u][3] = __ldcg(q + o1);
            }
#pragma unroll
            for (int u = 0; u < kFinUnroll; ++u) {
                re += v[u][0] - v[u][1];
                im -= v[u][2] + v[u][3];
            }
        }
        for (; z < nq; z += kFinWarps) {
            const float* q = Q + (size_t)z * st;
            re += __ldcg(q + o0) - __ldcg(q + o1 + kw);
            im -= __ldcg(q + o0 + kw) + __ldcg(q + o1);
        }
    }
    part[w][lane] = make_float2(re, im);
    __syncthreads();
    if (w != 0 || b >= kw) return;
    float2 v = part[0][lane];
    for (int i = 1; i < kFinWarps; ++i) v = cadd(v, part[i][lane]);
    out[a * kw + b] = make_float2(v.x * scale, v.y * scale);
}

void launch_spec_final(const float* Q, int nq, int ldq, int kw, float2* out, int n, cudaStream_t s) {
    const float scale = 1.0f / ((float)n * (float)n);
    prof_begin(PK_SPECTRUM_REDUCE, s);
    launch_pdl(k_spec_final, dim3(kw, (kw + 31) / 32), dim3(32 * kFinWarps), 0, s, Q, nq, ldq, kw, scale, out);
    prof_end(PK_SPECTRUM_REDUCE, s);
}

// --------------------------------------------------------------------------
// frequency-domain sums with the rank-K TCC (one warp per output frequency)
// --------------------------------------------------------------------------

// clips per block of the Hopkins sums (each TCC entry loaded once for all of them). The
// forward sum reads each clip's mhat (k^2 entries, 10 KB at k = 35), so four clips' share
// L1; the adjoint sum also reads rhat ((2k-1)^2 entries, 38 KB), and one clip per block
// keeps its working set in L1 (four per block measured 1.4x slower).
constexpr int kIhatClips = 4, kShatClips = 1;

// Tensor-core path: the four window spectrum entries Z(+-j1, +-j2) folded into the B
// operand of T = E Z over the folded table (rows c(j) = j: cos, s(j) = r + j: sin), as
// bf16 hi/lo [ldz][ldz] (row = output column of T, column = table row):
//   P = Z(j1, j2), Q = Z(j1, -j2), R = Z(-j1, j2), T = Z(-j1, -j2)
// (an entry whose sign flip is the same frequency, j = 0, is counted once). With
// T(y, u2) = sum_u1 e^{+i theta u1 y} Z(u1, u2) and the expansion's operand
// [T(y, j2) + T(y, -j2)] real part on cos rows, -[Im T(y, j2) - Im T(y, -j2)] on sin rows:
//   Zm[c(j2)][c(j1)] = Re (P + Q + R + T)            Zm[c(j2)][s(j1)] = -Im (P - R + Q - T)
//   Zm[s(j2)][c(j1)] = -Im (P - Q + R - T)            Zm[s(j2)][s(j1)] = Re (-P + Q + R - T)
__device__ __forceinline__ void put_zm_folded(__nv_bfloat16* hi, __nv_bfloat16* lo, int ldz, int r, int j1, int j2,
                                              float2 P, float2 Q, float2 R, float2 T) {
    auto put = [&](int row, int col, float x) {
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        hi[(size_t)row * ldz + col] = h;
        lo[(size_t)row * ldz + col] = __float2bfloat16_rn(x - __bfloat162float(h));
    };
    const bool hq = j2 > 0, hr = j1 > 0, ht = hq && hr;
    const float cc = P.x + (hq ? Q.x : 0.f) + (hr ? R.x : 0.f) + (ht ? T.x : 0.f);
    put(j2, j1, cc);
    if (hr) put(j2, r + j1, -((P.y - R.y) + (hq ? Q.y - T.y : 0.f)));
    if (hq) put(r + j2, j1, -((P.y - Q.y) + (hr ? R.y - T.y : 0.f)));
    if (ht) put(r + j2, r + j1, (-P.x + Q.x) + (R.x - T.x));
}

// Ihat(g) = sum_{a in rect(g)} Tdiff[off(g) + t] mhat(a) conj(mhat(a - g)), rect(g) = {a in W :
// a - g in W}, t = row-major index within rect(g). The aerial image is real, so
// Ihat(-g) = conj(Ihat(g)): one block per (j1, j2) in [0, r2]^2 and per CB clips of a batch,
// whose two halves of 128 threads sum g = (j1, j2) and g = (j1, -j2) (the latter when
// j1, j2 > 0) for each of its clips, every TCC entry loaded once for all of them; thread q
// then writes clip q's four entries (+-j1, +-j2), and for the tensor-core path their folded
// operand entries. Each clip's sum runs in the same order whatever CB is.
template <int CB>
__global__ void __launch_bounds__(256)
k_ihat_tcc(const float2* __restrict__ Tdiff, const int* __restrict__ goff,
           const float2* __restrict__ mhat, int k, int B, float2* __restrict__ Ihat, __nv_bfloat16* __restrict__ zhi,
           __nv_bfloat16* __restrict__ zlo, int ldz) {
    __shared__ float2 sh[CB][8];
    const int k2 = 2 * k - 1, r2 = k - 1, kk = k * k;
    const int j1 = blockIdx.x / (r2 + 1), j2 = blockIdx.x - j1 * (r2 + 1);
    const int c0 = blockIdx.y * CB, nc = min(CB, B - c0);
    const int half = threadIdx.x >> 7, tid = threadIdx.x & 127;
    const bool two = j1 > 0 && j2 > 0;
    const int c1 = r2 + j1, c2 = half ? r2 - j2 : r2 + j2;
    const bool active = half == 0 || two;
    const int a1lo = max(0, c1 - r2), a1hi = min(k, c1 - r2 + k);
    const int a2lo = max(0, c2 - r2), a2hi = min(k, c2 - r2 + k);
    const int n2 = a2hi - a2lo, total = (a1hi - a1lo) * n2;
    const float2* T = Tdiff + goff[c1 * k2 + c2];
    // the TCC entries (constant) into L2 while the previous kernel finishes
    pdl_trigger();
    if (active)
        for (int i = tid * 16; i < total; i += 128 * 16) prefetch_l2(T + i);
    pdl_wait();
    const float2* mh = mhat + (size_t)c0 * kk;
    float2 acc[CB];
#pragma unroll
    for (int q = 0; q < CB; ++q) acc[q] = make_float2(0.f, 0.f);
    if (active) {
#pragma unroll 2
        for (int t = tid; t < total; t += 128) {
            const int i1 = t / n2, i2 = t - i1 * n2;
            const int a1 = a1lo + i1, a2 = a2lo + i2;
            const int ia = a1 * k + a2, ib = (a1 - c1 + r2) * k + (a2 - c2 + r2);
            const float2 tv = __ldg(T + t);
#pragma unroll
            for (int q = 0; q < CB; ++q)
                if (q < nc)
                    acc[q] = cadd(acc[q], cmul(tv, cmulc(__ldg(mh + (size_t)q * kk + ia), __ldg(mh + (size_t)q * kk + ib))));
        }
    }
#pragma unroll
    for (int q = 0; q < CB; ++q) {
        const float2 v = warp_sum2(acc[q]);
        if ((threadIdx.x & 31) == 0) sh[q][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < nc) {
        const int q = threadIdx.x;
        const size_t c = (size_t)c0 + q;
        float2* Ih = Ihat + c * k2 * k2;
        const float2 A = cadd(cadd(sh[q][0], sh[q][1]), cadd(sh[q][2], sh[q][3]));
        const float2 Ac = make_float2(A.x, -A.y);
        const int g = c1 * k2 + (r2 + j2);
        Ih[g] = A;
        Ih[k2 * k2 - 1 - g] = Ac;
        float2 Bq = Ac, Bc = Ac;
        if (two) {
            Bq = cadd(cadd(sh[q][4], sh[q][5]), cadd(sh[q][6], sh[q][7]));
            Bc = make_float2(Bq.x, -Bq.y);
            const int gb = c1 * k2 + (r2 - j2);
            Ih[gb] = Bq;
            Ih[k2 * k2 - 1 - gb] = Bc;
        }
        // Q = Ihat(j1, -j2), R = Ihat(-j1, j2) = conj(Q), T = Ihat(-j1, -j2) = conj(A)
        if (zhi)
            put_zm_folded(zhi + c * ldz * ldz, zlo + c * ldz * ldz, ldz, r2, j1, j2, A, j1 > 0 ? Bq : Ac,
                          j2 > 0 ? Bc : Ac, Ac);
    }
}

// Shat(f) = sum_{a in W} conj(TCC[f][a]) mhat(a) rhat(f - a); with a second system (TCC2,
// rhat2: the defocused corner) its term is added. One block per (j1, j2) in [0, r]^2 and
// per CB clips of a batch, whose four groups of 128 threads sum f = (j1, j2), (j1, -j2),
// (-j1, j2), (-j1, -j2) (each sign flip taken only for j > 0) for each of its clips, every
// TCC entry loaded once for all of them; thread q then writes clip q's entries, and for the
// tensor-core path their folded operand entries. Each clip's sum runs in the same order
// whatever CB is.
template <int CB>
__global__ void __launch_bounds__(512)
k_shat_tcc(const float2* __restrict__ TCC, const float2* __restrict__ mhat,
           const float2* __restrict__ rhat, int k, int B, float2* __restrict__ Shat, __nv_bfloat16* __restrict__ zhi,
           __nv_bfloat16* __restrict__ zlo, int ldz, const float2* __restrict__ TCC2,
           const float2* __restrict__ rhat2) {
    __shared__ float2 sh[CB][16];
    const int k2 = 2 * k - 1, r2 = k - 1, kk = k * k, r = (k - 1) / 2, kk2 = k2 * k2;
    const int j1 = blockIdx.x / (r + 1), j2 = blockIdx.x - j1 * (r + 1);
    const int c0 = blockIdx.y * CB, nc = min(CB, B - c0);
    const int grp = threadIdx.x >> 7, tid = threadIdx.x & 127;
    const int s1 = (grp & 2) ? -1 : 1, s2 = (grp & 1) ? -1 : 1;
    const bool active = (s1 > 0 || j1 > 0) && (s2 > 0 || j2 > 0);
    const int f1 = r + s1 * j1, f2 = r + s2 * j2, f = f1 * k + f2;
    const float2* row = TCC + (size_t)f * kk;
    const float2* row2 = TCC2 ? TCC2 + (size_t)f * kk : nullptr;
    pdl_trigger();
    if (active)
        for (int i = tid * 16; i < kk; i += 128 * 16) {
            prefetch_l2(row + i);
            if (row2) prefetch_l2(row2 + i);
        }
    pdl_wait();
    const float2* mh = mhat + (size_t)c0 * kk;
    const float2* rh = rhat + (size_t)c0 * kk2;
    const float2* rh2 = rhat2 ? rhat2 + (size_t)c0 * kk2 : nullptr;
    float2 acc[CB];
#pragma unroll
    for (int q = 0; q < CB; ++q) acc[q] = make_float2(0.f, 0.f);
    if (active) {
#pragma unroll 4
        for (int a = tid; a < kk; a += 128) {
            const int a1 = a / k, a2 = a - a1 * k;
            const int g = (f1 - a1 + r2) * k2 + (f2 - a2 + r2);
            const float2 ta = __ldg(row + a);
            const float2 tb = row2 ? __ldg(row2 + a) : make_float2(0.f, 0.f);
#pragma unroll
            for (int q = 0; q < CB; ++q)
                if (q < nc) {
                    const float2 ma = __ldg(mh + (size_t)q * kk + a);
                    acc[q] = cadd(acc[q], cmulc(cmul(ma, __ldg(rh + (size_t)q * kk2 + g)), ta));
                    if (row2)  // the defocused system's term (its TCC, its dL/dI spectrum, the same mask)
                        acc[q] = cadd(acc[q], cmulc(cmul(ma, __ldg(rh2 + (size_t)q * kk2 + g)), tb));
                }
        }
    }
#pragma unroll
    for (int q = 0; q < CB; ++q) {
        const float2 v = warp_sum2(acc[q]);
        if ((threadIdx.x & 31) == 0) sh[q][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    if (threadIdx.x < nc) {
        const int q = threadIdx.x;
        const size_t c = (size_t)c0 + q;
        float2 res[4];
        for (int g = 0; g < 4; ++g)
            res[g] = cadd(cadd(sh[q][4 * g], sh[q][4 * g + 1]), cadd(sh[q][4 * g + 2], sh[q][4 * g + 3]));
        float2* Sh = Shat + c * kk;
        for (int g = 0; g < 4; ++g) {
            const int t1 = (g & 2) ? -1 : 1, t2 = (g & 1) ? -1 : 1;
            if ((t1 > 0 || j1 > 0) && (t2 > 0 || j2 > 0)) Sh[(r + t1 * j1) * k + (r + t2 * j2)] = res[g];
        }
        if (zhi) put_zm_folded(zhi + c * ldz * ldz, zlo + c * ldz * ldz, ldz, r, j1, j2, res[0], res[1], res[2], res[3]);
    }
}

// FP32 path: T(y, b) = sum_a e^{+i theta_a y} Z(a, b) -> Acat[y] = [Re T | -Im T | 0 ...]
// (ldk columns). A block of 256 threads takes kTRows rows; Z and
// the rows' cos / sin values are staged in shared memory; a warp per row, lane l computes
// the columns b = l, l + 32, ... (and writes the zero padding beyond 2 kw).
constexpr int kTRows = 8;

__global__ void __launch_bounds__(256)
k_expand_T(const float2* __restrict__ Z, const float* __restrict__ basisT, int n, int kw, int ldk,
           float* __restrict__ Af) {
    extern __shared__ float2 zs[];  // [kw * kw] Z, then [kTRows][ldk] floats of basisT
    float* gs = reinterpret_cast<float*>(zs + kw * kw);
    pdl_trigger();
    pdl_wait();
    const int y0 = blockIdx.x * kTRows;
    // stage Z with batches of independent loads in flight (latency, not bandwidth, bound)
    {
        const int nz = kw * kw;
        for (int i0 = threadIdx.x; i0 < nz; i0 += 8 * blockDim.x) {
            float2 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int i = i0 + u * blockDim.x;
                v[u] = i < nz ? __ldg(Z + i) : make_float2(0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int i = i0 + u * blockDim.x;
                if (i < nz) zs[i] = v[u];
            }
        }
        const int ng = kTRows * ldk;
        for (int i0 = threadIdx.x; i0 < ng; i0 += 8 * blockDim.x) {
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int i = i0 + u * blockDim.x;
                const int r = i / ldk, c = i - r * ldk;
                v[u] = i < ng ? __ldg(basisT + (size_t)min(y0 + r, n - 1) * ldk + c) : 0.f;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int i = i0 + u * blockDim.x;
                if (i < ng) gs[i] = v[u];
            }
        }
    }
    __syncthreads();
    const int r = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int y = y0 + r;
    if (y >= n) return;
    const float* g = gs + r * ldk;
    const size_t base = (size_t)y * ldk;
    for (int b = lane; b < ldk - kw; b += 32) {
        float v0 = 0.f, v1 = 0.f;
        if (b < kw) {
            float tr = 0.f, ti = 0.f;
            for (int a = 0; a < kw; ++a) {
                const float2 z = zs[a * kw + b];
                const float c = g[a], s = g[kw + a];
                tr = fmaf(c, z.x, fmaf(-s, z.y, tr));
                ti = fmaf(c, z.y, fmaf(s, z.x, ti));
            }
            v0 = tr;
            v1 = -ti;
        }
        if (b < kw) Af[base + b] = v0;
        Af[base + kw + b] = v1;
    }
}

template <typename TA, typename TB, int EPI, bool BN_MAJOR = false>
int gemm_nt(const TA* A, int lda, const TB* B, int ldb, int M, int N, int K, int splits, const EpiArgs& ep, int kind,
            cudaStream_t s, const char* what) {
    const int kchunk = ((K + splits - 1) / splits + gBK - 1) / gBK * gBK;
    dim3 grid((N + gBN - 1) / gBN, (M + gBM - 1) / gBM, splits);
    prof_begin(kind, s);
    cudaError_t e = launch_pdl(k_gemm_nt<TA, TB, EPI, BN_MAJOR>, grid, dim3(kThreads), 0, s, A, lda, B, ldb, M, N, K,
                               kchunk, ep);
    prof_end(kind, s);
    if (e != cudaSuccess) return cuda_error(e, what);
    return DEVEL_OK;
}

const TcWindow& tc_window(const devel_optics* o, const Window& w) { return (&w == &o->W) ? o->tcW : o->tcW2; }

// stage 1 of the FP32 reduction: P slices in ws.Ppart ([nsplit][n][ldk])
template <typename TX>
int reduce_stage1(const devel_optics* o, const TX* X, const Window& w, cudaStream_t s) {
    const int n = o->n;
    const Workspace& ws = o->ws;
    EpiArgs ep;
    ep.C = ws.Ppart;
    ep.ldc = w.ldk;
    ep.split_stride = (size_t)n * w.ldk;
    ep.scale = 1.0f;
    return gemm_nt<TX, float, EPI_STORE>(X, n, w.basis, n, n, w.ldk, n, o->nsplit, ep, PK_SPECTRUM, s,
                                         "k_gemm_nt(spectrum)");
}

// stages 2-3 of the reduction from the slices P[z][y][c] in ws.Ppart
int reduce_finish(const devel_optics* o, const Window& w, float2* out, cudaStream_t s) {
    const int n = o->n;
    const Workspace& ws = o->ws;
    const size_t len = (size_t)n * w.ldk;
    prof_begin(PK_SPECTRUM_STAGE2, s);
    cudaError_t e = launch_pdl(k_sum_slices, dim3((unsigned)std::min<size_t>((len + 255) / 256, 4 * 148)), dim3(256), 0,
                               s, (const float*)ws.Ppart, o->nsplit, len, ws.P);
    prof_end(PK_SPECTRUM_STAGE2, s);
    if (e != cudaSuccess) return cuda_error(e, "k_sum_slices");
    EpiArgs ep;
    ep.C = ws.Q;
    ep.ldc = w.ldk;
    ep.split_stride = (size_t)w.ldk * w.ldk;
    ep.scale = 1.0f;
    int rc = gemm_nt<float, float, EPI_STORE, true>(w.basis, n, ws.P, w.ldk, w.ldk, w.ldk, n, o->nq, ep,
                                                    PK_SPECTRUM_STAGE2, s, "k_gemm_nt(stage2)");
    if (rc) return rc;
    launch_spec_final(ws.Q, o->nq, w.ldk, w.kw, out, n, s);
    DEVEL_LAUNCH_CHECK("k_spec_final");
    return DEVEL_OK;
}

// tensor-core reduction: both contractions and the complex combination per CTA (bf16
// operand already in Xhi/Xlo), then the sum of the CTAs' partial spectra
int reduce_tc(const devel_optics* o, const Window& w, int use_alo, float2* out, cudaStream_t s) {
    const TcWindow& tw = tc_window(o, w);
    tc::Operands op{&o->m_X_hi, &o->m_X_lo, &tw.m_basis_hi, &tw.m_basis_lo, use_alo};
    return tc::launch_spectrum2(op, &tw.m_basis128_hi, &tw.m_basis128_lo, tw.ldf, w.kw, o->n, o->n, o->ldn,
                                o->tc_split, o->batch, o->ws.Q, out, o->tc_err, s);
}

}  // namespace

int litho_init_attrs() {
    const int big = 200 * 1024;
    DEVEL_CUDA_TRY(cudaFuncSetAttribute(k_expand_T, cudaFuncAttributeMaxDynamicSharedMemorySize, big));
    return DEVEL_OK;
}

int launch_spectrum_f32(const devel_optics* o, const float* X, const Window& w, float2* out, cudaStream_t s) {
    if (o->precision == DEVEL_PREC_BF16X3) {
        int rc = tc::launch_split(X, o->n, o->n, o->n, o->ldn, o->Xhi, o->Xlo, s);
        return rc ? rc : reduce_tc(o, w, 1, out, s);
    }
    int rc = reduce_stage1<float>(o, X, w, s);
    return rc ? rc : reduce_finish(o, w, out, s);
}
int launch_spectrum_u8(const devel_optics* o, const unsigned char* X, const Window& w, float2* out,
                       cudaStream_t s) {
    if (o->precision == DEVEL_PREC_BF16X3) {
        int rc = tc::launch_mask_bf16(X, o->n, o->ldn, o->Xhi, s);
        return rc ? rc : reduce_tc(o, w, 0, out, s);
    }
    int rc = reduce_stage1<unsigned char>(o, X, w, s);
    return rc ? rc : reduce_finish(o, w, out, s);
}

int launch_spectrum_mask_resident(const devel_optics* o, const Window& w, float2* out, cudaStream_t s) {
    return reduce_tc(o, w, 0, out, s);
}

int launch_spectrum_resident(const devel_optics* o, const Window& w, float2* out, cudaStream_t s) {
    return reduce_tc(o, w, 1, out, s);
}

int launch_ihat(const devel_optics* o, cudaStream_t s) {
    prof_begin(PK_HOPKINS, s);
    const bool tcp = o->precision == DEVEL_PREC_BF16X3;
    // one instantiation for every batch size (a clip's arithmetic never depends on it)
    const int chunks = (o->batch + kIhatClips - 1) / kIhatClips;
    cudaError_t e = launch_pdl(k_ihat_tcc<kIhatClips>, dim3(o->k * o->k, chunks), dim3(256), 0, s, (const float2*)o->Tdiff, (const int*)o->goff,
                               (const float2*)o->ws.mhat, o->k, o->batch, o->ws.Ihat,
                               tcp ? o->tcW2.zm_hi : nullptr, tcp ? o->tcW2.zm_lo : nullptr, o->tcW2.ldf);
    prof_end(PK_HOPKINS, s);
    if (e != cudaSuccess) return cuda_error(e, "k_ihat_tcc");
    return DEVEL_OK;
}

int launch_shat(const devel_optics* o, cudaStream_t s, const devel_optics* od) {
    prof_begin(PK_ADJ_WINDOW, s);
    const bool tcp = o->precision == DEVEL_PREC_BF16X3;
    cudaError_t e = launch_pdl(k_shat_tcc<kShatClips>,
                               dim3((o->r + 1) * (o->r + 1), (o->batch + kShatClips - 1) / kShatClips),
                               dim3(512), 0, s, (const float2*)o->TCC, (const float2*)o->ws.mhat,
                               (const float2*)o->ws.rhat, o->k, o->batch, o->ws.Shat,
                               tcp ? o->tcW.zm_hi : nullptr, tcp ? o->tcW.zm_lo : nullptr, o->tcW.ldf,
                               od ? (const float2*)od->TCC : nullptr, od ? (const float2*)od->ws.rhat : nullptr);
    prof_end(PK_ADJ_WINDOW, s);
    if (e != cudaSuccess) return cuda_error(e, "k_shat_tcc");
    return DEVEL_OK;
}

int launch_expand(const devel_optics* o, const float2* Z, const Window& w, int epi, const EpiArgs& ep_in,
                  int* nparts, cudaStream_t s) {
    const int n = o->n;
    const Workspace& ws = o->ws;
    const bool tcp = o->precision == DEVEL_PREC_BF16X3;
    EpiArgs ep = ep_in;
    ep.n = n;
    ep.ldc = n;
    ep.split_stride = 0;
    ep.vpart = ws.vpart;
    if (tcp) {
        const TcWindow& tw = tc_window(o, w);
        // T = E Z on the tensor cores (Z is in tw.zm, written by the Hopkins sum that
        // produced it), as the bf16 hi/lo operand of the expansion
        // a batch: one CTA per 128 rows and clip spans the whole table width (enough CTAs);
        // one clip: 16-column tiles, so that its 128-row blocks spread over more SMs
        const bool wide = o->batch > 1;
        tc::Operands opT{&tw.m_basisT_hi, &tw.m_basisT_lo, wide ? &tw.m_zmw_hi : &tw.m_zm_hi,
                         wide ? &tw.m_zmw_lo : &tw.m_zm_lo, 1};
        EpiArgs et;
        et.Chi = o->Acat_hi;
        et.Clo = o->Acat_lo;
        et.ldh = tw.ldf;
        et.split_stride = (size_t)n * tw.ldf;  // clip stride of the operand
        int rc = tc::launch_gemm_split(opT, wide ? tw.ldf : kTileT, PK_EXPAND_T, n, tw.ldf, tw.ldf, o->batch, et,
                                       o->tc_err, s);
        if (rc) return rc;
        const int bn = o->tc_expand_bn;
        tc::Operands op{&tw.m_acat_hi, &tw.m_acat_lo, bn == 64 ? &tw.m_basisT64_hi : &tw.m_basisT_hi,
                        bn == 64 ? &tw.m_basisT64_lo : &tw.m_basisT_lo, 1};
        if (nparts) *nparts = tc::expand_grid(n, n, bn);
        ep.split_stride = (size_t)n * n;  // clip stride of the output image
        ep.vbits = ws.vbits;
        return tc::launch_expand(op, bn, epi, n, n, tw.ldf, o->batch, ep, o->tc_err, s);
    }
    prof_begin(PK_EXPAND_T, s);
    cudaError_t e = launch_pdl(k_expand_T, dim3((n + kTRows - 1) / kTRows), dim3(256),
                               sizeof(float2) * w.kw * w.kw + sizeof(float) * kTRows * w.ldk, s, Z,
                               (const float*)w.basisT, n, w.kw, w.ldk, ws.Acat);
    prof_end(PK_EXPAND_T, s);
    if (e != cudaSuccess) return cuda_error(e, "k_expand_T");
    if (nparts) *nparts = expand_parts(n);
    if (epi == EPI_VEL)
        return gemm_nt<float, float, EPI_VEL>(ws.Acat, w.ldk, w.basisT, w.ldk, n, n, w.ldk, 1, ep, PK_EXPAND_GEMM,
                                              s, "k_gemm_nt(expand)");
    return gemm_nt<float, float, EPI_STORE>(ws.Acat, w.ldk, w.basisT, w.ldk, n, n, w.ldk, 1, ep, PK_EXPAND_GEMM, s,
                                            "k_gemm_nt(expand)");
}

int expand_parts(int n) { return ((n + gBN - 1) / gBN) * ((n + gBM - 1) / gBM); }

}  // namespace devel
