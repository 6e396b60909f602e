// Per-pixel sigmoid resist, DSO loss terms and dL/dI (Sec. III-A), and the
// fixed-order block reduction of the loss partials.
#pragma once

#include "common.cuh"

namespace devel {

inline ResistArgs make_resist_args(const devel_resist_params& p) {
    const double log2e = 1.4426950408889634;
    const double sz = p.sigma_z, d2i = (double)p.dose_in * p.dose_in, d2o = (double)p.dose_out * p.dose_out;
    ResistArgs a;
    a.I_th = p.I_th;
    a.d2in = (float)d2i;
    a.d2out = (float)d2o;
    a.a_nom = (float)(-log2e * sz);
    a.a_in = (float)(-log2e * sz * d2i);
    a.a_out = (float)(-log2e * sz * d2o);
    a.b = (float)(log2e * sz * p.I_th);
    a.k_nom = (float)(2.0 * sz * p.alpha);
    a.k_in = (float)(2.0 * sz * p.beta * d2i);
    a.k_out = (float)(2.0 * sz * p.beta * d2o);
    a.pad_ = 0.f;
    a.a_nom2 = make_float2(a.a_nom, a.a_nom);
    a.a_in2 = make_float2(a.a_in, a.a_in);
    a.a_out2 = make_float2(a.a_out, a.a_out);
    a.b2 = make_float2(a.b, a.b);
    a.d2in2 = make_float2(a.d2in, a.d2in);
    a.d2out2 = make_float2(a.d2out, a.d2out);
    a.k_nom2 = make_float2(a.k_nom, a.k_nom);
    a.k_in2 = make_float2(a.k_in, a.k_in);
    a.k_out2 = make_float2(a.k_out, a.k_out);
    return a;
}

// Loss accumulators of one thread: FP32 sums of a few pixels and the two
// binary-metric counts.
struct LossAcc {
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
    int l2 = 0, pvb = 0;
};

// 2^u and 1/x by the SFU (relative errors of a few 2^-23; subnormal results flush
// to zero, which only happens where Z saturates).
__device__ __forceinline__ float sfu_exp2(float u) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(u));
    return r;
}
__device__ __forceinline__ float sfu_rcp(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// min(a, b) that returns NaN when either operand is NaN (fminf would drop it).
__device__ __forceinline__ float min_nan(float a, float b) {
    float r;
    asm("min.NaN.f32 %0, %1, %2;" : "=f"(r) : "f"(a), "f"(b));
    return r;
}

// One corner: e = 2^u, Z = 1 / (1 + e) and the slope Z (1 - Z) = e Z^2 (no
// cancellation near Z = 1).
struct Corner {
    float z, ez2;
};

// The three corners of one pixel with one reciprocal: with q_c = 1 + e_c and
// r = 1 / (q_1 q_2 q_3), Z_1 = q_2 q_3 r and so on. u is capped at 40 (a NaN stays NaN),
// so the product stays below 2^121; where the cap applies Z is below 2^-40 and its
// absolute error is too.
__device__ __forceinline__ void resist_corners(float I1, float I2, float I3, float a1, float a2, float a3, float b,
                                               Corner& c1, Corner& c2, Corner& c3) {
    const float e1 = sfu_exp2(min_nan(fmaf(a1, I1, b), 40.f));
    const float e2 = sfu_exp2(min_nan(fmaf(a2, I2, b), 40.f));
    const float e3 = sfu_exp2(min_nan(fmaf(a3, I3, b), 40.f));
    const float q1 = 1.f + e1, q2 = 1.f + e2, q3 = 1.f + e3;
    const float q23 = q2 * q3;
    const float r = sfu_rcp(q1 * q23);
    const float z1 = q23 * r, z2 = (q1 * q3) * r, z3 = (q1 * q2) * r;
    c1 = Corner{z1, e1 * z1 * z1};
    c2 = Corner{z2, e2 * z2 * z2};
    c3 = Corner{z3, e3 * z3 * z3};
}

// Z_c = sigmoid(sigma_z (d_c^2 I - I_th)) at nominal / inner / outer dose;
// returns dL/dI = sum_c coef_c 2 (Z_c - Z_t) sigma_z Z_c (1 - Z_c) d_c^2.
__device__ __forceinline__ float resist_px(float I, bool zt_on, const ResistArgs& p, LossAcc& a) {
    const float zt = zt_on ? 1.f : 0.f;
    Corner cn, ci, co;
    resist_corners(I, I, I, p.a_nom, p.a_in, p.a_out, p.b, cn, ci, co);
    const float en = cn.z - zt, ei = ci.z - zt, eo = co.z - zt;
    a.s0 = fmaf(en, en, a.s0);
    a.s1 = fmaf(ei, ei, a.s1);
    a.s2 = fmaf(eo, eo, a.s2);
    a.l2 += ((I >= p.I_th) != zt_on);
    a.pvb += ((p.d2in * I >= p.I_th) != (p.d2out * I >= p.I_th));
    float g = (p.k_nom * en) * cn.ez2;
    g = fmaf(p.k_in * ei, ci.ez2, g);
    return fmaf(p.k_out * eo, co.ez2, g);
}

// Two pixels at once on the packed FP32 pipe (f32x2 add / mul / fma: the same IEEE
// round-to-nearest operations, so each pixel's dL/dI is bit-identical to resist_px): the
// parameters pre-broadcast in ResistArgs, the exponentials and the reciprocal per pixel. The squared
// errors accumulate per lane of s (pixel pairs (0, 2), (1, 3) of a group of four), folded
// into the thread's sums once at the end (a fixed order).
__device__ __forceinline__ float2 sfu_exp2_capped2(float2 u) {
    return make_float2(sfu_exp2(min_nan(u.x, 40.f)), sfu_exp2(min_nan(u.y, 40.f)));
}
__device__ __forceinline__ float2 resist_pair(float2 I, bool zt0, bool zt1, const ResistArgs& p, LossAcc& a,
                                              float2 (&s)[3]) {
    const float2 one = make_float2(1.f, 1.f);
    const float2 e1 = sfu_exp2_capped2(__ffma2_rn(p.a_nom2, I, p.b2));
    const float2 e2 = sfu_exp2_capped2(__ffma2_rn(p.a_in2, I, p.b2));
    const float2 e3 = sfu_exp2_capped2(__ffma2_rn(p.a_out2, I, p.b2));
    const float2 q1 = __fadd2_rn(one, e1), q2 = __fadd2_rn(one, e2), q3 = __fadd2_rn(one, e3);
    const float2 q23 = __fmul2_rn(q2, q3);
    const float2 pr = __fmul2_rn(q1, q23);
    const float2 r = make_float2(sfu_rcp(pr.x), sfu_rcp(pr.y));
    const float2 z1 = __fmul2_rn(q23, r), z2 = __fmul2_rn(__fmul2_rn(q1, q3), r), z3 = __fmul2_rn(__fmul2_rn(q1, q2), r);
    const float2 g1 = __fmul2_rn(__fmul2_rn(e1, z1), z1), g2 = __fmul2_rn(__fmul2_rn(e2, z2), z2),
                 g3 = __fmul2_rn(__fmul2_rn(e3, z3), z3);
    const float2 nzt = make_float2(zt0 ? -1.f : -0.f, zt1 ? -1.f : -0.f);  // z - zt as z + (-zt)
    const float2 en = __fadd2_rn(z1, nzt), ei = __fadd2_rn(z2, nzt), eo = __fadd2_rn(z3, nzt);
    s[0] = __ffma2_rn(en, en, s[0]);
    s[1] = __ffma2_rn(ei, ei, s[1]);
    s[2] = __ffma2_rn(eo, eo, s[2]);
    a.l2 += ((I.x >= p.I_th) != zt0) + ((I.y >= p.I_th) != zt1);
    const float2 di = __fmul2_rn(p.d2in2, I), dd = __fmul2_rn(p.d2out2, I);
    a.pvb += ((di.x >= p.I_th) != (dd.x >= p.I_th)) + ((di.y >= p.I_th) != (dd.y >= p.I_th));
    float2 g = __fmul2_rn(__fmul2_rn(p.k_nom2, en), g1);
    g = __ffma2_rn(__fmul2_rn(p.k_in2, ei), g2, g);
    return __ffma2_rn(__fmul2_rn(p.k_out2, eo), g3, g);
}

// Defocused process corner (Sec. II-C): the inner corner images through the defocused
// system (In: nominal-focus image, Id: defocused image). Returns dL/dIn (nominal and
// outer terms) and sets gD = dL/dId (inner term).
__device__ __forceinline__ float resist_px2(float In, float Id, bool zt_on, const ResistArgs& p, LossAcc& a,
                                            float& gD) {
    const float zt = zt_on ? 1.f : 0.f;
    Corner cn, ci, co;
    resist_corners(In, Id, In, p.a_nom, p.a_in, p.a_out, p.b, cn, ci, co);
    const float en = cn.z - zt, ei = ci.z - zt, eo = co.z - zt;
    a.s0 = fmaf(en, en, a.s0);
    a.s1 = fmaf(ei, ei, a.s1);
    a.s2 = fmaf(eo, eo, a.s2);
    a.l2 += ((In >= p.I_th) != zt_on);
    a.pvb += ((p.d2in * Id >= p.I_th) != (p.d2out * In >= p.I_th));
    gD = (p.k_in * ei) * ci.ez2;
    return fmaf(p.k_out * eo, co.ez2, (p.k_nom * en) * cn.ez2);
}

// Reduction of the accumulators of each group of 256 threads (a logical block) in a
// fixed order (FP32 / int within the group); the first thread of group j writes its
// partial to qpart[(part0 + j) * 3 + {0,1,2}] (fixed point, to_q32) and
// lpart[(part0 + j) * 2 + {0,1}]. Every thread of the CTA (at most 1024) must call
// it. sf/si: shared scratch of >= 32 entries.
__device__ __forceinline__ void block_store_loss(const LossAcc& a, int part0, long long* qpart, long long* lpart,
                                                 float (*sf)[32], int (*si)[32]) {
    float s0 = a.s0, s1 = a.s1, s2 = a.s2;
    int l2 = a.l2, pvb = a.pvb;
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_down_sync(0xffffffffu, s0, o);
        s1 += __shfl_down_sync(0xffffffffu, s1, o);
        s2 += __shfl_down_sync(0xffffffffu, s2, o);
        l2 += __shfl_down_sync(0xffffffffu, l2, o);
        pvb += __shfl_down_sync(0xffffffffu, pvb, o);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        sf[0][w] = s0;
        sf[1][w] = s1;
        sf[2][w] = s2;
        si[0][w] = l2;
        si[1][w] = pvb;
    }
    __syncthreads();
    if ((threadIdx.x & 255) == 0) {  // the group's 8 warps, in order
        const int w0 = threadIdx.x >> 5;
        float x0 = 0.f, x1 = 0.f, x2 = 0.f;
        int c0 = 0, c1 = 0;
        for (int i = w0; i < w0 + 8; ++i) {
            x0 += sf[0][i];
            x1 += sf[1][i];
            x2 += sf[2][i];
            c0 += si[0][i];
            c1 += si[1][i];
        }
        const int part = part0 + (threadIdx.x >> 8);
        qpart[part * 3 + 0] = to_q32(x0);
        qpart[part * 3 + 1] = to_q32(x1);
        qpart[part * 3 + 2] = to_q32(x2);
        lpart[part * 2 + 0] = c0;
        lpart[part * 2 + 1] = c1;
    }
}

}  // namespace devel
