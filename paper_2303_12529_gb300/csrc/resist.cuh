// Per-pixel sigmoid resist, DSO loss terms and dL/dI (Sec. III-A), shared by
// the standalone resist kernel and the fused epilogues of the expansion
// GEMMs; plus the fixed-order block reduction of the loss partials.
#pragma once

#include "common.cuh"

namespace devel {

inline ResistArgs make_resist_args(const devel_resist_params& p) {
    ResistArgs a;
    a.sigma_z = p.sigma_z;
    a.I_th = p.I_th;
    a.alpha = p.alpha;
    a.beta = p.beta;
    a.d2in = p.dose_in * p.dose_in;
    a.d2out = p.dose_out * p.dose_out;
    return a;
}

// Loss accumulators of one thread: FP32 sums of a few pixels (FP64 from the
// warp level up) and the two binary-metric counts.
struct LossAcc {
    float s0 = 0.f, s1 = 0.f, s2 = 0.f;
    int l2 = 0, pvb = 0;
};

// Z = 1 / (1 + e), e = exp(-t), and the slope Z (1 - Z) = e Z^2 (no cancellation
// near Z = 1). Hardware exp2 and reciprocal: relative error a few ulp for
// |t| of order 1, where dL/dI peaks; larger |t| only in saturated pixels.
__device__ __forceinline__ void sigmoid_slope(float t, float& z, float& dz) {
    const float e = __expf(-t);
    z = __fdividef(1.f, 1.f + e);
    dz = e * z * z;
}

// Z_c = sigmoid(sigma_z (d_c^2 I - I_th)) at nominal / inner / outer dose;
// returns dL/dI = sum_c coef_c 2 (Z_c - Z_t) sigma_z Z_c (1 - Z_c) d_c^2.
__device__ __forceinline__ float resist_px(float I, bool zt_on, const ResistArgs& p, LossAcc& a) {
    const float zt = zt_on ? 1.f : 0.f;
    const float Ii = p.d2in * I, Io = p.d2out * I;
    float zn, zi, zo, dn, di, dd;
    sigmoid_slope(p.sigma_z * (I - p.I_th), zn, dn);
    sigmoid_slope(p.sigma_z * (Ii - p.I_th), zi, di);
    sigmoid_slope(p.sigma_z * (Io - p.I_th), zo, dd);
    const float en = zn - zt, ei = zi - zt, eo = zo - zt;
    a.s0 = fmaf(en, en, a.s0);
    a.s1 = fmaf(ei, ei, a.s1);
    a.s2 = fmaf(eo, eo, a.s2);
    a.l2 += ((I >= p.I_th) != zt_on);
    a.pvb += ((Ii >= p.I_th) != (Io >= p.I_th));
    const float gn = p.alpha * en * dn;
    const float gi = p.beta * ei * di * p.d2in;
    const float go = p.beta * eo * dd * p.d2out;
    return 2.f * p.sigma_z * (gn + gi + go);
}

// Block reduction of the accumulators in a fixed order; thread 0 writes the
// block's partial to dpart[part * 3 + {0,1,2}] and lpart[part * 2 + {0,1}].
// Every thread of the block must call it. sd/sl: shared scratch of >= 32 entries.
__device__ __forceinline__ void block_store_loss(const LossAcc& a, int part, double* dpart, long long* lpart,
                                                 double (*sd)[32], long long (*sl)[32]) {
    double s0 = a.s0, s1 = a.s1, s2 = a.s2;
    long long l2 = a.l2, pvb = a.pvb;
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
        const int nw = (blockDim.x + 31) >> 5;
        double x0 = 0, x1 = 0, x2 = 0;
        long long c0 = 0, c1 = 0;
        for (int i = 0; i < nw; ++i) {
            x0 += sd[0][i];
            x1 += sd[1][i];
            x2 += sd[2][i];
            c0 += sl[0][i];
            c1 += sl[1][i];
        }
        dpart[part * 3 + 0] = x0;
        dpart[part * 3 + 1] = x1;
        dpart[part * 3 + 2] = x2;
        lpart[part * 2 + 0] = c0;
        lpart[part * 2 + 1] = c1;
    }
}

}  // namespace devel
