// Host interface of the tcgen05 forward convolution of the DSN (conv_tc.cu).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "common.cuh"

namespace devel {

// Layers the tensor-core kernel takes: Cin a multiple of 16, and either Cout in
// {32, 64, 128} on planes of side >= 128 (a multiple of 8; one 128-pixel row segment per
// MMA tile) or Cout = 256 on planes of side 64 (operands swapped: one 64-pixel row per
// MMA tile, 128 output channels per MMA).
bool conv3_tc_supported(int Cin, int Cout, int side);
// bf16 elements of the prepared weights Wtc[ceil(Cin / 64)][9][Cout][64] (for Cout = 32 in
// the order [cb][dx][2 - dy], the same count)
size_t conv3_tc_weight_elems(int Cin, int Cout);
// shared-memory opt-in of the kernel instances (once per device, outside any capture)
int conv3_tc_init_attrs();
// TMA map over the prepared weights: one [Cout x 64] box per (channel block, tap)
int conv3_tc_make_map(CUtensorMap* tm, const __nv_bfloat16* Wt, int Cin, int Cout);
// Wtc from the FP32 weights W[Cout][Cin][3][3]
int launch_prep_wtc(const float* W, int Cout, int Cin, __nv_bfloat16* Wt, cudaStream_t s);
// Y[nb][Cout][side][side] = ReLU(conv3x3([XA; XB]) + bias), bf16 NCHW, zero padding
int launch_conv3_tc(const __nv_bfloat16* XA, int CA, const __nv_bfloat16* XB, int CB, const CUtensorMap& tmW,
                    const float* bias, __nv_bfloat16* Y, int Cout, int nb, int side, cudaStream_t s);

}  // namespace devel
