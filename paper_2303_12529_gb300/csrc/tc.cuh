// Host interface of the tcgen05 contraction kernels (tc.cu).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "common.cuh"

namespace devel {
namespace tc {

// The four operand tensor maps of one GEMM (see make_map). use_alo = 0 skips
// the A_lo term (A exact in bf16).
struct Operands {
    const CUtensorMap* Ahi;
    const CUtensorMap* Alo;
    const CUtensorMap* Bhi;
    const CUtensorMap* Blo;
    int use_alo;
};

// bf16 tensor map over a row-major [rows][cols] array with row pitch ld
// elements; boxes of 64 columns x box_rows rows, 128-byte swizzle, zero fill.
int make_map(CUtensorMap* tm, const void* base, int rows, int cols, int ld, int box_rows);
// The same over `depth` such arrays, array d at base + d * dld elements (one per clip of a
// batch; loads give the clip as the third coordinate).
int make_map3(CUtensorMap* tm, const void* base, int depth, int rows, int cols, int ld, size_t dld, int box_rows);
// 3-D bf16 map without swizzle: dims (d0 innermost, d1, d2), byte strides s1 and s2 of dims 1
// and 2, box (b0, b1, b2) (b0 * 2 bytes a multiple of 16), zero fill.
int make_map_plain3(CUtensorMap* tm, const void* base, uint64_t d0, uint64_t d1, uint64_t d2, uint64_t s1,
                    uint64_t s2, uint32_t b0, uint32_t b1, uint32_t b2);

// D = ep.scale * A B^T (M x N, contraction length K, a multiple of 16, all of it in
// one CTA), tiles of 128 x BN (BN a multiple of 16 up to 256, the B map's box height),
// written as bf16 hi/lo into ep.Chi / ep.Clo with row pitch ep.ldh; for B clips, B is a
// 3-D map over them and clip c's D goes to ep.Chi / ep.Clo + c * ep.split_stride.
int launch_gemm_split(const Operands& op, int BN, int prof_kind, int M, int N, int K, int B, const EpiArgs& ep,
                      int* err, cudaStream_t s);

// A window reduction (k_tc_spec2, then k_spec_sum) over the folded table: the phase-1
// operands as in launch_gemm (A = image [M rows][K], B = folded basis [BN rows][K]),
// Chi/Clo = the same tables with 128-row boxes (the phase-2 A operand); BN = the table's
// ldf, kw the window side (kw <= BN), K a multiple of 64. The image maps are 3-D over
// B clips. Each CTA takes 128 rows and `split` columns of one clip's image (split a
// multiple of 64) and stores its kw x kw block of cos / sin products as one of the clip's
// spectrum2_slices(M, K, split) slices of G ([B][slices][kw][round_up(kw, 16)] floats);
// the slices are then added in order and combined, clip c into out + c kw^2:
// out[a][b] = n^-2 sum_p X(p) e^{-2 pi i ((a-r) y + (b-r) x) / n}.
int spectrum2_slices(int M, int K, int split);
int launch_spectrum2(const Operands& op, const CUtensorMap* Chi, const CUtensorMap* Clo, int BN, int kw, int n,
                     int M, int K, int split, int B, float* G, float2* out, int* err, cudaStream_t s);

// Persistent expansion D = ep.scale * A B^T (k_tc_expand) for B clips, clip c's M x N
// output row-major at ep.C + c * ep.split_stride with pitch ep.ldc; A a 3-D map over the
// clips' [M][K] operands with 128-row boxes, B the [N][K] table map with BN-row boxes (BN =
// 64 or 128, the output tile width); K a multiple of 16 up to 256.
// epi: EPI_STORE, or EPI_VEL (also max |D| of each clip into ep.vmax[c] as FP64, through the
// zeroed words ep.vbits[c], which the kernel leaves zeroed; ep.counter a zeroed word).
int launch_expand(const Operands& op, int BN, int epi, int M, int N, int K, int B, const EpiArgs& ep, int* err,
                  cudaStream_t s);
int expand_grid(int M, int N, int BN);

// One CTA whose thread waits (bounded) on an mbarrier that nothing signals: sets
// *err = DEVEL_ETIMEOUT after the wait limit (about one second).
int launch_wait_selftest(int* err, cudaStream_t s);

// Shared-memory opt-in of all tensor-core kernels (once per device).
int init_attrs();

// hi/lo split of a row-major float array [rows][cols] (pitch ldx) into
// [rows][ldo] bf16 arrays, zero beyond cols; lo may be NULL.
int launch_split(const float* X, int rows, int cols, int ldx, int ldo, __nv_bfloat16* hi, __nv_bfloat16* lo,
                 cudaStream_t s);
// 0/1 mask (uint8 [n][n]) to bf16 [n][ldo], zero beyond n (B masks n^2 apart into outputs
// n ldo apart).
int launch_mask_bf16(const unsigned char* M, int n, int ldo, __nv_bfloat16* hi, cudaStream_t s, int B = 1);

}  // namespace tc
}  // namespace devel
