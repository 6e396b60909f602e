// Internal declarations shared by the CUDA sources of libdevelset.
#pragma once

#include <climits>

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/develset.h"

namespace devel {

// ---------------------------------------------------------------------------
// error reporting (thread-local message, see devel_last_error)
// ---------------------------------------------------------------------------
int set_error(int code, const char* fmt, ...);
int cuda_error(cudaError_t e, const char* where);

#define DEVEL_CUDA_TRY(call)                                       \
    do {                                                           \
        cudaError_t _e = (call);                                   \
        if (_e != cudaSuccess) return ::devel::cuda_error(_e, #call); \
    } while (0)

#define DEVEL_LAUNCH_CHECK(where)                                  \
    do {                                                           \
        cudaError_t _e = cudaGetLastError();                       \
        if (_e != cudaSuccess) return ::devel::cuda_error(_e, where); \
    } while (0)

// ---------------------------------------------------------------------------
// programmatic dependent launch
// ---------------------------------------------------------------------------
// The kernels of the solve loop are launched with programmatic stream serialization: a
// kernel may be scheduled while the previous kernel on its stream is still running, so
// that its launch and prologue (barrier set-up, TMEM allocation, loads of the constant
// DFT and TCC tables) overlap that kernel's tail. Every such kernel
//   - calls pdl_trigger() as it starts (its dependents may then be scheduled once all of
//     its CTAs are resident), and
//   - calls pdl_wait() before it reads anything the previous kernel writes and before it
//     writes global memory; pdl_wait() returns once the previous kernel has completed and
//     its writes are visible. Since each kernel completes only after its own wait, that
//     covers every earlier kernel of the stream too.
// Both are no-ops for a kernel launched without the attribute. DEVEL_NO_PDL=1 in the
// environment launches every kernel with plain stream serialization.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

bool pdl_enabled();

template <typename... P, typename... A>
inline cudaError_t launch_pdl(void (*kernel)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              A&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = pdl_enabled() ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<A&&>(args)...);
}

// kernel classes of the optional event profiler (prof.cu)
enum ProfKind {
    PK_SPECTRUM = 0, PK_SPECTRUM_REDUCE, PK_SOCS_Y, PK_HOPKINS, PK_ADJ_WINDOW,
    PK_EXPAND_T, PK_EXPAND_GEMM, PK_VMAX, PK_RESIST, PK_RESIST_FINAL,
    PK_STEP, PK_MASK, PK_EDT_COLS, PK_EDT_ROWS, PK_U8F32,
    PK_TC_EXPAND, PK_TC_SPECTRUM, PK_SPECTRUM_STAGE2, PK_TC_SPLIT, PK_CG_DOTS, PK_CG_UPDATE,
    PK_DSN_CONV, PK_DSN_MISC, PK_RESAMPLE, PROF_NKINDS
};
bool prof_on();
unsigned prof_generation();
void prof_begin(int kind, cudaStream_t s);
void prof_end(int kind, cudaStream_t s);

// Per-corner constants of the resist (Sec. III-A), folded on the host:
// exponent u_c = a_c I + b = -log2(e) sigma_z (d_c^2 I - I_th), so that Z_c = 1 / (1 + 2^u_c);
// gradient coefficient k_c = 2 sigma_z coef_c d_c^2 (coef = alpha at nominal, beta at the corners).
struct ResistArgs {
    float I_th, d2in, d2out;
    float a_nom, a_in, a_out, b;
    float k_nom, k_in, k_out;
    float pad_;
    // the same values broadcast to pairs, for the packed FP32 path (kernel-parameter
    // operands: no registers held for them)
    float2 a_nom2, a_in2, a_out2, b2, d2in2, d2out2, k_nom2, k_in2, k_out2;
};

// N tile of the tensor-core GEMM T = E Z (a multiple of 16): narrow, so that the
// GEMM over n rows and ldk <= 256 columns still spreads over several CTAs per row block.
constexpr int kTileT = 16;

// Epilogues of the contraction GEMMs.
enum { EPI_STORE = 0, EPI_VEL = 1, EPI_SPLIT = 2 };

struct EpiArgs {
    float* C = nullptr;              // output
    int ldc = 0;
    size_t split_stride = 0;         // FP32 GEMM: offset of split-K slice z (C + z * split_stride);
                                     // tensor-core GEMMs: offset of clip z's output
    float scale = 1.f;
    float* vpart = nullptr;          // EPI_VEL (FP32 GEMM): per-CTA max |out|
    int n = 0;
    // EPI_VEL: the last CTA reduces the maxima into vmax (FP64), flags non-finite in *status
    unsigned* counter = nullptr;
    double* vmax = nullptr;          // tensor-core expansion: [nclips]
    int* status = nullptr;
    unsigned* vbits = nullptr;       // tensor-core expansion: [nclips] zeroed words (max |out| bits)
    int nclips = 1;
    // EPI_SPLIT: out = bf16 hi/lo pair, row pitch ldh (elements)
    __nv_bfloat16* Chi = nullptr;
    __nv_bfloat16* Clo = nullptr;
    int ldh = 0;
};


// Called by every thread of every block of an EPI_VEL expansion after the block has
// stored its max |V| in vpart[its index]: the last block to arrive reduces all nparts
// values (max is exact, so order does not matter), writes *vmax in FP64, flags a
// non-finite value in *status, and resets *counter to zero.
__device__ __forceinline__ void vmax_last_block(const float* vpart, int nparts, unsigned* counter, double* vmax,
                                                int* status) {
    __shared__ bool s_last;
    __shared__ float s_red[32];
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(counter, 1u) == (unsigned)nparts - 1u;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    float m = 0.f;
    bool bad = false;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
        const float v = __ldcg(vpart + i);
        if (!(v == v) || isinf(v)) bad = true;
        m = fmaxf(m, v);
    }
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = m;
    bad = __syncthreads_or(bad);
    if (threadIdx.x == 0) {
        float r = s_red[0];
        for (int w = 1; w < (int)((blockDim.x + 31) >> 5); ++w) r = fmaxf(r, s_red[w]);
        *vmax = (double)r;
        if (bad && status) *status = DEVEL_ENAN;
        *counter = 0u;
    }
}

// x * 2^32 as an int64, rounded toward zero, from the bits of an FP32 value with
// |x| < 2^30 (integer ALU only: FP64 instructions are slow here); kQBad for a
// non-finite x. Summing these is exact and independent of the order; a partial of
// squared errors of values in [0, 1] (each term <= 1) never approaches 2^30.
constexpr long long kQBad = LLONG_MIN;
__device__ __forceinline__ long long to_q32(float x) {
    const unsigned u = __float_as_uint(x);
    const int e = (int)((u >> 23) & 0xffu);
    if (e == 0xff) return kQBad;
    if (e == 0) return 0;  // zero or subnormal
    const long long m = (long long)((u & 0x7fffffu) | 0x800000u);
    const int sh = e - 118;  // x 2^32 = m 2^(e - 127 - 23 + 32)
    if (sh > 38) return kQBad;
    const long long q = sh >= 0 ? (m << sh) : (sh <= -24 ? 0 : (m >> -sh));
    return (u >> 31) ? -q : q;
}

// Device-side limit of the window side handled by the FP32 kernels.
constexpr int kMaxWindow = 63;

// ---------------------------------------------------------------------------
// the imaging model and its workspace
// ---------------------------------------------------------------------------
// A centred frequency window of side kw and its DFT tables.
struct Window {
    int kw = 0;              // window side (odd)
    int ldk = 0;             // round_up(2 kw, 16): padded contraction length
    float* basis = nullptr;  // [ldk][n]: rows a: cos(2 pi (a-r) x/n), rows kw+a: sin(...), rest 0
    float* basisT = nullptr; // [n][ldk]: the transpose
};

struct Workspace {
    float* Ppart = nullptr;    // [nsplit][n][ldk2] split-K slices of P (reduction stage 1)
    float* P = nullptr;        // [n][ldk2] stage-1 slices summed
    float* Q = nullptr;        // [slices][ldk2][ldk2] partial sums of reduction stage 2
    float2* mhat = nullptr;    // [k*k]   mask spectrum on W, scaled 1/n^2
    float2* Ihat = nullptr;    // [k2*k2] aerial-image spectrum on W2
    float2* rhat = nullptr;    // [k2*k2] dL/dI spectrum on W2, scaled 1/n^2
    float2* Shat = nullptr;    // [k*k]   adjoint spectrum on W
    float* Acat = nullptr;     // [n][ldk2] expansion operand [Re T | -Im T]
    long long* qpart = nullptr; // loss partials, fixed point (x 2^32), 3 per block
    long long* lpart = nullptr;// reduction partials, counts
    float* vpart = nullptr;    // per-block max |V| (FP32 path)
    unsigned* vbits = nullptr; // [batch] zeroed words: max |V| bit patterns (tensor-core path)
    // solver buffers
    float* bufI = nullptr;     // [n*n] intensity, then dL/dI (in place)
    float* bufV = nullptr;     // [n*n] dL/dM
    float* phi2 = nullptr;     // [n*n] ping-pong level set
    unsigned char* M = nullptr;// [n*n] mask
    int* d2 = nullptr;         // [n*n] EDT scratch
    double* vmax = nullptr;    // [1]
    double* loss4 = nullptr;   // [4]
    long long* cnt2 = nullptr; // [2]
    unsigned* counters = nullptr;  // [8] zeroed: last-block counters (0: resist, 1: max |V|,
                                   //     2: CG dot products, 3: max |D|, 4: AHF loss)
    // conjugate-gradient state (Sec. III-C)
    float* cgpart = nullptr;   // [3 * cg_parts] FP32 block sums of V.V, V.Vp, Vp.Vp
    float* cgvpart = nullptr;  // [cg_parts] per-block max |D|
    float* cgbeta = nullptr;   // [1] beta of the current iteration
    double* cg_vmax = nullptr; // [1] max |D|
    float* cgV = nullptr;      // [n*n] velocity of the previous iteration (solve only)
    float* cgD = nullptr;      // [n*n] direction (solve only)
};

// bf16 hi/lo tables and tensor maps of one window for the tensor-core path.
// The images are real, so each frequency pair +-j needs one cosine and one sine row:
// the folded table has kw = 2r + 1 rows, row j = cos(2 pi j x / n) for j = 0..r and
// row r + j = sin(2 pi j x / n) for j = 1..r, zero-padded to ldf = round_up(kw, 16)
// (about half the 2 kw rows of the FP32 path's tables, so every contraction of the
// tensor-core path is about half as wide).
struct TcWindow {
    int ldf = 0;                         // rows of the folded table: round_up(kw, 16)
    __nv_bfloat16* basis_hi = nullptr;   // [round_up(ldf, 128)][ldn], rows >= kw zero
    __nv_bfloat16* basis_lo = nullptr;
    __nv_bfloat16* basisT_hi = nullptr;  // [n][ldf]
    __nv_bfloat16* basisT_lo = nullptr;
    CUtensorMap m_basis_hi, m_basis_lo, m_basisT_hi, m_basisT_lo, m_acat_hi, m_acat_lo;
    CUtensorMap m_basis128_hi, m_basis128_lo;  // same tables, 128-row boxes (fused reduction, phase 2)
    CUtensorMap m_basisT64_hi, m_basisT64_lo;  // basis^T with 64-row boxes (expansion tiles of width 64)
    // the window spectrum Z folded onto the table's rows, as the B operand of T = E Z
    // (ldf x ldf; written by the Hopkins sums, see put_zm_folded)
    __nv_bfloat16* zm_hi = nullptr;
    __nv_bfloat16* zm_lo = nullptr;
    CUtensorMap m_zm_hi, m_zm_lo;    // boxes of kTileT rows (the N tile of T = E Z)
    CUtensorMap m_zmw_hi, m_zmw_lo;  // boxes of ldf rows (one N tile over the whole width)
};

}  // namespace devel

struct devel_optics {
    int n, K, k, r, k2, r2, precision;
    // clips whose workspace this struct describes: 1 for a handle; a batch's view of its
    // handle (devel_batch) shares the handle's tables and has B clips' workspace, every
    // per-clip array holding clip c at c times its single-clip size
    int batch = 1;
    int ldn = 0;                  // tensor-core path: round_up(n, 64)
    devel::TcWindow tcW, tcW2;
    __nv_bfloat16* Xhi = nullptr;     // [n][ldn] operand of the reductions
    __nv_bfloat16* Xlo = nullptr;
    __nv_bfloat16* Acat_hi = nullptr; // [n][ldf] operand of the expansions (ldf of the window)
    __nv_bfloat16* Acat_lo = nullptr;
    CUtensorMap m_X_hi, m_X_lo;
    int* tc_err = nullptr;            // device flag: DEVEL_ETIMEOUT from a bounded wait
    // tile shapes of the tensor-core path (devel_optics_autotune may change them)
    int tc_expand_bn = 128;           // output tile width of the expansion (64 or 128)
    int tc_split = 256;               // image columns per CTA of the fused reduction
    int tc_split_min = 256;           // smallest split the Q workspace is sized for
    int nsplit;               // split-K slices of reduction stage 1 (over x)
    int nq;                   // split-K slices of reduction stage 2 (over y)
    int npart_red;            // size of the generic reduction partial arrays
    devel::Window W, W2;      // the kernel window and the difference window
    float2* TCC = nullptr;    // [k*k][k*k] TCC_K(a, b) = sum_j w_j H_j(a) conj(H_j(b))
    float2* Tdiff = nullptr;  // k^4 entries: TCC_K(a, a - g) grouped by g in W2
    int* goff = nullptr;      // [k2*k2] offset of each g's group in Tdiff
    devel::Workspace ws;
};

namespace devel {

// ---------------------------------------------------------------------------
// launchers (litho.cu)
// ---------------------------------------------------------------------------
// spectrum of an n x n real image on window w (output scaled 1/n^2):
// out[a][b] = n^-2 sum_p X(p) e^{-2 pi i ((a-r)y + (b-r)x)/n}
int launch_spectrum_f32(const devel_optics* o, const float* X, const Window& w, float2* out, cudaStream_t s);
int launch_spectrum_u8(const devel_optics* o, const unsigned char* X, const Window& w, float2* out,
                       cudaStream_t s);
// tensor-core path: spectrum of the image already split into Xhi/Xlo
int launch_spectrum_resident(const devel_optics* o, const Window& w, float2* out, cudaStream_t s);
// Ihat (on W2) from mhat with the rank-K TCC
int launch_ihat(const devel_optics* o, cudaStream_t s);
// Shat (on W) from mhat and rhat with the rank-K TCC
// od: a second (defocused) system whose term is added (its TCC and rhat)
int launch_shat(const devel_optics* o, cudaStream_t s, const devel_optics* od = nullptr);
// out = mult * Re sum_{a,b} Z[a][b] e^{+2 pi i ((a-r)y + (b-r)x)/n} on window w; optional max|out|
// epi: EPI_STORE (ep.C = out) or EPI_VEL (ep.C, max |out| partials);
// *nparts = number of CTA partials.
int launch_expand(const devel_optics* o, const float2* Z, const Window& w, int epi, const EpiArgs& ep,
                  int* nparts, cudaStream_t s);

int expand_parts(int n);


// resist.cu
// dL/dI of the image I (n x n): into R (FP32, n x n) and/or into bf16 hi/lo
// arrays of pitch ldr; loss partials, then the final reduction.
// (one kernel: the last block to finish also does the final FP64 sums; `counter`
// is a zeroed device word that the kernel leaves zeroed). alone: no other kernel runs
// beside this one (one CTA per SM); else CTAs of 256 threads. Identical results.
// B > 1: a batch of B clips (256-thread CTAs, grid nparts x B): clip c's image and target
// at c n^2, its bf16 outputs at c n ldr, partials at c 3 nparts / c 2 nparts, counter
// counter + c, history entries at c hist_stride; loss4 / cnt2 must then be NULL.
int launch_resist(int n, const float* I, const unsigned char* Zt, const devel_resist_params& p,
                  float* R, __nv_bfloat16* Rhi, __nv_bfloat16* Rlo, int ldr, long long* qpart,
                  long long* lpart, int nparts, double* loss4, long long* cnt2, double* loss_hist,
                  long long* l2_hist, long long* pvb_hist, int* status, unsigned* counter, cudaStream_t s,
                  bool alone = true, int B = 1, int hist_stride = 0);
int resist_parts(int n);
// Defocused inner corner: images In (nominal focus) and Id (defocused); dL/dIn and dL/dId as
// FP32 images (Rn, Rd; may alias In, Id) or bf16 hi/lo operands (Rnhi.. with pitch ldr).
int launch_resist_defocus(int n, const float* In, const float* Id, const unsigned char* Zt,
                          const devel_resist_params& p, float* Rn, float* Rd, __nv_bfloat16* Rnhi,
                          __nv_bfloat16* Rnlo, __nv_bfloat16* Rdhi, __nv_bfloat16* Rdlo, int ldr, long long* qpart,
                          long long* lpart, int nparts, double* loss4, long long* cnt2, double* loss_hist,
                          long long* l2_hist, long long* pvb_hist, int* status, unsigned* counter, cudaStream_t s,
                          bool alone = true);

// levelset.cu
// mask_bf (optional): the new mask also as a bf16 [n][ldb] operand of the next reduction
// upwind: DEVEL_UPWIND_GODUNOV1 or DEVEL_UPWIND_WENO5 (one-sided derivatives of |grad phi|)
// modulation.cu: candidate maps H(phi + dh_j) (m: float[ncand][n*n]); AHF loss (qpart:
// long long[>= nparts], counter: one zeroed word, loss: device double).
int launch_mod_candidates(int n, const float* phi, int ncand, const float* dh_host, float* m, cudaStream_t s);
// *best = argmin_j hist[j * ldh + col] over finite entries (ties: the first)
int launch_argmin_final(const double* hist, int ncand, int ldh, int col, int* best, cudaStream_t s);
int launch_ahf_loss(int n, const float* phi, const float* mgt, float eps, float* grad, long long* qpart, int nparts,
                    unsigned* counter, double* loss, cudaStream_t s);
// cg.cu: D = V + beta D (PR+ beta from V, Vp; restart: D = V), Vp = V, max|D| -> vmax.
// part: float[3 * cg_parts(n)], vpart: float[cg_parts(n)], counters: 2 zeroed words.
int cg_parts(int n);
int launch_cg_direction(int n, const float* V, float* Vp, float* D, bool restart, float* part, float* vpart,
                        float* beta_f, double* beta_out, unsigned* counters, double* vmax, int* status,
                        cudaStream_t s);
// B > 1: a batch of B clips, each array's clip c at c n^2 (mask_bf: c n ldb, vmax: c; m: c n^2
// or NULL). phi_out, mask_out or mask_bf NULL: that output is not written.
int launch_levelset_step(int n, const float* phi, const float* V, const double* vmax,
                         const float* m, float dt, float lambda, float* phi_out,
                         unsigned char* mask_out, __nv_bfloat16* mask_bf, int ldb, cudaStream_t s,
                         int upwind = DEVEL_UPWIND_GODUNOV1, int B = 1);
// tensor-core path: spectrum of the mask already in Xhi (bf16, exact)
int launch_spectrum_mask_resident(const devel_optics* o, const Window& w, float2* out, cudaStream_t s);
int launch_mask_from_phi(int n, const float* phi, unsigned char* M, cudaStream_t s, int B = 1);
int launch_u8_to_f32(int n, const unsigned char* M, float* out, cudaStream_t s);

// one-time kernel attributes (api.cu calls them once per device)
int litho_init_attrs();
int reinit_init_attrs();

// reinit.cu
// B > 1: a batch of B clips, each array's clip c at c n^2. want_d2 false: d2 is scratch
// only (it then holds the packed column distances, and the row pass skips its store)
int launch_reinit(int n, const unsigned char* mask, float* phi, int* d2, float d_lo, float d_hi,
                  cudaStream_t s, int B = 1, bool want_d2 = true);

// forward / adjoint bodies shared by the ABI and the solver (api.cu)
int forward_from_mhat(const devel_optics* o, float* I, cudaStream_t s);
int forward_loss_from_mhat(const devel_optics* o, const unsigned char* target, const devel_resist_params& rp,
                           double* loss4, long long* cnt2, double* lh, long long* l2h, long long* pvbh,
                           int* status, cudaStream_t s);
int adjoint_from_mhat(const devel_optics* o, const float* R, float* V, double* vmax, int* status,
                      cudaStream_t s);
// adjoint from ws.mhat and the spectrum ws.rhat of dL/dI: Shat, then V with max |V| in vmax
// (od: a second, defocused system whose term is added, or NULL)
int adjoint_from_rhat(const devel_optics* o, float* V, double* vmax, int* status, cudaStream_t s,
                      const devel_optics* od = nullptr);

}  // namespace devel
