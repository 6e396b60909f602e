/*
 * develset.h -- C ABI of the GB300 level-set inverse-lithography (ILT) library.
 *
 * The library runs the per-iteration hot path of the DevelSet-Optimizer
 * (DSO) loop of "DevelSet: Deep Neural Level Set for Instant Mask
 * Optimization" (Chen et al., arXiv 2303.12529) as CUDA kernels for sm_103a:
 *
 *   devel_reinit_sdf      Eqs. (sdf), (tsdf), Alg. 1 CUDA_TSDF     TSDF of a mask
 *   devel_reinit_sdf_batch  the same for a batch of masks in one launch
 *   devel_litho_forward   Sec. II-B SOCS imaging                   I = sum_j w_j |M (*) h_j|^2
 *   devel_resist_loss     Sec. III-A sigmoid resist, L_ilt, L_pvb; Sec. II-C L2, PVBand
 *   devel_litho_adjoint   Eqs. (ilt_gradient), (pvb_gradient), (vel)  dL/dM from dL/dI
 *   devel_levelset_step   Eqs. (dso_evolution), (numerical-settings), (curva_numer), (phi2mask)
 *   devel_levelset_step_weno5   the same step with WENO5 one-sided derivatives (Sec. III-C)
 *   devel_cg_direction    Sec. III-C conjugate-gradient direction of the velocity
 *   devel_modulation_candidates, devel_ahf_loss   Sec. III-B modulation-branch supervision
 *   devel_dsn_*           Sec. III-B DSN level-set branch: learned initial level set, training
 *   devel_phi_downsample, devel_phi_upsample   level sets between a clip's grid and the DSN's
 *   devel_shot_count      Sec. II-C.3 mask fracturing shot count (host)
 *   devel_ilt_solve       Sec. III-A / III-C: the whole loop for a batch of clips
 *   devel_ilt_solve_batch the same loop with each stage launched once over all clips
 *
 * Conventions shared by every call
 * --------------------------------
 * - Images are n x n, row-major, index p = y * n + x (y = row, x = column).
 *   Lithography is periodic (circular convolution on the n x n torus).
 * - Optical kernel j is given by its spectrum on a k x k window centred on
 *   DC (k odd, r = (k-1)/2): H[j][a][b] is the value at frequency
 *   (u, v) = (a - r, b - r) cycles per n pixels, u along rows (y), v along
 *   columns (x). The spatial kernel is h_j = IDFT_n(zero-padded H_j), with
 *   the 1/n^2 on the inverse. Complex values are interleaved (re, im) float.
 * - Pointers are DEVICE pointers owned by the caller unless marked "host".
 *   Device arrays must be 16-byte aligned (any cudaMalloc / PyTorch
 *   allocation is). Nothing is allocated after devel_optics_create.
 * - Every call enqueues work on `stream` and returns without waiting, so
 *   CUDA errors from the kernels themselves surface at the caller's next
 *   synchronisation. Calls that share one devel_optics handle must not run
 *   concurrently (the handle holds the per-iteration workspace).
 * - Return value: DEVEL_OK, or a negative code; devel_last_error() then
 *   returns a thread-local message naming the argument or the CUDA error.
 *   Argument checks happen before any work is enqueued.
 */
#ifndef DEVELSET_H
#define DEVELSET_H

#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DEVEL_OK 0
#define DEVEL_EINVAL (-1)   /* bad size, null or misaligned pointer, bad option */
#define DEVEL_ECUDA (-2)    /* a CUDA runtime call or kernel launch failed       */
#define DEVEL_ENOMEM (-3)   /* devel_optics_create could not allocate            */
#define DEVEL_ETIMEOUT (-4) /* a bounded device-side wait gave up                */
#define DEVEL_ENAN (-5)     /* a non-finite loss or velocity maximum was found   */

/* Arithmetic of the truncated-DFT contractions (forward and adjoint). */
#define DEVEL_PREC_FP32 0   /* FP32 FMA on the CUDA cores                         */
#define DEVEL_PREC_BF16X3 1 /* tcgen05 BF16 hi+lo split, 3 products, FP32 accumulate */

/* Upwind schemes of the level-set transport term (Sec. III-C names WENO for
 * |grad phi| without specifying it): Godunov's flux with first-order one-sided
 * differences, or with fifth-order WENO one-sided derivatives (Hamilton-Jacobi
 * WENO: three third-order ENO candidates, ideal weights 0.1 / 0.6 / 0.3,
 * smoothness indicators, eps = 1e-6 max v^2). */
#define DEVEL_UPWIND_GODUNOV1 0
#define DEVEL_UPWIND_WENO5 1

/* Optimisers of the solve (Sec. III-C: DSO optimises with conjugate gradient, the
 * paper gives no update rule): the front moves with the velocity V = dL/dM itself
 * (steepest descent), or with the nonlinear conjugate-gradient direction
 * D = V + beta D_prev, beta = max(0, <V, V - V_prev> / <V_prev, V_prev>) (Polak-Ribiere,
 * clipped at zero), restarted (D = V) at the first iteration of a solve and at every
 * iteration that follows a re-initialisation. Either is normalised by its max. */
#define DEVEL_OPT_STEEPEST 0
#define DEVEL_OPT_CG 1

/* Thread-local text of the last error returned on this thread ("" if none). */
const char* devel_last_error(void);

/* ABI version: (major << 16) | minor. */
int devel_version(void);

/* ------------------------------------------------------------------------ */
/* Optics handle                                                            */
/* ------------------------------------------------------------------------ */
typedef struct devel_optics devel_optics;

/*
 * Create the imaging model for n x n clips: K SOCS kernels (Sec. II-B; the
 * paper uses N_k = 24) on a k x k window.
 *   H_host  host, float[K][k][k][2]: kernel spectra (see conventions)
 *   w_host  host, float[K]: SOCS weights sigma_j >= 0
 *   precision DEVEL_PREC_FP32 or DEVEL_PREC_BF16X3
 * Requires 16 <= n <= 8192, k odd, 3 <= k, 2k - 1 <= n, 1 <= K <= k*k.
 * Copies everything it needs to the device (Sec. III-A keeps the optical
 * kernels and weights resident on the GPU for the whole optimisation) and
 * allocates the workspace of devel_litho_*, devel_cg_direction and
 * devel_ilt_solve for this n (about 29 bytes per pixel plus O(n k) tables).
 * *out receives the handle; on error *out is left NULL.
 * Returns DEVEL_EINVAL, DEVEL_ENOMEM or DEVEL_ECUDA on failure.
 */
int devel_optics_create(int n, int K, int k, const float* H_host, const float* w_host,
                        int precision, devel_optics** out);

/* Wait for the device, then free the handle and its device memory. NULL is a no-op. */
int devel_optics_destroy(devel_optics* optics);

/* n of the handle (or -1 for NULL). */
int devel_optics_n(const devel_optics* optics);

/*
 * Synchronise `stream`, then report (and clear) the handle's device error
 * flag: DEVEL_ETIMEOUT if a tensor-core kernel's bounded wait gave up during
 * an earlier devel_litho_* call on this handle, else DEVEL_OK.
 */
int devel_optics_check(const devel_optics* optics, cudaStream_t stream);

/*
 * Diagnostic (no counterpart in the paper): launches one thread that waits on a
 * device barrier nothing signals, through the same bounded wait the tensor-core
 * kernels use. The wait gives up after about one second and records
 * DEVEL_ETIMEOUT in the handle's flag, which the next devel_optics_check
 * returns (and clears); the context stays usable. Asynchronous on `stream`.
 */
int devel_selftest_bounded_wait(const devel_optics* optics, cudaStream_t stream);

/*
 * Tile-shape tuner (no counterpart in the paper; it serves batches of clips of
 * uneven sizes). Times the candidate tile shapes of the handle's tensor-core
 * kernels on its own workspace (the output tile width of the expansions, the
 * image columns per CTA of the reductions) and keeps the fastest for later
 * calls. Synchronises `stream`; overwrites the handle's workspace, so call it
 * between solves, not while a call on the handle is in flight. Results of later
 * calls may differ from earlier ones in the last bits (the summation order
 * depends on the tiles). A no-op for DEVEL_PREC_FP32 handles.
 */
int devel_optics_autotune(devel_optics* optics, cudaStream_t stream);
/* The tile shapes in use (0 for FP32 handles). Either pointer may be NULL. */
int devel_optics_config(const devel_optics* optics, int* expand_tile_n, int* reduce_split);

/* ------------------------------------------------------------------------ */
/* Lithography                                                              */
/* ------------------------------------------------------------------------ */

/*
 * Aerial image of a real mask (Sec. II-B):
 *   I(p) = sum_j w_j |A_j(p)|^2,  A_j = mask (*) h_j  (circular).
 *   mask       device float[n*n], any real values (the solver passes 0/1)
 *   intensity  device float[n*n], written
 * The mask may not alias intensity.
 */
int devel_litho_forward(const devel_optics* optics, const float* mask, float* intensity,
                        cudaStream_t stream);

/* Resist and loss parameters, Sec. III-A and IV (sigma_z = 50, alpha = 1, beta = 7.5). */
typedef struct {
    float sigma_z;   /* sigmoid steepness                                    */
    float I_th;      /* print threshold                                      */
    float alpha;     /* weight of L_ilt (nominal condition)                  */
    float beta;      /* weight of L_pvb (inner + outer corners)              */
    float dose_in;   /* inner-corner dose, image scales by dose_in^2 (0.98)  */
    float dose_out;  /* outer-corner dose, image scales by dose_out^2 (1.02) */
} devel_resist_params;

/*
 * Sigmoid resist Z_c = 1/(1+exp(-sigma_z (d_c^2 I - I_th))) at the three
 * conditions c = nominal (d=1), inner, outer, and
 *   L    = alpha sum (Z_nom - Z_t)^2 + beta [sum (Z_in - Z_t)^2 + sum (Z_out - Z_t)^2]
 *   dLdI = sum_c coef_c 2 (Z_c - Z_t) sigma_z Z_c (1 - Z_c) d_c^2
 *   L2   = #{[I >= I_th] != Z_t},  PVB = #{[d_in^2 I >= I_th] xor [d_out^2 I >= I_th]}
 *   intensity  device float[n*n]
 *   target     device uint8[n*n], 0/1
 *   params     host
 *   dLdI       device float[n*n], written (may alias intensity)
 *   loss_out   device double[4]: {L, sum (Z_nom-Z_t)^2, sum (Z_in-Z_t)^2, sum (Z_out-Z_t)^2}
 *   counts_out device long long[2]: {L2, PVB}
 * n is the handle's; its workspace holds the reduction partials. The sums
 * are FP32 within blocks of 256 threads and exact fixed-point (2^-32)
 * across blocks, returned as FP64; reproducible bit for bit.
 */
int devel_resist_loss(const devel_optics* optics, const float* intensity, const unsigned char* target,
                      const devel_resist_params* params, float* dLdI, double* loss_out,
                      long long* counts_out, cudaStream_t stream);

/*
 * Gradient of a loss L(I) with respect to the mask, given R = dL/dI
 * (Eq. ilt_gradient with the weights and the sum over kernels written out):
 *   dLdM(q) = sum_j 2 w_j Re sum_p R(p) conj(A_j(p)) h_j(p - q)
 *   mask   device float[n*n] (the mask the forward image was taken of)
 *   dLdI   device float[n*n]
 *   dLdM   device float[n*n], written
 *   vmax   device double[1], written with max_q |dLdM(q)|
 */
int devel_litho_adjoint(const devel_optics* optics, const float* mask, const float* dLdI,
                        float* dLdM, double* vmax, cudaStream_t stream);

/* ------------------------------------------------------------------------ */
/* Level set                                                                */
/* ------------------------------------------------------------------------ */

/*
 * One explicit level-set update, Eq. (dso_evolution) with the descent sign
 * (the velocity is V = +dL/dM), central differences of Eq.
 * (numerical-settings), curvature term of Eq. (curva_numer):
 *   F        = -dt V / vmax                 (transport skipped if vmax == 0)
 *   phi_out  = phi - [max(F,0) |grad phi|^+ + min(F,0) |grad phi|^-]
 *                  + dt lambda m Kc
 *   Kc       = (phi_xx phi_y^2 - 2 phi_x phi_y phi_xy + phi_yy phi_x^2)/(phi_x^2 + phi_y^2)
 *              (0 where phi_x^2 + phi_y^2 < 1e-12)
 *   mask_out = [phi_out <= 0]                                   Eq. (phi2mask)
 * |grad phi|^+- are Godunov's first-order upwind magnitudes; borders
 * replicate the edge pixel.
 *   phi      device float[n*n]         V      device float[n*n]
 *   vmax     device double[1]          m      device float[n*n] or NULL (m = 1)
 *   phi_out  device float[n*n], must not alias phi
 *   mask_out device uint8[n*n] or NULL
 */
int devel_levelset_step(int n, const float* phi, const float* V, const double* vmax,
                        const float* m, float dt, float lambda, float* phi_out,
                        unsigned char* mask_out, cudaStream_t stream);
/* The same update with the WENO5 one-sided derivatives in the transport term
 * (DEVEL_UPWIND_WENO5); same arguments and layout. */
int devel_levelset_step_weno5(int n, const float* phi, const float* V, const double* vmax,
                              const float* m, float dt, float lambda, float* phi_out,
                              unsigned char* mask_out, cudaStream_t stream);

/*
 * Truncated signed distance of a mask, Eqs. (sdf), (tsdf) (Alg. 1 CUDA_TSDF):
 *   phi = +(sqrt(d2) - 1/2)  outside (mask == 0),
 *   phi = -(sqrt(d2) - 1/2)  inside  (mask != 0),
 * clamped to [d_lo, d_hi] (the paper: D_l = -100, D_u = 900), where d2 is
 * the exact squared Euclidean distance between pixel centres to the nearest
 * pixel of the other class. [phi <= 0] reproduces the mask.
 *   mask   device uint8[n*n] (0 = outside, nonzero = inside)
 *   phi    device float[n*n], written
 *   d2     device int[n*n], scratch; on return d2[p] is the exact integer
 *          squared distance of p to the other class, or -1 if that class is empty
 * Requires 1 <= n <= 8192 and d_lo <= d_hi.
 */
int devel_reinit_sdf(int n, const unsigned char* mask, float* phi, int* d2, float d_lo,
                     float d_hi, cudaStream_t stream);

/*
 * devel_reinit_sdf of nb masks at once (Eqs. (sdf), (tsdf)): clip c's mask, phi and d2
 * at offset c*n*n of each array; one launch of each pass over the whole batch, and
 * per clip the same arithmetic in the same order, so every clip's phi and d2 are
 * bit-identical to devel_reinit_sdf on it alone.
 *   mask   device uint8[nb][n*n];  phi  device float[nb][n*n], written
 *   d2     device int[nb][n*n], scratch and output as in devel_reinit_sdf
 * Requires 1 <= n <= 8192, 1 <= nb <= 65535, d_lo <= d_hi; 16-byte-aligned arrays.
 */
int devel_reinit_sdf_batch(int n, int nb, const unsigned char* mask, float* phi, int* d2,
                           float d_lo, float d_hi, cudaStream_t stream);

/*
 * Allocation-free re-initialisation (the paper has no counterpart).
 *
 * Same result as devel_reinit_sdf (same kernels, bit-identical phi), for
 * callers that cannot allocate device memory and so cannot supply the d2
 * scratch: for example an embedder whose device memory is all owned by its
 * own pool allocator, or a latency-critical loop that must not pay the
 * device-wide synchronisation a cudaMalloc/cudaFree can cause. The n*n
 * distance scratch lives instead in a static device array inside the library:
 *   - n <= DEVEL_REINIT_STATIC_MAX_N (2048); larger n returns DEVEL_EINVAL.
 *     The array (2048*2048 32-bit words, 16 MiB) is reserved on every GPU
 *     that loads the library, until the process exits.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture begins. The address is kept for the life of
 *     the process: after a cudaDeviceReset of that device it is stale, so do
 *     not call this entry point again in a process that reset the device.
 *   - All calls share the one array: calls whose kernels overlap on the GPU
 *     (other streams, other threads) race on it; serialise them.
 *   - The array keeps the last call's contents; a call writes every word it
 *     reads before reading it, so nothing needs clearing.
 *   - Calls no cudaMalloc, cudaFree or other allocating routine.
 *   mask  device uint8[n*n]      phi  device float[n*n], written
 */
#define DEVEL_REINIT_STATIC_MAX_N 2048
int devel_reinit_sdf_static(int n, const unsigned char* mask, float* phi, float d_lo, float d_hi,
                            cudaStream_t stream);

/* ------------------------------------------------------------------------ */
/* Whole loop                                                               */
/* ------------------------------------------------------------------------ */

typedef struct {
    devel_resist_params resist;
    float dt;            /* CFL number eta: the front moves at most dt px per iteration */
    float lambda;        /* curvature weight                                              */
    float d_lo, d_hi;    /* TSDF clamp, Eq. (tsdf)                                        */
    int iters;           /* iterations T                                                  */
    int reinit_every;    /* re-initialise after iteration i when (i+1) % reinit_every == 0 (0 = never) */
    int start_iter;      /* global index of the first iteration (resume)                  */
    int use_graph;       /* 1: capture the solve into a CUDA graph on first use and replay it
                            on later calls with identical params and clip list (kernel
                            arguments are baked in; the data behind the pointers is read at
                            replay); 0: launch kernel by kernel. Ignored while a profile is open. */
    int upwind;          /* one-sided derivatives of |grad phi|: DEVEL_UPWIND_GODUNOV1 (first order)
                            or DEVEL_UPWIND_WENO5 (fifth-order WENO, Sec. III-C)                */
    int optimizer;       /* DEVEL_OPT_STEEPEST or DEVEL_OPT_CG (Sec. III-C). With CG, a solve
                            resumed at a multiple of reinit_every is bit-identical to the
                            unsplit run (the direction restarts there)                     */
} devel_ilt_params;

typedef struct {
    const devel_optics* optics;    /* imaging model; fixes n                              */
    const unsigned char* target;   /* device uint8[n*n], Z_t                              */
    float* phi;                    /* device float[n*n]: in = phi_0 if phi_given, out = phi_T */
    int phi_given;                 /* 0: phi_0 = TSDF(target) (the paper's start, Sec. III-A) */
    const float* m;                /* device float[n*n] curvature modulation m_theta, or NULL */
    unsigned char* mask_out;       /* device uint8[n*n] or NULL: [phi_T <= 0]            */
    double* loss_hist;             /* device double[iters+1] or NULL: L of the mask imaged
                                      by iteration i; entry iters is the final mask's    */
    long long* l2_hist;            /* device long long[iters+1] or NULL                  */
    long long* pvb_hist;           /* device long long[iters+1] or NULL                  */
    const devel_optics* optics_defocus; /* NULL: dose-only process corners (I_c = d_c^2 I). Else
                                      the defocused optical system of the inner corner (Sec. II-C:
                                      inner = defocus at dose_in, outer = nominal focus at dose_out):
                                      same n, window and precision as `optics`, a handle of its own
                                      (its workspace is used; no other clip of the call may use it) */
} devel_clip;

/*
 * Conjugate-gradient direction of the level-set velocity (Sec. III-C; the rule
 * of DEVEL_OPT_CG above):
 *   restart != 0:  D = V, beta = 0
 *   else:          beta = max(0, <V, V - Vprev> / <Vprev, Vprev>)  (0 if <Vprev, Vprev> = 0),
 *                  D = V + beta D
 * then Vprev = V and vmax_out = max |D| (the normaliser of the next
 * devel_levelset_step, which takes D as its V). <.,.> sums over the n*n
 * pixels: FP32 in a fixed order (reproducible); beta is computed in FP32.
 *   V         device float[n*n]             Vprev  device float[n*n], in/out
 *   D         device float[n*n], in/out (ignored on input when restarting)
 *   beta_out  device double[1] or NULL      vmax_out device double[1]
 *   status    device int[1] or NULL: set to DEVEL_ENAN if a dot product or D
 *             is not finite
 * V, Vprev and D must be distinct arrays; n is the handle's (its workspace
 * holds the partial sums).
 */
int devel_cg_direction(const devel_optics* optics, const float* V, float* Vprev, float* D, int restart,
                       double* beta_out, double* vmax_out, int* status, cudaStream_t stream);

/*
 * Supervision of the curvature modulation m_theta (Sec. III-B, modulation branch).
 *
 * Candidate maps: m_out[j][p] = H(phi_gt[p] + dh[j]) with the Heaviside of Eq.
 * (heaviside), H(z) = 1 for z >= 0 (the sum in FP32), else 0; the paper draws dh
 * from U[-20, 20]. The label m_gt is the candidate whose DSO run (a devel_ilt_solve
 * with clip.m = m_out[j]) ends with the smallest L_DSO: run the candidates as clips of
 * one devel_ilt_solve, each with a handle of its own to run them concurrently.
 *   phi_gt  device float[n*n]           dh_host host float[ncand], finite
 *   m_out   device float[ncand][n*n]    1 <= ncand <= DEVEL_MOD_MAX_CANDIDATES
 */
#define DEVEL_MOD_MAX_CANDIDATES 64
int devel_modulation_candidates(int n, const float* phi_gt, int ncand, const float* dh_host, float* m_out,
                                cudaStream_t stream);

/*
 * The label search of the modulation branch (Sec. III-B) in one call: the candidate
 * maps m_out[j] = H(phi_gt + dh[j]) (as devel_modulation_candidates), a DSO solve of
 * every candidate with clip.m = m_out[j] from the TSDF of the target (the candidates are
 * the clips of one devel_ilt_solve, candidate j on handles[j], so distinct handles run
 * concurrently), and the index of the smallest final L_DSO (ties: the first; a non-finite
 * loss never wins) written to *best_dev. Everything is enqueued on `stream`; nothing is
 * read back. The solves' status word (as devel_ilt_solve's) goes to *status_dev.
 *   params    the solve's parameters (params->iters >= 0)
 *   handles   host array of ncand handles of side n (distinct handles run concurrently)
 *   target    device uint8[n*n]          phi_gt  device float[n*n]
 *   dh_host   host float[ncand], finite  1 <= ncand <= DEVEL_MOD_MAX_CANDIDATES
 *   m_out     device float[ncand][n*n]   the candidate maps (written)
 *   phi_work  device float[ncand][n*n]   the candidates' level sets (written)
 *   loss_hist device double[ncand][ldh]  per-candidate L_DSO history (iters + 1 entries
 *             per row); ldh >= iters + 1, even (16-byte rows)
 *   best_dev  device int[1]              status_dev device int[1]
 */
int devel_modulation_search(const devel_ilt_params* params, int ncand, devel_optics* const* handles,
                            const unsigned char* target, const float* phi_gt, const float* dh_host, float* m_out,
                            float* phi_work, double* loss_hist, int ldh, int* best_dev, int* status_dev,
                            cudaStream_t stream);

/*
 * Loss of the modulation branch against its label (Sec. III-B) with the approximated
 * Heaviside H_eps(phi) = (1 + (2/pi) atan(phi / eps)) / 2 (the paper: eps = 0.03):
 *   loss_out[0] = sum_p (H_eps(phi_m[p]) - m_gt[p])^2
 *   grad_out[p] = 2 (H_eps(phi_m[p]) - m_gt[p]) (eps / pi) / (eps^2 + phi_m[p]^2)
 * FP32 per pixel and within blocks, exact fixed point across blocks, FP64 result
 * (NaN if any term is not finite).
 *   phi_m, m_gt device float[n*n]   loss_out device double[1]
 *   grad_out    device float[n*n] or NULL
 * n is the handle's (its workspace holds the partial sums).
 */
int devel_ahf_loss(const devel_optics* optics, const float* phi_m, const float* m_gt, float eps,
                   double* loss_out, float* grad_out, cudaStream_t stream);

/*
 * Mask fracturing shot count (Sec. II-C.3): the number of rectangles the mask is
 * fractured into, read as the minimum number of non-overlapping axis-aligned
 * rectangles whose union is the mask (exact: per 4-connected piece, vertices / 2 +
 * holes - g - 1 with g the largest set of non-intersecting chords between reflex
 * vertices, from a bipartite matching). Host code, synchronous.
 *   mask_host  host uint8[n*n] (nonzero = mask)    count_out  host long long[1]
 */
int devel_shot_count(int n, const unsigned char* mask_host, long long* count_out);

/*
 * Level-set branch of DevelSet-Net (Sec. III-B): a convolutional encoder-decoder
 * that predicts the initial level set of DSO from the target (the paper gives no
 * layer list; this one has four levels of widths w, 2w, 4w, 8w with two 3x3
 * convolutions + ReLU each, 2x2 average pooling, nearest 2x upsampling with the
 * encoder's level concatenated after it, and a 1x1 head added to the input).
 * Input x = clip(tsdf, -band, band) / band of the target's TSDF; output
 * phi0 = band * (x + head(...)), so zero head weights give back the band-limited
 * TSDF (the plain DSO start). Trained with the mean squared error between
 * x + head and clip(phi_gt, -band, band) / band (phi_gt: the level set DSO
 * converges to) and Adam (lr given, beta1 0.9, beta2 0.999, eps 1e-8).
 * Activations BF16, weights used in BF16 (FP32 master copy), FP32 accumulation,
 * FP32 gradients; reductions in a fixed order (reproducible).
 * Tensors are device float [nb][side][side], nb <= batch; side a multiple of 16.
 * Parameters: a flat FP32 vector, per layer (in the order above, head last) the
 * weights [cout][cin][k][k] then the biases [cout].
 */
typedef struct devel_dsn devel_dsn;
int devel_dsn_create(int side, int batch, int width, devel_dsn** out);
int devel_dsn_destroy(devel_dsn* dsn);
long long devel_dsn_param_count(const devel_dsn* dsn);
/* He-normal weights (splitmix64 + Box-Muller from seed), zero biases; resets Adam. */
int devel_dsn_init(devel_dsn* dsn, unsigned long long seed);
/* Host float[param_count] in / out (synchronous); set_params resets Adam. */
int devel_dsn_set_params(devel_dsn* dsn, const float* host);
int devel_dsn_get_params(const devel_dsn* dsn, float* host);
/* Gradients of the last train step, host float[param_count] (synchronous). */
int devel_dsn_grads(const devel_dsn* dsn, float* host);
int devel_dsn_forward(devel_dsn* dsn, int nb, const float* tsdf, float band, float* phi0, cudaStream_t stream);
/* One Adam step on a batch; loss_out: device double[1] (mean squared error before the
 * step) or NULL. */
int devel_dsn_train_step(devel_dsn* dsn, int nb, const float* tsdf, const float* phi_gt, float band, float lr,
                         double* loss_out, cudaStream_t stream);
/* The same network as the modulation branch (Sec. III-B): its output y is read as
 * phi_m and m = H_eps(y) = (1 + (2/pi) atan(y / eps)) / 2 (the approximated Heaviside;
 * the paper: eps = 0.03). forward_ahf writes m (device float [nb][side][side]);
 * train_step_ahf takes one Adam step on mean (H_eps(y) - m_gt)^2 (the per-pixel L_m,
 * averaged) against 0 / 1 label maps m_gt (devel_modulation_candidates, picked by the
 * label search). */
int devel_dsn_forward_ahf(devel_dsn* dsn, int nb, const float* tsdf, float band, float eps, float* m_out,
                          cudaStream_t stream);
int devel_dsn_train_step_ahf(devel_dsn* dsn, int nb, const float* tsdf, const float* m_gt, float band, float eps,
                             float lr, double* loss_out, cudaStream_t stream);

/*
 * Level sets between a fine n x n grid and the coarse (n/f) x (n/f) grid a DSN runs
 * on, for clips larger than the network's side (Sec. III-B/C: the network predicts
 * phi_0, DSO refines it at the clip's own resolution). Distances are kept in the
 * pixels of each grid, so both maps also scale values by f.
 *   downsample: coarse[b][I][J] = (1 / f^3) sum_{u,v < f} fine[b][f I + u][f J + v]
 *               (the mean over the f x f block, in coarse pixels; the block mean of
 *               an affine function is its value at the block centre).
 *   upsample:   fine[b][p][q] = f * bilinear(coarse[b], (p + 1/2) / f - 1/2,
 *               (q + 1/2) / f - 1/2), pixel centres aligned, coarse indices clamped
 *               to the grid (constant beyond the outer coarse centres).
 * fine: device float [nb][n][n]; coarse: device float [nb][n/f][n/f]; both 16-byte
 * aligned, not overlapping. n >= 1, f >= 1, n % f == 0, nb >= 0 (0: nothing to do);
 * otherwise DEVEL_EINVAL. Asynchronous on `stream`; FP32, sums in a fixed order.
 */
int devel_phi_downsample(int n, int f, int nb, const float* fine, float* coarse, cudaStream_t stream);
int devel_phi_upsample(int n, int f, int nb, const float* coarse, float* fine, cudaStream_t stream);

/*
 * Run `params->iters` DSO iterations on each clip (host array of nclips):
 * image, resist loss, adjoint velocity, level-set step, periodic TSDF
 * re-initialisation, all on `stream`, nothing copied to the host.
 *   status_dev  device int[1]: set to 0, then to DEVEL_ENAN by the device if a
 *               loss or max|V| is not finite (read it after synchronising).
 * Clips may have different n; each clip's handle must not be used by any
 * other concurrent call. With use_graph, the first call with a given
 * argument set captures the work on an internal stream (not on `stream`)
 * and later calls replay it: one graph launch on `stream`.
 */
int devel_ilt_solve(const devel_ilt_params* params, int nclips, const devel_clip* clips,
                    int* status_dev, cudaStream_t stream);

/*
 * Batched solve (Sec. III-A / III-C, the loop of devel_ilt_solve): up to `capacity`
 * clips on one compensated-BF16 optics handle, every stage of every iteration launched
 * once over all clips of the call (the reduction, Hopkins sums, expansions, resist,
 * level-set step and re-initialisation each take the clip as one more grid dimension),
 * so each launch moves the whole batch's data. Results per clip equal devel_ilt_solve's
 * up to FP32 rounding (the same arithmetic per clip; only the resist kernel's CTA shape
 * and the reduction's partial-spectrum order may differ).
 * devel_batch_create: the batch's workspace for `capacity` clips of the handle's n (about
 * 90 MB per clip at n = 2048); the handle must be DEVEL_PREC_BF16X3 and must outlive the
 * batch; its tables are shared, not copied. DEVEL_EINVAL for a bad argument, DEVEL_ENOMEM.
 * devel_ilt_solve_batch: nclips in [0, capacity]; arrays hold clip c at c times the
 * per-clip size:
 *   target     device uint8 [nclips][n*n]       phi   device float [nclips][n*n], in/out
 *   phi_given  0: phi_0 = TSDF(target)           m     device float [nclips][n*n] or NULL
 *   mask_out   device uint8 [nclips][n*n] or NULL
 *   loss_hist, l2_hist, pvb_hist  device [nclips][ldh] or NULL (ldh >= iters + 1)
 *   status_dev device int[1], as devel_ilt_solve's
 * params: the steepest-descent optimizer, either upwind scheme; DEVEL_EINVAL otherwise.
 * With use_graph the first call with an argument set is captured and later calls replay
 * it. Calls on one batch must not run concurrently.
 */
typedef struct devel_batch devel_batch;
int devel_batch_create(const devel_optics* optics, int capacity, devel_batch** out);
int devel_batch_destroy(devel_batch* batch);
int devel_ilt_solve_batch(const devel_ilt_params* params, devel_batch* batch, int nclips,
                          const unsigned char* target, float* phi, int phi_given, const float* m,
                          unsigned char* mask_out, double* loss_hist, long long* l2_hist, long long* pvb_hist,
                          int ldh, int* status_dev, cudaStream_t stream);

/* ------------------------------------------------------------------------ */
/* Optional kernel timing (tracing)                                          */
/* ------------------------------------------------------------------------ */

/*
 * Open a profile: until devel_profile_stop, every kernel launch of the
 * library is bracketed by two CUDA events on its stream (at most `capacity`
 * launches; events are created here, on the host, not on the hot path).
 * A solve captured into a graph meanwhile records the events inside the
 * graph (such graphs are dropped when the profile closes). One profile at a
 * time per process.
 */
int devel_profile_start(int capacity);
/*
 * Wait for the events recorded so far and add their launch counts and times
 * to the per-kernel totals. Events of kernel-by-kernel launches are counted
 * once (their slots are released); a solve captured into a CUDA graph while
 * the profile is open records its events on every replay, so call it after
 * each replay (both kinds may be mixed).
 */
int devel_profile_collect(void);
/* Close the profile (the totals stay readable). */
int devel_profile_stop(void);
/* Number of kernel classes. */
int devel_profile_kinds(void);
/* Restrict the events of the next profiles to the kernel classes whose bit
 * (1 << kind) is set in kind_mask (all classes by default): fewer events
 * disturb the timing of the selected kernels less. DEVEL_EINVAL while a
 * profile is open. */
int devel_profile_select(unsigned long long kind_mask);
/* Name, launch count and summed device time (ms) of kernel class `kind`
 * accumulated by devel_profile_collect. */
int devel_profile_query(int kind, const char** name, int* launches, double* total_ms);

#ifdef __cplusplus
}
#endif

#endif /* DEVELSET_H */
