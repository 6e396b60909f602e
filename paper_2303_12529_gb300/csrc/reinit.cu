// Re-initialisation of the level set to a truncated signed distance.
//
// Eqs. (sdf), (tsdf) and Alg. 1 (CUDA_TSDF). Instead of the paper's search
// over all boundary pixels, the exact squared Euclidean distance is computed
// separably (d2(y,x) = min_x' [(x - x')^2 + g(y,x')^2], g the distance along
// the column):
//
//   k_edt_cols  one pass per column strip: g to the nearest pixel of each
//               class along the column, both packed in one 32-bit word
//               (two 16-bit distances, 0xFFFF = none), from per-segment bit
//               masks and scans over the segments;
//   k_edt_rows  one block per row: the row of packed g in shared memory; each
//               pixel searches outwards |dx| = 1, 2, ... while dx^2 is below
//               its best candidate, so the work per pixel is its distance.
//               Writes the exact d2 (or -1) over the packed words, and phi.
//
// Integer arithmetic throughout; sqrtf is IEEE round-to-nearest (no fast
// math), so phi is the correctly rounded sqrt(d2) minus one half.
#include <climits>
#include <mutex>

#include "common.cuh"

namespace devel {
namespace {

constexpr unsigned kNone = 0xFFFFu;
constexpr int kSegRows = 64;   // rows per column segment (one 64-bit mask)
constexpr int kSegMax = 128;   // segments per column (n <= 8192)
constexpr int kSegPerWarp = kSegMax / 32;
constexpr unsigned kLastNone = 0xFFFFFFFFu;   // packed (-1, -1): no pixel of either class
constexpr unsigned kFirstNone = 0x7FFF7FFFu;  // packed (32767, 32767), beyond any row

// Column pass. Lane x of warp w holds, for column x of the block's 32 and each segment
// s = w, w + 32, .. of 64 rows, the segment's mask bits in one 64-bit word (loaded one row
// at a time: a warp reads 32 consecutive bytes of a row, its stores write 128). The
// nearest pixel of each class above a segment is the prefix maximum of the segments' last
// positions, the nearest below the suffix minimum of their first positions: per column
// one sequential scan over the segments in shared memory, both classes at once as signed
// 16-bit halves (positions < 8192). The rows of a segment then take their distances from
// the runs of equal rows (below), and g is written once.
__global__ void __launch_bounds__(1024)
k_edt_cols(const unsigned char* __restrict__ mask, int n, unsigned* __restrict__ g) {
    __shared__ unsigned sL[kSegMax][32], sF[kSegMax][32];  // packed (class 0 | class 1 << 16)
    pdl_trigger();
    pdl_wait();
    mask += (size_t)blockIdx.y * n * n;  // clip blockIdx.y of a batch
    g += (size_t)blockIdx.y * n * n;
    const int lane = threadIdx.x, w = threadIdx.y, nw = blockDim.y;
    const int x = blockIdx.x * 32 + lane;
    const int S = (n + kSegRows - 1) / kSegRows;
    unsigned long long bits[kSegPerWarp];
#pragma unroll
    for (int j = 0; j < kSegPerWarp; ++j) {
        const int sg = w + j * nw, ys = sg * kSegRows, len = min(kSegRows, n - ys);
        bits[j] = 0ull;
        if (sg < S && x < n) {
            const unsigned char* p = mask + (size_t)ys * n + x;
#pragma unroll 16
            for (int i = 0; i < len; ++i)
                if (p[(size_t)i * n]) bits[j] |= 1ull << i;
        }
        if (sg < S) {
            const unsigned long long valid = len >= 64 ? ~0ull : ((1ull << len) - 1ull);
            const unsigned long long b1 = bits[j], b0 = ~b1 & valid;
            const int l0 = b0 ? ys + 63 - __clzll((long long)b0) : -1;
            const int l1 = b1 ? ys + 63 - __clzll((long long)b1) : -1;
            const int f0 = b0 ? ys + __ffsll((long long)b0) - 1 : 0x7FFF;
            const int f1 = b1 ? ys + __ffsll((long long)b1) - 1 : 0x7FFF;
            sL[sg][lane] = ((unsigned)l0 & 0xFFFFu) | ((unsigned)l1 << 16);
            sF[sg][lane] = (unsigned)f0 | ((unsigned)f1 << 16);
        }
    }
    __syncthreads();
    if (w == 0) {  // inclusive prefix maxima of the last positions, top down
        unsigned acc = kLastNone;
#pragma unroll 8
        for (int sg = 0; sg < S; ++sg) {
            acc = __vmaxs2(acc, sL[sg][lane]);
            sL[sg][lane] = acc;
        }
    }
    if (w == (nw > 1 ? 1 : 0)) {  // inclusive suffix minima of the first positions, bottom up
        unsigned acc = kFirstNone;
#pragma unroll 8
        for (int sg = S - 1; sg >= 0; --sg) {
            acc = __vmins2(acc, sF[sg][lane]);
            sF[sg][lane] = acc;
        }
    }
    __syncthreads();
    if (x >= n) return;
#pragma unroll
    for (int j = 0; j < kSegPerWarp; ++j) {
        const int sg = w + j * nw;
        if (sg >= S) break;
        const int ys = sg * kSegRows, len = min(kSegRows, n - ys);
        const unsigned up = sg > 0 ? sL[sg - 1][lane] : kLastNone;
        const unsigned dn = sg + 1 < S ? sF[sg + 1][lane] : kFirstNone;
        const int up0 = (int)(short)(up & 0xFFFFu), up1 = (int)(short)(up >> 16);
        const int dn0 = (int)(dn & 0xFFFFu), dn1 = (int)(dn >> 16);
        const unsigned long long valid = len >= 64 ? ~0ull : ((1ull << len) - 1ull);
        const unsigned long long b1 = bits[j];
        // A pixel's own class is at distance 0; the other class is nearest just outside the
        // pixel's run of equal rows. Bit i of t: rows i and i + 1 differ. At a run's first
        // row the run's end (the next set bit of t) and the nearest other-class rows above
        // and below are found once; every row of the run then needs a few operations.
        const unsigned long long t = (b1 ^ (b1 >> 1)) & (valid >> 1);
        int re = -1, above = -1, below = 0x7FFF;
        unsigned cls = 0u;
        unsigned* gp = g + (size_t)ys * n + x;
        for (int i = 0; i < len; ++i) {
            const int y = ys + i;
            if (i > re) {  // a run starts at row i
                cls = (unsigned)(b1 >> i) & 1u;
                const unsigned long long nt = t >> i;
                re = nt ? i + __ffsll((long long)nt) - 1 : len - 1;
                above = i > 0 ? y - 1 : (cls ? up0 : up1);
                below = re < len - 1 ? ys + re + 1 : (cls ? dn0 : dn1);
            }
            unsigned d = above >= 0 ? (unsigned)(y - above) : kNone;
            if (below != 0x7FFF) d = min(d, (unsigned)(below - y));
            gp[(size_t)i * n] = cls ? d : (d << 16);  // (class 0 | class 1 << 16), own class 0
        }
    }
}

// Row pass: d2(x) = min_x' [(x - x')^2 + f(x')] with f = g^2 over the columns x' where
// the wanted class occurs (an inside pixel looks for class 0, an outside one for class 1).
// One block per row, the row's f of both classes in shared memory, with lower bounds on
// 16-column blocks k (columns b0 .. b1): the block minimum of f and the lower envelope at
// both edges, eR(k) = min (b1 - x')^2 + f(x'), eL(k) = min (x' - b0)^2 + f(x'). For x > b1
// every column of k costs at least (x - b1)^2 + eR(k), since
// (x - x')^2 >= (x - b1)^2 + (b1 - x')^2 (symmetrically eL for x < b0).
// A warp takes 32 consecutive pixels and searches for all of them together, so that its
// control flow is uniform: it scans the tile's own two blocks unless no lane's bound can
// win, then walks outwards block by block while some lane's distance to the block is below
// its best candidate, scanning (all 16 columns, every lane) each block whose bound can win
// for some lane. Every skipped column provably cannot lower a lane's minimum, so the result
// is the exact minimum.
constexpr int kBlk = 16;
constexpr int kEnvMaxN = 8192;

// Squared column distance, or kFar when the column has no pixel of the class; kFar
// plus a few squared distances (each < 2^26 for n <= 8192) stays below INT_MAX.
constexpr int kFar = 1 << 30;

__host__ __device__ constexpr int edt_nb(int n) { return (n + kBlk - 1) / kBlk; }

// all 32 lanes: best = min(best, (x - x')^2 + f(x')) over the 16 columns of block k
__device__ __forceinline__ int scan_block(const int* f, int x, int k, int best) {
    const int b0 = k * kBlk;
#pragma unroll
    for (int j = 0; j < kBlk; ++j) {
        const int d = x - (b0 + j);
        best = min(best, d * d + f[b0 + j]);
    }
    return best;
}

__global__ void __launch_bounds__(256)
k_edt_rows(const unsigned char* __restrict__ mask, int n, unsigned* __restrict__ g,
           float* __restrict__ phi, float d_lo, float d_hi, int store_d2) {
    extern __shared__ int sfx[];
    pdl_trigger();
    pdl_wait();
    mask += (size_t)blockIdx.y * n * n;  // clip blockIdx.y of a batch
    g += (size_t)blockIdx.y * n * n;
    phi += (size_t)blockIdx.y * n * n;
    const int nb = edt_nb(n), npad = nb * kBlk;
    // per class c: f at c npad, then the block minima, eL and eR at 2 npad + (0 / 2 / 4 + c) nb
    int* const F = sfx;
    int* const BM = sfx + 2 * npad;
    int* const EL = BM + 2 * nb;
    int* const ER = BM + 4 * nb;
    unsigned char* const SM = reinterpret_cast<unsigned char*>(BM + 6 * nb);  // the row's mask bytes
    const int y = blockIdx.x;
    const size_t base = (size_t)y * n;
    // the row's packed column distances and mask bytes, eight columns per thread with all
    // their loads issued before the first use
    constexpr int kFill = 8;
    for (int x0 = threadIdx.x; x0 < npad; x0 += kFill * blockDim.x) {
        unsigned w[kFill];
        unsigned char mk[kFill];
#pragma unroll
        for (int u = 0; u < kFill; ++u) {
            const int x = x0 + u * blockDim.x;
            w[u] = kNone | (kNone << 16);
            mk[u] = 0;
            if (x < n) {
                w[u] = g[base + x];
                mk[u] = mask[base + x];
            }
        }
#pragma unroll
        for (int u = 0; u < kFill; ++u) {
            const int x = x0 + u * blockDim.x;
            if (x < npad) {
                const unsigned a = w[u] & 0xFFFFu, b = w[u] >> 16;
                F[x] = a == kNone ? kFar : (int)(a * a);
                F[npad + x] = b == kNone ? kFar : (int)(b * b);
                SM[x] = mk[u];
            }
        }
    }
    __syncthreads();
    bool any0 = false, any1 = false;
    for (int i = threadIdx.x; i < 2 * nb; i += blockDim.x) {  // (class, block) pairs
        const int c = i / nb, k = i - c * nb;
        const int* fc = F + c * npad + k * kBlk;
        int m = kFar, l = kFar, r = kFar;
#pragma unroll
        for (int j = 0; j < kBlk; ++j) {
            const int v = fc[j];
            m = min(m, v);
            l = min(l, v + j * j);
            r = min(r, v + (kBlk - 1 - j) * (kBlk - 1 - j));
        }
        BM[c * nb + k] = m;
        EL[c * nb + k] = l;
        ER[c * nb + k] = r;
        if (c == 0) any0 |= m < kFar;
        else any1 |= m < kFar;
    }
    // rows in which a class never occurs (in any column) need no search for it
    const bool has0 = __syncthreads_or(any0), has1 = __syncthreads_or(any1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    for (int x0 = warp * 32; x0 < n; x0 += nwarps * 32) {
        const int x = x0 + lane;
        const bool valid = x < n;
        const bool inside = valid && SM[x] != 0;
        const int c = inside ? 0 : 1;
        const int* f = F + c * npad;
        const int* bm = BM + c * nb;
        const int* el = EL + c * nb;
        const int* er = ER + c * nb;
        const bool active = valid && (inside ? has0 : has1);
        int best = valid ? f[x] : kFar;
        // the tile's own blocks
        const int tb0 = x0 / kBlk, tb1 = min(nb - 1, (x0 + 31) / kBlk);
        for (int k = tb0; k <= tb1; ++k) {
            const int b0 = k * kBlk, b1 = b0 + kBlk - 1;
            int bound;
            if (x < b0) bound = (b0 - x) * (b0 - x) + el[k];
            else if (x > b1) bound = (x - b1) * (x - b1) + er[k];
            else bound = 1 + bm[k];  // every other column of x's own block is >= 1 away
            if (__any_sync(0xffffffffu, active && bound < best)) best = scan_block(f, x, k, best);
        }
        for (int k = tb0 - 1; k >= 0; --k) {  // blocks to the left, nearest first
            const int d = x - (k * kBlk + kBlk - 1), dd = d * d;
            const bool alive = active && dd < best;
            if (!__any_sync(0xffffffffu, alive)) break;
            if (__any_sync(0xffffffffu, alive && dd + er[k] < best)) best = scan_block(f, x, k, best);
        }
        for (int k = tb1 + 1; k < nb; ++k) {  // blocks to the right
            const int d = k * kBlk - x, dd = d * d;
            const bool alive = active && dd < best;
            if (!__any_sync(0xffffffffu, alive)) break;
            if (__any_sync(0xffffffffu, alive && dd + el[k] < best)) best = scan_block(f, x, k, best);
        }
        if (valid) {
            float v;
            int d2;
            if (best >= kFar) {
                d2 = -1;
                v = inside ? d_lo : d_hi;
            } else {
                d2 = best;
                const float dist = sqrtf((float)best) - 0.5f;
                v = inside ? -dist : dist;
                v = fminf(fmaxf(v, d_lo), d_hi);
            }
            if (store_d2) g[base + x] = (unsigned)d2;
            phi[base + x] = v;
        }
    }
}

}  // namespace

static size_t edt_rows_smem(int n) { return sizeof(int) * (2 * edt_nb(n) * kBlk + 6 * edt_nb(n)) + edt_nb(n) * kBlk; }

int reinit_init_attrs() {
    DEVEL_CUDA_TRY(cudaFuncSetAttribute(k_edt_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)edt_rows_smem(kEnvMaxN)));
    return DEVEL_OK;
}

int launch_reinit(int n, const unsigned char* mask, float* phi, int* d2, float d_lo, float d_hi,
                  cudaStream_t s, int B, bool want_d2) {
    prof_begin(PK_EDT_COLS, s);
    const int segs = (n + kSegRows - 1) / kSegRows;
    cudaError_t e = launch_pdl(k_edt_cols, dim3((n + 31) / 32, B), dim3(32, std::min(32, segs)), 0, s, mask, n,
                               reinterpret_cast<unsigned*>(d2));
    prof_end(PK_EDT_COLS, s);
    if (e != cudaSuccess) return cuda_error(e, "k_edt_cols");
    prof_begin(PK_EDT_ROWS, s);
    e = launch_pdl(k_edt_rows, dim3(n, B), dim3(256), edt_rows_smem(n), s, mask, n, reinterpret_cast<unsigned*>(d2), phi,
                   d_lo, d_hi, want_d2 ? 1 : 0);
    prof_end(PK_EDT_ROWS, s);
    if (e != cudaSuccess) return cuda_error(e, "k_edt_rows");
    return DEVEL_OK;
}

}  // namespace devel

// ---------------------------------------------------------------------------
// Allocation-free variant: the distance scratch lives in a static device array.
// ---------------------------------------------------------------------------
// Some callers cannot allocate device memory (their memory is owned by another
// allocator, or they must not pay cudaMalloc's implicit synchronisation), so
// devel_reinit_sdf_static needs no scratch argument. The array below is
// reserved on every GPU that loads this library, for the life of the process.
static __device__ __align__(256) unsigned g_reinit_scratch[(size_t)DEVEL_REINIT_STATIC_MAX_N *
                                                           DEVEL_REINIT_STATIC_MAX_N];

namespace devel {
namespace {
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_addr[kMaxDevices] = {};
}  // namespace
}  // namespace devel

extern "C" int devel_reinit_sdf_static(int n, const unsigned char* mask, float* phi, float d_lo,
                                       float d_hi, cudaStream_t s) {
    using namespace devel;
    if (n < 1 || n > DEVEL_REINIT_STATIC_MAX_N || n > kEnvMaxN)
        return set_error(DEVEL_EINVAL,
                         "devel_reinit_sdf_static: n=%d outside [1, %d] (size of the static scratch)", n,
                         DEVEL_REINIT_STATIC_MAX_N);
    if (!mask || !phi) return set_error(DEVEL_EINVAL, "devel_reinit_sdf_static: mask/phi is NULL");
    if ((reinterpret_cast<uintptr_t>(mask) | reinterpret_cast<uintptr_t>(phi)) & 15u)
        return set_error(DEVEL_EINVAL, "devel_reinit_sdf_static: mask/phi not 16-byte aligned");
    if (!(d_lo <= d_hi)) return set_error(DEVEL_EINVAL, "devel_reinit_sdf_static: d_lo > d_hi");
    int dev = 0;
    DEVEL_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices)
        return set_error(DEVEL_EINVAL, "devel_reinit_sdf_static: device %d beyond %d", dev, kMaxDevices);
    void* scratch = nullptr;
    {
        // set-up on the first call per device, with that device current: the host
        // symbol is only a stand-in, the kernels need the array's device address
        std::lock_guard<std::mutex> lock(g_scratch_mu);
        scratch = g_scratch_addr[dev];
        if (!scratch) {
            cudaError_t e = cudaGetSymbolAddress(&scratch, g_reinit_scratch);
            if (e != cudaSuccess) return cuda_error(e, "devel_reinit_sdf_static: cudaGetSymbolAddress");
            g_scratch_addr[dev] = scratch;
        }
    }
    // every scratch word the kernels read is written earlier in the same call,
    // so the previous call's contents need no clearing
    return launch_reinit(n, mask, phi, static_cast<int*>(scratch), d_lo, d_hi, s, 1, false);
}
