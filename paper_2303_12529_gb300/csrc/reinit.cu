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

constexpr int kCX = 8;     // columns per block
constexpr int kSegs = 128; // segments per column (<= 64 rows each for n <= 8192)
constexpr unsigned kNone = 0xFFFFu;
constexpr int kNoPos = INT_MAX;

// Column pass. Thread (column x, segment sg) holds its segment's mask bits in one
// 64-bit word; the nearest pixel of each class above the segment is the prefix
// maximum of the segments' last positions, the nearest below the suffix minimum of
// their first positions (Hillis-Steele scans over the block's segments). Every row
// of the segment then finds its nearest pixel of each class on either side with one
// leading/trailing-bit count, and g is written once.
__global__ void __launch_bounds__(kCX * kSegs)
k_edt_cols(const unsigned char* __restrict__ mask, int n, unsigned* __restrict__ g) {
    __shared__ int sc[2][4][kSegs][kCX];  // [buffer][last0, last1, first0, first1][segment][column]
    pdl_trigger();
    pdl_wait();
    mask += (size_t)blockIdx.y * n * n;  // clip blockIdx.y of a batch
    g += (size_t)blockIdx.y * n * n;
    const int cx = threadIdx.x, sg = threadIdx.y;
    const int x = blockIdx.x * kCX + cx;
    const int L = (n + kSegs - 1) / kSegs;
    const int ys = min(n, sg * L), len = min(n, ys + L) - ys;
    unsigned long long bits = 0ull;
    if (x < n) {
        for (int i = 0; i < len; ++i)
            if (mask[(size_t)(ys + i) * n + x]) bits |= 1ull << i;
    }
    const unsigned long long valid = len >= 64 ? ~0ull : ((1ull << len) - 1ull);
    const unsigned long long b1 = bits, b0 = ~bits & valid;
    sc[0][0][sg][cx] = b0 ? ys + 63 - __clzll((long long)b0) : -1;
    sc[0][1][sg][cx] = b1 ? ys + 63 - __clzll((long long)b1) : -1;
    sc[0][2][sg][cx] = b0 ? ys + __ffsll((long long)b0) - 1 : kNoPos;
    sc[0][3][sg][cx] = b1 ? ys + __ffsll((long long)b1) - 1 : kNoPos;
    int cur = 0;
    for (int off = 1; off < kSegs; off <<= 1) {
        __syncthreads();
        int l0 = sc[cur][0][sg][cx], l1 = sc[cur][1][sg][cx];
        int f0 = sc[cur][2][sg][cx], f1 = sc[cur][3][sg][cx];
        if (sg >= off) {
            l0 = max(l0, sc[cur][0][sg - off][cx]);
            l1 = max(l1, sc[cur][1][sg - off][cx]);
        }
        if (sg + off < kSegs) {
            f0 = min(f0, sc[cur][2][sg + off][cx]);
            f1 = min(f1, sc[cur][3][sg + off][cx]);
        }
        sc[cur ^ 1][0][sg][cx] = l0;
        sc[cur ^ 1][1][sg][cx] = l1;
        sc[cur ^ 1][2][sg][cx] = f0;
        sc[cur ^ 1][3][sg][cx] = f1;
        cur ^= 1;
    }
    __syncthreads();
    if (x >= n || len == 0) return;
    const int up0 = sg > 0 ? sc[cur][0][sg - 1][cx] : -1;
    const int up1 = sg > 0 ? sc[cur][1][sg - 1][cx] : -1;
    const int dn0 = sg + 1 < kSegs ? sc[cur][2][sg + 1][cx] : kNoPos;
    const int dn1 = sg + 1 < kSegs ? sc[cur][3][sg + 1][cx] : kNoPos;
    for (int i = 0; i < len; ++i) {
        const int y = ys + i;
        const unsigned long long le = (2ull << i) - 1ull, ge = ~0ull << i;
        const unsigned long long a0 = b0 & le, a1 = b1 & le, c0 = b0 & ge, c1 = b1 & ge;
        const int pa0 = a0 ? ys + 63 - __clzll((long long)a0) : up0;
        const int pa1 = a1 ? ys + 63 - __clzll((long long)a1) : up1;
        const int pb0 = c0 ? ys + __ffsll((long long)c0) - 1 : dn0;
        const int pb1 = c1 ? ys + __ffsll((long long)c1) - 1 : dn1;
        unsigned d0 = pa0 >= 0 ? (unsigned)(y - pa0) : kNone;
        unsigned d1 = pa1 >= 0 ? (unsigned)(y - pa1) : kNone;
        if (pb0 != kNoPos) d0 = min(d0, (unsigned)(pb0 - y));
        if (pb1 != kNoPos) d1 = min(d1, (unsigned)(pb1 - y));
        g[(size_t)y * n + x] = d0 | (d1 << 16);
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
           float* __restrict__ phi, float d_lo, float d_hi) {
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
    const int y = blockIdx.x;
    const size_t base = (size_t)y * n;
    for (int x = threadIdx.x; x < npad; x += blockDim.x) {
        const unsigned w = x < n ? g[base + x] : (kNone | (kNone << 16));
        const unsigned a = w & 0xFFFFu, b = w >> 16;
        F[x] = a == kNone ? kFar : (int)(a * a);
        F[npad + x] = b == kNone ? kFar : (int)(b * b);
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
        const bool inside = valid && mask[base + x] != 0;
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
            g[base + x] = (unsigned)d2;
            phi[base + x] = v;
        }
    }
}

}  // namespace

static size_t edt_rows_smem(int n) { return sizeof(int) * (2 * edt_nb(n) * kBlk + 6 * edt_nb(n)); }

int reinit_init_attrs() {
    DEVEL_CUDA_TRY(cudaFuncSetAttribute(k_edt_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)edt_rows_smem(kEnvMaxN)));
    return DEVEL_OK;
}

int launch_reinit(int n, const unsigned char* mask, float* phi, int* d2, float d_lo, float d_hi,
                  cudaStream_t s, int B) {
    prof_begin(PK_EDT_COLS, s);
    cudaError_t e = launch_pdl(k_edt_cols, dim3((n + kCX - 1) / kCX, B), dim3(kCX, kSegs), 0, s, mask, n,
                               reinterpret_cast<unsigned*>(d2));
    prof_end(PK_EDT_COLS, s);
    if (e != cudaSuccess) return cuda_error(e, "k_edt_cols");
    prof_begin(PK_EDT_ROWS, s);
    e = launch_pdl(k_edt_rows, dim3(n, B), dim3(256), edt_rows_smem(n), s, mask, n, reinterpret_cast<unsigned*>(d2), phi,
                   d_lo, d_hi);
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
    return launch_reinit(n, mask, phi, static_cast<int*>(scratch), d_lo, d_hi, s);
}
