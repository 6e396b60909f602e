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

// Row pass: d2(x) = min_x' [(x - x')^2 + g(x')^2] over the columns x' where the
// wanted class occurs. One block per row, the row of packed g in shared memory;
// each pixel searches outwards |x - x'| = 1, 2, ... while (x - x')^2 is below its
// best candidate. Per 16-column block the smaller g of each class is kept, and
// the search skips the rest of a block when even its best case (distance to the
// nearest unscanned column squared plus the block minimum squared) cannot beat
// the candidate (about 6 steps per pixel on a Manhattan clip).
constexpr int kBlk = 16;
constexpr int kEnvMaxN = 8192;

// Squared column distance, or kFar when the column has no pixel of the class; kFar
// plus any squared row distance (< 2^28 for n <= 8192) stays below INT_MAX.
constexpr int kFar = 1 << 30;

__global__ void __launch_bounds__(256)
k_edt_rows(const unsigned char* __restrict__ mask, int n, unsigned* __restrict__ g,
           float* __restrict__ phi, float d_lo, float d_hi) {
    extern __shared__ int sfx[];  // f0[n], f1[n]: g^2 per class; b0[nb], b1[nb]: block minima
    const int nb = (n + kBlk - 1) / kBlk;
    int* f0 = sfx;
    int* f1 = f0 + n;
    int* b0 = f1 + n;
    int* b1 = b0 + nb;
    const int y = blockIdx.x;
    const size_t base = (size_t)y * n;
    for (int x = threadIdx.x; x < n; x += blockDim.x) {
        const unsigned w = g[base + x];
        const unsigned a = w & 0xFFFFu, b = w >> 16;
        f0[x] = a == kNone ? kFar : (int)(a * a);
        f1[x] = b == kNone ? kFar : (int)(b * b);
    }
    __syncthreads();
    bool any0 = false, any1 = false;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        int m0 = kFar, m1 = kFar;
        for (int x = b * kBlk; x < min(n, (b + 1) * kBlk); ++x) {
            m0 = min(m0, f0[x]);
            m1 = min(m1, f1[x]);
        }
        b0[b] = m0;
        b1[b] = m1;
        any0 |= m0 < kFar;
        any1 |= m1 < kFar;
    }
    // rows in which a class never occurs (in any column) need no search for it
    const bool has0 = __syncthreads_or(any0), has1 = __syncthreads_or(any1);
    for (int x = threadIdx.x; x < n; x += blockDim.x) {
        const bool inside = mask[base + x] != 0;
        // an inside pixel looks for class 0, an outside one for class 1
        const int* f = inside ? f0 : f1;
        const int* bm = inside ? b0 : b1;
        int best = f[x];
        if (inside ? has0 : has1) {
            int L = x - 1, R = x + 1;
            while (true) {
                const int dl = x - L, dr = R - x;
                const int dl2 = dl * dl, dr2 = dr * dr;
                const bool lok = L >= 0 && dl2 < best;
                const bool rok = R < n && dr2 < best;
                if (!lok && !rok) break;
                // skip the rest of the 16-column block holding L (or R) when even the block's
                // minimum at the nearest unscanned column cannot win; valid at any position,
                // since every unscanned column of the block is at least that far
                if (lok) {
                    if (dl2 + bm[L >> 4] >= best) {
                        L = (L & ~(kBlk - 1)) - 1;
                    } else {
                        best = min(best, dl2 + f[L]);
                        --L;
                    }
                }
                if (rok) {
                    if (dr2 + bm[R >> 4] >= best) {
                        R = (R | (kBlk - 1)) + 1;
                    } else {
                        best = min(best, dr2 + f[R]);
                        ++R;
                    }
                }
            }
        }
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

}  // namespace

static size_t edt_rows_smem(int n) { return sizeof(int) * 2 * (n + (n + kBlk - 1) / kBlk); }

int reinit_init_attrs() {
    DEVEL_CUDA_TRY(cudaFuncSetAttribute(k_edt_rows, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)edt_rows_smem(kEnvMaxN)));
    return DEVEL_OK;
}

int launch_reinit(int n, const unsigned char* mask, float* phi, int* d2, float d_lo, float d_hi,
                  cudaStream_t s) {
    prof_begin(PK_EDT_COLS, s);
    k_edt_cols<<<(n + kCX - 1) / kCX, dim3(kCX, kSegs), 0, s>>>(mask, n, reinterpret_cast<unsigned*>(d2));
    prof_end(PK_EDT_COLS, s);
    DEVEL_LAUNCH_CHECK("k_edt_cols");
    prof_begin(PK_EDT_ROWS, s);
    k_edt_rows<<<n, 256, edt_rows_smem(n), s>>>(mask, n, reinterpret_cast<unsigned*>(d2), phi, d_lo, d_hi);
    prof_end(PK_EDT_ROWS, s);
    DEVEL_LAUNCH_CHECK("k_edt_rows");
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
