// C ABI of libdevelset: argument checks, the optics handle, and the
// forward / adjoint / solve sequences built from the kernels of the other
// translation units.
#include <algorithm>
#include <mutex>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "tc.cuh"

namespace devel {

static thread_local char g_err[512] = "";

int set_error(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

int cuda_error(cudaError_t e, const char* where) {
    return set_error(DEVEL_ECUDA, "%s: %s (%s)", where, cudaGetErrorName(e), cudaGetErrorString(e));
}

int expand_parts(int n);

bool pdl_enabled() {
    static const bool on = [] {
        const char* v = std::getenv("DEVEL_NO_PDL");
        return !(v && v[0] && v[0] != '0');
    }();
    return on;
}

// Shared-memory opt-ins of every kernel, once per device, outside any stream capture.
static int init_device_attrs() {
    static std::mutex mu;
    static bool done[64] = {};
    int dev = 0;
    DEVEL_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return set_error(DEVEL_EINVAL, "device index %d", dev);
    std::lock_guard<std::mutex> lock(mu);
    if (done[dev]) return DEVEL_OK;
    int rc = litho_init_attrs();
    if (!rc) rc = reinit_init_attrs();
    if (!rc) rc = tc::init_attrs();
    if (!rc) done[dev] = true;
    return rc;
}

static bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

#define CHECK_PTR(p, name)                                                             \
    do {                                                                               \
        if (!(p)) return set_error(DEVEL_EINVAL, "%s: %s is NULL", __func__, name);    \
        if (!aligned16(p))                                                             \
            return set_error(DEVEL_EINVAL, "%s: %s is not 16-byte aligned", __func__, name); \
    } while (0)

#define CHECK_OPT_PTR(p, name)                                                         \
    do {                                                                               \
        if ((p) && !aligned16(p))                                                      \
            return set_error(DEVEL_EINVAL, "%s: %s is not 16-byte aligned", __func__, name); \
    } while (0)

// forward image from ws.mhat: Ihat on W2, then the expansion (plain store)
int forward_from_mhat(const devel_optics* o, float* I, cudaStream_t s) {
    int rc = launch_ihat(o, s);
    if (rc) return rc;
    EpiArgs ep;
    ep.C = I;
    return launch_expand(o, o->ws.Ihat, o->W2, EPI_STORE, ep, nullptr, s);
}

// forward image and resist loss: I into ws.bufI, then dL/dI into ws.bufI (FP32
// path, in place) or into the bf16 reduction operand Xhi/Xlo (tensor-core path);
// the loss and metrics of this image go to the history slots (or loss4/cnt2).
int forward_loss_from_mhat(const devel_optics* o, const unsigned char* target, const devel_resist_params& rp,
                           double* loss4, long long* cnt2, double* lh, long long* l2h, long long* pvbh,
                           int* status, cudaStream_t s, bool alone = true) {
    int rc = forward_from_mhat(o, o->ws.bufI, s);
    if (rc) return rc;
    const bool tcp = o->precision == DEVEL_PREC_BF16X3;
    return launch_resist(o->n, o->ws.bufI, target, rp, tcp ? nullptr : o->ws.bufI, tcp ? o->Xhi : nullptr,
                         tcp ? o->Xlo : nullptr, o->ldn, o->ws.qpart, o->ws.lpart, o->npart_red, loss4, cnt2, lh,
                         l2h, pvbh, status, o->ws.counters, s, alone);
}

// adjoint from ws.mhat (spectrum of the imaged mask) and the spectrum rhat of R
int adjoint_from_rhat(const devel_optics* o, float* V, double* vmax, int* status, cudaStream_t s,
                      const devel_optics* od) {
    int rc = launch_shat(o, s, od);
    if (rc) return rc;
    EpiArgs ep;
    ep.C = V;
    ep.scale = 2.0f;
    ep.counter = o->ws.counters + 1;
    ep.vmax = vmax;
    ep.status = status;
    return launch_expand(o, o->ws.Shat, o->W, EPI_VEL, ep, nullptr, s);
}

// adjoint with R given as an FP32 image
int adjoint_from_mhat(const devel_optics* o, const float* R, float* V, double* vmax, int* status,
                      cudaStream_t s) {
    int rc = launch_spectrum_f32(o, R, o->W2, o->ws.rhat, s);
    if (rc) return rc;
    return adjoint_from_rhat(o, V, vmax, status, s);
}

// adjoint with R where forward_loss_from_mhat left it
static int adjoint_resident(const devel_optics* o, float* V, double* vmax, int* status, cudaStream_t s) {
    int rc = o->precision == DEVEL_PREC_BF16X3 ? launch_spectrum_resident(o, o->W2, o->ws.rhat, s)
                                               : launch_spectrum_f32(o, o->ws.bufI, o->W2, o->ws.rhat, s);
    if (rc) return rc;
    return adjoint_from_rhat(o, V, vmax, status, s);
}

static void free_optics(devel_optics* o) {
    if (!o) return;
    void* ptrs[] = {o->W.basis, o->W.basisT, o->W2.basis, o->W2.basisT, o->TCC, o->Tdiff, o->goff,
                    o->ws.Ppart, o->ws.P, o->ws.Q, o->ws.mhat, o->ws.Ihat, o->ws.rhat, o->ws.Shat,
                    o->ws.Acat, o->ws.qpart, o->ws.lpart, o->ws.vpart, o->ws.vbits, o->ws.bufI, o->ws.bufV, o->ws.phi2,
                    o->ws.M, o->ws.d2, o->ws.vmax, o->ws.loss4, o->ws.cnt2,
                    o->ws.cgpart, o->ws.cgvpart, o->ws.cgbeta, o->ws.cg_vmax, o->ws.cgV, o->ws.cgD,
                    o->tcW.basis_hi, o->tcW.basis_lo, o->tcW.basisT_hi, o->tcW.basisT_lo,
                    o->tcW2.basis_hi, o->tcW2.basis_lo, o->tcW2.basisT_hi, o->tcW2.basisT_lo,
                    o->tcW.zm_hi, o->tcW.zm_lo, o->tcW2.zm_hi, o->tcW2.zm_lo,
                    o->Xhi, o->Xlo, o->Acat_hi, o->Acat_lo, o->tc_err, o->ws.counters};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete o;
}

static int round_up(int v, int m) { return (v + m - 1) / m * m; }

// cos / sin table of a centred window of side kw, padded to ldk rows:
// rows 0..kw-1 cos, kw..2kw-1 sin, rest 0; angle 2 pi ((a - r) x mod n) / n
// reduced exactly in integers and evaluated in double. Also its transpose.
static void make_basis(int n, int kw, int ldk, std::vector<float>& t, std::vector<float>& tT) {
    const int r = (kw - 1) / 2;
    t.assign((size_t)ldk * n, 0.f);
    tT.assign((size_t)n * ldk, 0.f);
    for (int a = 0; a < kw; ++a) {
        const long long u = a - r;
        for (int x = 0; x < n; ++x) {
            long long m = (u * x) % n;
            if (m < 0) m += n;
            const double ang = 2.0 * M_PI * (double)m / (double)n;
            const float c = (float)std::cos(ang), sn = (float)std::sin(ang);
            t[(size_t)a * n + x] = c;
            t[(size_t)(kw + a) * n + x] = sn;
            tT[(size_t)x * ldk + a] = c;
            tT[(size_t)x * ldk + kw + a] = sn;
        }
    }
}

// Folded table of the tensor-core path as bf16 hi/lo pairs (x = hi + lo, hi = rn(x),
// lo = rn(x - hi), x the FP32 value): row j = cos(2 pi j x / n), j = 0..r, row r + j =
// sin(2 pi j x / n), j = 1..r; basis [rows][ldn] (rows >= kw and columns >= n zero) and
// its transpose basisT [n][ldf] (columns >= kw zero). Angles reduced exactly in integers
// and evaluated in double, as in make_basis.
static void make_basis_folded(int n, int kw, int ldf, int rows, int ldn, std::vector<__nv_bfloat16>& bh,
                              std::vector<__nv_bfloat16>& bl, std::vector<__nv_bfloat16>& th,
                              std::vector<__nv_bfloat16>& tl) {
    const int r = (kw - 1) / 2;
    const __nv_bfloat16 z = __float2bfloat16_rn(0.f);
    bh.assign((size_t)rows * ldn, z);
    bl.assign((size_t)rows * ldn, z);
    th.assign((size_t)n * ldf, z);
    tl.assign((size_t)n * ldf, z);
    for (int j = 0; j <= r; ++j) {
        for (int x = 0; x < n; ++x) {
            const long long m = ((long long)j * x) % n;
            const double ang = 2.0 * M_PI * (double)m / (double)n;
            const float v[2] = {(float)std::cos(ang), (float)std::sin(ang)};
            for (int q = 0; q < 2; ++q) {
                if (q == 1 && j == 0) continue;
                const int row = q == 0 ? j : r + j;
                const __nv_bfloat16 h = __float2bfloat16_rn(v[q]);
                const __nv_bfloat16 l = __float2bfloat16_rn(v[q] - __bfloat162float(h));
                bh[(size_t)row * ldn + x] = h;
                bl[(size_t)row * ldn + x] = l;
                th[(size_t)x * ldf + row] = h;
                tl[(size_t)x * ldf + row] = l;
            }
        }
    }
}

}  // namespace devel

using namespace devel;

// All iterations of one clip on stream s (the clip's optics workspace is used
// exclusively by this sequence of launches).
// alone: no other clip's kernels run beside this clip's (the resist kernel then takes
// one CTA per SM; with concurrent clips, CTAs of 256 threads that pack between theirs)
static int enqueue_clip(const devel_ilt_params* p, const devel_clip& cl, int* status, cudaStream_t s,
                        bool alone) {
    const devel_optics* o = cl.optics;
    const devel_optics* od = cl.optics_defocus;
    const int n = o->n;
    const Workspace& w = o->ws;
    float* phi = cl.phi;
    float* phi_alt = w.phi2;
    int rc;
    if (!cl.phi_given) {
        rc = launch_reinit(n, cl.target, phi, w.d2, p->d_lo, p->d_hi, s, 1, false);
        if (rc) return rc;
    }
    const bool tcp = o->precision == DEVEL_PREC_BF16X3;
    rc = launch_mask_from_phi(n, phi, w.M, s);
    if (rc) return rc;
    if (tcp) {  // later masks come out of the level-set step already in bf16
        rc = tc::launch_mask_bf16(w.M, n, o->ldn, o->Xhi, s);
        if (rc) return rc;
    }
    for (int t = 0; t <= p->iters; ++t) {
        // image the current mask, resist loss and dL/dI (in place in bufI)
        rc = tcp ? launch_spectrum_mask_resident(o, o->W, w.mhat, s) : launch_spectrum_u8(o, w.M, o->W, w.mhat, s);
        if (rc) return rc;
        double* lh = cl.loss_hist ? cl.loss_hist + t : nullptr;
        long long* l2h = cl.l2_hist ? cl.l2_hist + t : nullptr;
        long long* pvbh = cl.pvb_hist ? cl.pvb_hist + t : nullptr;
        if (od) {
            // defocused inner corner: both systems image the same mask (same spectrum)
            DEVEL_CUDA_TRY(cudaMemcpyAsync(od->ws.mhat, w.mhat, sizeof(float2) * o->k * o->k,
                                           cudaMemcpyDeviceToDevice, s));
            rc = forward_from_mhat(o, w.bufI, s);
            if (!rc) rc = forward_from_mhat(od, od->ws.bufI, s);
            if (!rc)
                rc = launch_resist_defocus(n, w.bufI, od->ws.bufI, cl.target, p->resist, tcp ? nullptr : w.bufI,
                                           tcp ? nullptr : od->ws.bufI, tcp ? o->Xhi : nullptr,
                                           tcp ? o->Xlo : nullptr, tcp ? od->Xhi : nullptr,
                                           tcp ? od->Xlo : nullptr, o->ldn, w.qpart, w.lpart, o->npart_red,
                                           nullptr, nullptr, lh, l2h, pvbh, status, w.counters, s, alone);
        } else {
            rc = forward_loss_from_mhat(o, cl.target, p->resist, nullptr, nullptr, lh, l2h, pvbh, status, s, alone);
        }
        if (rc) return rc;
        if (t == p->iters) break;  // the final mask is imaged for its metrics only
        if (od) {
            rc = tcp ? launch_spectrum_resident(o, o->W2, w.rhat, s)
                     : launch_spectrum_f32(o, w.bufI, o->W2, w.rhat, s);
            if (!rc)
                rc = tcp ? launch_spectrum_resident(od, od->W2, od->ws.rhat, s)
                         : launch_spectrum_f32(od, od->ws.bufI, od->W2, od->ws.rhat, s);
            if (!rc) rc = adjoint_from_rhat(o, w.bufV, w.vmax, status, s, od);
        } else {
            rc = adjoint_resident(o, w.bufV, w.vmax, status, s);
        }
        if (rc) return rc;
        const float* vel = w.bufV;
        const double* velmax = w.vmax;
        const int gi = p->start_iter + t;
        if (p->optimizer == DEVEL_OPT_CG) {
            // conjugate-gradient direction; restarts at the first iteration and after each
            // re-initialisation (global index), so a run resumed there is bit-identical
            const bool restart = t == 0 || (p->reinit_every > 0 && gi % p->reinit_every == 0);
            rc = launch_cg_direction(n, w.bufV, w.cgV, w.cgD, restart, w.cgpart, w.cgvpart, w.cgbeta, nullptr,
                                     w.counters + 2, w.cg_vmax, status, s);
            if (rc) return rc;
            vel = w.cgD;
            velmax = w.cg_vmax;
        }
        // the tensor-core forward reads the bf16 mask; the u8 mask then only feeds a
        // re-initialisation (which also overwrites phi) and the final mask output
        const bool reinit = p->reinit_every > 0 && (gi + 1) % p->reinit_every == 0;
        const bool keep_mask = !tcp || reinit || (t + 1 == p->iters && cl.mask_out);
        rc = launch_levelset_step(n, phi, vel, velmax, cl.m, p->dt, p->lambda, reinit ? nullptr : phi_alt,
                                  keep_mask ? w.M : nullptr, tcp ? o->Xhi : nullptr, o->ldn, s, p->upwind);
        if (rc) return rc;
        float* tmp = phi;
        phi = phi_alt;
        phi_alt = tmp;
        if (reinit) {
            rc = launch_reinit(n, w.M, phi, w.d2, p->d_lo, p->d_hi, s, 1, false);
            if (rc) return rc;
        }
    }
    if (phi != cl.phi)
        DEVEL_CUDA_TRY(cudaMemcpyAsync(cl.phi, phi, sizeof(float) * n * n, cudaMemcpyDeviceToDevice, s));
    if (cl.mask_out)
        DEVEL_CUDA_TRY(cudaMemcpyAsync(cl.mask_out, w.M, (size_t)n * n, cudaMemcpyDeviceToDevice, s));
    return DEVEL_OK;
}

// Several clips: clips that share an optics handle (and so its workspace) form a chain
// run in order; chains are spread over up to kBranches streams forked from s and
// joined back into it, so that independent clips' kernels run concurrently (as
// parallel branches when captured into a graph). Chains go longest first to the
// branch with the least work so far (work ~ n^2 per clip).
constexpr int kBranches = 16;
// Concurrent branches of a batch: kBranches, or DEVEL_MAX_BRANCHES (1 .. kBranches) from
// the environment.
static int branch_limit() {
    static const int lim = [] {
        const char* v = std::getenv("DEVEL_MAX_BRANCHES");
        const int b = v ? std::atoi(v) : 0;
        return b >= 1 && b <= kBranches ? b : kBranches;
    }();
    return lim;
}
struct BranchPool {
    cudaStream_t st[kBranches] = {};
    cudaEvent_t fork = nullptr, join[kBranches] = {};
    bool ready = false;
};
std::mutex g_branch_mu;
BranchPool g_branch[64];

// Streams and events of the device's branch pool (created on first use, outside any capture).
static int branch_pool(int dev, BranchPool** out) {
    BranchPool& b = g_branch[dev];
    if (!b.ready) {
        for (int i = 0; i < kBranches; ++i) {
            DEVEL_CUDA_TRY(cudaStreamCreateWithFlags(&b.st[i], cudaStreamNonBlocking));
            DEVEL_CUDA_TRY(cudaEventCreateWithFlags(&b.join[i], cudaEventDisableTiming));
        }
        DEVEL_CUDA_TRY(cudaEventCreateWithFlags(&b.fork, cudaEventDisableTiming));
        b.ready = true;
    }
    *out = &b;
    return DEVEL_OK;
}

static int enqueue_solve(const devel_ilt_params* p, int nclips, const devel_clip* clips, int* status,
                         cudaStream_t s, BranchPool* pool) {
    DEVEL_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), s));
    std::vector<const devel_optics*> handles;
    std::vector<std::vector<int>> chains;
    for (int c = 0; c < nclips; ++c) {
        size_t h = 0;
        while (h < handles.size() && handles[h] != clips[c].optics) ++h;
        if (h == handles.size()) {
            handles.push_back(clips[c].optics);
            chains.emplace_back();
        }
        chains[h].push_back(c);
    }
    if (chains.size() <= 1 || !pool) {
        for (int c = 0; c < nclips; ++c) {
            int rc = enqueue_clip(p, clips[c], status, s, true);
            if (rc) return rc;
        }
        return DEVEL_OK;
    }
    const int nb = (int)std::min<size_t>(chains.size(), (size_t)branch_limit());
    std::vector<double> cost(chains.size(), 0.0), load(nb, 0.0);
    std::vector<int> order(chains.size());
    for (size_t h = 0; h < chains.size(); ++h) {
        for (int c : chains[h]) cost[h] += (double)clips[c].optics->n * clips[c].optics->n;
        order[h] = (int)h;
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    std::vector<std::vector<int>> branch(nb);
    for (int h : order) {
        const int b = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        load[b] += cost[h];
        branch[b].push_back(h);
    }
    DEVEL_CUDA_TRY(cudaEventRecord(pool->fork, s));
    for (int b = 0; b < nb; ++b) {
        cudaStream_t bs = pool->st[b];
        DEVEL_CUDA_TRY(cudaStreamWaitEvent(bs, pool->fork, 0));
        for (int h : branch[b])
            for (int c : chains[h]) {
                int rc = enqueue_clip(p, clips[c], status, bs, false);
                if (rc) return rc;
            }
        DEVEL_CUDA_TRY(cudaEventRecord(pool->join[b], bs));
        DEVEL_CUDA_TRY(cudaStreamWaitEvent(s, pool->join[b], 0));
    }
    return DEVEL_OK;
}


// ---------------------------------------------------------------------------
// CUDA-graph replay of whole solves
// ---------------------------------------------------------------------------
// A solve is captured once per distinct (params, clip list) into a graph on an
// internal capture stream, then replayed with one cudaGraphLaunch on the
// caller's stream. Kernel arguments (pointers, sizes) are baked into the
// graph; the data they point to is read at replay time.
namespace {
struct GraphEntry {
    std::vector<unsigned char> key;
    cudaGraphExec_t exec = nullptr;
    int device = -1;
};
std::mutex g_graph_mu;
std::vector<GraphEntry> g_graphs;  // most recent last
constexpr size_t kMaxGraphs = 8;
cudaStream_t g_capture_stream[64] = {};

// A graph captured while a profile is open records the profiler's events; it is
// keyed by the profile generation (device slot replaced by ~generation) so it is
// never replayed after that profile closes.
std::vector<unsigned char> solve_key(const devel_ilt_params* p, int nclips, const devel_clip* clips, int* status,
                                     int device) {
    std::vector<unsigned char> k(sizeof(devel_ilt_params) + sizeof(int) * 2 + sizeof(int*) +
                                 sizeof(devel_clip) * nclips);
    unsigned char* q = k.data();
    std::memcpy(q, p, sizeof(devel_ilt_params));
    q += sizeof(devel_ilt_params);
    std::memcpy(q, &nclips, sizeof(int));
    q += sizeof(int);
    const int tag = prof_on() ? (int)(~prof_generation()) : device;
    std::memcpy(q, &tag, sizeof(int));
    q += sizeof(int);
    std::memcpy(q, &status, sizeof(int*));
    q += sizeof(int*);
    if (nclips) std::memcpy(q, clips, sizeof(devel_clip) * nclips);
    return k;
}
}  // namespace

static int solve_graph(const devel_ilt_params* p, int nclips, const devel_clip* clips, int* status,
                       cudaStream_t s) {
    int dev = 0;
    DEVEL_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return enqueue_solve(p, nclips, clips, status, s, nullptr);
    std::vector<unsigned char> key = solve_key(p, nclips, clips, status, dev);
    std::lock_guard<std::mutex> lock(g_graph_mu);
    for (size_t i = 0; i < g_graphs.size(); ++i) {
        if (g_graphs[i].device == dev && g_graphs[i].key == key) {
            GraphEntry e = g_graphs[i];
            g_graphs.erase(g_graphs.begin() + i);
            g_graphs.push_back(e);
            DEVEL_CUDA_TRY(cudaGraphLaunch(e.exec, s));
            return DEVEL_OK;
        }
    }
    if (!g_capture_stream[dev])
        DEVEL_CUDA_TRY(cudaStreamCreateWithFlags(&g_capture_stream[dev], cudaStreamNonBlocking));
    cudaStream_t cs = g_capture_stream[dev];
    BranchPool* pool = nullptr;
    {
        std::lock_guard<std::mutex> bl(g_branch_mu);
        int rc0 = branch_pool(dev, &pool);
        if (rc0) return rc0;
    }
    DEVEL_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_solve(p, nclips, clips, status, cs, pool);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(cs, &graph);
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return cuda_error(e, "devel_ilt_solve: cudaStreamEndCapture");
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_error(e, "devel_ilt_solve: cudaGraphInstantiate");
    if (g_graphs.size() >= kMaxGraphs) {
        cudaGraphExecDestroy(g_graphs.front().exec);
        g_graphs.erase(g_graphs.begin());
    }
    g_graphs.push_back(GraphEntry{key, exec, dev});
    DEVEL_CUDA_TRY(cudaGraphLaunch(exec, s));
    return DEVEL_OK;
}

// Drop cached graphs that reference a handle about to be destroyed.
static void drop_graphs_of(const devel_optics* o) {
    std::lock_guard<std::mutex> lock(g_graph_mu);
    for (size_t i = 0; i < g_graphs.size();) {
        const std::vector<unsigned char>& k = g_graphs[i].key;
        const size_t head = sizeof(devel_ilt_params) + sizeof(int) * 2 + sizeof(int*);
        bool uses = false;
        for (size_t off = head; off + sizeof(devel_clip) <= k.size(); off += sizeof(devel_clip)) {
            devel_clip c;
            std::memcpy(&c, k.data() + off, sizeof(devel_clip));
            if (c.optics == o || c.optics_defocus == o) uses = true;
        }
        if (uses) {
            cudaGraphExecDestroy(g_graphs[i].exec);
            g_graphs.erase(g_graphs.begin() + i);
        } else {
            ++i;
        }
    }
}

extern "C" {

const char* devel_last_error(void) { return g_err; }

int devel_version(void) { return (1 << 16) | 0; }

int devel_optics_n(const devel_optics* o) { return o ? o->n : -1; }

int devel_optics_create(int n, int K, int k, const float* H_host, const float* w_host,
                        int precision, devel_optics** out) {
    if (!out) return set_error(DEVEL_EINVAL, "devel_optics_create: out is NULL");
    *out = nullptr;
    if (!H_host || !w_host) return set_error(DEVEL_EINVAL, "devel_optics_create: H_host/w_host is NULL");
    if (n < 16 || n > 8192) return set_error(DEVEL_EINVAL, "devel_optics_create: n=%d outside [16, 8192]", n);
    if (k < 3 || (k % 2) == 0 || k > kMaxWindow)
        return set_error(DEVEL_EINVAL, "devel_optics_create: k=%d must be odd in [3, %d]", k, kMaxWindow);
    if (2 * k - 1 > n) return set_error(DEVEL_EINVAL, "devel_optics_create: 2k-1=%d exceeds n=%d", 2 * k - 1, n);
    if (K < 1 || K > k * k) return set_error(DEVEL_EINVAL, "devel_optics_create: K=%d outside [1, k*k]", K);
    if (precision != DEVEL_PREC_FP32 && precision != DEVEL_PREC_BF16X3)
        return set_error(DEVEL_EINVAL, "devel_optics_create: unknown precision %d", precision);
    for (int j = 0; j < K; ++j)
        if (!(w_host[j] >= 0.f) || !std::isfinite(w_host[j]))
            return set_error(DEVEL_EINVAL, "devel_optics_create: w[%d] must be finite and >= 0", j);

    {
        int rc0 = init_device_attrs();
        if (rc0) return rc0;
    }
    devel_optics* o = new devel_optics();
    o->n = n;
    o->K = K;
    o->k = k;
    o->r = (k - 1) / 2;
    o->k2 = 2 * k - 1;
    o->r2 = k - 1;
    o->precision = precision;
    o->W.kw = k;
    o->W.ldk = round_up(2 * k, 16);
    o->W2.kw = o->k2;
    o->W2.ldk = round_up(2 * o->k2, 16);
    o->ldn = round_up(n, 64);
    if (precision == DEVEL_PREC_BF16X3) {
        o->nsplit = o->ldn / 256 + (o->ldn % 256 ? 1 : 0);  // 256-wide K slices of the tc reduction
    } else {
        int ns = (n + 255) / 256;
        o->nsplit = ns < 1 ? 1 : (ns > 16 ? 16 : ns);
    }
    const size_t npix = (size_t)n * n;
    const int kk = k * k, kk2 = o->k2 * o->k2;
    const int nred = std::max(resist_parts(n), expand_parts(n));  // CTA partials of any loss reduction
    o->npart_red = resist_parts(n);
    const int ld2 = o->W2.ldk;

#define ALLOC(ptr, bytes)                                                                  \
    do {                                                                                   \
        cudaError_t e_ = cudaMalloc((void**)&(ptr), (bytes));                              \
        if (e_ != cudaSuccess) {                                                           \
            cudaGetLastError();                                                            \
            free_optics(o);                                                                \
            return set_error(DEVEL_ENOMEM, "devel_optics_create: cudaMalloc(%zu): %s",     \
                             (size_t)(bytes), cudaGetErrorString(e_));                     \
        }                                                                                  \
    } while (0)

    ALLOC(o->W.basis, sizeof(float) * o->W.ldk * n);
    ALLOC(o->W.basisT, sizeof(float) * o->W.ldk * n);
    ALLOC(o->W2.basis, sizeof(float) * ld2 * n);
    ALLOC(o->W2.basisT, sizeof(float) * ld2 * n);
    ALLOC(o->TCC, sizeof(float2) * (size_t)kk * kk);
    ALLOC(o->Tdiff, sizeof(float2) * (size_t)kk * kk);
    ALLOC(o->goff, sizeof(int) * kk2);
    ALLOC(o->ws.Ppart, sizeof(float) * (size_t)o->nsplit * n * ld2);
    o->nq = std::max(1, std::min(16, n / 128));
    ALLOC(o->ws.P, sizeof(float) * (size_t)n * ld2);
    // the fused reduction's slices, for the narrowest split the tuner may pick (at most
    // 256 slices)
    if (precision == DEVEL_PREC_BF16X3) {
        o->tc_split = std::min(256, o->ldn);
        o->tc_split_min = o->tc_split;
        while (o->tc_split_min > 64 && tc::spectrum2_slices(n, o->ldn, o->tc_split_min / 2) <= 256)
            o->tc_split_min /= 2;
    }
    const size_t nslices = precision == DEVEL_PREC_BF16X3
                               ? (size_t)std::max(o->nq, tc::spectrum2_slices(n, o->ldn, o->tc_split_min))
                               : (size_t)o->nq;
    ALLOC(o->ws.Q, sizeof(float) * nslices * ld2 * ld2);
    ALLOC(o->ws.mhat, sizeof(float2) * kk);
    ALLOC(o->ws.Ihat, sizeof(float2) * kk2);
    ALLOC(o->ws.rhat, sizeof(float2) * kk2);
    ALLOC(o->ws.Shat, sizeof(float2) * kk);
    ALLOC(o->ws.Acat, sizeof(float) * (size_t)n * ld2);
    ALLOC(o->ws.qpart, sizeof(long long) * 3 * nred);
    ALLOC(o->ws.lpart, sizeof(long long) * 2 * nred);
    ALLOC(o->ws.vpart, sizeof(float) * expand_parts(n));
    ALLOC(o->ws.vbits, sizeof(unsigned));
    ALLOC(o->ws.bufI, sizeof(float) * npix);
    ALLOC(o->ws.bufV, sizeof(float) * npix);
    ALLOC(o->ws.phi2, sizeof(float) * npix);
    ALLOC(o->ws.M, npix);
    ALLOC(o->ws.d2, sizeof(int) * npix);
    ALLOC(o->ws.vmax, sizeof(double));
    ALLOC(o->ws.loss4, sizeof(double) * 4);
    ALLOC(o->ws.cnt2, sizeof(long long) * 2);
    ALLOC(o->tc_err, sizeof(int));
    ALLOC(o->ws.counters, sizeof(unsigned) * 8);
    ALLOC(o->ws.cgpart, sizeof(float) * 3 * cg_parts(n));
    ALLOC(o->ws.cgvpart, sizeof(float) * cg_parts(n));
    ALLOC(o->ws.cgbeta, sizeof(float));
    ALLOC(o->ws.cg_vmax, sizeof(double));
    ALLOC(o->ws.cgV, sizeof(float) * npix);
    ALLOC(o->ws.cgD, sizeof(float) * npix);
    if (precision == DEVEL_PREC_BF16X3) {
        const size_t bf = sizeof(__nv_bfloat16);
        o->tcW.ldf = round_up(k, 16);
        o->tcW2.ldf = round_up(o->k2, 16);
        for (TcWindow* tw : {&o->tcW, &o->tcW2}) {
            const int ldf = tw->ldf;
            ALLOC(tw->basis_hi, bf * round_up(ldf, 128) * o->ldn);
            ALLOC(tw->basis_lo, bf * round_up(ldf, 128) * o->ldn);
            ALLOC(tw->basisT_hi, bf * (size_t)n * ldf);
            ALLOC(tw->basisT_lo, bf * (size_t)n * ldf);
            ALLOC(tw->zm_hi, bf * (size_t)ldf * ldf);
            ALLOC(tw->zm_lo, bf * (size_t)ldf * ldf);
        }
        ALLOC(o->Xhi, bf * (size_t)n * o->ldn);
        ALLOC(o->Xlo, bf * (size_t)n * o->ldn);
        ALLOC(o->Acat_hi, bf * (size_t)n * o->tcW2.ldf);
        ALLOC(o->Acat_lo, bf * (size_t)n * o->tcW2.ldf);
    }
#undef ALLOC

    // DFT tables of both windows
    std::vector<float> b1, b1T, b2, b2T;
    make_basis(n, k, o->W.ldk, b1, b1T);
    make_basis(n, o->k2, ld2, b2, b2T);
    // rank-K TCC in double: TCC(a, b) = sum_j w_j H_j(a) conj(H_j(b))  (Sec. II-B)
    std::vector<double> Hr((size_t)K * kk), Hi((size_t)K * kk);
    for (int j = 0; j < K; ++j) {
        const double sw = std::sqrt((double)w_host[j]);
        for (int i = 0; i < kk; ++i) {
            Hr[(size_t)j * kk + i] = sw * H_host[((size_t)j * kk + i) * 2];
            Hi[(size_t)j * kk + i] = sw * H_host[((size_t)j * kk + i) * 2 + 1];
        }
    }
    std::vector<float2> tcc((size_t)kk * kk);
    for (int a = 0; a < kk; ++a) {
        for (int b = 0; b < kk; ++b) {
            double re = 0.0, im = 0.0;
            for (int j = 0; j < K; ++j) {
                const double ar = Hr[(size_t)j * kk + a], ai = Hi[(size_t)j * kk + a];
                const double br = Hr[(size_t)j * kk + b], bi = Hi[(size_t)j * kk + b];
                re += ar * br + ai * bi;
                im += ai * br - ar * bi;
            }
            tcc[(size_t)a * kk + b] = make_float2((float)re, (float)im);
        }
    }
    // grouped by difference g = a - b in W2: rect(g) = {a : a - g in W}, row-major
    std::vector<float2> tdiff((size_t)kk * kk);
    std::vector<int> goff(kk2);
    {
        size_t off = 0;
        const int r2 = o->r2;
        for (int c1 = 0; c1 < o->k2; ++c1) {
            for (int c2 = 0; c2 < o->k2; ++c2) {
                goff[c1 * o->k2 + c2] = (int)off;
                const int a1lo = std::max(0, c1 - r2), a1hi = std::min(k, c1 - r2 + k);
                const int a2lo = std::max(0, c2 - r2), a2hi = std::min(k, c2 - r2 + k);
                for (int a1 = a1lo; a1 < a1hi; ++a1)
                    for (int a2 = a2lo; a2 < a2hi; ++a2) {
                        const int b1 = a1 - c1 + r2, b2 = a2 - c2 + r2;
                        tdiff[off++] = tcc[(size_t)(a1 * k + a2) * kk + (b1 * k + b2)];
                    }
            }
        }
    }
    cudaError_t e = cudaSuccess;
    struct Cp { void* d; const void* h; size_t bytes; } cps[] = {
        {o->W.basis, b1.data(), b1.size() * sizeof(float)},
        {o->W.basisT, b1T.data(), b1T.size() * sizeof(float)},
        {o->W2.basis, b2.data(), b2.size() * sizeof(float)},
        {o->W2.basisT, b2T.data(), b2T.size() * sizeof(float)},
        {o->TCC, tcc.data(), tcc.size() * sizeof(float2)},
        {o->Tdiff, tdiff.data(), tdiff.size() * sizeof(float2)},
        {o->goff, goff.data(), goff.size() * sizeof(int)},
    };
    for (const Cp& c : cps)
        if (e == cudaSuccess) e = cudaMemcpy(c.d, c.h, c.bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(o->tc_err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(o->ws.counters, 0, sizeof(unsigned) * 8);
    if (e == cudaSuccess) e = cudaMemset(o->ws.vbits, 0, sizeof(unsigned));
    if (e != cudaSuccess) {
        free_optics(o);
        return cuda_error(e, "devel_optics_create: cudaMemcpy");
    }
    if (precision == DEVEL_PREC_BF16X3) {
        // folded bf16 hi/lo DFT tables and their tensor maps
        int rc = DEVEL_OK;
        std::vector<__nv_bfloat16> bh, bl, th, tl;
        for (int wi = 0; wi < 2 && rc == DEVEL_OK; ++wi) {
            const Window& w = wi ? o->W2 : o->W;
            TcWindow& tw = wi ? o->tcW2 : o->tcW;
            const int ldf = tw.ldf, rows128 = round_up(ldf, 128);
            make_basis_folded(n, w.kw, ldf, rows128, o->ldn, bh, bl, th, tl);
            const size_t bf = sizeof(__nv_bfloat16);
            if (cudaMemcpy(tw.basis_hi, bh.data(), bf * bh.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
                cudaMemcpy(tw.basis_lo, bl.data(), bf * bl.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
                cudaMemcpy(tw.basisT_hi, th.data(), bf * th.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
                cudaMemcpy(tw.basisT_lo, tl.data(), bf * tl.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
                rc = set_error(DEVEL_ECUDA, "devel_optics_create: cudaMemcpy of the folded tables");
                break;
            }
            rc = tc::make_map(&tw.m_basis128_hi, tw.basis_hi, rows128, o->ldn, o->ldn, 128);
            if (!rc) rc = tc::make_map(&tw.m_basis128_lo, tw.basis_lo, rows128, o->ldn, o->ldn, 128);
            if (!rc) rc = tc::make_map(&tw.m_basis_hi, tw.basis_hi, ldf, o->ldn, o->ldn, ldf);
            if (!rc) rc = tc::make_map(&tw.m_basis_lo, tw.basis_lo, ldf, o->ldn, o->ldn, ldf);
            if (!rc) rc = tc::make_map(&tw.m_basisT_hi, tw.basisT_hi, n, ldf, ldf, 128);
            if (!rc) rc = tc::make_map(&tw.m_basisT_lo, tw.basisT_lo, n, ldf, ldf, 128);
            // Zm entries outside the window's kw x kw block are never written: zero them once
            if (!rc && (cudaMemset(tw.zm_hi, 0, bf * ldf * ldf) != cudaSuccess ||
                        cudaMemset(tw.zm_lo, 0, bf * ldf * ldf) != cudaSuccess))
                rc = set_error(DEVEL_ECUDA, "devel_optics_create: cudaMemset");
            if (!rc) rc = tc::make_map3(&tw.m_zm_hi, tw.zm_hi, 1, ldf, ldf, ldf, (size_t)ldf * ldf, kTileT);
            if (!rc) rc = tc::make_map3(&tw.m_zm_lo, tw.zm_lo, 1, ldf, ldf, ldf, (size_t)ldf * ldf, kTileT);
            if (!rc) rc = tc::make_map3(&tw.m_zmw_hi, tw.zm_hi, 1, ldf, ldf, ldf, (size_t)ldf * ldf, ldf);
            if (!rc) rc = tc::make_map3(&tw.m_zmw_lo, tw.zm_lo, 1, ldf, ldf, ldf, (size_t)ldf * ldf, ldf);
            if (!rc) rc = tc::make_map(&tw.m_basisT64_hi, tw.basisT_hi, n, ldf, ldf, 64);
            if (!rc) rc = tc::make_map(&tw.m_basisT64_lo, tw.basisT_lo, n, ldf, ldf, 64);
            if (!rc) rc = tc::make_map3(&tw.m_acat_hi, o->Acat_hi, 1, n, ldf, ldf, (size_t)n * ldf, 128);
            if (!rc) rc = tc::make_map3(&tw.m_acat_lo, o->Acat_lo, 1, n, ldf, ldf, (size_t)n * ldf, 128);
        }
        // the operand's pad columns [n, ldn) must read as zeros: only kernels that
        // write zeros there (or nothing) ever touch them afterwards
        if (!rc && (cudaMemset(o->Xhi, 0, sizeof(__nv_bfloat16) * (size_t)n * o->ldn) != cudaSuccess ||
                    cudaMemset(o->Xlo, 0, sizeof(__nv_bfloat16) * (size_t)n * o->ldn) != cudaSuccess))
            rc = set_error(DEVEL_ECUDA, "devel_optics_create: cudaMemset");
        if (!rc) rc = tc::make_map3(&o->m_X_hi, o->Xhi, 1, n, o->ldn, o->ldn, (size_t)n * o->ldn, 128);
        if (!rc) rc = tc::make_map3(&o->m_X_lo, o->Xlo, 1, n, o->ldn, o->ldn, (size_t)n * o->ldn, 128);
        if (!rc) {
            cudaError_t e2 = cudaDeviceSynchronize();
            if (e2 != cudaSuccess) rc = cuda_error(e2, "devel_optics_create: table split");
        }
        if (rc) {
            free_optics(o);
            return rc;
        }
    }
    *out = o;
    return DEVEL_OK;
}

int devel_optics_destroy(devel_optics* o) {
    if (!o) return DEVEL_OK;
    drop_graphs_of(o);
    cudaError_t e = cudaDeviceSynchronize();
    free_optics(o);
    if (e != cudaSuccess) return cuda_error(e, "devel_optics_destroy: cudaDeviceSynchronize");
    return DEVEL_OK;
}

// Tile-shape tuner: times each candidate on the handle's own tables and workspace
// (whatever they hold; the timing does not depend on the values) and keeps the fastest.
// Tuned: the output tile width of the tensor-core expansion and the image columns per
// CTA of the fused reduction (which sets its grid: narrow clips want narrow slices to
// fill the SMs). The FP32 path has nothing to tune.
int devel_optics_autotune(devel_optics* o, cudaStream_t s) {
    if (!o) return set_error(DEVEL_EINVAL, "devel_optics_autotune: optics is NULL");
    if (o->precision != DEVEL_PREC_BF16X3) return DEVEL_OK;
    int rc = init_device_attrs();
    if (rc) return rc;
    cudaEvent_t a = nullptr, b = nullptr;
    DEVEL_CUDA_TRY(cudaEventCreate(&a));
    cudaError_t ce = cudaEventCreate(&b);
    if (ce != cudaSuccess) {
        cudaEventDestroy(a);
        return cuda_error(ce, "devel_optics_autotune: cudaEventCreate");
    }
    constexpr int kReps = 5;
    // the two expansions and the two reductions of one iteration
    auto expand_pair = [&]() -> int {
        EpiArgs e1;
        e1.C = o->ws.bufI;
        int r = launch_expand(o, o->ws.Ihat, o->W2, EPI_STORE, e1, nullptr, s);
        EpiArgs e2;
        e2.C = o->ws.bufV;
        return r ? r : launch_expand(o, o->ws.Shat, o->W, EPI_STORE, e2, nullptr, s);
    };
    auto reduce_pair = [&]() -> int {
        int r = launch_spectrum_mask_resident(o, o->W, o->ws.mhat, s);
        return r ? r : launch_spectrum_resident(o, o->W2, o->ws.rhat, s);
    };
    auto time_of = [&](auto&& fn, float* ms) -> int {
        int r = fn();  // warm-up
        for (int i = 0; i < kReps && !r; ++i) {
            if (i == 0 && cudaEventRecord(a, s) != cudaSuccess) r = set_error(DEVEL_ECUDA, "autotune: event");
            if (!r) r = fn();
        }
        if (!r && (cudaEventRecord(b, s) != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess ||
                   cudaEventElapsedTime(ms, a, b) != cudaSuccess))
            r = set_error(DEVEL_ECUDA, "devel_optics_autotune: event timing");
        return r;
    };
    float best = 1e30f, t = 0.f;
    int best_bn = o->tc_expand_bn, best_split = o->tc_split;
    for (int bn : {64, 128}) {
        o->tc_expand_bn = bn;
        rc = time_of(expand_pair, &t);
        if (rc) break;
        if (t < best) {
            best = t;
            best_bn = bn;
        }
    }
    o->tc_expand_bn = best_bn;
    best = 1e30f;
    for (int split = o->tc_split_min; !rc && split <= std::min(512, o->ldn); split *= 2) {
        if (o->ldn % 64) break;
        o->tc_split = split;
        rc = time_of(reduce_pair, &t);
        if (!rc && t < best) {
            best = t;
            best_split = split;
        }
    }
    o->tc_split = best_split;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    drop_graphs_of(o);  // graphs captured with the old shapes
    return rc;
}

int devel_optics_config(const devel_optics* o, int* expand_tile_n, int* reduce_split) {
    if (!o) return set_error(DEVEL_EINVAL, "devel_optics_config: optics is NULL");
    if (expand_tile_n) *expand_tile_n = o->precision == DEVEL_PREC_BF16X3 ? o->tc_expand_bn : 0;
    if (reduce_split) *reduce_split = o->precision == DEVEL_PREC_BF16X3 ? o->tc_split : 0;
    return DEVEL_OK;
}

int devel_selftest_bounded_wait(const devel_optics* o, cudaStream_t s) {
    if (!o) return set_error(DEVEL_EINVAL, "devel_selftest_bounded_wait: optics is NULL");
    return tc::launch_wait_selftest(o->tc_err, s);
}

int devel_optics_check(const devel_optics* o, cudaStream_t s) {
    if (!o) return set_error(DEVEL_EINVAL, "devel_optics_check: optics is NULL");
    DEVEL_CUDA_TRY(cudaStreamSynchronize(s));
    int flag = 0;
    DEVEL_CUDA_TRY(cudaMemcpy(&flag, o->tc_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (flag) {
        DEVEL_CUDA_TRY(cudaMemset(o->tc_err, 0, sizeof(int)));
        return set_error(flag, "devel_optics_check: a bounded device wait gave up (code %d)", flag);
    }
    return DEVEL_OK;
}

int devel_litho_forward(const devel_optics* o, const float* mask, float* intensity, cudaStream_t s) {
    if (!o) return set_error(DEVEL_EINVAL, "devel_litho_forward: optics is NULL");
    CHECK_PTR(mask, "mask");
    CHECK_PTR(intensity, "intensity");
    if ((const void*)mask == (const void*)intensity)
        return set_error(DEVEL_EINVAL, "devel_litho_forward: mask aliases intensity");
    int rc = launch_spectrum_f32(o, mask, o->W, o->ws.mhat, s);
    if (rc) return rc;
    return forward_from_mhat(o, intensity, s);
}

int devel_resist_loss(const devel_optics* o, const float* intensity, const unsigned char* target,
                      const devel_resist_params* p, float* dLdI, double* loss_out,
                      long long* counts_out, cudaStream_t s) {
    if (!o) return set_error(DEVEL_EINVAL, "devel_resist_loss: optics is NULL");
    if (!p) return set_error(DEVEL_EINVAL, "devel_resist_loss: params is NULL");
    CHECK_PTR(intensity, "intensity");
    CHECK_PTR(target, "target");
    CHECK_PTR(dLdI, "dLdI");
    CHECK_PTR(loss_out, "loss_out");
    CHECK_PTR(counts_out, "counts_out");
    return launch_resist(o->n, intensity, target, *p, dLdI, nullptr, nullptr, 0, o->ws.qpart, o->ws.lpart,
                         o->npart_red, loss_out, counts_out, nullptr, nullptr, nullptr, nullptr, o->ws.counters, s);
}

int devel_litho_adjoint(const devel_optics* o, const float* mask, const float* dLdI, float* dLdM,
                        double* vmax, cudaStream_t s) {
    if (!o) return set_error(DEVEL_EINVAL, "devel_litho_adjoint: optics is NULL");
    CHECK_PTR(mask, "mask");
    CHECK_PTR(dLdI, "dLdI");
    CHECK_PTR(dLdM, "dLdM");
    CHECK_PTR(vmax, "vmax");
    int rc = launch_spectrum_f32(o, mask, o->W, o->ws.mhat, s);
    if (rc) return rc;
    return adjoint_from_mhat(o, dLdI, dLdM, vmax, nullptr, s);
}

static int levelset_step_checked(int n, const float* phi, const float* V, const double* vmax, const float* m,
                                 float dt, float lambda, float* phi_out, unsigned char* mask_out, cudaStream_t s,
                                 int upwind) {
    if (n < 1 || n > 16384) return set_error(DEVEL_EINVAL, "devel_levelset_step: n=%d outside [1, 16384]", n);
    CHECK_PTR(phi, "phi");
    CHECK_PTR(V, "V");
    CHECK_PTR(vmax, "vmax");
    CHECK_PTR(phi_out, "phi_out");
    CHECK_OPT_PTR(m, "m");
    CHECK_OPT_PTR(mask_out, "mask_out");
    if (phi == phi_out) return set_error(DEVEL_EINVAL, "devel_levelset_step: phi_out aliases phi");
    if (!std::isfinite(dt) || !std::isfinite(lambda))
        return set_error(DEVEL_EINVAL, "devel_levelset_step: dt/lambda not finite");
    return launch_levelset_step(n, phi, V, vmax, m, dt, lambda, phi_out, mask_out, nullptr, 0, s, upwind);
}

int devel_levelset_step(int n, const float* phi, const float* V, const double* vmax, const float* m,
                        float dt, float lambda, float* phi_out, unsigned char* mask_out, cudaStream_t s) {
    return levelset_step_checked(n, phi, V, vmax, m, dt, lambda, phi_out, mask_out, s, DEVEL_UPWIND_GODUNOV1);
}

int devel_levelset_step_weno5(int n, const float* phi, const float* V, const double* vmax, const float* m,
                              float dt, float lambda, float* phi_out, unsigned char* mask_out, cudaStream_t s) {
    return levelset_step_checked(n, phi, V, vmax, m, dt, lambda, phi_out, mask_out, s, DEVEL_UPWIND_WENO5);
}

int devel_reinit_sdf(int n, const unsigned char* mask, float* phi, int* d2, float d_lo, float d_hi,
                     cudaStream_t s) {
    if (n < 1 || n > 8192) return set_error(DEVEL_EINVAL, "devel_reinit_sdf: n=%d outside [1, 8192]", n);
    CHECK_PTR(mask, "mask");
    CHECK_PTR(phi, "phi");
    CHECK_PTR(d2, "d2");
    if (!(d_lo <= d_hi)) return set_error(DEVEL_EINVAL, "devel_reinit_sdf: d_lo > d_hi");
    int rc = init_device_attrs();
    if (rc) return rc;
    return launch_reinit(n, mask, phi, d2, d_lo, d_hi, s);
}

int devel_reinit_sdf_batch(int n, int nb, const unsigned char* mask, float* phi, int* d2, float d_lo, float d_hi,
                           cudaStream_t s) {
    if (n < 1 || n > 8192) return set_error(DEVEL_EINVAL, "devel_reinit_sdf_batch: n=%d outside [1, 8192]", n);
    if (nb < 1 || nb > 65535) return set_error(DEVEL_EINVAL, "devel_reinit_sdf_batch: nb=%d outside [1, 65535]", nb);
    CHECK_PTR(mask, "mask");
    CHECK_PTR(phi, "phi");
    CHECK_PTR(d2, "d2");
    if (!(d_lo <= d_hi)) return set_error(DEVEL_EINVAL, "devel_reinit_sdf_batch: d_lo > d_hi");
    int rc = init_device_attrs();
    if (rc) return rc;
    return launch_reinit(n, mask, phi, d2, d_lo, d_hi, s, nb);
}

int devel_modulation_candidates(int n, const float* phi_gt, int ncand, const float* dh_host, float* m_out,
                                cudaStream_t s) {
    if (n < 1 || n > 8192) return set_error(DEVEL_EINVAL, "devel_modulation_candidates: n=%d outside [1, 8192]", n);
    if (ncand < 1 || ncand > DEVEL_MOD_MAX_CANDIDATES)
        return set_error(DEVEL_EINVAL, "devel_modulation_candidates: ncand=%d outside [1, %d]", ncand,
                         DEVEL_MOD_MAX_CANDIDATES);
    CHECK_PTR(phi_gt, "phi_gt");
    CHECK_PTR(m_out, "m_out");
    if (!dh_host) return set_error(DEVEL_EINVAL, "devel_modulation_candidates: dh_host is NULL");
    for (int j = 0; j < ncand; ++j)
        if (!std::isfinite(dh_host[j]))
            return set_error(DEVEL_EINVAL, "devel_modulation_candidates: dh[%d] is not finite", j);
    return launch_mod_candidates(n, phi_gt, ncand, dh_host, m_out, s);
}

int devel_modulation_search(const devel_ilt_params* p, int ncand, devel_optics* const* handles,
                            const unsigned char* target, const float* phi_gt, const float* dh_host, float* m_out,
                            float* phi_work, double* loss_hist, int ldh, int* best_dev, int* status_dev,
                            cudaStream_t s) {
    if (!p) return set_error(DEVEL_EINVAL, "devel_modulation_search: params is NULL");
    if (ncand < 1 || ncand > DEVEL_MOD_MAX_CANDIDATES)
        return set_error(DEVEL_EINVAL, "devel_modulation_search: ncand=%d outside [1, %d]", ncand,
                         DEVEL_MOD_MAX_CANDIDATES);
    if (!handles || !handles[0]) return set_error(DEVEL_EINVAL, "devel_modulation_search: handles is NULL");
    const int n = handles[0]->n;
    for (int j = 1; j < ncand; ++j)
        if (!handles[j] || handles[j]->n != n)
            return set_error(DEVEL_EINVAL, "devel_modulation_search: handle %d missing or of another size", j);
    if (p->iters < 0 || ldh < p->iters + 1 || (ldh & 1))
        return set_error(DEVEL_EINVAL, "devel_modulation_search: ldh=%d must be even and >= iters + 1", ldh);
    CHECK_PTR(target, "target");
    CHECK_PTR(phi_gt, "phi_gt");
    CHECK_PTR(m_out, "m_out");
    CHECK_PTR(phi_work, "phi_work");
    CHECK_PTR(loss_hist, "loss_hist");
    CHECK_PTR(best_dev, "best_dev");
    CHECK_PTR(status_dev, "status_dev");
    if (!dh_host) return set_error(DEVEL_EINVAL, "devel_modulation_search: dh_host is NULL");
    for (int j = 0; j < ncand; ++j)
        if (!std::isfinite(dh_host[j]))
            return set_error(DEVEL_EINVAL, "devel_modulation_search: dh[%d] is not finite", j);
    int rc = launch_mod_candidates(n, phi_gt, ncand, dh_host, m_out, s);
    if (rc) return rc;
    const size_t N = (size_t)n * n;
    std::vector<devel_clip> clips(ncand);
    for (int j = 0; j < ncand; ++j) {
        devel_clip& c = clips[j];
        std::memset(&c, 0, sizeof(c));
        c.optics = handles[j];
        c.target = target;
        c.phi = phi_work + (size_t)j * N;
        c.phi_given = 0;
        c.m = m_out + (size_t)j * N;
        c.loss_hist = loss_hist + (size_t)j * ldh;
    }
    rc = devel_ilt_solve(p, ncand, clips.data(), status_dev, s);
    if (rc) return rc;
    return launch_argmin_final(loss_hist, ncand, ldh, p->iters, best_dev, s);
}

int devel_ahf_loss(const devel_optics* o, const float* phi_m, const float* m_gt, float eps, double* loss_out,
                   float* grad_out, cudaStream_t s) {
    if (!o) return set_error(DEVEL_EINVAL, "devel_ahf_loss: optics is NULL");
    CHECK_PTR(phi_m, "phi_m");
    CHECK_PTR(m_gt, "m_gt");
    CHECK_PTR(loss_out, "loss_out");
    CHECK_OPT_PTR(grad_out, "grad_out");
    if (!(eps > 0.f) || !std::isfinite(eps)) return set_error(DEVEL_EINVAL, "devel_ahf_loss: eps must be > 0");
    return launch_ahf_loss(o->n, phi_m, m_gt, eps, grad_out, o->ws.qpart, o->npart_red, o->ws.counters + 4, loss_out,
                           s);
}

int devel_cg_direction(const devel_optics* o, const float* V, float* Vprev, float* D, int restart,
                       double* beta_out, double* vmax_out, int* status, cudaStream_t s) {
    if (!o) return set_error(DEVEL_EINVAL, "devel_cg_direction: optics is NULL");
    CHECK_PTR(V, "V");
    CHECK_PTR(Vprev, "Vprev");
    CHECK_PTR(D, "D");
    CHECK_PTR(vmax_out, "vmax_out");
    CHECK_OPT_PTR(beta_out, "beta_out");
    CHECK_OPT_PTR(status, "status");
    if ((const void*)V == (const void*)Vprev || (const void*)V == (const void*)D || Vprev == D)
        return set_error(DEVEL_EINVAL, "devel_cg_direction: V, Vprev and D must be distinct arrays");
    return launch_cg_direction(o->n, V, Vprev, D, restart != 0, o->ws.cgpart, o->ws.cgvpart, o->ws.cgbeta,
                               beta_out, o->ws.counters + 2, vmax_out, status, s);
}

int devel_ilt_solve(const devel_ilt_params* p, int nclips, const devel_clip* clips, int* status,
                    cudaStream_t s) {
    if (!p) return set_error(DEVEL_EINVAL, "devel_ilt_solve: params is NULL");
    if (nclips < 0 || (nclips > 0 && !clips)) return set_error(DEVEL_EINVAL, "devel_ilt_solve: bad clip list");
    CHECK_PTR(status, "status_dev");
    if (p->iters < 0 || p->reinit_every < 0 || p->start_iter < 0)
        return set_error(DEVEL_EINVAL, "devel_ilt_solve: negative iters/reinit_every/start_iter");
    if (!(p->d_lo <= p->d_hi)) return set_error(DEVEL_EINVAL, "devel_ilt_solve: d_lo > d_hi");
    if (p->upwind != DEVEL_UPWIND_GODUNOV1 && p->upwind != DEVEL_UPWIND_WENO5)
        return set_error(DEVEL_EINVAL, "devel_ilt_solve: unknown upwind scheme %d", p->upwind);
    if (p->optimizer != DEVEL_OPT_STEEPEST && p->optimizer != DEVEL_OPT_CG)
        return set_error(DEVEL_EINVAL, "devel_ilt_solve: unknown optimizer %d", p->optimizer);
    for (int c = 0; c < nclips; ++c) {
        const devel_clip& cl = clips[c];
        if (!cl.optics) return set_error(DEVEL_EINVAL, "devel_ilt_solve: clip %d has no optics", c);
        CHECK_PTR(cl.target, "clip.target");
        CHECK_PTR(cl.phi, "clip.phi");
        CHECK_OPT_PTR(cl.m, "clip.m");
        CHECK_OPT_PTR(cl.mask_out, "clip.mask_out");
        CHECK_OPT_PTR(cl.loss_hist, "clip.loss_hist");
        CHECK_OPT_PTR(cl.l2_hist, "clip.l2_hist");
        CHECK_OPT_PTR(cl.pvb_hist, "clip.pvb_hist");
        if (const devel_optics* od = cl.optics_defocus) {
            if (od == cl.optics || od->n != cl.optics->n || od->k != cl.optics->k ||
                od->precision != cl.optics->precision)
                return set_error(DEVEL_EINVAL,
                                 "devel_ilt_solve: clip %d: the defocus optics must be a separate handle with the "
                                 "same n, window and precision",
                                 c);
            for (int d = 0; d < nclips; ++d) {  // its workspace belongs to this clip's chain alone
                if (clips[d].optics == od ||
                    (clips[d].optics_defocus == od && clips[d].optics != cl.optics))
                    return set_error(DEVEL_EINVAL, "devel_ilt_solve: clip %d: defocus handle shared", c);
            }
        }
    }
    if (p->use_graph) return solve_graph(p, nclips, clips, status, s);
    int dev = 0;
    DEVEL_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return enqueue_solve(p, nclips, clips, status, s, nullptr);
    std::lock_guard<std::mutex> bl(g_branch_mu);  // the pool's events serve one call at a time
    BranchPool* pool = nullptr;
    int rc = branch_pool(dev, &pool);
    if (rc) return rc;
    return enqueue_solve(p, nclips, clips, status, s, pool);
}

}  // extern "C"
