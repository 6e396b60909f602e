// Batched DSO solve (Sec. III-A / III-C): the loop of devel_ilt_solve with every stage
// launched once over a batch of clips that share one compensated-BF16 optics handle.
//
// A batch owns the per-clip workspace of `capacity` clips (clip c of every array at c
// times its single-clip size, the tensor maps of the operands 3-D over the clips) and a
// view of its handle: a copy of the handle's struct whose tables (DFT tables, TCC) are
// the handle's and whose workspace pointers and maps are the batch's, with `batch` set to
// the number of clips of the call. The launchers that serve a single clip then launch one
// grid over all clips (the clip is one more grid dimension, or part of a persistent
// kernel's tile range), so each launch moves the whole batch's images.
#include <algorithm>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "tc.cuh"

struct devel_batch {
    const devel_optics* base = nullptr;
    int capacity = 0;
    devel_optics view;               // the handle's tables, this batch's workspace
    unsigned* rcount = nullptr;      // [capacity] zeroed: the resist's last-block counters
    std::vector<void*> owned;        // device allocations of the batch
    struct Graph {
        std::vector<unsigned char> key;
        cudaGraphExec_t exec = nullptr;
    };
    std::vector<Graph> graphs;       // captured solves, most recent last
    cudaStream_t capture = nullptr;  // internal capture stream
};

namespace devel {
namespace {

constexpr size_t kMaxBatchGraphs = 4;

void free_batch(devel_batch* b) {
    if (!b) return;
    for (auto& g : b->graphs)
        if (g.exec) cudaGraphExecDestroy(g.exec);
    for (void* p : b->owned)
        if (p) cudaFree(p);
    if (b->capture) cudaStreamDestroy(b->capture);
    delete b;
}

int round_up16(int v) { return (v + 15) / 16 * 16; }

}  // namespace
}  // namespace devel

using namespace devel;

extern "C" int devel_batch_create(const devel_optics* o, int capacity, devel_batch** out) {
    if (!out) return set_error(DEVEL_EINVAL, "devel_batch_create: out is NULL");
    *out = nullptr;
    if (!o) return set_error(DEVEL_EINVAL, "devel_batch_create: optics is NULL");
    if (o->precision != DEVEL_PREC_BF16X3 || o->batch != 1)
        return set_error(DEVEL_EINVAL, "devel_batch_create: the handle must be a DEVEL_PREC_BF16X3 handle");
    if (capacity < 1 || capacity > 4096)
        return set_error(DEVEL_EINVAL, "devel_batch_create: capacity %d outside [1, 4096]", capacity);
    devel_batch* b = new devel_batch();
    b->base = o;
    b->capacity = capacity;
    b->view = *o;
    b->view.batch = capacity;
    b->view.ws = Workspace{};
    const size_t C = (size_t)capacity, n = (size_t)o->n, npix = n * n, ldn = (size_t)o->ldn;
    const size_t k = (size_t)o->k, k2 = (size_t)o->k2;
    const size_t ldf1 = (size_t)o->tcW.ldf, ldf2 = (size_t)o->tcW2.ldf;
    const size_t nslices = (size_t)tc::spectrum2_slices(o->n, o->ldn, o->tc_split_min);
    const size_t nparts = (size_t)o->npart_red;
    int rc = DEVEL_OK;
    auto alloc = [&](void** p, size_t bytes, bool zero) {
        if (rc) return;
        cudaError_t e = cudaMalloc(p, bytes);
        if (e == cudaSuccess) {
            b->owned.push_back(*p);
            if (zero) e = cudaMemset(*p, 0, bytes);
        }
        if (e != cudaSuccess) {
            cudaGetLastError();
            rc = set_error(e == cudaErrorMemoryAllocation ? DEVEL_ENOMEM : DEVEL_ECUDA,
                           "devel_batch_create: %zu bytes: %s", bytes, cudaGetErrorString(e));
        }
    };
    devel_optics& v = b->view;
    Workspace& w = v.ws;
    // the reduction's slices of the wider window (the other window's fit in them)
    alloc((void**)&w.Q, sizeof(float) * C * nslices * k2 * (size_t)round_up16((int)k2), false);
    alloc((void**)&w.mhat, sizeof(float2) * C * k * k, false);
    alloc((void**)&w.Ihat, sizeof(float2) * C * k2 * k2, false);
    alloc((void**)&w.rhat, sizeof(float2) * C * k2 * k2, false);
    alloc((void**)&w.Shat, sizeof(float2) * C * k * k, false);
    alloc((void**)&w.qpart, sizeof(long long) * C * 3 * nparts, false);
    alloc((void**)&w.lpart, sizeof(long long) * C * 2 * nparts, false);
    alloc((void**)&w.vbits, sizeof(unsigned) * C, true);
    alloc((void**)&w.vmax, sizeof(double) * C, false);
    alloc((void**)&w.counters, sizeof(unsigned) * 8, true);
    alloc((void**)&b->rcount, sizeof(unsigned) * C, true);
    alloc((void**)&w.bufI, sizeof(float) * C * npix, false);
    alloc((void**)&w.bufV, sizeof(float) * C * npix, false);
    alloc((void**)&w.phi2, sizeof(float) * C * npix, false);
    alloc((void**)&w.M, C * npix, false);
    alloc((void**)&w.d2, sizeof(int) * C * npix, false);
    // the reduction operand's pad columns [n, ldn) must read as zeros
    alloc((void**)&v.Xhi, sizeof(__nv_bfloat16) * C * n * ldn, true);
    alloc((void**)&v.Xlo, sizeof(__nv_bfloat16) * C * n * ldn, true);
    alloc((void**)&v.Acat_hi, sizeof(__nv_bfloat16) * C * n * ldf2, false);
    alloc((void**)&v.Acat_lo, sizeof(__nv_bfloat16) * C * n * ldf2, false);
    // Zm entries outside the window's kw x kw block are never written
    alloc((void**)&v.tcW.zm_hi, sizeof(__nv_bfloat16) * C * ldf1 * ldf1, true);
    alloc((void**)&v.tcW.zm_lo, sizeof(__nv_bfloat16) * C * ldf1 * ldf1, true);
    alloc((void**)&v.tcW2.zm_hi, sizeof(__nv_bfloat16) * C * ldf2 * ldf2, true);
    alloc((void**)&v.tcW2.zm_lo, sizeof(__nv_bfloat16) * C * ldf2 * ldf2, true);
    const int ci = capacity, ni = o->n;
    if (!rc) rc = tc::make_map3(&v.m_X_hi, v.Xhi, ci, ni, o->ldn, o->ldn, n * ldn, 128);
    if (!rc) rc = tc::make_map3(&v.m_X_lo, v.Xlo, ci, ni, o->ldn, o->ldn, n * ldn, 128);
    for (TcWindow* tw : {&v.tcW, &v.tcW2}) {
        const int ldf = tw->ldf;
        if (!rc) rc = tc::make_map3(&tw->m_zm_hi, tw->zm_hi, ci, ldf, ldf, ldf, (size_t)ldf * ldf, kTileT);
        if (!rc) rc = tc::make_map3(&tw->m_zm_lo, tw->zm_lo, ci, ldf, ldf, ldf, (size_t)ldf * ldf, kTileT);
        if (!rc) rc = tc::make_map3(&tw->m_zmw_hi, tw->zm_hi, ci, ldf, ldf, ldf, (size_t)ldf * ldf, ldf);
        if (!rc) rc = tc::make_map3(&tw->m_zmw_lo, tw->zm_lo, ci, ldf, ldf, ldf, (size_t)ldf * ldf, ldf);
        if (!rc) rc = tc::make_map3(&tw->m_acat_hi, v.Acat_hi, ci, ni, ldf, ldf, n * ldf, 128);
        if (!rc) rc = tc::make_map3(&tw->m_acat_lo, v.Acat_lo, ci, ni, ldf, ldf, n * ldf, 128);
    }
    if (!rc) {
        cudaError_t e = cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking);
        if (e != cudaSuccess) rc = cuda_error(e, "devel_batch_create: cudaStreamCreate");
    }
    if (rc) {
        free_batch(b);
        return rc;
    }
    *out = b;
    return DEVEL_OK;
}

extern "C" int devel_batch_destroy(devel_batch* b) {
    if (!b) return DEVEL_OK;
    cudaError_t e = cudaDeviceSynchronize();
    free_batch(b);
    if (e != cudaSuccess) return cuda_error(e, "devel_batch_destroy: cudaDeviceSynchronize");
    return DEVEL_OK;
}

namespace devel {
namespace {

struct BatchArgs {
    const unsigned char* target;
    float* phi;
    int phi_given;
    const float* m;
    unsigned char* mask_out;
    double* loss_hist;
    long long* l2_hist;
    long long* pvb_hist;
    int ldh;
    int* status;
};

// Every iteration of the batch on stream s, in the order of the single-clip loop: the
// reduction of the masks, Ihat, the forward expansion, resist / loss / dL/dI, the
// reduction of dL/dI, Shat, the adjoint expansion with each clip's max |V|, the level-set
// step, and the re-initialisation every reinit_every iterations (global index).
int enqueue_batch(const devel_ilt_params* p, devel_batch* b, int B, const BatchArgs& a, cudaStream_t s) {
    devel_optics v = b->view;
    v.batch = B;
    v.tc_split = b->base->tc_split;  // the handle's tuned tile shapes
    v.tc_expand_bn = b->base->tc_expand_bn;
    const Workspace& w = v.ws;
    const int n = v.n;
    const size_t npix = (size_t)n * n;
    DEVEL_CUDA_TRY(cudaMemsetAsync(a.status, 0, sizeof(int), s));
    float* phi = a.phi;
    float* phi_alt = w.phi2;
    int rc;
    if (!a.phi_given) {
        rc = launch_reinit(n, a.target, phi, w.d2, p->d_lo, p->d_hi, s, B, false);
        if (rc) return rc;
    }
    rc = launch_mask_from_phi(n, phi, w.M, s, B);
    if (!rc) rc = tc::launch_mask_bf16(w.M, n, v.ldn, v.Xhi, s, B);
    if (rc) return rc;
    for (int t = 0; t <= p->iters; ++t) {
        rc = launch_spectrum_mask_resident(&v, v.W, w.mhat, s);
        if (!rc) rc = forward_from_mhat(&v, w.bufI, s);
        if (!rc)
            rc = launch_resist(n, w.bufI, a.target, p->resist, nullptr, v.Xhi, v.Xlo, v.ldn, w.qpart, w.lpart,
                               v.npart_red, nullptr, nullptr, a.loss_hist ? a.loss_hist + t : nullptr,
                               a.l2_hist ? a.l2_hist + t : nullptr, a.pvb_hist ? a.pvb_hist + t : nullptr,
                               a.status, b->rcount, s, false, B, a.ldh);
        if (rc) return rc;
        if (t == p->iters) break;  // the final masks are imaged for their metrics only
        rc = launch_spectrum_resident(&v, v.W2, w.rhat, s);
        if (!rc) rc = adjoint_from_rhat(&v, w.bufV, w.vmax, a.status, s);
        // the next forward reads the bf16 mask; the u8 mask only feeds a re-initialisation
        // (which also overwrites phi) and the final mask output
        const int gi = p->start_iter + t;
        const bool reinit = p->reinit_every > 0 && (gi + 1) % p->reinit_every == 0;
        const bool keep_mask = reinit || (t + 1 == p->iters && a.mask_out);
        if (!rc)
            rc = launch_levelset_step(n, phi, w.bufV, w.vmax, a.m, p->dt, p->lambda, reinit ? nullptr : phi_alt,
                                      keep_mask ? w.M : nullptr, v.Xhi, v.ldn, s, p->upwind, B);
        if (rc) return rc;
        std::swap(phi, phi_alt);
        if (reinit) {
            rc = launch_reinit(n, w.M, phi, w.d2, p->d_lo, p->d_hi, s, B, false);
            if (rc) return rc;
        }
    }
    if (phi != a.phi)
        DEVEL_CUDA_TRY(cudaMemcpyAsync(a.phi, phi, sizeof(float) * npix * B, cudaMemcpyDeviceToDevice, s));
    if (a.mask_out) DEVEL_CUDA_TRY(cudaMemcpyAsync(a.mask_out, w.M, npix * B, cudaMemcpyDeviceToDevice, s));
    return DEVEL_OK;
}

std::vector<unsigned char> batch_key(const devel_ilt_params* p, const devel_batch* b, int B, const BatchArgs& a,
                                     int device) {
    // field by field (no padding bytes in the key)
    const int tag = prof_on() ? (int)(~prof_generation()) : device;
    const void* ptrs[8] = {a.target, a.phi, a.m, a.mask_out, a.loss_hist, a.l2_hist, a.pvb_hist, a.status};
    const int ints[6] = {B, a.phi_given, a.ldh, tag, b->base->tc_split, b->base->tc_expand_bn};
    std::vector<unsigned char> k(sizeof(devel_ilt_params) + sizeof(ptrs) + sizeof(ints));
    unsigned char* q = k.data();
    std::memcpy(q, p, sizeof(devel_ilt_params));
    q += sizeof(devel_ilt_params);
    std::memcpy(q, ptrs, sizeof(ptrs));
    q += sizeof(ptrs);
    std::memcpy(q, ints, sizeof(ints));
    return k;
}

}  // namespace
}  // namespace devel

#define CHECK_ARR(ptr, name, need)                                                                \
    do {                                                                                          \
        if ((need) && !(ptr)) return set_error(DEVEL_EINVAL, "devel_ilt_solve_batch: %s is NULL", name); \
        if ((ptr) && (reinterpret_cast<uintptr_t>(ptr) & 15u))                                    \
            return set_error(DEVEL_EINVAL, "devel_ilt_solve_batch: %s is not 16-byte aligned", name); \
    } while (0)

extern "C" int devel_ilt_solve_batch(const devel_ilt_params* p, devel_batch* b, int nclips,
                                     const unsigned char* target, float* phi, int phi_given, const float* m,
                                     unsigned char* mask_out, double* loss_hist, long long* l2_hist,
                                     long long* pvb_hist, int ldh, int* status, cudaStream_t s) {
    if (!p) return set_error(DEVEL_EINVAL, "devel_ilt_solve_batch: params is NULL");
    if (!b) return set_error(DEVEL_EINVAL, "devel_ilt_solve_batch: batch is NULL");
    if (nclips < 0 || nclips > b->capacity)
        return set_error(DEVEL_EINVAL, "devel_ilt_solve_batch: nclips %d outside [0, %d]", nclips, b->capacity);
    if (p->iters < 0 || p->reinit_every < 0 || p->start_iter < 0)
        return set_error(DEVEL_EINVAL, "devel_ilt_solve_batch: negative iters/reinit_every/start_iter");
    if (!(p->d_lo <= p->d_hi)) return set_error(DEVEL_EINVAL, "devel_ilt_solve_batch: d_lo > d_hi");
    if (p->upwind != DEVEL_UPWIND_GODUNOV1 && p->upwind != DEVEL_UPWIND_WENO5)
        return set_error(DEVEL_EINVAL, "devel_ilt_solve_batch: unknown upwind scheme %d", p->upwind);
    if (p->optimizer != DEVEL_OPT_STEEPEST)
        return set_error(DEVEL_EINVAL, "devel_ilt_solve_batch: only the steepest-descent optimizer is batched");
    CHECK_ARR(status, "status", true);
    CHECK_ARR(target, "target", nclips > 0);
    CHECK_ARR(phi, "phi", nclips > 0);
    CHECK_ARR(m, "m", false);
    CHECK_ARR(mask_out, "mask_out", false);
    CHECK_ARR(loss_hist, "loss_hist", false);
    CHECK_ARR(l2_hist, "l2_hist", false);
    CHECK_ARR(pvb_hist, "pvb_hist", false);
    if ((loss_hist || l2_hist || pvb_hist) && ldh < p->iters + 1)
        return set_error(DEVEL_EINVAL, "devel_ilt_solve_batch: ldh %d < iters + 1", ldh);
    if (nclips == 0) {
        DEVEL_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(int), s));
        return DEVEL_OK;
    }
    const BatchArgs a{target, phi, phi_given, m, mask_out, loss_hist, l2_hist, pvb_hist, ldh, status};
    if (!p->use_graph) return enqueue_batch(p, b, nclips, a, s);
    int dev = 0;
    DEVEL_CUDA_TRY(cudaGetDevice(&dev));
    std::vector<unsigned char> key = batch_key(p, b, nclips, a, dev);
    for (size_t i = 0; i < b->graphs.size(); ++i) {
        if (b->graphs[i].key == key) {
            devel_batch::Graph g = b->graphs[i];
            b->graphs.erase(b->graphs.begin() + i);
            b->graphs.push_back(g);
            DEVEL_CUDA_TRY(cudaGraphLaunch(g.exec, s));
            return DEVEL_OK;
        }
    }
    DEVEL_CUDA_TRY(cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_batch(p, b, nclips, a, b->capture);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->capture, &graph);
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return cuda_error(e, "devel_ilt_solve_batch: cudaStreamEndCapture");
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_error(e, "devel_ilt_solve_batch: cudaGraphInstantiate");
    if (b->graphs.size() >= kMaxBatchGraphs) {
        cudaGraphExecDestroy(b->graphs.front().exec);
        b->graphs.erase(b->graphs.begin());
    }
    b->graphs.push_back(devel_batch::Graph{key, exec});
    DEVEL_CUDA_TRY(cudaGraphLaunch(exec, s));
    return DEVEL_OK;
}
