// Optional per-kernel timing with CUDA events (tracing; no counterpart in the paper).
//
// When a profile is open (devel_profile_start), every kernel launch of the
// library is bracketed by two events recorded on the launching stream; after
// devel_profile_stop the host reads per-kernel launch counts and summed
// device time. Off by default; when off the cost is one branch per launch.
// devel_profile_select limits the events to some kernel classes (fewer events
// disturb the timed kernels less).
#include <algorithm>
#include <cstring>
#include <vector>

#include "common.cuh"

namespace devel {

static const char* kNames[PROF_NKINDS] = {
    "spectrum_gemm", "spectrum_reduce", "unused",     "ihat_tcc",  "shat_tcc",
    "expand_T",      "expand_gemm",     "vmax_final", "resist",    "resist_final",
    "levelset_step", "mask_from_phi",   "edt_cols",   "edt_rows",  "u8_to_f32",
    "tc_expand",     "tc_spectrum",     "spectrum_stage2", "tc_split",  "cg_dots",
    "cg_update",     "dsn_conv",        "dsn_misc",   "phi_resample",
};

struct Slot {
    int kind;
    cudaEvent_t a, b;
    bool captured;  // recorded into a captured graph (re-timestamped by every replay)
};

static bool g_on = false;
static std::vector<Slot> g_pool;
static size_t g_used = 0;
static int g_open_kind = -1;
static int g_launches[PROF_NKINDS];
static double g_ms[PROF_NKINDS];
static bool g_overflow = false;
static unsigned g_generation = 0;  // bumped by every devel_profile_start
static unsigned long long g_select = ~0ull;  // kernel classes that get events

bool prof_on() { return g_on; }
unsigned prof_generation() { return g_generation; }

// Inside a stream capture an external record becomes an event-record node that
// timestamps the event on every replay (not a capture-internal dependency); outside a
// capture a plain record (the external flag is only valid while capturing).
static bool capturing(cudaStream_t s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    return cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive;
}
static void record(cudaEvent_t e, cudaStream_t s) {
    if (capturing(s))
        cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
    else
        cudaEventRecord(e, s);
}

void prof_begin(int kind, cudaStream_t s) {
    if (!g_on || !((g_select >> kind) & 1ull)) return;
    if (g_used >= g_pool.size()) {
        g_overflow = true;
        g_open_kind = -1;
        return;
    }
    g_pool[g_used].kind = kind;
    g_pool[g_used].captured = capturing(s);
    record(g_pool[g_used].a, s);
    g_open_kind = kind;
}

void prof_end(int kind, cudaStream_t s) {
    if (!g_on || g_open_kind != kind) return;
    record(g_pool[g_used].b, s);
    ++g_used;
    g_open_kind = -1;
}

}  // namespace devel

using namespace devel;

extern "C" {

int devel_profile_select(unsigned long long kind_mask) {
    if (g_on) return set_error(DEVEL_EINVAL, "devel_profile_select: a profile is open");
    g_select = kind_mask;
    return DEVEL_OK;
}

int devel_profile_start(int capacity) {
    if (capacity < 1 || capacity > (1 << 22))
        return set_error(DEVEL_EINVAL, "devel_profile_start: capacity %d outside [1, 4194304]", capacity);
    if (g_on) return set_error(DEVEL_EINVAL, "devel_profile_start: a profile is already open");
    if ((int)g_pool.size() < capacity) {
        for (size_t i = g_pool.size(); i < (size_t)capacity; ++i) {
            Slot sl{0, nullptr, nullptr, false};
            DEVEL_CUDA_TRY(cudaEventCreate(&sl.a));
            DEVEL_CUDA_TRY(cudaEventCreate(&sl.b));
            g_pool.push_back(sl);
        }
    }
    g_used = 0;
    g_overflow = false;
    std::memset(g_launches, 0, sizeof(g_launches));
    for (int i = 0; i < PROF_NKINDS; ++i) g_ms[i] = 0.0;
    ++g_generation;
    g_on = true;
    return DEVEL_OK;
}

int devel_profile_collect(void) {
    for (size_t i = 0; i < g_used; ++i) {
        DEVEL_CUDA_TRY(cudaEventSynchronize(g_pool[i].b));
        float ms = 0.f;
        DEVEL_CUDA_TRY(cudaEventElapsedTime(&ms, g_pool[i].a, g_pool[i].b));
        g_launches[g_pool[i].kind] += 1;
        g_ms[g_pool[i].kind] += ms;
    }
    // events of direct launches are counted once: their slots go back to the pool, while
    // the slots of captured graphs stay (every replay records into them again)
    std::stable_partition(g_pool.begin(), g_pool.begin() + (long)g_used, [](const Slot& sl) { return sl.captured; });
    size_t kept = 0;
    while (kept < g_used && g_pool[kept].captured) ++kept;
    g_used = kept;
    if (g_overflow) return set_error(DEVEL_EINVAL, "devel_profile_collect: capacity exceeded, profile truncated");
    return DEVEL_OK;
}

int devel_profile_stop(void) {
    if (!g_on) return set_error(DEVEL_EINVAL, "devel_profile_stop: no profile open");
    g_on = false;
    ++g_generation;
    return DEVEL_OK;
}

int devel_profile_kinds(void) { return PROF_NKINDS; }

int devel_profile_query(int kind, const char** name, int* launches, double* total_ms) {
    if (kind < 0 || kind >= PROF_NKINDS) return set_error(DEVEL_EINVAL, "devel_profile_query: bad kind %d", kind);
    if (name) *name = kNames[kind];
    if (launches) *launches = g_launches[kind];
    if (total_ms) *total_ms = g_ms[kind];
    return DEVEL_OK;
}

}  // extern "C"
