// ks_api.cu -- extern "C" entry points of include/ks.h: dispatch to the
// compiled (nx, ny) instantiations, workspace queries and status handling.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/ks.h"
#include "ks_impl.cuh"
#include "ks_mixed.cuh"

namespace ks {

extern const VTable kImpl_2_1;
extern const VTable kImpl_4_2;
extern const VTable kImpl_6_3;
extern const VTable kImpl_8_4;
extern const VTable kImpl_32_8;

static const VTable* const kImpls[] = {&kImpl_2_1, &kImpl_4_2, &kImpl_6_3, &kImpl_8_4, &kImpl_32_8};

const VTable* find_impl(int nx, int ny) {
    for (const VTable* v : kImpls)
        if (v->nx == nx && v->ny == ny) return v;
    return nullptr;
}

static const VTable* find_nx(int nx) {
    for (const VTable* v : kImpls)
        if (v->nx == nx) return v;
    return nullptr;
}

// ---- steps-per-thread rules (ks_set_chunk_rules); slot 0: mixed-size
// batches, 1..3: nx = 2, 4, 6.  Host state of the process, guarded by a mutex.
namespace {
constexpr int kMaxRules = 16;
struct RuleSet {
    int count = 0;   // 0: built-in table
    int64_t below[kMaxRules];
    int choice[kMaxRules];   // chunk index | fold << 2
};
std::mutex g_rules_mutex;
RuleSet g_rules[4];

int rule_slot(int nx) { return nx == 0 ? 0 : nx == 2 ? 1 : nx == 4 ? 2 : nx == 6 ? 3 : -1; }
int steps_index(int steps) { return steps == 4 ? 0 : steps == 8 ? 1 : steps == 16 ? 2 : steps == 32 ? 3 : -1; }
}  // namespace

int chunk_choice(int nx, int64_t T) {
    const int sl = rule_slot(nx);
    if (sl >= 0) {
        std::lock_guard<std::mutex> lock(g_rules_mutex);
        const RuleSet& r = g_rules[sl];
        for (int i = 0; i < r.count; ++i)
            if (T < r.below[i]) return r.choice[i];
        if (r.count > 0) return r.choice[r.count - 1];
    }
    return builtin_chunk_index(T) | (builtin_fold(nx, T) ? 4 : 0);
}

extern const MixedVariant kMixed4, kMixed8, kMixed16, kMixed32;
static const MixedVariant* const kMixed[4] = {&kMixed4, &kMixed8, &kMixed16, &kMixed32};

// Slots (nx = 6, 4, 2) of a mixed batch's groups; KS_OK or an error code.
static int mixed_slots(int G, const ks_batch_group* gs, bool check_data, int (&slot)[3], int64_t* total) {
    slot[0] = slot[1] = slot[2] = -1;
    if (G < 1 || G > 3 || !gs) return KS_EINVAL;
    int64_t sum = 0;
    for (int i = 0; i < G; ++i) {
        const ks_batch_group& g = gs[i];
        const ks_model_batch& mb = g.models;
        const int s = (mb.nx == 6 && mb.ny == 3) ? 0 : (mb.nx == 4 && mb.ny == 2) ? 1
                    : (mb.nx == 2 && mb.ny == 1) ? 2 : -1;
        if (mb.nx < 1 || mb.ny < 1) return KS_EINVAL;
        if (s < 0) return KS_EUNSUPPORTED;
        if (slot[s] >= 0) return KS_EINVAL;   // two groups of one size
        if (mb.B < 1 || g.total_T < mb.B || g.total_T > 0x7fffffffLL) return KS_EINVAL;
        if (check_data) {
            if (!mb.F || !mb.Q || !mb.H || !mb.R || !mb.m0 || !mb.P0 || !mb.offsets) return KS_EINVAL;
            const void* p[5] = {g.y, g.fmean, g.fcov, g.smean, g.scov};
            for (const void* q : p)
                if (!q || (reinterpret_cast<uintptr_t>(q) & 15u) != 0) return KS_EINVAL;
        }
        slot[s] = i;
        sum += g.total_T;
    }
    if (sum > 0x7fffffffLL) return KS_EINVAL;
    *total = sum;
    return KS_OK;
}

static int check_nx_ny(const ks_model* m, const VTable** out) {
    if (!m) return KS_EINVAL;
    if (m->nx < 1 || m->ny < 1) return KS_EINVAL;
    const VTable* v = find_impl(m->nx, m->ny);
    if (!v) return KS_EUNSUPPORTED;
    *out = v;
    return KS_OK;
}

// Look-back settings in the workspace header (ks_workspace_set_waits).
__global__ void set_header_kernel(uint32_t* hdr, uint32_t wait_polls, uint32_t first_tile) {
    hdr[HDR_WAIT] = wait_polls;
    hdr[HDR_FIRST_TILE] = first_tile;
}

}  // namespace ks

using namespace ks;

extern "C" {

int ks_version(void) { return 100; }

int ks_supported(int nx, int ny) { return find_impl(nx, ny) != nullptr ? 1 : 0; }

const char* ks_strerror(int code) {
    switch (code) {
        case KS_OK: return "ok";
        case KS_EINVAL: return "invalid argument (size, null or misaligned pointer, workspace too small)";
        case KS_ECUDA: return "CUDA launch or copy failed";
        case KS_ENUMERIC: return "non-finite value or failed factorisation on the device";
        case KS_ETIMEOUT: return "look-back wait on the device ran out";
        case KS_EUNSUPPORTED: return "size not compiled into this library, or a model form this entry point does not take";
        default: return "unknown status code";
    }
}

size_t ks_workspace_bytes(const ks_model* m, int64_t T, int purpose) {
    const VTable* v = nullptr;
    if (check_nx_ny(m, &v) || T < 1 || T > 0x7fffffffLL) return 0;
    const Layout L = v->layout(T, 1);
    if (m->time_varying) {   // time-varying smoothing keeps per-step elements or constants
        if (m->time_varying != 1 || !v->tv_bytes) return 0;
        return (purpose == KS_WS_SMOOTH || purpose == KS_WS_ELEMENTS) ? v->tv_bytes(T) : 0;
    }
    if (purpose == KS_WS_SMOOTH) return L.bytes_smooth;
    if (purpose == KS_WS_ELEMENTS) return L.bytes_elements;
    return 0;
}

int ks_workspace_init(void* ws, size_t ws_bytes, void* stream) {
    if (!ws || ws_bytes < 256 || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0) return KS_EINVAL;
    return cudaMemsetAsync(ws, 0, 256, static_cast<cudaStream_t>(stream)) == cudaSuccess ? KS_OK : KS_ECUDA;
}

int ks_elements_layout_get(const ks_model* m, int64_t T, ks_elements_layout* out) {
    const VTable* v = nullptr;
    int rc = check_nx_ny(m, &v);
    if (rc) return rc;
    if (!out || T < 1 || T > 0x7fffffffLL) return KS_EINVAL;
    const Layout L = v->layout(T, 1);
    const int64_t n = m->nx, f = 4 * L.ld;
    out->ld = L.ld;
    out->offset_A = (int64_t)L.off_elems;
    out->offset_b = out->offset_A + n * n * f;
    out->offset_C = out->offset_b + n * f;
    out->offset_eta = out->offset_C + n * n * f;
    out->offset_J = out->offset_eta + n * f;
    return KS_OK;
}

int ks_build_elements(const ks_model* m, const float* y, int64_t T, void* ws, size_t ws_bytes, void* stream) {
    const VTable* v = nullptr;
    int rc = check_nx_ny(m, &v);
    if (rc) return rc;
    return v->build_elements(m, y, T, ws, ws_bytes, static_cast<cudaStream_t>(stream));
}

int ks_filter_scan(const ks_model* m, int64_t T, void* ws, size_t ws_bytes, float* fmean, float* fcov,
                   void* stream) {
    const VTable* v = nullptr;
    int rc = check_nx_ny(m, &v);
    if (rc) return rc;
    return v->filter_scan(m, T, ws, ws_bytes, fmean, fcov, static_cast<cudaStream_t>(stream));
}

int ks_smooth_scan(const ks_model* m, int64_t T, const float* fmean, const float* fcov, void* ws,
                   size_t ws_bytes, float* smean, float* scov, void* stream) {
    const VTable* v = nullptr;
    int rc = check_nx_ny(m, &v);
    if (rc) return rc;
    return v->smooth_scan(m, T, fmean, fcov, ws, ws_bytes, smean, scov, static_cast<cudaStream_t>(stream));
}

int ks_smooth(const ks_model* m, const float* y, int64_t T, void* ws, size_t ws_bytes, float* fmean,
              float* fcov, float* smean, float* scov, void* stream) {
    const VTable* v = nullptr;
    int rc = check_nx_ny(m, &v);
    if (rc) return rc;
    return v->smooth(m, y, T, ws, ws_bytes, fmean, fcov, smean, scov, static_cast<cudaStream_t>(stream),
                     nullptr);
}

int ks_smooth_traced(const ks_model* m, const float* y, int64_t T, void* ws, size_t ws_bytes, float* fmean,
                     float* fcov, float* smean, float* scov, void* stream, void* const* events) {
    const VTable* v = nullptr;
    int rc = check_nx_ny(m, &v);
    if (rc) return rc;
    return v->smooth(m, y, T, ws, ws_bytes, fmean, fcov, smean, scov, static_cast<cudaStream_t>(stream),
                     events);
}

size_t ks_workspace_bytes_aggregate(const ks_model* m, int64_t T) {
    const VTable* v = nullptr;
    if (check_nx_ny(m, &v) || T < 1 || T > 0x7fffffffLL) return 0;
    return v->agg_bytes(T);
}

int ks_filter_aggregate(const ks_model* m, const float* y, int64_t T, int first, void* ws, size_t ws_bytes,
                        float* out, void* stream) {
    const VTable* v = nullptr;
    int rc = check_nx_ny(m, &v);
    if (rc) return rc;
    return v->faggregate(m, y, T, first, ws, ws_bytes, out, static_cast<cudaStream_t>(stream));
}

int ks_smoother_aggregate(const ks_model* m, int64_t T, const float* fmean, const float* fcov, int last, void* ws,
                          size_t ws_bytes, float* out, void* stream) {
    const VTable* v = nullptr;
    int rc = check_nx_ny(m, &v);
    if (rc) return rc;
    return v->saggregate(m, T, fmean, fcov, last, ws, ws_bytes, out, static_cast<cudaStream_t>(stream));
}

size_t ks_workspace_bytes_batch(int nx, int ny, int B, int64_t total_T) {
    const VTable* v = find_impl(nx, ny);
    if (!v || B < 1 || total_T < B || total_T > 0x7fffffffLL) return 0;
    return v->layout(total_T, B).bytes_smooth;
}

int ks_smooth_batch(const ks_model_batch* mb, const float* y, int64_t total_T, void* ws, size_t ws_bytes,
                    float* fmean, float* fcov, float* smean, float* scov, void* stream) {
    if (!mb || mb->nx < 1 || mb->ny < 1) return KS_EINVAL;
    const VTable* v = find_impl(mb->nx, mb->ny);
    if (!v) return KS_EUNSUPPORTED;
    return v->smooth_batch(mb, y, total_T, ws, ws_bytes, fmean, fcov, smean, scov,
                           static_cast<cudaStream_t>(stream));
}

size_t ks_workspace_bytes_batched(int G, const ks_batch_group* groups) {
    int slot[3];
    int64_t total = 0;
    if (mixed_slots(G, groups, false, slot, &total) != KS_OK) return 0;
    size_t need = 0, base[3];
    for (const MixedVariant* v : kMixed) need = std::max(need, v->regions(groups, slot, base));
    return need;
}

int ks_smooth_batched(int G, const ks_batch_group* groups, void* ws, size_t ws_bytes, void* stream) {
    int slot[3];
    int64_t total = 0;
    int rc = mixed_slots(G, groups, true, slot, &total);
    if (rc) return rc;
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0) return KS_EINVAL;
    const int c = chunk_choice(0, total);
    return kMixed[c & 3]->run(groups, slot, ws, ws_bytes, static_cast<cudaStream_t>(stream), (c & 4) != 0);
}

int ks_set_chunk_rules(int nx, int count, const ks_chunk_rule* rules) {
    const int sl = rule_slot(nx);
    if (sl < 0 || count < 0 || count > kMaxRules || (count > 0 && !rules)) return KS_EINVAL;
    RuleSet r;
    r.count = count;
    for (int i = 0; i < count; ++i) {
        const int ix = steps_index(rules[i].steps);
        if (ix < 0 || rules[i].T_below < 1 || (i > 0 && rules[i].T_below <= rules[i - 1].T_below)) return KS_EINVAL;
        if (rules[i].fold != 0 && rules[i].fold != 1) return KS_EINVAL;
        r.below[i] = rules[i].T_below;
        r.choice[i] = ix | (rules[i].fold << 2);
    }
    std::lock_guard<std::mutex> lock(g_rules_mutex);
    g_rules[sl] = r;
    return KS_OK;
}

int ks_chunk_steps(int nx, int64_t T) {
    if (rule_slot(nx) < 0 || T < 1) return 0;
    static const int kSteps[4] = {4, 8, 16, 32};
    return kSteps[chunk_index_for(nx, T)];
}

int ks_chunk_fold(int nx, int64_t T) {
    if (rule_slot(nx) < 0 || T < 1) return 0;
    return (chunk_choice(nx, T) & 4) ? 1 : 0;
}

int ks_status(void* ws, void* stream) {
    if (!ws) return KS_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint32_t h = 0;
    if (cudaMemcpyAsync(&h, ws, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess) return KS_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return KS_ECUDA;
    if (cudaMemsetAsync(ws, 0, sizeof(h), s) != cudaSuccess) return KS_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return KS_ECUDA;
    if (h & ST_BADARG) return KS_EINVAL;
    if (h & ST_TIMEOUT) return KS_ETIMEOUT;
    if (h & ST_NUMERIC) return KS_ENUMERIC;
    return KS_OK;
}

int ks_workspace_set_waits(void* ws, size_t ws_bytes, uint32_t wait_polls, uint32_t first_tile, void* stream) {
    if (!ws || ws_bytes < 256 || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0 || first_tile > 1u)
        return KS_EINVAL;
    set_header_kernel<<<1, 1, 0, static_cast<cudaStream_t>(stream)>>>(static_cast<uint32_t*>(ws), wait_polls,
                                                                       first_tile);
    return launch_status();
}

int ks_refinements(void* ws, void* stream, uint32_t* count) {
    if (!ws || !count) return KS_EINVAL;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint32_t* ctr = static_cast<uint32_t*>(ws) + 1;
    uint32_t h = 0;
    if (cudaMemcpyAsync(&h, ctr, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess) return KS_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return KS_ECUDA;
    if (cudaMemsetAsync(ctr, 0, sizeof(h), s) != cudaSuccess) return KS_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return KS_ECUDA;
    *count = h;
    return KS_OK;
}

static int combine_args(int nx, int64_t count, const float* l, const float* r, float* o, void* ws,
                        size_t ws_bytes) {
    if (nx < 1 || count < 0 || !ws || ws_bytes < 256 || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0)
        return KS_EINVAL;
    if (count > 0 && (!l || !r || !o)) return KS_EINVAL;
    return KS_OK;
}

int ks_filter_combine_batch(int nx, int64_t count, const float* left, const float* right, float* out,
                            void* ws, size_t ws_bytes, void* stream) {
    int rc = combine_args(nx, count, left, right, out, ws, ws_bytes);
    if (rc) return rc;
    const VTable* v = find_nx(nx);
    if (!v) return KS_EUNSUPPORTED;
    return v->fcomb_batch(count, left, right, out, ws, static_cast<cudaStream_t>(stream));
}

int ks_smoother_combine_batch(int nx, int64_t count, const float* left, const float* right, float* out,
                              void* ws, size_t ws_bytes, void* stream) {
    int rc = combine_args(nx, count, left, right, out, ws, ws_bytes);
    if (rc) return rc;
    const VTable* v = find_nx(nx);
    if (!v) return KS_EUNSUPPORTED;
    return v->scomb_batch(count, left, right, out, ws, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
