// ks_noalloc.cu -- ks_smooth_noalloc: the end-to-end filter + smoother with
// its scratch in a file-scope device array instead of a caller workspace, for
// callers that cannot allocate device memory.
//
// The array below is a host-side stand-in in host code: its device address is
// fetched with cudaGetSymbolAddress, with the calling device current, at the
// start of every call (a host-side query; the first call on a device also
// loads the module there).  Asking on every call instead of caching keeps the
// address valid after a cudaDeviceReset, which gives the array a new address.
// Every call on a device shares the array; calls that overlap on the GPU race
// on it.  The status word is cleared at the start of each call and the scan
// state is cleared by the model-preparation kernel, so a call never depends
// on what an earlier call left behind.
#include <cuda_runtime.h>

#include "../../include/ks.h"
#include "ks_impl.cuh"

namespace ks {
extern const VTable kImpl32_4_2;

namespace {

static __device__ __align__(256) unsigned char g_noalloc_scratch[KS_NOALLOC_SCRATCH_BYTES];

// Device address of the scratch array on the current device.
int scratch_on_current_device(void** out) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return KS_ECUDA;
    *out = p;
    return KS_OK;
}

}  // namespace
}  // namespace ks

extern "C" int ks_smooth_noalloc(const ks_model* m, const float* y, int64_t T, float* fmean, float* fcov,
                                 float* smean, float* scov, int32_t* status_out, void* stream) {
    using namespace ks;
    if (!m) return KS_EINVAL;
    if (m->nx != 4 || m->ny != 2 || m->time_varying != 0) return KS_EUNSUPPORTED;
    if (T < 1 || T > KS_NOALLOC_MAX_T) return KS_EINVAL;
    if (!fmean || !fcov) return KS_EINVAL;
    if ((smean == nullptr) != (scov == nullptr)) return KS_EINVAL;   // both NULL: filtering only
    const VTable* v = &kImpl32_4_2;   // 32 steps per thread: the smallest scratch layout
    if (v->layout(T, 1).bytes_smooth > (size_t)KS_NOALLOC_SCRATCH_BYTES) return KS_EINVAL;
    void* ws = nullptr;
    int rc = scratch_on_current_device(&ws);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(ws, 0, 256, st) != cudaSuccess) return KS_ECUDA;   // status word
    rc = v->smooth(m, y, T, ws, (size_t)KS_NOALLOC_SCRATCH_BYTES, fmean, fcov, smean, scov, st, nullptr);
    if (rc) return rc;
    if (status_out &&
        cudaMemcpyAsync(status_out, ws, sizeof(int32_t), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return KS_ECUDA;
    return KS_OK;
}
