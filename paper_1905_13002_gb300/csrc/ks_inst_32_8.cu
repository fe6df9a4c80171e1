// Instantiation nx = 32, ny = 8: single sequences on the tensor-core scans
// (ks_timpl.cuh), segmented batches on the CUDA-core group kernels
// (ks_gimpl.cuh).
#include "ks_timpl.cuh"

namespace ks {
namespace {

// 3 chains of 72 steps per tile: T = 65536 is then one wave of 304 tiles
// (two per SM).
using TC = TImpl<32, 8, 3, 72>;
using GR = GImpl<32, 8, 3, 64>;

// One layout entry serves both: a single sequence (B = 1) gets the
// tensor-core layout, with its sizes raised to cover a one-segment batch.
Layout layout_32_8(int64_t T, int B) {
    if (B > 1) return GR::layout(T, B);
    Layout L = TC::layout(T);
    const Layout G = GR::layout(T, 1);
    if (G.bytes_smooth > L.bytes_smooth) L.bytes_smooth = G.bytes_smooth;
    if (L.bytes_elements < L.bytes_smooth) L.bytes_elements = L.bytes_smooth;
    return L;
}

}  // namespace

extern const VTable kImpl_32_8 = VTable{32,
                                        8,
                                        &layout_32_8,
                                        &GR::build_elements,
                                        &GR::filter_scan,
                                        &TC::smooth_scan,
                                        &TC::smooth,
                                        &GR::smooth_batch,
                                        &GR::no_comb,
                                        &GR::no_comb,
                                        &GR::no_agg_bytes,
                                        &GR::no_fagg,
                                        &GR::no_sagg,
                                        nullptr};
}  // namespace ks
