// Instantiation nx = 4, ny = 2 (2-D Wiener-velocity tracking model of Section V).
#include "ks_impl.cuh"

namespace ks {
extern const ChunkVariant kChunk_4_2_4, kChunk_4_2_8, kChunk_4_2_16;   // ks_chunk*.cu
static constexpr ChunkVariant kChunk_4_2_32 = Impl<4, 2>::chunk_variant();
template <>
const ChunkVariant* const ChunkTable<4, 2>::v[4] = {&kChunk_4_2_4, &kChunk_4_2_8, &kChunk_4_2_16,
                                                   &kChunk_4_2_32};
extern const VTable kImpl_4_2 = Tuned<4, 2>::vtable();
extern const VTable kImpl32_4_2 = Impl<4, 2>::vtable();   // fixed 32 steps per thread (ks_noalloc.cu)
}
