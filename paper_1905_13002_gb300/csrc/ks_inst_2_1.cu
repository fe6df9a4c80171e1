// Instantiation nx = 2, ny = 1.
#include "ks_impl.cuh"

namespace ks {
extern const ChunkVariant kChunk_2_1_4, kChunk_2_1_8, kChunk_2_1_16;   // ks_chunk*.cu
static constexpr ChunkVariant kChunk_2_1_32 = Impl<2, 1>::chunk_variant();
template <>
const ChunkVariant* const ChunkTable<2, 1>::v[4] = {&kChunk_2_1_4, &kChunk_2_1_8, &kChunk_2_1_16,
                                                   &kChunk_2_1_32};
extern const VTable kImpl_2_1 = Tuned<2, 1>::vtable();
}
