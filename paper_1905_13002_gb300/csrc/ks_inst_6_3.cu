// Instantiation nx = 6, ny = 3.
#include "ks_impl.cuh"

namespace ks {
extern const ChunkVariant kChunk_6_3_4, kChunk_6_3_8, kChunk_6_3_16;   // ks_chunk*.cu
static constexpr ChunkVariant kChunk_6_3_32 = Impl<6, 3>::chunk_variant();
template <>
const ChunkVariant* const ChunkTable<6, 3>::v[4] = {&kChunk_6_3_4, &kChunk_6_3_8, &kChunk_6_3_16,
                                                   &kChunk_6_3_32};
extern const VTable kImpl_6_3 = Tuned<6, 3>::vtable();
}
