// The 8-steps-per-thread variants of the fused smooth / smooth_batch for
// nx = 2, 4 and 6 (chosen per call by chunk_choice, ks_api.cu).
#include "ks_impl.cuh"

namespace ks {
extern const ChunkVariant kChunk_2_1_8 = Impl<2, 1, 8>::chunk_variant();
extern const ChunkVariant kChunk_4_2_8 = Impl<4, 2, 8>::chunk_variant();
extern const ChunkVariant kChunk_6_3_8 = Impl<6, 3, 8>::chunk_variant();
}
