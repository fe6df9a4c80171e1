// The 16-steps-per-thread variants of the fused smooth / smooth_batch for
// nx = 2, 4 and 6 (chosen per call by chunk_choice, ks_api.cu).
#include "ks_impl.cuh"

namespace ks {
extern const ChunkVariant kChunk_2_1_16 = Impl<2, 1, 16>::chunk_variant();
extern const ChunkVariant kChunk_4_2_16 = Impl<4, 2, 16>::chunk_variant();
extern const ChunkVariant kChunk_6_3_16 = Impl<6, 3, 16>::chunk_variant();
}
