// Mixed-size batches (ks_smooth_batched) at 16 steps per thread.
#include "ks_mixed.cuh"

namespace ks {
extern const MixedVariant kMixed16 = mixed_variant<16>();
}
