// Mixed-size batches (ks_smooth_batched) at 32 steps per thread.
#include "ks_mixed.cuh"

namespace ks {
extern const MixedVariant kMixed32 = mixed_variant<32>();
}
