// Mixed-size batches (ks_smooth_batched) at 4 steps per thread.
#include "ks_mixed.cuh"

namespace ks {
extern const MixedVariant kMixed4 = mixed_variant<4>();
}
