// Mixed-size batches (ks_smooth_batched) at 8 steps per thread.
#include "ks_mixed.cuh"

namespace ks {
extern const MixedVariant kMixed8 = mixed_variant<8>();
}
