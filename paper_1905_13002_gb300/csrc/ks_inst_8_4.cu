// Instantiation nx = 8, ny = 4: one 8-lane group per chain, four chains (one
// warp) per tile of 4 x 32 steps.
#include "ks_gimpl.cuh"

namespace ks {
extern const VTable kImpl_8_4 = GImpl<8, 4, 1, 32>::vtable();
}
