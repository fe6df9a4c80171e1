// Instantiation nx = 32, ny = 8 (one warp per chain).
#include "ks_gimpl.cuh"

namespace ks {
extern const VTable kImpl_32_8 = GImpl<32, 8, 3, 64>::vtable();
}
