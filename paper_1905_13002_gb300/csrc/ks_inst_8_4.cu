// Instantiation nx = 8, ny = 4 (one warp per chain).
#include "ks_gimpl.cuh"

namespace ks {
extern const VTable kImpl_8_4 = GImpl<8, 4, 4, 32>::vtable();
}
