// Instantiation nx = 4, ny = 2 (2-D Wiener-velocity tracking model of Section V).
#include "ks_impl.cuh"

namespace ks {
extern const VTable kImpl_4_2 = Impl<4, 2>::vtable();
}
