// Instantiation nx = 2, ny = 1.
#include "ks_impl.cuh"

namespace ks {
extern const VTable kImpl_2_1 = Impl<2, 1>::vtable();
}
