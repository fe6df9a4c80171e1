// Instantiation nx = 6, ny = 3.
#include "ks_impl.cuh"

namespace ks {
extern const VTable kImpl_6_3 = Impl<6, 3>::vtable();
}
