// Instantiations of the order-3 kernels (elastic and 3-mechanism anelastic).
#include "launch.h"

namespace ltsdev {
Launchers launchers_o3(int m) { return m == 0 ? Impl<3, 0>::make() : Impl<3, 3>::make(); }
}  // namespace ltsdev
