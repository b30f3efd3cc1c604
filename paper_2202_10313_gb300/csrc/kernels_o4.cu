// Instantiations of the order-4 kernels (elastic and 3-mechanism anelastic).
#include "launch.h"

namespace ltsdev {
Launchers launchers_o4(int m) { return m == 0 ? Impl<4, 0>::make() : Impl<4, 3>::make(); }
}  // namespace ltsdev
