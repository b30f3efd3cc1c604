// Instantiations of the order-5 kernels (elastic and 3-mechanism anelastic).
#include "launch.h"

namespace ltsdev {
Launchers launchers_o5(int m) { return m == 0 ? Impl<5, 0>::make() : Impl<5, 3>::make(); }
}  // namespace ltsdev
