// Instantiations of the order-4 kernels (elastic and 3-mechanism anelastic).
#include "launch.h"

namespace ltsdev {
Launchers launchers_o4(int m, bool fused) {
  if (fused) return m == 0 ? Impl<4, 0, FUSED_GROUP>::make() : Impl<4, 3, FUSED_GROUP>::make();
  return m == 0 ? Impl<4, 0, 1>::make() : Impl<4, 3, 1>::make();
}
}  // namespace ltsdev
