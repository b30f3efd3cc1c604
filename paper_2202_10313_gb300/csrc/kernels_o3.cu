// Instantiations of the order-3 kernels (elastic and 3-mechanism anelastic).
#include "launch.h"

namespace ltsdev {
Launchers launchers_o3(int m, bool fused) {
  if (fused) return m == 0 ? Impl<3, 0, FUSED_GROUP>::make() : Impl<3, 3, FUSED_GROUP>::make();
  return m == 0 ? Impl<3, 0, 1>::make() : Impl<3, 3, 1>::make();
}
}  // namespace ltsdev
