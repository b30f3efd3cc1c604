// Instantiations of the order-5 kernels (elastic and 3-mechanism anelastic).
#include "launch.h"

namespace ltsdev {
Launchers launchers_o5(int m, bool fused) {
  if (fused) return m == 0 ? Impl<5, 0, FUSED_GROUP>::make() : Impl<5, 3, FUSED_GROUP>::make();
  return m == 0 ? Impl<5, 0, 1>::make() : Impl<5, 3, 1>::make();
}
}  // namespace ltsdev
