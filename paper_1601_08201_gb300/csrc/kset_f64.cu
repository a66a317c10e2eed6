// Launchers of the f64 precision mode (vectors: double, A's values: double).
#include "sgtv_kset.cuh"

namespace sgtv {
const KernelSet kset_f64 = Impl<double, double>::make();
}  // namespace sgtv
