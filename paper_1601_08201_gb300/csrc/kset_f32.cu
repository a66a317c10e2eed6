// Launchers of the f32 precision mode (vectors: float, A's values: float).
#include "sgtv_kset.cuh"

namespace sgtv {
const KernelSet kset_f32 = Impl<float, float>::make();
}  // namespace sgtv
