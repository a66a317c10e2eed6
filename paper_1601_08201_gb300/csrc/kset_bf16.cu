// Launchers of the bf16 precision mode (vectors: float, A's values: __nv_bfloat16).
#include "sgtv_kset.cuh"

namespace sgtv {
const KernelSet kset_bf16 = Impl<float, __nv_bfloat16>::make();
}  // namespace sgtv
