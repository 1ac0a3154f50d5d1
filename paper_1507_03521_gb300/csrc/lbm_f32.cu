// FP32 instantiation: populations and arithmetic in FP32.
#include "lbm_ops.cuh"

namespace lbm {
const Ops *ops_f32() { return OpsImpl<float, PlainStore<float>, 2, 128, 1>::ops("f32"); }
}  // namespace lbm
