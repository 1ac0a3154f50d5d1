// 16-bit deviation storage instantiations (Store16D): FP32 arithmetic,
// f_0..8 and g_1..8 stored as deviations from the rest equilibrium of the
// cell they sit on, in scaled FP16 or BF16, g_0 in FP32.  Single domains
// only, on 120-column strips of 128 threads.
#include "lbm_ops.cuh"

namespace lbm {
const Ops *ops_f16d() { return OpsImpl<float, Store16D<__half>, 2, 120, 2>::ops("f16d"); }
const Ops *ops_bf16d() { return OpsImpl<float, Store16D<__nv_bfloat16>, 2, 120, 2>::ops("bf16d"); }
}  // namespace lbm
