// 16-bit storage instantiations: FP32 arithmetic, f_0..8 and g_1..8 stored
// as FP16 (scaled) or BF16, g_0 in FP32.
#include "lbm_ops.cuh"

namespace lbm {
const Ops *ops_f16s() { return OpsImpl<float, Store16<__half>, 2, 128, 2>::ops("f16s"); }
const Ops *ops_bf16s() { return OpsImpl<float, Store16<__nv_bfloat16>, 2, 128, 2>::ops("bf16s"); }
}  // namespace lbm
