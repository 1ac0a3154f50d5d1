// FP32 instantiation: populations and arithmetic in FP32.  Single domains
// and slabs run 120-column strips on 128 threads (every step of a row in
// one pass); batches run 128-column strips.
#include "lbm_ops.cuh"

namespace lbm {
const Ops *ops_f32() {
    using Batch = OpsImpl<float, PlainStore<float>, 2, 128, 1>;
    using Narrow = OpsImpl<float, PlainStore<float>, 2, 64, 1>;
    return OpsImpl<float, PlainStore<float>, 2, 120, 1>::ops_batch_from<Batch, Narrow>("f32");
}
}  // namespace lbm
