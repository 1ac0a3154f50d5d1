// FP64 instantiation.  Built with --fmad=false so that every product and sum
// is rounded separately, as in the FP64 CPU statement of the scheme.
#include "lbm_ops.cuh"

namespace lbm {
const Ops *ops_f64() { return OpsImpl<double, PlainStore<double>, 2, 64, 1>::ops("f64"); }
}  // namespace lbm
