// fk_dc_kf64.cu -- engine instantiations for Laplacian kernel sums on the
// all-FP64 path.
#include "fk_dc_ops.cuh"

namespace fk {
namespace dc {
FK_DC_SWEEP_DEF(sweep_kd1, PolKD<1>)
FK_DC_SWEEP_DEF(sweep_kd2, PolKD<2>)
}  // namespace dc
}  // namespace fk
