// fk_dc_orth.cu -- engine instantiations for orthant sums (counts, FP64 and
// compensated-FP32 weights).
#include "fk_dc_ops.cuh"

namespace fk {
namespace dc {
FK_DC_SWEEP_DEF(sweep_count, PolCount)
FK_DC_SWEEP_DEF(sweep_w64, PolW64)
FK_DC_SWEEP_DEF(sweep_wff, PolWFF)
}  // namespace dc
}  // namespace fk
