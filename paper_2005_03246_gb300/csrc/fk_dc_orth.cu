// fk_dc_orth.cu -- engine instantiations for weighted orthant sums (FP64 and
// compensated-FP32 weights; counts use the dominance engine of fk_dom.cu).
#include "fk_dc_ops.cuh"

namespace fk {
namespace dc {
FK_DC_SWEEP_DEF(sweep_w64, PolW64)
FK_DC_SWEEP_DEF(sweep_wff, PolWFF)
}  // namespace dc
}  // namespace fk
