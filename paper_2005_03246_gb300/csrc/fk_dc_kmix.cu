// fk_dc_kmix.cu -- engine instantiations for Laplacian kernel sums on the
// mixed-precision path (KDE: one weight channel; Nadaraya-Watson: two).
#include "fk_dc_ops.cuh"

namespace fk {
namespace dc {
FK_DC_SWEEP_DEF(sweep_kf1, PolKF<1>)
FK_DC_SWEEP_DEF(sweep_kf2, PolKF<2>)
}  // namespace dc
}  // namespace fk
