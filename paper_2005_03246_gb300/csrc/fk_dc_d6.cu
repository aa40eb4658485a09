// fk_dc_d6.cu -- engine instantiations for d = 6 at the sample points: 4
// enclosing class bits, 32 sweep channels.  One-channel
// policies only (weighted orthant sums, the Laplacian KDE on both paths), in a
// translation unit of their own so that they compile beside the others.
#include "fk_dc_ops.cuh"

namespace fk {
namespace dc {

#define FK_DC_SWEEP_HD_DEF(POL)                                                                      \
    fk_status sweep_d6(int d_eff, int64_t n, const uint32_t* const* P, const uint32_t* seq_top,     \
                       const POL& pol, Arena& ar, cudaStream_t st, int levels, int opts) {          \
        switch (d_eff) {                                                                            \
            case 6: return dc_sweep<POL, 4>(d_eff, n, P, seq_top, pol, ar, st, levels, opts);       \
            default: return set_error(FK_ERR_UNSUPPORTED, "sample-point path supports d <= 6");     \
        }                                                                                           \
    }
FK_DC_SWEEP_HD_DEF(PolW64)
FK_DC_SWEEP_HD_DEF(PolWFF)
FK_DC_SWEEP_HD_DEF(PolKF<1>)
FK_DC_SWEEP_HD_DEF(PolKD<1>)
#undef FK_DC_SWEEP_HD_DEF

}  // namespace dc
}  // namespace fk
