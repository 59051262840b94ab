// dbm_step_acc_s1.cu -- the fused step with the FP32 arithmetic options
// (FP64 thermo, stochastic rounding) instantiated for 1 species.
#include "dbm_step_impl.cuh"

namespace dbm {
template int launch_step_tma_t<1, tma_tile_x(1), tma_tile_y(1), 1, true>(dbm_handle *, const CUtensorMap *, const void *, void *, cudaStream_t);
}  // namespace dbm
