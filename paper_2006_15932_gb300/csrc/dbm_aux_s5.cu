// dbm_aux_s5.cu -- the output and initialisation launches for 5 species.
#include "dbm_aux_impl.cuh"

namespace dbm {
template void aux_set_state<5>(dbm_handle *, void *, const double *, const double *, const double *, const double *,
                                cudaStream_t);
template void aux_moments<5>(dbm_handle *, const void *, double *, cudaStream_t);
template void aux_noneq<5>(dbm_handle *, const void *, double *, cudaStream_t);
template void aux_cons<5>(dbm_handle *, const void *, double *, double *, cudaStream_t);
}  // namespace dbm
