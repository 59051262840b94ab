// dbm_aux_s3.cu -- the output and initialisation launches for 3 species.
#include "dbm_aux_impl.cuh"

namespace dbm {
template void aux_set_state<3>(dbm_handle *, void *, const double *, const double *, const double *, const double *,
                                cudaStream_t);
template void aux_moments<3>(dbm_handle *, const void *, double *, cudaStream_t);
template void aux_noneq<3>(dbm_handle *, const void *, double *, cudaStream_t);
template void aux_cons<3>(dbm_handle *, const void *, double *, double *, cudaStream_t);
}  // namespace dbm
