// placeholder until the tensor-core pass lands
#include "ctx.h"
cudaError_t launch_sym_pass_tc(cudaStream_t, int, const float *, int64_t, int64_t, const float *,
                               int64_t, int, const double *, float *, int64_t, int, uint16_t *,
                               uint16_t *, int64_t, int *)
{
    return cudaErrorNotSupported;
}
cudaError_t launch_syrk_tc(cudaStream_t, int, const float *, int64_t, int64_t, int, const int *,
                           float *, int64_t, int, uint16_t *, uint16_t *, int64_t, int *)
{
    return cudaErrorNotSupported;
}
