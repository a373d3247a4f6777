// mca.cu -- maximal causes analysis (Table 1, max superposition) E-step.
#include "internal.cuh"
namespace prosper {
int launch_mca_prep(prosper_ctx *, const float *, cudaStream_t) { set_error("MCA not built yet"); return PROSPER_EINVAL; }
int launch_mca_estep(prosper_ctx *, const float *, const double *, const float *, int64_t, prosper_stats *,
                     int16_t *, float *, int16_t *, float *, float *, cudaStream_t) { set_error("MCA not built yet"); return PROSPER_EINVAL; }
}
