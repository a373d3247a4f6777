// gsc.cu -- Gaussian sparse coding (Table 1, spike-and-slab) E-step.
#include "internal.cuh"
namespace prosper {
int launch_gsc_prep(prosper_ctx *, const prosper_params *, cudaStream_t) { set_error("GSC not built yet"); return PROSPER_EINVAL; }
int launch_gsc_estep(prosper_ctx *, const prosper_params *, const float *, int64_t, prosper_stats *,
                     int16_t *, float *, int16_t *, float *, float *, cudaStream_t) { set_error("GSC not built yet"); return PROSPER_EINVAL; }
}
