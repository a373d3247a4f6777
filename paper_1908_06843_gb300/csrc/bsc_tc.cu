// bsc_tc.cu -- BF16 tcgen05 projection for BSC preselection.
#include "internal.cuh"
namespace prosper {
int launch_bsc_proj_bf16(prosper_ctx *, const float *, const float *, int64_t, cudaStream_t) { set_error("BF16 path not built yet"); return PROSPER_EINVAL; }
}
