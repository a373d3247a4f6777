// serve.cu -- continuous-batching encode service.
#include "internal.cuh"
extern "C" {
int prosper_serve_start(prosper_ctx *, const prosper_params *, int, int) { return PROSPER_EINVAL; }
int prosper_serve_submit(prosper_ctx *, const float *, int, uint64_t *) { return PROSPER_EINVAL; }
int prosper_serve_wait(prosper_ctx *, uint64_t, int, int16_t *, float *, int16_t *, float *, float *, int64_t *, int64_t *) { return PROSPER_EINVAL; }
int prosper_serve_stop(prosper_ctx *) { return PROSPER_OK; }
}
