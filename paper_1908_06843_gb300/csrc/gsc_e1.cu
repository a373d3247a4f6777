// gsc_e1.cu -- GSC E-step instantiations for Hprime 1..3 (see gsc_estep.cuh).
#include "gsc_estep.cuh"

namespace prosper {

int gsc_launch_1_3(int Hp, GscArgs &A, bool enc, int grid, cudaStream_t s) {
    switch (Hp) {
        case 1: return gsc_launch<1>(A, enc, grid, s);
        case 2: return gsc_launch<2>(A, enc, grid, s);
        case 3: return gsc_launch<3>(A, enc, grid, s);
        default: set_error("GSC: unsupported Hprime %d", Hp); return PROSPER_EINVAL;
    }
}

}  // namespace prosper
