// gsc_e4.cu -- GSC E-step instantiations for Hprime 9..10 (see gsc_estep.cuh).
#include "gsc_estep.cuh"

namespace prosper {

int gsc_launch_9_10(int Hp, GscArgs &A, bool enc, int grid, cudaStream_t s) {
    switch (Hp) {
        case 9: return gsc_launch<9>(A, enc, grid, s);
        case 10: return gsc_launch<10>(A, enc, grid, s);
        default: set_error("GSC: unsupported Hprime %d", Hp); return PROSPER_EINVAL;
    }
}

}  // namespace prosper
