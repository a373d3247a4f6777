// gsc_e3.cu -- GSC E-step instantiations for Hprime 7..8 (see gsc_estep.cuh).
#include "gsc_estep.cuh"

namespace prosper {

int gsc_launch_7_8(int Hp, GscArgs &A, bool enc, int grid, cudaStream_t s) {
    switch (Hp) {
        case 7: return gsc_launch<7>(A, enc, grid, s);
        case 8: return gsc_launch<8>(A, enc, grid, s);
        default: set_error("GSC: unsupported Hprime %d", Hp); return PROSPER_EINVAL;
    }
}

}  // namespace prosper
