// gsc_e2.cu -- GSC E-step instantiations for Hprime 4..6 (see gsc_estep.cuh).
#include "gsc_estep.cuh"

namespace prosper {

int gsc_launch_4_6(int Hp, GscArgs &A, bool enc, int grid, cudaStream_t s) {
    switch (Hp) {
        case 4: return gsc_launch<4>(A, enc, grid, s);
        case 5: return gsc_launch<5>(A, enc, grid, s);
        case 6: return gsc_launch<6>(A, enc, grid, s);
        default: set_error("GSC: unsupported Hprime %d", Hp); return PROSPER_EINVAL;
    }
}

}  // namespace prosper
