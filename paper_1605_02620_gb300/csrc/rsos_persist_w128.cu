// Persistent engine kernels for 128-lane words (four 32-lane words per
// thread) on 4x4 sub-tiles (8x8 DT tiles).
#include "rsos_persist_launch.cuh"

namespace rsos {

cudaError_t plan_persist_w128(const JobDev& J, int block_tiles, int phase_lag, PersistPlan* out)
{
    switch (J.N) {
        case 1: return plan_persist_t<1, Word128, 4>(J, block_tiles, phase_lag, out);
        case 2: return plan_persist_t<2, Word128, 4>(J, block_tiles, phase_lag, out);
        case 3: return plan_persist_t<3, Word128, 4>(J, block_tiles, phase_lag, out);
        case 4: return plan_persist_t<4, Word128, 4>(J, block_tiles, phase_lag, out);
        case 5: return plan_persist_t<5, Word128, 4>(J, block_tiles, phase_lag, out);
        case 6: return plan_persist_t<6, Word128, 4>(J, block_tiles, phase_lag, out);
        case 7: return plan_persist_t<7, Word128, 4>(J, block_tiles, phase_lag, out);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_persist_w128(const JobDev& J, const PersistArgs& A, const PersistPlan& P, cudaStream_t s)
{
    switch (J.N) {
        case 1: return launch_persist_t<1, Word128, 4>(A, P, s);
        case 2: return launch_persist_t<2, Word128, 4>(A, P, s);
        case 3: return launch_persist_t<3, Word128, 4>(A, P, s);
        case 4: return launch_persist_t<4, Word128, 4>(A, P, s);
        case 5: return launch_persist_t<5, Word128, 4>(A, P, s);
        case 6: return launch_persist_t<6, Word128, 4>(A, P, s);
        case 7: return launch_persist_t<7, Word128, 4>(A, P, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace rsos
