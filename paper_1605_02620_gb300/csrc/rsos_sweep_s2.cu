// Phase kernels for 2x2 sub-tiles (4x4 DT tiles).
#include "rsos_sweep.cuh"
RSOS_DEFINE_SX(2)
