// Phase kernels for 4x4 sub-tiles (8x8 DT tiles).
#include "rsos_sweep.cuh"
RSOS_DEFINE_SX(4)
