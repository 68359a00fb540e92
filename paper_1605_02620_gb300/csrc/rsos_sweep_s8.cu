// Phase kernels for 8x8 sub-tiles (16x16 DT tiles).
#include "rsos_sweep.cuh"
RSOS_DEFINE_SX(8)
