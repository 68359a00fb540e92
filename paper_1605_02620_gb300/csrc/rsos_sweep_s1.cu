// Phase kernels for 1x1 sub-tiles (2x2 DT tiles).
#include "rsos_sweep.cuh"
RSOS_DEFINE_SX(1)
