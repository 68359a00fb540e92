// Persistent engine kernels for 1x1 sub-tiles (2x2 DT tiles).
#include "rsos_persist_launch.cuh"
RSOS_DEFINE_PERSIST(1)
