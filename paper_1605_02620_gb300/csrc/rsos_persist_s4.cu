// Persistent engine kernels for 4x4 sub-tiles (8x8 DT tiles).
#include "rsos_persist_launch.cuh"
RSOS_DEFINE_PERSIST(4)
