// Persistent engine kernels for 8x8 sub-tiles (16x16 DT tiles).
#include "rsos_persist_launch.cuh"
RSOS_DEFINE_PERSIST(8)
