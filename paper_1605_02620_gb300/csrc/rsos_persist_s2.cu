// Persistent engine kernels for 2x2 sub-tiles (4x4 DT tiles).
#include "rsos_persist_launch.cuh"
RSOS_DEFINE_PERSIST(2)
