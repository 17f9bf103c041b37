// Float instantiation of the hot-path launch sequences.
#include "hobc_run.cuh"
HOBC_INSTANTIATE(float)
