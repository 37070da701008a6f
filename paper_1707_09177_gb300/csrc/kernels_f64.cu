// float64 instantiation of the pass kernels.
#define GAD_REAL double
#include "kernels_impl.cuh"
