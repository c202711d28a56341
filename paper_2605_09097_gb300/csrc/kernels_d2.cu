// Kernels and launchers of the 2D FP64 path.
#include "osmpm_kernels.cuh"

template struct osmpm::Kernels<2, double>;
