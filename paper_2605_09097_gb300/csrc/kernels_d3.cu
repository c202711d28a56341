// Kernels and launchers of the 3D FP64 path.
#include "osmpm_kernels.cuh"

template struct osmpm::Kernels<3, double>;
