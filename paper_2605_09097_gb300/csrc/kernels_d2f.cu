// Kernels and launchers of the 2D mixed-precision path.
#include "osmpm_kernels.cuh"

template struct osmpm::Kernels<2, float>;
template struct osmpm::MultiKernels<2>;
