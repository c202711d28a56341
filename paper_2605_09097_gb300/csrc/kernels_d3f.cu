// Kernels and launchers of the 3D mixed-precision path.
#include "osmpm_kernels.cuh"

template struct osmpm::Kernels<3, float>;
template struct osmpm::MultiKernels<3>;
