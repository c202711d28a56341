// Kernels and launchers of the 3D path.
#include "osmpm_kernels.cuh"

template struct osmpm::Kernels<3>;
