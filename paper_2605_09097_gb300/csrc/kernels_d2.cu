// Kernels and launchers of the 2D path.
#include "osmpm_kernels.cuh"

template struct osmpm::Kernels<2>;
