// Surrogate MLP kernels (filled in by the surrogate component).
#include "rad_internal.cuh"
