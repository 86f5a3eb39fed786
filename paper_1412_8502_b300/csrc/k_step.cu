// The per-step kernels of the library in one translation unit: the cell and
// list build, the integrator and the pair forces, plus the persistent step
// kernel that runs all of them in one launch (k_persist.cuh), which needs
// their device code in the same unit.
#include "k_build.cuh"
#include "k_integrate.cuh"
#include "k_force.cuh"
#include "k_persist.cuh"
