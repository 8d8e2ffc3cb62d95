// Evaluator classes of part 2 of the kernels (see qmc_kernels.cu): compiled
// as their own translation unit so that the build runs in parallel.
#define QMC_PART 2
#include "qmc_kernels.cu"
