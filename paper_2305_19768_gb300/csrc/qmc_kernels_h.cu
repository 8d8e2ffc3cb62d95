// Evaluator classes of part 3 of the kernels (see qmc_kernels.cu): compiled
// as their own translation unit so that the build runs in parallel.
#define QMC_PART 3
#include "qmc_kernels.cu"
