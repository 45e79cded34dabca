// The mixed form's sweep kernel (k_sample<float>) with the register budget
// that keeps three CTAs per SM resident, for systems whose walkers fit three
// or more per SM in shared memory.  The kernel is the one of vmc_walker.cu;
// this unit instantiates only that variant, so that the two build in
// parallel.
#define VMC_SWEEP_V3_ONLY
#include "vmc_walker.cu"
