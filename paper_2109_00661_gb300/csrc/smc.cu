// RJSMC stage kernels (reweight with TESS bisection, within-model systematic
// resampling, RJ mutation, model odds).  Filled in by the SMC build-out.
#include "aem_internal.h"
