// One instance of the factor kernel (factor_kernel.cuh): the arithmetic of its O(B^3) work
// (HSAD_FI_AR: 0 float-float, 1 FP64) and the working precision of the whitening operand
// it writes (HSAD_FI_PREC: a Prec value). The build compiles this file once per pair, in
// parallel; the host dispatch in k_factor.cu picks the instance per launch.
#include "factor_kernel.cuh"

#ifndef HSAD_FI_AR
#define HSAD_FI_AR 0
#endif
#ifndef HSAD_FI_PREC
#define HSAD_FI_PREC 0
#endif

#define HSAD_FI_CAT2(a, b) a##b
#define HSAD_FI_CAT(a, b) HSAD_FI_CAT2(a, b)
#define HSAD_FI_SUFFIX HSAD_FI_CAT(HSAD_FI_CAT(a, HSAD_FI_AR), HSAD_FI_CAT(_p, HSAD_FI_PREC))

#if HSAD_FI_AR == 0
#define HSAD_FI_ARITH fk::ArFF
#else
#define HSAD_FI_ARITH fk::ArF64
#endif

// one more level so that the suffix macro is expanded before it is pasted
#define HSAD_FI_INSTANCE(ar, prec, suffix) HSAD_FACTOR_INSTANCE(ar, prec, suffix)

namespace hsad {
HSAD_FI_INSTANCE(HSAD_FI_ARITH, HSAD_FI_PREC, HSAD_FI_SUFFIX)
}  // namespace hsad
