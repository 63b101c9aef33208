// FP64 instantiation of the sine-transform passes.
#define CSL_T double
#include "csl_pass_impl.cuh"
