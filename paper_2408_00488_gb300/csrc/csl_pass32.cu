// FP32 instantiation of the sine-transform passes.
#define CSL_T float
#include "csl_pass_impl.cuh"
