// FP32 instantiation of the long-line sine-transform passes.
#define CSL_T float
#include "csl_pass_big_impl.cuh"
