// FP64 instantiation of the long-line sine-transform passes.
#define CSL_T double
#include "csl_pass_big_impl.cuh"
