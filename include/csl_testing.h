/*
 * csl_testing.h -- test hooks of libcsl.so.  They are not part of the method
 * (the paper has no counterpart); they expose, element by element, the
 * format conversions that the FP32-form kernels perform with integer field
 * moves instead of the hardware conversion (which issues on the FP64 pipe),
 * so that tests can compare them bit for bit with the hardware results.
 *
 * Arguments: in / out are DEVICE pointers owned by the caller, n >= 0
 * elements; stream is a cudaStream_t (NULL = legacy default stream).  The
 * call is stream-ordered and does not synchronise.  Returns CSL_OK,
 * CSL_INVALID_ARG (null pointer with n > 0, or n < 0) or CSL_CUDA_ERROR.
 */
#ifndef CSL_TESTING_H
#define CSL_TESTING_H

#include <stdint.h>

#include "csl.h"

#ifdef __cplusplus
extern "C" {
#endif

/* out[i] = in[i] rounded to nearest-even float (IEEE binary32) */
csl_status csl_test_convert_d2f(const double* in, float* out, int64_t n, void* stream);

/* out[i] = in[i] widened exactly to double */
csl_status csl_test_convert_f2d(const float* in, double* out, int64_t n, void* stream);

#ifdef __cplusplus
}
#endif

#endif
