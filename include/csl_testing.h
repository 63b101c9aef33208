/*
 * csl_testing.h -- test and measurement hooks of libcsl.so.  They are not
 * part of the method (the paper has no counterpart).  The conversion hooks
 * expose, element by element, the format conversions that the FP32-form
 * kernels perform with integer field moves instead of the hardware
 * conversion (which issues on the FP64 pipe), so that tests can compare them
 * bit for bit with the hardware results.
 *
 * Conversion hooks: in / out are DEVICE pointers owned by the caller, n >= 0
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

/*
 * Measurement hook (no counterpart in the paper): the cost of one
 * synchronisation point between two dependent stages of an iteration, on the
 * current device, in the two forms a device-resident solver can take.
 *   out[0]  microseconds per kernel of a CUDA graph of `kernels` kernels
 *           without work, launched with programmatic dependent launch (the
 *           form the solver's graph uses); grid 2 CTAs per SM, 256 threads,
 *           48 KB dynamic shared memory, each waiting on its predecessor;
 *   out[1]  the same without programmatic dependent launch;
 *   out[2]  microseconds per grid barrier of one cooperative kernel of
 *           (resident CTAs per SM, at most 2) x SMs CTAs crossing `barriers`
 *           barriers (an arrival counter in global memory and a spin).
 * Every spin is bounded: about one second, or, with `unreachable` != 0,
 * about one millisecond with every barrier target one arrival above what the
 * grid provides, so that every wait runs out.  A CTA whose wait runs out
 * records it in a flag and returns (it has nothing in flight), and the call
 * returns CSL_TIMEOUT; the context stays usable.
 * kernels in [1, 100000], barriers in [1, 1000000], out a HOST array of 3
 * (out[2] is filled also on CSL_TIMEOUT).  Synchronous; allocates 16 bytes of
 * device memory and a stream for the call.  Returns CSL_OK, CSL_TIMEOUT,
 * CSL_INVALID_ARG, CSL_UNSUPPORTED_SIZE (no cooperative launch) or
 * CSL_CUDA_ERROR.
 */
csl_status csl_probe_sync_cost(int kernels, int barriers, int unreachable, double out[3]);

#ifdef __cplusplus
}
#endif

#endif
