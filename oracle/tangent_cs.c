/*
 * Complex-step build of the FP64 oracle: the same source with every real
 * quantity (fields, populations and parameters) complex.  Perturbing an input
 * by i*h (h ~ 1e-30) and reading Im(output)/h gives the exact directional
 * derivative of the step (no subtractive cancellation), which pins the
 * hand-written adjoint through <u, J v> = <J^T u, v>.
 *
 * TEST INFRASTRUCTURE ONLY, like the oracle itself.  Every operation of the
 * step is analytic (products, sums, quotients and the square root in the unit
 * normal, whose argument has a positive real part), so the complex step is valid.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif
/* the system headers above are included before the type is redefined */
#define ORACLE_TANGENT_BUILD 1
#define double double _Complex
#define sqrt csqrt
#include "lbpf_oracle.c"
