// adjoint.cu -- placeholder until the adjoint kernels land.
#include "../../include/schur_gb300.h"
extern "C" int schur_eig_backward(int, const double*, int, const double*, int, const double*, const double*,
                                  const double*, const double*, double*, int, const schur_opts*) {
  return SCHUR_ERR_UNSUPPORTED;
}
extern "C" int schur_eig_backward_batched(int, const int*, double* const*, const int*, double* const*, const int*,
                                          double* const*, double* const*, double* const*, double* const*,
                                          double* const*, const int*, const schur_opts*) {
  return SCHUR_ERR_UNSUPPORTED;
}
