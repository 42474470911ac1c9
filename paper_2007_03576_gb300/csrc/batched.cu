// batched.cu -- placeholder until the persistent batched kernel lands.
#include "../../include/schur_gb300.h"
extern "C" int schur_hessenberg_batched(int, const int*, double* const*, const int*, double* const*, const int*,
                                        double* const*, double* const*, int*, const schur_opts*) {
  return SCHUR_ERR_UNSUPPORTED;
}
