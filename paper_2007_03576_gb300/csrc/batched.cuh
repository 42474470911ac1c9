// batched.cuh -- types of the batched engine shared by the translation units
// that launch it (batched.cu, noalloc.cu).
#pragma once

#include "common.cuh"

#define B_MAX_BUCKETS 8
#define B_NW_MAX 128       // AED window limit of the batched engine
#define B_STAGE_COLS 32    // vectors staged per chunk of a window product

struct BatchedParams {
  int nmin, nibble, mode, exc_period;
  double thold;
  int nbuckets;
  int bucket_max_n[B_MAX_BUCKETS];  // bucket b holds m <= bucket_max_n[b]
  int ns[B_MAX_BUCKETS];
  int nw[B_MAX_BUCKETS];
  int nw_max;                       // largest window in the table (smem sizing)
};

struct BatchedDesc {
  double* H;
  double* Z;
  double* wr;
  double* wi;
  long long ldh, ldz;
  int n;
  int pad;
};

struct BatchedScratch {   // per thread block, global memory
  double* V;        // nw_max^2
  double* vbuf;     // 4 nw_max
  double* cand_re;  // nw_max
  double* cand_im;
  double* pairs;    // 2 * (MAX_BULGES_PER_CHAIN + 4)
  double* flops;    // 1: algorithmic flops this block applied (accumulated over its matrices)
};

struct BShared;

__global__ void k_batched(const BatchedDesc* __restrict__ desc, const int* __restrict__ order, int batch, int* counter,
                          int* info, BatchedScratch* scratch, BatchedParams P);
__global__ void k_batched_prep_z(const BatchedDesc* desc, int batch, int zinit);
