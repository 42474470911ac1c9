// gemm.cuh -- batched FP64 GEMM used by the eigenvector and adjoint entry
// points: C = alpha * op(A) * op(B) + beta * C, column-major, op(X) = X or X^T.
// Several independent products ("tasks") run in one launch; a block finds its
// task by binary search over the tasks' first tile index.  Internal linkage:
// each translation unit that includes it gets its own copy.
#pragma once

#include <cuda_runtime.h>

namespace {

// ---------------------------------------------------------------------------
// Batched FP64 GEMM: C = alpha * op(A) * op(B) + beta * C (column-major; op(X) =
// X or X^T), 64 x 64 output tiles, K in chunks of 16 through shared memory,
// 4 x 4 outputs per thread.
// ---------------------------------------------------------------------------
struct GemmTask {
  const double* A;
  const double* B;
  double* C;
  long long lda, ldb, ldc;
  int M, N, K, transB;
  double alpha, beta;
  int tile0, tiles_n, ntile, transA;
};

__global__ void __launch_bounds__(256) k_gemm(const GemmTask* __restrict__ tasks, int ntask, int total) {
  __shared__ double As[16][64 + 1];
  __shared__ double Bs[16][64 + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  for (int tile = blockIdx.x; tile < total; tile += gridDim.x) {
    int lo = 0, hi = ntask - 1;
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (tasks[mid].tile0 <= tile) lo = mid; else hi = mid - 1;
    }
    const GemmTask& t = tasks[lo];
    const int local = tile - t.tile0;
    const int m0 = (local / t.tiles_n) * 64, n0 = (local % t.tiles_n) * 64;
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
    for (int k0 = 0; k0 < t.K; k0 += 16) {
      for (int idx = threadIdx.x; idx < 16 * 64; idx += 256) {
        int i = idx & 63, kk = idx >> 6;
        int r = m0 + i, c = k0 + kk;
        As[kk][i] = (r < t.M && c < t.K) ? (t.transA ? t.A[c + (long long)r * t.lda] : t.A[r + (long long)c * t.lda])
                                         : 0.0;
        int j, kb;
        if (t.transB) {
          j = idx & 63;
          kb = idx >> 6;
        } else {
          kb = idx & 15;
          j = idx >> 4;
        }
        int col = n0 + j, kr = k0 + kb;
        double v = 0.0;
        if (col < t.N && kr < t.K)
          v = t.transB ? t.B[col + (long long)kr * t.ldb] : t.B[kr + (long long)col * t.ldb];
        Bs[kb][j] = v;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < 16; ++kk) {
        double av[4], bv[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) av[a] = As[kk][ty * 4 + a];
#pragma unroll
        for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][tx * 4 + b];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = fma(av[a], bv[b], acc[a][b]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        int r = m0 + ty * 4 + a, c = n0 + tx * 4 + b;
        if (r < t.M && c < t.N) {
          double* cp = t.C + r + (long long)c * t.ldc;
          *cp = (t.beta == 0.0) ? t.alpha * acc[a][b] : fma(t.alpha, acc[a][b], t.beta * *cp);
        }
      }
  }
}

}  // namespace
