// hessred.cu -- Householder reduction of a general matrix to upper Hessenberg
// form, A = Q H Q^T: phase (i) of the eigenvalue computation that precedes
// the multishift QR iteration (Sec. 1; the paper times it with the rest of
// the pipeline in Sec. 5.5).
//
// Method: the textbook unblocked reduction (Golub & Van Loan, Alg. 7.4.2)
// with LAPACK's reflector convention (dlarfg: beta = -sign(alpha) ||x||,
// v(1) = 1), so H agrees with dgehrd's up to rounding.  Step j builds
// P_j = I - tau v v^T on rows/columns j+1..n-1 from x = A[j+1:n, j] and
// applies it from both sides.  Q is formed afterwards, backward
// (Q = P_0 (P_1 (... P_{n-3}))), as dorghr does: each P_j then meets only the
// trailing (n-j-1)^2 block, (4/3) n^3 flops instead of 2 n^3 forward.
//
// Why unblocked on this GPU: its FP64 tensor-core rate equals its FP64 FMA
// rate, so the blocked (BLAS-3) form buys no arithmetic speed; what it buys
// is less memory traffic.  The unblocked step moves each trailing entry once
// to and from DRAM (the second pass of a kernel re-reads it from L2), 16 bytes
// per 4 flops: at the FP64 peak that is ~4.4 TB/s, inside HBM bandwidth, so
// the reduction is bound by the FP64 pipe either way, and the unblocked form
// has no panel factorisation on the critical path.
//
// Storage, as in LAPACK: after step j, column j holds beta_j on the
// subdiagonal and the reflector's vector v_{j+2..n-1} below it (v_{j+1} = 1
// is implicit); the entries below the subdiagonal are set to zero once Q has
// been formed from them.  Every product uses the scaled v (|v_p| <= 1), so the
// reduction overflows only where the matrix entries themselves approach the
// overflow threshold.
//
// Kernels per step j (stream-ordered; no atomics, so results are
// bit-reproducible):
//   k_hr_refl   one block: sigma^2 from the previous step's partial sums of
//               squares (fixed order), (tau, beta), v = x / (alpha - beta)
//               written over x;
//   k_hr_left   A[j+1:, c] <- P_j A[j+1:, c] for c >= j+1, one warp per
//               column (dot pass, then update pass re-reading from L1/L2);
//   k_hr_right  A[:, j+1:] <- A[:, j+1:] P_j on 8-row slabs (quarter-warps on
//               consecutive rows of one column: 64-byte segments); each slab
//               also writes its part of the sum of squares of the new column
//               j+1 below row j+2, the norm of step j+1's reflector.
// Q formation reuses k_hr_left with the stored tau_j and v_j.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>

#include "../../include/schur_gb300.h"
#include "host.h"

namespace {

constexpr int HR_THREADS = 256;       // 8 warps
constexpr int HR_WARPS = HR_THREADS / 32;
constexpr int HR_SLAB = 8;            // rows per block of k_hr_right
constexpr int HR_GROUPS = HR_THREADS / HR_SLAB;   // column groups per slab

// Deterministic block sum: strided per-thread sums, a fixed shuffle tree,
// then the warps' sums in warp order.  Every thread gets the result.
__device__ double hr_block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < HR_WARPS; ++w) t += red[w];
  return t;
}

__device__ double hr_block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < HR_WARPS; ++w) t = fmax(t, red[w]);
  return t;
}

// Reflector of step j from column j (alpha = x[j+1], tail x[j+2..n-1]) and
// sigma^2 = the sum of the partials, in one block: tau = 0 when the tail is
// zero (P_j = I, beta = alpha); else beta = -sign(alpha) hypot(alpha, sigma),
// tau = (beta - alpha) / beta, and the tail is overwritten by
// v = x / (alpha - beta).  When sigma^2 lies outside [2^-960, 2^960] (tail
// entries near the underflow or overflow threshold, or a zero sum, which can
// come from squares that underflowed) the norm is recomputed from the column
// scaled by its largest magnitude; that largest magnitude is what tells a
// zero tail.  refl[2j] = tau,
// refl[2j+1] = beta; x[j+1] is left as alpha (its final value, beta, is
// written by k_hr_finish).
__global__ void __launch_bounds__(HR_THREADS) k_hr_refl(double* __restrict__ A, long long lda, int n, int j,
                                                        const double* __restrict__ part, int npart,
                                                        double* __restrict__ refl) {
  __shared__ double red[HR_WARPS];
  double* x = A + (long long)j * lda;
  double a = 0.0;
  for (int i = threadIdx.x; i < npart; i += blockDim.x) a += part[i];
  const double ss = hr_block_sum(a, red);
  const double alpha = x[j + 1];
  double sigma;
  if (ss >= 0x1p-960 && ss <= 0x1p960) {
    sigma = sqrt(ss);
  } else {   // also ss = 0: a zero tail, or squares that underflowed
    double m = 0.0;
    for (int p = j + 2 + threadIdx.x; p < n; p += blockDim.x) m = fmax(m, fabs(x[p]));
    m = hr_block_max(m, red);
    if (m > 0.0 && m <= 1.7976931348623157e308) {
      const double r = 1.0 / m;
      double q = 0.0;
      for (int p = j + 2 + threadIdx.x; p < n; p += blockDim.x) {
        const double t = x[p] * r;
        q = fma(t, t, q);
      }
      sigma = m * sqrt(hr_block_sum(q, red));
    } else {
      sigma = sqrt(ss);
    }
  }
  double tau = 0.0, beta = alpha;
  if (sigma != 0.0) {
    beta = -copysign(hypot(alpha, sigma), alpha);
    tau = (beta - alpha) / beta;
    const double d = alpha - beta;
    for (int p = j + 2 + threadIdx.x; p < n; p += blockDim.x) x[p] = x[p] / d;
  }
  if (threadIdx.x == 0) {
    refl[2 * j] = tau;
    refl[2 * j + 1] = beta;
  }
}

// M[j+1:n, c] <- P_j M[j+1:n, c] for c = j+1..n-1, one warp per column; v
// below row j+1 of column j of A.
__global__ void __launch_bounds__(HR_THREADS) k_hr_left(double* __restrict__ M, long long ldm,
                                                        const double* __restrict__ A, long long lda, int n, int j,
                                                        const double* __restrict__ refl) {
  const double tau = refl[2 * j];
  if (tau == 0.0) return;
  const double* v = A + (long long)j * lda;
  const int lane = threadIdx.x & 31;
  const int nwarp = gridDim.x * HR_WARPS;
  for (int c = j + 1 + blockIdx.x * HR_WARPS + (threadIdx.x >> 5); c < n; c += nwarp) {
    double* mc = M + (long long)c * ldm;
    double d0 = 0.0, d1 = 0.0, d2 = 0.0, d3 = 0.0;
    int p = j + 2 + lane;
    for (; p + 96 < n; p += 128) {
      d0 = fma(v[p], mc[p], d0);
      d1 = fma(v[p + 32], mc[p + 32], d1);
      d2 = fma(v[p + 64], mc[p + 64], d2);
      d3 = fma(v[p + 96], mc[p + 96], d3);
    }
    for (; p < n; p += 32) d0 = fma(v[p], mc[p], d0);
    double d = (d0 + d1) + (d2 + d3);
    for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
    const double w = tau * (mc[j + 1] + d);
    __syncwarp();
    if (lane == 0) mc[j + 1] -= w;
    for (p = j + 2 + lane; p + 96 < n; p += 128) {
      const double e0 = mc[p], e1 = mc[p + 32], e2 = mc[p + 64], e3 = mc[p + 96];
      const double v0 = v[p], v1 = v[p + 32], v2 = v[p + 64], v3 = v[p + 96];
      mc[p] = fma(-w, v0, e0);
      mc[p + 32] = fma(-w, v1, e1);
      mc[p + 64] = fma(-w, v2, e2);
      mc[p + 96] = fma(-w, v3, e3);
    }
    for (; p < n; p += 32) mc[p] = fma(-w, v[p], mc[p]);
  }
}

// A[:, j+1:n] <- A[:, j+1:n] P_j for the HR_SLAB rows of this block; writes
// the block's part of sum_{r >= j+3} A[r, j+1]^2 (after the update) to
// part[].  Each thread walks its row through every HR_GROUPS-th column, four
// columns per iteration with their loads issued together (the kernel is
// limited by load latency, not by the FP64 pipe, when fewer loads are in
// flight).
__global__ void __launch_bounds__(HR_THREADS) k_hr_right(double* __restrict__ A, long long lda, int n, int j,
                                                         const double* __restrict__ refl, double* __restrict__ part) {
  __shared__ double red[HR_GROUPS][HR_SLAB + 1];
  __shared__ double gsh[HR_SLAB];
  const double tau = refl[2 * j];
  const double* x = A + (long long)j * lda;   // v of step j below row j+1
  const int rl = threadIdx.x % HR_SLAB;
  const int g = threadIdx.x / HR_SLAB;
  const int row = blockIdx.x * HR_SLAB + rl;
  const bool rok = row < n;
  double* Ar = A + row;
  const long long step = (long long)HR_GROUPS * lda;
  if (tau != 0.0) {
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    if (rok) {
      int c = j + 2 + g;
      const double* e = Ar + (long long)c * lda;
      for (; c + 3 * HR_GROUPS < n; c += 4 * HR_GROUPS, e += 4 * step) {
        const double e0 = e[0], e1 = e[step], e2 = e[2 * step], e3 = e[3 * step];
        const double v0 = x[c], v1 = x[c + HR_GROUPS], v2 = x[c + 2 * HR_GROUPS], v3 = x[c + 3 * HR_GROUPS];
        a0 = fma(e0, v0, a0);
        a1 = fma(e1, v1, a1);
        a2 = fma(e2, v2, a2);
        a3 = fma(e3, v3, a3);
      }
      for (; c < n; c += HR_GROUPS, e += step) a0 = fma(e[0], x[c], a0);
    }
    red[g][rl] = (a0 + a1) + (a2 + a3);
  }
  __syncthreads();
  if (threadIdx.x < HR_SLAB) {
    double* a1p = A + (long long)(j + 1) * lda + row;
    double a1 = rok ? *a1p : 0.0;
    double gv = 0.0;
    if (tau != 0.0) {
      double S = 0.0;
      for (int k = 0; k < HR_GROUPS; ++k) S += red[k][rl];
      const double f = tau * (a1 + S);
      a1 -= f;
      if (rok) *a1p = a1;
      gv = f;
    }
    gsh[rl] = gv;
    double sq = (rok && row >= j + 3) ? a1 * a1 : 0.0;
    for (int o = HR_SLAB / 2; o > 0; o >>= 1) sq += __shfl_xor_sync((1u << HR_SLAB) - 1u, sq, o);
    if (threadIdx.x == 0) part[blockIdx.x] = sq;
  }
  __syncthreads();
  if (tau != 0.0 && rok) {
    const double gv = gsh[rl];
    int c = j + 2 + g;
    double* e = Ar + (long long)c * lda;
    for (; c + 3 * HR_GROUPS < n; c += 4 * HR_GROUPS, e += 4 * step) {
      const double e0 = e[0], e1 = e[step], e2 = e[2 * step], e3 = e[3 * step];
      const double v0 = x[c], v1 = x[c + HR_GROUPS], v2 = x[c + 2 * HR_GROUPS], v3 = x[c + 3 * HR_GROUPS];
      e[0] = fma(-gv, v0, e0);
      e[step] = fma(-gv, v1, e1);
      e[2 * step] = fma(-gv, v2, e2);
      e[3 * step] = fma(-gv, v3, e3);
    }
    for (; c < n; c += HR_GROUPS, e += step) e[0] = fma(-gv, x[c], e[0]);
  }
}

// part[0] = sum_{p >= 2} A[p, 0]^2 (the norm for step 0).
__global__ void __launch_bounds__(HR_THREADS) k_hr_part0(const double* __restrict__ A, int n,
                                                         double* __restrict__ part) {
  __shared__ double red[HR_WARPS];
  double a = 0.0;
  for (int p = 2 + threadIdx.x; p < n; p += blockDim.x) a = fma(A[p], A[p], a);
  a = hr_block_sum(a, red);
  if (threadIdx.x == 0) part[0] = a;
}

// flag <- 1 if A has a non-finite entry.
__global__ void k_hr_check(const double* __restrict__ A, long long lda, int n, int* flag) {
  for (int c = blockIdx.x; c < n; c += gridDim.x) {
    const double* ac = A + (long long)c * lda;
    for (int r = threadIdx.x; r < n; r += blockDim.x)
      if (!isfinite(ac[r])) *flag = 1;
  }
}

__global__ void k_hr_eye(double* __restrict__ Q, long long ldq, int n) {
  for (int c = blockIdx.x; c < n; c += gridDim.x)
    for (int r = threadIdx.x; r < n; r += blockDim.x) Q[r + (long long)c * ldq] = (r == c) ? 1.0 : 0.0;
}

// Column j <- (..., beta_j, 0, ..., 0) for j = 0..n-3.
__global__ void k_hr_finish(double* __restrict__ A, long long lda, int n, const double* __restrict__ refl) {
  for (int j = blockIdx.x; j < n - 2; j += gridDim.x) {
    double* aj = A + (long long)j * lda;
    if (threadIdx.x == 0) aj[j + 1] = refl[2 * j + 1];
    for (int p = j + 2 + threadIdx.x; p < n; p += blockDim.x) aj[p] = 0.0;
  }
}

}  // namespace

using schur::ck_at;

extern "C" int schur_hessenberg_reduce_workspace(int n, size_t* bytes) {
  if (n < 0) return -1;
  if (!bytes) return -2;
  const size_t slabs = (size_t)(n + HR_SLAB - 1) / HR_SLAB;
  *bytes = ((2 * (size_t)std::max(n, 1) + slabs + 1) * sizeof(double) + 255) / 256 * 256 + 256;
  return SCHUR_OK;
}

extern "C" int schur_hessenberg_reduce(int n, double* A, int lda, double* Q, int ldq, const schur_opts* opts) {
  if (n < 0) return -1;
  if (n > 0 && A == nullptr) return -2;
  if (lda < std::max(1, n)) return -3;
  if (Q != nullptr && ldq < std::max(1, n)) return -5;
  memset(&schur::g_stats, 0, sizeof(schur::g_stats));
  if (n == 0) return SCHUR_OK;
  schur_opts o;
  schur::read_opts(opts, &o);
  cudaStream_t st = (cudaStream_t)o.stream;
  size_t need = 0;
  schur_hessenberg_reduce_workspace(n, &need);
  char* mem = nullptr;
  bool own = false;
  if (o.workspace) {
    if (schur::workspace_unusable(o, need)) return SCHUR_ERR_WORKSPACE;
    mem = (char*)o.workspace;
  } else {
    if (cudaMalloc((void**)&mem, need) != cudaSuccess) {
      cudaGetLastError();
      return SCHUR_ERR_NOMEM;
    }
    own = true;
  }
  int rc = SCHUR_OK;
  try {
    double* refl = (double*)mem;
    const int slabs = (n + HR_SLAB - 1) / HR_SLAB;
    double* part = refl + 2 * (size_t)n;
    int* flag = (int*)(mem + need - 256);
    long long launches = 0;
    const int nsm = schur::num_sms();
    ck_at(cudaMemsetAsync(flag, 0, sizeof(int), st), __LINE__);
    k_hr_check<<<std::min(n, 4 * nsm), 256, 0, st>>>(A, lda, n, flag);
    ck_at(cudaGetLastError(), __LINE__);
    ++launches;
    int hflag = 0;
    ck_at(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st), __LINE__);
    ck_at(cudaStreamSynchronize(st), __LINE__);
    if (hflag) {
      rc = SCHUR_ERR_NONFINITE;
    } else {
      double flops = 0.0;
      if (n > 2) {
        k_hr_part0<<<1, HR_THREADS, 0, st>>>(A, n, part);
        ck_at(cudaGetLastError(), __LINE__);
        ++launches;
        for (int j = 0; j + 2 < n; ++j) {
          const int m = n - j - 1;
          const int lgrid = std::max(1, std::min((m + HR_WARPS - 1) / HR_WARPS, 4 * nsm));
          k_hr_refl<<<1, HR_THREADS, 0, st>>>(A, lda, n, j, part, j == 0 ? 1 : slabs, refl);
          k_hr_left<<<lgrid, HR_THREADS, 0, st>>>(A, lda, A, lda, n, j, refl);
          k_hr_right<<<slabs, HR_THREADS, 0, st>>>(A, lda, n, j, refl, part);
          launches += 3;
          flops += 4.0 * m * m + 4.0 * n * m;
        }
        ck_at(cudaGetLastError(), __LINE__);
      }
      if (Q != nullptr) {
        k_hr_eye<<<std::min(n, 4 * nsm), 256, 0, st>>>(Q, ldq, n);
        ++launches;
        for (int j = n - 3; j >= 0; --j) {
          const int m = n - j - 1;
          const int lgrid = std::max(1, std::min((m + HR_WARPS - 1) / HR_WARPS, 4 * nsm));
          k_hr_left<<<lgrid, HR_THREADS, 0, st>>>(Q, ldq, A, lda, n, j, refl);
          ++launches;
          flops += 4.0 * m * m;
        }
        ck_at(cudaGetLastError(), __LINE__);
      }
      if (n > 2) {
        k_hr_finish<<<std::min(n - 2, 4 * nsm), 256, 0, st>>>(A, lda, n, refl);
        ck_at(cudaGetLastError(), __LINE__);
        ++launches;
      }
      ck_at(cudaStreamSynchronize(st), __LINE__);
      schur::g_stats.kernel_launches = launches;
      schur::g_stats.flops = flops;
    }
  } catch (const schur::CudaError&) {
    rc = SCHUR_ERR_CUDA;
  }
  if (own) cudaFree(mem);
  return rc;
}
