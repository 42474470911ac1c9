// eigvec.cu -- right eigenvectors from the real Schur form: phase (iii) of
// the eigenvalue computation (Sec. 1: H = Z S Z^T, then eigenvectors of S
// are carried back by Z).
//
// For each eigenvalue lambda_i of the standardised quasi-triangular S, x_i
// solves (S - lambda_i I) x = 0 with x_i zero below its own diagonal block:
// the block's part is fixed (1 for a 1x1 block; for the 2x2 block
// [[a, b], [c, d]] of a complex pair, (b, lambda - a), or (lambda - d, c) when
// both b and lambda - a vanish), the rows above follow by back substitution
// over the diagonal blocks, and the result is scaled to unit 2-norm and
// multiplied by Z.  A pivot below smin = max(u ||S||_F, 1e-300), u = 2^-52,
// is replaced by smin (the usual perturbation of nearly repeated
// eigenvalues).  Output in LAPACK's real format: column i = x_i for a real
// lambda_i; for a pair (i, i+1) with wi[i] > 0, columns i and i+1 hold the
// real and imaginary parts of x_i (x_{i+1} is its conjugate).
//
// Blocked back substitution (the standard right-looking scheme: all
// eigenvectors advance together, block row by block row, from the bottom):
// rows are cut into blocks K = [k0, k1) of ~64 rows that never split a 2x2
// diagonal block.  For each K, bottom to top:
//   k_ev_diag  every eigenvector with index >= k0 solves its rows in K: one
//              thread per eigenvector (shifts differ per eigenvector), S[K, K]
//              in shared memory, the thread's x[K] in shared memory
//              (thread-fastest, no bank conflicts), right-hand sides from
//              XS[K, i] (the updates from the blocks below);
//   k_gemm     XS[0:k0, k0:n] -= S[0:k0, K] XS[K, k0:n]  (FP64 tiles).
// All flops but O(n^2 b) are in the GEMMs: n^3/3 for the substitution and n^3
// for X = Z XS, where XS is upper triangular (plus one subdiagonal entry per
// pair), so column block J needs only the first (last column of J) + 2 rows.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/schur_gb300.h"
#include "gemm.cuh"
#include "host.h"

using schur::ck_at;

namespace {

constexpr int EV_B = 64;           // nominal rows per block row
constexpr int EV_BMAX = EV_B + 1;  // a block grows by one row to keep a 2x2 block whole
constexpr int EV_T = 64;           // eigenvectors (threads) per k_ev_diag block
constexpr int EV_FRO_BLOCKS = 256;

struct cx {
  double r, i;
};
__device__ __forceinline__ cx cx_sub(cx a, cx b) { return {a.r - b.r, a.i - b.i}; }
__device__ __forceinline__ cx cx_mul(cx a, cx b) { return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r}; }
__device__ __forceinline__ cx cx_scale(double s, cx a) { return {s * a.r, s * a.i}; }
__device__ __forceinline__ double cx_abs(cx a) { return hypot(a.r, a.i); }
__device__ __forceinline__ cx cx_div(cx a, cx b) {
  if (b.i == 0.0) return {a.r / b.r, a.i / b.r};
  const double d = b.r * b.r + b.i * b.i;
  return {(a.r * b.r + a.i * b.i) / d, (a.i * b.r - a.r * b.i) / d};
}

// Partial sums of squares of the quasi-triangular part of S (rows <= c + 1 of
// column c), one per block; k_ev_smin adds them in order.
__global__ void __launch_bounds__(256) k_ev_fro(const double* __restrict__ S, long long lds, int n,
                                                double* __restrict__ part) {
  __shared__ double red[8];
  double a = 0.0;
  for (int c = blockIdx.x; c < n; c += gridDim.x) {
    const double* sc = S + (long long)c * lds;
    const int hi = min(c + 1, n - 1);
    for (int r = threadIdx.x; r <= hi; r += blockDim.x) a = fma(sc[r], sc[r], a);
  }
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}

__global__ void k_ev_smin(const double* __restrict__ part, int np, double* __restrict__ smin) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double t = 0.0;
  for (int i = 0; i < np; ++i) t += part[i];
  *smin = fmax(0x1p-52 * sqrt(t), 1e-300);
}

// Rows K = [k0, k1) of every eigenvector with index >= k0 (see the header).
__global__ void __launch_bounds__(EV_T) k_ev_diag(const double* __restrict__ S, long long lds,
                                                  const double* __restrict__ wr, const double* __restrict__ wi,
                                                  double* __restrict__ XS, long long ldx, int n, int k0, int k1,
                                                  const double* __restrict__ sminp) {
  extern __shared__ double ev_smem[];
  const int B = k1 - k0;
  double* Ss = ev_smem;              // S[K, K], column-major, leading dimension B
  double* xr = Ss + B * B;           // x[K] of the block's eigenvectors, thread-fastest
  double* xi = xr + B * EV_T;
  for (int idx = threadIdx.x; idx < B * B; idx += EV_T) {
    const int r = idx % B, c = idx / B;
    Ss[idx] = S[(k0 + r) + (long long)(k0 + c) * lds];
  }
  __syncthreads();
  const int t = threadIdx.x;
  const int c = k0 + blockIdx.x * EV_T + t;
  if (c >= n) return;
  const double wic = wi[c];
  if (wic < 0.0) return;          // second column of a pair: written with the first
  const bool cpx = wic > 0.0 && c + 1 < n;
  const cx lam{wr[c], cpx ? wic : 0.0};
  const double smin = *sminp;
  const int top = cpx ? c + 1 : c;   // last row of the eigenvector's own block
  const int hi = min(top, k1 - 1);   // last row of K that is nonzero
  auto SS = [&](int row, int col) { return Ss[row - k0 + (col - k0) * B]; };
  auto XV = [&](int row) { return cx{xr[(row - k0) * EV_T + t], xi[(row - k0) * EV_T + t]}; };
  auto XSET = [&](int row, cx v) {
    xr[(row - k0) * EV_T + t] = v.r;
    xi[(row - k0) * EV_T + t] = v.i;
  };
  int k;
  if (top < k1) {
    if (!cpx) {
      XSET(c, cx{1.0, 0.0});
    } else {
      const double a = SS(c, c), b = SS(c, c + 1), cc = SS(c + 1, c), d = SS(c + 1, c + 1);
      const cx lma{lam.r - a, lam.i};
      if (fabs(b) + cx_abs(lma) > 0.0) {
        XSET(c, cx{b, 0.0});
        XSET(c + 1, lma);
      } else {
        XSET(c, cx{lam.r - d, lam.i});
        XSET(c + 1, cx{cc, 0.0});
      }
    }
    k = c - 1;
  } else {
    k = k1 - 1;
  }
  const double* xs_r = XS + (long long)c * ldx;
  const double* xs_i = cpx ? XS + (long long)(c + 1) * ldx : nullptr;
  while (k >= k0) {
    const bool two = (k - 1 >= k0) && SS(k, k - 1) != 0.0;
    if (!two) {
      cx r{xs_r[k], cpx ? xs_i[k] : 0.0};
      for (int l = k + 1; l <= hi; ++l) {
        const double s = SS(k, l);
        const cx xl = XV(l);
        r.r = fma(-s, xl.r, r.r);
        r.i = fma(-s, xl.i, r.i);
      }
      cx dd{SS(k, k) - lam.r, -lam.i};
      if (cx_abs(dd) < smin) dd = cx{smin, 0.0};
      XSET(k, cx_div(r, dd));
      k -= 1;
    } else {
      const int k1r = k - 1;   // rows (k - 1, k)
      cx r0{xs_r[k1r], cpx ? xs_i[k1r] : 0.0};
      cx r1{xs_r[k], cpx ? xs_i[k] : 0.0};
      for (int l = k + 1; l <= hi; ++l) {
        const double s0 = SS(k1r, l), s1 = SS(k, l);
        const cx xl = XV(l);
        r0.r = fma(-s0, xl.r, r0.r);
        r0.i = fma(-s0, xl.i, r0.i);
        r1.r = fma(-s1, xl.r, r1.r);
        r1.i = fma(-s1, xl.i, r1.i);
      }
      const cx m00{SS(k1r, k1r) - lam.r, -lam.i}, m11{SS(k, k) - lam.r, -lam.i};
      const double m01 = SS(k1r, k), m10 = SS(k, k1r);
      cx det = cx_mul(m00, m11);
      det.r -= m01 * m10;
      const double mx = fmax(fmax(cx_abs(m00), cx_abs(m11)), fmax(fabs(m01), fabs(m10)));
      const double lim = smin * fmax(1.0, mx);
      if (cx_abs(det) < lim) det = cx{lim, 0.0};
      const cx n0 = cx_sub(cx_mul(m11, r0), cx_scale(m01, r1));
      const cx n1 = cx_sub(cx_mul(m00, r1), cx_scale(m10, r0));
      XSET(k1r, cx_div(n0, det));
      XSET(k, cx_div(n1, det));
      k -= 2;
    }
  }
  double* wr_col = XS + (long long)c * ldx;
  for (int r = k0; r <= hi; ++r) wr_col[r] = xr[(r - k0) * EV_T + t];
  if (cpx) {
    double* wi_col = XS + (long long)(c + 1) * ldx;
    for (int r = k0; r <= hi; ++r) wi_col[r] = xi[(r - k0) * EV_T + t];
  }
}

// Scale every eigenvector (a column, or the column pair of a complex pair) to
// unit 2-norm; one warp per eigenvector.
__global__ void __launch_bounds__(256) k_ev_norm(double* __restrict__ XS, long long ldx,
                                                 const double* __restrict__ wi, int n) {
  const int lane = threadIdx.x & 31;
  for (int c = blockIdx.x * 8 + (threadIdx.x >> 5); c < n; c += gridDim.x * 8) {
    const double w = wi[c];
    if (w < 0.0) continue;
    const bool cpx = w > 0.0 && c + 1 < n;
    const int rows = min(n, c + (cpx ? 2 : 1));
    double* a = XS + (long long)c * ldx;
    double* b = cpx ? a + ldx : nullptr;
    double q = 0.0;
    for (int r = lane; r < rows; r += 32) {
      q = fma(a[r], a[r], q);
      if (cpx) q = fma(b[r], b[r], q);
    }
    for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
    double scale;
    if (q >= 0x1p-960 && q <= 0x1p960) {
      scale = 1.0 / sqrt(q);
    } else {
      // entries near the underflow / overflow threshold: scale by the largest
      double m = 0.0;
      for (int r = lane; r < rows; r += 32) {
        m = fmax(m, fabs(a[r]));
        if (cpx) m = fmax(m, fabs(b[r]));
      }
      for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
      double qq = 0.0;
      const double rm = (m > 0.0) ? 1.0 / m : 0.0;
      for (int r = lane; r < rows; r += 32) {
        const double u = a[r] * rm;
        qq = fma(u, u, qq);
        if (cpx) {
          const double v = b[r] * rm;
          qq = fma(v, v, qq);
        }
      }
      for (int o = 16; o > 0; o >>= 1) qq += __shfl_xor_sync(0xffffffffu, qq, o);
      scale = (m > 0.0) ? rm / sqrt(qq) : 0.0;
    }
    for (int r = lane; r < rows; r += 32) {
      a[r] *= scale;
      if (cpx) b[r] *= scale;
    }
  }
}

constexpr size_t EV_DIAG_SMEM = (EV_BMAX * EV_BMAX + 2 * EV_BMAX * EV_T) * sizeof(double);

// k_ev_diag's dynamic shared-memory limit, raised once per device.
std::mutex g_ev_mu;
bool g_ev_done[64] = {false};

void ev_raise_limit() {
  int dev = 0;
  ck_at(cudaGetDevice(&dev), __LINE__);
  if (dev < 0 || dev >= 64) throw schur::CudaError{cudaErrorInvalidDevice};
  std::lock_guard<std::mutex> lock(g_ev_mu);
  if (g_ev_done[dev]) return;
  ck_at(cudaFuncSetAttribute(k_ev_diag, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)EV_DIAG_SMEM), __LINE__);
  g_ev_done[dev] = true;
}

size_t tasks_bytes(int n) {
  const size_t nblk = (size_t)(n + EV_B - 1) / EV_B + 2;
  return ((2 * nblk) * sizeof(GemmTask) + 255) / 256 * 256;
}

size_t workspace_need(int n, bool backtransform) {
  size_t b = 0;
  if (backtransform) b += ((size_t)n * n * sizeof(double) + 255) / 256 * 256;
  b += tasks_bytes(n);
  b += (EV_FRO_BLOCKS + 1) * sizeof(double) + 256;
  return b;
}

}  // namespace

extern "C" int schur_eigenvectors_workspace(int n, int with_z, size_t* bytes) {
  if (n < 0) return -1;
  if (!bytes) return -3;
  *bytes = workspace_need(std::max(n, 1), with_z != 0);
  return SCHUR_OK;
}

namespace schur {

size_t eigvec_workspace(int n, bool with_z) { return workspace_need(std::max(n, 1), with_z); }

// The body of schur_eigenvectors on stream st with scratch `mem`
// (eigvec_workspace(n, Z != nullptr) bytes); hwi is a host copy of wi (the
// pair structure).  Does not synchronise; adds its launches and GEMM flops.
void eigvec_run(int n, const double* S, int lds, const double* Z, int ldz, const double* wr, const double* wi,
                const double* hwi, double* X, int ldx, cudaStream_t st, char* mem, long long* launches,
                double* flops) {
  const bool bt = Z != nullptr;
  char* p = mem;
  double* XS = X;
  long long ldxs = ldx;
  if (bt) {
    XS = (double*)p;
    ldxs = n;
    p += ((size_t)n * n * sizeof(double) + 255) / 256 * 256;
  }
  GemmTask* dtask = (GemmTask*)p;
  p += tasks_bytes(n);
  double* part = (double*)p;
  double* smin = part + EV_FRO_BLOCKS;
  const int nsm = num_sms();
  ev_raise_limit();

  std::vector<int> starts;   // block starts, bottom block first
  for (int k1 = n; k1 > 0;) {
    int k0 = std::max(0, k1 - EV_B);
    if (k0 > 0 && hwi[k0 - 1] > 0.0) --k0;   // keep the pair (k0 - 1, k0) together
    starts.push_back(k0);
    k1 = k0;
  }

  // every GEMM task of the call, uploaded once
  std::vector<GemmTask> tasks;
  auto task = [&](const double* A, long long lda, const double* Bm, long long ldb, double* C, long long ldc, int M,
                  int N, int K, double alpha, double beta) {
    GemmTask tk;
    memset(&tk, 0, sizeof(tk));
    tk.A = A; tk.B = Bm; tk.C = C; tk.lda = lda; tk.ldb = ldb; tk.ldc = ldc;
    tk.M = M; tk.N = N; tk.K = K; tk.transB = 0; tk.alpha = alpha; tk.beta = beta;
    tk.tiles_n = (N + 63) / 64;
    tk.ntile = ((M + 63) / 64) * tk.tiles_n;
    tasks.push_back(tk);
  };
  int k1 = n;
  std::vector<int> sub_task(starts.size(), -1);
  for (size_t bi = 0; bi < starts.size(); ++bi) {
    const int k0 = starts[bi];
    if (k0 > 0) {
      sub_task[bi] = (int)tasks.size();
      task(S + (long long)k0 * lds, lds, XS + k0 + (long long)k0 * ldxs, ldxs, XS + (long long)k0 * ldxs, ldxs, k0,
           n - k0, k1 - k0, -1.0, 1.0);
      *flops += 2.0 * k0 * (double)(n - k0) * (k1 - k0);
    }
    k1 = k0;
  }
  const int bt_first = (int)tasks.size();
  if (bt) {
    int tile = 0;
    for (int c0 = 0; c0 < n; c0 += 64) {
      const int c1 = std::min(n, c0 + 64);
      const int K = std::min(n, c1 + 1);
      task(Z, ldz, XS + (long long)c0 * ldxs, ldxs, X + (long long)c0 * ldx, ldx, n, c1 - c0, K, 1.0, 0.0);
      tasks.back().tile0 = tile;
      tile += tasks.back().ntile;
      *flops += 2.0 * n * (double)(c1 - c0) * K;
    }
  }
  if (!tasks.empty())
    ck_at(cudaMemcpyAsync(dtask, tasks.data(), tasks.size() * sizeof(GemmTask), cudaMemcpyHostToDevice, st),
          __LINE__);

  // XS = 0 (entries below each eigenvector's block stay zero)
  ck_at(cudaMemset2DAsync(XS, ldxs * sizeof(double), 0, n * sizeof(double), n, st), __LINE__);
  k_ev_fro<<<EV_FRO_BLOCKS, 256, 0, st>>>(S, lds, n, part);
  k_ev_smin<<<1, 32, 0, st>>>(part, EV_FRO_BLOCKS, smin);
  *launches += 2;
  k1 = n;
  for (size_t bi = 0; bi < starts.size(); ++bi) {
    const int k0 = starts[bi];
    const int cols = n - k0;
    const size_t smem = ((size_t)(k1 - k0) * (k1 - k0) + 2 * (size_t)(k1 - k0) * EV_T) * sizeof(double);
    k_ev_diag<<<(cols + EV_T - 1) / EV_T, EV_T, smem, st>>>(S, lds, wr, wi, XS, ldxs, n, k0, k1, smin);
    ++*launches;
    if (sub_task[bi] >= 0) {
      const GemmTask& tk = tasks[sub_task[bi]];
      k_gemm<<<std::min(tk.ntile, 4 * nsm), 256, 0, st>>>(dtask + sub_task[bi], 1, tk.ntile);
      ++*launches;
    }
    k1 = k0;
  }
  ck_at(cudaGetLastError(), __LINE__);
  k_ev_norm<<<std::min((n + 7) / 8, 8 * nsm), 256, 0, st>>>(XS, ldxs, wi, n);
  ++*launches;
  if (bt) {
    int total = 0;
    for (size_t i = bt_first; i < tasks.size(); ++i) total += tasks[i].ntile;
    k_gemm<<<std::min(total, 4 * nsm), 256, 0, st>>>(dtask + bt_first, (int)tasks.size() - bt_first, total);
    ++*launches;
  }
  ck_at(cudaGetLastError(), __LINE__);
}

}  // namespace schur

extern "C" int schur_eigenvectors(int n, const double* S, int lds, const double* Z, int ldz, const double* wr,
                                  const double* wi, double* X, int ldx, const schur_opts* opts) {
  if (n < 0) return -1;
  if (n > 0 && S == nullptr) return -2;
  if (lds < std::max(1, n)) return -3;
  if (Z != nullptr && ldz < std::max(1, n)) return -5;
  if (n > 0 && wr == nullptr) return -6;
  if (n > 0 && wi == nullptr) return -7;
  if (n > 0 && X == nullptr) return -8;
  if (ldx < std::max(1, n)) return -9;
  memset(&schur::g_stats, 0, sizeof(schur::g_stats));
  if (n == 0) return SCHUR_OK;
  schur_opts o;
  schur::read_opts(opts, &o);
  cudaStream_t st = (cudaStream_t)o.stream;
  const size_t need = workspace_need(n, Z != nullptr);
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
    // pair structure (host copy of wi) for the block rows
    std::vector<double> hwi(n);
    ck_at(cudaMemcpyAsync(hwi.data(), wi, n * sizeof(double), cudaMemcpyDeviceToHost, st), __LINE__);
    ck_at(cudaStreamSynchronize(st), __LINE__);
    long long launches = 0;
    double flops = 0.0;
    schur::eigvec_run(n, S, lds, Z, ldz, wr, wi, hwi.data(), X, ldx, st, mem, &launches, &flops);
    ck_at(cudaStreamSynchronize(st), __LINE__);
    schur::g_stats.kernel_launches = launches;
    schur::g_stats.flops = flops;
  } catch (const schur::CudaError&) {
    rc = SCHUR_ERR_CUDA;
  }
  if (own) cudaFree(mem);
  return rc;
}
