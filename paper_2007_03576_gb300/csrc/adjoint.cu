// adjoint.cu -- eigenvalue adjoint dL/dH (not in the paper).
//
// For cotangents g_k = dL/dRe(lambda_k) + i dL/dIm(lambda_k), first-order
// perturbation theory (d lambda = y^H dH x / y^H x) gives
//     dL/dH = Z G Z^T,   G = Re( sum_k conj(g_k) / c_k  w_k x_k^T ),
// with x_k, w_k = conj(y_k) the right eigenvectors of S and of S^T
// (S x = lambda x, S^T w = lambda w) and c_k = w_k^T x_k.  For a complex pair
// (lambda, conj(lambda)) the two terms combine into
//     Re( (conj(g_k) + g_{k+1}) / c_k  w_k x_k^T )
// (the partner's vectors are the conjugates), so one complex vector pair per
// diagonal block is computed:
//   * k_adj_vectors: one warp per diagonal block; x by block back
//     substitution in column (axpy) order -- after x_j is final, column j of
//     S updates the right-hand sides above it, reading S contiguously --; w by
//     forward substitution with the dot products over contiguous columns of
//     S; c = w_b^T x_b involves the block rows only.  Writes
//     XR = Re x, XI = Im x, P = Re(e w), Q = Im(e w) with e the coefficient
//     above (zero columns for the second row of a pair).
//   * k_gemm: G = P XR^T - Q XI^T, T = Z G, dH = T Z^T (FP64 FFMA tiles).
// That per-warp path serves the batched entry point and single matrices below
// ADJ_BLOCKED_MIN (where it is also the faster one: 4.3 / 6.9 / 13.9 ms against
// 10.7 / 15.4 / 21.7 ms at n = 512 / 768 / 1024 on a GB300, the blocked path's
// launches and serial block rows dominating there).  Larger single matrices
// (any order) take both vector sets
// from the blocked back substitution of the eigenvector solver (eigvec.cu):
//   * x_k: the right eigenvectors X of S in LAPACK's real format;
//   * w_k: with R the reversal permutation (R e_i = e_{n-1-i}),
//     S' = R S^T R is upper quasi-triangular with the same 2x2 blocks (a
//     standardised [[a, b], [c, a]] maps to itself), and S^T w = lam w iff
//     S' (R w) = lam (R w): w_k = R x'_{n-1-k} with x' the right eigenvectors
//     of S' (a pair (k, k+1) of S sits at (n-2-k, n-1-k) of S', the
//     eigenvalue with positive imaginary part first: wi' = -R wi);
//   * k_adj_combine: c_k, e_k and P with G = P X^T (P column k = Re(e w),
//     column k+1 = -Im(e w) for a pair);
//   * three GEMM launches that skip the known zeros: P is lower triangular
//     and X upper triangular up to one entry per pair, so G(i, j) = 0 for
//     i < j - 2 and its column block J needs only k >= j0 - 1 and, for rows
//     below i1, k <= i1; T = Z G needs k >= j0 - 2; dH = T Z^T is dense.
//     About n^3/3 + n^3 + 2 n^3 flops, plus n^3/3 for each vector set.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/schur_gb300.h"
#include "common.cuh"
#include "gemm.cuh"
#include "host.h"

#define ADJ_WARPS 8          // warps (vector blocks) per thread block
#define ADJ_NMAX 1024        // largest order of the per-warp path (its shared-memory rows)
#define ADJ_BLOCKED_MIN 1025 // single matrices of this order or more: blocked vectors, any order
#define ADJ_CH 512           // row chunk of the G = P X^T tasks

struct AdjDesc {
  const double* S;
  const double* Z;
  const double* wr;
  const double* wi;
  const double* gwr;
  const double* gwi;
  double* dH;
  double* ws;         // 5 n^2 doubles: XR, XI, P, Q, T (each n x n, ld n)
  long long lds, ldz, lddh;
  int n;
  int item0;          // first global item (= eigenvalue index) of this matrix
};

// complex helpers (pairs of doubles)
struct cplx {
  double r, i;
};
__device__ __forceinline__ cplx cmul(cplx a, cplx b) { return {fma(a.r, b.r, -a.i * b.i), fma(a.r, b.i, a.i * b.r)}; }
__device__ __forceinline__ cplx cdiv(cplx a, cplx b, double smin2) {
  double d = fma(b.r, b.r, b.i * b.i);
  if (d < smin2) d = smin2;  // perturbation of a (nearly) repeated eigenvalue
  double rd = fast_rcp(d);
  return {fma(a.r, b.r, a.i * b.i) * rd, fma(a.i, b.r, -a.r * b.i) * rd};
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_absmax(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Solve (B - lam I) x = r for the 1x1 / 2x2 real block B (transposed when
// trans), complex lam and r.
__device__ inline void block_solve(int sz, const double* B, bool trans, cplx lam, const cplx* r, cplx* x,
                                   double smin2) {
  if (sz == 1) {
    x[0] = cdiv(r[0], cplx{B[0] - lam.r, -lam.i}, smin2);
    return;
  }
  // B column-major 2x2: B[0]=b00, B[1]=b10, B[2]=b01, B[3]=b11
  double b00 = B[0], b10 = trans ? B[2] : B[1], b01 = trans ? B[1] : B[2], b11 = B[3];
  cplx m00{b00 - lam.r, -lam.i}, m11{b11 - lam.r, -lam.i};
  cplx det = cmul(m00, m11);
  det.r -= b01 * b10;
  cplx n0 = cmul(m11, r[0]);
  n0.r -= b01 * r[1].r;
  n0.i -= b01 * r[1].i;
  cplx n1 = cmul(m00, r[1]);
  n1.r -= b10 * r[0].r;
  n1.i -= b10 * r[0].i;
  x[0] = cdiv(n0, det, smin2);
  x[1] = cdiv(n1, det, smin2);
}

// ---------------------------------------------------------------------------
// One warp per eigenvalue index k (global item); the warp of the second row
// of a 2x2 block writes zero columns.  Per-warp shared buffer of 2 n doubles.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(32 * ADJ_WARPS) k_adj_vectors(const AdjDesc* __restrict__ descs, int ndesc,
                                                               int nitems, int nst) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int item = blockIdx.x * ADJ_WARPS + warp;
  if (item >= nitems) return;
  int b = 0;
  {
    int lo = 0, hi = ndesc - 1;  // last descriptor with item0 <= item
    while (lo < hi) {
      int mid = (lo + hi + 1) >> 1;
      if (descs[mid].item0 <= item) lo = mid; else hi = mid - 1;
    }
    b = lo;
  }
  const AdjDesc& d = descs[b];
  const int n = d.n;
  const int k = item - d.item0;
  if (k < 0 || k >= n) return;
  Mat S{const_cast<double*>(d.S), d.lds};
  const long long nn = (long long)n * n;
  double* XR = d.ws;
  double* XI = XR + nn;
  double* PP = XI + nn;
  double* QQ = PP + nn;
  double* xr = smem + (size_t)warp * 2 * nst;
  double* xi = xr + nst;
  const bool second = (k > 0 && S(k, k - 1) != 0.0);
  if (second) {
    for (int r = lane; r < n; r += 32) {
      XR[r + (long long)k * n] = 0.0;
      XI[r + (long long)k * n] = 0.0;
      PP[r + (long long)k * n] = 0.0;
      QQ[r + (long long)k * n] = 0.0;
    }
    return;
  }
  const int sz = (k + 1 < n && S(k + 1, k) != 0.0) ? 2 : 1;
  const cplx lam{d.wr[k], (sz == 2) ? d.wi[k] : 0.0};
  // smallest pivot: u * max |S_jj| (perturbation of repeated eigenvalues)
  double smax = 0.0;
  for (int r = lane; r < n; r += 32) smax = fmax(smax, fabs(S(r, r)));
  smax = warp_absmax(smax);
  double smin = fmax(SCHUR_U * smax, 1e-290);
  double smin2 = smin * smin;
  double Bk[4] = {S(k, k), (sz == 2) ? S(k + 1, k) : 0.0, (sz == 2) ? S(k, k + 1) : 0.0,
                  (sz == 2) ? S(k + 1, k + 1) : 0.0};
  // ---- right vector: block part, then back substitution upward
  for (int r = lane; r < n; r += 32) {
    xr[r] = 0.0;
    xi[r] = 0.0;
  }
  __syncwarp();
  cplx xb[2];
  if (sz == 1) {
    xb[0] = {1.0, 0.0};
  } else {
    double a = Bk[0], bb = Bk[2], c = Bk[1], dd = Bk[3];
    cplx u0{bb, 0.0}, u1{lam.r - a, lam.i};
    if (fabs(u0.r) + fabs(u1.r) + fabs(u1.i) == 0.0) {
      u0 = {lam.r - dd, lam.i};
      u1 = {c, 0.0};
    }
    xb[0] = u0;
    xb[1] = u1;
  }
  // rhs rows < k from the block's columns
  for (int t = 0; t < sz; ++t) {
    const double* col = &S(0, k + t);
    for (int r = lane; r < k; r += 32) {
      xr[r] = fma(-col[r], xb[t].r, xr[r]);
      xi[r] = fma(-col[r], xb[t].i, xi[r]);
    }
  }
  if (lane == 0) {
    for (int t = 0; t < sz; ++t) {
      xr[k + t] = xb[t].r;
      xi[k + t] = xb[t].i;
    }
  }
  __syncwarp();
  int j = k - 1;
  while (j >= 0) {
    int bs = (j >= 1 && S(j, j - 1) != 0.0) ? 2 : 1;
    int j0 = j - bs + 1;
    cplx xs[2];
    if (lane == 0) {
      double B[4] = {S(j0, j0), (bs == 2) ? S(j0 + 1, j0) : 0.0, (bs == 2) ? S(j0, j0 + 1) : 0.0,
                     (bs == 2) ? S(j0 + 1, j0 + 1) : 0.0};
      cplx rr[2] = {{xr[j0], xi[j0]}, {(bs == 2) ? xr[j0 + 1] : 0.0, (bs == 2) ? xi[j0 + 1] : 0.0}};
      block_solve(bs, B, false, lam, rr, xs, smin2);
      for (int t = 0; t < bs; ++t) {
        xr[j0 + t] = xs[t].r;
        xi[j0 + t] = xs[t].i;
      }
    }
    __syncwarp();
    for (int t = 0; t < bs; ++t) {
      double vr = xr[j0 + t], vi = xi[j0 + t];
      const double* col = &S(0, j0 + t);
      for (int r = lane; r < j0; r += 32) {
        xr[r] = fma(-col[r], vr, xr[r]);
        xi[r] = fma(-col[r], vi, xi[r]);
      }
    }
    __syncwarp();
    j = j0 - 1;
  }
  // normalise by max |x| and store
  double mx = 0.0;
  for (int r = lane; r < k + sz; r += 32) mx = fmax(mx, fmax(fabs(xr[r]), fabs(xi[r])));
  mx = warp_absmax(mx);
  double rs = (mx > 0.0) ? fast_rcp(mx) : 1.0;
  for (int r = lane; r < n; r += 32) {
    bool in = r < k + sz;
    XR[r + (long long)k * n] = in ? xr[r] * rs : 0.0;
    XI[r + (long long)k * n] = in ? xi[r] * rs : 0.0;
  }
  cplx xbs[2] = {{xr[k] * rs, xi[k] * rs}, {(sz == 2) ? xr[k + 1] * rs : 0.0, (sz == 2) ? xi[k + 1] * rs : 0.0}};
  __syncwarp();
  // ---- left vector (S^T w = lam w): block part, forward substitution
  for (int r = lane; r < n; r += 32) {
    xr[r] = 0.0;
    xi[r] = 0.0;
  }
  __syncwarp();
  cplx wb[2];
  if (sz == 1) {
    wb[0] = {1.0, 0.0};
  } else {
    double a = Bk[0], bb = Bk[2], c = Bk[1], dd = Bk[3];
    cplx u0{c, 0.0}, u1{lam.r - a, lam.i};
    if (fabs(u0.r) + fabs(u1.r) + fabs(u1.i) == 0.0) {
      u0 = {lam.r - dd, lam.i};
      u1 = {bb, 0.0};
    }
    wb[0] = u0;
    wb[1] = u1;
  }
  if (lane == 0)
    for (int t = 0; t < sz; ++t) {
      xr[k + t] = wb[t].r;
      xi[k + t] = wb[t].i;
    }
  __syncwarp();
  j = k + sz;
  while (j < n) {
    int bs = (j + 1 < n && S(j + 1, j) != 0.0) ? 2 : 1;
    cplx rr[2];
    for (int t = 0; t < bs; ++t) {
      const double* col = &S(0, j + t);
      double sr = 0.0, si = 0.0;
      for (int r = k + lane; r < j; r += 32) {
        sr = fma(col[r], xr[r], sr);
        si = fma(col[r], xi[r], si);
      }
      rr[t] = {-warp_sum(sr), -warp_sum(si)};
    }
    if (lane == 0) {
      double B[4] = {S(j, j), (bs == 2) ? S(j + 1, j) : 0.0, (bs == 2) ? S(j, j + 1) : 0.0,
                     (bs == 2) ? S(j + 1, j + 1) : 0.0};
      cplx ws2[2];
      block_solve(bs, B, true, lam, rr, ws2, smin2);
      for (int t = 0; t < bs; ++t) {
        xr[j + t] = ws2[t].r;
        xi[j + t] = ws2[t].i;
      }
    }
    __syncwarp();
    j += bs;
  }
  mx = 0.0;
  for (int r = k + lane; r < n; r += 32) mx = fmax(mx, fmax(fabs(xr[r]), fabs(xi[r])));
  mx = warp_absmax(mx);
  rs = (mx > 0.0) ? fast_rcp(mx) : 1.0;
  // c = w_b^T x_b (block rows only); e = g_r / c (real) or
  // (conj(g_k) + g_{k+1}) / c (pair)
  cplx c{0.0, 0.0};
  for (int t = 0; t < sz; ++t) {
    cplx wv{xr[k + t] * rs, xi[k + t] * rs};
    cplx p = cmul(wv, xbs[t]);
    c.r += p.r;
    c.i += p.i;
  }
  cplx num;
  if (sz == 1) {
    num = {d.gwr[k], 0.0};
  } else {
    num = {d.gwr[k] + d.gwr[k + 1], -d.gwi[k] + d.gwi[k + 1]};
  }
  cplx e = cdiv(num, c, 1e-300);
  for (int r = lane; r < n; r += 32) {
    bool in = r >= k;
    cplx wv{in ? xr[r] * rs : 0.0, in ? xi[r] * rs : 0.0};
    cplx ew = cmul(e, wv);
    PP[r + (long long)k * n] = ew.r;
    QQ[r + (long long)k * n] = ew.i;
  }
}

// ---------------------------------------------------------------------------
// Blocked path, step 1: S' = R S^T R, i.e. S'(i, j) = S(n-1-j, n-1-i), by
// 32 x 32 tiles through shared memory (both sides coalesced), and
// wr' = R wr, wi' = -R wi.  Grid (ceil(n/32), ceil(n/32)), 256 threads.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_adj_revT(const double* __restrict__ S, long long lds, int n,
                                                 double* __restrict__ Sp, const double* __restrict__ wr,
                                                 const double* __restrict__ wi, double* __restrict__ wrp,
                                                 double* __restrict__ wip) {
  __shared__ double tile[32][33];
  const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;   // tile of S': rows i0.., columns j0..
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int r = ty; r < 32; r += 8) {                       // tile[r][tx] = S'(i0 + r, j0 + tx)
    const int i = i0 + r, j = j0 + tx;
    tile[r][tx] = (i < n && j < n) ? S[(n - 1 - j) + (long long)(n - 1 - i) * lds] : 0.0;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int i = i0 + tx, j = j0 + r;
    if (i < n && j < n) Sp[i + (long long)j * n] = tile[tx][r];
  }
  if (blockIdx.y == 0 && threadIdx.x < 32) {
    const int i = i0 + threadIdx.x;
    if (i < n) {
      const double w = wi[n - 1 - i];
      wrp[i] = wr[n - 1 - i];
      wip[i] = (w == 0.0) ? 0.0 : -w;
    }
  }
}

// ---------------------------------------------------------------------------
// Blocked path, step 2: one warp per eigenvalue index k (the first of a
// pair; the second's warp returns).  X, Wp (= the right eigenvectors of S')
// and P are n x n with leading dimension n.  c = w^T x over the block rows
// (the only rows where both are nonzero), e = g / c (real) or
// (conj(g_k) + g_{k+1}) / c (pair); P column k = Re(e w), column k+1 =
// -Im(e w), so that P X^T = Re(e w x^T).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_adj_combine(const double* __restrict__ X, const double* __restrict__ Wp,
                                                    const double* __restrict__ wi, const double* __restrict__ gwr,
                                                    const double* __restrict__ gwi, double* __restrict__ P, int n) {
  const int lane = threadIdx.x & 31;
  const int k = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (k >= n) return;
  const double wk = wi[k];
  if (wk < 0.0) return;
  const bool pair = wk > 0.0 && k + 1 < n;
  const long long ln = n;
  cplx c{0.0, 0.0}, num;
  if (!pair) {
    c.r = X[k + k * ln] * Wp[(n - 1 - k) + (n - 1 - k) * ln];
    num = {gwr[k], 0.0};
  } else {
    for (int t = 0; t < 2; ++t) {
      const int r = k + t;
      const cplx x{X[r + k * ln], X[r + (k + 1) * ln]};
      const cplx w{Wp[(n - 1 - r) + (n - 2 - k) * ln], Wp[(n - 1 - r) + (n - 1 - k) * ln]};
      const cplx p = cmul(w, x);
      c.r += p.r;
      c.i += p.i;
    }
    num = {gwr[k] + gwr[k + 1], gwi[k + 1] - gwi[k]};
  }
  const cplx e = cdiv(num, c, 1e-300);
  double* p0 = P + k * ln;
  if (!pair) {
    const double* wc = Wp + (n - 1 - k) * ln;
    for (int r = lane; r < n; r += 32) p0[r] = e.r * wc[n - 1 - r];
  } else {
    const double* wre = Wp + (n - 2 - k) * ln;
    const double* wim = Wp + (n - 1 - k) * ln;
    double* p1 = p0 + ln;
    for (int r = lane; r < n; r += 32) {
      const cplx ew = cmul(e, cplx{wre[n - 1 - r], wim[n - 1 - r]});
      p0[r] = ew.r;
      p1[r] = -ew.i;
    }
  }
}

// ===========================================================================
// Host side
// ===========================================================================
namespace {

struct AdjMatrix {
  int n;
  const double *S, *Z, *wr, *wi, *gwr, *gwi;
  double* dH;
  int lds, ldz, lddh;
};

using schur::ck_at;
using schur::CudaError;

// k_adj_vectors' shared-memory limit is raised to the device maximum once per
// device (never lowered), so that concurrent calls on other host threads never
// see a limit below the size they launch with.
static std::mutex g_adj_mu;
static bool g_adj_done[64] = {false};

static void adj_raise_limit() {
  int dev = 0;
  ck_at(cudaGetDevice(&dev), __LINE__);
  if (dev < 0 || dev >= 64) throw CudaError{cudaErrorInvalidDevice};
  std::lock_guard<std::mutex> lock(g_adj_mu);
  if (g_adj_done[dev]) return;
  int optin = 0;
  ck_at(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev), __LINE__);
  cudaFuncAttributes fa;
  ck_at(cudaFuncGetAttributes(&fa, k_adj_vectors), __LINE__);
  ck_at(cudaFuncSetAttribute(k_adj_vectors, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin - (int)fa.sharedSizeBytes), __LINE__);
  g_adj_done[dev] = true;
}

size_t warp_path_bytes(const std::vector<int>& ns) {
  size_t ws_doubles = 0;
  for (int n : ns) ws_doubles += 5 * (size_t)n * n;
  const size_t nb = ns.size();
  size_t desc_bytes = (nb * sizeof(AdjDesc) + 255) & ~(size_t)255;
  size_t task_bytes = ((size_t)4 * nb * sizeof(GemmTask) + 255) & ~(size_t)255;
  return ws_doubles * sizeof(double) + desc_bytes + task_bytes;
}

int run_backward(const std::vector<AdjMatrix>& ms, const schur_opts* opts) {
  schur_opts o;
  schur::read_opts(opts, &o);
  cudaStream_t st = (cudaStream_t)o.stream;
  const int nb = (int)ms.size();
  size_t ws_doubles = 0;
  int nmax = 1, items = 0;
  for (auto& m : ms) {
    ws_doubles += 5 * (size_t)m.n * m.n;
    nmax = std::max(nmax, m.n);
    items += m.n;
  }
  size_t desc_bytes = ((size_t)nb * sizeof(AdjDesc) + 255) & ~(size_t)255;
  std::vector<int> ns;
  for (auto& m : ms) ns.push_back(m.n);
  const size_t need = warp_path_bytes(ns);
  char* mem = nullptr;
  bool own = false;
  int rc = SCHUR_OK;
  if (o.workspace && schur::workspace_unusable(o, need)) return SCHUR_ERR_WORKSPACE;
  try {
    schur::init_kernel_attributes();
    adj_raise_limit();
    if (o.workspace) {
      mem = (char*)o.workspace;
    } else {
      if (cudaMalloc((void**)&mem, need) != cudaSuccess) {
        cudaGetLastError();
        return SCHUR_ERR_NOMEM;
      }
      own = true;
    }
    double* wsbase = (double*)mem;
    std::vector<AdjDesc> hd(nb);
    size_t off = 0;
    int item0 = 0;
    for (int b = 0; b < nb; ++b) {
      const AdjMatrix& m = ms[b];
      hd[b] = AdjDesc{m.S, m.Z, m.wr, m.wi, m.gwr, m.gwi, m.dH, wsbase + off, m.lds, m.ldz, m.lddh, m.n, item0};
      off += 5 * (size_t)m.n * m.n;
      item0 += m.n;
    }
    AdjDesc* ddesc = (AdjDesc*)(mem + ws_doubles * sizeof(double));
    GemmTask* dtask = (GemmTask*)((char*)ddesc + desc_bytes);
    ck_at(cudaMemcpyAsync(ddesc, hd.data(), nb * sizeof(AdjDesc), cudaMemcpyHostToDevice, st), __LINE__);
    size_t smem = (size_t)ADJ_WARPS * 2 * nmax * sizeof(double);
    k_adj_vectors<<<(items + ADJ_WARPS - 1) / ADJ_WARPS, 32 * ADJ_WARPS, smem, st>>>(ddesc, nb, items, nmax);
    ck_at(cudaGetLastError(), __LINE__);
    ++schur::g_stats.kernel_launches;
    // three GEMM phases: G = P XR^T - Q XI^T (into T), W = Z G (into P),
    // dH = W Z^T
    std::vector<GemmTask> tasks;
    auto add = [&](const double* A, long long lda, const double* B, long long ldb, double* C, long long ldc, int M,
                   int N, int K, int transB, double alpha, double beta) {
      GemmTask t;
      memset(&t, 0, sizeof(t));
      t.A = A; t.B = B; t.C = C; t.lda = lda; t.ldb = ldb; t.ldc = ldc;
      t.M = M; t.N = N; t.K = K; t.transB = transB; t.alpha = alpha; t.beta = beta;
      tasks.push_back(t);
    };
    auto launch = [&]() {
      int tile = 0;
      for (auto& t : tasks) {
        t.tiles_n = (t.N + 63) / 64;
        t.ntile = ((t.M + 63) / 64) * t.tiles_n;
        t.tile0 = tile;
        tile += t.ntile;
      }
      ck_at(cudaMemcpyAsync(dtask, tasks.data(), tasks.size() * sizeof(GemmTask), cudaMemcpyHostToDevice, st),
            __LINE__);
      k_gemm<<<std::min(tile, 4 * schur::num_sms()), 256, 0, st>>>(dtask, (int)tasks.size(), tile);
      ck_at(cudaGetLastError(), __LINE__);
      ++schur::g_stats.kernel_launches;
      // the task array is reused by the next phase: wait for this one
      ck_at(cudaStreamSynchronize(st), __LINE__);
      tasks.clear();
    };
    for (int b = 0; b < nb; ++b) {
      const AdjDesc& d = hd[b];
      long long nn = (long long)d.n * d.n;
      double *XR = d.ws, *XI = XR + nn, *PP = XI + nn, *QQ = PP + nn, *TT = QQ + nn;
      add(PP, d.n, XR, d.n, TT, d.n, d.n, d.n, d.n, 1, 1.0, 0.0);
    }
    launch();
    for (int b = 0; b < nb; ++b) {
      const AdjDesc& d = hd[b];
      long long nn = (long long)d.n * d.n;
      double *XR = d.ws, *XI = XR + nn, *PP = XI + nn, *QQ = PP + nn, *TT = QQ + nn;
      add(QQ, d.n, XI, d.n, TT, d.n, d.n, d.n, d.n, 1, -1.0, 1.0);
    }
    launch();
    for (int b = 0; b < nb; ++b) {
      const AdjDesc& d = hd[b];
      long long nn = (long long)d.n * d.n;
      double *PP = d.ws + 2 * nn, *TT = d.ws + 4 * nn;
      add(d.Z, d.ldz, TT, d.n, PP, d.n, d.n, d.n, d.n, 0, 1.0, 0.0);
    }
    launch();
    for (int b = 0; b < nb; ++b) {
      const AdjDesc& d = hd[b];
      long long nn = (long long)d.n * d.n;
      double* PP = d.ws + 2 * nn;
      add(PP, d.n, d.Z, d.ldz, d.dH, d.lddh, d.n, d.n, d.n, 1, 1.0, 0.0);
    }
    launch();
  } catch (const CudaError&) {
    rc = SCHUR_ERR_CUDA;
  }
  if (own && mem) cudaFree(mem);
  return rc;
}

// ----------------------------------------------------------- blocked path
size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

// The GEMM tasks of the blocked path (pointers may be null when only the
// count is wanted): G = P X^T by (64-column block, ADJ_CH-row chunk), then
// T = Z G by column block, then dH = T Z^T.  first[0..2] = index of each
// group's first task; returns the flops.
double blocked_tasks(int n, const double* P, const double* X, double* G, const double* Z, long long ldz, double* T,
                     double* dH, long long lddh, std::vector<GemmTask>* tasks, int first[3]) {
  double flops = 0.0;
  const long long ln = n;
  auto add = [&](const double* A, long long lda, const double* B, long long ldb, int transB, double* C,
                 long long ldc, int M, int N, int K) {
    GemmTask t;
    memset(&t, 0, sizeof(t));
    t.A = A; t.B = B; t.C = C; t.lda = lda; t.ldb = ldb; t.ldc = ldc;
    t.M = M; t.N = N; t.K = K; t.transB = transB; t.alpha = 1.0; t.beta = 0.0;
    t.tiles_n = (N + 63) / 64;
    t.ntile = ((M + 63) / 64) * t.tiles_n;
    tasks->push_back(t);
    flops += 2.0 * M * (double)N * K;
  };
  first[0] = (int)tasks->size();
  for (int j0 = 0; j0 < n; j0 += 64) {
    const int j1 = std::min(n, j0 + 64);
    const int k0 = std::max(0, j0 - 1);
    for (int i0 = std::max(0, j0 - 2); i0 < n; i0 += ADJ_CH) {
      const int i1 = std::min(n, i0 + ADJ_CH);
      const int k1 = std::min(n, i1 + 1);
      add(P ? P + i0 + k0 * ln : nullptr, ln, X ? X + j0 + k0 * ln : nullptr, ln, 1, G ? G + i0 + j0 * ln : nullptr,
          ln, i1 - i0, j1 - j0, k1 - k0);
    }
  }
  first[1] = (int)tasks->size();
  for (int j0 = 0; j0 < n; j0 += 64) {
    const int j1 = std::min(n, j0 + 64);
    const int k0 = std::max(0, j0 - 2);
    add(Z ? Z + k0 * ldz : nullptr, ldz, G ? G + k0 + j0 * ln : nullptr, ln, 0, T ? T + j0 * ln : nullptr, ln, n,
        j1 - j0, n - k0);
  }
  first[2] = (int)tasks->size();
  add(T, ln, Z, ldz, 1, dH, lddh, n, n, n);
  return flops;
}

struct BlockedLayout {
  size_t buf0, buf1, buf2, wrp, wip, ev, task, total;
  int ntask;
};

BlockedLayout blocked_layout(int n) {
  BlockedLayout L;
  const size_t nn = al256((size_t)n * n * sizeof(double));
  const size_t vec = al256((size_t)n * sizeof(double));
  std::vector<GemmTask> tk;
  int first[3];
  blocked_tasks(n, nullptr, nullptr, nullptr, nullptr, n, nullptr, nullptr, n, &tk, first);
  L.ntask = (int)tk.size();
  L.buf0 = 0;
  L.buf1 = nn;
  L.buf2 = 2 * nn;
  L.wrp = 3 * nn;
  L.wip = L.wrp + vec;
  L.ev = L.wip + vec;
  L.task = L.ev + al256(schur::eigvec_workspace(n, false));
  L.total = L.task + al256((size_t)L.ntask * sizeof(GemmTask));
  return L;
}

int run_backward_blocked(const AdjMatrix& m, const schur_opts* opts) {
  schur_opts o;
  schur::read_opts(opts, &o);
  cudaStream_t st = (cudaStream_t)o.stream;
  const int n = m.n;
  const BlockedLayout L = blocked_layout(n);
  char* mem = nullptr;
  bool own = false;
  if (o.workspace) {
    if (schur::workspace_unusable(o, L.total)) return SCHUR_ERR_WORKSPACE;
    mem = (char*)o.workspace;
  } else {
    if (cudaMalloc((void**)&mem, L.total) != cudaSuccess) {
      cudaGetLastError();
      return SCHUR_ERR_NOMEM;
    }
    own = true;
  }
  int rc = SCHUR_OK;
  try {
    schur::init_kernel_attributes();
    double* b0 = (double*)(mem + L.buf0);   // S', then X
    double* b1 = (double*)(mem + L.buf1);   // W' (vectors of S'), then G
    double* b2 = (double*)(mem + L.buf2);   // P, then T
    double* wrp = (double*)(mem + L.wrp);
    double* wip = (double*)(mem + L.wip);
    GemmTask* dtask = (GemmTask*)(mem + L.task);
    long long launches = 0;
    double flops = 0.0;
    std::vector<double> hwi(n), hwip(n);
    ck_at(cudaMemcpyAsync(hwi.data(), m.wi, n * sizeof(double), cudaMemcpyDeviceToHost, st), __LINE__);
    ck_at(cudaStreamSynchronize(st), __LINE__);
    for (int i = 0; i < n; ++i) hwip[i] = (hwi[n - 1 - i] == 0.0) ? 0.0 : -hwi[n - 1 - i];
    const int nt = (n + 31) / 32;
    k_adj_revT<<<dim3(nt, nt), 256, 0, st>>>(m.S, m.lds, n, b0, m.wr, m.wi, wrp, wip);
    ck_at(cudaGetLastError(), __LINE__);
    ++launches;
    schur::eigvec_run(n, b0, n, nullptr, 0, wrp, wip, hwip.data(), b1, n, st, mem + L.ev, &launches, &flops);
    schur::eigvec_run(n, m.S, m.lds, nullptr, 0, m.wr, m.wi, hwi.data(), b0, n, st, mem + L.ev, &launches, &flops);
    k_adj_combine<<<(n + 7) / 8, 256, 0, st>>>(b0, b1, m.wi, m.gwr, m.gwi, b2, n);
    ck_at(cudaGetLastError(), __LINE__);
    ++launches;
    std::vector<GemmTask> tasks;
    int first[3];
    // T overwrites P, which the G launch has finished reading
    flops += blocked_tasks(n, b2, b0, b1, m.Z, m.ldz, b2, m.dH, m.lddh, &tasks, first);
    if ((int)tasks.size() != L.ntask) throw CudaError{cudaErrorInvalidValue};
    // one launch per group (G, then T, then dH: each reads the previous
    // one's output); tile indices count from 0 within a group
    const int bounds[4] = {first[0], first[1], first[2], (int)tasks.size()};
    int ntile[3];
    for (int g = 0; g < 3; ++g) {
      int tile = 0;
      for (int i = bounds[g]; i < bounds[g + 1]; ++i) {
        tasks[i].tile0 = tile;
        tile += tasks[i].ntile;
      }
      ntile[g] = tile;
    }
    ck_at(cudaMemcpyAsync(dtask, tasks.data(), tasks.size() * sizeof(GemmTask), cudaMemcpyHostToDevice, st),
          __LINE__);
    ck_at(cudaMemsetAsync(b1, 0, (size_t)n * n * sizeof(double), st), __LINE__);   // G's known zeros
    const int nsm = schur::num_sms();
    for (int g = 0; g < 3; ++g) {
      k_gemm<<<std::min(ntile[g], 4 * nsm), 256, 0, st>>>(dtask + bounds[g], bounds[g + 1] - bounds[g], ntile[g]);
      ck_at(cudaGetLastError(), __LINE__);
      ++launches;
    }
    ck_at(cudaStreamSynchronize(st), __LINE__);
    schur::g_stats.kernel_launches = launches;
    schur::g_stats.flops = flops;
  } catch (const CudaError&) {
    rc = SCHUR_ERR_CUDA;
  }
  if (own && mem) cudaFree(mem);
  return rc;
}

}  // namespace

extern "C" int schur_eig_backward_workspace(int n, size_t* bytes) {
  if (n < 0) return -1;
  if (!bytes) return -2;
  *bytes = (n >= ADJ_BLOCKED_MIN) ? blocked_layout(n).total : warp_path_bytes({std::max(n, 1)});
  return SCHUR_OK;
}

extern "C" int schur_eig_backward(int n, const double* S, int lds, const double* Z, int ldz, const double* wr,
                                  const double* wi, const double* gwr, const double* gwi, double* dH, int lddh,
                                  const schur_opts* opts) {
  if (n < 0) return -1;
  if (n == 0) return SCHUR_OK;
  if (!S) return -2;
  if (lds < n) return -3;
  if (!Z) return -4;
  if (ldz < n) return -5;
  if (!wr) return -6;
  if (!wi) return -7;
  if (!gwr) return -8;
  if (!gwi) return -9;
  if (!dH) return -10;
  if (lddh < n) return -11;
  memset(&schur::g_stats, 0, sizeof(schur::g_stats));
  const AdjMatrix m{n, S, Z, wr, wi, gwr, gwi, dH, lds, ldz, lddh};
  if (n >= ADJ_BLOCKED_MIN) return run_backward_blocked(m, opts);
  return run_backward(std::vector<AdjMatrix>{m}, opts);
}

extern "C" int schur_eig_backward_batched(int batch, const int* n, double* const* S, const int* lds, double* const* Z,
                                          const int* ldz, double* const* wr, double* const* wi, double* const* gwr,
                                          double* const* gwi, double* const* dH, const int* lddh,
                                          const schur_opts* opts) {
  if (batch < 0) return -1;
  if (batch == 0) return SCHUR_OK;
  if (!n) return -2;
  if (!S) return -3;
  if (!lds) return -4;
  if (!Z) return -5;
  if (!ldz) return -6;
  if (!wr) return -7;
  if (!wi) return -8;
  if (!gwr) return -9;
  if (!gwi) return -10;
  if (!dH) return -11;
  if (!lddh) return -12;
  std::vector<AdjMatrix> ms(batch);
  for (int b = 0; b < batch; ++b) {
    if (n[b] < 1 || n[b] > ADJ_NMAX) return -2;
    if (!S[b]) return -3;
    if (lds[b] < n[b]) return -4;
    if (!Z[b]) return -5;
    if (ldz[b] < n[b]) return -6;
    if (!wr[b]) return -7;
    if (!wi[b]) return -8;
    if (!gwr[b]) return -9;
    if (!gwi[b]) return -10;
    if (!dH[b]) return -11;
    if (lddh[b] < n[b]) return -12;
    ms[b] = AdjMatrix{n[b], S[b], Z[b], wr[b], wi[b], gwr[b], gwi[b], dH[b], lds[b], ldz[b], lddh[b]};
  }
  return run_backward(ms, opts);
}
