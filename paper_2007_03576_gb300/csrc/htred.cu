// htred.cu -- Hessenberg-triangular reduction of a matrix pair on the GPU:
// the first phase of the generalized case (Sec. 1 remark: (A, B) -> (H, R)
// with H upper Hessenberg and R upper triangular, A = Q H Z^T, B = Q R Z^T,
// before the QZ iteration of qz.cu).
//
// The classical two-stage method (Golub & Van Loan, Alg. 7.7.1):
//   1. a Householder QR of B (reflectors with v_0 = 1, LAPACK's sign
//      convention) applied to A from the left and accumulated into Q;
//   2. for each column j of A, bottom to top, a left Givens rotation of rows
//      (i - 1, i) zeroes A[i, j]; it leaves a fill-in R[i, i - 1], which a
//      right rotation of columns (i - 1, i) removes (applied to A, R and Z).
// The order of the transformations is the oracle's (oracle/qz.py,
// hessenberg_triangular), so both give the same pair up to rounding.
//
// One thread block per pair, the pair in global memory (like the QZ kernel):
//   * stage 1: the column norm is a block reduction (scaled by the largest
//     entry, so no overflow or underflow), v overwrites B's column below the
//     diagonal, then one warp per column applies the reflector to B and A and
//     one thread per row to Q;
//   * stage 2: the rotation pair of a step comes from five entries
//     (A[i-1, j], A[i, j], R[i-1, i-1], R[i-1, i], R[i, i]); thread 0 builds
//     the next step's pair while the other threads apply the current one in
//     one pass: the left rotation to rows i-1, i of A and R outside columns
//     i-1, i, the right one to columns i-1, i of A, R and Z outside rows
//     i-1, i (and outside R's row i-2), Q's columns by the left one.  Thread 0
//     applies both to the 2x2 blocks of A and R (left first) and the right
//     one to R's row i-2, which gives it every input of the next pair; one
//     barrier per step.
// About n^2 / 2 rotation steps of O(n) work each: a latency-bound kernel
// meant for batches of small and medium pairs (one SM per pair).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/schur_gb300.h"
#include "host.h"

namespace {

constexpr int HT_THREADS = 256;        // pairs of order < HT_BIG_N
constexpr int HT_THREADS_BIG = 1024;
constexpr int HT_BIG_N = 384;

struct HtDesc {
  double *A, *B, *Q, *Z;
  long long lda, ldb, ldq, ldz;
  int n, pad;
};

struct GMat {
  double* p;
  long long ld;
  __device__ double& operator()(int r, int c) const { return p[r + c * ld]; }
};

// block-wide max / sum (every thread gets the result); red has NT / 32 slots
template <int NT, bool MAX>
__device__ double block_reduce(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) {
    const double w = __shfl_xor_sync(0xffffffffu, v, o);
    v = MAX ? fmax(v, w) : v + w;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();   // red may still be read from the previous reduction
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < NT / 32; ++w) t = MAX ? fmax(t, red[w]) : t + red[w];
  return t;
}

// (c, s) of a left rotation of rows (i, k) that zeroes b: (a, b) -> (r, 0)
__device__ __forceinline__ void ht_rot_second(double a, double b, double& c, double& s) {
  if (b == 0.0) {
    c = 1.0;
    s = 0.0;
    return;
  }
  const double r = hypot(a, b);
  c = a / r;
  s = b / r;
}

// (c, s) of a right rotation of columns (i, k) with c a + s b = 0
__device__ __forceinline__ void ht_rot_first(double a, double b, double& c, double& s) {
  if (a == 0.0) {
    c = 1.0;
    s = 0.0;
    return;
  }
  const double r = hypot(a, b);
  c = b / r;
  s = -a / r;
}

// The rotation pair of one step from A[i-1, j] = a, A[i, j] = b and R's
// block (r11, r12; 0, r22): the left rotation zeroing b, then the right one
// zeroing the fill-in f21 it leaves in R.  out = (c1, s1, c2, s2, f21, f22).
__device__ __forceinline__ void ht_build_pair(double a, double b, double r11, double r12, double r22,
                                              double* out) {
  double c1, s1, c2, s2;
  ht_rot_second(a, b, c1, s1);
  const double f21 = -s1 * r11, f22 = fma(-s1, r12, c1 * r22);   // R[i, i-1], R[i, i] after the left rotation
  ht_rot_first(f21, f22, c2, s2);
  out[0] = c1;
  out[1] = s1;
  out[2] = c2;
  out[3] = s2;
  out[4] = f21;
  out[5] = f22;
}

template <int NT>
__device__ void ht_pair(const HtDesc& d, bool want_qz, int z_init, int* info_b, double* red,
                        double (*rotb)[8]) {
  const int n = d.n;
  const GMat A{d.A, d.lda}, B{d.B, d.ldb}, Q{d.Q, d.ldq}, Z{d.Z, d.ldz};
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = NT / 32;

  // non-finite input: nothing is changed
  {
    double bad = 0.0;
    for (long long e = tid; e < (long long)n * n; e += NT) {
      const int r = (int)(e % n), c = (int)(e / n);
      if (!isfinite(A(r, c)) || !isfinite(B(r, c))) bad = 1.0;
    }
    if (block_reduce<NT, true>(bad, red) != 0.0) {
      if (tid == 0) *info_b = SCHUR_ERR_NONFINITE;
      return;
    }
  }
  if (want_qz && z_init == 0) {
    for (long long e = tid; e < (long long)n * n; e += NT) {
      const int r = (int)(e % n), c = (int)(e / n);
      Q(r, c) = (r == c) ? 1.0 : 0.0;
      Z(r, c) = (r == c) ? 1.0 : 0.0;
    }
  }
  __syncthreads();

  // ---- stage 1: B = Q1 R (Householder), A <- Q1^T A, Q <- Q Q1
  for (int j = 0; j + 1 < n; ++j) {
    double m = 0.0;
    for (int r = j + 1 + tid; r < n; r += NT) m = fmax(m, fabs(B(r, j)));
    m = block_reduce<NT, true>(m, red);
    if (m == 0.0) continue;   // B[j+1:, j] is already zero: the identity
    const double rm = 1.0 / m;
    double q = 0.0;
    for (int r = j + 1 + tid; r < n; r += NT) {
      const double x = B(r, j) * rm;
      q = fma(x, x, q);
    }
    q = block_reduce<NT, false>(q, red);
    const double alpha = B(j, j);
    const double sigma = m * sqrt(q);
    const double beta = -copysign(hypot(alpha, sigma), alpha);
    const double tau = (beta - alpha) / beta;
    const double scal = 1.0 / (alpha - beta);
    __syncthreads();   // every thread has read the column before v overwrites it
    for (int r = j + 1 + tid; r < n; r += NT) B(r, j) *= scal;   // v below the diagonal, v_0 = 1
    __syncthreads();
    // one warp per column: B columns j+1.., A columns 0..
    for (int c = warp; c < 2 * n - j - 1; c += NW) {
      const GMat& M = (c < n - j - 1) ? B : A;
      const int col = (c < n - j - 1) ? j + 1 + c : c - (n - j - 1);
      double s = (lane == 0) ? M(j, col) : 0.0;
      for (int r = j + 1 + lane; r < n; r += 32) s = fma(B(r, j), M(r, col), s);
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      s *= tau;
      if (lane == 0) M(j, col) -= s;
      for (int r = j + 1 + lane; r < n; r += 32) M(r, col) = fma(-s, B(r, j), M(r, col));
    }
    if (want_qz) {
      // one thread per row of Q: Q[r, j:] <- Q[r, j:] (I - tau v v^T)
      for (int r = tid; r < n; r += NT) {
        double s = Q(r, j);
        for (int k = j + 1; k < n; ++k) s = fma(Q(r, k), B(k, j), s);
        s *= tau;
        Q(r, j) -= s;
        for (int k = j + 1; k < n; ++k) Q(r, k) = fma(-s, B(k, j), Q(r, k));
      }
    }
    __syncthreads();
    if (tid == 0) B(j, j) = beta;
    for (int r = j + 1 + tid; r < n; r += NT) B(r, j) = 0.0;
    __syncthreads();
  }

  // ---- stage 2: zero A below the subdiagonal, keep R triangular.  Thread 0
  // builds step i's rotation pair during step i + 1 (double-buffered in
  // shared memory), from values it carries or owns: A[i-1, j] (untouched
  // until step i), A[i, j] (the left rotation of step i + 1 applied to the
  // pair it carries), R[i-1, i-1] (untouched), R[i-1, i] (the right rotation
  // of step i + 1 on row i - 1, its own item) and R[i, i] (the 2x2 block of
  // step i + 1, its own item).  The other threads apply the current pair.
  for (int j = 0; j + 2 < n; ++j) {
    double aa = 0.0, bb = 0.0;   // thread 0: the (A[i-1, j], A[i, j]) the current pair was built from
    if (tid == 0) {
      const int i = n - 1;
      aa = A(i - 1, j);
      bb = A(i, j);
      ht_build_pair(aa, bb, B(i - 1, i - 1), B(i - 1, i), B(i, i), rotb[0]);
    }
    __syncthreads();
    int buf = 0;
    for (int i = n - 1; i >= j + 2; --i, buf ^= 1) {
      const double c1 = rotb[buf][0], s1 = rotb[buf][1], c2 = rotb[buf][2], s2 = rotb[buf][3];
      if (tid == 0) {
        // the 2x2 blocks on rows and columns (i-1, i): left rotation, then right
        const double a11 = A(i - 1, i - 1), a12 = A(i - 1, i), a21 = A(i, i - 1), a22 = A(i, i);
        const double t11 = fma(c1, a11, s1 * a21), t21 = fma(-s1, a11, c1 * a21);
        const double t12 = fma(c1, a12, s1 * a22), t22 = fma(-s1, a12, c1 * a22);
        A(i - 1, i - 1) = fma(c2, t11, s2 * t12);
        A(i - 1, i) = fma(-s2, t11, c2 * t12);
        A(i, i - 1) = fma(c2, t21, s2 * t22);
        A(i, i) = fma(-s2, t21, c2 * t22);
        // R: the left rotation gives (g11, g12; f21, f22), the right one zeroes f21
        const double r11 = B(i - 1, i - 1), r12 = B(i - 1, i), r22 = B(i, i);
        const double f21 = rotb[buf][4], f22 = rotb[buf][5];
        const double g11 = c1 * r11, g12 = fma(c1, r12, s1 * r22);
        const double n11 = fma(c2, g11, s2 * g12);
        B(i - 1, i - 1) = n11;
        B(i - 1, i) = fma(-s2, g11, c2 * g12);
        B(i, i - 1) = 0.0;
        B(i, i) = fma(-s2, f21, c2 * f22);
        // the right rotation on R's row i - 2
        const double x = B(i - 2, i - 1), y = B(i - 2, i);
        const double m12 = fma(c2, x, s2 * y);
        B(i - 2, i - 1) = m12;
        B(i - 2, i) = fma(-s2, x, c2 * y);
        if (i - 1 >= j + 2) {   // the next step's pair
          const double na = A(i - 2, j), nb = fma(c1, aa, s1 * bb);
          ht_build_pair(na, nb, B(i - 2, i - 2), m12, n11, rotb[buf ^ 1]);
          aa = na;
          bb = nb;
        }
      } else {
        // work items: [A left: columns j..n-1 except i-1, i] [R left: columns i+1..n-1]
        // [A right: rows except i-1, i] [R right: rows 0..i-3] [Q: rows] [Z: rows]
        const int nal = n - j - 2, nrl = n - i - 1, nar = n - 2, nrr = i - 2;
        const int nq = want_qz ? n : 0;
        const int total = nal + nrl + nar + nrr + 2 * nq;
        for (int t = tid - 1; t < total; t += NT - 1) {
          int u = t;
          if (u < nal) {
            const int c = (u < i - 1 - j) ? j + u : u + j + 2;   // skip columns i-1, i
            const double x = A(i - 1, c), y = A(i, c);
            A(i - 1, c) = fma(c1, x, s1 * y);
            A(i, c) = (c == j) ? 0.0 : fma(-s1, x, c1 * y);
            continue;
          }
          u -= nal;
          if (u < nrl) {
            const int c = i + 1 + u;
            const double x = B(i - 1, c), y = B(i, c);
            B(i - 1, c) = fma(c1, x, s1 * y);
            B(i, c) = fma(-s1, x, c1 * y);
            continue;
          }
          u -= nrl;
          if (u < nar) {
            const int r = (u < i - 1) ? u : u + 2;   // skip rows i-1, i
            const double x = A(r, i - 1), y = A(r, i);
            A(r, i - 1) = fma(c2, x, s2 * y);
            A(r, i) = fma(-s2, x, c2 * y);
            continue;
          }
          u -= nar;
          if (u < nrr) {
            const double x = B(u, i - 1), y = B(u, i);
            B(u, i - 1) = fma(c2, x, s2 * y);
            B(u, i) = fma(-s2, x, c2 * y);
            continue;
          }
          u -= nrr;
          if (u < nq) {
            const double x = Q(u, i - 1), y = Q(u, i);
            Q(u, i - 1) = fma(c1, x, s1 * y);
            Q(u, i) = fma(-s1, x, c1 * y);
            continue;
          }
          u -= nq;
          const double x = Z(u, i - 1), y = Z(u, i);
          Z(u, i - 1) = fma(c2, x, s2 * y);
          Z(u, i) = fma(-s2, x, c2 * y);
        }
      }
      __syncthreads();
    }
  }
  if (tid == 0) *info_b = 0;
}

template <int NT>
__global__ void __launch_bounds__(NT) k_ht(const HtDesc* __restrict__ descs, int nb, int want_qz, int z_init,
                                           int* __restrict__ info) {
  __shared__ double red[NT / 32];
  __shared__ double rotb[2][8];
  for (int b = blockIdx.x; b < nb; b += gridDim.x) {
    const HtDesc d = descs[b];
    ht_pair<NT>(d, want_qz != 0 && d.Q != nullptr, z_init, info + b, red, rotb);
    __syncthreads();
  }
}

struct HtPair {
  int n;
  double *A, *B, *Q, *Z;
  int lda, ldb, ldq, ldz;
};

int run_ht(const std::vector<HtPair>& ps, int* info_out, const schur_opts* opts) {
  schur_opts o;
  schur::read_opts(opts, &o);
  cudaStream_t st = (cudaStream_t)o.stream;
  const int nb = (int)ps.size();
  const size_t desc_bytes = ((size_t)nb * sizeof(HtDesc) + 255) / 256 * 256;
  const size_t need = desc_bytes + (size_t)nb * sizeof(int);
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
    std::vector<HtDesc> hd(nb);
    int nmax = 0;
    for (int b = 0; b < nb; ++b) {
      const HtPair& p = ps[b];
      hd[b] = HtDesc{p.A, p.B, p.Q, p.Z, p.lda, p.ldb, p.ldq, p.ldz, p.n, 0};
      nmax = std::max(nmax, p.n);
    }
    HtDesc* dd = (HtDesc*)mem;
    int* dinfo = (int*)(mem + desc_bytes);
    schur::ck_at(cudaMemcpyAsync(dd, hd.data(), nb * sizeof(HtDesc), cudaMemcpyHostToDevice, st), __LINE__);
    const int grid = std::min(nb, 8 * schur::num_sms());
    if (nmax >= HT_BIG_N)
      k_ht<HT_THREADS_BIG><<<grid, HT_THREADS_BIG, 0, st>>>(dd, nb, o.want_z, o.z_init, dinfo);
    else
      k_ht<HT_THREADS><<<grid, HT_THREADS, 0, st>>>(dd, nb, o.want_z, o.z_init, dinfo);
    schur::ck_at(cudaGetLastError(), __LINE__);
    schur::ck_at(cudaMemcpyAsync(info_out, dinfo, nb * sizeof(int), cudaMemcpyDeviceToHost, st), __LINE__);
    schur::ck_at(cudaStreamSynchronize(st), __LINE__);
    schur::g_stats.kernel_launches = 1;
  } catch (const schur::CudaError&) {
    rc = SCHUR_ERR_CUDA;
  }
  if (own) cudaFree(mem);
  return rc;
}

}  // namespace

extern "C" int schur_ht_reduce(int n, double* A, int lda, double* B, int ldb, double* Q, int ldq, double* Z, int ldz,
                               const schur_opts* opts) {
  if (n < 0) return -1;
  if (n > 0 && A == nullptr) return -2;
  if (lda < std::max(1, n)) return -3;
  if (n > 0 && B == nullptr) return -4;
  if (ldb < std::max(1, n)) return -5;
  schur_opts oq;
  schur::read_opts(opts, &oq);
  const int want_qz = oq.want_z;
  if (want_qz && n > 0 && Q == nullptr) return -6;
  if (want_qz && ldq < std::max(1, n)) return -7;
  if (want_qz && n > 0 && Z == nullptr) return -8;
  if (want_qz && ldz < std::max(1, n)) return -9;
  memset(&schur::g_stats, 0, sizeof(schur::g_stats));
  if (n == 0) return SCHUR_OK;
  std::vector<HtPair> ps{HtPair{n, A, B, want_qz ? Q : nullptr, want_qz ? Z : nullptr, lda, ldb,
                                want_qz ? ldq : 1, want_qz ? ldz : 1}};
  int info = 0;
  const int rc = run_ht(ps, &info, opts);
  return rc ? rc : info;
}

extern "C" int schur_ht_reduce_batched(int batch, const int* n, double* const* A, const int* lda, double* const* B,
                                       const int* ldb, double* const* Q, const int* ldq, double* const* Z,
                                       const int* ldz, int* info, const schur_opts* opts) {
  if (batch < 0) return -1;
  if (batch == 0) return SCHUR_OK;
  if (!n) return -2;
  if (!A) return -3;
  if (!lda) return -4;
  if (!B) return -5;
  if (!ldb) return -6;
  schur_opts oq;
  schur::read_opts(opts, &oq);
  const int want_qz = oq.want_z;
  if (want_qz && !Q) return -7;
  if (want_qz && !ldq) return -8;
  if (want_qz && !Z) return -9;
  if (want_qz && !ldz) return -10;
  if (!info) return -11;
  std::vector<HtPair> ps(batch);
  for (int b = 0; b < batch; ++b) {
    if (n[b] < 1) return -2;
    if (!A[b]) return -3;
    if (lda[b] < n[b]) return -4;
    if (!B[b]) return -5;
    if (ldb[b] < n[b]) return -6;
    if (want_qz && !Q[b]) return -7;
    if (want_qz && ldq[b] < n[b]) return -8;
    if (want_qz && !Z[b]) return -9;
    if (want_qz && ldz[b] < n[b]) return -10;
    ps[b] = HtPair{n[b], A[b], B[b], want_qz ? Q[b] : nullptr, want_qz ? Z[b] : nullptr, lda[b], ldb[b],
                   want_qz ? ldq[b] : 1, want_qz ? ldz[b] : 1};
  }
  memset(&schur::g_stats, 0, sizeof(schur::g_stats));
  return run_ht(ps, info, opts);
}
