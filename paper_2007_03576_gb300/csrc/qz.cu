// qz.cu -- generalized real Schur form of Hessenberg-triangular pairs (the
// QZ algorithm), the generalized case of the paper's remarks: Sec. 1 (the
// pair (H, T) and its generalized Schur form), Sec. 2.1 (LAPACK's convention:
// |T_ii| <= u ||T||_F is an infinite eigenvalue, T_ii set to zero), Sec. 2.2
// (shifts from the trailing 2x2 pair; bulge vector
// v = (H T^-1 - l1)(H T^-1 - l2) e1; left 3x3 reflectors plus right reflectors
// that restore T's triangular form) and Sec. 3.4 (infinite eigenvalues chased
// to the upper-left corner of the active block).
//
// One thread block owns one pair and runs the whole iteration on it in
// global memory (the pairs of a batch stay L2-resident at the orders this
// entry point is meant for): the deflation scan and the search for negligible
// T_ii are block reductions; each reflector or rotation is built by thread 0
// and applied by all threads, columns or rows in parallel.  The order of the
// transformations is the oracle's (oracle/qz.py), so one sweep with the same
// shifts gives the same pair up to rounding.
//
// This is the double-shift form of the iteration (one bulge per sweep, no
// AED): the multishift / AED machinery of the standard case is not carried
// over to pairs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/schur_gb300.h"
#include "common.cuh"
#include "host.h"

namespace {

constexpr int QZ_THREADS = 256;        // pairs of order < QZ_BIG_N
constexpr int QZ_THREADS_BIG = 1024;   // larger pairs: one column / row per thread
constexpr int QZ_BIG_N = 384;
constexpr int QZ_WARPS = QZ_THREADS_BIG / 32;
constexpr double QZ_U = 0x1p-52;

struct QzDesc {
  double *H, *T, *Q, *Z, *ar, *ai, *be;
  long long ldh, ldt, ldq, ldz;
  int n, pad;
};

struct QzShared {
  double w[4];        // current transform: w0, w1, w2, tau (reflector) or c, s (rotation)
  double m[8];        // 2x2 orthogonal factors (U, V) of a standardisation
  double x[3];        // the bulge column
  double red[QZ_WARPS];
  int ired[QZ_WARPS];
  int iv[4];
};

struct GM {
  double* p;
  long long ld;
  __device__ double& operator()(int r, int c) const { return p[r + c * ld]; }
};

// (c, s) of a left rotation of rows (i, k) that zeroes b (the pair (a, b)
// becomes (hypot(a, b), 0)).
__device__ void rot_second(double a, double b, double& c, double& s) {
  if (b == 0.0) {
    c = 1.0;
    s = 0.0;
    return;
  }
  const double r = hypot(a, b);
  c = a / r;
  s = b / r;
}

// (c, s) of a right rotation of columns (i, k) that zeroes a: c a + s b = 0.
__device__ void rot_first(double a, double b, double& c, double& s) {
  if (a == 0.0) {
    c = 1.0;
    s = 0.0;
    return;
  }
  const double r = hypot(a, b);
  c = b / r;
  s = -a / r;
}

// ---------------------------------------------------- block-wide products

// M[r..r+nr-1, c0..c1-1] <- (I - tau w w^T) M[...], w = (w0, w1, w2).
__device__ void left_apply(const GM& M, int r, int nr, int c0, int c1, double w0, double w1, double w2, double tau) {
  if (tau == 0.0) return;
  for (int c = c0 + (int)threadIdx.x; c < c1; c += blockDim.x) {
    const double a0 = M(r, c), a1 = M(r + 1, c), a2 = (nr == 3) ? M(r + 2, c) : 0.0;
    const double s = tau * fma(w2, a2, fma(w1, a1, w0 * a0));
    M(r, c) = fma(-s, w0, a0);
    M(r + 1, c) = fma(-s, w1, a1);
    if (nr == 3) M(r + 2, c) = fma(-s, w2, a2);
  }
}

// M[r0..r1-1, c..c+nr-1] <- M[...] (I - tau w w^T).
__device__ void right_apply(const GM& M, int c, int nr, int r0, int r1, double w0, double w1, double w2,
                            double tau) {
  if (tau == 0.0) return;
  for (int r = r0 + (int)threadIdx.x; r < r1; r += blockDim.x) {
    const double a0 = M(r, c), a1 = M(r, c + 1), a2 = (nr == 3) ? M(r, c + 2) : 0.0;
    const double s = tau * fma(w2, a2, fma(w1, a1, w0 * a0));
    M(r, c) = fma(-s, w0, a0);
    M(r, c + 1) = fma(-s, w1, a1);
    if (nr == 3) M(r, c + 2) = fma(-s, w2, a2);
  }
}

// rows (i, k) <- [c s; -s c] rows (i, k), columns c0..c1-1
__device__ void rot_rows(const GM& M, int i, int k, double c, double s, int c0, int c1) {
  for (int j = c0 + (int)threadIdx.x; j < c1; j += blockDim.x) {
    const double x = M(i, j), y = M(k, j);
    M(i, j) = c * x + s * y;
    M(k, j) = -s * x + c * y;
  }
}

// columns (i, k) <- (columns i, k) [c -s; s c], rows r0..r1-1
__device__ void rot_cols(const GM& M, int i, int k, double c, double s, int r0, int r1) {
  for (int j = r0 + (int)threadIdx.x; j < r1; j += blockDim.x) {
    const double x = M(j, i), y = M(j, k);
    M(j, i) = c * x + s * y;
    M(j, k) = -s * x + c * y;
  }
}

// rows (k, k+1) <- U^T rows (k, k+1) (U = [u0 u2; u1 u3], column-major), columns c0..c1-1
__device__ void mat_rows(const GM& M, int k, const double* U, int c0, int c1) {
  for (int j = c0 + (int)threadIdx.x; j < c1; j += blockDim.x) {
    const double x = M(k, j), y = M(k + 1, j);
    M(k, j) = U[0] * x + U[1] * y;
    M(k + 1, j) = U[2] * x + U[3] * y;
  }
}

// columns (k, k+1) <- columns (k, k+1) V, rows r0..r1-1
__device__ void mat_cols(const GM& M, int k, const double* V, int r0, int r1) {
  for (int j = r0 + (int)threadIdx.x; j < r1; j += blockDim.x) {
    const double x = M(j, k), y = M(j, k + 1);
    M(j, k) = x * V[0] + y * V[1];
    M(j, k + 1) = x * V[2] + y * V[3];
  }
}

__device__ double block_sum(double v, QzShared* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh->red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh->red[w];
  __syncthreads();
  return t;
}

// op 0: max, op 1: min
__device__ int block_ireduce(int v, int op, QzShared* sh) {
  for (int o = 16; o > 0; o >>= 1) {
    const int u = __shfl_xor_sync(0xffffffffu, v, o);
    v = op ? min(v, u) : max(v, u);
  }
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh->ired[threadIdx.x >> 5] = v;
  __syncthreads();
  int t = sh->ired[0];
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w) t = op ? min(t, sh->ired[w]) : max(t, sh->ired[w]);
  __syncthreads();
  return t;
}

// eigenvalues of the 2x2 pair (S2, T2) with T2 upper triangular, nonsingular:
// those of M = S2 T2^-1 (closed form); returns true for a complex pair
// (re +- i im), else the real roots r1 >= r2 in (re, im).
__device__ bool pair_eigs(double s00, double s01, double s10, double s11, double t00, double t01, double t11,
                          double& re, double& im) {
  // M = S2 T2^-1, T2^-1 = [1/t00, -t01/(t00 t11); 0, 1/t11]
  const double i00 = 1.0 / t00, i11 = 1.0 / t11, i01 = -t01 * i00 * i11;
  const double m00 = s00 * i00, m01 = s00 * i01 + s01 * i11;
  const double m10 = s10 * i00, m11 = s10 * i01 + s11 * i11;
  const double tr = m00 + m11, det = m00 * m11 - m01 * m10;
  const double disc = 0.25 * tr * tr - det;
  if (disc >= 0.0) {
    const double r = sqrt(disc);
    re = 0.5 * tr + r;
    im = 0.5 * tr - r;
    return false;
  }
  re = 0.5 * tr;
  im = sqrt(-disc);
  return true;
}

}  // namespace

namespace {

// Infinite eigenvalue at T[j, j] = 0 on the block lo..hi: chase the zero to
// (lo, lo) and split the 1x1 pair off there (the oracle's
// chase_infinite_to_top).
__device__ void qz_chase_infinite(const GM& H, const GM& T, const GM& Q, const GM& Z, int n, int lo, int hi, int j,
                                  bool wz, QzShared* sh) {
  for (int i = j; i > lo; --i) {
    if (threadIdx.x == 0) rot_first(T(i - 1, i - 1), T(i - 1, i), sh->w[0], sh->w[1]);
    __syncthreads();
    double c = sh->w[0], s = sh->w[1];
    rot_cols(T, i - 1, i, c, s, 0, i + 1);
    rot_cols(H, i - 1, i, c, s, 0, min(i + 1, hi) + 1);
    if (wz) rot_cols(Z, i - 1, i, c, s, 0, n);
    __syncthreads();
    if (threadIdx.x == 0) {
      T(i - 1, i - 1) = 0.0;
      T(i, i - 1) = 0.0;
      if (i + 1 <= hi) rot_second(H(i, i - 1), H(i + 1, i - 1), sh->w[2], sh->w[3]);
    }
    __syncthreads();
    if (i + 1 <= hi) {
      c = sh->w[2];
      s = sh->w[3];
      rot_rows(H, i, i + 1, c, s, i - 1, n);
      rot_rows(T, i, i + 1, c, s, i, n);
      if (wz) rot_cols(Q, i, i + 1, c, s, 0, n);
      __syncthreads();
      if (threadIdx.x == 0) {
        H(i + 1, i - 1) = 0.0;
        T(i + 1, i) = 0.0;
      }
      __syncthreads();
    }
  }
  if (lo < hi) {
    if (threadIdx.x == 0) rot_second(H(lo, lo), H(lo + 1, lo), sh->w[0], sh->w[1]);
    __syncthreads();
    const double c = sh->w[0], s = sh->w[1];
    rot_rows(H, lo, lo + 1, c, s, lo, n);
    rot_rows(T, lo, lo + 1, c, s, lo, n);
    if (wz) rot_cols(Q, lo, lo + 1, c, s, 0, n);
    __syncthreads();
    if (threadIdx.x == 0) {
      H(lo + 1, lo) = 0.0;
      T(lo, lo) = 0.0;
      T(lo + 1, lo) = 0.0;
    }
    __syncthreads();
  }
}

// The 2x2 diagonal block pair at k, k+1 (T's block nonsingular): split a real
// pair, or make T's block diagonal and positive for a complex pair (the
// oracle's standardize_pair_block).
__device__ void qz_standardize(const GM& H, const GM& T, const GM& Q, const GM& Z, int n, int k, bool wz,
                               QzShared* sh) {
  if (threadIdx.x == 0) {
    const double s00 = H(k, k), s01 = H(k, k + 1), s10 = H(k + 1, k), s11 = H(k + 1, k + 1);
    const double t00 = T(k, k), t01 = T(k, k + 1), t11 = T(k + 1, k + 1);
    double re, im;
    const bool cpx = pair_eigs(s00, s01, s10, s11, t00, t01, t11, re, im);
    sh->iv[0] = cpx ? 1 : 0;
    if (!cpx) {
      const double l1 = re;
      const double k00 = s00 - l1 * t00, k01 = s01 - l1 * t01, k10 = s10, k11 = s11 - l1 * t11;
      double x0, x1;
      if (hypot(k00, k01) >= hypot(k10, k11)) {
        x0 = -k01;
        x1 = k00;
      } else {
        x0 = -k11;
        x1 = k10;
      }
      double h = hypot(x0, x1);
      if (h == 0.0) {
        x0 = 1.0;
        x1 = 0.0;
        h = 1.0;
      }
      sh->w[0] = x0 / h;   // first column of the right rotation = the eigenvector
      sh->w[1] = x1 / h;
    } else {
      // T2 = U diag(s1, s2) V^T: V diagonalises T2^T T2 (a Jacobi rotation),
      // U's columns are those of T2 V scaled to unit length
      const double f = t00, g = t01, hh = t11;
      const double th = 0.5 * atan2(2.0 * f * g, f * f - g * g - hh * hh);
      const double cs = cos(th), sn = sin(th);
      const double v00 = cs, v10 = sn, v01 = -sn, v11 = cs;
      const double w00 = f * v00 + g * v10, w10 = hh * v10;
      const double w01 = f * v01 + g * v11, w11 = hh * v11;
      const double n0 = hypot(w00, w10), n1 = hypot(w01, w11);
      sh->m[0] = w00 / n0;
      sh->m[1] = w10 / n0;
      sh->m[2] = w01 / n1;
      sh->m[3] = w11 / n1;
      sh->m[4] = v00;
      sh->m[5] = v10;
      sh->m[6] = v01;
      sh->m[7] = v11;
      sh->x[0] = n0;
      sh->x[1] = n1;
    }
  }
  __syncthreads();
  if (sh->iv[0] == 0) {
    const double c = sh->w[0], s = sh->w[1];
    rot_cols(H, k, k + 1, c, s, 0, k + 2);
    rot_cols(T, k, k + 1, c, s, 0, k + 2);
    if (wz) rot_cols(Z, k, k + 1, c, s, 0, n);
    __syncthreads();
    if (threadIdx.x == 0) rot_second(T(k, k), T(k + 1, k), sh->w[2], sh->w[3]);
    __syncthreads();
    const double c2 = sh->w[2], s2 = sh->w[3];
    rot_rows(H, k, k + 1, c2, s2, k, n);
    rot_rows(T, k, k + 1, c2, s2, k, n);
    if (wz) rot_cols(Q, k, k + 1, c2, s2, 0, n);
    __syncthreads();
    if (threadIdx.x == 0) {
      H(k + 1, k) = 0.0;
      T(k + 1, k) = 0.0;
    }
  } else {
    mat_rows(H, k, sh->m, k, n);
    mat_rows(T, k, sh->m, k, n);
    if (wz) mat_cols(Q, k, sh->m, 0, n);
    __syncthreads();
    mat_cols(H, k, sh->m + 4, 0, k + 2);
    mat_cols(T, k, sh->m + 4, 0, k + 2);
    if (wz) mat_cols(Z, k, sh->m + 4, 0, n);
    __syncthreads();
    if (threadIdx.x == 0) {
      T(k, k) = sh->x[0];
      T(k, k + 1) = 0.0;
      T(k + 1, k) = 0.0;
      T(k + 1, k + 1) = sh->x[1];
    }
  }
  __syncthreads();
}

// (ssum, sprod) of the trailing 2x2 of M = H T^-1 on lo..hi (hi - lo >= 2),
// or the exceptional pair; thread 0 only.
__device__ void qz_shifts(const GM& H, const GM& T, int lo, int hi, bool exceptional, double& ssum, double& sprod) {
  if (exceptional) {
    const double mhh = H(hi, hi) / T(hi, hi);
    const double s = fabs(H(hi, hi - 1) / T(hi - 1, hi - 1)) +
                     ((hi - 2 >= lo) ? fabs(H(hi - 1, hi - 2) / T(hi - 2, hi - 2)) : 0.0);
    const double a = mhh + 0.75 * s;
    ssum = 2.0 * a;
    sprod = a * a + 0.4375 * s * s;
    return;
  }
  const int a = hi - 2;
  // inverse of the 3x3 upper triangular T[a:hi+1, a:hi+1], columns 1 and 2
  const double t00 = T(a, a), t01 = T(a, a + 1), t02 = T(a, a + 2);
  const double t11 = T(a + 1, a + 1), t12 = T(a + 1, a + 2), t22 = T(a + 2, a + 2);
  const double i11 = 1.0 / t11, i22 = 1.0 / t22, i00 = 1.0 / t00;
  const double i01 = -t01 * i00 * i11;
  const double i12 = -t12 * i11 * i22;
  const double i02 = -(t01 * i12 + t02 * i22) * i00;
  // M = H[hi-1:hi+1, a:hi+1] @ Ti[:, 1:3]; H(hi-1, a) is the subdiagonal, H(hi, a) = 0
  const double h10 = H(hi - 1, a), h11 = H(hi - 1, a + 1), h12 = H(hi - 1, a + 2);
  const double h21 = H(hi, a + 1), h22 = H(hi, a + 2);
  const double m00 = h10 * i01 + h11 * i11;
  const double m01 = h10 * i02 + h11 * i12 + h12 * i22;
  const double m10 = h21 * i11;
  const double m11 = h21 * i12 + h22 * i22;
  ssum = m00 + m11;
  sprod = m00 * m11 - m01 * m10;
}

// left reflector (1, v1, v2) applied to one column's entries (a0, a1, a2):
// the arithmetic of left_apply, so that thread 0 can predict the values the
// block writes
__device__ __forceinline__ void left3_col(double v1, double v2, double tau, double& a0, double& a1, double& a2) {
  const double s = tau * fma(v2, a2, fma(v1, a1, a0));
  a0 = fma(-s, 1.0, a0);
  a1 = fma(-s, v1, a1);
  a2 = fma(-s, v2, a2);
}

// one double-shift sweep on lo..hi (the oracle's qz_sweep).  Reflectors come
// from house3, the short-chain reflector of the standard case: the oracle's
// convention (beta = -sign(x0) ||x||, tau = (beta - x0) / beta,
// v = (1, x1, x2) / (x0 - beta), identity for a zero tail), built from FP32
// seeds and one Newton step instead of IEEE division and square root.  Per
// position
// thread 0 builds all three reflectors at once -- the left one from the
// bulge column, the two right ones from T's 3x3 diagonal block after the
// left one, computed with the same arithmetic as the block's own updates --
// so a position costs three block barriers: left products, right products
// (both right reflectors applied by the thread that owns a row), bookkeeping.
__device__ void qz_sweep_dev(const GM& H, const GM& T, const GM& Q, const GM& Z, int n, int lo, int hi, double ssum,
                             double sprod, bool wz, QzShared* sh) {
  double x0 = 0.0, x1 = 0.0, x2 = 0.0;   // the bulge column (thread 0)
  if (threadIdx.x == 0) {
    const double m00 = H(lo, lo) / T(lo, lo), m10 = H(lo + 1, lo) / T(lo, lo);
    const double tl = T(lo, lo + 1), t11 = T(lo + 1, lo + 1);
    const double m01 = (H(lo, lo + 1) - m00 * tl) / t11;
    const double m11 = (H(lo + 1, lo + 1) - m10 * tl) / t11;
    const double m21 = H(lo + 2, lo + 1) / t11;
    x0 = m00 * m00 + m10 * m01 - ssum * m00 + sprod;
    x1 = m00 * m10 + m10 * m11 - ssum * m10;
    x2 = m10 * m21;
  }
  for (int k = lo; k < hi - 1; ++k) {
    if (threadIdx.x == 0) {
      if (k > lo) {
        x0 = H(k, k - 1);
        x1 = H(k + 1, k - 1);
        x2 = H(k + 2, k - 1);
      }
      double v1, v2, tau, beta;
      house3(3, x0, x1, x2, v1, v2, tau, beta);
      // T[k..k+2, k..k+2] after the left reflector (lower part exactly zero)
      double b00 = T(k, k), b10 = 0.0, b20 = 0.0;
      double b01 = T(k, k + 1), b11 = T(k + 1, k + 1), b21 = 0.0;
      double b02 = T(k, k + 2), b12 = T(k + 1, k + 2), b22 = T(k + 2, k + 2);
      if (tau != 0.0) {
        left3_col(v1, v2, tau, b00, b10, b20);
        left3_col(v1, v2, tau, b01, b11, b21);
        left3_col(v1, v2, tau, b02, b12, b22);
      }
      // first right reflector: row k+2 -> (0, 0, *), w = (u2, u1, 1)
      double u1, u2, t1, g1;
      house3(3, b22, b21, b20, u1, u2, t1, g1);
      // its effect on row k+1 (right_apply's arithmetic), then the second
      // right reflector from (T[k+1, k], T[k+1, k+1]), w = (z1, 1)
      if (t1 != 0.0) {
        const double s = t1 * fma(1.0, b12, fma(u1, b11, u2 * b10));
        b10 = fma(-s, u2, b10);
        b11 = fma(-s, u1, b11);
      }
      double z1, z2, t2, g2;
      house3(2, b11, b10, 0.0, z1, z2, t2, g2);
      sh->w[0] = v1;
      sh->w[1] = v2;
      sh->w[2] = tau;
      sh->w[3] = beta;
      sh->m[0] = u2;
      sh->m[1] = u1;
      sh->m[2] = t1;
      sh->m[3] = z1;
      sh->m[4] = t2;
    }
    __syncthreads();
    {
      const double v1 = sh->w[0], v2 = sh->w[1], tau = sh->w[2];
      const int c0 = (k > lo) ? k - 1 : lo;
      // H's columns c0..n-1, T's columns k..n-1 and Q's rows in one pass,
      // so that the three matrices' loads overlap
      if (tau != 0.0) {
        const int nh = n - c0, nt = n - k, total = nh + nt + (wz ? n : 0);
        for (int it = threadIdx.x; it < total; it += blockDim.x) {
          if (it < nh) {
            const int c = c0 + it;
            double a0 = H(k, c), a1 = H(k + 1, c), a2 = H(k + 2, c);
            left3_col(v1, v2, tau, a0, a1, a2);
            H(k, c) = a0;
            H(k + 1, c) = a1;
            H(k + 2, c) = a2;
          } else if (it < nh + nt) {
            const int c = k + (it - nh);
            double a0 = T(k, c), a1 = T(k + 1, c), a2 = T(k + 2, c);
            left3_col(v1, v2, tau, a0, a1, a2);
            T(k, c) = a0;
            T(k + 1, c) = a1;
            T(k + 2, c) = a2;
          } else {
            const int r = it - nh - nt;
            double a0 = Q(r, k), a1 = Q(r, k + 1), a2 = Q(r, k + 2);
            left3_col(v1, v2, tau, a0, a1, a2);
            Q(r, k) = a0;
            Q(r, k + 1) = a1;
            Q(r, k + 2) = a2;
          }
        }
      }
    }
    __syncthreads();
    if (threadIdx.x == 0 && k > lo) {
      H(k, k - 1) = sh->w[3];
      H(k + 1, k - 1) = 0.0;
      H(k + 2, k - 1) = 0.0;
    }
    {
      const double a0w = sh->m[0], a1w = sh->m[1], t1 = sh->m[2], z1 = sh->m[3], t2 = sh->m[4];
      const int rmax = min(k + 3, hi);
      // one row per thread: the 3x3 reflector on columns k..k+2, then the
      // 2x2 on columns k, k+1 (rows past k+1 of T get only the first)
      auto both = [&](const GM& M, int r, bool second) {
        double e0 = M(r, k), e1 = M(r, k + 1), e2 = M(r, k + 2);
        if (t1 != 0.0) {
          const double s = t1 * fma(1.0, e2, fma(a1w, e1, a0w * e0));
          e0 = fma(-s, a0w, e0);
          e1 = fma(-s, a1w, e1);
          e2 = fma(-s, 1.0, e2);
        }
        if (second && t2 != 0.0) {
          const double s = t2 * fma(0.0, 0.0, fma(1.0, e1, z1 * e0));
          e0 = fma(-s, z1, e0);
          e1 = fma(-s, 1.0, e1);
        }
        M(r, k) = e0;
        M(r, k + 1) = e1;
        M(r, k + 2) = e2;
      };
      const int nh = rmax + 1, nt = k + 3, total = nh + nt + (wz ? n : 0);
      for (int it = threadIdx.x; it < total; it += blockDim.x) {
        if (it < nh)
          both(H, it, true);
        else if (it < nh + nt)
          both(T, it - nh, it - nh <= k + 1);
        else
          both(Z, it - nh - nt, true);
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      T(k + 2, k) = 0.0;
      T(k + 2, k + 1) = 0.0;
      T(k + 1, k) = 0.0;
    }
  }
  // last position: rows / columns hi-1, hi
  const int k = hi - 1;
  if (threadIdx.x == 0) {
    x0 = H(k, k - 1);
    x1 = H(k + 1, k - 1);
    double v1, v2, tau, beta;
    house3(2, x0, x1, 0.0, v1, v2, tau, beta);
    double b10 = 0.0, b11 = T(k + 1, k + 1);
    if (tau != 0.0) {   // column k: (T(k, k), 0); column k+1: (T(k, k+1), T(k+1, k+1))
      const double a0 = T(k, k), a1 = 0.0;
      const double s0 = tau * fma(0.0, 0.0, fma(v1, a1, a0));
      b10 = fma(-s0, v1, a1);
      const double c0 = T(k, k + 1), c1 = T(k + 1, k + 1);
      const double s1 = tau * fma(0.0, 0.0, fma(v1, c1, c0));
      b11 = fma(-s1, v1, c1);
    }
    double z1, z2, t2, g2;
    house3(2, b11, b10, 0.0, z1, z2, t2, g2);
    sh->w[0] = v1;
    sh->w[2] = tau;
    sh->w[3] = beta;
    sh->m[3] = z1;
    sh->m[4] = t2;
  }
  __syncthreads();
  {
    const double v1 = sh->w[0], tau = sh->w[2];
    left_apply(H, k, 2, k - 1, n, 1.0, v1, 0.0, tau);
    left_apply(T, k, 2, k, n, 1.0, v1, 0.0, tau);
    if (wz) right_apply(Q, k, 2, 0, n, 1.0, v1, 0.0, tau);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    H(k, k - 1) = sh->w[3];
    H(k + 1, k - 1) = 0.0;
  }
  {
    const double z1 = sh->m[3], t2 = sh->m[4];
    right_apply(H, k, 2, 0, hi + 1, z1, 1.0, 0.0, t2);
    right_apply(T, k, 2, 0, k + 2, z1, 1.0, 0.0, t2);
    if (wz) right_apply(Z, k, 2, 0, n, z1, 1.0, 0.0, t2);
  }
  __syncthreads();
  if (threadIdx.x == 0) T(k + 1, k) = 0.0;
  __syncthreads();
}

// The whole iteration on one pair (the oracle's qz driver).  Returns 0, 1 +
// the top row of a block that did not converge, or SCHUR_ERR_NONFINITE.
__device__ int qz_pair(const QzDesc& d, bool wz, int z_init, QzShared* sh) {
  const int n = d.n;
  const GM H{d.H, d.ldh}, T{d.T, d.ldt}, Q{d.Q, d.ldq}, Z{d.Z, d.ldz};
  // input check and ||T||_F (upper triangle), H below the subdiagonal and T
  // below the diagonal set to zero
  double ss = 0.0;
  int bad = 0;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int r = idx % n, c = idx / n;
    const double h = H(r, c), t = T(r, c);
    if (r <= c + 1 && !isfinite(h)) bad = 1;
    if (r <= c && !isfinite(t)) bad = 1;
    if (r <= c) ss = fma(t, t, ss);
  }
  if (block_ireduce(bad, 0, sh)) return SCHUR_ERR_NONFINITE;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int r = idx % n, c = idx / n;
    if (r > c + 1) H(r, c) = 0.0;
    if (r > c) T(r, c) = 0.0;
    if (wz && z_init == 0) {
      Q(r, c) = (r == c) ? 1.0 : 0.0;
      Z(r, c) = (r == c) ? 1.0 : 0.0;
    }
  }
  const double tthr = QZ_U * sqrt(block_sum(ss, sh));
  const double sml = 0x1p-1022 * ((double)n / QZ_U);
  __syncthreads();
  int hi = n - 1, its = 0, info = 0;
  while (hi >= 0) {
    // lo: the largest k <= hi with a negligible H[k, k-1] (0 if none)
    int cand = 0;
    for (int k = 1 + (int)threadIdx.x; k <= hi; k += blockDim.x) {
      const double sub = fabs(H(k, k - 1));
      if (sub <= fmax(QZ_U * (fabs(H(k - 1, k - 1)) + fabs(H(k, k))), sml)) cand = max(cand, k);
    }
    const int lo = block_ireduce(cand, 0, sh);
    if (threadIdx.x == 0 && lo > 0) H(lo, lo - 1) = 0.0;
    // negligible T_jj in [lo, hi]: set to zero, the first one is chased
    int jinf = n;
    for (int jj = lo + (int)threadIdx.x; jj <= hi; jj += blockDim.x)
      if (fabs(T(jj, jj)) <= tthr) {
        T(jj, jj) = 0.0;
        jinf = min(jinf, jj);
      }
    jinf = block_ireduce(jinf, 1, sh);
    if (jinf < n && hi > lo) {
      qz_chase_infinite(H, T, Q, Z, n, lo, hi, jinf, wz, sh);
      its = 0;
      continue;
    }
    const int size = hi - lo + 1;
    if (size == 1) {
      hi -= 1;
      its = 0;
      continue;
    }
    if (size == 2) {
      qz_standardize(H, T, Q, Z, n, lo, wz, sh);
      hi -= 2;
      its = 0;
      continue;
    }
    ++its;
    if (its > 30 * size) {
      info = lo + 1;
      break;
    }
    if (threadIdx.x == 0) {
      double ssum, sprod;
      qz_shifts(H, T, lo, hi, its % 10 == 0, ssum, sprod);
      sh->red[0] = ssum;
      sh->red[1] = sprod;
    }
    __syncthreads();
    const double ssum = sh->red[0], sprod = sh->red[1];
    __syncthreads();
    qz_sweep_dev(H, T, Q, Z, n, lo, hi, ssum, sprod, wz, sh);
  }
  // eigenvalues: (alphar + i alphai) / beta per block
  __syncthreads();
  if (threadIdx.x == 0) {
    int k = 0;
    while (k < n) {
      if (k + 1 < n && H(k + 1, k) != 0.0) {
        double re, im;
        pair_eigs(H(k, k), H(k, k + 1), H(k + 1, k), H(k + 1, k + 1), T(k, k), T(k, k + 1), T(k + 1, k + 1), re, im);
        const double b0 = T(k, k), b1 = T(k + 1, k + 1);
        d.ar[k] = re * b0;
        d.ai[k] = im * b0;
        d.be[k] = b0;
        d.ar[k + 1] = re * b1;
        d.ai[k + 1] = -im * b1;
        d.be[k + 1] = b1;
        k += 2;
      } else {
        const double sg = (T(k, k) < 0.0) ? -1.0 : 1.0;
        d.ar[k] = sg * H(k, k);
        d.ai[k] = 0.0;
        d.be[k] = sg * T(k, k);
        k += 1;
      }
    }
  }
  __syncthreads();
  return info;
}

template <int NT>
__global__ void __launch_bounds__(NT) k_qz(const QzDesc* __restrict__ descs, int batch, int want_z, int z_init,
                                                   int* __restrict__ info) {
  __shared__ QzShared sh;
  for (int b = blockIdx.x; b < batch; b += gridDim.x) {
    const int r = qz_pair(descs[b], want_z != 0, z_init, &sh);
    if (threadIdx.x == 0) info[b] = r;
    __syncthreads();
  }
}

// one sweep with given shifts (the single-step parity entry point)
__global__ void __launch_bounds__(QZ_THREADS_BIG) k_qz_sweep(QzDesc d, int lo, int hi, double ssum, double sprod) {
  __shared__ QzShared sh;
  const GM H{d.H, d.ldh}, T{d.T, d.ldt}, Q{d.Q, d.ldq}, Z{d.Z, d.ldz};
  qz_sweep_dev(H, T, Q, Z, d.n, lo, hi, ssum, sprod, d.Q != nullptr, &sh);
}

struct QzPair {
  int n;
  double *H, *T, *Q, *Z, *ar, *ai, *be;
  int ldh, ldt, ldq, ldz;
};

int run_qz(const std::vector<QzPair>& ps, int* info_out, const schur_opts* opts) {
  schur_opts o;
  schur::read_opts(opts, &o);
  cudaStream_t st = (cudaStream_t)o.stream;
  const int nb = (int)ps.size();
  const size_t desc_bytes = ((size_t)nb * sizeof(QzDesc) + 255) / 256 * 256;
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
    std::vector<QzDesc> hd(nb);
    for (int b = 0; b < nb; ++b) {
      const QzPair& p = ps[b];
      hd[b] = QzDesc{p.H, p.T, p.Q, p.Z, p.ar, p.ai, p.be, p.ldh, p.ldt, p.ldq, p.ldz, p.n, 0};
    }
    QzDesc* dd = (QzDesc*)mem;
    int* dinfo = (int*)(mem + desc_bytes);
    schur::ck_at(cudaMemcpyAsync(dd, hd.data(), nb * sizeof(QzDesc), cudaMemcpyHostToDevice, st), __LINE__);
    const int grid = std::min(nb, 8 * schur::num_sms());
    int nmax = 0;
    for (const QzPair& p : ps) nmax = std::max(nmax, p.n);
    if (nmax >= QZ_BIG_N)
      k_qz<QZ_THREADS_BIG><<<grid, QZ_THREADS_BIG, 0, st>>>(dd, nb, o.want_z, o.z_init, dinfo);
    else
      k_qz<QZ_THREADS><<<grid, QZ_THREADS, 0, st>>>(dd, nb, o.want_z, o.z_init, dinfo);
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

extern "C" int schur_qz(int n, double* H, int ldh, double* T, int ldt, double* Q, int ldq, double* Z, int ldz,
                        double* alphar, double* alphai, double* beta, const schur_opts* opts) {
  if (n < 0) return -1;
  if (n > 0 && H == nullptr) return -2;
  if (ldh < std::max(1, n)) return -3;
  if (n > 0 && T == nullptr) return -4;
  if (ldt < std::max(1, n)) return -5;
  schur_opts oq;
  schur::read_opts(opts, &oq);
  const int want_z = oq.want_z;
  if (want_z && n > 0 && Q == nullptr) return -6;
  if (want_z && ldq < std::max(1, n)) return -7;
  if (want_z && n > 0 && Z == nullptr) return -8;
  if (want_z && ldz < std::max(1, n)) return -9;
  if (n > 0 && alphar == nullptr) return -10;
  if (n > 0 && alphai == nullptr) return -11;
  if (n > 0 && beta == nullptr) return -12;
  memset(&schur::g_stats, 0, sizeof(schur::g_stats));
  if (n == 0) return SCHUR_OK;
  std::vector<QzPair> ps{QzPair{n, H, T, Q, Z, alphar, alphai, beta, ldh, ldt, ldq, ldz}};
  int info = 0;
  const int rc = run_qz(ps, &info, opts);
  return rc ? rc : info;
}

extern "C" int schur_qz_batched(int batch, const int* n, double* const* H, const int* ldh, double* const* T,
                                const int* ldt, double* const* Q, const int* ldq, double* const* Z, const int* ldz,
                                double* const* alphar, double* const* alphai, double* const* beta, int* info,
                                const schur_opts* opts) {
  if (batch < 0) return -1;
  if (batch == 0) return SCHUR_OK;
  if (!n) return -2;
  if (!H) return -3;
  if (!ldh) return -4;
  if (!T) return -5;
  if (!ldt) return -6;
  schur_opts oq;
  schur::read_opts(opts, &oq);
  const int want_z = oq.want_z;
  if (want_z && !Q) return -7;
  if (want_z && !ldq) return -8;
  if (want_z && !Z) return -9;
  if (want_z && !ldz) return -10;
  if (!alphar) return -11;
  if (!alphai) return -12;
  if (!beta) return -13;
  if (!info) return -14;
  std::vector<QzPair> ps(batch);
  for (int b = 0; b < batch; ++b) {
    if (n[b] < 1) return -2;
    if (!H[b]) return -3;
    if (ldh[b] < n[b]) return -4;
    if (!T[b]) return -5;
    if (ldt[b] < n[b]) return -6;
    if (want_z && !Q[b]) return -7;
    if (want_z && ldq[b] < n[b]) return -8;
    if (want_z && !Z[b]) return -9;
    if (want_z && ldz[b] < n[b]) return -10;
    if (!alphar[b]) return -11;
    if (!alphai[b]) return -12;
    if (!beta[b]) return -13;
    ps[b] = QzPair{n[b], H[b], T[b], want_z ? Q[b] : nullptr, want_z ? Z[b] : nullptr, alphar[b], alphai[b], beta[b],
                   ldh[b], ldt[b], want_z ? ldq[b] : 1, want_z ? ldz[b] : 1};
  }
  memset(&schur::g_stats, 0, sizeof(schur::g_stats));
  return run_qz(ps, info, opts);
}

extern "C" int schur_qz_sweep(int n, double* H, int ldh, double* T, int ldt, double* Q, int ldq, double* Z, int ldz,
                              int lo, int hi, double ssum, double sprod, const schur_opts* opts) {
  if (n < 3) return -1;
  if (H == nullptr) return -2;
  if (ldh < n) return -3;
  if (T == nullptr) return -4;
  if (ldt < n) return -5;
  if ((Q == nullptr) != (Z == nullptr)) return Q ? -8 : -6;
  if (Q && ldq < n) return -7;
  if (Z && ldz < n) return -9;
  if (lo < 0 || lo > n - 3) return -10;
  if (hi < lo + 2 || hi > n - 1) return -11;
  schur_opts o;
  schur::read_opts(opts, &o);
  cudaStream_t st = (cudaStream_t)o.stream;
  QzDesc d{H, T, Q, Z, nullptr, nullptr, nullptr, ldh, ldt, Q ? ldq : 1, Z ? ldz : 1, n, 0};
  k_qz_sweep<<<1, n >= QZ_BIG_N ? QZ_THREADS_BIG : QZ_THREADS, 0, st>>>(d, lo, hi, ssum, sprod);
  if (cudaGetLastError() != cudaSuccess) return SCHUR_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return SCHUR_ERR_CUDA;
  return SCHUR_OK;
}
