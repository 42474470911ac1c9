// cta.cuh -- one-thread-block building blocks of the QR iteration.
//
// Every function here is called by all threads of a block with uniform
// arguments; scalar decisions are taken by thread 0 and broadcast through
// shared memory.  Matrices are column-major views (Mat) that may live in
// shared or global memory.  Used by the small-block double-shift QR
// (Sec. 2.2 / the "small Schur" task of Sec. 3.2), the AED step (Sec. 2.5:
// window Schur form, deflation checks, reordering, spike elimination) and the
// batched persistent kernel.
#pragma once

#include "common.cuh"

struct CtaShared {
  double r[8];       // reflector / rotation broadcast
  double q[16];      // 4x4 orthogonal factor of a swap
  double d[16];      // new 4x4 diagonal block of a swap
  double red[32];    // block reductions
  int iv[8];         // integer broadcast
};

__device__ __forceinline__ int cta_tid() { return threadIdx.x; }
__device__ __forceinline__ int cta_nt() { return blockDim.x; }

// ---------------------------------------------------------------------------
// Reflector of order nr (2 or 3) at rows k..k+nr-1.
// ---------------------------------------------------------------------------

// rows k..k+nr-1, columns c0..c1: X <- (I - tau v v^T) X
__device__ __forceinline__ void cta_refl_left(const Mat& M, int k, int nr, double v1, double v2, double tau,
                                              int c0, int c1) {
  if (tau == 0.0) return;
  for (int j = c0 + cta_tid(); j <= c1; j += cta_nt()) {
    double* col = &M(k, j);
    double x0 = col[0], x1 = col[1];
    double x2 = (nr == 3) ? col[2] : 0.0;
    double s = tau * (x0 + v1 * x1 + v2 * x2);
    col[0] = x0 - s;
    col[1] = x1 - s * v1;
    if (nr == 3) col[2] = x2 - s * v2;
  }
}

// columns k..k+nr-1, rows r0..r1: X <- X (I - tau v v^T)
__device__ __forceinline__ void cta_refl_right(const Mat& M, int k, int nr, double v1, double v2, double tau,
                                               int r0, int r1) {
  if (tau == 0.0) return;
  double* c0p = &M(0, k);
  double* c1p = c0p + M.ld;
  double* c2p = c1p + M.ld;
  for (int i = r0 + cta_tid(); i <= r1; i += cta_nt()) {
    double x0 = c0p[i], x1 = c1p[i];
    double x2 = (nr == 3) ? c2p[i] : 0.0;
    double s = tau * (x0 + v1 * x1 + v2 * x2);
    c0p[i] = x0 - s;
    c1p[i] = x1 - s * v1;
    if (nr == 3) c2p[i] = x2 - s * v2;
  }
}

// ---------------------------------------------------------------------------
// Vigilant deflation scan: largest k in (lo, hi] with a negligible H(k, k-1)
// (set to zero), else lo.
// ---------------------------------------------------------------------------
__device__ inline int cta_find_ktop(const Mat& H, int lo, int hi, const DeflParams& dp, CtaShared* sh) {
  if (cta_tid() == 0) sh->iv[0] = lo;
  __syncthreads();
  for (int k = hi - cta_tid(); k > lo; k -= cta_nt()) {
    if (H(k, k - 1) == 0.0 || subdiag_negligible(H, k, lo, hi, dp)) {
      atomicMax(&sh->iv[0], k);
      break;  // smaller k of this thread cannot beat this one
    }
  }
  __syncthreads();
  int l = sh->iv[0];
  __syncthreads();
  if (cta_tid() == 0 && l > lo) H(l, l - 1) = 0.0;
  __syncthreads();
  return l;
}

// ---------------------------------------------------------------------------
// Standardise the decoupled 2x2 block at (k, k) (eq. 2by2_blocks) and apply
// its rotation to rows k, k+1 (columns k+2..ncols-1), columns k, k+1
// (rows 0..k-1) and to U's columns k, k+1 (rows 0..urows-1).
// ---------------------------------------------------------------------------
__device__ inline void cta_standardize_block(const Mat& T, int k, int ncols, const Mat& U, int urows,
                                             CtaShared* sh) {
  if (cta_tid() == 0) {
    double cs, sn, B[4];
    standardize2x2(T(k, k), T(k, k + 1), T(k + 1, k), T(k + 1, k + 1), cs, sn, B);
    sh->r[0] = cs;
    sh->r[1] = sn;
    sh->r[2] = B[0];
    sh->r[3] = B[1];
    sh->r[4] = B[2];
    sh->r[5] = B[3];
  }
  __syncthreads();
  double cs = sh->r[0], sn = sh->r[1];
  if (!(cs == 1.0 && sn == 0.0)) {
    for (int j = k + 2 + cta_tid(); j < ncols; j += cta_nt()) {
      double a = T(k, j), b = T(k + 1, j);
      T(k, j) = cs * a + sn * b;
      T(k + 1, j) = -sn * a + cs * b;
    }
    for (int i = cta_tid(); i < k; i += cta_nt()) {
      double a = T(i, k), b = T(i, k + 1);
      T(i, k) = cs * a + sn * b;
      T(i, k + 1) = -sn * a + cs * b;
    }
    if (U.p) {
      for (int i = cta_tid(); i < urows; i += cta_nt()) {
        double a = U(i, k), b = U(i, k + 1);
        U(i, k) = cs * a + sn * b;
        U(i, k + 1) = -sn * a + cs * b;
      }
    }
  }
  __syncthreads();
  if (cta_tid() == 0) {
    T(k, k) = sh->r[2];
    T(k, k + 1) = sh->r[3];
    T(k + 1, k) = sh->r[4];
    T(k + 1, k + 1) = sh->r[5];
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// One Francis double-shift sweep on [l, i] of the m x m matrix T (full Schur
// mode within T: columns up to m-1, rows from 0), accumulated into U.
// Per reflector: thread 0 builds it (a short FP64 chain, see house3), then
// the left product on rows k..k+2 and the right product on columns k..k+2
// (and U) run over all threads, separated by a barrier because they meet on
// the 3x3 diagonal block.
// ---------------------------------------------------------------------------
__device__ inline void cta_double_shift_sweep(const Mat& T, int m, int l, int i, double ssum, double sprod,
                                              const Mat& U, int urows, CtaShared* sh) {
  for (int k = l; k < i; ++k) {
    int nr = min(3, i - k + 1);
    if (cta_tid() == 0) {
      double x0, x1, x2 = 0.0;
      if (k == l) {
        double h00 = T(l, l), h01 = T(l, l + 1), h10 = T(l + 1, l), h11 = T(l + 1, l + 1);
        x0 = fma(h00, h00, fma(h01, h10, fma(-ssum, h00, sprod)));
        x1 = h10 * (h00 + h11 - ssum);
        if (nr == 3) x2 = h10 * T(l + 2, l + 1);
      } else {
        x0 = T(k, k - 1);
        x1 = T(k + 1, k - 1);
        if (nr == 3) x2 = T(k + 2, k - 1);
      }
      double v1, v2, tau, beta;
      house3(nr, x0, x1, x2, v1, v2, tau, beta);
      if (k > l) {
        T(k, k - 1) = beta;
        T(k + 1, k - 1) = 0.0;
        if (nr == 3) T(k + 2, k - 1) = 0.0;
      }
      sh->r[0] = v1;
      sh->r[1] = v2;
      sh->r[2] = tau;
    }
    __syncthreads();
    double v1 = sh->r[0], v2 = sh->r[1], tau = sh->r[2];
    if (tau != 0.0) {
      for (int j = k + cta_tid(); j < m; j += cta_nt()) {
        double* col = &T(k, j);
        double a0 = col[0], a1 = col[1], a2 = (nr == 3) ? col[2] : 0.0;
        double s = tau * fma(v2, a2, fma(v1, a1, a0));
        col[0] = a0 - s;
        col[1] = fma(-s, v1, a1);
        if (nr == 3) col[2] = fma(-s, v2, a2);
      }
      __syncthreads();
      const int nrr = min(k + 3, i) + 1;   // rows 0..min(k+3, i) of T
      const int nu = U.p ? urows : 0;
      for (int it = cta_tid(); it < nrr + nu; it += cta_nt()) {
        const Mat& M = (it < nrr) ? T : U;
        int r = (it < nrr) ? it : it - nrr;
        double* c0 = &M(r, k);
        double a0 = c0[0], a1 = c0[M.ld], a2 = (nr == 3) ? c0[2 * M.ld] : 0.0;
        double s = tau * fma(v2, a2, fma(v1, a1, a0));
        c0[0] = a0 - s;
        c0[M.ld] = fma(-s, v1, a1);
        if (nr == 3) c0[2 * M.ld] = fma(-s, v2, a2);
      }
    }
    __syncthreads();
  }
}

// Exceptional double shift (EISPACK's ad-hoc shift): s = |h_{i,i-1}| +
// |h_{i-1,i-2}|, a = h_ii + 0.75 s, pair a +- i sqrt(0.4375) s.
__device__ __forceinline__ void exceptional_pair(const Mat& T, int lo, int i, double& ssum, double& sprod) {
  double s = fabs(T(i, i - 1)) + ((i - 2 >= lo) ? fabs(T(i - 1, i - 2)) : 0.0);
  double a = T(i, i) + 0.75 * s;
  ssum = 2.0 * a;
  sprod = a * a + 0.4375 * s * s;
}

// ---------------------------------------------------------------------------
// Francis double-shift QR (Sec. 2.2) of the block [lo, hi] of the m x m T,
// full Schur form within T, accumulated into U (urows x m).  Returns 0 or
// i+1 when the iteration limit 30*max(10, hi-lo+1) is reached with rows
// lo..i unreduced.
// ---------------------------------------------------------------------------
__device__ inline int cta_francis(const Mat& T, int m, int lo, int hi, const Mat& U, int urows, const DeflParams& dp,
                                  CtaShared* sh) {
  int i = hi;
  int itmax = 30 * max(10, hi - lo + 1);
  int total = 0;
  while (i >= lo) {
    int its = 0;
    int l;
    while (true) {
      l = cta_find_ktop(T, lo, i, dp, sh);
      if (l >= i - 1) break;
      ++its;
      ++total;
      if (total > itmax) return i + 1;
      double ssum, sprod;
      if (its % 10 == 0) {
        exceptional_pair(T, l, i, ssum, sprod);
      } else {
        double a = T(i - 1, i - 1), b = T(i - 1, i), c = T(i, i - 1), d = T(i, i);
        ssum = a + d;
        sprod = a * d - b * c;
      }
      cta_double_shift_sweep(T, m, l, i, ssum, sprod, U, urows, sh);
    }
    if (l == i) {
      i -= 1;
    } else {
      cta_standardize_block(T, i - 1, m, U, urows, sh);
      i -= 2;
    }
  }
  return 0;
}

// ---------------------------------------------------------------------------
// Swap of adjacent diagonal blocks (Bai & Demmel direct swap, cited in
// Sec. 2.5): T[j:j+p] (p x p) and the following q x q block.
// ---------------------------------------------------------------------------

// Householder vector of x (length len <= 4): (I - tau v v^T) x = beta e_1.
__device__ inline void house_small(int len, const double* x, double* v, double& tau, double& beta) {
  v[0] = 1.0;
  long long rest = 0;
  for (int t = 1; t < len; ++t) rest |= fm_abs_key(x[t]);
  if (rest == 0) {
    for (int t = 1; t < len; ++t) v[t] = 0.0;
    tau = 0.0;
    beta = x[0];
    return;
  }
  bool safe = true;
  for (int t = 0; t < len; ++t) {
    int e = fm_exponent(x[t]);
    if (fm_abs_key(x[t]) != 0 && (e <= -480 || e >= 480)) safe = false;
  }
  const bool neg = __double2hiint(x[0]) < 0;
  if (safe) {
    double a = 0.0;
    for (int t = 0; t < len; ++t) a = fma(x[t], x[t], a);
    double r = fast_rsqrt(a);
    double nrm = a * r;
    beta = neg ? nrm : -nrm;
    double d = x[0] - beta;
    double rd = fast_rcp(d);
    for (int t = 1; t < len; ++t) v[t] = x[t] * rd;
    tau = neg ? -d * r : d * r;
    return;
  }
  double sig = 0.0;
  for (int t = 1; t < len; ++t) sig = hypot(sig, x[t]);
  double nrm = hypot(x[0], sig);
  beta = neg ? nrm : -nrm;
  double d = x[0] - beta;
  for (int t = 1; t < len; ++t) v[t] = x[t] / d;
  tau = (beta - x[0]) / beta;
}

// Householder QR of the m x q matrix W (m <= 4, q <= 2); returns the m x m
// orthogonal factor in Q (column-major, leading dimension 4).
__device__ inline void small_qr_q(double W[4][2], int m, int q, double* Q) {
  for (int a = 0; a < m; ++a)
    for (int b = 0; b < m; ++b) Q[a + 4 * b] = (a == b) ? 1.0 : 0.0;
  for (int c = 0; c < q; ++c) {
    int len = m - c;
    double x[4], v[4], tau, beta;
    for (int t = 0; t < len; ++t) x[t] = W[c + t][c];
    house_small(len, x, v, tau, beta);
    if (tau == 0.0) continue;
    for (int cc = c; cc < q; ++cc) {
      double s = 0.0;
      for (int t = 0; t < len; ++t) s = fma(v[t], W[c + t][cc], s);
      s *= tau;
      for (int t = 0; t < len; ++t) W[c + t][cc] = fma(-s, v[t], W[c + t][cc]);
    }
    for (int r = 0; r < m; ++r) {
      double s = 0.0;
      for (int t = 0; t < len; ++t) s = fma(Q[r + 4 * (c + t)], v[t], s);
      s *= tau;
      for (int t = 0; t < len; ++t) Q[r + 4 * (c + t)] = fma(-s, v[t], Q[r + 4 * (c + t)]);
    }
  }
}

// Warp 0 part of the swap (all 32 lanes call it).  Lane 0 solves the
// Sylvester equation A11 X - X A22 = A12 (its Kronecker form, complete
// pivoting by magnitude keys, a pivot below sml replaced by sml as Bai &
// Demmel do for nearly equal eigenvalues) and factors [-X; I] = Q [R; 0];
// lanes (a, b) then form D = Q^T A Q in parallel, D's (2,1) block is the
// residual of the swap (accepted if <= max(10 u ||A||_F, nu n / u)) and is
// set to zero.  Two 1x1 blocks [[a, b], [0, c]] swap by the rotation whose
// first column is (b, c - a)/norm, which the Sylvester solution
// x = b / (a - c) gives; its residual is zero by construction.
// Results: sh->q (Q), sh->d (D), sh->iv[1] (1 = accepted).
__device__ inline void warp_swap_compute(const Mat& T, int nT, int j, int p, int q, CtaShared* sh) {
  const int lane = threadIdx.x & 31;
  const int m = p + q;
  double* Q = sh->q;
  double* D = sh->d;
  if (p == 1 && q == 1) {
    if (lane == 0) {
      double a = T(j, j), b = T(j, j + 1), c = T(j + 1, j + 1);
      double u0 = b, u1 = c - a;
      double cs = 1.0, sn = 0.0;
      if ((fm_abs_key(u0) | fm_abs_key(u1)) != 0) {
        if (fm_safe_range3(u0, u1, 0.0)) {
          double r = fast_rsqrt(fma(u0, u0, u1 * u1));
          cs = u0 * r;
          sn = u1 * r;
        } else {
          double r = hypot(u0, u1);
          cs = u0 / r;
          sn = u1 / r;
        }
      }
      double t00 = fma(a, cs, b * sn), t01 = fma(-a, sn, b * cs);
      double t10 = c * sn, t11 = c * cs;
      D[0] = fma(cs, t00, sn * t10);
      D[1] = 0.0;
      D[4] = fma(cs, t01, sn * t11);
      D[5] = fma(-sn, t01, cs * t11);
      Q[0] = cs; Q[1] = sn; Q[4] = -sn; Q[5] = cs;
      sh->iv[1] = 1;
    }
    return;
  }
  if (lane == 0) {
    int pq = p * q;
    double K[4][4], rhs[4];
    long long kmax = 0;
    for (int c = 0; c < q; ++c)
      for (int r = 0; r < p; ++r) {
        int row = r + c * p;
        rhs[row] = T(j + r, j + p + c);
        for (int c2 = 0; c2 < q; ++c2)
          for (int r2 = 0; r2 < p; ++r2) {
            int col = r2 + c2 * p;
            double v = ((c == c2) ? T(j + r, j + r2) : 0.0) - ((r == r2) ? T(j + p + c2, j + p + c) : 0.0);
            K[row][col] = v;
            long long kk = fm_abs_key(v);
            kmax = kk > kmax ? kk : kmax;
          }
      }
    double sml = fmax(SCHUR_U * __longlong_as_double(kmax), smlnum_of(nT));
    long long smlk = fm_abs_key(sml);
    int perm[4] = {0, 1, 2, 3};
    double inv[4];
    for (int i = 0; i < pq; ++i) {
      int br = i, bc = i;
      long long best = -1;
      for (int r = i; r < pq; ++r)
        for (int c = i; c < pq; ++c) {
          long long kk = fm_abs_key(K[r][c]);
          if (kk > best) {
            best = kk;
            br = r;
            bc = c;
          }
        }
      if (br != i) {
        for (int c = 0; c < pq; ++c) {
          double t = K[i][c]; K[i][c] = K[br][c]; K[br][c] = t;
        }
        double t = rhs[i]; rhs[i] = rhs[br]; rhs[br] = t;
      }
      if (bc != i) {
        for (int r = 0; r < pq; ++r) {
          double t = K[r][i]; K[r][i] = K[r][bc]; K[r][bc] = t;
        }
        int t = perm[i]; perm[i] = perm[bc]; perm[bc] = t;
      }
      if (best < smlk) K[i][i] = sml;
      inv[i] = fast_rcp(K[i][i]);
      for (int r = i + 1; r < pq; ++r) {
        double f = K[r][i] * inv[i];
        for (int c = i + 1; c < pq; ++c) K[r][c] = fma(-f, K[i][c], K[r][c]);
        rhs[r] = fma(-f, rhs[i], rhs[r]);
      }
    }
    double y[4], x[4];
    for (int i = pq - 1; i >= 0; --i) {
      double s = rhs[i];
      for (int c = i + 1; c < pq; ++c) s = fma(-K[i][c], y[c], s);
      y[i] = s * inv[i];
    }
    for (int i = 0; i < pq; ++i) x[perm[i]] = y[i];
    double W[4][2];
    for (int r = 0; r < m; ++r)
      for (int c = 0; c < 2; ++c) W[r][c] = 0.0;
    for (int c = 0; c < q; ++c) {
      for (int r = 0; r < p; ++r) W[r][c] = -x[r + c * p];
      W[p + c][c] = 1.0;
    }
    small_qr_q(W, m, q, Q);
  }
  __syncwarp();
  // D = Q^T A Q, one entry per lane
  const int a = lane & 3, b = lane >> 2;
  const bool mine = lane < 16 && a < m && b < m;
  double dab = 0.0, fro = 0.0;
  if (mine) {
    for (int t = 0; t < m; ++t) {
      double aq = 0.0;
      for (int s2 = 0; s2 < m; ++s2) aq = fma(T(j + t, j + s2), Q[s2 + 4 * b], aq);
      dab = fma(Q[t + 4 * a], aq, dab);
    }
    double av = T(j + a, j + b);
    fro = av * av;
  }
  double res = (mine && a >= q && b < q) ? dab * dab : 0.0;
  for (int o = 16; o > 0; o >>= 1) {
    res += __shfl_xor_sync(0xffffffffu, res, o);
    fro += __shfl_xor_sync(0xffffffffu, fro, o);
  }
  if (mine) D[a + 4 * b] = (a >= q && b < q) ? 0.0 : dab;
  if (lane == 0) {
    double tol = 10.0 * SCHUR_U;
    double sml = smlnum_of(nT);
    sh->iv[1] = (res <= fmax(tol * tol * fro, sml * sml)) ? 1 : 0;
  }
}

// Swap the adjacent blocks (sizes p, q) starting at row j of the nT x nT
// quasi-triangular T, accumulating into V (vrows x nT).  Returns false (T, V
// untouched) when the swap is rejected.  The swapped blocks are left as the
// orthogonal factor produces them (not re-standardised: callers standardise
// a block when its standard form is needed).  Two barriers: the diagonal
// block is written from D while the other threads apply Q to the rest of the
// rows (columns >= j+m), the rest of the columns (rows < j) and V.
__device__ inline bool cta_swap(const Mat& T, int nT, int j, int p, int q, const Mat& V, int vrows, CtaShared* sh) {
  if (cta_tid() < 32) warp_swap_compute(T, nT, j, p, q, sh);
  __syncthreads();
  if (sh->iv[1] == 0) {
    __syncthreads();
    return false;
  }
  const int m = p + q;
  const double* Q = sh->q;
  const int nrest_c = nT - (j + m);  // columns right of the block
  const int nrest_r = j;             // rows above the block
  const int total = nrest_c + nrest_r + vrows + 1;
  for (int it = cta_tid(); it < total; it += cta_nt()) {
    double x[4], y[4];
    if (it < nrest_c) {
      int c = j + m + it;
      for (int t = 0; t < m; ++t) x[t] = T(j + t, c);
      for (int a = 0; a < m; ++a) {
        double s = 0.0;
        for (int t = 0; t < m; ++t) s += Q[t + 4 * a] * x[t];
        y[a] = s;
      }
      for (int t = 0; t < m; ++t) T(j + t, c) = y[t];
    } else if (it < nrest_c + nrest_r) {
      int r = it - nrest_c;
      for (int t = 0; t < m; ++t) x[t] = T(r, j + t);
      for (int b = 0; b < m; ++b) {
        double s = 0.0;
        for (int t = 0; t < m; ++t) s += x[t] * Q[t + 4 * b];
        y[b] = s;
      }
      for (int t = 0; t < m; ++t) T(r, j + t) = y[t];
    } else if (it < nrest_c + nrest_r + vrows) {
      int r = it - nrest_c - nrest_r;
      for (int t = 0; t < m; ++t) x[t] = V(r, j + t);
      for (int b = 0; b < m; ++b) {
        double s = 0.0;
        for (int t = 0; t < m; ++t) s += x[t] * Q[t + 4 * b];
        y[b] = s;
      }
      for (int t = 0; t < m; ++t) V(r, j + t) = y[t];
    } else {
      for (int a = 0; a < m; ++a)
        for (int b = 0; b < m; ++b) T(j + a, j + b) = sh->d[a + 4 * b];
    }
  }
  __syncthreads();
  return true;
}

// Move the block of size p starting at ifst up to start at ilst (a block
// boundary) by adjacent swaps; false if a swap was rejected.
__device__ inline bool cta_move_block_up(const Mat& T, int nT, int ifst, int ilst, int p, const Mat& V, int vrows,
                                         CtaShared* sh) {
  int here = ifst;
  while (here > ilst) {
    int q = (here >= 2 && here - 2 >= ilst && T(here - 1, here - 2) != 0.0) ? 2 : 1;
    if (!cta_swap(T, nT, here - q, q, p, V, vrows, sh)) return false;
    here -= q;
  }
  return true;
}

// ---------------------------------------------------------------------------
// Householder reflector of arbitrary length from x (contiguous, length len),
// v written to vbuf (v[0] = 1); tau, beta returned (uniform).
// ---------------------------------------------------------------------------
__device__ inline void cta_house_vec(const double* x, int len, double* vbuf, double& tau, double& beta,
                                     CtaShared* sh) {
  // scaled 2-norm of x[1:]
  double mx = 0.0;
  for (int t = 1 + cta_tid(); t < len; t += cta_nt()) mx = fmax(mx, fabs(x[t]));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((cta_tid() & 31) == 0) sh->red[cta_tid() >> 5] = mx;
  __syncthreads();
  if (cta_tid() == 0) {
    double m = 0.0;
    for (int w = 0; w < (cta_nt() + 31) / 32; ++w) m = fmax(m, sh->red[w]);
    sh->r[6] = m;
  }
  __syncthreads();
  double scale = sh->r[6];
  double ss = 0.0;
  if (scale > 0.0) {
    double rsc = fast_rcp(scale);
    for (int t = 1 + cta_tid(); t < len; t += cta_nt()) {
      double z = x[t] * rsc;
      ss = fma(z, z, ss);
    }
  }
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  __syncthreads();
  if ((cta_tid() & 31) == 0) sh->red[cta_tid() >> 5] = ss;
  __syncthreads();
  if (cta_tid() == 0) {
    double s = 0.0;
    for (int w = 0; w < (cta_nt() + 31) / 32; ++w) s += sh->red[w];
    double alpha = x[0];
    if (scale == 0.0 || s == 0.0) {
      sh->r[6] = 0.0;   // tau
      sh->r[7] = alpha; // beta
      sh->r[5] = 0.0;
    } else {
      double sig = scale * sqrt(s);
      double b = -copysign(hypot(alpha, sig), alpha);
      sh->r[6] = (b - alpha) / b;
      sh->r[7] = b;
      sh->r[5] = 1.0 / (alpha - b);   // reciprocal of the scaling denominator
    }
  }
  __syncthreads();
  tau = sh->r[6];
  beta = sh->r[7];
  double rden = sh->r[5];
  for (int t = cta_tid(); t < len; t += cta_nt()) vbuf[t] = (t == 0) ? 1.0 : ((tau == 0.0) ? 0.0 : x[t] * rden);
  __syncthreads();
}

// X[r0:r0+len, c0:c1] <- (I - tau v v^T) X
__device__ inline void cta_house_left(const Mat& M, const double* v, int len, double tau, int r0, int c0, int c1) {
  if (tau == 0.0) return;
  for (int c = c0 + cta_tid(); c <= c1; c += cta_nt()) {
    double* col = &M(r0, c);
    double s = 0.0;
    for (int t = 0; t < len; ++t) s += v[t] * col[t];
    s *= tau;
    for (int t = 0; t < len; ++t) col[t] -= s * v[t];
  }
}

// X[rlo:rhi+1, c0:c0+len] <- X (I - tau v v^T)
__device__ inline void cta_house_right(const Mat& M, const double* v, int len, double tau, int c0, int rlo, int rhi) {
  if (tau == 0.0) return;
  for (int r = rlo + cta_tid(); r <= rhi; r += cta_nt()) {
    double s = 0.0;
    for (int t = 0; t < len; ++t) s += M(r, c0 + t) * v[t];
    s *= tau;
    for (int t = 0; t < len; ++t) M(r, c0 + t) -= s * v[t];
  }
}

// ---------------------------------------------------------------------------
// AED steps 2 and 3 (Sec. 2.5) on a window T (nw x nw) already in Schur form
// (rows 0..info-1 possibly unconverged), with V the accumulated transform and
// s = h_{kwtop, kwtop-1}.  Deflation checks bottom-up, failed blocks moved to
// the top of the unevaluated part (halt on a rejected swap), candidates
// written top to bottom, and -- if something deflated -- the spike of the
// undeflated part reflected onto its first entry and that part returned to
// Hessenberg form.  Returns nd; *top receives the new h_{kwtop, kwtop-1}.
// vbuf: scratch of length >= nw.
// ---------------------------------------------------------------------------
__device__ inline int cta_aed_post(const Mat& T, int nw, int info, double s, const Mat& V, const DeflParams& dp,
                                   double* vbuf, double* cand_re, double* cand_im, int* ncand_out, double* top_out,
                                   int* swap_fail_out, CtaShared* sh, long long* cyc = nullptr) {
  long long c0 = clock64();
  int ns = nw;
  int ilst = info;
  int failed = 0;
  for (int guard = 0; guard < 2 * nw + 2 && ilst < ns; ++guard) {
    // the bottom 2x2 block is put in standard form before it is tested
    // (swaps leave moved blocks unstandardised)
    if (ns >= 2 && T(ns - 1, ns - 2) != 0.0) cta_standardize_block(T, ns - 2, nw, V, nw, sh);
    // decision by thread 0
    if (cta_tid() == 0) {
      int bs = (ns >= 2 && T(ns - 1, ns - 2) != 0.0) ? 2 : 1;
      double spj = s * V(0, ns - 1);
      double spm = (bs == 2) ? s * V(0, ns - 2) : 0.0;
      bool defl = spike_deflatable(T, spj, spm, ns - 1, bs, dp);
      sh->iv[2] = bs;
      sh->iv[3] = defl ? 1 : 0;
    }
    __syncthreads();
    int bs = sh->iv[2];
    bool defl = sh->iv[3] != 0;
    __syncthreads();
    if (defl) {
      ns -= bs;
      continue;
    }
    if (!cta_move_block_up(T, nw, ns - bs, ilst, bs, V, nw, sh)) {
      failed = 1;
      break;
    }
    ilst += bs;
  }
  int nd = nw - ns;
  long long c1 = clock64();
  // candidates of the undeflated part (converged rows info..ns-1)
  if (cta_tid() == 0) {
    int c = 0;
    int j = info;
    while (j < ns) {
      if (j + 1 < ns && T(j + 1, j) != 0.0) {
        double r1, i1, r2, i2;
        eig2x2(T(j, j), T(j, j + 1), T(j + 1, j), T(j + 1, j + 1), r1, i1, r2, i2);
        cand_re[c] = r1; cand_im[c] = i1; ++c;
        cand_re[c] = r2; cand_im[c] = i2; ++c;
        j += 2;
      } else {
        cand_re[c] = T(j, j);
        cand_im[c] = 0.0;
        ++c;
        j += 1;
      }
    }
    *ncand_out = c;
    *swap_fail_out = failed;
  }
  __syncthreads();
  double top = 0.0;
  if (nd > 0 && ns >= 1) {
    if (ns == 1) {
      top = s * V(0, 0);
    } else if (s != 0.0) {
      // reflect the spike s * V(0, 0:ns) onto e_1
      for (int t = cta_tid(); t < ns; t += cta_nt()) vbuf[nw + t] = s * V(0, t);
      __syncthreads();
      double tau, beta;
      cta_house_vec(vbuf + nw, ns, vbuf, tau, beta, sh);
      cta_house_left(T, vbuf, ns, tau, 0, 0, nw - 1);
      __syncthreads();
      cta_house_right(T, vbuf, ns, tau, 0, 0, ns - 1);
      cta_house_right(V, vbuf, ns, tau, 0, 0, nw - 1);
      __syncthreads();
      top = beta;
      // Householder Hessenberg reduction of T[0:ns, 0:ns]
      for (int j = 0; j < ns - 2; ++j) {
        int len = ns - j - 1;
        double tj, bj;
        cta_house_vec(&T(j + 1, j), len, vbuf, tj, bj, sh);
        cta_house_left(T, vbuf, len, tj, j + 1, j + 1, nw - 1);
        __syncthreads();
        cta_house_right(T, vbuf, len, tj, j + 1, 0, ns - 1);
        cta_house_right(V, vbuf, len, tj, j + 1, 0, nw - 1);
        __syncthreads();
        if (cta_tid() == 0) {
          T(j + 1, j) = bj;
          for (int t = j + 2; t < ns; ++t) T(t, j) = 0.0;
        }
        __syncthreads();
      }
    }
  }
  *top_out = top;
  if (cyc && cta_tid() == 0) {
    cyc[0] += c1 - c0;
    cyc[1] += clock64() - c1;
  }
  return nd;
}

// ---------------------------------------------------------------------------
// Shift pairs for the next sweep (one thread).  Reading of Sec. 2.5: the
// undeflated AED candidates become the shifts -- the bottom-most ones, complex
// conjugates kept together, real shifts paired in order of appearance; an
// exceptional pair every exc_period-th iteration without deflation
// (ndfl % exc_period == 0); the trailing 2x2 when no candidate is left.
// Writes (sum, product) pairs and returns their count (at most
// min(ns_max, m - 1) / 2 for the active block [ktop, kbot] of m rows).
// ---------------------------------------------------------------------------
__device__ inline int make_shift_pairs(const Mat& H, int ktop, int kbot, int ns_max, int ndfl, int exc_period,
                                       const double* cand_re, const double* cand_im, int ncand, double* pairs) {
  int m = kbot - ktop + 1;
  int ns = min(ns_max, m - 1);
  ns -= ns % 2;
  int want = ns / 2;
  int np = 0;
  if (m < 3 || want <= 0) return 0;
  if (ndfl % exc_period == 0) {
    for (int i = kbot; np < want && i > ktop; i -= 2) {
      double ss, sp;
      exceptional_pair(H, ktop, i, ss, sp);
      pairs[2 * np] = ss;
      pairs[2 * np + 1] = sp;
      ++np;
    }
    return np;
  }
  bool pending = false;
  double pv = 0.0;
  int i = ncand - 1;
  while (i >= 0 && np < want) {
    double re = cand_re[i], im = cand_im[i];
    if (im != 0.0) {
      pairs[2 * np] = 2.0 * re;
      pairs[2 * np + 1] = re * re + im * im;
      ++np;
      i -= 2;
      continue;
    }
    if (!pending) {
      pending = true;
      pv = re;
    } else {
      pairs[2 * np] = pv + re;
      pairs[2 * np + 1] = pv * re;
      ++np;
      pending = false;
    }
    i -= 1;
  }
  if (np == 0) {
    double a = H(kbot - 1, kbot - 1), b = H(kbot - 1, kbot), c = H(kbot, kbot - 1), d = H(kbot, kbot);
    pairs[0] = a + d;
    pairs[1] = a * d - b * c;
    np = 1;
  }
  return np;
}
