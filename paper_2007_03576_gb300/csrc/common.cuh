// common.cuh -- shared definitions of the GB300 FP64 multishift QR library.
//
// Host/device structures, constants and scalar device helpers: Householder
// reflectors of order 2/3 (the 3x3 reflectors of Sec. 2.2), 2x2 eigenvalues
// and standardisation (eq. 2by2_blocks), and the deflation conditions of
// Sec. 5.6.  All arithmetic is IEEE FP64.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fastmath.cuh"

#define SCHUR_U (2.220446049250313080847e-16)     /* u = 2^-52, Sec. 5.4 */
#define SCHUR_NU (2.225073858507201383090e-308)   /* nu = DBL_MIN, Sec. 5.6 */

// Bounds of the one-block kernels.
#define CTA_THREADS 256
#define CHASE_THREADS 512    // threads of a bulge-chase block (one warp per bulge or two)
#define KWIN_MAX 112         // largest bulge-chase window (window + U in shared memory: 2 (k+1) k doubles)
#define NW_SMEM_MAX 160      // AED windows / small blocks held in shared memory
#define MAX_CHAINS 32        // bulge chains chased concurrently in one launch
#define MAX_BULGES_PER_CHAIN 32
#define MAX_UPD_TASKS (3 * MAX_CHAINS + 4)
// doubles per chase window in the U buffers: U (kwin x kwin) followed by the
// row range of U's nonzeros in each column (kwin int2)
#define CHASE_USLOT(kwin) ((kwin) * (kwin) + (kwin))

struct DeflParams {
  int mode;        // 0 lapack, 1 norm, 2 fixed
  double thold;    // fixed threshold
  double normH;    // ||H||_F of the input (norm-stable mode)
  int n;           // order used in nu * n / u
};

// Control block written by the device, mirrored to pinned host memory once
// per iteration of the driver.
struct Ctl {
  int ktop;      // start of the bottom unreduced block (scan)
  int nd;        // eigenvalues deflated by the last AED
  int ncand;     // undeflated AED candidates
  int npairs;    // shift pairs prepared for the next sweep
  int ndfl;      // iterations since the last deflation (exceptional shifts)
  int info;      // nonzero: small-QR / window-QR iteration limit
  int swap_fail; // a reordering swap was rejected in the last AED
  int nswaps;    // swaps performed by the last AED
  long long cyc_schur, cyc_defl, cyc_hess;  // clock64 cycles of the AED sub-steps (accumulated)
  int sync_err;  // the AED kernel's two blocks lost contact (a bounded wait ran out)
  int recomputed;  // shift recomputations after AED (accumulated)
};

// One bulge chain in one launch of the chase kernel (Sec. 2.3 / 2.4: a set of
// tightly-coupled bulges moved through one diagonal window).
struct ChainDesc {
  int ws, we;      // window rows/cols ws..we (inclusive, global indices)
  int tau0, tau1;  // chain-local steps processed: [tau0, tau1)
  int pair0;       // index of this chain's first shift pair
  int nb;          // bulges in the chain
  int uoff;        // offset (doubles) of this window's U in the U buffer
  int pad;
};

struct ChaseArgs {
  int nchain;
  int lo, hi;      // active block
  int ldu;         // leading dimension of every U
  ChainDesc c[MAX_CHAINS];
};

// One off-window product (Sec. 3.2.1): side 0 -> X <- U^T X on the column
// vectors of X (X = A[r0:r0+L, c0:c0+nvec]); side 1 -> X <- X U on the row
// vectors of X (X = A[r0:r0+nvec, c0:c0+L]).
struct UpdTask {
  double* A;
  const double* U;
  long long lda;
  int ldu;
  int side;
  int r0, c0;
  int L;       // order of U
  int nvec;    // vectors (columns for side 0, rows for side 1)
  int tile0;   // first tile index of this task in the launch
  int ntile;
  const int* gate;  // optional: skip when *gate == 0 (e.g. AED deflated nothing)
  int lbw, ubw;     // U[k, i] = 0 when k - i > lbw or i - k > ubw (L = dense)
  const int2* rng;  // optional (device): U[k, i] = 0 unless rng[i].x <= k <= rng[i].y
  const int2* hrng; // the same ranges on the host (executed-flop count); nullptr = none
};

struct UpdArgs {
  int ntask;
  int tn;      // vectors per tile
  UpdTask t[MAX_UPD_TASKS];
};

#ifdef __CUDACC__

struct Mat {
  double* p;
  long long ld;
  __device__ __forceinline__ double& operator()(int i, int j) const { return p[i + (long long)j * ld]; }
};

__device__ __forceinline__ double smlnum_of(int n) { return SCHUR_NU * ((double)n / SCHUR_U); }

// Householder reflector (I - tau v v^T), v = (1, v1, v2) (v2 = 0 when nr == 2),
// with (I - tau v v^T) x = beta e_1, beta = -sign(x0) ||x||.
//
// This is the innermost link of every serial chain of the method (the next
// reflector of a bulge depends on the previous one), so it is arranged for
// the fewest dependent FP64 operations.  With r = 1/||x||:
//   tau = (beta - x0) / beta = 1 + |x0| r,  in [1, 2];
//   v_i = x_i / (x0 - beta) = sign(x0) x_i r / tau;
// so one reciprocal square root (of ||x||^2) and one reciprocal of tau are
// needed.  The FP32 seed of 1/tau is formed from the FP32 seed of r beside
// the FP64 chain, and both are refined by one third-order Newton step
// (fastmath.cuh): 12 dependent FP64 operations in all.  The magnitude tests
// are integer operations, evaluated beside the chain; operands whose squares
// could overflow or underflow take the hypot path afterwards.
__device__ __forceinline__ void house3(int nr, double x0, double x1, double x2, double& v1, double& v2,
                                       double& tau, double& beta) {
  if (nr < 3) x2 = 0.0;
  const bool trivial = nr < 2 || (fm_abs_key(x1) | fm_abs_key(x2)) == 0;
  const bool safe = fm_safe_range3(x0, x1, x2);
  const int h0 = __double2hiint(x0);
  const double ax0 = fabs(x0);
  const double a = fma(x0, x0, fma(x1, x1, x2 * x2));
  const int ha = __double2hiint(a);
  const int e = ((ha >> 20) & 0x7ff) - 1023;
  const int k = e >> 1;
  // FP32 seed of (a 2^-2k)^(-1/2), and of 1/tau from |x0| 2^-k in FP32
  const float sf = fm_rsqrt_approx_f32(fm_mantissa_f32(ha, __double2loint(a), e & 1));
  const double y = fm_f32_to_f64_scaled(sf, -k);
  const int e0 = ((h0 >> 20) & 0x7ff) - 1023 - k;
  const float x0f = (e0 < -126 || (fm_abs_key(x0) == 0))
                        ? 0.0f
                        : __uint_as_float(((unsigned)(e0 + 127) << 23) | (((unsigned)h0 & 0xfffffu) << 3) |
                                          ((unsigned)__double2loint(x0) >> 29));
  const float rtf = fm_rcp_approx_f32(fmaf(x0f, sf, 1.0f));
  // r = a^(-1/2): one third-order step
  const double ay = a * y;
  const double ee = fma(-ay, y, 1.0);
  const double ye = y * ee;
  const double pp = fma(0.375, ee, 0.5);
  const double r = fma(ye, pp, y);
  tau = fma(ax0, r, 1.0);
  const double rs = copysign(r, x0);
  const double xr1 = x1 * rs, xr2 = x2 * rs;
  beta = -copysign(a * r, x0);
  // 1/tau, tau in [1, 2]: one third-order step from the FP32 seed
  double z = fm_f32_to_f64_scaled(rtf, 0);
  const double et = fma(-tau, z, 1.0);
  const double pt = fma(et, et, et);
  z = fma(z, pt, z);
  v1 = xr1 * z;
  v2 = xr2 * z;
  if (trivial) {
    v1 = 0.0;
    v2 = 0.0;
    tau = 0.0;
    beta = x0;
  } else if (!safe) {
    double sig = hypot(x1, x2);
    double nrm = hypot(x0, sig);
    beta = -copysign(nrm, x0);
    tau = (beta - x0) / beta;
    double den = x0 - beta;
    v1 = x1 / den;
    v2 = x2 / den;
  }
}

// Eigenvalues of [[a, b], [c, d]]; for a complex pair im1 > 0.
__device__ __forceinline__ void eig2x2(double a, double b, double c, double d, double& re1, double& im1,
                                       double& re2, double& im2) {
  double p = 0.5 * (a - d);
  double disc = p * p + b * c;
  double mid = 0.5 * (a + d);
  if (disc >= 0.0) {
    double r = sqrt(disc);
    re1 = mid + r;
    re2 = mid - r;
    im1 = im2 = 0.0;
  } else {
    double r = sqrt(-disc);
    re1 = re2 = mid;
    im1 = r;
    im2 = -r;
  }
}

// Rotation G = [[cs, -sn], [sn, cs]] with G^T A G in standard form
// (eq. 2by2_blocks): complex pair -> equal diagonal, b'c' < 0; real
// eigenvalues -> c' = 0.  Real case: G e_1 is a unit eigenvector of the
// eigenvalue (a+d)/2 + sign(a-d) r.  Complex case: the diagonal difference
// of G^T A G is (a-d) cos 2t + (b+c) sin 2t, zero for
// (cos 2t, sin 2t) = (|b+c|, -sign(b+c) (a-d)) / rho, rho = ||(a-d, b+c)||
// (the root with cos 2t >= 0), and cos t = sqrt((1 + cos 2t)/2),
// sin t = sin 2t / (2 cos t).  Writes the new block to B[4] = a', b', c', d'.
__device__ inline void standardize2x2(double a, double b, double c, double d, double& cs, double& sn, double* B) {
  if (fm_abs_key(c) == 0) {
    cs = 1.0;
    sn = 0.0;
    B[0] = a; B[1] = b; B[2] = 0.0; B[3] = d;
    return;
  }
  for (int pass = 0; pass < 2; ++pass) {
    double p = 0.5 * (a - d);
    double disc = fma(p, p, b * c);
    bool real = __double2hiint(disc) >= 0;
    double c1 = 1.0, s1 = 0.0;
    if (real) {
      double r = (fm_abs_key(disc) == 0) ? 0.0 : disc * fast_rsqrt(disc);
      double z = p + copysign(r, p);
      double lam1 = d + z;
      double u0 = z, u1 = c, w0 = b, w1 = lam1 - a;
      if (fabs(u0) + fabs(u1) < fabs(w0) + fabs(w1)) { u0 = w0; u1 = w1; }
      if (fm_safe_range3(u0, u1, 0.0)) {
        double rn = fast_rsqrt(fma(u0, u0, u1 * u1));
        c1 = u0 * rn;
        s1 = u1 * rn;
      } else {
        double nrm = hypot(u0, u1);
        c1 = u0 / nrm;
        s1 = u1 / nrm;
      }
    } else {
      double am = a - d, bp = b + c;
      double rho2 = fma(am, am, bp * bp);
      if (fm_abs_key(rho2) != 0 && fm_safe_range3(am, bp, 0.0)) {
        double rr = fast_rsqrt(rho2);
        double c2 = fabs(bp) * rr;
        double s2 = (__double2hiint(bp) < 0 ? am : -am) * rr;
        double h = 0.5 * (1.0 + c2);
        double rs = fast_rsqrt(h);
        c1 = h * rs;
        s1 = 0.5 * s2 * rs;
      } else if (fm_abs_key(rho2) != 0) {
        double t = 0.5 * atan2(-(a - d), b + c);
        c1 = cos(t);
        s1 = sin(t);
      }
    }
    // B = G^T A G
    double t00 = a * c1 + b * s1, t01 = -a * s1 + b * c1;
    double t10 = c * c1 + d * s1, t11 = -c * s1 + d * c1;
    double na = c1 * t00 + s1 * t10, nb = c1 * t01 + s1 * t11;
    double nc = -s1 * t00 + c1 * t10, nd = -s1 * t01 + c1 * t11;
    if (pass == 0) {
      cs = c1;
      sn = s1;
    } else {
      double cc = cs * c1 - sn * s1, ss = sn * c1 + cs * s1;
      cs = cc;
      sn = ss;
    }
    if (real) {
      B[0] = na; B[1] = nb; B[2] = 0.0; B[3] = nd;
      return;
    }
    double m = 0.5 * (na + nd);
    if (nb * nc < 0.0) {
      B[0] = m; B[1] = nb; B[2] = nc; B[3] = m;
      return;
    }
    // rounding made the pair real: triangularise the rotated block
    a = m; b = nb; c = nc; d = m;
    if (fm_abs_key(c) == 0) {
      B[0] = a; B[1] = b; B[2] = 0.0; B[3] = d;
      return;
    }
  }
}

// Vigilant-deflation test of H(k, k-1) inside the block [lo, hi]
// (Sec. 2.1 / Sec. 5.6; LAPACK-style mode: below u (|h_{k-1,k-1}| + |h_kk|)
// and the Ahues-Tisseur refinement).
__device__ inline bool subdiag_negligible(const Mat& H, int k, int lo, int hi, const DeflParams& dp) {
  double h21 = fabs(H(k, k - 1));
  if (dp.mode == 1) return h21 <= SCHUR_U * dp.normH;
  if (dp.mode == 2) return h21 <= dp.thold;
  double sml = smlnum_of(dp.n);
  if (h21 <= sml) return true;
  double tst = fabs(H(k - 1, k - 1)) + fabs(H(k, k));
  if (tst == 0.0) {
    if (k - 2 >= lo) tst += fabs(H(k - 1, k - 2));
    if (k + 1 <= hi) tst += fabs(H(k + 1, k));
  }
  if (h21 > SCHUR_U * tst) return false;
  double h12 = fabs(H(k - 1, k));
  double dd = fabs(H(k - 1, k - 1) - H(k, k));
  double h22 = fabs(H(k, k));
  double ab = fmax(h21, h12), ba = fmin(h21, h12);
  double aa = fmax(h22, dd), bb = fmin(h22, dd);
  double rs = fast_rcp(aa + ab);
  return ba * (ab * rs) <= fmax(sml, SCHUR_U * (bb * (aa * rs)));
}

// AED deflation test (Sec. 5.6) of a diagonal block of size bs, given by
// its entries [[a, b], [c, d]] (bs == 2) or d (bs == 1), against the spike
// entries sp_j of its last row (and sp_{j-1} of the row above for bs == 2).
__device__ inline bool spike_deflatable_blk(double a, double b, double c, double d, double spj, double spjm1, int bs,
                                            const DeflParams& dp) {
  double s = (bs == 1) ? fabs(spj) : fmax(fabs(spj), fabs(spjm1));
  if (dp.mode == 1) return s <= SCHUR_U * dp.normH;
  if (dp.mode == 2) return s <= dp.thold;
  if (bs == 1) return s <= fmax(smlnum_of(dp.n), SCHUR_U * fabs(d));
  double hhat = sqrt(fabs(d * a)) + sqrt(fabs(b * c));
  return s <= fmax(smlnum_of(dp.n), SCHUR_U * hhat);
}

// The same test for the block of T ending at row j.
__device__ inline bool spike_deflatable(const Mat& T, double spj, double spjm1, int j, int bs, const DeflParams& dp) {
  if (bs == 1) return spike_deflatable_blk(0.0, 0.0, 0.0, T(j, j), spj, spjm1, 1, dp);
  return spike_deflatable_blk(T(j - 1, j - 1), T(j - 1, j), T(j, j - 1), T(j, j), spj, spjm1, 2, dp);
}

#endif  // __CUDACC__
