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
  double red[32];    // block reductions
  int iv[8];         // integer broadcast
};

__device__ __forceinline__ int cta_tid() { return threadIdx.x; }
__device__ __forceinline__ int cta_nt() { return blockDim.x; }

// ---------------------------------------------------------------------------
// Transform stream between the two blocks of a cluster.
//
// The window Schur form of AED accumulates its reflectors and rotations into
// V, which the Francis chain never reads.  In the AED kernel block 0 reduces
// the window and pushes every transform, in order, through distributed
// shared memory to block 1, which keeps V in its own shared memory and
// applies them there.  A ring of VRING_OPS slots in block 1 holds the
// transforms; block 0 publishes how many it wrote (release store at cluster
// scope) and block 1 how many it applied, which block 0 waits for before it
// reuses a slot.  Every wait gives up after VRING_TIMEOUT cycles and sets
// err; both blocks meet at a cluster barrier after the exchange, so neither
// touches the other's shared memory after the other has left.
// ---------------------------------------------------------------------------
#define VRING_OPS 256
#define VRING_TIMEOUT 4000000000LL   // SM cycles (about 2 s)

struct VOp {
  double a, b, c;   // reflector: v1, v2, tau; rotation: cs, sn
  int k;            // first column
  int kind;         // 2 or 3: reflector of that order; 1: rotation; 0: end
};

struct VRing {
  VOp ops[VRING_OPS];   // consumer: the transforms
  unsigned count;       // consumer: transforms published
  unsigned consumed;    // producer: transforms the consumer has applied
  unsigned pushed;      // producer: transforms pushed so far (one thread)
  int err;              // a wait timed out
  VRing* remote;        // the other block's ring (generic address)
};

__device__ __forceinline__ unsigned vr_ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.cluster.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void vr_st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.cluster.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Called by one thread of the producer block, in transform order.
__device__ inline void vring_push(VRing* r, double a, double b, double c, int k, int kind) {
  const unsigned q = r->pushed;
  r->pushed = q + 1;
  if (r->err) return;
  if (q >= VRING_OPS) {
    const long long t0 = clock64();
    while (vr_ld_acquire(&r->consumed) + VRING_OPS <= q) {
      if (clock64() - t0 > VRING_TIMEOUT) {
        r->err = 1;
        return;
      }
    }
  }
  VOp* d = &r->remote->ops[q % VRING_OPS];
  d->a = a;
  d->b = b;
  d->c = c;
  d->k = k;
  d->kind = kind;
  vr_st_release(&r->remote->count, q + 1);
}

// The consumer block: applies the stream to the rows 0..nrows-1 of V (one
// thread per row) until the end mark; returns 1 if a wait timed out.
__device__ inline int vring_consume(VRing* r, const Mat& V, int nrows) {
  __shared__ unsigned s_avail;
  const int tid = threadIdx.x;
  unsigned done = 0;
  int ended = 0, timed_out = 0;
  while (!ended) {
    if (tid == 0) {
      const long long t0 = clock64();
      unsigned c;
      while ((c = vr_ld_acquire(&r->count)) == done) {
        if (clock64() - t0 > VRING_TIMEOUT) break;
      }
      s_avail = c;
    }
    __syncthreads();
    const unsigned c = s_avail;
    if (c == done) {   // timed out (uniform: every thread reads s_avail)
      timed_out = 1;
      break;
    }
    unsigned q = done;
    for (; q < c; ++q) {
      const VOp op = r->ops[q % VRING_OPS];
      if (op.kind == 0) {
        ended = 1;
        break;
      }
      if (tid < nrows) {
        double* row = &V(tid, op.k);
        const long long ld = V.ld;
        if (op.kind == 1) {
          const double x = row[0], y = row[ld];
          row[0] = op.a * x + op.b * y;
          row[ld] = -op.b * x + op.a * y;
        } else {
          const double x0 = row[0], x1 = row[ld], x2 = (op.kind == 3) ? row[2 * ld] : 0.0;
          const double s = op.c * fma(op.b, x2, fma(op.a, x1, x0));
          row[0] = x0 - s;
          row[ld] = fma(-s, op.a, x1);
          if (op.kind == 3) row[2 * ld] = fma(-s, op.b, x2);
        }
      }
    }
    done = ended ? q + 1 : c;
    __syncthreads();   // every thread is done with the slots read above
    if (tid == 0) vr_st_release(&r->remote->consumed, done);
  }
  return timed_out;
}

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
                                             CtaShared* sh, VRing* ring = nullptr) {
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
  if (ring && cta_tid() == 128 && !(cs == 1.0 && sn == 0.0)) vring_push(ring, cs, sn, 0.0, k, 1);
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
//
// The sweep is a chain: the reflector P_{k+1} is built from column k of
// P_k T P_k, so the time of a step is the length of that chain.  On this GPU
// a dependent FP64 operation costs ~64 cycles, and a sub-partition of the SM
// issues one FP64 warp instruction per ~64 cycles whatever the number of
// active lanes; so the chain runs alone on one lane of warp 0, whose
// sub-partition does no other FP64 work, and it touches no other data than a
// register copy of the 4 x 3 block B_k = T[k..k+3, k..k+2]:
//   y  = column k of B_k P_k  (rows k..k+3),
//   x  = rows k+1..k+3 of P_k y  (6 dependent operations in all),
//   P_{k+1} = house3(x).
// Beside it, per step (one barrier per step):
//   - warp 1 applies P_k to the diagonal block T[k..k+3, k..k+3] (left
//     product on rows k..k+2, then right product on columns k..k+2, so every
//     entry receives the same operations in the same order as with the left
//     product applied first), writes it back, and hands B_{k+1} to the chain
//     lane through a double buffer;
//   - the warps of the other three sub-partitions apply P_k to the rest of
//     rows k..k+2 (columns k+4..m-1), of columns k..k+2 (rows 0..k-1) and
//     to U.
// These regions are disjoint; the chain lane writes the new column k
// (beta, 0, 0) below the diagonal itself.  Reflectors alternate between two
// slots of sh->r.
// ---------------------------------------------------------------------------
// The next reflector of the Francis chain on the lanes of one warp.
//
// Each sub-partition of the SM issues one FP64 warp instruction per ~64
// cycles whatever the number of active lanes, so a chain of scalar FP64
// operations costs 64 cycles per instruction, even when some of them are
// independent.  Independent operations are therefore put in different
// lanes of the same instruction, and values move between lanes by shuffles
// (not on the FP64 unit):
//   - lane r (< 4) holds row r of B = T[k..k+3, k..k+2] and computes
//     y_r = (B P)(r, 0) (3 instructions for the four rows);
//   - x = rows 1..3 of P y: q = w^T y, x_r = y_r - (tau q) w_r (4);
//   - house3 of x: ||x||^2 (3), a^(-1/2) by one third-order step from an
//     integer-built seed (4, the two middle products in two lanes), then
//     tau = 1 + |x0| r, ||x|| = a r, x1 r and x2 r in four lanes of one
//     instruction (1), 1/tau by one third-order step from an FP32 seed formed
//     beside the chain (3), and v1, v2 in two lanes (1).
// 20 FP64 instructions, against ~40 for the scalar evaluation.  The result
// is the reflector of house3 (same formulas), up to rounding.  Every lane of
// the warp executes the same instructions; all lanes return (v1, v2, tau,
// beta).  b0, b1, b2: this lane's row of B (lanes >= 4: anything finite).
__device__ __forceinline__ double warp_bcast(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }

__device__ __forceinline__ void warp_next_reflector(double b0, double b1, double b2, double v1, double v2, double tau,
                                                    int nr1, double& ov1, double& ov2, double& otau, double& obeta) {
  const int lane = threadIdx.x & 31;
  // y = column 0 of B P
  const double in = fma(v2, b2, fma(v1, b1, b0));
  const double y = fma(-tau, in, b0);
  const double y0 = warp_bcast(y, 0), y1 = warp_bcast(y, 1), y2 = warp_bcast(y, 2);
  // x = rows 1..3 of P y (row 3 unchanged by the left product)
  const double q = fma(v2, y2, fma(v1, y1, y0));
  const double tq = tau * q;
  const double w = (lane == 1) ? v1 : ((lane == 2) ? v2 : 0.0);
  const double xl = fma(-tq, w, y);
  const double x0 = warp_bcast(xl, 1), x1 = warp_bcast(xl, 2);
  const double x2 = (nr1 == 3) ? warp_bcast(xl, 3) : 0.0;
  // house3(x)
  const bool trivial = (fm_abs_key(x1) | fm_abs_key(x2)) == 0;
  const bool safe = fm_safe_range3(x0, x1, x2);
  const int h0 = __double2hiint(x0);
  const double a = fma(x0, x0, fma(x1, x1, x2 * x2));
  const int ha = __double2hiint(a);
  const int e = ((ha >> 20) & 0x7ff) - 1023;
  const int k = e >> 1;
  const float sf = fm_rsqrt_approx_f32(fm_mantissa_f32(ha, __double2loint(a), e & 1));
  const double ys = fm_f32_to_f64_scaled(sf, -k);
  const int e0 = ((h0 >> 20) & 0x7ff) - 1023 - k;
  const float x0f = (e0 < -126 || (fm_abs_key(x0) == 0))
                        ? 0.0f
                        : __uint_as_float(((unsigned)(e0 + 127) << 23) | (((unsigned)h0 & 0xfffffu) << 3) |
                                          ((unsigned)__double2loint(x0) >> 29));
  const float rtf = fm_rcp_approx_f32(fmaf(x0f, sf, 1.0f));
  const double ay = a * ys;
  const double ee = fma(-ay, ys, 1.0);
  // lane 0: y e; lane 1: 3/8 e + 1/2
  const double t = fma((lane == 1) ? 0.375 : ys, ee, (lane == 1) ? 0.5 : 0.0);
  const double ye = warp_bcast(t, 0), pp = warp_bcast(t, 1);
  const double r = fma(ye, pp, ys);
  const double rs = copysign(r, x0);
  // lane 0: tau = 1 + |x0| r; lane 1: ||x|| = a r; lane 2: x1 r; lane 3: x2 r (signed)
  const double m1 = (lane == 0) ? fabs(x0) : ((lane == 1) ? a : ((lane == 2) ? x1 : x2));
  const double m2 = (lane <= 1) ? r : rs;
  const double u = fma(m1, m2, (lane == 0) ? 1.0 : 0.0);
  const double tv = warp_bcast(u, 0), nrm = warp_bcast(u, 1), xr1 = warp_bcast(u, 2), xr2 = warp_bcast(u, 3);
  double z = fm_f32_to_f64_scaled(rtf, 0);
  const double et = fma(-tv, z, 1.0);
  const double pt = fma(et, et, et);
  z = fma(z, pt, z);
  const double vv = ((lane == 1) ? xr2 : xr1) * z;
  ov1 = warp_bcast(vv, 0);
  ov2 = warp_bcast(vv, 1);
  otau = tv;
  obeta = -copysign(nrm, x0);
  if (trivial) {
    ov1 = 0.0;
    ov2 = 0.0;
    otau = 0.0;
    obeta = x0;
  } else if (!safe) {
    double sig = hypot(x1, x2);
    double nr = hypot(x0, sig);
    obeta = -copysign(nr, x0);
    otau = (obeta - x0) / obeta;
    double den = x0 - obeta;
    ov1 = x1 / den;
    ov2 = x2 / den;
  }
}

__device__ __forceinline__ void refl3_apply(double* p, long long stride, int nr, double v1, double v2, double tau) {
  double a0 = p[0], a1 = p[stride], a2 = (nr == 3) ? p[2 * stride] : 0.0;
  double s = tau * fma(v2, a2, fma(v1, a1, a0));
  p[0] = a0 - s;
  p[stride] = fma(-s, v1, a1);
  if (nr == 3) p[2 * stride] = fma(-s, v2, a2);
}

// the warps that apply a step's reflector away from the diagonal block: all
// but warp 0 (the chain), warp 1 (the block) and warp 4 (warp 0's
// sub-partition)
__device__ __forceinline__ bool francis_far_warp(int warp) { return warp >= 2 && warp != 4; }
__device__ __forceinline__ int francis_far_rank(int warp) { return warp - 2 - (warp > 4 ? 1 : 0); }

__device__ inline void cta_double_shift_sweep(const Mat& T, int m, int l, int i, double ssum, double sprod,
                                              const Mat& U, int urows, CtaShared* sh, VRing* ring = nullptr) {
  __shared__ double bnext[2][16];   // B_k for the chain lane, by step parity (row r, column c at r + 4c)
  const int tid = cta_tid(), nt = cta_nt(), lane = tid & 31, warp = tid >> 5;
  // far warps: 2..nwarps-1 without 4 (blocks of at least 3 warps; the kernels use 8)
  const int nwarps = nt >> 5;
  const int nfar = nwarps - 2 - (nwarps > 4 ? 1 : 0);
  // the chain warp's state: the current reflector (the same in every lane)
  double cv1 = 0.0, cv2 = 0.0, ctau = 0.0;
  if (tid == 0) {
    const int nr = min(3, i - l + 1);
    double h00 = T(l, l), h01 = T(l, l + 1), h10 = T(l + 1, l), h11 = T(l + 1, l + 1);
    double x0 = fma(h00, h00, fma(h01, h10, fma(-ssum, h00, sprod)));
    double x1 = h10 * (h00 + h11 - ssum);
    double x2 = (nr == 3) ? h10 * T(l + 2, l + 1) : 0.0;
    double beta;
    house3(nr, x0, x1, x2, cv1, cv2, ctau, beta);
    sh->r[0] = cv1;
    sh->r[1] = cv2;
    sh->r[2] = ctau;
    // B_l (rows l..l+3, columns l..l+2; zero outside the block)
    for (int r = 0; r < 4; ++r)
      for (int c = 0; c < 3; ++c)
        bnext[(l & 1)][r + 4 * c] = (l + r <= i && r <= c + 1) ? T(l + r, l + c) : 0.0;
  }
  __syncthreads();
  if (warp == 0) {   // every lane of the chain warp carries the current reflector
    cv1 = sh->r[0];
    cv2 = sh->r[1];
    ctau = sh->r[2];
  }
  // with a transform stream the accumulation happens in the other block
  const int nu = (U.p && !ring) ? urows : 0;
  for (int k = l; k < i; ++k) {
    const int nr = min(3, i - k + 1);
    const int slot = ((k - l) & 1) * 4;
    if (ring && tid == 128 && sh->r[slot + 2] != 0.0)
      vring_push(ring, sh->r[slot], sh->r[slot + 1], sh->r[slot + 2], k, nr);
    if (warp == 0) {
      if (k + 1 < i) {
        // here nr == 3; the next reflector from column k of P_k B_k P_k
        const double* B = bnext[k & 1];
        const int rr = lane & 3;
        const double b0 = B[rr], b1 = B[rr + 4], b2 = B[rr + 8];
        const int k1 = k + 1, nr1 = min(3, i - k1 + 1);
        double beta;
        warp_next_reflector(b0, b1, b2, cv1, cv2, ctau, nr1, cv1, cv2, ctau, beta);
        if (lane == 0) {
          T(k1, k) = beta;
          T(k1 + 1, k) = 0.0;
          if (nr1 == 3) T(k1 + 2, k) = 0.0;
          const int s1 = 4 - slot;
          sh->r[s1] = cv1;
          sh->r[s1 + 1] = cv2;
          sh->r[s1 + 2] = ctau;
        }
      }
    } else if (warp == 1) {
      const double v1 = sh->r[slot], v2 = sh->r[slot + 1], tau = sh->r[slot + 2];
      // lane = r + 4 c (r, c < 4): entry T(k + r, k + c) of the diagonal block
      const int r = lane & 3, c = (lane >> 2) & 3;
      const bool valid = lane < 16 && k + r <= i && k + c <= m - 1;
      double a = valid ? T(k + r, k + c) : 0.0;
      if (tau != 0.0) {
        // left product on rows k..k+nr-1 of each column
        const double a0 = __shfl_sync(0xffffffffu, a, 4 * c + 0);
        const double a1 = __shfl_sync(0xffffffffu, a, 4 * c + 1);
        const double a2 = __shfl_sync(0xffffffffu, a, 4 * c + 2);
        const double s = tau * fma(v2, (nr == 3) ? a2 : 0.0, fma(v1, a1, a0));
        if (r < nr) a = fma(-s, (r == 0) ? 1.0 : ((r == 1) ? v1 : v2), a);
        // right product on columns k..k+nr-1 of each row
        const double b0 = __shfl_sync(0xffffffffu, a, r + 0);
        const double b1 = __shfl_sync(0xffffffffu, a, r + 4);
        const double b2 = __shfl_sync(0xffffffffu, a, r + 8);
        const double t = tau * fma(v2, (nr == 3) ? b2 : 0.0, fma(v1, b1, b0));
        if (c < nr) a = fma(-t, (c == 0) ? 1.0 : ((c == 1) ? v1 : v2), a);
      }
      // column k below the diagonal belongs to the chain lane when a next
      // reflector follows
      if (valid && !(c == 0 && r >= 1 && k + 1 < i)) T(k + r, k + c) = a;
      if (k + 1 < i) {
        double* Bn = bnext[(k + 1) & 1];
        if (lane < 16 && r >= 1 && c >= 1) Bn[(r - 1) + 4 * (c - 1)] = valid ? a : 0.0;
        if (lane == 16) {
          Bn[3] = 0.0;
          Bn[7] = 0.0;
          Bn[11] = (k + 4 <= i && k + 3 <= m - 1) ? T(k + 4, k + 3) : 0.0;
        }
      }
    } else if (francis_far_warp(warp)) {
      const double v1 = sh->r[slot], v2 = sh->r[slot + 1], tau = sh->r[slot + 2];
      if (tau != 0.0) {
        // items: rows of U first (global memory, the longest loads), then rows
        // 0..k-1 of T, then columns k+4..m-1 of T; each thread loads both of
        // its items of a round before computing either
        const int c0 = k + 4;
        const int nB = max(0, m - c0);
        const int total = nu + k + nB;
        const int bt = francis_far_rank(warp) * 32 + lane, bn = nfar * 32;
        for (int base = 0; base < total; base += 2 * bn) {
          double* p[2];
          long long sd[2];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int it = base + bt + h * bn;
            if (it < nu) {
              p[h] = &U(it, k);
              sd[h] = U.ld;
            } else if (it < nu + k) {
              p[h] = &T(it - nu, k);
              sd[h] = T.ld;
            } else if (it < total) {
              p[h] = &T(k, c0 + (it - nu - k));
              sd[h] = 1;
            } else {
              p[h] = nullptr;
              sd[h] = 0;
            }
          }
          double a[2][3];
#pragma unroll
          for (int h = 0; h < 2; ++h)
            if (p[h]) {
              a[h][0] = p[h][0];
              a[h][1] = p[h][sd[h]];
              a[h][2] = (nr == 3) ? p[h][2 * sd[h]] : 0.0;
            }
#pragma unroll
          for (int h = 0; h < 2; ++h)
            if (p[h]) {
              double s = tau * fma(v2, a[h][2], fma(v1, a[h][1], a[h][0]));
              p[h][0] = a[h][0] - s;
              p[h][sd[h]] = fma(-s, v1, a[h][1]);
              if (nr == 3) p[h][2 * sd[h]] = fma(-s, v2, a[h][2]);
            }
        }
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
// flops (optional, thread 0 only): adds the algorithmic flops of the
// reflectors applied (4 nr per entry of a row or column they touch).
__device__ inline int cta_francis(const Mat& T, int m, int lo, int hi, const Mat& U, int urows, const DeflParams& dp,
                                  CtaShared* sh, VRing* ring = nullptr, double* flops = nullptr) {
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
      cta_double_shift_sweep(T, m, l, i, ssum, sprod, U, urows, sh, ring);
      if (flops && cta_tid() == 0) {
        double e = 0.0;
        for (int k = l; k < i; ++k) e += 4.0 * min(3, i - k + 1) * ((min(k + 3, i) + 1) + (m - k) + (U.p ? urows : 0));
        *flops += e;
      }
    }
    if (l == i) {
      i -= 1;
    } else {
      cta_standardize_block(T, i - 1, m, ring ? Mat{nullptr, 1} : U, urows, sh, ring);
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

// Factor of one swap, computed by one thread (each thread of a block may
// compute a different swap).  Solves the Sylvester equation
// A11 X - X A22 = A12 (its Kronecker form, complete pivoting by magnitude
// keys, a pivot below sml replaced by sml as Bai & Demmel do for nearly equal
// eigenvalues) and factors [-X; I] = Q [R; 0].  The swap is accepted when the
// (2,1) block of Q^T A Q -- the part that must vanish -- is at most
// max(10 u ||A||_F, nu n / u); the product itself is left to the caller.  Two
// 1x1 blocks [[a, b], [0, c]] swap by the rotation whose first column is
// (b, c - a)/norm, which the Sylvester solution x = b / (a - c) gives; its
// residual is zero by construction.  Q (m x m, m = p + q) is written
// column-major with leading dimension 4 to Qo.
__device__ inline bool lane_swap_factor(const Mat& T, int nT, int j, int p, int q, double* Qo) {
  const int m = p + q;
  if (p == 1 && q == 1) {
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
    Qo[0] = cs; Qo[1] = sn; Qo[4] = -sn; Qo[5] = cs;
    return true;
  }
  const int pq = p * q;
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
  double Q[16];
  small_qr_q(W, m, q, Q);
  // residual: rows q..m-1, columns 0..q-1 of Q^T A Q
  double res = 0.0, fro = 0.0;
  for (int b = 0; b < q; ++b) {
    double aq[4];
    for (int t = 0; t < m; ++t) {
      double acc = 0.0;
      for (int s2 = 0; s2 < m; ++s2) acc = fma(T(j + t, j + s2), Q[s2 + 4 * b], acc);
      aq[t] = acc;
    }
    for (int a = q; a < m; ++a) {
      double d = 0.0;
      for (int t = 0; t < m; ++t) d = fma(Q[t + 4 * a], aq[t], d);
      res = fma(d, d, res);
    }
  }
  for (int t = 0; t < m; ++t)
    for (int s2 = 0; s2 < m; ++s2) {
      double av = T(j + t, j + s2);
      fro = fma(av, av, fro);
    }
  for (int b = 0; b < m; ++b)
    for (int a = 0; a < m; ++a) Qo[a + 4 * b] = Q[a + 4 * b];
  const double tol = 10.0 * SCHUR_U;
  return res <= fmax(tol * tol * fro, sml * sml);
}

// ---------------------------------------------------------------------------
// Deflation checks and reordering of AED step 2 (Sec. 2.5), pipelined.
//
// The sequential procedure checks the bottom unevaluated block; a block that
// fails is moved by adjacent swaps to just below the blocks that failed
// before it, and the next bottom block is checked.  A failed block's later
// swaps act on rows and columns above the blocks that are still to be
// checked, so they can run while those are checked, and swaps of disjoint
// pairs of adjacent blocks commute.  Here every failed block that still has
// an unevaluated block directly above it swaps with that block in each round,
// and the bottom block is checked in the same round when it is unevaluated:
// the same swaps and checks as in the sequential order, each failed block
// moving up one block per round behind the one before it.  Per round, one
// thread computes each swap's factor, then warps apply the factors to the rows
// (left products, disjoint rows) and, after a barrier, to the columns of T and
// V (right products, disjoint columns).  A checked 2x2 block is tested in its
// standardised form (computed by the checking thread); the standardising
// rotation is applied when the block deflates, or splits into two 1x1 blocks.
// A rejected swap ends the reordering (the blocks stay where they are and
// count as undeflated), as the sequential procedure halts.
// ---------------------------------------------------------------------------
#define DEFL_MAX_OPS 48       // swaps per round (further ones wait a round)
#define DEFL_MAX_BLOCKS 1024  // diagonal blocks of a window (nw <= 1024)

struct DeflState {
  unsigned char bsz[DEFL_MAX_BLOCKS];  // block sizes of rows [info, ns), top to bottom
  unsigned char bst[DEFL_MAX_BLOCKS];  // 0 not yet checked, 1 failed its check
  double Q[DEFL_MAX_OPS][16];          // the round's swap factors
  int opj[DEFL_MAX_OPS];               // first row of the pair
  int opk[DEFL_MAX_OPS];               // list index of the pair's upper block
  unsigned char opp[DEFL_MAX_OPS], opq[DEFL_MAX_OPS], opacc[DEFL_MAX_OPS];
  double rot[6];                       // cs, sn and the standardised block of the checked 2x2 block
  int nblk, ns, nops, chk, rot_k, halt, done;
};

// Warp 0: this round's swaps (pairs "unevaluated above failed") and whether
// the bottom block is checked.
__device__ inline void defl_schedule(int info, DeflState* ds) {
  const int lane = threadIdx.x & 31;
  const int nb = ds->nblk;
  const int per = (nb + 31) / 32;
  const int k0 = min(lane * per, nb), k1 = min(k0 + per, nb);
  int rows = 0, pairs = 0;
  for (int k = k0; k < k1; ++k) {
    rows += ds->bsz[k];
    if (k > 0 && ds->bst[k] == 1 && ds->bst[k - 1] == 0) ++pairs;
  }
  int rs = rows, ps = pairs;
  for (int o = 1; o < 32; o <<= 1) {
    int a = __shfl_up_sync(0xffffffffu, rs, o);
    int b = __shfl_up_sync(0xffffffffu, ps, o);
    if (lane >= o) {
      rs += a;
      ps += b;
    }
  }
  int pos = info + rs - rows, op = ps - pairs;
  for (int k = k0; k < k1; ++k) {
    if (k > 0 && ds->bst[k] == 1 && ds->bst[k - 1] == 0) {
      if (op < DEFL_MAX_OPS) {
        int p = ds->bsz[k - 1];
        ds->opj[op] = pos - p;
        ds->opk[op] = k - 1;
        ds->opp[op] = (unsigned char)p;
        ds->opq[op] = ds->bsz[k];
      }
      ++op;
    }
    pos += ds->bsz[k];
  }
  const int total = __shfl_sync(0xffffffffu, ps, 31);
  if (lane == 0) {
    const int nops = min(total, DEFL_MAX_OPS);
    const int chk = (nb > 0 && ds->bst[nb - 1] == 0) ? 1 : 0;
    ds->nops = nops;
    ds->chk = chk;
    ds->rot_k = -1;
    ds->done = (nops == 0 && !chk) ? 1 : 0;
  }
}

// The checking thread: bottom block of rows [info, ns).
__device__ inline void defl_check(const Mat& T, double s, const Mat& V, const DeflParams& dp, DeflState* ds) {
  const int nb = ds->nblk, ns = ds->ns;
  const int bs = ds->bsz[nb - 1];
  const int jb = ns - 1;
  if (bs == 1) {
    bool defl = spike_deflatable_blk(0.0, 0.0, 0.0, T(jb, jb), s * V(0, jb), 0.0, 1, dp);
    if (defl) {
      ds->nblk = nb - 1;
      ds->ns = ns - 1;
    } else {
      ds->bst[nb - 1] = 1;
    }
    return;
  }
  double cs, sn, B[4];
  standardize2x2(T(jb - 1, jb - 1), T(jb - 1, jb), T(jb, jb - 1), T(jb, jb), cs, sn, B);
  ds->rot[0] = cs;
  ds->rot[1] = sn;
  for (int t = 0; t < 4; ++t) ds->rot[2 + t] = B[t];
  if (B[2] == 0.0) {
    // real pair: two 1x1 blocks, checked from the next round on
    ds->rot_k = jb - 1;
    ds->bsz[nb - 1] = 1;
    ds->bst[nb - 1] = 0;
    ds->bsz[nb] = 1;
    ds->bst[nb] = 0;
    ds->nblk = nb + 1;
    return;
  }
  const double v0 = V(0, jb - 1), v1 = V(0, jb);
  const double w0 = fma(cs, v0, sn * v1), w1 = fma(-sn, v0, cs * v1);
  bool defl = spike_deflatable_blk(B[0], B[1], B[2], B[3], s * w1, s * w0, 2, dp);
  if (defl) {
    ds->rot_k = jb - 1;
    ds->nblk = nb - 1;
    ds->ns = ns - 2;
  } else {
    ds->bst[nb - 1] = 1;
  }
}

// y = Q^T x on rows j..j+M-1 of the columns c of T (lanes over columns).
template <int M>
__device__ __forceinline__ void defl_left(const Mat& T, int nT, int j, const double* Q, int lane) {
  for (int c = j + lane; c < nT; c += 32) {
    double x[M];
#pragma unroll
    for (int t = 0; t < M; ++t) x[t] = T(j + t, c);
#pragma unroll
    for (int a = 0; a < M; ++a) {
      double acc = 0.0;
#pragma unroll
      for (int t = 0; t < M; ++t) acc = fma(Q[t + 4 * a], x[t], acc);
      T(j + a, c) = acc;
    }
  }
}

// x Q on columns j..j+M-1 of rows 0..j+M-1 of T and of all vrows rows of V;
// rows j+q.. of T get exact zeros in columns j..j+q-1 (the swap's residual).
template <int M>
__device__ __forceinline__ void defl_right(const Mat& T, const Mat& V, int vrows, int j, int q, const double* Q,
                                           int lane) {
  const int nr = j + M;
  for (int it = lane; it < nr + vrows; it += 32) {
    const bool onT = it < nr;
    const Mat& X = onT ? T : V;
    const int r = onT ? it : it - nr;
    double x[M];
#pragma unroll
    for (int t = 0; t < M; ++t) x[t] = X(r, j + t);
    const bool low = onT && r >= j + q;
#pragma unroll
    for (int b = 0; b < M; ++b) {
      double acc = 0.0;
#pragma unroll
      for (int t = 0; t < M; ++t) acc = fma(x[t], Q[t + 4 * b], acc);
      X(r, j + b) = (low && b < q) ? 0.0 : acc;
    }
  }
}

// Runs the checks and the reordering on rows [info, nw) of T (V: the
// accumulated transform, vrows rows).  Returns ns (rows ns..nw-1 deflated);
// failed = 1 when a swap was rejected (or the round limit was reached).
__device__ inline int cta_aed_deflate(const Mat& T, int nw, int info, double s, const Mat& V, int vrows,
                                      const DeflParams& dp, int& failed) {
  __shared__ DeflState ds;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps = (blockDim.x + 31) >> 5;
  if (tid == 0) {
    int nb = 0;
    for (int j = info; j < nw;) {
      int b = (j + 1 < nw && T(j + 1, j) != 0.0) ? 2 : 1;
      ds.bsz[nb] = (unsigned char)b;
      ds.bst[nb] = 0;
      ++nb;
      j += b;
    }
    ds.nblk = nb;
    ds.ns = nw;
    ds.halt = 0;
  }
  __syncthreads();
  const int max_rounds = 4 * nw + 16;
  int round = 0;
  for (; round < max_rounds; ++round) {
    if (tid < 32) defl_schedule(info, &ds);
    __syncthreads();
    if (ds.done || ds.halt) break;
    const int nops = ds.nops;
    if (tid < nops) {
      const int j = ds.opj[tid], p = ds.opp[tid], q = ds.opq[tid];
      const bool acc = lane_swap_factor(T, nw, j, p, q, ds.Q[tid]);
      ds.opacc[tid] = acc ? 1 : 0;
      if (acc) {
        const int k = ds.opk[tid];
        ds.bsz[k] = (unsigned char)q;
        ds.bsz[k + 1] = (unsigned char)p;
        ds.bst[k] = 1;
        ds.bst[k + 1] = 0;
      } else {
        ds.halt = 1;
      }
    }
    if (tid == (int)blockDim.x - 1 && ds.chk) defl_check(T, s, V, dp, &ds);
    __syncthreads();
    const int rk = ds.rot_k;
    const double cs = ds.rot[0], sn = ds.rot[1];
    const bool rot = rk >= 0 && !(cs == 1.0 && sn == 0.0);
    // left products (rows of each pair / of the rotated block)
    for (int o = warp; o <= nops; o += nwarps) {
      if (o < nops) {
        if (!ds.opacc[o]) continue;
        const int j = ds.opj[o], m = ds.opp[o] + ds.opq[o];
        if (m == 2) defl_left<2>(T, nw, j, ds.Q[o], lane);
        else if (m == 3) defl_left<3>(T, nw, j, ds.Q[o], lane);
        else defl_left<4>(T, nw, j, ds.Q[o], lane);
      } else if (rot) {
        for (int c = rk + 2 + lane; c < nw; c += 32) {
          double a = T(rk, c), b = T(rk + 1, c);
          T(rk, c) = fma(cs, a, sn * b);
          T(rk + 1, c) = fma(-sn, a, cs * b);
        }
      }
    }
    __syncthreads();
    // right products (columns of each pair / of the rotated block, T and V)
    for (int o = warp; o <= nops; o += nwarps) {
      if (o < nops) {
        if (!ds.opacc[o]) continue;
        const int j = ds.opj[o], q = ds.opq[o], m = ds.opp[o] + q;
        if (m == 2) defl_right<2>(T, V, vrows, j, q, ds.Q[o], lane);
        else if (m == 3) defl_right<3>(T, V, vrows, j, q, ds.Q[o], lane);
        else defl_right<4>(T, V, vrows, j, q, ds.Q[o], lane);
      } else if (rk >= 0) {
        if (rot) {
          for (int it = lane; it < rk + vrows; it += 32) {
            const bool onT = it < rk;
            const Mat& X = onT ? T : V;
            const int r = onT ? it : it - rk;
            double a = X(r, rk), b = X(r, rk + 1);
            X(r, rk) = fma(cs, a, sn * b);
            X(r, rk + 1) = fma(-sn, a, cs * b);
          }
        }
        if (lane == 0) {
          T(rk, rk) = ds.rot[2];
          T(rk, rk + 1) = ds.rot[3];
          T(rk + 1, rk) = ds.rot[4];
          T(rk + 1, rk + 1) = ds.rot[5];
        }
      }
    }
    __syncthreads();
  }
  const int ns = ds.ns;
  failed = (ds.halt || round >= max_rounds) ? 1 : 0;
  __syncthreads();
  return ns;
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
  int failed = 0;
  int ns = cta_aed_deflate(T, nw, info, s, V, nw, dp, failed);
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
