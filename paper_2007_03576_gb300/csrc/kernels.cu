// kernels.cu -- device kernels of the single-matrix path.
//
//   k_prep          input check (finite), zero below the subdiagonal, Z = I
//   k_scan          vigilant-deflation scan of the subdiagonal (Sec. 2.1)
//   k_std2          standardise a decoupled 2x2 block (eq. 2by2_blocks)
//   k_smallqr       double-shift QR of a small block in shared memory,
//                   transform accumulated into U (Sec. 2.2, "small Schur")
//   k_aed_small     whole AED step for windows <= NW_SMEM_MAX (Sec. 2.5)
//   k_copy_window / k_aed_big_post
//                   AED for larger windows: copy out, (recursive QR on the
//                   host-driven path), then deflation checks, reordering and
//                   spike elimination on the window in global memory
//   k_make_pairs    next sweep's shift pairs from the AED candidates
//                   (or exceptional shifts)
//   k_chase         windowed bulge chase of several chains (Sec. 2.3, 2.4),
//                   window and accumulator U in shared memory
//   k_apply_u       off-window products U^T X / X U (Sec. 3.2.1), FP64 FFMA
//   k_extract_eigs  eigenvalues from the standardised diagonal blocks
#include <cooperative_groups.h>

#include "cta.cuh"
#include "kernels.cuh"

namespace cg = cooperative_groups;

// ---------------------------------------------------------------------------
__global__ void k_set_int(int* p, int v) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *p = v;
}

__global__ void k_prep(double* H, long long ldh, int n, double* Z, long long ldz, int zinit, int* nonfinite) {
  for (int j = blockIdx.x; j < n; j += gridDim.x) {
    double* col = H + (long long)j * ldh;
    int bad = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      if (i > j + 1)
        col[i] = 0.0;
      else if (!isfinite(col[i]))
        bad = 1;
    }
    if (bad) atomicOr(nonfinite, 1);
    if (Z != nullptr && zinit == 0) {
      double* zc = Z + (long long)j * ldz;
      for (int i = threadIdx.x; i < n; i += blockDim.x) zc[i] = (i == j) ? 1.0 : 0.0;
    }
  }
}

__global__ void k_scan(double* H, long long ldh, int lo, int hi, DeflParams dp, Ctl* ctl) {
  __shared__ CtaShared sh;
  Mat Hm{H, ldh};
  int l = cta_find_ktop(Hm, lo, hi, dp, &sh);
  if (threadIdx.x == 0) ctl->ktop = l;
}

__global__ void k_std2(double* H, long long ldh, int n, double* Z, long long ldz, int zrows, int k) {
  __shared__ CtaShared sh;
  Mat Hm{H, ldh};
  Mat Zm{Z, ldz};
  cta_standardize_block(Hm, k, n, Zm, zrows, &sh);
}

// ---------------------------------------------------------------------------
// Small block [ilo, ihi] (m <= NW_SMEM_MAX): copy to shared memory, Francis
// QR with the transform accumulated into U (m x m, global), copy back.  The
// off-window rows/columns and Z are updated afterwards by k_apply_u.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(CTA_THREADS) k_smallqr(double* H, long long ldh, int ilo, int ihi, double* U,
                                                         int ldu, DeflParams dp, Ctl* ctl) {
  extern __shared__ double smem[];
  __shared__ CtaShared sh;
  int m = ihi - ilo + 1;
  int ldt = m | 1;
  Mat T{smem, ldt};
  Mat Um{U, ldu};
  for (int j = 0; j < m; ++j)
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      T(i, j) = (i <= j + 1) ? H[(ilo + i) + (long long)(ilo + j) * ldh] : 0.0;
      Um(i, j) = (i == j) ? 1.0 : 0.0;
    }
  __syncthreads();
  int info = cta_francis(T, m, 0, m - 1, Um, m, dp, &sh);
  for (int j = 0; j < m; ++j)
    for (int i = threadIdx.x; i < m; i += blockDim.x)
      H[(ilo + i) + (long long)(ilo + j) * ldh] = (i <= j + 1) ? T(i, j) : 0.0;
  if (threadIdx.x == 0) ctl->info = info ? (ilo + info) : 0;
}

// ---------------------------------------------------------------------------
// AED on the trailing window [kwtop, kbot] of the active block [ktop, kbot]
// with the window held in shared memory.
// ---------------------------------------------------------------------------
__device__ void aed_write_back(double* H, long long ldh, int ktop, int kwtop, int nw, const Mat& T, double top) {
  for (int j = 0; j < nw; ++j)
    for (int i = threadIdx.x; i < nw; i += blockDim.x)
      H[(kwtop + i) + (long long)(kwtop + j) * ldh] = (i <= j + 1) ? T(i, j) : 0.0;
  if (kwtop > ktop) {
    for (int i = threadIdx.x; i < nw; i += blockDim.x)
      H[(kwtop + i) + (long long)(kwtop - 1) * ldh] = (i == 0) ? top : 0.0;
  }
}

// The AED kernel runs as a cluster of two blocks (Sec. 2.5 step 1 on block
// 0, the accumulation of its transform V on block 1, see the transform
// stream in cta.cuh); block 0 then runs steps 2-3 with V in global memory.
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(CTA_THREADS)
    k_aed_small(double* H, long long ldh, int ktop, int kbot, int nw, double* V, int ldv, double* cand_re,
                double* cand_im, double* vbuf, DeflParams dp, DeflParams dpw, Ctl* ctl) {
  extern __shared__ double smem[];
  __shared__ CtaShared sh;
  __shared__ int s_ncand, s_swf;
  __shared__ VRing ring;
  cg::cluster_group cluster = cg::this_cluster();
  const unsigned rank = cluster.block_rank();
  int kwtop = kbot - nw + 1;
  int ldt = nw | 1;
  if (threadIdx.x == 0) {
    ring.count = 0;
    ring.consumed = 0;
    ring.pushed = 0;
    ring.err = 0;
    ring.remote = cluster.map_shared_rank(&ring, rank ^ 1u);
  }
  cluster.sync();
  if (rank == 1) {
    Mat Vs{smem, ldt};
    for (int j = 0; j < nw; ++j)
      for (int i = threadIdx.x; i < nw; i += blockDim.x) Vs(i, j) = (i == j) ? 1.0 : 0.0;
    __syncthreads();
    const int timed_out = vring_consume(&ring, Vs, nw);
    for (int j = 0; j < nw; ++j)
      for (int i = threadIdx.x; i < nw; i += blockDim.x) V[i + (long long)j * ldv] = Vs(i, j);
    if (timed_out && threadIdx.x == 0) atomicOr(&ctl->sync_err, 1);
    cluster.sync();   // V is complete in global memory
    return;
  }
  Mat T{smem, ldt};
  Mat Vm{V, ldv};
  for (int j = 0; j < nw; ++j)
    for (int i = threadIdx.x; i < nw; i += blockDim.x)
      T(i, j) = (i <= j + 1) ? H[(kwtop + i) + (long long)(kwtop + j) * ldh] : 0.0;
  double s = (kwtop > ktop) ? H[kwtop + (long long)(kwtop - 1) * ldh] : 0.0;
  __syncthreads();
  long long c0 = clock64();
  int info = cta_francis(T, nw, 0, nw - 1, Vm, nw, dpw, &sh, &ring);
  if (threadIdx.x == 128) vring_push(&ring, 0.0, 0.0, 0.0, 0, 0);   // end of the stream
  cluster.sync();   // block 1 has applied the stream and written V
  if (threadIdx.x == 0) {
    ctl->cyc_schur += clock64() - c0;
    if (ring.err) atomicOr(&ctl->sync_err, 1);
  }
  double top;
  int nd = cta_aed_post(T, nw, info, s, Vm, dp, vbuf, cand_re, cand_im, &s_ncand, &top, &s_swf, &sh,
                        &ctl->cyc_defl);
  if (nd > 0) aed_write_back(H, ldh, ktop, kwtop, nw, T, top);
  if (threadIdx.x == 0) {
    ctl->nd = nd;
    ctl->ncand = s_ncand;
    ctl->swap_fail = s_swf;
  }
}

__global__ void k_copy_window(const double* H, long long ldh, int kwtop, int nw, double* T, int ldt, double* V,
                              int ldv) {
  for (int j = blockIdx.x; j < nw; j += gridDim.x)
    for (int i = threadIdx.x; i < nw; i += blockDim.x) {
      T[i + (long long)j * ldt] = (i <= j + 1) ? H[(kwtop + i) + (long long)(kwtop + j) * ldh] : 0.0;
      V[i + (long long)j * ldv] = (i == j) ? 1.0 : 0.0;
    }
}

// AED steps 2-3 for a window whose Schur form T (global, with transform V)
// was computed by the recursive driver; inner_info = its return code
// (rows 0..inner_info-1 unreduced).
__global__ void __launch_bounds__(CTA_THREADS) k_aed_big_post(double* H, long long ldh, int ktop, int kbot, int nw,
                                                              double* T, int ldt, double* V, int ldv,
                                                              double* cand_re, double* cand_im, double* vbuf,
                                                              DeflParams dp, Ctl* ctl, int inner_info) {
  __shared__ CtaShared sh;
  __shared__ int s_ncand, s_swf;
  int kwtop = kbot - nw + 1;
  Mat Tm{T, ldt};
  Mat Vm{V, ldv};
  int info = inner_info;
  double s = (kwtop > ktop) ? H[kwtop + (long long)(kwtop - 1) * ldh] : 0.0;
  double top;
  int nd = cta_aed_post(Tm, nw, info, s, Vm, dp, vbuf, cand_re, cand_im, &s_ncand, &top, &s_swf, &sh,
                        &ctl->cyc_defl);
  __syncthreads();
  if (nd > 0) aed_write_back(H, ldh, ktop, kwtop, nw, Tm, top);
  if (threadIdx.x == 0) {
    ctl->nd = nd;
    ctl->ncand = s_ncand;
    ctl->swap_fail = s_swf;
  }
}

// ---------------------------------------------------------------------------
// Shift recomputation after AED (opts.recompute_shifts; LAPACK's rule): when
// a sweep follows and AED left at most ns/2 undeflated candidates, the
// candidates become the eigenvalues of the trailing r x r principal
// submatrix of the active block (r = min(ns, NW_SMEM_MAX, rows)), computed by
// double-shift QR on a copy in shared memory; on a QR failure the AED
// candidates are kept.  kbot_old: the block's last row before AED.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(CTA_THREADS) k_recompute_shifts(const double* H, long long ldh, int ktop,
                                                                  int kbot_old, int ns_max, int nw, int nibble,
                                                                  int nmin, double* cand_re, double* cand_im,
                                                                  DeflParams dp, Ctl* ctl) {
  extern __shared__ double smem[];
  __shared__ CtaShared sh;
  const int nd = ctl->nd;
  const int kbot = kbot_old - nd;
  const int mblk = kbot - ktop + 1;
  // the same decisions as the driver: no sweep follows in these cases
  if (mblk <= nmin) return;
  if (nd > 0 && 100 * nd > nibble * nw) return;
  int ns = min(ns_max, mblk - 1);
  ns -= ns % 2;
  if (ctl->ncand > ns / 2) return;
  const int m = min(min(ns, NW_SMEM_MAX), mblk);
  if (m < 2) return;
  const int ks = kbot - m + 1;
  const int ldt = m | 1;
  Mat T{smem, ldt};
  for (int j = 0; j < m; ++j)
    for (int i = threadIdx.x; i < m; i += blockDim.x)
      T(i, j) = (i <= j + 1) ? H[(ks + i) + (long long)(ks + j) * ldh] : 0.0;
  __syncthreads();
  DeflParams dpw = dp;
  dpw.n = m;
  const int info = cta_francis(T, m, 0, m - 1, Mat{nullptr, 1}, 0, dpw, &sh);
  __syncthreads();
  if (info != 0 || threadIdx.x != 0) return;
  int c = 0, j = 0;
  while (j < m) {
    if (j + 1 < m && T(j + 1, j) != 0.0) {
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
  ctl->ncand = c;
  ctl->recomputed += 1;
}

// ---------------------------------------------------------------------------
// Shift pairs for the next sweep (one thread).  Reading of Sec. 2.5: the
// undeflated AED candidates become the shifts -- the bottom-most ones, complex
// conjugates kept together, real shifts paired in order of appearance; an
// exceptional pair every exc_period-th iteration without deflation; the
// trailing 2x2 when no candidate is left.
// ---------------------------------------------------------------------------
__global__ void k_make_pairs(const double* H, long long ldh, int ktop, int kbot_old, int ns_max, int ndfl_host,
                             int exc_period, const double* cand_re, const double* cand_im, double* pairs, Ctl* ctl) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  Mat Hm{const_cast<double*>(H), ldh};
  int nd = ctl->nd;
  int ndfl = (nd > 0) ? 1 : ndfl_host + 1;
  ctl->npairs = make_shift_pairs(Hm, ktop, kbot_old - nd, ns_max, ndfl, exc_period, cand_re, cand_im, ctl->ncand,
                                 pairs);
  ctl->ndfl = ndfl;
}

// ---------------------------------------------------------------------------
// Windowed bulge chase (Sec. 2.3, Fig. 2; several chains as in Fig. 3).
//
// Block c moves chain c through its window [ws, we]: chain-local steps
// tau0..tau1-1, bulge j of the chain at row k = lo + tau - 3 j.  Per step:
// (A) every bulge's reflector is built from the window (the shift vector at
// k = lo, else column k-1), (B) all left products on the in-window columns,
// (C) all right products on the in-window rows and on the accumulator U.
// Doing the bulges of a step bottom-first in this three-phase order gives the
// reflectors of introducing the bulges one at a time and chasing each just far
// enough (different bulges touch disjoint rows/columns except where a left
// and a right product meet, and those commute).  The window and U are then
// written back; k_apply_u applies U off-window.
// ---------------------------------------------------------------------------
size_t chase_smem_bytes(int kwin) {
  size_t ld = (size_t)(kwin | 1);
  return 2 * ld * (size_t)kwin * sizeof(double);
}

#define CHASE_G 2

// One product phase of k_chase over all bulges: SIDE 0 the left products
// (rows kl..kl+2 of the window, columns kl..L-1), SIDE 1 the right products
// (columns kl..kl+2 of window rows 0..min(kl+3, hil) and of U rows
// ulo..uhi, the rows where U's columns kl..kl+2 can be nonzero).  Warp w
// takes bulges w, w + nwarps, ...; its lanes run over the concatenated items
// of those bulges, CHASE_G per thread with all loads issued before the
// arithmetic.
template <int SIDE>
__device__ __forceinline__ void chase_phase(const Mat& W, const Mat& Us, int L, int ld, int nb, int hil,
                                            const double* rv1, const double* rv2, const double* rtau,
                                            const int* rk, const int* rnr, const int* rulo, const int* ruhi) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  int end[4], kls[4], jj[4], nws[4];
  int nmy = 0, tot = 0;
  for (int j = warp; j < nb && nmy < 4; j += nwarps) {
    if (rnr[j] == 0 || rtau[j] == 0.0) continue;
    const int kl = rk[j];
    const int nwr = (SIDE == 0) ? 0 : min(kl + 3, hil) + 1;
    tot += (SIDE == 0) ? (L - kl) : (nwr + ruhi[j] - rulo[j] + 1);
    end[nmy] = tot;
    kls[nmy] = kl;
    jj[nmy] = j;
    nws[nmy] = nwr;
    ++nmy;
  }
  for (int base = lane; base < tot; base += CHASE_G * 32) {
    double* p[CHASE_G];
    long long sd[CHASE_G];
    int ms[CHASE_G];
#pragma unroll
    for (int g = 0; g < CHASE_G; ++g) {
      const int it = base + g * 32;
      p[g] = nullptr;
      sd[g] = 0;
      ms[g] = 0;
      if (it >= tot) continue;
      int m = 0;
      while (it >= end[m]) ++m;
      const int q = it - (m ? end[m - 1] : 0);
      const int kl = kls[m];
      if (SIDE == 0) {
        p[g] = &W(kl, kl + q);
        sd[g] = 1;
      } else if (q < nws[m]) {
        p[g] = &W(q, kl);
        sd[g] = ld;
      } else {
        p[g] = &Us(q - nws[m] + rulo[jj[m]], kl);
        sd[g] = ld;
      }
      ms[g] = m;
    }
    double a[CHASE_G][3];
#pragma unroll
    for (int g = 0; g < CHASE_G; ++g)
      if (p[g]) {
        const int nr = rnr[jj[ms[g]]];
        a[g][0] = p[g][0];
        a[g][1] = p[g][sd[g]];
        a[g][2] = (nr == 3) ? p[g][2 * sd[g]] : 0.0;
      }
#pragma unroll
    for (int g = 0; g < CHASE_G; ++g)
      if (p[g]) {
        const int j = jj[ms[g]];
        const int nr = rnr[j];
        const double v1 = rv1[j], v2 = rv2[j], t = rtau[j];
        double s = t * (a[g][0] + v1 * a[g][1] + v2 * a[g][2]);
        p[g][0] = a[g][0] - s;
        p[g][sd[g]] = a[g][1] - s * v1;
        if (nr == 3) p[g][2 * sd[g]] = a[g][2] - s * v2;
      }
  }
}

__global__ void __launch_bounds__(CHASE_THREADS) k_chase(double* H, long long ldh, const double* pairs, double* Ubuf,
                                                       const __grid_constant__ ChaseArgs args) {
  extern __shared__ double smem[];
  __shared__ double rv1[MAX_BULGES_PER_CHAIN], rv2[MAX_BULGES_PER_CHAIN], rtau[MAX_BULGES_PER_CHAIN];
  __shared__ int rk[MAX_BULGES_PER_CHAIN], rnr[MAX_BULGES_PER_CHAIN];
  // rows ulo[c]..uhi[c] hold U's nonzeros in column c (U starts as I; a
  // reflector on columns kl..kl+2 merges their ranges)
  __shared__ short ulo[KWIN_MAX], uhi[KWIN_MAX];
  __shared__ int rulo[MAX_BULGES_PER_CHAIN], ruhi[MAX_BULGES_PER_CHAIN];
  const ChainDesc& d = args.c[blockIdx.x];
  const int ws = d.ws;
  const int L = d.we - d.ws + 1;
  const int ld = L | 1;
  Mat W{smem, ld};
  Mat Us{smem + (size_t)ld * L, ld};
  const int lo = args.lo, hi = args.hi;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int j = 0; j < L; ++j)
    for (int i = tid; i < L; i += nt) {
      W(i, j) = H[(ws + i) + (long long)(ws + j) * ldh];
      Us(i, j) = (i == j) ? 1.0 : 0.0;
    }
  for (int c = tid; c < L; c += nt) {
    ulo[c] = (short)c;
    uhi[c] = (short)c;
  }
  __syncthreads();
  const int nb = d.nb;
  const int hil = hi - ws;  // local index of hi
  for (int tau = d.tau0; tau < d.tau1; ++tau) {
    // (A) reflectors
    if (tid < nb) {
      int j = tid;
      int k = lo + tau - 3 * j;
      if (k >= lo && k <= hi - 1) {
        int nr = min(3, hi - k + 1);
        int kl = k - ws;
        double x0, x1, x2 = 0.0;
        if (k == lo) {
          double ssum = pairs[2 * (d.pair0 + j)], sprod = pairs[2 * (d.pair0 + j) + 1];
          double h00 = W(kl, kl), h01 = W(kl, kl + 1), h10 = W(kl + 1, kl), h11 = W(kl + 1, kl + 1);
          x0 = h00 * h00 + h01 * h10 - ssum * h00 + sprod;
          x1 = h10 * (h00 + h11 - ssum);
          if (nr == 3) x2 = h10 * W(kl + 2, kl + 1);
        } else {
          x0 = W(kl, kl - 1);
          x1 = W(kl + 1, kl - 1);
          if (nr == 3) x2 = W(kl + 2, kl - 1);
        }
        double v1, v2, t, beta;
        house3(nr, x0, x1, x2, v1, v2, t, beta);
        if (k > lo) {
          W(kl, kl - 1) = beta;
          W(kl + 1, kl - 1) = 0.0;
          if (nr == 3) W(kl + 2, kl - 1) = 0.0;
        }
        rv1[j] = v1;
        rv2[j] = v2;
        rtau[j] = t;
        rk[j] = kl;
        rnr[j] = nr;
        int a0 = ulo[kl], b0 = uhi[kl];
        for (int t2 = 1; t2 < nr; ++t2) {
          a0 = min(a0, (int)ulo[kl + t2]);
          b0 = max(b0, (int)uhi[kl + t2]);
        }
        for (int t2 = 0; t2 < nr; ++t2) {
          ulo[kl + t2] = (short)a0;
          uhi[kl + t2] = (short)b0;
        }
        rulo[j] = a0;
        ruhi[j] = b0;
      } else {
        rnr[j] = 0;
      }
    }
    __syncthreads();
    // (B) left products: slot -> (bulge j, window column c), active for
    // c >= kl_j; (C) right products: slot -> (bulge j, row q), q < L a window
    // row (active for q <= min(kl_j + 3, hil)), q >= L row q - L of U.
    // Consecutive threads take consecutive columns / rows of one bulge; each
    // thread loads the operands of CHASE_G slots before computing any.
    chase_phase<0>(W, Us, L, ld, nb, hil, rv1, rv2, rtau, rk, rnr, rulo, ruhi);
    __syncthreads();
    chase_phase<1>(W, Us, L, ld, nb, hil, rv1, rv2, rtau, rk, rnr, rulo, ruhi);
    __syncthreads();
  }
  double* Uout = Ubuf + d.uoff;
  for (int j = 0; j < L; ++j)
    for (int i = tid; i < L; i += nt) {
      H[(ws + i) + (long long)(ws + j) * ldh] = W(i, j);
      Uout[i + (long long)j * args.ldu] = Us(i, j);
    }
  // the row range of U's nonzeros in each column, for the products
  int2* Urng = (int2*)(Uout + (size_t)args.ldu * args.ldu);
  for (int c = tid; c < L; c += nt) Urng[c] = make_int2(ulo[c], uhi[c]);
}

// ---------------------------------------------------------------------------
// Off-window products (Sec. 3.2.1 left/right update), FP64 FFMA.
//
// A tile is TN vectors of one task, all L entries each, so a block owns its
// output and updates A in place.  y = U^T x for every vector x (a column of X
// for side 0; a row of X for side 1, where X U = (U^T X^T)^T).  U streams
// through shared memory in chunks of KC rows; each thread keeps RM x 4
// accumulators (rows rg + RG*t, vectors 4*vg .. 4*vg+3).
// ---------------------------------------------------------------------------
int apply_u_tn(int maxL) {
  if (maxL <= 128) return 64;
  if (maxL <= 256) return 32;
  if (maxL <= 512) return 16;
  return 8;
}

// Rows of U staged per chunk: at most half of L (rounded up to 16), so that
// the chase windows' products (L <= 112, 64 vectors) take ~87 KB of shared
// memory and two blocks share an SM, and at most 16384 / (L + 1) in general.
__host__ __device__ static inline int apply_u_kc(int L) {
  int kc = 16384 / (L + 1);
  int half = ((L + 1) / 2 + 15) / 16 * 16;
  if (kc > half) kc = half;
  return kc < L ? (kc < 1 ? 1 : kc) : L;
}

size_t apply_u_smem_bytes(int tn, int maxL) {
  size_t ldv = (size_t)tn + 1;
  size_t kc = (size_t)apply_u_kc(maxL);
  return ((size_t)maxL * ldv + kc * ((size_t)maxL + 1)) * sizeof(double);
}

// One k of the register tile: the thread's CN vector entries of row k of X
// (vectors vg, vg + VG, vg + 2 VG, ...: consecutive lanes read consecutive
// words, no bank conflicts) are loaded once and multiplied into every active
// row block a.
template <int CN, int VG>
__device__ __forceinline__ void apply_u_k_impl(const double* sX, const double* sU, int krow, int kk, int LDV, int LDU,
                                               int vg, int rg, int RG, int L, unsigned act, double (&acc)[8][CN]) {
  const double* xr = sX + (size_t)krow * LDV + vg;
  double x[CN];
#pragma unroll
  for (int c = 0; c < CN; ++c) x[c] = xr[c * VG];
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    if (act & (1u << a)) {
      const int i = rg + RG * a;
      const double u = (i < L) ? sU[(size_t)kk * LDU + i] : 0.0;
#pragma unroll
      for (int c = 0; c < CN; ++c) acc[a][c] = fma(u, x[c], acc[a][c]);
    }
  }
}
// row blocks a whose range [klo[a], khi[a]] contains k
__device__ __forceinline__ unsigned fine_mask(int k, const int (&klo)[8], const int (&khi)[8]) {
  unsigned m = 0;
#pragma unroll
  for (int a = 0; a < 8; ++a) m |= (k >= klo[a] && k <= khi[a]) ? (1u << a) : 0u;
  return m;
}

template <int TN>
__global__ void __launch_bounds__(CTA_THREADS, 2) k_apply_u(const __grid_constant__ UpdArgs args) {
  extern __shared__ double smem[];
  constexpr int CN = 4;
  constexpr int VG = TN / CN;          // vector groups
  constexpr int RG = CTA_THREADS / VG; // row groups
  constexpr int LDV = TN + 1;
  const int tid = threadIdx.x;
  const int vg = tid % VG, rg = tid / VG;
  const UpdTask& last = args.t[args.ntask - 1];
  const int total = last.tile0 + last.ntile;
  for (int tile = blockIdx.x; tile < total; tile += gridDim.x) {
    int ti = 0;
    while (ti + 1 < args.ntask && args.t[ti + 1].tile0 <= tile) ++ti;
    const UpdTask& t = args.t[ti];
    if (t.gate != nullptr && *t.gate == 0) continue;
    const int L = t.L;
    const int v0 = (tile - t.tile0) * TN;
    const int nv = min(TN, t.nvec - v0);
    const int RM = (L + RG - 1) / RG;
    const int KC = apply_u_kc(L);
    // rows k of U that can be nonzero in the output rows of this warp, per
    // row block a: the union of the columns' ranges over the warp's rows
    // (warp-uniform, so the per-k skip below never diverges inside a warp)
    int klo[8], khi[8];
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int i = rg + RG * a;
      int lo = L, hi = -1;
      if (a < RM && i < L) {
        if (t.rng != nullptr) {
          const int2 r = t.rng[i];
          lo = r.x;
          hi = r.y;
        } else {
          lo = 0;
          hi = L - 1;
        }
      }
#pragma unroll
      for (int o = VG; o < 32; o <<= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
      }
      klo[a] = lo;
      khi[a] = hi;
    }
    const int LDU = L + 1;
    double* sX = smem;                       // [L][LDV]: sX[k*LDV + v]
    double* sU = smem + (size_t)L * LDV;     // [KC][LDU]: sU[kk*LDU + i]
    const long long lda = t.lda;
    // load the TN vectors
    if (t.side == 0) {
      for (int idx = tid; idx < L * TN; idx += CTA_THREADS) {
        int k = idx % L, v = idx / L;
        sX[k * LDV + v] = (v < nv) ? t.A[(t.r0 + k) + (long long)(t.c0 + v0 + v) * lda] : 0.0;
      }
    } else {
      for (int idx = tid; idx < L * TN; idx += CTA_THREADS) {
        int v = idx % TN, k = idx / TN;
        sX[k * LDV + v] = (v < nv) ? t.A[(t.r0 + v0 + v) + (long long)(t.c0 + k) * lda] : 0.0;
      }
    }
    double acc[8][CN];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int c = 0; c < CN; ++c) acc[a][c] = 0.0;
    for (int kc = 0; kc < L; kc += KC) {
      const int kn = min(KC, L - kc);
      __syncthreads();
      for (int idx = tid; idx < kn * L; idx += CTA_THREADS) {
        int kk = idx % kn, i = idx / kn;
        sU[kk * LDU + i] = t.U[(kc + kk) + (long long)i * t.ldu];
      }
      __syncthreads();
      // k in blocks of 16; a block of output rows (rows RG*a .. RG*a+RG-1) is
      // skipped where U[k, i] is structurally zero for all its rows:
      // k - i > lbw or i - k > ubw (banded window transforms of the chase)
      for (int k16 = 0; k16 < kn; k16 += 16) {
        const int kg0 = kc + k16;
        const int kend = min(kn, k16 + 16);
        const int kg1 = kc + kend - 1;
        // row blocks with a nonzero of U in this k block (uniform over the
        // block: the test depends on a, not on the thread)
        unsigned act = 0;
#pragma unroll
        for (int a = 0; a < 8; ++a)
          if (a < RM && !((kg0 - (RG * a + RG - 1) > t.lbw) || (RG * a - kg1 > t.ubw))) act |= 1u << a;
        if (act == 0) continue;
        if (kend - k16 == 16) {
#pragma unroll 4
          for (int kk = k16; kk < k16 + 16; ++kk)
            apply_u_k_impl<CN, VG>(sX, sU, kc + kk, kk, LDV, LDU, vg, rg, RG, L, act & fine_mask(kc + kk, klo, khi), acc);
        } else {
          for (int kk = k16; kk < kend; ++kk)
            apply_u_k_impl<CN, VG>(sX, sU, kc + kk, kk, LDV, LDU, vg, rg, RG, L, act & fine_mask(kc + kk, klo, khi), acc);
        }
      }
    }
    __syncthreads();
    // stage the outputs (i-major) and store
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      if (a < RM) {
        int i = rg + RG * a;
        if (i < L) {
#pragma unroll
          for (int c = 0; c < CN; ++c) sX[i * LDV + vg + VG * c] = acc[a][c];
        }
      }
    }
    __syncthreads();
    if (t.side == 0) {
      for (int idx = tid; idx < L * TN; idx += CTA_THREADS) {
        int k = idx % L, v = idx / L;
        if (v < nv) t.A[(t.r0 + k) + (long long)(t.c0 + v0 + v) * lda] = sX[k * LDV + v];
      }
    } else {
      for (int idx = tid; idx < L * TN; idx += CTA_THREADS) {
        int v = idx % TN, k = idx / TN;
        if (v < nv) t.A[(t.r0 + v0 + v) + (long long)(t.c0 + k) * lda] = sX[k * LDV + v];
      }
    }
    __syncthreads();
  }
}

cudaError_t launch_apply_u(int tn, int grid, size_t smem, cudaStream_t st, const UpdArgs& a) {
  switch (tn) {
    case 64: k_apply_u<64><<<grid, CTA_THREADS, smem, st>>>(a); break;
    case 32: k_apply_u<32><<<grid, CTA_THREADS, smem, st>>>(a); break;
    case 16: k_apply_u<16><<<grid, CTA_THREADS, smem, st>>>(a); break;
    default: k_apply_u<8><<<grid, CTA_THREADS, smem, st>>>(a); break;
  }
  return cudaGetLastError();
}

int apply_u_blocks_per_sm(int tn, size_t smem) {
  int nb = 0;
  cudaError_t e;
  switch (tn) {
    case 64: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_apply_u<64>, CTA_THREADS, smem); break;
    case 32: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_apply_u<32>, CTA_THREADS, smem); break;
    case 16: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_apply_u<16>, CTA_THREADS, smem); break;
    default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_apply_u<8>, CTA_THREADS, smem); break;
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return nb > 0 ? nb : 1;
}

cudaError_t apply_u_set_smem(int bytes) {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_apply_u<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes))) return e;
  if ((e = cudaFuncSetAttribute(k_apply_u<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes))) return e;
  if ((e = cudaFuncSetAttribute(k_apply_u<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes))) return e;
  return cudaFuncSetAttribute(k_apply_u<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

// ---------------------------------------------------------------------------
__global__ void k_extract_eigs(const double* H, long long ldh, int n, double* wr, double* wi) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    int s = -1;
    if (j + 1 < n && H[(j + 1) + (long long)j * ldh] != 0.0) s = j;
    else if (j > 0 && H[j + (long long)(j - 1) * ldh] != 0.0) s = j - 1;
    if (s < 0) {
      wr[j] = H[j + (long long)j * ldh];
      wi[j] = 0.0;
    } else {
      double r1, i1, r2, i2;
      eig2x2(H[s + (long long)s * ldh], H[s + (long long)(s + 1) * ldh], H[(s + 1) + (long long)s * ldh],
             H[(s + 1) + (long long)(s + 1) * ldh], r1, i1, r2, i2);
      wr[j] = (j == s) ? r1 : r2;
      wi[j] = (j == s) ? i1 : i2;
    }
  }
}

// ---------------------------------------------------------------------------
// FP64 FMA throughput probe: every thread runs FM_CHAINS independent
// dependent chains of fused multiply-adds (the instruction the off-window
// products execute), so every sub-partition always has an FP64 instruction
// ready; the result is written so that nothing is optimised away.
#define FM_CHAINS 8
__global__ void __launch_bounds__(256) k_fma_probe(int iters, double* out) {
  double a[FM_CHAINS];
#pragma unroll
  for (int c = 0; c < FM_CHAINS; ++c) a[c] = 1.0 + 1e-9 * (threadIdx.x + c);
  const double m = 0.9999999999, b = 1e-10;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < FM_CHAINS; ++c) a[c] = fma(a[c], m, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < FM_CHAINS; ++c) s += a[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

int fma_probe_launch(int iters, int blocks, double* out, cudaStream_t st) {
  k_fma_probe<<<blocks, 256, 0, st>>>(iters, out);
  return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

// ---------------------------------------------------------------------------
// Diagnostics: the deflation tests of Sec. 5.6 on given data.
__global__ void k_vigilant_eval(int count, const double* H, DeflParams dp, int* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    Mat Hm{const_cast<double*>(H) + 16 * (long long)i, 4};
    out[i] = subdiag_negligible(Hm, 2, 0, 3, dp) ? 1 : 0;
  }
}

__global__ void k_spike_eval(int count, const double* blk, DeflParams dp, int* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
    const double* r = blk + 7 * (long long)i;
    const int bs = (r[6] == 2.0) ? 2 : 1;
    out[i] = spike_deflatable_blk(r[0], r[1], r[2], r[3], r[4], r[5], bs, dp) ? 1 : 0;
  }
}

// ---------------------------------------------------------------------------
// Diagnostic: the low-latency reciprocal / reciprocal square root of
// fastmath.cuh next to CUDA's IEEE division and square root.
__global__ void k_fastmath_eval(int n, const double* x, double* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double v = x[i];
    out[4 * i + 0] = fast_rcp(v);
    out[4 * i + 1] = 1.0 / v;
    out[4 * i + 2] = (v > 0.0) ? fast_rsqrt(v) : 0.0;
    out[4 * i + 3] = (v > 0.0) ? 1.0 / sqrt(v) : 0.0;
  }
}
