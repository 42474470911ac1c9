// batched.cu -- many independent Hessenberg matrices in one persistent launch.
//
// Not in the paper (batching of the method).  Each thread block takes matrices
// from an atomic work queue, largest first, and runs the whole iteration of
// Sec. 2.1 on its matrix: vigilant-deflation scan, double-shift QR for blocks
// of at most nmin rows (Sec. 2.2), AED with the window held in shared memory
// (Sec. 2.5) and tightly-coupled multishift sweeps (Sec. 2.3).  One block owns
// the whole matrix, so reflectors are applied directly to H and Z (no window
// accumulation: it would only add flops); within a sweep step every bulge's
// reflector is built at once by its own thread and the left/right products of
// all bulges run in two phases.  Shifts/window per size bucket come from the
// autotuner (api.autotune_batched) or the default table.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/schur_gb300.h"
#include "cta.cuh"
#include "host.h"

#include "batched.cuh"

struct BShared {
  double v1[MAX_BULGES_PER_CHAIN], v2[MAX_BULGES_PER_CHAIN], tau[MAX_BULGES_PER_CHAIN];
  int k[MAX_BULGES_PER_CHAIN], nr[MAX_BULGES_PER_CHAIN];
  int ival[4];
  double dval[2];
};

// ---------------------------------------------------------------------------
// Block-level products with an L x L transform V (global, ld = L):
//   side 0: X = A[r0:r0+L, c0:c0+nv] <- V^T X      (columns of X staged)
//   side 1: X = A[r0:r0+nv, c0:c0+L] <- X V        (rows of X staged)
// stage: shared memory for L x B_STAGE_COLS doubles.
// ---------------------------------------------------------------------------
__device__ void cta_window_product(const Mat& A, int side, int r0, int c0, int nv, int L, const double* V,
                                   double* stage) {
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int v0 = 0; v0 < nv; v0 += B_STAGE_COLS) {
    const int cb = min(B_STAGE_COLS, nv - v0);
    // stage[k * B_STAGE_COLS + v] = element k of vector v
    for (int idx = tid; idx < L * cb; idx += nt) {
      int k, v;
      if (side == 0) {
        k = idx % L;
        v = idx / L;
        stage[k * B_STAGE_COLS + v] = A(r0 + k, c0 + v0 + v);
      } else {
        v = idx % cb;
        k = idx / cb;
        stage[k * B_STAGE_COLS + v] = A(r0 + v0 + v, c0 + k);
      }
    }
    __syncthreads();
    // outputs (i, v): y_v[i] = sum_k V[k, i] x_v[k]; at most
    // B_NW_MAX * B_STAGE_COLS / blockDim = 16 outputs per thread
    double acc[16];
    int cnt = 0;
    for (int o = tid; o < L * cb && cnt < 16; o += nt, ++cnt) {
      int v = o % cb, i = o / cb;
      const double* vc = V + (long long)i * L;
      double a = 0.0;
      for (int k = 0; k < L; ++k) a = fma(vc[k], stage[k * B_STAGE_COLS + v], a);
      acc[cnt] = a;
    }
    __syncthreads();
    cnt = 0;
    for (int o = tid; o < L * cb && cnt < 16; o += nt, ++cnt) {
      int v = o % cb, i = o / cb;
      if (side == 0)
        A(r0 + i, c0 + v0 + v) = acc[cnt];
      else
        A(r0 + v0 + v, c0 + i) = acc[cnt];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Multishift sweep (Sec. 2.3) on [lo, hi] of the n x n H, reflectors applied
// directly to all of H's columns/rows and to Z.  Bulge j (pair j) sits at row
// k = lo + t - 3 j at step t; per step: (A) each bulge's reflector by its own
// thread, (B) all left products, (C) all right products (and Z).
// ---------------------------------------------------------------------------
__device__ void cta_ms_sweep(const Mat& H, int n, int lo, int hi, const double* pairs, int nb, const Mat& Z,
                             int zrows, BShared* bs, double* flops) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int steps = (hi - lo) + 3 * (nb - 1);
  for (int t = 0; t < steps; ++t) {
    if (tid < nb) {
      int j = tid;
      int k = lo + t - 3 * j;
      if (k >= lo && k <= hi - 1) {
        int nr = min(3, hi - k + 1);
        double x0, x1, x2 = 0.0;
        if (k == lo) {
          double ssum = pairs[2 * j], sprod = pairs[2 * j + 1];
          double h00 = H(lo, lo), h01 = H(lo, lo + 1), h10 = H(lo + 1, lo), h11 = H(lo + 1, lo + 1);
          x0 = fma(h00, h00, fma(h01, h10, fma(-ssum, h00, sprod)));
          x1 = h10 * (h00 + h11 - ssum);
          if (nr == 3) x2 = h10 * H(lo + 2, lo + 1);
        } else {
          x0 = H(k, k - 1);
          x1 = H(k + 1, k - 1);
          if (nr == 3) x2 = H(k + 2, k - 1);
        }
        double v1, v2, tau, beta;
        house3(nr, x0, x1, x2, v1, v2, tau, beta);
        if (k > lo) {
          H(k, k - 1) = beta;
          H(k + 1, k - 1) = 0.0;
          if (nr == 3) H(k + 2, k - 1) = 0.0;
        }
        bs->v1[j] = v1;
        bs->v2[j] = v2;
        bs->tau[j] = tau;
        bs->k[j] = k;
        bs->nr[j] = nr;
      } else {
        bs->nr[j] = 0;
      }
    }
    __syncthreads();
    if (tid == 0) {   // algorithmic flops: 4 nr per row / column entry of each reflector
      double e = 0.0;
      for (int j = 0; j < nb; ++j)
        if (bs->nr[j] != 0 && bs->tau[j] != 0.0)
          e += 4.0 * bs->nr[j] * ((n - bs->k[j]) + (min(bs->k[j] + 3, hi) + 1) + zrows);
      *flops += e;
    }
    {  // (B) left products, items spread over all threads
      int base = 0;
      for (int j = 0; j < nb; ++j) {
        int nr = bs->nr[j];
        if (nr == 0 || bs->tau[j] == 0.0) continue;
        int k = bs->k[j];
        int cnt = n - k;
        double v1 = bs->v1[j], v2 = bs->v2[j], tau = bs->tau[j];
        int start = (tid - base) % nt;
        if (start < 0) start += nt;
        for (int c = start; c < cnt; c += nt) {
          double* col = &H(k, k + c);
          double a0 = col[0], a1 = col[1], a2 = (nr == 3) ? col[2] : 0.0;
          double s = tau * fma(v2, a2, fma(v1, a1, a0));
          col[0] = a0 - s;
          col[1] = fma(-s, v1, a1);
          if (nr == 3) col[2] = fma(-s, v2, a2);
        }
        base += cnt;
      }
    }
    __syncthreads();
    {  // (C) right products on H rows 0..min(k+3, hi) and Z rows 0..zrows-1
      int base = 0;
      for (int j = 0; j < nb; ++j) {
        int nr = bs->nr[j];
        if (nr == 0 || bs->tau[j] == 0.0) continue;
        int k = bs->k[j];
        double v1 = bs->v1[j], v2 = bs->v2[j], tau = bs->tau[j];
        int rh = min(k + 3, hi) + 1;
        int cnt = rh + zrows;
        int start = (tid - base) % nt;
        if (start < 0) start += nt;
        for (int it = start; it < cnt; it += nt) {
          const Mat& M = (it < rh) ? H : Z;
          int r = (it < rh) ? it : it - rh;
          double* c0 = &M(r, k);
          double a0 = c0[0], a1 = c0[M.ld], a2 = (nr == 3) ? c0[2 * M.ld] : 0.0;
          double s = tau * fma(v2, a2, fma(v1, a1, a0));
          c0[0] = a0 - s;
          c0[M.ld] = fma(-s, v1, a1);
          if (nr == 3) c0[2 * M.ld] = fma(-s, v2, a2);
        }
        base += cnt;
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// AED (Sec. 2.5) on the trailing nw x nw window of [ktop, kbot]: window in
// shared memory (T), transform V in global scratch; window and spike written
// back and V applied to the rest of H and to Z only if something deflated.
// Returns nd; candidates in scratch, their count in bs->ival[1].
// ---------------------------------------------------------------------------
__device__ int cta_aed_direct(const Mat& H, int n, const Mat& Z, int ktop, int kbot, int nw, const DeflParams& dp,
                              const BatchedScratch& sc, double* smem_T, double* stage, CtaShared* sh, BShared* bs) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int kwtop = kbot - nw + 1;
  const int ldt = nw | 1;
  Mat T{smem_T, ldt};
  Mat V{sc.V, nw};
  for (int j = 0; j < nw; ++j)
    for (int i = tid; i < nw; i += nt) {
      T(i, j) = (i <= j + 1) ? H(kwtop + i, kwtop + j) : 0.0;
      V(i, j) = (i == j) ? 1.0 : 0.0;
    }
  double s = (kwtop > ktop) ? H(kwtop, kwtop - 1) : 0.0;
  __syncthreads();
  DeflParams dpw = dp;
  dpw.n = nw;
  int info = cta_francis(T, nw, 0, nw - 1, V, nw, dpw, sh, nullptr, &bs->dval[1]);
  double top;
  int nd = cta_aed_post(T, nw, info, s, V, dp, sc.vbuf, sc.cand_re, sc.cand_im, &bs->ival[1], &top, &bs->ival[2], sh);
  __syncthreads();
  if (nd > 0) {
    for (int j = 0; j < nw; ++j)
      for (int i = tid; i < nw; i += nt) H(kwtop + i, kwtop + j) = (i <= j + 1) ? T(i, j) : 0.0;
    if (kwtop > ktop)
      for (int i = tid; i < nw; i += nt) H(kwtop + i, kwtop - 1) = (i == 0) ? top : 0.0;
    __syncthreads();
    if (tid == 0) bs->dval[1] += 2.0 * nw * nw * ((double)(n - kbot - 1) + kwtop + n);
    if (kbot + 1 < n) cta_window_product(H, 0, kwtop, kbot + 1, n - kbot - 1, nw, sc.V, stage);
    if (kwtop > 0) cta_window_product(H, 1, 0, kwtop, kwtop, nw, sc.V, stage);
    cta_window_product(Z, 1, 0, kwtop, n, nw, sc.V, stage);
  }
  return nd;
}

// ---------------------------------------------------------------------------
// The iteration of Sec. 2.1 on one matrix (same rules as the single-matrix
// driver).  Returns 0 or 1 + the last row of the block that hit the
// iteration limit.
// ---------------------------------------------------------------------------
__device__ int cta_schur_one(const Mat& H, int n, const Mat& Z, const BatchedParams& P, const DeflParams& dp,
                             const BatchedScratch& sc, double* smem_T, double* stage, CtaShared* sh, BShared* bs) {
  int kbot = n - 1;
  const int itmax = 30 * max(10, n);
  int it = 0, ndfl = 1;
  for (int guard = 0; guard < 64 * max(10, n) && kbot >= 0; ++guard) {
    int ktop = cta_find_ktop(H, 0, kbot, dp, sh);
    int m = kbot - ktop + 1;
    if (m == 1) {
      kbot -= 1;
      ndfl = 1;
      continue;
    }
    if (m == 2) {
      cta_standardize_block(H, ktop, n, Z, n, sh);
      kbot -= 2;
      ndfl = 1;
      continue;
    }
    if (m <= P.nmin) {
      int info = cta_francis(H, n, ktop, kbot, Z, n, dp, sh, nullptr, &bs->dval[1]);
      if (info) return info;
      kbot = ktop - 1;
      ndfl = 1;
      continue;
    }
    if (++it > itmax) return kbot + 1;
    int b = 0;
    while (b + 1 < P.nbuckets && m > P.bucket_max_n[b]) ++b;
    int ns_max = min(P.ns[b], 2 * MAX_BULGES_PER_CHAIN);
    int nw = min(min(P.nw[b], m), P.nw_max);
    int nd = cta_aed_direct(H, n, Z, ktop, kbot, nw, dp, sc, smem_T, stage, sh, bs);
    kbot -= nd;
    ndfl = (nd > 0) ? 1 : ndfl + 1;
    m = kbot - ktop + 1;
    if (m <= P.nmin) continue;
    if (nd > 0 && 100 * nd > P.nibble * nw) continue;
    if (threadIdx.x == 0)
      bs->ival[0] = make_shift_pairs(H, ktop, kbot, ns_max, ndfl, P.exc_period, sc.cand_re, sc.cand_im, bs->ival[1],
                                     sc.pairs);
    __syncthreads();
    int np = bs->ival[0];
    __syncthreads();
    if (np > 0) cta_ms_sweep(H, n, ktop, kbot, sc.pairs, np, Z, n, bs, &bs->dval[1]);
  }
  return (kbot >= 0) ? kbot + 1 : 0;
}

__global__ void __launch_bounds__(CTA_THREADS, 3) k_batched(const BatchedDesc* __restrict__ desc,
                                                         const int* __restrict__ order, int batch, int* counter,
                                                         int* info, BatchedScratch* scratch, BatchedParams P) {
  extern __shared__ double smem[];
  __shared__ CtaShared sh;
  __shared__ BShared bs;
  __shared__ int s_item;
  double* smem_T = smem;
  double* stage = smem + (size_t)(P.nw_max | 1) * P.nw_max;
  const BatchedScratch sc = scratch[blockIdx.x];
  if (threadIdx.x == 0) bs.dval[1] = 0.0;
  // bounded: every iteration consumes one queue entry
  for (int guard = 0; guard <= batch; ++guard) {
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    int item = s_item;
    __syncthreads();
    if (item >= batch) break;
    const BatchedDesc d = desc[order[item]];
    const int n = d.n;
    Mat H{d.H, d.ldh};
    Mat Z{d.Z, d.ldz};
    // zero below the subdiagonal
    for (int j = 0; j < n; ++j)
      for (int i = j + 2 + threadIdx.x; i < n; i += blockDim.x) H(i, j) = 0.0;
    DeflParams dp;
    dp.mode = P.mode;
    dp.thold = P.thold;
    dp.n = n;
    dp.normH = 0.0;
    if (P.mode == 1) {  // ||H||_F for the norm-stable conditions
      double ssq = 0.0;
      for (int j = 0; j < n; ++j)
        for (int i = threadIdx.x; i <= min(j + 1, n - 1); i += blockDim.x) ssq = fma(H(i, j), H(i, j), ssq);
      for (int o = 16; o > 0; o >>= 1) ssq += __shfl_xor_sync(0xffffffffu, ssq, o);
      if ((threadIdx.x & 31) == 0) sh.red[threadIdx.x >> 5] = ssq;
      __syncthreads();
      if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += sh.red[w];
        bs.dval[0] = sqrt(t);
      }
      __syncthreads();
      dp.normH = bs.dval[0];
    }
    __syncthreads();
    int rc = (n >= 1) ? cta_schur_one(H, n, Z, P, dp, sc, smem_T, stage, &sh, &bs) : 0;
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      int s = -1;
      if (j + 1 < n && H(j + 1, j) != 0.0) s = j;
      else if (j > 0 && H(j, j - 1) != 0.0) s = j - 1;
      if (s < 0) {
        d.wr[j] = H(j, j);
        d.wi[j] = 0.0;
      } else {
        double r1, i1, r2, i2;
        eig2x2(H(s, s), H(s, s + 1), H(s + 1, s), H(s + 1, s + 1), r1, i1, r2, i2);
        d.wr[j] = (j == s) ? r1 : r2;
        d.wi[j] = (j == s) ? i1 : i2;
      }
    }
    if (threadIdx.x == 0) info[order[item]] = rc;
    __syncthreads();
  }
  if (threadIdx.x == 0 && sc.flops) *sc.flops += bs.dval[1];
}

__global__ void k_batched_prep_z(const BatchedDesc* desc, int batch, int zinit) {
  if (zinit) return;
  for (int b = blockIdx.x; b < batch; b += gridDim.x) {
    const BatchedDesc d = desc[b];
    for (int j = 0; j < d.n; ++j)
      for (int i = threadIdx.x; i < d.n; i += blockDim.x) d.Z[i + (long long)j * d.ldz] = (i == j) ? 1.0 : 0.0;
  }
}

// ===========================================================================
// Host side
// ===========================================================================
namespace schur {

// Default per-bucket table and double-shift crossover: the autotuner's choice
// (tune.autotune_batched and tune.autotune_batched_nmin on GB300, one wave of
// hess_n matrices per bucket; timings in the profiles folder).  Windows are
// capped for the batched engine's shared-memory window.
static void default_batched_params(BatchedParams& P) {
  memset(&P, 0, sizeof(P));
  P.nmin = 48;
  P.nibble = 14;
  P.exc_period = 6;
  P.nbuckets = 4;
  int mx[4] = {149, 299, 589, 1 << 30};
  int ns[4] = {8, 8, 32, 32};
  int nw[4] = {24, 24, 64, 64};
  for (int b = 0; b < 4; ++b) {
    P.bucket_max_n[b] = mx[b];
    P.ns[b] = ns[b];
    P.nw[b] = nw[b];
  }
  P.nw_max = 64;
}

thread_local BatchedParams g_bparams;
thread_local bool g_bparams_set = false;

}  // namespace schur

using namespace schur;

extern "C" int schur_batched_set_table(int nbuckets, const int* max_n, const int* ns, const int* nw) {
  if (nbuckets < 0 || nbuckets > B_MAX_BUCKETS) return -1;
  if (nbuckets == 0) {
    g_bparams_set = false;
    return SCHUR_OK;
  }
  if (!max_n) return -2;
  if (!ns) return -3;
  if (!nw) return -4;
  BatchedParams P;
  default_batched_params(P);
  P.nbuckets = nbuckets;
  P.nw_max = 4;
  for (int b = 0; b < nbuckets; ++b) {
    if (nw[b] < 4 || nw[b] > B_NW_MAX) return -4;
    if (ns[b] < 2 || ns[b] > 2 * MAX_BULGES_PER_CHAIN) return -3;
    P.bucket_max_n[b] = max_n[b];
    P.ns[b] = ns[b];
    P.nw[b] = nw[b];
    P.nw_max = std::max(P.nw_max, nw[b]);
  }
  P.bucket_max_n[nbuckets - 1] = 1 << 30;
  g_bparams = P;
  g_bparams_set = true;
  return SCHUR_OK;
}

static size_t batched_smem(const BatchedParams& P) {
  return ((size_t)(P.nw_max | 1) * P.nw_max + (size_t)P.nw_max * B_STAGE_COLS) * sizeof(double);
}

// One captured graph per batch shape (batch size, grid, parameters, Z
// initialisation, device): its device buffer holds the descriptors, the
// largest-first order, the queue counter, the per-matrix status, the
// per-block scratch and flop counters.  A call uploads the descriptors and
// the order (the matrices' pointers may change between calls), replays the
// graph (counter reset, Z = I, the persistent kernel) and reads the status
// back.  At most BGRAPH_CACHE shapes are kept; the least recently used one
// is released.
#define BGRAPH_CACHE 4

struct BGraph {
  int dev = -1, batch = 0, grid = 0, zinit = 0;
  BatchedParams P;
  char* mem = nullptr;
  size_t off_desc = 0, off_ord = 0, off_cnt = 0, off_info = 0, off_scr = 0, off_flops = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  unsigned long long used = 0;
  void release() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (mem) cudaFree(mem);
    exec = nullptr;
    graph = nullptr;
    mem = nullptr;
    batch = 0;
  }
};

static std::mutex g_bgraph_mu;
static BGraph g_bgraph[BGRAPH_CACHE];
static unsigned long long g_bgraph_clock = 0;

// Builds the graph of one shape into e (device buffers, scratch layout,
// capture, instantiation).  Throws CudaError.
static void bgraph_build(BGraph& e, int dev, int batch, int grid, int zinit, const BatchedParams& P, size_t smem,
                         cudaStream_t st) {
  e.dev = dev;
  e.batch = batch;
  e.grid = grid;
  e.zinit = zinit;
  e.P = P;
  size_t per_block = ((size_t)P.nw_max * P.nw_max + 6 * (size_t)P.nw_max + 2 * (MAX_BULGES_PER_CHAIN + 4)) *
                     sizeof(double);
  per_block = (per_block + 255) & ~(size_t)255;
  e.off_desc = 0;
  e.off_ord = (e.off_desc + batch * sizeof(BatchedDesc) + 255) & ~(size_t)255;
  e.off_cnt = (e.off_ord + batch * sizeof(int) + 255) & ~(size_t)255;
  e.off_info = e.off_cnt + 256;
  e.off_flops = (e.off_info + batch * sizeof(int) + 255) & ~(size_t)255;
  e.off_scr = (e.off_flops + grid * sizeof(double) + 255) & ~(size_t)255;
  const size_t off_sd = (e.off_scr + grid * sizeof(BatchedScratch) + 255) & ~(size_t)255;
  const size_t total = off_sd + grid * per_block;
  if (cudaMalloc((void**)&e.mem, total) != cudaSuccess) {
    cudaGetLastError();
    e.mem = nullptr;
    throw CudaError{cudaErrorMemoryAllocation};
  }
  std::vector<BatchedScratch> hs(grid);
  for (int g = 0; g < grid; ++g) {
    double* base = (double*)(e.mem + off_sd + g * per_block);
    hs[g].V = base;
    hs[g].vbuf = base + (size_t)P.nw_max * P.nw_max;
    hs[g].cand_re = hs[g].vbuf + 4 * P.nw_max;
    hs[g].cand_im = hs[g].cand_re + P.nw_max;
    hs[g].pairs = hs[g].cand_im + P.nw_max;
    hs[g].flops = (double*)(e.mem + e.off_flops) + g;
  }
  ck_at(cudaMemcpyAsync(e.mem + e.off_scr, hs.data(), grid * sizeof(BatchedScratch), cudaMemcpyHostToDevice, st),
        __LINE__);
  ck_at(cudaStreamSynchronize(st), __LINE__);
  cudaStream_t cap = nullptr;
  ck_at(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), __LINE__);
  cudaError_t err = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (err == cudaSuccess) {
    cudaMemsetAsync(e.mem + e.off_cnt, 0, sizeof(int), cap);
    cudaMemsetAsync(e.mem + e.off_flops, 0, grid * sizeof(double), cap);
    k_batched_prep_z<<<std::min(batch, 4 * num_sms()), CTA_THREADS, 0, cap>>>((BatchedDesc*)(e.mem + e.off_desc),
                                                                              batch, zinit);
    k_batched<<<grid, CTA_THREADS, smem, cap>>>((BatchedDesc*)(e.mem + e.off_desc), (int*)(e.mem + e.off_ord), batch,
                                                (int*)(e.mem + e.off_cnt), (int*)(e.mem + e.off_info),
                                                (BatchedScratch*)(e.mem + e.off_scr), P);
    err = cudaStreamEndCapture(cap, &e.graph);
  }
  cudaStreamDestroy(cap);
  ck_at(err, __LINE__);
  ck_at(cudaGraphInstantiate(&e.exec, e.graph, 0), __LINE__);
}

extern "C" int schur_hessenberg_batched(int batch, const int* n, double* const* H, const int* ldh, double* const* Z,
                                        const int* ldz, double* const* wr, double* const* wi, int* info,
                                        const schur_opts* opts) {
  if (batch < 0) return -1;
  if (batch == 0) return SCHUR_OK;
  if (!n) return -2;
  if (!H) return -3;
  if (!ldh) return -4;
  if (!Z) return -5;
  if (!ldz) return -6;
  if (!wr) return -7;
  if (!wi) return -8;
  if (!info) return -9;
  for (int b = 0; b < batch; ++b) {
    if (n[b] < 1 || n[b] > 1024) return -2;
    if (!H[b]) return -3;
    if (ldh[b] < n[b]) return -4;
    if (!Z[b]) return -5;
    if (ldz[b] < n[b]) return -6;
    if (!wr[b]) return -7;
    if (!wi[b]) return -8;
  }
  schur_opts o;
  read_opts(opts, &o);
  cudaStream_t st = (cudaStream_t)o.stream;
  BatchedParams P;
  if (g_bparams_set)
    P = g_bparams;
  else
    default_batched_params(P);
  if (o.nmin > 0) P.nmin = std::min(o.nmin, NW_SMEM_MAX);
  if (o.nibble > 0) P.nibble = o.nibble;
  P.mode = o.deflation;
  P.thold = o.fixed_thold;
  int rc = SCHUR_OK;
  std::lock_guard<std::mutex> lock(g_bgraph_mu);
  try {
    init_kernel_attributes();
    int dev = 0;
    ck_at(cudaGetDevice(&dev), __LINE__);
    size_t smem = batched_smem(P);
    int per_sm = 0;
    ck_at(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batched, CTA_THREADS, smem), __LINE__);
    int grid = std::min(batch, num_sms() * std::max(1, per_sm));
    const int zinit = o.z_init ? 1 : 0;
    // the cached graph of this shape, else build one in the least recently used slot
    BGraph* e = nullptr;
    for (auto& c : g_bgraph)
      if (c.exec && c.dev == dev && c.batch == batch && c.grid == grid && c.zinit == zinit &&
          memcmp(&c.P, &P, sizeof(P)) == 0)
        e = &c;
    bool built = false;
    if (!e) {
      e = &g_bgraph[0];
      for (auto& c : g_bgraph)
        if (!c.exec || c.used < e->used) e = &c;
      e->release();
      try {
        bgraph_build(*e, dev, batch, grid, zinit, P, smem, st);
      } catch (const CudaError&) {
        e->release();
        throw;
      }
      built = true;
    }
    e->used = ++g_bgraph_clock;
    // this call's descriptors and largest-first order
    std::vector<BatchedDesc> hd(batch);
    std::vector<int> ord(batch);
    for (int b = 0; b < batch; ++b) {
      hd[b] = BatchedDesc{H[b], Z[b], wr[b], wi[b], ldh[b], ldz[b], n[b], 0};
      ord[b] = b;
    }
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int c) { return n[a] > n[c]; });
    ck_at(cudaMemcpyAsync(e->mem + e->off_desc, hd.data(), batch * sizeof(BatchedDesc), cudaMemcpyHostToDevice, st),
          __LINE__);
    ck_at(cudaMemcpyAsync(e->mem + e->off_ord, ord.data(), batch * sizeof(int), cudaMemcpyHostToDevice, st),
          __LINE__);
    ck_at(cudaGraphLaunch(e->exec, st), __LINE__);
    memset(&g_stats, 0, sizeof(g_stats));
    g_stats.kernel_launches = 2;
    g_stats.graph_built = built ? 1 : 0;
    std::vector<double> fl(grid);
    ck_at(cudaMemcpyAsync(info, e->mem + e->off_info, batch * sizeof(int), cudaMemcpyDeviceToHost, st), __LINE__);
    ck_at(cudaMemcpyAsync(fl.data(), e->mem + e->off_flops, grid * sizeof(double), cudaMemcpyDeviceToHost, st),
          __LINE__);
    ck_at(cudaStreamSynchronize(st), __LINE__);
    double tot = 0.0;
    for (double f : fl) tot += f;
    g_stats.reflector_flops = tot;
  } catch (const CudaError&) {
    rc = SCHUR_ERR_CUDA;
  }
  return rc;
}
