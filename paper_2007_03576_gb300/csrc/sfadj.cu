// sfadj.cu -- adjoint of the real Schur factors (not in the paper): dL/dH for
// a loss L(S, Z) of the standardised factors H = Z S Z^T.
//
// First-order change: dZ = Z Omega (Omega skew), E = Z^T dH Z and
//     dS = E + S Omega - Omega S.
// Omega is fixed by the structure of S: dS stays zero below the diagonal
// blocks, and every 2x2 block stays standardised (equal diagonal entries).
// With blocks p, q (sizes 1 or 2) the conditions below the blocks read
//     S_pp O_pq - O_pq S_qq + sum_{r>p} S_pr O_rq - sum_{r<q} O_pr S_rq = -E_pq,
// a block-triangular Sylvester system for the blocks O_pq (p > q); each 2x2
// block's rotation w_p (Omega's entry inside the block) follows from
//     2 (b_p + c_p) w_p + [...] = -(E_kk - E_k+1,k+1),  S_pp = [[a, b], [c, a]].
// Reverse mode: with G = S^T Sbar - Sbar S^T + Z^T Zbar and W = G - G^T, the
// cotangents of the unknowns are W's entries there; the transposed system
// M^T y = -W is solved in the reverse order -- block columns q from right to
// left, and in each column p from top to bottom:
//     S_pp^T y_pq - y_pq S_qq^T = -W_pq + sum_{q<q'<p} y_pq' S_qq'^T
//                                - sum_{q<p'<p} S_p'p^T y_p'q - (rotation terms),
// the rotation terms coming from eta_p = -W_{k+1,k} / (2 (b_p + c_p)) of the
// 2x2 blocks.  Then Ebar = Sbar + y (on the entries below the blocks) + eta
// (+ on S_kk, - on S_k+1,k+1) and dL/dH = Z Ebar Z^T.
//
// Kernels: three GEMM tasks for G (k_gemm), k_sfa_solve (one block per
// matrix: per block column a parallel pass builds every right-hand side of the
// column, then the column is solved top-down, each solved block updating the
// right-hand sides below it), two GEMMs for Z Ebar Z^T.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/schur_gb300.h"
#include "gemm.cuh"
#include "host.h"

#define SFA_THREADS 256
#define SFA_NMAX 1024

namespace {

struct SfaDesc {
  const double *S, *Z, *Sb, *Zb;
  double* dH;
  double* ws;   // 4 n^2 doubles: G, Y, E, T (each n x n, ld n)
  long long lds, ldz, ldsb, ldzb, lddh;
  int n, pad;
};

// Solve the (sp sq) x (sp sq) Kronecker form of A^T Y - Y B^T = R (A sp x sp,
// B sq x sq, column-major 2x2 arrays) by Gaussian elimination with partial
// pivoting; a pivot below smin is replaced by smin.
__device__ void small_sylvester_t(int sp, int sq, const double* A, const double* B, const double* R, double* Y,
                                  double smin) {
  const int nn = sp * sq;
  double K[4][5];
  // unknown index u = r + sp * c  (Y(r, c)); (A^T Y)(r, c) = sum_k A(k, r) Y(k, c);
  // (Y B^T)(r, c) = sum_k Y(r, k) B(c, k)
  for (int u = 0; u < nn; ++u) {
    const int r = u % sp, c = u / sp;
    for (int v = 0; v < nn; ++v) {
      const int rr = v % sp, cc = v / sp;
      double val = 0.0;
      if (cc == c) val += A[rr + 2 * r];
      if (rr == r) val -= B[c + 2 * cc];
      K[u][v] = val;
    }
    K[u][nn] = R[r + 2 * c];
  }
  for (int col = 0; col < nn; ++col) {
    int piv = col;
    for (int r = col + 1; r < nn; ++r)
      if (fabs(K[r][col]) > fabs(K[piv][col])) piv = r;
    if (piv != col)
      for (int c = 0; c <= nn; ++c) {
        const double t = K[col][c];
        K[col][c] = K[piv][c];
        K[piv][c] = t;
      }
    if (fabs(K[col][col]) < smin) K[col][col] = (K[col][col] < 0.0) ? -smin : smin;
    for (int r = col + 1; r < nn; ++r) {
      const double f = K[r][col] / K[col][col];
      for (int c = col; c <= nn; ++c) K[r][c] = fma(-f, K[col][c], K[r][c]);
    }
  }
  double x[4];
  for (int r = nn - 1; r >= 0; --r) {
    double s = K[r][nn];
    for (int c = r + 1; c < nn; ++c) s = fma(-K[r][c], x[c], s);
    x[r] = s / K[r][r];
  }
  for (int u = 0; u < nn; ++u) Y[(u % sp) + 2 * (u / sp)] = x[u];
}

__global__ void __launch_bounds__(SFA_THREADS) k_sfa_solve(const SfaDesc* __restrict__ descs, int ndesc) {
  extern __shared__ double smem[];
  const SfaDesc& d = descs[blockIdx.x];
  const int n = d.n;
  double* rhs0 = smem;             // right-hand sides of the current block column (column 0 / 1 of q)
  double* rhs1 = rhs0 + n;
  double* eta = rhs1 + n;          // per row: eta of the 2x2 block the row starts (0 otherwise)
  int* bstart = (int*)(eta + n);   // per row: first row of its diagonal block
  __shared__ double ysh[4];
  __shared__ double fro;
  (void)ndesc;
  const double* S = d.S;
  const long long lds = d.lds;
  const double* G = d.ws;
  double* Y = d.ws + (long long)n * n;
  double* E = Y + (long long)n * n;
  auto Sx = [&](int i, int j) { return S[i + j * lds]; };
  auto Wx = [&](int i, int j) { return G[i + (long long)j * n] - G[j + (long long)i * n]; };
  // block structure (rows of a 2x2 block share its first row) and ||S||_F
  __shared__ double red[SFA_THREADS / 32];
  if (threadIdx.x == 0) {
    int i = 0;
    while (i < n) {
      if (i + 1 < n && Sx(i + 1, i) != 0.0) {
        bstart[i] = i;
        bstart[i + 1] = i;
        i += 2;
      } else {
        bstart[i] = i;
        i += 1;
      }
    }
  }
  double a = 0.0;
  for (long long idx = threadIdx.x; idx < (long long)n * n; idx += blockDim.x) {
    const int i = (int)(idx % n), j = (int)(idx / n);
    Y[i + (long long)j * n] = 0.0;
    if (i <= j + 1) {
      const double v = Sx(i, j);
      a = fma(v, v, a);
    }
  }
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < SFA_THREADS / 32; ++w) t += red[w];
    fro = t;
  }
  // eta of each 2x2 block (b + c = 0 leaves its rotation free: eta = 0)
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    double e = 0.0;
    if (bstart[i] == i && i + 1 < n && bstart[i + 1] == i) {
      const double bc = Sx(i, i + 1) + Sx(i + 1, i);
      if (bc != 0.0) e = -Wx(i + 1, i) / (2.0 * bc);
    }
    eta[i] = e;
  }
  __syncthreads();
  const double smin = fmax(0x1p-52 * sqrt(fro), 1e-300);
  // block columns q from the right
  int q1 = n;   // one past the last row of block q
  while (q1 > 0) {
    const int q0 = bstart[q1 - 1];
    const int sq = q1 - q0;
    // (a) right-hand sides of every row below block q
    for (int i = q1 + threadIdx.x; i < n; i += blockDim.x) {
      const int p0 = bstart[i];
      const int r = i - p0;
      const int sp = (p0 + 1 < n && bstart[p0 + 1] == p0) ? 2 : 1;
      for (int c = 0; c < sq; ++c) {
        double v = -Wx(i, q0 + c);
        double acc = 0.0;
        for (int cc = q1; cc < p0; ++cc) acc = fma(Y[i + (long long)cc * n], Sx(q0 + c, cc), acc);
        v += acc;
        const double sqp = Sx(q0 + c, i);
        const double dc = (c == 0) ? 1.0 : -1.0, dr = (r == 0) ? 1.0 : -1.0;
        if (sq == 2) v -= eta[q0] * dc * sqp;
        if (sp == 2) v += eta[p0] * dr * sqp;
        if (c == 0) rhs0[i] = v; else rhs1[i] = v;
      }
    }
    __syncthreads();
    // (b) the column, top-down
    int p0 = q1;
    while (p0 < n) {
      const int sp = (p0 + 1 < n && bstart[p0 + 1] == p0) ? 2 : 1;
      if (threadIdx.x == 0) {
        double A[4] = {Sx(p0, p0), sp == 2 ? Sx(p0 + 1, p0) : 0.0, sp == 2 ? Sx(p0, p0 + 1) : 0.0,
                       sp == 2 ? Sx(p0 + 1, p0 + 1) : 0.0};
        double B[4] = {Sx(q0, q0), sq == 2 ? Sx(q0 + 1, q0) : 0.0, sq == 2 ? Sx(q0, q0 + 1) : 0.0,
                       sq == 2 ? Sx(q0 + 1, q0 + 1) : 0.0};
        double R[4] = {rhs0[p0], sp == 2 ? rhs0[p0 + 1] : 0.0, sq == 2 ? rhs1[p0] : 0.0,
                       (sp == 2 && sq == 2) ? rhs1[p0 + 1] : 0.0};
        double Yv[4] = {0.0, 0.0, 0.0, 0.0};
        small_sylvester_t(sp, sq, A, B, R, Yv, smin);
        for (int c = 0; c < sq; ++c)
          for (int r = 0; r < sp; ++r) {
            ysh[r + 2 * c] = Yv[r + 2 * c];
            Y[(p0 + r) + (long long)(q0 + c) * n] = Yv[r + 2 * c];
          }
      }
      __syncthreads();
      // rows below block p: rhs -= S_{p,p''}^T y_pq
      for (int i = p0 + sp + threadIdx.x; i < n; i += blockDim.x) {
        const double s0 = Sx(p0, i), s1 = (sp == 2) ? Sx(p0 + 1, i) : 0.0;
        rhs0[i] -= fma(s1, ysh[1], s0 * ysh[0]);
        if (sq == 2) rhs1[i] -= fma(s1, ysh[3], s0 * ysh[2]);
      }
      __syncthreads();
      p0 += sp;
    }
    q1 = q0;
  }
  // Ebar = Sbar + y below the blocks + eta on the 2x2 blocks' diagonals
  const double* Sb = d.Sb;
  for (long long idx = threadIdx.x; idx < (long long)n * n; idx += blockDim.x) {
    const int i = (int)(idx % n), j = (int)(idx / n);
    double v = Sb[i + j * d.ldsb];
    if (bstart[i] > bstart[j]) v += Y[i + (long long)j * n];
    if (i == j) {
      const int b0 = bstart[i];
      if (b0 + 1 < n && bstart[b0 + 1] == b0) v += (i == b0) ? eta[b0] : -eta[b0];
    }
    E[i + (long long)j * n] = v;
  }
}

struct SfaMatrix {
  int n;
  const double *S, *Z, *Sb, *Zb;
  double* dH;
  int lds, ldz, ldsb, ldzb, lddh;
};

int run_sfa(const std::vector<SfaMatrix>& ms, const schur_opts* opts) {
  schur_opts o;
  schur::read_opts(opts, &o);
  cudaStream_t st = (cudaStream_t)o.stream;
  const int nb = (int)ms.size();
  size_t ws_doubles = 0;
  int nmax = 1;
  for (auto& m : ms) {
    ws_doubles += 4 * (size_t)m.n * m.n;
    nmax = std::max(nmax, m.n);
  }
  const size_t desc_bytes = ((size_t)nb * sizeof(SfaDesc) + 255) / 256 * 256;
  const size_t task_bytes = ((size_t)5 * nb * sizeof(GemmTask) + 255) / 256 * 256;
  const size_t need = ws_doubles * sizeof(double) + desc_bytes + task_bytes;
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
    double* wsb = (double*)mem;
    SfaDesc* dd = (SfaDesc*)(mem + ws_doubles * sizeof(double));
    GemmTask* dt = (GemmTask*)((char*)dd + desc_bytes);
    std::vector<SfaDesc> hd(nb);
    std::vector<GemmTask> tasks;
    auto task = [&](const double* A, long long lda, int ta, const double* B, long long ldb, int tb, double* C,
                    long long ldc, int N, double alpha, double beta) {
      GemmTask t;
      memset(&t, 0, sizeof(t));
      t.A = A; t.B = B; t.C = C; t.lda = lda; t.ldb = ldb; t.ldc = ldc;
      t.M = N; t.N = N; t.K = N; t.transA = ta; t.transB = tb; t.alpha = alpha; t.beta = beta;
      t.tiles_n = (N + 63) / 64;
      t.ntile = t.tiles_n * t.tiles_n;
      tasks.push_back(t);
    };
    size_t off = 0;
    for (int b = 0; b < nb; ++b) {
      const SfaMatrix& m = ms[b];
      hd[b] = SfaDesc{m.S, m.Z, m.Sb, m.Zb, m.dH, wsb + off, m.lds, m.ldz, m.ldsb, m.ldzb, m.lddh, m.n, 0};
      off += 4 * (size_t)m.n * m.n;
    }
    // phase k of every matrix is task k * nb + b
    for (int b = 0; b < nb; ++b) {
      const SfaDesc& d = hd[b];
      task(d.S, d.lds, 1, d.Sb, d.ldsb, 0, d.ws, d.n, d.n, 1.0, 0.0);            // G = S^T Sbar
    }
    for (int b = 0; b < nb; ++b) {
      const SfaDesc& d = hd[b];
      task(d.Sb, d.ldsb, 0, d.S, d.lds, 1, d.ws, d.n, d.n, -1.0, 1.0);           // G -= Sbar S^T
    }
    for (int b = 0; b < nb; ++b) {
      const SfaDesc& d = hd[b];
      task(d.Z, d.ldz, 1, d.Zb, d.ldzb, 0, d.ws, d.n, d.n, 1.0, 1.0);            // G += Z^T Zbar
    }
    for (int b = 0; b < nb; ++b) {
      const SfaDesc& d = hd[b];
      const long long nn = (long long)d.n * d.n;
      task(d.Z, d.ldz, 0, d.ws + 2 * nn, d.n, 0, d.ws + 3 * nn, d.n, d.n, 1.0, 0.0);   // T = Z Ebar
    }
    for (int b = 0; b < nb; ++b) {
      const SfaDesc& d = hd[b];
      const long long nn = (long long)d.n * d.n;
      task(d.ws + 3 * nn, d.n, 0, d.Z, d.ldz, 1, d.dH, d.lddh, d.n, 1.0, 0.0);   // dH = T Z^T
    }
    std::vector<int> phase_tiles(5, 0);
    for (int ph = 0; ph < 5; ++ph) {
      int tile = 0;
      for (int b = 0; b < nb; ++b) {
        GemmTask& t = tasks[ph * nb + b];
        t.tile0 = tile;
        tile += t.ntile;
      }
      phase_tiles[ph] = tile;
    }
    schur::ck_at(cudaMemcpyAsync(dd, hd.data(), nb * sizeof(SfaDesc), cudaMemcpyHostToDevice, st), __LINE__);
    schur::ck_at(cudaMemcpyAsync(dt, tasks.data(), tasks.size() * sizeof(GemmTask), cudaMemcpyHostToDevice, st),
                 __LINE__);
    const int nsm = schur::num_sms();
    auto gemm_phase = [&](int ph) {
      k_gemm<<<std::min(phase_tiles[ph], 4 * nsm), 256, 0, st>>>(dt + ph * nb, nb, phase_tiles[ph]);
      schur::ck_at(cudaGetLastError(), __LINE__);
    };
    gemm_phase(0);
    gemm_phase(1);
    gemm_phase(2);
    const size_t smem = (size_t)nmax * (3 * sizeof(double) + sizeof(int));
    k_sfa_solve<<<nb, SFA_THREADS, smem, st>>>(dd, nb);
    schur::ck_at(cudaGetLastError(), __LINE__);
    gemm_phase(3);
    gemm_phase(4);
    schur::ck_at(cudaStreamSynchronize(st), __LINE__);
    schur::g_stats.kernel_launches = 6;
  } catch (const schur::CudaError&) {
    rc = SCHUR_ERR_CUDA;
  }
  if (own) cudaFree(mem);
  return rc;
}

}  // namespace

extern "C" int schur_factor_backward(int n, const double* S, int lds, const double* Z, int ldz, const double* Sbar,
                                     int ldsb, const double* Zbar, int ldzb, double* dH, int lddh,
                                     const schur_opts* opts) {
  if (n < 0 || n > SFA_NMAX) return -1;
  if (n == 0) return SCHUR_OK;
  if (!S) return -2;
  if (lds < n) return -3;
  if (!Z) return -4;
  if (ldz < n) return -5;
  if (!Sbar) return -6;
  if (ldsb < n) return -7;
  if (!Zbar) return -8;
  if (ldzb < n) return -9;
  if (!dH) return -10;
  if (lddh < n) return -11;
  memset(&schur::g_stats, 0, sizeof(schur::g_stats));
  std::vector<SfaMatrix> ms{SfaMatrix{n, S, Z, Sbar, Zbar, dH, lds, ldz, ldsb, ldzb, lddh}};
  return run_sfa(ms, opts);
}

extern "C" int schur_factor_backward_batched(int batch, const int* n, double* const* S, const int* lds,
                                             double* const* Z, const int* ldz, double* const* Sbar, const int* ldsb,
                                             double* const* Zbar, const int* ldzb, double* const* dH,
                                             const int* lddh, const schur_opts* opts) {
  if (batch < 0) return -1;
  if (batch == 0) return SCHUR_OK;
  if (!n) return -2;
  if (!S) return -3;
  if (!lds) return -4;
  if (!Z) return -5;
  if (!ldz) return -6;
  if (!Sbar) return -7;
  if (!ldsb) return -8;
  if (!Zbar) return -9;
  if (!ldzb) return -10;
  if (!dH) return -11;
  if (!lddh) return -12;
  std::vector<SfaMatrix> ms(batch);
  for (int b = 0; b < batch; ++b) {
    if (n[b] < 1 || n[b] > SFA_NMAX) return -2;
    if (!S[b]) return -3;
    if (lds[b] < n[b]) return -4;
    if (!Z[b]) return -5;
    if (ldz[b] < n[b]) return -6;
    if (!Sbar[b]) return -7;
    if (ldsb[b] < n[b]) return -8;
    if (!Zbar[b]) return -9;
    if (ldzb[b] < n[b]) return -10;
    if (!dH[b]) return -11;
    if (lddh[b] < n[b]) return -12;
    ms[b] = SfaMatrix{n[b], S[b], Z[b], Sbar[b], Zbar[b], dH[b], lds[b], ldz[b], ldsb[b], ldzb[b], lddh[b]};
  }
  memset(&schur::g_stats, 0, sizeof(schur::g_stats));
  return run_sfa(ms, opts);
}
