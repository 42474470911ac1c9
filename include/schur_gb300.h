/*
 * schur_gb300.h -- C ABI of the GB300 (sm_103a) FP64 Hessenberg -> real Schur
 * library: multishift QR with aggressive early deflation (AED).
 *
 * The method is the one of Myllykoski, "Algorithm 1019: A task-based
 * multi-shift QR/QZ algorithm with aggressive early deflation", ACM TOMS
 * 48(1), 2021:
 *   - Sec. 2.1   the iteration: deflate, decouple, iterate, fail at a limit;
 *   - Sec. 2.2   shifts and bulge chasing (Fig. 1);
 *   - Sec. 2.3   tightly-coupled multishift bulge chains chased through
 *                diagonal windows with an accumulated transform U, applied
 *                off-window by matrix-matrix products (Fig. 2, Fig. 3);
 *   - Sec. 2.5   aggressive early deflation (Fig. 4);
 *   - Sec. 5.6   the deflation conditions (LAPACK-style, norm-stable, fixed).
 * The real Schur form is eq. (schur_form) with the 2x2 blocks of
 * eq. (2by2_blocks), returned in standardised form (equal diagonal entries,
 * off-diagonal entries of opposite sign).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Matrices are FP64, column-major, with a leading dimension ld >= n
 *    (entry (i, j) at p[i + j * ld]).
 *  - Every matrix / vector pointer is a DEVICE pointer owned by the caller,
 *    unless the argument's comment says "host".  The library never frees
 *    caller memory.
 *  - Work is issued on opts->stream (a cudaStream_t; NULL = the legacy default
 *    stream).  The functions return after the result is complete (they read
 *    a few control scalars back from the device during the iteration).
 *  - Scratch: if opts->workspace is non-NULL and opts->workspace_bytes is at
 *    least the size reported by the matching *_workspace_size call, the
 *    library allocates no device memory; otherwise it allocates (and frees)
 *    its own scratch inside the call.  A caller workspace must be 256-byte
 *    aligned (cudaMalloc's alignment); a smaller or misaligned one returns
 *    SCHUR_ERR_WORKSPACE before any device work.
 *  - Return codes: SCHUR_OK (0) on success; a negative value -(i) when
 *    argument i (1-based) is invalid; SCHUR_ERR_* below for other errors;
 *    a positive value k > 0 when the iteration limit was reached: rows
 *    0..k-1 may still contain unreduced blocks (H and Z then hold a valid
 *    orthogonal similarity of the input, as in LAPACK's dhseqr).
 *  - No C++ exception crosses this interface.
 */
#ifndef SCHUR_GB300_H
#define SCHUR_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SCHUR_OK 0
#define SCHUR_ERR_NONFINITE (-1001) /* H contains NaN or Inf */
#define SCHUR_ERR_CUDA (-1002)      /* a CUDA runtime call failed */
#define SCHUR_ERR_NOMEM (-1003)     /* scratch allocation failed */
#define SCHUR_ERR_WORKSPACE (-1004) /* caller workspace too small */
#define SCHUR_ERR_UNSUPPORTED (-1005)
#define SCHUR_ERR_TOO_LARGE (-1006) /* order above the fixed limit of schur_hessenberg_noalloc */

/* Deflation conditions of Sec. 5.6. */
#define SCHUR_DEFLATION_LAPACK 0 /* item 1 (the paper's experiments) */
#define SCHUR_DEFLATION_NORM 1   /* item 2, norm-stable */
#define SCHUR_DEFLATION_FIXED 2  /* item 3, |entry| <= fixed_thold */

typedef struct {
  int struct_size;     /* sizeof(schur_opts); set by schur_default_opts.
                          Every entry point reads the first struct_size
                          bytes over the defaults; struct_size <= 0 reads
                          the whole struct of this header's layout */
  int n_shifts;        /* shifts per sweep (even); 0 = size table */
  int aed_window;      /* AED window nw; 0 = size table */
  int bulges_per_chain;/* bulges chased together in one window; 0 = auto */
  int nmin;            /* blocks of at most nmin rows use double-shift QR; 0 = 75 */
  int nibble;          /* repeat AED when it deflates > nibble % of nw; 0 = 14 */
  int deflation;       /* SCHUR_DEFLATION_* */
  double fixed_thold;  /* threshold for SCHUR_DEFLATION_FIXED */
  int want_z;          /* 1: accumulate Z (default), 0: Z is not referenced */
  int z_init;          /* 0: Z is set to I on entry; 1: Z holds Q1 and is
                          multiplied in place (Z <- Z * Z_QR) */
  void* stream;        /* cudaStream_t */
  void* workspace;     /* optional device scratch (see conventions) */
  size_t workspace_bytes;
  int timing;          /* 1: record per-phase device time (CUDA events) in
                          schur_stats; 0 (default): no events */
  int nmin_window;     /* AED windows of at most this order are reduced to
                          Schur form by double-shift QR in one thread block;
                          larger ones by the multishift iteration itself
                          (one recursion level; the windows of that level use
                          double-shift QR).  The crossover plays the role of
                          LAPACK's NMIN for the small AED task of Sec. 3.2.
                          0 = 160, the largest window one block holds;
                          values above 160 act as 160 */
  int recompute_shifts;/* 1: when AED leaves at most ns/2 undeflated
                          candidates, the next sweep's shifts are the
                          eigenvalues of the trailing min(ns, 160) rows of the
                          active block (LAPACK's rule, which the paper's
                          Sec. 5 names as the source of its shift quality
                          differences); 0 (default): the AED candidates */
  int split_products;  /* 1: a sweep's left products of each chase step are
                          split into the columns the next chase step needs
                          (main stream) and the rest (a fourth stream, beside
                          the next chase step, with the blocks where another
                          window's right products meet them); right products
                          leave those blocks out (schur_sweep_split_tasks
                          lists the pieces).  Same results up to rounding
                          order; at n = 20000 on the bench's workload 3 %
                          faster end to end, with every product launch slower
                          because more of them overlap.  0 (default): left
                          products of a step on the main stream, right
                          products on the side stream */
} schur_opts;

/* Statistics of the last schur_hessenberg call on this host thread. */
typedef struct {
  int aed_steps;        /* AED steps (Sec. 2.5) at the top level */
  int sweeps;           /* multishift sweeps (Sec. 2.3) at the top level */
  int small_qr;         /* blocks finished by double-shift QR (Sec. 2.2) */
  int deflated_by_aed;  /* eigenvalues deflated by AED at the top level */
  int window_launches;  /* bulge-chase window launches (all levels) */
  double sweep_gemm_flops;  /* executed FP64 flops of the off-window updates */
  double aed_gemm_flops;
  double reflector_flops;   /* algorithmic flops of direct reflector application */
  int update_launches;      /* off-window product launches of the sweeps */
  int chase_launches;       /* bulge-chase launches at the top level */
  /* device time per phase in ms (opts->timing = 1 only): */
  double t_chase_ms;        /* bulge-chase windows of the sweeps */
  double t_update_ms;       /* off-window products of the sweeps on H (main and side streams) */
  double t_aed_ms;          /* AED: window Schur form, deflation, reordering */
  double t_aed_update_ms;   /* off-window products of AED */
  double t_small_ms;        /* double-shift QR of small blocks (+ products) */
  /* SM clock cycles spent by the top-level AED kernels in the window Schur
   * form (Sec. 2.5 step 1; windows held in shared memory only) and in the
   * deflation checks + reordering + spike elimination (steps 2-3): */
  double aed_cycles_schur;
  double aed_cycles_post;
  long long kernel_launches; /* kernels launched by the call (all levels) */
  double t_z_ms;            /* products applied to Z on the Z stream (overlaps the rest) */
  int graph_built;          /* schur_hessenberg_batched: 1 if this call captured a new graph, 0 if it
                               replayed the one cached for its batch shape */
  int shift_recomputations; /* sweeps whose shifts were recomputed (opts->recompute_shifts) */
  double flops;             /* schur_hessenberg_reduce, schur_eigenvectors: algorithmic FP64 flops of
                               the call (LAPACK's operation counts for the same work) */
} schur_stats;

/* Fill *opts with the defaults listed above. Returns SCHUR_OK. */
int schur_default_opts(schur_opts* opts);

/* Human-readable text for a return code (static storage). */
const char* schur_status_string(int code);

/* Device scratch (bytes) needed by schur_hessenberg for order n and *opts
 * (opts may be NULL for the defaults). */
int schur_workspace_size(int n, const schur_opts* opts, size_t* bytes);

/*
 * schur_hessenberg -- reduce the upper Hessenberg H (n x n) to real Schur form
 * S = Z^T H Z (Sec. 2, eqs. hessenberg_form .. 2by2_blocks).
 *   n      order, n >= 0                                            (arg 1)
 *   H      device, ldh x n; on entry the upper Hessenberg matrix (entries
 *          below the first subdiagonal are ignored); on exit S, standardised
 *          quasi-triangular, zero below the subdiagonal                (arg 2)
 *   ldh    >= max(1, n)                                             (arg 3)
 *   Z      device, ldz x n; see opts->z_init; on exit Z_in * Z_QR; may be
 *          NULL when opts->want_z == 0                              (arg 4)
 *   ldz    >= max(1, n) when Z is referenced                        (arg 5)
 *   wr,wi  device, length n: eigenvalues; a complex pair is adjacent with
 *          the positive imaginary part first (the order of S's diagonal)
 *                                                                    (args 6, 7)
 *   opts   may be NULL (defaults)                                   (arg 8)
 * Streams: the call creates three streams of its own and joins them to
 * opts->stream by events (its first kernel waits for the work already on
 * opts->stream; opts->stream waits for its last one).  The main stream has
 * the greatest priority and carries the scan, the AED and the chase; a side
 * stream one level lower carries each chase step's products on the rows
 * above its windows; a least-priority stream carries every product on Z
 * (Sec. 3.4: updates outside the critical path are delayed).  The call is
 * therefore not capturable into a CUDA graph; schur_hessenberg_batched is.
 * With the environment variable SCHUR_TRACE=<file> set (timing is then on
 * whatever opts->timing says), every timed bracket of the call is written to
 * <file> as CSV
 * "stream,phase,start_ms,end_ms" (streams 0 main, 1 Z, 2 side; phases as in
 * schur_stats: 0 chase, 1 products, 2 AED, 3 AED products, 4 small QR, 5 Z).
 */
int schur_hessenberg(int n, double* H, int ldh, double* Z, int ldz, double* wr, double* wi,
                     const schur_opts* opts);

/*
 * schur_hessenberg_noalloc -- schur_hessenberg for callers that cannot
 * allocate memory during the call (no counterpart in the paper).  Examples:
 * a host framework that owns every device allocation through its own pool,
 * a real-time loop with a fixed memory budget, code that must avoid the
 * implicit device synchronisation of cudaMalloc / cudaFree.  Arguments and
 * results as in schur_hessenberg (device pointers; Z is required and is set
 * to I on entry unless opts->z_init == 1; opts may be NULL).  One thread block
 * reduces the matrix with the batched engine (AED windows of at most 64
 * rows), so it suits small and medium orders.
 *   - Allocates nothing: its scratch (about 37 KB) is a fixed array in
 *     device memory that every device holding the library keeps until the
 *     process exits.  The first call on a device sets the entry point up
 *     there (the device must be current): it looks up that array's device
 *     address and raises the shared-memory limits of the library's kernels
 *     to the device maximum, once; make that first call before any stream
 *     capture.  No call changes a kernel attribute afterwards, so calls of
 *     the other entry points on other host threads are not affected.
 *   - n > 1024 returns SCHUR_ERR_TOO_LARGE without touching the device.
 *   - All calls share the one array: calls that may overlap on the GPU
 *     (different streams or host threads) race and must be serialised by
 *     the caller.  Each call resets the parts that must start at zero.
 *   - Synchronises opts->stream before returning (it returns the status).
 */
int schur_hessenberg_noalloc(int n, double* H, int ldh, double* Z, int ldz, double* wr, double* wi,
                             const schur_opts* opts);

/* Statistics of the last schur_hessenberg call made by this host thread. */
int schur_last_stats(schur_stats* out);

/* Text of the last CUDA error seen by this host thread (which runtime call
 * failed and where); "" if none.  Static storage, per host thread. */
const char* schur_last_error_detail(void);

/*
 * schur_hessenberg_batched -- the same reduction for `batch` independent
 * matrices of uneven sizes in ONE persistent kernel launch, replayed from a
 * captured CUDA graph (not in the paper: batching of the method).  The graph
 * and its device buffers are cached per batch shape (batch size, the
 * size table, deflation mode, opts->z_init; up to 4 shapes, least recently
 * used released): a call with a cached shape uploads its descriptors and
 * replays the graph.  Calls are serialised by a lock.  schur_last_stats
 * reports graph_built and, in reflector_flops, the algorithmic flops the
 * kernel applied (4 nr per row or column entry of each reflector of order
 * nr, 2 nw^2 per vector of each AED window product).  Each
 * matrix is reduced by one thread block with the same iteration as
 * schur_hessenberg (AED, multishift sweeps, double-shift QR for small
 * blocks, the same deflation conditions), with reflectors applied directly
 * instead of through windows.
 *   batch        number of matrices, >= 0                            (arg 1)
 *   n            host array [batch]: orders, 1 <= n[b] <= 1024          (arg 2)
 *   H            host array [batch] of device pointers (as in schur_hessenberg)
 *                                                                     (arg 3)
 *   ldh          host array [batch], ldh[b] >= n[b]                   (arg 4)
 *   Z            host array [batch] of device pointers (always accumulated;
 *                opts->z_init applies)                               (arg 5)
 *   ldz          host array [batch], ldz[b] >= n[b]                   (arg 6)
 *   wr, wi       host arrays [batch] of device pointers, length n[b] each
 *                                                                (args 7, 8)
 *   info         host array [batch] (output): per-matrix status as in
 *                schur_hessenberg                                     (arg 9)
 *   opts         may be NULL                                          (arg 10)
 * Returns SCHUR_OK if the launch succeeded (check info[] per matrix).
 */
int schur_hessenberg_batched(int batch, const int* n, double* const* H, const int* ldh, double* const* Z,
                             const int* ldz, double* const* wr, double* const* wi, int* info,
                             const schur_opts* opts);

/*
 * schur_batched_set_table -- per-size-bucket (shifts, AED window) table used by
 * schur_hessenberg_batched on this host thread (the autotuner's output; not
 * in the paper).  Bucket b covers active blocks of at most max_n[b] rows (the
 * last bucket covers all larger ones); 2 <= ns[b] <= 64, 4 <= nw[b] <= 128.
 * nbuckets = 0 restores the built-in table.  All arrays are host arrays of
 * nbuckets entries (nbuckets <= 8).
 */
int schur_batched_set_table(int nbuckets, const int* max_n, const int* ns, const int* nw);

/*
 * schur_eig_backward -- adjoint of the eigenvalues (not in the paper).  For
 * a real loss L(lambda_1..lambda_n) with cotangents g_k = dL/dRe(lambda_k) +
 * i dL/dIm(lambda_k), returns dL/dH = Z G Z^T with
 *     G = Re( sum_k conj(g_k) / (y_k^H x_k) * conj(y_k) x_k^T ),
 * x_k, y_k the right / left eigenvectors of S (first-order eigenvalue
 * perturbation: d lambda = y^H dH x / y^H x).  The eigenvectors come from
 * block back / forward substitution on the quasi-triangular S: up to order
 * 1024 one warp per eigenvalue; above that the blocked solver of
 * schur_eigenvectors, run on S and on the reversed transpose of S (whose
 * right eigenvectors are y reversed), then three FP64 GEMMs that skip the
 * triangular factors' zeros (about 3.3 n^3 + 2 n^3/3 flops).  A pivot below
 * a small multiple of u ||S|| (nearly repeated eigenvalues) is replaced by
 * it.
 *   n          order, n >= 0                                        (arg 1)
 *   S, lds     device, the standardised Schur factor from schur_hessenberg
 *                                                                (args 2, 3)
 *   Z, ldz     device, the Schur vectors from schur_hessenberg       (args 4, 5)
 *   wr, wi     device, eigenvalues in S's order                      (args 6, 7)
 *   gwr, gwi   device, length n: cotangents of Re / Im of each eigenvalue
 *                                                                (args 8, 9)
 *   dH, lddh   device, output n x n                                  (args 10, 11)
 *   opts       may be NULL (stream, workspace)                        (arg 12)
 * Scratch: schur_eig_backward_workspace(n) bytes (5 n^2 doubles up to order
 * 1024, 3 n^2 above, plus small tables), from opts->workspace when set
 * (SCHUR_ERR_WORKSPACE if smaller), else allocated for the call.
 * Synchronises opts->stream before returning.
 */
int schur_eig_backward_workspace(int n, size_t* bytes);
int schur_eig_backward(int n, const double* S, int lds, const double* Z, int ldz, const double* wr,
                       const double* wi, const double* gwr, const double* gwi, double* dH, int lddh,
                       const schur_opts* opts);

/*
 * schur_factor_backward -- adjoint of the Schur factors themselves (not in
 * the paper): for a real loss L(S, Z) of the standardised factors of
 * H = Z S Z^T (schur_hessenberg's output), with cotangents Sbar = dL/dS and
 * Zbar = dL/dZ, returns dL/dH (n x n).  The first-order change of the
 * factors is dZ = Z Omega (Omega skew), dS = Z^T dH Z + S Omega - Omega S,
 * with Omega fixed by keeping S quasi-triangular with standardised 2x2 blocks;
 * the adjoint solves the transposed block-triangular Sylvester system on S
 * (one thread block, block column by block column) between two sets of FP64
 * GEMMs.  Requires the diagonal blocks of S to have distinct eigenvalues (the
 * factors are not differentiable otherwise; a pivot below 2^-52 ||S||_F of a
 * 2x2 or 4x4 block equation is replaced by that value).  A 2x2 block with
 * b + c = 0 is invariant under the rotations that keep it standardised; its
 * rotation term is taken as zero.
 *   n          order, 0 <= n <= 1024                                (arg 1)
 *   S, Z       device, the factors (args 2-5); Sbar, Zbar device cotangents
 *              (args 6-9); dH device output (args 10-11)
 * Scratch 4 n^2 doubles (+ descriptors), from opts->workspace when set.
 */
int schur_factor_backward(int n, const double* S, int lds, const double* Z, int ldz, const double* Sbar, int ldsb,
                          const double* Zbar, int ldzb, double* dH, int lddh, const schur_opts* opts);

/* schur_factor_backward for `batch` matrices: host arrays of device
 * pointers and host arrays of ints as in schur_eig_backward_batched; one
 * thread block per matrix for the Sylvester solve, the GEMMs of all matrices
 * in shared launches.  A bad argument i returns -i. */
int schur_factor_backward_batched(int batch, const int* n, double* const* S, const int* lds, double* const* Z,
                                  const int* ldz, double* const* Sbar, const int* ldsb, double* const* Zbar,
                                  const int* ldzb, double* const* dH, const int* lddh, const schur_opts* opts);

/* schur_eig_backward for `batch` matrices in one launch sequence; arrays as
 * in schur_hessenberg_batched (host arrays of device pointers; n, lds, ldz
 * and lddh host arrays of ints).  A bad argument i returns -i, also when
 * only one matrix's entry of that array is bad. */
int schur_eig_backward_batched(int batch, const int* n, double* const* S, const int* lds, double* const* Z,
                               const int* ldz, double* const* wr, double* const* wi, double* const* gwr,
                               double* const* gwi, double* const* dH, const int* lddh,
                               const schur_opts* opts);

/* ---------------------------------------------------------------------
 * The phases around the QR iteration (Sec. 1): reduction of a general
 * matrix to Hessenberg form before it (phase i) and eigenvectors from the
 * Schur form after it (phase iii).  Together with schur_hessenberg they give
 * the eigen-decomposition of a general matrix on the device:
 *   schur_hessenberg_reduce(A -> H, Q);  schur_hessenberg(H -> S, Z = Q Z_QR,
 *   opts.z_init = 1);  schur_eigenvectors(S, Z -> X).
 * Same conventions as above: device pointers owned by the caller,
 * column-major, synchronous on opts->stream, no exceptions.
 * --------------------------------------------------------------------- */

/*
 * schur_hessenberg_reduce -- Householder reduction A = Q H Q^T of a general
 * n x n matrix (phase (i), Sec. 1; the textbook unblocked reduction with
 * LAPACK dgehrd's reflector convention beta = -sign(alpha) ||x||, so H equals
 * dgehrd's up to rounding).
 *   A   in: the matrix; out: H, with the entries below the first
 *       subdiagonal set to 0.                                      (args 2-3)
 *   Q   out: the orthogonal factor (n x n), or NULL to skip it.    (args 4-5)
 * Scratch: schur_hessenberg_reduce_workspace(n) bytes, from
 * opts->workspace when it is set (SCHUR_ERR_WORKSPACE if smaller), else
 * allocated and freed by the call.  Returns SCHUR_ERR_NONFINITE (A is left
 * unchanged) if A holds a NaN or Inf.  Sets schur_stats.flops
 * ((10/3) n^3 for H, (4/3) n^3 more for Q) and kernel_launches.
 */
int schur_hessenberg_reduce(int n, double* A, int lda, double* Q, int ldq, const schur_opts* opts);
int schur_hessenberg_reduce_workspace(int n, size_t* bytes);

/*
 * schur_eigenvectors -- right eigenvectors of H = Z S Z^T from its real
 * Schur form (phase (iii), Sec. 1).
 *   S      the standardised quasi-triangular factor (schur_hessenberg's output
 *          H); only its upper quasi-triangular part is read.      (args 2-3)
 *   Z      the Schur vectors (n x n); NULL: X receives the eigenvectors of S
 *          itself.                                                  (args 4-5)
 *   wr, wi the eigenvalues schur_hessenberg returned for this S (device,
 *          length n; a pair has wi > 0 first).                      (args 6-7)
 *   X      out (n x n): column i = the eigenvector of a real lambda_i; for a
 *          pair (i, i+1), columns i and i+1 = real and imaginary parts of
 *          the eigenvector of wr[i] + i wi[i] (its conjugate belongs to
 *          lambda_{i+1}).  Every (complex) vector has unit 2-norm; the phase
 *          is that of the back substitution started from 1 (1x1 block) or
 *          from (b, lambda - a) on a 2x2 block [[a, b], [c, d]].    (args 8-9)
 * A pivot of magnitude below smin = max(2^-52 ||S||_F, 1e-300) is replaced by
 * smin (nearly repeated eigenvalues).  The vectors are not protected against
 * overflow beyond that (growth past ~1e300 needs a departure from normality
 * of that order).  Scratch: schur_eigenvectors_workspace(n, Z != NULL)
 * bytes (an n x n buffer when Z is given), from opts->workspace when set,
 * else allocated by the call.  Sets schur_stats.flops (n^3/3 + n^3 with Z).
 */
int schur_eigenvectors(int n, const double* S, int lds, const double* Z, int ldz, const double* wr,
                       const double* wi, double* X, int ldx, const schur_opts* opts);
int schur_eigenvectors_workspace(int n, int with_z, size_t* bytes);

/* ---------------------------------------------------------------------
 * The generalized case (the paper's remarks in Sec. 1, 2.1, 2.2 and 3.4):
 * the generalized real Schur form (S, T) = Q^T (H, T0) Z of a
 * Hessenberg-triangular pair, by the double-shift QZ iteration.
 * --------------------------------------------------------------------- */

/*
 * schur_ht_reduce -- Hessenberg-triangular reduction of a general pair (the
 * generalized case's first phase, Sec. 1 remark): (A, B) -> (H, R) with H
 * upper Hessenberg and R upper triangular, A = Q H Z^T and B = Q R Z^T.  A
 * Householder QR of B applied to A, then Givens rotations that zero A below
 * its subdiagonal column by column from the bottom, each followed by the
 * right rotation that removes its fill-in in R (Golub & Van Loan Alg. 7.7.1;
 * the order of the oracle's reduction).  One thread block per pair; the
 * result is schur_qz's input.
 *   n          order, n >= 0                                        (arg 1)
 *   A, lda     device, overwritten by H (zeros below the subdiagonal) (args 2, 3)
 *   B, ldb     device, overwritten by R (zeros below the diagonal)  (args 4, 5)
 *   Q, ldq     device n x n: set to the left transformation (I on entry
 *              unless opts->z_init == 1, then multiplied in place)  (args 6, 7)
 *   Z, ldz     device n x n: the right transformation, the same way (args 8, 9)
 *              (Q and Z are not referenced when opts->want_z == 0)
 *   opts       may be NULL                                         (arg 10)
 * Returns SCHUR_OK, SCHUR_ERR_NONFINITE (a NaN or Inf in A or B: nothing
 * changed), or an error code.  Synchronises opts->stream before returning.
 */
int schur_ht_reduce(int n, double* A, int lda, double* B, int ldb, double* Q, int ldq, double* Z, int ldz,
                    const schur_opts* opts);

/* schur_ht_reduce for `batch` pairs in one launch (one thread block per
 * pair): host arrays of device pointers and of ints as in
 * schur_qz_batched; info[b] is the per-pair status.  A bad argument i
 * returns -i. */
int schur_ht_reduce_batched(int batch, const int* n, double* const* A, const int* lda, double* const* B,
                            const int* ldb, double* const* Q, const int* ldq, double* const* Z, const int* ldz,
                            int* info, const schur_opts* opts);

/*
 * schur_qz -- (H, T) upper Hessenberg / upper triangular (n x n, device)
 * are overwritten by S (quasi upper triangular) and T (upper triangular):
 *   - a 2x2 diagonal block of S holds a complex conjugate pair, and T's block
 *     there is diagonal with positive entries (LAPACK's standardised form);
 *     a pair with real eigenvalues is split;
 *   - |T_ii| <= 2^-52 ||T||_F is an infinite eigenvalue: T_ii is set to 0 and
 *     the zero is chased up to the top of its unreduced block and split off
 *     there (Sec. 2.1 / 3.4);
 *   - entries of H below the subdiagonal and of T below the diagonal are
 *     ignored on entry and zero on exit.
 *   Q, Z (args 6-9): when opts->want_z (default 1), the transformations are
 *     accumulated: z_init = 0 sets Q = Z = I first, z_init = 1 multiplies the
 *     given Q1, Z1 (e.g. from a Hessenberg-triangular reduction) in place.
 *   alphar, alphai, beta (device, length n; args 10-12): eigenvalue i is
 *     (alphar_i + i alphai_i) / beta_i; beta_i = 0 for an infinite one; a
 *     complex pair has alphai > 0 first.
 * Method: one thread block runs the whole double-shift iteration on the pair
 * (bulge of (H T^-1 - l1)(H T^-1 - l2) e1, left 3x3 reflectors, right
 * reflectors restoring T, Sec. 2.2 remark), exceptional shifts every 10th
 * iteration without deflation; no multishift sweeps or AED for pairs.
 * Returns SCHUR_OK, 1 + the top row of a block that did not converge within
 * 30 x (its order) iterations, SCHUR_ERR_NONFINITE (pair unchanged) or
 * another negative error.  Sets schur_stats.kernel_launches.
 */
int schur_qz(int n, double* H, int ldh, double* T, int ldt, double* Q, int ldq, double* Z, int ldz,
             double* alphar, double* alphai, double* beta, const schur_opts* opts);

/* schur_qz for `batch` pairs in one launch, one thread block per pair; the
 * arrays are host arrays of device pointers / ints as in
 * schur_hessenberg_batched; info (host, length batch) receives each pair's
 * schur_qz status.  Returns SCHUR_OK or a negative error (a bad argument i
 * returns -i, also when only one pair's entry is bad). */
int schur_qz_batched(int batch, const int* n, double* const* H, const int* ldh, double* const* T, const int* ldt,
                     double* const* Q, const int* ldq, double* const* Z, const int* ldz, double* const* alphar,
                     double* const* alphai, double* const* beta, int* info, const schur_opts* opts);

/* ---------------------------------------------------------------------
 * Single steps of the method, exported so that each can be checked on its
 * own against the CPU oracle.  Same conventions as above.
 * --------------------------------------------------------------------- */

/*
 * schur_qz_sweep -- one double-shift QZ sweep (Sec. 2.2 remark) on the
 * unreduced block lo..hi (0-based, hi - lo >= 2) of the Hessenberg-triangular
 * pair (H, T) with the shift pair given as ssum = l1 + l2, sprod = l1 l2,
 * full generalized Schur form mode (rows 0.. and columns ..n-1 updated);
 * Q and Z (both or neither) accumulate the transformations.  T's diagonal
 * entries lo, lo+1 and hi-2..hi must be nonzero.
 */
int schur_qz_sweep(int n, double* H, int ldh, double* T, int ldt, double* Q, int ldq, double* Z, int ldz, int lo,
                   int hi, double ssum, double sprod, const schur_opts* opts);

/*
 * schur_sweep -- one tightly-coupled multishift sweep (Sec. 2.3, Fig. 2/3)
 * on the unreduced block rows/cols ilo..ihi (0-based, inclusive) of the
 * n x n H, full Schur form mode (rows 0.. and columns ..n-1 are updated,
 * and Z's columns ilo..ihi when Z != NULL).
 *   pairs  HOST array of 2*npairs doubles: (s1+s2, s1*s2) for each shift
 *          pair; pair b drives the b-th bulge introduced.          (arg 8)
 *   bulges_per_chain: bulges chased together in one window (0 = auto).
 */
int schur_sweep(int n, double* H, int ldh, double* Z, int ldz, int ilo, int ihi, const double* pairs,
                int npairs, int bulges_per_chain, const schur_opts* opts);

/*
 * schur_aed -- one AED step (Sec. 2.5) on the trailing nw x nw window of the
 * active block ktop..kbot (0-based, inclusive).  On exit *nd (host) is the
 * number of deflated eigenvalues; cand_re / cand_im (HOST arrays of length
 * >= nw) receive the undeflated candidates top to bottom and *ncand (host)
 * their count.  H and Z are updated in place (window written back only if
 * *nd > 0).
 */
int schur_aed(int n, double* H, int ldh, double* Z, int ldz, int ktop, int kbot, int nw, int* nd,
              double* cand_re, double* cand_im, int* ncand, const schur_opts* opts);

/*
 * schur_small_qr -- double-shift QR (Sec. 2.2) of the block ilo..ihi, full
 * Schur form mode, run by one thread block (the "small Schur" step used for
 * blocks of at most nmin rows; ihi - ilo + 1 <= 160).
 */
int schur_small_qr(int n, double* H, int ldh, double* Z, int ldz, int ilo, int ihi, const schur_opts* opts);

/*
 * schur_apply_u -- off-window update (Sec. 3.2.1 "left/right update"):
 * side 0: X <- U^T X with X = rows r0..r0+k-1, columns c0..c0+m-1 of A;
 * side 1: X <- X U   with X = rows r0..r0+m-1, columns c0..c0+k-1 of A.
 * U is k x k (device, ldu).  1 <= k <= 1024.
 */
int schur_apply_u(int side, double* A, int lda, int r0, int c0, int m, int k, const double* U, int ldu,
                  const schur_opts* opts);

/*
 * schur_fastmath_eval -- diagnostic of the FP64 reciprocal and reciprocal
 * square root used on the latency-bound scalar paths (Newton-Raphson from an
 * FP32 seed; not in the paper).  For each x[i] (device, length n) writes
 * out[4i..4i+3] (device) = {fast 1/x, IEEE 1/x, fast 1/sqrt(x), IEEE
 * 1/sqrt(x)} (the square-root pair is 0 for x <= 0).
 */
int schur_fastmath_eval(int n, const double* x, double* out, const schur_opts* opts);

/*
 * schur_fp64_fma_probe -- FP64 fused multiply-add throughput of this GPU
 * (not in the paper; the denominator of the off-window products' roofline,
 * which execute FP64 FMAs).  Launches `blocks` blocks of 256 threads, each
 * thread running 8 independent dependent chains of `iters` FMAs, on
 * opts->stream WITHOUT synchronising: the caller times it with events on
 * that stream.
 *   iters   >= 1                                                       (arg 1)
 *   blocks  >= 1 (a multiple of the SM count fills the GPU)             (arg 2)
 *   out     device, blocks * 256 doubles (results, keeps the work)      (arg 3)
 *   flops   host (output): the FP64 flops the launch executes (2 per FMA)
 *                                                                       (arg 4)
 *   opts    may be NULL (stream)                                        (arg 5)
 */
int schur_fp64_fma_probe(int iters, int blocks, double* out, double* flops, const schur_opts* opts);

/*
 * schur_sweep_split_tasks -- the products of every chase step of a sweep on
 * rows lo..hi of an n x n H, as the single-matrix path issues them at the
 * top level with opts.split_products = 1 (host only, no device work).  Record q (8 ints at rec + 8 q):
 *   step, kind, chain, side, r0, c0, L, nvec
 * kind 0 near left products (main stream), 1 far left products (far
 * stream), 2 cross blocks (far stream, after the step's near products),
 * 3 right products (side stream), 4 Z products; side 0: rows r0..r0+L-1,
 * columns c0..c0+nvec-1; side 1: rows r0..r0+nvec-1, columns c0..c0+L-1
 * (kind 4: the rows of Z, nvec = n).  *count = records (all of them, even
 * when more than cap); rec may be NULL when cap = 0.
 */
int schur_sweep_split_tasks(int n, int lo, int hi, int npairs, int bulges_per_chain, int cap, int* rec, int* count);

/*
 * schur_chase_schedule -- the window schedule of one multishift sweep as the
 * driver issues it (Sec. 2.3 / 2.4, Fig. 3; host computation only, no
 * device work).  npairs bulges are chased in chains of at most
 * bulges_per_chain (0 = the driver's default, 16); every launch moves each
 * chain in flight through one diagonal window.
 *   lo, hi    the active block, 0 <= lo, hi >= lo + 2                (args 1, 2)
 *   npairs    bulges (shift pairs), 1 <= npairs <= 1024                (arg 3)
 *   bulges_per_chain  >= 0                                             (arg 4)
 *   cap       capacity of rec in records, >= 0                         (arg 5)
 *   rec       host, cap x 7 ints: per window (launch index, ws, we, tau0,
 *             tau1, first pair, bulges): the window rows/columns ws..we and
 *             the chain-local steps tau0..tau1-1 moved in it; bulge j of the
 *             chain sits at row lo + tau - 3 j at step tau            (arg 6)
 *   count     host (output): number of windows of the sweep; records
 *             beyond cap are not written                               (arg 7)
 *   kwin, delta  host (output, may be NULL): the window order bound and
 *             the steps per launch                                 (args 8, 9)
 */
int schur_chase_schedule(int lo, int hi, int npairs, int bulges_per_chain, int cap, int* rec, int* count,
                         int* kwin, int* delta);

/*
 * schur_vigilant_eval -- the device's vigilant-deflation test of a
 * subdiagonal entry (Sec. 2.1; the conditions of Sec. 5.6), evaluated on
 * given matrices so that it can be checked against the CPU oracle.
 *   count   number of matrices, >= 0                                  (arg 1)
 *   H       device, count 4x4 matrices, column-major, each 16 doubles
 *           apart; the entry tested is H(2, 1) of the active block rows
 *           0..3 (its neighbours H(1, 0) and H(3, 2) enter the test when
 *           the two diagonal entries are zero)                         (arg 2)
 *   mode    SCHUR_DEFLATION_*                                          (arg 3)
 *   thold   threshold of SCHUR_DEFLATION_FIXED                         (arg 4)
 *   normH   ||H||_F of SCHUR_DEFLATION_NORM                            (arg 5)
 *   n       order in the absolute floor nu n / u, >= 1                 (arg 6)
 *   out     device, count ints: 1 negligible, 0 not                    (arg 7)
 *   opts    may be NULL (stream)                                       (arg 8)
 * Synchronises opts->stream before returning.
 */
int schur_vigilant_eval(int count, const double* H, int mode, double thold, double normH, int n, int* out,
                        const schur_opts* opts);

/*
 * schur_spike_eval -- the device's AED deflation test (Sec. 5.6) of a 1x1
 * or 2x2 diagonal block of the window's Schur form against its spike
 * entries, evaluated on given blocks.
 *   count   number of blocks, >= 0                                    (arg 1)
 *   blk     device, count records of 7 doubles: a, b, c, d (the block
 *           [[a, b], [c, d]]; only d for a 1x1 block), s_j (the spike
 *           entry of the block's last row), s_{j-1} (of the row above, 2x2
 *           only) and the block size (1.0 or 2.0)                      (arg 2)
 *   mode, thold, normH, n   as in schur_vigilant_eval              (args 3-6)
 *   out     device, count ints: 1 deflatable, 0 not                    (arg 7)
 *   opts    may be NULL (stream)                                       (arg 8)
 * Synchronises opts->stream before returning.
 */
int schur_spike_eval(int count, const double* blk, int mode, double thold, double normH, int n, int* out,
                     const schur_opts* opts);

#ifdef __cplusplus
}
#endif

#endif /* SCHUR_GB300_H */
