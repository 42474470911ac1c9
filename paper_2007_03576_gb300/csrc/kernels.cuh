// kernels.cuh -- declarations of the kernels launched by the host driver.
#pragma once

#include "common.cuh"

__global__ void k_prep(double* H, long long ldh, int n, double* Z, long long ldz, int zinit, int* nonfinite);
__global__ void k_scan(double* H, long long ldh, int lo, int hi, DeflParams dp, Ctl* ctl);
__global__ void k_std2(double* H, long long ldh, int n, double* Z, long long ldz, int zrows, int k);
__global__ void k_smallqr(double* H, long long ldh, int ilo, int ihi, double* U, int ldu, DeflParams dp, Ctl* ctl);
__global__ void k_aed_small(double* H, long long ldh, int ktop, int kbot, int nw, double* V, int ldv,
                            double* cand_re, double* cand_im, double* vbuf, DeflParams dp, DeflParams dpw, Ctl* ctl);
__global__ void k_copy_window(const double* H, long long ldh, int kwtop, int nw, double* T, int ldt, double* V,
                              int ldv);
__global__ void k_aed_big_post(double* H, long long ldh, int ktop, int kbot, int nw, double* T, int ldt, double* V,
                               int ldv, double* cand_re, double* cand_im, double* vbuf, DeflParams dp, Ctl* ctl,
                               int inner_info);
__global__ void k_recompute_shifts(const double* H, long long ldh, int ktop, int kbot_old, int ns_max, int nw,
                                   int nibble, int nmin, double* cand_re, double* cand_im, DeflParams dp, Ctl* ctl);
__global__ void k_make_pairs(const double* H, long long ldh, int ktop, int kbot_old, int ns_max, int ndfl_host,
                             int exc_period, const double* cand_re, const double* cand_im, double* pairs, Ctl* ctl);
__global__ void k_chase(double* H, long long ldh, const double* pairs, double* Ubuf,
                        const __grid_constant__ ChaseArgs args);
__global__ void k_extract_eigs(const double* H, long long ldh, int n, double* wr, double* wi);
__global__ void k_set_int(int* p, int v);
__global__ void k_fastmath_eval(int n, const double* x, double* out);
int fma_probe_launch(int iters, int blocks, double* out, cudaStream_t st);   // 256 threads x 8 FMA chains
__global__ void k_vigilant_eval(int count, const double* H, DeflParams dp, int* out);
__global__ void k_spike_eval(int count, const double* blk, DeflParams dp, int* out);

// off-window products (TN = vectors per tile, 64/32/16/8)
cudaError_t launch_apply_u(int tn, int grid, size_t smem, cudaStream_t st, const UpdArgs& a);
cudaError_t apply_u_set_smem(int bytes);
int apply_u_blocks_per_sm(int tn, size_t smem);   // resident k_apply_u blocks per SM

size_t chase_smem_bytes(int kwin);
size_t apply_u_smem_bytes(int tn, int maxL);
int apply_u_tn(int maxL);
