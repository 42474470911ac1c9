// noalloc.cu -- a reduction entry point that allocates no memory.
//
// Some callers cannot allocate device memory while they call into this
// library: a framework that owns every device allocation through its own
// pool, a real-time loop with a fixed memory budget, or code that must not
// risk the implicit device synchronisation of cudaMalloc / cudaFree.  For
// them schur_hessenberg_noalloc reduces one Hessenberg matrix with the
// batched engine's kernel (one thread block, reflectors applied directly)
// and takes all of its scratch -- the work-queue counter, the status word,
// the matrix descriptor and the per-block workspace -- from one file-scope
// device array of fixed size.  That array exists once per device for the
// life of the process and is shared by every call.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "../../include/schur_gb300.h"
#include "batched.cuh"
#include "host.h"

#define NA_NW 64                 // AED window limit of this entry point
#define NA_NMAX 1024             // largest order accepted
#define NA_MAX_DEVICES 64

// Layout of the scratch array (bytes): counter, status, descriptor, order,
// block-scratch struct, then the block workspace (V, vbuf, candidates, pairs).
#define NA_OFF_COUNTER 0
#define NA_OFF_INFO 8
#define NA_OFF_ORDER 16
#define NA_OFF_DESC 256
#define NA_OFF_SCRATCH 512
#define NA_OFF_WORK 1024
#define NA_WORK_DOUBLES (NA_NW * NA_NW + 6 * NA_NW + 2 * (MAX_BULGES_PER_CHAIN + 4))
#define NA_BYTES (NA_OFF_WORK + NA_WORK_DOUBLES * 8)

static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

// Device address of g_noalloc_scratch per device, set up once per device
// (with that device current) together with the kernels' shared-memory limits,
// which are raised to their maximum there and never changed per call.
static char* g_scratch_ptr[NA_MAX_DEVICES] = {nullptr};
static std::mutex g_setup_mu;

static int noalloc_setup(int dev) {
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (g_scratch_ptr[dev] != nullptr) return SCHUR_OK;
  try {
    schur::init_kernel_attributes();
  } catch (const schur::CudaError&) {
    return SCHUR_ERR_CUDA;
  }
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) {
    cudaGetLastError();
    return SCHUR_ERR_CUDA;
  }
  g_scratch_ptr[dev] = (char*)p;
  return SCHUR_OK;
}

extern "C" int schur_hessenberg_noalloc(int n, double* H, int ldh, double* Z, int ldz, double* wr, double* wi,
                                        const schur_opts* opts) {
  if (n < 0) return -1;
  if (n > NA_NMAX) return SCHUR_ERR_TOO_LARGE;
  if (n == 0) return SCHUR_OK;
  if (!H) return -2;
  if (ldh < n) return -3;
  if (!Z) return -4;
  if (ldz < n) return -5;
  if (!wr) return -6;
  if (!wi) return -7;
  schur_opts o;
  schur::read_opts(opts, &o);
  cudaStream_t st = (cudaStream_t)o.stream;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return SCHUR_ERR_CUDA;
  if (g_scratch_ptr[dev] == nullptr) {
    int rc = noalloc_setup(dev);
    if (rc != SCHUR_OK) return rc;
  }
  char* base = g_scratch_ptr[dev];
  // parameters: the built-in size table with windows capped at NA_NW
  BatchedParams P;
  memset(&P, 0, sizeof(P));
  P.nmin = (o.nmin > 0) ? std::min(o.nmin, NW_SMEM_MAX) : 75;
  P.nibble = (o.nibble > 0) ? o.nibble : 14;
  P.exc_period = 6;
  P.mode = o.deflation;
  P.thold = o.fixed_thold;
  P.nbuckets = 3;
  const int mx[3] = {149, 589, 1 << 30}, ns[3] = {8, 8, 32}, nw[3] = {24, 32, NA_NW};
  for (int b = 0; b < 3; ++b) {
    P.bucket_max_n[b] = mx[b];
    P.ns[b] = ns[b];
    P.nw[b] = nw[b];
  }
  P.nw_max = NA_NW;
  // descriptor, order and block-scratch pointers (all inside the array);
  // the counter and the status word must start at zero
  BatchedDesc d{H, Z, wr, wi, (long long)ldh, (long long)ldz, n, 0};
  double* work = (double*)(base + NA_OFF_WORK);
  BatchedScratch sc;
  sc.V = work;
  sc.vbuf = sc.V + NA_NW * NA_NW;
  sc.cand_re = sc.vbuf + 4 * NA_NW;
  sc.cand_im = sc.cand_re + NA_NW;
  sc.pairs = sc.cand_im + NA_NW;
  sc.flops = nullptr;
  const int zero2[4] = {0, 0, 0, 0};
  const int order0 = 0;
  size_t smem = ((size_t)(NA_NW | 1) * NA_NW + (size_t)NA_NW * B_STAGE_COLS) * sizeof(double);
  int info = 0;
  if (cudaMemcpyAsync(base + NA_OFF_COUNTER, zero2, 16, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(base + NA_OFF_ORDER, &order0, sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(base + NA_OFF_DESC, &d, sizeof(d), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaMemcpyAsync(base + NA_OFF_SCRATCH, &sc, sizeof(sc), cudaMemcpyHostToDevice, st) != cudaSuccess) {
    cudaGetLastError();
    return SCHUR_ERR_CUDA;
  }
  k_batched_prep_z<<<1, CTA_THREADS, 0, st>>>((const BatchedDesc*)(base + NA_OFF_DESC), 1, o.z_init);
  k_batched<<<1, CTA_THREADS, smem, st>>>((const BatchedDesc*)(base + NA_OFF_DESC), (const int*)(base + NA_OFF_ORDER),
                                          1, (int*)(base + NA_OFF_COUNTER), (int*)(base + NA_OFF_INFO),
                                          (BatchedScratch*)(base + NA_OFF_SCRATCH), P);
  if (cudaGetLastError() != cudaSuccess) return SCHUR_ERR_CUDA;
  if (cudaMemcpyAsync(&info, base + NA_OFF_INFO, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return SCHUR_ERR_CUDA;
  }
  return info;
}
