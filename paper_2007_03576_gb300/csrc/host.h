// host.h -- host-side solver state shared by the C ABI translation units.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "../../include/schur_gb300.h"
#include "common.cuh"


#include <array>
#include <deque>

namespace schur {


struct CudaError {
  cudaError_t e;
};

// A matrix being reduced (full Schur form: every transform reaches all of H's
// rows/columns and zrows rows of Z).
struct Mat3 {
  double* H;
  long long ldh;
  int n;
  double* Z;
  long long ldz;
  int zrows;
};

// Device buffers of one recursion level (level 0 = the input matrix, level 1
// = an AED window reduced by the same iteration).
struct Level {
  int n = 0, nwmax = 0, nsmax = 0;
  Ctl* ctl = nullptr;
  double* ubuf = nullptr;
  double* V = nullptr;
  double* T = nullptr;
  double* cand_re = nullptr;
  double* cand_im = nullptr;
  double* pairs = nullptr;
  double* vbuf = nullptr;
  double* usmall = nullptr;
};

// Per-phase device timing with CUDA events (opts.timing = 1).
enum Phase { PH_CHASE = 0, PH_UPDATE = 1, PH_AED = 2, PH_AED_UPDATE = 3, PH_SMALL = 4, PH_Z = 5, PH_COUNT = 6 };

struct PhaseTimer {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  std::vector<int> phase_of;   // phase of event pair i
  size_t used = 0;             // event pairs recorded since the last flush
  int depth = 0;               // > 0 while inside a timed region (nested launches not timed)
  double ms[PH_COUNT] = {0, 0, 0, 0, 0, 0};
  // optional timeline: (stream id, phase, start ms, end ms) relative to
  // *base, appended as pairs are collected
  int sid = 0;
  cudaEvent_t* base = nullptr;
  std::vector<std::array<double, 4>>* trace = nullptr;
  void collect(size_t i);
  int begin(cudaStream_t st, int phase);
  void end(cudaStream_t st, int token);
  void flush();                // after a stream synchronisation
  void flush_completed();      // pairs whose end event has completed (other stream)
  ~PhaseTimer();
};

struct Solver {
  schur_opts opts;
  cudaStream_t st = nullptr;
  Ctl* hctl = nullptr;       // pinned mirror of the control block
  char* owned = nullptr;     // scratch allocated by the library
  int* flag = nullptr;
  double normH = 0.0;
  double* cur_flops = nullptr;
  int cur_update_phase = PH_UPDATE;
  bool count_launches = false;
  PhaseTimer timer;
  // Z is only ever multiplied from the right and nothing on H's side reads
  // it, so at level 0 its updates run on a second, low-priority stream (zst)
  // behind events; the chase / AED transforms they read sit in an arena whose
  // regions are reused only after zst has consumed them.  A sweep's Z
  // products are held back (zpending) until the sweep's H updates have been
  // issued, so that they fill the SMs that the next (one-block) AED leaves idle
  // instead of competing with the sweep's own H updates.
  cudaStream_t zst = nullptr;
  PhaseTimer ztimer;
  // At level 0 the call runs on its own streams, joined to the caller's
  // stream (ust) by events at the start and the end: the main stream (st) at
  // the greatest priority, zst at the least, and a side stream (sst, greatest
  // priority) for each chase step's products on the rows above its windows,
  // which nothing in the next chase step reads: they run beside it.
  cudaStream_t ust = nullptr, own_st = nullptr, sst = nullptr;
  PhaseTimer stimer;
  cudaEvent_t ev_t1 = nullptr, ev_t2 = nullptr, ev_join = nullptr;
  // far-column left products and the cross blocks of a chase step run on
  // fst beside the next chase step (their timer reports as the side stream)
  cudaStream_t fst = nullptr;
  PhaseTimer ftimer;
  cudaEvent_t ev_c = nullptr, ev_n = nullptr, ev_f = nullptr;
  bool f_pending = false;
  size_t f_a = 0, f_b = 0;
  // SCHUR_TRACE=<file>: every timed bracket of the call is written there as
  // "stream,phase,start_ms,end_ms" (streams 0 main, 1 Z, 2 side)
  cudaEvent_t ev_base = nullptr;
  std::vector<std::array<double, 4>> trace;
  const char* trace_path = nullptr;
  void write_trace();
  bool t2_pending = false;   // ev_t2 recorded and not yet waited for by st
  size_t t2_a = 0, t2_b = 0; // arena region [t2_a, t2_b) that the pending side-stream products read
  int side_reserve = 0;      // SMs the side stream's products leave to the next chase step
  cudaEvent_t ev_ready = nullptr, ev_zdone = nullptr;
  // Circular arena (level 0) holding the chase U's and AED V's that the Z
  // stream has not consumed yet; a region is reused only after the event
  // recorded behind its last Z-stream reader.
  struct Region {
    size_t a, b;           // [a, b) in doubles
    cudaEvent_t ev;        // nullptr: only main-stream readers
  };
  double* arena = nullptr;
  size_t arena_cap = 0, arena_cur = 0;
  std::deque<Region> live;
  struct PendingZ {
    std::vector<UpdTask> tasks;
    size_t a, b;           // arena region the tasks read
  };
  std::vector<PendingZ> zpending;
  std::vector<cudaEvent_t> spare_events;
  double* arena_alloc(size_t n);                 // waits (on st) for overlapping live regions
  void arena_release(double* p, size_t n, bool z_reader);  // after the readers were issued
  std::vector<Level> levels;
  // host copies of the chase windows' column ranges of the current sweep
  // (executed-flop counts of its products); cleared at the end of the sweep
  std::deque<std::vector<int2>> host_ranges;

  explicit Solver(const schur_opts* o);
  ~Solver();
  int setup(int n);
  void carve(char* base, int n);
  void read_ctl(const Ctl* d);
  DeflParams defl(int n) const;
  void run_updates(std::vector<UpdTask>& tasks, cudaStream_t s = nullptr, bool on_z = false);
  void apply_block_transform(const Mat3& M, int k0, int L, const double* U, int ldu, const int* gate,
                             bool with_z = true);
  void z_async(std::vector<UpdTask>& tasks, cudaEvent_t done);   // Z tasks on zst after st's current point
  void z_defer(std::vector<UpdTask>& tasks, const double* p, size_t n);  // held until z_flush
  void sweep_step_split(const Mat3& M, const struct SweepPlan& plan, int lo, int hi, int s, const ChaseArgs& a,
                        int na, double* ubase, size_t need, bool zasync, bool use_arena);
  void z_flush();                                                // issue zpending on zst after st's current point
  void drain_z();                                                // st waits for all of zst's work
  void init_streams(bool with_z);                               // see ust / sst / zst
  void join_caller();                                            // ust waits for st
  void sweep(const Mat3& M, int lev, int lo, int hi, const double* dpairs, int npairs, int nbc_req);
  int qr_block(const Mat3& M, int lev, int ilo, int ihi);
  int aed(const Mat3& M, int lev, int ktop, int kbot, int nw, int ns_max, int ndfl);
};

extern thread_local schur_stats g_stats;
extern thread_local char g_err_detail[256];
void ck_at(cudaError_t e, int line);
void init_kernel_attributes();   // once per device (thread-safe); throws CudaError
int num_sms();                   // SMs of the current device
// *out = the defaults overlaid with the first in->struct_size bytes of *in
// (the whole struct when struct_size <= 0); in may be NULL.
void read_opts(const schur_opts* in, schur_opts* out);
void default_ns_nw(int m, int* ns, int* nw);
size_t workspace_bytes(int n, const schur_opts& o);
// A caller workspace (o.workspace non-NULL) that cannot hold `need` bytes or
// is not 256-byte aligned (buffers are laid out at 256-byte offsets from it,
// so a misaligned base would misalign every FP64 access).
inline bool workspace_unusable(const schur_opts& o, size_t need) {
  return o.workspace_bytes < need || ((size_t)o.workspace & 255) != 0;
}
const char* status_string(int code);

// Right eigenvectors of a standardised quasi-triangular S, the work of
// schur_eigenvectors (eigvec.cu), on stream st: scratch `mem` of
// eigvec_workspace(n, Z != nullptr) bytes, hwi a host copy of wi (the pair
// structure).  Does not synchronise; adds its launches and GEMM flops to
// *launches / *flops; throws CudaError.
size_t eigvec_workspace(int n, bool with_z);
void eigvec_run(int n, const double* S, int lds, const double* Z, int ldz, const double* wr, const double* wi,
                const double* hwi, double* X, int ldx, cudaStream_t st, char* mem, long long* launches,
                double* flops);

}  // namespace schur
