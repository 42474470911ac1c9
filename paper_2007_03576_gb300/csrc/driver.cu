// driver.cu -- host driver and C ABI of the single-matrix path.
//
// The iteration of Sec. 2.1 runs on the host as a short control loop over
// device-resident data; every arithmetic step is a kernel of kernels.cu.  Per
// iteration the host reads back one small control block (Ctl) twice: after
// the deflation scan (where the bottom unreduced block starts) and after AED
// (how many eigenvalues deflated, how many shift pairs are ready).  A sweep is
// then issued without further synchronisation as a sequence of window steps:
// one k_chase launch (one block per bulge chain, Sec. 2.4) followed by the
// step's off-window products on three streams of the call (priorities as in
// Sec. 3.4): the left products of H on the main stream, the right products on
// the rows above the windows on a side stream, beside the next k_chase
// launch, and the products on Z on a least-priority stream, released at the
// end of the sweep so that they run beside the next AED.  Left and right
// products meet on blocks H[window_i, window_j], where they commute but would
// race; the next step's left products wait for the side stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "../../include/schur_gb300.h"
#include "batched.cuh"
#include "kernels.cuh"
#include "host.h"

namespace schur {

thread_local schur_stats g_stats;

const char* status_string(int code) {
  switch (code) {
    case SCHUR_OK: return "success";
    case SCHUR_ERR_NONFINITE: return "input contains NaN or Inf";
    case SCHUR_ERR_CUDA: return "CUDA runtime error";
    case SCHUR_ERR_NOMEM: return "device memory allocation failed";
    case SCHUR_ERR_WORKSPACE: return "workspace too small";
    case SCHUR_ERR_UNSUPPORTED: return "unsupported argument combination";
    case SCHUR_ERR_TOO_LARGE: return "order above the fixed limit (1024) of the no-allocation entry point";
    default: break;
  }
  if (code < 0) return "invalid argument";
  return "iteration limit reached (unreduced blocks remain)";
}

// Default (shifts, AED window) for an active block of m rows.  The paper has
// no table (windows are sized by tiles, Sec. 3.2); the same table is used by
// the oracle.
void default_ns_nw(int m, int* ns, int* nw) {
  if (m < 150) { *ns = 8; *nw = 24; return; }
  if (m < 590) { *ns = 8; *nw = 32; return; }
  if (m < 3000) { *ns = 64; *nw = 96; return; }
  if (m < 6000) { *ns = 64; *nw = 128; return; }
  *ns = 256;
  *nw = std::min(1024, std::max(3 * 256 / 2, (int)std::lround(0.03 * m)));
}

// ---------------------------------------------------------------------------
// Workspace
// ---------------------------------------------------------------------------
static size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

struct LevelSizes {
  int n;       // order of the matrix at this level
  int nwmax;   // largest AED window
  int nsmax;   // most shifts
  size_t arena;  // level 0: doubles of the arena behind the Z stream
  int fmax;      // windows above this order are reduced recursively (need the copy T)
  // AED candidates, or the eigenvalues of a trailing block of up to
  // min(nsmax, NW_SMEM_MAX) rows when shifts are recomputed
  int cand_len() const { return std::max(std::max(nwmax, std::min(nsmax + 8, NW_SMEM_MAX)), 4); }
  size_t bytes() const {
    size_t b = 0;
    b += align_up(sizeof(Ctl));
    b += align_up((size_t)MAX_CHAINS * CHASE_USLOT(KWIN_MAX) * sizeof(double));  // chase U + column ranges
    b += align_up((size_t)nwmax * nwmax * sizeof(double));                       // V
    b += align_up(arena * sizeof(double));
    b += (nwmax > fmax) ? align_up((size_t)nwmax * nwmax * sizeof(double)) : 0;  // T
    b += 2 * align_up((size_t)cand_len() * sizeof(double));                      // candidates
    b += align_up((size_t)(nsmax + 8) * sizeof(double));                         // pairs
    b += align_up((size_t)4 * std::max(nwmax, 4) * sizeof(double));              // vbuf
    b += align_up((size_t)NW_SMEM_MAX * NW_SMEM_MAX * sizeof(double));           // small-QR U
    return b;
  }
};

// Largest AED window reduced by double-shift QR in one thread block at the
// top level (the crossover to the recursive multishift iteration).
static int window_francis_max(const schur_opts& o) {
  return (o.nmin_window > 0) ? std::min(o.nmin_window, NW_SMEM_MAX) : NW_SMEM_MAX;
}

static void level_plan(int n, const schur_opts& o, std::vector<LevelSizes>& out) {
  out.clear();
  int m = n;
  for (int lev = 0; lev < 3 && m > 0; ++lev) {
    int ns, nw;
    default_ns_nw(m, &ns, &nw);
    if (lev == 0) {
      if (o.n_shifts > 0) ns = o.n_shifts;
      if (o.aed_window > 0) nw = o.aed_window;
    }
    nw = std::min(std::min(nw, m), 1024);
    size_t arena = 0;
    if (lev == 0) {
      // one sweep's window transforms plus an AED's V: chains x steps x kwin^2
      int nbc = o.bulges_per_chain > 0 ? o.bulges_per_chain : 16;
      nbc = std::max(1, std::min(nbc, MAX_BULGES_PER_CHAIN));
      int kwin = std::min(KWIN_MAX, std::max(6 * nbc, 48));
      int delta = std::max(1, kwin - 3 * nbc - 1);
      size_t nchain = (size_t)std::max(1, (ns / 2 + nbc - 1) / nbc);
      size_t steps = (size_t)m / delta + 3 * nchain * ((size_t)(2 * kwin + 4 * nbc) / delta + 2) + 8;
      arena = (nchain * steps + 2) * (size_t)CHASE_USLOT(kwin) + 2 * (size_t)nw * nw;
      arena = std::min(arena, (size_t)(1ull << 27));                       // at most 1 GiB
      arena = std::max(arena, (size_t)MAX_CHAINS * CHASE_USLOT(KWIN_MAX) + (size_t)nw * nw);
    }
    LevelSizes L{m, nw, ns, arena, lev == 0 ? window_francis_max(o) : NW_SMEM_MAX};
    out.push_back(L);
    if (nw <= L.fmax) break;
    m = nw;
  }
}

size_t workspace_bytes(int n, const schur_opts& o) {
  std::vector<LevelSizes> lv;
  level_plan(n, o, lv);
  size_t b = align_up(sizeof(int)) + 256;
  for (auto& L : lv) b += L.bytes();
  return b;
}

void Solver::carve(char* base, int n) {
  std::vector<LevelSizes> lv;
  level_plan(n, opts, lv);
  char* p = base;
  auto take = [&](size_t bytes) {
    char* q = p;
    p += align_up(bytes);
    return q;
  };
  flag = (int*)take(sizeof(int));
  levels.clear();
  for (auto& L : lv) {
    Level v;
    v.n = L.n;
    v.nwmax = L.nwmax;
    v.nsmax = L.nsmax;
    v.ctl = (Ctl*)take(sizeof(Ctl));
    v.ubuf = (double*)take((size_t)MAX_CHAINS * CHASE_USLOT(KWIN_MAX) * sizeof(double));
    v.V = (double*)take((size_t)L.nwmax * L.nwmax * sizeof(double));
    if (L.arena) {
      arena = (double*)take(L.arena * sizeof(double));
      arena_cap = L.arena;
      arena_cur = 0;
    }
    v.T = (L.nwmax > L.fmax) ? (double*)take((size_t)L.nwmax * L.nwmax * sizeof(double)) : nullptr;
    v.cand_re = (double*)take((size_t)L.cand_len() * sizeof(double));
    v.cand_im = (double*)take((size_t)L.cand_len() * sizeof(double));
    v.pairs = (double*)take((size_t)(L.nsmax + 8) * sizeof(double));
    v.vbuf = (double*)take((size_t)4 * std::max(L.nwmax, 4) * sizeof(double));
    v.usmall = (double*)take((size_t)NW_SMEM_MAX * NW_SMEM_MAX * sizeof(double));
    levels.push_back(v);
  }
}

// ---------------------------------------------------------------------------
// Solver
// ---------------------------------------------------------------------------
// Kernel attributes are per device: they are raised once for each device,
// under a lock, the first time a call runs with that device current.
#define ATTR_MAX_DEVICES 64
static std::mutex g_attr_mu;
static bool g_attr_done[ATTR_MAX_DEVICES] = {false};
static int g_num_sms[ATTR_MAX_DEVICES] = {0};

thread_local char g_err_detail[256] = "";

void ck_at(cudaError_t e, int line) {
  if (e != cudaSuccess) {
    snprintf(g_err_detail, sizeof(g_err_detail), "%s (%d) at driver.cu:%d", cudaGetErrorString(e), (int)e, line);
    cudaGetLastError();
    throw CudaError{e};
  }
}
#define ck(x) ck_at((x), __LINE__)

int PhaseTimer::begin(cudaStream_t st, int phase) {
  if (!on || depth > 0) return -1;
  ++depth;
  size_t i = used++;
  if (pool.size() < 2 * used) {
    cudaEvent_t a, b;
    ck(cudaEventCreate(&a));
    ck(cudaEventCreate(&b));
    pool.push_back(a);
    pool.push_back(b);
    phase_of.push_back(phase);
  }
  phase_of[i] = phase;
  ck(cudaEventRecord(pool[2 * i], st));
  return (int)i;
}

void PhaseTimer::end(cudaStream_t st, int token) {
  if (token < 0) return;
  --depth;
  ck(cudaEventRecord(pool[2 * token + 1], st));
}

void PhaseTimer::collect(size_t i) {
  float t = 0.f;
  if (cudaEventElapsedTime(&t, pool[2 * i], pool[2 * i + 1]) == cudaSuccess) ms[phase_of[i]] += t;
  if (trace && base) {
    float a = 0.f, b = 0.f;
    if (cudaEventElapsedTime(&a, *base, pool[2 * i]) == cudaSuccess &&
        cudaEventElapsedTime(&b, *base, pool[2 * i + 1]) == cudaSuccess)
      trace->push_back({(double)sid, (double)phase_of[i], (double)a, (double)b});
  }
  cudaGetLastError();
}

void PhaseTimer::flush() {
  if (depth > 0) return;  // a bracket is still open: its end event is not recorded yet
  for (size_t i = 0; i < used; ++i) collect(i);
  used = 0;
}

void PhaseTimer::flush_completed() {
  size_t i = 0;
  for (; i < used; ++i) {
    if (cudaEventQuery(pool[2 * i + 1]) != cudaSuccess) break;
    collect(i);
  }
  cudaGetLastError();
  if (i == 0) return;
  // keep the unfinished pairs at the front (swap events and phases)
  size_t k = 0;
  for (size_t j = i; j < used; ++j, ++k) {
    std::swap(pool[2 * k], pool[2 * j]);
    std::swap(pool[2 * k + 1], pool[2 * j + 1]);
    phase_of[k] = phase_of[j];
  }
  used = k;
}

PhaseTimer::~PhaseTimer() {
  for (auto e : pool) cudaEventDestroy(e);
}

void init_kernel_attributes() {
  int dev = 0;
  ck(cudaGetDevice(&dev));
  if (dev < 0 || dev >= ATTR_MAX_DEVICES) throw CudaError{cudaErrorInvalidDevice};
  std::lock_guard<std::mutex> lock(g_attr_mu);
  if (g_attr_done[dev]) return;
  ck(cudaDeviceGetAttribute(&g_num_sms[dev], cudaDevAttrMultiProcessorCount, dev));
  // every kernel with dynamic shared memory may take what the block limit
  // leaves beside its static shared memory; raised once and never lowered, so
  // that no entry point changes a limit that another one relies on
  int optin = 0;
  ck(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  auto allow = [&](const void* k) {
    cudaFuncAttributes fa;
    ck(cudaFuncGetAttributes(&fa, k));
    ck(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes));
  };
  allow((const void*)k_chase);
  allow((const void*)k_smallqr);
  allow((const void*)k_aed_small);
  allow((const void*)k_batched);
  allow((const void*)k_recompute_shifts);
  ck(apply_u_set_smem(220 * 1024));
  g_attr_done[dev] = true;
}

int num_sms() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= ATTR_MAX_DEVICES) {
    cudaGetLastError();
    return 152;
  }
  return g_num_sms[dev] > 0 ? g_num_sms[dev] : 152;
}

void read_opts(const schur_opts* in, schur_opts* out) {
  schur_default_opts(out);
  if (!in) return;
  size_t sz = (in->struct_size <= 0) ? sizeof(schur_opts) : std::min((size_t)in->struct_size, sizeof(schur_opts));
  memcpy(out, in, sz);
  out->struct_size = (int)sizeof(schur_opts);
}

Solver::Solver(const schur_opts* o) {
  read_opts(o, &opts);
  st = (cudaStream_t)opts.stream;
  timer.on = opts.timing != 0;
  if (opts.nmin <= 0) opts.nmin = 75;
  if (opts.nmin > NW_SMEM_MAX) opts.nmin = NW_SMEM_MAX;
  if (opts.nibble <= 0) opts.nibble = 14;
  ck(cudaMallocHost((void**)&hctl, sizeof(Ctl)));
}

Solver::~Solver() {
  for (cudaStream_t x : {zst, sst, fst, own_st})
    if (x) {
      cudaStreamSynchronize(x);
      cudaStreamDestroy(x);
    }
  for (cudaEvent_t e : {ev_t1, ev_t2, ev_join, ev_base, ev_c, ev_n, ev_f})
    if (e) cudaEventDestroy(e);
  for (auto& r : live)
    if (r.ev) cudaEventDestroy(r.ev);
  for (auto& e : spare_events) cudaEventDestroy(e);
  if (ev_ready) cudaEventDestroy(ev_ready);
  if (ev_zdone) cudaEventDestroy(ev_zdone);
  if (hctl) cudaFreeHost(hctl);
  if (owned) cudaFree(owned);
}

// Streams of a full reduction (level 0); st becomes the call's own stream.
void Solver::init_streams(bool with_z) {
  int least = 0, greatest = 0;
  ck(cudaDeviceGetStreamPriorityRange(&least, &greatest));
  ck(cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming));
  ck(cudaEventCreateWithFlags(&ev_t1, cudaEventDisableTiming));
  ck(cudaEventCreateWithFlags(&ev_t2, cudaEventDisableTiming));
  ck(cudaStreamCreateWithPriority(&own_st, cudaStreamNonBlocking, greatest));
  // one level below the main stream, so that a chase step's blocks are
  // placed before the side stream's
  ck(cudaStreamCreateWithPriority(&sst, cudaStreamNonBlocking, greatest < least ? greatest + 1 : greatest));
  ck(cudaStreamCreateWithPriority(&fst, cudaStreamNonBlocking, greatest < least ? greatest + 1 : greatest));
  ck(cudaEventCreateWithFlags(&ev_c, cudaEventDisableTiming));
  ck(cudaEventCreateWithFlags(&ev_n, cudaEventDisableTiming));
  ck(cudaEventCreateWithFlags(&ev_f, cudaEventDisableTiming));
  ust = st;
  ck(cudaEventRecord(ev_join, ust));
  ck(cudaStreamWaitEvent(own_st, ev_join, 0));
  st = own_st;
  trace_path = getenv("SCHUR_TRACE");
  if (trace_path && *trace_path) {
    timer.on = true;
    ck(cudaEventCreate(&ev_base));
    ck(cudaEventRecord(ev_base, st));
    PhaseTimer* ts[4] = {&timer, &ztimer, &stimer, &ftimer};
    for (int k = 0; k < 4; ++k) {
      ts[k]->sid = (k == 3) ? 2 : k;
      ts[k]->base = &ev_base;
      ts[k]->trace = &trace;
    }
  } else {
    trace_path = nullptr;
  }
  stimer.on = timer.on;
  ftimer.on = timer.on;
  if (with_z) {
    ck(cudaStreamCreateWithPriority(&zst, cudaStreamNonBlocking, least));
    ck(cudaEventCreateWithFlags(&ev_ready, cudaEventDisableTiming));
    ck(cudaEventCreateWithFlags(&ev_zdone, cudaEventDisableTiming));
    ztimer.on = timer.on;
  }
}

void Solver::write_trace() {
  if (!trace_path) return;
  FILE* f = fopen(trace_path, "w");
  if (!f) return;
  fprintf(f, "stream,phase,start_ms,end_ms\n");
  for (auto& r : trace) fprintf(f, "%d,%d,%.4f,%.4f\n", (int)r[0], (int)r[1], r[2], r[3]);
  fclose(f);
}

void Solver::join_caller() {
  if (!own_st) return;
  ck(cudaEventRecord(ev_join, st));
  ck(cudaStreamWaitEvent(ust, ev_join, 0));
}

// Regions of the arena are handed out in order, wrapping at the end; a new
// region waits (on the main stream) for every older live region up to the
// last one it overlaps.
double* Solver::arena_alloc(size_t n) {
  size_t a = (arena_cur + n > arena_cap) ? 0 : arena_cur;
  size_t b = a + n;
  // a region still held by deferred Z products is handed to zst first
  for (const PendingZ& p : zpending)
    if (p.a < b && a < p.b) {
      z_flush();
      break;
    }
  int last = -1;
  for (size_t i = 0; i < live.size(); ++i)
    if (live[i].a < b && a < live[i].b) last = (int)i;
  // the side stream (and the far stream) may still read the last chase step's region
  if (t2_pending && t2_a < b && a < t2_b) ck(cudaStreamWaitEvent(st, ev_t2, 0));
  if (f_pending && f_a < b && a < f_b) ck(cudaStreamWaitEvent(st, ev_f, 0));
  for (int i = 0; i <= last; ++i) {
    Region r = live.front();
    live.pop_front();
    if (r.ev) {
      ck(cudaStreamWaitEvent(st, r.ev, 0));
      spare_events.push_back(r.ev);
    }
  }
  arena_cur = b;
  return arena + a;
}

void Solver::arena_release(double* p, size_t n, bool z_reader) {
  Region r{(size_t)(p - arena), (size_t)(p - arena) + n, nullptr};
  if (z_reader) {
    if (spare_events.empty()) {
      cudaEvent_t e;
      ck(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      spare_events.push_back(e);
    }
    r.ev = spare_events.back();
    spare_events.pop_back();
    ck(cudaEventRecord(r.ev, zst));
  }
  live.push_back(r);
}

void Solver::z_defer(std::vector<UpdTask>& tasks, const double* p, size_t n) {
  zpending.push_back(PendingZ{std::move(tasks), (size_t)(p - arena), (size_t)(p - arena) + n});
}

// The deferred tasks go to zst in the order they were deferred (Z's columns
// overlap between chase steps); their arena regions become live, each behind
// the event recorded after the last of them.
void Solver::z_flush() {
  if (zpending.empty()) return;
  std::vector<PendingZ> pend;
  pend.swap(zpending);
  ck(cudaEventRecord(ev_ready, st));
  ck(cudaStreamWaitEvent(zst, ev_ready, 0));
  for (PendingZ& p : pend) run_updates(p.tasks, zst, true);
  for (PendingZ& p : pend) arena_release(arena + p.a, p.b - p.a, true);
}

void Solver::z_async(std::vector<UpdTask>& tasks, cudaEvent_t done) {
  z_flush();
  ck(cudaEventRecord(ev_ready, st));
  ck(cudaStreamWaitEvent(zst, ev_ready, 0));
  run_updates(tasks, zst, true);
  if (done) ck(cudaEventRecord(done, zst));
}

void Solver::drain_z() {
  if (!zst) return;
  z_flush();
  ck(cudaEventRecord(ev_zdone, zst));
  ck(cudaStreamWaitEvent(st, ev_zdone, 0));
}

int Solver::setup(int n) {
  size_t need = workspace_bytes(n, opts);
  if (opts.workspace != nullptr && workspace_unusable(opts, need)) return SCHUR_ERR_WORKSPACE;
  init_kernel_attributes();
  char* base = nullptr;
  if (opts.workspace != nullptr) {
    base = (char*)opts.workspace;
  } else {
    if (cudaMalloc((void**)&owned, need) != cudaSuccess) {
      owned = nullptr;
      cudaGetLastError();
      return SCHUR_ERR_NOMEM;
    }
    base = (char*)owned;
  }
  carve(base, n);
  for (auto& L : levels) ck(cudaMemsetAsync(L.ctl, 0, sizeof(Ctl), st));
  return SCHUR_OK;
}

void Solver::read_ctl(const Ctl* dctl) {
  ck(cudaMemcpyAsync(hctl, dctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
  ck(cudaStreamSynchronize(st));
  timer.flush();
  if (zst) ztimer.flush_completed();
  if (sst) stimer.flush_completed();
  if (fst) ftimer.flush_completed();
}

DeflParams Solver::defl(int n) const {
  DeflParams d;
  d.mode = opts.deflation;
  d.thold = opts.fixed_thold;
  d.normH = normH;
  d.n = n;
  return d;
}

static double apply_u_entries(const UpdTask& q, int tn);

// Issue a list of off-window products (split in launches of at most
// MAX_UPD_TASKS tasks; tasks within a launch must not overlap).
void Solver::run_updates(std::vector<UpdTask>& tasks, cudaStream_t sarg, bool on_z) {
  const bool on_far = !on_z && sarg != nullptr && sarg == fst;
  const bool on_side = !on_z && sarg != nullptr && (sarg == sst || on_far);
  cudaStream_t s = (on_z || on_side) ? sarg : st;
  PhaseTimer& tm = on_z ? ztimer : (on_far ? ftimer : (on_side ? stimer : timer));
  const int phase = on_z ? PH_Z : cur_update_phase;
  size_t i = 0;
  while (i < tasks.size()) {
    UpdArgs a;
    memset(&a, 0, sizeof(a));
    int maxL = 1;
    int cnt = 0;
    for (; i < tasks.size() && cnt < MAX_UPD_TASKS; ++i) {
      if (tasks[i].nvec <= 0 || tasks[i].L <= 0) continue;
      a.t[cnt++] = tasks[i];
      maxL = std::max(maxL, tasks[i].L);
    }
    if (cnt == 0) continue;
    a.ntask = cnt;
    int tn = apply_u_tn(maxL);
    a.tn = tn;
    int tile = 0;
    const int RG = CTA_THREADS / (tn / 4);  // output rows per row block of k_apply_u
    for (int t = 0; t < cnt; ++t) {
      a.t[t].tile0 = tile;
      a.t[t].ntile = (a.t[t].nvec + tn - 1) / tn;
      tile += a.t[t].ntile;
      // flops the kernel executes: (row block, 16 k) tiles outside the band
      // are skipped, and inside a kept tile each warp skips the k outside
      // the union of its rows' ranges, exactly as in k_apply_u
      const UpdTask& q = a.t[t];
      if (cur_flops) *cur_flops += 2.0 * apply_u_entries(q, tn) * q.nvec;
    }
    size_t smem = apply_u_smem_bytes(tn, maxL);
    // one tile per block: blocks stay short (~0.3 ms), so that when the two
    // streams compete the block scheduler can hand freed SMs to the
    // high-priority stream (H updates, chase, AED) between tiles
    int grid = std::min(tile, 1 << 20);
    // the side stream's products leave SMs free for the chase step that
    // runs beside them
    if (on_side && side_reserve > 0)
      grid = std::min(grid, apply_u_blocks_per_sm(tn, smem) * std::max(1, num_sms() - side_reserve));
    int tok = tm.begin(s, phase);
    ++g_stats.kernel_launches;
    ck(launch_apply_u(tn, grid, smem, s, a));
    tm.end(s, tok);
    if (cur_update_phase == PH_UPDATE && timer.depth == 0 && count_launches) g_stats.update_launches += 1;
  }
}

// Entries of U (row k, output row i) that k_apply_u multiplies for one
// vector of task q at tn vectors per tile (its skip rules mirrored).
static double apply_u_entries(const UpdTask& q, int tn) {
  const int VG = tn / 4, RG = CTA_THREADS / VG, rows_per_warp = 32 / VG;
  double entries = 0.0;
  for (int r0 = 0; r0 < q.L; r0 += RG)
    for (int k0 = 0; k0 < q.L; k0 += 16) {
      const int k1 = std::min(q.L, k0 + 16) - 1;
      const bool skip = (k0 - (r0 + RG - 1) > q.lbw) || (r0 - k1 > q.ubw);
      if (skip) continue;
      // warps of the row block: rows r0 + w * rows_per_warp .. + rows_per_warp - 1
      for (int w0 = r0; w0 < std::min(q.L, r0 + RG); w0 += rows_per_warp) {
        const int w1 = std::min(q.L, w0 + rows_per_warp) - 1;
        int lo = 0, hi = q.L - 1;
        if (q.hrng) {
          lo = q.L;
          hi = -1;
          for (int i = w0; i <= w1; ++i) {
            lo = std::min(lo, q.hrng[i].x);
            hi = std::max(hi, q.hrng[i].y);
          }
        }
        const int ka = std::max(k0, lo), kb = std::min(k1, hi);
        if (kb >= ka) entries += (double)(w1 - w0 + 1) * (kb - ka + 1);
      }
    }
  return entries;
}

static UpdTask make_task(double* A, long long lda, int side, int r0, int c0, int L, int nvec, const double* U, int ldu,
                         const int* gate) {
  UpdTask t;
  memset(&t, 0, sizeof(t));
  t.A = A;
  t.lda = lda;
  t.side = side;
  t.r0 = r0;
  t.c0 = c0;
  t.L = L;
  t.nvec = nvec;
  t.U = U;
  t.ldu = ldu;
  t.gate = gate;
  t.lbw = L;
  t.ubw = L;
  return t;
}

// Band of the accumulated transform U of one chase window (U = product of the
// window's reflectors in order; U[r, c] can be nonzero only if column c is
// reached from row r by overlapping reflectors applied later):
//  - downward an index only follows the bulge that first covers it (the bulge
//    ahead is three rows lower and is moved first in every step), so
//    c - r <= (steps in the window - 1) + 2 <= delta + 1;
//  - upward it passes to the next bulge above once per step, two rows each
//    time, so r - c <= 2 + 2 min(nb - 1, delta - 1).
// Entries outside the band are exact zeros of the identity U starts from.
static void set_chase_band(UpdTask& t, int nb, int delta) {
  t.lbw = std::min(t.L, 2 + 2 * std::min(nb - 1, delta - 1));
  t.ubw = std::min(t.L, delta + 1);
}

// Apply an accumulated L x L transform of the diagonal block [k0, k0+L) to
// the rest of H (full Schur form: columns right of the block, rows above it)
// and to Z's columns k0..k0+L-1.
void Solver::apply_block_transform(const Mat3& M, int k0, int L, const double* U, int ldu, const int* gate,
                                   bool with_z) {
  std::vector<UpdTask> t1, t2;
  if (k0 + L < M.n) t1.push_back(make_task(M.H, M.ldh, 0, k0, k0 + L, L, M.n - k0 - L, U, ldu, gate));
  if (M.Z && with_z) t1.push_back(make_task(M.Z, M.ldz, 1, 0, k0, L, M.zrows, U, ldu, gate));
  if (k0 > 0) t2.push_back(make_task(M.H, M.ldh, 1, 0, k0, L, k0, U, ldu, gate));
  // left products and right products touch H[k0.., k0..] on disjoint sets:
  // left: rows k0..k0+L-1, columns >= k0+L; right: rows < k0, columns of
  // the block -- so they can share a launch.
  for (auto& x : t2) t1.push_back(x);
  run_updates(t1);
}

// ---------------------------------------------------------------------------
// One multishift sweep (Sec. 2.3) on [lo, hi] with npairs pairs (device).
// ---------------------------------------------------------------------------
// Row range of the nonzeros in each column of one chase window's U (U starts
// as I; a reflector on columns kl..kl+nr-1 gives all of them the union of
// their ranges): the chase kernel's own bookkeeping, replayed on the host to
// count the products' executed flops.  It depends on the schedule only.
static void chase_u_ranges(int lo, int hi, int ws, int we, int tau0, int tau1, int nb, std::vector<int2>& r) {
  const int L = we - ws + 1;
  r.resize(L);
  for (int c = 0; c < L; ++c) r[c] = make_int2(c, c);
  for (int tau = tau0; tau < tau1; ++tau)
    for (int j = 0; j < nb; ++j) {
      const int k = lo + tau - 3 * j;
      if (k < lo || k > hi - 1) continue;
      const int nr = std::min(3, hi - k + 1), kl = k - ws;
      int a = r[kl].x, b = r[kl].y;
      for (int t = 1; t < nr; ++t) {
        a = std::min(a, r[kl + t].x);
        b = std::max(b, r[kl + t].y);
      }
      for (int t = 0; t < nr; ++t) r[kl + t] = make_int2(a, b);
    }
}

// The window schedule of one sweep (Sec. 2.3 / 2.4, Fig. 3): npairs bulges
// in chains of at most nbc; chain c starts S launches after chain c-1 so that
// its window stays clear of the chain ahead; in every launch each chain in
// flight moves delta steps inside a window of at most kwin rows.
struct SweepPlan {
  int nbc = 1, kwin = 0, delta = 1, nchain = 0, S = 1, last = 0;
  std::vector<int> nbs, tend, start;
};

static SweepPlan plan_sweep(int lo, int hi, int npairs, int nbc) {
  SweepPlan P;
  nbc = std::max(1, std::min(nbc, std::min(npairs, MAX_BULGES_PER_CHAIN)));
  // every chain in flight must fit one launch (MAX_CHAINS blocks)
  nbc = std::max(nbc, (npairs + MAX_CHAINS - 1) / MAX_CHAINS);
  int kwin = std::min(KWIN_MAX, std::max(6 * nbc, 48));
  int delta = kwin - 3 * nbc - 1;
  if (delta < 1) {
    kwin = 3 * nbc + 2;
    delta = 1;
  }
  P.nbc = nbc;
  P.kwin = kwin;
  P.delta = delta;
  P.nchain = (npairs + nbc - 1) / nbc;
  const int D = kwin + delta + 3 * nbc + 2;
  P.S = (D + delta - 1) / delta;
  P.nbs.resize(P.nchain);
  P.tend.resize(P.nchain);
  P.start.resize(P.nchain);
  for (int c = 0; c < P.nchain; ++c) {
    P.nbs[c] = std::min(nbc, npairs - c * nbc);
    P.tend[c] = (hi - lo - 1) + 3 * (P.nbs[c] - 1);
    P.start[c] = c * P.S;
    const int nl = (P.tend[c] + delta) / delta;  // launches of this chain
    P.last = std::max(P.last, P.start[c] + nl);
  }
  return P;
}

// The chains of launch s (chains in order 0 = ahead, lowest); returns their
// number (<= MAX_CHAINS); window i's U is at uoff = i * CHASE_USLOT(kwin),
// its column ranges kwin^2 doubles further.
static int chase_launch(const SweepPlan& P, int lo, int hi, int s, ChaseArgs& a) {
  memset(&a, 0, sizeof(a));
  a.lo = lo;
  a.hi = hi;
  a.ldu = P.kwin;
  int na = 0;
  for (int c = 0; c < P.nchain && na < MAX_CHAINS; ++c) {
    if (s < P.start[c]) continue;
    const int tau0 = (s - P.start[c]) * P.delta;
    if (tau0 > P.tend[c]) continue;
    const int tau1 = std::min(tau0 + P.delta, P.tend[c] + 1);
    const int nb = P.nbs[c];
    const int kmin = std::max(lo, lo + tau0 - 3 * (nb - 1));
    const int kmax = std::min(hi - 1, lo + tau1 - 1);
    if (kmin > kmax) continue;
    ChainDesc& d = a.c[na];
    d.ws = (kmin == lo) ? lo : kmin - 1;
    d.we = std::min(kmax + 3, hi);
    d.tau0 = tau0;
    d.tau1 = tau1;
    d.pair0 = c * P.nbc;
    d.nb = nb;
    d.uoff = na * CHASE_USLOT(P.kwin);
    ++na;
  }
  a.nchain = na;
  return na;
}

// Products of one chase step on four streams (level 0, opts.split_products).  For each window
// (rows/columns ws..we, transform U):
//   near   U^T on rows ws..we, the columns up to the last column of any next-
//          step window sharing its rows: all the next chase step needs -- on
//          the main stream;
//   far    U^T on the remaining columns -- on the far stream, beside the
//          next chase step;
//   right  H U on the rows above the window, the rows of the windows above it
//          left out -- on the side stream;
//   cross  H U on the rows of each window above it (the blocks where another
//          window's left products meet this window's right products) -- on
//          the far stream after that window's near and far products;
//   Z      as before, deferred to the Z stream.
// Order between steps: near(s) after far/cross(s-1) and right(s-1) (the rows
// of a window overlap those of the previous step); far(s) after right(s-1);
// right(s) after far/cross(s-1).  Right products never meet the next chase
// step's windows (the schedule is built that way).
// The products of chase step s as rectangles of H (or Z), by kind:
// 0 near (main), 1 far (far stream), 2 cross (far stream, after near),
// 3 right (side stream), 4 Z.  side 0: rows r0..r0+L-1, columns
// c0..c0+nvec-1; side 1: rows r0..r0+nvec-1, columns c0..c0+L-1.
struct SplitRect {
  int kind, chain, side, r0, c0, L, nvec;
};

static void split_rects(const SweepPlan& plan, int lo, int hi, int s, const ChaseArgs& a, int na, int n, bool with_z,
                        std::vector<SplitRect>& out) {
  ChaseArgs an;
  const int nan = (s + 1 < plan.last) ? chase_launch(plan, lo, hi, s + 1, an) : 0;
  for (int i = 0; i < na; ++i) {
    const ChainDesc& d = a.c[i];
    const int L = d.we - d.ws + 1;
    auto add = [&](int kind, int side, int r0, int c0, int nvec) {
      if (nvec > 0) out.push_back(SplitRect{kind, i, side, r0, c0, L, nvec});
    };
    // near: up to the last column of any next-step window that shares rows
    int near_end = d.we;
    for (int k = 0; k < nan; ++k)
      if (an.c[k].ws <= d.we && d.ws <= an.c[k].we) near_end = std::max(near_end, an.c[k].we);
    near_end = std::min(near_end, n - 1);
    add(0, 0, d.ws, d.we + 1, near_end - d.we);
    add(1, 0, d.ws, near_end + 1, n - near_end - 1);
    if (with_z) add(4, 1, 0, d.ws, n);
    // rows above the window: the gaps between the windows above are right
    // products, the windows' own rows cross blocks
    std::vector<std::pair<int, int>> above;
    for (int j = 0; j < na; ++j)
      if (a.c[j].we < d.ws) above.push_back({a.c[j].ws, a.c[j].we});
    std::sort(above.begin(), above.end());
    int cur = 0;
    for (auto& w : above) {
      add(3, 1, cur, d.ws, w.first - cur);
      add(2, 1, w.first, d.ws, w.second - w.first + 1);
      cur = w.second + 1;
    }
    add(3, 1, cur, d.ws, d.ws - cur);
  }
}

void Solver::sweep_step_split(const Mat3& M, const SweepPlan& plan, int lo, int hi, int s, const ChaseArgs& a,
                              int na, double* ubase, size_t need, bool zasync, bool use_arena) {
  const int kwin = plan.kwin, delta = plan.delta;
  std::vector<SplitRect> rects;
  split_rects(plan, lo, hi, s, a, na, M.n, M.Z != nullptr, rects);
  std::vector<UpdTask> tn, tf, tx, t2, tz;
  std::vector<const int2*> hr(na);
  for (int i = 0; i < na; ++i) {
    const ChainDesc& d = a.c[i];
    host_ranges.emplace_back();
    chase_u_ranges(lo, hi, d.ws, d.we, d.tau0, d.tau1, d.nb, host_ranges.back());
    hr[i] = host_ranges.back().data();
  }
  for (const SplitRect& r : rects) {
    const ChainDesc& d = a.c[r.chain];
    const double* U = ubase + d.uoff;
    std::vector<UpdTask>& v = (r.kind == 0) ? tn : (r.kind == 1) ? tf : (r.kind == 2) ? tx : (r.kind == 3) ? t2
                              : (zasync ? tz : tf);
    double* A = (r.kind == 4) ? M.Z : M.H;
    const long long ld = (r.kind == 4) ? M.ldz : M.ldh;
    const int nvec = (r.kind == 4) ? M.zrows : r.nvec;
    v.push_back(make_task(A, ld, r.side, r.r0, r.c0, r.L, nvec, U, kwin, nullptr));
    set_chase_band(v.back(), d.nb, delta);
    v.back().rng = (const int2*)(U + (size_t)kwin * kwin);
    v.back().hrng = hr[r.chain];
  }
  if (zasync) z_defer(tz, ubase, need);
  else if (use_arena) arena_release(ubase, need, false);
  // main: the next chase step needs only the near products
  ck(cudaEventRecord(ev_c, st));
  if (f_pending) ck(cudaStreamWaitEvent(st, ev_f, 0));
  if (t2_pending) ck(cudaStreamWaitEvent(st, ev_t2, 0));
  run_updates(tn);
  ck(cudaEventRecord(ev_n, st));
  // side: right products after this step's transforms and the previous
  // far/cross products; far: after this step's transforms and the previous
  // right products.  (Holding both back until the near products are done
  // keeps the next chase step's SMs free but leaves the products less time:
  // measured slower.)
  ck(cudaStreamWaitEvent(sst, ev_c, 0));
  if (f_pending) ck(cudaStreamWaitEvent(sst, ev_f, 0));
  ck(cudaStreamWaitEvent(fst, ev_c, 0));
  if (t2_pending) ck(cudaStreamWaitEvent(fst, ev_t2, 0));
  run_updates(tf, fst);
  if (!tx.empty()) {
    ck(cudaStreamWaitEvent(fst, ev_n, 0));
    run_updates(tx, fst);
  }
  ck(cudaEventRecord(ev_f, fst));
  f_pending = true;
  f_a = use_arena ? (size_t)(ubase - arena) : 0;
  f_b = use_arena ? f_a + need : 0;
  run_updates(t2, sst);
  ck(cudaEventRecord(ev_t2, sst));
  t2_pending = true;
  t2_a = f_a;
  t2_b = f_b;
}

void Solver::sweep(const Mat3& M, int lev, int lo, int hi, const double* dpairs, int npairs, int nbc_req) {
  Level& Lv = levels[lev];
  const int nbc0 = nbc_req > 0 ? nbc_req : (opts.bulges_per_chain > 0 ? opts.bulges_per_chain : 16);
  const SweepPlan plan = plan_sweep(lo, hi, npairs, nbc0);
  const int kwin = plan.kwin, delta = plan.delta, nchain = plan.nchain, last = plan.last;
  size_t smem = chase_smem_bytes(kwin);
  const bool zasync = (lev == 0 && zst != nullptr && M.Z != nullptr);
  const bool side = (lev == 0 && sst != nullptr);
  const bool use_arena = zasync || side;
  side_reserve = std::min(nchain, MAX_CHAINS) + 2;
  for (int s = 0; s < last; ++s) {
    ChaseArgs a;
    const int na = chase_launch(plan, lo, hi, s, a);
    if (na == 0) continue;
    // this step's window transforms: from the arena while the Z or the side
    // stream may still need them, else the level's buffer
    const size_t need = (size_t)na * CHASE_USLOT(kwin);
    double* ubase = use_arena ? arena_alloc(need) : Lv.ubuf;
    int tok = timer.begin(st, PH_CHASE);
    ++g_stats.kernel_launches;
    k_chase<<<na, CHASE_THREADS, smem, st>>>(M.H, M.ldh, dpairs, ubase, a);
    ck(cudaGetLastError());
    timer.end(st, tok);
    g_stats.window_launches += 1;
    if (lev == 0) g_stats.chase_launches += 1;
    count_launches = (lev == 0);
    if (side && fst && opts.split_products) {
      sweep_step_split(M, plan, lo, hi, s, a, na, ubase, need, zasync, use_arena);
      continue;
    }
    std::vector<UpdTask> t1, t2, tz;
    for (int i = 0; i < na; ++i) {
      const ChainDesc& d = a.c[i];
      int L = d.we - d.ws + 1;
      const double* U = ubase + d.uoff;
      const int2* rng = (const int2*)(U + (size_t)kwin * kwin);
      host_ranges.emplace_back();
      chase_u_ranges(lo, hi, d.ws, d.we, d.tau0, d.tau1, d.nb, host_ranges.back());
      const int2* hrng = host_ranges.back().data();
      auto ranged = [&](UpdTask& t) {
        t.rng = rng;
        t.hrng = hrng;
      };
      if (d.we + 1 < M.n) {
        t1.push_back(make_task(M.H, M.ldh, 0, d.ws, d.we + 1, L, M.n - d.we - 1, U, kwin, nullptr));
        set_chase_band(t1.back(), d.nb, delta);
        ranged(t1.back());
      }
      if (M.Z) {
        std::vector<UpdTask>& tzv = zasync ? tz : t1;
        tzv.push_back(make_task(M.Z, M.ldz, 1, 0, d.ws, L, M.zrows, U, kwin, nullptr));
        set_chase_band(tzv.back(), d.nb, delta);
        ranged(tzv.back());
      }
      if (d.ws > 0) {
        t2.push_back(make_task(M.H, M.ldh, 1, 0, d.ws, L, d.ws, U, kwin, nullptr));
        set_chase_band(t2.back(), d.nb, delta);
        ranged(t2.back());
      }
    }
    if (zasync) z_defer(tz, ubase, need);   // issued on zst at the end of the sweep
    else if (use_arena) arena_release(ubase, need, false);
    if (side) {
      // t1 meets the previous step's t2 where a chain's rows cross the
      // columns of the chain ahead of it
      if (t2_pending) ck(cudaStreamWaitEvent(st, ev_t2, 0));
      run_updates(t1);
      if (!t2.empty()) {
        ck(cudaEventRecord(ev_t1, st));
        ck(cudaStreamWaitEvent(sst, ev_t1, 0));
        run_updates(t2, sst);
        ck(cudaEventRecord(ev_t2, sst));
        t2_pending = true;
        t2_a = use_arena ? (size_t)(ubase - arena) : 0;
        t2_b = use_arena ? t2_a + need : 0;
      } else {
        t2_pending = false;
      }
    } else {
      run_updates(t1);
      run_updates(t2);
    }
  }
  if (t2_pending) {
    ck(cudaStreamWaitEvent(st, ev_t2, 0));
    t2_pending = false;
  }
  if (f_pending) {
    ck(cudaStreamWaitEvent(st, ev_f, 0));
    f_pending = false;
  }
  if (zasync) z_flush();
  host_ranges.clear();   // every task of the sweep has been issued
  if (lev == 0) {
    // algorithmic flops of applying the reflectors directly (12 flops per
    // row/column entry of each 3x3 reflector): every bulge passes rows
    // lo..hi; a reflector at row k touches n-k columns, k+4 rows and zrows
    // rows of Z.
    double m = hi - lo + 1;
    double avgk = 0.5 * (lo + hi);
    g_stats.reflector_flops += 12.0 * npairs * m * ((M.n - avgk) + (avgk + 4) + (M.Z ? M.zrows : 0));
  }
}

// ---------------------------------------------------------------------------
// The iteration of Sec. 2.1 on rows/cols ilo..ihi of M (full Schur form).
// ---------------------------------------------------------------------------
int Solver::qr_block(const Mat3& M, int lev, int ilo, int ihi) {
  Level& Lv = levels[lev];
  DeflParams dp = defl(M.n);
  int kbot = ihi;
  int itmax = 30 * std::max(10, ihi - ilo + 1);
  int it = 0;
  int ndfl = 1;
  while (kbot >= ilo) {
    ++g_stats.kernel_launches;
    k_scan<<<1, CTA_THREADS, 0, st>>>(M.H, M.ldh, ilo, kbot, dp, Lv.ctl);
    ck(cudaGetLastError());
    read_ctl(Lv.ctl);
    int ktop = hctl->ktop;
    int m = kbot - ktop + 1;
    if (m == 1) {
      kbot -= 1;
      ndfl = 1;
      continue;
    }
    if (m == 2) {
      if (lev == 0) drain_z();
      ++g_stats.kernel_launches;
      k_std2<<<1, CTA_THREADS, 0, st>>>(M.H, M.ldh, M.n, M.Z, M.ldz, M.Z ? M.zrows : 0, ktop);
      ck(cudaGetLastError());
      kbot -= 2;
      ndfl = 1;
      continue;
    }
    if (m <= opts.nmin) {
      if (lev == 0) drain_z();
      size_t smem = (size_t)(m | 1) * m * sizeof(double);
      int tok = timer.begin(st, PH_SMALL);
      ++g_stats.kernel_launches;
      k_smallqr<<<1, CTA_THREADS, smem, st>>>(M.H, M.ldh, ktop, kbot, Lv.usmall, m, dp, Lv.ctl);
      ck(cudaGetLastError());
      apply_block_transform(M, ktop, m, Lv.usmall, m, nullptr);
      timer.end(st, tok);
      read_ctl(Lv.ctl);
      if (lev == 0) g_stats.small_qr += 1;
      if (hctl->info) return hctl->info;
      kbot = ktop - 1;
      ndfl = 1;
      continue;
    }
    ++it;
    if (it > itmax) return kbot + 1;
    int ns_max, nw;
    default_ns_nw(m, &ns_max, &nw);
    if (lev == 0) {
      if (opts.n_shifts > 0) ns_max = opts.n_shifts;
      if (opts.aed_window > 0) nw = opts.aed_window;
    }
    nw = std::min(std::min(std::min(nw, m), Lv.nwmax), 1024);
    int nd = aed(M, lev, ktop, kbot, nw, ns_max, ndfl);
    if (lev == 0) {
      g_stats.aed_steps += 1;
      g_stats.deflated_by_aed += nd;
    }
    kbot -= nd;
    ndfl = hctl->ndfl;
    int npairs = hctl->npairs;
    m = kbot - ktop + 1;
    if (m <= opts.nmin) continue;
    if (nd > 0 && 100 * nd > opts.nibble * nw) continue;
    if (npairs <= 0) continue;
    sweep(M, lev, ktop, kbot, Lv.pairs, npairs, 0);
    if (lev == 0) g_stats.sweeps += 1;
  }
  return 0;
}

// AED (Sec. 2.5) on the trailing nw x nw window of [ktop, kbot]; returns nd
// and leaves the control block (npairs, ndfl, ncand) in hctl.
int Solver::aed(const Mat3& M, int lev, int ktop, int kbot, int nw, int ns_max, int ndfl) {
  Level& Lv = levels[lev];
  DeflParams dp = defl(M.n);
  DeflParams dpw = defl(nw);
  int kwtop = kbot - nw + 1;
  double* saved = cur_flops;
  if (lev == 0) cur_flops = &g_stats.aed_gemm_flops;
  // ring slot of V (reused only after the Z stream has applied it)
  const bool zasync = (lev == 0 && zst != nullptr && M.Z != nullptr);
  double* V = zasync ? arena_alloc((size_t)nw * nw) : Lv.V;
  int tok = timer.begin(st, PH_AED);
  // the window's Schur form: double-shift QR in one block up to the
  // crossover, the recursive iteration above it; windows of windows always
  // use double-shift QR
  const bool in_block = nw <= NW_SMEM_MAX && (lev > 0 || nw <= window_francis_max(opts));
  if (in_block) {
    size_t smem = (size_t)(nw | 1) * nw * sizeof(double);
    ++g_stats.kernel_launches;
    // a cluster of two blocks: the window on one, its transform V on the other
    k_aed_small<<<2, CTA_THREADS, smem, st>>>(M.H, M.ldh, ktop, kbot, nw, V, nw, Lv.cand_re, Lv.cand_im, Lv.vbuf,
                                             dp, dpw, Lv.ctl);
    ck(cudaGetLastError());
  } else {
    ++g_stats.kernel_launches;
    k_copy_window<<<std::min(nw, 4 * num_sms()), CTA_THREADS, 0, st>>>(M.H, M.ldh, kwtop, nw, Lv.T, nw, V, nw);
    ck(cudaGetLastError());
    Mat3 W{Lv.T, nw, nw, V, nw, nw};
    double* keep = cur_flops;
    cur_flops = nullptr;
    int inner = qr_block(W, lev + 1, 0, nw - 1);
    cur_flops = keep;
    ++g_stats.kernel_launches;
    k_aed_big_post<<<1, CTA_THREADS, 0, st>>>(M.H, M.ldh, ktop, kbot, nw, Lv.T, nw, V, nw, Lv.cand_re, Lv.cand_im,
                                              Lv.vbuf, dp, Lv.ctl, inner);
    ck(cudaGetLastError());
  }
  timer.end(st, tok);
  int saved_phase = cur_update_phase;
  cur_update_phase = PH_AED_UPDATE;
  apply_block_transform(M, kwtop, nw, V, nw, &Lv.ctl->nd, !zasync);
  if (opts.recompute_shifts) {
    const int r = std::min(std::min(ns_max, NW_SMEM_MAX), kbot - ktop + 1);
    ++g_stats.kernel_launches;
    k_recompute_shifts<<<1, CTA_THREADS, (size_t)(r | 1) * r * sizeof(double), st>>>(
        M.H, M.ldh, ktop, kbot, ns_max, nw, opts.nibble, opts.nmin, Lv.cand_re, Lv.cand_im, dp, Lv.ctl);
    ck(cudaGetLastError());
  }
  ++g_stats.kernel_launches;
  k_make_pairs<<<1, 32, 0, st>>>(M.H, M.ldh, ktop, kbot, std::min(ns_max, Lv.nsmax + 8 - 4), ndfl, 6, Lv.cand_re,
                                 Lv.cand_im, Lv.pairs, Lv.ctl);
  ck(cudaGetLastError());
  read_ctl(Lv.ctl);
  if (hctl->sync_err) {
    snprintf(g_err_detail, sizeof(g_err_detail), "the AED kernel's transform stream between its two blocks timed out");
    throw CudaError{cudaErrorLaunchTimeout};
  }
  if (zasync) {
    if (hctl->nd > 0) {
      std::vector<UpdTask> tz{make_task(M.Z, M.ldz, 1, 0, kwtop, nw, M.zrows, V, nw, nullptr)};
      z_async(tz, nullptr);
    }
    arena_release(V, (size_t)nw * nw, hctl->nd > 0);
  }
  cur_update_phase = saved_phase;
  cur_flops = saved;
  return hctl->nd;
}

}  // namespace schur

// ===========================================================================
// C ABI
// ===========================================================================
using namespace schur;

extern "C" int schur_default_opts(schur_opts* o) {
  if (!o) return -1;
  memset(o, 0, sizeof(*o));
  o->struct_size = (int)sizeof(schur_opts);
  o->nmin = 75;
  o->nibble = 14;
  o->deflation = SCHUR_DEFLATION_LAPACK;
  o->want_z = 1;
  o->z_init = 0;
  return SCHUR_OK;
}

extern "C" const char* schur_status_string(int code) { return status_string(code); }

extern "C" int schur_workspace_size(int n, const schur_opts* opts, size_t* bytes) {
  if (n < 0) return -1;
  if (!bytes) return -3;
  schur_opts o;
  read_opts(opts, &o);
  *bytes = workspace_bytes(std::max(n, 1), o);
  return SCHUR_OK;
}

extern "C" const char* schur_last_error_detail(void) { return g_err_detail; }

extern "C" int schur_last_stats(schur_stats* out) {
  if (!out) return -1;
  *out = g_stats;
  return SCHUR_OK;
}

static int frob_norm(const double* H, long long ldh, int n, cudaStream_t st, double* out);

extern "C" int schur_hessenberg(int n, double* H, int ldh, double* Z, int ldz, double* wr, double* wi,
                                const schur_opts* opts) {
  if (n < 0) return -1;
  if (n > 0 && H == nullptr) return -2;
  if (ldh < std::max(1, n)) return -3;
  schur_opts oq;
  schur::read_opts(opts, &oq);
  int want_z = oq.want_z;
  if (want_z && n > 0 && Z == nullptr) return -4;
  if (want_z && ldz < std::max(1, n)) return -5;
  if (n > 0 && wr == nullptr) return -6;
  if (n > 0 && wi == nullptr) return -7;
  memset(&g_stats, 0, sizeof(g_stats));
  if (n == 0) return SCHUR_OK;
  try {
    Solver s(opts);
    if (!s.opts.want_z) Z = nullptr;
    int rc = s.setup(n);
    if (rc) return rc;
    ck(cudaMemsetAsync(s.flag, 0, sizeof(int), s.st));
    int grid = std::min(n, 8 * num_sms());
    ++g_stats.kernel_launches;
    k_prep<<<grid, CTA_THREADS, 0, s.st>>>(H, ldh, n, Z, ldz, s.opts.z_init, s.flag);
    ck(cudaGetLastError());
    int hflag = 0;
    ck(cudaMemcpyAsync(&hflag, s.flag, sizeof(int), cudaMemcpyDeviceToHost, s.st));
    ck(cudaStreamSynchronize(s.st));
    if (hflag) return SCHUR_ERR_NONFINITE;
    if (s.opts.deflation == SCHUR_DEFLATION_NORM) {
      int r = frob_norm(H, ldh, n, s.st, &s.normH);
      if (r) return r;
    }
    Mat3 M{H, ldh, n, Z, ldz, n};
    s.cur_flops = &g_stats.sweep_gemm_flops;
    s.init_streams(Z != nullptr);
    int info = s.qr_block(M, 0, 0, n - 1);
    s.drain_z();
    ++g_stats.kernel_launches;
    k_extract_eigs<<<std::max(1, std::min((n + 255) / 256, 4 * num_sms())), 256, 0, s.st>>>(H, ldh, n, wr, wi);
    ck(cudaGetLastError());
    s.join_caller();
    ck(cudaStreamSynchronize(s.st));
    s.timer.flush();
    s.read_ctl(s.levels[0].ctl);
    for (cudaStream_t x : {s.zst, s.sst, s.fst})
      if (x) ck(cudaStreamSynchronize(x));
    s.ztimer.flush_completed();
    s.stimer.flush_completed();
    s.ftimer.flush_completed();
    for (int ph = 0; ph < PH_COUNT; ++ph) s.timer.ms[ph] += s.ztimer.ms[ph] + s.stimer.ms[ph] + s.ftimer.ms[ph];
    s.write_trace();
    g_stats.aed_cycles_schur = (double)s.hctl->cyc_schur;
    g_stats.shift_recomputations = s.hctl->recomputed;
    g_stats.aed_cycles_post = (double)s.hctl->cyc_defl;
    g_stats.t_chase_ms = s.timer.ms[PH_CHASE];
    g_stats.t_update_ms = s.timer.ms[PH_UPDATE];
    g_stats.t_aed_ms = s.timer.ms[PH_AED];
    g_stats.t_aed_update_ms = s.timer.ms[PH_AED_UPDATE];
    g_stats.t_small_ms = s.timer.ms[PH_SMALL];
    g_stats.t_z_ms = s.timer.ms[PH_Z];
    return info;
  } catch (const CudaError&) {
    return SCHUR_ERR_CUDA;
  }
}

// ---------------------------------------------------------------------------
// ||H||_F of the Hessenberg part (norm-stable deflation, Sec. 5.6 item 2)
// ---------------------------------------------------------------------------
__global__ void k_frob(const double* H, long long ldh, int n, double* out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int j = blockIdx.x; j < n; j += gridDim.x)
    for (int i = threadIdx.x; i <= min(j + 1, n - 1); i += blockDim.x) {
      double v = H[i + (long long)j * ldh];
      s += v * v;
    }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) t += red[w];
    atomicAdd(out, t);
  }
}

static int frob_norm(const double* H, long long ldh, int n, cudaStream_t st, double* out) {
  double* d = nullptr;
  if (cudaMalloc((void**)&d, sizeof(double)) != cudaSuccess) return SCHUR_ERR_NOMEM;
  cudaMemsetAsync(d, 0, sizeof(double), st);
  k_frob<<<std::min(n, 4 * num_sms()), 256, 0, st>>>(H, ldh, n, d);
  double h = 0.0;
  cudaMemcpyAsync(&h, d, sizeof(double), cudaMemcpyDeviceToHost, st);
  cudaError_t e = cudaStreamSynchronize(st);
  cudaFree(d);
  if (e != cudaSuccess) return SCHUR_ERR_CUDA;
  *out = sqrt(h);
  return SCHUR_OK;
}

// ---------------------------------------------------------------------------
// Single steps (parity tests)
// ---------------------------------------------------------------------------
extern "C" int schur_sweep(int n, double* H, int ldh, double* Z, int ldz, int ilo, int ihi, const double* pairs,
                           int npairs, int bulges_per_chain, const schur_opts* opts) {
  if (n < 1) return -1;
  if (!H) return -2;
  if (ldh < n) return -3;
  if (Z && ldz < n) return -5;
  if (ilo < 0 || ilo >= n) return -6;
  if (ihi < ilo + 2 || ihi >= n) return -7;
  if (!pairs) return -8;
  if (npairs < 1 || npairs > MAX_CHAINS * MAX_BULGES_PER_CHAIN) return -9;
  try {
    Solver s(opts);
    int rc = s.setup(n);
    if (rc) return rc;
    double* dpairs = nullptr;
    ck(cudaMalloc((void**)&dpairs, 2 * npairs * sizeof(double)));
    ck(cudaMemcpyAsync(dpairs, pairs, 2 * npairs * sizeof(double), cudaMemcpyHostToDevice, s.st));
    Mat3 M{H, ldh, n, Z, ldz, n};
    s.sweep(M, 0, ilo, ihi, dpairs, npairs, bulges_per_chain);
    ck(cudaStreamSynchronize(s.st));
    cudaFree(dpairs);
    return SCHUR_OK;
  } catch (const CudaError&) {
    return SCHUR_ERR_CUDA;
  }
}

extern "C" int schur_aed(int n, double* H, int ldh, double* Z, int ldz, int ktop, int kbot, int nw, int* nd,
                         double* cand_re, double* cand_im, int* ncand, const schur_opts* opts) {
  if (n < 1) return -1;
  if (!H) return -2;
  if (ldh < n) return -3;
  if (Z && ldz < n) return -5;
  if (ktop < 0 || ktop >= n) return -6;
  if (kbot < ktop || kbot >= n) return -7;
  if (nw < 1 || nw > kbot - ktop + 1) return -8;
  if (!nd) return -9;
  try {
    schur_opts o;
    read_opts(opts, &o);
    o.aed_window = nw;
    Solver s(&o);
    int rc = s.setup(n);
    if (rc) return rc;
    if (s.opts.deflation == SCHUR_DEFLATION_NORM) {
      int r = frob_norm(H, ldh, n, s.st, &s.normH);
      if (r) return r;
    }
    Mat3 M{H, ldh, n, Z, ldz, n};
    int d = s.aed(M, 0, ktop, kbot, nw, 8, 1);
    *nd = d;
    int nc = s.hctl->ncand;
    if (ncand) *ncand = nc;
    if (cand_re && nc > 0) ck(cudaMemcpy(cand_re, s.levels[0].cand_re, nc * sizeof(double), cudaMemcpyDeviceToHost));
    if (cand_im && nc > 0) ck(cudaMemcpy(cand_im, s.levels[0].cand_im, nc * sizeof(double), cudaMemcpyDeviceToHost));
    return SCHUR_OK;
  } catch (const CudaError&) {
    return SCHUR_ERR_CUDA;
  }
}

extern "C" int schur_small_qr(int n, double* H, int ldh, double* Z, int ldz, int ilo, int ihi, const schur_opts* opts) {
  if (n < 1) return -1;
  if (!H) return -2;
  if (ldh < n) return -3;
  if (Z && ldz < n) return -5;
  if (ilo < 0 || ilo >= n) return -6;
  if (ihi < ilo || ihi >= n || ihi - ilo + 1 > NW_SMEM_MAX) return -7;
  try {
    Solver s(opts);
    int rc = s.setup(n);
    if (rc) return rc;
    int m = ihi - ilo + 1;
    Mat3 M{H, ldh, n, Z, ldz, n};
    DeflParams dp = s.defl(n);
    size_t smem = (size_t)(m | 1) * m * sizeof(double);
    ++g_stats.kernel_launches;
    k_smallqr<<<1, CTA_THREADS, smem, s.st>>>(H, ldh, ilo, ihi, s.levels[0].usmall, m, dp, s.levels[0].ctl);
    ck(cudaGetLastError());
    s.apply_block_transform(M, ilo, m, s.levels[0].usmall, m, nullptr);
    s.read_ctl(s.levels[0].ctl);
    return s.hctl->info;
  } catch (const CudaError&) {
    return SCHUR_ERR_CUDA;
  }
}

extern "C" int schur_apply_u(int side, double* A, int lda, int r0, int c0, int m, int k, const double* U, int ldu,
                             const schur_opts* opts) {
  if (side != 0 && side != 1) return -1;
  if (!A) return -2;
  if (lda < 1) return -3;
  if (r0 < 0) return -4;
  if (c0 < 0) return -5;
  if (m < 0) return -6;
  if (k < 1 || k > 1024) return -7;
  if (!U) return -8;
  if (ldu < k) return -9;
  try {
    Solver s(opts);
    init_kernel_attributes();
    std::vector<UpdTask> t;
    t.push_back(make_task(A, lda, side, r0, c0, k, m, U, ldu, nullptr));
    s.run_updates(t);
    ck(cudaStreamSynchronize(s.st));
    return SCHUR_OK;
  } catch (const CudaError&) {
    return SCHUR_ERR_CUDA;
  }
}

extern "C" int schur_fastmath_eval(int n, const double* x, double* out, const schur_opts* opts) {
  if (n < 0) return -1;
  if (n > 0 && !x) return -2;
  if (n > 0 && !out) return -3;
  if (n == 0) return SCHUR_OK;
  schur_opts o;
  read_opts(opts, &o);
  cudaStream_t st = (cudaStream_t)o.stream;
  k_fastmath_eval<<<std::min((n + 255) / 256, 1024), 256, 0, st>>>(n, x, out);
  if (cudaGetLastError() != cudaSuccess) return SCHUR_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return SCHUR_ERR_CUDA;
  return SCHUR_OK;
}

static int deflation_eval(int which, int count, const double* data, int mode, double thold, double normH, int n,
                          int* out, const schur_opts* opts) {
  if (count < 0) return -1;
  if (count > 0 && !data) return -2;
  if (mode < SCHUR_DEFLATION_LAPACK || mode > SCHUR_DEFLATION_FIXED) return -3;
  if (n < 1) return -6;
  if (count > 0 && !out) return -7;
  if (count == 0) return SCHUR_OK;
  schur_opts o;
  read_opts(opts, &o);
  cudaStream_t st = (cudaStream_t)o.stream;
  DeflParams dp;
  dp.mode = mode;
  dp.thold = thold;
  dp.normH = normH;
  dp.n = n;
  const int grid = std::min((count + 255) / 256, 1024);
  if (which == 0)
    k_vigilant_eval<<<grid, 256, 0, st>>>(count, data, dp, out);
  else
    k_spike_eval<<<grid, 256, 0, st>>>(count, data, dp, out);
  if (cudaGetLastError() != cudaSuccess) return SCHUR_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return SCHUR_ERR_CUDA;
  return SCHUR_OK;
}

extern "C" int schur_vigilant_eval(int count, const double* H, int mode, double thold, double normH, int n, int* out,
                                   const schur_opts* opts) {
  return deflation_eval(0, count, H, mode, thold, normH, n, out, opts);
}

extern "C" int schur_spike_eval(int count, const double* blk, int mode, double thold, double normH, int n, int* out,
                                const schur_opts* opts) {
  return deflation_eval(1, count, blk, mode, thold, normH, n, out, opts);
}

// ---------------------------------------------------------------------------
// The chase schedule of a sweep, as the driver issues it (host only).
// ---------------------------------------------------------------------------
extern "C" int schur_chase_schedule(int lo, int hi, int npairs, int bulges_per_chain, int cap, int* rec, int* count,
                                    int* kwin, int* delta) {
  if (lo < 0) return -1;
  if (hi < lo + 2) return -2;
  if (npairs < 1 || npairs > MAX_CHAINS * MAX_BULGES_PER_CHAIN) return -3;
  if (bulges_per_chain < 0) return -4;
  if (cap < 0) return -5;
  if (cap > 0 && !rec) return -6;
  if (!count) return -7;
  const SweepPlan P = plan_sweep(lo, hi, npairs, bulges_per_chain > 0 ? bulges_per_chain : 16);
  if (kwin) *kwin = P.kwin;
  if (delta) *delta = P.delta;
  int nrec = 0;
  for (int s = 0; s < P.last; ++s) {
    ChaseArgs a;
    const int na = chase_launch(P, lo, hi, s, a);
    for (int i = 0; i < na; ++i, ++nrec) {
      if (nrec >= cap) continue;
      int* r = rec + 7 * (size_t)nrec;
      const ChainDesc& d = a.c[i];
      r[0] = s;
      r[1] = d.ws;
      r[2] = d.we;
      r[3] = d.tau0;
      r[4] = d.tau1;
      r[5] = d.pair0;
      r[6] = d.nb;
    }
  }
  *count = nrec;
  return SCHUR_OK;
}

// ---------------------------------------------------------------------------
// FP64 FMA throughput probe (the roofline's in-run peak).
// ---------------------------------------------------------------------------
extern "C" int schur_sweep_split_tasks(int n, int lo, int hi, int npairs, int bulges_per_chain, int cap, int* rec,
                                      int* count) {
  if (n < 1) return -1;
  if (lo < 0 || lo > n - 1) return -2;
  if (hi <= lo || hi > n - 1) return -3;
  if (npairs < 1 || npairs > 1024) return -4;
  if (bulges_per_chain < 0) return -5;
  if (cap < 0) return -6;
  if (cap > 0 && !rec) return -7;
  if (!count) return -8;
  const SweepPlan plan = plan_sweep(lo, hi, npairs, bulges_per_chain > 0 ? bulges_per_chain : 16);
  int cnt = 0;
  for (int s = 0; s < plan.last; ++s) {
    ChaseArgs a;
    const int na = chase_launch(plan, lo, hi, s, a);
    if (na == 0) continue;
    std::vector<SplitRect> rects;
    split_rects(plan, lo, hi, s, a, na, n, true, rects);
    for (const SplitRect& r : rects) {
      if (cnt < cap) {
        int* q = rec + 8 * cnt;
        q[0] = s;
        q[1] = r.kind;
        q[2] = r.chain;
        q[3] = r.side;
        q[4] = r.r0;
        q[5] = r.c0;
        q[6] = r.L;
        q[7] = r.nvec;
      }
      ++cnt;
    }
  }
  *count = cnt;
  return SCHUR_OK;
}

extern "C" int schur_fp64_fma_probe(int iters, int blocks, double* out, double* flops, const schur_opts* opts) {
  if (iters < 1) return -1;
  if (blocks < 1) return -2;
  if (!out) return -3;
  if (!flops) return -4;
  schur_opts o;
  read_opts(opts, &o);
  if (fma_probe_launch(iters, blocks, out, (cudaStream_t)o.stream)) return SCHUR_ERR_CUDA;
  *flops = 2.0 * 8.0 * (double)iters * 256.0 * (double)blocks;
  return SCHUR_OK;
}
