// engine.cu -- host engine and C ABI (include/bdm.h) of the GB300
// mechanical-interaction iteration.
//
// The simulation owns all device memory.  One iteration is one captured CUDA
// graph (geometry -> brick ranks -> keys -> brick scan -> scatter -> brick
// sort -> [sort-step gather] -> force/displacement/behaviours -> [division
// merge] -> finish) replayed on an internal stream that is fenced against the
// caller's stream.  The number of agents, the grid geometry and every size
// the kernels need live in device memory, so one graph serves every
// iteration; grid capacities that turn out too small are reported by the
// kernels through a sticky error word before any agent state changes, and the
// host grows the buffers, recaptures and repeats the iteration.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "bdm_internal.cuh"
#include "bdm.h"

#define BDM_ABI_VERSION 200

namespace {
thread_local std::string g_create_error = "no error";

}  // namespace

struct bdm_sim {
  bdm_params P{};
  DevParams dp{};
  cudaStream_t user = nullptr;
  cudaStream_t own = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  // bdm_set_agents: a second stream that copies and checks the positions
  // while the other input arrays are still crossing the host link
  cudaStream_t aux = nullptr;
  cudaEvent_t ev_a = nullptr, ev_b = nullptr;
  std::string err = "no error";
  long long cap = 0;
  int n_sims = 1;
  int sm_count = 152;
  // device memory
  AgentSet sets[2]{};     // host copies of the two sets' pointers
  AgentSet *d_sets = nullptr;  // device: [0] = current, [1] = other (swapped by the sort)
  DevBufs B{};
  LaunchCfg lc{};
  DevCounters *d_ctr = nullptr;
  DevCounters *h_ctr = nullptr;  // pinned
  SimGeom *d_geom = nullptr;
  std::vector<double> dt_sim;
  std::vector<long long> sim_off;
  void *dbg_scratch = nullptr;
  size_t dbg_scratch_bytes = 0;
  bool have_agents = false;
  cudaGraphExec_t exec = nullptr;
  bool graph_ok = false;
  std::vector<void *> allocs_agents, allocs_grid;
  long long kernels = 0;   // kernels launched so far (all entry points)
  // phase profiling (bdm_profile_begin / bdm_profile_end)
  bool prof_on = false;
  std::vector<cudaEvent_t> prof_ev;
  size_t prof_used = 0;
  std::vector<int> prof_phase;  // phase of the interval that starts at event i
  double prof_ms[16] = {0};
  long long prof_launch[16] = {0};
};

// phases of one iteration (bdm_phase_name)
enum Phase { PH_GEOMETRY, PH_BRICK_RANK, PH_KEYS, PH_BRICK_SCAN, PH_SCATTER, PH_BRICK_SORT, PH_GATHER, PH_FORCE,
             PH_FORCE_FIX, PH_DIVIDE, PH_FINISH, PH_COUNT };
static const char *kPhaseNames[PH_COUNT] = {"geometry", "brick_rank", "keys", "brick_scan", "scatter",
                                            "brick_sort", "gather", "force", "force_fix", "divide", "finish"};
static const int kPhaseLaunches[PH_COUNT] = {1, 1, 1, 3, 1, 2, 2, 2, 1, 3, 1};

// ------------------------------------------------------------------ helpers
static int fail(bdm_sim *s, int code, const std::string &msg) {
  if (s) s->err = msg; else g_create_error = msg;
  return code;
}

static int cuda_fail(bdm_sim *s, cudaError_t e, const char *what) {
  return fail(s, BDM_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                        \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(s, e_, #call); \
  } while (0)

static int dmalloc(bdm_sim *s, void **p, size_t bytes, std::vector<void *> &list) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(s, BDM_ENOMEM, std::string("cudaMalloc of ") + std::to_string(bytes) + " bytes failed: " +
                                   cudaGetErrorString(e));
  }
  list.push_back(*p);
  return BDM_OK;
}

static void free_list(std::vector<void *> &list) {
  for (void *p : list) cudaFree(p);
  list.clear();
}

// device-side parameters (params.cu)
DevParams make_dev_params(const bdm_params &P);


static void make_launch_cfg(bdm_sim *s) {
  const long long sm = s->sm_count;
  auto clampb = [](long long v, long long lo, long long hi) { return (int)std::max(lo, std::min(v, hi)); };
  s->lc.agent_blocks = clampb((s->cap + 255) / 256, 1, sm * 8);
  s->lc.brick_blocks = clampb((s->B.brick_cap + 255) / 256, 1, sm * 8);
  s->lc.scan_blocks = clampb((s->B.brick_cap + SCAN_TILE - 1) / SCAN_TILE, 1, 1LL << 30);
  s->lc.agent_scan_blocks = clampb((s->cap + SCAN_TILE - 1) / SCAN_TILE, 1, 1LL << 30);
  s->lc.occ_blocks = clampb(s->B.occ_cap, 1, sm * 4);
  s->lc.force_blocks = clampb(s->B.occ_cap, 1, sm * 4);
}

static int alloc_grid(bdm_sim *s, long long brick_cap, long long occ_cap) {
  if (s->graph_ok) {
    cudaGraphExecDestroy(s->exec);
    s->exec = nullptr;
    s->graph_ok = false;
  }
  cudaStreamSynchronize(s->own);
  free_list(s->allocs_grid);
  DevBufs &B = s->B;
  B.brick_cap = brick_cap;
  B.occ_cap = occ_cap;
  const long long scan_n = (std::max(brick_cap, s->cap) + SCAN_TILE - 1) / SCAN_TILE + 2;
  int rc = BDM_OK;
  auto A = [&](void **p, size_t bytes) {
    if (rc == BDM_OK) rc = dmalloc(s, p, bytes, s->allocs_grid);
  };
  A((void **)&B.brick_table, sizeof(int32_t) * brick_cap);
  A((void **)&B.brick_count, sizeof(uint32_t) * brick_cap);
  A((void **)&B.brick_start, sizeof(uint32_t) * brick_cap);
  A((void **)&B.brick_occ, sizeof(int32_t) * brick_cap);
  A((void **)&B.dirty, sizeof(unsigned long long) * brick_cap);
  A((void **)&B.occ_list, sizeof(int32_t) * occ_cap);
  A((void **)&B.occ_info, sizeof(int4) * occ_cap);
  A((void **)&B.heavy, sizeof(int32_t) * occ_cap);
  A((void **)&B.need, sizeof(unsigned long long) * occ_cap);
  A((void **)&B.worklist, sizeof(int32_t) * occ_cap);
  A((void **)&B.box_start, sizeof(uint32_t) * occ_cap * 64);
  A((void **)&B.box_cnt, sizeof(uint32_t) * occ_cap * 64);
  A((void **)&B.scan_a, sizeof(uint32_t) * scan_n);
  A((void **)&B.scan_b, sizeof(uint32_t) * scan_n);
  make_launch_cfg(s);
  return rc;
}

static int alloc_agents(bdm_sim *s) {
  const long long cap = s->cap;
  const bool f64 = s->P.precision == BDM_FP64;
  const bool grow = s->dp.grow != 0;
  int rc = BDM_OK;
  auto A = [&](void **p, size_t bytes) {
    if (rc == BDM_OK) rc = dmalloc(s, p, bytes, s->allocs_agents);
  };
  for (int t = 0; t < 2; ++t) {
    AgentSet &S = s->sets[t];
    for (int b = 0; b < 2; ++b) {
      A((void **)&S.x[b], sizeof(double) * cap);
      A((void **)&S.y[b], sizeof(double) * cap);
      A((void **)&S.z[b], sizeof(double) * cap);
    }
    A(&S.diam, (f64 ? sizeof(double) : sizeof(float)) * cap);
    if (grow) A((void **)&S.vol, sizeof(double) * cap);
    else S.vol = nullptr;
    A((void **)&S.uid, sizeof(uint64_t) * cap);
    A((void **)&S.beh, cap);
    A((void **)&S.flags, cap);
    A((void **)&S.nz, sizeof(uint16_t) * cap);
  }
  DevBufs &B = s->B;
  A((void **)&s->d_sets, sizeof(AgentSet) * 2);
  A((void **)&s->d_ctr, sizeof(DevCounters));
  A((void **)&s->d_geom, sizeof(SimGeom) * s->n_sims);
  A((void **)&B.sim_off, sizeof(long long) * (s->n_sims + 1));
  A((void **)&B.brick_base, sizeof(long long) * (s->n_sims + 1));
  A((void **)&B.bbox, sizeof(unsigned long long) * 12 * s->n_sims);
  A((void **)&B.key, sizeof(uint32_t) * cap);
  A((void **)&B.arrival, sizeof(uint32_t) * cap);
  A((void **)&B.bucket, sizeof(uint32_t) * cap);
  A((void **)&B.perm, sizeof(uint32_t) * cap);
  A((void **)&B.c32, sizeof(float4) * cap);
  if (f64) A((void **)&B.c64, sizeof(dbl4) * cap);
  else B.c64 = nullptr;
  if (grow) {
    A((void **)&B.stash, sizeof(dbl4) * cap);
  } else {
    B.stash = nullptr;
  }
  if (s->dp.die) {
    A((void **)&B.ghost, sizeof(dbl4) * cap);
  } else {
    B.ghost = nullptr;
  }
  if (!f64) {
    A((void **)&B.fix, sizeof(uint4) * cap);
  } else {
    B.fix = nullptr;
  }
  if (s->dp.n_types > 1) {
    A((void **)&B.tp, cap);
  } else {
    B.tp = nullptr;
  }
  if (s->P.keep_forces) A((void **)&B.fdbg, sizeof(double) * 3 * cap);
  if (rc) return rc;
  B.A = s->d_sets;
  B.A_alt = s->d_sets + 1;
  B.ctr = s->d_ctr;
  B.geom = s->d_geom;
  B.cap = cap;
  return BDM_OK;
}

static int fence_in(bdm_sim *s) {
  CK(cudaEventRecord(s->ev_in, s->user));
  CK(cudaStreamWaitEvent(s->own, s->ev_in, 0));
  return BDM_OK;
}
static int fence_out(bdm_sim *s) {
  CK(cudaEventRecord(s->ev_out, s->own));
  CK(cudaStreamWaitEvent(s->user, s->ev_out, 0));
  return BDM_OK;
}

static int read_counters(bdm_sim *s) {
  CK(cudaMemcpyAsync(s->h_ctr, s->d_ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, s->own));
  CK(cudaStreamSynchronize(s->own));
  return BDM_OK;
}

static int clear_error(bdm_sim *s) {
  CK(cudaMemsetAsync(&s->d_ctr->error, 0, sizeof(int32_t), s->own));
  return BDM_OK;
}

// grid build of the current state (no agent state changes)
static void enqueue_grid(bdm_sim *s) {
  launch_geometry(s->B, s->dp, s->own);
  launch_brick_rank(s->B, s->dp, s->lc, s->own);
  launch_keys(s->B, s->dp, s->lc, s->own);
  launch_brick_scan(s->B, s->dp, s->lc, s->own);
  launch_scatter(s->B, s->dp, s->lc, s->own);
  launch_brick_sort(s->B, s->dp, s->lc, s->own);
}

static void enqueue_step(bdm_sim *s) {
  enqueue_grid(s);
  launch_gather(s->B, s->dp, s->lc, s->own);
  launch_force(s->B, s->dp, s->lc, FM_STEP, s->own);
  launch_force_fix(s->B, s->dp, s->lc, FM_STEP, s->own);
  launch_divide(s->B, s->dp, s->lc, s->own);
  launch_finish(s->B, s->dp, s->own);
}

static int phase_launches(const bdm_sim *s, int p) {
  if (p == PH_DIVIDE) return divide_launches(s->dp);
  if (p == PH_FORCE) return force_launches(s->dp);
  if (p == PH_FORCE_FIX) return force_fix_launches(s->dp);
  return kPhaseLaunches[p];
}

static long long kernels_per_step(const bdm_sim *s) {
  long long k = 0;
  for (int p = 0; p < PH_COUNT; ++p) k += phase_launches(s, p);
  if (s->dp.detect_static) k += 1;  // the static pass before the force kernel
  return k;
}

static int prof_mark(bdm_sim *s, int phase) {
  if (s->prof_used == s->prof_ev.size()) {
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    s->prof_ev.push_back(e);
    s->prof_phase.push_back(-1);
  }
  s->prof_phase[s->prof_used] = phase;
  CK(cudaEventRecord(s->prof_ev[s->prof_used], s->own));
  s->prof_used++;
  return BDM_OK;
}

// one iteration launched kernel by kernel with an event before every phase
static int enqueue_step_profiled(bdm_sim *s) {
  int rc;
  for (int p = 0; p < PH_COUNT; ++p) {
    if (phase_launches(s, p) == 0) continue;
    if ((rc = prof_mark(s, p))) return rc;
    switch (p) {
      case PH_GEOMETRY: launch_geometry(s->B, s->dp, s->own); break;
      case PH_BRICK_RANK: launch_brick_rank(s->B, s->dp, s->lc, s->own); break;
      case PH_KEYS: launch_keys(s->B, s->dp, s->lc, s->own); break;
      case PH_BRICK_SCAN: launch_brick_scan(s->B, s->dp, s->lc, s->own); break;
      case PH_SCATTER: launch_scatter(s->B, s->dp, s->lc, s->own); break;
      case PH_BRICK_SORT: launch_brick_sort(s->B, s->dp, s->lc, s->own); break;
      case PH_GATHER: launch_gather(s->B, s->dp, s->lc, s->own); break;
      case PH_FORCE: launch_force(s->B, s->dp, s->lc, FM_STEP, s->own); break;
      case PH_FORCE_FIX: launch_force_fix(s->B, s->dp, s->lc, FM_STEP, s->own); break;
      case PH_DIVIDE: launch_divide(s->B, s->dp, s->lc, s->own); break;
      default: launch_finish(s->B, s->dp, s->own); break;
    }
    s->prof_launch[p] += phase_launches(s, p);
  }
  if ((rc = prof_mark(s, -1))) return rc;  // end of the iteration
  s->kernels += kernels_per_step(s);
  return BDM_OK;
}

static int capture_step(bdm_sim *s) {
  if (s->graph_ok) return BDM_OK;
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(s->own, cudaStreamCaptureModeThreadLocal));
  enqueue_step(s);
  cudaError_t e = cudaStreamEndCapture(s->own, &g);
  if (e != cudaSuccess) return cuda_fail(s, e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&s->exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return cuda_fail(s, e, "cudaGraphInstantiate");
  s->graph_ok = true;
  return BDM_OK;
}

// Handle the sticky device error after a batch: grow grid buffers (returns
// 1 = retry), or map it to an API error (negative), or 0 = no error.
static int handle_device_error(bdm_sim *s) {
  const DevCounters &h = *s->h_ctr;
  if (h.error == DEV_OK) return 0;
  const int e = h.error;
  int rc = clear_error(s);
  if (rc) return rc;
  if (e == DEV_ECAP_BRICKS || e == DEV_ECAP_OCC) {
    long long nb = s->B.brick_cap, no = s->B.occ_cap;
    if (e == DEV_ECAP_BRICKS) nb = std::max(nb, (long long)(h.need_bricks * 1.25) + 1024);
    if (e == DEV_ECAP_OCC) no = std::max(no, (long long)(h.need_occ * 1.25) + 1024);
    if (nb > (1LL << 26)) return fail(s, BDM_EINVAL, "grid needs more than 2^26 bricks (4x4x4 boxes)");
    rc = alloc_grid(s, nb, no);
    if (rc) return rc;
    return 1;
  }
  if (e == DEV_ECAP_AGENTS) return fail(s, BDM_ECAPACITY, "daughters would exceed the agent capacity");
  if (e == DEV_ERANGE) return fail(s, BDM_EINVAL, "a simulation spans more than 2^21 boxes along an axis");
  if (e == DEV_EBOX) return fail(s, BDM_EINVAL, "more than 65536 agents in one box");
  if (e == DEV_ECHECK)
    return fail(s, BDM_ECUDA, "device bounds check failed (source line " + std::to_string(h.check_line) + ")");
  return fail(s, BDM_EINVAL, "device error " + std::to_string(e));
}

// run the grid build (debug / sort) with capacity growth
static int run_grid(bdm_sim *s, bool gather) {
  for (int attempt = 0; attempt < 8; ++attempt) {
    enqueue_grid(s);
    if (gather) launch_gather(s->B, s->dp, s->lc, s->own);
    int rc = read_counters(s);
    if (rc) return rc;
    rc = handle_device_error(s);
    if (rc == 0) return BDM_OK;
    if (rc < 0) return rc;
    if (gather) {
      int one = 1;
      CK(cudaMemcpyAsync(&s->d_ctr->force_sort, &one, sizeof(int), cudaMemcpyHostToDevice, s->own));
      CK(cudaStreamSynchronize(s->own));
    }
  }
  return fail(s, BDM_ENOMEM, "grid capacity did not converge");
}

static int ensure_dbg_scratch(bdm_sim *s, size_t bytes) {
  if (s->dbg_scratch_bytes >= bytes) return BDM_OK;
  if (s->dbg_scratch) cudaFree(s->dbg_scratch);
  s->dbg_scratch = nullptr;
  s->dbg_scratch_bytes = 0;
  cudaError_t e = cudaMalloc(&s->dbg_scratch, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(s, BDM_ENOMEM, "debug scratch allocation failed");
  }
  s->dbg_scratch_bytes = bytes;
  return BDM_OK;
}

static int current_set(bdm_sim *s, AgentSet *out) {
  CK(cudaMemcpyAsync(out, s->d_sets, sizeof(AgentSet), cudaMemcpyDeviceToHost, s->own));
  CK(cudaStreamSynchronize(s->own));
  return BDM_OK;
}

// ------------------------------------------------------------------ C ABI
extern "C" {

int bdm_version(void) { return BDM_ABI_VERSION; }

const char *bdm_last_error(const bdm_sim *sim) {
  return sim ? sim->err.c_str() : g_create_error.c_str();
}

int bdm_create(const bdm_params *params, void *stream, bdm_sim **out) {
  if (!params || !out) return fail(nullptr, BDM_EINVAL, "NULL params or out");
  *out = nullptr;
  const bdm_params &P = *params;
  const double L = P.box_edge > 0.0 ? P.box_edge : P.interaction_radius;
  if (!(P.interaction_radius > 0.0) || !std::isfinite(P.interaction_radius))
    return fail(nullptr, BDM_EINVAL, "interaction_radius must be positive and finite");
  if (!(L >= P.interaction_radius) || !std::isfinite(L)) return fail(nullptr, BDM_EINVAL, "box_edge must be >= R");
  if (P.n_sims < 1) return fail(nullptr, BDM_EINVAL, "n_sims must be >= 1");
  if (P.capacity < 1 || P.capacity > (1LL << 31) - 1)
    return fail(nullptr, BDM_EINVAL, "capacity must be in [1, 2^31)");
  if (P.precision != BDM_FP64 && P.precision != BDM_FP32_FORCE) return fail(nullptr, BDM_EINVAL, "unknown precision");
  if (P.growth_per_step > 0.0 && (P.n_sims > 1 || P.precision != BDM_FP64))
    return fail(nullptr, BDM_EINVAL, "growth and division need n_sims == 1 and BDM_FP64");
  if (P.growth_per_step > 0.0 && !(P.ratio_hi >= P.ratio_lo && P.ratio_lo > 0.0 && P.divide_volume > 0.0))
    return fail(nullptr, BDM_EINVAL, "division needs 0 < ratio_lo <= ratio_hi and divide_volume > 0");
  if (!(P.dt >= 0.0) || !(P.max_displacement >= 0.0) || !(P.adherence >= 0.0) || !(P.walk_step >= 0.0))
    return fail(nullptr, BDM_EINVAL, "dt, max_displacement, adherence and walk_step must be >= 0");
  if (P.sort_every < 0) return fail(nullptr, BDM_EINVAL, "sort_every must be >= 0");
  if (!(P.death_prob >= 0.0 && P.death_prob <= 1.0)) return fail(nullptr, BDM_EINVAL, "death_prob must be in [0, 1]");
  if (P.death_prob > 0.0 && P.n_sims > 1) return fail(nullptr, BDM_EINVAL, "removal needs n_sims == 1");
  if (P.n_types < 0 || P.n_types > 4) return fail(nullptr, BDM_EINVAL, "n_types must be in [0, 4]");
  if (P.curve != BDM_CURVE_MORTON && P.curve != BDM_CURVE_HILBERT)
    return fail(nullptr, BDM_EINVAL, "curve must be BDM_CURVE_MORTON or BDM_CURVE_HILBERT");
  for (int a = 0; a < P.n_types && P.n_types > 1; ++a)
    for (int b = 0; b < P.n_types; ++b) {
      const double k = P.type_k[4 * a + b], g = P.type_gamma[4 * a + b];
      if (!(std::isfinite(k) && std::isfinite(g) && k >= 0.0 && g >= 0.0))
        return fail(nullptr, BDM_EINVAL, "type_k and type_gamma must be finite and >= 0");
      if (k != P.type_k[4 * b + a] || g != P.type_gamma[4 * b + a])
        return fail(nullptr, BDM_EINVAL, "type_k and type_gamma must be symmetric");
    }

  bdm_sim *s = new bdm_sim();
  s->P = P;
  s->dp = make_dev_params(P);
  s->user = (cudaStream_t)stream;
  s->cap = P.capacity;
  s->n_sims = P.n_sims;
  s->dt_sim.assign(P.n_sims, P.dt);
  if (P.dt_per_sim)
    for (int i = 0; i < P.n_sims; ++i) s->dt_sim[i] = P.dt_per_sim[i];
  int dev = 0;
  int rc = BDM_OK;
  auto bail = [&](int code) {
    g_create_error = s->err;
    bdm_destroy(s);
    return code;
  };
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&s->sm_count, cudaDevAttrMultiProcessorCount, dev) !=
                                                cudaSuccess) {
    cudaGetLastError();
    s->err = "no CUDA device";
    return bail(BDM_ECUDA);
  }
  if (cudaStreamCreateWithFlags(&s->own, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&s->aux, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->ev_out, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->ev_a, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&s->ev_b, cudaEventDisableTiming) != cudaSuccess ||
      cudaMallocHost((void **)&s->h_ctr, sizeof(DevCounters)) != cudaSuccess) {
    cudaGetLastError();
    s->err = "stream/event/pinned allocation failed";
    return bail(BDM_ECUDA);
  }
  rc = alloc_agents(s);
  if (rc) return bail(rc);
  rc = alloc_grid(s, 1 << 16, std::max<long long>(1024, s->cap / 16));
  if (rc) return bail(rc);
  // device-side constant state
  if (cudaMemcpy(s->d_sets, s->sets, sizeof(AgentSet) * 2, cudaMemcpyHostToDevice) != cudaSuccess) {
    s->err = "copy of agent sets failed";
    return bail(BDM_ECUDA);
  }
  std::vector<SimGeom> geo(s->n_sims);
  std::memset(geo.data(), 0, sizeof(SimGeom) * s->n_sims);
  for (int i = 0; i < s->n_sims; ++i) {
    geo[i].dt = s->dt_sim[i];
    geo[i].dt_f = (float)s->dt_sim[i];
  }
  DevCounters z{};
  if (cudaMemcpy(s->d_geom, geo.data(), sizeof(SimGeom) * s->n_sims, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(s->d_ctr, &z, sizeof(DevCounters), cudaMemcpyHostToDevice) != cudaSuccess) {
    s->err = "initial copies failed";
    return bail(BDM_ECUDA);
  }
  *out = s;
  return BDM_OK;
}

void bdm_destroy(bdm_sim *s) {
  if (!s) return;
  if (s->own) cudaStreamSynchronize(s->own);
  if (s->exec) cudaGraphExecDestroy(s->exec);
  free_list(s->allocs_grid);
  free_list(s->allocs_agents);
  if (s->dbg_scratch) cudaFree(s->dbg_scratch);
  if (s->B.nbr_count) cudaFree(s->B.nbr_count);
  if (s->B.nbr_off) cudaFree(s->B.nbr_off);
  if (s->B.nbr_out) cudaFree(s->B.nbr_out);
  if (s->B.dbg_i32) cudaFree(s->B.dbg_i32);
  if (!s->P.keep_forces && s->B.fdbg) cudaFree(s->B.fdbg);
  for (cudaEvent_t e : s->prof_ev) cudaEventDestroy(e);
  if (s->h_ctr) cudaFreeHost(s->h_ctr);
  if (s->ev_in) cudaEventDestroy(s->ev_in);
  if (s->ev_out) cudaEventDestroy(s->ev_out);
  if (s->ev_a) cudaEventDestroy(s->ev_a);
  if (s->ev_b) cudaEventDestroy(s->ev_b);
  if (s->aux) cudaStreamDestroy(s->aux);
  if (s->own) cudaStreamDestroy(s->own);
  delete s;
}

int bdm_set_stream(bdm_sim *s, void *stream) {
  if (!s) return BDM_EINVAL;
  s->user = (cudaStream_t)stream;
  return BDM_OK;
}

int bdm_set_agents(bdm_sim *s, int64_t n, const double *xyz, const double *diam, const double *vol,
                   const uint64_t *uid, const uint8_t *behavior, const int64_t *sim_offsets, int64_t step,
                   uint64_t next_uid, int mem) {
  if (!s) return BDM_EINVAL;
  if (n < 0) return fail(s, BDM_EINVAL, "n must be >= 0");
  if (n > s->cap) return fail(s, BDM_ECAPACITY, "n exceeds capacity");
  if (n > 0 && (!xyz || !diam)) return fail(s, BDM_EINVAL, "xyz and diam are required");
  if (mem != BDM_HOST && mem != BDM_DEVICE) return fail(s, BDM_EINVAL, "mem must be BDM_HOST or BDM_DEVICE");
  if (step < 0) return fail(s, BDM_EINVAL, "step must be >= 0");
  const cudaMemcpyKind kind = (mem == BDM_HOST) ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  int rc = fence_in(s);
  if (rc) return rc;
  // simulation offsets
  std::vector<long long> off(s->n_sims + 1, 0);
  if (s->n_sims == 1) {
    off[1] = n;
  } else {
    if (!sim_offsets) return fail(s, BDM_EINVAL, "sim_offsets required when n_sims > 1");
    if (mem == BDM_HOST) {
      for (int i = 0; i <= s->n_sims; ++i) off[i] = sim_offsets[i];
    } else {
      CK(cudaMemcpyAsync(off.data(), sim_offsets, sizeof(long long) * (s->n_sims + 1), cudaMemcpyDeviceToHost, s->own));
      CK(cudaStreamSynchronize(s->own));
    }
    if (off[0] != 0 || off[s->n_sims] != n) return fail(s, BDM_EINVAL, "sim_offsets must start at 0 and end at n");
    for (int i = 0; i < s->n_sims; ++i)
      if (off[i + 1] < off[i]) return fail(s, BDM_EINVAL, "sim_offsets must be non-decreasing");
  }
  // the current set becomes set 0 again
  CK(cudaMemcpyAsync(s->d_sets, s->sets, sizeof(AgentSet) * 2, cudaMemcpyHostToDevice, s->own));
  const AgentSet &A = s->sets[0];
  const AgentSet &T = s->sets[1];  // staging
  if (n > 0) {
    // P_t into both position buffers (no movement history yet), checked on
    // the way (finite positions within +-1e9 um, then finite positive
    // diameters in the init kernel); a failure leaves no agents set.  From
    // host memory the positions cross the link first, and their second copy
    // and check run on the auxiliary stream while the diameters cross.
    int *bad = (int *)s->B.scan_b;  // scratch
    CK(cudaMemsetAsync(bad, 0, sizeof(int), s->own));
    if (mem == BDM_HOST) {
      CK(cudaMemcpyAsync(A.x[0], xyz, sizeof(double) * n, kind, s->own));
      CK(cudaMemcpyAsync(A.y[0], xyz + n, sizeof(double) * n, kind, s->own));
      CK(cudaMemcpyAsync(A.z[0], xyz + 2 * n, sizeof(double) * n, kind, s->own));
      CK(cudaEventRecord(s->ev_a, s->own));
      CK(cudaStreamWaitEvent(s->aux, s->ev_a, 0));
      launch_positions_in(A.x[0], A.y[0], A.z[0], A, n, bad, s->lc, s->aux);
      CK(cudaEventRecord(s->ev_b, s->aux));
    } else {
      launch_positions_in(xyz, xyz + n, xyz + 2 * n, A, n, bad, s->lc, s->own);
    }
    const double *d_diam = diam;
    const double *d_vol = nullptr;
    const uint64_t *d_uid = nullptr;
    const uint8_t *d_beh = nullptr;
    if (mem == BDM_HOST) {
      CK(cudaMemcpyAsync(T.x[0], diam, sizeof(double) * n, kind, s->own));
      d_diam = T.x[0];
      if (vol) { CK(cudaMemcpyAsync(T.x[1], vol, sizeof(double) * n, kind, s->own)); d_vol = T.x[1]; }
      if (uid) { CK(cudaMemcpyAsync(T.y[0], uid, sizeof(uint64_t) * n, kind, s->own)); d_uid = (const uint64_t *)T.y[0]; }
      if (behavior) { CK(cudaMemcpyAsync(T.beh, behavior, n, kind, s->own)); d_beh = T.beh; }
    } else {
      d_vol = vol;
      d_uid = uid;
      d_beh = behavior;
    }
    launch_init_agents(s->B, s->dp, s->lc, d_diam, d_vol, d_uid, d_beh, n, bad, s->own);
    if (mem == BDM_HOST) CK(cudaStreamWaitEvent(s->own, s->ev_b, 0));
    int hb = 0;
    CK(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, s->own));
    CK(cudaStreamSynchronize(s->own));
    s->kernels += 2;
    if (hb) {
      s->have_agents = false;
      return fail(s, BDM_EINVAL, "non-finite or out-of-range position or diameter (no agents are set)");
    }
  }
  // offsets, counters, bounding box
  std::vector<long long> base(s->n_sims + 1, 0);
  CK(cudaMemcpyAsync(s->B.sim_off, off.data(), sizeof(long long) * (s->n_sims + 1), cudaMemcpyHostToDevice, s->own));
  DevCounters z{};
  z.n = n;
  z.step = step;
  z.next_uid = next_uid;
  *s->h_ctr = z;
  CK(cudaMemcpyAsync(s->d_ctr, s->h_ctr, sizeof(DevCounters), cudaMemcpyHostToDevice, s->own));
  launch_bbox(s->B, s->dp, s->lc, s->own);
  s->kernels += 2;
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s->own));
  s->sim_off = off;
  s->have_agents = true;
  return fence_out(s);
}

int bdm_step(bdm_sim *s, int n_steps) {
  if (!s) return BDM_EINVAL;
  if (n_steps < 0) return fail(s, BDM_EINVAL, "n_steps must be >= 0");
  if (!s->have_agents) return fail(s, BDM_ESTATE, "bdm_set_agents must come first");
  int rc = fence_in(s);
  if (rc) return rc;
  rc = read_counters(s);
  if (rc) return rc;
  const long long target = s->h_ctr->step + n_steps;
  for (int guard = 0; guard < 64 && s->h_ctr->step < target; ++guard) {
    rc = capture_step(s);
    if (rc) return rc;
    const long long todo = target - s->h_ctr->step;
    if (s->prof_on) {
      for (long long t = 0; t < todo; ++t)
        if ((rc = enqueue_step_profiled(s))) return rc;
    } else {
      for (long long t = 0; t < todo; ++t) CK(cudaGraphLaunch(s->exec, s->own));
      s->kernels += todo * kernels_per_step(s);
    }
    rc = read_counters(s);
    if (rc) return rc;
    rc = handle_device_error(s);
    if (rc < 0) return rc;
    rc = read_counters(s);
    if (rc) return rc;
  }
  if (s->h_ctr->step < target) return fail(s, BDM_ENOMEM, "grid capacity did not converge");
  return fence_out(s);
}

int bdm_sort(bdm_sim *s) {
  if (!s) return BDM_EINVAL;
  if (!s->have_agents) return fail(s, BDM_ESTATE, "bdm_set_agents must come first");
  int rc = fence_in(s);
  if (rc) return rc;
  int one = 1;
  CK(cudaMemcpyAsync(&s->d_ctr->force_sort, &one, sizeof(int), cudaMemcpyHostToDevice, s->own));
  rc = run_grid(s, true);
  if (rc) return rc;
  return fence_out(s);
}

int bdm_get_agents(bdm_sim *s, int64_t cap, double *xyz, double *diam, double *vol, uint64_t *uid,
                   uint8_t *behavior, int64_t *sim_offsets, int64_t *n_out, int64_t *step, uint64_t *next_uid,
                   int mem) {
  if (!s) return BDM_EINVAL;
  if (mem != BDM_HOST && mem != BDM_DEVICE) return fail(s, BDM_EINVAL, "mem must be BDM_HOST or BDM_DEVICE");
  int rc = fence_in(s);
  if (rc) return rc;
  rc = read_counters(s);
  if (rc) return rc;
  const long long n = s->h_ctr->n;
  if (n_out) *n_out = n;
  if (step) *step = s->h_ctr->step;
  if (next_uid) *next_uid = s->h_ctr->next_uid;
  if (cap < n && (xyz || diam || vol || uid || behavior)) return fail(s, BDM_ECAPACITY, "output capacity < n");
  const cudaMemcpyKind kind = (mem == BDM_HOST) ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  AgentSet A, T;
  rc = current_set(s, &A);
  if (rc) return rc;
  CK(cudaMemcpyAsync(&T, s->d_sets + 1, sizeof(AgentSet), cudaMemcpyDeviceToHost, s->own));
  CK(cudaStreamSynchronize(s->own));
  const int cur = (int)(s->h_ctr->step & 1);
  if (n > 0) {
    if (xyz) {
      CK(cudaMemcpyAsync(xyz, A.x[cur], sizeof(double) * n, kind, s->own));
      CK(cudaMemcpyAsync(xyz + cap, A.y[cur], sizeof(double) * n, kind, s->own));
      CK(cudaMemcpyAsync(xyz + 2 * cap, A.z[cur], sizeof(double) * n, kind, s->own));
    }
    if (diam) {
      if (s->P.precision == BDM_FP64) {
        CK(cudaMemcpyAsync(diam, A.diam, sizeof(double) * n, kind, s->own));
      } else {
        launch_diam_to_f64(s->B, s->dp, s->lc, T.x[0], s->own);
        CK(cudaMemcpyAsync(diam, T.x[0], sizeof(double) * n, kind, s->own));
      }
    }
    if (vol) {
      if (A.vol) {
        CK(cudaMemcpyAsync(vol, A.vol, sizeof(double) * n, kind, s->own));
      } else if (mem == BDM_HOST) {
        // pi/6 d^3 from the stored diameter
        std::vector<double> d(n);
        if (s->P.precision == BDM_FP64) {
          CK(cudaMemcpyAsync(d.data(), A.diam, sizeof(double) * n, cudaMemcpyDeviceToHost, s->own));
        } else {
          launch_diam_to_f64(s->B, s->dp, s->lc, T.x[0], s->own);
          CK(cudaMemcpyAsync(d.data(), T.x[0], sizeof(double) * n, cudaMemcpyDeviceToHost, s->own));
        }
        CK(cudaStreamSynchronize(s->own));
        const double c = 3.141592653589793 / 6.0;
        for (long long i = 0; i < n; ++i) vol[i] = ((c * d[i]) * d[i]) * d[i];
      } else {
        return fail(s, BDM_EINVAL, "volume is not stored without growth; request it into host memory");
      }
    }
    if (uid) CK(cudaMemcpyAsync(uid, A.uid, sizeof(uint64_t) * n, kind, s->own));
    if (behavior) CK(cudaMemcpyAsync(behavior, A.beh, n, kind, s->own));
  }
  CK(cudaStreamSynchronize(s->own));
  if (sim_offsets) {
    std::vector<long long> off = s->sim_off;
    if (s->n_sims == 1) off = {0, n};
    if (mem == BDM_HOST) std::memcpy(sim_offsets, off.data(), sizeof(long long) * (s->n_sims + 1));
    else CK(cudaMemcpy(sim_offsets, off.data(), sizeof(long long) * (s->n_sims + 1), cudaMemcpyHostToDevice));
  }
  return fence_out(s);
}

int bdm_get_counters(bdm_sim *s, bdm_counters *out) {
  if (!s || !out) return BDM_EINVAL;
  int rc = read_counters(s);
  if (rc) return rc;
  const DevCounters &h = *s->h_ctr;
  out->n_agents = h.n;
  out->step = h.step;
  out->next_uid = h.next_uid;
  out->n_static = (int64_t)h.l_static;
  out->n_moved = (int64_t)h.l_moved;
  out->n_divided = (int64_t)h.l_div;
  out->n_removed = (int64_t)h.l_rm;
  out->n_fp64_fixup = (int64_t)h.l_fix;
  out->n_candidates = (int64_t)h.l_cand;
  out->n_neighbors = (int64_t)h.l_nbr;
  out->n_contacts = (int64_t)h.l_contact;
  out->n_exact_fallback = (int64_t)h.l_exact;
  out->n_boxes = h.l_boxes;
  out->n_bricks = h.l_bricks;
  out->n_occupied_bricks = h.l_occ;
  out->max_brick_agents = h.l_max_brick;
  out->kernels_launched = s->kernels;
  out->history_valid = h.history_valid;
  out->error = h.error;
  return BDM_OK;
}

static int apply_params(bdm_sim *s, const bdm_params &P, int lanes) {
  s->P = P;
  DevParams d = make_dev_params(P);
  d.lanes_fixed = lanes;
  s->dp = d;
  if (s->graph_ok) {
    cudaGraphExecDestroy(s->exec);
    s->exec = nullptr;
    s->graph_ok = false;
  }
  return BDM_OK;
}

int bdm_set_force_kernel(bdm_sim *s, int lanes) {
  if (!s) return BDM_EINVAL;
  if (!(lanes == FORCE_HYBRID || lanes == FORCE_SPARSE || lanes == -1 || lanes == FORCE_TILE || lanes == 1 ||
        lanes == 2 || lanes == 4 || lanes == 8 || lanes == 16 || lanes == 32))
    return fail(s, BDM_EINVAL, "lanes must be -4, -3, -1, 0, 1, 2, 4, 8, 16 or 32");
  return apply_params(s, s->P, lanes);
}

int bdm_autotune(bdm_sim *s, int trial_steps, int what, bdm_tuning *out) {
  if (!s || trial_steps < 1) return s ? fail(s, BDM_EINVAL, "trial_steps must be >= 1") : BDM_EINVAL;
  if (!s->have_agents) return fail(s, BDM_ESTATE, "bdm_set_agents must come first");
  int rc = read_counters(s);
  if (rc) return rc;
  const long long n = s->h_ctr->n;
  const int64_t step0 = s->h_ctr->step;
  const uint64_t uid0 = s->h_ctr->next_uid;
  // snapshot of the state in the layout bdm_set_agents takes
  const size_t per = 8 * 3 + 8 + 8 + 8 + 1;
  void *snap = nullptr;
  if (cudaMalloc(&snap, per * (size_t)std::max<long long>(n, 1) + 256) != cudaSuccess) {
    cudaGetLastError();
    return fail(s, BDM_ENOMEM, "autotune snapshot allocation failed");
  }
  double *xyz = (double *)snap;
  double *dia = xyz + 3 * n;
  double *vol = dia + n;
  uint64_t *uid = (uint64_t *)(vol + n);
  uint8_t *beh = (uint8_t *)(uid + n);
  const bool have_vol = s->sets[0].vol != nullptr;
  int64_t nn = 0, st = 0;
  uint64_t nu = 0;
  rc = bdm_get_agents(s, n, xyz, dia, have_vol ? vol : nullptr, uid, beh, nullptr, &nn, &st, &nu, BDM_DEVICE);
  std::vector<int64_t> off_h(s->sim_off.begin(), s->sim_off.end());
  if (s->n_sims == 1) off_h = {0, (int64_t)n};
  // bdm_set_agents with BDM_DEVICE reads sim_offsets from device memory
  long long *d_off = nullptr;
  if (rc == BDM_OK && s->n_sims > 1) {
    if (cudaMalloc(&d_off, sizeof(long long) * (s->n_sims + 1)) != cudaSuccess ||
        cudaMemcpy(d_off, off_h.data(), sizeof(long long) * (s->n_sims + 1), cudaMemcpyHostToDevice) != cudaSuccess) {
      cudaGetLastError();
      rc = fail(s, BDM_ENOMEM, "autotune offsets allocation failed");
    }
  }
  auto restore_dev = [&]() {
    return bdm_set_agents(s, n, xyz, dia, have_vol ? vol : nullptr, uid, beh, (const int64_t *)d_off, step0, uid0,
                          BDM_DEVICE);
  };
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (rc == BDM_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) {
    cudaGetLastError();
    rc = fail(s, BDM_ECUDA, "autotune events");
  }
  const bdm_params base = s->P;
  const double R = base.interaction_radius;
  bdm_params best = base;
  int best_lanes = s->dp.lanes_fixed;
  double best_ms = 1e300;
  int trials = 0;
  auto trial = [&](const bdm_params &P, int lanes, double *ms) -> int {
    int r = apply_params(s, P, lanes);
    if (r) return r;
    if ((r = restore_dev())) return r;
    if ((r = bdm_step(s, 1))) return r;
    CK(cudaEventRecord(e0, s->own));
    if ((r = bdm_step(s, trial_steps))) return r;
    CK(cudaEventRecord(e1, s->own));
    CK(cudaEventSynchronize(e1));
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, e0, e1));
    *ms = t / trial_steps;
    trials++;
    return BDM_OK;
  };
  if (rc == BDM_OK) {
    double ms = 0;
    rc = trial(best, best_lanes, &best_ms);
    if (rc == BDM_OK && (what & BDM_TUNE_BOX_EDGE)) {
      const double f[4] = {1.0, 1.125, 1.25, 1.5};
      bdm_params b = best;
      for (int i = 0; i < 4 && rc == BDM_OK; ++i) {
        bdm_params P = b;
        P.box_edge = R * f[i];
        if ((rc = trial(P, best_lanes, &ms)) == BDM_OK && ms < best_ms) { best_ms = ms; best = P; }
      }
    }
    if (rc == BDM_OK && (what & BDM_TUNE_LANES) && base.precision == BDM_FP32_FORCE) {
      const int opts[4] = {FORCE_LANES_DEFAULT, 4, FORCE_SPARSE, FORCE_TILE};
      int bl = best_lanes;
      for (int i = 0; i < 4 && rc == BDM_OK; ++i)
        if ((rc = trial(best, opts[i], &ms)) == BDM_OK && ms < best_ms) { best_ms = ms; bl = opts[i]; }
      best_lanes = bl;
    }
    if (rc == BDM_OK && (what & BDM_TUNE_SORT)) {
      const int opts[4] = {0, 5, 10, 20};
      bdm_params b = best;
      for (int i = 0; i < 4 && rc == BDM_OK; ++i) {
        bdm_params P = b;
        P.sort_every = opts[i];
        if ((rc = trial(P, best_lanes, &ms)) == BDM_OK && ms < best_ms) { best_ms = ms; best = P; }
      }
    }
  }
  // keep the best setting and the original state
  int rc2 = apply_params(s, best, best_lanes);
  if (rc2 == BDM_OK) rc2 = restore_dev();
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (d_off) cudaFree(d_off);
  cudaFree(snap);
  if (rc) return rc;
  if (rc2) return rc2;
  if (out) {
    out->box_edge = best.box_edge > 0.0 ? best.box_edge : R;
    out->ms_per_step = best_ms;
    out->lanes = best_lanes;
    out->sort_every = best.sort_every;
    out->n_trials = trials;
    out->reserved = 0;
  }
  return BDM_OK;
}

int bdm_profile_begin(bdm_sim *s) {
  if (!s) return BDM_EINVAL;
  s->prof_on = true;
  s->prof_used = 0;
  for (int p = 0; p < PH_COUNT; ++p) { s->prof_ms[p] = 0.0; s->prof_launch[p] = 0; }
  return BDM_OK;
}

int bdm_profile_end(bdm_sim *s, double *ms, int64_t *launches, int cap, int *n_phases) {
  if (!s) return BDM_EINVAL;
  if (n_phases) *n_phases = PH_COUNT;
  CK(cudaStreamSynchronize(s->own));
  for (size_t i = 0; i + 1 < s->prof_used; ++i) {
    const int p = s->prof_phase[i];
    if (p < 0) continue;
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, s->prof_ev[i], s->prof_ev[i + 1]));
    s->prof_ms[p] += t;
  }
  for (int p = 0; p < PH_COUNT && p < cap; ++p) {
    if (ms) ms[p] = s->prof_ms[p];
    if (launches) launches[p] = s->prof_launch[p];
  }
  s->prof_on = false;
  s->prof_used = 0;
  return BDM_OK;
}

const char *bdm_phase_name(int phase) {
  return (phase >= 0 && phase < PH_COUNT) ? kPhaseNames[phase] : "";
}

int bdm_get_debug(bdm_sim *s, int what, void *out, int64_t cap, int64_t *n_out) {
  if (!s) return BDM_EINVAL;
  if (!s->have_agents) return fail(s, BDM_ESTATE, "bdm_set_agents must come first");
  int rc = fence_in(s);
  if (rc) return rc;
  rc = read_counters(s);
  if (rc) return rc;
  const long long n = s->h_ctr->n;
  AgentSet A;
  rc = current_set(s, &A);
  if (rc) return rc;
  auto need = [&](long long m) -> int {
    if (n_out) *n_out = m;
    if (cap < m || (m > 0 && !out)) return fail(s, BDM_ECAPACITY, "debug output capacity too small");
    return BDM_OK;
  };
  switch (what) {
    case BDM_DBG_FORCES: {
      if (!s->P.keep_forces) return fail(s, BDM_EINVAL, "BDM_DBG_FORCES needs keep_forces");
      if ((rc = need(3 * n))) return rc;
      for (int d = 0; d < 3; ++d)
        CK(cudaMemcpyAsync((double *)out + d * n, s->B.fdbg + d * s->cap, sizeof(double) * n, cudaMemcpyDeviceToHost,
                           s->own));
      break;
    }
    case BDM_DBG_NZ: {
      if ((rc = need(n))) return rc;
      std::vector<uint16_t> v(n);
      CK(cudaMemcpyAsync(v.data(), A.nz, sizeof(uint16_t) * n, cudaMemcpyDeviceToHost, s->own));
      CK(cudaStreamSynchronize(s->own));
      for (long long i = 0; i < n; ++i) ((int32_t *)out)[i] = v[i];
      break;
    }
    case BDM_DBG_STATIC: {
      if ((rc = need(n))) return rc;
      CK(cudaMemcpyAsync(out, A.flags, n, cudaMemcpyDeviceToHost, s->own));
      CK(cudaStreamSynchronize(s->own));
      for (long long i = 0; i < n; ++i) ((uint8_t *)out)[i] = (((uint8_t *)out)[i] & FL_STATIC) ? 1 : 0;
      break;
    }
    case BDM_DBG_GRID_BOX:
    case BDM_DBG_GRID_ORDER:
    case BDM_DBG_GRID_GEOMETRY:
    case BDM_DBG_BRICK_RANK: {
      const long long m = (what == BDM_DBG_GRID_BOX) ? 3 * n : (what == BDM_DBG_GRID_GEOMETRY ? 6LL * s->n_sims : n);
      if ((rc = need(m))) return rc;
      rc = run_grid(s, false);
      if (rc) return rc;
      if (what == BDM_DBG_GRID_ORDER) {
        std::vector<uint32_t> v(n);
        CK(cudaMemcpyAsync(v.data(), s->B.perm, sizeof(uint32_t) * n, cudaMemcpyDeviceToHost, s->own));
        CK(cudaStreamSynchronize(s->own));
        for (long long i = 0; i < n; ++i) ((int64_t *)out)[i] = v[i];
      } else if (what == BDM_DBG_GRID_GEOMETRY) {
        std::vector<SimGeom> g(s->n_sims);
        CK(cudaMemcpyAsync(g.data(), s->d_geom, sizeof(SimGeom) * s->n_sims, cudaMemcpyDeviceToHost, s->own));
        CK(cudaStreamSynchronize(s->own));
        for (int i = 0; i < s->n_sims; ++i)
          for (int d = 0; d < 3; ++d) {
            ((double *)out)[6 * i + d] = g[i].lo[d];
            ((double *)out)[6 * i + 3 + d] = (double)g[i].nb[d];
          }
      } else {
        if ((rc = ensure_dbg_scratch(s, (size_t)n * 20 + 64))) return rc;
        int32_t *box = (int32_t *)s->dbg_scratch;
        long long *rk = (long long *)((char *)s->dbg_scratch + ((size_t)n * 12 + 15) / 16 * 16);
        launch_debug_boxes(s->B, s->dp, s->lc, box, rk, s->own);
        if (what == BDM_DBG_GRID_BOX)
          CK(cudaMemcpyAsync(out, box, sizeof(int32_t) * 3 * n, cudaMemcpyDeviceToHost, s->own));
        else
          CK(cudaMemcpyAsync(out, rk, sizeof(long long) * n, cudaMemcpyDeviceToHost, s->own));
      }
      break;
    }
    case BDM_DBG_NEIGHBORS: {
      rc = run_grid(s, false);
      if (rc) return rc;
      if (!s->B.nbr_count) {
        if (cudaMalloc(&s->B.nbr_count, sizeof(int32_t) * s->cap) != cudaSuccess ||
            cudaMalloc(&s->B.nbr_off, sizeof(long long) * (s->cap + 1)) != cudaSuccess) {
          cudaGetLastError();
          return fail(s, BDM_ENOMEM, "neighbour count allocation failed");
        }
      }
      launch_force(s->B, s->dp, s->lc, FM_COUNT_NBR, s->own);
      launch_nbr_offsets(s->B, s->dp, s->own);
      long long total = 0;
      CK(cudaMemcpyAsync(&total, s->B.nbr_off + n, sizeof(long long), cudaMemcpyDeviceToHost, s->own));
      CK(cudaStreamSynchronize(s->own));
      if ((rc = need(n + 1 + total))) return rc;
      if (s->B.nbr_cap < total) {
        if (s->B.nbr_out) cudaFree(s->B.nbr_out);
        s->B.nbr_out = nullptr;
        if (cudaMalloc(&s->B.nbr_out, sizeof(long long) * (total + 1)) != cudaSuccess) {
          cudaGetLastError();
          s->B.nbr_cap = 0;
          return fail(s, BDM_ENOMEM, "neighbour list allocation failed");
        }
        s->B.nbr_cap = total;
      }
      launch_force(s->B, s->dp, s->lc, FM_LIST_NBR, s->own);
      CK(cudaMemcpyAsync(out, s->B.nbr_off, sizeof(long long) * (n + 1), cudaMemcpyDeviceToHost, s->own));
      CK(cudaMemcpyAsync((long long *)out + n + 1, s->B.nbr_out, sizeof(long long) * total, cudaMemcpyDeviceToHost,
                         s->own));
      break;
    }
    case BDM_DBG_FORCES_NOW: {
      if ((rc = need(3 * n + n))) return rc;  // counted in doubles: 3n doubles + 2n int32
      rc = run_grid(s, false);
      if (rc) return rc;
      if (!s->B.fdbg) {
        if (cudaMalloc(&s->B.fdbg, sizeof(double) * 3 * s->cap) != cudaSuccess) {
          cudaGetLastError();
          return fail(s, BDM_ENOMEM, "force buffer allocation failed");
        }
      }
      if (!s->B.dbg_i32) {
        if (cudaMalloc(&s->B.dbg_i32, sizeof(int32_t) * 2 * s->cap) != cudaSuccess) {
          cudaGetLastError();
          return fail(s, BDM_ENOMEM, "debug buffer allocation failed");
        }
      }
      launch_force(s->B, s->dp, s->lc, FM_FORCES, s->own);
      for (int d = 0; d < 3; ++d)
        CK(cudaMemcpyAsync((double *)out + d * n, s->B.fdbg + d * s->cap, sizeof(double) * n, cudaMemcpyDeviceToHost,
                           s->own));
      int32_t *ip = (int32_t *)((double *)out + 3 * n);
      CK(cudaMemcpyAsync(ip, s->B.dbg_i32, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s->own));
      CK(cudaMemcpyAsync(ip + n, s->B.dbg_i32 + s->cap, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, s->own));
      break;
    }
    default:
      return fail(s, BDM_EINVAL, "unknown debug selector");
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s->own));
  rc = read_counters(s);
  if (rc) return rc;
  if (s->h_ctr->error) {
    rc = handle_device_error(s);
    if (rc < 0) return rc;
  }
  return fence_out(s);
}

}  // extern "C"
