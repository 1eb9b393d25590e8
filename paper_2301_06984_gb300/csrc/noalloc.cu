// noalloc.cu -- an entry point that allocates no memory.
//
// bdm_forces_noalloc() evaluates the summed overlap force of every agent of
// one simulation (FP64 form, the same kernels as bdm_get_debug's
// BDM_DBG_FORCES_NOW) for callers that cannot call cudaMalloc: host
// applications whose own allocator owns all device memory (a cudaMalloc
// behind its back would break its accounting or fail against its pool), and
// plug-ins or embedded solvers that their host forbids to allocate.  The
// caller passes device inputs and outputs; every intermediate (grid tables,
// sorted records, counters) lives in one file-scope device array of fixed
// size, which every GPU that loads this library holds until the process
// exits.  The call waits for its work to finish before it returns.
#include <cstring>
#include <mutex>

#include "bdm_internal.cuh"
#include "bdm.h"

DevParams make_dev_params_for(const bdm_params &P);  // params.cu

namespace {

// capacity of the static scratch array
constexpr long long NA_MAX_AGENTS = 131072;
constexpr long long NA_MAX_BRICKS = 262144;
constexpr long long NA_MAX_OCC = 16384;

constexpr size_t align_up(size_t v) { return (v + 255) / 256 * 256; }

// byte offsets of each table inside the scratch array
constexpr size_t OFF_SETS = 0;
constexpr size_t OFF_CTR = align_up(OFF_SETS + 2 * sizeof(AgentSet));
constexpr size_t OFF_GEOM = align_up(OFF_CTR + sizeof(DevCounters));
constexpr size_t OFF_SIMOFF = align_up(OFF_GEOM + sizeof(SimGeom));
constexpr size_t OFF_BBASE = align_up(OFF_SIMOFF + 2 * sizeof(long long));
constexpr size_t OFF_BBOX = align_up(OFF_BBASE + 2 * sizeof(long long));
constexpr size_t OFF_FLAGS = align_up(OFF_BBOX + 12 * sizeof(unsigned long long));
constexpr size_t OFF_KEY = align_up(OFF_FLAGS + NA_MAX_AGENTS);
constexpr size_t OFF_ARR = align_up(OFF_KEY + NA_MAX_AGENTS * 4);
constexpr size_t OFF_BUCKET = align_up(OFF_ARR + NA_MAX_AGENTS * 4);
constexpr size_t OFF_PERM = align_up(OFF_BUCKET + NA_MAX_AGENTS * 4);
constexpr size_t OFF_C32 = align_up(OFF_PERM + NA_MAX_AGENTS * 4);
constexpr size_t OFF_C64 = align_up(OFF_C32 + NA_MAX_AGENTS * sizeof(float4));
constexpr size_t OFF_BTABLE = align_up(OFF_C64 + NA_MAX_AGENTS * sizeof(dbl4));
constexpr size_t OFF_BCOUNT = align_up(OFF_BTABLE + NA_MAX_BRICKS * 4);
constexpr size_t OFF_BSTART = align_up(OFF_BCOUNT + NA_MAX_BRICKS * 4);
constexpr size_t OFF_BOCC = align_up(OFF_BSTART + NA_MAX_BRICKS * 4);
constexpr size_t OFF_DIRTY = align_up(OFF_BOCC + NA_MAX_BRICKS * 4);
constexpr size_t OFF_OCCL = align_up(OFF_DIRTY + NA_MAX_BRICKS * 8);
constexpr size_t OFF_OCCI = align_up(OFF_OCCL + NA_MAX_OCC * 4);
constexpr size_t OFF_HEAVY = align_up(OFF_OCCI + NA_MAX_OCC * sizeof(int4));
constexpr size_t OFF_BOXS = align_up(OFF_HEAVY + NA_MAX_OCC * 4);
constexpr size_t OFF_BOXC = align_up(OFF_BOXS + NA_MAX_OCC * 64 * 4);
constexpr size_t SCAN_N = (NA_MAX_BRICKS + SCAN_TILE - 1) / SCAN_TILE + 2;
constexpr size_t OFF_SCANA = align_up(OFF_BOXC + NA_MAX_OCC * 64 * 4);
constexpr size_t OFF_SCANB = align_up(OFF_SCANA + SCAN_N * 4);
constexpr size_t SCRATCH_BYTES = align_up(OFF_SCANB + SCAN_N * 4);

// the scratch array (about 23 MB); host code must not use its name as an
// address: the device address comes from cudaGetSymbolAddress
static __device__ __align__(256) unsigned char g_noalloc_scratch[SCRATCH_BYTES];

constexpr int NA_MAX_DEVICES = 64;
unsigned char *g_scratch_ptr[NA_MAX_DEVICES] = {nullptr};
std::mutex g_setup_mutex;
thread_local char g_noalloc_err[256] = "no error";

int na_fail(int code, const char *msg) {
  std::strncpy(g_noalloc_err, msg, sizeof(g_noalloc_err) - 1);
  g_noalloc_err[sizeof(g_noalloc_err) - 1] = 0;
  return code;
}

}  // namespace

extern "C" int bdm_forces_noalloc(int64_t n, const double *xyz, const double *diam, double interaction_radius,
                                  double box_edge, double k, double gamma, double *forces, int32_t *counts,
                                  void *stream) {
  const cudaStream_t st = (cudaStream_t)stream;
  if (n < 0 || (n > 0 && (!xyz || !diam || !forces || !counts)))
    return na_fail(BDM_EINVAL, "bdm_forces_noalloc: n < 0 or a NULL pointer");
  if (n > NA_MAX_AGENTS) return na_fail(BDM_ECAPACITY, "bdm_forces_noalloc: at most 131072 agents");
  const double L = box_edge > 0.0 ? box_edge : interaction_radius;
  if (!(interaction_radius > 0.0) || !(L >= interaction_radius))
    return na_fail(BDM_EINVAL, "bdm_forces_noalloc: need R > 0 and box_edge >= R");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES)
    return na_fail(BDM_ECUDA, "bdm_forces_noalloc: no current CUDA device");
  unsigned char *base = nullptr;
  {
    // once per device, with that device current: the array's device address
    // (cached for the life of the process; a cudaDeviceReset, which unloads
    // this module from the device, invalidates it -- see bdm.h)
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_ptr[dev]) {
      cudaError_t e = cudaGetSymbolAddress((void **)&g_scratch_ptr[dev], g_noalloc_scratch);
      if (e != cudaSuccess) {
        g_scratch_ptr[dev] = nullptr;
        return na_fail(BDM_ECUDA, "bdm_forces_noalloc: cudaGetSymbolAddress failed");
      }
    }
    base = g_scratch_ptr[dev];
  }
  if (n == 0) return BDM_OK;

  bdm_params bp{};
  bp.interaction_radius = interaction_radius;
  bp.box_edge = L;
  bp.k = k;
  bp.gamma = gamma;
  bp.precision = BDM_FP64;
  bp.n_sims = 1;
  bp.capacity = n;
  DevParams dp = make_dev_params_for(bp);

  // the agent set points at the caller's inputs (read only here)
  AgentSet hs{};
  hs.x[0] = hs.x[1] = const_cast<double *>(xyz);
  hs.y[0] = hs.y[1] = const_cast<double *>(xyz + n);
  hs.z[0] = hs.z[1] = const_cast<double *>(xyz + 2 * n);
  hs.diam = const_cast<double *>(diam);
  hs.flags = (uint8_t *)(base + OFF_FLAGS);
  AgentSet sets[2] = {hs, hs};
  DevCounters zc{};
  zc.n = n;

  DevBufs B{};
  B.A = (AgentSet *)(base + OFF_SETS);
  B.A_alt = B.A + 1;
  B.ctr = (DevCounters *)(base + OFF_CTR);
  B.geom = (SimGeom *)(base + OFF_GEOM);
  B.sim_off = (long long *)(base + OFF_SIMOFF);
  B.brick_base = (long long *)(base + OFF_BBASE);
  B.bbox = (unsigned long long *)(base + OFF_BBOX);
  B.brick_table = (int32_t *)(base + OFF_BTABLE);
  B.brick_count = (uint32_t *)(base + OFF_BCOUNT);
  B.brick_start = (uint32_t *)(base + OFF_BSTART);
  B.brick_occ = (int32_t *)(base + OFF_BOCC);
  B.dirty = (unsigned long long *)(base + OFF_DIRTY);
  B.occ_list = (int32_t *)(base + OFF_OCCL);
  B.occ_info = (int4 *)(base + OFF_OCCI);
  B.heavy = (int32_t *)(base + OFF_HEAVY);
  B.box_start = (uint32_t *)(base + OFF_BOXS);
  B.box_cnt = (uint32_t *)(base + OFF_BOXC);
  B.key = (uint32_t *)(base + OFF_KEY);
  B.arrival = (uint32_t *)(base + OFF_ARR);
  B.bucket = (uint32_t *)(base + OFF_BUCKET);
  B.perm = (uint32_t *)(base + OFF_PERM);
  B.c32 = (float4 *)(base + OFF_C32);
  B.c64 = (dbl4 *)(base + OFF_C64);
  B.scan_a = (uint32_t *)(base + OFF_SCANA);
  B.scan_b = (uint32_t *)(base + OFF_SCANB);
  B.fdbg = forces;      // 3 x n, written as x[0..n), y[0..n), z[0..n)
  B.dbg_i32 = counts;   // contacts[0..n) then neighbours[0..n)
  B.brick_cap = NA_MAX_BRICKS;
  B.occ_cap = NA_MAX_OCC;
  B.cap = n;

  LaunchCfg lc{};
  lc.agent_blocks = (int)((n + 255) / 256 < 1216 ? (n + 255) / 256 : 1216);
  lc.brick_blocks = 1024;
  lc.scan_blocks = (int)((NA_MAX_BRICKS + SCAN_TILE - 1) / SCAN_TILE);
  lc.agent_scan_blocks = (int)((n + SCAN_TILE - 1) / SCAN_TILE);
  lc.occ_blocks = 608;
  lc.force_blocks = 608;

  // state every call starts from: agent sets, counters (zero but n),
  // flags zero; the tables the kernels fill are rebuilt on every call
  cudaError_t e = cudaMemcpyAsync(B.A, sets, sizeof(sets), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(B.ctr, &zc, sizeof(zc), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(hs.flags, 0, (size_t)n, st);
  if (e != cudaSuccess) return na_fail(BDM_ECUDA, "bdm_forces_noalloc: initial copies failed");
  launch_bbox(B, dp, lc, st);
  launch_geometry(B, dp, st);
  launch_brick_rank(B, dp, lc, st);
  launch_keys(B, dp, lc, st);
  launch_brick_scan(B, dp, lc, st);
  launch_scatter(B, dp, lc, st);
  launch_brick_sort(B, dp, lc, st);
  launch_force(B, dp, lc, FM_FORCES, st);
  // a launch the runtime rejected (no kernel image, bad configuration) would
  // otherwise leave the outputs unwritten with the device error word still 0
  e = cudaGetLastError();
  if (e != cudaSuccess) return na_fail(BDM_ECUDA, "bdm_forces_noalloc: a kernel launch failed");
  int32_t err = 0;
  e = cudaMemcpyAsync(&err, &B.ctr->error, sizeof(err), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return na_fail(BDM_ECUDA, "bdm_forces_noalloc: kernel or copy failed");
  if (err == DEV_ECAP_BRICKS) return na_fail(BDM_ECAPACITY, "bdm_forces_noalloc: grid exceeds 262144 bricks");
  if (err == DEV_ECAP_OCC) return na_fail(BDM_ECAPACITY, "bdm_forces_noalloc: more than 16384 occupied bricks");
  if (err != 0) return na_fail(BDM_EINVAL, "bdm_forces_noalloc: device error (range or box occupancy)");
  return BDM_OK;
}

extern "C" const char *bdm_noalloc_last_error(void) { return g_noalloc_err; }
