// bdm_internal.cuh -- device data layout, shared device helpers and kernel
// launchers of the GB300 mechanical-interaction iteration.
//
// Data layout in HBM (structure of arrays, storage order, capacity `cap`):
//   X[b][axis]  double   two position buffers; buffer t % 2 holds P_t, buffer
//                        (t + 1) % 2 holds P_(t-1) (read by the static marking)
//   diam        double (FP64 form) or float (FP32-force form)
//   vol, uid, beh, flags, nz   per-agent state and static-detection history
// Grid of one iteration (Sec. 3.1), in Morton order (Sec. 4.2):
//   boxes are grouped in 4x4x4 bricks; a brick's Morton rank among the
//   in-domain bricks orders the bricks, the 6-bit Morton code of the box inside
//   the brick orders the boxes; key = brick rank * 64 + local code.  Agents are
//   counting-sorted into bricks, then each occupied brick is sorted by (box,
//   storage index) on chip, so a box is a contiguous range of sorted positions.
//   c32[k] (float4: box-local x, y, z, radius) and, in the FP64 form,
//   c64[k] (dbl4: x, y, z, radius) hold the agent at sorted position k.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define BDM_MAX_SIMS_SMEM 1024

// 32-byte aligned (x, y, z, w) record of doubles
struct __align__(32) dbl4 {
  double x, y, z, w;
};
__host__ __device__ __forceinline__ dbl4 mk_dbl4(double x, double y, double z, double w) {
  dbl4 r;
  r.x = x; r.y = y; r.z = z; r.w = w;
  return r;
}

// device error word (sticky; kernels return early once it is set)
enum DevError : int32_t {
  DEV_OK = 0,
  DEV_ECAP_BRICKS = 1,  // grid has more bricks than allocated (host regrows)
  DEV_ECAP_OCC = 2,     // more occupied bricks than allocated (host regrows)
  DEV_ECAP_AGENTS = 3,  // daughters would exceed the agent capacity
  DEV_ERANGE = 4,       // a simulation spans more than 2^21 boxes per axis
  DEV_EBOX = 5,         // more than BDM_MAX_BOX_AGENTS agents in one box
  DEV_ENONFINITE = 6,   // a position became non-finite
  DEV_ECHECK = 7,       // a bounds check of the -DBDM_CHECK build failed (line in check_line)
};

#define BDM_MAX_BOX_AGENTS 65536

// agent flag bits
#define FL_CHANGED 1u  // moved, resized or created during the previous iteration
#define FL_MOVED 2u    // position changed during the previous iteration
#define FL_STATIC 4u   // skipped as static in the last iteration
#define FL_DIVIDE 8u   // divides in the current iteration (scratch)
#define FL_REMOVE 16u  // removed at the end of the current iteration (scratch)

#define BEH_GROW 1u
#define BEH_WALK 2u
#define BEH_DIE 4u
#define BEH_TYPE_SHIFT 4  // bits 4-5 of the behaviour byte: the agent's type

struct AgentSet {
  double *x[2], *y[2], *z[2];
  void *diam;  // double* or float*
  double *vol;
  uint64_t *uid;
  uint8_t *beh;
  uint8_t *flags;
  uint16_t *nz;
};

struct SimGeom {
  double lo[3];         // grid origin per axis
  int32_t nb[3];        // boxes per axis
  int32_t nr[3];        // bricks per axis
  int64_t brick_base;   // first global brick index of this simulation
  int64_t n_bricks;     // bricks of this simulation
  int32_t levels;       // Morton levels of the brick grid
  int32_t pad0;
  float lo_f[3];        // lo truncated to float (fast box path)
  float pad1;
  long long lo_fix[3];  // lo in fixed point (scale 2^fix_shift)
  double dt;            // time step
  float dt_f;
  float pad2;
};

struct DevCounters {
  long long n;          // agents
  long long step;       // iterations completed
  unsigned long long next_uid;
  int32_t error;
  int32_t history_valid;
  int32_t check_line;   // -DBDM_CHECK build: source line of the first failed bounds check
  int32_t pad_check;
  long long total_bricks, total_boxes, n_occ, n_div, max_brick;
  long long need_bricks, need_occ;
  int32_t sort_now, force_sort;
  unsigned long long work_next;  // dynamic brick fetch of the force kernel
  unsigned long long work_next2; // the same for the light bricks of the hybrid force launch
  // the force kernels take the heaviest bricks first: bricks of at least
  // FORCE_HEAVY_HI agents (heavy list front), then of at least FORCE_HEAVY_LO
  // (heavy list back), then the rest in Morton order
  unsigned long long heavy_n[2], heavy_take[2];
  unsigned long long work_n;     // entries of the static pass's work list
  // removal (Sec. 3.2): agents removed this iteration, the size after the
  // commit, the holes below it; ghosts = agents removed in the previous
  // iteration, whose boxes the static test marks dirty
  long long n_rm, rm_m;
  unsigned long long rm_h;
  long long n_ghost;
  unsigned long long fix_n;      // FP32 form: agents listed for the FP64 fix-up pass
  // per-iteration accumulators (reset by the geometry kernel)
  unsigned long long a_static, a_moved, a_cand, a_nbr, a_contact, a_exact;
  // snapshot of the last completed iteration
  unsigned long long l_static, l_moved, l_cand, l_nbr, l_contact, l_exact, l_div, l_rm, l_fix;
  long long l_boxes, l_bricks, l_occ, l_max_brick;
};

struct DevParams {
  double R, R2, L;
  double dt, dmax, k, gamma, adherence;
  double growth, divide_volume, ratio_lo, ratio_hi, walk_step;
  double death_prob;                // per-iteration removal probability of BEH_DIE agents
  uint64_t death_thr;               // ceil(death_prob * 2^53): the integer form of u < death_prob
  uint64_t seed;
  float Rf, R2_lo_f, R2_hi_f, Lf;   // FP32 prefilter: certain neighbour / certain not
  float cband1, cband2;             // contact band: W = cband1 * s + cband2 * s^2
  float kf, gammaf, dmaxf, adherencef, walkf, invLf;
  float box_eps;                    // relative error bound of the fast box path
  float graze;                      // FP32 overlaps below this (um) are "grazing"
  float graze_e;                    // error bound of an FP32 overlap (um)
  float graze_exact;                // FP32 overlaps below this (um) are evaluated in FP64
  float rel_tol, abs_tol;           // FP32-form force tolerance the refinement keeps
  float low_scale;                  // agents whose summed pair-force magnitude is below this
                                    // are evaluated in FP64
  float close2;                     // FP32 form: pairs closer than this (um^2) are evaluated
                                    // in FP64 (their FP32 direction is too rough)
  int32_t fix_shift;                // fixed-point scale bits of the local coordinates
  int32_t df_shift;                 // fixed-point bits of contact_df's differences (|D| 2^s < 2^46)
  int32_t brick_class;              // bricks a force launch takes: 0 all, 1 not light, 2 light only
  uint32_t light_max;               // hybrid force launch: bricks of fewer agents are light
  long long L_fix;                  // box edge in fixed point (multiple of 128)
  int32_t precision, detect_static, sort_every, n_sims, keep_forces, grow, walk, die;
  int32_t n_types;                  // > 1: the pair's constants are type_k / type_gamma[4 a + b]
  int32_t curve;                    // brick order: 0 Morton, 1 Hilbert
  double type_k[16], type_gamma[16];  // of the agents' types a, b (bits 4-5 of the behaviour)
  int32_t lanes_fixed;              // FP32 form: > 0 lanes per agent of the force kernel; -1
                                    // lanes chosen per box by its cost model
};

// Everything a kernel reaches, passed by value.
struct DevBufs {
  AgentSet *A;          // device-resident current agent set (swapped by the sort)
  AgentSet *A_alt;      // device-resident other set
  DevCounters *ctr;
  SimGeom *geom;
  long long *sim_off;   // n_sims + 1 (static in ensembles)
  long long *brick_base;// n_sims + 1
  unsigned long long *bbox;  // [2][n_sims][6] order-preserving encodings
  int32_t *brick_table;      // (sim, linear brick) -> global brick rank
  uint32_t *brick_count, *brick_start;
  int32_t *brick_occ;        // global brick rank -> occupied index or -1
  unsigned long long *dirty; // global brick rank -> 64-box dirty mask
  int32_t *occ_list;         // occupied index -> global brick rank
  int4 *occ_info;            // occupied index -> (Bx, By, Bz, sim)
  uint32_t *box_start, *box_cnt;  // occupied index * 64 + local code
  uint32_t *key, *arrival, *bucket, *perm;
  float4 *c32;
  dbl4 *c64;
  uint32_t *scan_a, *scan_b;      // block partials of the scans
  uint32_t *div_rank;
  dbl4 *stash;                 // daughter (x, y, z, volume) by mother index
  dbl4 *ghost;                 // positions of the agents removed in the last iteration
  uint4 *fix;                  // FP32 form: (sorted index, occupied brick * 64 + box, contacts,
                               // neighbours) of the agents the FP64 fix-up pass evaluates
  uint8_t *tp;                 // n_types > 1: the type of the agent at each sorted position
  double *fdbg;                   // 3 x cap forces (debug)
  int32_t *nbr_count;             // debug neighbour lists
  long long *nbr_off;
  long long *nbr_out;
  int32_t *dbg_i32;               // debug: contacts / neighbours
  int32_t *heavy;                 // occ_cap: occupied indices of heavy bricks (both ends)
  unsigned long long *need;       // occ_cap: boxes with non-static agents (static pass)
  int32_t *worklist;              // occ_cap: light bricks with work left (static pass)
  long long brick_cap, occ_cap, cap, nbr_cap;
};

// ----------------------------------------------------------------- bounds checks
// The -DBDM_CHECK build evaluates BDM_IN(counters, condition) at every index
// that a kernel derives from device data before it reads or writes through it
// (box and brick indices, sorted positions, slots against capacities,
// shared-memory tiles and queues).  A failed check sets the sticky error word
// to DEV_ECHECK, records the source line, and the caller substitutes a safe
// index or skips the access, so an out-of-range index becomes a reported
// error instead of a fault.  The regular build compiles the checks away.
#ifdef BDM_CHECK
__device__ __forceinline__ bool bdm_check_in(DevCounters *C, bool ok, int line) {
  if (!ok && atomicCAS(&C->error, 0, (int)DEV_ECHECK) == 0) C->check_line = line;
  return ok;
}
#define BDM_IN(C, cond) bdm_check_in((C), (cond), __LINE__)
#else
#define BDM_IN(C, cond) true
#endif

// ----------------------------------------------------------------- helpers
__device__ __forceinline__ unsigned long long enc_f64(double v) {
  unsigned long long b = (unsigned long long)__double_as_longlong(v);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double dec_f64(unsigned long long e) {
  unsigned long long b = (e >> 63) ? (e & 0x7FFFFFFFFFFFFFFFull) : ~e;
  return __longlong_as_double((long long)b);
}

// truncating double -> float through the bit pattern (error < 1 float ulp);
// keeps the conversion off the FP64 pipe
__device__ __forceinline__ float dtof_trunc(double v) {
  unsigned long long b = (unsigned long long)__double_as_longlong(v);
  unsigned hi = (unsigned)(b >> 32);
  int e = (int)((hi >> 20) & 0x7FF);
  int fe = e - 896;
  if (fe <= 0 || fe >= 255) return (e == 0) ? 0.0f : __double2float_rz(v);
  unsigned mant = (unsigned)((b >> 29) & 0x7FFFFFull);
  return __uint_as_float((hi & 0x80000000u) | ((unsigned)fe << 23) | mant);
}

// exact float -> double through the bit pattern (normal floats and zero)
__device__ __forceinline__ double ftod_exact(float f) {
  unsigned u = __float_as_uint(f);
  unsigned e = (u >> 23) & 0xFF;
  if (e == 0 || e == 255) return (double)f;
  unsigned long long b = ((unsigned long long)(u & 0x80000000u) << 32) |
                         ((unsigned long long)(e - 127 + 1023) << 52) |
                         ((unsigned long long)(u & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)b);
}

// double -> fixed point (truncation of |v| * 2^s), without the FP64 pipe
__device__ __forceinline__ long long to_fixed(double v, int s) {
  unsigned long long b = (unsigned long long)__double_as_longlong(v);
  int e = (int)((b >> 52) & 0x7FF);
  if (e == 0) return 0;
  long long m = (long long)((b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull);
  int sh = e - 1075 + s;
  long long r;
  if (sh >= 0) r = (sh > 9) ? (1ll << 62) : (m << sh);
  else r = (sh <= -63) ? 0 : (m >> (-sh));
  return (b >> 63) ? -r : r;
}

// 2-bit-per-axis Morton code of a box inside its brick (x low bit)
__device__ __forceinline__ int local_code(int lx, int ly, int lz) {
  return (lx & 1) | ((ly & 1) << 1) | ((lz & 1) << 2) | ((lx & 2) << 2) | ((ly & 2) << 3) | ((lz & 2) << 4);
}
__device__ __forceinline__ void local_decode(int c, int &lx, int &ly, int &lz) {
  lx = (c & 1) | ((c >> 2) & 2);
  ly = ((c >> 1) & 1) | ((c >> 3) & 2);
  lz = ((c >> 2) & 1) | ((c >> 4) & 2);
}

// The 27-box stencil of a local box as masks over the bricks around its
// brick: for local box lb, up to 8 (brick, 64-bit box mask) pairs; bo is the
// brick's index among the 27 ((dz + 1) 9 + (dy + 1) 3 + (dx + 1)).  A box is
// dirty when some pair's mask meets that brick's dirty mask.  The table is
// built at compile time (the same Morton code as local_code).
struct StencilMasks {
  unsigned long long m[64][8];
  unsigned char b[64][8];
  unsigned char n[64];
};
constexpr StencilMasks make_stencil_masks() {
  StencilMasks S{};
  for (int lb = 0; lb < 64; ++lb) {
    const int lx = (lb & 1) | ((lb >> 2) & 2), ly = ((lb >> 1) & 1) | ((lb >> 3) & 2),
              lz = ((lb >> 2) & 1) | ((lb >> 4) & 2);
    int n = 0;
    for (int t = 0; t < 27; ++t) {
      const int ax = lx + t % 3 - 1, ay = ly + (t / 3) % 3 - 1, az = lz + t / 9 - 1;
      const int bo = ((az < 0) ? 0 : (az > 3 ? 2 : 1)) * 9 + ((ay < 0) ? 0 : (ay > 3 ? 2 : 1)) * 3 +
                     ((ax < 0) ? 0 : (ax > 3 ? 2 : 1));
      const int x = ax & 3, y = ay & 3, z = az & 3;
      const int code = (x & 1) | ((y & 1) << 1) | ((z & 1) << 2) | ((x & 2) << 2) | ((y & 2) << 3) | ((z & 2) << 4);
      int e = 0;
      while (e < n && S.b[lb][e] != bo) ++e;
      if (e == n) {
        S.b[lb][e] = (unsigned char)bo;
        ++n;
      }
      S.m[lb][e] |= 1ull << code;
    }
    S.n[lb] = (unsigned char)n;
  }
  return S;
}
__device__ const StencilMasks g_stencil_masks = make_stencil_masks();
// whether a box of the stencil of local box lb is dirty (dm: the 27 bricks'
// dirty masks)
__device__ __forceinline__ bool stencil_dirty(const unsigned long long *dm, int lb) {
  const StencilMasks &S = g_stencil_masks;
  unsigned long long any = 0ull;
  const int n = __ldg(&S.n[lb]);
  for (int e = 0; e < n; ++e) any |= dm[__ldg(&S.b[lb][e])] & __ldg(&S.m[lb][e]);
  return any != 0ull;
}

__device__ __forceinline__ int sim_of_agent(const long long *sim_off, int n_sims, long long i) {
  int lo = 0, hi = n_sims - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (sim_off[mid] <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Box coordinate of one axis: exactly floor(fl(fl(p - lo) / L)), the FP64
// definition; an FP32 estimate decides whenever its error bound cannot cross
// an integer, the FP64 path runs otherwise.
__device__ __forceinline__ int box_axis(double p, double lo, float lo_f, const DevParams &P, bool &fallback) {
  float pf = dtof_trunc(p);
  float a = pf - lo_f;
  float q = a * P.invLf;
  float m = (fabsf(pf) + fabsf(lo_f)) * P.invLf * P.box_eps + fabsf(q) * (4.0f * 1.1920929e-7f) + 1e-30f;
  float f0 = floorf(q - m), f1 = floorf(q + m);
  if (f0 == f1 && fabsf(q) < 1.0e9f) {
    fallback = false;
    return (int)f0;
  }
  fallback = true;
  double qd = floor(__ddiv_rn(__dsub_rn(p, lo), P.L));
  if (qd < -1.0e9) return -1000000000;
  if (qd > 1.0e9) return 1000000000;
  return (int)qd;
}

// ----------------------------------------------------------------- Philox
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of two
// 64x64->128 products with the round multipliers; key bumped by the Weyl
// constants between rounds.
__device__ __forceinline__ void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += W0; k1 += W1; }
    const uint64_t hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
    const uint64_t hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
    const uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
  }
}

#define PURPOSE_DEATH 3ull

// Death of a BEH_DIE agent in iteration `step`: Philox4x64-10 with counter
// (uid, step, PURPOSE_DEATH, 0) and key (seed, 0); the first word's top 53
// bits give u in [0, 1), and the agent is removed iff u < death_prob, taken
// exactly in integers as (w >> 11) < death_thr, death_thr = ceil(death_prob 2^53).
__device__ __forceinline__ bool agent_dies(const DevParams &P, uint64_t uid, long long step) {
  uint64_t c[4] = {uid, (uint64_t)step, PURPOSE_DEATH, 0ull};
  philox4x64_10(c, P.seed, 0ull);
  return (c[0] >> 11) < P.death_thr;
}

// ----------------------------------------------------------------- launchers
struct LaunchCfg {
  int agent_blocks;   // grid-stride agent kernels
  int brick_blocks;   // grid-stride brick kernels
  int scan_blocks;    // ceil(brick_cap / SCAN_TILE)
  int agent_scan_blocks;
  int occ_blocks;
  int force_blocks;    // k_force
};

// FP32 force kernel choice (DevParams::lanes_fixed): FORCE_TILE selects the
// tiled kernel (k_force_tile), FORCE_SPARSE the sparse kernel
// (k_force_sparse), FORCE_HYBRID the sparse kernel for light bricks and the
// lane-per-agent kernel with 4 lanes for the others, a positive value the
// lane-per-agent kernel with that many lanes per agent (4: adapted per pass to
// the agents left in the box), -1 the lane-per-agent kernel with the lanes
// chosen per box by a cost model.  The default: the hybrid launch
#define FORCE_TILE 0
#define FORCE_SPARSE (-3)
#define FORCE_HYBRID (-4)  // the sparse kernel for light bricks, the lane-per-agent kernel (4) for the others
#define FORCE_LIGHT_MAX 192
#define FORCE_LANES_DEFAULT FORCE_HYBRID

// brick weight classes of the force kernels' largest-first order (agents)
#define FORCE_HEAVY_HI 1024
#define FORCE_HEAVY_LO 256
// the hybrid launch's light bricks are never on the heavy lists (which the
// lane-per-agent kernel takes whatever their class)
static_assert(FORCE_LIGHT_MAX <= FORCE_HEAVY_LO, "light bricks must not be heavy-listed");


#define SCAN_TILE 2048
#define SCAN_THREADS 256

enum ForceMode : int32_t { FM_STEP = 0, FM_FORCES = 1, FM_COUNT_NBR = 2, FM_LIST_NBR = 3 };

void launch_geometry(const DevBufs &B, const DevParams &P, cudaStream_t s);
void launch_brick_rank(const DevBufs &B, const DevParams &P, const LaunchCfg &c, cudaStream_t s);
void launch_keys(const DevBufs &B, const DevParams &P, const LaunchCfg &c, cudaStream_t s);
void launch_brick_scan(const DevBufs &B, const DevParams &P, const LaunchCfg &c, cudaStream_t s);
void launch_scatter(const DevBufs &B, const DevParams &P, const LaunchCfg &c, cudaStream_t s);
void launch_brick_sort(const DevBufs &B, const DevParams &P, const LaunchCfg &c, cudaStream_t s);
void launch_gather(const DevBufs &B, const DevParams &P, const LaunchCfg &c, cudaStream_t s);
void launch_force(const DevBufs &B, const DevParams &P, const LaunchCfg &c, int mode, cudaStream_t s);
void launch_divide(const DevBufs &B, const DevParams &P, const LaunchCfg &c, cudaStream_t s);
int divide_launches(const DevParams &P);  // kernels launch_divide enqueues
int force_launches(const DevParams &P);   // kernels launch_force enqueues (without the static pass)
void launch_force_fix(const DevBufs &B, const DevParams &P, const LaunchCfg &c, int mode, cudaStream_t s);
int force_fix_launches(const DevParams &P);
void launch_finish(const DevBufs &B, const DevParams &P, cudaStream_t s);
void launch_bbox(const DevBufs &B, const DevParams &P, const LaunchCfg &c, cudaStream_t s);
void launch_debug_boxes(const DevBufs &B, const DevParams &P, const LaunchCfg &c, int32_t *out_box,
                        long long *out_rank, cudaStream_t s);
void launch_diam_to_f64(const DevBufs &B, const DevParams &P, const LaunchCfg &c, double *out, cudaStream_t s);
void launch_init_agents(const DevBufs &B, const DevParams &P, const LaunchCfg &c, const double *diam_in,
                        const double *vol_in, const uint64_t *uid_in, const uint8_t *beh_in, long long n, int *bad,
                        cudaStream_t s);
void launch_positions_in(const double *x, const double *y, const double *z, const AgentSet &A, long long n, int *bad,
                         const LaunchCfg &c, cudaStream_t s);
void launch_nbr_offsets(const DevBufs &B, const DevParams &P, cudaStream_t s);
