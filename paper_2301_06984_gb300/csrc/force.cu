// force.cu -- the 27-box overlap force, clamped displacement, behaviours
// (random walk, growth, division) and the parallel merge of daughters.
//
// Force (Sec. 5; the paper defers to the Cortex3D collision force):
//   for neighbours j != i with d^2 < R^2 and delta = r_i + r_j - d > 0:
//   F = k delta - gamma sqrt(rbar delta), rbar = r_i r_j / (r_i + r_j),
//   f_i += F (p_i - p_j) / d; displacement dt * sum f unless |sum f| <=
//   adherence, clamped to max_displacement; random walk added after the clamp.
//
// Work decomposition: one CTA per occupied 4x4x4 brick (fetched dynamically),
// one warp per box.  The warp resolves the 27 stencil boxes once (lanes 0..26),
// then takes the box's agents in passes: S lanes per agent split the staged
// candidates (FP32 form; with 4 lanes per agent, S follows the agents left in
// the box: 2 while 11 or more are left, 4, and 8 to 32 for a last pass of 4 or
// fewer; lanes = -1 chooses S per box by a cost model) and a shuffle tree
// reduces the S partial sums.  The FP64 form keeps one lane
// per agent and the canonical summation order (stencil boxes dz, dy, dx
// ascending; ascending storage index inside a box), which makes it bit-equal
// to the FP64 oracle.  Both forms decide "neighbour" (d^2 < R^2) and
// "contact" (delta > 0) exactly as FP64 does: an FP32 estimate with a rigorous
// error band decides outside the band, FP64 decides inside it.
#include <type_traits>

#include "bdm_internal.cuh"

namespace {

#define PURPOSE_RATIO 0ull
#define PURPOSE_AXIS 1ull
#define PURPOSE_WALK 2ull
#define MAX_DRAWS 1000

__device__ __forceinline__ double u53(uint64_t w) {
  return __dmul_rn(__ull2double_rn(w >> 11), 1.0 / 9007199254740992.0);
}

// Marsaglia (1972) disc method in FP64, operation for operation as the
// contract states it: x1, x2 = 2u - 1; accept 0 < s = x1^2 + x2^2 < 1;
// u = (2 x1 sqrt(1-s), 2 x2 sqrt(1-s), 1 - 2 s); two attempts per block.
__device__ void unit_vector_f64(uint64_t seed, uint64_t uid, uint64_t step, uint64_t purpose, double out[3]) {
  for (uint64_t draw = 0; draw < MAX_DRAWS; ++draw) {
    uint64_t c[4] = {uid, step, purpose, draw};
    philox4x64_10(c, seed, 0ull);
    for (int a = 0; a < 2; ++a) {
      const double x1 = __dsub_rn(__dmul_rn(2.0, u53(c[2 * a])), 1.0);
      const double x2 = __dsub_rn(__dmul_rn(2.0, u53(c[2 * a + 1])), 1.0);
      const double s = __dadd_rn(__dmul_rn(x1, x1), __dmul_rn(x2, x2));
      if (s > 0.0 && s < 1.0) {
        const double q = __dsqrt_rn(__dsub_rn(1.0, s));
        out[0] = __dmul_rn(__dmul_rn(2.0, x1), q);
        out[1] = __dmul_rn(__dmul_rn(2.0, x2), q);
        out[2] = __dsub_rn(1.0, __dmul_rn(2.0, s));
        return;
      }
    }
  }
  out[0] = 0.0; out[1] = 0.0; out[2] = 1.0;
}

// Same accept/reject decisions as the FP64 method, taken in exact integer
// arithmetic (x = A 2^-52 exactly; s = (A^2 + B^2) 2^-104), with FP64 only
// when the sum lies within the FP64 rounding band around 1; the components
// are then formed in FP32 (1 - s exact from the integers).
__device__ void unit_vector_f32(uint64_t seed, uint64_t uid, uint64_t step, uint64_t purpose, float out[3]) {
  for (uint64_t draw = 0; draw < MAX_DRAWS; ++draw) {
    uint64_t c[4] = {uid, step, purpose, draw};
    philox4x64_10(c, seed, 0ull);
    for (int a = 0; a < 2; ++a) {
      const long long A = (long long)(c[2 * a] >> 11) - (1ll << 52);
      const long long Bv = (long long)(c[2 * a + 1] >> 11) - (1ll << 52);
      const uint64_t ua = (uint64_t)(A < 0 ? -A : A), ub = (uint64_t)(Bv < 0 ? -Bv : Bv);
      const uint64_t alo = ua * ua, ahi = __umul64hi(ua, ua);
      const uint64_t blo = ub * ub, bhi = __umul64hi(ub, ub);
      const uint64_t slo = alo + blo;
      const uint64_t shi = ahi + bhi + (slo < alo ? 1ull : 0ull);
      if (shi == 0 && slo == 0) continue;  // s == 0: reject
      // one = 2^104 = (2^40, 0); band = 2^54 around it
      const uint64_t one_hi = 1ull << 40;
      // S < 2^104 - 2^54 ?
      const bool below = (shi < one_hi - 1) || (shi == one_hi - 1 && slo < (0ull - (1ull << 54)));
      // S > 2^104 + 2^54 ?
      const bool above = (shi > one_hi) || (shi == one_hi && slo > (1ull << 54));
      bool accept;
      if (below) accept = true;
      else if (above) accept = false;
      else {
        const double x1 = __dsub_rn(__dmul_rn(2.0, u53(c[2 * a])), 1.0);
        const double x2 = __dsub_rn(__dmul_rn(2.0, u53(c[2 * a + 1])), 1.0);
        const double s = __dadd_rn(__dmul_rn(x1, x1), __dmul_rn(x2, x2));
        accept = (s > 0.0 && s < 1.0);
      }
      if (!accept) continue;
      // 1 - s = D 2^-104 with D = 2^104 - S (exact; 0 when S >= 2^104)
      float oms = 0.0f;
      if (shi < one_hi) {
        const uint64_t dlo = 0ull - slo;
        const uint64_t dhi = one_hi - shi - (slo != 0 ? 1ull : 0ull);
        oms = __ull2float_rn(dhi) * 9.094947e-13f /* 2^-40 */ + __ull2float_rn(dlo) * 4.9303807e-32f /* 2^-104 */;
      }
      const float q = sqrtf(fmaxf(oms, 0.0f));
      const float x1f = (float)(int)(A >> 29) * 1.1920929e-7f;
      const float x2f = (float)(int)(Bv >> 29) * 1.1920929e-7f;
      out[0] = 2.0f * x1f * q;
      out[1] = 2.0f * x2f * q;
      out[2] = 2.0f * oms - 1.0f;
      return;
    }
  }
  out[0] = 0.f; out[1] = 0.f; out[2] = 1.f;
}

// Cube root by Newton's method after an exact power-of-two range reduction
// (x = m 2^(3q), m in [0.5, 4)); six steps y <- y - (y^3 - m) / (3 y^2) from
// the first guess 0.6 + 0.25 m, every step a single IEEE operation.
__device__ double cbrt_newton(double x) {
  if (x == 0.0 || !isfinite(x)) return x;
  double sgn = 1.0;
  if (x < 0.0) { sgn = -1.0; x = -x; }
  int e;
  double m = frexp(x, &e);
  int q = e / 3, r = e % 3;
  if (r < 0) { r += 3; q -= 1; }
  m = ldexp(m, r);
  double y = __dadd_rn(0.6, __dmul_rn(0.25, m));
  for (int it = 0; it < 6; ++it) {
    const double y2 = __dmul_rn(y, y);
    const double y3 = __dmul_rn(y2, y);
    y = __dsub_rn(y, __ddiv_rn(__dsub_rn(y3, m), __dmul_rn(3.0, y2)));
  }
  return __dmul_rn(sgn, ldexp(y, q));
}

__device__ __forceinline__ double uniform_draw(uint64_t seed, uint64_t uid, uint64_t step, uint64_t purpose) {
  uint64_t c[4] = {uid, step, purpose, 0ull};
  philox4x64_10(c, seed, 0ull);
  return u53(c[0]);
}

// ---------------------------------------------------------------- pair work
constexpr float TINY2 = 1.0e-6f;  // d^2 below this (um^2) goes to FP64

template <int PREC>
__device__ __forceinline__ dbl4 exact_of(const DevBufs &B, const AgentSet &A, int cur, unsigned k) {
  if (PREC == 0) return B.c64[k];
  const uint32_t i = B.perm[k];
  return mk_dbl4(A.x[cur][i], A.y[cur][i], A.z[cur][i], ftod_exact(B.c32[k].w));
}

// FP64 pair: returns 0 not a neighbour, 1 neighbour without force, 2 contact
// (force added to f*)
__device__ __forceinline__ int pair_f64_k(double R2, double k, double gamma, const dbl4 &q, const dbl4 &c, double &fx,
                                          double &fy, double &fz) {
  const double ddx = __dsub_rn(q.x, c.x), ddy = __dsub_rn(q.y, c.y), ddz = __dsub_rn(q.z, c.z);
  const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy)), __dmul_rn(ddz, ddz));
  if (!(d2 < R2)) return 0;
  if (d2 == 0.0) return 1;
  const double d = __dsqrt_rn(d2);
  const double delta = __dsub_rn(__dadd_rn(q.w, c.w), d);
  if (!(delta > 0.0)) return 1;
  const double rbar = __ddiv_rn(__dmul_rn(q.w, c.w), __dadd_rn(q.w, c.w));
  const double F = __dsub_rn(__dmul_rn(k, delta), __dmul_rn(gamma, __dsqrt_rn(__dmul_rn(rbar, delta))));
  const double sc = __ddiv_rn(F, d);
  fx = __dadd_rn(fx, __dmul_rn(sc, ddx));
  fy = __dadd_rn(fy, __dmul_rn(sc, ddy));
  fz = __dadd_rn(fz, __dmul_rn(sc, ddz));
  return 2;
}
// The same pair as pair_f64_k, returning the three products sc * (q - c) that
// pair_f64_k adds to the running sum (so a caller can add them later, in the
// same order, with the same IEEE operations).
__device__ __forceinline__ int pair_f64_terms(const DevParams &P, double k, double gamma, const dbl4 &q, const dbl4 &c,
                                              double &tx, double &ty, double &tz) {
  const double ddx = __dsub_rn(q.x, c.x), ddy = __dsub_rn(q.y, c.y), ddz = __dsub_rn(q.z, c.z);
  const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy)), __dmul_rn(ddz, ddz));
  if (!(d2 < P.R2)) return 0;
  if (d2 == 0.0) return 1;
  const double d = __dsqrt_rn(d2);
  const double delta = __dsub_rn(__dadd_rn(q.w, c.w), d);
  if (!(delta > 0.0)) return 1;
  const double rbar = __ddiv_rn(__dmul_rn(q.w, c.w), __dadd_rn(q.w, c.w));
  const double F = __dsub_rn(__dmul_rn(k, delta), __dmul_rn(gamma, __dsqrt_rn(__dmul_rn(rbar, delta))));
  const double sc = __ddiv_rn(F, d);
  tx = __dmul_rn(sc, ddx);
  ty = __dmul_rn(sc, ddy);
  tz = __dmul_rn(sc, ddz);
  return 2;
}

__device__ __forceinline__ bool is_nbr_f64(const DevParams &P, const dbl4 &q, const dbl4 &c) {
  const double ddx = __dsub_rn(q.x, c.x), ddy = __dsub_rn(q.y, c.y), ddz = __dsub_rn(q.z, c.z);
  const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy)), __dmul_rn(ddz, ddz));
  return d2 < P.R2;
}

__device__ __forceinline__ unsigned long long wmin64(unsigned long long v) {
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = (w < v) ? w : v;
  }
  return v;
}
__device__ __forceinline__ unsigned long long wmax64(unsigned long long v) {
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = (w > v) ? w : v;
  }
  return v;
}
__device__ __forceinline__ unsigned long long wsum64(unsigned long long v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ void flush_bbox(const DevBufs &B, const DevParams &P, int nxt, int sim,
                                           unsigned long long bmin[3], unsigned long long bmax[3]) {
  unsigned long long v[6];
  for (int d = 0; d < 3; ++d) { v[d] = wmin64(bmin[d]); v[3 + d] = wmax64(bmax[d]); }
  if ((threadIdx.x & 31) == 0 && sim >= 0 && v[0] != ~0ull) {
    unsigned long long *bb = B.bbox + ((size_t)nxt * P.n_sims + sim) * 6;
    for (int d = 0; d < 3; ++d) { atomicMin(&bb[d], v[d]); atomicMax(&bb[3 + d], v[3 + d]); }
  }
  for (int d = 0; d < 3; ++d) { bmin[d] = ~0ull; bmax[d] = 0ull; }
}

#define FORCE_WARPS 8
#define CHUNK 96

// Next occupied brick for a force-kernel CTA (called by one thread; phase is
// that thread's cursor, starting at 0): the heaviest bricks first, so that no
// CTA starts a dense brick when the others are about to run out of work.
// Returns -1 when every brick has been handed out.
// With static detection (use_static) only bricks with work left after
// k_static are handed out: heavy ones whose need mask is not empty, then the
// work list.
// With brick_class 1 (the hybrid launch's dense part) light bricks (fewer than
// light_max agents) are skipped; with brick_class 2 only light bricks are
// handed out, from their own cursor.
__device__ __forceinline__ long long next_force_brick(const DevBufs &B, const DevParams &P, DevCounters *C,
                                                      long long n_occ, int &phase, bool use_static) {
  if (P.brick_class == 2) {
    while (true) {
      const long long u = (long long)atomicAdd(&C->work_next2, 1ull);
      long long o;
      if (use_static) {
        if (u >= (long long)C->work_n) return -1;
        o = B.worklist[u];
      } else {
        if (u >= n_occ) return -1;
        o = u;
      }
      if (B.brick_count[B.occ_list[o]] < P.light_max) return o;
    }
  }
  while (true) {
    if (phase < 2) {
      const unsigned long long u = atomicAdd(&C->heavy_take[phase], 1ull);
      if (u < C->heavy_n[phase]) {
        const long long o = phase == 0 ? B.heavy[u] : B.heavy[B.occ_cap - 1 - (long long)u];
        if (!use_static || B.need[o]) return o;
        continue;
      }
      phase++;
      continue;
    }
    const long long u = (long long)atomicAdd(&C->work_next, 1ull);
    long long o;
    if (use_static) {
      if (u >= (long long)C->work_n) return -1;
      o = B.worklist[u];
    } else {
      if (u >= n_occ) return -1;
      o = u;
      if (B.brick_count[B.occ_list[o]] >= FORCE_HEAVY_LO) continue;  // heavy ones were listed
    }
    if (P.brick_class == 1 && B.brick_count[B.occ_list[o]] < P.light_max) continue;
    return o;
  }
}

// flush a warp's shared bounding-box accumulator into the simulation's
__device__ __forceinline__ void flush_bbox_warp(const DevBufs &B, const DevParams &P, int nxt, int sim,
                                                unsigned long long *bb_w) {
  __syncwarp();
  if ((threadIdx.x & 31) == 0 && sim >= 0 && bb_w[0] != ~0ull) {
    unsigned long long *bb = B.bbox + ((size_t)nxt * P.n_sims + sim) * 6;
    for (int d = 0; d < 3; ++d) { atomicMin(&bb[d], bb_w[d]); atomicMax(&bb[3 + d], bb_w[3 + d]); }
  }
  __syncwarp();
  if ((threadIdx.x & 31) < 6) bb_w[threadIdx.x & 31] = ((threadIdx.x & 31) < 3) ? ~0ull : 0ull;
  __syncwarp();
}

// FP32 form of the displacement before the random walk (Sec. 5): dt F when
// |F| exceeds the adherence, scaled down to the maximum displacement.
__device__ __forceinline__ void displacement_f32(const DevParams &P, float dt_f, float fx, float fy, float fz,
                                                 float &ux, float &uy, float &uz) {
  ux = uy = uz = 0.f;
  const float fn2 = fmaf(fx, fx, fmaf(fy, fy, fz * fz));
  if (fn2 > P.adherencef * P.adherencef) {
    ux = dt_f * fx; uy = dt_f * fy; uz = dt_f * fz;
    const float dn2 = fmaf(ux, ux, fmaf(uy, uy, uz * uz));
    if (dn2 > P.dmaxf * P.dmaxf) {
      const float c = P.dmaxf * rsqrtf(dn2);
      ux *= c; uy *= c; uz *= c;
    }
  }
}

// Per-agent end of the force kernels (px, py, pz: the agent's position P_t).
// FM_FORCES records the summed force and the contact and neighbour counts in
// the debug buffers.  FM_STEP forms the displacement
// (Sec. 5: dt F unless |F| <= adherence, clamped to the
// maximum displacement, random walk added after the clamp), grows and divides
// (FP64 form), writes the new position when it or the previous one moved,
// and records the flags and the simulation's bounding box.
template <int PREC, int MODE>
__device__ __forceinline__ void finish_agent(const DevBufs &B, const DevParams &P, const AgentSet &A, int cur, int nxt,
                                             long long step, double dt, float dt_f, uint32_t iq, uint8_t fl,
                                             bool is_static, float ffx, float ffy, float ffz, double dfx, double dfy,
                                             double dfz, unsigned nnb, unsigned ncont, unsigned &c_static,
                                             unsigned &c_moved, unsigned long long *bb_w, double px, double py,
                                             double pz) {
  double Fx, Fy, Fz;
  if (PREC == 0) { Fx = dfx; Fy = dfy; Fz = dfz; }
  else { Fx = ftod_exact(ffx); Fy = ftod_exact(ffy); Fz = ftod_exact(ffz); }
  if (MODE == FM_FORCES) {
    B.fdbg[iq] = Fx; B.fdbg[B.cap + iq] = Fy; B.fdbg[2 * B.cap + iq] = Fz;
    B.dbg_i32[iq] = (int32_t)ncont;
    B.dbg_i32[B.cap + iq] = (int32_t)nnb;
    return;
  }
  // ----------------------------------------------------- FM_STEP epilogue
  double nx = px, ny = py, nzp = pz;
  uint8_t nfl = 0;
  bool write_pos = (fl & FL_MOVED) != 0;
  if (is_static) {
    nfl = FL_STATIC;
    c_static++;
    Fx = Fy = Fz = 0.0;
  } else {
    const uint8_t beh = (P.walk || P.grow || P.die) ? A.beh[iq] : (uint8_t)0;
    if (P.die && (beh & BEH_DIE) && agent_dies(P, A.uid[iq], step)) {
      // removed at the end of this iteration (Sec. 3.2): no displacement,
      // growth or division, and no part in the next grid's bounding box
      A.flags[iq] = FL_REMOVE;
      A.nz[iq] = (uint16_t)min(ncont, 65535u);
      return;
    }
    if (PREC == 1) {
      float ux, uy, uz;
      displacement_f32(P, dt_f, ffx, ffy, ffz, ux, uy, uz);
      if (P.walk && (beh & BEH_WALK)) {
        float u[3];
        unit_vector_f32(P.seed, A.uid[iq], (uint64_t)step, PURPOSE_WALK, u);
        ux = fmaf(P.walkf, u[0], ux);
        uy = fmaf(P.walkf, u[1], uy);
        uz = fmaf(P.walkf, u[2], uz);
      }
      if (ux != 0.f) nx = __dadd_rn(px, ftod_exact(ux));
      if (uy != 0.f) ny = __dadd_rn(py, ftod_exact(uy));
      if (uz != 0.f) nzp = __dadd_rn(pz, ftod_exact(uz));
    } else {
      double ux = 0.0, uy = 0.0, uz = 0.0;
      const double fn = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(dfx, dfx), __dmul_rn(dfy, dfy)), __dmul_rn(dfz, dfz)));
      if (fn > P.adherence) {
        ux = __dmul_rn(dt, dfx); uy = __dmul_rn(dt, dfy); uz = __dmul_rn(dt, dfz);
        const double dn = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(ux, ux), __dmul_rn(uy, uy)), __dmul_rn(uz, uz)));
        if (dn > P.dmax) {
          const double c = __ddiv_rn(P.dmax, dn);
          ux = __dmul_rn(ux, c); uy = __dmul_rn(uy, c); uz = __dmul_rn(uz, c);
        }
      }
      if (P.walk && (beh & BEH_WALK)) {
        double u[3];
        unit_vector_f64(P.seed, A.uid[iq], (uint64_t)step, PURPOSE_WALK, u);
        ux = __dadd_rn(ux, __dmul_rn(P.walk_step, u[0]));
        uy = __dadd_rn(uy, __dmul_rn(P.walk_step, u[1]));
        uz = __dadd_rn(uz, __dmul_rn(P.walk_step, u[2]));
      }
      nx = __dadd_rn(px, ux);
      ny = __dadd_rn(py, uy);
      nzp = __dadd_rn(pz, uz);
    }
    const bool moved = (nx != px) || (ny != py) || (nzp != pz);
    bool changed = moved;
    if (PREC == 0 && P.grow && (beh & BEH_GROW)) {
      const double pi = 3.141592653589793;
      const double v = __dadd_rn(A.vol[iq], P.growth);
      changed = true;
      if (v >= P.divide_volume) {
        const uint64_t uid = A.uid[iq];
        const double u0 = uniform_draw(P.seed, uid, (uint64_t)step, PURPOSE_RATIO);
        const double rho = __dadd_rn(P.ratio_lo, __dmul_rn(__dsub_rn(P.ratio_hi, P.ratio_lo), u0));
        const double v1 = __ddiv_rn(__dmul_rn(v, rho), __dadd_rn(1.0, rho));
        const double v2 = __ddiv_rn(v, __dadd_rn(1.0, rho));
        double ax[3];
        unit_vector_f64(P.seed, uid, (uint64_t)step, PURPOSE_AXIS, ax);
        const double rad = __dmul_rn(cbrt_newton(__ddiv_rn(__dmul_rn(6.0, v), pi)), 0.5);
        const double a1 = __dmul_rn(rad, __ddiv_rn(v2, v)), a2 = __dmul_rn(rad, __ddiv_rn(v1, v));
        const double cx = nx, cy = ny, cz = nzp;
        nx = __dadd_rn(cx, __dmul_rn(a1, ax[0]));
        ny = __dadd_rn(cy, __dmul_rn(a1, ax[1]));
        nzp = __dadd_rn(cz, __dmul_rn(a1, ax[2]));
        B.stash[iq] = mk_dbl4(__dsub_rn(cx, __dmul_rn(a2, ax[0])), __dsub_rn(cy, __dmul_rn(a2, ax[1])),
                                   __dsub_rn(cz, __dmul_rn(a2, ax[2])), v2);
        A.vol[iq] = v1;
        ((double *)A.diam)[iq] = cbrt_newton(__ddiv_rn(__dmul_rn(6.0, v1), pi));
        nfl |= FL_DIVIDE | FL_MOVED;
        write_pos = true;
      } else {
        A.vol[iq] = v;
        ((double *)A.diam)[iq] = cbrt_newton(__ddiv_rn(__dmul_rn(6.0, v), pi));
      }
    }
    if (moved) { nfl |= FL_MOVED; c_moved++; write_pos = true; }
    if (changed) nfl |= FL_CHANGED;
    A.nz[iq] = (uint16_t)min(ncont, 65535u);
  }
  if (write_pos) {
    A.x[nxt][iq] = nx;
    A.y[nxt][iq] = ny;
    A.z[nxt][iq] = nzp;
  }
  A.flags[iq] = nfl;
  if (P.keep_forces) { B.fdbg[iq] = Fx; B.fdbg[B.cap + iq] = Fy; B.fdbg[2 * B.cap + iq] = Fz; }
  atomicMin(&bb_w[0], enc_f64(nx));
  atomicMax(&bb_w[3], enc_f64(nx));
  atomicMin(&bb_w[1], enc_f64(ny));
  atomicMax(&bb_w[4], enc_f64(ny));
  atomicMin(&bb_w[2], enc_f64(nzp));
  atomicMax(&bb_w[5], enc_f64(nzp));
}
// x and y components of a - b in one packed FP32 subtraction (sub.f32x2,
// sm_100 and later): each half is rounded like a scalar subtraction, so the
// result is bit-identical to two scalar ones at half the issue slots.
__device__ __forceinline__ float2 sub_xy(const float4 &a, const float4 &b) {
  float2 r;
  asm("{\n .reg .b64 ra, rb, rd;\n mov.b64 ra, {%2, %3};\n mov.b64 rb, {%4, %5};\n"
      " sub.rn.f32x2 rd, ra, rb;\n mov.b64 {%0, %1}, rd;\n}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}

// FP32 squared distance of the prefilter, fma(ex, ex, fma(ey, ey, ez ez)).
__device__ __forceinline__ float dist2_f32(const float4 &q, const float4 &c) {
  const float2 e = sub_xy(q, c);
  const float ez = q.z - c.z;
  return fmaf(e.x, e.x, fmaf(e.y, e.y, ez * ez));
}

// One lane's share of a staged chunk: candidates sub, sub + S, sub + 2S, ...
// below fill, each queued (its chunk position, one byte per slot, slots 32
// bytes apart) when its FP32 squared distance is below R2.  SS > 0 fixes the
// stride at compile time.  Returns the number of queued candidates; the queue
// keeps the candidates' order.
template <int SS>
__device__ __forceinline__ unsigned scan_chunk(const float4 *sc, uint8_t *q, const float4 cq, unsigned sub,
                                               unsigned S_, unsigned fill, float R2) {
  const unsigned S = SS > 0 ? (unsigned)SS : S_;
  uint8_t *const q0 = q;
  unsigned i = sub;
  // four independent candidates per iteration (latency hiding)
  for (; i + 3u * S < fill; i += 4u * S) {
    const float e0 = dist2_f32(cq, sc[i]), e1 = dist2_f32(cq, sc[i + S]);
    const float e2 = dist2_f32(cq, sc[i + 2 * S]), e3 = dist2_f32(cq, sc[i + 3 * S]);
    if (e0 < R2) { *q = (uint8_t)i; q += 32; }
    if (e1 < R2) { *q = (uint8_t)(i + S); q += 32; }
    if (e2 < R2) { *q = (uint8_t)(i + 2 * S); q += 32; }
    if (e3 < R2) { *q = (uint8_t)(i + 3 * S); q += 32; }
  }
  for (; i < fill; i += S)
    if (dist2_f32(cq, sc[i]) < R2) { *q = (uint8_t)i; q += 32; }
  return (unsigned)(q - q0) >> 5;
}

// Force of a certain contact from the exact geometry, for the FP32 form's
// contacts whose box-local FP32 records are too coarse (grazing contacts,
// forces near the sign change of k delta - gamma sqrt(rbar delta), close
// pairs).  The two FP64 positions are converted to the grid's fixed point (the
// truncation of each coordinate is below 2^-fs um), so the difference D and
// N = S^2 - |D|^2 (S = r_i + r_j, radii exact in the fixed point) are exact
// integers; delta = N / (S + d) then carries only the FP32 rounding of the
// quotient (about 3e-7 relative) and the direction D / d that of d, all
// without the FP64 pipe.  pq and pc: x, y, z in FP64 and the radius in w.
// Returns the force vector on the agent at pq and |F|.
__device__ __forceinline__ float contact_int(const dbl4 &pq, const dbl4 &pc, int fs, float k, float gamma, float &fx,
                                             float &fy, float &fz) {
  const long long dx = to_fixed(pq.x, fs) - to_fixed(pc.x, fs);
  const long long dy = to_fixed(pq.y, fs) - to_fixed(pc.y, fs);
  const long long dz = to_fixed(pq.z, fs) - to_fixed(pc.z, fs);
  const long long D2 = dx * dx + dy * dy + dz * dz;  // |D| < 2^30: no overflow
  const float rq = (float)pq.w, rc = (float)pc.w;     // exact: the radii are floats
  const float scale = __int_as_float((127 + fs) << 23), unscale = __int_as_float((127 - fs) << 23);
  const long long S = (long long)__fmul_rn(rq, scale) + (long long)__fmul_rn(rc, scale);
  const long long N = S * S - D2;
  fx = fy = fz = 0.f;
  if (D2 <= 0 || N <= 0) return 0.f;
  const float d = sqrtf((float)D2);
  const float delta = __fmul_rn(__fdiv_rn((float)N, __fadd_rn((float)S, d)), unscale);
  const float rbar = __fdiv_rn(__fmul_rn(rq, rc), __fadd_rn(rq, rc));
  const float F = fmaf(k, delta, -__fmul_rn(gamma, sqrtf(__fmul_rn(rbar, delta))));
  const float sc = __fdiv_rn(F, d);
  fx = __fmul_rn(sc, (float)dx);
  fy = __fmul_rn(sc, (float)dy);
  fz = __fmul_rn(sc, (float)dz);
  return fabsf(F);
}

// ---------------------------------------------------------------- double-float contact
// Unevaluated sums h + l of two FP32 numbers (about 44 significant bits),
// formed with error-free transformations: Knuth's TwoSum, the fast two-sum
// for |a| >= |b|, and the product's exact error from one fused multiply-add
// (Dekker 1971; the double-float arithmetic of Hida, Li and Bailey).  Every
// operation is an explicitly rounded intrinsic, so no contraction changes them.
struct DF {
  float h, l;
};
__device__ __forceinline__ DF df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ DF df_fast(float a, float b) {  // |a| >= |b| or a == 0
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DF df_two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, fmaf(a, b, -p)};
}
__device__ __forceinline__ DF df_add(DF x, DF y) {
  const DF s = df_two_sum(x.h, y.h);
  return df_fast(s.h, __fadd_rn(s.l, __fadd_rn(x.l, y.l)));
}
__device__ __forceinline__ DF df_mul(DF x, DF y) {
  const float p = __fmul_rn(x.h, y.h);
  const float e = fmaf(x.h, y.l, fmaf(x.l, y.h, fmaf(x.h, y.h, -p)));
  return df_fast(p, e);
}
// x / y and sqrt(x): an FP32 first approximation (the approximate reciprocal
// and reciprocal square root suffice) corrected once by the exactly formed
// residual
__device__ __forceinline__ DF df_div(DF x, DF y) {
  const float ry = __fdividef(1.0f, y.h);
  const float q1 = __fmul_rn(x.h, ry);
  const DF p = df_mul({q1, 0.f}, y);
  const float r = __fadd_rn(__fsub_rn(__fsub_rn(x.h, p.h), p.l), x.l);  // x - q1 y
  return df_fast(q1, __fmul_rn(r, ry));
}
__device__ __forceinline__ DF df_sqrt(DF x) {  // x > 0
  const float rs = rsqrtf(x.h);
  const float s = __fmul_rn(x.h, rs);
  const DF p = df_two_prod(s, s);
  const float r = __fadd_rn(__fsub_rn(__fsub_rn(x.h, p.h), p.l), x.l);  // x - s^2
  return df_fast(s, __fmul_rn(r, __fmul_rn(0.5f, rs)));
}
// an integer v, |v| < 2^46, times 2^-sh, as a double-float (exact)
__device__ __forceinline__ DF df_of_fixed(long long v, int sh) {
  const int hi = (int)(v >> 22);         // floor(v / 2^22), |hi| < 2^24
  const int lo = (int)(v & 0x3FFFFFll);  // v - hi 2^22, in [0, 2^22)
  const float sc = __int_as_float((127 - sh) << 23);
  const DF r = df_fast(__fmul_rn((float)hi, 4194304.0f), (float)lo);
  return {__fmul_rn(r.h, sc), __fmul_rn(r.l, sc)};
}
__device__ __forceinline__ int exp_of(double v) {  // |v| < 2^exp_of(v)
  return (int)((__double_as_longlong(v) >> 52) & 0x7FF) - 1022;
}

// Force of a certain contact in double-float arithmetic, for the contacts
// whose FP32 and exact-integer forms are too coarse: a force magnitude near
// the sign change of k delta - gamma sqrt(rbar delta), where an absolute error
// of eps delta in delta becomes about k/2 eps delta in F.  The positions'
// differences are taken in fixed point 2^-sh (sh = 40, fewer bits where the
// coordinates or the cutoff R need them: the truncation is below 2^-sh um per
// coordinate), d, delta, rbar, sqrt(rbar delta) and F in double-float, the
// direction (p_i - p_j) / d in FP32.  k and gamma: double-float pair constants.
// Returns |F| and the force vector on the agent at pq.
__device__ __forceinline__ float contact_df(const DevParams &P, const dbl4 &pq, const dbl4 &pc, DF k, DF gamma,
                                            float &fx, float &fy, float &fz) {
  int e = max(max(exp_of(pq.x), exp_of(pq.y)), max(exp_of(pq.z), exp_of(pc.x)));
  e = max(e, max(exp_of(pc.y), exp_of(pc.z)));
  const int sh = max(0, min(P.df_shift, 61 - e));
  const DF Dx = df_of_fixed(to_fixed(pq.x, sh) - to_fixed(pc.x, sh), sh);
  const DF Dy = df_of_fixed(to_fixed(pq.y, sh) - to_fixed(pc.y, sh), sh);
  const DF Dz = df_of_fixed(to_fixed(pq.z, sh) - to_fixed(pc.z, sh), sh);
  fx = fy = fz = 0.f;
  const DF d2 = df_add(df_add(df_mul(Dx, Dx), df_mul(Dy, Dy)), df_mul(Dz, Dz));
  if (!(d2.h > 0.f)) return 0.f;
  const DF d = df_sqrt(d2);
  const float rq = (float)pq.w, rc = (float)pc.w;  // exact: the radii are floats
  const DF S = df_two_sum(rq, rc);
  const DF delta = df_add(S, {-d.h, -d.l});
  if (!(delta.h > 0.f)) return 0.f;
  const DF rbar = df_div(df_two_prod(rq, rc), S);
  const DF sq = df_sqrt(df_mul(rbar, delta));
  const DF gs = df_mul(gamma, sq);
  const DF F = df_add(df_mul(k, delta), {-gs.h, -gs.l});
  const float Ff = __fadd_rn(F.h, F.l);
  const float sc = __fdividef(Ff, d.h);
  fx = __fmul_rn(sc, Dx.h);
  fy = __fmul_rn(sc, Dy.h);
  fz = __fmul_rn(sc, Dz.h);
  return fabsf(Ff);
}


// FP32 force of a certain contact at squared distance d2 (s = r_i + r_j, pi =
// r_i r_j): overlap delta, the scale F / d of the difference vector, and the
// force F itself.  Every operation is rounded as written (the fused
// multiply-adds are explicit), so the force kernel and the FP64 fix-up pass
// form the same bits for the contacts both evaluate in FP32.
struct ContactF32 {
  float inv_d, delta, rbar, sq, fm, scf;
};
__device__ __forceinline__ ContactF32 contact_f32(float d2, float s, float pi, float k, float gamma) {
  ContactF32 c;
  c.inv_d = rsqrtf(d2);
  c.delta = fmaf(-d2, c.inv_d, s);
  c.rbar = __fdividef(pi, s);
  const float rd = __fmul_rn(c.rbar, c.delta);  // > 0 for a certain contact
  c.sq = __fmul_rn(rd, rsqrtf(rd));
  c.fm = fmaf(k, c.delta, -__fmul_rn(gamma, c.sq));
  c.scf = __fmul_rn(c.fm, c.inv_d);
  return c;
}

// SPLIT (FP32 step without random walk or growth only): the agent's lanes
// finish one axis each.  A separate instantiation, so that the other forms
// keep the register allocation they have without that code.
// TYPES: several agent types (the pair constants from the type tables).
template <int PREC, int MODE, bool SPLIT = false, bool TYPES = false>
__global__ void __launch_bounds__(FORCE_WARPS * 32, 4) k_force(DevBufs B, DevParams P) {
  static_assert(!SPLIT || (PREC == 1 && MODE == FM_STEP), "the split epilogue is the FP32 step's");
  __shared__ int s_nocc[27];
  __shared__ unsigned long long s_ndirty[27];
  __shared__ int s_next;
  __shared__ unsigned s_bcnt[64];
  __shared__ uint8_t s_order[64];
  __shared__ unsigned long long s_need;
  __shared__ long long s_o;
  // per-warp statistics in shared memory rather than registers (fewer spills):
  // candidates, neighbours, contacts, FP64 decisions (32-bit shared atomics)
  __shared__ unsigned s_ctr[FORCE_WARPS][4];
  __shared__ double s_pos[FORCE_WARPS][32];  // SPLIT: each lane's position, copied ahead
  __shared__ float4 s_off[27];
  __shared__ unsigned long long s_bb[FORCE_WARPS][6];
  // per warp: a staged chunk of candidate records (box offset applied) and
  // their sorted positions, and per-lane queues of the chunk entries that
  // passed the FP32 prefilter ([warp][slot][lane]: each lane its own bank)
  __shared__ float4 s_c[FORCE_WARPS][CHUNK];
  __shared__ uint32_t s_kj[FORCE_WARPS][CHUNK];
  __shared__ uint8_t s_q[FORCE_WARPS][CHUNK][32];
  __shared__ unsigned s_pre[FORCE_WARPS][32], s_kb[FORCE_WARPS][32];
  // several agent types: the staged candidates' types and the pair constants
  __shared__ uint8_t s_tp[FORCE_WARPS][CHUNK];
  __shared__ float s_tkf[16], s_tgf[16];
  __shared__ double s_tkd[16], s_tgd[16];
  DevCounters *C = B.ctr;
  if (C->error) return;
  const AgentSet A = *B.A;
  const int cur = (int)(C->step & 1), nxt = cur ^ 1;
  const bool use_static = (MODE == FM_STEP) && P.detect_static && C->history_valid;
  const long long n_occ = C->n_occ;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long step = C->step;
  unsigned c_static = 0, c_moved = 0;
  int wsim = -1;
  int fetch_phase = 0;
  if (threadIdx.x < 27) {
    const int t = threadIdx.x;
    s_off[t] = make_float4((float)(t % 3 - 1) * P.Lf, (float)((t / 3) % 3 - 1) * P.Lf, (float)(t / 9 - 1) * P.Lf, 0.f);
  }
  if (lane < 6) s_bb[warp][lane] = (lane < 3) ? ~0ull : 0ull;
  if (lane < 4) s_ctr[warp][lane] = 0u;
  if (TYPES && threadIdx.x < 16) {
    s_tkd[threadIdx.x] = P.type_k[threadIdx.x];
    s_tgd[threadIdx.x] = P.type_gamma[threadIdx.x];
    s_tkf[threadIdx.x] = (float)P.type_k[threadIdx.x];
    s_tgf[threadIdx.x] = (float)P.type_gamma[threadIdx.x];
  }

  // One block per occupied brick (taken from a global counter); its warps
  // take the brick's 64 boxes from a block counter.
  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) {
      s_o = next_force_brick(B, P, C, n_occ, fetch_phase, use_static);
      s_next = 0;
    }
    __syncthreads();
    long long o = s_o;
    if (o < 0) break;
    if (!BDM_IN(B.ctr, o < n_occ)) break;  // block-uniform
    const int4 info = B.occ_info[o];
    const SimGeom &G = B.geom[info.w];
    if (threadIdx.x < 27) {
      const int t = threadIdx.x;
      const int X = info.x + t % 3 - 1, Y = info.y + (t / 3) % 3 - 1, Z = info.z + t / 9 - 1;
      int occ = -1;
      unsigned long long dm = 0ull;
      if (X >= 0 && X < G.nr[0] && Y >= 0 && Y < G.nr[1] && Z >= 0 && Z < G.nr[2]) {
        const int rank = B.brick_table[G.brick_base + ((long long)Z * G.nr[1] + Y) * G.nr[0] + X];
        occ = B.brick_occ[rank];
        if (use_static) dm = B.dirty[rank];
      }
      s_nocc[t] = occ;
      s_ndirty[t] = dm;
    }
    if (threadIdx.x >= 64 && threadIdx.x < 128) s_bcnt[threadIdx.x - 64] = B.box_cnt[o * 64 + threadIdx.x - 64];
    if (threadIdx.x == 32) s_need = use_static ? B.need[o] : ~0ull;
    __syncthreads();
    if (MODE == FM_STEP && info.w != wsim) {
      flush_bbox_warp(B, P, nxt, wsim, s_bb[warp]);
      wsim = info.w;
    }

    const double dt = G.dt;
    const float dt_f = G.dt_f;
    // the warps take the brick's boxes heaviest first (fewest idle warps at
    // the brick's end): rank by agent count, ties by box index
    if (threadIdx.x < 64) {
      const unsigned c = s_bcnt[threadIdx.x];
      unsigned r = 0;
      for (int q = 0; q < 64; ++q) {
        const unsigned cq = s_bcnt[q];
        r += (cq > c) || (cq == c && q < (int)threadIdx.x);
      }
      s_order[r] = (uint8_t)threadIdx.x;
    }
    __syncthreads();

    while (true) {
      int kb = 0;
      if (lane == 0) kb = atomicAdd(&s_next, 1);
      kb = __shfl_sync(0xffffffffu, kb, 0);
      if (kb >= 64) break;
      const int lb = s_order[kb];
      if (!((s_need >> lb) & 1ull)) continue;  // nothing left after the static pass
      const unsigned qbase = B.box_start[o * 64 + lb], nq = B.box_cnt[o * 64 + lb];
      if (nq == 0) continue;
      int lx, ly, lz;
      local_decode(lb, lx, ly, lz);
      unsigned nb_st = 0, nb_cnt = 0;
      bool nb_dirty = false;
      if (lane < 27) {
        const int ax = lx + lane % 3 - 1, ay = ly + (lane / 3) % 3 - 1, az = lz + lane / 9 - 1;
        const int bo = ((az < 0) ? 0 : (az > 3 ? 2 : 1)) * 9 + ((ay < 0) ? 0 : (ay > 3 ? 2 : 1)) * 3 +
                       ((ax < 0) ? 0 : (ax > 3 ? 2 : 1));
        const int lc = local_code(ax & 3, ay & 3, az & 3);
        const int occ = s_nocc[bo];
        if (occ >= 0) {
          nb_st = B.box_start[(long long)occ * 64 + lc];
          nb_cnt = B.box_cnt[(long long)occ * 64 + lc];
        }
        nb_dirty = (s_ndirty[bo] >> lc) & 1ull;
      }
      const bool clean = !__any_sync(0xffffffffu, nb_dirty);
      // exclusive prefix of the stencil box counts (canonical box order)
      unsigned pre = nb_cnt;
      for (int of = 1; of < 32; of <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, pre, of);
        if (lane >= of) pre += y;
      }
      const unsigned ctot = __shfl_sync(0xffffffffu, pre, 31);
      // box starts in the stencil (s_pre[27] = ctot, then UINT_MAX: the
      // staging's search needs no range test) and each box's first sorted
      // position minus its start
      s_pre[warp][lane] = (lane <= 27) ? pre - nb_cnt : 0xFFFFFFFFu;
      s_kb[warp][lane] = nb_st - (pre - nb_cnt);
      __syncwarp();
      // lanes per agent: split the candidates of small boxes over several lanes
      int S = 1;
      if (PREC == 1 && (MODE == FM_STEP || MODE == FM_FORCES) && P.lanes_fixed > 0) {
        S = P.lanes_fixed;
      } else if (PREC == 1 && (MODE == FM_STEP || MODE == FM_FORCES)) {
        unsigned best = 0xffffffffu;
        for (int ls = 0; ls <= 5; ++ls) {
          const unsigned passes = (nq + (32u >> ls) - 1) >> (5 - ls);
          const unsigned cost = passes * (((ctot + (1u << ls) - 1) >> ls) + 2u);
          if (cost < best) { best = cost; S = 1 << ls; }
        }
      }
      // With 4 lanes per agent the lanes follow the agents still to do: 2
      // lanes (16 agents a pass) while 11 or more are left, so that a crowded
      // box stages its stencil fewer times, and a last pass of 4 agents or
      // fewer spread over the whole warp (8, 16 or 32 lanes per agent).  One
      // lane per agent would stage less again, but its single FP32 sum over a
      // crowded stencil loses accuracy.
      const int S0 = S;
      for (unsigned q0 = 0; q0 < nq; q0 += 32u / (unsigned)S) {
        if (PREC == 1 && S0 == 4) {
          const unsigned rem = nq - q0;
          S = (rem >= 11u) ? 2 : (rem <= 1u) ? 32 : (rem <= 2u) ? 16 : (rem <= 4u) ? 8 : 4;
        }
        const int sub = lane & (S - 1);
        const unsigned qi = q0 + (unsigned)(lane / S);
        bool valid = qi < nq;
        unsigned kq = qbase + (valid ? qi : 0u);
        if (!BDM_IN(B.ctr, (long long)kq < C->n)) { kq = 0; valid = false; }
        uint32_t iq = B.perm[kq];
        if (!BDM_IN(B.ctr, (long long)iq < B.cap)) { iq = 0; valid = false; }
        const float4 cq = B.c32[kq];
        dbl4 dq = mk_dbl4(0.0, 0.0, 0.0, 0.0);
        if (PREC == 0) dq = B.c64[kq];
        const uint8_t fl = valid ? A.flags[iq] : (uint8_t)0;
        const bool is_static = use_static && clean && valid && !(fl & FL_CHANGED) && A.nz[iq] <= 1;
        const int tq4 = TYPES ? 4 * (int)B.tp[kq] : 0;  // the agent's row of the type tables
        if (SPLIT && S >= 4 && valid && !is_static && sub < 3) {
          // this lane's axis of the agent's position, copied to shared memory
          // while the pairs are evaluated (waited for in the epilogue)
          const double *const gp = ((sub == 0) ? A.x[cur] : (sub == 1) ? A.y[cur] : A.z[cur]) + iq;
          const unsigned sa = (unsigned)__cvta_generic_to_shared(&s_pos[warp][lane]);
          asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gp) : "memory");
          asm volatile("cp.async.commit_group;\n" ::: "memory");
        }
        const bool compute = valid && !is_static;
        {
          // candidates tested in pass 0: the whole stencil for each computing agent
          const unsigned na = __popc(__ballot_sync(0xffffffffu, compute));
          if (lane == 0) s_ctr[warp][0] += ctot * (na / (unsigned)S);
        }
        float ffx = 0.f, ffy = 0.f, ffz = 0.f, gbound = 0.f, fscale = 0.f;
        double dfx = 0.0, dfy = 0.0, dfz = 0.0;
        unsigned ncont = 0, nnb = 0;
        long long lbase = 0;
        if (MODE == FM_LIST_NBR && valid) lbase = B.nbr_off[iq];
        {
          if (__any_sync(0xffffffffu, compute)) {
            // The warp stages its stencil's candidates in chunks of CHUNK
            // records in shared memory (coalesced copies, neighbour-box offset
            // applied once), every lane tests its share of the chunk in FP32
            // and queues the ones that may be neighbours, then the queued pairs
            // are evaluated with every lane busy.  Chunks follow the canonical
            // order and queues keep each lane's order, so the FP64 form keeps
            // the canonical summation order.
            float4 *const sc = s_c[warp];
            uint32_t *const skj = s_kj[warp];
            unsigned c0 = 0;
            while (true) {
              // ---- stage the next chunk: every lane locates its positions in
              // the stencil (binary search over the box prefix sums), so all
              // loads of a chunk are independent and in flight together
              const unsigned fill = (c0 < ctot) ? min((unsigned)CHUNK, ctot - c0) : 0u;
              constexpr int PER_LANE = (CHUNK + 31) / 32;
              unsigned kjs[PER_LANE];
              int boxs[PER_LANE];
#pragma unroll
              for (int m = 0; m < PER_LANE; ++m) {
                // branch-free binary search: last stencil box starting at or
                // before this chunk position (empty boxes are skipped because
                // the next box starts at the same position)
                const unsigned p = c0 + lane + 32u * m;
                int lo = 0;
#pragma unroll
                for (int step = 16; step > 0; step >>= 1)
                  if (s_pre[warp][lo + step] <= p) lo += step;
                boxs[m] = lo;
                kjs[m] = s_kb[warp][lo] + p;
                if (!BDM_IN(B.ctr, p >= ctot || (long long)kjs[m] < C->n)) kjs[m] = 0;
              }
              float4 cs[PER_LANE];
#pragma unroll
              for (int m = 0; m < PER_LANE; ++m)
                if (lane + 32u * m < fill) cs[m] = __ldg(&B.c32[kjs[m]]);
#pragma unroll
              for (int m = 0; m < PER_LANE; ++m) {
                const unsigned t = lane + 32u * m;
                if (t < fill) {
                  const float4 of = s_off[boxs[m]];
                  sc[t] = make_float4(cs[m].x + of.x, cs[m].y + of.y, cs[m].z + of.z, cs[m].w);
                  skj[t] = kjs[m];
                  if (TYPES) s_tp[warp][t] = B.tp[kjs[m]];
                }
              }
              c0 += fill;
              if (fill == 0) break;
              __syncwarp();
              // ---- test the chunk in FP32, queue the candidates inside the band
              unsigned qlen = 0;
              if (compute) {
                // the stride of 4 lanes per agent with constant offsets
                qlen = (S == 4) ? scan_chunk<4>(sc, &s_q[warp][0][lane], cq, (unsigned)sub, 4u, fill, P.R2_hi_f)
                                : scan_chunk<0>(sc, &s_q[warp][0][lane], cq, (unsigned)sub, (unsigned)S, fill,
                                                P.R2_hi_f);
              }
              // ---- evaluate the queued pairs
              if (PREC == 0 && (MODE == FM_STEP || MODE == FM_FORCES)) {
                // FP64 form: the warp evaluates the pooled queues of its lanes
                // 32 pairs at a time (every lane busy on the slow FP64 pipe),
                // writing each pair's terms to shared memory (aliasing the
                // staged FP32 records, which the FP64 pairs do not read); each
                // owner lane then adds its own pairs' terms in its queue order,
                // the canonical order, with the same IEEE operations as one
                // lane evaluating its queue.
                unsigned inc = qlen;
                for (int of = 1; of < 32; of <<= 1) {
                  const unsigned y = __shfl_up_sync(0xffffffffu, inc, of);
                  if (lane >= of) inc += y;
                }
                const unsigned tot = __shfl_sync(0xffffffffu, inc, 31), mine = inc - qlen;
                double *const tr = (double *)sc;               // [3][32] terms of a tile
                int *const rr = (int *)(tr + 96);              // [32] pair results
                uint32_t *const qs = (uint32_t *)(rr + 32);    // [32] pooled queue starts
                uint32_t *const kqs = qs + 32;                 // [32] the lanes' agents
                __syncwarp();
                qs[lane] = mine;
                kqs[lane] = kq;
                __syncwarp();
                for (unsigned t0 = 0; t0 < tot; t0 += 32) {
                  const unsigned e = t0 + (unsigned)lane;
                  double tx = 0.0, ty = 0.0, tz = 0.0;
                  int r = 0;
                  if (e < tot) {
                    int ow = 0;  // the lane whose queue holds pooled entry e
                    for (int st = 16; st > 0; st >>= 1)
                      if (ow + st < 32 && qs[ow + st] <= e) ow += st;
                    const unsigned kj = skj[s_q[warp][e - qs[ow]][ow]];
                    const unsigned ko = kqs[ow];
                    double kk = P.k, gg = P.gamma;
                    if (TYPES) {
                      const int ab = 4 * (int)B.tp[ko] + (int)B.tp[kj];
                      kk = s_tkd[ab];
                      gg = s_tgd[ab];
                    }
                    if (kj != ko) r = pair_f64_terms(P, kk, gg, B.c64[ko], B.c64[kj], tx, ty, tz);
                  }
                  __syncwarp();
                  tr[lane] = tx;
                  tr[32 + lane] = ty;
                  tr[64 + lane] = tz;
                  rr[lane] = r;
                  __syncwarp();
                  const unsigned lo = max(mine, t0), hi = min(mine + qlen, t0 + 32u);
                  for (unsigned u = lo; u < hi; ++u) {
                    const unsigned t = u - t0;
                    const int ru = rr[t];
                    nnb += (ru > 0);
                    if (ru == 2) {
                      ncont++;
                      dfx = __dadd_rn(dfx, tr[t]);
                      dfy = __dadd_rn(dfy, tr[32 + t]);
                      dfz = __dadd_rn(dfz, tr[64 + t]);
                    }
                  }
                  __syncwarp();
                }
                continue;
              }
              const unsigned mx = __reduce_max_sync(0xffffffffu, qlen);
              for (unsigned m = 0; m < mx; ++m) {
                if (m >= qlen) continue;
                const unsigned i = s_q[warp][m][lane];
                const unsigned kj = (PREC == 0) ? skj[i] : 0u;
                if (PREC == 0 && kj == kq) continue;  // the agent itself
                if (PREC == 0) {
                  const dbl4 cj = B.c64[kj];
                  if (MODE == FM_COUNT_NBR || MODE == FM_LIST_NBR) {
                    if (is_nbr_f64(P, dq, cj)) {
                      if (MODE == FM_LIST_NBR) B.nbr_out[lbase + nnb] = (long long)B.perm[kj];
                      nnb++;
                    }
                    continue;
                  }
                  const int ab = tq4 + (TYPES ? (int)B.tp[kj] : 0);
                  const int r = pair_f64_k(P.R2, TYPES ? s_tkd[ab] : P.k, TYPES ? s_tgd[ab] : P.gamma, dq, cj, dfx,
                                           dfy, dfz);
                  nnb += (r > 0);
                  ncont += (r == 2);
                  continue;
                }
                const float4 c = sc[i];
                const float ex = __fsub_rn(cq.x, c.x), ey = __fsub_rn(cq.y, c.y), ez = __fsub_rn(cq.z, c.z);
                const float d2 = fmaf(ex, ex, fmaf(ey, ey, __fmul_rn(ez, ez)));
                // the agent itself: its own staged record, at d2 = 0 exactly
                if (d2 < TINY2 && skj[i] == kq) continue;
                const bool band = (d2 > P.R2_lo_f) || (d2 < TINY2);
                if (MODE == FM_COUNT_NBR || MODE == FM_LIST_NBR) {
                  bool isn = true;
                  if (band && d2 > P.R2_lo_f) {
                    atomicAdd(&s_ctr[warp][3], 1u);
                    isn = is_nbr_f64(P, exact_of<1>(B, A, cur, kq), exact_of<1>(B, A, cur, skj[i]));
                  }
                  if (isn) {
                    if (MODE == FM_LIST_NBR) B.nbr_out[lbase + nnb] = (long long)B.perm[skj[i]];
                    nnb++;
                  }
                  continue;
                }
                const float s = __fadd_rn(cq.w, c.w), s2 = s * s;
                const float W = fmaf(s, P.cband1, s2 * P.cband2);
                const int ab = tq4 + (TYPES ? (int)s_tp[warp][i] : 0);
                const float kf = TYPES ? s_tkf[ab] : P.kf, gf = TYPES ? s_tgf[ab] : P.gammaf;
                bool exact = band || (d2 > s2 - W && d2 < s2 + W);  // cutoff or contact decided in FP64
                ContactF32 k = {};
                if (!exact) {
                  if (d2 >= s2 + W) {  // a neighbour, certainly no contact
                    nnb++;
                    continue;
                  }
                  k = contact_f32(d2, s, __fmul_rn(cq.w, c.w), kf, gf);
                  // from the exact geometry instead: a contact so shallow that
                  // gamma sqrt(rbar delta) is too steep for the FP32 overlap, or
                  // a pair so close that the FP32 rounding of its difference
                  // vector turns its direction too much
                  if (k.delta < P.graze_exact || d2 < P.close2) {
                    atomicAdd(&s_ctr[warp][3], 1u);
                    float tx, ty, tz;
                    fscale += contact_int(exact_of<1>(B, A, cur, kq), exact_of<1>(B, A, cur, skj[i]), P.fix_shift,
                                          kf, gf, tx, ty, tz);
                    ffx += tx; ffy += ty; ffz += tz;
                    nnb++;
                    ncont++;
                    continue;
                  }
                }
                if (exact) {
                  atomicAdd(&s_ctr[warp][3], 1u);
                  double gx = 0.0, gy = 0.0, gz = 0.0;
                  const int r = pair_f64_k(P.R2, TYPES ? s_tkd[ab] : P.k, TYPES ? s_tgd[ab] : P.gamma,
                                           exact_of<1>(B, A, cur, kq), exact_of<1>(B, A, cur, skj[i]), gx, gy, gz);
                  nnb += (r > 0);
                  if (r == 2) {
                    ncont++;
                    const float tx = (float)gx, ty = (float)gy, tz = (float)gz;
                    ffx += tx; ffy += ty; ffz += tz;
                    fscale += sqrtf(fmaf(tx, tx, fmaf(ty, ty, tz * tz)));
                  }
                  continue;
                }
                nnb++;
                const float delta = k.delta, rbar = k.rbar, sq = k.sq, fm = k.fm, scf = k.scf;
                ffx = fmaf(scf, ex, ffx);
                ffy = fmaf(scf, ey, ffy);
                ffz = fmaf(scf, ez, ffz);
                // error bound of a grazing contact: sqrt(rbar delta) is steep
                // in delta
                if (delta < P.graze)
                  gbound += (sq > 1e-18f) ? fminf(gf * rbar * P.graze_e * 0.5f * __frcp_rn(sq),
                                                  gf * sqrtf(rbar * P.graze_e))
                                          : gf * sqrtf(rbar * P.graze_e);
                fscale += fabsf(fm);
                ncont++;
              }
              __syncwarp();
            }
          }
          // reduce the S partial sums of an agent
          for (int of = S >> 1; of > 0; of >>= 1) {
            ffx += __shfl_xor_sync(0xffffffffu, ffx, of);
            ffy += __shfl_xor_sync(0xffffffffu, ffy, of);
            ffz += __shfl_xor_sync(0xffffffffu, ffz, of);
            ncont += __shfl_xor_sync(0xffffffffu, ncont, of);
            nnb += __shfl_xor_sync(0xffffffffu, nnb, of);
            if (PREC == 1) {
              gbound += __shfl_xor_sync(0xffffffffu, gbound, of);
              fscale += __shfl_xor_sync(0xffffffffu, fscale, of);
            }
          }
        }
        // FP32 form: the agent's tolerance is rel_tol * S + abs_tol, S =
        // fscale, the sum of its pair-force magnitudes.  When the bound of its
        // grazing contacts' FP32 error is not a small part of it, or S is so
        // small that the absolute floor dominates (S < low_scale: the
        // coordinates' rounding, about 1e-6 um per contact, is no longer
        // negligible), the agent goes to the FP64 fix-up pass, which
        // evaluates and finishes it.
        bool need_fix = false;
        if (PREC == 1 && (MODE == FM_STEP || MODE == FM_FORCES)) {
          need_fix = compute && ncont > 0 &&
                     (fscale < P.low_scale || gbound > 0.25f * (P.rel_tol * fscale + P.abs_tol));
          if (need_fix && sub == 0) {
            const unsigned long long e = atomicAdd(&C->fix_n, 1ull);
            if (BDM_IN(B.ctr, (long long)e < B.cap)) B.fix[e] = make_uint4(kq, (uint32_t)(o * 64 + lb), ncont, nnb);
          }
        }
        if (SPLIT && S >= 4) {
          // Lanes 0, 1 and 2 of the agent finish one axis each (one FP64
          // position addition, store and bounding-box update per lane),
          // with the same arithmetic as finish_agent's FP32 form.
          float ux, uy, uz;
          displacement_f32(P, dt_f, ffx, ffy, ffz, ux, uy, uz);
          if (valid && !is_static && sub < 3) asm volatile("cp.async.wait_all;\n" ::: "memory");
          const bool live = valid && !is_static && !need_fix && sub < 3;
          double p = 0.0, np = 0.0;
          if (live) {
            p = s_pos[warp][lane];
            const float u = (sub == 0) ? ux : (sub == 1) ? uy : uz;
            np = (u != 0.f) ? __dadd_rn(p, ftod_exact(u)) : p;
          }
          const unsigned mv = __ballot_sync(0xffffffffu, live && np != p);
          const bool moved = ((mv >> (lane - sub)) & 7u) != 0u;
          if (live) {
            if ((fl & FL_MOVED) || moved) ((sub == 0) ? A.x[nxt] : (sub == 1) ? A.y[nxt] : A.z[nxt])[iq] = np;
            if (P.keep_forces) B.fdbg[(size_t)sub * B.cap + iq] = ftod_exact((sub == 0) ? ffx : (sub == 1) ? ffy : ffz);
            atomicMin(&s_bb[warp][sub], enc_f64(np));
            atomicMax(&s_bb[warp][3 + sub], enc_f64(np));
            if (sub == 0) {
              c_moved += moved;
              A.nz[iq] = (uint16_t)min(ncont, 65535u);
              A.flags[iq] = moved ? (uint8_t)(FL_MOVED | FL_CHANGED) : (uint8_t)0;
            }
          }
          {
            const unsigned gn = __reduce_add_sync(0xffffffffu, (valid && sub == 0) ? nnb : 0u);
            const unsigned gc = __reduce_add_sync(0xffffffffu, (valid && sub == 0) ? ncont : 0u);
            if (lane == 0) { atomicAdd(&s_ctr[warp][1], gn); atomicAdd(&s_ctr[warp][2], gc); }
          }
          continue;
        }
        if (!valid || sub != 0) continue;
        atomicAdd(&s_ctr[warp][1], nnb);
        atomicAdd(&s_ctr[warp][2], ncont);
        if (MODE == FM_COUNT_NBR) { B.nbr_count[iq] = (int32_t)nnb; continue; }
        if (MODE == FM_LIST_NBR) continue;
        if (is_static) continue;  // finished by the static pass
        if (need_fix) continue;   // finished by the FP64 fix-up pass
        double px = 0.0, py = 0.0, pz = 0.0;
        if (MODE == FM_STEP) { px = A.x[cur][iq]; py = A.y[cur][iq]; pz = A.z[cur][iq]; }
        finish_agent<PREC, MODE>(B, P, A, cur, nxt, step, dt, dt_f, iq, fl, is_static, ffx, ffy, ffz, dfx, dfy, dfz,
                                 nnb, ncont, c_static, c_moved, s_bb[warp], px, py, pz);
      }
    }
  }
  if (MODE == FM_STEP) flush_bbox_warp(B, P, nxt, wsim, s_bb[warp]);
  __syncwarp();
  const unsigned long long t_static = wsum64(c_static), t_moved = wsum64(c_moved), t_cand = s_ctr[warp][0],
                           t_nbr = s_ctr[warp][1], t_cont = s_ctr[warp][2], t_exact = s_ctr[warp][3];
  if (lane == 0) {
    if (t_static) atomicAdd(&C->a_static, t_static);
    if (t_moved) atomicAdd(&C->a_moved, t_moved);
    if (t_cand) atomicAdd(&C->a_cand, t_cand);
    if (t_nbr) atomicAdd(&C->a_nbr, t_nbr);
    if (t_cont) atomicAdd(&C->a_contact, t_cont);
    if (t_exact) atomicAdd(&C->a_exact, t_exact);
  }
}

// ---------------------------------------------------------------- tiled FP32 force kernel
// FP32 form, FM_STEP and FM_FORCES (lanes = 0).  A warp takes a box and its
// agents in groups of up to 32 (lane a owns agent a of the group), stages the
// box's 27-box stencil in chunks of TCH candidate records (neighbour-box
// offset applied, as k_force stages them) and, per chunk:
//  1. tests every computing agent of the group against the chunk, lane t
//     holding candidates t and t + 32 in registers: the FP32 prefilter
//     d^2 < R2_hi of k_force, bit for bit.  One ballot per candidate slot
//     appends the passing (agent, candidate) pairs to the warp's pair list,
//     agent after agent, so that each agent's pairs are contiguous and in
//     candidate order;
//  2. evaluates the list 32 pairs per warp instruction with k_force's
//     decisions (FP32 outside the error bands, FP64 inside them) and its FP32
//     arithmetic, each lane writing its pair's force over the list entry;
//     the contacts whose FP32 force is not within the tolerance on their own
//     (|F| below low_scale, near the sign change of k delta - gamma
//     sqrt(rbar delta); grazing, delta < graze; close, d^2 < close2) go to a
//     second list that is evaluated in double-float arithmetic (contact_df),
//     again 32 pairs per warp instruction;
//  3. has each owner lane add its agent's segment of the list in list order
//     (summed per segment, then into the agent's total).
// Every test slot and every evaluation slot is a lane of work whatever the
// box's agent count.  Every contact's force is within the FP32 form's
// tolerance where it is formed, so no agent needs the fix-up pass.  The sums
// are deterministic (the same bits on every run), in a different order from
// k_force's.
#define TILE_WARPS 8
#define TCH 64    // candidates per staged chunk (2 per lane)
#define TPL 192   // entries of a warp's pair list (>= TCH: one agent's worst case)
template <int MODE, bool TYPES>
__global__ void __launch_bounds__(TILE_WARPS * 32, 4) k_force_tile(DevBufs B, DevParams P) {
  static_assert(MODE == FM_STEP || MODE == FM_FORCES, "the tiled kernel computes forces");
  __shared__ int s_nocc[27];
  __shared__ unsigned long long s_ndirty[27];
  __shared__ int s_next;
  __shared__ unsigned s_bcnt[64];
  __shared__ uint8_t s_order[64];
  __shared__ unsigned long long s_need;
  __shared__ long long s_o;
  __shared__ unsigned s_ctr[TILE_WARPS][4];  // candidates, neighbours, contacts, exact pairs
  __shared__ float4 s_off[27];
  __shared__ unsigned long long s_bb[TILE_WARPS][6];
  __shared__ unsigned s_pre[TILE_WARPS][32], s_kb[TILE_WARPS][32];
  __shared__ float4 s_own[TILE_WARPS][32];          // the group's agents' FP32 records
  __shared__ uint8_t s_otp[TILE_WARPS][32];         // TYPES: their types
  __shared__ float4 s_c[TILE_WARPS][TCH];           // the staged chunk (offset applied)
  __shared__ uint32_t s_kj[TILE_WARPS][TCH];        // its sorted positions
  __shared__ uint8_t s_tp[TILE_WARPS][TCH];         // TYPES: its types
  __shared__ float4 s_rec[TILE_WARPS][TPL];         // the pair list: entry, then result
  __shared__ uint16_t s_dfl[TILE_WARPS][TPL];       // its contacts for the double-float pass
  __shared__ float s_tkf[16], s_tgf[16];
  __shared__ double s_tkd[16], s_tgd[16];
  __shared__ DF s_tk2[16], s_tg2[16];
  DevCounters *C = B.ctr;
  if (C->error) return;
  const AgentSet A = *B.A;
  const int cur = (int)(C->step & 1), nxt = cur ^ 1;
  const bool use_static = (MODE == FM_STEP) && P.detect_static && C->history_valid;
  const long long n_occ = C->n_occ;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const long long step = C->step;
  unsigned c_static = 0, c_moved = 0;
  int wsim = -1;
  int fetch_phase = 0;
  if (threadIdx.x < 27) {
    const int t = threadIdx.x;
    s_off[t] = make_float4((float)(t % 3 - 1) * P.Lf, (float)((t / 3) % 3 - 1) * P.Lf, (float)(t / 9 - 1) * P.Lf, 0.f);
  }
  if (lane < 6) s_bb[warp][lane] = (lane < 3) ? ~0ull : 0ull;
  if (lane < 4) s_ctr[warp][lane] = 0u;
  if (threadIdx.x < 16) {  // one type: every entry holds k and gamma
    s_tkd[threadIdx.x] = P.type_k[threadIdx.x];
    s_tgd[threadIdx.x] = P.type_gamma[threadIdx.x];
    s_tkf[threadIdx.x] = (float)P.type_k[threadIdx.x];
    s_tgf[threadIdx.x] = (float)P.type_gamma[threadIdx.x];
    const float kh = (float)P.type_k[threadIdx.x], gh = (float)P.type_gamma[threadIdx.x];
    s_tk2[threadIdx.x] = {kh, (float)(P.type_k[threadIdx.x] - (double)kh)};
    s_tg2[threadIdx.x] = {gh, (float)(P.type_gamma[threadIdx.x] - (double)gh)};
  }
  // a staged slot past the chunk's end: a record no agent is near
  const float4 far = make_float4(3.0e38f, 3.0e38f, 3.0e38f, 0.f);

  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) {
      s_o = next_force_brick(B, P, C, n_occ, fetch_phase, use_static);
      s_next = 0;
    }
    __syncthreads();
    const long long o = s_o;
    if (o < 0) break;
    if (!BDM_IN(B.ctr, o < n_occ)) break;  // block-uniform
    const int4 info = B.occ_info[o];
    const SimGeom &G = B.geom[info.w];
    if (threadIdx.x < 27) {
      const int t = threadIdx.x;
      const int X = info.x + t % 3 - 1, Y = info.y + (t / 3) % 3 - 1, Z = info.z + t / 9 - 1;
      int occ = -1;
      unsigned long long dm = 0ull;
      if (X >= 0 && X < G.nr[0] && Y >= 0 && Y < G.nr[1] && Z >= 0 && Z < G.nr[2]) {
        const int rank = B.brick_table[G.brick_base + ((long long)Z * G.nr[1] + Y) * G.nr[0] + X];
        occ = B.brick_occ[rank];
        if (use_static) dm = B.dirty[rank];
      }
      s_nocc[t] = occ;
      s_ndirty[t] = dm;
    }
    if (threadIdx.x >= 64 && threadIdx.x < 128) s_bcnt[threadIdx.x - 64] = B.box_cnt[o * 64 + threadIdx.x - 64];
    if (threadIdx.x == 32) s_need = use_static ? B.need[o] : ~0ull;
    __syncthreads();
    if (MODE == FM_STEP && info.w != wsim) {
      flush_bbox_warp(B, P, nxt, wsim, s_bb[warp]);
      wsim = info.w;
    }
    const double dt = G.dt;
    const float dt_f = G.dt_f;
    // boxes heaviest first (ties by box index)
    if (threadIdx.x < 64) {
      const unsigned c = s_bcnt[threadIdx.x];
      unsigned r = 0;
      for (int q = 0; q < 64; ++q) {
        const unsigned cq = s_bcnt[q];
        r += (cq > c) || (cq == c && q < (int)threadIdx.x);
      }
      s_order[r] = (uint8_t)threadIdx.x;
    }
    __syncthreads();

    while (true) {
      int kb = 0;
      if (lane == 0) kb = atomicAdd(&s_next, 1);
      kb = __shfl_sync(0xffffffffu, kb, 0);
      if (kb >= 64) break;
      const int lb = s_order[kb];
      if (!((s_need >> lb) & 1ull)) continue;  // nothing left after the static pass
      const unsigned qbase = B.box_start[o * 64 + lb], nq = B.box_cnt[o * 64 + lb];
      if (nq == 0) continue;
      int lx, ly, lz;
      local_decode(lb, lx, ly, lz);
      unsigned nb_st = 0, nb_cnt = 0;
      bool nb_dirty = false;
      if (lane < 27) {
        const int ax = lx + lane % 3 - 1, ay = ly + (lane / 3) % 3 - 1, az = lz + lane / 9 - 1;
        const int bo = ((az < 0) ? 0 : (az > 3 ? 2 : 1)) * 9 + ((ay < 0) ? 0 : (ay > 3 ? 2 : 1)) * 3 +
                       ((ax < 0) ? 0 : (ax > 3 ? 2 : 1));
        const int lc = local_code(ax & 3, ay & 3, az & 3);
        const int occ = s_nocc[bo];
        if (occ >= 0) {
          nb_st = B.box_start[(long long)occ * 64 + lc];
          nb_cnt = B.box_cnt[(long long)occ * 64 + lc];
        }
        nb_dirty = (s_ndirty[bo] >> lc) & 1ull;
      }
      const bool clean = !__any_sync(0xffffffffu, nb_dirty);
      unsigned pre = nb_cnt;
      for (int of = 1; of < 32; of <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, pre, of);
        if (lane >= of) pre += y;
      }
      const unsigned ctot = __shfl_sync(0xffffffffu, pre, 31);
      // box starts in the stencil (s_pre[27] = ctot, then UINT_MAX: the
      // staging's search needs no range test) and each box's first sorted
      // position minus its start
      s_pre[warp][lane] = (lane <= 27) ? pre - nb_cnt : 0xFFFFFFFFu;
      s_kb[warp][lane] = nb_st - (pre - nb_cnt);
      __syncwarp();
      for (unsigned q0 = 0; q0 < nq; q0 += 32) {
        const unsigned qi = q0 + (unsigned)lane;
        bool valid = qi < nq;
        unsigned kq = qbase + (valid ? qi : 0u);
        if (!BDM_IN(B.ctr, (long long)kq < C->n)) { kq = 0; valid = false; }
        uint32_t iq = B.perm[kq];
        if (!BDM_IN(B.ctr, (long long)iq < B.cap)) { iq = 0; valid = false; }
        const float4 cq = B.c32[kq];
        const uint8_t fl = valid ? A.flags[iq] : (uint8_t)0;
        const bool is_static = use_static && clean && valid && !(fl & FL_CHANGED) && A.nz[iq] <= 1;
        const bool compute = valid && !is_static;
        const unsigned cmask = __ballot_sync(0xffffffffu, compute);
        __syncwarp();  // the previous group's readers of s_own are done
        s_own[warp][lane] = cq;
        if (TYPES) s_otp[warp][lane] = B.tp[kq];
        if (lane == 0) s_ctr[warp][0] += ctot * (unsigned)__popc(cmask);
        float ffx = 0.f, ffy = 0.f, ffz = 0.f;  // this lane's agent's force
        unsigned ncont = 0, nnb = 0;
        unsigned my_lo = 0, my_hi = 0;  // this lane's agent's segment of the list
        __syncwarp();
        for (unsigned c0 = 0; cmask != 0u && c0 < ctot; c0 += TCH) {
          // ---- stage the chunk: each lane locates its two positions in the
          // stencil (binary search over the box prefix sums), loads them, and
          // keeps them in registers for the test
          float4 cr[2];
          {
            unsigned kjs[2];
            int boxs[2];
#pragma unroll
            for (int m = 0; m < 2; ++m) {
              const unsigned p = c0 + (unsigned)lane + 32u * m;
              int lo = 0;
#pragma unroll
              for (int st = 16; st > 0; st >>= 1)
                if (s_pre[warp][lo + st] <= p) lo += st;
              boxs[m] = lo;
              kjs[m] = s_kb[warp][lo] + p;
              if (!BDM_IN(B.ctr, p >= ctot || (long long)kjs[m] < C->n)) kjs[m] = 0;
            }
            float4 cs[2];
#pragma unroll
            for (int m = 0; m < 2; ++m)
              if (c0 + (unsigned)lane + 32u * m < ctot) cs[m] = __ldg(&B.c32[kjs[m]]);
#pragma unroll
            for (int m = 0; m < 2; ++m) {
              const unsigned t = (unsigned)lane + 32u * m;
              cr[m] = far;
              if (c0 + t < ctot) {
                const float4 of = s_off[boxs[m]];
                cr[m] = make_float4(cs[m].x + of.x, cs[m].y + of.y, cs[m].z + of.z, cs[m].w);
                s_c[warp][t] = cr[m];
                s_kj[warp][t] = kjs[m];
                if (TYPES) s_tp[warp][t] = B.tp[kjs[m]];
              }
            }
          }
          unsigned am = cmask;  // agents still to test against this chunk
          while (true) {
            // ---- test agents until the list could overflow
            unsigned base = 0;
            while (am != 0u && base + TCH <= TPL) {
              const int a = __ffs(am) - 1;
              am &= am - 1u;
              const float4 qa = s_own[warp][a];
              const bool p0 = dist2_f32(qa, cr[0]) < P.R2_hi_f;
              const bool p1 = dist2_f32(qa, cr[1]) < P.R2_hi_f;
              const unsigned b0 = __ballot_sync(0xffffffffu, p0), b1 = __ballot_sync(0xffffffffu, p1);
              const unsigned n0 = __popc(b0);
              const unsigned tag = ((unsigned)a << 8) | (unsigned)lane;
              if (p0) reinterpret_cast<unsigned &>(s_rec[warp][base + __popc(b0 & lt)].x) = tag;
              if (p1) reinterpret_cast<unsigned &>(s_rec[warp][base + n0 + __popc(b1 & lt)].x) = tag + 32u;
              if (lane == a) my_lo = base;
              base += n0 + __popc(b1);
              if (lane == a) my_hi = base;
            }
            __syncwarp();
            // ---- evaluate the list, 32 pairs per warp instruction
            unsigned ndf = 0;  // contacts listed for the double-float pass
            for (unsigned p0 = 0; p0 < base; p0 += 32u) {
              const unsigned e = p0 + (unsigned)lane;
              int r = 0;  // 0: no neighbour, 1: neighbour without force, 2: contact
              bool risky = false;
              if (e < base) {
                const unsigned ent = reinterpret_cast<const unsigned &>(s_rec[warp][e].x);
                const int a = (int)(ent >> 8);
                const unsigned t = ent & 255u;
                const unsigned kqa = qbase + q0 + (unsigned)a;
                const unsigned kj = s_kj[warp][t];
                float4 res = make_float4(0.f, 0.f, 0.f, 0.f);  // force on agent a
                if (kj != kqa) {
                  const float4 qa = s_own[warp][a];
                  const float4 c = s_c[warp][t];
                  const float ex = __fsub_rn(qa.x, c.x), ey = __fsub_rn(qa.y, c.y), ez = __fsub_rn(qa.z, c.z);
                  const float d2 = fmaf(ex, ex, fmaf(ey, ey, __fmul_rn(ez, ez)));
                  const bool band = (d2 > P.R2_lo_f) || (d2 < TINY2);
                  const float s = __fadd_rn(qa.w, c.w), s2 = s * s;
                  const float W = fmaf(s, P.cband1, s2 * P.cband2);
                  const int ab = TYPES ? 4 * (int)s_otp[warp][a] + (int)s_tp[warp][t] : 0;
                  const float kf = TYPES ? s_tkf[ab] : P.kf, gf = TYPES ? s_tgf[ab] : P.gammaf;
                  const bool exact = band || (d2 > s2 - W && d2 < s2 + W);  // cutoff or contact in FP64
                  if (!exact && d2 >= s2 + W) {
                    r = 1;  // a neighbour, certainly no contact
                  } else if (!exact) {
                    r = 2;
                    const ContactF32 k = contact_f32(d2, s, __fmul_rn(qa.w, c.w), kf, gf);
                    // a contact whose FP32 force is not within the tolerance on
                    // its own: near the sign change of F (|F| < low_scale),
                    // grazing (delta < graze: sqrt(rbar delta) is steep in
                    // delta) or close (d^2 < close2: the direction); it keeps
                    // its list entry for the double-float pass
                    risky = fabsf(k.fm) < P.low_scale || k.delta < P.graze || d2 < P.close2;
                    res = make_float4(__fmul_rn(k.scf, ex), __fmul_rn(k.scf, ey), __fmul_rn(k.scf, ez), 0.f);
                  } else {
                    atomicAdd(&s_ctr[warp][3], 1u);
                    double gx = 0.0, gy = 0.0, gz = 0.0;
                    r = pair_f64_k(P.R2, TYPES ? s_tkd[ab] : P.k, TYPES ? s_tgd[ab] : P.gamma,
                                   exact_of<1>(B, A, cur, kqa), exact_of<1>(B, A, cur, kj), gx, gy, gz);
                    if (r == 2) res = make_float4((float)gx, (float)gy, (float)gz, 0.f);
                  }
                }
                if (!risky) s_rec[warp][e] = res;
              }
              {
                const unsigned bd = __ballot_sync(0xffffffffu, risky);
                if (risky) s_dfl[warp][ndf + __popc(bd & lt)] = (uint16_t)e;
                ndf += __popc(bd);
              }
              // this window's neighbours and contacts of each owner's agent
              const unsigned bn = __ballot_sync(0xffffffffu, r > 0), bc = __ballot_sync(0xffffffffu, r == 2);
              if (my_hi > p0 && my_lo < p0 + 32u) {
                const unsigned lo = (my_lo > p0 ? my_lo : p0) - p0, hi = (my_hi < p0 + 32u ? my_hi : p0 + 32u) - p0;
                const unsigned msk = ((hi == 32u) ? 0xffffffffu : ((1u << hi) - 1u)) & ~((1u << lo) - 1u);
                nnb += __popc(bn & msk);
                ncont += __popc(bc & msk);
              }
            }
            __syncwarp();
            // ---- the listed contacts in double-float (contact_df), 32 per
            // warp instruction; each result replaces its entry
            for (unsigned d0 = 0; d0 < ndf; d0 += 32u) {
              if (d0 + (unsigned)lane < ndf) {
                const unsigned e = s_dfl[warp][d0 + lane];
                const unsigned ent = reinterpret_cast<const unsigned &>(s_rec[warp][e].x);
                const int a = (int)(ent >> 8);
                const unsigned t = ent & 255u;
                const int ab = TYPES ? 4 * (int)s_otp[warp][a] + (int)s_tp[warp][t] : 0;
                float4 res = make_float4(0.f, 0.f, 0.f, 0.f);
                contact_df(P, exact_of<1>(B, A, cur, qbase + q0 + (unsigned)a), exact_of<1>(B, A, cur, s_kj[warp][t]),
                           s_tk2[ab], s_tg2[ab], res.x, res.y, res.z);
                s_rec[warp][e] = res;
              }
            }
            if (lane == 0 && ndf) s_ctr[warp][3] += ndf;
            __syncwarp();
            // ---- each owner sums its agent's segment in list order, then
            // adds that sum to the agent's (a two-level sum: the rounding of
            // a long sequential sum of large, cancelling pair forces is what
            // a dense cluster would feel)
            {
              float sx = 0.f, sy = 0.f, sz = 0.f;
              for (unsigned u = my_lo; u < my_hi; ++u) {
                const float4 v = s_rec[warp][u];
                sx += v.x;
                sy += v.y;
                sz += v.z;
              }
              ffx += sx;
              ffy += sy;
              ffz += sz;
            }
            my_lo = my_hi = 0;
            __syncwarp();
            if (am == 0u) break;
          }
        }
        // ---- per agent: the epilogue
        {
          const unsigned gn = __reduce_add_sync(0xffffffffu, valid ? nnb : 0u);
          const unsigned gc = __reduce_add_sync(0xffffffffu, valid ? ncont : 0u);
          if (lane == 0) { s_ctr[warp][1] += gn; s_ctr[warp][2] += gc; }
        }
        if (!compute) continue;  // static agents: finished by the static pass
        double px = 0.0, py = 0.0, pz = 0.0;
        if (MODE == FM_STEP) { px = A.x[cur][iq]; py = A.y[cur][iq]; pz = A.z[cur][iq]; }
        finish_agent<1, MODE>(B, P, A, cur, nxt, step, dt, dt_f, iq, fl, false, ffx, ffy, ffz, 0.0, 0.0, 0.0, nnb,
                              ncont, c_static, c_moved, s_bb[warp], px, py, pz);
      }
    }
  }
  if (MODE == FM_STEP) flush_bbox_warp(B, P, nxt, wsim, s_bb[warp]);
  __syncwarp();
  const unsigned long long t_static = wsum64(c_static), t_moved = wsum64(c_moved), t_cand = s_ctr[warp][0],
                           t_nbr = s_ctr[warp][1], t_cont = s_ctr[warp][2], t_exact = s_ctr[warp][3];
  if (lane == 0) {
    if (t_static) atomicAdd(&C->a_static, t_static);
    if (t_moved) atomicAdd(&C->a_moved, t_moved);
    if (t_cand) atomicAdd(&C->a_cand, t_cand);
    if (t_nbr) atomicAdd(&C->a_nbr, t_nbr);
    if (t_cont) atomicAdd(&C->a_contact, t_cont);
    if (t_exact) atomicAdd(&C->a_exact, t_exact);
  }
}

// ---------------------------------------------------------------- sparse FP32 force kernel
// FP32 form, FM_STEP and FM_FORCES (lanes = -3), for sparse tissue: boxes of
// one to a few agents (a shell around a static core, the small simulations of
// an ensemble), where the per-box work of the box-per-warp kernels (stencil
// set-up, staging, lists) is shared by too few agents.  One warp per occupied
// brick (heaviest first, the static pass's work list as in k_force; no block
// barriers); its lanes take the agents of the brick's boxes with work one per
// lane, in rounds of 32, and each lane walks its own agent's 27-box stencil in
// the canonical order,
// testing every candidate with k_force's FP32 prefilter and deciding
// neighbour and contact exactly as k_force does (FP32 outside the error
// bands, FP64 in place inside them).  A contact the FP32 error analysis covers
// is added in place; the others (|F| < low_scale, delta < graze, d^2 < close2)
// are queued per lane and evaluated by the warp in double-float (contact_df),
// 32 pairs per warp instruction, after each round; the owner lane adds their
// results in its queue order.  A lane whose queue is full evaluates the contact
// itself.  No agent is listed for the fix-up pass.
#define SP_WARPS 4
#define SP_Q 4    // double-float contacts a lane queues per round
template <int MODE, bool TYPES>
__global__ void __launch_bounds__(SP_WARPS * 32, 8) k_force_sparse(DevBufs B, DevParams P) {
  static_assert(MODE == FM_STEP || MODE == FM_FORCES, "the sparse kernel computes forces");
  // per warp: its brick's 27 neighbour bricks (occupied index, dirty mask),
  // box starts (and end), and the agents of boxes with work before each box
  __shared__ int s_nocc[SP_WARPS][27];
  __shared__ unsigned long long s_ndirty[SP_WARPS][27];
  __shared__ unsigned s_bst[SP_WARPS][65];
  // and the first sorted position and agent count of each box of the 6 x 6 x 6
  // region around the brick (local box coordinates -1..4)
  __shared__ unsigned s_rst[SP_WARPS][216], s_rcnt[SP_WARPS][216];
  __shared__ float4 s_off[27];
  __shared__ unsigned long long s_bb[SP_WARPS][6];
  __shared__ uint32_t s_dq[SP_WARPS][SP_Q][32];   // each lane's queued candidates (sorted positions)
  __shared__ float4 s_dr[SP_WARPS][SP_Q][32];     // and their double-float forces
  __shared__ uint32_t s_dk[SP_WARPS][32];         // each lane's agent (sorted position)
  __shared__ unsigned s_ncum[SP_WARPS][65];
  __shared__ float s_tkf[16], s_tgf[16];
  __shared__ double s_tkd[16], s_tgd[16];
  __shared__ DF s_tk2[16], s_tg2[16];
  DevCounters *C = B.ctr;
  if (C->error) return;
  const AgentSet A = *B.A;
  const int cur = (int)(C->step & 1), nxt = cur ^ 1;
  const bool use_static = (MODE == FM_STEP) && P.detect_static && C->history_valid;
  const long long n_occ = C->n_occ;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long step = C->step;
  unsigned c_static = 0, c_moved = 0;
  int wsim = -1;
  int fetch_phase = 0;
  if (threadIdx.x < 27) {
    const int t = threadIdx.x;
    s_off[t] = make_float4((float)(t % 3 - 1) * P.Lf, (float)((t / 3) % 3 - 1) * P.Lf, (float)(t / 9 - 1) * P.Lf, 0.f);
  }
  if (lane < 6) s_bb[warp][lane] = (lane < 3) ? ~0ull : 0ull;
  if (threadIdx.x < 16) {  // one type: every entry holds k and gamma
    s_tkd[threadIdx.x] = P.type_k[threadIdx.x];
    s_tgd[threadIdx.x] = P.type_gamma[threadIdx.x];
    s_tkf[threadIdx.x] = (float)P.type_k[threadIdx.x];
    s_tgf[threadIdx.x] = (float)P.type_gamma[threadIdx.x];
    const float kh = (float)P.type_k[threadIdx.x], gh = (float)P.type_gamma[threadIdx.x];
    s_tk2[threadIdx.x] = {kh, (float)(P.type_k[threadIdx.x] - (double)kh)};
    s_tg2[threadIdx.x] = {gh, (float)(P.type_gamma[threadIdx.x] - (double)gh)};
  }
  unsigned n_cand = 0, n_nbr = 0, n_cont = 0, n_exact = 0;  // this thread's statistics

  __syncthreads();  // the block's tables are written
  // one brick per warp (taken from the global brick order): no block barriers,
  // so a warp on a brick with few agents to compute does not hold the others
  while (true) {
    long long o = 0;
    if (lane == 0) o = next_force_brick(B, P, C, n_occ, fetch_phase, use_static);
    o = __shfl_sync(0xffffffffu, o, 0);
    if (o < 0) break;
    if (!BDM_IN(B.ctr, o < n_occ)) break;  // warp-uniform
    const int4 info = B.occ_info[o];
    const SimGeom &G = B.geom[info.w];
    __syncwarp();  // the previous brick's readers of the warp's tables are done
    if (lane < 27) {
      const int X = info.x + lane % 3 - 1, Y = info.y + (lane / 3) % 3 - 1, Z = info.z + lane / 9 - 1;
      int occ = -1;
      unsigned long long dm = 0ull;
      if (X >= 0 && X < G.nr[0] && Y >= 0 && Y < G.nr[1] && Z >= 0 && Z < G.nr[2]) {
        const int rank = B.brick_table[G.brick_base + ((long long)Z * G.nr[1] + Y) * G.nr[0] + X];
        occ = B.brick_occ[rank];
        if (use_static) dm = B.dirty[rank];
      }
      s_nocc[warp][lane] = occ;
      s_ndirty[warp][lane] = dm;
    }
    s_bst[warp][lane] = B.box_start[o * 64 + lane];
    s_bst[warp][lane + 32] = B.box_start[o * 64 + lane + 32];
    if (lane == 0) s_bst[warp][64] = B.box_start[o * 64 + 63] + B.box_cnt[o * 64 + 63];
    const unsigned long long need = use_static ? B.need[o] : ~0ull;  // boxes with work
    __syncwarp();
    for (int rb = lane; rb < 216; rb += 32) {
      const int ax = rb % 6 - 1, ay = (rb / 6) % 6 - 1, az = rb / 36 - 1;
      const int bo = ((az < 0) ? 0 : (az > 3 ? 2 : 1)) * 9 + ((ay < 0) ? 0 : (ay > 3 ? 2 : 1)) * 3 +
                     ((ax < 0) ? 0 : (ax > 3 ? 2 : 1));
      const int occ = s_nocc[warp][bo];
      unsigned st = 0, cnt = 0;
      if (occ >= 0) {
        const long long bx = (long long)occ * 64 + local_code(ax & 3, ay & 3, az & 3);
        st = B.box_start[bx];
        cnt = B.box_cnt[bx];
      }
      s_rst[warp][rb] = st;
      s_rcnt[warp][rb] = cnt;
    }
    // boxes with a clean stencil (no dirty box in it)
    unsigned long long clean = 0ull;
    if (use_static) {
      const bool c0 = !stencil_dirty(s_ndirty[warp], lane), c1 = !stencil_dirty(s_ndirty[warp], lane + 32);
      clean = (unsigned long long)__ballot_sync(0xffffffffu, c0) |
              ((unsigned long long)__ballot_sync(0xffffffffu, c1) << 32);
    }
    {
      // exclusive prefix of the agent counts of the boxes with work (two
      // boxes per lane)
      const int l2 = 2 * lane;
      const unsigned a0 = ((need >> l2) & 1ull) ? s_bst[warp][l2 + 1] - s_bst[warp][l2] : 0u;
      const unsigned a1 = ((need >> (l2 + 1)) & 1ull) ? s_bst[warp][l2 + 2] - s_bst[warp][l2 + 1] : 0u;
      unsigned inc = a0 + a1;
      for (int of = 1; of < 32; of <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, inc, of);
        if (lane >= of) inc += y;
      }
      s_ncum[warp][l2] = inc - a0 - a1;
      s_ncum[warp][l2 + 1] = inc - a1;
      if (lane == 31) s_ncum[warp][64] = inc;
    }
    __syncwarp();
    if (MODE == FM_STEP && info.w != wsim) {
      flush_bbox_warp(B, P, nxt, wsim, s_bb[warp]);
      wsim = info.w;
    }
    const double dt = G.dt;
    const float dt_f = G.dt_f;
    const unsigned nw = s_ncum[warp][64];  // agents of the brick's boxes with work
    // rounds of one agent per lane (warp-uniform trip count)
    for (unsigned r0 = 0; r0 < nw; r0 += 32u) {
      const unsigned i = r0 + (unsigned)lane;
      bool valid = i < nw;
      int lb = 0;  // the agent's box: the last box with work whose first agent is at or before i
#pragma unroll
      for (int st = 32; st > 0; st >>= 1)
        if (lb + st < 64 && s_ncum[warp][lb + st] <= i) lb += st;
      const unsigned kq = valid ? s_bst[warp][lb] + (i - s_ncum[warp][lb]) : s_bst[warp][0];
      if (!BDM_IN(B.ctr, !valid || (long long)kq < C->n)) valid = false;
      uint32_t iq = valid ? B.perm[kq] : 0u;
      if (!BDM_IN(B.ctr, (long long)iq < B.cap)) { iq = 0; valid = false; }
      const uint8_t fl = valid ? A.flags[iq] : (uint8_t)0;
      const bool is_static = use_static && valid && ((clean >> lb) & 1ull) && !(fl & FL_CHANGED) && A.nz[iq] <= 1;
      const bool compute = valid && !is_static;
      const float4 cq = B.c32[kq];
      const int tq4 = TYPES ? 4 * (int)B.tp[kq] : 0;
      s_dk[warp][lane] = kq;
      float ffx = 0.f, ffy = 0.f, ffz = 0.f;
      unsigned nnb = 0, ncont = 0, nq = 0;
      if (compute) {
        int lx, ly, lz;
        local_decode(lb, lx, ly, lz);
        for (int sb = 0; sb < 27; ++sb) {
          const int rb = (lx + sb % 3) + 6 * (ly + (sb / 3) % 3) + 36 * (lz + sb / 9);
          const unsigned st = s_rst[warp][rb], cnt = s_rcnt[warp][rb];
          n_cand += cnt;
          const float4 of = s_off[sb];
          for (unsigned j = 0; j < cnt; ++j) {
            const unsigned kj = st + j;
            if (!BDM_IN(B.ctr, (long long)kj < C->n)) break;
            const float4 cs = __ldg(&B.c32[kj]);
            const float4 c = make_float4(cs.x + of.x, cs.y + of.y, cs.z + of.z, cs.w);
            const float d2 = dist2_f32(cq, c);
            if (!(d2 < P.R2_hi_f) || kj == kq) continue;
            const bool band = (d2 > P.R2_lo_f) || (d2 < TINY2);
            const float s = __fadd_rn(cq.w, c.w), s2 = s * s;
            const float W = fmaf(s, P.cband1, s2 * P.cband2);
            if (!band && d2 >= s2 + W) {  // a neighbour, certainly no contact
              nnb++;
              continue;
            }
            const int ab = tq4 + (TYPES ? (int)B.tp[kj] : 0);
            if (band || d2 > s2 - W) {  // cutoff or contact undecided in FP32: FP64
              n_exact++;
              double gx = 0.0, gy = 0.0, gz = 0.0;
              const int r = pair_f64_k(P.R2, TYPES ? s_tkd[ab] : P.k, TYPES ? s_tgd[ab] : P.gamma,
                                       exact_of<1>(B, A, cur, kq), exact_of<1>(B, A, cur, kj), gx, gy, gz);
              nnb += (r > 0);
              ncont += (r == 2);
              if (r == 2) { ffx += (float)gx; ffy += (float)gy; ffz += (float)gz; }
              continue;
            }
            nnb++;
            ncont++;
            const float kf = TYPES ? s_tkf[ab] : P.kf, gf = TYPES ? s_tgf[ab] : P.gammaf;
            const ContactF32 k = contact_f32(d2, s, __fmul_rn(cq.w, c.w), kf, gf);
            if (fabsf(k.fm) < P.low_scale || k.delta < P.graze || d2 < P.close2) {
              // not covered by the FP32 error analysis: double-float, queued
              // for the warp (or here when the queue is full)
              n_exact++;
              if (nq < SP_Q) {
                s_dq[warp][nq][lane] = kj;
                nq++;
              } else {
                float tx, ty, tz;
                contact_df(P, exact_of<1>(B, A, cur, kq), exact_of<1>(B, A, cur, kj), s_tk2[ab], s_tg2[ab], tx, ty,
                           tz);
                ffx += tx; ffy += ty; ffz += tz;
              }
              continue;
            }
            ffx = fmaf(k.scf, __fsub_rn(cq.x, c.x), ffx);
            ffy = fmaf(k.scf, __fsub_rn(cq.y, c.y), ffy);
            ffz = fmaf(k.scf, __fsub_rn(cq.z, c.z), ffz);
          }
        }
      }
      // ---- the warp's queued contacts in double-float, 32 per warp
      // instruction (lanes' queues pooled in lane order), then each owner
      // adds its own in its queue order
      {
        unsigned inc = nq;
        for (int of = 1; of < 32; of <<= 1) {
          const unsigned y = __shfl_up_sync(0xffffffffu, inc, of);
          if (lane >= of) inc += y;
        }
        const unsigned tot = __shfl_sync(0xffffffffu, inc, 31);
        if (tot) {
          __syncwarp();  // the lanes' queues and agents are written
          const unsigned mine = inc - nq;
          // pooled entry e belongs to the last lane whose first entry is <= e
          // (a lane without entries starts where the next one does)
          for (unsigned t0 = 0; t0 < tot; t0 += 32u) {
            const unsigned e = t0 + (unsigned)lane;
            int ow = 0;
            for (int of = 16; of > 0; of >>= 1) {
              const unsigned so = __shfl_sync(0xffffffffu, mine, ow + of);
              if (so <= e) ow += of;
            }
            const unsigned sow = __shfl_sync(0xffffffffu, mine, ow);
            if (e < tot) {
              const unsigned sl = e - sow;
              const unsigned kj = s_dq[warp][sl][ow], kqo = s_dk[warp][ow];
              const int ab = TYPES ? 4 * (int)B.tp[kqo] + (int)B.tp[kj] : 0;
              float4 rr = make_float4(0.f, 0.f, 0.f, 0.f);
              contact_df(P, exact_of<1>(B, A, cur, kqo), exact_of<1>(B, A, cur, kj), s_tk2[ab], s_tg2[ab], rr.x, rr.y,
                         rr.z);
              s_dr[warp][sl][ow] = rr;
            }
          }
          __syncwarp();
          for (unsigned u = 0; u < nq; ++u) {
            const float4 v = s_dr[warp][u][lane];
            ffx += v.x;
            ffy += v.y;
            ffz += v.z;
          }
          __syncwarp();
        }
      }
      if (valid) { n_nbr += nnb; n_cont += ncont; }
      if (!compute) continue;  // static agents: finished by the static pass
      double px = 0.0, py = 0.0, pz = 0.0;
      if (MODE == FM_STEP) { px = A.x[cur][iq]; py = A.y[cur][iq]; pz = A.z[cur][iq]; }
      finish_agent<1, MODE>(B, P, A, cur, nxt, step, dt, dt_f, iq, fl, false, ffx, ffy, ffz, 0.0, 0.0, 0.0, nnb,
                            ncont, c_static, c_moved, s_bb[warp], px, py, pz);
    }
  }
  if (MODE == FM_STEP) flush_bbox_warp(B, P, nxt, wsim, s_bb[warp]);
  __syncwarp();
  const unsigned long long t_moved = wsum64(c_moved), t_cand = wsum64(n_cand), t_nbr = wsum64(n_nbr),
                           t_cont = wsum64(n_cont), t_exact = wsum64(n_exact);
  if (lane == 0) {
    if (t_moved) atomicAdd(&C->a_moved, t_moved);
    if (t_cand) atomicAdd(&C->a_cand, t_cand);
    if (t_nbr) atomicAdd(&C->a_nbr, t_nbr);
    if (t_cont) atomicAdd(&C->a_contact, t_cont);
    if (t_exact) atomicAdd(&C->a_exact, t_exact);
  }
}

// ---------------------------------------------------------------- static pass
// Static agents (FM_STEP with static detection, before the force kernel).  A
// box is clean when no box of its 27-box stencil is dirty; an agent of a clean
// box that did not change in the previous iteration and had at most one
// contact is static.  One warp per occupied brick finishes the brick's static
// agents in a streaming pass (flag, bounding box, zero force: what the per-box
// path does for a static agent) and stores in need[o] the brick's boxes that
// still hold non-static agents; bricks with such boxes and fewer than
// FORCE_HEAVY_LO agents go to the work list the force kernel takes them from
// (heavier ones stay on the heavy lists).  High occupancy hides the per-brick
// latency that a force-kernel block would serialise.
#define KS_WARPS 8
__global__ void __launch_bounds__(KS_WARPS * 32, 8) k_static(DevBufs B, DevParams P) {
  __shared__ unsigned long long s_dm[KS_WARPS][27];
  __shared__ unsigned s_bst[KS_WARPS][64], s_bcnt[KS_WARPS][64], s_work[KS_WARPS][64];
  DevCounters *C = B.ctr;
  if (C->error || !(P.detect_static && C->history_valid)) return;
  const AgentSet &A = *B.A;
  const int cur = (int)(C->step & 1), nxt = cur ^ 1;
  const long long n_occ = C->n_occ;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned c_static = 0;
  unsigned long long mn[3] = {~0ull, ~0ull, ~0ull}, mx[3] = {0ull, 0ull, 0ull};
  int wsim = -1;
  auto flush = [&]() {
    unsigned long long v[6];
    for (int d = 0; d < 3; ++d) { v[d] = wmin64(mn[d]); v[3 + d] = wmax64(mx[d]); mn[d] = ~0ull; mx[d] = 0ull; }
    if (lane == 0 && wsim >= 0 && v[0] != ~0ull) {
      unsigned long long *bb = B.bbox + ((size_t)nxt * P.n_sims + wsim) * 6;
      for (int d = 0; d < 3; ++d) { atomicMin(&bb[d], v[d]); atomicMax(&bb[3 + d], v[3 + d]); }
    }
  };
  for (long long o = (long long)blockIdx.x * KS_WARPS + w; o < n_occ; o += (long long)gridDim.x * KS_WARPS) {
    const int4 info = B.occ_info[o];
    if (info.w != wsim) {
      flush();
      wsim = info.w;
    }
    const SimGeom &G = B.geom[info.w];
    if (lane < 27) {
      const int X = info.x + lane % 3 - 1, Y = info.y + (lane / 3) % 3 - 1, Z = info.z + lane / 9 - 1;
      unsigned long long dm = 0ull;
      if (X >= 0 && X < G.nr[0] && Y >= 0 && Y < G.nr[1] && Z >= 0 && Z < G.nr[2])
        dm = B.dirty[B.brick_table[G.brick_base + ((long long)Z * G.nr[1] + Y) * G.nr[0] + X]];
      s_dm[w][lane] = dm;
    }
    s_bst[w][lane] = B.box_start[o * 64 + lane];
    s_bst[w][lane + 32] = B.box_start[o * 64 + lane + 32];
    s_bcnt[w][lane] = B.box_cnt[o * 64 + lane];
    s_bcnt[w][lane + 32] = B.box_cnt[o * 64 + lane + 32];
    __syncwarp();
    // clean boxes (the per-box path's stencil test), lane and lane + 32
    unsigned long long cm = 0ull;
    for (int h = 0; h < 2; ++h) {
      const int lb = lane + 32 * h;
      const bool dirty = stencil_dirty(s_dm[w], lb);
      s_work[w][lb] = dirty ? s_bcnt[w][lb] : 0u;
      cm |= (unsigned long long)__ballot_sync(0xffffffffu, !dirty) << (32 * h);
    }
    __syncwarp();
    const unsigned S0 = s_bst[w][0], m = s_bst[w][63] + s_bcnt[w][63] - S0;
    for (unsigned k = lane; k < m; k += 32) {
      // the box holding sorted position S0 + k: the last one starting at or
      // before it (an empty box starts where the next one does)
      int lb = 0;
      for (int st = 32; st > 0; st >>= 1)
        if (lb + st < 64 && s_bst[w][lb + st] <= S0 + k) lb += st;
      if (!((cm >> lb) & 1ull)) continue;
      const uint32_t iq = B.perm[S0 + k];
      const uint8_t fl = A.flags[iq];
      if ((fl & FL_CHANGED) || A.nz[iq] > 1) {
        atomicAdd(&s_work[w][lb], 1u);
        continue;
      }
      if (P.die && (A.beh[iq] & BEH_DIE) && agent_dies(P, A.uid[iq], C->step)) {
        A.flags[iq] = FL_STATIC | FL_REMOVE;  // removed at the end of the iteration
        if (P.keep_forces) { B.fdbg[iq] = 0.0; B.fdbg[B.cap + iq] = 0.0; B.fdbg[2 * B.cap + iq] = 0.0; }
        c_static++;
        continue;
      }
      if (fl != FL_STATIC) A.flags[iq] = FL_STATIC;
      const unsigned long long e[3] = {enc_f64(A.x[cur][iq]), enc_f64(A.y[cur][iq]), enc_f64(A.z[cur][iq])};
      for (int d = 0; d < 3; ++d) { mn[d] = min(mn[d], e[d]); mx[d] = max(mx[d], e[d]); }
      if (P.keep_forces) { B.fdbg[iq] = 0.0; B.fdbg[B.cap + iq] = 0.0; B.fdbg[2 * B.cap + iq] = 0.0; }
      c_static++;
    }
    __syncwarp();
    const unsigned long long need = (unsigned long long)__ballot_sync(0xffffffffu, s_work[w][lane] > 0u) |
                                    ((unsigned long long)__ballot_sync(0xffffffffu, s_work[w][lane + 32] > 0u) << 32);
    if (lane == 0) {
      B.need[o] = need;
      if (need && m < FORCE_HEAVY_LO) {
        const unsigned long long e = atomicAdd(&C->work_n, 1ull);
        if (BDM_IN(B.ctr, (long long)e < B.occ_cap)) B.worklist[e] = (int32_t)o;
      }
    }
    __syncwarp();
  }
  flush();
  const unsigned long long t = wsum64(c_static);
  if (lane == 0 && t) atomicAdd(&C->a_static, t);
}

__global__ void k_reset_work(DevBufs B) {
  B.ctr->work_next = 0;
  B.ctr->work_next2 = 0;
  B.ctr->heavy_take[0] = B.ctr->heavy_take[1] = 0;
  B.ctr->fix_n = 0;
}

// ---------------------------------------------------------------- fix-up pass (FP32 form)
// The FP32-form agents that the lane-per-agent force kernel listed (an FP32
// error bound not small against the agent's tolerance, or a summed pair-force
// magnitude so small that the absolute floor dominates) are evaluated again
// here, FIX_LANES lanes per listed agent: each lane walks every FIX_LANES-th
// box of the agent's 27-box stencil, with k_force's FP32 prefilter and
// decisions (FP64 inside the error bands); every contact the FP32 error
// analysis does not cover (|F| < low_scale, delta < graze, d^2 < close2) in
// double-float (contact_df), the others with the force kernel's FP32
// arithmetic; the contributions summed in FP64 (per lane, then over the
// agent's lanes in a fixed tree), rounded to FP32 once.  The listed agents are
// few (1-2% of a dense tissue), so the pass takes a few waves, and its time
// is a warp's latency: 16 lanes per agent split that walk, and the FP64 and
// double-float pairs of a warp's 2 agents, where a lane per agent would
// serialise those of 32.
#define FIXT_THREADS 128
#define FIX_LANES 16
template <int MODE>
__global__ void __launch_bounds__(FIXT_THREADS, 8) k_force_fix(DevBufs B, DevParams P) {
  __shared__ float s_tkf[16], s_tgf[16];
  __shared__ double s_tkd[16], s_tgd[16];
  __shared__ DF s_tk2[16], s_tg2[16];
  __shared__ unsigned long long s_bb[FIXT_THREADS / 32][6];
  DevCounters *C = B.ctr;
  if (C->error) return;
  const unsigned long long nfix = C->fix_n;
  if (nfix == 0) return;
  if (threadIdx.x < 16) {
    s_tkd[threadIdx.x] = P.type_k[threadIdx.x];
    s_tgd[threadIdx.x] = P.type_gamma[threadIdx.x];
    s_tkf[threadIdx.x] = (float)P.type_k[threadIdx.x];
    s_tgf[threadIdx.x] = (float)P.type_gamma[threadIdx.x];
    const float kh = (float)P.type_k[threadIdx.x], gh = (float)P.type_gamma[threadIdx.x];
    s_tk2[threadIdx.x] = {kh, (float)(P.type_k[threadIdx.x] - (double)kh)};
    s_tg2[threadIdx.x] = {gh, (float)(P.type_gamma[threadIdx.x] - (double)gh)};
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane < 6) s_bb[warp][lane] = (lane < 3) ? ~0ull : 0ull;
  __syncthreads();
  const AgentSet A = *B.A;
  const int cur = (int)(C->step & 1), nxt = cur ^ 1;
  const long long step = C->step;
  unsigned c_static = 0, c_moved = 0, n_exact = 0;
  int wsim = -1;
  // FIX_LANES lanes per listed agent, each walking every FIX_LANES-th box of
  // its stencil; warp-uniform trip count (the bounding-box flushes and the
  // lanes' sums are warp-wide)
  const int sub = lane & (FIX_LANES - 1);
  const unsigned long long stride = (unsigned long long)gridDim.x * (FIXT_THREADS / FIX_LANES);
  for (unsigned long long e0 = (unsigned long long)blockIdx.x * (FIXT_THREADS / FIX_LANES) +
                               (threadIdx.x & ~31u) / FIX_LANES;
       e0 < nfix; e0 += stride) {
    const unsigned long long e = e0 + (unsigned long long)(lane / FIX_LANES);
    bool valid = e < nfix && BDM_IN(B.ctr, (long long)e < B.cap);
    const uint4 ent = valid ? B.fix[e] : make_uint4(0u, 0u, 0u, 0u);
    const unsigned kq = ent.x;
    const long long o = (long long)(ent.y >> 6);
    const int lb = (int)(ent.y & 63u);
    if (valid && !BDM_IN(B.ctr, o < C->n_occ && (long long)kq < C->n)) valid = false;
    const int4 info = valid ? B.occ_info[o] : make_int4(0, 0, 0, 0);
    // the warp's bounding-box accumulator holds one simulation at a time; a
    // warp whose agents belong to several simulations updates each agent's
    // simulation box directly
    bool same = true;
    if (MODE == FM_STEP) {
      const int sim0 = __shfl_sync(0xffffffffu, valid ? info.w : -1, 0);
      same = __all_sync(0xffffffffu, !valid || info.w == sim0);
      if (same && sim0 != wsim) {
        flush_bbox_warp(B, P, nxt, wsim, s_bb[warp]);
        wsim = sim0;
      }
    }
    double hx = 0.0, hy = 0.0, hz = 0.0;
    const SimGeom &G = B.geom[info.w];
    if (valid) {
      const float4 cq = B.c32[kq];
      const dbl4 dq = exact_of<1>(B, A, cur, kq);
      const int tq4 = (P.n_types > 1) ? 4 * (int)B.tp[kq] : 0;
      int lx, ly, lz;
      local_decode(lb, lx, ly, lz);
      for (int sb = sub; sb < 27; sb += FIX_LANES) {
        const int ax = lx + sb % 3 - 1, ay = ly + (sb / 3) % 3 - 1, az = lz + sb / 9 - 1;
        const int X = info.x + ((ax < 0) ? -1 : (ax > 3 ? 1 : 0));
        const int Y = info.y + ((ay < 0) ? -1 : (ay > 3 ? 1 : 0));
        const int Z = info.z + ((az < 0) ? -1 : (az > 3 ? 1 : 0));
        if (X < 0 || X >= G.nr[0] || Y < 0 || Y >= G.nr[1] || Z < 0 || Z >= G.nr[2]) continue;
        const int rank = B.brick_table[G.brick_base + ((long long)Z * G.nr[1] + Y) * G.nr[0] + X];
        const int occ = B.brick_occ[rank];
        if (occ < 0) continue;
        const long long bx = (long long)occ * 64 + local_code(ax & 3, ay & 3, az & 3);
        const unsigned st = B.box_start[bx], cnt = B.box_cnt[bx];
        const float ofx = (float)(sb % 3 - 1) * P.Lf, ofy = (float)((sb / 3) % 3 - 1) * P.Lf,
                    ofz = (float)(sb / 9 - 1) * P.Lf;
        for (unsigned j = 0; j < cnt; ++j) {
          const unsigned kj = st + j;
          if (!BDM_IN(B.ctr, (long long)kj < C->n)) break;
          const float4 cs = __ldg(&B.c32[kj]);
          const float4 c = make_float4(cs.x + ofx, cs.y + ofy, cs.z + ofz, cs.w);
          const float d2 = dist2_f32(cq, c);
          if (!(d2 < P.R2_hi_f) || kj == kq) continue;
          const bool band = (d2 > P.R2_lo_f) || (d2 < TINY2);
          const float s = __fadd_rn(cq.w, c.w), s2 = s * s;
          const float W = fmaf(s, P.cband1, s2 * P.cband2);
          if (!band && d2 >= s2 + W) continue;  // a neighbour, certainly no contact
          const int ab = tq4 + ((P.n_types > 1) ? (int)B.tp[kj] : 0);
          n_exact++;
          if (band || d2 > s2 - W) {  // cutoff or contact undecided in FP32: FP64
            pair_f64_k(P.R2, s_tkd[ab], s_tgd[ab], dq, exact_of<1>(B, A, cur, kj), hx, hy, hz);
            continue;
          }
          const ContactF32 k = contact_f32(d2, s, __fmul_rn(cq.w, c.w), s_tkf[ab], s_tgf[ab]);
          if (fabsf(k.fm) < P.low_scale || k.delta < P.graze || d2 < P.close2) {
            float tx, ty, tz;
            contact_df(P, dq, exact_of<1>(B, A, cur, kj), s_tk2[ab], s_tg2[ab], tx, ty, tz);
            hx += (double)tx; hy += (double)ty; hz += (double)tz;
          } else {
            n_exact--;
            hx += (double)__fmul_rn(k.scf, __fsub_rn(cq.x, c.x));
            hy += (double)__fmul_rn(k.scf, __fsub_rn(cq.y, c.y));
            hz += (double)__fmul_rn(k.scf, __fsub_rn(cq.z, c.z));
          }
        }
      }
    }
    for (int of = FIX_LANES >> 1; of > 0; of >>= 1) {
      hx += __shfl_xor_sync(0xffffffffu, hx, of);
      hy += __shfl_xor_sync(0xffffffffu, hy, of);
      hz += __shfl_xor_sync(0xffffffffu, hz, of);
    }
    if (valid && sub == 0) {
      const uint32_t iq = B.perm[kq];
      double px = 0.0, py = 0.0, pz = 0.0;
      if (MODE == FM_STEP) { px = A.x[cur][iq]; py = A.y[cur][iq]; pz = A.z[cur][iq]; }
      // the force kernel's neighbour and contact counts (ent.w, ent.z)
      finish_agent<1, MODE>(B, P, A, cur, nxt, step, G.dt, G.dt_f, iq, A.flags[iq], false, (float)hx, (float)hy,
                            (float)hz, 0.0, 0.0, 0.0, ent.w, ent.z, c_static, c_moved,
                            same ? s_bb[warp] : B.bbox + ((size_t)nxt * P.n_sims + info.w) * 6, px, py, pz);
    }
  }
  if (MODE == FM_STEP) flush_bbox_warp(B, P, nxt, wsim, s_bb[warp]);
  const unsigned long long t_moved = wsum64(c_moved), t_exact = wsum64(n_exact);
  if (lane == 0) {
    if (t_moved) atomicAdd(&C->a_moved, t_moved);
    if (t_exact) atomicAdd(&C->a_exact, t_exact);
  }
}

// ---------------------------------------------------------------- division merge
// Daughter slot = n + (number of dividing agents with a smaller storage
// index): a tile-wise exclusive scan of the divide flags in storage order.
__device__ unsigned blk_scan(unsigned v, unsigned *sm, unsigned *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  unsigned x = v;
  for (int o = 1; o < 32; o <<= 1) {
    unsigned y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sm[warp] = x;
  __syncthreads();
  if (warp == 0) {
    unsigned w = (lane < nw) ? sm[lane] : 0u;
    for (int o = 1; o < 32; o <<= 1) {
      unsigned y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    sm[lane] = w;
  }
  __syncthreads();
  const unsigned base = warp ? sm[warp - 1] : 0u;
  *total = sm[nw - 1];
  __syncthreads();
  return base + x - v;
}

// Per tile of SCAN_TILE agents: the number of dividing agents (low 16 bits)
// and of removed agents (high 16 bits) in one packed word (a tile holds at
// most 2048 of each, so the halves never carry into each other).
__device__ __forceinline__ unsigned commit_flags(uint8_t f) {
  return ((f & FL_DIVIDE) ? 1u : 0u) | ((f & FL_REMOVE) ? 0x10000u : 0u);
}

__global__ void k_div_reduce(DevBufs B) {
  __shared__ unsigned sm[32];
  const DevCounters *C = B.ctr;
  if (C->error) return;
  const long long n = C->n;
  const long long t0 = (long long)blockIdx.x * SCAN_TILE;
  if (t0 >= n) return;
  const AgentSet A = *B.A;
  unsigned c = 0;
  for (int e = 0; e < SCAN_TILE / SCAN_THREADS; ++e) {
    const long long i = t0 + threadIdx.x * (SCAN_TILE / SCAN_THREADS) + e;
    if (i < n) c += commit_flags(A.flags[i]);
  }
  unsigned tot;
  blk_scan(c, sm, &tot);
  if (threadIdx.x == 0) {
    B.scan_a[blockIdx.x] = tot & 0xffffu;
    B.scan_b[blockIdx.x] = tot >> 16;
  }
}

// Exclusive scans over the tiles of the division counts (scan_a) and the
// removal counts (scan_b); totals n_div and n_rm; the size after the commit
// m = n + n_div - n_rm.
__global__ void k_div_top(DevBufs B) {
  __shared__ unsigned sm[32];
  DevCounters *C = B.ctr;
  if (C->error) return;
  const long long n = C->n;
  const long long nblk = (n + SCAN_TILE - 1) / SCAN_TILE;
  unsigned carry = 0, carry_rm = 0;
  for (long long b0 = 0; b0 < nblk; b0 += blockDim.x) {
    const long long b = b0 + threadIdx.x;
    const unsigned v = (b < nblk) ? B.scan_a[b] : 0u;
    const unsigned w = (b < nblk) ? B.scan_b[b] : 0u;
    unsigned t, t_rm;
    const unsigned e = blk_scan(v, sm, &t);
    const unsigned e_rm = blk_scan(w, sm, &t_rm);
    if (b < nblk) { B.scan_a[b] = carry + e; B.scan_b[b] = carry_rm + e_rm; }
    carry += t;
    carry_rm += t_rm;
  }
  if (threadIdx.x == 0) {
    C->n_div = carry;
    C->n_rm = carry_rm;
    C->rm_m = n + (long long)carry - (long long)carry_rm;
    C->rm_h = 0;
  }
}

__global__ void k_div_write(DevBufs B, DevParams P) {
  __shared__ unsigned sm[32];
  DevCounters *C = B.ctr;
  if (C->error) return;
  const long long n = C->n;
  const long long t0 = (long long)blockIdx.x * SCAN_TILE;
  if (t0 >= n) return;
  const AgentSet A = *B.A;
  const int nxt = (int)((C->step & 1) ^ 1);
  constexpr int E = SCAN_TILE / SCAN_THREADS;
  unsigned c = 0;
  for (int e = 0; e < E; ++e) {
    const long long i = t0 + threadIdx.x * E + e;
    if (i < n) c += (A.flags[i] & FL_DIVIDE) ? 1u : 0u;
  }
  unsigned tot;
  unsigned r = blk_scan(c, sm, &tot) + B.scan_a[blockIdx.x];
  const double pi = 3.141592653589793;
  unsigned long long bmin[3] = {~0ull, ~0ull, ~0ull}, bmax[3] = {0ull, 0ull, 0ull};
  for (int e = 0; e < E; ++e) {
    const long long i = t0 + threadIdx.x * E + e;
    if (i >= n || !(A.flags[i] & FL_DIVIDE)) continue;
    const long long d = n + r;
    if (d >= B.cap) {  // cannot happen when the up-front count is right; never write out of bounds
      atomicCAS(&C->error, 0, (int)DEV_ECAP_AGENTS);
      break;
    }
    const dbl4 sd = B.stash[i];
    for (int b = 0; b < 2; ++b) { A.x[b][d] = sd.x; A.y[b][d] = sd.y; A.z[b][d] = sd.z; }
    A.vol[d] = sd.w;
    ((double *)A.diam)[d] = cbrt_newton(__ddiv_rn(__dmul_rn(6.0, sd.w), pi));
    A.uid[d] = C->next_uid + r;
    A.beh[d] = A.beh[i];
    A.flags[d] = FL_CHANGED;
    A.nz[d] = 0;
    if (P.keep_forces) { B.fdbg[d] = 0.0; B.fdbg[B.cap + d] = 0.0; B.fdbg[2 * B.cap + d] = 0.0; }
    A.flags[i] &= (uint8_t)~FL_DIVIDE;
    const unsigned long long e0 = enc_f64(sd.x), e1 = enc_f64(sd.y), e2 = enc_f64(sd.z);
    bmin[0] = min(bmin[0], e0); bmax[0] = max(bmax[0], e0);
    bmin[1] = min(bmin[1], e1); bmax[1] = max(bmax[1], e1);
    bmin[2] = min(bmin[2], e2); bmax[2] = max(bmax[2], e2);
    ++r;
  }
  flush_bbox(B, P, nxt, 0, bmin, bmax);
}

// ---------------------------------------------------------------- removal
// Removal (Sec. 3.2), after the daughters are appended: the vector of
// n' = n + n_div agents keeps no empty element.  With m = n' - n_rm the new
// size, a removed agent at i < m is a hole; the survivors at i >= m fill the
// holes, the k-th survivor (ascending index) the k-th hole (ascending index),
// which is the paper's swap step with the removed list in storage order.
// The work is O(n) flag reads (one byte per agent) for the holes, and
// O(n_rm) for the moves.  The removed agents' positions P_t are kept as
// ghosts: their boxes are dirty in the next iteration's static test.
__global__ void k_rm_holes(DevBufs B, DevParams P) {
  __shared__ unsigned sm[32];
  DevCounters *C = B.ctr;
  if (C->error) return;
  const long long n = C->n;
  const long long t0 = (long long)blockIdx.x * SCAN_TILE;
  if (t0 >= n) return;
  const AgentSet A = *B.A;
  const int cur = (int)(C->step & 1);
  const long long m = C->rm_m;
  constexpr int E = SCAN_TILE / SCAN_THREADS;
  unsigned c = 0;
  for (int e = 0; e < E; ++e) {
    const long long i = t0 + threadIdx.x * E + e;
    if (i < n) c += (A.flags[i] & FL_REMOVE) ? 1u : 0u;
  }
  unsigned tot;
  unsigned r = blk_scan(c, sm, &tot) + B.scan_b[blockIdx.x];
  unsigned holes = 0;
  for (int e = 0; e < E; ++e) {
    const long long i = t0 + threadIdx.x * E + e;
    if (i >= n || !(A.flags[i] & FL_REMOVE)) continue;
    B.ghost[r] = mk_dbl4(A.x[cur][i], A.y[cur][i], A.z[cur][i], 0.0);
    if (i < m) {
      B.bucket[r] = (uint32_t)i;
      holes = r + 1;
    }
    ++r;
  }
  if (holes) atomicMax(&C->rm_h, (unsigned long long)holes);
}

__device__ __forceinline__ void move_agent(const DevBufs &B, const DevParams &P, const AgentSet &A, long long src,
                                           long long dst) {
  for (int b = 0; b < 2; ++b) {
    A.x[b][dst] = A.x[b][src];
    A.y[b][dst] = A.y[b][src];
    A.z[b][dst] = A.z[b][src];
  }
  if (P.precision == 0) ((double *)A.diam)[dst] = ((const double *)A.diam)[src];
  else ((float *)A.diam)[dst] = ((const float *)A.diam)[src];
  if (A.vol) A.vol[dst] = A.vol[src];
  A.uid[dst] = A.uid[src];
  A.beh[dst] = A.beh[src];
  A.flags[dst] = A.flags[src];
  A.nz[dst] = A.nz[src];
  if (P.keep_forces)
    for (int d = 0; d < 3; ++d) B.fdbg[(size_t)d * B.cap + dst] = B.fdbg[(size_t)d * B.cap + src];
}

// The survivors at i in [m, n'): block b takes the b-th tile that meets the
// tail.  Survivor i is the k-th of the tail, k = (i - m) - (removed agents in
// [m, i)).  Only flags at indices >= m are read: the moves write holes, all
// below m, concurrently.  For a tile starting at t0 > m, the removed agents in
// [m, t0) are rr(t0) - h, with rr(t0) = the tile's exclusive removal prefix
// and h the number of holes (removed agents below m).
__global__ void k_rm_move(DevBufs B, DevParams P) {
  __shared__ unsigned sm[32];
  DevCounters *C = B.ctr;
  if (C->error) return;
  const long long n = C->n;
  const long long n2 = n + C->n_div;
  const long long m = C->rm_m;
  if (m >= n2) return;
  const long long tile = m / SCAN_TILE + blockIdx.x;
  const long long t0 = tile * SCAN_TILE;
  if (t0 >= n2) return;
  const AgentSet A = *B.A;
  const long long ntiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  const long long h = (long long)C->rm_h;
  constexpr int E = SCAN_TILE / SCAN_THREADS;
  unsigned c = 0;
  for (int e = 0; e < E; ++e) {
    const long long i = t0 + threadIdx.x * E + e;
    if (i >= m && i < n) c += (A.flags[i] & FL_REMOVE) ? 1u : 0u;
  }
  unsigned tot;
  long long before = 0;  // removed agents in [m, t0)
  if (t0 > m) before = ((tile < ntiles) ? (long long)B.scan_b[tile] : (long long)C->n_rm) - h;
  long long rt = (long long)blk_scan(c, sm, &tot) + before;
  for (int e = 0; e < E; ++e) {
    const long long i = t0 + threadIdx.x * E + e;
    if (i >= n2) break;
    if (i < m) continue;
    const bool removed = i < n && (A.flags[i] & FL_REMOVE);
    if (!removed) {
      const long long k = (i - m) - rt;
      if (!BDM_IN(B.ctr, k >= 0 && k < h)) break;
      const long long dst = (long long)B.bucket[k];
      if (!BDM_IN(B.ctr, dst < m)) break;
      move_agent(B, P, A, i, dst);
    }
    rt += removed ? 1 : 0;
  }
}

__global__ void k_finish(DevBufs B) {
  DevCounters *C = B.ctr;
  if (C->error) return;
  const long long nd = C->n_div, nr = C->n_rm;
  C->n += nd - nr;
  C->next_uid += (unsigned long long)nd;
  C->l_rm = (unsigned long long)nr;
  C->l_fix = C->fix_n;
  C->n_ghost = nr;
  C->l_static = C->a_static;
  C->l_moved = C->a_moved;
  C->l_cand = C->a_cand;
  C->l_nbr = C->a_nbr;
  C->l_contact = C->a_contact;
  C->l_exact = C->a_exact;
  C->l_div = (unsigned long long)nd;
  C->l_boxes = C->total_boxes;
  C->l_bricks = C->total_bricks;
  C->l_occ = C->n_occ;
  C->l_max_brick = C->max_brick;
  C->step += 1;
  C->history_valid = 1;
}

// neighbour-list offsets (debug): exclusive scan of per-agent counts, serial
// per block tile, sufficient for diagnostic sizes
__global__ void k_nbr_offsets(DevBufs B) {
  __shared__ unsigned sm[32];
  const long long n = B.ctr->n;
  long long carry = 0;
  for (long long b0 = 0; b0 < n; b0 += blockDim.x) {
    const long long i = b0 + threadIdx.x;
    const unsigned v = (i < n) ? (unsigned)B.nbr_count[i] : 0u;
    unsigned t;
    const unsigned e = blk_scan(v, sm, &t);
    if (i < n) B.nbr_off[i] = carry + e;
    carry += t;
  }
  if (threadIdx.x == 0) B.nbr_off[n] = carry;
}

}  // namespace

void launch_force(const DevBufs &B, const DevParams &P, const LaunchCfg &c, int mode, cudaStream_t s) {
  k_reset_work<<<1, 1, 0, s>>>(B);
  if (mode == FM_STEP && P.detect_static) k_static<<<2 * c.occ_blocks, KS_WARPS * 32, 0, s>>>(B, P);
  const int g = c.force_blocks;
  const bool ty = P.n_types > 1;
#define LF(PR, MO, SP, TY) k_force<PR, MO, SP, TY><<<g, FORCE_WARPS * 32, 0, s>>>(B, P)
#define LT(MO, TY) k_force_tile<MO, TY><<<g, TILE_WARPS * 32, 0, s>>>(B, P)
#define LS(MO, TY) k_force_sparse<MO, TY><<<2 * g, SP_WARPS * 32, 0, s>>>(B, P)
  // the hybrid launch: the lane-per-agent kernel (4 lanes per agent, adapted
  // per pass) on the bricks that are not light, then the sparse kernel on the
  // light ones
  DevParams Pd = P, Pl = P;
  Pd.brick_class = 1;
  Pd.lanes_fixed = 4;
  Pl.brick_class = 2;
  if (P.precision == 0) {
    switch (mode) {
      case FM_STEP: if (ty) LF(0, FM_STEP, false, true); else LF(0, FM_STEP, false, false); break;
      case FM_FORCES: if (ty) LF(0, FM_FORCES, false, true); else LF(0, FM_FORCES, false, false); break;
      case FM_COUNT_NBR: LF(0, FM_COUNT_NBR, false, false); break;
      default: LF(0, FM_LIST_NBR, false, false); break;
    }
  } else {
    switch (mode) {
      case FM_STEP:
        if (P.lanes_fixed == FORCE_TILE) {
          if (ty) LT(FM_STEP, true); else LT(FM_STEP, false);
        } else if (P.lanes_fixed == FORCE_SPARSE) {
          if (ty) LS(FM_STEP, true); else LS(FM_STEP, false);
        } else if (P.lanes_fixed == FORCE_HYBRID) {
          if (ty) {
            k_force<1, FM_STEP, false, true><<<g, FORCE_WARPS * 32, 0, s>>>(B, Pd);
            k_force_sparse<FM_STEP, true><<<2 * g, SP_WARPS * 32, 0, s>>>(B, Pl);
          } else {
            if (!P.walk && !P.grow && !P.die) k_force<1, FM_STEP, true, false><<<g, FORCE_WARPS * 32, 0, s>>>(B, Pd);
            else k_force<1, FM_STEP, false, false><<<g, FORCE_WARPS * 32, 0, s>>>(B, Pd);
            k_force_sparse<FM_STEP, false><<<2 * g, SP_WARPS * 32, 0, s>>>(B, Pl);
          }
        } else if (ty) LF(1, FM_STEP, false, true);
        else if (!P.walk && !P.grow && !P.die) LF(1, FM_STEP, true, false);
        else LF(1, FM_STEP, false, false);
        break;
      case FM_FORCES:
        if (P.lanes_fixed == FORCE_TILE) {
          if (ty) LT(FM_FORCES, true); else LT(FM_FORCES, false);
        } else if (P.lanes_fixed == FORCE_SPARSE) {
          if (ty) LS(FM_FORCES, true); else LS(FM_FORCES, false);
        } else if (P.lanes_fixed == FORCE_HYBRID) {
          if (ty) {
            k_force<1, FM_FORCES, false, true><<<g, FORCE_WARPS * 32, 0, s>>>(B, Pd);
            k_force_sparse<FM_FORCES, true><<<2 * g, SP_WARPS * 32, 0, s>>>(B, Pl);
          } else {
            k_force<1, FM_FORCES, false, false><<<g, FORCE_WARPS * 32, 0, s>>>(B, Pd);
            k_force_sparse<FM_FORCES, false><<<2 * g, SP_WARPS * 32, 0, s>>>(B, Pl);
          }
        } else if (ty) LF(1, FM_FORCES, false, true);
        else LF(1, FM_FORCES, false, false);
        break;
      case FM_COUNT_NBR: LF(1, FM_COUNT_NBR, false, false); break;
      default: LF(1, FM_LIST_NBR, false, false); break;
    }
  }
#undef LF
#undef LT
#undef LS
  if (mode == FM_FORCES) launch_force_fix(B, P, c, mode, s);
}

// the FP64 fix-up pass of the FP32 form, after launch_force (FM_STEP: its own
// phase of an iteration; FM_FORCES: part of launch_force)
void launch_force_fix(const DevBufs &B, const DevParams &P, const LaunchCfg &c, int mode, cudaStream_t s) {
  // the tiled and sparse kernels list no agent
  if (P.precision != 1 || P.lanes_fixed == FORCE_TILE || P.lanes_fixed == FORCE_SPARSE) return;
  if (mode == FM_STEP) k_force_fix<FM_STEP><<<2 * c.occ_blocks, FIXT_THREADS, 0, s>>>(B, P);
  if (mode == FM_FORCES) k_force_fix<FM_FORCES><<<2 * c.occ_blocks, FIXT_THREADS, 0, s>>>(B, P);
}

// kernels of an iteration's force phase: k_reset_work, k_static (static
// detection), the force kernel (two for the hybrid launch)
int force_launches(const DevParams &P) {
  return 2 + (P.detect_static ? 1 : 0) + ((P.precision == 1 && P.lanes_fixed == FORCE_HYBRID) ? 1 : 0);
}
int force_fix_launches(const DevParams &P) {
  return (P.precision == 1 && P.lanes_fixed != FORCE_TILE && P.lanes_fixed != FORCE_SPARSE) ? 1 : 0;
}

void launch_divide(const DevBufs &B, const DevParams &P, const LaunchCfg &c, cudaStream_t s) {
  if (!P.grow && !P.die) return;
  k_div_reduce<<<c.agent_scan_blocks, SCAN_THREADS, 0, s>>>(B);
  k_div_top<<<1, 1024, 0, s>>>(B);
  if (P.grow) k_div_write<<<c.agent_scan_blocks, SCAN_THREADS, 0, s>>>(B, P);
  if (P.die) {
    k_rm_holes<<<c.agent_scan_blocks, SCAN_THREADS, 0, s>>>(B, P);
    k_rm_move<<<c.agent_scan_blocks + 1, SCAN_THREADS, 0, s>>>(B, P);
  }
}

int divide_launches(const DevParams &P) { return (P.grow || P.die) ? 2 + (P.grow ? 1 : 0) + (P.die ? 2 : 0) : 0; }

void launch_finish(const DevBufs &B, const DevParams &P, cudaStream_t s) {
  (void)P;
  k_finish<<<1, 1, 0, s>>>(B);
}

void launch_nbr_offsets(const DevBufs &B, const DevParams &P, cudaStream_t s) {
  (void)P;
  k_nbr_offsets<<<1, 1024, 0, s>>>(B);
}
