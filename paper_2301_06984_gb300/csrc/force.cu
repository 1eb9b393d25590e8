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
// then takes the box's agents in groups: S lanes per agent split the candidate
// boxes (FP32 form; S chosen per box from its occupancy and candidate count)
// and a shuffle tree reduces the S partial sums.  The FP64 form keeps one lane
// per agent and the canonical summation order (stencil boxes dz, dy, dx
// ascending; ascending storage index inside a box), which makes it bit-equal
// to the FP64 oracle.  Both forms decide "neighbour" (d^2 < R^2) and
// "contact" (delta > 0) exactly as FP64 does: an FP32 estimate with a rigorous
// error band decides outside the band, FP64 decides inside it.
#include <type_traits>

#include "bdm_internal.cuh"

namespace {

// ---------------------------------------------------------------- Philox
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
__device__ __forceinline__ int pair_f64(const DevParams &P, const dbl4 &q, const dbl4 &c, double &fx, double &fy,
                                        double &fz) {
  return pair_f64_k(P.R2, P.k, P.gamma, q, c, fx, fy, fz);
}
// The same pair as pair_f64, returning the three products sc * (q - c) that
// pair_f64 adds to the running sum (so a caller can add them later, in the
// same order, with the same IEEE operations).
__device__ __forceinline__ int pair_f64_terms(const DevParams &P, const dbl4 &q, const dbl4 &c, double &tx, double &ty,
                                              double &tz) {
  const double ddx = __dsub_rn(q.x, c.x), ddy = __dsub_rn(q.y, c.y), ddz = __dsub_rn(q.z, c.z);
  const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(ddx, ddx), __dmul_rn(ddy, ddy)), __dmul_rn(ddz, ddz));
  if (!(d2 < P.R2)) return 0;
  if (d2 == 0.0) return 1;
  const double d = __dsqrt_rn(d2);
  const double delta = __dsub_rn(__dadd_rn(q.w, c.w), d);
  if (!(delta > 0.0)) return 1;
  const double rbar = __ddiv_rn(__dmul_rn(q.w, c.w), __dadd_rn(q.w, c.w));
  const double F = __dsub_rn(__dmul_rn(P.k, delta), __dmul_rn(P.gamma, __dsqrt_rn(__dmul_rn(rbar, delta))));
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
__device__ __forceinline__ long long next_force_brick(const DevBufs &B, DevCounters *C, long long n_occ, int &phase,
                                                      bool use_static) {
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
    if (use_static) return u < (long long)C->work_n ? (long long)B.worklist[u] : -1;
    if (u >= n_occ) return -1;
    if (B.brick_count[B.occ_list[u]] < FORCE_HEAVY_LO) return u;  // heavy ones were listed
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
    const uint8_t beh = (P.walk || P.grow) ? A.beh[iq] : (uint8_t)0;
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

// SPLIT (FP32 step without random walk or growth only): the agent's lanes
// finish one axis each.  A separate instantiation, so that the other forms
// keep the register allocation they have without that code.
template <int PREC, int MODE, bool SPLIT = false>
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
  __shared__ unsigned s_pre[FORCE_WARPS][28], s_st[FORCE_WARPS][28];
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

  // One block per occupied brick (taken from a global counter); its warps
  // take the brick's 64 boxes from a block counter.
  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) {
      s_o = next_force_brick(B, C, n_occ, fetch_phase, use_static);
      s_next = 0;
    }
    __syncthreads();
    const long long o = s_o;
    if (o < 0) break;
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
      if (lane < 27) {
        s_pre[warp][lane] = pre - nb_cnt;
        s_st[warp][lane] = nb_st;
      }
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
      const int sub = lane & (S - 1);
      const unsigned G_ = 32u / S;
      for (unsigned q0 = 0; q0 < nq; q0 += G_) {
        const unsigned qi = q0 + (unsigned)(lane / S);
        const bool valid = qi < nq;
        const unsigned kq = qbase + (valid ? qi : 0u);
        const uint32_t iq = B.perm[kq];
        const float4 cq = B.c32[kq];
        dbl4 dq = mk_dbl4(0.0, 0.0, 0.0, 0.0);
        if (PREC == 0) dq = B.c64[kq];
        const uint8_t fl = valid ? A.flags[iq] : (uint8_t)0;
        const bool is_static = use_static && clean && valid && !(fl & FL_CHANGED) && A.nz[iq] <= 1;
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
        float ffx = 0.f, ffy = 0.f, ffz = 0.f;
        float gfx = 0.f, gfy = 0.f, gfz = 0.f, gbound = 0.f, fscale = 0.f;
        double dfx = 0.0, dfy = 0.0, dfz = 0.0;
        unsigned ncont = 0, nnb = 0;
        long long lbase = 0;
        if (MODE == FM_LIST_NBR && valid) lbase = B.nbr_off[iq];
        bool refine = false;
        double hx = 0.0, hy = 0.0, hz = 0.0;
        for (int pass = 0; pass < 2; ++pass) {
          const bool act = (pass == 0) ? compute : refine;
          if (__any_sync(0xffffffffu, act)) {
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
                  if (lo + step <= 26 && s_pre[warp][lo + step] <= p) lo += step;
                boxs[m] = lo;
                kjs[m] = s_st[warp][lo] + (p - s_pre[warp][lo]);
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
                }
              }
              c0 += fill;
              if (fill == 0) break;
              __syncwarp();
              // ---- test the chunk in FP32, queue the candidates inside the band
              unsigned qlen = 0;
              if (act) {
                // the default stride (4 lanes per agent) with constant offsets
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
                    if (kj != ko) r = pair_f64_terms(P, B.c64[ko], B.c64[kj], tx, ty, tz);
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
                const unsigned kj = skj[i];
                if (kj == kq) continue;  // the agent itself
                if (PREC == 0) {
                  const dbl4 cj = B.c64[kj];
                  if (MODE == FM_COUNT_NBR || MODE == FM_LIST_NBR) {
                    if (is_nbr_f64(P, dq, cj)) {
                      if (MODE == FM_LIST_NBR) B.nbr_out[lbase + nnb] = (long long)B.perm[kj];
                      nnb++;
                    }
                    continue;
                  }
                  const int r = pair_f64(P, dq, cj, dfx, dfy, dfz);
                  nnb += (r > 0);
                  ncont += (r == 2);
                  continue;
                }
                const float4 c = sc[i];
                const float ex = cq.x - c.x, ey = cq.y - c.y, ez = cq.z - c.z;
                const float d2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
                const bool band = (d2 > P.R2_lo_f) || (d2 < TINY2);
                if (MODE == FM_COUNT_NBR || MODE == FM_LIST_NBR) {
                  bool isn = true;
                  if (band && d2 > P.R2_lo_f) {
                    atomicAdd(&s_ctr[warp][3], 1u);
                    isn = is_nbr_f64(P, exact_of<1>(B, A, cur, kq), exact_of<1>(B, A, cur, kj));
                  }
                  if (isn) {
                    if (MODE == FM_LIST_NBR) B.nbr_out[lbase + nnb] = (long long)B.perm[kj];
                    nnb++;
                  }
                  continue;
                }
                const float s = cq.w + c.w, s2 = s * s;
                const float W = fmaf(s, P.cband1, s2 * P.cband2);
                if (pass == 1 && (band || d2 > s2 - W)) continue;  // not an FP32 contact
                if (band || (d2 > s2 - W && d2 < s2 + W)) {
                  // cutoff or contact decided in FP64
                  atomicAdd(&s_ctr[warp][3], 1u);
                  double gx = 0.0, gy = 0.0, gz = 0.0;
                  const int r = pair_f64(P, exact_of<1>(B, A, cur, kq), exact_of<1>(B, A, cur, kj), gx, gy, gz);
                  nnb += (r > 0);
                  if (r == 2) {
                    ncont++;
                    ffx += (float)gx; ffy += (float)gy; ffz += (float)gz;
                  }
                  continue;
                }
                if (pass == 0) nnb++;
                if (d2 >= s2 + W) continue;  // certainly no contact
                const float inv_d = rsqrtf(d2);
                const float d = d2 * inv_d;
                const float delta = s - d;
                const float rbar = __fdividef(cq.w * c.w, s);
                const float rd = rbar * delta;            // > 0: a certain contact
                const float sq = rd * rsqrtf(rd);
                const float kd = P.kf * delta, gs = P.gammaf * sq;
                const float scf = (kd - gs) * inv_d;
                if (pass == 1) {
                  // refinement: the grazing contacts of pass 0, classified by the
                  // same FP32 arithmetic, redone in FP64
                  if (delta < P.graze) {
                    atomicAdd(&s_ctr[warp][3], 1u);
                    pair_f64(P, exact_of<1>(B, A, cur, kq), exact_of<1>(B, A, cur, kj), hx, hy, hz);
                  }
                  continue;
                }
                if (delta < P.graze) {
                  // grazing contact: d/d(delta) of sqrt(rbar delta) is large,
                  // so keep it apart with a bound of its FP32 error
                  gfx = fmaf(scf, ex, gfx);
                  gfy = fmaf(scf, ey, gfy);
                  gfz = fmaf(scf, ez, gfz);
                  gbound += (sq > 1e-18f) ? fminf(P.gammaf * rbar * P.graze_e * 0.5f * __frcp_rn(sq),
                                                  P.gammaf * sqrtf(rbar * P.graze_e))
                                          : P.gammaf * sqrtf(rbar * P.graze_e);
                } else {
                  ffx = fmaf(scf, ex, ffx);
                  ffy = fmaf(scf, ey, ffy);
                  ffz = fmaf(scf, ez, ffz);
                }
                fscale += kd + gs;
                ncont++;
              }
              __syncwarp();
            }
          }
          if (pass == 1) {
            for (int of = S >> 1; of > 0; of >>= 1) {
              hx += __shfl_xor_sync(0xffffffffu, hx, of);
              hy += __shfl_xor_sync(0xffffffffu, hy, of);
              hz += __shfl_xor_sync(0xffffffffu, hz, of);
            }
            if (refine) { gfx = (float)hx; gfy = (float)hy; gfz = (float)hz; }
            break;
          }
          // reduce the S partial sums of an agent
          for (int of = S >> 1; of > 0; of >>= 1) {
            ffx += __shfl_xor_sync(0xffffffffu, ffx, of);
            ffy += __shfl_xor_sync(0xffffffffu, ffy, of);
            ffz += __shfl_xor_sync(0xffffffffu, ffz, of);
            ncont += __shfl_xor_sync(0xffffffffu, ncont, of);
            nnb += __shfl_xor_sync(0xffffffffu, nnb, of);
            if (PREC == 1) {
              gfx += __shfl_xor_sync(0xffffffffu, gfx, of);
              gfy += __shfl_xor_sync(0xffffffffu, gfy, of);
              gfz += __shfl_xor_sync(0xffffffffu, gfz, of);
              gbound += __shfl_xor_sync(0xffffffffu, gbound, of);
              fscale += __shfl_xor_sync(0xffffffffu, fscale, of);
            }
          }
          if (PREC != 1 || !(MODE == FM_STEP || MODE == FM_FORCES)) break;
          // accept the grazing sum when its error bound is a small part of the
          // agent's tolerance; otherwise redo those pairs in FP64 (pass 1)
          refine = compute && gbound > 0.25f * (P.rel_tol * fscale + P.abs_tol);
          if (!__any_sync(0xffffffffu, refine)) break;
        }
        if (PREC == 1 && (MODE == FM_STEP || MODE == FM_FORCES)) {
          ffx += gfx;
          ffy += gfy;
          ffz += gfz;
        }
        if (SPLIT && S >= 4) {
          // Lanes 0, 1 and 2 of the agent finish one axis each (one FP64
          // position addition, store and bounding-box update per lane),
          // with the same arithmetic as finish_agent's FP32 form.
          float ux, uy, uz;
          displacement_f32(P, dt_f, ffx, ffy, ffz, ux, uy, uz);
          const bool live = valid && !is_static && sub < 3;
          double p = 0.0, np = 0.0;
          if (live) {
            asm volatile("cp.async.wait_all;\n" ::: "memory");
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

// Exact FP64 inputs of a pair, for the out-of-line settle step of k_force32.
struct ExactSrc {
  const uint32_t *perm;
  const double *x, *y, *z;
  const float4 *c32;
  double R2, k, gamma;
};

// Settle the deferred pairs of a k_force32 warp (called by the whole warp).
// Entry e holds the candidate's sorted index and the agent slot and kind in
// dw[e], and for a grazing pair its FP32 contribution and error bound in
// dc[e].  Band pairs are evaluated in FP64 and added with their neighbour and
// contact counts; the grazing pairs of agents in rmask are redone in FP64,
// replacing their FP32 contribution and removing their bound.  Each agent's
// owner lane adds its settled pairs in list order.  kq0 is the sorted index of
// agent slot 0.  Returns this lane's count of FP64 pair evaluations.
#define DA_EXACT 0x100u
#define DA_NBR 0x200u
#define DA_CONT 0x400u
__device__ __noinline__ unsigned settle_deferred(ExactSrc X, unsigned kq0, unsigned dlen, unsigned rmask, float4 *dc,
                                                 uint2 *dw, float4 *acc, float *bnd, uint32_t *nnb_s,
                                                 uint32_t *nct_s) {
  const unsigned lane = threadIdx.x & 31;
  unsigned n_exact = 0;
  for (unsigned e0 = 0; e0 < dlen; e0 += 32) {
    const unsigned e = e0 + lane;
    bool need = false;
    if (e < dlen) {
      const uint2 w = dw[e];
      const unsigned a = w.y & 0xffu;
      const bool ex = (w.y & DA_EXACT) != 0;
      need = ex || ((rmask >> a) & 1u);
      if (need) {
        n_exact++;
        const unsigned kq = kq0 + a, kj = w.x;
        const uint32_t iq = X.perm[kq], ij = X.perm[kj];
        const dbl4 pq = mk_dbl4(X.x[iq], X.y[iq], X.z[iq], ftod_exact(X.c32[kq].w));
        const dbl4 pj = mk_dbl4(X.x[ij], X.y[ij], X.z[ij], ftod_exact(X.c32[kj].w));
        double gx = 0.0, gy = 0.0, gz = 0.0;
        const int r = pair_f64_k(X.R2, X.k, X.gamma, pq, pj, gx, gy, gz);
        if (ex) {
          dc[e] = make_float4((float)gx, (float)gy, (float)gz, 0.f);
          dw[e].y = w.y | (r > 0 ? DA_NBR : 0u) | (r == 2 ? DA_CONT : 0u);
        } else {
          // FP64 contribution in place of the FP32 one; its bound goes
          const float4 d = dc[e];
          dc[e] = make_float4((float)gx - d.x, (float)gy - d.y, (float)gz - d.z, d.w);
        }
      }
    }
    unsigned nm = __ballot_sync(0xffffffffu, need);
    __syncwarp();
    for (; nm; nm &= nm - 1) {
      const unsigned e1 = e0 + (unsigned)(__ffs(nm) - 1);
      const unsigned w = dw[e1].y;
      if (lane == (w & 0xffu)) {
        const float4 d = dc[e1];
        float4 t = acc[lane];
        t.x += d.x; t.y += d.y; t.z += d.z;
        acc[lane] = t;
        if (w & DA_EXACT) {
          nnb_s[lane] += (w & DA_NBR) ? 1u : 0u;
          nct_s[lane] += (w & DA_CONT) ? 1u : 0u;
        } else {
          bnd[lane] -= d.w;
        }
      }
      __syncwarp();
    }
  }
  __syncwarp();
  return n_exact;
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
__global__ void __launch_bounds__(KS_WARPS * 32) k_static(DevBufs B, DevParams P) {
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
      int lx, ly, lz;
      local_decode(lb, lx, ly, lz);
      bool dirty = false;
      for (int t = 0; t < 27; ++t) {
        const int ax = lx + t % 3 - 1, ay = ly + (t / 3) % 3 - 1, az = lz + t / 9 - 1;
        const int bo = ((az < 0) ? 0 : (az > 3 ? 2 : 1)) * 9 + ((ay < 0) ? 0 : (ay > 3 ? 2 : 1)) * 3 +
                       ((ax < 0) ? 0 : (ax > 3 ? 2 : 1));
        dirty |= ((s_dm[w][bo] >> local_code(ax & 3, ay & 3, az & 3)) & 1ull) != 0ull;
      }
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
      if (need && m < FORCE_HEAVY_LO) B.worklist[atomicAdd(&C->work_n, 1ull)] = (int32_t)o;
    }
    __syncwarp();
  }
  flush();
  const unsigned long long t = wsum64(c_static);
  if (lane == 0 && t) atomicAdd(&C->a_static, t);
}

// ---------------------------------------------------------------- FP32 form: pair-ring kernel
// The FP32 form's production kernel.  Same work decomposition as k_force
// (one CTA per occupied brick, one warp per box), but the pairs are not
// evaluated lane-per-agent.  For a group of up to 32 agents of a box the warp
// stages the stencil's candidates in shared memory (up to F32_CHUNK at a
// time; most stencils fit at once); for every agent it tests 32 candidates
// per instruction in FP32 and appends the (agent, candidate) indices of those
// inside the cutoff band to a ring (ballot + popcount positions).  Whenever
// the ring holds 32 pairs they are evaluated with every lane busy, and a
// segmented shuffle reduction over the agent index folds them into per-agent
// sums in shared memory.  Pairs that FP32 cannot decide (cutoff or contact
// band) and grazing contacts are also written to the warp's deferred list in
// global memory, settled in FP64 at the end of the group: band pairs always,
// grazing pairs when the agent's summed FP32 error bound is not a small part
// of its tolerance (their FP32 contribution is then replaced).
#define F32_WARPS FORCE32_WARPS
#define F32_MINB FORCE32_CTAS_PER_SM
#define F32_CHUNK 448
#define F32_RING 512
#define F32_DCAP FORCE32_DCAP
// per warp: staged chunk (float4 + index), the ring, the group's agents,
// their sums (float4 each) and positions (three doubles), bounds and the two
// counts (one word each)
#define F32_WARP_SMEM (F32_CHUNK * 20 + F32_RING * 4 + 32 * 16 * 2 + 32 * 8 * 3 + 32 * 4 * 3)

template <int MODE>
__global__ void __launch_bounds__(F32_WARPS * 32, F32_MINB) k_force32(DevBufs B, DevParams P) {
  __shared__ int s_nocc[27];
  __shared__ unsigned long long s_ndirty[27];
  __shared__ int s_next;
  __shared__ unsigned s_bcnt[64];
  __shared__ uint8_t s_order[64];
  __shared__ unsigned long long s_need;
  __shared__ long long s_o;
  __shared__ float4 s_off[27];
  __shared__ unsigned long long s_bb[F32_WARPS][6];
  __shared__ unsigned s_pre[F32_WARPS][28], s_st[F32_WARPS][28];
  extern __shared__ __align__(16) unsigned char dyn_smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float4 *const sc = (float4 *)(dyn_smem + (size_t)warp * F32_WARP_SMEM);  // staged candidates
  float4 *const ag = sc + F32_CHUNK;                                       // the group's agents
  float4 *const acc = ag + 32;                                             // their sums (f, scale)
  double *const pos_s = (double *)(acc + 32);                              // their P_t (x, y, z rows)
  uint32_t *const skj = (uint32_t *)(pos_s + 96);                          // staged: sorted index
  uint32_t *const ring = skj + F32_CHUNK;                                  // (agent << 16) | chunk index
  float *const bnd = (float *)(ring + F32_RING);                           // summed error bounds
  uint32_t *const nnb_s = (uint32_t *)(bnd + 32);                          // neighbour counts
  uint32_t *const nct_s = nnb_s + 32;                                      // contact counts
  const size_t dbase = ((size_t)blockIdx.x * F32_WARPS + warp) * F32_DCAP;
  float4 *const dc = B.defer_c + dbase;  // deferred: FP32 contribution, bound
  uint2 *const dw = B.defer_w + dbase;   // deferred: sorted index, agent | kind

  DevCounters *C = B.ctr;
  if (C->error) return;
  const AgentSet &A = *B.A;  // read at the use sites: no registers held
  const int cur = (int)(C->step & 1), nxt = cur ^ 1;
  const bool use_static = (MODE == FM_STEP) && P.detect_static && C->history_valid;
  const long long n_occ = C->n_occ;
  const long long step = C->step;
  const unsigned lt_mask = (1u << lane) - 1u;
  unsigned c_static = 0, c_moved = 0, c_cand = 0, c_nbr = 0, c_cont = 0, c_exact = 0;
  int wsim = -1;
  int fetch_phase = 0;
  if (threadIdx.x < 27) {
    const int t = threadIdx.x;
    s_off[t] = make_float4((float)(t % 3 - 1) * P.Lf, (float)((t / 3) % 3 - 1) * P.Lf, (float)(t / 9 - 1) * P.Lf, 0.f);
  }
  if (lane < 6) s_bb[warp][lane] = (lane < 3) ? ~0ull : 0ull;

  while (true) {
    __syncthreads();
    if (threadIdx.x == 0) {
      s_o = next_force_brick(B, C, n_occ, fetch_phase, use_static);
      s_next = 0;
    }
    __syncthreads();
    const long long o = s_o;
    if (o < 0) break;
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
      unsigned pre = nb_cnt;
      for (int of = 1; of < 32; of <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, pre, of);
        if (lane >= of) pre += y;
      }
      const unsigned ctot = __shfl_sync(0xffffffffu, pre, 31);
      if (lane < 27) {
        s_pre[warp][lane] = pre - nb_cnt;
        s_st[warp][lane] = nb_st;
      }
      __syncwarp();

      for (unsigned q0 = 0; q0 < nq; q0 += 32) {
        const unsigned ng = min(32u, nq - q0);
        const bool valid = (unsigned)lane < ng;
        const unsigned kq = qbase + q0 + (valid ? (unsigned)lane : 0u);
        const uint32_t iq = B.perm[kq];
        const float4 cq = B.c32[kq];
        const uint8_t fl = valid ? A.flags[iq] : (uint8_t)0;
        const bool is_static = use_static && clean && valid && !(fl & FL_CHANGED) && A.nz[iq] <= 1;
        const bool compute = valid && !is_static;
        ag[lane] = cq;
        acc[lane] = make_float4(0.f, 0.f, 0.f, 0.f);
        bnd[lane] = 0.f;
        nnb_s[lane] = 0u;
        nct_s[lane] = 0u;
        if (MODE == FM_STEP && valid && !is_static) {
          // the epilogue's P_t, fetched while the pairs are evaluated
          const unsigned sa = (unsigned)__cvta_generic_to_shared(pos_s + lane);
          asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(A.x[cur] + iq) : "memory");
          asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa + 256u), "l"(A.y[cur] + iq) : "memory");
          asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa + 512u), "l"(A.z[cur] + iq) : "memory");
          asm volatile("cp.async.commit_group;\n" ::: "memory");
        }
        const unsigned cmask = __ballot_sync(0xffffffffu, compute);
        __syncwarp();
        if (cmask) {
          unsigned dlen = 0;
          // evaluate cnt (<= 32) ring pairs starting at ring position h
          auto drain = [&](unsigned h, unsigned cnt) {
            const bool v = (unsigned)lane < cnt;
            const unsigned ent = v ? ring[(h & (F32_RING - 1)) + (unsigned)lane] : 0u;
            const unsigned a = ent >> 16, i = ent & 0xffffu;
            const float4 q = ag[a];
            const float4 c = sc[i];
            const float ex = q.x - c.x, ey = q.y - c.y, ez = q.z - c.z;
            const float d2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
            const bool band = (d2 > P.R2_lo_f) || (d2 < TINY2);
            const float s = q.w + c.w, s2 = s * s;
            const float W = fmaf(s, P.cband1, s2 * P.cband2);
            const bool exact = v && (band || (d2 > s2 - W && d2 < s2 + W));
            const bool cont = v && !exact && d2 <= s2 - W;
            float vx = 0.f, vy = 0.f, vz = 0.f, vs = 0.f, vb = 0.f;
            bool graze = false;
            if (cont) {
              const float inv_d = rsqrtf(d2);
              const float d = d2 * inv_d;
              const float delta = s - d;
              const float rbar = __fdividef(q.w * c.w, s);
              const float rd = rbar * delta;
              const float sq = rd * rsqrtf(rd);
              const float kd = P.kf * delta, gs = P.gammaf * sq;
              const float scf = (kd - gs) * inv_d;
              vx = scf * ex;
              vy = scf * ey;
              vz = scf * ez;
              vs = kd + gs;
              graze = delta < P.graze;
              if (graze) {
                // d/d(delta) of sqrt(rbar delta) is large: bound its FP32 error
                vb = (sq > 1e-18f) ? fminf(P.gammaf * rbar * P.graze_e * 0.5f * __frcp_rn(sq),
                                           P.gammaf * sqrtf(rbar * P.graze_e))
                                   : P.gammaf * sqrtf(rbar * P.graze_e);
              }
            }
            const bool defer = exact || graze;
            const unsigned dbal = __ballot_sync(0xffffffffu, defer);
            if (dbal) {
              if (dlen + (unsigned)__popc(dbal) > F32_DCAP) {
                // full list: settle it now, redoing every grazing pair in it
                c_exact += settle_deferred(ExactSrc{B.perm, A.x[cur], A.y[cur], A.z[cur], B.c32, P.R2, P.k, P.gamma},
                                           qbase + q0, dlen, 0xffffffffu, dc, dw, acc, bnd, nnb_s, nct_s);
                dlen = 0;
              }
              if (defer) {
                const unsigned p = dlen + (unsigned)__popc(dbal & lt_mask);
                dc[p] = make_float4(vx, vy, vz, vb);
                dw[p] = make_uint2(skj[i], a | (exact ? DA_EXACT : 0u));
              }
              dlen += (unsigned)__popc(dbal);
            }
            const unsigned nbal = __ballot_sync(0xffffffffu, v && !exact);
            const unsigned cbal = __ballot_sync(0xffffffffu, cont);
            // segmented reduction over runs of equal agent index
            const unsigned key = v ? a : 32u + (unsigned)lane;
            const unsigned prev = __shfl_up_sync(0xffffffffu, key, 1);
            const bool is_head = lane == 0 || prev != key;
            const unsigned heads = __ballot_sync(0xffffffffu, is_head);
            const unsigned above = heads & ~(0xffffffffu >> (31 - lane));
            const unsigned end = above ? (unsigned)(__ffs(above) - 1) : 32u;
#pragma unroll
            for (int off = 1; off < 32; off <<= 1) {
              const float tx = __shfl_down_sync(0xffffffffu, vx, off);
              const float ty = __shfl_down_sync(0xffffffffu, vy, off);
              const float tz = __shfl_down_sync(0xffffffffu, vz, off);
              const float ts = __shfl_down_sync(0xffffffffu, vs, off);
              const float tb = __shfl_down_sync(0xffffffffu, vb, off);
              if ((unsigned)lane + off < end) { vx += tx; vy += ty; vz += tz; vs += ts; vb += tb; }
            }
            const unsigned segm = (end == 32u ? 0xffffffffu : ((1u << end) - 1u)) & ~lt_mask;
            // a run whose agent is not above the previous run's starts a new
            // epoch; within an epoch the runs' agents are distinct
            const unsigned desc = __ballot_sync(0xffffffffu, is_head && lane > 0 && key < prev);
            const unsigned ep = (unsigned)__popc(desc & (lt_mask | (1u << lane)));
            const unsigned nep = (unsigned)__popc(desc);
            for (unsigned e = 0; e <= nep; ++e) {
              if (is_head && v && ep == e) {
                float4 t = acc[a];
                t.x += vx; t.y += vy; t.z += vz; t.w += vs;
                acc[a] = t;
                bnd[a] += vb;
                nnb_s[a] += (unsigned)__popc(nbal & segm);
                nct_s[a] += (unsigned)__popc(cbal & segm);
              }
              __syncwarp();
            }
          };

          // Producer/consumer loop: scan (agent, 32-candidate block) steps
          // until the ring holds 32 pairs, then evaluate one ring window.  A
          // chunk is restaged only once the ring is empty (its entries index
          // the staged chunk).
          unsigned head = 0, tail = 0;
          const unsigned own0 = s_pre[warp][13] + q0;  // stencil position of agent q0 itself
          unsigned cnext = 0, cstart = 0, fill = 0, nblk = 0, am = 0, a = 0, b = 0, own = 0;
          float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
          while (true) {
            while (tail - head < 32u) {
              if (am == 0) {
                if (cnext >= ctot || tail != head) break;
                // stage the next chunk (coalesced copies, box offset applied)
                cstart = cnext;
                fill = min((unsigned)F32_CHUNK, ctot - cstart);
                cnext += fill;
                __syncwarp();
                for (unsigned g0 = 0; g0 < fill; g0 += 128u) {
                  unsigned kjs[4];
                  int boxs[4];
#pragma unroll
                  for (int m = 0; m < 4; ++m) {
                    const unsigned p = cstart + g0 + lane + 32u * m;
                    int lo = 0;
#pragma unroll
                    for (int st = 16; st > 0; st >>= 1)
                      if (lo + st <= 26 && s_pre[warp][lo + st] <= p) lo += st;
                    boxs[m] = lo;
                    kjs[m] = s_st[warp][lo] + (p - s_pre[warp][lo]);
                  }
                  float4 cs[4];
#pragma unroll
                  for (int m = 0; m < 4; ++m)
                    if (g0 + lane + 32u * m < fill) cs[m] = __ldg(&B.c32[kjs[m]]);
#pragma unroll
                  for (int m = 0; m < 4; ++m) {
                    const unsigned t = g0 + lane + 32u * m;
                    if (t < fill) {
                      const float4 of = s_off[boxs[m]];
                      sc[t] = make_float4(cs[m].x + of.x, cs[m].y + of.y, cs[m].z + of.z, cs[m].w);
                      skj[t] = kjs[m];
                    }
                  }
                }
                __syncwarp();
                if (lane == 0) c_cand += (unsigned)__popc(cmask) * fill;
                nblk = (fill + 31u) >> 5;
                am = cmask;
                b = 0;
                a = (unsigned)(__ffs(am) - 1);
                q = ag[a];
                own = own0 + a - cstart;
              }
              // eight (or, for the last few, four) candidate blocks of agent a
              // per step: independent chains
              auto scan_step = [&](auto width) {
                constexpr int NW = decltype(width)::value;
                unsigned bal[NW];
#pragma unroll
                for (int u = 0; u < NW; ++u) {
                  const unsigned i = (b + u) * 32u + (unsigned)lane;
                  const float4 c = sc[min(i, (unsigned)F32_CHUNK - 1u)];
                  const float ex = q.x - c.x, ey = q.y - c.y, ez = q.z - c.z;
                  const float d2 = fmaf(ex, ex, fmaf(ey, ey, ez * ez));
                  bal[u] = __ballot_sync(0xffffffffu, i < fill && d2 < P.R2_hi_f && i != own);
                }
#pragma unroll
                for (int u = 0; u < NW; ++u) {
                  if ((bal[u] >> lane) & 1u)
                    ring[(tail + (unsigned)__popc(bal[u] & lt_mask)) & (F32_RING - 1)] = (a << 16) | ((b + u) * 32u + lane);
                  tail += (unsigned)__popc(bal[u]);
                }
                b += NW;
              };
              if (nblk - b > 4u) scan_step(std::integral_constant<int, 8>());
              else scan_step(std::integral_constant<int, 4>());
              if (b >= nblk) {
                b = 0;
                am &= am - 1;
                if (am) {
                  a = (unsigned)(__ffs(am) - 1);
                  q = ag[a];
                  own = own0 + a - cstart;
                }
              }
            }
            // the producer stops short of 32 pairs only to restage or finish
            const bool flush = tail - head < 32u;
            const unsigned cnt = min(32u, tail - head);
            if (cnt) {
              __syncwarp();
              drain(head, cnt);
            }
            if (flush) {
              head = tail = 0;  // the ring is empty now
              if (am == 0 && cnext >= ctot) break;
            } else {
              head += 32u;
            }
          }
          if (dlen) {
            // end of the group: refine the agents whose bound is too large
            const float4 t = acc[lane];
            const unsigned rmask = __ballot_sync(0xffffffffu, bnd[lane] > 0.25f * (P.rel_tol * t.w + P.abs_tol));
            c_exact += settle_deferred(ExactSrc{B.perm, A.x[cur], A.y[cur], A.z[cur], B.c32, P.R2, P.k, P.gamma},
                                       qbase + q0, dlen, rmask, dc, dw, acc, bnd, nnb_s, nct_s);
          }
        }
        if (valid && !is_static) {  // static agents were finished by the static pass
          const float4 t = acc[lane];
          const unsigned nnb = nnb_s[lane], ncont = nct_s[lane];
          c_nbr += nnb;
          c_cont += ncont;
          double px = 0.0, py = 0.0, pz = 0.0;
          if (MODE == FM_STEP) {
            // P_t, copied to shared memory asynchronously at the group's start
            asm volatile("cp.async.wait_all;\n" ::: "memory");
            px = pos_s[lane];
            py = pos_s[32 + lane];
            pz = pos_s[64 + lane];
          }
          finish_agent<1, MODE>(B, P, A, cur, nxt, step, dt, dt_f, iq, fl, is_static, t.x, t.y, t.z, 0.0, 0.0, 0.0,
                                nnb, ncont, c_static, c_moved, s_bb[warp], px, py, pz);
        }
      }
    }
  }
  if (MODE == FM_STEP) asm volatile("cp.async.wait_all;\n" ::: "memory");  // none left in flight at exit
  if (MODE == FM_STEP) flush_bbox_warp(B, P, nxt, wsim, s_bb[warp]);
  const unsigned long long t_static = wsum64(c_static), t_moved = wsum64(c_moved), t_cand = wsum64(c_cand),
                           t_nbr = wsum64(c_nbr), t_cont = wsum64(c_cont), t_exact = wsum64(c_exact);
  if (lane == 0) {
    if (t_static) atomicAdd(&C->a_static, t_static);
    if (t_moved) atomicAdd(&C->a_moved, t_moved);
    if (t_cand) atomicAdd(&C->a_cand, t_cand);
    if (t_nbr) atomicAdd(&C->a_nbr, t_nbr);
    if (t_cont) atomicAdd(&C->a_contact, t_cont);
    if (t_exact) atomicAdd(&C->a_exact, t_exact);
  }
}

__global__ void k_reset_work(DevBufs B) {
  B.ctr->work_next = 0;
  B.ctr->heavy_take[0] = B.ctr->heavy_take[1] = 0;
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
    if (i < n) c += (A.flags[i] & FL_DIVIDE) ? 1u : 0u;
  }
  unsigned tot;
  blk_scan(c, sm, &tot);
  if (threadIdx.x == 0) B.scan_a[blockIdx.x] = tot;
}

__global__ void k_div_top(DevBufs B) {
  __shared__ unsigned sm[32];
  DevCounters *C = B.ctr;
  if (C->error) return;
  const long long n = C->n;
  const long long nblk = (n + SCAN_TILE - 1) / SCAN_TILE;
  unsigned carry = 0;
  for (long long b0 = 0; b0 < nblk; b0 += blockDim.x) {
    const long long b = b0 + threadIdx.x;
    const unsigned v = (b < nblk) ? B.scan_a[b] : 0u;
    unsigned t;
    const unsigned e = blk_scan(v, sm, &t);
    if (b < nblk) B.scan_a[b] = carry + e;
    carry += t;
  }
  if (threadIdx.x == 0) C->n_div = carry;
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

__global__ void k_finish(DevBufs B) {
  DevCounters *C = B.ctr;
  if (C->error) return;
  const long long nd = C->n_div;
  C->n += nd;
  C->next_uid += (unsigned long long)nd;
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
  if (P.precision == 1 && P.lanes_fixed == 0 && (mode == FM_STEP || mode == FM_FORCES)) {
    // the FP32 form's pair-ring kernel (dynamic shared memory above 48 KB)
    constexpr int smem = F32_WARPS * F32_WARP_SMEM;
    if (mode == FM_STEP) {
      cudaFuncSetAttribute(k_force32<FM_STEP>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      k_force32<FM_STEP><<<c.force32_blocks, F32_WARPS * 32, smem, s>>>(B, P);
    } else {
      cudaFuncSetAttribute(k_force32<FM_FORCES>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
      k_force32<FM_FORCES><<<c.force32_blocks, F32_WARPS * 32, smem, s>>>(B, P);
    }
    return;
  }
  const int g = c.force_blocks;
#define LF(PR, MO) k_force<PR, MO><<<g, FORCE_WARPS * 32, 0, s>>>(B, P)
  if (P.precision == 0) {
    switch (mode) {
      case FM_STEP: LF(0, FM_STEP); break;
      case FM_FORCES: LF(0, FM_FORCES); break;
      case FM_COUNT_NBR: LF(0, FM_COUNT_NBR); break;
      default: LF(0, FM_LIST_NBR); break;
    }
  } else {
    switch (mode) {
      case FM_STEP:
        if (!P.walk && !P.grow) k_force<1, FM_STEP, true><<<g, FORCE_WARPS * 32, 0, s>>>(B, P);
        else LF(1, FM_STEP);
        break;
      case FM_FORCES: LF(1, FM_FORCES); break;
      case FM_COUNT_NBR: LF(1, FM_COUNT_NBR); break;
      default: LF(1, FM_LIST_NBR); break;
    }
  }
#undef LF
}

void launch_divide(const DevBufs &B, const DevParams &P, const LaunchCfg &c, cudaStream_t s) {
  k_div_reduce<<<c.agent_scan_blocks, SCAN_THREADS, 0, s>>>(B);
  k_div_top<<<1, 1024, 0, s>>>(B);
  k_div_write<<<c.agent_scan_blocks, SCAN_THREADS, 0, s>>>(B, P);
}

void launch_finish(const DevBufs &B, const DevParams &P, cudaStream_t s) {
  (void)P;
  k_finish<<<1, 1, 0, s>>>(B);
}

void launch_nbr_offsets(const DevBufs &B, const DevParams &P, cudaStream_t s) {
  (void)P;
  k_nbr_offsets<<<1, 1024, 0, s>>>(B);
}
