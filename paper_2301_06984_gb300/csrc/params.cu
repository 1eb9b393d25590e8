// params.cu -- the device-side parameters of a simulation: derived
// constants of the fixed-point local frame, the FP32 error bands that keep
// the neighbour and contact decisions equal to FP64's, and the error bound of
// an FP32 overlap used for the grazing contacts.
#include <algorithm>
#include <cmath>

#include "bdm_internal.cuh"
#include "bdm.h"

namespace {
inline double pow2i(int e) { return std::ldexp(1.0, e); }
}  // namespace

DevParams make_dev_params(const bdm_params &P) {
  DevParams d{};
  d.R = P.interaction_radius;
  d.R2 = d.R * d.R;
  d.L = P.box_edge > 0.0 ? P.box_edge : d.R;
  d.dt = P.dt;
  d.dmax = P.max_displacement;
  d.k = P.k;
  d.gamma = P.gamma;
  d.adherence = P.adherence;
  d.growth = P.growth_per_step;
  d.divide_volume = P.divide_volume;
  d.ratio_lo = P.ratio_lo;
  d.ratio_hi = P.ratio_hi;
  d.walk_step = P.walk_step;
  d.seed = P.seed;
  d.precision = P.precision;
  d.detect_static = P.detect_static ? 1 : 0;
  d.sort_every = P.sort_every;
  d.n_sims = P.n_sims;
  d.keep_forces = P.keep_forces ? 1 : 0;
  d.grow = P.growth_per_step > 0.0 ? 1 : 0;
  d.walk = P.walk_step > 0.0 ? 1 : 0;
  d.death_prob = P.death_prob;
  d.n_types = P.n_types > 1 ? P.n_types : 0;
  d.curve = P.curve;
  for (int e = 0; e < 16; ++e) {
    d.type_k[e] = d.n_types ? P.type_k[e] : P.k;
    d.type_gamma[e] = d.n_types ? P.type_gamma[e] : P.gamma;
  }
  d.die = P.death_prob > 0.0 ? 1 : 0;
  // u = k 2^-53 (k an integer below 2^53) is below p iff k < ceil(p 2^53)
  d.death_thr = P.death_prob >= 1.0 ? (1ull << 53) : (uint64_t)std::ceil(P.death_prob * 9007199254740992.0);
  // fixed-point local coordinates: L 2^s < 2^29, box step a multiple of 128
  int lg = (int)std::ceil(std::log2(d.L * 1.0000001));
  int sft = 29 - lg;
  if (sft > 40) sft = 40;
  if (sft < 0) sft = 0;
  d.fix_shift = sft;
  // contact_df: a contact's coordinate differences (|D| < R) in fixed point
  // 2^-s with |D| 2^s < 2^46 (two exact 24-bit halves), at most 2^-40 um
  {
    const int lr = (int)std::ceil(std::log2(std::max(d.R, 1.0) * 1.0000001));
    d.df_shift = std::max(0, std::min(40, 46 - lr));
  }
  double Lfix = std::round(d.L * pow2i(sft) / 128.0) * 128.0;
  d.L_fix = (long long)Lfix;
  d.Lf = (float)(Lfix * pow2i(-sft));
  d.invLf = (float)(1.0 / d.L);
  d.box_eps = (float)pow2i(-22);
  // error bound E of an FP32 coordinate difference (um): truncation and
  // int->float rounding of both local coordinates (<= 130 units of 2^-s),
  // plus the two FP32 operations forming it (<= 2^-22 * 3 L)
  const double E = 256.0 * pow2i(-sft) + pow2i(-22) * 3.0 * d.L;
  const double R = d.R;
  const double W = 2.0 * (2.0 * std::sqrt(3.0) * R * E + 3.0 * pow2i(-23) * R * R + 4.0 * pow2i(-52) * R * R);
  d.Rf = (float)R;
  d.R2_lo_f = (float)(d.R2 - W);
  d.R2_hi_f = (float)(d.R2 + W);
  // grazing contacts: an overlap error e changes gamma sqrt(rbar delta) by up
  // to gamma sqrt(rbar) e / (2 sqrt(delta)); overlaps below `graze` are summed
  // apart and redone in FP64 when their bound is not small against the
  // agent's tolerance 2e-5 * sum(k delta + gamma sqrt(rbar delta)) + 1e-6
  d.graze = 0.2f;
  {
    // error bound of an FP32 overlap delta = s - d: each component of the
    // difference carries the conversion of both local coordinates (<= 17
    // units of 2^-s each: truncation to fixed point, int->float rounding) and
    // the two FP32 operations forming it (<= half an ulp of a value below
    // 2.02 L each); d adds the rounding of d^2 (1.5 2^-24 d), rsqrtf (2 ulp)
    // and the product d^2 rsqrt(d^2) (2^-24 d), with d below 1.01 R; a
    // grazing pair has s = d + delta below 1.01 R + graze, and the rounding of
    // s = r_i + r_j and of s - d adds 2^-24 (s + graze)
    const double half_ulp = std::ldexp(1.0, (int)std::ceil(std::log2(2.02 * d.L)) - 25);
    const double Ec = 34.0 * pow2i(-sft) + 2.0 * half_ulp;
    const double Rm = 1.01 * R;
    d.graze_e = (float)(std::sqrt(3.0) * Ec + (1.5 * pow2i(-24) + pow2i(-22) + pow2i(-24)) * Rm +
                        pow2i(-24) * (Rm + 2.0 * (double)d.graze));
    // the difference vector's error is at most sqrt(3) Ec, so the unit
    // direction of a pair at distance d is off by at most sqrt(3) Ec / d
    // (5e-6 / d at R = L = 11 um): pairs closer than 0.5 um, where that
    // reaches 1e-5 of the pair's force, are evaluated in FP64
    d.close2 = 0.25f;
    // grazing contacts shallower than 2e-3 um go to FP64 in place: above it
    // the bound gamma sqrt(rbar) graze_e / (2 sqrt(delta)) of one contact
    // stays near 2e-4, a small part of a dense agent's tolerance
    d.graze_exact = 2e-3f;
  }
  d.rel_tol = 2e-5f;
  d.abs_tol = 1e-6f;
  // below S = 4 abs_tol / rel_tol (0.2) the tolerance rel_tol S + abs_tol is
  // under 5e-6, a few times the FP32 error of one contact (the coordinates'
  // rounding, about 1e-6 um), so such agents are evaluated in FP64
  d.low_scale = 4.0f * d.abs_tol / d.rel_tol;
  d.cband1 = (float)(4.0 * std::sqrt(3.0) * E);
  d.cband2 = (float)(10.0 * pow2i(-23));
  d.lanes_fixed = FORCE_LANES_DEFAULT;
  d.brick_class = 0;
  d.light_max = FORCE_LIGHT_MAX;
  d.kf = (float)P.k;
  d.gammaf = (float)P.gamma;
  d.dmaxf = (float)P.max_displacement;
  d.adherencef = (float)P.adherence;
  d.walkf = (float)P.walk_step;
  return d;
}

// device parameters of a parameter block (also used by bdm_forces_noalloc)

DevParams make_dev_params_for(const bdm_params &P) { return make_dev_params(P); }
