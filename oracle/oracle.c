/*
 * oracle.c -- plain, slow FP64 CPU oracle for one mechanical-interaction
 * iteration over spherical agents (BioDynaMo, PPoPP'23, arXiv 2301.06984).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code, header, table or constant
 * generator with the CUDA library; the two are written independently from
 * the paper and the contract below.
 *
 * Build: cc -O2 -std=c11 -ffp-contract=off -fno-fast-math -fPIC -shared
 * (-ffp-contract=off matters: aarch64 GCC contracts a*b+c into an FMA by
 * default, which would change the rounding of every expression below).
 *
 * What each function follows (sections of the paper):
 *   Algorithm 1 (simulation loop)           -> orc_step ordering
 *   Sec. 3.1 (uniform grid, 3x3x3 boxes)     -> grid geometry, box lists
 *   Sec. 3.2 (additions at end of iteration)-> division merge (parent order)
 *   Sec. 3.2 (removal in five steps)         -> orc_remove (swap from the tail)
 *   Sec. 4.2 (Morton order, gap/offset DFS)  -> orc_morton_offsets, sort step
 *   Sec. 4.2 (Hilbert order, compared there) -> orc_hilbert3, orc_curve_order
 *   Sec. 5  (static-agent conditions i-iv)   -> static contract
 *   Sec. 5  defers the pair force to Cortex3D without a formula; the force
 *   used here is F = k*delta - gamma*sqrt(rbar*delta) along the centre line,
 *   delta = r_i + r_j - d, rbar = r_i r_j / (r_i + r_j), k = 2, gamma = 1.
 *   Sec. 6.5 (cell sorting, differential adhesion between cell types)  ->
 *   with n_types > 1 the pair's constants are k and gamma of its two types,
 *   the type being bits 4-5 of the agent's behaviour byte.
 *
 * Pins (tests/test_oracle_pins.py): brute-force O(N^2) neighbour sets, the
 * hand-worked two/three-sphere forces, antisymmetry, translation invariance,
 * the 3x3-in-4x4 Morton example of Sec. 4.2, brute-force Morton ranks,
 * Philox against numpy's Philox bit generator, cube root against numpy,
 * static-skip == no-skip trajectories, division invariants.
 * Parity unpinned: the division geometry and the random-walk direction have
 * no printed reference; only their invariants are pinned.  Removal is pinned
 * by hand-worked examples of its five steps and by invariants; which agents
 * die (a Philox draw per agent and iteration) has no printed reference.
 */
#include <math.h>
#ifdef ORC_OPENMP
#include <omp.h>
#endif
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)
#define ORC_ECAPACITY (-4)

#define BEH_GROW 1u
#define BEH_WALK 2u
#define BEH_DIE 4u
#define TYPE_OF(beh) (((beh) >> 4) & 3u)

typedef struct {
  double R;          /* interaction radius: neighbour iff d^2 < R^2, j != i   */
  double L;          /* box edge, >= R                                         */
  double dt;         /* time step (used when dt_sim is NULL)                   */
  double dmax;       /* displacement clamp                                     */
  double k, gamma;   /* force constants                                        */
  double adherence;  /* no displacement if |sum F| <= adherence                */
  int32_t detect_static;
  int32_t sort_every;
  double growth;         /* volume added per iteration to GROW agents          */
  double divide_volume;  /* divide when volume >= this                          */
  double ratio_lo, ratio_hi;
  double walk_step;      /* random-walk step length for WALK agents             */
  uint64_t seed;
  double death_prob;     /* per-iteration probability that a DIE agent is removed */
  int32_t n_types;       /* > 1: per-type-pair force constants below              */
  int32_t curve;         /* storage order of the sort step: 0 Morton, 1 Hilbert   */
  double type_k[16];     /* k of the types (a, b) at [4 a + b]                    */
  double type_gamma[16]; /* gamma of the types (a, b) at [4 a + b]                */
} orc_params;

typedef struct {
  int64_t n, cap;
  int32_t n_sims, history_valid;
  double *x, *y, *z, *diam, *vol;
  uint64_t *uid;
  uint8_t *beh;
  int64_t *sim_off;      /* n_sims + 1 entries; agents of sim s are [off[s], off[s+1]) */
  const double *dt_sim;  /* nullable: per-simulation time step                */
  uint8_t *changed;      /* history: agent changed during the previous step   */
  int32_t *nz;           /* history: contacts (delta > 0) in the previous step */
  double *px, *py, *pz;  /* history: positions before the previous step       */
  int64_t step;
  uint64_t next_uid;
  /* outputs of the last orc_step (nullable arrays) */
  double *fx, *fy, *fz;
  uint8_t *is_static;
  int64_t n_divided, n_static, n_coincident;
  /* history: positions (at the start of the previous step) of the agents
   * removed during it; their boxes are dirty for the static test */
  double *gx, *gy, *gz;
  int64_t n_ghost;
  int64_t n_removed; /* output: agents removed by the last orc_step */
} orc_state;

/* ------------------------------------------------------------------------ */
/* Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11), written from the      */
/* published definition: 10 rounds, each (L0,R0,L1,R1) -> two 64x64->128     */
/* multiplies by the round constants, key bumped by the Weyl constants.      */
/* ------------------------------------------------------------------------ */
static void mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo) {
  unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
  *lo = (uint64_t)p;
  *hi = (uint64_t)(p >> 64);
}

void orc_philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4]) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
  const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
  uint64_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint64_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += W0; k1 += W1; }
    uint64_t hi0, lo0, hi1, lo1;
    mulhilo64(M0, c0, &hi0, &lo0);
    mulhilo64(M1, c2, &hi1, &lo1);
    uint64_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* uniform double in [0,1) from the top 53 bits of a 64-bit word */
static double u53(uint64_t w) { return (double)(w >> 11) * (1.0 / 9007199254740992.0); }

/* Random stream ids: counter = (uid, step, purpose, draw), key = (seed, 0). */
#define PURPOSE_RATIO 0u
#define PURPOSE_AXIS 1u
#define PURPOSE_WALK 2u
#define PURPOSE_DEATH 3u

/* Unit vector by Marsaglia's (1972) disc method: draw x1, x2 uniform in
 * [-1,1) until 0 < s = x1^2 + x2^2 < 1; then
 * u = (2 x1 sqrt(1-s), 2 x2 sqrt(1-s), 1 - 2s).  Each Philox block gives two
 * attempts: words (0,1) then (2,3); the draw index advances per block. */
void orc_unit_vector(uint64_t seed, uint64_t uid, uint64_t step, uint64_t purpose, double out[3]) {
  uint64_t key[2] = {seed, 0};
  for (uint64_t draw = 0;; ++draw) {
    uint64_t ctr[4] = {uid, step, purpose, draw}, w[4];
    orc_philox4x64_10(ctr, key, w);
    for (int a = 0; a < 2; ++a) {
      double x1 = 2.0 * u53(w[2 * a]) - 1.0;
      double x2 = 2.0 * u53(w[2 * a + 1]) - 1.0;
      double s = x1 * x1 + x2 * x2;
      if (s > 0.0 && s < 1.0) {
        double q = sqrt(1.0 - s);
        out[0] = (2.0 * x1) * q;
        out[1] = (2.0 * x2) * q;
        out[2] = 1.0 - 2.0 * s;
        return;
      }
    }
  }
}

double orc_uniform(uint64_t seed, uint64_t uid, uint64_t step, uint64_t purpose) {
  uint64_t key[2] = {seed, 0}, ctr[4] = {uid, step, purpose, 0}, w[4];
  orc_philox4x64_10(ctr, key, w);
  return u53(w[0]);
}

/* ------------------------------------------------------------------------ */
/* Cube root by Newton's method on y^3 = m after an exact power-of-two       */
/* range reduction (x = m 2^(3q), m in [0.5, 4)).  Six Newton steps from a  */
/* linear first guess; every operation is a single IEEE operation so the     */
/* CUDA library reaches the same bits with the same sequence.               */
/* ------------------------------------------------------------------------ */
double orc_cbrt(double x) {
  if (x == 0.0 || !isfinite(x)) return x;
  double sgn = 1.0;
  if (x < 0.0) { sgn = -1.0; x = -x; }
  int e;
  double m = frexp(x, &e); /* x = m 2^e, m in [0.5, 1) */
  int q = e / 3, r = e % 3;
  if (r < 0) { r += 3; q -= 1; }
  m = ldexp(m, r); /* m in [0.5, 4), x = m 2^(3q) */
  double y = 0.6 + 0.25 * m;
  for (int it = 0; it < 6; ++it) {
    double y2 = y * y;
    double y3 = y2 * y;
    y = y - (y3 - m) / (3.0 * y2);
  }
  return sgn * ldexp(y, q);
}

/* ------------------------------------------------------------------------ */
/* Hilbert index of the cell (x, y, z) of a 2^bits cube, by Skilling's        */
/* transpose method (J. Skilling, "Programming the Hilbert curve", AIP Conf. */
/* Proc. 707, 2004): going down from the top bit, undo on the lower bits the */
/* reflection or the exchange of axes the curve applies in the sub-cube the */
/* point lies in; Gray-encode the axes; then read the index with x's bit    */
/* most significant in each 3-bit digit.                                    */
/* ------------------------------------------------------------------------ */
uint64_t orc_hilbert3(uint64_t x, uint64_t y, uint64_t z, int bits) {
  if (bits <= 0) return 0;
  uint64_t X[3] = {x, y, z};
  const uint64_t M = 1ULL << (bits - 1);
  for (uint64_t Q = M; Q > 1; Q >>= 1) {
    const uint64_t P = Q - 1;
    for (int i = 0; i < 3; ++i) {
      if (X[i] & Q) {
        X[0] ^= P; /* reflect the lower bits of axis 0 */
      } else {     /* exchange the lower bits of axes 0 and i */
        const uint64_t t = (X[0] ^ X[i]) & P;
        X[0] ^= t;
        X[i] ^= t;
      }
    }
  }
  X[1] ^= X[0]; /* Gray encode */
  X[2] ^= X[1];
  uint64_t t = 0;
  for (uint64_t Q = M; Q > 1; Q >>= 1)
    if (X[2] & Q) t ^= Q - 1;
  for (int i = 0; i < 3; ++i) X[i] ^= t;
  uint64_t h = 0;
  for (int b = bits - 1; b >= 0; --b)
    for (int i = 0; i < 3; ++i) h = (h << 1) | ((X[i] >> b) & 1ULL);
  return h;
}

/* ------------------------------------------------------------------------ */
/* Morton codes and the gap/offset algorithm of Sec. 4.2                     */
/* ------------------------------------------------------------------------ */
/* x -> bit 3k, y -> bit 3k+1, z -> bit 3k+2 (21 bits per axis) */
uint64_t orc_morton3(uint64_t x, uint64_t y, uint64_t z) {
  uint64_t c = 0;
  for (int b = 0; b < 21; ++b) {
    c |= ((x >> b) & 1ULL) << (3 * b);
    c |= ((y >> b) & 1ULL) << (3 * b + 1);
    c |= ((z >> b) & 1ULL) << (3 * b + 2);
  }
  return c;
}

/* 2D variant (x -> bit 2k, y -> bit 2k+1), for the worked example */
uint64_t orc_morton2(uint64_t x, uint64_t y) {
  uint64_t c = 0;
  for (int b = 0; b < 31; ++b) {
    c |= ((x >> b) & 1ULL) << (2 * b);
    c |= ((y >> b) & 1ULL) << (2 * b + 1);
  }
  return c;
}

typedef struct {
  int D;
  int64_t n[3];
  int64_t box_counter, offset;
  int found_gap;
  int64_t n_out, cap;
  int64_t *out_counter, *out_offset;
} gap_walk;

/* number of in-domain leaves under a node [lo, lo + s) per axis */
static int64_t node_inside(const gap_walk *g, const int64_t lo[3], int64_t s) {
  int64_t cnt = 1;
  for (int d = 0; d < g->D; ++d) {
    int64_t hi = lo[d] + s;
    if (hi > g->n[d]) hi = g->n[d];
    int64_t w = hi - lo[d];
    if (w <= 0) return 0;
    cnt *= w;
  }
  return cnt;
}

/* Depth-first traversal of the implicit quad/octree in Morton order.  A node
 * is complete (all leaves inside), empty (none inside) or partial; only
 * partial inner nodes are descended.  Complete nodes and inside leaves emit
 * (box_counter, offset) when a gap preceded them, then advance box_counter by
 * their leaf count; empty nodes advance offset and set found_gap. */
static void gap_dfs(gap_walk *g, const int64_t lo[3], int64_t s) {
  int64_t leaves = 1;
  for (int d = 0; d < g->D; ++d) leaves *= s;
  int64_t inside = node_inside(g, lo, s);
  if (inside == leaves) {
    if (g->found_gap) {
      if (g->n_out < g->cap) {
        g->out_counter[g->n_out] = g->box_counter;
        g->out_offset[g->n_out] = g->offset;
      }
      g->n_out++;
      g->found_gap = 0;
    }
    g->box_counter += leaves;
    return;
  }
  if (inside == 0) {
    g->offset += leaves;
    g->found_gap = 1;
    return;
  }
  int64_t h = s / 2;
  int nchild = 1 << g->D;
  for (int c = 0; c < nchild; ++c) {
    int64_t clo[3] = {0, 0, 0};
    for (int d = 0; d < g->D; ++d) clo[d] = lo[d] + (((c >> d) & 1) ? h : 0);
    gap_dfs(g, clo, h);
  }
}

/* Returns the number of (box_counter, offset) entries; writes at most cap.
 * D = 2 or 3, n = grid extent per axis.  Morton rank of an in-domain code c is
 * c - offset_e with e the last entry whose box_counter + offset_e <= c. */
int64_t orc_morton_offsets(int32_t D, const int64_t *n, int64_t *out_counter, int64_t *out_offset,
                           int64_t cap) {
  if (D < 2 || D > 3) return ORC_EINVAL;
  gap_walk g;
  memset(&g, 0, sizeof g);
  g.D = D;
  int64_t mx = 1;
  for (int d = 0; d < D; ++d) {
    if (n[d] <= 0) return 0;
    g.n[d] = n[d];
    if (n[d] > mx) mx = n[d];
  }
  int64_t s = 1;
  while (s < mx) s *= 2;
  g.found_gap = 1;
  g.cap = cap;
  g.out_counter = out_counter;
  g.out_offset = out_offset;
  int64_t lo[3] = {0, 0, 0};
  gap_dfs(&g, lo, s);
  return g.n_out;
}

/* ------------------------------------------------------------------------ */
/* Grid (Sec. 3.1): per simulation, lo_d = floor(min_d/L) L - L and          */
/* n_d = floor((max_d - lo_d)/L) + 2 boxes; an agent's box is                */
/* floor((p_d - lo_d)/L) clamped to [1, n_d - 2], so every 3x3x3 stencil    */
/* stays inside the grid.                                                    */
/* ------------------------------------------------------------------------ */
typedef struct {
  double lo[3];
  int64_t nb[3];
} sim_grid;

static void grid_geometry(const orc_state *st, const orc_params *P, int s, sim_grid *g) {
  int64_t a0 = st->sim_off[s], a1 = st->sim_off[s + 1];
  double mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (int64_t i = a0; i < a1; ++i) {
    double p[3] = {st->x[i], st->y[i], st->z[i]};
    for (int d = 0; d < 3; ++d) {
      if (p[d] < mn[d]) mn[d] = p[d];
      if (p[d] > mx[d]) mx[d] = p[d];
    }
  }
  for (int d = 0; d < 3; ++d) {
    if (a1 <= a0) { g->lo[d] = 0.0; g->nb[d] = 0; continue; }
    g->lo[d] = floor(mn[d] / P->L) * P->L - P->L;
    g->nb[d] = (int64_t)floor((mx[d] - g->lo[d]) / P->L) + 2;
  }
}

static int64_t box_coord_raw(double p, double lo, double L) { return (int64_t)floor((p - lo) / L); }

static int64_t box_coord(double p, double lo, double L, int64_t n) {
  int64_t b = box_coord_raw(p, lo, L);
  if (b < 1) b = 1;
  if (b > n - 2) b = n - 2;
  return b;
}

static int64_t box_linear(const sim_grid *g, int64_t bx, int64_t by, int64_t bz) {
  return (bz * g->nb[1] + by) * g->nb[0] + bx;
}

typedef struct {
  int64_t key; /* (sim, linear box) flattened via per-sim base */
  int64_t idx;
} key_idx;

static int cmp_key_idx(const void *a, const void *b) {
  const key_idx *p = (const key_idx *)a, *q = (const key_idx *)b;
  if (p->key != q->key) return p->key < q->key ? -1 : 1;
  if (p->idx != q->idx) return p->idx < q->idx ? -1 : 1;
  return 0;
}

static int cmp_i64(const void *a, const void *b) {
  int64_t p = *(const int64_t *)a, q = *(const int64_t *)b;
  return p < q ? -1 : (p > q ? 1 : 0);
}

typedef struct {
  int n_sims;
  sim_grid *g;
  int64_t *base;   /* per-sim base of the flattened linear box id */
  int64_t *sim_of; /* per agent */
  int64_t *bx, *by, *bz;
  key_idx *sorted; /* agents sorted by (flattened box, storage index) */
  int64_t n;
} grid_t;

static void grid_free(grid_t *G) {
  free(G->g); free(G->base); free(G->sim_of); free(G->bx); free(G->by); free(G->bz); free(G->sorted);
  memset(G, 0, sizeof *G);
}

static int grid_build(const orc_state *st, const orc_params *P, grid_t *G) {
  memset(G, 0, sizeof *G);
  int64_t n = st->n;
  G->n = n;
  G->n_sims = st->n_sims;
  G->g = (sim_grid *)calloc((size_t)st->n_sims, sizeof(sim_grid));
  G->base = (int64_t *)calloc((size_t)st->n_sims + 1, sizeof(int64_t));
  G->sim_of = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  G->bx = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  G->by = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  G->bz = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  G->sorted = (key_idx *)malloc(sizeof(key_idx) * (size_t)(n > 0 ? n : 1));
  if (!G->g || !G->base || !G->sim_of || !G->bx || !G->by || !G->bz || !G->sorted) {
    grid_free(G);
    return ORC_ENOMEM;
  }
  for (int s = 0; s < st->n_sims; ++s) {
    grid_geometry(st, P, s, &G->g[s]);
    G->base[s + 1] = G->base[s] + G->g[s].nb[0] * G->g[s].nb[1] * G->g[s].nb[2];
  }
  for (int s = 0; s < st->n_sims; ++s) {
    const sim_grid *g = &G->g[s];
    for (int64_t i = st->sim_off[s]; i < st->sim_off[s + 1]; ++i) {
      G->sim_of[i] = s;
      G->bx[i] = box_coord(st->x[i], g->lo[0], P->L, g->nb[0]);
      G->by[i] = box_coord(st->y[i], g->lo[1], P->L, g->nb[1]);
      G->bz[i] = box_coord(st->z[i], g->lo[2], P->L, g->nb[2]);
      G->sorted[i].key = G->base[s] + box_linear(g, G->bx[i], G->by[i], G->bz[i]);
      G->sorted[i].idx = i;
    }
  }
  qsort(G->sorted, (size_t)n, sizeof(key_idx), cmp_key_idx);
  return ORC_OK;
}

/* [first, last) of the agents in flattened box `key` within the sorted list */
static void grid_range(const grid_t *G, int64_t key, int64_t *first, int64_t *last) {
  int64_t lo = 0, hi = G->n;
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (G->sorted[mid].key < key) lo = mid + 1; else hi = mid;
  }
  *first = lo;
  hi = G->n;
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (G->sorted[mid].key <= key) lo = mid + 1; else hi = mid;
  }
  *last = lo;
}

/* ------------------------------------------------------------------------ */
/* Pair force and neighbour enumeration                                      */
/* ------------------------------------------------------------------------ */
typedef struct {
  double fx, fy, fz;
  double scale;     /* sum over contacts of k*delta + gamma*sqrt(rbar*delta) (term magnitudes) */
  double scale_abs; /* sum over contacts of |k*delta - gamma*sqrt(rbar*delta)| (pair-force magnitudes) */
  int32_t nz;   /* contacts: neighbours with delta > 0 */
  int32_t nnb;  /* neighbours: d^2 < R^2, j != i */
  int32_t ncoincident;
} force_acc;

/* Canonical order: stencil boxes with dz outermost, then dy, then dx, each in
 * -1, 0, +1; inside a box, ascending storage index. */
static void force_on(const orc_state *st, const orc_params *P, const grid_t *G, int64_t i, force_acc *a,
                     int64_t *nbr_out, int64_t *nbr_cnt) {
  int s = (int)G->sim_of[i];
  const sim_grid *g = &G->g[s];
  double R2 = P->R * P->R;
  double xi = st->x[i], yi = st->y[i], zi = st->z[i], ri = st->diam[i] * 0.5;
  a->fx = a->fy = a->fz = 0.0;
  a->scale = 0.0;
  a->scale_abs = 0.0;
  a->nz = a->nnb = a->ncoincident = 0;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        int64_t key = G->base[s] + box_linear(g, G->bx[i] + dx, G->by[i] + dy, G->bz[i] + dz);
        int64_t f, l;
        grid_range(G, key, &f, &l);
        for (int64_t m = f; m < l; ++m) {
          int64_t j = G->sorted[m].idx;
          if (j == i) continue;
          double ddx = xi - st->x[j], ddy = yi - st->y[j], ddz = zi - st->z[j];
          double d2 = (ddx * ddx + ddy * ddy) + ddz * ddz;
          if (!(d2 < R2)) continue;
          a->nnb++;
          if (nbr_out) nbr_out[(*nbr_cnt)++] = j;
          if (d2 == 0.0) { a->ncoincident++; continue; }
          double d = sqrt(d2);
          double rj = st->diam[j] * 0.5;
          double delta = (ri + rj) - d;
          if (!(delta > 0.0)) continue;
          double rbar = (ri * rj) / (ri + rj);
          double k = P->k, gamma = P->gamma;
          if (P->n_types > 1) {
            const unsigned ab = 4u * TYPE_OF(st->beh[i]) + TYPE_OF(st->beh[j]);
            k = P->type_k[ab];
            gamma = P->type_gamma[ab];
          }
          double kd = k * delta, gs = gamma * sqrt(rbar * delta);
          double F = kd - gs;
          double sc = F / d;
          a->scale += kd + gs;
          a->scale_abs += fabs(F);
          a->fx = a->fx + sc * ddx;
          a->fy = a->fy + sc * ddy;
          a->fz = a->fz + sc * ddz;
          a->nz++;
        }
      }
}

/* ------------------------------------------------------------------------ */
/* Public helpers used by the tests                                          */
/* ------------------------------------------------------------------------ */

static int check_state(const orc_state *st, const orc_params *P) {
  if (!st || !P) return ORC_EINVAL;
  if (st->n < 0 || st->n > st->cap || st->n_sims < 1) return ORC_EINVAL;
  if (!(P->R > 0.0) || !(P->L >= P->R)) return ORC_EINVAL;
  if (st->sim_off[0] != 0 || st->sim_off[st->n_sims] != st->n) return ORC_EINVAL;
  return ORC_OK;
}

/* Per-agent box coordinates, Morton code of the box, and per-simulation grid
 * geometry (lo[3 * n_sims], nb[3 * n_sims]) of the grid the next iteration
 * builds. */
int orc_grid(const orc_state *st, const orc_params *P, int64_t *bxyz, uint64_t *morton, double *lo,
             int64_t *nb) {
  int rc = check_state(st, P);
  if (rc) return rc;
  grid_t G;
  rc = grid_build(st, P, &G);
  if (rc) return rc;
  for (int64_t i = 0; i < st->n; ++i) {
    if (bxyz) { bxyz[3 * i] = G.bx[i]; bxyz[3 * i + 1] = G.by[i]; bxyz[3 * i + 2] = G.bz[i]; }
    if (morton) morton[i] = orc_morton3((uint64_t)G.bx[i], (uint64_t)G.by[i], (uint64_t)G.bz[i]);
  }
  for (int s = 0; s < st->n_sims; ++s)
    for (int d = 0; d < 3; ++d) {
      if (lo) lo[3 * s + d] = G.g[s].lo[d];
      if (nb) nb[3 * s + d] = G.g[s].nb[d];
    }
  grid_free(&G);
  return ORC_OK;
}

typedef struct {
  int64_t sim;
  uint64_t code;
  int64_t idx;
} sort_rec;

static int cmp_sort_rec(const void *a, const void *b) {
  const sort_rec *p = (const sort_rec *)a, *q = (const sort_rec *)b;
  if (p->sim != q->sim) return p->sim < q->sim ? -1 : 1;
  if (p->code != q->code) return p->code < q->code ? -1 : 1;
  if (p->idx != q->idx) return p->idx < q->idx ? -1 : 1;
  return 0;
}

/* Stable order by (simulation, Morton code of the box): perm[k] = storage
 * index of the agent at sorted position k. */
int orc_morton_order(const orc_state *st, const orc_params *P, int64_t *perm) {
  int rc = check_state(st, P);
  if (rc) return rc;
  grid_t G;
  rc = grid_build(st, P, &G);
  if (rc) return rc;
  sort_rec *r = (sort_rec *)malloc(sizeof(sort_rec) * (size_t)(st->n > 0 ? st->n : 1));
  if (!r) { grid_free(&G); return ORC_ENOMEM; }
  for (int64_t i = 0; i < st->n; ++i) {
    r[i].sim = G.sim_of[i];
    r[i].code = orc_morton3((uint64_t)G.bx[i], (uint64_t)G.by[i], (uint64_t)G.bz[i]);
    r[i].idx = i;
  }
  qsort(r, (size_t)st->n, sizeof(sort_rec), cmp_sort_rec);
  for (int64_t k = 0; k < st->n; ++k) perm[k] = r[k].idx;
  free(r);
  grid_free(&G);
  return ORC_OK;
}

/* Neighbour lists through the grid, canonical order; CSR (off[n+1], nbr). */
int64_t orc_neighbors(const orc_state *st, const orc_params *P, int64_t *off, int64_t *nbr, int64_t cap) {
  int rc = check_state(st, P);
  if (rc) return rc;
  grid_t G;
  rc = grid_build(st, P, &G);
  if (rc) return rc;
  int64_t total = 0;
  int64_t *tmp = (int64_t *)malloc(sizeof(int64_t) * (size_t)(st->n > 0 ? st->n : 1));
  if (!tmp) { grid_free(&G); return ORC_ENOMEM; }
  off[0] = 0;
  for (int64_t i = 0; i < st->n; ++i) {
    force_acc a;
    int64_t cnt = 0;
    force_on(st, P, &G, i, &a, tmp, &cnt);
    for (int64_t m = 0; m < cnt; ++m) {
      if (total + m < cap) nbr[total + m] = tmp[m];
    }
    total += cnt;
    off[i + 1] = total;
  }
  free(tmp);
  grid_free(&G);
  return total;
}

/* Brute force O(N^2) neighbour lists (same simulation only), ascending j. */
int64_t orc_neighbors_brute(const orc_state *st, const orc_params *P, int64_t *off, int64_t *nbr, int64_t cap) {
  int rc = check_state(st, P);
  if (rc) return rc;
  double R2 = P->R * P->R;
  int64_t total = 0;
  off[0] = 0;
  for (int s = 0; s < st->n_sims; ++s) {
    for (int64_t i = st->sim_off[s]; i < st->sim_off[s + 1]; ++i) {
      for (int64_t j = st->sim_off[s]; j < st->sim_off[s + 1]; ++j) {
        if (j == i) continue;
        double ddx = st->x[i] - st->x[j], ddy = st->y[i] - st->y[j], ddz = st->z[i] - st->z[j];
        double d2 = (ddx * ddx + ddy * ddy) + ddz * ddz;
        if (d2 < R2) {
          if (total < cap) nbr[total] = j;
          total++;
        }
      }
      off[i + 1] = total;
    }
  }
  return total;
}

/* Threads the force loops run on: 1, or the OpenMP thread count of the
 * timing build. */
int orc_threads(void) {
#ifdef ORC_OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Summed pair force on selected agents (all when q == NULL), without the
 * static skip; f is 3 x nq SoA.  Optional outputs: nz (contacts), nnb
 * (neighbours), scale (sum over contacts of the magnitudes of the two force
 * terms) and scale_abs (sum over contacts of the pair-force magnitude |F_ij|,
 * the base of the FP32 form's relative force tolerance). */
int orc_forces(const orc_state *st, const orc_params *P, int64_t nq, const int64_t *q, double *f,
               int32_t *nz, int32_t *nnb, double *scale, double *scale_abs) {
  int rc = check_state(st, P);
  if (rc) return rc;
  grid_t G;
  rc = grid_build(st, P, &G);
  if (rc) return rc;
  if (!q) nq = st->n;
  for (int64_t m = 0; m < nq; ++m) {
    int64_t i = q ? q[m] : m;
    if (i < 0 || i >= st->n) { grid_free(&G); return ORC_EINVAL; }
    force_acc a;
    force_on(st, P, &G, i, &a, NULL, NULL);
    f[m] = a.fx; f[nq + m] = a.fy; f[2 * nq + m] = a.fz;
    if (nz) nz[m] = a.nz;
    if (nnb) nnb[m] = a.nnb;
    if (scale) scale[m] = a.scale;
    if (scale_abs) scale_abs[m] = a.scale_abs;
  }
  grid_free(&G);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* One iteration (Algorithm 1 with the mechanical operation of Sec. 5).      */
/* ------------------------------------------------------------------------ */
static void permute_f64(double *a, const int64_t *perm, int64_t n, double *tmp) {
  if (!a) return;
  for (int64_t k = 0; k < n; ++k) tmp[k] = a[perm[k]];
  memcpy(a, tmp, sizeof(double) * (size_t)n);
}

/* Storage order of a sort step for the curve P->curve: perm[k] = storage
 * index of the agent at sorted position k.  Morton: by the Morton code of the
 * box.  Hilbert: by the Hilbert index of the box's 4x4x4-box brick over the
 * simulation's brick grid (bits = ceil(log2) of its longest side), then by the
 * Morton code of the box inside the brick.  Both stable (storage index). */
int orc_curve_order(const orc_state *st, const orc_params *P, int64_t *perm) {
  if (P->curve != 1) return orc_morton_order(st, P, perm);
  int rc = check_state(st, P);
  if (rc) return rc;
  grid_t G;
  rc = grid_build(st, P, &G);
  if (rc) return rc;
  sort_rec *r = (sort_rec *)malloc(sizeof(sort_rec) * (size_t)(st->n > 0 ? st->n : 1));
  if (!r) { grid_free(&G); return ORC_ENOMEM; }
  for (int64_t i = 0; i < st->n; ++i) {
    const sim_grid *g = &G.g[G.sim_of[i]];
    int64_t longest = 1;
    for (int d = 0; d < 3; ++d) {
      const int64_t bricks = (g->nb[d] + 3) / 4;
      if (bricks > longest) longest = bricks;
    }
    int bits = 0;
    while ((1LL << bits) < longest) ++bits;
    const uint64_t h = orc_hilbert3((uint64_t)(G.bx[i] >> 2), (uint64_t)(G.by[i] >> 2), (uint64_t)(G.bz[i] >> 2), bits);
    r[i].sim = G.sim_of[i];
    r[i].code = (h << 6) | orc_morton3((uint64_t)(G.bx[i] & 3), (uint64_t)(G.by[i] & 3), (uint64_t)(G.bz[i] & 3));
    r[i].idx = i;
  }
  qsort(r, (size_t)st->n, sizeof(sort_rec), cmp_sort_rec);
  for (int64_t k = 0; k < st->n; ++k) perm[k] = r[k].idx;
  free(r);
  grid_free(&G);
  return ORC_OK;
}

static int apply_sort(orc_state *st, const orc_params *P) {
  int64_t n = st->n;
  if (n <= 0) return ORC_OK;
  int64_t *perm = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  double *tmp = (double *)malloc(sizeof(double) * (size_t)n);
  if (!perm || !tmp) { free(perm); free(tmp); return ORC_ENOMEM; }
  int rc = orc_curve_order(st, P, perm);
  if (rc) { free(perm); free(tmp); return rc; }
  permute_f64(st->x, perm, n, tmp);
  permute_f64(st->y, perm, n, tmp);
  permute_f64(st->z, perm, n, tmp);
  permute_f64(st->diam, perm, n, tmp);
  permute_f64(st->vol, perm, n, tmp);
  permute_f64(st->px, perm, n, tmp);
  permute_f64(st->py, perm, n, tmp);
  permute_f64(st->pz, perm, n, tmp);
  uint64_t *tu = (uint64_t *)tmp;
  for (int64_t k = 0; k < n; ++k) tu[k] = st->uid[perm[k]];
  memcpy(st->uid, tu, sizeof(uint64_t) * (size_t)n);
  int32_t *ti = (int32_t *)tmp;
  for (int64_t k = 0; k < n; ++k) ti[k] = st->nz[perm[k]];
  memcpy(st->nz, ti, sizeof(int32_t) * (size_t)n);
  uint8_t *tb = (uint8_t *)tmp;
  for (int64_t k = 0; k < n; ++k) tb[k] = st->beh[perm[k]];
  memcpy(st->beh, tb, (size_t)n);
  for (int64_t k = 0; k < n; ++k) tb[k] = st->changed[perm[k]];
  memcpy(st->changed, tb, (size_t)n);
  free(perm);
  free(tmp);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Removal (Sec. 3.2): the agent vector has no empty elements, so a removed  */
/* agent left of the new size leaves a hole that a surviving agent from the */
/* right of it fills.  The paper's five steps, on one thread, with the       */
/* removed list in ascending storage index.                                  */
/* ------------------------------------------------------------------------ */
static void move_agent(orc_state *st, int64_t from, int64_t to) {
  st->x[to] = st->x[from]; st->y[to] = st->y[from]; st->z[to] = st->z[from];
  st->px[to] = st->px[from]; st->py[to] = st->py[from]; st->pz[to] = st->pz[from];
  st->diam[to] = st->diam[from];
  if (st->vol) st->vol[to] = st->vol[from];
  st->uid[to] = st->uid[from];
  st->beh[to] = st->beh[from];
  st->changed[to] = st->changed[from];
  st->nz[to] = st->nz[from];
  if (st->fx) { st->fx[to] = st->fx[from]; st->fy[to] = st->fy[from]; st->fz[to] = st->fz[from]; }
  if (st->is_static) st->is_static[to] = st->is_static[from];
}

/* Remove the agents i < st->n with rm[i] != 0.  Returns the number of agents
 * moved (at most the number removed), or a negative error. */
int64_t orc_remove(orc_state *st, const uint8_t *rm) {
  const int64_t n = st->n;
  /* step 1: number of removed agents, the new size, two auxiliary arrays of
   * that length */
  int64_t removed = 0;
  for (int64_t i = 0; i < n; ++i) removed += rm[i] ? 1 : 0;
  const int64_t new_size = n - removed;
  if (removed == 0) return 0;
  int64_t *to_right = (int64_t *)malloc(sizeof(int64_t) * (size_t)removed);
  int64_t *to_left = (int64_t *)malloc(sizeof(int64_t) * (size_t)removed);
  uint8_t *not_to_left = (uint8_t *)calloc((size_t)removed, 1);
  if (!to_right || !to_left || !not_to_left) {
    free(to_right); free(to_left); free(not_to_left);
    return ORC_ENOMEM;
  }
  /* step 2: a removed agent left of the new size is a hole (to_right holds
   * its index, the others hold "none"); one right of it marks not_to_left at
   * idx - new_size */
  const int64_t NONE = -1;
  int64_t k = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (!rm[i]) continue;
    if (i < new_size) {
      to_right[k] = i;
    } else {
      to_right[k] = NONE;
      not_to_left[i - new_size] = 1;
    }
    ++k;
  }
  /* step 3: move the entries that mean a swap to the front: the holes in
   * to_right, and, with not_to_left read as to_left, each zero entry as
   * array index + new_size (a survivor right of the new size) */
  int64_t swaps_right = 0, swaps_left = 0;
  for (int64_t e = 0; e < removed; ++e)
    if (to_right[e] != NONE) to_right[swaps_right++] = to_right[e];
  for (int64_t e = 0; e < removed; ++e)
    if (!not_to_left[e]) to_left[swaps_left++] = e + new_size;
  /* step 4: the swaps (the prefix sum of the per-thread swap counts is
   * trivial with one thread); both lists have one entry per hole */
  const int64_t swaps = swaps_right < swaps_left ? swaps_right : swaps_left;
  for (int64_t e = 0; e < swaps; ++e) move_agent(st, to_left[e], to_right[e]);
  /* step 5: shrink */
  st->n = new_size;
  free(to_right); free(to_left); free(not_to_left);
  return swaps;
}

static int agent_dt(const orc_state *st, const orc_params *P, int64_t sim, double *dt) {
  *dt = st->dt_sim ? st->dt_sim[sim] : P->dt;
  return 0;
}

int orc_step(orc_state *st, const orc_params *P) {
  int rc = check_state(st, P);
  if (rc) return rc;
  if (st->n_sims > 1 && (P->growth > 0.0 || P->death_prob > 0.0))
    return ORC_EINVAL; /* ensembles neither divide nor remove */
  if (!st->gx || !st->gy || !st->gz) return ORC_EINVAL;
  int64_t n = st->n;
  const double pi = 3.141592653589793;

  /* 1. sort step: stable Morton order of grid t, before the grid build */
  if (P->sort_every > 0 && (st->step % P->sort_every) == 0) {
    rc = apply_sort(st, P);
    if (rc) return rc;
  }

  /* 2. grid on P_t */
  grid_t G;
  rc = grid_build(st, P, &G);
  if (rc) return rc;

  /* 3. static marking: dirty boxes hold the old or the new position of an
   *    agent that changed during the previous step */
  uint8_t *stat = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
  int64_t *dirty = (int64_t *)malloc(sizeof(int64_t) * (size_t)(2 * n + st->n_ghost + 1));
  if (!stat || !dirty) { free(stat); free(dirty); grid_free(&G); return ORC_ENOMEM; }
  int64_t ndirty = 0;
  int use_static = P->detect_static && st->history_valid;
  if (use_static) {
    for (int64_t j = 0; j < n; ++j) {
      if (!st->changed[j]) continue;
      int s = (int)G.sim_of[j];
      const sim_grid *g = &G.g[s];
      dirty[ndirty++] = G.base[s] + box_linear(g, G.bx[j], G.by[j], G.bz[j]);
      int64_t ox = box_coord_raw(st->px[j], g->lo[0], P->L);
      int64_t oy = box_coord_raw(st->py[j], g->lo[1], P->L);
      int64_t oz = box_coord_raw(st->pz[j], g->lo[2], P->L);
      if (ox >= 0 && ox < g->nb[0] && oy >= 0 && oy < g->nb[1] && oz >= 0 && oz < g->nb[2])
        dirty[ndirty++] = G.base[s] + box_linear(g, ox, oy, oz);
    }
    /* agents removed during the previous step: their last boxes are dirty */
    for (int64_t k = 0; k < st->n_ghost; ++k) {
      const sim_grid *g = &G.g[0];
      int64_t ox = box_coord_raw(st->gx[k], g->lo[0], P->L);
      int64_t oy = box_coord_raw(st->gy[k], g->lo[1], P->L);
      int64_t oz = box_coord_raw(st->gz[k], g->lo[2], P->L);
      if (ox >= 0 && ox < g->nb[0] && oy >= 0 && oy < g->nb[1] && oz >= 0 && oz < g->nb[2])
        dirty[ndirty++] = G.base[0] + box_linear(g, ox, oy, oz);
    }
    qsort(dirty, (size_t)ndirty, sizeof(int64_t), cmp_i64);
    for (int64_t i = 0; i < n; ++i) {
      if (st->changed[i] || st->nz[i] > 1) continue;
      int s = (int)G.sim_of[i];
      const sim_grid *g = &G.g[s];
      int clean = 1;
      for (int dz = -1; dz <= 1 && clean; ++dz)
        for (int dy = -1; dy <= 1 && clean; ++dy)
          for (int dx = -1; dx <= 1 && clean; ++dx) {
            int64_t key = G.base[s] + box_linear(g, G.bx[i] + dx, G.by[i] + dy, G.bz[i] + dz);
            if (bsearch(&key, dirty, (size_t)ndirty, sizeof(int64_t), cmp_i64)) clean = 0;
          }
      stat[i] = (uint8_t)clean;
    }
  }

  /* 4. forces and displacement (Jacobi: every force reads P_t) */
  double *nx = (double *)malloc(sizeof(double) * (size_t)(3 * n + 1));
  int32_t *nnz = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n + 1));
  uint8_t *moved = (uint8_t *)calloc((size_t)(n + 1), 1);
  uint8_t *divide = (uint8_t *)calloc((size_t)(n + 1), 1);
  if (!nx || !nnz || !moved || !divide) {
    free(nx); free(nnz); free(moved); free(divide); free(stat); free(dirty); grid_free(&G);
    return ORC_ENOMEM;
  }
  double *ny = nx + n, *nzp = nx + 2 * n;
  int64_t n_static = 0, n_coincident = 0;
  /* each agent's sum is serial in the canonical order, so the timing build's
   * parallel loop (ORC_OPENMP) gives the same bits as the serial one */
#ifdef ORC_OPENMP
#pragma omp parallel for schedule(dynamic, 256) reduction(+ : n_static, n_coincident)
#endif
  for (int64_t i = 0; i < n; ++i) {
    double dxv = 0.0, dyv = 0.0, dzv = 0.0;
    double fxv = 0.0, fyv = 0.0, fzv = 0.0;
    if (stat[i]) {
      nnz[i] = st->nz[i];
      n_static++;
    } else {
      force_acc a;
      force_on(st, P, &G, i, &a, NULL, NULL);
      n_coincident += a.ncoincident;
      nnz[i] = a.nz;
      fxv = a.fx; fyv = a.fy; fzv = a.fz;
      double fn = sqrt((a.fx * a.fx + a.fy * a.fy) + a.fz * a.fz);
      if (fn > P->adherence) {
        double dt;
        agent_dt(st, P, G.sim_of[i], &dt);
        dxv = dt * a.fx; dyv = dt * a.fy; dzv = dt * a.fz;
        double dn = sqrt((dxv * dxv + dyv * dyv) + dzv * dzv);
        if (dn > P->dmax) {
          double c = P->dmax / dn;
          dxv = dxv * c; dyv = dyv * c; dzv = dzv * c;
        }
      }
    }
    if (!stat[i] && (st->beh[i] & BEH_WALK) && P->walk_step > 0.0) {
      double u[3];
      orc_unit_vector(P->seed, st->uid[i], (uint64_t)st->step, PURPOSE_WALK, u);
      dxv = dxv + P->walk_step * u[0];
      dyv = dyv + P->walk_step * u[1];
      dzv = dzv + P->walk_step * u[2];
    }
    nx[i] = st->x[i] + dxv;
    ny[i] = st->y[i] + dyv;
    nzp[i] = st->z[i] + dzv;
    moved[i] = (uint8_t)(nx[i] != st->x[i] || ny[i] != st->y[i] || nzp[i] != st->z[i]);
    if (st->fx) { st->fx[i] = fxv; st->fy[i] = fyv; st->fz[i] = fzv; }
    if (st->is_static) st->is_static[i] = stat[i];
  }
  st->n_static = n_static;
  st->n_coincident = n_coincident;
  free(stat);
  free(dirty);

  /* 5. behaviours: death (an agent removed at the end of this step neither
   *    grows nor divides), growth and the division decision (on the grown
   *    volume) */
  uint8_t *resized = (uint8_t *)calloc((size_t)(n + 1), 1);
  uint8_t *rm = (uint8_t *)calloc((size_t)(st->cap + 1), 1);
  if (!resized || !rm) { free(nx); free(nnz); free(moved); free(divide); free(resized); free(rm); grid_free(&G); return ORC_ENOMEM; }
  for (int64_t i = 0; i < n; ++i)
    if ((st->beh[i] & BEH_DIE) && P->death_prob > 0.0)
      rm[i] = (uint8_t)(orc_uniform(P->seed, st->uid[i], (uint64_t)st->step, PURPOSE_DEATH) < P->death_prob);
  int64_t ndiv = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (rm[i]) continue;
    if (!((st->beh[i] & BEH_GROW) && P->growth > 0.0)) continue;
    double v = st->vol[i] + P->growth;
    if (v >= P->divide_volume) { divide[i] = 1; ndiv++; }
    resized[i] = 1;
  }
  if (n + ndiv > st->cap) {
    free(nx); free(nnz); free(moved); free(divide); free(resized); free(rm); grid_free(&G);
    return ORC_ECAPACITY;
  }

  /* 6. commit: history of the previous positions, new positions, sizes;
   *    daughters are appended in parent storage order (Sec. 3.2) */
  int64_t rank = 0;
  for (int64_t i = 0; i < n; ++i) {
    st->px[i] = st->x[i]; st->py[i] = st->y[i]; st->pz[i] = st->z[i];
    st->x[i] = nx[i]; st->y[i] = ny[i]; st->z[i] = nzp[i];
    st->nz[i] = nnz[i];
    st->changed[i] = (uint8_t)(moved[i] || resized[i]);
    if (!resized[i]) continue;
    double v = st->vol[i] + P->growth;
    if (!divide[i]) {
      st->vol[i] = v;
      st->diam[i] = orc_cbrt((6.0 * v) / pi);
      continue;
    }
    double u0 = orc_uniform(P->seed, st->uid[i], (uint64_t)st->step, PURPOSE_RATIO);
    double rho = P->ratio_lo + (P->ratio_hi - P->ratio_lo) * u0;
    double v1 = (v * rho) / (1.0 + rho);
    double v2 = v / (1.0 + rho);
    double ax[3];
    orc_unit_vector(P->seed, st->uid[i], (uint64_t)st->step, PURPOSE_AXIS, ax);
    double rad = orc_cbrt((6.0 * v) / pi) * 0.5;
    double a1 = rad * (v2 / v), a2 = rad * (v1 / v);
    double cx = st->x[i], cy = st->y[i], cz = st->z[i];
    int64_t dgt = n + rank;
    st->x[i] = cx + a1 * ax[0]; st->y[i] = cy + a1 * ax[1]; st->z[i] = cz + a1 * ax[2];
    st->vol[i] = v1;
    st->diam[i] = orc_cbrt((6.0 * v1) / pi);
    st->changed[i] = 1;
    st->x[dgt] = cx - a2 * ax[0]; st->y[dgt] = cy - a2 * ax[1]; st->z[dgt] = cz - a2 * ax[2];
    st->px[dgt] = st->x[dgt]; st->py[dgt] = st->y[dgt]; st->pz[dgt] = st->z[dgt];
    st->vol[dgt] = v2;
    st->diam[dgt] = orc_cbrt((6.0 * v2) / pi);
    st->uid[dgt] = st->next_uid + (uint64_t)rank;
    st->beh[dgt] = st->beh[i];
    st->changed[dgt] = 1;
    st->nz[dgt] = 0;
    if (st->fx) { st->fx[dgt] = 0.0; st->fy[dgt] = 0.0; st->fz[dgt] = 0.0; }
    if (st->is_static) st->is_static[dgt] = 0;
    rank++;
  }
  st->n = n + ndiv;

  /* 7. removals, after the additions (Sec. 3.2): the removed agents' boxes of
   *    this step are remembered for the next step's static test, then the
   *    vector is compacted by swaps from its tail */
  st->n_ghost = 0;
  for (int64_t i = 0; i < n; ++i) {
    if (!rm[i]) continue;
    st->gx[st->n_ghost] = st->px[i]; st->gy[st->n_ghost] = st->py[i]; st->gz[st->n_ghost] = st->pz[i];
    st->n_ghost++;
  }
  int64_t moved_by_removal = orc_remove(st, rm);
  if (moved_by_removal < 0) {
    free(nx); free(nnz); free(moved); free(divide); free(resized); free(rm); grid_free(&G);
    return ORC_ENOMEM;
  }
  st->n_removed = st->n_ghost;

  st->sim_off[st->n_sims] = st->n; /* division and removal only in single-simulation runs */
  st->next_uid += (uint64_t)ndiv;
  st->n_divided = ndiv;
  st->step += 1;
  st->history_valid = 1;
  free(nx); free(nnz); free(moved); free(divide); free(resized); free(rm);
  grid_free(&G);
  return ORC_OK;
}
