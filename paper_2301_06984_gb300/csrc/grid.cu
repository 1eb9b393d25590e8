// grid.cu -- uniform-grid build of one iteration (Sec. 3.1 of the paper) as a
// counting sort of Morton keys (Sec. 4.2), plus the sort-step gather.
//
//   k_geometry    per simulation: lo = floor(min/L) L - L, n = floor((max-lo)/L)+2
//                 boxes per axis (one-box margin), 4x4x4 bricks, brick bases
//   k_brick_rank  Morton rank of every in-domain brick (the paper's gap/offset
//                 mapping rank = code - offset(code), evaluated per brick as a
//                 prefix count of in-domain cells, O(levels) per brick)
//   k_keys        box of every agent, key = brick rank * 64 + local Morton
//                 code, warp-aggregated atomics for per-brick arrival slots,
//                 dirty-box marking for the static contract (Sec. 5)
//   k_scan_*      exclusive scan of per-brick counts and occupancy
//   k_scatter     agents into their brick's bucket (arrival order)
//   k_brick_rank  rank of every brick among the in-domain bricks of its
//                 simulation along the Morton curve (Sec. 4.2's order) or,
//                 with curve = 1, along the Hilbert curve Sec. 4.2 compares
//   k_brick_sort  per occupied brick, on chip: order by (box, storage index),
//                 box ranges, and the compact per-agent records the force
//                 kernel streams (box-local FP32 coordinates and radius)
//   k_gather      sort step: storage <- grid order for every agent array
#include "bdm_internal.cuh"

#include <cooperative_groups.h>

namespace {

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// block-wide exclusive scan of one 32-bit value per thread; returns the
// exclusive prefix, writes the block total to *total.  blockDim.x <= 1024.
__device__ unsigned block_excl_scan(unsigned v, unsigned *smem32, unsigned *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  unsigned x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) smem32[warp] = x;
  __syncthreads();
  if (warp == 0) {
    unsigned w = (lane < nw) ? smem32[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      unsigned y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    smem32[lane] = w;  // inclusive warp totals
  }
  __syncthreads();
  unsigned base = (warp > 0) ? smem32[warp - 1] : 0u;
  *total = smem32[nw - 1];
  __syncthreads();
  return base + x - v;
}

__device__ long long block_excl_scan64(long long v, long long *smem64, long long *total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  long long x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) smem64[warp] = x;
  __syncthreads();
  if (warp == 0) {
    long long w = (lane < nw) ? smem64[lane] : 0ll;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      long long y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    smem64[lane] = w;
  }
  __syncthreads();
  long long base = (warp > 0) ? smem64[warp - 1] : 0ll;
  *total = smem64[nw - 1];
  __syncthreads();
  return base + x - v;
}

// Number of in-domain cells (x < n0, y < n1, z < n2) whose Morton code is
// smaller than that of (x, y, z): walk the code from its top bit; every 1 bit
// adds the in-domain cells of the lower half of the current node.
__device__ long long morton_rank3(int x, int y, int z, int n0, int n1, int n2, int levels) {
  long long rank = 0;
  int lo[3] = {0, 0, 0}, sz[3], n[3] = {n0, n1, n2}, v[3] = {x, y, z};
  sz[0] = sz[1] = sz[2] = 1 << levels;
  for (int k = levels - 1; k >= 0; --k) {
    const int half = 1 << k;
    for (int a = 2; a >= 0; --a) {
      if ((v[a] >> k) & 1) {
        long long c = 1;
        for (int b = 0; b < 3; ++b) {
          int l = lo[b];
          int h = (b == a) ? lo[b] + half : lo[b] + sz[b];
          if (h > n[b]) h = n[b];
          int w = h - l;
          if (w <= 0) { c = 0; break; }
          c *= w;
        }
        rank += c;
        lo[a] += half;
      }
      sz[a] = half;
    }
  }
  return rank;
}

// Number of in-domain cells (x < n0, y < n1, z < n2) that come before (x, y,
// z) on the 3D Hilbert curve of the 2^levels cube (the curve of Skilling's
// transpose method: at each level the sub-cubes are visited in the Gray-code
// order of their transformed bits, and the curve reflects or exchanges axes
// on the lower levels according to the sub-cube it is in).  Going down the
// levels, the state is the transform of the current node (which original axis
// each transformed axis reads, and whether it is reflected) and the parity of
// the final flip; at each level the in-domain cells of the sibling octants
// whose digit is smaller than the target's are added.
__device__ long long hilbert_rank3(int x, int y, int z, int n0, int n1, int n2, int levels) {
  const int v[3] = {x, y, z}, n[3] = {n0, n1, n2};
  int lo[3] = {0, 0, 0}, perm[3] = {0, 1, 2}, flip[3] = {0, 0, 0};
  int tpar = 0;
  long long rank = 0;
  for (int q = levels - 1; q >= 0; --q) {
    const int half = 1 << q;
    const int b[3] = {(v[0] >> q) & 1, (v[1] >> q) & 1, (v[2] >> q) & 1};
    // digit of a child with original bits c: transform, Gray-encode, flip
    auto digit = [&](const int c[3]) {
      const int X0 = c[perm[0]] ^ flip[0], X1 = c[perm[1]] ^ flip[1], X2 = c[perm[2]] ^ flip[2];
      const int g0 = X0, g1 = X0 ^ X1, g2 = g1 ^ X2;
      return ((g0 ^ tpar) << 2) | ((g1 ^ tpar) << 1) | (g2 ^ tpar);
    };
    const int dt = digit(b);
    for (int cc = 0; cc < 8; ++cc) {
      const int c[3] = {cc & 1, (cc >> 1) & 1, (cc >> 2) & 1};
      if (digit(c) >= dt) continue;
      long long cnt = 1;
      for (int d = 0; d < 3; ++d) {
        const int a0 = lo[d] + c[d] * half;
        const int a1 = min(a0 + half, n[d]);
        cnt *= (a1 > a0) ? (long long)(a1 - a0) : 0ll;
      }
      rank += cnt;
    }
    // the curve's transform for the lower levels (the target's sub-cube)
    const int X[3] = {b[perm[0]] ^ flip[0], b[perm[1]] ^ flip[1], b[perm[2]] ^ flip[2]};
    const int gpar = X[0] ^ X[1] ^ X[2];
    for (int i = 0; i < 3; ++i) {
      if (X[i]) {
        flip[0] ^= 1;
      } else {
        const int tp = perm[0], tf = flip[0];
        perm[0] = perm[i]; flip[0] = flip[i];
        perm[i] = tp; flip[i] = tf;
      }
    }
    tpar ^= gpar;
    for (int d = 0; d < 3; ++d) lo[d] += b[d] * half;
  }
  return rank;
}

__device__ __forceinline__ int sim_of_brick(const long long *base, int n_sims, long long g) {
  int lo = 0, hi = n_sims - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (base[mid] <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// --------------------------------------------------------------- geometry
__global__ void k_geometry(DevBufs B, DevParams P) {
  __shared__ long long s64[32];
  DevCounters *C = B.ctr;
  if (C->error) return;
  const int S = P.n_sims;
  const int par = (int)(C->step & 1);
  const long long n = C->n;
  long long carry = 0, boxes = 0;
  int bad = 0;
  for (int s0 = 0; s0 < S; s0 += blockDim.x) {
    const int s = s0 + threadIdx.x;
    long long nbk = 0;
    if (s < S) {
      const long long a0 = (S == 1) ? 0 : B.sim_off[s];
      const long long a1 = (S == 1) ? n : B.sim_off[s + 1];
      SimGeom *g = &B.geom[s];
      if (a1 > a0) {
        const unsigned long long *bb = B.bbox + ((size_t)par * S + s) * 6;
        int nb[3], nr[3];
        for (int d = 0; d < 3; ++d) {
          double mn = dec_f64(bb[d]), mx = dec_f64(bb[3 + d]);
          double lo = __dsub_rn(__dmul_rn(floor(__ddiv_rn(mn, P.L)), P.L), P.L);
          double cnt = floor(__ddiv_rn(__dsub_rn(mx, lo), P.L)) + 2.0;
          if (!(cnt >= 3.0 && cnt <= 2097152.0)) { bad = 1; cnt = 3.0; }
          nb[d] = (int)cnt;
          nr[d] = (nb[d] + 3) >> 2;
          g->lo[d] = lo;
          g->lo_f[d] = dtof_trunc(lo);
          g->lo_fix[d] = to_fixed(lo, P.fix_shift);
          g->nb[d] = nb[d];
          g->nr[d] = nr[d];
        }
        int mxr = max(nr[0], max(nr[1], nr[2])), lv = 0;
        while ((1 << lv) < mxr) ++lv;
        g->levels = lv;
        nbk = (long long)nr[0] * nr[1] * nr[2];
        boxes += (long long)nb[0] * nb[1] * nb[2];
      } else {
        for (int d = 0; d < 3; ++d) {
          g->lo[d] = 0.0; g->lo_f[d] = 0.f; g->lo_fix[d] = 0; g->nb[d] = 0; g->nr[d] = 0;
        }
        g->levels = 0;
      }
      g->n_bricks = nbk;
    }
    long long tot;
    long long ex = block_excl_scan64(nbk, s64, &tot);
    if (s < S) {
      B.geom[s].brick_base = carry + ex;
      B.brick_base[s] = carry + ex;
    }
    carry += tot;
  }
  // totals
  __shared__ int s_bad;
  __shared__ unsigned long long s_boxes;
  if (threadIdx.x == 0) { s_bad = 0; s_boxes = 0; }
  __syncthreads();
  if (bad) atomicOr(&s_bad, 1);
  atomicAdd(&s_boxes, (unsigned long long)boxes);
  __syncthreads();
  // reset the accumulator of the next positions' bounding box
  const int np = par ^ 1;
  for (int i = threadIdx.x; i < S * 6; i += blockDim.x) {
    B.bbox[(size_t)np * S * 6 + i] = ((i % 6) < 3) ? ~0ull : 0ull;
  }
  if (threadIdx.x == 0) {
    B.brick_base[S] = carry;
    C->total_bricks = carry;
    C->total_boxes = (long long)s_boxes;
    if (s_bad) {
      C->error = DEV_ERANGE;
    } else if (carry > B.brick_cap) {
      C->error = DEV_ECAP_BRICKS;
      C->need_bricks = carry;
    }
    C->a_static = C->a_moved = C->a_cand = C->a_nbr = C->a_contact = C->a_exact = 0;
    C->n_div = 0;
    C->max_brick = 0;
    C->n_occ = 0;
    C->heavy_n[0] = C->heavy_n[1] = 0;
    C->work_n = 0;
    C->sort_now = ((P.sort_every > 0 && (C->step % P.sort_every) == 0) || C->force_sort) ? 1 : 0;
    C->force_sort = 0;
  }
}

__global__ void k_brick_rank(DevBufs B, DevParams P) {
  const DevCounters *C = B.ctr;
  if (C->error) return;
  const long long total = C->total_bricks;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
       g += (long long)gridDim.x * blockDim.x) {
    const int s = (P.n_sims == 1) ? 0 : sim_of_brick(B.brick_base, P.n_sims, g);
    const SimGeom &G = B.geom[s];
    const long long base = G.brick_base;
    const long long local = g - base;
    const int ix = (int)(local % G.nr[0]);
    const long long t = local / G.nr[0];
    const int iy = (int)(t % G.nr[1]);
    const int iz = (int)(t / G.nr[1]);
    const long long r = (P.curve == 1) ? hilbert_rank3(ix, iy, iz, G.nr[0], G.nr[1], G.nr[2], G.levels)
                                       : morton_rank3(ix, iy, iz, G.nr[0], G.nr[1], G.nr[2], G.levels);
    B.brick_table[g] = (int32_t)(base + r);
    B.brick_count[g] = 0;
    B.dirty[g] = 0ull;
  }
}

// brick rank and local code of a (clamped or raw) box
__device__ __forceinline__ void box_key(const DevBufs &B, const SimGeom &G, int bx, int by, int bz, int &rank,
                                        int &lc) {
  const int Bx = bx >> 2, By = by >> 2, Bz = bz >> 2;
  long long lin = ((long long)Bz * G.nr[1] + By) * G.nr[0] + Bx;
  if (!BDM_IN(B.ctr, bx >= 0 && by >= 0 && bz >= 0 && Bx < G.nr[0] && By < G.nr[1] && Bz < G.nr[2] &&
                         G.brick_base + lin < B.brick_cap))
    lin = -G.brick_base;
  rank = B.brick_table[G.brick_base + lin];
  if (!BDM_IN(B.ctr, rank >= 0 && rank < B.brick_cap)) rank = 0;
  lc = local_code(bx & 3, by & 3, bz & 3);
}

// 8 blocks of 256 per SM (32 registers): the pass is bound by the latency of
// its loads and atomics, and the extra warps hide it (2.32 -> 1.64 ms at 150M
// core + shell agents, measured, despite a few spilled registers)
__global__ void __launch_bounds__(256, 8) k_keys(DevBufs B, DevParams P) {
  DevCounters *C = B.ctr;
  if (C->error) return;
  const AgentSet A = *B.A;
  const long long n = C->n;
  const int cur = (int)(C->step & 1);
  const bool use_static = P.detect_static && C->history_valid;
  const int lane = threadIdx.x & 31;
  unsigned long long ndiv = 0;
  for (long long base = blockIdx.x * (long long)blockDim.x; base < n; base += (long long)gridDim.x * blockDim.x) {
    const long long i = base + threadIdx.x;
    const bool active = i < n;
    const unsigned mask = __ballot_sync(0xffffffffu, active);
    if (!active) continue;
    const int s = (P.n_sims == 1) ? 0 : sim_of_agent(B.sim_off, P.n_sims, i);
    const SimGeom &G = B.geom[s];
    const double x = A.x[cur][i], y = A.y[cur][i], z = A.z[cur][i];
    bool fb;
    int bx = box_axis(x, G.lo[0], G.lo_f[0], P, fb);
    int by = box_axis(y, G.lo[1], G.lo_f[1], P, fb);
    int bz = box_axis(z, G.lo[2], G.lo_f[2], P, fb);
    bx = min(max(bx, 1), G.nb[0] - 2);
    by = min(max(by, 1), G.nb[1] - 2);
    bz = min(max(bz, 1), G.nb[2] - 2);
    int rank, lc;
    box_key(B, G, bx, by, bz, rank, lc);
    B.key[i] = (uint32_t)rank * 64u + (uint32_t)lc;
    // warp-aggregated arrival slot in the brick
    const unsigned m = __match_any_sync(mask, rank);
    const int leader = __ffs(m) - 1;
    unsigned slot = 0;
    if (lane == leader) slot = atomicAdd(&B.brick_count[rank], (unsigned)__popc(m));
    slot = __shfl_sync(m, slot, leader);
    B.arrival[i] = slot + (unsigned)__popc(m & lanemask_lt());
    if (use_static && (A.flags[i] & FL_CHANGED)) {
      atomicOr(&B.dirty[rank], 1ull << lc);
      const int o = cur ^ 1;
      int ox = box_axis(A.x[o][i], G.lo[0], G.lo_f[0], P, fb);
      int oy = box_axis(A.y[o][i], G.lo[1], G.lo_f[1], P, fb);
      int oz = box_axis(A.z[o][i], G.lo[2], G.lo_f[2], P, fb);
      if (ox >= 0 && ox < G.nb[0] && oy >= 0 && oy < G.nb[1] && oz >= 0 && oz < G.nb[2]) {
        int r2, l2;
        box_key(B, G, ox, oy, oz, r2, l2);
        atomicOr(&B.dirty[r2], 1ull << l2);
      }
    }
    if (P.grow && (A.beh[i] & BEH_GROW)) {
      // an agent removed in this iteration does not divide
      if (__dadd_rn(A.vol[i], P.growth) >= P.divide_volume &&
          !(P.die && (A.beh[i] & BEH_DIE) && agent_dies(P, A.uid[i], C->step)))
        ndiv++;
    }
  }
  if (use_static) {
    // the boxes the agents removed in the previous iteration left (their
    // position at its start) are dirty: their neighbours lost a neighbour
    const long long ng = C->n_ghost;
    const SimGeom &G = B.geom[0];
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < ng;
         g += (long long)gridDim.x * blockDim.x) {
      const dbl4 q = B.ghost[g];
      bool fb;
      const int ox = box_axis(q.x, G.lo[0], G.lo_f[0], P, fb);
      const int oy = box_axis(q.y, G.lo[1], G.lo_f[1], P, fb);
      const int oz = box_axis(q.z, G.lo[2], G.lo_f[2], P, fb);
      if (ox >= 0 && ox < G.nb[0] && oy >= 0 && oy < G.nb[1] && oz >= 0 && oz < G.nb[2]) {
        int r2, l2;
        box_key(B, G, ox, oy, oz, r2, l2);
        atomicOr(&B.dirty[r2], 1ull << l2);
      }
    }
  }
  if (P.grow) {
    for (int o = 16; o > 0; o >>= 1) ndiv += __shfl_down_sync(0xffffffffu, ndiv, o);
    if (lane == 0 && ndiv) atomicAdd((unsigned long long *)&C->n_div, ndiv);
  }
}

// --------------------------------------------------------------- brick scan
__global__ void k_scan_reduce(DevBufs B) {
  __shared__ unsigned s32[32];
  const DevCounters *C = B.ctr;
  if (C->error) return;
  const long long total = C->total_bricks;
  const long long t0 = (long long)blockIdx.x * SCAN_TILE;
  if (t0 >= total) return;
  unsigned sum = 0, occ = 0, mx = 0;
  for (int e = 0; e < SCAN_TILE / SCAN_THREADS; ++e) {
    const long long g = t0 + threadIdx.x * (SCAN_TILE / SCAN_THREADS) + e;
    if (g < total) {
      unsigned c = B.brick_count[g];
      sum += c;
      occ += (c > 0);
      mx = max(mx, c);
    }
  }
  unsigned tot;
  block_excl_scan(sum, s32, &tot);
  unsigned tot_occ;
  block_excl_scan(occ, s32, &tot_occ);
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_down_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) atomicMax((unsigned long long *)&B.ctr->max_brick, (unsigned long long)mx);
  if (threadIdx.x == 0) {
    B.scan_a[blockIdx.x] = tot;
    B.scan_b[blockIdx.x] = tot_occ;
  }
}

__global__ void k_scan_top(DevBufs B, DevParams P) {
  __shared__ unsigned s32[32];
  DevCounters *C = B.ctr;
  if (C->error) return;
  const long long total = C->total_bricks;
  const long long nblk = (total + SCAN_TILE - 1) / SCAN_TILE;
  unsigned carry_a = 0, carry_b = 0;
  for (long long b0 = 0; b0 < nblk; b0 += blockDim.x) {
    const long long b = b0 + threadIdx.x;
    unsigned va = (b < nblk) ? B.scan_a[b] : 0u, vb = (b < nblk) ? B.scan_b[b] : 0u;
    unsigned ta, tb;
    unsigned ea = block_excl_scan(va, s32, &ta);
    unsigned eb = block_excl_scan(vb, s32, &tb);
    if (b < nblk) {
      B.scan_a[b] = carry_a + ea;
      B.scan_b[b] = carry_b + eb;
    }
    carry_a += ta;
    carry_b += tb;
  }
  if (threadIdx.x == 0) {
    C->n_occ = carry_b;
    if ((long long)carry_b > B.occ_cap) {
      C->error = DEV_ECAP_OCC;
      C->need_occ = carry_b;
    } else if (P.grow && C->n + C->n_div > B.cap) {
      C->error = DEV_ECAP_AGENTS;
    }
  }
}

__global__ void k_scan_down(DevBufs B) {
  __shared__ unsigned s32[32];
  const DevCounters *C = B.ctr;
  if (C->error) return;
  const long long total = C->total_bricks;
  const long long t0 = (long long)blockIdx.x * SCAN_TILE;
  if (t0 >= total) return;
  constexpr int E = SCAN_TILE / SCAN_THREADS;
  unsigned c[E];
  unsigned sum = 0, occ = 0;
  for (int e = 0; e < E; ++e) {
    const long long g = t0 + threadIdx.x * E + e;
    c[e] = (g < total) ? B.brick_count[g] : 0u;
    sum += c[e];
    occ += (c[e] > 0);
  }
  unsigned tt;
  unsigned ps = block_excl_scan(sum, s32, &tt) + B.scan_a[blockIdx.x];
  unsigned po = block_excl_scan(occ, s32, &tt) + B.scan_b[blockIdx.x];
  for (int e = 0; e < E; ++e) {
    const long long g = t0 + threadIdx.x * E + e;
    if (g < total) {
      B.brick_start[g] = ps;
      if (c[e] > 0) {
        B.brick_occ[g] = (int32_t)po;
        B.occ_list[po] = (int32_t)g;
        ++po;
      } else {
        B.brick_occ[g] = -1;
      }
      ps += c[e];
    }
  }
}

__global__ void k_scatter(DevBufs B) {
  const DevCounters *C = B.ctr;
  if (C->error) return;
  const long long n = C->n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const uint32_t r = B.key[i] >> 6;
    if (!BDM_IN(B.ctr, r < (uint32_t)B.brick_cap)) continue;
    const unsigned long long dst = (unsigned long long)B.brick_start[r] + B.arrival[i];
    if (!BDM_IN(B.ctr, dst < (unsigned long long)n)) continue;
    B.bucket[dst] = (uint32_t)i;
  }
}

// --------------------------------------------------------------- brick sort
#define BS_THREADS 256

// Bricks of at most BSW_MAX agents (most bricks of sparse workloads, and the
// bricks of a tissue at one to four agents per box) are sorted by
// k_brick_sort_small, one warp per brick, with the same result; k_brick_sort
// takes the rest, one block per brick.
#define BSW_MAX 320
static_assert(BSW_MAX < FORCE_HEAVY_HI, "the warp-per-brick sort lists no brick at the heavy list front");
#define BSW_WARPS 8
#define BS_SMEM_M 4096

// box-local compact record of agent i in its box (bx, by, bz)
__device__ __forceinline__ void write_compact(const DevBufs &B, const DevParams &P, const AgentSet &A, int cur,
                                              const SimGeom &G, long long i, long long k, int bx, int by, int bz,
                                              double x, double y, double z) {
  const long long ox = G.lo_fix[0] + (long long)bx * P.L_fix;
  const long long oy = G.lo_fix[1] + (long long)by * P.L_fix;
  const long long oz = G.lo_fix[2] + (long long)bz * P.L_fix;
  const float sc = __int_as_float((127 - P.fix_shift) << 23);
  const float xl = (float)(int)(to_fixed(x, P.fix_shift) - ox) * sc;
  const float yl = (float)(int)(to_fixed(y, P.fix_shift) - oy) * sc;
  const float zl = (float)(int)(to_fixed(z, P.fix_shift) - oz) * sc;
  float r;
  double rd;
  if (P.precision == 0) {
    rd = __dmul_rn(((const double *)A.diam)[i], 0.5);
    r = dtof_trunc(rd);
    B.c64[k] = mk_dbl4(x, y, z, rd);
  } else {
    r = ((const float *)A.diam)[i] * 0.5f;
  }
  B.c32[k] = make_float4(xl, yl, zl, r);
  if (P.n_types > 1) B.tp[k] = (uint8_t)((A.beh[i] >> BEH_TYPE_SHIFT) & 3u);
}

// The brick of agent idx (the same for every agent with the same brick
// rank): its coordinates and simulation, from the agent's clamped box exactly
// as k_keys formed the agent's key.
__device__ __forceinline__ int4 brick_of_agent(const DevBufs &B, const DevParams &P, const AgentSet &A, int cur,
                                               uint32_t idx) {
  const int s = (P.n_sims == 1) ? 0 : sim_of_agent(B.sim_off, P.n_sims, idx);
  const SimGeom &G = B.geom[s];
  bool fb;
  const int bx = min(max(box_axis(A.x[cur][idx], G.lo[0], G.lo_f[0], P, fb), 1), G.nb[0] - 2);
  const int by = min(max(box_axis(A.y[cur][idx], G.lo[1], G.lo_f[1], P, fb), 1), G.nb[1] - 2);
  const int bz = min(max(box_axis(A.z[cur][idx], G.lo[2], G.lo_f[2], P, fb), 1), G.nb[2] - 2);
  return make_int4(bx >> 2, by >> 2, bz >> 2, s);
}

// Agent idx at sorted position kk of occupied brick o (br: the brick, from
// brick_of_agent; lc: the agent's local box code): its storage index, its
// box-local compact record and, for the brick's first agent, the brick's
// coordinates and simulation.  The agent's box is the brick's corner box plus
// its local box, so no box is computed per agent.
__device__ __forceinline__ void place_agent(const DevBufs &B, const DevParams &P, const AgentSet &A, int cur,
                                            long long o, uint32_t idx, unsigned lc, int4 br, long long kk, bool first) {
  if (!BDM_IN(B.ctr, kk >= 0 && kk < B.ctr->n && idx < (uint32_t)B.cap && o < B.occ_cap && br.w >= 0 &&
                         br.w < P.n_sims)) return;
  B.perm[kk] = idx;
  const SimGeom &G = B.geom[br.w];
  int lx, ly, lz;
  local_decode((int)lc, lx, ly, lz);
  const double x = A.x[cur][idx], y = A.y[cur][idx], z = A.z[cur][idx];
  write_compact(B, P, A, cur, G, idx, kk, 4 * br.x + lx, 4 * br.y + ly, 4 * br.z + lz, x, y, z);
  if (first) B.occ_info[o] = br;
}

__global__ void __launch_bounds__(BS_THREADS) k_brick_sort(DevBufs B, DevParams P) {
  __shared__ uint32_t s_idx[BS_SMEM_M];
  __shared__ uint32_t s_grp[BS_SMEM_M];
  __shared__ uint8_t s_l[BS_SMEM_M];
  __shared__ uint8_t s_gl[BS_SMEM_M];
  __shared__ unsigned s_cnt[64], s_off[64], s_cur[64];
  __shared__ int s_abort;
  __shared__ int4 s_br;
  __shared__ long long s_list[BS_THREADS];
  __shared__ int s_nlist;
  DevCounters *C = B.ctr;
  if (C->error) return;
  const AgentSet A = *B.A;
  const int cur = (int)(C->step & 1);
  const long long n_occ = C->n_occ;
  // The block's bricks are o = blockIdx.x + i gridDim.x.  Its threads test
  // BS_THREADS of them at a time and list those above BSW_MAX agents (the
  // others are k_brick_sort_small's), so that the block does not walk the
  // many light bricks one dependent load pair at a time.  The bricks are
  // independent: the order in which a block sorts them changes no result.
  for (long long r0 = 0; (long long)blockIdx.x + (long long)gridDim.x * r0 < n_occ; r0 += BS_THREADS) {
    __syncthreads();
    if (threadIdx.x == 0) s_nlist = 0;
    __syncthreads();
    {
      const long long ot = (long long)blockIdx.x + (long long)gridDim.x * (r0 + threadIdx.x);
      if (ot < n_occ && B.brick_count[B.occ_list[ot]] > BSW_MAX) s_list[atomicAdd(&s_nlist, 1)] = ot;
    }
    __syncthreads();
    const int nl = s_nlist;
    for (int li = 0; li < nl; ++li) {
      const long long o = s_list[li];
      const int g = B.occ_list[o];
      const unsigned S0 = B.brick_start[g];
      const unsigned m = B.brick_count[g];
      const bool onchip = m <= BS_SMEM_M;
      if (threadIdx.x == 0 && m >= FORCE_HEAVY_LO) {
        // heavy bricks, listed for the force kernels' largest-first order
        if (m >= FORCE_HEAVY_HI) B.heavy[atomicAdd(&C->heavy_n[0], 1ull)] = (int32_t)o;
        else B.heavy[B.occ_cap - 1 - (long long)atomicAdd(&C->heavy_n[1], 1ull)] = (int32_t)o;
      }
      __syncthreads();
      if (threadIdx.x < 64) s_cnt[threadIdx.x] = 0;
      if (threadIdx.x == 0) {
        s_abort = 0;
        s_br = brick_of_agent(B, P, A, cur, B.bucket[S0]);
      }
      __syncthreads();
#pragma unroll 4
      for (unsigned k = threadIdx.x; k < m; k += blockDim.x) {
        if (!BDM_IN(B.ctr, (long long)S0 + k < B.ctr->n)) break;
        const uint32_t idx = B.bucket[S0 + k];
        if (!BDM_IN(B.ctr, idx < (uint32_t)B.cap)) continue;
        const unsigned l = B.key[idx] & 63u;
        if (onchip) { s_idx[k] = idx; s_l[k] = (uint8_t)l; }
        atomicAdd(&s_cnt[l], 1u);
      }
      __syncthreads();
      if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        unsigned a = s_cnt[lane], b = s_cnt[lane + 32];
        unsigned xa = a, xb = b;
        for (int d = 1; d < 32; d <<= 1) {
          unsigned ya = __shfl_up_sync(0xffffffffu, xa, d), yb = __shfl_up_sync(0xffffffffu, xb, d);
          if (lane >= d) { xa += ya; xb += yb; }
        }
        unsigned ta = __shfl_sync(0xffffffffu, xa, 31);
        s_off[lane] = xa - a;
        s_off[lane + 32] = ta + xb - b;
        s_cur[lane] = xa - a;
        s_cur[lane + 32] = ta + xb - b;
        unsigned mx = max(a, b);
        for (int d = 16; d > 0; d >>= 1) mx = max(mx, __shfl_down_sync(0xffffffffu, mx, d));
        if (lane == 0 && mx > BDM_MAX_BOX_AGENTS) {
          atomicCAS(&C->error, 0, (int)DEV_EBOX);
          s_abort = 1;
        }
      }
      __syncthreads();
      if (s_abort) return;  // block-uniform
      // group by box (arrival order inside a group)
      for (unsigned k = threadIdx.x; k < m; k += blockDim.x) {
        uint32_t idx;
        unsigned l;
        if (onchip) { idx = s_idx[k]; l = s_l[k]; }
        else { idx = B.bucket[S0 + k]; l = B.key[idx] & 63u; }
        const unsigned pos = atomicAdd(&s_cur[l], 1u);
        if (!BDM_IN(B.ctr, pos < m && (!onchip || pos < BS_SMEM_M))) continue;
        if (onchip) { s_grp[pos] = idx; s_gl[pos] = (uint8_t)l; }
        else B.arrival[S0 + pos] = idx;
      }
      __syncthreads();
      // stable rank inside the box = members with a smaller storage index
#pragma unroll 2
      for (unsigned k = threadIdx.x; k < m; k += blockDim.x) {
        uint32_t idx;
        unsigned l;
        if (onchip) { idx = s_grp[k]; l = s_gl[k]; }
        else { idx = B.arrival[S0 + k]; l = B.key[idx] & 63u; }
        const unsigned lo = s_off[l], cnt = s_cnt[l];
        unsigned r = 0;
        if (onchip) {
          for (unsigned q = 0; q < cnt; ++q) r += (s_grp[lo + q] < idx);
        } else {
          for (unsigned q = 0; q < cnt; ++q) r += (B.arrival[S0 + lo + q] < idx);
        }
        place_agent(B, P, A, cur, o, idx, l, s_br, (long long)S0 + lo + r, lo + r == 0);
      }
      if (threadIdx.x < 64) {
        B.box_start[o * 64 + threadIdx.x] = S0 + s_off[threadIdx.x];
        B.box_cnt[o * 64 + threadIdx.x] = s_cnt[threadIdx.x];
      }
    }
  }
}

// One warp per brick of at most BSW_MAX agents: per-box counts (shared
// atomics), exclusive scan of the 64 counts, grouping by box, then the stable
// rank inside each box by storage index, exactly as k_brick_sort.
__global__ void __launch_bounds__(BSW_WARPS * 32) k_brick_sort_small(DevBufs B, DevParams P) {
  __shared__ uint32_t s_idx[BSW_WARPS][BSW_MAX], s_grp[BSW_WARPS][BSW_MAX];
  __shared__ uint8_t s_l[BSW_WARPS][BSW_MAX], s_gl[BSW_WARPS][BSW_MAX];
  __shared__ unsigned s_cnt[BSW_WARPS][64], s_off[BSW_WARPS][64], s_cur[BSW_WARPS][64];
  DevCounters *C = B.ctr;
  if (C->error) return;
  const AgentSet A = *B.A;
  const int cur = (int)(C->step & 1);
  const long long n_occ = C->n_occ;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long nw = (long long)gridDim.x * BSW_WARPS;
  for (long long o = (long long)blockIdx.x * BSW_WARPS + w; o < n_occ; o += nw) {
    const int g = B.occ_list[o];
    const unsigned S0 = B.brick_start[g], m = B.brick_count[g];
    if (m > BSW_MAX) continue;  // warp-uniform: k_brick_sort's brick
    if (lane == 0 && m >= FORCE_HEAVY_LO) {
      // heavy bricks (below FORCE_HEAVY_HI here), listed for the force
      // kernels' largest-first order
      B.heavy[B.occ_cap - 1 - (long long)atomicAdd(&C->heavy_n[1], 1ull)] = (int32_t)o;
    }
    s_cnt[w][lane] = 0u;
    s_cnt[w][lane + 32] = 0u;
    int4 br = make_int4(0, 0, 0, 0);
    if (lane == 0) br = brick_of_agent(B, P, A, cur, B.bucket[S0]);
    br.x = __shfl_sync(0xffffffffu, br.x, 0);
    br.y = __shfl_sync(0xffffffffu, br.y, 0);
    br.z = __shfl_sync(0xffffffffu, br.z, 0);
    br.w = __shfl_sync(0xffffffffu, br.w, 0);
    __syncwarp();
    // unrolled: several agents' loads in flight per lane
#pragma unroll 4
    for (unsigned k = lane; k < m; k += 32) {
      const uint32_t idx = B.bucket[S0 + k];
      if (!BDM_IN(B.ctr, k < BSW_MAX && idx < (uint32_t)B.cap)) continue;
      const unsigned l = B.key[idx] & 63u;
      s_idx[w][k] = idx;
      s_l[w][k] = (uint8_t)l;
      atomicAdd(&s_cnt[w][l], 1u);
    }
    __syncwarp();
    {
      const unsigned a = s_cnt[w][lane], b = s_cnt[w][lane + 32];
      unsigned xa = a, xb = b;
      for (int d = 1; d < 32; d <<= 1) {
        const unsigned ya = __shfl_up_sync(0xffffffffu, xa, d), yb = __shfl_up_sync(0xffffffffu, xb, d);
        if (lane >= d) { xa += ya; xb += yb; }
      }
      const unsigned ta = __shfl_sync(0xffffffffu, xa, 31);
      s_off[w][lane] = s_cur[w][lane] = xa - a;
      s_off[w][lane + 32] = s_cur[w][lane + 32] = ta + xb - b;
    }
    __syncwarp();
    // group by box (arrival order inside a group)
    for (unsigned k = lane; k < m; k += 32) {
      const unsigned l = s_l[w][k];
      const unsigned pos = atomicAdd(&s_cur[w][l], 1u);
      if (!BDM_IN(B.ctr, pos < m && pos < BSW_MAX)) continue;
      s_grp[w][pos] = s_idx[w][k];
      s_gl[w][pos] = (uint8_t)l;
    }
    __syncwarp();
    // stable rank inside the box = members with a smaller storage index
#pragma unroll 2
    for (unsigned k = lane; k < m; k += 32) {
      const uint32_t idx = s_grp[w][k];
      const unsigned l = s_gl[w][k];
      const unsigned lo = s_off[w][l], cnt = s_cnt[w][l];
      unsigned r = 0;
      for (unsigned q = 0; q < cnt; ++q) r += (s_grp[w][lo + q] < idx);
      place_agent(B, P, A, cur, o, idx, l, br, (long long)S0 + lo + r, lo + r == 0);
    }
    B.box_start[o * 64 + lane] = S0 + s_off[w][lane];
    B.box_start[o * 64 + lane + 32] = S0 + s_off[w][lane + 32];
    B.box_cnt[o * 64 + lane] = s_cnt[w][lane];
    B.box_cnt[o * 64 + lane + 32] = s_cnt[w][lane + 32];
    __syncwarp();
  }
}

// --------------------------------------------------------------- sort step
__global__ void k_gather(DevBufs B, DevParams P) {
  const DevCounters *C = B.ctr;
  if (C->error || !C->sort_now) return;
  const AgentSet A = *B.A, D = *B.A_alt;
  const long long n = C->n;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    const uint32_t i = B.perm[k];
    if (!BDM_IN(B.ctr, (long long)i < n)) continue;
    for (int b = 0; b < 2; ++b) {
      D.x[b][k] = A.x[b][i];
      D.y[b][k] = A.y[b][i];
      D.z[b][k] = A.z[b][i];
    }
    if (P.precision == 0) ((double *)D.diam)[k] = ((const double *)A.diam)[i];
    else ((float *)D.diam)[k] = ((const float *)A.diam)[i];
    if (A.vol) D.vol[k] = A.vol[i];
    D.uid[k] = A.uid[i];
    D.beh[k] = A.beh[i];
    D.flags[k] = A.flags[i];
    D.nz[k] = A.nz[i];
    B.perm[k] = (uint32_t)k;
  }
}

__global__ void k_swap(DevBufs B) {
  const DevCounters *C = B.ctr;
  if (C->error || !C->sort_now) return;
  const AgentSet t = *B.A;
  *B.A = *B.A_alt;
  *B.A_alt = t;
}

// --------------------------------------------------------------- bbox / init
__global__ void k_bbox_reset(DevBufs B, DevParams P) {
  const int par = (int)(B.ctr->step & 1);
  for (int i = threadIdx.x; i < P.n_sims * 6; i += blockDim.x)
    B.bbox[(size_t)par * P.n_sims * 6 + i] = ((i % 6) < 3) ? ~0ull : 0ull;
}

__global__ void k_bbox(DevBufs B, DevParams P) {
  // per-thread min/max of the encoded coordinates, flushed when the
  // simulation changes; a single simulation reduces over the warp and the
  // block first, so each block issues six atomics
  __shared__ unsigned long long s_v[32][6];
  const DevCounters *C = B.ctr;
  const AgentSet A = *B.A;
  const long long n = C->n;
  const int par = (int)(C->step & 1);
  int cs = -1;
  unsigned long long v[6] = {~0ull, ~0ull, ~0ull, 0ull, 0ull, 0ull};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int s = (P.n_sims == 1) ? 0 : sim_of_agent(B.sim_off, P.n_sims, i);
    if (s != cs) {
      if (cs >= 0) {
        unsigned long long *bb = B.bbox + ((size_t)par * P.n_sims + cs) * 6;
        for (int d = 0; d < 3; ++d) { atomicMin(&bb[d], v[d]); atomicMax(&bb[3 + d], v[3 + d]); }
      }
      cs = s;
      v[0] = v[1] = v[2] = ~0ull;
      v[3] = v[4] = v[5] = 0ull;
    }
    const unsigned long long e[3] = {enc_f64(A.x[par][i]), enc_f64(A.y[par][i]), enc_f64(A.z[par][i])};
    for (int d = 0; d < 3; ++d) {
      v[d] = min(v[d], e[d]);
      v[3 + d] = max(v[3 + d], e[d]);
    }
  }
  if (P.n_sims > 1) {
    if (cs >= 0) {
      unsigned long long *bb = B.bbox + ((size_t)par * P.n_sims + cs) * 6;
      for (int d = 0; d < 3; ++d) { atomicMin(&bb[d], v[d]); atomicMax(&bb[3 + d], v[3 + d]); }
    }
    return;
  }
  for (int o = 16; o > 0; o >>= 1)
    for (int d = 0; d < 3; ++d) {
      v[d] = min(v[d], __shfl_xor_sync(0xffffffffu, v[d], o));
      v[3 + d] = max(v[3 + d], __shfl_xor_sync(0xffffffffu, v[3 + d], o));
    }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0)
    for (int d = 0; d < 6; ++d) s_v[warp][d] = v[d];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < nw; ++w)
      for (int d = 0; d < 3; ++d) {
        v[d] = min(v[d], s_v[w][d]);
        v[3 + d] = max(v[3 + d], s_v[w][3 + d]);
      }
    if (v[0] != ~0ull) {
      unsigned long long *bb = B.bbox + (size_t)par * 6;
      for (int d = 0; d < 3; ++d) { atomicMin(&bb[d], v[d]); atomicMax(&bb[3 + d], v[3 + d]); }
    }
  }
}

__global__ void k_debug_boxes(DevBufs B, DevParams P, int32_t *out_box, long long *out_rank) {
  const DevCounters *C = B.ctr;
  const AgentSet A = *B.A;
  const long long n = C->n;
  const int cur = (int)(C->step & 1);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int s = (P.n_sims == 1) ? 0 : sim_of_agent(B.sim_off, P.n_sims, i);
    const SimGeom &G = B.geom[s];
    bool fb;
    int bx = min(max(box_axis(A.x[cur][i], G.lo[0], G.lo_f[0], P, fb), 1), G.nb[0] - 2);
    int by = min(max(box_axis(A.y[cur][i], G.lo[1], G.lo_f[1], P, fb), 1), G.nb[1] - 2);
    int bz = min(max(box_axis(A.z[cur][i], G.lo[2], G.lo_f[2], P, fb), 1), G.nb[2] - 2);
    out_box[i] = bx;
    out_box[n + i] = by;
    out_box[2 * n + i] = bz;
    out_rank[i] = (long long)(B.key[i] >> 6) - G.brick_base;
  }
}

__global__ void k_diam_to_f64(DevBufs B, DevParams P, double *out) {
  const DevCounters *C = B.ctr;
  const AgentSet A = *B.A;
  const long long n = C->n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = (P.precision == 0) ? ((const double *)A.diam)[i] : (double)((const float *)A.diam)[i];
}

// The other agent arrays from the caller's diameters (checked: finite,
// positive, below 1e6 um; *bad is set when one is not) and optional arrays.
__global__ void k_init_agents(DevBufs B, DevParams P, const double *diam_in, const double *vol_in,
                              const uint64_t *uid_in, const uint8_t *beh_in, long long n, int *bad) {
  const AgentSet A = *B.A;
  const double pi = 3.141592653589793;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double d = diam_in[i];
    if (!(isfinite(d) && d > 0.0 && d < 1e6)) atomicOr(bad, 1);
    if (P.precision == 0) ((double *)A.diam)[i] = d;
    else ((float *)A.diam)[i] = __double2float_rn(d);
    if (A.vol) A.vol[i] = vol_in ? vol_in[i] : __dmul_rn(__dmul_rn(__dmul_rn(pi / 6.0, d), d), d);
    A.uid[i] = uid_in ? uid_in[i] : (uint64_t)i;
    A.beh[i] = beh_in ? beh_in[i] : (uint8_t)((P.grow ? BEH_GROW : 0) | (P.walk ? BEH_WALK : 0));
    A.flags[i] = 0;
    A.nz[i] = 0;
  }
}

// The caller's positions into both position buffers (the second one: no
// movement history yet), checked on the way (finite, within +-1e9 um); *bad
// is set when one is not.  (sx, sy, sz) may be set 0's own first buffers, which
// are then not written again.
__global__ void k_positions_in(const double *sx, const double *sy, const double *sz, AgentSet A, long long n,
                               int *bad) {
  const bool copy0 = sx != A.x[0];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double a = sx[i], b = sy[i], c = sz[i];
    if (copy0) { A.x[0][i] = a; A.y[0][i] = b; A.z[0][i] = c; }
    A.x[1][i] = a;
    A.y[1][i] = b;
    A.z[1][i] = c;
    const bool ok = isfinite(a) && isfinite(b) && isfinite(c) && fabs(a) < 1e9 && fabs(b) < 1e9 && fabs(c) < 1e9;
    if (!ok) atomicOr(bad, 1);
  }
}

}  // namespace

// --------------------------------------------------------------- launchers
void launch_geometry(const DevBufs &B, const DevParams &P, cudaStream_t s) {
  k_geometry<<<1, 1024, 0, s>>>(B, P);
}
void launch_brick_rank(const DevBufs &B, const DevParams &P, const LaunchCfg &c, cudaStream_t s) {
  k_brick_rank<<<c.brick_blocks, 256, 0, s>>>(B, P);
}
void launch_keys(const DevBufs &B, const DevParams &P, const LaunchCfg &c, cudaStream_t s) {
  k_keys<<<c.agent_blocks, 256, 0, s>>>(B, P);
}
void launch_brick_scan(const DevBufs &B, const DevParams &P, const LaunchCfg &c, cudaStream_t s) {
  k_scan_reduce<<<c.scan_blocks, SCAN_THREADS, 0, s>>>(B);
  k_scan_top<<<1, 1024, 0, s>>>(B, P);
  k_scan_down<<<c.scan_blocks, SCAN_THREADS, 0, s>>>(B);
}
void launch_scatter(const DevBufs &B, const DevParams &P, const LaunchCfg &c, cudaStream_t s) {
  (void)P;
  k_scatter<<<c.agent_blocks, 256, 0, s>>>(B);
}
void launch_brick_sort(const DevBufs &B, const DevParams &P, const LaunchCfg &c, cudaStream_t s) {
  k_brick_sort_small<<<c.occ_blocks, BSW_WARPS * 32, 0, s>>>(B, P);
  // the block-per-brick sort with twice the blocks of the other grid kernels:
  // each block sorts one brick at a time, so more bricks are in flight per SM
  k_brick_sort<<<2 * c.occ_blocks, BS_THREADS, 0, s>>>(B, P);
}
void launch_gather(const DevBufs &B, const DevParams &P, const LaunchCfg &c, cudaStream_t s) {
  k_gather<<<c.agent_blocks, 256, 0, s>>>(B, P);
  k_swap<<<1, 1, 0, s>>>(B);
}
void launch_bbox(const DevBufs &B, const DevParams &P, const LaunchCfg &c, cudaStream_t s) {
  k_bbox_reset<<<1, 256, 0, s>>>(B, P);
  k_bbox<<<c.agent_blocks, 256, 0, s>>>(B, P);
}
void launch_debug_boxes(const DevBufs &B, const DevParams &P, const LaunchCfg &c, int32_t *out_box,
                        long long *out_rank, cudaStream_t s) {
  k_debug_boxes<<<c.agent_blocks, 256, 0, s>>>(B, P, out_box, out_rank);
}
void launch_diam_to_f64(const DevBufs &B, const DevParams &P, const LaunchCfg &c, double *out, cudaStream_t s) {
  k_diam_to_f64<<<c.agent_blocks, 256, 0, s>>>(B, P, out);
}
void launch_init_agents(const DevBufs &B, const DevParams &P, const LaunchCfg &c, const double *diam_in,
                        const double *vol_in, const uint64_t *uid_in, const uint8_t *beh_in, long long n, int *bad,
                        cudaStream_t s) {
  k_init_agents<<<c.agent_blocks, 256, 0, s>>>(B, P, diam_in, vol_in, uid_in, beh_in, n, bad);
}
void launch_positions_in(const double *x, const double *y, const double *z, const AgentSet &A, long long n, int *bad,
                         const LaunchCfg &c, cudaStream_t s) {
  k_positions_in<<<c.agent_blocks, 256, 0, s>>>(x, y, z, A, n, bad);
}
