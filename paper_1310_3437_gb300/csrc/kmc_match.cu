// kmc_match.cu -- exact candidate test, mutual-choice matching and the collision
// update (Sec. 2: "a closer partner replaces the one found so far"; "two particles
// only collide if they have both found each other"; positions and velocities of
// the colliding pair are then updated).
//
// All binary64 arithmetic goes through the __d*_rn intrinsics (never contracted),
// in the operation order of the definitions below, so every value is bit-identical
// to the binary64 definition evaluated on any IEEE-754 machine.
//
//   k_refine  exact test of every pair emitted by the search:
//             r = x_j - x_i (minimum image on periodic axes), v = v_j - v_i,
//             t* = -(r.v)/|v|^2, d_min^2 = |r x v|^2/|v|^2; candidate iff |v| != 0,
//             0 <= t* < dt, d_min^2 < d0^2, and the pair is not the pair that last
//             collided for both of its members.  Survivors take a slot in each
//             endpoint's candidate list.
//   k_alloc   each particle with candidates gets a contiguous list (one warp-
//             aggregated atomic per warp) and a place on the first round's work list;
//             only the particles with candidates are touched, no pass over all n.
//   k_fill    the lists: (other end, pair) per slot.
//   k_best    per round, over the round's work list: every unmatched particle picks
//             its unmatched candidate of least key (d_min^2, t*, partner id) -- a
//             total order, so the choice does not depend on the order of the list.
//   k_mutual  per round, over the same list: pairs that picked each other are
//             matched (warp-aggregated appends); a particle left unmatched that still
//             had an unmatched candidate goes on the next round's list, so later
//             rounds only visit the few particles they can still match.
//   k_collide isotropic centre-of-mass scatter at the time of closest approach.
#include <algorithm>

#include "kmc_internal.cuh"
#include "kmc_rng.cuh"

namespace kmc {

// Point on the unit sphere by Marsaglia's method (Ann. Math. Stat. 43, 1972):
// u1, u2 uniform in [-1, 1) from 32-bit words, s = u1^2 + u2^2 accepted if
// 0 < s < 1, n = (2 u1 sqrt(1-s), 2 u2 sqrt(1-s), 1 - 2 s).  Counter (id, step lo,
// k, step hi), key (seed lo, seed hi); two attempts per Philox call.
__device__ bool sphere_point(uint64_t seed, uint64_t step, uint32_t id, double nv[3]) {
  for (uint32_t k = 0; k < 64; ++k) {
    uint32_t c[4] = {id, (uint32_t)step, k, (uint32_t)(step >> 32)};
    philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    // both attempts of the call are evaluated and the first accepted one is kept, so
    // that lanes whose first attempt fails do not split the warp
    const double u1a = word_uniform(c[0]), u2a = word_uniform(c[1]);
    const double u1b = word_uniform(c[2]), u2b = word_uniform(c[3]);
    const double sa = dadd(dmul(u1a, u1a), dmul(u2a, u2a));
    const double sb = dadd(dmul(u1b, u1b), dmul(u2b, u2b));
    const bool oka = sa > 0.0 && sa < 1.0, okb = sb > 0.0 && sb < 1.0;
    if (oka || okb) {
      const double u1 = oka ? u1a : u1b, u2 = oka ? u2a : u2b, s = oka ? sa : sb;
      const double q = dsqrt(dsub(1.0, s));
      nv[0] = dmul(dadd(u1, u1), q);
      nv[1] = dmul(dadd(u2, u2), q);
      nv[2] = dsub(1.0, dadd(s, s));
      return true;
    }
  }
  return false;
}

// Planar mode: a direction uniform on the unit circle from the same counters.  A point
// (u1, u2) uniform in the unit disk (the same rejection) has a uniform polar angle;
// the vector at twice that angle, ((u1^2 - u2^2)/s, (2 u1 u2)/s), is uniform on the
// circle (von Neumann's method, no trigonometric function).
__device__ bool circle_point(uint64_t seed, uint64_t step, uint32_t id, double nv[3]) {
  for (uint32_t k = 0; k < 64; ++k) {
    uint32_t c[4] = {id, (uint32_t)step, k, (uint32_t)(step >> 32)};
    philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    const double u1a = word_uniform(c[0]), u2a = word_uniform(c[1]);
    const double u1b = word_uniform(c[2]), u2b = word_uniform(c[3]);
    const double sa = dadd(dmul(u1a, u1a), dmul(u2a, u2a));
    const double sb = dadd(dmul(u1b, u1b), dmul(u2b, u2b));
    const bool oka = sa > 0.0 && sa < 1.0, okb = sb > 0.0 && sb < 1.0;
    if (oka || okb) {
      const double u1 = oka ? u1a : u1b, u2 = oka ? u2a : u2b, s = oka ? sa : sb;
      nv[0] = ddiv(dsub(dmul(u1, u1), dmul(u2, u2)), s);
      nv[1] = ddiv(dmul(dadd(u1, u1), u2), s);
      nv[2] = 0.0;
      return true;
    }
  }
  return false;
}

__device__ __forceinline__ double min_image(double r, double L) {
  double h = dmul(L, 0.5);
  if (r > h) return dsub(r, L);
  if (r < -h) return dadd(r, L);
  return r;
}

// ---- dealing a batch's items to the blocks ---------------------------------- //
// The items of all members (candidate pairs, work-list entries, colliding pairs) form
// one sequence dealt to the blocks: member k's first item goes to the block after the
// one that took member k - 1's last, so a batch of many small members spreads over the
// whole grid instead of piling onto the grid's first blocks.  A block reads the counts
// of up to kEdgeBlock members at once, one thread each (walked one member after
// another, the counts were a chain of dependent loads of about a microsecond per
// member and kernel), places the members by a block-wide scan of the blocks each one
// spans, and visits only the members it holds items of.  count(s) gives member s's
// items from fields that stay fixed during the launch, so every block deals alike; the
// status word is read once per member and block.  body(s, first, trips) does the
// block's share: items first, first + stride, ..., trips of them per thread, the same
// trips for every thread of the block (the last may lie past the end), so body may use
// block-wide appends.  Blocks of kEdgeBlock threads.
template <class Count, class Body>
__device__ __forceinline__ void for_dealt(const Batch& B, Count count, Body body) {
  __shared__ uint32_t s_first[kEdgeBlock], s_trips[kEdgeBlock], s_wsum[kEdgeBlock / 32];
  const uint32_t nb = gridDim.x, stride = nb * (uint32_t)kEdgeBlock;
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  uint32_t base = 0;  // the block where the chunk's first member starts
  for (int k0 = 0; k0 < B.nsims; k0 += kEdgeBlock) {
    const int k = k0 + (int)threadIdx.x;
    uint32_t c = 0;
    bool live = false;
    if (k < B.nsims) {
      const SimDev& s = *B.sims[k];
      c = count(s);
      live = s.d.status == 0;
    }
    // blocks the member spans, modulo the grid
    const uint32_t span = (uint32_t)((((uint64_t)c + kEdgeBlock - 1) / kEdgeBlock) % nb);
    uint32_t incl = span;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
      if (lane >= (uint32_t)o) incl += y;
    }
    if (lane == 31) s_wsum[warp] = incl;
    __syncthreads();
    uint32_t before = 0, total = 0;
#pragma unroll
    for (int w = 0; w < kEdgeBlock / 32; ++w) {
      const uint32_t v = s_wsum[w];
      if (w < (int)warp) before += v;
      total += v;
    }
    const uint32_t start = (base + before + incl - span) % nb;
    const uint32_t at = ((blockIdx.x + nb - start) % nb) * (uint32_t)kEdgeBlock;
    s_first[threadIdx.x] = at;
    s_trips[threadIdx.x] =
        (live && c > at) ? (uint32_t)(((uint64_t)(c - at) + stride - 1) / stride) : 0u;
    base = (base + total) % nb;
    __syncthreads();
    const int kn = B.nsims - k0 < kEdgeBlock ? B.nsims - k0 : kEdgeBlock;
    for (int j = 0; j < kn; ++j) {
      const uint32_t trips = s_trips[j];
      if (trips) body(*B.sims[k0 + j], s_first[j] + threadIdx.x, trips);
    }
    __syncthreads();  // the tables are rewritten for the next chunk
  }
}

// candidate pairs the search stored (a member whose buffer overflowed is not live)
__device__ __forceinline__ uint32_t raw_pairs(const SimDev& s) {
  return s.d.n_raw < s.edge_cap ? s.d.n_raw : s.edge_cap;
}

// ---- k_refine ------------------------------------------------------------ //
// MIX: the plan has a mixture (per-pair contact distance, mass-weighted scatter)
template <bool MIX>
__global__ void __launch_bounds__(kEdgeBlock) k_refine(Batch B) {
  for_dealt(B, [](const SimDev& s) { return sim_scheduled(s) ? raw_pairs(s) : 0u; },
            [](SimDev& s, uint32_t first, uint32_t) {
    const int cur = s.d.parity ^ 1;
    const uint32_t nraw = raw_pairs(s);
    uint32_t found = 0;
    for (uint32_t e = first; e < nraw; e += gridDim.x * kEdgeBlock) {
      uint2 pr = s.edge[e];
      uint32_t i = pr.x, j = pr.y;
      bool cand = false;
      double d2 = 0.0, t = 0.0;
      uint32_t idi = s.id[cur][i], idj = s.id[cur][j];
      // contact distance: d0, or in a mixture the sum of the two effective radii (the
      // search tested against d0, at least every such sum)
      double c2 = s.d0sq;
      if (MIX && s.mix) {
        const double c = dadd(s.sp_radius[s.species[idi]], s.sp_radius[s.species[idj]]);
        c2 = dmul(c, c);
      }
      if (!(s.last[cur][i] == idj && s.last[cur][j] == idi)) {
        double r[3], v[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          double dd = dsub(s.x[cur][a][j], s.x[cur][a][i]);
          r[a] = s.bc[a] == KMC_PERIODIC ? min_image(dd, s.box[a]) : dd;
          v[a] = dsub(s.v[cur][a][j], s.v[cur][a][i]);
        }
        double vv = dadd(dadd(dmul(v[0], v[0]), dmul(v[1], v[1])), dmul(v[2], v[2]));
        if (vv != 0.0) {
          double rv = dadd(dadd(dmul(r[0], v[0]), dmul(r[1], v[1])), dmul(r[2], v[2]));
          t = ddiv(-rv, vv);
          double wx = dsub(dmul(r[1], v[2]), dmul(r[2], v[1]));
          double wy = dsub(dmul(r[2], v[0]), dmul(r[0], v[2]));
          double wz = dsub(dmul(r[0], v[1]), dmul(r[1], v[0]));
          d2 = ddiv(dadd(dadd(dmul(wx, wx), dmul(wy, wy)), dmul(wz, wz)), vv);
          cand = t >= 0.0 && t < s.dt && d2 < c2;
        }
      }
      if (cand) {
        s.e_d2[e] = d2;
        s.e_t[e] = t;
        uint32_t si = atomicAdd(&s.deg[i], 1u);
        uint32_t sj = atomicAdd(&s.deg[j], 1u);
        s.e_slot[e] = make_uint2(si, sj);
        ++found;
      } else {
        s.e_slot[e] = make_uint2(kNone, kNone);
      }
    }
    block_append(&s.d.n_edges, found);  // one atomic per block
  });
}

// ---- candidate lists -------------------------------------------------------- //

// the pair whose slot is 0 at an endpoint opens that endpoint's list
__global__ void __launch_bounds__(kEdgeBlock) k_alloc(Batch B) {
  for_dealt(B, [](const SimDev& s) { return sim_scheduled(s) ? raw_pairs(s) : 0u; },
            [](SimDev& s, uint32_t first, uint32_t trips) {
    const uint32_t nraw = raw_pairs(s);
    const uint32_t stride = gridDim.x * kEdgeBlock;
    // the block's trip count, the same for all its threads: the appends are block-wide
    uint32_t e = first;
    for (uint32_t t = 0; t < trips; ++t, e += stride) {
      uint32_t i = kNone, j = kNone, di = 0, dj = 0;
      if (e < nraw) {
        const uint2 sl = s.e_slot[e];
        if (sl.x != kNone) {
          const uint2 pr = s.edge[e];
          if (sl.x == 0) { i = pr.x; di = s.deg[i]; }
          if (sl.y == 0) { j = pr.y; dj = s.deg[j]; }
        }
      }
      const uint32_t at = block_append(&s.d.adj_used, di + dj);
      const uint32_t wa = block_append(&s.d.wl_len[0], (i != kNone ? 1u : 0u) + (j != kNone ? 1u : 0u));
      if (i != kNone) { s.off[i] = at; s.wl[0][wa] = i; }
      if (j != kNone) { s.off[j] = at + di; s.wl[0][wa + (i != kNone ? 1u : 0u)] = j; }
    }
  });
}

__global__ void __launch_bounds__(kEdgeBlock) k_fill(Batch B) {
  for_dealt(B, [](const SimDev& s) { return sim_scheduled(s) ? raw_pairs(s) : 0u; },
            [](SimDev& s, uint32_t first, uint32_t) {
    const uint32_t nraw = raw_pairs(s);
    for (uint32_t e = first; e < nraw; e += gridDim.x * kEdgeBlock) {
      uint2 sl = s.e_slot[e];
      if (sl.x == kNone) continue;
      uint2 pr = s.edge[e];
      s.adj[s.off[pr.x] + sl.x] = make_uint2(pr.y, e);
      s.adj[s.off[pr.y] + sl.y] = make_uint2(pr.x, e);
    }
  });
}

// ---- matching rounds ------------------------------------------------------ //
__device__ __forceinline__ bool key_less(double d2a, double ta, uint32_t ja, double d2b, double tb,
                                         uint32_t jb) {
  if (d2a < d2b) return true;
  if (d2a > d2b) return false;
  if (ta < tb) return true;
  if (ta > tb) return false;
  return ja < jb;
}

// The work list of round r holds every particle that is unmatched after round r - 1
// and had an unmatched candidate in round r - 1 (round 0: every particle with a
// candidate).  A particle left off it has no unmatched candidate, so it can neither
// pick nor be picked: the rounds over the lists match exactly the pairs that rounds
// over all particles would.
__device__ __forceinline__ uint32_t round_list(const SimDev& s, int round) {
  return sim_scheduled(s) && round < s.max_rounds ? s.d.wl_len[round] : 0u;
}

__global__ void __launch_bounds__(kEdgeBlock) k_best(Batch B, int round) {
  for_dealt(B, [round](const SimDev& s) { return round_list(s, round); },
            [round](SimDev& s, uint32_t first, uint32_t) {
    const int cur = s.d.parity ^ 1;
    const uint32_t len = s.d.wl_len[round];
    const uint32_t* __restrict__ list = s.wl[round & 1];
    for (uint32_t t = first; t < len; t += gridDim.x * kEdgeBlock) {
      const uint32_t i = list[t];
      const uint32_t q0 = s.off[i], q1 = q0 + s.deg[i];
      uint32_t bj = kNone, be = kNone, bid = kNone;
      double bd2 = 0.0, bt = 0.0;
      for (uint32_t q = q0; q < q1; ++q) {
        const uint2 a = s.adj[q];
        const uint32_t j = a.x;
        if (s.partner[j] != kNone) continue;
        const double d2 = s.e_d2[a.y], tt = s.e_t[a.y];
        const uint32_t idj = s.id[cur][j];
        if (bj == kNone || key_less(d2, tt, idj, bd2, bt, bid)) {
          bj = j; be = a.y; bid = idj; bd2 = d2; bt = tt;
        }
      }
      s.best[i] = bj;
      s.best_e[i] = be;
    }
  });
}

__global__ void __launch_bounds__(kEdgeBlock) k_mutual(Batch B, int round) {
  for_dealt(B, [round](const SimDev& s) { return round_list(s, round); },
            [round](SimDev& s, uint32_t first, uint32_t trips) {
    const int cur = s.d.parity ^ 1;
    const uint32_t len = s.d.wl_len[round];
    const uint32_t* __restrict__ list = s.wl[round & 1];
    uint32_t* __restrict__ next = s.wl[(round + 1) & 1];
    const uint32_t stride = gridDim.x * kEdgeBlock;
    // the block's trip count, the same for all its threads: the appends are block-wide
    uint32_t t = first;
    for (uint32_t q = 0; q < trips; ++q, t += stride) {
      bool pair = false, again = false;
      uint32_t i = kNone;
      if (t < len) {
        i = list[t];
        const uint32_t j = s.best[i];
        if (j != kNone) {
          if (s.best[j] == i) {
            s.partner[i] = j;
            s.medge[i] = s.best_e[i];
            pair = s.id[cur][i] < s.id[cur][j];
          } else {
            again = true;
          }
        }
      }
      const uint32_t at = block_append(&s.d.n_pairs, pair ? 1u : 0u, &s.d.round_pairs[round]);
      if (pair) s.pairs[at] = i;
      if (round + 1 < s.max_rounds) {
        const uint32_t w = block_append(&s.d.wl_len[round + 1], again ? 1u : 0u);
        if (again) next[w] = i;
      }
    }
  });
}

// ---- collision update ------------------------------------------------------ //
// For the pair (a, b) with a the smaller id: stream both to t*, scatter
//   g = v_a - v_b, V = (v_a + v_b) * 0.5, G = |g|,  v_a' = V + (G/2) n,  v_b' = V - (G/2) n,
// then stream the rest of the step:  x' = (x + v t*) + v' (dt - t*).
template <bool MIX>
__global__ void __launch_bounds__(kEdgeBlock) k_collide(Batch B) {
  for_dealt(B, [](const SimDev& s) { return sim_scheduled(s) ? s.d.n_pairs : 0u; },
            [](SimDev& s, uint32_t first, uint32_t) {
    const int cur = s.d.parity ^ 1;
    const uint32_t total = s.d.n_pairs;
    for (uint32_t q = first; q < total; q += gridDim.x * kEdgeBlock) {
      // the pair list holds each colliding pair once, by its smaller-id member
      const uint32_t i = s.pairs[q];
      const uint32_t j = s.partner[i];
      const uint32_t ida = s.id[cur][i];
      double t = s.e_t[s.medge[i]];
      double nv[3];
      if (!(s.planar ? circle_point(s.seed, s.d.step, ida, nv) : sphere_point(s.seed, s.d.step, ida, nv))) {
        atomicOr(&s.d.status, ST_RANDOM);
        continue;
      }
      // equal masses: V = (v_a + v_b)/2 and both get half the relative speed; a mixture:
      // V = (m_a v_a + m_b v_b)/M, v_a' = V + (m_b/M) G n, v_b' = V - (m_a/M) G n
      const bool mixed = MIX && s.mix;
      double ma = 1.0, mb = 1.0;
      if (mixed) {
        ma = s.sp_mass[s.species[ida]];
        mb = s.sp_mass[s.species[s.id[cur][j]]];
      }
      double va[3], vb[3], g[3], V[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        va[c] = s.v[cur][c][i];
        vb[c] = s.v[cur][c][j];
        g[c] = dsub(va[c], vb[c]);
      }
      double fa = 0.5, fb = 0.5;
      if (mixed) {
        const double M = dadd(ma, mb);
#pragma unroll
        for (int c = 0; c < 3; ++c) V[c] = ddiv(dadd(dmul(ma, va[c]), dmul(mb, vb[c])), M);
        fa = ddiv(mb, M);
        fb = ddiv(ma, M);
      } else {
#pragma unroll
        for (int c = 0; c < 3; ++c) V[c] = dmul(dadd(va[c], vb[c]), 0.5);
      }
      double G = dsqrt(dadd(dadd(dmul(g[0], g[0]), dmul(g[1], g[1])), dmul(g[2], g[2])));
      const double hGa = dmul(fa, G);
      const double hGb = dmul(fb, G);
      double rest = dsub(s.dt, t);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        double na = dadd(V[c], dmul(hGa, nv[c]));
        double nb = dsub(V[c], dmul(hGb, nv[c]));
        double xa = s.x[cur][c][i], xb = s.x[cur][c][j];
        s.x[cur][c][i] = dadd(dadd(xa, dmul(va[c], t)), dmul(na, rest));
        s.x[cur][c][j] = dadd(dadd(xb, dmul(vb[c], t)), dmul(nb, rest));
        s.v[cur][c][i] = na;
        s.v[cur][c][j] = nb;
      }
    }
  });
}

int launch_match_lists(const LaunchPlan& L, cudaStream_t st) {
  const int nb = L.edge_blocks;
  if (L.mix) k_refine<true><<<nb, kEdgeBlock, 0, st>>>(L.b);
  else k_refine<false><<<nb, kEdgeBlock, 0, st>>>(L.b);
  k_alloc<<<nb, kEdgeBlock, 0, st>>>(L.b);
  k_fill<<<nb, kEdgeBlock, 0, st>>>(L.b);
  return 3;
}

int launch_collide(const LaunchPlan& L, cudaStream_t st) {
  const int nb = L.edge_blocks;
  if (L.mix) k_collide<true><<<nb, kEdgeBlock, 0, st>>>(L.b);
  else k_collide<false><<<nb, kEdgeBlock, 0, st>>>(L.b);
  return 1;
}

int launch_match(const LaunchPlan& L, int max_rounds, cudaStream_t st) {
  const int nb = L.edge_blocks;
  int n = launch_match_lists(L, st);
  for (int r = 0; r < max_rounds; ++r) {
    // the later rounds' work lists hold a few percent of the first round's: a grid of
    // one block per SM covers them (grid-stride) without launching idle blocks
    const int nr = r == 0 ? nb : std::max(1, nb / 8);
    k_best<<<nr, kEdgeBlock, 0, st>>>(L.b, r);
    k_mutual<<<nr, kEdgeBlock, 0, st>>>(L.b, r);
    n += 2;
  }
  return n + launch_collide(L, st);
}

}  // namespace kmc
