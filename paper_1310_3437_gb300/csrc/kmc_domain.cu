// kmc_domain.cu -- domain decomposition of one simulation into x slabs (Sec. 4,
// "Hybrid Simulations": the space is cut into equal domains along one axis, each
// domain keeps copies of its neighbours' particles near the cut as ghosts, and four
// communication phases per step keep the domains consistent).
//
// Each domain is a simulation of the whole box that holds every particle slot; a
// slot is present in the domain when its particle is owned there (x inside the
// domain's slab) or is a ghost (x within the reach R = d0 + 2 v_max dt of the slab),
// absent otherwise.  Absent slots carry the last-partner marker KMC_ABSORBED, so the
// sort parks them after every cell and the step kernels skip them, exactly as they
// skip particles that left through an absorbing wall.  The domains step together as
// one batch; between the kernels of a step the four phases of Sec. 4 run through
// id-indexed exchange buffers:
//   1. ghosts (and migration): every owned particle's state after the previous step
//      sits in the id-order buffer; each domain takes from it the particles it owns
//      and its ghosts (k_dom_refresh), so a particle that crossed a cut is owned by
//      its new domain from this step on;
//   2. global v_max: a max-reduction over the id-order buffer gives the common ghost
//      reach (k_dom_owner, k_dom_reach);
//   3. collision partners: in every matching round each domain publishes the best
//      partner (and then the match) of the particles it owns, and every domain
//      replaces its ghosts' choices by their owners' (k_dom_publish, k_dom_import),
//      so mutual choice across a cut is decided with the owner's complete candidate
//      set -- the paper's reason for this phase;
//   4. migration: each domain writes back the particles it owned at the start of
//      the step (k_dom_gather); ownership is recomputed from the new positions.
// A pair (a, b) is counted (candidate edges, collisions) by the domain that owns its
// smaller id, so the totals equal those of one domain.  The result is the
// single-domain result bit for bit: every candidate pair of an owned particle has
// both members present in its domain, the pair keys are the same binary64 values,
// and both domains of a pair across a cut apply the same collision update.
#include "kmc_internal.cuh"

namespace kmc {

namespace {

__device__ __forceinline__ int dom_of(const DomainDev& D, double x) {
  int lo = 0, hi = D.P;  // largest k with X[k] <= x, clamped to [0, P - 1]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (D.X[mid] <= x) lo = mid; else hi = mid;
  }
  return lo;
}

// distance along x from x to domain k's slab [X[k], X[k+1]) (on a periodic x axis the
// shorter way round); rounding only moves it by a few ulps, which the reach's margin
// covers (an extra ghost changes no result)
__device__ __forceinline__ double dom_dist(const DomainDev& D, int k, double x) {
  const double a = D.X[k], b = D.X[k + 1];
  if (x >= a && x < b) return 0.0;
  double d = x < a ? dsub(a, x) : dsub(x, b);
  if (D.periodic_x) {
    const double w = x < a ? dadd(dsub(x, b), D.Lx) : dadd(dsub(a, x), D.Lx);
    d = w < d ? w : d;
  }
  return d;
}

__device__ __forceinline__ uint32_t block_sum(uint32_t v) {
  __shared__ uint32_t ws[32];
  const uint32_t lane = threadIdx.x & 31u, w = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
  __syncthreads();
  if (lane == 0) ws[w] = v;
  __syncthreads();
  uint32_t t = 0;
  if (threadIdx.x == 0)
    for (uint32_t i = 0; i < (blockDim.x + 31u) / 32u; ++i) t += ws[i];
  return t;  // valid in thread 0
}

// phase 2 (and the owners of this step): owner domain and |v|^2 of every particle
__global__ void k_dom_owner(DomainDev* Dp) {
  DomainDev& D = *Dp;
  unsigned long long m = 0ull;
  for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < D.n; g += gridDim.x * blockDim.x) {
    D.owner[g] = (uint8_t)dom_of(D, D.x[0][g]);
    const double vx = D.v[0][g], vy = D.v[1][g], vz = D.v[2][g];
    const double q = dadd(dadd(dmul(vx, vx), dmul(vy, vy)), dmul(vz, vz));
    const unsigned long long b = (unsigned long long)__double_as_longlong(q);
    m = b > m ? b : m;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long y = __shfl_xor_sync(0xFFFFFFFFu, m, o);
    m = y > m ? y : m;
  }
  if ((threadIdx.x & 31u) == 0 && m) atomicMax(&D.vmax2_bits, m);
}

// ghost reach of the step: R = (d0 + 2 v_max dt), widened by a relative 2^-20 so that
// the rounding of R and of the distances can only add ghosts; clears the step's counters
__global__ void k_dom_reach(DomainDev* Dp) {
  DomainDev& D = *Dp;
  const double vmax = dsqrt(__longlong_as_double((long long)D.vmax2_bits));
  const double R = dadd(D.d0, dmul(dmul(2.0, vmax), D.dt));
  D.reach = dadd(dmul(R, 1.0 + 0x1p-20), 0x1p-1000);
  D.vmax2_bits = 0ull;
  for (int k = 0; k < D.P; ++k) D.owned[k] = D.ghosts[k] = 0;
  D.acc_edges = 0;
  for (int r = 0; r < 4; ++r) D.acc_round[r] = 0;
}

// phase 1: each domain takes its owned particles and its ghosts from the id-order
// buffer into its current state buffer; every other slot becomes absent
__global__ void __launch_bounds__(kTile) k_dom_refresh(Batch B, DomainDev* Dp) {
  DomainDev& D = *Dp;
  const int k = find_sim(B.ptile, B.nsims, blockIdx.x);
  SimDev& s = *B.sims[k];
  const uint32_t p = (blockIdx.x - B.ptile[k]) * kTile + threadIdx.x;
  bool own = false, ghost = false;
  if (p < s.n) {
    const int par = s.d.parity;
    const uint32_t g = s.id[par][p];
    const double x0 = D.x[0][g];
    own = D.owner[g] == (uint8_t)k;
    ghost = !own && dom_dist(D, k, x0) < D.reach;
    if (own || ghost) {
      s.x[par][0][p] = x0;
      s.x[par][1][p] = D.x[1][g];
      s.x[par][2][p] = D.x[2][g];
      for (int a = 0; a < 3; ++a) s.v[par][a][p] = D.v[a][g];
      s.last[par][p] = D.last[g];
    } else {
      s.last[par][p] = KMC_ABSORBED;
    }
  }
  const uint32_t no = block_sum(own ? 1u : 0u);
  const uint32_t ng = block_sum(ghost ? 1u : 0u);
  if (threadIdx.x == 0) {
    if (no) atomicAdd(&D.owned[k], no);
    if (ng) atomicAdd(&D.ghosts[k], ng);
  }
}

// after the sort: where each id sits in each domain's order (kNone if absent)
__global__ void __launch_bounds__(kTile) k_dom_loc(Batch B, DomainDev* Dp) {
  DomainDev& D = *Dp;
  const int k = find_sim(B.ptile, B.nsims, blockIdx.x);
  SimDev& s = *B.sims[k];
  const uint32_t p = (blockIdx.x - B.ptile[k]) * kTile + threadIdx.x;
  if (p >= s.n || !sim_active(s)) return;
  const int cur = s.d.parity ^ 1;
  D.loc[(size_t)k * D.n + s.id[cur][p]] = p < live_count(s) ? p : kNone;
}

// candidate edges counted by the domain that owns the smaller id
__global__ void __launch_bounds__(kEdgeBlock) k_dom_edges(Batch B, DomainDev* Dp) {
  DomainDev& D = *Dp;
  for (int k = 0; k < B.nsims; ++k) {
    SimDev& s = *B.sims[k];
    if (!sim_active(s)) continue;
    const int cur = s.d.parity ^ 1;
    const uint32_t nraw = s.d.n_raw < s.edge_cap ? s.d.n_raw : s.edge_cap;
    uint32_t c = 0;
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < nraw; e += gridDim.x * blockDim.x) {
      if (s.e_slot[e].x == kNone) continue;
      const uint2 pr = s.edge[e];
      const uint32_t a = s.id[cur][pr.x], b = s.id[cur][pr.y];
      if (D.owner[a < b ? a : b] == (uint8_t)k) ++c;
    }
    const uint32_t t = block_sum(c);
    if (threadIdx.x == 0 && t) atomicAdd(&D.acc_edges, t);
  }
}

// ---- matching rounds with the partner exchange ------------------------------ //
// Every round visits the particles that have candidates (the first round's list) and
// skips the matched ones.
__device__ __forceinline__ bool key_less(double d2a, double ta, uint32_t ja, double d2b, double tb,
                                         uint32_t jb) {
  if (d2a < d2b) return true;
  if (d2a > d2b) return false;
  if (ta < tb) return true;
  if (ta > tb) return false;
  return ja < jb;
}

__global__ void __launch_bounds__(kEdgeBlock) k_dom_best(Batch B) {
  for (int k = 0; k < B.nsims; ++k) {
    SimDev& s = *B.sims[k];
    if (!sim_active(s)) continue;
    const int cur = s.d.parity ^ 1;
    const uint32_t len = s.d.wl_len[0];
    const uint32_t* __restrict__ list = s.wl[0];
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < len; t += gridDim.x * blockDim.x) {
      const uint32_t i = list[t];
      uint32_t bj = kNone, be = kNone, bid = kNone;
      if (s.partner[i] == kNone) {
        double bd2 = 0.0, bt = 0.0;
        const uint32_t q0 = s.off[i], q1 = q0 + s.deg[i];
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
      }
      s.best[i] = bj;
      s.best_e[i] = be;
    }
  }
}

// what = 0: best partners, 1: matches.  Owned particles write the global id of their
// choice (or match) into the id-indexed buffer.
__global__ void __launch_bounds__(kEdgeBlock) k_dom_publish(Batch B, DomainDev* Dp, int what) {
  DomainDev& D = *Dp;
  uint32_t* out = what == 0 ? D.bestG : D.partnerG;
  for (int k = 0; k < B.nsims; ++k) {
    SimDev& s = *B.sims[k];
    if (!sim_active(s)) continue;
    const int cur = s.d.parity ^ 1;
    const uint32_t len = s.d.wl_len[0];
    const uint32_t* __restrict__ list = s.wl[0];
    const uint32_t* src = what == 0 ? s.best : s.partner;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < len; t += gridDim.x * blockDim.x) {
      const uint32_t i = list[t];
      const uint32_t g = s.id[cur][i];
      if (D.owner[g] != (uint8_t)k) continue;
      const uint32_t j = src[i];
      out[g] = j == kNone ? kNone : s.id[cur][j];
    }
  }
}

// Ghosts take their owners' choice (what = 0; the pair's edge is looked up in the
// ghost's candidate list: both members are present, so the pair is a candidate here
// too) or match (what = 1: a ghost matched to a particle this domain lacks is marked
// kElsewhere -- no longer available -- and, after the last round, kNone, so that the
// push never reads through it).
__global__ void __launch_bounds__(kEdgeBlock) k_dom_import(Batch B, DomainDev* Dp, int what,
                                                           int last_round) {
  DomainDev& D = *Dp;
  for (int k = 0; k < B.nsims; ++k) {
    SimDev& s = *B.sims[k];
    if (!sim_active(s)) continue;
    const int cur = s.d.parity ^ 1;
    const uint32_t len = s.d.wl_len[0];
    const uint32_t* __restrict__ list = s.wl[0];
    const uint32_t* __restrict__ loc = D.loc + (size_t)k * D.n;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < len; t += gridDim.x * blockDim.x) {
      const uint32_t i = list[t];
      const uint32_t g = s.id[cur][i];
      if (D.owner[g] == (uint8_t)k) continue;
      if (what == 0) {
        const uint32_t b = D.bestG[g];
        uint32_t j = b == kNone ? kNone : loc[b], e = kNone;
        if (j != kNone) {
          const uint32_t q0 = s.off[i], q1 = q0 + s.deg[i];
          for (uint32_t q = q0; q < q1; ++q) {
            const uint2 a = s.adj[q];
            if (a.x == j) { e = a.y; break; }
          }
          if (e == kNone) j = kNone;  // cannot happen (see above): never pair through it
        }
        s.best[i] = j;
        s.best_e[i] = e;
      } else {
        const uint32_t m = D.partnerG[g];
        if (m == kNone) continue;
        const uint32_t j = loc[m];
        s.partner[i] = j != kNone ? j : (last_round ? kNone : kElsewhere);
      }
    }
  }
}

__global__ void __launch_bounds__(kEdgeBlock) k_dom_mutual(Batch B, DomainDev* Dp, int round) {
  DomainDev& D = *Dp;
  for (int k = 0; k < B.nsims; ++k) {
    SimDev& s = *B.sims[k];
    if (!sim_active(s)) continue;
    const int cur = s.d.parity ^ 1;
    const uint32_t len = s.d.wl_len[0];
    const uint32_t* __restrict__ list = s.wl[0];
    const uint32_t stride = gridDim.x * blockDim.x;
    const uint32_t span = ((len + stride - 1) / stride) * stride;  // block-wide appends
    uint32_t counted = 0;
    for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < span; t += stride) {
      bool pair = false;
      uint32_t i = kNone;
      if (t < len) {
        i = list[t];
        const uint32_t j = s.best[i];
        if (s.partner[i] == kNone && j != kNone && s.best[j] == i) {
          s.partner[i] = j;
          s.medge[i] = s.best_e[i];
          const uint32_t gi = s.id[cur][i];
          pair = gi < s.id[cur][j];
          if (pair && D.owner[gi] == (uint8_t)k) ++counted;
        }
      }
      const uint32_t at = block_append(&s.d.n_pairs, pair ? 1u : 0u, &s.d.round_pairs[round]);
      if (pair) s.pairs[at] = i;
    }
    const uint32_t c = block_sum(counted);
    if (threadIdx.x == 0 && c) atomicAdd(&D.acc_round[round], c);
  }
}

// phase 4: after the push (the domains' current buffers hold the new state), each
// domain writes back the particles it owned at the start of the step, with the
// global id of their partner in the step
__global__ void __launch_bounds__(kTile) k_dom_gather(Batch B, DomainDev* Dp) {
  DomainDev& D = *Dp;
  const int k = find_sim(B.ptile, B.nsims, blockIdx.x);
  SimDev& s = *B.sims[k];
  const uint32_t p = (blockIdx.x - B.ptile[k]) * kTile + threadIdx.x;
  if (p >= s.n) return;
  const int par = s.d.parity;
  if (s.last[par][p] == KMC_ABSORBED) return;  // absent
  const uint32_t g = s.id[par][p];
  if (D.owner[g] != (uint8_t)k) return;
  for (int a = 0; a < 3; ++a) {
    D.x[a][g] = s.x[par][a][p];
    D.v[a][g] = s.v[par][a][p];
  }
  D.last[g] = s.last[par][p];
  const uint32_t q = s.partner[p];
  D.partner_out[g] = q == kNone ? kNone : s.id[par][q];
}

// the step's record: counts of the owning domains, pair tests and cells of all domains
__global__ void k_dom_record(Batch B, DomainDev* Dp) {
  DomainDev& D = *Dp;
  kmc_step_counts rec = {};
  const SimDev& s0 = *B.sims[0];
  rec.step = s0.d.step - 1;
  uint32_t coll = 0;
  for (int r = 0; r < 4; ++r) {
    rec.round_pairs[r] = D.acc_round[r];
    coll += D.acc_round[r];
  }
  rec.collisions = coll;
  rec.edges = D.acc_edges;
  for (int k = 0; k < B.nsims; ++k) {
    const SimDev& s = *B.sims[k];
    if (s.d.hist_count == 0) continue;
    const kmc_step_counts& h = s.hist[(s.d.hist_count - 1) % s.hist_cap];
    rec.pair_tests += h.pair_tests;
    rec.survivors += h.survivors;
    rec.cells += h.cells;
  }
  rec.live = D.n;
  D.hist[D.hist_count % D.hist_cap] = rec;
  D.hist_count += 1;
}

// KMC_OBS_EDGES of a decomposition: the last step's candidate pairs, each from the
// domain that owns its smaller id
__global__ void k_dom_gather_edges(Batch B, DomainDev* Dp, uint32_t cap, uint2* out, uint32_t* count) {
  DomainDev& D = *Dp;
  for (int k = 0; k < B.nsims; ++k) {
    const SimDev& s = *B.sims[k];
    const int par = s.d.parity;
    const uint32_t nraw = s.d.last_raw < s.edge_cap ? s.d.last_raw : s.edge_cap;
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < nraw; e += gridDim.x * blockDim.x) {
      if (s.e_slot[e].x == kNone) continue;
      const uint2 pr = s.edge[e];
      const uint32_t a = s.id[par][pr.x], b = s.id[par][pr.y];
      const uint32_t lo = a < b ? a : b, hi = a < b ? b : a;
      if (D.owner[lo] != (uint8_t)k) continue;
      const uint32_t pos = atomicAdd(count, 1u);
      if (pos < cap) out[pos] = make_uint2(lo, hi);
    }
  }
}

__global__ void k_dom_vmax(const DomainDev* Dp, unsigned long long* acc) {
  const DomainDev& D = *Dp;
  unsigned long long m = 0ull;
  for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < D.n; g += gridDim.x * blockDim.x) {
    const double vx = D.v[0][g], vy = D.v[1][g], vz = D.v[2][g];
    const double q = dadd(dadd(dmul(vx, vx), dmul(vy, vy)), dmul(vz, vz));
    const unsigned long long b = (unsigned long long)__double_as_longlong(q);
    m = b > m ? b : m;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long y = __shfl_xor_sync(0xFFFFFFFFu, m, o);
    m = y > m ? y : m;
  }
  if ((threadIdx.x & 31u) == 0 && m) atomicMax(acc, m);
}

__global__ void k_dom_vmax_sqrt(const unsigned long long* acc, double* out) {
  out[0] = dsqrt(__longlong_as_double((long long)*acc));
}

}  // namespace

int launch_domain_step(const LaunchPlan& L, DomainDev* D, uint32_t n, int precision, int K,
                       int max_rounds, cudaStream_t st) {
  const int nb = L.edge_blocks;
  int c = 0;
  k_dom_owner<<<4 * 152, 256, 0, st>>>(D);
  k_dom_reach<<<1, 1, 0, st>>>(D);
  k_dom_refresh<<<L.ptiles, kTile, 0, st>>>(L.b, D);
  c += 3;
  c += launch_init_grid(L, st);  // each domain's grid from the particles it now holds
  c += launch_sort(L, st);
  k_dom_loc<<<L.ptiles, kTile, 0, st>>>(L.b, D);
  c += 1;
  c += launch_search(L, precision, K, st);
  c += launch_match_lists(L, st);
  k_dom_edges<<<nb, kEdgeBlock, 0, st>>>(L.b, D);
  c += 1;
  for (int r = 0; r < max_rounds; ++r) {
    const int last = r + 1 == max_rounds;
    k_dom_best<<<nb, kEdgeBlock, 0, st>>>(L.b);
    k_dom_publish<<<nb, kEdgeBlock, 0, st>>>(L.b, D, 0);
    k_dom_import<<<nb, kEdgeBlock, 0, st>>>(L.b, D, 0, last);
    k_dom_mutual<<<nb, kEdgeBlock, 0, st>>>(L.b, D, r);
    k_dom_publish<<<nb, kEdgeBlock, 0, st>>>(L.b, D, 1);
    k_dom_import<<<nb, kEdgeBlock, 0, st>>>(L.b, D, 1, last);
    c += 6;
  }
  c += launch_collide(L, st);
  c += launch_push(L, st);
  k_dom_gather<<<L.ptiles, kTile, 0, st>>>(L.b, D);
  k_dom_record<<<1, 1, 0, st>>>(L.b, D);
  (void)n;
  return c + 2;
}

void launch_domain_edges(const LaunchPlan& L, DomainDev* D, uint32_t cap, uint2* out,
                         uint32_t* count, cudaStream_t st) {
  k_dom_gather_edges<<<304, 256, 0, st>>>(L.b, D, cap, out, count);
}

void launch_domain_vmax(const DomainDev* D, unsigned long long* acc, double* out, cudaStream_t st) {
  cudaMemsetAsync(acc, 0, sizeof(unsigned long long), st);
  k_dom_vmax<<<304, 256, 0, st>>>(D, acc);
  k_dom_vmax_sqrt<<<1, 1, 0, st>>>(acc, out);
}

}  // namespace kmc
