// kmc_push.cu -- free streaming, boundaries, observables and the end-of-step
// bookkeeping (Sec. 2: positions updated, boundary conditions applied to particles
// that reach the walls; output at fixed intervals).
//
//   k_push      x += v dt for particles that did not collide (colliders were
//               streamed by k_collide), then the boundaries per axis:
//                 periodic   one wrap into [0, L), x == L mapped to 0;
//                 reflecting lower wall at 0; upper wall at L, or on x at the piston
//                            X = x0 - u ((step+1) dt): x -> 2X - x, v -> -v - 2u
//                            (specular reflection in the frame of the moving wall).
//               It also records the last partner and a binary32 upper bound of
//               max |v|^2 (directed rounding) for the next step's cell size.
//   k_profile   every profile_every steps: per x-bin count, sum v and sum v^2, in
//               exact fixed point (int64 digits), so the sums do not depend on the
//               order of the particles.
//   k_finalize  one thread per simulation: step record, step counter, the next
//               grid (kmc_grid.cuh) and the per-step counters reset.
#include "kmc_grid.cuh"
#include "kmc_internal.cuh"

namespace kmc {

__device__ __forceinline__ void block_max_to(uint32_t* dst, float v) {
  __shared__ float wmax[kTile / 32];
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_down_sync(0xFFFFFFFFu, v, o));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    float m = 0.0f;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) m = fmaxf(m, wmax[w]);
    atomicMax(dst, __float_as_uint(m));
  }
}

// Comparisons of finite doubles on the integer pipes (the binary64 pipe is the
// scarce one on this part).  For a finite x and a positive finite bound y the order
// of the values is the order of the bit patterns read as signed integers; negative
// x (including -0.0) compare below every positive y.
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ bool lt_zero(double x) {  // x < 0.0 (false for -0.0)
  return (unsigned long long)dbits(x) > 0x8000000000000000ull;
}

// ---- k_push ---------------------------------------------------------------- //
// The boundary fix-ups are rare (particles that crossed a wall or the periodic
// boundary in this step).  They sit in out-of-line functions so that their binary64
// operations issue only for the lanes that call them, instead of being predicated
// into every lane's instruction stream.
struct XV {
  double x, v;
};

// periodic axis: one wrap into [0, L), x == L mapped to 0
__device__ __noinline__ double wrap_periodic(double x, double L) {
  if (dbits(x) >= dbits(L)) x = dsub(x, L);
  if (lt_zero(x)) {
    x = dadd(x, L);
    if (dbits(x) == dbits(L)) x = 0.0;
  }
  return x;
}

// reflecting axis: lower wall at 0, upper wall (or piston) at X moving with u
__device__ __noinline__ XV reflect_walls(double x, double v, double X, double u) {
  if (lt_zero(x)) {
    x = -x;
    v = -v;
  }
  if (dbits(X) > 0 ? dbits(x) > dbits(X) : x > X) {
    x = dsub(dadd(X, X), x);
    v = dsub(-v, dadd(u, u));
  }
  return {x, v};
}

// Free streaming and walls of one particle (sorted position p); returns the binary32
// upper bound of its |v|^2 (0 if it left).  ABS: the simulation has absorbing walls.
template <bool ABS>
__device__ __forceinline__ float push_particle(SimDev& s, int cur, uint32_t p, double dt, double sX,
                                               bool& gone) {
  const uint32_t q = s.partner[p];
  double vv[3];
  if (!ABS) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      double x = s.x[cur][a][p];
      double v = s.v[cur][a][p];
      if (q == kNone) x = dadd(x, dmul(v, dt));
      if (s.bc[a] == KMC_PERIODIC) {
        const double L = s.box[a];  // > 0
        if (dbits(x) >= dbits(L) || lt_zero(x)) x = wrap_periodic(x, L);
      } else {
        const double X = a == 0 ? sX : s.box[a];
        const double u = a == 0 ? s.piston_u : 0.0;
        if (lt_zero(x) || (dbits(X) > 0 ? dbits(x) > dbits(X) : x > X)) {
          const XV r = reflect_walls(x, v, X, u);
          x = r.x;
          v = r.v;
          s.v[cur][a][p] = v;
        }
      }
      s.x[cur][a][p] = x;
      vv[a] = v;
    }
    if (q != kNone) s.last[cur][p] = s.id[cur][q];
    return vmag2_up(vv[0], vv[1], vv[2]);
  }
  double xs[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    xs[a] = s.x[cur][a][p];
    vv[a] = s.v[cur][a][p];
    if (q == kNone) xs[a] = dadd(xs[a], dmul(vv[a], dt));
  }
  // beyond an absorbing wall at the end of the step: the particle leaves the gas with
  // this position and velocity (tested before any other axis' boundary)
#pragma unroll
  for (int a = 0; a < 3; ++a)
    if (s.bc[a] == KMC_ABSORB && (lt_zero(xs[a]) || xs[a] > s.box[a])) gone = true;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    double x = xs[a];
    double v = vv[a];
    if (gone || s.bc[a] == KMC_ABSORB) {
      // no wall acts (inside on this axis, or the particle has left)
    } else if (s.bc[a] == KMC_PERIODIC) {
      const double L = s.box[a];
      if (dbits(x) >= dbits(L) || lt_zero(x)) x = wrap_periodic(x, L);
    } else {
      const double X = a == 0 ? sX : s.box[a];
      const double u = a == 0 ? s.piston_u : 0.0;
      if (lt_zero(x) || (dbits(X) > 0 ? dbits(x) > dbits(X) : x > X)) {
        const XV r = reflect_walls(x, v, X, u);
        x = r.x;
        v = r.v;
        s.v[cur][a][p] = v;
      }
    }
    s.x[cur][a][p] = x;
    vv[a] = v;
  }
  if (gone) s.last[cur][p] = KMC_ABSORBED;
  else if (q != kNone) s.last[cur][p] = s.id[cur][q];
  return gone ? 0.0f : vmag2_up(vv[0], vv[1], vv[2]);
}

template <bool ABS>
__global__ void __launch_bounds__(kTile) k_push(Batch B) {
  __shared__ double sX;                       // piston position at the end of the step
  __shared__ uint32_t scnt[kSplitTrials];     // particles above each trial threshold
  __shared__ uint32_t sgone;                  // particles absorbed in this block
  int k = find_sim(B.ptile, B.nsims, blockIdx.x);
  SimDev& s = *B.sims[k];
  if (!sim_active(s)) return;
  const int cur = s.d.parity ^ 1;
  const uint64_t step = s.d.step;
  const double dt = s.dt;
  if (threadIdx.x == 0)
    sX = s.bc[0] == KMC_PERIODIC ? 0.0
                                 : dsub(s.piston_x0, dmul(s.piston_u, dmul((double)(step + 1), dt)));
  if (threadIdx.x < kSplitTrials) scnt[threadIdx.x] = 0;
  if (ABS && threadIdx.x == 0) sgone = 0;
  __syncthreads();
  uint32_t p = (blockIdx.x - B.ptile[k]) * kTile + threadIdx.x;
  float vm = 0.0f;
  // absorbing walls: particles that left earlier sit at the end of the order and stay
  // as they are (live_count is this step's sort's count of the others)
  const uint32_t n_in = ABS ? live_count(s) : s.n;
  bool gone = false;
  if (p < n_in) vm = (ABS && s.absorb) ? push_particle<true>(s, cur, p, dt, sX, gone)
                                       : push_particle<false>(s, cur, p, dt, sX, gone);
  if (ABS && s.absorb) {
    const unsigned m = __ballot_sync(0xFFFFFFFFu, gone);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(&sgone, (uint32_t)__popc(m));
  }
  if (s.split_ok) {
    // particles above each trial split threshold: warp ballots, shared counters, one
    // global atomic per block and trial; each particle keeps how many thresholds it
    // exceeds, which is all the next step's count needs to classify it
    const bool valid = p < n_in && !gone;
    uint32_t above = 0;
#pragma unroll
    for (int t = 1; t < kSplitTrials; ++t) {
      const bool hi = valid && vm > s.d.split_thr[t];
      above += hi ? 1u : 0u;
      unsigned m = __ballot_sync(0xFFFFFFFFu, hi);
      if ((threadIdx.x & 31) == 0 && m) atomicAdd(&scnt[t], (uint32_t)__popc(m));
    }
    if (valid) s.vbucket[p] = (uint8_t)above;
  }
  block_max_to(&s.d.vmax2_acc, vm);  // its block barrier also orders the shared counters
  if (s.split_ok && threadIdx.x > 0 && threadIdx.x < kSplitTrials && scnt[threadIdx.x])
    atomicAdd(&s.d.split_cnt[threadIdx.x], scnt[threadIdx.x]);
  if (ABS && s.absorb && threadIdx.x == 0 && sgone) atomicAdd(&s.d.n_absorbed, sgone);
}

template <bool ABS>
__global__ void __launch_bounds__(kTile) k_profile(Batch B) {
  extern __shared__ long long acc[];
  int k = find_sim(B.prtile, B.nsims, blockIdx.x);
  SimDev& s = *B.sims[k];
  if (!sim_active(s) || !s.d.prof_due) return;
  const int nb = s.profile_bins;
  for (int i = threadIdx.x; i < nb * kProfQ; i += blockDim.x) acc[i] = 0;
  __syncthreads();
  const int cur = s.d.parity ^ 1;
  const double scale = ddiv((double)nb, s.profile_range);
  uint32_t base = (blockIdx.x - B.prtile[k]) * kProfTile;
  for (uint32_t i = threadIdx.x; i < kProfTile; i += blockDim.x) {
    uint32_t p = base + i;
    if (p >= s.n) break;
    if (ABS && s.absorb && s.last[cur][p] == KMC_ABSORBED) continue;  // out of the gas
    double x = s.x[cur][0][p];
    if (!(x >= 0.0)) continue;
    double f = dmul(x, scale);
    if (f >= (double)nb) continue;
    int b = (int)f;
    const double v[3] = {s.v[cur][0][p], s.v[cur][1][p], s.v[cur][2][p]};
    profile_add(acc + b * kProfQ, v);
  }
  __syncthreads();
  long long* out = s.prof_acc + (size_t)(s.d.prof_count % s.prof_cap) * nb * kProfQ;
  for (int i = threadIdx.x; i < nb * kProfQ; i += blockDim.x)
    if (acc[i]) atomicAdd((unsigned long long*)&out[i], (unsigned long long)acc[i]);
}

// ---- end of step ------------------------------------------------------------ //
__device__ void reset_step_counters(SimDev& s) {
  s.d.n_raw = 0;
  s.d.n_edges = 0;
  for (int r = 0; r < 4; ++r) s.d.round_pairs[r] = 0;
  s.d.n_pairs = 0;
  s.d.adj_used = 0;
  for (int r = 0; r < 5; ++r) s.d.wl_len[r] = 0;
  s.d.pair_tests = 0;
  s.d.fast_tests = 0;
  s.d.n_absorbed = 0;
  s.d.vmax2_acc = 0;
}

__device__ void set_prof_due(SimDev& s) {
  s.d.prof_due = (s.profile_bins > 0 && s.profile_every > 0 &&
                  (s.d.step + 1) % (uint64_t)s.profile_every == 0) ? 1u : 0u;
}

// one warp per simulation: lane 0 keeps the books, the warp builds the next grid
__global__ void k_finalize(Batch B) {
  const uint32_t lane = threadIdx.x & 31u;
  const int nwarps = (int)(gridDim.x * blockDim.x / 32u);
  for (int k = (int)((blockIdx.x * blockDim.x + threadIdx.x) / 32u); k < B.nsims; k += nwarps) {
    SimDev& s = *B.sims[k];
    if (!sim_active(s)) continue;
    if (lane == 0) {
      kmc_step_counts rec;
      rec.step = s.d.step;
      uint32_t coll = 0;
      for (int r = 0; r < 4; ++r) {
        rec.round_pairs[r] = s.d.round_pairs[r];
        coll += s.d.round_pairs[r];
      }
      rec.collisions = coll;
      rec.edges = s.d.n_edges;
      rec.survivors = s.d.n_raw;
      rec.cells = s.d.grid.nkeys;
      rec.pair_tests = s.d.pair_tests;
      rec.fast_tests = s.d.fast_tests;
      rec.absorbed = s.d.n_absorbed;
      rec.live = live_count(s) - s.d.n_absorbed;  // this step's grid, before the next one
      s.hist[s.d.hist_count % s.hist_cap] = rec;
      s.d.hist_count += 1;
      if (s.d.prof_due) {
        s.prof_step[s.d.prof_count % s.prof_cap] = s.d.step;
        s.d.prof_count += 1;
      }
      s.d.last_raw = s.d.n_raw;
      s.d.have_counts = s.split_ok ? 1u : 0u;
      s.d.parity ^= 1u;
      s.d.step += 1;
      s.d.steps_left -= 1;
      s.d.vmax2 = __uint_as_float(s.d.vmax2_acc);
    }
    __syncwarp();
    compute_grid(s, s.d.vmax2, s.d.step, lane);
    __syncwarp();
    if (lane == 0) {
      reset_step_counters(s);
      set_prof_due(s);
    }
    __syncwarp();
    if (s.d.prof_due) {
      long long* out = s.prof_acc + (size_t)(s.d.prof_count % s.prof_cap) * s.profile_bins * kProfQ;
      for (int i = (int)lane; i < s.profile_bins * kProfQ; i += 32) out[i] = 0;
    }
    __syncwarp();
  }
}

// ---- initial grid (creation, resume, after an error is cleared) ------------ //
template <bool ABS>
__global__ void __launch_bounds__(kTile) k_vmax(Batch B) {
  int k = find_sim(B.ptile, B.nsims, blockIdx.x);
  SimDev& s = *B.sims[k];
  uint32_t p = (blockIdx.x - B.ptile[k]) * kTile + threadIdx.x;
  float vm = 0.0f;
  if (p < s.n) {
    int par = s.d.parity;
    if (!(ABS && s.absorb && s.last[par][p] == KMC_ABSORBED))
      vm = vmag2_up(s.v[par][0][p], s.v[par][1][p], s.v[par][2][p]);
  }
  block_max_to(&s.d.vmax2_acc, vm);
}

// the trial thresholds of the speed split from the state's bound of max |v|^2
__global__ void k_init_thresholds(Batch B) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < B.nsims; k += gridDim.x * blockDim.x) {
    SimDev& s = *B.sims[k];
    s.d.vmax2 = __uint_as_float(s.d.vmax2_acc);
    set_split_thresholds(s, s.d.vmax2);
  }
}

// particles above each trial threshold, and each particle's speed class, as the push
// counts them at the end of a step: the first step can split the fast particles off
template <bool ABS>
__global__ void __launch_bounds__(kTile) k_split_count(Batch B) {
  __shared__ uint32_t scnt[kSplitTrials];
  const int k = find_sim(B.ptile, B.nsims, blockIdx.x);
  SimDev& s = *B.sims[k];
  if (!s.split_ok) return;
  if (threadIdx.x < kSplitTrials) scnt[threadIdx.x] = 0;
  __syncthreads();
  const uint32_t p = (blockIdx.x - B.ptile[k]) * kTile + threadIdx.x;
  const int par = s.d.parity;
  const bool valid = p < s.n && !(ABS && s.absorb && s.last[par][p] == KMC_ABSORBED);
  const float vm = valid ? vmag2_up(s.v[par][0][p], s.v[par][1][p], s.v[par][2][p]) : 0.0f;
  uint32_t above = 0;
#pragma unroll
  for (int t = 1; t < kSplitTrials; ++t) {
    const bool hi = valid && vm > s.d.split_thr[t];
    above += hi ? 1u : 0u;
    const unsigned m = __ballot_sync(0xFFFFFFFFu, hi);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(&scnt[t], (uint32_t)__popc(m));
  }
  if (valid) s.vbucket[p] = (uint8_t)above;
  __syncthreads();
  if (threadIdx.x > 0 && threadIdx.x < kSplitTrials && scnt[threadIdx.x])
    atomicAdd(&s.d.split_cnt[threadIdx.x], scnt[threadIdx.x]);
}

// one warp per simulation, as k_finalize
__global__ void k_init_grid(Batch B) {
  const uint32_t lane = threadIdx.x & 31u;
  const int nwarps = (int)(gridDim.x * blockDim.x / 32u);
  for (int k = (int)((blockIdx.x * blockDim.x + threadIdx.x) / 32u); k < B.nsims; k += nwarps) {
    SimDev& s = *B.sims[k];
    if (lane == 0) s.d.have_counts = s.split_ok ? 1u : 0u;  // k_split_count's
    __syncwarp();
    compute_grid(s, s.d.vmax2, s.d.step, lane);
    __syncwarp();
    if (lane == 0) {
      reset_step_counters(s);
      set_prof_due(s);
    }
    __syncwarp();
    if (s.d.prof_due && s.prof_acc) {
      long long* out = s.prof_acc + (size_t)(s.d.prof_count % s.prof_cap) * s.profile_bins * kProfQ;
      for (int i = (int)lane; i < s.profile_bins * kProfQ; i += 32) out[i] = 0;
    }
    __syncwarp();
  }
}

__global__ void k_zero_vmax(Batch B) {
  for (int k = threadIdx.x; k < B.nsims; k += blockDim.x) B.sims[k]->d.vmax2_acc = 0;
}

int launch_init_grid(const LaunchPlan& L, cudaStream_t st) {
  k_zero_vmax<<<1, 256, 0, st>>>(L.b);
  if (L.absorb) k_vmax<true><<<L.ptiles, kTile, 0, st>>>(L.b);
  else k_vmax<false><<<L.ptiles, kTile, 0, st>>>(L.b);
  k_init_thresholds<<<(L.b.nsims + 255) / 256, 256, 0, st>>>(L.b);
  if (L.absorb) k_split_count<true><<<L.ptiles, kTile, 0, st>>>(L.b);
  else k_split_count<false><<<L.ptiles, kTile, 0, st>>>(L.b);
  k_init_grid<<<(L.b.nsims + 7) / 8, 256, 0, st>>>(L.b);
  return 5;
}

int launch_push(const LaunchPlan& L, cudaStream_t st) {
  if (L.absorb) {
    k_push<true><<<L.ptiles, kTile, 0, st>>>(L.b);
    k_profile<true><<<L.prtiles, kTile, 256 * kProfQ * sizeof(long long), st>>>(L.b);
  } else {
    k_push<false><<<L.ptiles, kTile, 0, st>>>(L.b);
    k_profile<false><<<L.prtiles, kTile, 256 * kProfQ * sizeof(long long), st>>>(L.b);
  }
  k_finalize<<<(L.b.nsims + 7) / 8, 256, 0, st>>>(L.b);
  return 3;
}

__global__ void k_add_steps(SimDev* d, uint64_t n) { d->d.steps_left += n; }
void launch_add_steps(SimDev* d, uint64_t nsteps, cudaStream_t st) {
  k_add_steps<<<1, 1, 0, st>>>(d, nsteps);
}

// ---- observables ------------------------------------------------------------ //
// The state in id order (x, y, z, vx, vy, vz as n binary64 each, then n last
// partners).  Written as a gather: k_state_where scatters each particle's sorted
// position into the last-partner section (one 4-byte store per particle), then
// k_gather_state walks the ids in order, reads every field from that position and
// writes all seven arrays with coalesced stores (the last partner replaces the
// position it was read from).  Scattering the seven fields directly, 8-byte stores
// to random addresses, made the memory system read back most sectors it wrote.
__global__ void k_state_where(SimDev* d, void* out) {
  SimDev& s = *d;
  const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= s.n) return;
  uint32_t* ol = (uint32_t*)((double*)out + (size_t)6 * s.n);
  ol[s.id[s.d.parity][p]] = p;
}

__global__ void k_gather_state(SimDev* d, void* out) {
  SimDev& s = *d;
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= s.n) return;
  const int par = s.d.parity;
  double* o = (double*)out;
  uint32_t* ol = (uint32_t*)(o + (size_t)6 * s.n);
  const uint32_t p = ol[i];
  for (int a = 0; a < 3; ++a) {
    o[(size_t)a * s.n + i] = s.x[par][a][p];
    o[(size_t)(3 + a) * s.n + i] = s.v[par][a][p];
  }
  ol[i] = s.last[par][p];
}

__global__ void k_gather_partners(SimDev* d, uint32_t* out) {
  SimDev& s = *d;
  uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= s.n) return;
  // partners refer to the buffer the last step ran on, which is the current one
  int par = s.d.parity;
  uint32_t q = s.partner[p];
  out[s.id[par][p]] = q == kNone ? kNone : s.id[par][q];
}

__global__ void k_gather_edges(SimDev* d, uint32_t cap, uint2* out, uint32_t* count) {
  SimDev& s = *d;
  int par = s.d.parity;
  uint32_t nraw = s.d.last_raw < s.edge_cap ? s.d.last_raw : s.edge_cap;
  for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < nraw; e += gridDim.x * blockDim.x) {
    uint2 sl = s.e_slot[e];
    if (sl.x == kNone) continue;
    uint2 pr = s.edge[e];
    uint32_t a = s.id[par][pr.x], b = s.id[par][pr.y];
    uint32_t pos = atomicAdd(count, 1u);
    if (pos < cap) out[pos] = a < b ? make_uint2(a, b) : make_uint2(b, a);
  }
}

__global__ void k_profile_convert(SimDev* d, uint32_t first, uint32_t count, uint32_t bins, double* out) {
  SimDev& s = *d;
  uint32_t total = count * bins * 7;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    uint32_t snap = i / (bins * 7), rem = i % (bins * 7), b = rem / 7, q = rem % 7;
    const long long* src = s.prof_acc + ((size_t)((first + snap) % s.prof_cap) * bins + b) * kProfQ;
    out[i] = profile_value(src, (int)q);
  }
}

// KMC_OBS_VMAX: max over the particles in the gas of (vx*vx + vy*vy) + vz*vz, each
// operation correctly rounded; the squares are non-negative, so their bit patterns
// order as their values and one 64-bit atomicMax per warp reduces them exactly
__global__ void k_vmax_exact(SimDev* d, unsigned long long* acc) {
  SimDev& s = *d;
  const int par = s.d.parity;
  unsigned long long m = 0ull;
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < s.n; p += gridDim.x * blockDim.x) {
    if (s.absorb && s.last[par][p] == KMC_ABSORBED) continue;
    const double vx = s.v[par][0][p], vy = s.v[par][1][p], vz = s.v[par][2][p];
    const double q = dadd(dadd(dmul(vx, vx), dmul(vy, vy)), dmul(vz, vz));
    const unsigned long long b = (unsigned long long)__double_as_longlong(q);
    m = b > m ? b : m;
  }
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long o = __shfl_xor_sync(0xFFFFFFFFu, m, off);
    m = o > m ? o : m;
  }
  if ((threadIdx.x & 31u) == 0 && m) atomicMax(acc, m);
}

__global__ void k_vmax_sqrt(const unsigned long long* acc, double* out) {
  out[0] = dsqrt(__longlong_as_double((long long)*acc));
}

void launch_vmax_exact(SimDev* d, unsigned long long* acc, double* out, cudaStream_t st) {
  cudaMemsetAsync(acc, 0, sizeof(unsigned long long), st);
  k_vmax_exact<<<304, 256, 0, st>>>(d, acc);
  k_vmax_sqrt<<<1, 1, 0, st>>>(acc, out);
}

// particles outside the box at creation: count them (host reports KMC_EINVAL)
__global__ void k_validate(SimDev* d, uint32_t* bad) {
  SimDev& s = *d;
  uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= s.n) return;
  bool out = false;
  // a particle that already left through an absorbing wall may lie anywhere (finite)
  const bool left = s.absorb && s.last[s.d.parity][p] == KMC_ABSORBED;
  for (int a = 0; a < 3; ++a) {
    double q = s.x[s.d.parity][a][p];
    double hi = (a == 0 && s.bc[0] == KMC_REFLECT) ? s.piston_x0 : s.box[a];
    bool periodic = s.bc[a] == KMC_PERIODIC;
    if (left ? !(fabs(q) < 1e300) : (!(q >= 0.0) || (periodic ? !(q < hi) : !(q <= hi)))) out = true;
    if (!(fabs(s.v[s.d.parity][a][p]) < 1e15)) out = true;
  }
  if (s.planar && s.v[s.d.parity][2][p] != 0.0) out = true;
  if (s.mix && s.species[s.id[s.d.parity][p]] >= (uint32_t)s.mix_n) out = true;
  if (out) atomicAdd(bad, 1u);
}

void launch_validate(SimDev* d, uint32_t n, uint32_t* bad, cudaStream_t st) {
  k_validate<<<(n + 255) / 256, 256, 0, st>>>(d, bad);
}

void launch_gather_state(SimDev* d, uint32_t n, void* out, cudaStream_t st) {
  if (n == 0) return;
  k_state_where<<<(n + 255) / 256, 256, 0, st>>>(d, out);
  k_gather_state<<<(n + 255) / 256, 256, 0, st>>>(d, out);
}
void launch_gather_partners(SimDev* d, uint32_t n, uint32_t* out, cudaStream_t st) {
  k_gather_partners<<<(n + 255) / 256, 256, 0, st>>>(d, out);
}
void launch_gather_edges(SimDev* d, uint32_t cap, uint2* out, uint32_t* count, cudaStream_t st) {
  k_gather_edges<<<304, 256, 0, st>>>(d, cap, out, count);
}
void launch_profile_convert(SimDev* d, uint32_t first, uint32_t count, uint32_t bins, double* out,
                            cudaStream_t st) {
  if (count == 0) return;
  k_profile_convert<<<152, 256, 0, st>>>(d, first, count, bins, out);
}

}  // namespace kmc
