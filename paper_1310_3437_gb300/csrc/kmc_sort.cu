// kmc_sort.cu -- binning of the particles into cells (Sec. 2: every particle is
// appended to the list of its bin; the grid is rebuilt every step).
//
// GB300 form: a counting sort into a column-Morton cell order.
//   k_count   cell key per particle; rank inside the cell by a warp-aggregated
//             atomic increment (a run of equal keys in neighbouring lanes shares one
//             atomic).
//   scan      segmented exclusive scan of the counts -> cell_start (one launch,
//             decoupled look-back); clears the counts for the next step.
//   k_scatter records the source of every position of the new order;
//   k_gather  permutes the binary64 state into the other buffer, writes the
//             binary32 mirror (box coordinates and velocity) for the guarded
//             search and resets the per-particle step arrays.
// The order inside a cell depends on atomic timing; nothing downstream depends on
// it (argmin over a total order, integer counters, order-free profile sums).
#include "kmc_internal.cuh"

namespace kmc {

// --------------------------------------------------------------------------- //
// run of equal keys in consecutive lanes: rank of each valid lane, one atomic per run
__device__ __forceinline__ uint32_t run_rank(uint32_t* counts, uint32_t key, bool valid, uint32_t lane) {
  // warp aggregation over runs of equal keys: the particles come in the previous
  // step's cell order, so equal keys mostly sit in neighbouring lanes.  Each run of
  // equal keys in consecutive lanes takes one atomic for all its members (a key that
  // appears in two runs takes two; the ranks stay distinct either way).
  const uint32_t prev = __shfl_up_sync(0xFFFFFFFFu, key, 1);
  const bool head = valid && (lane == 0 || prev != key);  // valid lanes are a prefix
  const unsigned heads = __ballot_sync(0xFFFFFFFFu, head);
  const unsigned vmask = __ballot_sync(0xFFFFFFFFu, valid);
  // this lane's run: from the last head at or below it to the next head (or the end
  // of the valid lanes)
  const unsigned le = heads & (0xFFFFFFFFu >> (31u - lane));
  const int lead = 31 - __clz((int)le);
  uint32_t base = 0;
  if (head) {
    const unsigned above = heads & ~(0xFFFFFFFFu >> (31u - lane));  // heads past this lane
    const int next = above ? __ffs((int)above) - 1 : 32 - __clz((int)vmask);
    base = atomicAdd(&counts[key], (uint32_t)(next - (int)lane));
  }
  base = __shfl_sync(0xFFFFFFFFu, base, lead < 0 ? 0 : lead);
  return base + (lane - (uint32_t)lead);
}

// two particles per thread, half a tile apart: both sets of loads are in flight
// before either key is needed (the kernel is bound by memory latency)
// ABS: the plan has a simulation with absorbing walls (their absorbed particles take
// the key after every cell)
template <bool ABS>
__global__ void __launch_bounds__(kTile / 2) k_count(Batch B) {
  // the scan that follows hands out its tiles from 0 and starts a new epoch
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    B.scan_ctl[0] = 0u;
    B.scan_ctl[1] += 1u;
  }
  int k = find_sim(B.ptile, B.nsims, blockIdx.x);
  SimDev& s = *B.sims[k];
  if (!sim_active(s)) return;
  const Grid& g = s.d.grid;
  const uint32_t p0 = (blockIdx.x - B.ptile[k]) * kTile + threadIdx.x;
  const uint32_t pp[2] = {p0, p0 + kTile / 2};
  const int par = s.d.parity;
  double xs[2][3];
  uint32_t vb[2];
  bool valid[2], gone[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    valid[h] = pp[h] < s.n;
    const uint32_t q = valid[h] ? pp[h] : 0u;
#pragma unroll
    for (int a = 0; a < 3; ++a) xs[h][a] = s.x[par][a][q];
    vb[h] = g.split ? (uint32_t)s.vbucket[q] : 0u;
    gone[h] = ABS && s.absorb && s.last[par][q] == KMC_ABSORBED;
  }
  const uint32_t lane = threadIdx.x & 31u;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    uint32_t key = 0;
    if (valid[h] && gone[h]) {
      key = graveyard_key(g);  // left through an absorbing wall: after every cell
    } else if (valid[h]) {
      const int cx = cell_coord(g, 0, xs[h][0]);
      const int cy = cell_coord(g, 1, xs[h][1]);
      const int cz = cell_coord(g, 2, xs[h][2]);
      key = col_code(g, (uint32_t)cy, (uint32_t)cz) * (uint32_t)g.nc[0] + (uint32_t)cx;
      // fast particles (speed bound above the split threshold) form the second population
      // (the trial thresholds decrease with their index, so |v|^2 > threshold[split_t]
      // exactly when the bound exceeds at least 7 - split_t of the six trial values)
      if (g.split && (int)vb[h] >= kSplitTrials - g.split_t) key += g.nkeys;
    }
    const uint32_t rank = run_rank(s.cell_count, key, valid[h], lane);
    if (valid[h]) {
      s.key[pp[h]] = key;
      s.rank[pp[h]] = rank;
    }
  }
}

// --------------------------------------------------------------------------- //
// Segmented exclusive scan of the cell counts -> cell_start (the counts are cleared
// for the next step).  Element `len` is a virtual zero, so out[len] receives the total.
struct ScanView {
  const uint32_t* in;
  uint32_t* out;
  uint32_t* clear;
  uint32_t len;
};

__device__ __forceinline__ ScanView scan_view(SimDev& s) {
  ScanView v;
  v.in = s.cell_count; v.out = s.cell_start; v.clear = s.cell_count;
  v.len = graveyard_key(s.d.grid) + (s.absorb ? 1u : 0u);
  return v;
}

// Single-pass segmented scan with decoupled look-back (Merrill and Garland, "Single-
// pass Parallel Prefix Scan with Decoupled Look-back", NVIDIA technical report, 2016).
// Tiles are handed out in launch order by an atomic counter, so every tile a block
// waits for belongs to a block that is already running.  Each tile publishes its own
// sum at once, then its inclusive prefix once it knows it; a tile's exclusive prefix
// is the sum of its predecessors' published values back to the first inclusive prefix
// (or to the start of its simulation's segment, which starts at zero).  Status words
// carry the epoch of the scan, so the words of the previous step read as not ready.
// The wait for a predecessor is bounded: if it runs out the simulation gets the
// ST_SCAN_WAIT status (sim_sync reports KMC_ETIMEOUT) instead of the block spinning on.
constexpr unsigned long long kStAgg = 1ull, kStIncl = 2ull;
constexpr int kScanWaitLimit = 1 << 20;  // spins of at least 0.1 us: about a second

__device__ __forceinline__ unsigned long long scan_word(uint32_t epoch, unsigned long long state,
                                                        uint32_t value) {
  return ((unsigned long long)epoch << 34) | (state << 32) | (unsigned long long)value;
}

__global__ void __launch_bounds__(kTile) k_scan_onepass(Batch B, uint32_t ntiles) {
  __shared__ uint32_t s_tile, s_excl;
  if (threadIdx.x == 0) s_tile = atomicAdd(&B.scan_ctl[0], 1u);
  __syncthreads();
  const uint32_t tile = s_tile;
  if (tile >= ntiles) return;
  const uint32_t* pre = B.stile_c;
  const int k = find_sim(pre, B.nsims, tile);
  SimDev& s = *B.sims[k];
  // a tile that waited too long sets the status word while the scan runs: the block
  // takes one answer (every thread reaches the barriers below or none does)
  if (!__syncthreads_and(sim_active(s))) return;
  const ScanView v = scan_view(s);
  const uint32_t first = pre[k];
  const uint32_t base = (tile - first) * kScanTile;
  if (base > v.len) return;  // past the key space: no later tile of this segment waits
  const uint32_t epoch = *(volatile uint32_t*)&B.scan_ctl[1] & 0x3FFFFFFFu;
  volatile unsigned long long* status = B.tile_status;
  // The tile in the warps' layout: warp w holds keys [512 w, 512 w + 512) of the tile
  // and lane l the four 16-byte groups 512 w + 128 q + 4 l (q = 0..3), so every load
  // and store instruction of a warp covers 512 contiguous bytes.  Groups that reach
  // past the key space are read and written element by element.
  constexpr int kGroups = kScanTile / kTile / 4;
  constexpr uint32_t kWarpKeys = kScanTile / (kTile / 32);
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const uint32_t eb = base + warp * kWarpKeys + lane * 4u;  // this lane's group q = 0
  uint4 val[kGroups];
  uint32_t gsum[kGroups], goff[kGroups];
#pragma unroll
  for (int q = 0; q < kGroups; ++q) {
    const uint32_t e = eb + 128u * q;
    if (e + 3u < v.len) {
      val[q] = *reinterpret_cast<const uint4*>(v.in + e);
    } else {
      val[q].x = e < v.len ? v.in[e] : 0u;
      val[q].y = e + 1u < v.len ? v.in[e + 1u] : 0u;
      val[q].z = e + 2u < v.len ? v.in[e + 2u] : 0u;
      val[q].w = 0u;
    }
    gsum[q] = val[q].x + val[q].y + val[q].z + val[q].w;
  }
  // exclusive prefix of each group within the warp, groups in (q, lane) order
  uint32_t wrun = 0;
#pragma unroll
  for (int q = 0; q < kGroups; ++q) {
    uint32_t incl = gsum[q];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
      if (lane >= (uint32_t)o) incl += y;
    }
    goff[q] = wrun + incl - gsum[q];
    wrun += __shfl_sync(0xFFFFFFFFu, incl, 31);
  }
  // the warps' totals -> each warp's offset in the tile, and the tile's sum
  __shared__ uint32_t s_w[kTile / 32 + 1];
  if (lane == 0) s_w[warp] = wrun;
  __syncthreads();
  if (warp == 0) {
    const uint32_t w = lane < kTile / 32 ? s_w[lane] : 0u;
    uint32_t wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, wi, o);
      if (lane >= (uint32_t)o) wi += y;
    }
    if (lane < kTile / 32) s_w[lane] = wi - w;
    if (lane == kTile / 32 - 1) s_w[kTile / 32] = wi;
  }
  __syncthreads();
  const uint32_t woff = s_w[warp];
  const uint32_t agg = s_w[kTile / 32];
  // publish the tile's sum, then look back with the whole block, kTile predecessors
  // per read (all tiles start at about the same time, so the nearest inclusive prefix
  // can be far back: a tile reads about t / kTile windows)
  __shared__ uint32_t s_stop, s_val[kTile / 32];
  __shared__ int s_done;
  if (tile == first) {
    if (threadIdx.x == 0) {
      status[tile] = scan_word(epoch, kStIncl, agg);
      s_excl = 0;
    }
  } else {
    if (threadIdx.x == 0) status[tile] = scan_word(epoch, kStAgg, agg);
    // the failure-path test waits for an epoch that no tile writes
    const uint32_t want = s.scan_wait_test ? ((epoch + 1u) & 0x3FFFFFFFu) : epoch;
    uint32_t excl = 0;
    bool timed_out = false;
    long long top = (long long)tile - 1;  // thread t reads tile top - t
    for (;;) {
      const long long p = top - (long long)threadIdx.x;
      const bool in_seg = p >= (long long)first;
      unsigned long long w = 0ull;
      int spins = 0;
      for (;;) {
        w = in_seg ? status[p] : 0ull;
        const bool ready = !in_seg || ((uint32_t)(w >> 34) == want && ((w >> 32) & 3ull) != 0ull);
        if (__syncthreads_and(ready)) break;
        if (++spins > kScanWaitLimit) { timed_out = true; break; }
        if (spins > 16) __nanosleep(100);
      }
      if (timed_out) break;
      // the nearest inclusive prefix (lowest thread index) ends the look-back; the
      // segment's first tile always publishes one, so some window finds it
      if (threadIdx.x == 0) s_stop = 0xFFFFFFFFu;
      __syncthreads();
      const bool incl = in_seg && ((w >> 32) & 3ull) == kStIncl;
      if (incl) atomicMin(&s_stop, threadIdx.x);
      __syncthreads();
      const uint32_t stop = s_stop;
      uint32_t val = (in_seg && threadIdx.x <= stop) ? (uint32_t)w : 0u;
      for (int o = 16; o > 0; o >>= 1) val += __shfl_xor_sync(0xFFFFFFFFu, val, o);
      if (lane == 0) s_val[warp] = val;
      __syncthreads();
      if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int i = 0; i < kTile / 32; ++i) t += s_val[i];
        excl += t;
        s_done = (stop != 0xFFFFFFFFu || top - (kTile - 1) <= (long long)first) ? 1 : 0;
      }
      __syncthreads();
      if (s_done) break;
      top -= kTile;
    }
    if (threadIdx.x == 0) {
      if (timed_out) atomicOr(&s.d.status, ST_SCAN_WAIT);
      status[tile] = scan_word(epoch, kStIncl, excl + agg);
      s_excl = excl;
    }
  }
  __syncthreads();
  const uint32_t tb = s_excl + woff;
#pragma unroll
  for (int q = 0; q < kGroups; ++q) {
    const uint32_t e = eb + 128u * q;
    uint4 st;
    st.x = tb + goff[q];
    st.y = st.x + val[q].x;
    st.z = st.y + val[q].y;
    st.w = st.z + val[q].z;
    // element len (a virtual zero) receives the total
    if (e + 3u <= v.len) {
      *reinterpret_cast<uint4*>(v.out + e) = st;
    } else {
      if (e <= v.len) v.out[e] = st.x;
      if (e + 1u <= v.len) v.out[e + 1u] = st.y;
      if (e + 2u <= v.len) v.out[e + 2u] = st.z;
    }
    if (v.clear && gsum[q]) {  // the counts are cleared for the next step
      if (e + 3u < v.len) {
        *reinterpret_cast<uint4*>(v.clear + e) = make_uint4(0u, 0u, 0u, 0u);
      } else {
        if (e < v.len) v.clear[e] = 0u;
        if (e + 1u < v.len) v.clear[e + 1u] = 0u;
        if (e + 2u < v.len) v.clear[e + 2u] = 0u;
      }
    }
  }
}

// --------------------------------------------------------------------------- //
// The permutation is applied as a gather: k_scatter only records, for every
// position of the new cell order, which particle goes there (4 bytes, scattered over
// nearby positions -- particles move less than a cell per step); k_gather then walks
// the new order, reads each particle from its old position (nearby reads share
// sectors) and writes the permuted state, the mirror and the per-particle step
// arrays with coalesced stores.
// Both kernels take two particles per thread, half a tile apart, so that both
// dependent load chains (key -> cell start; source -> state) are in flight at once.
__global__ void __launch_bounds__(kTile / 2) k_scatter(Batch B) {
  int k = find_sim(B.ptile, B.nsims, blockIdx.x);
  SimDev& s = *B.sims[k];
  if (!sim_active(s)) return;
  const uint32_t p0 = (blockIdx.x - B.ptile[k]) * kTile + threadIdx.x;
  const uint32_t pp[2] = {p0, p0 + kTile / 2};
  uint32_t key[2], rank[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const uint32_t q = pp[h] < s.n ? pp[h] : 0u;
    key[h] = s.key[q];
    rank[h] = s.rank[q];
  }
  uint32_t dst[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) dst[h] = s.cell_start[key[h]] + rank[h];
#pragma unroll
  for (int h = 0; h < 2; ++h)
    if (pp[h] < s.n) s.src[dst[h]] = pp[h];
}

__global__ void __launch_bounds__(kTile / 2) k_gather(Batch B) {
  int k = find_sim(B.ptile, B.nsims, blockIdx.x);
  SimDev& s = *B.sims[k];
  if (!sim_active(s)) return;
  const uint32_t d0 = (blockIdx.x - B.ptile[k]) * kTile + threadIdx.x;
  const uint32_t dd[2] = {d0, d0 + kTile / 2};
  const int from = s.d.parity, to = from ^ 1;
  uint32_t pp[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) pp[h] = s.src[dd[h] < s.n ? dd[h] : 0u];
  double xs[2][3], vs[2][3];
  uint32_t id[2], last[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      xs[h][a] = s.x[from][a][pp[h]];
      vs[h][a] = s.v[from][a][pp[h]];
    }
    id[h] = s.id[from][pp[h]];
    last[h] = s.last[from][pp[h]];
  }
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const uint32_t d = dd[h];
    if (d >= s.n) continue;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      s.x[to][a][d] = xs[h][a];
      s.v[to][a][d] = vs[h][a];
    }
    s.id[to][d] = id[h];
    s.last[to][d] = last[h];
    s.deg[d] = 0;
    s.partner[d] = kNone;
    if (s.precision == KMC_GUARDED_FP32) {
      // box coordinates and velocity, each rounded once to binary32
      mirror_store(s.mir, d, d2f_rn(xs[h][0]), d2f_rn(xs[h][1]), d2f_rn(xs[h][2]),
                   d2f_rn(vs[h][0]), d2f_rn(vs[h][1]), d2f_rn(vs[h][2]));
    }
  }
}

// --------------------------------------------------------------------------- //
int launch_cell_scan(const LaunchPlan& L, cudaStream_t st) {
  const uint32_t nt = L.stiles_c;
  k_scan_onepass<<<nt, kTile, 0, st>>>(L.b, nt);
  return 1;
}

int launch_sort(const LaunchPlan& L, cudaStream_t st) {
  if (L.absorb) k_count<true><<<L.ptiles, kTile / 2, 0, st>>>(L.b);
  else k_count<false><<<L.ptiles, kTile / 2, 0, st>>>(L.b);
  int n = launch_cell_scan(L, st);
  k_scatter<<<L.ptiles, kTile / 2, 0, st>>>(L.b);
  k_gather<<<L.ptiles, kTile / 2, 0, st>>>(L.b);
  return n + 3;
}

}  // namespace kmc
