// kmc_internal.cuh -- device data layout and helpers shared by the libkmc kernels.
//
// Every kernel is written for a *batch* of simulations: it receives a device table
// of SimDev pointers and a prefix array that maps its tiles (blocks) onto the
// simulations.  A lone simulation is a batch of one.  Per-step quantities that the
// host never needs (cell grid, counters, step index) live in device memory, so the
// launch sequence of a step is fixed and can be captured once in a CUDA graph.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kmc.h"

namespace kmc {

constexpr int kTile = 256;          // particles per block in particle kernels
constexpr int kScanTile = 8192;     // keys per tile of the cell scan
constexpr int kProfTile = 8192;     // particles per block in the profile kernel
constexpr int kEdgeBlock = 256;     // threads per block in edge / adjacency kernels
constexpr int kSearchBuf = 512;     // per-block shared-memory staging of emitted pairs
constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr int kProfQ = 20;          // int64 counters per profile bin (see profile_add below)
constexpr int kMaxGroup = 4096;     // simulations per batch
constexpr int kSplitTrials = 7;     // trial thresholds of the speed split (index 0: none)

// trial thresholds of the speed split as fractions of vmax (index 0: no split)
__device__ __forceinline__ float split_frac(int t) {
  return t == 0 ? 1.0f : t == 1 ? 0.85f : t == 2 ? 0.72f : t == 3 ? 0.6f : t == 4 ? 0.5f
                 : t == 5 ? 0.42f : 0.35f;
}

enum : uint32_t {
  ST_EDGE_OVERFLOW = 1u << 0,  // candidate-pair buffer too small (host grows it)
  ST_RANDOM = 1u << 1,         // 128 rejected sphere-point draws
  ST_CELL_OVERFLOW = 1u << 2,  // grid key space above capacity (cannot happen: coarsened)
  ST_SCAN_WAIT = 1u << 3,      // a scan tile waited too long for its predecessor's sum
};

// Search grid of the current step.  Cells are keyed column-major along x inside a
// tiled Z-order (Morton) walk over the (y, z) columns: key = col(cy, cz) * nc[0] + cx.
struct Grid {
  int32_t nc[3];      // cells per axis; 1 means the axis is one cell (no stencil on it)
  int32_t K;          // stencil radius in cells
  int32_t mode;       // search kernel of this step: KMC_SEARCH_PARTICLE, _CELL or _ROW
  int32_t split_t;    // trial threshold index of the split (0: no split)
  uint32_t split;     // 1: particles with |v|^2 above s1sq form a second population
  float s1sq;         // binary32 split threshold on the upper bound of |v|^2
  int32_t cfast[3];   // fast particles search cfast cells on each side (split axes)
  uint32_t nkeys;     // size of the key space (padded Morton columns x nc[0])
  uint32_t col_shift; // log2 of the Morton tile edge T (T <= 8)
  uint32_t col_tz;    // tiles along z
  int32_t kx;         // cells per stencil radius along x (K, or 2K under the row search)
  double w[3];        // cell widths
  float wf[3];        // cell widths (binary32)
  float inv_wf[3];    // cells per unit length (binary32, cell assignment)
  // guarded binary32 pre-tests (kmc_search.cu derives them; kmc_push.cu sets them)
  float s_c0, s_c1;   // sphere test: drop if R > s_c0 + s_c1 * B
  float a_g;          // approach test: drop if A < -a_g
  float t_g, dtf;     // time test: drop if A - dtf * B > t_g
  float d0up, b_rel, b_abs, w_e, w_rel;  // distance test (see kmc_search.cu)
  float Lf[3], halfLf[3], tief[3];        // one-cell periodic axes: minimum image
  // row trimming of the binary32 row search: slow-slow candidates lie within the reach
  // d0 + 2 S1 dt; r2 bounds its square, eps the binary32 error of a distance from a
  // cell edge, pad the error of a coordinate (all rounded up).  Per particle i the
  // reach is d0 + (|v_i| + S1) dt: at most row_a + row_b |v_i| (both rounded up); for a
  // fast particle i (partners up to the bound V of max |v|) at most fast_a + row_b |v_i|
  float row_r2, row_eps, row_pad, row_a, row_b, fast_a;
  // binary64 sphere pre-test: drop if R > c0 + c1 * B (B >= 2^-900)
  double c0, c1;
};

struct Dyn {
  uint64_t step;        // absolute index of the next step
  uint64_t steps_left;  // step budget; kernels skip the simulation when 0
  uint32_t parity;      // state buffer holding the state at the start of the step
  uint32_t status;      // ST_* bits; kernels skip the simulation when non-zero
  uint32_t vmax2_acc;   // binary32 bits of an upper bound of max |v|^2 (atomicMax)
  float vmax2;          // bound the current grid was built from
  Grid grid;
  uint32_t n_raw;       // pairs emitted by the search (may exceed edge_cap)
  uint32_t n_edges;     // candidate pairs after the exact test
  uint32_t round_pairs[4];
  uint32_t n_pairs;     // entries of the pair list
  uint32_t adj_used;    // candidate-list entries handed out this step
  uint32_t wl_len[5];   // particles on the work list of matching round r (0: all with
                        // candidates; r + 1 is filled by round r)
  unsigned long long pair_tests;
  unsigned long long fast_tests;  // the part of pair_tests done by the fast-particle search
  uint32_t last_raw;    // n_raw of the last completed step (its pair buffer is kept)
  uint32_t have_counts; // split_cnt holds counts of the current state
  float split_thr[kSplitTrials];     // trial thresholds on |v|^2 (set with the grid)
  uint32_t split_cnt[kSplitTrials];  // particles above each trial threshold
  uint32_t prof_due;    // the step being run ends with a profile
  uint32_t prof_count;  // snapshots written
  uint64_t hist_count;  // step records written
  uint32_t n_absorbed;  // particles that left through absorbing walls this step
};

struct SimDev {
  // ---- parameters ----
  uint32_t n;
  int32_t bc[3];
  int32_t max_rounds, precision, profile_bins, profile_every, K, search_kernel;
  int32_t split_ok;     // 0: never split, 1: split when cheaper, 2: split whenever possible
  int32_t planar;       // 1: x-y dynamics (vz = 0), scatter directions in the plane
  double split_min_occ; // smallest mean occupancy of the slow grid under a split
  double box[3];
  double piston_x0, piston_u, d0, dt, d0sq;
  double profile_range, cell_scale;
  uint64_t seed;
  uint32_t cell_cap, edge_cap, hist_cap, prof_cap;
  // ---- state, double-buffered by the sort ----
  double* x[2][3];
  double* v[2][3];
  uint32_t* id[2];
  uint32_t* last[2];
  // ---- per-step work arrays ----
  float4* mir;          // binary32 mirror in pair records (mirror_load / mirror_store)
  void* mir_spare;      // unused: keeps the offsets of the fields below
  uint32_t* key;        // cell key per particle (pre-sort order)
  uint32_t* rank;       // rank inside the cell (pre-sort order)
  uint8_t* vbucket;     // per particle: how many of the trial split thresholds its
                        // |v|^2 bound exceeds (written by the push, read by the count)
  uint32_t* src;        // pre-sort position of the particle at each sorted position
  uint32_t* cell_count; // nkeys counters, all zero between steps
  uint32_t* cell_start; // nkeys + 1
  uint32_t* deg;        // candidate pairs per particle
  uint32_t* off;        // start of each particle's candidate list in adj (set for deg > 0)
  uint2* edge;          // emitted pairs (sorted indices, owner first)
  double* e_d2;         // binary64 key of each pair
  double* e_t;
  uint2* e_slot;        // slot of the pair in each endpoint's list, x = kNone if rejected
  uint2* adj;           // candidate lists, each particle's contiguous: (other end, pair)
  uint32_t* wl[2];      // work lists of the matching rounds (unmatched particles that
                        // still had an unmatched candidate), used alternately
  uint32_t* best;       // best unmatched candidate (sorted index) in the current round
  uint32_t* best_e;
  uint32_t* partner;    // partner (sorted index) this step, kNone if none
  uint32_t* medge;      // pair index of the collision
  uint32_t* pairs;      // colliding pairs of the step, by their smaller-id member
  kmc_step_counts* hist;
  long long* prof_acc;  // prof_cap x bins x kProfQ fixed-point counters
  uint64_t* prof_step;
  Dyn d;
  // ---- variants (after the fields every step reads, which keep their offsets) ----
  int32_t absorb;       // 1: some axis has absorbing walls (the sort keeps the particles
                        // that left in one extra key after every cell: see graveyard_key)
  int32_t mix;          // 1: a mixture (per-particle species: mass and effective radius)
  int32_t mix_n;        // number of species
  // mixture: species by particle id, mass and radius by species
  uint8_t* species;
  double* sp_mass;
  double* sp_radius;
  int32_t scan_wait_test;  // KMC_FLAG_SCAN_WAIT_TEST: the scan waits for a word never written
};

// ---- batch mapping ------------------------------------------------------- //
struct Batch {
  SimDev* const* sims;     // device table
  int nsims;
  const uint32_t* ptile;   // prefix of ceil(n / kTile) per simulation
  const uint32_t* stile_c; // prefix of ceil((cell_cap + 2) / kScanTile)
  const uint32_t* prtile;  // prefix of ceil(n / kProfTile)
  // single-pass segmented scan: per tile a status word (epoch << 34 | state << 32 |
  // value), and the control words [0] next tile to hand out, [1] current epoch
  unsigned long long* tile_status;
  uint32_t* scan_ctl;
};

__device__ __forceinline__ int find_sim(const uint32_t* prefix, int nsims, uint32_t tile) {
  int lo = 0, hi = nsims;  // prefix[lo] <= tile < prefix[hi]
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (__ldg(prefix + mid) <= tile) lo = mid; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ bool sim_active(const SimDev& s) {
  return s.d.status == 0 && s.d.steps_left > 0;
}

// A member that runs this step.  Unlike the status word, which the searches, the scan
// and the collision set while they run, steps_left changes only between kernels (the
// step's last one counts it down), so every thread and block of a launch reads the
// same value.  Control flow that reaches a barrier, or that blocks must agree on
// (dealing a batch's items), decides on this and the launch-fixed grid fields; the
// status word only gates the work, read once per block or per warp.
__device__ __forceinline__ bool sim_scheduled(const SimDev& s) { return s.d.steps_left > 0; }

// Absorbing walls: the particles that have left sort into one extra key after every
// cell key (and after the fast population's keys), so that they occupy the end of the
// sorted order, [live, n), and no cell holds them.
__device__ __forceinline__ uint32_t graveyard_key(const Grid& g) {
  return g.nkeys * (g.split ? 2u : 1u);
}
// particles in the gas at the start of the step (after this step's sort); without
// absorbing walls the scan's total at that key is n
__device__ __forceinline__ uint32_t live_count(const SimDev& s) {
  return __ldg(s.cell_start + graveyard_key(s.d.grid));
}

// ---- exact binary64 arithmetic (never contracted into FMA) --------------- //
__device__ __forceinline__ double dadd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double dsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double dmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double ddiv(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ double dsqrt(double a) { return __dsqrt_rn(a); }

// ---- fixed-point profile counters ----------------------------------------- //
// A profile bin keeps kProfQ int64 counters: [0] the particle count, [1 + 3a + c]
// digit c of sum v_a, [10 + 3a + c] digit c of sum v_a^2, [19] the terms that were
// out of range.  A term q is |q| 2^64 truncated, split into three 32-bit digits with
// the sign of q; the digits are summed exactly in int64 (below 2^31 terms per bin),
// so the sums do not depend on the order of the atomic additions.  A term with
// |q| >= 2^31 (|v_a| >= 46341 for the squares) does not fit the three digits: it is
// counted in [19] instead, and the bin's six velocity sums convert to NaN.
__device__ __forceinline__ bool fx_digits(double q, long long d[3]) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(q);
  const bool neg = (bits >> 63) != 0;
  const int ex = (int)((bits >> 52) & 0x7FF);
  d[0] = d[1] = d[2] = 0;
  if (ex == 0) return true;      // zero or subnormal: below 2^-64
  const int sh = ex - 1075 + 64; // |q| 2^64 = man 2^sh
  if (sh > 42) return false;     // |q| >= 2^31, infinity or NaN
  const unsigned long long man = (bits & ((1ull << 52) - 1)) | (1ull << 52);
  unsigned __int128 f;
  if (sh >= 0) f = (unsigned __int128)man << sh;
  else if (sh > -64) f = (unsigned __int128)(man >> (-sh));
  else f = 0;
  long long d0 = (long long)(uint32_t)f, d1 = (long long)(uint32_t)(f >> 32),
            d2 = (long long)(uint32_t)(f >> 64);
  if (neg) { d0 = -d0; d1 = -d1; d2 = -d2; }
  d[0] = d0; d[1] = d1; d[2] = d2;
  return true;
}

// add one particle (velocity v) to the counters q of its bin (shared or global memory)
__device__ __forceinline__ void profile_add(long long* q, const double v[3]) {
  atomicAdd((unsigned long long*)&q[0], 1ull);
  unsigned long long bad = 0;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    long long d[3];
    if (fx_digits(v[a], d)) {
      for (int c = 0; c < 3; ++c) atomicAdd((unsigned long long*)&q[1 + 3 * a + c], (unsigned long long)d[c]);
    } else {
      ++bad;
    }
    if (fx_digits(__dmul_rn(v[a], v[a]), d)) {
      for (int c = 0; c < 3; ++c) atomicAdd((unsigned long long*)&q[10 + 3 * a + c], (unsigned long long)d[c]);
    } else {
      ++bad;
    }
  }
  if (bad) atomicAdd((unsigned long long*)&q[19], bad);
}

// value k (0: count, 1..3: sum v_a, 4..6: sum v_a^2) of a bin's counters, in binary64:
// (d2 2^64 + d1 2^32 + d0) 2^-64 from a signed 128-bit total, rounded once; NaN for a
// velocity sum of a bin with out-of-range terms
__device__ __forceinline__ double profile_value(const long long* src, int k) {
  if (k == 0) return (double)src[0];
  if (src[19] != 0) return __longlong_as_double(0x7FF8000000000000ll);
  const long long* dg = src + 1 + 3 * (k - 1);
  const __int128 tot = ((__int128)dg[2] << 64) + ((__int128)dg[1] << 32) + (__int128)dg[0];
  const bool neg = tot < 0;
  const unsigned __int128 mag = neg ? (unsigned __int128)(-tot) : (unsigned __int128)tot;
  const double hi = (double)(unsigned long long)(mag >> 64);
  const double lo = (double)(unsigned long long)mag;
  const double val = __dadd_rn(__dmul_rn(hi, 1.0), __dmul_rn(lo, 0x1p-64));
  return neg ? -val : val;
}

// Block-aggregated append: one atomic per block on the shared counter (a counter that
// every warp of the grid hits is a hot spot: its atomics serialise in L2).  Every
// thread of the block must call it; *also, if given, is advanced by the same total.
// Returns this thread's first index in the buffer behind *counter.
__device__ __forceinline__ uint32_t block_append(uint32_t* counter, uint32_t want,
                                                 uint32_t* also = nullptr) {
  constexpr int kW = kEdgeBlock / 32;  // blocks of kEdgeBlock threads
  __shared__ uint32_t wsum[kW], wbase[kW], bbase;
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  uint32_t incl = want;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
    if (lane >= (uint32_t)o) incl += y;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const uint32_t v = lane < (uint32_t)kW ? wsum[lane] : 0u;
    uint32_t vi = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, vi, o);
      if (lane >= (uint32_t)o) vi += y;
    }
    if (lane < (uint32_t)kW) wbase[lane] = vi - v;
    if (lane == (uint32_t)kW - 1) {
      bbase = vi ? atomicAdd(counter, vi) : 0u;
      if (also && vi) atomicAdd(also, vi);
    }
  }
  __syncthreads();
  const uint32_t r = bbase + wbase[warp] + incl - want;
  __syncthreads();  // the slots are free for the next call
  return r;
}

// ---- guarded-binary32 mirror ------------------------------------------------ //
// Box coordinates and velocity of every particle (sorted order), each rounded once to
// binary32, in pair records: particles 2k and 2k + 1 share three float4,
//   (x0, x1, y0, y1), (z0, z1, vx0, vx1), (vy0, vy1, vz0, vz1),
// so that a 16-byte load gives one component of two consecutive partners already
// paired for the packed f32x2 arithmetic of the row search.
__device__ __forceinline__ void mirror_load(const float4* __restrict__ M, uint32_t j, float4& a,
                                            float2& b) {
  const float* r = reinterpret_cast<const float*>(M + 3 * (size_t)(j >> 1)) + (j & 1u);
  a = make_float4(__ldg(r), __ldg(r + 2), __ldg(r + 4), __ldg(r + 6));
  b = make_float2(__ldg(r + 8), __ldg(r + 10));
}
__device__ __forceinline__ void mirror_store(float4* M, uint32_t j, float x, float y, float z,
                                             float vx, float vy, float vz) {
  float* r = reinterpret_cast<float*>(M + 3 * (size_t)(j >> 1)) + (j & 1u);
  r[0] = x;
  r[2] = y;
  r[4] = z;
  r[6] = vx;
  r[8] = vy;
  r[10] = vz;
}

// ---- Morton column code --------------------------------------------------- //
__device__ __forceinline__ uint32_t dilate16(uint32_t x) {
  x &= 0xFFFFu;
  x = (x | (x << 8)) & 0x00FF00FFu;
  x = (x | (x << 4)) & 0x0F0F0F0Fu;
  x = (x | (x << 2)) & 0x33333333u;
  x = (x | (x << 1)) & 0x55555555u;
  return x;
}
__device__ __forceinline__ uint32_t compact16(uint32_t x) {
  x &= 0x55555555u;
  x = (x | (x >> 1)) & 0x33333333u;
  x = (x | (x >> 2)) & 0x0F0F0F0Fu;
  x = (x | (x >> 4)) & 0x00FF00FFu;
  x = (x | (x >> 8)) & 0x0000FFFFu;
  return x;
}
// Column order: the (y, z) plane is cut into T x T tiles (T = 2^col_shift <= 8)
// walked row by row; inside a tile the columns follow the Z-order (Morton) curve.
// Padding is below T per axis.
__device__ __forceinline__ uint32_t col_code(const Grid& g, uint32_t cy, uint32_t cz) {
  const uint32_t t = g.col_shift, mask = (1u << t) - 1u;
  const uint32_t tile = (cy >> t) * g.col_tz + (cz >> t);
  return (tile << (2 * t)) | dilate16(cy & mask) | (dilate16(cz & mask) << 1);
}
__device__ __forceinline__ void key_decode(const Grid& g, uint32_t key, int& cx, int& cy, int& cz) {
  const uint32_t nx = (uint32_t)g.nc[0];
  const uint32_t col = key / nx;
  cx = (int)(key - col * nx);
  const uint32_t t = g.col_shift;
  const uint32_t tile = col >> (2 * t);
  const uint32_t in = col & ((1u << (2 * t)) - 1u);
  const uint32_t by = tile / g.col_tz, bz = tile - by * g.col_tz;
  cy = (int)((by << t) | compact16(in));
  cz = (int)((bz << t) | compact16(in >> 1));
}

// binary64 -> binary32 conversions on the integer pipes (on this part the hardware
// conversion issues on the binary64 pipe, which runs at 1/72 of the binary32 rate).
// IEEE 754 round to nearest even, with no hardware fallback: a fallback branch that
// the compiler turns into a predicated conversion would still occupy the binary64
// pipe.  Normal results round the 29 dropped bits; results below the binary32 normal
// range are k 2^-149 with k = M 2^(e-926) rounded (M the 53-bit significand);
// overflow gives infinity and NaN a quiet NaN.
__device__ __forceinline__ float d2f_rn(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const uint32_t sign = (uint32_t)(b >> 63) << 31;
  const int e = (int)((b >> 52) & 0x7FF);
  const int fe = e - 1023 + 127;
  if (fe >= 1 && fe <= 254) {
    const uint32_t top = (uint32_t)((b >> 29) & 0x7FFFFFu);
    const uint32_t rest = (uint32_t)(b & 0x1FFFFFFFu);
    const uint32_t up = (rest > 0x10000000u || (rest == 0x10000000u && (top & 1u))) ? 1u : 0u;
    return __uint_as_float(sign | (((uint32_t)fe << 23) + top + up));  // carry may reach inf
  }
  if (fe > 254) {
    const bool nan = e == 0x7FF && (b & 0xFFFFFFFFFFFFFull) != 0ull;
    return __uint_as_float(nan ? 0x7FFFFFFFu : (sign | 0x7F800000u));
  }
  const int sh = 926 - e;  // >= 30 here
  if (e == 0 || sh > 54) return __uint_as_float(sign);  // below half the least subnormal
  const unsigned long long M = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  unsigned long long k = M >> sh;
  const unsigned long long rem = M & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
  k += (rem > half || (rem == half && (k & 1ull))) ? 1ull : 0ull;
  return __uint_as_float(sign | (uint32_t)k);
}
// |x| rounded up to binary32 (integer pipes, no hardware fallback)
__device__ __forceinline__ float d2f_abs_ru(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
  const int e = (int)(b >> 52);
  const int fe = e - 1023 + 127;
  if (fe >= 1 && fe <= 254) {
    const uint32_t top = (uint32_t)((b >> 29) & 0x7FFFFFu);
    const uint32_t up = (b & 0x1FFFFFFFull) ? 1u : 0u;
    return __uint_as_float(((uint32_t)fe << 23) + top + up);
  }
  if (fe > 254) return __uint_as_float(e == 0x7FF && (b & 0xFFFFFFFFFFFFFull) ? 0x7FFFFFFFu : 0x7F800000u);
  if (b == 0ull) return 0.0f;
  const int sh = 926 - e;
  if (e == 0 || sh > 63) return __uint_as_float(1u);  // the least subnormal
  const unsigned long long M = (b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
  const unsigned long long k = (M >> sh) + ((M & ((1ull << sh) - 1ull)) ? 1ull : 0ull);
  return __uint_as_float((uint32_t)k);
}

// upper bound of |v|^2 in binary32 (directed rounding; used to size cells and to
// split fast from slow particles, never in a result)
__device__ __forceinline__ float vmag2_up(double vx, double vy, double vz) {
  float ax = d2f_abs_ru(vx), ay = d2f_abs_ru(vy), az = d2f_abs_ru(vz);
  return __fadd_ru(__fadd_ru(__fmul_ru(ax, ax), __fmul_ru(ay, ay)), __fmul_ru(az, az));
}

// cell coordinate along one axis, binary32 (only the speed depends on it); from the
// binary32 coordinate (the mirror's) it is the same cell as from the binary64 one
__device__ __forceinline__ int cell_coord_f(const Grid& g, int k, float xf) {
  if (g.nc[k] == 1) return 0;
  float f = floorf(xf * g.inv_wf[k]);
  int c = (int)f;
  c = c < 0 ? 0 : c;
  c = c >= g.nc[k] ? g.nc[k] - 1 : c;
  return c;
}
__device__ __forceinline__ int cell_coord(const Grid& g, int k, double x) {
  return cell_coord_f(g, k, d2f_rn(x));
}

// ---- domain decomposition (kmc_domain.cu) ---------------------------------- //
constexpr int kMaxDomains = 64;
constexpr uint32_t kElsewhere = 0xFFFFFFFDu;  // partner of a ghost matched to a particle
                                              // that its domain does not hold

struct DomainDev {
  uint32_t n;                   // particles (global ids 0..n-1)
  int32_t P;                    // domains: x slabs
  int32_t periodic_x;
  double Lx;                    // box length along x
  double X[kMaxDomains + 1];    // domain k owns X[k] <= x < X[k+1] (the last one all above)
  double d0, dt;
  // id-order exchange buffers: the state (52 n bytes: x, y, z, vx, vy, vz, last)
  double* x[3];
  double* v[3];
  uint32_t* last;
  uint8_t* owner;               // domain owning each particle during the current step
  uint32_t* bestG;              // round's best partner (global id) of each owned particle
  uint32_t* partnerG;           // round's match (global id) of each owned particle
  uint32_t* partner_out;        // partner (global id) in the last step, KMC_NONE if none
  uint32_t* loc;                // P x n: position of each id in each domain (kNone: absent)
  unsigned long long vmax2_bits;
  double reach;                 // ghost reach of the step (d0 + 2 v_max dt, widened)
  uint32_t owned[kMaxDomains], ghosts[kMaxDomains];
  uint32_t acc_edges, acc_round[4];
  kmc_step_counts* hist;
  uint32_t hist_cap;
  uint64_t hist_count;
};

// ---- launch helpers (host) ----------------------------------------------- //
struct LaunchPlan {
  Batch b;
  uint32_t ptiles, stiles_c, prtiles;
  int edge_blocks;
  int cell_blocks;  // persistent grid of the warp-per-cell search
  int part_blocks;  // grid-stride grids of the particle, row and fast searches
  int row_blocks;     // row search, no periodic x axis
  int row_blocks_px;  // row search, periodic x axis
  int fast_blocks;
  // some simulation of the plan has absorbing walls / is a mixture: the kernels that
  // handle either are launched in their general form only then
  bool absorb = false;
  bool mix = false;
};

// each returns the number of kernels it launched
int launch_sort(const LaunchPlan& L, cudaStream_t st);
// ev_slow (optional, two events): recorded around the slow-population search kernels
int launch_search(const LaunchPlan& L, int precision, int K, cudaStream_t st,
                  cudaEvent_t* ev_slow = nullptr);
// resident-block grids of the search kernels (and the row search's shared-memory
// attribute); called when a launch plan is built, before any capture
void search_grids(int precision, int K, int num_sms, uint32_t ptiles, LaunchPlan& L);
int launch_match(const LaunchPlan& L, int max_rounds, cudaStream_t st);
// the parts of launch_match around the rounds: exact test and candidate lists; collision
int launch_match_lists(const LaunchPlan& L, cudaStream_t st);
int launch_collide(const LaunchPlan& L, cudaStream_t st);
int launch_push(const LaunchPlan& L, cudaStream_t st);
int launch_init_grid(const LaunchPlan& L, cudaStream_t st);
int launch_cell_scan(const LaunchPlan& L, cudaStream_t st);

// one step of a domain decomposition (the members of L are its domains, in order)
int launch_domain_step(const LaunchPlan& L, DomainDev* D, uint32_t n, int precision, int K,
                       int max_rounds, cudaStream_t st);
void launch_domain_edges(const LaunchPlan& L, DomainDev* D, uint32_t cap, uint2* out,
                         uint32_t* count, cudaStream_t st);
void launch_domain_vmax(const DomainDev* D, unsigned long long* acc, double* out, cudaStream_t st);

// observe helpers
void launch_gather_state(SimDev* d, uint32_t n, void* out, cudaStream_t st);
void launch_gather_partners(SimDev* d, uint32_t n, uint32_t* out, cudaStream_t st);
void launch_gather_edges(SimDev* d, uint32_t cap, uint2* out, uint32_t* count, cudaStream_t st);
void launch_profile_convert(SimDev* d, uint32_t first, uint32_t count, uint32_t bins,
                            double* out, cudaStream_t st);
void launch_add_steps(SimDev* d, uint64_t nsteps, cudaStream_t st);
void launch_validate(SimDev* d, uint32_t n, uint32_t* bad, cudaStream_t st);
// KMC_OBS_VMAX: acc is 8 bytes of device scratch, out one binary64 (device)
void launch_vmax_exact(SimDev* d, unsigned long long* acc, double* out, cudaStream_t st);

// device-side initial state (kmc_init.cu): writes buffer 0 of the state in id order,
// the ids and last = kNone; counts particles whose rejection loops ran out in *fails
struct InitLaunch {
  uint32_t n;
  int32_t kind;
  int32_t planar;
  uint64_t n_hot;
  uint64_t seed;
  double sigma, speed, sigma_hot, radius;
  double center[3];
  double box[3];
  double* x[3];
  double* v[3];
  uint32_t* id;
  uint32_t* last;
  uint32_t* fails;
};
void launch_init_state(const InitLaunch& L, cudaStream_t st);

}  // namespace kmc
