// kmc_grid.cuh -- per-step search grid and the guard bands of the binary32
// pre-tests, computed on the device by one thread per simulation.
//
// Cell size.  A candidate pair has |r| <= d_min + |v| t* < d0 + |v_i - v_j| dt
// <= d0 + (s_i + s_j) dt with s = |v| (Sec. 2: the partner must reach its distance
// of closest approach within the next time step).  With every particle at most S
// fast, cells at least d0 + 2 S dt wide hold each partner in the same or a
// neighbouring cell (Sec. 2: 26 neighbours in 3D).  With stencil K the cell is 1/K of
// that and K cells are searched on each side.  The width gets a relative margin m
// for the binary32 cell assignment, and cell_scale >= 1 only enlarges it.
//
// Speed split.  The fastest particle sets S = vmax, although nearly all particles
// are much slower.  The grid may instead be sized for a threshold S1 < vmax: the
// particles faster than S1 ("fast") are sorted into a second population.  Slow-slow
// pairs are searched on the S1 grid as above; every fast particle searches c cells
// on each side, c = ceil((d0 + 2 vmax dt) / w), over both populations (fast-fast
// pairs once, by the lower index).  Each candidate pair is still tested exactly
// once.  S1 is chosen per step from the number of particles above a few trial
// thresholds (counted by the push of the previous step) with a cost estimate.
// None of this can change a result, only the amount of work.  An axis with fewer
// than 2K+1 cells becomes a single cell (searched once, no duplicate neighbours).
#pragma once

#include "kmc_internal.cuh"

namespace kmc {

__device__ __forceinline__ float f_up(double x) { return __double2float_ru(x); }

struct CellPlan {
  int nc[3];
  double m;
  uint32_t col_shift, col_tz, nkeys;
  bool ok;
};

// cells for search radius h (before the stencil split); key space capped by max_keys.
// Along x the radius is split into K * kxm cells (kxm = 2: narrow cells along the rows
// of the row search), along y and z into K.
__device__ inline CellPlan plan_cells(const double ext[3], double h, int K, uint64_t max_keys,
                                      int kxm = 1) {
  const double u32 = 0x1p-24;
  CellPlan p;
  p.ok = false;
  p.m = 0.0;
  p.col_shift = 0;
  p.col_tz = 1;
  p.nkeys = 1;
  p.nc[0] = p.nc[1] = p.nc[2] = 1;
  for (int attempt = 0; attempt < 64; ++attempt) {
    // margin for binary32 cell assignment: index error <= 4 u32 n per particle
    double nmax = 0.0;
    for (int a = 0; a < 3; ++a) {
      double q = ext[a] * (a == 0 ? K * kxm : K) / h;
      nmax = q > nmax ? q : nmax;
    }
    if (nmax > 65535.0) nmax = 65535.0;
    p.m = 1e-4 + 16.0 * u32 * nmax;
    for (int a = 0; a < 3; ++a) {
      const int Ka = a == 0 ? K * kxm : K;
      const double wt = h * (1.0 + p.m) / Ka;  // target cell width
      double q = floor(ext[a] / wt);
      int c = q > 65535.0 ? 65535 : (int)q;
      if (c < 2 * Ka + 1) c = 1;
      p.nc[a] = c;
    }
    // key space of the tiled column order: T x T Morton tiles, T = 2^t <= 8
    const uint32_t ny = (uint32_t)p.nc[1], nz = (uint32_t)p.nc[2];
    const uint32_t small = ny < nz ? ny : nz;
    uint32_t t = 0;
    while (t < 3 && (1u << (t + 1)) <= small) ++t;
    const uint64_t T = 1ull << t;
    const uint64_t ty = (ny + T - 1) / T, tz = (nz + T - 1) / T;
    const uint64_t nkeys = ty * tz * T * T * (uint64_t)p.nc[0];
    if (nkeys <= max_keys) {
      p.col_shift = t;
      p.col_tz = (uint32_t)tz;
      p.nkeys = (uint32_t)nkeys;
      p.ok = true;
      return p;
    }
    h *= 1.25;  // coarsen until the key space fits
  }
  return p;
}

// Cost estimates for the choice of the split threshold, in units of one pair test of
// the row search (measured on GB300 at 2^24 particles; only the ratios matter):
// a slow particle costs its trimmed half-stencil, about 5 tests per particle per cell
// (rho = particles per cell of width w), plus its set-up (about 6 tests' time; the
// warp-per-cell search at high occupancy tests 13.5 rho pairs per particle at about 2.6
// times the rate, the same cost); a fast particle costs its reach-trimmed stencil
// (about 1.4 times the sphere of radius R_f, at about 2 tests' time per test) plus 15
// per (y, z) column it walks.
__device__ inline double slow_cost(double n, double rho) { return n * (5.0 * rho + 6.0); }
// The binary64 path has no row search (thread per particle or warp per cell, whole
// stencil, binary64 pre-tests): its cost is the half stencil's pair tests, inflated
// when cells hold fewer particles than a warp's lanes can use; a fast particle costs
// its whole stencil at 3 units per test.
__device__ inline double slow_cost_f64(double n, double rho, int K) {
  const double st = (2 * K + 1.0) * (2 * K + 1.0) * (2 * K + 1.0) * 0.5;
  const double eff = rho < 16.0 ? sqrt(16.0 / (rho > 0.25 ? rho : 0.25)) : 1.0;
  return n * st * rho * eff;
}
__device__ inline double fast_cost(double nfast, double rho, double rf_cells, double ncol) {
  const double tests = rho * 1.4 * 4.18879 * rf_cells * rf_cells * rf_cells;
  return nfast * (2.0 * tests + 15.0 * ncol);
}

// Trial thresholds of the speed split, fractions of the bound V of max |v| (squares
// rounded down), with their particle counts cleared for the next count.
__device__ inline void set_split_thresholds(SimDev& s, float vmax2_bound) {
  const double V = sqrt((double)vmax2_bound) * (1.0 + 0x1p-20);
  for (int t = 0; t < kSplitTrials; ++t) {
    const double f = (double)split_frac(t);
    s.d.split_thr[t] = __double2float_rd(f * V * f * V);
    s.d.split_cnt[t] = 0;
  }
}

// Called by all 32 lanes of a warp: lane t < kSplitTrials estimates the cost of
// trial threshold t, lane 0 chooses and writes the grid (the others only read).
__device__ inline void compute_grid(SimDev& s, float vmax2_bound, uint64_t step, uint32_t lane) {
  Grid& g = s.d.grid;
  const double u32 = 0x1p-24, u64 = 0x1p-53;
  const int K = s.K;
  const double scale = s.cell_scale > 1.0 ? s.cell_scale : 1.0;
  const double V = sqrt((double)vmax2_bound) * (1.0 + 0x1p-20);  // upper bound of max |v|
  const double Rfull = s.d0 + 2.0 * V * s.dt;
  double ext[3];
  for (int a = 0; a < 3; ++a) {
    ext[a] = s.box[a];
    if (a == 0 && s.bc[0] == KMC_REFLECT) {
      // upper x wall at the start of this step (particles are below it)
      double X = s.piston_x0 - s.piston_u * ((double)step * s.dt);
      ext[0] = X > 0.0 ? X : s.box[0];
    }
  }

  // ---- split threshold: estimated pair-test cost of each trial (one lane each) --
  const bool can_split = s.split_ok && s.d.have_counts;
  bool my_feasible = false;
  double my_cost = 0.0;
  if (lane < (uint32_t)kSplitTrials) {
    const int t = (int)lane;
    bool feasible_t = false;
    double cost_t = 0.0;
    do {
    if (t > 0 && !can_split) break;
    // trial thresholds were set from the previous step's bound; the slow cell must
    // cover the threshold actually used for classification (a binary32 square)
    const float sq = t == 0 ? 0.0f : s.d.split_thr[t];
    const double S1 = t == 0 ? V : sqrt((double)sq);
    if (t > 0 && !(S1 < V)) break;
    const double hs = (s.d0 + 2.0 * S1 * s.dt) * scale;
    CellPlan p = plan_cells(ext, hs, K, (uint64_t)s.cell_cap / (t == 0 ? 1 : 2));
    if (!p.ok) break;
    const double cells = (double)p.nc[0] * p.nc[1] * p.nc[2];
    const double rho = (double)s.n / cells;
    const bool f64 = s.precision == KMC_FP64;
    if (t == 0) {
      cost_t = f64 ? slow_cost_f64((double)s.n, rho, K) : slow_cost((double)s.n, rho);
      feasible_t = true;
      break;
    }
    if (s.split_ok == 1 && rho < s.split_min_occ) break;
    // fast stencil: c cells on each side per split axis; periodic axes must hold it,
    // and no axis may be a one-cell periodic axis (no minimum-image test there)
    const double nfast = (double)s.d.split_cnt[t];
    double ncol = 1.0, wmin = 0.0, fast_cells = 1.0;
    bool fits = true;
    for (int a = 0; a < 3; ++a) {
      if (p.nc[a] == 1) {
        if (s.bc[a] == KMC_PERIODIC) fits = false;
        continue;
      }
      const double w = ext[a] / p.nc[a];
      wmin = wmin == 0.0 || w < wmin ? w : wmin;
      int c = (int)ceil(Rfull * (1.0 + p.m) / w);
      if (c < K) c = K;
      if (s.bc[a] == KMC_PERIODIC && p.nc[a] < 2 * c + 2) fits = false;
      if (a > 0) ncol *= (2.0 * c + 1.0);
      fast_cells *= (2.0 * c + 1.0);
    }
    if (!fits) break;
    // a fast particle's reach, its speed taken just above the threshold
    const double rf = s.d0 + (1.15 * S1 + V) * s.dt;
    const double rf_cells = wmin > 0.0 ? rf / wmin : 1.0;
    cost_t = f64 ? slow_cost_f64((double)s.n - nfast, rho, K) + nfast * fast_cells * rho * 3.0
                 : slow_cost((double)s.n - nfast, rho) + fast_cost(nfast, rho, rf_cells, ncol);
    feasible_t = true;
    } while (false);
    my_feasible = feasible_t;
    my_cost = cost_t;
  }
  bool feasible[kSplitTrials];
  double cost[kSplitTrials];
  for (int t = 0; t < kSplitTrials; ++t) {
    feasible[t] = __shfl_sync(0xFFFFFFFFu, my_feasible ? 1 : 0, t) != 0;
    cost[t] = __shfl_sync(0xFFFFFFFFu, my_cost, t);
  }
  if (lane != 0) return;  // lane 0 chooses the threshold and writes the grid
  int best = 0;
  if (s.split_ok == 2) {
    // forced: cycle through the feasible trial thresholds step by step
    const int want = (int)(step % (uint64_t)(kSplitTrials - 1));
    for (int d = 0; d < kSplitTrials - 1; ++d) {
      const int t = 1 + (want + d) % (kSplitTrials - 1);
      if (feasible[t]) { best = t; break; }
    }
  } else {
    for (int t = 1; t < kSplitTrials; ++t)
      if (feasible[t] && cost[t] < 0.9 * cost[best]) best = t;
  }
  const float s1sq = best > 0 ? s.d.split_thr[best] : 0.0f;
  const bool split = best > 0;
  const double S1 = split ? sqrt((double)s1sq) : V;
  g.split = split ? 1u : 0u;
  g.split_t = best;
  g.s1sq = s1sq;
  // trial thresholds for the next step (counted by the push of this step)
  set_split_thresholds(s, vmax2_bound);

  CellPlan p = plan_cells(ext, (s.d0 + 2.0 * S1 * s.dt) * scale, K,
                          (uint64_t)s.cell_cap / (split ? 2 : 1));
  {
    // search kernel for the slow population: warp per cell when cells are well
    // filled; the binary32 warp-per-cell search handles no one-cell periodic axis
    // (the row search does)
    const double cells = (double)p.nc[0] * p.nc[1] * p.nc[2];
    const double occ = (double)s.n / cells;
    bool cp = false;
    for (int a = 0; a < 3; ++a) cp = cp || (p.nc[a] == 1 && s.bc[a] == KMC_PERIODIC);
    int mode = s.search_kernel;
    const bool fp32 = s.precision == KMC_GUARDED_FP32;
    if (mode == 0) {
      if (fp32) mode = occ >= 16.0 ? KMC_SEARCH_CELL : KMC_SEARCH_ROW;
      else mode = occ >= 4.0 ? KMC_SEARCH_CELL : KMC_SEARCH_PARTICLE;
    }
    if (mode == KMC_SEARCH_ROW && !fp32) mode = KMC_SEARCH_CELL;
    if (mode == KMC_SEARCH_CELL && cp && fp32) mode = KMC_SEARCH_ROW;
    g.mode = mode;
    g.kx = K;
    if (mode == KMC_SEARCH_ROW && p.nc[0] > 1) {
      // rows of half-width cells: each particle's row is trimmed to its reach in
      // half-cell steps (the grid is otherwise the same)
      const CellPlan q = plan_cells(ext, (s.d0 + 2.0 * S1 * s.dt) * scale, K,
                                    (uint64_t)s.cell_cap / (split ? 2 : 1), 2);
      if (q.ok && q.nc[0] > 1 && q.nc[1] == p.nc[1] && q.nc[2] == p.nc[2]) {
        p = q;
        g.kx = 2 * K;
      }
    }
  }
  if (!p.ok) s.d.status |= ST_CELL_OVERFLOW;
  const int* nc = p.nc;
  const double m = p.m;
  g.col_shift = p.col_shift;
  g.col_tz = p.col_tz;
  g.nkeys = p.nkeys;
  g.K = K;
  int cfast[3] = {0, 0, 0};
  for (int a = 0; a < 3; ++a) {
    if (!split || nc[a] == 1) continue;
    const int Ka = a == 0 ? g.kx : K;
    const double w = ext[a] / nc[a];
    int c = (int)ceil(Rfull * (1.0 + m) / w);
    if (c < Ka) c = Ka;
    cfast[a] = c;
  }
  for (int a = 0; a < 3; ++a) g.cfast[a] = cfast[a];
  for (int a = 0; a < 3; ++a) {
    g.nc[a] = nc[a];
    g.w[a] = nc[a] == 1 ? ext[a] : ext[a] / nc[a];
    g.wf[a] = (float)g.w[a];
    g.inv_wf[a] = nc[a] == 1 ? 0.0f : (float)((double)nc[a] / ext[a]);
  }

  // ---- binary64 sphere pre-test: R > c0 + c1 B  =>  not a candidate ----------
  // Exactly, |r|^2 |v|^2 = (r.v)^2 + |r x v|^2, so |r|^2 = t*^2 |v|^2 + d_min^2 <
  // dt^2 |v|^2 + d0^2 for a candidate; with the roundings of the test this holds
  // with a relative slack below 30 u64, far inside the 2^-40 used here.
  g.c0 = s.d0sq * (1.0 + 0x1p-40) * (1.0 + 0x1p-50);
  g.c1 = s.dt * s.dt * (1.0 + 0x1p-40) * (1.0 + 0x1p-50);

  // ---- binary32 pre-tests ------------------------------------------------------
  // The binary32 mirror holds box coordinates and velocities, each rounded once.
  // Error of the binary32 separation against the binary64 one, per component:
  //   multi-cell axis: both coordinates (u32 L each), a periodic image shifts one
  //     side by the rounded box length (u32 L) and that sum is rounded (u32 L); the
  //     difference itself rounds with u32 |r|: 4 u32 L + u32 rb, plus 8 u64 L for the
  //     binary64 separation's own rounding;
  //   one-cell axis (minimum image in binary32): u32 * 6.1 * extent + 8 u64 L.
  // Velocity difference: 4.1 u32 V.  Component bounds: |r_k| <= rb_k, |v_k| <= 2V.
  double er = 0.0, rn2 = 0.0, rbmax = 0.0;
  for (int a = 0; a < 3; ++a) {
    const double L = s.box[a] > ext[a] ? s.box[a] : ext[a];
    const int Ka = a == 0 ? g.kx : K;
    const int Ke = cfast[a] > Ka ? cfast[a] : Ka;
    double e, rb;
    if (nc[a] == 1) {
      e = 6.1 * u32 * L + 8.0 * u64 * L;
      rb = s.bc[a] == KMC_PERIODIC ? 0.5 * L * (1.0 + 8.0 * u32) + 2.0 * e : L;
    } else {
      rb = (Ke + 1.0 + 2.0 * m) * g.w[a];
      e = u32 * (4.0 * L + rb) * (1.0 + 1e-3) + 8.0 * u64 * L;
    }
    er = e > er ? e : er;
    rbmax = rb > rbmax ? rb : rbmax;
    rn2 += rb * rb;
    g.Lf[a] = (float)s.box[a];
    g.halfLf[a] = (float)(0.5 * s.box[a]);
    g.tief[a] = f_up(4.0 * e);
  }
  {
    // row trimming: a slow-slow candidate has |r| < d0 + (|v_i| + |v_j|) dt <= d0 + 2 S1 dt
    double Lmax = 0.0;
    for (int a = 0; a < 3; ++a) {
      const double L = s.box[a] > ext[a] ? s.box[a] : ext[a];
      Lmax = L > Lmax ? L : Lmax;
    }
    const double reach = (s.d0 + 2.0 * S1 * s.dt) * (1.0 + 1e-6);
    g.row_r2 = f_up(reach * reach * (1.0 + 1e-6));
    // per particle: (i, j) with j slow has |r| < d0 + (|v_i| + |v_j|) dt <= d0 + S1 dt + |v_i| dt
    g.row_a = f_up((s.d0 + S1 * s.dt) * (1.0 + 1e-6));
    g.row_b = f_up(s.dt * (1.0 + 1e-6));
    g.fast_a = f_up((s.d0 + V * s.dt) * (1.0 + 1e-6));
    g.row_eps = f_up(16.0 * u32 * Lmax);
    g.row_pad = f_up(4.0 * u32 * Lmax);
  }
  const double rn = sqrt(rn2) * (1.0 + 1e-6);
  const double ev = 4.1 * u32 * V;
  const double g3 = 3.0 * u32 / (1.0 - 3.0 * u32);
  const double g3d = 3.0 * u64 / (1.0 - 3.0 * u64);
  const double g2 = 2.0 * u32 / (1.0 - 2.0 * u32);
  const double up2 = 1.0 + 2.0 * u32, up4 = 1.0 + 4.0 * u32;
  const double rel40 = 1.0 + 0x1p-40;
  const double s3 = 1.7320508075688772 * (1.0 + 1e-15);
  const double bslack = 7.0 * ev * V + 3.0 * ev * ev;  // |v|^2 - |v~|^2 slack, absolute
  const double dt = s.dt, d0sq = s.d0sq;
  // sphere test
  const double c0 = (rel40 * (d0sq + dt * dt * bslack) + 2.0 * s3 * er * rn) * (1.0 + g3);
  const double c1 = dt * dt * rel40 * (1.0 + g3) / (1.0 - g3);
  g.s_c0 = f_up(c0 * up2);
  g.s_c1 = f_up(c1 * up2);
  // approach test (t* >= 0): |A~ - A64| <= a_g
  const double Ga = (s3 * (ev * rn + 2.0 * V * er) + g3 * rn * 2.0 * V * 1.01 + g3d * rn * 2.0 * V) *
                    (1.0 + 1e-3);
  g.a_g = f_up(Ga);
  // time test (t* < dt): X~ = A~ - dt B~ > t_g  =>  A64 >= dt B64
  const double Ex = u32 * (rn * 2.0 * V * 1.01 + 2.0 * dt * 4.0 * V * V * 1.02);
  const double Gt = (Ex + Ga + dt * (8.1 * V * V * g3 + bslack)) * (1.0 + 1e-3);
  g.t_g = f_up(Gt);
  g.dtf = (float)dt;
  // distance test (d_min < d0): |w~| >= w_e + d0 sqrt(B_up)  =>  W64 >= d0^2 B64
  const double ew = (2.0 * (rbmax * ev + 2.0 * V * er) * 1.001 + g2 * 2.0 * rbmax * 2.0 * V * 1.01) +
                    2.0 * (2.0 * u64) * rbmax * 2.0 * V;
  g.w_e = f_up(s3 * ew * up4);
  g.b_rel = f_up((1.0 / (1.0 - g3)) * (1.0 + g3d) * up2);
  g.b_abs = f_up(bslack * (1.0 + g3d) * up2);
  g.d0up = f_up(s.d0 * rel40 / sqrt(1.0 - g3d) * up4 * (1.0 + 4.0 * u32));
  g.w_rel = f_up((1.0 + g3) * up4);
}

}  // namespace kmc
