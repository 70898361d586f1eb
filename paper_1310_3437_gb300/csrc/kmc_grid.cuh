// kmc_grid.cuh -- per-step search grid and the guard bands of the binary32
// pre-tests, computed on the device by one thread per simulation.
//
// Cell size.  A candidate pair has |r| <= d_min + |v| t* < d0 + 2 vmax dt (the
// relative speed is at most 2 vmax), so with cells at least h = d0 + 2 vmax dt wide
// the partner lies in the same or a neighbouring cell (Sec. 2: 26 neighbours in 3D).
// With stencil K the cell is h/K wide and K cells are searched on each side.  The
// cell width gets a relative margin m that covers the binary32 rounding of the
// cell assignment, and cell_scale >= 1 only enlarges it: none of this can change a
// result, only the amount of work.  An axis with fewer than 2K+1 cells becomes a
// single cell (searched once, no duplicate neighbours).
#pragma once

#include "kmc_internal.cuh"

namespace kmc {

__device__ __forceinline__ float f_up(double x) { return __double2float_ru(x); }

__device__ inline void compute_grid(SimDev& s, float vmax2_bound, uint64_t step) {
  Grid& g = s.d.grid;
  const double u32 = 0x1p-24, u64 = 0x1p-53;
  const int K = s.K;
  double V = sqrt((double)vmax2_bound) * (1.0 + 0x1p-20);  // upper bound of max |v|
  double hmin = s.d0 + 2.0 * V * s.dt;
  double ext[3];
  for (int a = 0; a < 3; ++a) {
    ext[a] = s.box[a];
    if (a == 0 && s.bc[0] == KMC_REFLECT) {
      // upper x wall at the start of this step (particles are below it)
      double X = s.piston_x0 - s.piston_u * ((double)step * s.dt);
      ext[0] = X > 0.0 ? X : s.box[0];
    }
  }
  double h = hmin * (s.cell_scale > 1.0 ? s.cell_scale : 1.0);
  int nc[3];
  double m = 0.0;
  for (int attempt = 0; attempt < 64; ++attempt) {
    // margin for binary32 cell assignment: index error <= 4 u32 n per particle
    double nmax = 0.0;
    for (int a = 0; a < 3; ++a) {
      double q = ext[a] * K / h;
      nmax = q > nmax ? q : nmax;
    }
    if (nmax > 65535.0) nmax = 65535.0;
    m = 1e-4 + 16.0 * u32 * nmax;
    double wt = h * (1.0 + m) / K;  // target cell width
    for (int a = 0; a < 3; ++a) {
      double q = floor(ext[a] / wt);
      int c = q > 65535.0 ? 65535 : (int)q;
      if (c < 2 * K + 1) c = 1;
      nc[a] = c;
    }
    // key space of the column-Morton order
    uint32_t ny = (uint32_t)nc[1], nz = (uint32_t)nc[2];
    uint32_t small = ny < nz ? ny : nz, large = ny < nz ? nz : ny;
    uint32_t sh = 0;
    while ((1u << sh) < small) ++sh;
    uint64_t P = 1ull << sh;
    uint64_t cols = ((large + P - 1) / P) * P * P;
    uint64_t nkeys = cols * (uint64_t)nc[0];
    if (nkeys <= (uint64_t)s.cell_cap && sh <= 15) {
      g.col_shift = sh;
      g.y_major = ny >= nz ? 1u : 0u;
      g.nkeys = (uint32_t)nkeys;
      break;
    }
    h *= 1.25;  // coarsen until the key space fits
    if (attempt == 63) s.d.status |= ST_CELL_OVERFLOW;
  }
  g.K = K;
  {
    // search kernel: warp per cell when cells hold enough particles to fill a warp's
    // lanes with partners; the binary32 warp-per-cell search handles no one-cell
    // periodic axis (those need the minimum image per pair)
    double cells = (double)nc[0] * nc[1] * nc[2];
    double occ = (double)s.n / cells;
    bool cp = false;
    for (int a = 0; a < 3; ++a) cp = cp || (nc[a] == 1 && s.bc[a] == KMC_PERIODIC);
    int mode = s.search_kernel;
    if (mode == 0) mode = occ >= 4.0 ? KMC_SEARCH_CELL : KMC_SEARCH_PARTICLE;
    if (mode == KMC_SEARCH_CELL && cp && s.precision == KMC_GUARDED_FP32) mode = KMC_SEARCH_PARTICLE;
    g.mode = mode;
  }
  double wmax = 0.0;
  for (int a = 0; a < 3; ++a) {
    g.nc[a] = nc[a];
    g.w[a] = nc[a] == 1 ? ext[a] : ext[a] / nc[a];
    g.wf[a] = (float)g.w[a];
    g.inv_wf[a] = nc[a] == 1 ? 0.0f : (float)((double)nc[a] / ext[a]);
    wmax = g.w[a] > wmax ? g.w[a] : wmax;
  }

  // ---- binary64 sphere pre-test: R > c0 + c1 B  =>  not a candidate ----------
  // Exactly, |r|^2 |v|^2 = (r.v)^2 + |r x v|^2, so |r|^2 = t*^2 |v|^2 + d_min^2 <
  // dt^2 |v|^2 + d0^2 for a candidate; with the roundings of the test this holds
  // with a relative slack below 30 u64, far inside the 2^-40 used here.
  g.c0 = s.d0sq * (1.0 + 0x1p-40) * (1.0 + 0x1p-50);
  g.c1 = s.dt * s.dt * (1.0 + 0x1p-40) * (1.0 + 0x1p-50);

  // ---- binary32 pre-tests ------------------------------------------------------
  // Error of the binary32 separation against the binary64 one, per component:
  //   split axis: offsets from the cell corner (binary64 difference rounded once)
  //     plus the stencil shift: u32 w (3K + 5) + 8 u64 L;
  //   one-cell axis: u32 * 6.1 * extent + 8 u64 L.
  // Velocity difference: 4.1 u32 V.  Component bounds: |r_k| <= rb_k, |v_k| <= 2V.
  double Lmax = 0.0, er = 0.0, rn2 = 0.0, rbmax = 0.0;
  for (int a = 0; a < 3; ++a) {
    double L = s.box[a] > ext[a] ? s.box[a] : ext[a];
    Lmax = L > Lmax ? L : Lmax;
    double e, rb;
    if (nc[a] == 1) {
      e = 6.1 * u32 * L + 8.0 * u64 * L;
      rb = s.bc[a] == KMC_PERIODIC ? 0.5 * L * (1.0 + 8.0 * u32) + 2.0 * e : L;
    } else {
      e = u32 * g.w[a] * (3.0 * K + 5.0) * (1.0 + 1e-3) + 8.0 * u64 * L;
      rb = (K + 1.0 + 2.0 * m) * g.w[a];
    }
    er = e > er ? e : er;
    rbmax = rb > rbmax ? rb : rbmax;
    rn2 += rb * rb;
    g.Lf[a] = (float)s.box[a];
    g.halfLf[a] = (float)(0.5 * s.box[a]);
    g.tief[a] = f_up(4.0 * e);
  }
  double rn = sqrt(rn2) * (1.0 + 1e-6);
  double ev = 4.1 * u32 * V;
  double g3 = 3.0 * u32 / (1.0 - 3.0 * u32);
  double g3d = 3.0 * u64 / (1.0 - 3.0 * u64);
  double g2 = 2.0 * u32 / (1.0 - 2.0 * u32);
  double up2 = 1.0 + 2.0 * u32, up4 = 1.0 + 4.0 * u32;
  double rel40 = 1.0 + 0x1p-40;
  double s3 = 1.7320508075688772 * (1.0 + 1e-15);
  double bslack = 7.0 * ev * V + 3.0 * ev * ev;  // |v|^2 - |v~|^2 slack, absolute
  double dt = s.dt, d0sq = s.d0sq;
  // sphere test
  double c0 = (rel40 * (d0sq + dt * dt * bslack) + 2.0 * s3 * er * rn) * (1.0 + g3);
  double c1 = dt * dt * rel40 * (1.0 + g3) / (1.0 - g3);
  g.s_c0 = f_up(c0 * up2);
  g.s_c1 = f_up(c1 * up2);
  // approach test (t* >= 0): |A~ - A64| <= a_g
  double Ga = (s3 * (ev * rn + 2.0 * V * er) + g3 * rn * 2.0 * V * 1.01 + g3d * rn * 2.0 * V) *
              (1.0 + 1e-3);
  g.a_g = f_up(Ga);
  // time test (t* < dt): X~ = A~ - dt B~ > t_g  =>  A64 >= dt B64
  double Ex = u32 * (rn * 2.0 * V * 1.01 + 2.0 * dt * 4.0 * V * V * 1.02);
  double Gt = (Ex + Ga + dt * (8.1 * V * V * g3 + bslack)) * (1.0 + 1e-3);
  g.t_g = f_up(Gt);
  g.dtf = (float)dt;
  // distance test (d_min < d0): |w~| >= w_e + d0 sqrt(B_up)  =>  W64 >= d0^2 B64
  double ew = (2.0 * (rbmax * ev + 2.0 * V * er) * 1.001 + g2 * 2.0 * rbmax * 2.0 * V * 1.01) +
              2.0 * (2.0 * u64) * rbmax * 2.0 * V;
  g.w_e = f_up(s3 * ew * up4);
  g.b_rel = f_up((1.0 / (1.0 - g3)) * (1.0 + g3d) * up2);
  g.b_abs = f_up(bslack * (1.0 + g3d) * up2);
  g.d0up = f_up(s.d0 * rel40 / sqrt(1.0 - g3d) * up4 * (1.0 + 4.0 * u32));
  g.w_rel = f_up((1.0 + g3) * up4);
  (void)Lmax;
}

}  // namespace kmc
