// kmc_search.cu -- neighbourhood search for collision candidates (Sec. 2: every
// particle of a bin is compared with the particles of its own and the neighbouring
// bins; the cost is O(B * N_bin^2 / P), eq. "eff").
//
// GB300 form.  One thread per particle, particles in cell order, so the lanes of a
// warp sit in the same or adjacent cells and read the same partner records
// (broadcast loads, L1/L2 reuse of the neighbour cells).  Each unordered pair is
// tested once: the thread of particle p visits the "forward half" of the stencil
// (own cell with j > p, then the cells whose offset (dz, dy, dx) is
// lexicographically positive).  The search does no division: it only culls pairs
// that provably fail the paper's criteria, and emits the survivors; kmc_match.cu
// re-tests every survivor with the exact binary64 predicate.
//
//   KMC_FP64          binary64 sphere test |r|^2 > d0^2 + dt^2 |v|^2 (+2^-40 slack).
//   KMC_GUARDED_FP32  binary32 on cell-local offsets: sphere test, then approach,
//                     time and distance tests, each widened by a guard band that
//                     bounds the binary32 error (kmc_grid.cuh derives the bands).
// A pair that passes the binary64 predicate is never culled by either variant, so
// both variants produce exactly the candidate list of the binary64 definition.
#include <algorithm>

#include "kmc_internal.cuh"

namespace kmc {

struct Own32 {
  float ox, oy, oz, vx, vy, vz;
};

// Two binary32 values in one 64-bit register, and the packed (f32x2) arithmetic of
// sm_100-class GPUs on them: each half is rounded exactly as the scalar operation.
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 pack2(float a, float b) {
  f32x2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void unpack2(f32x2 r, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ f32x2 sub2(f32x2 a, f32x2 b) {
  f32x2 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
  f32x2 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
  f32x2 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

__device__ __forceinline__ void min_image_f(float& r, float halfL, float L, float tie, bool& keep) {
  float ar = fabsf(r);
  if (fabsf(ar - halfL) <= tie) keep = true;
  else if (ar > halfL) r = r > 0.f ? r - L : r + L;
}

// block-uniform: does any simulation of the batch run this step with the given search
// (mode < 0: the fast-particle search, i.e. any simulation under the speed split)?
__device__ __forceinline__ bool batch_uses(const Batch& B, int mode) {
  bool any = false;
  for (int q = threadIdx.x; q < B.nsims; q += blockDim.x) {
    const SimDev& t = *B.sims[q];
    any = any || (sim_active(t) && (mode < 0 ? t.d.grid.split != 0u : t.d.grid.mode == mode));
  }
  return __syncthreads_or(any) != 0;
}

// Conservative binary64 approach and time pre-tests on a sphere survivor.  The search
// computes r = x_j - x_i, v = v_j - v_i, |v|^2 and r.v with the same operations as the
// exact test (k_refine), so rv is its value bit for bit; the exact test needs
// t* = fl(-rv / vv) >= 0 and < dt.  Dropped here only when that provably fails:
//   rv > vv 2^-1000: -rv / vv <= -2^-1000 (too large to round to -0.0, which would
//     count as >= 0), so t* < 0;
//   -rv >= fl(fl(dt vv)(1 + 2^-48)) >= dt vv (1 + 2^-50): fl(-rv / vv) >= dt.
// (vv >= 2^-900 here; rounding of the two thresholds only makes the drops rarer.)
__device__ __forceinline__ bool f64_cannot_approach(double rv, double vv, double dt) {
  return rv > dmul(vv, 0x1p-1000) || -rv >= dmul(dmul(dt, vv), 1.0 + 0x1p-48);
}

template <int PREC, int K>
__global__ void __launch_bounds__(kTile) k_search(Batch B) {
  __shared__ uint2 sbuf[kSearchBuf];
  __shared__ uint32_t scnt, sbase;
  __shared__ unsigned long long stests;
  // grid-stride over tiles of kTile particles (an occupancy-sized grid: the kernel is
  // launched every step and exits at once when the step runs another search)
  if (!batch_uses(B, KMC_SEARCH_PARTICLE)) return;
  const uint32_t ntiles = B.ptile[B.nsims];
  for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    int k = find_sim(B.ptile, B.nsims, tile);
    SimDev& s = *B.sims[k];
    if (s.d.grid.mode != KMC_SEARCH_PARTICLE) continue;
    // the previous tile's flush has read the staging buffer; the status word can change
    // while the search runs (a full pair buffer), so the block takes one answer
    if (!__syncthreads_and(sim_active(s))) continue;
    if (threadIdx.x == 0) { scnt = 0; stests = 0; }
    __syncthreads();

    const Grid g = s.d.grid;
    const uint32_t n = s.n;
    const int cur = s.d.parity ^ 1;
    const uint32_t* __restrict__ cs = s.cell_start;
    const uint32_t edge_cap = s.edge_cap;
    uint2* __restrict__ edges = s.edge;
    const int nx = g.nc[0], ny = g.nc[1], nz = g.nc[2];
    const int Kx = nx == 1 ? 0 : K, Ky = ny == 1 ? 0 : K, Kz = nz == 1 ? 0 : K;
    const bool px = s.bc[0] == KMC_PERIODIC, py = s.bc[1] == KMC_PERIODIC,
               pz = s.bc[2] == KMC_PERIODIC;
    unsigned long long tests = 0;

    uint32_t p = (tile - B.ptile[k]) * kTile + threadIdx.x;
    // with the speed split only the slow population (keys below nkeys) is searched here;
    // particles that left through absorbing walls sit after every cell key
    const uint32_t nslow = (g.split || s.absorb) ? __ldg(cs + g.nkeys) : n;
    if (p < nslow) {
      // the particle's cell, recomputed as the sort computed it
      const int cx = cell_coord(g, 0, s.x[cur][0][p]), cy = cell_coord(g, 1, s.x[cur][1][p]),
                cz = cell_coord(g, 2, s.x[cur][2][p]);

      // own record
      double xo[3], vo[3];
      Own32 o32;
      const double* __restrict__ X0 = s.x[cur][0];
      const double* __restrict__ X1 = s.x[cur][1];
      const double* __restrict__ X2 = s.x[cur][2];
      const double* __restrict__ V0 = s.v[cur][0];
      const double* __restrict__ V1 = s.v[cur][1];
      const double* __restrict__ V2 = s.v[cur][2];
      const float4* __restrict__ MM = s.mir;
      if (PREC == KMC_FP64) {
        xo[0] = X0[p]; xo[1] = X1[p]; xo[2] = X2[p];
        vo[0] = V0[p]; vo[1] = V1[p]; vo[2] = V2[p];
      } else {
        float4 a;
        float2 b;
        mirror_load(MM, p, a, b);
        o32 = {a.x, a.y, a.z, a.w, b.x, b.y};
      }
      // one-cell periodic axes need the minimum image explicitly
      const bool cp0 = nx == 1 && px, cp1 = ny == 1 && py, cp2 = nz == 1 && pz;
      const bool any_cp = cp0 || cp1 || cp2;
      const double L0 = s.box[0], L1 = s.box[1], L2 = s.box[2];

      // a neighbour reached across a periodic boundary is seen as its image: wrap
      // flags -1 (below 0) or +1 (at or above the extent) per axis
      for (int dz = 0; dz <= Kz; ++dz) {
        int qz = cz + dz, wz = 0;
        if (qz >= nz) {
          if (!pz) break;
          qz -= nz;
          wz = 1;
        }
        for (int dy = (dz == 0 ? 0 : -Ky); dy <= Ky; ++dy) {
          int qy = cy + dy, wy = 0;
          if (qy < 0) {
            if (!py) continue;
            qy += ny;
            wy = -1;
          } else if (qy >= ny) {
            if (!py) continue;
            qy -= ny;
            wy = 1;
          }
          const uint32_t colbase = col_code(g, (uint32_t)qy, (uint32_t)qz) * (uint32_t)nx;
          const int dx0 = (dz == 0 && dy == 0) ? 0 : -Kx;
          for (int dx = dx0; dx <= Kx; ++dx) {
            int qx = cx + dx, wx = 0;
            if (qx < 0) {
              if (!px) continue;
              qx += nx;
              wx = -1;
            } else if (qx >= nx) {
              if (!px) continue;
              qx -= nx;
              wx = 1;
            }
            const uint32_t key = colbase + (uint32_t)qx;
            uint32_t beg = __ldg(cs + key), end = __ldg(cs + key + 1);
            if (dz == 0 && dy == 0 && dx == 0) beg = p + 1;
            if (beg >= end) continue;
            tests += end - beg;
            if (PREC == KMC_FP64) {
              for (uint32_t j = beg; j < end; ++j) {
                double r0 = dsub(__ldg(X0 + j), xo[0]);
                double r1 = dsub(__ldg(X1 + j), xo[1]);
                double r2 = dsub(__ldg(X2 + j), xo[2]);
                if (px) { if (r0 > 0.5 * L0) r0 = dsub(r0, L0); else if (r0 < -0.5 * L0) r0 = dadd(r0, L0); }
                if (py) { if (r1 > 0.5 * L1) r1 = dsub(r1, L1); else if (r1 < -0.5 * L1) r1 = dadd(r1, L1); }
                if (pz) { if (r2 > 0.5 * L2) r2 = dsub(r2, L2); else if (r2 < -0.5 * L2) r2 = dadd(r2, L2); }
                double g0 = dsub(__ldg(V0 + j), vo[0]);
                double g1 = dsub(__ldg(V1 + j), vo[1]);
                double g2 = dsub(__ldg(V2 + j), vo[2]);
                double R = dadd(dadd(dmul(r0, r0), dmul(r1, r1)), dmul(r2, r2));
                double Bv = dadd(dadd(dmul(g0, g0), dmul(g1, g1)), dmul(g2, g2));
                if (Bv >= 0x1p-900 && R > dadd(g.c0, dmul(g.c1, Bv))) continue;
                if (Bv >= 0x1p-900 &&
                    f64_cannot_approach(dadd(dadd(dmul(r0, g0), dmul(r1, g1)), dmul(r2, g2)), Bv, s.dt))
                  continue;
                uint32_t pos = atomicAdd(&scnt, 1u);
                if (pos < (uint32_t)kSearchBuf) {
                  sbuf[pos] = make_uint2(p, j);
                } else {
                  uint32_t gpos = atomicAdd(&s.d.n_raw, 1u);
                  if (gpos < edge_cap) edges[gpos] = make_uint2(p, j);
                  else atomicOr(&s.d.status, ST_EDGE_OVERFLOW);
                }
              }
            } else {
              // own coordinates moved by the image shift (j seen at x_j + w L)
              const float sx = o32.ox - (float)wx * g.Lf[0];
              const float sy = o32.oy - (float)wy * g.Lf[1];
              const float sz = o32.oz - (float)wz * g.Lf[2];
              for (uint32_t j = beg; j < end; ++j) {
                float4 a;
                float2 b;
                mirror_load(MM, j, a, b);
                float rx = a.x - sx, ry = a.y - sy, rz = a.z - sz;
                bool keep = false;
                if (any_cp) {
                  // minimum image on one-cell periodic axes; near the tie the two
                  // images are both possible in binary64: keep the pair unculled
                  if (cp0) min_image_f(rx, g.halfLf[0], g.Lf[0], g.tief[0], keep);
                  if (cp1) min_image_f(ry, g.halfLf[1], g.Lf[1], g.tief[1], keep);
                  if (cp2) min_image_f(rz, g.halfLf[2], g.Lf[2], g.tief[2], keep);
                }
                const float gx = a.w - o32.vx, gy = b.x - o32.vy, gz = b.y - o32.vz;
                const float R = fmaf(rz, rz, fmaf(ry, ry, rx * rx));
                const float Bv = fmaf(gz, gz, fmaf(gy, gy, gx * gx));
                if (!keep) {
                  if (R > fmaf(g.s_c1, Bv, g.s_c0)) continue;
                  // rare: full guarded test on the sphere survivors
                  const float A = -fmaf(rz, gz, fmaf(ry, gy, rx * gx));
                  if (A < -g.a_g) continue;
                  if (fmaf(-g.dtf, Bv, A) > g.t_g) continue;
                  const float wx = fmaf(ry, gz, -(rz * gy));
                  const float wy = fmaf(rz, gx, -(rx * gz));
                  const float wz = fmaf(rx, gy, -(ry * gx));
                  const float W = fmaf(wz, wz, fmaf(wy, wy, wx * wx));
                  const float thr = fmaf(g.d0up, sqrtf(fmaf(Bv, g.b_rel, g.b_abs)), g.w_e);
                  if (W > thr * thr * g.w_rel) continue;
                }
                uint32_t pos = atomicAdd(&scnt, 1u);
                if (pos < (uint32_t)kSearchBuf) {
                  sbuf[pos] = make_uint2(p, j);
                } else {
                  uint32_t gpos = atomicAdd(&s.d.n_raw, 1u);
                  if (gpos < edge_cap) edges[gpos] = make_uint2(p, j);
                  else atomicOr(&s.d.status, ST_EDGE_OVERFLOW);
                }
              }
            }
          }
        }
      }
    }

    // block totals: pair tests and the staged pairs
    for (int o = 16; o > 0; o >>= 1) tests += __shfl_down_sync(0xFFFFFFFFu, tests, o);
    if ((threadIdx.x & 31) == 0 && tests) atomicAdd(&stests, tests);
    __syncthreads();
    uint32_t cnt = scnt < (uint32_t)kSearchBuf ? scnt : (uint32_t)kSearchBuf;
    if (threadIdx.x == 0) {
      if (stests) atomicAdd(&s.d.pair_tests, stests);
      sbase = cnt ? atomicAdd(&s.d.n_raw, cnt) : 0u;
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < cnt; i += kTile) {
      uint32_t gpos = sbase + i;
      if (gpos < edge_cap) edges[gpos] = sbuf[i];
      else atomicOr(&s.d.status, ST_EDGE_OVERFLOW);
    }
  }
}

// --------------------------------------------------------------------------- //
// Warp-per-cell search.  A warp owns one cell A.  For every forward column run of
// the stencil, the run's particles (contiguous in cell order) are loaded 32 at a
// time, one partner j per lane, with coalesced loads; the particles i of A are
// staged in shared memory and read by broadcast in a warp-uniform loop.  Each lane
// thus tests its j against every i of A with no divergence and no per-pair address
// arithmetic.  Emitted pairs go through a per-warp shared-memory buffer (one global
// atomic per flush).
constexpr int kCellWarps = 8;
constexpr int kWarpBuf = 64;

struct WarpEmit {
  uint2* buf;        // this warp's staging buffer in shared memory
  uint32_t count;    // warp-uniform fill level
};

__device__ __forceinline__ void warp_flush(WarpEmit& w, SimDev& s, uint32_t lane) {
  __syncwarp();
  if (w.count) {
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(&s.d.n_raw, w.count);
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    for (uint32_t k = lane; k < w.count; k += 32) {
      uint32_t g = base + k;
      if (g < s.edge_cap) s.edge[g] = w.buf[k];
      else atomicOr(&s.d.status, ST_EDGE_OVERFLOW);
    }
    w.count = 0;
  }
  __syncwarp();
}

__device__ __forceinline__ void warp_emit(WarpEmit& w, SimDev& s, uint32_t lane, bool emit,
                                          uint32_t i, uint32_t j) {
  unsigned m = __ballot_sync(0xFFFFFFFFu, emit);
  if (!m) return;
  uint32_t c = (uint32_t)__popc(m);
  if (w.count + c > (uint32_t)kWarpBuf) warp_flush(w, s, lane);
  if (emit) w.buf[w.count + __popc(m & ((1u << lane) - 1u))] = make_uint2(i, j);
  w.count += c;
  __syncwarp();
}

template <int PREC, int K>
__global__ void __launch_bounds__(kCellWarps * 32) k_search_cell(Batch B) {
  constexpr int ICAP = PREC == KMC_FP64 ? 32 : 64;
  constexpr int NF = PREC == KMC_FP64 ? 1 : kCellWarps;
  constexpr int ND = PREC == KMC_FP64 ? kCellWarps : 1;
  __shared__ float4 sa[NF][PREC == KMC_FP64 ? 1 : ICAP];
  __shared__ float2 sb[NF][PREC == KMC_FP64 ? 1 : ICAP];
  __shared__ double sd[ND][6][PREC == KMC_FP64 ? ICAP : 1];
  __shared__ uint2 wbuf[kCellWarps][kWarpBuf];
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const uint32_t gwarp = blockIdx.x * kCellWarps + warp, nwarps = gridDim.x * kCellWarps;

  // The cells of the batch's simulations are dealt to the warps as one sequence: a
  // simulation's cells start at the warp after the previous simulation's last.  Every
  // warp walks the simulations in the same order and decides on fields that stay fixed
  // during the launch, so all agree on the running base; the status word, which the
  // search itself can set (a full pair buffer), only gates the work.  Dealt from warp 0
  // each time, the small simulations of a batch all landed on the same few blocks.
  uint32_t base = 0;
  for (int k = 0; k < B.nsims; ++k) {
    SimDev& s = *B.sims[k];
    if (!sim_scheduled(s) || s.d.grid.mode != KMC_SEARCH_CELL) continue;
    const uint32_t first = (gwarp + nwarps - base) % nwarps;
    base = (base + s.d.grid.nkeys % nwarps) % nwarps;
    if (!__all_sync(0xFFFFFFFFu, sim_active(s))) continue;
    const Grid& G = s.d.grid;
    const int nx = G.nc[0], ny = G.nc[1], nz = G.nc[2];
    const int Kx = nx == 1 ? 0 : K, Ky = ny == 1 ? 0 : K, Kz = nz == 1 ? 0 : K;
    const bool px = s.bc[0] == KMC_PERIODIC, py = s.bc[1] == KMC_PERIODIC,
               pz = s.bc[2] == KMC_PERIODIC;
    const uint32_t nkeys = G.nkeys;
    const uint32_t* __restrict__ cs = s.cell_start;
    const int cur = s.d.parity ^ 1;
    const float wx = G.wf[0], wy = G.wf[1], wz = G.wf[2];
    const float c0 = G.s_c0, c1 = G.s_c1, ag = G.a_g, tg = G.t_g, dtf = G.dtf;
    const float d0up = G.d0up, brel = G.b_rel, babs = G.b_abs, we = G.w_e, wrel = G.w_rel;
    const double C0 = G.c0, C1 = G.c1;
    const double L0 = s.box[0], L1 = s.box[1], L2 = s.box[2];
    const float4* __restrict__ MM = s.mir;
    const double* __restrict__ X0 = s.x[cur][0];
    const double* __restrict__ X1 = s.x[cur][1];
    const double* __restrict__ X2 = s.x[cur][2];
    const double* __restrict__ V0 = s.v[cur][0];
    const double* __restrict__ V1 = s.v[cur][1];
    const double* __restrict__ V2 = s.v[cur][2];
    WarpEmit we_ = {wbuf[warp], 0u};
    unsigned long long tests = 0;

    for (uint32_t key = first; key < nkeys; key += nwarps) {
      const uint32_t startA = __ldg(cs + key), endA = __ldg(cs + key + 1);
      if (startA == endA) continue;
      int cx, cy, cz;
      key_decode(G, key, cx, cy, cz);
      for (uint32_t i0 = startA; i0 < endA; i0 += ICAP) {
        const uint32_t nI = endA - i0 < (uint32_t)ICAP ? endA - i0 : (uint32_t)ICAP;
        __syncwarp();
        for (uint32_t t = lane; t < nI; t += 32) {
          if (PREC == KMC_FP64) {
            sd[warp][0][t] = X0[i0 + t]; sd[warp][1][t] = X1[i0 + t]; sd[warp][2][t] = X2[i0 + t];
            sd[warp][3][t] = V0[i0 + t]; sd[warp][4][t] = V1[i0 + t]; sd[warp][5][t] = V2[i0 + t];
          } else {
            float4 a;
            float2 b;
            mirror_load(MM, i0 + t, a, b);
            sa[warp][t] = a;
            sb[warp][t] = b;
          }
        }
        __syncwarp();
        for (int dz = 0; dz <= Kz; ++dz) {
          int qz = cz + dz;
          if (qz >= nz) {
            if (!pz) break;
            qz -= nz;
          }
          for (int dy = (dz == 0 ? 0 : -Ky); dy <= Ky; ++dy) {
            int qy = cy + dy;
            if (qy < 0) {
              if (!py) continue;
              qy += ny;
            } else if (qy >= ny) {
              if (!py) continue;
              qy -= ny;
            }
            const uint32_t colbase = col_code(G, (uint32_t)qy, (uint32_t)qz) * (uint32_t)nx;
            const bool own_col = dz == 0 && dy == 0;
            const float shy = (float)dy * wy, shz = (float)dz * wz;
            // split the x run into pieces of consecutive cells (periodic wrap)
            int dx = own_col ? 0 : -Kx;
            while (dx <= Kx) {
              const int q0 = cx + dx;  // unwrapped cell index
              const int region = q0 < 0 ? -1 : (q0 >= nx ? 1 : 0);
              if (region != 0 && !px) { ++dx; continue; }
              const int qx = q0 - region * nx;
              // extend the piece while the next cell lies in the same wrap region, so
              // that its cells are consecutive keys of the column
              int m = 1;
              while (dx + m <= Kx) {
                const int q2 = cx + dx + m;
                const int r2 = q2 < 0 ? -1 : (q2 >= nx ? 1 : 0);
                if (r2 != region) break;
                ++m;
              }
              const int dxa = dx;
              dx += m;
              const uint32_t jbeg = __ldg(cs + colbase + qx), jend = __ldg(cs + colbase + qx + m);
              if (jbeg == jend) continue;
              uint32_t bnd[2 * K];
#pragma unroll
              for (int t = 0; t < 2 * K; ++t) bnd[t] = (t + 1 < m) ? __ldg(cs + colbase + qx + t + 1) : jend;
              const bool has_own = own_col && dxa <= 0 && dxa + m > 0;
              // analytic count of the pair tests of this piece
              if (lane == 0) {
                uint64_t len = jend - jbeg;
                if (has_own) {
                  uint64_t nA = endA - startA;
                  uint64_t inc = (uint64_t)nI * (endA - i0 - 1) - (uint64_t)nI * (nI - 1) / 2;
                  tests += (uint64_t)nI * (len - nA) + inc;
                } else {
                  tests += (uint64_t)nI * len;
                }
              }
              for (uint32_t cb = jbeg; cb < jend; cb += 32) {
                const uint32_t j = cb + lane;
                const bool jv = j < jend;
                const bool jown = has_own && j >= startA && j < endA;
                if (PREC == KMC_FP64) {
                  double xj0 = 0, xj1 = 0, xj2 = 0, vj0 = 0, vj1 = 0, vj2 = 0;
                  if (jv) {
                    xj0 = X0[j]; xj1 = X1[j]; xj2 = X2[j];
                    vj0 = V0[j]; vj1 = V1[j]; vj2 = V2[j];
                  }
                  for (uint32_t ii = 0; ii < nI; ++ii) {
                    const uint32_t i = i0 + ii;
                    bool valid = jv && (!jown || j > i);
                    double r0 = dsub(xj0, sd[warp][0][ii]);
                    double r1 = dsub(xj1, sd[warp][1][ii]);
                    double r2 = dsub(xj2, sd[warp][2][ii]);
                    if (px) { if (r0 > 0.5 * L0) r0 = dsub(r0, L0); else if (r0 < -0.5 * L0) r0 = dadd(r0, L0); }
                    if (py) { if (r1 > 0.5 * L1) r1 = dsub(r1, L1); else if (r1 < -0.5 * L1) r1 = dadd(r1, L1); }
                    if (pz) { if (r2 > 0.5 * L2) r2 = dsub(r2, L2); else if (r2 < -0.5 * L2) r2 = dadd(r2, L2); }
                    double g0 = dsub(vj0, sd[warp][3][ii]);
                    double g1 = dsub(vj1, sd[warp][4][ii]);
                    double g2 = dsub(vj2, sd[warp][5][ii]);
                    double R = dadd(dadd(dmul(r0, r0), dmul(r1, r1)), dmul(r2, r2));
                    double Bv = dadd(dadd(dmul(g0, g0), dmul(g1, g1)), dmul(g2, g2));
                    bool emit = valid && !(Bv >= 0x1p-900 && R > dadd(C0, dmul(C1, Bv)));
                    if (emit && Bv >= 0x1p-900 &&
                        f64_cannot_approach(dadd(dadd(dmul(r0, g0), dmul(r1, g1)), dmul(r2, g2)), Bv, s.dt))
                      emit = false;
                    warp_emit(we_, s, lane, emit, i, j);
                  }
                } else {
                  float jx = 0.f, jy = 0.f, jz = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
                  if (jv) {
                    float4 a;
                    float2 b;
                    mirror_load(MM, j, a, b);
                    int t = 0;
#pragma unroll
                    for (int q = 0; q < 2 * K; ++q) t += j >= bnd[q] ? 1 : 0;
                    // partner coordinates moved into the frame of cell A's corner
                    jx = a.x + (float)(dxa + t) * wx;
                    jy = a.y + shy;
                    jz = a.z + shz;
                    gx = a.w; gy = b.x; gz = b.y;
                  }
                  for (uint32_t ii = 0; ii < nI; ++ii) {
                    const uint32_t i = i0 + ii;
                    const float4 ia = sa[warp][ii];
                    const float2 ib = sb[warp][ii];
                    const bool valid = jv && (!jown || j > i);
                    const float rx = jx - ia.x, ry = jy - ia.y, rz = jz - ia.z;
                    const float vx = gx - ia.w, vy = gy - ib.x, vz = gz - ib.y;
                    const float R = fmaf(rz, rz, fmaf(ry, ry, rx * rx));
                    const float Bv = fmaf(vz, vz, fmaf(vy, vy, vx * vx));
                    bool cand = valid && !(R > fmaf(c1, Bv, c0));
                    if (__any_sync(0xFFFFFFFFu, cand)) {
                      if (cand) {
                        // full guarded test on the sphere survivors
                        const float A = -fmaf(rz, vz, fmaf(ry, vy, rx * vx));
                        if (A < -ag) cand = false;
                        if (fmaf(-dtf, Bv, A) > tg) cand = false;
                        const float w0 = fmaf(ry, vz, -(rz * vy));
                        const float w1 = fmaf(rz, vx, -(rx * vz));
                        const float w2 = fmaf(rx, vy, -(ry * vx));
                        const float W = fmaf(w2, w2, fmaf(w1, w1, w0 * w0));
                        const float thr = fmaf(d0up, sqrtf(fmaf(Bv, brel, babs)), we);
                        if (W > thr * thr * wrel) cand = false;
                      }
                      warp_emit(we_, s, lane, cand, i, j);
                    }
                  }
                }
              }
            }
          }
        }
      }
    }
    warp_flush(we_, s, lane);
    if (lane == 0 && tests) atomicAdd(&s.d.pair_tests, tests);
  }
}

// --------------------------------------------------------------------------- //
// Binary32 warp-per-cell search, unrolled.  The particles i of cell A are staged as
// structure-of-arrays in shared memory, padded to a multiple of 4 with a sentinel
// position (-1e30) that every sphere test rejects; lanes past the end of a partner
// chunk carry the opposite sentinel (+1e30).  Four pairs per lane are tested per
// iteration with one warp vote, so the loop body is pure arithmetic plus four
// 16-byte shared-memory broadcasts.
struct Guard32 {
  float c0, c1, ag, tg, dtf, d0up, brel, babs, we, wrel;
};

// exact guarded test of one pair on the sphere survivors (rare path)
__device__ __forceinline__ bool full_test32(const Guard32& q, float rx, float ry, float rz,
                                            float vx, float vy, float vz, float Bv) {
  const float A = -fmaf(rz, vz, fmaf(ry, vy, rx * vx));
  if (A < -q.ag) return false;
  if (fmaf(-q.dtf, Bv, A) > q.tg) return false;
  const float w0 = fmaf(ry, vz, -(rz * vy));
  const float w1 = fmaf(rz, vx, -(rx * vz));
  const float w2 = fmaf(rx, vy, -(ry * vx));
  const float W = fmaf(w2, w2, fmaf(w1, w1, w0 * w0));
  const float thr = fmaf(q.d0up, sqrtf(fmaf(Bv, q.brel, q.babs)), q.we);
  return !(W > thr * thr * q.wrel);
}

// The same test behind a real call: inlined, the compiler predicates it into every
// lane's instruction stream (about 30 instructions per pair although only the rare
// sphere survivors need it); as a call it issues only when some lane of the warp
// takes the branch.
__device__ __noinline__ bool full_test32_call(const Guard32& q, float rx, float ry, float rz,
                                              float vx, float vy, float vz, float Bv) {
  return full_test32(q, rx, ry, rz, vx, vy, vz, Bv);
}

// Emission from divergent lanes: a shared-memory counter per warp; entries that do
// not fit in the warp's buffer go straight to the global list.
__device__ __forceinline__ void emit_lane(uint2* buf, uint32_t* count, SimDev& s, uint32_t i,
                                          uint32_t j) {
  uint32_t pos = atomicAdd(count, 1u);
  if (pos < (uint32_t)kWarpBuf) {
    buf[pos] = make_uint2(i, j);
  } else {
    uint32_t g = atomicAdd(&s.d.n_raw, 1u);
    if (g < s.edge_cap) s.edge[g] = make_uint2(i, j);
    else atomicOr(&s.d.status, ST_EDGE_OVERFLOW);
  }
}

// warp-uniform: move the buffered pairs to the global list
__device__ __forceinline__ void flush_lanes(uint2* buf, uint32_t* count, SimDev& s, uint32_t lane) {
  __syncwarp();
  uint32_t c = *count;
  c = c < (uint32_t)kWarpBuf ? c : (uint32_t)kWarpBuf;
  if (c) {
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(&s.d.n_raw, c);
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    for (uint32_t k = lane; k < c; k += 32) {
      uint32_t g = base + k;
      if (g < s.edge_cap) s.edge[g] = buf[k];
      else atomicOr(&s.d.status, ST_EDGE_OVERFLOW);
    }
  }
  __syncwarp();
  if (lane == 0) *count = 0;
  __syncwarp();
}

template <bool OWN>
__device__ __forceinline__ void cell32_sweep(const float* __restrict__ si, uint32_t nI4, uint32_t i0,
                                             float jx, float jy, float jz, float gx, float gy,
                                             float gz, uint32_t j, bool jown, float c0, float c1,
                                             const Guard32& q, uint2* buf, uint32_t* count,
                                             SimDev& s) {
  const float* sx = si;
  const float* sy = si + 1 * 64;
  const float* sz = si + 2 * 64;
  const float* su = si + 3 * 64;
  const float* sv = si + 4 * 64;
  const float* sw = si + 5 * 64;
  // the four own particles of an iteration as two packed pairs (adjacent in shared
  // memory), the lane's partner broadcast to both halves
  const f32x2 JX = pack2(jx, jx), JY = pack2(jy, jy), JZ = pack2(jz, jz);
  const f32x2 GX = pack2(gx, gx), GY = pack2(gy, gy), GZ = pack2(gz, gz);
  const f32x2 C0 = pack2(c0, c0), C1 = pack2(c1, c1);
  for (uint32_t ii = 0; ii < nI4; ii += 4) {
    const ulonglong2 X = *reinterpret_cast<const ulonglong2*>(sx + ii);
    const ulonglong2 Y = *reinterpret_cast<const ulonglong2*>(sy + ii);
    const ulonglong2 Z = *reinterpret_cast<const ulonglong2*>(sz + ii);
    const ulonglong2 U = *reinterpret_cast<const ulonglong2*>(su + ii);
    const ulonglong2 V = *reinterpret_cast<const ulonglong2*>(sv + ii);
    const ulonglong2 W = *reinterpret_cast<const ulonglong2*>(sw + ii);
    unsigned mask = 0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const f32x2 rx = sub2(JX, h ? X.y : X.x), ry = sub2(JY, h ? Y.y : Y.x), rz = sub2(JZ, h ? Z.y : Z.x);
      const f32x2 vx = sub2(GX, h ? U.y : U.x), vy = sub2(GY, h ? V.y : V.x), vz = sub2(GZ, h ? W.y : W.x);
      const f32x2 R = fma2(rz, rz, fma2(ry, ry, mul2(rx, rx)));
      const f32x2 Bv = fma2(vz, vz, fma2(vy, vy, mul2(vx, vx)));
      float R0, R1, T0, T1;
      unpack2(R, R0, R1);
      unpack2(fma2(C1, Bv, C0), T0, T1);
      bool c_0 = R0 <= T0, c_1 = R1 <= T1;
      if (OWN) {
        c_0 = c_0 && (!jown || j > i0 + ii + (uint32_t)(2 * h));
        c_1 = c_1 && (!jown || j > i0 + ii + (uint32_t)(2 * h + 1));
      }
      mask |= (c_0 ? (1u << (2 * h)) : 0u) | (c_1 ? (2u << (2 * h)) : 0u);
    }
    if (mask) {
      // rare and divergent: only the lanes with sphere survivors run the full test
      do {
        const int u = __ffs(mask) - 1;
        mask &= mask - 1;
        const uint32_t t = ii + (uint32_t)u;
        const float rx = jx - sx[t], ry = jy - sy[t], rz = jz - sz[t];
        const float vx = gx - su[t], vy = gy - sv[t], vz = gz - sw[t];
        const float Bv = fmaf(vz, vz, fmaf(vy, vy, vx * vx));
        if (full_test32(q, rx, ry, rz, vx, vy, vz, Bv)) emit_lane(buf, count, s, i0 + t, j);
      } while (mask);
    }
  }
}

template <int K>
__global__ void __launch_bounds__(kCellWarps * 32, 3) k_search_cell32(Batch B) {
  constexpr int ICAP = 64;
  __shared__ __align__(16) float si[kCellWarps][6 * ICAP];
  __shared__ uint2 wbuf[kCellWarps][kWarpBuf];
  __shared__ uint32_t wcount[kCellWarps];
  __shared__ Guard32 sq;
  const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
  const uint32_t gwarp = blockIdx.x * kCellWarps + warp, nwarps = gridDim.x * kCellWarps;

  // The cells of the batch's simulations are dealt to the warps as one sequence (see
  // k_search_cell: the dealing decides on launch-fixed fields only).
  uint32_t base = 0;
  for (int k = 0; k < B.nsims; ++k) {
    SimDev& s = *B.sims[k];
    if (!sim_scheduled(s) || s.d.grid.mode != KMC_SEARCH_CELL) continue;
    const uint32_t first = (gwarp + nwarps - base) % nwarps;
    base = (base + s.d.grid.nkeys % nwarps) % nwarps;
    // every warp is done with the previous simulation's constants; the status word can
    // change while the search runs, so the block takes one answer
    if (!__syncthreads_and(sim_active(s))) continue;
    if (threadIdx.x == 0) {
      const Grid& G0 = s.d.grid;
      sq.c0 = G0.s_c0; sq.c1 = G0.s_c1; sq.ag = G0.a_g; sq.tg = G0.t_g; sq.dtf = G0.dtf;
      sq.d0up = G0.d0up; sq.brel = G0.b_rel; sq.babs = G0.b_abs; sq.we = G0.w_e; sq.wrel = G0.w_rel;
    }
    if (lane == 0) wcount[warp] = 0;
    __syncthreads();
    const Grid& G = s.d.grid;
    const int nx = G.nc[0], ny = G.nc[1], nz = G.nc[2];
    const int Kx = nx == 1 ? 0 : K, Ky = ny == 1 ? 0 : K, Kz = nz == 1 ? 0 : K;
    const bool px = s.bc[0] == KMC_PERIODIC, py = s.bc[1] == KMC_PERIODIC,
               pz = s.bc[2] == KMC_PERIODIC;
    const uint32_t nkeys = G.nkeys;
    const uint32_t* __restrict__ cs = s.cell_start;
    const float Lx = G.Lf[0], Ly = G.Lf[1], Lz = G.Lf[2];
    const float c0 = G.s_c0, c1 = G.s_c1;
    const float4* __restrict__ MM = s.mir;
    float* my = si[warp];
    uint2* buf = wbuf[warp];
    uint32_t* cnt = &wcount[warp];
    unsigned long long tests = 0;

    for (uint32_t key = first; key < nkeys; key += nwarps) {
      const uint32_t startA = __ldg(cs + key), endA = __ldg(cs + key + 1);
      if (startA == endA) continue;
      int cx, cy, cz;
      key_decode(G, key, cx, cy, cz);
      for (uint32_t i0 = startA; i0 < endA; i0 += ICAP) {
        const uint32_t nI = endA - i0 < (uint32_t)ICAP ? endA - i0 : (uint32_t)ICAP;
        const uint32_t nI4 = (nI + 3u) & ~3u;
        __syncwarp();
        for (uint32_t t = lane; t < nI4; t += 32) {
          if (t < nI) {
            float4 a;
            float2 b;
            mirror_load(MM, i0 + t, a, b);
            my[t] = a.x; my[ICAP + t] = a.y; my[2 * ICAP + t] = a.z;
            my[3 * ICAP + t] = a.w; my[4 * ICAP + t] = b.x; my[5 * ICAP + t] = b.y;
          } else {
            my[t] = -1e30f; my[ICAP + t] = 0.f; my[2 * ICAP + t] = 0.f;
            my[3 * ICAP + t] = 0.f; my[4 * ICAP + t] = 0.f; my[5 * ICAP + t] = 0.f;
          }
        }
        __syncwarp();
        for (int dz = 0; dz <= Kz; ++dz) {
          int qz = cz + dz, wrz = 0;
          if (qz >= nz) {
            if (!pz) break;
            qz -= nz;
            wrz = 1;
          }
          for (int dy = (dz == 0 ? 0 : -Ky); dy <= Ky; ++dy) {
            int qy = cy + dy, wry = 0;
            if (qy < 0) {
              if (!py) continue;
              qy += ny;
              wry = -1;
            } else if (qy >= ny) {
              if (!py) continue;
              qy -= ny;
              wry = 1;
            }
            const uint32_t colbase = col_code(G, (uint32_t)qy, (uint32_t)qz) * (uint32_t)nx;
            const bool own_col = dz == 0 && dy == 0;
            // image shifts of partners reached across a periodic boundary
            const float shy = (float)wry * Ly, shz = (float)wrz * Lz;
            int dx = own_col ? 0 : -Kx;
            while (dx <= Kx) {
              const int q0 = cx + dx;
              const int region = q0 < 0 ? -1 : (q0 >= nx ? 1 : 0);
              if (region != 0 && !px) { ++dx; continue; }
              const int qx = q0 - region * nx;
              int m = 1;
              while (dx + m <= Kx) {
                const int q2 = cx + dx + m;
                const int r2 = q2 < 0 ? -1 : (q2 >= nx ? 1 : 0);
                if (r2 != region) break;
                ++m;
              }
              const int dxa = dx;
              dx += m;
              const uint32_t jbeg = __ldg(cs + colbase + qx), jend = __ldg(cs + colbase + qx + m);
              if (jbeg == jend) continue;
              const float shx = (float)region * Lx;
              const bool has_own = own_col && dxa <= 0 && dxa + m > 0;
              if (lane == 0) {
                uint64_t len = jend - jbeg;
                if (has_own) {
                  uint64_t nA = endA - startA;
                  uint64_t inc = (uint64_t)nI * (endA - i0 - 1) - (uint64_t)nI * (nI - 1) / 2;
                  tests += (uint64_t)nI * (len - nA) + inc;
                } else {
                  tests += (uint64_t)nI * len;
                }
              }
              for (uint32_t cb = jbeg; cb < jend; cb += 32) {
                const uint32_t j = cb + lane;
                float jx = 1e30f, jy = 0.f, jz = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
                if (j < jend) {
                  float4 a;
                  float2 b;
                  mirror_load(MM, j, a, b);
                  jx = a.x + shx;
                  jy = a.y + shy;
                  jz = a.z + shz;
                  gx = a.w; gy = b.x; gz = b.y;
                }
                if (has_own) {
                  const bool jown = j >= startA && j < endA;
                  cell32_sweep<true>(my, nI4, i0, jx, jy, jz, gx, gy, gz, j, jown, c0, c1, sq, buf, cnt, s);
                } else {
                  cell32_sweep<false>(my, nI4, i0, jx, jy, jz, gx, gy, gz, j, false, c0, c1, sq, buf, cnt, s);
                }
                __syncwarp();
                if (*cnt >= (uint32_t)(kWarpBuf / 2)) flush_lanes(buf, cnt, s, lane);
              }
            }
          }
        }
      }
    }
    flush_lanes(buf, cnt, s, lane);
    if (lane == 0 && tests) atomicAdd(&s.d.pair_tests, tests);
  }
}

// --------------------------------------------------------------------------- //
// Row search (binary32), for sparsely filled cells.  One lane per slow particle i,
// 32 consecutive particles (cell order) per warp.  With the mirror in box
// coordinates a stencil row -- the 2K+1 cells along x of one forward (y, z) column,
// or in i's own column the cells from its own on with only j > i -- is one
// contiguous range of partners; a row that crosses a periodic x boundary splits
// into two pieces, the far one seen through its image.  Each lane lists its
// non-empty pieces in shared memory and then walks them as one sequence of tests,
// one test per iteration, so no per-cell loop and no per-cell shift remain.  The
// warp runs as many iterations as its busiest lane needs.  Rows split only on a
// periodic x axis (PX); without one the piece lists take half the shared memory,
// which leaves more of the SM's L1 to cache the partner records.
template <int K, bool PX>
struct RowLayout {
  static constexpr int kCols = 1 + K + K * (2 * K + 1);  // own column + forward columns
  static constexpr int kPieces = PX ? 2 * kCols : kCols; // a row splits at most once
  static constexpr int kWarps = kTile / 32;
  static constexpr size_t kPieceBytes = (size_t)kWarps * kPieces * 32 * sizeof(uint2);
  static constexpr size_t kCodeBytes = (size_t)kWarps * kPieces * 32;
  static constexpr size_t kBytes = kPieceBytes + kCodeBytes + (size_t)kWarps * kWarpBuf * sizeof(uint2);
};

// image flags of a piece: bit 0 / 1 = seen at +L / -L along x, bits 2-3 y, bits 4-5 z
__device__ __forceinline__ uint32_t image_code(int wx, int wy, int wz) {
  return (uint32_t)(wx > 0) | ((uint32_t)(wx < 0) << 1) | ((uint32_t)(wy > 0) << 2) |
         ((uint32_t)(wy < 0) << 3) | ((uint32_t)(wz > 0) << 4) | ((uint32_t)(wz < 0) << 5);
}

template <int K, bool PX>
__global__ void __launch_bounds__(kTile, 4) k_search_rows32(Batch B) {
  using RL = RowLayout<K, PX>;
  constexpr int NP = RL::kPieces;
  extern __shared__ __align__(16) unsigned char rows_smem[];
  __shared__ uint32_t wcount[RL::kWarps];
  __shared__ Guard32 sq;
  __shared__ float4 shift_tab[64];  // image shift (x, y, z) of each image code
  __shared__ int s_live;            // the current simulation runs this step
  // grid-stride over tiles of kTile particles: the kernel is launched every step on an
  // occupancy-sized grid and exits at once when the step runs another search
  if (!batch_uses(B, KMC_SEARCH_ROW)) return;
  const uint32_t ntiles = B.ptile[B.nsims];
  int kcur = -1;  // simulation whose constants the shared tables hold
  // The warp's pair tests and emitted pairs go to the simulation's counters only when
  // the simulation changes, the staging buffer is half full, or at the end: per-tile
  // atomics on these two counters from every warp serialise in L2.  The running
  // counts live in shared memory (registers are the row search's limit).
  __shared__ unsigned long long wtests[RL::kWarps];
  auto warp_buf = [&]() {
    return reinterpret_cast<uint2*>(rows_smem + RL::kPieceBytes + RL::kCodeBytes) +
           (size_t)(threadIdx.x >> 5) * kWarpBuf;
  };
  auto warp_flush = [&](SimDev& f) {
    const uint32_t w = threadIdx.x >> 5, l = threadIdx.x & 31u;
    flush_lanes(warp_buf(), &wcount[w], f, l);
    if (l == 0 && wtests[w]) atomicAdd(&f.d.pair_tests, wtests[w]);
    if (l == 0) wtests[w] = 0;
    __syncwarp();
  };
  if ((threadIdx.x & 31u) == 0) {
    wcount[threadIdx.x >> 5] = 0;
    wtests[threadIdx.x >> 5] = 0;
  }
  __syncwarp();
  for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int k = find_sim(B.ptile, B.nsims, tile);
    SimDev& s = *B.sims[k];
    // launch-fixed fields only: the barriers below depend on it
    if (!sim_scheduled(s) || s.d.grid.mode != KMC_SEARCH_ROW || (s.bc[0] == KMC_PERIODIC) != PX)
      continue;
    const Grid& g = s.d.grid;
    // The shared constants change only with the simulation (block-uniform: every warp
    // walks the same tiles), so the warps of a block need not wait for each other at
    // every tile: each runs on to its part of the next tile.
    if (k != kcur) {
      if (kcur >= 0) warp_flush(*B.sims[kcur]);  // staged pairs and counts of the last one
      __syncthreads();  // every warp is done with the previous simulation's constants
      if (threadIdx.x == 0) {
        sq.c0 = g.s_c0; sq.c1 = g.s_c1; sq.ag = g.a_g; sq.tg = g.t_g; sq.dtf = g.dtf;
        sq.d0up = g.d0up; sq.brel = g.b_rel; sq.babs = g.b_abs; sq.we = g.w_e; sq.wrel = g.w_rel;
        // the status word, read once per simulation and block (the search itself can set
        // it: a full pair buffer only stops the stores, which are bounds-checked)
        s_live = sim_active(s) ? 1 : 0;
      }
      if (threadIdx.x < 64) {
        const uint32_t c = threadIdx.x;
        const float w0 = (float)((int)(c & 1u) - (int)((c >> 1) & 1u));
        const float w1 = (float)((int)((c >> 2) & 1u) - (int)((c >> 3) & 1u));
        const float w2 = (float)((int)((c >> 4) & 1u) - (int)((c >> 5) & 1u));
        shift_tab[c] = make_float4(w0 * g.Lf[0], w1 * g.Lf[1], w2 * g.Lf[2], 0.f);
      }
      __syncthreads();
      kcur = k;
    }
    if (!s_live) continue;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t nslow = (g.split || s.absorb) ? __ldg(s.cell_start + g.nkeys) : s.n;
    const uint32_t p = (tile - B.ptile[k]) * kTile + threadIdx.x;
    if (p - lane >= nslow) continue;  // the whole warp is past the slow population
    uint2* pc = reinterpret_cast<uint2*>(rows_smem) + (size_t)warp * NP * 32;
    uint8_t* cd = rows_smem + RL::kPieceBytes + (size_t)warp * NP * 32;
    uint2* buf = warp_buf();
    uint32_t* cnt = &wcount[warp];

    const bool valid = p < nslow;
    const int nx = g.nc[0], ny = g.nc[1], nz = g.nc[2];
    // along x the grid may have narrower cells under the row search (kx per radius)
    const int Kx = nx == 1 ? 0 : g.kx, Ky = ny == 1 ? 0 : K, Kz = nz == 1 ? 0 : K;
    constexpr bool px = PX;
    const bool py = s.bc[1] == KMC_PERIODIC, pz = s.bc[2] == KMC_PERIODIC;
    // one-cell periodic axes need the minimum image explicitly
    const bool cp0 = nx == 1 && px, cp1 = ny == 1 && py, cp2 = nz == 1 && pz;
    const bool any_cp = cp0 || cp1 || cp2;
    const uint32_t* __restrict__ cs = s.cell_start;
    const float4* __restrict__ MM = s.mir;

    // 1. the lane's non-empty pieces, column by column
    int np = 0;
    uint32_t total = 0, iters = 0;  // tests; iterations of up to two tests of one piece
    Own32 o = {0, 0, 0, 0, 0, 0};
    int cx = 0, cy = 0, cz = 0;
    if (valid) {
      float4 a;
      float2 b;
      mirror_load(MM, p, a, b);
      o = {a.x, a.y, a.z, a.w, b.x, b.y};
      // the particle's cell, recomputed from the mirror as the sort computed it
      cx = cell_coord_f(g, 0, a.x);
      cy = cell_coord_f(g, 1, a.y);
      cz = cell_coord_f(g, 2, a.z);
    }
    // Nearly every warp lies in one (y, z) column (a column holds thousands of
    // particles in cell order).  Then the forward columns are the same for all lanes:
    // lane c works out column c (whether it exists, its key base, its image code)
    // once for the warp.  Lane 0 is valid whenever any lane is.
    const int cy0 = __shfl_sync(0xFFFFFFFFu, cy, 0), cz0 = __shfl_sync(0xFFFFFFFFu, cz, 0);
    const bool uni = __all_sync(0xFFFFFFFFu, !valid || (cy == cy0 && cz == cz0));
    uint32_t ctab = kNone, ctag = 0;
    if (uni && lane < (uint32_t)RL::kCols) {
      const int c = (int)lane;
      const int dz = c <= K ? 0 : 1 + (c - K - 1) / (2 * K + 1);
      const int dy = c == 0 ? 0 : (c <= K ? c : (c - K - 1) % (2 * K + 1) - K);
      int qz = cz0 + dz, wz = 0, qy = cy0 + dy, wy = 0;
      bool ok = !(dz > Kz || dy > Ky || dy < -Ky);
      if (qz >= nz) { ok = ok && pz; qz -= nz; wz = 1; }
      if (qy < 0) { ok = ok && py; qy += ny; wy = -1; }
      else if (qy >= ny) { ok = ok && py; qy -= ny; wy = 1; }
      if (ok) {
        ctab = col_code(g, (uint32_t)qy, (uint32_t)qz) * (uint32_t)nx;
        ctag = (uint32_t)(wy & 3) | ((uint32_t)(wz & 3) << 2);
      }
    }
    {
      // row trimming: the part of each row within the reach of this particle.  A
      // column whose cells lie farther than the reach in (y, z) is skipped; in the
      // others only the cells with x within sqrt(reach^2 - d^2) are kept (d the
      // column's distance in (y, z), taken from the cell edges and rounded down; the
      // x extent rounded up).  Rows that cross a periodic x boundary keep their full
      // length on the crossing side.
      // the reach of this particle: |v_i| from its binary32 velocity (each component
      // within u32 of the binary64 one, the sum of squares within 3 u32, the square
      // root within 3 ulp; the argument kept normal, which only enlarges it) times
      // 1 + 4e-6 bounds |v_i| from above; the products and the square get 1e-6 each.
      // The smaller of this and the common reach holds.
      const float sv2 = fmaxf(fmaf(o.vz, o.vz, fmaf(o.vy, o.vy, o.vx * o.vx)), 1e-30f);
      // (the square root from the approximate reciprocal root: 3 ulp, inside the margin)
      const float si = sv2 * rsqrtf(sv2) * 1.000004f;
      const float Ri = fmaf(si, g.row_b, g.row_a) * 1.000001f;
      const float R2 = fminf(g.row_r2, Ri * Ri * 1.000001f);
      const float eps = g.row_eps, pad = g.row_pad;
      const float wyf = g.wf[1], wzf = g.wf[2], ivx = g.inv_wf[0];
#pragma unroll
      for (int c = 0; c < RL::kCols; ++c) {
        const int dz = c <= K ? 0 : 1 + (c - K - 1) / (2 * K + 1);
        const int dy = c == 0 ? 0 : (c <= K ? c : (c - K - 1) % (2 * K + 1) - K);
        // the column's key base and image flags (warp table, or this lane's own)
        uint32_t colb, wtag;
        if (uni) {
          colb = __shfl_sync(0xFFFFFFFFu, ctab, c);
          wtag = __shfl_sync(0xFFFFFFFFu, ctag, c);
          if (colb == kNone) continue;
        } else {
          if (dz > Kz || dy > Ky || dy < -Ky) continue;
          int qz = cz + dz, wz = 0;
          if (qz >= nz) {
            if (!pz) continue;
            qz -= nz;
            wz = 1;
          }
          int qy = cy + dy, wy = 0;
          if (qy < 0) {
            if (!py) continue;
            qy += ny;
            wy = -1;
          } else if (qy >= ny) {
            if (!py) continue;
            qy -= ny;
            wy = 1;
          }
          colb = col_code(g, (uint32_t)qy, (uint32_t)qz) * (uint32_t)nx;
          wtag = (uint32_t)(wy & 3) | ((uint32_t)(wz & 3) << 2);
        }
        if (!valid) continue;
        const int wy = (wtag & 3u) == 3u ? -1 : (int)(wtag & 3u);
        const int wz = (int)((wtag >> 2) & 3u);
        float d2 = 0.f;
        if (dy != 0) {
          const float e = dy > 0 ? (float)(cy + dy) * wyf - o.oy : o.oy - (float)(cy + dy + 1) * wyf;
          const float el = fmaxf(e - eps, 0.f);
          d2 = el * el;
        }
        if (dz != 0) {  // forward columns only: dz > 0
          const float e = (float)(cz + dz) * wzf - o.oz;
          const float el = fmaxf(e - eps, 0.f);
          d2 = fmaf(el, el, d2);
        }
        d2 *= 0.9999995f;
        if (d2 >= R2) continue;
        // x extent sqrt(R2 - d2) from the approximate reciprocal square root (at most
        // 2 ulp off, 3 ulp with the product), widened by 33 ulp; the argument is kept
        // normal, which only widens it
        const float t2 = fmaxf(R2 - d2, 1e-30f);
        const float ex = fmaf(t2 * rsqrtf(t2), 1.000004f, pad);
        int xa = c == 0 ? cx : cx - Kx, xb = cx + Kx;  // cells of the row, unwrapped
        if (Kx > 0) {
          const int ta = (int)floorf((o.ox - ex) * ivx), tb = (int)floorf((o.ox + ex) * ivx);
          if (ta >= 0 && ta > xa) xa = ta;
          if (tb <= nx - 1 && tb < xb) xb = tb;
          if (xb < xa) continue;
        }
        {
          const int a0 = xa < 0 ? 0 : xa, b0 = xb >= nx ? nx - 1 : xb;
          const uint32_t jb = c == 0 ? p + 1 : __ldg(cs + colb + a0);
          const uint32_t je = __ldg(cs + colb + b0 + 1);
          if (je > jb) {
            pc[np * 32 + lane] = make_uint2(jb, je);
            cd[np * 32 + lane] = (uint8_t)image_code(0, wy, wz);
            ++np;
            total += je - jb;
            iters += ((je + 1u) >> 1) - (jb >> 1);  // pair slots
          }
        }
        if (px && xa < 0) {  // cells [xa + nx, nx) seen through the image at -L
          const uint32_t jb = __ldg(cs + colb + xa + nx), je = __ldg(cs + colb + nx);
          if (je > jb) {
            pc[np * 32 + lane] = make_uint2(jb, je);
            cd[np * 32 + lane] = (uint8_t)image_code(-1, wy, wz);
            ++np;
            total += je - jb;
            iters += ((je + 1u) >> 1) - (jb >> 1);  // pair slots
          }
        }
        if (px && xb >= nx) {  // cells [0, xb - nx] seen through the image at +L
          const uint32_t jb = __ldg(cs + colb), je = __ldg(cs + colb + xb - nx + 1);
          if (je > jb) {
            pc[np * 32 + lane] = make_uint2(jb, je);
            cd[np * 32 + lane] = (uint8_t)image_code(1, wy, wz);
            ++np;
            total += je - jb;
            iters += ((je + 1u) >> 1) - (jb >> 1);  // pair slots
          }
        }
      }
    }

    // 2. walk the pieces in pair slots of the mirror, two tests per iteration (a half
    //    outside the piece masked), the binary32 pre-tests in packed f32x2 arithmetic
    const uint32_t T = __reduce_max_sync(0xFFFFFFFFu, any_cp ? total : iters);
    uint32_t j = 0, je = 0;
    int r = 0;
    float sx = o.ox, sy = o.oy, sz = o.oz;
    if (np > 0) {
      const uint2 q = pc[lane];
      const float4 sh = shift_tab[cd[lane]];
      j = q.x;
      je = q.y;
      sx = o.ox - sh.x;
      sy = o.oy - sh.y;
      sz = o.oz - sh.z;
    }
    const float c0 = g.s_c0, c1 = g.s_c1;
    if (any_cp) {
      // one-cell periodic axes (thin slabs): one test per iteration with the minimum image
      for (uint32_t t = 0; t < T; ++t) {
        if (j < je) {
          float4 a;
          float2 b;
          mirror_load(MM, j, a, b);
          float rx = a.x - sx, ry = a.y - sy, rz = a.z - sz;
          bool keep = false;
          if (cp0) min_image_f(rx, g.halfLf[0], g.Lf[0], g.tief[0], keep);
          if (cp1) min_image_f(ry, g.halfLf[1], g.Lf[1], g.tief[1], keep);
          if (cp2) min_image_f(rz, g.halfLf[2], g.Lf[2], g.tief[2], keep);
          const float gx = a.w - o.vx, gy = b.x - o.vy, gz = b.y - o.vz;
          const float R = fmaf(rz, rz, fmaf(ry, ry, rx * rx));
          const float Bv = fmaf(gz, gz, fmaf(gy, gy, gx * gx));
          if (keep || (R <= fmaf(c1, Bv, c0) && full_test32_call(sq, rx, ry, rz, gx, gy, gz, Bv)))
            emit_lane(buf, cnt, s, p, j);
          if (++j == je && r + 1 < np) {
            ++r;
            const uint2 q = pc[r * 32 + lane];
            const float4 sh = shift_tab[cd[r * 32 + lane]];
            j = q.x;
            je = q.y;
            sx = o.ox - sh.x;
            sy = o.oy - sh.y;
            sz = o.oz - sh.z;
          }
        }
      }
    } else {
      const f32x2 C0 = pack2(c0, c0), C1 = pack2(c1, c1);
      const f32x2 VX = pack2(o.vx, o.vx), VY = pack2(o.vy, o.vy), VZ = pack2(o.vz, o.vz);
      f32x2 SX = pack2(sx, sx), SY = pack2(sy, sy), SZ = pack2(sz, sz);
      // the piece [j, je) in pair slots: slot k holds particles 2k and 2k + 1, three
      // 16-byte loads give each component of both already paired; a half outside the
      // piece (its first slot's lower, its last slot's upper half) is masked
      const ulonglong2* __restrict__ MP = reinterpret_cast<const ulonglong2*>(MM);
      uint32_t k = j >> 1, ke = (je + 1u) >> 1;
      for (uint32_t t = 0; t < T; ++t) {
        if (k < ke) {
          const ulonglong2* rec = MP + 3 * (size_t)k;
          const ulonglong2 Q0 = __ldg(rec), Q1 = __ldg(rec + 1), Q2 = __ldg(rec + 2);
          const f32x2 rx = sub2(Q0.x, SX), ry = sub2(Q0.y, SY), rz = sub2(Q1.x, SZ);
          const f32x2 gx = sub2(Q1.y, VX), gy = sub2(Q2.x, VY), gz = sub2(Q2.y, VZ);
          const f32x2 R = fma2(rz, rz, fma2(ry, ry, mul2(rx, rx)));
          const f32x2 Bv = fma2(gz, gz, fma2(gy, gy, mul2(gx, gx)));
          const f32x2 bound = fma2(C1, Bv, C0);
          float R0, R1, T0, T1;
          unpack2(R, R0, R1);
          unpack2(bound, T0, T1);
          const uint32_t j0 = 2u * k;
          const bool s0 = j0 >= j && R0 <= T0, s1 = j0 + 1u < je && R1 <= T1;
          if (s0 || s1) {  // rare: a sphere survivor
            float rx0, rx1, ry0, ry1, rz0, rz1, gx0, gx1, gy0, gy1, gz0, gz1, B0, B1;
            unpack2(rx, rx0, rx1);
            unpack2(ry, ry0, ry1);
            unpack2(rz, rz0, rz1);
            unpack2(gx, gx0, gx1);
            unpack2(gy, gy0, gy1);
            unpack2(gz, gz0, gz1);
            unpack2(Bv, B0, B1);
            if (s0 && full_test32_call(sq, rx0, ry0, rz0, gx0, gy0, gz0, B0))
              emit_lane(buf, cnt, s, p, j0);
            if (s1 && full_test32_call(sq, rx1, ry1, rz1, gx1, gy1, gz1, B1))
              emit_lane(buf, cnt, s, p, j0 + 1u);
          }
          if (++k == ke && r + 1 < np) {
            ++r;
            const uint2 q = pc[r * 32 + lane];
            const float4 sh = shift_tab[cd[r * 32 + lane]];
            j = q.x;
            je = q.y;
            k = j >> 1;
            ke = (je + 1u) >> 1;
            SX = pack2(o.ox - sh.x, o.ox - sh.x);
            SY = pack2(o.oy - sh.y, o.oy - sh.y);
            SZ = pack2(o.oz - sh.z, o.oz - sh.z);
          }
        }
      }
    }
    __syncwarp();
    if (*cnt >= (uint32_t)(kWarpBuf / 2)) flush_lanes(buf, cnt, s, lane);
    unsigned long long tests = total;
    for (int off = 16; off > 0; off >>= 1) tests += __shfl_down_sync(0xFFFFFFFFu, tests, off);
    if (lane == 0) wtests[warp] += tests;
  }
  if (kcur >= 0) warp_flush(*B.sims[kcur]);
}


// --------------------------------------------------------------------------- //
// Fast particles of the speed split: one warp per fast particle p, searching cfast
// cells on each side over both populations -- every slow particle, and the fast
// particles j > p (each fast-fast pair once).  The stencil is walked by (y, z)
// columns: the lanes take one column each, trim its row of cells along x to p's
// reach (as the row search does) and read its slow and fast partner ranges -- a row
// is contiguous in the cell order, so a column costs four loads of the cell table
// whatever its length.  A warp prefix sum over the lanes' test counts then deals the
// tests of 32 columns out to the lanes, so every lane tests a pair in every
// iteration whatever the occupancies.  The pair tests are those of the
// thread-per-particle search.
template <int PREC>
__global__ void __launch_bounds__(kCellWarps * 32, 4) k_search_fast(Batch B) {
  __shared__ uint2 wbuf[kCellWarps][kWarpBuf];
  __shared__ uint32_t wcount[kCellWarps];
  // per column of the current batch (one per lane): its first test within the batch,
  // and up to four partner ranges (slow and fast population, each in at most two x
  // segments on a periodic x axis): first partner, length, image flags of the segment
  constexpr int kFastPieces = 4;
  __shared__ uint32_t sjb[kCellWarps][kFastPieces][32], sln[kCellWarps][kFastPieces][32];
  __shared__ uint8_t scd[kCellWarps][kFastPieces][32];
  // the batch's pieces laid end to end (column by column): first test, first partner,
  // image flags
  __shared__ uint32_t fst[kCellWarps][kFastPieces * 32], fjb[kCellWarps][kFastPieces * 32];
  __shared__ uint8_t fcd[kCellWarps][kFastPieces * 32];
  // grid-stride over tiles (an occupancy-sized grid); the warps of tile t take the
  // fast particles f = 8 (t - first tile) + warp, stepping by 8 tiles per simulation
  if (!batch_uses(B, -1)) return;
  const uint32_t ntiles = B.ptile[B.nsims];
  for (uint32_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int k = find_sim(B.ptile, B.nsims, tile);
    SimDev& s = *B.sims[k];
    // launch-fixed fields first; the status word (the search itself can set it) as one
    // answer per warp
    if (!sim_scheduled(s) || !s.d.grid.split) continue;
    if (!__all_sync(0xFFFFFFFFu, sim_active(s))) continue;
    const Grid& g = s.d.grid;
    const uint32_t* __restrict__ cs = s.cell_start;
    const uint32_t nk = g.nkeys;
    const uint32_t n = __ldg(cs + 2 * nk);  // end of the fast keys (n without absorption)
    const uint32_t nslow = __ldg(cs + nk);
    const uint32_t nfast = n - nslow;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t blk = tile - B.ptile[k];
    // tiles past the fast population have nothing to do (no block-wide barrier below)
    if (blk * kCellWarps >= nfast) continue;
    const uint32_t wstride = (B.ptile[k + 1] - B.ptile[k]) * kCellWarps;
    uint2* buf = wbuf[warp];
    uint32_t* cnt = &wcount[warp];
    if (lane == 0) *cnt = 0;
    __syncwarp();

    const int cur = s.d.parity ^ 1;
    const int nx = g.nc[0], ny = g.nc[1], nz = g.nc[2];
    const int Cx = g.cfast[0], Cy = g.cfast[1], Cz = g.cfast[2];
    const bool px = s.bc[0] == KMC_PERIODIC, py = s.bc[1] == KMC_PERIODIC,
               pz = s.bc[2] == KMC_PERIODIC;
    const double* __restrict__ X0 = s.x[cur][0];
    const double* __restrict__ X1 = s.x[cur][1];
    const double* __restrict__ X2 = s.x[cur][2];
    const double* __restrict__ V0 = s.v[cur][0];
    const double* __restrict__ V1 = s.v[cur][1];
    const double* __restrict__ V2 = s.v[cur][2];
    const float4* __restrict__ MM = s.mir;
    const double L0 = s.box[0], L1 = s.box[1], L2 = s.box[2];
    Guard32 q;
    q.c0 = g.s_c0; q.c1 = g.s_c1; q.ag = g.a_g; q.tg = g.t_g; q.dtf = g.dtf;
    q.d0up = g.d0up; q.brel = g.b_rel; q.babs = g.b_abs; q.we = g.w_e; q.wrel = g.w_rel;
    const float Lf0 = g.Lf[0], Lf1 = g.Lf[1], Lf2 = g.Lf[2];
    unsigned long long tests = 0;

    for (uint32_t f = blk * kCellWarps + warp; f < nfast; f += wstride) {
      const uint32_t p = nslow + f;
      // the particle's cell, recomputed as the sort computed it
      const int cx = cell_coord(g, 0, X0[p]), cy = cell_coord(g, 1, X1[p]), cz = cell_coord(g, 2, X2[p]);
      double xo[3] = {0, 0, 0}, vo[3] = {0, 0, 0};
      Own32 o32 = {0, 0, 0, 0, 0, 0};
      if (PREC == KMC_FP64) {
        xo[0] = X0[p]; xo[1] = X1[p]; xo[2] = X2[p];
        vo[0] = V0[p]; vo[1] = V1[p]; vo[2] = V2[p];
        // binary32 position and velocity for the cell trimming only
        o32 = {d2f_rn(xo[0]), d2f_rn(xo[1]), d2f_rn(xo[2]), d2f_rn(vo[0]), d2f_rn(vo[1]),
               d2f_rn(vo[2])};
      } else {
        float4 a;
        float2 b;
        mirror_load(MM, p, a, b);
        o32 = {a.x, a.y, a.z, a.w, b.x, b.y};
      }
      // cell trimming: a pair (p, j) has |r| < d0 + (|v_p| + |v_j|) dt <= d0 + (|v_p| + V) dt,
      // so a stencil cell farther than that from p holds no candidate.  |v_p| from the
      // binary32 velocity times 1 + 2e-6 bounds it from above; the distance to a cell is
      // taken from its edges less eps (the binary32 error of a coordinate against a
      // cell edge), rounded down.
      const float sp = sqrtf(fmaf(o32.vz, o32.vz, fmaf(o32.vy, o32.vy, o32.vx * o32.vx))) * 1.000002f;
      const float Rp = fmaf(sp, g.row_b, g.fast_a) * 1.000001f;
      const float Rp2 = Rp * Rp * 1.000001f;
      const float teps = g.row_eps;
      const int Wy = 2 * Cy + 1;
      const int ncol = Wy * (2 * Cz + 1);
      const float ivx = g.inv_wf[0], pad = g.row_pad;
      for (int c0 = 0; c0 < ncol; c0 += 32) {
        // this lane's column: its row of cells trimmed to p's reach, split at a periodic
        // x boundary, and the slow and fast partner ranges of each segment
        const int c = c0 + (int)lane;
        int np = 0;
        uint32_t tot = 0;
        if (c < ncol) {
          const int dz = c / Wy - Cz;
          const int dy = c - (dz + Cz) * Wy - Cy;
          int qy = cy + dy, qz = cz + dz;
          const int wy = qy < 0 ? -1 : (qy >= ny ? 1 : 0);
          const int wz = qz < 0 ? -1 : (qz >= nz ? 1 : 0);
          bool ok = (wy == 0 || py) && (wz == 0 || pz);
          // squared distance from p to the column (unwrapped: the image frame of p)
          float d2 = 0.f;
          if (dy != 0 && ny > 1) {
            const float e = dy > 0 ? (float)(cy + dy) * g.wf[1] - o32.oy
                                   : o32.oy - (float)(cy + dy + 1) * g.wf[1];
            const float el = fmaxf(e - teps, 0.f);
            d2 = el * el;
          }
          if (dz != 0 && nz > 1) {
            const float e = dz > 0 ? (float)(cz + dz) * g.wf[2] - o32.oz
                                   : o32.oz - (float)(cz + dz + 1) * g.wf[2];
            const float el = fmaxf(e - teps, 0.f);
            d2 = fmaf(el, el, d2);
          }
          if (d2 * 0.9999995f >= Rp2) ok = false;
          if (ok) {
            qy -= wy * ny;
            qz -= wz * nz;
            const uint32_t colb = col_code(g, (uint32_t)qy, (uint32_t)qz) * (uint32_t)nx;
            // the cells along x within the reach: sqrt(Rp2 - d2) from the approximate
            // reciprocal square root (3 ulp), widened by 33 ulp and the coordinate error
            int xa = 0, xb = 0;
            if (nx > 1) {
              const float t2 = fmaxf(Rp2 - d2, 1e-30f);
              const float ex = fmaf(t2 * rsqrtf(t2), 1.000004f, pad);
              const int ta = (int)floorf((o32.ox - ex) * ivx), tb = (int)floorf((o32.ox + ex) * ivx);
              xa = ta > cx - Cx ? ta : cx - Cx;
              xb = tb < cx + Cx ? tb : cx + Cx;
              if (!px) {
                xa = xa < 0 ? 0 : xa;
                xb = xb > nx - 1 ? nx - 1 : xb;
              }
            }
            const uint32_t code_yz = (uint32_t)((wy > 0) ? 4 : 0) | (uint32_t)((wy < 0) ? 8 : 0) |
                                     (uint32_t)((wz > 0) ? 16 : 0) | (uint32_t)((wz < 0) ? 32 : 0);
            // x segments: [xa, xb] within [0, nx), and the part past a periodic boundary
            auto segment = [&](int a0, int b0, uint32_t code) {
              const uint32_t k0 = colb + (uint32_t)a0, k1 = colb + (uint32_t)b0 + 1u;
              const uint32_t sb0 = __ldg(cs + k0), se0 = __ldg(cs + k1);
              uint32_t sb1 = __ldg(cs + nk + k0);
              const uint32_t se1 = __ldg(cs + nk + k1);
              if (sb1 <= p) sb1 = p + 1;  // fast partners j > p only
              if (se0 > sb0) {
                sjb[warp][np][lane] = sb0; sln[warp][np][lane] = se0 - sb0; scd[warp][np][lane] = (uint8_t)code;
                tot += se0 - sb0;
                ++np;
              }
              if (se1 > sb1) {
                sjb[warp][np][lane] = sb1; sln[warp][np][lane] = se1 - sb1; scd[warp][np][lane] = (uint8_t)code;
                tot += se1 - sb1;
                ++np;
              }
            };
            if (xb >= xa) {
              const int a0 = xa < 0 ? 0 : xa, b0 = xb > nx - 1 ? nx - 1 : xb;
              if (b0 >= a0) segment(a0, b0, code_yz);
              if (xa < 0) segment(xa + nx, nx - 1, code_yz | 2u);            // seen at -L
              else if (xb > nx - 1) segment(0, xb - nx, code_yz | 1u);      // seen at +L
            }
          }
        }
        // lay the batch's pieces end to end: piece base and first test of each column
        uint32_t incl = tot, pincl = (uint32_t)np;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
          const uint32_t z = __shfl_up_sync(0xFFFFFFFFu, pincl, o);
          if (lane >= (uint32_t)o) {
            incl += y;
            pincl += z;
          }
        }
        const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
        const uint32_t npw = __shfl_sync(0xFFFFFFFFu, pincl, 31);
        tests += tot;
        {
          uint32_t at = pincl - (uint32_t)np, st = incl - tot;
          for (int r = 0; r < np; ++r) {
            fst[warp][at] = st;
            fjb[warp][at] = sjb[warp][r][lane];
            fcd[warp][at] = scd[warp][r][lane];
            st += sln[warp][r][lane];
            ++at;
          }
        }
        __syncwarp();
        // walk the batch's tests 32 at a time: lane l takes test kb + l.  P is the piece
        // holding test kb; the pieces starting inside the pass (at most 31, each
        // non-empty) are among P + 1 .. P + 31 and mark their first test in one OR
        uint32_t P = 0;
        for (uint32_t kb = 0; kb < total; kb += 32) {
          const uint32_t qp = P + lane;
          const uint32_t st = qp < npw ? fst[warp][qp] : 0xFFFFFFFFu;
          const uint32_t bit = (st >= kb && st - kb < 32u) ? 1u << (st - kb) : 0u;
          const uint32_t mask = __reduce_or_sync(0xFFFFFFFFu, bit);
          const uint32_t before = __shfl_sync(0xFFFFFFFFu, st < kb ? 1u : 0u, 0);
          const uint32_t pi = P - 1u + before + __popc(mask & (0xFFFFFFFFu >> (31u - lane)));
          const uint32_t qi = kb + lane;
          if (qi < total) {
            const uint32_t j = fjb[warp][pi] + (qi - fst[warp][pi]);
            const uint32_t d = fcd[warp][pi];
            bool emit;
            if (PREC == KMC_FP64) {
              double r0 = dsub(__ldg(X0 + j), xo[0]);
              double r1 = dsub(__ldg(X1 + j), xo[1]);
              double r2 = dsub(__ldg(X2 + j), xo[2]);
              if (px) { if (r0 > 0.5 * L0) r0 = dsub(r0, L0); else if (r0 < -0.5 * L0) r0 = dadd(r0, L0); }
              if (py) { if (r1 > 0.5 * L1) r1 = dsub(r1, L1); else if (r1 < -0.5 * L1) r1 = dadd(r1, L1); }
              if (pz) { if (r2 > 0.5 * L2) r2 = dsub(r2, L2); else if (r2 < -0.5 * L2) r2 = dadd(r2, L2); }
              const double g0 = dsub(__ldg(V0 + j), vo[0]);
              const double g1 = dsub(__ldg(V1 + j), vo[1]);
              const double g2 = dsub(__ldg(V2 + j), vo[2]);
              const double R = dadd(dadd(dmul(r0, r0), dmul(r1, r1)), dmul(r2, r2));
              const double Bv = dadd(dadd(dmul(g0, g0), dmul(g1, g1)), dmul(g2, g2));
              emit = !(Bv >= 0x1p-900 && R > dadd(g.c0, dmul(g.c1, Bv)));
              if (emit && Bv >= 0x1p-900 &&
                  f64_cannot_approach(dadd(dadd(dmul(r0, g0), dmul(r1, g1)), dmul(r2, g2)), Bv, s.dt))
                emit = false;
            } else {
              // own coordinates moved by the image shift (j seen at x_j + w L)
              const float wxf = (float)((int)(d & 1u) - (int)((d >> 1) & 1u));
              const float wyf = (float)((int)((d >> 2) & 1u) - (int)((d >> 3) & 1u));
              const float wzf = (float)((int)((d >> 4) & 1u) - (int)((d >> 5) & 1u));
              const float sx = o32.ox - wxf * Lf0;
              const float sy = o32.oy - wyf * Lf1;
              const float sz = o32.oz - wzf * Lf2;
              float4 a;
              float2 b;
              mirror_load(MM, j, a, b);
              const float rx = a.x - sx, ry = a.y - sy, rz = a.z - sz;
              const float gx = a.w - o32.vx, gy = b.x - o32.vy, gz = b.y - o32.vz;
              const float R = fmaf(rz, rz, fmaf(ry, ry, rx * rx));
              const float Bv = fmaf(gz, gz, fmaf(gy, gy, gx * gx));
              emit = R <= fmaf(q.c1, Bv, q.c0) && full_test32(q, rx, ry, rz, gx, gy, gz, Bv);
            }
            if (emit) emit_lane(buf, cnt, s, p, j);
          }
          // the next pass starts in lane 31's piece or in the one after it
          uint32_t nextP = 0;
          if (lane == 31u) {
            const uint32_t end = pi + 1u < npw ? fst[warp][pi + 1u] : total;
            nextP = kb + 32u >= end ? pi + 1u : pi;
          }
          P = __shfl_sync(0xFFFFFFFFu, nextP, 31);
          __syncwarp();
          if (*cnt >= (uint32_t)(kWarpBuf / 2)) flush_lanes(buf, cnt, s, lane);
        }
        __syncwarp();
      }
    }
    flush_lanes(buf, cnt, s, lane);
    for (int o = 16; o > 0; o >>= 1) tests += __shfl_down_sync(0xFFFFFFFFu, tests, o);
    if (lane == 0 && tests) {
      atomicAdd(&s.d.pair_tests, tests);
      atomicAdd(&s.d.fast_tests, tests);
    }
  }
}

namespace {
// resident blocks of a kernel on the whole GPU (occupancy x SMs)
template <typename F>
int resident_blocks(F kernel, int threads, size_t smem, int num_sms) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess ||
      per_sm < 1) {
    cudaGetLastError();
    per_sm = 2;
  }
  return per_sm * num_sms;
}
}  // namespace

void search_grids(int precision, int K, int num_sms, uint32_t ptiles, LaunchPlan& L) {
  auto cap = [&](int blocks) { return (int)std::min<uint32_t>((uint32_t)blocks, std::max(ptiles, 1u)); };
  if (precision == KMC_FP64) {
    L.cell_blocks = K == 2 ? resident_blocks(k_search_cell<KMC_FP64, 2>, kCellWarps * 32, 0, num_sms)
                           : resident_blocks(k_search_cell<KMC_FP64, 1>, kCellWarps * 32, 0, num_sms);
    L.part_blocks = cap(K == 2 ? resident_blocks(k_search<KMC_FP64, 2>, kTile, 0, num_sms)
                               : resident_blocks(k_search<KMC_FP64, 1>, kTile, 0, num_sms));
    L.row_blocks = 0;
    L.row_blocks_px = 0;
    L.fast_blocks = cap(resident_blocks(k_search_fast<KMC_FP64>, kCellWarps * 32, 0, num_sms));
    return;
  }
  // the row search keeps its piece lists in dynamic shared memory (above 48 KB for
  // K = 2); set before any launch or capture
  if (K == 2) {
    cudaFuncSetAttribute(k_search_rows32<2, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)RowLayout<2, true>::kBytes);
    cudaFuncSetAttribute(k_search_rows32<2, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)RowLayout<2, false>::kBytes);
    L.cell_blocks = resident_blocks(k_search_cell32<2>, kCellWarps * 32, 0, num_sms);
    L.part_blocks = cap(resident_blocks(k_search<KMC_GUARDED_FP32, 2>, kTile, 0, num_sms));
    L.row_blocks = cap(resident_blocks(k_search_rows32<2, false>, kTile, RowLayout<2, false>::kBytes, num_sms));
    L.row_blocks_px = cap(resident_blocks(k_search_rows32<2, true>, kTile, RowLayout<2, true>::kBytes, num_sms));
  } else {
    cudaFuncSetAttribute(k_search_rows32<1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)RowLayout<1, true>::kBytes);
    cudaFuncSetAttribute(k_search_rows32<1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)RowLayout<1, false>::kBytes);
    L.cell_blocks = resident_blocks(k_search_cell32<1>, kCellWarps * 32, 0, num_sms);
    L.part_blocks = cap(resident_blocks(k_search<KMC_GUARDED_FP32, 1>, kTile, 0, num_sms));
    L.row_blocks = cap(resident_blocks(k_search_rows32<1, false>, kTile, RowLayout<1, false>::kBytes, num_sms));
    L.row_blocks_px = cap(resident_blocks(k_search_rows32<1, true>, kTile, RowLayout<1, true>::kBytes, num_sms));
  }
  L.fast_blocks = cap(resident_blocks(k_search_fast<KMC_GUARDED_FP32>, kCellWarps * 32, 0, num_sms));
}

int launch_search(const LaunchPlan& L, int precision, int K, cudaStream_t st, cudaEvent_t* ev_slow) {
  // every search kernel is launched; each simulation runs in the one its grid selected
  // (the others return at once)
  const int cb = L.cell_blocks;
  if (ev_slow) cudaEventRecord(ev_slow[0], st);
  if (precision == KMC_FP64) {
    if (K == 2) {
      k_search<KMC_FP64, 2><<<L.part_blocks, kTile, 0, st>>>(L.b);
      k_search_cell<KMC_FP64, 2><<<cb, kCellWarps * 32, 0, st>>>(L.b);
    } else {
      k_search<KMC_FP64, 1><<<L.part_blocks, kTile, 0, st>>>(L.b);
      k_search_cell<KMC_FP64, 1><<<cb, kCellWarps * 32, 0, st>>>(L.b);
    }
  } else {
    if (K == 2) {
      k_search<KMC_GUARDED_FP32, 2><<<L.part_blocks, kTile, 0, st>>>(L.b);
      k_search_cell32<2><<<cb, kCellWarps * 32, 0, st>>>(L.b);
      k_search_rows32<2, false><<<L.row_blocks, kTile, RowLayout<2, false>::kBytes, st>>>(L.b);
      k_search_rows32<2, true><<<L.row_blocks_px, kTile, RowLayout<2, true>::kBytes, st>>>(L.b);
    } else {
      k_search<KMC_GUARDED_FP32, 1><<<L.part_blocks, kTile, 0, st>>>(L.b);
      k_search_cell32<1><<<cb, kCellWarps * 32, 0, st>>>(L.b);
      k_search_rows32<1, false><<<L.row_blocks, kTile, RowLayout<1, false>::kBytes, st>>>(L.b);
      k_search_rows32<1, true><<<L.row_blocks_px, kTile, RowLayout<1, true>::kBytes, st>>>(L.b);
    }
  }
  if (ev_slow) cudaEventRecord(ev_slow[1], st);
  if (precision == KMC_FP64) k_search_fast<KMC_FP64><<<L.fast_blocks, kCellWarps * 32, 0, st>>>(L.b);
  else k_search_fast<KMC_GUARDED_FP32><<<L.fast_blocks, kCellWarps * 32, 0, st>>>(L.b);
  return precision == KMC_FP64 ? 3 : 5;
}

}  // namespace kmc
