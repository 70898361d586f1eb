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
#include "kmc_internal.cuh"

namespace kmc {

struct Own32 {
  float ox, oy, oz, vx, vy, vz;
};

__device__ __forceinline__ void min_image_f(float& r, float halfL, float L, float tie, bool& keep) {
  float ar = fabsf(r);
  if (fabsf(ar - halfL) <= tie) keep = true;
  else if (ar > halfL) r = r > 0.f ? r - L : r + L;
}

template <int PREC, int K>
__global__ void __launch_bounds__(kTile) k_search(Batch B) {
  __shared__ uint2 sbuf[kSearchBuf];
  __shared__ uint32_t scnt, sbase;
  __shared__ unsigned long long stests;
  int k = find_sim(B.ptile, B.nsims, blockIdx.x);
  SimDev& s = *B.sims[k];
  if (!sim_active(s)) return;
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

  uint32_t p = (blockIdx.x - B.ptile[k]) * kTile + threadIdx.x;
  if (p < n) {
    int cx, cy, cz;
    key_decode(g, s.skey[p], cx, cy, cz);

    // own record
    double xo[3], vo[3];
    Own32 o32;
    const double* __restrict__ X0 = s.x[cur][0];
    const double* __restrict__ X1 = s.x[cur][1];
    const double* __restrict__ X2 = s.x[cur][2];
    const double* __restrict__ V0 = s.v[cur][0];
    const double* __restrict__ V1 = s.v[cur][1];
    const double* __restrict__ V2 = s.v[cur][2];
    const float4* __restrict__ MA = s.mir_a;
    const float2* __restrict__ MB = s.mir_b;
    if (PREC == KMC_FP64) {
      xo[0] = X0[p]; xo[1] = X1[p]; xo[2] = X2[p];
      vo[0] = V0[p]; vo[1] = V1[p]; vo[2] = V2[p];
    } else {
      float4 a = MA[p];
      float2 b = MB[p];
      o32 = {a.x, a.y, a.z, a.w, b.x, b.y};
    }
    // one-cell periodic axes need the minimum image explicitly
    const bool cp0 = nx == 1 && px, cp1 = ny == 1 && py, cp2 = nz == 1 && pz;
    const bool any_cp = cp0 || cp1 || cp2;
    const double L0 = s.box[0], L1 = s.box[1], L2 = s.box[2];

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
        const uint32_t colbase = col_code(g, (uint32_t)qy, (uint32_t)qz) * (uint32_t)nx;
        const int dx0 = (dz == 0 && dy == 0) ? 0 : -Kx;
        for (int dx = dx0; dx <= Kx; ++dx) {
          int qx = cx + dx;
          if (qx < 0) {
            if (!px) continue;
            qx += nx;
          } else if (qx >= nx) {
            if (!px) continue;
            qx -= nx;
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
            // own coordinates shifted into the frame of the neighbour cell's corner
            const float sx = o32.ox - (float)dx * g.wf[0];
            const float sy = o32.oy - (float)dy * g.wf[1];
            const float sz = o32.oz - (float)dz * g.wf[2];
            for (uint32_t j = beg; j < end; ++j) {
              const float4 a = __ldg(MA + j);
              const float2 b = __ldg(MB + j);
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

int launch_search(const LaunchPlan& L, int precision, int K, cudaStream_t st) {
  if (precision == KMC_FP64) {
    if (K == 2) k_search<KMC_FP64, 2><<<L.ptiles, kTile, 0, st>>>(L.b);
    else k_search<KMC_FP64, 1><<<L.ptiles, kTile, 0, st>>>(L.b);
  } else {
    if (K == 2) k_search<KMC_GUARDED_FP32, 2><<<L.ptiles, kTile, 0, st>>>(L.b);
    else k_search<KMC_GUARDED_FP32, 1><<<L.ptiles, kTile, 0, st>>>(L.b);
  }
  return 1;
}

}  // namespace kmc
