// kmc_init.cu -- initial states drawn on the device from Philox4x32-10.
//
// The paper describes its initial states in words only (Sec. 2: particles in a box;
// Sec. 3 and Sec. 4: random positions, one common speed, random directions).  This
// kernel draws them without a host round trip, from counters that the collision
// update never uses, so that a state of any size is created in a few milliseconds:
//
//   key (seed lo, seed hi); counter (id, 0xFFFFFFFF, k, 0xFFFFFFFF), i.e. the
//   collision counter of step 2^64 - 1, a step no run reaches.
//   positions  attempt a = 0..63 uses blocks k = 2a and 2a+1; a coordinate is the
//              53-bit uniform u = ((w0 >> 5) 2^26 + (w1 >> 6)) 2^-53 of two words
//              (x: block 2a words 0-1, y: block 2a words 2-3, z: block 2a+1 words
//              0-1), x = u L, or the largest double below L if the product rounds
//              up to L.  Box states take attempt 0.  Blast: ids below n_hot take
//              x = (c - r) + (2r) u per axis and keep the attempt if
//              (dx^2 + dy^2) + dz^2 < r^2; the others take x = u L and keep it if not.
//   velocities blocks k = 128 + j (j = 0..63), two attempts per block (words 0-1, then
//              2-3); u = w 2^-31 - 1, s = u1^2 + u2^2, kept if 0 < s < 1.
//              Gaussian components by Marsaglia's polar method (SIAM Review 6, 1964):
//              f = sqrt((-2 ln s) / s); the first kept attempt gives (u1 f, u2 f), the
//              second u1 f; v = sigma g.  One speed: the first kept attempt gives the
//              direction (sphere: (2u1 sqrt(1-s), 2u2 sqrt(1-s), 1 - 2s); planar:
//              ((u1^2 - u2^2)/s, (2u1) u2/s, 0)), v = speed n.
//   planar     z = box_z / 2, vz = 0.
// ln s comes from ln_series below (+, -, *, / only), so the arrays are bit-identical
// to any implementation of the same definition on an IEEE-754 machine; every binary64
// operation is a __d*_rn intrinsic in the order written.
#include "kmc_internal.cuh"
#include "kmc_rng.cuh"

namespace kmc {

// Natural logarithm of a positive normal s: s = m 2^e with m in [1, 2) from the bits
// (exact); if m exceeds the double nearest sqrt 2, m is halved and e raised, so m lies
// in (0.707, 1.415).  ln m = 2 atanh(f), f = (m - 1)/(m + 1), |f| < 0.172, summed as
// 2f (1 + f^2/3 + ... + f^22/23) (the next term is below 2^-63 relative) in Horner
// form with each coefficient 1/(2k+1) one correctly rounded division; ln s = e ln2 +
// ln m with ln2 the double nearest ln 2.
__device__ double ln_series(double s) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(s);
  int e = (int)((b >> 52) & 0x7FFull) - 1023;
  double m = __longlong_as_double((long long)((b & 0x000FFFFFFFFFFFFFull) | (1023ull << 52)));
  if (m > 0x1.6a09e667f3bcdp+0) {
    m = dmul(m, 0.5);
    e += 1;
  }
  const double f = ddiv(dsub(m, 1.0), dadd(m, 1.0));
  const double z = dmul(f, f);
  double poly = ddiv(1.0, 23.0);
#pragma unroll
  for (int k = 10; k >= 0; --k) poly = dadd(dmul(poly, z), ddiv(1.0, (double)(2 * k + 1)));
  const double lnm = dmul(dadd(f, f), poly);
  return dadd(dmul((double)e, 0x1.62e42fefa39efp-1), lnm);
}

__device__ __forceinline__ double u53(uint32_t w0, uint32_t w1) {
  // (w0 >> 5) 2^26 + (w1 >> 6) < 2^53: every step is exact
  return dmul(dadd(dmul((double)(w0 >> 5), 67108864.0), (double)(w1 >> 6)), 0x1p-53);
}

__device__ __forceinline__ double scale_into(double u, double L) {
  const double x = dmul(u, L);
  // the largest double below a positive normal L
  return x < L ? x : __longlong_as_double(__double_as_longlong(L) - 1);
}

__device__ __forceinline__ void init_block(uint32_t id, uint32_t k, uint64_t seed, uint32_t w[4]) {
  w[0] = id; w[1] = 0xFFFFFFFFu; w[2] = k; w[3] = 0xFFFFFFFFu;
  philox4x32_10(w, (uint32_t)seed, (uint32_t)(seed >> 32));
}

__global__ void __launch_bounds__(256) k_init_state(InitLaunch L) {
  const uint32_t id = blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= L.n) return;
  const bool blast = L.kind == KMC_INIT_BLAST;
  const bool hot = blast && (uint64_t)id < L.n_hot;
  double x[3] = {0.0, 0.0, 0.0};
  bool placed = false;
  for (uint32_t a = 0; a < 64 && !placed; ++a) {
    uint32_t w0[4], w1[4];
    init_block(id, 2 * a, L.seed, w0);
    init_block(id, 2 * a + 1, L.seed, w1);
    const double u[3] = {u53(w0[0], w0[1]), u53(w0[2], w0[3]), u53(w1[0], w1[1])};
#pragma unroll
    for (int k = 0; k < 3; ++k)
      x[k] = hot ? dadd(dsub(L.center[k], L.radius), dmul(dadd(L.radius, L.radius), u[k]))
                 : scale_into(u[k], L.box[k]);
    if (L.planar) x[2] = dmul(L.box[2], 0.5);
    placed = true;
    if (blast) {
      const double d0 = dsub(x[0], L.center[0]), d1 = dsub(x[1], L.center[1]), d2 = dsub(x[2], L.center[2]);
      const double r2 = dadd(dadd(dmul(d0, d0), dmul(d1, d1)), dmul(d2, d2));
      placed = (r2 < dmul(L.radius, L.radius)) == hot;
    }
  }
  double v[3] = {0.0, 0.0, 0.0};
  const int want = (L.kind == KMC_INIT_EQUAL_SPEED || L.planar) ? 1 : 2;
  int got = 0;
  double g[4] = {0.0, 0.0, 0.0, 0.0};
  for (uint32_t j = 0; j < 64 && got < want; ++j) {
    uint32_t w[4];
    init_block(id, 128 + j, L.seed, w);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (got >= want) break;
      const double u1 = word_uniform(w[2 * h]), u2 = word_uniform(w[2 * h + 1]);
      const double s = dadd(dmul(u1, u1), dmul(u2, u2));
      if (!(s > 0.0 && s < 1.0)) continue;
      if (L.kind == KMC_INIT_EQUAL_SPEED) {
        if (L.planar) {
          v[0] = dmul(L.speed, ddiv(dsub(dmul(u1, u1), dmul(u2, u2)), s));
          v[1] = dmul(L.speed, ddiv(dmul(dadd(u1, u1), u2), s));
        } else {
          const double q = dsqrt(dsub(1.0, s));
          v[0] = dmul(L.speed, dmul(dadd(u1, u1), q));
          v[1] = dmul(L.speed, dmul(dadd(u2, u2), q));
          v[2] = dmul(L.speed, dsub(1.0, dadd(s, s)));
        }
      } else {
        const double f = dsqrt(ddiv(dmul(-2.0, ln_series(s)), s));
        g[2 * got] = dmul(u1, f);
        g[2 * got + 1] = dmul(u2, f);
      }
      ++got;
    }
  }
  if (L.kind != KMC_INIT_EQUAL_SPEED) {
    const double sg = hot ? L.sigma_hot : L.sigma;
    v[0] = dmul(sg, g[0]);
    v[1] = dmul(sg, g[1]);
    v[2] = L.planar ? 0.0 : dmul(sg, g[2]);
  }
  if (!placed || got < want) atomicAdd(L.fails, 1u);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    L.x[k][id] = x[k];
    L.v[k][id] = v[k];
  }
  L.id[id] = id;
  L.last[id] = kNone;
}

void launch_init_state(const InitLaunch& L, cudaStream_t st) {
  if (L.n == 0) return;
  k_init_state<<<(L.n + 255) / 256, 256, 0, st>>>(L);
}

}  // namespace kmc
