/*
 * kmc_oracle.c -- plain, slow, FP64 CPU oracle for one time step of the kinetic
 * Monte Carlo hard-sphere gas of Howell et al., "Parallelization of Kinetic Theory
 * Simulations" (Sec. 2 "Initial Simulation Setup").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load this library.  It shares no code, header or
 * constant with the CUDA library; the two meet only through the seeded inputs.
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math -fopenmp -shared -fPIC.
 * Every floating-point operation below is one correctly rounded IEEE-754 binary64
 * +, -, *, / or sqrt, in the order written (no contraction), so the result is
 * the same on every host that honours IEEE-754.
 *
 * What each part follows:
 *   - Binning into cells: Sec. 2 (grid of bins, particles appended to their bin).
 *     Here it is only an acceleration of brute force: the cell search returns
 *     exactly the pairs the O(N^2) search returns (pinned by a test).
 *   - Candidate test: Sec. 2, the three criteria (inside the neighbourhood, within
 *     the effective radii, closest approach reached within the next time step),
 *     with t* = -r.v/|v|^2 and d_min^2 = |r x v|^2/|v|^2.
 *   - Best partner: Sec. 2 (a closer partner replaces the one found so far);
 *     ties broken on (t*, partner id).
 *   - Mutual choice: Sec. 2 (two particles collide only if each found the other),
 *     repeated over the particles still unmatched for up to max_rounds rounds.
 *   - Collision update: Sec. 2 says only that positions and velocities are updated;
 *     the update used is an isotropic centre-of-mass elastic scatter whose
 *     direction comes from Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and
 *     Marsaglia's (1972) method for a point on the unit sphere; in the planar mode
 *     (the paper's two-dimensional runs, Sec. 2 and Sec. 4: 8 neighbouring bins)
 *     the direction is uniform on the unit circle (von Neumann's method).
 *   - Boundaries: Sec. 2 (reflective or periodic box), plus a moving piston wall.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_NONE 0xFFFFFFFFu
#define OR_PERIODIC 0
#define OR_REFLECT 1
#define OR_ABSORB 2           /* walls at 0 and L remove the particles that cross them */
#define OR_ABSORBED 0xFFFFFFFEu /* last-partner value of a particle that has left */

typedef struct or_params {
  uint32_t n;
  uint32_t pad0;
  double box[3];
  int32_t bc[3];
  int32_t max_rounds;
  double piston_x0, piston_u;
  double d0, dt;
  uint64_t seed;
  int32_t profile_bins, profile_every;
  double profile_range;
  int32_t search;  /* 0: brute force O(N^2), 1: cell search */
  int32_t threads; /* 0: library default */
  int32_t planar;  /* 1: two-dimensional dynamics in the x-y plane (z and vz constant,
                      vz = 0); scatter directions isotropic in the plane */
  int32_t nspecies; /* 0: one species (m = 1, contact distance d0); else a mixture */
  /* Mixture (Sec. 2: every particle carries its mass and effective radius): species[i]
   * indexes mass[] and radius[]; a pair (i, j) is in contact at r_i + r_j; d0 must be
   * at least the largest contact distance (it sets the search reach). */
  const uint8_t* species;
  const double* mass;
  const double* radius;
} or_params;

/* Per-step record: collisions (matched pairs), candidate pairs, and the pairs
 * matched in each of up to four rounds. */
typedef struct or_counts {
  uint64_t step;
  uint32_t collisions;
  uint32_t edges;
  uint32_t round_pairs[4];
  uint32_t absorbed; /* particles that left through an absorbing wall in this step */
  uint32_t live;     /* particles still in the box after the step */
} or_counts;

static int is_gone(const uint32_t* last, uint32_t i) { return last != NULL && last[i] == OR_ABSORBED; }

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon et al., SC'11, Sec. "Philox"): ten rounds of the
 * Philox S-box with the two 32-bit multipliers, key bumped by the Weyl constants
 * between rounds. */
static void mulhilo32(uint32_t a, uint32_t b, uint32_t* hi, uint32_t* lo) {
  uint64_t p = (uint64_t)a * (uint64_t)b;
  *hi = (uint32_t)(p >> 32);
  *lo = (uint32_t)p;
}

void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    uint32_t hi0, lo0, hi1, lo1;
    mulhilo32(0xD2511F53u, c0, &hi0, &lo0);
    mulhilo32(0xCD9E8D57u, c2, &hi1, &lo1);
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Unit vector for the pair whose smaller id is `id`, at absolute step `step`.
 * Counter (id, step lo, k, step hi), key (seed lo, seed hi); each Philox call gives
 * two Marsaglia attempts.  A 32-bit word w maps to u = w*2^-31 - 1 in [-1, 1),
 * exactly.  Accept when 0 < s = u1^2 + u2^2 < 1; then
 * n = (2 u1 sqrt(1-s), 2 u2 sqrt(1-s), 1 - 2 s).
 * Returns the number of attempts used (1..128) or -1 if all 128 were rejected. */
int or_unit_vector(uint64_t seed, uint64_t step, uint32_t id, double nvec[3]) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (uint32_t k = 0; k < 64; ++k) {
    uint32_t ctr[4] = {id, (uint32_t)step, k, (uint32_t)(step >> 32)};
    uint32_t w[4];
    or_philox4x32_10(ctr, key, w);
    for (int a = 0; a < 2; ++a) {
      double u1 = (double)w[2 * a] * 0x1p-31 - 1.0;
      double u2 = (double)w[2 * a + 1] * 0x1p-31 - 1.0;
      double s = u1 * u1 + u2 * u2;
      if (s > 0.0 && s < 1.0) {
        double q = sqrt(1.0 - s);
        nvec[0] = (u1 + u1) * q;
        nvec[1] = (u2 + u2) * q;
        nvec[2] = 1.0 - (s + s);
        return (int)(2 * k + a + 1);
      }
    }
  }
  return -1;
}

/* Unit vector in the x-y plane for the planar (two-dimensional) mode, from the same
 * counters as or_unit_vector.  A point (u1, u2) uniform in the unit disk (the same
 * rejection) has a uniform polar angle phi; the vector at twice that angle,
 * (cos 2phi, sin 2phi) = ((u1^2 - u2^2)/s, (2 u1 u2)/s) with s = u1^2 + u2^2, is
 * uniform on the unit circle (von Neumann's method, no trigonometric function).
 * Written n = ((u1*u1 - u2*u2) / s, ((u1 + u1) * u2) / s, 0).
 * Returns the number of attempts used (1..128) or -1 if all 128 were rejected. */
int or_circle_vector(uint64_t seed, uint64_t step, uint32_t id, double nvec[3]) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  for (uint32_t k = 0; k < 64; ++k) {
    uint32_t ctr[4] = {id, (uint32_t)step, k, (uint32_t)(step >> 32)};
    uint32_t w[4];
    or_philox4x32_10(ctr, key, w);
    for (int a = 0; a < 2; ++a) {
      double u1 = (double)w[2 * a] * 0x1p-31 - 1.0;
      double u2 = (double)w[2 * a + 1] * 0x1p-31 - 1.0;
      double s = u1 * u1 + u2 * u2;
      if (s > 0.0 && s < 1.0) {
        nvec[0] = (u1 * u1 - u2 * u2) / s;
        nvec[1] = ((u1 + u1) * u2) / s;
        nvec[2] = 0.0;
        return (int)(2 * k + a + 1);
      }
    }
  }
  return -1;
}

/* ------------------------------------------------------------------------- */
/* Pair geometry and the candidate test (Sec. 2, the three criteria).
 * r = x_j - x_i per axis; on a periodic axis the minimum image is taken with
 * "if r > L/2 then r -= L, else if r < -L/2 then r += L".  v = v_j - v_i.
 * vv = |v|^2, rv = r.v, w = r x v, t = -rv/vv, d2 = |w|^2/vv.
 * Candidate iff vv != 0, 0 <= t < dt, d2 < d0^2, and the pair is not the pair that
 * collided last for both of its members (each member's last partner is the other). */
static inline double min_image(double r, double L, double halfL) {
  if (r > halfL) return r - L;
  if (r < -halfL) return r + L;
  return r;
}

typedef struct geo {
  double L[3], halfL[3];
  int periodic[3];
  double dt, d0sq;
  const uint8_t* species; /* mixture: contact distance radius[s_i] + radius[s_j] */
  const double* radius;
} geo;

static void make_geo(const or_params* p, geo* g) {
  for (int k = 0; k < 3; ++k) {
    g->L[k] = p->box[k];
    g->halfL[k] = p->box[k] * 0.5;
    g->periodic[k] = (p->bc[k] == OR_PERIODIC);
  }
  g->dt = p->dt;
  g->d0sq = p->d0 * p->d0;
  g->species = p->nspecies > 0 ? p->species : NULL;
  g->radius = p->radius;
}

/* Returns 1 and fills (d2, t) if (i, j) is a candidate pair. */
static int pair_test(const geo* g, const double* const st[6], const uint32_t* last,
                     uint32_t i, uint32_t j, double* d2_out, double* t_out) {
  if (last != NULL && last[i] == j && last[j] == i) return 0;
  if (is_gone(last, i) || is_gone(last, j)) return 0; /* absorbed: out of the gas */
  double r[3], v[3];
  for (int k = 0; k < 3; ++k) {
    double d = st[k][j] - st[k][i];
    r[k] = g->periodic[k] ? min_image(d, g->L[k], g->halfL[k]) : d;
    v[k] = st[3 + k][j] - st[3 + k][i];
  }
  double vv = (v[0] * v[0] + v[1] * v[1]) + v[2] * v[2];
  if (vv == 0.0) return 0;
  double rv = (r[0] * v[0] + r[1] * v[1]) + r[2] * v[2];
  double t = (-rv) / vv;
  double wx = r[1] * v[2] - r[2] * v[1];
  double wy = r[2] * v[0] - r[0] * v[2];
  double wz = r[0] * v[1] - r[1] * v[0];
  double d2 = ((wx * wx + wy * wy) + wz * wz) / vv;
  double c2 = g->d0sq;
  if (g->species) {
    double c = g->radius[g->species[i]] + g->radius[g->species[j]];
    c2 = c * c;
  }
  if (t >= 0.0 && t < g->dt && d2 < c2) {
    *d2_out = d2;
    *t_out = t;
    return 1;
  }
  return 0;
}

int or_pair(const or_params* p, const double* const st[6], const uint32_t* last,
            uint32_t i, uint32_t j, double* d2, double* t) {
  geo g;
  make_geo(p, &g);
  return pair_test(&g, st, last, i, j, d2, t);
}

/* ------------------------------------------------------------------------- */
/* Candidate lists: for every particle i, every j != i that passes the test.
 * Stored as CSR (off[n+1], nbr[], d2[], t[]), each list sorted by j. */
typedef struct adjacency {
  int64_t* off;
  uint32_t* nbr;
  double* d2;
  double* t;
  int64_t total;
} adjacency;

static void adj_free(adjacency* a) {
  free(a->off); free(a->nbr); free(a->d2); free(a->t);
  memset(a, 0, sizeof(*a));
}

typedef struct entry { uint32_t j; double d2, t; } entry;

static int entry_cmp(const void* a, const void* b) {
  uint32_t ja = ((const entry*)a)->j, jb = ((const entry*)b)->j;
  return (ja > jb) - (ja < jb);
}

/* growable per-chunk buffer */
typedef struct ebuf { entry* e; int64_t n, cap; int64_t* cnt; } ebuf;

static int ebuf_push(ebuf* b, uint32_t j, double d2, double t) {
  if (b->n == b->cap) {
    int64_t nc = b->cap ? 2 * b->cap : 256;
    entry* ne = (entry*)realloc(b->e, (size_t)nc * sizeof(entry));
    if (!ne) return -1;
    b->e = ne; b->cap = nc;
  }
  b->e[b->n].j = j; b->e[b->n].d2 = d2; b->e[b->n].t = t;
  b->n++;
  return 0;
}

/* The cell grid used to accelerate the search.  Cell width per axis is at least
 * 1.01*(d0 + 2 vmax dt): any candidate has |r| <= d_min + |v| t* < d0 + 2 vmax dt, so
 * its partner lies in the same or an adjacent cell.  An axis with fewer than three
 * cells becomes a single cell so that no neighbour is visited twice. */
typedef struct cgrid {
  int nc[3];
  double lo[3], w[3];
  int64_t ncell;
  int64_t* start; /* ncell+1 */
  uint32_t* perm; /* particles grouped by cell, increasing id inside a cell */
} cgrid;

static int build_cells(const or_params* p, const double* const st[6], const uint32_t* last,
                       cgrid* cg) {
  uint32_t n = p->n;
  double vmax2 = 0.0;
  uint32_t first = 0; /* first particle still in the box (absorbed ones are not binned) */
  while (first < n && is_gone(last, first)) ++first;
  for (uint32_t i = 0; i < n; ++i) {
    if (is_gone(last, i)) continue;
    double s = (st[3][i] * st[3][i] + st[4][i] * st[4][i]) + st[5][i] * st[5][i];
    if (s > vmax2) vmax2 = s;
  }
  double h = (p->d0 + 2.0 * sqrt(vmax2) * p->dt) * 1.01;
  for (int k = 0; k < 3; ++k) {
    double lo, hi;
    if (p->bc[k] == OR_PERIODIC) {
      lo = 0.0; hi = p->box[k];
    } else {
      lo = first < n ? st[k][first] : 0.0;
      hi = lo;
      for (uint32_t i = first; i < n; ++i) {
        if (is_gone(last, i)) continue;
        if (st[k][i] < lo) lo = st[k][i];
        if (st[k][i] > hi) hi = st[k][i];
      }
    }
    double ext = hi - lo;
    double f = floor(ext / h);
    int c = (f > 1e6) ? 1000000 : (int)f;
    if (c < 3) c = 1;
    cg->nc[k] = c;
    cg->lo[k] = lo;
    cg->w[k] = (c == 1) ? (ext > 0 ? ext : 1.0) : ext / c;
  }
  cg->ncell = (int64_t)cg->nc[0] * cg->nc[1] * cg->nc[2];
  cg->start = (int64_t*)calloc((size_t)cg->ncell + 1, sizeof(int64_t));
  cg->perm = (uint32_t*)malloc((size_t)(n ? n : 1) * sizeof(uint32_t));
  int64_t* cell = (int64_t*)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
  if (!cg->start || !cg->perm || !cell) { free(cell); return -1; }
  for (uint32_t i = 0; i < n; ++i) {
    int64_t c[3];
    if (is_gone(last, i)) { cell[i] = -1; continue; }
    for (int k = 0; k < 3; ++k) {
      double f = floor((st[k][i] - cg->lo[k]) / cg->w[k]);
      int64_t ci = (f < 0.0) ? 0 : (f >= cg->nc[k] ? cg->nc[k] - 1 : (int64_t)f);
      c[k] = ci;
    }
    cell[i] = (c[2] * cg->nc[1] + c[1]) * cg->nc[0] + c[0];
    cg->start[cell[i] + 1]++;
  }
  for (int64_t c = 0; c < cg->ncell; ++c) cg->start[c + 1] += cg->start[c];
  int64_t* fill = (int64_t*)malloc((size_t)cg->ncell * sizeof(int64_t));
  if (!fill) { free(cell); return -1; }
  memcpy(fill, cg->start, (size_t)cg->ncell * sizeof(int64_t));
  for (uint32_t i = 0; i < n; ++i)
    if (cell[i] >= 0) cg->perm[fill[cell[i]]++] = i; /* ids increase */
  free(fill);
  free(cell);
  return 0;
}

static void free_cells(cgrid* cg) { free(cg->start); free(cg->perm); }

static int cell_of(const cgrid* cg, const or_params* p, const double* const st[6], uint32_t i,
                   int c[3]) {
  for (int k = 0; k < 3; ++k) {
    double f = floor((st[k][i] - cg->lo[k]) / cg->w[k]);
    c[k] = (f < 0.0) ? 0 : (f >= cg->nc[k] ? cg->nc[k] - 1 : (int)f);
  }
  (void)p;
  return 0;
}

int or_candidates_csr(const or_params* p, const double* const st[6], const uint32_t* last,
                      adjacency* out) {
  uint32_t n = p->n;
  geo g;
  make_geo(p, &g);
  memset(out, 0, sizeof(*out));
  out->off = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  if (!out->off) return -1;
  cgrid cg;
  memset(&cg, 0, sizeof(cg));
  if (p->search == 1 && n > 0) {
    if (build_cells(p, st, last, &cg)) { free_cells(&cg); return -1; }
  }
  const int64_t chunk = 512;
  int64_t nchunks = ((int64_t)n + chunk - 1) / chunk;
  ebuf* bufs = (ebuf*)calloc((size_t)(nchunks ? nchunks : 1), sizeof(ebuf));
  int fail = 0;
#ifdef _OPENMP
  int nthr = p->threads > 0 ? p->threads : omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthr)
#endif
  for (int64_t ch = 0; ch < nchunks; ++ch) {
    ebuf* b = &bufs[ch];
    b->cnt = (int64_t*)calloc((size_t)chunk, sizeof(int64_t));
    uint32_t i0 = (uint32_t)(ch * chunk);
    uint32_t i1 = (uint32_t)((ch + 1) * chunk < (int64_t)n ? (ch + 1) * chunk : n);
    for (uint32_t i = i0; i < i1; ++i) {
      int64_t before = b->n;
      double d2, t;
      if (p->search == 0) {
        for (uint32_t j = 0; j < n; ++j) {
          if (j == i) continue;
          if (pair_test(&g, st, last, i, j, &d2, &t)) {
            if (ebuf_push(b, j, d2, t)) fail = 1;
          }
        }
      } else if (!is_gone(last, i)) {
        int c[3];
        cell_of(&cg, p, st, i, c);
        int lo[3], hi[3];
        for (int k = 0; k < 3; ++k) {
          if (cg.nc[k] == 1) { lo[k] = 0; hi[k] = 0; }
          else { lo[k] = -1; hi[k] = 1; }
        }
        for (int dz = lo[2]; dz <= hi[2]; ++dz)
          for (int dy = lo[1]; dy <= hi[1]; ++dy)
            for (int dx = lo[0]; dx <= hi[0]; ++dx) {
              int q[3] = {c[0] + dx, c[1] + dy, c[2] + dz};
              int skip = 0;
              for (int k = 0; k < 3; ++k) {
                if (cg.nc[k] == 1) { q[k] = 0; continue; }
                if (q[k] < 0 || q[k] >= cg.nc[k]) {
                  if (g.periodic[k]) q[k] = (q[k] + cg.nc[k]) % cg.nc[k];
                  else skip = 1;
                }
              }
              if (skip) continue;
              int64_t cell = ((int64_t)q[2] * cg.nc[1] + q[1]) * cg.nc[0] + q[0];
              for (int64_t s = cg.start[cell]; s < cg.start[cell + 1]; ++s) {
                uint32_t j = cg.perm[s];
                if (j == i) continue;
                if (pair_test(&g, st, last, i, j, &d2, &t)) {
                  if (ebuf_push(b, j, d2, t)) fail = 1;
                }
              }
            }
      }
      if (b->n > before) qsort(b->e + before, (size_t)(b->n - before), sizeof(entry), entry_cmp);
      b->cnt[i - i0] = b->n - before;
    }
  }
  if (p->search == 1) free_cells(&cg);
  int64_t total = 0;
  for (int64_t ch = 0; ch < nchunks; ++ch) {
    if (!bufs[ch].cnt) fail = 1;
    else {
      uint32_t i0 = (uint32_t)(ch * chunk);
      uint32_t i1 = (uint32_t)((ch + 1) * chunk < (int64_t)n ? (ch + 1) * chunk : n);
      for (uint32_t i = i0; i < i1; ++i) {
        out->off[i] = total;
        total += bufs[ch].cnt[i - i0];
      }
    }
  }
  out->off[n] = total;
  out->total = total;
  size_t tb = (size_t)(total ? total : 1);
  out->nbr = (uint32_t*)malloc(tb * sizeof(uint32_t));
  out->d2 = (double*)malloc(tb * sizeof(double));
  out->t = (double*)malloc(tb * sizeof(double));
  if (!out->nbr || !out->d2 || !out->t) fail = 1;
  int64_t pos = 0;
  for (int64_t ch = 0; ch < nchunks && !fail; ++ch) {
    for (int64_t e = 0; e < bufs[ch].n; ++e) {
      out->nbr[pos] = bufs[ch].e[e].j;
      out->d2[pos] = bufs[ch].e[e].d2;
      out->t[pos] = bufs[ch].e[e].t;
      ++pos;
    }
  }
  for (int64_t ch = 0; ch < nchunks; ++ch) { free(bufs[ch].e); free(bufs[ch].cnt); }
  free(bufs);
  if (fail) { adj_free(out); return -1; }
  return 0;
}

/* Exported: candidate pairs (i < j) in increasing (i, j) order with their keys.
 * Returns the number of pairs, or -(needed) if cap is too small, or INT64_MIN on
 * allocation failure. */
int64_t or_candidate_pairs(const or_params* p, const double* const st[6], const uint32_t* last,
                           uint32_t* pi, uint32_t* pj, double* pd2, double* pt, int64_t cap) {
  adjacency a;
  if (or_candidates_csr(p, st, last, &a)) return INT64_MIN;
  int64_t cnt = 0;
  for (uint32_t i = 0; i < p->n; ++i)
    for (int64_t e = a.off[i]; e < a.off[i + 1]; ++e)
      if (a.nbr[e] > i) {
        if (cnt < cap) {
          pi[cnt] = i; pj[cnt] = a.nbr[e]; pd2[cnt] = a.d2[e]; pt[cnt] = a.t[e];
        }
        ++cnt;
      }
  adj_free(&a);
  return cnt <= cap ? cnt : -cnt;
}

/* ------------------------------------------------------------------------- */
/* Mutual-choice matching (Sec. 2): in each round every unmatched particle picks
 * the unmatched candidate with the smallest key (d2, t, partner id); pairs that
 * picked each other collide.  Rounds stop at max_rounds or when a round matches
 * nobody (every later round would repeat it). */
static int key_less(double d2a, double ta, uint32_t ja, double d2b, double tb, uint32_t jb) {
  if (d2a < d2b) return 1;
  if (d2a > d2b) return 0;
  if (ta < tb) return 1;
  if (ta > tb) return 0;
  return ja < jb;
}

static void match(const or_params* p, const adjacency* a, uint32_t* partner, int64_t* pedge,
                  uint32_t round_pairs[4]) {
  uint32_t n = p->n;
  uint32_t* best = (uint32_t*)malloc((size_t)(n ? n : 1) * sizeof(uint32_t));
  int64_t* bedge = (int64_t*)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
  for (uint32_t i = 0; i < n; ++i) { partner[i] = OR_NONE; pedge[i] = -1; }
  for (int r = 0; r < 4; ++r) round_pairs[r] = 0;
  for (int r = 0; r < p->max_rounds; ++r) {
    for (uint32_t i = 0; i < n; ++i) {
      best[i] = OR_NONE;
      bedge[i] = -1;
      if (partner[i] != OR_NONE) continue;
      for (int64_t e = a->off[i]; e < a->off[i + 1]; ++e) {
        uint32_t j = a->nbr[e];
        if (partner[j] != OR_NONE) continue;
        if (best[i] == OR_NONE ||
            key_less(a->d2[e], a->t[e], j, a->d2[bedge[i]], a->t[bedge[i]], best[i])) {
          best[i] = j;
          bedge[i] = e;
        }
      }
    }
    uint32_t pairs = 0;
    for (uint32_t i = 0; i < n; ++i) {
      uint32_t j = best[i];
      if (j != OR_NONE && best[j] == i) {
        partner[i] = j;
        pedge[i] = bedge[i];
        if (i < j) ++pairs;
      }
    }
    if (r < 4) round_pairs[r] = pairs;
    if (pairs == 0) break;
  }
  free(best);
  free(bedge);
}

/* ------------------------------------------------------------------------- */
/* Boundaries after streaming.  Periodic: one wrap into [0, L) with x == L mapped
 * to 0.  Reflecting: lower wall at 0; upper wall at L, or for the x axis at the
 * piston X = x0 - u*((step+1)*dt) (end of the step); specular reflection in the
 * frame of the wall: x -> 2X - x, v -> -v - 2u.  Absorbing (Sec. 2 names
 * absorptive walls beside reflective and periodic ones): walls at 0 and L that
 * remove a particle whose end-of-step position lies beyond them (x < 0 or x > L,
 * the reflecting test); it keeps that position and its velocity, its last partner
 * becomes OR_ABSORBED, and it takes no further part (no search, no streaming, no
 * profile).  Tested on every absorbing axis before the other axes' boundaries. */
static void apply_bc(const or_params* p, uint64_t step, double* x, double* v, int k) {
  if (p->bc[k] == OR_PERIODIC) {
    double L = p->box[k];
    if (*x >= L) *x = *x - L;
    if (*x < 0.0) {
      *x = *x + L;
      if (*x == L) *x = 0.0;
    }
    return;
  }
  double X, u;
  if (k == 0) {
    u = p->piston_u;
    X = p->piston_x0 - u * ((double)(step + 1) * p->dt);
  } else {
    u = 0.0;
    X = p->box[k];
  }
  if (*x < 0.0) {
    *x = -*x;
    *v = -*v;
  }
  if (*x > X) {
    *x = (X + X) - *x;
    *v = (-*v) - (u + u);
  }
}

/* One step.  state: st[0..2] positions, st[3..5] velocities (id order, id = index);
 * last: last collision partner per particle (OR_NONE if none).
 * partner_out (optional, n): this step's partner per particle, OR_NONE if none.
 * prof (optional): profile_bins*7 sums written when the step is a profile step. */
int or_step(const or_params* p, double* const st[6], uint32_t* last, uint64_t step,
            or_counts* counts, uint32_t* partner_out, double* prof, int* profiled) {
  uint32_t n = p->n;
  adjacency a;
  if (or_candidates_csr(p, (const double* const*)st, last, &a)) return -1;
  uint32_t* partner = (uint32_t*)malloc((size_t)(n ? n : 1) * sizeof(uint32_t));
  int64_t* pedge = (int64_t*)malloc((size_t)(n ? n : 1) * sizeof(int64_t));
  uint8_t* moved = (uint8_t*)calloc((size_t)(n ? n : 1), 1);
  if (!partner || !pedge || !moved) { adj_free(&a); free(partner); free(pedge); free(moved); return -1; }
  counts->step = step;
  counts->edges = (uint32_t)(a.total / 2);
  match(p, &a, partner, pedge, counts->round_pairs);
  uint32_t coll = 0;
  int rc = 0;
  /* collisions: stream to t*, scatter, stream the rest of the step */
  for (uint32_t ia = 0; ia < n; ++ia) {
    uint32_t ib = partner[ia];
    if (ib == OR_NONE || ib < ia) continue;
    ++coll;
    double t = a.t[pedge[ia]];
    double nv[3];
    if ((p->planar ? or_circle_vector(p->seed, step, ia, nv) : or_unit_vector(p->seed, step, ia, nv)) < 0) {
      rc = -2;
      continue;
    }
    double g[3], V[3];
    /* centre-of-mass velocity and the shares of the relative speed: equal masses
     * V = (v_a + v_b)/2, both shares G/2; a mixture V = (m_a v_a + m_b v_b)/M,
     * v_a' = V + (m_b/M) G n, v_b' = V - (m_a/M) G n (M = m_a + m_b), which is the
     * equal-mass update, bit for bit, when m_a = m_b */
    double ma = 1.0, mb = 1.0;
    if (p->nspecies > 0) {
      ma = p->mass[p->species[ia]];
      mb = p->mass[p->species[ib]];
    }
    double M = ma + mb;
    for (int k = 0; k < 3; ++k) {
      g[k] = st[3 + k][ia] - st[3 + k][ib];
      if (p->nspecies > 0) V[k] = (ma * st[3 + k][ia] + mb * st[3 + k][ib]) / M;
      else V[k] = (st[3 + k][ia] + st[3 + k][ib]) * 0.5;
    }
    double G = sqrt((g[0] * g[0] + g[1] * g[1]) + g[2] * g[2]);
    double hGa = (p->nspecies > 0 ? mb / M : 0.5) * G;
    double hGb = (p->nspecies > 0 ? ma / M : 0.5) * G;
    double rest = p->dt - t;
    for (int k = 0; k < 3; ++k) {
      double va = V[k] + hGa * nv[k];
      double vb = V[k] - hGb * nv[k];
      double xa = st[k][ia], xb = st[k][ib];
      double oa = st[3 + k][ia], ob = st[3 + k][ib];
      st[k][ia] = (xa + oa * t) + va * rest;
      st[k][ib] = (xb + ob * t) + vb * rest;
      st[3 + k][ia] = va;
      st[3 + k][ib] = vb;
    }
    moved[ia] = moved[ib] = 1;
  }
  counts->collisions = coll;
  uint32_t absorbed = 0, live = 0;
  for (uint32_t i = 0; i < n; ++i) {
    if (is_gone(last, i)) continue;
    for (int k = 0; k < 3; ++k)
      if (!moved[i]) st[k][i] = st[k][i] + st[3 + k][i] * p->dt;
    int gone = 0;
    for (int k = 0; k < 3; ++k)
      if (p->bc[k] == OR_ABSORB && (st[k][i] < 0.0 || st[k][i] > p->box[k])) gone = 1;
    if (gone) {
      last[i] = OR_ABSORBED;
      ++absorbed;
      continue;
    }
    for (int k = 0; k < 3; ++k)
      if (p->bc[k] != OR_ABSORB) apply_bc(p, step, &st[k][i], &st[3 + k][i], k);
    if (partner[i] != OR_NONE) last[i] = partner[i];
    ++live;
  }
  counts->absorbed = absorbed;
  counts->live = live;
  if (partner_out) memcpy(partner_out, partner, (size_t)n * sizeof(uint32_t));
  if (profiled) *profiled = 0;
  if (prof && p->profile_every > 0 && p->profile_bins > 0 &&
      (step + 1) % (uint64_t)p->profile_every == 0) {
    int nb = p->profile_bins;
    double scale = (double)nb / p->profile_range;
    memset(prof, 0, (size_t)nb * 7 * sizeof(double));
    for (uint32_t i = 0; i < n; ++i) {
      double x = st[0][i];
      if (is_gone(last, i) || !(x >= 0.0)) continue;
      double f = x * scale;
      if (f >= (double)nb) continue;
      int b = (int)f;
      double* q = prof + (size_t)b * 7;
      q[0] += 1.0;
      for (int k = 0; k < 3; ++k) {
        double vk = st[3 + k][i];
        q[1 + k] += vk;
        q[4 + k] += vk * vk;
      }
    }
    if (profiled) *profiled = 1;
  }
  adj_free(&a);
  free(partner);
  free(pedge);
  free(moved);
  return rc;
}

/* Run nsteps steps from absolute step step0.  counts: nsteps records.
 * prof: (number of profile steps) * bins * 7 doubles, in step order.
 * Returns 0, -1 on allocation failure, -2 if a scatter direction was not found. */
int or_run(const or_params* p, double* const st[6], uint32_t* last, uint64_t step0,
           uint32_t nsteps, or_counts* counts, double* prof) {
  int64_t nprof = 0;
  for (uint32_t s = 0; s < nsteps; ++s) {
    int profiled = 0;
    double* pp = prof ? prof + (size_t)nprof * (size_t)(p->profile_bins > 0 ? p->profile_bins : 0) * 7 : NULL;
    int rc = or_step(p, st, last, step0 + s, &counts[s], NULL, pp, &profiled);
    if (rc) return rc;
    nprof += profiled;
  }
  return 0;
}

/* max |v|^2 over particles, each |v|^2 = (vx^2 + vy^2) + vz^2 */
double or_vmax2(uint32_t n, const double* vx, const double* vy, const double* vz) {
  double m = 0.0;
  for (uint32_t i = 0; i < n; ++i) {
    double s = (vx[i] * vx[i] + vy[i] * vy[i]) + vz[i] * vz[i];
    if (s > m) m = s;
  }
  return m;
}

int or_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* Initial states drawn from Philox4x32-10 (the library's device-side
 * initialisation).  The paper describes its initial states only in words (Sec. 2:
 * particles in a box; Sec. 3 and Sec. 4: random positions, one speed, random
 * directions); this generator fixes one counter-based reading so that two
 * independent implementations produce the same arrays.
 *
 * Draws for particle `id`: key (seed lo, seed hi), counter (id, 0xFFFFFFFF, k,
 * 0xFFFFFFFF), i.e. the scatter counter of step 2^64 - 1, a step no run reaches.
 *   positions: attempt a (0..63) uses blocks k = 2a, 2a+1; each coordinate is a
 *     53-bit uniform u = ((w0 >> 5) 2^26 + (w1 >> 6)) 2^-53 in [0, 1) from two
 *     words (x: block 2a words 0-1, y: block 2a words 2-3, z: block 2a+1 words 0-1);
 *     x = u L (the largest double below L if the product rounds to L).  Box
 *     states accept attempt 0.  The blast's hot particles (id < n_hot) take
 *     x = (c - r) + (2r) u per axis and accept |x - c|^2 < r^2; the others take
 *     x = u L and accept |x - c|^2 >= r^2, with |x - c|^2 summed as (dx^2 + dy^2) + dz^2.
 *   velocities: blocks k = 128 + j (j = 0..63), two attempts per block (words 0-1,
 *     words 2-3), u = w 2^-31 - 1, s = u1^2 + u2^2, accept 0 < s < 1.
 *     Gaussian (Marsaglia's polar method, SIAM Rev. 6, 1964): f = sqrt((-2 ln s) / s),
 *     the first accepted attempt gives (u1 f, u2 f) = (gx, gy), the second gives
 *     gz (its u1 f); v = sigma g.  Equal speed: the first accepted attempt gives the
 *     direction n (sphere: (2 u1 sqrt(1-s), 2 u2 sqrt(1-s), 1 - 2s); planar:
 *     ((u1^2 - u2^2)/s, (2 u1) u2 / s, 0)), v = speed n.
 *   planar: z = box_z / 2 and vz = 0 (only two Gaussians are used).
 * ln s is or_log below. */

/* Natural logarithm from +, -, *, / only (so that two implementations that follow
 * the same operations agree bit for bit): s = m 2^e with m in [1, 2) read from the
 * bits (exact), m halved and e raised when m > sqrt(2) (the double nearest sqrt 2),
 * so m in (0.707, 1.415); ln m = 2 atanh(f) with f = (m - 1)/(m + 1), |f| < 0.172,
 * by the series 2 f (1 + f^2/3 + f^4/5 + ... + f^22/23) (f^24/25 < 2^-63) in
 * Horner form with coefficients 1/(2k+1) formed by one division each; then
 * ln s = e ln2 + ln m with ln2 the double nearest ln 2.  For positive normal s. */
double or_log(double s) {
  uint64_t b;
  memcpy(&b, &s, sizeof b);
  int e = (int)((b >> 52) & 0x7FF) - 1023;
  b = (b & 0x000FFFFFFFFFFFFFull) | ((uint64_t)1023 << 52);
  double m;
  memcpy(&m, &b, sizeof m);
  if (m > 0x1.6a09e667f3bcdp+0) {
    m = m * 0.5;
    e = e + 1;
  }
  double f = (m - 1.0) / (m + 1.0);
  double z = f * f;
  double poly = 1.0 / 23.0;
  for (int k = 10; k >= 0; --k) poly = poly * z + 1.0 / (double)(2 * k + 1);
  double lnm = (f + f) * poly;
  return (double)e * 0x1.62e42fefa39efp-1 + lnm;
}

typedef struct or_init {
  int32_t kind;   /* 1 Maxwellian box, 2 equal speed, 3 blast */
  int32_t pad0;
  uint64_t n_hot; /* blast: ids below n_hot are hot */
  double sigma;   /* Maxwellian / blast background: per-component standard deviation */
  double speed;   /* equal speed */
  double sigma_hot;
  double center[3];
  double radius;
} or_init;

static double u53(uint32_t w0, uint32_t w1) {
  return ((double)(w0 >> 5) * 67108864.0 + (double)(w1 >> 6)) * 0x1p-53;
}

static double below(double L) { return nextafter(L, 0.0); }

static double scale_into(double u, double L) {
  double x = u * L;
  return x < L ? x : below(L);
}

/* one particle; returns 0, or -1 when a rejection loop ran out of attempts */
static int init_one(const or_init* in, const or_params* p, uint32_t id, double out[6]) {
  const uint32_t key[2] = {(uint32_t)p->seed, (uint32_t)(p->seed >> 32)};
  const int blast = in->kind == 3;
  const int hot = blast && (uint64_t)id < in->n_hot;
  int placed = 0;
  for (uint32_t a = 0; a < 64 && !placed; ++a) {
    uint32_t c0[4] = {id, 0xFFFFFFFFu, 2 * a, 0xFFFFFFFFu}, c1[4] = {id, 0xFFFFFFFFu, 2 * a + 1, 0xFFFFFFFFu};
    uint32_t w0[4], w1[4];
    or_philox4x32_10(c0, key, w0);
    or_philox4x32_10(c1, key, w1);
    double u[3] = {u53(w0[0], w0[1]), u53(w0[2], w0[3]), u53(w1[0], w1[1])};
    double x[3];
    for (int k = 0; k < 3; ++k) {
      if (hot) {
        x[k] = (in->center[k] - in->radius) + (in->radius + in->radius) * u[k];
      } else {
        x[k] = scale_into(u[k], p->box[k]);
      }
    }
    if (p->planar) x[2] = p->box[2] * 0.5;
    if (blast) {
      double d[3];
      for (int k = 0; k < 3; ++k) d[k] = x[k] - in->center[k];
      double r2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
      int inside = r2 < in->radius * in->radius;
      if (inside != hot) continue;
    }
    for (int k = 0; k < 3; ++k) out[k] = x[k];
    placed = 1;
  }
  if (!placed) return -1;
  /* velocities */
  double g[4];
  int got = 0;
  const int want = in->kind == 2 ? 1 : (p->planar ? 1 : 2); /* accepted attempts needed */
  for (uint32_t j = 0; j < 64 && got < want; ++j) {
    uint32_t c[4] = {id, 0xFFFFFFFFu, 128 + j, 0xFFFFFFFFu};
    uint32_t w[4];
    or_philox4x32_10(c, key, w);
    for (int h = 0; h < 2 && got < want; ++h) {
      double u1 = (double)w[2 * h] * 0x1p-31 - 1.0;
      double u2 = (double)w[2 * h + 1] * 0x1p-31 - 1.0;
      double s = u1 * u1 + u2 * u2;
      if (!(s > 0.0 && s < 1.0)) continue;
      if (in->kind == 2) {
        if (p->planar) {
          out[3] = in->speed * ((u1 * u1 - u2 * u2) / s);
          out[4] = in->speed * (((u1 + u1) * u2) / s);
          out[5] = 0.0;
        } else {
          double q = sqrt(1.0 - s);
          out[3] = in->speed * ((u1 + u1) * q);
          out[4] = in->speed * ((u2 + u2) * q);
          out[5] = in->speed * (1.0 - (s + s));
        }
      } else {
        double f = sqrt((-2.0 * or_log(s)) / s);
        g[2 * got] = u1 * f;
        g[2 * got + 1] = u2 * f;
      }
      ++got;
    }
  }
  if (got < want) return -1;
  if (in->kind != 2) {
    double sg = hot ? in->sigma_hot : in->sigma;
    out[3] = sg * g[0];
    out[4] = sg * g[1];
    out[5] = p->planar ? 0.0 : sg * g[2];
  }
  return 0;
}

/* Initial state of the listed particle ids (out[k][i] for ids[i]); returns the
 * number of ids whose rejection loops ran out of attempts (0 normally). */
int64_t or_init_particles(const or_init* in, const or_params* p, const uint32_t* ids, int64_t m,
                          double* const out[6]) {
  int64_t fails = 0;
#pragma omp parallel for schedule(static) reduction(+ : fails)
  for (int64_t i = 0; i < m; ++i) {
    double o[6] = {0, 0, 0, 0, 0, 0};
    if (init_one(in, p, ids[i], o)) ++fails;
    for (int k = 0; k < 6; ++k) out[k][i] = o[k];
  }
  return fails;
}

/* or_log over an array (for tests) */
void or_log_many(const double* s, double* out, int64_t m) {
  for (int64_t i = 0; i < m; ++i) out[i] = or_log(s[i]);
}
