// kmc_api.cu -- host side of the C ABI declared in include/kmc.h.
//
// A simulation owns its device buffers and a device descriptor (SimDev).  Stepping
// goes through a LaunchPlan: a device table of descriptors plus tile prefixes,
// built for one simulation (sim_step) or for a group (sim_group_step).  The kernel
// sequence of one step is captured once in a CUDA graph and replayed per step; the
// step index, cell grid and counters live on the device, so replays need no host
// work.  Device-side failures set status bits that every later kernel of the
// simulation checks; sim_sync reads them, grows an overflowed pair buffer and
// re-runs the steps that were skipped (the state of the last completed step is
// untouched because the sort writes the other buffer).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "kmc_internal.cuh"

using namespace kmc;

namespace {

thread_local std::string g_create_error;

struct Plan {
  LaunchPlan L{};
  SimDev** d_table = nullptr;
  uint32_t* d_pre = nullptr;  // one allocation for the four prefix arrays + scratch
  cudaGraphExec_t graph = nullptr;
  bool graph_tried = false;
  int precision = 0, K = 1, max_rounds = 4;
  int launches_per_step = 0;
  bool has_profiles = false;
};

int g_num_sms = 0;

int num_sms() {
  if (g_num_sms == 0) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
      g_num_sms = v;
    else
      g_num_sms = 152;
  }
  return g_num_sms;
}

}  // namespace

struct kmc_group;

struct kmc_sim {
  kmc_params p{};
  SimDev h{};            // host mirror of the descriptor (parameters and pointers)
  SimDev* d = nullptr;   // device descriptor
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  kmc_group* group = nullptr;
  Plan solo;
  bool solo_built = false;
  std::vector<void*> allocs;
  void* stage = nullptr;
  size_t stage_bytes = 0;
  uint64_t hist_read = 0, prof_read = 0;
  uint64_t launches = 0;     // kernel launches enqueued for this simulation
  bool timing = false;       // per-phase CUDA-event timing (no graph)
  double phase_ms[5] = {0, 0, 0, 0, 0};  // sort, search, match, push; slow search kernels
  uint64_t timed_steps = 0;
  // in a group: the step index at the group's last sync (or at joining) and the
  // group's issued-step count then, so that a sync can tell how many of the group's
  // steps this member missed after an overflow
  uint64_t sync_step = 0, issued_base = 0;
  // a decomposition into x slabs (sim_create_domains): the steps run on its domains
  struct Domains* dom = nullptr;
  std::string err;
};

// Domain decomposition (Sec. 4): the member simulations are the domains, stepped as
// one batch; the exchange buffers live in DomainDev (kmc_domain.cu).
struct Domains {
  std::vector<kmc_sim*> members;
  Plan plan;
  DomainDev h{};
  DomainDev* d = nullptr;
  void* state = nullptr;  // id-order state, 52 n bytes (the layout of KMC_OBS_STATE)
  std::vector<void*> allocs;
  cudaGraphExec_t graph = nullptr;
  bool graph_tried = false;
  int launches_per_step = 0;
  uint64_t hist_read = 0;
};

struct kmc_group {
  std::vector<kmc_sim*> members;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  Plan plan;
  bool built = false;
  uint64_t issued = 0;  // group steps enqueued since the last sync
  std::string err;
};

namespace {

#define KCHECK(call, who)                                                        \
  do {                                                                           \
    cudaError_t e_ = (call);                                                     \
    if (e_ != cudaSuccess) {                                                     \
      (who) = std::string(#call) + ": " + cudaGetErrorString(e_);                \
      return KMC_ECUDA;                                                          \
    }                                                                            \
  } while (0)

uint32_t ceil_div(uint64_t a, uint64_t b) { return (uint32_t)((a + b - 1) / b); }

uint32_t default_edge_cap(uint32_t n) { return std::max<uint32_t>(4096u, n / 4u + 1024u); }
uint32_t default_cell_cap(uint32_t n) { return 2u * n + 4096u; }

struct Sizes {
  uint32_t n, cell_cap, edge_cap, hist_cap, prof_cap, bins;
  bool fp32;
};

Sizes sizes_of(const kmc_params& p) {
  Sizes z;
  z.n = p.n;
  z.cell_cap = default_cell_cap(p.n);
  z.edge_cap = p.edge_cap ? p.edge_cap : default_edge_cap(p.n);
  z.hist_cap = p.history_cap ? p.history_cap : 4096u;
  z.prof_cap = p.profile_cap ? p.profile_cap : 64u;
  z.bins = p.profile_bins > 0 ? (uint32_t)p.profile_bins : 0u;
  z.fp32 = p.precision == KMC_GUARDED_FP32;
  return z;
}

size_t edge_bytes(uint32_t cap) {
  // pairs, keys, slots; candidate lists (2 per pair) and the two round work lists
  return (size_t)cap * (sizeof(uint2) + 2 * sizeof(double) + sizeof(uint2)) +
         (size_t)2 * cap * (sizeof(uint2) + 2 * sizeof(uint32_t));
}

size_t bytes_for(const Sizes& z) {
  size_t n = z.n;
  size_t b = 0;
  b += 2 * 6 * n * sizeof(double) + 2 * 2 * n * sizeof(uint32_t);  // state, double-buffered
  if (z.fp32) b += (n + 1) / 2 * 3 * sizeof(float4);               // binary32 mirror
  b += 3 * n * sizeof(uint32_t) + n;                                  // key, rank, src, speed class
  b += n + 4096;                                                      // mixture species (if any)
  b += 2 * ((size_t)z.cell_cap + 2) * sizeof(uint32_t);               // cell count / start
  b += n * sizeof(uint32_t) + (n + 1) * sizeof(uint32_t);             // deg, list starts
  b += 4 * n * sizeof(uint32_t);                                      // best, best_e, partner, medge
  b += (n / 2 + 1) * sizeof(uint32_t);                                // pair list
  b += edge_bytes(z.edge_cap);
  b += (size_t)z.hist_cap * sizeof(kmc_step_counts);
  if (z.bins) b += (size_t)z.prof_cap * z.bins * kProfQ * sizeof(long long) + z.prof_cap * sizeof(uint64_t);
  b += sizeof(SimDev);
  return b;
}

int validate(const kmc_params* p, std::string& err) {
  if (!p) { err = "params is NULL"; return KMC_EINVAL; }
  if (p->n == 0) { err = "n must be >= 1"; return KMC_EINVAL; }
  if (p->flags & ~(uint32_t)(KMC_FLAG_NO_SPLIT | KMC_FLAG_FORCE_SPLIT | KMC_FLAG_PLANAR |
                             KMC_FLAG_SCAN_WAIT_TEST)) {
    err = "unknown flags";
    return KMC_EINVAL;
  }
  if ((p->flags & KMC_FLAG_NO_SPLIT) && (p->flags & KMC_FLAG_FORCE_SPLIT)) { err = "conflicting split flags"; return KMC_EINVAL; }
  for (int a = 0; a < 3; ++a) {
    if (!(p->box[a] > 0.0)) { err = "box extents must be > 0"; return KMC_EINVAL; }
    if (p->bc[a] != KMC_PERIODIC && p->bc[a] != KMC_REFLECT && p->bc[a] != KMC_ABSORB) {
      err = "bad boundary kind";
      return KMC_EINVAL;
    }
  }
  if (!(p->d0 > 0.0) || !(p->dt > 0.0)) { err = "d0 and dt must be > 0"; return KMC_EINVAL; }
  if (p->max_rounds < 0 || p->max_rounds > 4) { err = "max_rounds must be in 0..4"; return KMC_EINVAL; }
  if (p->precision != KMC_FP64 && p->precision != KMC_GUARDED_FP32) { err = "bad precision"; return KMC_EINVAL; }
  if (p->stencil < 0 || p->stencil > 2) { err = "stencil must be 0, 1 or 2"; return KMC_EINVAL; }
  if (p->profile_bins < 0 || p->profile_bins > 256) { err = "profile_bins must be in 0..256"; return KMC_EINVAL; }
  if (p->profile_every < 0) { err = "profile_every must be >= 0"; return KMC_EINVAL; }
  if (p->profile_bins > 0 && !(p->profile_range > 0.0)) { err = "profile_range must be > 0"; return KMC_EINVAL; }
  if (p->cell_scale != 0.0 && !(p->cell_scale >= 1.0)) { err = "cell_scale must be 0 or >= 1"; return KMC_EINVAL; }
  if (p->bc[0] == KMC_REFLECT && !(p->piston_x0 > 0.0)) { err = "reflecting x axis needs piston_x0 > 0"; return KMC_EINVAL; }
  // the cell tables hold 2 n + 4096 keys in uint32 indices
  if (p->n > 0x7FFFF000u) { err = "n too large (at most 2^31 - 4096)"; return KMC_EINVAL; }
  if (p->search_kernel < 0 || p->search_kernel > 3) { err = "bad search_kernel"; return KMC_EINVAL; }
  if (p->split_min_occ < 0.0) { err = "split_min_occ must be >= 0"; return KMC_EINVAL; }
  return KMC_OK;
}

bool is_device_ptr(const void* ptr) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <typename T>
int dalloc(kmc_sim* s, T** out, size_t count) {
  void* ptr = nullptr;
  size_t bytes = std::max<size_t>(count * sizeof(T), 16);
  cudaError_t e = cudaMalloc(&ptr, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    s->err = std::string("cudaMalloc failed: ") + cudaGetErrorString(e);
    return KMC_ENOMEM;
  }
  s->allocs.push_back(ptr);
  *out = (T*)ptr;
  return KMC_OK;
}

void dfree(kmc_sim* s, void* ptr) {
  if (!ptr) return;
  auto it = std::find(s->allocs.begin(), s->allocs.end(), ptr);
  if (it != s->allocs.end()) s->allocs.erase(it);
  cudaFree(ptr);
}

int alloc_edges(kmc_sim* s, uint32_t cap) {
  int rc;
  SimDev& h = s->h;
  if ((rc = dalloc(s, &h.edge, cap))) return rc;
  if ((rc = dalloc(s, &h.e_d2, cap))) return rc;
  if ((rc = dalloc(s, &h.e_t, cap))) return rc;
  if ((rc = dalloc(s, &h.e_slot, cap))) return rc;
  if ((rc = dalloc(s, &h.adj, 2 * (size_t)cap))) return rc;
  if ((rc = dalloc(s, &h.wl[0], 2 * (size_t)cap))) return rc;
  if ((rc = dalloc(s, &h.wl[1], 2 * (size_t)cap))) return rc;
  h.edge_cap = cap;
  return KMC_OK;
}

void free_edges(kmc_sim* s) {
  SimDev& h = s->h;
  void* ptrs[] = {h.edge, h.e_d2, h.e_t, h.e_slot, h.adj, h.wl[0], h.wl[1]};
  for (void* q : ptrs) dfree(s, q);
  h.edge = nullptr; h.e_d2 = nullptr; h.e_t = nullptr; h.e_slot = nullptr;
  h.adj = nullptr; h.wl[0] = h.wl[1] = nullptr;
}

// ---- plans ----------------------------------------------------------------- //
void free_plan(Plan& P) {
  if (P.graph) cudaGraphExecDestroy(P.graph);
  if (P.d_table) cudaFree(P.d_table);
  if (P.d_pre) cudaFree(P.d_pre);
  P = Plan();
}

int build_plan(Plan& P, const std::vector<kmc_sim*>& sims, cudaStream_t st, std::string& err) {
  free_plan(P);
  int m = (int)sims.size();
  std::vector<uint32_t> pt(m + 1), sc(m + 1), pr(m + 1);
  std::vector<SimDev*> table(m);
  pt[0] = sc[0] = pr[0] = 0;
  P.precision = sims[0]->h.precision;
  P.K = sims[0]->h.K;
  P.max_rounds = 0;
  for (int k = 0; k < m; ++k) {
    const SimDev& h = sims[k]->h;
    table[k] = sims[k]->d;
    pt[k + 1] = pt[k] + ceil_div(h.n, kTile);
    sc[k + 1] = sc[k] + ceil_div((uint64_t)h.cell_cap + 2, kScanTile);
    pr[k + 1] = pr[k] + ceil_div(h.n, kProfTile);
    P.max_rounds = std::max(P.max_rounds, h.max_rounds);
    if (h.profile_bins > 0) P.has_profiles = true;
    if (h.absorb) P.L.absorb = true;
    if (h.mix) P.L.mix = true;
  }
  // prefixes (3 (m + 1) words, padded to an even count), the scan's two control
  // words, then one 64-bit status word per scan tile
  const size_t head = (3 * (size_t)(m + 1) + 1) & ~(size_t)1;
  size_t words = head + 2 + 2 * ((size_t)sc[m] + 1);
  if (cudaMalloc(&P.d_table, sizeof(SimDev*) * m) != cudaSuccess ||
      cudaMalloc(&P.d_pre, words * sizeof(uint32_t)) != cudaSuccess) {
    cudaGetLastError();
    err = "cudaMalloc failed for the launch plan";
    free_plan(P);
    return KMC_ENOMEM;
  }
  std::vector<uint32_t> host(3 * (m + 1));
  std::copy(pt.begin(), pt.end(), host.begin());
  std::copy(sc.begin(), sc.end(), host.begin() + (m + 1));
  std::copy(pr.begin(), pr.end(), host.begin() + 2 * (m + 1));
  KCHECK(cudaMemcpyAsync(P.d_table, table.data(), sizeof(SimDev*) * m, cudaMemcpyHostToDevice, st), err);
  KCHECK(cudaMemsetAsync(P.d_pre, 0, words * sizeof(uint32_t), st), err);
  KCHECK(cudaMemcpyAsync(P.d_pre, host.data(), host.size() * sizeof(uint32_t), cudaMemcpyHostToDevice, st), err);
  KCHECK(cudaStreamSynchronize(st), err);
  LaunchPlan& L = P.L;
  L.b.sims = P.d_table;
  L.b.nsims = m;
  L.b.ptile = P.d_pre;
  L.b.stile_c = P.d_pre + (m + 1);
  L.b.prtile = P.d_pre + 2 * (m + 1);
  L.b.scan_ctl = P.d_pre + head;
  L.b.tile_status = reinterpret_cast<unsigned long long*>(P.d_pre + head + 2);
  L.ptiles = pt[m];
  L.stiles_c = sc[m];
  L.prtiles = pr[m];
  L.edge_blocks = 8 * num_sms();
  search_grids(P.precision, P.K, num_sms(), L.ptiles, L);
  return KMC_OK;
}

int enqueue_step(const Plan& P, cudaStream_t st) {
  int n = launch_sort(P.L, st);
  n += launch_search(P.L, P.precision, P.K, st);
  n += launch_match(P.L, P.max_rounds, st);
  n += launch_push(P.L, st);
  return n;
}

// Diagnostic stepping: phases launched one by one between CUDA events on the
// stream, waiting for each step.
int run_steps_timed(Plan& P, cudaStream_t st, uint64_t nsteps, kmc_sim* s) {
  cudaEvent_t ev[7];
  for (int i = 0; i < 7; ++i) KCHECK(cudaEventCreate(&ev[i]), s->err);
  int rc = KMC_OK;
  for (uint64_t k = 0; k < nsteps && rc == KMC_OK; ++k) {
    int n = 0;
    cudaEventRecord(ev[0], st);
    n += launch_sort(P.L, st);
    cudaEventRecord(ev[1], st);
    n += launch_search(P.L, P.precision, P.K, st, ev + 5);
    cudaEventRecord(ev[2], st);
    n += launch_match(P.L, P.max_rounds, st);
    cudaEventRecord(ev[3], st);
    n += launch_push(P.L, st);
    cudaEventRecord(ev[4], st);
    cudaError_t e = cudaEventSynchronize(ev[4]);
    if (e != cudaSuccess) {
      s->err = std::string("timed step: ") + cudaGetErrorString(e);
      rc = KMC_ECUDA;
      break;
    }
    for (int i = 0; i < 4; ++i) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, ev[i], ev[i + 1]);
      s->phase_ms[i] += ms;
    }
    float ms_slow = 0.f;
    cudaEventElapsedTime(&ms_slow, ev[5], ev[6]);
    s->phase_ms[4] += ms_slow;
    s->timed_steps += 1;
    s->launches += n;
  }
  for (int i = 0; i < 7; ++i) cudaEventDestroy(ev[i]);
  return rc;
}

// Replay the captured step nsteps times (capture on first use; plain launches if
// the stream cannot be captured).  Returns launches through *launched.
int run_steps(Plan& P, cudaStream_t st, uint64_t nsteps, std::string& err, uint64_t* launched) {
  if (!P.graph_tried) {
    P.graph_tried = true;
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      P.launches_per_step = enqueue_step(P, st);
      cudaError_t e = cudaStreamEndCapture(st, &graph);
      if (e == cudaSuccess && graph) {
        if (cudaGraphInstantiate(&P.graph, graph, 0) != cudaSuccess) P.graph = nullptr;
        cudaGraphDestroy(graph);
      }
    }
    cudaGetLastError();
  }
  for (uint64_t i = 0; i < nsteps; ++i) {
    if (P.graph) {
      KCHECK(cudaGraphLaunch(P.graph, st), err);
      *launched += P.launches_per_step;
    } else {
      *launched += enqueue_step(P, st);
    }
  }
  KCHECK(cudaGetLastError(), err);
  return KMC_OK;
}

int ensure_solo(kmc_sim* s) {
  if (s->solo_built) return KMC_OK;
  std::vector<kmc_sim*> one{s};
  int rc = build_plan(s->solo, one, s->stream, s->err);
  if (rc) return rc;
  s->solo_built = true;
  return KMC_OK;
}

int read_dyn(kmc_sim* s, Dyn* out, cudaStream_t st) {
  KCHECK(cudaMemcpyAsync(out, &s->d->d, sizeof(Dyn), cudaMemcpyDeviceToHost, st), s->err);
  KCHECK(cudaStreamSynchronize(st), s->err);
  return KMC_OK;
}

int write_dyn(kmc_sim* s, const Dyn* in, cudaStream_t st) {
  KCHECK(cudaMemcpyAsync(&s->d->d, in, sizeof(Dyn), cudaMemcpyHostToDevice, st), s->err);
  KCHECK(cudaStreamSynchronize(st), s->err);
  return KMC_OK;
}

// Grow the pair buffer of a simulation whose step overflowed it and clear the
// error; the step is re-run later from the unchanged state.
int recover_overflow(kmc_sim* s, Dyn& dy, cudaStream_t st) {
  uint64_t need = (uint64_t)dy.n_raw + dy.n_raw / 4 + 1024;
  uint64_t cap = std::max<uint64_t>(2ull * s->h.edge_cap, need);
  if (cap > 0x7FFFFFFFull) cap = 0x7FFFFFFFull;
  if (cap <= s->h.edge_cap) {
    s->err = "candidate-pair buffer cannot grow further";
    return KMC_EOVERFLOW;
  }
  KCHECK(cudaStreamSynchronize(st), s->err);
  free_edges(s);
  int rc = alloc_edges(s, (uint32_t)cap);
  if (rc) return rc;
  KCHECK(cudaMemcpyAsync(s->d, &s->h, offsetof(SimDev, d), cudaMemcpyHostToDevice, st), s->err);
  dy.status = 0;
  dy.n_raw = 0;
  dy.n_edges = 0;
  for (int r = 0; r < 4; ++r) dy.round_pairs[r] = 0;
  dy.n_pairs = 0;
  dy.adj_used = 0;
  for (int r = 0; r < 5; ++r) dy.wl_len[r] = 0;
  dy.pair_tests = 0;
  dy.fast_tests = 0;
  // the push of the failed step never ran: keep the bound of the previous step
  dy.vmax2_acc = 0;
  return write_dyn(s, &dy, st);
}

int status_code(uint32_t status, std::string& err) {
  if (status & ST_RANDOM) { err = "128 rejected sphere-point draws"; return KMC_ERANDOM; }
  if (status & ST_CELL_OVERFLOW) { err = "cell grid exceeds capacity"; return KMC_EOVERFLOW; }
  if (status & ST_SCAN_WAIT) { err = "a scan tile's wait for its predecessor ran out"; return KMC_ETIMEOUT; }
  if (status & ST_EDGE_OVERFLOW) { err = "candidate-pair buffer overflow"; return KMC_EOVERFLOW; }
  return KMC_OK;
}

int stage_reserve(kmc_sim* s, size_t bytes) {
  if (s->stage_bytes >= bytes) return KMC_OK;
  if (s->stage) {
    cudaStreamSynchronize(s->stream);
    dfree(s, s->stage);
    s->stage = nullptr;
    s->stage_bytes = 0;
  }
  void* p = nullptr;
  int rc = dalloc(s, (char**)&p, bytes);
  if (rc) return rc;
  s->stage = p;
  s->stage_bytes = bytes;
  return KMC_OK;
}

cudaStream_t sim_work_stream(kmc_sim* s) { return s->group ? s->group->stream : s->stream; }

}  // namespace

// =========================================================================== //
extern "C" {

size_t sim_bytes_required(const kmc_params* p) {
  std::string e;
  if (validate(p, e)) return 0;
  return bytes_for(sizes_of(*p));
}

const char* sim_last_error(const kmc_sim* s) {
  if (!s) return g_create_error.c_str();
  return s->err.c_str();
}

int sim_destroy(kmc_sim* s) {
  if (!s) return KMC_OK;
  if (s->group) sim_group_remove(s->group, s);
  cudaStreamSynchronize(s->stream);
  if (s->dom) {
    Domains* D = s->dom;
    for (kmc_sim* m : D->members) sim_destroy(m);
    if (D->graph) cudaGraphExecDestroy(D->graph);
    free_plan(D->plan);
    for (void* q : D->allocs) cudaFree(q);  // the device descriptor D->d is one of them
    delete D;
    s->dom = nullptr;
  }
  free_plan(s->solo);
  for (void* q : s->allocs) cudaFree(q);
  s->allocs.clear();
  if (s->d) cudaFree(s->d);
  if (s->own_stream) cudaStreamDestroy(s->stream);
  delete s;
  return KMC_OK;
}

}  // extern "C"

namespace {

int validate_init(const kmc_params* p, const kmc_init* in, std::string& err) {
  if (!in) { err = "init descriptor is NULL"; return KMC_EINVAL; }
  const bool planar = (p->flags & KMC_FLAG_PLANAR) != 0;
  switch (in->kind) {
    case KMC_INIT_MAXWELL:
      if (!(in->sigma >= 0.0) || !std::isfinite(in->sigma)) { err = "sigma must be finite and >= 0"; return KMC_EINVAL; }
      break;
    case KMC_INIT_EQUAL_SPEED:
      if (!(in->speed >= 0.0) || !std::isfinite(in->speed)) { err = "speed must be finite and >= 0"; return KMC_EINVAL; }
      break;
    case KMC_INIT_BLAST:
      if (planar) { err = "BLAST cannot be planar"; return KMC_EINVAL; }
      if (!(in->sigma >= 0.0) || !std::isfinite(in->sigma) || !(in->sigma_hot >= 0.0) ||
          !std::isfinite(in->sigma_hot)) {
        err = "sigma and sigma_hot must be finite and >= 0";
        return KMC_EINVAL;
      }
      if (in->n_hot > p->n) { err = "n_hot exceeds n"; return KMC_EINVAL; }
      if (!(in->radius > 0.0) || !std::isfinite(in->radius)) { err = "radius must be finite and > 0"; return KMC_EINVAL; }
      for (int a = 0; a < 3; ++a) {
        if (!(in->center[a] - in->radius > 0.0) || !(in->center[a] + in->radius < p->box[a])) {
          err = "the ball must lie strictly inside the box";
          return KMC_EINVAL;
        }
      }
      break;
    default:
      err = "unknown init kind";
      return KMC_EINVAL;
  }
  return KMC_OK;
}

struct Mixture {
  const uint8_t* species;
  uint32_t nspecies;
  const double* mass;
  const double* radius;
};

int validate_mixture(const kmc_params* p, const Mixture* m, std::string& err) {
  if (!m->species || !m->mass || !m->radius) { err = "NULL mixture array"; return KMC_EINVAL; }
  if (m->nspecies < 1 || m->nspecies > 256) { err = "nspecies must be in 1..256"; return KMC_EINVAL; }
  double rmax = 0.0;
  for (uint32_t k = 0; k < m->nspecies; ++k) {
    if (!(m->mass[k] > 0.0) || !std::isfinite(m->mass[k])) { err = "masses must be finite and > 0"; return KMC_EINVAL; }
    if (!(m->radius[k] > 0.0) || !std::isfinite(m->radius[k])) { err = "radii must be finite and > 0"; return KMC_EINVAL; }
    rmax = std::max(rmax, m->radius[k]);
  }
  if (!(rmax + rmax <= p->d0)) { err = "d0 must be at least the largest contact distance 2 max(radius)"; return KMC_EINVAL; }
  return KMC_OK;
}

// shared body of sim_create (src: six state arrays), sim_create_init (init) and
// sim_create_mixture (mix)
int create_impl(const kmc_params* p, const double* const* src6, const uint32_t* last,
                const kmc_init* init, const Mixture* mix, void* stream, kmc_sim** out) {
  if (out) *out = nullptr;
  g_create_error.clear();
  int rc = validate(p, g_create_error);
  if (rc) return rc;
  if (init && (rc = validate_init(p, init, g_create_error))) return rc;
  if (mix && (rc = validate_mixture(p, mix, g_create_error))) return rc;
  if (!out || (!init && (!src6[0] || !src6[1] || !src6[2] || !src6[3] || !src6[4] || !src6[5]))) {
    g_create_error = "NULL array or output pointer";
    return KMC_EINVAL;
  }
  kmc_sim* s = new (std::nothrow) kmc_sim();
  if (!s) { g_create_error = "out of host memory"; return KMC_ENOMEM; }
  s->p = *p;
  if (stream) {
    s->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
      g_create_error = "cudaStreamCreate failed";
      delete s;
      return KMC_ECUDA;
    }
    s->own_stream = true;
  }
  Sizes zs = sizes_of(*p);
  SimDev& h = s->h;
  h.n = p->n;
  for (int a = 0; a < 3; ++a) { h.bc[a] = p->bc[a]; h.box[a] = p->box[a]; }
  h.max_rounds = p->max_rounds ? p->max_rounds : 4;
  h.precision = p->precision;
  h.profile_bins = (int32_t)zs.bins;
  h.profile_every = p->profile_every;
  h.K = p->stencil ? p->stencil : 1;
  h.search_kernel = p->search_kernel;
  h.split_ok = (p->flags & KMC_FLAG_NO_SPLIT) ? 0 : ((p->flags & KMC_FLAG_FORCE_SPLIT) ? 2 : 1);
  h.planar = (p->flags & KMC_FLAG_PLANAR) ? 1 : 0;
  h.scan_wait_test = (p->flags & KMC_FLAG_SCAN_WAIT_TEST) ? 1 : 0;
  h.absorb = (p->bc[0] == KMC_ABSORB || p->bc[1] == KMC_ABSORB || p->bc[2] == KMC_ABSORB) ? 1 : 0;
  h.mix = mix ? 1 : 0;
  h.mix_n = mix ? (int32_t)mix->nspecies : 0;
  h.split_min_occ = p->split_min_occ;
  h.piston_x0 = p->bc[0] == KMC_REFLECT ? p->piston_x0 : p->box[0];
  h.piston_u = p->bc[0] == KMC_REFLECT ? p->piston_u : 0.0;
  h.d0 = p->d0;
  h.dt = p->dt;
  h.d0sq = p->d0 * p->d0;
  h.profile_range = p->profile_range;
  h.cell_scale = p->cell_scale >= 1.0 ? p->cell_scale : 1.0;
  h.seed = p->seed;
  h.cell_cap = zs.cell_cap;
  h.hist_cap = zs.hist_cap;
  h.prof_cap = zs.prof_cap;
  size_t n = p->n;
  auto fail = [&](int code) {
    g_create_error = s->err;
    sim_destroy(s);
    return code;
  };
  if (cudaMalloc(&s->d, sizeof(SimDev)) != cudaSuccess) {
    cudaGetLastError();
    s->err = "cudaMalloc failed for the descriptor";
    return fail(KMC_ENOMEM);
  }
  for (int b = 0; b < 2; ++b) {
    for (int a = 0; a < 3; ++a) {
      if ((rc = dalloc(s, &h.x[b][a], n))) return fail(rc);
      if ((rc = dalloc(s, &h.v[b][a], n))) return fail(rc);
    }
    if ((rc = dalloc(s, &h.id[b], n))) return fail(rc);
    if ((rc = dalloc(s, &h.last[b], n))) return fail(rc);
  }
  if (zs.fp32) {
    if ((rc = dalloc(s, &h.mir, 3 * ((n + 1) / 2)))) return fail(rc);
  }
  if (mix) {
    if ((rc = dalloc(s, &h.species, n))) return fail(rc);
    if ((rc = dalloc(s, &h.sp_mass, mix->nspecies))) return fail(rc);
    if ((rc = dalloc(s, &h.sp_radius, mix->nspecies))) return fail(rc);
  }
  if ((rc = dalloc(s, &h.key, n))) return fail(rc);
  if ((rc = dalloc(s, &h.rank, n))) return fail(rc);
  if ((rc = dalloc(s, &h.src, n))) return fail(rc);
  if ((rc = dalloc(s, &h.vbucket, n))) return fail(rc);
  // cell keys (at most cell_cap), the absorbed particles' key, the total
  if ((rc = dalloc(s, &h.cell_count, (size_t)zs.cell_cap + 2))) return fail(rc);
  if ((rc = dalloc(s, &h.cell_start, (size_t)zs.cell_cap + 2))) return fail(rc);
  if ((rc = dalloc(s, &h.deg, n))) return fail(rc);
  if ((rc = dalloc(s, &h.off, n + 1))) return fail(rc);
  if ((rc = dalloc(s, &h.best, n))) return fail(rc);
  if ((rc = dalloc(s, &h.best_e, n))) return fail(rc);
  if ((rc = dalloc(s, &h.partner, n))) return fail(rc);
  if ((rc = dalloc(s, &h.medge, n))) return fail(rc);
  if ((rc = dalloc(s, &h.pairs, n / 2 + 1))) return fail(rc);
  if ((rc = alloc_edges(s, zs.edge_cap))) return fail(rc);
  if ((rc = dalloc(s, &h.hist, zs.hist_cap))) return fail(rc);
  if (zs.bins) {
    if ((rc = dalloc(s, &h.prof_acc, (size_t)zs.prof_cap * zs.bins * kProfQ))) return fail(rc);
    if ((rc = dalloc(s, &h.prof_step, zs.prof_cap))) return fail(rc);
  }
  cudaStream_t st = s->stream;
  auto ck = [&](cudaError_t e) {
    if (e != cudaSuccess) {
      s->err = std::string("CUDA error during creation: ") + cudaGetErrorString(e);
      return false;
    }
    return true;
  };
  bool ok = true;
  // bad[0]: particles outside the box / non-finite; bad[1]: exhausted init draws
  uint32_t* bad = nullptr;
  if ((rc = dalloc(s, &bad, 2))) return fail(rc);
  ok = ck(cudaMemsetAsync(bad, 0, 2 * sizeof(uint32_t), st));
  if (mix) {
    ok = ok && ck(cudaMemcpyAsync(h.species, mix->species, n, cudaMemcpyDefault, st)) &&
         ck(cudaMemcpyAsync(h.sp_mass, mix->mass, mix->nspecies * sizeof(double), cudaMemcpyDefault, st)) &&
         ck(cudaMemcpyAsync(h.sp_radius, mix->radius, mix->nspecies * sizeof(double), cudaMemcpyDefault, st));
  }
  if (init) {
    InitLaunch L;
    std::memset(&L, 0, sizeof(L));
    L.n = p->n;
    L.kind = (int32_t)init->kind;
    L.planar = h.planar;
    L.n_hot = init->n_hot;
    L.seed = p->seed;
    L.sigma = init->sigma;
    L.speed = init->speed;
    L.sigma_hot = init->sigma_hot;
    L.radius = init->radius;
    for (int a = 0; a < 3; ++a) {
      L.center[a] = init->center[a];
      L.box[a] = p->box[a];
      L.x[a] = h.x[0][a];
      L.v[a] = h.v[0][a];
    }
    L.id = h.id[0];
    L.last = h.last[0];
    L.fails = bad + 1;
    if (ok) launch_init_state(L, st);
    ok = ok && ck(cudaGetLastError());
  } else {
    for (int a = 0; a < 3 && ok; ++a) {
      ok = ck(cudaMemcpyAsync(h.x[0][a], src6[a], n * sizeof(double), cudaMemcpyDefault, st)) &&
           ck(cudaMemcpyAsync(h.v[0][a], src6[3 + a], n * sizeof(double), cudaMemcpyDefault, st));
    }
    std::vector<uint32_t> ids(n);
    for (size_t i = 0; i < n; ++i) ids[i] = (uint32_t)i;
    ok = ok && ck(cudaMemcpyAsync(h.id[0], ids.data(), n * sizeof(uint32_t), cudaMemcpyHostToDevice, st));
    if (last) ok = ok && ck(cudaMemcpyAsync(h.last[0], last, n * sizeof(uint32_t), cudaMemcpyDefault, st));
    else ok = ok && ck(cudaMemsetAsync(h.last[0], 0xFF, n * sizeof(uint32_t), st));
  }
  ok = ok && ck(cudaMemsetAsync(h.cell_count, 0, ((size_t)zs.cell_cap + 2) * sizeof(uint32_t), st));
  ok = ok && ck(cudaMemsetAsync(h.partner, 0xFF, n * sizeof(uint32_t), st));
  ok = ok && ck(cudaMemsetAsync(h.e_slot, 0xFF, (size_t)h.edge_cap * sizeof(uint2), st));
  if (zs.bins) ok = ok && ck(cudaMemsetAsync(h.prof_acc, 0, (size_t)zs.prof_cap * zs.bins * kProfQ * sizeof(long long), st));
  if (!ok) return fail(KMC_ECUDA);
  Dyn dy;
  std::memset(&dy, 0, sizeof(dy));
  dy.step = p->step0;
  dy.steps_left = 0;
  dy.parity = 0;
  if (!ck(cudaMemcpyAsync(s->d, &h, sizeof(SimDev), cudaMemcpyHostToDevice, st))) return fail(KMC_ECUDA);
  if (!ck(cudaMemcpyAsync(&s->d->d, &dy, sizeof(Dyn), cudaMemcpyHostToDevice, st))) return fail(KMC_ECUDA);
  // positions must lie in the box, velocities must be finite
  uint32_t nbad[2] = {0, 0};
  launch_validate(s->d, p->n, bad, st);
  if (!ck(cudaMemcpyAsync(nbad, bad, 2 * sizeof(uint32_t), cudaMemcpyDeviceToHost, st)) ||
      !ck(cudaStreamSynchronize(st)))
    return fail(KMC_ECUDA);
  dfree(s, bad);
  if (nbad[1]) {
    s->err = std::to_string(nbad[1]) + " particle(s) ran out of initialisation draws";
    return fail(KMC_ERANDOM);
  }
  if (nbad[0]) {
    s->err = std::to_string(nbad[0]) + " particle(s) outside the box or with non-finite velocity" +
             std::string(h.planar ? " (or, planar, with vz != 0)" : "") +
             std::string(mix ? " (or with a species index >= nspecies)" : "");
    return fail(KMC_EINVAL);
  }
  if ((rc = ensure_solo(s))) return fail(rc);
  launch_init_grid(s->solo.L, st);
  if (!ck(cudaGetLastError()) || !ck(cudaStreamSynchronize(st))) return fail(KMC_ECUDA);
  *out = s;
  return KMC_OK;
}

// ---- domain decomposition (Sec. 4) ------------------------------------------ //
template <typename T>
int dom_alloc(Domains* D, T** out, size_t count, std::string& err) {
  void* ptr = nullptr;
  const cudaError_t e = cudaMalloc(&ptr, std::max<size_t>(count * sizeof(T), 16));
  if (e != cudaSuccess) {
    cudaGetLastError();
    err = std::string("cudaMalloc failed: ") + cudaGetErrorString(e);
    return KMC_ENOMEM;
  }
  D->allocs.push_back(ptr);
  *out = (T*)ptr;
  return KMC_OK;
}

int dom_create(const kmc_params* p, uint32_t ndom, const double* const* src6, const uint32_t* last,
               void* stream, kmc_sim** out) {
  if (out) *out = nullptr;
  g_create_error.clear();
  int rc = validate(p, g_create_error);
  if (rc) return rc;
  if (ndom < 1 || ndom > (uint32_t)kMaxDomains) { g_create_error = "ndomains must be in 1..64"; return KMC_EINVAL; }
  for (int a = 0; a < 3; ++a)
    if (p->bc[a] == KMC_ABSORB) { g_create_error = "a decomposition has no absorbing walls"; return KMC_EINVAL; }
  if (p->profile_bins != 0) { g_create_error = "a decomposition keeps no profiles (profile_bins must be 0)"; return KMC_EINVAL; }
  if (!out || !src6[0] || !src6[1] || !src6[2] || !src6[3] || !src6[4] || !src6[5]) {
    g_create_error = "NULL array or output pointer";
    return KMC_EINVAL;
  }
  kmc_sim* s = new (std::nothrow) kmc_sim();
  if (!s) { g_create_error = "out of host memory"; return KMC_ENOMEM; }
  Domains* D = new (std::nothrow) Domains();
  if (!D) { delete s; g_create_error = "out of host memory"; return KMC_ENOMEM; }
  s->dom = D;
  s->p = *p;
  s->h.n = p->n;
  s->h.precision = p->precision;
  s->h.hist_cap = p->history_cap ? p->history_cap : 4096u;
  if (stream) {
    s->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete D;
      delete s;
      g_create_error = "cudaStreamCreate failed";
      return KMC_ECUDA;
    }
    s->own_stream = true;
  }
  auto fail = [&](int code) {
    g_create_error = s->err.empty() ? g_create_error : s->err;
    sim_destroy(s);
    return code;
  };
  const size_t n = p->n;
  cudaStream_t st = s->stream;
  DomainDev& h = D->h;
  char* state = nullptr;
  if ((rc = dom_alloc(D, &state, 52 * n, s->err))) return fail(rc);
  D->state = state;
  for (int a = 0; a < 3; ++a) {
    h.x[a] = (double*)state + (size_t)a * n;
    h.v[a] = (double*)state + (size_t)(3 + a) * n;
  }
  h.last = (uint32_t*)((double*)state + 6 * n);
  bool ok = true;
  for (int a = 0; a < 3 && ok; ++a) {
    ok = cudaMemcpyAsync(h.x[a], src6[a], n * sizeof(double), cudaMemcpyDefault, st) == cudaSuccess &&
         cudaMemcpyAsync(h.v[a], src6[3 + a], n * sizeof(double), cudaMemcpyDefault, st) == cudaSuccess;
  }
  if (ok && last) ok = cudaMemcpyAsync(h.last, last, n * sizeof(uint32_t), cudaMemcpyDefault, st) == cudaSuccess;
  if (ok && !last) ok = cudaMemsetAsync(h.last, 0xFF, n * sizeof(uint32_t), st) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    s->err = "copying the initial state failed";
    return fail(KMC_ECUDA);
  }
  // the domains: simulations of the whole box over every particle slot (ids 0..n-1),
  // slots outside the domain absent (the absorbed-particle marker); each step's grid,
  // speed split included, is built afresh from the particles a domain holds
  kmc_params q = *p;
  // a domain cannot regrow its candidate-pair buffer mid-run (the others have moved
  // on): start it at one pair per particle slot unless the caller chose a size
  if (q.edge_cap == 0) q.edge_cap = std::max<uint32_t>(4096u, p->n);
  const double* mem6[6] = {h.x[0], h.x[1], h.x[2], h.v[0], h.v[1], h.v[2]};
  for (uint32_t k = 0; k < ndom; ++k) {
    kmc_sim* m = nullptr;
    rc = create_impl(&q, mem6, h.last, nullptr, nullptr, st, &m);
    if (rc) {
      s->err = g_create_error;
      return fail(rc);
    }
    D->members.push_back(m);
    m->h.absorb = 1;
    const int32_t one = 1;
    if (cudaMemcpyAsync(&m->d->absorb, &one, sizeof(one), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      cudaGetLastError();
      s->err = "descriptor update failed";
      return fail(KMC_ECUDA);
    }
  }
  if ((rc = build_plan(D->plan, D->members, st, s->err))) return fail(rc);
  h.n = p->n;
  h.P = (int32_t)ndom;
  h.periodic_x = p->bc[0] == KMC_PERIODIC ? 1 : 0;
  h.Lx = p->box[0];
  const double xmax = p->bc[0] == KMC_REFLECT ? std::max(p->box[0], p->piston_x0) : p->box[0];
  for (uint32_t k = 0; k <= ndom; ++k) h.X[k] = xmax * (double)k / (double)ndom;
  h.d0 = p->d0;
  h.dt = p->dt;
  h.hist_cap = s->h.hist_cap;
  if ((rc = dom_alloc(D, &h.owner, n, s->err)) || (rc = dom_alloc(D, &h.bestG, n, s->err)) ||
      (rc = dom_alloc(D, &h.partnerG, n, s->err)) || (rc = dom_alloc(D, &h.partner_out, n, s->err)) ||
      (rc = dom_alloc(D, &h.loc, (size_t)ndom * n, s->err)) ||
      (rc = dom_alloc(D, &h.hist, h.hist_cap, s->err)) || (rc = dom_alloc(D, &D->d, 1, s->err)))
    return fail(rc);
  ok = cudaMemsetAsync(h.partner_out, 0xFF, n * sizeof(uint32_t), st) == cudaSuccess &&
       cudaMemsetAsync(h.bestG, 0xFF, n * sizeof(uint32_t), st) == cudaSuccess &&
       cudaMemsetAsync(h.partnerG, 0xFF, n * sizeof(uint32_t), st) == cudaSuccess &&
       cudaMemcpyAsync(D->d, &h, sizeof(DomainDev), cudaMemcpyHostToDevice, st) == cudaSuccess &&
       cudaStreamSynchronize(st) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    s->err = "initialising the exchange buffers failed";
    return fail(KMC_ECUDA);
  }
  *out = s;
  return KMC_OK;
}

int dom_enqueue(Domains* D, cudaStream_t st) {
  const Plan& P = D->plan;
  return launch_domain_step(P.L, D->d, D->h.n, P.precision, P.K, P.max_rounds, st);
}

int dom_step(kmc_sim* s, uint32_t nsteps) {
  Domains* D = s->dom;
  cudaStream_t st = s->stream;
  for (kmc_sim* m : D->members) launch_add_steps(m->d, nsteps, st);
  s->launches += D->members.size();
  if (!D->graph_tried) {
    D->graph_tried = true;
    cudaGraph_t graph = nullptr;
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      D->launches_per_step = dom_enqueue(D, st);
      const cudaError_t e = cudaStreamEndCapture(st, &graph);
      if (e == cudaSuccess && graph) {
        if (cudaGraphInstantiate(&D->graph, graph, 0) != cudaSuccess) D->graph = nullptr;
        cudaGraphDestroy(graph);
      }
    }
    cudaGetLastError();
  }
  for (uint32_t i = 0; i < nsteps; ++i) {
    if (D->graph) {
      KCHECK(cudaGraphLaunch(D->graph, st), s->err);
      s->launches += D->launches_per_step;
    } else {
      s->launches += dom_enqueue(D, st);
    }
  }
  KCHECK(cudaGetLastError(), s->err);
  return KMC_OK;
}

int dom_sync(kmc_sim* s) {
  KCHECK(cudaStreamSynchronize(s->stream), s->err);
  for (kmc_sim* m : s->dom->members) {
    Dyn dy;
    int rc = read_dyn(m, &dy, s->stream);
    if (rc) { s->err = m->err; return rc; }
    if (dy.status) {
      rc = status_code(dy.status, s->err);
      if (dy.status & ST_EDGE_OVERFLOW)
        s->err = "candidate-pair buffer of a domain overflowed: create it with a larger edge_cap";
      return rc;
    }
  }
  return KMC_OK;
}

int64_t dom_observe(kmc_sim* s, int what, void* dst, size_t dst_bytes) {
  Domains* D = s->dom;
  cudaStream_t st = s->stream;
  const uint32_t n = D->h.n;
  int rc;
  switch (what) {
    case KMC_OBS_STATE: {
      const size_t need = (size_t)n * 52;
      if (dst_bytes < need) { s->err = "dst too small for STATE"; return KMC_EINVAL; }
      KCHECK(cudaMemcpyAsync(dst, D->state, need, cudaMemcpyDefault, st), s->err);
      KCHECK(cudaStreamSynchronize(st), s->err);
      return 1;
    }
    case KMC_OBS_PARTNERS: {
      const size_t need = (size_t)n * sizeof(uint32_t);
      if (dst_bytes < need) { s->err = "dst too small for PARTNERS"; return KMC_EINVAL; }
      KCHECK(cudaMemcpyAsync(dst, D->h.partner_out, need, cudaMemcpyDefault, st), s->err);
      KCHECK(cudaStreamSynchronize(st), s->err);
      return n;
    }
    case KMC_OBS_EDGES: {
      const uint32_t cap = (uint32_t)std::min<size_t>(dst_bytes / sizeof(uint2), 0xFFFFFFFFu);
      if ((rc = stage_reserve(s, (size_t)cap * sizeof(uint2) + 16))) return rc;
      uint32_t* cnt = (uint32_t*)s->stage;
      uint2* buf = (uint2*)((char*)s->stage + 16);
      KCHECK(cudaMemsetAsync(cnt, 0, sizeof(uint32_t), st), s->err);
      launch_domain_edges(D->plan.L, D->d, cap, buf, cnt, st);
      KCHECK(cudaGetLastError(), s->err);
      uint32_t count = 0;
      KCHECK(cudaMemcpyAsync(&count, cnt, sizeof(uint32_t), cudaMemcpyDeviceToHost, st), s->err);
      KCHECK(cudaStreamSynchronize(st), s->err);
      if (count > cap) { s->err = "dst too small for EDGES"; return KMC_EINVAL; }
      KCHECK(cudaMemcpyAsync(dst, buf, (size_t)count * sizeof(uint2), cudaMemcpyDefault, st), s->err);
      KCHECK(cudaStreamSynchronize(st), s->err);
      return count;
    }
    case KMC_OBS_COUNTS: {
      uint64_t hc = 0;
      KCHECK(cudaMemcpyAsync(&hc, &D->d->hist_count, sizeof(hc), cudaMemcpyDeviceToHost, st), s->err);
      KCHECK(cudaStreamSynchronize(st), s->err);
      uint64_t avail = hc - D->hist_read, first = D->hist_read;
      if (avail > D->h.hist_cap) {
        first = hc - D->h.hist_cap;
        avail = D->h.hist_cap;
      }
      if (avail > dst_bytes / sizeof(kmc_step_counts)) { s->err = "dst too small for COUNTS"; return KMC_EINVAL; }
      kmc_step_counts* o = (kmc_step_counts*)dst;
      for (uint64_t i = 0; i < avail;) {
        const uint64_t slot = (first + i) % D->h.hist_cap;
        const uint64_t run = std::min<uint64_t>(avail - i, D->h.hist_cap - slot);
        KCHECK(cudaMemcpyAsync(o + i, D->h.hist + slot, run * sizeof(kmc_step_counts), cudaMemcpyDefault, st), s->err);
        i += run;
      }
      KCHECK(cudaStreamSynchronize(st), s->err);
      D->hist_read = hc;
      return (int64_t)avail;
    }
    case KMC_OBS_DOMAINS: {
      const size_t need = (size_t)2 * D->h.P * sizeof(uint32_t);
      if (dst_bytes < need) { s->err = "dst too small for DOMAINS"; return KMC_EINVAL; }
      std::vector<uint32_t> v(2 * D->h.P);
      KCHECK(cudaMemcpyAsync(v.data(), D->d->owned, D->h.P * sizeof(uint32_t), cudaMemcpyDeviceToHost, st), s->err);
      KCHECK(cudaMemcpyAsync(v.data() + D->h.P, D->d->ghosts, D->h.P * sizeof(uint32_t), cudaMemcpyDeviceToHost, st), s->err);
      KCHECK(cudaStreamSynchronize(st), s->err);
      KCHECK(cudaMemcpy(dst, v.data(), need, cudaMemcpyDefault), s->err);
      return 2 * D->h.P;
    }
    case KMC_OBS_VMAX: {
      if (dst_bytes < sizeof(double)) { s->err = "dst too small for VMAX"; return KMC_EINVAL; }
      if ((rc = stage_reserve(s, 16))) return rc;
      unsigned long long* acc = (unsigned long long*)s->stage;
      double* val = (double*)((char*)s->stage + 8);
      launch_domain_vmax(D->d, acc, val, st);
      KCHECK(cudaGetLastError(), s->err);
      KCHECK(cudaMemcpyAsync(dst, val, sizeof(double), cudaMemcpyDefault, st), s->err);
      KCHECK(cudaStreamSynchronize(st), s->err);
      return 1;
    }
    case KMC_OBS_STEP:
      return sim_observe(D->members[0], what, dst, dst_bytes);
    case KMC_OBS_LAUNCHES: {
      if (dst_bytes < sizeof(uint64_t)) { s->err = "dst too small for LAUNCHES"; return KMC_EINVAL; }
      KCHECK(cudaMemcpy(dst, &s->launches, sizeof(uint64_t), cudaMemcpyDefault), s->err);
      return 1;
    }
    case KMC_OBS_PROFILES:
      return 0;
    default:
      s->err = "observable not available for a decomposition";
      return KMC_EINVAL;
  }
}

}  // namespace

extern "C" {

int sim_create(const kmc_params* p, const double* x, const double* y, const double* z,
               const double* vx, const double* vy, const double* vz, const uint32_t* last,
               void* stream, kmc_sim** out) {
  const double* src[6] = {x, y, z, vx, vy, vz};
  return create_impl(p, src, last, nullptr, nullptr, stream, out);
}

int sim_create_mixture(const kmc_params* p, const double* x, const double* y, const double* z,
                       const double* vx, const double* vy, const double* vz, const uint32_t* last,
                       const uint8_t* species, uint32_t nspecies, const double* mass,
                       const double* radius, void* stream, kmc_sim** out) {
  const double* src[6] = {x, y, z, vx, vy, vz};
  Mixture m{species, nspecies, mass, radius};
  return create_impl(p, src, last, nullptr, &m, stream, out);
}

int sim_create_domains(const kmc_params* p, uint32_t ndomains, const double* x, const double* y,
                       const double* z, const double* vx, const double* vy, const double* vz,
                       const uint32_t* last, void* stream, kmc_sim** out) {
  const double* src6[6] = {x, y, z, vx, vy, vz};
  return dom_create(p, ndomains, src6, last, stream, out);
}

int sim_create_init(const kmc_params* p, const kmc_init* init, void* stream, kmc_sim** out) {
  if (out) *out = nullptr;
  if (!init) {
    g_create_error = "init descriptor is NULL";
    return KMC_EINVAL;
  }
  return create_impl(p, nullptr, nullptr, init, nullptr, stream, out);
}

int sim_step(kmc_sim* s, uint32_t nsteps) {
  if (!s) return KMC_EINVAL;
  if (s->group) { s->err = "simulation belongs to a group"; return KMC_ESTATE; }
  if (nsteps == 0) return KMC_OK;
  if (s->dom) return dom_step(s, nsteps);
  int rc = ensure_solo(s);
  if (rc) return rc;
  launch_add_steps(s->d, nsteps, s->stream);
  s->launches += 1;
  if (s->timing) return run_steps_timed(s->solo, s->stream, nsteps, s);
  return run_steps(s->solo, s->stream, nsteps, s->err, &s->launches);
}

int sim_set_timing(kmc_sim* s, int enable) {
  if (!s) return KMC_EINVAL;
  s->timing = enable != 0;
  return KMC_OK;
}

int sim_sync(kmc_sim* s) {
  if (!s) return KMC_EINVAL;
  if (s->dom) return dom_sync(s);
  if (s->group) {
    // the group's sync knows how many group steps a recovering member missed
    const int rc = sim_group_sync(s->group);
    if (rc) s->err = s->group->err;
    return rc;
  }
  cudaStream_t st = sim_work_stream(s);
  for (int attempt = 0; attempt < 64; ++attempt) {
    KCHECK(cudaStreamSynchronize(st), s->err);
    Dyn dy;
    int rc = read_dyn(s, &dy, st);
    if (rc) return rc;
    if (dy.status == 0) return KMC_OK;
    if (dy.status == ST_EDGE_OVERFLOW) {
      if ((rc = recover_overflow(s, dy, st))) return rc;
      if (dy.steps_left) {
        if ((rc = run_steps(s->solo, st, dy.steps_left, s->err, &s->launches))) return rc;
      }
      continue;
    }
    return status_code(dy.status, s->err);
  }
  s->err = "overflow recovery did not converge";
  return KMC_EOVERFLOW;
}

int64_t sim_observe(kmc_sim* s, int what, void* dst, size_t dst_bytes) {
  if (!s) return KMC_EINVAL;
  if (!dst) { s->err = "dst is NULL"; return KMC_EINVAL; }
  if (s->dom) return dom_observe(s, what, dst, dst_bytes);
  cudaStream_t st = sim_work_stream(s);
  uint32_t n = s->h.n;
  bool dev = is_device_ptr(dst);
  int rc;
  switch (what) {
    case KMC_OBS_STATE: {
      size_t need = (size_t)n * (6 * sizeof(double) + sizeof(uint32_t));
      if (dst_bytes < need) { s->err = "dst too small for STATE"; return KMC_EINVAL; }
      void* target = dst;
      if (!dev) {
        if ((rc = stage_reserve(s, need))) return rc;
        target = s->stage;
      }
      launch_gather_state(s->d, n, target, st);
      KCHECK(cudaGetLastError(), s->err);
      if (!dev) {
        KCHECK(cudaMemcpyAsync(dst, target, need, cudaMemcpyDeviceToHost, st), s->err);
        KCHECK(cudaStreamSynchronize(st), s->err);
      }
      return 1;
    }
    case KMC_OBS_PARTNERS: {
      size_t need = (size_t)n * sizeof(uint32_t);
      if (dst_bytes < need) { s->err = "dst too small for PARTNERS"; return KMC_EINVAL; }
      void* target = dst;
      if (!dev) {
        if ((rc = stage_reserve(s, need))) return rc;
        target = s->stage;
      }
      launch_gather_partners(s->d, n, (uint32_t*)target, st);
      KCHECK(cudaGetLastError(), s->err);
      if (!dev) {
        KCHECK(cudaMemcpyAsync(dst, target, need, cudaMemcpyDeviceToHost, st), s->err);
        KCHECK(cudaStreamSynchronize(st), s->err);
      }
      return n;
    }
    case KMC_OBS_EDGES: {
      uint32_t cap = (uint32_t)std::min<size_t>(dst_bytes / sizeof(uint2), 0xFFFFFFFFu);
      size_t need = (size_t)cap * sizeof(uint2) + 16;
      if ((rc = stage_reserve(s, need))) return rc;
      uint32_t* cnt = (uint32_t*)s->stage;
      uint2* buf = (uint2*)((char*)s->stage + 16);
      KCHECK(cudaMemsetAsync(cnt, 0, sizeof(uint32_t), st), s->err);
      launch_gather_edges(s->d, cap, buf, cnt, st);
      KCHECK(cudaGetLastError(), s->err);
      uint32_t count = 0;
      KCHECK(cudaMemcpyAsync(&count, cnt, sizeof(uint32_t), cudaMemcpyDeviceToHost, st), s->err);
      KCHECK(cudaStreamSynchronize(st), s->err);
      if (count > cap) { s->err = "dst too small for EDGES"; return KMC_EINVAL; }
      KCHECK(cudaMemcpyAsync(dst, buf, (size_t)count * sizeof(uint2), cudaMemcpyDefault, st), s->err);
      KCHECK(cudaStreamSynchronize(st), s->err);
      return count;
    }
    case KMC_OBS_COUNTS: {
      Dyn dy;
      if ((rc = read_dyn(s, &dy, st))) return rc;
      uint64_t avail = dy.hist_count - s->hist_read;
      uint64_t first = s->hist_read;
      if (avail > s->h.hist_cap) {
        first = dy.hist_count - s->h.hist_cap;
        avail = s->h.hist_cap;
      }
      uint64_t fit = dst_bytes / sizeof(kmc_step_counts);
      if (avail > fit) { s->err = "dst too small for COUNTS"; return KMC_EINVAL; }
      kmc_step_counts* o = (kmc_step_counts*)dst;
      for (uint64_t i = 0; i < avail;) {
        uint64_t slot = (first + i) % s->h.hist_cap;
        uint64_t run = std::min<uint64_t>(avail - i, s->h.hist_cap - slot);
        KCHECK(cudaMemcpyAsync(o + i, s->h.hist + slot, run * sizeof(kmc_step_counts), cudaMemcpyDefault, st), s->err);
        i += run;
      }
      KCHECK(cudaStreamSynchronize(st), s->err);
      s->hist_read = dy.hist_count;
      return (int64_t)avail;
    }
    case KMC_OBS_PROFILES: {
      if (s->h.profile_bins == 0) return 0;
      Dyn dy;
      if ((rc = read_dyn(s, &dy, st))) return rc;
      uint64_t avail = dy.prof_count - s->prof_read;
      uint64_t first = s->prof_read;
      if (avail > s->h.prof_cap) {
        first = dy.prof_count - s->h.prof_cap;
        avail = s->h.prof_cap;
      }
      size_t per = (size_t)s->h.profile_bins * 7 * sizeof(double);
      if (avail * per > dst_bytes) { s->err = "dst too small for PROFILES"; return KMC_EINVAL; }
      if (avail == 0) return 0;
      if ((rc = stage_reserve(s, avail * per))) return rc;
      launch_profile_convert(s->d, (uint32_t)(first % s->h.prof_cap), (uint32_t)avail,
                             (uint32_t)s->h.profile_bins, (double*)s->stage, st);
      KCHECK(cudaGetLastError(), s->err);
      KCHECK(cudaMemcpyAsync(dst, s->stage, avail * per, cudaMemcpyDefault, st), s->err);
      KCHECK(cudaStreamSynchronize(st), s->err);
      s->prof_read = dy.prof_count;
      return (int64_t)avail;
    }
    case KMC_OBS_LAUNCHES: {
      if (dst_bytes < sizeof(uint64_t)) { s->err = "dst too small for LAUNCHES"; return KMC_EINVAL; }
      KCHECK(cudaMemcpy(dst, &s->launches, sizeof(uint64_t), cudaMemcpyDefault), s->err);
      return 1;
    }
    case KMC_OBS_PHASE_MS: {
      if (dst_bytes < 5 * sizeof(double)) { s->err = "dst too small for PHASE_MS"; return KMC_EINVAL; }
      double v[6] = {s->phase_ms[0], s->phase_ms[1], s->phase_ms[2], s->phase_ms[3],
                     (double)s->timed_steps, s->phase_ms[4]};
      const size_t m = dst_bytes >= sizeof(v) ? 6 : 5;
      KCHECK(cudaMemcpy(dst, v, m * sizeof(double), cudaMemcpyDefault), s->err);
      return (int64_t)m;
    }
    case KMC_OBS_VMAX: {
      if (dst_bytes < sizeof(double)) { s->err = "dst too small for VMAX"; return KMC_EINVAL; }
      if ((rc = stage_reserve(s, 16))) return rc;
      unsigned long long* acc = (unsigned long long*)s->stage;
      double* val = (double*)((char*)s->stage + 8);
      launch_vmax_exact(s->d, acc, dev ? (double*)dst : val, st);
      KCHECK(cudaGetLastError(), s->err);
      if (!dev) {
        KCHECK(cudaMemcpyAsync(dst, val, sizeof(double), cudaMemcpyDeviceToHost, st), s->err);
        KCHECK(cudaStreamSynchronize(st), s->err);
      }
      return 1;
    }
    case KMC_OBS_STEP: {
      if (dst_bytes < sizeof(uint64_t)) { s->err = "dst too small for STEP"; return KMC_EINVAL; }
      Dyn dy;
      if ((rc = read_dyn(s, &dy, st))) return rc;
      KCHECK(cudaMemcpyAsync(dst, &dy.step, sizeof(uint64_t), cudaMemcpyDefault, st), s->err);
      KCHECK(cudaStreamSynchronize(st), s->err);
      return 1;
    }
    default:
      s->err = "unknown observable";
      return KMC_EINVAL;
  }
}

// ---- groups ------------------------------------------------------------------ //
int sim_group_create(kmc_sim* const* sims, uint32_t count, void* stream, kmc_group** out) {
  if (out) *out = nullptr;
  if (!sims || count == 0 || !out || count > (uint32_t)kMaxGroup) {
    g_create_error = "bad group arguments";
    return KMC_EINVAL;
  }
  for (uint32_t i = 0; i < count; ++i) {
    if (!sims[i] || sims[i]->group) { g_create_error = "member NULL or already grouped"; return KMC_EINVAL; }
    if (sims[i]->dom) { g_create_error = "a decomposition cannot join a group"; return KMC_EINVAL; }
    if (sims[i]->h.precision != sims[0]->h.precision || sims[i]->h.K != sims[0]->h.K) {
      g_create_error = "members must share precision and stencil";
      return KMC_EINVAL;
    }
    for (uint32_t j = 0; j < i; ++j)
      if (sims[j] == sims[i]) { g_create_error = "duplicate member"; return KMC_EINVAL; }
  }
  kmc_group* g = new (std::nothrow) kmc_group();
  if (!g) return KMC_ENOMEM;
  if (stream) {
    g->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete g;
      g_create_error = "cudaStreamCreate failed";
      return KMC_ECUDA;
    }
    g->own_stream = true;
  }
  for (uint32_t i = 0; i < count; ++i) {
    cudaStreamSynchronize(sims[i]->stream);
    Dyn dy;
    if (read_dyn(sims[i], &dy, sims[i]->stream) == KMC_OK) sims[i]->sync_step = dy.step;
    sims[i]->issued_base = 0;
    sims[i]->group = g;
    g->members.push_back(sims[i]);
  }
  *out = g;
  return KMC_OK;
}

int sim_group_add(kmc_group* g, kmc_sim* s) {
  if (!g || !s) return KMC_EINVAL;
  if (s->group) { g->err = "simulation already grouped"; return KMC_EINVAL; }
  if (s->dom) { g->err = "a decomposition cannot join a group"; return KMC_EINVAL; }
  if (g->members.size() >= (size_t)kMaxGroup) { g->err = "group full"; return KMC_EINVAL; }
  if (!g->members.empty() && (s->h.precision != g->members[0]->h.precision || s->h.K != g->members[0]->h.K)) {
    g->err = "members must share precision and stencil";
    return KMC_EINVAL;
  }
  cudaStreamSynchronize(s->stream);
  Dyn dy;
  int rc = read_dyn(s, &dy, s->stream);
  if (rc) return rc;
  s->sync_step = dy.step;
  s->issued_base = g->issued;
  s->group = g;
  g->members.push_back(s);
  g->built = false;
  return KMC_OK;
}

int sim_group_remove(kmc_group* g, kmc_sim* s) {
  if (!g || !s || s->group != g) return KMC_EINVAL;
  cudaStreamSynchronize(g->stream);
  g->members.erase(std::remove(g->members.begin(), g->members.end(), s), g->members.end());
  s->group = nullptr;
  g->built = false;
  return KMC_OK;
}

int sim_group_budget(kmc_group* g, kmc_sim* s, uint32_t nsteps) {
  if (!g || !s || s->group != g) return KMC_EINVAL;
  launch_add_steps(s->d, nsteps, g->stream);
  s->launches += 1;
  KCHECK(cudaGetLastError(), g->err);
  return KMC_OK;
}

int sim_group_step(kmc_group* g, uint32_t nsteps) {
  if (!g) return KMC_EINVAL;
  if (g->members.empty() || nsteps == 0) return KMC_OK;
  if (!g->built) {
    cudaStreamSynchronize(g->stream);
    int rc = build_plan(g->plan, g->members, g->stream, g->err);
    if (rc) return rc;
    g->built = true;
  }
  uint64_t launched = 0;
  int rc = run_steps(g->plan, g->stream, nsteps, g->err, &launched);
  for (kmc_sim* s : g->members) s->launches += launched;
  g->issued += nsteps;
  return rc;
}

int64_t sim_group_steps_left(kmc_group* g, kmc_sim* s) {
  if (!g || !s || s->group != g) return KMC_EINVAL;
  Dyn dy;
  int rc = read_dyn(s, &dy, g->stream);
  if (rc) return rc;
  return (int64_t)dy.steps_left;
}

int sim_group_sync(kmc_group* g) {
  if (!g) return KMC_EINVAL;
  int worst = KMC_OK;
  for (int attempt = 0; attempt < 64; ++attempt) {
    KCHECK(cudaStreamSynchronize(g->stream), g->err);
    bool rerun = false;
    worst = KMC_OK;
    for (kmc_sim* s : g->members) {
      Dyn dy;
      int rc = read_dyn(s, &dy, g->stream);
      if (rc) return rc;
      if (dy.status == 0) {
        s->sync_step = dy.step;
        s->issued_base = 0;
        continue;
      }
      if (dy.status == ST_EDGE_OVERFLOW) {
        rc = recover_overflow(s, dy, g->stream);
        if (rc == KMC_OK) {
          // the group's steps after the overflow skipped this member: it runs the ones
          // it missed since the last sync on its own (within its budget), so that a
          // sync leaves every member where the group's steps should have taken it
          const uint64_t window = g->issued > s->issued_base ? g->issued - s->issued_base : 0;
          const uint64_t taken = dy.step - s->sync_step;
          uint64_t lost = window > taken ? window - taken : 0;
          if (lost > dy.steps_left) lost = dy.steps_left;
          if (lost) {
            rc = ensure_solo(s);
            if (rc == KMC_OK) rc = run_steps(s->solo, g->stream, lost, s->err, &s->launches);
            rerun = true;
          }
        }
      } else {
        rc = status_code(dy.status, s->err);
      }
      if (rc) {
        g->err = s->err;
        worst = rc;
      }
    }
    if (!rerun) {
      // the next sync counts the group's steps from here for every member, including
      // one whose recovery failed (its issued_base must not stay above the new count)
      g->issued = 0;
      for (kmc_sim* s : g->members) {
        Dyn dy;
        if (s->issued_base != 0 && read_dyn(s, &dy, g->stream) == KMC_OK) s->sync_step = dy.step;
        s->issued_base = 0;
      }
      return worst;
    }
  }
  g->err = "overflow recovery did not converge";
  return KMC_EOVERFLOW;
}

int sim_group_destroy(kmc_group* g) {
  if (!g) return KMC_OK;
  cudaStreamSynchronize(g->stream);
  for (kmc_sim* s : g->members) s->group = nullptr;
  free_plan(g->plan);
  if (g->own_stream) cudaStreamDestroy(g->stream);
  delete g;
  return KMC_OK;
}

}  // extern "C"
