// kmc_noalloc.cu -- x-profile of a particle state for callers that cannot allocate.
//
// Who needs this.  Some host programs cannot call cudaMalloc at the point where they
// want an observable: an application that hands all device memory to its own pool
// allocator and forbids outside allocations, an in-situ analysis hook running
// inside a host code's time loop where an allocation would synchronise the device,
// or a tool that only receives device pointers to someone else's arrays.  This
// entry point computes the same 7 x bins profile as KMC_OBS_PROFILES (count,
// sum v, sum v^2 per x bin) from caller-owned device arrays, and allocates nothing:
// its only scratch is the fixed-size array below, which lives in the library's
// device image.
//
// The scratch array holds kStaticBins x 19 int64 fixed-point counters (38,912
// bytes).  Every GPU that loads the library keeps its own copy until the process
// exits.  All calls on a device share it and it keeps the last call's contents;
// each call clears the counters it uses before accumulating.  Two calls whose work
// overlaps on the GPU (different streams, no ordering between them) race on the
// counters and give wrong sums: order such calls on one stream or with events.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "kmc_internal.cuh"

namespace {

constexpr int kStaticBins = 256;  // largest supported number of bins
constexpr int kQ = 19;            // counters per bin: count, 3 x 3 digits of sum v, of sum v^2
constexpr int kMaxDevices = 64;

}  // namespace

// fixed-point profile counters (see the file comment): 256 x 19 x 8 = 38,912 bytes
static __device__ __align__(256) long long kmc_profile_scratch[kStaticBins * kQ];

namespace {

// |q| * 2^64 truncated, as three 32-bit digits with the sign of q (|q| < 2^31)
__device__ __forceinline__ void digits3(double q, long long d[3]) {
  unsigned long long bits = (unsigned long long)__double_as_longlong(q);
  bool neg = (bits >> 63) != 0;
  int ex = (int)((bits >> 52) & 0x7FF);
  d[0] = d[1] = d[2] = 0;
  if (ex == 0) return;
  unsigned long long man = (bits & ((1ull << 52) - 1)) | (1ull << 52);
  int sh = ex - 1075 + 64;
  unsigned __int128 f;
  if (sh >= 0) f = (unsigned __int128)man << (sh > 42 ? 42 : sh);
  else if (sh > -64) f = (unsigned __int128)(man >> (-sh));
  else f = 0;
  long long d0 = (long long)(uint32_t)f, d1 = (long long)(uint32_t)(f >> 32),
            d2 = (long long)(uint32_t)(f >> 64);
  if (neg) { d0 = -d0; d1 = -d1; d2 = -d2; }
  d[0] = d0; d[1] = d1; d[2] = d2;
}

__global__ void k_static_clear(long long* acc, int count) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) acc[i] = 0;
}

// per-block shared-memory counters, then one global atomic per non-zero counter
__global__ void __launch_bounds__(256) k_static_profile(const double* __restrict__ x,
                                                        const double* __restrict__ vx,
                                                        const double* __restrict__ vy,
                                                        const double* __restrict__ vz, uint32_t n,
                                                        int nb, double range, long long* acc) {
  extern __shared__ long long sh[];
  for (int i = threadIdx.x; i < nb * kQ; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  const double scale = kmc::ddiv((double)nb, range);
  const double* vel[3] = {vx, vy, vz};
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    double xp = x[p];
    if (!(xp >= 0.0)) continue;
    double f = kmc::dmul(xp, scale);
    if (f >= (double)nb) continue;
    long long* q = sh + (int)f * kQ;
    atomicAdd((unsigned long long*)&q[0], 1ull);
    for (int a = 0; a < 3; ++a) {
      double v = vel[a][p];
      long long d[3];
      digits3(v, d);
      for (int c = 0; c < 3; ++c) atomicAdd((unsigned long long*)&q[1 + 3 * a + c], (unsigned long long)d[c]);
      digits3(kmc::dmul(v, v), d);
      for (int c = 0; c < 3; ++c) atomicAdd((unsigned long long*)&q[10 + 3 * a + c], (unsigned long long)d[c]);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nb * kQ; i += blockDim.x)
    if (sh[i]) atomicAdd((unsigned long long*)&acc[i], (unsigned long long)sh[i]);
}

// counters -> binary64: count, sum vx, sum vy, sum vz, sum vx^2, sum vy^2, sum vz^2
__global__ void k_static_convert(const long long* acc, int nb, double* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nb * 7; i += gridDim.x * blockDim.x) {
    int b = i / 7, q = i % 7;
    const long long* src = acc + b * kQ;
    double val;
    if (q == 0) {
      val = (double)src[0];
    } else {
      const long long* dg = src + 1 + 3 * (q - 1);
      __int128 tot = ((__int128)dg[2] << 64) + ((__int128)dg[1] << 32) + (__int128)dg[0];
      bool neg = tot < 0;
      unsigned __int128 mag = neg ? (unsigned __int128)(-tot) : (unsigned __int128)tot;
      double hi = (double)(unsigned long long)(mag >> 64);
      double lo = (double)(unsigned long long)mag;
      val = kmc::dadd(kmc::dmul(hi, 1.0), kmc::dmul(lo, 0x1p-64));
      val = neg ? -val : val;
    }
    out[i] = val;
  }
}

std::mutex g_setup_mutex;
long long* g_scratch_addr[kMaxDevices] = {nullptr};
int g_num_sms[kMaxDevices] = {0};

bool on_device(const void* ptr) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

int reject(const char* why) {
  std::fprintf(stderr, "sim_profile_static: %s\n", why);
  return KMC_EINVAL;
}

}  // namespace

extern "C" int sim_profile_static(const double* x, const double* vx, const double* vy,
                                  const double* vz, uint32_t n, int32_t bins, double range,
                                  double* out, void* stream) {
  if (bins < 1 || bins > kStaticBins) return reject("bins must be in 1..256 (size of the static scratch)");
  if (!(range > 0.0)) return reject("range must be > 0");
  if (!out) return reject("out is NULL");
  if (n > 0 && (!x || !vx || !vy || !vz)) return reject("a particle array is NULL");
  if (!on_device(out) || (n > 0 && (!on_device(x) || !on_device(vx) || !on_device(vy) || !on_device(vz))))
    return reject("all arrays must be device memory");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return KMC_ECUDA;
  }
  long long* acc = nullptr;
  int sms = 0;
  {
    // once per device, with that device current: the device address of the scratch
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, kmc_profile_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return KMC_ECUDA;
      }
      int v = 0;
      if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) {
        cudaGetLastError();
        v = 152;
      }
      g_num_sms[dev] = v;
      g_scratch_addr[dev] = (long long*)p;
    }
    acc = g_scratch_addr[dev];
    sms = g_num_sms[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int count = bins * kQ;
  k_static_clear<<<(count + 255) / 256, 256, 0, st>>>(acc, count);
  if (n > 0) {
    int blocks = 2 * sms;
    k_static_profile<<<blocks, 256, (size_t)count * sizeof(long long), st>>>(x, vx, vy, vz, n, bins, range, acc);
  }
  k_static_convert<<<(bins * 7 + 255) / 256, 256, 0, st>>>(acc, bins, out);
  if (cudaGetLastError() != cudaSuccess) return KMC_ECUDA;
  return KMC_OK;
}
