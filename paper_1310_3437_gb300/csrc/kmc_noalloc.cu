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
// The scratch array holds kStaticBins x 20 int64 fixed-point counters (40,960
// bytes): per bin the count, three 32-bit digits of each velocity sum and of each
// sum of squares, and the number of terms out of the digits' range (profile_add in
// kmc_internal.cuh; the profile kernel of the simulations uses the same helpers).
// Every GPU that loads the library keeps its own copy until the process exits.
// All calls on a device share it and it keeps the last call's contents; each call
// clears the counters it uses before accumulating.  Two calls whose work overlaps
// on the GPU (different streams, no ordering between them) race on the counters
// and give wrong sums: order such calls on one stream or with events.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "kmc_internal.cuh"

namespace {

constexpr int kStaticBins = 256;  // largest supported number of bins
constexpr int kQ = kmc::kProfQ;   // counters per bin (see profile_add)
constexpr int kMaxDevices = 64;

}  // namespace

// fixed-point profile counters (see the file comment): 256 x 20 x 8 = 40,960 bytes
static __device__ __align__(256) long long kmc_profile_scratch[kStaticBins * kQ];

namespace {

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
  for (uint32_t p = blockIdx.x * blockDim.x + threadIdx.x; p < n; p += gridDim.x * blockDim.x) {
    double xp = x[p];
    if (!(xp >= 0.0)) continue;
    double f = kmc::dmul(xp, scale);
    if (f >= (double)nb) continue;
    const double v[3] = {vx[p], vy[p], vz[p]};
    kmc::profile_add(sh + (int)f * kQ, v);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nb * kQ; i += blockDim.x)
    if (sh[i]) atomicAdd((unsigned long long*)&acc[i], (unsigned long long)sh[i]);
}

// counters -> binary64: count, sum vx, sum vy, sum vz, sum vx^2, sum vy^2, sum vz^2
__global__ void k_static_convert(const long long* acc, int nb, double* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nb * 7; i += gridDim.x * blockDim.x)
    out[i] = kmc::profile_value(acc + (i / 7) * kQ, i % 7);
}

std::mutex g_setup_mutex;
long long* g_scratch_addr[kMaxDevices] = {nullptr};
int g_num_sms[kMaxDevices] = {0};

// device memory of the current device dev (or managed memory): a pointer to another
// GPU's memory would be dereferenced without a peer mapping
bool on_device(const void* ptr, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
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
  if (n >= 0x80000000u) return reject("n must be below 2^31 (int64 digit sums)");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return KMC_ECUDA;
  }
  if (!on_device(out, dev) ||
      (n > 0 && (!on_device(x, dev) || !on_device(vx, dev) || !on_device(vy, dev) || !on_device(vz, dev))))
    return reject("all arrays must be device memory of the current device");
  if (stream) {
    int sdev = -1;
    if (cudaStreamGetDevice((cudaStream_t)stream, &sdev) != cudaSuccess) {
      cudaGetLastError();
      return reject("stream is not a valid CUDA stream");
    }
    if (sdev != dev) return reject("stream belongs to another device");
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
