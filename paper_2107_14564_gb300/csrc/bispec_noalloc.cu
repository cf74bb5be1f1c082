// Triple-product sums without any memory allocation (bsp_triple_sums_noalloc).
//
// This is a variant of the CUDA-core contraction for callers that cannot call cudaMalloc:
// code that runs inside a framework whose allocator owns the whole device-memory budget (a
// raw cudaMalloc there bypasses its accounting and can fail or fragment the pool), or a
// latency-critical loop that must never enter the driver's allocator once it is set up.
// Instead of plan-owned buffers, the per-block partial sums live in one file-scope device
// array of fixed size. Every GPU that loads this library holds that array until the process
// exits.
#include <mutex>

#include "common.cuh"

namespace bsp {
namespace {

constexpr int kNaThreads = 256;
constexpr int kNaPerThread = BSP_NOALLOC_MAX_TRIPLETS / kNaThreads;  // bins per thread
constexpr int kNaChunk = 64;                                        // voxels per shared chunk
constexpr int kNaFlush = 16;                                        // FP32 runs of 1024 voxels
constexpr int kNaMaxDevices = 64;

// Partial sums [block][bin] of the last call; every call overwrites the part it reads.
static __device__ __align__(256) double g_noalloc_partial[BSP_NOALLOC_MAX_BLOCKS * BSP_NOALLOC_MAX_TRIPLETS];

// Device address of g_noalloc_partial, looked up once per device.
static void* g_partial_addr[kNaMaxDevices];
static int g_num_sms[kNaMaxDevices];
static std::mutex g_setup_mutex;

__global__ void __launch_bounds__(kNaThreads)
noalloc_contract_kernel(const float* __restrict__ fields, int ns, long long nvox,
                        const int* __restrict__ trip, int n_trip, double* partial,
                        long long vox_per_block) {
  __shared__ float dsm[BSP_NOALLOC_MAX_SHELLS * (kNaChunk + 1)];
  constexpr int LD = kNaChunk + 1;
  int ia[kNaPerThread], ib[kNaPerThread], ic[kNaPerThread];
  float acc[kNaPerThread];
  double acc64[kNaPerThread];
  unsigned bad = 0;  // bit k: bin k of this thread names a shell outside [0, ns)
#pragma unroll
  for (int k = 0; k < kNaPerThread; ++k) {
    const int t = threadIdx.x + k * kNaThreads;
    const bool ok = t < n_trip;
    const int a = ok ? trip[3 * t + 0] : 0;
    const int b = ok ? trip[3 * t + 1] : 0;
    const int c = ok ? trip[3 * t + 2] : 0;
    const bool in = a >= 0 && a < ns && b >= 0 && b < ns && c >= 0 && c < ns;
    // a bin with a shell index outside the fields reads shell 0 instead and reports NaN
    ia[k] = in ? a : 0;
    ib[k] = in ? b : 0;
    ic[k] = in ? c : 0;
    bad |= in ? 0u : 1u << k;
    acc[k] = 0.f;
    acc64[k] = 0.0;
  }
  const long long v_begin = (long long)blockIdx.x * vox_per_block;
  const long long v_end = min(v_begin + vox_per_block, nvox);
  int run = 0;
  for (long long vb = v_begin; vb < v_end; vb += kNaChunk) {
    __syncthreads();
    for (int i = threadIdx.x; i < ns * kNaChunk; i += kNaThreads) {
      const int n = i / kNaChunk;
      const int v = i - n * kNaChunk;
      const long long gv = vb + v;
      dsm[n * LD + v] = gv < v_end ? fields[(long long)n * nvox + gv] : 0.f;
    }
    __syncthreads();
    for (int v = 0; v < kNaChunk; ++v) {
#pragma unroll
      for (int k = 0; k < kNaPerThread; ++k)
        acc[k] = fmaf(dsm[ia[k] * LD + v] * dsm[ib[k] * LD + v], dsm[ic[k] * LD + v], acc[k]);
    }
    if (++run == kNaFlush) {
      run = 0;
#pragma unroll
      for (int k = 0; k < kNaPerThread; ++k) { acc64[k] += (double)acc[k]; acc[k] = 0.f; }
    }
  }
#pragma unroll
  for (int k = 0; k < kNaPerThread; ++k) {
    const int t = threadIdx.x + k * kNaThreads;
    if (t < n_trip)
      partial[(long long)blockIdx.x * n_trip + t] = (bad >> k) & 1u ? __longlong_as_double(0x7ff8000000000000LL)
                                                                      : acc64[k] + (double)acc[k];
  }
}

__global__ void noalloc_reduce_kernel(const double* partial, int nblocks, int n_trip, double* msum) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_trip) return;
  double s = 0.0;
  for (int b = 0; b < nblocks; ++b) s += partial[(long long)b * n_trip + t];
  msum[t] = s;
}

// Once per device, with that device current: the device address of the scratch array.
bsp_status noalloc_setup(int dev, void** addr, int* n_sm) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (g_partial_addr[dev] == nullptr) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partial);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_partial)");
    int sms = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    g_num_sms[dev] = sms;
    g_partial_addr[dev] = p;
  }
  *addr = g_partial_addr[dev];
  *n_sm = g_num_sms[dev];
  return BSP_OK;
}

}  // namespace
}  // namespace bsp

using namespace bsp;

extern "C" bsp_status bsp_triple_sums_noalloc(const float* fields, int n_shells, long long n_vox,
                                              const int* triplets, int n_triplets, double* msum,
                                              void* stream) {
  if (!fields || !triplets || !msum) return fail_c(BSP_ERR_INVALID_ARG, "NULL argument");
  if (n_shells < 1 || n_shells > BSP_NOALLOC_MAX_SHELLS)
    return fail_c(BSP_ERR_INVALID_ARG,
                  "bsp_triple_sums_noalloc: n_shells must be in [1, BSP_NOALLOC_MAX_SHELLS = 64]");
  if (n_triplets < 1 || n_triplets > BSP_NOALLOC_MAX_TRIPLETS)
    return fail_c(BSP_ERR_INVALID_ARG,
                  "bsp_triple_sums_noalloc: n_triplets must be in [1, BSP_NOALLOC_MAX_TRIPLETS = 4096] "
                  "(its scratch array has a fixed size)");
  if (n_vox < 1) return fail_c(BSP_ERR_INVALID_ARG, "bsp_triple_sums_noalloc: n_vox must be >= 1");
  int dev = 0;
  BSP_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNaMaxDevices) return fail_c(BSP_ERR_NOT_SUPPORTED, "bsp_triple_sums_noalloc: device index >= 64");
  void* scratch = nullptr;
  int n_sm = 0;
  bsp_status st = noalloc_setup(dev, &scratch, &n_sm);
  if (st != BSP_OK) return st;
  const long long chunks = (n_vox + kNaChunk - 1) / kNaChunk;
  long long blocks = std::min<long long>(std::min<long long>(2LL * n_sm, BSP_NOALLOC_MAX_BLOCKS), chunks);
  if (blocks < 1) blocks = 1;
  const long long vpb = ((chunks + blocks - 1) / blocks) * kNaChunk;
  const int nb = (int)((n_vox + vpb - 1) / vpb);  // blocks that own voxels; all write their part
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double* partial = static_cast<double*>(scratch);
  noalloc_contract_kernel<<<nb, kNaThreads, 0, s>>>(fields, n_shells, n_vox, triplets, n_triplets, partial, vpb);
  BSP_CUDA(cudaGetLastError());
  noalloc_reduce_kernel<<<(n_triplets + 255) / 256, 256, 0, s>>>(partial, nb, n_triplets, msum);
  BSP_CUDA(cudaGetLastError());
  return BSP_OK;
}
