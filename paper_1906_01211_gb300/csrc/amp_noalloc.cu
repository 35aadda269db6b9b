// Polarization energy for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc when they need this number: a host
// framework that owns all device memory through its own pool and forbids
// other allocations, or a time-critical loop that cannot afford the implicit
// device synchronisation cudaMalloc/cudaFree may cause. For them this file
// provides amp_polarization_energy_noalloc: the same reduction as
// amp_polarization_energy, but context-free, with its only scratch (one float64
// partial sum per block of 256 atoms) in a fixed array in device global memory
// that this library defines. Nothing is allocated by the call.
//
// Limits and sharing rules:
//   - at most kNoallocMaxBlocks = 4096 blocks, i.e. n_atoms <= 1,048,576
//     (AMP_NOALLOC_MAX_ATOMS); larger inputs are rejected with
//     AMP_ERR_TOO_LARGE before anything is launched;
//   - the array (32 KiB) lives on every GPU that loads the library, until the
//     process exits;
//   - all calls share it and it keeps the last call's partial sums. Each call
//     writes every partial it later reads, so nothing has to start at zero;
//     calls whose kernels overlap on the GPU (different streams or threads
//     without ordering) race on the array and give wrong results;
//   - the first call on each device looks up the array's device address with
//     cudaGetSymbolAddress (host code cannot use the symbol itself: on the host
//     it names a stand-in, not device memory); make that first call before any
//     stream capture.
#include <mutex>

#include "amp_internal.cuh"

// The scratch array: one partial sum per block of 256 atoms.
static __device__ __align__(256) double g_energy_partials[4096];

namespace amp {
namespace {

constexpr int kNoallocThreads = 256;  // atoms per block
constexpr int kNoallocMaxBlocks = 4096;
constexpr int kMaxDevices = 64;
static_assert((long long)kNoallocThreads * kNoallocMaxBlocks == AMP_NOALLOC_MAX_ATOMS, "limit mismatch");
static_assert(sizeof(g_energy_partials) == sizeof(double) * kNoallocMaxBlocks, "scratch size");

std::mutex g_setup_mutex;
double* g_partials_ptr[kMaxDevices] = {nullptr};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double s[kNoallocThreads / 32];
  __shared__ double total;
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) s[w] = v;
  __syncthreads();
  if (w == 0) {
    double x = l < kNoallocThreads / 32 ? s[l] : 0.0;
    x = warp_sum(x);
    if (l == 0) total = x;
  }
  __syncthreads();
  return total;
}

// One block per 256 atoms: partial[b] = sum over its atoms of mu . E0.
__global__ void __launch_bounds__(kNoallocThreads) k_energy_partials_noalloc(int n, const double* __restrict__ mu,
                                                                             const double* __restrict__ e0,
                                                                             double* __restrict__ partials) {
  const int s = blockIdx.x * kNoallocThreads + threadIdx.x;
  double v = 0.0;
  if (s < n) v = mu[3 * s] * e0[3 * s] + mu[3 * s + 1] * e0[3 * s + 1] + mu[3 * s + 2] * e0[3 * s + 2];
  v = block_sum(v);
  if (threadIdx.x == 0) partials[blockIdx.x] = v;
}

// U = -1/2 C sum of the partials, summed in a fixed order.
__global__ void __launch_bounds__(kNoallocThreads) k_energy_finish_noalloc(int nblocks,
                                                                           const double* __restrict__ partials,
                                                                           double* __restrict__ U) {
  double v = 0.0;
  for (int k = threadIdx.x; k < nblocks; k += kNoallocThreads) v += partials[k];
  v = block_sum(v);
  if (threadIdx.x == 0) *U = -0.5 * kCoulomb * v;
}

// Device address of the partials array for the current device (looked up once).
int partials_address(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return AMP_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_partials_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_energy_partials) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return AMP_ERR_CUDA;
    }
    g_partials_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_partials_ptr[dev];
  return AMP_OK;
}

}  // namespace
}  // namespace amp

extern "C" int amp_polarization_energy_noalloc(int n_atoms, const double* mu, const double* E0, double* U,
                                               void* cuda_stream) {
  using namespace amp;
  if (n_atoms < 1 || !mu || !E0 || !U) return AMP_ERR_ARG;
  if (n_atoms > AMP_NOALLOC_MAX_ATOMS) return AMP_ERR_TOO_LARGE;
  double* partials = nullptr;
  int r = partials_address(&partials);
  if (r != AMP_OK) return r;
  // An error left by an earlier, unrelated call on this thread is not ours to
  // consume: it stays pending for its owner, and nothing is launched.
  if (cudaPeekAtLastError() != cudaSuccess) return AMP_ERR_CUDA;
  const int nblocks = (n_atoms + kNoallocThreads - 1) / kNoallocThreads;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  k_energy_partials_noalloc<<<nblocks, kNoallocThreads, 0, st>>>(n_atoms, mu, E0, partials);
  k_energy_finish_noalloc<<<1, kNoallocThreads, 0, st>>>(nblocks, partials, U);
  if (cudaPeekAtLastError() != cudaSuccess) {
    cudaGetLastError();  // this call's own launch error, reported through the return code
    return AMP_ERR_CUDA;
  }
  return AMP_OK;
}
