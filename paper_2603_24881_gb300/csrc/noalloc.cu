// gpw_lda_x_noalloc: Slater exchange potential and energy of a density grid, for callers
// that cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is not available or not allowed — a host
// application whose memory pool owns all device memory and forbids allocations behind
// its back, a real-time loop that must not block in the driver's allocator, or a library
// linked into a process whose CUDA context and memory budget belong to someone else.
// Every other libgpw call needs a plan, and building a plan allocates.  This entry point
// needs none: the caller passes the density and the two outputs, and the only working
// memory is a fixed array in the library's own device image, reserved when the library is
// loaded onto a GPU and held by that GPU until the process exits.
//
// It is the allocation-free variant of the exchange step of gpw_fock, whose kernel keeps
// its per-block partial energies in plan-owned scratch.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "gpw.h"

namespace gpw {
void set_error(const std::string& msg);
}

namespace {

constexpr int kNaThreads = 256;
constexpr int kNaPerThread = 64;
constexpr long long kNaChunk = (long long)kNaThreads * kNaPerThread;  // points per block
constexpr int kNaMaxBlocks = GPW_LDA_NOALLOC_MAX_POINTS / (kNaThreads * kNaPerThread);
static_assert((long long)kNaMaxBlocks * kNaChunk == GPW_LDA_NOALLOC_MAX_POINTS,
              "maximum must be a whole number of blocks");

// The scratch: one partial energy per block (32 KB).  Device code may name it directly;
// host code must use the address obtained with cudaGetSymbolAddress.
static __device__ __align__(256) double g_lda_noalloc_partials[kNaMaxBlocks];

constexpr int kNaMaxDevices = 64;
std::mutex g_na_mutex;
double* g_na_scratch[kNaMaxDevices] = {};

__global__ void lda_noalloc_blocks(const double* __restrict__ rho, long long n,
                                   double* __restrict__ vx, double* __restrict__ partials) {
  __shared__ double sh[kNaThreads];
  const double cx = 0.98474502184269641;  // (3/pi)^(1/3)
  const long long base = (long long)blockIdx.x * kNaChunk;
  double part = 0.0;
  for (int j = 0; j < kNaPerThread; ++j) {
    const long long i = base + (long long)j * kNaThreads + threadIdx.x;
    if (i < n) {
      const double r = fmax(rho[i], 0.0);
      const double c = cbrt(r);
      vx[i] = -cx * c;
      part += -0.75 * cx * r * c;
    }
  }
  sh[threadIdx.x] = part;
  __syncthreads();
  for (int s = kNaThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

__global__ void lda_noalloc_total(const double* __restrict__ partials, int nblocks,
                                  double weight, double* __restrict__ ex) {
  __shared__ double sh[kNaThreads];
  double v = 0.0;
  for (int i = threadIdx.x; i < nblocks; i += kNaThreads) v += partials[i];
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = kNaThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *ex = weight * sh[0];
}

}  // namespace

extern "C" int gpw_lda_x_noalloc(const double* rho, long long n, double weight, double* v_x,
                                 double* e_x, void* stream) {
  if (!rho || !v_x || !e_x || n <= 0) {
    gpw::set_error("gpw_lda_x_noalloc: NULL pointer or empty grid");
    return GPW_EINVAL;
  }
  if (n > (long long)GPW_LDA_NOALLOC_MAX_POINTS) {
    gpw::set_error("gpw_lda_x_noalloc: grid of " + std::to_string(n) +
                   " points exceeds the fixed maximum of " +
                   std::to_string((long long)GPW_LDA_NOALLOC_MAX_POINTS) + " points");
    return GPW_ERANGE;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) {
    gpw::set_error(std::string("gpw_lda_x_noalloc: no usable current device: ") +
                   cudaGetErrorString(e));
    return GPW_ECUDA;
  }
  double* scratch = nullptr;
  {
    // first call on a device: look up the scratch array's device address (the device is
    // current); later calls reuse it
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_scratch[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_lda_noalloc_partials);
      if (e != cudaSuccess || !p) {
        gpw::set_error(std::string("gpw_lda_x_noalloc: cudaGetSymbolAddress: ") +
                       cudaGetErrorString(e));
        return GPW_ECUDA;
      }
      g_na_scratch[dev] = static_cast<double*>(p);
    }
    scratch = g_na_scratch[dev];
  }
  // every block writes its partial before the total reads it: nothing needs clearing
  const int nblocks = (int)((n + kNaChunk - 1) / kNaChunk);
  cudaStream_t s = (cudaStream_t)stream;
  lda_noalloc_blocks<<<nblocks, kNaThreads, 0, s>>>(rho, n, v_x, scratch);
  e = cudaGetLastError();
  if (e == cudaSuccess) {
    lda_noalloc_total<<<1, kNaThreads, 0, s>>>(scratch, nblocks, weight, e_x);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    gpw::set_error(std::string("gpw_lda_x_noalloc: launch: ") + cudaGetErrorString(e));
    return GPW_ECUDA;
  }
  return GPW_OK;
}
