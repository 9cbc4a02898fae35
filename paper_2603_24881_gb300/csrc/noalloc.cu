// gpw_lda_x_noalloc: Slater exchange potential and energy of a density grid, for callers
// that cannot allocate device memory.
//
// Who needs it: code that runs where cudaMalloc is not available or not allowed — a host
// application whose memory pool owns all device memory and forbids allocations behind
// its back, a real-time loop that must not block in the driver's allocator, or a library
// linked into a process whose CUDA context and memory budget belong to someone else.
// Every other libgpw call needs a plan, and building a plan allocates.  This entry point
// needs none: the caller passes the density and the two outputs, and the only working
// memory is a fixed array in the library's own device image, held by each GPU that loaded
// it until the process exits.  With lazy module loading (CUDA's default) the image, and so
// the array, is loaded onto a device by the first call there (its address lookup), and
// that load may allocate inside the driver: make the first call on each device during
// set-up.  Later calls allocate nothing.
//
// It is the allocation-free variant of the exchange step of gpw_fock, whose kernel keeps
// its per-block partial energies in plan-owned scratch.
#include <cuda.h>
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

std::mutex g_na_mutex;

// Scratch addresses by CUDA context id, filled round robin.
constexpr int kNaCache = 64;
unsigned long long g_na_ctx[kNaCache] = {};
double* g_na_ptr[kNaCache] = {};
int g_na_next = 0;

double* cached_scratch(unsigned long long ctx) {
  for (int i = 0; i < kNaCache; ++i)
    if (g_na_ptr[i] && g_na_ctx[i] == ctx) return g_na_ptr[i];
  return nullptr;
}

void cache_scratch(unsigned long long ctx, double* p) {
  g_na_ctx[g_na_next] = ctx;
  g_na_ptr[g_na_next] = p;
  g_na_next = (g_na_next + 1) % kNaCache;
}

// Process-unique id of the current context (cuCtxGetCurrent + cuCtxGetId, reached through
// the runtime's driver entry points: no link against the driver library).  False when no
// context is current or the driver does not provide them.
bool current_context_id(unsigned long long* id) {
  using GetCurrent = CUresult (*)(CUcontext*);
  using GetId = CUresult (*)(CUcontext, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrent>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetId>(f);
  });
  if (!get_current || !get_id) return false;
  CUcontext c = nullptr;
  if (get_current(&c) != CUDA_SUCCESS || !c) return false;
  return get_id(c, id) == CUDA_SUCCESS;
}

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
  if (e != cudaSuccess) {
    gpw::set_error(std::string("gpw_lda_x_noalloc: no usable current device: ") +
                   cudaGetErrorString(e));
    return GPW_ECUDA;
  }
  // The array's device address belongs to the current context: it is cached per context
  // (keyed by the context's process-unique id, so a context created after a device reset
  // is never given an address of the old one).  The first call in a context looks it up,
  // which with lazy module loading also loads the library's device image there.
  double* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_na_mutex);
    unsigned long long ctx = 0;
    const bool have_ctx = current_context_id(&ctx);
    if (have_ctx) scratch = cached_scratch(ctx);
    if (!scratch) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_lda_noalloc_partials);
      if (e != cudaSuccess || !p) {
        gpw::set_error(std::string("gpw_lda_x_noalloc: cudaGetSymbolAddress: ") +
                       cudaGetErrorString(e));
        return GPW_ECUDA;
      }
      scratch = static_cast<double*>(p);
      // the lookup has made the device's primary context current if none was
      if (have_ctx || current_context_id(&ctx)) cache_scratch(ctx, scratch);
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  // every block writes its partial before the total reads it: nothing needs clearing
  const int nblocks = (int)((n + kNaChunk - 1) / kNaChunk);
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
