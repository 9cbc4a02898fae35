// Real 3-D transforms of the multigrid combine and restriction (Sec. II: the level
// densities to the finest spectrum, the potential back to the levels) as complex
// transforms of half the length along z.
//
// A real grid x[n0][n1][n2] with N2 even is read as the complex grid
// z[n0][n1][m] = x[..][2m] + i x[..][2m+1], m < M = N2/2, and transformed as a whole (cuFFT
// Z2Z over N0 x N1 x M).  With E and O the transforms of the even and the odd samples,
// Z = E + i O, and E, O are Hermitian (their samples are real), so for k2 = 0..M
//   E(k) = (Z(k) + conj Z(-k)) / 2,  O(k) = (Z(k) - conj Z(-k)) / (2i),
//   X(k0, k1, k2) = E(k0, k1, k2 mod M) + w^k2 O(k0, k1, k2 mod M),  w = exp(-2 pi i / N2),
// which is the half spectrum of the real transform (rfft_untangle).  The inverse runs the
// same steps backwards: from the stored half spectrum and its Hermitian mirror,
//   2E = X(k) + X(k + M e2),  2O = (X(k) - X(k + M e2)) / w^k2,
// Z = 2E + 2i O, and the complex inverse transform of Z over N0 x N1 x M is
// N0 N1 N2 (x[2m] + i x[2m+1]), the unnormalised real inverse transform read as pairs
// (rfft_pack).  The half-length complex transform takes about 30% less time on this GPU
// than the real-to-complex transform of the full length.
#include <cuda_runtime.h>
#include <cufft.h>

#include <cmath>
#include <vector>

#include "gpw_internal.h"
#include "kernels.h"

namespace gpw {
namespace {

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }

// Z: N0 x N1 x M complex (the half-length transform); X: N0 x N1 x (M + 1), the half
// spectrum; tw[k2] = w^k2 (k2 = 0..M, from the plan: a sine or cosine per element would
// cost more FP64 work than the transform saves).  One thread per output element, one
// row of blocks per plane k0 (blockIdx.y).
__global__ void rfft_untangle_kernel(const double2* __restrict__ Z, double2* __restrict__ X,
                                     const double2* __restrict__ tw, int N0, int N1, int M) {
  const int plane = N1 * (M + 1);
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < plane) {
    const int k0 = blockIdx.y, k1 = j / (M + 1), k2 = j - k1 * (M + 1);
    const long long i = (long long)k0 * plane + j;
    const int q2 = k2 == M ? 0 : k2;
    const int m0 = k0 == 0 ? 0 : N0 - k0, m1 = k1 == 0 ? 0 : N1 - k1, mq = q2 == 0 ? 0 : M - q2;
    const double2 zk = Z[((long long)k0 * N1 + k1) * M + q2];
    const double2 zm = cconj(Z[((long long)m0 * N1 + m1) * M + mq]);
    const double2 s = cadd(zk, zm), d = csub(zk, zm);
    const double2 E = make_double2(0.5 * s.x, 0.5 * s.y);
    const double2 O = make_double2(0.5 * d.y, -0.5 * d.x);  // d / (2i)
    X[i] = cadd(E, cmul(__ldg(tw + k2), O));
  }
}

// X: N0 x N1 x (M + 1) half spectrum; Z: N0 x N1 x M; tw as above (its conjugate is
// 1 / w^k2).  One thread per element of Z, one row of blocks per plane k0.
__global__ void rfft_pack_kernel(const double2* __restrict__ X, double2* __restrict__ Z,
                                 const double2* __restrict__ tw, int N0, int N1, int M) {
  const int plane = N1 * M;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < plane) {
    const int k0 = blockIdx.y, k1 = j / M, k2 = j - k1 * M;
    const long long i = (long long)k0 * plane + j;
    const long long row = ((long long)k0 * N1 + k1) * (M + 1);
    const double2 x = X[row + k2];
    double2 xp;  // X(k0, k1, k2 + M): stored for k2 = 0, else the Hermitian mirror
    if (k2 == 0) {
      xp = X[row + M];
    } else {
      const int m0 = k0 == 0 ? 0 : N0 - k0, m1 = k1 == 0 ? 0 : N1 - k1;
      xp = cconj(X[((long long)m0 * N1 + m1) * (M + 1) + (M - k2)]);
    }
    const double2 t = cmul(cconj(__ldg(tw + k2)), csub(x, xp));  // 2 O
    Z[i] = make_double2(x.x + xp.x - t.y, x.y + xp.y + t.x);   // 2E + i 2O
  }
}

dim3 grid_for(int plane, int N0) { return dim3((unsigned)((plane + 255) / 256), (unsigned)N0); }

}  // namespace

cudaError_t launch_rfft_untangle(const cufftDoubleComplex* Z, cufftDoubleComplex* X,
                                 const cufftDoubleComplex* tw, const int* N, cudaStream_t s) {
  rfft_untangle_kernel<<<grid_for(N[1] * (N[2] / 2 + 1), N[0]), 256, 0, s>>>(
      reinterpret_cast<const double2*>(Z), reinterpret_cast<double2*>(X),
      reinterpret_cast<const double2*>(tw), N[0], N[1], N[2] / 2);
  return cudaGetLastError();
}

cudaError_t launch_rfft_pack(const cufftDoubleComplex* X, cufftDoubleComplex* Z,
                             const cufftDoubleComplex* tw, const int* N, cudaStream_t s) {
  rfft_pack_kernel<<<grid_for(N[1] * (N[2] / 2), N[0]), 256, 0, s>>>(
      reinterpret_cast<const double2*>(X), reinterpret_cast<double2*>(Z),
      reinterpret_cast<const double2*>(tw), N[0], N[1], N[2] / 2);
  return cudaGetLastError();
}

void rfft_twiddles(int N2, std::vector<cufftDoubleComplex>* out) {
  const int M = N2 / 2;
  const double pi = 3.14159265358979323846;
  for (int k = 0; k <= M; ++k) {
    // w^k = exp(-2 pi i k / N2), with the exact values at k = 0 and k = M
    cufftDoubleComplex w;
    w.x = k == 0 ? 1.0 : (k == M ? -1.0 : std::cos(2.0 * pi * k / N2));
    w.y = (k == 0 || k == M) ? 0.0 : -std::sin(2.0 * pi * k / N2);
    out->push_back(w);
  }
}

}  // namespace gpw
