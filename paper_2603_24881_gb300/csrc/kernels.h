// Launch wrappers of the libgpw CUDA kernels (sm_103a).  Not part of the C ABI.
#pragma once

#include "gpw_internal.h"

namespace gpw {

struct KLevels {
  LevelInfo lv[GPW_MAX_LEVELS];
  int nlev;
  int skew;       // non-orthogonal cell: |G|^2 has cross terms
  double gq[3];   // their coefficients 2 (2 pi)^2 (b0.b1, b0.b2, b1.b2)
  double rec[9];  // reciprocal rows b_d (Cartesian G = 2 pi sum_d s_d b_d)
  double invn[GPW_MAX_LEVELS];  // 1 / (N0 N1 N2) of every level
};

KLevels make_klevels(const Plan& p, bool integ);

// Launch shape of a grid kernel: sub-box, warps per block, factor rows, staging, smem.
struct GridLaunch {
  int tile[3];
  int nw, lp, stg;
  size_t smem;
  int ldeg = 0;  // collocation: degree added to every pair's L (2 for the kinetic density)
  int skew = 0;  // non-orthogonal cells: the kernels with cross factors
  int zwin = 0;  // integration: z window of the sub-boxes (tile[2]: plain tiling)
};
cudaError_t launch_collocate_views(const GridLaunch& cfg, const PlanView* views, const int4* work,
                                   long long nwork, const CoefTables* tabs, cudaStream_t s);
cudaError_t launch_integrate_views(const GridLaunch& cfg, int lext, const PlanView* views,
                                   const int4* work, long long nwork, const CoefTables* tabs,
                                   cudaStream_t s);
cudaError_t configure_batch(const int* tile_c, const int* tile_i, int zwin_i, int lmax, int nw_req,
                            GridLaunch* colloc,
                            GridLaunch* integ1, int skew = 0);

cudaError_t launch_tables(const Plan& p, cudaStream_t s);
cudaError_t launch_pair_coef(const Plan& p, const double* D, cudaStream_t s);
cudaError_t launch_pair_coef_tau(const Plan& p, const double* D, cudaStream_t s);
cudaError_t launch_assemble_V_tau(const Plan& p, int lext, double* V, cudaStream_t s);
cudaError_t launch_grad_tau(const Plan& p, const double* D, double* grad, cudaStream_t s);
cudaError_t launch_fourier_deriv(const Plan& p, int axis, const cufftDoubleComplex* in,
                                 cufftDoubleComplex* out, bool subtract, cudaStream_t s);
cudaError_t launch_pbe_x(const Plan& p, const double* rho, double* grad3, double* v_rho,
                         cudaStream_t s);
cudaError_t launch_spec_combine(const Plan& p, const cufftDoubleComplex* fa,
                                const cufftDoubleComplex* fb, cufftDoubleComplex* out,
                                cudaStream_t s);
// the x and then the y contraction of collocation, once per pair (ldeg: degree raise)
cudaError_t launch_xcontract(const Plan& p, cudaStream_t s, int ldeg = 0);
cudaError_t launch_collocate(const Plan& p, cudaStream_t s, int ldeg = 0);
cudaError_t launch_integrate(const Plan& p, int lext, cudaStream_t s);
cudaError_t launch_reduce_parts(const Plan& p, int lext, cudaStream_t s);
cudaError_t launch_assemble_V(const Plan& p, int lext, double* V, cudaStream_t s);
cudaError_t launch_grad(const Plan& p, const double* D, double* grad, cudaStream_t s);
cudaError_t launch_combine(const Plan& p, cudaStream_t s);
cudaError_t launch_restrict(const Plan& p, int level, const cufftDoubleComplex* fa,
                            const cufftDoubleComplex* fb, cudaStream_t s);
cudaError_t launch_poisson(const Plan& p, cudaStream_t s);
cudaError_t launch_lda(const Plan& p, const double* rho, const double* vH, double* v_out,
                       cudaStream_t s);
cudaError_t launch_energy_final(const Plan& p, int slot, int nparts, cudaStream_t s);
// GPW_DEBUG_CHECKS: error code 16 if any of x[0..n) is not finite; code 17 if a task list
// (integ: the integration list) is inconsistent with its sub-boxes and pair boxes
cudaError_t launch_finite_check(const Plan& p, const double* x, long long n, cudaStream_t s);
cudaError_t launch_validate_tasks(const Plan& p, bool integ, cudaStream_t s);
cudaError_t configure_kernels(Plan* p);
// rfft.cu: real 3-D transforms of an N[0] x N[1] x N[2] grid (N[2] even) through the
// complex transform of N[0] x N[1] x N[2]/2: the half spectrum X from that transform Z
// (untangle), and the Z whose inverse transform is the real inverse of X (pack).
// tw: the twiddles w^k2 = exp(-2 pi i k2 / N[2]), k2 = 0..N[2]/2 (rfft_twiddles).
cudaError_t launch_rfft_untangle(const cufftDoubleComplex* Z, cufftDoubleComplex* X,
                                 const cufftDoubleComplex* tw, const int* N, cudaStream_t s);
cudaError_t launch_rfft_pack(const cufftDoubleComplex* X, cufftDoubleComplex* Z,
                             const cufftDoubleComplex* tw, const int* N, cudaStream_t s);
void rfft_twiddles(int N2, std::vector<cufftDoubleComplex>* out);

constexpr int kRedBlocks = 304;
constexpr int kRedThreads = 256;

}  // namespace gpw
