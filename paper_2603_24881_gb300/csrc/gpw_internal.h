// Internal layout of a libgpw plan: host-side screening results and the device arrays
// the kernels read.  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <cufft.h>

#include <string>
#include <vector>

#include "gpw.h"

extern "C" int gpw_tile_supported(int t0, int t1, int t2);

namespace gpw {

constexpr int kShellLmax = 3;                   // Cartesian shells up to f
constexpr int kLmax = 2 * kShellLmax;           // la + lb
constexpr int kLextMax = kLmax + 1;             // one more for the centre derivatives
// highest degree of any pair tensor: the kinetic-energy-density gradient (L + 3)
constexpr int kDegMax = kLmax + 3;
constexpr int kNc3Max = (kDegMax + 1) * (kDegMax + 2) * (kDegMax + 3) / 6;  // 220
constexpr int kNc2Max = (kDegMax + 1) * (kDegMax + 2) / 2;                   // 55

// Default sub-box (tile) owned by one thread block: T0 x T1 x T2 grid points, the last
// along the fastest grid index.  The shape is a plan parameter (see kTileShapes).
constexpr int kT0 = 4, kT1 = 8, kT2 = 16;

// Integration work items hold at most max(kChunkMin, ~tasks / kChunkDiv) tasks (about
// four per resident block of 2 x 152 SMs).
constexpr long long kChunkMin = 64;
constexpr long long kChunkDiv = 4 * 2 * 152;
// Work-list band (items): a few times the blocks resident in one launch.
constexpr long long kBand = 2048;

// Non-orthogonal cells: the Cartesian monomials (r - A)^k of degree n <= kSkewDeg are
// re-expanded in the grid-unit displacements xi_d along the lattice rows,
// (r - A)_c = sum_d (R_d)_c / N_d xi_d; per level and degree n a block of
// nh(n) x nh(n) coefficients (row: Cartesian monomial, column: lattice monomial, both
// numbered l2 outer, l1 inner), blocks at mono_off(n), levels kMonoStride apart.
constexpr int kSkewDeg = kDegMax;
__host__ __device__ constexpr int nh(int n) { return (n + 1) * (n + 2) / 2; }
__host__ __device__ constexpr int mono_off(int n) {
  return n == 0 ? 0 : mono_off(n - 1) + nh(n - 1) * nh(n - 1);
}
constexpr int kMonoStride = mono_off(kSkewDeg + 1);
__host__ __device__ constexpr int hidx(int n, int k1, int k2) { return k2 * (n + 1) - (k2 * (k2 - 1)) / 2 + k1; }

// Number of monomials x^l0 y^l1 z^l2 with l0 + l1 + l2 <= L, and of (l1, l2) pairs.
__host__ __device__ constexpr int nc3(int L) { return (L + 1) * (L + 2) * (L + 3) / 6; }
__host__ __device__ constexpr int nc2(int L) { return (L + 1) * (L + 2) / 2; }

// Flat order of the pair coefficient tensors D[l0,l1,l2] / V[l0,l1,l2] of total degree
// <= L (Eqs. rho1 and the V tensor of Sec. III A):
//   for l2 in 0..L, for l1 in 0..L-l2 (the (l2,l1) index c21), for l0 in 0..L-l2-l1.
// Decode tables for every L <= kDegMax live in one small device array:
//   dec21[L][c21] = l2 | l1 << 8 | base3 << 16   (base3 = flat index of (0,l1,l2))
//   dec3[L][c]    = c21 | l0 << 8
struct CoefTables {
  int dec21[kDegMax + 1][kNc2Max];
  int dec3[kDegMax + 1][kNc3Max];
  int c21base[kDegMax + 1][kDegMax + 1];  // c21 of (l2, 0)
};
void build_coef_tables(CoefTables* t);

// GPW_FAST_BLOCK_PRUNE: a pair's centre in fractional coordinates and its extent R_p
struct alignas(16) PairQ {
  double x, y, z, w;
};

struct LevelInfo {
  int N[3];
  int nsb[3];            // sub-boxes per dimension (ceil(N / tile))
  long long grid_off;    // offset of the level grid in the level-grid buffer
  long long spec_off;    // offset of the level half spectrum (complex elements)
  long long sub_base;    // first sub-box of this level in the task CSR (collocation)
  double Gk2;            // cutoff sphere: |G|^2 < Gk2
  double weight;         // Omega / (N0 N1 N2)
  double h[3];           // grid spacing L_d / N_d
  // non-orthogonal cells: metric of the grid step vectors dR_d = R_d / N_d
  // (dR0.dR0, dR1.dR1, dR2.dR2, dR0.dR1, dR0.dR2, dR1.dR2) and the map from Cartesian
  // positions to grid units, x_d = sum_c fr[3 d + c] r_c (fr = N_d times the
  // reciprocal row b_d)
  double gm[6];
  double fr[9];
};

// Everything a grid kernel needs from one plan, in device memory, so that one launch can
// serve the tasks of many plans (work items carry the index of their plan's view).
struct PlanView {
  LevelInfo lc[GPW_MAX_LEVELS];  // levels with the collocation sub-box fields
  LevelInfo li[GPW_MAX_LEVELS];  // levels with the integration sub-box fields
  const int4* task_c;
  const long long* sub_off_c;
  const int4* task_i;
  const long long* sub_off_i;
  const long long* tab_off;
  const long long* coef_off;
  const long long* part_off;
  const long long* xt_off;
  const long long* yt_off;
  const double* tab;
  const double* coef;
  double* part;
  const double* xt;
  const double* yt;
  double* grids;
  int* err;
  int chunk_i;  // tasks per integration work item (items carry level | chunk << 4)
  int xr;       // extra 1-D table rows per dimension (table rows = L + 2 + xr)
  int skew;     // non-orthogonal cell: the grid kernels apply the cross factors
  const double* geo;
  const int4* hot_a;
};

struct DeviceArrays {
  // per pair (SoA)
  int4* hot_a = nullptr;      // lo0, lo1, lo2, L = la + lb
  int4* hot_b = nullptr;      // n0, n1, n2, level      (n = box extent)
  int4* ids = nullptr;        // la, lb, ao_a, ao_b
  int4* ids2 = nullptr;       // atom_a, atom_b, w (2 if a < b else 1), nentries
  double* geo = nullptr;      // 8 per pair: A[3], B[3] (image of b), alpha_a, alpha_b
  double* cab = nullptr;      // c_a N_a c_b N_b
  double* pref = nullptr;     // c_a N_a c_b N_b K_ab (K_ab = exp(-a b |A-B|^2/(a+b)))
  long long* tab_off = nullptr;   // 1-D factor tables
  long long* coef_off = nullptr;  // D tensor (rho) / reduced V tensor (stride nc3(L+1))
  long long* part_off = nullptr;  // per-pair block of task W tensors (nc2(L+1) n0 ns12)
  long long* xt_off = nullptr;    // x-contracted D tables (nc2(L) rows of n0)
  long long* yt_off = nullptr;    // x- and y-contracted D tables (L+1 planes of n0 x n1)
  // tasks of the collocation (c) and integration (i) sub-box shapes
  int4* task_c = nullptr;     // 2 per task: {pair, m|L, u, rank}, {t|n per dimension}
  long long* sub_off_c = nullptr;  // CSR offsets over all sub-boxes of all levels
  int4* work_c = nullptr;     // {plan slot (0), level, sub-box, tasks}, heaviest first
  int4* task_i = nullptr;
  long long* sub_off_i = nullptr;
  int4* work_i = nullptr;
  // V assembly: groups of pairs sharing a contracted shell pair
  int4* groups = nullptr;     // shell a, shell b, first pair, end pair
  // gradient assembly
  long long* atom_off = nullptr;  // CSR over atoms
  int* atom_list = nullptr;       // 2 * pair + side
  // tables and buffers
  double* tab = nullptr;
  double* coef = nullptr;     // per call: D tensors / reduced V tensors
  double* part = nullptr;     // per call: task W tensors, or the x-contracted D tables
  double* pgrad = nullptr;    // 6 per pair
  double* grids = nullptr;    // level real grids
  cufftDoubleComplex* spec = nullptr;   // level half spectra
  cufftDoubleComplex* fspec = nullptr;  // finest half spectrum (work)
  cufftDoubleComplex* fspec2 = nullptr; // copy (C2R overwrites its input)
  double* fine_a = nullptr;   // finest real scratch
  double* fine_b = nullptr;
  double* red = nullptr;      // reduction partials
  double* g2tab = nullptr;    // ((2 pi s)/L_d)^2 per finest-mesh index along each axis
  double* g1tab = nullptr;    // (2 pi s)/L_d, 0 on the Nyquist plane of an even axis
  double* mono_t = nullptr;   // non-orthogonal cells: monomial transforms per level
  double* grad3 = nullptr;    // GGA: three finest real grids (grad rho, then de/d grad rho)
  cufftDoubleComplex* fspec3 = nullptr;  // GGA: finest half spectrum (work)
  double* energies = nullptr; // E_H, E_x (device)
  int* err = nullptr;         // device error word
  PairQ* prune = nullptr;   // GPW_FAST_BLOCK_PRUNE: per pair {f_0(P), f_1(P), f_2(P), R_p}
  // gpw_fock_grad_host: device copies of D, V and the gradient (made by its first call)
  double* xfer_D = nullptr;
  double* xfer_V = nullptr;
  double* xfer_g = nullptr;
  cufftDoubleComplex* fft_pack = nullptr;  // half-length complex grid of the real transforms
  cufftDoubleComplex* fft_tw = nullptr;    // their twiddles, per level (Plan::tw_off)
  CoefTables* tabs = nullptr;
  PlanView* view = nullptr;   // this plan's view (device)
};

struct Plan {
  int device = 0;
  int nao = 0, natm = 0, nlev = 0, lmax = 0;
  int nprim = 0, nshell = 0;
  int tile[3] = {kT0, kT1, kT2};      // collocation sub-box
  int tile_i[3] = {8, 8, 32};         // integration sub-box (along z: window stride)
  int zwin_i = 32;                    // z window of the integration sub-boxes
  int chunk_i = 0;                    // most tasks per integration work item
  double L[3] = {0, 0, 0};   // lattice lengths |R_d|
  double omega = 0;
  bool skew = false;         // non-orthogonal cell (App., non-orthogonal lattices)
  bool skew_zc = false;      // ... whose third row is not orthogonal to the first two
  double lat[9] = {0};       // lattice rows R_d
  double rec[9] = {0};       // reciprocal rows b_d (b_d . R_e = delta_de)
  double E[GPW_MAX_LEVELS] = {0};
  LevelInfo lev[GPW_MAX_LEVELS];     // sub-box fields for the collocation tile
  LevelInfo lev_i[GPW_MAX_LEVELS];   // same levels, sub-box fields for the integration tile
  long long npairs = 0, nent = 0, nwork = 0, nsub_total = 0, ngroups = 0;
  long long nent_i = 0, nwork_i = 0, nsub_i = 0;
  bool tasks_on_device = false;  // task records built on the device at commit
  bool prune = false;            // GPW_FAST_BLOCK_PRUNE: collocation tasks screened per block
  bool debug = false;            // GPW_DEBUG_CHECKS
  double prune_blen[3] = {0, 0, 0};  // |b_d| of the block screening (1 / L_d orthorhombic)
  double prune_lam = 0;      // a lower bound of the lattice metric's smallest eigenvalue
  long long tab_total = 0, coef_total = 0, part_total = 0, xt_total = 0;
  long long yt_base = 0, yt_total = 0;  // the y-contracted tables: part[yt_base, + yt_total)
  long long grid_total = 0, spec_total = 0, fine_n = 0, fine_spec_n = 0;
  long long pair_points = 0;
  long long pair_points_level[GPW_MAX_LEVELS] = {0};
  long long pair_points_L[8] = {0};
  long long npairs_level[GPW_MAX_LEVELS] = {0};
  double flops_rho = 0, flops_mat = 0, flops_ip1 = 0;
  long long device_bytes = 0;
  // host copies needed after construction
  std::vector<int> h_ab, h_img, h_lev, h_lo, h_hi;   // screened pair table (pair order)
  std::vector<int> prim_atom;                          // per primitive
  std::vector<double> prim_alpha;
  std::vector<int> pair_a, pair_b;                     // primitive indices per pair
  std::vector<double> coords;                          // natm * 3
  DeviceArrays d;
  bool committed = false;
  struct HostArrays* host = nullptr;       // host staging between prepare and commit
  std::vector<int4> work_c_host, work_i_host;   // copies kept for batch merging
  struct FftEntry* fft_d2z[GPW_MAX_LEVELS] = {nullptr};  // shared cuFFT handles (cache)
  struct FftEntry* fft_z2d[GPW_MAX_LEVELS] = {nullptr};
  // complex transforms of N0 x N1 x N2/2 for the real ones (N2 even; else nullptr)
  struct FftEntry* fft_z2z[GPW_MAX_LEVELS] = {nullptr};
  long long tw_off[GPW_MAX_LEVELS] = {0};  // level twiddles in d.fft_tw
  double* fft_work = nullptr;          // this plan's cuFFT work area
  cudaStream_t alloc_stream = nullptr; // stream of the plan's stream-ordered allocations
  int red_blocks = 0;
  size_t smem_colloc = 0, smem_integ = 0, smem_integ1 = 0;
  // kinetic-energy-density passes (GPW_TAU): collocation at degree L+2, integration at
  // degree L+2 / L+3
  size_t smem_colloc_t = 0, smem_integ3 = 0;
  int stg_colloc_t = 0, nw_colloc_t = 8, stg_integ3 = 0;
  int nw_colloc = 8, nw_integ = 8;     // warps per thread block
  int nw_colloc_req = 0;               // requested collocation warps (0 = occupancy pick)
  int xc = GPW_XC_LDA_X;               // exchange functional
  int xr = 0;                          // extra 1-D table rows (2 with GPW_TAU)
  int stg_colloc = 0, stg_integ = 0, stg_integ1 = 0;  // per-warp staging doubles
  // profiler: event pairs per phase, recorded on the calling stream when enabled
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  // gpw_fock_grad_host: a stream that copies V back while the gradient kernels run, and
  // the event that marks V complete (made by its first call)
  cudaStream_t xfer_stream = nullptr;
  cudaEvent_t xfer_ev = nullptr;
  std::vector<int> ev_phase;   // phase of each recorded pair (pool index / 2)
  size_t ev_used = 0;
  double prof_ms[GPW_NPHASES] = {0};
  long long prof_n[GPW_NPHASES] = {0};
  mutable long long launches = 0;
};

// plan.cpp (host): screening and task lists; fills everything except device arrays.
int build_host_plan(const gpw_desc* desc, Plan* plan, struct HostArrays* host);
// kernels.cu: shared memory of one integration thread block (eval_mat_ip1, degree
// lmax + 1) for the sub-boxes `tile` with z windows of zwin points; 0 if no kernel exists
// for that shape.  Host arithmetic only (no device query).
size_t integ_block_smem(const int* tile, int zwin, int lmax);
PlanView make_view(const Plan& p);

void set_error(const std::string& msg);

}  // namespace gpw
