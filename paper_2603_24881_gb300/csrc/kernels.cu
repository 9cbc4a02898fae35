// libgpw CUDA kernels for sm_103a, all arithmetic in FP64.
//
// GB300 issues one warp-wide FP64 FMA per 64 cycles per SM sub-partition, while
// integer, FP32 and shared-memory instructions issue every cycle.  The kernels are
// therefore organised to spend as few FP64 instructions as possible per pair-point and
// to keep every lane of each FP64 instruction busy; index arithmetic uses INT32/FP32.
//
// Collocation (Algorithm 1) and integration (Algorithm 2) both use the separable,
// binomially expanded form of the pair product (Eqs. gx, gab, binomial, gab_lp, rho1
// and the V tensor): a pair contributes
//     sum_{l0+l1+l2 <= L} D[l0,l1,l2] g0[l0](x0) g1[l1](x1) g2[l2](x2)
// with g_d[l](x) = (x - A_d)^l exp(-alpha_p (x - P_d)^2).  The 1-D factors are tabulated
// once per plan; a thread block owns one kT0 x kT1 x kT2 sub-box of a level grid and
// contracts the three dimensions one after another for every (pair, sub-box) task.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <cstdint>

#include "gpw_internal.h"
#include "kernels.h"

namespace gpw {

namespace {

// The integration kernel keeps the dec21 block of the decode tables (the first member of
// CoefTables) in shared memory, padded to a whole number of int4.
constexpr int kDec21Ints = (((kDegMax + 1) * kNc2Max) + 3) & ~3;
static_assert(offsetof(CoefTables, dec21) == 0, "dec21 leads CoefTables");
static_assert(sizeof(CoefTables) >= kDec21Ints * sizeof(int), "CoefTables layout");

__device__ __forceinline__ int fdiv(int x, float inv) {
  // exact floor(x / m) for 0 <= x < 4096, m <= 512, inv = 1/m rounded to fp32
  return __float2int_rz(((float)x + 0.5f) * inv);
}

__device__ __forceinline__ void cart_comp(int l, int idx, int* c) {
  int n = 0;
  for (int ix = l; ix >= 0; --ix)
    for (int iy = l - ix; iy >= 0; --iy) {
      if (n == idx) {
        c[0] = ix;
        c[1] = iy;
        c[2] = l - ix - iy;
        return;
      }
      ++n;
    }
  c[0] = c[1] = c[2] = 0;
}

__constant__ double c_binom[6][6] = {{1, 0, 0, 0, 0, 0}, {1, 1, 0, 0, 0, 0},
                                     {1, 2, 1, 0, 0, 0}, {1, 3, 3, 1, 0, 0},
                                     {1, 4, 6, 4, 1, 0}, {1, 5, 10, 10, 5, 1}};

// n <= 5: an f exponent plus two (the second centre derivative of an f function)
__device__ __forceinline__ double binom(int n, int k) { return c_binom[n][k]; }

__device__ __forceinline__ void set_err(int* err, int code) { atomicCAS(err, 0, code); }

// Asynchronous global -> shared copies (LDGSTS): the next task's factor windows are
// fetched while the current task computes.
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__device__ __forceinline__ void load_dec21(int* dst, const CoefTables* src, int tid, int nthr) {
  const int4* s4 = reinterpret_cast<const int4*>(src);
  int4* d4 = reinterpret_cast<int4*>(dst);
  for (int i = tid; i < kDec21Ints / 4; i += nthr) d4[i] = s4[i];
}

// ----------------------------------------------------------------------------------
// 1-D factor tables (Eq. gab_lp with the exponential of Eq. gab):
//   g_d[l](i) = (x - A_d)^l exp(-alpha_p (x - P_d)^2),  x = (lo_d + i) h_d,  l <= L + 1 + xr
//   (xr = 2 for plans with the kinetic-energy-density kernels),
// laid out per pair as [d][l][n_d].  Also pref = c_a N_a c_b N_b K_ab.  One warp per pair.
__global__ void tables_kernel(long long np, const KLevels K, const int4* __restrict__ hot_a,
                              const int4* __restrict__ hot_b, const double* __restrict__ geo,
                              const double* __restrict__ cab,
                              const long long* __restrict__ tab_off, double* __restrict__ tab,
                              double* __restrict__ pref, int xr, int skew) {
  const int lane = threadIdx.x & 31;
  long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long sw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long p = gw; p < np; p += sw) {
    const int4 ha = hot_a[p];
    const int4 hb = hot_b[p];
    const int L = ha.w;
    const LevelInfo& lv = K.lv[hb.w];
    const double* g = geo + 8 * p;
    const double aa = g[6], ab = g[7], ap = aa + ab;
    double P[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) P[d] = (aa * g[d] + ab * g[3 + d]) / ap;
    if (lane == 0) {
      double ab2 = 0.0;
#pragma unroll
      for (int d = 0; d < 3; ++d) ab2 += (g[d] - g[3 + d]) * (g[d] - g[3 + d]);
      pref[p] = cab[p] * exp(-aa * ab * ab2 / ap);
    }
    const int n[3] = {hb.x, hb.y, hb.z};
    const int lo[3] = {ha.x, ha.y, ha.z};
    const int ntot = n[0] + n[1] + n[2];
    const long long base = tab_off[p];
    // non-orthogonal cell: A and P in grid units along the rows (x_d = fr_d . r)
    double ag[3] = {0.0, 0.0, 0.0}, pg[3] = {0.0, 0.0, 0.0};
    if (skew) {
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        ag[d] = lv.fr[3 * d] * g[0] + lv.fr[3 * d + 1] * g[1] + lv.fr[3 * d + 2] * g[2];
        pg[d] = lv.fr[3 * d] * P[0] + lv.fr[3 * d + 1] * P[1] + lv.fr[3 * d + 2] * P[2];
      }
    }
    for (int it = lane; it < ntot; it += 32) {
      int d = it < n[0] ? 0 : (it < n[0] + n[1] ? 1 : 2);
      int off = d == 0 ? 0 : (d == 1 ? n[0] : n[0] + n[1]);
      int i = it - off;
      double u, v;
      if (skew) {
        // xi^l exp(-alpha_p |dR_d|^2 eta^2): the diagonal part of |r - P|^2 on the grid;
        // the cross terms between rows are applied by the grid kernels
        const double x = (double)(lo[d] + i);
        u = x - ag[d];
        const double t = x - pg[d];
        v = exp(-ap * lv.gm[d] * t * t);
      } else {
        double x = (double)(lo[d] + i) * lv.h[d];
        u = x - g[d];
        double t = x - P[d];
        v = exp(-ap * t * t);
      }
      double* dst = tab + base + (long long)(L + 2 + xr) * off + i;
      for (int l = 0; l <= L + 1 + xr; ++l) {
        dst[(long long)l * n[d]] = v;
        v *= u;
      }
    }
    if (skew) {
      // cross-factor tables over the pair box, after the 1-D tables: for the row pairs
      // (0,1), (0,2), (1,2), R_de[x][y] = exp(c a_d(x) a_e(y)), a_d(x) = lo_d + x - p_d,
      // c = -2 alpha_p G_de; each row is geometric in y (two exp, then products)
      double* sd = tab + base + (long long)(L + 2 + xr) * ntot;
      const int pd[3][3] = {{0, 1, 3}, {0, 2, 4}, {1, 2, 5}};
      const long long soff[3] = {0, (long long)n[0] * n[1], (long long)n[0] * (n[1] + n[2])};
      const int rows = 2 * n[0] + n[1];
      for (int it = lane; it < rows; it += 32) {
        const int k = it < n[0] ? 0 : (it < 2 * n[0] ? 1 : 2);
        const int x = it - (k == 0 ? 0 : (k == 1 ? n[0] : 2 * n[0]));
        const int d = pd[k][0], e = pd[k][1];
        const double c = -2.0 * ap * lv.gm[pd[k][2]];
        const double ad = (double)(lo[d] + x) - pg[d];
        const double ae = (double)lo[e] - pg[e];
        const int len = n[e];
        double v = exp(c * ad * ae);
        const double q = exp(c * ad);
        double* row = sd + soff[k] + (long long)x * len;
        for (int y = 0; y < len; ++y) {
          row[y] = v;
          v *= q;
        }
      }
    }
  }
}

// ----------------------------------------------------------------------------------
// Pair coefficient tensor for collocation (Eq. rho1): contract the density-matrix block
// of the pair with the binomial expansion of Eq. (binomial) in every dimension,
//   D[k0,k1,k2] = w pref sum_{mu in a, nu in b} D_mu,nu prod_d C(b_d, k_d - a_d) (A_d - B_d)^(a_d + b_d - k_d)
// w = 2 for a < b (the pair also stands for (b, a, -T)).  One thread per pair.
__global__ void pair_coef_kernel(long long np, const int4* __restrict__ hot_a,
                                 const int4* __restrict__ ids, const int4* __restrict__ ids2,
                                 const double* __restrict__ geo, const double* __restrict__ pref,
                                 const long long* __restrict__ coef_off,
                                 const CoefTables* __restrict__ tabs, const double* __restrict__ D,
                                 int nao, double* __restrict__ coef) {
  long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const int4 id = ids[p];
  const int la = id.x, lb = id.y, L = la + lb;
  const int na = (la + 1) * (la + 2) / 2, nb = (lb + 1) * (lb + 2) / 2;
  const double* g = geo + 8 * p;
  double pw[3][4];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    double ab = g[d] - g[3 + d];
    pw[d][0] = 1.0;
    pw[d][1] = ab;
    pw[d][2] = ab * ab;
    pw[d][3] = ab * ab * ab;
  }
  double acc[nc3(kLmax)];
  const int nc = nc3(L);
  for (int c = 0; c < nc; ++c) acc[c] = 0.0;
  const double scale = (double)ids2[p].z * pref[p];
  for (int mu = 0; mu < na; ++mu) {
    int ca[3];
    cart_comp(la, mu, ca);
    const double* Drow = D + (long long)(id.z + mu) * nao + id.w;
    for (int nu = 0; nu < nb; ++nu) {
      int cb[3];
      cart_comp(lb, nu, cb);
      const double dmn = scale * Drow[nu];
      for (int t2 = 0; t2 <= cb[2]; ++t2) {
        const double c2 = dmn * binom(cb[2], t2) * pw[2][cb[2] - t2];
        const int k2 = ca[2] + t2;
        for (int t1 = 0; t1 <= cb[1]; ++t1) {
          const double c21 = c2 * binom(cb[1], t1) * pw[1][cb[1] - t1];
          const int k1 = ca[1] + t1;
          const int base = tabs->dec21[L][tabs->c21base[L][k2] + k1] >> 16;
          for (int t0 = 0; t0 <= cb[0]; ++t0)
            acc[base + ca[0] + t0] += c21 * binom(cb[0], t0) * pw[0][cb[0] - t0];
        }
      }
    }
  }
  double* out = coef + coef_off[p];
  for (int c = 0; c < nc; ++c) out[c] = acc[c];
}

// First contraction of collocation, once per pair over its whole box extent n0:
//   X[l2,l1](i) = sum_{l0 <= L - l1 - l2} D[l0,l1,l2] g0[l0](i),   0 <= i < n0,
// stored as nc2(L) rows of n0 (row c21 = c21base[l2] + l1).  Every task of the pair reads
// its m0-column window of it instead of forming the same sums again.  One warp per pair.
__global__ void xcontract_kernel(long long np, const int4* __restrict__ hot_a,
                                 const int4* __restrict__ hot_b,
                                 const long long* __restrict__ tab_off, const double* __restrict__ tab,
                                 const long long* __restrict__ coef_off,
                                 const double* __restrict__ coef,
                                 const long long* __restrict__ xt_off,
                                 const CoefTables* __restrict__ tabs, double* __restrict__ xt,
                                 int ldeg) {
  const int lane = threadIdx.x & 31;
  long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long sw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long p = gw; p < np; p += sw) {
    const int L = hot_a[p].w + ldeg, n0 = hot_b[p].x;
    const double* g0 = tab + tab_off[p];
    const double* Dp = coef + coef_off[p];
    double* out = xt + xt_off[p];
    const int items = nc2(L) * n0;
    for (int it = lane; it < items; it += 32) {
      const int c21 = it / n0, i = it - c21 * n0;
      const int dc = __ldg(&tabs->dec21[L][c21]);
      const int l2 = dc & 255, l1 = (dc >> 8) & 255, b3 = dc >> 16;
      double a = 0.0;
      for (int l0 = 0; l0 <= L - l2 - l1; ++l0) a = fma(Dp[b3 + l0], g0[l0 * n0 + i], a);
      out[(long long)c21 * n0 + i] = a;
    }
  }
}

// Second contraction of collocation, also once per pair, over its box extents n0 x n1:
//   Y[l2](i0, i1) = sum_{l1 <= L - l2} X[l2,l1](i0) g1[l1](i1)
// (times the cross factor R01(i0, i1) of a non-orthogonal cell), stored as L + 1 planes of
// n0 x n1 (i1 fastest).  A pair box spans several sub-boxes along z; each of those tasks
// reads its m0 x m1 window of Y and is left with the z contraction alone.  One warp per
// pair, one lane per (i0, i1), the pair's degree a compile-time constant: a lane keeps
// its g1 column in registers and the lanes write consecutive entries.
template <int L, bool SKEW>
__device__ __forceinline__ void ycontract_pair(int n0, int n1, const double* __restrict__ X,
                                               const double* __restrict__ g1,
                                               const double* __restrict__ r01,
                                               double* __restrict__ out, int lane) {
  const long long n01 = (long long)n0 * n1;
  // (i0, i1) of item it = i0 n1 + i1, advanced by 32 items with a carry (no division
  // per item)
  const int dq = 32 / n1, di = 32 - dq * n1;
  int i0 = lane / n1, i1 = lane - (lane / n1) * n1;
  for (long long it = lane; it < n01; it += 32) {
    double g[L + 1];
#pragma unroll
    for (int l1 = 0; l1 <= L; ++l1) g[l1] = g1[l1 * n1 + i1];
    double f = 1.0;
    if constexpr (SKEW) f = r01[it];
    const double* x = X + i0;
#pragma unroll
    for (int l2 = 0; l2 <= L; ++l2) {
      // X row of (l2, l1): l2 (L + 1) - l2 (l2 - 1) / 2 + l1
      const int row = l2 * (L + 1) - ((l2 * (l2 - 1)) >> 1);
      double a = 0.0;
#pragma unroll
      for (int l1 = 0; l1 <= L - l2; ++l1) a = fma(x[(long long)(row + l1) * n0], g[l1], a);
      if constexpr (SKEW) a *= f;
      out[l2 * n01 + it] = a;
    }
    i0 += dq;
    i1 += di;
    if (i1 >= n1) {
      i1 -= n1;
      ++i0;
    }
  }
}

__global__ void ycontract_kernel(long long np, const int4* __restrict__ hot_a,
                                 const int4* __restrict__ hot_b,
                                 const long long* __restrict__ tab_off, const double* __restrict__ tab,
                                 const long long* __restrict__ xt_off, const double* __restrict__ xt,
                                 const long long* __restrict__ yt_off, double* __restrict__ yt,
                                 int ldeg, int xr, int skew, int* __restrict__ err) {
  const int lane = threadIdx.x & 31;
  long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long sw = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long p = gw; p < np; p += sw) {
    const int Lp = hot_a[p].w, L = Lp + ldeg;
    const int n0 = hot_b[p].x, n1 = hot_b[p].y, n2 = hot_b[p].z;
    const int trows = Lp + 2 + xr;  // rows of each 1-D table of the pair
    const double* g1 = tab + tab_off[p] + (long long)trows * n0;
    const double* r01 = skew ? tab + tab_off[p] + (long long)trows * (n0 + n1 + n2) : nullptr;  // [n0][n1]
    const double* X = xt + xt_off[p];
    double* out = yt + yt_off[p];
    switch (L) {
#define GPW_YC(LL) \
  case LL:         \
    if (skew)      \
      ycontract_pair<LL, true>(n0, n1, X, g1, r01, out, lane); \
    else           \
      ycontract_pair<LL, false>(n0, n1, X, g1, r01, out, lane); \
    break;
      GPW_YC(0) GPW_YC(1) GPW_YC(2) GPW_YC(3) GPW_YC(4) GPW_YC(5) GPW_YC(6) GPW_YC(7) GPW_YC(8)
      GPW_YC(9)
#undef GPW_YC
      default:
        if (lane == 0) set_err(err, 1);
    }
  }
}

// A task is one (pair, sub-box copy) intersection, precomputed by the plan as two int4:
//   r0 = {pair, m0 | m1 << 8 | m2 << 16 | L << 24, u0 | u1 << 8 | u2 << 16, rank}
//   r1 = {t0 | n0 << 16, t1 | n1 << 16, t2 | n2 << 16, 0}
// m = intersection extent, u = its offset in the sub-box, t = its offset in the pair box
// (column of the 1-D tables), n = pair box extent (table row length), rank = index of
// the task among the pair's tasks.
struct Task {
  int p, L, rank;
  int m[3], u[3], t[3], n[3];
};

__device__ __forceinline__ Task decode_task(const int4 r0, const int4 r1) {
  Task t;
  t.p = r0.x;
  t.m[0] = r0.y & 255;
  t.m[1] = (r0.y >> 8) & 255;
  t.m[2] = (r0.y >> 16) & 255;
  t.L = (r0.y >> 24) & 255;
  t.u[0] = r0.z & 255;
  t.u[1] = (r0.z >> 8) & 255;
  t.u[2] = (r0.z >> 16) & 255;
  t.rank = r0.w;
  t.t[0] = r1.x & 0xffff;
  t.n[0] = (r1.x >> 16) & 0xffff;
  t.t[1] = r1.y & 0xffff;
  t.n[1] = (r1.y >> 16) & 0xffff;
  t.t[2] = r1.z & 0xffff;
  t.n[2] = (r1.z >> 16) & 0xffff;
  return t;
}

struct SubBox {
  int s[3], ext[3];
  long long eb, ee;
};

// Sub-box `sub` of a level cut into T0 x T1 x T2 sub-boxes; along z its thread block's
// window spans W2 points from the sub-box start (W2 > T2: windows of neighbouring
// sub-boxes overlap, see the integration kernel).
template <int T0, int T1, int T2, int W2 = T2>
__device__ __forceinline__ SubBox sub_box(const LevelInfo& lv, int sub, const long long* sub_off) {
  SubBox b;
  const int j2 = sub % lv.nsb[2];
  const int j1 = (sub / lv.nsb[2]) % lv.nsb[1];
  const int j0 = sub / (lv.nsb[2] * lv.nsb[1]);
  b.s[0] = j0 * T0;
  b.s[1] = j1 * T1;
  b.s[2] = j2 * T2;
  b.ext[0] = min(T0, lv.N[0] - b.s[0]);
  b.ext[1] = min(T1, lv.N[1] - b.s[1]);
  b.ext[2] = min(W2, lv.N[2] - b.s[2]);
  b.eb = sub_off[lv.sub_base + sub];
  b.ee = sub_off[lv.sub_base + sub + 1];
  return b;
}

// Valid task for a sub-box: non-empty intersection inside the sub-box and inside the
// pair's tables, and a degree the staging buffers were sized for.
__device__ __forceinline__ bool task_ok(const Task& tk, int lx, int lrows, const SubBox& sb) {
  bool ok = lx + 1 <= lrows;
#pragma unroll
  for (int d = 0; d < 3; ++d)
    ok = ok && tk.m[d] >= 1 && tk.u[d] + tk.m[d] <= sb.ext[d] && tk.t[d] + tk.m[d] <= tk.n[d];
  return ok;
}

// Issue asynchronous copies of rows l < rows of the y and z 1-D factor windows of a
// task into shared memory (row strides P1, P2).
template <int P1, int P2>
__device__ __forceinline__ void stage_yz_async(const double* tb, const Task& tk, int rows,
                                               int trows, double* sg1, double* sg2, int lane) {
  const double* t1 = tb + trows * tk.n[0] + tk.t[1];
  const double* t2 = tb + trows * (tk.n[0] + tk.n[1]) + tk.t[2];
  const int m1 = tk.m[1], m2 = tk.m[2];
  const float i1f = __frcp_rn((float)m1), i2f = __frcp_rn((float)m2);
  for (int it = lane; it < rows * m1; it += 32) {
    int l = fdiv(it, i1f), i = it - l * m1;
    cp_async8(sg1 + l * P1 + i, t1 + l * tk.n[1] + i);
  }
  for (int it = lane; it < rows * m2; it += 32) {
    int l = fdiv(it, i2f), i = it - l * m2;
    cp_async8(sg2 + l * P2 + i, t2 + l * tk.n[2] + i);
  }
}

// The per-task contraction of collocation for a pair of total degree L (a compile-time
// constant, so it unrolls completely), from the task's window of the pair's y-contracted
// table (ycontract_kernel) staged as sT2[l2 Q + q], q = i0 m1 + i1:
//   acc(q, i2) += sum_{l2 <= L} T2[l2](q) g2[l2](i2)
// The items (q, i2) are spread over the lanes flat so that partial tasks keep the lanes
// busy; the item index advances by 32 with a carry.
// SK: 0 orthogonal rows or, on a non-orthogonal cell, only the R01 cross factor (folded
// into the table); 1 non-orthogonal cells, of which those with zc (the third row not
// orthogonal to the others) also take R02(i0, i2) R12(i1, i2) at every point, from the
// windows in sR ([T0][T2] then [T1][T2])
template <int L, int T0, int T1, int T2, int SK = 0>
__device__ __forceinline__ void colloc_task(int m01, int m2, const double* __restrict__ sT2,
                                            const double* __restrict__ sg2,
                                            const int* __restrict__ s_row,
                                            const int* __restrict__ s_qi, double* __restrict__ acc,
                                            int lane, const double* __restrict__ sR = nullptr,
                                            bool zc = false) {
  constexpr int Q = T0 * T1;
  const float inv2 = __frcp_rn((float)m2);
  {
    const int dq = fdiv(32, inv2), di = 32 - dq * m2;
    int qA = fdiv(lane, inv2), iA = lane - qA * m2;
    const int items = m01 * m2;
    for (int base = 0; base < items; base += 64) {
      int qB = qA + dq, iB = iA + di;
      if (iB >= m2) {
        iB -= m2;
        ++qB;
      }
      const bool okA = qA < m01, okB = qB < m01;
      const int qa = okA ? qA : 0, qb = okB ? qB : 0;
      double* pa = acc + s_row[qa] + iA;
      double* pb = acc + s_row[qb] + iB;
      const double* ta = sT2 + qa;
      const double* tb = sT2 + qb;
      const double* ga = sg2 + iA;
      const double* gb = sg2 + iB;
      bool zcross = false;
      if constexpr (SK == 1) zcross = zc;
      if (zcross) {
        // non-orthogonal cell: R01 is in T2 already; times R02(i0, i2) R12(i1, i2)
        // (zc false: the plan's third row is orthogonal to the others, R02 = R12 = 1)
        const double* r02 = sR;
        const double* r12 = r02 + T0 * T2;
        const int pa_i = s_qi[qa], pb_i = s_qi[qb];
        if (base + 32 < items) {
          double sa = 0.0, sb = 0.0;
#pragma unroll
          for (int l2 = 0; l2 <= L; ++l2) {
            sa = fma(ta[l2 * Q], ga[l2 * T2], sa);
            sb = fma(tb[l2 * Q], gb[l2 * T2], sb);
          }
          const double ea = r02[(pa_i & 255) * T2 + iA] * r12[(pa_i >> 8) * T2 + iA];
          const double eb = r02[(pb_i & 255) * T2 + iB] * r12[(pb_i >> 8) * T2 + iB];
          if (okA) *pa = fma(ea, sa, *pa);
          if (okB) *pb = fma(eb, sb, *pb);
        } else if (okA) {
          double sa = 0.0;
#pragma unroll
          for (int l2 = 0; l2 <= L; ++l2) sa = fma(ta[l2 * Q], ga[l2 * T2], sa);
          *pa = fma(r02[(pa_i & 255) * T2 + iA] * r12[(pa_i >> 8) * T2 + iA], sa, *pa);
        }
      } else if (base + 32 < items) {
        double ra = okA ? *pa : 0.0, rb = okB ? *pb : 0.0;
#pragma unroll
        for (int l2 = 0; l2 <= L; ++l2) {
          ra = fma(ta[l2 * Q], ga[l2 * T2], ra);
          rb = fma(tb[l2 * Q], gb[l2 * T2], rb);
        }
        if (okA) *pa = ra;
        if (okB) *pb = rb;
      } else if (okA) {
        double ra = *pa;
#pragma unroll
        for (int l2 = 0; l2 <= L; ++l2) ra = fma(ta[l2 * Q], ga[l2 * T2], ra);
        *pa = ra;
      }
      qA = qB + dq;
      iA = iB + di;
      if (iA >= m2) {
        iA -= m2;
        ++qA;
      }
    }
  }
}

// Non-orthogonal cells (App., non-orthogonal lattices): on the grid of a level,
// |r - P|^2 = sum_de G_de eta_d eta_e with eta_d the grid-unit offset of the point from P
// along row d and G the metric of the step vectors.  The 1-D tables hold the diagonal
// part; a task's cross factor is
//   E(i0, i1, i2) = R01(i0, i1) R02(i0, i2) R12(i1, i2),  Rde = exp(-2 alpha_p G_de eta_d eta_e),
// each R row geometric in its second index (eta = eta0 + i): one lane per row takes two
// exp and multiplies along the row.  Rows go to sR ([T0][T1], [T0][T2], [T1][T2]).
template <int T0, int T1, int T2>
struct CrossWindows {
  // a task's windows of the pair's cross-factor tables: R01 [T0][T1], R02 [T0][T2],
  // R12 [T1][T2] (the pair's tables follow its 1-D tables: R01 [n0][n1], R02 [n0][n2],
  // R12 [n1][n2])
  static constexpr int kSize = T0 * T1 + T0 * T2 + T1 * T2;
};

// Stage a task's windows of its pair's cross-factor tables (tables_kernel) into shared
// memory with cp.async, next to its other windows: R01 always, R02 and R12 when zc.
template <int T0, int T1, int T2>
__device__ __forceinline__ void stage_cross(const double* __restrict__ tab, long long toff,
                                            const Task& tk, int xr, double* __restrict__ sR,
                                            int lane, bool zc) {
  const int n0 = tk.n[0], n1 = tk.n[1], n2 = tk.n[2];
  const int m0 = tk.m[0], m1 = tk.m[1], m2 = tk.m[2];
  const int t0 = tk.t[0], t1 = tk.t[1], t2 = tk.t[2];
  const double* sd = tab + toff + (long long)(tk.L + 2 + xr) * (n0 + n1 + n2);
  const float i1f = __frcp_rn((float)m1), i2f = __frcp_rn((float)m2);
  for (int it = lane; it < m0 * m1; it += 32) {
    const int i = fdiv(it, i1f), j = it - i * m1;
    cp_async8(sR + i * T1 + j, sd + (long long)(t0 + i) * n1 + t1 + j);
  }
  if (!zc) return;
  const double* r02 = sd + (long long)n0 * n1;
  const double* r12 = r02 + (long long)n0 * n2;
  for (int it = lane; it < m0 * m2; it += 32) {
    const int i = fdiv(it, i2f), j = it - i * m2;
    cp_async8(sR + T0 * T1 + i * T2 + j, r02 + (long long)(t0 + i) * n2 + t2 + j);
  }
  for (int it = lane; it < m1 * m2; it += 32) {
    const int i = fdiv(it, i2f), j = it - i * m2;
    cp_async8(sR + T0 * T1 + T0 * T2 + i * T2 + j, r12 + (long long)(t1 + i) * n2 + t2 + j);
  }
}

// Collocation's cross-factor windows (non-orthogonal cells with every cross term): R02
// [T0][T2] then R12 [T1][T2] (R01 is in the y-contracted table)
template <int T0, int T1, int T2>
struct CrossWindowsZ {
  static constexpr int kSize = T0 * T2 + T1 * T2;
};

template <int T0, int T1, int T2>
__device__ __forceinline__ void stage_cross_z(const double* __restrict__ tab, long long toff,
                                              const Task& tk, int xr, double* __restrict__ sR,
                                              int lane) {
  const int n0 = tk.n[0], n1 = tk.n[1], n2 = tk.n[2];
  const int m0 = tk.m[0], m1 = tk.m[1], m2 = tk.m[2];
  const int t0 = tk.t[0], t1 = tk.t[1], t2 = tk.t[2];
  const double* r02 = tab + toff + (long long)(tk.L + 2 + xr) * (n0 + n1 + n2) + (long long)n0 * n1;
  const double* r12 = r02 + (long long)n0 * n2;
  const float i2f = __frcp_rn((float)m2);
  for (int it = lane; it < m0 * m2; it += 32) {
    const int i = fdiv(it, i2f), j = it - i * m2;
    cp_async8(sR + i * T2 + j, r02 + (long long)(t0 + i) * n2 + t2 + j);
  }
  for (int it = lane; it < m1 * m2; it += 32) {
    const int i = fdiv(it, i2f), j = it - i * m2;
    cp_async8(sR + T0 * T2 + i * T2 + j, r12 + (long long)(t1 + i) * n2 + t2 + j);
  }
}

template <int T0, int T1, int T2>
struct CollocLayout {
  // one staging buffer: the task's window of the y-contracted table (lp planes of T0 T1,
  // compact: plane l2, entry q = i0 m1 + i1) and its z factor window (lp rows of T2)
  __host__ __device__ static int buf(int lp) { return (lp * (T0 * T1 + T2) + 1) & ~1; }
  // per-warp staging: two buffers and two row tables (T0*T1 ints each: q -> accumulator
  // offset of the row, q -> (i0, i1))
  __host__ __device__ static int stage(int lp) { return 2 * buf(lp) + T0 * T1; }
};

// ----------------------------------------------------------------------------------
// Collocation (Algorithm 1, two-stage: accumulate on chip, write each point once).
// One thread block per sub-box with tasks; warp w takes tasks w, w + NW, ... of the
// sub-box's list and accumulates into its own copy of the sub-box in shared memory;
// the NW copies are summed in a fixed order and written once (coalesced, no atomics).
// The first two of the three contractions are done once per pair beforehand
// (xcontract_kernel, ycontract_kernel); per task, with m the intersection extents and T2
// the pair's y-contracted table, only the third remains:
//   rho(i0,i1,i2) += sum_l2 T2[l2](t0+i0, t1+i1) g2[l2](t2+i2)        (L+1) m0 m1 m2 FMAs
// The next task's windows are copied in (cp.async) while the current one computes.
template <int T0, int T1, int T2, int NW, int SK = 0>
__global__ void __launch_bounds__(NW * 32, 24 / NW)
    collocate_kernel(const PlanView* __restrict__ views, const int4* __restrict__ work,
                     const CoefTables* __restrict__ tabs, int lp, int stg, int ldeg) {
  using Lay = CollocLayout<T0, T1, T2>;
  constexpr int kTileN = T0 * T1 * T2;
  extern __shared__ __align__(16) double sm[];
  double* acc_all = sm;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int i = tid; i < NW * kTileN; i += NW * 32) acc_all[i] = 0.0;

  const int4 item = work[blockIdx.x];
  const PlanView& pv = views[item.x];
  const LevelInfo& lv = pv.lc[item.y];
  const int4* __restrict__ task = pv.task_c;
  const long long* __restrict__ tab_off = pv.tab_off;
  const long long* __restrict__ yt_off = pv.yt_off;
  const double* __restrict__ tab = pv.tab;
  const double* __restrict__ yt = pv.yt;
  double* __restrict__ grids = pv.grids;
  int* __restrict__ err = pv.err;
  const SubBox sb = sub_box<T0, T1, T2>(lv, item.z, pv.sub_off_c);

  double* acc = acc_all + warp * kTileN;
  double* stage_base = acc_all + NW * kTileN + warp * stg;
  const int bufn = Lay::buf(lp);
  constexpr int Q = T0 * T1;
  int* s_row = reinterpret_cast<int*>(stage_base + 2 * bufn);
  int* s_qi = s_row + Q;
  // non-orthogonal cells: the task's cross-factor windows, one per staging buffer, after
  // the regular per-warp staging
  double* sRb = stage_base + ((Lay::stage(lp) + 1) & ~1);
  const bool zc = SK == 1 && pv.skew != 2;  // cross terms with the third row (R02, R12)
  __syncthreads();

  // staging buffer b: [T2 window lp planes of Q][g2 window lp rows of T2]
  auto issue = [&](const Task& tk, long long toff, long long yoff, int b) {
    double* sY = stage_base + b * bufn;
    double* sg2 = sY + lp * Q;
    const int L = tk.L + ldeg, m0 = tk.m[0], m1 = tk.m[1], m2 = tk.m[2];
    const int m01 = m0 * m1, n1 = tk.n[1];
    const long long n01 = (long long)tk.n[0] * n1;
    const int trows = tk.L + 2 + pv.xr;  // table rows of the pair
    const double* y = yt + yoff + (long long)tk.t[0] * n1 + tk.t[1];
    const double* t2 = tab + toff + trows * (tk.n[0] + tk.n[1]) + tk.t[2];
    const float i01f = __frcp_rn((float)m01), i1f = __frcp_rn((float)m1), i2f = __frcp_rn((float)m2);
    for (int it = lane; it < (L + 1) * m01; it += 32) {
      const int l = fdiv(it, i01f), q = it - l * m01;
      const int i0 = fdiv(q, i1f), i1 = q - i0 * m1;
      cp_async8(sY + l * Q + q, y + l * n01 + (long long)i0 * n1 + i1);
    }
    for (int it = lane; it < (L + 1) * m2; it += 32) {
      const int l = fdiv(it, i2f), i = it - l * m2;
      cp_async8(sg2 + l * T2 + i, t2 + l * tk.n[2] + i);
    }
    if constexpr (SK == 1)
      if (zc) stage_cross_z<T0, T1, T2>(tab, toff, tk, pv.xr, sRb + b * CrossWindowsZ<T0, T1, T2>::kSize, lane);
  };

  long long e = sb.eb + warp;
  int4 a0 = make_int4(0, 0, 0, 0), a1 = a0, b0 = a0, b1 = a0;
  long long btoff = 0, bxoff = 0;
  if (e < sb.ee) {
    a0 = __ldg(task + 2 * e);
    a1 = __ldg(task + 2 * e + 1);
    const long long atoff = __ldg(tab_off + a0.x);
    const long long axoff = __ldg(yt_off + a0.x);
    const Task tk = decode_task(a0, a1);
    if (task_ok(tk, tk.L + ldeg, lp, sb)) issue(tk, atoff, axoff, 0);
    cp_async_commit();
  }
  if (e + NW < sb.ee) {
    b0 = __ldg(task + 2 * (e + NW));
    b1 = __ldg(task + 2 * (e + NW) + 1);
    btoff = __ldg(tab_off + b0.x);
    bxoff = __ldg(yt_off + b0.x);
  }
  int buf = 0;
  for (; e < sb.ee; e += NW, buf ^= 1) {
    cp_async_wait_all();
    __syncwarp();
    // fetch the next task's windows into the other buffer
    if (e + NW < sb.ee) {
      const Task tn = decode_task(b0, b1);
      if (task_ok(tn, tn.L + ldeg, lp, sb)) issue(tn, btoff, bxoff, buf ^ 1);
      cp_async_commit();
    }
    int4 c0 = b0, c1 = b1;
    if (e + 2 * NW < sb.ee) {
      c0 = __ldg(task + 2 * (e + 2 * NW));
      c1 = __ldg(task + 2 * (e + 2 * NW) + 1);
    }
    const Task tk = decode_task(a0, a1);
    const int L = tk.L + ldeg;
    const int m0 = tk.m[0], m1 = tk.m[1], m2 = tk.m[2];
    if (!task_ok(tk, L, lp, sb)) {
      if (lane == 0) set_err(err, 1);
    } else {
      const double* sY = stage_base + buf * bufn;
      const double* sg2 = sY + lp * Q;
      const int m01 = m0 * m1;
      const float inv1 = __frcp_rn((float)m1);
      // per-task row tables: q = i0 m1 + i1 -> (i0, i1) and accumulator offset of the row
      for (int q = lane; q < m01; q += 32) {
        const int i0 = fdiv(q, inv1), i1 = q - i0 * m1;
        s_qi[q] = i0 | (i1 << 8);
        s_row[q] = ((tk.u[0] + i0) * T1 + (tk.u[1] + i1)) * T2 + tk.u[2];
      }
      const double* sR = sRb + buf * CrossWindowsZ<T0, T1, T2>::kSize;
      __syncwarp();
#define GPW_COLLOC_L(LL)                                                              \
  case LL:                                                                            \
    colloc_task<LL, T0, T1, T2, SK>(m01, m2, sY, sg2, s_row, s_qi, acc, lane, sR, zc); \
    break;
      switch (L) {
        GPW_COLLOC_L(0) GPW_COLLOC_L(1) GPW_COLLOC_L(2) GPW_COLLOC_L(3) GPW_COLLOC_L(4)
        GPW_COLLOC_L(5) GPW_COLLOC_L(6) GPW_COLLOC_L(7) GPW_COLLOC_L(8)
        default:
          if (lane == 0) set_err(err, 1);
      }
#undef GPW_COLLOC_L
    }
    long long ctoff = btoff, cxoff = bxoff;
    if (e + 2 * NW < sb.ee) {
      ctoff = __ldg(tab_off + c0.x);
      cxoff = __ldg(yt_off + c0.x);
    }
    __syncwarp();
    a0 = b0;
    a1 = b1;
    b0 = c0;
    b1 = c1;
    btoff = ctoff;
    bxoff = cxoff;
  }
  cp_async_wait_all();
  __syncthreads();
  // sum the warp copies in warp order and write the sub-box once
  double* out = grids + lv.grid_off;
  const int e12 = sb.ext[1] * sb.ext[2];
  const int npts = sb.ext[0] * e12;
  for (int pt = tid; pt < npts; pt += NW * 32) {
    const int i0 = pt / e12, r = pt - i0 * e12, i1 = r / sb.ext[2], i2 = r - i1 * sb.ext[2];
    const int ti = (i0 * T1 + i1) * T2 + i2;
    double v = acc_all[ti];
#pragma unroll
    for (int w = 1; w < NW; ++w) v += acc_all[w * kTileN + ti];
    out[((long long)(sb.s[0] + i0) * lv.N[1] + (sb.s[1] + i1)) * lv.N[2] + (sb.s[2] + i2)] = v;
  }
}

// ----------------------------------------------------------------------------------
// Integration (Algorithm 2 and, with lext = 1, the gradient of Algorithm 3): the
// thread block stages its sub-box of the level potential in shared memory once; every
// task contracts it with the pair's 1-D factors (towards the V tensor of Sec. III A):
//   U[l2](i0,i1) = sum_i2 v(i0,i1,i2) g2[l2](i2)        (Lx+1) m0 m1 m2 FMAs
//   W[l2,l1](i0) = sum_i1 U[l2](i0,i1) g1[l1](i1)        nc2(Lx) m0 m1
// and stores W for the task.  The last contraction, V[l0,l1,l2] = sum_i0 W[l2,l1](i0)
// g0[l0](i0), is linear in W, so reduce_parts_kernel first sums the W tensors of the
// pair's tasks that share an x-segment and contracts once per segment (fixed order).
// Lx = L + lext.  Shared rows are padded to an odd number of doubles (P = T + 1) so
// that lanes walking different rows hit different banks.
// Along z a block may stage a window of T2 points while the sub-boxes start every S2 <
// T2 points: the plan then cuts a pair box along z where a window opened in its current
// sub-box ends, so that most pair boxes take one task per (x, y) window instead of one
// per sub-box they cross, and the W contraction (and its store) runs once for them.
template <int T0, int T1, int T2>
struct IntegLayout {
  static constexpr int P0 = T0 + 1, P1 = T1 + 1, P2 = T2 + 1;
  static constexpr int kSV = T0 * T1 * P2;  // padded potential tile
  static constexpr int kUS = T1 * P0;       // one l2 slab of U: [i1][i0]
  __host__ __device__ static int buf(int lpx) { return (lpx * (P1 + P2) + 1) & ~1; }
  // per-warp staging: two factor-window buffers plus the U intermediate
  __host__ __device__ static int stage(int lpx) { return 2 * buf(lpx) + lpx * kUS; }
};

template <int T0, int T1, int T2, int NW, int SK = 0, int S2 = T2>
__global__ void __launch_bounds__(NW * 32)
    integrate_kernel(const PlanView* __restrict__ views, const int4* __restrict__ work,
                     const CoefTables* __restrict__ tabs, int lext, int lpx, int stg) {
  using Lay = IntegLayout<T0, T1, T2>;
  constexpr int P0 = Lay::P0, P1 = Lay::P1, P2 = Lay::P2, kUS = Lay::kUS;
  extern __shared__ __align__(16) double sm[];
  int* s_tab = reinterpret_cast<int*>(sm);
  const int(*s_dec21)[kNc2Max] = reinterpret_cast<const int(*)[kNc2Max]>(s_tab);
  double* sv = sm + kDec21Ints / 2;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  load_dec21(s_tab, tabs, tid, NW * 32);

  const int4 item = work[blockIdx.x];
  const PlanView& pv = views[item.x];
  const LevelInfo& lv = pv.li[item.y & 15];
  const int4* __restrict__ task = pv.task_i;
  const long long* __restrict__ tab_off = pv.tab_off;
  const long long* __restrict__ part_off = pv.part_off;
  const double* __restrict__ tab = pv.tab;
  const double* __restrict__ grids = pv.grids;
  double* __restrict__ part = pv.part;
  int* __restrict__ err = pv.err;
  SubBox sb = sub_box<T0, T1, S2, T2>(lv, item.z, pv.sub_off_i);
  sb.eb += (long long)(item.y >> 4) * pv.chunk_i;  // this item's chunk of the task list
  sb.ee = min(sb.ee, sb.eb + pv.chunk_i);
  {
    const double* vin = grids + lv.grid_off;
    const int e12 = sb.ext[1] * sb.ext[2];
    const int npts = sb.ext[0] * e12;
    for (int pt = tid; pt < npts; pt += NW * 32) {
      const int i0 = pt / e12, r = pt - i0 * e12, i1 = r / sb.ext[2], i2 = r - i1 * sb.ext[2];
      sv[(i0 * T1 + i1) * P2 + i2] = __ldg(
          vin + ((long long)(sb.s[0] + i0) * lv.N[1] + (sb.s[1] + i1)) * lv.N[2] + (sb.s[2] + i2));
    }
  }
  double* stage_base = sv + Lay::kSV + warp * stg;
  const int bufn = Lay::buf(lpx);
  double* sU = stage_base + 2 * bufn;
  // non-orthogonal cells: the task's window of the potential times its cross factors,
  // and the factor rows, after the regular per-warp staging
  // (the potential window times the cross factors last: plans whose third row is
  // orthogonal to the others do not use it and are launched without it)
  double* sRb = stage_base + ((Lay::stage(lpx) + 1) & ~1);
  double* sVE = sRb + 2 * CrossWindows<T0, T1, T2>::kSize;
  const bool zc = SK == 1 && pv.skew != 2;  // cross terms with the third row (R02, R12)
  __syncthreads();

  auto issue = [&](const Task& tk, long long toff, int b) {
    double* sg1 = stage_base + b * bufn;
    stage_yz_async<P1, P2>(tab + toff, tk, tk.L + lext + 1, tk.L + 2 + pv.xr, sg1,
                           sg1 + lpx * P1, lane);
    if constexpr (SK != 0) stage_cross<T0, T1, T2>(tab, toff, tk, pv.xr, sRb + b * CrossWindows<T0, T1, T2>::kSize, lane, zc);
  };

  long long e = sb.eb + warp;
  int4 a0 = make_int4(0, 0, 0, 0), a1 = a0, b0 = a0, b1 = a0;
  long long apoff = 0, btoff = 0, bpoff = 0;
  if (e < sb.ee) {
    a0 = __ldg(task + 2 * e);
    a1 = __ldg(task + 2 * e + 1);
    const long long atoff = __ldg(tab_off + a0.x);
    apoff = __ldg(part_off + a0.x);
    const Task tk = decode_task(a0, a1);
    if (task_ok(tk, tk.L + lext, lpx, sb)) issue(tk, atoff, 0);
    cp_async_commit();
  }
  if (e + NW < sb.ee) {
    b0 = __ldg(task + 2 * (e + NW));
    b1 = __ldg(task + 2 * (e + NW) + 1);
    btoff = __ldg(tab_off + b0.x);
    bpoff = __ldg(part_off + b0.x);
  }
  int buf = 0;
  for (; e < sb.ee; e += NW, buf ^= 1) {
    cp_async_wait_all();
    __syncwarp();
    if (e + NW < sb.ee) {
      const Task tn = decode_task(b0, b1);
      if (task_ok(tn, tn.L + lext, lpx, sb)) issue(tn, btoff, buf ^ 1);
      cp_async_commit();
    }
    int4 c0 = b0, c1 = b1;
    if (e + 2 * NW < sb.ee) {
      c0 = __ldg(task + 2 * (e + 2 * NW));
      c1 = __ldg(task + 2 * (e + 2 * NW) + 1);
    }
    const Task tk = decode_task(a0, a1);
    const int L = tk.L, Lx = L + lext;
    const int m0 = tk.m[0], m1 = tk.m[1], m2 = tk.m[2];
    if (!task_ok(tk, Lx, lpx, sb)) {
      if (lane == 0) set_err(err, 3);
    } else {
      const double* sg1 = stage_base + buf * bufn;
      const double* sg2 = sg1 + lpx * P1;
      const int m01 = m0 * m1;
      const double* vbase = sv;
      int u0 = tk.u[0], u1 = tk.u[1], u2 = tk.u[2];
      const double* sR = sRb + buf * CrossWindows<T0, T1, T2>::kSize;
      if (SK == 1 && zc) {
        const double* r02 = sR + T0 * T1;
        const double* r12 = r02 + T0 * T2;
        const float inv2 = __frcp_rn((float)m2), inv1 = __frcp_rn((float)m1);
        for (int it = lane; it < m01 * m2; it += 32) {
          const int q = fdiv(it, inv2), i2 = it - q * m2;
          const int i0 = fdiv(q, inv1), i1 = q - i0 * m1;
          sVE[(i0 * T1 + i1) * P2 + i2] = sv[((u0 + i0) * T1 + (u1 + i1)) * P2 + u2 + i2] *
                                          (r02[i0 * T2 + i2] * r12[i1 * T2 + i2]);
        }
        __syncwarp();
        vbase = sVE;
        u0 = u1 = u2 = 0;
      }
      // U[l2](i1, i0): lanes walk consecutive i1 (rows P2 apart: conflict free).  Items
      // go 32 at a time; a last round of at most 16 items gives each item two lanes, the
      // lower and the upper half of its z sum, added with one shuffle (lanes k and
      // k + 16): ceil(m2 / 2) + 1 FP64 instructions instead of m2 with half the lanes idle
      {
        const float inv01 = __frcp_rn((float)m01), inv1 = __frcp_rn((float)m1);
        const int items = (Lx + 1) * m01;
        const int full = items & ~31, rem = items - full;
        auto u_item = [&](int it, int z0, int z1, bool store, bool pair) {
          const int l2 = fdiv(it, inv01), q = it - l2 * m01;
          const int i0 = fdiv(q, inv1), i1 = q - i0 * m1;
          const double* vr = vbase + ((u0 + i0) * T1 + (u1 + i1)) * P2 + u2;
          const double* gr = sg2 + l2 * P2;
          double a = 0.0;
          for (int i2 = z0; i2 < z1; ++i2) a = fma(vr[i2], gr[i2], a);
          if (pair) a += __shfl_down_sync(0xffffffffu, a, 16);
          if constexpr (SK != 0) a *= sR[i0 * T1 + i1];  // R01(i0, i1)
          if (store) sU[l2 * kUS + i1 * P0 + i0] = a;
        };
        for (int it = lane; it < full; it += 32) u_item(it, 0, m2, true, false);
        if (rem > 16) {
          if (lane < rem) u_item(full + lane, 0, m2, true, false);
        } else if (rem > 0) {
          const int k = lane & 15, up = lane >> 4, h = (m2 + 1) >> 1;
          u_item(full + (k < rem ? k : 0), up ? h : 0, up ? m2 : h, up == 0 && k < rem, true);
        }
      }
      __syncwarp();
      // W[c21](i0) -> the task's slot (compact: item it = c21 m0 + i0, coalesced); the
      // last round split in two halves of the y sum as above
      {
        const float inv0 = __frcp_rn((float)m0);
        const int items = nc2(Lx) * m0;
        const int full = items & ~31, rem = items - full;
        double* dst = part + apoff + a1.w;
        auto w_item = [&](int it, int y0, int y1, bool store, bool pair) {
          const int c21 = fdiv(it, inv0), i0 = it - c21 * m0;
          const int dc = s_dec21[Lx][c21];
          const int l2 = dc & 255, l1 = (dc >> 8) & 255;
          const double* ur = sU + l2 * kUS + i0;
          const double* gr = sg1 + l1 * P1;
          double a = 0.0;
          for (int i1 = y0; i1 < y1; ++i1) a = fma(ur[i1 * P0], gr[i1], a);
          if (pair) a += __shfl_down_sync(0xffffffffu, a, 16);
          if (store) dst[it] = a;
        };
        for (int it = lane; it < full; it += 32) w_item(it, 0, m1, true, false);
        if (rem > 16) {
          if (lane < rem) w_item(full + lane, 0, m1, true, false);
        } else if (rem > 0) {
          const int k = lane & 15, up = lane >> 4, h = (m1 + 1) >> 1;
          w_item(full + (k < rem ? k : 0), up ? h : 0, up ? m1 : h, up == 0 && k < rem, true);
        }
      }
    }
    long long ctoff = btoff, cpoff = bpoff;
    if (e + 2 * NW < sb.ee) {
      ctoff = __ldg(tab_off + c0.x);
      cpoff = __ldg(part_off + c0.x);
    }
    __syncwarp();
    a0 = b0;
    a1 = b1;
    apoff = bpoff;
    b0 = c0;
    b1 = c1;
    btoff = ctoff;
    bpoff = cpoff;
  }
  cp_async_wait_all();
}

// Extent of the x-segment of a pair box that starts at grid index i (hi = last index of
// the box): segments end at sub-box boundaries (multiples of T) and at the periodic
// boundaries of the N-point mesh, as the plan cut the tasks.
__device__ __forceinline__ int seg_len(int i, int hi, int N, int T) {
  const int k = i >= 0 ? i / N : -((-i + N - 1) / N);
  const int ip = i - k * N;
  const int end = k * N + min((ip / T + 1) * T, N) - 1;
  return min(hi, end) - i + 1;
}

// Per-pair V tensor from the task W tensors (the x contraction of the integration),
//   V[l0,l1,l2] = w_k sum_segments sum_i0 g0[l0](t0 + i0) sum_{tasks of the segment} W[l2,l1](i0)
// with the level weight w_k = Omega / N_k (Sec. III A); sums in a fixed order.  One warp
// per pair; T0 = x extent of the integration sub-box.  The pair's x-segments are taken
// in chunks of at most kRedX points and kRedCap summed values: the lanes stage the
// chunk's g0 rows and its segment map in shared memory, sum the task W tensors of every
// (segment, c21, i0) into rows Wsum[c21][x] (flat over the chunk, so the lanes stay
// busy), then contract them with g0.  When V has fewer than 32 entries, G = 32 / C lane
// groups (C = nc rounded up to a power of two) take every G-th x and a fixed butterfly
// of shuffles adds the groups at the end.
// a + b[0] + b[ts] + ... + b[(N-1) ts], added in that order; all N loads are issued
// before the first add
template <int N>
__device__ __forceinline__ double sum_strided(const double* __restrict__ b, long long ts, double a) {
  double x[N];
#pragma unroll
  for (int j = 0; j < N; ++j) x[j] = b[j * ts];
#pragma unroll
  for (int j = 0; j < N; ++j) a += x[j];
  return a;
}

constexpr int kRedCap = 512;
constexpr int kRedX = 64;
constexpr int kRedPW = 4;  // warps per block (static shared memory stays under 48 KB)
// NK: V entries per lane in steps of 32 (nc3(Lx) <= 32 NK); 4 up to degree kLextMax, 8 for
// the kinetic-energy-density tensors (degree up to kDegMax, 220 entries)
template <int NK>
__global__ void __launch_bounds__(kRedPW * 32, 6)
    reduce_parts_kernel(long long np, const KLevels K, int T0, const int4* __restrict__ hot_a,
                        const int4* __restrict__ hot_b, const int4* __restrict__ ids2,
                        const long long* __restrict__ part_off,
                        const long long* __restrict__ coef_off,
                        const long long* __restrict__ tab_off, const double* __restrict__ tab,
                        const double* __restrict__ part, const CoefTables* __restrict__ tabs,
                        double* __restrict__ coef, int lext, int xr) {
  constexpr int kRows = NK == 4 ? kLextMax + 1 : kDegMax + 1;
  static_assert(nc3(kRows - 1) <= 32 * NK, "entries per lane");
  __shared__ double s_w[kRedPW][kRedCap];
  __shared__ double s_g[kRedPW][kRows * kRedX];
  __shared__ int s_seg[kRedPW][kRedX];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long sw = ((long long)gridDim.x * blockDim.x) >> 5;
  double* sW = s_w[wib];
  double* sG = s_g[wib];
  int* sSeg = s_seg[wib];
  for (long long p = gw; p < np; p += sw) {
    const int4 ha = hot_a[p], hb = hot_b[p];
    const int L = ha.w, Lx = L + lext, nc = nc3(Lx), n2c = nc2(Lx), S = nc2(L + 1 + xr);
    const int lo0 = ha.x, n0 = hb.x, hi0 = lo0 + n0 - 1;
    const LevelInfo& lv = K.lv[hb.w];
    const int N0 = lv.N[0];
    int nsx = 0;
    for (int t0 = 0; t0 < n0; t0 += seg_len(lo0 + t0, hi0, N0, T0)) ++nsx;
    const int ns12 = ids2[p].w / nsx;
    const double* src = part + part_off[p];
    const double* g0 = tab + tab_off[p];
    const float inv2c = __frcp_rn((float)n2c);
    // lane -> (group g, entries c = cidx + 32 k)
    int C = 32;
    while (C >= 2 * nc && C > 1) C >>= 1;
    const int G = 32 / C, g = lane / C, cidx = lane - g * C;
    double v[NK];
    int cc[NK], cl[NK];
#pragma unroll
    for (int k = 0; k < NK; ++k) {
      v[k] = 0.0;
      const int c = cidx + 32 * k;
      const int dc = c < nc ? __ldg(&tabs->dec3[Lx][c]) : 0;
      cc[k] = dc & 255;
      cl[k] = dc >> 8;
    }
    for (int x0 = 0; x0 < n0;) {
      // chunk [x0, x1): whole segments (one segment always fits)
      int x1 = x0 + seg_len(lo0 + x0, hi0, N0, T0);
      while (x1 < n0) {
        const int m = seg_len(lo0 + x1, hi0, N0, T0);
        if (n2c * (x1 + m - x0) > kRedCap || x1 + m - x0 > kRedX) break;
        x1 += m;
      }
      const int E = x1 - x0;
      // segment map (x -> segment start, length) and g0 rows of the chunk
      for (int xr = lane; xr < E; xr += 32) {
        const int i = lo0 + x0 + xr;
        const int kk = i >= 0 ? i / N0 : -((-i + N0 - 1) / N0);
        const int t0 = max(lo0, kk * N0 + ((i - kk * N0) / T0) * T0) - lo0;
        sSeg[xr] = (t0 - x0) | (seg_len(lo0 + t0, hi0, N0, T0) << 16);
      }
      for (int it = lane; it < (Lx + 1) * E; it += 32) {
        const int l = it / E, xr = it - l * E;
        sG[it] = __ldg(g0 + (long long)l * n0 + x0 + xr);
      }
      __syncwarp();
      // one sum per (segment, c21, i0); one FP64 add per task W value (the adds, not the
      // loads, set the pace: loads are unrolled ahead of the add chain)
      for (int it = lane; it < n2c * E; it += 32) {
        const int sg = sSeg[fdiv(it, inv2c)];
        const int tr = sg & 0xffff, m0 = sg >> 16;
        const int rem = it - n2c * tr;
        const int c21 = fdiv(rem, __frcp_rn((float)m0)), i0 = rem - c21 * m0;
        const double* b = src + (long long)S * (x0 + tr) * ns12 + rem;
        const long long ts = (long long)S * m0;
        double a = 0.0;
        int r = 0;
        for (; r + 8 <= ns12; r += 8) a = sum_strided<8>(b + r * ts, ts, a);
        switch (ns12 - r) {
          case 1: a = sum_strided<1>(b + r * ts, ts, a); break;
          case 2: a = sum_strided<2>(b + r * ts, ts, a); break;
          case 3: a = sum_strided<3>(b + r * ts, ts, a); break;
          case 4: a = sum_strided<4>(b + r * ts, ts, a); break;
          case 5: a = sum_strided<5>(b + r * ts, ts, a); break;
          case 6: a = sum_strided<6>(b + r * ts, ts, a); break;
          case 7: a = sum_strided<7>(b + r * ts, ts, a); break;
          default: break;
        }
        sW[c21 * E + tr + i0] = a;
      }
      __syncwarp();
#pragma unroll
      for (int k = 0; k < NK; ++k) {
        if (cidx + 32 * k < nc) {
          const double* wr = sW + cc[k] * E;
          const double* gr = sG + cl[k] * E;
          for (int xr = g; xr < E; xr += G) v[k] = fma(wr[xr], gr[xr], v[k]);
        }
      }
      __syncwarp();
      x0 = x1;
    }
    for (int o = C; o < 32; o <<= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
    const double wgt = lv.weight;
    double* dst = coef + coef_off[p];
    if (g == 0) {
#pragma unroll
      for (int k = 0; k < NK; ++k)
        if (cidx + 32 * k < nc) dst[cidx + 32 * k] = wgt * v[k];
    }
  }
}

// Non-orthogonal cells: re-expand a pair's tensor over the monomials of degree <= L + lext
// (flat order of mono_index) between Cartesian monomials (r - A)^k and grid-unit lattice
// monomials xi^k' of the pair's level, with T the level's transform ((r - A)^k =
// sum_k' T[k][k'] xi^k', degree by degree):
//   dir 0, density coefficients:  C'[k'] = sum_k T[k][k'] C[k]   (Cartesian -> lattice)
//   dir 1, potential moments:      W[k]  = sum_k' T[k][k'] W'[k'] (lattice -> Cartesian)
// One thread per pair.
__device__ __forceinline__ int mono_index(int k0, int k1, int k2, int M);

__global__ void mono_transform_kernel(long long np, const int4* __restrict__ hot_a,
                                      const int4* __restrict__ hot_b,
                                      const long long* __restrict__ coef_off,
                                      double* __restrict__ coef, const double* __restrict__ mono_t,
                                      int lext, int dir) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const int L = hot_a[p].w + lext;
  const double* T = mono_t + (long long)kMonoStride * hot_b[p].w;
  double* c = coef + coef_off[p];
  double in[kNc3Max];
  const int nc = nc3(L);
  for (int i = 0; i < nc; ++i) in[i] = c[i];
  for (int n = 0; n <= L; ++n) {
    const double* blk = T + mono_off(n);
    const int m = nh(n);
    for (int a2 = 0; a2 <= n; ++a2)
      for (int a1 = 0; a1 <= n - a2; ++a1) {
        const int ha = hidx(n, a1, a2);
        double acc = 0.0;
        for (int b2 = 0; b2 <= n; ++b2)
          for (int b1 = 0; b1 <= n - b2; ++b1) {
            const int hb = hidx(n, b1, b2);
            // dir 0: output lattice a from Cartesian b (T[b][a]); dir 1: the transpose
            const double t = dir == 0 ? blk[hb * m + ha] : blk[ha * m + hb];
            acc = fma(t, in[mono_index(n - b1 - b2, b1, b2, L)], acc);
          }
        c[mono_index(n - a1 - a2, a1, a2, L)] = acc;
      }
  }
}

// V assembly: one warp per contracted shell pair (sa, sb), lanes over its (mu, nu)
// elements; each element sums over the group's pairs
//   X_mu,nu = pref sum_k V[k] prod_d C(b_d, k_d - a_d) (A_d - B_d)^(a_d + b_d - k_d)
// (Eq. binomial contracted with the V tensor).  A pair a < b in a diagonal shell
// block also contributes X^T (its mirror (b, a, -T)); off-diagonal blocks are written
// together with their transpose.
__device__ double contract_elem(const int* ca, const int* cb, const double pw[3][4],
                                const double* V, int L, const int (*dec21)[kNc2Max],
                                const int (*c21b)[kDegMax + 1]) {
  double s = 0.0;
  for (int t2 = 0; t2 <= cb[2]; ++t2) {
    const double c2 = binom(cb[2], t2) * pw[2][cb[2] - t2];
    const int k2 = ca[2] + t2;
    for (int t1 = 0; t1 <= cb[1]; ++t1) {
      const double c21 = c2 * binom(cb[1], t1) * pw[1][cb[1] - t1];
      const int k1 = ca[1] + t1;
      const int base = dec21[L][c21b[L][k2] + k1] >> 16;
      double s0 = 0.0;
      for (int t0 = 0; t0 <= cb[0]; ++t0) s0 += binom(cb[0], t0) * pw[0][cb[0] - t0] * V[base + ca[0] + t0];
      s += c21 * s0;
    }
  }
  return s;
}

// One warp per contracted shell pair (group of primitive pairs); a group with fewer than
// 32 elements spreads its pairs over G = 32 / C lane groups (C = the element count rounded
// up to a power of two): lane group g sums the pairs g, g + G, ... of the group for its
// element, and a fixed butterfly of shuffles adds the groups.
__global__ void assemble_V_kernel(long long ngroups, const int4* __restrict__ groups,
                                  const int4* __restrict__ ids, const int4* __restrict__ ids2,
                                  const double* __restrict__ geo, const double* __restrict__ pref,
                                  const long long* __restrict__ coef_off,
                                  const double* __restrict__ coef,
                                  const CoefTables* __restrict__ tabs, int nao, int lext,
                                  double* __restrict__ V) {
  const int lane = threadIdx.x & 31;
  long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (gw >= ngroups) return;
  const int4 gr = groups[gw];
  const int4 id0 = ids[gr.z];
  const int la = id0.x, lb = id0.y, Lx = la + lb + lext;
  const int na = (la + 1) * (la + 2) / 2, nb = (lb + 1) * (lb + 2) / 2;
  const int nel = na * nb;
  const bool diag = gr.x == gr.y;
  int C = 1;
  while (C < nel && C < 32) C <<= 1;
  const int G = 32 / C, g = lane / C, e = lane - g * C;
  for (int base = 0; base < nel; base += C) {
    const int el = base + e;
    double tot = 0.0;
    if (el < nel) {
      const int mu = el / nb, nu = el - mu * nb;
      int ca[3], cb[3];
      cart_comp(la, mu, ca);
      cart_comp(lb, nu, cb);
      for (int p = gr.z + g; p < gr.w; p += G) {
        const double* gp = geo + 8LL * p;
        double pw[3][4];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          double ab = gp[d] - gp[3 + d];
          pw[d][0] = 1.0;
          pw[d][1] = ab;
          pw[d][2] = ab * ab;
          pw[d][3] = ab * ab * ab;
        }
        const double* Vp = coef + coef_off[p];
        double x = contract_elem(ca, cb, pw, Vp, Lx, tabs->dec21, tabs->c21base);
        if (diag && ids2[p].z == 2) {
          int ca2[3], cb2[3];
          cart_comp(la, nu, ca2);
          cart_comp(lb, mu, cb2);
          x += contract_elem(ca2, cb2, pw, Vp, Lx, tabs->dec21, tabs->c21base);
        }
        tot += pref[p] * x;
      }
    }
    for (int o = C; o < 32; o <<= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
    if (g == 0 && el < nel) {
      const int mu = el / nb, nu = el - mu * nb;
      V[(long long)(id0.z + mu) * nao + id0.w + nu] = tot;
      if (!diag) V[(long long)(id0.w + nu) * nao + id0.z + mu] = tot;
    }
  }
}

// Flat index of the monomial (k0, k1, k2) in the coefficient order of total degree <= M
// (l2 outer, l1, l0 inner): the l2 blocks before k2, the l1 rows before k1, then k0.
__device__ __forceinline__ int mono_index(int k0, int k1, int k2, int M) {
  const int r = M - k2;
  return nc3(M) - nc3(r) + k1 * (r + 1) - ((k1 * (k1 - 1)) >> 1) + k0;
}

// Gradient contraction per pair (Algorithm 3).  The centre derivative of the product
// (x - A)^a exp(-alpha_a (x - A)^2) brings -a_d (x - A)^(a - e_d) + 2 alpha_a (x - A)^(a + e_d);
// expanding (x - B)^b about A (Eq. binomial) turns the density-matrix block into
//   Dt[k]   = sum_{mu,nu} D_mu,nu prod_d C(b_d, t_d) (A_d - B_d)^(b_d - t_d),  k = a + t
//   Dm_d[k] = sum_{mu,nu} D_mu,nu a_d prod_d C(b_d, t_d) (A_d - B_d)^(b_d - t_d),  k = a - e_d + t
// so that with the pair's degree-(L+1) V tensor
//   dE/dA_d = w pref [ 2 alpha_a sum_k Dt[k] V[k + e_d] - sum_k Dm_d[k] V[k] ].
// The product depends on x - A and x - B only, so d/dA + d/dB = -d/dx, and
//   dE/dB_d = -dE/dA_d - w pref sum_k Dt[k] [ k_d V[k - e_d] - 2 alpha_p (V[k + e_d] + (A_d - P_d) V[k]) ]
// (the x derivative of (x - A)^k exp(-alpha_p (x - P)^2), summed on the same grid points).
// One thread per pair.
__global__ void grad_pair_kernel(long long np, const int4* __restrict__ ids,
                                 const int4* __restrict__ ids2, const double* __restrict__ geo,
                                 const double* __restrict__ pref,
                                 const long long* __restrict__ coef_off,
                                 const double* __restrict__ coef, const double* __restrict__ D,
                                 int nao, double* __restrict__ pgrad) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const int4 id = ids[p];
  const int la = id.x, lb = id.y, L = la + lb, Lx = L + 1;
  const int na = (la + 1) * (la + 2) / 2, nb = (lb + 1) * (lb + 2) / 2;
  const double* g = geo + 8 * p;
  const double aa = g[6], ab = g[7], ap = aa + ab;
  double pw[3][4], amp[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double t = g[d] - g[3 + d];
    pw[d][0] = 1.0;
    pw[d][1] = t;
    pw[d][2] = t * t;
    pw[d][3] = t * t * t;
    amp[d] = ab * t / ap;  // A_d - P_d
  }
  double Dt[nc3(kLmax)];
  double Dm[3][nc3(kLmax - 1)];
  const int nt = nc3(L), nm = L >= 1 ? nc3(L - 1) : 0;
  for (int c = 0; c < nt; ++c) Dt[c] = 0.0;
  for (int c = 0; c < nm; ++c) Dm[0][c] = Dm[1][c] = Dm[2][c] = 0.0;
  for (int mu = 0; mu < na; ++mu) {
    int a[3];
    cart_comp(la, mu, a);
    const double* Drow = D + (long long)(id.z + mu) * nao + id.w;
    for (int nu = 0; nu < nb; ++nu) {
      int b[3];
      cart_comp(lb, nu, b);
      const double dmn = Drow[nu];
      for (int t2 = 0; t2 <= b[2]; ++t2) {
        const double c2 = dmn * binom(b[2], t2) * pw[2][b[2] - t2];
        for (int t1 = 0; t1 <= b[1]; ++t1) {
          const double c21 = c2 * binom(b[1], t1) * pw[1][b[1] - t1];
          for (int t0 = 0; t0 <= b[0]; ++t0) {
            const double c = c21 * binom(b[0], t0) * pw[0][b[0] - t0];
            const int k0 = a[0] + t0, k1 = a[1] + t1, k2 = a[2] + t2;
            Dt[mono_index(k0, k1, k2, L)] += c;
            if (a[0] > 0) Dm[0][mono_index(k0 - 1, k1, k2, L - 1)] += a[0] * c;
            if (a[1] > 0) Dm[1][mono_index(k0, k1 - 1, k2, L - 1)] += a[1] * c;
            if (a[2] > 0) Dm[2][mono_index(k0, k1, k2 - 1, L - 1)] += a[2] * c;
          }
        }
      }
    }
  }
  const double* V = coef + coef_off[p];
  double sA[3] = {0.0, 0.0, 0.0}, sX[3] = {0.0, 0.0, 0.0}, sC[3] = {0.0, 0.0, 0.0};
  int c = 0;
  for (int k2 = 0; k2 <= L; ++k2)
    for (int k1 = 0; k1 <= L - k2; ++k1)
      for (int k0 = 0; k0 <= L - k2 - k1; ++k0, ++c) {
        const double dt = Dt[c];
        const double v0 = V[mono_index(k0, k1, k2, Lx)];
        const int k[3] = {k0, k1, k2};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const double vp = V[mono_index(k0 + (d == 0), k1 + (d == 1), k2 + (d == 2), Lx)];
          const double vm = k[d] > 0 ? V[mono_index(k0 - (d == 0), k1 - (d == 1), k2 - (d == 2), Lx)] : 0.0;
          sA[d] += dt * vp;
          sX[d] += dt * (k[d] * vm - 2.0 * ap * (vp + amp[d] * v0));
        }
      }
  c = 0;
  for (int k2 = 0; k2 < L; ++k2)
    for (int k1 = 0; k1 < L - k2; ++k1)
      for (int k0 = 0; k0 < L - k2 - k1; ++k0, ++c) {
        const double v0 = V[mono_index(k0, k1, k2, Lx)];
#pragma unroll
        for (int d = 0; d < 3; ++d) sC[d] += Dm[d][c] * v0;
      }
  const double scale = (double)ids2[p].z * pref[p];
  double* out = pgrad + 6 * p;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double gA = scale * (2.0 * aa * sA[d] - sC[d]);
    out[d] = gA;
    out[3 + d] = -gA - scale * sX[d];
  }
}

// Per-atom sums of the per-pair gradient sextets: one warp per atom, lanes stride its
// (pair, side) list in order and a fixed shuffle tree combines them (deterministic).
__global__ void grad_atom_kernel(int natm, const long long* __restrict__ atom_off,
                                 const int* __restrict__ atom_list,
                                 const double* __restrict__ pgrad, double* __restrict__ grad) {
  const int lane = threadIdx.x & 31;
  const int atom = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (atom >= natm) return;
  double s0 = 0.0, s1 = 0.0, s2 = 0.0;
  for (long long i = atom_off[atom] + lane; i < atom_off[atom + 1]; i += 32) {
    const int code = atom_list[i];
    const double* g = pgrad + 6LL * (code >> 1) + 3 * (code & 1);
    s0 += g[0];
    s1 += g[1];
    s2 += g[2];
  }
  for (int o = 16; o > 0; o >>= 1) {
    s0 += __shfl_xor_sync(0xffffffffu, s0, o);
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  }
  if (lane == 0) {
    grad[3 * atom] = s0;
    grad[3 * atom + 1] = s1;
    grad[3 * atom + 2] = s2;
  }
}

// ----------------------------------------------------------------------------------
// Spectral steps.  |G|^2 is formed exactly as ((2 pi s)/L)^2 summed in index order,
// without FMA contraction, so the strict sphere test |G| < G_k is the same decision as
// the oracle's (Sec. II multigrid, Eq. vHG).  Non-orthogonal cells add the cross terms.
__device__ __forceinline__ int signed_freq(int m, int N) { return m < (N + 1) / 2 ? m : m - N; }

// |G|^2 from per-axis tables of ((2 pi s)/L_d)^2 (built on the host, indexed by the
// finest-mesh index), summed in axis order without FMA.
__device__ __forceinline__ double gsq(int f0, int f1, int f2, const double* __restrict__ g2t,
                                      const int* Nf) {
  return __dadd_rn(__dadd_rn(__ldg(g2t + f0), __ldg(g2t + Nf[0] + f1)),
                   __ldg(g2t + Nf[0] + Nf[1] + f2));
}

// |G|^2 of a non-orthogonal cell: the per-axis tables hold (2 pi s_d |b_d|)^2, plus the
// cross terms 2 (2 pi)^2 (b_d . b_e) s_d s_e of G = 2 pi sum_d s_d b_d.
__device__ __forceinline__ double gsq_k(int f0, int f1, int f2, const double* __restrict__ g2t,
                                        const int* Nf, const KLevels& K) {
  double g = gsq(f0, f1, f2, g2t, Nf);
  if (K.skew) {
    const double s0 = signed_freq(f0, Nf[0]), s1 = signed_freq(f1, Nf[1]), s2 = signed_freq(f2, Nf[2]);
    g += K.gq[0] * s0 * s1 + K.gq[1] * s0 * s2 + K.gq[2] * s1 * s2;
  }
  return g;
}

// Fine spectrum S(G) = sum_k [|G| < G_k] rho^_k(G) / N_k (unnormalised level DFTs):
// Fourier interpolation of every level onto the finest grid; one C2R then gives rho.
// One block row per plane m0 (blockIdx.y), the plane's N1 x (N2/2 + 1) elements along x.
__global__ void combine_kernel(const KLevels K, const double* __restrict__ g2t,
                               const cufftDoubleComplex* __restrict__ spec,
                               cufftDoubleComplex* __restrict__ fspec) {
  const LevelInfo& f = K.lv[0];
  const int h2 = f.N[2] / 2 + 1;
  const int plane = f.N[1] * h2;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < plane) {
    const int m0 = blockIdx.y;
    const int m1 = j / h2, m2 = j - m1 * h2;
    const long long idx = (long long)m0 * plane + j;
    const int s0 = signed_freq(m0, f.N[0]), s1 = signed_freq(m1, f.N[1]), s2 = m2;
    const double G2 = gsq_k(m0, m1, m2, g2t, f.N, K);
    double re = 0.0, im = 0.0;
    for (int k = 0; k < K.nlev; ++k) {
      const LevelInfo& lv = K.lv[k];
      if (!(G2 < lv.Gk2)) continue;
      if (2 * abs(s0) > lv.N[0] - 1 || 2 * abs(s1) > lv.N[1] - 1 || 2 * s2 > lv.N[2] - 1) continue;
      const int i0 = s0 < 0 ? s0 + lv.N[0] : s0;
      const int i1 = s1 < 0 ? s1 + lv.N[1] : s1;
      const double inv = K.invn[k];
      const cufftDoubleComplex z =
          spec[lv.spec_off + ((long long)i0 * lv.N[1] + i1) * (lv.N[2] / 2 + 1) + s2];
      re += z.x * inv;
      im += z.y * inv;
    }
    fspec[idx].x = re;
    fspec[idx].y = im;
  }
}

// Level spectrum from fine spectra: T_k(G) = [|G| < G_k] (fa(G) sa + fb(G)), where fa is
// an unnormalised DFT (sa = 1/N_fine) and fb, if given, is already a normalised spectrum.
__global__ void restrict_kernel(const KLevels K, const double* __restrict__ g2t, int level,
                                const cufftDoubleComplex* __restrict__ fa,
                                const cufftDoubleComplex* __restrict__ fb,
                                cufftDoubleComplex* __restrict__ spec) {
  const LevelInfo& f = K.lv[0];
  const LevelInfo& lv = K.lv[level];
  const int h2 = lv.N[2] / 2 + 1, fh2 = f.N[2] / 2 + 1;
  const long long total = (long long)lv.N[0] * lv.N[1] * h2;
  const double inv = 1.0 / ((double)f.N[0] * f.N[1] * f.N[2]);
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int m2 = (int)(idx % h2);
    const long long r = idx / h2;
    const int m1 = (int)(r % lv.N[1]);
    const int m0 = (int)(r / lv.N[1]);
    const int s0 = signed_freq(m0, lv.N[0]), s1 = signed_freq(m1, lv.N[1]), s2 = m2;
    cufftDoubleComplex out;
    out.x = 0.0;
    out.y = 0.0;
    const int i0 = s0 < 0 ? s0 + f.N[0] : s0;
    const int i1 = s1 < 0 ? s1 + f.N[1] : s1;
    const double G2 = gsq_k(i0, i1, s2, g2t, f.N, K);
    if (G2 < lv.Gk2 && 2 * abs(s0) <= lv.N[0] - 1 && 2 * abs(s1) <= lv.N[1] - 1 &&
        2 * s2 <= lv.N[2] - 1) {
      const long long fi = ((long long)i0 * f.N[1] + i1) * fh2 + s2;
      const cufftDoubleComplex z = fa[fi];
      out.x = z.x * inv;
      out.y = z.y * inv;
      if (fb) {
        const cufftDoubleComplex w = fb[fi];
        out.x += w.x;
        out.y += w.y;
      }
    }
    spec[lv.spec_off + idx] = out;
  }
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
  const int tid = threadIdx.x;
  sh[tid] = v;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (tid < s) sh[tid] += sh[tid + s];
    __syncthreads();
  }
  return sh[0];
}

// Poisson in place on the fine spectrum (Eqs. vH, vHG): S <- 4 pi S / |G|^2, G = 0
// dropped; E_H = (Omega/2) sum_G |S|^2 4 pi / |G|^2 over the full spectrum (half
// spectrum weighted by Hermitian symmetry), block partials to red.
__global__ void poisson_kernel(const KLevels K, const double* __restrict__ g2t, double omega,
                               cufftDoubleComplex* __restrict__ fspec, double* __restrict__ red) {
  __shared__ double sh[kRedThreads];
  const LevelInfo& f = K.lv[0];
  const int h2 = f.N[2] / 2 + 1;
  const long long total = (long long)f.N[0] * f.N[1] * h2;
  double part = 0.0;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int m2 = (int)(idx % h2);
    const long long r = idx / h2;
    const int m1 = (int)(r % f.N[1]);
    const int m0 = (int)(r / f.N[1]);
    const double G2 = gsq_k(m0, m1, m2, g2t, f.N, K);
    cufftDoubleComplex z = fspec[idx];
    double kern = G2 > 0.0 ? (4.0 * 3.141592653589793) / G2 : 0.0;
    const double mult = (m2 == 0 || (f.N[2] % 2 == 0 && m2 == f.N[2] / 2)) ? 1.0 : 2.0;
    part += mult * kern * (z.x * z.x + z.y * z.y);
    z.x *= kern;
    z.y *= kern;
    fspec[idx] = z;
  }
  const double s = block_sum(part, sh);
  if (threadIdx.x == 0) red[blockIdx.x] = 0.5 * omega * s;
}

// Slater exchange on the fine grid (Sec. II, LDA), summed with v_H:
// v_out = v_H - (3/pi)^(1/3) rho+^(1/3); E_x partials (Omega/N) sum -(3/4)(3/pi)^(1/3) rho+^(4/3).
__global__ void lda_kernel(long long n, double wgt, const double* __restrict__ rho,
                           const double* __restrict__ vH, double* __restrict__ vout,
                           double* __restrict__ red) {
  __shared__ double sh[kRedThreads];
  const double cx = 0.98474502184269641;  // (3/pi)^(1/3)
  double part = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double r = fmax(rho[i], 0.0);
    const double c = cbrt(r);
    vout[i] = (vH ? vH[i] : 0.0) - cx * c;
    part += -0.75 * cx * r * c;
  }
  const double s = block_sum(part, sh);
  if (threadIdx.x == 0) red[blockIdx.x] = wgt * s;
}

// ----------------------------------------------------------------------------------
// Kinetic energy density of meta-GGA functionals (Sec. II, meta-GGA):
//   tau(r) = (1/2) sum D_mu,nu grad phi_mu . grad phi_nu,
// and its Fock term (1/2) int v_tau grad phi_mu . grad phi_nu (Eq. J_metaGGA).  Per
// dimension d, d/dx_d of (x - A)^a exp(-alpha_a (x - A)^2) is a_d (x - A)^(a - e_d) -
// 2 alpha_a (x - A)^(a + e_d) (times the exponential), so grad phi_a . grad phi_b is a
// sum of twelve shifted pair products; expanding (x - B)^b' about A (Eq. binomial) gives
// a coefficient tensor of degree L + 2 over the monomials (x - A)^k, which the
// collocation kernel contracts like the density's (its degree raised by 2).

// Term of d/dx_d on a monomial exponent c (shift -1: c_d, shift +1: -2 alpha).
__device__ __forceinline__ double dcoef(int cd, int shift, double alpha) {
  return shift < 0 ? (double)cd : -2.0 * alpha;
}

// Pair coefficient tensor of tau: Dt[k] = w pref (1/2) sum_mu,nu D_mu,nu sum_d sum of the
// four (a +- e_d, b +- e_d) terms, binomially expanded about A.  One thread per pair.
__global__ void pair_coef_tau_kernel(long long np, const int4* __restrict__ ids,
                                     const int4* __restrict__ ids2, const double* __restrict__ geo,
                                     const double* __restrict__ pref,
                                     const long long* __restrict__ coef_off,
                                     const double* __restrict__ D, int nao,
                                     double* __restrict__ coef) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const int4 id = ids[p];
  const int la = id.x, lb = id.y, Lt = la + lb + 2;
  const int na = (la + 1) * (la + 2) / 2, nb = (lb + 1) * (lb + 2) / 2;
  const double* g = geo + 8 * p;
  const double aa = g[6], ab = g[7];
  double pw[3][5];  // (A_d - B_d)^j, j <= lb + 1
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double t = g[d] - g[3 + d];
    pw[d][0] = 1.0;
#pragma unroll
    for (int k = 1; k < 5; ++k) pw[d][k] = pw[d][k - 1] * t;
  }
  double acc[nc3(kLmax + 2)];
  const int nc = nc3(Lt);
  for (int c = 0; c < nc; ++c) acc[c] = 0.0;
  const double scale = 0.5 * (double)ids2[p].z * pref[p];
  for (int mu = 0; mu < na; ++mu) {
    int a[3];
    cart_comp(la, mu, a);
    const double* Drow = D + (long long)(id.z + mu) * nao + id.w;
    for (int nu = 0; nu < nb; ++nu) {
      int b[3];
      cart_comp(lb, nu, b);
      const double dmn = scale * Drow[nu];
      for (int d = 0; d < 3; ++d)
        for (int sa = -1; sa <= 1; sa += 2)
          for (int sb = -1; sb <= 1; sb += 2) {
            const double c = dmn * dcoef(a[d], sa, aa) * dcoef(b[d], sb, ab);
            int a2[3] = {a[0], a[1], a[2]}, b2[3] = {b[0], b[1], b[2]};
            a2[d] += sa;
            b2[d] += sb;
            if (c == 0.0 || a2[d] < 0 || b2[d] < 0) continue;
            for (int t2 = 0; t2 <= b2[2]; ++t2) {
              const double c2 = c * binom(b2[2], t2) * pw[2][b2[2] - t2];
              for (int t1 = 0; t1 <= b2[1]; ++t1) {
                const double c21 = c2 * binom(b2[1], t1) * pw[1][b2[1] - t1];
                for (int t0 = 0; t0 <= b2[0]; ++t0)
                  acc[mono_index(a2[0] + t0, a2[1] + t1, a2[2] + t2, Lt)] +=
                      c21 * binom(b2[0], t0) * pw[0][b2[0] - t0];
              }
            }
          }
    }
  }
  double* out = coef + coef_off[p];
  for (int c = 0; c < nc; ++c) out[c] = acc[c];
}

// Coefficients of the i-th derivative of (x - X)^c e^{-alpha (x - X)^2}: sum over the
// returned shifts s of w_s (x - X)^(c + s) (times the exponential); returns the count.
__device__ __forceinline__ int deriv_terms(int c, int i, double alpha, int* sh, double* w) {
  const double cd = (double)c;
  if (i == 0) {
    sh[0] = 0;
    w[0] = 1.0;
    return 1;
  }
  if (i == 1) {
    sh[0] = -1;
    w[0] = cd;
    sh[1] = 1;
    w[1] = -2.0 * alpha;
    return 2;
  }
  sh[0] = -2;
  w[0] = cd * (cd - 1.0);
  sh[1] = 0;
  w[1] = -2.0 * alpha * (2.0 * cd + 1.0);
  sh[2] = 2;
  w[2] = 4.0 * alpha * alpha;
  return 3;
}

// 1-D product u^(i) w^(j) in powers of (x - A): out[k], k <= a + b + i + j (<= 9);
// pw[m] = (A - B)^m.
__device__ __forceinline__ void prod_1d(int a, int b, int i, int j, double aa, double ab,
                                       const double* pw, double* out) {
#pragma unroll
  for (int k = 0; k < 10; ++k) out[k] = 0.0;
  int su[3], sw[3];
  double wu[3], ww[3];
  const int nu = deriv_terms(a, i, aa, su, wu), nw = deriv_terms(b, j, ab, sw, ww);
  for (int p = 0; p < nu; ++p) {
    const int ea = a + su[p];
    if (ea < 0 || wu[p] == 0.0) continue;
    for (int q = 0; q < nw; ++q) {
      const int eb = b + sw[q];
      if (eb < 0 || ww[q] == 0.0) continue;
      const double c = wu[p] * ww[q];
      // (x - B)^eb = sum_m C(eb, m) (A - B)^(eb - m) (x - A)^m
      for (int m = 0; m <= eb; ++m) out[ea + m] += c * binom(eb, m) * pw[eb - m];
    }
  }
}

// sum_{k0,k1,k2} f0[k0] f1[k1] f2[k2] V[k0,k1,k2] over k_c <= n_c (n0 + n1 + n2 <= Lx)
__device__ __forceinline__ double contract3(const double* f0, int n0, const double* f1, int n1,
                                            const double* f2, int n2, const double* V, int Lx) {
  double s0 = 0.0;
  for (int k0 = 0; k0 <= n0; ++k0) {
    if (f0[k0] == 0.0) continue;
    double s1 = 0.0;
    for (int k1 = 0; k1 <= n1; ++k1) {
      if (f1[k1] == 0.0) continue;
      double s2 = 0.0;
      for (int k2 = 0; k2 <= n2; ++k2) s2 = fma(f2[k2], V[mono_index(k0, k1, k2, Lx)], s2);
      s1 = fma(f1[k1], s2, s1);
    }
    s0 = fma(f0[k0], s1, s0);
  }
  return s0;
}

// (1/2) grad phi_a . grad phi_b integrated against the potential, from the pair's V
// tensor of degree Lx: per dimension d the product d_d phi_a d_d phi_b is the 1-D factor
// u' w' in d times u w in the other two, each expanded in powers of (x - A).
__device__ double xtau(const int* a, const int* b, double aa, double ab, const double (*pw)[6],
                       const double* V, int Lx) {
  double P0[3][10], P1[3][10];
  for (int c = 0; c < 3; ++c) {
    prod_1d(a[c], b[c], 0, 0, aa, ab, pw[c], P0[c]);
    prod_1d(a[c], b[c], 1, 1, aa, ab, pw[c], P1[c]);
  }
  const int n0[3] = {a[0] + b[0], a[1] + b[1], a[2] + b[2]};
  double s = contract3(P1[0], n0[0] + 2, P0[1], n0[1], P0[2], n0[2], V, Lx);
  s += contract3(P0[0], n0[0], P1[1], n0[1] + 2, P0[2], n0[2], V, Lx);
  s += contract3(P0[0], n0[0], P0[1], n0[1], P1[2], n0[2] + 2, V, Lx);
  return 0.5 * s;
}

// V^tau assembly: one warp per contracted shell pair, lanes over its elements and lane
// groups over its pairs (as assemble_V_kernel, with xtau in place of the plain pair
// product).
__global__ void assemble_V_tau_kernel(long long ngroups, const int4* __restrict__ groups,
                                      const int4* __restrict__ ids, const int4* __restrict__ ids2,
                                      const double* __restrict__ geo,
                                      const double* __restrict__ pref,
                                      const long long* __restrict__ coef_off,
                                      const double* __restrict__ coef,
                                      const CoefTables* __restrict__ tabs, int nao, int lext,
                                      double* __restrict__ V) {
  const int lane = threadIdx.x & 31;
  long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (gw >= ngroups) return;
  const int4 gr = groups[gw];
  const int4 id0 = ids[gr.z];
  const int la = id0.x, lb = id0.y, Lx = la + lb + lext;
  const int na = (la + 1) * (la + 2) / 2, nb = (lb + 1) * (lb + 2) / 2;
  const int nel = na * nb;
  const bool diag = gr.x == gr.y;
  int C = 1;
  while (C < nel && C < 32) C <<= 1;
  const int G = 32 / C, g = lane / C, e = lane - g * C;
  for (int base = 0; base < nel; base += C) {
    const int el = base + e;
    double tot = 0.0;
    if (el < nel) {
      const int mu = el / nb, nu = el - mu * nb;
      int ca[3], cb[3];
      cart_comp(la, mu, ca);
      cart_comp(lb, nu, cb);
      for (int p = gr.z + g; p < gr.w; p += G) {
        const double* gp = geo + 8LL * p;
        double pw[3][6];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          const double t = gp[d] - gp[3 + d];
          pw[d][0] = 1.0;
#pragma unroll
          for (int k = 1; k < 6; ++k) pw[d][k] = pw[d][k - 1] * t;
        }
        const double* Vp = coef + coef_off[p];
        double x = xtau(ca, cb, gp[6], gp[7], pw, Vp, Lx);
        if (diag && ids2[p].z == 2) {
          int ca2[3], cb2[3];
          cart_comp(la, nu, ca2);
          cart_comp(lb, mu, cb2);
          x += xtau(ca2, cb2, gp[6], gp[7], pw, Vp, Lx);
        }
        tot += pref[p] * x;
      }
    }
    for (int o = C; o < 32; o <<= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
    if (g == 0 && el < nel) {
      const int mu = el / nb, nu = el - mu * nb;
      V[(long long)(id0.z + mu) * nao + id0.w + nu] = tot;
      if (!diag) V[(long long)(id0.w + nu) * nao + id0.z + mu] = tot;
    }
  }
}

// Nuclear gradient of <v_tau, tau(D)> per pair from its degree-(L+3) V tensor: the centre
// derivative of grad phi_a is minus its Hessian in x, so
//   dE/dA_d = -w pref (1/2) sum_mu,nu D_mu,nu sum_e <d_d d_e phi_a, d_e phi_b>,
//   dE/dB_d = -w pref (1/2) sum_mu,nu D_mu,nu sum_e <d_e phi_a, d_d d_e phi_b>.
// Every bracket is a product over the three dimensions of 1-D factors
// u^(i)(x) w^(j)(x), u = (x - A)^a e^{-alpha_a (x - A)^2} and w likewise about B, i and j
// the derivative orders in that dimension: (2,1) or (1,0)/(1,1) for the A brackets,
// (1,2) or (0,1)/(1,1) for the B brackets, (0,0) elsewhere.  Per (mu, nu) the six 1-D
// products of each dimension are expanded once in powers of (x - A) (Eq. binomial), and
// each bracket is the triple contraction of three of them with V.  One thread per pair
// (pairs of one class are adjacent, so the threads of a warp do equal work).

__global__ void grad_tau_pair_kernel(long long np, const int4* __restrict__ ids,
                                     const int4* __restrict__ ids2, const double* __restrict__ geo,
                                     const double* __restrict__ pref,
                                     const long long* __restrict__ coef_off,
                                     const double* __restrict__ coef,
                                     const CoefTables* __restrict__ tabs,
                                     const double* __restrict__ D, int nao,
                                     double* __restrict__ pgrad) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const int4 id = ids[p];
  const int la = id.x, lb = id.y, Lx = la + lb + 3;
  const int na = (la + 1) * (la + 2) / 2, nb = (lb + 1) * (lb + 2) / 2;
  const double* g = geo + 8 * p;
  const double aa = g[6], ab = g[7];
  double pw[3][6];  // (A_d - B_d)^j, j <= lb + 2
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double t = g[d] - g[3 + d];
    pw[d][0] = 1.0;
#pragma unroll
    for (int k = 1; k < 6; ++k) pw[d][k] = pw[d][k - 1] * t;
  }
  const double* Vp = coef + coef_off[p];
  const double scale = -0.5 * (double)ids2[p].z * pref[p];
  // derivative orders (i, j) of the six 1-D products: 00, 10, 01, 11, 21, 12
  const int ti[6] = {0, 1, 0, 1, 2, 1}, tj[6] = {0, 0, 1, 1, 1, 2};
  double gA[3] = {0.0, 0.0, 0.0}, gB[3] = {0.0, 0.0, 0.0};
  double P[3][6][10];
  int deg[3][6];
  for (int mu = 0; mu < na; ++mu) {
    int a[3];
    cart_comp(la, mu, a);
    const double* Drow = D + (long long)(id.z + mu) * nao + id.w;
    for (int nu = 0; nu < nb; ++nu) {
      int b[3];
      cart_comp(lb, nu, b);
      const double dmn = scale * Drow[nu];
      for (int c = 0; c < 3; ++c)
        for (int t = 0; t < 6; ++t) {
          prod_1d(a[c], b[c], ti[t], tj[t], aa, ab, pw[c], P[c][t]);
          deg[c][t] = a[c] + b[c] + ti[t] + tj[t];
        }
      for (int d = 0; d < 3; ++d) {
        const int e1 = (d + 1) % 3, e2 = (d + 2) % 3;
        // types per dimension of the brackets, dimension order (d, e1, e2) mapped to (0,1,2)
        int tA[3][3], tB[3][3];
        for (int r = 0; r < 3; ++r)
          for (int c = 0; c < 3; ++c) tA[r][c] = tB[r][c] = 0;
        tA[0][d] = 4;                 // e = d: (2,1) in d
        tA[1][d] = 1; tA[1][e1] = 3;  // e = e1: (1,0) in d, (1,1) in e1
        tA[2][d] = 1; tA[2][e2] = 3;
        tB[0][d] = 5;                 // e = d: (1,2) in d
        tB[1][d] = 2; tB[1][e1] = 3;  // e = e1: (0,1) in d, (1,1) in e1
        tB[2][d] = 2; tB[2][e2] = 3;
        double sA = 0.0, sB = 0.0;
        for (int r = 0; r < 3; ++r) {
          sA += contract3(P[0][tA[r][0]], deg[0][tA[r][0]], P[1][tA[r][1]], deg[1][tA[r][1]],
                          P[2][tA[r][2]], deg[2][tA[r][2]], Vp, Lx);
          sB += contract3(P[0][tB[r][0]], deg[0][tB[r][0]], P[1][tB[r][1]], deg[1][tB[r][1]],
                          P[2][tB[r][2]], deg[2][tB[r][2]], Vp, Lx);
        }
        gA[d] += dmn * sA;
        gB[d] += dmn * sB;
      }
    }
  }
  double* out = pgrad + 6 * p;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    out[d] = gA[d];
    out[3 + d] = gB[d];
  }
}

// Fourier derivative on the finest half spectrum (Sec. II, GGA): out = i G_d in, or
// out -= i G_d in (subtract).  G_d = (2 pi s)/L_d from a host table that is zero on the
// Nyquist plane of an even axis.
__global__ void fourier_deriv_kernel(const KLevels K, const double* __restrict__ g1t, int axis,
                                     const cufftDoubleComplex* __restrict__ in,
                                     cufftDoubleComplex* __restrict__ out, int subtract) {
  const LevelInfo& f = K.lv[0];
  const int h2 = f.N[2] / 2 + 1;
  const long long total = (long long)f.N[0] * f.N[1] * h2;
  const int off = axis == 0 ? 0 : (axis == 1 ? f.N[0] : f.N[0] + f.N[1]);
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int m2 = (int)(idx % h2);
    const long long r = idx / h2;
    const int m1 = (int)(r % f.N[1]);
    const int m0 = (int)(r / f.N[1]);
    const int m = axis == 0 ? m0 : (axis == 1 ? m1 : m2);
    // orthorhombic: the axis table holds (2 pi s)/L_d; non-orthogonal: the tables hold
    // 2 pi s per mesh axis and the Cartesian component is sum_d 2 pi s_d (b_d)_axis
    const double g = K.skew ? __ldg(g1t + m0) * K.rec[axis] + __ldg(g1t + f.N[0] + m1) * K.rec[3 + axis] +
                                  __ldg(g1t + f.N[0] + f.N[1] + m2) * K.rec[6 + axis]
                            : __ldg(g1t + off + m);
    const cufftDoubleComplex z = in[idx];
    if (subtract) {
      cufftDoubleComplex o = out[idx];
      o.x += g * z.y;
      o.y -= g * z.x;
      out[idx] = o;
    } else {
      cufftDoubleComplex o;
      o.x = -g * z.y;
      o.y = g * z.x;
      out[idx] = o;
    }
  }
}

// PBE exchange at every finest-grid point (spin-unpolarised, rho+ = max(rho, 0)):
//   e = e_x^LDA F_x(s), e_x^LDA = -(3/4)(3/pi)^(1/3) rho^(4/3),
//   s^2 = sigma / (4 k_F^2 rho^2), k_F^2 = (3 pi^2 rho)^(2/3), sigma = |grad rho|^2,
//   F_x = 1 + kappa - kappa / (1 + mu s^2 / kappa),
// writes de/drho to v_rho and 2 de/dsigma grad rho over grad (in place); e = 0 where
// rho <= 1e-12.  Per-block partial sums of (Omega/N) e.
__global__ void pbe_x_kernel(long long n, double wgt, const double* __restrict__ rho,
                             double* __restrict__ gx, double* __restrict__ gy,
                             double* __restrict__ gz, double* __restrict__ v_rho,
                             double* __restrict__ red) {
  __shared__ double sh[kRedThreads];
  const double cx = 0.98474502184269641;        // (3/pi)^(1/3)
  const double three_pi2 = 29.608813203268074;  // 3 pi^2
  const double kappa = 0.804, mu = 0.21951497276451704;
  double part = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const double r = fmax(rho[i], 0.0);
    const double x = gx[i], y = gy[i], z = gz[i];
    double e = 0.0, dedr = 0.0, deds = 0.0;
    if (r > 1e-12) {
      const double r13 = cbrt(r);
      const double elda = -0.75 * cx * r * r13;
      const double delda = -cx * r13;
      const double c = cbrt(three_pi2 * r);
      const double ds2 = 1.0 / (4.0 * (c * c) * r * r);  // d s^2 / d sigma
      const double s2 = (x * x + y * y + z * z) * ds2;
      const double den = 1.0 + mu * s2 / kappa;
      const double F = 1.0 + kappa - kappa / den;
      const double dF = mu / (den * den);
      e = elda * F;
      dedr = delda * F + elda * dF * (-8.0 / 3.0) * s2 / r;
      deds = elda * dF * ds2;
    }
    v_rho[i] = dedr;
    gx[i] = 2.0 * deds * x;
    gy[i] = 2.0 * deds * y;
    gz[i] = 2.0 * deds * z;
    part += e;
  }
  const double s = block_sum(part, sh);
  if (threadIdx.x == 0) red[blockIdx.x] = wgt * s;
}

// out = fa / N_fine + fb on the finest half spectrum (the potential's spectrum)
__global__ void spec_combine_kernel(long long total, double inv,
                                    const cufftDoubleComplex* __restrict__ fa,
                                    const cufftDoubleComplex* __restrict__ fb,
                                    cufftDoubleComplex* __restrict__ out) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    cufftDoubleComplex o;
    o.x = fa[i].x * inv + fb[i].x;
    o.y = fa[i].y * inv + fb[i].y;
    out[i] = o;
  }
}

__global__ void energy_final_kernel(const double* __restrict__ red, int nparts,
                                    double* __restrict__ out) {
  __shared__ double sh[kRedThreads];
  double v = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) v += red[i];
  const double s = block_sum(v, sh);
  if (threadIdx.x == 0) *out = s;
}

// GPW_DEBUG_CHECKS: a value that is not finite in an output
__global__ void finite_check_kernel(const double* __restrict__ x, long long n, int* err) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    if (!isfinite(x[i])) {
      set_err(err, 16);
      return;
    }
}

// GPW_DEBUG_CHECKS at commit: every task of a list against its sub-box (one thread per
// sub-box): the pair exists, its level is the sub-box's, the record's degree and pair-box
// extents are the pair's, the intersection lies inside the sub-box and the pair box and
// sits, wrapped, where the record says, and the pairs come in order.
__global__ void validate_tasks_kernel(const KLevels K, int T0, int T1, int T2, int W2, long long nsub,
                                      const long long* __restrict__ sub_off,
                                      const int4* __restrict__ task,
                                      const int4* __restrict__ hot_a,
                                      const int4* __restrict__ hot_b, long long np, int* err) {
  const int T[3] = {T0, T1, T2}, Wd[3] = {T0, T1, W2};
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < nsub;
       g += (long long)gridDim.x * blockDim.x) {
    int k = 0;
    while (k + 1 < K.nlev && K.lv[k + 1].sub_base <= g) ++k;
    const LevelInfo& lv = K.lv[k];
    const long long sub = g - lv.sub_base;
    const long long j2 = sub % lv.nsb[2], j1 = (sub / lv.nsb[2]) % lv.nsb[1],
                    j0 = sub / ((long long)lv.nsb[2] * lv.nsb[1]);
    const long long j[3] = {j0, j1, j2};
    bool ok = sub_off[g] <= sub_off[g + 1];
    long long prev = -1;
    for (long long e = sub_off[g]; ok && e < sub_off[g + 1]; ++e) {
      const int4 r0 = task[2 * e], r1 = task[2 * e + 1];
      const long long p = r0.x;
      ok = p >= 0 && p < np && p >= prev;
      if (!ok) break;
      prev = p;
      const int4 ha = hot_a[p], hb = hot_b[p];
      const int lo[3] = {ha.x, ha.y, ha.z}, n[3] = {hb.x, hb.y, hb.z};
      const int rt[3] = {r1.x, r1.y, r1.z};
      ok = hb.w == k && ((r0.y >> 24) & 255) == ha.w;
      for (int d = 0; d < 3 && ok; ++d) {
        const int m = (r0.y >> (8 * d)) & 255, u = (r0.z >> (8 * d)) & 255;
        const int t = rt[d] & 0xffff, nn = (rt[d] >> 16) & 0xffff;
        const long long s0 = j[d] * T[d];
        const long long ext = min((long long)Wd[d], (long long)lv.N[d] - s0);
        const long long i = (long long)lo[d] + t;
        const long long w = ((i % lv.N[d]) + lv.N[d]) % lv.N[d];
        ok = nn == n[d] && m >= 1 && u + m <= ext && t + m <= n[d] && w == s0 + u;
      }
    }
    if (!ok) set_err(err, 17);
  }
}

int even(int x) { return (x + 1) & ~1; }

constexpr int kNW = 8;

// Sub-box shapes with compiled kernels: collocation, and integration (a superset).
#define GPW_COLLOC_SHAPES(X) \
  X(8, 8, 16) X(4, 8, 32) X(8, 8, 32) X(4, 8, 64) X(4, 8, 16) X(4, 4, 16) X(2, 8, 16) X(4, 4, 32)
#define GPW_INTEG_SHAPES(X) GPW_COLLOC_SHAPES(X) X(8, 8, 64) X(8, 4, 64)
// Integration sub-boxes (a, b, c) with z windows of w > c points (overlapping windows).
#define GPW_INTEG_WSHAPES(X) X(8, 8, 16, 48)

// per-warp staging doubles of the non-orthogonal variants (cross factors and their rows)
template <int T0, int T1, int T2>
int colloc_skew_extra(bool zc) { return zc ? 2 * CrossWindowsZ<T0, T1, T2>::kSize : 0; }
// collocation staging of the non-orthogonal variants (SK = 1 with every cross term adds
// the R02 and R12 windows)
template <int T0, int T1, int T2>
int colloc_skew_stage(bool zc, int lp) {
  return even(even(CollocLayout<T0, T1, T2>::stage(lp)) + colloc_skew_extra<T0, T1, T2>(zc));
}
template <int T0, int T1, int T2>
int integ_skew_extra(bool zc) {
  return (zc ? IntegLayout<T0, T1, T2>::kSV : 0) + 2 * CrossWindows<T0, T1, T2>::kSize;
}

template <int T0, int T1, int T2>
size_t colloc_smem(int stg, int nw) {
  return sizeof(double) * (size_t)nw * (T0 * T1 * T2 + stg);
}

template <int T0, int T1, int T2>
size_t integ_smem(int stg) {
  return sizeof(int) * kDec21Ints + sizeof(double) * ((size_t)IntegLayout<T0, T1, T2>::kSV + (size_t)kNW * stg);
}

// Warps per collocation block: the candidate with the most resident warps per SM, as the
// occupancy calculator reports it for this shared-memory size (registers included), the
// larger block on a tie.
template <int T0, int T1, int T2, int SK = 0>
int pick_colloc_warps(int stg, int want, int* nw_out, size_t* smem_out) {
  int best = 0;
  // a tie in resident warps goes to the larger block: smaller blocks make each sub-box
  // take longer, which the launch's tail pays on small cells (4-warp blocks ran the
  // 32-water collocation 30% slower, for 1% on the 256-water one)
  const void* fns[3] = {(const void*)collocate_kernel<T0, T1, T2, 8, SK>,
                        (const void*)collocate_kernel<T0, T1, T2, 6, SK>,
                        (const void*)collocate_kernel<T0, T1, T2, 4, SK>};
  const int nws[3] = {8, 6, 4};
  for (int i = 0; i < 3; ++i) {
    if (want != 0 && nws[i] != want) continue;  // a requested count (still must fit)
    const size_t need = colloc_smem<T0, T1, T2>(stg, nws[i]);
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fns[i], nws[i] * 32, need) != cudaSuccess)
      continue;
    if (blocks * nws[i] > best) {
      best = blocks * nws[i];
      *nw_out = nws[i];
      *smem_out = need;
    }
  }
  return best;
}

}  // namespace

extern "C" int gpw_tile_supported(int t0, int t1, int t2) {
  int r = 0;
#define GPW_TILE_CHECK_C(a, b, c) \
  if (t0 == a && t1 == b && t2 == c) r |= GPW_TILE_COLLOC;
#define GPW_TILE_CHECK_I(a, b, c) \
  if (t0 == a && t1 == b && t2 == c) r |= GPW_TILE_INTEG;
  GPW_COLLOC_SHAPES(GPW_TILE_CHECK_C)
  GPW_INTEG_SHAPES(GPW_TILE_CHECK_I)
#undef GPW_TILE_CHECK_C
#undef GPW_TILE_CHECK_I
  return r;
}

extern "C" int gpw_integ_zwin_supported(int t0, int t1, int t2, int zwin) {
  if (zwin == t2) return (gpw_tile_supported(t0, t1, t2) & GPW_TILE_INTEG) ? 1 : 0;
#define GPW_ZWIN_CHECK(a, b, c, w) \
  if (t0 == a && t1 == b && t2 == c && zwin == w) return 1;
  GPW_INTEG_WSHAPES(GPW_ZWIN_CHECK)
#undef GPW_ZWIN_CHECK
  return 0;
}

KLevels make_klevels(const Plan& p, bool integ) {
  KLevels k;
  for (int i = 0; i < GPW_MAX_LEVELS; ++i) k.lv[i] = integ ? p.lev_i[i] : p.lev[i];
  k.nlev = p.nlev;
  k.skew = p.skew ? 1 : 0;
  const double tp2 = 2.0 * (2.0 * M_PI) * (2.0 * M_PI);
  const int pd[3][2] = {{0, 1}, {0, 2}, {1, 2}};
  for (int i = 0; i < 3; ++i) {
    const double* bd = p.rec + 3 * pd[i][0];
    const double* be = p.rec + 3 * pd[i][1];
    k.gq[i] = p.skew ? tp2 * (bd[0] * be[0] + bd[1] * be[1] + bd[2] * be[2]) : 0.0;
  }
  for (int i = 0; i < 9; ++i) k.rec[i] = p.rec[i];
  for (int i = 0; i < GPW_MAX_LEVELS; ++i) {
    const LevelInfo& l = integ ? p.lev_i[i] : p.lev[i];
    k.invn[i] = i < p.nlev ? 1.0 / ((double)l.N[0] * l.N[1] * l.N[2]) : 0.0;
  }
  return k;
}

size_t integ_block_smem(const int* tile, int zwin, int lmax) {
#define GPW_SMEM_IW(a, b, c, w)                                                       \
  if (tile[0] == a && tile[1] == b && tile[2] == c && zwin == w)                      \
    return integ_smem<a, b, w>(even(IntegLayout<a, b, w>::stage(lmax + 2)));
#define GPW_SMEM_I(a, b, c) GPW_SMEM_IW(a, b, c, c)
  GPW_INTEG_SHAPES(GPW_SMEM_I)
  GPW_INTEG_WSHAPES(GPW_SMEM_IW)
#undef GPW_SMEM_I
#undef GPW_SMEM_IW
  return 0;
}

cudaError_t configure_kernels(Plan* p) {
  const int lp = p->lmax + 1;
  int found = 0;
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  // the attribute is per function and shared by all plans: raise it to the device
  // maximum (before the occupancy queries below), each launch asks for what it needs
#define GPW_TILE_ATTR(a, b, c)                                                                    \
  e = cudaFuncSetAttribute(collocate_kernel<a, b, c, 8>,                                          \
                           cudaFuncAttributeMaxDynamicSharedMemorySize, optin);                   \
  if (e != cudaSuccess) return e;                                                                 \
  e = cudaFuncSetAttribute(collocate_kernel<a, b, c, 6>,                                          \
                           cudaFuncAttributeMaxDynamicSharedMemorySize, optin);                   \
  if (e != cudaSuccess) return e;                                                                 \
  e = cudaFuncSetAttribute(collocate_kernel<a, b, c, 4>,                                          \
                           cudaFuncAttributeMaxDynamicSharedMemorySize, optin);                   \
  if (e != cudaSuccess) return e;
#define GPW_TILE_ATTR_I(a, b, c)                                                                  \
  e = cudaFuncSetAttribute(integrate_kernel<a, b, c, kNW>,                                        \
                           cudaFuncAttributeMaxDynamicSharedMemorySize, optin);                   \
  if (e != cudaSuccess) return e;
#define GPW_TILE_ATTR_W(a, b, c, w)                                                               \
  e = cudaFuncSetAttribute(integrate_kernel<a, b, w, kNW, 0, c>,                                  \
                           cudaFuncAttributeMaxDynamicSharedMemorySize, optin);                   \
  if (e != cudaSuccess) return e;
  GPW_COLLOC_SHAPES(GPW_TILE_ATTR)
  GPW_INTEG_SHAPES(GPW_TILE_ATTR_I)
  GPW_INTEG_WSHAPES(GPW_TILE_ATTR_W)
#undef GPW_TILE_ATTR
#undef GPW_TILE_ATTR_I
#undef GPW_TILE_ATTR_W
  // the non-orthogonal variants (4x8x16 sub-boxes)
  for (const void* f : {(const void*)collocate_kernel<kT0, kT1, kT2, 8, 1>,
                        (const void*)collocate_kernel<kT0, kT1, kT2, 6, 1>,
                        (const void*)collocate_kernel<kT0, kT1, kT2, 4, 1>,
                        (const void*)integrate_kernel<kT0, kT1, kT2, kNW, 1>,
                        (const void*)collocate_kernel<kT0, kT1, kT2, 8, 2>,
                        (const void*)collocate_kernel<kT0, kT1, kT2, 6, 2>,
                        (const void*)collocate_kernel<kT0, kT1, kT2, 4, 2>,
                        (const void*)integrate_kernel<kT0, kT1, kT2, kNW, 2>}) {
    e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e != cudaSuccess) return e;
  }
  if (p->skew) {
    if (!(p->tile[0] == kT0 && p->tile[1] == kT1 && p->tile[2] == kT2 && p->tile_i[0] == kT0 &&
          p->tile_i[1] == kT1 && p->tile_i[2] == kT2))
      return cudaErrorInvalidValue;
    using IL = IntegLayout<kT0, kT1, kT2>;
    const bool zc = p->skew_zc;
    const auto pick = zc ? pick_colloc_warps<kT0, kT1, kT2, 1> : pick_colloc_warps<kT0, kT1, kT2, 2>;
    p->stg_colloc = colloc_skew_stage<kT0, kT1, kT2>(zc, lp);
    if (pick(p->stg_colloc, p->nw_colloc_req, &p->nw_colloc,
                                                &p->smem_colloc) == 0)
      return cudaErrorInvalidValue;
    p->stg_integ = even(even(IL::stage(p->lmax + 1)) + integ_skew_extra<kT0, kT1, kT2>(zc));
    p->stg_integ1 = even(even(IL::stage(p->lmax + 2)) + integ_skew_extra<kT0, kT1, kT2>(zc));
    p->smem_integ = integ_smem<kT0, kT1, kT2>(p->stg_integ);
    p->smem_integ1 = integ_smem<kT0, kT1, kT2>(p->stg_integ1);
    p->nw_integ = kNW;
    if ((size_t)optin < std::max(p->smem_colloc, std::max(p->smem_integ, p->smem_integ1)))
      return cudaErrorInvalidValue;
    if (p->xr) {
      // kinetic-energy density: collocation at degree L+2, integration at L+2 / L+3
      p->stg_colloc_t = colloc_skew_stage<kT0, kT1, kT2>(zc, p->lmax + 3);
      if (pick(p->stg_colloc_t, p->nw_colloc_req,
                                                  &p->nw_colloc_t, &p->smem_colloc_t) == 0)
        return cudaErrorInvalidValue;
      p->stg_integ3 = even(even(IL::stage(p->lmax + 4)) + integ_skew_extra<kT0, kT1, kT2>(zc));
      p->smem_integ3 = integ_smem<kT0, kT1, kT2>(p->stg_integ3);
      if ((size_t)optin < std::max(p->smem_colloc_t, p->smem_integ3)) return cudaErrorInvalidValue;
    }
    return cudaSuccess;
  }
#define GPW_TILE_CONF(a, b, c)                                                      \
  if (p->tile[0] == a && p->tile[1] == b && p->tile[2] == c) {                      \
    found |= 1;                                                                     \
    p->stg_colloc = even(CollocLayout<a, b, c>::stage(lp));                         \
    if (pick_colloc_warps<a, b, c>(p->stg_colloc, p->nw_colloc_req, &p->nw_colloc,         \
                                   &p->smem_colloc) == 0)                                \
      return cudaErrorInvalidValue;                                                 \
  }
#define GPW_TILE_CONF_IW(a, b, c, w)                                                \
  if (p->tile_i[0] == a && p->tile_i[1] == b && p->tile_i[2] == c && p->zwin_i == w) { \
    found |= 2;                                                                     \
    p->stg_integ = even(IntegLayout<a, b, w>::stage(p->lmax + 1));                  \
    p->stg_integ1 = even(IntegLayout<a, b, w>::stage(p->lmax + 2));                 \
    p->smem_integ = integ_smem<a, b, w>(p->stg_integ);                              \
    p->smem_integ1 = integ_smem<a, b, w>(p->stg_integ1);                            \
  }
#define GPW_TILE_CONF_I(a, b, c) GPW_TILE_CONF_IW(a, b, c, c)
  GPW_COLLOC_SHAPES(GPW_TILE_CONF)
  GPW_INTEG_SHAPES(GPW_TILE_CONF_I)
  GPW_INTEG_WSHAPES(GPW_TILE_CONF_IW)
#undef GPW_TILE_CONF
#undef GPW_TILE_CONF_I
#undef GPW_TILE_CONF_IW
  if (found != 3) return cudaErrorInvalidValue;
  p->nw_integ = kNW;
  if (p->xr) {
#define GPW_TILE_CONF_T(a, b, c)                                                             \
  if (p->tile[0] == a && p->tile[1] == b && p->tile[2] == c) {                               \
    p->stg_colloc_t = even(CollocLayout<a, b, c>::stage(p->lmax + 3));                       \
    if (pick_colloc_warps<a, b, c>(p->stg_colloc_t, p->nw_colloc_req, &p->nw_colloc_t,      \
                                   &p->smem_colloc_t) == 0)                                 \
      return cudaErrorInvalidValue;                                                          \
  }
#define GPW_TILE_CONF_I3W(a, b, c, w)                                                        \
  if (p->tile_i[0] == a && p->tile_i[1] == b && p->tile_i[2] == c && p->zwin_i == w) {      \
    p->stg_integ3 = even(IntegLayout<a, b, w>::stage(p->lmax + 4));                          \
    p->smem_integ3 = integ_smem<a, b, w>(p->stg_integ3);                                     \
  }
#define GPW_TILE_CONF_I3(a, b, c) GPW_TILE_CONF_I3W(a, b, c, c)
    GPW_COLLOC_SHAPES(GPW_TILE_CONF_T)
    GPW_INTEG_SHAPES(GPW_TILE_CONF_I3)
    GPW_INTEG_WSHAPES(GPW_TILE_CONF_I3W)
#undef GPW_TILE_CONF_T
#undef GPW_TILE_CONF_I3
#undef GPW_TILE_CONF_I3W
    if ((size_t)optin < std::max(p->smem_colloc_t, p->smem_integ3)) return cudaErrorInvalidValue;
  }
  if ((size_t)optin < std::max(p->smem_colloc, std::max(p->smem_integ, p->smem_integ1)))
    return cudaErrorInvalidValue;
  return cudaSuccess;
}

cudaError_t launch_finite_check(const Plan& p, const double* x, long long n, cudaStream_t s) {
  if (!p.debug || !x || n <= 0) return cudaSuccess;
  ++p.launches;
  const long long blocks = std::min<long long>((n + 255) / 256, 152LL * 8);
  finite_check_kernel<<<(int)blocks, 256, 0, s>>>(x, n, p.d.err);
  return cudaGetLastError();
}

cudaError_t launch_validate_tasks(const Plan& p, bool integ, cudaStream_t s) {
  const long long nsub = integ ? p.nsub_i : p.nsub_total;
  if (!p.debug || nsub <= 0) return cudaSuccess;
  const int* T = integ ? p.tile_i : p.tile;
  ++p.launches;
  const long long blocks = std::min<long long>((nsub + 127) / 128, 152LL * 16);
  validate_tasks_kernel<<<(int)blocks, 128, 0, s>>>(
      make_klevels(p, integ), T[0], T[1], T[2], integ ? p.zwin_i : T[2], nsub,
      integ ? p.d.sub_off_i : p.d.sub_off_c,
      integ ? p.d.task_i : p.d.task_c, p.d.hot_a, p.d.hot_b, p.npairs, p.d.err);
  return cudaGetLastError();
}

cudaError_t launch_tables(const Plan& p, cudaStream_t s) {
  if (p.npairs == 0) return cudaSuccess;
  long long blocks = std::min<long long>((p.npairs + 7) / 8, 152LL * 64);
  ++p.launches;
  tables_kernel<<<(int)blocks, 256, 0, s>>>(p.npairs, make_klevels(p, false), p.d.hot_a, p.d.hot_b,
                                             p.d.geo, p.d.cab, p.d.tab_off, p.d.tab, p.d.pref,
                                             p.xr, p.skew ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_pair_coef(const Plan& p, const double* D, cudaStream_t s) {
  if (p.npairs == 0) return cudaSuccess;
  ++p.launches;
  pair_coef_kernel<<<(int)((p.npairs + 127) / 128), 128, 0, s>>>(
      p.npairs, p.d.hot_a, p.d.ids, p.d.ids2, p.d.geo, p.d.pref, p.d.coef_off, p.d.tabs, D,
      p.nao, p.d.coef);
  if (p.skew) {
    ++p.launches;
    mono_transform_kernel<<<(int)((p.npairs + 127) / 128), 128, 0, s>>>(
        p.npairs, p.d.hot_a, p.d.hot_b, p.d.coef_off, p.d.coef, p.d.mono_t, 0, 0);
  }
  return cudaGetLastError();
}

cudaError_t launch_xcontract(const Plan& p, cudaStream_t s, int ldeg) {
  if (p.npairs == 0) return cudaSuccess;
  long long blocks = std::min<long long>((p.npairs + 7) / 8, 152LL * 64);
  ++p.launches;
  xcontract_kernel<<<(int)blocks, 256, 0, s>>>(p.npairs, p.d.hot_a, p.d.hot_b, p.d.tab_off, p.d.tab,
                                                p.d.coef_off, p.d.coef, p.d.xt_off, p.d.tabs, p.d.part,
                                                ldeg);
  ++p.launches;
  ycontract_kernel<<<(int)blocks, 256, 0, s>>>(p.npairs, p.d.hot_a, p.d.hot_b, p.d.tab_off, p.d.tab,
                                                p.d.xt_off, p.d.part, p.d.yt_off, p.d.part + p.yt_base,
                                                ldeg, p.xr, p.skew ? 1 : 0, p.d.err);
  return cudaGetLastError();
}

// Collocation over `nwork` work items of the views in `views` (one plan, or a batch of
// plans sharing the sub-box shapes); cfg gives the launch shape.
cudaError_t launch_collocate_views(const GridLaunch& cfg, const PlanView* views, const int4* work,
                                   long long nwork, const CoefTables* tabs, cudaStream_t s) {
  if (nwork == 0) return cudaSuccess;
  const int t0 = cfg.tile[0], t1 = cfg.tile[1], t2 = cfg.tile[2];
  if (cfg.skew) {
    if (!(t0 == kT0 && t1 == kT1 && t2 == kT2)) return cudaErrorInvalidValue;
#define GPW_COLLOC_SK(NWV, SKV)                                                            \
  if (cfg.nw == NWV && cfg.skew == SKV) {                                                  \
    collocate_kernel<kT0, kT1, kT2, NWV, SKV><<<(int)nwork, NWV * 32, cfg.smem, s>>>(      \
        views, work, tabs, cfg.lp, cfg.stg, cfg.ldeg);                                     \
    return cudaGetLastError();                                                             \
  }
    GPW_COLLOC_SK(8, 1) GPW_COLLOC_SK(6, 1) GPW_COLLOC_SK(4, 1)
    GPW_COLLOC_SK(8, 2) GPW_COLLOC_SK(6, 2) GPW_COLLOC_SK(4, 2)
#undef GPW_COLLOC_SK
    return cudaErrorInvalidValue;
  }
#define GPW_COLLOC_NW(a, b, c, NWV)                                                        \
  if (t0 == a && t1 == b && t2 == c && cfg.nw == NWV) {                                    \
    collocate_kernel<a, b, c, NWV><<<(int)nwork, NWV * 32, cfg.smem, s>>>(                 \
        views, work, tabs, cfg.lp, cfg.stg, cfg.ldeg);                                     \
    return cudaGetLastError();                                                             \
  }
#define GPW_LAUNCH_COLLOC(a, b, c) GPW_COLLOC_NW(a, b, c, 8) GPW_COLLOC_NW(a, b, c, 6) GPW_COLLOC_NW(a, b, c, 4)
  GPW_COLLOC_SHAPES(GPW_LAUNCH_COLLOC)
#undef GPW_LAUNCH_COLLOC
#undef GPW_COLLOC_NW
  return cudaErrorInvalidValue;
}

cudaError_t launch_integrate_views(const GridLaunch& cfg, int lext, const PlanView* views,
                                   const int4* work, long long nwork, const CoefTables* tabs,
                                   cudaStream_t s) {
  if (nwork == 0) return cudaSuccess;
  const int t0 = cfg.tile[0], t1 = cfg.tile[1], t2 = cfg.tile[2];
  if (cfg.skew) {
    if (!(t0 == kT0 && t1 == kT1 && t2 == kT2)) return cudaErrorInvalidValue;
    if (cfg.skew == 1)
      integrate_kernel<kT0, kT1, kT2, kNW, 1><<<(int)nwork, kNW * 32, cfg.smem, s>>>(
          views, work, tabs, lext, cfg.lp, cfg.stg);
    else
      integrate_kernel<kT0, kT1, kT2, kNW, 2><<<(int)nwork, kNW * 32, cfg.smem, s>>>(
          views, work, tabs, lext, cfg.lp, cfg.stg);
    return cudaGetLastError();
  }
  const int zw = cfg.zwin ? cfg.zwin : t2;
#define GPW_LAUNCH_INTEGW(a, b, c, w)                                                        \
  if (t0 == a && t1 == b && t2 == c && zw == w) {                                          \
    integrate_kernel<a, b, w, kNW, 0, c><<<(int)nwork, kNW * 32, cfg.smem, s>>>(           \
        views, work, tabs, lext, cfg.lp, cfg.stg);                                         \
    return cudaGetLastError();                                                             \
  }
#define GPW_LAUNCH_INTEG(a, b, c) GPW_LAUNCH_INTEGW(a, b, c, c)
  GPW_INTEG_SHAPES(GPW_LAUNCH_INTEG)
  GPW_INTEG_WSHAPES(GPW_LAUNCH_INTEGW)
#undef GPW_LAUNCH_INTEG
#undef GPW_LAUNCH_INTEGW
  return cudaErrorInvalidValue;
}

cudaError_t launch_collocate(const Plan& p, cudaStream_t s, int ldeg) {
  if (p.nwork == 0) return cudaSuccess;
  if (ldeg && !p.xr) return cudaErrorInvalidValue;
  ++p.launches;
  GridLaunch cfg;
  for (int d = 0; d < 3; ++d) cfg.tile[d] = p.tile[d];
  cfg.nw = ldeg ? p.nw_colloc_t : p.nw_colloc;
  cfg.lp = p.lmax + 1 + ldeg;
  cfg.stg = ldeg ? p.stg_colloc_t : p.stg_colloc;
  cfg.smem = ldeg ? p.smem_colloc_t : p.smem_colloc;
  cfg.ldeg = ldeg;
  cfg.skew = p.skew ? (p.skew_zc ? 1 : 2) : 0;
  return launch_collocate_views(cfg, p.d.view, p.d.work_c, p.nwork, p.d.tabs, s);
}

cudaError_t launch_integrate(const Plan& p, int lext, cudaStream_t s) {
  if (p.nwork_i == 0) return cudaSuccess;
  ++p.launches;
  GridLaunch cfg;
  for (int d = 0; d < 3; ++d) cfg.tile[d] = p.tile_i[d];
  cfg.zwin = p.zwin_i;
  cfg.nw = kNW;
  if (lext > 1 + p.xr) return cudaErrorInvalidValue;
  cfg.lp = p.lmax + lext + 1;
  cfg.stg = lext > 1 ? p.stg_integ3 : (lext ? p.stg_integ1 : p.stg_integ);
  cfg.smem = lext > 1 ? p.smem_integ3 : (lext ? p.smem_integ1 : p.smem_integ);
  cfg.skew = p.skew ? (p.skew_zc ? 1 : 2) : 0;
  return launch_integrate_views(cfg, lext, p.d.view, p.d.work_i, p.nwork_i, p.d.tabs, s);
}

// Launch shapes for a batch of plans with the same sub-boxes and largest degree lmax.
cudaError_t configure_batch(const int* tile_c, const int* tile_i, int zwin_i, int lmax, int nw_req,
                            GridLaunch* colloc,
                            GridLaunch* integ1, int skew) {
  int dev = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess)
    e = cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  if (e != cudaSuccess) return e;
  int found = 0;
  for (int d = 0; d < 3; ++d) {
    colloc->tile[d] = tile_c[d];
    integ1->tile[d] = tile_i[d];
  }
  integ1->zwin = zwin_i;
  colloc->lp = lmax + 1;
  integ1->lp = lmax + 2;
  integ1->nw = kNW;
#define GPW_TILE_BCONF(a, b, c)                                                             \
  if (tile_c[0] == a && tile_c[1] == b && tile_c[2] == c) {                                 \
    found |= 1;                                                                             \
    colloc->stg = even(CollocLayout<a, b, c>::stage(lmax + 1));                             \
    if (pick_colloc_warps<a, b, c>(colloc->stg, nw_req, &colloc->nw, &colloc->smem) == 0) \
      return cudaErrorInvalidValue;                                                         \
  }
#define GPW_TILE_BCONF_IW(a, b, c, w)                                                       \
  if (tile_i[0] == a && tile_i[1] == b && tile_i[2] == c && zwin_i == w) {                  \
    found |= 2;                                                                             \
    integ1->stg = even(IntegLayout<a, b, w>::stage(lmax + 2));                              \
    integ1->smem = integ_smem<a, b, w>(integ1->stg);                                        \
  }
#define GPW_TILE_BCONF_I(a, b, c) GPW_TILE_BCONF_IW(a, b, c, c)
  GPW_COLLOC_SHAPES(GPW_TILE_BCONF)
  GPW_INTEG_SHAPES(GPW_TILE_BCONF_I)
  GPW_INTEG_WSHAPES(GPW_TILE_BCONF_IW)
#undef GPW_TILE_BCONF
#undef GPW_TILE_BCONF_I
#undef GPW_TILE_BCONF_IW
  if (found != 3) return cudaErrorInvalidValue;
  colloc->skew = integ1->skew = skew;
  if (skew) {
    // non-orthogonal plans: the cross-factor variants and their larger staging
    if (!(tile_c[0] == kT0 && tile_c[1] == kT1 && tile_c[2] == kT2 && tile_i[0] == kT0 &&
          tile_i[1] == kT1 && tile_i[2] == kT2))
      return cudaErrorInvalidValue;
    colloc->stg = colloc_skew_stage<kT0, kT1, kT2>(skew == 1, lmax + 1);
    const auto pick = skew == 1 ? pick_colloc_warps<kT0, kT1, kT2, 1> : pick_colloc_warps<kT0, kT1, kT2, 2>;
    if (pick(colloc->stg, nw_req, &colloc->nw, &colloc->smem) == 0)
      return cudaErrorInvalidValue;
    integ1->stg = even(even(IntegLayout<kT0, kT1, kT2>::stage(lmax + 2)) +
                       integ_skew_extra<kT0, kT1, kT2>(skew == 1));
    integ1->smem = integ_smem<kT0, kT1, kT2>(integ1->stg);
  }
  return cudaSuccess;
}

PlanView make_view(const Plan& p) {
  PlanView v;
  for (int k = 0; k < GPW_MAX_LEVELS; ++k) {
    v.lc[k] = p.lev[k];
    v.li[k] = p.lev_i[k];
  }
  v.task_c = p.d.task_c;
  v.sub_off_c = p.d.sub_off_c;
  v.task_i = p.d.task_i;
  v.sub_off_i = p.d.sub_off_i;
  v.tab_off = p.d.tab_off;
  v.coef_off = p.d.coef_off;
  v.part_off = p.d.part_off;
  v.tab = p.d.tab;
  v.coef = p.d.coef;
  v.part = p.d.part;
  v.xt_off = p.d.xt_off;
  v.xt = p.d.part;
  v.yt_off = p.d.yt_off;
  v.yt = p.d.part + p.yt_base;
  v.grids = p.d.grids;
  v.err = p.d.err;
  v.chunk_i = p.chunk_i;
  v.xr = p.xr;
  // 1: general non-orthogonal cell; 2: the third row orthogonal to the first two
  // (hexagonal, monoclinic with unique axis c), only the R01 cross factor
  v.skew = p.skew ? (p.skew_zc ? 1 : 2) : 0;
  v.geo = p.d.geo;
  v.hot_a = p.d.hot_a;
  return v;
}

cudaError_t launch_reduce_parts(const Plan& p, int lext, cudaStream_t s) {
  if (p.npairs == 0) return cudaSuccess;
  long long blocks = std::min<long long>((p.npairs + kRedPW - 1) / kRedPW, 152LL * 128);
  ++p.launches;
  if (p.lmax + lext <= kLextMax)
    reduce_parts_kernel<4><<<(int)blocks, kRedPW * 32, 0, s>>>(
        p.npairs, make_klevels(p, true), p.tile_i[0], p.d.hot_a, p.d.hot_b, p.d.ids2, p.d.part_off,
        p.d.coef_off, p.d.tab_off, p.d.tab, p.d.part, p.d.tabs, p.d.coef, lext, p.xr);
  else
    reduce_parts_kernel<8><<<(int)blocks, kRedPW * 32, 0, s>>>(
        p.npairs, make_klevels(p, true), p.tile_i[0], p.d.hot_a, p.d.hot_b, p.d.ids2, p.d.part_off,
        p.d.coef_off, p.d.tab_off, p.d.tab, p.d.part, p.d.tabs, p.d.coef, lext, p.xr);
  if (p.skew) {
    ++p.launches;
    mono_transform_kernel<<<(int)((p.npairs + 127) / 128), 128, 0, s>>>(
        p.npairs, p.d.hot_a, p.d.hot_b, p.d.coef_off, p.d.coef, p.d.mono_t, lext, 1);
  }
  return cudaGetLastError();
}

cudaError_t launch_assemble_V(const Plan& p, int lext, double* V, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(V, 0, sizeof(double) * (size_t)p.nao * p.nao, s);
  if (e != cudaSuccess || p.ngroups == 0) return e;
  ++p.launches;
  assemble_V_kernel<<<(int)((p.ngroups + 7) / 8), 256, 0, s>>>(
      p.ngroups, p.d.groups, p.d.ids, p.d.ids2, p.d.geo, p.d.pref, p.d.coef_off, p.d.coef,
      p.d.tabs, p.nao, lext, V);
  return cudaGetLastError();
}

cudaError_t launch_grad(const Plan& p, const double* D, double* grad, cudaStream_t s) {
  if (p.npairs > 0) {
    ++p.launches;
    grad_pair_kernel<<<(int)((p.npairs + 127) / 128), 128, 0, s>>>(
        p.npairs, p.d.ids, p.d.ids2, p.d.geo, p.d.pref, p.d.coef_off, p.d.coef, D, p.nao,
        p.d.pgrad);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  ++p.launches;
  grad_atom_kernel<<<(p.natm + 7) / 8, 256, 0, s>>>(p.natm, p.d.atom_off, p.d.atom_list,
                                                    p.d.pgrad, grad);
  return cudaGetLastError();
}

cudaError_t launch_combine(const Plan& p, cudaStream_t s) {
  ++p.launches;
  const LevelInfo& f = p.lev[0];
  const dim3 grid((unsigned)((f.N[1] * (f.N[2] / 2 + 1) + 255) / 256), (unsigned)f.N[0]);
  combine_kernel<<<grid, 256, 0, s>>>(make_klevels(p, false), p.d.g2tab, p.d.spec, p.d.fspec);
  return cudaGetLastError();
}

cudaError_t launch_restrict(const Plan& p, int level, const cufftDoubleComplex* fa,
                            const cufftDoubleComplex* fb, cudaStream_t s) {
  ++p.launches;
  restrict_kernel<<<152 * 8, 256, 0, s>>>(make_klevels(p, false), p.d.g2tab, level, fa, fb, p.d.spec);
  return cudaGetLastError();
}

cudaError_t launch_poisson(const Plan& p, cudaStream_t s) {
  ++p.launches;
  poisson_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(make_klevels(p, false), p.d.g2tab, p.omega,
                                                    p.d.fspec, p.d.red);
  return cudaGetLastError();
}

cudaError_t launch_lda(const Plan& p, const double* rho, const double* vH, double* v_out,
                       cudaStream_t s) {
  ++p.launches;
  lda_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(p.fine_n, p.omega / (double)p.fine_n, rho, vH, v_out,
                                                p.d.red + kRedBlocks);
  return cudaGetLastError();
}

cudaError_t launch_pair_coef_tau(const Plan& p, const double* D, cudaStream_t s) {
  if (p.npairs == 0) return cudaSuccess;
  if (!p.xr) return cudaErrorInvalidValue;
  ++p.launches;
  pair_coef_tau_kernel<<<(int)((p.npairs + 127) / 128), 128, 0, s>>>(
      p.npairs, p.d.ids, p.d.ids2, p.d.geo, p.d.pref, p.d.coef_off, D, p.nao, p.d.coef);
  if (p.skew) {
    ++p.launches;
    mono_transform_kernel<<<(int)((p.npairs + 127) / 128), 128, 0, s>>>(
        p.npairs, p.d.hot_a, p.d.hot_b, p.d.coef_off, p.d.coef, p.d.mono_t, 2, 0);
  }
  return cudaGetLastError();
}

cudaError_t launch_assemble_V_tau(const Plan& p, int lext, double* V, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(V, 0, sizeof(double) * (size_t)p.nao * p.nao, s);
  if (e != cudaSuccess || p.ngroups == 0) return e;
  ++p.launches;
  assemble_V_tau_kernel<<<(int)((p.ngroups + 7) / 8), 256, 0, s>>>(
      p.ngroups, p.d.groups, p.d.ids, p.d.ids2, p.d.geo, p.d.pref, p.d.coef_off, p.d.coef,
      p.d.tabs, p.nao, lext, V);
  return cudaGetLastError();
}

cudaError_t launch_grad_tau(const Plan& p, const double* D, double* grad, cudaStream_t s) {
  if (p.npairs > 0) {
    ++p.launches;
    grad_tau_pair_kernel<<<(int)((p.npairs + 127) / 128), 128, 0, s>>>(
        p.npairs, p.d.ids, p.d.ids2, p.d.geo, p.d.pref, p.d.coef_off, p.d.coef, p.d.tabs, D,
        p.nao, p.d.pgrad);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  ++p.launches;
  grad_atom_kernel<<<(p.natm + 7) / 8, 256, 0, s>>>(p.natm, p.d.atom_off, p.d.atom_list,
                                                    p.d.pgrad, grad);
  return cudaGetLastError();
}

cudaError_t launch_fourier_deriv(const Plan& p, int axis, const cufftDoubleComplex* in,
                                 cufftDoubleComplex* out, bool subtract, cudaStream_t s) {
  ++p.launches;
  fourier_deriv_kernel<<<152 * 8, 256, 0, s>>>(make_klevels(p, false), p.d.g1tab, axis, in, out,
                                               subtract ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_pbe_x(const Plan& p, const double* rho, double* grad3, double* v_rho,
                         cudaStream_t s) {
  ++p.launches;
  const long long n = p.fine_n;
  pbe_x_kernel<<<kRedBlocks, kRedThreads, 0, s>>>(n, p.omega / (double)n, rho, grad3,
                                                  grad3 + n, grad3 + 2 * n, v_rho,
                                                  p.d.red + kRedBlocks);
  return cudaGetLastError();
}

cudaError_t launch_spec_combine(const Plan& p, const cufftDoubleComplex* fa,
                                const cufftDoubleComplex* fb, cufftDoubleComplex* out,
                                cudaStream_t s) {
  ++p.launches;
  spec_combine_kernel<<<152 * 8, 256, 0, s>>>(p.fine_spec_n, 1.0 / (double)p.fine_n, fa, fb, out);
  return cudaGetLastError();
}

cudaError_t launch_energy_final(const Plan& p, int slot, int nparts, cudaStream_t s) {
  ++p.launches;
  energy_final_kernel<<<1, kRedThreads, 0, s>>>(p.d.red + slot * kRedBlocks, nparts,
                                                p.d.energies + slot);
  return cudaGetLastError();
}

}  // namespace gpw
