// Host part of gpw_plan: primitive normalisation, shell cutoff radii (Eq. cut), pair
// screening over lattice images (Sec. III A), multigrid level assignment (Sec. II),
// integer pair boxes and the per-level sub-box task lists that the collocation and
// integration kernels walk.  Compiled with -ffp-contract=off: every screening decision
// is an exact function of the inputs.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include <mutex>

#include <omp.h>

#include "gpw_internal.h"
#include "plan_host.h"

namespace gpw {

namespace {

double ipow(double x, int n) {
  double p = 1.0;
  for (int k = 0; k < n; ++k) p *= x;
  return p;
}

double dfact(int n) {
  double r = 1.0;
  while (n > 1) {
    r *= n;
    n -= 2;
  }
  return r;
}

// N_l(alpha): unit self-overlap of the x^l component of a primitive Cartesian Gaussian.
double prim_norm(int l, double alpha) {
  double ip = 1.0;
  for (int k = 0; k < l; ++k) ip *= 4.0 * alpha;
  return std::sqrt(std::pow(2.0 * alpha / M_PI, 1.5) * ip / dfact(2 * l - 1));
}

// Eq. (cut) for one primitive: f(r) = |c N| r^(l+2) exp(-alpha r^2); r_cut is the largest
// root of f = tau on the decreasing branch (64 bisection steps); -1 drops the primitive.
double prim_f(double cn, int l, double alpha, double r) {
  return cn * ipow(r, l + 2) * std::exp(-alpha * r * r);
}

double prim_rcut(double cn, int l, double alpha, double tau) {
  double r0 = std::sqrt((double)(l + 2) / (2.0 * alpha));
  if (prim_f(cn, l, alpha, r0) < tau) return -1.0;
  double hi = r0;
  for (int it = 0; it < 200 && prim_f(cn, l, alpha, hi) >= tau; ++it) hi *= 2.0;
  double lo = r0;
  for (int it = 0; it < 64; ++it) {
    double mid = 0.5 * (lo + hi);
    if (prim_f(cn, l, alpha, mid) >= tau) lo = mid; else hi = mid;
  }
  return hi;
}

// Eq. (cut) for the product Gaussian of Eq. (gab): magnitude bound at distance r from P,
// h(r) = |c_a N_a c_b N_b| K_ab (r + |P-A|)^la (r + |P-B|)^lb r^2 exp(-alpha_p r^2).
double pair_h(double cab, double kab, int la, int lb, double dA, double dB, double ap,
              double r) {
  return cab * kab * ipow(r + dA, la) * ipow(r + dB, lb) * r * r * std::exp(-ap * r * r);
}

// Integer box of a pair (reading of Eq. cut): R = the 64-step bisection root of h = tau,
// lo_d = ceil((P_d - R) N_d / L_d), hi_d = floor((P_d + R) N_d / L_d).  Both are monotone
// in R (correctly rounded operations, no contraction) and the final root lies inside every
// bracket of the bisection, so the bisection stops as soon as both ends of its bracket
// give the same box: the box is then that of the full 64 steps.  False drops the pair.
void box_at(double R, const double* P, const double* N, const double* L, int* lo, int* hi) {
  for (int d = 0; d < 3; ++d) {
    lo[d] = (int)std::ceil((P[d] - R) * N[d] / L[d]);
    hi[d] = (int)std::floor((P[d] + R) * N[d] / L[d]);
  }
}

// The box of a non-orthogonal cell (App., non-orthogonal lattices): the grid points whose
// fractional coordinate along R_d lies within R |b_d| of that of P,
//   lo_d = ceil((f_d(P) - R |b_d|) N_d),  hi_d = floor((f_d(P) + R |b_d|) N_d),
// f_d(P) = b_d . P summed over x, y, z in that order; monotone in R like box_at.
struct SkewBox {
  const double* rec;   // reciprocal rows b_d
  double blen[3];      // |b_d|
};

void box_at_skew(double R, const double* P, const double* N, const SkewBox& sk, int* lo, int* hi) {
  for (int d = 0; d < 3; ++d) {
    double f = 0.0;
    for (int c = 0; c < 3; ++c) f += sk.rec[3 * d + c] * P[c];
    lo[d] = (int)std::ceil((f - R * sk.blen[d]) * N[d]);
    hi[d] = (int)std::floor((f + R * sk.blen[d]) * N[d]);
  }
}

// d log h / dr: strictly decreasing in r, so h has one maximum, at r* <= r0.
double pair_dlogh(int la, int lb, double dA, double dB, double ap, double r) {
  return (double)la / (r + dA) + (double)lb / (r + dB) + 2.0 / r - 2.0 * ap * r;
}

// R_p = the largest root of h = tau.  With r0 = sqrt((la+lb+2)/(2 ap)): if h(r0) >= tau the
// root lies beyond r0 (bracketed by doubling); otherwise the maximum r* of h in (0, r0] is
// found by 64 bisection steps on the sign of d log h / dr, h(r*) < tau drops the pair, and
// the root is bisected on [r*, r0].  Either way h decreases on the bracket of the final
// bisection, whose upper end is R_p.
bool pair_box(double cab, double kab, int la, int lb, double dA, double dB, double ap,
              double tau, const double* P, const double* N, const double* L, int* lo_out,
              int* hi_out, const SkewBox* sk = nullptr, double* R_out = nullptr) {
  auto box = [&](double R, int* lo, int* hi) {
    if (sk)
      box_at_skew(R, P, N, *sk, lo, hi);
    else
      box_at(R, P, N, L, lo, hi);
  };
  double r0 = std::sqrt((double)(la + lb + 2) / (2.0 * ap));
  double lo, hi;
  if (pair_h(cab, kab, la, lb, dA, dB, ap, r0) >= tau) {
    hi = r0;
    for (int it = 0; it < 200 && pair_h(cab, kab, la, lb, dA, dB, ap, hi) >= tau; ++it) hi *= 2.0;
    lo = r0;
  } else {
    // Most pairs that reach here peak far below tau: a closed-form upper bound of h
    // rejects them before the bisection.  With D = max(dA, dB) and L = la + lb,
    // (r+dA)^la (r+dB)^lb <= (r+D)^L <= 2^(L-1) (r^L + D^L) (L >= 1), and
    // max r^k exp(-ap r^2) = (k / (2 e ap))^(k/2), so
    //   h <= C 2^(L-1) [((L+2) / (2 e ap))^((L+2)/2) + D^L / (e ap)]   (C / (e ap) for L = 0).
    // The margin keeps the decision that of the bisection despite rounding.
    const int L = la + lb;
    const double D = dA > dB ? dA : dB;
    const double eap = M_E * ap;
    double bound;
    if (L == 0) {
      bound = cab * kab / eap;
    } else {
      const double k = (double)(L + 2);
      bound = cab * kab * ipow(2.0, L - 1) *
              (std::pow(k / (2.0 * eap), 0.5 * k) + ipow(D, L) / eap);
    }
    if (bound < tau * (1.0 - 1e-12)) return false;
    double a = 0.0, b = r0;
    for (int it = 0; it < 64; ++it) {
      double mid = 0.5 * (a + b);
      if (pair_dlogh(la, lb, dA, dB, ap, mid) > 0.0) a = mid; else b = mid;
    }
    double rs = a > 0.0 ? a : b;
    if (pair_h(cab, kab, la, lb, dA, dB, ap, rs) < tau) return false;
    lo = rs;
    hi = r0;
  }
  for (int it = 0; it < 64; ++it) {
    double mid = 0.5 * (lo + hi);
    if (pair_h(cab, kab, la, lb, dA, dB, ap, mid) >= tau) lo = mid; else hi = mid;
    if (it >= 7 && (it & 3) == 3) {
      int a[3], b[3], c[3], e[3];
      box(lo, a, b);
      box(hi, c, e);
      bool same = true;
      for (int d = 0; d < 3; ++d) same = same && a[d] == c[d] && b[d] == e[d];
      if (same) break;
    }
  }
  box(hi, lo_out, hi_out);
  if (R_out) *R_out = hi;  // an upper bound of the root (the bisection may stop early)
  return true;
}

// A lower bound of the smallest eigenvalue of the lattice metric M_de = R_d . R_e (the
// closed form for a symmetric 3 x 3 matrix, then 1e-9 relative taken off for rounding):
// |sum_d f_d R_d|^2 >= lam |f|^2 for every fractional displacement f.
double metric_lambda_min(const double* lat) {
  double M[3][3];
  for (int d = 0; d < 3; ++d)
    for (int e = 0; e < 3; ++e)
      M[d][e] = lat[3 * d] * lat[3 * e] + lat[3 * d + 1] * lat[3 * e + 1] + lat[3 * d + 2] * lat[3 * e + 2];
  const double tr = (M[0][0] + M[1][1] + M[2][2]) / 3.0;
  const double p1 = M[0][1] * M[0][1] + M[0][2] * M[0][2] + M[1][2] * M[1][2];
  const double p2 = (M[0][0] - tr) * (M[0][0] - tr) + (M[1][1] - tr) * (M[1][1] - tr) +
                    (M[2][2] - tr) * (M[2][2] - tr) + 2.0 * p1;
  const double p = std::sqrt(p2 / 6.0);
  if (!(p > 0.0)) return tr * (1.0 - 1e-9);
  double B[3][3];
  for (int d = 0; d < 3; ++d)
    for (int e = 0; e < 3; ++e) B[d][e] = (M[d][e] - (d == e ? tr : 0.0)) / p;
  const double det = B[0][0] * (B[1][1] * B[2][2] - B[1][2] * B[2][1]) -
                     B[0][1] * (B[1][0] * B[2][2] - B[1][2] * B[2][0]) +
                     B[0][2] * (B[1][0] * B[2][1] - B[1][1] * B[2][0]);
  const double r = std::max(-1.0, std::min(1.0, det / 2.0));
  const double phi = std::acos(r) / 3.0;
  const double lmin = tr + 2.0 * p * std::cos(phi + 2.0 * M_PI / 3.0);
  return std::max(0.0, lmin) * (1.0 - 1e-9);
}

bool smooth7(int m) {
  for (int f : {2, 3, 5, 7})
    while (m % f == 0) m /= f;
  return m == 1;
}

int smooth7_even_at_least(int n) {
  int m = std::max(2, n);
  while (!(m % 2 == 0 && smooth7(m))) ++m;
  return m;
}

long long floordiv(long long a, long long b) {
  long long q = a / b;
  if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
  return q;
}

struct Prim {
  int atom, l, shell;
  long long ao;
  double alpha, cn, rcut;
};

struct PairTmp {
  int a, b, sa, sb;
  int img[3];
  int level;
  int lo[3], hi[3];
  PairQ q;  // GPW_FAST_BLOCK_PRUNE: fractional coordinates of P and R_p
};

struct Seg {
  int k, j;
};

// most sub-box segments of one pair box along one axis
constexpr size_t kSegMax = 512;

// Segments of [lo, hi] along an axis of N points cut into sub-boxes of T (the last one of
// each period clipped), whose thread blocks see windows of W >= T points from their
// sub-box start (W = T: plain tiling).  A segment starts at lo or where the previous one
// ended; it belongs to the sub-box j it starts in and ends where that sub-box's window
// (clipped at the period) ends.  With W = T the cells of the unwrapped axis are numbered
// g = period * nsb + sub-box, and [lo, hi] meets every cell from g(lo) to g(hi).
long long nseg(int lo, int hi, int N, int T, int W) {
  const long long nsb = (N + T - 1) / T;
  if (W == T) {
    auto g = [&](long long i) {
      const long long q = floordiv(i, N);
      return q * nsb + (i - q * N) / T;
    };
    return g(hi) - g(lo) + 1;
  }
  long long n = 0;
  for (long long i = lo; i <= hi; ++n) {
    const long long k = floordiv(i, N), j = (i - k * N) / T;
    i = k * N + std::min<long long>(j * T + W, N);
  }
  return n;
}

void segments(int lo, int hi, int N, int T, int W, std::vector<Seg>* out) {
  out->clear();
  long long i = lo;
  while (i <= hi) {
    long long k = floordiv(i, N);
    long long ip = i - k * N;
    long long j = ip / T;
    long long end = k * N + std::min<long long>(j * T + W, N) - 1;
    out->push_back({(int)k, (int)j});
    i = std::min<long long>(hi, end) + 1;
  }
}

struct PairBox {
  int level, lo[3], hi[3];
  PairQ q;  // GPW_FAST_BLOCK_PRUNE: fractional coordinates of P and R_p
};

// Spare task-record buffers of committed plans, kept with their pages so that the next
// plan (a server plans one small cell after another) neither faults them in nor zeroes
// fresh memory.  At most kTaskPoolBytes in total.
std::mutex g_task_pool_mu;
std::vector<std::vector<int4>> g_task_pool;
constexpr size_t kTaskPoolBytes = size_t(1) << 30;

std::vector<int4> take_task_buffer(size_t n) {
  std::lock_guard<std::mutex> lk(g_task_pool_mu);
  int best = -1;
  for (int i = 0; i < (int)g_task_pool.size(); ++i)
    if (g_task_pool[i].capacity() >= n &&
        (best < 0 || g_task_pool[i].capacity() < g_task_pool[best].capacity()))
      best = i;
  if (best < 0) return {};
  std::vector<int4> v = std::move(g_task_pool[best]);
  g_task_pool.erase(g_task_pool.begin() + best);
  v.clear();
  return v;
}

// Host threads for a loop over n items: all cores for large plans, one for small ones
// (a server plans several small cells at once on its own threads).
// gpw_desc.host_threads of the plan being built on this thread (0: no cap)
thread_local int g_host_threads = 0;

int plan_threads(long long n) {
  if (n < 20000) return 1;
  int cap = omp_get_max_threads();
  if (g_host_threads > 0) cap = std::min(cap, g_host_threads);
  return std::max(1, std::min<int>(cap, (int)(n / 20000)));
}

std::vector<PairBox> pairs_view(const std::vector<PairTmp>& pairs) {
  std::vector<PairBox> v(pairs.size());
  const int nthr = plan_threads((long long)pairs.size());
#pragma omp parallel for num_threads(nthr) schedule(static)
  for (long long i = 0; i < (long long)pairs.size(); ++i) {
    v[i].level = pairs[i].level;
    v[i].q = pairs[i].q;
    for (int d = 0; d < 3; ++d) {
      v[i].lo[d] = pairs[i].lo[d];
      v[i].hi[d] = pairs[i].hi[d];
    }
  }
  return v;
}

// Task lists for one sub-box shape T: per level, sub-boxes of T (the last ones clipped
// at the mesh edge), and for every pair each (sub-box, periodic copy) its box meets;
// along z the segments follow the windows of zwin points (zwin = T[2]: plain tiling).
// Fills lev[k].sub_base, the CSR offsets, the 2-int4 task records (sorted by pair
// inside every sub-box), the work list (heaviest sub-box first) and, if ranks is
// non-NULL (the integration tasks), the number of tasks of every pair, the size of its
// block of per-task W tensors (psize) and each task's offset in that block (record
// r1.w).  A pair's tasks are ranked x-segment first; the W tensor of a task (nc2(L+1)
// rows of m0) sits at nc2(L+1) (t0 ns12 + r12 m0), with ns12 the number of (y, z)
// segments and r12 the task's index among them, so the tasks of one x-segment are
// contiguous and every x-segment block starts at nc2(L+1) t0 ns12.
int build_tasks(Plan* plan, const std::vector<PairBox>& pairs, const std::vector<int4>& hot_a,
                const int* T, int zwin, LevelInfo* lev, std::vector<long long>* sub_off,
                std::vector<int4>* task, std::vector<int4>* work, long long* nent_out,
                long long* nwork_out, long long* nsub_out, std::vector<int>* ranks,
                std::vector<long long>* psize, long long* chunk_io, bool prune = false) {
  // GPW_FAST_BLOCK_PRUNE (collocation lists only): tasks whose box lies wholly beyond R_p
  // are left out; the others keep their rank among all of the pair's tasks
  auto beyond = [&](const PairBox& t, const LevelInfo& lv, const long long* a, const long long* b) {
    if (!prune) return false;
    const int ai[3] = {(int)a[0], (int)a[1], (int)a[2]}, bi[3] = {(int)b[0], (int)b[1], (int)b[2]};
    return block_beyond(t.q, ai, bi, lv.N, plan->prune_blen, !plan->skew, plan->prune_lam);
  };
  // unwrapped grid range [a, b] of segment s of [lo, hi] along an axis of N points
  const int Wd[3] = {T[0], T[1], zwin};
  auto seg_range = [](int lo, int hi, int N, int Td, int Wn, const Seg& s, long long* a,
                      long long* b) {
    const long long s0 = (long long)s.j * Td;
    const long long ext = std::min<long long>(Wn, N - s0);
    const long long o = (long long)s.k * N + s0;
    *a = std::max<long long>(lo, o);
    *b = std::min<long long>(hi, o + ext - 1);
  };
  const int K = plan->nlev;
  const long long np = (long long)pairs.size();
  long long nsub = 0;
  for (int k = 0; k < K; ++k) {
    lev[k].sub_base = nsub;
    nsub += (long long)lev[k].nsb[0] * lev[k].nsb[1] * lev[k].nsb[2];
  }
  *nsub_out = nsub;
  // Threads take contiguous ranges of pairs; every thread counts its tasks per sub-box,
  // the counts give each thread its first slot in every sub-box (threads in pair order),
  // so the task order inside a sub-box is the pair order whatever the thread count.
  const int nthr = plan_threads(np);
  std::vector<std::vector<long long>> tslot(nthr);
#pragma omp parallel num_threads(nthr)
  {
    const int th = omp_get_thread_num();
    const long long p0 = np * th / nthr, p1 = np * (th + 1) / nthr;
    std::vector<long long>& c = tslot[th];
    c.assign(nsub, 0);
    std::vector<Seg> sg[3];
    for (long long p = p0; p < p1; ++p) {
      const PairBox& t = pairs[p];
      const LevelInfo& lv = lev[t.level];
      for (int d = 0; d < 3; ++d) segments(t.lo[d], t.hi[d], lv.N[d], T[d], Wd[d], &sg[d]);
      long long a[3], b[3];
      for (auto& s0 : sg[0]) {
        seg_range(t.lo[0], t.hi[0], lv.N[0], T[0], Wd[0], s0, &a[0], &b[0]);
        for (auto& s1 : sg[1]) {
          seg_range(t.lo[1], t.hi[1], lv.N[1], T[1], Wd[1], s1, &a[1], &b[1]);
          for (auto& s2 : sg[2]) {
            seg_range(t.lo[2], t.hi[2], lv.N[2], T[2], Wd[2], s2, &a[2], &b[2]);
            if (beyond(t, lv, a, b)) continue;
            c[lv.sub_base + ((long long)s0.j * lv.nsb[1] + s1.j) * lv.nsb[2] + s2.j]++;
          }
        }
      }
    }
  }
  std::vector<long long> count(nsub + 1, 0);
  for (long long i = 0; i < nsub; ++i) {
    long long run = count[i];
    for (int th = 0; th < nthr; ++th) {
      const long long c = tslot[th][i];
      tslot[th][i] = run;
      run += c;
    }
    count[i + 1] = run;
  }
  const long long nent = count[nsub];
  *nent_out = nent;
  *task = take_task_buffer((size_t)(2 * nent));
  task->resize((size_t)(2 * nent));
  if (ranks) ranks->assign(np, 0);
  if (psize) psize->assign(np, 0);
  int fail = GPW_OK;
#pragma omp parallel num_threads(nthr)
  {
    const int th = omp_get_thread_num();
    const long long p0 = np * th / nthr, p1 = np * (th + 1) / nthr;
    std::vector<long long>& fill = tslot[th];
    std::vector<Seg> sg[3];
    for (long long p = p0; p < p1; ++p) {
      const PairBox& t = pairs[p];
      const LevelInfo& lv = lev[t.level];
      for (int d = 0; d < 3; ++d) segments(t.lo[d], t.hi[d], lv.N[d], T[d], Wd[d], &sg[d]);
      const int L = hot_a[p].w;
      int n[3];
      bool bad = false;
      for (int d = 0; d < 3; ++d) {
        n[d] = t.hi[d] - t.lo[d] + 1;
        bad = bad || n[d] > 65535;
      }
      const long long ns12 = (long long)sg[1].size() * sg[2].size();
      const long long S = nc2(L + 1 + plan->xr);
      if (psize) {
        (*psize)[p] = S * n[0] * ns12;
        bad = bad || (*psize)[p] > INT32_MAX;
      }
      if (bad) {
#pragma omp critical(gpw_plan_fail)
        fail = GPW_ERANGE;
        continue;
      }
      // per dimension and segment: packed (m, u, t) fields of the records and the
      // sub-box coordinate, computed once per pair
      int fm[3][kSegMax], fu[3][kSegMax], ft[3][kSegMax];
      long long fj[3][kSegMax], fa[3][kSegMax], fb[3][kSegMax];
      bool big = false;
      for (int d = 0; d < 3; ++d) {
        big = big || sg[d].size() > kSegMax;
        if (big) break;
        for (size_t k = 0; k < sg[d].size(); ++k) {
          const Seg& sgm = sg[d][k];
          const long long s0 = (long long)sgm.j * T[d];
          const long long ext = std::min<long long>(Wd[d], lv.N[d] - s0);
          const long long o = (long long)sgm.k * lv.N[d] + s0;
          const long long a = std::max<long long>(t.lo[d], o);
          const long long b = std::min<long long>(t.hi[d], o + ext - 1);
          const int shift = 8 * d;
          fm[d][k] = (int)(b - a + 1) << shift;
          fu[d][k] = (int)(a - o) << shift;
          ft[d][k] = (int)(a - t.lo[d]) | (n[d] << 16);
          fj[d][k] = sgm.j;
          fa[d][k] = a;
          fb[d][k] = b;
        }
      }
      if (big) {
#pragma omp critical(gpw_plan_fail)
        fail = GPW_ERANGE;
        continue;
      }
      const int ns0 = (int)sg[0].size(), ns1 = (int)sg[1].size(), ns2 = (int)sg[2].size();
      int rank = 0;
      for (int k0 = 0; k0 < ns0; ++k0) {
        const int m0 = fm[0][k0] & 255, tt0 = ft[0][k0] & 0xffff;
        for (int k1 = 0; k1 < ns1; ++k1) {
          const long long sub01 = lv.sub_base + (fj[0][k0] * lv.nsb[1] + fj[1][k1]) * lv.nsb[2];
          for (int k2 = 0; k2 < ns2; ++k2, ++rank) {
            if (prune) {
              const long long a[3] = {fa[0][k0], fa[1][k1], fa[2][k2]};
              const long long b[3] = {fb[0][k0], fb[1][k1], fb[2][k2]};
              if (beyond(t, lv, a, b)) continue;
            }
            const long long slot = fill[sub01 + fj[2][k2]]++;
            const int r12 = k1 * ns2 + k2;
            (*task)[2 * slot] = make_int4((int)p, fm[0][k0] | fm[1][k1] | fm[2][k2] | (L << 24),
                                          fu[0][k0] | fu[1][k1] | fu[2][k2], rank);
            (*task)[2 * slot + 1] =
                make_int4(ft[0][k0], ft[1][k1], ft[2][k2],
                          psize ? (int)(S * ((long long)tt0 * ns12 + (long long)r12 * m0)) : 0);
          }
        }
      }
      if (ranks) (*ranks)[p] = rank;
    }
  }
  if (fail != GPW_OK) {
    set_error("gpw_plan: pair box longer than 65535 grid points, more than 512 sub-box "
              "segments along one axis, or per-pair task block too large");
    return fail;
  }
  *sub_off = count;
  long long chunk = 0;
  if (chunk_io) {
    chunk = *chunk_io >= 0 ? *chunk_io : default_chunk(nent);
    *chunk_io = chunk;
  }
  return order_work(K, lev, count, chunk, work, nwork_out);
}

// The task counts of build_tasks without the records, which the device builds at commit
// (tasks.cu): sets lev[k].sub_base and *nsub_out, the exclusive prefix sums toff (np + 1)
// of the pairs' task counts in pair order and *nent_out, and, for the integration shape,
// each pair's task count (ranks) and W block size (psize).  Same limits as build_tasks.
int count_tasks(Plan* plan, const std::vector<PairBox>& pairs, const std::vector<int4>& hot_a,
                const int* T, int zwin, LevelInfo* lev, long long* nsub_out, std::vector<long long>* toff,
                long long* nent_out, std::vector<int>* ranks, std::vector<long long>* psize) {
  const int K = plan->nlev;
  const long long np = (long long)pairs.size();
  long long nsub = 0;
  for (int k = 0; k < K; ++k) {
    lev[k].sub_base = nsub;
    nsub += (long long)lev[k].nsb[0] * lev[k].nsb[1] * lev[k].nsb[2];
  }
  *nsub_out = nsub;
  toff->assign(np + 1, 0);
  if (ranks) ranks->assign(np, 0);
  if (psize) psize->assign(np, 0);
  bool bad = false;
  const int nthr = plan_threads(np);
#pragma omp parallel for num_threads(nthr) schedule(static) reduction(|| : bad)
  for (long long p = 0; p < np; ++p) {
    const PairBox& t = pairs[p];
    const LevelInfo& lv = lev[t.level];
    long long ns[3];
    int n[3];
    for (int d = 0; d < 3; ++d) {
      n[d] = t.hi[d] - t.lo[d] + 1;
      ns[d] = nseg(t.lo[d], t.hi[d], lv.N[d], T[d], d == 2 ? zwin : T[d]);
      bad = bad || n[d] > 65535 || ns[d] > (long long)kSegMax;
    }
    const long long c = ns[0] * ns[1] * ns[2];
    if (psize) {
      (*psize)[p] = nc2(hot_a[p].w + 1 + plan->xr) * n[0] * ns[1] * ns[2];
      bad = bad || (*psize)[p] > INT32_MAX;
    }
    if (ranks) (*ranks)[p] = (int)c;
    (*toff)[p + 1] = c;
  }
  for (long long p = 0; p < np; ++p) (*toff)[p + 1] += (*toff)[p];
  if (bad) {
    set_error("gpw_plan: pair box longer than 65535 grid points, more than 512 sub-box "
              "segments along one axis, or per-pair task block too large");
    return GPW_ERANGE;
  }
  *nent_out = (*toff)[np];
  return GPW_OK;
}

}  // namespace

// Monomial transforms of a non-orthogonal cell, per level (layout: gpw_internal.h): the
// Cartesian monomial prod_c (r - A)_c^(k_c) with (r - A)_c = sum_d M_cd xi_d,
// M_cd = (R_d)_c / N_d, expanded by multiplying out the linear forms one at a time.
void build_mono_transforms(const Plan& P, std::vector<double>* out) {
  out->assign((size_t)kMonoStride * P.nlev, 0.0);
  constexpr int D = kSkewDeg + 1;
  for (int k = 0; k < P.nlev; ++k) {
    double M[3][3];
    for (int c = 0; c < 3; ++c)
      for (int d = 0; d < 3; ++d) M[c][d] = P.lat[3 * d + c] / P.lev[k].N[d];
    double* blk = out->data() + (size_t)kMonoStride * k;
    for (int n = 0; n <= kSkewDeg; ++n)
      for (int c2 = 0; c2 <= n; ++c2)
        for (int c1 = 0; c1 <= n - c2; ++c1) {
          const int kc[3] = {n - c1 - c2, c1, c2};
          // poly[x0][x1][x2]: coefficient of xi0^x0 xi1^x1 xi2^x2
          std::vector<double> poly(D * D * D, 0.0), nxt(D * D * D);
          poly[0] = 1.0;
          int deg = 0;
          for (int c = 0; c < 3; ++c)
            for (int r = 0; r < kc[c]; ++r) {
              std::fill(nxt.begin(), nxt.end(), 0.0);
              for (int x2 = 0; x2 <= deg; ++x2)
                for (int x1 = 0; x1 <= deg - x2; ++x1) {
                  const int x0 = deg - x1 - x2;
                  const double v = poly[(x0 * D + x1) * D + x2];
                  if (v == 0.0) continue;
                  nxt[((x0 + 1) * D + x1) * D + x2] += v * M[c][0];
                  nxt[(x0 * D + x1 + 1) * D + x2] += v * M[c][1];
                  nxt[(x0 * D + x1) * D + x2 + 1] += v * M[c][2];
                }
              poly.swap(nxt);
              ++deg;
            }
          double* row = blk + mono_off(n) + (size_t)hidx(n, c1, c2) * nh(n);
          for (int x2 = 0; x2 <= n; ++x2)
            for (int x1 = 0; x1 <= n - x2; ++x1) row[hidx(n, x1, x2)] = poly[((n - x1 - x2) * D + x1) * D + x2];
        }
  }
}

long long default_chunk(long long nent) {
  return std::min<long long>(INT32_MAX, std::max(kChunkMin, (nent + kChunkDiv - 1) / kChunkDiv));
}

// Work list of one task-list shape from its sub-box CSR offsets `count` (nsub + 1):
// items {plan slot, level | chunk << 4, sub-box, tasks}; with chunk > 0 a sub-box with
// more tasks is cut into items of `chunk` consecutive tasks (integration only: its tasks
// write separate slots).
int order_work(int K, const LevelInfo* lev, const std::vector<long long>& count, long long chunk,
               std::vector<int4>* work, long long* nwork_out) {
  const long long nsub = (long long)count.size() - 1;
  // Order: items in Morton order of their sub-box (per level) are cut into bands of
  // kBand items; each band runs heaviest first and bands run by decreasing mean weight.
  // Blocks resident at the same time then work on nearby sub-boxes, whose pairs' factor
  // tables are shared in L2, while the light items still come last.
  struct W {
    long long c, sidx, j;
    unsigned long long key;
  };
  auto spread = [](unsigned long long x) {
    unsigned long long r = 0;
    for (int b = 0; b < 20; ++b) r |= ((x >> b) & 1ULL) << (3 * b);
    return r;
  };
  std::vector<W> w;
  for (long long sidx = 0; sidx < nsub; ++sidx) {
    const long long c = count[sidx + 1] - count[sidx];
    if (c <= 0) continue;
    int k = 0;
    while (k + 1 < K && lev[k + 1].sub_base <= sidx) ++k;
    const long long loc = sidx - lev[k].sub_base;
    const long long j2 = loc % lev[k].nsb[2], j1 = (loc / lev[k].nsb[2]) % lev[k].nsb[1];
    const long long j0 = loc / ((long long)lev[k].nsb[2] * lev[k].nsb[1]);
    const unsigned long long key =
        ((unsigned long long)k << 60) | (spread(j0) << 2) | (spread(j1) << 1) | spread(j2);
    if (chunk <= 0 || c <= chunk) {
      w.push_back({c, sidx, 0, key});
    } else {
      for (long long j = 0; j * chunk < c; ++j)
        w.push_back({std::min(chunk, c - j * chunk), sidx, j, key});
    }
  }
  std::stable_sort(w.begin(), w.end(), [](const W& a, const W& b) { return a.key < b.key; });
  std::vector<std::pair<double, size_t>> bands;  // (-mean weight, first item)
  for (size_t b = 0; b < w.size(); b += kBand) {
    const size_t e = std::min(w.size(), b + (size_t)kBand);
    std::stable_sort(w.begin() + b, w.begin() + e, [](const W& x, const W& y) { return x.c > y.c; });
    double sum = 0;
    for (size_t i = b; i < e; ++i) sum += (double)w[i].c;
    bands.push_back({-sum / (double)(e - b), b});
  }
  std::stable_sort(bands.begin(), bands.end(),
                   [](const std::pair<double, size_t>& x, const std::pair<double, size_t>& y) {
                     return x.first < y.first;
                   });
  std::vector<W> ordered;
  ordered.reserve(w.size());
  for (const auto& bd : bands)
    for (size_t i = bd.second; i < std::min(w.size(), bd.second + (size_t)kBand); ++i)
      ordered.push_back(w[i]);
  w.swap(ordered);
  work->resize(w.size());
  for (size_t i = 0; i < w.size(); ++i) {
    const long long sidx = w[i].sidx;
    int k = 0;
    while (k + 1 < K && lev[k + 1].sub_base <= sidx) ++k;
    if (w[i].j >= (1LL << 27)) {
      set_error("gpw_plan: too many work chunks in one sub-box");
      return GPW_ERANGE;
    }
    (*work)[i] = make_int4(0, k | (int)(w[i].j << 4), (int)(sidx - lev[k].sub_base),
                           (int)std::min<long long>(w[i].c, 1 << 30));
  }
  *nwork_out = (long long)w.size();
  return GPW_OK;
}

int build_host_plan(const gpw_desc* desc, Plan* plan, HostArrays* H) {
  if (!desc || !plan || !H) {
    set_error("gpw_plan: NULL argument");
    return GPW_EINVAL;
  }
  const double* lat = desc->lattice;
  for (int i = 0; i < 9; ++i) plan->lat[i] = lat[i];
  plan->skew = false;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      if (i != j && lat[3 * i + j] != 0.0) plan->skew = true;
  if (!plan->skew) {
    for (int d = 0; d < 3; ++d) {
      plan->L[d] = lat[4 * d];
      if (!(plan->L[d] > 0)) {
        set_error("gpw_plan: lattice lengths must be positive");
        return GPW_EINVAL;
      }
    }
    plan->omega = plan->L[0] * plan->L[1] * plan->L[2];
  } else {
    // rows R_d, lengths |R_d|, reciprocal rows b_0 = R_1 x R_2 / V, b_1 = R_2 x R_0 / V,
    // b_2 = R_0 x R_1 / V with V = R_0 . (R_1 x R_2)
    const double* R[3] = {lat, lat + 3, lat + 6};
    double cr[3][3];
    for (int d = 0; d < 3; ++d) {
      const double* a = R[(d + 1) % 3];
      const double* b = R[(d + 2) % 3];
      cr[d][0] = a[1] * b[2] - a[2] * b[1];
      cr[d][1] = a[2] * b[0] - a[0] * b[2];
      cr[d][2] = a[0] * b[1] - a[1] * b[0];
      plan->L[d] = std::sqrt(R[d][0] * R[d][0] + R[d][1] * R[d][1] + R[d][2] * R[d][2]);
    }
    const double V = R[0][0] * cr[0][0] + R[0][1] * cr[0][1] + R[0][2] * cr[0][2];
    if (!(std::fabs(V) > 0) || !std::isfinite(V)) {
      set_error("gpw_plan: the lattice rows must be linearly independent");
      return GPW_EINVAL;
    }
    for (int d = 0; d < 3; ++d)
      for (int c = 0; c < 3; ++c) plan->rec[3 * d + c] = cr[d][c] / V;
    plan->omega = std::fabs(V);
  }
  if (desc->nlevels < 1 || desc->nlevels > GPW_MAX_LEVELS) {
    set_error("gpw_plan: nlevels must be in 1..GPW_MAX_LEVELS");
    return GPW_EINVAL;
  }
  if (desc->natm < 1 || desc->nshell < 1 || !desc->coords || !desc->shell_atom ||
      !desc->shell_l || !desc->shell_nprim || !desc->shell_prim_off || !desc->exponents ||
      !desc->coeffs) {
    set_error("gpw_plan: empty or missing basis/atoms");
    return GPW_EINVAL;
  }
  if (!(desc->tau > 0)) {
    set_error("gpw_plan: tau must be positive");
    return GPW_EINVAL;
  }
  const int K = desc->nlevels;
  plan->nlev = K;
  if (desc->tile[0] || desc->tile[1] || desc->tile[2]) {
    if (!(gpw_tile_supported(desc->tile[0], desc->tile[1], desc->tile[2]) & GPW_TILE_COLLOC)) {
      set_error("gpw_plan: unsupported tile shape");
      return GPW_EINVAL;
    }
    for (int d = 0; d < 3; ++d) plan->tile[d] = desc->tile[d];
  }
  const bool integ_default = !(desc->tile_integ[0] || desc->tile_integ[1] || desc->tile_integ[2]);
  if (!integ_default) {
    const int zw = desc->integ_zwin ? desc->integ_zwin : desc->tile_integ[2];
    if (!gpw_integ_zwin_supported(desc->tile_integ[0], desc->tile_integ[1], desc->tile_integ[2], zw)) {
      set_error("gpw_plan: unsupported integration tile shape or z window");
      return GPW_EINVAL;
    }
    for (int d = 0; d < 3; ++d) plan->tile_i[d] = desc->tile_integ[d];
    plan->zwin_i = zw;
  } else if (desc->integ_zwin) {
    set_error("gpw_plan: integ_zwin needs an explicit tile_integ");
    return GPW_EINVAL;
  }
  if (desc->colloc_warps != 0 && desc->colloc_warps != 4 && desc->colloc_warps != 6 &&
      desc->colloc_warps != 8) {
    set_error("gpw_plan: colloc_warps must be 0, 4, 6 or 8");
    return GPW_EINVAL;
  }
  if (desc->integ_chunk < 0) {
    set_error("gpw_plan: integ_chunk must be >= 0");
    return GPW_EINVAL;
  }
  if (desc->xc != GPW_XC_LDA_X && desc->xc != GPW_XC_PBE_X) {
    set_error("gpw_plan: unknown exchange functional (xc)");
    return GPW_EINVAL;
  }
  plan->xc = desc->xc;
  if (desc->host_threads < 0) {
    set_error("gpw_plan: host_threads must be >= 0");
    return GPW_EINVAL;
  }
  g_host_threads = desc->host_threads;
  if (desc->flags & ~(GPW_TAU | GPW_HOST_TASKS | GPW_FAST_BLOCK_PRUNE | GPW_DEBUG_CHECKS)) {
    set_error("gpw_plan: unknown flags");
    return GPW_EINVAL;
  }
  plan->xr = (desc->flags & GPW_TAU) ? 2 : 0;
  plan->debug = (desc->flags & GPW_DEBUG_CHECKS) != 0;
  if (plan->skew) {
    // the non-orthogonal kernels use 4x8x16 sub-boxes for both passes
    const bool tc = desc->tile[0] || desc->tile[1] || desc->tile[2];
    const bool ti = desc->tile_integ[0] || desc->tile_integ[1] || desc->tile_integ[2];
    if ((tc && !(desc->tile[0] == kT0 && desc->tile[1] == kT1 && desc->tile[2] == kT2)) ||
        (ti && !(desc->tile_integ[0] == kT0 && desc->tile_integ[1] == kT1 &&
                 desc->tile_integ[2] == kT2))) {
      set_error("gpw_plan: non-orthogonal cells use the 4x8x16 sub-box for both passes");
      return GPW_EINVAL;
    }
    plan->tile_i[0] = kT0;
    plan->tile_i[1] = kT1;
    plan->tile_i[2] = kT2;
    plan->zwin_i = kT2;
  }
  plan->nw_colloc_req = desc->colloc_warps;
  plan->natm = desc->natm;
  plan->nshell = desc->nshell;
  plan->coords.assign(desc->coords, desc->coords + 3 * desc->natm);
  const double rel = desc->rel_cutoff > 0 ? desc->rel_cutoff : 40.0;

  // ---- multigrid levels (Sec. II): cutoffs E_k and meshes
  int mesh[GPW_MAX_LEVELS][3];
  for (int k = 0; k < K; ++k) {
    if (desc->meshes) {
      double G = 1e300;
      for (int d = 0; d < 3; ++d) {
        mesh[k][d] = desc->meshes[3 * k + d];
        if (mesh[k][d] < 2) {
          set_error("gpw_plan: explicit meshes must be >= 2");
          return GPW_EINVAL;
        }
        G = std::min(G, 2.0 * M_PI * (double)((mesh[k][d] - 1) / 2) / plan->L[d]);
      }
      plan->E[k] = 0.5 * G * G;
    } else {
      if (!(desc->cutoff_ha > 0) || !(desc->level_ratio > 1.0)) {
        set_error("gpw_plan: cutoff_ha > 0 and level_ratio > 1 required without meshes");
        return GPW_EINVAL;
      }
      double div = 1.0;
      for (int i = 0; i < k; ++i) div *= desc->level_ratio;
      plan->E[k] = desc->cutoff_ha / div;
      double G = std::sqrt(2.0 * plan->E[k]);
      for (int d = 0; d < 3; ++d)
        mesh[k][d] = smooth7_even_at_least(2 * (int)std::ceil(G * plan->L[d] / (2.0 * M_PI)) + 1);
    }
  }
  for (int k = 0; k < K; ++k) {
    LevelInfo& lv = plan->lev[k];
    double G = std::sqrt(2.0 * plan->E[k]);
    lv.Gk2 = G * G;
    for (int d = 0; d < 3; ++d) {
      lv.N[d] = mesh[k][d];
      lv.h[d] = plan->L[d] / lv.N[d];
      // the strict sphere |G| < G_k must stay inside |m_d| <= (N_d - 1)/2 on its level
      // and on the finest level, so the field stays real and no Nyquist plane is used
      if (!(G * plan->L[d] / (2.0 * M_PI) <= (double)((lv.N[d] - 1) / 2)) ||
          mesh[k][d] > mesh[0][d]) {
        set_error("gpw_plan: level mesh too small for its cutoff sphere");
        return GPW_EINVAL;
      }
    }
    for (int d = 0; d < 3; ++d) lv.nsb[d] = (lv.N[d] + plan->tile[d] - 1) / plan->tile[d];
    lv.weight = plan->omega / ((double)lv.N[0] * lv.N[1] * lv.N[2]);
    for (int i = 0; i < 6; ++i) lv.gm[i] = 0.0;
    for (int i = 0; i < 9; ++i) lv.fr[i] = 0.0;
    if (plan->skew) {
      static const int pd[6][2] = {{0, 0}, {1, 1}, {2, 2}, {0, 1}, {0, 2}, {1, 2}};
      for (int i = 0; i < 6; ++i) {
        const int d = pd[i][0], e = pd[i][1];
        double g = 0.0;
        for (int c = 0; c < 3; ++c) g += (lat[3 * d + c] / lv.N[d]) * (lat[3 * e + c] / lv.N[e]);
        lv.gm[i] = g;
      }
      for (int d = 0; d < 3; ++d)
        for (int c = 0; c < 3; ++c) lv.fr[3 * d + c] = lv.N[d] * plan->rec[3 * d + c];
    }
  }
  plan->skew_zc = false;
  for (int k = 0; k < K; ++k)
    plan->skew_zc = plan->skew_zc || plan->lev[k].gm[4] != 0.0 || plan->lev[k].gm[5] != 0.0;
  for (int k = 1; k < K; ++k)
    if (plan->E[k] > plan->E[k - 1]) {
      set_error("gpw_plan: level cutoffs must decrease from level 0");
      return GPW_EINVAL;
    }

  // ---- primitives
  std::vector<Prim> prims;
  std::vector<long long> ao_off(desc->nshell + 1, 0);
  for (int s = 0; s < desc->nshell; ++s) {
    int l = desc->shell_l[s];
    if (l < 0 || l > kShellLmax) {
      set_error("gpw_plan: shell angular momentum must be 0..3");
      return GPW_EINVAL;
    }
    int a = desc->shell_atom[s];
    if (a < 0 || a >= desc->natm) {
      set_error("gpw_plan: shell_atom out of range");
      return GPW_EINVAL;
    }
    ao_off[s + 1] = ao_off[s] + (l + 1) * (l + 2) / 2;
    for (int k = 0; k < desc->shell_nprim[s]; ++k) {
      double alpha = desc->exponents[desc->shell_prim_off[s] + k];
      double c = desc->coeffs[desc->shell_prim_off[s] + k];
      if (!(alpha > 0)) {
        set_error("gpw_plan: exponents must be positive");
        return GPW_EINVAL;
      }
      Prim p;
      p.atom = a;
      p.l = l;
      p.shell = s;
      p.ao = ao_off[s];
      p.alpha = alpha;
      p.cn = c * prim_norm(l, alpha);
      p.rcut = prim_rcut(std::fabs(p.cn), l, alpha, desc->tau);
      prims.push_back(p);
    }
  }
  plan->nao = (int)ao_off[desc->nshell];
  plan->nprim = (int)prims.size();
  plan->prim_atom.resize(prims.size());
  plan->prim_alpha.resize(prims.size());
  for (size_t i = 0; i < prims.size(); ++i) {
    plan->prim_atom[i] = prims[i].atom;
    plan->prim_alpha[i] = prims[i].alpha;
  }

  // ---- pair screening over images (Sec. III A, Eq. cut)
  const int natm = desc->natm;
  std::vector<std::vector<int>> atom_prims(natm);
  std::vector<double> atom_rmax(natm, -1.0);
  for (int i = 0; i < (int)prims.size(); ++i) {
    if (prims[i].rcut < 0) continue;
    atom_prims[prims[i].atom].push_back(i);
    atom_rmax[prims[i].atom] = std::max(atom_rmax[prims[i].atom], prims[i].rcut);
  }
  // each atom's primitives by decreasing r_cut: the distance test r_a + r_b > |A - B_T|
  // then fails for all later b once it fails for one (the order of the pairs found does
  // not matter, they are sorted below)
  for (auto& v : atom_prims)
    std::stable_sort(v.begin(), v.end(), [&](int x, int y) { return prims[x].rcut > prims[y].rcut; });
  const double* X = desc->coords;
  SkewBox skb;
  skb.rec = plan->rec;
  for (int d = 0; d < 3; ++d)
    skb.blen[d] = std::sqrt(plan->rec[3 * d] * plan->rec[3 * d] +
                            plan->rec[3 * d + 1] * plan->rec[3 * d + 1] +
                            plan->rec[3 * d + 2] * plan->rec[3 * d + 2]);
  plan->prune = (desc->flags & GPW_FAST_BLOCK_PRUNE) != 0;
  for (int d = 0; d < 3; ++d) plan->prune_blen[d] = plan->skew ? skb.blen[d] : 1.0 / plan->L[d];
  plan->prune_lam = plan->skew ? metric_lambda_min(plan->lat) : 0.0;
  // atoms are screened in parallel (each thread keeps its own pair list); the sort
  // below fixes one order whatever the thread count
  // (the work is about one candidate pair per two primitive pairs within reach: 4.4e5
  // for the 32-water cell's 832 primitives)
  const int sthr = plan_threads((long long)prims.size() * prims.size() / 2);
  std::vector<std::vector<PairTmp>> tpairs(sthr);
#pragma omp parallel for num_threads(sthr) schedule(dynamic, 1)
  for (int ia = 0; ia < natm; ++ia) {
    std::vector<PairTmp>& pairs = tpairs[omp_get_thread_num()];
    if (atom_rmax[ia] < 0) continue;
    for (int ib = 0; ib < natm; ++ib) {
      if (atom_rmax[ib] < 0) continue;
      double rsum_max = atom_rmax[ia] + atom_rmax[ib];
      int nlo[3], nhi[3];
      for (int d = 0; d < 3; ++d) {
        if (!plan->skew) {
          double dd = X[3 * ia + d] - X[3 * ib + d];
          // one more image on each side than the atom-level bound: the exact
          // per-primitive distance test below decides
          nlo[d] = (int)std::floor((dd - rsum_max) / plan->L[d]) - 1;
          nhi[d] = (int)std::ceil((dd + rsum_max) / plan->L[d]) + 1;
        } else {
          // |f_d(A - B - T)| <= |A - B - T| |b_d| along the reciprocal row b_d
          double f = 0.0;
          for (int c = 0; c < 3; ++c) f += plan->rec[3 * d + c] * (X[3 * ia + c] - X[3 * ib + c]);
          nlo[d] = (int)std::floor(f - rsum_max * skb.blen[d]) - 1;
          nhi[d] = (int)std::ceil(f + rsum_max * skb.blen[d]) + 1;
        }
      }
      for (int n0 = nlo[0]; n0 <= nhi[0]; ++n0)
        for (int n1 = nlo[1]; n1 <= nhi[1]; ++n1)
          for (int n2 = nlo[2]; n2 <= nhi[2]; ++n2) {
            const int nn[3] = {n0, n1, n2};
            double Bt[3], AB2 = 0.0;
            for (int d = 0; d < 3; ++d) {
              Bt[d] = plan->skew ? X[3 * ib + d] + (((double)n0 * lat[d] + (double)n1 * lat[3 + d]) +
                                                    (double)n2 * lat[6 + d])
                                 : X[3 * ib + d] + (double)nn[d] * plan->L[d];
              double t = X[3 * ia + d] - Bt[d];
              AB2 += t * t;
            }
            if (std::sqrt(AB2) >= rsum_max + 1e-9 * (1.0 + rsum_max)) continue;
            const double dist = std::sqrt(AB2);
            for (int a : atom_prims[ia]) {
              if (!(dist < prims[a].rcut + atom_rmax[ib])) break;
              for (int b : atom_prims[ib]) {
                const Prim& pa = prims[a];
                const Prim& pb = prims[b];
                double rsum = pa.rcut + pb.rcut;
                if (!(dist < rsum)) break;
                if (a > b) continue;
                double aa = pa.alpha, ab = pb.alpha, ap = aa + ab;
                double P[3], dA2 = 0.0, dB2 = 0.0;
                for (int d = 0; d < 3; ++d) {
                  P[d] = (aa * X[3 * ia + d] + ab * Bt[d]) / ap;
                  double ta = P[d] - X[3 * ia + d], tb = P[d] - Bt[d];
                  dA2 += ta * ta;
                  dB2 += tb * tb;
                }
                double kab = std::exp(-aa * ab * AB2 / ap);
                double cab = std::fabs(pa.cn * pb.cn);
                int level = 0;
                for (int k = K - 1; k >= 0; --k)
                  if (plan->E[k] >= rel * ap) {
                    level = k;
                    break;
                  }
                PairTmp t;
                const double Nl[3] = {(double)mesh[level][0], (double)mesh[level][1],
                                      (double)mesh[level][2]};
                double Rp = 0.0;
                if (!pair_box(cab, kab, pa.l, pb.l, std::sqrt(dA2), std::sqrt(dB2), ap,
                              desc->tau, P, Nl, plan->L, t.lo, t.hi,
                              plan->skew ? &skb : nullptr, &Rp))
                  continue;
                if (plan->prune) {
                  // P's fractional coordinates as the boxes take them, and R_p
                  double fp[3];
                  for (int d = 0; d < 3; ++d) {
                    if (plan->skew) {
                      fp[d] = 0.0;
                      for (int c = 0; c < 3; ++c) fp[d] += plan->rec[3 * d + c] * P[c];
                    } else {
                      fp[d] = P[d] / plan->L[d];
                    }
                  }
                  t.q = PairQ{fp[0], fp[1], fp[2], Rp};
                } else {
                  t.q = PairQ{0.0, 0.0, 0.0, 0.0};
                }
                t.a = a;
                t.b = b;
                t.sa = pa.shell;
                t.sb = pb.shell;
                t.level = level;
                for (int d = 0; d < 3; ++d) t.img[d] = nn[d];
                if (t.hi[0] < t.lo[0] || t.hi[1] < t.lo[1] || t.hi[2] < t.lo[2]) continue;
                pairs.push_back(t);
              }
            }
          }
    }
  }
  // deterministic order: contracted shell pair, then primitives, then image.  The keys
  // are unique, so the order does not depend on how it is reached: the pairs are
  // bucketed by their first shell and the buckets sorted in parallel.  Where the fields
  // fit, each pair's key is packed into 64 bits in that order (shells 16 bits each, the
  // primitives' places in their shells 4 bits each, the image 8 bits per component): the
  // threads' lists scatter (key, source) records into the buckets in parallel, the
  // buckets are sorted, and the pairs are gathered once in key order.
  std::vector<PairTmp> pairs;
  {
    const int nsh = desc->nshell;
    const int nt = (int)tpairs.size();
    std::vector<long long> tbase(nt + 1, 0);
    for (int t = 0; t < nt; ++t) tbase[t + 1] = tbase[t] + (long long)tpairs[t].size();
    const long long total = tbase[nt];
    std::vector<int> shell_first(nsh + 1, 0);
    bool packable = nsh <= 65536;
    for (int i = 0; i < nsh; ++i) {
      shell_first[i + 1] = shell_first[i] + desc->shell_nprim[i];
      packable = packable && desc->shell_nprim[i] <= 16;
    }
    // per thread list and bucket: counts, then the start of its run in the bucket
    std::vector<long long> cnt((size_t)nt * (nsh + 1), 0);
#pragma omp parallel for num_threads(nt) schedule(static, 1) reduction(&& : packable)
    for (int t = 0; t < nt; ++t) {
      long long* c = cnt.data() + (size_t)t * (nsh + 1);
      for (const PairTmp& q : tpairs[t]) {
        ++c[q.sa];
        for (int d = 0; d < 3; ++d) packable = packable && q.img[d] >= -128 && q.img[d] < 128;
      }
    }
    std::vector<long long> boff(nsh + 1, 0);
    {
      long long run = 0;
      for (int i = 0; i < nsh; ++i) {
        boff[i] = run;
        for (int t = 0; t < nt; ++t) {
          long long& c = cnt[(size_t)t * (nsh + 1) + i];
          const long long n = c;
          c = run;  // now the start of thread t's run in bucket i
          run += n;
        }
      }
      boff[nsh] = run;
    }
    const int sthr2 = plan_threads(total);
    pairs.resize(total);
    if (packable) {
      struct KeyIdx {
        uint64_t key;
        long long src;  // tbase[thread] + index in its list
      };
      std::vector<KeyIdx> kv(total);
#pragma omp parallel for num_threads(nt) schedule(static, 1)
      for (int t = 0; t < nt; ++t) {
        long long* c = cnt.data() + (size_t)t * (nsh + 1);
        const std::vector<PairTmp>& v = tpairs[t];
        for (size_t i = 0; i < v.size(); ++i) {
          const PairTmp& q = v[i];
          uint64_t k = (uint64_t)q.sa << 48 | (uint64_t)q.sb << 32 |
                       (uint64_t)(q.a - shell_first[q.sa]) << 28 |
                       (uint64_t)(q.b - shell_first[q.sb]) << 24;
          for (int d = 0; d < 3; ++d) k |= (uint64_t)(q.img[d] + 128) << (16 - 8 * d);
          kv[c[q.sa]++] = KeyIdx{k, tbase[t] + (long long)i};
        }
      }
#pragma omp parallel for num_threads(sthr2) schedule(dynamic, 4)
      for (int i = 0; i < nsh; ++i)
        std::sort(kv.begin() + boff[i], kv.begin() + boff[i + 1],
                  [](const KeyIdx& x, const KeyIdx& y) { return x.key < y.key; });
#pragma omp parallel for num_threads(sthr2) schedule(static)
      for (long long j = 0; j < total; ++j) {
        const long long src = kv[j].src;
        const int t = (int)(std::upper_bound(tbase.begin(), tbase.end(), src) - tbase.begin()) - 1;
        pairs[j] = tpairs[t][src - tbase[t]];
      }
    } else {
      auto less = [](const PairTmp& x, const PairTmp& y) {
        if (x.sa != y.sa) return x.sa < y.sa;
        if (x.sb != y.sb) return x.sb < y.sb;
        if (x.a != y.a) return x.a < y.a;
        if (x.b != y.b) return x.b < y.b;
        for (int d = 0; d < 3; ++d)
          if (x.img[d] != y.img[d]) return x.img[d] < y.img[d];
        return false;
      };
#pragma omp parallel for num_threads(nt) schedule(static, 1)
      for (int t = 0; t < nt; ++t) {
        long long* c = cnt.data() + (size_t)t * (nsh + 1);
        for (const PairTmp& q : tpairs[t]) pairs[c[q.sa]++] = q;
      }
#pragma omp parallel for num_threads(sthr2) schedule(dynamic, 4)
      for (int i = 0; i < nsh; ++i) std::sort(pairs.begin() + boff[i], pairs.begin() + boff[i + 1], less);
    }
    std::vector<std::vector<PairTmp>>().swap(tpairs);
  }
  const long long np = (long long)pairs.size();
  plan->npairs = np;
  if (np > (1LL << 31) - 1) {
    set_error("gpw_plan: too many pairs");
    return GPW_ERANGE;
  }

  // ---- per-pair arrays
  H->hot_a.resize(np);
  H->hot_b.resize(np);
  H->ids.resize(np);
  H->ids2.resize(np);
  H->geo.resize(8 * np);
  H->cab.resize(np);
  H->tab_off.resize(np);
  H->coef_off.resize(np);
  H->part_off.resize(np);
  H->xt_off.resize(np);
  H->yt_off.resize(np);
  plan->h_ab.resize(2 * np);
  plan->h_img.resize(3 * np);
  plan->h_lev.resize(np);
  plan->h_lo.resize(3 * np);
  plan->h_hi.resize(3 * np);
  plan->pair_a.resize(np);
  plan->pair_b.resize(np);
  // per-pair records in parallel, then the offsets and statistics in pair order
  const int pthr = plan_threads(np);
#pragma omp parallel for num_threads(pthr) schedule(static)
  for (long long p = 0; p < np; ++p) {
    const PairTmp& t = pairs[p];
    const Prim& pa = prims[t.a];
    const Prim& pb = prims[t.b];
    const int L = pa.l + pb.l;
    int n[3];
    for (int d = 0; d < 3; ++d) n[d] = t.hi[d] - t.lo[d] + 1;
    H->hot_a[p] = make_int4(t.lo[0], t.lo[1], t.lo[2], L);
    H->hot_b[p] = make_int4(n[0], n[1], n[2], t.level);
    H->ids[p] = make_int4(pa.l, pb.l, (int)pa.ao, (int)pb.ao);
    H->ids2[p] = make_int4(pa.atom, pb.atom, t.a < t.b ? 2 : 1, 0);
    for (int d = 0; d < 3; ++d) {
      H->geo[8 * p + d] = X[3 * pa.atom + d];
      H->geo[8 * p + 3 + d] =
          plan->skew ? X[3 * pb.atom + d] + (((double)t.img[0] * lat[d] + (double)t.img[1] * lat[3 + d]) +
                                             (double)t.img[2] * lat[6 + d])
                     : X[3 * pb.atom + d] + (double)t.img[d] * plan->L[d];
    }
    H->geo[8 * p + 6] = pa.alpha;
    H->geo[8 * p + 7] = pb.alpha;
    H->cab[p] = pa.cn * pb.cn;
    plan->h_ab[2 * p] = t.a;
    plan->h_ab[2 * p + 1] = t.b;
    plan->pair_a[p] = t.a;
    plan->pair_b[p] = t.b;
    for (int d = 0; d < 3; ++d) {
      plan->h_img[3 * p + d] = t.img[d];
      plan->h_lo[3 * p + d] = t.lo[d];
      plan->h_hi[3 * p + d] = t.hi[d];
    }
    plan->h_lev[p] = t.level;
  }
  long long tab_total = 0, coef_total = 0, xt_total = 0, yt_total = 0;
  int lmax = 0;
  for (long long p = 0; p < np; ++p) {
    const int L = H->hot_a[p].w, lev = H->hot_b[p].w;
    const int n[3] = {H->hot_b[p].x, H->hot_b[p].y, H->hot_b[p].z};
    lmax = std::max(lmax, L);
    H->tab_off[p] = tab_total;
    tab_total += (long long)(L + 2 + plan->xr) * (n[0] + n[1] + n[2]);
    // non-orthogonal cells: the cross-factor tables R01, R02, R12 after the 1-D tables
    if (plan->skew)
      tab_total += (long long)n[0] * n[1] + (long long)n[0] * n[2] + (long long)n[1] * n[2];
    H->coef_off[p] = coef_total;
    coef_total += nc3(L + 1 + plan->xr);
    H->xt_off[p] = xt_total;
    xt_total += (long long)nc2(L + plan->xr) * n[0];
    H->yt_off[p] = yt_total;
    yt_total += (long long)(L + 1 + plan->xr) * n[0] * n[1];
    long long pts = (long long)n[0] * n[1] * n[2];
    plan->pair_points += pts;
    plan->pair_points_level[lev] += pts;
    plan->pair_points_L[L] += pts;
    plan->npairs_level[lev] += 1;
    plan->flops_rho += 2.0 * (L + 1) * (double)pts;
    plan->flops_mat += 2.0 * (L + 1) * (double)pts;
    plan->flops_ip1 += 2.0 * (L + 2) * (double)pts;
  }
  plan->lmax = lmax;
  if (integ_default && !plan->skew) {
    // default integration sub-boxes: 8x8x16 with 48-point z windows (a pair box crosses
    // fewer window ends than sub-box ends: fewer tasks, one y contraction per window)
    // when the staging of this plan's degrees leaves two thread blocks per SM (228 KB of
    // shared memory, 1 KB of it reserved per block), else plain 8x8x32 sub-boxes
    const int tw[3] = {8, 8, 16};
    const size_t two_blocks = (228 * 1024 - 2 * 1024) / 2;
    const size_t need = integ_block_smem(tw, 48, lmax);
    const bool win = need > 0 && need <= two_blocks;
    for (int d = 0; d < 3; ++d) plan->tile_i[d] = win ? tw[d] : (d == 2 ? 32 : 8);
    plan->zwin_i = win ? 48 : 32;
  }
  plan->tab_total = tab_total;
  plan->coef_total = coef_total;
  plan->xt_total = xt_total;
  plan->yt_base = (xt_total + 1) & ~1LL;  // after the x-contracted tables, 16-byte aligned
  plan->yt_total = yt_total;

  // ---- per-level sub-box task lists (CSR), one task per (pair, sub-box, image shift),
  // for the collocation tile and for the integration tile
  std::vector<int> ranks;
  std::vector<long long> psize;
  // by default only the per-pair task counts are taken here and the device builds the
  // records at commit; GPW_HOST_TASKS builds them on the host
  const bool host_tasks = (desc->flags & GPW_HOST_TASKS) != 0;
  plan->tasks_on_device = !host_tasks;
  const std::vector<PairBox> pv = pairs_view(pairs);
  if (plan->prune && !host_tasks) {
    H->prune.resize(pv.size());
    for (size_t p = 0; p < pv.size(); ++p) H->prune[p] = pv[p].q;
  }
  int rc = host_tasks
               ? build_tasks(plan, pv, H->hot_a, plan->tile, plan->tile[2], plan->lev,
                             &H->sub_off_c, &H->task_c,
                             &H->work_c, &plan->nent, &plan->nwork, &plan->nsub_total, nullptr,
                             nullptr, nullptr, plan->prune)
               : count_tasks(plan, pv, H->hot_a, plan->tile, plan->tile[2], plan->lev,
                             &plan->nsub_total,
                             &H->toff_c, &plan->nent, nullptr, nullptr);
  if (rc) return rc;
  for (int k = 0; k < K; ++k) plan->lev_i[k] = plan->lev[k];
  for (int k = 0; k < K; ++k)
    for (int d = 0; d < 3; ++d)
      plan->lev_i[k].nsb[d] = (plan->lev[k].N[d] + plan->tile_i[d] - 1) / plan->tile_i[d];
  long long nsub_i = 0;
  // integration chunks (auto): about four items per resident block of the whole launch,
  // so that no sub-box with many tasks is left running alone at the end
  long long chunk = desc->integ_chunk > 0 ? desc->integ_chunk : -1;
  if (host_tasks) {
    rc = build_tasks(plan, pv, H->hot_a, plan->tile_i, plan->zwin_i, plan->lev_i,
                     &H->sub_off_i, &H->task_i,
                     &H->work_i, &plan->nent_i, &plan->nwork_i, &nsub_i, &ranks, &psize, &chunk);
  } else {
    rc = count_tasks(plan, pv, H->hot_a, plan->tile_i, plan->zwin_i, plan->lev_i, &nsub_i,
                     &H->toff_i,
                     &plan->nent_i, &ranks, &psize);
    if (chunk < 0) chunk = default_chunk(plan->nent_i);
  }
  plan->chunk_i = (int)chunk;
  plan->nsub_i = nsub_i;
  if (rc) return rc;
  long long part_total = 0;
  for (long long p = 0; p < np; ++p) {
    H->ids2[p].w = ranks[p];
    H->part_off[p] = part_total;
    part_total += psize[p];
  }
  // the part buffer holds the task W tensors of the integration, or the two contracted D
  // tables of the collocation
  plan->part_total = std::max(part_total, plan->yt_base + yt_total);

  if (plan->skew) build_mono_transforms(*plan, &H->mono_t);

  // ---- V assembly groups: runs of pairs with the same contracted shell pair
  for (long long p = 0; p < np;) {
    long long q = p;
    while (q < np && pairs[q].sa == pairs[p].sa && pairs[q].sb == pairs[p].sb) ++q;
    H->groups.push_back(make_int4(pairs[p].sa, pairs[p].sb, (int)p, (int)q));
    p = q;
  }
  plan->ngroups = (long long)H->groups.size();

  // ---- gradient assembly: per atom, the (pair, side) contributions in pair order
  std::vector<long long> acount(natm + 1, 0);
  for (long long p = 0; p < np; ++p) {
    acount[prims[pairs[p].a].atom + 1]++;
    acount[prims[pairs[p].b].atom + 1]++;
  }
  for (int i = 0; i < natm; ++i) acount[i + 1] += acount[i];
  H->atom_off = acount;
  H->atom_list.resize(2 * np);
  std::vector<long long> afill(acount.begin(), acount.end() - 1);
  for (long long p = 0; p < np; ++p) {
    H->atom_list[afill[prims[pairs[p].a].atom]++] = (int)(2 * p);
    H->atom_list[afill[prims[pairs[p].b].atom]++] = (int)(2 * p + 1);
  }

  // ---- spectral sizes
  plan->grid_total = 0;
  plan->spec_total = 0;
  for (int k = 0; k < K; ++k) {
    LevelInfo& lv = plan->lev[k];
    lv.grid_off = plan->grid_total;
    lv.spec_off = plan->spec_total;
    plan->grid_total += (long long)lv.N[0] * lv.N[1] * lv.N[2];
    plan->spec_total += (long long)lv.N[0] * lv.N[1] * (lv.N[2] / 2 + 1);
  }
  // the integration-tile level table shares everything but its sub-box fields
  for (int k = 0; k < K; ++k) {
    plan->lev_i[k].grid_off = plan->lev[k].grid_off;
    plan->lev_i[k].spec_off = plan->lev[k].spec_off;
  }
  plan->fine_n = (long long)plan->lev[0].N[0] * plan->lev[0].N[1] * plan->lev[0].N[2];
  plan->fine_spec_n = (long long)plan->lev[0].N[0] * plan->lev[0].N[1] * (plan->lev[0].N[2] / 2 + 1);
  return GPW_OK;
}

void recycle_host_arrays(HostArrays* H) {
  if (!H) return;
  std::lock_guard<std::mutex> lk(g_task_pool_mu);
  for (std::vector<int4>* v : {&H->task_c, &H->task_i}) {
    if (v->capacity() == 0) continue;
    g_task_pool.push_back(std::move(*v));
    v->clear();
  }
  // keep the largest buffers within the byte cap
  std::sort(g_task_pool.begin(), g_task_pool.end(),
            [](const std::vector<int4>& a, const std::vector<int4>& b) {
              return a.capacity() > b.capacity();
            });
  std::vector<std::vector<int4>> kept;
  size_t total = 0;
  for (auto& v : g_task_pool) {
    const size_t b = v.capacity() * sizeof(int4);
    if (total + b > kTaskPoolBytes) continue;
    total += b;
    kept.push_back(std::move(v));
  }
  g_task_pool.swap(kept);
}

void build_coef_tables(CoefTables* t) {
  std::memset(t, 0, sizeof(*t));
  for (int L = 0; L <= kDegMax; ++L) {
    int c21 = 0, flat = 0;
    for (int l2 = 0; l2 <= L; ++l2) {
      t->c21base[L][l2] = c21;
      for (int l1 = 0; l1 <= L - l2; ++l1) {
        t->dec21[L][c21] = l2 | (l1 << 8) | (flat << 16);
        for (int l0 = 0; l0 <= L - l2 - l1; ++l0) t->dec3[L][flat++] = c21 | (l0 << 8);
        ++c21;
      }
    }
  }
}

}  // namespace gpw
