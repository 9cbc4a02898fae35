/*
 * Plain FP64 CPU oracle for the multigrid GPW pair <-> grid contractions.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference leg may load this library.  It shares no code with the
 * CUDA path and must never be linked into it.
 *
 * What it computes (arXiv 2603.24881):
 *   - shell cutoff radius, Eq. (cut):  r^2 phi_R(r) < tau, here with the angular
 *     factor r^l folded into phi_R, i.e. f(r) = |c N| r^(l+2) exp(-alpha r^2);
 *   - screened primitive pairs (a in the home cell, b at image T), Sec. III A
 *     ("single lattice sum plus folding", Eqs. rho_wrap and J_wrap), kept when
 *     |A - B - T| < r_a + r_b;
 *   - the Gaussian product centre and exponent of Eq. (gab);
 *   - density on each multigrid level, Eq. (rho_wrap), evaluated point by point
 *     ("plain": every phi_mu phi_nu from scratch) or from per-dimension 1-D
 *     factors with direct exp ("separable", the factorisation of Eq. gx/gab,
 *     exact algebra; no recursion, no binomial expansion);
 *   - the potential integral, Eq. (J_wrap), with the weight Omega/N of the
 *     level grid (Sec. III A, the V tensor definition);
 *   - the nuclear-gradient contraction of Algorithm 3: D, v and the analytic
 *     derivative of each primitive with respect to its centre.
 *
 * Lattices: `lat` holds the three lattice vectors as rows (lat[3 d + c] = component c of
 * R_d); grid point (i0, i1, i2) of an N-point level mesh sits at sum_d (i_d / N_d) R_d
 * and an image is T = sum_d n_d R_d.  With a diagonal lattice every formula reduces to
 * the orthorhombic one operation for operation (the off-diagonal terms add exact
 * zeros).  The separable mode is orthorhombic only; a non-orthogonal cell (App.,
 * non-orthogonal lattices) is evaluated point by point.
 * All arithmetic in double.  Build with -ffp-contract=off so that the screening
 * decisions are reproducible.  Collocation runs OpenMP over pairs with a static
 * pair-to-thread map into per-thread grids summed in thread order, so a density is
 * reproducible bit for bit at a given thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXCART 10

/* Cartesian components of angular momentum l, x^l first (xx, xy, xz, yy, ...). */
static int orc_cart(int l, int comp[][3]) {
  int n = 0;
  for (int ix = l; ix >= 0; --ix)
    for (int iy = l - ix; iy >= 0; --iy) {
      comp[n][0] = ix;
      comp[n][1] = iy;
      comp[n][2] = l - ix - iy;
      ++n;
    }
  return n;
}

static double orc_ipow(double x, int n) {
  double p = 1.0;
  for (int k = 0; k < n; ++k) p *= x;
  return p;
}

/* f(r) = cn * r^(l+2) * exp(-alpha r^2), Eq. (cut) with the r^2 volume factor. */
/* grid step vectors of a level: H[d][c] = R_dc / N_d */
static void orc_steps(const double* lat, const int* N, double H[3][3]) {
  for (int d = 0; d < 3; ++d)
    for (int c = 0; c < 3; ++c) H[d][c] = lat[3 * d + c] / (double)N[d];
}

/* Cartesian position of grid index (i0, i1, i2): sum_d i_d H[d] */
static void orc_point(const double H[3][3], long i0, long i1, long i2, double* r) {
  for (int c = 0; c < 3; ++c) r[c] = ((double)i0 * H[0][c] + (double)i1 * H[1][c]) + (double)i2 * H[2][c];
}

static int orc_diagonal(const double* lat) {
  return lat[1] == 0.0 && lat[2] == 0.0 && lat[3] == 0.0 && lat[5] == 0.0 && lat[6] == 0.0 &&
         lat[7] == 0.0;
}

/* cell volume |det R| ((L0 L1) L2 for a diagonal lattice) */
double orc_volume(const double* lat) {
  if (orc_diagonal(lat)) return lat[0] * lat[4] * lat[8];
  double d = lat[0] * (lat[4] * lat[8] - lat[5] * lat[7]) - lat[1] * (lat[3] * lat[8] - lat[5] * lat[6]) +
             lat[2] * (lat[3] * lat[7] - lat[4] * lat[6]);
  return fabs(d);
}

static double orc_prim_f(double cn, int l, double alpha, double r) {
  return cn * orc_ipow(r, l + 2) * exp(-alpha * r * r);
}

/* Largest root of f(r) = tau on the decreasing branch r >= sqrt((l+2)/(2 alpha)),
 * by 64 bisection steps; -1 when f stays below tau (the primitive is dropped). */
double orc_rcut(double cn, int l, double alpha, double tau) {
  double r0 = sqrt((double)(l + 2) / (2.0 * alpha));
  if (orc_prim_f(cn, l, alpha, r0) < tau) return -1.0;
  double hi = r0;
  for (int it = 0; it < 200 && orc_prim_f(cn, l, alpha, hi) >= tau; ++it) hi *= 2.0;
  double lo = r0;
  for (int it = 0; it < 64; ++it) {
    double mid = 0.5 * (lo + hi);
    if (orc_prim_f(cn, l, alpha, mid) >= tau) lo = mid; else hi = mid;
  }
  return hi;
}

/* Pair magnitude bound h(r) along the distance r from P, Eq. (cut) applied to
 * the product Gaussian of Eq. (gab):
 *   h(r) = cab * kab * (r + dA)^la * (r + dB)^lb * r^2 * exp(-ap r^2). */
static double orc_pair_h(double cab, double kab, int la, int lb, double dA, double dB,
                         double ap, double r) {
  return cab * kab * orc_ipow(r + dA, la) * orc_ipow(r + dB, lb) * r * r * exp(-ap * r * r);
}

/* d log h / dr = la/(r+dA) + lb/(r+dB) + 2/r - 2 ap r: strictly decreasing in r, so h has
 * a single maximum, at the zero of this function, never beyond sqrt((la+lb+2)/(2 ap)). */
static double orc_pair_dlogh(int la, int lb, double dA, double dB, double ap, double r) {
  return (double)la / (r + dA) + (double)lb / (r + dB) + 2.0 / r - 2.0 * ap * r;
}

/* Pair extent R_p: the largest root of h(r) = tau (Eq. cut applied to the pair), -1 when
 * h stays below tau for every r (pair dropped).  With r0 = sqrt((la+lb+2)/(2 ap)):
 *   h(r0) >= tau: the root lies beyond r0, where h decreases; bracket it by doubling and
 *     bisect 64 times;
 *   h(r0) <  tau: the maximum r* of h lies in (0, r0] (64 bisection steps on the sign of
 *     d log h / dr); h(r*) < tau drops the pair, otherwise the root is bisected 64 times
 *     on [r*, r0], where h decreases.
 * The returned value is the upper end of the final bracket: h(R_p) < tau. */
static double orc_pair_extent(double cab, double kab, int la, int lb, double dA, double dB,
                              double ap, double tau) {
  double r0 = sqrt((double)(la + lb + 2) / (2.0 * ap));
  double lo, hi;
  if (orc_pair_h(cab, kab, la, lb, dA, dB, ap, r0) >= tau) {
    hi = r0;
    for (int it = 0; it < 200 && orc_pair_h(cab, kab, la, lb, dA, dB, ap, hi) >= tau; ++it)
      hi *= 2.0;
    lo = r0;
  } else {
    double a = 0.0, b = r0;
    for (int it = 0; it < 64; ++it) {
      double mid = 0.5 * (a + b);
      if (orc_pair_dlogh(la, lb, dA, dB, ap, mid) > 0.0) a = mid; else b = mid;
    }
    double rs = a > 0.0 ? a : b;
    if (orc_pair_h(cab, kab, la, lb, dA, dB, ap, rs) < tau) return -1.0;
    lo = rs;
    hi = r0;
  }
  for (int it = 0; it < 64; ++it) {
    double mid = 0.5 * (lo + hi);
    if (orc_pair_h(cab, kab, la, lb, dA, dB, ap, mid) >= tau) lo = mid; else hi = mid;
  }
  return hi;
}

/*
 * Enumerate the screened pairs.  Primitive a <= b (global order), every lattice
 * image T = (n0 L0, n1 L1, n2 L2) of b with |A - B - T| < rc_a + rc_b (Sec. III A).
 * For each kept pair: level = coarsest level k with Ek[k] >= rel * alpha_p
 * (finest level when none qualifies), extent R_p, and the integer box
 * lo_d = ceil((P_d - R_p) N_d / L_d), hi_d = floor((P_d + R_p) N_d / L_d)
 * on that level's mesh.  Returns the number of pairs; arrays are filled for the
 * first `cap` of them.
 */
long orc_pairs(int npr, const double* pc, const int* pl, const double* pal,
               const double* pcn, const double* prc, const double* Ld, int nlev,
               const int* mesh, const double* Ek, double rel, double tau, long cap,
               int* out_ab, int* out_img, int* out_lev, int* out_lo, int* out_hi,
               double* out_R) {
  long n = 0;
  for (int a = 0; a < npr; ++a) {
    if (prc[a] < 0) continue;
    for (int b = a; b < npr; ++b) {
      if (prc[b] < 0) continue;
      double rsum = prc[a] + prc[b];
      int nlo[3], nhi[3];
      for (int d = 0; d < 3; ++d) {
        double dd = pc[3 * a + d] - pc[3 * b + d];
        nlo[d] = (int)ceil((dd - rsum) / Ld[d]);
        nhi[d] = (int)floor((dd + rsum) / Ld[d]);
      }
      for (int n0 = nlo[0]; n0 <= nhi[0]; ++n0)
        for (int n1 = nlo[1]; n1 <= nhi[1]; ++n1)
          for (int n2 = nlo[2]; n2 <= nhi[2]; ++n2) {
            int nn[3] = {n0, n1, n2};
            double B[3], AB2 = 0.0;
            for (int d = 0; d < 3; ++d) {
              B[d] = pc[3 * b + d] + (double)nn[d] * Ld[d];
              double t = pc[3 * a + d] - B[d];
              AB2 += t * t;
            }
            if (!(sqrt(AB2) < rsum)) continue;
            double aa = pal[a], ab = pal[b], ap = aa + ab;
            double P[3], dA2 = 0.0, dB2 = 0.0;
            for (int d = 0; d < 3; ++d) {
              P[d] = (aa * pc[3 * a + d] + ab * B[d]) / ap;
              double ta = P[d] - pc[3 * a + d], tb = P[d] - B[d];
              dA2 += ta * ta;
              dB2 += tb * tb;
            }
            double kab = exp(-aa * ab * AB2 / ap);
            double cab = fabs(pcn[a] * pcn[b]);
            double R = orc_pair_extent(cab, kab, pl[a], pl[b], sqrt(dA2), sqrt(dB2), ap, tau);
            if (R < 0) continue;
            int lev = 0;
            for (int k = nlev - 1; k >= 0; --k)
              if (Ek[k] >= rel * ap) { lev = k; break; }
            if (n < cap) {
              out_ab[2 * n] = a;
              out_ab[2 * n + 1] = b;
              for (int d = 0; d < 3; ++d) {
                out_img[3 * n + d] = nn[d];
                double Nd = (double)mesh[3 * lev + d];
                out_lo[3 * n + d] = (int)ceil((P[d] - R) * Nd / Ld[d]);
                out_hi[3 * n + d] = (int)floor((P[d] + R) * Nd / Ld[d]);
              }
              out_lev[n] = lev;
              out_R[n] = R;
            }
            ++n;
          }
    }
  }
  return n;
}

/*
 * orc_pairs for any lattice (rows of lat; rec = the reciprocal rows b_d with
 * b_d . R_e = delta_de).  Images: |f_d(A - B - T)| <= |A - B - T| |b_d| for the
 * fractional coordinate f_d = b_d . r, so n_d runs over
 * [ceil(f_d(A - B) - rsum |b_d|), floor(f_d(A - B) + rsum |b_d|)].  Box on the level
 * mesh: lo_d = ceil((f_d(P) - R_p |b_d|) N_d), hi_d = floor((f_d(P) + R_p |b_d|) N_d),
 * the grid points whose fractional coordinate along R_d can lie within R_p of P.
 */
long orc_pairs_lat(int npr, const double* pc, const int* pl, const double* pal,
                   const double* pcn, const double* prc, const double* lat, const double* rec,
                   int nlev, const int* mesh, const double* Ek, double rel, double tau, long cap,
                   int* out_ab, int* out_img, int* out_lev, int* out_lo, int* out_hi,
                   double* out_R) {
  double blen[3];
  for (int d = 0; d < 3; ++d)
    blen[d] = sqrt(rec[3 * d] * rec[3 * d] + rec[3 * d + 1] * rec[3 * d + 1] + rec[3 * d + 2] * rec[3 * d + 2]);
  long n = 0;
  for (int a = 0; a < npr; ++a) {
    if (prc[a] < 0) continue;
    for (int b = a; b < npr; ++b) {
      if (prc[b] < 0) continue;
      double rsum = prc[a] + prc[b];
      int nlo[3], nhi[3];
      for (int d = 0; d < 3; ++d) {
        double f = 0.0;
        for (int c = 0; c < 3; ++c) f += rec[3 * d + c] * (pc[3 * a + c] - pc[3 * b + c]);
        nlo[d] = (int)ceil(f - rsum * blen[d]);
        nhi[d] = (int)floor(f + rsum * blen[d]);
      }
      for (int n0 = nlo[0]; n0 <= nhi[0]; ++n0)
        for (int n1 = nlo[1]; n1 <= nhi[1]; ++n1)
          for (int n2 = nlo[2]; n2 <= nhi[2]; ++n2) {
            int nn[3] = {n0, n1, n2};
            double B[3], AB2 = 0.0;
            for (int c = 0; c < 3; ++c) {
              B[c] = pc[3 * b + c] + (((double)n0 * lat[c] + (double)n1 * lat[3 + c]) + (double)n2 * lat[6 + c]);
              double t = pc[3 * a + c] - B[c];
              AB2 += t * t;
            }
            if (!(sqrt(AB2) < rsum)) continue;
            double aa = pal[a], ab = pal[b], ap = aa + ab;
            double P[3], dA2 = 0.0, dB2 = 0.0;
            for (int c = 0; c < 3; ++c) {
              P[c] = (aa * pc[3 * a + c] + ab * B[c]) / ap;
              double ta = P[c] - pc[3 * a + c], tb = P[c] - B[c];
              dA2 += ta * ta;
              dB2 += tb * tb;
            }
            double kab = exp(-aa * ab * AB2 / ap);
            double cab = fabs(pcn[a] * pcn[b]);
            double R = orc_pair_extent(cab, kab, pl[a], pl[b], sqrt(dA2), sqrt(dB2), ap, tau);
            if (R < 0) continue;
            int lev = 0;
            for (int k = nlev - 1; k >= 0; --k)
              if (Ek[k] >= rel * ap) { lev = k; break; }
            if (n < cap) {
              out_ab[2 * n] = a;
              out_ab[2 * n + 1] = b;
              for (int d = 0; d < 3; ++d) {
                double f = 0.0;
                for (int c = 0; c < 3; ++c) f += rec[3 * d + c] * P[c];
                double Nd = (double)mesh[3 * lev + d];
                out_img[3 * n + d] = nn[d];
                out_lo[3 * n + d] = (int)ceil((f - R * blen[d]) * Nd);
                out_hi[3 * n + d] = (int)floor((f + R * blen[d]) * Nd);
              }
              out_lev[n] = lev;
              out_R[n] = R;
            }
            ++n;
          }
    }
  }
  return n;
}

static inline long orc_wrap(long i, long n) {
  long r = i % n;
  return r < 0 ? r + n : r;
}

typedef struct {
  int a, b, la, lb, na, nb, lev;
  int comp_a[ORC_MAXCART][3], comp_b[ORC_MAXCART][3];
  double A[3], B[3];
  double aa, ab, cna, cnb, w;
  long aoa, aob;
  int lo[3], hi[3];
} orc_pair_t;

static void orc_load_pair(orc_pair_t* q, long p, const int* ab, const int* img, const int* lev,
                          const int* lo, const int* hi, const double* pc, const int* pl,
                          const double* pal, const double* pcn, const long* pao,
                          const double* lat) {
  q->a = ab[2 * p];
  q->b = ab[2 * p + 1];
  q->la = pl[q->a];
  q->lb = pl[q->b];
  q->na = orc_cart(q->la, q->comp_a);
  q->nb = orc_cart(q->lb, q->comp_b);
  for (int d = 0; d < 3; ++d) {
    q->A[d] = pc[3 * q->a + d];
    q->B[d] = pc[3 * q->b + d] + (((double)img[3 * p] * lat[d] + (double)img[3 * p + 1] * lat[3 + d]) +
                                   (double)img[3 * p + 2] * lat[6 + d]);
    q->lo[d] = lo[3 * p + d];
    q->hi[d] = hi[3 * p + d];
  }
  q->aa = pal[q->a];
  q->ab = pal[q->b];
  q->cna = pcn[q->a];
  q->cnb = pcn[q->b];
  q->aoa = pao[q->a];
  q->aob = pao[q->b];
  q->lev = lev[p];
  /* a < b stands for both (a,b,T) and (b,a,-T), which fold onto the same cell
   * function; a == b keeps T and -T as separate pairs of weight 1. */
  q->w = (q->a < q->b) ? 2.0 : 1.0;
}

/* Value of the primitive Cartesian function at displacement (dx,dy,dz) from its
 * centre: cn * dx^ix dy^iy dz^iz * exp(-alpha r^2). */
static double orc_prim_val(double cn, const int* c, double alpha, double dx, double dy,
                           double dz) {
  return cn * orc_ipow(dx, c[0]) * orc_ipow(dy, c[1]) * orc_ipow(dz, c[2]) *
         exp(-alpha * (dx * dx + dy * dy + dz * dz));
}

/* Contribution of one pair at grid point r (absolute position), Eq. (rho_wrap):
 * w * sum_{mu in a, nu in b} D_mu,nu phi_mu(r) phi_nu(r - T). */
static double orc_pair_point_plain(const orc_pair_t* q, const double* D, long nao, double x,
                                   double y, double z) {
  double va[ORC_MAXCART], vb[ORC_MAXCART];
  for (int i = 0; i < q->na; ++i)
    va[i] = orc_prim_val(q->cna, q->comp_a[i], q->aa, x - q->A[0], y - q->A[1], z - q->A[2]);
  for (int j = 0; j < q->nb; ++j)
    vb[j] = orc_prim_val(q->cnb, q->comp_b[j], q->ab, x - q->B[0], y - q->B[1], z - q->B[2]);
  double s = 0.0;
  for (int i = 0; i < q->na; ++i)
    for (int j = 0; j < q->nb; ++j) s += D[(q->aoa + i) * nao + (q->aob + j)] * va[i] * vb[j];
  return q->w * s;
}

/* 1-D factors of one pair along dimension d over its box:
 * fa[k][t] = (x - A_d)^k exp(-aa (x - A_d)^2), fb likewise, x = (lo_d + t) * h_d. */
static void orc_pair_1d(const orc_pair_t* q, int d, double h, double* fa, double* fb, int n,
                        int lmax_a, int lmax_b) {
  for (int t = 0; t < n; ++t) {
    double x = (double)(q->lo[d] + t) * h;
    double ua = x - q->A[d], ub = x - q->B[d];
    double ea = exp(-q->aa * ua * ua), eb = exp(-q->ab * ub * ub);
    for (int k = 0; k <= lmax_a; ++k) fa[k * n + t] = orc_ipow(ua, k) * ea;
    for (int k = 0; k <= lmax_b; ++k) fb[k * n + t] = orc_ipow(ub, k) * eb;
  }
}

/*
 * eval_rho on every level: rho[level] += contributions of all pairs, each point of
 * the pair box folded into the cell (index mod N).  mode 0 = plain, 1 = separable.
 * grids: concatenated level grids, level k at grid_off[k], C order.
 * OpenMP over pairs with per-thread grids summed in thread order.
 */
void orc_collocate(int mode, long npairs, const int* ab, const int* img, const int* lev,
                   const int* lo, const int* hi, const double* pc, const int* pl,
                   const double* pal, const double* pcn, const long* pao, const double* lat,
                   const int* mesh, const long* grid_off, long grid_total, const double* D,
                   long nao, double* grids, int nthreads) {
  memset(grids, 0, sizeof(double) * grid_total);
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#else
  nthreads = 1;
#endif
  double* priv = (double*)calloc((size_t)nthreads * grid_total, sizeof(double));
#pragma omp parallel num_threads(nthreads)
  {
#ifdef _OPENMP
    int tid = omp_get_thread_num();
#else
    int tid = 0;
#endif
    double* g = priv + (size_t)tid * grid_total;
#pragma omp for schedule(static, 16)  /* fixed pair-to-thread map: deterministic sums */
    for (long p = 0; p < npairs; ++p) {
      orc_pair_t q;
      orc_load_pair(&q, p, ab, img, lev, lo, hi, pc, pl, pal, pcn, pao, lat);
      const int* N = mesh + 3 * q.lev;
      double H[3][3];
      orc_steps(lat, N, H);
      double h[3] = {H[0][0], H[1][1], H[2][2]};  /* separable mode: diagonal lattices */
      double* gl = g + grid_off[q.lev];
      int n[3] = {q.hi[0] - q.lo[0] + 1, q.hi[1] - q.lo[1] + 1, q.hi[2] - q.lo[2] + 1};
      if (n[0] <= 0 || n[1] <= 0 || n[2] <= 0) continue;
      if (mode == 0) {
        for (int i0 = q.lo[0]; i0 <= q.hi[0]; ++i0)
          for (int i1 = q.lo[1]; i1 <= q.hi[1]; ++i1)
            for (int i2 = q.lo[2]; i2 <= q.hi[2]; ++i2) {
              double r[3];
              orc_point(H, i0, i1, i2, r);
              double v = orc_pair_point_plain(&q, D, nao, r[0], r[1], r[2]);
              gl[(orc_wrap(i0, N[0]) * N[1] + orc_wrap(i1, N[1])) * N[2] + orc_wrap(i2, N[2])] += v;
            }
      } else {
        double* fa[3];
        double* fb[3];
        for (int d = 0; d < 3; ++d) {
          fa[d] = (double*)malloc(sizeof(double) * (q.la + 1) * n[d]);
          fb[d] = (double*)malloc(sizeof(double) * (q.lb + 1) * n[d]);
          orc_pair_1d(&q, d, h[d], fa[d], fb[d], n[d], q.la, q.lb);
        }
        double coef[ORC_MAXCART * ORC_MAXCART];
        for (int i = 0; i < q.na; ++i)
          for (int j = 0; j < q.nb; ++j)
            coef[i * q.nb + j] = q.w * q.cna * q.cnb * D[(q.aoa + i) * nao + (q.aob + j)];
        double s01[ORC_MAXCART * ORC_MAXCART];
        for (int t0 = 0; t0 < n[0]; ++t0) {
          long w0 = orc_wrap(q.lo[0] + t0, N[0]);
          for (int t1 = 0; t1 < n[1]; ++t1) {
            long w1 = orc_wrap(q.lo[1] + t1, N[1]);
            for (int i = 0; i < q.na; ++i)
              for (int j = 0; j < q.nb; ++j) {
                const int* ca = q.comp_a[i];
                const int* cb = q.comp_b[j];
                s01[i * q.nb + j] = coef[i * q.nb + j] * fa[0][ca[0] * n[0] + t0] *
                                    fb[0][cb[0] * n[0] + t0] * fa[1][ca[1] * n[1] + t1] *
                                    fb[1][cb[1] * n[1] + t1];
              }
            double* row = gl + (w0 * N[1] + w1) * N[2];
            for (int t2 = 0; t2 < n[2]; ++t2) {
              double v = 0.0;
              for (int i = 0; i < q.na; ++i)
                for (int j = 0; j < q.nb; ++j)
                  v += s01[i * q.nb + j] * fa[2][q.comp_a[i][2] * n[2] + t2] *
                       fb[2][q.comp_b[j][2] * n[2] + t2];
              row[orc_wrap(q.lo[2] + t2, N[2])] += v;
            }
          }
        }
        for (int d = 0; d < 3; ++d) {
          free(fa[d]);
          free(fb[d]);
        }
      }
    }
  }
  for (int t = 0; t < nthreads; ++t) {
    const double* g = priv + (size_t)t * grid_total;
    for (long i = 0; i < grid_total; ++i) grids[i] += g[i];
  }
  free(priv);
}

/* d/dC of u^i exp(-alpha u^2) with u = x - C, divided by exp(-alpha u^2):
 * -i u^(i-1) + 2 alpha u^(i+1). */
static double orc_dpoly(double u, int i, double alpha) {
  double t = 2.0 * alpha * orc_ipow(u, i + 1);
  if (i > 0) t -= (double)i * orc_ipow(u, i - 1);
  return t;
}

/*
 * Per-pair integrals of the level potential, Eq. (J_wrap) with the level weight
 * Omega/N_k:  X_p[i][j] = (Omega/N_k) sum_{r in box} v_k(r mod N) phi_i^a(r) phi_j^b(r - T),
 * stored at xout + xoff[p] (na*nb values, row i = component of a).  When
 * grad_D is non-NULL the same loop instead forms the Algorithm-3 gradient
 * contraction and stores 6 values per pair at xout + 6p:
 *   w * (Omega/N_k) sum_r v sum_ij D_ij [d phi_i^a / dA] phi_j^b   (3, atom of a)
 *   w * (Omega/N_k) sum_r v sum_ij D_ij phi_i^a [d phi_j^b / dB]   (3, atom of b)
 * with d/dA_x of (x-A)^i exp(-a (x-A)^2) = -i (x-A)^(i-1) e + 2 a (x-A)^(i+1) e.
 * Only the pairs listed in `sel` (or all when sel is NULL) are evaluated.
 */
void orc_integrate(long npairs, const long* sel, long nsel, const int* ab, const int* img,
                   const int* lev, const int* lo, const int* hi, const double* pc,
                   const int* pl, const double* pal, const double* pcn, const long* pao,
                   const double* lat, const int* mesh, const long* grid_off, const double* v,
                   const double* grad_D, long nao, const long* xoff, double* xout,
                   int nthreads) {
  long count = sel ? nsel : npairs;
  double omega = orc_volume(lat);
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#endif
#pragma omp parallel for schedule(dynamic, 8) num_threads(nthreads > 0 ? nthreads : 1)
  for (long s = 0; s < count; ++s) {
    long p = sel ? sel[s] : s;
    orc_pair_t q;
    orc_load_pair(&q, p, ab, img, lev, lo, hi, pc, pl, pal, pcn, pao, lat);
    const int* N = mesh + 3 * q.lev;
    double H[3][3];
    orc_steps(lat, N, H);
    double wgt = omega / ((double)N[0] * N[1] * N[2]);
    const double* vl = v + grid_off[q.lev];
    double X[ORC_MAXCART * ORC_MAXCART];
    double G[6] = {0, 0, 0, 0, 0, 0};
    memset(X, 0, sizeof(X));
    for (int i0 = q.lo[0]; i0 <= q.hi[0]; ++i0)
      for (int i1 = q.lo[1]; i1 <= q.hi[1]; ++i1)
        for (int i2 = q.lo[2]; i2 <= q.hi[2]; ++i2) {
          double r[3];
          orc_point(H, i0, i1, i2, r);
          double x = r[0], y = r[1], z = r[2];
          double vr = vl[(orc_wrap(i0, N[0]) * N[1] + orc_wrap(i1, N[1])) * N[2] +
                         orc_wrap(i2, N[2])];
          double ra[3] = {x - q.A[0], y - q.A[1], z - q.A[2]};
          double rb[3] = {x - q.B[0], y - q.B[1], z - q.B[2]};
          double ea = exp(-q.aa * (ra[0] * ra[0] + ra[1] * ra[1] + ra[2] * ra[2]));
          double eb = exp(-q.ab * (rb[0] * rb[0] + rb[1] * rb[1] + rb[2] * rb[2]));
          double va[ORC_MAXCART], vb[ORC_MAXCART];
          double dva[ORC_MAXCART][3], dvb[ORC_MAXCART][3];
          for (int i = 0; i < q.na; ++i) {
            const int* c = q.comp_a[i];
            double px = orc_ipow(ra[0], c[0]), py = orc_ipow(ra[1], c[1]), pz = orc_ipow(ra[2], c[2]);
            va[i] = q.cna * px * py * pz * ea;
            if (grad_D) {
              dva[i][0] = q.cna * orc_dpoly(ra[0], c[0], q.aa) * py * pz * ea;
              dva[i][1] = q.cna * px * orc_dpoly(ra[1], c[1], q.aa) * pz * ea;
              dva[i][2] = q.cna * px * py * orc_dpoly(ra[2], c[2], q.aa) * ea;
            }
          }
          for (int j = 0; j < q.nb; ++j) {
            const int* c = q.comp_b[j];
            double px = orc_ipow(rb[0], c[0]), py = orc_ipow(rb[1], c[1]), pz = orc_ipow(rb[2], c[2]);
            vb[j] = q.cnb * px * py * pz * eb;
            if (grad_D) {
              dvb[j][0] = q.cnb * orc_dpoly(rb[0], c[0], q.ab) * py * pz * eb;
              dvb[j][1] = q.cnb * px * orc_dpoly(rb[1], c[1], q.ab) * pz * eb;
              dvb[j][2] = q.cnb * px * py * orc_dpoly(rb[2], c[2], q.ab) * eb;
            }
          }
          if (!grad_D) {
            for (int i = 0; i < q.na; ++i)
              for (int j = 0; j < q.nb; ++j) X[i * q.nb + j] += vr * va[i] * vb[j];
          } else {
            for (int i = 0; i < q.na; ++i)
              for (int j = 0; j < q.nb; ++j) {
                double dij = grad_D[(q.aoa + i) * nao + (q.aob + j)] * vr;
                for (int d = 0; d < 3; ++d) {
                  G[d] += dij * dva[i][d] * vb[j];
                  G[3 + d] += dij * va[i] * dvb[j][d];
                }
              }
          }
        }
    if (!grad_D) {
      double* xo = xout + xoff[p];
      for (int k = 0; k < q.na * q.nb; ++k) xo[k] = wgt * X[k];
    } else {
      for (int d = 0; d < 6; ++d) xout[6 * s + d] = q.w * wgt * G[d];
    }
  }
}

/*
 * rho of one level at a list of grid points (indices in [0, N)), summing every
 * pair of that level whose box covers the point or one of its periodic copies.
 * Used to check large cells point by point.
 */
void orc_rho_points(long npairs, const int* ab, const int* img, const int* lev,
                    const int* lo, const int* hi, const double* pc, const int* pl,
                    const double* pal, const double* pcn, const long* pao, const double* lat,
                    const int* mesh, int level, long npts, const int* pts, const double* D,
                    long nao, double* out, int nthreads) {
  const int* N = mesh + 3 * level;
  double H[3][3];
  orc_steps(lat, N, H);
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads > 0 ? nthreads : 1)
  for (long s = 0; s < npts; ++s) {
    double acc = 0.0;
    for (long p = 0; p < npairs; ++p) {
      if (lev[p] != level) continue;
      int k0[3], k1[3];
      int skip = 0;
      for (int d = 0; d < 3; ++d) {
        /* unwrapped copies i = pts + k N inside [lo, hi] */
        long l0 = lo[3 * p + d], h0 = hi[3 * p + d], x = pts[3 * s + d];
        double a = (double)(l0 - x) / N[d], b = (double)(h0 - x) / N[d];
        k0[d] = (int)ceil(a);
        k1[d] = (int)floor(b);
        if (k0[d] > k1[d]) skip = 1;
      }
      if (skip) continue;
      orc_pair_t q;
      orc_load_pair(&q, p, ab, img, lev, lo, hi, pc, pl, pal, pcn, pao, lat);
      for (int a0 = k0[0]; a0 <= k1[0]; ++a0)
        for (int a1 = k0[1]; a1 <= k1[1]; ++a1)
          for (int a2 = k0[2]; a2 <= k1[2]; ++a2) {
            long i0 = pts[3 * s] + (long)a0 * N[0];
            long i1 = pts[3 * s + 1] + (long)a1 * N[1];
            long i2 = pts[3 * s + 2] + (long)a2 * N[2];
            double r[3];
            orc_point(H, i0, i1, i2, r);
            acc += orc_pair_point_plain(&q, D, nao, r[0], r[1], r[2]);
          }
    }
    out[s] = acc;
  }
}

/* ------------------------------------------------------------------------------------
 * Kinetic energy density of meta-GGA functionals (Sec. II, meta-GGA):
 *   tau(r) = (1/2) sum_mu,nu D_mu,nu grad phi_mu(r) . grad phi_nu(r),
 * and the matching Fock term (1/2) int v_tau grad phi_mu . grad phi_nu (Eq. J_metaGGA).
 * Per dimension, a primitive factor is f(u) = u^c exp(-alpha u^2), u = x - C, with
 *   f'(u)  = (c u^(c-1) - 2 alpha u^(c+1)) exp(-alpha u^2)
 *   f''(u) = (c (c-1) u^(c-2) - 2 alpha (2c+1) u^c + 4 alpha^2 u^(c+2)) exp(-alpha u^2).
 * Everything is evaluated point by point (no factorisation, no recursion).
 */
static double orc_f0(double u, int c) { return orc_ipow(u, c); }
static double orc_f1(double u, int c, double a) {
  double t = -2.0 * a * orc_ipow(u, c + 1);
  if (c > 0) t += (double)c * orc_ipow(u, c - 1);
  return t;
}
static double orc_f2(double u, int c, double a) {
  double t = -2.0 * a * (2.0 * c + 1.0) * orc_ipow(u, c) + 4.0 * a * a * orc_ipow(u, c + 2);
  if (c > 1) t += (double)c * (c - 1) * orc_ipow(u, c - 2);
  return t;
}

/* value, gradient and Hessian (xx, yy, zz, xy, xz, yz) of cn u^c exp(-alpha |u|^2) */
static void orc_prim_derivs(double cn, const int* c, double alpha, const double* u, double* val,
                            double* g, double* H) {
  double e = cn * exp(-alpha * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]));
  double f0[3], f1[3], f2[3];
  for (int d = 0; d < 3; ++d) {
    f0[d] = orc_f0(u[d], c[d]);
    f1[d] = orc_f1(u[d], c[d], alpha);
    f2[d] = orc_f2(u[d], c[d], alpha);
  }
  *val = e * f0[0] * f0[1] * f0[2];
  g[0] = e * f1[0] * f0[1] * f0[2];
  g[1] = e * f0[0] * f1[1] * f0[2];
  g[2] = e * f0[0] * f0[1] * f1[2];
  if (H) {
    H[0] = e * f2[0] * f0[1] * f0[2];
    H[1] = e * f0[0] * f2[1] * f0[2];
    H[2] = e * f0[0] * f0[1] * f2[2];
    H[3] = e * f1[0] * f1[1] * f0[2];
    H[4] = e * f1[0] * f0[1] * f1[2];
    H[5] = e * f0[0] * f1[1] * f1[2];
  }
}

static int orc_hidx(int d, int e) {
  if (d == e) return d;
  if (d > e) { int t = d; d = e; e = t; }
  return d == 0 ? (e == 1 ? 3 : 4) : 5;
}

/* tau on every level: w (1/2) sum_ij D_ij grad phi_i^a . grad phi_j^b at every point of
 * each pair box, folded into the cell; OpenMP over pairs, per-thread grids summed in
 * thread order. */
void orc_collocate_tau(long npairs, const int* ab, const int* img, const int* lev,
                       const int* lo, const int* hi, const double* pc, const int* pl,
                       const double* pal, const double* pcn, const long* pao, const double* lat,
                       const int* mesh, const long* grid_off, long grid_total, const double* D,
                       long nao, double* grids, int nthreads) {
  memset(grids, 0, sizeof(double) * grid_total);
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#else
  nthreads = 1;
#endif
  double* priv = (double*)calloc((size_t)nthreads * grid_total, sizeof(double));
#pragma omp parallel num_threads(nthreads)
  {
#ifdef _OPENMP
    int tid = omp_get_thread_num();
#else
    int tid = 0;
#endif
    double* g = priv + (size_t)tid * grid_total;
#pragma omp for schedule(static, 16)  /* fixed pair-to-thread map: deterministic sums */
    for (long p = 0; p < npairs; ++p) {
      orc_pair_t q;
      orc_load_pair(&q, p, ab, img, lev, lo, hi, pc, pl, pal, pcn, pao, lat);
      const int* N = mesh + 3 * q.lev;
      double H[3][3];
      orc_steps(lat, N, H);
      double* gl = g + grid_off[q.lev];
      for (int i0 = q.lo[0]; i0 <= q.hi[0]; ++i0)
        for (int i1 = q.lo[1]; i1 <= q.hi[1]; ++i1)
          for (int i2 = q.lo[2]; i2 <= q.hi[2]; ++i2) {
            double r[3];
            orc_point(H, i0, i1, i2, r);
            double ua[3], ub[3], va, vb, ga[ORC_MAXCART][3], gb[ORC_MAXCART][3];
            for (int d = 0; d < 3; ++d) {
              ua[d] = r[d] - q.A[d];
              ub[d] = r[d] - q.B[d];
            }
            for (int i = 0; i < q.na; ++i) orc_prim_derivs(q.cna, q.comp_a[i], q.aa, ua, &va, ga[i], NULL);
            for (int j = 0; j < q.nb; ++j) orc_prim_derivs(q.cnb, q.comp_b[j], q.ab, ub, &vb, gb[j], NULL);
            double s = 0.0;
            for (int i = 0; i < q.na; ++i)
              for (int j = 0; j < q.nb; ++j)
                s += D[(q.aoa + i) * nao + (q.aob + j)] *
                     (ga[i][0] * gb[j][0] + ga[i][1] * gb[j][1] + ga[i][2] * gb[j][2]);
            gl[(orc_wrap(i0, N[0]) * N[1] + orc_wrap(i1, N[1])) * N[2] + orc_wrap(i2, N[2])] +=
                0.5 * q.w * s;
          }
    }
  }
  for (int t = 0; t < nthreads; ++t) {
    const double* g = priv + (size_t)t * grid_total;
    for (long i = 0; i < grid_total; ++i) grids[i] += g[i];
  }
  free(priv);
}

/* Per-pair Fock blocks of a kinetic-energy-density potential (Eq. J_metaGGA, level
 * weight Omega/N_k): X_p[i][j] = (Omega/N_k) sum_r v(r) (1/2) grad phi_i^a . grad phi_j^b.
 * With grad_D, the nuclear gradient of sum_ij D_ij X_ij instead (6 values per pair):
 * d/dA of grad phi^a is minus the Hessian of phi^a in x, so
 *   dA_d = -w (Omega/N_k) sum_r v (1/2) sum_ij D_ij sum_e H^a_de grad_e phi^b, and likewise B. */
void orc_integrate_tau(long npairs, const long* sel, long nsel, const int* ab, const int* img,
                       const int* lev, const int* lo, const int* hi, const double* pc,
                       const int* pl, const double* pal, const double* pcn, const long* pao,
                       const double* lat, const int* mesh, const long* grid_off, const double* v,
                       const double* grad_D, long nao, const long* xoff, double* xout,
                       int nthreads) {
  long count = sel ? nsel : npairs;
  double omega = orc_volume(lat);
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#endif
#pragma omp parallel for schedule(dynamic, 8) num_threads(nthreads > 0 ? nthreads : 1)
  for (long s = 0; s < count; ++s) {
    long p = sel ? sel[s] : s;
    orc_pair_t q;
    orc_load_pair(&q, p, ab, img, lev, lo, hi, pc, pl, pal, pcn, pao, lat);
    const int* N = mesh + 3 * q.lev;
    double H[3][3];
    orc_steps(lat, N, H);
    double wgt = omega / ((double)N[0] * N[1] * N[2]);
    const double* vl = v + grid_off[q.lev];
    double X[ORC_MAXCART * ORC_MAXCART];
    double G[6] = {0, 0, 0, 0, 0, 0};
    memset(X, 0, sizeof(X));
    for (int i0 = q.lo[0]; i0 <= q.hi[0]; ++i0)
      for (int i1 = q.lo[1]; i1 <= q.hi[1]; ++i1)
        for (int i2 = q.lo[2]; i2 <= q.hi[2]; ++i2) {
          double r[3];
          orc_point(H, i0, i1, i2, r);
          double vr = vl[(orc_wrap(i0, N[0]) * N[1] + orc_wrap(i1, N[1])) * N[2] + orc_wrap(i2, N[2])];
          double ua[3], ub[3], va, vb;
          double ga[ORC_MAXCART][3], gb[ORC_MAXCART][3], Ha[ORC_MAXCART][6], Hb[ORC_MAXCART][6];
          for (int d = 0; d < 3; ++d) {
            ua[d] = r[d] - q.A[d];
            ub[d] = r[d] - q.B[d];
          }
          for (int i = 0; i < q.na; ++i)
            orc_prim_derivs(q.cna, q.comp_a[i], q.aa, ua, &va, ga[i], grad_D ? Ha[i] : NULL);
          for (int j = 0; j < q.nb; ++j)
            orc_prim_derivs(q.cnb, q.comp_b[j], q.ab, ub, &vb, gb[j], grad_D ? Hb[j] : NULL);
          if (!grad_D) {
            for (int i = 0; i < q.na; ++i)
              for (int j = 0; j < q.nb; ++j)
                X[i * q.nb + j] += vr * 0.5 *
                    (ga[i][0] * gb[j][0] + ga[i][1] * gb[j][1] + ga[i][2] * gb[j][2]);
          } else {
            for (int i = 0; i < q.na; ++i)
              for (int j = 0; j < q.nb; ++j) {
                double dij = grad_D[(q.aoa + i) * nao + (q.aob + j)] * vr * 0.5;
                for (int d = 0; d < 3; ++d) {
                  double sa = 0.0, sb = 0.0;
                  for (int e = 0; e < 3; ++e) {
                    sa += Ha[i][orc_hidx(d, e)] * gb[j][e];
                    sb += ga[i][e] * Hb[j][orc_hidx(d, e)];
                  }
                  G[d] -= dij * sa;
                  G[3 + d] -= dij * sb;
                }
              }
          }
        }
    if (!grad_D) {
      double* xo = xout + xoff[p];
      for (int k = 0; k < q.na * q.nb; ++k) xo[k] = wgt * X[k];
    } else {
      for (int d = 0; d < 6; ++d) xout[6 * s + d] = q.w * wgt * G[d];
    }
  }
}
