// Sub-box task lists built on the device at commit: the mapping of screened pairs to grid
// blocks of the paper's appendix (Algorithm 5: count the pairs of every block, offsets by
// a prefix sum, fill the per-block lists), here with one task per (pair, sub-box,
// periodic copy) as the grid kernels walk them.
//
// The host part of the plan only counted each pair's tasks (toff: prefix sums in pair
// order).  Task t of pair p is its r-th segment triple (x segment outer, z inner), so the
// tasks in index order are the host builder's enumeration.  Each task gets the key of its
// sub-box; a stable radix sort by key then gives every sub-box its tasks in pair order,
// the order build_tasks produces on the host, and the records are written at their
// sorted positions.  The work list is ordered on the host from the sub-box offsets.
#include <cub/device/device_radix_sort.cuh>

#include <algorithm>
#include <string>
#include <vector>

#include "gpw_internal.h"
#include "plan_host.h"

namespace gpw {
namespace {

struct TaskGeom {
  int T[3];
  int C[3];  // z windows of C[d] T[d] points (C = 1: plain tiling)
  int N[GPW_MAX_LEVELS][3];
  int nsb[GPW_MAX_LEVELS][3];
  long long sub_base[GPW_MAX_LEVELS];
  long long np, nent, nsub;
  int xr;
  int integ;  // integration records: offset of the task's W tensor in r1.w
  int prune;  // GPW_FAST_BLOCK_PRUNE on this list: tasks beyond R_p get the key nsub
  int ortho;
  double blen[3];
  double lam;
};

// block_beyond (plan_host.h) with every rounding spelt out, so that it decides as the host
// builder does: the task box [a_d, b_d] lies wholly farther than R_p from P
__device__ __forceinline__ bool block_beyond_d(const PairQ q, const long long* a,
                                               const long long* b, const int* N,
                                               const double* blen, int ortho, double lam) {
  const double fp[3] = {q.x, q.y, q.z};
  double f[3], s[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double fa = __ddiv_rn((double)a[d], (double)N[d]);
    const double fb = __ddiv_rn((double)b[d], (double)N[d]);
    f[d] = fp[d] < fa ? __dsub_rn(fa, fp[d]) : (fp[d] > fb ? __dsub_rn(fp[d], fb) : 0.0);
    s[d] = __ddiv_rn(f[d], blen[d]);
  }
  const double R2 = __dmul_rn(q.w, q.w);
  if (ortho) {
    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(s[0], s[0]), __dmul_rn(s[1], s[1])),
                                __dmul_rn(s[2], s[2]));
    return r2 > R2;
  }
  if (fmax(s[0], fmax(s[1], s[2])) > q.w) return true;
  const double f2 = __dadd_rn(__dadd_rn(__dmul_rn(f[0], f[0]), __dmul_rn(f[1], f[1])),
                              __dmul_rn(f[2], f[2]));
  return __dmul_rn(lam, f2) > R2;
}

__host__ __device__ __forceinline__ long long floordiv_d(long long a, long long b) {
  long long q = a / b;
  if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
  return q;
}

// Segments of a pair box along an axis of N points cut into nsb sub-boxes of T, whose
// blocks see windows of C T points from their sub-box start (C = 1: plain tiling): a
// segment starts at the box start or where the previous one ended, belongs to the
// sub-box it starts in and ends with that sub-box's window (clipped at the period).  In
// the box's first period (q0) segments start in sub-boxes j0, j0 + C, ...; in later ones
// in 0, C, 2C, ...
struct AxisSeg {
  long long q0, j0, nfirst, per;
};

__host__ __device__ __forceinline__ AxisSeg axis_seg(int lo, int N, int T, int nsb, int C) {
  AxisSeg a;
  a.q0 = floordiv_d(lo, N);
  a.j0 = ((long long)lo - a.q0 * N) / T;
  a.nfirst = (nsb - a.j0 + C - 1) / C;
  a.per = (nsb + C - 1) / C;
  return a;
}

// index of the segment holding grid index i >= lo
__host__ __device__ __forceinline__ long long seg_of(long long i, const AxisSeg& a, int N, int T, int C) {
  const long long q = floordiv_d(i, N);
  const long long j = (i - q * N) / T;
  if (q == a.q0) return (j - a.j0) / C;
  return a.nfirst + (q - a.q0 - 1) * a.per + j / C;
}

struct SegD {
  int m, u, t;
  long long j;
};

// segment k of the pair box [lo, lo + n - 1] along axis d: the packed record fields of
// build_tasks (length m, start u inside the sub-box, start t inside the pair box | n << 16)
// and the sub-box coordinate j
__host__ __device__ __forceinline__ SegD segment(int lo, int n, int N, int T, int nsb, int C,
                                                 long long k, int d) {
  const long long hi = (long long)lo + n - 1;
  const AxisSeg as = axis_seg(lo, N, T, nsb, C);
  long long q, j;
  if (k < as.nfirst) {
    q = as.q0;
    j = as.j0 + k * C;
  } else {
    const long long r = k - as.nfirst;
    q = as.q0 + 1 + r / as.per;
    j = (r % as.per) * C;
  }
  const long long s0 = j * T;
  const long long ext = std::min<long long>((long long)C * T, (long long)N - s0);
  const long long o = q * N + s0;
  const long long a = std::max<long long>(lo, o);
  const long long b = std::min<long long>(hi, o + ext - 1);
  SegD r;
  r.m = (int)(b - a + 1) << (8 * d);
  r.u = (int)(a - o) << (8 * d);
  r.t = (int)(a - lo) | (n << 16);
  r.j = j;
  return r;
}

__host__ __device__ __forceinline__ long long nseg_d(int lo, int n, int N, int T, int nsb, int C) {
  const AxisSeg as = axis_seg(lo, N, T, nsb, C);
  return seg_of((long long)lo + n - 1, as, N, T, C) + 1;
}

// pair of task t: the last p with toff[p] <= t
__host__ __device__ __forceinline__ long long pair_of(const long long* __restrict__ toff, long long np,
                                             long long t) {
  long long lo = 0, hi = np - 1;
  while (lo < hi) {
    const long long mid = (lo + hi + 1) >> 1;
    if (toff[mid] <= t)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

struct TaskPos {
  long long p, r, k0, k1, k2, ns1, ns2;
  int4 a, b;  // hot_a {lo, L}, hot_b {n, level}
};

__host__ __device__ __forceinline__ TaskPos locate(const TaskGeom& G, const int4* __restrict__ hot_a,
                                          const int4* __restrict__ hot_b,
                                          const long long* __restrict__ toff, long long t) {
  TaskPos q;
  q.p = pair_of(toff, G.np, t);
  q.r = t - toff[q.p];
  q.a = hot_a[q.p];
  q.b = hot_b[q.p];
  const int lev = q.b.w;
  q.ns1 = nseg_d(q.a.y, q.b.y, G.N[lev][1], G.T[1], G.nsb[lev][1], G.C[1]);
  q.ns2 = nseg_d(q.a.z, q.b.z, G.N[lev][2], G.T[2], G.nsb[lev][2], G.C[2]);
  q.k2 = q.r % q.ns2;
  q.k1 = (q.r / q.ns2) % q.ns1;
  q.k0 = q.r / (q.ns1 * q.ns2);
  return q;
}

// sub-box key of every task, and the identity permutation; a task left out by the block
// screening gets the key nsub, past every sub-box, so the sort puts it after them all
__global__ void task_keys_kernel(TaskGeom G, const int4* __restrict__ hot_a,
                                 const int4* __restrict__ hot_b,
                                 const long long* __restrict__ toff,
                                 const PairQ* __restrict__ pq, unsigned* __restrict__ keys,
                                 unsigned* __restrict__ vals) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < G.nent;
       t += (long long)gridDim.x * blockDim.x) {
    const TaskPos q = locate(G, hot_a, hot_b, toff, t);
    const int lev = q.b.w;
    const SegD s0 = segment(q.a.x, q.b.x, G.N[lev][0], G.T[0], G.nsb[lev][0], G.C[0], q.k0, 0);
    const SegD s1 = segment(q.a.y, q.b.y, G.N[lev][1], G.T[1], G.nsb[lev][1], G.C[1], q.k1, 1);
    const SegD s2 = segment(q.a.z, q.b.z, G.N[lev][2], G.T[2], G.nsb[lev][2], G.C[2], q.k2, 2);
    unsigned key = (unsigned)(G.sub_base[lev] + (s0.j * G.nsb[lev][1] + s1.j) * G.nsb[lev][2] + s2.j);
    if (G.prune) {
      // the task box: from its start in the pair box (t) and its length (m)
      const long long a[3] = {(long long)q.a.x + (s0.t & 0xffff), (long long)q.a.y + (s1.t & 0xffff),
                              (long long)q.a.z + (s2.t & 0xffff)};
      const long long b[3] = {a[0] + (s0.m & 255) - 1, a[1] + ((s1.m >> 8) & 255) - 1,
                              a[2] + ((s2.m >> 16) & 255) - 1};
      if (block_beyond_d(pq[q.p], a, b, G.N[lev], G.blen, G.ortho, G.lam)) key = (unsigned)G.nsub;
    }
    keys[t] = key;
    vals[t] = (unsigned)t;
  }
}

// the two int4 records of the task at sorted position s
__global__ void task_fill_kernel(TaskGeom G, const int4* __restrict__ hot_a,
                                 const int4* __restrict__ hot_b,
                                 const long long* __restrict__ toff,
                                 const unsigned* __restrict__ perm, int4* __restrict__ task) {
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < G.nent;
       s += (long long)gridDim.x * blockDim.x) {
    const TaskPos q = locate(G, hot_a, hot_b, toff, (long long)perm[s]);
    const int lev = q.b.w, L = q.a.w;
    const SegD s0 = segment(q.a.x, q.b.x, G.N[lev][0], G.T[0], G.nsb[lev][0], G.C[0], q.k0, 0);
    const SegD s1 = segment(q.a.y, q.b.y, G.N[lev][1], G.T[1], G.nsb[lev][1], G.C[1], q.k1, 1);
    const SegD s2 = segment(q.a.z, q.b.z, G.N[lev][2], G.T[2], G.nsb[lev][2], G.C[2], q.k2, 2);
    int w = 0;
    if (G.integ) {
      const long long S = nc2(L + 1 + G.xr);
      const long long ns12 = q.ns1 * q.ns2, r12 = q.k1 * q.ns2 + q.k2;
      const long long tt0 = s0.t & 0xffff, m0 = s0.m & 255;
      w = (int)(S * (tt0 * ns12 + r12 * m0));
    }
    task[2 * s] = make_int4((int)q.p, s0.m | s1.m | s2.m | (L << 24), s0.u | s1.u | s2.u, (int)q.r);
    task[2 * s + 1] = make_int4(s0.t, s1.t, s2.t, w);
  }
}

// CSR offsets from the sorted keys: sub_off[k] = first sorted position with key >= k
__global__ void sub_off_kernel(long long nent, long long nsub, const unsigned* __restrict__ keys,
                               long long* __restrict__ sub_off) {
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s <= nent;
       s += (long long)gridDim.x * blockDim.x) {
    const long long kp = s == 0 ? -1 : (long long)keys[s - 1];
    const long long kc = s == nent ? nsub : (long long)keys[s];
    for (long long k = kp + 1; k <= kc; ++k) sub_off[k] = s;
  }
}

#define GPW_TCK(x)                                                                  \
  do {                                                                              \
    cudaError_t e_ = (x);                                                           \
    if (e_ != cudaSuccess) {                                                        \
      set_error(std::string("device task lists: ") + #x + ": " + cudaGetErrorString(e_)); \
      return e_ == cudaErrorMemoryAllocation ? GPW_ENOMEM : GPW_ECUDA;              \
    }                                                                               \
  } while (0)

int key_bits(long long nsub) {
  int b = 1;
  while (b < 32 && (1LL << b) <= nsub) ++b;
  return b;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// sort temp bytes of cub for n items (no device work)
int sort_temp_bytes(long long n, int bits, size_t* out) {
  cub::DoubleBuffer<unsigned> k(nullptr, nullptr), v(nullptr, nullptr);
  *out = 0;
  if (n <= 0) return GPW_OK;
  GPW_TCK(cub::DeviceRadixSort::SortPairs(nullptr, *out, k, v, (int)n, 0, bits));
  return GPW_OK;
}

TaskGeom geom(const Plan& P, bool integ) {
  TaskGeom G{};
  const LevelInfo* lev = integ ? P.lev_i : P.lev;
  const int* T = integ ? P.tile_i : P.tile;
  for (int d = 0; d < 3; ++d) {
    G.T[d] = T[d];
    G.C[d] = 1;
  }
  if (integ) G.C[2] = P.zwin_i / P.tile_i[2];
  for (int k = 0; k < P.nlev; ++k) {
    for (int d = 0; d < 3; ++d) {
      G.N[k][d] = lev[k].N[d];
      G.nsb[k][d] = lev[k].nsb[d];
    }
    G.sub_base[k] = lev[k].sub_base;
  }
  G.np = P.npairs;
  G.nent = integ ? P.nent_i : P.nent;
  G.nsub = integ ? P.nsub_i : P.nsub_total;
  G.xr = P.xr;
  G.integ = integ ? 1 : 0;
  G.prune = (P.prune && !integ) ? 1 : 0;
  G.ortho = P.skew ? 0 : 1;
  for (int d = 0; d < 3; ++d) G.blen[d] = P.prune_blen[d];
  G.lam = P.prune_lam;
  return G;
}

}  // namespace

long long task_sort_bytes(const Plan& P) {
  // four key/value arrays of the larger list; the radix sort's own temp is bounded by a
  // few histograms per pass (checked at commit, where the exact figure is known)
  const long long n = std::max(P.nent, P.nent_i);
  return n > 0 ? 16 * n + (8 << 20) : 0;
}

int build_tasks_device(Plan* P, HostArrays& H, cudaStream_t s, long long* bytes) {
  DeviceArrays& d = P->d;
  const long long np = P->npairs;
  if (P->nent >= INT32_MAX || P->nent_i >= INT32_MAX || P->nsub_total >= INT32_MAX ||
      P->nsub_i >= INT32_MAX) {
    set_error("gpw_plan: more than 2^31 - 1 tasks or sub-boxes in one list");
    return GPW_ERANGE;
  }
  // scratch: the toff arrays, two key and two value buffers and the sort temp; in the
  // part buffer (W tensors, not live before the first integration) when it is large
  // enough, else allocated for the build and released after it
  const long long nmax = std::max(P->nent, P->nent_i);
  size_t temp = 0, temp_i = 0;
  int rc = sort_temp_bytes(P->nent, key_bits(P->nsub_total), &temp);
  if (!rc) rc = sort_temp_bytes(P->nent_i, key_bits(P->nsub_i), &temp_i);
  if (rc) return rc;
  temp = std::max(temp, temp_i);
  const size_t toff_b = align256(sizeof(long long) * (size_t)(np + 1));
  const size_t kv_b = align256(sizeof(unsigned) * (size_t)std::max<long long>(nmax, 1));
  const size_t need = 2 * toff_b + 4 * kv_b + align256(std::max<size_t>(temp, 1));
  char* scratch = nullptr;
  bool own = false;
  if ((size_t)P->part_total * sizeof(double) >= need) {
    scratch = reinterpret_cast<char*>(d.part);
  } else {
    GPW_TCK(cudaMallocAsync((void**)&scratch, need, s));
    own = true;
  }
  long long* toff_c = reinterpret_cast<long long*>(scratch);
  long long* toff_i = reinterpret_cast<long long*>(scratch + toff_b);
  unsigned* kv[4];
  for (int i = 0; i < 4; ++i) kv[i] = reinterpret_cast<unsigned*>(scratch + 2 * toff_b + i * kv_b);
  void* tmp = scratch + 2 * toff_b + 4 * kv_b;
  int out = GPW_OK;
  PairQ* pq = nullptr;  // the block screening's per-pair data (fractional P, R_p)
  auto body = [&]() -> int {
    if (P->prune) {
      GPW_TCK(cudaMallocAsync((void**)&pq, sizeof(PairQ) * (size_t)std::max<long long>(np, 1), s));
      if (np > 0)
        GPW_TCK(cudaMemcpyAsync(pq, H.prune.data(), sizeof(PairQ) * (size_t)np,
                                cudaMemcpyHostToDevice, s));
    }
    GPW_TCK(cudaMemcpyAsync(toff_c, H.toff_c.data(), sizeof(long long) * (size_t)(np + 1),
                            cudaMemcpyHostToDevice, s));
    GPW_TCK(cudaMemcpyAsync(toff_i, H.toff_i.data(), sizeof(long long) * (size_t)(np + 1),
                            cudaMemcpyHostToDevice, s));
    for (int integ = 0; integ < 2; ++integ) {
      const TaskGeom G = geom(*P, integ != 0);
      int4** task = integ ? &d.task_i : &d.task_c;
      long long** sub = integ ? &d.sub_off_i : &d.sub_off_c;
      GPW_TCK(cudaMallocAsync((void**)task, sizeof(int4) * (size_t)std::max<long long>(2 * G.nent, 1), s));
      *bytes += (long long)(sizeof(int4) * (size_t)std::max<long long>(2 * G.nent, 1));
      GPW_TCK(cudaMallocAsync((void**)sub, sizeof(long long) * (size_t)(G.nsub + 1), s));
      *bytes += (long long)(sizeof(long long) * (size_t)(G.nsub + 1));
      const unsigned* sorted_keys = kv[0];
      if (G.nent > 0) {
        const long long* toff = integ ? toff_i : toff_c;
        const int threads = 256;
        const int blocks = (int)std::min<long long>((G.nent + threads - 1) / threads, 152 * 16);
        task_keys_kernel<<<blocks, threads, 0, s>>>(G, d.hot_a, d.hot_b, toff, pq, kv[0], kv[2]);
        GPW_TCK(cudaGetLastError());
        cub::DoubleBuffer<unsigned> keys(kv[0], kv[1]), vals(kv[2], kv[3]);
        size_t tb = temp;
        GPW_TCK(cub::DeviceRadixSort::SortPairs(tmp, tb, keys, vals, (int)G.nent, 0,
                                                key_bits(G.nsub), s));
        task_fill_kernel<<<blocks, threads, 0, s>>>(G, d.hot_a, d.hot_b, toff, vals.Current(), *task);
        GPW_TCK(cudaGetLastError());
        sorted_keys = keys.Current();
      }
      const int sblocks = (int)std::min<long long>((G.nent + 256) / 256, 152 * 16);
      sub_off_kernel<<<sblocks, 256, 0, s>>>(G.nent, G.nsub, sorted_keys, *sub);
      GPW_TCK(cudaGetLastError());
      // the next list reuses the key buffers: keep the order on the stream
    }
    // work lists on the host, from the sub-box offsets
    H.sub_off_c.resize((size_t)(P->nsub_total + 1));
    H.sub_off_i.resize((size_t)(P->nsub_i + 1));
    GPW_TCK(cudaMemcpyAsync(H.sub_off_c.data(), d.sub_off_c, sizeof(long long) * H.sub_off_c.size(),
                            cudaMemcpyDeviceToHost, s));
    GPW_TCK(cudaMemcpyAsync(H.sub_off_i.data(), d.sub_off_i, sizeof(long long) * H.sub_off_i.size(),
                            cudaMemcpyDeviceToHost, s));
    GPW_TCK(cudaStreamSynchronize(s));
    // the block screening's dropped tasks sit past the last sub-box's
    P->nent = H.sub_off_c[(size_t)P->nsub_total];
    int r = order_work(P->nlev, P->lev, H.sub_off_c, 0, &H.work_c, &P->nwork);
    if (!r) r = order_work(P->nlev, P->lev_i, H.sub_off_i, P->chunk_i, &H.work_i, &P->nwork_i);
    if (r) return r;
    for (int integ = 0; integ < 2; ++integ) {
      const std::vector<int4>& w = integ ? H.work_i : H.work_c;
      int4** dst = integ ? &d.work_i : &d.work_c;
      GPW_TCK(cudaMallocAsync((void**)dst, sizeof(int4) * std::max<size_t>(w.size(), 1), s));
      *bytes += (long long)(sizeof(int4) * std::max<size_t>(w.size(), 1));
      if (!w.empty())
        GPW_TCK(cudaMemcpyAsync(*dst, w.data(), sizeof(int4) * w.size(), cudaMemcpyHostToDevice, s));
    }
    return GPW_OK;
  };
  out = body();
  if (own) cudaFreeAsync(scratch, s);
  if (pq) cudaFreeAsync(pq, s);
  return out;
}

}  // namespace gpw
