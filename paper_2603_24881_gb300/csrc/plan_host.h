// Host staging arrays produced by build_host_plan and uploaded by gpw_plan.
#pragma once

#include <algorithm>
#include <vector>

#include "gpw_internal.h"

namespace gpw {

struct HostArrays {
  std::vector<int4> hot_a, hot_b, ids, ids2;
  std::vector<double> geo, cab;
  std::vector<long long> tab_off, coef_off, part_off, xt_off, yt_off;
  std::vector<int4> task_c, task_i;   // 2 int4 per task
  std::vector<long long> sub_off_c, sub_off_i;
  std::vector<long long> toff_c, toff_i;  // per-pair task prefix sums (device-built lists)
  std::vector<PairQ> prune;  // GPW_FAST_BLOCK_PRUNE: per pair {f_0(P), f_1(P), f_2(P), R_p}
  std::vector<double> mono_t;  // non-orthogonal cells: monomial transforms per level
  std::vector<int4> work_c, work_i;   // {plan slot, level, sub-box, tasks}
  std::vector<int4> groups;
  std::vector<long long> atom_off;
  std::vector<int> atom_list;
};

// Monomial transforms of a non-orthogonal cell (one block per level).
void build_mono_transforms(const Plan& P, std::vector<double>* out);

// Default integration chunk for nent tasks: max(kChunkMin, ceil(nent / kChunkDiv)).
long long default_chunk(long long nent);

// Work list of one task-list shape from its sub-box CSR offsets (nsub + 1 entries):
// Morton bands of sub-boxes, heaviest first inside a band, bands by decreasing mean
// weight; sub-boxes with more than chunk > 0 tasks are cut into chunks.
int order_work(int K, const LevelInfo* lev, const std::vector<long long>& count, long long chunk,
               std::vector<int4>* work, long long* nwork_out);

// Device task lists of a plan whose host part only counted them (Plan::tasks_on_device):
// allocates and fills d.task_c/sub_off_c/work_c and d.task_i/sub_off_i/work_i on stream
// s, adds the persistent bytes to *bytes, fills H.work_c/work_i and P->nwork/nwork_i.
int build_tasks_device(Plan* P, HostArrays& H, cudaStream_t s, long long* bytes);

// Device bytes of the sort buffers build_tasks_device needs beyond the plan's part buffer.
long long task_sort_bytes(const Plan& P);

// GPW_FAST_BLOCK_PRUNE: true when the task box [a_d, b_d] (unwrapped grid indices of a
// level with N points along each row) lies wholly farther than R from P, given P's
// fractional coordinates fp_d, the reciprocal row lengths blen_d and, for other than
// orthorhombic rows, lam <= the smallest eigenvalue of the lattice metric R_d . R_e.
// With df_d the fractional distance from P to the box along row d: orthorhombic rows
// give the exact distance sqrt(sum (df_d / blen_d)^2); other rows two lower bounds of it,
// the largest slab distance df_d / blen_d and sqrt(lam sum df_d^2).  Plain correctly
// rounded operations, so that the host and the device builders (which spell out every
// rounding) decide alike.
inline bool block_beyond(const PairQ& q, const int* a, const int* b, const int* N,
                         const double* blen, bool ortho, double lam) {
  const double fp[3] = {q.x, q.y, q.z};
  double f[3], s[3];
  for (int d = 0; d < 3; ++d) {
    const double fa = (double)a[d] / (double)N[d], fb = (double)b[d] / (double)N[d];
    f[d] = fp[d] < fa ? fa - fp[d] : (fp[d] > fb ? fp[d] - fb : 0.0);
    s[d] = f[d] / blen[d];
  }
  if (ortho) {
    const double r2 = (s[0] * s[0] + s[1] * s[1]) + s[2] * s[2];
    return r2 > q.w * q.w;
  }
  if (std::max(s[0], std::max(s[1], s[2])) > q.w) return true;
  const double f2 = (f[0] * f[0] + f[1] * f[1]) + f[2] * f[2];
  return lam * f2 > q.w * q.w;
}

// Return the task-record buffers of a plan that no longer needs them (after commit) to
// the planner's pool of spare buffers.
void recycle_host_arrays(HostArrays* H);

}  // namespace gpw
