// Host staging arrays produced by build_host_plan and uploaded by gpw_plan.
#pragma once

#include <vector>

#include "gpw_internal.h"

namespace gpw {

struct HostArrays {
  std::vector<int4> hot_a, hot_b, ids, ids2;
  std::vector<double> geo, cab;
  std::vector<long long> tab_off, coef_off, part_off, xt_off;
  std::vector<int4> task_c, task_i;   // 2 int4 per task
  std::vector<long long> sub_off_c, sub_off_i;
  std::vector<long long> toff_c, toff_i;  // per-pair task prefix sums (device-built lists)
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

// Return the task-record buffers of a plan that no longer needs them (after commit) to
// the planner's pool of spare buffers.
void recycle_host_arrays(HostArrays* H);

}  // namespace gpw
