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
  std::vector<int4> work_c, work_i;   // {plan slot, level, sub-box, tasks}
  std::vector<int4> groups;
  std::vector<long long> atom_off;
  std::vector<int> atom_list;
};

// Return the task-record buffers of a plan that no longer needs them (after commit) to
// the planner's pool of spare buffers.
void recycle_host_arrays(HostArrays* H);

}  // namespace gpw
