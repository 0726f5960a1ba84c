// tqr_plan.h -- host-side task lists and their priority order.
//
// A plan is the list of tasks of one launch, in the order the device hands
// them out.  It is built in three steps:
//   1. enumerate the tasks of the mode in the sequential order of the
//      algorithm (Algorithm 1 for the factorization);
//   2. derive the DAG from the per-task rules of tqr_graph.h: for every slab
//      counter, the writers in sequential order; a wait for version v on a
//      counter depends on that counter's v-th writer.  This step also checks
//      the rules against the sequential order (every writer must wait for
//      exactly the number of writers before it);
//   3. simulate list scheduling on `workers` CTAs with a cost model and keep
//      the start order of the better of two priority policies: the paper's
//      static priorities (Section 3.3: GEQRT > TSQRT > LARFB > SSRFB, ties
//      by smaller k) or the longest remaining path ("bottom level").
#pragma once

#include <stdint.h>

#include <string>
#include <vector>

#include "tqr_graph.h"

namespace tqr {

struct PlanStats {
  double makespan_s = 0;     // simulated time of the chosen order
  double makespan_other = 0; // simulated time of the other policy
  int policy = 0;            // 0: paper priorities, 1: bottom level
  int64_t edges = 0;
  double critical_path_s = 0;
  double work_s = 0;         // sum of task costs
};

// Tree variant: the prefix table of writes per row (Inst.vtab), (kt+1) x p.
void tree_table(const Inst& I, std::vector<int32_t>& vt);

// Tasks of one instance in the sequential order of its mode.
void seq_tasks(const Inst& I, int inst_index, std::vector<TaskX>& out);

// Builds predecessor-count / successor lists (CSR) from the rules.  Returns
// false and sets *err when the rules contradict the sequential order.
bool build_dag(const std::vector<Inst>& insts, const std::vector<TaskX>& seq, std::vector<int>& indeg,
               std::vector<int64_t>& succ_ptr, std::vector<int>& succ, std::string* err);

// Cost model (seconds on one CTA) used by the simulation.
double task_cost(const Inst& I, const TaskX& t, int esize, int ctas_per_sm);

// Orders `seq` for `workers` CTAs.  Returns false on a rule error.
bool order_tasks(const std::vector<Inst>& insts, const std::vector<TaskX>& seq, int workers, int esize,
                 int ctas_per_sm, int policy /* -1: best of both */, std::vector<TaskX>& ordered,
                 PlanStats* stats, std::string* err);

// Orders a (possibly multi-instance) task set by decreasing bottom level
// (longest remaining path, cost model) without simulation and without
// materialising predecessor lists: one backward sweep over the sequential
// order propagates each task's bottom level to the writers it waits on.
// Sorting by strictly decreasing bottom level is a topological order because
// every task costs more than zero.  Used for large batches.
bool order_bottom_level(const std::vector<Inst>& insts, const std::vector<TaskX>& seq, int esize, int ctas_per_sm,
                        int workers, std::vector<TaskX>& ordered, PlanStats* stats, std::string* err);

// Critical path and total work (seconds of the cost model) of one
// instance's task graph, without building it: one pass over the sequential
// order, where every wait is on the preceding writer of its counter, so a
// task starts when the last writers of its counters finish.
void critical_path_estimate(const Inst& I, int esize, int ctas_per_sm, double* critical_path_s, double* work_s);

}  // namespace tqr
