// Fusion planner: gate sequences -> fused tile passes (host side).
#pragma once

#include "qsim_internal.h"

namespace qs {

// One op an item emits; `out` is the logical output it accumulates into
// (-1: none).  `coef` indexes the per-call coefficient table.
struct ItemOp {
  uint8_t type;
  uint8_t flags;
  int coef;
  int out;
  double weight;  // multiplies the accumulated partial when gathered into `out`
};

enum ItemKind { IK_DENSE1, IK_DENSE2, IK_DIAG, IK_GLOBAL_DIAG };

struct PlanItem {
  int kind;
  int nt;
  int t[2];
  uint64_t ctrl;     // control qubits
  uint64_t touched;  // every qubit the item reads or writes (ordering)
  std::vector<ItemOp> ops;
};

struct PlanParams {
  int n;       // qubits (>= kRegBits)
  int m;       // tile bits
  int c;       // low contiguous bits
  qs_dtype dt;
  bool micro = true;  // also lower qualifying passes to micro-ops (k_tile2.cu)
};

// Slots: every accumulating op of a pass gets a launch-local slot; the plan's
// slot table maps it to (output, weight).
struct SlotMap {
  std::vector<int> out;
  std::vector<double> weight;
};

// Plan a sequence of items into passes appended to `plan` with the given pass
// flags.  Grad/energy ops get slots appended to `slots`.
qs_status plan_items(const std::vector<PlanItem>& items, const PlanParams& pp, uint32_t flags, TilePlan* plan,
                     SlotMap* slots);

// Plan one pass over an explicit tile bit set (all items must fit).
qs_status plan_single_pass(const std::vector<PlanItem>& items, uint64_t S, const PlanParams& pp, uint32_t flags,
                           TilePlan* plan, SlotMap* slots);

}  // namespace qs
