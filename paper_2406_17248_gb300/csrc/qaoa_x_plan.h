// Host planner of the complex64 QAOA passes with separate forward and reverse
// tile shapes.
#pragma once

#include <utility>
#include <vector>

#include "plan.h"
#include "qaoa_x.h"

namespace qs {

// One pass of a sweep in global qubit masks: MIX(l1) on set1, then the
// diagonal step of layer ld (XDiag), then MIX(l3) on set3.
struct XSched {
  uint64_t S;
  uint64_t set1;
  int l1;
  int diag;
  int ld;
  uint64_t set3;
  int l3;
};

struct XBuild {
  int n, p;
  int mf, cf;  // forward tile bits / low bits
  int mr, cr;  // turnaround and reverse tile bits / low bits
  int n_edges;
  std::vector<std::pair<int, int>> edges;
};

// Forward sweep COST(0) MIX(0) ... MIX(p-1); the last pass completes MIX(p-1).
std::vector<XSched> qx_forward_schedule(int n, int p, int m, int c, int elem_bytes);
// Reverse sweep from MIX(p-1) with `rem0` still applied, down to COST(0).
std::vector<XSched> qx_reverse_schedule(int n, int p, int m, int c, uint64_t rem0, int elem_bytes);
// Descriptor of one pass (two_state: psi/lam kernel and the reverse tile shape);
// its in-tile edge-count table, if it has a diagonal step, is appended to *fs.
qs_status qx_build_pass(const XBuild& B, const XSched& s, bool two_state, uint32_t flags, int out_slots[3],
                        XPass* out, std::vector<uint8_t>* fs);

// Both plans of one engine: the gradient plan (forward passes, turnaround,
// reverse passes) and the energy plan, their output slots (output index:
// 0 = E, 1 + l = dgamma_l, 1 + p + l = dbeta_l) and the edge-count tables.
struct XPlans {
  std::vector<XPass> grad, energy;
  std::vector<int> grad_two, energy_two;
  SlotMap gslots, eslots;
  std::vector<uint8_t> fs;
  double bytes_grad = 0, bytes_energy = 0;
  int n_fwd = 0, n_rev = 0;  // forward passes (the turnaround included), reverse passes
  int n_coef = 0;            // complex entries of the per-call coefficient table
};
qs_status qx_make_plans(const XBuild& B, double gs, XPlans* X);

// The per-call coefficient table (interleaved FP64 complex, n_coef entries):
// per layer the renormalised cost LUTs and the scaled-mixer t of both sweep
// directions, then every pass's phase weights (see qaoa_x.h).  *flip: the
// energy plan leaves the state with every qubit flipped (an odd number of
// layers took the flipped mixer form).
qs_status qx_fill_coef(int n, int p, int n_edges, double gs, const double* gamma, const double* beta,
                       const std::vector<XPass>& grad, const std::vector<XPass>& energy, int n_coef,
                       std::vector<double>* tab, bool* flip);

}  // namespace qs
