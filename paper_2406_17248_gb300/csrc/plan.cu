// Fusion planner.  A pass is a tile bit set S (the low c qubits plus chosen
// higher ones) and the ops of the gates it absorbs; ops are grouped into
// register phases of kRegBits target bits.  Gates are absorbed in circuit
// order; a gate that cannot join blocks its qubits so that no later gate
// sharing a qubit jumps over it (gates on disjoint qubits commute).
#include <algorithm>
#include <cstring>

#include "plan.h"

namespace qs {

namespace {

inline int popc(uint64_t x) { return __builtin_popcountll(x); }

uint64_t item_need(const PlanItem& it) {
  if (it.kind == IK_DENSE1) return 1ull << it.t[0];
  if (it.kind == IK_DENSE2) return (1ull << it.t[0]) | (1ull << it.t[1]);
  return 0;
}

// Order the sub-cube bits so that the lowest W of them have distinct residues
// mod W (the shared-memory swizzle folds bit b onto bank bit b mod W), then the
// rest ascending.
std::vector<int> order_q(const std::vector<int>& rest, int W) {
  std::vector<int> q, used(rest.size(), 0);
  for (int r = 0; r < W; ++r) {
    for (size_t i = 0; i < rest.size(); ++i) {
      if (!used[i] && rest[i] % W == r) {
        q.push_back(rest[i]);
        used[i] = 1;
        break;
      }
    }
  }
  std::vector<int> tail;
  for (size_t i = 0; i < rest.size(); ++i)
    if (!used[i]) tail.push_back(rest[i]);
  std::sort(q.begin(), q.end());
  q.insert(q.end(), tail.begin(), tail.end());
  return q;
}

struct PassBuilder {
  const PlanParams& pp;
  uint64_t S;
  int local_of[64];
  int global_of[16];

  PassBuilder(const PlanParams& p, uint64_t s) : pp(p), S(s) {
    int k = 0;
    for (int q = 0; q < 64; ++q) local_of[q] = -1;
    for (int q = 0; q < pp.n; ++q)
      if ((S >> q) & 1) {
        local_of[q] = k;
        global_of[k] = q;
        ++k;
      }
  }

  // Emit the pass: phases built greedily from the items (in order).
  qs_status emit(const std::vector<const PlanItem*>& items, uint32_t flags, TilePlan* plan, SlotMap* slots) {
    PlannedPass P;
    std::memset(&P.hdr, 0, sizeof(P.hdr));
    P.hdr.m = pp.m;
    P.hdr.c = pp.c;
    P.hdr.flags = flags;
    int k = 0;
    for (int q = 0; q < pp.n; ++q)
      if (!((S >> q) & 1)) P.hdr.comp[k++] = (int8_t)q;
    P.hdr.ncomp = k;
    for (int i = 0; i < 64; ++i) {
      uint64_t a = 0, b = 0;
      for (int j = 0; j < 6; ++j) {
        const int la = pp.c + j, lb = pp.c + 6 + j;
        if ((i >> j) & 1) {
          if (la < pp.m) a |= 1ull << global_of[la];
          if (lb < pp.m) b |= 1ull << global_of[lb];
        }
      }
      P.hdr.hiA[i] = a;
      P.hdr.hiB[i] = b;
    }
    for (int i = 64; i < 128; ++i) P.hdr.hiB[i] = 0;
    for (const PlanItem* it : items)
      if (it->kind == IK_GLOBAL_DIAG) P.hdr.flags |= PF_NEED_CUT;

    const int W = pp.dt == QS_C64 ? 4 : 3;
    std::vector<char> taken(items.size(), 0);
    size_t n_taken = 0;
    int slot_count = 0;
    const int slot_base = (int)slots->out.size();
    while (n_taken < items.size()) {
      uint64_t R = 0;        // local-bit mask in registers
      uint64_t blocked = 0;  // global qubits of items skipped in this sweep
      std::vector<size_t> phase_items;
      for (size_t i = 0; i < items.size(); ++i) {
        if (taken[i]) continue;
        const PlanItem& it = *items[i];
        if (it.touched & blocked) {
          blocked |= it.touched;
          continue;
        }
        uint64_t needl = 0;
        const uint64_t need = item_need(it);
        for (int q = 0; q < pp.n; ++q)
          if ((need >> q) & 1) needl |= 1ull << local_of[q];
        if ((needl & ~R) == 0 || popc(R | needl) <= kRegBits) {
          R |= needl;
          phase_items.push_back(i);
          taken[i] = 1;
          ++n_taken;
        } else {
          blocked |= it.touched;
        }
      }
      if (phase_items.empty()) {
        set_error("planner: no progress (internal error)");
        return QS_ERR_UNSUPPORTED;
      }
      // pad R to kRegBits local bits, lowest free first
      for (int l = 0; l < pp.m && popc(R) < kRegBits; ++l)
        if (!((R >> l) & 1)) R |= 1ull << l;
      DevPhase ph;
      std::memset(&ph, 0, sizeof(ph));
      int ri = 0;
      int reg_of_local[16];
      for (int l = 0; l < 16; ++l) reg_of_local[l] = -1;
      for (int l = 0; l < pp.m; ++l)
        if ((R >> l) & 1) {
          reg_of_local[l] = ri;
          ph.R[ri++] = (int8_t)l;
        }
      std::vector<int> rest;
      for (int l = 0; l < pp.m; ++l)
        if (!((R >> l) & 1)) rest.push_back(l);
      std::vector<int> q = order_q(rest, W);
      ph.nq = (int16_t)q.size();
      for (size_t i = 0; i < q.size(); ++i) ph.Q[i] = (int8_t)q[i];
      ph.op_begin = (int)plan_ops_size(P);
      for (size_t idx : phase_items) {
        const PlanItem& it = *items[idx];
        for (const ItemOp& io : it.ops) {
          DevOp op;
          std::memset(&op, 0, sizeof(op));
          op.type = io.type;
          op.flags = io.flags;
          op.coef = (uint32_t)io.coef;
          op.dloc[0] = op.dloc[1] = -1;
          op.dglb[0] = op.dglb[1] = -1;
          for (int q2 = 0; q2 < pp.n; ++q2) {
            if (!((it.ctrl >> q2) & 1)) continue;
            const int l = local_of[q2];
            if (l < 0)
              op.gc |= 1ull << q2;
            else if (reg_of_local[l] >= 0)
              op.jc |= (uint16_t)(1u << reg_of_local[l]);
            else
              op.lc |= 1u << l;
          }
          if (it.kind == IK_DENSE1 || it.kind == IK_DENSE2) {
            op.rb0 = (uint8_t)reg_of_local[local_of[it.t[0]]];
            if (it.kind == IK_DENSE2) op.rb1 = (uint8_t)reg_of_local[local_of[it.t[1]]];
          } else if (it.kind == IK_DIAG) {
            for (int j = 0; j < it.nt; ++j) {
              const int l = local_of[it.t[j]];
              if (l >= 0)
                op.dloc[j] = (int8_t)l;
              else
                op.dglb[j] = (int8_t)it.t[j];
            }
          }
          if (io.out >= 0) {
            op.slot = (uint16_t)slot_count++;
            slots->out.push_back(io.out);
            slots->weight.push_back(io.weight);
          }
          P.ops.push_back(op);
        }
      }
      ph.op_end = (int)plan_ops_size(P);
      P.phases.push_back(ph);
    }
    if (slot_count > kMaxSlotsPerPass || (int)P.phases.size() > kMaxPhasesPerPass) {
      set_error("planner: pass exceeds slot/phase limits (internal error)");
      return QS_ERR_UNSUPPORTED;
    }
    P.hdr.n_slots = slot_count;
    P.hdr.slot_base = slot_base;
    P.hdr.n_phases = (int)P.phases.size();
    plan->passes.push_back(std::move(P));
    return QS_OK;
  }

  static size_t plan_ops_size(const PlannedPass& P) { return P.ops.size(); }
};

}  // namespace

qs_status plan_single_pass(const std::vector<PlanItem>& items, uint64_t S, const PlanParams& pp, uint32_t flags,
                           TilePlan* plan, SlotMap* slots) {
  std::vector<const PlanItem*> v;
  for (const auto& it : items) {
    if (item_need(it) & ~S) {
      set_error("planner: item outside the tile (internal error)");
      return QS_ERR_UNSUPPORTED;
    }
    v.push_back(&it);
  }
  PassBuilder b(pp, S);
  return b.emit(v, flags, plan, slots);
}

qs_status plan_items(const std::vector<PlanItem>& items, const PlanParams& pp, uint32_t flags, TilePlan* plan,
                     SlotMap* slots) {
  const uint64_t low = (pp.c >= 64) ? ~0ull : ((1ull << pp.c) - 1);
  std::vector<char> done(items.size(), 0);
  size_t n_done = 0;
  size_t first = 0;
  const size_t lookahead = 512;
  while (n_done < items.size()) {
    while (first < items.size() && done[first]) ++first;
    // choose S
    uint64_t S = low;
    uint64_t blocked = 0;
    size_t scanned = 0;
    for (size_t i = first; i < items.size() && scanned < lookahead; ++i) {
      if (done[i]) continue;
      ++scanned;
      const PlanItem& it = items[i];
      if (it.touched & blocked) {
        blocked |= it.touched;
        continue;
      }
      const uint64_t need = item_need(it);
      if (popc(S | need) <= pp.m)
        S |= need;
      else
        blocked |= it.touched;
    }
    for (int q = 0; q < pp.n && popc(S) < pp.m; ++q) S |= 1ull << q;
    // absorb
    std::vector<const PlanItem*> take;
    blocked = 0;
    int slot_est = 0;
    for (size_t i = first; i < items.size(); ++i) {
      if (done[i]) continue;
      const PlanItem& it = items[i];
      int it_slots = 0;
      for (const auto& o : it.ops) it_slots += o.out >= 0;
      if ((it.touched & blocked) || (item_need(it) & ~S) || slot_est + it_slots > kMaxSlotsPerPass ||
          take.size() >= 4096) {
        blocked |= it.touched;
        continue;
      }
      take.push_back(&it);
      slot_est += it_slots;
      done[i] = 1;
      ++n_done;
    }
    if (take.empty()) {
      set_error("planner: no progress (internal error)");
      return QS_ERR_UNSUPPORTED;
    }
    PassBuilder b(pp, S);
    QS_TRY(b.emit(take, flags, plan, slots));
  }
  return QS_OK;
}

void TilePlan::free_device() {
  if (d_pass) cudaFree(d_pass);
  if (d_phase) cudaFree(d_phase);
  if (d_ops) cudaFree(d_ops);
  d_pass = nullptr;
  d_phase = nullptr;
  d_ops = nullptr;
}

qs_status TilePlan::upload(cudaStream_t st) {
  free_device();
  std::vector<DevPass> hp;
  std::vector<DevPhase> hph;
  std::vector<DevOp> hops;
  for (auto& p : passes) {
    DevPass h = p.hdr;
    h.phase_begin = (int)hph.size();
    const int op_base = (int)hops.size();
    for (auto ph : p.phases) {
      ph.op_begin += op_base;
      ph.op_end += op_base;
      hph.push_back(ph);
    }
    hops.insert(hops.end(), p.ops.begin(), p.ops.end());
    h.n_phases = (int)p.phases.size();
    hp.push_back(h);
  }
  if (hops.empty()) hops.resize(1);
  if (hph.empty()) hph.resize(1);
  if (hp.empty()) hp.resize(1);
  QS_CUDA(cudaMalloc(&d_pass, hp.size() * sizeof(DevPass)));
  QS_CUDA(cudaMalloc(&d_phase, hph.size() * sizeof(DevPhase)));
  QS_CUDA(cudaMalloc(&d_ops, hops.size() * sizeof(DevOp)));
  QS_CUDA(cudaMemcpyAsync(d_pass, hp.data(), hp.size() * sizeof(DevPass), cudaMemcpyHostToDevice, st));
  QS_CUDA(cudaMemcpyAsync(d_phase, hph.data(), hph.size() * sizeof(DevPhase), cudaMemcpyHostToDevice, st));
  QS_CUDA(cudaMemcpyAsync(d_ops, hops.data(), hops.size() * sizeof(DevOp), cudaMemcpyHostToDevice, st));
  QS_CUDA(cudaStreamSynchronize(st));
  return QS_OK;
}

}  // namespace qs
