// Fusion planner.  A pass is a tile bit set S (the low c qubits plus chosen
// higher ones) and the ops of the gates it absorbs; ops are grouped into
// register phases of kRegBits target bits.  Gates are absorbed in circuit
// order; a gate that cannot join blocks its qubits so that no later gate
// sharing a qubit jumps over it (gates on disjoint qubits commute).
#include <algorithm>
#include <cstring>

#include "plan.h"
#include "t2gen.h"
#include "tma.h"

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

// Op types the interpreter kernel implements: X, real and unit-diagonal ops
// only in complex128 one-state passes, Z flips as unit diagonals there and as
// general diagonals elsewhere.
uint8_t interp_type(uint8_t t, qs_dtype dt, bool two_state) {
  const bool special = dt == QS_C128 && !two_state;
  if (t == OP_ZFLIP) return special ? OP_UDIAG : OP_DIAG;
  if (!special && (t == OP_X || t == OP_REAL1)) return OP_DENSE1;
  if (!special && t == OP_UDIAG) return OP_DIAG;
  return t;
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
    std::vector<std::vector<size_t>> phase_items_all;
    std::vector<uint64_t> phase_need;
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
      const uint64_t Rneed = R;
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
          op.type = interp_type(io.type, pp.dt, (flags & (PF_LOAD_LAM | PF_STORE_LAM)) != 0);
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
      phase_items_all.push_back(phase_items);
      phase_need.push_back(Rneed);
    }
    if (slot_count > kMaxSlotsPerPass || (int)P.phases.size() > kMaxPhasesPerPass) {
      set_error("planner: pass exceeds slot/phase limits (internal error)");
      return QS_ERR_UNSUPPORTED;
    }
    P.hdr.n_slots = slot_count;
    P.hdr.slot_base = slot_base;
    P.hdr.n_phases = (int)P.phases.size();
    lower_t2(items, phase_items_all, phase_need, flags, &P);
    plan->passes.push_back(std::move(P));
    return QS_OK;
  }

  // The micro-op form of the pass (complex64 only).  Registers: the phase's
  // needed bits padded from the top of the tile (the low local bits stay lane
  // bits for the bank columns).  Lanes: under the 128-byte swizzle an element's
  // 8-byte bank slot has bits b0, b1 ^ b4, b2 ^ b5, b3 ^ b6 of its local index,
  // so the first lane bits take one local bit of each class {0}, {1, 4},
  // {2, 5}, {3, 6} (with 16-byte accesses, when bit 0 is a register bit, the
  // first three lanes take classes 1..3).  Leaves P->t2 false when the pass does
  // not qualify; the interpreter kernel then runs it.
  void lower_t2(const std::vector<const PlanItem*>& items, const std::vector<std::vector<size_t>>& ph_items,
                const std::vector<uint64_t>& ph_need, uint32_t flags, PlannedPass* P) {
    P->t2 = false;
    if (!pp.micro || pp.dt != QS_C64 || pp.c < 4 || (flags & PF_NEED_CUT)) return;
    const int ns = (flags & (PF_LOAD_LAM | PF_STORE_LAM)) ? 2 : 1;
    if (pp.m > (ns == 2 ? 12 : 13) || pp.m < 9) return;
    if (ns == 2 && !((flags & PF_LOAD_PSI) && (flags & PF_LOAD_LAM))) return;
    TileMapDims md;
    if (!tile_map_dims(S, pp.n, 0, pp.m, 4, 4, 1024, &md)) return;
    {  // every box of the zero-offset tile lies inside the map's dimensions
      const uint32_t nb = 1u << (pp.m - md.lb);
      for (uint32_t j = 0; j < nb; ++j) {
        uint64_t g = 0;
        const uint32_t l = j << md.lb;
        for (int b = 0; b < pp.m; ++b)
          if ((l >> b) & 1u) g |= 1ull << global_of[b];
        for (int d = 0; d < 5; ++d) {
          const uint64_t x = (g >> md.a[d]) & ((1ull << md.w[d]) - 1ull);
          if (x + (1ull << md.bx[d]) > (1ull << md.w[d])) return;
        }
      }
    }
    T2Pass H;
    std::memset(&H, 0, sizeof(H));
    H.m = pp.m;
    H.ns = ns;
    H.flags = flags;
    for (int i = 0; i < 5; ++i) {
      H.ma[i] = md.a[i];
      H.mw[i] = md.w[i];
      H.mbx[i] = md.bx[i];
    }
    H.mlb = md.lb;
    int k = 0;
    for (int q = 0; q < pp.n; ++q)
      if (!((S >> q) & 1)) H.comp[k++] = (int8_t)q;
    H.ncomp = k;
    for (int i = 0; i < 64; ++i) {
      uint64_t a = 0;
      for (int j = 0; j < 6; ++j)
        if (((i >> j) & 1) && 4 + j < pp.m) a |= 1ull << global_of[4 + j];
      H.hiA[i] = a;
    }
    for (int i = 0; i < 128; ++i) {
      uint64_t b = 0;
      for (int j = 0; j < 7; ++j)
        if (((i >> j) & 1) && 10 + j < pp.m) b |= 1ull << global_of[10 + j];
      H.hiB[i] = b;
    }
    auto swz = [](uint32_t l) { return l ^ (((l >> 4) & 7u) << 1); };
    std::vector<T2Phase> phs;
    std::vector<T2Op> ops;
    int n_coef = 0, n_slots = 0;
    for (size_t pi = 0; pi < ph_items.size(); ++pi) {
      uint64_t R = ph_need[pi];
      for (int l = pp.m - 1; l >= 0 && popc(R) < kRegBits; --l)
        if (l >= 7 && !((R >> l) & 1)) R |= 1ull << l;
      for (int l = pp.m - 1; l >= 0 && popc(R) < kRegBits; --l)
        if (!((R >> l) & 1)) R |= 1ull << l;
      T2Phase ph;
      std::memset(&ph, 0, sizeof(ph));
      int reg_of[16], ri = 0;
      for (int l = 0; l < 16; ++l) reg_of[l] = -1;
      for (int l = 0; l < pp.m; ++l)
        if ((R >> l) & 1) {
          reg_of[l] = ri;
          ph.R[ri] = (uint8_t)l;
          ph.sp[ri] = swz(1u << l);
          ++ri;
        }
      ph.pair = ph.R[0] == 0;
      // lane order: one bit per bank class first, then the rest ascending
      std::vector<int> rest, q;
      for (int l = 0; l < pp.m; ++l)
        if (!((R >> l) & 1)) rest.push_back(l);
      const int cls[4][2] = {{0, -1}, {1, 4}, {2, 5}, {3, 6}};
      for (int c0 = ph.pair ? 1 : 0; c0 < 4; ++c0)
        for (int v : cls[c0])
          if (v >= 0 && v < pp.m && !((R >> v) & 1) &&
              std::find(q.begin(), q.end(), v) == q.end()) {
            q.push_back(v);
            break;
          }
      for (int v : rest)
        if (std::find(q.begin(), q.end(), v) == q.end()) q.push_back(v);
      if (q.size() > 9) return;
      for (int e = 0; e < 48; ++e) {
        const int first = e < 16 ? 0 : 4;
        const uint32_t bits = e < 16 ? (uint32_t)e : (uint32_t)(e - 16);
        uint32_t v = 0;
        for (int i = 0; i < 5 && first + i < (int)q.size(); ++i)
          if ((bits >> i) & 1u) v |= 1u << q[first + i];
        ph.l0tab[e] = v;
      }
      ph.op_begin = (uint16_t)ops.size();
      for (size_t idx : ph_items[pi]) {
        const PlanItem& it = *items[idx];
        for (const ItemOp& io : it.ops) {
          T2Op op;
          std::memset(&op, 0, sizeof(op));
          op.d0 = op.d1 = 0xFF;
          for (int q2 = 0; q2 < pp.n; ++q2) {
            if (!((it.ctrl >> q2) & 1)) continue;
            const int l = local_of[q2];
            if (l < 0)
              op.gc |= 1ull << q2;
            else if (reg_of[l] >= 0)
              op.jc |= (uint8_t)(1u << reg_of[l]);
            else
              op.lc |= 1u << l;
          }
          const bool jc = op.jc != 0;
          auto reg = [&](int qb) { return local_of[qb] >= 0 ? reg_of[local_of[qb]] : -1; };
          auto cbit = [&](int qb) { return (uint8_t)(local_of[qb] >= 0 ? local_of[qb] : 64 + qb); };
          int nc = 0;
          switch (io.type) {
            case OP_DENSE1: case OP_REAL1: case OP_RX: case OP_X: case OP_GRAD1: {
              const int r0 = reg(it.t[0]);
              if (r0 < 0) return;
              const int kind = io.type == OP_DENSE1 ? T2_U1 : io.type == OP_REAL1 ? T2_R1 : io.type == OP_RX ? T2_RX
                               : io.type == OP_X ? T2_X : T2_G1;
              op.code = (uint16_t)t2_code(kind, r0, 0, jc);
              nc = kind == T2_X ? 0 : kind == T2_RX ? 1 : 4;
              break;
            }
            case OP_DENSE2: case OP_GRAD2: {
              const int r0 = reg(it.t[0]), r1 = reg(it.t[1]);
              if (r0 < 0 || r1 < 0 || r0 == r1) return;
              op.code = (uint16_t)t2_code(io.type == OP_DENSE2 ? T2_U2 : T2_G2, r0, r1, jc);
              nc = 16;
              break;
            }
            case OP_ZFLIP: {
              const int r0 = reg(it.t[0]);
              if (r0 >= 0) {
                op.code = (uint16_t)t2_code(T2_Z, r0, 0, jc);
              } else {
                op.code = (uint16_t)t2_code(T2_ZC, 0, 0, jc);
                op.d0 = cbit(it.t[0]);
              }
              break;
            }
            case OP_DIAG: case OP_UDIAG: {
              const int r0 = reg(it.t[0]);
              if (it.nt == 1) {
                if (r0 >= 0) {
                  op.code = (uint16_t)t2_code(T2_D1R, r0, 0, jc);
                } else {
                  op.code = (uint16_t)t2_code(T2_D1C, 0, 0, jc);
                  op.d0 = cbit(it.t[0]);
                }
                nc = 2;
              } else {
                const int r1 = reg(it.t[1]);
                if (r0 >= 0 && r1 >= 0) {
                  op.code = (uint16_t)t2_code(T2_D2RR, r0, r1, jc);
                } else if (r0 >= 0) {
                  op.code = (uint16_t)t2_code(T2_D2RC, r0, 0, jc);
                  op.d1 = cbit(it.t[1]);
                } else if (r1 >= 0) {
                  op.code = (uint16_t)t2_code(T2_D2CR, 0, r1, jc);
                  op.d0 = cbit(it.t[0]);
                } else {
                  op.code = (uint16_t)t2_code(T2_D2CC, 0, 0, jc);
                  op.d0 = cbit(it.t[0]);
                  op.d1 = cbit(it.t[1]);
                }
                nc = 4;
              }
              break;
            }
            case OP_GRADDIAG: {
              auto enc = [&](int qb) {
                const int r = reg(qb);
                return r >= 0 ? (uint8_t)(128 + r) : cbit(qb);
              };
              op.code = (uint16_t)t2_code(T2_GD, 0, 0, jc);
              op.d0 = enc(it.t[0]);
              op.d1 = it.nt == 2 ? enc(it.t[1]) : 0xFF;
              nc = it.nt == 2 ? 4 : 2;
              break;
            }
            default:
              return;  // cost-value and other ops: interpreter only
          }
          if (op.lc || op.gc) op.code |= (uint16_t)T2_OUTSIDE;
          op.cs = (uint16_t)n_coef;
          op.coef = (uint32_t)io.coef;
          op.ncoef = (uint32_t)nc;
          n_coef += nc;
          if (io.out >= 0) op.slot = (uint16_t)n_slots++;
          ops.push_back(op);
        }
      }
      ph.op_end = (uint16_t)ops.size();
      phs.push_back(ph);
    }
    if (n_slots != P->hdr.n_slots) return;  // slots must match the interpreter's numbering
    H.n_phases = (int)phs.size();
    H.n_ops = (int)ops.size();
    H.n_coef = n_coef;
    H.n_slots = n_slots;
    H.slot_base = P->hdr.slot_base;
    const size_t T = (size_t)std::min(1 << (pp.m - kRegBits), ns == 2 ? 256 : 512);
    const size_t tiles = (size_t)3 * ns * ((size_t)8 << pp.m);
    size_t smem = 1024 + tiles + sizeof(T2Pass) + phs.size() * sizeof(T2Phase) + ops.size() * sizeof(T2Op) +
                  (size_t)n_coef * 8 + (size_t)n_slots * (T / 32) * 8 + 5 * 64 * 8 + 256;
    if (smem > 227 * 1024 - 512 || ops.size() > 65535 || n_coef > 65535) return;
    H.smem = (uint32_t)smem;
    P->t2 = true;
    P->t2hdr = H;
    P->t2ph = std::move(phs);
    P->t2ops = std::move(ops);
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
  if (d_t2pass) cudaFree(d_t2pass);
  if (d_t2ph) cudaFree(d_t2ph);
  if (d_t2ops) cudaFree(d_t2ops);
  d_pass = nullptr;
  d_phase = nullptr;
  d_ops = nullptr;
  d_t2pass = nullptr;
  d_t2ph = nullptr;
  d_t2ops = nullptr;
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
  std::vector<T2Pass> t2p(std::max<size_t>(passes.size(), 1));
  std::vector<T2Phase> t2ph;
  std::vector<T2Op> t2ops;
  t2_phase_off.assign(passes.size(), 0);
  t2_op_off.assign(passes.size(), 0);
  for (size_t i = 0; i < passes.size(); ++i) {
    std::memset(&t2p[i], 0, sizeof(T2Pass));
    if (!passes[i].t2) continue;
    t2p[i] = passes[i].t2hdr;
    t2_phase_off[i] = (int)t2ph.size();
    t2_op_off[i] = (int)t2ops.size();
    t2ph.insert(t2ph.end(), passes[i].t2ph.begin(), passes[i].t2ph.end());
    t2ops.insert(t2ops.end(), passes[i].t2ops.begin(), passes[i].t2ops.end());
  }
  if (t2ph.empty()) t2ph.resize(1);
  if (t2ops.empty()) t2ops.resize(1);
  QS_CUDA(cudaMalloc(&d_t2pass, t2p.size() * sizeof(T2Pass)));
  QS_CUDA(cudaMalloc(&d_t2ph, t2ph.size() * sizeof(T2Phase)));
  QS_CUDA(cudaMalloc(&d_t2ops, t2ops.size() * sizeof(T2Op)));
  QS_CUDA(cudaMemcpyAsync(d_t2pass, t2p.data(), t2p.size() * sizeof(T2Pass), cudaMemcpyHostToDevice, st));
  QS_CUDA(cudaMemcpyAsync(d_t2ph, t2ph.data(), t2ph.size() * sizeof(T2Phase), cudaMemcpyHostToDevice, st));
  QS_CUDA(cudaMemcpyAsync(d_t2ops, t2ops.data(), t2ops.size() * sizeof(T2Op), cudaMemcpyHostToDevice, st));
  QS_CUDA(cudaMalloc(&d_pass, hp.size() * sizeof(DevPass)));
  QS_CUDA(cudaMalloc(&d_phase, hph.size() * sizeof(DevPhase)));
  QS_CUDA(cudaMalloc(&d_ops, hops.size() * sizeof(DevOp)));
  QS_CUDA(cudaMemcpyAsync(d_pass, hp.data(), hp.size() * sizeof(DevPass), cudaMemcpyHostToDevice, st));
  QS_CUDA(cudaMemcpyAsync(d_phase, hph.data(), hph.size() * sizeof(DevPhase), cudaMemcpyHostToDevice, st));
  QS_CUDA(cudaMemcpyAsync(d_ops, hops.data(), hops.size() * sizeof(DevOp), cudaMemcpyHostToDevice, st));
  QS_CUDA(cudaStreamSynchronize(st));
  gen_fn.clear();
  if (gen > 0) QS_TRY(t2gen_build(*this));
  return QS_OK;
}

}  // namespace qs
