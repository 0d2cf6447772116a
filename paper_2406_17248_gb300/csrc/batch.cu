// Host side of the batched engine: argument checks, device tables, queue order.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "batch.h"
#include "handles.h"

using namespace qs;

// An instance too large for shared memory: it runs on the fused tile passes of
// its own circuit plan, on one of the batch's lanes.
struct BLarge {
  int inst = 0;
  int param_off = 0, n_params = 0;
  qs_circuit* c = nullptr;
  qs_ham* h = nullptr;
};

// A lane: a stream with its own psi, lam and scratch, so that large instances
// on different lanes overlap.
#ifndef QS_BATCH_LANES
#define QS_BATCH_LANES 32
#endif
constexpr int kBatchLanes = QS_BATCH_LANES;
struct BLane {
  cudaStream_t st = nullptr;
  cudaEvent_t done = nullptr;
  void* psi = nullptr;
  void* lam = nullptr;
  double* scratch = nullptr;
};

// Large instances of one qubit count run in lock-step: pass k of every member
// in one launch (instance = blockIdx.y), then one batched Hamiltonian apply,
// energy reduction, reverse passes, slot reduction and parameter gather.
struct BGroup {
  int ne = 0, m_fwd = 0, m_rev = 0, grid1 = 0, grid2 = 0, hgrid = 0;
  bool micro = false;          // every pass in micro-op form (k_tile2.cu), else every pass on the interpreter
  T2Args* d_fwd2 = nullptr;    // micro-op pass arguments, [pass k][member with that pass]
  T2Args* d_rev2 = nullptr;
  std::vector<uint32_t> fwd_smem, rev_smem;  // per pass index: the largest member's shared memory
  int gx_fwd = 1, gx_rev = 1;  // CTAs per member (each loops over several tiles)
  std::vector<int> members;  // indices into qs_batch::large
  void* psi = nullptr;       // members' states back to back
  void* lam = nullptr;
  double* scratch = nullptr;
  TileKArgs* d_fwd = nullptr;  // [pass k][member with that pass]
  TileKArgs* d_rev = nullptr;
  std::vector<int> fwd_off, fwd_cnt, rev_off, rev_cnt;
  HamMultiArgs* d_ham = nullptr;
  ReduceMultiArgs* d_red_e = nullptr;
  ReduceMultiArgs* d_red_s = nullptr;
  GatherMultiArgs* d_gather = nullptr;
  int n_red_s = 0, n_gather = 0, max_slots = 0, max_params = 0;
  cudaStream_t st = nullptr;
  cudaEvent_t done = nullptr;
};

struct qs_batch {
  qs_dtype dt = QS_C64;
  cudaStream_t st = nullptr;
  int n_inst = 0;
  int n_small = 0;                 // instances run by the persistent kernel (shared memory)
  std::vector<BLarge> large;       // instances run on fused tile passes
  std::vector<BGroup> groups;      // ... in lock-step by qubit count
  std::vector<char> in_group;      // per entry of `large`
  std::vector<BLane> lanes;        // ... or one by one on lanes (the rest)
  BCoefGate* d_cg = nullptr;       // coefficient-table entries of the large instances' gates
  int n_cg = 0;
  BCoefRun* d_runs = nullptr;      // fused single-qubit runs of their forward passes
  BCoefGate* d_run_members = nullptr;
  int n_runs = 0;
  cudaEvent_t ev_fill = nullptr;
  // the whole call (coefficients, lanes, persistent kernel) captured once as a
  // CUDA graph on the batch's own parameter/output buffers and replayed
  cudaGraphExec_t graph = nullptr;
  bool graph_failed = false;
  cudaStream_t cap_st = nullptr;   // the graph's stream (capture needs a non-default stream)
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  int n_params_total = 0;
  BInst* d_inst = nullptr;
  int* d_order = nullptr;
  BGate* d_gates = nullptr;
  DevHamGroup* d_groups = nullptr;
  DevHamTerm* d_terms = nullptr;
  double* d_params = nullptr;
  double* d_energy = nullptr;
  double* d_grad = nullptr;
  int* d_queue = nullptr;
  int smem_amps = 0, smem_gates = 0, smem_params = 0;
  int grid = 0;
};

namespace {

bool batch_kind_ok(int k) {
  return (k >= QS_GATE_I && k <= QS_GATE_SWAP) || (k >= QS_GATE_RX && k <= QS_GATE_RZZ);
}
bool batch_two_target(int k) { return k == QS_GATE_SWAP || k == QS_GATE_RXX || k == QS_GATE_RYY || k == QS_GATE_RZZ; }
bool batch_param_ok(int k) { return k >= QS_GATE_RX && k <= QS_GATE_RZZ; }

void free_batch(qs_batch* b) {
  if (!b) return;
  for (BLarge& L : b->large) {
    if (L.c) qs_circuit_destroy(L.c);
    if (L.h) qs_ham_destroy(L.h);
  }
  for (BGroup& G : b->groups) {
    for (void* p : {G.psi, G.lam, (void*)G.scratch, (void*)G.d_fwd, (void*)G.d_rev, (void*)G.d_ham,
                    (void*)G.d_red_e, (void*)G.d_red_s, (void*)G.d_gather, (void*)G.d_fwd2, (void*)G.d_rev2})
      if (p) cudaFree(p);
    if (G.st) cudaStreamDestroy(G.st);
    if (G.done) cudaEventDestroy(G.done);
  }
  for (BLane& L : b->lanes) {
    if (L.st) cudaStreamDestroy(L.st);
    if (L.done) cudaEventDestroy(L.done);
    for (void* p : {L.psi, L.lam, (void*)L.scratch})
      if (p) cudaFree(p);
  }
  if (b->d_cg) cudaFree(b->d_cg);
  if (b->d_runs) cudaFree(b->d_runs);
  if (b->d_run_members) cudaFree(b->d_run_members);
  if (b->ev_fill) cudaEventDestroy(b->ev_fill);
  if (b->graph) cudaGraphExecDestroy(b->graph);
  if (b->cap_st) cudaStreamDestroy(b->cap_st);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  for (void* p : {(void*)b->d_inst, (void*)b->d_order, (void*)b->d_gates, (void*)b->d_groups, (void*)b->d_terms,
                  (void*)b->d_params, (void*)b->d_energy, (void*)b->d_grad, (void*)b->d_queue})
    if (p) cudaFree(p);
  delete b;
}

template <class X>
qs_status upload(X** dst, const std::vector<X>& v) {
  const size_t n = std::max<size_t>(v.size(), 1);
  QS_CUDA(cudaMalloc(dst, n * sizeof(X)));
  if (!v.empty()) QS_CUDA(cudaMemcpy(*dst, v.data(), v.size() * sizeof(X), cudaMemcpyHostToDevice));
  return QS_OK;
}

// Energy and adjoint gradient of one large instance on a lane: psi = U|0> by
// the forward passes, lam = H psi with E, then the reverse passes with the
// gradient slots gathered into the instance's slice of the outputs.
qs_status run_large(const qs_batch* b, const BLarge& I, const BLane& L, double* energies, double* grads) {
  const CircuitPlan& P = I.c->plan;
  const qs_ham* h = I.h;
  const int ne = P.ne;
  const int n_slots = (int)P.rev_slots.out.size();
  const size_t part = (size_t)std::max(n_slots, 1) * P.grid2;
  double* d_part = L.scratch;
  double* d_slot = d_part + part;
  double* d_hpart = d_slot + n_slots + 1;
  const int hgrid = ham_grid_size(ne);
  QS_TRY(launch_set_basis(b->dt, L.psi, ne, 0, L.st));
  QS_TRY(run_passes(P.fwd, 0, (int)P.fwd.passes.size(), b->dt, L.psi, nullptr, P.d_coef, nullptr, d_part, ne, 0,
                    P.grid1, P.grid2, L.st));
  QS_TRY(launch_ham_apply(b->dt, L.psi, L.lam, ne, h->d_groups, h->n_groups, h->d_terms, d_hpart, hgrid, L.st));
  QS_TRY(launch_reduce_slots(d_hpart, 1, hgrid, nullptr, energies + I.inst, L.st));
  QS_TRY(run_passes(P.rev, 0, (int)P.rev.passes.size(), b->dt, L.psi, L.lam, P.d_coef, nullptr, d_part, ne, 0,
                    P.grid1, P.grid2, L.st));
  if (I.n_params > 0) {
    QS_TRY(launch_reduce_slots(d_part, n_slots, P.grid2, nullptr, d_slot, L.st));
    QS_TRY(launch_param_gather(d_slot, P.d_row, P.d_sidx, P.d_w, I.n_params, grads + I.param_off, L.st));
  }
  return QS_OK;
}

// One lock-step group: |0>, forward passes, lam = H psi and E, reverse passes,
// slot sums, gradient gather; every step one launch over all members.  The
// output pointers in the argument tables are the batch's own buffers.
qs_status run_group(const qs_batch* b, const BGroup& G, double* energies, double* grads) {
  (void)energies;
  (void)grads;
  QS_TRY(launch_set_zero_multi(b->dt, G.psi, G.ne, (int)G.members.size(), G.st));
  for (size_t k = 0; k < G.fwd_cnt.size(); ++k) {
    if (G.micro)
      QS_TRY(launch_tile2_multi(1, G.d_fwd2 + G.fwd_off[k], G.fwd_cnt[k], G.gx_fwd, G.fwd_smem[k], G.st));
    else
      QS_TRY(launch_tile_pass_multi(b->dt, 1, G.m_fwd, G.d_fwd + G.fwd_off[k], G.fwd_cnt[k], G.grid1, G.st));
  }
  QS_TRY(launch_ham_apply_multi(b->dt, G.d_ham, (int)G.members.size(), G.hgrid, G.st));
  QS_TRY(launch_reduce_multi(G.d_red_e, (int)G.members.size(), 1, G.st));
  for (size_t k = 0; k < G.rev_cnt.size(); ++k) {
    if (G.micro)
      QS_TRY(launch_tile2_multi(2, G.d_rev2 + G.rev_off[k], G.rev_cnt[k], G.gx_rev, G.rev_smem[k], G.st));
    else
      QS_TRY(launch_tile_pass_multi(b->dt, 2, G.m_rev, G.d_rev + G.rev_off[k], G.rev_cnt[k], G.grid2, G.st));
  }
  QS_TRY(launch_reduce_multi(G.d_red_s, G.n_red_s, G.max_slots, G.st));
  QS_TRY(launch_gather_multi(G.d_gather, G.n_gather, G.max_params, G.st));
  return QS_OK;
}

// Groups of large instances with one qubit count whose plans run only on the
// interpreter kernel (equal tile shapes and grids): built once, the argument
// tables pointing at the batch's parameter, energy and gradient buffers.
qs_status build_groups(qs_batch* b) {
  b->in_group.assign(b->large.size(), 0);
  std::vector<int> by_ne(64, -1);
  for (size_t k = 0; k < b->large.size(); ++k) {
    const CircuitPlan& P = b->large[k].c->plan;
    bool ok = P.valid && P.fuse >= 0 && P.ckpt.empty() && !P.fwd.passes.empty() && !P.rev.passes.empty();
    const bool micro = P.fwd.passes[0].t2;
    for (const auto& pp : P.fwd.passes) ok = ok && pp.t2 == micro;
    for (const auto& pp : P.rev.passes) ok = ok && pp.t2 == micro;
    if (!ok) continue;
    const int mf = P.fwd.passes[0].hdr.m, mr = P.rev.passes[0].hdr.m;
    for (const auto& pp : P.fwd.passes) ok = ok && pp.hdr.m == mf;
    for (const auto& pp : P.rev.passes) ok = ok && pp.hdr.m == mr;
    if (!ok) continue;
    int gi = by_ne[P.ne];
    if (gi >= 0) {
      const BGroup& G = b->groups[gi];
      if (G.m_fwd != mf || G.m_rev != mr || G.grid1 != P.grid1 || G.grid2 != P.grid2 || G.micro != micro) continue;
    } else {
      gi = (int)b->groups.size();
      by_ne[P.ne] = gi;
      b->groups.emplace_back();
      BGroup& G = b->groups.back();
      G.micro = micro;
      G.ne = P.ne;
      G.m_fwd = mf;
      G.m_rev = mr;
      G.grid1 = P.grid1;
      G.grid2 = P.grid2;
      G.hgrid = ham_grid_size(P.ne);
    }
    b->groups[gi].members.push_back((int)k);
    b->in_group[k] = 1;
  }
  const size_t amp = amp_bytes(b->dt);
  for (BGroup& G : b->groups) {
    const int cnt = (int)G.members.size();
    const size_t sb = amp << G.ne;
    QS_CUDA(cudaMalloc(&G.psi, sb * cnt));
    QS_CUDA(cudaMalloc(&G.lam, sb * cnt));
    QS_CUDA(cudaStreamCreateWithFlags(&G.st, cudaStreamNonBlocking));
    QS_CUDA(cudaEventCreateWithFlags(&G.done, cudaEventDisableTiming));
    // scratch per member: slot partials (slots x grid2), slot sums, Hamiltonian partials
    std::vector<size_t> off(cnt + 1, 0);
    for (int i = 0; i < cnt; ++i) {
      const CircuitPlan& P = b->large[G.members[i]].c->plan;
      const size_t ns = P.rev_slots.out.size();
      off[i + 1] = off[i] + std::max<size_t>(ns, 1) * G.grid2 + ns + (size_t)G.hgrid + 2;
    }
    QS_CUDA(cudaMalloc(&G.scratch, off[cnt] * sizeof(double)));
    auto state = [&](void* base, int i) { return (void*)((char*)base + sb * (size_t)i); };
    std::vector<TileKArgs> fwd, rev;
    std::vector<HamMultiArgs> ham;
    std::vector<ReduceMultiArgs> rede, reds;
    std::vector<GatherMultiArgs> gath;
    size_t max_f = 0, max_r = 0;
    for (int i = 0; i < cnt; ++i) {
      const CircuitPlan& P = b->large[G.members[i]].c->plan;
      max_f = std::max(max_f, P.fwd.passes.size());
      max_r = std::max(max_r, P.rev.passes.size());
    }
    auto targs = [&](const CircuitPlan& P, const TilePlan& T, int k, int i) {
      TileKArgs a;
      a.psi = state(G.psi, i);
      a.lam = state(G.lam, i);
      a.pass = T.d_pass + k;
      a.phases = T.d_phase;
      a.ops = T.d_ops;
      a.coef = P.d_coef;
      a.cut = nullptr;
      a.partials = G.scratch + off[i];
      a.n = G.ne;
      a.n_edges = 0;
      a.grid_stride = G.grid2;
      return a;
    };
    std::vector<T2Args> fwd2, rev2;
    // micro-op passes: CTAs per member so that each loops over about 8 tiles
    G.gx_fwd = (int)std::max<uint64_t>(1, (1ull << (G.ne - G.m_fwd)) / 8);
    G.gx_rev = (int)std::max<uint64_t>(1, (1ull << (G.ne - G.m_rev)) / 8);
    auto t2args = [&](const CircuitPlan& P, const TilePlan& T, int k, int i, T2Args* a) {
      return make_tile2_args(T, k, state(G.psi, i), state(G.lam, i), P.d_coef, G.scratch + off[i], G.grid2,
                             G.grid2, G.ne, a);
    };
    for (size_t k = 0; k < max_f; ++k) {
      G.fwd_off.push_back(G.micro ? (int)fwd2.size() : (int)fwd.size());
      uint32_t sm = 0;
      for (int i = 0; i < cnt; ++i) {
        const CircuitPlan& P = b->large[G.members[i]].c->plan;
        if (k >= P.fwd.passes.size()) continue;
        if (G.micro) {
          T2Args a;
          QS_TRY(t2args(P, P.fwd, (int)k, i, &a));
          fwd2.push_back(a);
          sm = std::max(sm, P.fwd.passes[k].t2hdr.smem);
        } else {
          fwd.push_back(targs(P, P.fwd, (int)k, i));
        }
      }
      G.fwd_cnt.push_back((G.micro ? (int)fwd2.size() : (int)fwd.size()) - G.fwd_off.back());
      G.fwd_smem.push_back(sm);
    }
    for (size_t k = 0; k < max_r; ++k) {
      G.rev_off.push_back(G.micro ? (int)rev2.size() : (int)rev.size());
      uint32_t sm = 0;
      for (int i = 0; i < cnt; ++i) {
        const CircuitPlan& P = b->large[G.members[i]].c->plan;
        if (k >= P.rev.passes.size()) continue;
        if (G.micro) {
          T2Args a;
          QS_TRY(t2args(P, P.rev, (int)k, i, &a));
          rev2.push_back(a);
          sm = std::max(sm, P.rev.passes[k].t2hdr.smem);
        } else {
          rev.push_back(targs(P, P.rev, (int)k, i));
        }
      }
      G.rev_cnt.push_back((G.micro ? (int)rev2.size() : (int)rev.size()) - G.rev_off.back());
      G.rev_smem.push_back(sm);
    }
    QS_TRY(upload(&G.d_fwd2, fwd2));
    QS_TRY(upload(&G.d_rev2, rev2));
    for (int i = 0; i < cnt; ++i) {
      const BLarge& L = b->large[G.members[i]];
      const CircuitPlan& P = L.c->plan;
      const size_t ns = P.rev_slots.out.size();
      double* part = G.scratch + off[i];
      double* slot = part + std::max<size_t>(ns, 1) * G.grid2;
      double* hpart = slot + ns + 1;
      HamMultiArgs h;
      h.psi = state(G.psi, i);
      h.lam = state(G.lam, i);
      h.groups = L.h->d_groups;
      h.terms = L.h->d_terms;
      h.partials = hpart;
      h.n = G.ne;
      h.n_groups = L.h->n_groups;
      ham.push_back(h);
      rede.push_back(ReduceMultiArgs{hpart, b->d_energy + L.inst, 1, G.hgrid});
      if (ns > 0 && L.n_params > 0) {
        reds.push_back(ReduceMultiArgs{part, slot, (int)ns, G.grid2});
        gath.push_back(GatherMultiArgs{slot, P.d_row, P.d_sidx, P.d_w, b->d_grad + L.param_off, L.n_params, 0});
        G.max_slots = std::max(G.max_slots, (int)ns);
        G.max_params = std::max(G.max_params, L.n_params);
      }
    }
    G.n_red_s = (int)reds.size();
    G.n_gather = (int)gath.size();
    QS_TRY(upload(&G.d_fwd, fwd));
    QS_TRY(upload(&G.d_rev, rev));
    QS_TRY(upload(&G.d_ham, ham));
    QS_TRY(upload(&G.d_red_e, rede));
    QS_TRY(upload(&G.d_red_s, reds));
    QS_TRY(upload(&G.d_gather, gath));
  }
  return QS_OK;
}

}  // namespace

// Enqueue one evaluation of every instance on st (lanes forked and joined).
static qs_status issue_all(qs_batch* b, cudaStream_t st, const double* dev_params, double* dev_energies,
                           double* dev_grads) {
  // large instances: matrices from the device parameters, then each instance's
  // fused passes on a lane (lanes run concurrently with each other and with the
  // persistent kernel)
  if (!b->large.empty()) {
    QS_TRY(launch_batch_coef(b->dt, b->d_cg, b->n_cg, dev_params, st));
    QS_TRY(launch_batch_runs(b->dt, b->d_runs, b->n_runs, b->d_run_members, dev_params, st));
    QS_CUDA(cudaEventRecord(b->ev_fill, st));
    for (BLane& L : b->lanes) QS_CUDA(cudaStreamWaitEvent(L.st, b->ev_fill, 0));
    for (BGroup& G : b->groups) {
      QS_CUDA(cudaStreamWaitEvent(G.st, b->ev_fill, 0));
      QS_TRY(run_group(b, G, dev_energies, dev_grads));
      QS_CUDA(cudaEventRecord(G.done, G.st));
    }
    size_t lane = 0;
    for (size_t k = 0; k < b->large.size(); ++k)
      if (!b->in_group[k]) QS_TRY(run_large(b, b->large[k], b->lanes[lane++ % b->lanes.size()], dev_energies, dev_grads));
    for (BLane& L : b->lanes) QS_CUDA(cudaEventRecord(L.done, L.st));
  }
  if (b->n_small > 0) {
    QS_CUDA(cudaMemsetAsync(b->d_queue, 0, sizeof(int), st));
    BatchArgs a;
    a.inst = b->d_inst;
    a.order = b->d_order;
    a.n_inst = b->n_small;
    a.gates = b->d_gates;
    a.groups = b->d_groups;
    a.terms = b->d_terms;
    a.params = dev_params;
    a.energy = dev_energies;
    a.grad = dev_grads;
    a.queue = b->d_queue;
    a.smem_amps = b->smem_amps;
    a.smem_gates = b->smem_gates;
    a.smem_params = b->smem_params;
    TraceRec* rec = trace_begin(st);
    QS_TRY(launch_batch(b->dt, a, b->grid, st));
    if (rec) {
      rec->bytes = 0;
      rec->kind = QS_TRACE_BATCH;
      QS_CUDA(cudaEventRecord(rec->end, st));
    }
  }
  for (BLane& L : b->lanes) QS_CUDA(cudaStreamWaitEvent(st, L.done, 0));
  for (BGroup& G : b->groups) QS_CUDA(cudaStreamWaitEvent(st, G.done, 0));
  return QS_OK;
}

extern "C" {

qs_status qs_batch_create(int n_inst, const int* n_qubits, const int* gate_offsets, const qs_batch_gate* gates,
                          const int* term_offsets, const uint64_t* xmask, const uint64_t* zmask, const double* coef,
                          const int* param_offsets, qs_dtype dtype, void* cuda_stream, qs_batch** out) {
  QS_CHECK(out != nullptr, "out is null");
  QS_CHECK(n_inst >= 1, "need at least one instance");
  QS_CHECK(n_qubits && gate_offsets && term_offsets && param_offsets, "null offset arrays");
  QS_CHECK(dtype == QS_C64 || dtype == QS_C128, "invalid dtype");
  QS_CHECK(gate_offsets[0] == 0 && term_offsets[0] == 0 && param_offsets[0] == 0, "offsets must start at 0");
  const int max_n = 26;
  std::vector<BInst> inst(n_inst);
  std::vector<BGate> bg;
  std::vector<DevHamGroup> groups;
  std::vector<DevHamTerm> terms;
  const int smem_n = dtype == QS_C64 ? 13 : 12;
  int big_n = 0;
  for (int i = 0; i < n_inst; ++i) {
    const int n = n_qubits[i];
    QS_CHECK(n >= 1 && n <= max_n, "instance qubit count must be in 1..26");
    QS_CHECK(gate_offsets[i + 1] >= gate_offsets[i] && term_offsets[i + 1] >= term_offsets[i] &&
                 param_offsets[i + 1] >= param_offsets[i],
             "offsets must be non-decreasing");
    const int np = param_offsets[i + 1] - param_offsets[i];
    BInst& I = inst[i];
    I.n = n;
    I.gate_begin = (int)bg.size();
    for (int k = gate_offsets[i]; k < gate_offsets[i + 1]; ++k) {
      QS_CHECK(gates != nullptr, "null gates");
      const qs_batch_gate& g = gates[k];
      QS_CHECK(batch_kind_ok(g.kind), "unsupported gate kind in a batch (MATRIX gates are not batched)");
      const int nt = batch_two_target(g.kind) ? 2 : 1;
      QS_CHECK(g.n_targets == nt, "wrong number of targets for this gate kind");
      uint64_t used = 0;
      for (int t = 0; t < nt; ++t) {
        QS_CHECK(g.targets[t] >= 0 && g.targets[t] < n, "target qubit out of range");
        QS_CHECK(!((used >> g.targets[t]) & 1), "duplicate target");
        used |= 1ull << g.targets[t];
      }
      QS_CHECK(g.ctrl_mask < (1ull << n) && !(g.ctrl_mask & used), "control mask out of range or overlaps a target");
      QS_CHECK(g.param >= -1 && g.param < np, "param index outside the instance's parameters");
      QS_CHECK(g.param == -1 || batch_param_ok(g.kind), "only RX/RY/RZ/PS/RXX/RYY/RZZ take a parameter");
      QS_CHECK(std::isfinite(g.coef) && std::isfinite(g.constant), "non-finite angle binding");
      BGate d;
      d.kind = (uint8_t)g.kind;
      d.nt = (uint8_t)nt;
      d.t0 = (uint8_t)g.targets[0];
      d.t1 = (uint8_t)(nt == 2 ? g.targets[1] : g.targets[0]);
      d.param = g.param;
      d.cmask = g.ctrl_mask;
      d.coef = g.coef;
      d.constant = g.constant;
      bg.push_back(d);
    }
    I.gate_end = (int)bg.size();
    // Hamiltonian: group the instance's terms by X mask, coefficient c * i^{#Y}
    std::vector<int> ord;
    for (int k = term_offsets[i]; k < term_offsets[i + 1]; ++k) {
      QS_CHECK(xmask && zmask && coef, "null term arrays");
      QS_CHECK(xmask[k] < (1ull << n) && zmask[k] < (1ull << n), "Pauli mask names a qubit >= the instance's n");
      QS_CHECK(std::isfinite(coef[k]), "non-finite coefficient");
      ord.push_back(k);
    }
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return xmask[a] < xmask[b]; });
    I.group_begin = (int)groups.size();
    const double cr[4] = {1, 0, -1, 0}, ci[4] = {0, 1, 0, -1};
    for (int k : ord) {
      if ((int)groups.size() == I.group_begin || groups.back().xmask != xmask[k]) {
        DevHamGroup G;
        G.xmask = xmask[k];
        G.begin = G.end = (int)terms.size();
        groups.push_back(G);
      }
      const int ny = __builtin_popcountll(xmask[k] & zmask[k]) & 3;
      DevHamTerm t;
      t.zmask = zmask[k];
      t.re = coef[k] * cr[ny];
      t.im = coef[k] * ci[ny];
      terms.push_back(t);
      groups.back().end = (int)terms.size();
    }
    I.group_end = (int)groups.size();
    I.param_off = param_offsets[i];
    I.n_params = np;
    const int max_p = dtype == QS_C64 ? kBatchMaxSmemParams : kBatchMaxSmemParams / 2;
    I.in_smem = (n <= smem_n && I.gate_end - I.gate_begin <= kBatchMaxSmemGates && np <= max_p) ? 1 : 0;
    I.pad = 0;
    I.cost = (double)(3 * (I.gate_end - I.gate_begin) + 2 * (I.group_end - I.group_begin) + 1) * (double)(1ull << n);
    if (!I.in_smem) big_n = std::max(big_n, n);
  }
  qs_batch* b = new qs_batch;
  b->dt = dtype;
  b->st = (cudaStream_t)cuda_stream;
  b->n_inst = n_inst;
  b->n_params_total = param_offsets[n_inst];
  {
    const size_t np = std::max(b->n_params_total, 1);
    cudaError_t e = cudaMalloc(&b->d_params, np * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_grad, np * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_energy, (size_t)n_inst * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_queue, sizeof(int));
    if (e != cudaSuccess) {
      free_batch(b);
      return cuda_fail(e, "cudaMalloc(batch outputs)");
    }
  }
  // shared memory sized for the largest shared-memory instance (more CTAs per SM
  // when all are small)
  int sm_n = 1, sm_g = 1, sm_p = 1;
  for (int i = 0; i < n_inst; ++i)
    if (inst[i].in_smem) {
      sm_n = std::max(sm_n, inst[i].n);
      sm_g = std::max(sm_g, inst[i].gate_end - inst[i].gate_begin);
      sm_p = std::max(sm_p, inst[i].n_params);
    }
  b->smem_amps = 1 << sm_n;
  b->smem_gates = sm_g;
  b->smem_params = sm_p;
  // the persistent kernel's queue holds the shared-memory instances, largest first
  std::vector<int> order;
  for (int i = 0; i < n_inst; ++i)
    if (inst[i].in_smem) order.push_back(i);
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return inst[a].cost > inst[c].cost; });
  b->n_small = (int)order.size();
  qs_status s = QS_OK;
  b->grid = batch_grid_size(dtype, b->smem_amps, b->smem_gates, b->smem_params);
  if (b->grid < 1) {
    free_batch(b);
    set_error("batch: the shared-memory states do not fit");
    return QS_ERR_UNSUPPORTED;
  }
  if (big_n) {
    // instances beyond shared memory: a circuit plan and a Hamiltonian each, run
    // on fused tile passes; their matrices are formed on the device per call
    std::vector<BCoefGate> cg, run_members;
    std::vector<BCoefRun> runs;
    size_t need = 16;
    int max_ne = kRegBits;
    for (int i = 0; i < n_inst; ++i) {
      if (inst[i].in_smem) continue;
      BLarge L;
      L.inst = i;
      L.param_off = param_offsets[i];
      L.n_params = param_offsets[i + 1] - param_offsets[i];
      b->large.push_back(L);
      BLarge& B = b->large.back();
      const int n = inst[i].n;
      if ((s = qs_circuit_create(n, &B.c)) != QS_OK) break;
      for (int k = gate_offsets[i]; k < gate_offsets[i + 1] && s == QS_OK; ++k) {
        const qs_batch_gate& g = gates[k];
        int ctrls[64], nc = 0;
        for (int q = 0; q < n; ++q)
          if ((g.ctrl_mask >> q) & 1ull) ctrls[nc++] = q;
        s = qs_circuit_add(B.c, g.kind, g.targets, g.n_targets, ctrls, nc, g.param, g.coef, g.constant, nullptr);
      }
      if (s == QS_OK) B.c->n_params = std::max(B.c->n_params, param_offsets[i + 1] - param_offsets[i]);
      // default plans: below 22 qubits the interpreter passes (micro-op passes
      // in lock-step groups measured slower there: 2048-instance batch 4970 ->
      // 4235 instances/s), micro-op passes from 22 qubits
      if (s == QS_OK) s = qs_circuit_finalize(B.c, dtype, nullptr);
      if (s == QS_OK) {
        const int t0 = term_offsets[i], nt = term_offsets[i + 1] - t0;
        s = qs_ham_create(n, nt, nt ? xmask + t0 : nullptr, nt ? zmask + t0 : nullptr, nt ? coef + t0 : nullptr, &B.h);
      }
      if (s != QS_OK) break;
      const CircuitPlan& P = B.c->plan;
      for (size_t gi = 0; gi < B.c->gates.size(); ++gi) {
        const HostGate& hg = B.c->gates[gi];
        BCoefGate d;
        d.table = P.d_coef;
        d.off_u = P.off_u[gi];
        d.off_ud = P.off_ud[gi];
        d.off_a = hg.param >= 0 ? P.off_a[gi] : -1;
        d.kind = (uint8_t)hg.kind;
        d.nt = (uint8_t)hg.nt;
        d.diag = (uint8_t)(P.gclass[gi] == GC_DIAG1 || P.gclass[gi] == GC_DIAG2);
        d.pad = 0;
        d.param = hg.param >= 0 ? param_offsets[i] + hg.param : -1;
        d.coef = hg.coef;
        d.constant = hg.constant;
        cg.push_back(d);
      }
      for (size_t r = 0; r < P.runs.size(); ++r) {
        BCoefRun R;
        R.table = P.d_coef;
        R.off = P.run_off[r];
        R.begin = (int)run_members.size();
        R.count = (int)P.runs[r].size();
        R.diag = P.run_diag[r] ? 1 : 0;
        for (int gi : P.runs[r]) {
          const HostGate& hg = B.c->gates[gi];
          BCoefGate d{};
          d.kind = (uint8_t)hg.kind;
          d.nt = 1;
          d.param = hg.param >= 0 ? param_offsets[i] + hg.param : -1;
          d.coef = hg.coef;
          d.constant = hg.constant;
          run_members.push_back(d);
        }
        runs.push_back(R);
      }
      const size_t n_slots = P.rev_slots.out.size();
      need = std::max(need, std::max<size_t>(n_slots, 1) * P.grid2 + n_slots + 1 +
                                (size_t)ham_grid_size(P.ne) + 16);
      max_ne = std::max(max_ne, P.ne);
    }
    if (s == QS_OK) s = upload(&b->d_cg, cg);
    b->n_cg = (int)cg.size();
    if (s == QS_OK) s = upload(&b->d_runs, runs);
    if (s == QS_OK) s = upload(&b->d_run_members, run_members);
    b->n_runs = (int)runs.size();
    if (s == QS_OK) {
      // instances of 14-17 qubits have only 4-32 tiles per pass: many lanes in
      // flight keep the SMs busy; the largest instances are dealt out first
      std::stable_sort(b->large.begin(), b->large.end(),
                       [&](const BLarge& x, const BLarge& y) { return inst[x.inst].cost > inst[y.inst].cost; });
      s = build_groups(b);
    }
    if (s == QS_OK) {
      int rest = 0;
      for (char g : b->in_group) rest += !g;
      const int n_lanes = std::min<int>(kBatchLanes, rest);
      const size_t state_bytes = amp_bytes(dtype) << max_ne;
      cudaError_t e = cudaEventCreateWithFlags(&b->ev_fill, cudaEventDisableTiming);
      for (int l = 0; l < n_lanes && e == cudaSuccess; ++l) {
        b->lanes.emplace_back();
        BLane& L = b->lanes.back();
        e = cudaStreamCreateWithFlags(&L.st, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMalloc(&L.psi, state_bytes);
        if (e == cudaSuccess) e = cudaMalloc(&L.lam, state_bytes);
        if (e == cudaSuccess) e = cudaMalloc(&L.scratch, need * sizeof(double));
      }
      if (e != cudaSuccess) s = cuda_fail(e, "batch lanes");
    }
    if (s != QS_OK) {
      free_batch(b);
      return s;
    }
  }
  if ((s = upload(&b->d_inst, inst)) != QS_OK || (s = upload(&b->d_order, order)) != QS_OK ||
      (s = upload(&b->d_gates, bg)) != QS_OK || (s = upload(&b->d_groups, groups)) != QS_OK ||
      (s = upload(&b->d_terms, terms)) != QS_OK) {
    free_batch(b);
    return s;
  }
  *out = b;
  return QS_OK;
}

qs_status qs_batch_destroy(qs_batch* b) {
  if (!b) return QS_OK;
  cudaDeviceSynchronize();
  free_batch(b);
  return QS_OK;
}

qs_status qs_batch_info(const qs_batch* b, int* n_instances, int* n_params, int* grid) {
  QS_CHECK(b != nullptr, "null batch");
  if (n_instances) *n_instances = b->n_inst;
  if (n_params) *n_params = b->n_params_total;
  if (grid) *grid = b->grid;
  return QS_OK;
}

qs_status qs_batch_expectation_with_grad_device(qs_batch* b, const double* dev_params, double* dev_energies,
                                                double* dev_grads) {
  QS_CHECK(b != nullptr, "null batch");
  QS_CHECK(dev_energies != nullptr && (b->n_params_total == 0 || (dev_params && dev_grads)), "null argument");
  // Many large instances mean tens of thousands of small launches: capture the
  // call once as a graph on the batch's own buffers and replay it (not while
  // launches are being traced, whose events must stay per launch).
  if (!b->large.empty() && !trace_active() && !b->graph_failed) {
    if (!b->graph) {
      cudaGraph_t g = nullptr;
      qs_status s = QS_OK;
      if (cudaStreamCreateWithFlags(&b->cap_st, cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess ||
          cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) != cudaSuccess ||
          cudaStreamBeginCapture(b->cap_st, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
        s = QS_ERR_CUDA;
      } else {
        s = issue_all(b, b->cap_st, b->d_params, b->d_energy, b->d_grad);
        if (cudaStreamEndCapture(b->cap_st, &g) != cudaSuccess) s = QS_ERR_CUDA;
      }
      if (s == QS_OK && cudaGraphInstantiate(&b->graph, g, 0) != cudaSuccess) s = QS_ERR_CUDA;
      if (g) cudaGraphDestroy(g);
      if (s != QS_OK) {
        (void)cudaGetLastError();
        b->graph = nullptr;
        b->graph_failed = true;  // fall back to direct launches from now on
      }
    }
    if (b->graph) {
      // ordered after the caller's stream, and the caller's stream after it
      const size_t np = (size_t)b->n_params_total * sizeof(double);
      QS_CUDA(cudaEventRecord(b->ev_in, b->st));
      QS_CUDA(cudaStreamWaitEvent(b->cap_st, b->ev_in, 0));
      if (np && dev_params != b->d_params)
        QS_CUDA(cudaMemcpyAsync(b->d_params, dev_params, np, cudaMemcpyDeviceToDevice, b->cap_st));
      QS_CUDA(cudaGraphLaunch(b->graph, b->cap_st));
      if (dev_energies != b->d_energy)
        QS_CUDA(cudaMemcpyAsync(dev_energies, b->d_energy, (size_t)b->n_inst * sizeof(double),
                                cudaMemcpyDeviceToDevice, b->cap_st));
      if (np && dev_grads != b->d_grad)
        QS_CUDA(cudaMemcpyAsync(dev_grads, b->d_grad, np, cudaMemcpyDeviceToDevice, b->cap_st));
      QS_CUDA(cudaEventRecord(b->ev_out, b->cap_st));
      QS_CUDA(cudaStreamWaitEvent(b->st, b->ev_out, 0));
      return QS_OK;
    }
  }
  // direct launches: the argument tables of the lock-step groups name the
  // batch's own buffers, so the call goes through them
  const size_t np = (size_t)b->n_params_total * sizeof(double);
  if (np && dev_params != b->d_params)
    QS_CUDA(cudaMemcpyAsync(b->d_params, dev_params, np, cudaMemcpyDeviceToDevice, b->st));
  QS_TRY(issue_all(b, b->st, b->d_params, b->d_energy, b->d_grad));
  if (dev_energies != b->d_energy)
    QS_CUDA(cudaMemcpyAsync(dev_energies, b->d_energy, (size_t)b->n_inst * sizeof(double), cudaMemcpyDeviceToDevice,
                            b->st));
  if (np && dev_grads != b->d_grad)
    QS_CUDA(cudaMemcpyAsync(dev_grads, b->d_grad, np, cudaMemcpyDeviceToDevice, b->st));
  return QS_OK;
}

qs_status qs_batch_expectation_with_grad(qs_batch* b, const double* params, double* energies, double* grads) {
  QS_CHECK(b != nullptr, "null batch");
  QS_CHECK(energies != nullptr && (b->n_params_total == 0 || (params && grads)), "null argument");
  if (b->n_params_total)
    QS_CUDA(cudaMemcpyAsync(b->d_params, params, b->n_params_total * sizeof(double), cudaMemcpyHostToDevice, b->st));
  QS_TRY(qs_batch_expectation_with_grad_device(b, b->d_params, b->d_energy, b->d_grad));
  QS_CUDA(cudaMemcpyAsync(energies, b->d_energy, b->n_inst * sizeof(double), cudaMemcpyDeviceToHost, b->st));
  if (b->n_params_total)
    QS_CUDA(cudaMemcpyAsync(grads, b->d_grad, b->n_params_total * sizeof(double), cudaMemcpyDeviceToHost, b->st));
  QS_CUDA(cudaStreamSynchronize(b->st));
  return QS_OK;
}

}  // extern "C"
