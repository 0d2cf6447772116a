// Host side of the batched engine: argument checks, device tables, queue order.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "batch.h"
#include "handles.h"

using namespace qs;

struct qs_batch {
  qs_dtype dt = QS_C64;
  cudaStream_t st = nullptr;
  int n_inst = 0;
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
  void* d_slots = nullptr;
  size_t slot_amps = 0;
  int smem_amps = 0;
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
  for (void* p : {(void*)b->d_inst, (void*)b->d_order, (void*)b->d_gates, (void*)b->d_groups, (void*)b->d_terms,
                  (void*)b->d_params, (void*)b->d_energy, (void*)b->d_grad, (void*)b->d_queue, b->d_slots})
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

}  // namespace

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
    I.in_smem = n <= smem_n ? 1 : 0;
    I.pad = 0;
    I.cost = (double)(3 * (I.gate_end - I.gate_begin) + 2 * (I.group_end - I.group_begin) + 1) * (double)(1ull << n);
    if (!I.in_smem) big_n = std::max(big_n, n);
  }
  qs_batch* b = new qs_batch;
  b->dt = dtype;
  b->st = (cudaStream_t)cuda_stream;
  b->n_inst = n_inst;
  b->n_params_total = param_offsets[n_inst];
  b->smem_amps = 1 << smem_n;
  std::vector<int> order(n_inst);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return inst[a].cost > inst[c].cost; });
  qs_status s = QS_OK;
  b->grid = batch_grid_size(dtype, b->smem_amps);
  if (b->grid < 1) {
    free_batch(b);
    set_error("batch: the shared-memory states do not fit");
    return QS_ERR_UNSUPPORTED;
  }
  if (big_n) {
    // per-CTA slots for psi and lam of the largest instance kept in global memory;
    // fewer CTAs if the slots would take more than a quarter of the free memory
    b->slot_amps = 1ull << big_n;
    const size_t per_cta = 2 * b->slot_amps * (dtype == QS_C64 ? 8 : 16);
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    const size_t cap = std::max<size_t>(1, (free_b / 4) / per_cta);
    if ((size_t)b->grid > cap) b->grid = (int)cap;
    cudaError_t e = cudaMalloc(&b->d_slots, per_cta * b->grid);
    if (e != cudaSuccess) {
      free_batch(b);
      return cuda_fail(e, "cudaMalloc(batch slots)");
    }
  }
  if ((s = upload(&b->d_inst, inst)) != QS_OK || (s = upload(&b->d_order, order)) != QS_OK ||
      (s = upload(&b->d_gates, bg)) != QS_OK || (s = upload(&b->d_groups, groups)) != QS_OK ||
      (s = upload(&b->d_terms, terms)) != QS_OK) {
    free_batch(b);
    return s;
  }
  const size_t np = std::max(b->n_params_total, 1);
  cudaError_t e = cudaMalloc(&b->d_params, np * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_grad, np * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_energy, (size_t)n_inst * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_queue, sizeof(int));
  if (e != cudaSuccess) {
    free_batch(b);
    return cuda_fail(e, "cudaMalloc(batch outputs)");
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
  QS_CUDA(cudaMemsetAsync(b->d_queue, 0, sizeof(int), b->st));
  BatchArgs a;
  a.inst = b->d_inst;
  a.order = b->d_order;
  a.n_inst = b->n_inst;
  a.gates = b->d_gates;
  a.groups = b->d_groups;
  a.terms = b->d_terms;
  a.params = dev_params;
  a.energy = dev_energies;
  a.grad = dev_grads;
  a.queue = b->d_queue;
  a.slots = b->d_slots;
  a.slot_amps = b->slot_amps;
  a.smem_amps = b->smem_amps;
  TraceRec* rec = trace_begin(b->st);
  QS_TRY(launch_batch(b->dt, a, b->grid, b->st));
  if (rec) {
    rec->bytes = 0;
    rec->kind = QS_TRACE_BATCH;
    QS_CUDA(cudaEventRecord(rec->end, b->st));
  }
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
