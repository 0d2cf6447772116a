// Opaque handle types behind the C ABI and the host helpers shared by api.cu
// and qaoa.cu.
#pragma once

#include <vector>

#include "plan.h"
#include "qsim_internal.h"

using namespace qs;


struct qs_state {
  int n = 0;   // qubits as created
  int ne = 0;  // qubits of the stored array (n padded up to kRegBits)
  qs_dtype dt = QS_C64;
  void* ptr = nullptr;
  bool owned = false;
  size_t bytes = 0;
  cudaStream_t st = nullptr;
  double* scratch = nullptr;
  size_t scratch_n = 0;
  void* save = nullptr;  // copy of the evolved state (several Hamiltonians in one gradient call)
  std::vector<double> host_out;
};

struct CircuitPlan {
  bool valid = false;
  qs_dtype dt = QS_C64;
  int fuse = 1, m = 0, c = 0, ne = 0;
  TilePlan fwd, rev;
  SlotMap rev_slots;
  std::vector<int> off_u, off_ud, off_a, gclass;
  // forward passes: runs of single-qubit, uncontrolled gates on one qubit with
  // nothing else on that qubit in between become one 2x2 op (product of the run)
  std::vector<int> run_head;                 // gate -> first gate of its run, -1 if not absorbed
  std::vector<std::vector<int>> runs;        // runs of >= 2 gates, in circuit order
  std::vector<int> run_off;                  // coefficient offset of each run's product
  std::vector<char> run_diag;                // every gate of the run is diagonal
  int n_coef = 0;
  void* d_coef = nullptr;
  int* d_row = nullptr;
  int* d_sidx = nullptr;
  double* d_w = nullptr;
  int n_params = 0;
  int grid1 = 1, grid2 = 1;
  // adjoint checkpoints: segment ends (pass indices) of the forward plan in
  // circuit order and of the reverse plan in reverse order, and one saved state
  // per inner segment boundary
  std::vector<int> fwd_seg_end, rev_seg_end;
  std::vector<void*> ckpt;
  void release() {
    for (void* b : ckpt) cudaFree(b);
    ckpt.clear();
    fwd_seg_end.clear();
    rev_seg_end.clear();
    fwd.free_device();
    rev.free_device();
    if (d_coef) cudaFree(d_coef);
    if (d_row) cudaFree(d_row);
    if (d_sidx) cudaFree(d_sidx);
    if (d_w) cudaFree(d_w);
    d_coef = nullptr;
    d_row = d_sidx = nullptr;
    d_w = nullptr;
    fwd = TilePlan();
    rev = TilePlan();
    rev_slots = SlotMap();
    valid = false;
  }
};

struct qs_circuit {
  int n = 0;
  int dm_n = 0;               // > 0: a density-matrix circuit of dm_n qubits (2 dm_n stored)
  bool has_channel = false;   // holds a channel (non-unitary): no adjoint gradient
  bool fuse_1q = true;        // forward passes merge runs of single-qubit gates into one 2x2 op
  std::vector<HostGate> gates;
  int n_params = 0;
  qs_options opts{};
  CircuitPlan plan;
  std::vector<double> host_coef;  // staging of the per-call coefficient table
};

struct qs_ham {
  int n = 0;
  std::vector<uint64_t> x, z;
  std::vector<double> c;
  DevHamGroup* d_groups = nullptr;
  DevHamTerm* d_terms = nullptr;
  int n_groups = 0;
};


namespace qs {
struct TraceRec {
  cudaEvent_t start, end;
  double bytes;
  int kind;  // qs_trace_kind
};
// Event pair for the next launch on `st` when tracing is on, else nullptr.
TraceRec* trace_begin(cudaStream_t st);
bool trace_active();
qs_status trace_enable(int on);
qs_status trace_read(int max, int* n, double* ms, double* bytes, int* kinds);
qs_status ensure_scratch(qs_state* s, size_t ndoubles);
qs_status upload_table(const std::vector<double>& tab, qs_dtype dt, void* d_dst, cudaStream_t st,
                       std::vector<double>& staging);
qs_status build_csr(const SlotMap& sm, int n_out, int** d_row, int** d_sidx, double** d_w, cudaStream_t st);
qs_status run_passes(const TilePlan& plan, int begin, int end, qs_dtype dt, void* psi, void* lam, const void* coef,
                     const uint8_t* cut, double* partials, int n, int n_edges, int grid1, int grid2, cudaStream_t st);
qs_status check_state(const qs_state* s);
size_t amp_bytes(qs_dtype dt);
}  // namespace qs
