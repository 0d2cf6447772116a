// Batched engine: many independent (circuit, Hamiltonian, parameters)
// instances evaluated (energy + adjoint gradient) in one persistent launch.
#pragma once

#include "qsim_internal.h"

namespace qs {

constexpr int kBatchThreads = 256;
// dynamic shared memory one CTA of the batched or trajectory kernels may use
constexpr size_t kBatchSmemBudget = 220 * 1024;
// instances with more gates or parameters than these run on fused tile passes
constexpr int kBatchMaxSmemGates = 1024;
constexpr int kBatchMaxSmemParams = 512;

// One gate of a batched circuit (device layout, 32 bytes).
struct BGate {
  uint8_t kind;   // qs_gate_kind (MATRIX is not supported in batches)
  uint8_t nt;     // targets (1 or 2)
  uint8_t t0, t1;
  int32_t param;  // -1: fixed angle
  uint64_t cmask;
  double coef, constant;
};

struct BInst {
  int n;
  int gate_begin, gate_end;
  int group_begin, group_end;  // Hamiltonian groups (terms sharing an X mask)
  int param_off, n_params;     // slice of the concatenated parameter / gradient arrays
  int in_smem;                 // psi and lam fit in shared memory (else: fused tile passes)
  int pad;
  double cost;                 // work estimate used to order the queue
};

struct BatchArgs {
  const BInst* inst;
  const int* order;        // instance indices by decreasing cost
  int n_inst;
  const BGate* gates;
  const DevHamGroup* groups;
  const DevHamTerm* terms;
  const double* params;    // concatenated
  double* energy;          // [n_inst]
  double* grad;            // concatenated, like params
  int* queue;              // work counter (zeroed before the launch)
  int smem_amps;           // amplitudes per state in shared memory
  int smem_gates;          // gate-data entries in shared memory (the most gates of an instance)
  int smem_params;         // gradient slots in shared memory (the most parameters of an instance)
};

qs_status launch_batch(qs_dtype dt, const BatchArgs& a, int grid, cudaStream_t st);

// One gate of an instance that runs on fused tile passes: where its matrices go
// in that instance's coefficient table (the layout the tile planner assigned).
struct BCoefGate {
  void* table;    // the instance's coefficient table (complex of the batch dtype)
  int off_u, off_ud, off_a;  // U, U^dag and (parametric gates) A = dU U^dag; -1 = none
  uint8_t kind, nt, diag, pad;
  int param;      // index into the concatenated parameters, -1 = fixed angle
  double coef, constant;
};
// Fill the tables of every such gate from the device parameters.
qs_status launch_batch_coef(qs_dtype dt, const BCoefGate* g, int n, const double* params, cudaStream_t st);

// A run of single-qubit gates fused into one 2x2 op of a forward pass: its
// product (members[begin .. begin + count), in circuit order) goes to table[off].
struct BCoefRun {
  void* table;
  int off;
  int begin, count;
  int diag;  // store the two diagonal entries only
};
qs_status launch_batch_runs(qs_dtype dt, const BCoefRun* runs, int n, const BCoefGate* members,
                            const double* params, cudaStream_t st);
int batch_grid_size(qs_dtype dt, int smem_amps, int smem_gates, int smem_params);

// Monte-Carlo trajectories of one noisy circuit (the state-vector treatment of
// channels, §3.3): each trajectory samples one branch operator per channel site
// and runs in one CTA's shared memory.  A site is a BGate of kind kGateChannel
// whose param is the site index.
constexpr int kGateChannel = 250;
constexpr int kTrajMaxSites = 4096;
constexpr int kTrajMaxKraus = 4;
struct BChannel {
  double K[kTrajMaxKraus][8];  // branch operators, 2x2 (re, im) row-major
  double w[kTrajMaxKraus];     // fixed branch weights (fixed = 1)
  int n_kraus;
  int fixed;  // 1: weights w and unitary branch operators (Pauli, depolarizing);
              // 0: w_i = ||K_i psi||^2, branch operator K_i / sqrt(w_i)
  int qubit;
  int pad;
};
struct TrajArgs {
  const BGate* gates;
  const BChannel* ch;
  const DevHamGroup* groups;
  const DevHamTerm* terms;
  const double* params;
  double* energy;     // [n_traj]
  double* grad;       // [n_traj * n_params] (gradient kernel)
  uint8_t* choice;    // [n_traj * n_sites] branches taken, or null
  void* state_out;    // final state of the launch's first trajectory, or null
  int* queue;         // work counter (zeroed before the launch)
  uint64_t seed;
  long long first;    // global index of the launch's first trajectory
  int n_traj, n, n_gates, n_sites, n_params, n_groups;
};
qs_status launch_traj(qs_dtype dt, bool grad, const TrajArgs& a, int grid, cudaStream_t st);
int traj_grid_size(qs_dtype dt, bool grad, int n, int n_gates, int n_params);
size_t traj_smem_bytes(qs_dtype dt, bool grad, int n, int n_gates, int n_params);
// out[c] = (sum over r of rows[r * n_cols + c]) / n_rows, rows summed in order.
qs_status launch_row_mean(const double* rows, int n_rows, int n_cols, double* out, cudaStream_t st);
size_t batch_smem_bytes(qs_dtype dt, int smem_amps, int smem_gates, int smem_params);
// Reduced density matrix of qubit q of psi (2^n amplitudes): partials[4][grid] =
// per-CTA FP64 sums of |a0|^2, |a1|^2, Re a0 conj(a1), Im a0 conj(a1) over the
// pairs (a0, a1) = (psi[x], psi[x | 2^q]).
qs_status launch_qubit_rdm(qs_dtype dt, const void* psi, int n, int q, double* partials, int grid,
                           cudaStream_t st);

}  // namespace qs
