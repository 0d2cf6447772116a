// Internal types shared by the host runtime (api.cu, plan.cu) and the kernels.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "qsim.h"
#include "t2_types.h"

namespace qs {

// ----------------------------------------------------------------------------- limits
constexpr int kMaxQubits = 34;
constexpr int kRegBits = 4;          // amplitudes per thread in a tile phase = 2^kRegBits
constexpr int kTileThreads = 256;    // threads of a fused tile CTA
constexpr int kTileWarps = kTileThreads / 32;
constexpr int kMaxTileBits = 13;     // 2^13 amplitudes per tile
// Largest tile whose two-state (psi, lam) pass fits in shared memory.
constexpr int max_tile_bits(qs_dtype dt) { return dt == QS_C64 ? 13 : 12; }
constexpr int kMinTileBits = 6;
constexpr int kMicroMinQubits = 22;  // default use of the complex64 micro-op tile passes
constexpr int kMaxSlotsPerPass = 256;  // gradient/energy accumulators of one launch
constexpr int kMaxPhasesPerPass = 64;
constexpr int kSmallMaxBytes = 96 * 1024;  // per-state bytes of the one-CTA engine

// ----------------------------------------------------------------------------- ops
// One instruction of a fused tile pass.  Register bits rb0/rb1 index the
// phase's register set (the 2^kRegBits amplitudes a thread holds at a time).
enum OpType : uint8_t {
  OP_DENSE1 = 1,    // 2x2 complex matrix on register bit rb0
  OP_DENSE2 = 2,    // 4x4 on register bits (rb0 = targets[0], rb1 = targets[1])
  OP_DIAG = 3,      // diagonal D[b0 + 2 b1] on up to two qubits (any bit of the index)
  OP_RX = 4,        // [[c, -is], [-is, c]] on rb0; coef = (c, s)
  OP_GRAD1 = 5,     // acc += 2 Re <lam| A |psi>, A 2x2 on rb0
  OP_GRAD2 = 6,     // acc += 2 Re <lam| A |psi>, A 4x4 on (rb0, rb1)
  OP_GRADDIAG = 7,  // acc += 2 Re <lam| D |psi>, D diagonal as OP_DIAG
  OP_GRADX = 8,     // acc += Im <lam| X_rb0 |psi>
  OP_COST = 9,      // psi_x *= lut[cut(x)]
  OP_GRADCOST = 10, // acc += C(x) Im(conj(lam_x) psi_x), C = n_edges - 2 cut
  OP_ENERGY = 11,   // acc += C(x) |psi_x|^2 and lam_x = C(x) psi_x
  OP_X = 12,        // X on rb0, complex128 one-state passes: a swap of the amplitude pairs (controls as OP_DENSE1)
  OP_REAL1 = 13,    // as OP_DENSE1 with real entries (H, RY; complex128 one-state passes): half the FP64 work
  OP_UDIAG = 14,    // as OP_DIAG with entries in {1, i, -1, -i} (Z, S, CZ; complex128 one-state passes): no FP64 work
  OP_ZFLIP = 15     // diag(1, -1) on one target (Z, CZ): a sign flip (lowered to OP_UDIAG / OP_DIAG for the
                    // interpreter kernel)
};

enum OpFlags : uint8_t { OPF_LAM = 1 };  // apply to lam as well as psi

struct DevOp {
  uint8_t type;
  uint8_t rb0, rb1;
  uint8_t flags;
  uint16_t jc;       // control bits that are register bits (mask over register index)
  uint16_t slot;     // accumulator slot within the launch
  uint32_t lc;       // control bits that are tile bits but not register bits (local mask)
  uint32_t coef;     // index of the first complex coefficient
  int8_t dloc[2];    // OP_DIAG/GRADDIAG: local bit of qubit 0/1, or -1
  int8_t dglb[2];    // ... or global bit (outside the tile), or -1
  uint32_t pad;
  uint64_t gc;       // control bits outside the tile (checked on the tile offset)
};

struct DevPhase {
  int8_t R[kRegBits];  // local bits held in registers (register bit i <-> local bit R[i])
  int8_t Q[16];        // local bits enumerated by the sub-cube index, low to high
  int16_t nq;
  int16_t pad;
  int op_begin, op_end;
};

struct DevPass {
  int m;          // tile bits
  int c;          // low contiguous bits (local bit i = global bit i for i < c)
  int n_phases;
  int phase_begin;
  int ncomp;      // global bits not in the tile
  uint32_t flags;
  int n_slots;
  int slot_base;
  int8_t comp[40];
  uint64_t hiA[64];  // deposit of local bits c..c+5 into their global positions
  uint64_t hiB[128]; // deposit of local bits c+6..c+12
};

// ----------------------------------------------------------------------------- host plans
struct HostGate {
  int kind;
  int nt;
  int t[2];
  std::vector<int> ctrls;
  int param;
  double coef, constant;
  std::vector<double> matrix;  // interleaved complex, for QS_GATE_MATRIX
};

// Class of a gate for the engines: which tile-pass op realises it.
enum GateClass { GC_DENSE1, GC_DENSE2, GC_DIAG1, GC_DIAG2 };

struct PlannedPass {
  DevPass hdr;
  std::vector<DevPhase> phases;
  std::vector<DevOp> ops;
  // the micro-op form, when the pass qualifies (complex64, 4 low bits, a
  // five-dimensional tile map, shared-memory budget)
  bool t2 = false;
  T2Pass t2hdr;
  std::vector<T2Phase> t2ph;
  std::vector<T2Op> t2ops;
};

// A compiled sequence of tile passes plus the coefficient recipe to fill per call.
struct TilePlan {
  int n = 0;
  qs_dtype dtype = QS_C64;
  int m = 0, c = 0;
  std::vector<PlannedPass> passes;
  int n_coef = 0;  // complex coefficients per call
  int n_slots = 0;
  // device copies
  DevPass* d_pass = nullptr;
  DevPhase* d_phase = nullptr;
  DevOp* d_ops = nullptr;
  T2Pass* d_t2pass = nullptr;   // per pass (unused entries for passes without the micro-op form)
  T2Phase* d_t2ph = nullptr;
  T2Op* d_t2ops = nullptr;
  std::vector<int> t2_phase_off, t2_op_off;  // per pass: first phase / op in the device arrays
  // per-circuit kernels (t2gen.cu), compiled at upload: gen = 1 for the
  // micro-op passes within the compile budget (t2gen_budget_ops), 2 for every
  // micro-op pass; the kernel of pass i in gen_fn[i] (null: the library's
  // micro-op kernel, the same arithmetic)
  int gen = 0;
  std::vector<void*> gen_fn;
  void free_device();
  qs_status upload(cudaStream_t st);
};

// ----------------------------------------------------------------------------- kernel launchers
struct TileLaunch {
  void* psi;
  void* lam;
  const void* coef;
  const uint8_t* cut;
  double* partials;  // [n_slots_total][grid]
  int n;
  int n_edges;
  int grid;    // CTAs of this launch
  int stride;  // stride of the partials array (the plan's 2-state grid)
};

// Kernel arguments of one instance's tile pass (device layout).
struct TileKArgs {
  void* psi;
  void* lam;
  const DevPass* pass;
  const DevPhase* phases;
  const DevOp* ops;
  const void* coef;
  const uint8_t* cut;
  double* partials;
  int n;
  int n_edges;
  int grid_stride;  // stride of the partials array (the plan's grid)
};
// The same pass index of `count` independent instances with equal tile bits m
// and equal grid, in one launch (interpreter kernel): instance i's arguments in
// d_argv[i].
qs_status launch_tile_pass_multi(qs_dtype dt, int ns, int m, const TileKArgs* d_argv, int count, int grid,
                                 cudaStream_t st);
qs_status launch_tile2_pass(const TilePlan& plan, int pass_index, const TileLaunch& L, cudaStream_t st);
qs_status make_tile2_args(const TilePlan& plan, int pass_index, void* psi, void* lam, const void* coef,
                          double* partials, int stride, int cols, int n, T2Args* out);
// Pass arguments of `count` instances (d_argv, 64-byte aligned), grid_x CTAs per
// instance, each looping over its share of the instance's tiles.
qs_status launch_tile2_multi(int ns, const T2Args* d_argv, int count, int grid_x, uint32_t smem, cudaStream_t st);
qs_status launch_tile_pass(qs_dtype dt, const TilePlan& plan, int pass_index, const TileLaunch& L,
                           cudaStream_t st);
int tile_grid_size(qs_dtype dt, int m, int ns, int n_tiles);
size_t tile_smem_bytes(qs_dtype dt, int m, int ns);

// Per-gate (unfused) kernels.
qs_status launch_gate_dense(qs_dtype dt, void* psi, int n, int nt, const int* t, uint64_t cmask,
                            const double* mat /* interleaved complex (2^nt)^2 */, cudaStream_t st);
qs_status launch_gate_diag(qs_dtype dt, void* psi, int n, int nt, const int* t, uint64_t cmask,
                           const double* diag /* interleaved complex 2^nt */, cudaStream_t st);

// States.
qs_status launch_set_basis(qs_dtype dt, void* psi, int n, uint64_t index, cudaStream_t st);
qs_status launch_set_plus(qs_dtype dt, void* psi, int n, cudaStream_t st);

// Hamiltonians: groups of terms sharing an X mask.
struct DevHamTerm {
  uint64_t zmask;
  double re, im;  // coef * i^{#Y}
};
struct DevHamGroup {
  uint64_t xmask;
  int begin, end;
};
qs_status launch_ham_apply(qs_dtype dt, const void* psi, void* lam /* nullable */, int n,
                           const DevHamGroup* groups, int n_groups, const DevHamTerm* terms,
                           double* partials, int grid, cudaStream_t st);
int ham_grid_size(int n);
qs_status launch_inner(qs_dtype dt, const void* a, const void* b, int n, double* partials /* [2][grid] */,
                       int grid, cudaStream_t st);
qs_status launch_norm2(qs_dtype dt, const void* a, int n, double* partials, int grid, cudaStream_t st);
// out[s] = sum_b partials[s * nb + b] * scale[s] (scale nullable), fixed order.
qs_status launch_reduce_slots(const double* partials, int n_slots, int nb, const double* scale,
                              double* out, cudaStream_t st);
// grad[p] = sum over gates g of param p: coef_g * gate_grad[g]  (CSR by parameter)
qs_status launch_param_gather(const double* gate_grad, const int* row_ptr, const int* gate_idx,
                              const double* gate_coef, int n_params, double* grad, cudaStream_t st);

// QAOA
qs_status launch_cut_values(uint8_t* cut, int n, const int* d_edges, int n_edges, cudaStream_t st);
// *d_out = max of v[0..n) (bytes); v 16-byte aligned
qs_status launch_max_u8(const uint8_t* v, uint64_t n, int* d_out, cudaStream_t st);

// Sampling
qs_status launch_sample(qs_dtype dt, const void* psi, int n, uint64_t shots, uint64_t seed,
                        double* scratch /* cdf of block sums */, uint64_t* d_out, cudaStream_t st);
size_t sample_scratch_doubles(int n);
// Projective measurement of qubit q: scratch holds 2 nb + 2 doubles; afterwards
// scratch[2 nb] = outcome, scratch[2 nb + 1] = 1/sqrt(P(outcome)).
qs_status launch_measure(qs_dtype dt, void* psi, int n, int q, uint64_t seed, double* scratch, int nb,
                         cudaStream_t st);

// Batched forms of the Hamiltonian apply, slot reduction and parameter gather:
// one launch, instance blockIdx.y.
struct HamMultiArgs {
  const void* psi;
  void* lam;
  const DevHamGroup* groups;
  const DevHamTerm* terms;
  double* partials;
  int n, n_groups;
};
struct ReduceMultiArgs {
  const double* partials;
  double* out;
  int n_slots, nb;
};
struct GatherMultiArgs {
  const double* gate_grad;
  const int* row_ptr;
  const int* gate_idx;
  const double* gate_coef;
  double* grad;
  int n_params, pad;
};
qs_status launch_ham_apply_multi(qs_dtype dt, const HamMultiArgs* d_argv, int count, int grid, cudaStream_t st);
qs_status launch_reduce_multi(const ReduceMultiArgs* d_argv, int count, int max_slots, cudaStream_t st);
qs_status launch_gather_multi(const GatherMultiArgs* d_argv, int count, int max_params, cudaStream_t st);
// psi_i = |0...0> for count states of 2^n amplitudes stored back to back
qs_status launch_set_zero_multi(qs_dtype dt, void* base, int n, int count, cudaStream_t st);


// ----------------------------------------------------------------------------- errors
void set_error(const std::string& msg);
qs_status cuda_fail(cudaError_t e, const char* what);

#define QS_CUDA(call)                                  \
  do {                                                 \
    cudaError_t _e = (call);                           \
    if (_e != cudaSuccess) return qs::cuda_fail(_e, #call); \
  } while (0)

#define QS_CHECK(cond, msg)                   \
  do {                                        \
    if (!(cond)) {                            \
      qs::set_error(msg);                     \
      return QS_ERR_INVALID_ARG;              \
    }                                         \
  } while (0)

#define QS_TRY(expr)                  \
  do {                                \
    qs_status _s = (expr);            \
    if (_s != QS_OK) return _s;       \
  } while (0)

}  // namespace qs
