/*
 * qsim.h -- C ABI of the GB300 state-vector engine for variational quantum
 * algorithms (MindSpore Quantum whitepaper, arXiv 2406.17248).
 *
 * Conventions shared by every call
 * --------------------------------
 * - A state of n qubits is 2^n complex amplitudes, little endian: qubit q is
 *   bit q of the amplitude index (§2.6 "Basic Usage of Simulator").  Storage is
 *   interleaved (re, im): float2 for QS_C64 (complex64), double2 for QS_C128
 *   (complex128) (§2.1 "Data Type").
 * - Every call returns a qs_status; nothing aborts.  On an error the call has
 *   not modified any output, and qs_last_error() returns a message (thread-local,
 *   valid until the next failing call on that thread).  Arguments are checked on
 *   the host before any launch.
 * - Device work is enqueued on the CUDA stream given at qs_state_create (the
 *   state's stream).  Calls that return host values (energies, gradients,
 *   samples, copies to host) synchronise that stream before returning; all
 *   other calls are asynchronous with respect to the host.
 * - Energies, gradients and inner products are returned in FP64 for both
 *   dtypes; complex64 reductions accumulate in FP32 per thread over a bounded
 *   run, then in FP64 in a fixed order, so results are bitwise repeatable for a
 *   given launch configuration.
 * - Pointers named dev_* are device pointers; every other pointer is host.
 * - Handles are opaque and owned by the library; *_destroy frees them.
 *   Device buffers passed in by the caller stay owned by the caller.
 */
#ifndef QSIM_H
#define QSIM_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define QS_API __attribute__((visibility("default")))
#else
#define QS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  QS_OK = 0,
  QS_ERR_INVALID_ARG = 1,   /* bad handle, qubit index, size or mismatched n/dtype */
  QS_ERR_OUT_OF_MEMORY = 2, /* a library allocation failed */
  QS_ERR_CUDA = 3,          /* a CUDA runtime call failed (message has the CUDA error) */
  QS_ERR_TIMEOUT = 4,       /* a bounded device-side wait ran out */
  QS_ERR_UNSUPPORTED = 5    /* valid request outside what this build implements */
} qs_status;

typedef enum { QS_C64 = 0, QS_C128 = 1 } qs_dtype;

/* Gate kinds.  Fixed gates §2.3.2; parameterised gates §2.3.3 with the
 * half-angle convention R_P(theta) = exp(-i theta P / 2), and RZZ/RXX/RYY(theta)
 * = exp(-i theta/2 P(x)P); PS(theta) = diag(1, e^{i theta}); custom matrix gates
 * §2.3.4.  Any gate may carry control qubits (§2.3.5): it acts where every
 * control bit is 1.  Two-target matrices use the basis index
 * bit(targets[0]) + 2 * bit(targets[1]). */
typedef enum {
  QS_GATE_I = 0,
  QS_GATE_X = 1,
  QS_GATE_Y = 2,
  QS_GATE_Z = 3,
  QS_GATE_H = 4,
  QS_GATE_S = 5,
  QS_GATE_SDG = 6,
  QS_GATE_T = 7,
  QS_GATE_TDG = 8,
  QS_GATE_SWAP = 9,
  QS_GATE_RX = 16,
  QS_GATE_RY = 17,
  QS_GATE_RZ = 18,
  QS_GATE_PS = 19,
  QS_GATE_RXX = 20,
  QS_GATE_RYY = 21,
  QS_GATE_RZZ = 22,
  QS_GATE_MATRIX = 32
} qs_gate_kind;

typedef struct qs_state qs_state;
typedef struct qs_circuit qs_circuit;
typedef struct qs_ham qs_ham;
typedef struct qs_qaoa qs_qaoa;

/* Execution options for a circuit plan.  Zero means "library default". */
typedef struct {
  int fuse;       /* 1 (default): fused shared-memory tile passes (complex64 states of 22 or more
                     qubits run the passes that qualify as micro-ops on TMA-fed tiles, each pass
                     of at most 192 ops (128 in adjoint passes) compiled for the circuit at
                     finalize by the runtime compiler, larger ones on the precompiled micro-op
                     kernels, the rest on the op interpreter); 2: all on the op interpreter; 3: micro-ops wherever a pass
                     qualifies, whatever the size, on the library's precompiled kernels (ops
                     dispatched from a table); 4: as 3, compiled for the circuit (the same
                     arithmetic as 3, bit for bit); -1: one kernel per gate.  Compiled passes
                     are cached by their source for the life of the process; finalize returns
                     QS_ERR_UNSUPPORTED if the runtime compiler fails. */
  int tile_bits;  /* log2 amplitudes per fused tile, 6..13 (default 12 for c64, 11 for c128) */
  int low_bits;   /* low (contiguous) qubits present in every tile, 1..tile_bits (default 4) */
  int checkpoint; /* adjoint state checkpoints, 0 (default): none.  Circuits: every `checkpoint`
                     gates the forward sweep saves psi (passes never span that boundary) and the
                     reverse sweep reloads it there instead of the uncomputed state, which bounds
                     the rounding drift of long uncompute chains; one extra state of memory per
                     checkpoint.  QAOA engine: every `checkpoint` layers (about two passes each). */
} qs_options;

/* Library version string and the last error message of this thread. */
QS_API const char* qs_version(void);
QS_API const char* qs_last_error(void);

/* ------------------------------------------------------------------ states */

/* Create a state of n_qubits (1..34) and dtype on `cuda_stream` (a cudaStream_t,
 * NULL = legacy default stream).  dev_buf: caller-owned device buffer of at
 * least buf_bytes >= 2^n * sizeof(amplitude), 256-byte aligned; NULL = the
 * library allocates (and later frees) the buffer.  Contents are undefined until
 * a set_* or copy_in call. */
QS_API qs_status qs_state_create(int n_qubits, qs_dtype dtype, void* dev_buf, size_t buf_bytes,
                          void* cuda_stream, qs_state** out);
QS_API qs_status qs_state_destroy(qs_state* s);
/* Device pointer of the amplitudes (for zero-copy views by the caller). */
QS_API qs_status qs_state_device_ptr(const qs_state* s, void** dev_ptr);
/* |index>  (§2.6: the simulator starts in |0...0>). */
QS_API qs_status qs_state_set_basis(qs_state* s, uint64_t index);
/* |+>^n = 2^{-n/2} sum_x |x>  (the QAOA start state, §5.2). */
QS_API qs_status qs_state_set_plus(qs_state* s);
/* set_qs / get_qs (§2.6.2, §6.2): copy 2^n amplitudes of the state's dtype in
 * or out.  src_on_device / dst_on_device: 1 = device pointer, 0 = host pointer. */
QS_API qs_status qs_state_copy_in(qs_state* s, const void* src, int src_on_device);
QS_API qs_status qs_state_copy_out(const qs_state* s, void* dst, int dst_on_device);
/* dst <- src (same n and dtype). */
QS_API qs_status qs_state_copy(qs_state* dst, const qs_state* src);
/* sum_x |psi_x|^2 in FP64. */
QS_API qs_status qs_state_norm2(const qs_state* s, double* out);

/* ---------------------------------------------------------------- circuits */

QS_API qs_status qs_circuit_create(int n_qubits, qs_circuit** out);
QS_API qs_status qs_circuit_destroy(qs_circuit* c);
/* Append one gate.  targets[n_t] (n_t = 1, or 2 for SWAP/RXX/RYY/RZZ/2-qubit
 * MATRIX), ctrls[n_c] (n_c >= 0), all distinct and < n_qubits.
 * Angle binding (§2.2 parameter resolver, linear in one parameter):
 *   angle = constant + coef * params[param_idx]; param_idx = -1 for a fixed angle.
 * matrix: for QS_GATE_MATRIX only, (2^n_t)^2 complex entries row-major as
 * interleaved (re, im) doubles; the library copies it.  Invalidates any plan. */
QS_API qs_status qs_circuit_add(qs_circuit* c, int kind, const int* targets, int n_t, const int* ctrls,
                         int n_c, int param_idx, double coef, double constant, const double* matrix);
/* Build the execution plan (fusion into tile passes) for `dtype`.  opts may be
 * NULL.  Called implicitly by the first apply if absent. */
QS_API qs_status qs_circuit_finalize(qs_circuit* c, qs_dtype dtype, const qs_options* opts);
/* Plan statistics: gates, parameters (max param_idx + 1), forward HBM passes. */
/* Per-circuit kernels of the complex64 micro-op passes (option fuse = 4), for
 * inspection and host-side tests; host only, no device work.  Plans the
 * circuit (which must not have been finalized) for complex64 with `opts`
 * (NULL or fuse 0: fuse = 4; tile_bits / low_bits as for finalize), writes the
 * CUDA source of the micro-op passes of the forward (which = 0) or adjoint
 * (which = 1) plan into src (at most cap - 1 characters and a terminating 0;
 * src may be NULL when cap = 0), its full length to *src_len and the number of
 * passes it holds to *n_gen, and with compile != 0 compiles it for sm_103a
 * with the runtime compiler (*cubin_bytes: the binary's size).  Returns
 * QS_ERR_UNSUPPORTED when the source cannot be generated or compiled (message:
 * the compiler's log).  The circuit is left unfinalized; out pointers may be
 * NULL. */
QS_API qs_status qs_circuit_codegen(qs_circuit* c, const qs_options* opts, int which, int compile, char* src,
                                    size_t cap, size_t* src_len, int* n_gen, size_t* cubin_bytes);
QS_API qs_status qs_circuit_info(const qs_circuit* c, int* n_gates, int* n_params, int* n_passes);

/* psi <- U(params) psi: the circuit applied in order (§2.6.1 apply_circuit).
 * params[n_params] on the host, n_params >= the circuit's parameter count. */
QS_API qs_status qs_apply_circuit(qs_state* s, qs_circuit* c, const double* params, int n_params);

/* psi <- U psi for a dense 2^k x 2^k complex matrix on k target qubits (a
 * custom gate, §2.3.4; equally the product of a run of gates fused into k
 * qubits).  matrix: host, row-major, (re, im) doubles, 2^k x 2^k; basis index
 * sum_b bit(targets[b]) 2^b.  k = 1..6, distinct targets < n.
 * engine: 0 = automatic, 1 = CUDA cores (the state's precision), 2 = tensor
 * cores (tcgen05 TF32 with head/tail operand splitting, float32 accuracy;
 * complex64, k = 4 or 5 and n - k >= 7 only, else QS_ERR_INVALID_ARG).  The
 * automatic choice takes the tensor cores where they apply.  Tensor-core calls
 * synchronise the stream and return QS_ERR_TIMEOUT if the MMA completion wait
 * gave up; CUDA-core calls are asynchronous. */
QS_API qs_status qs_apply_matrix(qs_state* s, int k, const int* targets, const double* matrix, int engine);

/* Autotuner of the fused passes: applies the circuit to `s` (whose contents
 * it overwrites) under each candidate tile shape -- tile bits m = largest, -1,
 * -2 for the dtype and state size, times contiguous low bits 2..5 -- timing
 * `reps` applications per candidate with CUDA events on s's stream, and keeps
 * the fastest plan in the circuit (fuse = 1).  chosen (may be NULL) receives the
 * options kept; best_ms (may be NULL) the time of one application.  Not part of
 * the paper: it picks the engine's tile shape by measurement.  Synchronises. */
QS_API qs_status qs_circuit_autotune(qs_circuit* c, qs_state* s, const double* params, int n_params, int reps,
                                     qs_options* chosen, double* best_ms);

/* ------------------------------------------------------------ Hamiltonians */

/* H = sum_k coef[k] P_k with real coefficients (§2.5.1), P_k given by masks:
 * bit q of xmask[k] / zmask[k] = X / Z on qubit q, both set = Y. */
QS_API qs_status qs_ham_create(int n_qubits, int n_terms, const uint64_t* xmask, const uint64_t* zmask,
                        const double* coef, qs_ham** out);
QS_API qs_status qs_ham_destroy(qs_ham* h);

/* dst <- H src, unnormalised (§2.6.1 apply_hamiltonian).  dst != src. */
QS_API qs_status qs_apply_hamiltonian(qs_state* dst, const qs_state* src, const qs_ham* h);
/* *energy = <psi|H|psi> (§2.6.2 get_expectation; real for real coefficients). */
QS_API qs_status qs_expectation(const qs_state* s, const qs_ham* h, double* energy);
/* out2[0] + i out2[1] = <bra|ket> (§2.6.2, the H = I case). */
QS_API qs_status qs_inner_product(const qs_state* bra, const qs_state* ket, double* out2);

/* Energy and its gradient with respect to every parameter by the adjoint
 * method (§4.1 get_expectation_with_grad; adjoint method named in §7.2):
 *   psi_N = U psi_0, E = <psi_N|H|psi_N>, lam = H psi_N, then for k = N..1:
 *   psi <- U_k^dag psi, grad[p(k)] += coef_k * 2 Re <lam| dU_k |psi>, lam <- U_k^dag lam.
 * psi: holds psi_0 on entry; on return it holds psi_0 again up to rounding.
 * lam: a second state of the same n and dtype, used as the adjoint buffer.
 * energy: host double; grad: host double[n_params] (overwritten). */
QS_API qs_status qs_expectation_with_grad(qs_state* psi, qs_state* lam, qs_circuit* c, const qs_ham* h,
                                   const double* params, int n_params, double* energy, double* grad);

/* Draw `shots` outcomes of measuring every qubit (§2.6.3 sampling): outcome s is
 * the smallest x with cdf(x) > u_s * cdf(2^n - 1), cdf the FP64 prefix sums of
 * |psi_x|^2 and u_s = splitmix64(seed + s * 0x9E3779B97F4A7C15) >> 11, times 2^-53.
 * out_bits: host uint64[shots], little-endian bitstrings. */
QS_API qs_status qs_sample(const qs_state* s, uint64_t shots, uint64_t seed, uint64_t* out_bits);

/* The same for a list of Hamiltonians, evaluated together (§4.1: the gradient
 * operator takes a list of observables; outputs [n_ham] energies and
 * [n_ham, n_params] gradients, here for one encoder input).  One forward sweep;
 * each Hamiltonian then forms lam = H_h psi_N and runs its own reverse sweep
 * from a copy of psi_N kept in a buffer the call allocates on psi (2^n
 * amplitudes, kept until psi is destroyed).  hams: host array of n_ham handles.
 * energies: host double[n_ham]; grads: host double[n_ham * n_params],
 * row-major.  Synchronises psi's stream. */
QS_API qs_status qs_expectation_with_grad_multi(qs_state* psi, qs_state* lam, qs_circuit* c, int n_ham,
                                                const qs_ham* const* hams, const double* params, int n_params,
                                                double* energies, double* grads);

/* Generalised expectation (§2.6.2 and §4.1: E = <phi|U_l^dag H U_r|psi>, which
 * gives the physical expectation for phi = psi, U_l = U_r, inner products for
 * H = I, and projections for H a projector) and its gradient with respect to
 * every parameter, complex in general:
 *   dE/dp = sum_{k in U_r} coef_k <phi_l|H|..dU_k..psi> + sum_{k in U_l} coef_k <..dU_k..phi|H|psi_r>,
 * both circuits reading the same parameter vector.  Each circuit runs forward
 * once and backward twice (adjoint sweeps with lam and with i lam give the real
 * and imaginary parts).  psi, phi: the right and left input states (restored on
 * return up to rounding); lam: a third state used as the adjoint buffer (all
 * three of one n and dtype, distinct).  c_left NULL: U_l = U_r.  energy2: host
 * double[2] (re, im); grad2: host double[2 * n_params] (re, im interleaved).
 * Synchronises psi's stream. */
QS_API qs_status qs_expectation_general(qs_state* psi, qs_state* phi, qs_state* lam, qs_circuit* c_right,
                                        qs_circuit* c_left, const qs_ham* h, const double* params, int n_params,
                                        double* energy2, double* grad2);

/* Projective measurement of one qubit in the computational basis, mid-circuit
 * (the measurement gate, §2.3; outcomes as in sampling, §2.6.3): with
 * P(1) = sum of |psi_x|^2 over x with bit `qubit` set and P(0) = total - P(1),
 * u = top 53 bits of splitmix64(seed) / 2^53, the outcome is 0 iff P(0) > u *
 * total; the state is projected onto the outcome and renormalised in place.
 * Sums are FP64 in a fixed order.  *outcome: host int.  Synchronises. */
QS_API qs_status qs_measure(qs_state* s, int qubit, uint64_t seed, int* outcome);

/* ------------------------------------------------------- density matrices */

/* Density-matrix simulation (§3.2: rho' = U rho U^dag, <H> = tr(rho H)) with
 * quantum channels (§3.3: Psi(rho) = sum_i K_i rho K_i^dag, sum K_i^dag K_i = I).
 * rho of n qubits is a qs_state of 2n qubits holding vec[x + 2^n y] = rho_{x,y};
 * set_basis(0) prepares |0..0><0..0|.  A density-matrix circuit is a 2n-qubit
 * qs_circuit: each gate is added on the low register and its complex conjugate
 * on the high register, each channel as its superoperator sum_i K_i (x)
 * conj(K_i) on (qubit, qubit + n).  Apply it with qs_apply_circuit; the adjoint
 * gradient is refused once a channel is present (channels are not unitary). */
typedef enum {
  QS_CH_PAULI = 0,              /* p = (px, py, pz): (1-px-py-pz) rho + px X rho X + py Y rho Y + pz Z rho Z */
  QS_CH_DEPOLARIZING = 1,       /* p = (p): (1 - p) rho + p/4 (I rho I + X rho X + Y rho Y + Z rho Z) */
  QS_CH_AMPLITUDE_DAMPING = 2,  /* p = (gamma): E0 = diag(1, sqrt(1-gamma)), E1 = sqrt(gamma) |0><1| */
  QS_CH_PHASE_DAMPING = 3,      /* p = (gamma): E0 = diag(1, sqrt(1-gamma)), E1 = sqrt(gamma) |1><1| */
  QS_CH_KRAUS = 4               /* n_kraus 2x2 operators, (re, im) row-major, 8 doubles each */
} qs_channel_kind;

/* A density-matrix circuit of n_qubits (1..17) qubits. */
QS_API qs_status qs_dm_circuit_create(int n_qubits, qs_circuit** out);
/* Gate U on the system qubits (arguments as qs_circuit_add): adds U and conj(U). */
QS_API qs_status qs_dm_add_gate(qs_circuit* c, int kind, const int* targets, int n_t, const int* ctrls, int n_c,
                                int param_idx, double coef, double constant, const double* matrix);
/* Channel on one system qubit; p: the kind's parameters (host), kraus: for
 * QS_CH_KRAUS only.  Invalid probabilities or incomplete Kraus sets return
 * QS_ERR_INVALID_ARG. */
QS_API qs_status qs_dm_add_channel(qs_circuit* c, int kind, int qubit, const double* p, int n_kraus,
                                   const double* kraus);
/* *energy = tr(rho H) for a Pauli sum H on the n system qubits (rho: 2n qubits). */
QS_API qs_status qs_dm_expectation(const qs_state* rho, const qs_ham* h, double* energy);

/* ------------------------------------------------ Monte-Carlo trajectories */

/* The state-vector treatment of channels (§3.3: each noise gate acts with some
 * probability; averaging over sampled runs of the circuit gives the noisy
 * result).  A trajectory starts from |0..0>; at channel site s (sites numbered
 * 0, 1, ... in the order they are added) it takes branch i with probability w_i
 * and replaces psi by the branch operator applied to psi:
 *   Pauli (px, py, pz):  w = (1 - px - py - pz, px, py, pz), operators I, X, Y, Z;
 *   depolarizing (p):    q = p / 4, w = (1 - q - q - q, q, q, q), operators I, X, Y, Z;
 *   damping / Kraus:     w_i = ||K_i psi||^2 (FP64 sums), operator K_i / sqrt(w_i)
 *                        (amplitude and phase damping as in qs_channel_kind).
 * The branch is the smallest i whose running sum w_0 + ... + w_i exceeds
 * u * (w_0 + ... + w_last), else the last i with w_i > 0, with
 * u = (splitmix64(seed + c * 0x9E3779B97F4A7C15) >> 11) * 2^-53 for the counter
 * c = t * n_sites + s of trajectory t (the published splitmix64 of Steele, Lea &
 * Flood 2014; the same generator as qs_sample).  The mean of the trajectory
 * energies estimates tr(rho H) of the density-matrix simulator.
 *
 * n_qubits 1..34.  A trajectory runs in one CTA's shared memory while its
 * state fits (n_qubits <= 14 complex64 or 13 complex128 for energies; with
 * gradients, psi and lam both: 13 and 12), many trajectories per launch.
 * Larger states run one trajectory after another on the fused tile passes in
 * HBM: the gates between damping / Kraus sites are planned once as circuits,
 * a Pauli / depolarizing site is a one-qubit matrix gate set to the sampled
 * Pauli, and the weights at a damping / Kraus site come from the qubit's
 * reduced density matrix (FP64 sums), with the same draws and the same rule.
 * cuda_stream: the engine's stream (NULL: legacy default). */
typedef struct qs_traj qs_traj;
QS_API qs_status qs_traj_create(int n_qubits, qs_dtype dtype, void* cuda_stream, qs_traj** out);
QS_API qs_status qs_traj_destroy(qs_traj* t);
/* A gate (arguments as qs_circuit_add; any kind but QS_GATE_MATRIX). */
QS_API qs_status qs_traj_add_gate(qs_traj* t, int kind, const int* targets, int n_t, const int* ctrls, int n_c,
                                  int param_idx, double coef, double constant);
/* A channel site on one qubit: kind a qs_channel_kind, p its parameters (host);
 * QS_CH_KRAUS: n_kraus (1..4) 2x2 operators, (re, im) row-major, 8 doubles each,
 * complete to 1e-9.  At most 4096 sites. */
QS_API qs_status qs_traj_add_channel(qs_traj* t, int kind, int qubit, const double* p, int n_kraus,
                                     const double* kraus);
/* Sites, parameters, and the persistent grid of the energy and gradient kernels
 * (0: the state does not fit in shared memory). */
QS_API qs_status qs_traj_info(const qs_traj* t, int* n_sites, int* n_params, int* grid_energy, int* grid_grad);
/* Trajectories first .. first + n_traj - 1 (1 <= n_traj <= 2^24):
 * energies[i] = <psi_t|H|psi_t> (host double[n_traj]).  grad_mean (host
 * double[n_params], or NULL for energies only) = the mean over the trajectories
 * of each trajectory's adjoint gradient (§4.1 / §7.2), each trajectory being the
 * fixed unitary circuit of its sampled Paulis; refused (QS_ERR_INVALID_ARG)
 * when a damping or Kraus channel is present.  choices (host
 * uint8[n_traj * n_sites] or NULL): the branch taken at every site.
 * Synchronises the engine's stream. */
QS_API qs_status qs_traj_run(qs_traj* t, const qs_ham* h, const double* params, int n_params, uint64_t seed,
                             long long first, int n_traj, double* energies, double* grad_mean,
                             unsigned char* choices);
/* The same on device buffers (d_params double[n_params], d_energies
 * double[n_traj], d_grad_mean double[n_params] or NULL), enqueued on the
 * engine's stream without synchronising while the state fits in shared
 * memory; larger states run the host loop above and synchronise. */
QS_API qs_status qs_traj_run_device(qs_traj* t, const qs_ham* h, const double* d_params, uint64_t seed,
                                    long long first, int n_traj, double* d_energies, double* d_grad_mean);
/* The final state of trajectory `traj` into `out` (n_qubits, same dtype). */
QS_API qs_status qs_traj_state(qs_traj* t, const double* params, int n_params, uint64_t seed, long long traj,
                               qs_state* out);

/* -------------------------------------------------------------------- QAOA */

/* MaxCut QAOA engine (§5.2 ansatz; QuPack QAOA simulator interface §6.2):
 * cost C(x) = sum_{(a,b) in edges} z_a z_b, z = 1 - 2 bit; start |+>^n; layer

 * (n_qubits >= 4) l = 1..p applies exp(-i gamma_scale * gamma_l * C) then RX(beta_l) on every
 * qubit.  gamma_scale = 1: the QuPack form; 0.5: RZZ(gamma_l) on every edge.
 * edges: host int[2 * n_edges] (pairs of distinct qubits, no repeats).
 * opts may be NULL. */
QS_API qs_status qs_qaoa_create(int n_qubits, const int* edges, int n_edges, int p, double gamma_scale,
                         qs_dtype dtype, const qs_options* opts, qs_qaoa** out);
QS_API qs_status qs_qaoa_destroy(qs_qaoa* q);
/* Forward passes and planned HBM traffic of one energy+gradient evaluation. */
QS_API qs_status qs_qaoa_info(const qs_qaoa* q, int* fwd_passes, int* rev_passes, double* bytes_per_eval);
/* *max_cut = max over x of cut(x), the MaxCut optimum by exhaustive search over
 * the engine's cut-value array (the brute-force maximum §5.2 compares against).
 * Host output; synchronises. */
QS_API qs_status qs_qaoa_max_cut(qs_qaoa* q, int* max_cut);
/* psi <- U(gamma, beta)|+>^n (QuPack evolution()). */
QS_API qs_status qs_qaoa_evolve(qs_qaoa* q, qs_state* psi, const double* gamma, const double* beta);
/* *energy = <psi(gamma,beta)|C|psi(gamma,beta)>; psi is overwritten with the final state. */
QS_API qs_status qs_qaoa_expectation(qs_qaoa* q, qs_state* psi, const double* gamma, const double* beta,
                              double* energy);
/* Energy and dE/dgamma[p], dE/dbeta[p] by the adjoint method (QuPack
 * get_expectation_with_grad).  psi, lam: work states (contents on entry
 * ignored; on return undefined).  Host outputs. */
QS_API qs_status qs_qaoa_expectation_with_grad(qs_qaoa* q, qs_state* psi, qs_state* lam, const double* gamma,
                                        const double* beta, double* energy, double* dgamma, double* dbeta);

/* Plan of the complex64 two-shape QAOA passes (options fuse = 2, tile_bits,
 * low_bits; host only, no device work), for inspection and host-side tests.
 * which: 0 = energy+gradient plan (forward passes, turnaround, reverse passes),
 * 1 = energy plan.  rec: long long[max_passes * QS_XPLAN_REC]; per pass:
 * [0] kernel (0: psi alone, 1: psi and lam interleaved), [1] flags (1 start
 * from |+>, 2 load psi with lam = 0, 4 store, 8 step-1 gradients, 16 step-3
 * gradients), [2] tile qubit mask, [3] phases, [4] step-1 coefficient offset,
 * [5] step-3 offset, [6] diagonal LUT offset (-1 none; offsets index the
 * per-layer table lut[|E|+1], lut_dag[|E|+1], (cos b/2, sin b/2),
 * (cos b/2, -sin b/2)), [7..9] output slot of accumulators 0..2 (-1 none),
 * [10] tile bits, [11] low bits, then per phase 7 entries: step-1 register
 * mask, step-3 register mask, diagonal (0 none, 1 cost, 2 cost gradient and
 * cost^dag, 3 energy), the qubits of register bits 0..3 (-1: none; 12 phase
 * slots), then at [96] and [113] the tile's load and store tensor maps, 17 entries each:
 * log2 of 8-byte words per amplitude, local bits covered by one box, and per
 * dimension 0..4 its first word-index bit, its width in bits and the box width
 * in bits, then at [130] the offset of the pass's phase weights in the
 * per-call coefficient table.  slot_out/slot_w: output (0 = E, 1 + l =
 * dgamma_l, 1 + p + l = dbeta_l) and weight per slot. */
#define QS_XPLAN_REC 131
QS_API qs_status qs_qaoa_xplan(int n_qubits, const int* edges, int n_edges, int p, double gamma_scale, int tile_bits,
                               int low_bits, int which, long long* rec, int max_passes, int* n_passes,
                               int* slot_out, double* slot_w, int max_slots, int* n_slots);

/* The per-call coefficient table of the same plans (host only), for
 * inspection and host-side tests: interleaved FP64 complex, *n_entries
 * entries (table: double[2 * max_entries]).  Per layer l at l * (2 |E| + 4):
 * the cost LUT exp(-i gs gamma_l C) for cut = 0..|E| times its renormalisation,
 * the reverse LUT (conjugate phases, its own renormalisation), then (t, 0) of
 * the scaled mixer of RX(beta_l) and of RX(-beta_l): [[1, -it], [-it, 1]]
 * with t = s/c when |c| >= |s| (c, s = cos, sin of the half angle), else
 * t = -c/s with every qubit the step rotates flipped in the data.  Then each
 * pass's phase weights (record [130]): per phase (w1, w3), (wd, 0), the factors
 * of the step-1, step-3 and diagonal sums.  *flip = 1: the energy plan leaves
 * every qubit flipped (the engine flips the state back). */
QS_API qs_status qs_qaoa_xcoef(int n_qubits, const int* edges, int n_edges, int p, double gamma_scale, int tile_bits,
                               int low_bits, const double* gamma, const double* beta, double* table, int max_entries,
                               int* n_entries, int* flip);

/* One evaluation without handles, in the shape of the QuPack QAOA call (§6.2):
 * graph, depth and angles in; energy and gradients out (host arrays of p
 * doubles).  Creates the engine and two library-owned states on the legacy
 * default stream and frees them before returning; synchronises. */
QS_API qs_status qs_qaoa_evaluate(int n_qubits, const int* edges, int n_edges, int p, double gamma_scale,
                                  const double* gamma, const double* beta, qs_dtype dtype, double* energy,
                                  double* dgamma, double* dbeta);

/* ----------------------------------------------------------------- batches */

/* Many independent instances (circuit, Hamiltonian, parameters) evaluated
 * together: the batch dimension of get_expectation_with_grad (§4.1, output
 * shapes [n_batch, ...]), here with one circuit and Hamiltonian per instance.
 * Instances whose psi and lam fit in shared memory (complex64 n <= 13,
 * complex128 n <= 12) run in ONE persistent launch: each CTA takes instances
 * from a work queue (largest first) and runs the full adjoint evaluation of one
 * instance at a time.  Larger instances get their own fused tile-pass plan at
 * creation and run concurrently on the batch's streams, their gate matrices
 * formed on the device from the device parameters.  A call is captured once as
 * a CUDA graph and replayed (launches are direct while qs_trace is enabled). */
typedef struct qs_batch qs_batch;

/* One gate of a batched circuit: kind (any qs_gate_kind but QS_GATE_MATRIX),
 * n_targets / targets as in qs_circuit_add, controls as a bit mask, and the
 * angle binding angle = constant + coef * params[param] with `param` indexing
 * the instance's own parameter slice (-1: fixed angle). */
typedef struct {
  int32_t kind;
  int32_t n_targets;
  int32_t targets[2];
  uint64_t ctrl_mask;
  int32_t param;
  int32_t pad;
  double coef;
  double constant;
} qs_batch_gate;

/* Instance i has n_qubits[i] (1..26) qubits, gates gates[gate_offsets[i] ..
 * gate_offsets[i+1]), Pauli terms (xmask, zmask, coef)[term_offsets[i] ..
 * term_offsets[i+1]) and parameters params[param_offsets[i] ..
 * param_offsets[i+1]).  Offsets arrays have n_inst + 1 entries starting at 0.
 * Every instance starts from |0...0>.  All arrays are host arrays and copied.
 * Work is enqueued on cuda_stream. */
QS_API qs_status qs_batch_create(int n_inst, const int* n_qubits, const int* gate_offsets,
                                 const qs_batch_gate* gates, const int* term_offsets, const uint64_t* xmask,
                                 const uint64_t* zmask, const double* coef, const int* param_offsets,
                                 qs_dtype dtype, void* cuda_stream, qs_batch** out);
QS_API qs_status qs_batch_destroy(qs_batch* b);
/* Instances, total parameters and the CTAs of the persistent launch. */
QS_API qs_status qs_batch_info(const qs_batch* b, int* n_instances, int* n_params, int* grid);
/* energies[i] = <psi_i|H_i|psi_i> and grads (laid out like params) by the
 * adjoint method, for every instance.  Host arrays; synchronises the stream. */
QS_API qs_status qs_batch_expectation_with_grad(qs_batch* b, const double* params, double* energies,
                                                double* grads);
/* The same with device arrays (no copies, no synchronisation). */
QS_API qs_status qs_batch_expectation_with_grad_device(qs_batch* b, const double* dev_params,
                                                       double* dev_energies, double* dev_grads);

/* ------------------------------------------- learned QAOA initialiser (GNN) */

/* A graph network that maps a MaxCut graph to 2p QAOA angles, trained on
 * angles the simulator optimised.  The paper trains QAOA angles by gradient
 * descent from a fixed start (§5.2) and motivates slowly varying schedules by
 * adiabatic evolution (§5.4); the network is this library's own:
 *   node features h0[v] = (1, deg(v) / 3);
 *   `layers` message-passing layers of width `hidden`:
 *     a[v] = mean of h[u] over the neighbours u of v (0 without neighbours),
 *     h'[v] = relu(Ws h[v] + Wn a[v] + b);
 *   readout r = mean over nodes of h_L (0 for an empty graph),
 *   y = W2 relu(W1 r + b1) + b2, out_dim outputs.
 * Parameters: one float32 vector, blocks in this order: per layer Ws [hidden x d],
 * Wn [hidden x d], b [hidden] (d = 2 for the first layer, hidden after), then
 * W1 [hidden x hidden], b1 [hidden], W2 [out_dim x hidden], b2 [out_dim];
 * matrices row-major (output, input).  The kernels compute with the weights
 * rounded to bfloat16 (nearest, ties to even) and float32 activations and sums;
 * Adam keeps the float32 master copy. */
typedef struct qs_gnn qs_gnn;
typedef struct qs_graphs qs_graphs;

/* A batch of undirected graphs, validated and copied to the device.
 * node_off[n_graphs + 1]: graph g owns global nodes node_off[g] .. node_off[g+1]-1
 * (at most 64 nodes per graph); adj_off[N + 1] (N = node_off[n_graphs]) and adj:
 * the neighbours of global node v are adj[adj_off[v] .. adj_off[v+1]), given as
 * indices LOCAL to v's graph.  The adjacency must be symmetric, without self
 * loops or repeats, at most 4096 entries per graph.  Host arrays; violations
 * return QS_ERR_INVALID_ARG. */
QS_API qs_status qs_graphs_create(int n_graphs, const int* node_off, const int* adj_off, const int* adj,
                                  qs_graphs** out);
QS_API qs_status qs_graphs_destroy(qs_graphs* g);
/* *n = number of float32 parameters for these dimensions (hidden even, 2..64;
 * layers 1..4; out_dim 1..64). */
QS_API qs_status qs_gnn_n_weights(int hidden, int layers, int out_dim, int* n);
/* A network with zero weights and zero Adam state; work goes on cuda_stream. */
QS_API qs_status qs_gnn_create(int hidden, int layers, int out_dim, void* cuda_stream, qs_gnn** out);
QS_API qs_status qs_gnn_destroy(qs_gnn* g);
/* Replace the float32 weights (host or device array of n_weights floats), form
 * the bfloat16 copy and reset the Adam moments and step count. */
QS_API qs_status qs_gnn_set_weights(qs_gnn* g, const float* w, int on_device);
/* Copy out the float32 master weights and/or their bfloat16 bit patterns
 * (either pointer may be NULL).  Host copies synchronise the stream. */
QS_API qs_status qs_gnn_get_weights(qs_gnn* g, float* w, uint16_t* w_bf16, int on_device);
/* Training state for checkpoint/resume: the float32 master weights, the Adam
 * moments m and v (host float[n_weights] each) and the Adam step count.  get
 * synchronises the stream; set re-forms the bfloat16 copy and synchronises. */
QS_API qs_status qs_gnn_get_state(qs_gnn* g, float* w, float* m, float* v, int* step);
QS_API qs_status qs_gnn_set_state(qs_gnn* g, const float* w, const float* m, const float* v, int step);
/* dev_out[g * out_dim + o] = y_o of graph g, device float32.  Asynchronous. */
QS_API qs_status qs_gnn_forward(qs_gnn* g, const qs_graphs* graphs, float* dev_out);
/* dev_grad[n_weights] = sum over graphs of dL/dw given dev_dout[g * out_dim + o]
 * = dL/dy (device float32), recomputing the forward pass.  Gradients are summed
 * in a fixed order: bitwise reproducible for a given batch.  Asynchronous. */
QS_API qs_status qs_gnn_backward(qs_gnn* g, const qs_graphs* graphs, const float* dev_dout, float* dev_grad);
/* One Adam step (Kingma & Ba 2015, with bias correction; the step count is kept
 * by the network) on the float32 weights, then refresh the bfloat16 copy. */
QS_API qs_status qs_gnn_adam_step(qs_gnn* g, const float* dev_grad, float lr, float beta1, float beta2, float eps);
/* One training step on a batch in two launches: per graph the forward pass,
 * dL/dy of L = mean over the batch's n_graphs * out_dim entries of (y - t)^2,
 * and the backward pass; then the gradient sums and the Adam update (as
 * qs_gnn_adam_step).  dev_targets: device float32 [n_graphs * out_dim];
 * dev_loss: device float32 (may be NULL) receives L.  Equivalent to
 * forward + qs_mse + backward + adam_step (same weights bit for bit; the loss
 * is summed in another order).  Asynchronous. */
QS_API qs_status qs_gnn_train_step(qs_gnn* g, const qs_graphs* graphs, const float* dev_targets, float lr,
                                   float beta1, float beta2, float eps, float* dev_loss);
/* *dev_loss = mean of (y - t)^2 over n entries and dev_dy = 2 (y - t) / n (either
 * output may be NULL).  Device float32 arrays, one CTA, fixed summation order. */
QS_API qs_status qs_mse(int n, const float* dev_y, const float* dev_target, float* dev_loss, float* dev_dy,
                        void* cuda_stream);
/* One Adam step on n float64 parameters in place (device arrays), step count t
 * >= 1 given by the caller; maximize = 1 ascends (uses -grad).  Used to optimise
 * batches of circuit angles without leaving the device. */
QS_API qs_status qs_adam_f64(int n, double* dev_w, double* dev_m, double* dev_v, const double* dev_grad, int t,
                             double lr, double beta1, double beta2, double eps, int maximize, void* cuda_stream);

/* ------------------------------------------------- allocation-free variant */

/* *energy = <psi|H|psi>, the same Pauli-sum kernel as qs_expectation, for
 * callers that must not have the library allocate device memory: their device
 * memory belongs to another allocator (a framework's caching allocator, a pool
 * reserved at start-up), or they cannot risk the device-wide synchronisation of
 * cudaFree/cudaMalloc in their loop.  The paper has no counterpart; this is a
 * deployment variant.
 *   dev_psi: caller-owned device array of 2^n_qubits amplitudes of `dtype`.
 *   xmask/zmask/coef: host arrays of n_terms Pauli terms as in qs_ham_create,
 *   at most 4096 terms (QS_ERR_INVALID_ARG beyond).  energy: host double.
 * The call allocates no device memory: its working memory is a fixed 256 KiB
 * array inside the library, held by every device that loads the library until
 * the process exits.  The first call on a device (with that device current)
 * looks up the array's device address.  All calls share the array and it keeps
 * the last call's contents;
 * calls that overlap on the GPU (other host threads, other streams) race on it,
 * so serialise them.  The call synchronises `cuda_stream` before returning. */
QS_API qs_status qs_expectation_noalloc(const void* dev_psi, int n_qubits, qs_dtype dtype, int n_terms,
                                        const uint64_t* xmask, const uint64_t* zmask, const double* coef,
                                        void* cuda_stream, double* energy);

/* ------------------------------------------------------- failure detection */

/* Self-test of the bounded device-side waits (the tensor-core kernel's MMA
 * completion wait): one CTA polls an mbarrier that nothing arrives on, a bounded
 * number of times, and gives up with nothing in flight.  Returns
 * QS_ERR_TIMEOUT with *timed_out = 1 (the expected outcome); the context stays
 * usable.  Synchronises the device. */
QS_API qs_status qs_selftest_wait_timeout(int* timed_out);

/* ----------------------------------------------------------------- tracing */

/* Kernel of a traced launch. */
typedef enum {
  QS_TRACE_TILE = 0,      /* generic fused tile pass (circuits) */
  QS_TRACE_QAOA_FWD = 1,  /* QAOA pass on psi alone */
  QS_TRACE_QAOA_TWO = 2,  /* QAOA pass on separate psi and lam tiles (turnaround) */
  QS_TRACE_QAOA_IL = 3,   /* QAOA reverse pass on interleaved psi/lam */
  QS_TRACE_BATCH = 4,     /* batched persistent launch */
  QS_TRACE_DENSE_TC = 5,  /* dense k-qubit block on the tensor cores */
  QS_TRACE_DENSE_CC = 6,  /* dense k-qubit block on the CUDA cores */
  QS_TRACE_QX_FWD = 7,    /* complex64 two-shape QAOA pass on psi alone (forward sweep) */
  QS_TRACE_QX_TURN = 8,   /* two-shape turnaround: psi in, interleaved (psi, lam) out */
  QS_TRACE_QX_REV = 9,    /* two-shape reverse pass on interleaved (psi, lam) */
  QS_TRACE_TILE2 = 10,    /* complex64 fused tile pass as micro-ops (TMA-fed) */
  QS_TRACE_TILE2GEN = 11  /* ... its per-circuit kernel (fuse = 4: compiled at finalize) */
} qs_trace_kind;

/* Tracing of the engine's launches: while enabled, every tile-pass or batch
 * launch is bracketed by a CUDA event pair recorded on its own stream, together
 * with the pass's algorithmic HBM bytes (state tiles loaded + stored, plus cut
 * values; 0 for batch launches) and its kernel kind.  Not part of the paper; it
 * exists to measure the engine.  enable: 1 = start (clears earlier records),
 * 0 = stop.  At most 65536 launches are kept. */
QS_API qs_status qs_trace_enable(int enable);
/* Synchronise the recorded events and copy out up to `max` records: duration in
 * ms, algorithmic bytes and qs_trace_kind per launch (any output may be NULL).
 * *n = number of records copied. */
QS_API qs_status qs_trace_read(int max, int* n, double* ms, double* bytes, int* kinds);

#ifdef __cplusplus
}
#endif

#endif /* QSIM_H */
