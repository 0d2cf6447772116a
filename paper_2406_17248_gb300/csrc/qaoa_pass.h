// Descriptors of the specialised QAOA tile passes (host planner <-> kernel).
#pragma once

#include "qsim_internal.h"

namespace qs {

constexpr int kQaoaMaxTileBits = 13;
constexpr int kQaoaMaxAcc = 4;     // accumulators (outputs) per pass
constexpr int kQaoaMaxPhases = 8;
constexpr int kQaoaMaxSteps = 8;
constexpr int kQaoaMaxLayersPerPass = 2;

enum QStepType : uint8_t {
  QST_COST = 1,       // psi *= lut[cut] (QSF_DAG: conjugate table; QSF_LAM: lam too)
  QST_RX = 2,         // RX on the masked register bits (QSF_DAG: RX^dag; QSF_LAM: lam too)
  QST_GRAD_RX = 3,    // acc += sum_masked Im <lam|X_q|psi>; then RX^dag on psi and lam
  QST_GRAD_COST = 4,  // acc += C Im(conj(lam) psi); QSF_LAM: then cost^dag on psi and lam
  QST_ENERGY = 5      // acc += C |psi|^2; lam = C psi
};
enum QStepFlags : uint8_t { QSF_DAG = 1, QSF_LAM = 2 };

struct QStep {
  uint8_t type;
  uint8_t mask;   // register bits the RX steps act on
  uint8_t flags;
  uint8_t acc;    // accumulator index
  uint16_t layer; // layer index relative to the pass's first staged layer
  uint16_t pad;
};

struct QPhase {
  int8_t R[4];   // local bits held in registers
  int8_t Q[12];  // sub-cube bits, low to high
  int8_t nq;
  int8_t n_steps;
  int8_t need_cut;  // a step reads the cut values
  int8_t pad;
  // The shared-memory swizzle is linear over GF(2): the position of local index
  // l = OR of disjoint bits is the XOR of the positions of those bits.  These
  // are the positions of the single register bits and sub-cube bits.
  uint16_t sreg[4];
  uint16_t sq[12];
  QStep steps[kQaoaMaxSteps];
};

// Shared-memory position of local index l (a bijection, linear over GF(2)).
// Tiles are filled by 16-byte asynchronous copies, so the swizzle permutes
// 16-byte chunks (8 per 128-byte bank row) and keeps the two complex64
// amplitudes of a chunk in place: the chunk's bank bits are XORed with a fold
// of its higher bits.  Host and device use this one definition.
__host__ __device__ __forceinline__ uint32_t qaoa_swizzle(bool c64, uint32_t l) {
  const uint32_t v = c64 ? (l >> 1) : l;  // chunk index
  const uint32_t f = ((v >> 3) ^ (v >> 6) ^ (v >> 9)) & 7u;
  return l ^ (c64 ? (f << 1) : f);
}

struct QPassDesc {
  int m, c, ncomp, n_phases;
  uint32_t flags;
  int n_acc;
  int slot_base;
  int layer_lo;   // first layer whose coefficients the pass stages
  int n_layers;   // staged layers (<= kQaoaMaxLayersPerPass)
  int pad;
  double plus_amp;
  int8_t comp[40];
  uint64_t hiA[64], hiB[64];
  QPhase phases[kQaoaMaxPhases];
};

// complex64 reverse sweep: psi and lam interleaved per amplitude,
// (psi.re, lam.re, psi.im, lam.im) = 16 bytes, amplitude x stored at
// il[0] + x for x < 2^(n-1) and il[1] + (x - 2^(n-1)) otherwise.
enum QPassFlags : uint32_t {
  PF_LOAD_IL = 1u << 8,   // load psi and lam from the interleaved buffer
  PF_STORE_IL = 1u << 9   // store psi and lam to the interleaved buffer
};

struct QaoaLaunch {
  void* il[2];
  void* psi;
  void* lam;
  const void* coef;  // per layer: lut[E+1], lut_dag[E+1], rx (c, s), rx_dag (c, -s)
  const uint8_t* cut;
  double* partials;
  int n, n_edges, stride, grid;
};

size_t qaoa_smem_bytes(qs_dtype dt, int m, int ns, int n_edges);
int qaoa_grid_size(qs_dtype dt, int m, int ns, int n_edges, uint64_t n_tiles);
qs_status launch_qaoa_pass(qs_dtype dt, const QPassDesc* d_pass, int ns, int m, uint32_t flags,
                           const QaoaLaunch& L, cudaStream_t st);
int qaoa_il_grid_size(int m, int n_edges, uint64_t n_tiles);

}  // namespace qs
