// Layouts shared by the host planner, the complex64 micro-op tile kernels
// compiled with the library, and the per-circuit pass kernels compiled at run
// time (t2gen.cu): plain structs with fixed-width fields and no other header,
// so the runtime compiler can include this file as it stands.
#pragma once

#ifdef __CUDACC_RTC__
typedef signed char int8_t;
typedef unsigned char uint8_t;
typedef unsigned short uint16_t;
typedef unsigned int uint32_t;
typedef unsigned long long uint64_t;
typedef decltype(sizeof(0)) size_t;
#else
#include <stdint.h>
#include <vector_types.h>
#endif

namespace qs {

enum PassFlags : uint32_t {
  PF_LOAD_PSI = 1,
  PF_LOAD_LAM = 2,
  PF_STORE_PSI = 4,
  PF_STORE_LAM = 8,
  PF_GEN_PLUS = 16,  // psi tile = 2^{-n/2} instead of a load
  PF_GEN_ZERO = 32,  // psi tile = |0...0> instead of a load
  PF_NEED_CUT = 64   // load the cut-value tile
};

// ---- the complex64 micro-op tile kernel: every op lowered on the host to a
// code naming its compiled body (register bits as template arguments), its
// shared-memory coefficients and its predicates.
enum T2Kind : uint8_t {
  T2_U1 = 1,     // 2x2 complex on register bit r0
  T2_R1 = 2,     // 2x2 real (the real parts of the entries) on r0
  T2_RX = 3,     // RX: coefficient (c, s) on r0
  T2_X = 4,      // X on r0 (a swap)
  T2_Z = 5,      // sign flip where the diagonal bit is 1: on register bit r0
  T2_ZC = 6,     // ... on a constant bit (d0)
  T2_D1R = 7,    // diagonal (D0, D1) on register bit r0
  T2_D1C = 8,    // ... on a constant bit d0: one factor per sub-cube
  T2_D2RR = 9,   // diagonal D[b0 + 2 b1] with b0 on r0, b1 on r1
  T2_D2RC = 10,  // b0 on r0, b1 constant (d1)
  T2_D2CR = 11,  // b0 constant (d0), b1 on r1
  T2_D2CC = 12,  // both constant
  T2_U2 = 13,    // 4x4 complex on (r0, r1)
  T2_G1 = 14,    // acc += 2 Re <lam|A|psi>, A 2x2 on r0
  T2_G2 = 15,    // ... A 4x4 on (r0, r1)
  T2_GD = 16     // ... A diagonal: (d0, d1) as register bits (bit 7 clear) or constant bits
};
// code = kind | r0 << 5 | r1 << 7 | (register controls ? 1 << 9 : 0); bit 10 (T2_OUTSIDE) of an op's
// code marks controls outside the registers (lc, gc), checked before the body runs
#if defined(__CUDACC__) || defined(__CUDACC_RTC__)
#define QS_T2_HD __host__ __device__
#else
#define QS_T2_HD
#endif
QS_T2_HD constexpr int t2_code(int kind, int r0, int r1, bool jc) {
  return kind | (r0 << 5) | (r1 << 7) | (jc ? 512 : 0);
}
constexpr int T2_OUTSIDE = 1024;

struct T2Op {
  uint16_t code;
  uint16_t cs;      // first coefficient in the pass's shared coefficient stage
  uint16_t slot;    // accumulator slot (gradient ops)
  uint8_t jc;       // controls among the register bits (mask over the register index)
  uint8_t d0, d1;   // constant diagonal bits: local bit l, 64 + global qubit q; GD: 128 + register bit
  uint8_t pad0[3];
  uint32_t lc;      // controls on local bits outside the registers
  uint64_t gc;      // controls outside the tile (checked on the tile offset)
  uint32_t coef;    // source of the coefficients in the call's table
  uint32_t ncoef;   // ... and their count
};

struct T2Phase {
  uint8_t R[4];          // local bits of register bits 0..3, ascending
  uint8_t pair;          // R[0] is local bit 0: register elements (2k, 2k+1) are one 16-byte access
  uint8_t pad0[3];
  uint16_t op_begin, op_end;  // ops of the phase (pass-relative)
  uint32_t sp[4];        // swizzled element offset of each register bit
  uint32_t l0tab[48];    // sub-cube index u -> local base: tab[u & 15] | tab[16 + (u >> 4)]
};

struct T2Pass {
  int m, ns, n_phases, n_ops, n_coef, n_slots, slot_base, ncomp;
  uint32_t flags;
  uint32_t smem;          // dynamic shared bytes
  int8_t comp[40];
  uint8_t ma[5], mw[5], mbx[5], mlb;  // tensor map of the tile (8-byte words, 128-byte swizzle)
  uint8_t pad0[4];
  uint64_t hiA[64], hiB[128];  // deposit of local bits c..c+5 / c+6..c+12 (c = 4)
};

// An encoded TMA tensor map (the driver's opaque 128-byte, 64-byte aligned object).
struct alignas(64) TmapBlob {
  uint64_t w[16];
};

// Kernel arguments of one instance's micro-op pass (device layout; the tensor
// maps are read by the TMA unit from wherever the arguments live).
struct T2Args {
  TmapBlob tm[2];  // psi, lam (8-byte words)
  const T2Pass* pass;
  const T2Phase* phases;
  const T2Op* ops;
  const float2* coef;
  float2* psi;
  float2* lam;
  double* partials;
  int stride;  // partials columns of one slot
  int cols;    // columns this launch fills (>= gridDim.x; the rest are zeros)
  int n;
  float plus_amp;
};

}  // namespace qs
