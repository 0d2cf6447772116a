// Descriptors of the complex64 QAOA passes with separate forward and reverse
// tile shapes (host planner <-> kernels).
//
// Scaled mixer.  RX(b) = [[c, -is], [-is, c]] is applied as c [[1, -it], [-it, 1]]
// with t = s/c when |c| >= |s| (one FMA per real output instead of a product
// and an FMA), and when |s| > |c| as (s/i) X [[1, -it'], [-it', 1]], t' = -c/s:
// the data then hold the state with that qubit flipped.  Every layer's mixer
// is complete before the next cost layer, so the flips there are none or all
// qubits, and C(x) = C(NOT x) for MaxCut: the cost layers, the energy and all
// the gradient terms read the flipped data unchanged.  The scalar the data
// carry (a product of 1/c and i/s factors) is tracked on the host: the cost
// LUTs fold in a renormalisation (so the data stay O(1) and the evolved state
// comes out exact), and each phase's gradient and energy sums are weighted by
// 1 / |scalar|^2 at the point where they are taken.
//
// A pass stages one tile (2^m amplitudes over a bit set S that holds the low c
// qubits) in shared memory and runs phases over it.  In a phase every thread
// holds 16 amplitudes (4 register bits) of one sub-cube and applies, in order:
//   step 1: RX on the register bits in m1 (coefficient c1),
//   a diagonal step (cost phase, its gradient, or the energy),
//   step 3: RX on the register bits in m3 (coefficient c3).
// The cost value C(x) = |E| - 2 cut(x) of an amplitude is not read from memory:
// cut(x) = fs[local index] + g(tile) + sum over the local bits set of w_i(tile),
// where fs counts the edges inside S, and g, w_i come from the edges that leave S
// and the tile's fixed (complement) bits.
#pragma once

#include "qsim_internal.h"

namespace qs {

constexpr int kXMaxPhases = 12;
constexpr int kXMaxM = 13;
constexpr int kXMaxComp = 40;

enum XDiag : uint8_t {
  XD_NONE = 0,
  XD_COST = 1,       // psi *= lut[cut]
  XD_COST_GRAD = 2,  // acc += C Im(conj(lam) psi); then psi, lam *= lut[cut]
  XD_ENERGY = 3      // acc += C |psi|^2 (two-state kernel: also lam = C psi)
};

enum XFlags : uint32_t {
  XF_GEN_PLUS = 1u,   // forward: the tile starts as |+> (nothing loaded)
  XF_LOAD_PSI = 2u,   // two-state kernel: psi from the plain state, lam = 0
  XF_STORE = 4u,      // store the tile (from the last phase's registers)
  XF_GRAD1 = 8u,      // two-state kernel: step 1 accumulates Im <lam|X_q|psi>
  XF_GRAD3 = 16u      // two-state kernel: step 3 accumulates Im <lam|X_q|psi>
};

struct XPhase {
  uint64_t gbit[4];  // global (qubit) bit of each register bit
  uint16_t lbit[4];  // local-index bit of each register bit
  int8_t q[kXMaxM];  // sub-cube local bits, lane order
  uint8_t nq;
  uint8_t m1, m3;    // register-bit masks of steps 1 and 3
  uint8_t diag;      // XDiag (at most one phase of a pass has one)
  uint8_t kq;        // sub-cube bits that are bank-column bits (lanes 0..kq-1)
  uint8_t kn;        // register bits that are bank-column bits, relabelled by lanes kq..kq+kn-1
  uint8_t kidx[4];   // their register-bit indices
};

struct XPass {
  int m, c, n_phases;
  uint32_t flags;
  int c1, c3, cd;    // coefficient-table offsets (complex64 entries): step-1 (c, s), step-3 (c, s), diag LUT
  int slot[3];       // output slot of accumulator 0 (step 1), 1 (diag), 2 (step 3); -1: none
  int fs_off;        // byte offset of this pass's in-tile edge-count table (2^m bytes)
  int ncomp;         // complement (tile-index) bits
  int n_cc;          // complement nodes with complement neighbours above them
  int cw;            // coefficient offset of the pass's phase weights: per phase (w1, w3), (wd, 0)
  int8_t comp[kXMaxComp];
  uint8_t ccnode[kXMaxComp];
  uint64_t ccmask[kXMaxComp];  // complement neighbours (above) of ccnode[k]
  uint64_t wmask[kXMaxM];      // complement neighbours of tile (local) bit i
  uint64_t hiA[64], hiB[64];   // global bits of local bits c..c+5 and c+6..c+11
  // TMA tensor maps of the tile, [0] load, [1] store.  The array is viewed as
  // 8-byte words (a 16-byte element is two words: me = 1); its word-index bits
  // are cut into five dimensions, dim i spanning bits [ma[i], ma[i] + mw[i]),
  // of which the box holds the low mbx[i].  The boxes cover the low mlb local
  // bits of the tile; the 2^(m - mlb) boxes of a tile differ in the higher ones.
  uint8_t ma[2][5], mw[2][5], mbx[2][5], me[2], mlb[2];
  uint8_t mpad[6];
  XPhase ph[kXMaxPhases];
};

// Splits the word-index bits of a tile (bit set S of an n-qubit array, words
// per amplitude 2^e) into the five dimensions of a tensor map; false when the
// tile needs more than 32 boxes or a dimension is wider than 31 bits.
bool qx_map_dims(uint64_t S, int n, int e, int m, uint8_t a[5], uint8_t w[5], uint8_t bx[5], uint8_t* lb);

struct XLaunch {
  float2* psi;                 // plain complex64 state
  float4* il;                  // interleaved (psi.re, lam.re, psi.im, lam.im) per amplitude, 2^n entries
  const float2* coef;
  const uint8_t* fs;
  double* partials;
  int stride, grid, n, n_edges;
};

// Register bits per phase: 4 (16 amplitudes per thread) for psi alone, 3 (8
// psi/lam pairs) in the two-state kernel, whose 2^(m-3) compute threads then
// fit in 96 registers: twice the warps of 4 register bits at 168.
constexpr int qx_reg_bits(bool two_state) { return two_state ? 3 : 4; }

// two_state = 0: forward kernel (psi alone, 8-byte elements); 1: psi and lam
// interleaved (16-byte elements).  Returns the resident CTAs per SM (0: does
// not fit) for a tile of 2^m amplitudes.
int qx_occupancy(int two_state, int m, int n_edges, int n_phases);
int qx_grid(int two_state, int m, int n_edges, int n_phases, uint64_t n_tiles);
qs_status launch_qx_pass(int two_state, const XPass* d_pass, const XPass& h_pass, const XLaunch& L,
                         cudaStream_t st);
// psi[x] <-> psi[NOT x] over the n-qubit complex64 state (n >= 2)
qs_status launch_qx_flip(float2* psi, int n, cudaStream_t st);

}  // namespace qs
