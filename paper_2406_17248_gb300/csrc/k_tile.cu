// Fused shared-memory tile passes.
//
// One pass streams the state once through shared memory: the CTA loads a tile
// of 2^m amplitudes whose index bits are a chosen set S of qubits (the low c
// qubits, contiguous in HBM, plus m - c gathered higher qubits), applies a run
// of gates whose non-diagonal targets lie in S, and stores the tile back.
// Inside the tile, work proceeds in phases: each thread holds 2^kRegBits
// amplitudes in registers, a sub-cube spanned by the phase's register bits R,
// applies every op of the phase to them, and writes them back.  Controls and
// diagonal gates may sit on any qubit: their bits are read from the local index
// or from the tile offset.  The reverse (adjoint) passes carry psi and lam
// together and accumulate <lam|A|psi> partials per gate (the adjoint gradient
// of §4.1 / §7.2), reduced per warp in registers and per CTA in FP64.
#include "qsim_internal.h"

namespace qs {

template <class T>
struct VecT;
template <>
struct VecT<float> {
  using V = float2;
  using V4 = float4;
};
template <>
struct VecT<double> {
  using V = double2;
  using V4 = double2;  // one amplitude per 16-byte chunk
};

__device__ __forceinline__ float fmaT(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fmaT(double a, double b, double c) { return __fma_rn(a, b, c); }

template <class V>
__device__ __forceinline__ V cmul(V a, V b) {
  V r;
  r.x = fmaT(a.x, b.x, -a.y * b.y);
  r.y = fmaT(a.x, b.y, a.y * b.x);
  return r;
}
template <class V>
__device__ __forceinline__ V cfma(V a, V b, V acc) {  // acc + a * b
  acc.x = fmaT(a.x, b.x, acc.x);
  acc.x = fmaT(-a.y, b.y, acc.x);
  acc.y = fmaT(a.x, b.y, acc.y);
  acc.y = fmaT(a.y, b.x, acc.y);
  return acc;
}
// Re(conj(a) * b)
template <class V>
__device__ __forceinline__ decltype(V::x) re_conj_mul(V a, V b) {
  return fmaT(a.x, b.x, a.y * b.y);
}
// Im(conj(a) * b)
template <class V>
__device__ __forceinline__ decltype(V::x) im_conj_mul(V a, V b) {
  return fmaT(a.x, b.y, -a.y * b.x);
}

// Bank-conflict swizzle of a local index: XOR the bank bits with a fold of the
// higher bits (a bijection that keeps pairs (2k, 2k+1) within one 16-byte chunk
// for complex64).
template <class T>
__device__ __forceinline__ uint32_t swz(uint32_t l);
template <>
__device__ __forceinline__ uint32_t swz<float>(uint32_t l) {
  uint32_t v = l >> 4;
  return l ^ ((v ^ (v >> 4) ^ (v >> 8)) & 15u);
}
template <>
__device__ __forceinline__ uint32_t swz<double>(uint32_t l) {
  uint32_t v = l >> 3;
  return l ^ ((v ^ (v >> 3) ^ (v >> 6) ^ (v >> 9)) & 7u);
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

constexpr int RN = 1 << kRegBits;
constexpr int kTileOpStage = 256;  // ops of a pass staged in shared memory (more: read from global)


template <int J>
__device__ __forceinline__ uint32_t off_of(const uint32_t (&rm)[kRegBits]) {
  uint32_t o = 0;
#pragma unroll
  for (int i = 0; i < kRegBits; ++i)
    if (J & (1 << i)) o |= rm[i];
  return o;
}

// 16-bit pattern over the register index j of one diagonal bit: local bit
// `dloc` (-1: the bit is outside the tile, with value g).  A local bit held in
// register bit i gives the fixed pattern of bit i of j; any other local bit is
// constant for the thread's sub-cube (all ones or all zeros).
__device__ __forceinline__ uint32_t diag_pattern(int dloc, bool g, uint32_t l0, const uint32_t (&rm)[kRegBits]) {
  if (dloc < 0) return g ? 0xFFFFu : 0u;
  const uint32_t bit = 1u << dloc;
  constexpr uint32_t kPat[4] = {0xAAAAu, 0xCCCCu, 0xF0F0u, 0xFF00u};
#pragma unroll
  for (int i = 0; i < kRegBits; ++i)
    if (rm[i] == bit) return kPat[i];
  return (l0 & bit) ? 0xFFFFu : 0u;
}

// JC: the op has controls among the register bits (mask jc over the register
// index); without them the whole loop is predicated by `ok` alone.
template <class V, int RB, bool JC>
__device__ __forceinline__ void op_dense1(V (&a)[RN], const V* M, uint32_t jc, bool ok) {
  const V m00 = M[0], m01 = M[1], m10 = M[2], m11 = M[3];
#pragma unroll
  for (int j = 0; j < RN; ++j) {
    if (j & (1 << RB)) continue;
    const int j1 = j | (1 << RB);
    if (ok && (!JC || ((uint32_t)j & jc) == jc)) {
      V x0 = a[j], x1 = a[j1];
      a[j] = cfma(m01, x1, cmul(m00, x0));
      a[j1] = cfma(m11, x1, cmul(m10, x0));
    }
  }
}

template <class V, int RB, bool JC>
__device__ __forceinline__ void op_rx(V (&a)[RN], V cs, uint32_t jc, bool ok) {
  // [[c, -is], [-is, c]]: out0 = c x0 - i s x1, out1 = c x1 - i s x0
  const auto c = cs.x, s = cs.y;
#pragma unroll
  for (int j = 0; j < RN; ++j) {
    if (j & (1 << RB)) continue;
    const int j1 = j | (1 << RB);
    if (ok && (!JC || ((uint32_t)j & jc) == jc)) {
      V x0 = a[j], x1 = a[j1], y0, y1;
      y0.x = fmaT(c, x0.x, s * x1.y);
      y0.y = fmaT(c, x0.y, -s * x1.x);
      y1.x = fmaT(c, x1.x, s * x0.y);
      y1.y = fmaT(c, x1.y, -s * x0.x);
      a[j] = y0;
      a[j1] = y1;
    }
  }
}

template <class V, int RB, bool JC>
__device__ __forceinline__ void op_x(V (&a)[RN], uint32_t jc, bool ok) {
#pragma unroll
  for (int j = 0; j < RN; ++j) {
    if (j & (1 << RB)) continue;
    const int j1 = j | (1 << RB);
    if (ok && (!JC || ((uint32_t)j & jc) == jc)) {
      const V x0 = a[j];
      a[j] = a[j1];
      a[j1] = x0;
    }
  }
}

// 2x2 matrix with real entries (the real parts of M): 4 instead of 8 products per pair.
template <class V, int RB, bool JC>
__device__ __forceinline__ void op_real1(V (&a)[RN], const V* M, uint32_t jc, bool ok) {
  const auto m00 = M[0].x, m01 = M[1].x, m10 = M[2].x, m11 = M[3].x;
#pragma unroll
  for (int j = 0; j < RN; ++j) {
    if (j & (1 << RB)) continue;
    const int j1 = j | (1 << RB);
    if (ok && (!JC || ((uint32_t)j & jc) == jc)) {
      const V x0 = a[j], x1 = a[j1];
      V y0, y1;
      y0.x = fmaT(m01, x1.x, m00 * x0.x);
      y0.y = fmaT(m01, x1.y, m00 * x0.y);
      y1.x = fmaT(m11, x1.x, m10 * x0.x);
      y1.y = fmaT(m11, x1.y, m10 * x0.y);
      a[j] = y0;
      a[j1] = y1;
    }
  }
}

// Exact product i^k a (k = 0..3): a swap of the components and sign-bit flips
// on the integer pipe.
__device__ __forceinline__ double flip_sign(double v, uint32_t neg) {
  return __longlong_as_double(__double_as_longlong(v) ^ ((long long)neg << 63));
}
template <class V>
__device__ __forceinline__ V mul_ik(uint32_t k, V a) {
  V r;
  r.x = flip_sign((k & 1u) ? a.y : a.x, ((k + 1u) >> 1) & 1u);  // k = 1, 2: -
  r.y = flip_sign((k & 1u) ? a.x : a.y, (k >> 1) & 1u);         // k = 2, 3: -
  return r;
}

// k of an entry i^k of a unit diagonal, from its bit pattern (the planner emits
// OP_UDIAG only for entries that are exactly 1, i, -1 or -i).
__device__ __forceinline__ uint32_t unit_code_of(double2 d) {
  const long long one = 0x3FF0000000000000ll, minus_one = (long long)0xBFF0000000000000ull;
  const long long re = __double_as_longlong(d.x), im = __double_as_longlong(d.y);
  return re == one ? 0u : im == one ? 1u : re == minus_one ? 2u : 3u;
}

template <class V, int RB0, int RB1, bool JC>
__device__ __forceinline__ void op_dense2(V (&a)[RN], const V* M, uint32_t jc, bool ok) {
#pragma unroll
  for (int j = 0; j < RN; ++j) {
    if (j & ((1 << RB0) | (1 << RB1))) continue;
    if (!(ok && (!JC || ((uint32_t)j & jc) == jc))) continue;
    const int idx[4] = {j, j | (1 << RB0), j | (1 << RB1), j | (1 << RB0) | (1 << RB1)};
    V x[4] = {a[idx[0]], a[idx[1]], a[idx[2]], a[idx[3]]};
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      V y = cmul(M[4 * r], x[0]);
      y = cfma(M[4 * r + 1], x[1], y);
      y = cfma(M[4 * r + 2], x[2], y);
      y = cfma(M[4 * r + 3], x[3], y);
      a[idx[r]] = y;
    }
  }
}

template <class V, int RB, bool JC>
__device__ __forceinline__ auto grad_dense1(const V (&a)[RN], const V (&b)[RN], const V* A, uint32_t jc,
                                            bool ok) -> decltype(V::x) {
  decltype(V::x) acc = 0;
  const V a00 = A[0], a01 = A[1], a10 = A[2], a11 = A[3];
#pragma unroll
  for (int j = 0; j < RN; ++j) {
    if (j & (1 << RB)) continue;
    const int j1 = j | (1 << RB);
    if (ok && (!JC || ((uint32_t)j & jc) == jc)) {
      V y0 = cfma(a01, a[j1], cmul(a00, a[j]));
      V y1 = cfma(a11, a[j1], cmul(a10, a[j]));
      acc += re_conj_mul(b[j], y0) + re_conj_mul(b[j1], y1);
    }
  }
  return 2 * acc;
}

template <class V, int RB0, int RB1, bool JC>
__device__ __forceinline__ auto grad_dense2(const V (&a)[RN], const V (&b)[RN], const V* M, uint32_t jc,
                                            bool ok) -> decltype(V::x) {
  decltype(V::x) acc = 0;
#pragma unroll
  for (int j = 0; j < RN; ++j) {
    if (j & ((1 << RB0) | (1 << RB1))) continue;
    if (!(ok && (!JC || ((uint32_t)j & jc) == jc))) continue;
    const int idx[4] = {j, j | (1 << RB0), j | (1 << RB1), j | (1 << RB0) | (1 << RB1)};
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      V y = cmul(M[4 * r], a[idx[0]]);
      y = cfma(M[4 * r + 1], a[idx[1]], y);
      y = cfma(M[4 * r + 2], a[idx[2]], y);
      y = cfma(M[4 * r + 3], a[idx[3]], y);
      acc += re_conj_mul(b[idx[r]], y);
    }
  }
  return 2 * acc;
}

template <class V, int RB, bool JC>
__device__ __forceinline__ auto grad_x(const V (&a)[RN], const V (&b)[RN], uint32_t jc, bool ok)
    -> decltype(V::x) {
  decltype(V::x) acc = 0;
#pragma unroll
  for (int j = 0; j < RN; ++j) {
    if (j & (1 << RB)) continue;
    const int j1 = j | (1 << RB);
    if (ok && (!JC || ((uint32_t)j & jc) == jc)) acc += im_conj_mul(b[j], a[j1]) + im_conj_mul(b[j1], a[j]);
  }
  return acc;
}

#define QS_RB_SWITCH(rb, CALL) \
  switch (rb) {                \
    case 0: CALL(0); break;    \
    case 1: CALL(1); break;    \
    case 2: CALL(2); break;    \
    default: CALL(3); break;   \
  }

#define QS_RB2_SWITCH(r0, r1, CALL)      \
  switch ((r0) * 4 + (r1)) {             \
    case 1: CALL(0, 1); break;           \
    case 2: CALL(0, 2); break;           \
    case 3: CALL(0, 3); break;           \
    case 4: CALL(1, 0); break;           \
    case 6: CALL(1, 2); break;           \
    case 7: CALL(1, 3); break;           \
    case 8: CALL(2, 0); break;           \
    case 9: CALL(2, 1); break;           \
    case 11: CALL(2, 3); break;          \
    case 12: CALL(3, 0); break;          \
    case 13: CALL(3, 1); break;          \
    default: CALL(3, 2); break;          \
  }

#ifndef QS_TILE_C64_MINB
#define QS_TILE_C64_MINB 2
#endif
// The pass body: one CTA's share (tiles blockIdx.x, + gridDim.x, ...) of one
// instance's pass, its gradient partials in column blockIdx.x.
template <class T, int NS>
__device__ __forceinline__ void tile_pass_body(const TileKArgs& args) {
  using V = typename VecT<T>::V;
  extern __shared__ __align__(16) unsigned char smem_raw[];

  const DevPass& P = *args.pass;
  const int m = P.m, c = P.c;
  const uint32_t flags = P.flags;
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const uint32_t tile_n = 1u << m;

  V* s_psi = reinterpret_cast<V*>(smem_raw);
  V* s_lam = s_psi + (NS == 2 ? tile_n : 0);
  uint8_t* s_cut = reinterpret_cast<uint8_t*>(s_psi + NS * tile_n);
  double* s_acc = reinterpret_cast<double*>(s_cut + ((flags & PF_NEED_CUT) ? tile_n : 0));
  uint64_t* s_hi = reinterpret_cast<uint64_t*>(s_acc + P.n_slots * kTileWarps);  // hiA[64], hiB[64]
  DevOp* s_ops = reinterpret_cast<DevOp*>(s_hi + 128);  // the pass's ops, when they fit

  for (int i = tid; i < 64; i += blockDim.x) {
    s_hi[i] = P.hiA[i];
    s_hi[64 + i] = P.hiB[i];
  }
  // Sub-cube bases of every phase: the local index l0 of sub-cube u deposits u's
  // bits into the phase's Q bits; split u = lo (4 bits) | hi (up to 5 bits) and
  // tabulate each half, so l0 = tab[lo] | tab[16 + hi].
  uint32_t* s_l0 = reinterpret_cast<uint32_t*>(s_ops + kTileOpStage);  // [phase][48]
  for (int e = tid; e < P.n_phases * 48; e += blockDim.x) {
    const int ph = e / 48, k = e % 48;
    const DevPhase& PH = args.phases[P.phase_begin + ph];
    const int first = k < 16 ? 0 : 4;
    const uint32_t bits = k < 16 ? (uint32_t)k : (uint32_t)(k - 16);
    uint32_t v = 0;
    for (int i = 0; i < 5 && first + i < PH.nq; ++i)
      if ((bits >> i) & 1u) v |= 1u << PH.Q[first + i];
    s_l0[e] = (k < 16 || bits < 32) ? v : 0u;
  }
  const int op_lo = P.n_phases ? args.phases[P.phase_begin].op_begin : 0;
  const int op_hi = P.n_phases ? args.phases[P.phase_begin + P.n_phases - 1].op_end : 0;
  const bool ops_staged = op_hi - op_lo <= kTileOpStage;
  if (ops_staged) {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(args.ops + op_lo);
    uint32_t* dst = reinterpret_cast<uint32_t*>(s_ops);
    for (int i = tid; i < (op_hi - op_lo) * (int)(sizeof(DevOp) / 4); i += blockDim.x) dst[i] = src[i];
  }
  for (int i = tid; i < P.n_slots * kTileWarps; i += blockDim.x) s_acc[i] = 0.0;
  __syncthreads();

  const V* coef = reinterpret_cast<const V*>(args.coef);
  V* g_psi = reinterpret_cast<V*>(args.psi);
  V* g_lam = reinterpret_cast<V*>(args.lam);
  const uint32_t lowmask = (1u << c) - 1u;
  const uint64_t n_tiles = 1ull << (args.n - m);
  const T plus_amp = (T)exp2(-0.5 * (double)args.n);
  const int n_edges = args.n_edges;

  for (uint64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    uint64_t toff = 0;
    for (int i = 0; i < P.ncomp; ++i) toff |= ((tile >> i) & 1ull) << P.comp[i];

    // ---------------------------------------------------------------- load
    if (sizeof(T) == 4) {
      const uint32_t nch = tile_n >> 1;
      for (uint32_t ch = tid; ch < nch; ch += blockDim.x) {
        const uint32_t l = ch << 1;
        const uint64_t g = toff | (l & lowmask) | s_hi[(l >> c) & 63] | s_hi[64 + (l >> (c + 6))];
        uint32_t p = swz<T>(l);
        const bool sw = p & 1;
        p &= ~1u;
#pragma unroll
        for (int s = 0; s < NS; ++s) {
          float4 v;
          if (s == 0 && (flags & (PF_GEN_PLUS | PF_GEN_ZERO))) {
            float a0 = (flags & PF_GEN_PLUS) ? (float)plus_amp : (g == 0 ? 1.f : 0.f);
            float a1 = (flags & PF_GEN_PLUS) ? (float)plus_amp : 0.f;
            v = make_float4(a0, 0.f, a1, 0.f);
          } else if ((s == 0 && (flags & PF_LOAD_PSI)) || (s == 1 && (flags & PF_LOAD_LAM))) {
            const float4* src = reinterpret_cast<const float4*>((s == 0 ? g_psi : g_lam) + g);
            v = __ldcs(src);
          } else {
            continue;
          }
          if (sw) v = make_float4(v.z, v.w, v.x, v.y);
          *reinterpret_cast<float4*>((s == 0 ? s_psi : s_lam) + p) = v;
        }
        if (flags & PF_NEED_CUT) {
          s_cut[l] = args.cut[g];
          s_cut[l + 1] = args.cut[g + 1];
        }
      }
    } else {
      for (uint32_t l = tid; l < tile_n; l += blockDim.x) {
        const uint64_t g = toff | (l & lowmask) | s_hi[(l >> c) & 63] | s_hi[64 + (l >> (c + 6))];
        const uint32_t p = swz<T>(l);
#pragma unroll
        for (int s = 0; s < NS; ++s) {
          V v;
          if (s == 0 && (flags & (PF_GEN_PLUS | PF_GEN_ZERO))) {
            v.x = (flags & PF_GEN_PLUS) ? plus_amp : (g == 0 ? (T)1 : (T)0);
            v.y = 0;
          } else if ((s == 0 && (flags & PF_LOAD_PSI)) || (s == 1 && (flags & PF_LOAD_LAM))) {
            v = __ldcs((s == 0 ? g_psi : g_lam) + g);
          } else {
            continue;
          }
          (s == 0 ? s_psi : s_lam)[p] = v;
        }
        if (flags & PF_NEED_CUT) s_cut[l] = args.cut[g];
      }
    }
    __syncthreads();

    // ---------------------------------------------------------------- phases
    for (int ph = 0; ph < P.n_phases; ++ph) {
      const DevPhase& PH = args.phases[P.phase_begin + ph];
      uint32_t rm[kRegBits], sm[kRegBits];
#pragma unroll
      for (int i = 0; i < kRegBits; ++i) {
        rm[i] = 1u << PH.R[i];
        sm[i] = swz<T>(rm[i]);  // the swizzle is linear over GF(2): positions XOR
      }
      const uint32_t* l0tab = s_l0 + ph * 48;
      const uint32_t nsub = tile_n >> kRegBits;
      const uint32_t iters = (nsub + blockDim.x - 1) / blockDim.x;
      for (uint32_t it = 0; it < iters; ++it) {
        const uint32_t u = tid + it * blockDim.x;
        const bool active = u < nsub;
        const uint32_t l0 = active ? (l0tab[u & 15u] | l0tab[16 + ((u >> 4) & 31u)]) : 0u;
        const uint32_t p0 = swz<T>(l0);
        // position and local index of register element j (constants per j)
#define TPOS(j) \
  (p0 ^ (((j) & 1) ? sm[0] : 0u) ^ (((j) & 2) ? sm[1] : 0u) ^ (((j) & 4) ? sm[2] : 0u) ^ (((j) & 8) ? sm[3] : 0u))
#define TLOC(j) \
  (l0 | (((j) & 1) ? rm[0] : 0u) | (((j) & 2) ? rm[1] : 0u) | (((j) & 4) ? rm[2] : 0u) | (((j) & 8) ? rm[3] : 0u))
        V a[RN], b[RN];
        if (active) {
#pragma unroll
          for (int j = 0; j < RN; ++j) {
            const uint32_t p = TPOS(j);
            a[j] = s_psi[p];
            if (NS == 2) b[j] = s_lam[p];
          }
        } else {
#pragma unroll
          for (int j = 0; j < RN; ++j) {
            a[j].x = a[j].y = 0;
            if (NS == 2) b[j].x = b[j].y = 0;
          }
        }
        for (int o = PH.op_begin; o < PH.op_end; ++o) {
          const DevOp op = ops_staged ? s_ops[o - op_lo] : args.ops[o];
          const bool ok = active && ((l0 & op.lc) == op.lc) && ((toff & op.gc) == op.gc);
          // an op that only transforms amplitudes is skipped outright where it
          // does not apply (ops with sums keep every lane for the warp shuffle)
          if (!ok && op.type <= OP_RX) continue;
          if (!ok && (op.type >= OP_X || op.type == OP_COST)) continue;
          const uint32_t jc = op.jc;
          const V* M = coef + op.coef;
          T contrib = 0;
          bool has_contrib = false;
          switch (op.type) {
            case OP_DENSE1: {
#define CALLJ(R, J)                          \
  op_dense1<V, R, J>(a, M, jc, ok);          \
  if (NS == 2 && (op.flags & OPF_LAM)) op_dense1<V, R, J>(b, M, jc, ok);
#define CALL(R) if (jc) { CALLJ(R, true) } else { CALLJ(R, false) }
              QS_RB_SWITCH(op.rb0, CALL)
#undef CALL
#undef CALLJ
              break;
            }
            case OP_X: {  // complex128 forward passes only (where the planner emits it)
              if constexpr (NS == 1 && sizeof(T) == 8) {
#define CALL(R) if (jc) { op_x<V, R, true>(a, jc, ok); } else { op_x<V, R, false>(a, jc, ok); }
                QS_RB_SWITCH(op.rb0, CALL)
#undef CALL
              }
              break;
            }
            case OP_REAL1: {  // complex128 one-state passes only (where the planner emits it)
              if constexpr (NS == 1 && sizeof(T) == 8) {
#define CALL(R) if (jc) { op_real1<V, R, true>(a, M, jc, ok); } else { op_real1<V, R, false>(a, M, jc, ok); }
                QS_RB_SWITCH(op.rb0, CALL)
#undef CALL
              }
              break;
            }
            case OP_UDIAG: {  // complex128 one-state passes only: entries i^k, no FP64 arithmetic
              if constexpr (NS == 1 && sizeof(T) == 8) {
                const bool g0 = op.dglb[0] >= 0 && ((toff >> op.dglb[0]) & 1ull);
                const bool g1 = op.dglb[1] >= 0 && ((toff >> op.dglb[1]) & 1ull);
                const uint32_t codes = unit_code_of(M[0]) | (unit_code_of(M[1]) << 2) | (unit_code_of(M[2]) << 4) |
                                       (unit_code_of(M[3]) << 6);
#pragma unroll
                for (int j = 0; j < RN; ++j) {
                  if (!(ok && ((uint32_t)j & jc) == jc)) continue;
                  const uint32_t b0 = op.dloc[0] >= 0 ? (TLOC(j) >> op.dloc[0]) & 1u : (uint32_t)g0;
                  const uint32_t b1 = op.dloc[1] >= 0 ? (TLOC(j) >> op.dloc[1]) & 1u : (uint32_t)g1;
                  a[j] = mul_ik((codes >> (2 * (b0 | (b1 << 1)))) & 3u, a[j]);
                }
              }
              break;
            }
            case OP_RX: {
              const V cs = M[0];
#define CALLJ(R, J)                        \
  op_rx<V, R, J>(a, cs, jc, ok);           \
  if (NS == 2 && (op.flags & OPF_LAM)) op_rx<V, R, J>(b, cs, jc, ok);
#define CALL(R) if (jc) { CALLJ(R, true) } else { CALLJ(R, false) }
              QS_RB_SWITCH(op.rb0, CALL)
#undef CALL
#undef CALLJ
              break;
            }
            case OP_DENSE2: {
#define CALLJ(R0, R1, J)                         \
  op_dense2<V, R0, R1, J>(a, M, jc, ok);         \
  if (NS == 2 && (op.flags & OPF_LAM)) op_dense2<V, R0, R1, J>(b, M, jc, ok);
#define CALL(R0, R1) if (jc) { CALLJ(R0, R1, true) } else { CALLJ(R0, R1, false) }
              QS_RB2_SWITCH(op.rb0, op.rb1, CALL)
#undef CALL
#undef CALLJ
              break;
            }
            case OP_DIAG:
            case OP_GRADDIAG: {
              const bool g0 = op.dglb[0] >= 0 && ((toff >> op.dglb[0]) & 1ull);
              const bool g1 = op.dglb[1] >= 0 && ((toff >> op.dglb[1]) & 1ull);
              // the four diagonal entries (every diagonal op's block has four
              // slots) in registers: a select per amplitude, not a load
              const V D0 = M[0], D1 = M[1], D2 = M[2], D3 = M[3];
              // complex64 (ALU-bound): each diagonal bit as a pattern over the
              // register index j -- a register bit varies with j, any other bit is
              // constant here, and with both constant one factor serves all j;
              // complex128 (FP64-bound) measured faster with per-j bit extraction
              const uint32_t P0 = diag_pattern(op.dloc[0], g0, l0, rm);
              const uint32_t P1 = diag_pattern(op.dloc[1], g1, l0, rm);
              if (sizeof(T) == 8) {
#pragma unroll
                for (int j = 0; j < RN; ++j) {
                  if (!(ok && ((uint32_t)j & jc) == jc)) continue;
                  const uint32_t b0 = op.dloc[0] >= 0 ? (TLOC(j) >> op.dloc[0]) & 1u : (uint32_t)g0;
                  const uint32_t b1 = op.dloc[1] >= 0 ? (TLOC(j) >> op.dloc[1]) & 1u : (uint32_t)g1;
                  const V d = b1 ? (b0 ? D3 : D2) : (b0 ? D1 : D0);
                  if (op.type == OP_DIAG) {
                    a[j] = cmul(d, a[j]);
                    if (NS == 2 && (op.flags & OPF_LAM)) b[j] = cmul(d, b[j]);
                  } else if (NS == 2) {
                    contrib += 2 * re_conj_mul(b[j], cmul(d, a[j]));
                  }
                }
              } else if ((P0 == 0u || P0 == 0xFFFFu) && (P1 == 0u || P1 == 0xFFFFu)) {
                const V d = P1 ? (P0 ? D3 : D2) : (P0 ? D1 : D0);  // one factor for all
#pragma unroll
                for (int j = 0; j < RN; ++j) {
                  if (!(ok && ((uint32_t)j & jc) == jc)) continue;
                  if (op.type == OP_DIAG) {
                    a[j] = cmul(d, a[j]);
                    if (NS == 2 && (op.flags & OPF_LAM)) b[j] = cmul(d, b[j]);
                  } else if (NS == 2) {
                    contrib += 2 * re_conj_mul(b[j], cmul(d, a[j]));
                  }
                }
              } else {
#pragma unroll
                for (int j = 0; j < RN; ++j) {
                  if (!(ok && ((uint32_t)j & jc) == jc)) continue;
                  const bool b0 = (P0 >> j) & 1u, b1 = (P1 >> j) & 1u;
                  const V d = b1 ? (b0 ? D3 : D2) : (b0 ? D1 : D0);
                  if (op.type == OP_DIAG) {
                    a[j] = cmul(d, a[j]);
                    if (NS == 2 && (op.flags & OPF_LAM)) b[j] = cmul(d, b[j]);
                  } else if (NS == 2) {
                    contrib += 2 * re_conj_mul(b[j], cmul(d, a[j]));
                  }
                }
              }
              has_contrib = op.type == OP_GRADDIAG;
              break;
            }
            case OP_GRAD1: {
              if (NS == 2) {
#define CALL(R) contrib = jc ? grad_dense1<V, R, true>(a, b, M, jc, ok) : grad_dense1<V, R, false>(a, b, M, jc, ok);
                QS_RB_SWITCH(op.rb0, CALL)
#undef CALL
              }
              has_contrib = true;
              break;
            }
            case OP_GRAD2: {
              if (NS == 2) {
#define CALL(R0, R1) \
  contrib = jc ? grad_dense2<V, R0, R1, true>(a, b, M, jc, ok) : grad_dense2<V, R0, R1, false>(a, b, M, jc, ok);
                QS_RB2_SWITCH(op.rb0, op.rb1, CALL)
#undef CALL
              }
              has_contrib = true;
              break;
            }
            case OP_GRADX: {
              if (NS == 2) {
#define CALL(R) contrib = jc ? grad_x<V, R, true>(a, b, jc, ok) : grad_x<V, R, false>(a, b, jc, ok);
                QS_RB_SWITCH(op.rb0, CALL)
#undef CALL
              }
              has_contrib = true;
              break;
            }
            case OP_COST: {
              if (active) {
#pragma unroll
                for (int j = 0; j < RN; ++j) {
                  const V d = M[s_cut[TLOC(j)]];
                  a[j] = cmul(d, a[j]);
                  if (NS == 2 && (op.flags & OPF_LAM)) b[j] = cmul(d, b[j]);
                }
              }
              break;
            }
            case OP_GRADCOST: {
              if (NS == 2 && active) {
#pragma unroll
                for (int j = 0; j < RN; ++j) {
                  const T C = (T)(n_edges - 2 * (int)s_cut[TLOC(j)]);
                  contrib += C * im_conj_mul(b[j], a[j]);
                }
              }
              has_contrib = true;
              break;
            }
            case OP_ENERGY: {
              if (active) {
#pragma unroll
                for (int j = 0; j < RN; ++j) {
                  const T C = (T)(n_edges - 2 * (int)s_cut[TLOC(j)]);
                  contrib += C * fmaT(a[j].x, a[j].x, a[j].y * a[j].y);
                  if (NS == 2) {
                    b[j].x = C * a[j].x;
                    b[j].y = C * a[j].y;
                  }
                }
              }
              has_contrib = true;
              break;
            }
            default:
              break;
          }
          if (has_contrib) {  // uniform across the CTA (depends on op only)
            const T w = warp_sum(contrib);
            if (lane == 0) s_acc[op.slot * kTileWarps + warp] += (double)w;
          }
        }
        if (active) {
#pragma unroll
          for (int j = 0; j < RN; ++j) {
            const uint32_t p = TPOS(j);
            s_psi[p] = a[j];
            if (NS == 2) s_lam[p] = b[j];
          }
        }
#undef TPOS
#undef TLOC
      }
      __syncthreads();
    }

    // ---------------------------------------------------------------- store
    if (flags & (PF_STORE_PSI | PF_STORE_LAM)) {
      if (sizeof(T) == 4) {
        const uint32_t nch = tile_n >> 1;
        for (uint32_t ch = tid; ch < nch; ch += blockDim.x) {
          const uint32_t l = ch << 1;
          const uint64_t g = toff | (l & lowmask) | s_hi[(l >> c) & 63] | s_hi[64 + (l >> (c + 6))];
          uint32_t p = swz<T>(l);
          const bool sw = p & 1;
          p &= ~1u;
#pragma unroll
          for (int s = 0; s < NS; ++s) {
            if (!((s == 0 && (flags & PF_STORE_PSI)) || (s == 1 && (flags & PF_STORE_LAM)))) continue;
            float4 v = *reinterpret_cast<const float4*>((s == 0 ? s_psi : s_lam) + p);
            if (sw) v = make_float4(v.z, v.w, v.x, v.y);
            __stcs(reinterpret_cast<float4*>((s == 0 ? g_psi : g_lam) + g), v);
          }
        }
      } else {
        for (uint32_t l = tid; l < tile_n; l += blockDim.x) {
          const uint64_t g = toff | (l & lowmask) | s_hi[(l >> c) & 63] | s_hi[64 + (l >> (c + 6))];
          const uint32_t p = swz<T>(l);
#pragma unroll
          for (int s = 0; s < NS; ++s) {
            if (!((s == 0 && (flags & PF_STORE_PSI)) || (s == 1 && (flags & PF_STORE_LAM)))) continue;
            __stcs((s == 0 ? g_psi : g_lam) + g, (s == 0 ? s_psi : s_lam)[p]);
          }
        }
      }
    }
    __syncthreads();
  }

  // ------------------------------------------------------------------ partials
  for (int s = tid; s < P.n_slots; s += blockDim.x) {
    double v = 0.0;
    for (int w = 0; w < kTileWarps; ++w) v += s_acc[s * kTileWarps + w];
    args.partials[(size_t)(P.slot_base + s) * args.grid_stride + blockIdx.x] = v;
  }
}

template <class T, int NS>
__global__ void __launch_bounds__(kTileThreads, sizeof(T) == 4 ? QS_TILE_C64_MINB : 1) tile_pass_kernel(TileKArgs args) {
  tile_pass_body<T, NS>(args);
}

// The same pass of many independent instances (equal tile shape and grid) in
// one launch: instance blockIdx.y, its arguments from a device table.
template <class T, int NS>
__global__ void __launch_bounds__(kTileThreads, sizeof(T) == 4 ? QS_TILE_C64_MINB : 1)
    tile_pass_multi_kernel(const TileKArgs* __restrict__ argv) {
  const TileKArgs args = argv[blockIdx.y];
  tile_pass_body<T, NS>(args);
}

size_t tile_smem_bytes(qs_dtype dt, int m, int ns) {
  const size_t amp = dt == QS_C64 ? 8 : 16;
  const size_t tile = (size_t)1 << m;
  return ns * tile * amp + tile /* cut */ + (size_t)kMaxSlotsPerPass * kTileWarps * 8 + 128 * 8 +
         (size_t)kTileOpStage * sizeof(DevOp) + (size_t)kMaxPhasesPerPass * 48 * 4;
}

template <class T, int NS>
static int occupancy_for(size_t smem) {
  static int cached[2] = {0, 0};
  static size_t cached_smem[2] = {0, 0};
  const int key = 0;
  if (cached[key] && cached_smem[key] == smem) return cached[key];
  int blocks = 0;
  if (cudaFuncSetAttribute(tile_pass_kernel<T, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, tile_pass_kernel<T, NS>, kTileThreads, smem) !=
          cudaSuccess ||
      blocks < 1) {
    (void)cudaGetLastError();  // the probe's error must not surface at a later launch check
    blocks = 1;
  }
  cached[key] = blocks;
  cached_smem[key] = smem;
  return blocks;
}

static int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

int tile_grid_size(qs_dtype dt, int m, int ns, int n_tiles) {
  const size_t smem = tile_smem_bytes(dt, m, ns);
  int occ;
  if (dt == QS_C64)
    occ = ns == 2 ? occupancy_for<float, 2>(smem) : occupancy_for<float, 1>(smem);
  else
    occ = ns == 2 ? occupancy_for<double, 2>(smem) : occupancy_for<double, 1>(smem);
  // the partials stride is shared by the 1- and 2-state passes of one plan: use
  // the 2-state occupancy for both (it is never larger)
  long g = (long)sm_count() * occ;
  if (g > n_tiles) g = n_tiles;
  return (int)(g < 1 ? 1 : g);
}

qs_status launch_tile_pass_multi(qs_dtype dt, int ns, int m, const TileKArgs* d_argv, int count, int grid,
                                 cudaStream_t st) {
  if (count <= 0) return QS_OK;
  const size_t smem = tile_smem_bytes(dt, m, ns);
  const dim3 g((unsigned)grid, (unsigned)count);
  auto prep = [&](const void* fn) { return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); };
  if (dt == QS_C64) {
    if (ns == 2) {
      QS_CUDA(prep((const void*)tile_pass_multi_kernel<float, 2>));
      tile_pass_multi_kernel<float, 2><<<g, kTileThreads, smem, st>>>(d_argv);
    } else {
      QS_CUDA(prep((const void*)tile_pass_multi_kernel<float, 1>));
      tile_pass_multi_kernel<float, 1><<<g, kTileThreads, smem, st>>>(d_argv);
    }
  } else {
    if (ns == 2) {
      QS_CUDA(prep((const void*)tile_pass_multi_kernel<double, 2>));
      tile_pass_multi_kernel<double, 2><<<g, kTileThreads, smem, st>>>(d_argv);
    } else {
      QS_CUDA(prep((const void*)tile_pass_multi_kernel<double, 1>));
      tile_pass_multi_kernel<double, 1><<<g, kTileThreads, smem, st>>>(d_argv);
    }
  }
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

qs_status launch_tile_pass(qs_dtype dt, const TilePlan& plan, int pi, const TileLaunch& L, cudaStream_t st) {
  const PlannedPass& pp = plan.passes[pi];
  if (pp.t2 && dt == QS_C64) return launch_tile2_pass(plan, pi, L, st);
  const uint32_t fl = pp.hdr.flags;
  const int ns = (fl & (PF_LOAD_LAM | PF_STORE_LAM)) ? 2 : 1;
  TileKArgs a;
  a.psi = L.psi;
  a.lam = L.lam;
  a.pass = plan.d_pass + pi;
  a.phases = plan.d_phase;
  a.ops = plan.d_ops;
  a.coef = L.coef;
  a.cut = L.cut;
  a.partials = L.partials;
  a.n = L.n;
  a.n_edges = L.n_edges;
  a.grid_stride = L.stride;
  const size_t smem = tile_smem_bytes(dt, pp.hdr.m, ns);
  if (dt == QS_C64) {
    if (ns == 2) {
      occupancy_for<float, 2>(smem);
      tile_pass_kernel<float, 2><<<L.grid, kTileThreads, smem, st>>>(a);
    } else {
      occupancy_for<float, 1>(smem);
      tile_pass_kernel<float, 1><<<L.grid, kTileThreads, smem, st>>>(a);
    }
  } else {
    if (ns == 2) {
      occupancy_for<double, 2>(smem);
      tile_pass_kernel<double, 2><<<L.grid, kTileThreads, smem, st>>>(a);
    } else {
      occupancy_for<double, 1>(smem);
      tile_pass_kernel<double, 1><<<L.grid, kTileThreads, smem, st>>>(a);
    }
  }
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

}  // namespace qs
