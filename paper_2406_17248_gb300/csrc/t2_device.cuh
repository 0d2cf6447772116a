// Device side of the complex64 micro-op tile passes (the GB300 form of the
// fused shared-memory pass: one streaming sweep of the state applies a run of
// gates), shared by the kernels compiled with the library (k_tile2.cu: the ops
// of a pass read from a table and dispatched one by one) and the per-circuit
// kernels compiled at run time (t2gen.cu: the ops of each phase as straight-line
// calls of the same bodies).  Self-contained, so that the runtime compiler
// includes it as it stands.
//
// A CTA holds 2^(m-4) compute threads (at most 512; 256 with psi and lam) and
// one producer warp, and loops over tiles through a ring of three tile
// buffers.  The producer moves tiles between HBM and shared memory with
// five-dimensional TMA tensor copies (one or a few boxes per tile, 128-byte
// swizzle) completing on mbarriers, so the compute warps never issue a global
// access.  Each phase gives a thread the 16 amplitudes of one sub-cube (4
// register bits) and runs the phase's micro-ops on them: a body compiled for
// its register bits (template arguments: no per-amplitude bit extraction,
// selects or op decoding), its coefficients in a shared-memory stage, and
// predicates for controls outside the registers.  Reverse (adjoint) passes
// carry psi and lam and accumulate 2 Re <lam|A|psi> per parametric gate (§4.1),
// reduced per warp and per CTA in FP64 in a fixed order.
#pragma once

#include "t2_types.h"
#include "tma_device.cuh"

namespace qs {
namespace t2d {

constexpr int kT2NB = 3;  // tile buffers


__device__ __forceinline__ float2 lds64(uint32_t a) {
  float2 v;
  asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];\n" : "=f"(v.x), "=f"(v.y) : "r"(a));
  return v;
}
__device__ __forceinline__ float4 lds128(uint32_t a) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];\n" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
  return v;
}
__device__ __forceinline__ void sts64(uint32_t a, float2 v) {
  asm volatile("st.shared.v2.f32 [%0], {%1, %2};\n" ::"r"(a), "f"(v.x), "f"(v.y));
}
__device__ __forceinline__ void sts128(uint32_t a, float2 v, float2 w) {
  asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};\n" ::"r"(a), "f"(v.x), "f"(v.y), "f"(w.x), "f"(w.y));
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(__fmaf_rn(a.x, b.x, -a.y * b.y), __fmaf_rn(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 cfma(float2 a, float2 b, float2 c) {  // c + a b
  c.x = __fmaf_rn(a.x, b.x, c.x);
  c.x = __fmaf_rn(-a.y, b.y, c.x);
  c.y = __fmaf_rn(a.x, b.y, c.y);
  c.y = __fmaf_rn(a.y, b.x, c.y);
  return c;
}
__device__ __forceinline__ float re_conj_mul(float2 a, float2 b) { return __fmaf_rn(a.x, b.x, a.y * b.y); }
__device__ __forceinline__ float2 neg(float2 a) { return make_float2(-a.x, -a.y); }

// A thread's sub-cube: psi (a) and, in two-state passes, lam (b).
template <int NS>
struct Sub {
  float2 a[16];
  float2 b[16];  // unused (and eliminated) in one-state passes
};

// register-control test of element j (JC: the op has controls among the register bits)
#define T2_CTL(j) (!JC || (((uint32_t)(j)) & jc) == jc)

template <int NS, int R, bool JC>
__device__ __forceinline__ void t2_u1(Sub<NS>& s, const float2* M, uint32_t jc) {
  const float2 m00 = M[0], m01 = M[1], m10 = M[2], m11 = M[3];
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    if (j & (1 << R)) continue;
    if (!T2_CTL(j)) continue;
    const int j1 = j | (1 << R);
    {
      const float2 x0 = s.a[j], x1 = s.a[j1];
      s.a[j] = cfma(m01, x1, cmul(m00, x0));
      s.a[j1] = cfma(m11, x1, cmul(m10, x0));
    }
    if (NS == 2) {
      const float2 x0 = s.b[j], x1 = s.b[j1];
      s.b[j] = cfma(m01, x1, cmul(m00, x0));
      s.b[j1] = cfma(m11, x1, cmul(m10, x0));
    }
  }
}

template <int NS, int R, bool JC>
__device__ __forceinline__ void t2_r1(Sub<NS>& s, const float2* M, uint32_t jc) {
  const float m00 = M[0].x, m01 = M[1].x, m10 = M[2].x, m11 = M[3].x;
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    if (j & (1 << R)) continue;
    if (!T2_CTL(j)) continue;
    const int j1 = j | (1 << R);
    auto f = [&](float2(&v)[16]) {
      const float2 x0 = v[j], x1 = v[j1];
      v[j] = make_float2(__fmaf_rn(m01, x1.x, m00 * x0.x), __fmaf_rn(m01, x1.y, m00 * x0.y));
      v[j1] = make_float2(__fmaf_rn(m11, x1.x, m10 * x0.x), __fmaf_rn(m11, x1.y, m10 * x0.y));
    };
    f(s.a);
    if (NS == 2) f(s.b);
  }
}

template <int NS, int R, bool JC>
__device__ __forceinline__ void t2_rx(Sub<NS>& s, const float2* M, uint32_t jc) {
  const float c = M[0].x, sn = M[0].y;  // [[c, -i s], [-i s, c]]
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    if (j & (1 << R)) continue;
    if (!T2_CTL(j)) continue;
    const int j1 = j | (1 << R);
    auto f = [&](float2(&v)[16]) {
      const float2 x0 = v[j], x1 = v[j1];
      v[j] = make_float2(__fmaf_rn(c, x0.x, sn * x1.y), __fmaf_rn(c, x0.y, -sn * x1.x));
      v[j1] = make_float2(__fmaf_rn(c, x1.x, sn * x0.y), __fmaf_rn(c, x1.y, -sn * x0.x));
    };
    f(s.a);
    if (NS == 2) f(s.b);
  }
}

template <int NS, int R, bool JC>
__device__ __forceinline__ void t2_x(Sub<NS>& s, uint32_t jc) {
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    if (j & (1 << R)) continue;
    if (!T2_CTL(j)) continue;
    const int j1 = j | (1 << R);
    auto f = [&](float2(&v)[16]) {
      const float2 t = v[j];
      v[j] = v[j1];
      v[j1] = t;
    };
    f(s.a);
    if (NS == 2) f(s.b);
  }
}

template <int NS, int R, bool JC>
__device__ __forceinline__ void t2_z(Sub<NS>& s, uint32_t jc) {
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    if (!(j & (1 << R)) || !T2_CTL(j)) continue;
    s.a[j] = neg(s.a[j]);
    if (NS == 2) s.b[j] = neg(s.b[j]);
  }
}

template <int NS, bool JC>
__device__ __forceinline__ void t2_scale_all(Sub<NS>& s, float2 d, uint32_t jc) {
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    if (!T2_CTL(j)) continue;
    s.a[j] = cmul(d, s.a[j]);
    if (NS == 2) s.b[j] = cmul(d, s.b[j]);
  }
}

template <int NS, bool JC>
__device__ __forceinline__ void t2_neg_all(Sub<NS>& s, uint32_t jc) {
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    if (!T2_CTL(j)) continue;
    s.a[j] = neg(s.a[j]);
    if (NS == 2) s.b[j] = neg(s.b[j]);
  }
}

// diagonal with the selecting bit(s) in registers: element j takes D[idx(j)]
// with idx = bit R0 of j (+ 2 bit R1 of j when R1 >= 0); lo/hi pairs given
template <int NS, int R0, bool JC>
__device__ __forceinline__ void t2_d1(Sub<NS>& s, float2 d0, float2 d1, uint32_t jc) {
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    if (!T2_CTL(j)) continue;
    const float2 d = (j & (1 << R0)) ? d1 : d0;
    s.a[j] = cmul(d, s.a[j]);
    if (NS == 2) s.b[j] = cmul(d, s.b[j]);
  }
}
template <int NS, int R0, int R1, bool JC>
__device__ __forceinline__ void t2_d2(Sub<NS>& s, const float2* M, uint32_t jc) {
  const float2 D[4] = {M[0], M[1], M[2], M[3]};
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    if (!T2_CTL(j)) continue;
    const float2 d = D[((j >> R0) & 1) | (((j >> R1) & 1) << 1)];
    s.a[j] = cmul(d, s.a[j]);
    if (NS == 2) s.b[j] = cmul(d, s.b[j]);
  }
}

template <int NS, int R0, int R1, bool JC>
__device__ __forceinline__ void t2_u2(Sub<NS>& s, const float2* M, uint32_t jc) {
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    if (j & ((1 << R0) | (1 << R1))) continue;
    if (!T2_CTL(j)) continue;
    const int idx[4] = {j, j | (1 << R0), j | (1 << R1), j | (1 << R0) | (1 << R1)};
    auto f = [&](float2(&v)[16]) {
      const float2 x[4] = {v[idx[0]], v[idx[1]], v[idx[2]], v[idx[3]]};
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        float2 y = cmul(M[4 * r], x[0]);
        y = cfma(M[4 * r + 1], x[1], y);
        y = cfma(M[4 * r + 2], x[2], y);
        y = cfma(M[4 * r + 3], x[3], y);
        v[idx[r]] = y;
      }
    };
    f(s.a);
    if (NS == 2) f(s.b);
  }
}

// 2 Re <lam|A|psi> over the sub-cube (psi = a, lam = b)
template <int R, bool JC>
__device__ __forceinline__ float t2_g1(const Sub<2>& s, const float2* A, uint32_t jc) {
  const float2 a00 = A[0], a01 = A[1], a10 = A[2], a11 = A[3];
  float acc = 0.f;
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    if (j & (1 << R)) continue;
    if (!T2_CTL(j)) continue;
    const int j1 = j | (1 << R);
    const float2 y0 = cfma(a01, s.a[j1], cmul(a00, s.a[j]));
    const float2 y1 = cfma(a11, s.a[j1], cmul(a10, s.a[j]));
    acc += re_conj_mul(s.b[j], y0) + re_conj_mul(s.b[j1], y1);
  }
  return 2.f * acc;
}
template <int R0, int R1, bool JC>
__device__ __forceinline__ float t2_g2(const Sub<2>& s, const float2* A, uint32_t jc) {
  float acc = 0.f;
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    if (j & ((1 << R0) | (1 << R1))) continue;
    if (!T2_CTL(j)) continue;
    const int idx[4] = {j, j | (1 << R0), j | (1 << R1), j | (1 << R0) | (1 << R1)};
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      float2 y = cmul(A[4 * r], s.a[idx[0]]);
      y = cfma(A[4 * r + 1], s.a[idx[1]], y);
      y = cfma(A[4 * r + 2], s.a[idx[2]], y);
      y = cfma(A[4 * r + 3], s.a[idx[3]], y);
      acc += re_conj_mul(s.b[idx[r]], y);
    }
  }
  return 2.f * acc;
}

// Value of a constant diagonal bit: local bit (< 64) of the sub-cube base or
// global qubit (64 + q) of the tile offset.
__device__ __forceinline__ uint32_t t2_cbit(uint8_t d, uint32_t l0, uint64_t toff) {
  return d < 64 ? (l0 >> d) & 1u : (uint32_t)((toff >> (d - 64)) & 1ull);
}

template <int NS>
__device__ __forceinline__ float t2_gd(const Sub<NS>& s, const float2* A, uint32_t d0, uint32_t d1, uint32_t l0,
                                       uint64_t toff, uint32_t jc) {
  float acc = 0.f;
  if constexpr (NS == 2) {
    // bit sources: register bit (128 + r: bit r of j) or constant
    const uint32_t c0 = d0 >= 128 ? 0u : t2_cbit(d0, l0, toff);
    const uint32_t c1 = d1 == 0xFF ? 0u : d1 >= 128 ? 0u : t2_cbit(d1, l0, toff);
    const int r0 = d0 >= 128 ? (int)d0 - 128 : -1, r1 = (d1 != 0xFF && d1 >= 128) ? (int)d1 - 128 : -1;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      if ((((uint32_t)j) & jc) != jc) continue;
      const uint32_t b0 = r0 >= 0 ? ((uint32_t)j >> r0) & 1u : c0;
      const uint32_t b1 = r1 >= 0 ? ((uint32_t)j >> r1) & 1u : c1;
      acc += re_conj_mul(s.b[j], cmul(A[b0 | (b1 << 1)], s.a[j]));
    }
  }
  return 2.f * acc;
}

#define T2_R4(F) F(0) F(1) F(2) F(3)
#define T2_P12(F) F(0, 1) F(0, 2) F(0, 3) F(1, 0) F(1, 2) F(1, 3) F(2, 0) F(2, 1) F(2, 3) F(3, 0) F(3, 1) F(3, 2)

// Runs one micro-op on the thread's sub-cube; returns its gradient contribution (0 for apply ops).
template <int NS>
__device__ __forceinline__ float t2_run(Sub<NS>& s, const T2Op& op, const float2* M, uint32_t l0, uint64_t toff) {
  const uint32_t jc = op.jc;
  switch (op.code & (T2_OUTSIDE - 1)) {
#define U1(R) case t2_code(T2_U1, R, 0, false): t2_u1<NS, R, false>(s, M, jc); break; \
              case t2_code(T2_U1, R, 0, true): t2_u1<NS, R, true>(s, M, jc); break;
    T2_R4(U1)
#undef U1
#define R1(R) case t2_code(T2_R1, R, 0, false): t2_r1<NS, R, false>(s, M, jc); break; \
              case t2_code(T2_R1, R, 0, true): t2_r1<NS, R, true>(s, M, jc); break;
    T2_R4(R1)
#undef R1
#define RX(R) case t2_code(T2_RX, R, 0, false): t2_rx<NS, R, false>(s, M, jc); break; \
              case t2_code(T2_RX, R, 0, true): t2_rx<NS, R, true>(s, M, jc); break;
    T2_R4(RX)
#undef RX
#define XX(R) case t2_code(T2_X, R, 0, false): t2_x<NS, R, false>(s, jc); break; \
              case t2_code(T2_X, R, 0, true): t2_x<NS, R, true>(s, jc); break;
    T2_R4(XX)
#undef XX
#define ZZ(R) case t2_code(T2_Z, R, 0, false): t2_z<NS, R, false>(s, jc); break; \
              case t2_code(T2_Z, R, 0, true): t2_z<NS, R, true>(s, jc); break;
    T2_R4(ZZ)
#undef ZZ
    case t2_code(T2_ZC, 0, 0, false):
      if (t2_cbit(op.d0, l0, toff)) t2_neg_all<NS, false>(s, jc);
      break;
    case t2_code(T2_ZC, 0, 0, true):
      if (t2_cbit(op.d0, l0, toff)) t2_neg_all<NS, true>(s, jc);
      break;
#define D1R(R) case t2_code(T2_D1R, R, 0, false): t2_d1<NS, R, false>(s, M[0], M[1], jc); break; \
               case t2_code(T2_D1R, R, 0, true): t2_d1<NS, R, true>(s, M[0], M[1], jc); break;
    T2_R4(D1R)
#undef D1R
    case t2_code(T2_D1C, 0, 0, false): t2_scale_all<NS, false>(s, M[t2_cbit(op.d0, l0, toff)], jc); break;
    case t2_code(T2_D1C, 0, 0, true): t2_scale_all<NS, true>(s, M[t2_cbit(op.d0, l0, toff)], jc); break;
#define D2RR(R0, R1) case t2_code(T2_D2RR, R0, R1, false): t2_d2<NS, R0, R1, false>(s, M, jc); break; \
                     case t2_code(T2_D2RR, R0, R1, true): t2_d2<NS, R0, R1, true>(s, M, jc); break;
    T2_P12(D2RR)
#undef D2RR
#define D2RC(R)                                                              \
  case t2_code(T2_D2RC, R, 0, false): {                                      \
    const uint32_t g = t2_cbit(op.d1, l0, toff) << 1;                        \
    t2_d1<NS, R, false>(s, M[g], M[g + 1], jc);                              \
    break;                                                                   \
  }                                                                          \
  case t2_code(T2_D2RC, R, 0, true): {                                       \
    const uint32_t g = t2_cbit(op.d1, l0, toff) << 1;                        \
    t2_d1<NS, R, true>(s, M[g], M[g + 1], jc);                               \
    break;                                                                   \
  }
    T2_R4(D2RC)
#undef D2RC
#define D2CR(R)                                                              \
  case t2_code(T2_D2CR, 0, R, false): {                                      \
    const uint32_t g = t2_cbit(op.d0, l0, toff);                             \
    t2_d1<NS, R, false>(s, M[g], M[g + 2], jc);                              \
    break;                                                                   \
  }                                                                          \
  case t2_code(T2_D2CR, 0, R, true): {                                       \
    const uint32_t g = t2_cbit(op.d0, l0, toff);                             \
    t2_d1<NS, R, true>(s, M[g], M[g + 2], jc);                               \
    break;                                                                   \
  }
    T2_R4(D2CR)
#undef D2CR
    case t2_code(T2_D2CC, 0, 0, false):
      t2_scale_all<NS, false>(s, M[t2_cbit(op.d0, l0, toff) | (t2_cbit(op.d1, l0, toff) << 1)], jc);
      break;
    case t2_code(T2_D2CC, 0, 0, true):
      t2_scale_all<NS, true>(s, M[t2_cbit(op.d0, l0, toff) | (t2_cbit(op.d1, l0, toff) << 1)], jc);
      break;
#define U2(R0, R1) case t2_code(T2_U2, R0, R1, false): t2_u2<NS, R0, R1, false>(s, M, jc); break; \
                   case t2_code(T2_U2, R0, R1, true): t2_u2<NS, R0, R1, true>(s, M, jc); break;
    T2_P12(U2)
#undef U2
    default:
      break;
  }
  if constexpr (NS == 2) {
    switch (op.code & (T2_OUTSIDE - 1)) {
#define G1(R) case t2_code(T2_G1, R, 0, false): return t2_g1<R, false>(s, M, jc); \
              case t2_code(T2_G1, R, 0, true): return t2_g1<R, true>(s, M, jc);
      T2_R4(G1)
#undef G1
#define G2(R0, R1) case t2_code(T2_G2, R0, R1, false): return t2_g2<R0, R1, false>(s, M, jc); \
                   case t2_code(T2_G2, R0, R1, true): return t2_g2<R0, R1, true>(s, M, jc);
      T2_P12(G2)
#undef G2
      case t2_code(T2_GD, 0, 0, false):
      case t2_code(T2_GD, 0, 0, true):
        return t2_gd<NS>(s, M, op.d0, op.d1, l0, toff, jc);
      default:
        break;
    }
  }
  return 0.f;
}

__device__ __forceinline__ bool t2_is_grad(uint16_t code) {
  const int k = code & 31;
  return k == T2_G1 || k == T2_G2 || k == T2_GD;
}

// What a pass program sees of the current tile: the tile buffer, the tile's
// offset, the shared stages, and the phase loop.
template <int NS>
struct T2Ctx {
  uint32_t tb;          // shared address of the tile buffer (psi; lam at + tile_bytes)
  uint32_t tile_bytes;
  uint32_t nsub;        // sub-cubes of a tile
  uint64_t toff;        // global offset of the tile
  int T, tid, lane, warp, W;
  const T2Phase* ph;    // shared phase table
  const T2Op* ops;      // shared op table
  const float2* coef;   // shared coefficient stage
  double* acc;          // shared accumulators [slot][warp]

  // Runs body(s, l0) on each of this thread's sub-cubes of phase p (s: the 16
  // amplitudes, l0: the sub-cube's local base), then waits for the compute
  // warps.  PAIR: 1 / 0 when the phase's pair form is known, -1 to read it.
  template <int PAIR, class F>
  __device__ __forceinline__ void phase(int p, const F& body) const {
    const T2Phase& PH = ph[p];
    const uint32_t sp0 = PH.sp[0], sp1 = PH.sp[1], sp2 = PH.sp[2], sp3 = PH.sp[3];
    const bool pair = PAIR < 0 ? (bool)PH.pair : PAIR == 1;
    for (uint32_t u = (uint32_t)tid; u < nsub; u += (uint32_t)T) {
      const uint32_t l0 = PH.l0tab[u & 15u] | PH.l0tab[16 + ((u >> 4) & 31u)];
      const uint32_t p0 = l0 ^ (((l0 >> 4) & 7u) << 1);
#define T2_POS(j) \
  (p0 ^ (((j) & 1) ? sp0 : 0u) ^ (((j) & 2) ? sp1 : 0u) ^ (((j) & 4) ? sp2 : 0u) ^ (((j) & 8) ? sp3 : 0u))
      Sub<NS> s;
      if (pair) {
#pragma unroll
        for (int j = 0; j < 16; j += 2) {
          const uint32_t ad = tb + 8u * T2_POS(j);
          const float4 v = lds128(ad);
          s.a[j] = make_float2(v.x, v.y);
          s.a[j + 1] = make_float2(v.z, v.w);
          if (NS == 2) {
            const float4 w = lds128(ad + tile_bytes);
            s.b[j] = make_float2(w.x, w.y);
            s.b[j + 1] = make_float2(w.z, w.w);
          }
        }
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const uint32_t ad = tb + 8u * T2_POS(j);
          s.a[j] = lds64(ad);
          if (NS == 2) s.b[j] = lds64(ad + tile_bytes);
        }
      }
      body(s, l0);
      if (pair) {
#pragma unroll
        for (int j = 0; j < 16; j += 2) {
          const uint32_t ad = tb + 8u * T2_POS(j);
          sts128(ad, s.a[j], s.a[j + 1]);
          if (NS == 2) sts128(ad + tile_bytes, s.b[j], s.b[j + 1]);
        }
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const uint32_t ad = tb + 8u * T2_POS(j);
          sts64(ad, s.a[j]);
          if (NS == 2) sts64(ad + tile_bytes, s.b[j]);
        }
      }
#undef T2_POS
    }
    bar_compute(T);
  }

  // A gradient op's contribution: summed over the warp, added by lane 0 to
  // the slot's column of this warp (every thread of the warp takes part).
  __device__ __forceinline__ void grad(float g, int slot) const {
#pragma unroll
    for (int sh = 16; sh > 0; sh >>= 1) g += __shfl_xor_sync(0xffffffffu, g, sh);
    if (lane == 0) acc[slot * W + warp] += (double)g;
  }
};

// The pass program of the kernels compiled with the library: each phase runs
// its ops from the shared op table through the dispatch of t2_run.
template <int NS>
struct T2InterpPhase {
  const T2Ctx<NS>& c;
  int ob, oe;
  __device__ __forceinline__ void operator()(Sub<NS>& s, uint32_t l0) const {
    for (int o = ob; o < oe; ++o) {
      const T2Op& op = c.ops[o];
      const uint32_t code = op.code;
      const bool ok = !(code & T2_OUTSIDE) || (((l0 & op.lc) == op.lc) && ((c.toff & op.gc) == op.gc));
      if (NS == 2 && t2_is_grad(code)) {
        c.grad(ok ? t2_run<NS>(s, op, c.coef + op.cs, l0, c.toff) : 0.f, op.slot);
        continue;
      }
      if (!ok) continue;
      t2_run<NS>(s, op, c.coef + op.cs, l0, c.toff);
    }
  }
};
struct T2Interp {
  template <int NS>
  __device__ __forceinline__ void operator()(const T2Ctx<NS>& c, int n_ph) const {
    for (int p = 0; p < n_ph; ++p)
      c.template phase<-1>(p, T2InterpPhase<NS>{c, c.ph[p].op_begin, c.ph[p].op_end});
  }
};

// One pass over the tiles of this CTA (blockIdx.x, + gridDim.x, ...): the
// producer warp streams tiles in and out, the compute warps run `prog` on each.
template <int NS, class Prog>
__device__ __forceinline__ void tile2_body(const T2Args& args, const TmapBlob* tmap, const Prog& prog) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(8) uint64_t s_full[kT2NB], s_done[kT2NB];
  __shared__ int s_bad;
  const int tid = threadIdx.x, NT = blockDim.x, T = NT - 32, lane = tid & 31, warp = tid >> 5;
  const bool producer = tid >= T;
  const int W = T / 32;

  // ---- shared memory: tiles (1024-aligned) | pass | phases | ops | coefficients | accumulators | tables
  const uint32_t base = tma_sh(smem);
  const uint32_t tile0 = (base + 1023u) & ~1023u;
  unsigned char* gp = smem + (tile0 - base);
  const T2Pass* gpass = args.pass;
  const int m = gpass->m;
  const uint32_t tile_n = 1u << m, tile_bytes = tile_n * 8u, buf_bytes = (uint32_t)NS * tile_bytes;
  unsigned char* p = gp + (size_t)kT2NB * buf_bytes;
  T2Pass* s_pass = reinterpret_cast<T2Pass*>(p);
  p += (sizeof(T2Pass) + 15) & ~(size_t)15;
  {
    const int* src = reinterpret_cast<const int*>(gpass);
    int* dst = reinterpret_cast<int*>(s_pass);
    for (int i = tid; i < (int)(sizeof(T2Pass) / 4); i += NT) dst[i] = src[i];
  }
  if (tid == 0) {
    s_bad = 0;
    for (int b = 0; b < kT2NB; ++b) {
      mbar_init(tma_sh(&s_full[b]), 1);
      mbar_init(tma_sh(&s_done[b]), (uint32_t)T);
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  const T2Pass& P = *s_pass;
  const int n_ph = P.n_phases, n_ops = P.n_ops;
  T2Phase* s_ph = reinterpret_cast<T2Phase*>(p);
  p += ((size_t)n_ph * sizeof(T2Phase) + 15) & ~(size_t)15;
  T2Op* s_ops = reinterpret_cast<T2Op*>(p);
  p += ((size_t)n_ops * sizeof(T2Op) + 15) & ~(size_t)15;
  float2* s_coef = reinterpret_cast<float2*>(p);
  p += ((size_t)P.n_coef * 8 + 15) & ~(size_t)15;
  double* s_acc = reinterpret_cast<double*>(p);
  p += (size_t)P.n_slots * W * 8;
  uint64_t* s_dep = reinterpret_cast<uint64_t*>(p);  // [5][64]: tile index bits -> complement qubits
  {
    const int* src = reinterpret_cast<const int*>(args.phases);
    int* dst = reinterpret_cast<int*>(s_ph);
    for (int i = tid; i < n_ph * (int)(sizeof(T2Phase) / 4); i += NT) dst[i] = src[i];
    const int4* so = reinterpret_cast<const int4*>(args.ops);
    int4* dop = reinterpret_cast<int4*>(s_ops);
    for (int i = tid; i < n_ops * (int)(sizeof(T2Op) / 16); i += NT) dop[i] = so[i];
  }
  for (int i = tid; i < P.n_slots * W; i += NT) s_acc[i] = 0.0;
  for (int i = tid; i < 5 * 64; i += NT) {
    const int tb = i >> 6, v = i & 63;
    uint64_t o = 0;
    for (int k = 0; k < 6; ++k)
      if (((v >> k) & 1) && 6 * tb + k < P.ncomp) o |= 1ull << P.comp[6 * tb + k];
    s_dep[i] = o;
  }
  __syncthreads();
  // coefficient stage: each op's block of the call's table
  for (int o = warp; o < n_ops; o += NT / 32) {
    const T2Op& op = s_ops[o];
    for (uint32_t k = lane; k < op.ncoef; k += 32) s_coef[op.cs + k] = args.coef[op.coef + k];
  }
  __syncthreads();

  const uint64_t n_tiles = 1ull << (args.n - m);
  auto toff_of = [&](uint64_t t) {
    return s_dep[t & 63] | s_dep[64 + ((t >> 6) & 63)] | s_dep[128 + ((t >> 12) & 63)] |
           s_dep[192 + ((t >> 18) & 63)] | s_dep[256 + ((t >> 24) & 63)];
  };
  auto l2g = [&](uint32_t l) {  // tile-local index (bits >= 4) -> global offset
    return (uint64_t)(l & 15u) | P.hiA[(l >> 4) & 63] | P.hiB[(l >> 10) & 127];
  };
  auto tsh = [&](int b) { return tile0 + (uint32_t)b * buf_bytes; };
  const uint32_t flags = P.flags;

  if (producer) {
    // ------------------------------------------------------------ producer warp
    const bool gen = (flags & (PF_GEN_PLUS | PF_GEN_ZERO)) != 0;
    const bool st_psi = (flags & PF_STORE_PSI) != 0, st_lam = NS == 2 && (flags & PF_STORE_LAM);
    const uint32_t nb = 1u << (m - P.mlb), bb = (1u << P.mlb) * 8u;
    auto load = [&](uint64_t t, int b) {
      if (t >= n_tiles) return;
      const uint32_t fb = tma_sh(&s_full[b]);
      if (gen) {
        if (lane == 0) mbar_arrive(fb);
        return;
      }
      if (lane == 0) mbar_arrive_expect(fb, buf_bytes);
      __syncwarp();
      const uint64_t toff = toff_of(t);
      for (uint32_t j = lane; j < nb; j += 32) {
        int x[5];
        tile_coords(P.ma, P.mw, toff + l2g(j << P.mlb), x);
        tma_load5(tsh(b) + j * bb, &tmap[0], x, fb);
        if (NS == 2) tma_load5(tsh(b) + tile_bytes + j * bb, &tmap[1], x, fb);
      }
    };
    auto store = [&](uint64_t t, int b) {
      const uint64_t toff = toff_of(t);
      for (uint32_t j = lane; j < nb; j += 32) {
        int x[5];
        tile_coords(P.ma, P.mw, toff + l2g(j << P.mlb), x);
        if (st_psi) tma_store5(&tmap[0], x, tsh(b) + j * bb);
        if (st_lam) tma_store5(&tmap[1], x, tsh(b) + tile_bytes + j * bb);
      }
      bulk_commit();
      bulk_wait_read0();  // the buffer may be refilled once the stores have read it
    };
    const bool do_store = st_psi || st_lam;
    uint64_t tile = blockIdx.x;
    load(tile, 0);
    load(tile + gridDim.x, 1);
    int i = 0;
    for (; tile < n_tiles; tile += gridDim.x, ++i) {
      const int b2 = (i + 2) % kT2NB;  // the previous tile's buffer, refilled with the tile two ahead
      if (i >= 1) {
        if (!mbar_wait(tma_sh(&s_done[b2]), (uint32_t)(((i - 1) / kT2NB) & 1))) s_bad = 1;
        if (do_store) store(tile - gridDim.x, b2);
      }
      load(tile + 2ull * gridDim.x, b2);
    }
    if (i >= 1) {
      const int bl = (i - 1) % kT2NB;
      if (!mbar_wait(tma_sh(&s_done[bl]), (uint32_t)(((i - 1) / kT2NB) & 1))) s_bad = 1;
      if (do_store) store(tile - gridDim.x, bl);
    }
    bulk_wait0();
  } else {
    // ------------------------------------------------------------ compute warps
    T2Ctx<NS> c;
    c.tile_bytes = tile_bytes;
    c.nsub = tile_n >> 4;
    c.T = T;
    c.tid = tid;
    c.lane = lane;
    c.warp = warp;
    c.W = W;
    c.ph = s_ph;
    c.ops = s_ops;
    c.coef = s_coef;
    c.acc = s_acc;
    int i = 0;
    for (uint64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++i) {
      const int cur = i % kT2NB;
      if (!mbar_wait(tma_sh(&s_full[cur]), (uint32_t)((i / kT2NB) & 1))) s_bad = 1;
      c.tb = tsh(cur);
      c.toff = toff_of(tile);
      if (flags & (PF_GEN_PLUS | PF_GEN_ZERO)) {  // the tile starts as |+>^n or |0...0>
        const float v = (flags & PF_GEN_PLUS) ? args.plus_amp : 0.f;
        for (uint32_t e = tid; e < tile_n; e += T) sts64(c.tb + 8u * e, make_float2(v, 0.f));
        if ((flags & PF_GEN_ZERO) && c.toff == 0 && tid == 0) sts64(c.tb, make_float2(1.f, 0.f));
        bar_compute(T);
      }
      prog(c, n_ph);
      fence_async_smem();              // this thread's shared writes, before the bulk stores read them
      mbar_arrive(tma_sh(&s_done[cur]));  // the producer may store and refill this buffer
    }
  }
  __syncthreads();

  // ---- per-CTA sums of the accumulators in a fixed order; a wait that ran out poisons them
  for (int sl = tid; sl < P.n_slots; sl += NT) {
    double v = 0.0;
    for (int w = 0; w < W; ++w) v += s_acc[sl * W + w];
    const size_t row = (size_t)(P.slot_base + sl) * args.stride;
    args.partials[row + blockIdx.x] = s_bad ? __longlong_as_double(0x7ff8000000000000ll) : v;
    if (blockIdx.x == 0)
      for (int col = gridDim.x; col < args.cols; ++col) args.partials[row + col] = 0.0;
  }
}

}  // namespace t2d
}  // namespace qs
