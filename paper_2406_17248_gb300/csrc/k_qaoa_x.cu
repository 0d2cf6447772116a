// Complex64 QAOA tile passes with separate forward and reverse tile shapes
// (§5.2 ansatz, §6.2 QuPack QAOA simulator): RX(beta) on the tile bits, the
// cost phase exp(-i gs gamma C(x)), the energy and the adjoint-gradient terms
// dE/dbeta = sum_q Im <lam|X_q|psi> and dE/dgamma = 2 gs Im <lam|C|psi>.
//
// Two kernels share one structure:
//   qx_kernel<false>: psi alone (8-byte amplitudes), the forward sweep;
//   qx_kernel<true>:  psi and lam interleaved per amplitude as
//                     (psi.re, lam.re, psi.im, lam.im), so one packed f32x2
//                     FMA updates both states; the turnaround and reverse sweep.
// A CTA holds 2^(m-4) compute threads and one producer warp, and loops over
// tiles through a ring of three tile buffers.  The producer moves whole rows
// (runs of 2^c contiguous amplitudes) between HBM and shared memory with bulk
// asynchronous copies completing on mbarriers, so no compute warp ever issues
// a global load or store and HBM back-pressure never stalls the arithmetic.
// Each phase gives every compute thread the 16 amplitudes of one sub-cube, runs
// straight-line code for its steps (one compiled body per step shape), and
// writes back to shared memory.  Tiles are plain copies of the HBM rows (bulk
// copies do not swizzle); where a phase's register bits include bank-column
// bits, a lane XOR-relabels its register index so the lanes of a quarter warp
// still hit distinct banks.  C(x) is assembled per amplitude from a per-pass
// table of in-tile edge counts and per-tile linear terms (computed by warp 0
// two tiles ahead), so no cut-value array is read.
#include <algorithm>
#include <cmath>
#include <map>
#include <type_traits>

#include "qaoa_pass.h"
#include "qaoa_x.h"
#include "tma.h"

namespace qs {

namespace {

constexpr int kXN = 16;  // amplitudes per thread per phase
constexpr int kXNB = 3;  // tile buffers: the current tile, the next one landing, the one after issued

__device__ __forceinline__ uint32_t xsh(const void* p) { return tma_sh(p); }
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
__device__ __forceinline__ uint32_t ldsu8(uint32_t a) {
  uint32_t v;
  asm volatile("ld.shared.u8 %0, [%1];\n" : "=r"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ void sts64(uint32_t a, float x, float y) {
  asm volatile("st.shared.v2.f32 [%0], {%1, %2};\n" ::"r"(a), "f"(x), "f"(y));
}
__device__ __forceinline__ void sts128(uint32_t a, float x, float y, float z, float w) {
  asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};\n" ::"r"(a), "f"(x), "f"(y), "f"(z), "f"(w));
}

struct XArgs {
  CUtensorMap tm[2];  // tile copies: [0] load, [1] store
  const XPass* pass;
  float2* psi;
  float4* il;
  const float2* coef;
  const uint8_t* fs;
  double* partials;
  float plus_amp;
  int stride, n, n_edges;
};

__device__ __forceinline__ uint64_t x_l2g(const XPass& P, uint32_t l) {
  return (uint64_t)(l & ((1u << P.c) - 1u)) | P.hiA[(l >> P.c) & 63] | P.hiB[(l >> (P.c + 6)) & 63];
}

// ---------------------------------------------------------------- one-state steps
// scaled mixer [[1, -it], [-it, 1]] on register bit RB: one FMA per real output
template <int RB>
__device__ __forceinline__ void xrx1(float2 (&a)[kXN], float t) {
#pragma unroll
  for (int j = 0; j < kXN; ++j) {
    if (j & (1 << RB)) continue;
    const int j1 = j | (1 << RB);
    const float2 x0 = a[j], x1 = a[j1];
    a[j].x = __fmaf_rn(t, x1.y, x0.x);
    a[j].y = __fmaf_rn(-t, x1.x, x0.y);
    a[j1].x = __fmaf_rn(t, x0.y, x1.x);
    a[j1].y = __fmaf_rn(-t, x0.x, x1.y);
  }
}
// ---------------------------------------------------------------- two-state steps
// RE = (psi.re, lam.re), IM = (psi.im, lam.im): the scaled mixer on both states
// at once, one packed FMA per pair of real outputs
template <int RB, int N>
__device__ __forceinline__ void xrx2(float2 (&RE)[N], float2 (&IM)[N], float2 t2, float2 mt2) {
#pragma unroll
  for (int j = 0; j < N; ++j) {
    if (j & (1 << RB)) continue;
    const int j1 = j | (1 << RB);
    const float2 r0 = RE[j], i0 = IM[j], r1 = RE[j1], i1 = IM[j1];
    RE[j] = __ffma2_rn(t2, i1, r0);
    IM[j] = __ffma2_rn(mt2, r1, i0);
    RE[j1] = __ffma2_rn(t2, i0, r1);
    IM[j1] = __ffma2_rn(mt2, r0, i1);
  }
}
// Im <lam|X_RB|psi> over the sub-cube (four independent partial sums)
template <int RB, int N>
__device__ __forceinline__ float xgx2(const float2 (&RE)[N], const float2 (&IM)[N]) {
  float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
  for (int j = 0; j < N; ++j) {
    if (j & (1 << RB)) continue;
    const int j1 = j | (1 << RB);
    s0 = __fmaf_rn(RE[j].y, IM[j1].x, s0);
    s1 = __fmaf_rn(-IM[j].y, RE[j1].x, s1);
    s2 = __fmaf_rn(RE[j1].y, IM[j].x, s2);
    s3 = __fmaf_rn(-IM[j1].y, RE[j].x, s3);
  }
  return (s0 + s1) + (s2 + s3);
}
__device__ __forceinline__ void xacc(float& hi, float& lo, float x) {  // compensated (TwoSum)
  const float s = hi + x;
  const float bb = s - hi;
  lo += (hi - (s - bb)) + (x - bb);
  hi = s;
}

// Per-phase context of one thread (all values uniform across the phase code).
struct XPh {
  uint32_t tb;                  // shared address of the tile buffer
  uint32_t pb;                  // byte offset of the sub-cube base element in the tile
  uint32_t sp0, sp1, sp2, sp3;  // byte offsets of the register bits (XOR)
  uint32_t l0, lb0, lb1, lb2, lb3;  // l0: local index of register index 0 (relabel bits included)
  int cutb, w0, w1, w2, w3;     // cut value = fs[l0 | L(j)] + cutb + W(j)
  uint32_t fs, lut;             // shared addresses of the edge-count table and the LUT
  int ne;
  float2 cs1, cs3;              // steps 1 and 3: (scaled-mixer t, weight 1 / |scale|^2 of the step's sums)
  float pw;                     // the |+> amplitude in a generating phase, else the diagonal sum's weight
};

// Register-index sums: L(j) = OR of the local bits, S(j) = XOR of the shared
// byte offsets, W(j) = sum of the linear cut weights, G(j) = sum of the HBM byte
// offsets of the register bits set in j.
#define XL(j) ((((j) & 1) ? h.lb0 : 0u) | (((j) & 2) ? h.lb1 : 0u) | (((j) & 4) ? h.lb2 : 0u) | (((j) & 8) ? h.lb3 : 0u))
#define XS(j) ((((j) & 1) ? h.sp0 : 0u) ^ (((j) & 2) ? h.sp1 : 0u) ^ (((j) & 4) ? h.sp2 : 0u) ^ (((j) & 8) ? h.sp3 : 0u))
#define XW(j) ((((j) & 1) ? h.w0 : 0) + (((j) & 2) ? h.w1 : 0) + (((j) & 4) ? h.w2 : 0) + (((j) & 8) ? h.w3 : 0))
// cut value of element j, kept inside the LUT (0..|E|) whatever the tables hold
#define XCUT(j) ((int)min((unsigned)((int)ldsu8(h.fs + (h.l0 ^ XL(j))) + h.cutb + XW(j)), (unsigned)h.ne))


// RX on the first K register bits
template <int K>
__device__ __forceinline__ void xrx1_k(float2 (&a)[kXN], float2 ts) {
  if (K > 0) xrx1<0>(a, ts.x);
  if (K > 1) xrx1<1>(a, ts.x);
  if (K > 2) xrx1<2>(a, ts.x);
  if (K > 3) xrx1<3>(a, ts.x);
}
// Im <lam|X_q|psi> of each of the first K register bits, each taken before its
// rotation, then the rotation; ts = (t, weight of the step's start).  Every
// scaled rotation multiplies the data's |scale|^2 by 1 + t^2 (= 1/c^2 or 1/s^2
// in the two forms), so term r carries the weight times kappa^r,
// kappa = 1 / (1 + t^2)
template <int K, int N>
__device__ __forceinline__ float xrx2_k(float2 (&RE)[N], float2 (&IM)[N], float2 ts) {
  const float2 t2 = make_float2(ts.x, ts.x), mt2 = make_float2(-ts.x, -ts.x);
  const float kap = __frcp_rn(__fmaf_rn(ts.x, ts.x, 1.f));
  float g = 0.f, sc = ts.y;  // the step's weight at its start
  if (K > 0) {
    g = sc * xgx2<0>(RE, IM);
    xrx2<0>(RE, IM, t2, mt2);
    sc *= kap;
  }
  if (K > 1) {
    g = __fmaf_rn(sc, xgx2<1>(RE, IM), g);
    xrx2<1>(RE, IM, t2, mt2);
    sc *= kap;
  }
  if (K > 2) {
    g = __fmaf_rn(sc, xgx2<2>(RE, IM), g);
    xrx2<2>(RE, IM, t2, mt2);
    sc *= kap;
  }
  if (K > 3) {
    g = __fmaf_rn(sc, xgx2<3>(RE, IM), g);
    xrx2<3>(RE, IM, t2, mt2);
  }
  return g;
}

// One phase of the one-state kernel: RX on K1 bits, diagonal DG, RX on K3 bits.
template <int K1, int DG, int K3, bool GEN>
__device__ __forceinline__ void xphase1(const XPh& h, float (&acc)[3]) {
  float2 a[kXN];
  if (GEN) {
#pragma unroll
    for (int j = 0; j < kXN; ++j) a[j] = make_float2(h.pw, 0.f);
  } else {
#pragma unroll
    for (int j = 0; j < kXN; ++j) a[j] = lds64(h.tb + (h.pb ^ XS(j)));
  }
  xrx1_k<K1>(a, h.cs1);
  if (DG == XD_COST) {
#pragma unroll
    for (int j = 0; j < kXN; ++j) {
      const float2 d = lds64(h.lut + 8u * XCUT(j));
      const float2 x = a[j];
      a[j].x = __fmaf_rn(d.x, x.x, -d.y * x.y);
      a[j].y = __fmaf_rn(d.x, x.y, d.y * x.x);
    }
  } else if (DG == XD_ENERGY) {
    float e0 = 0.f, e1 = 0.f;
#pragma unroll
    for (int j = 0; j < kXN; ++j) {
      const float C = (float)(h.ne - 2 * XCUT(j));
      const float pr = __fmaf_rn(a[j].x, a[j].x, a[j].y * a[j].y);
      if (j & 1) e1 = __fmaf_rn(C, pr, e1);
      else e0 = __fmaf_rn(C, pr, e0);
    }
    acc[1] = __fmaf_rn(h.pw, e0 + e1, acc[1]);
  }
  xrx1_k<K3>(a, h.cs3);
#pragma unroll
  for (int j = 0; j < kXN; ++j) sts64(h.tb + (h.pb ^ XS(j)), a[j].x, a[j].y);
}

// One phase of the two-state kernel: the mixer steps take Im <lam|X_q|psi>
// into acc[0] (step 1) and acc[2] (step 3) before rotating both states.
template <int K1, int DG, int K3>
__device__ __forceinline__ void xphase2(const XPh& h, float (&acc)[3]) {
  constexpr int N = 1 << qx_reg_bits(true);
  float2 RE[N], IM[N];
#pragma unroll
  for (int j = 0; j < N; ++j) {
    const float4 e = lds128(h.tb + (h.pb ^ XS(j)));
    RE[j] = make_float2(e.x, e.y);
    IM[j] = make_float2(e.z, e.w);
  }
  if (K1 > 0) acc[0] += xrx2_k<K1>(RE, IM, h.cs1);
  if (DG == XD_COST_GRAD) {
    float g0 = 0.f, g1 = 0.f;
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const int k = XCUT(j);
      const float C = (float)(h.ne - 2 * k);
      const float im = __fmaf_rn(RE[j].y, IM[j].x, -IM[j].y * RE[j].x);  // Im(conj(lam) psi)
      if (j & 1) g1 = __fmaf_rn(C, im, g1);
      else g0 = __fmaf_rn(C, im, g0);
      const float2 d = lds64(h.lut + 8u * (uint32_t)k);
      const float2 dr = make_float2(d.x, d.x), di = make_float2(d.y, d.y), mdi = make_float2(-d.y, -d.y);
      const float2 r = RE[j], i = IM[j];
      RE[j] = __ffma2_rn(dr, r, __fmul2_rn(mdi, i));
      IM[j] = __ffma2_rn(dr, i, __fmul2_rn(di, r));
    }
    acc[1] = __fmaf_rn(h.pw, g0 + g1, acc[1]);
  } else if (DG == XD_ENERGY) {
    float e0 = 0.f, e1 = 0.f;
#pragma unroll
    for (int j = 0; j < N; ++j) {
      const float C = (float)(h.ne - 2 * XCUT(j));
      const float pr = __fmaf_rn(RE[j].x, RE[j].x, IM[j].x * IM[j].x);
      if (j & 1) e1 = __fmaf_rn(C, pr, e1);
      else e0 = __fmaf_rn(C, pr, e0);
      RE[j].y = C * RE[j].x;  // lam = C psi
      IM[j].y = C * IM[j].x;
    }
    acc[1] = __fmaf_rn(h.pw, e0 + e1, acc[1]);
  }
  if (K3 > 0) acc[2] += xrx2_k<K3>(RE, IM, h.cs3);
#pragma unroll
  for (int j = 0; j < N; ++j) sts128(h.tb + (h.pb ^ XS(j)), RE[j].x, RE[j].y, IM[j].x, IM[j].y);
}

// Phase code: K1 + 5 DIAG + 25 K3 (+ 125 for the |+> start of the forward sweep).
__host__ __device__ constexpr int xcode(int k1, int dg, int k3) { return k1 + 5 * dg + 25 * k3; }

__device__ __forceinline__ bool xdispatch1(int code, const XPh& h, float (&acc)[3]) {
  switch (code) {
#define C1(K1, DG, K3) \
  case xcode(K1, DG, K3): xphase1<K1, DG, K3, false>(h, acc); return true;
    C1(1, 0, 0) C1(2, 0, 0) C1(3, 0, 0) C1(4, 0, 0)
    C1(0, 0, 1) C1(0, 0, 2) C1(0, 0, 3) C1(0, 0, 4)
    C1(0, XD_COST, 4) C1(1, XD_COST, 4) C1(2, XD_COST, 4) C1(3, XD_COST, 4) C1(4, XD_COST, 4)
    C1(0, XD_ENERGY, 0) C1(1, XD_ENERGY, 0) C1(2, XD_ENERGY, 0) C1(3, XD_ENERGY, 0) C1(4, XD_ENERGY, 0)
#undef C1
    case 125 + xcode(0, XD_COST, 4): xphase1<0, XD_COST, 4, true>(h, acc); return true;
    default: return false;
  }
}

__device__ __forceinline__ bool xdispatch2(int code, const XPh& h, float (&acc)[3]) {
  // bodies for 3 register bits (the planner emits these step shapes only)
  static_assert(qx_reg_bits(true) == 3, "two-state phase table is written for 3 register bits");
  switch (code) {
#define C2(K1, DG, K3) \
  case xcode(K1, DG, K3): xphase2<K1, DG, K3>(h, acc); return true;
    C2(1, 0, 0) C2(2, 0, 0) C2(3, 0, 0)
    C2(0, 0, 1) C2(0, 0, 2) C2(0, 0, 3)
    C2(0, XD_COST_GRAD, 3) C2(1, XD_COST_GRAD, 3) C2(2, XD_COST_GRAD, 3) C2(3, XD_COST_GRAD, 3)
    C2(0, XD_COST_GRAD, 0) C2(1, XD_COST_GRAD, 0) C2(2, XD_COST_GRAD, 0) C2(3, XD_COST_GRAD, 0)
    C2(0, XD_ENERGY, 3) C2(1, XD_ENERGY, 3) C2(2, XD_ENERGY, 3) C2(3, XD_ENERGY, 3)
#undef C2
    default: return false;
  }
}



// Block: T = 2^(m-R) compute threads plus one producer warp.  The producer
// moves every tile between HBM and shared memory (16-byte cp.async copies in,
// 16-byte stores out) through a ring of three tile buffers, so the compute warps
// never stall on HBM back-pressure; mbarriers hand buffers over: full[b] when a
// tile's copies have landed, done[b] when the compute warps have finished it.
template <bool TWO>
__global__ void __launch_bounds__(544, 1) qx_kernel(const __grid_constant__ XArgs args) {
  constexpr uint32_t ES = TWO ? 16 : 8;  // bytes per shared-memory element
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ XPass P;
  __shared__ uint64_t s_dep[5][64];
  __shared__ int s_lin[kXNB][16];  // per tile buffer: w_i of local bit i (i < 13), g at [15]
  __shared__ double s_red[17];
  __shared__ float s_w[4 * kXMaxPhases];  // per phase: w1, w3, wd (phase weights of the scaled mixer)
  __shared__ int s_bad;
  __shared__ __align__(8) uint64_t s_full[kXNB], s_done[kXNB];
  const int tid = threadIdx.x, NT = blockDim.x, T = NT - 32, lane = tid & 31, warp = tid >> 5;
  const bool producer = tid >= T;
  {
    const int* src = reinterpret_cast<const int*>(args.pass);
    int* dst = reinterpret_cast<int*>(&P);
    for (int i = tid; i < (int)(sizeof(XPass) / 4); i += NT) dst[i] = src[i];
    if (tid == 0) {
      s_bad = 0;
      for (int b = 0; b < kXNB; ++b) {
        mbar_init(xsh(&s_full[b]), 1);
        mbar_init(xsh(&s_done[b]), (uint32_t)T);
      }
    }
  }
  __syncthreads();
  const int m = P.m, n_ph = P.n_phases;
  const uint32_t flags = P.flags, tile_n = 1u << m, tile_bytes = tile_n * ES;
  const int E1 = args.n_edges + 1;
  bool has_diag = false;
  for (int i = 0; i < n_ph; ++i) has_diag |= P.ph[i].diag != XD_NONE;

  // ---- shared memory: LUT | in-tile edge counts | phase bases | tile buffers
  float2* s_lut = reinterpret_cast<float2*>(smem);
  size_t off = ((size_t)E1 * 8 + 127) & ~(size_t)127;
  uint8_t* s_fs = smem + off;
  off += ((size_t)tile_n + 127) & ~(size_t)127;
  uint32_t* s_pl = reinterpret_cast<uint32_t*>(smem + off);
  off += (size_t)n_ph * T * 4;
  // tiled tensor copies need 128-byte aligned shared addresses; the dynamic
  // shared block follows the static variables and is only 16-byte aligned
  const uint32_t tile0 = (xsh(smem) + (uint32_t)off + 127u) & ~127u;
  // shared address of tile buffer b (arithmetic: an indexed array would live in local memory)
  auto tsh = [&](int b) { return tile0 + (uint32_t)b * tile_bytes; };

  if (P.cd >= 0)
    for (int i = tid; i < E1; i += NT) s_lut[i] = args.coef[P.cd + i];
  if (has_diag && P.fs_off >= 0) {
    const uint4* src = reinterpret_cast<const uint4*>(args.fs + P.fs_off);
    for (uint32_t i = tid; i < (tile_n >> 4); i += NT) reinterpret_cast<uint4*>(s_fs)[i] = src[i];
  }
  for (int i = tid; i < 2 * n_ph; i += NT) {
    const float2 w = args.coef[P.cw + i];
    s_w[2 * i] = w.x;
    s_w[2 * i + 1] = w.y;
  }
  const float2 cs1 = P.c1 >= 0 ? args.coef[P.c1] : make_float2(1.f, 0.f);
  const float2 cs3 = P.c3 >= 0 ? args.coef[P.c3] : make_float2(1.f, 0.f);
  // phase bases of each compute thread: (local index << 8) | relabel mask.
  // Tiles are unswizzled copies of the HBM runs, so an element's bank column is
  // its low local bits; where some of those are register bits, lanes kq..kq+kn-1
  // XOR the thread's register index with a mask kappa: register j then holds
  // element l0 | L(j ^ kappa) = (l0 | L(kappa)) ^ L(j).  The RX butterflies and
  // the gradient sums are symmetric in the two elements of a pair, so they are
  // unchanged; addresses, cut indices and weights take the relabel into account.
  for (int i = tid; i < n_ph * T; i += NT) {
    const int ph = i / T, t = i % T;
    const XPhase& PH = P.ph[ph];
    uint32_t l0 = 0, kap = 0;
    for (int q = 0; q < PH.nq; ++q) l0 |= ((uint32_t)(t >> q) & 1u) << PH.q[q];
    for (int k = 0; k < PH.kn; ++k) kap |= ((uint32_t)(t >> (PH.kq + k)) & 1u) << PH.kidx[k];
    for (int r = 0; r < 4; ++r)
      if ((kap >> r) & 1u) l0 |= PH.lbit[r];
    s_pl[ph * T + t] = (l0 << 8) | kap;
  }
  // tile index -> complement bits, 6 bits per table
  for (int i = tid; i < 5 * 64; i += NT) {
    const int tb = i >> 6, v = i & 63;
    uint64_t o = 0;
    for (int k = 0; k < 6; ++k)
      if (((v >> k) & 1) && 6 * tb + k < P.ncomp) o |= 1ull << P.comp[6 * tb + k];
    s_dep[tb][v] = o;
  }
  constexpr uint64_t GST = TWO ? 16u : 8u;  // HBM bytes per amplitude of the stored array
  const bool ld_psi8 = TWO && (flags & XF_LOAD_PSI);
  const uint64_t GLD = (TWO && !ld_psi8) ? 16u : 8u;
  __syncthreads();

  const uint64_t n_tiles = 1ull << (args.n - m);
  auto toff_of = [&](uint64_t t) {
    return s_dep[0][t & 63] | s_dep[1][(t >> 6) & 63] | s_dep[2][(t >> 12) & 63] | s_dep[3][(t >> 18) & 63] |
           s_dep[4][(t >> 24) & 63];
  };
  float acc_hi[3] = {0.f, 0.f, 0.f}, acc_lo[3] = {0.f, 0.f, 0.f};

  if (producer) {
    // ------------------------------------------------------------ producer warp
    // a tile is 2^(m - mlb) boxes of one tensor map; lane j copies box j, whose
    // tile-local offset j 2^mlb sets the local bits above the box
    const bool gen = (flags & XF_GEN_PLUS) != 0, do_store = (flags & XF_STORE) != 0;
    auto coords = [&](int k, uint64_t amp, int (&x)[5]) { tile_coords(P.ma[k], P.mw[k], amp << P.me[k], x); };
    auto load = [&](uint64_t t, int b) {  // tile t into buffer b, completing full[b]
      if (t >= n_tiles) return;
      const uint32_t fb = xsh(&s_full[b]);
      if (gen) {
        if (lane == 0) mbar_arrive(fb);
        return;
      }
      if (lane == 0) mbar_arrive_expect(fb, tile_n * (uint32_t)GLD);
      __syncwarp();
      const uint64_t toff = toff_of(t);
      const uint32_t nb = 1u << (m - P.mlb[0]), bb = (1u << P.mlb[0]) * (uint32_t)GLD;
      for (uint32_t j = lane; j < nb; j += 32) {
        int x[5];
        coords(0, toff + x_l2g(P, j << P.mlb[0]), x);
        tma_load5(tsh(b) + j * bb, &args.tm[0], x, fb);
      }
    };
    auto store = [&](uint64_t t, int b) {  // tile t from buffer b to HBM
      const uint64_t toff = toff_of(t);
      const uint32_t nb = 1u << (m - P.mlb[1]), bb = (1u << P.mlb[1]) * (uint32_t)GST;
      for (uint32_t j = lane; j < nb; j += 32) {
        int x[5];
        coords(1, toff + x_l2g(P, j << P.mlb[1]), x);
        tma_store5(&args.tm[1], x, tsh(b) + j * bb);
      }
      bulk_commit();
      bulk_wait_read0();  // the buffer may be refilled once the stores have read it
    };
    uint64_t tile = blockIdx.x;
    load(tile, 0);
    load(tile + gridDim.x, 1);
    int i = 0;
    for (; tile < n_tiles; tile += gridDim.x, ++i) {
      const int b2 = (i + 2) % kXNB;  // the previous tile's buffer, refilled with the tile two ahead
      if (i >= 1) {
        if (!mbar_wait(xsh(&s_done[b2]), (uint32_t)(((i - 1) / kXNB) & 1))) s_bad = 2;
        if (do_store) store(tile - gridDim.x, b2);
      }
      load(tile + 2ull * gridDim.x, b2);
    }
    if (i >= 1) {  // the last tile
      const int bl = (i - 1) % kXNB;
      if (!mbar_wait(xsh(&s_done[bl]), (uint32_t)(((i - 1) / kXNB) & 1))) s_bad = 2;
      if (do_store) store(tile - gridDim.x, bl);
    }
    bulk_wait0();
  } else {
    // ------------------------------------------------------------ compute warps
    // linear terms of C for tile t (warp 0): w_i = deg_out(i) - 2 #(outside neighbours set), g
    auto lin_terms = [&](uint64_t t, int par) {
      const uint64_t toff = toff_of(t);
      int g = 0;
      if (lane < m) {
        const uint64_t wm = P.wmask[lane];
        const int set = __popcll(toff & wm);
        s_lin[par][lane] = __popcll(wm) - 2 * set;
        g += set;  // crossing edges (i, b): [x_i != x_b] = x_b + x_i (1 - 2 x_b)
      }
      for (int k = lane; k < P.n_cc; k += 32) {
        const int a = P.ccnode[k];
        const uint64_t cm = P.ccmask[k];
        const int cnt = __popcll(toff & cm);
        g += ((toff >> a) & 1ull) ? __popcll(cm) - cnt : cnt;
      }
      for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(0xffffffffu, g, o);
      if (lane == 0) s_lin[par][15] = g;
    };
    uint64_t tile = blockIdx.x;
    if (has_diag && warp == 0) {
      if (tile < n_tiles) lin_terms(tile, 0);
      if (tile + gridDim.x < n_tiles) lin_terms(tile + gridDim.x, 1);
    }
    bar_compute(T);
    int i = 0;
    for (; tile < n_tiles; tile += gridDim.x, ++i) {
      const int cur = i % kXNB;
      const uint64_t t2 = tile + 2ull * gridDim.x;
      if (has_diag && warp == 0 && t2 < n_tiles) lin_terms(t2, (i + 2) % kXNB);
      if (!mbar_wait(xsh(&s_full[cur]), (uint32_t)((i / kXNB) & 1))) s_bad = 2;
      const uint32_t tb = tsh(cur);
      if (ld_psi8) {  // turnaround: the tile came in as 8-byte psi amplitudes; expand them in place to
                      // (psi.re, 0, psi.im, 0) elements (all threads read, then all write)
        constexpr int EPT = 1 << qx_reg_bits(TWO);  // elements per compute thread
        float2 v[EPT];
#pragma unroll
        for (int k = 0; k < EPT; ++k) v[k] = lds64(tb + 8u * ((uint32_t)tid + (uint32_t)T * k));
        bar_compute(T);
#pragma unroll
        for (int k = 0; k < EPT; ++k) sts128(tb + 16u * ((uint32_t)tid + (uint32_t)T * k), v[k].x, 0.f, v[k].y, 0.f);
        bar_compute(T);
      }
      const int* lin = s_lin[cur];
      float acc[3] = {0.f, 0.f, 0.f};
      for (int ph = 0; ph < n_ph; ++ph) {
        const XPhase& PH = P.ph[ph];
        const uint32_t pl = s_pl[ph * T + tid];
        XPh h;
        h.l0 = pl >> 8;  // local index of register index 0, relabel bits included
        const uint32_t kap = pl & 0xffu;
        h.tb = tb;
        h.pb = h.l0 * ES;
        h.lb0 = PH.lbit[0];
        h.lb1 = PH.lbit[1];
        h.lb2 = PH.lbit[2];
        h.lb3 = PH.lbit[3];
        h.sp0 = h.lb0 * ES;
        h.sp1 = h.lb1 * ES;
        h.sp2 = h.lb2 * ES;
        h.sp3 = h.lb3 * ES;
        h.fs = xsh(s_fs);
        h.lut = xsh(s_lut);
        h.ne = args.n_edges;
        const bool gen = (flags & XF_GEN_PLUS) && ph == 0;
        h.pw = gen ? args.plus_amp : s_w[4 * ph + 2];
        h.cutb = h.w0 = h.w1 = h.w2 = h.w3 = 0;
        const int diag = PH.diag;
        if (diag) {  // cut values: fs[l] + g + sum of w over the set local bits
          int cb = lin[15];
          for (uint32_t x = h.l0; x; x &= x - 1) cb += lin[__ffs(x) - 1];
          h.cutb = cb;  // includes the weights of the relabel bits set in l0
          // a register bit set in kappa is set in l0 and flips in j: its weight enters with -1
          h.w0 = ((kap & 1u) ? -1 : 1) * lin[__ffs(h.lb0) - 1];
          h.w1 = ((kap & 2u) ? -1 : 1) * lin[__ffs(h.lb1) - 1];
          h.w2 = ((kap & 4u) ? -1 : 1) * lin[__ffs(h.lb2) - 1];
          h.w3 = h.lb3 ? ((kap & 8u) ? -1 : 1) * lin[__ffs(h.lb3) - 1] : 0;
        }
        const int code = xcode(__popc(PH.m1), diag, __popc(PH.m3)) + (gen ? 125 : 0);
        // the phase's sums are weighted by 1 / |data scale|^2 where each is taken
        h.cs1 = make_float2(cs1.x, s_w[4 * ph]);
        h.cs3 = make_float2(cs3.x, s_w[4 * ph + 1]);
        const bool ok = TWO ? xdispatch2(code, h, acc) : xdispatch1(code, h, acc);
        if (!ok && tid == 0) s_bad = 1;
        bar_compute(T);
      }
      fence_async_smem();              // this thread's shared writes, before the bulk stores read them
      mbar_arrive(xsh(&s_done[cur]));  // the producer may now store this buffer and refill it
#pragma unroll
      for (int k = 0; k < 3; ++k) xacc(acc_hi[k], acc_lo[k], acc[k]);
    }
  }
  __syncthreads();

  // ---- per-CTA sums of the accumulators, fixed order; a phase code without a
  // kernel body (a planner fault) poisons the results with NaN
  __syncthreads();
  for (int k = 0; k < 3; ++k) {
    if (P.slot[k] < 0) continue;
    double v = (double)acc_hi[k] + (double)acc_lo[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) s_red[warp] = v;
    __syncthreads();
    if (tid == 0) {
      double s = 0;
      for (int w = 0; w < NT / 32; ++w) s += s_red[w];
      args.partials[(size_t)P.slot[k] * args.stride + blockIdx.x] = s_bad ? __longlong_as_double(0x7ff8000000000000ll) : s;
    }
    __syncthreads();
  }
}

#undef XL
#undef XS
#undef XW
#undef XCUT

// Dynamic shared memory: LUT, edge counts and phase bases, then the tile buffers.
size_t qx_smem(int two_state, int m, int n_edges, int n_phases) {
  const size_t T = (size_t)1 << (m - qx_reg_bits(two_state));
  const size_t tile = ((size_t)1 << m) * (two_state ? 16 : 8);
  size_t off = ((size_t)(n_edges + 1) * 8 + 127) & ~(size_t)127;
  off += (((size_t)1 << m) + 127) & ~(size_t)127;
  off += ((size_t)n_phases * T * 4 + 127) & ~(size_t)127;
  return off + 128 + (size_t)kXNB * tile;
}

// psi[x] <-> psi[NOT x] (every qubit flipped): pairs of amplitudes (2k, 2k + 1)
// swap with (N - 1 - 2k, N - 2 - 2k), in 16-byte words
__global__ void qx_flip_kernel(float4* psi, uint64_t half_words, uint64_t words) {
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < half_words;
       k += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t r = words - 1 - k;
    const float4 a = psi[k], b = psi[r];
    psi[k] = make_float4(b.z, b.w, b.x, b.y);
    psi[r] = make_float4(a.z, a.w, a.x, a.y);
  }
}

}  // namespace

qs_status launch_qx_flip(float2* psi, int n, cudaStream_t st) {
  const uint64_t words = 1ull << (n - 1), half = words / 2;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = (int)std::min<uint64_t>((half + 255) / 256, (uint64_t)std::max(sms, 1) * 8);
  qx_flip_kernel<<<std::max(grid, 1), 256, 0, st>>>(reinterpret_cast<float4*>(psi), half, words);
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

int qx_occupancy(int two_state, int m, int n_edges, int n_phases) {
  static std::map<long long, int> cache[2];  // a few (m, edges, phases) shapes per engine
  if (m < 5 + qx_reg_bits(two_state) || m > (two_state ? 12 : kXMaxM)) return 0;
  const size_t smem = qx_smem(two_state, m, n_edges, n_phases);
  const long long key = ((long long)m * 1024 + n_edges) * 64 + n_phases;
  auto it = cache[two_state].find(key);
  if (it != cache[two_state].end()) return it->second;
  const void* fn = two_state ? (const void*)qx_kernel<true> : (const void*)qx_kernel<false>;
  int blocks = 0;
  static size_t set_smem[2] = {0, 0};  // the attribute only grows
  if ((smem > set_smem[two_state] &&
       cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fn, (1 << (m - qx_reg_bits(two_state))) + 32, smem) !=
          cudaSuccess ||
      blocks < 1) {
    (void)cudaGetLastError();
    blocks = 0;
  } else if (smem > set_smem[two_state]) {
    set_smem[two_state] = smem;
  }
  cache[two_state][key] = blocks;
  return blocks;
}

int qx_grid(int two_state, int m, int n_edges, int n_phases, uint64_t n_tiles) {
  const int occ = qx_occupancy(two_state, m, n_edges, n_phases);
  if (occ < 1) return 0;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  uint64_t g = (uint64_t)(sms > 0 ? sms : 1) * occ;
  if (g > n_tiles) g = n_tiles;
  return (int)(g < 1 ? 1 : g);
}

namespace {

qs_status encode_map(const XPass& h, int k, void* base, CUtensorMap* out) {
  TileMapDims d;
  for (int i = 0; i < 5; ++i) {
    d.a[i] = h.ma[k][i];
    d.w[i] = h.mw[k][i];
    d.bx[i] = h.mbx[k][i];
  }
  d.e = h.me[k];
  d.lb = h.mlb[k];
  return encode_tile_map(d, base, false, out);
}

}  // namespace

qs_status launch_qx_pass(int two_state, const XPass* d_pass, const XPass& h, const XLaunch& L, cudaStream_t st) {
  if (h.m < 5 + qx_reg_bits(two_state) || h.m > (two_state ? 12 : kXMaxM) || h.m > L.n || L.grid < 1) {
    set_error("qaoa: invalid pass shape (internal error)");
    return QS_ERR_UNSUPPORTED;
  }
  if (qx_occupancy(two_state, h.m, L.n_edges, h.n_phases) < 1) {
    set_error("qaoa: the tile does not fit in shared memory");
    return QS_ERR_UNSUPPORTED;
  }
  XArgs a;
  void* ld_base = two_state && !(h.flags & XF_LOAD_PSI) ? (void*)L.il : (void*)L.psi;
  void* st_base = two_state ? (void*)L.il : (void*)L.psi;
  QS_TRY(encode_map(h, 0, ld_base, &a.tm[0]));
  QS_TRY(encode_map(h, 1, st_base, &a.tm[1]));
  a.pass = d_pass;
  a.psi = L.psi;
  a.il = L.il;
  a.coef = L.coef;
  a.fs = L.fs;
  a.partials = L.partials;
  a.plus_amp = (float)std::pow(2.0, -0.5 * L.n);
  a.stride = L.stride;
  a.n = L.n;
  a.n_edges = L.n_edges;
  const size_t smem = qx_smem(two_state, h.m, L.n_edges, h.n_phases);
  const int threads = (1 << (h.m - qx_reg_bits(two_state))) + 32;  // compute threads + the producer warp
  if (two_state)
    qx_kernel<true><<<L.grid, threads, smem, st>>>(a);
  else
    qx_kernel<false><<<L.grid, threads, smem, st>>>(a);
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

}  // namespace qs
