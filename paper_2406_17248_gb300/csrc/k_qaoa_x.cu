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
// A CTA of 2^(m-4) threads loops over tiles with the next tile's 16-byte
// cp.async copies in flight.  Each phase gives every thread the 16 amplitudes of
// one sub-cube (4 register bits), runs straight-line code for its steps (no op
// interpreter), and writes back to shared memory; the last phase stores to HBM
// straight from registers.  Tile buffers are aligned to their size in the
// shared window, so an element's address is the XOR of a per-thread base and a
// per-register-index offset (the tile swizzle is linear over GF(2)).  C(x) is
// assembled per amplitude from a per-pass table of in-tile edge counts and
// per-tile linear terms (computed by warp 0 for the next tile while the current
// one is processed), so no cut-value array is read.
#include <cmath>
#include <type_traits>

#include "qaoa_pass.h"
#include "qaoa_x.h"

namespace qs {

namespace {

constexpr int kXN = 16;  // amplitudes per thread per phase
constexpr int kXNB = 2;  // tile buffers

__device__ __forceinline__ uint32_t xsh(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void xcp16(uint32_t s, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void xcommit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void xwait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void xwait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
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
__device__ __forceinline__ void sts64(uint32_t a, float x, float y) {
  asm volatile("st.shared.v2.f32 [%0], {%1, %2};\n" ::"r"(a), "f"(x), "f"(y));
}
__device__ __forceinline__ void sts128(uint32_t a, float x, float y, float z, float w) {
  asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};\n" ::"r"(a), "f"(x), "f"(y), "f"(z), "f"(w));
}

struct XArgs {
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
// RX(c, s) = [[c, -is], [-is, c]] on register bit RB
template <int RB>
__device__ __forceinline__ void xrx1(float2 (&a)[kXN], float c, float s) {
#pragma unroll
  for (int j = 0; j < kXN; ++j) {
    if (j & (1 << RB)) continue;
    const int j1 = j | (1 << RB);
    const float2 x0 = a[j], x1 = a[j1];
    a[j].x = __fmaf_rn(c, x0.x, s * x1.y);
    a[j].y = __fmaf_rn(c, x0.y, -s * x1.x);
    a[j1].x = __fmaf_rn(c, x1.x, s * x0.y);
    a[j1].y = __fmaf_rn(c, x1.y, -s * x0.x);
  }
}
// ---------------------------------------------------------------- two-state steps
// RE = (psi.re, lam.re), IM = (psi.im, lam.im): RX(c, s) on both states at once
template <int RB>
__device__ __forceinline__ void xrx2(float2 (&RE)[kXN], float2 (&IM)[kXN], float2 c2, float2 s2, float2 ms2) {
#pragma unroll
  for (int j = 0; j < kXN; ++j) {
    if (j & (1 << RB)) continue;
    const int j1 = j | (1 << RB);
    const float2 r0 = RE[j], i0 = IM[j], r1 = RE[j1], i1 = IM[j1];
    RE[j] = __ffma2_rn(c2, r0, __fmul2_rn(s2, i1));
    IM[j] = __ffma2_rn(c2, i0, __fmul2_rn(ms2, r1));
    RE[j1] = __ffma2_rn(c2, r1, __fmul2_rn(s2, i0));
    IM[j1] = __ffma2_rn(c2, i1, __fmul2_rn(ms2, r0));
  }
}
// Im <lam|X_RB|psi> over the sub-cube (four independent partial sums)
template <int RB>
__device__ __forceinline__ float xgx2(const float2 (&RE)[kXN], const float2 (&IM)[kXN]) {
  float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
  for (int j = 0; j < kXN; ++j) {
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
  uint32_t pb;                  // shared address of the sub-cube base element
  uint32_t sp0, sp1, sp2, sp3;  // byte offsets of the register bits (XOR)
  uint32_t l0, lb0, lb1, lb2, lb3;
  int cutb, w0, w1, w2, w3;     // cut value = fs[l0 | L(j)] + cutb + W(j)
  const uint8_t* fs;
  const float2* lut;
  int ne;
  float2 cs1, cs3;
  bool last, store;
  float plus;
  char* gbase;                  // HBM address of the sub-cube base (last phase)
  uint64_t gb0, gb1, gb2, gb3;  // byte offsets of the register bits in HBM
};

// Register-index sums: L(j) = OR of the local bits, S(j) = XOR of the shared
// byte offsets, W(j) = sum of the linear cut weights, G(j) = sum of the HBM byte
// offsets of the register bits set in j.
#define XL(j) ((((j) & 1) ? h.lb0 : 0u) | (((j) & 2) ? h.lb1 : 0u) | (((j) & 4) ? h.lb2 : 0u) | (((j) & 8) ? h.lb3 : 0u))
#define XS(j) ((((j) & 1) ? h.sp0 : 0u) ^ (((j) & 2) ? h.sp1 : 0u) ^ (((j) & 4) ? h.sp2 : 0u) ^ (((j) & 8) ? h.sp3 : 0u))
#define XW(j) ((((j) & 1) ? h.w0 : 0) + (((j) & 2) ? h.w1 : 0) + (((j) & 4) ? h.w2 : 0) + (((j) & 8) ? h.w3 : 0))
#define XG(j) ((((j) & 1) ? h.gb0 : 0ull) + (((j) & 2) ? h.gb1 : 0ull) + (((j) & 4) ? h.gb2 : 0ull) + (((j) & 8) ? h.gb3 : 0ull))
// cut value of element j, kept inside the LUT (0..|E|) whatever the tables hold
#define XCUT(j) ((int)min((unsigned)((int)h.fs[h.l0 | XL(j)] + h.cutb + XW(j)), (unsigned)h.ne))

// RX on the first K register bits
template <int K>
__device__ __forceinline__ void xrx1_k(float2 (&a)[kXN], float2 cs) {
  if (K > 0) xrx1<0>(a, cs.x, cs.y);
  if (K > 1) xrx1<1>(a, cs.x, cs.y);
  if (K > 2) xrx1<2>(a, cs.x, cs.y);
  if (K > 3) xrx1<3>(a, cs.x, cs.y);
}
template <int K>
__device__ __forceinline__ float xrx2_k(float2 (&RE)[kXN], float2 (&IM)[kXN], float2 cs) {
  const float2 c2 = make_float2(cs.x, cs.x), s2 = make_float2(cs.y, cs.y), ms2 = make_float2(-cs.y, -cs.y);
  float g = 0.f;
  if (K > 0) {
    g += xgx2<0>(RE, IM);
    xrx2<0>(RE, IM, c2, s2, ms2);
  }
  if (K > 1) {
    g += xgx2<1>(RE, IM);
    xrx2<1>(RE, IM, c2, s2, ms2);
  }
  if (K > 2) {
    g += xgx2<2>(RE, IM);
    xrx2<2>(RE, IM, c2, s2, ms2);
  }
  if (K > 3) {
    g += xgx2<3>(RE, IM);
    xrx2<3>(RE, IM, c2, s2, ms2);
  }
  return g;
}

// One phase of the one-state kernel: RX on K1 bits, diagonal DG, RX on K3 bits.
template <int K1, int DG, int K3, bool GEN>
__device__ __forceinline__ void xphase1(const XPh& h, float (&acc)[3]) {
  float2 a[kXN];
  if (GEN) {
#pragma unroll
    for (int j = 0; j < kXN; ++j) a[j] = make_float2(h.plus, 0.f);
  } else {
#pragma unroll
    for (int j = 0; j < kXN; ++j) a[j] = lds64(h.pb ^ XS(j));
  }
  xrx1_k<K1>(a, h.cs1);
  if (DG == XD_COST) {
#pragma unroll
    for (int j = 0; j < kXN; ++j) {
      const float2 d = h.lut[XCUT(j)];
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
    acc[1] += e0 + e1;
  }
  xrx1_k<K3>(a, h.cs3);
  if (!h.last) {
#pragma unroll
    for (int j = 0; j < kXN; ++j) sts64(h.pb ^ XS(j), a[j].x, a[j].y);
  } else if (h.store) {
    if (h.gb0 == 8) {  // register bit 0 is qubit 0: pairs are adjacent in HBM
#pragma unroll
      for (int j = 0; j < kXN; j += 2)
        __stcs(reinterpret_cast<float4*>(h.gbase + XG(j)), make_float4(a[j].x, a[j].y, a[j + 1].x, a[j + 1].y));
    } else {
#pragma unroll
      for (int j = 0; j < kXN; ++j) __stcs(reinterpret_cast<float2*>(h.gbase + XG(j)), a[j]);
    }
  }
}

// One phase of the two-state kernel: the mixer steps take Im <lam|X_q|psi>
// into acc[0] (step 1) and acc[2] (step 3) before rotating both states.
template <int K1, int DG, int K3>
__device__ __forceinline__ void xphase2(const XPh& h, float (&acc)[3]) {
  float2 RE[kXN], IM[kXN];
#pragma unroll
  for (int j = 0; j < kXN; ++j) {
    const float4 e = lds128(h.pb ^ XS(j));
    RE[j] = make_float2(e.x, e.y);
    IM[j] = make_float2(e.z, e.w);
  }
  if (K1 > 0) acc[0] += xrx2_k<K1>(RE, IM, h.cs1);
  if (DG == XD_COST_GRAD) {
    float g0 = 0.f, g1 = 0.f;
#pragma unroll
    for (int j = 0; j < kXN; ++j) {
      const int k = XCUT(j);
      const float C = (float)(h.ne - 2 * k);
      const float im = __fmaf_rn(RE[j].y, IM[j].x, -IM[j].y * RE[j].x);  // Im(conj(lam) psi)
      if (j & 1) g1 = __fmaf_rn(C, im, g1);
      else g0 = __fmaf_rn(C, im, g0);
      const float2 d = h.lut[k];
      const float2 dr = make_float2(d.x, d.x), di = make_float2(d.y, d.y), mdi = make_float2(-d.y, -d.y);
      const float2 r = RE[j], i = IM[j];
      RE[j] = __ffma2_rn(dr, r, __fmul2_rn(mdi, i));
      IM[j] = __ffma2_rn(dr, i, __fmul2_rn(di, r));
    }
    acc[1] += g0 + g1;
  } else if (DG == XD_ENERGY) {
    float e0 = 0.f, e1 = 0.f;
#pragma unroll
    for (int j = 0; j < kXN; ++j) {
      const float C = (float)(h.ne - 2 * XCUT(j));
      const float pr = __fmaf_rn(RE[j].x, RE[j].x, IM[j].x * IM[j].x);
      if (j & 1) e1 = __fmaf_rn(C, pr, e1);
      else e0 = __fmaf_rn(C, pr, e0);
      RE[j].y = C * RE[j].x;  // lam = C psi
      IM[j].y = C * IM[j].x;
    }
    acc[1] += e0 + e1;
  }
  if (K3 > 0) acc[2] += xrx2_k<K3>(RE, IM, h.cs3);
  if (!h.last) {
#pragma unroll
    for (int j = 0; j < kXN; ++j) sts128(h.pb ^ XS(j), RE[j].x, RE[j].y, IM[j].x, IM[j].y);
  } else if (h.store) {
#pragma unroll
    for (int j = 0; j < kXN; ++j)
      __stcs(reinterpret_cast<float4*>(h.gbase + XG(j)), make_float4(RE[j].x, RE[j].y, IM[j].x, IM[j].y));
  }
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
  switch (code) {
#define C2(K1, DG, K3) \
  case xcode(K1, DG, K3): xphase2<K1, DG, K3>(h, acc); return true;
    C2(1, 0, 0) C2(2, 0, 0) C2(3, 0, 0) C2(4, 0, 0)
    C2(0, 0, 1) C2(0, 0, 2) C2(0, 0, 3) C2(0, 0, 4)
    C2(0, XD_COST_GRAD, 4) C2(1, XD_COST_GRAD, 4) C2(2, XD_COST_GRAD, 4) C2(3, XD_COST_GRAD, 4)
    C2(4, XD_COST_GRAD, 4)
    C2(0, XD_COST_GRAD, 0) C2(1, XD_COST_GRAD, 0) C2(2, XD_COST_GRAD, 0) C2(3, XD_COST_GRAD, 0)
    C2(4, XD_COST_GRAD, 0)
    C2(0, XD_ENERGY, 4) C2(1, XD_ENERGY, 4) C2(2, XD_ENERGY, 4) C2(3, XD_ENERGY, 4) C2(4, XD_ENERGY, 4)
#undef C2
    default: return false;
  }
}

template <bool TWO>
__global__ void __launch_bounds__(TWO ? 256 : 512, 1) qx_kernel(XArgs args) {
  constexpr uint32_t ES = TWO ? 16 : 8;  // bytes per shared-memory element
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ XPass P;
  __shared__ uint64_t s_gk[16], s_dep[5][64];
  __shared__ uint32_t s_pk[16];
  __shared__ int s_lin[2][16];  // per tile parity: w_i of local bit i (i < 13), g at [15]
  __shared__ double s_red[16];
  __shared__ int s_bad;
  {
    const int* src = reinterpret_cast<const int*>(args.pass);
    int* dst = reinterpret_cast<int*>(&P);
    for (int i = threadIdx.x; i < (int)(sizeof(XPass) / 4); i += blockDim.x) dst[i] = src[i];
    if (threadIdx.x == 0) s_bad = 0;
  }
  __syncthreads();
  const int tid = threadIdx.x, T = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const int m = P.m, n_ph = P.n_phases;
  const uint32_t flags = P.flags, tile_n = 1u << m, tile_bytes = tile_n * ES;
  const int E1 = args.n_edges + 1;
  bool has_diag = false;
  for (int i = 0; i < n_ph; ++i) has_diag |= P.ph[i].diag != XD_NONE;

  // ---- shared memory: LUT | in-tile edge counts | phase bases | tiles (aligned to their size)
  float2* s_lut = reinterpret_cast<float2*>(smem);
  size_t off = ((size_t)E1 * 8 + 127) & ~(size_t)127;
  uint8_t* s_fs = smem + off;
  off += ((size_t)tile_n + 127) & ~(size_t)127;
  uint32_t* s_pl = reinterpret_cast<uint32_t*>(smem + off);
  off += (size_t)kXMaxPhases * T * 4;
  const uint32_t sh0 = xsh(smem);
  const uint32_t tile0 = (sh0 + (uint32_t)off + tile_bytes - 1) & ~(tile_bytes - 1);
  const uint32_t tsh[kXNB] = {tile0, tile0 + tile_bytes};

  if (P.cd >= 0)
    for (int i = tid; i < E1; i += T) s_lut[i] = args.coef[P.cd + i];
  if (has_diag && P.fs_off >= 0) {
    const uint4* src = reinterpret_cast<const uint4*>(args.fs + P.fs_off);
    for (uint32_t i = tid; i < (tile_n >> 4); i += T) reinterpret_cast<uint4*>(s_fs)[i] = src[i];
  }
  const float2 cs1 = P.c1 >= 0 ? args.coef[P.c1] : make_float2(1.f, 0.f);
  const float2 cs3 = P.c3 >= 0 ? args.coef[P.c3] : make_float2(1.f, 0.f);
  // phase bases of this thread: (local index << 16) | swizzled position
  for (int ph = 0; ph < n_ph; ++ph) {
    const XPhase& PH = P.ph[ph];
    uint32_t l0 = 0;
    for (int i = 0; i < PH.nq; ++i) l0 |= ((uint32_t)(tid >> i) & 1u) << PH.q[i];
    s_pl[ph * T + tid] = (l0 << 16) | qaoa_swizzle(!TWO, l0);
  }
  // global index of the last phase's sub-cube base (its stores go straight to HBM)
  const uint64_t g_last = x_l2g(P, s_pl[(n_ph - 1) * T + tid] >> 16);
  // tile index -> complement bits, 6 bits per table
  for (int i = tid; i < 5 * 64; i += T) {
    const int tb = i >> 6, v = i & 63;
    uint64_t o = 0;
    for (int k = 0; k < 6; ++k)
      if (((v >> k) & 1) && 6 * tb + k < P.ncomp) o |= 1ull << P.comp[6 * tb + k];
    s_dep[tb][v] = o;
  }
  // copy addressing: thread tid copies chunks ch = tid + k T of 16 bytes (two
  // amplitudes of psi, or one interleaved element; the turnaround reads psi
  // pairs into the slot of the pair's first element).  Global offsets are byte
  // offsets: the tile offset, the thread's part and the chunk's part cover
  // disjoint qubits, so they add.
  const bool rd_il = TWO && !(flags & XF_LOAD_PSI);
  const uint32_t EPC = rd_il ? 1u : 2u;
  const uint64_t GE = rd_il ? 16u : 8u;  // bytes per amplitude in HBM of the loaded array
  const uint32_t nk = tile_n / EPC / T;
  for (uint32_t k = tid; k < nk; k += T) {
    s_gk[k] = x_l2g(P, k * T * EPC) * GE;
    s_pk[k] = qaoa_swizzle(!TWO, k * T * EPC) * ES;
  }
  const uint64_t gt = x_l2g(P, tid * EPC) * GE;
  const uint32_t pt = qaoa_swizzle(!TWO, tid * EPC) * ES;
  const char* src_base = rd_il ? reinterpret_cast<const char*>(args.il) : reinterpret_cast<const char*>(args.psi);
  char* dst_base = TWO ? reinterpret_cast<char*>(args.il) : reinterpret_cast<char*>(args.psi);
  __syncthreads();

  const uint64_t n_tiles = 1ull << (args.n - m);
  auto toff_of = [&](uint64_t t) {
    return s_dep[0][t & 63] | s_dep[1][(t >> 6) & 63] | s_dep[2][(t >> 12) & 63] | s_dep[3][(t >> 18) & 63] |
           s_dep[4][(t >> 24) & 63];
  };
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
  auto issue = [&](uint64_t t, uint32_t tb) {
    if (!(flags & XF_GEN_PLUS)) {
      const char* gb = src_base + toff_of(t) * GE + gt;
      const uint32_t db = tb ^ pt;
      for (uint32_t k = 0; k < nk; ++k) xcp16(db ^ s_pk[k], gb + s_gk[k]);
    }
    xcommit();
  };

  float acc_hi[3] = {0.f, 0.f, 0.f}, acc_lo[3] = {0.f, 0.f, 0.f};

  uint64_t tile = blockIdx.x;
  if (tile < n_tiles) {
    issue(tile, tsh[0]);
    if (has_diag && warp == 0) lin_terms(tile, 0);
  } else {
    xcommit();
  }
  for (int it = 0; tile < n_tiles; ++it, tile += gridDim.x) {
    const int cur = it & 1;
    const uint64_t next = tile + gridDim.x;
    if (next < n_tiles) {
      issue(next, tsh[cur ^ 1]);
      if (has_diag && warp == 0) lin_terms(next, cur ^ 1);
    } else {
      xcommit();
    }
    xwait1();
    const uint32_t tb = tsh[cur];
    if (TWO && (flags & XF_LOAD_PSI)) {
      // turnaround: the pair (psi_l, psi_l+1) landed in the slot of l; spread it
      // into two elements (psi, lam = 0); slot(l + 1) = slot(l) ^ 1
      for (uint32_t k = 0; k < nk; ++k) {
        const uint32_t a = tb ^ pt ^ s_pk[k];
        const float4 v = lds128(a);
        sts128(a, v.x, 0.f, v.y, 0.f);
        sts128(a ^ 16u, v.z, 0.f, v.w, 0.f);
      }
    }
    __syncthreads();
    const uint64_t toff = toff_of(tile);
    const int* lin = s_lin[cur];
    float acc[3] = {0.f, 0.f, 0.f};

    for (int ph = 0; ph < n_ph; ++ph) {
      const XPhase& PH = P.ph[ph];
      const uint32_t pl = s_pl[ph * T + tid];
      XPh h;
      h.l0 = pl >> 16;
      h.pb = tb ^ ((pl & 0xffffu) * ES);
      h.sp0 = PH.spos[0] * ES;
      h.sp1 = PH.spos[1] * ES;
      h.sp2 = PH.spos[2] * ES;
      h.sp3 = PH.spos[3] * ES;
      h.lb0 = PH.lbit[0];
      h.lb1 = PH.lbit[1];
      h.lb2 = PH.lbit[2];
      h.lb3 = PH.lbit[3];
      h.fs = s_fs;
      h.lut = s_lut;
      h.ne = args.n_edges;
      h.cs1 = cs1;
      h.cs3 = cs3;
      h.plus = args.plus_amp;
      h.last = ph == n_ph - 1;
      h.store = (flags & XF_STORE) != 0;
      h.cutb = h.w0 = h.w1 = h.w2 = h.w3 = 0;
      const int diag = PH.diag;
      if (diag) {  // cut values: fs[l] + g + sum of w over the set local bits
        int cb = lin[15];
        for (uint32_t x = h.l0; x; x &= x - 1) cb += lin[__ffs(x) - 1];
        h.cutb = cb;
        h.w0 = lin[__ffs(h.lb0) - 1];
        h.w1 = lin[__ffs(h.lb1) - 1];
        h.w2 = lin[__ffs(h.lb2) - 1];
        h.w3 = lin[__ffs(h.lb3) - 1];
      }
      if (h.last) {
        h.gbase = dst_base + (toff + g_last) * ES;
        h.gb0 = PH.gbit[0] * ES;
        h.gb1 = PH.gbit[1] * ES;
        h.gb2 = PH.gbit[2] * ES;
        h.gb3 = PH.gbit[3] * ES;
      } else {
        h.gbase = nullptr;
        h.gb0 = h.gb1 = h.gb2 = h.gb3 = 0;
      }
      const int code = xcode(__popc(PH.m1), diag, __popc(PH.m3)) + ((flags & XF_GEN_PLUS) && ph == 0 ? 125 : 0);
      const bool ok = TWO ? xdispatch2(code, h, acc) : xdispatch1(code, h, acc);
      if (!ok && tid == 0) s_bad = 1;
      if (!h.last) __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) xacc(acc_hi[k], acc_lo[k], acc[k]);
    __syncthreads();  // this buffer is refilled by the copies issued in the next iteration
  }
  xwait0();

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
      for (int w = 0; w < (T + 31) / 32; ++w) s += s_red[w];
      args.partials[(size_t)P.slot[k] * args.stride + blockIdx.x] = s_bad ? __longlong_as_double(0x7ff8000000000000ll) : s;
    }
    __syncthreads();
  }
}

#undef XL
#undef XS
#undef XW
#undef XG
#undef XCUT

// Dynamic shared memory: LUT, edge counts and phase bases, then the tile
// buffers at the next multiple of their size (at most one tile of padding).
size_t qx_smem(int two_state, int m, int n_edges) {
  const size_t T = (size_t)1 << (m - 4);
  const size_t tile = ((size_t)1 << m) * (two_state ? 16 : 8);
  size_t off = ((size_t)(n_edges + 1) * 8 + 127) & ~(size_t)127;
  off += (((size_t)1 << m) + 127) & ~(size_t)127;
  off += (size_t)kXMaxPhases * T * 4;
  return off + tile + (size_t)kXNB * tile;
}

}  // namespace

int qx_occupancy(int two_state, int m, int n_edges, int /*n_phases*/) {
  static int last_key[2] = {-1, -1}, last_occ[2] = {0, 0};
  if (m < 9 || m > (two_state ? 12 : kXMaxM)) return 0;
  const size_t smem = qx_smem(two_state, m, n_edges);
  const int key = m * 1024 + n_edges;
  if (last_key[two_state] == key) return last_occ[two_state];
  const void* fn = two_state ? (const void*)qx_kernel<true> : (const void*)qx_kernel<false>;
  int blocks = 0;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fn, 1 << (m - 4), smem) != cudaSuccess || blocks < 1) {
    (void)cudaGetLastError();
    blocks = 0;
  }
  last_key[two_state] = key;
  last_occ[two_state] = blocks;
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

qs_status launch_qx_pass(int two_state, const XPass* d_pass, const XPass& h, const XLaunch& L, cudaStream_t st) {
  if (h.m < 9 || h.m > (two_state ? 12 : kXMaxM) || h.m > L.n || L.grid < 1) {
    set_error("qaoa: invalid pass shape (internal error)");
    return QS_ERR_UNSUPPORTED;
  }
  if (qx_occupancy(two_state, h.m, L.n_edges, h.n_phases) < 1) {
    set_error("qaoa: the tile does not fit in shared memory");
    return QS_ERR_UNSUPPORTED;
  }
  XArgs a;
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
  const size_t smem = qx_smem(two_state, h.m, L.n_edges);
  const int threads = 1 << (h.m - 4);
  if (two_state)
    qx_kernel<true><<<L.grid, threads, smem, st>>>(a);
  else
    qx_kernel<false><<<L.grid, threads, smem, st>>>(a);
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

}  // namespace qs
