// QAOA tile passes (§5.2 ansatz, §6.2 QuPack QAOA simulator): the mixer RX(beta)
// on every tile bit and the cost phase exp(-i gs gamma C(x)) from a per-amplitude
// cut-value array, with the adjoint gradient ops of the reverse sweep.
//
// Same tiling as the generic engine (a tile = 2^m amplitudes over a bit set S,
// staged in shared memory, processed in phases of 4 register bits), but the op
// stream is specialised: a phase applies RX to (up to) all 4 register bits at
// once, fully unrolled and without predicates; the cost phase, its gradient
// C(x) Im(conj(lam) psi), the energy C|psi|^2 and the mixer gradient
// Im <lam|X_q|psi> are fused into the same register pass.  Gradient partials
// stay in registers per thread (FP32 within a tile, FP64 across tiles) and are
// reduced once per CTA at the end.
//
// Tiles are double-buffered: while a CTA computes tile t, 16-byte cp.async
// copies of tile t+grid (psi, lam and the cut values) are already in flight,
// so HBM reads overlap the shared-memory compute of the previous tile.
#include <type_traits>

#include "qaoa_pass.h"

namespace qs {

namespace {

template <class T>
struct QV;
template <>
struct QV<float> {
  using V = float2;
};
template <>
struct QV<double> {
  using V = double2;
};

__device__ __forceinline__ float qfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double qfma(double a, double b, double c) { return __fma_rn(a, b, c); }

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

constexpr int QRN = 16;

// RX(c, s) = [[c, -is], [-is, c]] on register bit RB of a 16-amplitude sub-cube
template <int RB, class V, class T>
__device__ __forceinline__ void rx_bit(V (&a)[QRN], T c, T s) {
#pragma unroll
  for (int j = 0; j < QRN; ++j) {
    if (j & (1 << RB)) continue;
    const int j1 = j | (1 << RB);
    const V x0 = a[j], x1 = a[j1];
    V y0, y1;
    y0.x = qfma(c, x0.x, s * x1.y);
    y0.y = qfma(c, x0.y, -s * x1.x);
    y1.x = qfma(c, x1.x, s * x0.y);
    y1.y = qfma(c, x1.y, -s * x0.x);
    a[j] = y0;
    a[j1] = y1;
  }
}

// sum over pairs of Im(conj(b0) a1 + conj(b1) a0) = Im <b| X_RB |a> on the sub-cube
// (four independent partial sums: the FMA chains stay short)
template <int RB, class V, class T>
__device__ __forceinline__ T gradx_bit(const V (&a)[QRN], const V (&b)[QRN]) {
  T s0 = 0, s1 = 0, s2 = 0, s3 = 0;
#pragma unroll
  for (int j = 0; j < QRN; ++j) {
    if (j & (1 << RB)) continue;
    const int j1 = j | (1 << RB);
    s0 = qfma(b[j].x, a[j1].y, s0);
    s1 = qfma(-b[j].y, a[j1].x, s1);
    s2 = qfma(b[j1].x, a[j].y, s2);
    s3 = qfma(-b[j1].y, a[j].x, s3);
  }
  return (s0 + s1) + (s2 + s3);
}

template <class V>
__device__ __forceinline__ V qcmul(V d, V a) {
  V r;
  r.x = qfma(d.x, a.x, -d.y * a.y);
  r.y = qfma(d.x, a.y, d.y * a.x);
  return r;
}

struct QArgs {
  float4* il0;  // interleaved (psi, lam) buffer, amplitudes [0, il_half)
  float4* il1;  // ... amplitudes [il_half, 2^n)
  uint64_t il_half;
  void* psi;
  void* lam;
  const QPassDesc* pass;
  const void* coef;  // complex table: per layer lut[E+1], lut_dag[E+1], rx, rx_dag
  const uint8_t* cut;
  double* partials;
  int n;
  int n_edges;
  int stride;
};

// Global index of local index l (tile offset excluded): OR of the global bits of l.
__device__ __forceinline__ uint64_t local_to_global(const QPassDesc& P, uint32_t l) {
  return (l & ((1u << P.c) - 1u)) | P.hiA[(l >> P.c) & 63] | P.hiB[(l >> (P.c + 6)) & 63];
}

// Per-thread address tables of a pass.  Thread t handles the 16-byte chunks
// ch = t + 256 k of a tile; the global index and the swizzled position are both
// linear in the bits of the chunk's local index, so each splits into a
// per-thread part (bits of t) and a per-k part (bits of k) shared by all threads.
struct QAddr {
  uint64_t gt;  // global index of the thread's part
  uint32_t pt;  // swizzled position of the thread's part
  uint64_t gcut[2];  // global index of the thread's cut-value runs (within the tile)
};

__device__ __forceinline__ QAddr make_addr(const QPassDesc& P, int epc, bool sw64, uint64_t* s_gk, uint32_t* s_pk) {
  QAddr A;
  const uint32_t lt = (uint32_t)threadIdx.x * epc;
  A.gt = local_to_global(P, lt);
  A.pt = qaoa_swizzle(sw64, lt);
  const uint32_t nk = ((1u << P.m) / epc + kTileThreads - 1) / kTileThreads;
  for (uint32_t k = threadIdx.x; k < nk; k += blockDim.x) {
    const uint32_t lk = k * kTileThreads * epc;
    s_gk[k] = local_to_global(P, lk);
    s_pk[k] = qaoa_swizzle(sw64, lk);
  }
  const int run = P.c >= 4 ? 16 : 8;
  A.gcut[0] = local_to_global(P, (uint32_t)threadIdx.x * run);
  A.gcut[1] = local_to_global(P, (uint32_t)(threadIdx.x + kTileThreads) * run);
  return A;
}

__device__ __forceinline__ uint64_t tile_offset(const QPassDesc& P, uint64_t tile) {
  uint64_t toff = 0;
  for (int i = 0; i < P.ncomp; ++i) toff |= ((tile >> i) & 1ull) << P.comp[i];
  return toff;
}

// Asynchronous copies of the cut values of one tile, in local-index order.
__device__ __forceinline__ void issue_cut(const QPassDesc& P, uint64_t toff, const QAddr& A, const uint8_t* cut,
                                          uint8_t* b_cut) {
  const uint32_t tile_n = 1u << P.m;
  if (P.c >= 4) {  // runs of 16 contiguous bytes
    for (uint32_t r = threadIdx.x, i = 0; r < (tile_n >> 4); r += kTileThreads, ++i)
      cp_async16(b_cut + (r << 4), cut + (toff | (i == 0 ? A.gcut[0] : i == 1 ? A.gcut[1] : local_to_global(P, r << 4))));
  } else if (P.c == 3) {  // runs of 8
    for (uint32_t r = threadIdx.x, i = 0; r < (tile_n >> 3); r += kTileThreads, ++i)
      cp_async8(b_cut + (r << 3), cut + (toff | (i == 0 ? A.gcut[0] : i == 1 ? A.gcut[1] : local_to_global(P, r << 3))));
  } else {  // shorter runs: plain byte loads
    for (uint32_t l = threadIdx.x; l < tile_n; l += kTileThreads) b_cut[l] = cut[toff | local_to_global(P, l)];
  }
}

// Issue the asynchronous copies of one tile (psi, lam, cut) into one buffer.
template <class T, int NS>
__device__ __forceinline__ void issue_tile(const QPassDesc& P, uint64_t toff, const QArgs& args, const QAddr& A,
                                           const uint64_t* s_gk, const uint32_t* s_pk, typename QV<T>::V* b_psi,
                                           typename QV<T>::V* b_lam, uint8_t* b_cut) {
  using V = typename QV<T>::V;
  const uint32_t flags = P.flags;
  constexpr int EPC = sizeof(T) == 4 ? 2 : 1;  // amplitudes per 16-byte chunk
  const uint32_t nk = (1u << P.m) / EPC / kTileThreads;
  const V* g_psi = reinterpret_cast<const V*>(args.psi);
  const V* g_lam = reinterpret_cast<const V*>(args.lam);
  const bool ld_psi = flags & PF_LOAD_PSI;
  const bool ld_lam = NS == 2 && (flags & PF_LOAD_LAM);
  if (ld_psi || ld_lam) {
    if (nk == 0) {  // tiles smaller than one chunk per thread
      for (uint32_t ch = threadIdx.x; ch < (1u << P.m) / EPC; ch += blockDim.x) {
        const uint32_t l = ch * EPC;
        const uint64_t g = toff | local_to_global(P, l);
        const uint32_t p = qaoa_swizzle(sizeof(T) == 4, l);
        if (ld_psi) cp_async16(b_psi + p, g_psi + g);
        if (ld_lam) cp_async16(b_lam + p, g_lam + g);
      }
    } else {
      const uint64_t gb = toff | A.gt;
      for (uint32_t k = 0; k < nk; ++k) {
        const uint64_t g = gb | s_gk[k];
        const uint32_t p = A.pt ^ s_pk[k];
        if (ld_psi) cp_async16(b_psi + p, g_psi + g);
        if (ld_lam) cp_async16(b_lam + p, g_lam + g);
      }
    }
  }
  if (flags & PF_NEED_CUT) issue_cut(P, toff, A, args.cut, b_cut);
}

// Compensated FP32 accumulation (TwoSum): hi + lo carries about 48 bits, so the
// per-thread sums over all tiles of a launch stay accurate without FP64 work in
// the loop (FP64 instructions are slow on this GPU).
__device__ __forceinline__ void acc_add(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bb = s - hi;
  lo += (hi - (s - bb)) + (x - bb);
  hi = s;
}
__device__ __forceinline__ void acc_add(double& hi, double& lo, double x) { hi += x; }

template <class T, int NS>
__global__ void __launch_bounds__(kTileThreads, (sizeof(T) == 4 && NS == 1) ? 2 : 1) qaoa_pass_kernel(QArgs args) {
  using V = typename QV<T>::V;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ QPassDesc P;

  // ---- stage the pass descriptor and the coefficients of its layers
  {
    const int* src = reinterpret_cast<const int*>(args.pass);
    int* dst = reinterpret_cast<int*>(&P);
    for (int i = threadIdx.x; i < (int)(sizeof(QPassDesc) / 4); i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  const int E1 = args.n_edges + 1;
  const int per_layer = 2 * E1 + 2;
  const int n_coef = per_layer * kQaoaMaxLayersPerPass;
  V* s_coef = reinterpret_cast<V*>(smem);
  {
    const V* g = reinterpret_cast<const V*>(args.coef) + (size_t)P.layer_lo * per_layer;
    const int nc = per_layer * P.n_layers;
    for (int i = threadIdx.x; i < nc; i += blockDim.x) s_coef[i] = g[i];
  }
  const int m = P.m, c = P.c;
  const uint32_t flags = P.flags;
  const uint32_t tile_n = 1u << m;
  // layout: coef | buffer 0 (psi, lam, cut) | buffer 1 | reduction | per-thread FP64 | sub-cube bases
  unsigned char* base = smem + ((n_coef * sizeof(V) + 127) & ~(size_t)127);
  const size_t buf_bytes = ((size_t)NS * tile_n * sizeof(V) + tile_n + 127) & ~(size_t)127;
  // buffer b: psi at base + b * buf_bytes, then lam, then the cut values
  auto buf_psi = [&](int b) { return reinterpret_cast<V*>(base + b * buf_bytes); };
  auto buf_lam = [&](int b) { return buf_psi(b) + (NS == 2 ? tile_n : 0); };
  auto buf_cut = [&](int b) { return reinterpret_cast<uint8_t*>(buf_psi(b) + NS * tile_n); };
  double* s_red = reinterpret_cast<double*>(base + 2 * buf_bytes);  // [kTileWarps]
  double* s_accd = s_red + kTileWarps;                              // [kQaoaMaxAcc][kTileThreads]
  uint32_t* s_base = reinterpret_cast<uint32_t*>(s_accd + kQaoaMaxAcc * kTileThreads);  // [phase][sub-cube]

  const int tid = threadIdx.x;
  V* g_psi = reinterpret_cast<V*>(args.psi);
  V* g_lam = reinterpret_cast<V*>(args.lam);
  const uint32_t lowmask = (1u << c) - 1u;
  const uint64_t n_tiles = 1ull << (args.n - m);
  const int n_edges = args.n_edges;
  constexpr bool C64 = sizeof(T) == 4;

  // sub-cube base of every phase, packed as (local index << 16) | swizzled position
  const uint32_t nsub = tile_n >> 4;
  for (int ph = 0; ph < P.n_phases; ++ph) {
    const QPhase& PH = P.phases[ph];
    for (uint32_t u = tid; u < nsub; u += blockDim.x) {
      uint32_t p0 = 0, l0 = 0;
      for (int i = 0; i < PH.nq; ++i)
        if ((u >> i) & 1u) {
          p0 ^= PH.sq[i];
          l0 |= 1u << PH.Q[i];
        }
      s_base[ph * nsub + u] = (l0 << 16) | p0;
    }
  }
  __shared__ uint64_t s_gk[16];
  __shared__ uint32_t s_pk[16];
  constexpr int EPC = C64 ? 2 : 1;
  const QAddr A = make_addr(P, EPC, C64, s_gk, s_pk);
  const uint32_t nk = tile_n / EPC / kTileThreads;
  __syncthreads();
  // per-thread accumulators over every tile of the launch
  T acc_hi[kQaoaMaxAcc] = {0, 0, 0, 0}, acc_lo[kQaoaMaxAcc] = {0, 0, 0, 0};
  const int n_acc = P.n_acc;

  uint64_t tile = blockIdx.x;
  if (tile < n_tiles)
    issue_tile<T, NS>(P, tile_offset(P, tile), args, A, s_gk, s_pk, buf_psi(0), buf_lam(0), buf_cut(0));
  cp_async_commit();
  for (int it = 0; tile < n_tiles; ++it, tile += gridDim.x) {
    const int cur = it & 1;
    const uint64_t next = tile + gridDim.x;
    if (next < n_tiles)
      issue_tile<T, NS>(P, tile_offset(P, next), args, A, s_gk, s_pk, buf_psi(cur ^ 1), buf_lam(cur ^ 1),
                        buf_cut(cur ^ 1));
    cp_async_commit();
    cp_async_wait1();  // this tile's copies have landed (the next tile's may still fly)
    V* const bp = buf_psi(cur);
    V* const bl = buf_lam(cur);
    const uint8_t* const bc = buf_cut(cur);
    if (flags & PF_GEN_PLUS) {
      V v;
      v.x = (T)P.plus_amp;
      v.y = (T)0;
      for (uint32_t l = tid; l < tile_n; l += blockDim.x) bp[l] = v;  // a constant: no swizzle needed
    }
    __syncthreads();

    // ---------------------------------------------------------------- phases
    T acc[kQaoaMaxAcc] = {0, 0, 0, 0};
    for (int ph = 0; ph < P.n_phases; ++ph) {
      const QPhase& PH = P.phases[ph];
      // position of element j = position of the sub-cube base XOR the positions
      // of j's register bits (the swizzle is linear); the local index likewise
      const uint32_t s0 = PH.sreg[0], s1 = PH.sreg[1], s2 = PH.sreg[2], s3 = PH.sreg[3];
      const uint32_t r0 = 1u << PH.R[0], r1 = 1u << PH.R[1], r2 = 1u << PH.R[2], r3 = 1u << PH.R[3];
      const bool ph_cut = PH.need_cut;
      for (uint32_t u = tid; u < nsub; u += kTileThreads) {
        const uint32_t bw = s_base[ph * nsub + u];
        const uint32_t p0 = bw & 0xffffu, l0 = bw >> 16;
#define QPOS(j) \
  (p0 ^ (((j) & 1) ? s0 : 0u) ^ (((j) & 2) ? s1 : 0u) ^ (((j) & 4) ? s2 : 0u) ^ (((j) & 8) ? s3 : 0u))
#define QLOC(j) \
  (l0 | (((j) & 1) ? r0 : 0u) | (((j) & 2) ? r1 : 0u) | (((j) & 4) ? r2 : 0u) | (((j) & 8) ? r3 : 0u))
        uint32_t cw[QRN / 4] = {0, 0, 0, 0};
        V a[QRN], b[QRN];
#pragma unroll
        for (int j = 0; j < QRN; ++j) {
          const uint32_t p = QPOS(j);
          a[j] = bp[p];
          if (NS == 2) b[j] = bl[p];
          if (ph_cut) cw[j >> 2] |= (uint32_t)bc[QLOC(j)] << (8 * (j & 3));
        }
#define QCUT(j) ((int)((cw[(j) >> 2] >> (8 * ((j) & 3))) & 255u))
        for (int si = 0; si < PH.n_steps; ++si) {
          const QStep st = PH.steps[si];
          const V* lay = s_coef + st.layer * per_layer;
          T g = 0;
          switch (st.type) {
            case QST_COST: {
              const V* lut = lay + ((st.flags & QSF_DAG) ? E1 : 0);
#pragma unroll
              for (int j = 0; j < QRN; ++j) {
                const V d = lut[QCUT(j)];
                a[j] = qcmul(d, a[j]);
                if (NS == 2 && (st.flags & QSF_LAM)) b[j] = qcmul(d, b[j]);
              }
              break;
            }
            case QST_RX: {
              const V cs = lay[2 * E1 + ((st.flags & QSF_DAG) ? 1 : 0)];
              const T cc = cs.x, ss = cs.y;
              const bool both = NS == 2 && (st.flags & QSF_LAM);
              if (st.mask & 1) {
                rx_bit<0>(a, cc, ss);
                if (both) rx_bit<0>(b, cc, ss);
              }
              if (st.mask & 2) {
                rx_bit<1>(a, cc, ss);
                if (both) rx_bit<1>(b, cc, ss);
              }
              if (st.mask & 4) {
                rx_bit<2>(a, cc, ss);
                if (both) rx_bit<2>(b, cc, ss);
              }
              if (st.mask & 8) {
                rx_bit<3>(a, cc, ss);
                if (both) rx_bit<3>(b, cc, ss);
              }
              break;
            }
            case QST_GRAD_RX: {
              // mixer gradient Im <lam|X_q|psi> for each masked bit, then RX^dag on both
              const V cs = lay[2 * E1 + 1];
              const T cc = cs.x, ss = cs.y;
              if (NS == 2) {
                if (st.mask & 1) {
                  g += gradx_bit<0, V, T>(a, b);
                  rx_bit<0>(a, cc, ss);
                  rx_bit<0>(b, cc, ss);
                }
                if (st.mask & 2) {
                  g += gradx_bit<1, V, T>(a, b);
                  rx_bit<1>(a, cc, ss);
                  rx_bit<1>(b, cc, ss);
                }
                if (st.mask & 4) {
                  g += gradx_bit<2, V, T>(a, b);
                  rx_bit<2>(a, cc, ss);
                  rx_bit<2>(b, cc, ss);
                }
                if (st.mask & 8) {
                  g += gradx_bit<3, V, T>(a, b);
                  rx_bit<3>(a, cc, ss);
                  rx_bit<3>(b, cc, ss);
                }
              }
              break;
            }
            case QST_GRAD_COST: {
              // cost gradient C(x) Im(conj(lam) psi), then (optionally) cost^dag on both
              if (NS == 2) {
                const V* lut = lay + E1;
                T gq[4] = {0, 0, 0, 0};
#pragma unroll
                for (int j = 0; j < QRN; ++j) {
                  const int k = QCUT(j);
                  const T C = (T)(n_edges - 2 * k);
                  gq[j & 3] = qfma(C, qfma(b[j].x, a[j].y, -b[j].y * a[j].x), gq[j & 3]);
                  if (st.flags & QSF_LAM) {
                    const V d = lut[k];
                    a[j] = qcmul(d, a[j]);
                    b[j] = qcmul(d, b[j]);
                  }
                }
                g = (gq[0] + gq[1]) + (gq[2] + gq[3]);
              }
              break;
            }
            case QST_ENERGY: {
              T gq[4] = {0, 0, 0, 0};
#pragma unroll
              for (int j = 0; j < QRN; ++j) {
                const T C = (T)(n_edges - 2 * QCUT(j));
                gq[j & 3] = qfma(C, qfma(a[j].x, a[j].x, a[j].y * a[j].y), gq[j & 3]);
                b[j].x = C * a[j].x;
                b[j].y = C * a[j].y;
              }
              g = (gq[0] + gq[1]) + (gq[2] + gq[3]);
              break;
            }
            default:
              break;
          }
          if (st.type >= QST_GRAD_RX) {
#pragma unroll
            for (int k = 0; k < kQaoaMaxAcc; ++k)
              if (k == st.acc) acc[k] += g;
          }
        }
#undef QCUT
#pragma unroll
        for (int j = 0; j < QRN; ++j) {
          const uint32_t p = QPOS(j);
          bp[p] = a[j];
          if (NS == 2) bl[p] = b[j];
        }
#undef QPOS
#undef QLOC
      }
      __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < kQaoaMaxAcc; ++k)
      if (k < n_acc) acc_add(acc_hi[k], acc_lo[k], acc[k]);

    // ---------------------------------------------------------------- store
    if (flags & (PF_STORE_PSI | PF_STORE_LAM)) {
      const uint64_t gb = tile_offset(P, tile) | A.gt;
      using C16 = typename std::conditional<C64, float4, double2>::type;
      for (uint32_t k = 0; k < nk; ++k) {
        const uint64_t g = gb | s_gk[k];
        const uint32_t p = A.pt ^ s_pk[k];
        if (flags & PF_STORE_PSI) __stcs(reinterpret_cast<C16*>(g_psi + g), *reinterpret_cast<const C16*>(bp + p));
        if (NS == 2 && (flags & PF_STORE_LAM))
          __stcs(reinterpret_cast<C16*>(g_lam + g), *reinterpret_cast<const C16*>(bl + p));
      }
      if (nk == 0) {  // tiles smaller than one chunk per thread
        const uint64_t toff = tile_offset(P, tile);
        for (uint32_t ch = tid; ch < tile_n / EPC; ch += kTileThreads) {
          const uint32_t l = ch * EPC;
          const uint64_t g = toff | local_to_global(P, l);
          const uint32_t p = qaoa_swizzle(C64, l);
          if (flags & PF_STORE_PSI)
            __stcs(reinterpret_cast<C16*>(g_psi + g), *reinterpret_cast<const C16*>(bp + p));
          if (NS == 2 && (flags & PF_STORE_LAM))
            __stcs(reinterpret_cast<C16*>(g_lam + g), *reinterpret_cast<const C16*>(bl + p));
        }
      }
    }
    if (C64 && NS == 2 && (flags & PF_STORE_IL)) {
      // hand psi and lam to the reverse sweep interleaved per amplitude
      uint64_t toff = 0;
      for (int i = 0; i < P.ncomp; ++i) toff |= ((tile >> i) & 1ull) << P.comp[i];
      for (uint32_t l = tid; l < tile_n; l += kTileThreads) {
        const uint64_t g = toff | (l & lowmask) | P.hiA[(l >> c) & 63] | P.hiB[(l >> (c + 6)) & 63];
        const uint32_t p = qaoa_swizzle(true, l);
        const V x = bp[p], y = bl[p];
        float4* dst = g < args.il_half ? args.il0 + g : args.il1 + (g - args.il_half);
        __stcs(dst, make_float4((float)x.x, (float)y.x, (float)x.y, (float)y.y));
      }
    }
    __syncthreads();  // this buffer is refilled by the copies issued in the next iteration
  }
  cp_async_wait1();
#pragma unroll
  for (int k = 0; k < kQaoaMaxAcc; ++k) s_accd[k * kTileThreads + tid] = (double)acc_hi[k] + (double)acc_lo[k];

  // ------------------------------------------------------------------ per-CTA reduction, fixed order
  const int lane = tid & 31, warp = tid >> 5;
  for (int k = 0; k < P.n_acc; ++k) {
    double v = s_accd[k * kTileThreads + tid];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) s_red[warp] = v;
    __syncthreads();
    if (tid == 0) {
      double s = 0;
      for (int w = 0; w < kTileWarps; ++w) s += s_red[w];
      args.partials[(size_t)(P.slot_base + k) * args.stride + blockIdx.x] = s;
    }
    __syncthreads();
  }
}

// ============================================================================
// complex64 reverse passes on the interleaved (psi, lam) buffer.  A 16-byte
// shared-memory element (psi.re, lam.re, psi.im, lam.im) gives the packed
// operands RE = (psi.re, lam.re) and IM = (psi.im, lam.im) in one load, so
// RX^dag and cost^dag update both states with one f32x2 FMA per component.
// The gradient terms mix the two lanes and stay scalar.
// ============================================================================

template <int RB>
__device__ __forceinline__ void rx2_bit(float2 (&RE)[QRN], float2 (&IM)[QRN], float2 c2, float2 s2, float2 ms2) {
#pragma unroll
  for (int j = 0; j < QRN; ++j) {
    if (j & (1 << RB)) continue;
    const int j1 = j | (1 << RB);
    const float2 r0 = RE[j], i0 = IM[j], r1 = RE[j1], i1 = IM[j1];
    RE[j] = __ffma2_rn(c2, r0, __fmul2_rn(s2, i1));   // c re0 + s im1
    IM[j] = __ffma2_rn(c2, i0, __fmul2_rn(ms2, r1));  // c im0 - s re1
    RE[j1] = __ffma2_rn(c2, r1, __fmul2_rn(s2, i0));
    IM[j1] = __ffma2_rn(c2, i1, __fmul2_rn(ms2, r0));
  }
}

// Im <lam| X_RB |psi>: lam0.re psi1.im - lam0.im psi1.re + lam1.re psi0.im - lam1.im psi0.re
// (four independent partial sums: the FMA chains stay short)
template <int RB>
__device__ __forceinline__ float gradx2_bit(const float2 (&RE)[QRN], const float2 (&IM)[QRN]) {
  float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll
  for (int j = 0; j < QRN; ++j) {
    if (j & (1 << RB)) continue;
    const int j1 = j | (1 << RB);
    s0 = __fmaf_rn(RE[j].y, IM[j1].x, s0);
    s1 = __fmaf_rn(-IM[j].y, RE[j1].x, s1);
    s2 = __fmaf_rn(RE[j1].y, IM[j].x, s2);
    s3 = __fmaf_rn(-IM[j1].y, RE[j].x, s3);
  }
  return (s0 + s1) + (s2 + s3);
}

__device__ __forceinline__ void cmul2(float2 d, float2& RE, float2& IM) {
  const float2 dr = make_float2(d.x, d.x), di = make_float2(d.y, d.y), mdi = make_float2(-d.y, -d.y);
  const float2 r = RE, i = IM;
  RE = __ffma2_rn(dr, r, __fmul2_rn(mdi, i));
  IM = __ffma2_rn(dr, i, __fmul2_rn(di, r));
}

__device__ __forceinline__ const float4* il_src(const QArgs& args, uint64_t g) {
  return g < args.il_half ? args.il0 + g : args.il1 + (g - args.il_half);
}

__device__ __forceinline__ void issue_tile_il(const QPassDesc& P, uint64_t toff, const QArgs& args, const QAddr& A,
                                              const uint64_t* s_gk, const uint32_t* s_pk, float4* b_el,
                                              uint8_t* b_cut) {
  const uint32_t tile_n = 1u << P.m;
  const uint32_t nk = tile_n / kTileThreads;
  if (nk == 0) {
    for (uint32_t l = threadIdx.x; l < tile_n; l += blockDim.x)
      cp_async16(b_el + qaoa_swizzle(false, l), il_src(args, toff | local_to_global(P, l)));
  } else {
    const uint64_t gb = toff | A.gt;
    for (uint32_t k = 0; k < nk; ++k) cp_async16(b_el + (A.pt ^ s_pk[k]), il_src(args, gb | s_gk[k]));
  }
  if (P.flags & PF_NEED_CUT) issue_cut(P, toff, A, args.cut, b_cut);
}

// Tile buffers of the interleaved reverse kernel: one CTA per SM with the next
// kIlBufs - 1 tiles' copies in flight.  Measured at 30 qubits: 2 buffers 284 ms
// per evaluation in this kernel, 3 buffers 304 ms, and two single-buffered CTAs
// per SM at <= 128 registers 378 ms (spills, exposed load latency).
#ifndef QS_IL_NBUF
#define QS_IL_NBUF 2
#endif
constexpr int kIlBufs = QS_IL_NBUF;

template <int N>
__device__ __forceinline__ void cp_async_wait_n() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__global__ void __launch_bounds__(kTileThreads, 1) qaoa_il_kernel(QArgs args) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ QPassDesc P;
  {
    const int* src = reinterpret_cast<const int*>(args.pass);
    int* dst = reinterpret_cast<int*>(&P);
    for (int i = threadIdx.x; i < (int)(sizeof(QPassDesc) / 4); i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  const int E1 = args.n_edges + 1;
  const int per_layer = 2 * E1 + 2;
  const int n_coef = per_layer * kQaoaMaxLayersPerPass;
  float2* s_coef = reinterpret_cast<float2*>(smem);
  {
    const float2* g = reinterpret_cast<const float2*>(args.coef) + (size_t)P.layer_lo * per_layer;
    const int nc = per_layer * P.n_layers;
    for (int i = threadIdx.x; i < nc; i += blockDim.x) s_coef[i] = g[i];
  }
  const int m = P.m;
  const uint32_t flags = P.flags;
  const uint32_t tile_n = 1u << m;
  unsigned char* base = smem + ((n_coef * sizeof(float2) + 127) & ~(size_t)127);
  const size_t buf_bytes = ((size_t)tile_n * 16 + tile_n + 127) & ~(size_t)127;
  auto buf_el = [&](int b) { return reinterpret_cast<float4*>(base + b * buf_bytes); };
  auto buf_cut = [&](int b) { return reinterpret_cast<uint8_t*>(buf_el(b) + tile_n); };
  double* s_red = reinterpret_cast<double*>(base + kIlBufs * buf_bytes);
  double* s_accd = s_red + kTileWarps;
  uint32_t* s_base = reinterpret_cast<uint32_t*>(s_accd + kQaoaMaxAcc * kTileThreads);

  const int tid = threadIdx.x;
  const uint64_t n_tiles = 1ull << (args.n - m);
  const int n_edges = args.n_edges;

  const uint32_t nsub = tile_n >> 4;
  for (int ph = 0; ph < P.n_phases; ++ph) {
    const QPhase& PH = P.phases[ph];
    for (uint32_t u = tid; u < nsub; u += blockDim.x) {
      uint32_t p0 = 0, l0 = 0;
      for (int i = 0; i < PH.nq; ++i)
        if ((u >> i) & 1u) {
          p0 ^= PH.sq[i];
          l0 |= 1u << PH.Q[i];
        }
      s_base[ph * nsub + u] = (l0 << 16) | p0;
    }
  }
  __shared__ uint64_t s_gk[16];
  __shared__ uint32_t s_pk[16];
  const QAddr A = make_addr(P, 1, false, s_gk, s_pk);
  const uint32_t nk = tile_n / kTileThreads;
  __syncthreads();
  float acc_hi[kQaoaMaxAcc] = {0.f, 0.f, 0.f, 0.f}, acc_lo[kQaoaMaxAcc] = {0.f, 0.f, 0.f, 0.f};
  const int n_acc = P.n_acc;

  // ring of kIlBufs buffers: tile it + j lives in buffer (it + j) % kIlBufs
  uint64_t tile = blockIdx.x;
#pragma unroll
  for (int j = 0; j < kIlBufs - 1; ++j) {
    const uint64_t t = tile + (uint64_t)j * gridDim.x;
    if (t < n_tiles) issue_tile_il(P, tile_offset(P, t), args, A, s_gk, s_pk, buf_el(j), buf_cut(j));
    cp_async_commit();
  }
  for (int it = 0; tile < n_tiles; ++it, tile += gridDim.x) {
    const int cur = it % kIlBufs;
    {
      const uint64_t t = tile + (uint64_t)(kIlBufs - 1) * gridDim.x;
      const int b = (it + kIlBufs - 1) % kIlBufs;
      if (t < n_tiles) issue_tile_il(P, tile_offset(P, t), args, A, s_gk, s_pk, buf_el(b), buf_cut(b));
      cp_async_commit();
    }
    cp_async_wait_n<kIlBufs - 1>();  // this tile's copies have landed
    __syncthreads();
    float4* const be = buf_el(cur);
    const uint8_t* const bc = buf_cut(cur);

    float acc[kQaoaMaxAcc] = {0.f, 0.f, 0.f, 0.f};
    for (int ph = 0; ph < P.n_phases; ++ph) {
      const QPhase& PH = P.phases[ph];
      const uint32_t s0 = PH.sreg[0], s1 = PH.sreg[1], s2 = PH.sreg[2], s3 = PH.sreg[3];
      const uint32_t r0 = 1u << PH.R[0], r1 = 1u << PH.R[1], r2 = 1u << PH.R[2], r3 = 1u << PH.R[3];
      const bool ph_cut = PH.need_cut;
      for (uint32_t u = tid; u < nsub; u += kTileThreads) {
        const uint32_t bw = s_base[ph * nsub + u];
        const uint32_t p0 = bw & 0xffffu, l0 = bw >> 16;
#define QPOS(j) \
  (p0 ^ (((j) & 1) ? s0 : 0u) ^ (((j) & 2) ? s1 : 0u) ^ (((j) & 4) ? s2 : 0u) ^ (((j) & 8) ? s3 : 0u))
#define QLOC(j) \
  (l0 | (((j) & 1) ? r0 : 0u) | (((j) & 2) ? r1 : 0u) | (((j) & 4) ? r2 : 0u) | (((j) & 8) ? r3 : 0u))
        uint32_t cw[QRN / 4] = {0, 0, 0, 0};
        float2 RE[QRN], IM[QRN];
#pragma unroll
        for (int j = 0; j < QRN; ++j) {
          const float4 e = be[QPOS(j)];
          RE[j] = make_float2(e.x, e.y);
          IM[j] = make_float2(e.z, e.w);
          if (ph_cut) cw[j >> 2] |= (uint32_t)bc[QLOC(j)] << (8 * (j & 3));
        }
#define QCUT(j) ((int)((cw[(j) >> 2] >> (8 * ((j) & 3))) & 255u))
        for (int si = 0; si < PH.n_steps; ++si) {
          const QStep st = PH.steps[si];
          const float2* lay = s_coef + st.layer * per_layer;
          float g = 0.f;
          if (st.type == QST_GRAD_RX) {
            const float2 cs = lay[2 * E1 + 1];
            const float2 c2 = make_float2(cs.x, cs.x), sv = make_float2(cs.y, cs.y), ms2 = make_float2(-cs.y, -cs.y);
            if (st.mask & 1) {
              g += gradx2_bit<0>(RE, IM);
              rx2_bit<0>(RE, IM, c2, sv, ms2);
            }
            if (st.mask & 2) {
              g += gradx2_bit<1>(RE, IM);
              rx2_bit<1>(RE, IM, c2, sv, ms2);
            }
            if (st.mask & 4) {
              g += gradx2_bit<2>(RE, IM);
              rx2_bit<2>(RE, IM, c2, sv, ms2);
            }
            if (st.mask & 8) {
              g += gradx2_bit<3>(RE, IM);
              rx2_bit<3>(RE, IM, c2, sv, ms2);
            }
          } else if (st.type == QST_GRAD_COST) {
            const float2* lut = lay + E1;
            float gq[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int j = 0; j < QRN; ++j) {
              const int k = QCUT(j);
              const float C = (float)(n_edges - 2 * k);
              gq[j & 3] = __fmaf_rn(C, __fmaf_rn(RE[j].y, IM[j].x, -IM[j].y * RE[j].x), gq[j & 3]);
              if (st.flags & QSF_LAM) cmul2(lut[k], RE[j], IM[j]);
            }
            g = (gq[0] + gq[1]) + (gq[2] + gq[3]);
          }
#pragma unroll
          for (int k = 0; k < kQaoaMaxAcc; ++k)
            if (k == st.acc) acc[k] += g;
        }
#undef QCUT
#pragma unroll
        for (int j = 0; j < QRN; ++j) be[QPOS(j)] = make_float4(RE[j].x, RE[j].y, IM[j].x, IM[j].y);
#undef QPOS
#undef QLOC
      }
      __syncthreads();
    }
#pragma unroll
    for (int k = 0; k < kQaoaMaxAcc; ++k)
      if (k < n_acc) acc_add(acc_hi[k], acc_lo[k], acc[k]);

    if (flags & PF_STORE_IL) {
      const uint64_t toff = tile_offset(P, tile);
      if (nk == 0) {
        for (uint32_t l = tid; l < tile_n; l += kTileThreads)
          __stcs(const_cast<float4*>(il_src(args, toff | local_to_global(P, l))), be[qaoa_swizzle(false, l)]);
      } else {
        const uint64_t gb = toff | A.gt;
        for (uint32_t k = 0; k < nk; ++k)
          __stcs(const_cast<float4*>(il_src(args, gb | s_gk[k])), be[A.pt ^ s_pk[k]]);
      }
    }
    __syncthreads();
  }
  cp_async_wait0();
#pragma unroll
  for (int k = 0; k < kQaoaMaxAcc; ++k) s_accd[k * kTileThreads + tid] = (double)acc_hi[k] + (double)acc_lo[k];

  const int lane = tid & 31, warp = tid >> 5;
  for (int k = 0; k < P.n_acc; ++k) {
    double v = s_accd[k * kTileThreads + tid];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) s_red[warp] = v;
    __syncthreads();
    if (tid == 0) {
      double s = 0;
      for (int w = 0; w < kTileWarps; ++w) s += s_red[w];
      args.partials[(size_t)(P.slot_base + k) * args.stride + blockIdx.x] = s;
    }
    __syncthreads();
  }
}

size_t qaoa_il_smem_bytes(int m, int n_edges) {
  const size_t coef = ((size_t)(2 * (n_edges + 1) + 2) * kQaoaMaxLayersPerPass * 8 + 127) & ~(size_t)127;
  const size_t tile = (size_t)1 << m;
  const size_t buf = (tile * 16 + tile + 127) & ~(size_t)127;
  return coef + kIlBufs * buf + kTileWarps * 8 + (size_t)kQaoaMaxAcc * kTileThreads * 8 +
         (size_t)kQaoaMaxPhases * (tile >> 4) * 4;
}

int qaoa_il_occupancy(size_t smem) {
  static size_t last = 0;
  static int occ = 0;
  if (last == smem) return occ;
  int blocks = 0;
  if (cudaFuncSetAttribute(qaoa_il_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, qaoa_il_kernel, kTileThreads, smem) != cudaSuccess ||
      blocks < 1) {
    (void)cudaGetLastError();
    blocks = 0;
  }
  last = smem;
  occ = blocks;
  return blocks;
}

template <class T, int NS>
const void* kernel_ptr() {
  return (const void*)qaoa_pass_kernel<T, NS>;
}

const void* qaoa_kernel_of(qs_dtype dt, int ns) {
  if (dt == QS_C64) return ns == 2 ? kernel_ptr<float, 2>() : kernel_ptr<float, 1>();
  return ns == 2 ? kernel_ptr<double, 2>() : kernel_ptr<double, 1>();
}

// Allow `smem` dynamic shared memory and return the resident CTAs per SM (0 if it does not fit).
int qaoa_occupancy(qs_dtype dt, int ns, size_t smem) {
  static size_t last[4] = {0, 0, 0, 0};
  static int occ[4] = {0, 0, 0, 0};
  const int key = (dt == QS_C64 ? 0 : 2) + (ns == 2 ? 1 : 0);
  if (last[key] == smem) return occ[key];
  const void* fn = qaoa_kernel_of(dt, ns);
  int blocks = 0;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fn, kTileThreads, smem) != cudaSuccess || blocks < 1) {
    (void)cudaGetLastError();
    blocks = 0;
  }
  last[key] = smem;
  occ[key] = blocks;
  return blocks;
}

}  // namespace

size_t qaoa_smem_bytes(qs_dtype dt, int m, int ns, int n_edges) {
  const size_t amp = dt == QS_C64 ? 8 : 16;
  const size_t coef = ((size_t)(2 * (n_edges + 1) + 2) * kQaoaMaxLayersPerPass * amp + 127) & ~(size_t)127;
  const size_t tile = (size_t)1 << m;
  const size_t buf = (ns * tile * amp + tile + 127) & ~(size_t)127;
  return coef + 2 * buf + kTileWarps * 8 + (size_t)kQaoaMaxAcc * kTileThreads * 8 +
         (size_t)kQaoaMaxPhases * (tile >> 4) * 4;
}

int qaoa_grid_size(qs_dtype dt, int m, int ns, int n_edges, uint64_t n_tiles) {
  const size_t smem = qaoa_smem_bytes(dt, m, ns, n_edges);
  const int occ = qaoa_occupancy(dt, ns, smem);
  if (occ < 1) return 0;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  uint64_t g = (uint64_t)(sms > 0 ? sms : 1) * occ;
  if (g > n_tiles) g = n_tiles;
  return (int)(g < 1 ? 1 : g);
}

int qaoa_il_grid_size(int m, int n_edges, uint64_t n_tiles) {
  const int occ = qaoa_il_occupancy(qaoa_il_smem_bytes(m, n_edges));
  if (occ < 1) return 0;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  uint64_t g = (uint64_t)(sms > 0 ? sms : 1) * occ;
  if (g > n_tiles) g = n_tiles;
  return (int)(g < 1 ? 1 : g);
}

qs_status launch_qaoa_pass(qs_dtype dt, const QPassDesc* d_pass, int ns, int m, uint32_t flags,
                           const QaoaLaunch& L, cudaStream_t st) {
  QArgs a;
  a.il0 = reinterpret_cast<float4*>(L.il[0]);
  a.il1 = reinterpret_cast<float4*>(L.il[1]);
  a.il_half = 1ull << (L.n - 1);
  a.psi = L.psi;
  a.lam = L.lam;
  a.pass = d_pass;
  a.coef = L.coef;
  a.cut = L.cut;
  a.partials = L.partials;
  a.n = L.n;
  a.n_edges = L.n_edges;
  a.stride = L.stride;
  if (flags & PF_LOAD_IL) {
    const size_t smem = qaoa_il_smem_bytes(m, L.n_edges);
    if (dt != QS_C64 || qaoa_il_occupancy(smem) < 1) {
      set_error("qaoa: the interleaved tile does not fit in shared memory");
      return QS_ERR_UNSUPPORTED;
    }
    qaoa_il_kernel<<<L.grid, kTileThreads, smem, st>>>(a);
    QS_CUDA(cudaGetLastError());
    return QS_OK;
  }
  const size_t smem = qaoa_smem_bytes(dt, m, ns, L.n_edges);
  if (qaoa_occupancy(dt, ns, smem) < 1) {
    set_error("qaoa: the tile does not fit in shared memory");
    return QS_ERR_UNSUPPORTED;
  }
  if (dt == QS_C64) {
    if (ns == 2)
      qaoa_pass_kernel<float, 2><<<L.grid, kTileThreads, smem, st>>>(a);
    else
      qaoa_pass_kernel<float, 1><<<L.grid, kTileThreads, smem, st>>>(a);
  } else {
    if (ns == 2)
      qaoa_pass_kernel<double, 2><<<L.grid, kTileThreads, smem, st>>>(a);
    else
      qaoa_pass_kernel<double, 1><<<L.grid, kTileThreads, smem, st>>>(a);
  }
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

}  // namespace qs
