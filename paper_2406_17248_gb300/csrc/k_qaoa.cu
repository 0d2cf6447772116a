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
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

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
template <int RB, class V, class T>
__device__ __forceinline__ T gradx_bit(const V (&a)[QRN], const V (&b)[QRN]) {
  T acc = 0;
#pragma unroll
  for (int j = 0; j < QRN; ++j) {
    if (j & (1 << RB)) continue;
    const int j1 = j | (1 << RB);
    acc = qfma(b[j].x, a[j1].y, acc);
    acc = qfma(-b[j].y, a[j1].x, acc);
    acc = qfma(b[j1].x, a[j].y, acc);
    acc = qfma(-b[j1].y, a[j].x, acc);
  }
  return acc;
}

template <class V>
__device__ __forceinline__ V qcmul(V d, V a) {
  V r;
  r.x = qfma(d.x, a.x, -d.y * a.y);
  r.y = qfma(d.x, a.y, d.y * a.x);
  return r;
}

struct QArgs {
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

// Issue the asynchronous copies of one tile (psi, lam, cut) into one buffer.
template <class T, int NS>
__device__ __forceinline__ void issue_tile(const QPassDesc& P, uint64_t tile, const QArgs& args,
                                           typename QV<T>::V* b_psi, typename QV<T>::V* b_lam, uint8_t* b_cut) {
  using V = typename QV<T>::V;
  const int m = P.m, c = P.c;
  const uint32_t flags = P.flags;
  const uint32_t tile_n = 1u << m;
  const uint32_t lowmask = (1u << c) - 1u;
  uint64_t toff = 0;
  for (int i = 0; i < P.ncomp; ++i) toff |= ((tile >> i) & 1ull) << P.comp[i];
  constexpr int EPC = sizeof(T) == 4 ? 2 : 1;  // amplitudes per 16-byte chunk
  const V* g_psi = reinterpret_cast<const V*>(args.psi);
  const V* g_lam = reinterpret_cast<const V*>(args.lam);
  const bool ld_psi = flags & PF_LOAD_PSI;
  const bool ld_lam = NS == 2 && (flags & PF_LOAD_LAM);
  if (ld_psi || ld_lam) {
    for (uint32_t ch = threadIdx.x; ch < tile_n / EPC; ch += blockDim.x) {
      const uint32_t l = ch * EPC;
      const uint64_t g = toff | (l & lowmask) | P.hiA[(l >> c) & 63] | P.hiB[(l >> (c + 6)) & 63];
      const uint32_t p = qaoa_swizzle(sizeof(T) == 4, l);
      if (ld_psi) cp_async16(b_psi + p, g_psi + g);
      if (ld_lam) cp_async16(b_lam + p, g_lam + g);
    }
  }
  if (flags & PF_NEED_CUT) {
    // cut values in local-index order, in runs of min(2^c, 16) contiguous bytes
    if (c >= 4) {
      for (uint32_t k = threadIdx.x; k < (tile_n >> 4); k += blockDim.x) {
        const uint32_t l = k << 4;
        const uint64_t g = toff | (l & lowmask) | P.hiA[(l >> c) & 63] | P.hiB[(l >> (c + 6)) & 63];
        cp_async16(b_cut + l, args.cut + g);
      }
    } else if (c == 3) {
      for (uint32_t k = threadIdx.x; k < (tile_n >> 3); k += blockDim.x) {
        const uint32_t l = k << 3;
        const uint64_t g = toff | P.hiA[(l >> c) & 63] | P.hiB[(l >> (c + 6)) & 63];
        cp_async8(b_cut + l, args.cut + g);
      }
    } else {
      const uint32_t run = 1u << c;  // 2 or 4 bytes
      for (uint32_t k = threadIdx.x; k < (tile_n >> 2); k += blockDim.x) {
        const uint32_t l = k << 2;
        if (run == 4) {
          const uint64_t g = toff | P.hiA[(l >> c) & 63] | P.hiB[(l >> (c + 6)) & 63];
          cp_async4(b_cut + l, args.cut + g);
        } else {
          for (int e = 0; e < 4; ++e) {
            const uint32_t le = l + e;
            const uint64_t g = toff | (le & lowmask) | P.hiA[(le >> c) & 63] | P.hiB[(le >> (c + 6)) & 63];
            b_cut[le] = args.cut[g];
          }
        }
      }
    }
  }
}

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

  for (int k = 0; k < kQaoaMaxAcc; ++k) s_accd[k * kTileThreads + tid] = 0.0;
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
  __syncthreads();

  uint64_t tile = blockIdx.x;
  if (tile < n_tiles) issue_tile<T, NS>(P, tile, args, buf_psi(0), buf_lam(0), buf_cut(0));
  cp_async_commit();
  for (int it = 0; tile < n_tiles; ++it, tile += gridDim.x) {
    const int cur = it & 1;
    const uint64_t next = tile + gridDim.x;
    if (next < n_tiles) issue_tile<T, NS>(P, next, args, buf_psi(cur ^ 1), buf_lam(cur ^ 1), buf_cut(cur ^ 1));
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
#pragma unroll
                for (int j = 0; j < QRN; ++j) {
                  const int k = QCUT(j);
                  const T C = (T)(n_edges - 2 * k);
                  g = qfma(C, qfma(b[j].x, a[j].y, -b[j].y * a[j].x), g);
                  if (st.flags & QSF_LAM) {
                    const V d = lut[k];
                    a[j] = qcmul(d, a[j]);
                    b[j] = qcmul(d, b[j]);
                  }
                }
              }
              break;
            }
            case QST_ENERGY: {
#pragma unroll
              for (int j = 0; j < QRN; ++j) {
                const T C = (T)(n_edges - 2 * QCUT(j));
                g = qfma(C, qfma(a[j].x, a[j].x, a[j].y * a[j].y), g);
                b[j].x = C * a[j].x;
                b[j].y = C * a[j].y;
              }
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
    for (int k = 0; k < kQaoaMaxAcc; ++k) s_accd[k * kTileThreads + tid] += (double)acc[k];

    // ---------------------------------------------------------------- store
    if (flags & (PF_STORE_PSI | PF_STORE_LAM)) {
      uint64_t toff = 0;
      for (int i = 0; i < P.ncomp; ++i) toff |= ((tile >> i) & 1ull) << P.comp[i];
      constexpr int EPC = C64 ? 2 : 1;
      using C16 = typename std::conditional<C64, float4, double2>::type;
      for (uint32_t ch = tid; ch < tile_n / EPC; ch += kTileThreads) {
        const uint32_t l = ch * EPC;
        const uint64_t g = toff | (l & lowmask) | P.hiA[(l >> c) & 63] | P.hiB[(l >> (c + 6)) & 63];
        const uint32_t p = qaoa_swizzle(C64, l);
        if (flags & PF_STORE_PSI) __stcs(reinterpret_cast<C16*>(g_psi + g), *reinterpret_cast<const C16*>(bp + p));
        if (NS == 2 && (flags & PF_STORE_LAM))
          __stcs(reinterpret_cast<C16*>(g_lam + g), *reinterpret_cast<const C16*>(bl + p));
      }
    }
    __syncthreads();  // this buffer is refilled by the copies issued in the next iteration
  }
  cp_async_wait1();

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

qs_status launch_qaoa_pass(qs_dtype dt, const QPassDesc* d_pass, int ns, int m, const QaoaLaunch& L,
                           cudaStream_t st) {
  QArgs a;
  a.psi = L.psi;
  a.lam = L.lam;
  a.pass = d_pass;
  a.coef = L.coef;
  a.cut = L.cut;
  a.partials = L.partials;
  a.n = L.n;
  a.n_edges = L.n_edges;
  a.stride = L.stride;
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
