// Batched persistent engine: thousands of small, independent variational
// instances (the encoder batch of §4.1, here each with its own circuit,
// Hamiltonian and parameters) evaluated in ONE launch.  CTAs pull instances
// from an atomic work queue ordered by decreasing cost; an instance is owned by
// one CTA from start to finish: psi = U|0>, E = <psi|H|psi>, lam = H psi, then
// the adjoint sweep (the gradient rule of §4.1 / §7.2) gate by gate, with psi
// and lam in the CTA's shared memory.  (Instances too large for shared memory
// run on fused tile passes, see batch.cu.)  Gate matrices are formed on the
// device from the angle (the definitions of §2.3.2 / §2.3.3); every reduction
// has a fixed order.
#include <cmath>

#include "batch.h"

namespace qs {

namespace {

template <class T>
struct BV;
template <>
struct BV<float> {
  using V = float2;
};
template <>
struct BV<double> {
  using V = double2;
};

template <class V>
__device__ __forceinline__ V bmul(V a, V b) {
  V r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
template <class V>
__device__ __forceinline__ V badd(V a, V b) {
  a.x += b.x;
  a.y += b.y;
  return a;
}
template <class V, class T>
__device__ __forceinline__ V bmk(T re, T im) {
  V v;
  v.x = re;
  v.y = im;
  return v;
}
// Re(conj(a) b)
template <class V>
__device__ __forceinline__ auto bre(V a, V b) -> decltype(a.x) {
  return a.x * b.x + a.y * b.y;
}

__device__ __forceinline__ void bsincos(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ __forceinline__ void bsincos(double x, double* s, double* c) { sincos(x, s, c); }

__device__ __forceinline__ uint64_t bins0(uint64_t i, int q) {
  return ((i >> q) << (q + 1)) | (i & ((1ull << q) - 1));
}

constexpr int kMaxBatchWarps = kBatchThreads / 32;

// Gate classes (what the kernel does with the matrix)
__device__ __forceinline__ bool bdiag(int k) {
  return k == QS_GATE_I || k == QS_GATE_Z || k == QS_GATE_S || k == QS_GATE_SDG || k == QS_GATE_T ||
         k == QS_GATE_TDG || k == QS_GATE_RZ || k == QS_GATE_PS || k == QS_GATE_RZZ;
}

// U of a gate (row-major, basis index bit(t0) + 2 bit(t1)); dim 2 or 4.
template <class V, class T>
__device__ void bgate_matrix(int kind, T th, V (&U)[16]) {
  T s, c;
  bsincos(th * (T)0.5, &s, &c);
  const T r2 = (T)0.70710678118654752440;
  for (int i = 0; i < 16; ++i) U[i] = bmk<V, T>(0, 0);
  switch (kind) {
    case QS_GATE_I: U[0] = U[3] = bmk<V, T>(1, 0); break;
    case QS_GATE_X: U[1] = U[2] = bmk<V, T>(1, 0); break;
    case QS_GATE_Y: U[1] = bmk<V, T>(0, -1); U[2] = bmk<V, T>(0, 1); break;
    case QS_GATE_Z: U[0] = bmk<V, T>(1, 0); U[3] = bmk<V, T>(-1, 0); break;
    case QS_GATE_H: U[0] = U[1] = U[2] = bmk<V, T>(r2, 0); U[3] = bmk<V, T>(-r2, 0); break;
    case QS_GATE_S: U[0] = bmk<V, T>(1, 0); U[3] = bmk<V, T>(0, 1); break;
    case QS_GATE_SDG: U[0] = bmk<V, T>(1, 0); U[3] = bmk<V, T>(0, -1); break;
    case QS_GATE_T: U[0] = bmk<V, T>(1, 0); U[3] = bmk<V, T>(r2, r2); break;
    case QS_GATE_TDG: U[0] = bmk<V, T>(1, 0); U[3] = bmk<V, T>(r2, -r2); break;
    case QS_GATE_RX: U[0] = U[3] = bmk<V, T>(c, 0); U[1] = U[2] = bmk<V, T>(0, -s); break;
    case QS_GATE_RY: U[0] = U[3] = bmk<V, T>(c, 0); U[1] = bmk<V, T>(-s, 0); U[2] = bmk<V, T>(s, 0); break;
    case QS_GATE_RZ: U[0] = bmk<V, T>(c, -s); U[3] = bmk<V, T>(c, s); break;
    case QS_GATE_PS: {
      T s2, c2;
      bsincos(th, &s2, &c2);
      U[0] = bmk<V, T>(1, 0);
      U[3] = bmk<V, T>(c2, s2);
      break;
    }
    case QS_GATE_SWAP: U[0] = U[6] = U[9] = U[15] = bmk<V, T>(1, 0); break;
    case QS_GATE_RXX:
      for (int b = 0; b < 4; ++b) {
        U[b * 5] = bmk<V, T>(c, 0);
        U[b * 4 + 3 - b] = bmk<V, T>(0, -s);
      }
      break;
    case QS_GATE_RYY:
      for (int b = 0; b < 4; ++b) U[b * 5] = bmk<V, T>(c, 0);
      U[3] = bmk<V, T>(0, s);
      U[6] = bmk<V, T>(0, -s);
      U[9] = bmk<V, T>(0, -s);
      U[12] = bmk<V, T>(0, s);
      break;
    case QS_GATE_RZZ:
      U[0] = U[15] = bmk<V, T>(c, -s);
      U[5] = U[10] = bmk<V, T>(c, s);
      break;
    default: break;
  }
}

// A = (dU/dtheta) U^dag of the parametric gates: -i P / 2 for the rotations,
// diag(0, i) for PS (independent of the angle).
template <class V, class T>
__device__ void bgate_generator(int kind, V (&A)[16]) {
  for (int i = 0; i < 16; ++i) A[i] = bmk<V, T>(0, 0);
  const T h = (T)0.5;
  switch (kind) {
    case QS_GATE_RX: A[1] = A[2] = bmk<V, T>(0, -h); break;
    case QS_GATE_RY: A[1] = bmk<V, T>(-h, 0); A[2] = bmk<V, T>(h, 0); break;
    case QS_GATE_RZ: A[0] = bmk<V, T>(0, -h); A[3] = bmk<V, T>(0, h); break;
    case QS_GATE_PS: A[3] = bmk<V, T>(0, 1); break;
    case QS_GATE_RXX:
      for (int b = 0; b < 4; ++b) A[b * 4 + 3 - b] = bmk<V, T>(0, -h);
      break;
    case QS_GATE_RYY:  // -i/2 Y(x)Y
      A[3] = bmk<V, T>(0, h);
      A[6] = bmk<V, T>(0, -h);
      A[9] = bmk<V, T>(0, -h);
      A[12] = bmk<V, T>(0, h);
      break;
    case QS_GATE_RZZ:
      A[0] = A[15] = bmk<V, T>(0, -h);
      A[5] = A[10] = bmk<V, T>(0, h);
      break;
    default: break;
  }
}

// ---------------------------------------------------------------- reductions

template <class T>
__device__ __forceinline__ T wsum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Fixed-order block sum, FP64 across warps (all threads get the result).
template <class T>
__device__ double bsum_all(T v, double* sh) {
  v = wsum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = (double)v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[i];
    sh[kMaxBatchWarps] = s;
  }
  __syncthreads();
  return sh[kMaxBatchWarps];
}

// ------------------------------------------------------- gate data and apply

// Four complex numbers per gate, formed once from the angle and kept in shared
// memory: single-qubit dense gates their 2x2 (row-major), diagonal gates their
// diagonal (two entries, four for RZZ), RXX / RYY (cos, sin) of the half angle;
// SWAP and channel sites need none.
template <class V, class T>
__device__ void form_gate(const BGate& g, const double* params, V* out) {
  if (g.kind == kGateChannel || g.kind == QS_GATE_SWAP) return;
  const double th = g.param < 0 ? g.constant : g.constant + g.coef * params[g.param];
  if (g.kind == QS_GATE_RXX || g.kind == QS_GATE_RYY) {
    T s, c;
    bsincos((T)th * (T)0.5, &s, &c);
    out[0] = bmk<V, T>(c, s);
    return;
  }
  V U[16];
  bgate_matrix<V, T>(g.kind, (T)th, U);
  if (g.kind == QS_GATE_RZZ) {
    out[0] = U[0];
    out[1] = U[5];
    out[2] = U[10];
    out[3] = U[15];
  } else if (bdiag(g.kind)) {
    out[0] = U[0];
    out[1] = U[3];
  } else {
    for (int e = 0; e < 4; ++e) out[e] = U[e];
  }
}

template <class V, class T>
__device__ void form_gates(const BGate* gates, int begin, int end, const double* params, V* s_gd) {
  for (int i = begin + (int)threadIdx.x; i < end; i += blockDim.x) form_gate<V, T>(gates[i], params, s_gd + 4 * (i - begin));
}

template <class V>
__device__ __forceinline__ V bconj(V a) {
  a.y = -a.y;
  return a;
}
// Im(conj(l) a)
template <class V>
__device__ __forceinline__ auto bim(V l, V a) -> decltype(a.x) {
  return l.x * a.y - l.y * a.x;
}
// -i s x and +i s x
template <class V, class T>
__device__ __forceinline__ V mis(T s, V x) {
  return bmk<V, T>(s * x.y, -s * x.x);
}
template <class V, class T>
__device__ __forceinline__ V pis(T s, V x) {
  return bmk<V, T>(-s * x.y, s * x.x);
}

// psi <- M psi on qubit q where the control mask cm is set (with BOTH, lam too).
template <class T, bool BOTH>
__device__ __forceinline__ void apply_1q(typename BV<T>::V* psi, typename BV<T>::V* lam, int n, int q, uint64_t cm,
                                         typename BV<T>::V m00, typename BV<T>::V m01, typename BV<T>::V m10,
                                         typename BV<T>::V m11) {
  const uint64_t P = 1ull << (n - 1);
  for (uint64_t i = threadIdx.x; i < P; i += blockDim.x) {
    const uint64_t x0 = bins0(i, q);
    if ((x0 & cm) != cm) continue;
    const uint64_t x1 = x0 | (1ull << q);
    const auto a0 = psi[x0], a1 = psi[x1];
    psi[x0] = badd(bmul(m00, a0), bmul(m01, a1));
    psi[x1] = badd(bmul(m10, a0), bmul(m11, a1));
    if (BOTH) {
      const auto l0 = lam[x0], l1 = lam[x1];
      lam[x0] = badd(bmul(m00, l0), bmul(m01, l1));
      lam[x1] = badd(bmul(m10, l0), bmul(m11, l1));
    }
  }
}

// Apply gate g (DAG: its adjoint) to psi, with BOTH also to lam; with GRAD first
// return this thread's share of 2 Re <lam|A|psi>, A = (dU/dtheta) U^dag on the
// control subspace, written out per kind: RX Im(l0* a1 + l1* a0), RY
// Re(l1* a0 - l0* a1), RZ +-Im(l* a), PS -2 Im(l1* a1), RXX Im(sum l_b* a_(3-b)),
// RYY Im(-l0* a3 + l1* a2 + l2* a1 - l3* a0), RZZ +-Im(l* a).
template <class T, bool BOTH, bool GRAD, bool DAG>
__device__ T bapply(typename BV<T>::V* psi, typename BV<T>::V* lam, int n, const BGate& g,
                    const typename BV<T>::V* gd) {
  using V = typename BV<T>::V;
  T acc = 0;
  const uint64_t cm = g.cmask;
  const int kind = g.kind;
  if (bdiag(kind)) {
    V d0 = gd[0], d1 = gd[1], d2 = d0, d3 = d1;
    if (g.nt == 2) {
      d2 = gd[2];
      d3 = gd[3];
    }
    if (DAG) {
      d0 = bconj(d0);
      d1 = bconj(d1);
      d2 = bconj(d2);
      d3 = bconj(d3);
    }
    // gradient weights of Im(l* a) per basis index b
    T w0 = 0, w1 = 0, w2 = 0, w3 = 0;
    if (kind == QS_GATE_RZ) {
      w0 = 1;
      w1 = -1;
    } else if (kind == QS_GATE_PS) {
      w1 = -2;
    } else if (kind == QS_GATE_RZZ) {
      w0 = w3 = 1;
      w1 = w2 = -1;
    }
    const uint64_t N = 1ull << n;
    for (uint64_t x = threadIdx.x; x < N; x += blockDim.x) {
      if ((x & cm) != cm) continue;
      int b = (int)((x >> g.t0) & 1);
      if (g.nt == 2) b |= (int)((x >> g.t1) & 1) << 1;
      const V u = b == 0 ? d0 : (b == 1 ? d1 : (b == 2 ? d2 : d3));
      const V a = psi[x];
      if (GRAD) acc += (b == 0 ? w0 : (b == 1 ? w1 : (b == 2 ? w2 : w3))) * bim(lam[x], a);
      if (BOTH) lam[x] = bmul(u, lam[x]);
      psi[x] = bmul(u, a);
    }
  } else if (g.nt == 1) {
    V m00 = gd[0], m01 = gd[1], m10 = gd[2], m11 = gd[3];
    if (DAG) {
      m00 = bconj(gd[0]);
      m01 = bconj(gd[2]);
      m10 = bconj(gd[1]);
      m11 = bconj(gd[3]);
    }
    if (GRAD) {
      const uint64_t P = 1ull << (n - 1);
      for (uint64_t i = threadIdx.x; i < P; i += blockDim.x) {
        const uint64_t x0 = bins0(i, g.t0);
        if ((x0 & cm) != cm) continue;
        const uint64_t x1 = x0 | (1ull << g.t0);
        const V a0 = psi[x0], a1 = psi[x1], l0 = lam[x0], l1 = lam[x1];
        if (kind == QS_GATE_RX)
          acc += bim(l0, a1) + bim(l1, a0);
        else if (kind == QS_GATE_RY)
          acc += bre(l1, a0) - bre(l0, a1);
        psi[x0] = badd(bmul(m00, a0), bmul(m01, a1));
        psi[x1] = badd(bmul(m10, a0), bmul(m11, a1));
        lam[x0] = badd(bmul(m00, l0), bmul(m01, l1));
        lam[x1] = badd(bmul(m10, l0), bmul(m11, l1));
      }
    } else {
      apply_1q<T, BOTH>(psi, lam, n, g.t0, cm, m00, m01, m10, m11);
    }
  } else {
    const int lo = g.t0 < g.t1 ? g.t0 : g.t1, hi = g.t0 < g.t1 ? g.t1 : g.t0;
    T c = 1, s = 0;
    if (kind != QS_GATE_SWAP) {
      c = gd[0].x;
      s = DAG ? -gd[0].y : gd[0].y;
    }
    const uint64_t Q = 1ull << (n - 2);
    for (uint64_t i = threadIdx.x; i < Q; i += blockDim.x) {
      const uint64_t base = bins0(bins0(i, lo), hi);
      if ((base & cm) != cm) continue;
      uint64_t idx[4];
#pragma unroll
      for (int b = 0; b < 4; ++b)
        idx[b] = base | ((uint64_t)(b & 1) << g.t0) | ((uint64_t)((b >> 1) & 1) << g.t1);
#pragma unroll
      for (int st = 0; st < (BOTH ? 2 : 1); ++st) {
        V* v = st == 0 ? psi : lam;
        V a[4];
#pragma unroll
        for (int b = 0; b < 4; ++b) a[b] = v[idx[b]];
        if (GRAD && st == 0) {
          V l[4];
#pragma unroll
          for (int b = 0; b < 4; ++b) l[b] = lam[idx[b]];
          if (kind == QS_GATE_RXX)
            acc += bim(l[0], a[3]) + bim(l[1], a[2]) + bim(l[2], a[1]) + bim(l[3], a[0]);
          else if (kind == QS_GATE_RYY)
            acc += -bim(l[0], a[3]) + bim(l[1], a[2]) + bim(l[2], a[1]) - bim(l[3], a[0]);
        }
        V y[4];
        if (kind == QS_GATE_SWAP) {
          y[0] = a[0];
          y[1] = a[2];
          y[2] = a[1];
          y[3] = a[3];
        } else if (kind == QS_GATE_RXX) {
#pragma unroll
          for (int b = 0; b < 4; ++b) y[b] = badd(bmk<V, T>(c * a[b].x, c * a[b].y), mis<V, T>(s, a[3 - b]));
        } else {  // RYY
          y[0] = badd(bmk<V, T>(c * a[0].x, c * a[0].y), pis<V, T>(s, a[3]));
          y[1] = badd(bmk<V, T>(c * a[1].x, c * a[1].y), mis<V, T>(s, a[2]));
          y[2] = badd(bmk<V, T>(c * a[2].x, c * a[2].y), mis<V, T>(s, a[1]));
          y[3] = badd(bmk<V, T>(c * a[3].x, c * a[3].y), pis<V, T>(s, a[0]));
        }
#pragma unroll
        for (int b = 0; b < 4; ++b) v[idx[b]] = y[b];
      }
    }
  }
  return acc;
}

// lam = H psi (if LAM) and this thread's share of <psi|H|psi>.
template <class T, bool LAM>
__device__ T bham(const typename BV<T>::V* psi, typename BV<T>::V* lam, int n, const DevHamGroup* groups, int g_begin,
                  int g_end, const DevHamTerm* terms) {
  using V = typename BV<T>::V;
  const uint64_t N = 1ull << n;
  T e = 0;
  for (uint64_t y = threadIdx.x; y < N; y += blockDim.x) {
    T lr = 0, li = 0;
    for (int gg = g_begin; gg < g_end; ++gg) {
      const DevHamGroup G = groups[gg];
      const uint64_t x = y ^ G.xmask;
      const V v = psi[x];
      T fr = 0, fi = 0;
      for (int k = G.begin; k < G.end; ++k) {
        const DevHamTerm t = terms[k];
        const T sg = (__popcll(x & t.zmask) & 1) ? (T)-1 : (T)1;
        fr += sg * (T)t.re;
        fi += sg * (T)t.im;
      }
      lr += fr * v.x - fi * v.y;
      li += fr * v.y + fi * v.x;
    }
    if (LAM) lam[y] = bmk<V, T>(lr, li);
    const V p = psi[y];
    e += p.x * lr + p.y * li;
  }
  return e;
}

// Shared-memory regions of one CTA: psi, lam, gate data (4 per gate), gradient
// slots (per parameter, per warp).
template <class T>
struct BSmem {
  typename BV<T>::V *psi, *lam, *gd;
  T* slot;
};
template <class T>
__device__ BSmem<T> bsmem(unsigned char* smem, int amps, bool with_lam, int gates) {
  using V = typename BV<T>::V;
  BSmem<T> S;
  S.psi = reinterpret_cast<V*>(smem);
  S.lam = S.psi + (with_lam ? amps : 0);
  S.gd = S.lam + amps;
  S.slot = reinterpret_cast<T*>(S.gd + 4 * gates);
  return S;
}

// Reverse sweep step of a parametric gate: its gradient term summed over the
// warp in the state's precision and added to this warp's slot (no barrier).
template <class T>
__device__ __forceinline__ void slot_add(T* slot, int param, double coef, T part) {
  part = wsum(part);
  if ((threadIdx.x & 31) == 0) slot[param * kMaxBatchWarps + (threadIdx.x >> 5)] += (T)coef * part;
}

template <class T>
__device__ void run_instance(const BatchArgs& a, const BInst& I, const BSmem<T>& S, double* sh) {
  using V = typename BV<T>::V;
  const int n = I.n;
  const uint64_t N = 1ull << n;
  const double* params = a.params + I.param_off;
  form_gates<V, T>(a.gates, I.gate_begin, I.gate_end, params, S.gd);
  for (int i = threadIdx.x; i < I.n_params * kMaxBatchWarps; i += blockDim.x) S.slot[i] = 0;
  for (uint64_t x = threadIdx.x; x < N; x += blockDim.x) S.psi[x] = bmk<V, T>(x == 0 ? 1 : 0, 0);
  __syncthreads();
  // forward: psi = U_N ... U_1 |0>
  for (int gi = I.gate_begin; gi < I.gate_end; ++gi) {
    bapply<T, false, false, false>(S.psi, S.lam, n, a.gates[gi], S.gd + 4 * (gi - I.gate_begin));
    __syncthreads();
  }
  // lam = H psi and E = <psi|lam>
  const T e = bham<T, true>(S.psi, S.lam, n, a.groups, I.group_begin, I.group_end, a.terms);
  const double E = bsum_all(e, sh);
  if (threadIdx.x == 0) a.energy[&I - a.inst] = E;
  // reverse: gradient of every gate, psi and lam undone gate by gate
  for (int gi = I.gate_end - 1; gi >= I.gate_begin; --gi) {
    const BGate g = a.gates[gi];
    const V* gd = S.gd + 4 * (gi - I.gate_begin);
    if (g.param >= 0)
      slot_add(S.slot, g.param, g.coef, bapply<T, true, true, true>(S.psi, S.lam, n, g, gd));
    else
      bapply<T, true, false, true>(S.psi, S.lam, n, g, gd);
    __syncthreads();
  }
  double* grad = a.grad + I.param_off;
  for (int p = threadIdx.x; p < I.n_params; p += blockDim.x) {
    double s = 0;
    for (int w = 0; w < kMaxBatchWarps; ++w) s += (double)S.slot[p * kMaxBatchWarps + w];
    grad[p] = s;
  }
  __syncthreads();
}

template <class T>
__global__ void __launch_bounds__(kBatchThreads, 2) batch_kernel(BatchArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double sh[kMaxBatchWarps + 1];
  __shared__ int s_next;
  const BSmem<T> S = bsmem<T>(smem, a.smem_amps, true, a.smem_gates);
  while (true) {
    if (threadIdx.x == 0) s_next = atomicAdd(a.queue, 1);
    __syncthreads();
    const int i = s_next;
    __syncthreads();
    if (i >= a.n_inst) break;
    run_instance<T>(a, a.inst[a.order[i]], S, sh);
  }
}

// ------------------------------------------------------------ trajectories

// Uniform in [0, 1) of counter c: splitmix64 (Steele, Lea & Flood 2014) of the
// state seed + c * golden gamma, top 53 bits.
__device__ __forceinline__ double traj_uniform(uint64_t seed, uint64_t c) {
  uint64_t z = seed + c * 0x9E3779B97F4A7C15ull + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * 0x1.0p-53;
}

// One channel site of trajectory t: branch weights (fixed, or ||K_i psi||^2:
// per-thread sums in the state's precision, FP64 across warps), the branch whose
// running weight sum first exceeds u * total, then psi <- branch operator psi.
// Every thread takes the same decision (the sums are broadcast).
template <class T>
__device__ int traj_site(const TrajArgs& a, const BChannel& C, int site, long long t, typename BV<T>::V* psi,
                         double* sh) {
  using V = typename BV<T>::V;
  const int n = a.n, q = C.qubit, nk = C.n_kraus;
  double w[kTrajMaxKraus] = {0, 0, 0, 0};
  if (C.fixed) {
    for (int k = 0; k < nk; ++k) w[k] = C.w[k];
  } else {
    T acc[kTrajMaxKraus] = {0, 0, 0, 0};
    V K[kTrajMaxKraus][4];
#pragma unroll
    for (int k = 0; k < kTrajMaxKraus; ++k)
#pragma unroll
      for (int e = 0; e < 4; ++e) K[k][e] = bmk<V, T>((T)C.K[k][2 * e], (T)C.K[k][2 * e + 1]);
    const uint64_t P = 1ull << (n - 1);
    for (uint64_t i = threadIdx.x; i < P; i += blockDim.x) {
      const uint64_t x0 = bins0(i, q), x1 = x0 | (1ull << q);
      const V a0 = psi[x0], a1 = psi[x1];
#pragma unroll
      for (int k = 0; k < kTrajMaxKraus; ++k) {
        if (k >= nk) break;
        const V y0 = badd(bmul(K[k][0], a0), bmul(K[k][1], a1));
        const V y1 = badd(bmul(K[k][2], a0), bmul(K[k][3], a1));
        acc[k] += y0.x * y0.x + y0.y * y0.y + y1.x * y1.x + y1.y * y1.y;
      }
    }
    for (int k = 0; k < nk; ++k) w[k] = bsum_all(acc[k], sh);
  }
  double total = 0.0;
  for (int k = 0; k < nk; ++k) total += w[k];
  const double thr = traj_uniform(a.seed, (uint64_t)t * (uint64_t)a.n_sites + (uint64_t)site) * total;
  int c = -1;
  double cum = 0.0;
  for (int k = 0; k < nk; ++k) {
    cum += w[k];
    if (c < 0 && cum > thr) c = k;
  }
  if (c < 0)
    for (int k = 0; k < nk; ++k)
      if (w[k] > 0) c = k;
  if (c < 0) c = 0;
  const double sc = C.fixed ? 1.0 : (w[c] > 0 ? 1.0 / sqrt(w[c]) : 0.0);
  V M[4];
  for (int e = 0; e < 4; ++e) M[e] = bmk<V, T>((T)(C.K[c][2 * e] * sc), (T)(C.K[c][2 * e + 1] * sc));
  apply_1q<T, false>(psi, psi, n, q, 0, M[0], M[1], M[2], M[3]);
  __syncthreads();
  return c;
}

// Trajectories from a work queue: psi = (gates and sampled branches)|0>,
// E = <psi|H|psi>; with GRAD also lam = H psi and the adjoint sweep, each
// sampled (unitary) branch undone by its adjoint, the gradient of trajectory i
// in row i of a.grad.  The gate data is formed once per CTA (all trajectories
// share the circuit and the parameters).
template <class T, bool GRAD>
__global__ void __launch_bounds__(kBatchThreads, 2) traj_kernel(TrajArgs a) {
  using V = typename BV<T>::V;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double sh[kMaxBatchWarps + 1];
  __shared__ int s_next;
  __shared__ uint8_t s_choice[kTrajMaxSites];
  const int n = a.n;
  const uint64_t N = 1ull << n;
  const BSmem<T> S = bsmem<T>(smem, (int)N, GRAD, a.n_gates);
  form_gates<V, T>(a.gates, 0, a.n_gates, a.params, S.gd);
  while (true) {
    if (threadIdx.x == 0) s_next = atomicAdd(a.queue, 1);
    __syncthreads();
    const int i = s_next;
    __syncthreads();
    if (i >= a.n_traj) break;
    const long long t = a.first + i;
    if (GRAD)
      for (int p = threadIdx.x; p < a.n_params * kMaxBatchWarps; p += blockDim.x) S.slot[p] = 0;
    for (uint64_t x = threadIdx.x; x < N; x += blockDim.x) S.psi[x] = bmk<V, T>(x == 0 ? 1 : 0, 0);
    __syncthreads();
    for (int gi = 0; gi < a.n_gates; ++gi) {
      const BGate g = a.gates[gi];
      if (g.kind == kGateChannel) {
        const int c = traj_site<T>(a, a.ch[g.param], g.param, t, S.psi, sh);
        if (threadIdx.x == 0) s_choice[g.param] = (uint8_t)c;
        continue;
      }
      bapply<T, false, false, false>(S.psi, S.lam, n, g, S.gd + 4 * gi);
      __syncthreads();
    }
    const T e = bham<T, GRAD>(S.psi, S.lam, n, a.groups, 0, a.n_groups, a.terms);
    const double E = bsum_all(e, sh);
    if (threadIdx.x == 0) a.energy[i] = E;
    if (GRAD) {
      for (int gi = a.n_gates - 1; gi >= 0; --gi) {
        const BGate g = a.gates[gi];
        if (g.kind == kGateChannel) {
          const BChannel& C = a.ch[g.param];
          const int c = s_choice[g.param];
          V Md[4];
          for (int r = 0; r < 2; ++r)
            for (int k = 0; k < 2; ++k)
              Md[r * 2 + k] = bmk<V, T>((T)C.K[c][2 * (k * 2 + r)], (T)-C.K[c][2 * (k * 2 + r) + 1]);
          apply_1q<T, true>(S.psi, S.lam, n, C.qubit, 0, Md[0], Md[1], Md[2], Md[3]);
        } else if (g.param >= 0) {
          slot_add(S.slot, g.param, g.coef, bapply<T, true, true, true>(S.psi, S.lam, n, g, S.gd + 4 * gi));
        } else {
          bapply<T, true, false, true>(S.psi, S.lam, n, g, S.gd + 4 * gi);
        }
        __syncthreads();
      }
      double* grad = a.grad + (size_t)i * a.n_params;
      for (int p = threadIdx.x; p < a.n_params; p += blockDim.x) {
        double s = 0;
        for (int w = 0; w < kMaxBatchWarps; ++w) s += (double)S.slot[p * kMaxBatchWarps + w];
        grad[p] = s;
      }
    }
    if (a.choice)
      for (int s2 = threadIdx.x; s2 < a.n_sites; s2 += blockDim.x) a.choice[(size_t)i * a.n_sites + s2] = s_choice[s2];
    if (a.state_out && i == 0) {
      V* out = reinterpret_cast<V*>(a.state_out);
      for (uint64_t x = threadIdx.x; x < N; x += blockDim.x) out[x] = S.psi[x];
    }
    __syncthreads();
  }
}

__global__ void row_mean_kernel(const double* __restrict__ rows, int n_rows, int n_cols, double* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_cols) return;
  double s = 0.0;
  for (int r = 0; r < n_rows; ++r) s += rows[(size_t)r * n_cols + c];
  out[c] = s / (double)n_rows;
}

// Coefficient tables of the instances that run on fused tile passes, formed on
// the device from the device parameters (the same layout the host fills for a
// single circuit: diagonal gates store their diagonal, RX stores (cos, sin) of
// the half angle, other gates the full matrix; U^dag and A = dU U^dag beside).
template <class V>
__global__ void batch_coef_kernel(const BCoefGate* __restrict__ gates, int n, const double* __restrict__ params) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const BCoefGate g = gates[i];
  const double th = g.param < 0 ? g.constant : g.constant + g.coef * params[g.param];
  double2 U[16], A[16];
  bgate_matrix<double2, double>(g.kind, th, U);
  V* tab = reinterpret_cast<V*>(g.table);
  auto put = [&](int off, int k, double re, double im) {
    V v;
    v.x = (decltype(v.x))re;
    v.y = (decltype(v.x))im;
    tab[off + k] = v;
  };
  const int d = g.nt == 2 ? 4 : 2;
  if (g.diag) {
    for (int k = 0; k < d; ++k) {
      put(g.off_u, k, U[k * d + k].x, U[k * d + k].y);
      put(g.off_ud, k, U[k * d + k].x, -U[k * d + k].y);
    }
  } else if (g.kind == QS_GATE_RX) {
    double s, c;
    sincos(0.5 * th, &s, &c);
    put(g.off_u, 0, c, s);
    put(g.off_ud, 0, c, -s);
  } else {
    for (int r = 0; r < d; ++r)
      for (int col = 0; col < d; ++col) {
        put(g.off_u, r * d + col, U[r * d + col].x, U[r * d + col].y);
        put(g.off_ud, r * d + col, U[col * d + r].x, -U[col * d + r].y);
      }
  }
  if (g.off_a >= 0) {
    bgate_generator<double2, double>(g.kind, A);
    if (g.diag)
      for (int k = 0; k < d; ++k) put(g.off_a, k, A[k * d + k].x, A[k * d + k].y);
    else
      for (int k = 0; k < d * d; ++k) put(g.off_a, k, A[k].x, A[k].y);
  }
}

// Products of single-qubit runs (later gates multiply on the left), from the
// device parameters, into the fused op's table entries.
template <class V>
__global__ void batch_run_kernel(const BCoefRun* __restrict__ runs, int n, const BCoefGate* __restrict__ members,
                                 const double* __restrict__ params) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const BCoefRun R = runs[r];
  double2 M[4] = {{1, 0}, {0, 0}, {0, 0}, {1, 0}};
  for (int k = 0; k < R.count; ++k) {
    const BCoefGate g = members[R.begin + k];
    const double th = g.param < 0 ? g.constant : g.constant + g.coef * params[g.param];
    double2 U[16];
    bgate_matrix<double2, double>(g.kind, th, U);
    double2 N[4];
    for (int a = 0; a < 2; ++a)
      for (int b = 0; b < 2; ++b) {
        const double2 x = bmul(U[2 * a], M[b]), y = bmul(U[2 * a + 1], M[2 + b]);
        N[2 * a + b] = make_double2(x.x + y.x, x.y + y.y);
      }
    for (int e = 0; e < 4; ++e) M[e] = N[e];
  }
  V* tab = reinterpret_cast<V*>(R.table);
  auto put = [&](int k, double2 v) {
    V o;
    o.x = (decltype(o.x))v.x;
    o.y = (decltype(o.x))v.y;
    tab[R.off + k] = o;
  };
  if (R.diag) {
    put(0, M[0]);
    put(1, M[3]);
  } else {
    for (int e = 0; e < 4; ++e) put(e, M[e]);
  }
}

}  // namespace

qs_status launch_batch_runs(qs_dtype dt, const BCoefRun* runs, int n, const BCoefGate* members,
                            const double* params, cudaStream_t st) {
  if (n <= 0) return QS_OK;
  const int threads = 128, blocks = (n + threads - 1) / threads;
  if (dt == QS_C64)
    batch_run_kernel<float2><<<blocks, threads, 0, st>>>(runs, n, members, params);
  else
    batch_run_kernel<double2><<<blocks, threads, 0, st>>>(runs, n, members, params);
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

qs_status launch_batch_coef(qs_dtype dt, const BCoefGate* g, int n, const double* params, cudaStream_t st) {
  if (n <= 0) return QS_OK;
  const int threads = 128, blocks = (n + threads - 1) / threads;
  if (dt == QS_C64)
    batch_coef_kernel<float2><<<blocks, threads, 0, st>>>(g, n, params);
  else
    batch_coef_kernel<double2><<<blocks, threads, 0, st>>>(g, n, params);
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

namespace {
const void* traj_fn(qs_dtype dt, bool grad) {
  if (dt == QS_C64) return grad ? (const void*)traj_kernel<float, true> : (const void*)traj_kernel<float, false>;
  return grad ? (const void*)traj_kernel<double, true> : (const void*)traj_kernel<double, false>;
}
// psi (+ lam), gate data, gradient slots
size_t cta_smem(qs_dtype dt, size_t amps, bool lam, int gates, int params) {
  const size_t v = dt == QS_C64 ? 8 : 16, t = v / 2;
  return (lam ? 2 : 1) * amps * v + 4 * (size_t)gates * v + (size_t)params * kMaxBatchWarps * t;
}
int grid_for(const void* fn, size_t smem) {
  if (smem > kBatchSmemBudget) return 0;
  int occ = 0;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kBatchThreads, smem) != cudaSuccess || occ < 1) {
    (void)cudaGetLastError();
    return 0;
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return (sms > 0 ? sms : 1) * occ;
}
}  // namespace

size_t traj_smem_bytes(qs_dtype dt, bool grad, int n, int n_gates, int n_params) {
  return cta_smem(dt, (size_t)1 << n, grad, n_gates, grad ? n_params : 0);
}

int traj_grid_size(qs_dtype dt, bool grad, int n, int n_gates, int n_params) {
  return grid_for(traj_fn(dt, grad), traj_smem_bytes(dt, grad, n, n_gates, n_params));
}

qs_status launch_traj(qs_dtype dt, bool grad, const TrajArgs& a, int grid, cudaStream_t st) {
  const size_t smem = traj_smem_bytes(dt, grad, a.n, a.n_gates, a.n_params);
  if (dt == QS_C64) {
    if (grad)
      traj_kernel<float, true><<<grid, kBatchThreads, smem, st>>>(a);
    else
      traj_kernel<float, false><<<grid, kBatchThreads, smem, st>>>(a);
  } else {
    if (grad)
      traj_kernel<double, true><<<grid, kBatchThreads, smem, st>>>(a);
    else
      traj_kernel<double, false><<<grid, kBatchThreads, smem, st>>>(a);
  }
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

qs_status launch_row_mean(const double* rows, int n_rows, int n_cols, double* out, cudaStream_t st) {
  if (n_cols <= 0) return QS_OK;
  row_mean_kernel<<<(n_cols + 127) / 128, 128, 0, st>>>(rows, n_rows, n_cols, out);
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

size_t batch_smem_bytes(qs_dtype dt, int smem_amps, int smem_gates, int smem_params) {
  return cta_smem(dt, (size_t)smem_amps, true, smem_gates, smem_params);
}

int batch_grid_size(qs_dtype dt, int smem_amps, int smem_gates, int smem_params) {
  const void* fn = dt == QS_C64 ? (const void*)batch_kernel<float> : (const void*)batch_kernel<double>;
  return grid_for(fn, batch_smem_bytes(dt, smem_amps, smem_gates, smem_params));
}

qs_status launch_batch(qs_dtype dt, const BatchArgs& a, int grid, cudaStream_t st) {
  const size_t smem = batch_smem_bytes(dt, a.smem_amps, a.smem_gates, a.smem_params);
  if (dt == QS_C64)
    batch_kernel<float><<<grid, kBatchThreads, smem, st>>>(a);
  else
    batch_kernel<double><<<grid, kBatchThreads, smem, st>>>(a);
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

}  // namespace qs
