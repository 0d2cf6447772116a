// Per-gate kernels, state initialisation, Pauli-sum application and
// expectation, deterministic reductions, MaxCut cut values and sampling.
#include <algorithm>

#include "qsim_internal.h"

namespace qs {

namespace {

template <class T>
struct V2;
template <>
struct V2<float> {
  using V = float2;
};
template <>
struct V2<double> {
  using V = double2;
};

template <class V>
__device__ __forceinline__ V mulc(V a, V b) {
  V r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}

constexpr int kThreads = 256;

int blocks_for(uint64_t work, int per_block = kThreads) {
  uint64_t b = (work + per_block - 1) / per_block;
  if (b > (1u << 30)) b = 1u << 30;
  return (int)(b ? b : 1);
}

// Insert a zero bit at position q (bits >= q shift up).
__device__ __forceinline__ uint64_t insert0(uint64_t i, int q) {
  const uint64_t lo = i & ((1ull << q) - 1);
  return ((i >> q) << (q + 1)) | lo;
}

struct Mat4 {
  double re[16], im[16];
};

// --------------------------------------------------------------- per-gate dense
template <class T, int K>
__global__ void gate_dense_kernel(typename V2<T>::V* psi, int n, int t0, int t1, uint64_t cmask, Mat4 M) {
  using V = typename V2<T>::V;
  const uint64_t groups = 1ull << (n - K);
  const int lo = (K == 2 && t1 < t0) ? t1 : t0;
  const int hi = (K == 2 && t1 < t0) ? t0 : t1;
  constexpr int D = 1 << K;
  V m[D * D];
#pragma unroll
  for (int i = 0; i < D * D; ++i) {
    m[i].x = (T)M.re[i];
    m[i].y = (T)M.im[i];
  }
  for (uint64_t g = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; g < groups;
       g += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t base = insert0(g, lo);
    if (K == 2) base = insert0(base, hi);
    if ((base & cmask) != cmask) continue;
    uint64_t idx[D];
#pragma unroll
    for (int b = 0; b < D; ++b) {
      uint64_t x = base;
      if (b & 1) x |= 1ull << t0;
      if (K == 2 && (b & 2)) x |= 1ull << t1;
      idx[b] = x;
    }
    V in[D];
#pragma unroll
    for (int b = 0; b < D; ++b) in[b] = psi[idx[b]];
#pragma unroll
    for (int r = 0; r < D; ++r) {
      V acc;
      acc.x = 0;
      acc.y = 0;
#pragma unroll
      for (int cidx = 0; cidx < D; ++cidx) {
        V p = mulc(m[r * D + cidx], in[cidx]);
        acc.x += p.x;
        acc.y += p.y;
      }
      psi[idx[r]] = acc;
    }
  }
}

template <class T>
__global__ void gate_diag_kernel(typename V2<T>::V* psi, int n, int nt, int t0, int t1, uint64_t cmask, Mat4 D) {
  using V = typename V2<T>::V;
  const uint64_t N = 1ull << n;
  V d[4];
  for (int i = 0; i < 4; ++i) {
    d[i].x = (T)D.re[i];
    d[i].y = (T)D.im[i];
  }
  for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < N; x += (uint64_t)gridDim.x * blockDim.x) {
    if ((x & cmask) != cmask) continue;
    int b = (int)((x >> t0) & 1);
    if (nt == 2) b |= (int)((x >> t1) & 1) << 1;
    psi[x] = mulc(d[b], psi[x]);
  }
}

// --------------------------------------------------------------- per-gate at HBM speed
// A single-qubit dense gate or a diagonal gate on one or two qubits, applied to
// exactly the amplitudes it changes: work item i enumerates the free bits (every
// bit but the fixed ones, in increasing order), the fixed bits are deposited
// (controls and, for diagonal gates whose first entry is 1, the target as 1; the
// target of a dense gate as 0).  With bit 0 free a complex64 item covers two
// adjacent amplitudes per 16-byte access; each thread keeps kGateUnroll items in
// flight, streaming loads and stores (the state is touched once).
constexpr int kGateUnroll = 4;
constexpr int kMaxFixed = 8;
struct FixedBits {
  int k;
  int pos[kMaxFixed];  // increasing
  uint64_t ones;       // fixed bits deposited as 1
};

__device__ __forceinline__ uint64_t deposit(uint64_t i, const FixedBits& F) {
#pragma unroll
  for (int j = 0; j < kMaxFixed; ++j) {  // static indices: F stays in the parameter bank
    if (j < F.k) {
      const int q = F.pos[j];
      i = ((i >> q) << (q + 1)) | (i & ((1ull << q) - 1)) | (F.ones & (1ull << q));
    }
  }
  return i;
}

__device__ __forceinline__ float4 ldcs4(const float2* p) { return __ldcs(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ void stcs4(float2* p, float4 v) { __stcs(reinterpret_cast<float4*>(p), v); }

template <class V>
__device__ __forceinline__ V lin2(V m0, V a, V m1, V b) {
  V r;
  r.x = m0.x * a.x - m0.y * a.y + m1.x * b.x - m1.y * b.y;
  r.y = m0.x * a.y + m0.y * a.x + m1.x * b.y + m1.y * b.x;
  return r;
}

// complex64, bit 0 free: item = two pairs (x, x + 1) and (x | T, x + 1 | T).
__global__ void gate1_c64_vec_kernel(float2* __restrict__ psi, uint64_t items, int t, FixedBits F, float2 m00,
                                     float2 m01, float2 m10, float2 m11) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t T = 1ull << t;
  for (uint64_t i0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i0 < items; i0 += stride * kGateUnroll) {
    float4 a[kGateUnroll], b[kGateUnroll];
    uint64_t x[kGateUnroll];
#pragma unroll
    for (int u = 0; u < kGateUnroll; ++u) {
      const uint64_t i = i0 + u * stride;
      x[u] = i < items ? deposit(i, F) : 0;  // F fixes bit 0 (as 0)
      if (i < items) {
        a[u] = ldcs4(psi + x[u]);
        b[u] = ldcs4(psi + (x[u] | T));
      }
    }
#pragma unroll
    for (int u = 0; u < kGateUnroll; ++u) {
      if (i0 + u * stride >= items) continue;
      const float2 a0 = make_float2(a[u].x, a[u].y), a1 = make_float2(a[u].z, a[u].w);
      const float2 b0 = make_float2(b[u].x, b[u].y), b1 = make_float2(b[u].z, b[u].w);
      const float2 y0 = lin2(m00, a0, m01, b0), z0 = lin2(m10, a0, m11, b0);
      const float2 y1 = lin2(m00, a1, m01, b1), z1 = lin2(m10, a1, m11, b1);
      stcs4(psi + x[u], make_float4(y0.x, y0.y, y1.x, y1.y));
      stcs4(psi + (x[u] | T), make_float4(z0.x, z0.y, z1.x, z1.y));
    }
  }
}

// complex64 with the target on qubit 0: item = one pair in one 16-byte access.
__global__ void gate1_c64_q0_kernel(float2* __restrict__ psi, uint64_t items, FixedBits F, float2 m00, float2 m01,
                                    float2 m10, float2 m11) {
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i0 < items; i0 += stride * kGateUnroll) {
    float4 a[kGateUnroll];
    uint64_t x[kGateUnroll];
#pragma unroll
    for (int u = 0; u < kGateUnroll; ++u) {
      const uint64_t i = i0 + u * stride;
      x[u] = i < items ? deposit(i, F) : 0;
      if (i < items) a[u] = ldcs4(psi + x[u]);
    }
#pragma unroll
    for (int u = 0; u < kGateUnroll; ++u) {
      if (i0 + u * stride >= items) continue;
      const float2 a0 = make_float2(a[u].x, a[u].y), a1 = make_float2(a[u].z, a[u].w);
      const float2 y = lin2(m00, a0, m01, a1), z = lin2(m10, a0, m11, a1);
      stcs4(psi + x[u], make_float4(y.x, y.y, z.x, z.y));
    }
  }
}

// y = m0 a + m1 b for the matrix forms: 0 general complex, 1 real entries (H, RY,
// X: half the multiplications), 2 real diagonal and imaginary off-diagonal (RX).
template <int FORM, class V>
__device__ __forceinline__ V lin2f(V m0, V a, V m1, V b) {
  V r;
  if constexpr (FORM == 1) {
    r.x = m0.x * a.x + m1.x * b.x;
    r.y = m0.x * a.y + m1.x * b.y;
  } else if constexpr (FORM == 2) {  // m0 real on the diagonal, m1 = i m1.y off it
    r.x = m0.x * a.x - m1.y * b.y;
    r.y = m0.x * a.y + m1.y * b.x;
  } else {
    r = lin2(m0, a, m1, b);
  }
  return r;
}

// Exact product i^k a (k = 0..3): a swap of the components and sign-bit flips,
// done on the integer pipe (complex128 gates whose entries are 0, +-1 or +-i
// then need no FP64 arithmetic, which bounds the other complex128 kernels).
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

// Anti-diagonal gate with entries i^k01 (row 0) and i^k10 (row 1): X, Y and
// their controlled forms move amplitudes without arithmetic.
template <class T>
__global__ void gate1_perm_kernel(typename V2<T>::V* __restrict__ psi, uint64_t items, int t, FixedBits F,
                                  uint32_t k01, uint32_t k10) {
  using V = typename V2<T>::V;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t Tb = 1ull << t;
  for (uint64_t i0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i0 < items; i0 += stride * kGateUnroll) {
    V a[kGateUnroll], b[kGateUnroll];
    uint64_t x[kGateUnroll];
#pragma unroll
    for (int u = 0; u < kGateUnroll; ++u) {
      const uint64_t i = i0 + u * stride;
      x[u] = i < items ? deposit(i, F) : 0;
      if (i < items) {
        a[u] = __ldcs(psi + x[u]);
        b[u] = __ldcs(psi + (x[u] | Tb));
      }
    }
#pragma unroll
    for (int u = 0; u < kGateUnroll; ++u) {
      if (i0 + u * stride >= items) continue;
      __stcs(psi + x[u], mul_ik(k01, b[u]));
      __stcs(psi + (x[u] | Tb), mul_ik(k10, a[u]));
    }
  }
}

// One pair per item (complex128, or complex64 with bit 0 fixed by a control).
// FORM 3: [[h, h], [h, -h]] with real h (Hadamard): the product h b is shared
// by both outputs, 3 instead of 4 operations per component.
template <class T, int FORM>
__global__ void gate1_pair_kernel(typename V2<T>::V* __restrict__ psi, uint64_t items, int t, FixedBits F,
                                  typename V2<T>::V m00, typename V2<T>::V m01, typename V2<T>::V m10,
                                  typename V2<T>::V m11) {
  using V = typename V2<T>::V;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const uint64_t Tb = 1ull << t;
  for (uint64_t i0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i0 < items; i0 += stride * kGateUnroll) {
    V a[kGateUnroll], b[kGateUnroll];
    uint64_t x[kGateUnroll];
#pragma unroll
    for (int u = 0; u < kGateUnroll; ++u) {
      const uint64_t i = i0 + u * stride;
      x[u] = i < items ? deposit(i, F) : 0;
      if (i < items) {
        a[u] = __ldcs(psi + x[u]);
        b[u] = __ldcs(psi + (x[u] | Tb));
      }
    }
#pragma unroll
    for (int u = 0; u < kGateUnroll; ++u) {
      if (i0 + u * stride >= items) continue;
      if constexpr (FORM == 3) {
        const T h = m00.x;
        V hb, y0, y1;
        hb.x = h * b[u].x;
        hb.y = h * b[u].y;
        y0.x = fma(h, a[u].x, hb.x);
        y0.y = fma(h, a[u].y, hb.y);
        y1.x = fma(h, a[u].x, -hb.x);
        y1.y = fma(h, a[u].y, -hb.y);
        __stcs(psi + x[u], y0);
        __stcs(psi + (x[u] | Tb), y1);
      } else {
        __stcs(psi + x[u], lin2f<FORM>(m00, a[u], m01, b[u]));
        __stcs(psi + (x[u] | Tb), lin2f<FORM>(m11, b[u], m10, a[u]));
      }
    }
  }
}

// Diagonal: amplitude x gets d[bit t0 + 2 bit t1] (targets that are fixed bits
// contribute their deposited value).  VEC (complex64, bit 0 free): two adjacent
// amplitudes per item, which share the factor unless a target is qubit 0.
template <class T, bool VEC>
__global__ void diag_fast_kernel(typename V2<T>::V* __restrict__ psi, uint64_t items, int nt, int t0, int t1,
                                 FixedBits F, typename V2<T>::V d0, typename V2<T>::V d1, typename V2<T>::V d2,
                                 typename V2<T>::V d3) {
  using V = typename V2<T>::V;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i0 < items; i0 += stride * kGateUnroll) {
    uint64_t x[kGateUnroll];
    float4 a4[kGateUnroll];
    V a[kGateUnroll];
#pragma unroll
    for (int u = 0; u < kGateUnroll; ++u) {
      const uint64_t i = i0 + u * stride;
      x[u] = i < items ? deposit(i, F) : 0;  // VEC: F fixes bit 0 (as 0)
      if (i < items) {
        if constexpr (VEC)
          a4[u] = ldcs4(reinterpret_cast<const float2*>(psi) + x[u]);
        else
          a[u] = __ldcs(psi + x[u]);
      }
    }
#pragma unroll
    for (int u = 0; u < kGateUnroll; ++u) {
      if (i0 + u * stride >= items) continue;
      auto factor = [&](uint64_t y) {
        int b = (int)((y >> t0) & 1);
        if (nt == 2) b |= (int)((y >> t1) & 1) << 1;
        return b == 0 ? d0 : (b == 1 ? d1 : (b == 2 ? d2 : d3));
      };
      if constexpr (VEC) {
        const V f0 = factor(x[u]), f1 = factor(x[u] + 1);
        const V y0 = mulc(f0, make_float2(a4[u].x, a4[u].y)), y1 = mulc(f1, make_float2(a4[u].z, a4[u].w));
        stcs4(reinterpret_cast<float2*>(psi) + x[u], make_float4(y0.x, y0.y, y1.x, y1.y));
      } else {
        __stcs(psi + x[u], mulc(factor(x[u]), a[u]));
      }
    }
  }
}

// Diagonal whose entries are all powers of i (Z, S, CZ ...): amplitude x gets
// i^k with k = bits 2b..2b+1 of `codes`, b = bit t0 + 2 bit t1 of x.
template <class T>
__global__ void diag_unit_kernel(typename V2<T>::V* __restrict__ psi, uint64_t items, int nt, int t0, int t1,
                                 FixedBits F, uint32_t codes) {
  using V = typename V2<T>::V;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t i0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i0 < items; i0 += stride * kGateUnroll) {
    uint64_t x[kGateUnroll];
    V a[kGateUnroll];
#pragma unroll
    for (int u = 0; u < kGateUnroll; ++u) {
      const uint64_t i = i0 + u * stride;
      x[u] = i < items ? deposit(i, F) : 0;
      if (i < items) a[u] = __ldcs(psi + x[u]);
    }
#pragma unroll
    for (int u = 0; u < kGateUnroll; ++u) {
      if (i0 + u * stride >= items) continue;
      uint32_t b = (uint32_t)((x[u] >> t0) & 1);
      if (nt == 2) b |= (uint32_t)((x[u] >> t1) & 1) << 1;
      __stcs(psi + x[u], mul_ik((codes >> (2 * b)) & 3u, a[u]));
    }
  }
}

// k with (re, im) = i^k exactly, else -1.
int unit_code(double re, double im) {
  if (im == 0.0 && re == 1.0) return 0;
  if (re == 0.0 && im == 1.0) return 1;
  if (im == 0.0 && re == -1.0) return 2;
  if (re == 0.0 && im == -1.0) return 3;
  return -1;
}

int gate_grid(uint64_t work) {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  const uint64_t want = (work + (uint64_t)kThreads * kGateUnroll - 1) / ((uint64_t)kThreads * kGateUnroll);
  return (int)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)sms * 8));
}

// Sorted fixed bits from a position mask; false if there are too many.
bool fixed_from(uint64_t fixed_mask, uint64_t ones, FixedBits* F) {
  F->k = 0;
  F->ones = ones;
  for (int q = 0; q < 64; ++q)
    if ((fixed_mask >> q) & 1) {
      if (F->k == kMaxFixed) return false;
      F->pos[F->k++] = q;
    }
  return true;
}

// --------------------------------------------------------------- init
template <class T>
__global__ void set_plus_kernel(typename V2<T>::V* psi, uint64_t N, T amp) {
  for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < N; x += (uint64_t)gridDim.x * blockDim.x) {
    typename V2<T>::V v;
    v.x = amp;
    v.y = 0;
    psi[x] = v;
  }
}

template <class T>
__global__ void set_one_kernel(typename V2<T>::V* psi, uint64_t index) {
  typename V2<T>::V v;
  v.x = 1;
  v.y = 0;
  psi[index] = v;
}

// --------------------------------------------------------------- block reduction helpers
__device__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sh[i];
  }
  __syncthreads();
  return r;  // valid in thread 0
}

constexpr int kFlush = 16;  // FP32 partial sums are flushed to FP64 every kFlush elements

// lam_y = sum_g psi_{y^m_g} * sum_{k in g} c'_k (-1)^{popcount((y^m_g) & z_k)};  E += Re(conj(psi_y) lam_y)
template <class T>
__device__ __forceinline__ void ham_apply_kernel_body(const typename V2<T>::V* __restrict__ psi,
                                                      typename V2<T>::V* __restrict__ lam, int n,
                                                      const DevHamGroup* __restrict__ groups, int n_groups,
                                                      const DevHamTerm* __restrict__ terms, double* partials) {
  using V = typename V2<T>::V;
  __shared__ double sh[32];
  const uint64_t N = 1ull << n;
  double acc_d = 0;
  T acc = 0;
  int cnt = 0;
  for (uint64_t y = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; y < N; y += (uint64_t)gridDim.x * blockDim.x) {
    T lr = 0, li = 0;
    for (int g = 0; g < n_groups; ++g) {
      const DevHamGroup G = groups[g];
      const uint64_t x = y ^ G.xmask;
      const V a = psi[x];
      T fr = 0, fi = 0;
      for (int k = G.begin; k < G.end; ++k) {
        const DevHamTerm t = terms[k];
        const T s = (__popcll(x & t.zmask) & 1) ? (T)-1 : (T)1;
        fr += s * (T)t.re;
        fi += s * (T)t.im;
      }
      lr += fr * a.x - fi * a.y;
      li += fr * a.y + fi * a.x;
    }
    const V p = psi[y];
    if (lam) {
      V o;
      o.x = lr;
      o.y = li;
      lam[y] = o;
    }
    acc += p.x * lr + p.y * li;
    if (++cnt == kFlush) {
      acc_d += (double)acc;
      acc = 0;
      cnt = 0;
    }
  }
  acc_d += (double)acc;
  const double s = block_sum(acc_d, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

template <class T>
__global__ void ham_apply_kernel(const typename V2<T>::V* __restrict__ psi, typename V2<T>::V* __restrict__ lam, int n,
                                 const DevHamGroup* __restrict__ groups, int n_groups,
                                 const DevHamTerm* __restrict__ terms, double* partials) {
  ham_apply_kernel_body<T>(psi, lam, n, groups, n_groups, terms, partials);
}

template <class T>
__global__ void ham_apply_multi_kernel(const HamMultiArgs* __restrict__ argv) {
  const HamMultiArgs a = argv[blockIdx.y];
  ham_apply_kernel_body<T>(reinterpret_cast<const typename V2<T>::V*>(a.psi),
                           reinterpret_cast<typename V2<T>::V*>(a.lam), a.n, a.groups, a.n_groups, a.terms,
                           a.partials);
}

// <a|b> partials: [0][grid] real, [1][grid] imag
template <class T>
__global__ void inner_kernel(const typename V2<T>::V* __restrict__ a, const typename V2<T>::V* __restrict__ b, int n,
                             double* partials) {
  __shared__ double sh[32];
  const uint64_t N = 1ull << n;
  double re_d = 0, im_d = 0;
  T re = 0, im = 0;
  int cnt = 0;
  for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < N; x += (uint64_t)gridDim.x * blockDim.x) {
    const auto u = a[x], v = b[x];
    re += u.x * v.x + u.y * v.y;
    im += u.x * v.y - u.y * v.x;
    if (++cnt == kFlush) {
      re_d += re;
      im_d += im;
      re = im = 0;
      cnt = 0;
    }
  }
  re_d += re;
  im_d += im;
  const double r = block_sum(re_d, sh);
  const double i = block_sum(im_d, sh);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = r;
    partials[gridDim.x + blockIdx.x] = i;
  }
}

template <class T>
__global__ void norm2_kernel(const typename V2<T>::V* __restrict__ a, int n, double* partials) {
  __shared__ double sh[32];
  const uint64_t N = 1ull << n;
  double s_d = 0;
  T s = 0;
  int cnt = 0;
  for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < N; x += (uint64_t)gridDim.x * blockDim.x) {
    const auto u = a[x];
    s += u.x * u.x + u.y * u.y;
    if (++cnt == kFlush) {
      s_d += s;
      s = 0;
      cnt = 0;
    }
  }
  s_d += s;
  const double r = block_sum(s_d, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = r;
}

// Reduced density matrix of qubit q, FP64 sums over the pairs (a0, a1) =
// (psi[x], psi[x | 2^q]) with bit q of x clear: partials[k * grid + block] for
// k = 0: sum |a0|^2, 1: sum |a1|^2, 2: Re sum a0 conj(a1), 3: Im sum a0 conj(a1).
template <class T>
__global__ void qubit_rdm_kernel(const typename V2<T>::V* __restrict__ a, int n, int q, double* partials) {
  __shared__ double sh[32];
  const uint64_t P = 1ull << (n - 1), Q = 1ull << q;
  double r00 = 0, r11 = 0, re = 0, im = 0;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < P; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t x0 = insert0(i, q);
    const auto u = a[x0], v = a[x0 | Q];
    const double ux = u.x, uy = u.y, vx = v.x, vy = v.y;
    r00 += ux * ux + uy * uy;
    r11 += vx * vx + vy * vy;
    re += ux * vx + uy * vy;
    im += uy * vx - ux * vy;
  }
  const double s0 = block_sum(r00, sh);
  const double s1 = block_sum(r11, sh);
  const double s2 = block_sum(re, sh);
  const double s3 = block_sum(im, sh);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = s0;
    partials[gridDim.x + blockIdx.x] = s1;
    partials[2 * gridDim.x + blockIdx.x] = s2;
    partials[3 * gridDim.x + blockIdx.x] = s3;
  }
}

// One warp per slot, fixed order: lanes take strided partials, then a fixed tree.
__global__ void reduce_slots_kernel(const double* partials, int n_slots, int nb, const double* scale, double* out) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= n_slots) return;
  double v = 0;
  for (int b = lane; b < nb; b += 32) v += partials[(size_t)warp * nb + b];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) out[warp] = scale ? v * scale[warp] : v;
}

__global__ void reduce_multi_kernel(const ReduceMultiArgs* __restrict__ argv) {
  const ReduceMultiArgs a = argv[blockIdx.y];
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= a.n_slots) return;
  double v = 0;
  for (int b = lane; b < a.nb; b += 32) v += a.partials[(size_t)warp * a.nb + b];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) a.out[warp] = v;
}

__global__ void gather_multi_kernel(const GatherMultiArgs* __restrict__ argv) {
  const GatherMultiArgs a = argv[blockIdx.y];
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= a.n_params) return;
  double s = 0;
  for (int k = a.row_ptr[p]; k < a.row_ptr[p + 1]; ++k) s += a.gate_coef[k] * a.gate_grad[a.gate_idx[k]];
  a.grad[p] = s;
}

template <class T>
__global__ void set_zero_multi_kernel(typename V2<T>::V* base, uint64_t N, int count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) base[(uint64_t)i * N].x = (T)1;
}

__global__ void param_gather_kernel(const double* gate_grad, const int* row_ptr, const int* gate_idx,
                                    const double* gate_coef, int n_params, double* grad) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n_params) return;
  double s = 0;
  for (int k = row_ptr[p]; k < row_ptr[p + 1]; ++k) s += gate_coef[k] * gate_grad[gate_idx[k]];
  grad[p] = s;
}

// cut(x) = number of edges whose endpoints differ in x
__global__ void cut_values_kernel(uint8_t* cut, int n, const int* __restrict__ edges, int n_edges) {
  extern __shared__ int s_e[];
  for (int i = threadIdx.x; i < 2 * n_edges; i += blockDim.x) s_e[i] = edges[i];
  __syncthreads();
  const uint64_t N = 1ull << n;
  for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < N; x += (uint64_t)gridDim.x * blockDim.x) {
    int c = 0;
    for (int e = 0; e < n_edges; ++e) c += (int)(((x >> s_e[2 * e]) ^ (x >> s_e[2 * e + 1])) & 1ull);
    cut[x] = (uint8_t)c;
  }
}

// *out = max over x of cut(x) (the maximum cut), 16 bytes per thread step
__global__ void max_u8_kernel(const uint8_t* __restrict__ v, uint64_t n, int* out) {
  int m = 0;
  const uint64_t n16 = n / 16;
  const uint4* v16 = reinterpret_cast<const uint4*>(v);
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n16; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint4 w = v16[i];
    for (uint32_t word : {w.x, w.y, w.z, w.w})
      for (int b = 0; b < 4; ++b) m = max(m, (int)((word >> (8 * b)) & 0xffu));
  }
  for (uint64_t i = n16 * 16 + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    m = max(m, (int)v[i]);
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// --------------------------------------------------------------- sampling
constexpr int kChunkBits = 12;  // probabilities are summed in chunks of 4096 amplitudes

template <class T>
__device__ __forceinline__ double prob(const typename V2<T>::V& a) {
  // products of the stored components are formed in FP64
  return (double)a.x * (double)a.x + (double)a.y * (double)a.y;
}

// chunk sums, one warp per chunk, lanes own contiguous segments (fixed order)
template <class T>
__global__ void chunk_sum_kernel(const typename V2<T>::V* __restrict__ psi, int n, double* chunk) {
  const int cb = n < kChunkBits ? n : kChunkBits;
  const uint64_t n_chunks = 1ull << (n - cb);
  const uint64_t w = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= n_chunks) return;
  const uint64_t csize = 1ull << cb;
  const uint64_t seg = (csize + 31) / 32;
  const uint64_t b = w * csize + lane * seg;
  double s = 0;
  for (uint64_t i = 0; i < seg && lane * seg + i < csize; ++i) s += prob<T>(psi[b + i]);
  // exclusive scan over lanes (Hillis-Steele, fixed order) -> total in lane 31
  for (int o = 1; o < 32; o <<= 1) {
    const double t = __shfl_up_sync(0xffffffffu, s, o);
    if (lane >= o) s += t;
  }
  if (lane == 31) chunk[w] = s;
}

// exclusive prefix over chunk sums in place, single block; chunk[n_chunks] = total
__global__ void chunk_scan_kernel(double* chunk, uint64_t n_chunks) {
  __shared__ double sh[1024];
  const int t = threadIdx.x, T_ = blockDim.x;
  const uint64_t per = (n_chunks + T_ - 1) / T_;
  const uint64_t b = t * per;
  double s = 0;
  for (uint64_t i = 0; i < per && b + i < n_chunks; ++i) s += chunk[b + i];
  sh[t] = s;
  __syncthreads();
  if (t == 0) {
    double run = 0;
    for (int i = 0; i < T_; ++i) {
      const double v = sh[i];
      sh[i] = run;
      run += v;
    }
    chunk[n_chunks] = run;
  }
  __syncthreads();
  double run = sh[t];
  for (uint64_t i = 0; i < per && b + i < n_chunks; ++i) {
    const double v = chunk[b + i];
    chunk[b + i] = run;
    run += v;
  }
}

__device__ __forceinline__ uint64_t splitmix64_out(uint64_t state) {
  uint64_t z = state + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// ------------------------------------------------------- projective measurement
// One qubit measured in the computational basis (the measurement gate of
// §2.3 / §2.6.3): P(1) = sum |psi_x|^2 over x with bit q set, the outcome drawn
// with the sampling rule (u_0 from splitmix64 of the seed; outcome 0 iff
// P(0) > u_0 * total), then the state projected and renormalised.
template <class T>
__global__ void measure_mass_kernel(const typename V2<T>::V* __restrict__ psi, int n, int q, double* partials) {
  __shared__ double s1[kThreads / 32], st[kThreads / 32];
  double a1 = 0.0, at = 0.0;
  const uint64_t N = 1ull << n;
  for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < N; x += (uint64_t)gridDim.x * blockDim.x) {
    const double p = (double)psi[x].x * (double)psi[x].x + (double)psi[x].y * (double)psi[x].y;
    at += p;
    if ((x >> q) & 1ull) a1 += p;
  }
  for (int o = 16; o > 0; o >>= 1) {
    a1 += __shfl_xor_sync(0xffffffffu, a1, o);
    at += __shfl_xor_sync(0xffffffffu, at, o);
  }
  if ((threadIdx.x & 31) == 0) {
    s1[threadIdx.x >> 5] = a1;
    st[threadIdx.x >> 5] = at;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double b1 = 0.0, bt = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      b1 += s1[w];
      bt += st[w];
    }
    partials[2 * blockIdx.x] = b1;
    partials[2 * blockIdx.x + 1] = bt;
  }
}

// out[0] = outcome, out[1] = 1 / sqrt(P(outcome)) (doubles), fixed summation order.
__global__ void measure_decide_kernel(const double* partials, int nb, uint64_t seed, double* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double p1 = 0.0, tot = 0.0;
  for (int b = 0; b < nb; ++b) {
    p1 += partials[2 * b];
    tot += partials[2 * b + 1];
  }
  const double p0 = tot - p1;
  const uint64_t z = splitmix64_out(seed);
  const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
  const int outcome = p0 > u * tot ? 0 : 1;
  const double pk = outcome ? p1 : p0;
  out[0] = (double)outcome;
  out[1] = pk > 0.0 ? 1.0 / sqrt(pk) : 0.0;
}

template <class T>
__global__ void measure_collapse_kernel(typename V2<T>::V* __restrict__ psi, int n, int q, const double* out) {
  const uint64_t keep = (uint64_t)out[0];
  const T sc = (T)out[1];
  const uint64_t N = 1ull << n;
  for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < N; x += (uint64_t)gridDim.x * blockDim.x) {
    typename V2<T>::V v = psi[x];
    const bool on = ((x >> q) & 1ull) == keep;
    v.x = on ? v.x * sc : (T)0;
    v.y = on ? v.y * sc : (T)0;
    psi[x] = v;
  }
}

// one warp per shot
template <class T>
__global__ void sample_kernel(const typename V2<T>::V* __restrict__ psi, int n, const double* __restrict__ chunk,
                              uint64_t shots, uint64_t seed, uint64_t* out) {
  const uint64_t w = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= shots) return;
  const int cb = n < kChunkBits ? n : kChunkBits;
  const uint64_t n_chunks = 1ull << (n - cb);
  const double total = chunk[n_chunks];
  const uint64_t z = splitmix64_out(seed + w * 0x9E3779B97F4A7C15ull);
  const double u = (double)(z >> 11) * (1.0 / 9007199254740992.0);
  const double target = u * total;
  // last chunk k with prefix[k] <= target
  uint64_t lo = 0, hi = n_chunks - 1;
  while (lo < hi) {
    const uint64_t mid = (lo + hi + 1) >> 1;
    if (chunk[mid] <= target)
      lo = mid;
    else
      hi = mid - 1;
  }
  const uint64_t csize = 1ull << cb;
  const uint64_t seg = (csize + 31) / 32;
  const uint64_t base = lo * csize;
  double s = 0;
  for (uint64_t i = 0; i < seg && lane * seg + i < csize; ++i) s += prob<T>(psi[base + lane * seg + i]);
  double incl = s;
  for (int o = 1; o < 32; o <<= 1) {
    const double t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  const double start = chunk[lo] + (incl - s);
  const double end = chunk[lo] + incl;
  // first lane whose running sum passes the target
  const unsigned passed = __ballot_sync(0xffffffffu, end > target);
  uint64_t result = base + csize - 1;
  if (passed == 0) {
    // rounding left the target at or beyond this chunk's end: the last amplitude
    // with non-zero probability in the chunk
    if (lane == 0) {
      for (uint64_t i = csize; i-- > 0;) {
        if (prob<T>(psi[base + i]) > 0) {
          result = base + i;
          break;
        }
      }
    }
    result = __shfl_sync(0xffffffffu, result, 0);
  } else {
    const int L = __ffs(passed) - 1;
    if (lane == L) {
      double run = start;
      const uint64_t b0 = base + lane * seg;
      const uint64_t stop = base + (lane * seg + seg < csize ? lane * seg + seg : csize);
      uint64_t x = b0;
      for (; x < stop; ++x) {
        run += prob<T>(psi[x]);
        if (run > target) break;
      }
      result = x < stop ? x : stop - 1;
    }
    result = __shfl_sync(0xffffffffu, result, L);
  }
  if (lane == 0) out[w] = result;
}

}  // namespace

// ------------------------------------------------------------------------ launchers

qs_status launch_gate_dense(qs_dtype dt, void* psi, int n, int nt, const int* t, uint64_t cmask, const double* mat,
                            cudaStream_t st) {
  if (nt == 1) {
    const int q = t[0];
    FixedBits F;
    if (fixed_from(cmask | (1ull << q), cmask, &F)) {
      const int nfix = F.k;
      const uint64_t pairs = 1ull << (n - nfix);  // items of one pair each
      if (dt == QS_C64) {
        const float2 m00 = make_float2((float)mat[0], (float)mat[1]), m01 = make_float2((float)mat[2], (float)mat[3]);
        const float2 m10 = make_float2((float)mat[4], (float)mat[5]), m11 = make_float2((float)mat[6], (float)mat[7]);
        if (q == 0) {
          // the pair (x, x + 1) is one aligned 16-byte word; controls are fixed bits
          gate1_c64_q0_kernel<<<gate_grid(pairs), kThreads, 0, st>>>((float2*)psi, pairs, F, m00, m01, m10, m11);
        } else if (!(cmask & 1ull) && q != 0 && n - nfix >= 1) {
          // bit 0 free: fix it too, two amplitudes per access
          FixedBits F2;
          if (fixed_from(cmask | (1ull << q) | 1ull, cmask, &F2)) {
            gate1_c64_vec_kernel<<<gate_grid(pairs / 2), kThreads, 0, st>>>((float2*)psi, pairs / 2, q, F2, m00, m01,
                                                                            m10, m11);
          } else {
            gate1_pair_kernel<float, 0><<<gate_grid(pairs), kThreads, 0, st>>>((float2*)psi, pairs, q, F, m00, m01,
                                                                              m10, m11);
          }
        } else {
          gate1_pair_kernel<float, 0><<<gate_grid(pairs), kThreads, 0, st>>>((float2*)psi, pairs, q, F, m00, m01, m10,
                                                                            m11);
        }
      } else {
        const double2 m00 = make_double2(mat[0], mat[1]), m01 = make_double2(mat[2], mat[3]);
        const double2 m10 = make_double2(mat[4], mat[5]), m11 = make_double2(mat[6], mat[7]);
        // complex128 is bound by the FP64 rate: use the cheapest form the matrix allows
        const bool real = mat[1] == 0 && mat[3] == 0 && mat[5] == 0 && mat[7] == 0;
        const bool rxf = mat[1] == 0 && mat[7] == 0 && mat[2] == 0 && mat[4] == 0;
        const bool hada = real && mat[0] == mat[2] && mat[0] == mat[4] && mat[6] == -mat[0];
        const int k01 = unit_code(mat[2], mat[3]), k10 = unit_code(mat[4], mat[5]);
        const bool perm = mat[0] == 0 && mat[1] == 0 && mat[6] == 0 && mat[7] == 0 && k01 >= 0 && k10 >= 0;
        if (perm)
          gate1_perm_kernel<double><<<gate_grid(pairs), kThreads, 0, st>>>((double2*)psi, pairs, q, F, (uint32_t)k01,
                                                                          (uint32_t)k10);
        else if (hada)
          gate1_pair_kernel<double, 3><<<gate_grid(pairs), kThreads, 0, st>>>((double2*)psi, pairs, q, F, m00, m01,
                                                                             m10, m11);
        else if (real)
          gate1_pair_kernel<double, 1><<<gate_grid(pairs), kThreads, 0, st>>>((double2*)psi, pairs, q, F, m00, m01,
                                                                             m10, m11);
        else if (rxf)
          gate1_pair_kernel<double, 2><<<gate_grid(pairs), kThreads, 0, st>>>((double2*)psi, pairs, q, F, m00, m01,
                                                                             m10, m11);
        else
          gate1_pair_kernel<double, 0><<<gate_grid(pairs), kThreads, 0, st>>>((double2*)psi, pairs, q, F, m00, m01,
                                                                             m10, m11);
      }
      QS_CUDA(cudaGetLastError());
      return QS_OK;
    }
  }
  Mat4 M;
  const int D = 1 << nt;
  for (int i = 0; i < D * D; ++i) {
    M.re[i] = mat[2 * i];
    M.im[i] = mat[2 * i + 1];
  }
  const uint64_t groups = 1ull << (n - nt);
  const int grid = blocks_for(groups);
  const int g = grid > 65535 * 16 ? 65535 * 16 : grid;
  if (dt == QS_C64) {
    if (nt == 1)
      gate_dense_kernel<float, 1><<<g, kThreads, 0, st>>>((float2*)psi, n, t[0], t[0], cmask, M);
    else
      gate_dense_kernel<float, 2><<<g, kThreads, 0, st>>>((float2*)psi, n, t[0], t[1], cmask, M);
  } else {
    if (nt == 1)
      gate_dense_kernel<double, 1><<<g, kThreads, 0, st>>>((double2*)psi, n, t[0], t[0], cmask, M);
    else
      gate_dense_kernel<double, 2><<<g, kThreads, 0, st>>>((double2*)psi, n, t[0], t[1], cmask, M);
  }
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

qs_status launch_gate_diag(qs_dtype dt, void* psi, int n, int nt, const int* t, uint64_t cmask, const double* diag,
                           cudaStream_t st) {
  {
    // amplitudes left unchanged are skipped: a single-qubit diagonal with first
    // entry 1 (Z, S, T, phase shift) changes only the target's |1> half
    const bool first_one = nt == 1 && diag[0] == 1.0 && diag[1] == 0.0;
    uint64_t fixed = cmask, ones = cmask;
    if (first_one) {
      fixed |= 1ull << t[0];
      ones |= 1ull << t[0];
    }
    FixedBits F;
    if (fixed_from(fixed, ones, &F)) {
      const uint64_t amps = 1ull << (n - F.k);
      const int t0 = t[0], t1 = nt == 2 ? t[1] : t[0];
      if (dt == QS_C64) {
        float2 d[4];
        for (int i = 0; i < 4; ++i) d[i] = i < (1 << nt) ? make_float2((float)diag[2 * i], (float)diag[2 * i + 1])
                                                          : make_float2(1.f, 0.f);
        FixedBits F2;
        if (!(fixed & 1ull) && n - F.k >= 1 && fixed_from(fixed | 1ull, ones, &F2))
          diag_fast_kernel<float, true><<<gate_grid(amps / 2), kThreads, 0, st>>>((float2*)psi, amps / 2, nt, t0, t1, F2,
                                                                                  d[0], d[1], d[2], d[3]);
        else
          diag_fast_kernel<float, false><<<gate_grid(amps), kThreads, 0, st>>>((float2*)psi, amps, nt, t0, t1, F, d[0],
                                                                              d[1], d[2], d[3]);
      } else {
        double2 d[4];
        uint32_t codes = 0;
        bool unit = true;
        for (int i = 0; i < 4; ++i) {
          d[i] = i < (1 << nt) ? make_double2(diag[2 * i], diag[2 * i + 1]) : make_double2(1.0, 0.0);
          const int k = unit_code(d[i].x, d[i].y);
          unit = unit && k >= 0;
          codes |= (uint32_t)(k < 0 ? 0 : k) << (2 * i);
        }
        if (unit)
          diag_unit_kernel<double><<<gate_grid(amps), kThreads, 0, st>>>((double2*)psi, amps, nt, t0, t1, F, codes);
        else
          diag_fast_kernel<double, false><<<gate_grid(amps), kThreads, 0, st>>>((double2*)psi, amps, nt, t0, t1, F,
                                                                               d[0], d[1], d[2], d[3]);
      }
      QS_CUDA(cudaGetLastError());
      return QS_OK;
    }
  }
  Mat4 D;
  for (int i = 0; i < (1 << nt); ++i) {
    D.re[i] = diag[2 * i];
    D.im[i] = diag[2 * i + 1];
  }
  const int grid = blocks_for(1ull << n);
  const int g = grid > 65535 * 16 ? 65535 * 16 : grid;
  if (dt == QS_C64)
    gate_diag_kernel<float><<<g, kThreads, 0, st>>>((float2*)psi, n, nt, t[0], nt == 2 ? t[1] : 0, cmask, D);
  else
    gate_diag_kernel<double><<<g, kThreads, 0, st>>>((double2*)psi, n, nt, t[0], nt == 2 ? t[1] : 0, cmask, D);
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

qs_status launch_set_basis(qs_dtype dt, void* psi, int n, uint64_t index, cudaStream_t st) {
  const size_t bytes = (size_t)(dt == QS_C64 ? 8 : 16) << n;
  QS_CUDA(cudaMemsetAsync(psi, 0, bytes, st));
  if (dt == QS_C64)
    set_one_kernel<float><<<1, 1, 0, st>>>((float2*)psi, index);
  else
    set_one_kernel<double><<<1, 1, 0, st>>>((double2*)psi, index);
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

qs_status launch_set_plus(qs_dtype dt, void* psi, int n, cudaStream_t st) {
  const int grid = blocks_for(1ull << n);
  const int g = grid > 65535 * 16 ? 65535 * 16 : grid;
  const double amp = std::ldexp(1.0, -n / 2) * ((n & 1) ? 0.70710678118654752440 : 1.0);
  if (dt == QS_C64)
    set_plus_kernel<float><<<g, kThreads, 0, st>>>((float2*)psi, 1ull << n, (float)amp);
  else
    set_plus_kernel<double><<<g, kThreads, 0, st>>>((double2*)psi, 1ull << n, amp);
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

int ham_grid_size(int n) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms <= 0) sms = 1;
  const uint64_t need = ((1ull << n) + kThreads - 1) / kThreads;
  const uint64_t g = (uint64_t)sms * 8;
  return (int)(need < g ? need : g);
}

qs_status launch_ham_apply(qs_dtype dt, const void* psi, void* lam, int n, const DevHamGroup* groups, int n_groups,
                           const DevHamTerm* terms, double* partials, int grid, cudaStream_t st) {
  if (dt == QS_C64)
    ham_apply_kernel<float><<<grid, kThreads, 0, st>>>((const float2*)psi, (float2*)lam, n, groups, n_groups, terms,
                                                       partials);
  else
    ham_apply_kernel<double><<<grid, kThreads, 0, st>>>((const double2*)psi, (double2*)lam, n, groups, n_groups,
                                                        terms, partials);
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

qs_status launch_ham_apply_multi(qs_dtype dt, const HamMultiArgs* d_argv, int count, int grid, cudaStream_t st) {
  if (count <= 0) return QS_OK;
  const dim3 g((unsigned)grid, (unsigned)count);
  if (dt == QS_C64)
    ham_apply_multi_kernel<float><<<g, kThreads, 0, st>>>(d_argv);
  else
    ham_apply_multi_kernel<double><<<g, kThreads, 0, st>>>(d_argv);
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

qs_status launch_reduce_multi(const ReduceMultiArgs* d_argv, int count, int max_slots, cudaStream_t st) {
  if (count <= 0 || max_slots <= 0) return QS_OK;
  const dim3 g((unsigned)((max_slots * 32 + 255) / 256), (unsigned)count);
  reduce_multi_kernel<<<g, 256, 0, st>>>(d_argv);
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

qs_status launch_gather_multi(const GatherMultiArgs* d_argv, int count, int max_params, cudaStream_t st) {
  if (count <= 0 || max_params <= 0) return QS_OK;
  const dim3 g((unsigned)((max_params + 127) / 128), (unsigned)count);
  gather_multi_kernel<<<g, 128, 0, st>>>(d_argv);
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

qs_status launch_set_zero_multi(qs_dtype dt, void* base, int n, int count, cudaStream_t st) {
  if (count <= 0) return QS_OK;
  const size_t bytes = ((size_t)(dt == QS_C64 ? 8 : 16) << n) * (size_t)count;
  QS_CUDA(cudaMemsetAsync(base, 0, bytes, st));
  const int blocks = (count + 255) / 256;
  if (dt == QS_C64)
    set_zero_multi_kernel<float><<<blocks, 256, 0, st>>>((float2*)base, 1ull << n, count);
  else
    set_zero_multi_kernel<double><<<blocks, 256, 0, st>>>((double2*)base, 1ull << n, count);
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

qs_status launch_inner(qs_dtype dt, const void* a, const void* b, int n, double* partials, int grid,
                       cudaStream_t st) {
  if (dt == QS_C64)
    inner_kernel<float><<<grid, kThreads, 0, st>>>((const float2*)a, (const float2*)b, n, partials);
  else
    inner_kernel<double><<<grid, kThreads, 0, st>>>((const double2*)a, (const double2*)b, n, partials);
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

qs_status launch_qubit_rdm(qs_dtype dt, const void* psi, int n, int q, double* partials, int grid,
                           cudaStream_t st) {
  if (dt == QS_C64)
    qubit_rdm_kernel<float><<<grid, kThreads, 0, st>>>((const float2*)psi, n, q, partials);
  else
    qubit_rdm_kernel<double><<<grid, kThreads, 0, st>>>((const double2*)psi, n, q, partials);
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

qs_status launch_norm2(qs_dtype dt, const void* a, int n, double* partials, int grid, cudaStream_t st) {
  if (dt == QS_C64)
    norm2_kernel<float><<<grid, kThreads, 0, st>>>((const float2*)a, n, partials);
  else
    norm2_kernel<double><<<grid, kThreads, 0, st>>>((const double2*)a, n, partials);
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

qs_status launch_reduce_slots(const double* partials, int n_slots, int nb, const double* scale, double* out,
                              cudaStream_t st) {
  if (n_slots <= 0) return QS_OK;
  const int threads = 256;
  const int blocks = (n_slots * 32 + threads - 1) / threads;
  reduce_slots_kernel<<<blocks, threads, 0, st>>>(partials, n_slots, nb, scale, out);
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

qs_status launch_param_gather(const double* gate_grad, const int* row_ptr, const int* gate_idx,
                              const double* gate_coef, int n_params, double* grad, cudaStream_t st) {
  if (n_params <= 0) return QS_OK;
  param_gather_kernel<<<(n_params + 127) / 128, 128, 0, st>>>(gate_grad, row_ptr, gate_idx, gate_coef, n_params,
                                                              grad);
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

qs_status launch_cut_values(uint8_t* cut, int n, const int* d_edges, int n_edges, cudaStream_t st) {
  const int grid = blocks_for(1ull << n);
  const int g = grid > 65535 * 8 ? 65535 * 8 : grid;
  cut_values_kernel<<<g, kThreads, 2 * n_edges * sizeof(int), st>>>(cut, n, d_edges, n_edges);
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

qs_status launch_max_u8(const uint8_t* v, uint64_t n, int* d_out, cudaStream_t st) {
  QS_CUDA(cudaMemsetAsync(d_out, 0, sizeof(int), st));
  const uint64_t want = (n / 16 + kThreads - 1) / kThreads;
  const int g = (int)(want < 1 ? 1 : (want > 4096 ? 4096 : want));
  max_u8_kernel<<<g, kThreads, 0, st>>>(v, n, d_out);
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

qs_status launch_measure(qs_dtype dt, void* psi, int n, int q, uint64_t seed, double* scratch, int nb,
                         cudaStream_t st) {
  double* out = scratch + 2 * nb;
  if (dt == QS_C64) {
    measure_mass_kernel<float><<<nb, kThreads, 0, st>>>((const float2*)psi, n, q, scratch);
    measure_decide_kernel<<<1, 32, 0, st>>>(scratch, nb, seed, out);
    measure_collapse_kernel<float><<<nb, kThreads, 0, st>>>((float2*)psi, n, q, out);
  } else {
    measure_mass_kernel<double><<<nb, kThreads, 0, st>>>((const double2*)psi, n, q, scratch);
    measure_decide_kernel<<<1, 32, 0, st>>>(scratch, nb, seed, out);
    measure_collapse_kernel<double><<<nb, kThreads, 0, st>>>((double2*)psi, n, q, out);
  }
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

size_t sample_scratch_doubles(int n) {
  const int cb = n < kChunkBits ? n : kChunkBits;
  return (1ull << (n - cb)) + 1;
}

qs_status launch_sample(qs_dtype dt, const void* psi, int n, uint64_t shots, uint64_t seed, double* scratch,
                        uint64_t* d_out, cudaStream_t st) {
  const int cb = n < kChunkBits ? n : kChunkBits;
  const uint64_t n_chunks = 1ull << (n - cb);
  const int threads = 256;
  const uint64_t cblocks = (n_chunks * 32 + threads - 1) / threads;
  if (dt == QS_C64)
    chunk_sum_kernel<float><<<(unsigned)cblocks, threads, 0, st>>>((const float2*)psi, n, scratch);
  else
    chunk_sum_kernel<double><<<(unsigned)cblocks, threads, 0, st>>>((const double2*)psi, n, scratch);
  QS_CUDA(cudaGetLastError());
  chunk_scan_kernel<<<1, 1024, 0, st>>>(scratch, n_chunks);
  QS_CUDA(cudaGetLastError());
  if (shots) {
    const uint64_t sblocks = (shots * 32 + threads - 1) / threads;
    if (dt == QS_C64)
      sample_kernel<float><<<(unsigned)sblocks, threads, 0, st>>>((const float2*)psi, n, scratch, shots, seed, d_out);
    else
      sample_kernel<double><<<(unsigned)sblocks, threads, 0, st>>>((const double2*)psi, n, scratch, shots, seed,
                                                                   d_out);
    QS_CUDA(cudaGetLastError());
  }
  return QS_OK;
}

}  // namespace qs
