// Dense k-qubit blocks: psi <- U psi for a 2^k x 2^k complex matrix U on k
// target qubits (§2.3.4 custom gates; a block is also what gate fusion
// produces, the product of the gates that act inside k qubits).
//
// Viewed as a matrix, the state is X[r][j] (r: the other n - k index bits, j:
// the target bits) and the block is the product Y = X U^T: a dense
// contraction.  On sm_103a complex64 blocks with k = 4 or 5 run on the 5th
// generation tensor cores (tcgen05.mma, kind::tf32) in real form,
//   Y_re + i Y_im  <-  [X_re X_im] . [[U_re^T, U_im^T], [-U_im^T, U_re^T]],
// with every float32 operand split into a tf32 head and a tf32 tail
// (x = h + t) and three products h.h + h.t + t.h accumulated in float32 in
// tensor memory: the dropped t.t term and the tail rounding are ~2^-21
// relative, float32 accuracy overall.  One CTA of 256 threads takes tiles of
// 128 rows, two threads per row: each gathers half of its row from HBM, splits
// it and stores it in the no-swizzle K-major core-matrix layout; one thread
// issues the MMAs and commits them to an mbarrier; each warp reads its 32 TMEM
// lanes back (tcgen05.ld 32x32b, the columns of its half) and stores those
// outputs in place (k = 4; k = 5 runs the warp-specialised form below, whose
// roles overlap the chain of consecutive tiles).  Every other
// case (complex128, other k, small n) runs on the CUDA cores in the state's
// own precision.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "handles.h"

using namespace qs;

namespace {

constexpr int kDenseMaxK = 6;
constexpr int kTcRows = 128;     // rows (MMA M) per tile
// two threads per row: thread t takes row t & 127 and half t >> 7 of its
// amplitudes; warp w reads TMEM lanes 32 (w % 4) .. + 31 (its lane quarter),
// columns of its half
constexpr int kTcThreads = 256;
constexpr long long kWaitLimit = 1ll << 26;  // bounded mbarrier polling

// ------------------------------------------------------------------ PTX helpers

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Shared-memory matrix descriptor, no swizzle, K-major: lbo = byte distance
// between core matrices adjacent along K, sbo = between 8-row groups.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
  return d;                // base offset 0, layout type 0 (no swizzle)
}

// Instruction descriptor: kind::tf32, f32 accumulator, A and B K-major.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4)               // D format f32
         | (2u << 7)             // A format tf32
         | (2u << 10)            // B format tf32
         | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, int accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive f32 columns of this warp's 32 TMEM lanes (lane = thread)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Byte offset of element (row, kk) in a K-major operand with KR f32 columns:
// 8-row x 16-byte core matrices, K-adjacent cores 128 bytes apart (LBO),
// 8-row groups KR * 32 bytes apart (SBO).
__device__ __forceinline__ uint32_t op_offset(int row, int kk, int KR) {
  return (uint32_t)((row >> 3) * (KR * 32) + (kk >> 2) * 128 + (row & 7) * 16 + (kk & 3) * 4);
}

// index of the amplitude with other-bits value r and target-bits value j:
// both deposited by precomputed tables (others: per bit of r)
struct DenseGeom {
  int n, k;
  int n_other;
  int pair0;  // target 0 is qubit 0 and the state 16-byte aligned: columns (2c, 2c + 1) form one 16-byte word
  uint64_t tgt_off[1 << kDenseMaxK];  // deposit(j, targets)
  uint8_t other_bit[64];              // bit position of the b-th other bit
};

__device__ __forceinline__ uint64_t deposit_other(const DenseGeom& G, uint64_t r) {
  uint64_t x = 0;
  for (int b = 0; b < G.n_other; ++b) x |= ((r >> b) & 1ull) << G.other_bit[b];
  return x;
}

// ------------------------------------------------------------------ tensor-core kernel

template <int K>
struct TcCfg {
  static constexpr int KB = 1 << K;     // complex columns
  static constexpr int KR = 2 * KB;     // real K = real N
  static constexpr int A_BYTES = kTcRows * KR * 4;
  static constexpr int B_BYTES = KR * KR * 4;
  static constexpr int TMEM_COLS = KR < 32 ? 32 : KR;
  // + barrier, tile-bit tables, slack for align
  static constexpr size_t SMEM = 2 * (size_t)A_BYTES + 2 * (size_t)B_BYTES + 64 + 3 * 256 * 8 + 128;
};

template <int K>
__global__ void __launch_bounds__(kTcThreads) dense_tc_kernel(float2* __restrict__ psi, const DenseGeom G,
                                                              const double2* __restrict__ U, uint64_t n_tiles,
                                                              int* __restrict__ err) {
  using Cfg = TcCfg<K>;
  constexpr int KB = Cfg::KB, KR = Cfg::KR;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
  unsigned char* a_hi = smem;
  unsigned char* a_lo = a_hi + Cfg::A_BYTES;
  unsigned char* b_hi = a_lo + Cfg::A_BYTES;
  unsigned char* b_lo = b_hi + Cfg::B_BYTES;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(b_lo + Cfg::B_BYTES);
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(mbar + 1);
  uint64_t* s_dep = mbar + 8;  // [3][256]: tile bits 8c.. deposited into the other qubits
  __shared__ int s_abort;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row = tid & (kTcRows - 1), half = tid / kTcRows;
  constexpr int KH = KB / 2;  // amplitudes per thread
  // row index r = tile * 128 + row: offset deposit(row) | deposit(tile << 7)
  // (tiles < 2^24: n - k - 7 <= 23)
  for (int e = tid; e < 3 * 256; e += kTcThreads) {
    const int c = e >> 8, v = e & 255;
    uint64_t xd = 0;
    for (int i = 0; i < 8; ++i) {
      const int b = 7 + 8 * c + i;
      if (((v >> i) & 1) && b < G.n_other) xd |= 1ull << G.other_bit[b];
    }
    s_dep[e] = xd;
  }
  const uint64_t row_dep = deposit_other(G, (uint64_t)row);
  auto tile_dep = [&](uint64_t t) {
    return s_dep[t & 255] | s_dep[256 + ((t >> 8) & 255)] | s_dep[512 + ((t >> 16) & 255)];
  };
  auto gather = [&](uint64_t b, float2(&dst)[KH]) {
    if (G.pair0) {  // column pairs (2c, 2c + 1) as one 16-byte word
#pragma unroll
      for (int c = 0; c < KH / 2; ++c) {
        const float4 v = *reinterpret_cast<const float4*>(psi + (b | G.tgt_off[half * KH + 2 * c]));
        dst[2 * c] = make_float2(v.x, v.y);
        dst[2 * c + 1] = make_float2(v.z, v.w);
      }
    } else {
#pragma unroll
      for (int j = 0; j < KH; ++j) dst[j] = psi[b | G.tgt_off[half * KH + j]];
    }
  };
  // B[n][kk] = W[kk][n], W = real form of U^T (see the file comment); split h/t
  for (int e = tid; e < KR * KR; e += kTcThreads) {
    const int n = e / KR, kk = e % KR;
    const int i = n >> 1, cp = n & 1, j = kk >> 1, c = kk & 1;
    const double2 u = U[i * KB + j];
    const float w = (float)(cp == 0 ? (c == 0 ? u.x : -u.y) : (c == 0 ? u.y : u.x));
    const float h = tf32_round(w);
    const uint32_t off = op_offset(n, kk, KR);
    *reinterpret_cast<float*>(b_hi + off) = h;
    *reinterpret_cast<float*>(b_lo + off) = tf32_round(w - h);
  }
  if (tid == 0) {
    s_abort = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_tmem)),
                 "r"((uint32_t)Cfg::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;
  constexpr uint32_t idesc = idesc_tf32(kTcRows, KR);
  const uint32_t lbo = 128, sbo = KR * 32;
  const uint32_t a_hi_s = smem_u32(a_hi), a_lo_s = smem_u32(a_lo), b_hi_s = smem_u32(b_hi), b_lo_s = smem_u32(b_lo);
  uint32_t phase = 0;

  // Software pipeline: the rows of the next tile are loaded into registers
  // while the tensor cores work on this one and its results are stored.
  uint64_t tile = blockIdx.x;
  float2 x[KH];
  uint64_t base = 0;
  if (tile < n_tiles) {
    base = row_dep | tile_dep(tile);
    gather(base, x);
  }
  for (; tile < n_tiles; tile += gridDim.x) {
    // split this thread's half row into tf32 head and tail, K-major core-matrix layout
#pragma unroll
    for (int c = 0; c < KH / 2; ++c) {
      const float2 p0 = x[2 * c], p1 = x[2 * c + 1];
      float4 h, t;
      h.x = tf32_round(p0.x);
      h.y = tf32_round(p0.y);
      h.z = tf32_round(p1.x);
      h.w = tf32_round(p1.y);
      t.x = tf32_round(p0.x - h.x);
      t.y = tf32_round(p0.y - h.y);
      t.z = tf32_round(p1.x - h.z);
      t.w = tf32_round(p1.y - h.w);
      const uint32_t off = op_offset(row, half * KB + 4 * c, KR);
      *reinterpret_cast<float4*>(a_hi + off) = h;
      *reinterpret_cast<float4*>(a_lo + off) = t;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
#pragma unroll
      for (int s = 0; s < KR / 8; ++s) {
        const uint32_t ko = s * 256;  // 8 tf32 = two 16-byte core columns
        const uint64_t ah = smem_desc(a_hi_s + ko, lbo, sbo), al = smem_desc(a_lo_s + ko, lbo, sbo);
        const uint64_t bh = smem_desc(b_hi_s + ko, lbo, sbo), bl = smem_desc(b_lo_s + ko, lbo, sbo);
        mma_tf32(tmem, ah, bh, idesc, s > 0);
        mma_tf32(tmem, ah, bl, idesc, 1);
        mma_tf32(tmem, al, bh, idesc, 1);
      }
      mma_commit(smem_u32(mbar));
    }
    // next tile's rows in flight during the MMAs and the stores below
    const uint64_t next = tile + gridDim.x;
    uint64_t nbase = 0;
    float2 xn[KH];
    if (next < n_tiles) {
      nbase = row_dep | tile_dep(next);
      gather(nbase, xn);
    } else {
#pragma unroll
      for (int j = 0; j < KH; ++j) xn[j] = make_float2(0.f, 0.f);
    }
    // every thread waits for the MMAs (bounded)
    bool ok = false;
    for (long long it = 0; it < kWaitLimit; ++it)
      if (mbar_try_wait(smem_u32(mbar), phase)) {
        ok = true;
        break;
      }
    phase ^= 1u;
    if (!ok) atomicExch(&s_abort, 1);
    __syncthreads();
    if (s_abort) {
      if (tid == 0) {
        atomicExch(err, 1);
        // the committed MMAs may still be reading shared memory and writing
        // tensor memory: wait for their commit once more (bounded) before the
        // tensor memory is freed below
        for (long long it = 0; it < kWaitLimit; ++it)
          if (mbar_try_wait(smem_u32(mbar), phase ^ 1u)) break;
      }
      break;
    }
    tc_fence_after();
    // rows back from tensor memory: lane 32 (warp % 4) + l = row, columns 2i,
    // 2i + 1 = output i, this half's outputs only
    const uint32_t trow = tmem + ((uint32_t)((warp & 3) * 32) << 16);
#pragma unroll
    for (int c0 = half * KB; c0 < half * KB + KB; c0 += 16) {
      float v[16];
      tmem_ld16(trow + c0, v);
      if (G.pair0) {
#pragma unroll
        for (int q = 0; q < 8; q += 2)
          *reinterpret_cast<float4*>(psi + (base | G.tgt_off[c0 / 2 + q])) =
              make_float4(v[2 * q], v[2 * q + 1], v[2 * q + 2], v[2 * q + 3]);
      } else {
#pragma unroll
        for (int q = 0; q < 8; ++q) psi[base | G.tgt_off[c0 / 2 + q]] = make_float2(v[2 * q], v[2 * q + 1]);
      }
    }
    tc_fence_before();
    __syncthreads();
    base = nbase;
#pragma unroll
    for (int j = 0; j < KH; ++j) x[j] = xn[j];
  }
  tc_fence_after();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"((uint32_t)Cfg::TMEM_COLS)
                 : "memory");
  (void)lane;
}

// ------------------------------------------------------------------ warp-specialised tensor-core kernel
//
// The same contraction with the per-tile chain split over roles, so that
// gathering, tensor-core work and write-back of consecutive tiles overlap in
// one CTA: 16 producer warps (four threads per row) gather a tile's
// rows into one of two operand stages and split them; one MMA warp issues the
// three products per K-step into one of two TMEM accumulators and commits them
// to the stage's "empty" and the accumulator's "full" mbarriers; 4 epilogue
// warps (warp w: TMEM lanes 32 w..) read the accumulator back, store the rows
// and release it.  Every wait is bounded; a wait that runs out records an
// error and ends the role's loop.
constexpr int kWsProducers = 512, kWsThreads = kWsProducers + 32 + 128;  // producers: 4 threads per row

template <int K>
struct WsCfg {
  static constexpr int KB = 1 << K, KR = 2 * KB;
  static constexpr int A_BYTES = kTcRows * KR * 4, B_BYTES = KR * KR * 4;
  static constexpr int TMEM_COLS = 2 * KR < 32 ? 32 : 2 * KR;
  static constexpr size_t SMEM = 4 * (size_t)A_BYTES + 2 * (size_t)B_BYTES + 16 * 8 + 3 * 256 * 8 + 128;
};

__device__ __forceinline__ bool ws_wait(uint32_t mbar, uint32_t parity) {
  for (long long it = 0; it < kWaitLimit; ++it)
    if (mbar_try_wait(mbar, parity)) return true;
  return false;
}
__device__ __forceinline__ void ws_arrive(uint32_t mbar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(mbar) : "memory");
}

template <int K>
__global__ void __launch_bounds__(kWsThreads, 1) dense_ws_kernel(float2* __restrict__ psi, const DenseGeom G,
                                                                 const double2* __restrict__ U, uint64_t n_tiles,
                                                                 int* __restrict__ err) {
  using Cfg = WsCfg<K>;
  constexpr int KB = Cfg::KB, KR = Cfg::KR, KQ = KB / 4;  // amplitudes per producer thread
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
  // stage st: head at smem + 2 st A_BYTES, tail right after it (arithmetic, not
  // an indexed array, which would live in local memory)
  auto a_hi = [&](int st) { return smem + (size_t)(2 * st) * Cfg::A_BYTES; };
  auto a_lo = [&](int st) { return smem + (size_t)(2 * st + 1) * Cfg::A_BYTES; };
  unsigned char* b_hi = smem + 4 * Cfg::A_BYTES;
  unsigned char* b_lo = b_hi + Cfg::B_BYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(b_lo + Cfg::B_BYTES);
  // full[s], empty[s], tfull[a], tempty[a]
  const uint32_t full0 = smem_u32(bars), empty0 = smem_u32(bars + 2), tfull0 = smem_u32(bars + 4),
                 tempty0 = smem_u32(bars + 6);
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(bars + 8);
  // row index r = tile * 128 + row: its other-qubit offset is deposit(row) |
  // deposit(tile << 7); the tile part comes from three tables of 8 tile bits
  // (tiles < 2^24: n - k - 7 <= 23)
  uint64_t* s_dep = bars + 16;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int e = tid; e < 3 * 256; e += kWsThreads) {
    const int c = e >> 8, v = e & 255;
    uint64_t x = 0;
    for (int i = 0; i < 8; ++i) {
      const int b = 7 + 8 * c + i;
      if (((v >> i) & 1) && b < G.n_other) x |= 1ull << G.other_bit[b];
    }
    s_dep[e] = x;
  }
  auto tile_dep = [&](uint64_t t) {
    return s_dep[t & 255] | s_dep[256 + ((t >> 8) & 255)] | s_dep[512 + ((t >> 16) & 255)];
  };

  for (int e = tid; e < KR * KR; e += kWsThreads) {  // B = real form of U^T, split h/t (as above)
    const int n = e / KR, kk = e % KR;
    const int i = n >> 1, cp = n & 1, j = kk >> 1, c = kk & 1;
    const double2 u = U[i * KB + j];
    const float w = (float)(cp == 0 ? (c == 0 ? u.x : -u.y) : (c == 0 ? u.y : u.x));
    const float h = tf32_round(w);
    const uint32_t off = op_offset(n, kk, KR);
    *reinterpret_cast<float*>(b_hi + off) = h;
    *reinterpret_cast<float*>(b_lo + off) = tf32_round(w - h);
  }
  if (tid == 0) {
    for (int q = 0; q < 2; ++q) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(full0 + 8 * q), "r"(kWsProducers / 32) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(empty0 + 8 * q) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tfull0 + 8 * q) : "memory");
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(tempty0 + 8 * q) : "memory");
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(s_tmem)),
                 "r"((uint32_t)Cfg::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *s_tmem;
  bool bad = false;

  if (tid < kWsProducers) {
    // ------------------------------------------------------------ producers
    // thread: row tid % 128, quarter tid / 128 of its amplitudes; the two
    // following tiles' amplitudes are loaded before this tile's are split and
    // stored, so three tiles' gathers are in flight per thread
    const int row = tid & (kTcRows - 1), qt = tid / kTcRows;
    const uint64_t row_dep = deposit_other(G, (uint64_t)row);
    float2 xn[KQ], xnn[KQ];
    uint64_t tile = blockIdx.x;
    auto gather = [&](uint64_t t, float2(&dst)[KQ]) {
      if (t >= n_tiles) return;
      const uint64_t base = row_dep | tile_dep(t);
      if (G.pair0) {
#pragma unroll
        for (int c = 0; c < KQ / 2; ++c) {
          const float4 v = *reinterpret_cast<const float4*>(psi + (base | G.tgt_off[qt * KQ + 2 * c]));
          dst[2 * c] = make_float2(v.x, v.y);
          dst[2 * c + 1] = make_float2(v.z, v.w);
        }
      } else {
#pragma unroll
        for (int j = 0; j < KQ; ++j) dst[j] = psi[base | G.tgt_off[qt * KQ + j]];
      }
    };
    gather(tile, xn);
    gather(tile + gridDim.x, xnn);
    int i = 0;
    for (; tile < n_tiles; tile += gridDim.x, ++i) {
      const int st = i & 1;
      float2 x[KQ];
#pragma unroll
      for (int j = 0; j < KQ; ++j) {
        x[j] = xn[j];
        xn[j] = xnn[j];
      }
      gather(tile + 2ull * gridDim.x, xnn);
      if (i >= 2 && !ws_wait(empty0 + 8 * st, (uint32_t)(((i - 2) >> 1) & 1))) {
        bad = true;
        break;
      }
#pragma unroll
      for (int c = 0; c < KQ / 2; ++c) {
        const float2 p0 = x[2 * c], p1 = x[2 * c + 1];
        float4 h, t;
        h.x = tf32_round(p0.x);
        h.y = tf32_round(p0.y);
        h.z = tf32_round(p1.x);
        h.w = tf32_round(p1.y);
        t.x = tf32_round(p0.x - h.x);
        t.y = tf32_round(p0.y - h.y);
        t.z = tf32_round(p1.x - h.z);
        t.w = tf32_round(p1.y - h.w);
        const uint32_t off = op_offset(row, qt * (KB / 2) + 4 * c, KR);
        *reinterpret_cast<float4*>(a_hi(st) + off) = h;
        *reinterpret_cast<float4*>(a_lo(st) + off) = t;
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the tensor cores
      __syncwarp();
      if (lane == 0) ws_arrive(full0 + 8 * st);
    }
  } else if (tid < kWsProducers + 32) {
    // ------------------------------------------------------------ MMA warp
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_tf32(kTcRows, KR);
      const uint32_t lbo = 128, sbo = KR * 32;
      const uint32_t bh_s = smem_u32(b_hi), bl_s = smem_u32(b_lo);
      int i = 0;
      for (uint64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++i) {
        const int st = i & 1, ac = i & 1;
        if (!ws_wait(full0 + 8 * st, (uint32_t)((i >> 1) & 1))) {
          bad = true;
          break;
        }
        if (i >= 2 && !ws_wait(tempty0 + 8 * ac, (uint32_t)(((i - 2) >> 1) & 1))) {
          bad = true;
          break;
        }
        tc_fence_after();
        const uint32_t ah_s = smem_u32(a_hi(st)), al_s = smem_u32(a_lo(st));
        const uint32_t d = tmem + (uint32_t)(ac * KR);
#pragma unroll
        for (int s = 0; s < KR / 8; ++s) {
          const uint32_t ko = s * 256;
          const uint64_t ah = smem_desc(ah_s + ko, lbo, sbo), al = smem_desc(al_s + ko, lbo, sbo);
          const uint64_t bh = smem_desc(bh_s + ko, lbo, sbo), bl = smem_desc(bl_s + ko, lbo, sbo);
          mma_tf32(d, ah, bh, idesc, s > 0);
          mma_tf32(d, ah, bl, idesc, 1);
          mma_tf32(d, al, bh, idesc, 1);
        }
        mma_commit(empty0 + 8 * st);  // the stage may be refilled once these MMAs have read it
        mma_commit(tfull0 + 8 * ac);  // the accumulator holds the tile
      }
      // the last commits before the tensor memory is freed (bounded)
      if (i >= 1) (void)ws_wait(tfull0 + 8 * ((i - 1) & 1), (uint32_t)(((i - 1) >> 1) & 1));
    }
    __syncwarp();
  } else {
    // ------------------------------------------------------------ epilogue warps
    // a warp may access only the TMEM lanes of its quarter, 32 (warp % 4) ..; the
    // four epilogue warps (9..12) cover the quarters 1, 2, 3, 0
    const int ew = warp & 3;
    const int row = ew * 32 + lane;
    const uint64_t row_dep = deposit_other(G, (uint64_t)row);
    int i = 0;
    for (uint64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++i) {
      const int ac = i & 1;
      if (!ws_wait(tfull0 + 8 * ac, (uint32_t)((i >> 1) & 1))) {
        bad = true;
        break;
      }
      tc_fence_after();
      const uint64_t base = row_dep | tile_dep(tile);
      const uint32_t trow = tmem + ((uint32_t)(ew * 32) << 16) + (uint32_t)(ac * KR);
#pragma unroll
      for (int c0 = 0; c0 < KR; c0 += 16) {
        float v[16];
        tmem_ld16(trow + c0, v);
        if (G.pair0) {
#pragma unroll
          for (int q = 0; q < 8; q += 2)
            *reinterpret_cast<float4*>(psi + (base | G.tgt_off[c0 / 2 + q])) =
                make_float4(v[2 * q], v[2 * q + 1], v[2 * q + 2], v[2 * q + 3]);
        } else {
#pragma unroll
          for (int q = 0; q < 8; ++q) psi[base | G.tgt_off[c0 / 2 + q]] = make_float2(v[2 * q], v[2 * q + 1]);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) ws_arrive(tempty0 + 8 * ac);
    }
  }
  if (bad) atomicExch(err, 1);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)Cfg::TMEM_COLS)
                 : "memory");
}

// ------------------------------------------------------------------ CUDA-core kernel

template <class T>
struct Cplx;
template <>
struct Cplx<float> {
  using V = float2;
};
template <>
struct Cplx<double> {
  using V = double2;
};

// One thread per row: the row is staged in shared memory, each output is a
// dot product with a row of U (held in shared memory in the state's precision).
template <class T>
__global__ void dense_cc_kernel(typename Cplx<T>::V* __restrict__ psi, const DenseGeom G,
                                const double2* __restrict__ U, uint64_t n_rows) {
  using V = typename Cplx<T>::V;
  extern __shared__ __align__(16) unsigned char cc_smem_raw[];
  const int KB = 1 << G.k;
  V* sU = reinterpret_cast<V*>(cc_smem_raw);
  V* sRow = sU + KB * KB + threadIdx.x * KB;
  for (int e = threadIdx.x; e < KB * KB; e += blockDim.x) {
    const double2 u = U[e];
    sU[e].x = (T)u.x;
    sU[e].y = (T)u.y;
  }
  __syncthreads();
  for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < n_rows;
       r += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t base = deposit_other(G, r);
    for (int j = 0; j < KB; ++j) sRow[j] = psi[base | G.tgt_off[j]];
    for (int i = 0; i < KB; ++i) {
      T re = 0, im = 0;
      for (int j = 0; j < KB; ++j) {
        const V u = sU[i * KB + j], x = sRow[j];
        re = fma(u.x, x.x, re);
        re = fma(-u.y, x.y, re);
        im = fma(u.x, x.y, im);
        im = fma(u.y, x.x, im);
      }
      V o;
      o.x = re;
      o.y = im;
      psi[base | G.tgt_off[i]] = o;
    }
  }
}

size_t cc_smem(qs_dtype dt, int k, int threads) {
  const size_t KB = (size_t)1 << k, amp = dt == QS_C64 ? 8 : 16;
  return (KB * KB + (size_t)threads * KB) * amp;
}

int cc_threads(qs_dtype dt, int k) {
  const size_t KB = (size_t)1 << k, amp = dt == QS_C64 ? 8 : 16;
  int t = 128;
  while (t > 32 && (KB * KB + (size_t)t * KB) * amp > 160 * 1024) t >>= 1;
  return t;
}

template <int K>
qs_status launch_ws(float2* psi, const DenseGeom& G, const double2* dU, int* d_err, cudaStream_t st) {
  using Cfg = WsCfg<K>;
  const uint64_t n_tiles = (1ull << (G.n - K)) / kTcRows;
  int dev = 0, sms = 1;
  QS_CUDA(cudaGetDevice(&dev));
  QS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  QS_CUDA(cudaFuncSetAttribute(dense_ws_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM));
  const uint64_t grid = std::min<uint64_t>(n_tiles, (uint64_t)sms);  // one CTA per SM, looping over tiles
  dense_ws_kernel<K><<<(unsigned)grid, kWsThreads, Cfg::SMEM, st>>>(psi, G, dU, n_tiles, d_err);
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

template <int K>
qs_status launch_tc(float2* psi, const DenseGeom& G, const double2* dU, int* d_err, cudaStream_t st) {
  using Cfg = TcCfg<K>;
  const uint64_t n_rows = 1ull << (G.n - K);
  const uint64_t n_tiles = n_rows / kTcRows;
  int dev = 0, sms = 1, per_sm = 1;
  QS_CUDA(cudaGetDevice(&dev));
  QS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  QS_CUDA(cudaFuncSetAttribute(dense_tc_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM));
  // all of the unified L1 / shared memory as shared memory, so that two CTAs fit
  QS_CUDA(cudaFuncSetAttribute(dense_tc_kernel<K>, cudaFuncAttributePreferredSharedMemoryCarveout,
                               (int)cudaSharedmemCarveoutMaxShared));
  QS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dense_tc_kernel<K>, kTcThreads, Cfg::SMEM));
  // the CTAs the SM's shared memory holds (the query above has returned one
  // where two fit); CTAs beyond the resident ones would only wait their turn
  int smem_sm = 0, reserved = 0;
  cudaFuncAttributes fa{};
  QS_CUDA(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
  QS_CUDA(cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev));
  QS_CUDA(cudaFuncGetAttributes(&fa, dense_tc_kernel<K>));
  const size_t per_cta = Cfg::SMEM + fa.sharedSizeBytes + (size_t)reserved;
  per_sm = std::max(per_sm, (int)((size_t)smem_sm / per_cta));
  // tensor memory: at most 512 columns per SM among resident CTAs
  per_sm = std::max(1, std::min(per_sm, 512 / Cfg::TMEM_COLS));
  const uint64_t grid = std::min<uint64_t>(n_tiles, (uint64_t)sms * per_sm);
  dense_tc_kernel<K><<<(unsigned)grid, kTcThreads, Cfg::SMEM, st>>>(psi, G, dU, n_tiles, d_err);
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

}  // namespace

// Self-test of the bounded-wait path the tensor-core kernel relies on: one CTA
// polls an mbarrier that nothing arrives on, `limit` times, then records the
// timeout.  No asynchronous work is in flight, so giving up leaves nothing behind.
__global__ void wait_selftest_kernel(long long limit, int* status) {
  __shared__ __align__(8) uint64_t mbar;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  bool ok = false;
  for (long long it = 0; it < limit; ++it)
    if (mbar_try_wait(smem_u32(&mbar), 0)) {
      ok = true;
      break;
    }
  __syncthreads();
  if (threadIdx.x == 0) *status = ok ? 0 : 1;
}

extern "C" {

qs_status qs_apply_matrix(qs_state* s, int k, const int* targets, const double* matrix, int engine) {
  QS_TRY(check_state(s));
  QS_CHECK(k >= 1 && k <= kDenseMaxK, "k must be 1..6");
  QS_CHECK(k <= s->n, "more targets than qubits");
  QS_CHECK(targets != nullptr && matrix != nullptr, "null argument");
  QS_CHECK(engine >= 0 && engine <= 2, "engine must be 0 (auto), 1 (CUDA cores) or 2 (tensor cores)");
  uint64_t tmask = 0;
  for (int b = 0; b < k; ++b) {
    QS_CHECK(targets[b] >= 0 && targets[b] < s->n, "target out of range");
    QS_CHECK(!((tmask >> targets[b]) & 1ull), "repeated target");
    tmask |= 1ull << targets[b];
  }
  const int KB = 1 << k;
  for (int e = 0; e < 2 * KB * KB; ++e) QS_CHECK(std::isfinite(matrix[e]), "non-finite matrix entry");
  // With qubit 0 among the targets, list it first (the matrix's index bits
  // permuted to match: the same operator), so that each column pair of a row is
  // one 16-byte word of the state.
  int tg[kDenseMaxK];
  for (int b = 0; b < k; ++b) tg[b] = targets[b];
  std::vector<double> permuted;
  int b0 = -1;
  for (int b = 0; b < k; ++b)
    if (targets[b] == 0) b0 = b;
  if (b0 > 0) {
    auto old_index = [&](int jn) {  // new bit 0 <- old bit b0, new bits 1..b0 <- old bits 0..b0-1
      int jo = 0;
      for (int p = 0; p < k; ++p) jo |= ((jn >> p) & 1) << (p == 0 ? b0 : p <= b0 ? p - 1 : p);
      return jo;
    };
    permuted.resize(2 * (size_t)KB * KB);
    for (int r = 0; r < KB; ++r)
      for (int c = 0; c < KB; ++c)
        for (int z = 0; z < 2; ++z)
          permuted[2 * ((size_t)r * KB + c) + z] = matrix[2 * ((size_t)old_index(r) * KB + old_index(c)) + z];
    tg[0] = 0;
    for (int p = 1; p <= b0; ++p) tg[p] = targets[p - 1];
    targets = tg;
    matrix = permuted.data();
  }
  DenseGeom G{};
  G.n = s->ne;
  G.k = k;
  for (int j = 0; j < KB; ++j) {
    uint64_t x = 0;
    for (int b = 0; b < k; ++b) x |= (uint64_t)((j >> b) & 1) << targets[b];
    G.tgt_off[j] = x;
  }
  G.n_other = 0;
  for (int q = 0; q < s->ne; ++q)
    if (!((tmask >> q) & 1ull)) G.other_bit[G.n_other++] = (uint8_t)q;
  G.pair0 = (targets[0] == 0 && ((uintptr_t)s->ptr & 15) == 0) ? 1 : 0;
  const bool tc_ok = s->dt == QS_C64 && (k == 4 || k == 5) && (s->ne - k) >= 7;
  QS_CHECK(engine != 2 || tc_ok, "tensor-core blocks need complex64, k = 4 or 5 and at least 7 other qubits");
  const bool use_tc = engine == 2 || (engine == 0 && tc_ok);
  // matrix and error word in the state's scratch (doubles): [err | U]
  const size_t need = 2 + 2 * (size_t)KB * KB;
  QS_TRY(ensure_scratch(s, need));
  int* d_err = reinterpret_cast<int*>(s->scratch);
  double2* dU = reinterpret_cast<double2*>(s->scratch + 2);
  QS_CUDA(cudaMemcpyAsync(dU, matrix, sizeof(double) * 2 * KB * KB, cudaMemcpyHostToDevice, s->st));
  if (use_tc) {
    QS_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int), s->st));
    TraceRec* rec = trace_begin(s->st);
    // k = 5: the warp-specialised kernel (28 qubits, spread targets 0.874 vs
    // 0.933 ms; targets 0-4 2.31 vs 2.91 ms); k = 4: the serial one (0.92 vs
    // 1.18 ms: a 32-column tile leaves the pipeline's hand-offs uncovered)
    qs_status r = k == 4 ? launch_tc<4>(static_cast<float2*>(s->ptr), G, dU, d_err, s->st)
                         : launch_ws<5>(static_cast<float2*>(s->ptr), G, dU, d_err, s->st);
    if (r != QS_OK) return r;
    if (rec) {
      rec->bytes = 2.0 * 8.0 * (double)(1ull << s->ne);
      rec->kind = QS_TRACE_DENSE_TC;
      QS_CUDA(cudaEventRecord(rec->end, s->st));
    }
    int h_err = 0;
    QS_CUDA(cudaMemcpyAsync(&h_err, d_err, sizeof(int), cudaMemcpyDeviceToHost, s->st));
    QS_CUDA(cudaStreamSynchronize(s->st));
    if (h_err) {
      set_error("tensor-core block: MMA completion wait timed out");
      return QS_ERR_TIMEOUT;
    }
    return QS_OK;
  }
  const int threads = cc_threads(s->dt, k);
  const size_t sm = cc_smem(s->dt, k, threads);
  const uint64_t n_rows = 1ull << (s->ne - k);
  const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>((n_rows + threads - 1) / threads, 152 * 8));
  TraceRec* rec = trace_begin(s->st);
  if (s->dt == QS_C64) {
    QS_CUDA(cudaFuncSetAttribute(dense_cc_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    dense_cc_kernel<float><<<grid, threads, sm, s->st>>>(static_cast<float2*>(s->ptr), G, dU, n_rows);
  } else {
    QS_CUDA(cudaFuncSetAttribute(dense_cc_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    dense_cc_kernel<double><<<grid, threads, sm, s->st>>>(static_cast<double2*>(s->ptr), G, dU, n_rows);
  }
  QS_CUDA(cudaGetLastError());
  if (rec) {
    rec->bytes = 2.0 * (double)amp_bytes(s->dt) * (double)(1ull << s->ne);
    rec->kind = QS_TRACE_DENSE_CC;
    QS_CUDA(cudaEventRecord(rec->end, s->st));
  }
  return QS_OK;
}

qs_status qs_selftest_wait_timeout(int* timed_out) {
  QS_CHECK(timed_out != nullptr, "null argument");
  int* d = nullptr;
  QS_CUDA(cudaMalloc(&d, sizeof(int)));
  QS_CUDA(cudaMemset(d, 0xff, sizeof(int)));
  wait_selftest_kernel<<<1, 32>>>(1 << 16, d);
  cudaError_t e = cudaGetLastError();
  int h = -1;
  if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d);
  QS_CUDA(e);
  *timed_out = h;
  if (h == 1) {
    set_error("bounded wait ran out (self-test)");
    return QS_ERR_TIMEOUT;
  }
  return QS_OK;
}

}  // extern "C"
