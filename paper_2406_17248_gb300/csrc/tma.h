// Tensor-memory-accelerator (TMA) tile copies and mbarriers shared by the
// tile-pass kernels: a tile of 2^m amplitudes over a qubit set S is one or a
// few boxes of a five-dimensional tensor map whose dimensions follow the runs
// of S in the array's word index.
#pragma once

#include <cuda.h>

#include "qsim_internal.h"

namespace qs {

// ------------------------------------------------------------------ host side

// Dimensions of the tensor map that copies a tile over the qubit set S of an
// n-qubit array with 2^e 8-byte words per amplitude.  The word-index bits of S
// are cut into runs, each run into chunks (dimension 0 at most dim0_max bits,
// the others at most 8: a box edge holds <= 256 words); dimension i spans word
// bits [a[i], a[i] + w[i]) and its box the low bx[i] of them.  Up to five
// chunks are dimensions; the tile's remaining local bits are enumerated as
// separate boxes (box j at tile-local offset j 2^lb).  Returns false when S
// does not start with a run of at least dim0_min word bits, when a tile needs
// more than 32 boxes or boxes smaller than min_box_bytes, or when a dimension
// would be wider than 31 bits.
struct TileMapDims {
  uint8_t a[5], w[5], bx[5];
  uint8_t e, lb;
};
bool tile_map_dims(uint64_t S, int n, int e, int m, int dim0_min, int dim0_max, uint32_t min_box_bytes,
                   TileMapDims* out);

// Encodes the map of `d` over the array at `base` (8-byte words; 16-byte
// aligned).  swizzle128: 128-byte shared-memory swizzle (16-byte chunk c of
// each 128-byte row r lands at chunk c ^ (r mod 8)); dimension 0 must then span
// exactly 128 bytes.
qs_status encode_tile_map(const TileMapDims& d, void* base, bool swizzle128, CUtensorMap* out);

// ---------------------------------------------------------------- device side
#ifdef __CUDACC__
__device__ __forceinline__ uint32_t tma_sh(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void tma_load5(uint32_t dst, const CUtensorMap* map, const int (&x)[5], uint32_t mbar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5, "
      "%6}], [%7];\n" ::"r"(dst),
      "l"(map), "r"(x[0]), "r"(x[1]), "r"(x[2]), "r"(x[3]), "r"(x[4]), "r"(mbar)
      : "memory");
}
__device__ __forceinline__ void tma_store5(const CUtensorMap* map, const int (&x)[5], uint32_t src) {
  asm volatile("cp.async.bulk.tensor.5d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3, %4, %5}], [%6];\n" ::"l"(
                   map),
               "r"(x[0]), "r"(x[1]), "r"(x[2]), "r"(x[3]), "r"(x[4]), "r"(src)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;\n" ::: "memory"); }
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;\n" ::: "memory"); }
// generic-proxy shared writes made visible to the async proxy (bulk stores)
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory"); }

// word index -> the five coordinates of map dimensions (a, w)
__device__ __forceinline__ void tile_coords(const uint8_t (&a)[5], const uint8_t (&w)[5], uint64_t wi, int (&x)[5]) {
#pragma unroll
  for (int d = 0; d < 5; ++d) x[d] = (int)((wi >> a[d]) & ((1ull << w[d]) - 1ull));
}

// mbarrier helpers (shared::cta addresses).  Waits are bounded: on timeout
// they return false and the kernel records a fault instead of hanging.
__device__ __forceinline__ void mbar_init(uint32_t a, uint32_t count) {
  asm volatile("mbarrier.init.shared.b64 [%0], %1;\n" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t a) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared.b64 st, [%0];\n}\n" ::"r"(a) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect(uint32_t a, uint32_t bytes) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(a), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_wait(uint32_t a, uint32_t parity) {
  for (long long it = 0; it < (1ll << 26); ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
// named barrier 1 over the compute warps (the producer warp does not take part)
__device__ __forceinline__ void bar_compute(int nthreads) {
  asm volatile("bar.sync 1, %0;\n" ::"r"(nthreads) : "memory");
}
#endif

}  // namespace qs
