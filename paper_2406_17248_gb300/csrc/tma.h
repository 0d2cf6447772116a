// Tensor-memory-accelerator (TMA) tile copies and mbarriers shared by the
// tile-pass kernels: a tile of 2^m amplitudes over a qubit set S is one or a
// few boxes of a five-dimensional tensor map whose dimensions follow the runs
// of S in the array's word index.
#pragma once

#include <cuda.h>

#include "qsim_internal.h"
#ifdef __CUDACC__
#include "tma_device.cuh"  // device side: copies, bulk groups, mbarriers
#endif

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

}  // namespace qs
