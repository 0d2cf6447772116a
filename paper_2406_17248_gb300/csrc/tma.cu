// Host side of the TMA tile copies: tensor-map dimensions of a tile and their
// encoding through the driver entry point (no link against libcuda).
#include <algorithm>

#include "tma.h"

namespace qs {

bool tile_map_dims(uint64_t S, int n, int e, int m, int dim0_min, int dim0_max, uint32_t min_box_bytes,
                   TileMapDims* out) {
  const int N = n + e;  // word-index bits
  const uint64_t Sw = (S << e) | ((1ull << e) - 1);
  int st[64], ln[64], k = 0;
  for (int q = 0; q < N;) {
    if (!((Sw >> q) & 1)) {
      ++q;
      continue;
    }
    int r = q;
    const int cap = k == 0 ? dim0_max : 8;
    while (r < N && ((Sw >> r) & 1) && r - q < cap) ++r;
    st[k] = q;
    ln[k++] = r - q;
    q = r;
  }
  if (k == 0 || st[0] != 0 || ln[0] < dim0_min) return false;
  const int d = std::min(k, 5);
  int box_bits = 0;
  for (int i = 0; i < d; ++i) box_bits += ln[i];
  const int lb = box_bits - e;  // local (amplitude) bits a box covers
  if (lb < 0 || m - lb > 5 || (8ull << box_bits) < min_box_bytes) return false;
  for (int i = 0; i < 5; ++i) {
    if (i < d) {
      const int hi = i + 1 < d ? st[i + 1] : N;
      out->a[i] = (uint8_t)st[i];
      out->w[i] = (uint8_t)(hi - st[i]);
      out->bx[i] = (uint8_t)ln[i];
      if (out->w[i] > 31) return false;
    } else {  // unused dimension: one word above the array
      out->a[i] = (uint8_t)N;
      out->w[i] = 0;
      out->bx[i] = 0;
    }
  }
  out->e = (uint8_t)e;
  out->lb = (uint8_t)lb;
  return true;
}

namespace {

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(f);
    else
      (void)cudaGetLastError();
  }
  return fn;
}

}  // namespace

qs_status encode_tile_map(const TileMapDims& d, void* base, bool swizzle128, CUtensorMap* out) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) {
    set_error("cuTensorMapEncodeTiled is unavailable");
    return QS_ERR_CUDA;
  }
  if (swizzle128 && d.bx[0] != 4) {
    set_error("tile map: a 128-byte swizzle needs a 128-byte box row (internal error)");
    return QS_ERR_UNSUPPORTED;
  }
  cuuint64_t dim[5], stride[4];
  cuuint32_t box[5], estr[5];
  for (int i = 0; i < 5; ++i) {
    dim[i] = 1ull << d.w[i];
    box[i] = 1u << d.bx[i];
    estr[i] = 1;
    if (i > 0) stride[i - 1] = 8ull << d.a[i];
  }
  const CUresult r = fn(out, CU_TENSOR_MAP_DATA_TYPE_UINT64, 5, base, dim, stride, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("tensor map of a tile rejected (internal error)");
    return QS_ERR_CUDA;
  }
  return QS_OK;
}

}  // namespace qs
