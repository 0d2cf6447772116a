// Complex64 fused tile passes as micro-ops, compiled with the library: each
// phase dispatches the ops of a pass from its table (the device side, shared
// with the per-circuit kernels of t2gen.cu, is in t2_device.cuh).
#include <algorithm>
#include <cmath>

#include "qsim_internal.h"
#include "t2_device.cuh"
#include "t2gen.h"
#include "tma.h"

namespace qs {

namespace {

using t2d::T2Interp;
using t2d::tile2_body;

template <int NS>
__global__ void __launch_bounds__(NS == 2 ? 288 : 544, 1) tile2_kernel(const __grid_constant__ T2Args args) {
  tile2_body<NS>(args, args.tm, T2Interp{});
}

// The same pass of many instances in one launch: instance blockIdx.y, its
// arguments from a table in global memory (copied to shared memory, except
// the tensor maps, which the TMA unit reads where they are).
template <int NS>
__global__ void __launch_bounds__(NS == 2 ? 288 : 544, 1) tile2_multi_kernel(const T2Args* __restrict__ argv) {
  __shared__ T2Args s_args;
  const T2Args* g = argv + blockIdx.y;
  {
    const int* src = reinterpret_cast<const int*>(g);
    int* dst = reinterpret_cast<int*>(&s_args);
    for (int i = threadIdx.x; i < (int)(sizeof(T2Args) / 4); i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  tile2_body<NS>(s_args, g->tm, T2Interp{});
}

int sm_count2() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

}  // namespace

// Arguments of pass pi of one instance (tensor maps of its psi and lam).
static_assert(sizeof(TmapBlob) == sizeof(CUtensorMap) && alignof(TmapBlob) >= 64, "tensor map layout");

qs_status make_tile2_args(const TilePlan& plan, int pi, void* psi, void* lam, const void* coef, double* partials,
                          int stride, int cols, int n, T2Args* out) {
  const T2Pass& h = plan.passes[pi].t2hdr;
  T2Args& a = *out;
  TileMapDims d;
  for (int i = 0; i < 5; ++i) {
    d.a[i] = h.ma[i];
    d.w[i] = h.mw[i];
    d.bx[i] = h.mbx[i];
  }
  d.e = 0;
  d.lb = h.mlb;
  QS_TRY(encode_tile_map(d, psi, true, reinterpret_cast<CUtensorMap*>(&a.tm[0])));
  if (h.ns == 2) QS_TRY(encode_tile_map(d, lam, true, reinterpret_cast<CUtensorMap*>(&a.tm[1])));
  else a.tm[1] = a.tm[0];
  a.pass = plan.d_t2pass + pi;
  a.phases = plan.d_t2ph + plan.t2_phase_off[pi];
  a.ops = plan.d_t2ops + plan.t2_op_off[pi];
  a.coef = reinterpret_cast<const float2*>(coef);
  a.psi = reinterpret_cast<float2*>(psi);
  a.lam = reinterpret_cast<float2*>(lam);
  a.partials = partials;
  a.stride = stride;
  a.cols = cols;
  a.n = n;
  a.plus_amp = (float)std::pow(2.0, -0.5 * n);
  return QS_OK;
}

qs_status launch_tile2_multi(int ns, const T2Args* d_argv, int count, int grid_x, uint32_t smem, cudaStream_t st) {
  if (count <= 0) return QS_OK;
  const void* fn = ns == 2 ? (const void*)tile2_multi_kernel<2> : (const void*)tile2_multi_kernel<1>;
  QS_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const dim3 g((unsigned)std::max(grid_x, 1), (unsigned)count);
  if (ns == 2)
    tile2_multi_kernel<2><<<g, 256 + 32, smem, st>>>(d_argv);
  else
    tile2_multi_kernel<1><<<g, 512 + 32, smem, st>>>(d_argv);
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

// One pass in its micro-op form (complex64).  grid: the launch's partial columns
// (the kernel runs one CTA per SM at most and zero-fills the other columns).
qs_status launch_tile2_pass(const TilePlan& plan, int pi, const TileLaunch& L, cudaStream_t st) {
  const PlannedPass& pp = plan.passes[pi];
  const T2Pass& h = pp.t2hdr;
  const uint64_t n_tiles = 1ull << (L.n - h.m);
  uint64_t g = std::min<uint64_t>((uint64_t)sm_count2(), n_tiles);
  g = std::min<uint64_t>(g, (uint64_t)std::max(L.grid, 1));
  const int grid = (int)std::max<uint64_t>(g, 1);
  T2Args a;
  QS_TRY(make_tile2_args(plan, pi, L.psi, L.lam, L.coef, L.partials, L.stride, std::max(L.grid, grid), L.n, &a));
  const int T = std::min(1 << (h.m - kRegBits), h.ns == 2 ? 256 : 512);
  if (pi < (int)plan.gen_fn.size() && plan.gen_fn[pi]) return t2gen_launch(plan.gen_fn[pi], a, grid, T + 32, h.smem, st);
  const void* fn = h.ns == 2 ? (const void*)tile2_kernel<2> : (const void*)tile2_kernel<1>;
  static size_t set_smem[2] = {0, 0};
  const int k = h.ns == 2 ? 1 : 0;
  if (set_smem[k] < h.smem) {
    QS_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)h.smem));
    set_smem[k] = h.smem;
  }
  if (h.ns == 2)
    tile2_kernel<2><<<grid, T + 32, h.smem, st>>>(a);
  else
    tile2_kernel<1><<<grid, T + 32, h.smem, st>>>(a);
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

}  // namespace qs
