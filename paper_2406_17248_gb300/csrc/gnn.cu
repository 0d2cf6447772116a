// Learned QAOA initialiser: a message-passing graph network that maps a graph
// to 2p QAOA angles, with bfloat16 weights and float32 arithmetic; its
// forward and backward kernels, the MSE loss and Adam (float32 with a bfloat16
// shadow copy, and float64 for batches of circuit angles).
//
// The paper trains QAOA angles by gradient descent from a fixed start (§5.2)
// and motivates slowly varying schedules by adiabatic evolution (§5.4); the
// network itself is this library's definition (include/qsim.h states it).
//
// One CTA runs one graph at a time (graphs g = blockIdx.x, + gridDim.x, ...;
// two CTAs per SM when every graph of the batch has at most 32 nodes):
// the weights (bf16, rows padded by two elements so that both row and column
// walks are free of bank conflicts), the per-layer node embeddings and the
// adjacency live in shared memory.  The backward kernel recomputes the forward
// activations in shared memory and adds its weight gradients into a private
// float32 slice per CTA; a second kernel sums the slices in CTA order, so
// gradients are bitwise reproducible for a given batch.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <set>
#include <utility>
#include <vector>

#include "handles.h"

using namespace qs;

namespace {

constexpr int kGnnThreads = 256;
constexpr int kGnnMaxNodes = 64;
constexpr int kGnnMaxAdj = 4096;   // adjacency entries (2 |E|) of one graph
constexpr int kGnnMaxHidden = 64;
constexpr int kGnnMaxLayers = 4;
constexpr int kGnnMaxOut = 64;
constexpr int kGnnInDim = 2;       // node features (1, deg / 3)
constexpr int kGnnMaxGrid = 4096;  // CTAs of one launch (per-CTA loss partials)

struct GnnBlock {
  int off;   // offset in the flat parameter vector
  int rows, cols;
  int soff;  // offset in the shared bf16 weight array (rows padded to cols + 2)
};

// Blocks: per layer Ws, Wn, b; then W1, b1, W2, b2.
struct GnnDims {
  int H, L, O, P;
  int n_blocks;
  GnnBlock blk[3 * kGnnMaxLayers + 4];
  int s_w;  // bf16 elements of the shared weight array
};

GnnDims make_dims(int H, int L, int O) {
  GnnDims d{};
  d.H = H;
  d.L = L;
  d.O = O;
  int off = 0, soff = 0, nb = 0;
  auto add = [&](int rows, int cols) {
    GnnBlock& b = d.blk[nb++];
    b.off = off;
    b.rows = rows;
    b.cols = cols;
    b.soff = soff;
    off += rows * cols;
    soff += cols == 1 ? ((rows + 1) & ~1) : rows * (cols + 2);
  };
  int in = kGnnInDim;
  for (int l = 0; l < L; ++l) {
    add(H, in);
    add(H, in);
    add(H, 1);
    in = H;
  }
  add(H, H);
  add(H, 1);
  add(O, H);
  add(O, 1);
  d.n_blocks = nb;
  d.P = off;
  d.s_w = soff;
  return d;
}

// Shared-memory carve-up of one CTA for graphs of at most mn nodes (floats
// after the bf16 weights).  Batches of graphs with at most 32 nodes use mn = 32:
// half the activation storage, two CTAs per SM.
struct GnnSmem {
  size_t w_bytes, h_off, a_off, t0_off, t1_off, vec_off, adj_off, total;
};

GnnSmem smem_layout(const GnnDims& d, int mn) {
  GnnSmem s{};
  s.w_bytes = ((size_t)d.s_w * 2 + 15) & ~(size_t)15;
  const size_t nodeH = (size_t)mn * d.H * 4;
  s.h_off = s.w_bytes;                        // h_0 .. h_L, each [mn][H] (h_0 uses 2 columns)
  s.a_off = s.h_off + (d.L + 1) * nodeH;      // a: mean over neighbours (backward: also q)
  s.t0_off = s.a_off + nodeH;                 // backward: dh
  s.t1_off = s.t0_off + nodeH;                // backward: dpre
  s.vec_off = s.t1_off + nodeH;               // r, zpre, y / dy, dz, dr: 8 x 64 floats
  s.adj_off = s.vec_off + 8 * 64 * 4;         // local CSR: off[mn + 1] int + adj bytes
  s.total = s.adj_off + (kGnnMaxNodes + 1) * 4 + kGnnMaxAdj;
  return s;
}

__device__ __forceinline__ float bf(const __nv_bfloat16* w, int i) { return __bfloat162float(w[i]); }
__device__ __forceinline__ float2 bf2(const __nv_bfloat16* w, int i) {
  return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(w + i));
}

struct GraphView {
  const int* node_off;
  const int* adj_off;
  const int* adj;
};

// Load the weights (once per CTA) into the padded shared layout.
__device__ void load_weights(const GnnDims& D, const __nv_bfloat16* __restrict__ wb, __nv_bfloat16* sw) {
  for (int b = 0; b < D.n_blocks; ++b) {
    const GnnBlock B = D.blk[b];
    const int n = B.rows * B.cols;
    const int stride = B.cols == 1 ? 1 : B.cols + 2;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const int r = i / B.cols, c = i % B.cols;
      sw[B.soff + r * stride + c] = wb[B.off + i];
    }
  }
}

// Graph g into shared memory: local CSR offsets and neighbour bytes; returns nv.
__device__ int load_graph(const GraphView& G, int g, int* s_off, uint8_t* s_adj) {
  const int v0 = G.node_off[g], nv = G.node_off[g + 1] - v0;
  const int e0 = G.adj_off[v0];
  for (int v = threadIdx.x; v <= nv; v += blockDim.x) s_off[v] = G.adj_off[v0 + v] - e0;
  const int ne = G.adj_off[v0 + nv] - e0;
  for (int i = threadIdx.x; i < ne; i += blockDim.x) s_adj[i] = (uint8_t)G.adj[e0 + i];
  return nv;
}

// a[v][k] = mean of h[u][k] over the neighbours u of v (0 without neighbours).
__device__ void aggregate(int nv, int d, int H, const float* h, float* a, const int* s_off, const uint8_t* s_adj) {
  for (int w = threadIdx.x; w < nv * d; w += blockDim.x) {
    const int v = w / d, k = w % d;
    const int b = s_off[v], e = s_off[v + 1];
    float s = 0.f;
    for (int j = b; j < e; ++j) s += h[s_adj[j] * H + k];
    a[v * H + k] = e > b ? s / (float)(e - b) : 0.f;
  }
}

// hout[v][o] = relu(b[o] + sum_i Ws[o][i] h[v][i] + Wn[o][i] a[v][i]), 4 nodes per thread.
__device__ void transform(int nv, int d, int H, const __nv_bfloat16* sw, const GnnBlock& Bs, const GnnBlock& Bn,
                          const GnnBlock& Bb, const float* h, const float* a, float* hout) {
  const int nb4 = (nv + 3) >> 2;
  const int stride = d + 2;
  for (int w = threadIdx.x; w < H * nb4; w += blockDim.x) {
    const int o = w % H, v0 = (w / H) * 4;
    const float bias = bf(sw, Bb.soff + o);
    float acc[4] = {bias, bias, bias, bias};
    const int ws = Bs.soff + o * stride, wn = Bn.soff + o * stride;
    for (int i = 0; i < d; i += 2) {
      const float2 s = bf2(sw, ws + i), n = bf2(sw, wn + i);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float* hv = h + (v0 + j) * H + i;
        const float* av = a + (v0 + j) * H + i;
        acc[j] = fmaf(s.x, hv[0], acc[j]);
        acc[j] = fmaf(s.y, hv[1], acc[j]);
        acc[j] = fmaf(n.x, av[0], acc[j]);
        acc[j] = fmaf(n.y, av[1], acc[j]);
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (v0 + j < nv) hout[(v0 + j) * H + o] = fmaxf(acc[j], 0.f);
  }
}

// Forward pass of one graph, leaving h_0..h_L, r, zpre and y in shared memory.
__device__ void forward_graph(const GnnDims& D, int nv, int mn, const __nv_bfloat16* sw, float* sh, float* sa,
                              float* r, float* zpre, float* y, const int* s_off, const uint8_t* s_adj) {
  const int H = D.H;
  const size_t nodeH = (size_t)mn * H;
  for (int v = threadIdx.x; v < nv; v += blockDim.x) {
    sh[v * H + 0] = 1.f;
    sh[v * H + 1] = (float)(s_off[v + 1] - s_off[v]) / 3.f;
  }
  __syncthreads();
  int d = kGnnInDim;
  for (int l = 0; l < D.L; ++l) {
    const float* h = sh + l * nodeH;
    aggregate(nv, d, H, h, sa, s_off, s_adj);
    __syncthreads();
    transform(nv, d, H, sw, D.blk[3 * l], D.blk[3 * l + 1], D.blk[3 * l + 2], h, sa, sh + (l + 1) * nodeH);
    __syncthreads();
    d = H;
  }
  const float* hL = sh + D.L * nodeH;
  for (int k = threadIdx.x; k < H; k += blockDim.x) {
    float s = 0.f;
    for (int v = 0; v < nv; ++v) s += hL[v * H + k];
    r[k] = nv ? s / (float)nv : 0.f;
  }
  __syncthreads();
  const GnnBlock& W1 = D.blk[3 * D.L];
  const GnnBlock& b1 = D.blk[3 * D.L + 1];
  const GnnBlock& W2 = D.blk[3 * D.L + 2];
  const GnnBlock& b2 = D.blk[3 * D.L + 3];
  for (int j = threadIdx.x; j < H; j += blockDim.x) {
    float s = bf(sw, b1.soff + j);
    for (int k = 0; k < H; k += 2) {
      const float2 w = bf2(sw, W1.soff + j * (H + 2) + k);
      s = fmaf(w.x, r[k], s);
      s = fmaf(w.y, r[k + 1], s);
    }
    zpre[j] = s;
  }
  __syncthreads();
  for (int o = threadIdx.x; o < D.O; o += blockDim.x) {
    float s = bf(sw, b2.soff + o);
    for (int j = 0; j < H; j += 2) {
      const float2 w = bf2(sw, W2.soff + o * (H + 2) + j);
      s = fmaf(w.x, fmaxf(zpre[j], 0.f), s);
      s = fmaf(w.y, fmaxf(zpre[j + 1], 0.f), s);
    }
    y[o] = s;
  }
  __syncthreads();
}

struct GnnPtrs {
  float* sh;
  float* sa;
  float* t0;
  float* t1;
  float* vec;
  int* s_off;
  uint8_t* s_adj;
};

__device__ GnnPtrs carve(const GnnDims& D, unsigned char* smem, int mn) {
  // same arithmetic as smem_layout(), on the device
  const size_t w_bytes = ((size_t)D.s_w * 2 + 15) & ~(size_t)15;
  const size_t nodeH = (size_t)mn * D.H;
  GnnPtrs p;
  p.sh = reinterpret_cast<float*>(smem + w_bytes);
  p.sa = p.sh + (D.L + 1) * nodeH;
  p.t0 = p.sa + nodeH;
  p.t1 = p.t0 + nodeH;
  p.vec = p.t1 + nodeH;
  p.s_off = reinterpret_cast<int*>(p.vec + 8 * 64);
  p.s_adj = reinterpret_cast<uint8_t*>(p.s_off + kGnnMaxNodes + 1);
  return p;
}

__global__ void __launch_bounds__(kGnnThreads) gnn_forward_kernel(GnnDims D, const __nv_bfloat16* __restrict__ wb,
                                                                  GraphView G, int n_graphs, int mn,
                                                                  float* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem[];
  __nv_bfloat16* sw = reinterpret_cast<__nv_bfloat16*>(smem);
  const GnnPtrs p = carve(D, smem, mn);
  load_weights(D, wb, sw);
  for (int g = blockIdx.x; g < n_graphs; g += gridDim.x) {
    __syncthreads();
    const int nv = load_graph(G, g, p.s_off, p.s_adj);
    __syncthreads();
    float* y = p.vec + 2 * 64;
    forward_graph(D, nv, mn, sw, p.sh, p.sa, p.vec, p.vec + 64, y, p.s_off, p.s_adj);
    for (int o = threadIdx.x; o < D.O; o += blockDim.x) out[(size_t)g * D.O + o] = y[o];
  }
}

// Backward of one graph per iteration; weight gradients go to this CTA's slice
// part[blockIdx.x * P ...] (one owning thread per entry; the CTA's first graph
// writes every entry, later graphs add).  TRAIN: dL/dy = 2 (y - t) / n_out of
// the mean squared error is formed in place from the targets, and the CTA's sum
// of squared errors goes to loss_part[blockIdx.x] (a whole training step's
// network work in one launch).
template <bool TRAIN>
__global__ void __launch_bounds__(kGnnThreads) gnn_backward_kernel(GnnDims D, const __nv_bfloat16* __restrict__ wb,
                                                                   GraphView G, int n_graphs, int mn,
                                                                   const float* __restrict__ dy_all,
                                                                   float* __restrict__ part, float dy_scale,
                                                                   float* __restrict__ loss_part) {
  extern __shared__ __align__(16) unsigned char smem[];
  __nv_bfloat16* sw = reinterpret_cast<__nv_bfloat16*>(smem);
  const GnnPtrs p = carve(D, smem, mn);
  const int H = D.H, O = D.O;
  const size_t nodeH = (size_t)mn * H;
  float* gp = part + (size_t)blockIdx.x * D.P;
  float* r = p.vec;
  float* zpre = p.vec + 64;
  float* y = p.vec + 128;
  float* dy = p.vec + 192;
  float* dz = p.vec + 256;
  float* dr = p.vec + 320;
  load_weights(D, wb, sw);
  const GnnBlock& W1 = D.blk[3 * D.L];
  const GnnBlock& b1 = D.blk[3 * D.L + 1];
  const GnnBlock& W2 = D.blk[3 * D.L + 2];
  const GnnBlock& b2 = D.blk[3 * D.L + 3];
  float sse = 0.f;  // TRAIN: this CTA's sum of squared errors (thread 0)
  for (int g = blockIdx.x; g < n_graphs; g += gridDim.x) {
    const bool first = g == (int)blockIdx.x;
    // first graph of the CTA: assign, later graphs: accumulate
    auto put = [&](int idx, float v) {
      if (first)
        gp[idx] = v;
      else
        gp[idx] += v;
    };
    __syncthreads();
    const int nv = load_graph(G, g, p.s_off, p.s_adj);
    __syncthreads();
    forward_graph(D, nv, mn, sw, p.sh, p.sa, r, zpre, y, p.s_off, p.s_adj);
    if (TRAIN) {
      for (int o = threadIdx.x; o < O; o += blockDim.x) dy[o] = dy_scale * (y[o] - dy_all[(size_t)g * O + o]);
      if (threadIdx.x == 0)
        for (int o = 0; o < O; ++o) {
          const float e = y[o] - dy_all[(size_t)g * O + o];
          sse = fmaf(e, e, sse);
        }
    } else {
      for (int o = threadIdx.x; o < O; o += blockDim.x) dy[o] = dy_all[(size_t)g * O + o];
    }
    __syncthreads();
    // readout MLP
    for (int w = threadIdx.x; w < O * H; w += blockDim.x) {
      const int o = w / H, j = w % H;
      put(W2.off + w, dy[o] * fmaxf(zpre[j], 0.f));
    }
    for (int o = threadIdx.x; o < O; o += blockDim.x) put(b2.off + o, dy[o]);
    for (int j = threadIdx.x; j < H; j += blockDim.x) {
      float s = 0.f;
      for (int o = 0; o < O; ++o) s = fmaf(bf(sw, W2.soff + o * (H + 2) + j), dy[o], s);
      dz[j] = zpre[j] > 0.f ? s : 0.f;
    }
    __syncthreads();
    for (int w = threadIdx.x; w < H * H; w += blockDim.x) {
      const int j = w / H, k = w % H;
      put(W1.off + w, dz[j] * r[k]);
    }
    for (int j = threadIdx.x; j < H; j += blockDim.x) put(b1.off + j, dz[j]);
    for (int k = threadIdx.x; k < H; k += blockDim.x) {
      float s = 0.f;
      for (int j = 0; j < H; ++j) s = fmaf(bf(sw, W1.soff + j * (H + 2) + k), dz[j], s);
      dr[k] = s;
    }
    __syncthreads();
    float* dh = p.t0;
    float* dpre = p.t1;
    float* q = p.sa;  // the neighbour means of this layer are dead once its gradients are added
    const float inv_nv = nv ? 1.f / (float)nv : 0.f;
    for (int w = threadIdx.x; w < nv * H; w += blockDim.x) dh[w] = dr[w % H] * inv_nv;
    __syncthreads();
    for (int l = D.L - 1; l >= 0; --l) {
      const int d = l == 0 ? kGnnInDim : H;
      const float* h = p.sh + l * nodeH;
      const float* hn = p.sh + (l + 1) * nodeH;
      const GnnBlock& Bs = D.blk[3 * l];
      const GnnBlock& Bn = D.blk[3 * l + 1];
      const GnnBlock& Bb = D.blk[3 * l + 2];
      aggregate(nv, d, H, h, p.sa, p.s_off, p.s_adj);
      for (int w = threadIdx.x; w < nv * H; w += blockDim.x) dpre[w] = hn[w] > 0.f ? dh[w] : 0.f;
      __syncthreads();
      for (int w = threadIdx.x; w < H * d; w += blockDim.x) {
        const int o = w / d, i = w % d;
        float ss = 0.f, sn = 0.f;
        for (int v = 0; v < nv; ++v) {
          const float g_ = dpre[v * H + o];
          ss = fmaf(g_, h[v * H + i], ss);
          sn = fmaf(g_, p.sa[v * H + i], sn);
        }
        put(Bs.off + w, ss);
        put(Bn.off + w, sn);
      }
      for (int o = threadIdx.x; o < H; o += blockDim.x) {
        float s = 0.f;
        for (int v = 0; v < nv; ++v) s += dpre[v * H + o];
        put(Bb.off + o, s);
      }
      if (l == 0) break;
      __syncthreads();  // p.sa (a_l) is read above and becomes q below
      // q[v][i] = sum_o Wn[o][i] dpre[v][o] / deg(v)
      for (int w = threadIdx.x; w < nv * H; w += blockDim.x) {
        const int v = w / H, i = w % H;
        const int deg = p.s_off[v + 1] - p.s_off[v];
        float s = 0.f;
        for (int o = 0; o < H; ++o) s = fmaf(bf(sw, Bn.soff + o * (d + 2) + i), dpre[v * H + o], s);
        q[w] = deg ? s / (float)deg : 0.f;
      }
      __syncthreads();
      // dh[v][i] = sum_o Ws[o][i] dpre[v][o] + sum over neighbours u of q[u][i]
      for (int w = threadIdx.x; w < nv * H; w += blockDim.x) {
        const int v = w / H, i = w % H;
        float s = 0.f;
        for (int o = 0; o < H; ++o) s = fmaf(bf(sw, Bs.soff + o * (d + 2) + i), dpre[v * H + o], s);
        for (int j = p.s_off[v]; j < p.s_off[v + 1]; ++j) s += q[p.s_adj[j] * H + i];
        dh[w] = s;
      }
      __syncthreads();
    }
  }
  if (TRAIN && threadIdx.x == 0) loss_part[blockIdx.x] = sse;
}

// grad[i] = sum over CTA slices in CTA order.
__global__ void gnn_reduce_kernel(const float* __restrict__ part, int n_slices, int P, float* __restrict__ grad) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int c = 0; c < n_slices; ++c) s += part[(size_t)c * P + i];
    grad[i] = s;
  }
}

// Training step tail: grad[i] = sum of the CTA slices (CTA order), then Adam
// on weight i (as adam_f32_kernel) and its bf16 copy; block 0 also forms the
// loss = (sum of the CTAs' squared errors) / n_out.
__global__ void gnn_reduce_adam_kernel(const float* __restrict__ part, int n_slices, int P, float* __restrict__ w,
                                       float* __restrict__ m, float* __restrict__ v, float lr, float b1, float b2,
                                       float eps, float c1, float c2, __nv_bfloat16* __restrict__ wb,
                                       const float* __restrict__ loss_part, float inv_n_out,
                                       float* __restrict__ loss) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < P; i += gridDim.x * blockDim.x) {
    float gi = 0.f;
    for (int c = 0; c < n_slices; ++c) gi += part[(size_t)c * P + i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    w[i] = wi;
    wb[i] = __float2bfloat16_rn(wi);
  }
  if (loss && blockIdx.x == 0 && threadIdx.x == 0) {
    float s = 0.f;
    for (int c = 0; c < n_slices; ++c) s += loss_part[c];
    *loss = s * inv_n_out;
  }
}

// Squared error: loss = mean (y - t)^2, dy = 2 (y - t) / n; one CTA, fixed order.
__global__ void mse_kernel(int n, const float* __restrict__ y, const float* __restrict__ t, float* __restrict__ loss,
                           float* __restrict__ dy) {
  __shared__ float red[1024];
  float s = 0.f;
  const float sc = n ? 2.f / (float)n : 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float d = y[i] - t[i];
    s = fmaf(d, d, s);
    if (dy) dy[i] = sc * d;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0 && loss) *loss = n ? red[0] / (float)n : 0.f;
}

// Adam (Kingma & Ba, Algorithm 1); c1 = 1 / (1 - b1^t), c2 = 1 / (1 - b2^t).
__global__ void adam_f32_kernel(int n, float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                                const float* __restrict__ g, float lr, float b1, float b2, float eps, float c1,
                                float c2, __nv_bfloat16* __restrict__ wb) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    w[i] = wi;
    if (wb) wb[i] = __float2bfloat16_rn(wi);
  }
}

__global__ void adam_f64_kernel(int n, double* __restrict__ w, double* __restrict__ m, double* __restrict__ v,
                                const double* __restrict__ g, double lr, double b1, double b2, double eps, double c1,
                                double c2, int maximize) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double gi = maximize ? -g[i] : g[i];
    const double mi = b1 * m[i] + (1.0 - b1) * gi;
    const double vi = b2 * v[i] + (1.0 - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] = w[i] - lr * (mi * c1) / (sqrt(vi * c2) + eps);
  }
}

__global__ void to_bf16_kernel(int n, const float* __restrict__ w, __nv_bfloat16* __restrict__ wb) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    wb[i] = __float2bfloat16_rn(w[i]);
}

int blocks_for(int n, int threads) { return std::max(1, std::min((n + threads - 1) / threads, 4096)); }

}  // namespace

struct qs_graphs {
  int n_graphs = 0;
  int max_nodes = 0;
  int* d_node_off = nullptr;
  int* d_adj_off = nullptr;
  int* d_adj = nullptr;
};

struct qs_gnn {
  GnnDims D{};
  GnnSmem S[2]{};        // layouts for graphs of <= 32 and <= 64 nodes
  int grid_max[2] = {1, 1};
  cudaStream_t st = nullptr;
  float* d_w = nullptr;  // float32 master weights
  float* d_m = nullptr;
  float* d_v = nullptr;
  __nv_bfloat16* d_wb = nullptr;  // the bfloat16 copy the kernels compute with
  float* d_part = nullptr;
  size_t part_slices = 0;
  float* d_loss_part = nullptr;  // per-CTA squared errors of a training step
  int step = 0;
};

namespace {

void free_gnn(qs_gnn* g) {
  if (!g) return;
  for (void* p : {(void*)g->d_w, (void*)g->d_m, (void*)g->d_v, (void*)g->d_wb, (void*)g->d_part,
                  (void*)g->d_loss_part})
    if (p) cudaFree(p);
  delete g;
}

void free_graphs(qs_graphs* g) {
  if (!g) return;
  for (void* p : {(void*)g->d_node_off, (void*)g->d_adj_off, (void*)g->d_adj})
    if (p) cudaFree(p);
  delete g;
}

qs_status check_graphs(int n_graphs, const int* node_off, const int* adj_off, const int* adj, int* max_nodes) {
  QS_CHECK(n_graphs >= 0, "n_graphs must be >= 0");
  QS_CHECK(node_off != nullptr && adj_off != nullptr, "null graph arrays");
  QS_CHECK(node_off[0] == 0 && adj_off[0] == 0, "offsets must start at 0");
  *max_nodes = 0;
  for (int g = 0; g < n_graphs; ++g) {
    const int v0 = node_off[g], v1 = node_off[g + 1], nv = v1 - v0;
    QS_CHECK(nv >= 0 && nv <= kGnnMaxNodes, "a graph has more than 64 nodes (or negative size)");
    *max_nodes = std::max(*max_nodes, nv);
    QS_CHECK(adj_off[v1] - adj_off[v0] <= kGnnMaxAdj, "a graph has more than 2048 edges");
    std::set<std::pair<int, int>> arcs;
    for (int v = v0; v < v1; ++v) {
      QS_CHECK(adj_off[v + 1] >= adj_off[v], "adjacency offsets must not decrease");
      for (int j = adj_off[v]; j < adj_off[v + 1]; ++j) {
        QS_CHECK(adj != nullptr, "null adjacency");
        const int u = adj[j];
        QS_CHECK(u >= 0 && u < nv, "neighbour index out of range (indices are local to the graph)");
        QS_CHECK(u != v - v0, "self loop");
        QS_CHECK(arcs.insert({v - v0, u}).second, "repeated neighbour");
      }
    }
    for (const auto& a : arcs) QS_CHECK(arcs.count({a.second, a.first}), "adjacency is not symmetric");
  }
  return QS_OK;
}

GraphView view(const qs_graphs* G) { return GraphView{G->d_node_off, G->d_adj_off, G->d_adj}; }

// Layout index (0: graphs of <= 32 nodes, 1: <= 64), node capacity and grid of a batch.
int gnn_layout(const qs_graphs* G) { return G->max_nodes <= 32 ? 0 : 1; }
int gnn_mn(int li) { return li == 0 ? 32 : kGnnMaxNodes; }
int gnn_grid(const qs_gnn* g, int li, int n_graphs) { return std::max(1, std::min(n_graphs, g->grid_max[li])); }

}  // namespace

extern "C" {

qs_status qs_graphs_create(int n_graphs, const int* node_off, const int* adj_off, const int* adj, qs_graphs** out) {
  QS_CHECK(out != nullptr, "null output");
  *out = nullptr;
  int max_nodes = 0;
  QS_TRY(check_graphs(n_graphs, node_off, adj_off, adj, &max_nodes));
  const int N = node_off[n_graphs], E = adj_off[N];
  qs_graphs* G = new qs_graphs();
  G->n_graphs = n_graphs;
  G->max_nodes = max_nodes;
  auto up = [&](int** dst, const int* src, int n) -> qs_status {
    cudaError_t e = cudaMalloc(dst, std::max(n, 1) * sizeof(int));
    if (e == cudaSuccess && n > 0) e = cudaMemcpy(*dst, src, n * sizeof(int), cudaMemcpyHostToDevice);
    return e == cudaSuccess ? QS_OK : cuda_fail(e, "graph upload");
  };
  qs_status s = up(&G->d_node_off, node_off, n_graphs + 1);
  if (s == QS_OK) s = up(&G->d_adj_off, adj_off, N + 1);
  if (s == QS_OK) s = up(&G->d_adj, adj, E);
  if (s != QS_OK) {
    free_graphs(G);
    return s;
  }
  *out = G;
  return QS_OK;
}

qs_status qs_graphs_destroy(qs_graphs* g) {
  free_graphs(g);
  return QS_OK;
}

qs_status qs_gnn_n_weights(int hidden, int layers, int out_dim, int* n) {
  QS_CHECK(n != nullptr, "null output");
  QS_CHECK(hidden >= 2 && hidden <= kGnnMaxHidden && hidden % 2 == 0, "hidden must be even, 2..64");
  QS_CHECK(layers >= 1 && layers <= kGnnMaxLayers, "layers must be 1..4");
  QS_CHECK(out_dim >= 1 && out_dim <= kGnnMaxOut, "out_dim must be 1..64");
  *n = make_dims(hidden, layers, out_dim).P;
  return QS_OK;
}

qs_status qs_gnn_create(int hidden, int layers, int out_dim, void* cuda_stream, qs_gnn** out) {
  QS_CHECK(out != nullptr, "null output");
  *out = nullptr;
  int P = 0;
  QS_TRY(qs_gnn_n_weights(hidden, layers, out_dim, &P));
  qs_gnn* g = new qs_gnn();
  g->D = make_dims(hidden, layers, out_dim);
  g->S[0] = smem_layout(g->D, 32);
  g->S[1] = smem_layout(g->D, kGnnMaxNodes);
  g->st = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0, sms = 1, smem_optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess && (size_t)smem_optin < g->S[1].total) {
    free_gnn(g);
    set_error("GNN shared-memory layout exceeds the device limit");
    return QS_ERR_UNSUPPORTED;
  }
  const int smax = (int)g->S[1].total;
  if (e == cudaSuccess) e = cudaFuncSetAttribute(gnn_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(gnn_backward_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(gnn_backward_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax);
  for (int li = 0; li < 2 && e == cudaSuccess; ++li) {
    // resident CTAs per SM of the heavier (backward) kernel with this layout
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, gnn_backward_kernel<true>, kGnnThreads, g->S[li].total);
    g->grid_max[li] = sms * std::max(occ, 1);
  }
  const size_t P4 = (size_t)P * 4;
  if (e == cudaSuccess) e = cudaMalloc(&g->d_w, P4);
  if (e == cudaSuccess) e = cudaMalloc(&g->d_m, P4);
  if (e == cudaSuccess) e = cudaMalloc(&g->d_v, P4);
  if (e == cudaSuccess) e = cudaMalloc(&g->d_wb, (size_t)P * 2);
  if (e == cudaSuccess) e = cudaMemset(g->d_w, 0, P4);
  if (e == cudaSuccess) e = cudaMemset(g->d_m, 0, P4);
  if (e == cudaSuccess) e = cudaMemset(g->d_v, 0, P4);
  if (e == cudaSuccess) e = cudaMemset(g->d_wb, 0, (size_t)P * 2);
  if (e != cudaSuccess) {
    free_gnn(g);
    return cuda_fail(e, "qs_gnn_create");
  }
  *out = g;
  return QS_OK;
}

qs_status qs_gnn_destroy(qs_gnn* g) {
  free_gnn(g);
  return QS_OK;
}

qs_status qs_gnn_set_weights(qs_gnn* g, const float* w, int on_device) {
  QS_CHECK(g != nullptr && w != nullptr, "null argument");
  const int P = g->D.P;
  QS_CUDA(cudaMemcpyAsync(g->d_w, w, (size_t)P * 4, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                          g->st));
  QS_CUDA(cudaMemsetAsync(g->d_m, 0, (size_t)P * 4, g->st));
  QS_CUDA(cudaMemsetAsync(g->d_v, 0, (size_t)P * 4, g->st));
  to_bf16_kernel<<<blocks_for(P, 256), 256, 0, g->st>>>(P, g->d_w, g->d_wb);
  QS_CUDA(cudaGetLastError());
  g->step = 0;
  if (!on_device) QS_CUDA(cudaStreamSynchronize(g->st));
  return QS_OK;
}

qs_status qs_gnn_get_weights(qs_gnn* g, float* w, uint16_t* w_bf16, int on_device) {
  QS_CHECK(g != nullptr && (w != nullptr || w_bf16 != nullptr), "null argument");
  const int P = g->D.P;
  const cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (w) QS_CUDA(cudaMemcpyAsync(w, g->d_w, (size_t)P * 4, k, g->st));
  if (w_bf16) QS_CUDA(cudaMemcpyAsync(w_bf16, g->d_wb, (size_t)P * 2, k, g->st));
  if (!on_device) QS_CUDA(cudaStreamSynchronize(g->st));
  return QS_OK;
}

qs_status qs_gnn_get_state(qs_gnn* g, float* w, float* m, float* v, int* step) {
  QS_CHECK(g != nullptr && w != nullptr && m != nullptr && v != nullptr && step != nullptr, "null argument");
  const size_t bytes = (size_t)g->D.P * 4;
  QS_CUDA(cudaMemcpyAsync(w, g->d_w, bytes, cudaMemcpyDeviceToHost, g->st));
  QS_CUDA(cudaMemcpyAsync(m, g->d_m, bytes, cudaMemcpyDeviceToHost, g->st));
  QS_CUDA(cudaMemcpyAsync(v, g->d_v, bytes, cudaMemcpyDeviceToHost, g->st));
  QS_CUDA(cudaStreamSynchronize(g->st));
  *step = g->step;
  return QS_OK;
}

qs_status qs_gnn_set_state(qs_gnn* g, const float* w, const float* m, const float* v, int step) {
  QS_CHECK(g != nullptr && w != nullptr && m != nullptr && v != nullptr, "null argument");
  QS_CHECK(step >= 0, "step must be >= 0");
  const int P = g->D.P;
  const size_t bytes = (size_t)P * 4;
  QS_CUDA(cudaMemcpyAsync(g->d_w, w, bytes, cudaMemcpyHostToDevice, g->st));
  QS_CUDA(cudaMemcpyAsync(g->d_m, m, bytes, cudaMemcpyHostToDevice, g->st));
  QS_CUDA(cudaMemcpyAsync(g->d_v, v, bytes, cudaMemcpyHostToDevice, g->st));
  to_bf16_kernel<<<blocks_for(P, 256), 256, 0, g->st>>>(P, g->d_w, g->d_wb);
  QS_CUDA(cudaGetLastError());
  QS_CUDA(cudaStreamSynchronize(g->st));
  g->step = step;
  return QS_OK;
}

qs_status qs_gnn_forward(qs_gnn* g, const qs_graphs* graphs, float* dev_out) {
  QS_CHECK(g != nullptr && graphs != nullptr, "null argument");
  QS_CHECK(graphs->n_graphs == 0 || dev_out != nullptr, "null output");
  if (graphs->n_graphs == 0) return QS_OK;
  const int li = gnn_layout(graphs);
  const int grid = gnn_grid(g, li, graphs->n_graphs);
  gnn_forward_kernel<<<grid, kGnnThreads, g->S[li].total, g->st>>>(g->D, g->d_wb, view(graphs), graphs->n_graphs,
                                                                    gnn_mn(li), dev_out);
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

qs_status qs_gnn_backward(qs_gnn* g, const qs_graphs* graphs, const float* dev_dout, float* dev_grad) {
  QS_CHECK(g != nullptr && graphs != nullptr && dev_grad != nullptr, "null argument");
  QS_CHECK(graphs->n_graphs == 0 || dev_dout != nullptr, "null dout");
  const int P = g->D.P;
  const int li = gnn_layout(graphs);
  const int grid = gnn_grid(g, li, graphs->n_graphs);
  if ((size_t)grid > g->part_slices) {
    if (g->d_part) QS_CUDA(cudaFree(g->d_part));
    g->d_part = nullptr;
    g->part_slices = 0;
    QS_CUDA(cudaMalloc(&g->d_part, (size_t)grid * P * 4));
    g->part_slices = grid;
  }
  if (graphs->n_graphs > 0) {  // every CTA has a graph and writes its whole slice
    gnn_backward_kernel<false><<<grid, kGnnThreads, g->S[li].total, g->st>>>(
        g->D, g->d_wb, view(graphs), graphs->n_graphs, gnn_mn(li), dev_dout, g->d_part, 0.f, nullptr);
    QS_CUDA(cudaGetLastError());
  } else {
    QS_CUDA(cudaMemsetAsync(g->d_part, 0, (size_t)grid * P * 4, g->st));
  }
  gnn_reduce_kernel<<<blocks_for(P, 256), 256, 0, g->st>>>(g->d_part, grid, P, dev_grad);
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

qs_status qs_gnn_adam_step(qs_gnn* g, const float* dev_grad, float lr, float beta1, float beta2, float eps) {
  QS_CHECK(g != nullptr && dev_grad != nullptr, "null argument");
  QS_CHECK(beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f && beta2 < 1.f && eps > 0.f, "bad Adam hyper-parameters");
  g->step += 1;
  const double c1 = 1.0 / (1.0 - std::pow((double)beta1, g->step));
  const double c2 = 1.0 / (1.0 - std::pow((double)beta2, g->step));
  const int P = g->D.P;
  adam_f32_kernel<<<blocks_for(P, 256), 256, 0, g->st>>>(P, g->d_w, g->d_m, g->d_v, dev_grad, lr, beta1, beta2, eps,
                                                         (float)c1, (float)c2, g->d_wb);
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

qs_status qs_gnn_train_step(qs_gnn* g, const qs_graphs* graphs, const float* dev_targets, float lr, float beta1,
                            float beta2, float eps, float* dev_loss) {
  QS_CHECK(g != nullptr && graphs != nullptr, "null argument");
  QS_CHECK(graphs->n_graphs >= 1 && dev_targets != nullptr, "need at least one graph and its targets");
  QS_CHECK(beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f && beta2 < 1.f && eps > 0.f, "bad Adam hyper-parameters");
  const int P = g->D.P;
  const int li = gnn_layout(graphs);
  const int grid = gnn_grid(g, li, graphs->n_graphs);
  if ((size_t)grid > g->part_slices) {
    if (g->d_part) QS_CUDA(cudaFree(g->d_part));
    g->d_part = nullptr;
    g->part_slices = 0;
    QS_CUDA(cudaMalloc(&g->d_part, (size_t)grid * P * 4));
    g->part_slices = grid;
  }
  if (!g->d_loss_part) QS_CUDA(cudaMalloc(&g->d_loss_part, (size_t)4 * 2 * kGnnMaxGrid));
  QS_CHECK(grid <= 2 * kGnnMaxGrid, "too many CTAs for the loss buffer");
  const int n_out = graphs->n_graphs * g->D.O;
  gnn_backward_kernel<true><<<grid, kGnnThreads, g->S[li].total, g->st>>>(
      g->D, g->d_wb, view(graphs), graphs->n_graphs, gnn_mn(li), dev_targets, g->d_part, 2.f / (float)n_out,
      g->d_loss_part);
  QS_CUDA(cudaGetLastError());
  g->step += 1;
  const double c1 = 1.0 / (1.0 - std::pow((double)beta1, g->step));
  const double c2 = 1.0 / (1.0 - std::pow((double)beta2, g->step));
  gnn_reduce_adam_kernel<<<blocks_for(P, 256), 256, 0, g->st>>>(g->d_part, grid, P, g->d_w, g->d_m, g->d_v, lr, beta1,
                                                                beta2, eps, (float)c1, (float)c2, g->d_wb,
                                                                g->d_loss_part, 1.f / (float)n_out, dev_loss);
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

qs_status qs_mse(int n, const float* dev_y, const float* dev_target, float* dev_loss, float* dev_dy,
                 void* cuda_stream) {
  QS_CHECK(n >= 0 && n <= (1 << 26), "n must be 0..2^26");
  QS_CHECK(n == 0 || (dev_y != nullptr && dev_target != nullptr), "null argument");
  mse_kernel<<<1, 1024, 0, static_cast<cudaStream_t>(cuda_stream)>>>(n, dev_y, dev_target, dev_loss, dev_dy);
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

qs_status qs_adam_f64(int n, double* dev_w, double* dev_m, double* dev_v, const double* dev_grad, int t, double lr,
                      double beta1, double beta2, double eps, int maximize, void* cuda_stream) {
  QS_CHECK(n >= 0, "n must be >= 0");
  QS_CHECK(n == 0 || (dev_w && dev_m && dev_v && dev_grad), "null argument");
  QS_CHECK(t >= 1, "t counts steps from 1");
  QS_CHECK(beta1 >= 0.0 && beta1 < 1.0 && beta2 >= 0.0 && beta2 < 1.0 && eps > 0.0, "bad Adam hyper-parameters");
  if (n == 0) return QS_OK;
  const double c1 = 1.0 / (1.0 - std::pow(beta1, t)), c2 = 1.0 / (1.0 - std::pow(beta2, t));
  adam_f64_kernel<<<blocks_for(n, 256), 256, 0, static_cast<cudaStream_t>(cuda_stream)>>>(
      n, dev_w, dev_m, dev_v, dev_grad, lr, beta1, beta2, eps, c1, c2, maximize);
  QS_CUDA(cudaGetLastError());
  return QS_OK;
}

}  // extern "C"
