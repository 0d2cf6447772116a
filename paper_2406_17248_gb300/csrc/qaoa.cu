// MaxCut QAOA engine (§5.2 ansatz; the QuPack QAOA simulator interface of
// §6.2): |+>^n, then per layer exp(-i gs gamma_l C) and RX(beta_l) on every
// qubit; energy <C> and its adjoint gradient in gamma and beta.
//
// Schedule.  A pass covers a tile bit set S (the low c qubits plus others).
// The mixer RX(beta_l) of a layer is applied to the bits of S not yet mixed in
// this layer.  When a pass completes layer l it applies the next cost layer
// (elementwise, from the cut-value array) and the next mixer on every bit of S
// at once, so the bit sets rotate and a layer costs about 2 HBM passes instead
// of ceil(n / (m - c)).  The last forward pass also forms E = sum C|psi|^2 and
// lam = C psi and immediately runs its own reverse ops (the turnaround): psi is
// never written there, because the state before the pass is still in HBM.
// The reverse passes replay the forward passes backwards on (psi, lam):
//   dE/dbeta_l  = sum_q Im <lam|X_q|psi>   (taken before RX_q^dag; any point
//                 inside layer l's mixer gives the same value because RX on
//                 other qubits commutes with X_q),
//   dE/dgamma_l = 2 gs Im <lam|C|psi>      (between the mixer and cost of l).
// The last reverse pass stores nothing.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>

#include "handles.h"
#include "qaoa_pass.h"
#include "qaoa_x_plan.h"

using cd = std::complex<double>;
using namespace qs;

struct qs_qaoa {
  int n = 0, ne = 0, p = 0, n_edges = 0;
  double gs = 1.0;
  qs_dtype dt = QS_C64;
  int m = 0, c = 0;
  uint8_t* d_cut = nullptr;
  int* d_edges = nullptr;
  std::vector<QPassDesc> gpass, epass;  // gradient plan, energy plan
  std::vector<int> gns, ens;            // states carried by each pass (1 or 2)
  QPassDesc* d_gpass = nullptr;
  QPassDesc* d_epass = nullptr;
  SlotMap gslots, eslots;
  int n_fwd = 0, rev_passes = 0;
  void* d_coef = nullptr;
  int n_coef = 0;
  int *g_row = nullptr, *g_sidx = nullptr, *e_row = nullptr, *e_sidx = nullptr;
  double *g_w = nullptr, *e_w = nullptr;
  int grid1 = 1, grid2 = 1;
  double bytes_per_eval = 0;
  std::vector<double> host_coef;
  // complex64 reverse sweep on interleaved (psi, lam): the lam state's buffer
  // holds the first half of the amplitudes and this private buffer the second
  bool il = false;
  void* d_il_priv = nullptr;
  int* d_max = nullptr;  // qs_qaoa_max_cut result
  // adjoint checkpoints: psi saved after these forward passes, reloaded before
  // the reverse pass that undoes the next one
  std::vector<int> ck_after;
  std::vector<void*> ckpt;
  // complex64 passes with separate forward (psi alone, mf tile bits, cf low
  // bits) and reverse (psi/lam interleaved, mr, cr) tile shapes; cut values
  // are formed in the kernels, d_cut is only made for qs_qaoa_max_cut
  bool xp = false;
  int xmf = 0, xcf = 0, xmr = 0, xcr = 0;
  std::vector<XPass> xg, xe;       // gradient plan, energy plan
  std::vector<int> xg_two, xe_two; // kernel of each pass: 0 psi alone, 1 psi/lam
  XPass* d_xg = nullptr;
  XPass* d_xe = nullptr;
  uint8_t* d_xfs = nullptr;
  int xgrid_f = 1, xgrid_r = 1, xstride = 1;
  double xbytes_grad = 0, xbytes_energy = 0;
};

namespace {

// ---------------------------------------------------------------------------- checkpoints

// Reload psi into the interleaved reverse buffer: amplitude x is
// (psi.re, lam.re, psi.im, lam.im) at il0[x] for x < half, il1[x - half] after.
__global__ void il_reload_kernel(float4* __restrict__ il0, float4* __restrict__ il1, uint64_t half,
                                 const float2* __restrict__ ck, uint64_t N) {
  for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < N; x += (uint64_t)gridDim.x * blockDim.x) {
    float4* e = x < half ? il0 + x : il1 + (x - half);
    float4 v = *e;
    const float2 p = __ldcs(ck + x);
    v.x = p.x;
    v.z = p.y;
    *e = v;
  }
}

// ---------------------------------------------------------------------------- schedule

enum QOpKind { QO_RX, QO_COST, QO_GRAD_RX, QO_GRAD_COST, QO_ENERGY };
struct QOp {
  int kind;
  int layer;
  int bit;
};
struct SchedPass {
  uint64_t S;
  std::vector<QOp> ops;  // forward ops (QO_RX, QO_COST)
};

inline int popc(uint64_t x) { return __builtin_popcountll(x); }

std::vector<SchedPass> make_schedule(int n, int p, int m, int c) {
  std::vector<SchedPass> passes;
  const uint64_t all = (n >= 64) ? ~0ull : ((1ull << n) - 1);
  const uint64_t low = (1ull << c) - 1;
  auto fill = [&](uint64_t S) {
    for (int q = 0; q < n && popc(S) < m; ++q) S |= 1ull << q;
    return S;
  };
  SchedPass first;
  first.S = fill(low);
  first.ops.push_back({QO_COST, 0, -1});
  for (int q = 0; q < n; ++q)
    if ((first.S >> q) & 1) first.ops.push_back({QO_RX, 0, q});
  passes.push_back(first);
  int layer = 0;
  uint64_t done = first.S;
  while (!(layer == p - 1 && done == all)) {
    const uint64_t U = all & ~done;
    SchedPass P;
    if (popc(U | low) <= m) {
      P.S = fill(U | low);
      for (int q = 0; q < n; ++q)
        if ((U >> q) & 1) P.ops.push_back({QO_RX, layer, q});
      if (layer + 1 < p) {
        ++layer;
        P.ops.push_back({QO_COST, layer, -1});
        for (int q = 0; q < n; ++q)
          if ((P.S >> q) & 1) P.ops.push_back({QO_RX, layer, q});
        done = P.S;
      } else {
        done = all;
      }
    } else {
      uint64_t S = low;
      for (int q = 0; q < n && popc(S) < m; ++q)
        if ((U >> q) & 1) S |= 1ull << q;
      P.S = S;
      for (int q = 0; q < n; ++q)
        if (((U & S) >> q) & 1) P.ops.push_back({QO_RX, layer, q});
      done |= U & S;
    }
    passes.push_back(P);
  }
  return passes;
}

std::vector<QOp> reverse_ops(const std::vector<QOp>& fwd) {
  std::vector<QOp> r;
  for (size_t i = fwd.size(); i-- > 0;) {
    const QOp& o = fwd[i];
    r.push_back({o.kind == QO_RX ? QO_GRAD_RX : QO_GRAD_COST, o.layer, o.bit});
  }
  return r;
}

// ---------------------------------------------------------------------------- pass builder

// Order of the sub-cube bits.  Threads of a half-warp (complex64, 8-byte
// accesses) or quarter-warp (complex128) take consecutive sub-cubes, so the
// lowest sub-cube bits should spread their accesses over distinct bank slots:
// with the chunk swizzle, chunk bit b lands on slot bit b mod 3, and for
// complex64 local bit 0 picks the half of a chunk.
std::vector<int> order_q(const std::vector<int>& rest, bool c64) {
  std::vector<int> q, tail;
  std::vector<char> used(rest.size(), 0);
  if (c64)
    for (size_t i = 0; i < rest.size(); ++i)
      if (rest[i] == 0) {
        q.push_back(0);
        used[i] = 1;
      }
  for (int r = 0; r < 3; ++r)
    for (size_t i = 0; i < rest.size(); ++i) {
      const int chunk_bit = c64 ? rest[i] - 1 : rest[i];
      if (!used[i] && chunk_bit >= 0 && chunk_bit % 3 == r) {
        q.push_back(rest[i]);
        used[i] = 1;
        break;
      }
    }
  std::sort(q.begin(), q.end());
  for (size_t i = 0; i < rest.size(); ++i)
    if (!used[i]) tail.push_back(rest[i]);
  q.insert(q.end(), tail.begin(), tail.end());
  return q;
}

struct QBuild {
  int n, m, c, p;
  double gs;
  qs_dtype dt;
};

// Outputs: 0 = E, 1 + l = dgamma_l, 1 + p + l = dbeta_l.
qs_status build_qpass(const QBuild& B, uint64_t S, const std::vector<QOp>& ops, uint32_t flags, QPassDesc* out,
                      SlotMap* slots) {
  QPassDesc D;
  std::memset(&D, 0, sizeof(D));
  D.m = B.m;
  D.c = B.c;
  D.flags = flags;
  D.plus_amp = std::pow(2.0, -0.5 * B.n);
  int local_of[64], global_of[16], k = 0;
  for (int q = 0; q < 64; ++q) local_of[q] = -1;
  for (int q = 0; q < B.n; ++q)
    if ((S >> q) & 1) {
      local_of[q] = k;
      global_of[k++] = q;
    } else {
      D.comp[D.ncomp++] = (int8_t)q;
    }
  for (int i = 0; i < 64; ++i) {
    uint64_t a = 0, b = 0;
    for (int j = 0; j < 6; ++j)
      if ((i >> j) & 1) {
        if (B.c + j < B.m) a |= 1ull << global_of[B.c + j];
        if (B.c + 6 + j < B.m) b |= 1ull << global_of[B.c + 6 + j];
      }
    D.hiA[i] = a;
    D.hiB[i] = b;
  }
  int lo = 1 << 30, hi = -1;
  for (const QOp& o : ops) {
    lo = std::min(lo, o.layer);
    hi = std::max(hi, o.layer);
  }
  if (hi - lo + 1 > kQaoaMaxLayersPerPass) {
    set_error("qaoa planner: a pass spans more than two layers (internal error)");
    return QS_ERR_UNSUPPORTED;
  }
  D.layer_lo = lo;
  D.n_layers = hi - lo + 1;
  std::vector<int> acc_out;
  std::vector<double> acc_w;
  auto acc_of = [&](int o, double w) {
    for (size_t i = 0; i < acc_out.size(); ++i)
      if (acc_out[i] == o) return (int)i;
    acc_out.push_back(o);
    acc_w.push_back(w);
    return (int)acc_out.size() - 1;
  };
  // Phases hold up to 4 distinct RX bits.  A layer's block of RX ops is
  // reordered (RX on distinct qubits commute) to start with the bits already
  // held in registers by the current phase.
  std::vector<std::vector<int>> phase_bits(1);
  std::vector<std::vector<QStep>> phase_steps(1);
  size_t i = 0;
  while (i < ops.size()) {
    const QOp o = ops[i];
    if (o.kind == QO_RX || o.kind == QO_GRAD_RX) {
      size_t j = i;
      while (j < ops.size() && ops[j].kind == o.kind && ops[j].layer == o.layer) ++j;
      std::vector<int> block;
      for (size_t t = i; t < j; ++t) block.push_back(ops[t].bit);
      const std::vector<int> cur0 = phase_bits.back();
      std::stable_sort(block.begin(), block.end(), [&](int a, int b) {
        const bool ia = std::find(cur0.begin(), cur0.end(), a) != cur0.end();
        const bool ib = std::find(cur0.begin(), cur0.end(), b) != cur0.end();
        return ia > ib;
      });
      const uint8_t ty = o.kind == QO_RX ? QST_RX : QST_GRAD_RX;
      for (int bit : block) {
        auto* cur = &phase_bits.back();
        auto it = std::find(cur->begin(), cur->end(), bit);
        if (it == cur->end()) {
          if (cur->size() == 4 || phase_steps.back().size() >= (size_t)kQaoaMaxSteps) {
            phase_bits.emplace_back();
            phase_steps.emplace_back();
            cur = &phase_bits.back();
          }
          cur->push_back(bit);
          it = cur->end() - 1;
        }
        const int rb = (int)(it - cur->begin());
        auto& steps = phase_steps.back();
        if (!steps.empty() && steps.back().type == ty && steps.back().layer == o.layer - lo &&
            !(steps.back().mask & (1 << rb))) {
          steps.back().mask |= (uint8_t)(1 << rb);
        } else {
          if (steps.size() >= (size_t)kQaoaMaxSteps) {
            set_error("qaoa planner: too many steps in a phase (internal error)");
            return QS_ERR_UNSUPPORTED;
          }
          QStep st;
          std::memset(&st, 0, sizeof(st));
          st.type = ty;
          st.mask = (uint8_t)(1 << rb);
          st.layer = (uint16_t)(o.layer - lo);
          if (ty == QST_GRAD_RX) {
            st.acc = (uint8_t)acc_of(1 + B.p + o.layer, 1.0);
            st.flags = QSF_DAG | QSF_LAM;
          }
          steps.push_back(st);
        }
      }
      i = j;
      continue;
    }
    if (phase_steps.back().size() >= (size_t)kQaoaMaxSteps) {
      phase_bits.emplace_back();
      phase_steps.emplace_back();
    }
    QStep st;
    std::memset(&st, 0, sizeof(st));
    st.layer = (uint16_t)(o.layer - lo);
    if (o.kind == QO_COST) {
      st.type = QST_COST;
    } else if (o.kind == QO_GRAD_COST) {
      st.type = QST_GRAD_COST;
      st.flags = QSF_LAM;
      st.acc = (uint8_t)acc_of(1 + o.layer, 2.0 * B.gs);
    } else {
      st.type = QST_ENERGY;
      st.acc = (uint8_t)acc_of(0, 1.0);
    }
    phase_steps.back().push_back(st);
    ++i;
  }
  if (acc_out.size() > (size_t)kQaoaMaxAcc || phase_bits.size() > (size_t)kQaoaMaxPhases) {
    set_error("qaoa planner: pass exceeds accumulator/phase limits (internal error)");
    return QS_ERR_UNSUPPORTED;
  }
  // shared-memory elements: 8-byte complex64 amplitudes (two per swizzled
  // 16-byte chunk), or 16 bytes (complex128, or interleaved complex64 psi/lam)
  const bool el8 = B.dt == QS_C64 && !(flags & PF_LOAD_IL);
  D.n_phases = (int)phase_bits.size();
  for (int ph = 0; ph < D.n_phases; ++ph) {
    QPhase& P = D.phases[ph];
    uint32_t R = 0;
    int ri = 0;
    for (int bit : phase_bits[ph]) {
      P.R[ri++] = (int8_t)local_of[bit];
      R |= 1u << local_of[bit];
    }
    for (int l = 0; l < B.m && ri < 4; ++l)
      if (!((R >> l) & 1)) {
        P.R[ri++] = (int8_t)l;
        R |= 1u << l;
      }
    std::vector<int> rest;
    for (int l = 0; l < B.m; ++l)
      if (!((R >> l) & 1)) rest.push_back(l);
    const std::vector<int> q = order_q(rest, el8);
    P.nq = (int8_t)q.size();
    for (size_t t = 0; t < q.size(); ++t) {
      P.Q[t] = (int8_t)q[t];
      P.sq[t] = (uint16_t)qaoa_swizzle(el8, 1u << q[t]);
    }
    for (int r = 0; r < 4; ++r) P.sreg[r] = (uint16_t)qaoa_swizzle(el8, 1u << P.R[r]);
    P.n_steps = (int8_t)phase_steps[ph].size();
    P.need_cut = 0;
    for (size_t t = 0; t < phase_steps[ph].size(); ++t) {
      P.steps[t] = phase_steps[ph][t];
      const uint8_t ty = phase_steps[ph][t].type;
      if (ty == QST_COST || ty == QST_GRAD_COST || ty == QST_ENERGY) P.need_cut = 1;
    }
  }
  D.n_acc = (int)acc_out.size();
  D.slot_base = (int)slots->out.size();
  for (size_t a = 0; a < acc_out.size(); ++a) {
    slots->out.push_back(acc_out[a]);
    slots->weight.push_back(acc_w[a]);
  }
  *out = D;
  return QS_OK;
}

uint32_t cut_flag(const std::vector<QOp>& ops) {
  for (const auto& o : ops)
    if (o.kind != QO_RX && o.kind != QO_GRAD_RX) return PF_NEED_CUT;
  return 0;
}

struct CoefLayout {
  int per_layer, lut, lut_dag, rx, rx_dag;
  int at(int l, int which) const { return l * per_layer + which; }
};

CoefLayout layout_for(int n_edges) {
  CoefLayout L;
  L.lut = 0;
  L.lut_dag = n_edges + 1;
  L.rx = 2 * (n_edges + 1);
  L.rx_dag = L.rx + 1;
  L.per_layer = L.rx + 2;
  return L;
}

double pass_bytes(uint32_t f, double S, double N) {
  return S * (((f & PF_LOAD_PSI) ? 1 : 0) + ((f & PF_LOAD_LAM) ? 1 : 0) + ((f & PF_STORE_PSI) ? 1 : 0) +
              ((f & PF_STORE_LAM) ? 1 : 0) + ((f & PF_LOAD_IL) ? 2 : 0) + ((f & PF_STORE_IL) ? 2 : 0)) +
         ((f & PF_NEED_CUT) ? N : 0.0);
}

// ---------------------------------------------------------------------------- two-shape complex64 passes

qs_status build_x_engine(qs_qaoa* q, const std::vector<std::pair<int, int>>& es, const qs_options* opts) {
  const int eng = opts ? opts->fuse : 0;
  const int mr = (eng == 2 && opts->tile_bits) ? opts->tile_bits : 12;
  const int cr = (eng == 2 && opts->low_bits) ? opts->low_bits : 3;
  QS_CHECK(mr >= 9 && mr <= 12, "tile_bits of the complex64 two-shape QAOA passes must be 9..12");
  QS_CHECK(cr >= 2 && cr <= mr - 4, "low_bits of the complex64 two-shape QAOA passes must be 2..tile_bits-4");
  QS_CHECK(!(opts && opts->checkpoint), "QAOA checkpoints need the general passes (fuse = 1)");
  const int n = q->n, p = q->p;
  QS_CHECK(n > mr + 1, "the complex64 two-shape QAOA passes need n_qubits > tile_bits + 1");
  XBuild B;
  B.n = n;
  B.p = p;
  B.mf = mr + 1;
  B.cf = cr + 1;
  B.mr = mr;
  B.cr = cr;
  B.n_edges = q->n_edges;
  B.edges = es;
  XPlans X;
  QS_TRY(qx_make_plans(B, q->gs, &X));
  q->xmf = B.mf;
  q->xcf = B.cf;
  q->xmr = mr;
  q->xcr = cr;
  q->xg = X.grad;
  q->xg_two = X.grad_two;
  q->xe = X.energy;
  q->xe_two = X.energy_two;
  q->gslots = X.gslots;
  q->eslots = X.eslots;
  int ph_f = 1, ph_r = 1;  // the most phases of a pass of each kernel (shared-memory sizing)
  for (size_t i = 0; i < X.grad.size(); ++i) (X.grad_two[i] ? ph_r : ph_f) = std::max(X.grad_two[i] ? ph_r : ph_f, X.grad[i].n_phases);
  for (size_t i = 0; i < X.energy.size(); ++i) ph_f = std::max(ph_f, X.energy[i].n_phases);
  q->xgrid_f = qx_grid(0, B.mf, q->n_edges, ph_f, 1ull << (n - B.mf));
  q->xgrid_r = qx_grid(1, mr, q->n_edges, ph_r, 1ull << (n - mr));
  if (q->xgrid_f < 1 || q->xgrid_r < 1) {
    set_error("qaoa: the two-shape tiles do not fit in shared memory");
    return QS_ERR_UNSUPPORTED;
  }
  q->xstride = std::max(q->xgrid_f, q->xgrid_r);
  QS_CUDA(cudaMalloc(&q->d_xg, q->xg.size() * sizeof(XPass)));
  QS_CUDA(cudaMalloc(&q->d_xe, q->xe.size() * sizeof(XPass)));
  QS_CUDA(cudaMalloc(&q->d_xfs, X.fs.size()));
  QS_CUDA(cudaMemcpy(q->d_xg, q->xg.data(), q->xg.size() * sizeof(XPass), cudaMemcpyHostToDevice));
  QS_CUDA(cudaMemcpy(q->d_xe, q->xe.data(), q->xe.size() * sizeof(XPass), cudaMemcpyHostToDevice));
  QS_CUDA(cudaMemcpy(q->d_xfs, X.fs.data(), X.fs.size(), cudaMemcpyHostToDevice));
  {
    std::vector<int> ev;
    for (const auto& e : es) {
      ev.push_back(e.first);
      ev.push_back(e.second);
    }
    QS_CUDA(cudaMalloc(&q->d_edges, sizeof(int) * ev.size()));
    QS_CUDA(cudaMemcpy(q->d_edges, ev.data(), sizeof(int) * ev.size(), cudaMemcpyHostToDevice));
  }
  // psi and lam interleaved in one buffer of 16 bytes per amplitude (lam's own
  // buffer is left unused by these passes)
  QS_CUDA(cudaMalloc(&q->d_il_priv, (size_t)16 << n));
  q->il = true;
  q->n_coef = X.n_coef;
  QS_CUDA(cudaMalloc(&q->d_coef, (size_t)q->n_coef * 16));
  QS_TRY(build_csr(q->gslots, 1 + 2 * p, &q->g_row, &q->g_sidx, &q->g_w, nullptr));
  QS_TRY(build_csr(q->eslots, 1, &q->e_row, &q->e_sidx, &q->e_w, nullptr));
  q->xbytes_grad = X.bytes_grad;
  q->xbytes_energy = X.bytes_energy;
  q->n_fwd = X.n_fwd - 1;
  q->rev_passes = X.n_rev;
  q->bytes_per_eval = X.bytes_grad;
  q->xp = true;
  return QS_OK;
}

}  // namespace

extern "C" {

qs_status qs_qaoa_create(int n_qubits, const int* edges, int n_edges, int p, double gamma_scale, qs_dtype dtype,
                         const qs_options* opts, qs_qaoa** out) {
  QS_CHECK(out != nullptr, "out is null");
  QS_CHECK(n_qubits >= kRegBits && n_qubits <= kMaxQubits, "n_qubits must be in 4..34");
  QS_CHECK(n_edges >= 1 && n_edges <= 255 && edges != nullptr, "need 1..255 edges");
  QS_CHECK(p >= 1 && p <= 1024, "p must be in 1..1024");
  QS_CHECK(std::isfinite(gamma_scale), "gamma_scale must be finite");
  QS_CHECK(dtype == QS_C64 || dtype == QS_C128, "invalid dtype");
  std::vector<std::pair<int, int>> es;
  for (int e = 0; e < n_edges; ++e) {
    const int a = edges[2 * e], b = edges[2 * e + 1];
    QS_CHECK(a >= 0 && a < n_qubits && b >= 0 && b < n_qubits && a != b, "edge endpoint out of range or a self-loop");
    es.push_back({std::min(a, b), std::max(a, b)});
  }
  std::sort(es.begin(), es.end());
  QS_CHECK(std::adjacent_find(es.begin(), es.end()) == es.end(), "repeated edge");
  if (opts) {
    QS_CHECK(opts->tile_bits == 0 || (opts->tile_bits >= kMinTileBits && opts->tile_bits <= kMaxTileBits),
             "tile_bits must be 0 or 6..13");
    QS_CHECK(opts->low_bits >= 0 && opts->low_bits <= kMaxTileBits, "low_bits must be 0..13");
    QS_CHECK(opts->checkpoint >= 0, "checkpoint must be >= 0");
    QS_CHECK(opts->fuse >= 0 && opts->fuse <= 2,
             "QAOA fuse option must be 0 (automatic), 1 (general passes) or 2 (two-shape passes)");
    QS_CHECK(opts->fuse != 2 || dtype == QS_C64, "the two-shape QAOA passes are complex64 only");
  }

  qs_qaoa* q = new qs_qaoa;
  q->n = n_qubits;
  q->ne = n_qubits;
  q->p = p;
  q->n_edges = n_edges;
  q->gs = gamma_scale;
  q->dt = dtype;
  // engine: fuse 2 = complex64 two-shape passes, 1 = general passes, 0 = automatic
  // (two-shape passes for complex64 from 18 qubits when no tile option is set)
  const int eng = opts ? opts->fuse : 0;
  const bool want_x = dtype == QS_C64 &&
                      (eng == 2 || (eng == 0 && n_qubits >= 18 &&
                                    !(opts && (opts->tile_bits || opts->low_bits || opts->checkpoint))));
  if (want_x) {
    const qs_status xs = build_x_engine(q, es, opts);
    if (xs == QS_OK) {
      *out = q;
      return QS_OK;
    }
    if (eng == 2) {
      qs_qaoa_destroy(q);
      return xs;
    }
    // automatic choice: fall back to the general passes
    qs_qaoa* fresh = new qs_qaoa;
    fresh->n = q->n;
    fresh->ne = q->ne;
    fresh->p = q->p;
    fresh->n_edges = q->n_edges;
    fresh->gs = q->gs;
    fresh->dt = q->dt;
    qs_qaoa_destroy(q);
    q = fresh;
    (void)cudaGetLastError();
  }
  int mm = (opts && opts->tile_bits) ? opts->tile_bits : (dtype == QS_C64 ? 12 : 11);
  // double-buffered psi + lam tiles must fit twice in shared memory
  mm = std::max(kRegBits, std::min({mm, dtype == QS_C64 ? 12 : 11, q->n}));
  int cc = (opts && opts->low_bits) ? opts->low_bits : 0;
  if (cc == 0) {  // fewest passes; ties go to more contiguous bits
    int best = 1 << 30;
    for (int c = 2; c <= std::min(6, mm); ++c) {
      const int np = (int)make_schedule(q->n, p, mm, c).size();
      if (np <= best) {
        best = np;
        cc = c;
      }
    }
  }
  cc = std::max(1, std::min(cc, mm));
  if (mm - cc > 12) cc = mm - 12;
  q->m = mm;
  q->c = cc;
  if (dtype == QS_C64 && q->n >= 5 && qaoa_il_grid_size(mm, n_edges, 1ull << (q->n - mm)) > 0) {
    // the interleaved reverse sweep needs a buffer the size of one state; without
    // it the engine runs the reverse passes on separate psi and lam tiles
    if (cudaMalloc(&q->d_il_priv, (size_t)8 << q->n) == cudaSuccess)
      q->il = true;
    else
      (void)cudaGetLastError();
  }

  auto fail = [&](qs_status s) {
    qs_qaoa_destroy(q);
    return s;
  };
  const uint64_t N = 1ull << q->n;
  cudaError_t e = cudaMalloc(&q->d_cut, N);
  if (e != cudaSuccess) return fail(cuda_fail(e, "cudaMalloc(cut values)"));
  e = cudaMalloc(&q->d_edges, sizeof(int) * 2 * n_edges);
  if (e != cudaSuccess) return fail(cuda_fail(e, "cudaMalloc(edges)"));
  e = cudaMemcpy(q->d_edges, edges, sizeof(int) * 2 * n_edges, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fail(cuda_fail(e, "cudaMemcpy(edges)"));
  qs_status s = launch_cut_values(q->d_cut, q->n, q->d_edges, n_edges, nullptr);
  if (s != QS_OK) return fail(s);
  const CoefLayout L = layout_for(n_edges);
  q->n_coef = L.per_layer * p;
  e = cudaMalloc(&q->d_coef, (size_t)q->n_coef * 16);
  if (e != cudaSuccess) return fail(cuda_fail(e, "cudaMalloc(coefficients)"));

  const std::vector<SchedPass> sched = make_schedule(q->n, p, mm, cc);
  const int K = (int)sched.size();
  const QBuild B{q->n, mm, cc, p, gamma_scale, dtype};
  QPassDesc D;
  // gradient plan: forward 0..K-2, turnaround K-1, reverse K-2..0
  for (int i = 0; i < K - 1; ++i) {
    const uint32_t fl = (i == 0 ? PF_GEN_PLUS : PF_LOAD_PSI) | PF_STORE_PSI | cut_flag(sched[i].ops);
    if ((s = build_qpass(B, sched[i].S, sched[i].ops, fl, &D, &q->gslots)) != QS_OK) return fail(s);
    q->gpass.push_back(D);
    q->gns.push_back(1);
  }
  {
    std::vector<QOp> ops = sched[K - 1].ops;
    ops.push_back({QO_ENERGY, sched[K - 1].ops.back().layer, -1});
    const std::vector<QOp> r = reverse_ops(sched[K - 1].ops);
    ops.insert(ops.end(), r.begin(), r.end());
    const uint32_t out = (q->il && K > 1) ? (uint32_t)PF_STORE_IL : (uint32_t)PF_STORE_LAM;
    const uint32_t fl = (K == 1 ? PF_GEN_PLUS : PF_LOAD_PSI) | out | PF_NEED_CUT;
    if ((s = build_qpass(B, sched[K - 1].S, ops, fl, &D, &q->gslots)) != QS_OK) return fail(s);
    q->gpass.push_back(D);
    q->gns.push_back(2);
  }
  for (int i = K - 2; i >= 0; --i) {
    const std::vector<QOp> r = reverse_ops(sched[i].ops);
    const uint32_t st = i > 0 ? (PF_STORE_PSI | PF_STORE_LAM) : 0;
    const uint32_t fl = q->il ? (PF_LOAD_IL | (i > 0 ? PF_STORE_IL : 0u) | cut_flag(r))
                              : (PF_LOAD_PSI | PF_LOAD_LAM | st | cut_flag(r));
    if ((s = build_qpass(B, sched[i].S, r, fl, &D, &q->gslots)) != QS_OK) return fail(s);
    q->gpass.push_back(D);
    q->gns.push_back(2);
  }
  q->n_fwd = K - 1;
  q->rev_passes = K - 1;
  if (opts && opts->checkpoint > 0)  // about two forward passes per layer
    for (int i = 0; i + 1 < K - 1; ++i)
      if ((i + 1) % (2 * opts->checkpoint) == 0) q->ck_after.push_back(i);
  // energy plan: the forward passes with the energy appended to the last
  for (int i = 0; i < K; ++i) {
    std::vector<QOp> ops = sched[i].ops;
    uint32_t fl = (i == 0 ? PF_GEN_PLUS : PF_LOAD_PSI) | PF_STORE_PSI | cut_flag(ops);
    if (i == K - 1) {
      ops.push_back({QO_ENERGY, ops.back().layer, -1});
      fl |= PF_NEED_CUT;
    }
    if ((s = build_qpass(B, sched[i].S, ops, fl, &D, &q->eslots)) != QS_OK) return fail(s);
    q->epass.push_back(D);
    q->ens.push_back(1);
  }
  e = cudaMalloc(&q->d_gpass, q->gpass.size() * sizeof(QPassDesc));
  if (e == cudaSuccess) e = cudaMalloc(&q->d_epass, q->epass.size() * sizeof(QPassDesc));
  if (e == cudaSuccess)
    e = cudaMemcpy(q->d_gpass, q->gpass.data(), q->gpass.size() * sizeof(QPassDesc), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(q->d_epass, q->epass.data(), q->epass.size() * sizeof(QPassDesc), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fail(cuda_fail(e, "uploading the QAOA plan"));
  s = build_csr(q->gslots, 1 + 2 * p, &q->g_row, &q->g_sidx, &q->g_w, nullptr);
  if (s == QS_OK) s = build_csr(q->eslots, 1, &q->e_row, &q->e_sidx, &q->e_w, nullptr);
  if (s != QS_OK) return fail(s);
  const uint64_t n_tiles = 1ull << (q->n - mm);
  q->grid1 = qaoa_grid_size(dtype, mm, 1, n_edges, n_tiles);
  q->grid2 = qaoa_grid_size(dtype, mm, 2, n_edges, n_tiles);
  if (q->il) q->grid2 = std::min(q->grid2, qaoa_il_grid_size(mm, n_edges, n_tiles));
  if (q->grid1 < 1 || q->grid2 < 1) {
    set_error("qaoa: the tile does not fit in shared memory");
    return fail(QS_ERR_UNSUPPORTED);
  }
  const double Sb = (double)amp_bytes(dtype) * (double)N;
  for (const auto& P : q->gpass) q->bytes_per_eval += pass_bytes(P.flags, Sb, (double)N);
  *out = q;
  return QS_OK;
}

qs_status qs_qaoa_destroy(qs_qaoa* q) {
  if (!q) return QS_OK;
  cudaDeviceSynchronize();
  if (q->d_cut) cudaFree(q->d_cut);
  if (q->d_max) cudaFree(q->d_max);
  if (q->d_edges) cudaFree(q->d_edges);
  if (q->d_coef) cudaFree(q->d_coef);
  if (q->d_gpass) cudaFree(q->d_gpass);
  if (q->d_epass) cudaFree(q->d_epass);
  if (q->d_il_priv) cudaFree(q->d_il_priv);
  if (q->d_xg) cudaFree(q->d_xg);
  if (q->d_xe) cudaFree(q->d_xe);
  if (q->d_xfs) cudaFree(q->d_xfs);
  for (void* b : q->ckpt) cudaFree(b);
  for (int* pi : {q->g_row, q->g_sidx, q->e_row, q->e_sidx})
    if (pi) cudaFree(pi);
  for (double* pd : {q->g_w, q->e_w})
    if (pd) cudaFree(pd);
  delete q;
  return QS_OK;
}

qs_status qs_qaoa_info(const qs_qaoa* q, int* fwd_passes, int* rev_passes, double* bytes_per_eval) {
  QS_CHECK(q != nullptr, "null qaoa");
  if (fwd_passes) *fwd_passes = q->n_fwd + 1;
  if (rev_passes) *rev_passes = q->rev_passes;
  if (bytes_per_eval) *bytes_per_eval = q->bytes_per_eval;
  return QS_OK;
}

qs_status qs_qaoa_max_cut(qs_qaoa* q, int* max_cut) {
  QS_CHECK(q != nullptr && max_cut != nullptr, "null argument");
  if (!q->d_cut) {  // the two-shape passes form cut values in the kernels: build the array now
    QS_CUDA(cudaMalloc(&q->d_cut, 1ull << q->n));
    QS_TRY(launch_cut_values(q->d_cut, q->n, q->d_edges, q->n_edges, nullptr));
  }
  if (!q->d_max) QS_CUDA(cudaMalloc(&q->d_max, sizeof(int)));
  QS_TRY(launch_max_u8(q->d_cut, 1ull << q->n, q->d_max, nullptr));
  QS_CUDA(cudaMemcpy(max_cut, q->d_max, sizeof(int), cudaMemcpyDeviceToHost));
  return QS_OK;
}

}  // extern "C"

namespace {

qs_status fill_qaoa_coef(qs_qaoa* q, const double* gamma, const double* beta) {
  const CoefLayout L = layout_for(q->n_edges);
  std::vector<double>& tab = q->host_coef;
  tab.assign((size_t)q->n_coef * 2, 0.0);
  auto put = [&](int off, cd v) {
    tab[2 * off] = v.real();
    tab[2 * off + 1] = v.imag();
  };
  for (int l = 0; l < q->p; ++l) {
    QS_CHECK(std::isfinite(gamma[l]) && std::isfinite(beta[l]), "non-finite angle");
    for (int k = 0; k <= q->n_edges; ++k) {
      const double C = (double)(q->n_edges - 2 * k);
      const double ph = q->gs * gamma[l] * C;
      put(L.at(l, L.lut) + k, cd(std::cos(ph), -std::sin(ph)));
      put(L.at(l, L.lut_dag) + k, cd(std::cos(ph), std::sin(ph)));
    }
    const double c = std::cos(0.5 * beta[l]), s = std::sin(0.5 * beta[l]);
    put(L.at(l, L.rx), cd(c, s));
    put(L.at(l, L.rx_dag), cd(c, -s));
  }
  return QS_OK;
}

qs_status qaoa_check(qs_qaoa* q, qs_state* psi, const double* gamma, const double* beta) {
  QS_CHECK(q != nullptr, "null qaoa");
  QS_TRY(check_state(psi));
  QS_CHECK(psi->n == q->n && psi->dt == q->dt, "state n/dtype differs from the QAOA engine");
  QS_CHECK(gamma != nullptr && beta != nullptr, "null angles");
  return QS_OK;
}

qs_status run_qpasses(qs_qaoa* q, const std::vector<QPassDesc>& passes, const std::vector<int>& ns,
                      const QPassDesc* d_passes, void* psi, void* lam, double* partials, cudaStream_t st,
                      size_t begin = 0, size_t end = (size_t)-1) {
  end = std::min(end, passes.size());
  for (size_t i = begin; i < end; ++i) {
    QaoaLaunch L;
    L.il[0] = lam;  // the interleaved reverse sweep reuses lam's buffer as its first half
    L.il[1] = q->d_il_priv;
    L.psi = psi;
    L.lam = lam;
    L.coef = q->d_coef;
    L.cut = q->d_cut;
    L.partials = partials;
    L.n = q->n;
    L.n_edges = q->n_edges;
    L.stride = q->grid2;
    L.grid = (ns[i] == 2 || passes[i].n_acc > 0) ? q->grid2 : q->grid1;
    TraceRec* rec = trace_begin(st);
    QS_TRY(launch_qaoa_pass(q->dt, d_passes + i, ns[i], q->m, passes[i].flags, L, st));
    if (rec) {
      rec->bytes = pass_bytes(passes[i].flags, (double)amp_bytes(q->dt) * (double)(1ull << q->n),
                              (double)(1ull << q->n));
      rec->kind = (passes[i].flags & PF_LOAD_IL) ? QS_TRACE_QAOA_IL : ns[i] == 2 ? QS_TRACE_QAOA_TWO : QS_TRACE_QAOA_FWD;
      QS_CUDA(cudaEventRecord(rec->end, st));
    }
  }
  return QS_OK;
}

qs_status run_xpasses(qs_qaoa* q, const std::vector<XPass>& passes, const std::vector<int>& two,
                      const XPass* d_passes, void* psi, void* lam, double* partials, cudaStream_t st) {
  const double S = 8.0 * (double)(1ull << q->n);
  for (size_t i = 0; i < passes.size(); ++i) {
    XLaunch L;
    L.psi = reinterpret_cast<float2*>(psi);
    L.il = reinterpret_cast<float4*>(q->d_il_priv);  // (psi, lam) interleaved, 16 bytes per amplitude
    L.coef = reinterpret_cast<const float2*>(q->d_coef);
    L.fs = q->d_xfs;
    L.partials = partials;
    L.stride = q->xstride;
    L.grid = two[i] ? q->xgrid_r : q->xgrid_f;
    L.n = q->n;
    L.n_edges = q->n_edges;
    TraceRec* rec = trace_begin(st);
    QS_TRY(launch_qx_pass(two[i], d_passes + i, passes[i], L, st));
    if (rec) {
      const uint32_t f = passes[i].flags;
      double b = 0;
      if (!two[i]) {
        b = ((f & XF_GEN_PLUS) ? 0 : S) + ((f & XF_STORE) ? S : 0);
        rec->kind = QS_TRACE_QX_FWD;
      } else if (f & XF_LOAD_PSI) {
        b = S + ((f & XF_STORE) ? 2 * S : 0);
        rec->kind = QS_TRACE_QX_TURN;
      } else {
        b = 2 * S + ((f & XF_STORE) ? 2 * S : 0);
        rec->kind = QS_TRACE_QX_REV;
      }
      rec->bytes = b;
      QS_CUDA(cudaEventRecord(rec->end, st));
    }
  }
  return QS_OK;
}

// The call's coefficient table: the scaled-mixer table of the two-shape passes
// (and whether the energy plan leaves every qubit flipped), else the plain one.
qs_status fill_coef_for(qs_qaoa* q, const double* gamma, const double* beta, bool* flip) {
  *flip = false;
  if (!q->xp) return fill_qaoa_coef(q, gamma, beta);
  for (int l = 0; l < q->p; ++l)
    QS_CHECK(std::isfinite(gamma[l]) && std::isfinite(beta[l]), "non-finite angle");
  return qx_fill_coef(q->n, q->p, q->n_edges, q->gs, gamma, beta, q->xg, q->xe, q->n_coef, &q->host_coef, flip);
}

qs_status qaoa_energy(qs_qaoa* q, qs_state* psi, const double* gamma, const double* beta, double* energy) {
  QS_TRY(qaoa_check(q, psi, gamma, beta));
  cudaStream_t st = psi->st;
  bool flip = false;
  QS_TRY(fill_coef_for(q, gamma, beta, &flip));
  QS_TRY(upload_table(q->host_coef, q->dt, q->d_coef, st, psi->host_out));
  const int n_slots = (int)q->eslots.out.size();
  const size_t part = (size_t)std::max(n_slots, 1) * q->grid2;
  if (q->xp) {
    const size_t xpart = (size_t)std::max(n_slots, 1) * q->xstride;
    QS_TRY(ensure_scratch(psi, xpart + n_slots + 8));
    double* d_part = psi->scratch;
    double* d_slot = d_part + xpart;
    double* d_out = d_slot + n_slots;
    QS_CUDA(cudaMemsetAsync(d_part, 0, xpart * sizeof(double), st));
    QS_TRY(run_xpasses(q, q->xe, q->xe_two, q->d_xe, psi->ptr, nullptr, d_part, st));
    if (flip) QS_TRY(launch_qx_flip(reinterpret_cast<float2*>(psi->ptr), q->n, st));  // the evolved state exactly
    QS_TRY(launch_reduce_slots(d_part, n_slots, q->xstride, nullptr, d_slot, st));
    QS_TRY(launch_param_gather(d_slot, q->e_row, q->e_sidx, q->e_w, 1, d_out, st));
    if (energy) {
      QS_CUDA(cudaMemcpyAsync(energy, d_out, sizeof(double), cudaMemcpyDeviceToHost, st));
      QS_CUDA(cudaStreamSynchronize(st));
    }
    return QS_OK;
  }
  QS_TRY(ensure_scratch(psi, part + n_slots + 8));
  double* d_part = psi->scratch;
  double* d_slot = d_part + part;
  double* d_out = d_slot + n_slots;
  QS_TRY(run_qpasses(q, q->epass, q->ens, q->d_epass, psi->ptr, nullptr, d_part, st));
  QS_TRY(launch_reduce_slots(d_part, n_slots, q->grid2, nullptr, d_slot, st));
  QS_TRY(launch_param_gather(d_slot, q->e_row, q->e_sidx, q->e_w, 1, d_out, st));
  if (energy) {
    QS_CUDA(cudaMemcpyAsync(energy, d_out, sizeof(double), cudaMemcpyDeviceToHost, st));
    QS_CUDA(cudaStreamSynchronize(st));
  }
  return QS_OK;
}

}  // namespace

extern "C" {

qs_status qs_qaoa_evolve(qs_qaoa* q, qs_state* psi, const double* gamma, const double* beta) {
  return qaoa_energy(q, psi, gamma, beta, nullptr);
}

qs_status qs_qaoa_expectation(qs_qaoa* q, qs_state* psi, const double* gamma, const double* beta, double* energy) {
  QS_CHECK(energy != nullptr, "energy is null");
  return qaoa_energy(q, psi, gamma, beta, energy);
}

qs_status qs_qaoa_expectation_with_grad(qs_qaoa* q, qs_state* psi, qs_state* lam, const double* gamma,
                                        const double* beta, double* energy, double* dgamma, double* dbeta) {
  QS_TRY(qaoa_check(q, psi, gamma, beta));
  QS_TRY(check_state(lam));
  QS_CHECK(lam != psi && lam->ptr != psi->ptr, "psi and lam must be different states");
  QS_CHECK(lam->n == q->n && lam->dt == q->dt, "lam n/dtype differs from the QAOA engine");
  QS_CHECK(energy && dgamma && dbeta, "null output");
  if (lam->st != psi->st) QS_CUDA(cudaStreamSynchronize(lam->st));
  cudaStream_t st = psi->st;
  bool flip = false;  // psi and lam are undefined on return: no unflip needed
  QS_TRY(fill_coef_for(q, gamma, beta, &flip));
  QS_TRY(upload_table(q->host_coef, q->dt, q->d_coef, st, psi->host_out));
  const int n_slots = (int)q->gslots.out.size();
  const int n_out = 1 + 2 * q->p;
  const size_t part = (size_t)std::max(n_slots, 1) * (q->xp ? q->xstride : q->grid2);
  QS_TRY(ensure_scratch(psi, part + n_slots + n_out + 8));
  double* d_part = psi->scratch;
  double* d_slot = d_part + part;
  double* d_out = d_slot + n_slots;
  if (q->xp) {
    QS_CUDA(cudaMemsetAsync(d_part, 0, part * sizeof(double), st));
    QS_TRY(run_xpasses(q, q->xg, q->xg_two, q->d_xg, psi->ptr, lam->ptr, d_part, st));
    QS_TRY(launch_reduce_slots(d_part, n_slots, q->xstride, nullptr, d_slot, st));
  } else if (q->ck_after.empty()) {
    QS_TRY(run_qpasses(q, q->gpass, q->gns, q->d_gpass, psi->ptr, lam->ptr, d_part, st));
  } else {
    // checkpoints: psi saved after the chosen forward passes and reloaded before
    // the reverse pass that undoes the following one (gradient plan order:
    // forward 0..K-2, turnaround K-1, reverse of pass i at index 2K-2-i)
    const size_t bytes = amp_bytes(q->dt) << q->n;
    if (q->ckpt.size() != q->ck_after.size()) {
      for (void* b : q->ckpt) cudaFree(b);
      q->ckpt.assign(q->ck_after.size(), nullptr);
      for (auto& b : q->ckpt) QS_CUDA(cudaMalloc(&b, bytes));
    }
    const int K = q->n_fwd + 1;
    size_t b = 0;
    for (size_t j = 0; j < q->ck_after.size(); ++j) {
      const size_t e = (size_t)q->ck_after[j] + 1;
      QS_TRY(run_qpasses(q, q->gpass, q->gns, q->d_gpass, psi->ptr, lam->ptr, d_part, st, b, e));
      QS_CUDA(cudaMemcpyAsync(q->ckpt[j], psi->ptr, bytes, cudaMemcpyDeviceToDevice, st));
      b = e;
    }
    for (size_t jj = q->ck_after.size(); jj-- > 0;) {
      const size_t e = (size_t)(2 * K - 2 - q->ck_after[jj]);
      QS_TRY(run_qpasses(q, q->gpass, q->gns, q->d_gpass, psi->ptr, lam->ptr, d_part, st, b, e));
      if (q->il) {
        const uint64_t N = 1ull << q->n;
        const int grid = (int)std::min<uint64_t>((N + 255) / 256, 152 * 16);
        il_reload_kernel<<<grid, 256, 0, st>>>(reinterpret_cast<float4*>(lam->ptr),
                                               reinterpret_cast<float4*>(q->d_il_priv), N / 2,
                                               reinterpret_cast<const float2*>(q->ckpt[jj]), N);
        QS_CUDA(cudaGetLastError());
      } else {
        QS_CUDA(cudaMemcpyAsync(psi->ptr, q->ckpt[jj], bytes, cudaMemcpyDeviceToDevice, st));
      }
      b = e;
    }
    QS_TRY(run_qpasses(q, q->gpass, q->gns, q->d_gpass, psi->ptr, lam->ptr, d_part, st, b, q->gpass.size()));
  }
  if (!q->xp) QS_TRY(launch_reduce_slots(d_part, n_slots, q->grid2, nullptr, d_slot, st));
  QS_TRY(launch_param_gather(d_slot, q->g_row, q->g_sidx, q->g_w, n_out, d_out, st));
  std::vector<double> h(n_out);
  QS_CUDA(cudaMemcpyAsync(h.data(), d_out, n_out * sizeof(double), cudaMemcpyDeviceToHost, st));
  QS_CUDA(cudaStreamSynchronize(st));
  *energy = h[0];
  for (int l = 0; l < q->p; ++l) {
    dgamma[l] = h[1 + l];
    dbeta[l] = h[1 + q->p + l];
  }
  return QS_OK;
}

qs_status qs_qaoa_evaluate(int n_qubits, const int* edges, int n_edges, int p, double gamma_scale,
                           const double* gamma, const double* beta, qs_dtype dtype, double* energy, double* dgamma,
                           double* dbeta) {
  qs_qaoa* q = nullptr;
  qs_state *psi = nullptr, *lam = nullptr;
  qs_status s = qs_qaoa_create(n_qubits, edges, n_edges, p, gamma_scale, dtype, nullptr, &q);
  if (s == QS_OK) s = qs_state_create(n_qubits, dtype, nullptr, 0, nullptr, &psi);
  if (s == QS_OK) s = qs_state_create(n_qubits, dtype, nullptr, 0, nullptr, &lam);
  if (s == QS_OK) s = qs_qaoa_expectation_with_grad(q, psi, lam, gamma, beta, energy, dgamma, dbeta);
  qs_state_destroy(lam);
  qs_state_destroy(psi);
  qs_qaoa_destroy(q);
  return s;
}

}  // extern "C"
