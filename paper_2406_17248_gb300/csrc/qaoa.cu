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

using cd = std::complex<double>;
using namespace qs;

namespace {

struct SchedOp {
  int type;  // 0 = RX(layer, bit), 1 = COST(layer)
  int layer;
  int bit;
};
struct SchedPass {
  uint64_t S;
  std::vector<SchedOp> ops;
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
  // first pass: cost 0 then mixer 0 on the lowest m bits
  SchedPass first;
  first.S = fill(low);
  first.ops.push_back({1, 0, -1});
  for (int q = 0; q < n; ++q)
    if ((first.S >> q) & 1) first.ops.push_back({0, 0, q});
  passes.push_back(first);
  int layer = 0;
  uint64_t done = first.S;
  while (!(layer == p - 1 && done == all)) {
    const uint64_t U = all & ~done;
    SchedPass P;
    if (popc(U | low) <= m) {
      P.S = fill(U | low);
      for (int q = 0; q < n; ++q)
        if ((U >> q) & 1) P.ops.push_back({0, layer, q});
      if (layer + 1 < p) {
        ++layer;
        P.ops.push_back({1, layer, -1});
        for (int q = 0; q < n; ++q)
          if ((P.S >> q) & 1) P.ops.push_back({0, layer, q});
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
        if (((U & S) >> q) & 1) P.ops.push_back({0, layer, q});
      done |= U & S;
    }
    passes.push_back(P);
  }
  return passes;
}

struct CoefLayout {
  int per_layer, lut, lut_dag, rx, rx_dag;
  int n_edges;
  int at(int l, int which) const { return l * per_layer + which; }
};

CoefLayout layout_for(int n_edges) {
  CoefLayout L;
  L.n_edges = n_edges;
  L.lut = 0;
  L.lut_dag = n_edges + 1;
  L.rx = 2 * (n_edges + 1);
  L.rx_dag = L.rx + 1;
  L.per_layer = L.rx + 2;
  return L;
}

PlanItem rx_item(int bit, std::vector<ItemOp> ops) {
  PlanItem it;
  it.kind = IK_DENSE1;
  it.nt = 1;
  it.t[0] = it.t[1] = bit;
  it.ctrl = 0;
  it.touched = 1ull << bit;
  it.ops = std::move(ops);
  return it;
}

PlanItem global_item(uint64_t all, std::vector<ItemOp> ops) {
  PlanItem it;
  it.kind = IK_GLOBAL_DIAG;
  it.nt = 0;
  it.t[0] = it.t[1] = 0;
  it.ctrl = 0;
  it.touched = all;
  it.ops = std::move(ops);
  return it;
}

// Forward items of one scheduled pass.
std::vector<PlanItem> fwd_items(const SchedPass& sp, const CoefLayout& L, uint64_t all) {
  std::vector<PlanItem> v;
  for (const SchedOp& o : sp.ops) {
    if (o.type == 0)
      v.push_back(rx_item(o.bit, {ItemOp{OP_RX, 0, L.at(o.layer, L.rx), -1, 0}}));
    else
      v.push_back(global_item(all, {ItemOp{OP_COST, 0, L.at(o.layer, L.lut), -1, 0}}));
  }
  return v;
}

// Reverse items (adjoint of the pass, with gradient ops) in reverse order.
// Outputs: 0 = E, 1 + l = dgamma_l, 1 + p + l = dbeta_l.
std::vector<PlanItem> rev_items(const SchedPass& sp, const CoefLayout& L, uint64_t all, int p, double gs) {
  std::vector<PlanItem> v;
  for (size_t i = sp.ops.size(); i-- > 0;) {
    const SchedOp& o = sp.ops[i];
    if (o.type == 0)
      v.push_back(rx_item(o.bit, {ItemOp{OP_GRADX, 0, 0, 1 + p + o.layer, 1.0},
                                  ItemOp{OP_RX, OPF_LAM, L.at(o.layer, L.rx_dag), -1, 0}}));
    else
      v.push_back(global_item(all, {ItemOp{OP_GRADCOST, 0, 0, 1 + o.layer, 2.0 * gs},
                                    ItemOp{OP_COST, OPF_LAM, L.at(o.layer, L.lut_dag), -1, 0}}));
  }
  return v;
}

uint32_t cut_flag(const SchedPass& sp) {
  for (const auto& o : sp.ops)
    if (o.type == 1) return PF_NEED_CUT;
  return 0;
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
    int a = edges[2 * e], b = edges[2 * e + 1];
    QS_CHECK(a >= 0 && a < n_qubits && b >= 0 && b < n_qubits && a != b, "edge endpoint out of range or a self-loop");
    es.push_back({std::min(a, b), std::max(a, b)});
  }
  std::vector<std::pair<int, int>> sorted = es;
  std::sort(sorted.begin(), sorted.end());
  QS_CHECK(std::adjacent_find(sorted.begin(), sorted.end()) == sorted.end(), "repeated edge");

  qs_qaoa* q = new qs_qaoa;
  q->n = n_qubits;
  q->ne = std::max(n_qubits, kRegBits);
  q->p = p;
  q->n_edges = n_edges;
  q->gs = gamma_scale;
  q->dt = dtype;
  q->edges.assign(edges, edges + 2 * n_edges);
  int mm = (opts && opts->tile_bits) ? opts->tile_bits : (dtype == QS_C64 ? 12 : 11);
  mm = std::max(kRegBits, std::min({mm, max_tile_bits(dtype), q->ne}));
  int cc = (opts && opts->low_bits) ? opts->low_bits : 0;
  if (cc == 0) {
    // fewest passes; ties go to more contiguous bits
    int best = 1 << 30;
    for (int c = 2; c <= std::min(6, mm); ++c) {
      const int np = (int)make_schedule(q->ne, p, mm, c).size();
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

  auto fail = [&](qs_status s) {
    qs_qaoa_destroy(q);
    return s;
  };
  const uint64_t N = 1ull << q->ne;
  cudaError_t e = cudaMalloc(&q->d_cut, N);
  if (e != cudaSuccess) return fail(cuda_fail(e, "cudaMalloc(cut values)"));
  e = cudaMalloc(&q->d_edges, sizeof(int) * 2 * n_edges);
  if (e != cudaSuccess) return fail(cuda_fail(e, "cudaMalloc(edges)"));
  e = cudaMemcpy(q->d_edges, edges, sizeof(int) * 2 * n_edges, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fail(cuda_fail(e, "cudaMemcpy(edges)"));
  qs_status s = launch_cut_values(q->d_cut, q->ne, q->d_edges, n_edges, nullptr);
  if (s != QS_OK) return fail(s);

  const CoefLayout L = layout_for(n_edges);
  q->n_coef = L.per_layer * p;
  e = cudaMalloc(&q->d_coef, (size_t)q->n_coef * 16);
  if (e != cudaSuccess) return fail(cuda_fail(e, "cudaMalloc(coefficients)"));

  const std::vector<SchedPass> sched = make_schedule(q->ne, p, mm, cc);
  const int K = (int)sched.size();
  const uint64_t all = (1ull << q->ne) - 1;
  PlanParams pp{q->ne, mm, cc, dtype};

  // gradient plan: forward passes 0..K-2, turnaround K-1, reverse K-2..0
  for (int i = 0; i < K - 1; ++i) {
    const uint32_t fl = (i == 0 ? PF_GEN_PLUS : PF_LOAD_PSI) | PF_STORE_PSI | cut_flag(sched[i]);
    s = plan_single_pass(fwd_items(sched[i], L, all), sched[i].S, pp, fl, &q->gplan, &q->gslots);
    if (s != QS_OK) return fail(s);
  }
  {
    std::vector<PlanItem> items = fwd_items(sched[K - 1], L, all);
    items.push_back(global_item(all, {ItemOp{OP_ENERGY, 0, 0, 0, 1.0}}));
    std::vector<PlanItem> r = rev_items(sched[K - 1], L, all, p, gamma_scale);
    items.insert(items.end(), r.begin(), r.end());
    const uint32_t fl = (K == 1 ? PF_GEN_PLUS : PF_LOAD_PSI) | PF_STORE_LAM | PF_NEED_CUT;
    s = plan_single_pass(items, sched[K - 1].S, pp, fl, &q->gplan, &q->gslots);
    if (s != QS_OK) return fail(s);
  }
  for (int i = K - 2; i >= 0; --i) {
    const uint32_t st = i > 0 ? (PF_STORE_PSI | PF_STORE_LAM) : 0;
    const uint32_t fl = PF_LOAD_PSI | PF_LOAD_LAM | st | cut_flag(sched[i]);
    s = plan_single_pass(rev_items(sched[i], L, all, p, gamma_scale), sched[i].S, pp, fl, &q->gplan, &q->gslots);
    if (s != QS_OK) return fail(s);
  }
  q->n_fwd = K - 1;
  q->rev_passes = K - 1;
  // energy plan: forward passes with the energy op appended to the last
  for (int i = 0; i < K; ++i) {
    std::vector<PlanItem> items = fwd_items(sched[i], L, all);
    uint32_t fl = (i == 0 ? PF_GEN_PLUS : PF_LOAD_PSI) | PF_STORE_PSI | cut_flag(sched[i]);
    if (i == K - 1) {
      items.push_back(global_item(all, {ItemOp{OP_ENERGY, 0, 0, 0, 1.0}}));
      fl |= PF_NEED_CUT;
    }
    s = plan_single_pass(items, sched[i].S, pp, fl, &q->eplan, &q->eslots);
    if (s != QS_OK) return fail(s);
  }
  s = q->gplan.upload(nullptr);
  if (s == QS_OK) s = q->eplan.upload(nullptr);
  if (s == QS_OK) s = build_csr(q->gslots, 1 + 2 * p, &q->g_row, &q->g_sidx, &q->g_w, nullptr);
  if (s == QS_OK) s = build_csr(q->eslots, 1, &q->e_row, &q->e_sidx, &q->e_w, nullptr);
  if (s != QS_OK) return fail(s);
  const uint64_t n_tiles = 1ull << (q->ne - mm);
  q->grid1 = tile_grid_size(dtype, mm, 1, (int)std::min<uint64_t>(n_tiles, 1u << 30));
  q->grid2 = tile_grid_size(dtype, mm, 2, (int)std::min<uint64_t>(n_tiles, 1u << 30));
  // planned HBM traffic of one gradient evaluation (state reads + writes and cut reads)
  const double S = (double)amp_bytes(dtype) * (double)N;
  double bytes = 0;
  for (const auto& pass : q->gplan.passes) {
    const uint32_t f = pass.hdr.flags;
    bytes += S * (((f & PF_LOAD_PSI) ? 1 : 0) + ((f & PF_LOAD_LAM) ? 1 : 0) + ((f & PF_STORE_PSI) ? 1 : 0) +
                  ((f & PF_STORE_LAM) ? 1 : 0));
    if (f & PF_NEED_CUT) bytes += (double)N;
  }
  q->bytes_per_eval = bytes;
  *out = q;
  return QS_OK;
}

qs_status qs_qaoa_destroy(qs_qaoa* q) {
  if (!q) return QS_OK;
  cudaDeviceSynchronize();
  q->gplan.free_device();
  q->eplan.free_device();
  if (q->d_cut) cudaFree(q->d_cut);
  if (q->d_edges) cudaFree(q->d_edges);
  if (q->d_coef) cudaFree(q->d_coef);
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

qs_status qaoa_energy(qs_qaoa* q, qs_state* psi, const double* gamma, const double* beta, double* energy) {
  QS_TRY(qaoa_check(q, psi, gamma, beta));
  cudaStream_t st = psi->st;
  QS_TRY(fill_qaoa_coef(q, gamma, beta));
  QS_TRY(upload_table(q->host_coef, q->dt, q->d_coef, st, psi->host_out));
  const int n_slots = (int)q->eslots.out.size();
  const size_t part = (size_t)std::max(n_slots, 1) * q->grid2;
  QS_TRY(ensure_scratch(psi, part + n_slots + 8));
  double* d_part = psi->scratch;
  double* d_slot = d_part + part;
  double* d_out = d_slot + n_slots;
  QS_TRY(run_passes(q->eplan, 0, (int)q->eplan.passes.size(), q->dt, psi->ptr, nullptr, q->d_coef, q->d_cut, d_part,
                    q->ne, q->n_edges, q->grid1, q->grid2, st));
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
  QS_TRY(fill_qaoa_coef(q, gamma, beta));
  QS_TRY(upload_table(q->host_coef, q->dt, q->d_coef, st, psi->host_out));
  const int n_slots = (int)q->gslots.out.size();
  const int n_out = 1 + 2 * q->p;
  const size_t part = (size_t)std::max(n_slots, 1) * q->grid2;
  QS_TRY(ensure_scratch(psi, part + n_slots + n_out + 8));
  double* d_part = psi->scratch;
  double* d_slot = d_part + part;
  double* d_out = d_slot + n_slots;
  QS_TRY(run_passes(q->gplan, 0, (int)q->gplan.passes.size(), q->dt, psi->ptr, lam->ptr, q->d_coef, q->d_cut, d_part,
                    q->ne, q->n_edges, q->grid1, q->grid2, st));
  QS_TRY(launch_reduce_slots(d_part, n_slots, q->grid2, nullptr, d_slot, st));
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

}  // extern "C"
