// Host side of the Monte-Carlo trajectory engine (§3.3: the state-vector
// simulator treats channels by sampling, and the average over sampled runs is
// the noisy result): circuit and channel tables, argument checks, launches of
// the shared-memory trajectory kernel, and, for states too large for one CTA's
// shared memory, the loop that runs trajectories one by one on the fused tile
// passes.
#include <algorithm>
#include <cmath>
#include <vector>

#include "batch.h"
#include "handles.h"

using namespace qs;

// A segment of the large-state path: the gates up to a damping / Kraus site (or
// the end), planned once as a fused circuit, with a one-qubit MATRIX gate at
// each Pauli / depolarizing site inside it whose entries are set to the sampled
// Pauli before every trajectory (the plan depends on the gate's kind, not its
// entries, so it stays valid).
struct TrajSeg {
  qs_circuit* c = nullptr;
  int site_after = -1;               // the state-dependent site that ends it; -1: the end
  std::vector<int> ph_gate, ph_site;  // placeholder gate index in c, and its site
};

struct qs_traj {
  int n = 0;
  qs_dtype dt = QS_C64;
  cudaStream_t st = nullptr;
  std::vector<BGate> gates;
  std::vector<BChannel> ch;
  int n_params = 0;
  bool all_fixed = true;
  bool dirty = true;
  BGate* d_gates = nullptr;
  BChannel* d_ch = nullptr;
  size_t cap_gates = 0, cap_ch = 0;
  double* d_params = nullptr;
  size_t cap_params = 0;
  double* d_energy = nullptr;
  size_t cap_energy = 0;
  double* d_grad = nullptr;
  size_t cap_grad = 0;
  double* d_gmean = nullptr;
  size_t cap_gmean = 0;
  uint8_t* d_choice = nullptr;
  size_t cap_choice = 0;
  int* d_queue = nullptr;
  // states too large for one CTA's shared memory: fused tile passes in HBM
  std::vector<TrajSeg> segs;
  bool segs_valid = false;
  qs_state* lpsi = nullptr;
  qs_state* llam = nullptr;
};

namespace {

template <class P>
qs_status ensure(P** p, size_t* cap, size_t count) {
  count = std::max<size_t>(count, 1);
  if (*cap >= count) return QS_OK;
  if (*p) QS_CUDA(cudaFree(*p));
  *p = nullptr;
  QS_CUDA(cudaMalloc((void**)p, count * sizeof(P)));
  *cap = count;
  return QS_OK;
}

qs_status upload(qs_traj* t) {
  if (!t->dirty) return QS_OK;
  QS_TRY(ensure(&t->d_gates, &t->cap_gates, t->gates.size()));
  QS_TRY(ensure(&t->d_ch, &t->cap_ch, t->ch.size()));
  if (!t->gates.empty())
    QS_CUDA(cudaMemcpyAsync(t->d_gates, t->gates.data(), t->gates.size() * sizeof(BGate), cudaMemcpyHostToDevice,
                            t->st));
  if (!t->ch.empty())
    QS_CUDA(cudaMemcpyAsync(t->d_ch, t->ch.data(), t->ch.size() * sizeof(BChannel), cudaMemcpyHostToDevice, t->st));
  if (!t->d_queue) QS_CUDA(cudaMalloc(&t->d_queue, sizeof(int)));
  t->dirty = false;
  return QS_OK;
}

void set_op(BChannel& C, int k, double a_re, double a_im, double b_re, double b_im, double c_re, double c_im,
            double d_re, double d_im) {
  const double v[8] = {a_re, a_im, b_re, b_im, c_re, c_im, d_re, d_im};
  for (int e = 0; e < 8; ++e) C.K[k][e] = v[e];
}

// ------------------------------------------------------------------ large states

// The uniform of site s of trajectory t, counter c = t * n_sites + s: the
// published splitmix64 finaliser (Steele, Lea & Flood 2014) of
// seed + (c + 1) * 0x9E3779B97F4A7C15, top 53 bits (the same numbers the
// shared-memory engine draws).
double traj_uniform_host(uint64_t seed, uint64_t c) {
  uint64_t z = seed + c * 0x9E3779B97F4A7C15ull + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (double)(z >> 11) * 0x1.0p-53;
}

// The smallest branch whose running weight sum exceeds u * total, else the last
// branch with a positive weight.
int choose_branch(const double* w, int nk, double u) {
  double total = 0.0;
  for (int k = 0; k < nk; ++k) total += w[k];
  const double thr = u * total;
  int c = -1;
  double cum = 0.0;
  for (int k = 0; k < nk; ++k) {
    cum += w[k];
    if (c < 0 && cum > thr) c = k;
  }
  if (c < 0)
    for (int k = 0; k < nk; ++k)
      if (w[k] > 0) c = k;
  return c < 0 ? 0 : c;
}

void free_segs(qs_traj* t) {
  for (auto& S : t->segs) qs_circuit_destroy(S.c);
  t->segs.clear();
  t->segs_valid = false;
}

qs_status build_segs(qs_traj* t) {
  if (t->segs_valid) return QS_OK;
  free_segs(t);
  auto open = [&]() {
    t->segs.emplace_back();
    return qs_circuit_create(t->n, &t->segs.back().c);
  };
  QS_TRY(open());
  static const double kEye[8] = {1, 0, 0, 0, 0, 0, 1, 0};
  for (const BGate& g : t->gates) {
    if (g.kind == kGateChannel) {
      const BChannel& C = t->ch[g.param];
      if (C.fixed) {
        TrajSeg& S = t->segs.back();
        const int q = C.qubit;
        QS_TRY(qs_circuit_add(S.c, QS_GATE_MATRIX, &q, 1, nullptr, 0, -1, 1.0, 0.0, kEye));
        S.ph_gate.push_back((int)S.c->gates.size() - 1);
        S.ph_site.push_back(g.param);
      } else {
        t->segs.back().site_after = g.param;
        QS_TRY(open());
      }
      continue;
    }
    const int tg[2] = {g.t0, g.t1};
    int ctr[64], nc = 0;
    for (int q = 0; q < t->n; ++q)
      if ((g.cmask >> q) & 1ull) ctr[nc++] = q;
    QS_TRY(qs_circuit_add(t->segs.back().c, g.kind, tg, g.nt, ctr, nc, g.param, g.coef, g.constant, nullptr));
  }
  for (auto& S : t->segs) QS_TRY(qs_circuit_finalize(S.c, t->dt, nullptr));
  t->segs_valid = true;
  return QS_OK;
}

// Branch weights of a damping / Kraus site on the current state:
// ||K psi||^2 = sum_r sum_ab K_ra conj(K_rb) rho_ab, rho the site qubit's
// reduced density matrix (FP64 sums on the device).
qs_status site_weights(qs_traj* t, const BChannel& C, double* w) {
  qs_state* s = t->lpsi;
  const int grid = ham_grid_size(s->ne);
  QS_TRY(ensure_scratch(s, 4 * (size_t)grid + 4));
  double* part = s->scratch;
  double* out = part + 4 * (size_t)grid;
  QS_TRY(launch_qubit_rdm(s->dt, s->ptr, s->ne, C.qubit, part, grid, s->st));
  QS_TRY(launch_reduce_slots(part, 4, grid, nullptr, out, s->st));
  double r[4];
  QS_CUDA(cudaMemcpyAsync(r, out, sizeof(r), cudaMemcpyDeviceToHost, s->st));
  QS_CUDA(cudaStreamSynchronize(s->st));
  // rho_ab as (re, im): rho00, rho01, rho10, rho11
  const double rho[4][2] = {{r[0], 0.0}, {r[2], r[3]}, {r[2], -r[3]}, {r[1], 0.0}};
  for (int k = 0; k < C.n_kraus; ++k) {
    double acc = 0.0;
    for (int row = 0; row < 2; ++row)
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
          const double kr = C.K[k][2 * (2 * row + a)], ki = C.K[k][2 * (2 * row + a) + 1];
          const double lr = C.K[k][2 * (2 * row + b)], li = -C.K[k][2 * (2 * row + b) + 1];  // conj(K_rb)
          const double pr = kr * lr - ki * li, pi = kr * li + ki * lr;
          acc += pr * rho[2 * a + b][0] - pi * rho[2 * a + b][1];
        }
    w[k] = acc;
  }
  return QS_OK;
}

// Trajectories on the fused tile engine, one after another (host results):
// the Pauli sites' branches are drawn up front and set into their placeholder
// gates; at a damping / Kraus site the weights come from site_weights and the
// state is replaced by K_c psi / sqrt(w_c) (a one-qubit gate kernel).  With
// gradients (Pauli / depolarizing sites only: one segment, unitary) each
// trajectory is one adjoint evaluation of its circuit.
qs_status run_large(qs_traj* t, const qs_ham* h, const double* params, uint64_t seed, long long first, int n_traj,
                    double* energies, double* grad_mean, unsigned char* choices, qs_state* state_out) {
  QS_TRY(build_segs(t));
  if (!t->lpsi) QS_TRY(qs_state_create(t->n, t->dt, nullptr, 0, t->st, &t->lpsi));
  if (grad_mean && !t->llam) QS_TRY(qs_state_create(t->n, t->dt, nullptr, 0, t->st, &t->llam));
  const int S = (int)t->ch.size(), np = t->n_params;
  std::vector<double> g((size_t)std::max(np, 1)), acc((size_t)std::max(np, 1), 0.0);
  std::vector<int> pick((size_t)std::max(S, 1), 0);
  for (int i = 0; i < n_traj; ++i) {
    const uint64_t tr = (uint64_t)(first + i);
    for (auto& seg : t->segs)
      for (size_t k = 0; k < seg.ph_gate.size(); ++k) {
        const int site = seg.ph_site[k];
        const BChannel& C = t->ch[site];
        const int c = choose_branch(C.w, C.n_kraus, traj_uniform_host(seed, tr * (uint64_t)S + (uint64_t)site));
        pick[site] = c;
        seg.c->gates[seg.ph_gate[k]].matrix.assign(C.K[c], C.K[c] + 8);
      }
    double e = 0.0;
    QS_TRY(qs_state_set_basis(t->lpsi, 0));
    if (grad_mean) {
      QS_TRY(qs_expectation_with_grad(t->lpsi, t->llam, t->segs[0].c, h, params, np, &e, g.data()));
      for (int p = 0; p < np; ++p) acc[p] += g[p];
    } else {
      for (auto& seg : t->segs) {
        if (!seg.c->gates.empty()) QS_TRY(qs_apply_circuit(t->lpsi, seg.c, params, np));
        if (seg.site_after < 0) continue;
        const int site = seg.site_after;
        const BChannel& C = t->ch[site];
        double w[kTrajMaxKraus] = {0, 0, 0, 0};
        QS_TRY(site_weights(t, C, w));
        const int c = choose_branch(w, C.n_kraus, traj_uniform_host(seed, tr * (uint64_t)S + (uint64_t)site));
        pick[site] = c;
        const double sc = w[c] > 0 ? 1.0 / std::sqrt(w[c]) : 0.0;
        double M[8];
        for (int e2 = 0; e2 < 8; ++e2) M[e2] = C.K[c][e2] * sc;
        const int q = C.qubit;
        QS_TRY(launch_gate_dense(t->dt, t->lpsi->ptr, t->lpsi->ne, 1, &q, 0, M, t->lpsi->st));
      }
      if (h) QS_TRY(qs_expectation(t->lpsi, h, &e));
    }
    if (energies) energies[i] = e;
    if (choices)
      for (int site = 0; site < S; ++site) choices[(size_t)i * S + site] = (unsigned char)pick[site];
  }
  if (grad_mean)
    for (int p = 0; p < np; ++p) grad_mean[p] = acc[p] / n_traj;
  if (state_out) {  // the copy runs on the output's stream: the trajectory's work first
    QS_CUDA(cudaStreamSynchronize(t->lpsi->st));
    QS_TRY(qs_state_copy(state_out, t->lpsi));
    QS_CUDA(cudaStreamSynchronize(state_out->st));
  }
  return QS_OK;
}

bool use_large(const qs_traj* t, bool grad) {
  return traj_grid_size(t->dt, grad, t->n, (int)t->gates.size(), t->n_params) <= 0;
}

// Launch n_traj trajectories starting at global index `first`.
qs_status run(qs_traj* t, const qs_ham* h, const double* d_params, uint64_t seed, long long first, int n_traj,
              double* d_energy, bool grad, double* d_gmean, uint8_t* d_choice, void* state_out) {
  QS_TRY(upload(t));
  int grid = traj_grid_size(t->dt, grad, t->n, (int)t->gates.size(), t->n_params);
  QS_CHECK(grid > 0, grad ? "too many qubits, gates or parameters for shared-memory trajectories with gradients"
                          : "too many qubits or gates for shared-memory trajectories");
  grid = std::min(grid, n_traj);
  if (grad) QS_TRY(ensure(&t->d_grad, &t->cap_grad, (size_t)n_traj * std::max(t->n_params, 1)));
  QS_CUDA(cudaMemsetAsync(t->d_queue, 0, sizeof(int), t->st));
  TrajArgs a{};
  a.gates = t->d_gates;
  a.ch = t->d_ch;
  a.groups = h ? h->d_groups : nullptr;
  a.terms = h ? h->d_terms : nullptr;
  a.n_groups = h ? h->n_groups : 0;
  a.params = d_params;
  a.energy = d_energy;
  a.grad = grad ? t->d_grad : nullptr;
  a.choice = d_choice;
  a.state_out = state_out;
  a.queue = t->d_queue;
  a.seed = seed;
  a.first = first;
  a.n_traj = n_traj;
  a.n = t->n;
  a.n_gates = (int)t->gates.size();
  a.n_sites = (int)t->ch.size();
  a.n_params = t->n_params;
  QS_TRY(launch_traj(t->dt, grad, a, grid, t->st));
  if (grad) QS_TRY(launch_row_mean(t->d_grad, n_traj, t->n_params, d_gmean, t->st));
  return QS_OK;
}

qs_status check_run(const qs_traj* t, const qs_ham* h, int n_traj, long long first, bool grad) {
  QS_CHECK(t != nullptr, "null trajectory engine");
  QS_CHECK(h == nullptr || h->n == t->n, "Hamiltonian qubit count differs from the circuit's");
  QS_CHECK(n_traj >= 1 && n_traj <= (1 << 24), "n_traj must be in 1..2^24");
  QS_CHECK(first >= 0, "first trajectory index must be >= 0");
  QS_CHECK(!grad || t->all_fixed, "gradients need Pauli or depolarizing channels only (unitary branches)");
  return QS_OK;
}

}  // namespace

extern "C" {

qs_status qs_traj_create(int n_qubits, qs_dtype dtype, void* cuda_stream, qs_traj** out) {
  QS_CHECK(out != nullptr, "out is null");
  QS_CHECK(n_qubits >= 1 && n_qubits <= kMaxQubits, "n_qubits must be in 1..34");
  QS_CHECK(dtype == QS_C64 || dtype == QS_C128, "invalid dtype");
  qs_traj* t = new qs_traj;
  t->n = n_qubits;
  t->dt = dtype;
  t->st = (cudaStream_t)cuda_stream;
  *out = t;
  return QS_OK;
}

qs_status qs_traj_destroy(qs_traj* t) {
  if (!t) return QS_OK;
  cudaStreamSynchronize(t->st);
  cudaFree(t->d_gates);
  cudaFree(t->d_ch);
  cudaFree(t->d_params);
  cudaFree(t->d_energy);
  cudaFree(t->d_grad);
  cudaFree(t->d_gmean);
  cudaFree(t->d_choice);
  cudaFree(t->d_queue);
  free_segs(t);
  qs_state_destroy(t->lpsi);
  qs_state_destroy(t->llam);
  delete t;
  return QS_OK;
}

qs_status qs_traj_add_gate(qs_traj* t, int kind, const int* targets, int n_t, const int* ctrls, int n_c,
                           int param_idx, double coef, double constant) {
  QS_CHECK(t != nullptr, "null trajectory engine");
  const bool two = kind == QS_GATE_SWAP || kind == QS_GATE_RXX || kind == QS_GATE_RYY || kind == QS_GATE_RZZ;
  QS_CHECK((kind >= QS_GATE_I && kind <= QS_GATE_SWAP) || (kind >= QS_GATE_RX && kind <= QS_GATE_RZZ),
           "unsupported gate kind (MATRIX gates are not supported in trajectories)");
  QS_CHECK(targets != nullptr && n_t == (two ? 2 : 1), "wrong number of targets for this gate kind");
  uint64_t used = 0;
  for (int i = 0; i < n_t; ++i) {
    QS_CHECK(targets[i] >= 0 && targets[i] < t->n, "target qubit out of range");
    QS_CHECK(!((used >> targets[i]) & 1), "duplicate target");
    used |= 1ull << targets[i];
  }
  uint64_t cm = 0;
  QS_CHECK(n_c >= 0 && (n_c == 0 || ctrls != nullptr), "bad controls");
  for (int i = 0; i < n_c; ++i) {
    QS_CHECK(ctrls[i] >= 0 && ctrls[i] < t->n && !((used >> ctrls[i]) & 1) && !((cm >> ctrls[i]) & 1),
             "control out of range, repeated or a target");
    cm |= 1ull << ctrls[i];
  }
  QS_CHECK(param_idx >= -1 && param_idx < (1 << 20), "param index out of range");
  QS_CHECK(param_idx == -1 || kind >= QS_GATE_RX, "only RX/RY/RZ/PS/RXX/RYY/RZZ take a parameter");
  QS_CHECK(std::isfinite(coef) && std::isfinite(constant), "non-finite angle binding");
  BGate g{};
  g.kind = (uint8_t)kind;
  g.nt = (uint8_t)n_t;
  g.t0 = (uint8_t)targets[0];
  g.t1 = (uint8_t)(two ? targets[1] : targets[0]);
  g.param = param_idx;
  g.cmask = cm;
  g.coef = coef;
  g.constant = constant;
  t->gates.push_back(g);
  t->n_params = std::max(t->n_params, param_idx + 1);
  t->dirty = true;
  t->segs_valid = false;
  return QS_OK;
}

qs_status qs_traj_add_channel(qs_traj* t, int kind, int qubit, const double* p, int n_kraus, const double* kraus) {
  QS_CHECK(t != nullptr, "null trajectory engine");
  QS_CHECK(qubit >= 0 && qubit < t->n, "qubit out of range");
  QS_CHECK((int)t->ch.size() < kTrajMaxSites, "too many channel sites (at most 4096)");
  BChannel C{};
  C.qubit = qubit;
  if (kind == QS_CH_PAULI || kind == QS_CH_DEPOLARIZING) {
    QS_CHECK(p != nullptr, "null probabilities");
    C.fixed = 1;
    C.n_kraus = 4;
    if (kind == QS_CH_PAULI) {
      const double px = p[0], py = p[1], pz = p[2];
      QS_CHECK(px >= 0 && py >= 0 && pz >= 0 && px + py + pz <= 1.0 + 1e-12, "probabilities must be >= 0, sum <= 1");
      C.w[0] = std::max(0.0, 1.0 - px - py - pz);
      C.w[1] = px;
      C.w[2] = py;
      C.w[3] = pz;
    } else {
      QS_CHECK(p[0] >= 0.0 && p[0] <= 1.0, "probability outside [0, 1]");
      const double q = p[0] / 4.0;
      C.w[0] = 1.0 - q - q - q;
      C.w[1] = C.w[2] = C.w[3] = q;
    }
    set_op(C, 0, 1, 0, 0, 0, 0, 0, 1, 0);    // I
    set_op(C, 1, 0, 0, 1, 0, 1, 0, 0, 0);    // X
    set_op(C, 2, 0, 0, 0, -1, 0, 1, 0, 0);   // Y
    set_op(C, 3, 1, 0, 0, 0, 0, 0, -1, 0);   // Z
  } else if (kind == QS_CH_AMPLITUDE_DAMPING || kind == QS_CH_PHASE_DAMPING) {
    QS_CHECK(p != nullptr && p[0] >= 0.0 && p[0] <= 1.0, "gamma outside [0, 1]");
    const double g = p[0];
    C.n_kraus = 2;
    set_op(C, 0, 1, 0, 0, 0, 0, 0, std::sqrt(1 - g), 0);
    if (kind == QS_CH_AMPLITUDE_DAMPING)
      set_op(C, 1, 0, 0, std::sqrt(g), 0, 0, 0, 0, 0);
    else
      set_op(C, 1, 0, 0, 0, 0, 0, 0, std::sqrt(g), 0);
  } else if (kind == QS_CH_KRAUS) {
    QS_CHECK(n_kraus >= 1 && n_kraus <= kTrajMaxKraus && kraus != nullptr, "1..4 Kraus operators in trajectories");
    C.n_kraus = n_kraus;
    double s[8] = {0, 0, 0, 0, 0, 0, 0, 0};  // sum K^dag K, (re, im) row-major
    for (int k = 0; k < n_kraus; ++k) {
      for (int e = 0; e < 8; ++e) {
        QS_CHECK(std::isfinite(kraus[8 * k + e]), "non-finite Kraus entry");
        C.K[k][e] = kraus[8 * k + e];
      }
      for (int r = 0; r < 2; ++r)
        for (int c = 0; c < 2; ++c)
          for (int m = 0; m < 2; ++m) {
            const double ar = C.K[k][2 * (2 * m + r)], ai = -C.K[k][2 * (2 * m + r) + 1];  // conj(K[m][r])
            const double br = C.K[k][2 * (2 * m + c)], bi = C.K[k][2 * (2 * m + c) + 1];
            s[2 * (2 * r + c)] += ar * br - ai * bi;
            s[2 * (2 * r + c) + 1] += ar * bi + ai * br;
          }
    }
    QS_CHECK(std::fabs(s[0] - 1) < 1e-9 && std::fabs(s[1]) < 1e-9 && std::fabs(s[2]) < 1e-9 &&
                 std::fabs(s[3]) < 1e-9 && std::fabs(s[4]) < 1e-9 && std::fabs(s[5]) < 1e-9 &&
                 std::fabs(s[6] - 1) < 1e-9 && std::fabs(s[7]) < 1e-9,
             "Kraus operators are not complete (sum K^dag K != I)");
  } else {
    set_error("unknown channel kind");
    return QS_ERR_INVALID_ARG;
  }
  if (!C.fixed) t->all_fixed = false;
  BGate g{};
  g.kind = (uint8_t)kGateChannel;
  g.nt = 1;
  g.t0 = g.t1 = (uint8_t)qubit;
  g.param = (int)t->ch.size();
  t->gates.push_back(g);
  t->ch.push_back(C);
  t->dirty = true;
  t->segs_valid = false;
  return QS_OK;
}

qs_status qs_traj_info(const qs_traj* t, int* n_sites, int* n_params, int* grid_energy, int* grid_grad) {
  QS_CHECK(t != nullptr, "null trajectory engine");
  if (n_sites) *n_sites = (int)t->ch.size();
  if (n_params) *n_params = t->n_params;
  if (grid_energy) *grid_energy = traj_grid_size(t->dt, false, t->n, (int)t->gates.size(), t->n_params);
  if (grid_grad) *grid_grad = traj_grid_size(t->dt, true, t->n, (int)t->gates.size(), t->n_params);
  return QS_OK;
}

qs_status qs_traj_run(qs_traj* t, const qs_ham* h, const double* params, int n_params, uint64_t seed,
                      long long first, int n_traj, double* energies, double* grad_mean, unsigned char* choices) {
  const bool grad = grad_mean != nullptr;
  QS_TRY(check_run(t, h, n_traj, first, grad));
  QS_CHECK(h != nullptr && energies != nullptr, "null Hamiltonian or energies");
  QS_CHECK(n_params == t->n_params && (n_params == 0 || params != nullptr), "n_params differs from the circuit's");
  for (int i = 0; i < n_params; ++i) QS_CHECK(std::isfinite(params[i]), "non-finite parameter");
  if (use_large(t, grad)) return run_large(t, h, params, seed, first, n_traj, energies, grad_mean, choices, nullptr);
  QS_TRY(ensure(&t->d_params, &t->cap_params, (size_t)n_params));
  QS_TRY(ensure(&t->d_energy, &t->cap_energy, (size_t)n_traj));
  if (grad) QS_TRY(ensure(&t->d_gmean, &t->cap_gmean, (size_t)n_params));
  if (choices) QS_TRY(ensure(&t->d_choice, &t->cap_choice, (size_t)n_traj * std::max<size_t>(t->ch.size(), 1)));
  if (n_params)
    QS_CUDA(cudaMemcpyAsync(t->d_params, params, n_params * sizeof(double), cudaMemcpyHostToDevice, t->st));
  QS_TRY(run(t, h, t->d_params, seed, first, n_traj, t->d_energy, grad, t->d_gmean, choices ? t->d_choice : nullptr,
             nullptr));
  QS_CUDA(cudaMemcpyAsync(energies, t->d_energy, n_traj * sizeof(double), cudaMemcpyDeviceToHost, t->st));
  if (grad && n_params)
    QS_CUDA(cudaMemcpyAsync(grad_mean, t->d_gmean, n_params * sizeof(double), cudaMemcpyDeviceToHost, t->st));
  if (choices && !t->ch.empty())
    QS_CUDA(cudaMemcpyAsync(choices, t->d_choice, (size_t)n_traj * t->ch.size(), cudaMemcpyDeviceToHost, t->st));
  QS_CUDA(cudaStreamSynchronize(t->st));
  return QS_OK;
}

qs_status qs_traj_run_device(qs_traj* t, const qs_ham* h, const double* d_params, uint64_t seed, long long first,
                             int n_traj, double* d_energies, double* d_grad_mean) {
  const bool grad = d_grad_mean != nullptr;
  QS_TRY(check_run(t, h, n_traj, first, grad));
  QS_CHECK(h != nullptr && d_energies != nullptr, "null Hamiltonian or energies");
  QS_CHECK(t->n_params == 0 || d_params != nullptr, "null parameters");
  if (use_large(t, grad)) {  // host loop over trajectories; results copied to the device buffers
    std::vector<double> p((size_t)std::max(t->n_params, 1)), e((size_t)n_traj), gm((size_t)std::max(t->n_params, 1));
    if (t->n_params)
      QS_CUDA(cudaMemcpyAsync(p.data(), d_params, t->n_params * sizeof(double), cudaMemcpyDeviceToHost, t->st));
    QS_CUDA(cudaStreamSynchronize(t->st));
    QS_TRY(run_large(t, h, p.data(), seed, first, n_traj, e.data(), grad ? gm.data() : nullptr, nullptr, nullptr));
    QS_CUDA(cudaMemcpyAsync(d_energies, e.data(), n_traj * sizeof(double), cudaMemcpyHostToDevice, t->st));
    if (grad && t->n_params)
      QS_CUDA(cudaMemcpyAsync(d_grad_mean, gm.data(), t->n_params * sizeof(double), cudaMemcpyHostToDevice, t->st));
    QS_CUDA(cudaStreamSynchronize(t->st));
    return QS_OK;
  }
  return run(t, h, d_params, seed, first, n_traj, d_energies, grad, d_grad_mean, nullptr, nullptr);
}

qs_status qs_traj_state(qs_traj* t, const double* params, int n_params, uint64_t seed, long long traj,
                        qs_state* out) {
  QS_TRY(check_run(t, nullptr, 1, traj, false));
  QS_TRY(check_state(out));
  QS_CHECK(out->n == t->n && out->dt == t->dt, "state n/dtype differs from the trajectory engine");
  QS_CHECK(n_params == t->n_params && (n_params == 0 || params != nullptr), "n_params differs from the circuit's");
  if (use_large(t, false)) {
    QS_CUDA(cudaStreamSynchronize(out->st));
    return run_large(t, nullptr, params, seed, traj, 1, nullptr, nullptr, nullptr, out);
  }
  QS_TRY(ensure(&t->d_params, &t->cap_params, (size_t)n_params));
  QS_TRY(ensure(&t->d_energy, &t->cap_energy, 1));
  if (n_params)
    QS_CUDA(cudaMemcpyAsync(t->d_params, params, n_params * sizeof(double), cudaMemcpyHostToDevice, t->st));
  QS_CUDA(cudaStreamSynchronize(out->st));
  QS_CUDA(cudaMemsetAsync(out->ptr, 0, out->bytes, t->st));
  QS_TRY(run(t, nullptr, t->d_params, seed, traj, 1, t->d_energy, false, nullptr, nullptr, out->ptr));
  QS_CUDA(cudaStreamSynchronize(t->st));
  return QS_OK;
}

}  // extern "C"
