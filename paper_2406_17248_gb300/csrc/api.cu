// C ABI of the engine: handles, argument checks, gate matrices (FP64 host
// arithmetic, converted once per call), plan execution and result gathering.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "handles.h"
#include "t2gen.h"

using cd = std::complex<double>;

namespace qs {

static thread_local std::string g_last_error;

void set_error(const std::string& msg) { g_last_error = msg; }

qs_status cuda_fail(cudaError_t e, const char* what) {
  set_error(std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e));
  if (e == cudaErrorMemoryAllocation) return QS_ERR_OUT_OF_MEMORY;
  return QS_ERR_CUDA;
}

}  // namespace qs

using namespace qs;

// ============================================================================ helpers

namespace qs {

size_t amp_bytes(qs_dtype dt) { return dt == QS_C64 ? 8 : 16; }

bool valid_dtype(int dt) { return dt == QS_C64 || dt == QS_C128; }

qs_status ensure_scratch(qs_state* s, size_t ndoubles) {
  if (s->scratch_n >= ndoubles) return QS_OK;
  if (s->scratch) {
    QS_CUDA(cudaStreamSynchronize(s->st));
    cudaFree(s->scratch);
    s->scratch = nullptr;
    s->scratch_n = 0;
  }
  const size_t n = std::max<size_t>(ndoubles, 4096);
  QS_CUDA(cudaMalloc(&s->scratch, n * sizeof(double)));
  s->scratch_n = n;
  return QS_OK;
}

int gate_targets(int kind) {
  switch (kind) {
    case QS_GATE_SWAP:
    case QS_GATE_RXX:
    case QS_GATE_RYY:
    case QS_GATE_RZZ:
      return 2;
    default:
      return 1;
  }
}

bool gate_known(int k) {
  return (k >= QS_GATE_I && k <= QS_GATE_SWAP) || (k >= QS_GATE_RX && k <= QS_GATE_RZZ) || k == QS_GATE_MATRIX;
}

bool gate_parametric(int k) { return k >= QS_GATE_RX && k <= QS_GATE_RZZ; }

bool gate_diagonal(int k) {
  switch (k) {
    case QS_GATE_I:
    case QS_GATE_Z:
    case QS_GATE_S:
    case QS_GATE_SDG:
    case QS_GATE_T:
    case QS_GATE_TDG:
    case QS_GATE_RZ:
    case QS_GATE_PS:
    case QS_GATE_RZZ:
      return true;
    default:
      return false;
  }
}

// Gates whose unitary is real for every angle, and diagonal gates whose entries
// are all in {1, i, -1, -i}.
bool real_kind(int k) {
  return k == QS_GATE_I || k == QS_GATE_X || k == QS_GATE_Z || k == QS_GATE_H || k == QS_GATE_RY;
}
bool unit_diag_kind(int k) { return k == QS_GATE_I || k == QS_GATE_Z || k == QS_GATE_S || k == QS_GATE_SDG; }

// Unitary of one gate on its targets (basis index bit(t0) + 2 bit(t1)), row-major.
// Definitions: §2.3.2 fixed gates, §2.3.3 R_P(theta) = cos(theta/2) I - i sin(theta/2) P.
void gate_unitary(const HostGate& g, double th, cd* U, int* dim) {
  const double c = std::cos(0.5 * th), s = std::sin(0.5 * th);
  const cd I(0, 1);
  const double r2 = 0.70710678118654752440;
  int d = g.nt == 2 ? 4 : 2;
  if (g.kind == QS_GATE_MATRIX) {
    d = 1 << g.nt;
    for (int i = 0; i < d * d; ++i) U[i] = cd(g.matrix[2 * i], g.matrix[2 * i + 1]);
    *dim = d;
    return;
  }
  for (int i = 0; i < d * d; ++i) U[i] = 0;
  auto diag2 = [&](cd a, cd b) {
    U[0] = a;
    U[3] = b;
  };
  switch (g.kind) {
    case QS_GATE_I: diag2(1, 1); break;
    case QS_GATE_X: U[1] = U[2] = 1; break;
    case QS_GATE_Y: U[1] = -I; U[2] = I; break;
    case QS_GATE_Z: diag2(1, -1); break;
    case QS_GATE_H: U[0] = U[1] = U[2] = r2; U[3] = -r2; break;
    case QS_GATE_S: diag2(1, I); break;
    case QS_GATE_SDG: diag2(1, -I); break;
    case QS_GATE_T: diag2(1, cd(r2, r2)); break;
    case QS_GATE_TDG: diag2(1, cd(r2, -r2)); break;
    case QS_GATE_RX: U[0] = U[3] = c; U[1] = U[2] = -I * s; break;
    case QS_GATE_RY: U[0] = U[3] = c; U[1] = -s; U[2] = s; break;
    case QS_GATE_RZ: diag2(cd(c, -s), cd(c, s)); break;
    case QS_GATE_PS: diag2(1, cd(std::cos(th), std::sin(th))); break;
    case QS_GATE_SWAP: U[0] = U[6] = U[9] = U[15] = 1; break;
    case QS_GATE_RXX:  // c I - i s X(x)X : X(x)X maps b -> 3 - b
      for (int b = 0; b < 4; ++b) {
        U[b * 4 + b] = c;
        U[b * 4 + (3 - b)] = -I * s;
      }
      break;
    case QS_GATE_RYY: {  // Y(x)Y = [[0,0,0,-1],[0,0,1,0],[0,1,0,0],[-1,0,0,0]]
      for (int b = 0; b < 4; ++b) U[b * 4 + b] = c;
      U[0 * 4 + 3] = I * s;
      U[1 * 4 + 2] = -I * s;
      U[2 * 4 + 1] = -I * s;
      U[3 * 4 + 0] = I * s;
      break;
    }
    case QS_GATE_RZZ:
      U[0] = cd(c, -s);
      U[5] = cd(c, s);
      U[10] = cd(c, s);
      U[15] = cd(c, -s);
      break;
  }
  *dim = d;
}

// A = (dU/dtheta) U^dag for a parametric gate, from the same definitions.
void gate_generator(const HostGate& g, double th, cd* A, int* dim) {
  cd U[16], dU[16];
  int d = 0;
  gate_unitary(g, th, U, &d);
  // derivative of each matrix entry: entries are linear in cos(th/2), sin(th/2)
  // (or cos th, sin th for PS) -> differentiate analytically via a shifted copy:
  // d/dth [a cos(th/2) + b sin(th/2)] = 1/2 [a cos(th/2 + pi/2) + b sin(th/2 + pi/2)]
  if (g.kind == QS_GATE_PS) {
    for (int i = 0; i < d * d; ++i) dU[i] = 0;
    dU[3] = cd(-std::sin(th), std::cos(th));
  } else {
    cd Us[16];
    int d2;
    gate_unitary(g, th + M_PI, Us, &d2);  // cos/sin of (th + pi)/2 = th/2 + pi/2
    for (int i = 0; i < d * d; ++i) dU[i] = 0.5 * Us[i];
    // the identity part of Us at th + pi equals -sin(th/2) etc.; entries with no
    // th dependence do not occur in the rotation gates
  }
  for (int r = 0; r < d; ++r)
    for (int col = 0; col < d; ++col) {
      cd acc = 0;
      for (int k = 0; k < d; ++k) acc += dU[r * d + k] * std::conj(U[col * d + k]);
      A[r * d + col] = acc;
    }
  *dim = d;
}

int gate_class(const HostGate& g) {
  if (gate_diagonal(g.kind)) return g.nt == 2 ? GC_DIAG2 : GC_DIAG1;
  return g.nt == 2 ? GC_DENSE2 : GC_DENSE1;
}

double gate_angle(const HostGate& g, const double* params) {
  return g.param < 0 ? g.constant : g.constant + g.coef * params[g.param];
}

uint64_t ctrl_mask(const HostGate& g) {
  uint64_t m = 0;
  for (int q : g.ctrls) m |= 1ull << q;
  return m;
}

// Convert an FP64 interleaved table to the device dtype and upload it.
qs_status upload_table(const std::vector<double>& tab, qs_dtype dt, void* d_dst, cudaStream_t st,
                       std::vector<double>& staging) {
  if (dt == QS_C128) {
    QS_CUDA(cudaMemcpyAsync(d_dst, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  } else {
    staging.resize((tab.size() + 1) / 2);
    float* f = reinterpret_cast<float*>(staging.data());
    for (size_t i = 0; i < tab.size(); ++i) f[i] = (float)tab[i];
    QS_CUDA(cudaMemcpyAsync(d_dst, f, tab.size() * sizeof(float), cudaMemcpyHostToDevice, st));
  }
  // pageable source: the copy has consumed the host buffer when the call returns
  return QS_OK;
}

qs_status build_csr(const SlotMap& sm, int n_out, int** d_row, int** d_sidx, double** d_w, cudaStream_t st) {
  std::vector<int> row(n_out + 1, 0), sidx;
  std::vector<double> w;
  std::vector<std::vector<std::pair<int, double>>> by(n_out);
  for (size_t s = 0; s < sm.out.size(); ++s) by[sm.out[s]].push_back({(int)s, sm.weight[s]});
  for (int o = 0; o < n_out; ++o) {
    row[o + 1] = row[o] + (int)by[o].size();
    for (auto& e : by[o]) {
      sidx.push_back(e.first);
      w.push_back(e.second);
    }
  }
  if (sidx.empty()) {
    sidx.push_back(0);
    w.push_back(0);
  }
  QS_CUDA(cudaMalloc(d_row, row.size() * sizeof(int)));
  QS_CUDA(cudaMalloc(d_sidx, sidx.size() * sizeof(int)));
  QS_CUDA(cudaMalloc(d_w, w.size() * sizeof(double)));
  QS_CUDA(cudaMemcpyAsync(*d_row, row.data(), row.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  QS_CUDA(cudaMemcpyAsync(*d_sidx, sidx.data(), sidx.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  QS_CUDA(cudaMemcpyAsync(*d_w, w.data(), w.size() * sizeof(double), cudaMemcpyHostToDevice, st));
  QS_CUDA(cudaStreamSynchronize(st));
  return QS_OK;
}

void default_opts(qs_dtype dt, const qs_options* in, int ne, int* fuse, int* m, int* c) {
  *fuse = (in && in->fuse) ? in->fuse : 1;
  int mm = (in && in->tile_bits) ? in->tile_bits : (dt == QS_C64 ? 12 : 11);
  mm = std::max(kRegBits, std::min(mm, std::min(max_tile_bits(dt), ne)));
  int cc = (in && in->low_bits) ? in->low_bits : 4;
  cc = std::max(1, std::min(cc, mm));
  if (mm - cc > 12) cc = mm - 12;
  *m = mm;
  *c = cc;
}

qs_status check_state(const qs_state* s) {
  QS_CHECK(s != nullptr, "null state");
  QS_CHECK(s->ptr != nullptr, "state has no buffer");
  return QS_OK;
}

// ---------------------------------------------------------------------------- circuit plan

// host_only: plan on the host and stop before any device work (inspection).
qs_status finalize_plan(qs_circuit* c, qs_dtype dt, cudaStream_t st, bool host_only = false) {
  CircuitPlan& P = c->plan;
  P.release();
  P.dt = dt;
  P.ne = std::max(c->n, kRegBits);
  default_opts(dt, &c->opts, P.ne, &P.fuse, &P.m, &P.c);
  P.n_params = c->n_params;
  const size_t G = c->gates.size();
  P.off_u.assign(G, -1);
  P.off_ud.assign(G, -1);
  P.off_a.assign(G, -1);
  P.gclass.assign(G, 0);
  int off = 0;
  for (size_t i = 0; i < G; ++i) {
    const HostGate& g = c->gates[i];
    const int cls = gate_class(g);
    P.gclass[i] = cls;
    int cnt = 4;
    if (cls == GC_DENSE2) cnt = 16;
    P.off_u[i] = off;
    off += cnt;
    P.off_ud[i] = off;
    off += cnt;
    if (g.param >= 0) {
      P.off_a[i] = off;
      off += cnt;
    }
  }
  // runs of single-qubit gates for the forward passes
  P.run_head.assign(G, -1);
  P.runs.clear();
  P.run_off.clear();
  P.run_diag.clear();
  // checkpoint segments: gates [s K, (s + 1) K); no run and no pass crosses them
  const int ckK = c->opts.checkpoint > 0 ? c->opts.checkpoint : 0;
  auto seg_of = [&](size_t i) { return ckK > 0 ? (int)(i / (size_t)ckK) : 0; };
  const int n_seg = ckK > 0 ? std::max(1, (int)((G + ckK - 1) / ckK)) : 1;
  if (c->fuse_1q) {
    auto single = [&](const HostGate& g) { return g.nt == 1 && g.ctrls.empty() && g.kind != QS_GATE_I; };
    std::vector<int> last(64, -1);        // latest gate touching each qubit
    std::vector<int> run_of(G, -1);       // gate -> index in P.runs of the run it heads or joins
    for (size_t i = 0; i < G; ++i) {
      const HostGate& g = c->gates[i];
      if (g.kind == QS_GATE_I) continue;
      if (single(g)) {
        const int q = g.t[0], j = last[q];
        if (j >= 0 && single(c->gates[j]) && seg_of((size_t)j) == seg_of(i)) {
          int r = run_of[j];
          if (r < 0) {
            r = (int)P.runs.size();
            P.runs.push_back({j});
            run_of[j] = r;
          }
          P.runs[r].push_back((int)i);
          run_of[i] = r;
          P.run_head[i] = P.runs[r][0];
          last[q] = (int)i;
          continue;
        }
      }
      last[g.t[0]] = (int)i;
      if (g.nt == 2) last[g.t[1]] = (int)i;
      for (int q : g.ctrls) last[q] = (int)i;
    }
    for (const auto& r : P.runs) {
      bool diag = true;
      for (int i : r) diag = diag && gate_diagonal(c->gates[i].kind);
      P.run_diag.push_back(diag);
      P.run_off.push_back(off);
      off += 4;
    }
  }
  P.n_coef = std::max(off, 1);
  if (!host_only) QS_CUDA(cudaMalloc(&P.d_coef, (size_t)P.n_coef * 16));
  if (P.fuse < 0) {
    P.valid = true;
    return QS_OK;
  }
  // complex64 micro-op passes: without a tile option the forward sweep takes
  // 2^13-amplitude tiles (16 compute warps per SM) and the reverse sweep, which
  // carries psi and lam, 2^12 (three buffers of both fit in shared memory)
  // (states below 22 qubits have too few tiles to fill the GPU with one
  // 192 KB CTA per SM; their many small launches overlap better on the
  // interpreter kernel: the 2048-instance batch ran 5150 -> 3897 instances/s)
  // From 22 qubits the default compiles the micro-op passes for the circuit
  // (t2gen.cu: the op dispatch taken out; 28-qubit random circuit 46.4 -> 15.0
  // ms), each pass within the compile budget; fuse = 3 keeps the library's
  // micro-op kernels, fuse = 4 compiles every micro-op pass.
  const bool micro = dt == QS_C64 && (P.fuse == 3 || P.fuse == 4 || (P.fuse == 1 && P.ne >= kMicroMinQubits));
  const int gen = !micro || P.fuse == 3 ? 0 : P.fuse == 4 ? 2 : 1;
  int m_fwd = P.m, m_rev = P.m;
  if (micro && !c->opts.tile_bits) {
    m_fwd = std::min(13, P.ne);
    m_rev = std::min(12, P.ne);
  }
  PlanParams pp{P.ne, m_fwd, P.c, dt, micro};
  PlanParams pp_rev{P.ne, m_rev, P.c, dt, micro};
  if (pp.m - pp.c > 12) pp.c = pp.m - 12;
  auto make_item = [&](size_t i, bool reverse) {
    const HostGate& g = c->gates[i];
    PlanItem it;
    it.nt = g.nt;
    it.t[0] = g.t[0];
    it.t[1] = g.nt == 2 ? g.t[1] : g.t[0];
    it.ctrl = ctrl_mask(g);
    it.touched = it.ctrl | (1ull << g.t[0]) | (g.nt == 2 ? (1ull << g.t[1]) : 0);
    const int cls = P.gclass[i];
    it.kind = cls == GC_DENSE1 ? IK_DENSE1 : cls == GC_DENSE2 ? IK_DENSE2 : IK_DIAG;
    // The op names what the gate is: X gates (CNOT, Toffoli) as swaps, real
    // matrices (H, RY) with real arithmetic, Z (CZ) as a sign flip, other
    // diagonals of +-1, +-i as unit diagonals.  Each kernel lowers them to what
    // it implements (the complex64 interpreter kernel runs all of them as
    // general matrices: there an extra op type cost more issue slots than it
    // saved, 5541 -> 4625 gates/s; complex128 one-state passes are FP64-bound
    // and gain, 397 -> 467).
    const bool rx = g.kind == QS_GATE_RX, x = g.kind == QS_GATE_X;
    const bool real = real_kind(g.kind), unit = unit_diag_kind(g.kind), zf = g.kind == QS_GATE_Z && g.nt == 1;
    const uint8_t apply_type = cls == GC_DENSE1   ? (rx ? OP_RX : x ? OP_X : real ? OP_REAL1 : OP_DENSE1)
                               : cls == GC_DENSE2 ? OP_DENSE2
                                                  : (zf ? OP_ZFLIP : unit ? OP_UDIAG : OP_DIAG);
    if (!reverse) {
      it.ops.push_back(ItemOp{apply_type, 0, P.off_u[i], -1, 0.0});
    } else {
      if (g.param >= 0) {
        const uint8_t gt = cls == GC_DENSE1 ? OP_GRAD1 : cls == GC_DENSE2 ? OP_GRAD2 : OP_GRADDIAG;
        it.ops.push_back(ItemOp{gt, 0, P.off_a[i], g.param, g.coef});
      }
      it.ops.push_back(ItemOp{apply_type, OPF_LAM, P.off_ud[i], -1, 0.0});
    }
    return it;
  };
  std::vector<std::vector<PlanItem>> fwd(n_seg), rev(n_seg);
  std::vector<int> run_index(G, -1);  // head gate -> its run
  for (size_t r = 0; r < P.runs.size(); ++r) run_index[P.runs[r][0]] = (int)r;
  for (size_t i = 0; i < G; ++i) {
    if (c->gates[i].kind == QS_GATE_I || P.run_head[i] >= 0) continue;  // absorbed into its run's head
    PlanItem it = make_item(i, false);
    const int r = run_index[i];
    if (r >= 0) {  // the run's product replaces the head gate's op
      it.kind = P.run_diag[r] ? IK_DIAG : IK_DENSE1;
      // products of real matrices are real, products of i^k are i^k: exactly,
      // in complex arithmetic (the other parts stay exact zeros)
      bool real = true, unit = true;
      for (int j : P.runs[r]) {
        real = real && real_kind(c->gates[j].kind);
        unit = unit && unit_diag_kind(c->gates[j].kind);
      }
      const uint8_t ty = P.run_diag[r] ? (unit ? OP_UDIAG : OP_DIAG) : (real ? OP_REAL1 : OP_DENSE1);
      it.ops.clear();
      it.ops.push_back(ItemOp{ty, 0, P.run_off[r], -1, 0.0});
    }
    fwd[seg_of(i)].push_back(it);
  }
  for (size_t i = G; i-- > 0;)
    if (c->gates[i].kind != QS_GATE_I || c->gates[i].param >= 0) rev[seg_of(i)].push_back(make_item(i, true));
  SlotMap none;
  for (int sg = 0; sg < n_seg; ++sg) {
    if (!fwd[sg].empty()) QS_TRY(plan_items(fwd[sg], pp, PF_LOAD_PSI | PF_STORE_PSI, &P.fwd, &none));
    P.fwd_seg_end.push_back((int)P.fwd.passes.size());
  }
  for (int sg = n_seg - 1; sg >= 0; --sg) {
    if (!rev[sg].empty())
      QS_TRY(plan_items(rev[sg], pp_rev, PF_LOAD_PSI | PF_LOAD_LAM | PF_STORE_PSI | PF_STORE_LAM, &P.rev,
                        &P.rev_slots));
    P.rev_seg_end.push_back((int)P.rev.passes.size());
  }
  P.fwd.gen = P.rev.gen = gen;
  if (host_only) return QS_OK;
  QS_TRY(P.fwd.upload(st));
  QS_TRY(P.rev.upload(st));
  QS_TRY(build_csr(P.rev_slots, std::max(P.n_params, 1), &P.d_row, &P.d_sidx, &P.d_w, st));
  const uint64_t n_tiles = 1ull << (P.ne - m_fwd), n_tiles_rev = 1ull << (P.ne - m_rev);
  P.grid1 = tile_grid_size(dt, m_fwd, 1, (int)std::min<uint64_t>(n_tiles, 1u << 30));
  P.grid2 = tile_grid_size(dt, m_rev, 2, (int)std::min<uint64_t>(n_tiles_rev, 1u << 30));
  P.valid = true;
  return QS_OK;
}

qs_status fill_circuit_coef(qs_circuit* c, const double* params) {
  CircuitPlan& P = c->plan;
  std::vector<double>& tab = c->host_coef;
  tab.assign((size_t)P.n_coef * 2, 0.0);
  for (size_t i = 0; i < c->gates.size(); ++i) {
    const HostGate& g = c->gates[i];
    const double th = gate_angle(g, params);
    cd U[16], A[16];
    int d = 0;
    gate_unitary(g, th, U, &d);
    const int cls = P.gclass[i];
    auto put = [&](int off, int k, cd v) {
      tab[2 * (off + k)] = v.real();
      tab[2 * (off + k) + 1] = v.imag();
    };
    if (cls == GC_DIAG1 || cls == GC_DIAG2) {
      for (int k = 0; k < d; ++k) {
        put(P.off_u[i], k, U[k * d + k]);
        put(P.off_ud[i], k, std::conj(U[k * d + k]));
      }
    } else if (g.kind == QS_GATE_RX) {
      const double cth = std::cos(0.5 * th), sth = std::sin(0.5 * th);
      put(P.off_u[i], 0, cd(cth, sth));
      put(P.off_ud[i], 0, cd(cth, -sth));
    } else {
      for (int r = 0; r < d; ++r)
        for (int col = 0; col < d; ++col) {
          put(P.off_u[i], r * d + col, U[r * d + col]);
          put(P.off_ud[i], r * d + col, std::conj(U[col * d + r]));
        }
    }
    if (g.param >= 0) {
      gate_generator(g, th, A, &d);
      if (cls == GC_DIAG1 || cls == GC_DIAG2) {
        for (int k = 0; k < d; ++k) put(P.off_a[i], k, A[k * d + k]);
      } else {
        for (int k = 0; k < d * d; ++k) put(P.off_a[i], k, A[k]);
      }
    }
  }
  // products of the single-qubit runs (later gates multiply on the left)
  for (size_t r = 0; r < P.runs.size(); ++r) {
    cd M[4] = {1, 0, 0, 1};
    for (int i : P.runs[r]) {
      cd U[16];
      int d = 0;
      gate_unitary(c->gates[i], gate_angle(c->gates[i], params), U, &d);
      const cd N[4] = {U[0] * M[0] + U[1] * M[2], U[0] * M[1] + U[1] * M[3], U[2] * M[0] + U[3] * M[2],
                       U[2] * M[1] + U[3] * M[3]};
      for (int k = 0; k < 4; ++k) M[k] = N[k];
    }
    const int o = P.run_off[r];
    if (P.run_diag[r]) {
      tab[2 * o] = M[0].real();
      tab[2 * o + 1] = M[0].imag();
      tab[2 * (o + 1)] = M[3].real();
      tab[2 * (o + 1) + 1] = M[3].imag();
    } else {
      for (int k = 0; k < 4; ++k) {
        tab[2 * (o + k)] = M[k].real();
        tab[2 * (o + k) + 1] = M[k].imag();
      }
    }
  }
  return QS_OK;
}

qs_status run_passes(const TilePlan& plan, int begin, int end, qs_dtype dt, void* psi, void* lam, const void* coef,
                     const uint8_t* cut, double* partials, int n, int n_edges, int grid1, int grid2,
                     cudaStream_t st) {
  for (int i = begin; i < end; ++i) {
    const auto& hdr = plan.passes[i].hdr;
    TileLaunch L;
    L.psi = psi;
    L.lam = lam;
    L.coef = coef;
    L.cut = cut;
    L.partials = partials;
    L.n = n;
    L.n_edges = n_edges;
    const bool two = hdr.flags & (PF_LOAD_LAM | PF_STORE_LAM);
    L.grid = (two || hdr.n_slots > 0) ? grid2 : grid1;
    L.stride = grid2;
    TraceRec* rec = trace_begin(st);
    QS_TRY(launch_tile_pass(dt, plan, i, L, st));
    if (rec) {
      const double S = (double)amp_bytes(dt) * (double)(1ull << n);
      const uint32_t f = hdr.flags;
      rec->bytes = S * (((f & PF_LOAD_PSI) ? 1 : 0) + ((f & PF_LOAD_LAM) ? 1 : 0) + ((f & PF_STORE_PSI) ? 1 : 0) +
                        ((f & PF_STORE_LAM) ? 1 : 0)) +
                   ((f & PF_NEED_CUT) ? (double)(1ull << n) : 0.0);
      const bool gen = (size_t)i < plan.gen_fn.size() && plan.gen_fn[i];
      rec->kind = !plan.passes[i].t2 ? QS_TRACE_TILE : gen ? QS_TRACE_TILE2GEN : QS_TRACE_TILE2;
      QS_CUDA(cudaEventRecord(rec->end, st));
    }
  }
  return QS_OK;
}

// ---------------------------------------------------------------------------- tracing

static std::mutex g_trace_mu;
static bool g_trace_on = false;
static std::vector<TraceRec> g_trace;
static size_t g_trace_used = 0;
constexpr size_t kTraceMax = 65536;

bool trace_active() { return g_trace_on; }

TraceRec* trace_begin(cudaStream_t st) {
  if (!g_trace_on) return nullptr;
  std::lock_guard<std::mutex> lk(g_trace_mu);
  if (g_trace_used >= kTraceMax) return nullptr;
  if (g_trace_used == g_trace.size()) {
    TraceRec r;
    if (cudaEventCreate(&r.start) != cudaSuccess || cudaEventCreate(&r.end) != cudaSuccess) {
      (void)cudaGetLastError();
      return nullptr;
    }
    g_trace.push_back(r);
  }
  TraceRec* r = &g_trace[g_trace_used++];
  if (cudaEventRecord(r->start, st) != cudaSuccess) {
    (void)cudaGetLastError();
    --g_trace_used;
    return nullptr;
  }
  return r;
}

qs_status trace_enable(int on) {
  std::lock_guard<std::mutex> lk(g_trace_mu);
  g_trace_on = on != 0;
  if (on) g_trace_used = 0;
  return QS_OK;
}

qs_status trace_read(int max, int* n, double* ms, double* bytes, int* kinds) {
  std::lock_guard<std::mutex> lk(g_trace_mu);
  const int k = (int)std::min<size_t>(g_trace_used, (size_t)std::max(max, 0));
  for (int i = 0; i < k; ++i) {
    QS_CUDA(cudaEventSynchronize(g_trace[i].end));
    float t = 0;
    QS_CUDA(cudaEventElapsedTime(&t, g_trace[i].start, g_trace[i].end));
    if (ms) ms[i] = t;
    if (bytes) bytes[i] = g_trace[i].bytes;
    if (kinds) kinds[i] = g_trace[i].kind;
  }
  *n = k;
  return QS_OK;
}

qs_status apply_per_gate(qs_state* s, qs_circuit* c, const double* params) {
  for (const HostGate& g : c->gates) {
    if (g.kind == QS_GATE_I) continue;
    cd U[16];
    int d = 0;
    gate_unitary(g, gate_angle(g, params), U, &d);
    double buf[32];
    const uint64_t cm = ctrl_mask(g);
    if (gate_diagonal(g.kind)) {
      for (int k = 0; k < d; ++k) {
        buf[2 * k] = U[k * d + k].real();
        buf[2 * k + 1] = U[k * d + k].imag();
      }
      QS_TRY(launch_gate_diag(s->dt, s->ptr, s->ne, g.nt, g.t, cm, buf, s->st));
    } else {
      for (int k = 0; k < d * d; ++k) {
        buf[2 * k] = U[k].real();
        buf[2 * k + 1] = U[k].imag();
      }
      QS_TRY(launch_gate_dense(s->dt, s->ptr, s->ne, g.nt, g.t, cm, buf, s->st));
    }
  }
  return QS_OK;
}

qs_status ensure_plan(qs_circuit* c, qs_dtype dt, cudaStream_t st) {
  if (c->plan.valid && c->plan.dt == dt) return QS_OK;
  return finalize_plan(c, dt, st);
}

}  // namespace qs

// ============================================================================ C ABI

extern "C" {

const char* qs_version(void) { return "qsim-gb300 0.1 (sm_103a)"; }
const char* qs_last_error(void) { return g_last_error.c_str(); }

qs_status qs_state_create(int n_qubits, qs_dtype dtype, void* dev_buf, size_t buf_bytes, void* cuda_stream,
                          qs_state** out) {
  QS_CHECK(out != nullptr, "out is null");
  QS_CHECK(n_qubits >= 1 && n_qubits <= kMaxQubits, "n_qubits must be in 1..34");
  QS_CHECK(valid_dtype(dtype), "invalid dtype");
  qs_state* s = new qs_state;
  s->n = n_qubits;
  s->ne = std::max(n_qubits, kRegBits);
  s->dt = dtype;
  s->st = (cudaStream_t)cuda_stream;
  s->bytes = amp_bytes(dtype) << s->ne;
  if (dev_buf) {
    if (buf_bytes < s->bytes || ((uintptr_t)dev_buf & 255)) {
      delete s;
      set_error("dev_buf too small (needs 2^max(n,4) amplitudes) or not 256-byte aligned");
      return QS_ERR_INVALID_ARG;
    }
    s->ptr = dev_buf;
    s->owned = false;
  } else {
    cudaError_t e = cudaMalloc(&s->ptr, s->bytes);
    if (e != cudaSuccess) {
      delete s;
      return cuda_fail(e, "cudaMalloc(state)");
    }
    s->owned = true;
  }
  if (s->ne != s->n) {
    cudaError_t e = cudaMemsetAsync(s->ptr, 0, s->bytes, s->st);
    if (e != cudaSuccess) {
      if (s->owned) cudaFree(s->ptr);
      delete s;
      return cuda_fail(e, "cudaMemsetAsync");
    }
  }
  *out = s;
  return QS_OK;
}

qs_status qs_state_destroy(qs_state* s) {
  if (!s) return QS_OK;
  if (s->st) cudaStreamSynchronize(s->st);
  if (s->owned && s->ptr) cudaFree(s->ptr);
  if (s->scratch) cudaFree(s->scratch);
  if (s->save) cudaFree(s->save);
  delete s;
  return QS_OK;
}

qs_status qs_state_device_ptr(const qs_state* s, void** dev_ptr) {
  QS_TRY(check_state(s));
  QS_CHECK(dev_ptr != nullptr, "dev_ptr is null");
  *dev_ptr = s->ptr;
  return QS_OK;
}

qs_status qs_state_set_basis(qs_state* s, uint64_t index) {
  QS_TRY(check_state(s));
  QS_CHECK(index < (1ull << s->n), "basis index out of range");
  return launch_set_basis(s->dt, s->ptr, s->ne, index, s->st);
}

qs_status qs_state_set_plus(qs_state* s) {
  QS_TRY(check_state(s));
  if (s->ne == s->n) return launch_set_plus(s->dt, s->ptr, s->n, s->st);
  // padded state: the first 2^n amplitudes, the rest zero
  QS_CUDA(cudaMemsetAsync(s->ptr, 0, s->bytes, s->st));
  return launch_set_plus(s->dt, s->ptr, s->n, s->st);
}

qs_status qs_state_copy_in(qs_state* s, const void* src, int src_on_device) {
  QS_TRY(check_state(s));
  QS_CHECK(src != nullptr, "src is null");
  const size_t nb = amp_bytes(s->dt) << s->n;
  if (s->ne != s->n) QS_CUDA(cudaMemsetAsync(s->ptr, 0, s->bytes, s->st));
  QS_CUDA(cudaMemcpyAsync(s->ptr, src, nb, src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s->st));
  if (!src_on_device) QS_CUDA(cudaStreamSynchronize(s->st));
  return QS_OK;
}

qs_status qs_state_copy_out(const qs_state* s, void* dst, int dst_on_device) {
  QS_TRY(check_state(s));
  QS_CHECK(dst != nullptr, "dst is null");
  const size_t nb = amp_bytes(s->dt) << s->n;
  QS_CUDA(cudaMemcpyAsync(dst, s->ptr, nb, dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s->st));
  if (!dst_on_device) QS_CUDA(cudaStreamSynchronize(s->st));
  return QS_OK;
}

qs_status qs_state_copy(qs_state* dst, const qs_state* src) {
  QS_TRY(check_state(dst));
  QS_TRY(check_state(src));
  QS_CHECK(dst->n == src->n && dst->dt == src->dt, "states differ in n or dtype");
  QS_CUDA(cudaMemcpyAsync(dst->ptr, src->ptr, src->bytes, cudaMemcpyDeviceToDevice, dst->st));
  return QS_OK;
}

qs_status qs_state_norm2(const qs_state* s_, double* out) {
  QS_TRY(check_state(s_));
  QS_CHECK(out != nullptr, "out is null");
  qs_state* s = const_cast<qs_state*>(s_);
  const int grid = ham_grid_size(s->ne);
  QS_TRY(ensure_scratch(s, grid + 8));
  QS_TRY(launch_norm2(s->dt, s->ptr, s->ne, s->scratch, grid, s->st));
  QS_TRY(launch_reduce_slots(s->scratch, 1, grid, nullptr, s->scratch + grid, s->st));
  QS_CUDA(cudaMemcpyAsync(out, s->scratch + grid, sizeof(double), cudaMemcpyDeviceToHost, s->st));
  QS_CUDA(cudaStreamSynchronize(s->st));
  return QS_OK;
}

// ---------------------------------------------------------------------------- circuits

qs_status qs_circuit_create(int n_qubits, qs_circuit** out) {
  QS_CHECK(out != nullptr, "out is null");
  QS_CHECK(n_qubits >= 1 && n_qubits <= kMaxQubits, "n_qubits must be in 1..34");
  qs_circuit* c = new qs_circuit;
  c->n = n_qubits;
  *out = c;
  return QS_OK;
}

qs_status qs_circuit_destroy(qs_circuit* c) {
  if (!c) return QS_OK;
  cudaDeviceSynchronize();
  c->plan.release();
  delete c;
  return QS_OK;
}

qs_status qs_circuit_add(qs_circuit* c, int kind, const int* targets, int n_t, const int* ctrls, int n_c,
                         int param_idx, double coef, double constant, const double* matrix) {
  QS_CHECK(c != nullptr, "null circuit");
  QS_CHECK(gate_known(kind), "unknown gate kind");
  const int want = kind == QS_GATE_MATRIX ? n_t : gate_targets(kind);
  QS_CHECK(n_t == want && (n_t == 1 || n_t == 2), "wrong number of targets for this gate kind");
  QS_CHECK(targets != nullptr, "targets is null");
  QS_CHECK(n_c >= 0 && (n_c == 0 || ctrls != nullptr), "bad controls");
  QS_CHECK(n_c + n_t <= c->n, "more target+control qubits than the circuit has");
  uint64_t used = 0;
  for (int i = 0; i < n_t; ++i) {
    QS_CHECK(targets[i] >= 0 && targets[i] < c->n, "target qubit out of range");
    QS_CHECK(!((used >> targets[i]) & 1), "duplicate qubit");
    used |= 1ull << targets[i];
  }
  for (int i = 0; i < n_c; ++i) {
    QS_CHECK(ctrls[i] >= 0 && ctrls[i] < c->n, "control qubit out of range");
    QS_CHECK(!((used >> ctrls[i]) & 1), "control qubit repeats a target or control");
    used |= 1ull << ctrls[i];
  }
  QS_CHECK(param_idx >= -1, "param_idx must be >= -1");
  QS_CHECK(param_idx == -1 || gate_parametric(kind), "only RX/RY/RZ/PS/RXX/RYY/RZZ take a parameter");
  QS_CHECK(std::isfinite(coef) && std::isfinite(constant), "non-finite angle binding");
  if (kind == QS_GATE_MATRIX) QS_CHECK(matrix != nullptr, "MATRIX gate needs a matrix");
  HostGate g;
  g.kind = kind;
  g.nt = n_t;
  g.t[0] = targets[0];
  g.t[1] = n_t == 2 ? targets[1] : targets[0];
  g.ctrls.assign(ctrls, ctrls + n_c);
  g.param = param_idx;
  g.coef = coef;
  g.constant = constant;
  if (kind == QS_GATE_MATRIX) {
    const int d = 1 << n_t;
    g.matrix.assign(matrix, matrix + 2 * d * d);
    for (double v : g.matrix) QS_CHECK(std::isfinite(v), "non-finite matrix entry");
  }
  c->gates.push_back(g);
  if (param_idx >= 0) c->n_params = std::max(c->n_params, param_idx + 1);
  if (c->plan.valid) {
    cudaDeviceSynchronize();
    c->plan.release();
  }
  return QS_OK;
}

qs_status qs_circuit_finalize(qs_circuit* c, qs_dtype dtype, const qs_options* opts) {
  QS_CHECK(c != nullptr, "null circuit");
  QS_CHECK(valid_dtype(dtype), "invalid dtype");
  if (opts) {
    QS_CHECK(opts->tile_bits == 0 || (opts->tile_bits >= kMinTileBits && opts->tile_bits <= kMaxTileBits),
             "tile_bits must be 0 or 6..13");
    QS_CHECK(opts->low_bits >= 0 && opts->low_bits <= kMaxTileBits, "low_bits must be 0..13");
    QS_CHECK(opts->fuse >= -1 && opts->fuse <= 4, "fuse must be -1, 0, 1, 2, 3 or 4");
    QS_CHECK(opts->checkpoint >= 0, "checkpoint must be >= 0");
    c->opts = *opts;
  }
  cudaDeviceSynchronize();
  return finalize_plan(c, dtype, nullptr);
}

qs_status qs_circuit_codegen(qs_circuit* c, const qs_options* opts, int which, int compile, char* src, size_t cap,
                             size_t* src_len, int* n_gen, size_t* cubin_bytes) {
  QS_CHECK(c != nullptr, "null circuit");
  QS_CHECK(which == 0 || which == 1, "which must be 0 (forward plan) or 1 (reverse plan)");
  QS_CHECK(cap == 0 || src != nullptr, "src is null");
  QS_CHECK(c->dm_n == 0, "density-matrix circuits are planned by their own engine");
  QS_CHECK(!c->plan.valid, "qs_circuit_codegen takes a circuit that has not been finalized");
  if (opts) {
    QS_CHECK(opts->tile_bits == 0 || (opts->tile_bits >= kMinTileBits && opts->tile_bits <= kMaxTileBits),
             "tile_bits must be 0 or 6..13");
    QS_CHECK(opts->low_bits >= 0 && opts->low_bits <= kMaxTileBits, "low_bits must be 0..13");
    QS_CHECK(opts->fuse >= 0 && opts->fuse <= 4, "fuse must be 0..4 for a generated plan");
    QS_CHECK(opts->checkpoint >= 0, "checkpoint must be >= 0");
  }
  const qs_options saved = c->opts;
  qs_options o = opts ? *opts : qs_options{};
  if (!o.fuse) o.fuse = 4;
  c->opts = o;
  const qs_status st = finalize_plan(c, QS_C64, nullptr, true);
  c->opts = saved;
  auto done = [&](qs_status r) {
    c->plan.release();
    return r;
  };
  if (st != QS_OK) return done(st);
  const TilePlan& plan = which == 0 ? c->plan.fwd : c->plan.rev;
  std::string text;
  std::vector<int> ids;
  if (!t2gen_source(plan, &text, &ids)) {
    set_error("a micro-op pass holds an op the generator does not write out");
    return done(QS_ERR_UNSUPPORTED);
  }
  if (src_len) *src_len = text.size();
  if (n_gen) *n_gen = (int)ids.size();
  if (cap) {
    const size_t k = std::min(cap - 1, text.size());
    std::memcpy(src, text.data(), k);
    src[k] = 0;
  }
  if (cubin_bytes) *cubin_bytes = 0;
  if (compile && !ids.empty()) {  // as the plan's upload compiles them: one program per pass
    std::vector<std::string> srcs(ids.size());
    for (size_t k = 0; k < ids.size(); ++k) t2gen_pass_source(plan, ids[k], &srcs[k]);
    std::vector<std::vector<char>> cubins;
    const qs_status r = t2gen_compile(srcs, &cubins);
    if (r != QS_OK) return done(r);
    size_t tot = 0;
    for (const auto& cb : cubins) tot += cb.size();
    if (cubin_bytes) *cubin_bytes = tot;
  }
  return done(QS_OK);
}

qs_status qs_circuit_info(const qs_circuit* c, int* n_gates, int* n_params, int* n_passes) {
  QS_CHECK(c != nullptr, "null circuit");
  if (n_gates) *n_gates = (int)c->gates.size();
  if (n_params) *n_params = c->n_params;
  if (n_passes) {
    if (!c->plan.valid) *n_passes = -1;
    else if (c->plan.fuse < 0) *n_passes = (int)c->gates.size();
    else *n_passes = (int)c->plan.fwd.passes.size();
  }
  return QS_OK;
}

qs_status qs_apply_circuit(qs_state* s, qs_circuit* c, const double* params, int n_params) {
  QS_TRY(check_state(s));
  QS_CHECK(c != nullptr, "null circuit");
  QS_CHECK(c->n == s->n, "circuit and state differ in qubit count");
  QS_CHECK(n_params >= c->n_params, "too few parameters");
  QS_CHECK(c->n_params == 0 || params != nullptr, "params is null");
  QS_TRY(ensure_plan(c, s->dt, s->st));
  if (c->plan.fuse < 0) return apply_per_gate(s, c, params);
  if (c->plan.fwd.passes.empty()) return QS_OK;
  QS_TRY(fill_circuit_coef(c, params));
  QS_TRY(upload_table(c->host_coef, s->dt, c->plan.d_coef, s->st, s->host_out));
  QS_TRY(ensure_scratch(s, 8));
  return run_passes(c->plan.fwd, 0, (int)c->plan.fwd.passes.size(), s->dt, s->ptr, nullptr, c->plan.d_coef, nullptr,
                    s->scratch, s->ne, 0, c->plan.grid1, c->plan.grid2, s->st);
}

// ---------------------------------------------------------------------------- Hamiltonians

qs_status qs_ham_create(int n_qubits, int n_terms, const uint64_t* xmask, const uint64_t* zmask, const double* coef,
                        qs_ham** out) {
  QS_CHECK(out != nullptr, "out is null");
  QS_CHECK(n_qubits >= 1 && n_qubits <= kMaxQubits, "n_qubits must be in 1..34");
  QS_CHECK(n_terms >= 0, "n_terms < 0");
  QS_CHECK(n_terms == 0 || (xmask && zmask && coef), "null term arrays");
  const uint64_t lim = 1ull << n_qubits;
  for (int k = 0; k < n_terms; ++k) {
    QS_CHECK(xmask[k] < lim && zmask[k] < lim, "Pauli mask names a qubit >= n_qubits");
    QS_CHECK(std::isfinite(coef[k]), "non-finite coefficient");
  }
  qs_ham* h = new qs_ham;
  h->n = n_qubits;
  h->x.assign(xmask, xmask + n_terms);
  h->z.assign(zmask, zmask + n_terms);
  h->c.assign(coef, coef + n_terms);
  // group by X mask (stable), term coefficient c * i^{#Y}
  std::vector<int> order(n_terms);
  for (int k = 0; k < n_terms; ++k) order[k] = k;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return h->x[a] < h->x[b]; });
  std::vector<DevHamGroup> groups;
  std::vector<DevHamTerm> terms;
  for (int i = 0; i < n_terms; ++i) {
    const int k = order[i];
    if (groups.empty() || groups.back().xmask != h->x[k]) {
      DevHamGroup g;
      g.xmask = h->x[k];
      g.begin = g.end = (int)terms.size();
      groups.push_back(g);
    }
    const int ny = __builtin_popcountll(h->x[k] & h->z[k]) & 3;
    const double cr[4] = {1, 0, -1, 0}, ci[4] = {0, 1, 0, -1};
    DevHamTerm t;
    t.zmask = h->z[k];
    t.re = coef[k] * cr[ny];
    t.im = coef[k] * ci[ny];
    terms.push_back(t);
    groups.back().end = (int)terms.size();
  }
  h->n_groups = (int)groups.size();
  if (groups.empty()) {
    groups.resize(1);
    terms.resize(1);
  }
  cudaError_t e = cudaMalloc(&h->d_groups, groups.size() * sizeof(DevHamGroup));
  if (e == cudaSuccess) e = cudaMalloc(&h->d_terms, terms.size() * sizeof(DevHamTerm));
  if (e == cudaSuccess)
    e = cudaMemcpy(h->d_groups, groups.data(), groups.size() * sizeof(DevHamGroup), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(h->d_terms, terms.data(), terms.size() * sizeof(DevHamTerm), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    if (h->d_groups) cudaFree(h->d_groups);
    if (h->d_terms) cudaFree(h->d_terms);
    delete h;
    return cuda_fail(e, "qs_ham_create");
  }
  *out = h;
  return QS_OK;
}

qs_status qs_ham_destroy(qs_ham* h) {
  if (!h) return QS_OK;
  cudaDeviceSynchronize();
  if (h->d_groups) cudaFree(h->d_groups);
  if (h->d_terms) cudaFree(h->d_terms);
  delete h;
  return QS_OK;
}

static qs_status ham_energy(qs_state* s, const qs_state* src, void* lam, const qs_ham* h, double* d_energy) {
  const int grid = ham_grid_size(src->ne);
  QS_TRY(ensure_scratch(s, grid + 16));
  QS_TRY(launch_ham_apply(src->dt, src->ptr, lam, src->ne, h->d_groups, h->n_groups, h->d_terms, s->scratch, grid,
                          src->st));
  return launch_reduce_slots(s->scratch, 1, grid, nullptr, d_energy, src->st);
}

qs_status qs_apply_hamiltonian(qs_state* dst, const qs_state* src, const qs_ham* h) {
  QS_TRY(check_state(dst));
  QS_TRY(check_state(src));
  QS_CHECK(h != nullptr, "null hamiltonian");
  QS_CHECK(dst != src && dst->ptr != src->ptr, "dst must differ from src");
  QS_CHECK(dst->n == src->n && dst->dt == src->dt && h->n == src->n, "n/dtype mismatch");
  qs_state* s = const_cast<qs_state*>(src);
  const int grid = ham_grid_size(src->ne);
  QS_TRY(ensure_scratch(s, grid + 16));
  QS_TRY(launch_ham_apply(src->dt, src->ptr, dst->ptr, src->ne, h->d_groups, h->n_groups, h->d_terms, s->scratch,
                          grid, src->st));
  if (dst->st != src->st) QS_CUDA(cudaStreamSynchronize(src->st));
  return QS_OK;
}

qs_status qs_expectation(const qs_state* s_, const qs_ham* h, double* energy) {
  QS_TRY(check_state(s_));
  QS_CHECK(h != nullptr && energy != nullptr, "null argument");
  QS_CHECK(h->n == s_->n, "hamiltonian and state differ in qubit count");
  qs_state* s = const_cast<qs_state*>(s_);
  const int grid = ham_grid_size(s->ne);
  QS_TRY(ensure_scratch(s, grid + 16));
  QS_TRY(ham_energy(s, s, nullptr, h, s->scratch + grid));
  QS_CUDA(cudaMemcpyAsync(energy, s->scratch + grid, sizeof(double), cudaMemcpyDeviceToHost, s->st));
  QS_CUDA(cudaStreamSynchronize(s->st));
  return QS_OK;
}

qs_status qs_inner_product(const qs_state* bra, const qs_state* ket, double* out2) {
  QS_TRY(check_state(bra));
  QS_TRY(check_state(ket));
  QS_CHECK(out2 != nullptr, "out2 is null");
  QS_CHECK(bra->n == ket->n && bra->dt == ket->dt, "n/dtype mismatch");
  qs_state* s = const_cast<qs_state*>(ket);
  if (bra->st != ket->st) QS_CUDA(cudaStreamSynchronize(bra->st));
  const int grid = ham_grid_size(s->ne);
  QS_TRY(ensure_scratch(s, 2 * grid + 16));
  QS_TRY(launch_inner(s->dt, bra->ptr, ket->ptr, s->ne, s->scratch, grid, s->st));
  QS_TRY(launch_reduce_slots(s->scratch, 2, grid, nullptr, s->scratch + 2 * grid, s->st));
  QS_CUDA(cudaMemcpyAsync(out2, s->scratch + 2 * grid, 2 * sizeof(double), cudaMemcpyDeviceToHost, s->st));
  QS_CUDA(cudaStreamSynchronize(s->st));
  return QS_OK;
}

namespace {

// Forward passes of a plan on psi; with checkpoints, psi is saved after every
// inner segment boundary.
qs_status forward_sweep(CircuitPlan& P, qs_state* psi, double* d_part, cudaStream_t st) {
  const size_t bytes = amp_bytes(psi->dt) << psi->ne;
  const int nseg = (int)P.fwd_seg_end.size();
  if (nseg > 1 && (int)P.ckpt.size() != nseg - 1) {
    for (void* b : P.ckpt) cudaFree(b);
    P.ckpt.assign(nseg - 1, nullptr);
    for (auto& b : P.ckpt) QS_CUDA(cudaMalloc(&b, bytes));
  }
  int b = 0;
  for (int sg = 0; sg < nseg; ++sg) {
    QS_TRY(run_passes(P.fwd, b, P.fwd_seg_end[sg], psi->dt, psi->ptr, nullptr, P.d_coef, nullptr, d_part, psi->ne, 0,
                      P.grid1, P.grid2, st));
    b = P.fwd_seg_end[sg];
    if (sg + 1 < nseg) QS_CUDA(cudaMemcpyAsync(P.ckpt[sg], psi->ptr, bytes, cudaMemcpyDeviceToDevice, st));
  }
  return QS_OK;
}

// Reverse passes on (psi, lam); with checkpoints, psi is reloaded from the
// saved state at every inner segment boundary before that segment is undone.
qs_status reverse_sweep(CircuitPlan& P, qs_state* psi, qs_state* lam, double* d_part, cudaStream_t st) {
  const size_t bytes = amp_bytes(psi->dt) << psi->ne;
  const int nseg = (int)P.rev_seg_end.size();
  int b = 0;
  for (int r = 0; r < nseg; ++r) {
    const int sg = nseg - 1 - r;
    if (r > 0 && (int)P.ckpt.size() == nseg - 1)
      QS_CUDA(cudaMemcpyAsync(psi->ptr, P.ckpt[sg], bytes, cudaMemcpyDeviceToDevice, st));
    QS_TRY(run_passes(P.rev, b, P.rev_seg_end[r], psi->dt, psi->ptr, lam->ptr, P.d_coef, nullptr, d_part, psi->ne, 0,
                      P.grid1, P.grid2, st));
    b = P.rev_seg_end[r];
  }
  return QS_OK;
}

}  // namespace

qs_status qs_expectation_with_grad(qs_state* psi, qs_state* lam, qs_circuit* c, const qs_ham* h, const double* params,
                                   int n_params, double* energy, double* grad) {
  QS_TRY(check_state(psi));
  QS_TRY(check_state(lam));
  QS_CHECK(c != nullptr && h != nullptr && energy != nullptr, "null argument");
  QS_CHECK(psi != lam && psi->ptr != lam->ptr, "psi and lam must be different states");
  QS_CHECK(psi->n == lam->n && psi->dt == lam->dt, "psi/lam n or dtype mismatch");
  QS_CHECK(c->n == psi->n && h->n == psi->n, "circuit/hamiltonian/state qubit counts differ");
  QS_CHECK(n_params >= c->n_params, "too few parameters");
  QS_CHECK(c->n_params == 0 || (params != nullptr && grad != nullptr), "params/grad is null");
  QS_CHECK(c->dm_n == 0, "density-matrix circuits: expectation with qs_dm_expectation (no adjoint gradient)");
  if (lam->st != psi->st) QS_CUDA(cudaStreamSynchronize(lam->st));
  QS_TRY(ensure_plan(c, psi->dt, psi->st));
  if (c->plan.fuse < 0) {
    set_error("the adjoint gradient runs on fused tile passes (fuse = -1 is forward only)");
    return QS_ERR_UNSUPPORTED;
  }
  CircuitPlan& P = c->plan;
  cudaStream_t st = psi->st;
  QS_TRY(fill_circuit_coef(c, params));
  QS_TRY(upload_table(c->host_coef, psi->dt, P.d_coef, st, psi->host_out));
  const int n_slots = (int)P.rev_slots.out.size();
  const int hgrid = ham_grid_size(psi->ne);
  const size_t part = (size_t)std::max(n_slots, 1) * P.grid2;
  const size_t need = part + n_slots + 1 + std::max(n_params, 1) + hgrid + 16;
  QS_TRY(ensure_scratch(psi, need));
  double* d_part = psi->scratch;
  double* d_slot = d_part + part;
  double* d_E = d_slot + n_slots;
  double* d_grad = d_E + 1;
  double* d_hpart = d_grad + std::max(n_params, 1);
  QS_TRY(forward_sweep(P, psi, d_part, st));
  QS_TRY(launch_ham_apply(psi->dt, psi->ptr, lam->ptr, psi->ne, h->d_groups, h->n_groups, h->d_terms, d_hpart, hgrid,
                          st));
  QS_TRY(launch_reduce_slots(d_hpart, 1, hgrid, nullptr, d_E, st));
  QS_TRY(reverse_sweep(P, psi, lam, d_part, st));
  QS_TRY(launch_reduce_slots(d_part, n_slots, P.grid2, nullptr, d_slot, st));
  QS_TRY(launch_param_gather(d_slot, P.d_row, P.d_sidx, P.d_w, c->n_params, d_grad, st));
  QS_CUDA(cudaMemcpyAsync(energy, d_E, sizeof(double), cudaMemcpyDeviceToHost, st));
  if (c->n_params > 0)
    QS_CUDA(cudaMemcpyAsync(grad, d_grad, c->n_params * sizeof(double), cudaMemcpyDeviceToHost, st));
  QS_CUDA(cudaStreamSynchronize(st));
  for (int p = c->n_params; p < n_params; ++p) grad[p] = 0.0;
  return QS_OK;
}

qs_status qs_expectation_with_grad_multi(qs_state* psi, qs_state* lam, qs_circuit* c, int n_ham,
                                         const qs_ham* const* hams, const double* params, int n_params,
                                         double* energies, double* grads) {
  QS_CHECK(n_ham >= 1 && hams != nullptr && energies != nullptr, "need n_ham >= 1 Hamiltonians and outputs");
  for (int h = 0; h < n_ham; ++h) QS_CHECK(hams[h] != nullptr, "null Hamiltonian");
  if (n_ham == 1) return qs_expectation_with_grad(psi, lam, c, hams[0], params, n_params, energies, grads);
  QS_TRY(check_state(psi));
  QS_TRY(check_state(lam));
  QS_CHECK(c != nullptr, "null circuit");
  QS_CHECK(c->dm_n == 0, "density-matrix circuits: expectation with qs_dm_expectation (no adjoint gradient)");
  QS_CHECK(psi != lam && psi->ptr != lam->ptr, "psi and lam must be different states");
  QS_CHECK(psi->n == lam->n && psi->dt == lam->dt, "psi/lam n or dtype mismatch");
  QS_CHECK(c->n == psi->n, "circuit/state qubit counts differ");
  for (int h = 0; h < n_ham; ++h) QS_CHECK(hams[h]->n == psi->n, "hamiltonian/state qubit counts differ");
  QS_CHECK(n_params >= c->n_params, "too few parameters");
  QS_CHECK(c->n_params == 0 || (params != nullptr && grads != nullptr), "params/grads is null");
  if (lam->st != psi->st) QS_CUDA(cudaStreamSynchronize(lam->st));
  QS_TRY(ensure_plan(c, psi->dt, psi->st));
  if (c->plan.fuse < 0) {
    set_error("the adjoint gradient runs on fused tile passes (fuse = -1 is forward only)");
    return QS_ERR_UNSUPPORTED;
  }
  CircuitPlan& P = c->plan;
  cudaStream_t st = psi->st;
  QS_TRY(fill_circuit_coef(c, params));
  QS_TRY(upload_table(c->host_coef, psi->dt, P.d_coef, st, psi->host_out));
  const int n_slots = (int)P.rev_slots.out.size();
  const int hgrid = ham_grid_size(psi->ne);
  const int np = std::max(c->n_params, 1);
  const size_t part = (size_t)std::max(n_slots, 1) * P.grid2;
  const size_t need = part + n_slots + n_ham + (size_t)n_ham * np + hgrid + 16;
  QS_TRY(ensure_scratch(psi, need));
  double* d_part = psi->scratch;
  double* d_slot = d_part + part;
  double* d_E = d_slot + n_slots;
  double* d_grad = d_E + n_ham;
  double* d_hpart = d_grad + (size_t)n_ham * np;
  const size_t bytes = amp_bytes(psi->dt) << psi->ne;
  if (!psi->save) QS_CUDA(cudaMalloc(&psi->save, bytes));
  // one forward sweep; each Hamiltonian restarts the reverse sweep from its copy
  QS_TRY(forward_sweep(P, psi, d_part, st));
  QS_CUDA(cudaMemcpyAsync(psi->save, psi->ptr, bytes, cudaMemcpyDeviceToDevice, st));
  for (int h = 0; h < n_ham; ++h) {
    if (h > 0) QS_CUDA(cudaMemcpyAsync(psi->ptr, psi->save, bytes, cudaMemcpyDeviceToDevice, st));
    QS_TRY(launch_ham_apply(psi->dt, psi->ptr, lam->ptr, psi->ne, hams[h]->d_groups, hams[h]->n_groups,
                            hams[h]->d_terms, d_hpart, hgrid, st));
    QS_TRY(launch_reduce_slots(d_hpart, 1, hgrid, nullptr, d_E + h, st));
    QS_TRY(reverse_sweep(P, psi, lam, d_part, st));
    if (c->n_params > 0) {
      QS_TRY(launch_reduce_slots(d_part, n_slots, P.grid2, nullptr, d_slot, st));
      QS_TRY(launch_param_gather(d_slot, P.d_row, P.d_sidx, P.d_w, c->n_params, d_grad + (size_t)h * np, st));
    }
  }
  QS_CUDA(cudaMemcpyAsync(energies, d_E, n_ham * sizeof(double), cudaMemcpyDeviceToHost, st));
  std::vector<double> g((size_t)n_ham * np);
  if (c->n_params > 0) QS_CUDA(cudaMemcpyAsync(g.data(), d_grad, g.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  QS_CUDA(cudaStreamSynchronize(st));
  if (grads)
    for (int h = 0; h < n_ham; ++h)
      for (int p = 0; p < n_params; ++p) grads[(size_t)h * n_params + p] = p < c->n_params ? g[(size_t)h * np + p] : 0.0;
  return QS_OK;
}

qs_status qs_expectation_general(qs_state* psi, qs_state* phi, qs_state* lam, qs_circuit* c_right,
                                 qs_circuit* c_left, const qs_ham* h, const double* params, int n_params,
                                 double* energy2, double* grad2) {
  QS_TRY(check_state(psi));
  QS_TRY(check_state(phi));
  QS_TRY(check_state(lam));
  QS_CHECK(c_right != nullptr && h != nullptr && energy2 != nullptr, "null argument");
  qs_circuit* cr = c_right;
  qs_circuit* cl = c_left ? c_left : c_right;
  QS_CHECK(psi->ptr != phi->ptr && psi->ptr != lam->ptr && phi->ptr != lam->ptr, "psi, phi and lam must differ");
  QS_CHECK(psi->n == phi->n && psi->n == lam->n && psi->dt == phi->dt && psi->dt == lam->dt,
           "psi/phi/lam n or dtype mismatch");
  QS_CHECK(cr->n == psi->n && cl->n == psi->n && h->n == psi->n, "circuit/hamiltonian/state qubit counts differ");
  QS_CHECK(cr->dm_n == 0 && cl->dm_n == 0, "density-matrix circuits have no generalised expectation");
  const int np = std::max(cr->n_params, cl->n_params);
  QS_CHECK(n_params >= np, "too few parameters");
  QS_CHECK(np == 0 || (params != nullptr && grad2 != nullptr), "params/grad is null");
  cudaStream_t st = psi->st;
  if (phi->st != st) QS_CUDA(cudaStreamSynchronize(phi->st));
  if (lam->st != st) QS_CUDA(cudaStreamSynchronize(lam->st));
  QS_TRY(ensure_plan(cr, psi->dt, st));
  QS_TRY(ensure_plan(cl, psi->dt, st));
  QS_CHECK(cr->plan.fuse >= 0 && cl->plan.fuse >= 0,
           "the adjoint gradient runs on fused tile passes (fuse = -1 is forward only)");
  const int ne = psi->ne;
  const size_t bytes = amp_bytes(psi->dt) << ne;
  if (!psi->save) QS_CUDA(cudaMalloc(&psi->save, bytes));
  if (!phi->save) QS_CUDA(cudaMalloc(&phi->save, bytes));
  const int hgrid = ham_grid_size(ne);
  const int igrid = hgrid;
  const int slots = std::max<int>({(int)cr->plan.rev_slots.out.size(), (int)cl->plan.rev_slots.out.size(), 1});
  const size_t part = (size_t)slots * std::max(cr->plan.grid2, cl->plan.grid2);
  const int npp = std::max(np, 1);
  const size_t need = part + slots + 2 + 4 * (size_t)npp + hgrid + 2 * (size_t)igrid + 16;
  QS_TRY(ensure_scratch(psi, need));
  double* d_part = psi->scratch;
  double* d_slot = d_part + part;
  double* d_E = d_slot + slots;
  double* d_g = d_E + 2;  // [4][npp]: right Re, right Im, left Re, left Im (each 2 Re <.|A|.> sums)
  double* d_hpart = d_g + 4 * (size_t)npp;
  double* d_ipart = d_hpart + hgrid;
  QS_CUDA(cudaMemsetAsync(d_g, 0, 4 * (size_t)npp * sizeof(double), st));
  const int t0 = 0;
  const double times_i[4] = {0.0, 1.0, 0.0, 1.0};
  // coefficient tables (one fill when both sides are the same circuit)
  QS_TRY(fill_circuit_coef(cr, params));
  QS_TRY(upload_table(cr->host_coef, psi->dt, cr->plan.d_coef, st, psi->host_out));
  if (cl != cr) {
    QS_TRY(fill_circuit_coef(cl, params));
    QS_TRY(upload_table(cl->host_coef, psi->dt, cl->plan.d_coef, st, psi->host_out));
  }
  const CircuitPlan& R = cr->plan;
  const CircuitPlan& L = cl->plan;
  // forward: psi_r = U_r psi, phi_l = U_l phi
  QS_TRY(run_passes(R.fwd, 0, (int)R.fwd.passes.size(), psi->dt, psi->ptr, nullptr, R.d_coef, nullptr, d_part, ne, 0,
                    R.grid1, R.grid2, st));
  QS_TRY(run_passes(L.fwd, 0, (int)L.fwd.passes.size(), psi->dt, phi->ptr, nullptr, L.d_coef, nullptr, d_part, ne, 0,
                    L.grid1, L.grid2, st));
  QS_CUDA(cudaMemcpyAsync(psi->save, psi->ptr, bytes, cudaMemcpyDeviceToDevice, st));
  QS_CUDA(cudaMemcpyAsync(phi->save, phi->ptr, bytes, cudaMemcpyDeviceToDevice, st));
  // E = <H phi_l | psi_r>
  QS_TRY(launch_ham_apply(psi->dt, phi->ptr, lam->ptr, ne, h->d_groups, h->n_groups, h->d_terms, d_hpart, hgrid, st));
  QS_TRY(launch_inner(psi->dt, lam->ptr, psi->ptr, ne, d_ipart, igrid, st));
  QS_TRY(launch_reduce_slots(d_ipart, 2, igrid, nullptr, d_E, st));
  // Each side sweeps twice: with lam and with i lam, giving 2 Re and 2 Im of
  // sum_k coef_k <lam_k|A_k|x_k>.  Right: x = psi, lam = H phi_l.  Left:
  // x = phi, lam = H psi_r (its terms enter conjugated).
  for (int side = 0; side < 2; ++side) {
    qs_circuit* c = side == 0 ? cr : cl;
    const CircuitPlan& P = c->plan;
    qs_state* x = side == 0 ? psi : phi;
    const void* other = side == 0 ? phi->save : psi->save;
    // without parameters one sweep still brings x back to its input state
    const int sweeps = c->n_params > 0 ? 2 : 1;
    for (int im = 0; im < sweeps; ++im) {
      if (im == 1) QS_CUDA(cudaMemcpyAsync(x->ptr, x->save, bytes, cudaMemcpyDeviceToDevice, st));
      QS_TRY(launch_ham_apply(psi->dt, other, lam->ptr, ne, h->d_groups, h->n_groups, h->d_terms, d_hpart, hgrid, st));
      if (im == 1) QS_TRY(launch_gate_diag(psi->dt, lam->ptr, ne, 1, &t0, 0, times_i, st));
      QS_TRY(run_passes(P.rev, 0, (int)P.rev.passes.size(), psi->dt, x->ptr, lam->ptr, P.d_coef, nullptr, d_part, ne,
                        0, P.grid1, P.grid2, st));
      const int ns = (int)P.rev_slots.out.size();
      if (c->n_params == 0 || ns == 0) continue;
      QS_TRY(launch_reduce_slots(d_part, ns, P.grid2, nullptr, d_slot, st));
      QS_TRY(launch_param_gather(d_slot, P.d_row, P.d_sidx, P.d_w, c->n_params, d_g + (size_t)(2 * side + im) * npp,
                                 st));
    }
  }
  double E[2];
  std::vector<double> g(4 * (size_t)npp);
  QS_CUDA(cudaMemcpyAsync(E, d_E, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
  QS_CUDA(cudaMemcpyAsync(g.data(), d_g, g.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  QS_CUDA(cudaStreamSynchronize(st));
  energy2[0] = E[0];
  energy2[1] = E[1];
  if (grad2)
    for (int p = 0; p < n_params; ++p) {
      const bool in = p < np;
      grad2[2 * p] = in ? 0.5 * (g[p] + g[2 * (size_t)npp + p]) : 0.0;
      grad2[2 * p + 1] = in ? 0.5 * (g[(size_t)npp + p] - g[3 * (size_t)npp + p]) : 0.0;
    }
  return QS_OK;
}

qs_status qs_measure(qs_state* s, int qubit, uint64_t seed, int* outcome) {
  QS_TRY(check_state(s));
  QS_CHECK(qubit >= 0 && qubit < s->n, "qubit out of range");
  QS_CHECK(outcome != nullptr, "outcome is null");
  const uint64_t N = 1ull << s->ne;
  const int nb = (int)std::min<uint64_t>(std::max<uint64_t>((N + 255) / 256, 1), 1024);
  QS_TRY(ensure_scratch(s, 2 * (size_t)nb + 2));
  QS_TRY(launch_measure(s->dt, s->ptr, s->ne, qubit, seed, s->scratch, nb, s->st));
  double o = 0.0;
  QS_CUDA(cudaMemcpyAsync(&o, s->scratch + 2 * nb, sizeof(double), cudaMemcpyDeviceToHost, s->st));
  QS_CUDA(cudaStreamSynchronize(s->st));
  *outcome = (int)o;
  return QS_OK;
}

qs_status qs_circuit_autotune(qs_circuit* c, qs_state* s, const double* params, int n_params, int reps,
                              qs_options* chosen, double* best_ms) {
  QS_TRY(check_state(s));
  QS_CHECK(c != nullptr, "null circuit");
  QS_CHECK(c->n == s->n, "circuit and state differ in qubit count");
  QS_CHECK(n_params >= c->n_params && (c->n_params == 0 || params != nullptr), "too few parameters");
  QS_CHECK(reps >= 1 && reps <= 100, "reps must be 1..100");
  const int ne = std::max(c->n, kRegBits);
  const int mmax = std::min(max_tile_bits(s->dt), ne);
  std::vector<std::pair<int, int>> cand;  // (tile bits, low bits)
  for (int m = mmax; m >= std::max(kMinTileBits, mmax - 2); --m)
    for (int lb = 2; lb <= 5; ++lb)
      if (lb < m) cand.push_back({m, lb});
  if (cand.empty()) cand.push_back({mmax, std::max(1, std::min(4, mmax))});
  cudaEvent_t e0, e1;
  QS_CUDA(cudaEventCreate(&e0));
  QS_CUDA(cudaEventCreate(&e1));
  const qs_options saved = c->opts;
  double best = 1e300;
  qs_options bo = saved;
  qs_status st = QS_OK;
  for (const auto& mc : cand) {
    qs_options o = saved;
    o.fuse = 1;
    o.tile_bits = mc.first;
    o.low_bits = mc.second;
    c->opts = o;
    if ((st = finalize_plan(c, s->dt, s->st)) != QS_OK) break;
    if ((st = qs_apply_circuit(s, c, params, n_params)) != QS_OK) break;  // warm-up (uploads the plan's tables)
    if (cudaEventRecord(e0, s->st) != cudaSuccess) { st = QS_ERR_CUDA; break; }
    for (int r = 0; r < reps && st == QS_OK; ++r) st = qs_apply_circuit(s, c, params, n_params);
    if (st != QS_OK) break;
    float ms = 0.f;
    if (cudaEventRecord(e1, s->st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      st = QS_ERR_CUDA;
      break;
    }
    if (ms / reps < best) {
      best = ms / reps;
      bo = o;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->opts = st == QS_OK ? bo : saved;
  qs_status s2 = finalize_plan(c, s->dt, s->st);
  if (st != QS_OK) return st;
  if (s2 != QS_OK) return s2;
  if (chosen) *chosen = bo;
  if (best_ms) *best_ms = best;
  return QS_OK;
}

qs_status qs_trace_enable(int enable) { return trace_enable(enable); }

qs_status qs_trace_read(int max, int* n, double* ms, double* bytes, int* kinds) {
  QS_CHECK(n != nullptr, "n is null");
  return trace_read(max, n, ms, bytes, kinds);
}

qs_status qs_sample(const qs_state* s_, uint64_t shots, uint64_t seed, uint64_t* out_bits) {
  QS_TRY(check_state(s_));
  QS_CHECK(shots == 0 || out_bits != nullptr, "out_bits is null");
  QS_CHECK(shots <= (1ull << 31), "at most 2^31 shots per call");
  qs_state* s = const_cast<qs_state*>(s_);
  const size_t nd = sample_scratch_doubles(s->ne);
  QS_TRY(ensure_scratch(s, nd + shots + 8));
  uint64_t* d_out = reinterpret_cast<uint64_t*>(s->scratch + nd + 1);
  QS_TRY(launch_sample(s->dt, s->ptr, s->ne, shots, seed, s->scratch, d_out, s->st));
  if (shots) QS_CUDA(cudaMemcpyAsync(out_bits, d_out, shots * sizeof(uint64_t), cudaMemcpyDeviceToHost, s->st));
  QS_CUDA(cudaStreamSynchronize(s->st));
  return QS_OK;
}

}  // extern "C"
