// Host planner of the complex64 QAOA passes with separate forward and reverse
// tile shapes (kernels in k_qaoa_x.cu).
//
// The evaluation (§5.2 ansatz, energy and adjoint gradient as in §6.2's QuPack
// interface) is a sequence of operations on the state:
//   forward:  COST(0) MIX(0) COST(1) MIX(1) ... COST(p-1) MIX(p-1)
//   turnaround: E = <C>, lam = C psi, then the reverse starts
//   reverse:  MIX(p-1)^dag COST(p-1)^dag ... MIX(0)^dag COST(0)^dag, taking
//             dE/dbeta_l = sum_q Im <lam|X_q|psi> inside MIX(l) and
//             dE/dgamma_l = 2 gs Im <lam|C|psi> between MIX(l) and COST(l),
// where MIX(l) = RX(beta_l) on every qubit and COST(l) = exp(-i gs gamma_l C).
// A pass covers a tile bit set S (the low c qubits plus m - c others): it
// applies MIX to the bits of S still pending in the current layer and, when that
// completes the layer, the next COST and the next MIX on every bit of S.  With
// the non-low qubits split into g groups of at most m - c bits, a layer costs
// g - 1 passes (two for 30 qubits).
//
// DRAM: a tile is a gather of runs of 2^c contiguous amplitudes.  128-byte runs
// whose tile also holds a qubit of small address stride (<= 16 KB) stream at
// 6.0-6.4 TB/s on GB300, while tiles whose other qubits are all high ones fall
// to 4.8 TB/s; so the small-stride qubits are dealt round-robin to the groups.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>

#include "plan.h"
#include "qaoa_pass.h"
#include "qaoa_x.h"
#include "qaoa_x_plan.h"
#include "tma.h"

namespace qs {

namespace {

inline int popc(uint64_t x) { return __builtin_popcountll(x); }

// Non-low qubits c..n-1 split into groups of at most m - c, the small-stride
// qubits (2^q * elem_bytes <= 16 KB) dealt round-robin, the rest in blocks.
std::vector<uint64_t> make_groups(int n, int m, int c, int elem_bytes) {
  const int k = m - c;
  const int g = std::max(1, (n - c + k - 1) / k);
  std::vector<uint64_t> grp(g, 0);
  std::vector<int> small, big;
  for (int q = c; q < n; ++q) ((((uint64_t)1 << q) * (uint64_t)elem_bytes <= 16384ull) ? small : big).push_back(q);
  std::vector<int> cap(g, 0);
  for (int i = 0; i < g; ++i) cap[i] = (n - c) / g + (i < (n - c) % g ? 1 : 0);
  int gi = 0;
  for (int q : small) {
    for (int t = 0; t < g && popc(grp[gi]) >= cap[gi]; ++t) gi = (gi + 1) % g;
    grp[gi] |= 1ull << q;
    gi = (gi + 1) % g;
  }
  int b = 0;
  for (int i = 0; i < g; ++i)
    while (popc(grp[i]) < cap[i] && b < (int)big.size()) grp[i] |= 1ull << big[b++];
  return grp;
}

// Up to k bits of `rem`, whole groups first (in group order).
uint64_t pick(uint64_t rem, int k, const std::vector<uint64_t>& groups) {
  uint64_t T = 0;
  for (uint64_t gmask : groups)
    for (int q = 0; q < 64 && popc(T) < k; ++q)
      if (((gmask & rem) >> q) & 1) T |= 1ull << q;
  for (int q = 0; q < 64 && popc(T) < k; ++q)
    if ((rem >> q) & 1) T |= 1ull << q;
  return T;
}

// X plus the lowest other qubits up to m.
uint64_t fill(uint64_t X, int n, int m) {
  for (int q = 0; q < n && popc(X) < m; ++q) X |= 1ull << q;
  return X;
}

}  // namespace

// ---------------------------------------------------------------------------- sweeps

std::vector<XSched> qx_forward_schedule(int n, int p, int m, int c, int elem_bytes) {
  const uint64_t all = (n >= 64) ? ~0ull : ((1ull << n) - 1);
  const uint64_t low = (1ull << c) - 1;
  const std::vector<uint64_t> groups = make_groups(n, m, c, elem_bytes);
  std::vector<XSched> out;
  uint64_t S = fill(low | groups[0], n, m);
  out.push_back({S, 0, -1, XD_COST, 0, S, 0});
  uint64_t rem = all & ~S;
  int layer = 0;
  while (true) {
    if (popc(rem | low) <= m) {
      S = fill(rem | low, n, m);
      XSched x{S, rem, layer, XD_NONE, -1, 0, -1};
      if (layer + 1 < p) {
        x.diag = XD_COST;
        x.ld = layer + 1;
        x.set3 = S;
        x.l3 = layer + 1;
        rem = all & ~S;
        ++layer;
        out.push_back(x);
      } else {
        out.push_back(x);
        break;
      }
    } else {
      const uint64_t T = pick(rem & ~low, m - c, groups);
      const uint64_t set1 = T | (rem & low);
      out.push_back({low | T, set1, layer, XD_NONE, -1, 0, -1});
      rem &= ~set1;
    }
  }
  return out;
}

std::vector<XSched> qx_reverse_schedule(int n, int p, int m, int c, uint64_t rem0, int elem_bytes) {
  const uint64_t all = (n >= 64) ? ~0ull : ((1ull << n) - 1);
  const uint64_t low = (1ull << c) - 1;
  const std::vector<uint64_t> groups = make_groups(n, m, c, elem_bytes);
  std::vector<XSched> out;
  uint64_t rem = rem0;
  int layer = p - 1;
  while (true) {
    if (popc(rem | low) <= m) {
      const uint64_t S = fill(rem | low, n, m);
      XSched x{S, rem, layer, XD_COST_GRAD, layer, 0, -1};
      if (layer > 0) {
        x.set3 = S;
        x.l3 = layer - 1;
        rem = all & ~S;
        --layer;
        out.push_back(x);
      } else {
        out.push_back(x);
        break;
      }
    } else {
      const uint64_t T = pick(rem & ~low, m - c, groups);
      const uint64_t set1 = T | (rem & low);
      out.push_back({low | T, set1, layer, XD_NONE, -1, 0, -1});
      rem &= ~set1;
    }
  }
  return out;
}

// ---------------------------------------------------------------------------- phases

namespace {

// Tiles sit in shared memory unswizzled (a copy of the gathered HBM runs), so
// the bank column of an element is its low local bits: 3 bits for 16-byte
// elements (8 per 128-byte row, the lanes of a quarter-warp), 4 for 8-byte ones
// (a half-warp).  Lane order: the column bits among the sub-cube bits first
// (lanes then also touch contiguous addresses), then the rest.  Column bits
// held in registers are covered by the next lanes, which XOR-relabel the
// thread's register index (see the kernel).
std::vector<int> lane_order(const std::vector<int>& rest, int ncol) {
  std::vector<int> q;
  for (int b : rest)
    if (b < ncol) q.push_back(b);
  for (int b : rest)
    if (b >= ncol) q.push_back(b);
  return q;
}

struct PhasePlan {
  std::vector<int> reg;  // R local bits
  uint8_t m1 = 0, m3 = 0;
  uint8_t diag = XD_NONE;
};

// Register bits for a group of op bits, padded to R with bits that carry no op
// (non-low bits first, so the low bits stay lane bits).
std::vector<int> pad_reg(std::vector<int> bits, int m, int c, size_t R) {
  for (int b = m - 1; b >= c && bits.size() < R; --b)
    if (std::find(bits.begin(), bits.end(), b) == bits.end()) bits.push_back(b);
  for (int b = 0; b < c && bits.size() < R; ++b)
    if (std::find(bits.begin(), bits.end(), b) == bits.end()) bits.push_back(b);
  return bits;
}

std::vector<PhasePlan> plan_phases(int m, int c, uint32_t A, int diag, uint32_t B, size_t R) {
  auto bits_of = [&](uint32_t mask, bool low_first) {
    std::vector<int> v, lo;
    for (int b = 0; b < m; ++b)
      if ((mask >> b) & 1) (b < c ? lo : v).push_back(b);
    if (low_first) {
      lo.insert(lo.end(), v.begin(), v.end());
      return lo;
    }
    v.insert(v.end(), lo.begin(), lo.end());
    return v;
  };
  std::vector<PhasePlan> out;
  auto add = [&](const std::vector<int>& ops_bits, bool step1, bool step3, const std::vector<int>& ops3) {
    PhasePlan pp;
    pp.reg = pad_reg(ops_bits, m, c, R);
    for (size_t r = 0; r < pp.reg.size(); ++r) {
      if (step1 && std::find(ops_bits.begin(), ops_bits.end(), pp.reg[r]) != ops_bits.end()) pp.m1 |= 1u << r;
      if (step3 && std::find(ops3.begin(), ops3.end(), pp.reg[r]) != ops3.end()) pp.m3 |= 1u << r;
    }
    out.push_back(pp);
  };
  if (diag == XD_NONE) {
    // step 1 only; low bits first so the last phase keeps them as lane bits
    const std::vector<int> a = bits_of(A, true);
    for (size_t i = 0; i < a.size(); i += R) {
      std::vector<int> g(a.begin() + i, a.begin() + std::min(a.size(), i + R));
      add(g, true, false, {});
    }
    if (out.empty()) add({}, false, false, {});
    return out;
  }
  // before the diagonal: step-1 bits in groups of 4, the remainder goes to the diagonal phase
  const std::vector<int> a = bits_of(A, true);
  const size_t kA = std::max<size_t>(1, (a.size() + R - 1) / R);
  for (size_t i = 0; i + 1 < kA; ++i) add(std::vector<int>(a.begin() + R * i, a.begin() + R * i + R), true, false, {});
  std::vector<int> d(a.begin() + std::min(a.size(), R * (kA - 1)), a.end());
  const std::vector<int> d1 = d;  // bits that still take step 1 in the diagonal phase
  // fill the diagonal phase with step-3 bits: the low ones first (they then take
  // their step 3 here and stay lane bits in the last phase)
  for (int b : bits_of(B, true))
    if (d.size() < R && std::find(d.begin(), d.end(), b) == d.end()) d.push_back(b);
  {
    PhasePlan pp;
    pp.reg = pad_reg(d, m, c, R);
    pp.diag = (uint8_t)diag;
    for (size_t r = 0; r < pp.reg.size(); ++r) {
      if (std::find(d1.begin(), d1.end(), pp.reg[r]) != d1.end()) pp.m1 |= 1u << r;
      if ((B >> pp.reg[r]) & 1) pp.m3 |= 1u << r;
    }
    out.push_back(pp);
  }
  // after the diagonal: the remaining step-3 bits, low ones first
  uint32_t rest = B;
  for (int b : out.back().reg) rest &= ~(1u << b);
  const std::vector<int> r3 = bits_of(rest, true);
  for (size_t i = 0; i < r3.size(); i += R) {
    std::vector<int> g(r3.begin() + i, r3.begin() + std::min(r3.size(), i + R));
    add(g, false, true, g);
  }
  return out;
}

// In-tile edge counts fs[l] for the edges with both ends in S (local indices).
void edge_table(int m, const std::vector<std::pair<int, int>>& loc_edges, std::vector<uint8_t>* fs) {
  const uint32_t N = 1u << m;
  const size_t base = fs->size();
  fs->resize(base + N, 0);
  for (uint32_t l = 0; l < N; ++l) {
    int k = 0;
    for (const auto& e : loc_edges) k += (int)(((l >> e.first) ^ (l >> e.second)) & 1u);
    (*fs)[base + l] = (uint8_t)k;
  }
}

}  // namespace

bool qx_map_dims(uint64_t S, int n, int e, int m, uint8_t a[5], uint8_t w[5], uint8_t bx[5], uint8_t* lb) {
  TileMapDims d;
  if (!tile_map_dims(S, n, e, m, 1, 8, 128, &d)) return false;
  for (int i = 0; i < 5; ++i) {
    a[i] = d.a[i];
    w[i] = d.w[i];
    bx[i] = d.bx[i];
  }
  *lb = d.lb;
  return true;
}

qs_status qx_build_pass(const XBuild& B, const XSched& s, bool two_state, uint32_t flags, int out_slots[3],
                        XPass* out, std::vector<uint8_t>* fs) {
  XPass P;
  std::memset(&P, 0, sizeof(P));
  const int m = two_state ? B.mr : B.mf, c = two_state ? B.cr : B.cf;
  if (popc(s.S) != m || (s.S & ((1ull << c) - 1)) != ((1ull << c) - 1)) {
    set_error("qaoa planner: malformed tile bit set (internal error)");
    return QS_ERR_UNSUPPORTED;
  }
  P.m = m;
  P.c = c;
  P.flags = flags;
  int local_of[64], global_of[kXMaxM], k = 0;
  for (int q = 0; q < 64; ++q) local_of[q] = -1;
  for (int q = 0; q < B.n; ++q)
    if ((s.S >> q) & 1) {
      local_of[q] = k;
      global_of[k++] = q;
    } else {
      P.comp[P.ncomp++] = (int8_t)q;
    }
  for (int i = 0; i < 64; ++i) {
    uint64_t a = 0, b = 0;
    for (int j = 0; j < 6; ++j)
      if ((i >> j) & 1) {
        if (c + j < m) a |= 1ull << global_of[c + j];
        if (c + 6 + j < m) b |= 1ull << global_of[c + 6 + j];
      }
    P.hiA[i] = a;
    P.hiB[i] = b;
  }
  auto local_mask = [&](uint64_t g) {
    uint32_t l = 0;
    for (int q = 0; q < B.n; ++q)
      if ((g >> q) & 1) {
        if (local_of[q] < 0) return 0xffffffffu;
        l |= 1u << local_of[q];
      }
    return l;
  };
  const uint32_t A = local_mask(s.set1), Bm = local_mask(s.set3);
  if (A == 0xffffffffu || Bm == 0xffffffffu) {
    set_error("qaoa planner: mixer bits outside the tile (internal error)");
    return QS_ERR_UNSUPPORTED;
  }
  const int R = qx_reg_bits(two_state);
  const std::vector<PhasePlan> phs = plan_phases(m, c, A, s.diag, Bm, (size_t)R);
  if ((int)phs.size() > kXMaxPhases) {
    set_error("qaoa planner: too many phases (internal error)");
    return QS_ERR_UNSUPPORTED;
  }
  // every phase must have a compiled body in its kernel (k_qaoa_x.cu): steps on
  // a prefix of the register bits, k1 + diag + k3 combinations below
  for (size_t i = 0; i < phs.size(); ++i) {
    const int k1 = popc(phs[i].m1), k3 = popc(phs[i].m3), dg = phs[i].diag;
    const bool prefix = phs[i].m1 == (1u << k1) - 1 && phs[i].m3 == (1u << k3) - 1;
    bool ok;
    if (dg == XD_NONE) ok = (k1 > 0) != (k3 > 0);
    else if (!two_state) ok = (dg == XD_COST && k3 == R) || (dg == XD_ENERGY && k3 == 0);
    else ok = (dg == XD_COST_GRAD && (k3 == R || k3 == 0)) || (dg == XD_ENERGY && k3 == R);
    if (!prefix || !ok) {
      set_error("qaoa planner: a phase without a kernel body (internal error)");
      return QS_ERR_UNSUPPORTED;
    }
  }
  const bool el8 = !two_state;  // 8-byte elements (psi alone) or 16-byte (psi/lam)
  P.n_phases = (int)phs.size();
  for (int i = 0; i < P.n_phases; ++i) {
    XPhase& X = P.ph[i];
    uint32_t regmask = 0;
    for (int r = 0; r < 4; ++r) {  // unused register slots (R = 3): no bit
      if (r >= R) {
        X.lbit[r] = 0;
        X.gbit[r] = 0;
        continue;
      }
      X.lbit[r] = (uint16_t)(1u << phs[i].reg[r]);
      X.gbit[r] = 1ull << global_of[phs[i].reg[r]];
      regmask |= 1u << phs[i].reg[r];
    }
    std::vector<int> rest;
    for (int b = 0; b < m; ++b)
      if (!((regmask >> b) & 1)) rest.push_back(b);
    const int ncol = el8 ? 4 : 3;
    const std::vector<int> q = lane_order(rest, ncol);
    X.nq = (uint8_t)q.size();
    for (size_t t = 0; t < q.size(); ++t) X.q[t] = (int8_t)q[t];
    // register bits that are column bits: relabelled by the lanes after the
    // column lanes, so the first 2^ncol lanes still hit 2^ncol columns
    X.kq = 0;
    while (X.kq < X.nq && X.q[X.kq] < ncol) ++X.kq;
    X.kn = 0;
    for (int r = 0; r < R; ++r)
      if (phs[i].reg[r] < ncol) X.kidx[X.kn++] = (uint8_t)r;
    if (X.kq + X.kn != ncol || X.kq + X.kn > X.nq) {
      set_error("qaoa planner: bank-column lanes do not cover the columns (internal error)");
      return QS_ERR_UNSUPPORTED;
    }
    X.m1 = phs[i].m1;
    X.m3 = phs[i].m3;
    X.diag = phs[i].diag;
  }
  // tensor maps: loads of psi (8-byte words) or of the interleaved pair (two
  // words per amplitude), stores to the interleaved pair in the two-state kernel
  {
    const int e_ld = two_state && !(flags & XF_LOAD_PSI) ? 1 : 0, e_st = two_state ? 1 : 0;
    if (!qx_map_dims(s.S, B.n, e_ld, m, P.ma[0], P.mw[0], P.mbx[0], &P.mlb[0]) ||
        !qx_map_dims(s.S, B.n, e_st, m, P.ma[1], P.mw[1], P.mbx[1], &P.mlb[1])) {
      set_error("qaoa planner: the tile does not map onto a five-dimensional copy");
      return QS_ERR_UNSUPPORTED;
    }
    P.me[0] = (uint8_t)e_ld;
    P.me[1] = (uint8_t)e_st;
  }
  // coefficients: per layer lut[E+1], lut_dag[E+1], rx (c, s), rx_dag (c, -s)
  const int E1 = B.n_edges + 1, per_layer = 2 * E1 + 2;
  const bool rev = s.diag == XD_COST_GRAD;
  P.c1 = s.l1 >= 0 ? s.l1 * per_layer + 2 * E1 + (rev || (flags & XF_GRAD1) ? 1 : 0) : -1;
  P.c3 = s.l3 >= 0 ? s.l3 * per_layer + 2 * E1 + (rev || (flags & XF_GRAD3) ? 1 : 0) : -1;
  P.cd = (s.diag == XD_COST) ? s.ld * per_layer : (s.diag == XD_COST_GRAD) ? s.ld * per_layer + E1 : -1;
  for (int i = 0; i < 3; ++i) P.slot[i] = out_slots[i];
  // edges: in-tile table, crossing masks, complement-complement masks
  P.fs_off = -1;
  if (s.diag != XD_NONE) {
    std::vector<std::pair<int, int>> loc;
    for (int i = 0; i < kXMaxM; ++i) P.wmask[i] = 0;
    std::vector<uint64_t> cc(B.n, 0);
    for (const auto& e : B.edges) {
      const int la = local_of[e.first], lb = local_of[e.second];
      if (la >= 0 && lb >= 0) {
        loc.push_back({la, lb});
      } else if (la >= 0) {
        P.wmask[la] |= 1ull << e.second;
      } else if (lb >= 0) {
        P.wmask[lb] |= 1ull << e.first;
      } else {
        const int lo = std::min(e.first, e.second), hi = std::max(e.first, e.second);
        cc[lo] |= 1ull << hi;
      }
    }
    for (int a = 0; a < B.n; ++a)
      if (cc[a]) {
        if (P.n_cc >= kXMaxComp) {
          set_error("qaoa planner: too many complement nodes (internal error)");
          return QS_ERR_UNSUPPORTED;
        }
        P.ccnode[P.n_cc] = (uint8_t)a;
        P.ccmask[P.n_cc++] = cc[a];
      }
    P.fs_off = (int)fs->size();
    edge_table(m, loc, fs);
  }
  *out = P;
  return QS_OK;
}

qs_status qx_make_plans(const XBuild& B, double gs, XPlans* X) {
  const int n = B.n, p = B.p, mr = B.mr, cr = B.cr, mf = B.mf, cf = B.cf;
  if (n <= mf || mr < 9 || mr > 12 || cr < 2 || cr > mr - 4 || mf != mr + 1 || cf != cr + 1 || p < 1) {
    set_error("qaoa planner: unsupported two-shape tile (internal error)");
    return QS_ERR_UNSUPPORTED;
  }
  const uint64_t all = (1ull << n) - 1, lowr = (1ull << cr) - 1;
  const std::vector<XSched> fw = qx_forward_schedule(n, p, mf, cf, 8);
  if (fw.size() < 2) {
    set_error("qaoa planner: a single forward pass (internal error)");
    return QS_ERR_UNSUPPORTED;
  }
  auto slot = [](SlotMap& sm, int o, double w) {
    sm.out.push_back(o);
    sm.weight.push_back(w);
    return (int)sm.out.size() - 1;
  };
  int none[3] = {-1, -1, -1};
  XPass P;
  // gradient plan: forward passes, the turnaround (last forward pass, E and
  // lam = C psi, its own mixer bits undone), the reverse passes
  for (size_t i = 0; i + 1 < fw.size(); ++i) {
    QS_TRY(qx_build_pass(B, fw[i], false, (i == 0 ? XF_GEN_PLUS : 0u) | XF_STORE, none, &P, &X->fs));
    X->grad.push_back(P);
    X->grad_two.push_back(0);
  }
  const uint64_t rl = fw.back().set1;
  if (popc(rl | lowr) > mr) {
    set_error("qaoa planner: the turnaround does not fit the reverse tile (internal error)");
    return QS_ERR_UNSUPPORTED;
  }
  // the turnaround undoes the last mixer on every qubit of its tile (all of them
  // carry it by then), not only on the ones it applied
  const uint64_t St = fill(rl | lowr, n, mr);
  {
    const XSched t{St, rl, p - 1, XD_ENERGY, p - 1, St, p - 1};
    int ts[3] = {-1, slot(X->gslots, 0, 1.0), slot(X->gslots, 1 + p + (p - 1), 1.0)};
    QS_TRY(qx_build_pass(B, t, true, XF_LOAD_PSI | XF_STORE | XF_GRAD3, ts, &P, &X->fs));
    X->grad.push_back(P);
    X->grad_two.push_back(1);
  }
  const std::vector<XSched> rv = qx_reverse_schedule(n, p, mr, cr, all & ~St, 16);
  for (size_t i = 0; i < rv.size(); ++i) {
    const XSched& r = rv[i];
    int rs[3] = {r.set1 ? slot(X->gslots, 1 + p + r.l1, 1.0) : -1,
                 r.diag == XD_COST_GRAD ? slot(X->gslots, 1 + r.ld, 2.0 * gs) : -1,
                 r.set3 ? slot(X->gslots, 1 + p + r.l3, 1.0) : -1};
    const uint32_t fl = XF_GRAD1 | XF_GRAD3 | (i + 1 < rv.size() ? XF_STORE : 0u);
    QS_TRY(qx_build_pass(B, r, true, fl, rs, &P, &X->fs));
    X->grad.push_back(P);
    X->grad_two.push_back(1);
  }
  // energy plan: the forward passes, the energy taken in the last
  for (size_t i = 0; i < fw.size(); ++i) {
    XSched e = fw[i];
    int sl[3] = {-1, -1, -1};
    if (i + 1 == fw.size()) {
      e.diag = XD_ENERGY;
      e.ld = p - 1;
      sl[1] = slot(X->eslots, 0, 1.0);
    }
    QS_TRY(qx_build_pass(B, e, false, (i == 0 ? XF_GEN_PLUS : 0u) | XF_STORE, sl, &P, &X->fs));
    X->energy.push_back(P);
    X->energy_two.push_back(0);
  }
  if (X->fs.empty()) X->fs.assign(16, 0);
  {  // phase-weight blocks after the per-layer coefficients
    const int per_layer = 2 * (B.n_edges + 1) + 2;
    int off = p * per_layer;
    for (XPass& P : X->grad) {
      P.cw = off;
      off += 2 * kXMaxPhases;
    }
    for (XPass& P : X->energy) {
      P.cw = off;
      off += 2 * kXMaxPhases;
    }
    X->n_coef = off;
  }
  const double S = 8.0 * (double)(1ull << n);
  X->bytes_grad = S + 2 * S * (double)(fw.size() - 2) + 3 * S + 4 * S * (double)(rv.size() - 1) + 2 * S;
  X->bytes_energy = S + 2 * S * (double)(fw.size() - 1);
  X->n_fwd = (int)fw.size();
  X->n_rev = (int)rv.size();
  return QS_OK;
}

qs_status qx_fill_coef(int n, int p, int n_edges, double gs, const double* gamma, const double* beta,
                       const std::vector<XPass>& grad, const std::vector<XPass>& energy, int n_coef,
                       std::vector<double>* tab, bool* flip) {
  using cd = std::complex<double>;
  const int E1 = n_edges + 1, per_layer = 2 * E1 + 2;
  tab->assign((size_t)2 * n_coef, 0.0);
  auto put = [&](int o, cd v) {
    (*tab)[2 * (size_t)o] = v.real();
    (*tab)[2 * (size_t)o + 1] = v.imag();
  };
  // scaled mixer of layer l, direction d (0: RX(beta), 1: RX(-beta)): t and the factor g
  std::vector<double> tt(2 * p);
  std::vector<cd> gg(2 * p);
  std::vector<char> form_b(p);
  for (int l = 0; l < p; ++l) {
    const double c = std::cos(0.5 * beta[l]), s0 = std::sin(0.5 * beta[l]);
    form_b[l] = std::fabs(s0) > std::fabs(c);
    for (int d = 0; d < 2; ++d) {
      const double sd = d == 0 ? s0 : -s0;
      if (!form_b[l]) {
        tt[2 * l + d] = sd / c;
        gg[2 * l + d] = cd(1.0 / c, 0.0);
      } else {
        tt[2 * l + d] = -c / sd;
        gg[2 * l + d] = cd(0.0, 1.0 / sd);
      }
      put(l * per_layer + 2 * E1 + d, cd(tt[2 * l + d], 0.0));
    }
  }
  // renormalisation of each cost LUT (forward: index l, reverse: p + l), set where first met
  std::vector<cd> rho(2 * p, cd(0, 0));
  std::vector<char> have(2 * p, 0);
  auto ipow = [](cd g, int k) {
    cd r(1, 0);
    for (int i = 0; i < k; ++i) r *= g;
    return r;
  };
  auto step = [&](int off) -> int {  // coefficient offset -> 2 l + d
    const int l = off / per_layer, d = off % per_layer - 2 * E1;
    return 2 * l + d;
  };
  auto simulate = [&](const std::vector<XPass>& plan) {
    cd sigma(1, 0);
    for (const XPass& P : plan) {
      for (int ph = 0; ph < P.n_phases; ++ph) {
        const XPhase& X = P.ph[ph];
        const int k1 = __builtin_popcount(X.m1), k3 = __builtin_popcount(X.m3);
        const double w1 = 1.0 / std::norm(sigma);
        if (k1) sigma *= ipow(gg[step(P.c1)], k1);
        const double wd = 1.0 / std::norm(sigma);
        if (X.diag == XD_COST || X.diag == XD_COST_GRAD) {
          const int l = P.cd / per_layer, rev = X.diag == XD_COST_GRAD;
          const int key = rev * p + l;
          if (!have[key]) {
            if (!rev && l == p - 1)  // the state leaves the last mixer exactly
              rho[key] = 1.0 / (sigma * ipow(gg[2 * l], n));
            else
              rho[key] = 1.0 / std::abs(sigma);
            have[key] = 1;
          }
          sigma *= rho[key];
        }
        const double w3 = 1.0 / std::norm(sigma);
        if (k3) sigma *= ipow(gg[step(P.c3)], k3);
        put(P.cw + 2 * ph, cd(w1, w3));
        put(P.cw + 2 * ph + 1, cd(wd, 0.0));
      }
    }
    return sigma;
  };
  simulate(grad);
  const cd s_end = simulate(energy);
  if (std::abs(s_end - cd(1, 0)) > 1e-6) {
    set_error("qaoa: scaled-mixer bookkeeping does not close (internal error)");
    return QS_ERR_UNSUPPORTED;
  }
  for (int l = 0; l < p; ++l) {
    const cd rf = have[l] ? rho[l] : cd(1, 0), rr = have[p + l] ? rho[p + l] : cd(1, 0);
    for (int k = 0; k <= n_edges; ++k) {
      const double ph = gs * gamma[l] * (double)(n_edges - 2 * k);
      put(l * per_layer + k, cd(std::cos(ph), -std::sin(ph)) * rf);
      put(l * per_layer + E1 + k, cd(std::cos(ph), std::sin(ph)) * rr);
    }
  }
  int nb = 0;
  for (int l = 0; l < p; ++l) nb += form_b[l];
  *flip = (nb & 1) != 0;
  return QS_OK;
}

}  // namespace qs

// ---------------------------------------------------------------------------- inspection

using namespace qs;

extern "C" qs_status qs_qaoa_xplan(int n_qubits, const int* edges, int n_edges, int p, double gamma_scale,
                                   int tile_bits, int low_bits, int which, long long* rec, int max_passes,
                                   int* n_passes, int* slot_out, double* slot_w, int max_slots, int* n_slots) {
  QS_CHECK(edges != nullptr && n_edges >= 1 && n_edges <= 255, "need 1..255 edges");
  QS_CHECK(n_qubits >= 10 && n_qubits <= kMaxQubits, "n_qubits must be in 10..34");
  QS_CHECK(rec && n_passes && slot_out && slot_w && n_slots, "null output");
  XBuild B;
  B.n = n_qubits;
  B.p = p;
  B.mr = tile_bits ? tile_bits : 12;
  B.cr = low_bits ? low_bits : 3;
  B.mf = B.mr + 1;
  B.cf = B.cr + 1;
  B.n_edges = n_edges;
  for (int e = 0; e < n_edges; ++e) {
    const int a = edges[2 * e], b = edges[2 * e + 1];
    QS_CHECK(a >= 0 && a < n_qubits && b >= 0 && b < n_qubits && a != b, "edge endpoint out of range");
    B.edges.push_back({std::min(a, b), std::max(a, b)});
  }
  XPlans X;
  QS_TRY(qx_make_plans(B, gamma_scale, &X));
  const std::vector<XPass>& pl = which ? X.energy : X.grad;
  const std::vector<int>& two = which ? X.energy_two : X.grad_two;
  const SlotMap& sm = which ? X.eslots : X.gslots;
  QS_CHECK((int)pl.size() <= max_passes && (int)sm.out.size() <= max_slots, "output arrays too small");
  *n_passes = (int)pl.size();
  *n_slots = (int)sm.out.size();
  for (size_t i = 0; i < sm.out.size(); ++i) {
    slot_out[i] = sm.out[i];
    slot_w[i] = sm.weight[i];
  }
  for (size_t i = 0; i < pl.size(); ++i) {
    const XPass& P = pl[i];
    long long* r = rec + i * QS_XPLAN_REC;
    uint64_t S = 0;
    int gl[kXMaxM];
    for (int l = 0; l < P.m; ++l) {
      const uint64_t g = l < P.c ? (1ull << l) : (l < P.c + 6 ? P.hiA[1 << (l - P.c)] : P.hiB[1 << (l - P.c - 6)]);
      S |= g;
      gl[l] = __builtin_ctzll(g);
    }
    r[0] = two[i];
    r[1] = P.flags;
    r[2] = (long long)S;
    r[3] = P.n_phases;
    r[4] = P.c1;
    r[5] = P.c3;
    r[6] = P.cd;
    r[7] = P.slot[0];
    r[8] = P.slot[1];
    r[9] = P.slot[2];
    r[10] = P.m;
    r[11] = P.c;
    for (int ph = 0; ph < P.n_phases; ++ph) {
      long long* q = r + 12 + 7 * ph;
      const XPhase& X2 = P.ph[ph];
      q[0] = X2.m1;
      q[1] = X2.m3;
      q[2] = X2.diag;
      for (int k = 0; k < 4; ++k) q[3 + k] = X2.lbit[k] ? gl[__builtin_ctz(X2.lbit[k])] : -1;
    }
    r[12 + 7 * kXMaxPhases + 34] = P.cw;
    for (int k = 0; k < 2; ++k) {
      long long* t = r + 12 + 7 * kXMaxPhases + 17 * k;
      t[0] = P.me[k];
      t[1] = P.mlb[k];
      for (int d = 0; d < 5; ++d) {
        t[2 + d] = P.ma[k][d];
        t[7 + d] = P.mw[k][d];
        t[12 + d] = P.mbx[k][d];
      }
    }
  }
  return QS_OK;
}

extern "C" qs_status qs_qaoa_xcoef(int n_qubits, const int* edges, int n_edges, int p, double gamma_scale,
                                   int tile_bits, int low_bits, const double* gamma, const double* beta,
                                   double* table, int max_entries, int* n_entries, int* flip) {
  QS_CHECK(edges != nullptr && n_edges >= 1 && n_edges <= 255, "need 1..255 edges");
  QS_CHECK(n_qubits >= 10 && n_qubits <= kMaxQubits, "n_qubits must be in 10..34");
  QS_CHECK(gamma && beta && table && n_entries && flip, "null argument");
  XBuild B;
  B.n = n_qubits;
  B.p = p;
  B.mr = tile_bits ? tile_bits : 12;
  B.cr = low_bits ? low_bits : 3;
  B.mf = B.mr + 1;
  B.cf = B.cr + 1;
  B.n_edges = n_edges;
  for (int e = 0; e < n_edges; ++e) {
    const int a = edges[2 * e], b = edges[2 * e + 1];
    QS_CHECK(a >= 0 && a < n_qubits && b >= 0 && b < n_qubits && a != b, "edge endpoint out of range");
    B.edges.push_back({std::min(a, b), std::max(a, b)});
  }
  XPlans X;
  QS_TRY(qx_make_plans(B, gamma_scale, &X));
  QS_CHECK(X.n_coef <= max_entries, "table too small");
  std::vector<double> tab;
  bool fl = false;
  QS_TRY(qx_fill_coef(n_qubits, p, n_edges, gamma_scale, gamma, beta, X.grad, X.energy, X.n_coef, &tab, &fl));
  for (size_t i = 0; i < tab.size(); ++i) table[i] = tab[i];
  *n_entries = X.n_coef;
  *flip = fl ? 1 : 0;
  return QS_OK;
}
