// Density-matrix simulation (§3.2) with quantum channels (§3.3) on the same
// fused tile engine as pure states.
//
// rho (2^n x 2^n) is stored as a state of 2n qubits: vec[x + 2^n y] = rho_{x,y}.
// Then rho -> U rho U^dag is U on the low n qubits and conj(U) on the high n
// qubits, and a channel sum_i K_i rho K_i^dag on qubit q is the 4x4
// superoperator S = sum_i K_i (x) conj(K_i) on qubits (q, q + n).  A
// density-matrix circuit is therefore an ordinary 2n-qubit circuit (gates
// doubled, channels as 2-qubit MATRIX gates) and runs on the same fused passes.
// tr(rho H) for a Pauli sum: for P = c i^{#Y} X^m Z^z, P|x> = c i^{#Y}
// (-1)^{|x & z|} |x ^ m>, so tr(rho P) = sum_x rho_{x, x^m} c i^{#Y} (-1)^{|x & z|}.
#include <cuda_runtime.h>

#include <cmath>
#include <complex>
#include <vector>

#include "handles.h"

using namespace qs;

namespace {

using cd = std::complex<double>;
constexpr int kDmThreads = 256;

template <class T>
struct DmV;
template <>
struct DmV<float> {
  using V = float2;
};
template <>
struct DmV<double> {
  using V = double2;
};

template <class T>
__global__ void dm_expect_kernel(const typename DmV<T>::V* __restrict__ vec, int n,
                                 const DevHamGroup* __restrict__ groups, int n_groups,
                                 const DevHamTerm* __restrict__ terms, double* partials) {
  __shared__ double sh[kDmThreads / 32];
  const uint64_t N = 1ull << n;
  double acc = 0.0;
  for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < N; x += (uint64_t)gridDim.x * blockDim.x) {
    for (int g = 0; g < n_groups; ++g) {
      const DevHamGroup G = groups[g];
      const typename DmV<T>::V r = vec[x | ((x ^ G.xmask) << n)];  // rho_{x, x^m}
      double fr = 0.0, fi = 0.0;
      for (int k = G.begin; k < G.end; ++k) {
        const DevHamTerm t = terms[k];
        const double s = (__popcll(x & t.zmask) & 1) ? -1.0 : 1.0;
        fr += s * t.re;
        fi += s * t.im;
      }
      acc += fr * (double)r.x - fi * (double)r.y;  // Re(f * rho_{x, x^m})
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kDmThreads / 32; ++w) s += sh[w];
    partials[blockIdx.x] = s;
  }
}

// conj(U) of a gate as (kind, coef, constant, matrix) on the bra register.
qs_status conj_gate(int kind, double coef, double constant, const double* matrix, int n_t, int* ck, double* cc,
                    double* cconst, std::vector<double>* cm) {
  *ck = kind;
  *cc = coef;
  *cconst = constant;
  cm->clear();
  switch (kind) {
    case QS_GATE_I:
    case QS_GATE_X:
    case QS_GATE_Z:
    case QS_GATE_H:
    case QS_GATE_SWAP:
    case QS_GATE_RY:  // real matrices
      break;
    case QS_GATE_Y:  // conj(Y) = [[0, i], [-i, 0]]
      *ck = QS_GATE_MATRIX;
      *cm = {0, 0, 0, 1, 0, -1, 0, 0};
      break;
    case QS_GATE_S: *ck = QS_GATE_SDG; break;
    case QS_GATE_SDG: *ck = QS_GATE_S; break;
    case QS_GATE_T: *ck = QS_GATE_TDG; break;
    case QS_GATE_TDG: *ck = QS_GATE_T; break;
    case QS_GATE_RX:
    case QS_GATE_RZ:
    case QS_GATE_PS:
    case QS_GATE_RXX:
    case QS_GATE_RYY:
    case QS_GATE_RZZ:  // exp(-i theta P / 2) with P real: conj = exp(+i theta P / 2)
      *cc = -coef;
      *cconst = -constant;
      break;
    case QS_GATE_MATRIX: {
      const int d = 1 << n_t;
      cm->assign(matrix, matrix + 2 * d * d);
      for (int e = 0; e < d * d; ++e) (*cm)[2 * e + 1] = -(*cm)[2 * e + 1];
      break;
    }
    default:
      set_error("unknown gate kind");
      return QS_ERR_INVALID_ARG;
  }
  return QS_OK;
}

}  // namespace

extern "C" {

qs_status qs_dm_circuit_create(int n_qubits, qs_circuit** out) {
  QS_CHECK(out != nullptr, "out is null");
  QS_CHECK(n_qubits >= 1 && 2 * n_qubits <= kMaxQubits, "density matrices hold 1..17 qubits");
  QS_TRY(qs_circuit_create(2 * n_qubits, out));
  (*out)->dm_n = n_qubits;
  return QS_OK;
}

qs_status qs_dm_add_gate(qs_circuit* c, int kind, const int* targets, int n_t, const int* ctrls, int n_c,
                         int param_idx, double coef, double constant, const double* matrix) {
  QS_CHECK(c != nullptr && c->dm_n > 0, "not a density-matrix circuit");
  const int n = c->dm_n;
  QS_CHECK(targets != nullptr && n_t >= 1 && n_t <= 2 && n_c >= 0 && n_c <= n, "bad targets or controls");
  for (int i = 0; i < n_t; ++i) QS_CHECK(targets[i] >= 0 && targets[i] < n, "target qubit out of range");
  for (int i = 0; i < n_c; ++i) QS_CHECK(ctrls != nullptr && ctrls[i] >= 0 && ctrls[i] < n, "control out of range");
  QS_TRY(qs_circuit_add(c, kind, targets, n_t, ctrls, n_c, param_idx, coef, constant, matrix));
  int ck;
  double cc, cconst;
  std::vector<double> cm;
  QS_TRY(conj_gate(kind, coef, constant, matrix, n_t, &ck, &cc, &cconst, &cm));
  int t2[2], c2[64];
  for (int i = 0; i < n_t; ++i) t2[i] = targets[i] + n;
  for (int i = 0; i < n_c; ++i) c2[i] = ctrls[i] + n;
  return qs_circuit_add(c, ck, t2, n_t, c2, n_c, ck == QS_GATE_MATRIX ? -1 : param_idx, cc, cconst,
                        cm.empty() ? nullptr : cm.data());
}

qs_status qs_dm_add_channel(qs_circuit* c, int kind, int qubit, const double* p, int n_kraus, const double* kraus) {
  QS_CHECK(c != nullptr && c->dm_n > 0, "not a density-matrix circuit");
  const int n = c->dm_n;
  QS_CHECK(qubit >= 0 && qubit < n, "qubit out of range");
  std::vector<std::vector<cd>> K;  // 2x2 row-major
  auto mk = [](cd a, cd b, cd e, cd d) { return std::vector<cd>{a, b, e, d}; };
  if (kind == QS_CH_PAULI || kind == QS_CH_DEPOLARIZING) {
    QS_CHECK(p != nullptr, "null probabilities");
    double px, py, pz;
    if (kind == QS_CH_PAULI) {
      px = p[0], py = p[1], pz = p[2];
    } else {
      QS_CHECK(p[0] >= 0.0 && p[0] <= 1.0, "probability outside [0, 1]");
      px = py = pz = p[0] / 4.0;
    }
    QS_CHECK(px >= 0 && py >= 0 && pz >= 0 && px + py + pz <= 1.0 + 1e-12, "probabilities must be >= 0, sum <= 1");
    const double p0 = std::max(0.0, 1.0 - px - py - pz);
    K.push_back(mk(std::sqrt(p0), 0, 0, std::sqrt(p0)));
    K.push_back(mk(0, std::sqrt(px), std::sqrt(px), 0));
    K.push_back(mk(0, cd(0, -std::sqrt(py)), cd(0, std::sqrt(py)), 0));
    K.push_back(mk(std::sqrt(pz), 0, 0, -std::sqrt(pz)));
  } else if (kind == QS_CH_AMPLITUDE_DAMPING || kind == QS_CH_PHASE_DAMPING) {
    QS_CHECK(p != nullptr && p[0] >= 0.0 && p[0] <= 1.0, "gamma outside [0, 1]");
    const double g = p[0];
    K.push_back(mk(1, 0, 0, std::sqrt(1 - g)));
    if (kind == QS_CH_AMPLITUDE_DAMPING)
      K.push_back(mk(0, std::sqrt(g), 0, 0));
    else
      K.push_back(mk(0, 0, 0, std::sqrt(g)));
  } else if (kind == QS_CH_KRAUS) {
    QS_CHECK(n_kraus >= 1 && n_kraus <= 16 && kraus != nullptr, "1..16 Kraus operators");
    for (int i = 0; i < n_kraus; ++i) {
      std::vector<cd> k(4);
      for (int e = 0; e < 4; ++e) {
        QS_CHECK(std::isfinite(kraus[8 * i + 2 * e]) && std::isfinite(kraus[8 * i + 2 * e + 1]), "non-finite entry");
        k[e] = cd(kraus[8 * i + 2 * e], kraus[8 * i + 2 * e + 1]);
      }
      K.push_back(k);
    }
    // completeness: sum K^dag K = I (trace preserving)
    cd s[4] = {0, 0, 0, 0};
    for (const auto& k : K)
      for (int r = 0; r < 2; ++r)
        for (int col = 0; col < 2; ++col)
          for (int m = 0; m < 2; ++m) s[2 * r + col] += std::conj(k[2 * m + r]) * k[2 * m + col];
    QS_CHECK(std::abs(s[0] - 1.0) < 1e-9 && std::abs(s[1]) < 1e-9 && std::abs(s[2]) < 1e-9 &&
                 std::abs(s[3] - 1.0) < 1e-9,
             "Kraus operators are not complete (sum K^dag K != I)");
  } else {
    set_error("unknown channel kind");
    return QS_ERR_INVALID_ARG;
  }
  // superoperator on (qubit, qubit + n): S[a + 2b][c + 2d] = sum_i K_i[a][c] conj(K_i[b][d])
  std::vector<double> S(32, 0.0);
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b)
      for (int cc = 0; cc < 2; ++cc)
        for (int d = 0; d < 2; ++d) {
          cd v = 0;
          for (const auto& k : K) v += k[2 * a + cc] * std::conj(k[2 * b + d]);
          const int r = a + 2 * b, col = cc + 2 * d;
          S[2 * (4 * r + col)] = v.real();
          S[2 * (4 * r + col) + 1] = v.imag();
        }
  const int t[2] = {qubit, qubit + n};
  QS_TRY(qs_circuit_add(c, QS_GATE_MATRIX, t, 2, nullptr, 0, -1, 1.0, 0.0, S.data()));
  c->has_channel = true;
  return QS_OK;
}

qs_status qs_dm_expectation(const qs_state* rho, const qs_ham* h, double* energy) {
  QS_TRY(check_state(rho));
  QS_CHECK(h != nullptr && energy != nullptr, "null argument");
  QS_CHECK(rho->n % 2 == 0 && h->n == rho->n / 2, "rho must hold 2n qubits for an n-qubit Hamiltonian");
  qs_state* s = const_cast<qs_state*>(rho);
  const int n = rho->n / 2;
  const uint64_t N = 1ull << n;
  const int grid = (int)std::min<uint64_t>(std::max<uint64_t>((N + kDmThreads - 1) / kDmThreads, 1), 1024);
  QS_TRY(ensure_scratch(s, (size_t)grid + 2));
  if (h->n_groups > 0) {
    if (rho->dt == QS_C64)
      dm_expect_kernel<float><<<grid, kDmThreads, 0, s->st>>>((const float2*)rho->ptr, n, h->d_groups, h->n_groups,
                                                             h->d_terms, s->scratch);
    else
      dm_expect_kernel<double><<<grid, kDmThreads, 0, s->st>>>((const double2*)rho->ptr, n, h->d_groups,
                                                              h->n_groups, h->d_terms, s->scratch);
    QS_CUDA(cudaGetLastError());
    QS_TRY(launch_reduce_slots(s->scratch, 1, grid, nullptr, s->scratch + grid, s->st));
    QS_CUDA(cudaMemcpyAsync(energy, s->scratch + grid, sizeof(double), cudaMemcpyDeviceToHost, s->st));
    QS_CUDA(cudaStreamSynchronize(s->st));
  } else {
    *energy = 0.0;
  }
  return QS_OK;
}

}  // extern "C"
