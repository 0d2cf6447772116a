// <psi|H|psi> without any device allocation.
//
// Some callers cannot let a library call cudaMalloc: a process whose device
// memory is all owned by another allocator (a framework's caching allocator, or
// a pool reserved at start-up to a fixed budget), where a raw cudaMalloc fails or
// breaks the budget; or a latency-critical loop that must not risk the device-wide
// synchronisation that cudaFree performs and cudaMalloc may perform.  For them
// qs_expectation_noalloc runs the same Pauli-sum kernel as qs_expectation, with
// its working memory (term tables, per-CTA partial sums, the result slot) in the
// fixed array below instead of memory allocated per call or per handle.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

#include "handles.h"

namespace {

// Working memory of qs_expectation_noalloc.  256 KiB per device; a device that
// loads the library keeps it until the process exits.
constexpr size_t kNoallocBytes = 256 * 1024;
constexpr int kNoallocMaxTerms = 4096;
constexpr int kNoallocMaxGrid = 2048;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

// byte offsets inside the array
constexpr size_t kOffPartials = 0;                                        // double[kNoallocMaxGrid]
constexpr size_t kOffEnergy = kOffPartials + 8 * kNoallocMaxGrid;          // double[1] (+ pad)
constexpr size_t kOffGroups = kOffEnergy + 256;                            // DevHamGroup[kNoallocMaxTerms]
constexpr size_t kOffTerms = kOffGroups + sizeof(DevHamGroup) * kNoallocMaxTerms;  // DevHamTerm[...]
static_assert(kOffTerms + sizeof(DevHamTerm) * kNoallocMaxTerms <= kNoallocBytes, "noalloc layout");

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_dev_ptr[kMaxDevices] = {nullptr};

// Host staging for the term tables: fixed arrays, reused by every call under g_mu.
DevHamGroup g_h_groups[kNoallocMaxTerms];
DevHamTerm g_h_terms[kNoallocMaxTerms];
int g_h_order[kNoallocMaxTerms];

}  // namespace

extern "C" qs_status qs_expectation_noalloc(const void* dev_psi, int n_qubits, qs_dtype dtype, int n_terms,
                                            const uint64_t* xmask, const uint64_t* zmask, const double* coef,
                                            void* cuda_stream, double* energy) {
  QS_CHECK(dev_psi != nullptr && energy != nullptr, "null argument");
  QS_CHECK(n_qubits >= 1 && n_qubits <= kMaxQubits, "n_qubits must be in 1..34");
  QS_CHECK(dtype == QS_C64 || dtype == QS_C128, "invalid dtype");
  QS_CHECK(n_terms >= 0 && n_terms <= kNoallocMaxTerms,
           "qs_expectation_noalloc takes at most 4096 Pauli terms (its fixed working memory)");
  QS_CHECK(n_terms == 0 || (xmask && zmask && coef), "null term arrays");
  const uint64_t lim = 1ull << n_qubits;
  for (int k = 0; k < n_terms; ++k) {
    QS_CHECK(xmask[k] < lim && zmask[k] < lim, "Pauli mask names a qubit >= n_qubits");
    QS_CHECK(std::isfinite(coef[k]), "non-finite coefficient");
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;
  int dev = 0;
  QS_CUDA(cudaGetDevice(&dev));
  QS_CHECK(dev >= 0 && dev < kMaxDevices, "device index beyond the supported range");

  std::lock_guard<std::mutex> lk(g_mu);
  // Set-up, once per device with that device current: the device address of the
  // array (its name in host code is only a stand-in, not a device address).
  if (!g_dev_ptr[dev]) {
    void* p = nullptr;
    QS_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_dev_ptr[dev] = static_cast<unsigned char*>(p);
  }
  unsigned char* base = g_dev_ptr[dev];
  double* d_part = reinterpret_cast<double*>(base + kOffPartials);
  double* d_energy = reinterpret_cast<double*>(base + kOffEnergy);
  DevHamGroup* d_groups = reinterpret_cast<DevHamGroup*>(base + kOffGroups);
  DevHamTerm* d_terms = reinterpret_cast<DevHamTerm*>(base + kOffTerms);

  // Group the terms by X mask (order ties by input position: a stable grouping).
  for (int k = 0; k < n_terms; ++k) g_h_order[k] = k;
  std::sort(g_h_order, g_h_order + n_terms,
            [&](int a, int b) { return xmask[a] != xmask[b] ? xmask[a] < xmask[b] : a < b; });
  int n_groups = 0;
  const double cr[4] = {1, 0, -1, 0}, ci[4] = {0, 1, 0, -1};
  for (int i = 0; i < n_terms; ++i) {
    const int k = g_h_order[i];
    if (n_groups == 0 || g_h_groups[n_groups - 1].xmask != xmask[k]) {
      g_h_groups[n_groups].xmask = xmask[k];
      g_h_groups[n_groups].begin = g_h_groups[n_groups].end = i;
      ++n_groups;
    }
    const int ny = __builtin_popcountll(xmask[k] & zmask[k]) & 3;  // P = i^{#Y} X^x Z^z
    g_h_terms[i].zmask = zmask[k];
    g_h_terms[i].re = coef[k] * cr[ny];
    g_h_terms[i].im = coef[k] * ci[ny];
    g_h_groups[n_groups - 1].end = i + 1;
  }
  if (n_groups) {
    QS_CUDA(cudaMemcpyAsync(d_groups, g_h_groups, n_groups * sizeof(DevHamGroup), cudaMemcpyHostToDevice, st));
    QS_CUDA(cudaMemcpyAsync(d_terms, g_h_terms, n_terms * sizeof(DevHamTerm), cudaMemcpyHostToDevice, st));
  }
  const int grid = std::min(ham_grid_size(n_qubits), kNoallocMaxGrid);
  QS_TRY(launch_ham_apply(dtype, dev_psi, nullptr, n_qubits, d_groups, n_groups, d_terms, d_part, grid, st));
  QS_TRY(launch_reduce_slots(d_part, 1, grid, nullptr, d_energy, st));
  QS_CUDA(cudaMemcpyAsync(energy, d_energy, sizeof(double), cudaMemcpyDeviceToHost, st));
  // the host tables above are reused by the next call: wait for the copies here
  QS_CUDA(cudaStreamSynchronize(st));
  return QS_OK;
}
