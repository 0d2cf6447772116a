// Per-circuit kernels of the complex64 micro-op tile passes.  The passes of a
// plan are written out as CUDA source in which every phase is a straight-line
// sequence of calls of the op bodies of t2_device.cuh, with register bits,
// control masks, constant bits and coefficient offsets as literals, and
// compiled for sm_103a by the runtime compiler when the plan is uploaded.  The
// kernels are the library's micro-op kernels with the op dispatch taken out:
// the producer warp, the tile ring, the shared stages, the op bodies and the
// fixed-order FP64 reductions are the same code, so the results are the same
// bit for bit.  What the dispatch costs in the library kernel (the 32 live
// amplitudes held in fixed registers across a switch, every body ending by
// moving its results back, swaps and sign flips executed as moves) goes away:
// the compiler renames registers for X gates and folds sign flips into the
// next multiply.  Compiled modules are cached by their source for the life of
// the process.
#include <dlfcn.h>
#include <nvrtc.h>

#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "qsim_internal.h"
#include "t2gen.h"

namespace qs {

namespace {

void app(std::string& o, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
void app(std::string& o, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  const int k = std::vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (k > 0) o.append(buf, (size_t)std::min(k, (int)sizeof(buf) - 1));
}

// The call of one op, or false for a code outside the set the library
// kernel's dispatch knows (t2_run: such ops are skipped there too, and a plan
// that holds one is not generated).  M names the op's coefficients.
bool emit_op(std::string& o, const T2Op& op, int ns) {
  const int code = op.code & (T2_OUTSIDE - 1);
  const int kind = code & 31, r0 = (code >> 5) & 3, r1 = (code >> 7) & 3;
  const bool jc = (code >> 9) & 1;
  if (code & ~(31 | (3 << 5) | (3 << 7) | 512)) return false;
  const char* JC = jc ? "true" : "false";
  const unsigned J = op.jc;
  const bool grad = kind == T2_G1 || kind == T2_G2 || kind == T2_GD;
  if (grad && ns != 2) return true;  // no accumulator in one-state passes: skipped, as in t2_run
  std::string body;
  char M[32];
  std::snprintf(M, sizeof M, "(c.coef + %u)", (unsigned)op.cs);
  auto cbit = [&](unsigned d) {
    char b[64];
    std::snprintf(b, sizeof b, "t2_cbit(%uu, l0, c.toff)", d);
    return std::string(b);
  };
  const bool need_r1_zero = kind == T2_U1 || kind == T2_R1 || kind == T2_RX || kind == T2_X || kind == T2_Z ||
                            kind == T2_D1R || kind == T2_D2RC || kind == T2_G1;
  const bool need_both_zero = kind == T2_ZC || kind == T2_D1C || kind == T2_D2CC || kind == T2_GD;
  if (need_r1_zero && r1 != 0) return false;
  if (need_both_zero && (r0 | r1)) return false;
  if (kind == T2_D2CR && r0 != 0) return false;
  if ((kind == T2_D2RR || kind == T2_U2 || kind == T2_G2) && r0 == r1) return false;
  switch (kind) {
    case T2_U1: app(body, "t2_u1<%d, %d, %s>(s, %s, %uu);", ns, r0, JC, M, J); break;
    case T2_R1: app(body, "t2_r1<%d, %d, %s>(s, %s, %uu);", ns, r0, JC, M, J); break;
    case T2_RX: app(body, "t2_rx<%d, %d, %s>(s, %s, %uu);", ns, r0, JC, M, J); break;
    case T2_X: app(body, "t2_x<%d, %d, %s>(s, %uu);", ns, r0, JC, J); break;
    case T2_Z: app(body, "t2_z<%d, %d, %s>(s, %uu);", ns, r0, JC, J); break;
    case T2_ZC: app(body, "if (%s) t2_neg_all<%d, %s>(s, %uu);", cbit(op.d0).c_str(), ns, JC, J); break;
    case T2_D1R: app(body, "t2_d1<%d, %d, %s>(s, %s[0], %s[1], %uu);", ns, r0, JC, M, M, J); break;
    case T2_D1C: app(body, "t2_scale_all<%d, %s>(s, %s[%s], %uu);", ns, JC, M, cbit(op.d0).c_str(), J); break;
    case T2_D2RR: app(body, "t2_d2<%d, %d, %d, %s>(s, %s, %uu);", ns, r0, r1, JC, M, J); break;
    case T2_D2RC:
      app(body, "{ const uint32_t g = %s << 1; t2_d1<%d, %d, %s>(s, %s[g], %s[g + 1], %uu); }",
          cbit(op.d1).c_str(), ns, r0, JC, M, M, J);
      break;
    case T2_D2CR:
      app(body, "{ const uint32_t g = %s; t2_d1<%d, %d, %s>(s, %s[g], %s[g + 2], %uu); }", cbit(op.d0).c_str(),
          ns, r1, JC, M, M, J);
      break;
    case T2_D2CC:
      app(body, "t2_scale_all<%d, %s>(s, %s[%s | (%s << 1)], %uu);", ns, JC, M, cbit(op.d0).c_str(),
          cbit(op.d1).c_str(), J);
      break;
    case T2_U2: app(body, "t2_u2<%d, %d, %d, %s>(s, %s, %uu);", ns, r0, r1, JC, M, J); break;
    case T2_G1: app(body, "t2_g1<%d, %s>(s, %s, %uu)", r0, JC, M, J); break;
    case T2_G2: app(body, "t2_g2<%d, %d, %s>(s, %s, %uu)", r0, r1, JC, M, J); break;
    case T2_GD: app(body, "t2_gd<2>(s, %s, %uu, %uu, l0, c.toff, %uu)", M, (unsigned)op.d0, (unsigned)op.d1, J); break;
    default: return false;
  }
  const bool outside = (op.code & T2_OUTSIDE) != 0;
  char okc[128] = "true";
  if (outside)
    std::snprintf(okc, sizeof okc, "((l0 & %uu) == %uu) && ((c.toff & %lluull) == %lluull)", (unsigned)op.lc,
                  (unsigned)op.lc, (unsigned long long)op.gc, (unsigned long long)op.gc);
  if (grad) {
    if (outside)
      app(o, "      c.grad((%s) ? %s : 0.f, %u);\n", okc, body.c_str(), (unsigned)op.slot);
    else
      app(o, "      c.grad(%s, %u);\n", body.c_str(), (unsigned)op.slot);
  } else if (outside) {
    app(o, "      if (%s) { %s }\n", okc, body.c_str());
  } else {
    app(o, "      %s\n", body.c_str());
  }
  return true;
}

// Source of pass pi of a plan (its phase bodies, its program and its kernel
// qs_t2g_<pi>), or false when an op cannot be written out.
bool emit_pass(std::string& o, const PlannedPass& pp, int pi) {
  const T2Pass& h = pp.t2hdr;
  const int ns = h.ns;
  for (int p = 0; p < h.n_phases; ++p) {
    const T2Phase& ph = pp.t2ph[p];
    app(o, "struct Ph%d_%d {\n  const T2Ctx<%d>& c;\n", pi, p, ns);
    app(o, "  __device__ __forceinline__ void operator()(Sub<%d>& s, uint32_t l0) const {\n", ns);
    o += "    (void)l0;\n";
    for (int k = ph.op_begin; k < ph.op_end; ++k)
      if (!emit_op(o, pp.t2ops[k], ns)) return false;
    o += "  }\n};\n";
  }
  app(o, "struct Prog%d {\n  __device__ __forceinline__ void operator()(const T2Ctx<%d>& c, int) const {\n", pi, ns);
  for (int p = 0; p < h.n_phases; ++p)
    app(o, "    c.phase<%d>(%d, Ph%d_%d{c});\n", pp.t2ph[p].pair ? 1 : 0, p, pi, p);
  o += "  }\n};\n";
  app(o,
      "extern \"C\" __global__ void __launch_bounds__(%d, 1) qs_t2g_%d(const __grid_constant__ qs::T2Args args) {\n"
      "  tile2_body<%d>(args, args.tm, Prog%d{});\n}\n\n",
      ns == 2 ? 288 : 544, pi, ns, pi);
  return true;
}

}  // namespace

bool t2gen_source(const TilePlan& plan, std::string* src, std::vector<int>* passes) {
  std::string o =
      "// generated: complex64 micro-op tile passes of one plan\n"
      "#include \"t2_device.cuh\"\n"
      "using namespace qs;\nusing namespace qs::t2d;\n\n";
  passes->clear();
  for (int pi = 0; pi < (int)plan.passes.size(); ++pi) {
    if (!plan.passes[pi].t2) continue;
    if (!emit_pass(o, plan.passes[pi], pi)) return false;
    passes->push_back(pi);
  }
  *src = std::move(o);
  return true;
}

namespace {

// Directory of the kernel headers: csrc/ beside the library's _lib/ folder.
std::string header_dir() {
  Dl_info info;
  if (!dladdr(reinterpret_cast<void*>(&header_dir), &info) || !info.dli_fname) return "";
  std::string p = info.dli_fname;
  const size_t a = p.rfind('/');
  if (a == std::string::npos) return "";
  p.resize(a);  // .../_lib
  const size_t b = p.rfind('/');
  if (b == std::string::npos) return "";
  p.resize(b);
  return p + "/csrc";
}

typedef CUresult (*ModuleLoadDataFn)(CUmodule*, const void*);
typedef CUresult (*ModuleGetFunctionFn)(CUfunction*, CUmodule, const char*);
typedef CUresult (*FuncSetAttributeFn)(CUfunction, CUfunction_attribute, int);
typedef CUresult (*LaunchKernelFn)(CUfunction, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned, unsigned,
                                   CUstream, void**, void**);

struct DriverFns {
  ModuleLoadDataFn load = nullptr;
  ModuleGetFunctionFn get = nullptr;
  FuncSetAttributeFn attr = nullptr;
  LaunchKernelFn launch = nullptr;
  bool ok = false;
};

const DriverFns& driver() {
  static DriverFns d;
  static std::once_flag once;
  std::call_once(once, [] {
    auto get = [](const char* name, void** f) {
      cudaDriverEntryPointQueryResult q;
      return cudaGetDriverEntryPointByVersion(name, f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
             q == cudaDriverEntryPointSuccess && *f;
    };
    void *a = nullptr, *b = nullptr, *c = nullptr, *e = nullptr;
    d.ok = get("cuModuleLoadData", &a) && get("cuModuleGetFunction", &b) && get("cuFuncSetAttribute", &c) &&
           get("cuLaunchKernel", &e);
    d.load = reinterpret_cast<ModuleLoadDataFn>(a);
    d.get = reinterpret_cast<ModuleGetFunctionFn>(b);
    d.attr = reinterpret_cast<FuncSetAttributeFn>(c);
    d.launch = reinterpret_cast<LaunchKernelFn>(e);
  });
  return d;
}

// One pass's kernel, loaded.
struct GenKernel {
  CUmodule mod = nullptr;
  CUfunction fn = nullptr;
};

std::mutex g_mu;
std::map<std::string, GenKernel> g_cache;  // by device and source (modules stay loaded)

const char kPrefix[] =
    "// generated: complex64 micro-op tile pass\n"
    "#include \"t2_device.cuh\"\n"
    "using namespace qs;\nusing namespace qs::t2d;\n\n";

// Compiles one source for sm_103a; on failure returns the message instead of
// recording it (callers on other threads).
bool compile_one(const std::string& src, std::vector<char>* cubin, std::string* msg) {
  const std::string inc = "-I" + header_dir();
  const char* opts[] = {"-arch=sm_103a", "-std=c++17", inc.c_str()};
  nvrtcProgram prog;
  if (nvrtcCreateProgram(&prog, src.c_str(), "qs_t2gen.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS) {
    *msg = "nvrtcCreateProgram failed";
    return false;
  }
  const nvrtcResult r = nvrtcCompileProgram(prog, 3, opts);
  if (r != NVRTC_SUCCESS) {
    size_t n = 0;
    nvrtcGetProgramLogSize(prog, &n);
    std::string lg(n, '\0');
    if (n) nvrtcGetProgramLog(prog, &lg[0]);
    nvrtcDestroyProgram(&prog);
    *msg = std::string("runtime compilation of the generated passes failed: ") + nvrtcGetErrorString(r) + ": " +
           lg.substr(0, 1500);
    return false;
  }
  size_t cb = 0;
  nvrtcGetCUBINSize(prog, &cb);
  cubin->assign(cb, 0);
  const nvrtcResult r2 = cb ? nvrtcGetCUBIN(prog, cubin->data()) : NVRTC_ERROR_INVALID_INPUT;
  nvrtcDestroyProgram(&prog);
  if (r2 != NVRTC_SUCCESS) {
    *msg = "the runtime compiler returned no sm_103a binary";
    return false;
  }
  return true;
}

}  // namespace

bool t2gen_pass_source(const TilePlan& plan, int pi, std::string* src) {
  std::string o = kPrefix;
  if (!plan.passes[pi].t2 || !emit_pass(o, plan.passes[pi], pi)) return false;
  *src = std::move(o);
  return true;
}

qs_status t2gen_compile(const std::vector<std::string>& srcs, std::vector<std::vector<char>>* cubins) {
  const size_t n = srcs.size();
  cubins->assign(n, {});
  std::vector<std::string> msg(n);
  std::vector<char> ok(n, 0);
  const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  const size_t nth = std::min<size_t>(n, std::min(hw, 32u));
  std::atomic<size_t> next{0};
  auto work = [&] {
    for (size_t i; (i = next.fetch_add(1)) < n;) ok[i] = compile_one(srcs[i], &(*cubins)[i], &msg[i]);
  };
  std::vector<std::thread> th;
  for (size_t t = 1; t < nth; ++t) th.emplace_back(work);
  work();
  for (auto& t : th) t.join();
  for (size_t i = 0; i < n; ++i)
    if (!ok[i]) {
      set_error(msg[i]);
      return QS_ERR_UNSUPPORTED;
    }
  return QS_OK;
}

int t2gen_budget_ops(int ns) { return ns == 2 ? 128 : 192; }

qs_status t2gen_build(TilePlan& plan) {
  plan.gen_fn.assign(plan.passes.size(), nullptr);
  std::vector<int> ids;
  std::vector<std::string> srcs;
  for (int pi = 0; pi < (int)plan.passes.size(); ++pi) {
    if (!plan.passes[pi].t2) continue;
    const T2Pass& h = plan.passes[pi].t2hdr;
    if (plan.gen == 1 && h.n_ops > t2gen_budget_ops(h.ns)) continue;
    std::string src;
    if (!t2gen_pass_source(plan, pi, &src)) {
      set_error("a micro-op pass holds an op the generator does not write out");
      return QS_ERR_UNSUPPORTED;
    }
    ids.push_back(pi);
    srcs.push_back(std::move(src));
  }
  if (ids.empty()) return QS_OK;
  const DriverFns& d = driver();
  if (!d.ok) {
    set_error("the CUDA driver entry points for loading generated kernels are missing");
    return QS_ERR_CUDA;
  }
  int dev = 0;
  QS_CUDA(cudaGetDevice(&dev));
  QS_CUDA(cudaFree(nullptr));  // the device's primary context is current
  const std::string dk = std::to_string(dev) + "\n";
  std::vector<size_t> miss;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    for (size_t k = 0; k < ids.size(); ++k) {
      auto it = g_cache.find(dk + srcs[k]);
      if (it != g_cache.end()) plan.gen_fn[ids[k]] = reinterpret_cast<void*>(it->second.fn);
      else miss.push_back(k);
    }
  }
  if (miss.empty()) return QS_OK;
  std::vector<std::string> todo;
  for (size_t k : miss) todo.push_back(srcs[k]);
  std::vector<std::vector<char>> cubins;
  QS_TRY(t2gen_compile(todo, &cubins));
  for (size_t j = 0; j < miss.size(); ++j) {
    const int pi = ids[miss[j]];
    GenKernel gk;
    CUresult e = d.load(&gk.mod, cubins[j].data());
    if (e != CUDA_SUCCESS) {
      set_error("cuModuleLoadData failed on a generated pass (" + std::to_string((int)e) + ")");
      return QS_ERR_CUDA;
    }
    const std::string name = "qs_t2g_" + std::to_string(pi);
    e = d.get(&gk.fn, gk.mod, name.c_str());
    if (e != CUDA_SUCCESS) {
      set_error("cuModuleGetFunction failed for " + name);
      return QS_ERR_CUDA;
    }
    e = d.attr(gk.fn, CU_FUNC_ATTRIBUTE_MAX_DYNAMIC_SHARED_SIZE_BYTES, (int)plan.passes[pi].t2hdr.smem);
    if (e != CUDA_SUCCESS) {
      set_error("cuFuncSetAttribute failed for " + name);
      return QS_ERR_CUDA;
    }
    {
      std::lock_guard<std::mutex> lk(g_mu);
      g_cache.emplace(dk + srcs[miss[j]], gk);
    }
    plan.gen_fn[pi] = reinterpret_cast<void*>(gk.fn);
  }
  return QS_OK;
}

qs_status t2gen_launch(void* fn, const T2Args& a, int grid, int threads, uint32_t smem, cudaStream_t st) {
  const DriverFns& d = driver();
  T2Args arg = a;
  void* params[] = {&arg};
  const CUresult e = d.launch(reinterpret_cast<CUfunction>(fn), (unsigned)grid, 1, 1, (unsigned)threads, 1, 1, smem,
                              reinterpret_cast<CUstream>(st), params, nullptr);
  if (e != CUDA_SUCCESS) {
    set_error("cuLaunchKernel failed on a generated pass (" + std::to_string((int)e) + ")");
    return QS_ERR_CUDA;
  }
  return QS_OK;
}

}  // namespace qs
