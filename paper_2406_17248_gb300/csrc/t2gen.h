// Per-circuit kernels of the complex64 micro-op tile passes (t2gen.cu).
#pragma once

#include <string>
#include <vector>

#include "qsim_internal.h"

namespace qs {

// CUDA source of the plan's micro-op passes (kernel qs_t2g_<i> for pass i;
// `passes` lists the i).  False when a pass holds an op it cannot write out.
bool t2gen_source(const TilePlan& plan, std::string* src, std::vector<int>* passes);
// Source of pass pi alone (its kernel qs_t2g_<pi>); false as above.
bool t2gen_pass_source(const TilePlan& plan, int pi, std::string* src);
// Compiles generated sources for sm_103a on the host's cores (runtime
// compiler; needs no GPU).
qs_status t2gen_compile(const std::vector<std::string>& srcs, std::vector<std::vector<char>>* cubins);
// Ops above which a pass is left to the library kernel when plan.gen == 1
// (compile time grows with the ops of a pass: about 30 ms per op of a
// one-state pass and 45 ms of a two-state pass on one host core).
int t2gen_budget_ops(int ns);
// Compiles (or finds in the process cache) and loads the plan's generated
// passes; fills plan.gen_fn.
qs_status t2gen_build(TilePlan& plan);
// Launches a generated pass with the arguments of the library kernel.
qs_status t2gen_launch(void* fn, const T2Args& a, int grid, int threads, uint32_t smem, cudaStream_t st);

}  // namespace qs
