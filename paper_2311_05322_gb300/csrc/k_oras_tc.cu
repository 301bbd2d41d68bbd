// BF16 tensor-core ORAS apply: implemented in a later step.
#include "k_oras_tc.h"
#include "k_oras.h"
#include "mw_internal.h"

namespace mwk {
bool tc_plan_build(TcPlan&, const mw::Subdomains&, const std::function<void*(size_t)>&, cudaStream_t) {
  return false;
}
void tc_plan_free(TcPlan& p, const std::function<void(void*)>&) { p = TcPlan(); }
size_t tc_w_bytes(const TcPlan&) { return 16; }
size_t tc_scratch_bytes(const TcPlan&, int) { return 16; }
void tc_extract(const TcPlan&, const OrasBatch&, const OrasTopo&, int, const void*, void*, cudaStream_t) {}
void oras_apply_tc(const TcPlan&, const OrasTopo&, const void*, const float2*, float2*, int, void*, cudaStream_t) {}
}  // namespace mwk
