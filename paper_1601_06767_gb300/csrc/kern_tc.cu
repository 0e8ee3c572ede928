// Split-precision tensor-core contraction (tcgen05) - placeholder until the
// kernel lands; split plans are refused at plan creation.
#include "internal.h"

namespace chi0 {

bool tc_supported(std::string* why) {
  if (why) *why = "tensor-core contraction not built";
  return false;
}

size_t tc_pack_bytes(const chi0_plan_s*, int64_t, int) { return 0; }

cudaError_t launch_contract_tc(chi0_plan_s*, int, const float2*, int64_t, const double2*, double2*, cudaStream_t,
                               std::string* why) {
  if (why) *why = "not built";
  return cudaErrorNotSupported;
}

}  // namespace chi0
