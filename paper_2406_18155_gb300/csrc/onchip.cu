// On-chip evolution: placeholder until the per-column kernel lands.
#include "fast.h"
bool fast_onchip_available(const KPlan&, bool) { return false; }
sg_status fast_onchip_forward(sg_system* sys, const KPlan&, bool, const void*, double2*, int, double,
                              cudaStream_t, int*) {
  return sg_fail(sys->ctx, SG_E_UNSUPPORTED, "on-chip path not built");
}
