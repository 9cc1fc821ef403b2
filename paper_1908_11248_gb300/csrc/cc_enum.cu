// Result reconstruction (Section 4) on the device.
#include <cstdint>

#include "../../include/cc.h"
#include "cc_internal.h"

namespace cc {
struct Ctx;
struct Run;
int enumerate_run(Ctx *ctx, Run *run, uint64_t limit, int32_t *h_out, uint64_t *n_out,
                  uint64_t *n_total) {
  (void)ctx; (void)run; (void)limit; (void)h_out; (void)n_out; (void)n_total;
  return CC_EINVAL;
}
}  // namespace cc
