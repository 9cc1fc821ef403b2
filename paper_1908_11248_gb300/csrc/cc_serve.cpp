// Serving loop of the colour-coding library (cc_serve_* in include/cc.h).
#include <cstdint>

#include "../../include/cc.h"

extern "C" {

int cc_serve_start(cc_ctx *ctx, size_t mem_budget, int32_t max_inflight) {
  (void)ctx; (void)mem_budget; (void)max_inflight;
  return CC_EINVAL;
}

int cc_serve_submit(cc_ctx *ctx, int32_t pattern_id, uint64_t seed, int32_t trials, int32_t k,
                    int64_t *ticket) {
  (void)ctx; (void)pattern_id; (void)seed; (void)trials; (void)k; (void)ticket;
  return CC_EINVAL;
}

int cc_serve_poll(cc_ctx *ctx, int64_t ticket, int32_t *done, int32_t *status,
                  uint64_t *h_counts, uint8_t *h_exists, int64_t *latency_ns) {
  (void)ctx; (void)ticket; (void)done; (void)status; (void)h_counts; (void)h_exists;
  (void)latency_ns;
  return CC_EINVAL;
}

int cc_serve_stop(cc_ctx *ctx) {
  (void)ctx;
  return CC_OK;
}

}  // extern "C"
