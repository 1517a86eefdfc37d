// Serving entry points (placeholder until the request loop lands).
#include "swkb.h"

extern "C" {
swkb_status swkb_server_create(size_t, int32_t, int32_t, int32_t, swkb_server** out) {
  if (out) *out = nullptr;
  return SWKB_ERR_INVALID_ARG;
}
swkb_status swkb_submit(swkb_server*, const swkb_request*, uint64_t*) { return SWKB_ERR_INVALID_ARG; }
swkb_status swkb_poll(swkb_server*, uint64_t, double*, int32_t) { return SWKB_ERR_INVALID_ARG; }
swkb_status swkb_cancel(swkb_server*, uint64_t) { return SWKB_ERR_INVALID_ARG; }
swkb_status swkb_server_get_stats(swkb_server*, swkb_server_stats*) { return SWKB_ERR_INVALID_ARG; }
void swkb_server_destroy(swkb_server*) {}
}
