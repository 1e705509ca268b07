// Serving loop (continuous batching) -- placeholder until the step kernel lands.
#include "ahpp_host.h"

extern "C" {
int ahpp_server_start(ahpp_graph*, const ahpp_server_opts*, ahpp_server** out) {
  if (out) *out = nullptr;
  ahpp::set_error("serving loop not built yet");
  return AHPP_ESTATE;
}
int ahpp_submit(ahpp_server*, uint32_t, double, uint32_t, uint64_t*) { return AHPP_ESTATE; }
int ahpp_wait(ahpp_server*, uint64_t, int, uint32_t*, float*, uint32_t*, ahpp_stats*) { return AHPP_ESTATE; }
int ahpp_server_info_get(ahpp_server*, ahpp_server_info*) { return AHPP_ESTATE; }
int ahpp_server_stop(ahpp_server*) { return AHPP_OK; }
}
