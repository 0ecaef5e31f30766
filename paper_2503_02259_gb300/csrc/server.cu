// Continuous-batching request server (placeholder until the server is built).
#include "gp_api_internal.h"

extern "C" {
gp_status gp_server_create(size_t, int32_t, gp_server**) {
  gp::set_error("server not built yet");
  return GP_ERR_UNIMPLEMENTED;
}
gp_status gp_server_submit(gp_server*, const gp_request*, uint64_t*) { return GP_ERR_UNIMPLEMENTED; }
gp_status gp_server_poll(gp_server*, uint64_t, gp_result*) { return GP_ERR_UNIMPLEMENTED; }
gp_status gp_server_drain(gp_server*, double) { return GP_ERR_UNIMPLEMENTED; }
gp_status gp_server_destroy(gp_server*) { return GP_ERR_UNIMPLEMENTED; }
}
