// Entry points whose implementation is still to come: they report EUNSUPPORTED.
#include "litho_internal.h"

using namespace litho;

extern "C" {

litho_status litho_serve_create(size_t, int, int, litho_server** out) {
  if (out) *out = nullptr;
  set_error("not implemented yet");
  return LITHO_EUNSUPPORTED;
}
litho_status litho_serve_submit(litho_server*, const litho_request*, uint64_t*) { return LITHO_EUNSUPPORTED; }
litho_status litho_serve_poll(litho_server*, uint64_t, int) { return LITHO_EUNSUPPORTED; }
litho_status litho_serve_cancel(litho_server*, uint64_t) { return LITHO_EUNSUPPORTED; }
litho_status litho_serve_stats(litho_server*, litho_serve_stats_t*) { return LITHO_EUNSUPPORTED; }
void litho_serve_destroy(litho_server*) {}

}
