// Serving loop: continuous batching of integration requests on resident meshes.
#include "fe_runtime.h"

namespace fe {
struct ServeState {};
void serve_destroy(fe_ctx *ctx) { (void)ctx; }
}  // namespace fe

using namespace fe;
extern "C" {
fe_status fe_serve_submit(fe_ctx *ctx, const fe_request *, uint64_t *) {
    return set_error(ctx, FE_ERR_UNSUPPORTED, "not built yet");
}
fe_status fe_serve_poll(fe_ctx *ctx, uint64_t, fe_result *) { return set_error(ctx, FE_ERR_UNSUPPORTED, "not built yet"); }
fe_status fe_serve_release(fe_ctx *ctx, uint64_t) { return set_error(ctx, FE_ERR_UNSUPPORTED, "not built yet"); }
}
