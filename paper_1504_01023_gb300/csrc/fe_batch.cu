// Batched integration (persistent kernel, captured graph) and resident meshes.
#include "fe_runtime.h"

namespace fe {
struct BatchCache {};
void batch_destroy(fe_ctx *ctx) { (void)ctx; }
}  // namespace fe

using namespace fe;
extern "C" {
fe_status fe_mesh_register(fe_ctx *ctx, fe_elem_type, int64_t, const double *, fe_layout, fe_memory, int64_t *) {
    return set_error(ctx, FE_ERR_UNSUPPORTED, "not built yet");
}
fe_status fe_mesh_release(fe_ctx *ctx, int64_t) { return set_error(ctx, FE_ERR_UNSUPPORTED, "not built yet"); }
fe_status fe_batch_submit(fe_ctx *ctx, const fe_batch_item *, int, void *) {
    return set_error(ctx, FE_ERR_UNSUPPORTED, "not built yet");
}
}
