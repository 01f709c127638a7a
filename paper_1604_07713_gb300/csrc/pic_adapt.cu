// Mesh adaptation (§3.1, §4.3) and per-leaf split/merge particle management (§4.3).
#include "pic_internal.cuh"

namespace gbpic {

void adapt_mesh(pic_ctx *ctx, Instance &in) {
    (void)ctx; (void)in;
    fail(PIC_EINVAL, "mesh adaptation is not available in this build");
}

void split_merge(pic_ctx *ctx, Instance &in) {
    (void)ctx; (void)in;
    fail(PIC_EINVAL, "split/merge is not available in this build");
}

}  // namespace gbpic
