// pic_read_emag_noalloc: the |E| read-out of pic_read_fields(PIC_FIELD_EMAG) for callers that
// must not allocate device memory.  Its device scratch is a fixed file-scope array instead of
// a cudaMalloc'd buffer.
#include <mutex>

#include "pic_internal.cuh"

namespace {

// 131,072 leaves x 8 bytes = 1 MiB.  Every GPU that loads the library holds this array until
// the process exits.
constexpr int64_t kNoAllocMaxLeaves = 1 << 17;
static __device__ __align__(256) double g_emag_scratch[kNoAllocMaxLeaves];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
double *g_scratch_addr[kMaxDevices] = {};

struct Args {
    pic_ctx *ctx;
    int32_t inst;
    double *out;
    int64_t cap;
    int64_t *n_out;
};

// The array's name in host code is only a host-side stand-in; the device address comes from
// cudaGetSymbolAddress, once per device, with that device current.
double *scratch_for_current_device() {
    int dev = 0;
    GB_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) gbpic::fail(PIC_EINVAL, "device index beyond the no-alloc setup table");
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        GB_CUDA(cudaGetSymbolAddress(&p, g_emag_scratch));
        g_scratch_addr[dev] = static_cast<double *>(p);
    }
    return g_scratch_addr[dev];
}

pic_status run(void *v) {
    Args &a = *static_cast<Args *>(v);
    if (!a.ctx) gbpic::fail(PIC_EINVAL, "null context");
    if (a.inst < 0 || a.inst >= (int32_t)a.ctx->inst.size()) gbpic::fail(PIC_EINVAL, "instance index out of range");
    gbpic::Instance &in = a.ctx->inst[a.inst];
    if (!in.has_mesh) gbpic::fail(PIC_EINVAL, "mesh not set");
    const int64_t nl = in.nleaf;
    if (a.n_out) *a.n_out = nl;
    if (nl > kNoAllocMaxLeaves)
        gbpic::fail(PIC_EINVAL, "pic_read_emag_noalloc: " + std::to_string(nl) + " leaves exceed the fixed scratch of " +
                                    std::to_string(kNoAllocMaxLeaves) + " leaves; use pic_read_fields");
    if (!a.out || a.cap < nl) gbpic::fail(PIC_EINVAL, "output capacity too small");
    // the scratch is picked by the current device: it must be the context's, or the launch on
    // the context's stream would fail and poison the context
    int dev = -1;
    GB_CUDA(cudaGetDevice(&dev));
    if (dev != a.ctx->device)
        gbpic::fail(PIC_EINVAL, "pic_read_emag_noalloc: the current CUDA device (" + std::to_string(dev) +
                                    ") is not the context's device (" + std::to_string(a.ctx->device) + ")");
    double *scratch = scratch_for_current_device();
    double walls[4];
    gbpic::walls_at(in, a.ctx->step, walls);
    // every element read back below is written by this launch first: nothing to clear
    gbpic::cell_emag(a.ctx, in, walls, scratch);
    GB_CUDA(cudaMemcpyAsync(a.out, scratch, nl * sizeof(double), cudaMemcpyDeviceToHost, a.ctx->stream));
    GB_CUDA(cudaStreamSynchronize(a.ctx->stream));
    return PIC_OK;
}

}  // namespace

extern "C" pic_status pic_read_emag_noalloc(pic_ctx *ctx, int32_t inst, double *out, int64_t cap, int64_t *n_out) {
    Args a{ctx, inst, out, cap, n_out};
    return gbpic::guarded_call(ctx, run, &a);
}
