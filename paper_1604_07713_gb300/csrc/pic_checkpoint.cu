// Checkpoint and resume of one instance (no counterpart in the paper; the paper's method is
// a time integration, and a restart has to continue it exactly).  A checkpoint holds every
// piece of state that the following steps read:
//   - the leaf mesh (root, Morton code, level per leaf, in key order);
//   - the potential phi, the previous solution and the number of solves since the mesh was
//     set (the next solve's warm start extrapolates from them), and the wall potentials of
//     the last solve (the adaptation's |E| criterion reads them);
//   - the step counter (Philox counter word and RF phase) and the next particle id;
//   - per species the cell lists: per-leaf counts and the records in list order, in the
//     state's precision, plus the per-leaf weight sums (compensated pairs) that the last list
//     update left for the next deposit.
// Restoring it into a context with the same configuration continues bit for bit like the
// run it was taken from: the lists get fresh segments, but no result depends on where a
// segment lies.
//
// Byte layout (host order; every block starts on an 8-byte boundary):
//   Header, root u32[nl], morton u32[nl], level u8[nl], phi f64[nl], phi_prev f64[nl],
//   then per species: SpeciesHeader, count i32[nl], u, v, vx, vy, vz, w R[n], id u32[n],
//   and the per-leaf deposit sums stay_hi, stay_lo, ent_hi, ent_lo R[nl] when sums_valid.
#include <algorithm>
#include <cstring>

#include "pic_internal.cuh"

namespace gbpic {

namespace {
constexpr int kT = 256;
constexpr uint64_t kMagic = 0x314B435049504247ull;  // "GBPIPCK1"
constexpr uint32_t kVersion = 2;
inline unsigned warp_blocks(int64_t nw) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((nw + kT / 32 - 1) / (kT / 32), 1 << 20));
}
inline unsigned blocks_for(int64_t n) { return (unsigned)std::max<int64_t>(1, (n + kT - 1) / kT); }
inline int64_t pad8(int64_t b) { return (b + 7) & ~(int64_t)7; }

struct Header {
    uint64_t magic;
    uint32_t version, precision;
    int32_t n_species, nx0, ny0, max_level;
    double h0;
    int64_t nleaf, step, next_id;
    int32_t n_solves, pad_;
    double last_walls[4];
};
struct SpeciesHeader {
    int64_t n;
    int32_t present, sums_valid;
};

// Records of every leaf in list order into dense arrays (out0[L] = records before leaf L).
template <typename R>
__global__ void k_gather_records(int64_t nl, const int32_t *__restrict__ start, const int32_t *__restrict__ end,
                                 const int32_t *__restrict__ out0, SoA<R> d, SoA<R> o) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t L = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; L < nl; L += nw) {
        const int32_t p0 = start[L], p1 = end[L], o0 = out0[L];
        for (int32_t p = p0 + lane; p < p1; p += 32) {
            const int32_t q = o0 + (p - p0);
            o.u[q] = d.u[p]; o.v[q] = d.v[p]; o.vx[q] = d.vx[p]; o.vy[q] = d.vy[p]; o.vz[q] = d.vz[p];
            o.w[q] = d.w[p]; o.id[q] = d.id[p];
        }
    }
}

// Dense records (leaf-major, first[L] = records before leaf L) into the segments of fresh lists.
template <typename R>
__global__ void k_place_records(int64_t nl, const int32_t *__restrict__ first, const int32_t *__restrict__ start,
                                const int32_t *__restrict__ end, SoA<R> s, SoA<R> d) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t L = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; L < nl; L += nw) {
        const int32_t q0 = start[L], q1 = end[L], f0 = first[L];
        for (int32_t q = q0 + lane; q < q1; q += 32) {
            const int32_t p = f0 + (q - q0);
            d.u[q] = s.u[p]; d.v[q] = s.v[p]; d.vx[q] = s.vx[p]; d.vy[q] = s.vy[p]; d.vz[q] = s.vz[p];
            d.w[q] = s.w[p]; d.id[q] = s.id[p];
        }
    }
}

__global__ void k_leaf_counts(int64_t nl, const int32_t *__restrict__ start, const int32_t *__restrict__ end,
                              int32_t *__restrict__ cnt) {
    const int64_t L = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (L < nl) cnt[L] = end[L] - start[L];
}

template <typename R> SoA<R> dense_soa(DeviceArena &T, int64_t n) {
    SoA<R> o;
    o.u = dalloc<R>(T, n); o.v = dalloc<R>(T, n); o.vx = dalloc<R>(T, n); o.vy = dalloc<R>(T, n);
    o.vz = dalloc<R>(T, n); o.w = dalloc<R>(T, n); o.id = dalloc<uint32_t>(T, n);
    return o;
}

int64_t species_bytes(int64_t nl, int64_t n, size_t rs, bool sums) {
    return (int64_t)sizeof(SpeciesHeader) + pad8(4 * nl) + 6 * pad8(n * (int64_t)rs) + pad8(4 * n) +
           (sums ? 4 * pad8(nl * (int64_t)rs) : 0);
}

int64_t total_bytes(pic_ctx *ctx, Instance &in) {
    refresh_counts(ctx, in);
    const int64_t nl = in.nleaf;
    const size_t rs = in.cfg.precision == PIC_FP64 ? 8 : 4;
    int64_t b = (int64_t)sizeof(Header) + 2 * pad8(4 * nl) + pad8(nl) + 2 * 8 * nl;
    for (int s = 0; s < in.cfg.n_species; ++s) {
        const Species &sp = in.sp[s];
        b += species_bytes(nl, sp.start ? sp.n : 0, rs, sp.start && sp.sums_valid);
    }
    return b;
}

struct Writer {
    uint8_t *p;
    template <typename T> void put(const T &v) { std::memcpy(p, &v, sizeof(T)); p += sizeof(T); }
    void *take(int64_t bytes) { void *q = p; p += pad8(bytes); return q; }
};
struct Reader {
    const uint8_t *p, *end;
    template <typename T> T get() {
        if (p + sizeof(T) > end) fail(PIC_EINVAL, "checkpoint truncated");
        T v;
        std::memcpy(&v, p, sizeof(T));
        p += sizeof(T);
        return v;
    }
    const void *take(int64_t bytes) {
        if (bytes < 0 || p + pad8(bytes) > end) fail(PIC_EINVAL, "checkpoint truncated");
        const void *q = p;
        p += pad8(bytes);
        return q;
    }
};

template <typename R> void write_species(pic_ctx *ctx, Instance &in, int s, Writer &w) {
    cudaStream_t st = ctx->stream;
    Species &sp = in.sp[s];
    const int64_t nl = in.nleaf;
    SpeciesHeader h{sp.start ? sp.n : 0, sp.start ? 1 : 0, sp.start && sp.sums_valid ? 1 : 0};
    w.put(h);
    int32_t *cnt_h = (int32_t *)w.take(4 * nl);
    const int64_t n = h.n;
    R *arr_h[6];
    for (int k = 0; k < 6; ++k) arr_h[k] = (R *)w.take(n * (int64_t)sizeof(R));
    uint32_t *id_h = (uint32_t *)w.take(4 * n);
    void *sums_h[4] = {nullptr, nullptr, nullptr, nullptr};
    if (h.sums_valid)
        for (int k = 0; k < 4; ++k) sums_h[k] = w.take(nl * (int64_t)sizeof(R));
    if (!sp.start) {
        std::fill(cnt_h, cnt_h + nl, 0);
        return;
    }
    DeviceArena T(&ctx->cache);
    int32_t *cnt = dalloc<int32_t>(T, nl);
    k_leaf_counts<<<blocks_for(nl), kT, 0, st>>>(nl, sp.start, sp.end, cnt);
    count_launch(ctx);
    list_ranks(ctx, sp, nl);
    SoA<R> o = dense_soa<R>(T, n);
    k_gather_records<R><<<warp_blocks(nl), kT, 0, st>>>(nl, sp.start, sp.end, sp.rank0, soa<R>(sp, sp.cur), o);
    count_launch(ctx);
    check_launch("checkpoint_write");
    GB_CUDA(cudaMemcpyAsync(cnt_h, cnt, 4 * nl, cudaMemcpyDeviceToHost, st));
    R *src[6] = {o.u, o.v, o.vx, o.vy, o.vz, o.w};
    for (int k = 0; k < 6; ++k)
        if (n) GB_CUDA(cudaMemcpyAsync(arr_h[k], src[k], n * sizeof(R), cudaMemcpyDeviceToHost, st));
    if (n) GB_CUDA(cudaMemcpyAsync(id_h, o.id, 4 * n, cudaMemcpyDeviceToHost, st));
    if (h.sums_valid) {
        void *dev[4] = {sp.stay_hi, sp.stay_lo, sp.ent_hi, sp.ent_lo};
        for (int k = 0; k < 4; ++k)
            GB_CUDA(cudaMemcpyAsync(sums_h[k], dev[k], nl * sizeof(R), cudaMemcpyDeviceToHost, st));
    }
    GB_CUDA(cudaStreamSynchronize(st));
    T.release_all();
}

template <typename R> void read_species(pic_ctx *ctx, Instance &in, int s, Reader &r) {
    cudaStream_t st = ctx->stream;
    const int64_t nl = in.nleaf;
    const SpeciesHeader h = r.get<SpeciesHeader>();
    if (h.n < 0 || h.n >= (1ll << 31)) fail(PIC_EINVAL, "checkpoint: bad particle count");
    const int32_t *cnt_h = (const int32_t *)r.take(4 * nl);
    const int64_t n = h.n;
    const R *arr_h[6];
    for (int k = 0; k < 6; ++k) arr_h[k] = (const R *)r.take(n * (int64_t)sizeof(R));
    const uint32_t *id_h = (const uint32_t *)r.take(4 * n);
    const void *sums_h[4] = {nullptr, nullptr, nullptr, nullptr};
    if (h.sums_valid)
        for (int k = 0; k < 4; ++k) sums_h[k] = r.take(nl * (int64_t)sizeof(R));
    if (!h.present) return;
    int64_t total = 0;
    for (int64_t L = 0; L < nl; ++L) {
        if (cnt_h[L] < 0) fail(PIC_EINVAL, "checkpoint: negative leaf count");
        total += cnt_h[L];
    }
    if (total != n) fail(PIC_EINVAL, "checkpoint: leaf counts do not add up to the particle count");
    const pic_config &c = in.cfg;
    if (c.particle_capacity > 0 && c.particle_capacity < n) fail(PIC_ECAPACITY, "particle_capacity below the checkpoint's population");
    const int64_t cap = c.particle_capacity > 0 ? slots_for(c.particle_capacity, nl)
                                                : load_slots(n, nl);
    if (cap >= (1ll << 31) - 1) fail(PIC_ECAPACITY, "particle slots beyond 2^31");
    Species &sp = in.sp[s];
    species_alloc(ctx, in, s, cap);
    DeviceArena T(&ctx->cache);
    int32_t *cnt = dalloc<int32_t>(T, nl + 1), *first = dalloc<int32_t>(T, nl + 1);
    int32_t *scr = dalloc<int32_t>(T, scan_scratch_elems(nl));
    GB_CUDA(cudaMemcpyAsync(cnt, cnt_h, 4 * nl, cudaMemcpyHostToDevice, st));
    exclusive_scan_i32(ctx, cnt, first, nl, scr);
    lists_from_counts(ctx, sp, nl, cnt, sp.start, sp.end, sp.spawn_base + nl + 1);
    lists_installed(ctx, sp, nl);
    SoA<R> src = dense_soa<R>(T, n);
    R *dst[6] = {src.u, src.v, src.vx, src.vy, src.vz, src.w};
    for (int k = 0; k < 6; ++k)
        if (n) GB_CUDA(cudaMemcpyAsync(dst[k], arr_h[k], n * sizeof(R), cudaMemcpyHostToDevice, st));
    if (n) GB_CUDA(cudaMemcpyAsync(src.id, id_h, 4 * n, cudaMemcpyHostToDevice, st));
    k_place_records<R><<<warp_blocks(nl), kT, 0, st>>>(nl, first, sp.start, sp.end, src, soa<R>(sp, sp.cur));
    count_launch(ctx);
    check_launch("checkpoint_read");
    if (h.sums_valid) {
        void *dev[4] = {sp.stay_hi, sp.stay_lo, sp.ent_hi, sp.ent_lo};
        for (int k = 0; k < 4; ++k)
            GB_CUDA(cudaMemcpyAsync(dev[k], sums_h[k], nl * sizeof(R), cudaMemcpyHostToDevice, st));
        sp.sums_valid = true;
    }
    GB_CUDA(cudaStreamSynchronize(st));
    T.release_all();
    sp.n = n;
    sp.n_upper = n;
}
}  // namespace

int64_t checkpoint_write(pic_ctx *ctx, Instance &in, void *buf, int64_t cap) {
    const int64_t need = total_bytes(ctx, in);
    if (!buf || cap < need) return need;
    cudaStream_t st = ctx->stream;
    const int64_t nl = in.nleaf;
    Writer w{static_cast<uint8_t *>(buf)};
    std::memset(buf, 0, (size_t)need);
    Header h{};
    h.magic = kMagic;
    h.version = kVersion;
    h.precision = (uint32_t)in.cfg.precision;
    h.n_species = in.cfg.n_species;
    h.nx0 = in.nx0; h.ny0 = in.ny0; h.max_level = in.lmax;
    h.h0 = in.h0;
    h.nleaf = nl;
    h.step = ctx->step;
    unsigned long long nid = 0;
    GB_CUDA(cudaMemcpyAsync(&nid, in.d_next_id, 8, cudaMemcpyDeviceToHost, st));
    int32_t ns = in.n_solves;
    if (in.d_n_solves) GB_CUDA(cudaMemcpyAsync(&ns, in.d_n_solves, 4, cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaStreamSynchronize(st));
    h.next_id = (int64_t)nid;
    h.n_solves = ns;
    for (int k = 0; k < 4; ++k) h.last_walls[k] = in.last_walls[k];
    w.put(h);
    void *root = w.take(4 * nl), *mort = w.take(4 * nl), *lev = w.take(nl);
    void *phi = w.take(8 * nl), *prev = w.take(8 * nl);
    GB_CUDA(cudaMemcpyAsync(root, in.root, 4 * nl, cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaMemcpyAsync(mort, in.morton, 4 * nl, cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaMemcpyAsync(lev, in.lv[0].lev, nl, cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaMemcpyAsync(phi, in.phi, 8 * nl, cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaMemcpyAsync(prev, in.phi_prev, 8 * nl, cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaStreamSynchronize(st));
    for (int s = 0; s < in.cfg.n_species; ++s) {
        if (in.cfg.precision == PIC_FP64) write_species<double>(ctx, in, s, w);
        else write_species<float>(ctx, in, s, w);
    }
    return need;
}

void checkpoint_read(pic_ctx *ctx, Instance &in, const void *buf, int64_t bytes) {
    if (!buf || bytes < (int64_t)sizeof(Header)) fail(PIC_EINVAL, "checkpoint: buffer too small");
    Reader r{static_cast<const uint8_t *>(buf), static_cast<const uint8_t *>(buf) + bytes};
    const Header h = r.get<Header>();
    if (h.magic != kMagic || h.version != kVersion) fail(PIC_EINVAL, "checkpoint: not a gbpic checkpoint of this version");
    if ((int32_t)h.precision != in.cfg.precision || h.n_species != in.cfg.n_species)
        fail(PIC_EINVAL, "checkpoint: precision or species count differs from the instance's configuration");
    if (h.max_level != in.cfg.max_level) fail(PIC_EINVAL, "checkpoint: max_level differs from the configuration");
    if (h.nx0 < 1 || h.ny0 < 1 || !(h.h0 > 0.0) || h.nleaf < 1 || h.nleaf >= (1ll << 30) || h.step < 0 || h.next_id < 0)
        fail(PIC_EINVAL, "checkpoint: bad header");
    const int64_t nl = h.nleaf;
    const uint32_t *root = (const uint32_t *)r.take(4 * nl);
    const uint32_t *mort = (const uint32_t *)r.take(4 * nl);
    const uint8_t *lev = (const uint8_t *)r.take(nl);
    const double *phi = (const double *)r.take(8 * nl);
    const double *prev = (const double *)r.take(8 * nl);
    for (int64_t i = 0; i < nl; ++i)
        if (lev[i] > in.cfg.max_level) fail(PIC_EINVAL, "checkpoint: leaf level above max_level");
    set_mesh_impl(ctx, in, h.nx0, h.ny0, h.h0, nl, root, mort, lev);
    if (in.nleaf != nl) fail(PIC_EINVAL, "checkpoint: mesh size changed on rebuild");
    cudaStream_t st = ctx->stream;
    GB_CUDA(cudaMemcpyAsync(in.phi, phi, 8 * nl, cudaMemcpyHostToDevice, st));
    GB_CUDA(cudaMemcpyAsync(in.phi_prev, prev, 8 * nl, cudaMemcpyHostToDevice, st));
    in.n_solves = h.n_solves;
    if (in.d_n_solves) GB_CUDA(cudaMemcpyAsync(in.d_n_solves, &h.n_solves, 4, cudaMemcpyHostToDevice, st));
    for (int k = 0; k < 4; ++k) in.last_walls[k] = h.last_walls[k];
    for (int s = 0; s < in.cfg.n_species; ++s) {
        if (in.cfg.precision == PIC_FP64) read_species<double>(ctx, in, s, r);
        else read_species<float>(ctx, in, s, r);
    }
    unsigned long long nid = (unsigned long long)h.next_id;
    GB_CUDA(cudaMemcpyAsync(in.d_next_id, &nid, 8, cudaMemcpyHostToDevice, st));
    GB_CUDA(cudaStreamSynchronize(st));
    in.next_id = h.next_id;
    ctx->step = h.step;
}

}  // namespace gbpic
