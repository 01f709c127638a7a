// Cell lists with free slots (§3.1: each leaf keeps the list of its particles; a particle
// that crosses a face leaves its list and joins the neighbour's).
//
// Leaf L of a species owns the slot segment [start[L], lim[L]) of the species' buffers.
// Its records are [start[L], end[L]) in list order; the free slots [end[L], lim[L]) receive
// the particles that enter L during a step, so one push pass updates every list in place.
// Entering records that find no free slot left go to the overflow store, and their leaf
// moves to a fresh segment at the tail of the buffer (past every segment in use) with room
// for them.  Only when the tail is used up are all lists of the species laid out again, in
// leaf order with fresh free slots.  Both repairs sit behind IF nodes of a CUDA graph whose
// conditions a one-thread kernel sets from the device's overflow flags, so a step without
// overflow costs two tiny kernels and the host never waits; the order of records inside a
// list never depends on where its segment lies (order keys are list ranks, not slot numbers).
//
// This file holds the allocation of a species' buffers, the construction of segments from
// per-leaf counts, list ranks and record totals, and the two repairs.
#include <algorithm>
#include <cstring>

#include "pic_internal.cuh"

namespace gbpic {

namespace {
constexpr int kT = 256;
inline unsigned blocks_for(int64_t n, int t = kT) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }
inline unsigned warp_blocks(int64_t nw) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((nw + kT / 32 - 1) / (kT / 32), 1 << 20));
}

// seg[L] = c + list_slack(c) with c = a[L] (+ b[L]); with `room` (a re-layout: b = this
// step's entering records) the leaf also keeps room for one more step of that inflow.
__device__ __forceinline__ void seg_sizes(int64_t nl, const int32_t *__restrict__ a, const int32_t *__restrict__ b,
                                          int room, int32_t *__restrict__ seg, const int32_t *__restrict__ gate,
                                          int64_t i0, int64_t stride) {
    if (gate && *gate == 0) return;
    for (int64_t L = i0; L < nl; L += stride) {
        const int32_t c = a[L] + (b ? b[L] : 0);
        seg[L] = c + list_slack(c) + (room ? b[L] : 0);
    }
}
__global__ void k_seg_sizes(int64_t nl, const int32_t *__restrict__ a, const int32_t *__restrict__ b, int room,
                            int32_t *__restrict__ seg, const int32_t *__restrict__ gate) {
    seg_sizes(nl, a, b, room, seg, gate, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
              (int64_t)gridDim.x * blockDim.x);
}

// A re-layout whose inflow room does not fit the buffer lays out without it (flags[7]).
__global__ void k_relayout_fit(const int32_t *__restrict__ start_new, int64_t nl, int64_t cap,
                               int32_t *__restrict__ flags) {
    if (threadIdx.x == 0 && blockIdx.x == 0) flags[7] = (flags[5] && (int64_t)start_new[nl] > cap) ? 1 : 0;
}

// end[L] = start[L] + c[L]
__global__ void k_set_end(int64_t nl, const int32_t *__restrict__ start, const int32_t *__restrict__ cnt,
                          int32_t *__restrict__ end) {
    const int64_t L = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (L < nl) end[L] = start[L] + cnt[L];
}

// Segments in leaf order: lim[L] = start[L + 1]; the tail starts at start[nl].
__global__ void k_lists_installed(int64_t nl, const int32_t *__restrict__ start, int32_t *__restrict__ lim,
                                  int32_t *__restrict__ flags) {
    const int64_t L = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (L < nl) lim[L] = start[L + 1];
    if (L == 0) {
        flags[4] = start[nl];
        flags[5] = 0;
    }
}

__global__ void k_list_counts(int64_t nl, const int32_t *__restrict__ start, const int32_t *__restrict__ end,
                              int32_t *__restrict__ cnt) {
    const int64_t L = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (L < nl) cnt[L] = end[L] - start[L];
}

// total[0] += sum over leaves of end - start
__global__ void k_count_total(int64_t nl, const int32_t *__restrict__ start, const int32_t *__restrict__ end,
                              int32_t *__restrict__ total) {
    __shared__ int32_t part[kT / 32];
    int32_t s = 0;
    for (int64_t L = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; L < nl; L += (int64_t)gridDim.x * blockDim.x)
        s += end[L] - start[L];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
        atomicAdd(total, t);
    }
}

template <typename R>
__device__ __forceinline__ void copy_record(SoA<R> t, int64_t q, SoA<R> d, int64_t p) {
    t.u[q] = d.u[p]; t.v[q] = d.v[p]; t.vx[q] = d.vx[p]; t.vy[q] = d.vy[p]; t.vz[q] = d.vz[p];
    t.w[q] = d.w[p]; t.id[q] = d.id[p];
}

// Repair 1 (one warp per leaf that ran out of free slots): a segment at the tail with room
// for its staying and entering records and free slots, the staying records and the entering
// records already in free slots copied there.  A leaf that does not fit any more marks the
// tail as used up (flags[5]) and keeps its segment; the re-layout then takes over.
// The warp takes the moved leaves warp, warp + nw, ...
template <typename R>
__device__ __forceinline__ void move_to_tail(const int32_t *__restrict__ moved, int64_t nl, int64_t cap,
                                             int32_t *__restrict__ start, int32_t *__restrict__ end,
                                             int32_t *__restrict__ lim, const int32_t *__restrict__ stay,
                                             const int32_t *__restrict__ fill, SoA<R> d, uint32_t *__restrict__ key,
                                             uint32_t *__restrict__ aux, int32_t *__restrict__ flags, int64_t warp,
                                             int64_t nw) {
    if (flags[0] == 0) return;
    const int lane = threadIdx.x & 31;
    const int32_t nm = moved[nl];
    for (int64_t i = warp; i < nm; i += nw) {
        const int32_t L = moved[i];
        const int32_t ns = stay[L], f = fill[L], c = ns + f;
        const int32_t need = c + list_slack(c) + f;
        int32_t base = 0;
        if (lane == 0) base = atomicAdd(flags + 4, need);
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        if ((int64_t)base + need > cap) {
            if (lane == 0) flags[5] = 1;
            continue;
        }
        const int32_t s0 = start[L], e0 = end[L], room = lim[L] - e0;
        for (int32_t j = lane; j < ns; j += 32) copy_record(d, base + j, d, s0 + j);
        for (int32_t j = lane; j < room; j += 32) {
            copy_record(d, base + ns + j, d, e0 + j);
            key[base + ns + j] = key[e0 + j];
            aux[base + ns + j] = aux[e0 + j];
        }
        __syncwarp();
        if (lane == 0) {
            start[L] = base;
            end[L] = base + ns;
            lim[L] = base + need;
        }
    }
}
template <typename R>
__global__ void k_move_to_tail(const int32_t *__restrict__ moved, int64_t nl, int64_t cap,
                               int32_t *__restrict__ start, int32_t *__restrict__ end, int32_t *__restrict__ lim,
                               const int32_t *__restrict__ stay, const int32_t *__restrict__ fill, SoA<R> d,
                               uint32_t *__restrict__ key, uint32_t *__restrict__ aux, int32_t *__restrict__ flags) {
    move_to_tail<R>(moved, nl, cap, start, end, lim, stay, fill, d, key, aux, flags,
                    ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5, ((int64_t)gridDim.x * blockDim.x) >> 5);
}

// Repair 2: the overflow store's records join their moved leaf at their slot.
// The thread takes the records i0, i0 + stride, ...; `first` does the statistics.
template <typename R>
__device__ __forceinline__ void place_ovf(const int32_t *__restrict__ end, int64_t cap, SoA<R> o,
                                          const uint32_t *__restrict__ okey, const uint32_t *__restrict__ oaux,
                                          const int32_t *__restrict__ odest, const int32_t *__restrict__ oslot,
                                          SoA<R> d, uint32_t *__restrict__ key, uint32_t *__restrict__ aux,
                                          const int32_t *__restrict__ moved, int64_t nl, int32_t *__restrict__ flags,
                                          int64_t i0, int64_t stride, bool first) {
    const int32_t n = flags[0] < cap ? flags[0] : (int32_t)cap;  // beyond cap: err is set already
    if (n == 0) return;
    if (first) {  // statistics
        flags[3] += n;
        flags[6] += moved[nl];
    }
    if (flags[5]) return;  // the re-layout places them
    for (int64_t i = i0; i < n; i += stride) {
        const int32_t q = end[odest[i]] + oslot[i];
        copy_record(d, q, o, i);
        key[q] = okey[i];
        aux[q] = oaux[i];
    }
}
template <typename R>
__global__ void k_place_ovf(const int32_t *__restrict__ end, int64_t cap, SoA<R> o, const uint32_t *__restrict__ okey,
                            const uint32_t *__restrict__ oaux, const int32_t *__restrict__ odest,
                            const int32_t *__restrict__ oslot, SoA<R> d, uint32_t *__restrict__ key,
                            uint32_t *__restrict__ aux, const int32_t *__restrict__ moved, int64_t nl,
                            int32_t *__restrict__ flags) {
    place_ovf<R>(end, cap, o, okey, oaux, odest, oslot, d, key, aux, moved, nl, flags,
                 (int64_t)blockIdx.x * blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x,
                 blockIdx.x == 0 && threadIdx.x == 0);
}

// Re-layout, step 1 (one warp per leaf): the staying records and the entering records that
// found a free slot go to the scratch buffer at the new segment starts; staying records
// first, entering records at their slot after them.
template <typename R>
__device__ __forceinline__ void relayout_move(int64_t nl, const int32_t *__restrict__ start,
                                              const int32_t *__restrict__ end, const int32_t *__restrict__ lim,
                                              const int32_t *__restrict__ stay, const int32_t *__restrict__ fill,
                                              const int32_t *__restrict__ start_new, int64_t cap, SoA<R> d,
                                              const uint32_t *__restrict__ key, const uint32_t *__restrict__ aux,
                                              SoA<R> t, uint32_t *__restrict__ tkey, uint32_t *__restrict__ taux,
                                              const int32_t *__restrict__ flags, int32_t *__restrict__ err,
                                              int64_t warp, int64_t nw, bool first) {
    if (flags[5] == 0) return;
    if ((int64_t)start_new[nl] > cap) {
        if (first) atomicExch(err, 1);
        return;
    }
    const int lane = threadIdx.x & 31;
    for (int64_t L = warp; L < nl; L += nw) {
        const int32_t s0 = start[L], q0 = start_new[L], ns = stay[L];
        for (int32_t j = lane; j < ns; j += 32) copy_record(t, q0 + j, d, s0 + j);
        const int32_t e0 = end[L], room = lim[L] - e0;
        const int32_t k = fill[L] < room ? fill[L] : room;
        for (int32_t j = lane; j < k; j += 32) {
            const int32_t p = e0 + j, q = q0 + ns + j;
            copy_record(t, q, d, p);
            tkey[q] = key[p]; taux[q] = aux[p];
        }
    }
}
template <typename R>
__global__ void k_relayout_move(int64_t nl, const int32_t *__restrict__ start, const int32_t *__restrict__ end,
                                const int32_t *__restrict__ lim, const int32_t *__restrict__ stay,
                                const int32_t *__restrict__ fill, const int32_t *__restrict__ start_new, int64_t cap,
                                SoA<R> d, const uint32_t *__restrict__ key, const uint32_t *__restrict__ aux,
                                SoA<R> t, uint32_t *__restrict__ tkey, uint32_t *__restrict__ taux,
                                const int32_t *__restrict__ flags, int32_t *__restrict__ err) {
    relayout_move<R>(nl, start, end, lim, stay, fill, start_new, cap, d, key, aux, t, tkey, taux, flags, err,
                     ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5, ((int64_t)gridDim.x * blockDim.x) >> 5,
                     blockIdx.x == 0 && threadIdx.x == 0);
}

// Re-layout, step 2: the records of the overflow store join them at their slot.
template <typename R>
__device__ __forceinline__ void relayout_ovf(const int32_t *__restrict__ stay, const int32_t *__restrict__ start_new,
                                             int64_t nl, int64_t cap, SoA<R> o, const uint32_t *__restrict__ okey,
                                             const uint32_t *__restrict__ oaux, const int32_t *__restrict__ odest,
                                             const int32_t *__restrict__ oslot, SoA<R> t,
                                             uint32_t *__restrict__ tkey, uint32_t *__restrict__ taux,
                                             const int32_t *__restrict__ flags, int64_t i0, int64_t stride) {
    if (flags[5] == 0) return;
    const int32_t n = flags[0] < cap ? flags[0] : (int32_t)cap;
    if ((int64_t)start_new[nl] > cap) return;
    for (int64_t i = i0; i < n; i += stride) {
        const int32_t L = odest[i];
        const int32_t q = start_new[L] + stay[L] + oslot[i];
        copy_record(t, q, o, i);
        tkey[q] = okey[i]; taux[q] = oaux[i];
    }
}
template <typename R>
__global__ void k_relayout_ovf(const int32_t *__restrict__ stay, const int32_t *__restrict__ start_new, int64_t nl,
                               int64_t cap, SoA<R> o, const uint32_t *__restrict__ okey,
                               const uint32_t *__restrict__ oaux, const int32_t *__restrict__ odest,
                               const int32_t *__restrict__ oslot, SoA<R> t, uint32_t *__restrict__ tkey,
                               uint32_t *__restrict__ taux, const int32_t *__restrict__ flags) {
    relayout_ovf<R>(stay, start_new, nl, cap, o, okey, oaux, odest, oslot, t, tkey, taux, flags,
                    (int64_t)blockIdx.x * blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
}

// Re-layout, step 3: the scratch buffer back into the lists, the new segments, and end[L] at
// the first entering record (where the entering sort expects it).
template <typename R>
__device__ __forceinline__ void relayout_back(int64_t nl, const int32_t *__restrict__ start_new,
                                              const int32_t *__restrict__ stay, int64_t cap, SoA<R> t,
                                              const uint32_t *__restrict__ tkey, const uint32_t *__restrict__ taux,
                                              SoA<R> d, uint32_t *__restrict__ key, uint32_t *__restrict__ aux,
                                              int32_t *__restrict__ start, int32_t *__restrict__ end,
                                              int32_t *__restrict__ lim, int32_t *__restrict__ flags, int64_t i0,
                                              int64_t stride, bool first) {
    if (flags[5] == 0) return;
    const int64_t span = start_new[nl];
    if (span > cap) return;
    for (int64_t i = i0; i < span; i += stride) {
        copy_record(d, i, t, i);
        key[i] = tkey[i]; aux[i] = taux[i];
    }
    for (int64_t L = i0; L <= nl; L += stride) {
        start[L] = start_new[L];
        if (L < nl) {
            end[L] = start_new[L] + stay[L];
            lim[L] = start_new[L + 1];
        }
    }
    if (first) {
        flags[2] += 1;  // statistics
        flags[4] = (int32_t)span;
    }
}
template <typename R>
__global__ void k_relayout_back(int64_t nl, const int32_t *__restrict__ start_new, const int32_t *__restrict__ stay,
                                int64_t cap, SoA<R> t, const uint32_t *__restrict__ tkey,
                                const uint32_t *__restrict__ taux, SoA<R> d, uint32_t *__restrict__ key,
                                uint32_t *__restrict__ aux, int32_t *__restrict__ start, int32_t *__restrict__ end,
                                int32_t *__restrict__ lim, int32_t *__restrict__ flags) {
    relayout_back<R>(nl, start_new, stay, cap, t, tkey, taux, d, key, aux, start, end, lim, flags,
                     (int64_t)blockIdx.x * blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x,
                     blockIdx.x == 0 && threadIdx.x == 0);
}

// Every list of species s laid out again in leaf order with fresh free slots (the kernels
// return at once unless flags[5] is set).
template <typename R> void relayout_lists(pic_ctx *ctx, Instance &in, int s) {
    Species &sp = in.sp[s];
    cudaStream_t st = ctx->stream;
    const int64_t nl = in.nleaf;
    const SoA<R> d = soa<R>(sp, sp.cur), t = soa<R>(sp, sp.cur ^ 1);
    int32_t *scr = sp.spawn_base + nl + 1 + scan_scratch_elems(nl);
    // gated launches get small grids: a launch that returns at once still schedules every block
    const unsigned gb = std::min<unsigned>(blocks_for(nl), 152u * 2u);
    k_seg_sizes<<<gb, kT, 0, st>>>(nl, sp.stay, sp.fill, 1, sp.inc, sp.flags + 5);
    exclusive_scan_i32(ctx, sp.inc, sp.start_new, nl, scr, sp.flags + 5);
    k_relayout_fit<<<1, 32, 0, st>>>(sp.start_new, nl, sp.cap, sp.flags);
    k_seg_sizes<<<gb, kT, 0, st>>>(nl, sp.stay, sp.fill, 0, sp.inc, sp.flags + 7);
    exclusive_scan_i32(ctx, sp.inc, sp.start_new, nl, scr, sp.flags + 7);
    uint32_t *tkey = sp.key + sp.cap, *taux = sp.aux + sp.cap;
    k_relayout_move<R><<<std::min<unsigned>(warp_blocks(nl), 152u * 8u), kT, 0, st>>>(
        nl, sp.start, sp.end, sp.lim, sp.stay, sp.fill, sp.start_new, sp.cap, d, sp.key, sp.aux, t, tkey, taux,
        sp.flags, in.d_err);
    k_relayout_ovf<R><<<152 * 4, kT, 0, st>>>(sp.stay, sp.start_new, nl, sp.cap, soa_ovf<R>(sp), sp.ovf_key,
                                              sp.ovf_aux, sp.ovf_dest, sp.ovf_slot, t, tkey, taux, sp.flags);
    k_relayout_back<R><<<152 * 8, kT, 0, st>>>(nl, sp.start_new, sp.stay, sp.cap, t, tkey, taux, d, sp.key, sp.aux,
                                               sp.start, sp.end, sp.lim, sp.flags);
    count_launch(ctx, 6);
    check_launch("relayout_lists");
}

__global__ void k_set_if(cudaGraphConditionalHandle h, const int32_t *__restrict__ value) {
    if (threadIdx.x == 0 && blockIdx.x == 0) cudaGraphSetConditional(h, *value != 0 ? 1u : 0u);
}

// The repairs after a push, as two IF nodes so that a step without overflow runs two
// one-thread kernels instead of a dozen launches that return at once: records in the
// overflow store (flags[0]) -> move their leaves to the tail and place them; tail used up
// (flags[5]) -> lay every list out again.
template <typename R> void capture_repairs(pic_ctx *ctx, Instance &in, int s, cudaStream_t st) {
    Species &sp = in.sp[s];
    const int64_t nl = in.nleaf;
    capture_if(ctx, st, sp.flags + 0, [&]() {
        const SoA<R> d = soa<R>(sp, sp.cur);
        const SoA<R> o = soa_ovf<R>(sp);
        k_move_to_tail<R><<<152 * 4, kT, 0, ctx->stream>>>(sp.moved, nl, sp.cap, sp.start, sp.end, sp.lim, sp.stay,
                                                           sp.fill, d, sp.key, sp.aux, sp.flags);
        k_place_ovf<R><<<152 * 2, kT, 0, ctx->stream>>>(sp.end, sp.cap, o, sp.ovf_key, sp.ovf_aux, sp.ovf_dest,
                                                        sp.ovf_slot, d, sp.key, sp.aux, sp.moved, nl, sp.flags);
    });
    capture_if(ctx, st, sp.flags + 5, [&]() { relayout_lists<R>(ctx, in, s); });
}

template <typename R> void place_impl(pic_ctx *ctx, Instance &in, int s) {
    Species &sp = in.sp[s];
    if (ctx->capturing) {  // inside a captured step: the IF nodes go into that graph
        capture_repairs<R>(ctx, in, s, ctx->stream);
        count_launch(ctx, 2);
        return;
    }
    if (!sp.repair || sp.repair_mesh_epoch != ctx->mesh_epoch || sp.repair_lists_epoch != ctx->lists_epoch) {
        if (sp.repair) {
            cudaGraphExecDestroy(sp.repair);
            sp.repair = nullptr;
        }
        cudaStream_t cs;
        GB_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaStream_t saved = ctx->stream;
        const int64_t l0 = ctx->launches;
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        try {
            if (e != cudaSuccess) GB_CUDA(e);
            ctx->stream = cs;
            capture_repairs<R>(ctx, in, s, cs);
            ctx->stream = saved;
            e = cudaStreamEndCapture(cs, &g);
        } catch (...) {
            ctx->stream = saved;
            cudaStreamEndCapture(cs, &g);
            if (g) cudaGraphDestroy(g);
            ctx->launches = l0;
            cudaStreamDestroy(cs);
            throw;
        }
        ctx->launches = l0;
        cudaStreamDestroy(cs);
        if (e == cudaSuccess) e = cudaGraphInstantiate(&sp.repair, g, 0);
        if (g) cudaGraphDestroy(g);
        GB_CUDA(e);
        sp.repair_mesh_epoch = ctx->mesh_epoch;
        sp.repair_lists_epoch = ctx->lists_epoch;
    }
    GB_CUDA(cudaGraphLaunch(sp.repair, ctx->stream));
    count_launch(ctx, 2);  // the two condition kernels (the bodies run only when needed)
}

// Host-driven compaction: every record counts as staying, nothing enters.
__global__ void k_compact_prep(int64_t nl, const int32_t *__restrict__ start, const int32_t *__restrict__ end,
                               int32_t *__restrict__ stay, int32_t *__restrict__ fill, int32_t *__restrict__ flags) {
    const int64_t L = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (L < nl) {
        stay[L] = end[L] - start[L];
        fill[L] = 0;
    }
    if (L == 0) {
        flags[0] = 0;
        flags[5] = 1;
    }
}
__global__ void k_compact_done(int32_t *__restrict__ flags) {
    if (threadIdx.x == 0 && blockIdx.x == 0) flags[5] = 0;
}

// ---- the batched ensemble step: one entry per (instance, species) ------------------------
struct ListEntry {
    int64_t nl, cap;
    int32_t *start, *end, *lim, *stay, *fill, *flags, *moved, *inc;
    int32_t *spawn;  // ionizing electrons: spawn counts per leaf (else null)
    void *d[7], *o[7];  // record arrays of the current buffer and of the overflow store (id last)
    uint32_t *key, *aux, *okey, *oaux;
    int32_t *odest, *oslot;
    // the re-layout: new segment starts, the other buffer as scratch, the error flag
    int32_t *start_new, *err;
    void *t[7];
    uint32_t *tkey, *taux;
};
template <typename R> __device__ __forceinline__ SoA<R> soa_of(void *const p[7]) {
    SoA<R> a;
    a.u = (R *)p[0]; a.v = (R *)p[1]; a.vx = (R *)p[2]; a.vy = (R *)p[3]; a.vz = (R *)p[4]; a.w = (R *)p[5];
    a.id = (uint32_t *)p[6];
    return a;
}

// Before the pushes, per entry: what k_step_reset clears, and the record counts whose scan
// gives the list ranks (block = leaves [c.y, c.z) of entry c.x).
__global__ void k_lists_prep_batch(const ListEntry *__restrict__ tab, const int4 *__restrict__ chunks) {
    const int4 c = chunks[blockIdx.x];
    const ListEntry &e = tab[c.x];
    const int64_t L = (int64_t)c.y + threadIdx.x;
    if (L < c.z) {
        e.fill[L] = 0;
        if (e.spawn) e.spawn[L] = 0;
        e.inc[L] = e.end[L] - e.start[L];
    }
    if (L == 0) {
        e.flags[0] = 0;
        e.flags[5] = 0;
        e.moved[e.nl] = 0;
    }
}

// *out = 1 if flags[word] of any entry is nonzero, else 0 (one block).
__global__ void k_any_flag(const ListEntry *__restrict__ tab, int n, int word, int32_t *__restrict__ out) {
    int32_t any = 0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) any |= tab[i].flags[word] != 0 ? 1 : 0;
    any = __syncthreads_or(any);
    if (threadIdx.x == 0) *out = any;
}

// Repair 1 of every entry (blocks (x, entry)); entries without overflow return at once.
template <typename R> __global__ void k_move_to_tail_batch(const ListEntry *__restrict__ tab) {
    const ListEntry &e = tab[blockIdx.y];
    move_to_tail<R>(e.moved, e.nl, e.cap, e.start, e.end, e.lim, e.stay, e.fill, soa_of<R>(e.d), e.key, e.aux,
                    e.flags, ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5,
                    ((int64_t)gridDim.x * blockDim.x) >> 5);
}
template <typename R> __global__ void k_place_ovf_batch(const ListEntry *__restrict__ tab) {
    const ListEntry &e = tab[blockIdx.y];
    place_ovf<R>(e.end, e.cap, soa_of<R>(e.o), e.okey, e.oaux, e.odest, e.oslot, soa_of<R>(e.d), e.key, e.aux,
                 e.moved, e.nl, e.flags, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                 (int64_t)gridDim.x * blockDim.x, blockIdx.x == 0 && threadIdx.x == 0);
}

// The re-layout of every entry whose tail was used up (flags[5]); blocks (x, entry), the
// other entries return at once.  Same steps as relayout_lists.
__global__ void k_seg_sizes_batch(const ListEntry *__restrict__ tab, int room, int gate_word) {
    const ListEntry &e = tab[blockIdx.y];
    seg_sizes(e.nl, e.stay, e.fill, room, e.inc, e.flags + gate_word,
              (int64_t)blockIdx.x * blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
}
__global__ void k_relayout_fit_batch(const ListEntry *__restrict__ tab, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const ListEntry &e = tab[i];
        e.flags[7] = (e.flags[5] && (int64_t)e.start_new[e.nl] > e.cap) ? 1 : 0;
    }
}
template <typename R> __global__ void k_relayout_move_batch(const ListEntry *__restrict__ tab) {
    const ListEntry &e = tab[blockIdx.y];
    relayout_move<R>(e.nl, e.start, e.end, e.lim, e.stay, e.fill, e.start_new, e.cap, soa_of<R>(e.d), e.key, e.aux,
                     soa_of<R>(e.t), e.tkey, e.taux, e.flags, e.err,
                     ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5, ((int64_t)gridDim.x * blockDim.x) >> 5,
                     blockIdx.x == 0 && threadIdx.x == 0);
}
template <typename R> __global__ void k_relayout_ovf_batch(const ListEntry *__restrict__ tab) {
    const ListEntry &e = tab[blockIdx.y];
    relayout_ovf<R>(e.stay, e.start_new, e.nl, e.cap, soa_of<R>(e.o), e.okey, e.oaux, e.odest, e.oslot,
                    soa_of<R>(e.t), e.tkey, e.taux, e.flags, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                    (int64_t)gridDim.x * blockDim.x);
}
template <typename R> __global__ void k_relayout_back_batch(const ListEntry *__restrict__ tab) {
    const ListEntry &e = tab[blockIdx.y];
    relayout_back<R>(e.nl, e.start_new, e.stay, e.cap, soa_of<R>(e.t), e.tkey, e.taux, soa_of<R>(e.d), e.key, e.aux,
                     e.start, e.end, e.lim, e.flags, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                     (int64_t)gridDim.x * blockDim.x, blockIdx.x == 0 && threadIdx.x == 0);
}

template <typename R> void relayout_batch(pic_ctx *ctx) {
    const BatchTab &t = ctx->batch.lists;
    const ListEntry *tab = (const ListEntry *)t.tab;
    const unsigned n = (unsigned)t.n;
    cudaStream_t st = ctx->stream;
    // x blocks per entry: a re-laid-out species keeps 64 blocks busy (the other entries'
    // blocks return at once), so a few entries at a time still fill the GPU
    k_seg_sizes_batch<<<dim3(16, n), kT, 0, st>>>(tab, 1, 5);
    exclusive_scan_i32_batch(ctx, ctx->batch.relay5);
    k_relayout_fit_batch<<<(n + kT - 1) / kT, kT, 0, st>>>(tab, (int)n);
    k_seg_sizes_batch<<<dim3(16, n), kT, 0, st>>>(tab, 0, 7);
    exclusive_scan_i32_batch(ctx, ctx->batch.relay7);
    k_relayout_move_batch<R><<<dim3(64, n), kT, 0, st>>>(tab);
    k_relayout_ovf_batch<R><<<dim3(16, n), kT, 0, st>>>(tab);
    k_relayout_back_batch<R><<<dim3(64, n), kT, 0, st>>>(tab);
    count_launch(ctx, 6);
}

template <typename R> void repairs_batch_impl(pic_ctx *ctx) {
    const BatchTab &t = ctx->batch.lists;
    const ListEntry *tab = (const ListEntry *)t.tab;
    int32_t *flag = ctx->batch.flag;
    k_any_flag<<<1, kT, 0, ctx->stream>>>(tab, t.n, 0, flag);
    count_launch(ctx);
    capture_if(ctx, ctx->stream, flag, [&]() {
        k_move_to_tail_batch<R><<<dim3(8, (unsigned)t.n), kT, 0, ctx->stream>>>(tab);
        k_place_ovf_batch<R><<<dim3(8, (unsigned)t.n), kT, 0, ctx->stream>>>(tab);
        // a tail used up: those species' lists are laid out again
        k_any_flag<<<1, kT, 0, ctx->stream>>>(tab, t.n, 5, flag + 1);
        capture_if(ctx, ctx->stream, flag + 1, [&]() { relayout_batch<R>(ctx); });
    });
    count_launch(ctx);
}
}  // namespace

// Entries (instance, species) in instance order, and the prep blocks over their leaves.
BatchTab batch_prepare_lists(pic_ctx *ctx) {
    std::vector<ListEntry> tab;
    std::vector<int64_t> nls;
    for (Instance &in : ctx->inst) {
        const bool ionize = in.cfg.mcc && in.cfg.sigma_iz0 > 0.0;
        for (int s = 0; s < in.cfg.n_species; ++s) {
            Species &sp = in.sp[s];
            ListEntry e{};
            e.nl = in.nleaf;
            e.cap = sp.cap;
            e.start = sp.start; e.end = sp.end; e.lim = sp.lim; e.stay = sp.stay; e.fill = sp.fill;
            e.flags = sp.flags; e.moved = sp.moved; e.inc = sp.inc;
            e.spawn = s == 0 && ionize ? sp.spawn : nullptr;
            for (int k = 0; k < 6; ++k) {
                e.d[k] = sp.arr[sp.cur][k];
                e.o[k] = sp.ovf[k];
            }
            e.d[6] = sp.id[sp.cur];
            e.o[6] = sp.ovf_id;
            e.key = sp.key; e.aux = sp.aux; e.okey = sp.ovf_key; e.oaux = sp.ovf_aux;
            e.odest = sp.ovf_dest; e.oslot = sp.ovf_slot;
            e.start_new = sp.start_new;
            e.err = in.d_err;
            for (int k = 0; k < 6; ++k) e.t[k] = sp.arr[sp.cur ^ 1][k];
            e.t[6] = sp.id[sp.cur ^ 1];
            e.tkey = sp.key + sp.cap;
            e.taux = sp.aux + sp.cap;
            tab.push_back(e);
            nls.push_back(in.nleaf);
        }
    }
    // the re-layout's two gated scans of the new segment sizes
    std::vector<const int32_t *> in;
    std::vector<int32_t *> out;
    std::vector<const int32_t *> g5, g7;
    for (const ListEntry &e : tab) {
        in.push_back(e.inc);
        out.push_back(e.start_new);
        g5.push_back(e.flags + 5);
        g7.push_back(e.flags + 7);
    }
    ctx->batch.relay5 = scan_plan(ctx, in, out, nls, g5);
    ctx->batch.relay7 = scan_plan(ctx, in, out, nls, g7);
    const std::vector<int4> ch = batch_chunks(nls, kT);
    BatchTab t;
    t.tab = batch_upload(ctx, tab);
    t.chunks = batch_upload(ctx, ch);
    t.n = (int)tab.size();
    t.nchunks = (int)ch.size();
    return t;
}

void lists_prep_batch(pic_ctx *ctx) {
    const BatchTab &t = ctx->batch.lists;
    k_lists_prep_batch<<<(unsigned)t.nchunks, kT, 0, ctx->stream>>>((const ListEntry *)t.tab, t.chunks);
    count_launch(ctx);
    check_launch("lists_prep_batch");
}

// The overflow repairs of every entry: one reduction and one IF node per step; its body (run
// only when some entry has records in its overflow store) moves leaves to the tail and places
// the records for every entry at once, then re-lays out the species whose tail was used up.
void repairs_batch(pic_ctx *ctx) {
    if (ctx->inst.front().cfg.precision == PIC_FP64) repairs_batch_impl<double>(ctx);
    else repairs_batch_impl<float>(ctx);
    check_launch("repairs_batch");
}

// Per-leaf arrays of one species for nl leaves (segments empty).
void species_leaf_arrays(pic_ctx *ctx, Instance &in, int s, int64_t nl) {
    ++ctx->lists_epoch;
    Species &sp = in.sp[s];
    DeviceArena &A = in.part_mem[s];
    void *olds[] = {sp.start, sp.end, sp.lim, sp.rank0, sp.start_new, sp.stay, sp.inc, sp.fill, sp.big,
                    sp.moved, sp.spawn, sp.spawn_base, sp.stay_hi, sp.stay_lo, sp.ent_hi, sp.ent_lo};
    const size_t rs = in.cfg.precision == PIC_FP64 ? 8 : 4;
    sp.start = dalloc<int32_t>(A, nl + 1);
    sp.end = dalloc<int32_t>(A, nl + 1);
    sp.lim = dalloc<int32_t>(A, nl + 1);
    sp.rank0 = dalloc<int32_t>(A, nl + 1);
    sp.start_new = dalloc<int32_t>(A, nl + 1);
    sp.stay = dalloc<int32_t>(A, nl + 1);
    sp.inc = dalloc<int32_t>(A, nl + 1);
    sp.fill = dalloc<int32_t>(A, nl + 1);
    sp.big = dalloc<int32_t>(A, nl + 1);
    sp.moved = dalloc<int32_t>(A, nl + 1);
    sp.spawn = dalloc<int32_t>(A, nl + 1);
    // spawn_base [nl + 1] | scan scratch | scan scratch
    sp.spawn_base = dalloc<int32_t>(A, nl + 1 + 2 * scan_scratch_elems(nl) + 8);
    sp.stay_hi = A.alloc((nl + 1) * rs + 64);
    sp.stay_lo = A.alloc((nl + 1) * rs + 64);
    sp.ent_hi = A.alloc((nl + 1) * rs + 64);
    sp.ent_lo = A.alloc((nl + 1) * rs + 64);
    sp.sums_valid = false;
    cudaStream_t st = ctx->stream;
    GB_CUDA(cudaMemsetAsync(sp.start, 0, (nl + 1) * 4, st));
    GB_CUDA(cudaMemsetAsync(sp.end, 0, (nl + 1) * 4, st));
    GB_CUDA(cudaMemsetAsync(sp.lim, 0, (nl + 1) * 4, st));
    GB_CUDA(cudaMemsetAsync(sp.spawn_base, 0, (nl + 1 + 2 * scan_scratch_elems(nl) + 8) * 4, st));
    for (void *p : olds)
        if (p) A.release(p);
}

// Buffers of one species with `cap` slots each, and its per-leaf arrays (no records).  A
// species that already holds buffers of `cap` slots keeps them (a reload of the same
// population size costs no allocation): only their contents are dropped.
void species_alloc(pic_ctx *ctx, Instance &in, int s, int64_t cap) {
    ++ctx->lists_epoch;
    Species &sp = in.sp[s];
    DeviceArena &A = in.part_mem[s];
    if (sp.flags && sp.cap == cap && !A.blocks.empty()) {  // (a growth hands the old blocks over first)
        GB_CUDA(cudaMemsetAsync(sp.flags, 0, 8 * 4, ctx->stream));
        species_leaf_arrays(ctx, in, s, in.nleaf);
        sp.cur = 0;
        sp.n = 0;
        sp.n_upper = 0;
        return;
    }
    A.release_all();
    sp.flags = nullptr;
    sp.start = sp.end = sp.lim = sp.rank0 = sp.start_new = sp.stay = sp.inc = sp.fill = sp.big = sp.moved = nullptr;
    sp.spawn = sp.spawn_base = nullptr;
    sp.stay_hi = sp.stay_lo = nullptr;
    sp.ent_hi = sp.ent_lo = nullptr;
    const size_t rs = in.cfg.precision == PIC_FP64 ? 8 : 4;
    sp.cap = cap;
    for (int b = 0; b < 2; ++b) {
        for (int k = 0; k < 6; ++k) sp.arr[b][k] = A.alloc(cap * rs + 64);
        sp.id[b] = dalloc<uint32_t>(A, cap);
    }
    for (int k = 0; k < 6; ++k) sp.ovf[k] = A.alloc(cap * rs + 64);
    sp.ovf_id = dalloc<uint32_t>(A, cap);
    sp.ovf_key = dalloc<uint32_t>(A, cap);
    sp.ovf_aux = dalloc<uint32_t>(A, cap);
    sp.ovf_dest = dalloc<int32_t>(A, cap);
    sp.ovf_slot = dalloc<int32_t>(A, cap);
    sp.key = dalloc<uint32_t>(A, 2 * cap);
    sp.aux = dalloc<uint32_t>(A, 2 * cap);
    sp.flags = dalloc<int32_t>(A, 8);
    GB_CUDA(cudaMemsetAsync(sp.flags, 0, 8 * 4, ctx->stream));
    species_leaf_arrays(ctx, in, s, in.nleaf);
    sp.cur = 0;
    sp.n = 0;
    sp.n_upper = 0;
}

// start = exclusive scan of (cnt + free slots), end = start + cnt.  `start` has nl + 1
// entries (start[nl] = slot span); scratch: scan_scratch_elems(nl).  `start` must not
// alias cnt.  Installing them as a species' lists takes lists_installed() afterwards.
void lists_from_counts(pic_ctx *ctx, Species &sp, int64_t nl, const int32_t *cnt, int32_t *start, int32_t *end,
                       int32_t *scratch) {
    cudaStream_t st = ctx->stream;
    k_seg_sizes<<<blocks_for(nl), kT, 0, st>>>(nl, cnt, nullptr, 0, start, nullptr);
    count_launch(ctx);
    exclusive_scan_i32(ctx, start, start, nl, scratch);
    k_set_end<<<blocks_for(nl), kT, 0, st>>>(nl, start, cnt, end);
    count_launch(ctx);
    (void)sp;
}

// After a builder wrote sp.start (leaf order, nl + 1 entries) and sp.end: segment limits and
// the tail.
void lists_installed(pic_ctx *ctx, Species &sp, int64_t nl) {
    k_lists_installed<<<blocks_for(nl), kT, 0, ctx->stream>>>(nl, sp.start, sp.lim, sp.flags);
    count_launch(ctx);
    check_launch("lists_installed");
}

// rank0[L] = records of the leaves before L (list order), rank0[nl] = total.
void list_ranks(pic_ctx *ctx, Species &sp, int64_t nl) {
    k_list_counts<<<blocks_for(nl), kT, 0, ctx->stream>>>(nl, sp.start, sp.end, sp.inc);
    count_launch(ctx);
    exclusive_scan_i32(ctx, sp.inc, sp.rank0, nl, sp.spawn_base + nl + 1);
}

// flags[1] of every species := its record total (device side; read after a sync).
void count_totals(pic_ctx *ctx, Instance &in) {
    for (int s = 0; s < in.cfg.n_species; ++s) {
        Species &sp = in.sp[s];
        if (!sp.start) continue;
        GB_CUDA(cudaMemsetAsync(sp.flags + 1, 0, 4, ctx->stream));
        const unsigned nb = std::min<unsigned>(blocks_for(in.nleaf), 152u * 2u);
        k_count_total<<<nb, kT, 0, ctx->stream>>>(in.nleaf, sp.start, sp.end, sp.flags + 1);
        count_launch(ctx);
    }
    check_launch("count_totals");
}

void capture_if(pic_ctx *ctx, cudaStream_t st, const int32_t *value, const std::function<void()> &body) {
    cudaStreamCaptureStatus status = cudaStreamCaptureStatusNone;
    cudaGraph_t g = nullptr;
    const cudaGraphNode_t *deps = nullptr;
    size_t nd = 0;
    GB_CUDA(cudaStreamGetCaptureInfo(st, &status, nullptr, &g, &deps, nullptr, &nd));
    if (status != cudaStreamCaptureStatusActive) fail(PIC_ECUDA, "capture_if outside a stream capture");
    cudaGraphConditionalHandle h = 0;
    GB_CUDA(cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault));
    k_set_if<<<1, 32, 0, st>>>(h, value);
    GB_CUDA(cudaStreamGetCaptureInfo(st, &status, nullptr, &g, &deps, nullptr, &nd));
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeIf;
    np.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    GB_CUDA(cudaGraphAddNode(&node, g, deps, nullptr, nd, &np));
    GB_CUDA(cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    // the body, captured on a private stream into the node's body graph
    cudaStream_t bs;
    GB_CUDA(cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking));
    cudaStream_t saved = ctx->stream;
    const int64_t l0 = ctx->launches;
    cudaGraph_t bg = nullptr;
    cudaError_t e = cudaStreamBeginCaptureToGraph(bs, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                                  cudaStreamCaptureModeThreadLocal);
    try {
        if (e != cudaSuccess) GB_CUDA(e);
        ctx->stream = bs;
        body();
        ctx->stream = saved;
        e = cudaStreamEndCapture(bs, &bg);
    } catch (...) {
        ctx->stream = saved;
        cudaStreamEndCapture(bs, &bg);
        ctx->launches = l0;
        cudaStreamDestroy(bs);
        throw;
    }
    ctx->launches = l0;
    cudaStreamDestroy(bs);
    GB_CUDA(e);
}

void repairs_release(Instance &in) {
    for (Species &sp : in.sp)
        if (sp.repair) {
            cudaGraphExecDestroy(sp.repair);
            sp.repair = nullptr;
        }
}

void place_overflow(pic_ctx *ctx, Instance &in, int s) {
    if (in.cfg.precision == PIC_FP64) place_impl<double>(ctx, in, s);
    else place_impl<float>(ctx, in, s);
}

// Lay species s's lists out again in leaf order with fresh free slots (frees the tail).
void species_compact(pic_ctx *ctx, Instance &in, int s) {
    Species &sp = in.sp[s];
    const int64_t nl = in.nleaf;
    k_compact_prep<<<blocks_for(nl), kT, 0, ctx->stream>>>(nl, sp.start, sp.end, sp.stay, sp.fill, sp.flags);
    count_launch(ctx);
    if (in.cfg.precision == PIC_FP64) relayout_lists<double>(ctx, in, s);
    else relayout_lists<float>(ctx, in, s);
    k_compact_done<<<1, 32, 0, ctx->stream>>>(sp.flags);
    count_launch(ctx);
    sp.sums_valid = false;
}

}  // namespace gbpic
