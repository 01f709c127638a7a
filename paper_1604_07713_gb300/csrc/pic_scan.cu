// Exclusive prefix sums of int32 arrays (reduce -> scan of block totals -> rescan), used for
// the cell-list offsets, the spawn ranks and the multigrid level construction.
#include "pic_internal.cuh"

namespace gbpic {

namespace {
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ int32_t block_exclusive_scan(int32_t v, int32_t *total) {
    __shared__ int32_t warp_sums[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int32_t s = (lane < (int)(blockDim.x >> 5)) ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(0xFFFFFFFFu, s, o);
            if (lane >= o) s += y;
        }
        warp_sums[lane] = s;
    }
    __syncthreads();
    const int32_t before = (wid > 0 ? warp_sums[wid - 1] : 0) + x - v;
    *total = warp_sums[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before;
}

__global__ void k_tile_sums(const int32_t *__restrict__ in, int64_t n, int32_t *__restrict__ part,
                            const int32_t *__restrict__ gate) {
    if (gate && *gate == 0) return;
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < n) s += in[base + k];
    int32_t tot;
    block_exclusive_scan(s, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// One block scans the tile totals in chunks, carrying the running sum.
__global__ void k_scan_parts(int32_t *__restrict__ part, int64_t nparts, int32_t *__restrict__ total,
                             const int32_t *__restrict__ gate) {
    if (gate && *gate == 0) return;
    int32_t carry = 0;
    for (int64_t c0 = 0; c0 < nparts; c0 += kScanThreads) {
        const int64_t i = c0 + threadIdx.x;
        const int32_t v = i < nparts ? part[i] : 0;
        int32_t tot;
        const int32_t ex = block_exclusive_scan(v, &tot);
        if (i < nparts) part[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) *total = carry;
}

__global__ void k_tile_scan(const int32_t *__restrict__ in, int64_t n, const int32_t *__restrict__ part,
                            int32_t *__restrict__ out, const int32_t *__restrict__ gate) {
    if (gate && *gate == 0) return;
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int32_t v[kScanItems], s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0;
        s += v[k];
    }
    int32_t tot;
    int32_t run = block_exclusive_scan(s, &tot) + part[blockIdx.x];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
}
// The same three passes over many independent arrays at once (one launch per pass): block b
// takes tile tiles[b].y of segment tiles[b].x; the segment's tile totals sit at
// scratch[first tile + t].  Integer sums: the results equal the single-array scan's.
struct ScanSeg {
    const int32_t *in;
    int32_t *out;
    int64_t n;
    int32_t tile0, ntiles;
    const int32_t *gate;  // non-null: the segment is scanned only while *gate != 0
};

__global__ void k_tile_sums_seg(const ScanSeg *__restrict__ segs, const int2 *__restrict__ tiles,
                                int32_t *__restrict__ part) {
    const int2 bt = tiles[blockIdx.x];
    const ScanSeg sg = segs[bt.x];
    if (sg.gate && *sg.gate == 0) return;
    const int64_t base = (int64_t)bt.y * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int32_t s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k)
        if (base + k < sg.n) s += sg.in[base + k];
    int32_t tot;
    block_exclusive_scan(s, &tot);
    if (threadIdx.x == 0) part[sg.tile0 + bt.y] = tot;
}

__global__ void k_scan_parts_seg(const ScanSeg *__restrict__ segs, int32_t *__restrict__ part) {
    const ScanSeg sg = segs[blockIdx.x];
    if (sg.gate && *sg.gate == 0) return;
    int32_t carry = 0;
    for (int64_t c0 = 0; c0 < sg.ntiles; c0 += kScanThreads) {
        const int64_t i = c0 + threadIdx.x;
        const int32_t v = i < sg.ntiles ? part[sg.tile0 + i] : 0;
        int32_t tot;
        const int32_t ex = block_exclusive_scan(v, &tot);
        if (i < sg.ntiles) part[sg.tile0 + i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) sg.out[sg.n] = carry;
}

__global__ void k_tile_scan_seg(const ScanSeg *__restrict__ segs, const int2 *__restrict__ tiles,
                                const int32_t *__restrict__ part) {
    const int2 bt = tiles[blockIdx.x];
    const ScanSeg sg = segs[bt.x];
    if (sg.gate && *sg.gate == 0) return;
    const int64_t base = (int64_t)bt.y * kScanTile + (int64_t)threadIdx.x * kScanItems;
    int32_t v[kScanItems], s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        v[k] = (base + k < sg.n) ? sg.in[base + k] : 0;
        s += v[k];
    }
    int32_t tot;
    int32_t run = block_exclusive_scan(s, &tot) + part[sg.tile0 + bt.y];
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        if (base + k < sg.n) sg.out[base + k] = run;
        run += v[k];
    }
}
}  // namespace

int64_t scan_scratch_elems(int64_t n) { return (n + kScanTile - 1) / kScanTile + 2; }

// out[0..n-1] = exclusive prefix of in, out[n] = total.  scratch: scan_scratch_elems(n).
// `in` and `out` may alias.  With a gate, the kernels do nothing while *gate == 0 (a
// decision the device takes after the launches were queued).
void exclusive_scan_i32(pic_ctx *ctx, const int32_t *in, int32_t *out, int64_t n, int32_t *scratch,
                        const int32_t *gate) {
    const int64_t tiles = (n + kScanTile - 1) / kScanTile;
    if (tiles == 0) {
        if (gate) fail(PIC_EINVAL, "gated scan of an empty array");
        GB_CUDA(cudaMemsetAsync(out, 0, sizeof(int32_t), ctx->stream));
        return;
    }
    k_tile_sums<<<(unsigned)tiles, kScanThreads, 0, ctx->stream>>>(in, n, scratch, gate);
    k_scan_parts<<<1, kScanThreads, 0, ctx->stream>>>(scratch, tiles, out + n, gate);
    k_tile_scan<<<(unsigned)tiles, kScanThreads, 0, ctx->stream>>>(in, n, scratch, out, gate);
    count_launch(ctx, 3);
    check_launch("exclusive_scan_i32");
}

// Plan of a segmented scan (host tables uploaded now, outside any capture).  Every segment
// must hold at least one element.
ScanPlan scan_plan(pic_ctx *ctx, const std::vector<const int32_t *> &in, const std::vector<int32_t *> &out,
                   const std::vector<int64_t> &n, const std::vector<const int32_t *> &gate) {
    ScanPlan p;
    std::vector<ScanSeg> segs(in.size());
    std::vector<int2> tiles;
    int32_t t0 = 0;
    for (size_t k = 0; k < in.size(); ++k) {
        if (n[k] <= 0) fail(PIC_EINVAL, "segmented scan of an empty array");
        const int32_t nt = (int32_t)((n[k] + kScanTile - 1) / kScanTile);
        segs[k] = ScanSeg{in[k], out[k], n[k], t0, nt, gate.empty() ? nullptr : gate[k]};
        for (int32_t t = 0; t < nt; ++t) tiles.push_back(make_int2((int)k, t));
        t0 += nt;
    }
    p.nseg = (int)segs.size();
    p.ntiles = (int)tiles.size();
    if (p.nseg == 0) return p;
    p.segs = batch_upload(ctx, segs);
    p.tiles = batch_upload(ctx, tiles);
    p.scratch = (int32_t *)batch_upload(ctx, nullptr, (size_t)t0 * sizeof(int32_t));
    return p;
}

void exclusive_scan_i32_batch(pic_ctx *ctx, const ScanPlan &p) {
    if (p.nseg == 0) return;
    const ScanSeg *segs = (const ScanSeg *)p.segs;
    k_tile_sums_seg<<<(unsigned)p.ntiles, kScanThreads, 0, ctx->stream>>>(segs, p.tiles, p.scratch);
    k_scan_parts_seg<<<(unsigned)p.nseg, kScanThreads, 0, ctx->stream>>>(segs, p.scratch);
    k_tile_scan_seg<<<(unsigned)p.ntiles, kScanThreads, 0, ctx->stream>>>(segs, p.tiles, p.scratch);
    count_launch(ctx, 3);
    check_launch("exclusive_scan_i32_batch");
}

}  // namespace gbpic
