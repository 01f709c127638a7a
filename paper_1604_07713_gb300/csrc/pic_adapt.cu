// Mesh adaptation (§3.1: refined cells take their particles by position, coarsened cells
// their children's particles; §4.3: the AMR grid as particle management) and per-leaf particle
// splitting / merging (§4.3).  The rules (criteria, balance, list orders, merge grouping) are
// the readings written out in the oracle; every decision here takes the same inputs in the
// same order so the results agree exactly where the arithmetic is exact.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <utility>

#include "pic_internal.cuh"

namespace gbpic {

namespace {
constexpr int kT = 256;
inline unsigned blocks_for(int64_t n, int t = kT) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }
inline unsigned warp_blocks(int64_t nw) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((nw + 7) / 8, 1 << 20)); }

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// ------------------------------------------------------------------------------------
// Adaptation flags
// ------------------------------------------------------------------------------------
struct AdaptArgs {
    int64_t n;
    int lmax;
    const uint8_t *lev;
    const uint32_t *root, *morton;
    const int32_t *start_e, *end_e;  // electron lists
    const double *emag;
    int32_t refine_count, coarsen_count;
    double refine_e, coarsen_e;
};

__device__ __forceinline__ bool wants_refine(const AdaptArgs &a, int64_t l) {
    const int32_t c = a.end_e[l] - a.start_e[l];
    return a.lev[l] < a.lmax && (c > a.refine_count || a.emag[l] > a.refine_e);
}

// group[l] = first leaf of l's sibling quartet (4 consecutive leaves of one parent) or -1;
// gactive[first] = the quartet asks to coarsen.
__global__ void k_adapt_flags(AdaptArgs a, int32_t *__restrict__ refine, int32_t *__restrict__ group,
                              int32_t *__restrict__ gactive) {
    const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= a.n) return;
    refine[l] = wants_refine(a, l) ? 1 : 0;
    gactive[l] = 0;
    int32_t g = -1;
    const int lv = a.lev[l];
    if (lv >= 1) {
        const int64_t s = l - (int64_t)(a.morton[l] & 3u);
        if (s >= 0 && s + 3 < a.n) {
            bool ok = (a.morton[s] & 3u) == 0;
            for (int k = 0; k < 4 && ok; ++k)
                ok = a.lev[s + k] == lv && a.root[s + k] == a.root[s] && (a.morton[s + k] >> 2) == (a.morton[s] >> 2);
            if (ok) g = (int32_t)s;
        }
    }
    group[l] = g;
    if (g == (int32_t)l) {
        bool ok = true;
        int64_t tot = 0;
        for (int k = 0; k < 4; ++k) {
            ok = ok && !wants_refine(a, l + k) && a.emag[l + k] < a.coarsen_e;
            tot += a.end_e[l + k] - a.start_e[l + k];
        }
        gactive[l] = (ok && tot <= a.coarsen_count) ? 1 : 0;
    }
}

// One pass of the 2:1 closure over faces and corners: a leaf whose target level is more than
// one below a touching leaf's refines, or keeps its quartet from coarsening.  Only raises
// targets, so repeated passes reach the unique least balanced set whatever the order.
__global__ void k_adapt_balance(int64_t n, int lmax, const int32_t *__restrict__ map, int NX, int NY, int px,
                                int py, const int32_t *__restrict__ ix, const int32_t *__restrict__ iy,
                                const uint8_t *__restrict__ lev, int32_t *refine, const int32_t *__restrict__ group,
                                int32_t *gactive, int32_t *__restrict__ changed) {
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= n) return;
    auto target = [&](int64_t i) -> int {
        int t = lev[i] + (((volatile int32_t *)refine)[i] ? 1 : 0);
        const int32_t g = group[i];
        if (g >= 0 && ((volatile int32_t *)gactive)[g]) t -= 1;
        return t;
    };
    const int32_t x = ix[a], y = iy[a], s = 1 << (lmax - lev[a]);
    const int32_t P[12][2] = {{x - 1, y}, {x - 1, y + s - 1}, {x + s, y}, {x + s, y + s - 1},
                              {x, y - 1}, {x + s - 1, y - 1}, {x, y + s}, {x + s - 1, y + s},
                              {x - 1, y - 1}, {x + s, y - 1}, {x - 1, y + s}, {x + s, y + s}};
    const int32_t g = group[a];
    for (int k = 0; k < 12; ++k) {
        const int32_t b = lattice_leaf(map, NX, NY, px, py, P[k][0], P[k][1]);
        if (b < 0 || b == a) continue;
        if (g >= 0 && g == group[b]) continue;
        // decide and act on one snapshot of this leaf's own flags: refine only goes 0 -> 1 and
        // gactive 1 -> 0, so a stale snapshot at worst repeats a cancellation (and one more pass)
        const int act = g >= 0 ? ((volatile int32_t *)gactive)[g] : 0;
        const int ref = ((volatile int32_t *)refine)[a];
        const int ta = lev[a] + ref - act;
        const int tb = target(b);
        if (ta < tb - 1) {
            if (act) ((volatile int32_t *)gactive)[g] = 0;
            else if (!ref && lev[a] < lmax) ((volatile int32_t *)refine)[a] = 1;
            else continue;
            *changed = 1;
        }
    }
}

// Number of new leaves each old leaf emits: 4 (refine), 1 (kept; first of a coarsening
// quartet), 0 (other quartet members).
__global__ void k_adapt_emit_count(int64_t n, const int32_t *__restrict__ refine, const int32_t *__restrict__ group,
                                   const int32_t *__restrict__ gactive, int32_t *__restrict__ cnt) {
    const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n) return;
    const int32_t g = group[l];
    if (g >= 0 && gactive[g]) cnt[l] = (g == (int32_t)l) ? 1 : 0;
    else cnt[l] = refine[l] ? 4 : 1;
}

// New raw leaf description, index map old -> new, potential carried over.
__global__ void k_adapt_emit(int64_t n, const int32_t *__restrict__ refine, const int32_t *__restrict__ group,
                             const int32_t *__restrict__ gactive, const int32_t *__restrict__ pos,
                             const uint32_t *__restrict__ root, const uint32_t *__restrict__ morton,
                             const uint8_t *__restrict__ lev, const double *__restrict__ phi,
                             uint32_t *__restrict__ nroot, uint32_t *__restrict__ nmorton, uint8_t *__restrict__ nlev,
                             double *__restrict__ nphi, int32_t *__restrict__ new_of, int32_t *__restrict__ kind) {
    const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n) return;
    const int32_t g = group[l];
    if (g >= 0 && gactive[g]) {
        new_of[l] = pos[g];
        kind[l] = 2;  // coarsened into its quartet's parent
        if (g == (int32_t)l) {
            const int32_t o = pos[l];
            nroot[o] = root[l];
            nmorton[o] = morton[l] >> 2;
            nlev[o] = (uint8_t)(lev[l] - 1);
            nphi[o] = 0.25 * (((phi[l] + phi[l + 1]) + phi[l + 2]) + phi[l + 3]);
        }
    } else if (refine[l]) {
        const int32_t o = pos[l];
        new_of[l] = o;
        kind[l] = 1;  // refined into 4 children
        for (int c = 0; c < 4; ++c) {
            nroot[o + c] = root[l];
            nmorton[o + c] = (morton[l] << 2) | (uint32_t)c;
            nlev[o + c] = (uint8_t)(lev[l] + 1);
            nphi[o + c] = phi[l];
        }
    } else {
        const int32_t o = pos[l];
        new_of[l] = o;
        kind[l] = 0;
        nroot[o] = root[l];
        nmorton[o] = morton[l];
        nlev[o] = lev[l];
        nphi[o] = phi[l];
    }
}

// Particle counts of the new leaves (one warp per old leaf).
template <typename R>
__global__ void k_adapt_count(int64_t n, const int32_t *__restrict__ start, const int32_t *__restrict__ end,
                              const int32_t *__restrict__ kind, const int32_t *__restrict__ group,
                              const int32_t *__restrict__ new_of, SoA<R> d, int32_t *__restrict__ ncnt) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t l = warp; l < n; l += nw) {
        const int k = kind[l];
        if (k == 0) {
            if (lane == 0) ncnt[new_of[l]] = end[l] - start[l];
        } else if (k == 2) {
            if (lane == 0 && group[l] == (int32_t)l) {
                int32_t c = 0;
                for (int i = 0; i < 4; ++i) c += end[l + i] - start[l + i];
                ncnt[new_of[l]] = c;
            }
        } else {
            int32_t c4[4] = {0, 0, 0, 0};
            for (int32_t p0 = start[l]; p0 < end[l]; p0 += 32) {
                const int32_t p = p0 + lane;
                int ch = -1;
                if (p < end[l]) ch = (d.u[p] >= (R)0.5 ? 1 : 0) + (d.v[p] >= (R)0.5 ? 2 : 0);
                for (int c = 0; c < 4; ++c) c4[c] += __popc(__ballot_sync(0xFFFFFFFFu, ch == c));
            }
            if (lane == 0)
                for (int c = 0; c < 4; ++c) ncnt[new_of[l] + c] = c4[c];
        }
    }
}

// Move the records to the new lists; offsets re-expressed exactly in the new leaf.  A
// coarsened quartet's list is its children's lists one after another in Morton order.
template <typename R>
__global__ void k_adapt_move(int64_t n, const int32_t *__restrict__ start, const int32_t *__restrict__ end,
                             const int32_t *__restrict__ kind, const int32_t *__restrict__ group,
                             const int32_t *__restrict__ new_of, const uint32_t *__restrict__ morton,
                             const int32_t *__restrict__ nstart, SoA<R> s, SoA<R> d) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t l = warp; l < n; l += nw) {
        const int k = kind[l];
        const int32_t p0 = start[l], p1 = end[l];
        int32_t q0 = 0;  // first slot of this leaf's records in the new list
        if (k == 0) {
            q0 = nstart[new_of[l]];
        } else if (k == 2) {
            const int32_t g = group[l];
            q0 = nstart[new_of[l]];
            for (int32_t i = g; i < (int32_t)l; ++i) q0 += end[i] - start[i];
        }
        int32_t run[4] = {0, 0, 0, 0};
        for (int32_t c0 = p0; c0 < p1; c0 += 32) {
            const int32_t p = c0 + lane;
            const bool live = p < p1;
            R u = 0, v = 0;
            int32_t dst = -1;
            int ch = -1;
            if (live) {
                u = s.u[p];
                v = s.v[p];
            }
            if (k == 0) {
                dst = q0 + (p - p0);
            } else if (k == 2) {
                const R cx = (R)(morton[l] & 1u), cy = (R)((morton[l] >> 1) & 1u);
                dst = q0 + (p - p0);
                u = (cx + u) * (R)0.5;
                v = (cy + v) * (R)0.5;
            } else {
                ch = live ? (u >= (R)0.5 ? 1 : 0) + (v >= (R)0.5 ? 2 : 0) : -1;
                int32_t rank = 0;
                for (int c = 0; c < 4; ++c) {
                    const uint32_t m = __ballot_sync(0xFFFFFFFFu, ch == c);
                    if (ch == c) rank = run[c] + __popc(m & lanemask_lt());
                    run[c] += __popc(m);
                }
                if (live) {
                    dst = nstart[new_of[l] + ch] + rank;
                    u = (R)2 * u - (R)(ch & 1);
                    v = (R)2 * v - (R)(ch >> 1);
                }
            }
            if (live) {
                d.u[dst] = u; d.v[dst] = v;
                d.vx[dst] = s.vx[p]; d.vy[dst] = s.vy[p]; d.vz[dst] = s.vz[p]; d.w[dst] = s.w[p]; d.id[dst] = s.id[p];
            }
        }
    }
}

// Slots a coarsened quartet's list takes at the tail (its first sibling only; 0 elsewhere).
__global__ void k_adapt_tail_need(int64_t n, const int32_t *__restrict__ start, const int32_t *__restrict__ end,
                                  const int32_t *__restrict__ kind, const int32_t *__restrict__ group,
                                  int32_t *__restrict__ need) {
    const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n) return;
    int32_t v = 0;
    if (kind[l] == 2 && group[l] == (int32_t)l) {
        int32_t c = 0;
        for (int i = 0; i < 4; ++i) c += end[l + i] - start[l + i];
        v = c + list_slack(c);
    }
    need[l] = v;
}

// The lists of the new leaves, in place (one warp per old leaf):
// - an unchanged leaf keeps its segment;
// - a refined leaf's records are partitioned by quadrant inside its own segment (through the
//   scratch buffer), in list order, offsets re-expressed; its free slots are shared out;
// - a coarsened quartet's lists go, one after another in Morton order, to a segment at the
//   tail (tail0 + the scanned slot need of the quartets before it), offsets re-expressed.
template <typename R>
__global__ void k_adapt_inplace(int64_t n, const int32_t *__restrict__ start, const int32_t *__restrict__ end,
                                const int32_t *__restrict__ lim, const int32_t *__restrict__ kind,
                                const int32_t *__restrict__ group, const int32_t *__restrict__ new_of,
                                const uint32_t *__restrict__ morton, const int32_t *__restrict__ ncnt,
                                const int32_t *__restrict__ tail_off, int32_t tail0, SoA<R> d, SoA<R> t,
                                int32_t *__restrict__ nstart, int32_t *__restrict__ nend,
                                int32_t *__restrict__ nlim) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t l = warp; l < n; l += nw) {
        const int k = kind[l];
        const int32_t p0 = start[l], p1 = end[l];
        if (k == 0) {
            if (lane == 0) {
                const int32_t o = new_of[l];
                nstart[o] = p0; nend[o] = p1; nlim[o] = lim[l];
            }
        } else if (k == 1) {
            for (int32_t p = p0 + lane; p < p1; p += 32) {
                t.u[p] = d.u[p]; t.v[p] = d.v[p]; t.vx[p] = d.vx[p]; t.vy[p] = d.vy[p]; t.vz[p] = d.vz[p];
                t.w[p] = d.w[p]; t.id[p] = d.id[p];
            }
            __syncwarp();
            const int32_t o = new_of[l];
            int32_t off[4], cnt[4];
            const int32_t extra = (lim[l] - p0 - (p1 - p0)) / 4;  // free slots shared out
            int32_t acc = p0;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                cnt[c] = ncnt[o + c];
                off[c] = acc;
                acc += cnt[c] + extra;
            }
            if (lane < 4) {
                nstart[o + lane] = off[lane];
                nend[o + lane] = off[lane] + cnt[lane];
                nlim[o + lane] = lane == 3 ? lim[l] : off[lane] + cnt[lane] + extra;
            }
            int32_t run[4] = {0, 0, 0, 0};
            for (int32_t c0 = p0; c0 < p1; c0 += 32) {
                const int32_t p = c0 + lane;
                const bool live = p < p1;
                R u = 0, v = 0;
                int ch = -1;
                if (live) {
                    u = t.u[p];
                    v = t.v[p];
                    ch = (u >= (R)0.5 ? 1 : 0) + (v >= (R)0.5 ? 2 : 0);
                }
                int32_t rank = 0;
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const uint32_t m = __ballot_sync(0xFFFFFFFFu, ch == c);
                    if (ch == c) rank = run[c] + __popc(m & lanemask_lt());
                    run[c] += __popc(m);
                }
                if (live) {
                    int32_t q = 0;
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        if (ch == c) q = off[c] + rank;
                    d.u[q] = (R)2 * u - (R)(ch & 1);
                    d.v[q] = (R)2 * v - (R)(ch >> 1);
                    d.vx[q] = t.vx[p]; d.vy[q] = t.vy[p]; d.vz[q] = t.vz[p]; d.w[q] = t.w[p]; d.id[q] = t.id[p];
                }
            }
        } else if (group[l] == (int32_t)l) {
            const int32_t base = tail0 + tail_off[l];
            int32_t q0 = base;
            for (int i = 0; i < 4; ++i) {
                const int64_t li = l + i;
                const int32_t a0 = start[li], a1 = end[li];
                const R cx = (R)(morton[li] & 1u), cy = (R)((morton[li] >> 1) & 1u);
                for (int32_t p = a0 + lane; p < a1; p += 32) {
                    const int32_t q = q0 + (p - a0);
                    d.u[q] = (cx + d.u[p]) * (R)0.5;
                    d.v[q] = (cy + d.v[p]) * (R)0.5;
                    d.vx[q] = d.vx[p]; d.vy[q] = d.vy[p]; d.vz[q] = d.vz[p]; d.w[q] = d.w[p]; d.id[q] = d.id[p];
                }
                q0 += a1 - a0;
            }
            if (lane == 0) {
                const int32_t o = new_of[l], c = q0 - base;
                nstart[o] = base; nend[o] = q0; nlim[o] = base + c + list_slack(c);
            }
        }
    }
}

// ------------------------------------------------------------------------------------
// Split / merge
// ------------------------------------------------------------------------------------
struct SMArgs {
    int64_t n;
    const int32_t *start, *end;
    int32_t ppc_min, ppc_max, ppc_target;
};

__device__ __forceinline__ int split_rounds(int32_t c, int32_t ppc_min) {
    int r = 0;
    int64_t m = c;
    while (m < ppc_min) { m *= 4; ++r; }
    return r;
}

// Per leaf: records after the step, new ids, merge / split flags, and the tail slots a
// split leaf takes when its segment cannot hold its children.
__global__ void k_sm_count(SMArgs a, const int32_t *__restrict__ lim, int32_t *__restrict__ ncnt,
                           int32_t *__restrict__ nids, int32_t *__restrict__ merge_flag,
                           int32_t *__restrict__ split_flag, int32_t *__restrict__ tail_need) {
    const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= a.n) return;
    const int32_t c = a.end[l] - a.start[l];
    int32_t nc = c, ni = 0, mf = 0, sf = 0, tn = 0;
    if (c > 0 && c < a.ppc_min) {
        const int r = split_rounds(c, a.ppc_min);
        nc = c << (2 * r);
        ni = nc - c;
        sf = 1;
        if (nc > lim[l] - a.start[l]) tn = nc + list_slack(nc);
    } else if (c > a.ppc_max) {
        nc = a.ppc_target;
        mf = 1;
    }
    ncnt[l] = nc;
    nids[l] = ni;
    merge_flag[l] = mf;
    split_flag[l] = sf;
    tail_need[l] = tn;
}

// Split leaves, in place (one warp per listed leaf): the parents are copied to the scratch
// buffer, then each child k of parent j is written at slot j 4^r + k of the leaf's list,
// in its own segment or, when that is too small, in a segment at the tail.
template <typename R>
__global__ void k_sm_split(SMArgs a, const int32_t *__restrict__ slist, int32_t ns, int32_t *__restrict__ start,
                           int32_t *__restrict__ end, int32_t *__restrict__ lim,
                           const int32_t *__restrict__ tail_need, const int32_t *__restrict__ tail_off, int32_t tail0,
                           const int32_t *__restrict__ idbase, unsigned long long id0, SoA<R> d, SoA<R> t) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = warp; i < ns; i += nw) {
        const int32_t l = slist[i];
        const int32_t p0 = start[l], p1 = end[l], c = p1 - p0;
        for (int32_t p = p0 + lane; p < p1; p += 32) {
            t.u[p] = d.u[p]; t.v[p] = d.v[p]; t.vx[p] = d.vx[p]; t.vy[p] = d.vy[p]; t.vz[p] = d.vz[p];
            t.w[p] = d.w[p]; t.id[p] = d.id[p];
        }
        __syncwarp();
        const int r = split_rounds(c, a.ppc_min);
        const int32_t kids = 1 << (2 * r);
        const int32_t q0 = tail_need[l] > 0 ? tail0 + tail_off[l] : p0;
        // one child per lane-iteration: child k of parent j, k in depth-first (base-4) order
        for (int32_t tt = lane; tt < c * kids; tt += 32) {
            const int32_t j = tt / kids, k = tt - j * kids;
            const int32_t p = p0 + j;
            R u = t.u[p], v = t.v[p], w = t.w[p];
            for (int lvl = r - 1; lvl >= 0; --lvl) {
                const int digit = (k >> (2 * lvl)) & 3;
                R m = u < (R)1 - u ? u : (R)1 - u;
                m = m < v ? m : v;
                m = m < (R)1 - v ? m : (R)1 - v;
                R dd = (R)0.25 * m;
                dd = dd < (R)(1.0 / 1024.0) ? dd : (R)(1.0 / 1024.0);
                u = (digit & 1) ? u + dd : u - dd;
                v = (digit & 2) ? v + dd : v - dd;
                w = w * (R)0.25;
            }
            const int32_t q = q0 + tt;
            d.u[q] = u; d.v[q] = v; d.vx[q] = t.vx[p]; d.vy[q] = t.vy[p]; d.vz[q] = t.vz[p]; d.w[q] = w;
            d.id[q] = k == 0 ? t.id[p] : (uint32_t)(id0 + (unsigned long long)idbase[l] +
                                                    (unsigned long long)j * (kids - 1) + (k - 1));
        }
        __syncwarp();
        if (lane == 0) {
            start[l] = q0;
            end[l] = q0 + c * kids;
            if (tail_need[l] > 0) lim[l] = q0 + tail_need[l];
        }
    }
}

// Energy bin of one particle, decided in the state's precision with no contraction.
__device__ __forceinline__ float energy_f(float hm, float vx, float vy, float vz) {
    return __fmul_rn(hm, __fadd_rn(__fadd_rn(__fmul_rn(vx, vx), __fmul_rn(vy, vy)), __fmul_rn(vz, vz)));
}
__device__ __forceinline__ double energy_f(double hm, double vx, double vy, double vz) {
    return __dmul_rn(hm, __dadd_rn(__dadd_rn(__dmul_rn(vx, vx), __dmul_rn(vy, vy)), __dmul_rn(vz, vz)));
}
__device__ __forceinline__ int bin_of(float e, float lo, float rng) {
    if (rng == 0.0f) return 0;
    const float q = __fdiv_rn(__fmul_rn(__fsub_rn(e, lo), 16.0f), rng);
    const int b = (int)floorf(q);
    return b < 0 ? 0 : (b > 15 ? 15 : b);
}
__device__ __forceinline__ int bin_of(double e, double lo, double rng) {
    if (rng == 0.0) return 0;
    const double q = __ddiv_rn(__dmul_rn(__dsub_rn(e, lo), 16.0), rng);
    const int b = (int)floor(q);
    return b < 0 ? 0 : (b > 15 ? 15 : b);
}

constexpr int kMergeMax = 12288;  // particles of one leaf sorted in shared memory

// One block per merging leaf: sort by (energy bin, id), cut into ppc_target groups, merge.
// The merged records are written to the scratch buffer at the leaf's slots, then copied back
// in place, so no source record is overwritten before it is read.
template <typename R>
__global__ void __launch_bounds__(512) k_sm_merge(SMArgs a, const int32_t *__restrict__ mlist, int32_t nm,
                                                  int32_t *__restrict__ end, R half_m, SoA<R> s, SoA<R> d,
                                                  int32_t *__restrict__ err) {
    extern __shared__ unsigned long long keys[];  // (bin << 32 | id) , index in the low word after
    __shared__ R red_lo[16], red_hi[16];
    for (int32_t mi = blockIdx.x; mi < nm; mi += gridDim.x) {
        const int32_t l = mlist[mi];
        const int32_t p0 = a.start[l], c = a.end[l] - p0;
        if (c > kMergeMax) {
            if (threadIdx.x == 0) atomicExch(err, 1);
            continue;
        }
        // energy range
        R lo = (R)INFINITY, hi = (R)-INFINITY;
        for (int32_t i = threadIdx.x; i < c; i += blockDim.x) {
            const R e = energy_f(half_m, s.vx[p0 + i], s.vy[p0 + i], s.vz[p0 + i]);
            lo = e < lo ? e : lo;
            hi = e > hi ? e : hi;
        }
        for (int o = 16; o > 0; o >>= 1) {
            const R a1 = __shfl_xor_sync(0xFFFFFFFFu, lo, o), b1 = __shfl_xor_sync(0xFFFFFFFFu, hi, o);
            lo = a1 < lo ? a1 : lo;
            hi = b1 > hi ? b1 : hi;
        }
        if ((threadIdx.x & 31) == 0) { red_lo[threadIdx.x >> 5] = lo; red_hi[threadIdx.x >> 5] = hi; }
        __syncthreads();
        lo = red_lo[0]; hi = red_hi[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            lo = red_lo[w] < lo ? red_lo[w] : lo;
            hi = red_hi[w] > hi ? red_hi[w] : hi;
        }
        const R rng = hi - lo;
        // keys: bin (4 bits) | id (32 bits) | local index (14 bits), padded to a power of two
        int32_t np2 = 1;
        while (np2 < c) np2 <<= 1;
        for (int32_t i = threadIdx.x; i < np2; i += blockDim.x) {
            if (i < c) {
                const R e = energy_f(half_m, s.vx[p0 + i], s.vy[p0 + i], s.vz[p0 + i]);
                const unsigned long long b = (unsigned long long)bin_of(e, lo, rng);
                keys[i] = (b << 46) | ((unsigned long long)s.id[p0 + i] << 14) | (unsigned long long)i;
            } else {
                keys[i] = ~0ull;
            }
        }
        __syncthreads();
        // bitonic sort ascending
        for (int32_t k = 2; k <= np2; k <<= 1) {
            for (int32_t j = k >> 1; j > 0; j >>= 1) {
                for (int32_t i = threadIdx.x; i < np2; i += blockDim.x) {
                    const int32_t ij = i ^ j;
                    if (ij > i) {
                        const unsigned long long x = keys[i], y = keys[ij];
                        const bool up = (i & k) == 0;
                        if ((x > y) == up) { keys[i] = y; keys[ij] = x; }
                    }
                }
                __syncthreads();
            }
        }
        // groups: the first (c mod T) of size q + 1, the rest q
        const int32_t T = a.ppc_target, q = c / T, rem = c - q * T;
        const int32_t o0 = p0;
        for (int32_t g = threadIdx.x; g < T; g += blockDim.x) {
            const int32_t b0 = g < rem ? g * (q + 1) : rem * (q + 1) + (g - rem) * q;
            const int32_t sz = g < rem ? q + 1 : q;
            R W = 0, X = 0, Y = 0, VX = 0, VY = 0, VZ = 0;
            uint32_t idmin = 0xFFFFFFFFu;
            for (int32_t t = 0; t < sz; ++t) W += s.w[p0 + (int32_t)(keys[b0 + t] & 0x3FFFull)];
            for (int32_t t = 0; t < sz; ++t) {
                const int32_t p = p0 + (int32_t)(keys[b0 + t] & 0x3FFFull);
                const R wp = s.w[p];
                X += wp * s.u[p]; Y += wp * s.v[p];
                VX += wp * s.vx[p]; VY += wp * s.vy[p]; VZ += wp * s.vz[p];
                idmin = s.id[p] < idmin ? s.id[p] : idmin;
            }
            const int32_t o = o0 + g;
            R u = X / W, v = Y / W;
            u = u < (R)0 ? (R)0 : u;
            v = v < (R)0 ? (R)0 : v;
            d.u[o] = u; d.v[o] = v; d.vx[o] = VX / W; d.vy[o] = VY / W; d.vz[o] = VZ / W; d.w[o] = W;
            d.id[o] = idmin;
        }
        __syncthreads();
        for (int32_t g = threadIdx.x; g < T; g += blockDim.x) {
            const int32_t o = o0 + g;
            s.u[o] = d.u[o]; s.v[o] = d.v[o]; s.vx[o] = d.vx[o]; s.vy[o] = d.vy[o]; s.vz[o] = d.vz[o];
            s.w[o] = d.w[o]; s.id[o] = d.id[o];
        }
        if (threadIdx.x == 0) end[l] = o0 + T;
        __syncthreads();
    }
}

__global__ void k_compact_flags(int64_t n, const int32_t *__restrict__ flag, const int32_t *__restrict__ pos,
                                int32_t *__restrict__ list) {
    const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l < n && flag[l]) list[pos[l]] = (int32_t)l;
}

int32_t read_i32(pic_ctx *ctx, const int32_t *d) {
    int32_t h = 0;
    GB_CUDA(cudaMemcpyAsync(&h, d, 4, cudaMemcpyDeviceToHost, ctx->stream));
    GB_CUDA(cudaStreamSynchronize(ctx->stream));
    return h;
}

// Re-allocate one species' per-leaf arrays for a new leaf count; the records stay.  With
// nlim, the segments are taken as given (anywhere in the buffer) and the tail starts at
// `tail`; without, they are in leaf order (lim[L] = start[L + 1]).
void species_relist(pic_ctx *ctx, Instance &in, int s, int64_t nl, const int32_t *new_start,
                    const int32_t *new_end, const int32_t *nlim = nullptr, int32_t tail = 0) {
    Species &sp = in.sp[s];
    species_leaf_arrays(ctx, in, s, nl);
    GB_CUDA(cudaMemcpyAsync(sp.start, new_start, (nl + 1) * 4, cudaMemcpyDeviceToDevice, ctx->stream));
    GB_CUDA(cudaMemcpyAsync(sp.end, new_end, (nl + 1) * 4, cudaMemcpyDeviceToDevice, ctx->stream));
    if (nlim) {
        GB_CUDA(cudaMemcpyAsync(sp.lim, nlim, nl * 4, cudaMemcpyDeviceToDevice, ctx->stream));
        GB_CUDA(cudaMemcpyAsync(sp.flags + 4, &tail, 4, cudaMemcpyHostToDevice, ctx->stream));
    } else {
        lists_installed(ctx, sp, nl);
    }
    GB_CUDA(cudaStreamSynchronize(ctx->stream));
}

// Lists whose tail has used up more than a quarter of the buffer are laid out again first,
// so that repairs and adaptation do not keep growing the buffers.
void compact_if_crowded(pic_ctx *ctx, Instance &in, int s) {
    Species &sp = in.sp[s];
    const int32_t tail = read_i32(ctx, sp.flags + 4);
    if ((int64_t)tail > sp.cap - sp.cap / 4) species_compact(ctx, in, s);
}

template <typename R> void adapt_particles(pic_ctx *ctx, Instance &in, int64_t n_old, int64_t n_new,
                                           const int32_t *kind, const int32_t *group, const int32_t *new_of,
                                           const uint32_t *morton_old, DeviceArena &T) {
    cudaStream_t st = ctx->stream;
    for (int s = 0; s < in.cfg.n_species; ++s) {
        Species &sp = in.sp[s];
        compact_if_crowded(ctx, in, s);
        int32_t *ncnt = dalloc<int32_t>(T, n_new + 1);
        int32_t *need = dalloc<int32_t>(T, n_old + 1);
        int32_t *scr = dalloc<int32_t>(T, scan_scratch_elems(std::max(n_old, n_new)));
        GB_CUDA(cudaMemsetAsync(ncnt, 0, (n_new + 1) * 4, st));
        k_adapt_count<R><<<warp_blocks(n_old), kT, 0, st>>>(n_old, sp.start, sp.end, kind, group, new_of,
                                                           soa<R>(sp, sp.cur), ncnt);
        k_adapt_tail_need<<<blocks_for(n_old), kT, 0, st>>>(n_old, sp.start, sp.end, kind, group, need);
        count_launch(ctx, 2);
        exclusive_scan_i32(ctx, need, need, n_old, scr);
        // the coarsened quartets' lists go to the tail: make room for them first
        int32_t h[2] = {0, 0};
        GB_CUDA(cudaMemcpyAsync(&h[0], sp.flags + 4, 4, cudaMemcpyDeviceToHost, st));
        GB_CUDA(cudaMemcpyAsync(&h[1], need + n_old, 4, cudaMemcpyDeviceToHost, st));
        GB_CUDA(cudaStreamSynchronize(st));
        ensure_slots(ctx, in, s, (int64_t)h[0] + h[1]);
        int32_t *nstart = dalloc<int32_t>(T, n_new + 1), *nend = dalloc<int32_t>(T, n_new + 1);
        int32_t *nlim = dalloc<int32_t>(T, n_new + 1);
        k_adapt_inplace<R><<<warp_blocks(n_old), kT, 0, st>>>(n_old, sp.start, sp.end, sp.lim, kind, group, new_of,
                                                             morton_old, ncnt, need, h[0], soa<R>(sp, sp.cur),
                                                             soa<R>(sp, sp.cur ^ 1), nstart, nend, nlim);
        count_launch(ctx);
        check_launch("adapt_particles");
        species_relist(ctx, in, s, n_new, nstart, nend, nlim, h[0] + h[1]);
    }
}

template <typename R> void split_merge_impl(pic_ctx *ctx, Instance &in) {
    cudaStream_t st = ctx->stream;
    const int64_t nl = in.nleaf;
    DeviceArena T(&ctx->cache);
    unsigned long long next_id = 0;
    GB_CUDA(cudaMemcpyAsync(&next_id, in.d_next_id, 8, cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaStreamSynchronize(st));
    int32_t *err = dalloc<int32_t>(T, 1);
    GB_CUDA(cudaMemsetAsync(err, 0, 4, st));
    for (int s = 0; s < in.cfg.n_species; ++s) {
        Species &sp = in.sp[s];
        compact_if_crowded(ctx, in, s);
        int32_t *ncnt = dalloc<int32_t>(T, nl + 1), *nids = dalloc<int32_t>(T, nl + 1);
        int32_t *mflag = dalloc<int32_t>(T, nl + 1), *sflag = dalloc<int32_t>(T, nl + 1);
        int32_t *tneed = dalloc<int32_t>(T, nl + 1), *toff = dalloc<int32_t>(T, nl + 1);
        int32_t *idb = dalloc<int32_t>(T, nl + 1);
        int32_t *mpos = dalloc<int32_t>(T, nl + 1), *mlist = dalloc<int32_t>(T, nl + 1);
        int32_t *spos = dalloc<int32_t>(T, nl + 1), *slist = dalloc<int32_t>(T, nl + 1);
        int32_t *scr = dalloc<int32_t>(T, scan_scratch_elems(nl));
        {
            SMArgs a{nl, sp.start, sp.end, in.cfg.ppc_min, in.cfg.ppc_max, in.cfg.ppc_target};
            k_sm_count<<<blocks_for(nl), kT, 0, st>>>(a, sp.lim, ncnt, nids, mflag, sflag, tneed);
            count_launch(ctx);
        }
        exclusive_scan_i32(ctx, nids, idb, nl, scr);
        exclusive_scan_i32(ctx, mflag, mpos, nl, scr);
        exclusive_scan_i32(ctx, sflag, spos, nl, scr);
        exclusive_scan_i32(ctx, tneed, toff, nl, scr);
        int32_t tot[5];
        GB_CUDA(cudaMemcpyAsync(&tot[0], toff + nl, 4, cudaMemcpyDeviceToHost, st));
        GB_CUDA(cudaMemcpyAsync(&tot[1], idb + nl, 4, cudaMemcpyDeviceToHost, st));
        GB_CUDA(cudaMemcpyAsync(&tot[2], mpos + nl, 4, cudaMemcpyDeviceToHost, st));
        GB_CUDA(cudaMemcpyAsync(&tot[3], spos + nl, 4, cudaMemcpyDeviceToHost, st));
        GB_CUDA(cudaMemcpyAsync(&tot[4], sp.flags + 4, 4, cudaMemcpyDeviceToHost, st));
        GB_CUDA(cudaStreamSynchronize(st));
        if (in.cfg.particle_capacity > 0 && sp.n_upper + tot[1] > in.cfg.particle_capacity)
            fail(PIC_ECAPACITY, "split would exceed the particle capacity");
        // split leaves whose segment is too small go to the tail: make room first (may move
        // the lists to larger buffers)
        ensure_slots(ctx, in, s, (int64_t)tot[4] + tot[0]);
        SMArgs a{nl, sp.start, sp.end, in.cfg.ppc_min, in.cfg.ppc_max, in.cfg.ppc_target};
        k_compact_flags<<<blocks_for(nl), kT, 0, st>>>(nl, mflag, mpos, mlist);
        k_compact_flags<<<blocks_for(nl), kT, 0, st>>>(nl, sflag, spos, slist);
        count_launch(ctx, 2);
        if (tot[3] > 0) {
            k_sm_split<R><<<std::min<unsigned>(warp_blocks(tot[3]), 152u * 8u), kT, 0, st>>>(
                a, slist, tot[3], sp.start, sp.end, sp.lim, tneed, toff, tot[4], idb, next_id, soa<R>(sp, sp.cur),
                soa<R>(sp, sp.cur ^ 1));
            count_launch(ctx);
        }
        if (tot[2] > 0) {
            const size_t smem = 16384 * sizeof(unsigned long long);  // keys, padded to 2^14 >= kMergeMax
            GB_CUDA(cudaFuncSetAttribute(k_sm_merge<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            k_sm_merge<R><<<std::min<int32_t>(tot[2], 1024), 512, smem, st>>>(
                a, mlist, tot[2], sp.end, (R)(0.5 * in.cfg.m[s]), soa<R>(sp, sp.cur), soa<R>(sp, sp.cur ^ 1), err);
            count_launch(ctx);
        }
        check_launch("split_merge");
        const int32_t tail = tot[4] + tot[0];  // the split leaves moved to the tail took up to here
        GB_CUDA(cudaMemcpyAsync(sp.flags + 4, &tail, 4, cudaMemcpyHostToDevice, st));
        if (read_i32(ctx, err)) fail(PIC_EINVAL, "a leaf holds more particles than one merge block sorts (12288)");
        next_id += (unsigned long long)tot[1];
        sp.sums_valid = false;
    }
    GB_CUDA(cudaMemcpyAsync(in.d_next_id, &next_id, 8, cudaMemcpyHostToDevice, st));
    GB_CUDA(cudaStreamSynchronize(st));
    in.next_id = (int64_t)next_id;
    T.release_all();
    refresh_counts(ctx, in);
}

}  // namespace

// Any leaf refined or coarsened (its emitted count is not 1: 4 for a refined leaf, 0 or 1
// for the members of a coarsened quartet).
__global__ void k_adapt_changed(int64_t n, const int32_t *__restrict__ cnt, int32_t *__restrict__ changed) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && cnt[i] != 1) atomicOr(changed, 1);
}

void adapt_mesh(pic_ctx *ctx, Instance &in) {
    cudaStream_t st = ctx->stream;
    const int64_t n = in.nleaf;
    DeviceArena T(&ctx->cache);
    Level &g = in.lv[0];
    // |E| at leaf centres from the last solve
    double *emag = dalloc<double>(T, n);
    cell_emag(ctx, in, in.last_walls, emag);
    int32_t *refine = dalloc<int32_t>(T, n), *group = dalloc<int32_t>(T, n), *gactive = dalloc<int32_t>(T, n);
    AdaptArgs a{n, in.lmax, g.lev, in.root, in.morton, in.sp[0].start, in.sp[0].end, emag, in.cfg.refine_count,
                in.cfg.coarsen_count, in.cfg.refine_field * in.cfg.e_ref, in.cfg.coarsen_field * in.cfg.e_ref};
    k_adapt_flags<<<blocks_for(n), kT, 0, st>>>(a, refine, group, gactive);
    count_launch(ctx);
    int32_t *changed = dalloc<int32_t>(T, 1);
    // the closure settles in at most max_level sweeps; the bound is lower only under an
    // injected fault (pic_inject_fault), which tests the PIC_ETIMEOUT path
    const int max_sweeps = ctx->fault_balance_sweeps > 0 ? std::min(64, (int)ctx->fault_balance_sweeps) : 64;
    for (int it = 0; it < max_sweeps; ++it) {
        GB_CUDA(cudaMemsetAsync(changed, 0, 4, st));
        k_adapt_balance<<<blocks_for(n), kT, 0, st>>>(n, in.lmax, g.map, in.nx0 << in.lmax, in.ny0 << in.lmax,
                                                      in.cfg.bc_x == PIC_BC_PERIODIC, in.cfg.bc_y == PIC_BC_PERIODIC,
                                                      g.ix, g.iy, g.lev, refine, group, gactive, changed);
        count_launch(ctx);
        if (!read_i32(ctx, changed)) break;
        if (it == max_sweeps - 1)
            fail(PIC_ETIMEOUT, "2:1 balance closure did not settle in " + std::to_string(max_sweeps) + " sweeps");
    }
    int32_t *cnt = dalloc<int32_t>(T, n + 1), *pos = dalloc<int32_t>(T, n + 1);
    int32_t *scr = dalloc<int32_t>(T, scan_scratch_elems(n));
    k_adapt_emit_count<<<blocks_for(n), kT, 0, st>>>(n, refine, group, gactive, cnt);
    count_launch(ctx);
    exclusive_scan_i32(ctx, cnt, pos, n, scr);
    int32_t *grid_changed = dalloc<int32_t>(T, 1);
    GB_CUDA(cudaMemsetAsync(grid_changed, 0, 4, st));
    k_adapt_changed<<<blocks_for(n), kT, 0, st>>>(n, cnt, grid_changed);
    count_launch(ctx);
    const bool grid_did_change = read_i32(ctx, grid_changed) != 0;
    const int64_t n_new = read_i32(ctx, pos + n);
    uint32_t *nroot = dalloc<uint32_t>(T, n_new), *nmort = dalloc<uint32_t>(T, n_new);
    uint8_t *nlev = dalloc<uint8_t>(T, n_new);
    double *nphi = dalloc<double>(T, n_new);
    int32_t *new_of = dalloc<int32_t>(T, n), *kind = dalloc<int32_t>(T, n);
    k_adapt_emit<<<blocks_for(n), kT, 0, st>>>(n, refine, group, gactive, pos, in.root, in.morton, g.lev, in.phi,
                                               nroot, nmort, nlev, nphi, new_of, kind);
    count_launch(ctx);
    check_launch("adapt_mesh");
    // particles to the new lists (needs only the old lists and the old -> new map)
    uint32_t *morton_old = dalloc<uint32_t>(T, n);
    GB_CUDA(cudaMemcpyAsync(morton_old, in.morton, n * 4, cudaMemcpyDeviceToDevice, st));
    if (in.cfg.precision == PIC_FP64)
        adapt_particles<double>(ctx, in, n, n_new, kind, group, new_of, morton_old, T);
    else
        adapt_particles<float>(ctx, in, n, n_new, kind, group, new_of, morton_old, T);
    // rebuild the mesh structures from the new leaf description
    DeviceArena old_mesh = std::move(in.mesh_mem);
    in.mesh_mem = DeviceArena(&ctx->cache);
    DeviceArena &M = in.mesh_mem;
    uint32_t *r2 = dalloc<uint32_t>(M, n_new), *m2 = dalloc<uint32_t>(M, n_new);
    uint8_t *l2 = dalloc<uint8_t>(M, n_new);
    GB_CUDA(cudaMemcpyAsync(r2, nroot, n_new * 4, cudaMemcpyDeviceToDevice, st));
    GB_CUDA(cudaMemcpyAsync(m2, nmort, n_new * 4, cudaMemcpyDeviceToDevice, st));
    GB_CUDA(cudaMemcpyAsync(l2, nlev, n_new, cudaMemcpyDeviceToDevice, st));
    in.root = r2;
    in.morton = m2;
    in.nleaf = n_new;
    in.lv.clear();
    Level g0;
    g0.lev = l2;
    in.lv.push_back(g0);
    mesh_build_device(ctx, in, n_new);
    poisson_setup(ctx, in);
    GB_CUDA(cudaMemcpyAsync(in.phi, nphi, n_new * 8, cudaMemcpyDeviceToDevice, st));
    field_arrays(ctx, in);
    GB_CUDA(cudaStreamSynchronize(st));
    old_mesh.release_all();
    T.release_all();
    if (grid_did_change) diag_reset(ctx, in);  // §3.1: statistics counters restart when the grid changes
}

void split_merge(pic_ctx *ctx, Instance &in) {
    if (in.cfg.precision == PIC_FP64) split_merge_impl<double>(ctx, in);
    else split_merge_impl<float>(ctx, in);
}

}  // namespace gbpic
