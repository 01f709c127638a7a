// Checks of the explicit scheme's limits (§3: the explicit PIC needs cells smaller than about
// three Debye lengths and a time step below the inverse electron plasma frequency).
//
// For the electron population (species 0) of an instance: per leaf the weight sum W_l
// (particles per unit depth), so that the leaf's density is n_l = W_l / h_l^2, and the
// population's temperature from the weighted velocity variance, kT = m <|v - <v>|^2> / 3.
// Then
//     (h_l / lambda_D,l)^2 = h_l^2 n_l q^2 / (eps0 kT) = W_l q^2 / (eps0 kT),
//     (omega_pe,l dt)^2    = n_l q^2 dt^2 / (eps0 m),
// and the worst leaf of each decides.
#include <algorithm>
#include <cmath>

#include "pic_internal.cuh"

namespace gbpic {

namespace {
constexpr int kT = 256;

// The electrons' moments for the explicit-PIC limits, in two passes.  Pass 1, a fixed grid of
// kMomBlocks blocks (warps over leaves, grid-stride): per leaf the weight sum W_L (one warp
// reduction), its maximum and the maximum density W_L / h_L^2 over the warp's leaves; the
// weighted velocity sums (w v, w v^2 per component) per lane across all its leaves, reduced
// once at the end (FP64 lanes, fixed shuffle trees).  Each warp writes kMomWords words:
// {max W_L, max density, sum W_L, 3 x sum w v, 3 x sum w v^2}.  Pass 2, one block,
// combines the warps' words in a fixed tree (maxima for the first two).  The grid, the leaf
// assignment and both trees are fixed, so the result does not depend on scheduling.
constexpr int kMomBlocks = 152 * 4;
constexpr int kMomWarps = kMomBlocks * (kT / 32);
constexpr int kMomWords = 9;
template <typename R>
__global__ void __launch_bounds__(kT) k_leaf_moments(int64_t nl, const int32_t *__restrict__ start,
                                                     const int32_t *__restrict__ end, const uint8_t *__restrict__ lev,
                                                     int lmax, double hf, SoA<R> d, double *__restrict__ part) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    double m[6] = {0, 0, 0, 0, 0, 0};
    double w_max = 0.0, n_max = 0.0, w_tot = 0.0;
    for (int64_t L = warp; L < nl; L += kMomWarps) {
        double wl = 0.0;
        for (int32_t p = start[L] + lane; p < end[L]; p += 32) {
            const double w = (double)d.w[p], vx = (double)d.vx[p], vy = (double)d.vy[p], vz = (double)d.vz[p];
            wl += w;
            const double a = w * vx, b = w * vy, c = w * vz;
            m[0] += a; m[1] += b; m[2] += c;
            m[3] += a * vx; m[4] += b * vy; m[5] += c * vz;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) wl += __shfl_xor_sync(0xFFFFFFFFu, wl, o);
        const double h = (double)(1 << (lmax - lev[L])) * hf;
        w_max = fmax(w_max, wl);
        n_max = fmax(n_max, wl / (h * h));
        w_tot += wl;
    }
#pragma unroll
    for (int k = 0; k < 6; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m[k] += __shfl_xor_sync(0xFFFFFFFFu, m[k], o);
    if (lane == 0) {
        double *o = part + kMomWords * warp;
        o[0] = w_max; o[1] = n_max; o[2] = w_tot;
        for (int k = 0; k < 6; ++k) o[3 + k] = m[k];
    }
}

constexpr int kMomThreads = 512;
__global__ void __launch_bounds__(kMomThreads) k_moments_reduce(const double *__restrict__ part,
                                                                 double *__restrict__ out) {
    __shared__ double acc[kMomWords][kMomThreads];
    double a[kMomWords] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int wp = threadIdx.x; wp < kMomWarps; wp += kMomThreads) {
        const double *o = part + kMomWords * wp;
        a[0] = fmax(a[0], o[0]);
        a[1] = fmax(a[1], o[1]);
        for (int k = 2; k < kMomWords; ++k) a[k] += o[k];
    }
    for (int k = 0; k < kMomWords; ++k) acc[k][threadIdx.x] = a[k];
    __syncthreads();
    for (int h = kMomThreads / 2; h > 0; h >>= 1) {
        if ((int)threadIdx.x < h)
            for (int k = 0; k < kMomWords; ++k) {
                const double b = acc[k][threadIdx.x + h];
                acc[k][threadIdx.x] = k < 2 ? fmax(acc[k][threadIdx.x], b) : acc[k][threadIdx.x] + b;
            }
        __syncthreads();
    }
    if (threadIdx.x < kMomWords) out[threadIdx.x] = acc[threadIdx.x][0];
}

pic_status limits(const pic_config &c, double n_max, double w_max, double t_e_ev, double *dx_ld, double *wdt) {
    const double q2 = c.q[0] * c.q[0];
    const double kT = t_e_ev * c.qe;
    double a = 0.0, b = 0.0;
    if (w_max > 0.0) a = kT > 0.0 ? std::sqrt(w_max * q2 / (c.eps0 * kT)) : INFINITY;
    if (n_max > 0.0) b = std::sqrt(n_max * q2 / (c.eps0 * c.m[0])) * c.dt;
    if (dx_ld) *dx_ld = a;
    if (wdt) *wdt = b;
    return (a > 3.0 || b > 1.0) ? PIC_WARN_STABILITY : PIC_OK;
}
}  // namespace

// The two ratios for the current electron population of `in` (synchronises the stream).
pic_status stability_check(pic_ctx *ctx, Instance &in, double *dx_ld, double *wdt, double *t_e_ev) {
    Species &sp = in.sp[0];
    const int64_t nl = in.nleaf;
    if (!sp.start) {
        if (t_e_ev) *t_e_ev = 0.0;
        return limits(in.cfg, 0.0, 0.0, 0.0, dx_ld, wdt);
    }
    DeviceArena T(&ctx->cache);
    double *part = dalloc<double>(T, (size_t)kMomWords * kMomWarps + kMomWords);
    double *tot = part + (size_t)kMomWords * kMomWarps;
    const Level &g = in.lv[0];
    const double hf = in.h0 / (double)(1 << in.lmax);
    if (in.cfg.precision == PIC_FP64)
        k_leaf_moments<double><<<kMomBlocks, kT, 0, ctx->stream>>>(nl, sp.start, sp.end, g.lev, in.lmax, hf,
                                                                   soa<double>(sp, sp.cur), part);
    else
        k_leaf_moments<float><<<kMomBlocks, kT, 0, ctx->stream>>>(nl, sp.start, sp.end, g.lev, in.lmax, hf,
                                                                  soa<float>(sp, sp.cur), part);
    k_moments_reduce<<<1, kMomThreads, 0, ctx->stream>>>(part, tot);
    count_launch(ctx, 2);
    check_launch("stability_check");
    double r[kMomWords];
    GB_CUDA(cudaMemcpyAsync(r, tot, sizeof(r), cudaMemcpyDeviceToHost, ctx->stream));
    GB_CUDA(cudaStreamSynchronize(ctx->stream));
    T.release_all();
    const double w_max = r[0], n_max = r[1], W = r[2], *mv = r + 3, *mv2 = r + 6;
    double var = 0.0;
    if (W > 0.0)
        for (int k = 0; k < 3; ++k) var += std::max(0.0, mv2[k] / W - (mv[k] / W) * (mv[k] / W));
    const double te = in.cfg.m[0] * var / 3.0 / in.cfg.qe;
    if (t_e_ev) *t_e_ev = te;
    return limits(in.cfg, n_max, w_max, te, dx_ld, wdt);
}

}  // namespace gbpic

extern "C" pic_status pic_stability_limits(const pic_config *cfg, double n_e_max, double w_leaf_max, double t_e_ev,
                                           double *dx_over_debye, double *wpe_dt) {
    if (!cfg || !(n_e_max >= 0.0) || !(w_leaf_max >= 0.0) || !(t_e_ev >= 0.0) || !(cfg->eps0 > 0.0) ||
        !(cfg->m[0] > 0.0) || !(cfg->qe > 0.0)) {
        gbpic::set_error("pic_stability_limits: bad argument");
        return PIC_EINVAL;
    }
    gbpic::set_error("");
    return gbpic::limits(*cfg, n_e_max, w_leaf_max, t_e_ev, dx_over_debye, wpe_dt);
}

// ------------------------------------------------------------------------------------
// Time-averaged diagnostics (§3.3: the discharge's RF-cycle averages of n_e, n_i, T_e, phi
// and the EEDF; §3.1: statistics counters are reset when the grid changes).  Each step, after
// the field solve, the stored state (x^n, v^{n-1/2}, the potential of the step's solve) is
// added to per-leaf sums: the electron and ion weights, the electrons' weighted kinetic
// energy eps = m |v|^2 / (2 qe) [eV] and phi; and the electrons whose position lies in the
// region [x0, x1) x [y0, y1) add their weight to the bin floor(eps / d_eps) of the energy
// histogram (energies at or above eps_max are not binned).  Everything is summed in a fixed
// order: one warp per leaf with fixed shuffle trees, each warp's histogram in its own shared
// memory (lanes of one bin summed in lane order), the per-warp histograms then summed in
// warp order, so two runs give the same bits.
// ------------------------------------------------------------------------------------
namespace gbpic {

namespace {
constexpr int kDiagBlocks = 152 * 4;  // fixed grid: the histogram's summation order is fixed
constexpr int kDiagWarps = kDiagBlocks * (kT / 32);
constexpr int kMaxBins = 512;

struct DiagArgs {
    int64_t nl;
    int nsp, lmax, nbins;
    const int32_t *start[2], *end[2];
    const uint8_t *lev;
    const int32_t *ix, *iy;
    double hf, half_m_over_qe, inv_deps, eps_max;
    double region[4];
    const double *phi;
    double *leaf, *part;
};

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

template <typename R>
__global__ void __launch_bounds__(kT) k_diag_sample(DiagArgs a, SoA<R> e, SoA<R> ion) {
    extern __shared__ double hist_all[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    double *hist = hist_all + wib * a.nbins;
    for (int b = lane; b < a.nbins; b += 32) hist[b] = 0.0;
    __syncwarp();
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t L = warp; L < a.nl; L += nw) {
        const int32_t s = 1 << (a.lmax - a.lev[L]);
        const double x0 = (double)a.ix[L] * a.hf, y0 = (double)a.iy[L] * a.hf, hl = (double)s * a.hf;
        double we = 0.0, wee = 0.0;
        for (int32_t c0 = a.start[0][L]; c0 < a.end[0][L]; c0 += 32) {
            const int32_t p = c0 + lane;
            double w = 0.0, eps = 0.0;
            int bin = -1;
            if (p < a.end[0][L]) {
                w = (double)e.w[p];
                const double vx = (double)e.vx[p], vy = (double)e.vy[p], vz = (double)e.vz[p];
                // rounded step by step (no contraction), so that the bin is decided on the
                // value the oracle computes from the same velocities
                eps = __dmul_rn(a.half_m_over_qe, __dadd_rn(__dadd_rn(__dmul_rn(vx, vx), __dmul_rn(vy, vy)),
                                                            __dmul_rn(vz, vz)));
                const double x = x0 + (double)e.u[p] * hl, y = y0 + (double)e.v[p] * hl;
                if (x >= a.region[0] && x < a.region[1] && y >= a.region[2] && y < a.region[3] && eps < a.eps_max) {
                    bin = (int)floor(__dmul_rn(eps, a.inv_deps));
                    if (bin >= a.nbins) bin = -1;
                }
            }
            we += w;
            wee += w * eps;
            // lanes of one bin: their weights summed in lane order by the group's first lane
            const uint32_t peers = __match_any_sync(0xFFFFFFFFu, bin);
            double sum = 0.0;
            for (int j = 0; j < 32; ++j) {
                const double wj = __shfl_sync(0xFFFFFFFFu, w, j);
                if ((peers >> j) & 1u) sum += wj;
            }
            if (bin >= 0 && (peers & ((1u << lane) - 1u)) == 0) hist[bin] += sum;
            __syncwarp();
        }
        double wi = 0.0;
        if (a.nsp > 1)
            for (int32_t p = a.start[1][L] + lane; p < a.end[1][L]; p += 32) wi += (double)ion.w[p];
        we = warp_sum_d(we);
        wee = warp_sum_d(wee);
        wi = warp_sum_d(wi);
        if (lane == 0) {
            double *o = a.leaf + 4 * L;
            o[0] += we;
            o[1] += wi;
            o[2] += wee;
            o[3] += a.phi[L];
        }
    }
    __syncwarp();
    for (int b = lane; b < a.nbins; b += 32) a.part[warp * a.nbins + b] = hist[b];
}

// eedf[b] += sum over warps, in warp order, of the warps' histograms
__global__ void k_diag_eedf(int nbins, const double *__restrict__ part, double *__restrict__ eedf) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbins) return;
    double s = 0.0;
    for (int w = 0; w < kDiagWarps; ++w) s += part[(int64_t)w * nbins + b];
    eedf[b] += s;
}

__global__ void k_diag_field(int64_t nl, int field, int64_t samples, const double *__restrict__ leaf,
                             const uint8_t *__restrict__ lev, int lmax, double hf, double *__restrict__ out) {
    const int64_t L = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (L >= nl) return;
    const double h = (double)(1 << (lmax - lev[L])) * hf;
    const double *o = leaf + 4 * L;
    const double ns = samples > 0 ? (double)samples : 1.0;
    double r = 0.0;
    switch (field) {
    case PIC_FIELD_AVG_NE: r = o[0] / (ns * h * h); break;
    case PIC_FIELD_AVG_NI: r = o[1] / (ns * h * h); break;
    case PIC_FIELD_AVG_TE: r = o[0] > 0.0 ? (2.0 / 3.0) * o[2] / o[0] : 0.0; break;
    default: r = o[3] / ns; break;
    }
    out[L] = samples > 0 ? r : 0.0;
}
}  // namespace

void diag_reset(pic_ctx *ctx, Instance &in) {
    Diag &d = in.diag;
    if (!d.on) return;
    if (d.nleaf != in.nleaf || !d.leaf) {
        if (d.leaf) d.mem.release(d.leaf);
        d.leaf = dalloc<double>(d.mem, 4 * in.nleaf);
        d.nleaf = in.nleaf;
    }
    GB_CUDA(cudaMemsetAsync(d.leaf, 0, 4 * 8 * in.nleaf, ctx->stream));
    GB_CUDA(cudaMemsetAsync(d.eedf, 0, 8 * (size_t)d.nbins, ctx->stream));
    d.samples = 0;
}

void diag_accumulate(pic_ctx *ctx, Instance &in) {
    Diag &d = in.diag;
    if (!d.on) return;
    if (d.nleaf != in.nleaf) diag_reset(ctx, in);
    const pic_config &c = in.cfg;
    DiagArgs a{};
    a.nl = in.nleaf;
    a.nsp = c.n_species;
    a.lmax = in.lmax;
    a.nbins = d.nbins;
    for (int s = 0; s < 2; ++s) {
        const Species &sp = in.sp[std::min(s, c.n_species - 1)];
        a.start[s] = sp.start;
        a.end[s] = sp.end;
    }
    if (!a.start[0]) return;
    if (c.n_species > 1 && !in.sp[1].start) a.nsp = 1;
    const Level &g = in.lv[0];
    a.lev = g.lev; a.ix = g.ix; a.iy = g.iy;
    a.hf = in.h0 / (double)(1 << in.lmax);
    a.half_m_over_qe = 0.5 * c.m[0] / c.qe;
    a.eps_max = d.eps_max;
    a.inv_deps = (double)d.nbins / d.eps_max;
    for (int k = 0; k < 4; ++k) a.region[k] = d.region[k];
    a.phi = in.phi;
    a.leaf = d.leaf;
    a.part = d.part;
    const size_t smem = (size_t)(kT / 32) * d.nbins * sizeof(double);
    Species &e = in.sp[0];
    Species &ion = in.sp[a.nsp > 1 ? 1 : 0];
    if (c.precision == PIC_FP64)
        k_diag_sample<double><<<kDiagBlocks, kT, smem, ctx->stream>>>(a, soa<double>(e, e.cur), soa<double>(ion, ion.cur));
    else
        k_diag_sample<float><<<kDiagBlocks, kT, smem, ctx->stream>>>(a, soa<float>(e, e.cur), soa<float>(ion, ion.cur));
    k_diag_eedf<<<(d.nbins + kT - 1) / kT, kT, 0, ctx->stream>>>(d.nbins, d.part, d.eedf);
    count_launch(ctx, 2);
    check_launch("diag_accumulate");
    ++d.samples;
}

void diag_read_field(pic_ctx *ctx, Instance &in, int field, double *out_dev) {
    Diag &d = in.diag;
    const int64_t nl = in.nleaf;
    if (!d.on || d.nleaf != nl) {
        GB_CUDA(cudaMemsetAsync(out_dev, 0, 8 * nl, ctx->stream));
        return;
    }
    k_diag_field<<<(unsigned)std::max<int64_t>(1, (nl + kT - 1) / kT), kT, 0, ctx->stream>>>(
        nl, field, d.samples, d.leaf, in.lv[0].lev, in.lmax, in.h0 / (double)(1 << in.lmax), out_dev);
    count_launch(ctx);
    check_launch("diag_read_field");
}

void diag_enable(pic_ctx *ctx, Instance &in, int nbins, double eps_max, const double *region) {
    Diag &d = in.diag;
    d.mem.cache = &ctx->cache;
    d.mem.release_all();
    d.leaf = d.eedf = d.part = nullptr;
    d.nleaf = 0;
    d.on = nbins > 0;
    if (!d.on) return;
    if (nbins > kMaxBins) fail(PIC_EINVAL, "pic_diag_enable: at most 512 energy bins");
    if (!(eps_max > 0.0)) fail(PIC_EINVAL, "pic_diag_enable: eps_max must be positive");
    d.nbins = nbins;
    d.eps_max = eps_max;
    if (region) {
        for (int k = 0; k < 4; ++k) d.region[k] = region[k];
    } else {
        d.region[0] = d.region[2] = -INFINITY;
        d.region[1] = d.region[3] = INFINITY;
    }
    d.eedf = dalloc<double>(d.mem, nbins);
    d.part = dalloc<double>(d.mem, (size_t)kDiagWarps * nbins);
    static bool attr = false;
    if (!attr) {
        const int smax = (kT / 32) * kMaxBins * (int)sizeof(double);
        GB_CUDA(cudaFuncSetAttribute(k_diag_sample<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax));
        GB_CUDA(cudaFuncSetAttribute(k_diag_sample<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, smax));
        attr = true;
    }
    diag_reset(ctx, in);
}

void diag_read_eedf(pic_ctx *ctx, Instance &in, double *f, int64_t *samples) {
    Diag &d = in.diag;
    std::vector<double> h(d.nbins);
    GB_CUDA(cudaMemcpyAsync(h.data(), d.eedf, 8 * (size_t)d.nbins, cudaMemcpyDeviceToHost, ctx->stream));
    GB_CUDA(cudaStreamSynchronize(ctx->stream));
    double tot = 0.0;
    for (double v : h) tot += v;
    const double deps = d.eps_max / d.nbins;
    for (int b = 0; b < d.nbins; ++b) f[b] = tot > 0.0 ? h[b] / (tot * deps) : 0.0;
    if (samples) *samples = d.samples;
}

}  // namespace gbpic
