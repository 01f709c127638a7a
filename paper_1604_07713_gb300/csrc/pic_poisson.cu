// Poisson solve on the composite leaf mesh (§3: multigrid Poisson solver with the potential
// at cell centres).  Mixed precision: the residual b - A phi, its norm and the correction
// phi += e are FP64 (iterative refinement); each correction e comes from one FP32
// geometric-multigrid V-cycle over the tree-clamped and root-coarsened levels, with two
// red-black Gauss-Seidel sweeps before and after the coarse correction, summed restriction
// and piecewise-constant prolongation; the coarsest level (at most 64 cells) is solved by its
// dense inverse, built on the host in FP64, or else by conjugate gradients.  Levels of at
// most 8192 cells live in one block's shared memory; when every level does, the whole solve
// (FP64 residual, V-cycles, convergence test) is a single launch of a thread-block cluster
// that spreads the FP64 work over its SMs (one CTA per instance in a batch).  Larger meshes
// run one CUDA graph per solve whose WHILE node repeats the cycle until the device decides.
#include <algorithm>
#include <cmath>

#include <cooperative_groups.h>

#include "pic_internal.cuh"

namespace gbpic {

namespace {
constexpr int kT = 256;
constexpr int kRedBlocks = 304;  // 2 x 152 SMs: fixed so that the FP64 sums are deterministic
constexpr int kNu = 2;          // red-black Gauss-Seidel sweeps before and after the coarse correction
constexpr double kCoarseTol2 = 1e-10;  // coarsest solve (multi-block path): ||r|| <= 1e-5 ||b||
constexpr float kSmCoarseTol2 = 1e-6f; // coarsest solve inside a V-cycle in shared memory: 1e-3
inline unsigned blocks_for(int64_t n, int t = kT) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

// Launch with programmatic stream serialization (the kernel calls pdl_chain first).
template <typename... KArgs, typename... Args>
void pdl(void (*k)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t st, Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    GB_CUDA(cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...));
}

// Programmatic dependent launch: a kernel of the solve's chain lets the next one be scheduled
// at once and waits, before touching memory, for the previous one to complete (the waits are
// no-ops for a kernel launched without the programmatic-serialization attribute).
__device__ __forceinline__ void pdl_chain() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" :::);
}

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double sh[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
    __syncthreads();
    return s;  // valid in thread 0
}

// out = sums of the block partials (one warp: lanes in a fixed order, then a fixed tree,
// so the result does not depend on timing).
__global__ void k_finish_sums(int nparts, const double *__restrict__ part, double *__restrict__ out) {
    pdl_chain();
    const int lane = threadIdx.x & 31;
    if (threadIdx.x >= 32) return;
    double a = 0.0, b = 0.0;
    for (int k = lane; k < nparts; k += 32) { a += part[2 * k]; b += part[2 * k + 1]; }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xFFFFFFFFu, a, o);
        b += __shfl_down_sync(0xFFFFFFFFu, b, o);
    }
    if (lane == 0) { out[0] = a; out[1] = b; }
}

// The larger of two relative residuals, NaN if either is NaN: a non-finite residual (NaN or
// Inf in the charge density or the potential) stays visible to the host.
__device__ __forceinline__ double worst_residual(double a, double b) {
    return (a != a || b != b) ? __longlong_as_double(0x7FF8000000000000ll) : fmax(a, b);
}

// r = b - A phi (FP64) with r^2 and b^2 summed per block (fixed grid), then, in the block that
// arrives last on the ticket counter (after a fence, so every block's sums are visible), the
// block sums added as k_finish_sums adds them, the solve's statistics and whether another
// cycle runs (the condition of the graph's WHILE node; first = 1 before the first cycle),
// and the counter reset for the next launch.
__global__ void k_residual_decide(int64_t n, const int32_t *__restrict__ col, const double *__restrict__ val,
                                  const double *__restrict__ diag, const double *__restrict__ phi,
                                  const double *__restrict__ b, double *__restrict__ r, float *__restrict__ r32,
                                  double *__restrict__ part, uint32_t *__restrict__ ticket,
                                  cudaGraphConditionalHandle h, double tol, int maxc, double *__restrict__ stats,
                                  int first) {
    pdl_chain();
    __shared__ bool last;
    double rr = 0.0, bb = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double ax = diag[i] * phi[i];
#pragma unroll
        for (int j = 0; j < kEll; ++j) {
            const int32_t c = col[(int64_t)j * n + i];
            if (c >= 0) ax += val[(int64_t)j * n + i] * phi[c];
        }
        const double ri = b[i] - ax;
        r[i] = ri;
        r32[i] = (float)ri;
        rr += ri * ri;
        bb += b[i] * b[i];
    }
    const double s1 = block_sum(rr);
    const double s2 = block_sum(bb);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = s1;
        part[2 * blockIdx.x + 1] = s2;
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last || threadIdx.x >= 32) return;
    __threadfence();
    const int lane = threadIdx.x;
    double a = 0.0, c = 0.0;
    for (int k = lane; k < (int)gridDim.x; k += 32) { a += __ldcg(part + 2 * k); c += __ldcg(part + 2 * k + 1); }
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xFFFFFFFFu, a, o);
        c += __shfl_down_sync(0xFFFFFFFFu, c, o);
    }
    if (lane == 0) {
        *ticket = 0u;
        const double rel = c > 0.0 ? sqrt(a / c) : sqrt(a);
        const double cyc = first ? 0.0 : stats[0] + 1.0;
        const bool done = rel <= tol || (c == 0.0 && a == 0.0) || cyc >= (double)maxc;
        stats[0] = cyc;
        stats[1] = rel;
        if (done) stats[2] = worst_residual(stats[2], rel);
        cudaGraphSetConditional(h, done ? 0u : 1u);
    }
}

// Zero-mean projections for a fully periodic (singular) problem: area weights a = s^2.
__global__ void k_area_moments(int64_t n, const uint8_t *__restrict__ lev, int lmax, const double *__restrict__ v,
                               double *__restrict__ part) {
    double sv = 0.0, sa = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double s = (double)(1 << (lmax - lev[i]));
        sv += v[i];
        sa += s * s;
    }
    const double s1 = block_sum(sv), s2 = block_sum(sa);
    if (threadIdx.x == 0) { part[2 * blockIdx.x] = s1; part[2 * blockIdx.x + 1] = s2; }
}
__global__ void k_area_weighted(int64_t n, const uint8_t *__restrict__ lev, int lmax, const double *__restrict__ v,
                                double *__restrict__ part) {
    pdl_chain();
    double sv = 0.0, sa = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double s = (double)(1 << (lmax - lev[i]));
        sv += s * s * v[i];
        sa += s * s;
    }
    const double s1 = block_sum(sv), s2 = block_sum(sa);
    if (threadIdx.x == 0) { part[2 * blockIdx.x] = s1; part[2 * blockIdx.x + 1] = s2; }
}
// v -= mode * (sum / area_total): mode 0 subtracts an area-proportional share (RHS
// compatibility), mode 1 a constant (zero area-weighted mean of the potential).
__global__ void k_project(int64_t n, const uint8_t *__restrict__ lev, int lmax, const double *__restrict__ sums,
                          double *__restrict__ v, int mode) {
    pdl_chain();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double s = (double)(1 << (lmax - lev[i]));
    const double k = sums[0] / sums[1];
    v[i] -= mode == 0 ? k * s * s : k;
}

// Initial guess of a solve: phi <- 2 phi - phi_prev (linear extrapolation in time of the last
// two solutions), phi_prev <- phi.  With only one earlier solve: phi_prev <- phi.
__global__ void k_extrapolate(int64_t n, double *__restrict__ phi, double *__restrict__ prev, int both) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double p = phi[i];
    if (both) phi[i] = 2.0 * p - prev[i];
    prev[i] = p;
}

__global__ void k_add_correction(int64_t n, const float *__restrict__ e, double *__restrict__ phi) {
    pdl_chain();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) phi[i] += (double)e[i];
}

// One colour of a red-black Gauss-Seidel sweep, written out of place so that the result does
// not depend on thread order (cells of the same colour can touch on a non-uniform mesh):
// colour-c cells get D^-1 (b - offdiag x_in), others copy x_in.  zero_in: x_in is zero.
__global__ void k_rbgs_half(int64_t n, const int32_t *__restrict__ col, const float *__restrict__ val,
                            const float *__restrict__ dinv, const uint8_t *__restrict__ color, int c,
                            const float *__restrict__ b, const float *__restrict__ xin, float *__restrict__ xout,
                            int zero_in) {
    pdl_chain();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (color[i] != c) {
        xout[i] = zero_in ? 0.0f : xin[i];
        return;
    }
    float off = 0.0f;
    if (!zero_in) {
#pragma unroll
        for (int j = 0; j < kEll; ++j) {
            const int32_t cc = col[(int64_t)j * n + i];
            if (cc >= 0) off = fmaf(val[(int64_t)j * n + i], xin[cc], off);
        }
    }
    xout[i] = dinv[i] * (b[i] - off);
}

// The first two half sweeps of a pre-smoothing from x = 0 in one kernel: the first (colour 0
// from zero) leaves t = D^-1 (b - 0) on colour 0 and 0 elsewhere, which the second (colour 1)
// forms on the fly; the same arithmetic as the two half sweeps, so the same values.
__global__ void k_rbgs_first(int64_t n, const int32_t *__restrict__ col, const float *__restrict__ val,
                             const float *__restrict__ dinv, const uint8_t *__restrict__ color,
                             const float *__restrict__ b, float *__restrict__ xout) {
    pdl_chain();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (color[i] != 1) {
        xout[i] = dinv[i] * (b[i] - 0.0f);
        return;
    }
    float off = 0.0f;
#pragma unroll
    for (int j = 0; j < kEll; ++j) {
        const int32_t cc = col[(int64_t)j * n + i];
        if (cc >= 0) off = fmaf(val[(int64_t)j * n + i], color[cc] == 0 ? dinv[cc] * (b[cc] - 0.0f) : 0.0f, off);
    }
    xout[i] = dinv[i] * (b[i] - off);
}

// Injection of the coarse correction (x += xc[parent]) fused into the first half sweep after
// it: every value the sweep reads gets its correction added on the way, with the same
// additions as a separate injection pass.
__global__ void k_rbgs_half_prolong(int64_t n, const int32_t *__restrict__ col, const float *__restrict__ val,
                                    const float *__restrict__ dinv, const uint8_t *__restrict__ color, int c,
                                    const float *__restrict__ b, const float *__restrict__ xin,
                                    const int32_t *__restrict__ parent, const float *__restrict__ xc,
                                    float *__restrict__ xout) {
    pdl_chain();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (color[i] != c) {
        xout[i] = xin[i] + xc[parent[i]];
        return;
    }
    float off = 0.0f;
#pragma unroll
    for (int j = 0; j < kEll; ++j) {
        const int32_t cc = col[(int64_t)j * n + i];
        if (cc >= 0) off = fmaf(val[(int64_t)j * n + i], xin[cc] + xc[parent[cc]], off);
    }
    xout[i] = dinv[i] * (b[i] - off);
}

// Coarse right-hand side: summed residuals of the children; zero coarse iterate.
__global__ void k_restrict_residual(int64_t nc, const int32_t *__restrict__ child4, int64_t nf,
                                    const int32_t *__restrict__ col, const float *__restrict__ val,
                                    const float *__restrict__ dinv, const float *__restrict__ bf,
                                    const float *__restrict__ xf, float *__restrict__ bc, float *__restrict__ xc) {
    pdl_chain();
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nc) return;
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int32_t i = child4[4 * p + k];
        if (i < 0) continue;
        float ax = xf[i] / dinv[i];
#pragma unroll
        for (int j = 0; j < kEll; ++j) {
            const int32_t c = col[(int64_t)j * nf + i];
            if (c >= 0) ax = fmaf(val[(int64_t)j * nf + i], xf[c], ax);
        }
        s += bf[i] - ax;
    }
    bc[p] = s;
    xc[p] = 0.0f;
}


// One-block Jacobi-preconditioned CG on the coarsest level (symmetric: one uniform level).
__global__ void __launch_bounds__(1024) k_coarse_cg(int64_t n, const int32_t *__restrict__ col,
                                                    const float *__restrict__ val, const float *__restrict__ dinv,
                                                    const float *__restrict__ b, float *__restrict__ x,
                                                    float *__restrict__ r, float *__restrict__ p,
                                                    float *__restrict__ q, int singular, int maxit) {
    pdl_chain();
    __shared__ double red[32];
    __shared__ double bcast;
    auto bsum = [&](double v) -> double {
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
        if (lane == 0) red[wid] = v;
        __syncthreads();
        if (threadIdx.x == 0) {
            double s = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
            bcast = s;
        }
        __syncthreads();
        const double out = bcast;
        __syncthreads();
        return out;
    };
    double mb = 0.0;
    if (singular) {
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) mb += b[i];
        mb = bsum(mb) / (double)n;
    }
    double rz = 0.0, bb = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        const float ri = b[i] - (float)mb;
        x[i] = 0.0f;
        r[i] = ri;
        const float zi = dinv[i] * ri;
        p[i] = zi;
        rz += (double)ri * zi;
        bb += (double)ri * ri;
    }
    rz = bsum(rz);
    bb = bsum(bb);
    if (bb == 0.0) return;
    for (int it = 0; it < maxit; ++it) {
        double pq = 0.0;
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
            float ax = p[i] / dinv[i];
            for (int j = 0; j < kEll; ++j) {
                const int32_t c = col[(int64_t)j * n + i];
                if (c >= 0) ax = fmaf(val[(int64_t)j * n + i], p[c], ax);
            }
            q[i] = ax;
            pq += (double)p[i] * ax;
        }
        pq = bsum(pq);
        if (pq <= 0.0) break;
        const float alpha = (float)(rz / pq);
        double rr = 0.0, rz2 = 0.0;
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
            x[i] += alpha * p[i];
            const float ri = r[i] - alpha * q[i];
            r[i] = ri;
            rr += (double)ri * ri;
            rz2 += (double)ri * dinv[i] * ri;
        }
        rr = bsum(rr);
        rz2 = bsum(rz2);
        if (rr <= kCoarseTol2 * bb) break;
        const float beta = (float)(rz2 / rz);
        rz = rz2;
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) p[i] = dinv[i] * r[i] + beta * p[i];
        __syncthreads();
    }
    if (singular) {
        double mx = 0.0;
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) mx += x[i];
        mx = bsum(mx) / (double)n;
        for (int64_t i = threadIdx.x; i < n; i += blockDim.x) x[i] -= (float)mx;
    }
}

// ---- levels held in shared memory by one block (n <= kSmallN cells each) ----------------
constexpr int kSmallN = 8192;          // 8 cells per thread of a 1024-thread block
constexpr int kMaxSmallLevels = 16;
constexpr int kSmallSmemCap = 200 * 1024;

struct SmallLevel {
    int32_t n;
    const int32_t *col;
    const float *val, *dinv;
    const uint8_t *color;
    const int32_t *child4;  // children (in the finer level) of this level's cells
    const int32_t *parent;  // this level's cells -> cells of the next coarser level
    int32_t off;            // smem offset (floats) of x; b follows at off + n
    // A level of root boxes only (no refinement) is a row-major nx x ny grid whose operator
    // is the 5-point stencil; it is applied from the cell index, without the ELL arrays.
    int32_t uniform, nx, ny;
    uint32_t nx_magic;   // floor(i / nx) == mdiv(i, nx_magic) for every cell index i < n
    uint32_t nxh_magic;  // the same for nx / 2 (uniform levels with even nx)
};
struct SmallDesc {
    int nlev;  // levels g0 .. g0 + nlev - 1 live in shared memory
    int bcx, bcy;
    SmallLevel lv[kMaxSmallLevels];
    int32_t off_cg;  // smem offset of the coarsest CG vectors r, p, q (3 n)
    int32_t smem_floats;
    const double *cinv;  // coarsest level: dense FP64 inverse (n x n, row-major), or null (CG)
};

// floor(i / d) by a multiply-high reciprocal m = floor((2^32 - 1) / d) + 1; m = 0 stands for
// d = 1 (whose reciprocal 2^32 has no 32-bit form).
__host__ __device__ __forceinline__ uint32_t mdiv_magic(uint32_t d) { return d <= 1u ? 0u : 0xFFFFFFFFu / d + 1u; }
__device__ __forceinline__ int mdiv(int i, uint32_t m) { return m ? (int)__umulhi((uint32_t)i, m) : i; }

// Neighbour sum s and diagonal d of row i, so that (A x)_i = d x_i - s.  Uniform levels:
// face conductance 1 to each neighbour, 2 to a Dirichlet wall, none at a Neumann wall.
template <typename T>
__device__ __forceinline__ T uni_row(int nx, int ny, uint32_t magic, int bcx, int bcy, const T *x, int i, T &d) {
    const int iy = mdiv(i, magic), ix = i - iy * nx;
    T s = 0;
    int dd = 0;  // counted in integers: the diagonal is converted once
    if (ix > 0) { s += x[i - 1]; dd += 1; }
    else if (bcx == PIC_BC_PERIODIC) { s += x[i + nx - 1]; dd += 1; }
    else if (bcx == PIC_BC_DIRICHLET) dd += 2;
    if (ix < nx - 1) { s += x[i + 1]; dd += 1; }
    else if (bcx == PIC_BC_PERIODIC) { s += x[i - nx + 1]; dd += 1; }
    else if (bcx == PIC_BC_DIRICHLET) dd += 2;
    if (iy > 0) { s += x[i - nx]; dd += 1; }
    else if (bcy == PIC_BC_PERIODIC) { s += x[i + (ny - 1) * nx]; dd += 1; }
    else if (bcy == PIC_BC_DIRICHLET) dd += 2;
    if (iy < ny - 1) { s += x[i + nx]; dd += 1; }
    else if (bcy == PIC_BC_PERIODIC) { s += x[i - (ny - 1) * nx]; dd += 1; }
    else if (bcy == PIC_BC_DIRICHLET) dd += 2;
    d = (T)dd;
    return s;
}

__device__ __forceinline__ float sm_row(const SmallDesc &D, const SmallLevel &L, const float *x, int i, float &d,
                                        float &dinv) {
    if (L.uniform) {
        const float s = uni_row<float>(L.nx, L.ny, L.nx_magic, D.bcx, D.bcy, x, i, d);
        dinv = __frcp_rn(d);
        return s;
    }
    float off = 0.0f;
#pragma unroll
    for (int j = 0; j < kEll; ++j) {
        const int32_t c = L.col[(int64_t)j * L.n + i];
        if (c >= 0) off = fmaf(L.val[(int64_t)j * L.n + i], x[c], off);
    }
    dinv = L.dinv[i];
    d = __frcp_rn(dinv);
    return -off;
}
__device__ __forceinline__ float sm_row(const SmallDesc &D, const SmallLevel &L, const float *x, int i, float &d) {
    float dinv;
    return sm_row(D, L, x, i, d, dinv);
}

__device__ __forceinline__ int sm_color(const SmallLevel &L, int i) {
    if (!L.uniform) return L.color[i];
    const int iy = mdiv(i, L.nx_magic);
    return (i - iy * L.nx + iy) & 1;
}

// Red-black Gauss-Seidel sweep in shared memory; each colour's new values are computed from
// the current vector before any is written (deterministic on non-uniform meshes).  The block
// has 1024 threads; thread t owns cells t + 1024 k, k < 8, so the new values stay in registers.
constexpr int kPerThread = kSmallN / 1024;
__device__ void sm_smooth(const SmallDesc &D, const SmallLevel &L, float *x, const float *b, bool first) {
    if (first) {
        for (int i = threadIdx.x; i < L.n; i += blockDim.x) x[i] = 0.0f;
        __syncthreads();
    }
    if (L.uniform && (L.nx & 1) == 0) {
        // colour c of an even-width grid: in row iy the cells ix = 2m + ((c + iy) & 1)
        const int half = L.n >> 1, nxh = L.nx >> 1;
        for (int c = 0; c < 2; ++c) {
            float t[kPerThread / 2];
            int cell[kPerThread / 2];
#pragma unroll
            for (int k = 0; k < kPerThread / 2; ++k) {
                const int j = threadIdx.x + 1024 * k;
                cell[k] = -1;
                if (j < half) {
                    const int iy = mdiv(j, L.nxh_magic), m = j - iy * nxh;
                    const int i = iy * L.nx + 2 * m + ((c + iy) & 1);
                    float d, dinv;
                    const float sn = sm_row(D, L, x, i, d, dinv);
                    t[k] = (b[i] + sn) * dinv;
                    cell[k] = i;
                }
            }
            __syncthreads();
#pragma unroll
            for (int k = 0; k < kPerThread / 2; ++k)
                if (cell[k] >= 0) x[cell[k]] = t[k];
            __syncthreads();
        }
        return;
    }
    for (int c = 0; c < 2; ++c) {
        float t[kPerThread];
        bool mine[kPerThread];
#pragma unroll
        for (int k = 0; k < kPerThread; ++k) {
            const int i = threadIdx.x + 1024 * k;
            mine[k] = i < L.n && sm_color(L, i) == c;
            t[k] = 0.0f;
            if (mine[k]) {
                float d, dinv;
                const float sn = sm_row(D, L, x, i, d, dinv);
                t[k] = (b[i] + sn) * dinv;
            }
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kPerThread; ++k)
            if (mine[k]) x[threadIdx.x + 1024 * k] = t[k];
        __syncthreads();
    }
}



__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}
__device__ float sm_block_sumf(float v, float *red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_sumf(v);
    if (lane == 0) red[wid] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        red[32] = s;
    }
    __syncthreads();
    const float out = red[32];
    __syncthreads();
    return out;
}

// Coarsest level: Jacobi-preconditioned CG in shared memory (one uniform level: symmetric),
// all in FP32 (GB300's FP64 rate is a small fraction of FP32), to 1e-3 relative residual,
// which is all a coarse-grid correction needs.  Up to 256 cells it runs on the first warp.
__device__ void sm_coarse_cg(const SmallDesc &D, const SmallLevel &L, float *x, const float *b, float *r, float *p,
                             float *q, bool singular, float *red) {
    const int n = L.n;
    const int maxit = min(2 * n + 10, 500);
    const bool warp_only = n <= 256;
    if (warp_only && threadIdx.x >= 32) {
        __syncthreads();
        return;
    }
    const int stride = warp_only ? 32 : blockDim.x;
    auto sum = [&](float v) -> float { return warp_only ? warp_sumf(v) : sm_block_sumf(v, red); };
    auto sync = [&]() { if (warp_only) __syncwarp(); else __syncthreads(); };
    float mb = 0.0f;
    if (singular) {
        for (int i = threadIdx.x; i < n; i += stride) mb += b[i];
        mb = sum(mb) / (float)n;
    }
    float rz = 0.0f, bb = 0.0f;
    for (int i = threadIdx.x; i < n; i += stride) {
        float d, dinv;
        sm_row(D, L, b, i, d, dinv);  // diagonal only
        const float ri = b[i] - mb;
        x[i] = 0.0f;
        r[i] = ri;
        const float zi = ri * dinv;
        p[i] = zi;
        rz += ri * zi;
        bb += ri * ri;
    }
    rz = sum(rz);
    bb = sum(bb);
    sync();
    if (bb > 0.0f) {
        for (int it = 0; it < maxit; ++it) {
            float pq = 0.0f;
            for (int i = threadIdx.x; i < n; i += stride) {
                float d;
                const float sn = sm_row(D, L, p, i, d);
                const float ax = d * p[i] - sn;
                q[i] = ax;
                pq += p[i] * ax;
            }
            pq = sum(pq);
            if (!(pq > 0.0f)) break;
            const float alpha = rz / pq;
            float rr = 0.0f, rz2 = 0.0f;
            for (int i = threadIdx.x; i < n; i += stride) {
                float d, dinv;
                sm_row(D, L, p, i, d, dinv);
                x[i] += alpha * p[i];
                const float ri = r[i] - alpha * q[i];
                r[i] = ri;
                rr += ri * ri;
                rz2 += ri * ri * dinv;
            }
            rr = sum(rr);
            rz2 = sum(rz2);
            if (rr <= kSmCoarseTol2 * bb) break;
            const float beta = rz2 / rz;
            rz = rz2;
            sync();
            for (int i = threadIdx.x; i < n; i += stride) {
                float d, dinv;
                sm_row(D, L, p, i, d, dinv);
                p[i] = r[i] * dinv + beta * p[i];
            }
            sync();
        }
    }
    if (singular) {
        float mx = 0.0f;
        for (int i = threadIdx.x; i < n; i += stride) mx += x[i];
        mx = sum(mx) / (float)n;
        for (int i = threadIdx.x; i < n; i += stride) x[i] -= mx;
    }
    __syncthreads();
}

// Coarsest level by its dense inverse C (at most kDirectN cells), applied in FP64:
// x = C (b - mean(b)) with the mean taken out when the mesh is periodic in both directions (C
// then inverts A + 1 1^T / n, which maps a zero-mean right-hand side to the zero-mean
// solution).  Warp w forms rows w, w + 32, ...; all threads of the block call it.
__device__ void sm_coarse_direct(const SmallDesc &D, const SmallLevel &L, float *x, const float *b, bool singular,
                                 float *red) {
    const int n = L.n, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    double mb = 0.0;
    if (singular) {
        // every lane of warp 0 sums the (at most 64) values in the same order
        __shared__ double mean_sh;
        if (threadIdx.x < 32) {
            double sb = 0.0;
            for (int i = 0; i < n; ++i) sb += (double)b[i];
            if (threadIdx.x == 0) mean_sh = sb / (double)n;
        }
        __syncthreads();
        mb = mean_sh;
    }
    for (int r = threadIdx.x >> 5; r < n; r += nwarp) {
        double acc = 0.0;
        for (int c = lane; c < n; c += 32) acc = fma(__ldg(D.cinv + r * n + c), (double)b[c] - mb, acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
        if (lane == 0) x[r] = (float)acc;
    }
    __syncthreads();
}

// V-cycle over the shared-memory levels; b of the first level must be in place, x of the
// first level holds the correction on return.
__device__ void sm_vcycle(const SmallDesc &D, float *sm, bool singular, float *red) {
    const int last = D.nlev - 1;
    for (int g = 0; g < last; ++g) {
        const SmallLevel &L = D.lv[g], &Cc = D.lv[g + 1];
        float *x = sm + L.off, *b = x + L.n;
        for (int k = 0; k < kNu; ++k) sm_smooth(D, L, x, b, k == 0);
        float *bc = sm + Cc.off + Cc.n;
        for (int p = threadIdx.x; p < Cc.n; p += blockDim.x) {
            float s = 0.0f;
            if (L.uniform && Cc.uniform) {
                const int py = mdiv(p, Cc.nx_magic), px = p - py * Cc.nx;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int i = (2 * py + (k >> 1)) * L.nx + 2 * px + (k & 1);
                    float d;
                    const float sn = sm_row(D, L, x, i, d);
                    s += b[i] - (d * x[i] - sn);
                }
            } else {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const int32_t i = Cc.child4[4 * p + k];
                    if (i < 0) continue;
                    float d;
                    const float sn = sm_row(D, L, x, i, d);
                    s += b[i] - (d * x[i] - sn);
                }
            }
            bc[p] = s;
        }
        __syncthreads();
    }
    {
        const SmallLevel &L = D.lv[last];
        float *x = sm + L.off, *b = x + L.n;
        float *r = sm + D.off_cg;
        if (D.cinv) sm_coarse_direct(D, L, x, b, singular, red);
        else sm_coarse_cg(D, L, x, b, r, r + L.n, r + 2 * L.n, singular, red);
    }
    for (int g = last - 1; g >= 0; --g) {
        const SmallLevel &L = D.lv[g], &Cc = D.lv[g + 1];
        float *x = sm + L.off, *b = x + L.n;
        const float *xc = sm + Cc.off;
        if (L.uniform && Cc.uniform) {
            for (int i = threadIdx.x; i < L.n; i += blockDim.x) {
                const int iy = mdiv(i, L.nx_magic), ix = i - iy * L.nx;
                x[i] += xc[(iy >> 1) * Cc.nx + (ix >> 1)];
            }
        } else {
            for (int i = threadIdx.x; i < L.n; i += blockDim.x) x[i] += xc[L.parent[i]];
        }
        __syncthreads();
        for (int k = 0; k < kNu; ++k) sm_smooth(D, L, x, b, false);
    }
}

// Tail of a V-cycle started by the multi-block levels: b from global, x back to global.
__global__ void __launch_bounds__(1024, 1) k_tail_vcycle(SmallDesc D, const float *__restrict__ gb,
                                                       float *__restrict__ gx, int singular) {
    pdl_chain();
    extern __shared__ float sm[];
    __shared__ float redf[33];
    const SmallLevel &L = D.lv[0];
    for (int i = threadIdx.x; i < L.n; i += blockDim.x) sm[L.off + L.n + i] = gb[i];
    __syncthreads();
    sm_vcycle(D, sm, singular != 0, redf);
    for (int i = threadIdx.x; i < L.n; i += blockDim.x) gx[i] = sm[L.off + i];
}


// FP64 sums over the cells of a small solve that come out the same whatever the number C of
// CTAs in the instance's cluster: chunk c (cells 1024 c .. 1024 c + 1023) is summed by CTA
// c mod C as a fixed tree (warp shuffles, then the 32 warp sums in order), and the chunk
// sums by the leader CTA in chunk order.  f(i, a, b) adds cell i's terms to a and b; every
// thread of the cluster receives both totals.  Collective over the cluster.
constexpr int kSmallChunks = kSmallN / 1024;
template <typename F>
__device__ void cl_sums(cooperative_groups::cluster_group &cl, int C, int rank, int n, double *wsum, double *lpart,
                        double *louts, F f, double &s0, double &s1) {
    const int nch = (n + 1023) >> 10;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int c = rank; c < nch; c += C) {
        const int i = (c << 10) + (int)threadIdx.x;
        double a = 0.0, b = 0.0;
        if (i < n) f(i, a, b);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            a += __shfl_down_sync(0xFFFFFFFFu, a, o);
            b += __shfl_down_sync(0xFFFFFFFFu, b, o);
        }
        if (lane == 0) { wsum[wid] = a; wsum[32 + wid] = b; }
        __syncthreads();
        if (threadIdx.x == 0) {
            double x = 0.0, y = 0.0;
            for (int w = 0; w < 32; ++w) { x += wsum[w]; y += wsum[32 + w]; }
            lpart[2 * c] = x;
            lpart[2 * c + 1] = y;
        }
        __syncthreads();
    }
    cl.sync();
    if (rank == 0 && threadIdx.x == 0) {
        double x = 0.0, y = 0.0;
        for (int c = 0; c < nch; ++c) { x += lpart[2 * c]; y += lpart[2 * c + 1]; }
        louts[0] = x;
        louts[1] = y;
    }
    cl.sync();
    s0 = louts[0];
    s1 = louts[1];
}

// Whole solve for a mesh whose every level fits: FP64 residual and correction, FP32 V-cycles
// in shared memory, convergence test on the device.  One cluster of C CTAs per item (C = 1
// for a batch of instances, one launch for all; up to 8 for an instance alone): the leader
// CTA holds the levels and runs the V-cycles, and the FP64 work (warm start, residual,
// correction, norms) is split by chunks of 1024 cells over the cluster, each CTA writing its
// chunks' FP32 residual straight into the leader's shared memory.  GB300's FP64 rate per SM
// is low, so spreading it over the cluster's SMs is what bounds the solve.  The result does
// not depend on C.  stats: [cycles, rel. residual, max rel. since reset].
struct SmallSolve {
    SmallDesc D;
    const double *diag64, *val64;
    double *phi, *phi_prev, *bvec, *stats;
    const uint8_t *lev;
    int32_t *n_solves;  // device counter: the warm start extrapolates once two solves exist
    int lmax, singular, maxc;
    double tol;
};

__global__ void __launch_bounds__(1024, 1) k_small_solve(const SmallSolve *__restrict__ items) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks(), rank = (int)cl.block_rank();
    extern __shared__ float sm[];
    __shared__ float redf[33];
    __shared__ SmallDesc D;
    __shared__ double wsum[64], part[2 * kSmallChunks], outs[2];
    const SmallSolve &it = items[blockIdx.x / C];
    if (threadIdx.x == 0) D = it.D;
    __syncthreads();
    float *lsm = cl.map_shared_rank(sm, 0);  // the leader's levels
    double *lpart = cl.map_shared_rank(part, 0), *louts = cl.map_shared_rank(outs, 0);
    const double *__restrict__ diag64 = it.diag64;
    const double *__restrict__ val64 = it.val64;
    double *phi = it.phi;
    double *bvec = it.bvec;
    const uint8_t *__restrict__ lev = it.lev;
    const int lmax = it.lmax, singular = it.singular, maxc = it.maxc;
    const double tol = it.tol;
    const SmallLevel &L = D.lv[0];
    const int n = L.n, nch = (n + 1023) >> 10;
#define CL_FOR(i)                                                                    \
    for (int c_ = rank; c_ < nch; c_ += C)                                           \
        for (int i = (c_ << 10) + (int)threadIdx.x; i < n && i < ((c_ + 1) << 10); i += 1 << 30)
    {
        const int ns = *it.n_solves;
        if (ns >= 1)
            CL_FOR(i) {
                const double p = phi[i];
                if (ns >= 2) phi[i] = 2.0 * p - it.phi_prev[i];
                it.phi_prev[i] = p;
            }
        cl.sync();  // every CTA has read the counter and its chunks of phi
        if (rank == 0 && threadIdx.x == 0) *it.n_solves = ns + 1;
    }
    if (singular) {  // right-hand side compatibility: remove an area-proportional share
        double sb, sa;
        cl_sums(cl, C, rank, n, wsum, lpart, louts, [&](int i, double &a, double &b) {
            const double s = (double)(1 << (lmax - lev[i]));
            a += bvec[i];
            b += s * s;
        }, sb, sa);
        CL_FOR(i) {
            const double s = (double)(1 << (lmax - lev[i]));
            bvec[i] -= sb / sa * s * s;
        }
        cl.sync();
    }
    double bb, unused;
    cl_sums(cl, C, rank, n, wsum, lpart, louts, [&](int i, double &a, double &) { a += bvec[i] * bvec[i]; }, bb,
            unused);
    float *b0 = lsm + L.off + n, *x0 = lsm + L.off;
    int cyc = 0;
    double rel = 0.0;
    for (;;) {
        double rr;
        cl_sums(cl, C, rank, n, wsum, lpart, louts, [&](int i, double &a, double &) {
            double ax;
            if (L.uniform) {
                double d;
                const double sn = uni_row<double>(L.nx, L.ny, L.nx_magic, D.bcx, D.bcy, phi, i, d);
                ax = d * phi[i] - sn;
            } else {
                ax = diag64[i] * phi[i];
#pragma unroll
                for (int j = 0; j < kEll; ++j) {
                    const int32_t c = L.col[(int64_t)j * n + i];
                    if (c >= 0) ax += val64[(int64_t)j * n + i] * phi[c];
                }
            }
            const double ri = bvec[i] - ax;
            b0[i] = (float)ri;
            a += ri * ri;
        }, rr, unused);
        rel = bb > 0.0 ? sqrt(rr / bb) : sqrt(rr);
        if (rel <= tol || (bb == 0.0 && rr == 0.0) || cyc >= maxc) break;
        if (rank == 0) sm_vcycle(D, sm, singular != 0, redf);
        cl.sync();  // the correction is in the leader's x0
        CL_FOR(i) phi[i] += (double)x0[i];
        cl.sync();  // phi complete before the next residual (and x0 read before the next V-cycle)
        if (singular) {
            double sv, sa;
            cl_sums(cl, C, rank, n, wsum, lpart, louts, [&](int i, double &a, double &b) {
                const double s = (double)(1 << (lmax - lev[i]));
                a += s * s * phi[i];
                b += s * s;
            }, sv, sa);
            CL_FOR(i) phi[i] -= sv / sa;
            cl.sync();
        }
        ++cyc;
    }
#undef CL_FOR
    if (rank == 0 && threadIdx.x == 0) {
        it.stats[0] = (double)cyc;
        it.stats[1] = rel;
        it.stats[2] = worst_residual(it.stats[2], rel);
    }
}

// One launch of the small solve: n_items clusters of C CTAs.
void launch_small_solve(const void *items, int n_items, int C, size_t smem, cudaStream_t st) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(n_items * C));
    cfg.blockDim = dim3(1024);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    GB_CUDA(cudaLaunchKernelEx(&cfg, k_small_solve, (const SmallSolve *)items));
}

// The cluster size for an instance solved alone: one CTA per 1024-cell chunk, at most 8,
// reduced until the GPU can hold such a cluster.
int small_cluster(int n, size_t smem) {
    int C = std::min(8, std::max(1, (n + 1023) / 1024));
    for (; C > 1; C >>= 1) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)C);
        cfg.blockDim = dim3(1024);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int nc = 0;
        if (cudaOccupancyMaxActiveClusters(&nc, k_small_solve, &cfg) == cudaSuccess && nc >= 1) break;
        cudaGetLastError();
    }
    return C;
}

// Which suffix of the level list fits one block's shared memory.
int small_from(const Instance &in) {
    int g0 = (int)in.lv.size();
    int64_t floats = 0;
    for (int g = (int)in.lv.size() - 1; g >= 0; --g) {
        const Level &L = in.lv[g];
        const int64_t add = 2 * L.n + (g == (int)in.lv.size() - 1 ? 3 * L.n + 8 : 0);
        if (L.n > kSmallN || (int)in.lv.size() - g > kMaxSmallLevels || (floats + add) * 4 > kSmallSmemCap) break;
        floats += add;
        g0 = g;
    }
    return g0;
}

SmallDesc small_desc(const Instance &in, int g0) {
    SmallDesc D{};
    D.nlev = (int)in.lv.size() - g0;
    D.bcx = in.cfg.bc_x;
    D.bcy = in.cfg.bc_y;
    int32_t off = 0;
    for (int k = 0; k < D.nlev; ++k) {
        const Level &L = in.lv[g0 + k];
        SmallLevel &S = D.lv[k];
        S.n = (int32_t)L.n; S.col = L.col; S.val = L.val; S.dinv = L.dinv; S.color = L.color;
        S.child4 = L.child4; S.parent = L.parent; S.off = off;
        // (the implicit scheme's levels carry kappa in their ELL rows: no matrix-free stencil)
        S.uniform = L.lmax == 0 && !in.cfg.implicit ? 1 : 0;
        S.nx = L.nx0;
        S.ny = L.ny0;
        // multiply-high reciprocal: floor(i * m / 2^32) == floor(i / nx) for the i < n used here
        S.nx_magic = mdiv_magic((uint32_t)L.nx0);
        const uint32_t nxh = std::max(1, L.nx0 / 2);
        S.nxh_magic = mdiv_magic(nxh);
        auto q = [](int64_t i, uint32_t m) { return m ? (int64_t)(((uint64_t)i * m) >> 32) : i; };
        for (int64_t i = 0; i < L.n; ++i)
            if (q(i, S.nx_magic) != i / L.nx0 || q(i, S.nxh_magic) != i / (int64_t)nxh)
                fail(PIC_EINVAL, "index division check failed");
        off += 2 * (int32_t)L.n;
    }
    D.off_cg = off;
    off += 3 * (int32_t)in.lv.back().n + 8;
    D.smem_floats = off;
    D.cinv = in.coarse_inv;
    return D;
}

void vcycle(pic_ctx *ctx, Instance &in, size_t g, bool singular) {
    Level &L = in.lv[g];
    cudaStream_t s = ctx->stream;
    const int g0 = small_from(in);
    if ((int)g >= g0) {
        const SmallDesc D = small_desc(in, (int)g);
        const size_t bytes = (size_t)D.smem_floats * 4;
        pdl(k_tail_vcycle, 1, 1024, bytes, s, D, L.b, L.x, singular);
        count_launch(ctx);
        return;
    }
    if (g + 1 == in.lv.size()) {
        const int maxit = (int)std::min<int64_t>(2 * L.n + 10, 500);
        // r, p, q: three slices of the coarsest level's work buffer (allocated 3n)
        pdl(k_coarse_cg, 1, 1024, 0, s, L.n, L.col, L.val, L.dinv, L.b, L.x, L.t, L.t + L.n, L.t + 2 * L.n,
                                       singular, maxit);
        count_launch(ctx);
        return;
    }
    Level &C = in.lv[g + 1];
    const unsigned nb = blocks_for(L.n);
    // pre-smoothing (x starts at zero): the first sweep's two half sweeps in one kernel
    pdl(k_rbgs_first, nb, kT, 0, s, L.n, L.col, L.val, L.dinv, L.color, L.b, L.x);
    for (int k = 1; k < kNu; ++k)
        for (int c = 0; c < 2; ++c) {
            pdl(k_rbgs_half, nb, kT, 0, s, L.n, L.col, L.val, L.dinv, L.color, c, L.b, L.x, L.t, 0);
            std::swap(L.x, L.t);
        }
    pdl(k_restrict_residual, blocks_for(C.n), kT, 0, s, C.n, C.child4, L.n, L.col, L.val, L.dinv, L.b, L.x, C.b, C.x);
    count_launch(ctx, 2 * kNu);
    vcycle(ctx, in, g + 1, singular);
    // post-smoothing, the injection of the correction fused into its first half sweep
    pdl(k_rbgs_half_prolong, nb, kT, 0, s, L.n, L.col, L.val, L.dinv, L.color, 0, L.b, L.x, L.parent, C.x, L.t);
    std::swap(L.x, L.t);
    pdl(k_rbgs_half, nb, kT, 0, s, L.n, L.col, L.val, L.dinv, L.color, 1, L.b, L.x, L.t, 0);
    std::swap(L.x, L.t);
    for (int k = 1; k < kNu; ++k)
        for (int c = 0; c < 2; ++c) {
            pdl(k_rbgs_half, nb, kT, 0, s, L.n, L.col, L.val, L.dinv, L.color, c, L.b, L.x, L.t, 0);
            std::swap(L.x, L.t);
        }
    count_launch(ctx, 2 * kNu);
}
}  // namespace

namespace {
constexpr int kDirectN = 64;  // coarsest levels up to this size are solved by a dense inverse

// Dense inverse of the coarsest level's operator as the shared-memory V-cycle applies it
// (uniform levels: the 5-point stencil with the wall rules; otherwise the ELL rows with the
// diagonal 1 / dinv rounded to FP32), plus 1 1^T / n when the mesh is periodic in both
// directions.  Gauss-Jordan with partial pivoting in FP64; null (the CG is used) for a
// level larger than kDirectN cells or a singular matrix.
double *coarse_inverse(pic_ctx *ctx, Instance &in, bool singular) {
    const Level &L = in.lv.back();
    const int n = (int)L.n;
    if (n > kDirectN || n < 1) return nullptr;
    std::vector<double> A((size_t)n * n, 0.0);
    auto at = [&](int i, int j) -> double & { return A[(size_t)i * n + j]; };
    if (L.lmax == 0) {
        const int nx = L.nx0, ny = L.ny0, bx = in.cfg.bc_x, by = in.cfg.bc_y;
        for (int i = 0; i < n; ++i) {
            const int ix = i % nx, iy = i / nx;
            auto face = [&](bool inside, int j, int bc) {
                if (inside || bc == PIC_BC_PERIODIC) { at(i, j) -= 1.0; at(i, i) += 1.0; }
                else if (bc == PIC_BC_DIRICHLET) at(i, i) += 2.0;
            };
            face(ix > 0, ix > 0 ? i - 1 : i + nx - 1, bx);
            face(ix < nx - 1, ix < nx - 1 ? i + 1 : i - nx + 1, bx);
            face(iy > 0, iy > 0 ? i - nx : i + (ny - 1) * nx, by);
            face(iy < ny - 1, iy < ny - 1 ? i + nx : i - (ny - 1) * nx, by);
        }
    } else {
        std::vector<int32_t> col((size_t)kEll * n);
        std::vector<float> val((size_t)kEll * n), dinv(n);
        GB_CUDA(cudaMemcpyAsync(col.data(), L.col, col.size() * 4, cudaMemcpyDeviceToHost, ctx->stream));
        GB_CUDA(cudaMemcpyAsync(val.data(), L.val, val.size() * 4, cudaMemcpyDeviceToHost, ctx->stream));
        GB_CUDA(cudaMemcpyAsync(dinv.data(), L.dinv, dinv.size() * 4, cudaMemcpyDeviceToHost, ctx->stream));
        GB_CUDA(cudaStreamSynchronize(ctx->stream));
        for (int i = 0; i < n; ++i) {
            at(i, i) += (double)(1.0f / dinv[i]);
            for (int j = 0; j < kEll; ++j) {
                const int32_t c = col[(size_t)j * n + i];
                if (c >= 0) at(i, c) += (double)val[(size_t)j * n + i];
            }
        }
    }
    if (singular)
        for (double &a : A) a += 1.0 / n;
    // Gauss-Jordan on [A | I]
    std::vector<double> Inv((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) Inv[(size_t)i * n + i] = 1.0;
    double amax = 0.0;
    for (double a : A) amax = std::max(amax, std::fabs(a));
    for (int k = 0; k < n; ++k) {
        int piv = k;
        for (int i = k + 1; i < n; ++i)
            if (std::fabs(at(i, k)) > std::fabs(at(piv, k))) piv = i;
        if (!(std::fabs(at(piv, k)) > 1e-12 * amax)) return nullptr;
        if (piv != k)
            for (int j = 0; j < n; ++j) {
                std::swap(at(k, j), at(piv, j));
                std::swap(Inv[(size_t)k * n + j], Inv[(size_t)piv * n + j]);
            }
        const double p = 1.0 / at(k, k);
        for (int j = 0; j < n; ++j) { at(k, j) *= p; Inv[(size_t)k * n + j] *= p; }
        for (int i = 0; i < n; ++i) {
            if (i == k) continue;
            const double f = at(i, k);
            if (f == 0.0) continue;
            for (int j = 0; j < n; ++j) {
                at(i, j) -= f * at(k, j);
                Inv[(size_t)i * n + j] -= f * Inv[(size_t)k * n + j];
            }
        }
    }
    double *d = dalloc<double>(in.mesh_mem, Inv.size());
    GB_CUDA(cudaMemcpyAsync(d, Inv.data(), Inv.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
    GB_CUDA(cudaStreamSynchronize(ctx->stream));
    return d;
}
}  // namespace

void poisson_setup(pic_ctx *ctx, Instance &in) {
    if (in.mg_cycle) {
        cudaGraphExecDestroy(in.mg_cycle);
        in.mg_cycle = nullptr;
    }
    GB_CUDA(cudaFuncSetAttribute(k_tail_vcycle, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmallSmemCap));
    GB_CUDA(cudaFuncSetAttribute(k_small_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmallSmemCap));
    DeviceArena &A = in.mesh_mem;
    const int64_t n = in.lv[0].n;
    in.phi = dalloc<double>(A, n);
    in.phi_prev = dalloc<double>(A, n);
    in.n_solves = 0;
    in.d_n_solves = nullptr;
    in.bvec = dalloc<double>(A, n);
    in.res = dalloc<double>(A, n);
    in.charge = dalloc<double>(A, n);
    in.red = dalloc<double>(A, 2 * kRedBlocks + 8);  // block sums, totals, the residual's ticket
    GB_CUDA(cudaMemsetAsync(in.red, 0, (2 * kRedBlocks + 8) * sizeof(double), ctx->stream));
    in.mg_stats = dalloc<double>(A, 4);
    GB_CUDA(cudaMemsetAsync(in.mg_stats, 0, 4 * 8, ctx->stream));
    GB_CUDA(cudaMemsetAsync(in.phi, 0, n * 8, ctx->stream));
    GB_CUDA(cudaMemsetAsync(in.bvec, 0, n * 8, ctx->stream));
    GB_CUDA(cudaMemsetAsync(in.charge, 0, n * 8, ctx->stream));
    // coarsest-level CG needs three extra vectors: give it its own buffers
    Level &c = in.lv.back();
    c.t = dalloc<float>(A, 3 * c.n + 16);
    // (the implicit scheme's coarsest operator changes every step: the CG solves it)
    in.coarse_inv = in.cfg.implicit ? nullptr
                                    : coarse_inverse(ctx, in, in.cfg.bc_x == PIC_BC_PERIODIC && in.cfg.bc_y == PIC_BC_PERIODIC);
    // meshes whose every level fits one block: the whole solve is one block's work item
    in.small_item = nullptr;
    if (small_from(in) == 0) {
        SmallSolve it{};
        it.D = small_desc(in, 0);
        Level &L = in.lv[0];
        it.diag64 = L.diag64; it.val64 = L.val64;
        it.phi = in.phi; it.phi_prev = in.phi_prev; it.bvec = in.bvec; it.stats = in.mg_stats;
        it.lev = L.lev; it.lmax = L.lmax;
        it.singular = (in.cfg.bc_x == PIC_BC_PERIODIC && in.cfg.bc_y == PIC_BC_PERIODIC) ? 1 : 0;
        it.maxc = std::max(1, in.cfg.mg_max_cycles);
        it.tol = in.cfg.mg_rel_tol;
        int32_t *ns = dalloc<int32_t>(A, 1);
        GB_CUDA(cudaMemsetAsync(ns, 0, 4, ctx->stream));
        it.n_solves = ns;
        in.d_n_solves = ns;
        SmallSolve *d = (SmallSolve *)A.alloc(sizeof(SmallSolve));
        GB_CUDA(cudaMemcpyAsync(d, &it, sizeof(SmallSolve), cudaMemcpyHostToDevice, ctx->stream));
        GB_CUDA(cudaStreamSynchronize(ctx->stream));
        in.small_item = d;
        in.small_smem = (size_t)it.D.smem_floats * 4;
        in.small_cluster = small_cluster((int)L.n, in.small_smem);
    }
    ++ctx->mesh_epoch;
}

// After a solve that ended with a non-finite residual: the next solve starts from zero instead
// of extrapolating from a potential that holds NaN or Inf.
void poisson_reset_warm_start(pic_ctx *ctx, Instance &in) {
    const int64_t n = in.lv[0].n;
    GB_CUDA(cudaMemsetAsync(in.phi, 0, n * 8, ctx->stream));
    GB_CUDA(cudaMemsetAsync(in.phi_prev, 0, n * 8, ctx->stream));
    in.n_solves = 0;
    if (in.d_n_solves) GB_CUDA(cudaMemsetAsync(in.d_n_solves, 0, 4, ctx->stream));
}

// One launch for every instance whose mesh fits one block: block b solves instance b.
// The batched solver's item table for `list` (copies issued on the context's stream, so a
// step captured afterwards finds the table current and captures no copy).
void poisson_batch_items(pic_ctx *ctx, const std::vector<Instance *> &list) {
    if (ctx->batch_epoch != ctx->mesh_epoch || ctx->batch_n != (int)list.size()) {
        ctx->batch_mem.release_all();
        ctx->batch_items = ctx->batch_mem.alloc(list.size() * sizeof(SmallSolve));
        ctx->batch_smem = 0;
        // largest meshes first: the blocks start in this order, one per SM (each reserves the
        // largest instance's shared memory), so the longest solves begin in the first wave
        // and the short ones fill in behind them (every item writes only its own instance)
        std::vector<size_t> order(list.size());
        for (size_t k = 0; k < order.size(); ++k) order[k] = k;
        std::stable_sort(order.begin(), order.end(),
                         [&](size_t a, size_t b) { return list[a]->lv[0].n > list[b]->lv[0].n; });
        for (size_t k = 0; k < list.size(); ++k) {
            GB_CUDA(cudaMemcpyAsync((SmallSolve *)ctx->batch_items + k, list[order[k]]->small_item, sizeof(SmallSolve),
                                    cudaMemcpyDeviceToDevice, ctx->stream));
            ctx->batch_smem = std::max(ctx->batch_smem, list[order[k]]->small_smem);
        }
        ctx->batch_epoch = ctx->mesh_epoch;
        ctx->batch_n = (int)list.size();
    }
}

void poisson_solve_batch(pic_ctx *ctx, const std::vector<Instance *> &list, const std::vector<const double *> &walls) {
    if (list.empty()) return;
    poisson_batch_items(ctx, list);
    for (size_t k = 0; k < list.size(); ++k) {
        for (int w = 0; w < 4; ++w) list[k]->last_walls[w] = walls[k][w];
        list[k]->mg_on_device = true;
    }
    launch_small_solve(ctx->batch_items, (int)list.size(), 1, ctx->batch_smem, ctx->stream);
    count_launch(ctx);
    check_launch("poisson_solve_batch");
}

// Solve A phi = bvec to ||r|| <= mg_rel_tol ||b||, warm-started from the current phi.
void poisson_solve(pic_ctx *ctx, Instance &in, const double walls[4]) {
    for (int k = 0; k < 4; ++k) in.last_walls[k] = walls[k];
    Level &L = in.lv[0];
    cudaStream_t s = ctx->stream;
    const int64_t n = L.n;
    const bool singular = in.cfg.bc_x == PIC_BC_PERIODIC && in.cfg.bc_y == PIC_BC_PERIODIC;
    if (in.small_item) {
        launch_small_solve(in.small_item, 1, in.small_cluster, (size_t)in.small_smem, s);
        count_launch(ctx);
        check_launch("poisson_solve");
        in.mg_on_device = true;
        return;
    }
    if (in.n_solves >= 1) {
        k_extrapolate<<<blocks_for(n), kT, 0, s>>>(n, in.phi, in.phi_prev, in.n_solves >= 2 ? 1 : 0);
        count_launch(ctx);
    }
    ++in.n_solves;
    in.mg_on_device = false;
    if (singular) {
        k_area_moments<<<kRedBlocks, kT, 0, s>>>(n, L.lev, L.lmax, in.bvec, in.red);
        k_finish_sums<<<1, 32, 0, s>>>(kRedBlocks, in.red, in.red + 2 * kRedBlocks);
        k_project<<<blocks_for(n), kT, 0, s>>>(n, L.lev, L.lmax, in.red + 2 * kRedBlocks, in.bvec, 0);
        count_launch(ctx, 3);
    }
    const int maxc = std::max(1, in.cfg.mg_max_cycles);
    // launches go to ctx->stream, which is the capture stream while the solve is captured
    auto issue_residual = [&](int first, cudaGraphConditionalHandle h) {
        pdl(k_residual_decide, kRedBlocks, kT, 0, ctx->stream, n, L.col, L.val64, L.diag64, in.phi, in.bvec, in.res, L.b,
                                                              in.red, (uint32_t *)(in.red + 2 * kRedBlocks + 4), h,
                                                              in.cfg.mg_rel_tol, maxc, in.mg_stats, first);
        count_launch(ctx);
    };
    auto issue_cycle = [&](cudaGraphConditionalHandle h) {
        vcycle(ctx, in, 0, singular);
        pdl(k_add_correction, blocks_for(n), kT, 0, ctx->stream, n, L.x, in.phi);
        count_launch(ctx);
        if (singular) {
            pdl(k_area_weighted, kRedBlocks, kT, 0, ctx->stream, n, L.lev, L.lmax, in.phi, in.red);
            pdl(k_finish_sums, 1, 32, 0, ctx->stream, kRedBlocks, in.red, in.red + 2 * kRedBlocks);
            pdl(k_project, blocks_for(n), kT, 0, ctx->stream, n, L.lev, L.lmax, in.red + 2 * kRedBlocks, in.phi, 1);
            count_launch(ctx, 3);
        }
        issue_residual(0, h);
    };
    if (!in.mg_cycle) {
        // The whole solve as one graph: the residual of the warm start, then a WHILE node
        // whose body is one cycle (V-cycle, correction, FP64 residual); the residual's last
        // kernel decides on the device whether the body runs again, so the host never waits.
        // Captured on a private stream (the context's stream may be the legacy default
        // stream, which cannot be captured) and replayed on the context's stream.
        cudaStream_t cs;
        GB_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        cudaStream_t saved = ctx->stream;
        const int64_t l0 = ctx->launches;
        ctx->stream = cs;
        cudaGraph_t graph = nullptr;
        cudaGraphConditionalHandle h = 0;
        cudaError_t e = cudaGraphCreate(&graph, 0);
        if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, graph, 0, cudaGraphCondAssignDefault);
        if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(cs, graph, nullptr, nullptr, 0,
                                                                cudaStreamCaptureModeThreadLocal);
        cudaGraphNodeParams np = {};
        if (e == cudaSuccess) {
            issue_residual(1, h);
            cudaStreamCaptureStatus status;
            const cudaGraphNode_t *deps = nullptr;
            size_t nd = 0;
            e = cudaStreamGetCaptureInfo(cs, &status, nullptr, nullptr, &deps, nullptr, &nd);
            cudaGraphNode_t wn = nullptr;
            np.type = cudaGraphNodeTypeConditional;
            np.conditional.handle = h;
            np.conditional.type = cudaGraphCondTypeWhile;
            np.conditional.size = 1;
            if (e == cudaSuccess) e = cudaGraphAddNode(&wn, graph, deps, nullptr, nd, &np);
            if (e == cudaSuccess) e = cudaStreamUpdateCaptureDependencies(cs, &wn, nullptr, 1,
                                                                          cudaStreamSetCaptureDependencies);
            cudaGraph_t g2 = nullptr;
            const cudaError_t e2 = cudaStreamEndCapture(cs, &g2);
            if (e == cudaSuccess) e = e2;
        }
        in.mg_pre_nodes = ctx->launches - l0;
        if (e == cudaSuccess) {
            cudaGraph_t body = np.conditional.phGraph_out[0];
            e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                issue_cycle(h);
                cudaGraph_t b2 = nullptr;
                e = cudaStreamEndCapture(cs, &b2);
            }
        }
        ctx->stream = saved;
        in.mg_cycle_nodes = ctx->launches - l0 - in.mg_pre_nodes;
        ctx->launches = l0;
        cudaStreamDestroy(cs);
        if (e == cudaSuccess) e = cudaGraphInstantiate(&in.mg_cycle, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        GB_CUDA(e);
    }
    GB_CUDA(cudaGraphLaunch(in.mg_cycle, s));
    count_launch(ctx, in.mg_pre_nodes);  // the cycles' launches are counted when the stats are read
    in.mg_on_device = true;
    in.mg_count_cycles = true;
    check_launch("poisson_solve");
}

}  // namespace gbpic
