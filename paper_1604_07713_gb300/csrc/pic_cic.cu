// Cloud-in-cell shapes on a uniform mesh (§3: the momentum-conserving CIC-EM and the
// energy-conserving CIC-EC variants, on uniform meshes).
//
// Cells (i, j) of side h with centres at ((i + 1/2) h, (j + 1/2) h); on a uniform mesh the
// leaf index is i + j nx (root order).  A particle at offset (u, v) of its cell has the
// reference centre i0 = i - 1 + qx with qx = (u >= 1/2) and the fraction fx = u + 1/2 - qx
// (likewise in y): bilinear weights (1 - fx, fx) x (1 - fy, fy) on the centres i0, i0 + 1 and
// j0, j0 + 1.  A centre beyond a non-periodic wall is replaced by the boundary cell (its
// weight folds into it); periodic directions wrap.
//
// Deposit: one warp per leaf sums its particles' charge into the 3 x 3 block of cells around
// it (FP64 per lane, lanes combined by a fixed shuffle tree), then one thread per cell adds
// the contributions of its 9 neighbours in a fixed order: no atomics, the same bits every run.
//
// Field: for each leaf and each quarter (qx, qy) of it, the field over that quarter is a
// bilinear form in (fx, fy), e0 + fx e_x + fy (e_y + fx e_xy) per component, whose 4 x 2 x 4
// coefficients the push gathers by shuffles (lane k of the warp holds coefficient k):
//   CIC-EM: E at the four centres by central differences of phi (the Poisson operator's ghost
//           values beyond walls: Dirichlet 2 phi_wall - phi, Neumann phi), the centres
//           clamped at walls as in the deposit -- the deposit's weights gather it, so the
//           total force on the particles of a periodic box vanishes;
//   CIC-EC: E = -grad of the bilinear interpolant of phi over the four centres (ghost values
//           beyond walls) -- the gradient of the deposit's own weights.
#include <algorithm>

#include "pic_internal.cuh"

namespace gbpic {

namespace {
constexpr int kT = 256;
inline unsigned blocks_for(int64_t n) { return (unsigned)std::max<int64_t>(1, (n + kT - 1) / kT); }
inline unsigned warp_blocks(int64_t nw) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((nw + kT / 32 - 1) / (kT / 32), 1 << 20));
}

__host__ __device__ __forceinline__ int cic_cell(int i, int n, bool periodic) {
    if (periodic) return ((i % n) + n) % n;
    return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

struct CicGrid {
    int nx, ny, bcx, bcy;
    double h;
    double wall[4];
    const double *wall_dev;  // non-null: the wall potentials are read from here (captured steps)
};

// phi at lattice (i, j), with the ghost rule beyond walls (see the file comment)
__device__ __forceinline__ double phi_at(const CicGrid &g, const double *__restrict__ phi, const double *wall, int i,
                                         int j) {
    double add = 0.0, sgn = 1.0;
    if (i < 0 || i >= g.nx) {
        if (g.bcx == PIC_BC_PERIODIC) {
            i = ((i % g.nx) + g.nx) % g.nx;
        } else {
            const int in = i < 0 ? 0 : g.nx - 1;
            if (g.bcx == PIC_BC_DIRICHLET) { add = 2.0 * wall[i < 0 ? 0 : 1]; sgn = -1.0; }
            i = in;
        }
    }
    if (j < 0 || j >= g.ny) {
        if (g.bcy == PIC_BC_PERIODIC) {
            j = ((j % g.ny) + g.ny) % g.ny;
        } else {
            const int in = j < 0 ? 0 : g.ny - 1;
            if (g.bcy == PIC_BC_DIRICHLET) { add += 2.0 * wall[j < 0 ? 2 : 3] * sgn; sgn = -sgn; }
            j = in;
        }
    }
    return add + sgn * phi[i + (int64_t)g.nx * j];
}

// 32 coefficients per leaf: [quarter q = qx + 2 qy][component][e0, e_x, e_y, e_xy]
template <typename R>
__global__ void k_cic_patch(int64_t nl, CicGrid g, int shape, const double *__restrict__ phi, R *__restrict__ patch) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 4 * nl) return;
    double wall[4];
    for (int k = 0; k < 4; ++k) wall[k] = g.wall_dev ? g.wall_dev[k] : g.wall[k];
    const int64_t L = t >> 2;
    const int q = (int)(t & 3), qx = q & 1, qy = q >> 1;
    const int i = (int)(L % g.nx), j = (int)(L / g.nx);
    const int i0 = i - 1 + qx, j0 = j - 1 + qy;
    double ex[4], ey[4];  // corners 00, 10, 01, 11 of the quarter's bilinear form
    if (shape == PIC_SHAPE_CIC_EM) {
        const bool px = g.bcx == PIC_BC_PERIODIC, py = g.bcy == PIC_BC_PERIODIC;
        for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) {
                const int ci = cic_cell(i0 + a, g.nx, px), cj = cic_cell(j0 + b, g.ny, py);
                ex[a + 2 * b] = -(phi_at(g, phi, wall, ci + 1, cj) - phi_at(g, phi, wall, ci - 1, cj)) / (2.0 * g.h);
                ey[a + 2 * b] = -(phi_at(g, phi, wall, ci, cj + 1) - phi_at(g, phi, wall, ci, cj - 1)) / (2.0 * g.h);
            }
    } else {
        const double p00 = phi_at(g, phi, wall, i0, j0), p10 = phi_at(g, phi, wall, i0 + 1, j0);
        const double p01 = phi_at(g, phi, wall, i0, j0 + 1), p11 = phi_at(g, phi, wall, i0 + 1, j0 + 1);
        // E_x = -[(1 - fy)(p10 - p00) + fy (p11 - p01)] / h, E_y = -[(1 - fx)(p01 - p00) + fx (p11 - p10)] / h
        ex[0] = ex[1] = -(p10 - p00) / g.h;
        ex[2] = ex[3] = -(p11 - p01) / g.h;
        ey[0] = ey[2] = -(p01 - p00) / g.h;
        ey[1] = ey[3] = -(p11 - p10) / g.h;
    }
    R *o = patch + 32 * L + 8 * q;
    const double *e2[2] = {ex, ey};
    for (int c = 0; c < 2; ++c) {
        const double *e = e2[c];
        o[4 * c + 0] = (R)e[0];
        o[4 * c + 1] = (R)(e[1] - e[0]);
        o[4 * c + 2] = (R)(e[2] - e[0]);
        o[4 * c + 3] = (R)((e[0] - e[1]) - (e[2] - e[3]));
    }
}

// Per leaf: the charge its particles put on the 3 x 3 cells around it, part[9 L + (a + 1) + 3 (b + 1)].
struct CicDepositArgs {
    int64_t nl;
    int nsp;
    const int32_t *start[2], *end[2];
    const void *u[2], *v[2], *w[2];
    double q[2];
    double *part;
};

template <typename R>
__global__ void __launch_bounds__(kT) k_cic_deposit(CicDepositArgs a) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t L = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; L < a.nl; L += nw) {
        double acc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        for (int s = 0; s < a.nsp; ++s) {
            const R *U = (const R *)a.u[s], *V = (const R *)a.v[s], *Wt = (const R *)a.w[s];
            for (int32_t p = a.start[s][L] + lane; p < a.end[s][L]; p += 32) {
                const double u = (double)U[p], v = (double)V[p], qw = a.q[s] * (double)Wt[p];
                const int qx = u >= 0.5 ? 1 : 0, qy = v >= 0.5 ? 1 : 0;
                const double fx = u + 0.5 - qx, fy = v + 0.5 - qy;
                // centres i - 1 + qx + a', j - 1 + qy + b' -> slots (qx + a', qy + b') of the 3 x 3 block
#pragma unroll
                for (int bb = 0; bb < 2; ++bb)
#pragma unroll
                    for (int aa = 0; aa < 2; ++aa) {
                        const double wt = (aa ? fx : 1.0 - fx) * (bb ? fy : 1.0 - fy);
                        const int slot = (qx + aa) + 3 * (qy + bb);
#pragma unroll
                        for (int k = 0; k < 9; ++k)
                            if (k == slot) acc[k] += qw * wt;
                    }
            }
        }
#pragma unroll
        for (int k = 0; k < 9; ++k) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_xor_sync(0xFFFFFFFFu, acc[k], o);
        }
        if (lane < 9) {
            double v = 0.0;
#pragma unroll
            for (int k = 0; k < 9; ++k)
                if (k == lane) v = acc[k];
            a.part[9 * L + lane] = v;
        }
    }
}

// Per cell: the contributions of the 3 x 3 leaves around it whose (clamped or wrapped) target
// is this cell, in a fixed order; then b as the NGP deposit forms it.
__global__ void k_cic_charge(int64_t nl, CicGrid g, const double *__restrict__ part, double rho_bg, double inv_eps0,
                             const double *__restrict__ bcw, double *__restrict__ charge, double *__restrict__ b) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= nl) return;
    const int i = (int)(c % g.nx), j = (int)(c / g.nx);
    const bool px = g.bcx == PIC_BC_PERIODIC, py = g.bcy == PIC_BC_PERIODIC;
    double total = 0.0;
    int64_t seen[9];  // a leaf reached twice (a periodic direction of fewer than 3 cells) counts once
    int ns = 0;
    for (int sj = -1; sj <= 1; ++sj)
        for (int si = -1; si <= 1; ++si) {
            // the source leaf (i + si, j + sj): skip it beyond a wall, wrap it if periodic
            int li = i + si, lj = j + sj;
            if (li < 0 || li >= g.nx) { if (!px) continue; li = ((li % g.nx) + g.nx) % g.nx; }
            if (lj < 0 || lj >= g.ny) { if (!py) continue; lj = ((lj % g.ny) + g.ny) % g.ny; }
            const int64_t L = (int64_t)li + (int64_t)g.nx * lj;
            bool dup = false;
            for (int k = 0; k < ns; ++k) dup = dup || seen[k] == L;
            if (dup) continue;
            seen[ns++] = L;
            const double *src = part + 9 * L;
            for (int k = 0; k < 9; ++k) {
                const int di = k % 3 - 1, dj = k / 3 - 1;
                if (cic_cell(li + di, g.nx, px) == i && cic_cell(lj + dj, g.ny, py) == j) total += src[k];
            }
        }
    charge[c] = total;
    double bl = (total + rho_bg * g.h * g.h) * inv_eps0;
    for (int k = 0; k < 4; ++k) bl += bcw[4 * c + k] * (g.wall_dev ? g.wall_dev[k] : g.wall[k]);
    b[c] = bl;
}

CicGrid grid_of(pic_ctx *ctx, Instance &in, const double walls[4]) {
    CicGrid g{};
    g.nx = in.nx0;
    g.ny = in.ny0;
    g.bcx = in.cfg.bc_x;
    g.bcy = in.cfg.bc_y;
    g.h = in.h0;
    for (int k = 0; k < 4; ++k) g.wall[k] = walls[k];
    g.wall_dev = ctx->capturing ? in.d_walls : nullptr;
    return g;
}
}  // namespace

void cic_patch(pic_ctx *ctx, Instance &in, const double walls[4]) {
    const CicGrid g = grid_of(ctx, in, walls);
    const int64_t nl = in.nleaf;
    if (in.cfg.precision == PIC_FP64)
        k_cic_patch<double><<<blocks_for(4 * nl), kT, 0, ctx->stream>>>(nl, g, in.cfg.shape, in.phi, (double *)in.patch);
    else
        k_cic_patch<float><<<blocks_for(4 * nl), kT, 0, ctx->stream>>>(nl, g, in.cfg.shape, in.phi, (float *)in.patch);
    count_launch(ctx);
    check_launch("cic_patch");
}

void cic_deposit(pic_ctx *ctx, Instance &in, const double walls[4]) {
    const CicGrid g = grid_of(ctx, in, walls);
    const int64_t nl = in.nleaf;
    CicDepositArgs a{};
    a.nl = nl;
    for (int s = 0; s < in.cfg.n_species; ++s) {
        Species &sp = in.sp[s];
        if (!sp.start) continue;
        a.start[a.nsp] = sp.start;
        a.end[a.nsp] = sp.end;
        a.u[a.nsp] = sp.arr[sp.cur][0];
        a.v[a.nsp] = sp.arr[sp.cur][1];
        a.w[a.nsp] = sp.arr[sp.cur][5];
        a.q[a.nsp] = in.cfg.q[s];
        ++a.nsp;
    }
    a.part = in.cic_part;
    if (in.cfg.precision == PIC_FP64)
        k_cic_deposit<double><<<warp_blocks(nl), kT, 0, ctx->stream>>>(a);
    else
        k_cic_deposit<float><<<warp_blocks(nl), kT, 0, ctx->stream>>>(a);
    k_cic_charge<<<blocks_for(nl), kT, 0, ctx->stream>>>(nl, g, in.cic_part, in.cfg.rho_background, 1.0 / in.cfg.eps0,
                                                         in.lv[0].bcw, in.charge, in.bvec);
    count_launch(ctx, 2);
    check_launch("cic_deposit");
}

}  // namespace gbpic
