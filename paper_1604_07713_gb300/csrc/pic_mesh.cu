// Leaf mesh (§2.1 Morton-ordered forest of root boxes, §3.1 quad-tree) built on the device,
// the multigrid level hierarchy derived from it, the composite-mesh Poisson operator (§3)
// and the electric field on cell corners (§3).
#include <algorithm>
#include <cstring>

#include "pic_internal.cuh"

namespace gbpic {

namespace {

constexpr int kT = 256;
inline unsigned blocks_for(int64_t n, int t = kT) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

// ---- leaf keys: root * 4^lmax + (morton << 2 (lmax - level)) --------------------------
__global__ void k_leaf_keys(int64_t n, int nx0, int ny0, int lmax, const uint32_t *__restrict__ root,
                            const uint32_t *__restrict__ morton, const uint8_t *__restrict__ level,
                            uint32_t *__restrict__ key, int32_t *__restrict__ err) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t r = root[i], l = level[i], m = morton[i];
    if (r >= (uint32_t)(nx0 * ny0) || l > (uint32_t)lmax || (l < 16 && m >= (1u << (2 * l)))) {
        atomicExch(err, 1);
        key[i] = 0xFFFFFFFFu;
        return;
    }
    key[i] = r * (1u << (2 * lmax)) + (m << (2 * (lmax - l)));
}

// Counting placement by key: slot[key] = input index (keys are unique in a valid tiling).
__global__ void k_key_slots(int64_t n, const uint32_t *__restrict__ key, uint32_t nkeys,
                            int32_t *__restrict__ slot, int32_t *__restrict__ err) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t k = key[i];
    if (k >= nkeys) { atomicExch(err, 1); return; }
    if (atomicCAS(slot + k, -1, (int32_t)i) != -1) atomicExch(err, 2);
}

__global__ void k_flag_present(uint32_t nkeys, const int32_t *__restrict__ slot, int32_t *__restrict__ flag) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nkeys) flag[k] = slot[k] >= 0 ? 1 : 0;
}

// Gather the leaves in key order and derive their lattice geometry.
__global__ void k_gather_sorted(uint32_t nkeys, const int32_t *__restrict__ slot,
                                const int32_t *__restrict__ pos, const uint32_t *__restrict__ root_in,
                                const uint32_t *__restrict__ morton_in, const uint8_t *__restrict__ level_in,
                                int nx0, int lmax, uint32_t *__restrict__ key, uint32_t *__restrict__ root,
                                uint32_t *__restrict__ morton, uint8_t *__restrict__ lev,
                                int32_t *__restrict__ ix, int32_t *__restrict__ iy) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nkeys) return;
    const int32_t src = slot[k];
    if (src < 0) return;
    const int32_t o = pos[k];
    const uint32_t r = root_in[src], m = morton_in[src], l = level_in[src];
    key[o] = (uint32_t)k;
    root[o] = r;
    morton[o] = m;
    lev[o] = (uint8_t)l;
    const int32_t rx = (int32_t)(r % (uint32_t)nx0), ry = (int32_t)(r / (uint32_t)nx0);
    ix[o] = (rx << lmax) + (int32_t)(compact2(m) << (lmax - l));
    iy[o] = (ry << lmax) + (int32_t)(compact2(m >> 1) << (lmax - l));
}

// Tiling: consecutive leaves cover consecutive key ranges of s*s keys, from 0 to the end.
__global__ void k_check_tiling(int64_t n, const uint32_t *__restrict__ key, const uint8_t *__restrict__ lev,
                               int lmax, uint64_t nkeys, int32_t *__restrict__ err) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint64_t s = 1ull << (lmax - lev[i]);
    const uint64_t end = (uint64_t)key[i] + s * s;
    const uint64_t next = (i + 1 < n) ? (uint64_t)key[i + 1] : nkeys;
    if (end != next || (i == 0 && key[0] != 0)) atomicExch(err, 3);
}

// Each leaf paints its s x s lattice cells with its index.
__global__ void k_fill_map(int64_t n, const int32_t *__restrict__ ix, const int32_t *__restrict__ iy,
                           const uint8_t *__restrict__ lev, int lmax, int NX, int32_t *__restrict__ map) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int s = 1 << (lmax - lev[i]);
    const int x0 = ix[i], y0 = iy[i];
    for (int dy = 0; dy < s; ++dy)
        for (int dx = 0; dx < s; ++dx) map[(int64_t)(y0 + dy) * NX + x0 + dx] = (int32_t)i;
}

// ---- faces of the composite mesh --------------------------------------------------------
enum { FB = 0, FS = 1, FC = 2, FF = 3, FBAD = -1 };
struct Face { int type; int32_t n1, n2, sib; };

struct LatView {
    const int32_t *map;
    const int32_t *ix, *iy;
    const uint8_t *lev;
    int NX, NY, lmax;
    bool px, py;
    __device__ __forceinline__ int32_t at(int32_t I, int32_t J) const { return lattice_leaf(map, NX, NY, px, py, I, J); }
    __device__ __forceinline__ int32_t side(int32_t c) const { return 1 << (lmax - lev[c]); }
};

__device__ Face face_of(const LatView &L, int32_t c, int dir) {
    Face f{FBAD, -1, -1, -1};
    const int32_t x = L.ix[c], y = L.iy[c], s = L.side(c);
    int32_t I1, J1, I2, J2;
    if (dir == 0) { I1 = I2 = x - 1; J1 = y; J2 = y + s - 1; }
    else if (dir == 1) { I1 = I2 = x + s; J1 = y; J2 = y + s - 1; }
    else if (dir == 2) { J1 = J2 = y - 1; I1 = x; I2 = x + s - 1; }
    else { J1 = J2 = y + s; I1 = x; I2 = x + s - 1; }
    const int32_t a = L.at(I1, J1), b = L.at(I2, J2);
    if (a < 0 || b < 0) { f.type = (a < 0 && b < 0) ? FB : FBAD; return f; }
    if (a == b) {
        const int32_t sa = L.side(a);
        if (sa == s) { f.type = FS; f.n1 = a; return f; }
        if (sa == 2 * s) {
            int32_t sib;
            if (dir < 2) { const int32_t js = (y == L.iy[a]) ? y + s : y - s; sib = L.at(x, js); }
            else { const int32_t is = (x == L.ix[a]) ? x + s : x - s; sib = L.at(is, y); }
            if (sib < 0 || L.side(sib) != s) return f;
            f.type = FC; f.n1 = a; f.sib = sib;
        }
        return f;
    }
    if (2 * L.side(a) == s && 2 * L.side(b) == s) { f.type = FF; f.n1 = a; f.n2 = b; }
    return f;
}

// 2:1 balance across faces; periodic walls have no boundary faces.
__global__ void k_check_balance(int64_t n, LatView L, int32_t *__restrict__ err) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    for (int d = 0; d < 4; ++d) {
        const Face f = face_of(L, (int32_t)c, d);
        if (f.type == FBAD) atomicExch(err, 4);
    }
}

// ---- Poisson operator (divided by eps0):  sum_faces g (phi_c - phi_face) = b_c ----------
//   same level: g = 1 toward the neighbour;  coarse next to a fine pair: 4/3 toward the pair
//   average; fine next to coarse N with sibling S: (2/3)((phi_c + phi_S)/2 - phi_N);
//   Dirichlet wall: 2 toward the wall value; Neumann: nothing.
// kappa (may be null: 1 everywhere) is the direct implicit scheme's relative permittivity
// 1 + chi per cell: each face's conductance is multiplied by the face's kappa, the mean of
// its two sides (at a coarse-fine face the coarse cell and the mean of the fine pair, the
// same value in all three rows, so the operator stays conservative).
__global__ void k_assemble(int64_t n, LatView L, int bcx, int bcy, int32_t *__restrict__ col,
                           float *__restrict__ val, float *__restrict__ dinv, double *__restrict__ val64,
                           double *__restrict__ diag64, double *__restrict__ bcw, uint8_t *__restrict__ color,
                           int32_t *__restrict__ err, const double *__restrict__ kappa) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    {
        const int sh = L.lmax - L.lev[c];
        color[c] = (uint8_t)(((L.ix[c] >> sh) + (L.iy[c] >> sh)) & 1);
    }
    double diag = 0.0;
    int k = 0;
    int32_t cc[kEll];
    double vv[kEll];
    double wall[4] = {0, 0, 0, 0};
    for (int d = 0; d < 4; ++d) {
        const Face f = face_of(L, (int32_t)c, d);
        const int bc = d < 2 ? bcx : bcy;
        if (!kappa) {
            switch (f.type) {
            case FB:
                if (bc == PIC_BC_DIRICHLET) { diag += 2.0; wall[d] = 2.0; }
                break;
            case FS:
                diag += 1.0; cc[k] = f.n1; vv[k++] = -1.0;
                break;
            case FF:
                diag += 4.0 / 3.0;
                cc[k] = f.n1; vv[k++] = -2.0 / 3.0;
                cc[k] = f.n2; vv[k++] = -2.0 / 3.0;
                break;
            case FC:
                diag += 1.0 / 3.0;
                cc[k] = f.sib; vv[k++] = 1.0 / 3.0;
                cc[k] = f.n1; vv[k++] = -2.0 / 3.0;
                break;
            default:
                atomicExch(err, 5);
            }
            continue;
        }
        double kf;
        switch (f.type) {
        case FB:
            if (bc == PIC_BC_DIRICHLET) { diag += 2.0 * kappa[c]; wall[d] = 2.0 * kappa[c]; }
            break;
        case FS:
            kf = 0.5 * (kappa[c] + kappa[f.n1]);
            diag += kf; cc[k] = f.n1; vv[k++] = -kf;
            break;
        case FF:
            kf = 0.5 * (kappa[c] + 0.5 * (kappa[f.n1] + kappa[f.n2]));
            diag += 4.0 / 3.0 * kf;
            cc[k] = f.n1; vv[k++] = -2.0 / 3.0 * kf;
            cc[k] = f.n2; vv[k++] = -2.0 / 3.0 * kf;
            break;
        case FC:
            kf = 0.5 * (kappa[f.n1] + 0.5 * (kappa[c] + kappa[f.sib]));
            diag += 1.0 / 3.0 * kf;
            cc[k] = f.sib; vv[k++] = 1.0 / 3.0 * kf;
            cc[k] = f.n1; vv[k++] = -2.0 / 3.0 * kf;
            break;
        default:
            atomicExch(err, 5);
        }
    }
    for (int j = 0; j < kEll; ++j) {
        const int32_t cj = j < k ? cc[j] : -1;
        const double vj = j < k ? vv[j] : 0.0;
        col[(int64_t)j * n + c] = cj;
        val[(int64_t)j * n + c] = (float)vj;
        if (val64) val64[(int64_t)j * n + c] = vj;
    }
    dinv[c] = diag > 0.0 ? (float)(1.0 / diag) : 0.0f;
    if (diag64) diag64[c] = diag;
    if (bcw)
        for (int d = 0; d < 4; ++d) bcw[4 * c + d] = wall[d];
}

// ---- coarser multigrid levels -----------------------------------------------------------
// Clamp a tree level: cells at level lmax (side 1) merge with their 3 Morton siblings.
__global__ void k_clamp_flags(int64_t n, const int32_t *__restrict__ ix, const int32_t *__restrict__ iy,
                              const uint8_t *__restrict__ lev, int lmax, int32_t *__restrict__ keep) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int child = (ix[i] & 1) | ((iy[i] & 1) << 1);
    keep[i] = (lev[i] < lmax || child == 0) ? 1 : 0;
}

__global__ void k_clamp_build(int64_t n, const int32_t *__restrict__ ix, const int32_t *__restrict__ iy,
                              const uint8_t *__restrict__ lev, int lmax, const int32_t *__restrict__ pos,
                              int32_t *__restrict__ parent, int32_t *__restrict__ cix, int32_t *__restrict__ ciy,
                              uint8_t *__restrict__ clev, int32_t *__restrict__ child4) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const bool fine = lev[i] == lmax;
    const int child = fine ? ((ix[i] & 1) | ((iy[i] & 1) << 1)) : 0;
    const int32_t p = pos[i - child];
    parent[i] = p;
    child4[4 * (int64_t)p + child] = (int32_t)i;
    if (child == 0) {
        cix[p] = ix[i] >> 1;
        ciy[p] = iy[i] >> 1;
        clev[p] = (uint8_t)(fine ? lmax - 1 : lev[i]);
    }
}

// Root-box coarsening of a uniform level-0 grid (row-major): 2x2 cells -> 1.
__global__ void k_root_coarsen(int nx, int ny, int32_t *__restrict__ parent, int32_t *__restrict__ child4,
                               int32_t *__restrict__ cix, int32_t *__restrict__ ciy, uint8_t *__restrict__ clev) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)nx * ny) return;
    const int x = (int)(i % nx), y = (int)(i / nx);
    const int cnx = nx >> 1;
    const int32_t p = (y >> 1) * cnx + (x >> 1);
    parent[i] = p;
    child4[4 * (int64_t)p + ((x & 1) | ((y & 1) << 1))] = (int32_t)i;
    if (((x | y) & 1) == 0) {
        cix[p] = x >> 1;
        ciy[p] = y >> 1;
        clev[p] = 0;
    }
}

// ---- corner electric field ---------------------------------------------------------------
// Corner field from the cell potentials.  Differences of the FP64 potential are taken in
// FP64; the scaling by 1/h (exact powers of two times 1/h_finest) and the averaging run in T
// (float in FP32 mode, double in FP64 mode), with no divisions.
template <typename T> struct FieldView {
    LatView L;
    const double *phi;
    T inv_hf;  // 1 / (lattice cell side)
    int bcx, bcy;
    double wall[4];
    const double *wall_dev;  // non-null: the wall potentials are read from here (captured steps)

    __device__ __forceinline__ T inv_h(int32_t c) const { return inv_hf * ((T)1 / (T)L.side(c)); }

    // d phi / dx across the vertical lattice line x = I at lattice row J (operator's face rule)
    __device__ T grad_x(int32_t I, int32_t J) const {
        const int32_t A = L.at(I - 1, J), B = L.at(I, J);
        if (A < 0 && B < 0) return (T)0;
        if (A < 0) return bcx == PIC_BC_DIRICHLET ? (T)(phi[B] - wall[0]) * ((T)2 * inv_h(B)) : (T)0;
        if (B < 0) return bcx == PIC_BC_DIRICHLET ? (T)(wall[1] - phi[A]) * ((T)2 * inv_h(A)) : (T)0;
        const int32_t sA = L.side(A), sB = L.side(B);
        if (sA == sB) return (T)(phi[B] - phi[A]) * inv_h(A);
        if (sA > sB) {
            const int32_t c1 = L.at(L.ix[A] + sA, L.iy[A]), c2 = L.at(L.ix[A] + sA, L.iy[A] + sA - 1);
            return (T)(0.5 * (phi[c1] + phi[c2]) - phi[A]) * (inv_h(A) * (T)(4.0 / 3.0));
        }
        const int32_t c1 = L.at(L.ix[B] - 1, L.iy[B]), c2 = L.at(L.ix[B] - 1, L.iy[B] + sB - 1);
        return (T)(phi[B] - 0.5 * (phi[c1] + phi[c2])) * (inv_h(B) * (T)(4.0 / 3.0));
    }
    __device__ T grad_y(int32_t I, int32_t J) const {
        const int32_t A = L.at(I, J - 1), B = L.at(I, J);
        if (A < 0 && B < 0) return (T)0;
        if (A < 0) return bcy == PIC_BC_DIRICHLET ? (T)(phi[B] - wall[2]) * ((T)2 * inv_h(B)) : (T)0;
        if (B < 0) return bcy == PIC_BC_DIRICHLET ? (T)(wall[3] - phi[A]) * ((T)2 * inv_h(A)) : (T)0;
        const int32_t sA = L.side(A), sB = L.side(B);
        if (sA == sB) return (T)(phi[B] - phi[A]) * inv_h(A);
        if (sA > sB) {
            const int32_t c1 = L.at(L.ix[A], L.iy[A] + sA), c2 = L.at(L.ix[A] + sA - 1, L.iy[A] + sA);
            return (T)(0.5 * (phi[c1] + phi[c2]) - phi[A]) * (inv_h(A) * (T)(4.0 / 3.0));
        }
        const int32_t c1 = L.at(L.ix[B], L.iy[B] - 1), c2 = L.at(L.ix[B] + sB - 1, L.iy[B] - 1);
        return (T)(phi[B] - 0.5 * (phi[c1] + phi[c2])) * (inv_h(B) * (T)(4.0 / 3.0));
    }
    __device__ bool in_x(int32_t I) const { return L.px || (I >= 0 && I < L.NX); }
    __device__ bool in_y(int32_t J) const { return L.py || (J >= 0 && J < L.NY); }

    // E at lattice node (I, J): regular nodes average the incident face gradients; a node
    // inside a coarser leaf's edge takes the mean of that edge's end nodes (recursively).
    __device__ void node(int32_t I, int32_t J, T &ex, T &ey) const {
        int32_t sI[24], sJ[24];
        T sw[24];
        int top = 0;
        sI[0] = I; sJ[0] = J; sw[0] = (T)1; top = 1;
        ex = (T)0; ey = (T)0;
        while (top > 0) {
            --top;
            const int32_t i = sI[top], j = sJ[top];
            const T wt = sw[top];
            const int32_t LL = L.at(i - 1, j - 1), LR = L.at(i, j - 1), UL = L.at(i - 1, j), UR = L.at(i, j);
            int32_t q = -1;
            bool horiz = false;
            if (UL >= 0 && UL == UR) { q = UL; horiz = true; }
            else if (LL >= 0 && LL == LR) { q = LL; horiz = true; }
            else if (LL >= 0 && LL == UL) { q = LL; horiz = false; }
            else if (LR >= 0 && LR == UR) { q = LR; horiz = false; }
            if (q >= 0 && top + 2 <= 24) {
                const int32_t s = L.side(q);
                if (horiz) {
                    const int32_t off = (((i - L.ix[q]) % L.NX) + L.NX) % L.NX;
                    sI[top] = i - off; sJ[top] = j; sw[top] = (T)0.5 * wt; ++top;
                    sI[top] = i - off + s; sJ[top] = j; sw[top] = (T)0.5 * wt; ++top;
                } else {
                    const int32_t off = (((j - L.iy[q]) % L.NY) + L.NY) % L.NY;
                    sI[top] = i; sJ[top] = j - off; sw[top] = (T)0.5 * wt; ++top;
                    sI[top] = i; sJ[top] = j - off + s; sw[top] = (T)0.5 * wt; ++top;
                }
                continue;
            }
            T sx = 0, sy = 0;
            int nx = 0, ny = 0;
            if (in_y(j)) { sx += grad_x(i, j); ++nx; }
            if (in_y(j - 1)) { sx += grad_x(i, j - 1); ++nx; }
            if (in_x(i - 1)) { sy += grad_y(i - 1, j); ++ny; }
            if (in_x(i)) { sy += grad_y(i, j); ++ny; }
            ex -= wt * (nx == 2 ? (T)0.5 * sx : sx);
            ey -= wt * (ny == 2 ? (T)0.5 * sy : sy);
        }
    }
};

template <typename R>
__global__ void k_node_e(int64_t n, FieldView<R> F, R *__restrict__ stencil) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 4 * n) return;
    if (F.wall_dev)
        for (int k = 0; k < 4; ++k) F.wall[k] = F.wall_dev[k];
    const int32_t l = (int32_t)(t >> 2);
    const int c = (int)(t & 3);
    const int32_t s = F.L.side(l);
    R ex, ey;
    F.node(F.L.ix[l] + ((c & 1) ? s : 0), F.L.iy[l] + ((c & 2) ? s : 0), ex, ey);
    stencil[8 * (int64_t)l + 2 * c] = ex;
    stencil[8 * (int64_t)l + 2 * c + 1] = ey;
}

__global__ void k_cell_emag(int64_t n, FieldView<double> F, double *__restrict__ out) {
    const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= n) return;
    const int32_t x = F.L.ix[l], y = F.L.iy[l], s = F.L.side((int32_t)l);
    const double gxl = 0.5 * (F.grad_x(x, y) + F.grad_x(x, y + s - 1));
    const double gxr = 0.5 * (F.grad_x(x + s, y) + F.grad_x(x + s, y + s - 1));
    const double gyl = 0.5 * (F.grad_y(x, y) + F.grad_y(x + s - 1, y));
    const double gyh = 0.5 * (F.grad_y(x, y + s) + F.grad_y(x + s - 1, y + s));
    const double ex = -0.5 * (gxl + gxr), ey = -0.5 * (gyl + gyh);
    out[l] = sqrt(ex * ex + ey * ey);
}

int32_t read_err(pic_ctx *ctx, int32_t *d_err) {
    int32_t h = 0;
    GB_CUDA(cudaMemcpyAsync(&h, d_err, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
    GB_CUDA(cudaStreamSynchronize(ctx->stream));
    return h;
}

LatView view_of(const Instance &in, const Level &g) {
    LatView L;
    L.map = g.map; L.ix = g.ix; L.iy = g.iy; L.lev = g.lev;
    L.NX = g.nx0 << g.lmax; L.NY = g.ny0 << g.lmax; L.lmax = g.lmax;
    L.px = in.cfg.bc_x == PIC_BC_PERIODIC; L.py = in.cfg.bc_y == PIC_BC_PERIODIC;
    return L;
}

void assemble_level(pic_ctx *ctx, Instance &in, Level &g, bool finest, int32_t *d_err) {
    DeviceArena &A = in.mesh_mem;
    g.col = dalloc<int32_t>(A, kEll * g.n);
    g.val = dalloc<float>(A, kEll * g.n);
    g.dinv = dalloc<float>(A, g.n);
    g.color = dalloc<uint8_t>(A, g.n);
    if (finest) {
        g.val64 = dalloc<double>(A, kEll * g.n);
        g.diag64 = dalloc<double>(A, g.n);
        g.bcw = dalloc<double>(A, 4 * g.n);
    }
    g.x = dalloc<float>(A, g.n);
    g.b = dalloc<float>(A, g.n);
    g.t = dalloc<float>(A, g.n);
    g.kappa = in.cfg.implicit ? dalloc<double>(A, g.n) : nullptr;  // set per step (poisson_kappa)
    k_assemble<<<blocks_for(g.n), kT, 0, ctx->stream>>>(g.n, view_of(in, g), in.cfg.bc_x, in.cfg.bc_y, g.col,
                                                        g.val, g.dinv, g.val64, g.diag64, g.bcw, g.color, d_err,
                                                        nullptr);
    count_launch(ctx);
}

// A coarse cell's kappa: the mean over its children.
__global__ void k_kappa_restrict(int64_t nc, const int32_t *__restrict__ child4, const double *__restrict__ kf,
                                 double *__restrict__ kc) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nc) return;
    double s = 0.0;
    int m = 0;
    for (int k = 0; k < 4; ++k) {
        const int32_t i = child4[4 * p + k];
        if (i >= 0) { s += kf[i]; ++m; }
    }
    kc[p] = m ? s / (double)m : 1.0;
}

// b = (charge + rho_bg h^2) / eps0 + sum_walls bcw phi_wall (the deposit's right-hand side,
// formed again once the walls' coefficients carry kappa).
__global__ void k_rhs(int64_t n, const double *__restrict__ charge, const uint8_t *__restrict__ lev, int lmax,
                      double hf, double rho_bg, double inv_eps0, const double *__restrict__ bcw, double w0, double w1,
                      double w2, double w3, double *__restrict__ b) {
    const int64_t L = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (L >= n) return;
    const double h = (double)(1 << (lmax - lev[L])) * hf;
    const double wall[4] = {w0, w1, w2, w3};
    double bl = (charge[L] + rho_bg * h * h) * inv_eps0;
    for (int k = 0; k < 4; ++k) bl += bcw[4 * L + k] * wall[k];
    b[L] = bl;
}

void fill_map(pic_ctx *ctx, Instance &in, Level &g) {
    g.map = dalloc<int32_t>(in.mesh_mem, g.lat_n());
    k_fill_map<<<blocks_for(g.n), kT, 0, ctx->stream>>>(g.n, g.ix, g.iy, g.lev, g.lmax, g.nx0 << g.lmax, g.map);
    count_launch(ctx);
}

}  // namespace

// Build the leaf mesh from host arrays (NULL root = uniform level-0 mesh).
void mesh_build(pic_ctx *ctx, Instance &in, int nx0, int ny0, double h0, int64_t n,
                const uint32_t *root, const uint32_t *morton, const uint8_t *level) {
    const int lmax = in.cfg.max_level;
    in.mesh_mem.release_all();
    in.lv.clear();
    in.has_mesh = false;
    in.nx0 = nx0; in.ny0 = ny0; in.h0 = h0; in.lmax = lmax;
    std::vector<uint32_t> r, m;
    std::vector<uint8_t> l;
    if (!root) {
        r.resize(n); m.assign(n, 0); l.assign(n, 0);
        for (int64_t i = 0; i < n; ++i) r[i] = (uint32_t)i;
        root = r.data(); morton = m.data(); level = l.data();
    }
    DeviceArena &A = in.mesh_mem;
    uint32_t *d_root = dalloc<uint32_t>(A, n), *d_mort = dalloc<uint32_t>(A, n);
    uint8_t *d_lev = dalloc<uint8_t>(A, n);
    GB_CUDA(cudaMemcpyAsync(d_root, root, n * 4, cudaMemcpyHostToDevice, ctx->stream));
    GB_CUDA(cudaMemcpyAsync(d_mort, morton, n * 4, cudaMemcpyHostToDevice, ctx->stream));
    GB_CUDA(cudaMemcpyAsync(d_lev, level, n, cudaMemcpyHostToDevice, ctx->stream));
    in.root = d_root; in.morton = d_mort;
    in.nleaf = n;
    Level g0;
    g0.lev = d_lev;
    in.lv.push_back(g0);
    mesh_build_device(ctx, in, n);
}

// Device part: sort the raw leaves in in.root / in.morton / in.lv[0].lev by key, check the
// tiling and 2:1 balance, paint the lattice map, build the multigrid levels and operators.
void mesh_build_device(pic_ctx *ctx, Instance &in, int64_t n) {
    const int lmax = in.lmax, nx0 = in.nx0, ny0 = in.ny0;
    DeviceArena &A = in.mesh_mem;
    const uint64_t nkeys64 = (uint64_t)nx0 * ny0 << (2 * lmax);
    if (nkeys64 >= (1ull << 31)) fail(PIC_EINVAL, "lattice too large (nx0*ny0*4^max_level >= 2^31)");
    const uint32_t nkeys = (uint32_t)nkeys64;
    int32_t *d_err = dalloc<int32_t>(A, 1);
    GB_CUDA(cudaMemsetAsync(d_err, 0, 4, ctx->stream));
    uint32_t *raw_key = dalloc<uint32_t>(A, n);
    const uint32_t *raw_root = in.root, *raw_mort = in.morton;
    const uint8_t *raw_lev = in.lv[0].lev;
    k_leaf_keys<<<blocks_for(n), kT, 0, ctx->stream>>>(n, nx0, ny0, lmax, raw_root, raw_mort, raw_lev, raw_key, d_err);
    int32_t *slot = dalloc<int32_t>(A, nkeys + 1);
    int32_t *pos = dalloc<int32_t>(A, nkeys + 1);
    int32_t *scratch = dalloc<int32_t>(A, scan_scratch_elems(nkeys));
    GB_CUDA(cudaMemsetAsync(slot, 0xFF, (size_t)nkeys * 4, ctx->stream));
    k_key_slots<<<blocks_for(n), kT, 0, ctx->stream>>>(n, raw_key, nkeys, slot, d_err);
    k_flag_present<<<blocks_for(nkeys), kT, 0, ctx->stream>>>(nkeys, slot, pos);
    count_launch(ctx, 3);
    exclusive_scan_i32(ctx, pos, pos, nkeys, scratch);
    Level g;
    g.nx0 = nx0; g.ny0 = ny0; g.lmax = lmax; g.h0 = in.h0; g.n = n;
    g.ix = dalloc<int32_t>(A, n); g.iy = dalloc<int32_t>(A, n); g.lev = dalloc<uint8_t>(A, n);
    in.key = dalloc<uint32_t>(A, n);
    uint32_t *root = dalloc<uint32_t>(A, n), *mort = dalloc<uint32_t>(A, n);
    k_gather_sorted<<<blocks_for(nkeys), kT, 0, ctx->stream>>>(nkeys, slot, pos, raw_root, raw_mort, raw_lev, nx0,
                                                               lmax, in.key, root, mort, g.lev, g.ix, g.iy);
    k_check_tiling<<<blocks_for(n), kT, 0, ctx->stream>>>(n, in.key, g.lev, lmax, nkeys64, d_err);
    count_launch(ctx, 2);
    int32_t e = read_err(ctx, d_err);
    if (e) fail(PIC_EINVAL, "leaf set is not a tiling of the root boxes (code " + std::to_string(e) + ")");
    A.release(raw_key);
    A.release(slot);
    A.release(pos);
    A.release(scratch);
    in.root = root; in.morton = mort;
    fill_map(ctx, in, g);
    in.lv.clear();
    in.lv.push_back(g);
    k_check_balance<<<blocks_for(n), kT, 0, ctx->stream>>>(n, view_of(in, in.lv[0]), d_err);
    count_launch(ctx);
    e = read_err(ctx, d_err);
    if (e) fail(PIC_EINVAL, "leaf set is not 2:1 balanced across faces");
    assemble_level(ctx, in, in.lv[0], true, d_err);
    // coarser levels
    for (;;) {
        Level &f = in.lv.back();
        Level c;
        if (f.lmax > 0) {
            int32_t *keep = dalloc<int32_t>(A, f.n + 1);
            int32_t *sc = dalloc<int32_t>(A, scan_scratch_elems(f.n));
            k_clamp_flags<<<blocks_for(f.n), kT, 0, ctx->stream>>>(f.n, f.ix, f.iy, f.lev, f.lmax, keep);
            count_launch(ctx);
            exclusive_scan_i32(ctx, keep, keep, f.n, sc);
            int32_t nc = 0;
            GB_CUDA(cudaMemcpyAsync(&nc, keep + f.n, 4, cudaMemcpyDeviceToHost, ctx->stream));
            GB_CUDA(cudaStreamSynchronize(ctx->stream));
            c.nx0 = f.nx0; c.ny0 = f.ny0; c.lmax = f.lmax - 1; c.h0 = f.h0; c.n = nc;
            c.ix = dalloc<int32_t>(A, nc); c.iy = dalloc<int32_t>(A, nc); c.lev = dalloc<uint8_t>(A, nc);
            f.parent = dalloc<int32_t>(A, f.n);
            c.child4 = dalloc<int32_t>(A, 4 * (int64_t)nc);
            GB_CUDA(cudaMemsetAsync(c.child4, 0xFF, 16 * (size_t)nc, ctx->stream));
            k_clamp_build<<<blocks_for(f.n), kT, 0, ctx->stream>>>(f.n, f.ix, f.iy, f.lev, f.lmax, keep, f.parent,
                                                                   c.ix, c.iy, c.lev, c.child4);
            count_launch(ctx);
            A.release(keep);
            A.release(sc);
        } else {
            if ((f.nx0 & 1) || (f.ny0 & 1) || f.n <= 16) break;
            c.nx0 = f.nx0 / 2; c.ny0 = f.ny0 / 2; c.lmax = 0; c.h0 = f.h0 * 2; c.n = (int64_t)c.nx0 * c.ny0;
            c.ix = dalloc<int32_t>(A, c.n); c.iy = dalloc<int32_t>(A, c.n); c.lev = dalloc<uint8_t>(A, c.n);
            f.parent = dalloc<int32_t>(A, f.n);
            c.child4 = dalloc<int32_t>(A, 4 * c.n);
            GB_CUDA(cudaMemsetAsync(c.child4, 0xFF, 16 * (size_t)c.n, ctx->stream));
            k_root_coarsen<<<blocks_for(f.n), kT, 0, ctx->stream>>>(f.nx0, f.ny0, f.parent, c.child4, c.ix, c.iy, c.lev);
            count_launch(ctx);
        }
        in.lv.push_back(c);
        Level &cc = in.lv.back();
        fill_map(ctx, in, cc);
        assemble_level(ctx, in, cc, false, d_err);
    }
    e = read_err(ctx, d_err);
    if (e) fail(PIC_EINVAL, "multigrid level construction failed (code " + std::to_string(e) + ")");
    check_launch("mesh_build");
    in.has_mesh = true;
}

template <typename T> FieldView<T> field_view(const Instance &in, const double walls[4]) {
    FieldView<T> F;
    F.L = view_of(in, in.lv[0]);
    F.phi = in.phi;
    F.inv_hf = (T)((double)(1 << in.lmax) / in.h0);
    F.bcx = in.cfg.bc_x; F.bcy = in.cfg.bc_y;
    for (int k = 0; k < 4; ++k) F.wall[k] = walls[k];
    F.wall_dev = nullptr;
    return F;
}

// The corner field of every instance of an ensemble in one launch: block b takes the 4 corners
// of the leaves [c.y, c.z) of instance c.x, whose view (with the step's wall potentials read
// from the device) sits in shared memory.
template <typename R> struct NodeEEntry {
    FieldView<R> F;
    R *stencil;
};
template <typename R>
__global__ void __launch_bounds__(kT) k_node_e_batch(const NodeEEntry<R> *__restrict__ tab,
                                                     const int4 *__restrict__ chunks) {
    __shared__ NodeEEntry<R> se;
    const int4 c = chunks[blockIdx.x];
    {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(tab + c.x);
        uint32_t *dst = reinterpret_cast<uint32_t *>(&se);
        for (int k = threadIdx.x; k < (int)(sizeof(NodeEEntry<R>) / 4); k += blockDim.x) dst[k] = src[k];
    }
    __syncthreads();
    if (threadIdx.x < 4) se.F.wall[threadIdx.x] = se.F.wall_dev[threadIdx.x];
    __syncthreads();
    const int64_t l = (int64_t)c.y + (threadIdx.x >> 2);
    if (l >= c.z) return;
    const int cc = (int)(threadIdx.x & 3);
    const FieldView<R> &F = se.F;
    const int32_t s = F.L.side((int32_t)l);
    R ex, ey;
    F.node(F.L.ix[l] + ((cc & 1) ? s : 0), F.L.iy[l] + ((cc & 2) ? s : 0), ex, ey);
    se.stencil[8 * l + 2 * cc] = ex;
    se.stencil[8 * l + 2 * cc + 1] = ey;
}

template <typename R> void batch_prepare_node_e_impl(pic_ctx *ctx) {
    std::vector<NodeEEntry<R>> tab;
    std::vector<int64_t> nls;
    const double zero[4] = {0.0, 0.0, 0.0, 0.0};
    for (Instance &in : ctx->inst) {
        NodeEEntry<R> e;
        e.F = field_view<R>(in, zero);
        e.F.wall_dev = in.d_walls;
        e.stencil = (R *)in.stencil;
        tab.push_back(e);
        nls.push_back(in.lv[0].n);
    }
    const std::vector<int4> ch = batch_chunks(nls, kT / 4);
    BatchTab &t = ctx->batch.nodee;
    t.tab = batch_upload(ctx, tab);
    t.chunks = batch_upload(ctx, ch);
    t.n = (int)tab.size();
    t.nchunks = (int)ch.size();
}

void batch_prepare_node_e(pic_ctx *ctx) {
    if (ctx->inst.front().cfg.precision == PIC_FP64) batch_prepare_node_e_impl<double>(ctx);
    else batch_prepare_node_e_impl<float>(ctx);
}

void node_e_batch(pic_ctx *ctx) {
    const BatchTab &t = ctx->batch.nodee;
    if (ctx->inst.front().cfg.precision == PIC_FP64)
        k_node_e_batch<double><<<(unsigned)t.nchunks, kT, 0, ctx->stream>>>((const NodeEEntry<double> *)t.tab, t.chunks);
    else
        k_node_e_batch<float><<<(unsigned)t.nchunks, kT, 0, ctx->stream>>>((const NodeEEntry<float> *)t.tab, t.chunks);
    count_launch(ctx);
    check_launch("node_e_batch");
}

// The direct implicit scheme's operator for this step: kappa of the finest level (written by
// the deposit) restricted to every coarser level, every level assembled again with it, and
// the right-hand side formed with the new wall coefficients.
void poisson_kappa(pic_ctx *ctx, Instance &in, const double walls[4]) {
    cudaStream_t st = ctx->stream;
    for (size_t g = 1; g < in.lv.size(); ++g) {
        Level &C = in.lv[g];
        k_kappa_restrict<<<blocks_for(C.n), kT, 0, st>>>(C.n, C.child4, in.lv[g - 1].kappa, C.kappa);
        count_launch(ctx);
    }
    for (size_t g = 0; g < in.lv.size(); ++g) {
        Level &L = in.lv[g];
        k_assemble<<<blocks_for(L.n), kT, 0, st>>>(L.n, view_of(in, L), in.cfg.bc_x, in.cfg.bc_y, L.col, L.val,
                                                   L.dinv, L.val64, L.diag64, L.bcw, L.color, in.d_err, L.kappa);
        count_launch(ctx);
    }
    const Level &F = in.lv[0];
    k_rhs<<<blocks_for(F.n), kT, 0, st>>>(F.n, in.charge, F.lev, in.lmax, in.h0 / (double)(1 << in.lmax),
                                          in.cfg.rho_background, 1.0 / in.cfg.eps0, F.bcw, walls[0], walls[1],
                                          walls[2], walls[3], in.bvec);
    count_launch(ctx);
    check_launch("poisson_kappa");
}

void node_e(pic_ctx *ctx, Instance &in, const double walls[4]) {
    Level &g = in.lv[0];
    // a captured step reads the wall potentials of its time from the device
    const double *wd = ctx->capturing ? in.d_walls : nullptr;
    if (in.cfg.precision == PIC_FP64) {
        FieldView<double> F = field_view<double>(in, walls);
        F.wall_dev = wd;
        k_node_e<double><<<blocks_for(4 * g.n), kT, 0, ctx->stream>>>(g.n, F, (double *)in.stencil);
    } else {
        FieldView<float> F = field_view<float>(in, walls);
        F.wall_dev = wd;
        k_node_e<float><<<blocks_for(4 * g.n), kT, 0, ctx->stream>>>(g.n, F, (float *)in.stencil);
    }
    count_launch(ctx);
    check_launch("node_e");
    if (in.cfg.shape != PIC_SHAPE_NGP) cic_patch(ctx, in, walls);  // the push gathers from it
}

void cell_emag(pic_ctx *ctx, Instance &in, const double walls[4], double *out_dev) {
    Level &g = in.lv[0];
    k_cell_emag<<<blocks_for(g.n), kT, 0, ctx->stream>>>(g.n, field_view<double>(in, walls), out_dev);
    count_launch(ctx);
    check_launch("cell_emag");
}

}  // namespace gbpic
