/*
 * ORACLE — test infrastructure only.
 *
 * A plain, slow FP64 CPU restatement of the electrostatic PIC-MCC particle cycle on a
 * cell-based quadtree of Kolobov & Arslanbekov, "Electrostatic PIC with adaptive
 * Cartesian mesh" (arXiv:1604.07713).  Only the test-suite, the package's smoke check
 * and the CPU-baseline leg of the benchmark may load this library.  It shares no code,
 * header or table with the CUDA path.
 *
 * Conventions (one reading of the paper, applied identically everywhere):
 *   - Forest of nx0 x ny0 square root cells of side h0 (FOT boxes, §2.1); each root holds a
 *     quadtree of depth <= lmax.  The finest lattice has cells of side h0 / 2^lmax.
 *   - A leaf is (root, level, Morton code inside the root at that level).  Its sort key is
 *     root * 4^lmax + (morton << 2*(lmax-level)), i.e. the Morton index of its first finest
 *     cell (SFC ordering, §2.1).  A leaf covers keys [key, key + s*s), s = 2^(lmax-level).
 *   - Particles carry absolute FP64 positions here (the CUDA path stores cell offsets).
 *   - All arithmetic is FP64; build with -ffp-contract=off so no fused multiply-add.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------------------ */
/* Philox4x32-10 counter-based generator: Salmon, Moraes, Dror & Shaw, "Parallel random  */
/* numbers: as easy as 1, 2, 3", SC'11.  Ten rounds of the 4x32 Philox S-box with a      */
/* Weyl-sequence key schedule.                                                           */
/* ------------------------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Philox2x32-10 (same paper): a two-word counter, one 32 x 32 -> 64-bit product per round  */
/* (multiplier 0xD256D193), the Weyl key schedule k + r 0x9E3779B9, ten rounds.            */
void or_philox2x32_10(const uint32_t ctr_in[2], uint32_t key, uint32_t out[2])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) key += 0x9E3779B9u;
        uint64_t p = (uint64_t)0xD256D193u * (uint64_t)c0;
        uint32_t hi = (uint32_t)(p >> 32), lo = (uint32_t)p;
        c0 = hi ^ c1 ^ key;
        c1 = lo;
    }
    out[0] = c0; out[1] = c1;
}

/* Uniform in [0,1) from the top 24 bits: exactly representable in FP32 and FP64. */
static double u24(uint32_t r) { return (double)(r >> 8) * (1.0 / 16777216.0); }

/* Bulk draw for tests: counters (c0[i], c1, c2, c3) -> 4 words each. */
void or_philox_bulk(int64_t n, const uint32_t *c0, uint32_t c1, uint32_t c2, uint32_t c3,
                    uint32_t k0, uint32_t k1, uint32_t *out)
{
    uint32_t key[2] = {k0, k1};
    for (int64_t i = 0; i < n; ++i) {
        uint32_t ctr[4] = {c0[i], c1, c2, c3};
        or_philox4x32_10(ctr, key, out + 4 * i);
    }
}

/* ------------------------------------------------------------------------------------ */
/* Morton order (§2.1: SFC "currently based on Morton order")                            */
/* ------------------------------------------------------------------------------------ */
static uint32_t spread_bits(uint32_t v)
{
    uint32_t r = 0;
    for (int b = 0; b < 16; ++b)
        if (v & (1u << b)) r |= 1u << (2 * b);
    return r;
}
static uint32_t gather_bits(uint32_t v)
{
    uint32_t r = 0;
    for (int b = 0; b < 16; ++b)
        if (v & (1u << (2 * b))) r |= 1u << b;
    return r;
}
uint32_t or_morton(uint32_t cx, uint32_t cy) { return spread_bits(cx) | (spread_bits(cy) << 1); }

/* Leaf geometry on the finest lattice: corner (ix, iy), side s, sort key. */
int or_leaf_geometry(int64_t n, int32_t nx0, int32_t ny0, int32_t lmax, const int32_t *root,
                     const int32_t *level, const uint32_t *morton, int32_t *ix, int32_t *iy,
                     int32_t *s, int64_t *key)
{
    for (int64_t i = 0; i < n; ++i) {
        int32_t r = root[i], l = level[i];
        if (r < 0 || r >= nx0 * ny0 || l < 0 || l > lmax) return -1;
        uint32_t m = morton[i];
        if (l < 16 && (uint64_t)m >= ((uint64_t)1 << (2 * l))) return -1;
        uint32_t cx = gather_bits(m), cy = gather_bits(m >> 1);
        int32_t rx = r % nx0, ry = r / nx0;
        s[i] = 1 << (lmax - l);
        ix[i] = (rx << lmax) + (int32_t)(cx << (lmax - l));
        iy[i] = (ry << lmax) + (int32_t)(cy << (lmax - l));
        key[i] = (int64_t)r * ((int64_t)1 << (2 * lmax)) + ((int64_t)m << (2 * (lmax - l)));
    }
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Mesh and point location                                                               */
/* ------------------------------------------------------------------------------------ */
enum { BC_PERIODIC = 0, BC_DIRICHLET = 1, BC_NEUMANN = 2 };

typedef struct {
    int32_t nx0, ny0, lmax, bc_x, bc_y;
    int32_t pad_;
    double h0;
    int64_t nleaf;
    const int64_t *key; /* ascending */
    const int32_t *ix, *iy, *s;
} or_mesh;

static int32_t lat_nx(const or_mesh *m) { return m->nx0 << m->lmax; }
static int32_t lat_ny(const or_mesh *m) { return m->ny0 << m->lmax; }

/* Key of the finest lattice cell (I, J), which must lie inside the domain. */
static int64_t lattice_key(const or_mesh *m, int32_t I, int32_t J)
{
    int32_t mask = (1 << m->lmax) - 1;
    int64_t root = (int64_t)(I >> m->lmax) + (int64_t)(J >> m->lmax) * m->nx0;
    return root * ((int64_t)1 << (2 * m->lmax)) + or_morton((uint32_t)(I & mask), (uint32_t)(J & mask));
}

/* Leaf covering lattice cell (I, J): the last leaf whose key is <= the cell's key
 * (leaves tile the Morton curve in contiguous key ranges).  Periodic directions wrap;
 * outside a non-periodic wall returns -1. */
int64_t or_leaf_at(const or_mesh *m, int32_t I, int32_t J)
{
    int32_t NX = lat_nx(m), NY = lat_ny(m);
    if (I < 0 || I >= NX) {
        if (m->bc_x != BC_PERIODIC) return -1;
        I = ((I % NX) + NX) % NX;
    }
    if (J < 0 || J >= NY) {
        if (m->bc_y != BC_PERIODIC) return -1;
        J = ((J % NY) + NY) % NY;
    }
    int64_t K = lattice_key(m, I, J);
    int64_t lo = 0, hi = m->nleaf; /* first index with key > K */
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (m->key[mid] <= K) lo = mid + 1; else hi = mid;
    }
    return lo - 1;
}

/* Half-open point location: leaf l holds x if x in [x_l, x_l + h_l)^2 (floor rule). */
void or_locate(const or_mesh *m, int64_t n, const double *x, const double *y, int64_t *leaf)
{
    double hf = m->h0 / (double)(1 << m->lmax);
    for (int64_t i = 0; i < n; ++i) {
        int32_t I = (int32_t)floor(x[i] / hf), J = (int32_t)floor(y[i] / hf);
        if (I < 0 || I >= lat_nx(m) || J < 0 || J >= lat_ny(m)) { leaf[i] = -1; continue; }
        leaf[i] = or_leaf_at(m, I, J);
    }
}

/* Brute-force location over all leaves (pin for the key search on tiny trees). */
void or_locate_brute(const or_mesh *m, int64_t n, const double *x, const double *y, int64_t *leaf)
{
    double hf = m->h0 / (double)(1 << m->lmax);
    for (int64_t i = 0; i < n; ++i) {
        leaf[i] = -1;
        for (int64_t l = 0; l < m->nleaf; ++l) {
            double x0 = m->ix[l] * hf, y0 = m->iy[l] * hf, h = m->s[l] * hf;
            if (x[i] >= x0 && x[i] < x0 + h && y[i] >= y0 && y[i] < y0 + h) { leaf[i] = l; break; }
        }
    }
}

/* ------------------------------------------------------------------------------------ */
/* Faces of the composite leaf mesh.                                                      */
/* dir: 0 = -x, 1 = +x, 2 = -y, 3 = +y.                                                   */
/* ------------------------------------------------------------------------------------ */
enum { F_BOUNDARY = 0, F_SAME = 1, F_COARSER = 2, F_FINER = 3, F_BAD = -1 };

typedef struct {
    int type;
    int64_t n1, n2; /* SAME/COARSER: n1 = neighbour; FINER: the fine pair (n1 lower/left, n2 upper/right) */
    int64_t sib;    /* COARSER: the sibling of this leaf sharing the coarse neighbour's face */
} or_face;

static or_face face_of(const or_mesh *m, int64_t c, int dir)
{
    or_face f = {F_BAD, -1, -1, -1};
    int32_t ix = m->ix[c], iy = m->iy[c], s = m->s[c];
    int32_t I1, J1, I2, J2;
    switch (dir) {
    case 0: I1 = I2 = ix - 1; J1 = iy; J2 = iy + s - 1; break;
    case 1: I1 = I2 = ix + s; J1 = iy; J2 = iy + s - 1; break;
    case 2: J1 = J2 = iy - 1; I1 = ix; I2 = ix + s - 1; break;
    default: J1 = J2 = iy + s; I1 = ix; I2 = ix + s - 1; break;
    }
    int64_t a = or_leaf_at(m, I1, J1), b = or_leaf_at(m, I2, J2);
    if (a < 0 || b < 0) { f.type = (a < 0 && b < 0) ? F_BOUNDARY : F_BAD; return f; }
    if (a == b) {
        int32_t sn = m->s[a];
        if (sn == s) { f.type = F_SAME; f.n1 = a; return f; }
        if (sn == 2 * s) {
            f.type = F_COARSER; f.n1 = a;
            /* sibling: the other fine cell along the coarse neighbour's face */
            if (dir < 2) {
                int32_t jn = m->iy[a];
                int32_t js = (iy == jn) ? iy + s : iy - s;
                f.sib = or_leaf_at(m, ix, js);
            } else {
                int32_t in = m->ix[a];
                int32_t is = (ix == in) ? ix + s : ix - s;
                f.sib = or_leaf_at(m, is, iy);
            }
            if (f.sib < 0 || m->s[f.sib] != s) f.type = F_BAD;
            return f;
        }
        return f; /* unbalanced */
    }
    if (m->s[a] * 2 == s && m->s[b] * 2 == s) { f.type = F_FINER; f.n1 = a; f.n2 = b; }
    return f;
}

/* Validate tiling (consecutive key ranges, full coverage) and 2:1 face balance.
 * Returns 0 if valid. */
int or_check_tree(const or_mesh *m)
{
    int64_t total = (int64_t)m->nx0 * m->ny0 * ((int64_t)1 << (2 * m->lmax));
    int64_t expect = 0;
    for (int64_t i = 0; i < m->nleaf; ++i) {
        if (m->key[i] != expect) return 1;
        expect += (int64_t)m->s[i] * m->s[i];
    }
    if (expect != total) return 2;
    for (int64_t i = 0; i < m->nleaf; ++i)
        for (int d = 0; d < 4; ++d) {
            or_face f = face_of(m, i, d);
            if (f.type == F_BAD) return 3;
            if (f.type == F_BOUNDARY) {
                int is_x = d < 2;
                if ((is_x ? m->bc_x : m->bc_y) == BC_PERIODIC) return 4;
            }
        }
    return 0;
}

/* Face neighbour table for tests: per leaf and direction, type and up to two neighbours. */
void or_face_table(const or_mesh *m, int32_t *type, int64_t *n1, int64_t *n2, int64_t *sib)
{
    for (int64_t i = 0; i < m->nleaf; ++i)
        for (int d = 0; d < 4; ++d) {
            or_face f = face_of(m, i, d);
            type[4 * i + d] = f.type; n1[4 * i + d] = f.n1; n2[4 * i + d] = f.n2; sib[4 * i + d] = f.sib;
        }
}

/* ------------------------------------------------------------------------------------ */
/* Poisson operator (§3: multigrid Poisson solver with the potential at cell centres).    */
/* Cell-centred finite volumes on the composite leaf mesh, divided by eps0:               */
/*   sum_faces g_f (phi_C - phi_f) = rho_C h_C^2 / eps0                                    */
/*   same level:  g = 1 toward the neighbour;                                             */
/*   coarse C next to a fine pair (F1, F2): g = 4/3 toward (phi_F1 + phi_F2)/2, the pair  */
/*     average sits on the face normal at 3h_C/4;                                          */
/*   fine C next to coarse N, sibling S: each half face carries half of that flux:        */
/*     (2/3) ((phi_C + phi_S)/2 - phi_N);                                                  */
/*   Dirichlet wall: g = 2 toward the wall value (distance h/2);  Neumann wall: no flux.  */
/* The operator is conservative and reproduces linear potentials exactly.                 */
/* Emits COO triplets (row, col, val) and the per-leaf Dirichlet coefficients on the low  */
/* and high x and y walls (rhs += coef * phi_wall).  Returns the triplet count.           */
/* ------------------------------------------------------------------------------------ */
int64_t or_assemble(const or_mesh *m, int64_t *row, int64_t *col, double *val, double *bc_coef)
{
    int64_t k = 0;
    for (int64_t c = 0; c < m->nleaf; ++c) {
        double diag = 0.0;
        for (int w = 0; w < 4; ++w) bc_coef[4 * c + w] = 0.0;
        for (int d = 0; d < 4; ++d) {
            or_face f = face_of(m, c, d);
            int bc = (d < 2) ? m->bc_x : m->bc_y;
            switch (f.type) {
            case F_BOUNDARY:
                if (bc == BC_DIRICHLET) { diag += 2.0; bc_coef[4 * c + d] = 2.0; }
                break;
            case F_SAME:
                diag += 1.0;
                row[k] = c; col[k] = f.n1; val[k] = -1.0; ++k;
                break;
            case F_FINER:
                diag += 4.0 / 3.0;
                row[k] = c; col[k] = f.n1; val[k] = -2.0 / 3.0; ++k;
                row[k] = c; col[k] = f.n2; val[k] = -2.0 / 3.0; ++k;
                break;
            case F_COARSER:
                diag += 1.0 / 3.0;
                row[k] = c; col[k] = f.sib; val[k] = 1.0 / 3.0; ++k;
                row[k] = c; col[k] = f.n1; val[k] = -2.0 / 3.0; ++k;
                break;
            default:
                return -1;
            }
        }
        row[k] = c; col[k] = c; val[k] = diag; ++k;
    }
    return k;
}

/* The same operator with a relative permittivity kappa per leaf (the direct implicit       */
/* scheme's 1 + chi, §3): every face's conductance is multiplied by the face's kappa, the    */
/* mean of the kappa on its two sides:                                                     */
/*   same level: (k_C + k_N)/2;  Dirichlet wall: k_C;                                       */
/*   coarse C and fine pair (F1, F2): (k_C + (k_F1 + k_F2)/2)/2, the same value in the      */
/*   coarse cell's row and in both fine cells' rows, so the operator stays conservative.    */
int64_t or_assemble_kappa(const or_mesh *m, const double *kappa, int64_t *row, int64_t *col, double *val,
                          double *bc_coef)
{
    int64_t k = 0;
    for (int64_t c = 0; c < m->nleaf; ++c) {
        double diag = 0.0;
        for (int w = 0; w < 4; ++w) bc_coef[4 * c + w] = 0.0;
        for (int d = 0; d < 4; ++d) {
            or_face f = face_of(m, c, d);
            int bc = (d < 2) ? m->bc_x : m->bc_y;
            double kf;
            switch (f.type) {
            case F_BOUNDARY:
                if (bc == BC_DIRICHLET) { diag += 2.0 * kappa[c]; bc_coef[4 * c + d] = 2.0 * kappa[c]; }
                break;
            case F_SAME:
                kf = 0.5 * (kappa[c] + kappa[f.n1]);
                diag += kf;
                row[k] = c; col[k] = f.n1; val[k] = -kf; ++k;
                break;
            case F_FINER:
                kf = 0.5 * (kappa[c] + 0.5 * (kappa[f.n1] + kappa[f.n2]));
                diag += 4.0 / 3.0 * kf;
                row[k] = c; col[k] = f.n1; val[k] = -2.0 / 3.0 * kf; ++k;
                row[k] = c; col[k] = f.n2; val[k] = -2.0 / 3.0 * kf; ++k;
                break;
            case F_COARSER:
                kf = 0.5 * (kappa[f.n1] + 0.5 * (kappa[c] + kappa[f.sib]));
                diag += 1.0 / 3.0 * kf;
                row[k] = c; col[k] = f.sib; val[k] = 1.0 / 3.0 * kf; ++k;
                row[k] = c; col[k] = f.n1; val[k] = -2.0 / 3.0 * kf; ++k;
                break;
            default:
                return -1;
            }
        }
        row[k] = c; col[k] = c; val[k] = diag; ++k;
    }
    return k;
}

/* Gradient d(phi)/dx across the vertical lattice line x = I at lattice row J, using the
 * face rule of the operator above.  phi_lo / phi_hi are the wall values (x = 0, x = Lx). */
static double grad_x_at(const or_mesh *m, const double *phi, int32_t I, int32_t J,
                        double phi_lo, double phi_hi)
{
    double hf = m->h0 / (double)(1 << m->lmax);
    int64_t A = or_leaf_at(m, I - 1, J), B = or_leaf_at(m, I, J);
    if (A < 0 && B < 0) return 0.0;
    if (A < 0) { /* B is at the low x wall */
        if (m->bc_x == BC_DIRICHLET) return (phi[B] - phi_lo) / (0.5 * m->s[B] * hf);
        return 0.0;
    }
    if (B < 0) {
        if (m->bc_x == BC_DIRICHLET) return (phi_hi - phi[A]) / (0.5 * m->s[A] * hf);
        return 0.0;
    }
    double hA = m->s[A] * hf, hB = m->s[B] * hf;
    if (m->s[A] == m->s[B]) return (phi[B] - phi[A]) / hA;
    if (m->s[A] > m->s[B]) { /* A coarse: fine pair across A's +x face */
        or_face f = face_of(m, A, 1);
        return (0.5 * (phi[f.n1] + phi[f.n2]) - phi[A]) / (0.75 * hA);
    }
    or_face f = face_of(m, B, 0); /* B coarse: fine pair across B's -x face */
    return (phi[B] - 0.5 * (phi[f.n1] + phi[f.n2])) / (0.75 * hB);
}

static double grad_y_at(const or_mesh *m, const double *phi, int32_t I, int32_t J,
                        double phi_lo, double phi_hi)
{
    double hf = m->h0 / (double)(1 << m->lmax);
    int64_t A = or_leaf_at(m, I, J - 1), B = or_leaf_at(m, I, J);
    if (A < 0 && B < 0) return 0.0;
    if (A < 0) {
        if (m->bc_y == BC_DIRICHLET) return (phi[B] - phi_lo) / (0.5 * m->s[B] * hf);
        return 0.0;
    }
    if (B < 0) {
        if (m->bc_y == BC_DIRICHLET) return (phi_hi - phi[A]) / (0.5 * m->s[A] * hf);
        return 0.0;
    }
    double hA = m->s[A] * hf, hB = m->s[B] * hf;
    if (m->s[A] == m->s[B]) return (phi[B] - phi[A]) / hA;
    if (m->s[A] > m->s[B]) {
        or_face f = face_of(m, A, 3);
        return (0.5 * (phi[f.n1] + phi[f.n2]) - phi[A]) / (0.75 * hA);
    }
    or_face f = face_of(m, B, 2);
    return (phi[B] - 0.5 * (phi[f.n1] + phi[f.n2])) / (0.75 * hB);
}

/* ------------------------------------------------------------------------------------ */
/* Electric field on cell nodes/corners (§3: "components of the electric field vector on */
/* cell nodes/corners").  At a regular node, E = -(mean of the face-normal gradients of   */
/* the faces incident to the node); at a hanging node (inside the edge of a coarser leaf)*/
/* E is the mean of the values at the two ends of that edge, applied recursively.         */
/* walls[4] = phi on the x-low, x-high, y-low, y-high walls (Dirichlet only).              */
/* ------------------------------------------------------------------------------------ */
typedef struct { double ex, ey; } vec2;

static int in_y(const or_mesh *m, int32_t J) { return m->bc_y == BC_PERIODIC || (J >= 0 && J < lat_ny(m)); }
static int in_x(const or_mesh *m, int32_t I) { return m->bc_x == BC_PERIODIC || (I >= 0 && I < lat_nx(m)); }

static vec2 node_e(const or_mesh *m, const double *phi, const double *walls, int32_t I, int32_t J)
{
    int64_t LL = or_leaf_at(m, I - 1, J - 1), LR = or_leaf_at(m, I, J - 1);
    int64_t UL = or_leaf_at(m, I - 1, J), UR = or_leaf_at(m, I, J);
    /* hanging: the node lies strictly inside an edge of one leaf */
    int64_t q = -1;
    int horizontal = 0;
    if (UL >= 0 && UL == UR) { q = UL; horizontal = 1; }      /* bottom edge of q */
    else if (LL >= 0 && LL == LR) { q = LL; horizontal = 1; } /* top edge of q */
    else if (LL >= 0 && LL == UL) { q = LL; horizontal = 0; } /* right edge of q */
    else if (LR >= 0 && LR == UR) { q = LR; horizontal = 0; } /* left edge of q */
    if (q >= 0) {
        int32_t s = m->s[q];
        int32_t I0, J0, I1, J1;
        if (horizontal) {
            /* the edge's x-range is [ix, ix+s] in the periodic-unwrapped frame of the node */
            int32_t off = ((I - m->ix[q]) % lat_nx(m) + lat_nx(m)) % lat_nx(m);
            I0 = I - off; I1 = I0 + s; J0 = J1 = J;
        } else {
            int32_t off = ((J - m->iy[q]) % lat_ny(m) + lat_ny(m)) % lat_ny(m);
            J0 = J - off; J1 = J0 + s; I0 = I1 = I;
        }
        vec2 a = node_e(m, phi, walls, I0, J0), b = node_e(m, phi, walls, I1, J1);
        vec2 r = {0.5 * (a.ex + b.ex), 0.5 * (a.ey + b.ey)};
        return r;
    }
    double sx = 0.0, sy = 0.0;
    int nxs = 0, nys = 0;
    /* vertical segments (x-normal faces) above and below the node */
    if (in_y(m, J)) { sx += grad_x_at(m, phi, I, J, walls[0], walls[1]); ++nxs; }
    if (in_y(m, J - 1)) { sx += grad_x_at(m, phi, I, J - 1, walls[0], walls[1]); ++nxs; }
    /* horizontal segments (y-normal faces) left and right of the node */
    if (in_x(m, I - 1)) { sy += grad_y_at(m, phi, I - 1, J, walls[2], walls[3]); ++nys; }
    if (in_x(m, I)) { sy += grad_y_at(m, phi, I, J, walls[2], walls[3]); ++nys; }
    vec2 r = {nxs ? -sx / nxs : 0.0, nys ? -sy / nys : 0.0};
    return r;
}

/* Node E at the four corners of every leaf: out[8*l + 2*c + k], corners c = 0:(x0,y0),
 * 1:(x1,y0), 2:(x0,y1), 3:(x1,y1); k = 0: Ex, 1: Ey. */
void or_node_e(const or_mesh *m, const double *phi, const double *walls, double *out)
{
    for (int64_t l = 0; l < m->nleaf; ++l) {
        int32_t ix = m->ix[l], iy = m->iy[l], s = m->s[l];
        for (int c = 0; c < 4; ++c) {
            vec2 e = node_e(m, phi, walls, ix + ((c & 1) ? s : 0), iy + ((c & 2) ? s : 0));
            out[8 * l + 2 * c] = e.ex;
            out[8 * l + 2 * c + 1] = e.ey;
        }
    }
}

/* Cell-centred |E| per leaf from the face gradients (used by the refinement criterion). */
void or_cell_emag(const or_mesh *m, const double *phi, const double *walls, double *out)
{
    for (int64_t l = 0; l < m->nleaf; ++l) {
        int32_t ix = m->ix[l], iy = m->iy[l], s = m->s[l];
        /* mean over the faces on each side of the leaf; a face split into a fine pair is
         * sampled at both halves */
        double gxl, gxr, gyl, gyh;
        gxl = 0.5 * (grad_x_at(m, phi, ix, iy, walls[0], walls[1]) + grad_x_at(m, phi, ix, iy + s - 1, walls[0], walls[1]));
        gxr = 0.5 * (grad_x_at(m, phi, ix + s, iy, walls[0], walls[1]) + grad_x_at(m, phi, ix + s, iy + s - 1, walls[0], walls[1]));
        gyl = 0.5 * (grad_y_at(m, phi, ix, iy, walls[2], walls[3]) + grad_y_at(m, phi, ix + s - 1, iy, walls[2], walls[3]));
        gyh = 0.5 * (grad_y_at(m, phi, ix, iy + s, walls[2], walls[3]) + grad_y_at(m, phi, ix + s - 1, iy + s, walls[2], walls[3]));
        double ex = -0.5 * (gxl + gxr), ey = -0.5 * (gyl + gyh);
        out[l] = sqrt(ex * ex + ey * ey);
    }
}

/* ------------------------------------------------------------------------------------ */
/* Deposit (§3: NGP assignment of the particle charge to cell centres; §3.1: no weighting */
/* for the different cell volumes).  Q_l = sum q w over the leaf's list, in list order.    */
/* ------------------------------------------------------------------------------------ */
void or_deposit(int64_t nleaf, int64_t n, const int64_t *leaf, const double *w, double q, double *Q)
{
    for (int64_t i = 0; i < n; ++i)
        if (leaf[i] >= 0 && leaf[i] < nleaf) Q[leaf[i]] += q * w[i];
}

/* ------------------------------------------------------------------------------------ */
/* Push + boundary + location + Monte Carlo collisions (§3).                              */
/* ------------------------------------------------------------------------------------ */
typedef struct {
    double dt, q, m;
    int32_t species; /* 0: electrons (elastic + ionization); 1: ions (elastic, Maxwellian partner) */
    int32_t mcc;
    double ng, sigma_el, sigma_iz0, eps_th_ev, qe, m_neutral, t_gas_ev;
    uint32_t key0, key1, inst, step;
    double lx, ly;
    /* 0: leapfrog (kick, then drift by the new velocity); 1: the direct implicit scheme's
     * predictor (drift by the old velocity, no kick; collisions off by the caller); 2: its
     * corrector (kick, then drift by the kick's velocity increment times dt) */
    int32_t mode;
} or_push_params;

/* The collision test's uniform: Philox2x32-10 on the counter (id, step), keyed by the seed's */
/* two words, the instance and the id's high word.                                            */
static double draw_test(const or_push_params *p, uint64_t id)
{
    uint32_t ctr[2] = {(uint32_t)id, p->step}, r[2];
    uint32_t key = p->key0 ^ p->key1 ^ (p->inst << 24) ^ (uint32_t)(id >> 32);
    or_philox2x32_10(ctr, key, r);
    return u24(r[0]);
}

static void draw4(const or_push_params *p, uint64_t id, uint32_t purpose, double u[4])
{
    uint32_t ctr[4] = {(uint32_t)id, (uint32_t)(id >> 32) ^ (p->inst << 24), p->step, purpose};
    uint32_t key[2] = {p->key0, p->key1}, r[4];
    or_philox4x32_10(ctr, key, r);
    for (int k = 0; k < 4; ++k) u[k] = u24(r[k]);
}

/* Three standard normals by Box-Muller from the purpose-2 stream. */
static void normals3(const or_push_params *p, uint64_t id, double n[3])
{
    double u[4];
    draw4(p, id, 2, u);
    const double two_pi = 6.283185307179586;
    double r1 = sqrt(-2.0 * log(1.0 - u[0]));
    double r2 = sqrt(-2.0 * log(1.0 - u[2]));
    n[0] = r1 * cos(two_pi * u[1]);
    n[1] = r1 * sin(two_pi * u[1]);
    n[2] = r2 * cos(two_pi * u[3]);
}

static void iso_dir(double uc, double up, double d[3])
{
    const double two_pi = 6.283185307179586;
    double ct = 1.0 - 2.0 * uc;
    double st = sqrt(fmax(0.0, 1.0 - ct * ct));
    double ph = two_pi * up;
    d[0] = st * cos(ph);
    d[1] = st * sin(ph);
    d[2] = ct;
}

/*
 * One species, one step, in list order.  Inputs: positions x^n, velocities v^{n-1/2},
 * leaf of x^n, node E per leaf corner (or_node_e layout).  Outputs in place: v^{n+1/2}
 * (after collisions), x^{n+1}; new_leaf (-1 = absorbed).  Electrons that ionize set
 * spawn[i] = 1 and write the new electron velocity (spawn_v[3i..]) and new ion velocity
 * (spawn_vi[3i..]).  When dec is not NULL it receives the quantities of each particle's
 * collision decisions, dec[4i..4i+3] = (U0, P, U1 sigma_T, sigma_iz): collide iff U0 < P,
 * ionize iff U1 sigma_T < sigma_iz (electrons; ions 0, 0); U0 = -1 where no collision test
 * was made (absorbed particle, collisions off).  When e_part is not NULL it holds each
 * particle's field (ex, ey) at x^n, gathered with a cloud-in-cell shape, and replaces the
 * bilinear corner gather.  Returns the number of ionizations.
 */
int64_t or_push_mcc(const or_mesh *m, const or_push_params *p, const double *node_e_arr,
                    int64_t n, double *x, double *y, double *vx, double *vy, double *vz,
                    const uint64_t *id, const int64_t *leaf, int64_t *new_leaf, uint8_t *spawn,
                    double *spawn_v, double *spawn_vi, double *dec, const double *e_part)
{
    double hf = m->h0 / (double)(1 << m->lmax);
    int64_t nspawn = 0;
    for (int64_t i = 0; i < n; ++i) {
        spawn[i] = 0;
        if (dec) { dec[4 * i] = -1.0; dec[4 * i + 1] = 0.0; dec[4 * i + 2] = 0.0; dec[4 * i + 3] = 0.0; }
        int64_t l = leaf[i];
        double h = m->s[l] * hf;
        double u = (x[i] - m->ix[l] * hf) / h, v = (y[i] - m->iy[l] * hf) / h;
        double ex, ey;
        if (e_part) { /* a cloud-in-cell field gathered beforehand (or_cic_gather) */
            ex = e_part[2 * i];
            ey = e_part[2 * i + 1];
        } else {      /* bilinear over the leaf's corners */
            const double *E = node_e_arr + 8 * l;
            double w00 = (1 - u) * (1 - v), w10 = u * (1 - v), w01 = (1 - u) * v, w11 = u * v;
            ex = w00 * E[0] + w10 * E[2] + w01 * E[4] + w11 * E[6];
            ey = w00 * E[1] + w10 * E[3] + w01 * E[5] + w11 * E[7];
        }
        /* leapfrog kick and drift (the implicit scheme's predictor and corrector: see mode) */
        double qm = p->q / p->m;
        if (p->mode == 1) {
            x[i] += vx[i] * p->dt;
            y[i] += vy[i] * p->dt;
        } else {
            double dvx = qm * ex * p->dt, dvy = qm * ey * p->dt;
            vx[i] += dvx;
            vy[i] += dvy;
            if (p->mode == 2) {
                x[i] += dvx * p->dt;
                y[i] += dvy * p->dt;
            } else {
                x[i] += vx[i] * p->dt;
                y[i] += vy[i] * p->dt;
            }
        }
        /* walls: periodic wrap (modulo the period, however far the particle moved) or
         * absorption; a wrapped position that rounds onto the far wall is the near wall */
        int dead = 0;
        if (x[i] < 0.0 || x[i] >= p->lx) {
            if (m->bc_x == BC_PERIODIC) {
                x[i] -= p->lx * floor(x[i] / p->lx);
                if (x[i] >= p->lx || x[i] < 0.0) x[i] = 0.0;
            } else dead = 1;
        }
        if (y[i] < 0.0 || y[i] >= p->ly) {
            if (m->bc_y == BC_PERIODIC) {
                y[i] -= p->ly * floor(y[i] / p->ly);
                if (y[i] >= p->ly || y[i] < 0.0) y[i] = 0.0;
            } else dead = 1;
        }
        if (dead) { new_leaf[i] = -1; continue; }
        int64_t nl;
        or_locate(m, 1, x + i, y + i, &nl);
        new_leaf[i] = nl;
        if (!p->mcc) continue;

        /* Monte Carlo collision with the background gas */
        /* U[0] decides whether the particle collides; U[1..3] (the purpose-0 4x32 words     */
        /* after the first) decide the branch and the scattering angles                      */
        double U[4];
        draw4(p, id[i], 0, U);
        U[0] = draw_test(p, id[i]);
        if (p->species == 0) {
            double v2 = vx[i] * vx[i] + vy[i] * vy[i] + vz[i] * vz[i];
            double speed = sqrt(v2);
            double eps = 0.5 * p->m * v2 / p->qe; /* eV */
            double s_iz = eps > p->eps_th_ev ? p->sigma_iz0 * (1.0 - p->eps_th_ev / eps) : 0.0;
            double s_t = p->sigma_el + s_iz;
            double P = 1.0 - exp(-p->ng * s_t * speed * p->dt);
            if (dec) { dec[4 * i] = U[0]; dec[4 * i + 1] = P; dec[4 * i + 2] = U[1] * s_t; dec[4 * i + 3] = s_iz; }
            if (!(U[0] < P)) continue;
            if (U[1] * s_t < s_iz) {
                /* ionization: pay the threshold, share the rest, spawn an e-ion pair */
                double rest = eps - p->eps_th_ev;
                double e1 = U[2] * rest, e2 = (1.0 - U[2]) * rest;
                double V[4], d1[3], d2[3], nn[3];
                draw4(p, id[i], 1, V);
                iso_dir(V[0], V[1], d1);
                iso_dir(V[2], V[3], d2);
                double s1 = sqrt(2.0 * e1 * p->qe / p->m), s2 = sqrt(2.0 * e2 * p->qe / p->m);
                vx[i] = s1 * d1[0]; vy[i] = s1 * d1[1]; vz[i] = s1 * d1[2];
                spawn_v[3 * i] = s2 * d2[0]; spawn_v[3 * i + 1] = s2 * d2[1]; spawn_v[3 * i + 2] = s2 * d2[2];
                normals3(p, id[i], nn);
                double vt = sqrt(p->t_gas_ev * p->qe / p->m_neutral);
                spawn_vi[3 * i] = vt * nn[0]; spawn_vi[3 * i + 1] = vt * nn[1]; spawn_vi[3 * i + 2] = vt * nn[2];
                spawn[i] = 1;
                ++nspawn;
            } else {
                /* elastic, isotropic; energy loss 2m/M (1 - cos chi) */
                double d[3];
                iso_dir(U[2], U[3], d);
                double cchi = (vx[i] * d[0] + vy[i] * d[1] + vz[i] * d[2]) / speed;
                double eps2 = eps * (1.0 - 2.0 * p->m / p->m_neutral * (1.0 - cchi));
                double s2 = sqrt(2.0 * eps2 * p->qe / p->m);
                vx[i] = s2 * d[0]; vy[i] = s2 * d[1]; vz[i] = s2 * d[2];
            }
        } else {
            /* ion on a neutral partner drawn from the gas Maxwellian; isotropic in the
             * centre-of-mass frame */
            double nn[3];
            normals3(p, id[i], nn);
            double vt = sqrt(p->t_gas_ev * p->qe / p->m_neutral);
            double vn[3] = {vt * nn[0], vt * nn[1], vt * nn[2]};
            double g[3] = {vx[i] - vn[0], vy[i] - vn[1], vz[i] - vn[2]};
            double gm = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
            double P = 1.0 - exp(-p->ng * p->sigma_el * gm * p->dt);
            if (dec) { dec[4 * i] = U[0]; dec[4 * i + 1] = P; }
            if (!(U[0] < P)) continue;
            double d[3];
            iso_dir(U[2], U[3], d);
            double mt = p->m + p->m_neutral;
            double a = p->m_neutral / mt;
            double vc[3] = {(p->m * vx[i] + p->m_neutral * vn[0]) / mt, (p->m * vy[i] + p->m_neutral * vn[1]) / mt,
                            (p->m * vz[i] + p->m_neutral * vn[2]) / mt};
            vx[i] = vc[0] + a * gm * d[0];
            vy[i] = vc[1] + a * gm * d[1];
            vz[i] = vc[2] + a * gm * d[2];
        }
    }
    return nspawn;
}

/* ------------------------------------------------------------------------------------ */
/* Cloud-in-cell shapes on a uniform mesh (§3: the momentum-conserving CIC-EM and the     */
/* energy-conserving CIC-EC variants on uniform meshes).  nx x ny cells of side h, cell    */
/* (i, j) with its centre at ((i + 1/2) h, (j + 1/2) h), lattice index i + j nx.  A         */
/* particle at x has the reference centre i0 = floor(x / h - 1/2) and the fraction          */
/* fx = x / h - 1/2 - i0: weights 1 - fx and fx on the centres i0 and i0 + 1 (likewise in y, */
/* bilinear in 2D).  A centre beyond a non-periodic wall is replaced by the adjacent cell   */
/* (its weight folds into it, so charge is conserved); periodic directions wrap.            */
/* ------------------------------------------------------------------------------------ */
static int cic_cell(int i, int n, int periodic)
{
    if (periodic) return ((i % n) + n) % n;
    return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

static void cic_weights(double x, double h, int *i0, double *f)
{
    double g = x / h - 0.5;
    double fl = floor(g);
    *i0 = (int)fl;
    *f = g - fl;
}

/* Q[cell] += q w W(cell) for every particle (the charge per unit depth). */
void or_cic_deposit(int nx, int ny, double h, int px, int py, int64_t n, const double *x, const double *y,
                    const double *w, double q, double *Q)
{
    for (int64_t p = 0; p < n; ++p) {
        int i0, j0;
        double fx, fy;
        cic_weights(x[p], h, &i0, &fx);
        cic_weights(y[p], h, &j0, &fy);
        for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) {
                double wt = (a ? fx : 1.0 - fx) * (b ? fy : 1.0 - fy);
                int c = cic_cell(i0 + a, nx, px) + nx * cic_cell(j0 + b, ny, py);
                Q[c] += q * w[p] * wt;
            }
    }
}

/* phi at lattice (i, j) with the Poisson operator's ghost rule outside the walls:
 * periodic wrap; Dirichlet 2 phi_wall - phi_inside; Neumann phi_inside.
 * walls = phi on the x-low, x-high, y-low, y-high walls. */
static double cic_phi(int nx, int ny, int bcx, int bcy, const double *phi, const double *walls, int i, int j)
{
    double add = 0.0, sgn = 1.0;
    if (i < 0 || i >= nx) {
        if (bcx == BC_PERIODIC) i = ((i % nx) + nx) % nx;
        else {
            int in = i < 0 ? 0 : nx - 1;
            if (bcx == BC_DIRICHLET) { add = 2.0 * walls[i < 0 ? 0 : 1]; sgn = -1.0; }
            i = in;
        }
    }
    if (j < 0 || j >= ny) {
        if (bcy == BC_PERIODIC) j = ((j % ny) + ny) % ny;
        else {
            int in = j < 0 ? 0 : ny - 1;
            if (bcy == BC_DIRICHLET) { add += 2.0 * walls[j < 0 ? 2 : 3] * sgn; sgn = -sgn; }
            j = in;
        }
    }
    return add + sgn * phi[i + nx * j];
}

/* E at the particles.  shape 1 (CIC-EM): E at the cell centres by central differences of
 * phi (with the ghost rule), gathered with the particle's CIC weights (folded at walls as in
 * the deposit).  shape 2 (CIC-EC): E = -grad of the bilinear interpolant of phi over the cell
 * centres (ghost values beyond walls) at the particle. */
void or_cic_gather(int nx, int ny, double h, int bcx, int bcy, const double *phi, const double *walls, int shape,
                   int64_t n, const double *x, const double *y, double *ex, double *ey)
{
    int px = bcx == BC_PERIODIC, py = bcy == BC_PERIODIC;
    for (int64_t p = 0; p < n; ++p) {
        int i0, j0;
        double fx, fy;
        cic_weights(x[p], h, &i0, &fx);
        cic_weights(y[p], h, &j0, &fy);
        if (shape == 1) {
            double sx = 0.0, sy = 0.0;
            for (int b = 0; b < 2; ++b)
                for (int a = 0; a < 2; ++a) {
                    double wt = (a ? fx : 1.0 - fx) * (b ? fy : 1.0 - fy);
                    int i = cic_cell(i0 + a, nx, px), j = cic_cell(j0 + b, ny, py);
                    double gx = (cic_phi(nx, ny, bcx, bcy, phi, walls, i + 1, j) -
                                 cic_phi(nx, ny, bcx, bcy, phi, walls, i - 1, j)) / (2.0 * h);
                    double gy = (cic_phi(nx, ny, bcx, bcy, phi, walls, i, j + 1) -
                                 cic_phi(nx, ny, bcx, bcy, phi, walls, i, j - 1)) / (2.0 * h);
                    sx += wt * gx;
                    sy += wt * gy;
                }
            ex[p] = -sx;
            ey[p] = -sy;
        } else {
            double p00 = cic_phi(nx, ny, bcx, bcy, phi, walls, i0, j0);
            double p10 = cic_phi(nx, ny, bcx, bcy, phi, walls, i0 + 1, j0);
            double p01 = cic_phi(nx, ny, bcx, bcy, phi, walls, i0, j0 + 1);
            double p11 = cic_phi(nx, ny, bcx, bcy, phi, walls, i0 + 1, j0 + 1);
            ex[p] = -((1.0 - fy) * (p10 - p00) + fy * (p11 - p01)) / h;
            ey[p] = -((1.0 - fx) * (p01 - p00) + fx * (p11 - p10)) / h;
        }
    }
}
