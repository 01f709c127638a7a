// Particle side of the PIC-MCC cycle (§3, §3.1): NGP deposit, fused gather / leapfrog push /
// wall handling / leaf location / Monte Carlo collisions with electron-ion pair spawning,
// and the cell-list update.
//
// Storage: per species a structure of arrays in cell-list order: offsets (u, v) in [0, 1) of
// the leaf, velocity (vx, vy, vz), weight w in precision R, id as u32.  Leaf L's records are
// the slots [start[L], end[L]) of its segment [start[L], lim[L]); the leaf of a particle is
// implicit.  One warp walks one leaf, so the leaf's corner field and geometry are loaded
// once and broadcast.
//
// Cell-list update (§3.1: a particle that crosses a face leaves its cell's list and is added
// to the neighbour's list): the new list of a leaf is its staying particles in their old
// order, then the entering particles in the order of their old list position, then the
// electron-ion pairs spawned this step in the order of their parents.  One push pass per
// species does it in place: staying records are compacted to the front of their segment at
// their exact rank, entering and spawned records take an atomic free slot of their new
// leaf together with an order key (or the overflow store when the leaf has no free slot
// left, after which the leaf moves to a fresh segment).  A per-leaf sort of the entering
// slots by key then moves them behind the staying records, which makes the result
// deterministic.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "pic_internal.cuh"

namespace gbpic {

namespace {
constexpr int kT = 256;
constexpr int kWarpsPerBlock = kT / 32;
inline unsigned blocks_for(int64_t n, int t = kT) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }
inline unsigned warp_blocks(int64_t nwarps) {
    return (unsigned)std::max<int64_t>(1, std::min<int64_t>((nwarps + kWarpsPerBlock - 1) / kWarpsPerBlock, 1 << 20));
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Math in the state's precision.
__device__ __forceinline__ float m_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double m_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float m_expm1(float x) { return expm1f(x); }
__device__ __forceinline__ double m_expm1(double x) { return expm1(x); }
__device__ __forceinline__ float m_log(float x) { return logf(x); }
__device__ __forceinline__ double m_log(double x) { return log(x); }
__device__ __forceinline__ void m_sincospi(float x, float *s, float *c) { sincospif(x, s, c); }
__device__ __forceinline__ void m_sincospi(double x, double *s, double *c) { sincospi(x, s, c); }
__device__ __forceinline__ float m_floor(float x) { return floorf(x); }
// a / b: FP32 with the fast reciprocal-based division (2 ulp), FP64 correctly rounded
__device__ __forceinline__ float m_div(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double m_div(double a, double b) { return a / b; }
__device__ __forceinline__ double m_floor(double x) { return floor(x); }
template <typename R> __device__ __forceinline__ R below_one();
template <> __device__ __forceinline__ float below_one<float>() { return 0.99999994f; }
template <> __device__ __forceinline__ double below_one<double>() { return 0.99999999999999989; }

template <typename R> __device__ __forceinline__ R u24(uint32_t r) { return (R)(r >> 8) * (R)(1.0 / 16777216.0); }

// Compensated accumulation (Kahan) of one lane, and an error-free combination of the lanes'
// (sum, -compensation) pairs: every lane ends with the same (hi, lo).
template <typename R> __device__ __forceinline__ void kahan_add(R &sum, R &c, R x) {
    const R y = x - c;
    const R t = sum + y;
    c = (t - sum) - y;
    sum = t;
}
template <typename R> __device__ __forceinline__ void warp_two_sum(R &hi, R &lo) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const R oh = __shfl_xor_sync(0xFFFFFFFFu, hi, o), ol = __shfl_xor_sync(0xFFFFFFFFu, lo, o);
        const R t = hi + oh;
        const R bp = t - hi;
        const R err = (hi - (t - bp)) + (oh - bp);
        hi = t;
        lo = lo + ol + err;
    }
}

// ------------------------------------------------------------------------------------
// Deposit (§3 NGP at leaf centres; §3.1 no volume weighting): per leaf
//   charge = sum_s q_s sum_{p in list} w_p   (FP32 Kahan per lane, FP64 across lanes)
//   b      = (charge + rho_bg * area) / eps0 + sum_walls bcw * phi_wall
// ------------------------------------------------------------------------------------
struct DepositArgs {
    int64_t nleaf;
    int nsp;
    const int32_t *start[2], *end[2];
    const void *w[2];
    double q[2];
    const uint8_t *lev;
    int lmax;
    double hf, rho_bg, inv_eps0;
    const double *bcw;
    double wall[4];
    const double *wall_dev;  // non-null: the wall potentials are read from here (captured steps)
    double *charge, *b;
    double *kappa;           // implicit scheme: 1 + chi per leaf, chi = sum_s chi[s] W_s / h^2 (else null)
    double chi[2];           // dt^2 q_s^2 / (m_s eps0)
};

template <typename R>
__global__ void __launch_bounds__(kT) k_deposit(DepositArgs a) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t L = warp; L < a.nleaf; L += nw) {
        double total = 0.0, chi = 0.0;
        for (int s = 0; s < a.nsp; ++s) {
            const int32_t p0 = a.start[s][L], p1 = a.end[s][L];
            const R *w = (const R *)a.w[s];
            R sum = 0, c = 0;
            for (int32_t p = p0 + lane; p < p1; p += 128) {
                R x4[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) x4[k] = p + 32 * k < p1 ? w[p + 32 * k] : (R)0;
#pragma unroll
                for (int k = 0; k < 4; ++k) kahan_add(sum, c, x4[k]);
            }
            R hi = sum, lo = -c;
            warp_two_sum(hi, lo);
            const double Ws = (double)hi + (double)lo;
            total += a.q[s] * Ws;
            chi += a.chi[s] * Ws;
        }
        if (lane == 0) {
            const double h = (double)(1 << (a.lmax - a.lev[L])) * a.hf;
            if (a.kappa) a.kappa[L] = 1.0 + chi / (h * h);
            a.charge[L] = total;
            double bl = (total + a.rho_bg * h * h) * a.inv_eps0;
            for (int k = 0; k < 4; ++k) bl += a.bcw[4 * L + k] * (a.wall_dev ? a.wall_dev[k] : a.wall[k]);
            a.b[L] = bl;
        }
    }
}

// Deposit from the per-leaf weight sums that the last cell-list update left behind: the
// staying particles' compensated sum (hi, lo) from the move pass and the entering particles'
// (hi, lo) from the per-leaf sort, combined here in FP64 with one thread per leaf:
//   w_l = ((double) stay_hi + (double) stay_lo) + ((double) ent_hi + (double) ent_lo).
struct LeafSums {
    const void *stay_hi, *stay_lo, *ent_hi, *ent_lo;
};
template <typename R> __device__ __forceinline__ double leaf_weight(const LeafSums &w, int64_t L) {
    const double st = (double)((const R *)w.stay_hi)[L] + (double)((const R *)w.stay_lo)[L];
    return st + ((double)((const R *)w.ent_hi)[L] + (double)((const R *)w.ent_lo)[L]);
}
template <typename R>
__device__ __forceinline__ void deposit_sums_leaf(const DepositArgs &a, const LeafSums &w0, const LeafSums &w1,
                                                  int64_t L) {
    const double W0 = leaf_weight<R>(w0, L), W1 = a.nsp > 1 ? leaf_weight<R>(w1, L) : 0.0;
    double total = a.q[0] * W0;
    if (a.nsp > 1) total += a.q[1] * W1;
    const double h = (double)(1 << (a.lmax - a.lev[L])) * a.hf;
    if (a.kappa) {
        double chi = a.chi[0] * W0;
        if (a.nsp > 1) chi += a.chi[1] * W1;
        a.kappa[L] = 1.0 + chi / (h * h);
    }
    a.charge[L] = total;
    double bl = (total + a.rho_bg * h * h) * a.inv_eps0;
    for (int k = 0; k < 4; ++k) bl += a.bcw[4 * L + k] * (a.wall_dev ? a.wall_dev[k] : a.wall[k]);
    a.b[L] = bl;
}
template <typename R>
__global__ void k_deposit_sums(DepositArgs a, LeafSums w0, LeafSums w1) {
    const int64_t L = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (L < a.nleaf) deposit_sums_leaf<R>(a, w0, w1, L);
}
// Every instance of an ensemble: block b takes the leaves [c.y, c.z) of instance c.x.
struct DepositEntry {
    DepositArgs a;
    LeafSums w0, w1;
};
template <typename R>
__global__ void k_deposit_sums_batch(const DepositEntry *__restrict__ tab, const int4 *__restrict__ chunks) {
    const int4 c = chunks[blockIdx.x];
    const int64_t L = (int64_t)c.y + threadIdx.x;
    if (L < c.z) deposit_sums_leaf<R>(tab[c.x].a, tab[c.x].w0, tab[c.x].w1, L);
}

// ------------------------------------------------------------------------------------
// Fused gather - push - walls - locate - MCC, updating the cell lists in place.
// ------------------------------------------------------------------------------------
// Where the entering and spawned records of one species go: a free slot of the new leaf,
// else the overflow store (destination leaf and slot kept for the re-layout).
template <typename R> struct ListPut {
    SoA<R> d;
    uint32_t *key, *aux;
    const int32_t *end, *lim;
    int32_t *fill;
    int32_t *moved;  // leaves that ran out of free slots; their count at moved[nleaf]
    int64_t nleaf;
    SoA<R> ovf;
    uint32_t *ovf_key, *ovf_aux;
    int32_t *ovf_dest, *ovf_slot, *ovf_n;
    int32_t ovf_cap;
};

template <typename R>
__device__ __forceinline__ void list_put(const ListPut<R> &o, int32_t L, R u, R v, R vx, R vy, R vz, R w,
                                         uint32_t id, uint32_t key, uint32_t aux, int32_t *err) {
    const int32_t slot = atomicAdd(o.fill + L, 1);
    const int32_t q = o.end[L] + slot;
    const int32_t lim = o.lim[L];
    if (q < lim) {
        o.d.u[q] = u; o.d.v[q] = v; o.d.vx[q] = vx; o.d.vy[q] = vy; o.d.vz[q] = vz; o.d.w[q] = w;
        o.d.id[q] = id;
        o.key[q] = key;
        o.aux[q] = aux;
    } else {
        if (q == lim) o.moved[atomicAdd(o.moved + o.nleaf, 1)] = L;  // first record without a slot
        const int32_t i = atomicAdd(o.ovf_n, 1);
        if (i < o.ovf_cap) {
            o.ovf.u[i] = u; o.ovf.v[i] = v; o.ovf.vx[i] = vx; o.ovf.vy[i] = vy; o.ovf.vz[i] = vz; o.ovf.w[i] = w;
            o.ovf.id[i] = id;
            o.ovf_key[i] = key;
            o.ovf_aux[i] = aux;
            o.ovf_dest[i] = L;
            o.ovf_slot[i] = slot;
        } else {
            atomicExch(err, 1);
        }
    }
}

template <typename R> struct PushArgs {
    int64_t nleaf;
    int lmax, NX, NY;
    int px, py;
    R dth[kMaxLevel + 1];  // dt / h per level
    R qm_dt;               // (q/m) dt
    const int32_t *start, *end, *map, *ix, *iy;
    const int32_t *rank0;      // list rank of each leaf's first record; [nleaf] = species total
    const int32_t *ion_total;  // electrons with ionization: the ion total (spawned ions' keys)
    const uint8_t *lev;
    const R *stencil;
    const R *patch;       // cloud-in-cell shapes: 32 coefficients per leaf
    SoA<R> d;             // this species' lists, updated in place
    ListPut<R> self;      // entering records and spawned electrons of this species
    ListPut<R> ion;       // electrons with ionization: the spawned ions (ion.fill null otherwise)
    int32_t *stay;        // per leaf: staying records
    int32_t *spawn;       // electrons with ionization: per leaf, spawning electrons
    R *stay_hi, *stay_lo; // compensated weight sum of each leaf's staying particles
    int32_t *err;
    int self_wrap;        // some leaf spans a whole periodic direction (a particle may wrap back)
    // collisions
    int mcc, species;
    int drift_kick;  // the implicit scheme's corrector: drift by the kick's increment only
    R ng_dt, sig_el, sig_iz0, eps_th, half_m_over_qe, two_qe_over_m, two_m_over_mn;
    R vt_gas;       // neutral thermal speed sqrt(T qe / M)
    R red_a, red_m, red_mn;  // ions: M / (m + M), m / (m + M), M / (m + M)
    R g_partner_max, g_pad;  // ions: bound on the partner speed (8.2 v_t), rounding margin
    R p_pad;                 // rounding margin of the linear bound on the collision probability
    // the bound test of the pass: electrons sigma_el / sc, sigma_iz0 / sc, (n dt sc p_pad)^2 with
    // sc the larger nonzero cross section scale; ions 1 / (n dt sigma_el g_pad p_pad)
    R bnd_el, bnd_iz, bnd_q, bnd_inv;
    PhiloxKeys keys;    // round keys of the seed
    PhiloxKeys2 keys2;  // the collision test's uniform: Philox2x32-10 keyed by seed and instance
    uint32_t inst_word, step;
    const int64_t *step_dev;  // non-null: the step number is read from here (captured steps)
};

template <typename R> __device__ __forceinline__ void iso_dir(R uc, R up, R d[3]) {
    const R ct = (R)1 - (R)2 * uc;
    R st = (R)1 - ct * ct;
    st = st > (R)0 ? m_sqrt(st) : (R)0;
    R sp, cp;
    m_sincospi((R)2 * up, &sp, &cp);
    d[0] = st * cp; d[1] = st * sp; d[2] = ct;
}

template <typename R> __device__ __forceinline__ void normals3(const U4 &r, R n[3]) {
    const R u0 = u24<R>(r.x), u1 = u24<R>(r.y), u2 = u24<R>(r.z), u3 = u24<R>(r.w);
    const R r1 = m_sqrt((R)-2 * m_log((R)1 - u0)), r2 = m_sqrt((R)-2 * m_log((R)1 - u2));
    R s1, c1, s3, c3;
    m_sincospi((R)2 * u1, &s1, &c1);
    m_sincospi((R)2 * u3, &s3, &c3);
    n[0] = r1 * c1; n[1] = r1 * s1; n[2] = r2 * c3;
}

// Work that only some particles of a warp have, deferred so that it runs 32 particles at a
// time instead of with one or two lanes of a chunk: the location of a particle that left its
// leaf and its list slot there, and every collision beyond the bound test of the pass (the
// exact test, the scattering, the ionization with its pair, the ion's partner draw).  A
// per-warp ring of kQueue entries in shared memory holds them, in list order.
constexpr int kQueue = 64;

template <typename R> struct Queue {
    R a[kQueue], b[kQueue];  // new offsets in the old leaf (a leaver's lie outside [0, 1))
    R vx[kQueue], vy[kQueue], vz[kQueue], w[kQueue];
    uint32_t r0[kQueue];    // collision candidates: the test's uniform word
    uint32_t id[kQueue], key[kQueue], cand[kQueue];
    int32_t L[kQueue], dst[kQueue];  // dst: a stayer's slot, -1 for a leaver
};

// Deferred work of queue entry e; all 32 lanes call it (`valid`: the lane has an entry).
// Electrons that spawn are ranked among their leaf's spawning particles in list order: the
// entries are in list order, and (run_leaf, run_count) carry the count of the last leaf of
// the previous batch, whose entries may continue in this one.
template <typename R>
__device__ __forceinline__ void run_deferred(const PushArgs<R> &a, const Queue<R> &q, int e, bool valid, uint32_t span,
                                             uint32_t ion_span, uint32_t step, int32_t &run_leaf, int32_t &run_count) {
    R vx = 0, vy = 0, vz = 0, w = 0;
    uint32_t id = 0, cand = 0;
    int32_t L = -1, dst = -1;
    if (valid) {
        vx = q.vx[e]; vy = q.vy[e]; vz = q.vz[e]; w = q.w[e];
        id = q.id[e]; cand = q.cand[e];
        L = q.L[e]; dst = q.dst[e];
    }
    // a leaver: the finest-lattice cell of its new position, wrapped or absorbed at the walls
    // (an absorbed particle neither collides nor enters a list)
    R X = 0, Y = 0;
    int32_t I = 0, J = 0;
    bool alive = true;
    if (valid && dst < 0) {
        const int32_t s = 1 << (a.lmax - a.lev[L]);
        X = q.a[e] * (R)s; Y = q.b[e] * (R)s;  // exact: s is a power of two
        I = a.ix[L] + (int32_t)m_floor(X); J = a.iy[L] + (int32_t)m_floor(Y);
        // periodic directions wrap modulo the period, however far the particle moved
        if (I < 0 || I >= a.NX) {
            if (!a.px) alive = false;
            else { I %= a.NX; if (I < 0) I += a.NX; }
        }
        if (J < 0 || J >= a.NY) {
            if (!a.py) alive = false;
            else { J %= a.NY; if (J < 0) J += a.NY; }
        }
        if (!alive) cand = 0;
    }
    R sv[3] = {0, 0, 0}, si[3] = {0, 0, 0};
    bool spawns = false;
    if (cand) {
        const R v2 = vx * vx + vy * vy + vz * vz;
        const R U0 = u24<R>(q.r0[e]);
        const U4 r0 = philox4x32_10(id, a.inst_word, step, 0u, a.keys);  // the other uniforms
        if (a.species == 0) {
            // the exact test, from the same quantities as the bound of the pass
            const R eps = a.half_m_over_qe * v2;
            const R siz = eps > a.eps_th ? a.sig_iz0 * ((R)1 - m_div(a.eps_th, eps)) : (R)0;
            const R st = a.sig_el + siz;
            const R xc = a.ng_dt * st * m_sqrt(v2);
            if (U0 < -m_expm1(-xc)) {
                spawns = u24<R>(r0.y) * st < siz;
                const R speed = m_sqrt(v2);
                const R U2 = u24<R>(r0.z);
                if (spawns) {
                    const R rest = eps - a.eps_th;
                    const R e1 = U2 * rest, e2 = ((R)1 - U2) * rest;
                    const U4 r1 = philox4x32_10(id, a.inst_word, step, 1u, a.keys);
                    R d1[3], d2[3], nn[3];
                    iso_dir<R>(u24<R>(r1.x), u24<R>(r1.y), d1);
                    iso_dir<R>(u24<R>(r1.z), u24<R>(r1.w), d2);
                    const R s1 = m_sqrt(a.two_qe_over_m * e1), s2 = m_sqrt(a.two_qe_over_m * e2);
                    vx = s1 * d1[0]; vy = s1 * d1[1]; vz = s1 * d1[2];
                    sv[0] = s2 * d2[0]; sv[1] = s2 * d2[1]; sv[2] = s2 * d2[2];
                    const U4 r2 = philox4x32_10(id, a.inst_word, step, 2u, a.keys);
                    normals3<R>(r2, nn);
                    si[0] = a.vt_gas * nn[0]; si[1] = a.vt_gas * nn[1]; si[2] = a.vt_gas * nn[2];
                } else {
                    R d[3];
                    iso_dir<R>(U2, u24<R>(r0.w), d);
                    const R cchi = (vx * d[0] + vy * d[1] + vz * d[2]) / speed;
                    const R eps2 = eps * ((R)1 - a.two_m_over_mn * ((R)1 - cchi));
                    const R s2 = m_sqrt(a.two_qe_over_m * eps2);
                    vx = s2 * d[0]; vy = s2 * d[1]; vz = s2 * d[2];
                }
            }
        } else {
            // the partner is drawn and the exact test decides (the test in the pass was a bound)
            const U4 r2 = philox4x32_10(id, a.inst_word, step, 2u, a.keys);
            R nn[3];
            normals3<R>(r2, nn);
            const R vnx = a.vt_gas * nn[0], vny = a.vt_gas * nn[1], vnz = a.vt_gas * nn[2];
            const R gx = vx - vnx, gy = vy - vny, gz = vz - vnz;
            const R gm = m_sqrt(gx * gx + gy * gy + gz * gz);
            const R P = -m_expm1(-a.ng_dt * a.sig_el * gm);
            if (U0 < P) {
                R d[3];
                iso_dir<R>(u24<R>(r0.z), u24<R>(r0.w), d);
                const R cx = a.red_m * vx + a.red_mn * vnx, cy = a.red_m * vy + a.red_mn * vny,
                        cz = a.red_m * vz + a.red_mn * vnz;
                vx = cx + a.red_a * gm * d[0];
                vy = cy + a.red_a * gm * d[1];
                vz = cz + a.red_a * gm * d[2];
            }
        }
    }
    // spawn ranks and per-leaf spawn counts (valid lanes form a prefix of the warp)
    uint32_t rank = 0;
    const uint32_t smask = __ballot_sync(0xFFFFFFFFu, spawns);
    const uint32_t vmask = __ballot_sync(0xFFFFFFFFu, valid);
    const int32_t Llast = __shfl_sync(0xFFFFFFFFu, L, 31 - __clz(vmask));
    const uint32_t same_last = __ballot_sync(0xFFFFFFFFu, valid && L == Llast);
    if (smask) {
        const uint32_t same = __match_any_sync(0xFFFFFFFFu, L);
        const uint32_t before = smask & same & lanemask_lt();
        rank = (L == run_leaf ? (uint32_t)run_count : 0u) + __popc(before);
        if (spawns && before == 0) atomicAdd(a.spawn + L, __popc(smask & same));
    }
    run_count = (Llast == run_leaf ? run_count : 0) + __popc(smask & same_last);
    run_leaf = Llast;
    if (!valid || !alive) return;
    int32_t nl;
    R u, v;
    if (dst >= 0) {  // staying: the record is in place except its velocity
        a.d.vx[dst] = vx; a.d.vy[dst] = vy; a.d.vz[dst] = vz;
        nl = L;
        u = q.a[e]; v = q.b[e];
    } else {         // entering: locate, re-express the offsets in the new leaf, take a slot
        nl = __ldg(a.map + (int64_t)J * a.NX + I);
        const int32_t s2 = 1 << (a.lmax - a.lev[nl]);
        const R inv_s2 = (R)1 / (R)s2;
        // I - floor(X) is the old leaf's corner after the periodic wrap
        R un2 = ((R)(I - (int32_t)m_floor(X) - a.ix[nl]) + X) * inv_s2;
        R vn2 = ((R)(J - (int32_t)m_floor(Y) - a.iy[nl]) + Y) * inv_s2;
        un2 = un2 < (R)0 ? (R)0 : (un2 >= (R)1 ? below_one<R>() : un2);
        vn2 = vn2 < (R)0 ? (R)0 : (vn2 >= (R)1 ? below_one<R>() : vn2);
        u = un2; v = vn2;
        list_put(a.self, nl, u, v, vx, vy, vz, w, id, q.key[e], 0u, a.err);
    }
    if (spawns) {
        // the pair's ids follow from the parent's spawn rank once all leaves are counted:
        // the rank within the parent's leaf travels in the id word, the leaf in the aux word
        list_put(a.self, nl, u, v, sv[0], sv[1], sv[2], w, rank, span + q.key[e], (uint32_t)L, a.err);
        if (a.ion.fill)
            list_put(a.ion, nl, u, v, si[0], si[1], si[2], w, rank, ion_span + q.key[e], (uint32_t)L, a.err);
    }
}

// One warp per leaf (persistent warps).  A staying particle's record goes to slot
// start[L] + its rank among the leaf's staying particles, which is never past its own slot,
// so the leaf's own records are compacted in place; everything the warp reads of the next
// chunk lies beyond every slot it writes in this one.  Entering and spawned records only go
// to free slots past end[], which no warp reads during the pass.
// NT threads per block (a tuned launch shape); 768 threads per SM either way: 80 registers
// (a 64-register build for 1024 threads spills and runs slower).
// CIC: the field is gathered from the leaf's per-quarter cloud-in-cell coefficients (32 per
// leaf, lane k holding coefficient k) instead of the bilinear corner field.
// The warp walks the leaves first, first + nw, ... below last (all lanes call it).
template <typename R, int NT, bool CIC>
__device__ __forceinline__ void push_leaves(const PushArgs<R> &a, Queue<R> &q, const int64_t first, const int64_t last,
                                            const int64_t nw) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = first;
    // order keys: an entering record's list rank before the step; a spawned record's is the
    // species total plus its parent's rank, so it sorts after every entering record
    const uint32_t span = (uint32_t)a.rank0[a.nleaf];
    const uint32_t ion_span = a.ion_total ? (uint32_t)*a.ion_total : 0u;
    const uint32_t step = a.step_dev ? (uint32_t)*a.step_dev : a.step;
    int qhead = 0, qn = 0;  // ring of deferred entries
    int32_t run_leaf = -1, run_count = 0;  // spawn count of the last leaf seen by the deferred work
    // Persistent warps, software-pipelined: the next chunk's records are loaded while this
    // chunk computes, and during a leaf's last chunk that is the first chunk of the warp's
    // next leaf (whose list bounds are fetched when this leaf starts).  The next leaf's slots
    // are disjoint from every slot this warp writes while it finishes this leaf.
    R nu = 0, nv = 0, nvx = 0, nvy = 0, nvz = 0, nwt = 0;
    uint32_t nid = 0;
    auto fetch = [&](int32_t qq) {
        nu = a.d.u[qq]; nv = a.d.v[qq]; nvx = a.d.vx[qq]; nvy = a.d.vy[qq]; nvz = a.d.vz[qq];
        nid = a.d.id[qq]; nwt = a.d.w[qq];
    };
    int32_t np0 = 0, np1 = 0;
    if (warp < last) {
        np0 = a.start[warp]; np1 = a.end[warp];
        if (np0 + lane < np1) fetch(np0 + lane);
    }
    for (int64_t Lw = warp; Lw < last; Lw += nw) {
        const int32_t L = (int32_t)Lw;
        const int32_t p0 = np0, p1 = np1;
        np0 = np1 = 0;
        if (Lw + nw < last) { np0 = a.start[Lw + nw]; np1 = a.end[Lw + nw]; }
        if (p0 == p1) {
            if (lane == 0) {
                a.stay[L] = 0;
                a.stay_hi[L] = (R)0; a.stay_lo[L] = (R)0;
            }
            if (np0 + lane < np1) fetch(np0 + lane);
            continue;
        }
        R ws_sum = 0, ws_c = 0;  // staying particles' weights, in list order per lane
        const uint32_t key0 = (uint32_t)(a.rank0[L] - p0);
        const int lv = a.lev[L];
        const int32_t s = 1 << (a.lmax - lv);
        const int32_t lx = a.ix[L], ly = a.iy[L];
        const R dth = a.dth[lv];
        // the bilinear form in the leaf's corner field, E(u, v) = e0 + u e_u + v (e_v + u e_uv)
        // per component (corners 00, 10, 01, 11 at E[0..1], E[2..3], E[4..5], E[6..7])
        R Bx[4], By[4], pc = 0;
        if constexpr (CIC) {
            pc = a.patch[32 * (int64_t)L + lane];
        } else {
            R E[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) E[k] = a.stencil[8 * (int64_t)L + k];
            Bx[0] = E[0]; Bx[1] = E[2] - E[0]; Bx[2] = E[4] - E[0]; Bx[3] = (E[0] - E[2]) - (E[4] - E[6]);
            By[0] = E[1]; By[1] = E[3] - E[1]; By[2] = E[5] - E[1]; By[3] = (E[1] - E[3]) - (E[5] - E[7]);
        }
        int32_t stay_run = 0;
        for (int32_t c0 = p0; c0 < p1; c0 += 32) {
            const int32_t p = c0 + lane;
            const bool live = p < p1;
            bool stays = false, cand = false;
            R u = nu, v = nv, vx = nvx, vy = nvy, vz = nvz, w = nwt;
            uint32_t id = nid;
            if (p + 32 < p1) fetch(p + 32);
            else if (c0 + 32 >= p1 && np0 + lane < np1) fetch(np0 + lane);
            uint32_t r0x = 0u;
            R ex = 0, ey = 0;
            if constexpr (CIC) {
                // the quarter (qx, qy) of the leaf and the fractions (fx, fy) from its reference
                // cell centre; its 8 coefficients from the lanes that hold them (all lanes
                // take part in the shuffles)
                const int qx = u >= (R)0.5 ? 1 : 0, qy = v >= (R)0.5 ? 1 : 0;
                const R fx = u + (R)0.5 - (R)qx, fy = v + (R)0.5 - (R)qy;
                const int base = 8 * (qx + 2 * qy);
                R c[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) c[t] = __shfl_sync(0xFFFFFFFFu, pc, base + t);
                ex = c[0] + fx * c[1] + fy * (c[2] + fx * c[3]);
                ey = c[4] + fx * c[5] + fy * (c[6] + fx * c[7]);
            }
            if (live) {
                if constexpr (!CIC) {
                    // gather: bilinear in the leaf's corner field
                    ex = Bx[0] + u * Bx[1] + v * (Bx[2] + u * Bx[3]);
                    ey = By[0] + u * By[1] + v * (By[2] + u * By[3]);
                }
                // leapfrog kick and drift in leaf units (the implicit scheme's predictor has no
                // kick; its corrector drifts by the kick's increment)
                const R dvx = a.qm_dt * ex, dvy = a.qm_dt * ey;
                vx += dvx;
                vy += dvy;
                const R un = u + (a.drift_kick ? dvx : vx) * dth, vn = v + (a.drift_kick ? dvy : vy) * dth;
                if (un >= (R)0 && un < (R)1 && vn >= (R)0 && vn < (R)1) {
                    stays = true;
                    u = un; v = vn;
                } else {
                    // a leaver: its new cell, the walls and its list slot are deferred work
                    u = un; v = vn;
                    if (a.self_wrap) {
                        // a leaf as wide as a periodic domain can take its own particle back
                        const R X = un * (R)s, Y = vn * (R)s;  // exact: s is a power of two
                        int32_t I = lx + (int32_t)m_floor(X), J = ly + (int32_t)m_floor(Y);
                        bool in = true;
                        if (I < 0 || I >= a.NX) {
                            if (!a.px) in = false;
                            else { I %= a.NX; if (I < 0) I += a.NX; }
                        }
                        if (J < 0 || J >= a.NY) {
                            if (!a.py) in = false;
                            else { J %= a.NY; if (J < 0) J += a.NY; }
                        }
                        if (in && I >= lx && I < lx + s && J >= ly && J < ly + s) {
                            const R inv = (R)1 / (R)s;
                            R un2 = ((R)(I - (int32_t)m_floor(X) - lx) + X) * inv;
                            R vn2 = ((R)(J - (int32_t)m_floor(Y) - ly) + Y) * inv;
                            u = un2 < (R)0 ? (R)0 : (un2 >= (R)1 ? below_one<R>() : un2);
                            v = vn2 < (R)0 ? (R)0 : (vn2 >= (R)1 ? below_one<R>() : vn2);
                            stays = true;
                        }
                    }
                }
                if (a.mcc) {
                    const R v2 = vx * vx + vy * vy + vz * vz;
                    // the test's uniform: Philox2x32-10 on the counter (id, step); the deferred
                    // work draws the collision's other uniforms from the 4x32 purpose-0 stream
                    r0x = philox2x32_10_x(id, step, a.keys2);
                    const R U0 = u24<R>(r0x);
                    // 1 - exp(-x) <= x: a uniform at or above the bound x (with a rounding
                    // margin) means no collision; below it the deferred work makes the exact test
                    if (a.species == 0) {
                        // x = n dt sigma(eps) |v| with eps sigma(eps) = sc T(eps), squared so that
                        // neither a root nor a division is needed: U0 < x pad iff
                        // (U0 eps)^2 < (n dt sc pad)^2 v^2 T^2 (a zero uniform always goes on)
                        const R eps = a.half_m_over_qe * v2;
                        const R T = a.bnd_el * eps + a.bnd_iz * (eps > a.eps_th ? eps - a.eps_th : (R)0);
                        const R ue = U0 * eps;
                        cand = ue * ue < a.bnd_q * v2 * (T * T) || r0x < 256u;
                    } else {
                        // the Box-Muller partner speed is at most 8.157 v_t (24-bit uniforms):
                        // U0 < B (|v| + g) iff U0 / B - g < 0 or (U0 / B - g)^2 < v^2
                        const R x = U0 * a.bnd_inv - a.g_partner_max;
                        cand = x < (R)0 || x * x < v2;
                    }
                }
            }
            const uint32_t stay_mask = __ballot_sync(0xFFFFFFFFu, live && stays);
            const bool defer = live && (!stays || cand);
            const uint32_t defer_mask = __ballot_sync(0xFFFFFFFFu, defer);
            int32_t dst = -1;
            if (live && stays) {
                dst = p0 + stay_run + __popc(stay_mask & lanemask_lt());
                kahan_add(ws_sum, ws_c, w);
                a.d.u[dst] = u; a.d.v[dst] = v;
                if (!cand) { a.d.vx[dst] = vx; a.d.vy[dst] = vy; a.d.vz[dst] = vz; }
                if (dst != p) { a.d.w[dst] = w; a.d.id[dst] = id; }
            }
            if (defer_mask) {
                if (defer) {
                    const int e = (qhead + qn + __popc(defer_mask & lanemask_lt())) & (kQueue - 1);
                    q.a[e] = u; q.b[e] = v;
                    q.vx[e] = vx; q.vy[e] = vy; q.vz[e] = vz; q.w[e] = w;
                    q.cand[e] = cand ? 1u : 0u;
                    q.r0[e] = r0x;
                    q.id[e] = id; q.key[e] = key0 + (uint32_t)p;
                    q.L[e] = L; q.dst[e] = dst;
                }
                qn += __popc(defer_mask);
                if (qn >= 32) {
                    __syncwarp();
                    run_deferred(a, q, (qhead + lane) & (kQueue - 1), true, span, ion_span, step, run_leaf, run_count);
                    __syncwarp();
                    qhead = (qhead + 32) & (kQueue - 1);
                    qn -= 32;
                }
            }
            stay_run += __popc(stay_mask);
        }
        R hi = ws_sum, lo = -ws_c;
        warp_two_sum(hi, lo);
        if (lane == 0) {
            a.stay[L] = stay_run;
            a.stay_hi[L] = hi; a.stay_lo[L] = lo;
        }
    }
    __syncwarp();
    if (qn > 0) run_deferred(a, q, (qhead + lane) & (kQueue - 1), lane < qn, span, ion_span, step, run_leaf, run_count);
}

// One instance: persistent warps over all its leaves.
template <typename R, int NT, bool CIC>
__global__ void __launch_bounds__(NT, 768 / NT) k_push(const __grid_constant__ PushArgs<R> a) {
    extern __shared__ unsigned char push_smem[];
    Queue<R> &q = reinterpret_cast<Queue<R> *>(push_smem)[threadIdx.x >> 5];
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    push_leaves<R, NT, CIC>(a, q, warp, a.nleaf, nw);
}

// Every instance of an ensemble in one launch: block b takes the leaves [c.y, c.z) of
// instance c.x (c = chunks[b]), the instance's arguments copied to shared memory.
template <typename R, int NT, bool CIC>
__global__ void __launch_bounds__(NT, 768 / NT) k_push_batch(const PushArgs<R> *__restrict__ tab,
                                                             const int4 *__restrict__ chunks) {
    extern __shared__ unsigned char push_smem[];
    __shared__ PushArgs<R> sa;
    const int4 c = chunks[blockIdx.x];
    {
        const uint32_t *src = reinterpret_cast<const uint32_t *>(tab + c.x);
        uint32_t *dst = reinterpret_cast<uint32_t *>(&sa);
        for (int k = threadIdx.x; k < (int)(sizeof(PushArgs<R>) / 4); k += NT) dst[k] = src[k];
    }
    __syncthreads();
    Queue<R> &q = reinterpret_cast<Queue<R> *>(push_smem)[threadIdx.x >> 5];
    push_leaves<R, NT, CIC>(sa, q, (int64_t)c.y + (threadIdx.x >> 5), (int64_t)c.z, NT / 32);
}

__global__ void k_bump_next_id(unsigned long long *next_id, const int32_t *__restrict__ spawn_total) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *next_id += 2ull * (unsigned long long)(*spawn_total);
}

// ------------------------------------------------------------------------------------
// Per-leaf sort of the entering records [end[L], end[L] + n) by order key into their final
// slots [start[L] + stay[L], ...).  A spawned record (key >= span) gets its id here:
// next_id + 2 (spawn rank of its parent) (+ 1 for the ion), the rank being the parent
// leaf's spawn offset (aux word) plus the rank within that leaf (id word).
// ------------------------------------------------------------------------------------
struct SortArgs {
    int64_t nleaf;
    const int32_t *start, *stay, *fill, *lim;
    int32_t *end;
    uint32_t *key, *aux, *tkey, *taux;  // lists' and scratch buffer's key / aux words
    const int32_t *span;                // keys from *span on are spawned records (null: none)
    const int32_t *spawn_base;          // electrons' spawn offsets per parent leaf
    const unsigned long long *next_id;
    uint32_t ion_bit;                   // 1 for the ion list
    void *ent_hi, *ent_lo;              // non-null: the entering weights' compensated sum per leaf (R)
    int32_t *big;                       // long regions for k_sort_big, count at big[nleaf]
    int32_t *med;                       // medium regions for k_sort_medium, count at med[nleaf]
    int32_t *err;
};

// `nid` is *a.next_id, read once per warp (it holds still during the sorts).
__device__ __forceinline__ uint32_t spawn_id(const SortArgs &a, uint32_t span, unsigned long long nid, uint32_t key,
                                             uint32_t aux, uint32_t id) {
    if (key < span) return id;
    return (uint32_t)(nid + 2ull * ((unsigned long long)a.spawn_base[aux] + id) + a.ion_bit);
}

// Entering region of leaf L, or k < 0 when it cannot be (an aborted re-layout).
__device__ __forceinline__ void entering_region(const SortArgs &a, int64_t L, int32_t &b0, int32_t &k,
                                                int32_t &q0) {
    b0 = a.end[L];
    k = a.fill[L];
    q0 = a.start[L] + a.stay[L];
    if (b0 + k > a.lim[L] || q0 > b0) {
        k = -1;
        atomicExch(a.err, 1);
    }
}

constexpr int kSortSmem = 512;  // per-warp shared-memory sort capacity (keys + slots)
constexpr int kSortRegs = 160;  // entering regions up to this long sort in registers

// Sort the k <= 32 P entries at [b0, b0 + k) into [q0, q0 + k) in registers (one warp): lane
// j holds records b0 + j + 32 m; a record's rank is the number of smaller keys (keys are
// distinct), counted against every key broadcast by shuffles.  Every record is in registers
// before any is stored (the region and its destination may overlap).  Each record's key,
// aux word and payload are loaded together (the aux word serves spawned records only), and
// `nid` is the list's next id, read once by the caller.  With `wr` non-null the weights are
// also written there in key order (wr[rank]) for the caller's entering sum.
template <typename R, int P>
__device__ __forceinline__ void sort_region_regs(const SortArgs &a, uint32_t span, unsigned long long nid, int32_t b0,
                                                 int32_t k, int32_t q0, int lane, const SoA<R> &d, R *wr) {
    uint32_t key[P], aux[P], id[P];
    int rank[P];
    R u[P], v[P], vx[P], vy[P], vz[P], w[P];
#pragma unroll
    for (int m = 0; m < P; ++m) {
        const int32_t i = lane + 32 * m;
        const int32_t p = b0 + i;
        const bool act = i < k;
        key[m] = 0xFFFFFFFFu;
        aux[m] = 0;
        rank[m] = 0;
        u[m] = v[m] = vx[m] = vy[m] = vz[m] = w[m] = (R)0;
        id[m] = 0;
        if (act) {
            key[m] = a.key[p]; aux[m] = a.aux[p];
            u[m] = d.u[p]; v[m] = d.v[p]; vx[m] = d.vx[p]; vy[m] = d.vy[p]; vz[m] = d.vz[p]; w[m] = d.w[p];
            id[m] = d.id[p];
        }
    }
#pragma unroll
    for (int m = 0; m < P; ++m)
        if (key[m] >= span && lane + 32 * m < k)
            id[m] = (uint32_t)(nid + 2ull * ((unsigned long long)a.spawn_base[aux[m]] + id[m]) + a.ion_bit);
#pragma unroll
    for (int mm = 0; mm < P; ++mm) {
        const int nj = min(32, k - 32 * mm);  // keys of column mm (warp-uniform)
#pragma unroll 4
        for (int j = 0; j < nj; ++j) {
            const uint32_t o = __shfl_sync(0xFFFFFFFFu, key[mm], j);
#pragma unroll
            for (int m = 0; m < P; ++m) rank[m] += (o < key[m]) ? 1 : 0;
        }
    }
    __syncwarp();
#pragma unroll
    for (int m = 0; m < P; ++m)
        if (lane + 32 * m < k) {
            const int32_t q = q0 + rank[m];
            d.u[q] = u[m]; d.v[q] = v[m]; d.vx[q] = vx[m]; d.vy[q] = vy[m]; d.vz[q] = vz[m]; d.w[q] = w[m];
            d.id[q] = id[m];
            if (wr) wr[rank[m]] = w[m];
        }
    __syncwarp();
}

// Sort the k entries at [b0, b0 + k) into [q0, q0 + k) (one warp).  Up to kSortRegs entries
// sort in registers (their weights also go to `wr` in key order when it is non-null); up to
// 512 by a bitonic network on (key, slot) pairs in the warp's shared memory followed by a
// gather through the scratch buffer `t`.
template <typename R>
__device__ void sort_region(const SortArgs &a, uint32_t span, unsigned long long nid, int32_t b0, int32_t k, int32_t q0,
                            int lane, SoA<R> d, SoA<R> t, unsigned long long *wsm, R *wr) {
    if (k <= 32) { sort_region_regs<R, 1>(a, span, nid, b0, k, q0, lane, d, wr); return; }
    if (k <= 64) { sort_region_regs<R, 2>(a, span, nid, b0, k, q0, lane, d, wr); return; }
    if (k <= 96) { sort_region_regs<R, 3>(a, span, nid, b0, k, q0, lane, d, wr); return; }
    if (k <= 128) { sort_region_regs<R, 4>(a, span, nid, b0, k, q0, lane, d, wr); return; }
    if (k <= kSortRegs) { sort_region_regs<R, 5>(a, span, nid, b0, k, q0, lane, d, wr); return; }
    // copy the region to the scratch buffer
    for (int32_t p = b0 + lane; p < b0 + k; p += 32) {
        t.u[p] = d.u[p]; t.v[p] = d.v[p]; t.vx[p] = d.vx[p]; t.vy[p] = d.vy[p];
        t.vz[p] = d.vz[p]; t.w[p] = d.w[p]; t.id[p] = d.id[p]; a.tkey[p] = a.key[p]; a.taux[p] = a.aux[p];
    }
    __syncwarp();
    int32_t np2 = 64;
    while (np2 < k) np2 <<= 1;
    for (int32_t i = lane; i < np2; i += 32)
        wsm[i] = i < k ? (((unsigned long long)a.tkey[b0 + i] << 32) | (unsigned long long)i) : ~0ull;
    __syncwarp();
    for (int32_t kk = 2; kk <= np2; kk <<= 1) {
        for (int32_t j = kk >> 1; j > 0; j >>= 1) {
            for (int32_t i = lane; i < np2; i += 32) {
                const int32_t ij = i ^ j;
                if (ij > i) {
                    const unsigned long long x = wsm[i], y = wsm[ij];
                    if ((x > y) == ((i & kk) == 0)) { wsm[i] = y; wsm[ij] = x; }
                }
            }
            __syncwarp();
        }
    }
    for (int32_t r = lane; r < k; r += 32) {
        const int32_t p = b0 + (int32_t)(wsm[r] & 0xFFFFFFFFull), q = q0 + r;
        const uint32_t kk = (uint32_t)(wsm[r] >> 32);
        d.u[q] = t.u[p]; d.v[q] = t.v[p]; d.vx[q] = t.vx[p]; d.vy[q] = t.vy[p];
        d.vz[q] = t.vz[p]; d.w[q] = t.w[p];
        d.id[q] = spawn_id(a, span, nid, kk, kk >= span ? a.taux[p] : 0u, t.id[p]);
    }
    __syncwarp();
}

constexpr int kSortBig = 16384;  // one block sorts up to this many entries in shared memory

// Leaves whose entering region is longer than one warp's shared-memory sort: one block per
// leaf, bitonic network on (key, slot) pairs in dynamic shared memory, gather through the
// scratch buffer.  Regions longer than kSortBig rank every key against all others.
template <typename R>
__device__ __forceinline__ void sort_big_leaves(const SortArgs &a, const SoA<R> &d, const SoA<R> &t, int32_t first,
                                                int32_t stride, unsigned long long *bk, R *red_hi, R *red_lo) {
    const uint32_t span = a.span ? (uint32_t)*a.span : 0xFFFFFFFFu;
    const unsigned long long nid = a.span ? *a.next_id : 0ull;
    const int32_t nbig = a.big[a.nleaf];
    for (int32_t li = first; li < nbig; li += stride) {
        const int32_t L = a.big[li];
        int32_t b0, k, q0;
        entering_region(a, L, b0, k, q0);
        if (k < 0) continue;
        for (int32_t p = b0 + threadIdx.x; p < b0 + k; p += blockDim.x) {
            t.u[p] = d.u[p]; t.v[p] = d.v[p]; t.vx[p] = d.vx[p]; t.vy[p] = d.vy[p];
            t.vz[p] = d.vz[p]; t.w[p] = d.w[p]; t.id[p] = d.id[p]; a.tkey[p] = a.key[p]; a.taux[p] = a.aux[p];
        }
        __syncthreads();
        if (k <= kSortBig) {
            int32_t np2 = 1;
            while (np2 < k) np2 <<= 1;
            for (int32_t i = threadIdx.x; i < np2; i += blockDim.x)
                bk[i] = i < k ? (((unsigned long long)a.tkey[b0 + i] << 32) | (unsigned long long)i) : ~0ull;
            __syncthreads();
            for (int32_t kk = 2; kk <= np2; kk <<= 1) {
                for (int32_t j = kk >> 1; j > 0; j >>= 1) {
                    for (int32_t i = threadIdx.x; i < np2; i += blockDim.x) {
                        const int32_t ij = i ^ j;
                        if (ij > i) {
                            const unsigned long long x = bk[i], y = bk[ij];
                            if ((x > y) == ((i & kk) == 0)) { bk[i] = y; bk[ij] = x; }
                        }
                    }
                    __syncthreads();
                }
            }
            for (int32_t r = threadIdx.x; r < k; r += blockDim.x) {
                const int32_t p = b0 + (int32_t)(bk[r] & 0xFFFFFFFFull), q = q0 + r;
                const uint32_t kk = (uint32_t)(bk[r] >> 32);
                d.u[q] = t.u[p]; d.v[q] = t.v[p]; d.vx[q] = t.vx[p]; d.vy[q] = t.vy[p];
                d.vz[q] = t.vz[p]; d.w[q] = t.w[p];
                d.id[q] = spawn_id(a, span, nid, kk, kk >= span ? a.taux[p] : 0u, t.id[p]);
            }
        } else {
            for (int32_t p = b0 + threadIdx.x; p < b0 + k; p += blockDim.x) {
                const uint32_t kk = a.tkey[p];
                int32_t rank = 0;
                for (int32_t j = b0; j < b0 + k; ++j) rank += (a.tkey[j] < kk) ? 1 : 0;
                const int32_t q = q0 + rank;
                d.u[q] = t.u[p]; d.v[q] = t.v[p]; d.vx[q] = t.vx[p]; d.vy[q] = t.vy[p];
                d.vz[q] = t.vz[p]; d.w[q] = t.w[p];
                d.id[q] = spawn_id(a, span, nid, kk, kk >= span ? a.taux[p] : 0u, t.id[p]);
            }
        }
        __syncthreads();
        if (a.ent_hi) {  // entering weights in list order: per-thread Kahan, warps combined in order
            R sum = 0, c = 0;
            for (int32_t q = q0 + threadIdx.x; q < q0 + k; q += blockDim.x) kahan_add(sum, c, d.w[q]);
            R hi = sum, lo = -c;
            warp_two_sum(hi, lo);
            if ((threadIdx.x & 31) == 0) { red_hi[threadIdx.x >> 5] = hi; red_lo[threadIdx.x >> 5] = lo; }
            __syncthreads();
            if (threadIdx.x == 0) {
                double tt = 0.0;
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tt += (double)red_hi[w] + (double)red_lo[w];
                const R th = (R)tt;
                ((R *)a.ent_hi)[L] = th;
                ((R *)a.ent_lo)[L] = (R)(tt - (double)th);
            }
        }
        if (threadIdx.x == 0) a.end[L] = q0 + k;
        __syncthreads();
    }
}

template <typename R>
__global__ void __launch_bounds__(512) k_sort_big(SortArgs a, SoA<R> d, SoA<R> t) {
    extern __shared__ unsigned long long bk[];
    __shared__ R red_hi[16], red_lo[16];
    sort_big_leaves<R>(a, d, t, blockIdx.x, gridDim.x, bk, red_hi, red_lo);
}

constexpr int kSortLane = 8;  // entering regions up to this long are sorted by a leaf's 8-lane group

// Entering regions of every leaf, 8 lanes per leaf (4 leaves per warp pass): a short region
// (k <= kSortLane records) is sorted by its leaf's lane group, lane i holding record b0 + i,
// so that each of the record's arrays is read and written in one contiguous access per leaf;
// every record is in registers before any is written (the region and its destination may
// overlap).  Medium regions (up to kSortSmem) are queued for k_sort_medium, long ones for
// k_sort_big.  Sets end[L] and, with stay sums, the leaf's deposit weight: the staying sum
// plus the entering weights in key order.
// The warp takes the groups of 4 leaves W = first, first + stride, ... with leaves below last.
template <typename R>
__device__ __forceinline__ void sort_entering_groups(const SortArgs &a, const SoA<R> &d, const SoA<R> &t,
                                                     int64_t first, int64_t last, int64_t stride) {
    const uint32_t span = a.span ? (uint32_t)*a.span : 0xFFFFFFFFu;
    const unsigned long long nid = a.span ? *a.next_id : 0ull;
    const int lane = threadIdx.x & 31, g = lane >> 3, gl = lane & 7;
    for (int64_t W = first; W * 4 < last; W += stride) {
        const int64_t L = W * 4 + g;
        const bool has = L < last;
        int32_t b0 = 0, k = 0, q0 = 0;
        if (has && gl == 0) entering_region(a, L, b0, k, q0);
        b0 = __shfl_sync(0xFFFFFFFFu, b0, 0, 8);
        k = __shfl_sync(0xFFFFFFFFu, k, 0, 8);
        q0 = __shfl_sync(0xFFFFFFFFu, q0, 0, 8);
        const bool shortr = has && k >= 0 && k <= kSortLane;
        const bool mine = shortr && gl < k;
        const int32_t p = b0 + gl;
        R u = 0, v = 0, vx = 0, vy = 0, vz = 0, w = 0;
        uint32_t id = 0, key = 0xFFFFFFFFu;
        if (mine) {
            u = d.u[p]; v = d.v[p]; vx = d.vx[p]; vy = d.vy[p]; vz = d.vz[p]; w = d.w[p];
            id = d.id[p];
            key = a.key[p];
            id = spawn_id(a, span, nid, key, key >= span ? a.aux[p] : 0u, id);
        }
        // rank among the group's keys (keys are distinct)
        int r = 0;
#pragma unroll
        for (int j = 0; j < kSortLane; ++j) {
            const uint32_t kj = __shfl_sync(0xFFFFFFFFu, key, j, 8);
            r += (kj < key) ? 1 : 0;
        }
        __syncwarp();  // every load of the warp is done before any store
        if (mine) {
            const int32_t q = q0 + r;
            d.u[q] = u; d.v[q] = v; d.vx[q] = vx; d.vy[q] = vy; d.vz[q] = vz; d.w[q] = w; d.id[q] = id;
        }
        if (a.ent_hi) {
            // the entering weights in key order, summed by the group's first lane; the next
            // deposit combines the pair with the staying sum in FP64, one thread per leaf
            R sum = 0, c = 0;
#pragma unroll
            for (int rr = 0; rr < kSortLane; ++rr) {
                const uint32_t who = (__ballot_sync(0xFFFFFFFFu, mine && r == rr) >> (8 * g)) & 0xFFu;
                const R wr = __shfl_sync(0xFFFFFFFFu, w, who ? __ffs(who) - 1 : 0, 8);
                if (who) kahan_add(sum, c, wr);
            }
            if (shortr && gl == 0) {
                ((R *)a.ent_hi)[L] = sum;
                ((R *)a.ent_lo)[L] = -c;
            }
        }
        if (gl == 0 && has && k >= 0) {
            if (k <= kSortLane) a.end[L] = q0 + k;
            else if (k <= kSortSmem) a.med[atomicAdd(a.med + a.nleaf, 1)] = (int32_t)L;
            else a.big[atomicAdd(a.big + a.nleaf, 1)] = (int32_t)L;
        }
    }
}

template <typename R>
__global__ void __launch_bounds__(kT) k_sort_entering(SortArgs a, SoA<R> d, SoA<R> t) {
    sort_entering_groups<R>(a, d, t, ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5, a.nleaf,
                            ((int64_t)gridDim.x * blockDim.x) >> 5);
}

// Medium entering regions (kSortLane < k <= kSortSmem): one warp per listed leaf; the warp
// takes the list entries first, first + stride, ... below last.  Lane 0 fetches the next
// entry's leaf and region words while the current region is sorted.  A region sorted in
// registers leaves its weights in key order in the warp's shared memory, from which the
// entering sum is taken (the same order and arithmetic as from the sorted list).
template <typename R>
__device__ __forceinline__ void sort_medium_leaves(const SortArgs &a, const SoA<R> &d, const SoA<R> &t, int64_t first,
                                                   int64_t last, int64_t stride, unsigned long long *wsm) {
    const uint32_t span = a.span ? (uint32_t)*a.span : 0xFFFFFFFFu;
    const unsigned long long nid = a.span ? *a.next_id : 0ull;
    const int lane = threadIdx.x & 31;
    const int64_t nmed = min((int64_t)a.med[a.nleaf], last);
    int32_t nL = 0, nb0 = 0, nk = 0, nq0 = 0, nlim = 0;  // lane 0: the next entry's words
    auto fetch = [&](int64_t i) {
        if (lane == 0 && i < nmed) {
            nL = a.med[i];
            nb0 = a.end[nL]; nk = a.fill[nL]; nq0 = a.start[nL] + a.stay[nL]; nlim = a.lim[nL];
        }
    };
    fetch(first);
    R *wr = reinterpret_cast<R *>(wsm);
    for (int64_t i = first; i < nmed; i += stride) {
        int32_t L = nL, b0 = nb0, k = nk, q0 = nq0;
        if (lane == 0 && (b0 + k > nlim || q0 > b0)) {  // an aborted re-layout
            k = -1;
            atomicExch(a.err, 1);
        }
        L = __shfl_sync(0xFFFFFFFFu, L, 0);
        b0 = __shfl_sync(0xFFFFFFFFu, b0, 0);
        k = __shfl_sync(0xFFFFFFFFu, k, 0);
        q0 = __shfl_sync(0xFFFFFFFFu, q0, 0);
        fetch(i + stride);
        const bool staged = a.ent_hi && k <= kSortRegs;
        sort_region<R>(a, span, nid, b0, k, q0, lane, d, t, wsm, staged ? wr : nullptr);
        if (a.ent_hi) {
            if (k <= 16) {
                if (lane == 0) {
                    R sum = 0, c = 0;
                    for (int32_t r = 0; r < k; ++r) kahan_add(sum, c, wr[r]);
                    ((R *)a.ent_hi)[L] = sum;
                    ((R *)a.ent_lo)[L] = -c;
                }
            } else {
                R sum = 0, c = 0;
                for (int32_t r = lane; r < k; r += 32) kahan_add(sum, c, staged ? wr[r] : d.w[q0 + r]);
                R hi = sum, lo = -c;
                warp_two_sum(hi, lo);
                if (lane == 0) {
                    ((R *)a.ent_hi)[L] = hi;
                    ((R *)a.ent_lo)[L] = lo;
                }
            }
        }
        if (lane == 0) a.end[L] = q0 + k;
        __syncwarp();  // the staged weights are read before the next region overwrites them
    }
}

template <typename R>
__global__ void __launch_bounds__(kT, 3) k_sort_medium(SortArgs a, SoA<R> d, SoA<R> t) {
    __shared__ unsigned long long sm_keys[kWarpsPerBlock][kSortSmem];
    sort_medium_leaves<R>(a, d, t, ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5, a.nleaf,
                          ((int64_t)gridDim.x * blockDim.x) >> 5, sm_keys[threadIdx.x >> 5]);
}

// ---- the sorts of every (instance, species) of an ensemble, one launch per pass ----------
template <typename R> struct SortEntry {
    SortArgs a;
    SoA<R> d, t;
};
template <typename T> __device__ __forceinline__ void copy_words(T &dst, const T &src) {
    static_assert(sizeof(T) % 4 == 0, "word copy");
    const uint32_t *s = reinterpret_cast<const uint32_t *>(&src);
    uint32_t *o = reinterpret_cast<uint32_t *>(&dst);
    for (int k = threadIdx.x; k < (int)(sizeof(T) / 4); k += blockDim.x) o[k] = s[k];
}

// Before the entering sorts: the medium and long region lists of every entry are empty.
template <typename R> __global__ void k_sort_prep_batch(const SortEntry<R> *__restrict__ tab, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        tab[i].a.big[tab[i].a.nleaf] = 0;
        tab[i].a.med[tab[i].a.nleaf] = 0;
    }
}
// Block b: the leaves [c.y, c.z) of entry c.x (c.y a multiple of 4).
template <typename R>
__global__ void __launch_bounds__(kT) k_sort_entering_batch(const SortEntry<R> *__restrict__ tab,
                                                            const int4 *__restrict__ chunks) {
    __shared__ SortEntry<R> se;
    const int4 c = chunks[blockIdx.x];
    copy_words(se, tab[c.x]);
    __syncthreads();
    sort_entering_groups<R>(se.a, se.d, se.t, (int64_t)(c.y >> 2) + (threadIdx.x >> 5), (int64_t)c.z, kT / 32);
}
// Block b: the entries [c.y, c.z) of the medium-region list of entry c.x (the list can hold
// every leaf; blocks past its length return at once).
template <typename R>
__global__ void __launch_bounds__(kT, 4) k_sort_medium_batch(const SortEntry<R> *__restrict__ tab,
                                                          const int4 *__restrict__ chunks) {
    __shared__ unsigned long long sm_keys[kWarpsPerBlock][kSortSmem];
    __shared__ SortEntry<R> se;
    const int4 c = chunks[blockIdx.x];
    if (c.y >= tab[c.x].a.med[tab[c.x].a.nleaf]) return;
    copy_words(se, tab[c.x]);
    __syncthreads();
    sort_medium_leaves<R>(se.a, se.d, se.t, (int64_t)c.y + (threadIdx.x >> 5), (int64_t)c.z, kT / 32,
                          sm_keys[threadIdx.x >> 5]);
}
template <typename R>
__global__ void __launch_bounds__(512) k_sort_big_batch(const SortEntry<R> *__restrict__ tab) {
    extern __shared__ unsigned long long bk[];
    __shared__ R red_hi[16], red_lo[16];
    __shared__ SortEntry<R> se;
    copy_words(se, tab[blockIdx.y]);
    __syncthreads();
    sort_big_leaves<R>(se.a, se.d, se.t, blockIdx.x, gridDim.x, bk, red_hi, red_lo);
}

// After the sorts: every ionizing instance's next id moves past its spawned pairs.
struct BumpEntry {
    unsigned long long *next_id;
    const int32_t *spawn_total;
};
__global__ void k_bump_batch(const BumpEntry *__restrict__ tab, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) *tab[i].next_id += 2ull * (unsigned long long)(*tab[i].spawn_total);
}

// ------------------------------------------------------------------------------------
// Load: locate (FP64, floor rule on the finest lattice), slot per leaf, offsets.
// ------------------------------------------------------------------------------------
__global__ void k_locate_load(int64_t n, const double *__restrict__ x, const double *__restrict__ y, double hf,
                              int NX, int NY, const int32_t *__restrict__ map, int32_t *__restrict__ leaf,
                              int32_t *__restrict__ cnt, int32_t *__restrict__ slot, int32_t *__restrict__ err) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double fx = floor(x[i] / hf), fy = floor(y[i] / hf);
    if (!(fx >= 0.0 && fx < (double)NX && fy >= 0.0 && fy < (double)NY)) {
        atomicExch(err, 1);
        leaf[i] = -1;
        return;
    }
    const int32_t l = map[(int64_t)fy * NX + (int64_t)fx];
    leaf[i] = l;
    slot[i] = atomicAdd(cnt + l, 1);
}

// The loaded record i goes to slot q = start[leaf[i]] + slot[i] of its list: perm[q] = i
// (perm spans every slot of the lists, free ones included).
__global__ void k_load_perm(int64_t n, const int32_t *__restrict__ leaf, const int32_t *__restrict__ slot,
                            const int32_t *__restrict__ start, int32_t *__restrict__ perm) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) perm[start[leaf[i]] + slot[i]] = (int32_t)i;
}

// The loaded records in input order, converted to the list's precision with their offsets
// in their leaf, one aligned record of 8 words per particle, (u, v, vx, vy, vz, w) and two
// words of padding (32 bytes in FP32, 64 in FP64), so that the gather below reads one (FP32)
// or two (FP64) DRAM sectors per record.
template <typename R>
__global__ void k_pack_load(int64_t n, const double *__restrict__ x, const double *__restrict__ y,
                            const double *__restrict__ vx, const double *__restrict__ vy,
                            const double *__restrict__ vz, const double *__restrict__ w,
                            const int32_t *__restrict__ leaf, double hf, int lmax, const int32_t *__restrict__ ix,
                            const int32_t *__restrict__ iy, const uint8_t *__restrict__ lev, R *__restrict__ rec) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t l = leaf[i];
    const double h = (double)(1 << (lmax - lev[l])) * hf;
    R u = (R)((x[i] - (double)ix[l] * hf) / h), v = (R)((y[i] - (double)iy[l] * hf) / h);
    u = u < (R)0 ? (R)0 : (u >= (R)1 ? below_one<R>() : u);
    v = v < (R)0 ? (R)0 : (v >= (R)1 ? below_one<R>() : v);
    if constexpr (sizeof(R) == 4) {
        float4 *o = reinterpret_cast<float4 *>(rec + 8 * i);
        o[0] = make_float4(u, v, (float)vx[i], (float)vy[i]);
        o[1] = make_float4((float)vz[i], (float)w[i], 0.0f, 0.0f);
    } else {
        double2 *o = reinterpret_cast<double2 *>(rec + 8 * i);
        o[0] = make_double2(u, v);
        o[1] = make_double2(vx[i], vy[i]);
        o[2] = make_double2(vz[i], w[i]);
    }
}

// One warp per leaf: the leaf's cnt[L] loaded records, gathered from the packed input
// through perm, written to [start[L], start[L] + cnt[L]) with their id (given, or id0 +
// input index) and the input index as the order key.  Every array is written in
// contiguous runs.
template <typename R>
__global__ void k_gather_load(int64_t nleaf, const int32_t *__restrict__ start, const int32_t *__restrict__ cnt,
                              const int32_t *__restrict__ perm, const R *__restrict__ rec,
                              const unsigned long long *__restrict__ id, unsigned long long id0, SoA<R> d,
                              uint32_t *__restrict__ key) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t L = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; L < nleaf; L += nw) {
        const int32_t q0 = start[L], k = cnt[L];
        for (int32_t r = lane; r < k; r += 32) {
            const int32_t q = q0 + r, i = perm[q];
            if constexpr (sizeof(R) == 4) {
                const float4 *o = reinterpret_cast<const float4 *>(rec + 8 * (int64_t)i);
                const float4 A = __ldg(o), B = __ldg(o + 1);
                d.u[q] = A.x; d.v[q] = A.y; d.vx[q] = A.z; d.vy[q] = A.w; d.vz[q] = B.x; d.w[q] = B.y;
            } else {
                const double2 *o = reinterpret_cast<const double2 *>(rec + 8 * (int64_t)i);
                const double2 A = __ldg(o), B = __ldg(o + 1), C = __ldg(o + 2);
                d.u[q] = A.x; d.v[q] = A.y; d.vx[q] = B.x; d.vy[q] = B.y; d.vz[q] = C.x; d.w[q] = C.y;
            }
            d.id[q] = (uint32_t)(id ? id[i] : id0 + (unsigned long long)i);
            key[q] = (uint32_t)i;
        }
    }
}

// Read-back: absolute FP64 positions and leaf index per particle, at the particle's rank in
// the concatenated lists (out0[L] = records before leaf L).
template <typename R>
__global__ void k_read(int64_t nleaf, const int32_t *__restrict__ start, const int32_t *__restrict__ end,
                       const int32_t *__restrict__ out0, double hf, int lmax, const int32_t *__restrict__ ix,
                       const int32_t *__restrict__ iy, const uint8_t *__restrict__ lev, SoA<R> d,
                       double *__restrict__ x, double *__restrict__ y, double *__restrict__ vx,
                       double *__restrict__ vy, double *__restrict__ vz, double *__restrict__ w,
                       unsigned long long *__restrict__ id, uint32_t *__restrict__ leaf) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t L = warp; L < nleaf; L += nw) {
        const double s = (double)(1 << (lmax - lev[L]));
        const int32_t p0 = start[L], o0 = out0[L];
        for (int32_t p = p0 + lane; p < end[L]; p += 32) {
            const int32_t o = o0 + (p - p0);
            x[o] = ((double)ix[L] + (double)d.u[p] * s) * hf;
            y[o] = ((double)iy[L] + (double)d.v[p] * s) * hf;
            vx[o] = (double)d.vx[p]; vy[o] = (double)d.vy[p]; vz[o] = (double)d.vz[p];
            w[o] = (double)d.w[p];
            id[o] = d.id[p];
            leaf[o] = (uint32_t)L;
        }
    }
}

// Order the entering regions of every leaf: the warp-per-leaf pass (short regions, and the
// entering weight sums when a.ent_hi is given), then the long regions (one block each).
template <typename R> void sort_lists(pic_ctx *ctx, SortArgs a, SoA<R> d, SoA<R> t) {
    GB_CUDA(cudaMemsetAsync(a.big + a.nleaf, 0, 4, ctx->stream));
    GB_CUDA(cudaMemsetAsync(a.med + a.nleaf, 0, 4, ctx->stream));
    k_sort_entering<R><<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((a.nleaf + 31) / 32, 152 * 16)), kT, 0,
                         ctx->stream>>>(a, d, t);
    k_sort_medium<R><<<std::min<unsigned>(warp_blocks(a.nleaf), 152u * 8u), kT, 0, ctx->stream>>>(a, d, t);
    const size_t smem = (size_t)kSortBig * sizeof(unsigned long long);
    static bool attr = false;  // per R, set once (not while a step is being captured)
    if (!attr) {
        GB_CUDA(cudaFuncSetAttribute(k_sort_big<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        attr = true;
    }
    k_sort_big<R><<<152, 512, smem, ctx->stream>>>(a, d, t);
    count_launch(ctx, 3);
}

template <typename R> SortArgs sort_args(Instance &in, Species &sp) {
    SortArgs a{};
    a.nleaf = in.nleaf;
    a.start = sp.start; a.stay = sp.stay; a.fill = sp.fill; a.end = sp.end; a.lim = sp.lim;
    a.key = sp.key; a.aux = sp.aux; a.tkey = sp.key + sp.cap; a.taux = sp.aux + sp.cap;
    a.span = nullptr;
    a.spawn_base = nullptr;
    a.next_id = in.d_next_id;
    a.ion_bit = 0;
    a.ent_hi = a.ent_lo = nullptr;
    a.big = sp.big;
    a.med = sp.moved;  // the moved-leaf list is free once the overflow repairs ran
    a.err = in.d_err;
    return a;
}

template <typename R> ListPut<R> list_put_args(Species &sp, int64_t nl) {
    ListPut<R> o{};
    o.d = soa<R>(sp, sp.cur);
    o.key = sp.key; o.aux = sp.aux;
    o.end = sp.end; o.lim = sp.lim;
    o.fill = sp.fill;
    o.moved = sp.moved;
    o.nleaf = nl;
    o.ovf = soa_ovf<R>(sp);
    o.ovf_key = sp.ovf_key; o.ovf_aux = sp.ovf_aux; o.ovf_dest = sp.ovf_dest; o.ovf_slot = sp.ovf_slot;
    o.ovf_n = sp.flags;
    o.ovf_cap = (int32_t)sp.cap;
    return o;
}

template <typename R> PushArgs<R> push_args(Instance &in, int s, int64_t step) {
    const pic_config &c = in.cfg;
    Species &sp = in.sp[s];
    Level &g = in.lv[0];
    PushArgs<R> a{};
    a.nleaf = in.nleaf;
    a.lmax = in.lmax;
    a.NX = in.nx0 << in.lmax;
    a.NY = in.ny0 << in.lmax;
    a.px = c.bc_x == PIC_BC_PERIODIC;
    a.py = c.bc_y == PIC_BC_PERIODIC;
    for (int l = 0; l <= kMaxLevel; ++l) a.dth[l] = (R)(c.dt / (in.h0 / (double)(1 << l)));
    a.qm_dt = (R)(c.q[s] / c.m[s] * c.dt);
    a.start = sp.start; a.end = sp.end;
    a.rank0 = sp.rank0;
    a.ion_total = nullptr;
    a.map = g.map; a.ix = g.ix; a.iy = g.iy; a.lev = g.lev;
    a.stencil = (const R *)in.stencil;
    a.patch = (const R *)in.patch;
    a.d = soa<R>(sp, sp.cur);
    a.self = list_put_args<R>(sp, in.nleaf);
    a.ion = ListPut<R>{};
    a.stay = sp.stay;
    a.spawn = nullptr;
    a.stay_hi = (R *)sp.stay_hi;
    a.stay_lo = (R *)sp.stay_lo;
    a.err = in.d_err;
    a.self_wrap = (a.px && in.nx0 == 1) || (a.py && in.ny0 == 1);
    a.mcc = c.mcc ? 1 : 0;
    a.species = s;
    a.ng_dt = (R)(c.gas_density * c.dt);
    a.sig_el = (R)c.sigma_el;
    a.sig_iz0 = (R)c.sigma_iz0;
    a.eps_th = (R)c.eps_th_ev;
    a.half_m_over_qe = (R)(0.5 * c.m[s] / c.qe);
    a.two_qe_over_m = (R)(2.0 * c.qe / c.m[s]);
    a.two_m_over_mn = (R)(2.0 * c.m[s] / c.neutral_mass);
    a.vt_gas = (R)std::sqrt(c.gas_temperature_ev * c.qe / c.neutral_mass);
    const double mt = c.m[s] + c.neutral_mass;
    a.red_a = (R)(c.neutral_mass / mt);
    a.red_m = (R)(c.m[s] / mt);
    a.red_mn = (R)(c.neutral_mass / mt);
    a.g_partner_max = (R)(8.2 * std::sqrt(c.gas_temperature_ev * c.qe / c.neutral_mass));
    a.g_pad = (R)1.001;
    a.p_pad = (R)1.0001;
    {
        const double sc = c.sigma_el > 0.0 ? c.sigma_el : (c.sigma_iz0 > 0.0 ? c.sigma_iz0 : 1.0);
        const double A = c.gas_density * c.dt * sc * 1.0001;
        a.bnd_el = (R)(c.sigma_el / sc);
        a.bnd_iz = (R)(c.sigma_iz0 / sc);
        a.bnd_q = (R)(A * A);
        const double B = c.gas_density * c.dt * c.sigma_el * 1.001 * 1.0001;
        a.bnd_inv = B > 0.0 ? (R)(1.0 / B) : (R)INFINITY;
    }
    a.keys = philox_keys(c.seed);
    a.inst_word = (uint32_t)c.instance << 24;
    a.keys2 = philox2_keys((uint32_t)(c.seed & 0xFFFFFFFFu) ^ (uint32_t)(c.seed >> 32) ^ a.inst_word);
    a.step = (uint32_t)step;
    a.step_dev = nullptr;
    return a;
}

// The push of species s in a step: with ionization the electrons count their spawns per leaf
// and put the spawned ions into the ion lists.
template <typename R> PushArgs<R> step_push_args(Instance &in, int s, int64_t step, int mode = PUSH_LEAPFROG) {
    PushArgs<R> a = push_args<R>(in, s, step);
    if (mode == PUSH_PREDICT) {  // drift by the old velocity, no kick, no collisions
        a.qm_dt = (R)0;
        a.mcc = 0;
        return a;
    }
    a.drift_kick = mode == PUSH_CORRECT ? 1 : 0;
    const bool ionize = in.cfg.mcc && in.cfg.sigma_iz0 > 0.0;
    if (s == 0 && ionize) {
        a.spawn = in.sp[0].spawn;
        if (in.cfg.n_species > 1) {
            a.ion = list_put_args<R>(in.sp[1], in.nleaf);
            a.ion_total = in.sp[1].rank0 + in.nleaf;
        }
    }
    return a;
}

// The entering sort of species s in a step (spawned records get their ids; the entering
// weight sums feed the next deposit).
template <typename R> SortArgs step_sort_args(Instance &in, int s, int mode = PUSH_LEAPFROG) {
    Species &sp = in.sp[s];
    SortArgs a = sort_args<R>(in, sp);
    if (mode != PUSH_PREDICT && in.cfg.mcc && in.cfg.sigma_iz0 > 0.0) {
        a.span = sp.rank0 + in.nleaf;  // the species total before the step
        a.spawn_base = in.sp[0].spawn_base;
    }
    a.ion_bit = s == 1 ? 1u : 0u;
    a.ent_hi = sp.ent_hi;
    a.ent_lo = sp.ent_lo;
    return a;
}

// Per species before a push: no entering records yet, nothing in the overflow store, no
// moved leaves, the tail not used up, and (electrons with ionization) no spawns counted.
__global__ void k_step_reset(int64_t nl, int32_t *__restrict__ fill, int32_t *__restrict__ flags,
                             int32_t *__restrict__ moved, int32_t *__restrict__ spawn) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nl) {
        fill[i] = 0;
        if (spawn) spawn[i] = 0;
    }
    if (i == 0) {
        flags[0] = 0;
        flags[5] = 0;
        moved[nl] = 0;
    }
}

template <typename R> void step_impl(pic_ctx *ctx, Instance &in, int64_t step, int mode) {
    cudaStream_t st = ctx->stream;
    const int nsp = in.cfg.n_species;
    const int64_t nl = in.nleaf;
    // the push kernel runs persistent warps: as many blocks as are resident at once (or as the
    // tuned share allows), in blocks of 128 or 256 threads (a tuned launch shape)
    const int nt = ctx->tune.push_threads == 128 ? 128 : 256;
    const size_t push_smem = (size_t)(nt / 32) * sizeof(Queue<R>);
    // per process (one device model): resident blocks of [NGP, CIC][128, 256]
    static int resident[2][2] = {{0, 0}, {0, 0}}, sms = 0;
    if (!sms) {
        const size_t sm128 = 4 * sizeof(Queue<R>), sm256 = 8 * sizeof(Queue<R>);
        GB_CUDA(cudaFuncSetAttribute(k_push<R, 128, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm128));
        GB_CUDA(cudaFuncSetAttribute(k_push<R, 256, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm256));
        GB_CUDA(cudaFuncSetAttribute(k_push<R, 128, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm128));
        GB_CUDA(cudaFuncSetAttribute(k_push<R, 256, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm256));
        GB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident[0][0], k_push<R, 128, false>, 128, sm128));
        GB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident[0][1], k_push<R, 256, false>, 256, sm256));
        GB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident[1][0], k_push<R, 128, true>, 128, sm128));
        GB_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident[1][1], k_push<R, 256, true>, 256, sm256));
        for (auto &rr : resident)
            if (rr[0] < 1 || rr[1] < 1) fail(PIC_ECUDA, "push kernel does not fit on an SM");
        int dev = 0;
        GB_CUDA(cudaGetDevice(&dev));
        GB_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    }
    const bool cic = in.cfg.shape != PIC_SHAPE_NGP;
    const int wpb = nt / 32;
    const unsigned wb = (unsigned)std::max<int64_t>(1, (nl + wpb - 1) / wpb);
    int bps = resident[cic ? 1 : 0][nt == 128 ? 0 : 1];
    if (ctx->tune.push_bps > 0) bps = std::min(bps, ctx->tune.push_bps * (256 / nt));  // 256-thread units
    // a captured ensemble step runs instances on parallel branches: a push that takes a
    // share of the GPU lets several instances' pushes run side by side
    const unsigned full = (unsigned)(bps * sms);
    const unsigned pb = std::min<unsigned>(wb, ctx->capturing ? std::max(1u, full / (unsigned)std::max(1, ctx->tune.graph_div)) : full);
    const bool ionize = mode != PUSH_PREDICT && in.cfg.mcc && in.cfg.sigma_iz0 > 0.0;
    Species &e = in.sp[0];
    {
        Phase ph(ctx, PIC_PHASE_LISTS);
        for (int s = 0; s < nsp; ++s) {
            Species &sp = in.sp[s];
            k_step_reset<<<blocks_for(nl), kT, 0, st>>>(nl, sp.fill, sp.flags, sp.moved,
                                                        s == 0 && ionize ? sp.spawn : nullptr);
            count_launch(ctx);
            list_ranks(ctx, sp, nl);
        }
    }
    {
        Phase ph(ctx, PIC_PHASE_MOVE);
        for (int s = 0; s < nsp; ++s) {
            PushArgs<R> a = step_push_args<R>(in, s, step, mode);
            if (ctx->capturing) a.step_dev = ctx->d_step;  // a captured step reads its number on the device
            if (cic) {
                if (nt == 128) k_push<R, 128, true><<<pb, 128, push_smem, st>>>(a);
                else k_push<R, 256, true><<<pb, 256, push_smem, st>>>(a);
            } else {
                if (nt == 128) k_push<R, 128, false><<<pb, 128, push_smem, st>>>(a);
                else k_push<R, 256, false><<<pb, 256, push_smem, st>>>(a);
            }
            count_launch(ctx);
        }
    }
    {
        Phase ph(ctx, PIC_PHASE_SCAN);
        if (ionize) exclusive_scan_i32(ctx, e.spawn, e.spawn_base, nl, e.spawn_base + nl + 1 + scan_scratch_elems(nl));
        for (int s = 0; s < nsp; ++s) place_overflow(ctx, in, s);
    }
    {
        Phase ph(ctx, PIC_PHASE_SORT);
        for (int s = 0; s < nsp; ++s) {
            Species &sp = in.sp[s];
            sort_lists<R>(ctx, step_sort_args<R>(in, s, mode), soa<R>(sp, sp.cur), soa<R>(sp, sp.cur ^ 1));
            sp.sums_valid = true;
        }
        if (ionize) {
            k_bump_next_id<<<1, 32, 0, st>>>(in.d_next_id, e.spawn_base + nl);
            count_launch(ctx);
        }
    }
    check_launch("particle_step");
}

// Give species s `cap` slots per buffer, keeping its lists (records, segments, ends).
void grow_species(pic_ctx *ctx, Instance &in, int s, int64_t cap) {
    Species &sp = in.sp[s];
    if (cap >= (1ll << 31) - 1) fail(PIC_ECAPACITY, "particle slots beyond 2^31");
    const size_t rs = in.cfg.precision == PIC_FP64 ? 8 : 4;
    const int64_t nl = in.nleaf;
    int32_t span = 0;  // first unused slot (segments and the tail)
    GB_CUDA(cudaMemcpyAsync(&span, sp.flags + 4, 4, cudaMemcpyDeviceToHost, ctx->stream));
    GB_CUDA(cudaStreamSynchronize(ctx->stream));
    DeviceArena old = in.part_mem[s];
    Species os = sp;
    in.part_mem[s].blocks.clear();
    species_alloc(ctx, in, s, cap);
    for (int k = 0; k < 6; ++k)
        GB_CUDA(cudaMemcpyAsync(sp.arr[0][k], os.arr[os.cur][k], (size_t)span * rs, cudaMemcpyDeviceToDevice,
                                ctx->stream));
    GB_CUDA(cudaMemcpyAsync(sp.id[0], os.id[os.cur], (size_t)span * 4, cudaMemcpyDeviceToDevice, ctx->stream));
    GB_CUDA(cudaMemcpyAsync(sp.start, os.start, (nl + 1) * 4, cudaMemcpyDeviceToDevice, ctx->stream));
    GB_CUDA(cudaMemcpyAsync(sp.end, os.end, (nl + 1) * 4, cudaMemcpyDeviceToDevice, ctx->stream));
    GB_CUDA(cudaMemcpyAsync(sp.lim, os.lim, (nl + 1) * 4, cudaMemcpyDeviceToDevice, ctx->stream));
    GB_CUDA(cudaMemcpyAsync(sp.spawn_base, os.spawn_base, (nl + 1 + 2 * scan_scratch_elems(nl) + 8) * 4,
                            cudaMemcpyDeviceToDevice, ctx->stream));
    if (os.sums_valid) {
        for (auto pr : {std::make_pair(sp.stay_hi, os.stay_hi), std::make_pair(sp.stay_lo, os.stay_lo),
                        std::make_pair(sp.ent_hi, os.ent_hi), std::make_pair(sp.ent_lo, os.ent_lo)})
            GB_CUDA(cudaMemcpyAsync(pr.first, pr.second, nl * rs, cudaMemcpyDeviceToDevice, ctx->stream));
        sp.sums_valid = true;
    }
    GB_CUDA(cudaMemcpyAsync(sp.flags, os.flags, 8 * 4, cudaMemcpyDeviceToDevice, ctx->stream));  // tail, statistics
    GB_CUDA(cudaStreamSynchronize(ctx->stream));
    sp.n = os.n;
    sp.n_upper = os.n_upper;
    old.release_all();
}

}  // namespace

void walls_at(const Instance &in, int64_t step, double walls[4]) {
    const pic_config &c = in.cfg;
    const double t = (double)step * c.dt;
    walls[0] = c.phi_left_dc + c.phi_left_amp * std::sin(2.0 * M_PI * c.phi_left_freq * t);
    walls[1] = c.phi_right;
    walls[2] = 0.0;
    walls[3] = 0.0;
}

void particles_load(pic_ctx *ctx, Instance &in, int s, int64_t n, const double *x, const double *y,
                    const double *vx, const double *vy, const double *vz, const double *w,
                    const uint64_t *id) {
    cudaStream_t st = ctx->stream;
    Species &sp = in.sp[s];
    const int64_t nl = in.nleaf;
    unsigned long long next_id = 0;
    GB_CUDA(cudaMemcpyAsync(&next_id, in.d_next_id, 8, cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaStreamSynchronize(st));
    if (in.cfg.particle_capacity > 0 && in.cfg.particle_capacity < n)
        fail(PIC_ECAPACITY, "particle_capacity below the loaded population");
    const int64_t cap = in.cfg.particle_capacity > 0 ? slots_for(in.cfg.particle_capacity, nl) : load_slots(n, nl);
    if (cap >= (1ll << 31) - 1) fail(PIC_ECAPACITY, "particle slots beyond 2^31");
    if (id)
        for (int64_t i = 0; i < n; ++i)
            if (id[i] >= (1ull << 32)) fail(PIC_EINVAL, "particle id >= 2^32");
    species_alloc(ctx, in, s, cap);
    DeviceArena tmp(&ctx->cache);
    double *d[6];
    const double *h[6] = {x, y, vx, vy, vz, w};
    for (int k = 0; k < 6; ++k) d[k] = dalloc<double>(tmp, n);
    unsigned long long *did = id && n ? dalloc<unsigned long long>(tmp, n) : nullptr;
    // x and y on the context's stream, the rest on a side stream: the location and the list
    // layout run while the velocities, weights and ids are still copied
    if (!ctx->load_side) {
        GB_CUDA(cudaStreamCreateWithFlags(&ctx->load_side, cudaStreamNonBlocking));
        for (auto &ev : ctx->load_ev) GB_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    }
    cudaStream_t side = ctx->load_side;
    GB_CUDA(cudaEventRecord(ctx->load_ev[0], st));  // the side copies follow what the stream has queued
    GB_CUDA(cudaStreamWaitEvent(side, ctx->load_ev[0], 0));
    if (n) {
        for (int k = 0; k < 2; ++k) GB_CUDA(cudaMemcpyAsync(d[k], h[k], n * 8, cudaMemcpyHostToDevice, st));
        for (int k = 2; k < 6; ++k) GB_CUDA(cudaMemcpyAsync(d[k], h[k], n * 8, cudaMemcpyHostToDevice, side));
        if (did) GB_CUDA(cudaMemcpyAsync(did, id, n * 8, cudaMemcpyHostToDevice, side));
    }
    GB_CUDA(cudaEventRecord(ctx->load_ev[1], side));
    int32_t *leaf = dalloc<int32_t>(tmp, n), *slot = dalloc<int32_t>(tmp, n);
    // perm is indexed by list slot (free slots included, below cap): the scratch buffer's
    // id array holds cap words and is free until the entering sort
    int32_t *perm = reinterpret_cast<int32_t *>(sp.id[1]);
    int32_t *err = dalloc<int32_t>(tmp, 1);
    GB_CUDA(cudaMemsetAsync(err, 0, 4, st));
    GB_CUDA(cudaMemsetAsync(sp.fill, 0, (nl + 1) * 4, st));
    GB_CUDA(cudaMemsetAsync(sp.stay, 0, (nl + 1) * 4, st));
    Level &g = in.lv[0];
    const double hf = in.h0 / (double)(1 << in.lmax);
    if (n) {
        k_locate_load<<<blocks_for(n), kT, 0, st>>>(n, d[0], d[1], hf, in.nx0 << in.lmax, in.ny0 << in.lmax, g.map,
                                                    leaf, sp.fill, slot, err);
        count_launch(ctx);
    }
    int32_t herr = 0;
    GB_CUDA(cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaStreamSynchronize(st));
    if (herr) {
        GB_CUDA(cudaStreamSynchronize(side));  // no copy may still write a released block
        tmp.release_all();
        fail(PIC_EINVAL, "particle position outside the domain");
    }
    // segments with free slots; every loaded record enters its (empty) list: end = start,
    // stay = 0, fill = count, then the entering sort orders each list by input index
    lists_from_counts(ctx, sp, nl, sp.fill, sp.start, sp.end, sp.spawn_base + nl + 1);
    lists_installed(ctx, sp, nl);
    GB_CUDA(cudaMemcpyAsync(sp.end, sp.start, nl * 4, cudaMemcpyDeviceToDevice, st));
    const unsigned long long id0 = id ? 0ull : next_id;
    if (n) {
        k_load_perm<<<blocks_for(n), kT, 0, st>>>(n, leaf, slot, sp.start, perm);
        count_launch(ctx);
    }
    GB_CUDA(cudaStreamWaitEvent(st, ctx->load_ev[1], 0));  // every input array is on the device
    if (n) {
        const unsigned gb = (unsigned)std::min<int64_t>((nl + kT / 32 - 1) / (kT / 32), 152 * 64);
        if (in.cfg.precision == PIC_FP64) {
            double *rec = dalloc<double>(tmp, 8 * n);
            k_pack_load<double><<<blocks_for(n), kT, 0, st>>>(n, d[0], d[1], d[2], d[3], d[4], d[5], leaf, hf, in.lmax,
                                                              g.ix, g.iy, g.lev, rec);
            k_gather_load<double><<<gb, kT, 0, st>>>(nl, sp.start, sp.fill, perm, rec, did, id0, soa<double>(sp, 0),
                                                     sp.key);
        } else {
            float *rec = dalloc<float>(tmp, 8 * n);
            k_pack_load<float><<<blocks_for(n), kT, 0, st>>>(n, d[0], d[1], d[2], d[3], d[4], d[5], leaf, hf, in.lmax,
                                                             g.ix, g.iy, g.lev, rec);
            k_gather_load<float><<<gb, kT, 0, st>>>(nl, sp.start, sp.fill, perm, rec, did, id0, soa<float>(sp, 0),
                                                    sp.key);
        }
        count_launch(ctx, 2);
    }
    if (in.cfg.precision == PIC_FP64)
        sort_lists<double>(ctx, sort_args<double>(in, sp), soa<double>(sp, 0), soa<double>(sp, 1));
    else
        sort_lists<float>(ctx, sort_args<float>(in, sp), soa<float>(sp, 0), soa<float>(sp, 1));
    unsigned long long nid = next_id;
    if (id) {
        for (int64_t i = 0; i < n; ++i) nid = std::max<unsigned long long>(nid, id[i] + 1);
    } else {
        nid = next_id + (unsigned long long)n;
    }
    in.next_id = (int64_t)nid;
    GB_CUDA(cudaMemcpyAsync(in.d_next_id, &nid, 8, cudaMemcpyHostToDevice, st));
    GB_CUDA(cudaStreamSynchronize(st));
    tmp.release_all();
    sp.n = n;
    sp.n_upper = n;
    check_launch("particles_load");
}

void deposit(pic_ctx *ctx, Instance &in, const double walls[4]) {
    if (in.cfg.shape != PIC_SHAPE_NGP) {  // cloud-in-cell (pic_cic.cu)
        cic_deposit(ctx, in, walls);
        return;
    }
    DepositArgs a{};
    a.nleaf = in.nleaf;
    a.nsp = 0;
    for (int s = 0; s < in.cfg.n_species; ++s) {
        if (!in.sp[s].start) continue;
        a.start[a.nsp] = in.sp[s].start;
        a.end[a.nsp] = in.sp[s].end;
        a.w[a.nsp] = in.sp[s].arr[in.sp[s].cur][5];
        a.q[a.nsp] = in.cfg.q[s];
        a.chi[a.nsp] = in.cfg.dt * in.cfg.dt * in.cfg.q[s] * in.cfg.q[s] / (in.cfg.m[s] * in.cfg.eps0);
        ++a.nsp;
    }
    a.kappa = in.cfg.implicit ? in.lv[0].kappa : nullptr;
    a.lev = in.lv[0].lev;
    a.lmax = in.lmax;
    a.hf = in.h0 / (double)(1 << in.lmax);
    a.rho_bg = in.cfg.rho_background;
    a.inv_eps0 = 1.0 / in.cfg.eps0;
    a.bcw = in.lv[0].bcw;
    for (int k = 0; k < 4; ++k) a.wall[k] = walls[k];
    a.wall_dev = ctx->capturing ? in.d_walls : nullptr;  // a captured step: the step's own walls
    a.charge = in.charge;
    a.b = in.bvec;
    bool sums = true;
    for (int s = 0; s < in.cfg.n_species; ++s) sums = sums && in.sp[s].start && in.sp[s].sums_valid;
    if (sums) {
        const Species &s1 = in.sp[in.cfg.n_species > 1 ? 1 : 0];
        const LeafSums w0{in.sp[0].stay_hi, in.sp[0].stay_lo, in.sp[0].ent_hi, in.sp[0].ent_lo};
        const LeafSums w1{s1.stay_hi, s1.stay_lo, s1.ent_hi, s1.ent_lo};
        if (in.cfg.precision == PIC_FP64)
            k_deposit_sums<double><<<blocks_for(in.nleaf), kT, 0, ctx->stream>>>(a, w0, w1);
        else
            k_deposit_sums<float><<<blocks_for(in.nleaf), kT, 0, ctx->stream>>>(a, w0, w1);
    }
    else if (in.cfg.precision == PIC_FP64)
        k_deposit<double><<<warp_blocks(in.nleaf), kT, 0, ctx->stream>>>(a);
    else
        k_deposit<float><<<warp_blocks(in.nleaf), kT, 0, ctx->stream>>>(a);
    count_launch(ctx);
    check_launch("deposit");
    if (in.cfg.implicit) poisson_kappa(ctx, in, walls);  // the operator with this step's susceptibility
}

// Make sure a step cannot overflow the particle buffers: the electron count can at most
// double in one step (every electron ionizes once), the ion count grows by at most that, and
// a re-layout gives every leaf its free slots again.
void ensure_capacity(pic_ctx *ctx, Instance &in) {
    const bool ionize = in.cfg.mcc && in.cfg.sigma_iz0 > 0.0;
    const int nsp = in.cfg.n_species;
    const int64_t nl = in.nleaf;
    auto worst = [&](int s) -> int64_t {
        const int64_t ne = in.sp[0].n_upper;
        if (!ionize) return in.sp[s].n_upper;
        return s == 0 ? 2 * ne : in.sp[s].n_upper + ne;
    };
    const int64_t hard = in.cfg.particle_capacity;
    bool ok = true;
    for (int s = 0; s < nsp; ++s)
        ok = ok && slots_for(worst(s), nl) <= in.sp[s].cap && (hard <= 0 || worst(s) <= hard);
    if (ok) return;
    // exact counts
    count_totals(ctx, in);
    for (int s = 0; s < nsp; ++s)
        GB_CUDA(cudaMemcpyAsync(in.cnt_host + s, in.sp[s].flags + 1, 4, cudaMemcpyDeviceToHost, ctx->stream));
    GB_CUDA(cudaStreamSynchronize(ctx->stream));
    for (int s = 0; s < nsp; ++s) in.sp[s].n = in.sp[s].n_upper = in.cnt_host[s];
    for (int s = 0; s < nsp; ++s) {
        Species &sp = in.sp[s];
        const int64_t need = worst(s);
        if (hard > 0 && need > hard) fail(PIC_ECAPACITY, "particle population would exceed particle_capacity");
        if (slots_for(need, nl) <= sp.cap) continue;
        grow_species(ctx, in, s, std::max<int64_t>(slots_for(2 * need, nl), 2 * sp.cap));
    }
}

// Species s must hold `slots` slots (split/merge, adaptation): grow it if not.
void ensure_slots(pic_ctx *ctx, Instance &in, int s, int64_t slots) {
    Species &sp = in.sp[s];
    if (slots <= sp.cap) return;
    grow_species(ctx, in, s, std::max<int64_t>(slots + slots / 2, 2 * sp.cap));
}

void particle_step(pic_ctx *ctx, Instance &in, int64_t step, bool bookkeeping, int mode) {
    if (in.cfg.precision == PIC_FP64) step_impl<double>(ctx, in, step, mode);
    else step_impl<float>(ctx, in, step, mode);
    if (bookkeeping && mode != PUSH_PREDICT) particle_bookkeeping(in);  // the predictor spawns nothing
}

// Upper bounds of the populations after a step: every electron may have ionized once.
void particle_bookkeeping(Instance &in) {
    const bool ionize = in.cfg.mcc && in.cfg.sigma_iz0 > 0.0;
    if (ionize) {
        const int64_t ne = in.sp[0].n_upper;
        in.sp[0].n_upper = 2 * ne;
        if (in.cfg.n_species > 1) in.sp[1].n_upper += ne;
    }
}

// Exact record totals into sp.n (one sync).
void refresh_counts(pic_ctx *ctx, Instance &in) {
    count_totals(ctx, in);
    for (int s = 0; s < in.cfg.n_species; ++s)
        if (in.sp[s].start)
            GB_CUDA(cudaMemcpyAsync(in.cnt_host + s, in.sp[s].flags + 1, 4, cudaMemcpyDeviceToHost, ctx->stream));
    GB_CUDA(cudaStreamSynchronize(ctx->stream));
    for (int s = 0; s < in.cfg.n_species; ++s)
        if (in.sp[s].start) in.sp[s].n = in.sp[s].n_upper = in.cnt_host[s];
}

void particles_read(pic_ctx *ctx, Instance &in, int s, double *x, double *y, double *vx, double *vy,
                    double *vz, double *w, uint64_t *id, uint32_t *leaf) {
    Species &sp = in.sp[s];
    cudaStream_t st = ctx->stream;
    const int64_t n = sp.n, nl = in.nleaf;
    DeviceArena tmp(&ctx->cache);
    double *d[6];
    for (int k = 0; k < 6; ++k) d[k] = dalloc<double>(tmp, n);
    unsigned long long *did = dalloc<unsigned long long>(tmp, n);
    uint32_t *dleaf = dalloc<uint32_t>(tmp, n);
    list_ranks(ctx, sp, nl);
    const int32_t *out0 = sp.rank0;
    Level &g = in.lv[0];
    const double hf = in.h0 / (double)(1 << in.lmax);
    if (in.cfg.precision == PIC_FP64)
        k_read<double><<<warp_blocks(nl), kT, 0, st>>>(nl, sp.start, sp.end, out0, hf, in.lmax, g.ix, g.iy, g.lev,
                                                       soa<double>(sp, sp.cur), d[0], d[1], d[2], d[3], d[4], d[5],
                                                       did, dleaf);
    else
        k_read<float><<<warp_blocks(nl), kT, 0, st>>>(nl, sp.start, sp.end, out0, hf, in.lmax, g.ix, g.iy, g.lev,
                                                      soa<float>(sp, sp.cur), d[0], d[1], d[2], d[3], d[4], d[5],
                                                      did, dleaf);
    count_launch(ctx);
    double *h[6] = {x, y, vx, vy, vz, w};
    for (int k = 0; k < 6; ++k)
        if (h[k] && n) GB_CUDA(cudaMemcpyAsync(h[k], d[k], n * 8, cudaMemcpyDeviceToHost, st));
    if (id && n) GB_CUDA(cudaMemcpyAsync(id, did, n * 8, cudaMemcpyDeviceToHost, st));
    if (leaf && n) GB_CUDA(cudaMemcpyAsync(leaf, dleaf, n * 4, cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaStreamSynchronize(st));
    tmp.release_all();
    check_launch("particles_read");
}

// ------------------------------------------------------------------------------------
// The batched ensemble step: every instance's particle phases in one launch per phase,
// each block taking a range of leaves of one instance (or (instance, species) entry) from a
// table built here before the step is captured.  Each instance's arithmetic is the one of
// its own step (the same device functions on the same arguments), so a batched instance
// equals the instance run alone bit for bit.
// ------------------------------------------------------------------------------------
namespace {
template <typename R> void batch_prepare_impl(pic_ctx *ctx) {
    BatchStep &B = ctx->batch;
    std::vector<int64_t> nl_inst;
    std::vector<DepositEntry> dep;
    for (Instance &in : ctx->inst) {
        nl_inst.push_back(in.nleaf);
        DepositEntry e{};
        DepositArgs &a = e.a;
        a.nleaf = in.nleaf;
        a.nsp = in.cfg.n_species;
        for (int s = 0; s < a.nsp; ++s) {
            a.start[s] = in.sp[s].start;
            a.end[s] = in.sp[s].end;
            a.w[s] = in.sp[s].arr[in.sp[s].cur][5];
            a.q[s] = in.cfg.q[s];
        }
        a.lev = in.lv[0].lev;
        a.lmax = in.lmax;
        a.hf = in.h0 / (double)(1 << in.lmax);
        a.rho_bg = in.cfg.rho_background;
        a.inv_eps0 = 1.0 / in.cfg.eps0;
        a.bcw = in.lv[0].bcw;
        a.wall_dev = in.d_walls;
        a.charge = in.charge;
        a.b = in.bvec;
        const Species &s1 = in.sp[in.cfg.n_species > 1 ? 1 : 0];
        e.w0 = LeafSums{in.sp[0].stay_hi, in.sp[0].stay_lo, in.sp[0].ent_hi, in.sp[0].ent_lo};
        e.w1 = LeafSums{s1.stay_hi, s1.stay_lo, s1.ent_hi, s1.ent_lo};
        dep.push_back(e);
    }
    std::vector<int4> ch = batch_chunks(nl_inst, kT);
    B.dep.tab = batch_upload(ctx, dep);
    B.dep.chunks = batch_upload(ctx, ch);
    B.dep.n = (int)dep.size();
    B.dep.nchunks = (int)ch.size();

    B.lists = batch_prepare_lists(ctx);

    // pushes: species 0 of every instance, then species 1 of those that have it
    for (int s = 0; s < 2; ++s) {
        std::vector<PushArgs<R>> tab;
        std::vector<int64_t> nls;
        for (Instance &in : ctx->inst) {
            if (s >= in.cfg.n_species) continue;
            PushArgs<R> a = step_push_args<R>(in, s, ctx->step);
            a.step_dev = ctx->d_step;
            tab.push_back(a);
            nls.push_back(in.nleaf);
        }
        B.push[s] = BatchTab{};
        if (tab.empty()) continue;
        ch = batch_chunks(nls, std::max(32, ctx->tune.batch_leaves));
        B.push[s].tab = batch_upload(ctx, tab);
        B.push[s].chunks = batch_upload(ctx, ch);
        B.push[s].n = (int)tab.size();
        B.push[s].nchunks = (int)ch.size();
    }

    // list ranks of every entry; spawn offsets of every ionizing instance
    std::vector<const int32_t *> sin;
    std::vector<int32_t *> sout;
    std::vector<int64_t> sn;
    for (Instance &in : ctx->inst)
        for (int s = 0; s < in.cfg.n_species; ++s) {
            sin.push_back(in.sp[s].inc);
            sout.push_back(in.sp[s].rank0);
            sn.push_back(in.nleaf);
        }
    B.ranks = scan_plan(ctx, sin, sout, sn);
    sin.clear(); sout.clear(); sn.clear();
    std::vector<BumpEntry> bump;
    for (Instance &in : ctx->inst)
        if (in.cfg.mcc && in.cfg.sigma_iz0 > 0.0) {
            sin.push_back(in.sp[0].spawn);
            sout.push_back(in.sp[0].spawn_base);
            sn.push_back(in.nleaf);
            bump.push_back(BumpEntry{in.d_next_id, in.sp[0].spawn_base + in.nleaf});
        }
    B.spawns = scan_plan(ctx, sin, sout, sn);
    B.bump = BatchTab{};
    if (!bump.empty()) {
        B.bump.tab = batch_upload(ctx, bump);
        B.bump.n = (int)bump.size();
    }

    // sorts of every entry
    std::vector<SortEntry<R>> sorts;
    std::vector<int64_t> nls;
    for (Instance &in : ctx->inst)
        for (int s = 0; s < in.cfg.n_species; ++s) {
            Species &sp = in.sp[s];
            sorts.push_back(SortEntry<R>{step_sort_args<R>(in, s), soa<R>(sp, sp.cur), soa<R>(sp, sp.cur ^ 1)});
            nls.push_back(in.nleaf);
        }
    ch = batch_chunks(nls, kT);
    B.sort.tab = batch_upload(ctx, sorts);
    B.sort.chunks = batch_upload(ctx, ch);
    B.sort.n = (int)sorts.size();
    B.sort.nchunks = (int)ch.size();
    ch = batch_chunks(nls, 4 * (kT / 32));  // medium regions: 4 leaves per warp
    B.sort_med.tab = B.sort.tab;
    B.sort_med.chunks = batch_upload(ctx, ch);
    B.sort_med.n = B.sort.n;
    B.sort_med.nchunks = (int)ch.size();
    if (!B.flag) B.flag = (int32_t *)batch_upload(ctx, nullptr, 4 * sizeof(int32_t));

    // shared-memory limits of the batched kernels (set outside the capture)
    const size_t q256 = 8 * sizeof(Queue<R>), q128 = 4 * sizeof(Queue<R>);
    GB_CUDA(cudaFuncSetAttribute(k_push_batch<R, 256, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)q256));
    GB_CUDA(cudaFuncSetAttribute(k_push_batch<R, 128, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)q128));
    GB_CUDA(cudaFuncSetAttribute(k_sort_big_batch<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(kSortBig * sizeof(unsigned long long))));
}

template <typename R> void particle_step_batch_impl(pic_ctx *ctx) {
    BatchStep &B = ctx->batch;
    cudaStream_t st = ctx->stream;
    {
        Phase ph(ctx, PIC_PHASE_LISTS);
        lists_prep_batch(ctx);
        exclusive_scan_i32_batch(ctx, B.ranks);
    }
    {
        Phase ph(ctx, PIC_PHASE_MOVE);
        const int nt = ctx->tune.push_threads == 128 ? 128 : 256;
        const size_t smem = (size_t)(nt / 32) * sizeof(Queue<R>);
        for (int s = 0; s < 2; ++s) {
            const BatchTab &t = B.push[s];
            if (!t.n) continue;
            const PushArgs<R> *tab = (const PushArgs<R> *)t.tab;
            if (nt == 128) k_push_batch<R, 128, false><<<(unsigned)t.nchunks, 128, smem, st>>>(tab, t.chunks);
            else k_push_batch<R, 256, false><<<(unsigned)t.nchunks, 256, smem, st>>>(tab, t.chunks);
            count_launch(ctx);
        }
    }
    {
        Phase ph(ctx, PIC_PHASE_SCAN);
        exclusive_scan_i32_batch(ctx, B.spawns);
        repairs_batch(ctx);
    }
    {
        Phase ph(ctx, PIC_PHASE_SORT);
        const SortEntry<R> *tab = (const SortEntry<R> *)B.sort.tab;
        const unsigned n = (unsigned)B.sort.n;
        k_sort_prep_batch<R><<<(n + kT - 1) / kT, kT, 0, st>>>(tab, (int)n);
        k_sort_entering_batch<R><<<(unsigned)B.sort.nchunks, kT, 0, st>>>(tab, B.sort.chunks);
        k_sort_medium_batch<R><<<(unsigned)B.sort_med.nchunks, kT, 0, st>>>(tab, B.sort_med.chunks);
        k_sort_big_batch<R><<<dim3(2, n), 512, kSortBig * sizeof(unsigned long long), st>>>(tab);
        count_launch(ctx, 4);
        if (B.bump.n) {
            k_bump_batch<<<(unsigned)(B.bump.n + kT - 1) / kT, kT, 0, st>>>((const BumpEntry *)B.bump.tab, B.bump.n);
            count_launch(ctx);
        }
        for (Instance &in : ctx->inst)
            for (int s = 0; s < in.cfg.n_species; ++s) in.sp[s].sums_valid = true;
    }
    check_launch("particle_step_batch");
}
}  // namespace

void batch_prepare_particles(pic_ctx *ctx) {
    if (ctx->inst.front().cfg.precision == PIC_FP64) batch_prepare_impl<double>(ctx);
    else batch_prepare_impl<float>(ctx);
}

void deposit_batch(pic_ctx *ctx) {
    const BatchTab &t = ctx->batch.dep;
    const DepositEntry *tab = (const DepositEntry *)t.tab;
    if (ctx->inst.front().cfg.precision == PIC_FP64)
        k_deposit_sums_batch<double><<<(unsigned)t.nchunks, kT, 0, ctx->stream>>>(tab, t.chunks);
    else
        k_deposit_sums_batch<float><<<(unsigned)t.nchunks, kT, 0, ctx->stream>>>(tab, t.chunks);
    count_launch(ctx);
    check_launch("deposit_batch");
}

void particle_step_batch(pic_ctx *ctx) {
    if (ctx->inst.front().cfg.precision == PIC_FP64) particle_step_batch_impl<double>(ctx);
    else particle_step_batch_impl<float>(ctx);
}

}  // namespace gbpic
