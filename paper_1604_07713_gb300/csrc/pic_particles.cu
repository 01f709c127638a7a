// Particle side of the PIC-MCC cycle (§3, §3.1): NGP deposit, fused gather / leapfrog push /
// wall handling / leaf location / Monte Carlo collisions with electron-ion pair spawning,
// and the cell-list update.
//
// Storage: per species a structure of arrays in cell-list order (leaf by leaf, the order of
// the leaf's list inside): offsets (u, v) in [0, 1) of the leaf, velocity (vx, vy, vz),
// weight w in precision R, id as u32.  The leaf of a particle is implicit in the list offsets
// start[leaf] .. start[leaf + 1].  One warp walks one leaf, so the leaf's corner field and
// geometry are loaded once and broadcast.
//
// Cell-list update (§3.1: a particle that crosses a face leaves its cell's list and is added
// to the neighbour's list): the new list of a leaf is its staying particles in their old
// order, then the entering particles in the order of their old list position, then the
// electron-ion pairs spawned this step in the order of their parents.  It is built in two
// passes over the particles with identical arithmetic: a count pass (per-leaf staying and
// entering counts, spawn counts), prefix sums, a move pass that writes every record to its
// new list (staying: exact rank; entering: an atomic slot plus its order key), and a per-leaf
// sort of the entering slots by key, which makes the result deterministic.
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

template <typename R> struct SoA {
    R *u, *v, *vx, *vy, *vz, *w;
    uint32_t *id;
};
template <typename R> SoA<R> soa(Species &sp, int buf) {
    SoA<R> a;
    a.u = (R *)sp.arr[buf][0]; a.v = (R *)sp.arr[buf][1]; a.vx = (R *)sp.arr[buf][2];
    a.vy = (R *)sp.arr[buf][3]; a.vz = (R *)sp.arr[buf][4]; a.w = (R *)sp.arr[buf][5];
    a.id = sp.id[buf];
    return a;
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
    const int32_t *start[2];
    const void *w[2];
    double q[2];
    const uint8_t *lev;
    int lmax;
    double hf, rho_bg, inv_eps0;
    const double *bcw;
    double wall[4];
    double *charge, *b;
};

template <typename R>
__global__ void __launch_bounds__(kT) k_deposit(DepositArgs a) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t L = warp; L < a.nleaf; L += nw) {
        double total = 0.0;
        for (int s = 0; s < a.nsp; ++s) {
            const int32_t p0 = a.start[s][L], p1 = a.start[s][L + 1];
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
            total += a.q[s] * ((double)hi + (double)lo);
        }
        if (lane == 0) {
            const double h = (double)(1 << (a.lmax - a.lev[L])) * a.hf;
            a.charge[L] = total;
            double bl = (total + a.rho_bg * h * h) * a.inv_eps0;
            for (int k = 0; k < 4; ++k) bl += a.bcw[4 * L + k] * a.wall[k];
            a.b[L] = bl;
        }
    }
}

// Deposit from the per-leaf weight sums that the last cell-list update left behind
// (staying particles summed by the move pass, entering ones by the per-leaf sort).
__global__ void k_deposit_sums(DepositArgs a, const double *__restrict__ ws0, const double *__restrict__ ws1) {
    const int64_t L = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (L >= a.nleaf) return;
    double total = a.q[0] * ws0[L];
    if (a.nsp > 1) total += a.q[1] * ws1[L];
    const double h = (double)(1 << (a.lmax - a.lev[L])) * a.hf;
    a.charge[L] = total;
    double bl = (total + a.rho_bg * h * h) * a.inv_eps0;
    for (int k = 0; k < 4; ++k) bl += a.bcw[4 * L + k] * a.wall[k];
    a.b[L] = bl;
}

// ------------------------------------------------------------------------------------
// Fused gather - push - walls - locate - MCC, in count or move mode.
// ------------------------------------------------------------------------------------
template <typename R> struct PushArgs {
    int64_t nleaf;
    int lmax, NX, NY;
    int px, py;
    R dth[kMaxLevel + 1];  // dt / h per level
    R qm_dt;               // (q/m) dt
    const int32_t *start, *map, *ix, *iy;
    const uint8_t *lev;
    const R *stencil;
    SoA<R> in;
    int mode;  // 0 = count, 1 = move
    // counts (this species)
    int32_t *stay, *inc, *spawn;
    int32_t *inc_ion;  // electrons: entering counts of the ion lists (spawned ions)
    // move
    SoA<R> out;
    uint32_t *key_out;
    const int32_t *start_new, *stay_new;
    int32_t *fill;
    const int32_t *spawn_base;
    const unsigned long long *next_id;
    SoA<R> ion_out;
    uint32_t *ion_key;
    const int32_t *ion_start_new, *ion_stay, *ion_start_old;
    int32_t *ion_fill;
    R *stay_hi, *stay_lo;  // move pass: compensated weight sum of each leaf's staying particles
    int32_t cap, ion_cap;  // record capacity of the output buffers
    int32_t *err;          // set when a write would fall outside them (count/move mismatch)
    // collisions
    int mcc, species;
    R ng_dt, sig_el, sig_iz0, eps_th, half_m_over_qe, two_qe_over_m, two_m_over_mn;
    R vt_gas;       // neutral thermal speed sqrt(T qe / M)
    R red_a, red_m, red_mn;  // ions: M / (m + M), m / (m + M), M / (m + M)
    R g_partner_max, g_pad;  // ions: bound on the partner speed (8.2 v_t), rounding margin
    uint32_t k0, k1, inst_word, step;
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

template <typename R>
__global__ void __launch_bounds__(kT, 4) k_push(PushArgs<R> a) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int32_t n_old = a.start[a.nleaf];
    // persistent warps: the next leaf's list offsets are fetched while this leaf runs
    int32_t np0 = 0, np1 = 0;
    if (warp < a.nleaf) { np0 = a.start[warp]; np1 = a.start[warp + 1]; }
    for (int64_t Lw = warp; Lw < a.nleaf; Lw += nw) {
        const int32_t L = (int32_t)Lw;
        const int32_t p0 = np0, p1 = np1;
        if (Lw + nw < a.nleaf) { np0 = a.start[Lw + nw]; np1 = a.start[Lw + nw + 1]; }
        if (p0 == p1) {
            if (lane == 0) {
                if (a.mode == 0) { a.stay[L] = 0; if (a.spawn) a.spawn[L] = 0; }
                else { a.stay_hi[L] = (R)0; a.stay_lo[L] = (R)0; }
            }
            continue;
        }
        R ws_sum = 0, ws_c = 0;  // staying particles' weights, in list order per lane
        const int lv = a.lev[L];
        const int32_t s = 1 << (a.lmax - lv);
        const int32_t lx = a.ix[L], ly = a.iy[L];
        const R dth = a.dth[lv];
        R E[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) E[k] = a.stencil[8 * (int64_t)L + k];
        int32_t stay_run = 0, spawn_run = 0;
        const int32_t sbase = (a.mode == 1 && a.spawn_base) ? a.spawn_base[L] : 0;
        const int32_t dst0 = a.mode == 1 ? a.start_new[L] : 0;
        // software pipeline: the next chunk's record is loaded while this chunk computes
        R nu = 0, nv = 0, nvx = 0, nvy = 0, nvz = 0, nw = 0;
        uint32_t nid = 0;
        if (p0 + lane < p1) {
            const int32_t q = p0 + lane;
            nu = a.in.u[q]; nv = a.in.v[q]; nvx = a.in.vx[q]; nvy = a.in.vy[q]; nvz = a.in.vz[q];
            nid = a.in.id[q];
            if (a.mode == 1) nw = a.in.w[q];
        }
        for (int32_t c0 = p0; c0 < p1; c0 += 32) {
            const int32_t p = c0 + lane;
            const bool live = p < p1;
            bool alive = false, stays = false, spawns = false;
            int32_t nl = -1;
            R u = nu, v = nv, vx = nvx, vy = nvy, vz = nvz, w = nw;
            uint32_t id = nid;
            if (p + 32 < p1) {
                const int32_t q = p + 32;
                nu = a.in.u[q]; nv = a.in.v[q]; nvx = a.in.vx[q]; nvy = a.in.vy[q]; nvz = a.in.vz[q];
                nid = a.in.id[q];
                if (a.mode == 1) nw = a.in.w[q];
            }
            R sv[3] = {0, 0, 0}, si[3] = {0, 0, 0};
            if (live) {
                // gather: bilinear in the leaf's corner field
                const R w00 = ((R)1 - u) * ((R)1 - v), w10 = u * ((R)1 - v), w01 = ((R)1 - u) * v, w11 = u * v;
                const R ex = w00 * E[0] + w10 * E[2] + w01 * E[4] + w11 * E[6];
                const R ey = w00 * E[1] + w10 * E[3] + w01 * E[5] + w11 * E[7];
                // leapfrog kick and drift in leaf units
                vx += a.qm_dt * ex;
                vy += a.qm_dt * ey;
                R un = u + vx * dth, vn = v + vy * dth;
                alive = true;
                if (un >= (R)0 && un < (R)1 && vn >= (R)0 && vn < (R)1) {
                    stays = true;
                    nl = L;
                    u = un; v = vn;
                } else {
                    // locate on the finest lattice relative to this leaf, then re-express
                    const R X = un * (R)s, Y = vn * (R)s;  // exact: s is a power of two
                    const R fx = m_floor(X), fy = m_floor(Y);
                    int32_t I = lx + (int32_t)fx, J = ly + (int32_t)fy;
                    int32_t wx = 0, wy = 0;
                    if (I < 0 || I >= a.NX) {
                        if (!a.px) alive = false;
                        else { wx = I < 0 ? a.NX : -a.NX; I += wx; if (I < 0 || I >= a.NX) alive = false; }
                    }
                    if (J < 0 || J >= a.NY) {
                        if (!a.py) alive = false;
                        else { wy = J < 0 ? a.NY : -a.NY; J += wy; if (J < 0 || J >= a.NY) alive = false; }
                    }
                    if (alive) {
                        nl = __ldg(a.map + (int64_t)J * a.NX + I);
                        const int32_t s2 = 1 << (a.lmax - a.lev[nl]);
                        const R inv_s2 = (R)1 / (R)s2;
                        R un2 = ((R)(lx + wx - a.ix[nl]) + X) * inv_s2;
                        R vn2 = ((R)(ly + wy - a.iy[nl]) + Y) * inv_s2;
                        un2 = un2 < (R)0 ? (R)0 : (un2 >= (R)1 ? below_one<R>() : un2);
                        vn2 = vn2 < (R)0 ? (R)0 : (vn2 >= (R)1 ? below_one<R>() : vn2);
                        u = un2; v = vn2;
                        stays = nl == L;
                    }
                }
                // The count pass only needs the spawn decisions, which only electrons above the
                // ionization threshold can make; the move pass runs every collision.  v2 and eps
                // are computed once so both passes take the identical decision.
                const R v2 = vx * vx + vy * vy + vz * vz;
                const R eps = a.half_m_over_qe * v2;
                const bool collide_here = a.mode == 1 || (a.species == 0 && a.sig_iz0 > (R)0 && eps > a.eps_th);
                if (alive && a.mcc && collide_here) {
                    const U4 r0 = philox4x32_10(id, a.inst_word, a.step, 0u, a.k0, a.k1);
                    const R U0 = u24<R>(r0.x), U1 = u24<R>(r0.y), U2 = u24<R>(r0.z), U3 = u24<R>(r0.w);
                    if (a.species == 0) {
                        const R speed = m_sqrt(v2);
                        const R siz = eps > a.eps_th ? a.sig_iz0 * ((R)1 - a.eps_th / eps) : (R)0;
                        const R st = a.sig_el + siz;
                        const R P = -m_expm1(-a.ng_dt * st * speed);
                        if (U0 < P) {
                            if (U1 * st < siz) {
                                const R rest = eps - a.eps_th;
                                const R e1 = U2 * rest, e2 = ((R)1 - U2) * rest;
                                const U4 r1 = philox4x32_10(id, a.inst_word, a.step, 1u, a.k0, a.k1);
                                R d1[3], d2[3], nn[3];
                                iso_dir<R>(u24<R>(r1.x), u24<R>(r1.y), d1);
                                iso_dir<R>(u24<R>(r1.z), u24<R>(r1.w), d2);
                                const R s1 = m_sqrt(a.two_qe_over_m * e1), s2 = m_sqrt(a.two_qe_over_m * e2);
                                vx = s1 * d1[0]; vy = s1 * d1[1]; vz = s1 * d1[2];
                                sv[0] = s2 * d2[0]; sv[1] = s2 * d2[1]; sv[2] = s2 * d2[2];
                                const U4 r2 = philox4x32_10(id, a.inst_word, a.step, 2u, a.k0, a.k1);
                                normals3<R>(r2, nn);
                                si[0] = a.vt_gas * nn[0]; si[1] = a.vt_gas * nn[1]; si[2] = a.vt_gas * nn[2];
                                spawns = true;
                            } else {
                                R d[3];
                                iso_dir<R>(U2, U3, d);
                                const R cchi = (vx * d[0] + vy * d[1] + vz * d[2]) / speed;
                                const R eps2 = eps * ((R)1 - a.two_m_over_mn * ((R)1 - cchi));
                                const R s2 = m_sqrt(a.two_qe_over_m * eps2);
                                vx = s2 * d[0]; vy = s2 * d[1]; vz = s2 * d[2];
                            }
                        }
                    } else if (U0 < -m_expm1(-a.ng_dt * a.sig_el * a.g_pad *
                                             (m_sqrt(vx * vx + vy * vy + vz * vz) + a.g_partner_max))) {
                        // The Box-Muller partner speed is at most 8.157 v_t (24-bit uniforms), so
                        // U0 above the probability at |v| + that bound already means no collision;
                        // below it, the partner is drawn and the exact test decides.
                        const U4 r2 = philox4x32_10(id, a.inst_word, a.step, 2u, a.k0, a.k1);
                        R nn[3];
                        normals3<R>(r2, nn);
                        const R vnx = a.vt_gas * nn[0], vny = a.vt_gas * nn[1], vnz = a.vt_gas * nn[2];
                        const R gx = vx - vnx, gy = vy - vny, gz = vz - vnz;
                        const R gm = m_sqrt(gx * gx + gy * gy + gz * gz);
                        const R P = -m_expm1(-a.ng_dt * a.sig_el * gm);
                        if (U0 < P) {
                            R d[3];
                            iso_dir<R>(U2, U3, d);
                            const R cx = a.red_m * vx + a.red_mn * vnx, cy = a.red_m * vy + a.red_mn * vny,
                                    cz = a.red_m * vz + a.red_mn * vnz;
                            vx = cx + a.red_a * gm * d[0];
                            vy = cy + a.red_a * gm * d[1];
                            vz = cz + a.red_a * gm * d[2];
                        }
                    }
                }
            }
            const uint32_t stay_mask = __ballot_sync(0xFFFFFFFFu, live && alive && stays);
            const uint32_t spawn_mask = __ballot_sync(0xFFFFFFFFu, live && spawns);
            const bool enters = live && alive && !stays;
            if (a.mode == 0) {
                // entering particles and spawned pairs: per-destination counts
                if (enters || spawns) {
                    const uint32_t grp = __match_any_sync(__activemask(), nl);
                    const int nent = __popc(__ballot_sync(grp, enters));
                    const int nsp = __popc(__ballot_sync(grp, spawns));
                    if ((__ffs(grp) - 1) == lane) {
                        if (nent + nsp) atomicAdd(a.inc + nl, nent + nsp);
                        if (nsp && a.inc_ion) atomicAdd(a.inc_ion + nl, nsp);
                    }
                }
                stay_run += __popc(stay_mask);
                spawn_run += __popc(spawn_mask);
            } else {
                if (live && alive) {
                    int32_t dst;
                    if (stays) {
                        dst = dst0 + stay_run + __popc(stay_mask & lanemask_lt());
                    } else {
                        const int32_t slot = atomicAdd(a.fill + nl, 1);
                        dst = a.start_new[nl] + a.stay_new[nl] + slot;
                        if (dst >= 0 && dst < a.cap) a.key_out[dst] = (uint32_t)p;
                    }
                    if (dst < 0 || dst >= a.cap) { atomicExch(a.err, 1); dst = -1; }
                    if (stays) kahan_add(ws_sum, ws_c, w);
                    if (dst >= 0) {
                    a.out.u[dst] = u; a.out.v[dst] = v;
                    a.out.vx[dst] = vx; a.out.vy[dst] = vy; a.out.vz[dst] = vz;
                    a.out.w[dst] = w; a.out.id[dst] = id;
                    }
                }
                if (spawns) {
                    const int32_t rank = sbase + spawn_run + __popc(spawn_mask & lanemask_lt());
                    const unsigned long long base = *a.next_id + 2ull * (unsigned long long)rank;
                    const int32_t slot = atomicAdd(a.fill + nl, 1);
                    const int32_t dst = a.start_new[nl] + a.stay_new[nl] + slot;
                    if (dst < 0 || dst >= a.cap) {
                        atomicExch(a.err, 1);
                    } else {
                        a.key_out[dst] = (uint32_t)(n_old + p);
                        a.out.u[dst] = u; a.out.v[dst] = v;
                        a.out.vx[dst] = sv[0]; a.out.vy[dst] = sv[1]; a.out.vz[dst] = sv[2];
                        a.out.w[dst] = w; a.out.id[dst] = (uint32_t)base;
                    }
                    if (a.ion_fill) {
                        const int32_t islot = atomicAdd(a.ion_fill + nl, 1);
                        const int32_t idst = a.ion_start_new[nl] + a.ion_stay[nl] + islot;
                        if (idst < 0 || idst >= a.ion_cap) {
                            atomicExch(a.err, 1);
                        } else {
                        a.ion_key[idst] = (uint32_t)(a.ion_start_old[a.nleaf] + p);
                        a.ion_out.u[idst] = u; a.ion_out.v[idst] = v;
                        a.ion_out.vx[idst] = si[0]; a.ion_out.vy[idst] = si[1]; a.ion_out.vz[idst] = si[2];
                        a.ion_out.w[idst] = w; a.ion_out.id[idst] = (uint32_t)(base + 1);
                        }
                    }
                }
                stay_run += __popc(stay_mask);
                spawn_run += __popc(spawn_mask);
            }
        }
        if (a.mode == 0 && lane == 0) {
            a.stay[L] = stay_run;
            if (a.spawn) a.spawn[L] = spawn_run;
        }
        if (a.mode == 1) {
            R hi = ws_sum, lo = -ws_c;
            warp_two_sum(hi, lo);
            if (lane == 0) { a.stay_hi[L] = hi; a.stay_lo[L] = lo; }
        }
    }
}

__global__ void k_add_counts(int64_t n, const int32_t *__restrict__ a, int32_t *__restrict__ b) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = a[i] + b[i];
}

__global__ void k_bump_next_id(unsigned long long *next_id, const int32_t *__restrict__ spawn_total) {
    if (threadIdx.x == 0 && blockIdx.x == 0) *next_id += 2ull * (unsigned long long)(*spawn_total);
}

// Sort the slots [b0, b1) of one leaf by key (one warp).  Up to 32 entries sort in registers;
// longer runs go through the idle buffer `tmp`.
constexpr int kSortSmem = 512;  // per-warp shared-memory sort capacity (keys + slots)

// Sort the slots [b0, b1) of one leaf by key (one warp).  Up to 32 entries sort in registers;
// up to 512 by a bitonic network on (key, slot) pairs in the warp's shared memory followed by
// a gather through the idle buffer `tmp`; longer runs were sorted by k_sort_big already.
template <typename R>
__device__ void sort_region(int32_t b0, int32_t b1, int lane, SoA<R> d, uint32_t *__restrict__ key, SoA<R> tmp,
                            uint32_t *__restrict__ tkey, unsigned long long *wsm) {
    const int32_t k = b1 - b0;
    if (k <= 1 || k > kSortSmem) return;  // longer regions: k_sort_big
    if (k <= 32) {
        const bool act = lane < k;
        const uint32_t kk = act ? key[b0 + lane] : 0xFFFFFFFFu;
        int rank = 0;
        for (int j = 0; j < k; ++j) {
            const uint32_t o = __shfl_sync(0xFFFFFFFFu, kk, j);
            rank += (o < kk) ? 1 : 0;
        }
        R u = 0, v = 0, vx = 0, vy = 0, vz = 0, w = 0;
        uint32_t id = 0;
        if (act) {
            const int32_t p = b0 + lane;
            u = d.u[p]; v = d.v[p]; vx = d.vx[p]; vy = d.vy[p]; vz = d.vz[p]; w = d.w[p]; id = d.id[p];
        }
        __syncwarp();
        if (act) {
            const int32_t q = b0 + rank;
            d.u[q] = u; d.v[q] = v; d.vx[q] = vx; d.vy[q] = vy; d.vz[q] = vz; d.w[q] = w; d.id[q] = id;
            key[q] = kk;
        }
        __syncwarp();
        return;
    }
    // copy the region to the idle buffer
    for (int32_t p = b0 + lane; p < b1; p += 32) {
        tmp.u[p] = d.u[p]; tmp.v[p] = d.v[p]; tmp.vx[p] = d.vx[p]; tmp.vy[p] = d.vy[p];
        tmp.vz[p] = d.vz[p]; tmp.w[p] = d.w[p]; tmp.id[p] = d.id[p]; tkey[p] = key[p];
    }
    __syncwarp();
    {
        int32_t np2 = 64;
        while (np2 < k) np2 <<= 1;
        for (int32_t i = lane; i < np2; i += 32)
            wsm[i] = i < k ? (((unsigned long long)tkey[b0 + i] << 32) | (unsigned long long)i) : ~0ull;
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
            const int32_t p = b0 + (int32_t)(wsm[r] & 0xFFFFFFFFull), q = b0 + r;
            d.u[q] = tmp.u[p]; d.v[q] = tmp.v[p]; d.vx[q] = tmp.vx[p]; d.vy[q] = tmp.vy[p];
            d.vz[q] = tmp.vz[p]; d.w[q] = tmp.w[p]; d.id[q] = tmp.id[p]; key[q] = (uint32_t)(wsm[r] >> 32);
        }
        __syncwarp();
    }
}

constexpr int kSortBig = 16384;  // one block sorts up to this many entries in shared memory

// Leaves whose entering region is longer than one warp's shared-memory sort: one block per
// leaf, bitonic network on (key, slot) pairs in dynamic shared memory, gather through `tmp`.
// Regions longer than kSortBig rank every key against all others with the whole block.
template <typename R>
__global__ void __launch_bounds__(512) k_sort_big(const int32_t *__restrict__ list, const int32_t *__restrict__ count,
                                                  const int32_t *__restrict__ start,
                                                  const int32_t *__restrict__ stay, SoA<R> d,
                                                  uint32_t *__restrict__ key, SoA<R> tmp,
                                                  uint32_t *__restrict__ tkey, const R *__restrict__ stay_hi,
                                                  const R *__restrict__ stay_lo, double *__restrict__ wsum) {
    extern __shared__ unsigned long long bk[];
    __shared__ R red_hi[16], red_lo[16];
    const int32_t nbig = *count;
    for (int32_t li = blockIdx.x; li < nbig; li += gridDim.x) {
        const int32_t L = list[li];
        const int32_t b0 = start[L] + (stay ? stay[L] : 0), b1 = start[L + 1];
        const int32_t k = b1 - b0;
        for (int32_t p = b0 + threadIdx.x; p < b1; p += blockDim.x) {
            tmp.u[p] = d.u[p]; tmp.v[p] = d.v[p]; tmp.vx[p] = d.vx[p]; tmp.vy[p] = d.vy[p];
            tmp.vz[p] = d.vz[p]; tmp.w[p] = d.w[p]; tmp.id[p] = d.id[p]; tkey[p] = key[p];
        }
        __syncthreads();
        if (k <= kSortBig) {
            int32_t np2 = 1;
            while (np2 < k) np2 <<= 1;
            for (int32_t i = threadIdx.x; i < np2; i += blockDim.x)
                bk[i] = i < k ? (((unsigned long long)tkey[b0 + i] << 32) | (unsigned long long)i) : ~0ull;
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
                const int32_t p = b0 + (int32_t)(bk[r] & 0xFFFFFFFFull), q = b0 + r;
                d.u[q] = tmp.u[p]; d.v[q] = tmp.v[p]; d.vx[q] = tmp.vx[p]; d.vy[q] = tmp.vy[p];
                d.vz[q] = tmp.vz[p]; d.w[q] = tmp.w[p]; d.id[q] = tmp.id[p]; key[q] = (uint32_t)(bk[r] >> 32);
            }
        } else {
            for (int32_t p = b0 + threadIdx.x; p < b1; p += blockDim.x) {
                const uint32_t kk = tkey[p];
                int32_t rank = 0;
                for (int32_t j = b0; j < b1; ++j) rank += (tkey[j] < kk) ? 1 : 0;
                const int32_t q = b0 + rank;
                d.u[q] = tmp.u[p]; d.v[q] = tmp.v[p]; d.vx[q] = tmp.vx[p]; d.vy[q] = tmp.vy[p];
                d.vz[q] = tmp.vz[p]; d.w[q] = tmp.w[p]; d.id[q] = tmp.id[p]; key[q] = kk;
            }
        }
        __syncthreads();
        if (wsum) {  // entering weights in list order: per-thread Kahan, warps combined in order
            R sum = 0, c = 0;
            for (int32_t p = b0 + threadIdx.x; p < b1; p += blockDim.x) kahan_add(sum, c, d.w[p]);
            R hi = sum, lo = -c;
            warp_two_sum(hi, lo);
            if ((threadIdx.x & 31) == 0) { red_hi[threadIdx.x >> 5] = hi; red_lo[threadIdx.x >> 5] = lo; }
            __syncthreads();
            if (threadIdx.x == 0) {
                double t = (double)stay_hi[L] + (double)stay_lo[L];
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += (double)red_hi[w] + (double)red_lo[w];
                wsum[L] = t;
            }
            __syncthreads();
        }
    }
}

// ------------------------------------------------------------------------------------
// Per-leaf sort of the entering slots [start + stay, start_next) by key (one warp per leaf).
// Up to 32 entries sort in registers; longer runs go through the idle buffer `tmp`.
// ------------------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(kT) k_sort_entering(int64_t nleaf, const int32_t *__restrict__ start,
                                                      const int32_t *__restrict__ stay, SoA<R> d,
                                                      uint32_t *__restrict__ key, SoA<R> tmp,
                                                      uint32_t *__restrict__ tkey, const R *__restrict__ stay_hi,
                                                      const R *__restrict__ stay_lo, double *__restrict__ wsum,
                                                      int32_t *__restrict__ big_list, int32_t *__restrict__ big_count) {
    __shared__ unsigned long long sm_keys[kWarpsPerBlock][kSortSmem];
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t L = warp; L < nleaf; L += nw) {
        const int32_t b0 = start[L] + (stay ? stay[L] : 0), b1 = start[L + 1];
        if (b1 - b0 > kSortSmem) {  // long region: k_sort_big sorts it and sums its weights
            if (lane == 0) big_list[atomicAdd(big_count, 1)] = (int32_t)L;
            continue;
        }
        sort_region(b0, b1, lane, d, key, tmp, tkey, sm_keys[threadIdx.x >> 5]);
        if (wsum) {
            // the leaf's weight for the next deposit: staying sum + entering particles in order
            // (a few entering particles: one lane, in order; many: lanes, then an exact combine)
            __syncwarp();
            const int32_t k = b1 - b0;
            if (k <= 16) {
                if (lane == 0) {
                    R sum = 0, c = 0;
                    for (int32_t p = b0; p < b1; ++p) kahan_add(sum, c, d.w[p]);
                    wsum[L] = ((double)stay_hi[L] + (double)stay_lo[L]) + ((double)sum - (double)c);
                }
            } else {
                R sum = 0, c = 0;
                for (int32_t p = b0 + lane; p < b1; p += 32) kahan_add(sum, c, d.w[p]);
                R hi = sum, lo = -c;
                warp_two_sum(hi, lo);
                if (lane == 0) wsum[L] = ((double)stay_hi[L] + (double)stay_lo[L]) + ((double)hi + (double)lo);
            }
        }
    }
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

template <typename R>
__global__ void k_place_load(int64_t n, const double *__restrict__ x, const double *__restrict__ y,
                             const double *__restrict__ vx, const double *__restrict__ vy,
                             const double *__restrict__ vz, const double *__restrict__ w,
                             const unsigned long long *__restrict__ id, unsigned long long id0, double hf, int lmax,
                             const int32_t *__restrict__ ix, const int32_t *__restrict__ iy,
                             const uint8_t *__restrict__ lev, const int32_t *__restrict__ leaf,
                             const int32_t *__restrict__ slot, const int32_t *__restrict__ start, SoA<R> d,
                             uint32_t *__restrict__ key) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int32_t l = leaf[i];
    const int32_t q = start[l] + slot[i];
    const double h = (double)(1 << (lmax - lev[l])) * hf;
    R u = (R)((x[i] - (double)ix[l] * hf) / h), v = (R)((y[i] - (double)iy[l] * hf) / h);
    u = u < (R)0 ? (R)0 : (u >= (R)1 ? below_one<R>() : u);
    v = v < (R)0 ? (R)0 : (v >= (R)1 ? below_one<R>() : v);
    d.u[q] = u; d.v[q] = v;
    d.vx[q] = (R)vx[i]; d.vy[q] = (R)vy[i]; d.vz[q] = (R)vz[i]; d.w[q] = (R)w[i];
    d.id[q] = (uint32_t)(id ? id[i] : id0 + (unsigned long long)i);
    key[q] = (uint32_t)i;
}

// Read-back: absolute FP64 positions and leaf index per particle.
template <typename R>
__global__ void k_read(int64_t nleaf, const int32_t *__restrict__ start, double hf, int lmax,
                       const int32_t *__restrict__ ix, const int32_t *__restrict__ iy,
                       const uint8_t *__restrict__ lev, SoA<R> d, double *__restrict__ x, double *__restrict__ y,
                       double *__restrict__ vx, double *__restrict__ vy, double *__restrict__ vz,
                       double *__restrict__ w, unsigned long long *__restrict__ id, uint32_t *__restrict__ leaf) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t L = warp; L < nleaf; L += nw) {
        const double s = (double)(1 << (lmax - lev[L]));
        for (int32_t p = start[L] + lane; p < start[L + 1]; p += 32) {
            x[p] = ((double)ix[L] + (double)d.u[p] * s) * hf;
            y[p] = ((double)iy[L] + (double)d.v[p] * s) * hf;
            vx[p] = (double)d.vx[p]; vy[p] = (double)d.vy[p]; vz[p] = (double)d.vz[p];
            w[p] = (double)d.w[p];
            id[p] = d.id[p];
            leaf[p] = (uint32_t)L;
        }
    }
}

// Order the entering regions of every leaf: long regions first (one block each), then the
// warp-per-leaf pass (short regions, and the weight sums when wsum is given).
template <typename R>
void sort_lists(pic_ctx *ctx, int64_t nl, const int32_t *start, const int32_t *stay, SoA<R> d, uint32_t *key,
                SoA<R> tmp, uint32_t *tkey, const R *shi, const R *slo, double *wsum, int32_t *list) {
    // `list` holds nl + 1 ints: the long-region list and its counter at [nl]
    GB_CUDA(cudaMemsetAsync(list + nl, 0, 4, ctx->stream));
    k_sort_entering<R><<<warp_blocks(nl), kT, 0, ctx->stream>>>(nl, start, stay, d, key, tmp, tkey, shi, slo, wsum,
                                                                list, list + nl);
    const size_t smem = (size_t)kSortBig * sizeof(unsigned long long);
    GB_CUDA(cudaFuncSetAttribute(k_sort_big<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_sort_big<R><<<152, 512, smem, ctx->stream>>>(list, list + nl, start, stay, d, key, tmp, tkey, shi, slo, wsum);
    count_launch(ctx, 2);
}

template <typename R> PushArgs<R> push_args(pic_ctx *ctx, Instance &in, int s, int64_t step) {
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
    a.start = sp.start;
    a.map = g.map; a.ix = g.ix; a.iy = g.iy; a.lev = g.lev;
    a.stencil = (const R *)in.stencil;
    a.in = soa<R>(sp, sp.cur);
    a.out = soa<R>(sp, sp.cur ^ 1);
    a.stay = sp.stay; a.inc = sp.inc; a.spawn = nullptr; a.inc_ion = nullptr;
    a.key_out = sp.key;
    a.start_new = sp.start_new;
    a.stay_new = sp.stay;
    a.fill = sp.fill;
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
    a.k0 = (uint32_t)(c.seed & 0xFFFFFFFFu);
    a.k1 = (uint32_t)(c.seed >> 32);
    a.inst_word = (uint32_t)c.instance << 24;
    a.cap = (int32_t)sp.cap;
    a.stay_hi = (R *)sp.stay_hi;
    a.stay_lo = (R *)sp.stay_lo;
    a.ion_cap = in.cfg.n_species > 1 ? (int32_t)in.sp[1].cap : 0;
    a.err = in.d_err;
    a.step = (uint32_t)step;
    (void)ctx;
    return a;
}

template <typename R> void step_impl(pic_ctx *ctx, Instance &in, int64_t step) {
    cudaStream_t st = ctx->stream;
    const int nsp = in.cfg.n_species;
    const int64_t nl = in.nleaf;
    const unsigned wb = warp_blocks(nl);
    // the push kernel runs persistent warps: 4 resident blocks per SM (64 registers)
    const unsigned pb = std::min<unsigned>(wb, 152u * 4u);
    const bool ionize = in.cfg.mcc && in.cfg.sigma_iz0 > 0.0;
    Species &e = in.sp[0];
    Species *ion = nsp > 1 ? &in.sp[1] : nullptr;
    {
        Phase ph(ctx, PIC_PHASE_COUNT);
        for (int s = 0; s < nsp; ++s) {
            GB_CUDA(cudaMemsetAsync(in.sp[s].inc, 0, nl * 4, st));
            GB_CUDA(cudaMemsetAsync(in.sp[s].fill, 0, nl * 4, st));
        }
        for (int s = 0; s < nsp; ++s) {
            PushArgs<R> a = push_args<R>(ctx, in, s, step);
            a.mode = 0;
            if (s == 0 && ionize) {
                a.spawn = e.spawn;
                a.inc_ion = ion ? ion->inc : nullptr;
            }
            k_push<R><<<pb, kT, 0, st>>>(a);
            count_launch(ctx);
        }
    }
    {
        Phase ph(ctx, PIC_PHASE_SCAN);
        for (int s = 0; s < nsp; ++s) {
            Species &sp = in.sp[s];
            k_add_counts<<<blocks_for(nl), kT, 0, st>>>(nl, sp.stay, sp.inc);  // inc := stay + inc
            count_launch(ctx);
            exclusive_scan_i32(ctx, sp.inc, sp.start_new, nl, sp.spawn_base + nl + 1);
        }
        if (ionize) exclusive_scan_i32(ctx, e.spawn, e.spawn_base, nl, e.spawn_base + nl + 1 + scan_scratch_elems(nl));
    }
    {
        Phase ph(ctx, PIC_PHASE_MOVE);
        for (int s = nsp - 1; s >= 0; --s) {
            // ions first is not required; every write lands in its own slot
            PushArgs<R> a = push_args<R>(ctx, in, s, step);
            a.mode = 1;
            if (s == 0 && ionize) {
                a.spawn_base = e.spawn_base;
                a.next_id = in.d_next_id;
                if (ion) {
                    a.ion_out = soa<R>(*ion, ion->cur ^ 1);
                    a.ion_key = ion->key;
                    a.ion_start_new = ion->start_new;
                    a.ion_stay = ion->stay;
                    a.ion_start_old = ion->start;
                    a.ion_fill = ion->fill;
                }
            }
            k_push<R><<<pb, kT, 0, st>>>(a);
            count_launch(ctx);
        }
        if (ionize) {
            k_bump_next_id<<<1, 32, 0, st>>>(in.d_next_id, e.spawn_base + nl);
            count_launch(ctx);
        }
    }
    {
        Phase ph(ctx, PIC_PHASE_SORT);
        for (int s = 0; s < nsp; ++s) {
            Species &sp = in.sp[s];
            // entering region of leaf L: [start_new[L] + stay[L], start_new[L + 1])
            sort_lists<R>(ctx, nl, sp.start_new, sp.stay, soa<R>(sp, sp.cur ^ 1), sp.key, soa<R>(sp, sp.cur),
                          sp.key + sp.cap, (const R *)sp.stay_hi, (const R *)sp.stay_lo, sp.wsum, sp.fill);
            std::swap(sp.start, sp.start_new);
            sp.cur ^= 1;
            sp.sums_valid = true;
        }
    }
    check_launch("particle_step");
}

}  // namespace

// Device memory of one species: the two record buffers, keys (2 x cap) and per-leaf arrays.
void species_alloc(pic_ctx *ctx, Instance &in, int s, int64_t cap) {
    Species &sp = in.sp[s];
    DeviceArena &A = in.part_mem[s];
    A.release_all();
    const size_t rs = in.cfg.precision == PIC_FP64 ? 8 : 4;
    const int64_t nl = in.nleaf;
    sp.cap = cap;
    for (int b = 0; b < 2; ++b) {
        for (int k = 0; k < 6; ++k) sp.arr[b][k] = A.alloc(cap * rs + 64);
        sp.id[b] = dalloc<uint32_t>(A, cap);
    }
    sp.key = dalloc<uint32_t>(A, 2 * cap);
    sp.start = dalloc<int32_t>(A, nl + 1);
    sp.start_new = dalloc<int32_t>(A, nl + 1);
    sp.stay = dalloc<int32_t>(A, nl + 1);
    sp.inc = dalloc<int32_t>(A, nl + 1);
    sp.fill = dalloc<int32_t>(A, nl + 1);
    sp.spawn = dalloc<int32_t>(A, nl + 1);
    sp.stay_hi = A.alloc((nl + 1) * rs + 64);
    sp.stay_lo = A.alloc((nl + 1) * rs + 64);
    sp.wsum = dalloc<double>(A, nl + 1);
    sp.sums_valid = false;
    // spawn_base [nl + 1] | scan scratch | scan scratch
    sp.spawn_base = dalloc<int32_t>(A, nl + 1 + 2 * scan_scratch_elems(nl) + 8);
    GB_CUDA(cudaMemsetAsync(sp.start, 0, (nl + 1) * 4, ctx->stream));
    GB_CUDA(cudaMemsetAsync(sp.spawn_base, 0, (nl + 1 + 2 * scan_scratch_elems(nl) + 8) * 4, ctx->stream));
    sp.cur = 0;
    sp.n = 0;
    sp.n_upper = 0;
}

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
    int64_t cap = in.cfg.particle_capacity > 0 ? in.cfg.particle_capacity : std::max<int64_t>(2 * n + (1 << 16), 1 << 20);
    if (cap < n) fail(PIC_ECAPACITY, "particle_capacity below the loaded population");
    if (id)
        for (int64_t i = 0; i < n; ++i)
            if (id[i] >= (1ull << 32)) fail(PIC_EINVAL, "particle id >= 2^32");
    species_alloc(ctx, in, s, cap);
    DeviceArena tmp;
    double *d[6];
    const double *h[6] = {x, y, vx, vy, vz, w};
    for (int k = 0; k < 6; ++k) {
        d[k] = dalloc<double>(tmp, n);
        if (n) GB_CUDA(cudaMemcpyAsync(d[k], h[k], n * 8, cudaMemcpyHostToDevice, st));
    }
    unsigned long long *did = nullptr;
    if (id && n) {
        did = dalloc<unsigned long long>(tmp, n);
        GB_CUDA(cudaMemcpyAsync(did, id, n * 8, cudaMemcpyHostToDevice, st));
    }
    int32_t *leaf = dalloc<int32_t>(tmp, n), *slot = dalloc<int32_t>(tmp, n);
    int32_t *err = dalloc<int32_t>(tmp, 1);
    GB_CUDA(cudaMemsetAsync(err, 0, 4, st));
    GB_CUDA(cudaMemsetAsync(sp.inc, 0, nl * 4, st));
    Level &g = in.lv[0];
    const double hf = in.h0 / (double)(1 << in.lmax);
    if (n) {
        k_locate_load<<<blocks_for(n), kT, 0, st>>>(n, d[0], d[1], hf, in.nx0 << in.lmax, in.ny0 << in.lmax, g.map,
                                                    leaf, sp.inc, slot, err);
        count_launch(ctx);
    }
    int32_t herr = 0;
    GB_CUDA(cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaStreamSynchronize(st));
    if (herr) {
        tmp.release_all();
        fail(PIC_EINVAL, "particle position outside the domain");
    }
    exclusive_scan_i32(ctx, sp.inc, sp.start, nl, sp.spawn_base + nl + 1);
    const unsigned long long id0 = id ? 0ull : next_id;
    if (n) {
        if (in.cfg.precision == PIC_FP64)
            k_place_load<double><<<blocks_for(n), kT, 0, st>>>(n, d[0], d[1], d[2], d[3], d[4], d[5], did, id0, hf,
                                                               in.lmax, g.ix, g.iy, g.lev, leaf, slot, sp.start,
                                                               soa<double>(sp, 0), sp.key);
        else
            k_place_load<float><<<blocks_for(n), kT, 0, st>>>(n, d[0], d[1], d[2], d[3], d[4], d[5], did, id0, hf,
                                                              in.lmax, g.ix, g.iy, g.lev, leaf, slot, sp.start,
                                                              soa<float>(sp, 0), sp.key);
        count_launch(ctx);
        if (in.cfg.precision == PIC_FP64)
            sort_lists<double>(ctx, nl, sp.start, nullptr, soa<double>(sp, 0), sp.key, soa<double>(sp, 1),
                               sp.key + sp.cap, nullptr, nullptr, nullptr, sp.fill);
        else
            sort_lists<float>(ctx, nl, sp.start, nullptr, soa<float>(sp, 0), sp.key, soa<float>(sp, 1),
                              sp.key + sp.cap, nullptr, nullptr, nullptr, sp.fill);
    }
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
    DepositArgs a{};
    a.nleaf = in.nleaf;
    a.nsp = 0;
    for (int s = 0; s < in.cfg.n_species; ++s) {
        if (!in.sp[s].start) continue;
        a.start[a.nsp] = in.sp[s].start;
        a.w[a.nsp] = in.sp[s].arr[in.sp[s].cur][5];
        a.q[a.nsp] = in.cfg.q[s];
        ++a.nsp;
    }
    a.lev = in.lv[0].lev;
    a.lmax = in.lmax;
    a.hf = in.h0 / (double)(1 << in.lmax);
    a.rho_bg = in.cfg.rho_background;
    a.inv_eps0 = 1.0 / in.cfg.eps0;
    a.bcw = in.lv[0].bcw;
    for (int k = 0; k < 4; ++k) a.wall[k] = walls[k];
    a.charge = in.charge;
    a.b = in.bvec;
    bool sums = true;
    for (int s = 0; s < in.cfg.n_species; ++s) sums = sums && in.sp[s].start && in.sp[s].sums_valid;
    if (sums)
        k_deposit_sums<<<blocks_for(in.nleaf), kT, 0, ctx->stream>>>(a, in.sp[0].wsum,
                                                                   in.cfg.n_species > 1 ? in.sp[1].wsum : nullptr);
    else if (in.cfg.precision == PIC_FP64)
        k_deposit<double><<<warp_blocks(in.nleaf), kT, 0, ctx->stream>>>(a);
    else
        k_deposit<float><<<warp_blocks(in.nleaf), kT, 0, ctx->stream>>>(a);
    count_launch(ctx);
    check_launch("deposit");
}

// Make sure a step cannot overflow the particle buffers: the electron count can at most
// double in one step (every electron ionizes once), the ion count grows by at most that.
void ensure_capacity(pic_ctx *ctx, Instance &in) {
    const bool ionize = in.cfg.mcc && in.cfg.sigma_iz0 > 0.0;
    if (!ionize) return;
    const int nsp = in.cfg.n_species;
    const int64_t ne_up = in.sp[0].n_upper;
    bool ok = 2 * ne_up <= in.sp[0].cap && (nsp < 2 || in.sp[1].n_upper + ne_up <= in.sp[1].cap);
    if (ok) return;
    // read the exact counts
    for (int s = 0; s < nsp; ++s) {
        GB_CUDA(cudaMemcpyAsync(in.cnt_host + s, in.sp[s].start + in.nleaf, 4, cudaMemcpyDeviceToHost, ctx->stream));
    }
    GB_CUDA(cudaStreamSynchronize(ctx->stream));
    for (int s = 0; s < nsp; ++s) in.sp[s].n = in.sp[s].n_upper = in.cnt_host[s];
    const int64_t ne = in.sp[0].n;
    for (int s = 0; s < nsp; ++s) {
        Species &sp = in.sp[s];
        const int64_t need = s == 0 ? 2 * ne : sp.n + ne;
        if (need <= sp.cap) continue;
        if (in.cfg.particle_capacity > 0) fail(PIC_ECAPACITY, "particle population would exceed particle_capacity");
        int64_t cap = std::max<int64_t>(2 * need, sp.cap * 2);
        if (cap >= (1ll << 31)) fail(PIC_ECAPACITY, "particle population beyond 2^31");
        // grow: copy the current records and list offsets into fresh buffers
        const size_t rs = in.cfg.precision == PIC_FP64 ? 8 : 4;
        const int64_t n = sp.n, nl = in.nleaf;
        DeviceArena old = in.part_mem[s];
        Species os = sp;
        in.part_mem[s].blocks.clear();
        species_alloc(ctx, in, s, cap);
        for (int k = 0; k < 6; ++k)
            GB_CUDA(cudaMemcpyAsync(sp.arr[0][k], os.arr[os.cur][k], n * rs, cudaMemcpyDeviceToDevice, ctx->stream));
        GB_CUDA(cudaMemcpyAsync(sp.id[0], os.id[os.cur], n * 4, cudaMemcpyDeviceToDevice, ctx->stream));
        GB_CUDA(cudaMemcpyAsync(sp.start, os.start, (nl + 1) * 4, cudaMemcpyDeviceToDevice, ctx->stream));
        GB_CUDA(cudaMemcpyAsync(sp.spawn_base, os.spawn_base, (nl + 1 + 2 * scan_scratch_elems(nl) + 8) * 4,
                                cudaMemcpyDeviceToDevice, ctx->stream));
        GB_CUDA(cudaStreamSynchronize(ctx->stream));
        sp.n = sp.n_upper = n;
        old.release_all();
    }
}

void particle_step(pic_ctx *ctx, Instance &in, int64_t step) {
    if (in.cfg.precision == PIC_FP64) step_impl<double>(ctx, in, step);
    else step_impl<float>(ctx, in, step);
    const bool ionize = in.cfg.mcc && in.cfg.sigma_iz0 > 0.0;
    if (ionize) {
        const int64_t ne = in.sp[0].n_upper;
        in.sp[0].n_upper = 2 * ne;
        if (in.cfg.n_species > 1) in.sp[1].n_upper += ne;
    }
}

void particles_read(pic_ctx *ctx, Instance &in, int s, double *x, double *y, double *vx, double *vy,
                    double *vz, double *w, uint64_t *id, uint32_t *leaf) {
    Species &sp = in.sp[s];
    cudaStream_t st = ctx->stream;
    const int64_t n = sp.n;
    DeviceArena tmp;
    double *d[6];
    for (int k = 0; k < 6; ++k) d[k] = dalloc<double>(tmp, n);
    unsigned long long *did = dalloc<unsigned long long>(tmp, n);
    uint32_t *dleaf = dalloc<uint32_t>(tmp, n);
    Level &g = in.lv[0];
    const double hf = in.h0 / (double)(1 << in.lmax);
    if (in.cfg.precision == PIC_FP64)
        k_read<double><<<warp_blocks(in.nleaf), kT, 0, st>>>(in.nleaf, sp.start, hf, in.lmax, g.ix, g.iy, g.lev,
                                                             soa<double>(sp, sp.cur), d[0], d[1], d[2], d[3], d[4],
                                                             d[5], did, dleaf);
    else
        k_read<float><<<warp_blocks(in.nleaf), kT, 0, st>>>(in.nleaf, sp.start, hf, in.lmax, g.ix, g.iy, g.lev,
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

}  // namespace gbpic
