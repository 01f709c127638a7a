// Internal declarations shared by the gbpic translation units: context layout, device
// helpers (Philox, warp scans, leaf geometry) and host entry points of each unit.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <map>
#include <unordered_map>
#include <functional>
#include <vector>

#include "../../include/gbpic.h"

namespace gbpic {

// ------------------------------------------------------------------------------------
// Errors
// ------------------------------------------------------------------------------------
struct Error {
    pic_status code;
    std::string msg;
};
void set_error(const std::string &msg);
[[noreturn]] void fail(pic_status code, const std::string &msg);
void check_cuda(cudaError_t e, const char *what);
#define GB_CUDA(call) ::gbpic::check_cuda((call), #call)

constexpr int kEll = 8;           // off-diagonal slots per row of the Poisson operator
constexpr int kMaxLevel = 8;      // deepest supported refinement level
constexpr int kWarp = 32;

// ------------------------------------------------------------------------------------
// Device memory.  A context keeps the blocks it releases in a size-class cache and hands
// them out again, so a mesh rebuild (adaptation) or a temporary buffer costs no
// cudaMalloc / cudaFree (cudaFree also synchronizes the device).  Every user of a cache
// enqueues its work on the context's one stream, so a block released while kernels that
// read it are still queued is only rewritten by work queued after them.
// ------------------------------------------------------------------------------------
struct BlockCache {
    std::multimap<size_t, void *> idle;      // size class -> cached block
    std::unordered_map<void *, size_t> cls;  // every block from this cache -> its size class
    size_t idle_bytes = 0;
    int64_t fail_after = -1;  // injected fault: this many more blocks succeed, then one fails
    void *get(size_t bytes);
    void put(void *p);  // over the idle limit, the largest idle blocks are freed first
    void trim();  // cudaFree every cached block
};

struct DeviceArena {
    BlockCache *cache = nullptr;  // null: plain cudaMalloc / cudaFree
    std::vector<void *> blocks;
    DeviceArena() = default;
    explicit DeviceArena(BlockCache *c) : cache(c) {}
    void *alloc(size_t bytes);
    void release(void *p);
    void release_all();
};

template <typename T>
T *dalloc(DeviceArena &a, size_t n) { return static_cast<T *>(a.alloc(n * sizeof(T) + 16)); }

// ------------------------------------------------------------------------------------
// Multigrid level: a composite leaf mesh on its own lattice of (nx0 << lmax) x
// (ny0 << lmax) cells of side h0 / 2^lmax.
// ------------------------------------------------------------------------------------
struct Level {
    int nx0 = 0, ny0 = 0, lmax = 0;
    double h0 = 0;
    int64_t n = 0;
    int32_t *ix = nullptr, *iy = nullptr;  // lattice corner
    uint8_t *lev = nullptr;                // level (side = 1 << (lmax - lev) lattice cells)
    int32_t *map = nullptr;                // lattice cell -> cell index
    int32_t *parent = nullptr;             // cell -> cell of the next coarser level
    int32_t *child4 = nullptr;             // cell -> up to 4 cells of the next finer level
    int32_t *col = nullptr;                // ELL off-diagonal columns [kEll * n], -1 = empty
    float *val = nullptr;                  // ELL off-diagonal values (FP32)
    float *dinv = nullptr;                 // 1 / diagonal (FP32)
    uint8_t *color = nullptr;              // red-black colour of the cell on its own scale
    double *val64 = nullptr, *diag64 = nullptr;  // finest level only (FP64 residual)
    double *bcw = nullptr;                 // finest level: Dirichlet coefficients [4 * n]
    double *kappa = nullptr;               // implicit scheme: relative permittivity 1 + chi per cell
    float *x = nullptr, *b = nullptr, *t = nullptr;  // FP32 work vectors
    int64_t lat_n() const { return ((int64_t)nx0 << lmax) * ((int64_t)ny0 << lmax); }
};

// Cell lists with free slots.  Leaf L of a species owns the slot segment
// [start[L], lim[L]) of the species' buffers; its records are [start[L], end[L]) in list
// order and the free slots [end[L], lim[L]) take the particles that enter L during a step,
// so the push updates the lists in place.  A leaf that receives more particles than it has
// free slots moves to a fresh segment at the tail of the buffer (past every segment); only
// when the tail is used up are all lists of the species laid out again.  Every list builder
// (load, adaptation, split/merge, re-layout) gives a leaf with c records list_slack(c) free
// slots, segments in leaf order.
__host__ __device__ inline int32_t list_slack(int32_t c) { return 16 + (c >> 2); }
// Slots that lists of n records over nl leaves need, free slots included.
inline int64_t slots_for(int64_t n, int64_t nl) { return n + n / 4 + 16 * nl + 64; }
// Slots of a species loaded with n records (particle_capacity unset): room for the
// population to double (every electron ionizing once) before a regrow, plus a tail of about
// the population's size for the leaves whose free slots run out (each takes a fresh segment
// there; a re-layout, which copies every record twice, compacts the lists when the tail is
// used up).
inline int64_t load_slots(int64_t n, int64_t nl) {
    const int64_t s = slots_for(3 * n + (1 << 16), nl);
    return s > (1 << 20) ? s : (1 << 20);
}

// One species: SoA records (offsets u, v in [0,1) of the leaf, velocity, weight:
// precision R; id: u32) in three buffers of `cap` slots: the lists (arr[cur]), a scratch
// buffer (arr[cur ^ 1]: sorts, re-layout) and the overflow store (records whose leaf had
// no free slot left, with their destination).
struct Species {
    int64_t cap = 0;      // slots per buffer
    int64_t n = 0;        // exact count known to the host
    int64_t n_upper = 0;  // upper bound on the count while steps are in flight
    int cur = 0;
    void *arr[2][6] = {};      // u, v, vx, vy, vz, w
    uint32_t *id[2] = {};
    uint32_t *key = nullptr;   // [2 cap] sort key of entering records (lists | scratch)
    uint32_t *aux = nullptr;   // [2 cap] spawned records: the parent's leaf
    int32_t *start = nullptr;  // [nleaf + 1] first slot of each leaf's segment
    int32_t *end = nullptr;    // [nleaf + 1] end of each leaf's records
    int32_t *lim = nullptr;    // [nleaf + 1] end of each leaf's segment
    int32_t *rank0 = nullptr;  // [nleaf + 1] records before leaf L in list order; [nleaf] = total
    int32_t *start_new = nullptr;
    int32_t *stay = nullptr, *inc = nullptr, *fill = nullptr;  // [nleaf + 1]
    int32_t *big = nullptr;    // [nleaf + 1] long entering regions, their count at [nleaf]
    int32_t *moved = nullptr;  // [nleaf + 1] leaves that ran out of free slots, count at [nleaf]
    int32_t *spawn = nullptr, *spawn_base = nullptr;           // [nleaf], [nleaf + 1]
    // overflow store
    void *ovf[6] = {};
    uint32_t *ovf_id = nullptr, *ovf_key = nullptr, *ovf_aux = nullptr;
    int32_t *ovf_dest = nullptr, *ovf_slot = nullptr;
    // device words: [0] records in the overflow store, [1] record total, [2] re-layouts,
    // [3] records that went through the store, [4] first unused slot of the buffer (tail),
    // [5] tail used up this step (re-layout), [6] leaves moved to the tail (statistics),
    // [7] the re-layout drops the inflow room to fit the buffer
    int32_t *flags = nullptr;
    // per-leaf weight sums left by the last cell-list update for the next deposit: the staying
    // particles' compensated sum (move pass) and the entering particles' (per-leaf sort)
    void *stay_hi = nullptr, *stay_lo = nullptr;               // R [nleaf]
    void *ent_hi = nullptr, *ent_lo = nullptr;                 // R [nleaf]
    bool sums_valid = false;
    // the per-step list repairs as a graph of two IF nodes (pic_lists.cu), valid for the
    // mesh and list epochs it was built in
    cudaGraphExec_t repair = nullptr;
    int64_t repair_mesh_epoch = -1, repair_lists_epoch = -1;
};

template <typename R> struct SoA {
    R *u, *v, *vx, *vy, *vz, *w;
    uint32_t *id;
};
template <typename R> inline SoA<R> soa(Species &sp, int buf) {
    SoA<R> a;
    a.u = (R *)sp.arr[buf][0]; a.v = (R *)sp.arr[buf][1]; a.vx = (R *)sp.arr[buf][2];
    a.vy = (R *)sp.arr[buf][3]; a.vz = (R *)sp.arr[buf][4]; a.w = (R *)sp.arr[buf][5];
    a.id = sp.id[buf];
    return a;
}
template <typename R> inline SoA<R> soa_ovf(Species &sp) {
    SoA<R> a;
    a.u = (R *)sp.ovf[0]; a.v = (R *)sp.ovf[1]; a.vx = (R *)sp.ovf[2];
    a.vy = (R *)sp.ovf[3]; a.vz = (R *)sp.ovf[4]; a.w = (R *)sp.ovf[5];
    a.id = sp.ovf_id;
    return a;
}

// Time-averaged diagnostics of one instance (pic_diag_enable): per-leaf sums over the steps
// since the last reset, and the electron energy histogram of a region.
struct Diag {
    bool on = false;
    int nbins = 0;
    double eps_max = 0.0;                   // [eV]
    double region[4] = {0, 0, 0, 0};        // x0, x1, y0, y1 (absolute)
    int64_t samples = 0;                    // steps accumulated since the reset
    int64_t nleaf = 0;
    double *leaf = nullptr;                 // [4 nleaf]: sum w_e, sum w_i, sum w_e eps [eV], sum phi
    double *eedf = nullptr;                 // [nbins] sum of electron weights per energy bin
    double *part = nullptr;                 // per-warp partial histograms of one step
    DeviceArena mem;
};

struct Instance {
    pic_config cfg{};
    bool has_mesh = false;
    int nx0 = 0, ny0 = 0, lmax = 0;
    double h0 = 0;
    int64_t nleaf = 0;
    uint32_t *key = nullptr;     // leaf Morton keys
    uint32_t *root = nullptr;    // per leaf
    uint32_t *morton = nullptr;  // per leaf
    std::vector<Level> lv;       // lv[0] = the leaves
    double *phi = nullptr, *bvec = nullptr, *res = nullptr, *charge = nullptr;
    double *phi_prev = nullptr;  // previous solution: the next solve starts from 2 phi - phi_prev
    int n_solves = 0;            // solves since the mesh was set (extrapolation needs two)
    int32_t *d_n_solves = nullptr;  // the same count on the device, for meshes solved in one launch
    double last_walls[4] = {0, 0, 0, 0};  // wall potentials of the last solve
    double *red = nullptr;       // reduction scratch
    double *red_host = nullptr;  // pinned
    int32_t *cnt_host = nullptr; // pinned
    void *stencil = nullptr;     // node E per leaf corner: 8 x R per leaf
    void *patch = nullptr;       // cloud-in-cell shapes: per leaf 4 quarters x 2 components x 4 R
    double *cic_part = nullptr;  // cloud-in-cell deposit: per leaf its charge on the 3 x 3 cells around it
    Species sp[2];
    int64_t next_id = 0;                     // host mirror (exact after a sync)
    unsigned long long *d_next_id = nullptr; // device counter of the next particle id
    int32_t *d_err = nullptr;                // device-side consistency flag (0 = fine)
    double *d_walls = nullptr;               // the context's wall array for this instance (4)
    int32_t report_err = 0;                  // consistency flag read by the last report
    double mg_worst = 0;                     // worst relative residual of the solves since the reset
    int mg_cycles = 0;
    double mg_res = 0;
    double mg_res_max = 0;         // host-driven solves: worst relative residual since reset
    bool mg_on_device = false;     // last solve ran its loop on the device (stats below)
    double *mg_stats = nullptr;    // device: [cycles, rel. residual, max rel. since reset]
    double *coarse_inv = nullptr;        // coarsest multigrid level: dense FP64 inverse (small levels)
    void *small_item = nullptr;          // meshes that fit one block: the solve's work item
    size_t small_smem = 0;               // and its dynamic shared memory
    int small_cluster = 1;               // CTAs of its cluster when solved alone
    cudaGraphExec_t mg_cycle = nullptr;  // multi-block meshes: one captured cycle (V-cycle,
    int64_t mg_cycle_nodes = 0;          // correction, residual, norm read-back) and its launches
    int64_t mg_pre_nodes = 0;            // launches before the device-side cycle loop
    bool mg_count_cycles = false;        // add the device loop's cycles to the launch count
    Diag diag;                   // time-averaged diagnostics (off unless enabled)
    DeviceArena mesh_mem;        // freed on pic_set_mesh
    DeviceArena part_mem[2];     // freed on reload / regrow
};

struct TimingRec {
    int phase;
    cudaEvent_t a, b;
    int64_t launches;
};

}  // namespace gbpic

namespace gbpic {
// Launch shapes that no result depends on, chosen by pic_autotune (defaults until then).
struct Tuning {
    int push_threads = 256;  // block size of the push kernel (128 or 256)
    int push_bps = 0;        // resident push blocks per SM (0: as many as fit)
    int graph_div = 4;       // captured ensemble steps: each push takes 1/graph_div of the GPU
    int branches = 16;       // captured ensemble steps: parallel branches
    int batch_leaves = 64;   // batched ensemble steps: leaves per push block (a multiple of 32)
    double best_ms = 0.0;    // best step time the tuner measured
    int64_t epoch = 0;       // bumped on every change (a captured step is captured again)
};
// Device tables of the batched ensemble step (one launch per phase over every instance):
// `tab` holds one entry per instance or per (instance, species), `chunks` one int4
// {entry, first leaf, end leaf, 0} per block.  Built and uploaded before the step is
// captured; freed when it is captured again.
struct BatchTab {
    const void *tab = nullptr;
    const int4 *chunks = nullptr;
    int n = 0, nchunks = 0;
};
// A segmented exclusive scan: per segment {in, out, n, first tile}, per block {segment, tile}.
struct ScanPlan {
    const void *segs = nullptr;
    const int2 *tiles = nullptr;
    int nseg = 0, ntiles = 0;
    int32_t *scratch = nullptr;
};
struct BatchStep {
    bool on = false;  // the captured step is the batched one
    BatchTab dep, nodee, lists, push[2], sort, sort_med, bump;
    ScanPlan ranks, spawns, relay5, relay7;
    int32_t *flag = nullptr;  // device word: any instance has records in its overflow store
    std::vector<void *> bufs;
};
}  // namespace gbpic

struct pic_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool poisoned = false;
    int64_t step = 0;
    int64_t launches = 0;
    bool timing = false;
    std::vector<gbpic::TimingRec> trec;
    std::vector<cudaEvent_t> event_pool;  // created before a timed capture, taken by its phases
    std::vector<gbpic::Instance> inst;
    int precision = PIC_FP32;
    // batched one-block Poisson solves (instances whose meshes fit one block)
    int64_t mesh_epoch = 0, batch_epoch = -1;
    int batch_n = 0;
    void *batch_items = nullptr;
    size_t batch_smem = 0;
    gbpic::DeviceArena batch_mem;
    gbpic::BlockCache cache;  // device blocks released by this context, for reuse
    // captured multi-instance step (pic_graph.cu)
    bool capturing = false;          // launches are being captured: read step and walls on the device
    int64_t *d_step = nullptr;       // device copy of the step number
    double *d_walls = nullptr;       // per instance: the 4 wall potentials of the current step
    int64_t lists_epoch = 0;         // bumped whenever list buffers or per-leaf arrays are re-allocated
    cudaGraphExec_t step_graph = nullptr;
    int64_t graph_mesh_epoch = -1, graph_lists_epoch = -1;
    int64_t graph_nodes = 0;         // kernel launches of one replay
    std::vector<cudaStream_t> fork;  // branches of the captured step
    std::vector<cudaEvent_t> fork_ev;
    cudaStream_t load_side = nullptr;              // particle loads: copies beside the context's stream
    cudaEvent_t load_ev[2] = {nullptr, nullptr};
    void *report_dev = nullptr, *report_host = nullptr;  // end-of-call report, one entry per instance
    void *report_tab = nullptr;      // device table the report kernel reads
    int64_t report_epoch = -1;
    gbpic::Tuning tune;
    int64_t graph_tune_epoch = -1;
    gbpic::BatchStep batch;          // tables of the batched ensemble step (pic_graph.cu)
    // phase timing inside replays of the batched step: event nodes captured per phase (when
    // timing was on at the capture), read after each timed replay
    bool capture_phases = false, graph_timed = false;
    std::vector<gbpic::TimingRec> graph_trec;
    double graph_ms[16] = {};
    int64_t graph_launches[16] = {};
    int32_t fault_balance_sweeps = 0;  // injected fault: bound of the adaptation's balance closure (0: none)
};

namespace gbpic {

// Launch accounting / phase timing around a group of launches.
struct Phase {
    pic_ctx *ctx;
    int phase;
    int64_t launches0;
    cudaEvent_t a = nullptr;
    Phase(pic_ctx *c, int p);
    ~Phase();
};
inline void count_launch(pic_ctx *c, int64_t k = 1) { c->launches += k; }
void check_launch(const char *what);

// ------------------------------------------------------------------------------------
// Device helpers
// ------------------------------------------------------------------------------------
__host__ __device__ inline uint32_t spread2(uint32_t v) {
    v &= 0xFFFFu;
    v = (v | (v << 8)) & 0x00FF00FFu;
    v = (v | (v << 4)) & 0x0F0F0F0Fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}
__host__ __device__ inline uint32_t compact2(uint32_t v) {
    v &= 0x55555555u;
    v = (v | (v >> 1)) & 0x33333333u;
    v = (v | (v >> 2)) & 0x0F0F0F0Fu;
    v = (v | (v >> 4)) & 0x00FF00FFu;
    v = (v | (v >> 8)) & 0x0000FFFFu;
    return v;
}

// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): 10 rounds, Weyl key schedule.  The ten
// round keys of each word, (k + r W) mod 2^32, are computed once on the host (philox_keys), so
// a kernel that takes them as a parameter applies each as an operand of the round's XOR.
struct U4 { uint32_t x, y, z, w; };
struct PhiloxKeys { uint32_t k0[10], k1[10]; };
inline PhiloxKeys philox_keys(uint64_t seed) {
    PhiloxKeys K{};
    uint32_t k0 = (uint32_t)(seed & 0xFFFFFFFFu), k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        K.k0[r] = k0;
        K.k1[r] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return K;
}
__device__ __forceinline__ U4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                            const PhiloxKeys &K) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        // both halves of each 32 x 32 -> 64-bit product from one wide multiply
        const uint64_t p0 = (uint64_t)0xD2511F53u * c0, p1 = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t lo0 = (uint32_t)p0, hi0 = (uint32_t)(p0 >> 32);
        const uint32_t lo1 = (uint32_t)p1, hi1 = (uint32_t)(p1 >> 32);
        const uint32_t n0 = hi1 ^ c1 ^ K.k0[r], n2 = hi0 ^ c3 ^ K.k1[r];
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    return U4{c0, c1, c2, c3};
}

// Philox2x32-10 (same paper): a 2-word counter, one 32 x 32 -> 64-bit product per round and
// the Weyl key schedule k + r W.  Round keys precomputed on the host as for the 4x32 form.
struct PhiloxKeys2 { uint32_t k[10]; };
inline PhiloxKeys2 philox2_keys(uint32_t key) {
    PhiloxKeys2 K{};
    for (int r = 0; r < 10; ++r) {
        K.k[r] = key;
        key += 0x9E3779B9u;
    }
    return K;
}
__device__ __forceinline__ uint32_t philox2x32_10_x(uint32_t c0, uint32_t c1, const PhiloxKeys2 &K) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p = (uint64_t)0xD256D193u * c0;
        const uint32_t n0 = (uint32_t)(p >> 32) ^ c1 ^ K.k[r];
        c1 = (uint32_t)p;
        c0 = n0;
    }
    return c0;  // the first output word
}

// Leaf geometry on its level's lattice.
struct LeafGeom { int32_t ix, iy, s; };

// Finest-lattice lookup with wrap (periodic) or -1 outside a wall.
__device__ __forceinline__ int32_t lattice_leaf(const int32_t *__restrict__ map, int NX, int NY,
                                                bool px, bool py, int32_t I, int32_t J) {
    if (I < 0 || I >= NX) {
        if (!px) return -1;
        I = I < 0 ? I + NX : I - NX;
    }
    if (J < 0 || J >= NY) {
        if (!py) return -1;
        J = J < 0 ? J + NY : J - NY;
    }
    return __ldg(map + (int64_t)J * NX + I);
}

// ------------------------------------------------------------------------------------
// Entry points of the translation units (host side)
// ------------------------------------------------------------------------------------
// pic_mesh.cu
void mesh_build(pic_ctx *ctx, Instance &in, int nx0, int ny0, double h0, int64_t n,
                const uint32_t *root, const uint32_t *morton, const uint8_t *level);
void mesh_build_device(pic_ctx *ctx, Instance &in, int64_t n);  // from in.root/morton/lev
void node_e(pic_ctx *ctx, Instance &in, const double walls[4]);
void poisson_kappa(pic_ctx *ctx, Instance &in, const double walls[4]);  // implicit: operator of this step
void cell_emag(pic_ctx *ctx, Instance &in, const double walls[4], double *out_dev);
void batch_prepare_node_e(pic_ctx *ctx);
void node_e_batch(pic_ctx *ctx);
// pic_abi.cu
void set_mesh_impl(pic_ctx *ctx, Instance &in, int nx0, int ny0, double h0, int64_t n_leaves,
                   const uint32_t *root, const uint32_t *morton, const uint8_t *level);
// pic_poisson.cu
void poisson_setup(pic_ctx *ctx, Instance &in);
void poisson_solve(pic_ctx *ctx, Instance &in, const double walls[4]);
void poisson_reset_warm_start(pic_ctx *ctx, Instance &in);
void poisson_solve_batch(pic_ctx *ctx, const std::vector<Instance *> &list,
                         const std::vector<const double *> &walls);
void poisson_batch_items(pic_ctx *ctx, const std::vector<Instance *> &list);  // outside a capture
// pic_particles.cu
void particles_load(pic_ctx *ctx, Instance &in, int s, int64_t n, const double *x,
                    const double *y, const double *vx, const double *vy, const double *vz,
                    const double *w, const uint64_t *id);
void deposit(pic_ctx *ctx, Instance &in, const double walls[4]);
// The push passes of a step: the leapfrog, or the direct implicit scheme's predictor (drift by
// the old velocity, no kick, no collisions) and corrector (kick, drift by the kick's increment,
// then collisions).
enum { PUSH_LEAPFROG = 0, PUSH_PREDICT = 1, PUSH_CORRECT = 2 };
void particle_step(pic_ctx *ctx, Instance &in, int64_t step, bool bookkeeping = true, int mode = PUSH_LEAPFROG);
void particle_bookkeeping(Instance &in);  // host-side bounds after a step's launches
void particles_read(pic_ctx *ctx, Instance &in, int s, double *x, double *y, double *vx,
                    double *vy, double *vz, double *w, uint64_t *id, uint32_t *leaf);
void ensure_capacity(pic_ctx *ctx, Instance &in);
void ensure_slots(pic_ctx *ctx, Instance &in, int s, int64_t slots);
void refresh_counts(pic_ctx *ctx, Instance &in);  // sp.n := exact record totals (syncs)
void walls_at(const Instance &in, int64_t step, double walls[4]);
// the batched ensemble step: tables (before the capture), then the launches (captured)
void batch_prepare_particles(pic_ctx *ctx);
void deposit_batch(pic_ctx *ctx);
void particle_step_batch(pic_ctx *ctx);
// pic_lists.cu
void species_alloc(pic_ctx *ctx, Instance &in, int s, int64_t cap);
void species_leaf_arrays(pic_ctx *ctx, Instance &in, int s, int64_t nl);
void lists_from_counts(pic_ctx *ctx, Species &sp, int64_t nl, const int32_t *cnt, int32_t *start,
                       int32_t *end, int32_t *scratch);
void lists_installed(pic_ctx *ctx, Species &sp, int64_t nl);  // lim, tail after start / end are set
void list_ranks(pic_ctx *ctx, Species &sp, int64_t nl);       // rank0 from start / end
void count_totals(pic_ctx *ctx, Instance &in);  // flags[1] of every species, device side
void place_overflow(pic_ctx *ctx, Instance &in, int s);  // tail moves, else re-layout
void repairs_release(Instance &in);                       // the cached repair graphs
BatchTab batch_prepare_lists(pic_ctx *ctx);                // per (instance, species) list arrays
void lists_prep_batch(pic_ctx *ctx);                      // step reset and record counts
void repairs_batch(pic_ctx *ctx);                         // overflow repairs of every instance
// Capture into the graph that stream `st` is capturing: a one-thread kernel that reads *value,
// then an IF node whose body (the launches `body` issues on ctx->stream) runs when it was
// nonzero.  The body's launches are not counted (they run only when needed).
void capture_if(pic_ctx *ctx, cudaStream_t st, const int32_t *value, const std::function<void()> &body);
// pic_graph.cu
bool graph_step_possible(pic_ctx *ctx);
void one_step(pic_ctx *ctx);  // one step of every instance (graph replay or launches), step += 1
void graph_step(pic_ctx *ctx);            // one step of every instance as one graph replay
void graph_prepare(pic_ctx *ctx);         // capture (if out of date) and upload the step graph
void graph_release(pic_ctx *ctx);
bool batch_possible(pic_ctx *ctx);        // every instance NGP, one precision: one launch per phase
void *batch_upload(pic_ctx *ctx, const void *src, size_t bytes);  // device copy, freed with the tables
template <typename T> const T *batch_upload(pic_ctx *ctx, const std::vector<T> &v) {
    return (const T *)batch_upload(ctx, (const void *)v.data(), v.size() * sizeof(T));
}
// Blocks over the leaves of every entry: {entry, first, end, 0}, `per` leaves each.
std::vector<int4> batch_chunks(const std::vector<int64_t> &nleaf, int64_t per);
void report_all(pic_ctx *ctx);            // exact totals, error flags, solver stats of every instance (syncs)
void fields_all(pic_ctx *ctx, int64_t step);
void species_compact(pic_ctx *ctx, Instance &in, int s);  // leaf-order re-layout, tail freed
// pic_cic.cu (uniform meshes)
void cic_patch(pic_ctx *ctx, Instance &in, const double walls[4]);
void cic_deposit(pic_ctx *ctx, Instance &in, const double walls[4]);
void field_arrays(pic_ctx *ctx, Instance &in);  // corner field (and CIC arrays) for the current mesh
// pic_checkpoint.cu
int64_t checkpoint_write(pic_ctx *ctx, Instance &in, void *buf, int64_t cap);  // bytes needed
void checkpoint_read(pic_ctx *ctx, Instance &in, const void *buf, int64_t bytes);
// pic_diag.cu
pic_status stability_check(pic_ctx *ctx, Instance &in, double *dx_ld, double *wdt, double *t_e_ev);
void diag_reset(pic_ctx *ctx, Instance &in);       // zero the sums (and fit them to the mesh)
void diag_accumulate(pic_ctx *ctx, Instance &in);  // add this step's sample
void diag_read_field(pic_ctx *ctx, Instance &in, int field, double *out);  // PIC_FIELD_AVG_*
void diag_enable(pic_ctx *ctx, Instance &in, int nbins, double eps_max, const double *region);
void diag_read_eedf(pic_ctx *ctx, Instance &in, double *f, int64_t *samples);
// pic_adapt.cu
void adapt_mesh(pic_ctx *ctx, Instance &in);
void split_merge(pic_ctx *ctx, Instance &in);

// The larger of two relative residuals, NaN if either is NaN (so a non-finite field is reported).
inline double worst_residual_host(double a, double b) { return (a != a || b != b) ? a + b : (a > b ? a : b); }

// Runs fn(arg) with the ABI's error mapping (exceptions -> pic_status, last error, context
// poisoning on CUDA failures).  Allocates nothing on the device.
pic_status guarded_call(pic_ctx *ctx, pic_status (*fn)(void *), void *arg);

// scan helpers (pic_particles.cu): exclusive scan of n int32 into out[0..n] (out[n] = total)
void exclusive_scan_i32(pic_ctx *ctx, const int32_t *in, int32_t *out, int64_t n,
                        int32_t *scratch, const int32_t *gate = nullptr);
int64_t scan_scratch_elems(int64_t n);
// segments {in, out, n}: out[0..n) = exclusive scan of in, out[n] = total, one launch per pass
// With gates, segment k does nothing while *gate[k] == 0.
ScanPlan scan_plan(pic_ctx *ctx, const std::vector<const int32_t *> &in, const std::vector<int32_t *> &out,
                   const std::vector<int64_t> &n, const std::vector<const int32_t *> &gate = {});
void exclusive_scan_i32_batch(pic_ctx *ctx, const ScanPlan &p);

}  // namespace gbpic
