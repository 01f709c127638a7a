// C ABI of gbpic (include/gbpic.h): context lifetime, argument checks, error mapping, the
// step sequence of §3 (deposit -> Poisson -> corner E -> particle cycle) and read-outs.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <array>
#include <exception>
#include <iterator>
#include <new>

#include "pic_internal.cuh"

namespace gbpic {

namespace {
thread_local std::string g_last_error;

struct Failure : std::exception {
    pic_status code;
    std::string msg;
    Failure(pic_status c, std::string m) : code(c), msg(std::move(m)) {}
};
}  // namespace

void set_error(const std::string &msg) { g_last_error = msg; }

void fail(pic_status code, const std::string &msg) { throw Failure(code, msg); }

void check_cuda(cudaError_t e, const char *what) {
    if (e != cudaSuccess) {
        std::string m = std::string(what) + ": " + cudaGetErrorString(e);
        if (e == cudaErrorMemoryAllocation) throw Failure(PIC_ENOMEM, m);
        throw Failure(PIC_ECUDA, m);
    }
}

void check_launch(const char *what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) throw Failure(PIC_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

namespace {
// Size classes 1/8 of a power of two apart, so a buffer that grows or shrinks by a few
// percent between mesh rebuilds lands on a block it used before.
size_t size_class(size_t b) {
    b = std::max<size_t>(b, 256);
    int e = 63 - __builtin_clzll((unsigned long long)b);
    const size_t g = e >= 3 ? (size_t)1 << (e - 3) : 1;
    return (b + g - 1) / g * g;
}
constexpr size_t kCacheMaxBlock = (size_t)2 << 30;    // larger blocks are freed, not cached
constexpr size_t kCacheMaxIdle = (size_t)8 << 30;     // idle bytes kept at most

void *raw_alloc(size_t bytes) {
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}
}  // namespace

void *BlockCache::get(size_t bytes) {
    if (fail_after == 0) {
        fail_after = -1;
        throw Failure(PIC_ENOMEM, "injected allocation failure (" + std::to_string(bytes) + " bytes)");
    }
    if (fail_after > 0) --fail_after;
    const size_t c = size_class(bytes);
    auto it = idle.lower_bound(c);
    if (it != idle.end() && it->first <= c + c / 4) {
        void *p = it->second;
        idle_bytes -= it->first;
        idle.erase(it);
        return p;
    }
    void *p = raw_alloc(c);
    if (!p) {  // give the idle blocks back to the driver and try once more
        trim();
        p = raw_alloc(c);
    }
    if (!p) throw Failure(PIC_ENOMEM, "cudaMalloc(" + std::to_string(bytes) + " bytes) failed");
    cls[p] = c;
    return p;
}
void BlockCache::put(void *p) {
    auto it = cls.find(p);
    if (it == cls.end()) return;
    if (it->second > kCacheMaxBlock) {
        cudaFree(p);
        cls.erase(it);
        return;
    }
    idle.emplace(it->second, p);
    idle_bytes += it->second;
    // over the limit: the largest idle blocks go back to the driver first, so that a growth
    // of the particle buffers does not also evict the mesh's many small blocks (which the
    // next adaptation would then have to cudaMalloc again)
    while (idle_bytes > kCacheMaxIdle && !idle.empty()) {
        auto big = std::prev(idle.end());
        cudaFree(big->second);
        cls.erase(big->second);
        idle_bytes -= big->first;
        idle.erase(big);
    }
}
void BlockCache::trim() {
    for (auto &e : idle) {
        cudaFree(e.second);
        cls.erase(e.second);
    }
    idle.clear();
    idle_bytes = 0;
}

void *DeviceArena::alloc(size_t bytes) {
    void *p = nullptr;
    if (cache) {
        p = cache->get(bytes);
    } else {
        p = raw_alloc(std::max<size_t>(bytes, 16));
        if (!p) throw Failure(PIC_ENOMEM, "cudaMalloc(" + std::to_string(bytes) + " bytes) failed");
    }
    blocks.push_back(p);
    return p;
}
void DeviceArena::release(void *p) {
    auto it = std::find(blocks.begin(), blocks.end(), p);
    if (it != blocks.end()) {
        if (cache) cache->put(p);
        else cudaFree(p);
        blocks.erase(it);
    }
}
void DeviceArena::release_all() {
    for (void *p : blocks) {
        if (cache) cache->put(p);
        else cudaFree(p);
    }
    blocks.clear();
}

// Outside a capture the events are recorded on the stream; while a batched step is captured
// with phase timing they become event nodes of the graph (external records), read after each
// replay.
Phase::Phase(pic_ctx *c, int p) : ctx(c), phase(p), launches0(c->launches) {
    if (ctx->timing) {
        cudaEventCreate(&a);
        cudaEventRecord(a, ctx->stream);
    } else if (ctx->capturing && ctx->capture_phases && ctx->event_pool.size() >= 2) {
        a = ctx->event_pool.back();
        ctx->event_pool.pop_back();
        GB_CUDA(cudaEventRecordWithFlags(a, ctx->stream, cudaEventRecordExternal));
    }
}
Phase::~Phase() {
    if (ctx->timing && a) {
        cudaEvent_t b;
        cudaEventCreate(&b);
        cudaEventRecord(b, ctx->stream);
        ctx->trec.push_back(TimingRec{phase, a, b, ctx->launches - launches0});
    } else if (a && ctx->capturing && ctx->capture_phases) {
        cudaEvent_t b = ctx->event_pool.back();
        ctx->event_pool.pop_back();
        cudaEventRecordWithFlags(b, ctx->stream, cudaEventRecordExternal);
        ctx->graph_trec.push_back(TimingRec{phase, a, b, ctx->launches - launches0});
    }
}

}  // namespace gbpic

using namespace gbpic;

namespace {

template <typename F> pic_status guarded(pic_ctx *ctx, F &&f) {
    if (ctx && ctx->poisoned) {
        set_error("context poisoned by an earlier CUDA error");
        return PIC_ESTATE;
    }
    try {
        pic_status s = f();
        if (s == PIC_OK) set_error("");
        return s;
    } catch (const Failure &e) {
        set_error(e.msg);
        if (ctx && e.code == PIC_ECUDA) ctx->poisoned = true;
        return e.code;
    } catch (const std::bad_alloc &) {
        set_error("host allocation failed");
        return PIC_ENOMEM;
    } catch (const std::exception &e) {
        set_error(e.what());
        return PIC_EINVAL;
    }
}

void validate(const pic_config &c) {
    if (c.precision != PIC_FP32 && c.precision != PIC_FP64) fail(PIC_EINVAL, "precision must be PIC_FP32 or PIC_FP64");
    if (c.n_species < 1 || c.n_species > 2) fail(PIC_EINVAL, "n_species must be 1 or 2");
    if (!(c.dt > 0.0) || !(c.eps0 > 0.0)) fail(PIC_EINVAL, "dt and eps0 must be positive");
    for (int s = 0; s < c.n_species; ++s)
        if (!(c.m[s] > 0.0)) fail(PIC_EINVAL, "species mass must be positive");
    for (int b : {c.bc_x, c.bc_y})
        if (b < PIC_BC_PERIODIC || b > PIC_BC_NEUMANN) fail(PIC_EINVAL, "bad boundary condition");
    if (c.max_level < 0 || c.max_level > kMaxLevel) fail(PIC_EINVAL, "max_level must be in [0, 8]");
    if (c.mcc) {
        if (!(c.qe > 0.0) || !(c.neutral_mass > 0.0) || c.gas_density < 0.0)
            fail(PIC_EINVAL, "MCC needs qe > 0, neutral_mass > 0, gas_density >= 0");
    }
    if (c.instance < 0 || c.instance > 255) fail(PIC_EINVAL, "instance must be in [0, 255]");
    if (!(c.mg_rel_tol > 0.0)) fail(PIC_EINVAL, "mg_rel_tol must be positive");
    if (c.shape < PIC_SHAPE_NGP || c.shape > PIC_SHAPE_CIC_EC) fail(PIC_EINVAL, "unknown particle shape");
    if (c.shape != PIC_SHAPE_NGP && c.max_level != 0)
        fail(PIC_EINVAL, "cloud-in-cell shapes need a uniform mesh (max_level 0)");
    if (c.implicit != 0 && c.implicit != 1) fail(PIC_EINVAL, "implicit must be 0 or 1");
    if (c.implicit && c.shape != PIC_SHAPE_NGP) fail(PIC_EINVAL, "the implicit scheme uses the NGP shape");
}

Instance &get_inst(pic_ctx *ctx, int32_t inst) {
    if (!ctx) fail(PIC_EINVAL, "null context");
    if (inst < 0 || inst >= (int32_t)ctx->inst.size()) fail(PIC_EINVAL, "instance index out of range");
    return ctx->inst[inst];
}

void reset_solver_stats(pic_ctx *ctx, Instance &in) {
    in.mg_res_max = 0.0;
    if (in.mg_stats) GB_CUDA(cudaMemsetAsync(in.mg_stats + 2, 0, 8, ctx->stream));
}

// Worst relative residual of the solves since the last reset (synchronises the stream).
double collect_solver_stats(pic_ctx *ctx, Instance &in) {
    if (!in.mg_on_device || !in.mg_stats) return in.mg_res_max;
    GB_CUDA(cudaMemcpyAsync(in.red_host + 4, in.mg_stats, 3 * 8, cudaMemcpyDeviceToHost, ctx->stream));
    GB_CUDA(cudaStreamSynchronize(ctx->stream));
    in.mg_cycles = (int)in.red_host[4];
    in.mg_res = in.red_host[5];
    if (in.mg_count_cycles) {  // kernels of the device-side cycle loop of the last solve
        ctx->launches += (int64_t)in.mg_cycles * in.mg_cycle_nodes;
        in.mg_count_cycles = false;
    }
    return worst_residual_host(in.mg_res_max, in.red_host[6]);
}

void ensure_species(pic_ctx *ctx, Instance &in) {
    // a species never loaded is an empty population
    for (int s = 0; s < in.cfg.n_species; ++s)
        if (!in.sp[s].start) species_alloc(ctx, in, s, 1 << 16);
}

}  // namespace

// A new mesh for instance `in` (arguments checked by the caller): particles discarded, leaf
// arrays, multigrid levels and the corner-field array built.
void gbpic::set_mesh_impl(pic_ctx *ctx, Instance &in, int nx0, int ny0, double h0, int64_t n_leaves,
                          const uint32_t *root, const uint32_t *morton, const uint8_t *level) {
    in.part_mem[0].release_all();
    in.part_mem[1].release_all();
    for (auto &sp : in.sp) sp = Species();
    mesh_build(ctx, in, nx0, ny0, h0, n_leaves, root, morton, level);
    poisson_setup(ctx, in);
    diag_reset(ctx, in);
    field_arrays(ctx, in);
    GB_CUDA(cudaStreamSynchronize(ctx->stream));
}

// The corner field array (and, for cloud-in-cell shapes, the per-quarter coefficients and
// the deposit's per-leaf partial charges) of the current mesh, zeroed.
void gbpic::field_arrays(pic_ctx *ctx, Instance &in) {
    const size_t rs = in.cfg.precision == PIC_FP64 ? 8 : 4;
    in.stencil = in.mesh_mem.alloc(8 * rs * in.nleaf + 64);
    GB_CUDA(cudaMemsetAsync(in.stencil, 0, 8 * rs * in.nleaf, ctx->stream));
    in.patch = nullptr;
    in.cic_part = nullptr;
    if (in.cfg.shape != PIC_SHAPE_NGP) {
        in.patch = in.mesh_mem.alloc(32 * rs * in.nleaf + 64);
        GB_CUDA(cudaMemsetAsync(in.patch, 0, 32 * rs * in.nleaf, ctx->stream));
        in.cic_part = dalloc<double>(in.mesh_mem, 9 * in.nleaf);
    }
}

// Field half of a step for every instance: deposits, then one batched launch for all
// instances whose meshes fit one block (one block each), other instances one by one.
void gbpic::fields_all(pic_ctx *ctx, int64_t step) {
    std::vector<std::array<double, 4>> walls(ctx->inst.size());
    for (size_t i = 0; i < ctx->inst.size(); ++i) walls_at(ctx->inst[i], step, walls[i].data());
    {
        Phase ph(ctx, PIC_PHASE_DEPOSIT);
        for (size_t i = 0; i < ctx->inst.size(); ++i) deposit(ctx, ctx->inst[i], walls[i].data());
    }
    {
        Phase ph(ctx, PIC_PHASE_POISSON);
        std::vector<Instance *> small;
        std::vector<const double *> sw;
        for (size_t i = 0; i < ctx->inst.size(); ++i) {
            Instance &in = ctx->inst[i];
            if (in.small_item) {
                small.push_back(&in);
                sw.push_back(walls[i].data());
            } else {
                poisson_solve(ctx, in, walls[i].data());
            }
        }
        if (small.size() == 1) poisson_solve(ctx, *small[0], sw[0]);
        else poisson_solve_batch(ctx, small, sw);
    }
    {
        Phase ph(ctx, PIC_PHASE_NODE_E);
        for (size_t i = 0; i < ctx->inst.size(); ++i) node_e(ctx, ctx->inst[i], walls[i].data());
    }
}


pic_status gbpic::guarded_call(pic_ctx *ctx, pic_status (*fn)(void *), void *arg) {
    return guarded(ctx, [&]() -> pic_status { return fn(arg); });
}

namespace {
// After a call's steps: exact record totals (the next steps' capacity bound), consistency
// flags and solver statistics of every instance, in one read-back.
pic_status end_of_steps(pic_ctx *ctx) {
    report_all(ctx);
    pic_status st = PIC_OK;
    bool finite = true;
    for (Instance &in : ctx->inst) {
        if (!(in.mg_worst <= in.cfg.mg_rel_tol)) st = PIC_ENOTCONV;
        if (!std::isfinite(in.mg_worst)) {
            finite = false;
            poisson_reset_warm_start(ctx, in);
        }
        if (in.report_err != 0) {
            ctx->poisoned = true;
            fail(PIC_ESTATE, "particle bookkeeping violated a slot bound (overflow store or re-layout)");
        }
    }
    if (st != PIC_OK)
        set_error(finite ? "Poisson solve did not reach mg_rel_tol"
                         : "non-finite Poisson residual: NaN or Inf in the charge density or the potential");
    return st;
}

}  // namespace

extern "C" {

pic_status pic_create(const pic_config *cfg, int32_t n_instances, pic_ctx **out) {
    if (!out || !cfg || n_instances < 1) {
        set_error("pic_create: null argument or n_instances < 1");
        return PIC_EINVAL;
    }
    *out = nullptr;
    pic_ctx *ctx = nullptr;
    pic_status s = guarded(nullptr, [&]() -> pic_status {
        for (int i = 0; i < n_instances; ++i) validate(cfg[i]);
        ctx = new pic_ctx();
        GB_CUDA(cudaGetDevice(&ctx->device));
        ctx->inst.resize(n_instances);
        ctx->batch_mem.cache = &ctx->cache;
        for (int i = 0; i < n_instances; ++i) {
            Instance &in = ctx->inst[i];
            in.cfg = cfg[i];
            in.mesh_mem.cache = &ctx->cache;
            in.part_mem[0].cache = &ctx->cache;
            in.part_mem[1].cache = &ctx->cache;
            GB_CUDA(cudaMallocHost(&in.red_host, 64));
            GB_CUDA(cudaMallocHost(&in.cnt_host, 64));
            GB_CUDA(cudaMalloc(&in.d_next_id, 8));
            GB_CUDA(cudaMemset(in.d_next_id, 0, 8));
            GB_CUDA(cudaMalloc(&in.d_err, 4));
            GB_CUDA(cudaMemset(in.d_err, 0, 4));
        }
        // device step counter and wall potentials (read by captured ensemble steps)
        GB_CUDA(cudaMalloc(&ctx->d_step, 8));
        GB_CUDA(cudaMemset(ctx->d_step, 0, 8));
        GB_CUDA(cudaMalloc(&ctx->d_walls, 4 * 8 * (size_t)n_instances));
        for (int i = 0; i < n_instances; ++i) ctx->inst[i].d_walls = ctx->d_walls + 4 * i;
        ctx->precision = cfg[0].precision;
        return PIC_OK;
    });
    if (s != PIC_OK) {
        if (ctx) pic_destroy(ctx);
        return s;
    }
    *out = ctx;
    return PIC_OK;
}

pic_status pic_destroy(pic_ctx *ctx) {
    if (!ctx) return PIC_OK;
    cudaStreamSynchronize(ctx->stream);
    for (Instance &in : ctx->inst) {
        if (in.mg_cycle) cudaGraphExecDestroy(in.mg_cycle);
        repairs_release(in);
        in.mesh_mem.release_all();
        in.part_mem[0].release_all();
        in.part_mem[1].release_all();
        if (in.red_host) cudaFreeHost(in.red_host);
        if (in.cnt_host) cudaFreeHost(in.cnt_host);
        if (in.d_next_id) cudaFree(in.d_next_id);
        if (in.d_err) cudaFree(in.d_err);
    }
    for (auto &r : ctx->trec) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    ctx->batch_mem.release_all();
    graph_release(ctx);
    for (auto ev : ctx->event_pool) cudaEventDestroy(ev);
    if (ctx->load_side) cudaStreamDestroy(ctx->load_side);
    for (auto ev : ctx->load_ev)
        if (ev) cudaEventDestroy(ev);
    for (auto st : ctx->fork) cudaStreamDestroy(st);
    for (auto ev : ctx->fork_ev) cudaEventDestroy(ev);
    if (ctx->d_step) cudaFree(ctx->d_step);
    if (ctx->d_walls) cudaFree(ctx->d_walls);
    if (ctx->report_dev) cudaFree(ctx->report_dev);
    if (ctx->report_tab) cudaFree(ctx->report_tab);
    if (ctx->report_host) cudaFreeHost(ctx->report_host);
    ctx->cache.trim();
    for (auto &e : ctx->cache.cls) cudaFree(e.first);  // blocks an arena still held
    delete ctx;
    return PIC_OK;
}

pic_status pic_set_stream(pic_ctx *ctx, void *stream) {
    return guarded(ctx, [&]() -> pic_status {
        if (!ctx) fail(PIC_EINVAL, "null context");
        // cached blocks may still be read by work queued on the old stream
        GB_CUDA(cudaStreamSynchronize(ctx->stream));
        ctx->stream = (cudaStream_t)stream;
        return PIC_OK;
    });
}

pic_status pic_set_mesh(pic_ctx *ctx, int32_t inst, int32_t nx0, int32_t ny0, double h0, int64_t n_leaves,
                        const uint32_t *root, const uint32_t *morton, const uint8_t *level) {
    return guarded(ctx, [&]() -> pic_status {
        Instance &in = get_inst(ctx, inst);
        if (nx0 < 1 || ny0 < 1 || !(h0 > 0.0) || n_leaves < 1) fail(PIC_EINVAL, "bad mesh size");
        if (!root && n_leaves != (int64_t)nx0 * ny0) fail(PIC_EINVAL, "uniform mesh needs n_leaves == nx0 * ny0");
        if (root && (!morton || !level)) fail(PIC_EINVAL, "root, morton and level must all be given");
        if (n_leaves >= (1ll << 30)) fail(PIC_EINVAL, "too many leaves");
        if (level)
            for (int64_t i = 0; i < n_leaves; ++i)
                if (level[i] > in.cfg.max_level) fail(PIC_EINVAL, "leaf level above max_level");
        set_mesh_impl(ctx, in, nx0, ny0, h0, n_leaves, root, morton, level);
        return PIC_OK;
    });
}

pic_status pic_load_particles(pic_ctx *ctx, int32_t inst, int32_t species, int64_t n, const double *x,
                              const double *y, const double *vx, const double *vy, const double *vz,
                              const double *w, const uint64_t *id) {
    return guarded(ctx, [&]() -> pic_status {
        Instance &in = get_inst(ctx, inst);
        if (!in.has_mesh) fail(PIC_EINVAL, "pic_set_mesh must come first");
        if (species < 0 || species >= in.cfg.n_species) fail(PIC_EINVAL, "species out of range");
        if (n < 0 || n >= (1ll << 31)) fail(PIC_EINVAL, "bad particle count");
        if (n > 0 && (!x || !y || !vx || !vy || !vz || !w)) fail(PIC_EINVAL, "null particle array");
        particles_load(ctx, in, species, n, x, y, vx, vy, vz, w, id);
        if (species != 0) return PIC_OK;
        double a = 0.0, b = 0.0, te = 0.0;
        const pic_status st = stability_check(ctx, in, &a, &b, &te);
        if (st == PIC_WARN_STABILITY)
            set_error("explicit-PIC limits exceeded: max dx / lambda_D = " + std::to_string(a) +
                      " (limit 3), max omega_pe dt = " + std::to_string(b) + " (limit 1), T_e = " +
                      std::to_string(te) + " eV; the particles were loaded");
        return st;
    });
}

pic_status pic_compute_fields(pic_ctx *ctx) {
    return guarded(ctx, [&]() -> pic_status {
        if (!ctx) fail(PIC_EINVAL, "null context");
        pic_status st = PIC_OK;
        for (Instance &in : ctx->inst) {
            if (!in.has_mesh) fail(PIC_EINVAL, "mesh not set");
            ensure_species(ctx, in);
            reset_solver_stats(ctx, in);
        }
        fields_all(ctx, ctx->step);
        bool finite = true;
        for (Instance &in : ctx->inst) {
            const double worst = collect_solver_stats(ctx, in);
            if (!(worst <= in.cfg.mg_rel_tol)) st = PIC_ENOTCONV;
            if (!std::isfinite(worst)) {
                finite = false;
                poisson_reset_warm_start(ctx, in);
            }
        }
        if (st != PIC_OK)
            set_error(finite ? "Poisson solve did not reach mg_rel_tol"
                             : "non-finite Poisson residual: NaN or Inf in the charge density or the potential");
        return st;
    });
}

pic_status pic_step(pic_ctx *ctx, int32_t n_steps) {
    return guarded(ctx, [&]() -> pic_status {
        if (!ctx) fail(PIC_EINVAL, "null context");
        if (n_steps < 0) fail(PIC_EINVAL, "n_steps < 0");
        for (Instance &in : ctx->inst) {
            if (!in.has_mesh) fail(PIC_EINVAL, "mesh not set");
            ensure_species(ctx, in);
            reset_solver_stats(ctx, in);
        }
        for (int32_t k = 0; k < n_steps; ++k) one_step(ctx);
        return end_of_steps(ctx);
    });
}

// Launch-shape autotuner: one ordinary step per candidate configuration, timed with events
// on the context's stream; coordinate search, the best configuration kept.
pic_status pic_autotune(pic_ctx *ctx, int32_t max_steps, int32_t *steps_used) {
    return guarded(ctx, [&]() -> pic_status {
        if (!ctx) fail(PIC_EINVAL, "null context");
        if (max_steps < 0) fail(PIC_EINVAL, "max_steps < 0");
        for (Instance &in : ctx->inst) {
            if (!in.has_mesh) fail(PIC_EINVAL, "mesh not set");
            ensure_species(ctx, in);
            reset_solver_stats(ctx, in);
        }
        int32_t used = 0;
        // an ensemble reaches the state in which its steps replay as one graph after a step
        if (used < max_steps && !graph_step_possible(ctx)) {
            one_step(ctx);
            ++used;
        }
        const bool graph = graph_step_possible(ctx);
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        GB_CUDA(cudaEventCreate(&e0));
        GB_CUDA(cudaEventCreate(&e1));
        Tuning best = ctx->tune;
        double best_ms = 0.0;
        bool have = false;
        // a candidate runs kReps timed steps (the faster counts: the first replay of a fresh
        // capture can be slower) and replaces the best one only if at least 2 % faster
        constexpr int kReps = 2;
        auto trial = [&](Tuning t) {
            if (used + kReps > max_steps) return;
            if (have && t.push_threads == best.push_threads && t.push_bps == best.push_bps &&
                t.graph_div == best.graph_div && t.branches == best.branches)
                return;  // measured already
            t.epoch = ctx->tune.epoch + 1;
            ctx->tune = t;
            if (graph) graph_prepare(ctx);
            double ms = 0.0;
            for (int r = 0; r < kReps; ++r) {
                GB_CUDA(cudaEventRecord(e0, ctx->stream));
                one_step(ctx);
                GB_CUDA(cudaEventRecord(e1, ctx->stream));
                GB_CUDA(cudaEventSynchronize(e1));
                float m = 0.0f;
                GB_CUDA(cudaEventElapsedTime(&m, e0, e1));
                ms = r == 0 ? m : std::min(ms, (double)m);
                ++used;
            }
            if (!have || ms < 0.98 * best_ms) {
                best_ms = ms;
                best = t;
                have = true;
            }
        };
        try {
            for (int nt : {256, 128}) { Tuning t = best; t.push_threads = nt; trial(t); }
            if (graph) {
                for (int div : {4, 1, 2, 8}) { Tuning t = best; t.graph_div = div; trial(t); }
                for (int br : {16, 8, 32}) { Tuning t = best; t.branches = br; trial(t); }
            } else {
                for (int bps : {0, 2, 1}) { Tuning t = best; t.push_bps = bps; trial(t); }
            }
        } catch (...) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            throw;
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (have) {
            best.best_ms = best_ms;
            best.epoch = ctx->tune.epoch + 1;
            ctx->tune = best;
        }
        if (steps_used) *steps_used = used;
        return end_of_steps(ctx);
    });
}

pic_status pic_get_tuning(const pic_ctx *ctx, int32_t *push_threads, int32_t *push_blocks_per_sm,
                          int32_t *graph_push_div, int32_t *graph_branches, double *best_ms) {
    if (!ctx) {
        set_error("null context");
        return PIC_EINVAL;
    }
    const Tuning &t = ctx->tune;
    if (push_threads) *push_threads = t.push_threads;
    if (push_blocks_per_sm) *push_blocks_per_sm = t.push_bps;
    if (graph_push_div) *graph_push_div = t.graph_div;
    if (graph_branches) *graph_branches = t.branches;
    if (best_ms) *best_ms = t.best_ms;
    set_error("");
    return PIC_OK;
}

pic_status pic_adapt(pic_ctx *ctx, int32_t flags) {
    return guarded(ctx, [&]() -> pic_status {
        if (!ctx) fail(PIC_EINVAL, "null context");
        for (Instance &in : ctx->inst) {
            if (!in.has_mesh) fail(PIC_EINVAL, "mesh not set");
            ensure_species(ctx, in);
            if (flags & PIC_ADAPT_MESH) {
                Phase ph(ctx, PIC_PHASE_ADAPT);
                adapt_mesh(ctx, in);
            }
            if (flags & PIC_ADAPT_PARTICLES) {
                Phase ph(ctx, PIC_PHASE_SPLIT_MERGE);
                split_merge(ctx, in);
            }
        }
        return PIC_OK;
    });
}

pic_status pic_read_fields(pic_ctx *ctx, int32_t inst, int32_t field, double *out, int64_t cap, int64_t *n_out) {
    return guarded(ctx, [&]() -> pic_status {
        Instance &in = get_inst(ctx, inst);
        if (!in.has_mesh) fail(PIC_EINVAL, "mesh not set");
        const int64_t nl = in.nleaf;
        int64_t need = field == PIC_FIELD_NODE_E ? 8 * nl : nl;
        if (field < PIC_FIELD_PHI || field > PIC_FIELD_AVG_PHI) fail(PIC_EINVAL, "unknown field");
        if (n_out) *n_out = need;
        if (!out || cap < need) fail(PIC_EINVAL, "output capacity too small");
        cudaStream_t st = ctx->stream;
        std::vector<uint8_t> lev(nl);
        switch (field) {
        case PIC_FIELD_PHI:
            GB_CUDA(cudaMemcpyAsync(out, in.phi, nl * 8, cudaMemcpyDeviceToHost, st));
            GB_CUDA(cudaStreamSynchronize(st));
            break;
        case PIC_FIELD_RHO: {
            GB_CUDA(cudaMemcpyAsync(out, in.charge, nl * 8, cudaMemcpyDeviceToHost, st));
            GB_CUDA(cudaMemcpyAsync(lev.data(), in.lv[0].lev, nl, cudaMemcpyDeviceToHost, st));
            GB_CUDA(cudaStreamSynchronize(st));
            const double hf = in.h0 / (double)(1 << in.lmax);
            for (int64_t l = 0; l < nl; ++l) {
                const double h = (double)(1 << (in.lmax - lev[l])) * hf;
                out[l] = out[l] / (h * h) + in.cfg.rho_background;
            }
            break;
        }
        case PIC_FIELD_COUNT_E:
        case PIC_FIELD_COUNT_I: {
            const int s = field == PIC_FIELD_COUNT_E ? 0 : 1;
            if (s >= in.cfg.n_species || !in.sp[s].start) {
                std::fill(out, out + nl, 0.0);
                break;
            }
            std::vector<int32_t> st0(nl), en0(nl);
            GB_CUDA(cudaMemcpyAsync(st0.data(), in.sp[s].start, nl * 4, cudaMemcpyDeviceToHost, st));
            GB_CUDA(cudaMemcpyAsync(en0.data(), in.sp[s].end, nl * 4, cudaMemcpyDeviceToHost, st));
            GB_CUDA(cudaStreamSynchronize(st));
            for (int64_t l = 0; l < nl; ++l) out[l] = (double)(en0[l] - st0[l]);
            break;
        }
        case PIC_FIELD_NODE_E:
            if (in.cfg.precision == PIC_FP64) {
                GB_CUDA(cudaMemcpyAsync(out, in.stencil, 8 * nl * 8, cudaMemcpyDeviceToHost, st));
                GB_CUDA(cudaStreamSynchronize(st));
            } else {
                std::vector<float> tmp(8 * nl);
                GB_CUDA(cudaMemcpyAsync(tmp.data(), in.stencil, 8 * nl * 4, cudaMemcpyDeviceToHost, st));
                GB_CUDA(cudaStreamSynchronize(st));
                for (int64_t i = 0; i < 8 * nl; ++i) out[i] = tmp[i];
            }
            break;
        case PIC_FIELD_EMAG: {
            DeviceArena tmp(&ctx->cache);
            double *d = dalloc<double>(tmp, nl);
            double walls[4];
            walls_at(in, ctx->step, walls);
            cell_emag(ctx, in, walls, d);
            GB_CUDA(cudaMemcpyAsync(out, d, nl * 8, cudaMemcpyDeviceToHost, st));
            GB_CUDA(cudaStreamSynchronize(st));
            tmp.release_all();
            break;
        }
        default: {  // time averages
            DeviceArena tmp(&ctx->cache);
            double *d = dalloc<double>(tmp, nl);
            diag_read_field(ctx, in, field, d);
            GB_CUDA(cudaMemcpyAsync(out, d, nl * 8, cudaMemcpyDeviceToHost, st));
            GB_CUDA(cudaStreamSynchronize(st));
            tmp.release_all();
            break;
        }
        }
        return PIC_OK;
    });
}

pic_status pic_read_mesh(pic_ctx *ctx, int32_t inst, uint32_t *root, uint32_t *morton, uint8_t *level, int64_t cap,
                         int64_t *n_out) {
    return guarded(ctx, [&]() -> pic_status {
        Instance &in = get_inst(ctx, inst);
        if (!in.has_mesh) fail(PIC_EINVAL, "mesh not set");
        const int64_t nl = in.nleaf;
        if (n_out) *n_out = nl;
        if (cap < nl) fail(PIC_EINVAL, "output capacity too small");
        cudaStream_t st = ctx->stream;
        if (root) GB_CUDA(cudaMemcpyAsync(root, in.root, nl * 4, cudaMemcpyDeviceToHost, st));
        if (morton) GB_CUDA(cudaMemcpyAsync(morton, in.morton, nl * 4, cudaMemcpyDeviceToHost, st));
        if (level) GB_CUDA(cudaMemcpyAsync(level, in.lv[0].lev, nl, cudaMemcpyDeviceToHost, st));
        GB_CUDA(cudaStreamSynchronize(st));
        return PIC_OK;
    });
}

pic_status pic_read_particles(pic_ctx *ctx, int32_t inst, int32_t species, double *x, double *y, double *vx,
                              double *vy, double *vz, double *w, uint64_t *id, uint32_t *leaf, int64_t cap,
                              int64_t *n_out) {
    return guarded(ctx, [&]() -> pic_status {
        Instance &in = get_inst(ctx, inst);
        if (species < 0 || species >= in.cfg.n_species) fail(PIC_EINVAL, "species out of range");
        if (!in.has_mesh) fail(PIC_EINVAL, "mesh not set");
        ensure_species(ctx, in);
        Species &sp = in.sp[species];
        refresh_counts(ctx, in);
        if (n_out) *n_out = sp.n;
        if (cap < sp.n) fail(PIC_EINVAL, "output capacity too small");
        particles_read(ctx, in, species, x, y, vx, vy, vz, w, id, leaf);
        return PIC_OK;
    });
}

pic_status pic_get_list_stats(pic_ctx *ctx, int32_t inst, int32_t species, int64_t *relayouts,
                              int64_t *tail_moves, int64_t *overflowed) {
    return guarded(ctx, [&]() -> pic_status {
        Instance &in = get_inst(ctx, inst);
        if (species < 0 || species >= in.cfg.n_species) fail(PIC_EINVAL, "species out of range");
        Species &sp = in.sp[species];
        int32_t h[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (sp.flags) {
            GB_CUDA(cudaMemcpyAsync(in.cnt_host + 8, sp.flags, 8 * 4, cudaMemcpyDeviceToHost, ctx->stream));
            GB_CUDA(cudaStreamSynchronize(ctx->stream));
            for (int k = 0; k < 8; ++k) h[k] = in.cnt_host[8 + k];
        }
        if (relayouts) *relayouts = h[2];
        if (tail_moves) *tail_moves = h[6];
        if (overflowed) *overflowed = h[3];
        return PIC_OK;
    });
}

pic_status pic_get_counts(pic_ctx *ctx, int32_t inst, int64_t *n_leaves, int64_t *n_e, int64_t *n_i,
                          int32_t *mg_cycles, double *mg_rel_res) {
    return guarded(ctx, [&]() -> pic_status {
        Instance &in = get_inst(ctx, inst);
        int64_t c[2] = {0, 0};
        refresh_counts(ctx, in);
        for (int s = 0; s < in.cfg.n_species; ++s)
            if (in.sp[s].start) c[s] = in.sp[s].n;
        collect_solver_stats(ctx, in);
        if (n_leaves) *n_leaves = in.nleaf;
        if (n_e) *n_e = c[0];
        if (n_i) *n_i = c[1];
        if (mg_cycles) *mg_cycles = in.mg_cycles;
        if (mg_rel_res) *mg_rel_res = in.mg_res;
        return PIC_OK;
    });
}

pic_status pic_get_step(const pic_ctx *ctx, int64_t *step) {
    if (!ctx || !step) {
        set_error("null argument");
        return PIC_EINVAL;
    }
    *step = ctx->step;
    return PIC_OK;
}

pic_status pic_set_step(pic_ctx *ctx, int64_t step) {
    if (!ctx || step < 0) {
        set_error("bad argument");
        return PIC_EINVAL;
    }
    ctx->step = step;
    return PIC_OK;
}

pic_status pic_set_timing(pic_ctx *ctx, int32_t on) {
    return guarded(ctx, [&]() -> pic_status {
        if (!ctx) fail(PIC_EINVAL, "null context");
        GB_CUDA(cudaStreamSynchronize(ctx->stream));
        for (auto &r : ctx->trec) {
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
        ctx->trec.clear();
        for (int k = 0; k < 16; ++k) {
            ctx->graph_ms[k] = 0.0;
            ctx->graph_launches[k] = 0;
        }
        ctx->timing = on != 0;
        return PIC_OK;
    });
}

pic_status pic_get_timing(pic_ctx *ctx, double *ms, int64_t *launches, int32_t n) {
    return guarded(ctx, [&]() -> pic_status {
        if (!ctx) fail(PIC_EINVAL, "null context");
        GB_CUDA(cudaStreamSynchronize(ctx->stream));
        const int m = std::min<int>(n, PIC_N_PHASES);
        for (int k = 0; k < m; ++k) {
            if (ms) ms[k] = 0.0;
            if (launches) launches[k] = 0;
        }
        for (auto &r : ctx->trec) {
            if (r.phase >= m) continue;
            float t = 0.f;
            GB_CUDA(cudaEventElapsedTime(&t, r.a, r.b));
            if (ms) ms[r.phase] += t;
            if (launches) launches[r.phase] += r.launches;
        }
        for (int k = 0; k < m && k < 16; ++k) {  // phases inside graph replays
            if (ms) ms[k] += ctx->graph_ms[k];
            if (launches) launches[k] += ctx->graph_launches[k];
        }
        return PIC_OK;
    });
}

pic_status pic_diag_enable(pic_ctx *ctx, int32_t inst, int32_t n_bins, double eps_max_ev, const double *region) {
    return guarded(ctx, [&]() -> pic_status {
        Instance &in = get_inst(ctx, inst);
        if (!in.has_mesh) fail(PIC_EINVAL, "mesh not set");
        if (n_bins < 0) fail(PIC_EINVAL, "n_bins < 0");
        if (region && !(region[0] < region[1] && region[2] < region[3])) fail(PIC_EINVAL, "empty region");
        diag_enable(ctx, in, n_bins, eps_max_ev, region);
        return PIC_OK;
    });
}

pic_status pic_diag_reset(pic_ctx *ctx, int32_t inst) {
    return guarded(ctx, [&]() -> pic_status {
        Instance &in = get_inst(ctx, inst);
        diag_reset(ctx, in);
        return PIC_OK;
    });
}

pic_status pic_read_eedf(pic_ctx *ctx, int32_t inst, double *f, int64_t cap, int64_t *n_out, int64_t *samples) {
    return guarded(ctx, [&]() -> pic_status {
        Instance &in = get_inst(ctx, inst);
        if (!in.diag.on) fail(PIC_EINVAL, "diagnostics are off (pic_diag_enable)");
        if (n_out) *n_out = in.diag.nbins;
        if (!f || cap < in.diag.nbins) fail(PIC_EINVAL, "output capacity too small");
        diag_read_eedf(ctx, in, f, samples);
        return PIC_OK;
    });
}

pic_status pic_check_stability(pic_ctx *ctx, int32_t inst, double *dx_over_debye, double *wpe_dt, double *t_e_ev) {
    return guarded(ctx, [&]() -> pic_status {
        Instance &in = get_inst(ctx, inst);
        if (!in.has_mesh) fail(PIC_EINVAL, "mesh not set");
        const pic_status st = stability_check(ctx, in, dx_over_debye, wpe_dt, t_e_ev);
        if (st == PIC_WARN_STABILITY) set_error("explicit-PIC limits exceeded (dx > 3 lambda_D or omega_pe dt > 1)");
        return st;
    });
}

pic_status pic_inject_fault(pic_ctx *ctx, int32_t kind, int64_t count) {
    return guarded(ctx, [&]() -> pic_status {
        if (!ctx) fail(PIC_EINVAL, "null context");
        switch (kind) {
        case PIC_FAULT_NONE:
            ctx->cache.fail_after = -1;
            ctx->fault_balance_sweeps = 0;
            break;
        case PIC_FAULT_ALLOC:
            if (count < 0) fail(PIC_EINVAL, "count < 0");
            ctx->cache.fail_after = count;
            break;
        case PIC_FAULT_BALANCE:
            if (count < 1 || count > 64) fail(PIC_EINVAL, "balance sweeps must be in [1, 64]");
            ctx->fault_balance_sweeps = (int32_t)count;
            break;
        default:
            fail(PIC_EINVAL, "unknown fault kind");
        }
        return PIC_OK;
    });
}

pic_status pic_checkpoint_write(pic_ctx *ctx, int32_t inst, void *buf, int64_t cap, int64_t *bytes) {
    return guarded(ctx, [&]() -> pic_status {
        Instance &in = get_inst(ctx, inst);
        if (!in.has_mesh) fail(PIC_EINVAL, "mesh not set");
        const int64_t need = checkpoint_write(ctx, in, buf, cap);
        if (bytes) *bytes = need;
        if (!buf || cap < need) fail(PIC_EINVAL, "checkpoint buffer too small");
        return PIC_OK;
    });
}

pic_status pic_checkpoint_read(pic_ctx *ctx, int32_t inst, const void *buf, int64_t bytes) {
    return guarded(ctx, [&]() -> pic_status {
        Instance &in = get_inst(ctx, inst);
        GB_CUDA(cudaStreamSynchronize(ctx->stream));
        checkpoint_read(ctx, in, buf, bytes);
        return PIC_OK;
    });
}

pic_status pic_get_launch_count(const pic_ctx *ctx, int64_t *launches) {
    if (!ctx || !launches) {
        set_error("null argument");
        return PIC_EINVAL;
    }
    *launches = ctx->launches;
    return PIC_OK;
}

const char *pic_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
