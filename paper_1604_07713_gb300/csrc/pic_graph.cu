// A batched ensemble's step as one CUDA graph, and the end-of-call report of every instance.
//
// Every instance's step is a few dozen small launches (deposit, corner field, push, list
// repairs, sorts); with hundreds of instances the host spends more time launching them than
// the GPU spends running them.  Once every instance is in steady state (its Poisson solve fits
// the batched one-block solver, its deposit sums are valid), one step of all instances is
// captured as a graph and replayed: the launches of different instances sit on parallel
// branches (instances are independent), so their small kernels overlap on the GPU.  The step
// number and the wall potentials of each step are read on the device, from values the host
// writes there (from the same formula as an uncaptured step) before each replay.  The graph
// is captured again after anything that moves a buffer (load, adaptation, capacity growth,
// mesh change).
#include <algorithm>
#include <array>
#include <cmath>
#include <vector>

#include "pic_internal.cuh"

namespace gbpic {

namespace {
constexpr int kT = 256;

// One entry per instance: what the end-of-call report reads.
struct ReportTab {
    const int32_t *start[2], *end[2];
    int64_t nleaf;
    int32_t nsp;
    const int32_t *err;
    const double *mg_stats;  // null: the instance's solves report on the host
};
struct Report {
    int32_t tot[2];
    int32_t err, pad;
    double mg[3];  // cycles, relative residual, worst relative residual since the reset
};

// Blocks (x) over the leaves of instance y: record totals per species (out zeroed before),
// and from block 0 the consistency flag and the solver statistics.
__global__ void k_report(const ReportTab *__restrict__ tab, Report *__restrict__ out) {
    __shared__ int32_t part[kT / 32];
    const ReportTab &t = tab[blockIdx.y];
    Report &r = out[blockIdx.y];
    for (int s = 0; s < 2; ++s) {
        int32_t c = 0;
        if (s < t.nsp)
            for (int64_t L = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; L < t.nleaf;
                 L += (int64_t)gridDim.x * blockDim.x)
                c += t.end[s][L] - t.start[s][L];
        for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xFFFFFFFFu, c, o);
        if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = c;
        __syncthreads();
        if (threadIdx.x == 0) {
            int32_t tot = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) tot += part[w];
            if (tot) atomicAdd(&r.tot[s], tot);
        }
        __syncthreads();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        r.err = *t.err;
        r.pad = 0;
        for (int k = 0; k < 3; ++k) r.mg[k] = t.mg_stats ? t.mg_stats[k] : 0.0;
    }
}

// The parallel branches of a captured step (their number is a tuned launch shape).
void ensure_branches(pic_ctx *ctx) {
    const size_t nb = (size_t)std::max(1, ctx->tune.branches);
    if (ctx->fork.size() == nb) return;
    for (auto &s : ctx->fork) cudaStreamDestroy(s);
    for (auto &e : ctx->fork_ev) cudaEventDestroy(e);
    ctx->fork.assign(nb, nullptr);
    ctx->fork_ev.assign(nb + 1, nullptr);
    for (auto &s : ctx->fork) GB_CUDA(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    for (auto &e : ctx->fork_ev) GB_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
}

// The branches wait for what `main` has issued so far.
void fork_from(pic_ctx *ctx, cudaStream_t main) {
    GB_CUDA(cudaEventRecord(ctx->fork_ev[0], main));
    for (auto &s : ctx->fork) GB_CUDA(cudaStreamWaitEvent(s, ctx->fork_ev[0], 0));
}
// `main` waits for everything the branches have issued.
void join_into(pic_ctx *ctx, cudaStream_t main) {
    for (size_t j = 0; j < ctx->fork.size(); ++j) {
        GB_CUDA(cudaEventRecord(ctx->fork_ev[1 + j], ctx->fork[j]));
        GB_CUDA(cudaStreamWaitEvent(main, ctx->fork_ev[1 + j], 0));
    }
}

void capture_step(pic_ctx *ctx) {
    graph_release(ctx);
    const int n = (int)ctx->inst.size();
    std::vector<std::array<double, 4>> walls(n);
    for (int i = 0; i < n; ++i) walls_at(ctx->inst[i], ctx->step, walls[i].data());
    std::vector<Instance *> list;
    std::vector<const double *> wl;
    for (int i = 0; i < n; ++i) {
        list.push_back(&ctx->inst[i]);
        wl.push_back(walls[i].data());
    }
    const bool batched = batch_possible(ctx);
    if (batched) {  // the tables of the batched launches, uploaded before the capture
        poisson_batch_items(ctx, list);
        batch_prepare_particles(ctx);
        batch_prepare_node_e(ctx);
        GB_CUDA(cudaStreamSynchronize(ctx->stream));
    } else {
        ensure_branches(ctx);
    }
    cudaStream_t cs;
    GB_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaStream_t saved = ctx->stream;
    const bool saved_timing = ctx->timing;
    const int64_t l0 = ctx->launches;
    ctx->timing = false;
    ctx->capturing = true;
    ctx->capture_phases = batched && saved_timing;  // a linear graph: phases in sequence
    if (ctx->capture_phases)
        while (ctx->event_pool.size() < 32) {  // two per phase of the step
            cudaEvent_t ev = nullptr;
            GB_CUDA(cudaEventCreate(&ev));
            ctx->event_pool.push_back(ev);
        }
    ctx->stream = cs;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    try {
        if (e != cudaSuccess) GB_CUDA(e);
        if (batched) {
            // one launch per phase over every instance
            {
                Phase ph(ctx, PIC_PHASE_DEPOSIT);
                deposit_batch(ctx);
            }
            {
                Phase ph(ctx, PIC_PHASE_POISSON);
                poisson_solve_batch(ctx, list, wl);
            }
            {
                Phase ph(ctx, PIC_PHASE_NODE_E);
                node_e_batch(ctx);
            }
            particle_step_batch(ctx);
        } else {
            // deposits, branch per instance
            fork_from(ctx, cs);
            for (int i = 0; i < n; ++i) {
                ctx->stream = ctx->fork[i % ctx->fork.size()];
                deposit(ctx, ctx->inst[i], walls[i].data());
            }
            ctx->stream = cs;
            join_into(ctx, cs);
            // one launch solves every instance's Poisson problem
            poisson_solve_batch(ctx, list, wl);
            // corner fields and particle steps, branch per instance
            fork_from(ctx, cs);
            for (int i = 0; i < n; ++i) {
                ctx->stream = ctx->fork[i % ctx->fork.size()];
                node_e(ctx, ctx->inst[i], walls[i].data());
                particle_step(ctx, ctx->inst[i], ctx->step, false);
            }
            ctx->stream = cs;
            join_into(ctx, cs);
        }
        e = cudaStreamEndCapture(cs, &graph);
    } catch (...) {
        cudaStreamEndCapture(cs, &graph);
        if (graph) cudaGraphDestroy(graph);
        ctx->stream = saved;
        ctx->timing = saved_timing;
        ctx->capturing = false;
        ctx->capture_phases = false;
        ctx->launches = l0;
        cudaStreamDestroy(cs);
        throw;
    }
    ctx->stream = saved;
    ctx->timing = saved_timing;
    ctx->capturing = false;
    ctx->graph_timed = ctx->capture_phases;
    ctx->capture_phases = false;
    ctx->batch.on = batched;
    ctx->graph_nodes = ctx->launches - l0;
    ctx->launches = l0;
    cudaStreamDestroy(cs);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ctx->step_graph, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    GB_CUDA(e);
    ctx->graph_mesh_epoch = ctx->mesh_epoch;
    ctx->graph_lists_epoch = ctx->lists_epoch;
    ctx->graph_tune_epoch = ctx->tune.epoch;
}

bool graph_current(const pic_ctx *ctx) {
    // a batched step is captured with phase events exactly when timing is on
    const bool timed_ok = !batch_possible(const_cast<pic_ctx *>(ctx)) || ctx->graph_timed == ctx->timing;
    return ctx->step_graph && ctx->graph_mesh_epoch == ctx->mesh_epoch && ctx->graph_lists_epoch == ctx->lists_epoch &&
           ctx->graph_tune_epoch == ctx->tune.epoch && timed_ok;
}
}  // namespace

// Capture (if the captured step is out of date) and upload the step graph now, so that the
// next replay does no host work beyond the launch.
void graph_prepare(pic_ctx *ctx) {
    if (!graph_current(ctx)) capture_step(ctx);
    GB_CUDA(cudaGraphUpload(ctx->step_graph, ctx->stream));
}

void one_step(pic_ctx *ctx) {
    for (Instance &in : ctx->inst) ensure_capacity(ctx, in);
    if (graph_step_possible(ctx)) {
        graph_step(ctx);  // an ensemble in steady state: the whole step as one graph replay
    } else {
        // the direct implicit scheme (§3 DIPIC): the predictor before the field of the step
        for (Instance &in : ctx->inst)
            if (in.cfg.implicit) particle_step(ctx, in, ctx->step, true, PUSH_PREDICT);
        fields_all(ctx, ctx->step);
        for (Instance &in : ctx->inst) {
            diag_accumulate(ctx, in);  // time averages of the step's state (when enabled)
            particle_step(ctx, in, ctx->step, true, in.cfg.implicit ? PUSH_CORRECT : PUSH_LEAPFROG);
        }
    }
    ++ctx->step;
}

// Steady state of every instance of an ensemble: batched one-block Poisson solves and valid
// deposit sums for every species (so the step has no host decision left).
bool graph_step_possible(pic_ctx *ctx) {
    if (ctx->inst.size() < 2) return false;
    for (Instance &in : ctx->inst) {
        if (!in.has_mesh || !in.small_item || in.diag.on || in.cfg.implicit) return false;
        for (int s = 0; s < in.cfg.n_species; ++s)
            if (!in.sp[s].start || !in.sp[s].sums_valid) return false;
    }
    return true;
}

void graph_step(pic_ctx *ctx) {
    if (!graph_current(ctx)) capture_step(ctx);
    // this step's number and wall potentials, as an uncaptured step computes them (pageable
    // source: the copies are staged before they return, so the buffer may be reused)
    const int n = (int)ctx->inst.size();
    std::vector<double> walls(4 * (size_t)n);
    for (int i = 0; i < n; ++i) walls_at(ctx->inst[i], ctx->step, walls.data() + 4 * i);
    const int64_t step = ctx->step;
    GB_CUDA(cudaMemcpyAsync(ctx->d_walls, walls.data(), walls.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
    GB_CUDA(cudaMemcpyAsync(ctx->d_step, &step, 8, cudaMemcpyHostToDevice, ctx->stream));
    {
        Phase ph(ctx, PIC_PHASE_GRAPH);
        GB_CUDA(cudaGraphLaunch(ctx->step_graph, ctx->stream));
        count_launch(ctx, ctx->graph_nodes);
    }
    if (ctx->timing && ctx->graph_timed) {  // the phases inside this replay
        GB_CUDA(cudaStreamSynchronize(ctx->stream));
        for (const TimingRec &r : ctx->graph_trec) {
            float t = 0.f;
            GB_CUDA(cudaEventElapsedTime(&t, r.a, r.b));
            ctx->graph_ms[r.phase] += t;
            ctx->graph_launches[r.phase] += r.launches;
        }
    }
    // the host side of what the replay did
    for (Instance &in : ctx->inst) {
        walls_at(in, ctx->step, in.last_walls);
        in.mg_on_device = true;
        particle_bookkeeping(in);
    }
}

void graph_release(pic_ctx *ctx) {
    if (ctx->step_graph) {
        cudaGraphExecDestroy(ctx->step_graph);
        ctx->step_graph = nullptr;
    }
    if (!ctx->graph_trec.empty()) {
        cudaStreamSynchronize(ctx->stream);
        for (auto &r : ctx->graph_trec) {  // back to the pool
            ctx->event_pool.push_back(r.a);
            ctx->event_pool.push_back(r.b);
        }
        ctx->graph_trec.clear();
    }
    ctx->graph_timed = false;
    if (!ctx->batch.bufs.empty()) {  // a replay in flight may still read the tables
        cudaStreamSynchronize(ctx->stream);
        for (void *p : ctx->batch.bufs) cudaFree(p);
    }
    ctx->batch = BatchStep{};
}

// The batched step needs one kernel instantiation for all instances: every instance with the
// nearest-grid-point shape (the cloud-in-cell push gathers from a patch per leaf) and one
// precision.
bool batch_possible(pic_ctx *ctx) {
    for (const Instance &in : ctx->inst)
        if (in.cfg.shape != PIC_SHAPE_NGP || in.cfg.precision != ctx->inst.front().cfg.precision) return false;
    return !ctx->inst.empty();
}

void *batch_upload(pic_ctx *ctx, const void *src, size_t bytes) {
    void *p = nullptr;
    GB_CUDA(cudaMalloc(&p, std::max<size_t>(bytes, 16)));
    ctx->batch.bufs.push_back(p);
    if (src && bytes) GB_CUDA(cudaMemcpyAsync(p, src, bytes, cudaMemcpyHostToDevice, ctx->stream));
    else GB_CUDA(cudaMemsetAsync(p, 0, std::max<size_t>(bytes, 16), ctx->stream));
    GB_CUDA(cudaStreamSynchronize(ctx->stream));  // the host table may go out of scope
    return p;
}

std::vector<int4> batch_chunks(const std::vector<int64_t> &nleaf, int64_t per) {
    std::vector<int4> ch;
    for (size_t k = 0; k < nleaf.size(); ++k)
        for (int64_t lb = 0; lb < nleaf[k]; lb += per)
            ch.push_back(make_int4((int)k, (int)lb, (int)std::min<int64_t>(nleaf[k], lb + per), 0));
    return ch;
}

void report_all(pic_ctx *ctx) {
    const int n = (int)ctx->inst.size();
    cudaStream_t st = ctx->stream;
    const int64_t epoch = ctx->mesh_epoch * 1000003 + ctx->lists_epoch;
    if (!ctx->report_dev) {
        GB_CUDA(cudaMalloc(&ctx->report_dev, n * sizeof(Report)));
        GB_CUDA(cudaMallocHost(&ctx->report_host, n * sizeof(Report)));
        GB_CUDA(cudaMalloc(&ctx->report_tab, n * sizeof(ReportTab)));
    }
    if (ctx->report_epoch != epoch) {
        std::vector<ReportTab> tab(n);
        for (int i = 0; i < n; ++i) {
            Instance &in = ctx->inst[i];
            ReportTab &t = tab[i];
            t.nsp = in.cfg.n_species;
            t.nleaf = in.nleaf;
            for (int s = 0; s < 2; ++s) {
                t.start[s] = s < t.nsp ? in.sp[s].start : nullptr;
                t.end[s] = s < t.nsp ? in.sp[s].end : nullptr;
            }
            t.err = in.d_err;
            t.mg_stats = in.mg_stats;
        }
        GB_CUDA(cudaMemcpyAsync(ctx->report_tab, tab.data(), n * sizeof(ReportTab), cudaMemcpyHostToDevice, st));
        GB_CUDA(cudaStreamSynchronize(st));  // the host vector goes out of scope
        ctx->report_epoch = epoch;
    }
    int64_t maxl = 0;
    for (Instance &in : ctx->inst) maxl = std::max(maxl, in.nleaf);
    const dim3 grid((unsigned)std::min<int64_t>(std::max<int64_t>(1, (maxl + 8 * kT - 1) / (8 * kT)), 128), n);
    GB_CUDA(cudaMemsetAsync(ctx->report_dev, 0, n * sizeof(Report), st));
    k_report<<<grid, kT, 0, st>>>((const ReportTab *)ctx->report_tab, (Report *)ctx->report_dev);
    count_launch(ctx);
    GB_CUDA(cudaMemcpyAsync(ctx->report_host, ctx->report_dev, n * sizeof(Report), cudaMemcpyDeviceToHost, st));
    GB_CUDA(cudaStreamSynchronize(st));
    const Report *r = (const Report *)ctx->report_host;
    for (int i = 0; i < n; ++i) {
        Instance &in = ctx->inst[i];
        for (int s = 0; s < in.cfg.n_species; ++s) in.sp[s].n = in.sp[s].n_upper = r[i].tot[s];
        in.report_err = r[i].err;
        if (in.mg_on_device && in.mg_stats) {
            in.mg_cycles = (int)r[i].mg[0];
            in.mg_res = r[i].mg[1];
            in.mg_worst = worst_residual_host(in.mg_res_max, r[i].mg[2]);
            if (in.mg_count_cycles) {  // kernels of the device-side cycle loop of the last solve
                ctx->launches += (int64_t)in.mg_cycles * in.mg_cycle_nodes;
                in.mg_count_cycles = false;
            }
        } else {
            in.mg_worst = in.mg_res_max;
        }
    }
}

}  // namespace gbpic
