// lbm_engine.cu -- serving engine of liblbm.so (lbm_engine_*, declared in
// include/lbm.h): independent lattices resident on the device, admitted by device
// memory, advanced together by batched launches of the step kernel captured in CUDA
// graphs, retired as they finish so that queued requests take their place.
// Lattices with the near-contact force are batched too: their group's step starts
// with one batched launch of the near-contact pass over all of them.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/lbm.h"
#include "lbm_ctx.cuh"

using namespace lbm;

namespace lbm {
cudaError_t prepare_step_batched(int storage, bool unit_omega, int model);
}

namespace {

constexpr int kTileX = 32, kTileY = 8;
constexpr int kCandidates[] = {8, 16, 32, 64, 128};   // planes per CTA (block schedule)
constexpr int kDefaultT = 32;
constexpr int kTuneSteps = 4;                           // timed steps per candidate

struct Request {
    long long ticket = 0;
    lbm_params p{};
    size_t N = 0;
    std::vector<double> rr, rb, u;
    long long steps_total = 0, steps_done = 0;
    int state = 0;   // 0 queued, 1 resident, 2 finished, 3 result taken, 4 failed
    lbm_ctx* ctx = nullptr;
    size_t bytes = 0;
    long long t_submit = 0, t_admit = -1, t_retire = -1;
    std::vector<double> out_rr, out_rb, out_u, out_phi;
};

// Lattices of one storage format, relaxation class, model and near-contact class
// (none, or the halo class of h_cut): one batched launch of the step kernel per step,
// preceded for near-contact lattices by one batched launch of the near-contact pass
// (which also writes the ghost copies of their step's input), followed otherwise by
// one batched ghost-copy fill of the step's output.
struct Group {
    int storage = 0;
    bool unit = false;
    int model = 0;
    int nc = 0;          // 0: no near-contact force; else the halo class of the pass
    double h_cut = 0.0;
    std::vector<Request*> members;
    BatchLattice* d_tab[2] = {nullptr, nullptr};   // tables of the next two steps
    std::vector<BatchLattice> h_tab[2];
    NcBatchLattice* d_nc[2] = {nullptr, nullptr};  // near-contact tables of those steps
    std::vector<NcBatchLattice> h_nc[2];
    long long nc_blocks = 0, nc_ghost = 0;
    int ctas = 0;
    long long ghost = 0;
};

int nc_class(const lbm_ctx* c) {
    return c->p.A_nc > 0.0 ? nc_halo(ctx_h_cut(c)) : 0;
}

// Device memory a resident lattice holds: its context plus the FP64 staging of the
// host field exchanges (7 doubles per node).
size_t request_bytes(const lbm_params& p) {
    const size_t N = (size_t)p.nx * p.ny * p.nz;
    return lbm_footprint_bytes(&p) + 7 * N * sizeof(double);
}

}  // namespace

struct lbm_engine {
    lbm_engine_params ep{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int num_sms = 1;
    std::deque<Request*> queue;
    std::vector<Request*> resident;
    std::map<long long, std::unique_ptr<Request>> all;
    size_t used = 0, peak = 0;
    long long next_ticket = 1, ticks = 0;
    std::vector<Group> groups;
    cudaGraphExec_t graph = nullptr;
    bool graph_valid = false;
    int T = kDefaultT;
    std::map<std::string, int> tuned;
    std::string err;
};

namespace {

lbm_status efail(lbm_engine* e, lbm_status s, const std::string& msg) {
    if (e) e->err = msg;
    return s;
}

void free_groups(lbm_engine* e) {
    for (Group& g : e->groups)
        for (int j = 0; j < 2; ++j) {
            cudaFree(g.d_tab[j]);
            cudaFree(g.d_nc[j]);
        }
    e->groups.clear();
    if (e->graph) cudaGraphExecDestroy(e->graph);
    e->graph = nullptr;
    e->graph_valid = false;
}

// Batch composition: sizes, storage, relaxation class and model of the resident
// lattices.
std::string signature(const lbm_engine* e) {
    std::vector<std::string> parts;
    for (const Request* r : e->resident) {
        BatchLattice b;
        step_params_ahead(r->ctx, 0, 0, &b);
        const bool unit = !b.p.var_tau && b.p.omega0 == 1.0f;
        parts.push_back(std::to_string(r->p.nx) + "x" + std::to_string(r->p.ny) + "x" +
                        std::to_string(r->p.nz) + "s" + std::to_string(r->p.storage) +
                        (unit ? "u" : "v") + "m" + std::to_string(r->p.model) + "n" +
                        std::to_string(nc_class(r->ctx)));
    }
    std::sort(parts.begin(), parts.end());
    std::string s;
    for (const std::string& x : parts) s += x + ";";
    return s;
}

// One step of a group with the tables of step j (0 or 1): the batched near-contact
// pass (near-contact groups), the batched step kernel, and the batched ghost fill
// (other groups; near-contact groups get their ghost copies from the pass).
cudaError_t group_step(lbm_engine* e, Group& g, int j) {
    cudaError_t err = cudaSuccess;
    if (g.nc)
        err = launch_nc_batched(g.d_nc[j], (int)g.members.size(), g.nc_blocks, g.nc_ghost, g.storage,
                                g.h_cut, e->num_sms, e->stream);
    if (err == cudaSuccess)
        err = launch_step_batched(g.d_tab[j], (int)g.members.size(), g.ctas, g.storage, g.unit, g.model,
                                  e->stream);
    if (err == cudaSuccess && !g.nc && g.ghost > 0)
        err = launch_ghost_batched(g.d_tab[j], (int)g.members.size(), g.ghost, g.storage, e->num_sms,
                                   e->stream);
    return err;
}

// Tables of the next two steps for block schedule T and the graph replaying them.
cudaError_t build_batch(lbm_engine* e, int T) {
    free_groups(e);
    for (Request* r : e->resident) {
        BatchLattice b;
        step_params_ahead(r->ctx, 0, 0, &b);
        const bool unit = !b.p.var_tau && b.p.omega0 == 1.0f;
        const int ncc = nc_class(r->ctx);
        Group* g = nullptr;
        for (Group& x : e->groups)
            if (x.storage == r->p.storage && x.unit == unit && x.model == r->p.model && x.nc == ncc)
                g = &x;
        if (!g) {
            e->groups.emplace_back();
            g = &e->groups.back();
            g->storage = r->p.storage;
            g->unit = unit;
            g->model = r->p.model;
            g->nc = ncc;
            g->h_cut = ctx_h_cut(r->ctx);
        }
        g->members.push_back(r);
    }
    cudaError_t err = cudaSuccess;
    for (Group& g : e->groups) {
        err = prepare_step_batched(g.storage, g.unit, g.model);
        if (err == cudaSuccess && g.nc) err = prepare_nc_batched(g.storage, g.h_cut);
        if (err != cudaSuccess) return err;
        for (int j = 0; j < 2; ++j) {
            g.h_tab[j].resize(g.members.size());
            int ctas = 0;
            long long ghost = 0;
            for (size_t i = 0; i < g.members.size(); ++i) {
                const lbm_ctx* c = g.members[i]->ctx;
                const int nz = g.members[i]->p.nz;
                const int zparts = std::max(1, (nz + T - 1) / T);
                BatchLattice& b = g.h_tab[j][i];
                step_params_ahead(c, j, zparts, &b);
                b.cta_begin = ctas;
                b.ghost_begin = ghost;
                ctas += b.p.tiles_x * b.p.tiles_y * zparts;
                ghost += ghost_cells(b.p);
            }
            g.ctas = ctas;
            g.ghost = ghost;
            const size_t bytes = g.h_tab[j].size() * sizeof(BatchLattice);
            err = cudaMalloc((void**)&g.d_tab[j], bytes);
            if (err != cudaSuccess) return err;
            err = cudaMemcpyAsync(g.d_tab[j], g.h_tab[j].data(), bytes, cudaMemcpyHostToDevice, e->stream);
            if (err != cudaSuccess) return err;
            if (!g.nc) continue;
            // the near-contact pass of the same step: blocks and ghost-copy tasks of
            // every member, one after the other
            g.h_nc[j].resize(g.members.size());
            long long blocks = 0, gtasks = 0;
            for (size_t i = 0; i < g.members.size(); ++i) {
                NcBatchLattice& b = g.h_nc[j][i];
                nc_params_ahead(g.members[i]->ctx, j, &b);
                b.block_begin = blocks;
                b.ghost_begin = gtasks;
                blocks += nc_block_count(b.p);
                gtasks += b.p.ghost_f ? ghost_cells(b.p) : 0;
            }
            g.nc_blocks = blocks;
            g.nc_ghost = gtasks;
            const size_t nbytes = g.h_nc[j].size() * sizeof(NcBatchLattice);
            err = cudaMalloc((void**)&g.d_nc[j], nbytes);
            if (err != cudaSuccess) return err;
            err = cudaMemcpyAsync(g.d_nc[j], g.h_nc[j].data(), nbytes, cudaMemcpyHostToDevice, e->stream);
            if (err != cudaSuccess) return err;
        }
    }
    err = cudaStreamSynchronize(e->stream);
    if (err != cudaSuccess) return err;
    // the graph: two steps (tables 0 then 1), each one batched step launch and one
    // batched ghost fill per group
    cudaGraph_t graph = nullptr;
    err = cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal);
    if (err != cudaSuccess) return err;
    for (int j = 0; j < 2 && err == cudaSuccess; ++j)
        for (Group& g : e->groups)
            if (err == cudaSuccess) err = group_step(e, g, j);
    cudaError_t end = cudaStreamEndCapture(e->stream, &graph);
    if (err == cudaSuccess) err = end;
    if (err == cudaSuccess) err = cudaGraphInstantiate(&e->graph, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (err != cudaSuccess) return err;
    e->graph_valid = true;
    e->T = T;
    return cudaSuccess;
}

// One step with the step-0 tables, outside the graph (odd remainders).
cudaError_t single_step(lbm_engine* e) {
    cudaError_t err = cudaSuccess;
    for (Group& g : e->groups)
        if (err == cudaSuccess) err = group_step(e, g, 0);
    return err;
}

// Record k steps of the batched launches for the lattices they advance.
void advance_all(lbm_engine* e, long long k) {
    for (Request* r : e->resident) {
        advance_state(r->ctx, k);
        r->steps_done += k;
    }
}

// Graph replays of `pairs` x 2 steps, timed with events when ms != nullptr.
cudaError_t replay(lbm_engine* e, long long pairs, float* ms) {
    cudaEvent_t a = nullptr, b = nullptr;
    cudaError_t err = cudaSuccess;
    if (ms) {
        err = cudaEventCreate(&a);
        if (err == cudaSuccess) err = cudaEventCreate(&b);
        if (err == cudaSuccess) err = cudaEventRecord(a, e->stream);
    }
    for (long long i = 0; i < pairs && err == cudaSuccess; ++i) err = cudaGraphLaunch(e->graph, e->stream);
    if (ms && err == cudaSuccess) {
        err = cudaEventRecord(b, e->stream);
        if (err == cudaSuccess) err = cudaEventSynchronize(b);
        if (err == cudaSuccess) err = cudaEventElapsedTime(ms, a, b);
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    return err;
}

lbm_status admit(lbm_engine* e) {
    if (e->ep.policy == 1)   // shortest job first: fewest node-steps, then arrival
        std::stable_sort(e->queue.begin(), e->queue.end(), [](const Request* a, const Request* b) {
            return (double)a->N * a->steps_total < (double)b->N * b->steps_total;
        });
    while (!e->queue.empty() && (int)e->resident.size() < e->ep.max_slots) {
        Request* r = e->queue.front();
        if (e->used + r->bytes > e->ep.hbm_budget_bytes) break;   // in policy order
        e->queue.pop_front();
        lbm_params p = r->p;
        p.cuda_stream = e->stream;
        lbm_ctx* c = nullptr;
        lbm_status s = lbm_create(&p, &c);
        if (s == LBM_OK) s = lbm_set_fields(c, r->rr.data(), r->rb.data(), r->u.empty() ? nullptr : r->u.data(), 0);
        if (s != LBM_OK) {
            e->err = std::string("request ") + std::to_string(r->ticket) + ": " + lbm_last_error(c);
            lbm_destroy(c);
            r->state = 4;
            continue;
        }
        r->ctx = c;
        r->state = 1;
        r->t_admit = e->ticks;
        std::vector<double>().swap(r->rr);   // initial fields are on the device now
        std::vector<double>().swap(r->rb);
        std::vector<double>().swap(r->u);
        e->used += r->bytes;
        e->peak = std::max(e->peak, e->used);
        e->resident.push_back(r);
        e->graph_valid = false;
    }
    return LBM_OK;
}

lbm_status retire(lbm_engine* e, int* retired) {
    int n = 0;
    std::vector<Request*> keep;
    for (Request* r : e->resident) {
        if (r->steps_done < r->steps_total) {
            keep.push_back(r);
            continue;
        }
        r->out_rr.resize(r->N);
        r->out_rb.resize(r->N);
        r->out_u.resize(3 * r->N);
        r->out_phi.resize(r->N);
        const lbm_status s = lbm_get_fields(r->ctx, r->out_rr.data(), r->out_rb.data(), r->out_u.data(),
                                            r->out_phi.data(), 0);
        if (s != LBM_OK) e->err = std::string("request ") + std::to_string(r->ticket) + ": " + lbm_last_error(r->ctx);
        lbm_destroy(r->ctx);
        r->ctx = nullptr;
        r->state = s == LBM_OK ? 2 : 4;
        r->t_retire = e->ticks;
        e->used -= r->bytes;
        e->graph_valid = false;
        ++n;
    }
    e->resident.swap(keep);
    if (retired) *retired = n;
    return LBM_OK;
}

}  // namespace

extern "C" lbm_status lbm_engine_create(const lbm_engine_params* p, lbm_engine** out) {
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    if (!p || p->max_slots < 1 || p->chunk_steps < 2 || p->hbm_budget_bytes == 0 ||
        p->policy < 0 || p->policy > 1) {
        set_global_error("lbm_engine_create: need max_slots >= 1, chunk_steps >= 2, a budget, "
                         "policy 0 or 1");
        return LBM_EINVAL;
    }
    lbm_engine* e = new (std::nothrow) lbm_engine();
    if (!e) return LBM_ENOMEM;
    e->ep = *p;
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&e->num_sms, cudaDevAttrMultiProcessorCount, dev);
    e->stream = (cudaStream_t)p->cuda_stream;
    if (err == cudaSuccess && !e->stream) {
        // graphs are captured on the engine's stream: the legacy default stream cannot be
        err = cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking);
        e->own_stream = err == cudaSuccess;
    }
    if (err != cudaSuccess) {
        set_global_error(std::string("lbm_engine_create: ") + cudaGetErrorString(err));
        delete e;
        return LBM_ECUDA;
    }
    *out = e;
    return LBM_OK;
}

extern "C" lbm_status lbm_engine_submit(lbm_engine* e, const lbm_params* p, const double* rho_r,
                                        const double* rho_b, const double* u, long long steps,
                                        long long* ticket) {
    if (!e) return LBM_EINVAL;
    if (!p || !rho_r || !rho_b || !ticket) return efail(e, LBM_EINVAL, "p, rho_r, rho_b and ticket are required");
    if (steps < 1) return efail(e, LBM_EINVAL, "steps must be >= 1");
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return efail(e, LBM_EINVAL, "nx, ny, nz must be >= 1");
    if (p->inplace) return efail(e, LBM_EINVAL, "the engine keeps two population copies (inplace = 0)");
    std::unique_ptr<Request> r(new (std::nothrow) Request());
    if (!r) return efail(e, LBM_ENOMEM, "host allocation failed");
    r->p = *p;
    r->N = (size_t)p->nx * p->ny * p->nz;
    r->bytes = request_bytes(*p);
    if (r->bytes > e->ep.hbm_budget_bytes)
        return efail(e, LBM_ENOMEM, "request needs more device memory than the engine budget");
    r->rr.assign(rho_r, rho_r + r->N);
    r->rb.assign(rho_b, rho_b + r->N);
    if (u) r->u.assign(u, u + 3 * r->N);
    r->steps_total = steps;
    r->ticket = e->next_ticket++;
    r->t_submit = e->ticks;
    *ticket = r->ticket;
    e->queue.push_back(r.get());
    e->all[r->ticket] = std::move(r);
    return LBM_OK;
}

extern "C" lbm_status lbm_engine_tick(lbm_engine* e, int* resident, int* queued, int* retired,
                                      int* steps_advanced) {
    if (!e) return LBM_EINVAL;
    if (retired) *retired = 0;
    if (steps_advanced) *steps_advanced = 0;
    struct Range {   // host-side range over the tick (admission, steps, retirement)
        Range() { nvtxRangePushA("lbm_engine_tick"); }
        ~Range() { nvtxRangePop(); }
    } range;
    admit(e);
    if (resident) *resident = (int)e->resident.size();
    if (queued) *queued = (int)e->queue.size();
    if (e->resident.empty()) {
        ++e->ticks;
        return LBM_OK;
    }
    long long k = e->ep.chunk_steps;
    for (const Request* r : e->resident) k = std::min(k, r->steps_total - r->steps_done);
    if (k >= 2 && (k & 1)) --k;   // the graph runs pairs of steps
    cudaError_t err = cudaSuccess;
    long long done = 0;
    const bool have_batch = !e->resident.empty();
    if (have_batch && !e->graph_valid) {
        const std::string sig = signature(e);
        auto it = e->tuned.find(sig);
        const long long tune_need = (long long)kTuneSteps * (sizeof(kCandidates) / sizeof(int));
        if (it != e->tuned.end()) {
            err = build_batch(e, it->second);
        } else if (e->ep.autotune && k >= tune_need + 2) {
            // block schedule: time each candidate on real steps, keep the fastest
            int best_T = kDefaultT;
            float best = 1e30f;
            for (int T : kCandidates) {
                err = build_batch(e, T);
                float ms = 0.f;
                if (err == cudaSuccess) err = replay(e, 1, nullptr);   // first replay uploads the graph
                if (err == cudaSuccess) err = replay(e, kTuneSteps / 2 - 1, &ms);
                if (err != cudaSuccess) break;
                done += kTuneSteps;
                advance_all(e, kTuneSteps);
                if (ms < best) {
                    best = ms;
                    best_T = T;
                }
            }
            if (err == cudaSuccess) {
                e->tuned[sig] = best_T;
                err = build_batch(e, best_T);
            }
        } else {
            err = build_batch(e, kDefaultT);
        }
    }
    const long long left = have_batch ? k - done : 0;
    if (err == cudaSuccess && left >= 2) {
        err = replay(e, left / 2, nullptr);
        if (err == cudaSuccess) advance_all(e, left - (left & 1));
    }
    if (err == cudaSuccess && (left & 1)) {
        err = single_step(e);
        if (err == cudaSuccess) {
            advance_all(e, 1);
            e->graph_valid = false;   // the tables' step parity has flipped
        }
    }
    if (err == cudaSuccess) err = cudaStreamSynchronize(e->stream);
    if (err != cudaSuccess) {
        e->err = std::string("lbm_engine_tick: ") + cudaGetErrorString(err);
        return LBM_ECUDA;
    }
    for (Request* r : e->resident)
        if (check_errors(r->ctx) != LBM_OK) {
            e->err = std::string("request ") + std::to_string(r->ticket) + ": " + lbm_last_error(r->ctx);
            return LBM_ETIMEOUT;
        }
    if (steps_advanced) *steps_advanced = (int)k;
    retire(e, retired);
    if (!e->graph_valid) free_groups(e);
    ++e->ticks;
    return LBM_OK;
}

extern "C" int lbm_engine_state(const lbm_engine* e, long long ticket) {
    if (!e) return -1;
    auto it = e->all.find(ticket);
    return it == e->all.end() ? -1 : it->second->state;
}

extern "C" lbm_status lbm_engine_cancel(lbm_engine* e, long long ticket) {
    if (!e) return LBM_EINVAL;
    auto it = e->all.find(ticket);
    if (it == e->all.end()) return efail(e, LBM_EINVAL, "unknown ticket");
    Request* r = it->second.get();
    switch (r->state) {
        case 0:   // queued: leaves the queue
            e->queue.erase(std::remove(e->queue.begin(), e->queue.end(), r), e->queue.end());
            break;
        case 1: {   // resident: its lattice is freed once the queued work has drained
            cudaStreamSynchronize(e->stream);
            lbm_destroy(r->ctx);
            r->ctx = nullptr;
            e->used -= r->bytes;
            e->resident.erase(std::remove(e->resident.begin(), e->resident.end(), r),
                              e->resident.end());
            e->graph_valid = false;
            free_groups(e);
            break;
        }
        case 2:   // finished: its result is dropped
            break;
        default:
            return efail(e, LBM_ESTATE, "request already taken, failed or cancelled");
    }
    std::vector<double>().swap(r->rr);
    std::vector<double>().swap(r->rb);
    std::vector<double>().swap(r->u);
    std::vector<double>().swap(r->out_rr);
    std::vector<double>().swap(r->out_rb);
    std::vector<double>().swap(r->out_u);
    std::vector<double>().swap(r->out_phi);
    r->state = 5;
    return LBM_OK;
}

extern "C" lbm_status lbm_engine_result(lbm_engine* e, long long ticket, double* rho_r,
                                        double* rho_b, double* u, double* phi, long long info[4]) {
    if (!e) return LBM_EINVAL;
    auto it = e->all.find(ticket);
    if (it == e->all.end()) return efail(e, LBM_EINVAL, "unknown ticket");
    Request* r = it->second.get();
    if (r->state != 2) return efail(e, LBM_ESTATE, "request has not finished (or its result was taken)");
    const size_t N = r->N;
    if (rho_r) std::memcpy(rho_r, r->out_rr.data(), N * sizeof(double));
    if (rho_b) std::memcpy(rho_b, r->out_rb.data(), N * sizeof(double));
    if (u) std::memcpy(u, r->out_u.data(), 3 * N * sizeof(double));
    if (phi) std::memcpy(phi, r->out_phi.data(), N * sizeof(double));
    if (info) {
        info[0] = r->steps_done;
        info[1] = r->t_submit;
        info[2] = r->t_admit;
        info[3] = r->t_retire;
    }
    std::vector<double>().swap(r->out_rr);
    std::vector<double>().swap(r->out_rb);
    std::vector<double>().swap(r->out_u);
    std::vector<double>().swap(r->out_phi);
    r->state = 3;
    return LBM_OK;
}

extern "C" void lbm_engine_stats(const lbm_engine* e, long long out[7]) {
    if (!e || !out) return;
    out[0] = e->ticks;
    out[1] = (long long)e->resident.size();
    out[2] = (long long)e->queue.size();
    out[3] = (long long)e->used;
    out[4] = (long long)e->peak;
    out[5] = e->T;
    out[6] = (long long)e->groups.size();
}

extern "C" void lbm_engine_destroy(lbm_engine* e) {
    if (!e) return;
    if (e->stream) cudaStreamSynchronize(e->stream);
    free_groups(e);
    for (Request* r : e->resident) lbm_destroy(r->ctx);
    if (e->own_stream) cudaStreamDestroy(e->stream);
    delete e;
}

extern "C" const char* lbm_engine_last_error(const lbm_engine* e) {
    return e ? e->err.c_str() : "";
}
