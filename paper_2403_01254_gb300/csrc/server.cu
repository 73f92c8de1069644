// Request server: continuous batching of RKHS-BA solves on one GPU.
//
// Two host threads drive the device.  The admission thread takes queued
// requests while an in-flight slot is free and the device-memory budget has
// room, builds each problem (upload + grid step + the evaluation at the
// initial poses) on the slot's stream and hands it to the stepping thread.
//
// The stepping thread advances every admitted problem by one LM iteration
// per round (the loop of rkhsba_solve: solve, evaluate, accept; Sec. V-A,
// V-C).  In the default batched mode a round is: each problem's damped solve
// and query binning on its own stream (a replayed CUDA graph), then ONE
// persistent pair launch over the units of all problems that share a label
// layout (the sum of Eq. inner_product_actual_ba over every edge of every
// admitted problem, each problem adding into its own fixed-point
// accumulators), then each problem's FP64 assembly and accept/reject on its
// own stream (a second graph).  In the per-request mode each problem runs
// whole iterations on its own stream, a few per issue.  Requests whose LM
// state says done are finished after the round: poses copied out, context
// destroyed, slot and memory released, pollers and the admission thread
// woken.  Because every evaluation is exact in its reductions (fixed point)
// and stable in its sorts, a request's result does not depend on which other
// requests share the GPU, nor on the mode.
//
// With autotuning on, the first request of each workload class (label layout
// and density class) is timed under the autotuner's candidate settings
// (rkhsba_autotune) before it is built, and the chosen setting is used for it
// and every later request of that class.
#include "common.cuh"
#include "rkhsba.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

namespace {
using namespace rk;
using Clock = std::chrono::steady_clock;

enum ReqState { RQ_QUEUED = 0, RQ_RUNNING = 1, RQ_DONE = 2, RQ_FAILED = 3, RQ_CANCELLED = 4 };

struct Req {
    int64_t ticket = 0;
    int K = 0, E = 0;
    std::vector<int64_t> n;
    std::vector<double> xyz;
    std::vector<float> sem, rgb;
    std::vector<int32_t> edges;
    rkhsba_params p{};
    std::vector<double> poses0;
    size_t est = 0, bytes = 0;
    int state = RQ_QUEUED;
    int status = RKHSBA_OK;
    std::atomic<bool> cancel{false};
    rkhsba_ctx* ctx = nullptr;
    int slot = -1;
    cudaEvent_t ev = nullptr;        // end of the last issued work
    bool started = false;
    bool inflight = false;           // batched mode: an issued iteration has not completed
    LMState* mirror = nullptr;       // batched mode: pinned copy of the LM state after each iteration
    int cost_class = 0;              // batched mode: total points < 64k, < 256k, < 1M, more
    int issued = 0;
    Clock::time_point t_submit, t_admit, t_done;
    rkhsba_solve_info info{};
    std::vector<double> result;
};

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

// Device bytes a problem will hold, from its sizes (mirrors the buffers of
// rkhsba_create): points, labels, sort buffers, grids over the frames'
// bounding boxes, per-edge queries and home cells, and the 6K system.
size_t estimate_bytes(const Req& r) {
    const double rc = (r.p.cutoff_mult > 0 ? r.p.cutoff_mult : 3.0) * r.p.ell;
    const double h = rc * (1.0 + 1.0 / 1024.0);
    std::vector<double> cells(r.K, 1.0);
    long long off = 0;
    for (int m = 0; m < r.K; ++m) {
        if (r.n[m] > 0) {
            double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
            for (long long i = off; i < off + r.n[m]; ++i)
                for (int k = 0; k < 3; ++k) {
                    lo[k] = std::min(lo[k], r.xyz[3 * i + k]);
                    hi[k] = std::max(hi[k], r.xyz[3 * i + k]);
                }
            double c = 1.0;
            for (int k = 0; k < 3; ++k) c *= std::floor((hi[k] - lo[k]) / h) + 4.0;
            cells[m] = c;
        }
        off += r.n[m];
    }
    double N = (double)off, Q = 0, bins = 0, C = 0;
    for (int m = 0; m < r.K; ++m) C += cells[m];
    for (int e = 0; e < r.E; ++e) {
        int a = std::min(r.edges[2 * e], r.edges[2 * e + 1]), b = std::max(r.edges[2 * e], r.edges[2 * e + 1]);
        Q += (double)r.n[b];
        bins += cells[a];
    }
    const double D = r.p.sem_dim;
    const double bytes = N * (24 + 8 * D + 16 + 16 + 40 + 12) + Q * 68 + bins * 4 + C * 4 +
                         (double)r.K * r.K * 36 * 8 * 2 + (double)r.E * 1600 + (4 << 20);
    return (size_t)(bytes * 1.25);
}
}  // namespace

struct rkhsba_server {
    rkhsba_server_config cfg{};
    std::vector<cudaStream_t> streams;
    std::vector<int> free_slots;
    std::mutex mu;
    std::condition_variable cv_admit;   // admission thread: queue or resources changed
    std::condition_variable cv_done;    // pollers: a request ended
    std::condition_variable cv_step;    // stepping thread: new running request
    std::deque<Req*> queue;
    std::vector<Req*> running;
    std::unordered_map<int64_t, Req*> all;
    size_t mem_in_use = 0;
    int64_t next_ticket = 1;
    int64_t finished = 0;
    bool stop = false;
    std::thread admit_thr, step_thr;
    int device = 0;

    // batched mode: each round takes a free round slot -- a stream, pinned
    // host and device job records, unit counters and an event marking the
    // end of its batched launches -- so the launches of different rounds do
    // not wait for each other and no copy waits on the host.  A round holds
    // at least one request and a request is in at most one pending round, so
    // max_inflight + 1 slots always leave one free.
    struct RoundSlot {
        cudaStream_t stream = nullptr;
        cudaEvent_t ev_mid = nullptr;
        PairJob* h_jobs = nullptr;      // pinned [max_inflight]
        PairJob* d_jobs = nullptr;      // [max_inflight]
        int* d_counters = nullptr;      // [max_inflight]
    };
    std::vector<RoundSlot> rounds;
    LMState* h_mirror = nullptr;        // [max_inflight] pinned LM-state copies, one per request slot
    int num_sms = 1;

    // autotuning: per workload class (label layout, density class) the chosen setting
    struct Tuned { int key; rkhsba_tuning t; };
    std::vector<Tuned> tuned;
    std::mutex tune_mu;

    void release_rounds() {
        for (auto& x : rounds) {
            if (x.stream) {
                cudaStreamSynchronize(x.stream);
                cudaStreamDestroy(x.stream);
            }
            if (x.ev_mid) cudaEventDestroy(x.ev_mid);
            if (x.h_jobs) cudaFreeHost(x.h_jobs);
            cudaFree(x.d_jobs);
            cudaFree(x.d_counters);
        }
        rounds.clear();
        if (h_mirror) cudaFreeHost(h_mirror);
        h_mirror = nullptr;
    }
    void admit_loop();
    void step_loop();
    void step_loop_batched();
    void issue_round(const std::vector<Req*>& batch, int n_iter);
    bool tuning_for(Req* r, rkhsba_tuning* t);
    void finish(Req* r, int state, int status);   // called without mu held
};

void rkhsba_server::finish(Req* r, int state, int status) {
    if (r->ctx) {
        if (state == RQ_DONE) {
            LMState s{};
            cudaStream_t st = ctx_stream(r->ctx);
            cudaError_t e1 = cudaMemcpyAsync(&s, ctx_state_dev(r->ctx), sizeof(LMState), cudaMemcpyDeviceToHost, st);
            r->result.assign((size_t)16 * r->K, 0.0);
            cudaError_t e2 = cudaMemcpyAsync(r->result.data(), ctx_poses_dev(r->ctx), sizeof(double) * 16 * r->K,
                                             cudaMemcpyDeviceToHost, st);
            cudaError_t e3 = cudaStreamSynchronize(st);
            if (e1 != cudaSuccess || e2 != cudaSuccess || e3 != cudaSuccess) {
                state = RQ_FAILED;
                status = RKHSBA_ECUDA;
            } else {
                r->info.iters = s.iters;
                r->info.status = s.done ? s.status : RKHSBA_ENOTCONV;
                r->info.final_loss = -s.F_cur;
                r->info.lambda = s.lambda;
                r->info.pair_terms = s.pair_terms;
                status = r->info.status;
            }
        }
        rkhsba_destroy(r->ctx);
        r->ctx = nullptr;
    }
    if (r->ev) {
        cudaEventDestroy(r->ev);
        r->ev = nullptr;
    }
    {
        std::lock_guard<std::mutex> lk(mu);
        if (r->slot >= 0) free_slots.push_back(r->slot);
        r->slot = -1;
        mem_in_use -= std::min(mem_in_use, r->bytes);
        r->state = state;
        r->status = status;
        r->t_done = Clock::now();
        running.erase(std::remove(running.begin(), running.end(), r), running.end());
        r->xyz.clear(); r->xyz.shrink_to_fit();
        r->sem.clear(); r->sem.shrink_to_fit();
        r->rgb.clear(); r->rgb.shrink_to_fit();
        ++finished;
    }
    cv_done.notify_all();
    cv_admit.notify_all();
}

void rkhsba_server::admit_loop() {
    cudaSetDevice(device);
    for (;;) {
        Req* r = nullptr;
        int slot = -1;
        {
            std::unique_lock<std::mutex> lk(mu);
            for (;;) {
                if (stop) return;
                // drop cancelled requests at the head of the queue
                while (!queue.empty() && queue.front()->cancel) {
                    Req* c = queue.front();
                    queue.pop_front();
                    c->state = RQ_CANCELLED;
                    c->status = RKHSBA_OK;
                    c->t_done = Clock::now();
                    ++finished;
                    cv_done.notify_all();
                }
                if (!queue.empty() && !free_slots.empty()) {
                    Req* q = queue.front();
                    // admit by memory; a request larger than the whole budget
                    // runs alone once nothing else holds memory
                    if (mem_in_use + q->est <= (size_t)cfg.memory_budget || mem_in_use == 0) break;
                }
                cv_admit.wait(lk);
            }
            r = queue.front();
            queue.pop_front();
            slot = free_slots.back();
            free_slots.pop_back();
            r->slot = slot;
            mem_in_use += r->est;
            r->state = RQ_RUNNING;
            r->t_admit = Clock::now();
        }
        rkhsba_ctx* ctx = nullptr;
        rkhsba_tuning tune{};
        const bool tuned_ok = cfg.autotune && tuning_for(r, &tune);
        if (tuned_ok) r->p.cell_scale = tune.cell_scale;
        rkhsba_status s = rkhsba_create(&ctx, r->K, r->n.data(), r->xyz.data(), r->sem.empty() ? nullptr : r->sem.data(),
                                        r->rgb.empty() ? nullptr : r->rgb.data(), r->E, r->edges.data(), &r->p,
                                        (void*)streams[slot]);
        if (s == RKHSBA_OK && tuned_ok) s = rkhsba_set_tuning(ctx, tune.unit_queries, tune.ctas_per_sm);
        if (s == RKHSBA_OK) s = ctx_begin_solve(ctx, r->poses0.data());
        cudaEvent_t ev = nullptr;
        if (s == RKHSBA_OK && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) s = RKHSBA_ECUDA;
        if (s != RKHSBA_OK) {
            r->ctx = ctx;
            r->ev = ev;
            {
                std::lock_guard<std::mutex> lk(mu);
                mem_in_use -= std::min(mem_in_use, r->est);
                r->est = 0;
            }
            finish(r, RQ_FAILED, s);
            continue;
        }
        if (h_mirror) {
            r->mirror = h_mirror + slot;
            r->mirror->done = 0;
        }
        {
            std::lock_guard<std::mutex> lk(mu);
            r->ctx = ctx;
            r->ev = ev;
            const size_t real = ctx_bytes(ctx);
            mem_in_use = mem_in_use - std::min(mem_in_use, r->est) + real;
            r->bytes = real;
            running.push_back(r);
        }
        cv_step.notify_all();
    }
}

void rkhsba_server::step_loop() {
    cudaSetDevice(device);
    const int chunk = std::max(1, cfg.iters_per_issue);
    std::vector<Req*> snap;
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(mu);
            if (stop) return;
            if (running.empty()) cv_step.wait_for(lk, std::chrono::milliseconds(5));
            if (stop) return;
            snap = running;
        }
        bool issued = false;
        for (Req* r : snap) {
            if (r->cancel) {
                if (r->started) cudaEventSynchronize(r->ev);
                finish(r, RQ_CANCELLED, RKHSBA_OK);
                continue;
            }
            if (cfg.request_timeout_ms > 0 && ms_between(r->t_admit, Clock::now()) > cfg.request_timeout_ms) {
                if (r->started) cudaEventSynchronize(r->ev);
                finish(r, RQ_FAILED, RKHSBA_ETIMEOUT);
                continue;
            }
            if (!r->started) {
                r->started = true;
                ctx_iterate(r->ctx, chunk);
                r->issued = chunk;
                cudaEventRecord(r->ev, ctx_stream(r->ctx));
                issued = true;
                continue;
            }
            const cudaError_t q = cudaEventQuery(r->ev);
            if (q == cudaErrorNotReady) continue;
            if (q != cudaSuccess) {
                finish(r, RQ_FAILED, RKHSBA_ECUDA);
                continue;
            }
            LMState s{};
            cudaStream_t rs = ctx_stream(r->ctx);
            if (cudaMemcpyAsync(&s, ctx_state_dev(r->ctx), sizeof(LMState), cudaMemcpyDeviceToHost, rs) != cudaSuccess ||
                cudaStreamSynchronize(rs) != cudaSuccess) {
                finish(r, RQ_FAILED, RKHSBA_ECUDA);
                continue;
            }
            if (s.done || r->issued >= ctx_max_iters(r->ctx)) {
                finish(r, RQ_DONE, RKHSBA_OK);
                continue;
            }
            ctx_iterate(r->ctx, std::min(chunk, ctx_max_iters(r->ctx) - r->issued));
            r->issued += chunk;
            cudaEventRecord(r->ev, ctx_stream(r->ctx));
            issued = true;
        }
        if (!issued) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

// Workload class of a request for autotuning: its label layout (the
// template class of its pair kernel) and its density class (mean points per
// frame below 16k, below 64k, or more), since the best setting of a small
// problem is not that of a large one.
static int workload_class(const Req& r) {
    const rkhsba_params& p = r.p;
    const int pad = p.sem_dim > 0 ? (p.sem_dim + 3) / 4 : 0;
    const int layout = pad * 4 + (p.sem_bf16 ? 2 : 0) + ((!r.rgb.empty() && p.ell_color > 0.0) ? 1 : 0);
    long long n = 0;
    for (int64_t x : r.n) n += x;
    const double per_frame = (double)n / (r.K > 0 ? r.K : 1);
    const int size = per_frame < 16384.0 ? 0 : (per_frame < 65536.0 ? 1 : 2);
    return layout * 4 + size;
}

bool rkhsba_server::tuning_for(Req* r, rkhsba_tuning* t) {
    const int key = workload_class(*r);
    {
        std::lock_guard<std::mutex> lk(tune_mu);
        for (const Tuned& x : tuned)
            if (x.key == key) {
                *t = x.t;
                return true;
            }
    }
    rkhsba_tuning best{};
    const rkhsba_status s = rkhsba_autotune(r->K, r->n.data(), r->xyz.data(), r->sem.empty() ? nullptr : r->sem.data(),
                                            r->rgb.empty() ? nullptr : r->rgb.data(), r->E, r->edges.data(), &r->p, 0,
                                            r->poses0.data(), (void*)streams[r->slot], 2, &best, nullptr, 0, nullptr);
    if (s != RKHSBA_OK) return false;
    std::lock_guard<std::mutex> lk(tune_mu);
    tuned.push_back({key, best});
    *t = best;
    return true;
}

// n_iter LM iterations of every request in `batch` (requests whose first
// half -- damped solve and query binning -- has completed; r->ev marks its
// end), on one free round slot: per iteration one batched pair launch per
// label layout on the slot's stream, then on each request's stream the
// second half (assembly, accept/reject), a copy of the LM state to the
// request's pinned mirror, and at once the first half of the next
// iteration, so that the GPU does not wait for the host between iterations
// (a finished solve makes the rest no-ops).  Requests with the
// neighbour-limited variant (its own kernel) run whole iterations on their
// streams.
void rkhsba_server::issue_round(const std::vector<Req*>& batch, int n_iter) {
    struct Group { int key; GridParams layout; int ctas; int max_uq; std::vector<Req*> reqs; };
    std::vector<Group> groups;
    for (Req* r : batch) {
        const GridParams g = ctx_layout(r->ctx);
        if (g.top_k > 0) {
            cudaStream_t rs = ctx_stream(r->ctx);
            ctx_iterate(r->ctx, n_iter);
            cudaMemcpyAsync(r->mirror, ctx_state_dev(r->ctx), sizeof(LMState), cudaMemcpyDeviceToHost, rs);
            cudaEventRecord(r->ev, rs);
            continue;
        }
        // one launch serves one label layout, colour use and pruning use
        const bool prune = g.sem_min > -__builtin_huge_valf();
        const int key = g.sem_pad * 8 + (prune ? 4 : 0) + (g.sem_bf16 ? 2 : 0) + (g.color ? 1 : 0);
        Group* grp = nullptr;
        for (Group& x : groups)
            if (x.key == key && (int)x.reqs.size() < MAX_PAIR_JOBS) grp = &x;
        if (!grp) {
            groups.push_back({key, g, ctx_tune_ctas(r->ctx), 0, {}});
            grp = &groups.back();
        }
        grp->reqs.push_back(r);
        grp->max_uq = std::max(grp->max_uq, ctx_tune_uq(r->ctx));
    }
    if (groups.empty()) return;
    RoundSlot* rs_free = nullptr;
    for (RoundSlot& x : rounds)
        if (cudaEventQuery(x.ev_mid) == cudaSuccess) {
            rs_free = &x;
            break;
        }
    if (!rs_free) {                      // not reached (see RoundSlot); wait for the first slot
        cudaEventSynchronize(rounds[0].ev_mid);
        rs_free = &rounds[0];
    }
    cudaStream_t rst = rs_free->stream;
    PairJob* jobs = rs_free->d_jobs;
    PairJob* hjobs = rs_free->h_jobs;
    int* counters = rs_free->d_counters;
    {
        int off = 0;
        for (Group& grp : groups) {
            for (size_t k = 0; k < grp.reqs.size(); ++k) hjobs[off + k] = ctx_pair_job(grp.reqs[k]->ctx);
            off += (int)grp.reqs.size();
        }
        cudaMemcpyAsync(jobs, hjobs, sizeof(PairJob) * off, cudaMemcpyHostToDevice, rst);
    }
    for (int it = 0; it < n_iter; ++it) {
        int off = 0, gi = 0;
        for (Group& grp : groups) {
            const int n = (int)grp.reqs.size();
            for (Req* r : grp.reqs) cudaStreamWaitEvent(rst, r->ev, 0);
            cudaMemsetAsync(counters + gi, 0, sizeof(int), rst);
            launch_pairs_multi(jobs + off, n, grp.layout, grp.max_uq, counters + gi, num_sms, grp.ctas, rst);
            off += n;
            ++gi;
        }
        cudaEventRecord(rs_free->ev_mid, rst);
        for (Group& grp : groups)
            for (Req* r : grp.reqs) {
                cudaStream_t rs = ctx_stream(r->ctx);
                cudaStreamWaitEvent(rs, rs_free->ev_mid, 0);
                ctx_iter_post(r->ctx);
                cudaMemcpyAsync(r->mirror, ctx_state_dev(r->ctx), sizeof(LMState), cudaMemcpyDeviceToHost, rs);
                ctx_iter_pre(r->ctx);
                cudaEventRecord(r->ev, rs);
            }
    }
}

// Rolling rounds: every pass collects the requests whose issued work has
// completed (an event query, no waiting), ends those whose LM state (its
// pinned mirror, copied after the second half) says done or that reached
// max_iters, applies cancellations and the watchdog, and issues one round
// over the rest.  A newly admitted request first gets the first half of its
// first iteration.  Requests that are still running join a later round, so
// small problems are not held back by large ones, and problems that become
// ready together share one pair launch.
void rkhsba_server::step_loop_batched() {
    cudaSetDevice(device);
    std::vector<Req*> snap, batch;
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(mu);
            if (stop) return;
            if (running.empty()) cv_step.wait_for(lk, std::chrono::milliseconds(5));
            if (stop) return;
            snap = running;
        }
        batch.clear();
        for (Req* r : snap) {
            if (r->inflight) {
                const cudaError_t q = cudaEventQuery(r->ev);
                if (q == cudaErrorNotReady) continue;
                r->inflight = false;
                if (q != cudaSuccess) {
                    finish(r, RQ_FAILED, RKHSBA_ECUDA);
                    continue;
                }
                if (r->issued > 0 && (r->mirror->done || r->issued >= ctx_max_iters(r->ctx))) {
                    finish(r, RQ_DONE, RKHSBA_OK);
                    continue;
                }
            }
            if (r->cancel) {
                finish(r, RQ_CANCELLED, RKHSBA_OK);
                continue;
            }
            if (cfg.request_timeout_ms > 0 && ms_between(r->t_admit, Clock::now()) > cfg.request_timeout_ms) {
                finish(r, RQ_FAILED, RKHSBA_ETIMEOUT);
                continue;
            }
            if (!r->started) {
                r->started = true;
                r->inflight = true;
                if (ctx_layout(r->ctx).top_k == 0) {
                    ctx_iter_pre(r->ctx);
                    cudaEventRecord(r->ev, ctx_stream(r->ctx));
                } else {
                    cudaEventRecord(r->ev, ctx_stream(r->ctx));
                }
                continue;
            }
            batch.push_back(r);
        }
        if (batch.empty()) {
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            continue;
        }
        // one round per cost class (total points: < 64k, < 256k, < 1M, more),
        // each on its own round slot, so that a round's pair launch and the
        // iterations it gates do not hold small problems back behind large ones
        const int chunk = std::max(1, cfg.iters_per_issue);
        std::vector<Req*> part;
        for (int cls = 0; cls < 4; ++cls) {
            part.clear();
            for (Req* r : batch)
                if (r->cost_class == cls) part.push_back(r);
            if (part.empty()) continue;
            issue_round(part, chunk);
            for (Req* r : part) {
                r->inflight = true;
                r->issued += chunk;
            }
        }
    }
}

extern "C" {

rkhsba_status rkhsba_server_create(rkhsba_server** out, const rkhsba_server_config* cfg) {
    if (!out) return RKHSBA_EINVAL;
    *out = nullptr;
    rkhsba_server* s = new rkhsba_server();
    if (cfg) s->cfg = *cfg;
    if (s->cfg.max_inflight <= 0) s->cfg.max_inflight = 8;
    if (s->cfg.iters_per_issue <= 0) s->cfg.iters_per_issue = 4;
    if (s->cfg.max_inflight > 256) s->cfg.max_inflight = 256;
    if (s->cfg.mode < 0 || s->cfg.mode > 1) {
        delete s;
        set_thread_error("rkhsba_server_create: mode must be 0 (batched) or 1 (per request)");
        return RKHSBA_EINVAL;
    }
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        set_thread_error("no CUDA device");
        return RKHSBA_ECUDA;
    }
    if (s->cfg.memory_budget <= 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            delete s;
            set_thread_error("cudaMemGetInfo failed");
            return RKHSBA_ECUDA;
        }
        s->cfg.memory_budget = (int64_t)(fr / 2);
    }
    for (int i = 0; i < s->cfg.max_inflight; ++i) {
        cudaStream_t st;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            for (auto x : s->streams) cudaStreamDestroy(x);
            delete s;
            set_thread_error("stream creation failed");
            return RKHSBA_ECUDA;
        }
        s->streams.push_back(st);
        s->free_slots.push_back(s->cfg.max_inflight - 1 - i);
    }
    if (s->cfg.mode == 0) {
        cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, s->device);
        const int n = s->cfg.max_inflight;
        s->rounds.resize(n + 1);
        bool ok = cudaMallocHost(&s->h_mirror, sizeof(LMState) * n) == cudaSuccess;
        for (auto& x : s->rounds) {
            ok = ok && cudaStreamCreateWithFlags(&x.stream, cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&x.ev_mid, cudaEventDisableTiming) == cudaSuccess &&
                 cudaMallocHost(&x.h_jobs, sizeof(PairJob) * n) == cudaSuccess &&
                 cudaMalloc(&x.d_jobs, sizeof(PairJob) * n) == cudaSuccess &&
                 cudaMalloc(&x.d_counters, sizeof(int) * n) == cudaSuccess;
        }
        if (!ok) {
            cudaGetLastError();
            for (auto x : s->streams) cudaStreamDestroy(x);
            s->release_rounds();
            delete s;
            set_thread_error("batched-mode resources could not be created");
            return RKHSBA_ECUDA;
        }
        std::memset(s->h_mirror, 0, sizeof(LMState) * n);
    }
    s->admit_thr = std::thread([s] { s->admit_loop(); });
    if (s->cfg.mode == 0) s->step_thr = std::thread([s] { s->step_loop_batched(); });
    else s->step_thr = std::thread([s] { s->step_loop(); });
    *out = s;
    return RKHSBA_OK;
}

void rkhsba_server_destroy(rkhsba_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_admit.notify_all();
    s->cv_step.notify_all();
    s->admit_thr.join();
    s->step_thr.join();
    // cancel what is left: the threads are gone, so no lock contention
    std::vector<Req*> left = s->running;
    for (Req* r : left) {
        if (r->ev && r->started) cudaEventSynchronize(r->ev);
        s->finish(r, RQ_CANCELLED, RKHSBA_OK);
    }
    for (auto st : s->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    s->release_rounds();
    for (auto& kv : s->all) delete kv.second;
    delete s;
}

rkhsba_status rkhsba_submit(rkhsba_server* s, int32_t n_frames, const int64_t* n_points, const double* xyz,
                            const float* sem, const float* rgb, int32_t n_edges, const int32_t* edges,
                            const rkhsba_params* params, const double* poses0, int64_t* ticket) {
    if (!s || !n_points || !edges || !params || !poses0 || !ticket || n_frames < 1 || n_edges < 1) {
        set_thread_error("rkhsba_submit: bad arguments");
        return RKHSBA_EINVAL;
    }
    Req* r = new Req();
    r->K = n_frames;
    r->E = n_edges;
    r->n.assign(n_points, n_points + n_frames);
    long long N = 0;
    for (int m = 0; m < n_frames; ++m) {
        if (n_points[m] < 0) {
            delete r;
            set_thread_error("rkhsba_submit: negative point count");
            return RKHSBA_EINVAL;
        }
        N += n_points[m];
    }
    if (N > 0 && !xyz) {
        delete r;
        set_thread_error("rkhsba_submit: xyz is NULL");
        return RKHSBA_EINVAL;
    }
    r->xyz.assign(xyz, xyz + 3 * N);
    if (sem && params->sem_dim > 0) r->sem.assign(sem, sem + (size_t)N * params->sem_dim);
    if (rgb) r->rgb.assign(rgb, rgb + 3 * N);
    r->edges.assign(edges, edges + 2 * n_edges);
    r->p = *params;
    r->poses0.assign(poses0, poses0 + 16 * n_frames);
    if (!(r->p.ell > 0.0)) {
        delete r;
        set_thread_error("rkhsba_submit: params.ell must be > 0");
        return RKHSBA_EINVAL;
    }
    for (int e = 0; e < n_edges; ++e)
        if (edges[2 * e] < 0 || edges[2 * e] >= n_frames || edges[2 * e + 1] < 0 || edges[2 * e + 1] >= n_frames) {
            delete r;
            set_thread_error("rkhsba_submit: edge names a missing frame");
            return RKHSBA_EINVAL;
        }
    r->est = estimate_bytes(*r);
    r->cost_class = N < (1LL << 16) ? 0 : (N < (1LL << 18) ? 1 : (N < (1LL << 20) ? 2 : 3));
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) {
            delete r;
            return RKHSBA_EBUSY;
        }
        r->ticket = s->next_ticket++;
        s->all[r->ticket] = r;
        s->queue.push_back(r);
        *ticket = r->ticket;
    }
    s->cv_admit.notify_all();
    return RKHSBA_OK;
}

rkhsba_status rkhsba_poll(rkhsba_server* s, int64_t ticket, int32_t timeout_ms, double* poses,
                          rkhsba_request_info* info) {
    if (!s) return RKHSBA_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) {
        set_thread_error("rkhsba_poll: unknown ticket");
        return RKHSBA_EINVAL;
    }
    Req* r = it->second;
    auto ended = [r] { return r->state >= RQ_DONE; };
    if (!ended()) {
        if (timeout_ms < 0) s->cv_done.wait(lk, ended);
        else if (timeout_ms > 0) s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ended);
    }
    if (info) {
        info->state = r->state;
        info->status = r->status;
        info->solve = r->info;
        info->queue_ms = r->state == RQ_QUEUED ? ms_between(r->t_submit, Clock::now())
                                               : ms_between(r->t_submit, r->t_admit);
        info->latency_ms = ended() ? ms_between(r->t_submit, r->t_done) : ms_between(r->t_submit, Clock::now());
        info->device_bytes = (int64_t)r->bytes;
    }
    if (!ended()) return RKHSBA_EBUSY;
    if (poses && r->state == RQ_DONE) std::copy(r->result.begin(), r->result.end(), poses);
    s->all.erase(it);
    delete r;
    return RKHSBA_OK;
}

rkhsba_status rkhsba_cancel(rkhsba_server* s, int64_t ticket) {
    if (!s) return RKHSBA_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        auto it = s->all.find(ticket);
        if (it == s->all.end()) return RKHSBA_EINVAL;
        it->second->cancel = true;
    }
    s->cv_admit.notify_all();
    return RKHSBA_OK;
}

rkhsba_status rkhsba_server_stats(rkhsba_server* s, int64_t* queued, int64_t* running, int64_t* finished,
                                  int64_t* device_bytes) {
    if (!s) return RKHSBA_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (queued) *queued = (int64_t)s->queue.size();
    if (running) *running = (int64_t)s->running.size();
    if (finished) *finished = s->finished;
    if (device_bytes) *device_bytes = (int64_t)s->mem_in_use;
    return RKHSBA_OK;
}

}  // extern "C"
