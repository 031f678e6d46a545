// Serving: a request loop with continuous batching over device-resident plans.
//
// Requests (one particle configuration each, any N) are queued as they arrive.
// `lanes` worker threads each own a plan (same parameters; its matrices and
// pseudo-inverse stay resident) with its own stream and workspace.  A free
// lane takes the oldest waiting requests that fit -- at most max_batch systems
// and, together with the work the other lanes hold, at most the HBM budget --
// and runs them as one batched update step.  Requests that arrive while other
// lanes are on the GPU are admitted by the next free lane, so their device
// work overlaps with the batches in flight.  A request that alone exceeds the
// budget fails with HSMA_E_CAPACITY.
//
// Small requests (n <= express_max_n) queue apart from large ones.  The
// first express_lanes lanes serve only small requests, on the stream of
// highest priority, with persistent launches; the other (bulk) lanes serve
// only large requests (all requests when there is no express lane), on the
// stream of lowest priority, with their pair work launched as one CTA per
// work item (hsma_plan_set_preemptible): as bulk CTAs finish their items the
// SMs go to the express lanes' pending work, so a small request waits for
// work items of a large batch, not for the whole batch.  Optional medium
// lanes sit between the two: medium requests (express_max_n < n <=
// mid_max_n) on a stream of middle priority, with preemptible pair work and
// a workspace reserved at creation like the express lanes'.  Each system's arithmetic depends only on its own inputs
// and on how its sources are split into chunks, so a result is the same,
// within rounding of the chunk grouping, alone or in a mix.
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    int64_t id;
    int64_t n;
    std::vector<double> xyz, q;
    Clock::time_point t_submit, t_start, t_done;
    double energy = 0.0;
    std::vector<double> forces;
    int status = HSMA_E_AGAIN;
    int batch_size = 0;
};

}  // namespace

struct hsma_server_s {
    hsma_server_opts opts;
    int device = 0;
    std::vector<cudaStream_t> streams;
    std::vector<hsma_plan_t> plans;
    std::vector<std::thread> threads;
    std::vector<size_t> held;  // device bytes each lane holds for its current batch
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> queue, queue_small, queue_mid;  // large / small / medium requests, oldest first
    std::unordered_map<int64_t, Request *> all;
    int64_t next_id = 1;
    bool stop = false;
    long long completed = 0, failed = 0, batches = 0, batched_systems = 0, cancelled = 0;
    Clock::time_point t0;
    bool t0_set = false;
    Clock::time_point t_last_done;
};

namespace {

constexpr long long kBatchSizeRatio = 4;  // largest / smallest request size within one batch

void lane_main(hsma_server_s *s, int lane)
{
    cudaSetDevice(s->device);
    hsma_plan_t plan = s->plans[lane];
    const bool express = lane < s->opts.express_lanes;
    const bool mid = !express && lane < s->opts.express_lanes + s->opts.mid_lanes;
    std::vector<int64_t> offsets;
    std::vector<double> xyz, q, energies, forces;
    std::vector<int> status;
    // the queue this lane takes from: express lanes the small requests, bulk
    // lanes the large ones (and the small ones too when there is no express
    // lane); a small request on a bulk lane would run at the low priority
    // beside large work
    const bool bulk_takes_small = s->opts.express_lanes == 0;
    auto pick = [&]() -> std::deque<Request *> * {
        if (express) return s->queue_small.empty() ? nullptr : &s->queue_small;
        if (mid) return s->queue_mid.empty() ? nullptr : &s->queue_mid;
        if (!s->queue.empty()) return &s->queue;
        return (bulk_takes_small && !s->queue_small.empty()) ? &s->queue_small : nullptr;
    };
    for (;;) {
        std::vector<Request *> batch;
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] { return s->stop || pick() != nullptr; });
            std::deque<Request *> *qu = pick();
            if (!qu) return;  // stopping, and nothing left that this lane serves
            size_t others = 0;
            for (size_t l = 0; l < s->held.size(); ++l)
                if ((int)l != lane) others += s->held[l];
            size_t used = 0;
            // the oldest request, then the waiting ones within a factor
            // kBatchSizeRatio of its size: a request batched with much larger
            // ones would finish only when they do; the others stay queued, in
            // order, for the next free lane
            long long n_first = 0;
            for (size_t i = 0; i < qu->size() && (int)batch.size() < s->opts.max_batch;) {
                Request *r = (*qu)[i];
                size_t one = 0;
                hsma_plan_footprint(plan, r->n, &one);
                if (one > s->opts.hbm_budget_bytes) {  // can never run
                    qu->erase(qu->begin() + (std::ptrdiff_t)i);
                    r->status = HSMA_E_CAPACITY;
                    r->t_done = Clock::now();
                    r->t_start = r->t_done;
                    s->failed++;
                    s->cv_done.notify_all();
                    continue;
                }
                if (!batch.empty() && (r->n > kBatchSizeRatio * n_first || kBatchSizeRatio * r->n < n_first)) {
                    ++i;  // another size class: leave it for the next lane
                    continue;
                }
                if (others + used + one > s->opts.hbm_budget_bytes) break;  // wait for memory
                qu->erase(qu->begin() + (std::ptrdiff_t)i);
                if (batch.empty()) n_first = r->n;
                used += one;
                batch.push_back(r);
            }
            if (batch.empty()) {
                // memory is held by other lanes: wait for one of them to finish
                s->cv_done.wait_for(lk, std::chrono::milliseconds(2));
                continue;
            }
            s->held[lane] = used;
        }
        auto t_start = Clock::now();
        offsets.assign(1, 0);
        xyz.clear();
        q.clear();
        for (auto *r : batch) {
            offsets.push_back(offsets.back() + r->n);
            xyz.insert(xyz.end(), r->xyz.begin(), r->xyz.end());
            q.insert(q.end(), r->q.begin(), r->q.end());
        }
        const int nb = (int)batch.size();
        energies.assign(nb, 0.0);
        status.assign(nb, 0);
        forces.assign(3 * offsets.back(), 0.0);
        hsma_particles all;
        all.n = offsets.back();
        all.xyz = xyz.data();
        all.q = q.data();
        all.on_device = 0;
        int rc = hsma_energy_forces_batched(plan, nb, offsets.data(), &all, energies.data(), forces.data(), nullptr,
                                            status.data());
        auto t_done = Clock::now();
        {
            std::lock_guard<std::mutex> lk(s->mu);
            s->held[lane] = 0;
            // keep a bulk lane's cached workspace within what the budget leaves
            // (express and medium lanes keep the workspace reserved at creation:
            // freeing and growing it would synchronise the device behind bulk work)
            if (!express && !mid) {
                size_t others_now = 0;
                for (size_t l = 0; l < s->held.size(); ++l) others_now += s->held[l];
                size_t room = s->opts.hbm_budget_bytes > others_now ? s->opts.hbm_budget_bytes - others_now : 0;
                hsma::plan_trim_workspace(plan, room / s->plans.size());
            }
            s->batches++;
            s->batched_systems += nb;
            for (int i = 0; i < nb; ++i) {
                Request *r = batch[i];
                r->t_start = t_start;
                r->t_done = t_done;
                r->batch_size = nb;
                r->energy = energies[i];
                int code = (rc == HSMA_OK) ? HSMA_OK : (status[i] != HSMA_OK ? status[i] : rc);
                r->status = code;
                if (code == HSMA_OK) {
                    r->forces.assign(forces.begin() + 3 * offsets[i], forces.begin() + 3 * offsets[i + 1]);
                    s->completed++;
                } else {
                    s->failed++;
                }
                r->xyz.clear();
                r->xyz.shrink_to_fit();
                r->q.clear();
                r->q.shrink_to_fit();
            }
            s->t_last_done = t_done;
        }
        s->cv_done.notify_all();
    }
}

}  // namespace

extern "C" {

int hsma_server_opts_default(hsma_server_opts *o)
{
    if (!o) return HSMA_E_ARG;
    memset(o, 0, sizeof(*o));
    o->hbm_budget_bytes = 0;
    o->max_batch = 64;
    o->lanes = 2;
    o->precision = HSMA_FP32_ACC64;
    o->express_lanes = 1;
    o->express_max_n = 20000;
    o->mid_lanes = 0;
    o->mid_max_n = 60000;
    return HSMA_OK;
}

int hsma_server_create(hsma_server_t *out, const double box[3], int bc, int p, double R, int Q, int Kmon,
                       const hsma_server_opts *opts)
{
    if (!out) return HSMA_E_ARG;
    *out = nullptr;
    hsma_server_opts o;
    hsma_server_opts_default(&o);
    if (opts) o = *opts;
    if (o.lanes < 1 || o.lanes > 16 || o.max_batch < 1 || o.max_batch > 65528) return HSMA_E_ARG;
    if (o.express_lanes < 0 || o.mid_lanes < 0 || o.express_max_n < 0 ||
        (o.express_lanes + o.mid_lanes > 0 && o.express_lanes + o.mid_lanes >= o.lanes) ||
        (o.mid_lanes > 0 && o.mid_max_n < o.express_max_n))
        return HSMA_E_ARG;  // at least one bulk lane serves the large requests
    if (o.hbm_budget_bytes == 0) {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return HSMA_E_CUDA;
        o.hbm_budget_bytes = free_b / 2;
    }
    auto *s = new hsma_server_s();
    s->opts = o;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return HSMA_E_CUDA;
    }
    hsma_opts po;
    hsma_opts_default(&po);
    po.precision = o.precision;
    po.use_graphs = 0;  // batch shapes change from call to call: direct launches
    int prio_low = 0, prio_high = 0;  // numerically: greatest priority is the lowest number
    if (cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high) != cudaSuccess) {
        delete s;
        return HSMA_E_CUDA;
    }
    // numerically between the two (the same as the highest when the range has no middle)
    const int prio_mid = prio_low - prio_high >= 2 ? (prio_high + prio_low) / 2 : prio_high;
    for (int l = 0; l < o.lanes; ++l) {
        const bool express = l < o.express_lanes;
        const bool mid = !express && l < o.express_lanes + o.mid_lanes;
        cudaStream_t st = nullptr;
        const int prio = express ? prio_high : (mid ? prio_mid : prio_low);
        if (cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, prio) != cudaSuccess) {
            hsma_server_destroy(s);
            return HSMA_E_CUDA;
        }
        s->streams.push_back(st);
        po.stream = st;
        hsma_plan_t pl = nullptr;
        int rc = hsma_plan(&pl, box, bc, p, R, Q, Kmon, &po);
        if (!rc && !express) rc = hsma_plan_set_preemptible(pl, 1);
        // express and medium lanes never allocate while serving: their
        // workspace holds a full batch of the largest requests of their class
        // from the start (reserved after the preemptible setting, which sets
        // the number of partial records)
        if (!rc && express && o.express_max_n > 0)
            rc = hsma::plan_reserve(pl, o.max_batch, o.express_max_n);
        if (!rc && mid) rc = hsma::plan_reserve(pl, o.max_batch, o.mid_max_n);
        if (rc) {
            if (pl) hsma_plan_destroy(pl);
            hsma_server_destroy(s);
            return rc;
        }
        s->plans.push_back(pl);
    }
    // One- and two-system steps of a few charges on every lane before serving:
    // the CUDA runtime loads a kernel at its first launch, and a load can wait
    // for the work already on the device -- a lane's first request would
    // otherwise queue behind a large batch on another lane.
    {
        const int nw = 8;
        std::vector<double> wx(3 * 2 * nw), wq(2 * nw), we(2), wf(3 * 2 * nw);
        std::vector<int> ws(2);
        for (int i = 0; i < 2 * nw; ++i) {
            for (int a = 0; a < 3; ++a) wx[3 * i + a] = box[a] * (0.3 + 0.4 * (double)((i >> a) & 1) + 0.01 * i);
            wq[i] = (i & 1) ? -1.0 : 1.0;
        }
        for (int l = 0; l < o.lanes; ++l) {
            for (int k = 1; k <= 2; ++k) {
                const int64_t off[3] = {0, nw, 2 * nw};
                hsma_particles in{(int64_t)k * nw, wx.data(), wq.data(), 0};
                int rc = hsma_energy_forces_batched(s->plans[l], k, off, &in, we.data(), wf.data(), nullptr, ws.data());
                if (rc) {
                    hsma_server_destroy(s);
                    return rc;
                }
            }
        }
    }
    s->held.assign(o.lanes, 0);
    for (int l = 0; l < o.lanes; ++l) s->threads.emplace_back(lane_main, s, l);
    *out = s;
    return HSMA_OK;
}

int hsma_server_submit(hsma_server_t s, int64_t n, const double *xyz, const double *q, int64_t *ticket)
{
    if (!s || n < 1 || !xyz || !q || !ticket) return HSMA_E_ARG;
    auto *r = new Request();
    r->n = n;
    r->xyz.assign(xyz, xyz + 3 * n);
    r->q.assign(q, q + n);
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) {
            delete r;
            return HSMA_E_ARG;
        }
        r->id = s->next_id++;
        if (!s->t0_set) {
            s->t0 = r->t_submit;
            s->t0_set = true;
        }
        s->all[r->id] = r;
        if (n <= s->opts.express_max_n)
            s->queue_small.push_back(r);
        else if (s->opts.mid_lanes > 0 && n <= s->opts.mid_max_n)
            s->queue_mid.push_back(r);
        else
            s->queue.push_back(r);
        *ticket = r->id;
    }
    s->cv_work.notify_all();
    return HSMA_OK;
}

int hsma_server_result(hsma_server_t s, int64_t ticket, int wait, double *energy, double *forces,
                       hsma_request_info *info)
{
    if (!s) return HSMA_E_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return HSMA_E_NOT_FOUND;
    Request *r = it->second;
    if (r->status == HSMA_E_AGAIN) {
        if (!wait) return HSMA_E_AGAIN;
        s->cv_done.wait(lk, [&] { return r->status != HSMA_E_AGAIN; });
    }
    int code = r->status;
    if (energy) *energy = r->energy;
    if (forces && code == HSMA_OK) memcpy(forces, r->forces.data(), sizeof(double) * 3 * r->n);
    if (info) {
        info->n = r->n;
        info->latency_ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
        info->queue_ms = std::chrono::duration<double, std::milli>(r->t_start - r->t_submit).count();
        info->batch_size = r->batch_size;
        info->status = code;
    }
    s->all.erase(it);
    delete r;
    return code;
}

int hsma_server_cancel(hsma_server_t s, int64_t ticket)
{
    if (!s) return HSMA_E_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->all.find(ticket);
    if (it == s->all.end()) return HSMA_E_NOT_FOUND;
    Request *r = it->second;
    for (auto *qu : {&s->queue, &s->queue_small, &s->queue_mid})
        for (auto q = qu->begin(); q != qu->end(); ++q)
            if (*q == r) {
                qu->erase(q);
                r->status = HSMA_E_CANCELLED;
                r->t_done = Clock::now();
                r->t_start = r->t_done;
                s->cancelled++;
                s->cv_done.notify_all();
                return HSMA_OK;
            }
    return HSMA_E_AGAIN;  // already running or finished
}

int hsma_server_stats(hsma_server_t s, hsma_server_stats_t *st)
{
    if (!s || !st) return HSMA_E_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    st->completed = s->completed;
    st->failed = s->failed;
    st->cancelled = s->cancelled;
    st->queued = (int64_t)(s->queue.size() + s->queue_small.size() + s->queue_mid.size());
    st->batches = s->batches;
    st->mean_batch = s->batches ? (double)s->batched_systems / s->batches : 0.0;
    st->elapsed_s = s->t0_set ? std::chrono::duration<double>(s->t_last_done - s->t0).count() : 0.0;
    size_t held = 0;
    for (size_t h : s->held) held += h;
    st->hbm_held_bytes = held;
    st->hbm_budget_bytes = s->opts.hbm_budget_bytes;
    return HSMA_OK;
}

void hsma_server_destroy(hsma_server_t s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto &t : s->threads) t.join();
    for (auto &kv : s->all) delete kv.second;
    for (auto *pl : s->plans) hsma_plan_destroy(pl);
    for (auto st : s->streams) cudaStreamDestroy(st);
    delete s;
}

}  // extern "C"
