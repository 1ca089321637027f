// Query server over resident graphs: continuous batching of Kemeny queries and
// edge-update batches (the serving form of Sec. 3's estimate and Sec. 4's
// sample maintenance).  Host code only; every request runs through the C ABI
// of kc_api.cu on the worker's own CUDA stream, so requests on different graphs
// overlap on the device.  Per-graph order is submission order.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/kc_serve.h"
#include "kc_host_admit.h"
#include "kc_host_stop.h"

namespace {

struct Graph {
    kc_graph *h = nullptr;
    int64_t n = 0;
    bool dynamic = false;  // maintained pool (POOL_QUERY / UPDATE) vs fresh pools (QUERY)
    bool busy = false;     // a worker (or the dispatcher) is running one of its requests
    bool coalesced = false;  // its QUERY requests go to the dispatcher
    kc_config cfg{};
};

// A QUERY advanced by the dispatcher: kc_estimate's normal-approximation rule
// (kc_host_stop.h) as a state machine, one tree batch per round.
struct Active {
    int64_t ticket = 0;
    int64_t bytes = 0;
    int64_t pool = 0;     // trees drawn so far
    int round = -1;       // -1: the pilot batch is next; then checks 0 .. 63
    double z = 0;
    int64_t batch = 0, cap = 0;
};

struct Request {
    int32_t kind = KC_REQ_QUERY;
    int32_t graph = 0;
    uint64_t seed = 0;
    double eps = 0, delta = 0;
    std::vector<kc_edge_op> ops;
    int32_t mode = KC_UPDATE_ISM;
    bool done = false;
    kc_request_info info{};
};

}  // namespace

struct kc_server {
    kc_server_config cfg{};
    int device = 0;
    std::chrono::steady_clock::time_point t0;
    std::deque<Graph> graphs;                    // stable addresses while graphs are added
    std::vector<std::unique_ptr<Request>> reqs;  // by ticket (read under the lock)
    std::deque<int64_t> queue;                   // waiting tickets, submission order
    std::deque<int64_t> cqueue;                  // waiting coalesced QUERY tickets
    std::thread dispatcher;
    cudaStream_t dstream = nullptr;
    int64_t rounds = 0;                          // dispatcher rounds (kc_sample_multi calls)
    int64_t reserved = 0;                        // bytes reserved by running requests
    int64_t outstanding = 0;                     // submitted and not yet done
    bool stop = false;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::vector<std::thread> workers;
    std::vector<cudaStream_t> streams;

    double now_ms() const {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0)
            .count();
    }

    // device bytes a request on graph g reserves
    int64_t reserve_for(const Graph &g) const {
        const int64_t per_tree = 40 * g.n + 512;
        const int64_t want = 4096 * per_tree;
        return want < cfg.request_bytes ? want : cfg.request_bytes;
    }

    // the first waiting request of q that may start now (kc_host_admit.h)
    bool pick(int64_t *ticket, int64_t *bytes, std::deque<int64_t> *qp = nullptr) {
        std::deque<int64_t> &queue = qp ? *qp : this->queue;
        auto it = kc_host::first_admissible(
            queue.begin(), queue.end(), graphs.size(),
            [&](int64_t t) { return reqs[(size_t)t]->graph; },
            [&](size_t gi) { return graphs[gi].busy; },
            [&](size_t gi) { return reserve_for(graphs[gi]); }, reserved, cfg.budget_bytes,
            bytes);
        if (it == queue.end()) return false;
        *ticket = *it;
        queue.erase(it);
        return true;
    }

    void run(int wid) {
        cudaSetDevice(device);
        for (;;) {
            int64_t ticket = -1, bytes = 0;
            Request *rp = nullptr;
            Graph *gp = nullptr;
            {
                std::unique_lock<std::mutex> lk(mu);
                cv_work.wait(lk, [&] { return stop || (!queue.empty() && pick(&ticket, &bytes)); });
                if (ticket < 0) return;  // stop requested and nothing admissible
                rp = reqs[(size_t)ticket].get();
                gp = &graphs[(size_t)rp->graph];
                gp->busy = true;
                reserved += bytes;
            }
            Request &r = *rp;
            Graph &g = *gp;
            r.info.t_start_ms = now_ms();
            r.info.worker = wid;
            r.info.workspace_bytes = bytes;
            kc_status st = kc_graph_set_stream(g.h, streams[(size_t)wid]);
            if (st == KC_OK) st = kc_graph_set_workspace_limit(g.h, bytes - bytes / 8);
            double K = 0;
            if (st == KC_OK) {
                if (r.kind == KC_REQ_QUERY) {
                    st = kc_graph_reset(g.h, r.seed, 0);
                    if (st == KC_OK) st = kc_estimate(g.h, r.eps, r.delta, &K);
                } else if (r.kind == KC_REQ_POOL_QUERY) {
                    st = kc_estimate(g.h, r.eps, r.delta, &K);
                } else {
                    st = kc_update(g.h, r.ops.data(), (int64_t)r.ops.size(), r.mode);
                }
            }
            kc_graph_release_workspace(g.h);
            cudaStreamSynchronize(streams[(size_t)wid]);
            kc_stats_t stt;
            std::memset(&stt, 0, sizeof(stt));
            if (kc_stats(g.h, &stt) == KC_OK) r.info.trees = stt.pool_trees;
            r.info.status = st;
            r.info.K = K;
            r.info.t_end_ms = now_ms();
            {
                std::lock_guard<std::mutex> lk(mu);
                g.busy = false;
                reserved -= bytes;
                r.done = true;
                --outstanding;
            }
            cv_work.notify_all();
            cv_done.notify_all();
        }
    }
};

// The coalescing dispatcher.  Between rounds it admits waiting coalesced
// queries (submission order per graph, within the budget), then gives every
// admitted query its next batch: the pilot, or what the stopping rule asks
// for after the previous batch (kc_host::clt_more on the pool's sums).  A query
// whose rule says stop, or that has had 64 checks, takes K from its pool and
// leaves.  The batches of one round run as one kc_sample_multi call (all
// walks in one launch) on the dispatcher's stream.
void dispatch_loop(kc_server *s) {
    cudaSetDevice(s->device);
    std::vector<Active> act;
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(s->mu);
            int64_t ticket = -1, bytes = 0;
            // sleep only when nothing runs here and nothing waiting fits
            s->cv_work.wait(lk, [&] {
                return s->stop || !act.empty() ||
                       (!s->cqueue.empty() && s->pick(&ticket, &bytes, &s->cqueue));
            });
            for (;;) {
                if (ticket < 0 && (s->cqueue.empty() || !s->pick(&ticket, &bytes, &s->cqueue)))
                    break;
                Request &r = *s->reqs[(size_t)ticket];
                Graph &g = s->graphs[(size_t)r.graph];
                g.busy = true;
                s->reserved += bytes;
                Active a;
                a.ticket = ticket;
                a.bytes = bytes;
                a.z = kc_host::inv_normal_upper(r.delta / 2.0);
                a.batch = g.cfg.batch_trees > 0 ? g.cfg.batch_trees : 1024;
                a.cap = g.cfg.max_trees > 0 ? g.cfg.max_trees : ((int64_t)1 << 24);
                act.push_back(a);
                r.info.t_start_ms = s->now_ms();
                r.info.worker = -1;
                r.info.workspace_bytes = bytes;
                ticket = -1;
            }
            if (act.empty() && s->stop) return;
            if (act.empty()) continue;
        }
        // set up newly admitted queries (fresh pool under the request's seed)
        std::vector<kc_graph *> hs;
        std::vector<uint64_t> seeds;
        std::vector<int64_t> ks;
        std::vector<size_t> who;
        std::vector<std::pair<size_t, kc_status>> finished;
        for (size_t i = 0; i < act.size(); ++i) {
            Active &a = act[i];
            Request &r = *s->reqs[(size_t)a.ticket];
            kc_graph *h = s->graphs[(size_t)r.graph].h;
            kc_status st = KC_OK;
            int64_t k = 0;
            if (a.round < 0) {
                st = kc_graph_set_stream(h, s->dstream);
                if (st == KC_OK) st = kc_graph_set_workspace_limit(h, a.bytes - a.bytes / 8);
                if (st == KC_OK) st = kc_graph_reset(h, r.seed, 0);
                k = std::max<int64_t>(64, std::min(a.batch, a.cap));  // the pilot
                a.round = 0;
            } else if (a.round >= 64) {
                k = 0;
            } else {
                kc_pool_sums ps;
                st = kc_get_pool_sums(h, &ps);
                if (st == KC_OK)
                    k = kc_host::clt_more(kc_host::Moments{ps.count, ps.wf_sum, ps.w_sum, ps.x2_sum},
                                          a.z, r.eps, a.batch, a.cap, a.pool);
                ++a.round;
            }
            if (st != KC_OK || k <= 0) {
                finished.push_back({i, st});
                continue;
            }
            hs.push_back(h);
            seeds.push_back(r.seed);
            ks.push_back(k);
            who.push_back(i);
        }
        if (!hs.empty()) {
            const kc_status st = kc_sample_multi(hs.data(), seeds.data(), ks.data(), (int32_t)hs.size());
            ++s->rounds;
            for (size_t j = 0; j < who.size(); ++j) {
                if (st != KC_OK) finished.push_back({who[j], st});
                else act[who[j]].pool += ks[j];
            }
        }
        // finish: K from the pool (the exact int128 numerator), release
        std::vector<char> gone(act.size(), 0);
        for (auto &fs : finished) {
            Active &a = act[fs.first];
            Request &r = *s->reqs[(size_t)a.ticket];
            Graph &g = s->graphs[(size_t)r.graph];
            kc_status st = fs.second;
            double K = 0;
            if (st == KC_OK) st = kc_estimate(g.h, 0.0, 0.0, &K);
            kc_graph_release_workspace(g.h);
            cudaStreamSynchronize(s->dstream);
            kc_stats_t stt;
            std::memset(&stt, 0, sizeof(stt));
            if (kc_stats(g.h, &stt) == KC_OK) r.info.trees = stt.pool_trees;
            r.info.status = st;
            r.info.K = K;
            r.info.t_end_ms = s->now_ms();
            {
                std::lock_guard<std::mutex> lk(s->mu);
                g.busy = false;
                s->reserved -= a.bytes;
                r.done = true;
                --s->outstanding;
            }
            gone[fs.first] = 1;
        }
        if (!finished.empty()) {
            std::vector<Active> keep;
            for (size_t i = 0; i < act.size(); ++i)
                if (!gone[i]) keep.push_back(act[i]);
            act.swap(keep);
            s->cv_work.notify_all();
            s->cv_done.notify_all();
        }
    }
}

extern "C" {

void kc_server_config_default(kc_server_config *cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->struct_size = sizeof(kc_server_config);
    cfg->workers = 4;
}

kc_status kc_server_create(const kc_server_config *cfg_in, kc_server **out) {
    if (!out) return KC_ERR_INVALID_ARG;
    *out = nullptr;
    kc_server_config cfg;
    kc_server_config_default(&cfg);
    if (cfg_in) {
        if (cfg_in->struct_size != sizeof(kc_server_config)) return KC_ERR_INVALID_ARG;
        cfg = *cfg_in;
    }
    if (cfg.workers <= 0) cfg.workers = 4;
    if (cfg.workers > 64 || cfg.budget_bytes < 0 || cfg.request_bytes < 0)
        return KC_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        (void)cudaGetLastError();
        return KC_ERR_NO_DEVICE;
    }
    kc_server *s = new (std::nothrow) kc_server();
    if (!s) return KC_ERR_OUT_OF_MEMORY;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        delete s;
        return KC_ERR_CUDA;
    }
    if (cfg.budget_bytes == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            delete s;
            return KC_ERR_CUDA;
        }
        cfg.budget_bytes = (int64_t)(fr / 2);
    }
    if (cfg.request_bytes == 0) cfg.request_bytes = cfg.budget_bytes / cfg.workers;
    s->cfg = cfg;
    s->t0 = std::chrono::steady_clock::now();
    for (int i = 0; i < cfg.workers; ++i) {
        cudaStream_t st = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
            delete s;
            return KC_ERR_CUDA;
        }
        s->streams.push_back(st);
    }
    if (cfg.coalesce) {
        if (cfg.coalesce_max_n <= 0) cfg.coalesce_max_n = (int64_t)1 << 18;
        s->cfg = cfg;
        if (cudaStreamCreateWithFlags(&s->dstream, cudaStreamNonBlocking) != cudaSuccess) {
            for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
            delete s;
            return KC_ERR_CUDA;
        }
        s->dispatcher = std::thread([s] { dispatch_loop(s); });
    }
    for (int i = 0; i < cfg.workers; ++i) s->workers.emplace_back([s, i] { s->run(i); });
    *out = s;
    return KC_OK;
}

kc_status kc_server_drain(kc_server *s) {
    if (!s) return KC_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    s->cv_done.wait(lk, [&] { return s->outstanding == 0; });
    return KC_OK;
}

kc_status kc_server_destroy(kc_server *s) {
    if (!s) return KC_OK;
    kc_server_drain(s);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto &t : s->workers) t.join();
    if (s->dispatcher.joinable()) s->dispatcher.join();
    for (auto &g : s->graphs) kc_graph_destroy(g.h);
    for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
    if (s->dstream) cudaStreamDestroy(s->dstream);
    delete s;
    (void)cudaGetLastError();  // nothing the teardown above reports outlives this call
    return KC_OK;
}

kc_status kc_server_add_graph(kc_server *s, int64_t n, const int64_t *row_off, const int32_t *col,
                              const kc_config *cfg_in, uint64_t pool_seed, int64_t pool_trees,
                              int32_t *graph_id) {
    if (!s || !graph_id || pool_trees < 0) return KC_ERR_INVALID_ARG;
    kc_config cfg;
    kc_config_default(&cfg);
    if (cfg_in) {
        if (cfg_in->struct_size != sizeof(kc_config)) return KC_ERR_INVALID_ARG;
        cfg = *cfg_in;
    }
    cfg.keep_trees = pool_trees > 0 ? 1 : 0;
    kc_graph *h = nullptr;
    kc_status st = kc_graph_create(n, row_off, col, &cfg, &h);
    if (st != KC_OK) return st;
    if (pool_trees > 0) {
        st = kc_sample(h, pool_seed, pool_trees);
        if (st == KC_OK) st = kc_graph_release_workspace(h);
        if (st != KC_OK) {
            kc_graph_destroy(h);
            return st;
        }
    }
    std::lock_guard<std::mutex> lk(s->mu);
    Graph g;
    g.h = h;
    g.n = n;
    g.dynamic = pool_trees > 0;
    g.cfg = cfg;
    // a round lasts as long as its slowest walk: graphs with a deep tau0 (the
    // BIT variant: long walks, e.g. road-shaped ones) stay with the workers
    kc_stats_t stt;
    std::memset(&stt, 0, sizeof(stt));
    const bool shallow = kc_stats(h, &stt) == KC_OK && stt.ttf_variant == KC_TTF_SCAN;
    g.coalesced = s->cfg.coalesce && !g.dynamic && n <= s->cfg.coalesce_max_n && shallow &&
                  cfg.stop_rule == KC_STOP_CLT && cfg.reject_steps == 0 && !cfg.autotune;
    s->graphs.push_back(g);
    *graph_id = (int32_t)(s->graphs.size() - 1);
    return KC_OK;
}

static kc_status submit(kc_server *s, std::unique_ptr<Request> r, int64_t *ticket) {
    {
        std::lock_guard<std::mutex> lk(s->mu);
        r->info.kind = r->kind;
        r->info.graph = r->graph;
        r->info.worker = -1;
        r->info.t_submit_ms = s->now_ms();
        const int64_t t = (int64_t)s->reqs.size();
        const bool co = r->kind == KC_REQ_QUERY && s->graphs[(size_t)r->graph].coalesced;
        s->reqs.push_back(std::move(r));
        (co ? s->cqueue : s->queue).push_back(t);
        ++s->outstanding;
        *ticket = t;
    }
    s->cv_work.notify_all();
    return KC_OK;
}

static kc_status check_graph(kc_server *s, int32_t graph, bool dynamic) {
    std::lock_guard<std::mutex> lk(s->mu);
    if (graph < 0 || graph >= (int32_t)s->graphs.size()) return KC_ERR_INVALID_ARG;
    if (s->graphs[(size_t)graph].dynamic != dynamic) return KC_ERR_INVALID_ARG;
    return KC_OK;
}

kc_status kc_server_submit_query(kc_server *s, int32_t graph, uint64_t seed, double eps,
                                 double delta, int64_t *ticket) {
    if (!s || !ticket || !(eps > 0) || !(delta > 0 && delta < 1)) return KC_ERR_INVALID_ARG;
    kc_status st = check_graph(s, graph, false);
    if (st != KC_OK) return st;
    auto r = std::make_unique<Request>();
    r->kind = KC_REQ_QUERY;
    r->graph = graph;
    r->seed = seed;
    r->eps = eps;
    r->delta = delta;
    return submit(s, std::move(r), ticket);
}

kc_status kc_server_submit_pool_query(kc_server *s, int32_t graph, double eps, double delta,
                                      int64_t *ticket) {
    if (!s || !ticket || !(eps > 0) || !(delta > 0 && delta < 1)) return KC_ERR_INVALID_ARG;
    kc_status st = check_graph(s, graph, true);
    if (st != KC_OK) return st;
    auto r = std::make_unique<Request>();
    r->kind = KC_REQ_POOL_QUERY;
    r->graph = graph;
    r->eps = eps;
    r->delta = delta;
    return submit(s, std::move(r), ticket);
}

kc_status kc_server_submit_update(kc_server *s, int32_t graph, const kc_edge_op *ops,
                                  int64_t n_ops, int32_t mode, int64_t *ticket) {
    if (!s || !ticket || n_ops < 0 || (n_ops > 0 && !ops)) return KC_ERR_INVALID_ARG;
    if (mode != KC_UPDATE_BSM && mode != KC_UPDATE_ISM) return KC_ERR_INVALID_ARG;
    kc_status st = check_graph(s, graph, true);
    if (st != KC_OK) return st;
    auto r = std::make_unique<Request>();
    r->kind = KC_REQ_UPDATE;
    r->graph = graph;
    r->mode = mode;
    r->ops.assign(ops, ops + n_ops);
    return submit(s, std::move(r), ticket);
}

kc_status kc_server_wait(kc_server *s, int64_t ticket, kc_request_info *info) {
    if (!s) return KC_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    if (ticket < 0 || ticket >= (int64_t)s->reqs.size()) return KC_ERR_INVALID_ARG;
    Request &r = *s->reqs[(size_t)ticket];
    s->cv_done.wait(lk, [&] { return r.done; });
    if (info) *info = r.info;
    return KC_OK;
}

kc_status kc_server_poll(kc_server *s, int64_t ticket, int32_t *done, kc_request_info *info) {
    if (!s || !done) return KC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    if (ticket < 0 || ticket >= (int64_t)s->reqs.size()) return KC_ERR_INVALID_ARG;
    Request &r = *s->reqs[(size_t)ticket];
    *done = r.done ? 1 : 0;
    if (r.done && info) *info = r.info;
    return KC_OK;
}

}  // extern "C"
