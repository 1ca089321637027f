/*
 * kc_serve.h -- a query server over resident graphs (continuous batching).
 *
 * Serving form of the method: graphs (and, for dynamic graphs, their sample
 * pools maintained by Algorithm 2 / Algorithm 3) stay resident on the device;
 * Kemeny queries at a requested (eps, delta) and edge-update batches arrive at
 * any time and are admitted as a worker and workspace memory free up.  Every
 * worker drives its own CUDA stream, so the walks and traversals of requests
 * on different graphs run on the GPU at the same time.  This interface has no
 * counterpart in the paper; it packages the paper's static estimate (Sec. 3)
 * and sample maintenance (Sec. 4) for a serving loop.
 *
 * Conventions (as in kc.h): plain C types; input arrays are host pointers
 * copied by the library; every call returns a kc_status.  The server is used
 * from one host thread at a time (its workers are internal threads).
 *
 * Determinism: requests on one graph execute in submission order.  A QUERY
 * draws a fresh pool under its own seed (sample ids from 0), so its result
 * depends only on (graph, seed, eps, delta), alone or in any mix of traffic.
 * POOL_QUERY and UPDATE act on the graph's maintained pool in submission order,
 * so their results depend only on that graph's request sequence.
 */
#ifndef KC_SERVE_H
#define KC_SERVE_H

#include "kc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kc_server kc_server; /* opaque */

typedef struct {
    uint32_t struct_size;   /* sizeof(kc_server_config), for ABI growth                  */
    int32_t workers;        /* requests in flight at once: host threads, one CUDA stream
                               each (0: 4; at most 64)                                  */
    int64_t budget_bytes;   /* device bytes shared by the workspaces of in-flight
                               requests (0: half the free device memory at creation)    */
    int64_t request_bytes;  /* workspace cap of one request (0: budget / workers); a
                               request reserves min(cap, 4096 trees' worth) until done  */
    int32_t coalesce;       /* 1: QUERY requests on graphs of at most coalesce_max_n
                               vertices are run together by a dispatcher thread: in
                               each round every admitted query draws its next batch of
                               trees, and the walks of all of them share one launch
                               (kc_sample_multi); queries join and leave between rounds.
                               Each query draws the same trees and takes the same
                               stopping decisions as kc_estimate, so its K is the one
                               it gets alone.  Larger graphs, graphs whose path tree
                               is deep (the BIT variant: long walks, which would hold
                               up every query of a round), and graphs with the
                               Hoeffding rule, rejection or the autotuner stay with
                               the workers.  0: off                                 */
    int32_t reserved;
    int64_t coalesce_max_n; /* 0: 2^18                                                */
} kc_server_config;

/* Request kinds. */
enum { KC_REQ_QUERY = 0,       /* K at (eps, delta) from a fresh pool under the request's seed */
       KC_REQ_POOL_QUERY = 1,  /* K at (eps, delta) from the graph's maintained pool         */
       KC_REQ_UPDATE = 2 };    /* an edge-update batch (kc_update semantics)                  */

typedef struct {
    int32_t status;          /* kc_status of the request (KC_OK when done without error) */
    int32_t kind;            /* KC_REQ_*                                                  */
    int32_t graph;           /* graph id                                                  */
    int32_t worker;          /* worker (stream) that ran it                               */
    double K;                /* estimate (queries), 0 for updates                         */
    int64_t trees;           /* trees in the graph's pool when the request finished      */
    double t_submit_ms;      /* host steady clock, ms since the server was created        */
    double t_start_ms;
    double t_end_ms;
    int64_t workspace_bytes; /* device bytes reserved for the request                     */
} kc_request_info;

/* Fill *cfg with the defaults above. */
void kc_server_config_default(kc_server_config *cfg);

/* Start the workers on the current device.  Errors: INVALID_ARG, NO_DEVICE, CUDA. */
kc_status kc_server_create(const kc_server_config *cfg, kc_server **out);

/* Finish every submitted request, stop the workers, free every graph. */
kc_status kc_server_destroy(kc_server *s);

/*
 * Make a graph resident (kc_graph_create semantics for n, row_off, col, cfg,
 * except that cfg->keep_trees is replaced: 1 for a dynamic graph, else 0).
 * pool_trees > 0 makes it a dynamic graph: a pool of that many trees is drawn
 * under pool_seed (trees retained) and serves POOL_QUERY and UPDATE; otherwise
 * it serves QUERY.  *graph_id receives the id (0, 1, ...).
 * Errors: those of kc_graph_create and kc_sample.
 */
kc_status kc_server_add_graph(kc_server *s, int64_t n, const int64_t *row_off, const int32_t *col,
                              const kc_config *cfg, uint64_t pool_seed, int64_t pool_trees,
                              int32_t *graph_id);

/* Queue a request; *ticket identifies it (0, 1, ...).  Arguments are checked
 * here (INVALID_ARG: unknown graph, wrong graph kind, eps <= 0, delta outside
 * (0, 1)); the update ops are copied. */
kc_status kc_server_submit_query(kc_server *s, int32_t graph, uint64_t seed, double eps,
                                 double delta, int64_t *ticket);
kc_status kc_server_submit_pool_query(kc_server *s, int32_t graph, double eps, double delta,
                                      int64_t *ticket);
kc_status kc_server_submit_update(kc_server *s, int32_t graph, const kc_edge_op *ops,
                                  int64_t n_ops, int32_t mode, int64_t *ticket);

/* Block until the request is done; *info receives its record. */
kc_status kc_server_wait(kc_server *s, int64_t ticket, kc_request_info *info);

/* Non-blocking: *done = 1 and *info filled when finished, else *done = 0. */
kc_status kc_server_poll(kc_server *s, int64_t ticket, int32_t *done, kc_request_info *info);

/* Block until every submitted request is done. */
kc_status kc_server_drain(kc_server *s);

#ifdef __cplusplus
}
#endif

#endif /* KC_SERVE_H */
