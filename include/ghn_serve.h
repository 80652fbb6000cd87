/*
 * ghn_serve.h: C ABI of the serving engine of the grid-hashing KNN library.
 *
 * The paper answers one observation at a time (Sec. III.B, Algorithm 2); a
 * server answers many callers whose requests target many indexes.  It keeps
 * indexes resident in device memory, admits index builds by memory, and
 * serves query requests by continuous batching:
 *   - every query request queued when a batch slot frees up joins the next
 *     batch (any index, any k and head), up to the batch capacity;
 *   - a batch is one host->device copy, one persistent query launch per
 *     dimension with per-query work stealing across its requests (the
 *     kernels of knn_batch_query), and one device->host copy, on the slot's
 *     own stream;
 *   - up to max_inflight batches are on the GPU at once, so requests that
 *     arrive while batches run form the next batch and its work overlaps
 *     theirs on the device;
 *   - builds run on a stream of their own, overlapping query batches.
 * Each request's results equal those of knn_query on the same index with the
 * same arguments (every query is computed independently of its batch).
 *
 * Threads: all entry points may be called from any host thread.  Requests
 * complete asynchronously; knn_server_wait / knn_server_test return their
 * outcome and release the ticket.
 */
#ifndef GHN_SERVE_H
#define GHN_SERVE_H

#include "ghn_knn.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ghn_server ghn_server; /* opaque */

/* Zero fields take the defaults given here. */
typedef struct {
    int64_t memory_budget;      /* device bytes the server may hold: its batch buffers, the
                                   resident indexes and the builds in progress (60 GiB) */
    int64_t max_batch_queries;  /* queries per batch (262144) */
    int64_t max_batch_outputs;  /* neighbour rows per batch, the sum of m*k (16x queries) */
    int32_t max_batch_requests; /* requests per batch (4096) */
    int32_t max_inflight;       /* batches on the GPU at once (3) */
    int32_t device;             /* CUDA device; 0 is device 0 */
    int32_t reserved;           /* must be 0 */
} knn_server_config;

/* Outcome of a request. */
typedef struct {
    int32_t status;        /* knn_status of the request itself */
    int32_t kind;          /* 0 query, 1 build, 2 drop */
    int64_t index_id;      /* index the request names (a build: the new index) */
    int64_t batch;         /* batch that served a query request, else -1 */
    int64_t t_submit_ns;   /* CLOCK_MONOTONIC times: submission, */
    int64_t t_dispatch_ns; /* start (batch launch, or build admission), */
    int64_t t_done_ns;     /* and completion (results in the caller's buffers) */
} knn_ticket_info;

typedef struct {
    int64_t batches;          /* query batches launched */
    int64_t requests_done;    /* query requests completed */
    int64_t queries_done;     /* queries of those requests */
    int64_t builds_done;      /* builds completed (successful or not) */
    int64_t drops_done;
    int64_t indexes;          /* indexes known (building or resident) */
    int64_t resident_bytes;   /* device bytes of the resident indexes */
    int64_t reserved_bytes;   /* bound on the builds in progress */
    int64_t buffer_bytes;     /* the server's own batch buffers */
    int64_t budget_bytes;
    int64_t queued_requests;  /* query requests not yet in a batch */
    int64_t waiting_builds;   /* builds not yet admitted */
    int64_t inflight_batches;
    int64_t max_batch_requests_seen;
    int64_t max_batch_queries_seen;
    int64_t pack_ns;          /* host time packing and launching batches */
    int64_t wait_ns;          /* host time waiting for batches to finish */
    int64_t scatter_ns;       /* host time copying results to the callers' buffers */
} knn_server_stats_t;

/*
 * knn_server_create: a server on cfg->device (cfg may be NULL: defaults).
 * Allocates the batch buffers (device and pinned host) and starts the
 * server's threads.  KNN_EINVAL for a bad field; KNN_ENOMEM when the buffers
 * do not fit the budget or the device.
 */
knn_status knn_server_create(const knn_server_config* cfg, ghn_server** out);

/*
 * knn_server_build: request a new index (the arguments of knn_build; points
 * and labels host or device, borrowed until the request completes).  Returns
 * at once with the new index's id and a ticket.  The build starts when a
 * bound on its peak footprint fits the budget beside what the server holds;
 * builds start in arrival order.  Queries may be submitted against the id at
 * once: they wait for the build.  KNN_ENOMEM when the build could not fit
 * even in an empty server; build errors are the ticket's status.
 */
knn_status knn_server_build(ghn_server* server, const float* points, const void* labels,
                            int64_t n, int32_t d, float cell_width, int32_t table,
                            int64_t* index_id, int64_t* ticket);

/*
 * knn_server_build_bytes: the device bytes a build of n points in d
 * dimensions (with or without labels) is admitted with: a bound on its peak
 * footprint (staged inputs, sort buffers, the largest table it may choose).
 * Once built, an index counts with its actual size.
 */
int64_t knn_server_build_bytes(int64_t n, int32_t d, int32_t labels);

/*
 * knn_server_drop: release an index once the requests submitted before the
 * drop have completed.  Later requests naming it get KNN_EINVAL.
 */
knn_status knn_server_drop(ghn_server* server, int64_t index_id, int64_t* ticket);

/*
 * knn_server_submit: a query request (the arguments of knn_query; results as
 * knn_query's with KNN_QUERY_CHECKED: the ticket's status is KNN_EINVAL for
 * a non-finite query and KNN_ELIMIT for one that reached its work bound, as knn_query).
 *   flags    0 or KNN_QUERY_EXACT (the certified stop for this request).
 *   queries  host, m*d float32 of the index's d; borrowed until completion.
 *   ids      host, m*k int32; dist2 host m*k float32 or NULL; pred host m
 *            values (int32 for KNN_VOTE, float32 for KNN_MEAN / KNN_MEDIAN)
 *            or NULL.  Written before the ticket completes.
 * KNN_EINVAL for bad arguments, an unknown or dropped index, or a request
 * larger than one batch (m > max_batch_queries or m*k > max_batch_outputs).
 */
knn_status knn_server_submit(ghn_server* server, int64_t index_id, const float* queries,
                             int64_t m, int32_t k, int32_t mode, int32_t* ids, float* dist2,
                             void* pred, int32_t flags, int64_t* ticket);

/*
 * knn_server_submit_many: `count` query requests in one call (host arrays of
 * count entries, each as knn_server_submit's argument of the same name;
 * dist2, pred and flags may be NULL for none).  Every request is checked
 * before any is queued: on an error nothing is queued, and the message names
 * the request.  tickets receives count tickets.
 */
knn_status knn_server_submit_many(ghn_server* server, int32_t count, const int64_t* index_ids,
                                  const float* const* queries, const int64_t* m, const int32_t* k,
                                  const int32_t* mode, int32_t* const* ids, float* const* dist2,
                                  void* const* pred, const int32_t* flags, int64_t* tickets);

/*
 * knn_server_wait: wait up to timeout_us (negative: no limit) for a ticket.
 * KNN_OK when it completed (info, may be NULL, receives its outcome, and the
 * ticket is released); KNN_ETIMEDOUT when it has not completed yet;
 * KNN_EINVAL for an unknown ticket.
 */
knn_status knn_server_wait(ghn_server* server, int64_t ticket, int64_t timeout_us,
                           knn_ticket_info* info);

/*
 * knn_server_index: the resident index behind an id, for plain calls
 * (knn_query, knn_index_info) beside the server.  Borrowed: valid until the
 * index is dropped or the server destroyed; never pass it to knn_free.
 * KNN_EINVAL when the id is unknown, dropped or not built yet.
 */
knn_status knn_server_index(ghn_server* server, int64_t index_id, const ghn_index** index);

/* knn_server_test: knn_server_wait without waiting (*done = 0 or 1). */
knn_status knn_server_test(ghn_server* server, int64_t ticket, int32_t* done,
                           knn_ticket_info* info);

knn_status knn_server_stats(ghn_server* server, knn_server_stats_t* stats);

/* CLOCK_MONOTONIC now, in ns (the clock of knn_ticket_info). */
int64_t knn_server_clock_ns(void);

/*
 * knn_server_destroy: finish every admitted request, fail builds still
 * waiting for memory (KNN_ENOMEM), release every index and buffer.
 * NULL-safe.  Tickets not yet waited for are released.
 */
void knn_server_destroy(ghn_server* server);

#ifdef __cplusplus
}
#endif

#endif /* GHN_SERVE_H */
