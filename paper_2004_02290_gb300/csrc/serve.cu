// Serving engine: resident indexes, memory-admitted builds and continuous
// batching of query requests (the C ABI of include/ghn_serve.h).
//
// Three host threads share the server's state under one mutex:
//   dispatcher  when a batch slot is free and requests are queued, takes the
//               queued requests in arrival order up to the batch capacity,
//               packs them into the slot's pinned buffer (arguments, offsets,
//               queries), and on the slot's stream issues one host->device
//               copy, one persistent batched query launch per dimension (each
//               request is one entry of the launch; warps steal queries across
//               all of them) and one device->host copy of the results;
//   completers  (one per slot) each take the next launched slot, wait for
//               it, scatter each request's rows to the caller's buffers and
//               complete its ticket; the copies of consecutive batches run
//               in parallel;
//   builder     runs admitted builds (knn_build) on a stream of its own.
// Up to max_inflight slots are on the GPU at once: requests that arrive while
// batches run are queued and form the next batch as soon as a slot frees, and
// that batch's kernels overlap the tail of the ones before it.
//
// Memory admission: a build starts when the server's buffers, the resident
// indexes, the bounds of the builds in progress and the new build's bound fit
// the budget.  The bound is the largest footprint a build of n points in d
// dimensions can reach: its staged inputs, the sort buffers and the largest
// table the build may choose.  Once built, the index counts with its actual
// size.

#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>
#include <time.h>

#include <algorithm>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <numeric>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/ghn_serve.h"
#include "ghn_internal.cuh"

using ghn::BatchArgs;
using ghn::QueryArgs;

namespace {

constexpr int kQuery = 0, kBuild = 1, kDrop = 2;
// launch groups of a batch: (d, buffer width, table kind, stop rule)
constexpr int kGroups = 8 * (ghn::kMaxD + 1);

long long clock_ns()
{
    timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (long long)ts.tv_sec * 1000000000ll + ts.tv_nsec;
}

size_t align16(size_t v) { return (v + 15) & ~size_t(15); }

void set_errf(const char* fmt, ...)
{
    char buf[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    ghn::set_error(buf);
}

struct Ticket {
    long long id = 0;
    int kind = kQuery;
    long long index_id = -1;
    // query request
    const float* q = nullptr;
    long long m = 0;
    int k = 0;
    int mode = -1;
    int d = 0;
    int exact = 0;  // certified stop
    int32_t* ids = nullptr;
    float* dist2 = nullptr;
    void* pred = nullptr;
    const ghn_index* x = nullptr;  // set at dispatch
    int group = 0;                 // launch group within its batch
    // build request
    const float* points = nullptr;
    const void* labels = nullptr;
    long long n = 0;
    float w = 0.0f;
    int table = 0;
    long long reserve = 0;
    // outcome
    int status = KNN_OK;
    bool done = false;
    long long batch = -1;
    long long t_submit = 0, t_dispatch = 0, t_done = 0;
};
using TicketP = std::shared_ptr<Ticket>;

struct IndexEntry {
    ghn_index* x = nullptr;
    int d = 0;
    bool has_labels = false;
    bool building = true;   // build requested, not finished
    bool ready = false;     // built and resident
    bool dropping = false;  // no new requests
    long long queued = 0;   // requests submitted and not yet dispatched (parked included)
    long long inflight = 0; // requests in batches on the GPU
    long long bytes = 0;
    std::vector<TicketP> parked;  // requests that arrived during the build
    TicketP drop;
};

// One batch slot: buffers for the largest batch, a stream and an event.
struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t event = nullptr;
    char* dmeta = nullptr;  // device: arguments, offsets, counters, queries
    char* hmeta = nullptr;  // pinned mirror
    char* dout = nullptr;   // device: status words, predictions, ids, distances
    char* hout = nullptr;   // pinned mirror
    unsigned int* dheavy = nullptr;
    // the batch on the slot
    long long batch = -1;
    std::vector<TicketP> reqs;   // in launch order (grouped by dimension)
    std::vector<size_t> q_at;    // per request: first query of the batch
    std::vector<size_t> o_at;    // per request: first neighbour row
    size_t off_status = 0, off_pred = 0, off_ids = 0, off_d2 = 0;
    int launch_status = KNN_OK;
};

// Largest device footprint of a build of n points: staged inputs, keys and
// values double-buffered for the sort, cell lists and scan space, the rows,
// and the largest table the build may pick (dense: at most 4n + 1024
// entries; hash: at most 4n slots of 16 bytes plus an occupancy bitmap of at
// most 64n bytes).
long long build_bound(long long n, int d, bool labels)
{
    const long long P = ghn::row_floats(d);
    long long b = n * d * 4 + (labels ? n * 8 : 0);  // staged points, labels, kept labels
    b += n * (16 + 8) + n * 8 + n * 12;              // sort pairs, flags/ids, cells
    b += n * (P * 4 + 4);                            // rows, row ids
    b += std::max(n * 4 * 4 + 4096, n * 64 + n * 64);  // table
    return b + (64ll << 20);                          // sort and scan scratch
}

}  // namespace

struct ghn_server {
    knn_server_config cfg{};
    int sms = 0;
    std::mutex mu;
    std::condition_variable cv_dispatch, cv_complete, cv_build, cv_done;
    bool stop = false;
    long long next_ticket = 1, next_index = 1, next_batch = 0;
    std::unordered_map<long long, TicketP> tickets;
    std::unordered_map<long long, IndexEntry> indexes;
    std::deque<TicketP> queue;            // query requests whose index is resident
    std::deque<TicketP> builds_waiting;   // not admitted yet
    std::deque<TicketP> builds_admitted;  // admitted, not started
    int builds_running = 0;
    std::vector<Slot> slots;
    std::vector<int> free_slots;
    std::deque<int> launched;  // slots on the GPU not yet taken by a completer, in launch order
    int inflight = 0;          // slots launched and not yet completed
    long long resident = 0, reserved = 0, buffers = 0;
    knn_server_stats_t st{};
    cudaStream_t build_stream = nullptr;
    std::thread dispatcher, builder;
    std::vector<std::thread> completers;

    size_t cap_args() const { return align16((size_t)cfg.max_batch_requests * sizeof(QueryArgs)); }
    size_t cap_qoff() const { return align16(((size_t)cfg.max_batch_requests + kGroups) * 8); }
    size_t cap_cnt() const { return align16((size_t)kGroups * 32); }
    size_t meta_bytes() const
    {
        return cap_args() + cap_qoff() + cap_cnt() +
               align16((size_t)cfg.max_batch_queries * ghn::kMaxD * 4);
    }
    size_t out_bytes() const
    {
        return align16((size_t)cfg.max_batch_requests * 4) +
               align16((size_t)cfg.max_batch_queries * 4) +
               2 * align16((size_t)cfg.max_batch_outputs * 4);
    }

    void dispatch_loop();
    void complete_loop();
    void build_loop();
    void pack_and_launch(Slot& sl);
    void admit_builds();            // under mu
    void finish_drop(long long id);  // under mu
    void complete(const TicketP& t, int status, long long when);  // under mu
};

// ---------------------------------------------------------------------------
// Bookkeeping (all under mu)
// ---------------------------------------------------------------------------

void ghn_server::complete(const TicketP& t, int status, long long when)
{
    t->status = status;
    t->t_done = when;
    t->done = true;
    cv_done.notify_all();
}

void ghn_server::admit_builds()
{
    while (!builds_waiting.empty()) {
        const TicketP& t = builds_waiting.front();
        if (buffers + resident + reserved + t->reserve > cfg.memory_budget) break;
        reserved += t->reserve;
        t->t_dispatch = clock_ns();
        builds_admitted.push_back(t);
        builds_waiting.pop_front();
        cv_build.notify_one();
    }
}

// Release a dropped index once nothing submitted before the drop still needs it.
void ghn_server::finish_drop(long long id)
{
    auto it = indexes.find(id);
    if (it == indexes.end()) return;
    IndexEntry& e = it->second;
    if (!e.dropping || !e.drop || e.building || e.queued > 0 || e.inflight > 0) return;
    if (e.x) knn_free(e.x);
    resident -= e.bytes;
    TicketP d = e.drop;
    indexes.erase(it);
    ++st.drops_done;
    complete(d, KNN_OK, clock_ns());
    admit_builds();
}

// ---------------------------------------------------------------------------
// Dispatcher: batch formation and launch
// ---------------------------------------------------------------------------

void ghn_server::dispatch_loop()
{
    cudaSetDevice(cfg.device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        cv_dispatch.wait(lk, [&] { return stop || (!queue.empty() && !free_slots.empty()); });
        if (queue.empty() || free_slots.empty()) {
            if (stop) break;
            continue;
        }
        const int si = free_slots.back();
        free_slots.pop_back();
        Slot& sl = slots[si];
        sl.reqs.clear();
        long long nq = 0, no = 0;
        while (!queue.empty() && (long long)sl.reqs.size() < cfg.max_batch_requests) {
            const TicketP& t = queue.front();
            if (nq + t->m > cfg.max_batch_queries || no + t->m * t->k > cfg.max_batch_outputs) break;
            nq += t->m;
            no += t->m * t->k;
            IndexEntry& e = indexes[t->index_id];
            --e.queued;
            ++e.inflight;
            t->x = e.x;
            sl.reqs.push_back(t);
            queue.pop_front();
        }
        sl.batch = next_batch++;
        const long long now = clock_ns();
        for (auto& t : sl.reqs) {
            t->t_dispatch = now;
            t->batch = sl.batch;
        }
        ++st.batches;
        st.max_batch_requests_seen = std::max(st.max_batch_requests_seen, (int64_t)sl.reqs.size());
        st.max_batch_queries_seen = std::max(st.max_batch_queries_seen, (int64_t)nq);
        lk.unlock();
        const long long t0 = clock_ns();
        pack_and_launch(sl);
        const long long t1 = clock_ns();
        lk.lock();
        st.pack_ns += t1 - t0;
        ++inflight;
        launched.push_back(si);
        cv_complete.notify_one();
    }
}

void ghn_server::pack_and_launch(Slot& sl)
{
    const size_t E = sl.reqs.size();
    // group the requests by dimension, buffer width (k <= 32 or not) and table
    // kind (stable: arrival order inside a group); each group is one launch of
    // a kernel specialised for all three
    for (auto& t : sl.reqs) {
        QueryArgs a;
        memset(&a, 0, sizeof(a));
        ghn::index_query_args(t->x, a);
        t->group = t->d * 8 + (t->k > 32 ? 4 : 0) + (a.dense ? 2 : 0) + t->exact;
    }
    std::stable_sort(sl.reqs.begin(), sl.reqs.end(),
                     [](const TicketP& a, const TicketP& b) { return a->group < b->group; });
    sl.q_at.assign(E, 0);
    sl.o_at.assign(E, 0);
    size_t nq = 0, no = 0, nf = 0;
    for (size_t i = 0; i < E; ++i) {
        sl.q_at[i] = nq;
        sl.o_at[i] = no;
        nq += (size_t)sl.reqs[i]->m;
        no += (size_t)sl.reqs[i]->m * (size_t)sl.reqs[i]->k;
        nf += (size_t)sl.reqs[i]->m * (size_t)sl.reqs[i]->d;
    }
    // compact layouts of this batch
    const size_t off_args = 0;
    const size_t off_qoff = align16(E * sizeof(QueryArgs));
    const size_t off_cnt = off_qoff + align16((E + kGroups) * 8);
    const size_t off_q = off_cnt + cap_cnt();
    const size_t meta = off_q + nf * 4;
    sl.off_status = 0;
    sl.off_pred = align16(E * 4);
    sl.off_ids = sl.off_pred + align16(nq * 4);
    sl.off_d2 = sl.off_ids + align16(no * 4);
    const size_t out = sl.off_d2 + no * 4;

    QueryArgs* ha = reinterpret_cast<QueryArgs*>(sl.hmeta + off_args);
    unsigned long long* hq = reinterpret_cast<unsigned long long*>(sl.hmeta + off_qoff);
    memset(sl.hmeta + off_cnt, 0, cap_cnt());
    float* hqf = reinterpret_cast<float*>(sl.hmeta + off_q);
    const QueryArgs* da = reinterpret_cast<const QueryArgs*>(sl.dmeta + off_args);
    const unsigned long long* dq = reinterpret_cast<const unsigned long long*>(sl.dmeta + off_qoff);
    unsigned long long* dc = reinterpret_cast<unsigned long long*>(sl.dmeta + off_cnt);
    const float* dqf = reinterpret_cast<const float*>(sl.dmeta + off_q);

    std::vector<BatchArgs> groups;
    size_t qf = 0, qoff_at = 0;
    for (size_t i = 0; i < E;) {
        const int d = sl.reqs[i]->d, key = sl.reqs[i]->group;
        size_t j = i;
        BatchArgs g{};
        g.args = da + i;
        g.qoff = dq + qoff_at;
        g.d = d;
        g.ns = (key & 4) ? 2 : 1;
        g.dense = (key >> 1) & 1;
        g.exact = key & 1;
        unsigned long long acc = 0;
        for (; j < E && sl.reqs[j]->group == key; ++j) {
            const Ticket& t = *sl.reqs[j];
            QueryArgs a;
            memset(&a, 0, sizeof(a));
            ghn::index_query_args(t.x, a);
            memcpy(hqf + qf, t.q, (size_t)t.m * (size_t)d * 4);
            a.q = dqf + qf;
            qf += (size_t)t.m * (size_t)d;
            a.m = t.m;
            a.k = t.k;
            a.mode = t.mode;
            a.ids = reinterpret_cast<int*>(sl.dout + sl.off_ids) + sl.o_at[j];
            a.dist2 = reinterpret_cast<float*>(sl.dout + sl.off_d2) + sl.o_at[j];
            a.pred = t.mode >= 0 ? (void*)(reinterpret_cast<unsigned int*>(sl.dout + sl.off_pred) +
                                           sl.q_at[j])
                                 : nullptr;
            a.status = reinterpret_cast<unsigned int*>(sl.dout + sl.off_status) + j;
            a.exact = t.exact;
            ha[j] = a;
            hq[qoff_at + (j - i)] = acc;
            acc += (unsigned long long)t.m;
        }
        hq[qoff_at + (j - i)] = acc;
        g.count = (int)(j - i);
        g.total = acc;
        unsigned long long* c = dc + 4 * groups.size();
        g.counter = c;
        g.heavy_count = reinterpret_cast<unsigned int*>(c + 1);
        g.heavy_cursor = reinterpret_cast<unsigned int*>(c + 2);
        g.heavy_list = sl.dheavy;
        groups.push_back(g);
        qoff_at += (j - i) + 1;
        i = j;
    }

    cudaError_t e = cudaMemcpyAsync(sl.dmeta, sl.hmeta, meta, cudaMemcpyHostToDevice, sl.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(sl.dout, 0, E * 4, sl.stream);
    // the groups share the deferral list: they run one after another on the stream
    for (const BatchArgs& g : groups)
        if (e == cudaSuccess) e = ghn::launch_batch_query(g, sms, sl.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sl.hout, sl.dout, out, cudaMemcpyDeviceToHost, sl.stream);
    if (e == cudaSuccess) e = cudaEventRecord(sl.event, sl.stream);
    sl.launch_status = e == cudaSuccess ? KNN_OK : KNN_ECUDA;
}

// ---------------------------------------------------------------------------
// Completer: results back to the callers, in launch order
// ---------------------------------------------------------------------------

void ghn_server::complete_loop()
{
    cudaSetDevice(cfg.device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        cv_complete.wait(lk, [&] { return stop || !launched.empty(); });
        if (launched.empty()) {
            if (stop) break;
            continue;
        }
        const int si = launched.front();
        launched.pop_front();
        lk.unlock();
        Slot& sl = slots[si];
        const long long t0 = clock_ns();
        int batch_status = sl.launch_status;
        if (batch_status == KNN_OK && cudaEventSynchronize(sl.event) != cudaSuccess)
            batch_status = KNN_ECUDA;
        const long long t1 = clock_ns();
        if (batch_status != KNN_OK) {
            // whatever was queued before the failure finishes before the
            // slot's buffers are reused
            cudaStreamSynchronize(sl.stream);
            cudaGetLastError();
        }
        std::vector<int> status(sl.reqs.size(), batch_status);
        long long nq = 0;
        if (batch_status == KNN_OK) {
            const unsigned int* hs = reinterpret_cast<const unsigned int*>(sl.hout + sl.off_status);
            for (size_t i = 0; i < sl.reqs.size(); ++i) {
                const Ticket& t = *sl.reqs[i];
                const unsigned int w = hs[i];
                status[i] = (w & ghn::kStatusNonFinite) ? KNN_EINVAL
                            : (w & ghn::kStatusLimit)   ? KNN_ELIMIT
                                                        : KNN_OK;
                const size_t rows = (size_t)t.m * (size_t)t.k;
                memcpy(t.ids, sl.hout + sl.off_ids + sl.o_at[i] * 4, rows * 4);
                if (t.dist2) memcpy(t.dist2, sl.hout + sl.off_d2 + sl.o_at[i] * 4, rows * 4);
                if (t.pred && t.mode >= 0)
                    memcpy(t.pred, sl.hout + sl.off_pred + sl.q_at[i] * 4, (size_t)t.m * 4);
                nq += t.m;
            }
        }
        const long long now = clock_ns();
        lk.lock();
        st.wait_ns += t1 - t0;
        st.scatter_ns += now - t1;
        --inflight;
        for (size_t i = 0; i < sl.reqs.size(); ++i) {
            const TicketP& t = sl.reqs[i];
            complete(t, status[i], now);
            auto it = indexes.find(t->index_id);
            if (it != indexes.end()) {
                --it->second.inflight;
                finish_drop(t->index_id);
            }
        }
        st.requests_done += (int64_t)sl.reqs.size();
        st.queries_done += nq;
        sl.reqs.clear();
        free_slots.push_back(si);
        cv_dispatch.notify_one();
        cv_done.notify_all();
    }
}

// ---------------------------------------------------------------------------
// Builder: admitted builds on the build stream
// ---------------------------------------------------------------------------

void ghn_server::build_loop()
{
    cudaSetDevice(cfg.device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        cv_build.wait(lk, [&] { return stop || !builds_admitted.empty(); });
        if (builds_admitted.empty()) {
            if (stop) break;
            continue;
        }
        TicketP t = builds_admitted.front();
        builds_admitted.pop_front();
        ++builds_running;
        lk.unlock();
        ghn_index* x = nullptr;
        int status = knn_build(t->points, t->labels, t->n, t->d, t->w, t->table, build_stream, &x);
        if (status == KNN_OK && cudaStreamSynchronize(build_stream) != cudaSuccess) {
            status = KNN_ECUDA;
            knn_free(x);
            x = nullptr;
        }
        const long long bytes = x ? ghn::index_bytes(x) : 0;
        const long long now = clock_ns();
        lk.lock();
        --builds_running;
        reserved -= t->reserve;
        ++st.builds_done;
        IndexEntry& e = indexes[t->index_id];
        e.building = false;
        if (status == KNN_OK) {
            e.x = x;
            e.ready = true;
            e.bytes = bytes;
            resident += bytes;
            for (auto& q : e.parked) queue.push_back(q);
            if (!e.parked.empty()) cv_dispatch.notify_one();
        } else {
            // requests waiting for the index fail with it
            for (auto& q : e.parked) {
                complete(q, KNN_EINVAL, now);
                --e.queued;
            }
        }
        e.parked.clear();
        complete(t, status, now);
        if (e.dropping)
            finish_drop(t->index_id);
        else if (status != KNN_OK)
            indexes.erase(t->index_id);
        admit_builds();
    }
}

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------

namespace {

// True for device (or managed) memory; host, pinned and NULL pointers are not.
bool on_device(const void* p)
{
    if (!p) return false;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void fill_info(const Ticket& t, knn_ticket_info* info)
{
    if (!info) return;
    info->status = t.status;
    info->kind = t.kind;
    info->index_id = t.index_id;
    info->batch = t.batch;
    info->t_submit_ns = t.t_submit;
    info->t_dispatch_ns = t.t_dispatch;
    info->t_done_ns = t.t_done;
}

void release_slots(ghn_server* s)
{
    for (Slot& sl : s->slots) {
        if (sl.dmeta) cudaFree(sl.dmeta);
        if (sl.dout) cudaFree(sl.dout);
        if (sl.dheavy) cudaFree(sl.dheavy);
        if (sl.hmeta) cudaFreeHost(sl.hmeta);
        if (sl.hout) cudaFreeHost(sl.hout);
        if (sl.event) cudaEventDestroy(sl.event);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    s->slots.clear();
    if (s->build_stream) cudaStreamDestroy(s->build_stream);
    s->build_stream = nullptr;
}

}  // namespace

extern "C" {

int64_t knn_server_clock_ns(void) { return clock_ns(); }

int64_t knn_server_build_bytes(int64_t n, int32_t d, int32_t labels)
{
    if (n < 1 || d < 1 || d > ghn::kMaxD) return 0;
    return build_bound(n, d, labels != 0);
}

knn_status knn_server_create(const knn_server_config* cfg_in, ghn_server** out)
{
    if (!out) {
        ghn::set_error("knn_server_create: out is NULL");
        return KNN_EINVAL;
    }
    *out = nullptr;
    knn_server_config c{};
    if (cfg_in) c = *cfg_in;
    if (c.memory_budget == 0) c.memory_budget = 60ll << 30;
    if (c.max_batch_queries == 0) c.max_batch_queries = 262144;
    if (c.max_batch_outputs == 0) c.max_batch_outputs = 16 * c.max_batch_queries;
    if (c.max_batch_requests == 0) c.max_batch_requests = 4096;
    if (c.max_inflight == 0) c.max_inflight = 3;
    if (c.memory_budget < 0 || c.max_batch_queries < 1 || c.max_batch_queries > (1ll << 30) ||
        c.max_batch_outputs < 1 || c.max_batch_outputs > (1ll << 31) ||
        c.max_batch_requests < 1 || c.max_batch_requests > (1 << 20) || c.max_inflight < 1 ||
        c.max_inflight > 64 || c.device < 0 || c.reserved != 0) {
        ghn::set_error("knn_server_create: a configuration field is out of range");
        return KNN_EINVAL;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || c.device >= ndev) {
        cudaGetLastError();
        set_errf("knn_server_create: no CUDA device %d", c.device);
        return KNN_EINVAL;
    }
    ghn_server* s = new ghn_server();
    s->cfg = c;
    s->buffers = (long long)c.max_inflight *
                 (long long)(s->meta_bytes() + s->out_bytes() + (size_t)c.max_batch_queries * 4);
    if (s->buffers > c.memory_budget) {
        set_errf("knn_server_create: the batch buffers (%lld bytes) exceed the budget",
                 s->buffers);
        delete s;
        return KNN_ENOMEM;
    }
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(c.device);
    s->sms = ghn::device_sms(c.device);
    cudaError_t e = cudaStreamCreateWithFlags(&s->build_stream, cudaStreamNonBlocking);
    s->slots.resize((size_t)c.max_inflight);
    for (Slot& sl : s->slots) {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.event, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMalloc(&sl.dmeta, s->meta_bytes());
        if (e == cudaSuccess) e = cudaMalloc(&sl.dout, s->out_bytes());
        if (e == cudaSuccess) e = cudaMalloc(&sl.dheavy, (size_t)c.max_batch_queries * 4);
        if (e == cudaSuccess) e = cudaMallocHost(&sl.hmeta, s->meta_bytes());
        if (e == cudaSuccess) e = cudaMallocHost(&sl.hout, s->out_bytes());
    }
    if (e != cudaSuccess) {
        set_errf("knn_server_create: %s", cudaGetErrorString(e));
        cudaGetLastError();
        release_slots(s);
        delete s;
        cudaSetDevice(prev);
        return e == cudaErrorMemoryAllocation ? KNN_ENOMEM : KNN_ECUDA;
    }
    for (int i = 0; i < c.max_inflight; ++i) s->free_slots.push_back(i);
    s->st.buffer_bytes = s->buffers;
    s->st.budget_bytes = c.memory_budget;
    s->dispatcher = std::thread([s] { s->dispatch_loop(); });
    for (int i = 0; i < c.max_inflight; ++i)
        s->completers.emplace_back([s] { s->complete_loop(); });
    s->builder = std::thread([s] { s->build_loop(); });
    cudaSetDevice(prev);
    *out = s;
    return KNN_OK;
}

knn_status knn_server_build(ghn_server* s, const float* points, const void* labels, int64_t n,
                            int32_t d, float cell_width, int32_t table, int64_t* index_id,
                            int64_t* ticket)
{
    if (!s || !points || !index_id || !ticket) {
        ghn::set_error("knn_server_build: NULL argument");
        return KNN_EINVAL;
    }
    // the arguments knn_build checks without the device, checked here so that
    // a bad request fails at once
    if (n < 1 || n >= (1ll << 31) || d < 1 || d > ghn::kMaxD || !(cell_width > 0.0f) ||
        !(cell_width < INFINITY) || table < 0 || table > 2) {
        ghn::set_error("knn_server_build: bad n, d, cell width or table");
        return KNN_EINVAL;
    }
    auto t = std::make_shared<Ticket>();
    t->kind = kBuild;
    t->points = points;
    t->labels = labels;
    t->n = n;
    t->d = d;
    t->w = cell_width;
    t->table = table;
    t->reserve = build_bound(n, d, labels != nullptr);
    t->t_submit = clock_ns();
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->buffers + t->reserve > s->cfg.memory_budget) {
        set_errf("knn_server_build: a build of %lld points may need %lld bytes, more than the "
                 "budget leaves beside the batch buffers", (long long)n, t->reserve);
        return KNN_ENOMEM;
    }
    t->id = s->next_ticket++;
    t->index_id = s->next_index++;
    IndexEntry& e = s->indexes[t->index_id];
    e.d = d;
    e.has_labels = labels != nullptr;
    s->tickets[t->id] = t;
    s->builds_waiting.push_back(t);
    s->admit_builds();
    *index_id = t->index_id;
    *ticket = t->id;
    return KNN_OK;
}

knn_status knn_server_drop(ghn_server* s, int64_t index_id, int64_t* ticket)
{
    if (!s || !ticket) {
        ghn::set_error("knn_server_drop: NULL argument");
        return KNN_EINVAL;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->indexes.find(index_id);
    if (it == s->indexes.end() || it->second.dropping) {
        set_errf("knn_server_drop: unknown or dropped index %lld", (long long)index_id);
        return KNN_EINVAL;
    }
    auto t = std::make_shared<Ticket>();
    t->kind = kDrop;
    t->index_id = index_id;
    t->t_submit = t->t_dispatch = clock_ns();
    t->id = s->next_ticket++;
    s->tickets[t->id] = t;
    it->second.dropping = true;
    it->second.drop = t;
    *ticket = t->id;
    s->finish_drop(index_id);
    return KNN_OK;
}

}  // extern "C"

namespace {

// Checks of a query request that need no lock; the request's ticket on success.
knn_status make_request(ghn_server* s, int64_t index_id, const float* queries, int64_t m,
                        int32_t k, int32_t mode, int32_t* ids, float* dist2, void* pred,
                        int32_t flags, const char* who, TicketP& out)
{
    if (flags & ~KNN_QUERY_EXACT) {
        set_errf("%s: flags may only hold KNN_QUERY_EXACT", who);
        return KNN_EINVAL;
    }
    if (m < 0 || k < 1 || k > ghn::kMaxK || mode < -1 || mode > 2) {
        set_errf("%s: m must be >= 0, k in [1, 64], mode in {-1, 0, 1, 2}", who);
        return KNN_EINVAL;
    }
    if (m > 0 && (!queries || !ids || (mode >= 0 && !pred))) {
        set_errf("%s: queries, ids (and pred for a prediction) are required", who);
        return KNN_EINVAL;
    }
    if (m > 0 && (on_device(queries) || on_device(ids) || on_device(dist2) || on_device(pred))) {
        set_errf("%s: queries and outputs must be host memory", who);
        return KNN_EINVAL;
    }
    if (m > s->cfg.max_batch_queries || m * (int64_t)k > s->cfg.max_batch_outputs) {
        set_errf("%s: %lld queries x k = %d exceed one batch", who, (long long)m, k);
        return KNN_EINVAL;
    }
    auto t = std::make_shared<Ticket>();
    t->kind = kQuery;
    t->index_id = index_id;
    t->q = queries;
    t->m = m;
    t->k = k;
    t->mode = mode;
    t->ids = ids;
    t->dist2 = dist2;
    t->pred = mode >= 0 ? pred : nullptr;
    t->exact = (flags & KNN_QUERY_EXACT) ? 1 : 0;
    out = std::move(t);
    return KNN_OK;
}

// The checks against the server's indexes (under mu).
knn_status check_index(ghn_server* s, const Ticket& t, const char* who)
{
    auto it = s->indexes.find(t.index_id);
    if (it == s->indexes.end() || it->second.dropping) {
        set_errf("%s: unknown or dropped index %lld", who, (long long)t.index_id);
        return KNN_EINVAL;
    }
    if (t.mode >= 0 && !it->second.has_labels) {
        set_errf("%s: a prediction needs an index built with labels", who);
        return KNN_EINVAL;
    }
    return KNN_OK;
}

// Register a checked request and queue it (under mu).
int64_t enqueue(ghn_server* s, const TicketP& t, long long now)
{
    IndexEntry& e = s->indexes[t->index_id];
    t->d = e.d;
    t->t_submit = now;
    t->id = s->next_ticket++;
    s->tickets[t->id] = t;
    if (t->m == 0) {
        t->t_dispatch = now;
        s->complete(t, KNN_OK, now);
        return t->id;
    }
    ++e.queued;
    if (e.ready) {
        s->queue.push_back(t);
    } else {
        e.parked.push_back(t);
    }
    return t->id;
}

}  // namespace

extern "C" {

knn_status knn_server_submit(ghn_server* s, int64_t index_id, const float* queries, int64_t m,
                             int32_t k, int32_t mode, int32_t* ids, float* dist2, void* pred,
                             int32_t flags, int64_t* ticket)
{
    if (!s || !ticket) {
        ghn::set_error("knn_server_submit: NULL argument");
        return KNN_EINVAL;
    }
    TicketP t;
    knn_status st = make_request(s, index_id, queries, m, k, mode, ids, dist2, pred, flags,
                                 "knn_server_submit", t);
    if (st != KNN_OK) return st;
    const long long now = clock_ns();
    std::lock_guard<std::mutex> lk(s->mu);
    if ((st = check_index(s, *t, "knn_server_submit")) != KNN_OK) return st;
    *ticket = enqueue(s, t, now);
    s->cv_dispatch.notify_one();
    return KNN_OK;
}

knn_status knn_server_submit_many(ghn_server* s, int32_t count, const int64_t* index_ids,
                                  const float* const* queries, const int64_t* m, const int32_t* k,
                                  const int32_t* mode, int32_t* const* ids, float* const* dist2,
                                  void* const* pred, const int32_t* flags, int64_t* tickets)
{
    if (!s || count < 0 || (count > 0 && (!index_ids || !queries || !m || !k || !mode || !ids ||
                                          !tickets))) {
        ghn::set_error("knn_server_submit_many: NULL argument or negative count");
        return KNN_EINVAL;
    }
    std::vector<TicketP> ts((size_t)count);
    for (int32_t i = 0; i < count; ++i) {
        char who[64];
        snprintf(who, sizeof who, "knn_server_submit_many: request %d", i);
        knn_status st = make_request(s, index_ids[i], queries[i], m[i], k[i], mode[i], ids[i],
                                     dist2 ? dist2[i] : nullptr, pred ? pred[i] : nullptr,
                                     flags ? flags[i] : 0, who, ts[(size_t)i]);
        if (st != KNN_OK) return st;
    }
    const long long now = clock_ns();
    std::lock_guard<std::mutex> lk(s->mu);
    for (int32_t i = 0; i < count; ++i) {
        char who[64];
        snprintf(who, sizeof who, "knn_server_submit_many: request %d", i);
        knn_status st = check_index(s, *ts[(size_t)i], who);
        if (st != KNN_OK) return st;  // nothing queued yet
    }
    for (int32_t i = 0; i < count; ++i) tickets[i] = enqueue(s, ts[(size_t)i], now);
    s->cv_dispatch.notify_one();
    return KNN_OK;
}

static knn_status wait_impl(ghn_server* s, int64_t ticket, int64_t timeout_us,
                            knn_ticket_info* info, int32_t* done_out)
{
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->tickets.find(ticket);
    if (it == s->tickets.end()) {
        set_errf("knn_server_wait: unknown ticket %lld", (long long)ticket);
        return KNN_EINVAL;
    }
    TicketP t = it->second;
    if (timeout_us < 0)
        s->cv_done.wait(lk, [&] { return t->done; });
    else if (timeout_us > 0)
        s->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return t->done; });
    if (done_out) *done_out = t->done ? 1 : 0;
    if (!t->done) return done_out ? KNN_OK : KNN_ETIMEDOUT;
    fill_info(*t, info);
    s->tickets.erase(ticket);
    return KNN_OK;
}

knn_status knn_server_wait(ghn_server* s, int64_t ticket, int64_t timeout_us,
                           knn_ticket_info* info)
{
    if (!s) {
        ghn::set_error("knn_server_wait: NULL server");
        return KNN_EINVAL;
    }
    return wait_impl(s, ticket, timeout_us, info, nullptr);
}

knn_status knn_server_test(ghn_server* s, int64_t ticket, int32_t* done, knn_ticket_info* info)
{
    if (!s || !done) {
        ghn::set_error("knn_server_test: NULL argument");
        return KNN_EINVAL;
    }
    return wait_impl(s, ticket, 0, info, done);
}

knn_status knn_server_index(ghn_server* s, int64_t index_id, const ghn_index** index)
{
    if (!s || !index) {
        ghn::set_error("knn_server_index: NULL argument");
        return KNN_EINVAL;
    }
    *index = nullptr;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->indexes.find(index_id);
    if (it == s->indexes.end() || it->second.dropping || !it->second.ready) {
        set_errf("knn_server_index: index %lld is unknown, dropped or not built", (long long)index_id);
        return KNN_EINVAL;
    }
    *index = it->second.x;
    return KNN_OK;
}

knn_status knn_server_stats(ghn_server* s, knn_server_stats_t* out)
{
    if (!s || !out) {
        ghn::set_error("knn_server_stats: NULL argument");
        return KNN_EINVAL;
    }
    std::lock_guard<std::mutex> lk(s->mu);
    knn_server_stats_t v = s->st;
    v.indexes = (int64_t)s->indexes.size();
    v.resident_bytes = s->resident;
    v.reserved_bytes = s->reserved;
    v.buffer_bytes = s->buffers;
    v.budget_bytes = s->cfg.memory_budget;
    long long queued = (long long)s->queue.size();
    for (auto& kv : s->indexes) queued += (long long)kv.second.parked.size();
    v.queued_requests = queued;
    v.waiting_builds = (int64_t)s->builds_waiting.size();
    v.inflight_batches = (int64_t)s->inflight;
    *out = v;
    return KNN_OK;
}

void knn_server_destroy(ghn_server* s)
{
    if (!s) return;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        // builds still waiting for memory will not get it: fail them
        const long long now = clock_ns();
        for (auto& t : s->builds_waiting) {
            s->complete(t, KNN_ENOMEM, now);
            IndexEntry& e = s->indexes[t->index_id];
            for (auto& q : e.parked) s->complete(q, KNN_EINVAL, now);
            s->indexes.erase(t->index_id);
        }
        s->builds_waiting.clear();
        // finish everything admitted
        s->cv_done.wait(lk, [&] {
            return s->queue.empty() && s->inflight == 0 && s->builds_admitted.empty() &&
                   s->builds_running == 0;
        });
        s->stop = true;
        s->cv_dispatch.notify_all();
        s->cv_complete.notify_all();
        s->cv_build.notify_all();
    }
    s->dispatcher.join();
    for (auto& t : s->completers) t.join();
    s->builder.join();
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(s->cfg.device);
    for (auto& kv : s->indexes)
        if (kv.second.x) knn_free(kv.second.x);
    s->indexes.clear();
    cudaDeviceSynchronize();
    release_slots(s);
    cudaSetDevice(prev);
    delete s;
}

}  // extern "C"
