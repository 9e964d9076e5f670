// server.cu -- the served form: continuous batching of arriving transactions.
//
// Every lane owns a ring of `depth` batch slots, each with pinned host and
// device buffers sized for a full batch.  Arriving transactions are copied
// into the lane's forming slot; a slot launches when it is full (transaction
// cap or write-set budget), when its oldest request has waited max_delay, or
// as soon as none of the lane's batches is in flight.
// A launch is three stream-ordered steps on three streams per lane:
//   h2d stream   : inputs host -> device, event `in`
//   exec stream  : waits `in`, gcc_execute on the lane's database, event `exec`
//   d2h stream   : waits `exec`, results, read values and batch state back,
//                  event `out`
// so the next batch's upload overlaps the current execution, and lanes on
// different databases execute concurrently.  A trace run gives every lane two
// host threads -- a feeder (admission, batch forming, launches) and a
// completer (finished batches, completions, freeing slots) -- since at
// millions of requests per second the host work per request, not the GPU,
// bounds one thread.  They hand slots over through each slot's state word and
// a ring of launched slots (release/acquire); lanes share no state but the
// server's read-only parameters.  Batches of one lane run in the
// order they were launched on its exec stream; a slot becomes free when its
// `out` event has completed and its completions have been emitted.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "runtime.cuh"

using namespace gcc::rt;

namespace {

uint64_t now_ns() {
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

enum SlotState { FREE, FORMING, INFLIGHT };

struct Slot {
    gcc_txn* h_txns = nullptr;
    gcc_op* h_ops = nullptr;
    gcc_operand* h_opd = nullptr;
    gcc_txn_result* h_res = nullptr;
    gcc_operand* h_reads = nullptr;
    gcc::BatchState* h_state = nullptr;
    gcc_txn* d_txns = nullptr;
    gcc_op* d_ops = nullptr;
    gcc_operand* d_opd = nullptr;
    gcc_txn_result* d_res = nullptr;
    gcc_operand* d_reads = nullptr;
    cudaEvent_t ev_in = nullptr, ev_exec = nullptr, ev_out = nullptr;
    uint32_t n_txns = 0;
    uint64_t n_ops = 0, write_bytes = 0, seq = 0, oldest = 0;
    std::vector<uint64_t> req, arrival;
    int state = FREE;                   // SlotState; read and written atomically
};

// A slot's state is the hand-off between a lane's feeder (FREE -> FORMING ->
// INFLIGHT) and its completer (INFLIGHT -> FREE): release stores, acquire loads.
int state_of(const Slot& sl) { return __atomic_load_n(&sl.state, __ATOMIC_ACQUIRE); }
void set_state(Slot& sl, int st) { __atomic_store_n(&sl.state, st, __ATOMIC_RELEASE); }

// A request waiting for a free slot.  Requests of a trace point into the
// trace's arrays, which outlive the run; requests enqueued one by one own a
// copy (the caller may reuse its buffers).
struct Pending {
    gcc_txn txn;
    const gcc_op* ops;                 // ops and operands of the request: either
    const gcc_operand* opd;            // the caller's, or own_ops / own_opd
    std::vector<gcc_op> own_ops;
    std::vector<gcc_operand> own_opd;
    uint64_t arrival, id;
};

struct Lane {
    gcc_server_lane cfg{};
    uint64_t ops_cap = 0;
    cudaStream_t h2d = nullptr, exec = nullptr, d2h = nullptr;
    std::vector<Slot> slots;
    int forming = -1;
    // launched slots in launch order: a ring written by the feeder (tail) and
    // read by the completer (head), depth <= 8 entries
    int ring[8] = {0};
    uint32_t head = 0, tail = 0;
    std::deque<Pending> backlog;
    uint64_t next_seq = 0;
    uint64_t committed = 0, aborts = 0, batches = 0;
    uint64_t trace_done = 0;            // trace run: this lane's completions so far
};

}  // namespace

struct gcc_server {
    int device = 0;
    gcc_exec_params params{};
    std::vector<Lane> lanes;
    std::deque<gcc_completion> done;
    std::deque<std::vector<gcc_operand>> done_reads;
    uint64_t next_id = 0;
    // trace mode: results land directly in caller arrays
    gcc_completion* trace_out = nullptr;
    gcc_operand* trace_reads = nullptr;
    const gcc_txn* trace_txns = nullptr;
};

namespace {

void free_server(gcc_server* s) {
    cudaSetDevice(s->device);
    for (Lane& l : s->lanes) {
        for (cudaStream_t st : {l.h2d, l.exec, l.d2h})
            if (st) cudaStreamSynchronize(st);
        for (Slot& sl : l.slots) {
            cudaFreeHost(sl.h_txns);
            cudaFreeHost(sl.h_ops);
            cudaFreeHost(sl.h_opd);
            cudaFreeHost(sl.h_res);
            cudaFreeHost(sl.h_reads);
            cudaFreeHost(sl.h_state);
            cudaFree(sl.d_txns);
            cudaFree(sl.d_ops);
            cudaFree(sl.d_opd);
            cudaFree(sl.d_res);
            cudaFree(sl.d_reads);
            for (cudaEvent_t e : {sl.ev_in, sl.ev_exec, sl.ev_out})
                if (e) cudaEventDestroy(e);
        }
        for (cudaStream_t st : {l.h2d, l.exec, l.d2h})
            if (st) cudaStreamDestroy(st);
    }
    delete s;
}

bool writes(uint8_t kind) { return gcc::kind_writes(kind); }

gcc_status launch(gcc_server* s, Lane& l) {
    Slot& sl = l.slots[l.forming];
    l.forming = -1;
    sl.seq = l.next_seq++;
    set_state(sl, INFLIGHT);
    const uint64_t tb = (uint64_t)sl.n_txns * sizeof(gcc_txn), ob = sl.n_ops * sizeof(gcc_op),
                   pb = sl.n_ops * sizeof(gcc_operand);
    cudaError_t e = cudaSuccess;
    if (tb) e = cudaMemcpyAsync(sl.d_txns, sl.h_txns, tb, cudaMemcpyHostToDevice, l.h2d);
    if (!e && ob) e = cudaMemcpyAsync(sl.d_ops, sl.h_ops, ob, cudaMemcpyHostToDevice, l.h2d);
    if (!e && pb) e = cudaMemcpyAsync(sl.d_opd, sl.h_opd, pb, cudaMemcpyHostToDevice, l.h2d);
    if (!e) e = cudaEventRecord(sl.ev_in, l.h2d);
    if (!e) e = cudaStreamWaitEvent(l.exec, sl.ev_in, 0);
    if (e) return fail(GCC_ERR_CUDA, "server upload: %s", cudaGetErrorString(e));
    gcc_status st = gcc_execute(l.cfg.db, (gcc_scheme)l.cfg.scheme, sl.d_txns, sl.n_txns, sl.d_ops,
                                sl.d_opd, sl.n_ops, &s->params, sl.d_res, sl.d_reads, l.exec);
    if (st) return st;
    // the batch state is per database: read it before the lane's next batch resets it
    e = cudaMemcpyAsync(sl.h_state, l.cfg.db->st, sizeof(gcc::BatchState), cudaMemcpyDeviceToHost,
                        l.exec);
    if (!e) e = cudaEventRecord(sl.ev_exec, l.exec);
    if (!e) e = cudaStreamWaitEvent(l.d2h, sl.ev_exec, 0);
    if (!e && sl.n_txns)
        e = cudaMemcpyAsync(sl.h_res, sl.d_res, (uint64_t)sl.n_txns * sizeof(gcc_txn_result),
                            cudaMemcpyDeviceToHost, l.d2h);
    if (!e && sl.n_ops) e = cudaMemcpyAsync(sl.h_reads, sl.d_reads, pb, cudaMemcpyDeviceToHost, l.d2h);
    if (!e) e = cudaEventRecord(sl.ev_out, l.d2h);
    if (e) return fail(GCC_ERR_CUDA, "server download: %s", cudaGetErrorString(e));
    // into the ring only once its last event is recorded: the completer
    // queries that event, and an event never recorded reads as complete
    const uint32_t t = __atomic_load_n(&l.tail, __ATOMIC_RELAXED);
    l.ring[t % 8] = (int)(&sl - l.slots.data());
    __atomic_store_n(&l.tail, t + 1, __ATOMIC_RELEASE);
    return GCC_OK;
}

bool ring_empty(const Lane& l) {
    return __atomic_load_n(&l.head, __ATOMIC_ACQUIRE) == __atomic_load_n(&l.tail, __ATOMIC_ACQUIRE);
}

int take_free(Lane& l) {
    for (size_t i = 0; i < l.slots.size(); ++i)
        if (state_of(l.slots[i]) == FREE) {
            Slot& sl = l.slots[i];
            set_state(sl, FORMING);
            sl.n_txns = 0;
            sl.n_ops = 0;
            sl.write_bytes = 0;
            sl.req.clear();
            sl.arrival.clear();
            return (int)i;
        }
    return -1;
}

// A request fits an empty batch of the lane: no more ops than a transaction
// of the database may have, nor than a batch holds (max_batch_ops may be the
// smaller).  Admission relies on it: every request fits a fresh slot.
bool op_count_fits(const Lane& l, uint32_t nops) {
    return nops <= l.cfg.db->d.max_ops_per_txn && nops <= l.ops_cap;
}

// Append to the forming slot; false when it must launch first.
bool fits(const Lane& l, const Slot& sl, uint32_t nops, uint64_t wbytes) {
    return sl.n_txns < l.cfg.max_batch_txns && sl.n_ops + nops <= l.ops_cap &&
           (sl.n_txns == 0 || sl.write_bytes + wbytes <= l.cfg.write_budget_bytes);
}

void append(Slot& sl, const gcc_txn& t, const gcc_op* ops, const gcc_operand* opd, uint64_t wbytes,
            uint64_t arrival, uint64_t id) {
    gcc_txn x = t;
    x.first_op = (uint32_t)sl.n_ops;
    sl.h_txns[sl.n_txns++] = x;
    std::memcpy(sl.h_ops + sl.n_ops, ops, sizeof(gcc_op) * t.n_ops);
    std::memcpy(sl.h_opd + sl.n_ops, opd, sizeof(gcc_operand) * t.n_ops);
    sl.n_ops += t.n_ops;
    sl.write_bytes += wbytes;
    if (sl.req.empty()) sl.oldest = arrival;
    sl.req.push_back(id);
    sl.arrival.push_back(arrival);
}

void park(Lane& l, const gcc_txn& t, const gcc_op* ops, const gcc_operand* opd,
          uint64_t arrival, uint64_t id, bool borrowed) {
    Pending p{t, ops, opd, {}, {}, arrival, id};
    if (!borrowed) {
        p.own_ops.assign(ops, ops + t.n_ops);
        p.own_opd.assign(opd, opd + t.n_ops);
        p.ops = nullptr;                           // resolved to the copies when used
        p.opd = nullptr;
    }
    l.backlog.push_back(std::move(p));
}

const gcc_op* ops_of(const Pending& p) { return p.ops ? p.ops : p.own_ops.data(); }
const gcc_operand* opd_of(const Pending& p) { return p.opd ? p.opd : p.own_opd.data(); }

// Admit one request; launches the forming batch when it is full.  `borrowed`:
// ops and opd stay valid until the request is appended to a batch.
gcc_status admit(gcc_server* s, uint32_t li, const gcc_txn& t, const gcc_op* ops,
                 const gcc_operand* opd, uint64_t arrival, uint64_t id, bool borrowed) {
    Lane& l = s->lanes[li];
    if (!l.backlog.empty()) {                      // keep arrival order behind the backlog
        park(l, t, ops, opd, arrival, id, borrowed);
        return GCC_OK;
    }
    uint64_t wbytes = 0;
    for (uint32_t j = 0; j < t.n_ops; ++j) wbytes += writes(ops[j].kind) ? 16 : 0;
    if (l.forming >= 0 && !fits(l, l.slots[l.forming], t.n_ops, wbytes)) {
        gcc_status st = launch(s, l);
        if (st) return st;
    }
    if (l.forming < 0) l.forming = take_free(l);
    if (l.forming < 0) {                           // every slot in flight: wait in the backlog
        park(l, t, ops, opd, arrival, id, borrowed);
        return GCC_OK;
    }
    append(l.slots[l.forming], t, ops, opd, wbytes, arrival, id);
    return GCC_OK;
}

void emit(gcc_server* s, uint32_t li, Slot& sl, uint64_t t_done) {
    for (uint32_t i = 0; i < sl.n_txns; ++i) {
        gcc_completion c{};
        c.request = sl.req[i];
        c.lane = li;
        c.status = sl.h_res[i].status;
        c.batch_seq = sl.seq;
        c.commit_order = sl.h_res[i].commit_order;
        c.arrival_ns = sl.arrival[i];
        c.done_ns = t_done;
        const gcc_operand* r = sl.h_reads + sl.h_txns[i].first_op;
        if (s->trace_out) {
            s->trace_out[c.request] = c;
            if (s->trace_reads)
                std::memcpy(s->trace_reads + s->trace_txns[c.request].first_op, r,
                            sizeof(gcc_operand) * sl.h_txns[i].n_ops);
        } else {
            s->done.push_back(c);
            s->done_reads.emplace_back(r, r + sl.h_txns[i].n_ops);
        }
    }
    if (s->trace_out) __atomic_fetch_add(&s->lanes[li].trace_done, (uint64_t)sl.n_txns, __ATOMIC_RELEASE);
}

// Finished batches of one lane, in launch order: their completions are
// emitted and their slots freed (the lane's completer).
gcc_status lane_collect(gcc_server* s, uint32_t li) {
    Lane& l = s->lanes[li];
    while (!ring_empty(l)) {
        const uint32_t h = __atomic_load_n(&l.head, __ATOMIC_RELAXED);
        Slot& sl = l.slots[l.ring[h % 8]];
        const cudaError_t q = cudaEventQuery(sl.ev_out);
        if (q == cudaErrorNotReady) break;
        if (q != cudaSuccess) return fail(GCC_ERR_CUDA, "batch failed: %s", cudaGetErrorString(q));
        emit(s, li, sl, now_ns());
        l.committed += sl.h_state->committed;
        l.aborts += sl.h_state->aborts;
        l.batches++;
        set_state(sl, FREE);
        __atomic_store_n(&l.head, h + 1, __ATOMIC_RELEASE);
    }
    return GCC_OK;
}

// Backlog into free slots and a due launch of one lane (the lane's feeder).
gcc_status lane_feed(gcc_server* s, uint32_t li, bool flush_all, uint64_t t) {
    Lane& l = s->lanes[li];
    while (!l.backlog.empty()) {
        if (l.forming < 0) l.forming = take_free(l);
        if (l.forming < 0) break;
        Pending& p = l.backlog.front();
        const gcc_op* pops = ops_of(p);
        uint64_t wbytes = 0;
        for (uint32_t j = 0; j < p.txn.n_ops; ++j) wbytes += writes(pops[j].kind) ? 16 : 0;
        if (!fits(l, l.slots[l.forming], p.txn.n_ops, wbytes)) {
            gcc_status st = launch(s, l);
            if (st) return st;
            continue;
        }
        append(l.slots[l.forming], p.txn, pops, opd_of(p), wbytes, p.arrival, p.id);
        l.backlog.pop_front();
    }
    // a forming batch launches past its delay, at once when none of the
    // lane's batches is in flight (waiting gains nothing while the lane's GPU
    // work is idle), and always when draining
    if (l.forming >= 0) {
        Slot& sl = l.slots[l.forming];
        if (sl.n_txns && (flush_all || t - sl.oldest >= l.cfg.max_delay_ns || ring_empty(l))) {
            gcc_status st = launch(s, l);
            if (st) return st;
        }
    }
    return GCC_OK;
}

// Completions, backlog and a due launch of one lane, on one thread.
gcc_status pump_lane(gcc_server* s, uint32_t li, bool flush_all, uint64_t t) {
    gcc_status st = lane_collect(s, li);
    if (!st) st = lane_feed(s, li, flush_all, t);
    return st;
}

gcc_status pump(gcc_server* s, bool flush_all) {
    const uint64_t t = now_ns();
    for (uint32_t li = 0; li < s->lanes.size(); ++li) {
        const gcc_status st = pump_lane(s, li, flush_all, t);
        if (st) return st;
    }
    return GCC_OK;
}

bool idle(const gcc_server* s) {
    for (const Lane& l : s->lanes)
        if (!ring_empty(l) || !l.backlog.empty() ||
            (l.forming >= 0 && l.slots[l.forming].n_txns))
            return false;
    return true;
}

}  // namespace

extern "C" {

uint64_t gcc_server_now_ns(void) { return now_ns(); }

gcc_status gcc_server_create(const gcc_server_lane* lanes, uint32_t n, const gcc_exec_params* params,
                             gcc_server** out) {
    if (!lanes || !out || n == 0) return fail(GCC_ERR_INVALID, "null argument or no lanes");
    *out = nullptr;
    const int dev = lanes[0].db ? lanes[0].db->d.device : 0;
    for (uint32_t i = 0; i < n; ++i) {
        const gcc_server_lane& c = lanes[i];
        if (!c.db || c.db->d.device != dev) return fail(GCC_ERR_INVALID, "lane %u: bad database", i);
        for (uint32_t j = 0; j < i; ++j)
            if (lanes[j].db == c.db) return fail(GCC_ERR_INVALID, "lane %u: database used twice", i);
        if (c.scheme > GCC_MVCC)
            return fail(GCC_ERR_INVALID, "lane %u: unknown scheme", i);
        if (c.max_batch_txns == 0 || c.max_batch_txns > c.db->d.max_batch_txns)
            return fail(GCC_ERR_INVALID, "lane %u: max_batch_txns out of range", i);
        if (c.depth > 8) return fail(GCC_ERR_INVALID, "lane %u: depth must be at most 8", i);
    }
    gcc_exec_params p = merged(params);
    gcc_status st = validate_params(p);
    if (st) return st;
    if (cudaSetDevice(dev) != cudaSuccess) return fail(GCC_ERR_CUDA, "cannot select device");
    gcc_server* s = new (std::nothrow) gcc_server();
    if (!s) return fail(GCC_ERR_NOMEM, "host allocation failed");
    s->device = dev;
    s->params = p;
    s->lanes.resize(n);
    for (uint32_t i = 0; i < n; ++i) {
        Lane& l = s->lanes[i];
        l.cfg = lanes[i];
        if (!l.cfg.write_budget_bytes) l.cfg.write_budget_bytes = 256ull * l.cfg.max_batch_txns;
        if (!l.cfg.max_delay_ns) l.cfg.max_delay_ns = 200000;
        if (!l.cfg.depth) l.cfg.depth = 3;
        l.ops_cap = std::min<uint64_t>((uint64_t)l.cfg.max_batch_txns * l.cfg.db->d.max_ops_per_txn,
                                       l.cfg.db->d.max_batch_ops);
        bool ok = cudaStreamCreateWithFlags(&l.h2d, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&l.exec, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&l.d2h, cudaStreamNonBlocking) == cudaSuccess;
        l.slots.resize(l.cfg.depth);
        const uint64_t T = l.cfg.max_batch_txns, O = l.ops_cap;
        for (Slot& sl : l.slots) {
            ok = ok && cudaMallocHost(&sl.h_txns, T * sizeof(gcc_txn)) == cudaSuccess &&
                 cudaMallocHost(&sl.h_ops, O * sizeof(gcc_op)) == cudaSuccess &&
                 cudaMallocHost(&sl.h_opd, O * sizeof(gcc_operand)) == cudaSuccess &&
                 cudaMallocHost(&sl.h_res, T * sizeof(gcc_txn_result)) == cudaSuccess &&
                 cudaMallocHost(&sl.h_reads, O * sizeof(gcc_operand)) == cudaSuccess &&
                 cudaMallocHost(&sl.h_state, sizeof(gcc::BatchState)) == cudaSuccess &&
                 cudaMalloc(&sl.d_txns, T * sizeof(gcc_txn)) == cudaSuccess &&
                 cudaMalloc(&sl.d_ops, O * sizeof(gcc_op)) == cudaSuccess &&
                 cudaMalloc(&sl.d_opd, O * sizeof(gcc_operand)) == cudaSuccess &&
                 cudaMalloc(&sl.d_res, T * sizeof(gcc_txn_result)) == cudaSuccess &&
                 cudaMalloc(&sl.d_reads, O * sizeof(gcc_operand)) == cudaSuccess &&
                 cudaEventCreateWithFlags(&sl.ev_in, cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&sl.ev_exec, cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&sl.ev_out, cudaEventDisableTiming) == cudaSuccess;
            sl.req.reserve(T);
            sl.arrival.reserve(T);
        }
        if (!ok) {
            free_server(s);
            return fail(GCC_ERR_NOMEM, "cannot allocate lane %u buffers", i);
        }
    }
    *out = s;
    return GCC_OK;
}

gcc_status gcc_server_enqueue(gcc_server* s, uint32_t lane, const gcc_txn* txn, const gcc_op* ops,
                              const gcc_operand* operands, uint64_t arrival_ns, uint64_t* id) {
    if (!s || !txn || (txn->n_ops && (!ops || !operands)) || lane >= s->lanes.size())
        return fail(GCC_ERR_INVALID, "bad argument");
    if (!op_count_fits(s->lanes[lane], txn->n_ops))
        return fail(GCC_ERR_CAPACITY, "transaction has more ops than the lane's batches hold");
    if (cudaSetDevice(s->device) != cudaSuccess) return fail(GCC_ERR_CUDA, "cannot select device");
    const uint64_t rid = s->next_id++;
    if (id) *id = rid;
    return admit(s, lane, *txn, ops, operands, arrival_ns, rid, false);
}

gcc_status gcc_server_pump(gcc_server* s) {
    if (!s) return fail(GCC_ERR_INVALID, "null server");
    if (cudaSetDevice(s->device) != cudaSuccess) return fail(GCC_ERR_CUDA, "cannot select device");
    return pump(s, false);
}

gcc_status gcc_server_drain(gcc_server* s) {
    if (!s) return fail(GCC_ERR_INVALID, "null server");
    if (cudaSetDevice(s->device) != cudaSuccess) return fail(GCC_ERR_CUDA, "cannot select device");
    while (!idle(s)) {
        gcc_status st = pump(s, true);
        if (st) return st;
        std::this_thread::yield();
    }
    return GCC_OK;
}

gcc_status gcc_server_completions(gcc_server* s, gcc_completion* out, gcc_operand* reads_out,
                                  uint64_t reads_capacity, uint32_t max, uint32_t* n_out) {
    if (!s || !n_out || (max && !out)) return fail(GCC_ERR_INVALID, "bad argument");
    uint32_t k = 0;
    uint64_t used = 0;
    while (k < max && !s->done.empty()) {
        const std::vector<gcc_operand>& r = s->done_reads.front();
        if (reads_out && used + r.size() > reads_capacity) break;
        out[k] = s->done.front();
        if (reads_out) std::memcpy(reads_out + used, r.data(), r.size() * sizeof(gcc_operand));
        used += r.size();
        s->done.pop_front();
        s->done_reads.pop_front();
        ++k;
    }
    *n_out = k;
    return GCC_OK;
}

gcc_status gcc_server_run_trace(gcc_server* s, uint32_t n, const uint32_t* lane_of,
                                const gcc_txn* txns, const gcc_op* ops,
                                const gcc_operand* operands, const uint64_t* arrival_offset_ns,
                                gcc_completion* out, gcc_operand* reads_out) {
    if (!s || (n && (!lane_of || !txns || !ops || !operands || !arrival_offset_ns || !out)))
        return fail(GCC_ERR_INVALID, "bad argument");
    if (!idle(s) || !s->done.empty()) return fail(GCC_ERR_INVALID, "server is busy");
    for (uint32_t i = 0; i < n; ++i)
        if (lane_of[i] >= s->lanes.size() || !op_count_fits(s->lanes[lane_of[i]], txns[i].n_ops))
            return fail(GCC_ERR_INVALID, "request %u: bad lane or too many ops", i);
    if (cudaSetDevice(s->device) != cudaSuccess) return fail(GCC_ERR_CUDA, "cannot select device");
    s->trace_out = out;
    s->trace_reads = reads_out;
    s->trace_txns = txns;
    const uint32_t nl = (uint32_t)s->lanes.size();
    std::vector<std::vector<uint32_t>> mine(nl);       // each lane's requests, in trace order
    for (uint32_t i = 0; i < n; ++i) mine[lane_of[i]].push_back(i);
    for (Lane& l : s->lanes) l.trace_done = 0;
    // two threads per lane: the feeder admits arrivals, forms and launches
    // batches; the completer collects finished batches and frees their
    // slots.  An error on either stops both threads of its lane.
    std::vector<gcc_status> status(2 * nl, GCC_OK);
    std::vector<std::string> message(2 * nl);
    std::vector<int> stop(nl, 0);
    const uint64_t t0 = now_ns();
    auto stopped = [&](uint32_t li) { return __atomic_load_n(&stop[li], __ATOMIC_ACQUIRE) != 0; };
    auto halt = [&](uint32_t li, uint32_t w, gcc_status st) {
        status[w] = st;
        message[w] = gcc_last_error();
        __atomic_store_n(&stop[li], 1, __ATOMIC_RELEASE);
    };
    auto feeder = [&](uint32_t li) {
        if (cudaSetDevice(s->device) != cudaSuccess) {
            halt(li, 2 * li, fail(GCC_ERR_CUDA, "cannot select device"));
            return;
        }
        const std::vector<uint32_t>& idx = mine[li];
        const Lane& l = s->lanes[li];
        size_t next = 0;
        gcc_status st = GCC_OK;
        while (!st && !stopped(li)) {
            const uint64_t now = now_ns() - t0;
            while (!st && next < idx.size() && arrival_offset_ns[idx[next]] <= now) {
                // the trace's arrays outlive the run: a parked request points into them
                const uint32_t i = idx[next];
                st = admit(s, li, txns[i], ops + txns[i].first_op, operands + txns[i].first_op,
                           t0 + arrival_offset_ns[i], i, true);
                ++next;
            }
            if (!st) st = lane_feed(s, li, next == idx.size(), now_ns());
            if (next == idx.size() && l.backlog.empty() &&
                (l.forming < 0 || l.slots[l.forming].n_txns == 0))
                break;                                   // everything launched
        }
        if (st) halt(li, 2 * li, st);
    };
    auto completer = [&](uint32_t li) {
        if (cudaSetDevice(s->device) != cudaSuccess) {
            halt(li, 2 * li + 1, fail(GCC_ERR_CUDA, "cannot select device"));
            return;
        }
        const Lane& l = s->lanes[li];
        const uint64_t want = mine[li].size();
        while (!stopped(li) && __atomic_load_n(&l.trace_done, __ATOMIC_ACQUIRE) < want) {
            const gcc_status st = lane_collect(s, li);
            if (st) { halt(li, 2 * li + 1, st); return; }
        }
    };
    {
        std::vector<std::thread> workers;
        workers.reserve(2 * nl);
        for (uint32_t li = 0; li < nl; ++li) {
            workers.emplace_back(feeder, li);
            workers.emplace_back(completer, li);
        }
        for (std::thread& w : workers) w.join();
    }
    gcc_status st = GCC_OK;
    for (uint32_t w = 0; w < 2 * nl && !st; ++w)
        if (status[w]) st = fail(status[w], "lane %u: %s", w / 2, message[w].c_str());
    s->trace_out = nullptr;
    s->trace_reads = nullptr;
    s->trace_txns = nullptr;
    return st;
}

gcc_status gcc_server_lane_totals(gcc_server* s, uint32_t lane, uint64_t* committed,
                                  uint64_t* aborts, uint64_t* batches) {
    if (!s || lane >= s->lanes.size()) return fail(GCC_ERR_INVALID, "bad server or lane");
    const Lane& l = s->lanes[lane];
    if (committed) *committed = l.committed;
    if (aborts) *aborts = l.aborts;
    if (batches) *batches = l.batches;
    return GCC_OK;
}

gcc_status gcc_server_destroy(gcc_server* s) {
    if (!s) return GCC_OK;
    gcc_server_drain(s);
    free_server(s);
    return GCC_OK;
}

}  // extern "C"
