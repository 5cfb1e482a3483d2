// Serving runtime: continuous batching of many superiorized solves on one
// GPU (the C ABI suppy_server_* in include/suppy.h; the paper runs one solve
// at a time and has no counterpart).
//
// Every registered matrix is served by batched contexts (api.cu) whose
// right-hand sides are slots: a slot holds one request's bounds, iterate,
// exponent and stopping state on the device, and a free slot is marked
// stopped so that every kernel skips it.  A round of suppy_server_step never
// blocks on the device: a context whose last chunk of iterations finished
// (its event completed) has its stopped requests retired (x copied out) and
// its slots refilled from the queue, then gets the next chunk; contexts run
// on their own streams, so different matrices overlap on the GPU.  New
// contexts are created while the device-memory budget allows, after idle
// contexts of other matrices have been released.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <memory>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"

using namespace suppy;

namespace {

struct MatrixDef {
    int m = 0, n = 0;
    std::vector<int32_t> row_ptr, col;
    std::vector<float> val;
    std::vector<float> box_lo, box_hi;
    std::vector<int32_t> blocks;
    std::vector<float> c_lin;
    std::vector<int32_t> o_rp, o_col;      // objective rows (mean dose), when given
    std::vector<float> o_val;
    int o_m = 0;
    suppy_opts opts{};
    suppy_params params{};
    size_t bytes = 0;                      // measured device bytes of one context (0: unknown)
    int64_t nnz() const { return (int64_t)col.size(); }
};

struct Request {
    int64_t id = 0;
    int matrix = 0;
    std::vector<float> l, u;
    std::vector<float> x;
    int state = 0;                         // 0 waiting, 1 running, 2 done
    int engine = -1, slot = -1;
    RhsState st{};
    double t_submit = 0, t_start = 0, t_done = 0;
};

struct Engine {
    int matrix = 0;
    suppy_ctx* ctx = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    RhsState* h_st = nullptr;              // pinned
    float* d_x = nullptr;                  // one column
    float* h_x = nullptr;                  // pinned, one column
    std::vector<int64_t> slot_req;         // request index per slot, -1 free
    int running = 0;
    bool inflight = false;
    double last_used = 0;
    size_t bytes = 0;
};

}  // namespace

struct suppy_server {
    suppy_server_opts o{};
    std::chrono::steady_clock::time_point t0;
    std::vector<MatrixDef> mats;
    std::vector<Request> reqs;
    std::deque<int64_t> queue;             // waiting request indices, arrival order
    std::vector<std::unique_ptr<Engine>> engines;
    size_t used = 0;
    std::string err;
};

namespace {

double now_s(const suppy_server* s) {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - s->t0).count();
}

suppy_status sfail(suppy_server* s, suppy_status st, const std::string& msg) {
    if (s) s->err = msg;
    else set_thread_error(msg);
    return st;
}

#define SCK(call)                                                                          \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            cudaGetLastError();                                                            \
            return sfail(srv, SUPPY_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
        }                                                                                  \
    } while (0)

// Device bytes a new context of this matrix is expected to hold: the measured
// figure of an earlier context, else an upper estimate (two copies of A,
// per-row and per-column vectors of every slot, some slack).
size_t expected_bytes(const MatrixDef& d, int slots) {
    if (d.bytes) return d.bytes;
    const size_t vsz = d.opts.a_dtype == SUPPY_F32 ? 4 : 2;
    const size_t B = slots > 1 ? std::max(4, 1 << (32 - __builtin_clz((unsigned)(slots - 1)))) : 1;
    const size_t nnz_pad = (size_t)d.nnz() + 3 * (size_t)d.m + 3 * (size_t)d.n + 8192;
    return 2 * nnz_pad * (vsz + 4) + (size_t)d.m * (24 + 16 * B) + (size_t)d.n * (16 + 20 * B) +
           (size_t)4096 * 16 * B + ((size_t)1 << 20);
}

void release_engine(suppy_server* srv, size_t i) {
    Engine& e = *srv->engines[i];
    if (e.ctx) suppy_destroy(e.ctx);
    if (e.ev) cudaEventDestroy(e.ev);
    if (e.stream) cudaStreamDestroy(e.stream);
    if (e.h_st) cudaFreeHost(e.h_st);
    if (e.h_x) cudaFreeHost(e.h_x);
    if (e.d_x) cudaFree(e.d_x);
    srv->used -= std::min(srv->used, e.bytes);
    srv->engines.erase(srv->engines.begin() + (long)i);
    // keep the requests' engine indices valid
    for (auto& r : srv->reqs)
        if (r.state == 1 && r.engine > (int)i) r.engine -= 1;
}

// A new context for matrix mi, if the budget allows one (idle contexts of
// other matrices are released, least recently used first, to make room).  A
// server that holds nothing creates the context whatever the estimate says,
// so that no request waits forever; the budget caps concurrency.
suppy_status new_engine(suppy_server* srv, int mi, int* out) {
    *out = -1;
    MatrixDef& d = srv->mats[mi];
    const int slots = srv->o.slots;
    const size_t need = expected_bytes(d, slots) + (size_t)d.n * 4;
    while (srv->used > 0 && srv->used + need > (size_t)srv->o.hbm_budget) {
        int victim = -1;
        for (size_t i = 0; i < srv->engines.size(); ++i) {
            const Engine& e = *srv->engines[i];
            if (e.running == 0 && !e.inflight && e.matrix != mi &&
                (victim < 0 || e.last_used < srv->engines[victim]->last_used))
                victim = (int)i;
        }
        if (victim < 0) return SUPPY_OK;   // no room now: the request waits
        release_engine(srv, (size_t)victim);
    }
    std::unique_ptr<Engine> e(new Engine());
    e->matrix = mi;
    SCK(cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking));
    SCK(cudaEventCreateWithFlags(&e->ev, cudaEventDisableTiming));
    suppy_csr A;
    A.m = d.m;
    A.n = d.n;
    A.nnz = d.nnz();
    A.row_ptr = d.row_ptr.data();
    A.col = d.col.data();
    A.val = d.val.data();
    A.on_device = 0;
    suppy_csr S{};
    suppy_opts o = d.opts;
    o.nrhs = slots;
    o.block_of_row = d.blocks.empty() ? nullptr : d.blocks.data();
    o.c_lin = d.c_lin.empty() ? nullptr : d.c_lin.data();
    if (!d.o_rp.empty()) {
        S.m = d.o_m;
        S.n = d.n;
        S.nnz = (int64_t)d.o_col.size();
        S.row_ptr = d.o_rp.data();
        S.col = d.o_col.data();
        S.val = d.o_val.data();
        S.on_device = 0;
        o.obj_rows = &S;
    } else {
        o.obj_rows = nullptr;
    }
    // placeholder bounds (every slot is stopped until a request is loaded)
    std::vector<float> lo((size_t)d.m * slots, -INFINITY), hi((size_t)d.m * slots, INFINITY);
    suppy_status st = suppy_create(&A, lo.data(), hi.data(), d.box_lo.data(), d.box_hi.data(), &o,
                                   e->stream, &e->ctx);
    if (st != SUPPY_OK) {
        const std::string msg = suppy_last_error(nullptr);
        cudaEventDestroy(e->ev);
        cudaStreamDestroy(e->stream);
        return sfail(srv, st, "creating a context: " + msg);
    }
    ctx_set_sweep_budget(e->ctx, d.params.max_sweeps);
    for (int b = 0; b < slots; ++b)
        if ((st = ctx_slot_stop(e->ctx, b)) != SUPPY_OK) return sfail(srv, st, ctx_error(e->ctx));
    SCK(cudaMallocHost(&e->h_st, sizeof(RhsState) * slots));
    SCK(cudaMallocHost(&e->h_x, sizeof(float) * (size_t)d.n));
    SCK(cudaMalloc(&e->d_x, sizeof(float) * (size_t)d.n));
    e->slot_req.assign(slots, -1);
    e->bytes = ctx_device_bytes(e->ctx) + (size_t)d.n * 4;
    if (!d.bytes) d.bytes = ctx_device_bytes(e->ctx);
    e->last_used = now_s(srv);
    srv->used += e->bytes;
    srv->engines.push_back(std::move(e));
    *out = (int)srv->engines.size() - 1;
    return SUPPY_OK;
}

// Finished chunk of engine ei: copy the stopped requests' x out, free slots.
suppy_status retire(suppy_server* srv, int ei) {
    Engine& e = *srv->engines[ei];
    const MatrixDef& d = srv->mats[e.matrix];
    for (int b = 0; b < (int)e.slot_req.size(); ++b) {
        const int64_t ri = e.slot_req[b];
        if (ri < 0 || !e.h_st[b].stopped) continue;
        Request& r = srv->reqs[ri];
        suppy_status st = ctx_slot_extract(e.ctx, b, e.d_x);
        if (st != SUPPY_OK) return sfail(srv, st, ctx_error(e.ctx));
        SCK(cudaMemcpyAsync(e.h_x, e.d_x, sizeof(float) * d.n, cudaMemcpyDeviceToHost, e.stream));
        SCK(cudaStreamSynchronize(e.stream));
        r.x.assign(e.h_x, e.h_x + d.n);
        r.st = e.h_st[b];
        r.state = 2;
        r.t_done = now_s(srv);
        r.l.clear();
        r.l.shrink_to_fit();
        r.u.clear();
        r.u.shrink_to_fit();
        e.slot_req[b] = -1;
        e.running -= 1;
    }
    return SUPPY_OK;
}

// Place waiting requests into free slots (existing contexts first).
suppy_status admit(suppy_server* srv) {
    size_t scanned = srv->queue.size();
    while (scanned-- > 0) {
        const int64_t ri = srv->queue.front();
        srv->queue.pop_front();
        Request& r = srv->reqs[ri];
        int ei = -1, slot = -1;
        for (size_t i = 0; i < srv->engines.size() && ei < 0; ++i) {
            Engine& e = *srv->engines[i];
            if (e.matrix != r.matrix || e.inflight) continue;
            for (int b = 0; b < (int)e.slot_req.size(); ++b)
                if (e.slot_req[b] < 0) {
                    ei = (int)i;
                    slot = b;
                    break;
                }
        }
        if (ei < 0) {
            // a context of this matrix still busy with a chunk keeps the
            // request waiting for its slots rather than opening another one
            // while that one has free slots
            bool busy_with_room = false;
            for (auto& ep : srv->engines)
                if (ep->matrix == r.matrix && ep->running < (int)ep->slot_req.size())
                    busy_with_room = true;
            if (!busy_with_room) {
                suppy_status st = new_engine(srv, r.matrix, &ei);
                if (st != SUPPY_OK) return st;
                slot = 0;
            }
        }
        if (ei < 0) {
            srv->queue.push_back(ri);   // stays waiting, order kept
            continue;
        }
        Engine& e = *srv->engines[ei];
        suppy_status st = ctx_slot_load(e.ctx, slot, r.l.data(), r.u.data());
        if (st != SUPPY_OK) return sfail(srv, st, ctx_error(e.ctx));
        e.slot_req[slot] = ri;
        e.running += 1;
        r.state = 1;
        r.engine = ei;
        r.slot = slot;
        r.t_start = now_s(srv);
    }
    return SUPPY_OK;
}

}  // namespace

extern "C" {

suppy_status suppy_server_create(const suppy_server_opts* o, suppy_server** out) {
    if (!out) return sfail(nullptr, SUPPY_EINVAL, "out is NULL");
    *out = nullptr;
    suppy_server_opts so{};
    if (o) so = *o;
    if (so.slots == 0) so.slots = 32;
    if (so.check_every == 0) so.check_every = 8;
    if (so.slots < 1 || so.slots > kMaxRhs || so.check_every < 1 || so.hbm_budget < 0)
        return sfail(nullptr, SUPPY_EINVAL, "server options out of range");
    if (so.hbm_budget == 0) {
        size_t fr = 0, tot = 0;
        cudaError_t e = cudaMemGetInfo(&fr, &tot);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return sfail(nullptr, SUPPY_ECUDA, std::string("cudaMemGetInfo: ") + cudaGetErrorString(e));
        }
        so.hbm_budget = (int64_t)(0.8 * (double)fr);
    }
    suppy_server* s = new suppy_server();
    s->o = so;
    s->t0 = std::chrono::steady_clock::now();
    *out = s;
    return SUPPY_OK;
}

void suppy_server_destroy(suppy_server* srv) {
    if (!srv) return;
    while (!srv->engines.empty()) release_engine(srv, srv->engines.size() - 1);
    delete srv;
}

suppy_status suppy_server_add_matrix(suppy_server* srv, const suppy_csr* A, const float* box_lo,
                                     const float* box_hi, const suppy_opts* o,
                                     const suppy_params* p, int32_t* matrix_id) {
    if (!srv) return sfail(nullptr, SUPPY_EINVAL, "server is NULL");
    if (!A || !box_lo || !box_hi || !o || !p || !matrix_id)
        return sfail(srv, SUPPY_EINVAL, "NULL argument");
    if (A->on_device) return sfail(srv, SUPPY_EINVAL, "the server takes host arrays");
    if (A->m < 0 || A->n < 1 || A->nnz < 0 || !A->row_ptr || (A->nnz && (!A->col || !A->val)))
        return sfail(srv, SUPPY_EINVAL, "bad CSR shape or pointers");
    if (o->box_len != 1 && o->box_len != A->n) return sfail(srv, SUPPY_EINVAL, "box_len must be 1 or n");
    if (p->max_sweeps < 1) return sfail(srv, SUPPY_EINVAL, "params->max_sweeps must be >= 1");
    MatrixDef d;
    d.m = A->m;
    d.n = A->n;
    d.row_ptr.assign(A->row_ptr, A->row_ptr + A->m + 1);
    d.col.assign(A->col, A->col + A->nnz);
    d.val.assign(A->val, A->val + A->nnz);
    d.box_lo.assign(box_lo, box_lo + o->box_len);
    d.box_hi.assign(box_hi, box_hi + o->box_len);
    if (o->mode == SUPPY_BIP && o->block_of_row) d.blocks.assign(o->block_of_row, o->block_of_row + A->m);
    if (o->obj == SUPPY_OBJ_LINEAR) {
        if (o->obj_rows) {
            const suppy_csr* S = o->obj_rows;
            if (S->on_device || S->n != A->n || !S->row_ptr)
                return sfail(srv, SUPPY_EINVAL, "objective rows: host CSR with n columns");
            d.o_m = S->m;
            d.o_rp.assign(S->row_ptr, S->row_ptr + S->m + 1);
            d.o_col.assign(S->col, S->col + S->nnz);
            d.o_val.assign(S->val, S->val + S->nnz);
        } else if (o->c_lin) {
            d.c_lin.assign(o->c_lin, o->c_lin + A->n);
        }
    }
    d.opts = *o;
    d.params = *p;
    srv->mats.push_back(std::move(d));
    *matrix_id = (int32_t)srv->mats.size() - 1;
    return SUPPY_OK;
}

suppy_status suppy_server_submit(suppy_server* srv, int32_t matrix_id, const float* l,
                                 const float* u, int64_t* request_id) {
    if (!srv) return sfail(nullptr, SUPPY_EINVAL, "server is NULL");
    if (matrix_id < 0 || matrix_id >= (int)srv->mats.size())
        return sfail(srv, SUPPY_EINVAL, "unknown matrix id");
    if (!l || !u) return sfail(srv, SUPPY_EINVAL, "NULL bounds");
    const int m = srv->mats[matrix_id].m;
    Request r;
    r.id = (int64_t)srv->reqs.size();
    r.matrix = matrix_id;
    r.l.assign(l, l + m);
    r.u.assign(u, u + m);
    for (int i = 0; i < m; ++i)
        if (std::isnan(r.l[i]) || std::isnan(r.u[i]) || !(r.l[i] <= r.u[i]))
            return sfail(srv, SUPPY_EINVAL, "bounds need l <= u and no NaN");
    r.t_submit = now_s(srv);
    srv->reqs.push_back(std::move(r));
    srv->queue.push_back((int64_t)srv->reqs.size() - 1);
    if (request_id) *request_id = (int64_t)srv->reqs.size() - 1;
    return SUPPY_OK;
}

suppy_status suppy_server_step(suppy_server* srv, int32_t* running, int32_t* waiting) {
    if (!srv) return sfail(nullptr, SUPPY_EINVAL, "server is NULL");
    bool progressed = false;
    // 1. contexts whose chunk finished: retire stopped requests
    for (size_t i = 0; i < srv->engines.size(); ++i) {
        Engine& e = *srv->engines[i];
        if (!e.inflight) continue;
        const cudaError_t q = cudaEventQuery(e.ev);
        if (q == cudaErrorNotReady) continue;
        if (q != cudaSuccess) {
            cudaGetLastError();
            return sfail(srv, SUPPY_ECUDA, std::string("context chunk: ") + cudaGetErrorString(q));
        }
        e.inflight = false;
        suppy_status st = retire(srv, (int)i);
        if (st != SUPPY_OK) return st;
        progressed = true;
    }
    // 2. admissions
    const size_t before = srv->queue.size();
    suppy_status st = admit(srv);
    if (st != SUPPY_OK) return st;
    progressed = progressed || srv->queue.size() != before;
    // 3. next chunk on every idle context with running requests
    for (auto& ep : srv->engines) {
        Engine& e = *ep;
        if (e.inflight || e.running == 0) continue;
        const MatrixDef& d = srv->mats[e.matrix];
        if ((st = ctx_iterate(e.ctx, &d.params, srv->o.check_every)) != SUPPY_OK)
            return sfail(srv, st, ctx_error(e.ctx));
        if ((st = ctx_states_async(e.ctx, e.h_st)) != SUPPY_OK) return sfail(srv, st, ctx_error(e.ctx));
        SCK(cudaEventRecord(e.ev, e.stream));
        e.inflight = true;
        e.last_used = now_s(srv);
        progressed = true;
    }
    if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(20));
    int run = 0;
    for (auto& ep : srv->engines) run += ep->running;
    if (running) *running = run;
    if (waiting) *waiting = (int32_t)srv->queue.size();
    return SUPPY_OK;
}

suppy_status suppy_server_query(suppy_server* srv, int64_t request_id, suppy_request_info* info,
                                float* x) {
    if (!srv) return sfail(nullptr, SUPPY_EINVAL, "server is NULL");
    if (request_id < 0 || request_id >= (int64_t)srv->reqs.size())
        return sfail(srv, SUPPY_EINVAL, "unknown request id");
    const Request& r = srv->reqs[request_id];
    if (info) {
        info->state = r.state;
        info->sweeps = r.st.k;
        info->accepted = r.st.accepted_total;
        info->trials = r.st.trials_total;
        info->proximity = r.st.last_prox;
        info->objective = r.st.f_prev;
        info->t_submit = r.t_submit;
        info->t_start = r.t_start;
        info->t_done = r.t_done;
    }
    if (x && r.state == 2) std::memcpy(x, r.x.data(), sizeof(float) * r.x.size());
    return SUPPY_OK;
}

double suppy_server_clock(const suppy_server* srv) { return srv ? now_s(srv) : 0.0; }

int64_t suppy_server_device_bytes(const suppy_server* srv) { return srv ? (int64_t)srv->used : 0; }

const char* suppy_server_last_error(const suppy_server* srv) {
    return srv ? srv->err.c_str() : "";
}

}  // extern "C"
