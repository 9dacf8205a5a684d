// Serving loop for randomized PCA requests (include/rsvd.h, rsvd_server_*):
// continuous batching with HBM admission.
//
// One device arena (cudaMalloc'd once) holds the plan workspaces of admitted
// requests; the first-fit Arena tracks it.  Requests wait in arrival order.
// Every poll first retires batches whose completion event has fired (their
// workspaces return to the arena), then admits from the head of the queue:
// a batch takes the oldest waiting request and the requests queued directly
// behind it that share its l, q and storage type, while their workspaces fit
// and the batch is not full.  The head is never skipped (no starvation of large requests).
// Each batch runs on a slot of its own (a batch stream, one stream per problem,
// pinned result words, a completion event), so batches admitted while others
// run overlap on the device.
#include <cuda_runtime.h>

#include <chrono>
#include <deque>
#include <new>
#include <vector>

#include "arena.h"
#include "common.cuh"

namespace {

using Clock = std::chrono::steady_clock;

struct Request {
    int64_t id, m, n;
    int k, p, q;
    rsvd_dtype dtype;
    double t;
    const void *A;
    const float *sc, *Om;
    double *S;
    float *U, *V;
    size_t ws;
    double submit_ms;
};

struct Slot {
    cudaStream_t bs = nullptr;
    std::vector<cudaStream_t> ps;
    gbr::ServeBatch *sb = nullptr;
    int *host_out = nullptr;  // pinned, 3 ints per problem
    cudaEvent_t done = nullptr;
    bool busy = false;
};

struct Running {
    int slot;
    std::vector<Request> reqs;
    std::vector<rsvd_plan_t> plans;
    std::vector<size_t> offs;
    double start_ms;
};

}  // namespace

struct rsvd_server {
    char *base = nullptr;
    gbr::Arena arena;
    int max_batch = 1;
    std::vector<Slot> slots;
    std::deque<Request> queue;
    std::vector<Running> running;
    std::deque<rsvd_completion> ready;
    cudaEvent_t ref = nullptr;
    Clock::time_point t0;
    double ref_ms = 0.0;

    double now_ms() const { return std::chrono::duration<double, std::milli>(Clock::now() - t0).count(); }
};

namespace {

void free_slot(Slot &s) {
    if (s.done) cudaEventDestroy(s.done);
    if (s.host_out) cudaFreeHost(s.host_out);
    if (s.sb) gbr::serve_batch_free(s.sb);
    for (cudaStream_t x : s.ps)
        if (x) cudaStreamDestroy(x);
    if (s.bs) cudaStreamDestroy(s.bs);
    s = Slot();
}

// Retire one finished batch: completions to `ready`, workspaces back to the arena.
void retire(rsvd_server *S, size_t r) {
    Running &run = S->running[r];
    Slot &slot = S->slots[run.slot];
    float dev_ms = 0.f;
    cudaEventElapsedTime(&dev_ms, S->ref, slot.done);
    const double done_ms = S->ref_ms + dev_ms;
    const int count = (int)run.reqs.size();
    for (int i = 0; i < count; i++) {
        rsvd_completion c;
        c.id = run.reqs[i].id;
        c.status = gbr::serve_status(slot.host_out[3 * i], slot.host_out[3 * i + 2]);
        c.K = slot.host_out[3 * i + 1];
        c.batch = count;
        c.submit_ms = run.reqs[i].submit_ms;
        c.start_ms = run.start_ms;
        c.done_ms = done_ms;
        S->ready.push_back(c);
        rsvd_plan_destroy(run.plans[i]);
        S->arena.release(run.offs[i], run.reqs[i].ws);
    }
    slot.busy = false;
    S->running.erase(S->running.begin() + (long)r);
}

int free_slot_index(rsvd_server *S) {
    for (size_t i = 0; i < S->slots.size(); i++)
        if (!S->slots[i].busy) return (int)i;
    return -1;
}

// Admit and launch one batch from the head of the queue; false when nothing can start.
bool admit_one(rsvd_server *S, rsvd_status *err) {
    *err = RSVD_OK;
    if (S->queue.empty()) return false;
    const int si = free_slot_index(S);
    if (si < 0) return false;
    Slot &slot = S->slots[si];
    Running run;
    run.slot = si;
    const Request &head = S->queue.front();
    const int l = head.k + head.p, q = head.q;
    const rsvd_dtype dt = head.dtype;
    while (!S->queue.empty() && (int)run.reqs.size() < S->max_batch) {
        const Request &rq = S->queue.front();
        if (rq.k + rq.p != l || rq.q != q || rq.dtype != dt) break;
        size_t off = 0;
        if (!S->arena.alloc(rq.ws, &off)) break;
        run.reqs.push_back(rq);
        run.offs.push_back(off);
        S->queue.pop_front();
    }
    if (run.reqs.empty()) return false;
    const int count = (int)run.reqs.size();
    std::vector<const void *> A(count);
    std::vector<const float *> Om(count), Sc(count);
    std::vector<double *> Sg(count);
    std::vector<float *> U(count), V(count);
    std::vector<double> t(count);
    for (int i = 0; i < count; i++) {
        const Request &rq = run.reqs[i];
        rsvd_plan_t P = nullptr;
        rsvd_status st = rsvd_plan_create_in(&P, rq.m, rq.n, rq.k, rq.p, rq.q, rq.dtype, slot.ps[i],
                                             S->base + run.offs[i], rq.ws);
        if (st != RSVD_OK) {  // the whole batch fails with this status (nothing was launched)
            const double now = S->now_ms();
            for (rsvd_plan_t x : run.plans) rsvd_plan_destroy(x);
            for (int j = 0; j < count; j++) {
                S->arena.release(run.offs[j], run.reqs[j].ws);
                S->ready.push_back(rsvd_completion{run.reqs[j].id, st, 0, count, run.reqs[j].submit_ms, now, now});
            }
            return true;
        }
        run.plans.push_back(P);
        A[i] = rq.A;
        Sc[i] = rq.sc;
        Om[i] = rq.Om;
        Sg[i] = rq.S;
        U[i] = rq.U;
        V[i] = rq.V;
        t[i] = rq.t;
    }
    run.start_ms = S->now_ms();
    rsvd_status st = gbr::serve_batch_launch(slot.sb, count, run.plans.data(), A.data(), Sc.data(), Om.data(),
                                             Sg.data(), U.data(), V.data(), t.data(), slot.host_out);
    if (st == RSVD_OK && cudaEventRecord(slot.done, slot.bs) != cudaSuccess) st = RSVD_ERR_CUDA;
    if (st != RSVD_OK) {
        *err = st;
        return false;
    }
    slot.busy = true;
    S->running.push_back(std::move(run));
    return true;
}

}  // namespace

extern "C" {

rsvd_status rsvd_server_create(rsvd_server_t *server, size_t hbm_bytes, int max_batch, int max_inflight) {
    if (!server) return RSVD_ERR_ARG;
    *server = nullptr;
    if (hbm_bytes < gbr::Arena::kAlign || max_batch < 1 || max_batch > RSVD_BATCH_MAX || max_inflight < 1 ||
        max_inflight > 64)
        return RSVD_ERR_ARG;
    rsvd_server *S = new (std::nothrow) rsvd_server();
    if (!S) return RSVD_ERR_OOM;
    S->max_batch = max_batch;
    S->arena.init(hbm_bytes);
    bool ok = cudaMalloc(&S->base, S->arena.size()) == cudaSuccess;
    S->slots.resize(max_inflight);
    for (int i = 0; ok && i < max_inflight; i++) {
        Slot &s = S->slots[i];
        ok = cudaStreamCreateWithFlags(&s.bs, cudaStreamNonBlocking) == cudaSuccess;
        s.ps.assign(max_batch, nullptr);
        for (int j = 0; ok && j < max_batch; j++)
            ok = cudaStreamCreateWithFlags(&s.ps[j], cudaStreamNonBlocking) == cudaSuccess;
        ok = ok && (s.sb = gbr::serve_batch_new(s.bs, max_batch)) != nullptr;
        ok = ok && cudaMallocHost(&s.host_out, sizeof(int) * 3 * (size_t)max_batch) == cudaSuccess;
        ok = ok && cudaEventCreate(&s.done) == cudaSuccess;
    }
    ok = ok && cudaEventCreate(&S->ref) == cudaSuccess;
    if (ok) {  // anchor device event times to the host clock
        S->t0 = Clock::now();
        ok = cudaEventRecord(S->ref, S->slots[0].bs) == cudaSuccess && cudaEventSynchronize(S->ref) == cudaSuccess;
        S->ref_ms = S->now_ms();
    }
    if (!ok) {
        cudaGetLastError();
        rsvd_server_destroy(S);
        return RSVD_ERR_OOM;
    }
    *server = S;
    return RSVD_OK;
}

rsvd_status rsvd_server_submit_ex(rsvd_server_t S, int64_t id, int64_t m, int64_t n, int k, int p, int q,
                                  rsvd_dtype dtype, double t, const void *A, const float *col_scales,
                                  const float *Omega, double *Sg, float *U, float *V) {
    if (!S || !A || !Omega || !Sg || !U || !V || !(t > 0.0) || t > 1.0) return RSVD_ERR_ARG;
    if (dtype == RSVD_F64) return RSVD_ERR_UNSUPPORTED;                   // float32 outputs only
    if ((col_scales != nullptr) != (dtype == RSVD_FP8_E4M3)) return RSVD_ERR_ARG;
    size_t ws = 0;
    const rsvd_status st = rsvd_workspace_query(m, n, k, p, q, dtype, &ws);
    if (st != RSVD_OK) return st;
    if (gbr::Arena::round(ws) > S->arena.size()) return RSVD_ERR_OOM;
    S->queue.push_back(Request{id, m, n, k, p, q, dtype, t, A, col_scales, Omega, Sg, U, V, ws, S->now_ms()});
    return RSVD_OK;
}

rsvd_status rsvd_server_submit(rsvd_server_t S, int64_t id, int64_t m, int64_t n, int k, int p, int q, double t,
                               const float *A, const float *Omega, double *Sg, float *U, float *V) {
    return rsvd_server_submit_ex(S, id, m, n, k, p, q, RSVD_F32, t, A, nullptr, Omega, Sg, U, V);
}

int rsvd_server_poll(rsvd_server_t S, rsvd_completion *out, int max_out) {
    if (!S || (max_out > 0 && !out)) return RSVD_ERR_ARG;
    for (size_t r = 0; r < S->running.size();) {
        const cudaError_t e = cudaEventQuery(S->slots[S->running[r].slot].done);
        if (e == cudaSuccess) {
            retire(S, r);
        } else if (e == cudaErrorNotReady) {
            r++;
        } else {
            cudaGetLastError();
            return RSVD_ERR_CUDA;
        }
    }
    rsvd_status err = RSVD_OK;
    while (admit_one(S, &err)) {
    }
    if (err != RSVD_OK) return err;
    int w = 0;
    while (w < max_out && !S->ready.empty()) {
        out[w++] = S->ready.front();
        S->ready.pop_front();
    }
    return w;
}

int rsvd_server_pending(rsvd_server_t S) {
    if (!S) return 0;
    size_t n = S->queue.size() + S->ready.size();
    for (const Running &r : S->running) n += r.reqs.size();
    return (int)n;
}

rsvd_status rsvd_server_destroy(rsvd_server_t S) {
    if (!S) return RSVD_OK;
    for (Slot &s : S->slots) {
        if (s.bs) cudaStreamSynchronize(s.bs);
        for (cudaStream_t x : s.ps)
            if (x) cudaStreamSynchronize(x);
    }
    for (Running &r : S->running)
        for (rsvd_plan_t p : r.plans) rsvd_plan_destroy(p);
    for (Slot &s : S->slots) free_slot(s);
    if (S->ref) cudaEventDestroy(S->ref);
    if (S->base) cudaFree(S->base);
    delete S;
    return RSVD_OK;
}

}  // extern "C"
