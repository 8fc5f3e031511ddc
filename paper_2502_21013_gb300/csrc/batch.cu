// Batched solve of many independent instances (uneven mesh sizes and N).
//
// Each instance is a set-up context with its own stream and buffers.  One
// outer fixed-point step of every instance is captured into a single CUDA
// graph as parallel branches forked from, and joined back into, the batch
// stream, so one graph launch advances all instances by one step and their
// kernels run concurrently (small instances fill the SMs that a large one
// leaves idle).  An instance that has met its stopping rule keeps launching
// inside the graph but every kernel of it returns at once (its device flag),
// so its iterate is the one that converged.  The host reads all statuses
// every check_every steps and stops when every instance is done.
#include <chrono>
#include <cstring>
#include <vector>

#include "common.h"

namespace ptp {
Ctx* ctx_of(ptp_ctx* h);
}

struct ptp_batch {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::vector<ptp_ctx*> items;
    cudaGraphExec_t exec = nullptr;
    std::vector<int64_t> keys;  // step keys of the captured graph
    std::vector<int64_t> per_step;
    std::vector<cudaEvent_t> events;
    std::string err;
};

namespace {

void drop_graph(ptp_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    b->keys.clear();
}

template <typename F>
int batch_guard(ptp_batch* b, F&& f) {
    if (!b) return PTP_EINVAL;
    try {
        b->err.clear();
        PTP_CUDA(cudaSetDevice(b->device));
        return f();
    } catch (const ptp::Error& e) {
        b->err = e.what();
        return e.code;
    } catch (const std::exception& e) {
        b->err = e.what();
        return PTP_EINVAL;
    }
}

}  // namespace

extern "C" {

int ptp_batch_create(ptp_batch** out, int device) {
    if (!out || device < 0) return PTP_EINVAL;
    *out = nullptr;
    ptp_batch* b = new (std::nothrow) ptp_batch();
    if (!b) return PTP_ENOMEM;
    b->device = device;
    int rc = batch_guard(b, [&]() {
        PTP_CUDA(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
        return PTP_OK;
    });
    if (rc != PTP_OK) {
        delete b;
        return rc;
    }
    *out = b;
    return PTP_OK;
}

void ptp_batch_destroy(ptp_batch* b) {
    if (!b) return;
    cudaSetDevice(b->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    drop_graph(b);
    for (auto e : b->events) cudaEventDestroy(e);
    if (b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

const char* ptp_batch_last_error(const ptp_batch* b) { return b ? b->err.c_str() : "null batch"; }

int ptp_batch_add(ptp_batch* b, ptp_ctx* h) {
    return batch_guard(b, [&]() {
        ptp::Ctx* c = ptp::ctx_of(h);
        PTP_REQUIRE(c, "ptp_batch_add: null context");
        PTP_REQUIRE(c->ready, "ptp_batch_add: the context is not set up");
        PTP_REQUIRE(c->device == b->device, "ptp_batch_add: the context is on another device");
        for (auto* x : b->items) PTP_REQUIRE(x != h, "ptp_batch_add: context added twice");
        b->items.push_back(h);
        drop_graph(b);
        return PTP_OK;
    });
}

int ptp_batch_size(const ptp_batch* b) { return b ? (int)b->items.size() : PTP_EINVAL; }

int ptp_batch_result_dev(ptp_batch* b, int i, double* U) {
    return batch_guard(b, [&]() {
        PTP_REQUIRE(i >= 0 && i < (int)b->items.size() && U, "ptp_batch_result_dev: bad index or pointer");
        ptp::Ctx* c = ptp::ctx_of(b->items[i]);
        const size_t cnt = (size_t)c->n * c->N;
        PTP_CUDA(cudaMemcpyAsync(U, c->U.p, cnt * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
        PTP_CUDA(cudaStreamSynchronize(c->stream));
        return PTP_OK;
    });
}

int ptp_batch_solve(ptp_batch* b, const ptp_opts* opts, ptp_stats* stats, int* n_converged) {
    return batch_guard(b, [&]() {
        PTP_REQUIRE(opts && opts->max_outer >= 1 && opts->tol >= 0, "ptp_batch_solve: bad options");
        const int K = (int)b->items.size();
        PTP_REQUIRE(K > 0, "ptp_batch_solve: empty batch");
        const auto t0 = std::chrono::steady_clock::now();
        std::vector<ptp::Ctx*> cs(K);
        for (int i = 0; i < K; ++i) {
            cs[i] = ptp::ctx_of(b->items[i]);
            PTP_REQUIRE(cs[i]->ready, "ptp_batch_solve: a context is no longer set up");
            // solver options from the call; hierarchy and precision from each set-up
            ptp_opts o = *opts;
            o.precision = cs[i]->opts.precision;
            o.spatial_prec = cs[i]->opts.spatial_prec;
            o.time_levels = cs[i]->opts.time_levels;
            o.coarse_steps = cs[i]->opts.coarse_steps;
            o.coarse_solver = cs[i]->opts.coarse_solver;
            ptp::set_row_block(cs[i]->row_block);
            ptp::solve_begin(*cs[i], o, nullptr, ptp::STEP_FORWARD);
        }
        // capture one step of every instance (re-captured when any step changes)
        std::vector<int64_t> keys(K);
        for (int i = 0; i < K; ++i) keys[i] = ptp::step_key(*cs[i], cs[i]->opts);
        if (!b->exec || b->keys != keys) {
            drop_graph(b);
            while ((int)b->events.size() < K + 1) {
                cudaEvent_t e;
                PTP_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
                b->events.push_back(e);
            }
            b->per_step.assign(K, 0);
            cudaGraph_t g;
            PTP_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
            try {
                PTP_CUDA(cudaEventRecord(b->events[K], b->stream));
                for (int i = 0; i < K; ++i) {
                    PTP_CUDA(cudaStreamWaitEvent(cs[i]->stream, b->events[K], 0));
                    ptp::set_row_block(cs[i]->row_block);
                    b->per_step[i] = ptp::enqueue_step(*cs[i], ptp::STEP_FORWARD);
                    PTP_CUDA(cudaEventRecord(b->events[i], cs[i]->stream));
                    PTP_CUDA(cudaStreamWaitEvent(b->stream, b->events[i], 0));
                }
            } catch (...) {
                cudaStreamEndCapture(b->stream, &g);
                throw;
            }
            PTP_CUDA(cudaStreamEndCapture(b->stream, &g));
            PTP_CUDA(cudaGraphInstantiate(&b->exec, g, 0));
            cudaGraphDestroy(g);
            b->keys = keys;
        }
        // every context's stream must see its set-up work before the graph runs
        for (int i = 0; i < K; ++i) PTP_CUDA(cudaStreamSynchronize(cs[i]->stream));
        cudaEvent_t e0, e1;
        PTP_CUDA(cudaEventCreate(&e0));
        PTP_CUDA(cudaEventCreate(&e1));
        PTP_CUDA(cudaEventRecord(e0, b->stream));
        const int every = std::max(1, opts->check_every);
        int launched = 0, slot = 0, pending = -1;
        bool stop = false;
        cudaEvent_t chk[2];
        PTP_CUDA(cudaEventCreateWithFlags(&chk[0], cudaEventDisableTiming));
        PTP_CUDA(cudaEventCreateWithFlags(&chk[1], cudaEventDisableTiming));
        while (launched < opts->max_outer && !stop) {
            const int chunk = std::min(every, opts->max_outer - launched);
            for (int k = 0; k < chunk; ++k) PTP_CUDA(cudaGraphLaunch(b->exec, b->stream));
            launched += chunk;
            for (int i = 0; i < K; ++i)
                PTP_CUDA(cudaMemcpyAsync(&cs[i]->h_status[slot], cs[i]->status.p, sizeof(ptp::Status),
                                         cudaMemcpyDeviceToHost, b->stream));
            PTP_CUDA(cudaEventRecord(chk[slot], b->stream));
            if (pending >= 0) {
                PTP_CUDA(cudaEventSynchronize(chk[pending]));
                bool all = true;
                for (int i = 0; i < K; ++i) all = all && cs[i]->h_status[pending].done != 0;
                stop = all;
            }
            pending = slot;
            slot ^= 1;
        }
        PTP_CUDA(cudaEventRecord(e1, b->stream));
        PTP_CUDA(cudaStreamSynchronize(b->stream));
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaEventDestroy(chk[0]);
        cudaEventDestroy(chk[1]);
        const double wall = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        int conv = 0, worst = PTP_OK;
        for (int i = 0; i < K; ++i) {
            ptp::set_row_block(cs[i]->row_block);
            ptp_stats st;
            std::memset(&st, 0, sizeof(st));
            const int rc = ptp::solve_end(*cs[i], &st, ptp::STEP_FORWARD, (int64_t)launched * b->per_step[i], wall, ms);
            if (stats) stats[i] = st;
            if (rc == PTP_OK) ++conv;
            else if (worst == PTP_OK || rc == PTP_ENAN) worst = rc;
        }
        if (n_converged) *n_converged = conv;
        return worst;
    });
}

}  // extern "C"
