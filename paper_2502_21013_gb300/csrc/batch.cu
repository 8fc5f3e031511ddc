// Batched solve of many independent instances (uneven mesh sizes and N).
//
// Each instance is a set-up context with its own buffers.  One outer
// fixed-point step of every instance is first RECORDED: its launchers append
// (kernel kind, launch shape, argument struct) instead of launching.  The
// recorded programs are then merged into one: each instance's launches keep
// their order, and launches of the same kind (same batched kernel, block size,
// vector width and variant) at aligned positions become ONE launch over the
// work-list of those instances, every instance getting its own virtual grid
// (a contiguous range of the launch's blocks).  The alignment is a shortest
// common supersequence built instance by instance from longest common
// subsequences of the kind sequences, so instances of the same hierarchy
// share every launch and deeper ones add only their extra levels; the number
// of launches per step does not grow with the number of instances.  The
// merged program is captured into one CUDA graph per step.  An instance whose
// step has work without a batched form (another residual law, the ELL path,
// the DFT solver) runs as a parallel branch of the same graph instead.
//
// An instance that has met its stopping rule keeps its entries, but every
// kernel body of it returns at once (its device flag), so its iterate is the
// one that converged.  The host reads all statuses every check_every steps
// and stops when every instance is done.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <numeric>
#include <vector>

#include "common.h"
#include "kernels.h"

namespace ptp {
Ctx* ctx_of(ptp_ctx* h);

Recorder*& active_recorder() {
    static thread_local Recorder* r = nullptr;
    return r;
}
}  // namespace ptp

namespace {

using ptp::BatchLaunch;
using ptp::KShape;
using ptp::RecordedLaunch;

struct MergedOp {
    BatchLaunch fn = nullptr;
    KShape shape;                              // common kind; the largest dynamic shared memory
    std::vector<int> inst;                     // instance of each entry
    std::vector<const RecordedLaunch*> rec;    // its recorded launch
    size_t off_args = 0, off_inst = 0, off_geo = 0;
    int blocks = 0;
};

bool same_kind(const MergedOp& m, const RecordedLaunch& r) {
    return m.fn == r.fn && m.shape.block == r.shape.block && m.shape.vec == r.shape.vec &&
           m.shape.variant == r.shape.variant && m.rec.front()->args.size() == r.args.size();
}

MergedOp single(int inst, const RecordedLaunch& r) {
    MergedOp m;
    m.fn = r.fn;
    m.shape = r.shape;
    m.inst.push_back(inst);
    m.rec.push_back(&r);
    return m;
}

// merges program `ops` of instance `inst` into `seq` (longest common subsequence of kinds)
std::vector<MergedOp> merge(std::vector<MergedOp>&& seq, int inst, const std::vector<RecordedLaunch>& ops) {
    const size_t A = seq.size(), B = ops.size();
    std::vector<int> dp((A + 1) * (B + 1), 0);
    auto at = [&](size_t a, size_t b) -> int& { return dp[a * (B + 1) + b]; };
    for (size_t a = 1; a <= A; ++a)
        for (size_t b = 1; b <= B; ++b)
            at(a, b) = same_kind(seq[a - 1], ops[b - 1]) ? at(a - 1, b - 1) + 1 : std::max(at(a - 1, b), at(a, b - 1));
    std::vector<MergedOp> out;
    out.reserve(A + B);
    size_t a = A, b = B;
    while (a > 0 || b > 0) {
        if (a > 0 && b > 0 && same_kind(seq[a - 1], ops[b - 1]) && at(a, b) == at(a - 1, b - 1) + 1) {
            MergedOp m = std::move(seq[a - 1]);
            m.inst.push_back(inst);
            m.rec.push_back(&ops[b - 1]);
            m.shape.smem = std::max(m.shape.smem, ops[b - 1].shape.smem);
            out.push_back(std::move(m));
            --a;
            --b;
        } else if (a > 0 && (b == 0 || at(a - 1, b) >= at(a, b - 1))) {
            out.push_back(std::move(seq[a - 1]));
            --a;
        } else {
            out.push_back(single(inst, ops[b - 1]));
            --b;
        }
    }
    std::reverse(out.begin(), out.end());
    return out;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

struct ptp_batch {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::vector<ptp_ctx*> items;
    cudaGraphExec_t exec = nullptr;
    std::vector<int64_t> keys;  // step keys of the captured graph
    std::vector<int64_t> per_step;
    std::vector<cudaEvent_t> events;
    std::string err;
    int mode = PTP_BATCH_AUTO;      // requested layout
    int groups = 4;                 // merged programs that run concurrently (PTP_BATCH_MERGED)
    int use_mode = PTP_BATCH_MERGED, use_groups = 4;   // layout of the captured step
    std::vector<cudaStream_t> gstreams;
    std::vector<cudaEvent_t> gevents;
    // the merged programs, one per group of instances
    std::vector<ptp::Recorder> recs;
    std::vector<std::vector<MergedOp>> merged;
    std::vector<int> branch;        // instances that run as graph branches
    unsigned char* blob = nullptr;  // device work-lists (argument structs and virtual grids)
    int64_t step_launches = 0;      // kernels per batched step
    int merged_instances = 0;
};

namespace {

void drop_graph(ptp_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    b->keys.clear();
    if (b->blob) cudaFree(b->blob);
    b->blob = nullptr;
    b->merged.clear();
    b->recs.clear();
    b->branch.clear();
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

struct RecordGuard {
    explicit RecordGuard(ptp::Recorder* r) { ptp::active_recorder() = r; }
    ~RecordGuard() { ptp::active_recorder() = nullptr; }
};

// records every instance's step and merges those without foreign work
void plan(ptp_batch* b, const std::vector<ptp::Ctx*>& cs) {
    const int K = (int)cs.size();
    b->recs.assign(K, ptp::Recorder{});
    b->per_step.assign(K, 0);
    std::vector<int> mergeable;
    for (int i = 0; i < K; ++i) {
        if (b->use_mode != PTP_BATCH_MERGED) {
            b->branch.push_back(i);
            continue;
        }
        ptp::apply_schedule(*cs[i]);
        {
            RecordGuard g(&b->recs[i]);
            b->per_step[i] = ptp::enqueue_step(*cs[i], ptp::STEP_FORWARD);
        }
        if (b->recs[i].foreign == 0 && !b->recs[i].ops.empty()) mergeable.push_back(i);
        else b->branch.push_back(i);
    }
    // groups balanced by space-time size (largest first onto the lightest
    // group); inside a group the longest programs form the backbone
    const int G = std::max(1, std::min(b->use_groups, (int)mergeable.size()));
    std::vector<std::vector<int>> grp(G);
    {
        std::vector<int> order = mergeable;
        auto size_of = [&](int i) { return (double)cs[i]->n * cs[i]->N; };
        std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return size_of(x) > size_of(y); });
        std::vector<double> load(G, 0.0);
        for (int i : order) {
            const int g = (int)(std::min_element(load.begin(), load.end()) - load.begin());
            grp[g].push_back(i);
            load[g] += size_of(i);
        }
    }
    std::vector<std::vector<MergedOp>> seqs(G);
    for (int g = 0; g < G; ++g) {
        std::stable_sort(grp[g].begin(), grp[g].end(),
                         [&](int x, int y) { return b->recs[x].ops.size() > b->recs[y].ops.size(); });
        for (int i : grp[g]) seqs[g] = merge(std::move(seqs[g]), i, b->recs[i].ops);
    }
    // work-lists: argument structs, the instance of every block and the
    // virtual grid of every instance, for every merged launch
    size_t bytes = 0;
    for (auto& seq : seqs)
    for (MergedOp& m : seq) {
        const size_t k = m.inst.size();
        long total = 0;
        for (size_t j = 0; j < k; ++j) total += (long)m.rec[j]->shape.gx * std::max(1, m.rec[j]->shape.gy);
        PTP_REQUIRE(total < (1L << 31), "batched launch: too many blocks");
        m.blocks = (int)total;
        m.off_args = bytes = align_up(bytes, 256);
        bytes += k * m.rec.front()->args.size();
        m.off_geo = bytes = align_up(bytes, 16);
        bytes += k * sizeof(int4);
        m.off_inst = bytes = align_up(bytes, 16);
        bytes += (size_t)total * sizeof(int);
    }
    std::vector<unsigned char> host(std::max<size_t>(bytes, 1), 0);
    for (auto& seq : seqs)
    for (MergedOp& m : seq) {
        const size_t k = m.inst.size(), asz = m.rec.front()->args.size();
        int4* geo = reinterpret_cast<int4*>(host.data() + m.off_geo);
        int* inst_of = reinterpret_cast<int*>(host.data() + m.off_inst);
        int start = 0;
        for (size_t j = 0; j < k; ++j) {
            std::memcpy(host.data() + m.off_args + j * asz, m.rec[j]->args.data(), asz);
            const int gx = m.rec[j]->shape.gx, gy = std::max(1, m.rec[j]->shape.gy);
            geo[j] = make_int4(start, gx, gy, 0);
            for (int t = 0; t < gx * gy; ++t) inst_of[start + t] = (int)j;
            start += gx * gy;
        }
    }
    if (bytes > 0) {
        PTP_CUDA(cudaMalloc((void**)&b->blob, bytes));
        PTP_CUDA(cudaMemcpy(b->blob, host.data(), bytes, cudaMemcpyHostToDevice));
    }
    b->merged = std::move(seqs);
    b->merged_instances = (int)mergeable.size();
    while (b->gstreams.size() < b->merged.size()) {
        cudaStream_t st;
        PTP_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        b->gstreams.push_back(st);
        cudaEvent_t e;
        PTP_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        b->gevents.push_back(e);
    }
}

// the step of every instance: merged launches on the batch stream, branches on their own
void enqueue_batched_step(ptp_batch* b, const std::vector<ptp::Ctx*>& cs) {
    const int K = (int)cs.size();
    PTP_CUDA(cudaEventRecord(b->events[K], b->stream));
    int64_t launches = 0;
    for (int i : b->branch) {
        PTP_CUDA(cudaStreamWaitEvent(cs[i]->stream, b->events[K], 0));
        ptp::apply_schedule(*cs[i]);
        b->per_step[i] = ptp::enqueue_step(*cs[i], ptp::STEP_FORWARD);
        launches += b->per_step[i];
        PTP_CUDA(cudaEventRecord(b->events[i], cs[i]->stream));
    }
    // one group on the batch stream, the others forked onto their own streams
    const int G = (int)b->merged.size();
    for (int g = 0; g < G; ++g) {
        cudaStream_t st = g == 0 ? b->stream : b->gstreams[g];
        if (g > 0) PTP_CUDA(cudaStreamWaitEvent(st, b->events[K], 0));
        for (const MergedOp& m : b->merged[g]) {
            ptp::BatchMap map;
            map.inst_of = reinterpret_cast<const int*>(b->blob + m.off_inst);
            map.geo = reinterpret_cast<const int4*>(b->blob + m.off_geo);
            map.n = (int)m.inst.size();
            launches += m.fn(b->blob + m.off_args, map, m.blocks, m.shape, st);
        }
        if (g > 0) PTP_CUDA(cudaEventRecord(b->gevents[g], st));
    }
    for (int g = 1; g < G; ++g) PTP_CUDA(cudaStreamWaitEvent(b->stream, b->gevents[g], 0));
    for (int i : b->branch) PTP_CUDA(cudaStreamWaitEvent(b->stream, b->events[i], 0));
    b->step_launches = launches;
}

// plan and capture one step of every instance in the layout b->use_mode / use_groups
void capture_step(ptp_batch* b, const std::vector<ptp::Ctx*>& cs) {
    plan(b, cs);
    cudaGraph_t g;
    PTP_CUDA(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    try {
        enqueue_batched_step(b, cs);
    } catch (...) {
        cudaStreamEndCapture(b->stream, &g);
        throw;
    }
    PTP_CUDA(cudaStreamEndCapture(b->stream, &g));
    PTP_CUDA(cudaGraphInstantiate(&b->exec, g, 0));
    cudaGraphDestroy(g);
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
    for (auto e : b->gevents) cudaEventDestroy(e);
    for (auto st : b->gstreams) cudaStreamDestroy(st);
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

int ptp_batch_set_mode(ptp_batch* b, int mode) {
    return batch_guard(b, [&]() {
        PTP_REQUIRE(mode == PTP_BATCH_MERGED || mode == PTP_BATCH_BRANCHES || mode == PTP_BATCH_AUTO,
                    "ptp_batch_set_mode: bad mode");
        if (mode != b->mode) drop_graph(b);
        b->mode = mode;
        return PTP_OK;
    });
}

int ptp_batch_plan_info(const ptp_batch* b, int64_t* launches_per_step, int* merged_instances, int* merged_launches) {
    if (!b) return PTP_EINVAL;
    if (!b->exec) return PTP_ESTATE;
    if (launches_per_step) *launches_per_step = b->step_launches;
    if (merged_instances) *merged_instances = b->merged_instances;
    if (merged_launches) {
        size_t m = 0;
        for (const auto& seq : b->merged) m += seq.size();
        *merged_launches = (int)m;
    }
    return PTP_OK;
}

int ptp_batch_set_groups(ptp_batch* b, int groups) {
    return batch_guard(b, [&]() {
        PTP_REQUIRE(groups >= 1 && groups <= 64, "ptp_batch_set_groups: 1..64 groups");
        if (groups != b->groups) drop_graph(b);
        b->groups = groups;
        return PTP_OK;
    });
}

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
            ptp::apply_schedule(*cs[i]);
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
            if (b->mode == PTP_BATCH_AUTO) {
                // layout autotuner: a few steps of each candidate, the fastest kept;
                // then every instance starts again from zero
                struct Layout { int mode, groups; };
                const Layout cands[3] = {{PTP_BATCH_BRANCHES, 1}, {PTP_BATCH_MERGED, 1}, {PTP_BATCH_MERGED, 4}};
                cudaEvent_t e0, e1;
                PTP_CUDA(cudaEventCreate(&e0));
                PTP_CUDA(cudaEventCreate(&e1));
                double best = 1e300;
                Layout bl = cands[0];
                for (const Layout& cd : cands) {
                    if (cd.groups > 1 && K < 2 * cd.groups) continue;
                    b->use_mode = cd.mode;
                    b->use_groups = cd.groups;
                    capture_step(b, cs);
                    for (int i = 0; i < K; ++i) PTP_CUDA(cudaStreamSynchronize(cs[i]->stream));
                    for (int r = 0; r < 2; ++r) PTP_CUDA(cudaGraphLaunch(b->exec, b->stream));
                    PTP_CUDA(cudaEventRecord(e0, b->stream));
                    for (int r = 0; r < 3; ++r) PTP_CUDA(cudaGraphLaunch(b->exec, b->stream));
                    PTP_CUDA(cudaEventRecord(e1, b->stream));
                    PTP_CUDA(cudaEventSynchronize(e1));
                    float ms = 0;
                    PTP_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                    if (ms < best) {
                        best = ms;
                        bl = cd;
                    }
                    drop_graph(b);
                }
                cudaEventDestroy(e0);
                cudaEventDestroy(e1);
                b->use_mode = bl.mode;
                b->use_groups = bl.groups;
                for (int i = 0; i < K; ++i) {
                    ptp::apply_schedule(*cs[i]);
                    ptp::solve_begin(*cs[i], cs[i]->opts, nullptr, ptp::STEP_FORWARD);
                }
            } else {
                b->use_mode = b->mode;
                b->use_groups = b->groups;
            }
            capture_step(b, cs);
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
            ptp::apply_schedule(*cs[i]);
            ptp_stats st;
            std::memset(&st, 0, sizeof(st));
            const int rc = ptp::solve_end(*cs[i], &st, ptp::STEP_FORWARD, (int64_t)launched * b->step_launches, wall, ms);
            if (stats) stats[i] = st;
            if (rc == PTP_OK) ++conv;
            else if (worst == PTP_OK || rc == PTP_ENAN) worst = rc;
        }
        if (n_converged) *n_converged = conv;
        return worst;
    });
}

}  // extern "C"
