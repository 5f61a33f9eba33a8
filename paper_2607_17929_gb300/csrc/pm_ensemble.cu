// Batched ensemble: many independent boxes (each its own size, box length and
// seed) stepped together.  Every box is a full single-box context; one
// ensemble step issues all boxes' steps on K streams and captures them into
// one CUDA graph, so the small boxes' kernels run concurrently and the CPU
// issues one graph launch per step.  K is chosen by pm_ensemble_tune, which
// times ensemble steps for a few candidate stream counts.  With K > 1 the
// boxes of the largest mesh go, in order, to stream 0, whose large grids fill
// the GPU anyway; the smaller boxes spread over streams 1 .. K-1, so that
// their small, launch-bound kernels run beside the large ones.  The step is
// captured afresh each time (the potential ring, the particle ping-pong and
// the step's scalars change from step to step) but the topology does not, so
// the executable graph of the previous step is updated in place rather than
// instantiated again.
#include <algorithm>
#include <chrono>
#include <vector>

#include "pm_internal.cuh"


struct pm_ensemble {
    std::vector<pm_ctx *> box;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> joins;
    cudaStream_t origin = nullptr;
    cudaEvent_t fork = nullptr, t0 = nullptr, t1 = nullptr;
    cudaGraphExec_t exec = nullptr;  // executable graph of the last captured step
    int exec_k = 0;                  // stream count it was captured with
    int k = 1;                       // streams in use
    int nmax = 0;                    // largest mesh side in the ensemble
    std::string err;

    // stream of box b for the current stream count
    cudaStream_t stream_of(size_t b) const
    {
        if (k == 1) return streams[0];
        if (box[b]->c.N == nmax) return streams[0];
        size_t r = 0;   // rank of b among the smaller boxes
        for (size_t i = 0; i < b; i++) r += box[i]->c.N != nmax;
        return streams[1 + r % (size_t)(k - 1)];
    }
};

namespace {

constexpr int ENS_MAX_STREAMS = 32;

pm_status ens_fail(pm_ensemble *e, pm_status st, const char *msg)
{
    e->err = msg;
    return st;
}

// one ensemble step: fork from the origin stream to k streams, step every box
// on stream (box % k), join back; with capture, the whole step becomes the graph
// e->exec (updated in place when the previous one has the same topology)
pm_status ens_issue(pm_ensemble *e, bool capture)
{
    cudaGraph_t graph = nullptr;
    if (capture && cudaStreamBeginCapture(e->origin, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return ens_fail(e, PM_ERR_CUDA, "cudaStreamBeginCapture failed");
    cudaEventRecord(e->fork, e->origin);
    for (int s = 0; s < e->k; s++) cudaStreamWaitEvent(e->streams[s], e->fork, 0);
    pm_status st = PM_OK;
    for (size_t b = 0; b < e->box.size() && st == PM_OK; b++) {
        pm::Ctx &c = e->box[b]->c;
        c.stream = e->stream_of(b);
        c.no_timing = capture;
        st = pm_step(e->box[b]);
        c.no_timing = false;
    }
    for (int s = 0; s < e->k; s++) {
        cudaEventRecord(e->joins[s], e->streams[s]);
        cudaStreamWaitEvent(e->origin, e->joins[s], 0);
    }
    if (!capture) return st;
    cudaError_t ce = cudaStreamEndCapture(e->origin, &graph);
    if (st != PM_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (ce != cudaSuccess || !graph) return ens_fail(e, PM_ERR_CUDA, "cudaStreamEndCapture failed");
    bool updated = false;
    if (e->exec && e->exec_k == e->k) {
        cudaGraphExecUpdateResultInfo info{};
        updated = cudaGraphExecUpdate(e->exec, graph, &info) == cudaSuccess;
        if (!updated) cudaGetLastError();
    }
    if (!updated) {
        if (e->exec) cudaGraphExecDestroy(e->exec);
        e->exec = nullptr;
        ce = cudaGraphInstantiate(&e->exec, graph, 0);
        if (ce != cudaSuccess) {
            e->exec = nullptr;
            cudaGraphDestroy(graph);
            return ens_fail(e, PM_ERR_CUDA, "cudaGraphInstantiate failed");
        }
        e->exec_k = e->k;
    }
    cudaGraphDestroy(graph);
    return PM_OK;
}

}  // namespace

extern "C" {

pm_status pm_ensemble_init(const pm_config *cfgs, int32_t nbox, pm_ensemble **out)
{
    if (!cfgs || !out || nbox < 1) return PM_ERR_INVALID_ARG;
    *out = nullptr;
    for (int b = 0; b < nbox; b++)
        if (cfgs[b].n_steps != cfgs[0].n_steps) return PM_ERR_INVALID_ARG;  // boxes step in lockstep
    pm_ensemble *e = new (std::nothrow) pm_ensemble();
    if (!e) return PM_ERR_OOM;
    e->streams.resize(ENS_MAX_STREAMS);
    e->joins.resize(ENS_MAX_STREAMS);
    bool ok = cudaStreamCreateWithFlags(&e->origin, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&e->fork, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreate(&e->t0) == cudaSuccess && cudaEventCreate(&e->t1) == cudaSuccess;
    for (int s = 0; s < ENS_MAX_STREAMS && ok; s++)
        ok = cudaStreamCreateWithFlags(&e->streams[s], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&e->joins[s], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        pm_ensemble_destroy(e);
        return PM_ERR_CUDA;
    }
    e->k = nbox < 8 ? nbox : 8;
    for (int b = 0; b < nbox; b++) e->nmax = std::max(e->nmax, (int)cfgs[b].n_mesh);
    for (int b = 0; b < nbox; b++) {
        pm_config cfg = cfgs[b];
        cfg.stream = e->streams[0];
        pm_ctx *c = nullptr;
        pm_status st = pm_init(&cfg, &c);
        if (st != PM_OK) {
            pm_ensemble_destroy(e);
            return st;
        }
        e->box.push_back(c);
    }
    *out = e;
    return PM_OK;
}

void pm_ensemble_destroy(pm_ensemble *e)
{
    if (!e) return;
    if (e->origin) cudaStreamSynchronize(e->origin);
    if (e->exec) cudaGraphExecDestroy(e->exec);
    for (pm_ctx *c : e->box) pm_destroy(c);
    for (size_t s = 0; s < e->streams.size(); s++) {
        if (e->streams[s]) cudaStreamDestroy(e->streams[s]);
        if (e->joins[s]) cudaEventDestroy(e->joins[s]);
    }
    if (e->fork) cudaEventDestroy(e->fork);
    if (e->t0) cudaEventDestroy(e->t0);
    if (e->t1) cudaEventDestroy(e->t1);
    if (e->origin) cudaStreamDestroy(e->origin);
    cudaGetLastError();
    delete e;
}

const char *pm_ensemble_last_error(const pm_ensemble *e)
{
    return e ? e->err.c_str() : "null ensemble";
}

pm_status pm_ensemble_box(pm_ensemble *e, int32_t box, pm_ctx **ctx)
{
    if (!e || !ctx || box < 0 || box >= (int32_t)e->box.size()) return PM_ERR_INVALID_ARG;
    *ctx = e->box[box];
    return PM_OK;
}

pm_status pm_ensemble_set_particles(pm_ensemble *e, int32_t box, const double *pos, const double *mom)
{
    if (!e || box < 0 || box >= (int32_t)e->box.size()) return PM_ERR_INVALID_ARG;
    pm_ctx *c = e->box[box];
    c->c.stream = e->stream_of((size_t)box);
    pm_status st = pm_set_particles(c, pos, mom);
    if (st == PM_OK && cudaStreamSynchronize(c->c.stream) != cudaSuccess) return PM_ERR_CUDA;
    return st;
}

pm_status pm_ensemble_step(pm_ensemble *e, int32_t use_graph)
{
    if (!e) return PM_ERR_INVALID_ARG;
    if (!use_graph) return ens_issue(e, false);
    pm_status st = ens_issue(e, true);
    if (st != PM_OK) return st;
    cudaError_t ce = cudaGraphLaunch(e->exec, e->origin);
    return ce == cudaSuccess ? PM_OK : ens_fail(e, PM_ERR_CUDA, "cudaGraphLaunch failed");
}

pm_status pm_ensemble_sync(pm_ensemble *e)
{
    if (!e) return PM_ERR_INVALID_ARG;
    return cudaStreamSynchronize(e->origin) == cudaSuccess ? PM_OK : PM_ERR_CUDA;
}

pm_status pm_ensemble_stream(pm_ensemble *e, void **stream)
{
    if (!e || !stream) return PM_ERR_INVALID_ARG;
    *stream = e->origin;
    return PM_OK;
}

pm_status pm_ensemble_set_streams(pm_ensemble *e, int32_t n_streams)
{
    if (!e || n_streams < 1 || n_streams > ENS_MAX_STREAMS) return PM_ERR_INVALID_ARG;
    e->k = n_streams;
    return PM_OK;
}

pm_status pm_ensemble_tune(pm_ensemble *e, int32_t *n_streams)
{
    if (!e) return PM_ERR_INVALID_ARG;
    // FFT column-pass shapes, once per distinct mesh size
    for (size_t b = 0; b < e->box.size(); b++) {
        pm::Ctx &c = e->box[b]->c;
        size_t first = b;
        for (size_t a = 0; a < b; a++)
            if (e->box[a]->c.N == c.N && e->box[a]->c.mixed == c.mixed) {
                first = a;
                break;
            }
        c.stream = e->stream_of(b);
        pm_status st = first == b ? pm_fft_shapes(e->box[b], -1, -1, nullptr, nullptr)
                                  : pm_fft_shapes(e->box[b], e->box[first]->c.col_shape[0],
                                                  e->box[first]->c.col_shape[1], nullptr, nullptr);
        if (st != PM_OK) return st;
    }
    const int cand[] = {1, 2, 4, 8};
    constexpr int TRIAL_STEPS = 2;
    float best = 1e30f;
    int best_k = e->k;
    for (int k : cand) {
        if (k > (int)e->box.size() || k > ENS_MAX_STREAMS) break;
        // one untimed step (it instantiates the graph of the new stream layout), then TRIAL_STEPS timed
        // graph steps (the boxes advance: tuning consumes schedule steps)
        e->k = k;
        pm_status st0 = pm_ensemble_step(e, 1);
        if (st0 != PM_OK) return st0;
        if (cudaEventRecord(e->t0, e->origin) != cudaSuccess) return PM_ERR_CUDA;
        for (int t = 0; t < TRIAL_STEPS; t++) {
            pm_status st = pm_ensemble_step(e, 1);
            if (st != PM_OK) return st;
        }
        cudaEventRecord(e->t1, e->origin);
        if (cudaEventSynchronize(e->t1) != cudaSuccess) return PM_ERR_CUDA;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e->t0, e->t1);
        if (ms < best) {
            best = ms;
            best_k = k;
        }
    }
    e->k = best_k;
    if (n_streams) *n_streams = best_k;
    return PM_OK;
}

}  // extern "C"
