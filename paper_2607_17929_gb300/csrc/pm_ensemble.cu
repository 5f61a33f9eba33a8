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
//
// Batched mode (pm_ensemble_set_batched, or chosen by pm_ensemble_tune): the
// particle kernels of all boxes run as one launch each, over a work list of
// (box, tile) items that spans every box of a precision: one deposit launch
// (each CTA finds its box in a prefix table of tile counts and takes that box's
// parameters from the launch's parameter block), then every box's transforms
// and Fourier solve on the K streams, then one gather + kick + drift launch,
// then every box's counting sort on the K streams.  Small boxes then no longer
// leave most of the GPU idle in their own short particle launches.
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
    bool batched = false;            // particle kernels as one launch over all boxes
    int exec_batched = -1;           // mode the executable graph was captured in
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

void ens_fork(pm_ensemble *e)
{
    cudaEventRecord(e->fork, e->origin);
    for (int s = 0; s < e->k; s++) cudaStreamWaitEvent(e->streams[s], e->fork, 0);
}

void ens_join(pm_ensemble *e)
{
    for (int s = 0; s < e->k; s++) {
        cudaEventRecord(e->joins[s], e->streams[s]);
        cudaStreamWaitEvent(e->origin, e->joins[s], 0);
    }
}

// the batched step of the boxes: one deposit and one kick launch per precision (and deposit shape) over all
// boxes, the per-box transforms, solves and sorts on the k streams in between
template <class T>
void ens_particles(std::vector<pm::Ctx *> &cs, std::vector<pm::StepScalars> &ss, cudaStream_t st, bool deposit)
{
    if (cs.empty()) return;
    if (!deposit) {
        pm::launch_kick_batch<T>(cs.data(), ss.data(), (int)cs.size(), st);
        return;
    }
    for (int v = 0; v < 2; v++) {
        std::vector<pm::Ctx *> cv;
        std::vector<pm::StepScalars> sv;
        for (size_t i = 0; i < cs.size(); i++)
            if (cs[i]->dep_shape == v) {
                cv.push_back(cs[i]);
                sv.push_back(ss[i]);
            }
        if (!cv.empty()) pm::launch_project_batch<T>(cv.data(), sv.data(), (int)cv.size(), v, st);
    }
}

pm_status ens_step_batched(pm_ensemble *e)
{
    const size_t nb = e->box.size();
    for (size_t b = 0; b < nb; b++) {
        const pm::Ctx &c = e->box[b]->c;
        if (c.poisoned) return ens_fail(e, PM_ERR_STATE, "a box is poisoned by an earlier CUDA error");
        if (!c.have_particles || c.stage != 0) return ens_fail(e, PM_ERR_STATE, "a box has no particles or is mid-step");
        if (c.step >= c.cfg.n_steps) return ens_fail(e, PM_ERR_STATE, "schedule exhausted");
    }
    std::vector<pm::Ctx *> c32, c64;
    std::vector<pm::StepScalars> s32, s64;
    for (size_t b = 0; b < nb; b++) {
        pm::Ctx &c = e->box[b]->c;
        c.stepc++;
        (c.mixed ? c32 : c64).push_back(&c);
        (c.mixed ? s32 : s64).push_back(pm::scalars(c, c.step, false));
    }
    ens_particles<float>(c32, s32, e->origin, true);
    ens_particles<double>(c64, s64, e->origin, true);
    ens_fork(e);
    for (size_t b = 0; b < nb; b++) {
        pm::Ctx &c = e->box[b]->c;
        c.stream = e->stream_of(b);
        c.stage = 1;
        const pm_status st = c.mixed ? pm::do_solve<float>(c, false) : pm::do_solve<double>(c, false);
        if (st != PM_OK) return ens_fail(e, st, "box solve failed");
        c.stage = 2;
    }
    ens_join(e);
    for (size_t b = 0; b < nb; b++) {
        pm::Ctx &c = e->box[b]->c;
        if (!c.corr) continue;
        c.stream = e->origin;
        const pm::StepScalars s = pm::scalars(c, c.step, false);
        if (c.mixed) pm::launch_corr_kick<float>(c, s);
        else pm::launch_corr_kick<double>(c, s);
    }
    ens_particles<float>(c32, s32, e->origin, false);
    ens_particles<double>(c64, s64, e->origin, false);
    ens_fork(e);
    for (size_t b = 0; b < nb; b++) {
        pm::Ctx &c = e->box[b]->c;
        c.stream = e->stream_of(b);
        if (c.mixed) pm::launch_sort<float>(c);
        else pm::launch_sort<double>(c);
        pm::rotate(c);
        c.step += 1;
        c.stage = 0;
    }
    ens_join(e);
    if (cudaGetLastError() != cudaSuccess) return ens_fail(e, PM_ERR_CUDA, "batched launch failed");
    return PM_OK;
}

// one ensemble step: fork from the origin stream to k streams, step every box
// on stream (box % k), join back (or the batched form); with capture, the whole
// step becomes the graph e->exec (updated in place when the previous one has
// the same topology)
pm_status ens_issue(pm_ensemble *e, bool capture)
{
    cudaGraph_t graph = nullptr;
    if (capture && cudaStreamBeginCapture(e->origin, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return ens_fail(e, PM_ERR_CUDA, "cudaStreamBeginCapture failed");
    pm_status st = PM_OK;
    if (e->batched) {
        for (size_t b = 0; b < e->box.size(); b++) e->box[b]->c.no_timing = true;
        st = ens_step_batched(e);
        for (size_t b = 0; b < e->box.size(); b++) e->box[b]->c.no_timing = false;
    } else {
        ens_fork(e);
        for (size_t b = 0; b < e->box.size() && st == PM_OK; b++) {
            pm::Ctx &c = e->box[b]->c;
            c.stream = e->stream_of(b);
            c.no_timing = capture;
            st = pm_step(e->box[b]);
            c.no_timing = false;
        }
        ens_join(e);
    }
    if (!capture) return st;
    cudaError_t ce = cudaStreamEndCapture(e->origin, &graph);
    if (st != PM_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (ce != cudaSuccess || !graph) return ens_fail(e, PM_ERR_CUDA, "cudaStreamEndCapture failed");
    bool updated = false;
    if (e->exec && e->exec_k == e->k && e->exec_batched == (int)e->batched) {
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
        e->exec_batched = (int)e->batched;
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

pm_status pm_ensemble_set_batched(pm_ensemble *e, int32_t batched)
{
    if (!e || batched < 0 || batched > 1) return PM_ERR_INVALID_ARG;
    e->batched = batched != 0;
    return PM_OK;
}

pm_status pm_ensemble_get_mode(pm_ensemble *e, int32_t *n_streams, int32_t *batched)
{
    if (!e) return PM_ERR_INVALID_ARG;
    if (n_streams) *n_streams = e->k;
    if (batched) *batched = (int32_t)e->batched;
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
    // deposit chunk capacity, once per distinct mesh size and precision (between steps, so side-effect free)
    for (size_t b = 0; b < e->box.size(); b++) {
        pm::Ctx &c = e->box[b]->c;
        size_t first = b;
        for (size_t a = 0; a < b; a++)
            if (e->box[a]->c.N == c.N && e->box[a]->c.mixed == c.mixed) {
                first = a;
                break;
            }
        c.stream = e->stream_of(b);
        pm_status st = first == b ? pm_deposit_shape(e->box[b], -1, nullptr)
                                  : pm_deposit_shape(e->box[b], e->box[first]->c.dep_shape, nullptr);
        if (st != PM_OK) return st;
    }
    // the stream count and the batched or per-box particle kernels
    const int cand[] = {1, 2, 4, 8};
    constexpr int TRIAL_STEPS = 2;
    float best = 1e30f;
    int best_k = e->k;
    bool best_batched = e->batched;
    for (int trial = 0; trial < 8; trial++) {
        const int k = cand[trial % 4];
        const bool batched = trial >= 4;
        if (k > (int)e->box.size() || k > ENS_MAX_STREAMS) continue;
        // one untimed step (it instantiates the graph of the new stream layout), then TRIAL_STEPS timed
        // graph steps (the boxes advance: tuning consumes schedule steps)
        e->k = k;
        e->batched = batched;
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
            best_batched = batched;
        }
    }
    e->k = best_k;
    e->batched = best_batched;
    if (n_streams) *n_streams = best_k;
    return PM_OK;
}

}  // extern "C"
