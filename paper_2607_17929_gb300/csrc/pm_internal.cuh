// Internal declarations of libpm (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>
#include <vector>

#include "../../include/pm.h"

namespace pm {

// ---------------------------------------------------------------------------
// Precision traits.  FP64: f64 everywhere.  Mixed: f32 offsets, momenta,
// fields and FFTs; per-cell deposit sums in compensated f32 (float-float,
// about 48 significant bits) and the k = 0 mode in f64.
// ---------------------------------------------------------------------------
template <class T> struct Cplx;
template <> struct Cplx<double> { using type = double2; };
template <> struct Cplx<float> { using type = float2; };

// Particle record: cell index + offset inside the cell + momentum + id.
// 32 bytes in mixed precision, 64 bytes in FP64 (one/two 32-byte sectors).
template <class T> struct alignas(16) Particle;
template <> struct alignas(16) Particle<float> {
    int32_t cell;
    uint32_t id;
    float f[3];
    float u[3];
};
template <> struct alignas(16) Particle<double> {
    int32_t cell;
    uint32_t id;
    double f[3];
    double u[3];
    double pad;
};
static_assert(sizeof(Particle<float>) == 32, "mixed particle must be 32 B");
static_assert(sizeof(Particle<double>) == 64, "fp64 particle must be 64 B");

// Up to 16 device pointers for batched multi-field launches.
struct Ptrs {
    void *p[16];
};

// Per-step scalars (computed in FP64 on the host).
struct StepScalars {
    double a;            // a_n
    double hc;           // Hc(a_n)
    double c_phi_dt;     // 3 Hc / dtau_{n-1} (0 in the bootstrap and Newtonian mode)
    double c_phi_h2;     // 3 Hc^2 (0 in Newtonian mode)
    double inv_dtau_prev2;  // 1 / dtau_{n-2} for phi'
    double dtau;         // dtau_n (tensor step, drift)
    double dtau_kick;    // (dtau_{n-1} + dtau_n) / 2
    double a_half;       // a_{n+1/2}
    double hc_half;      // Hc(a_{n+1/2})
    double four_pi_g;
    double mass;
    double omega_m;
    int newtonian;
    int bootstrap;
    int full_hc;         // remainder of Eq. fullHc in the phi source (not in the bootstrap)
    int b_space;         // B from Eq. spacespace
    int b_seed;          // with b_space: this step takes B from the momentum constraint (step 0)
    double dtau_prev;    // dtau_{n-1}
    double b_decay;      // (a_{n-1} / a_n)^2
};

struct FftPlan {
    int n;
    int nst;
    int radix[12];
};

FftPlan make_plan(int n);

// ---------------------------------------------------------------------------
// Context.
// ---------------------------------------------------------------------------
struct Ctx {
    pm_config cfg;
    cudaStream_t stream = nullptr;
    int device = 0;
    bool poisoned = false;
    std::string err;
    int N = 0;
    int64_t nc = 0;    // N^3
    int64_t nh = 0;    // N * N * (N/2 + 1)
    int64_t np = 0;
    bool mixed = false;
    bool newtonian = false;
    bool full_hc = false;       // PM_FULL_HC
    bool b_space = false;       // PM_B_SPACESPACE
    int col_shape[2] = {0, 0};  // shapes of the y and z column FFT passes (pm_fft_shapes)
    int dep_shape = 0;          // record capacity of the deposit's shared-memory chunks (pm_deposit_shape)

    // schedule (host, FP64)
    std::vector<double> a_n, dtau, a_half;
    double h0 = 0, four_pi_g = 0, mass = 0;
    int step = 0;           // completed steps
    int stage = 0;          // 0: ready to project, 1: projected, 2: solved
    bool have_particles = false;

    // device buffers
    void *part[2] = {nullptr, nullptr};  // Particle<T> ping-pong
    int cur = 0;
    int32_t *count = nullptr;   // nc
    int32_t *start = nullptr;   // nc + 1
    int32_t *blocksum = nullptr;   // scan tile sums: one int per 4096 counts, more than the scan's tiles need
    int64_t nblocksum = 0;
    void *phi[3] = {nullptr, nullptr, nullptr};  // ring: phi_{n-2}, phi_{n-1}, phi_n
    int iphi_prev2 = 0, iphi_prev = 1, iphi_new = 2;
    void *chi = nullptr;        // chi_{n-1} before the solve, chi_n after it
    void *B = nullptr;          // 3 * nc
    void *src = nullptr;        // 9 * nc real sources
    void *spec = nullptr;       // 9 * nh complex
    void *tens = nullptr;       // 4 * nh complex tensor state
    void *bstate = nullptr;     // 3 * nh complex B_k between steps (PM_B_SPACESPACE only)
    void *corr = nullptr;       // force correction FP32 [cell][8] (channels 0..2) kicked in by pm_update; not owned
    float corr_scale = 1.f;     // force units per unit of corr
    void *ktab = nullptr;       // N values of ktilde(n)
    void *tw = nullptr;         // N twiddles exp(-2 pi i k / N)
    void *tw2 = nullptr;        // per-stage twiddles of the compile-time-N passes
    double *dscal = nullptr;    // device f64 scalars: [0] k=0 particle sum, [1..3] mean phi per ring slot,
                                // [4] (int) record check of a load, [5] (int) latched check of the async puts
    void *stage_buf = nullptr;  // host-transfer staging (f64)
    int64_t stage_elems = 0;
    FftPlan plan;

    // per-kernel CUDA events of the last RING steps (timing window) and the
    // number of library kernels launched
    static constexpr int RING = 64, NEV = 12;
    cudaEvent_t evr[RING][NEV] = {};
    bool timing_on = false;   // marks are recorded only inside pm_project/solve/update
    int64_t stepc = 0;        // steps started (selects the ring slot)
    int64_t window = 0;       // completed steps in the current timing window
    int64_t launches = 0, launches_mark = 0;

    bool no_timing = false;   // set while a step is captured into a CUDA graph (ensemble, pm_step_graph)

    // pm_step_graph: each pm_step is captured on gstream into one graph and launched on stream; two
    // executable graphs alternate, so the one being updated is never the one still running
    bool graph_step = false;
    cudaStream_t gstream = nullptr;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    int gslot = 0;

    // overlapped packed I/O (pm_put_particles_packed_async / pm_get_particles_packed_async): copy-engine
    // transfers on their own streams between pinned host memory and two device staging buffers
    cudaStream_t io_up = nullptr, io_down = nullptr;
    cudaEvent_t ev_in_ready = nullptr, ev_in_free = nullptr, ev_out_ready = nullptr, ev_out_free = nullptr;
    void *in_stage = nullptr, *out_stage = nullptr;   // n_part packed records each

    void mark(int point)
    {
        if (timing_on && !no_timing) cudaEventRecord(evr[stepc % RING][point], stream);
    }
};

// Event points inside one step.
enum { EV_START = 0, EV_PROJECT = 1, EV_FWD_X = 2, EV_FWD_Y = 3, EV_FWD_Z = 4, EV_SOLVE = 5,
       EV_INV_Z = 6, EV_INV_Y = 7, EV_INV_X = 8, EV_KICK = 9, EV_SCAN = 10, EV_END = 11 };

// True the first time it is called with `mask` on the current device (for per-device one-time set-up
// such as kernel attributes; a repeated set-up from a racing thread is harmless).
inline bool first_on_device(std::atomic<uint64_t> &mask)
{
    int d = 0;
    cudaGetDevice(&d);
    const uint64_t bit = 1ull << (d & 63);
    return (mask.fetch_or(bit) & bit) == 0;
}

// ---------------------------------------------------------------------------
// Launchers (implemented in pm_fft.cu, pm_particles.cu, pm_solve.cu).
// ---------------------------------------------------------------------------
template <class T>
void fft_forward(Ctx &c, int nfields, const void *const *real_in, void *const *spec_out);
template <class T>
void fft_inverse(Ctx &c, int nfields, void *const *spec_in, void *const *real_out);

template <class T>
void launch_project(Ctx &c, const StepScalars &s);
template <class T>
void launch_solve(Ctx &c, const StepScalars &s);
template <class T>
void launch_kick_drift(Ctx &c, const StepScalars &s);
// batched forms for the ensemble: one launch over n boxes of one precision (and one deposit shape)
template <class T>
void launch_project_batch(Ctx *const *cs, const StepScalars *ss, int n, int shape, cudaStream_t st);
template <class T>
void launch_kick_batch(Ctx *const *cs, const StepScalars *ss, int n, cudaStream_t st);
// times the deposit shapes on the context's current state and keeps the fastest (returns it)
template <class T>
int tune_deposit_shape(Ctx &c, const StepScalars &s);
template <class T>
void launch_sort(Ctx &c);
template <class T>
void launch_corr_kick(Ctx &c, const StepScalars &s);
template <class T>
void launch_load_particles(Ctx &c, const double *d_pos, const double *d_mom, int64_t first, int64_t count,
                           int *d_nonfinite);
template <class T>
void launch_store_particles(Ctx &c, double *d_pos, double *d_mom, int64_t first, int64_t count);
template <class T>
void launch_store_particles_scatter(Ctx &c, double *d_pos, double *d_mom);
// packed records (mixed form): load into the current buffer with checks; store from the id-ordered buffer
void launch_load_packed(Ctx &c, const pm_packed_particle *in, int64_t first, int64_t count, int *d_bad);
// all n_part records from device memory counted, checked and placed in cell order (the particle state)
void launch_put_packed_sorted(Ctx &c, const pm_packed_particle *in, int *d_bad);
void launch_store_packed(Ctx &c, pm_packed_particle *out, int64_t first, int64_t count);
template <class T>
void launch_density(Ctx &c, void *real_out);
template <class T>
void launch_pk_bin(Ctx &c, const void *spec_in, int nbins, double *d_acc);
template <class T>
void launch_to_f64(Ctx &c, const void *src, double *dst, int64_t n);
template <class T>
void launch_from_f64(Ctx &c, const double *src, void *dst, int64_t n);
template <class T>
void launch_check_finite(Ctx &c, const double *d, int64_t n, int *d_flag);

void launch_scan(Ctx &c);

// step pieces shared by the single-box calls and the batched ensemble (pm_api.cu)
StepScalars scalars(const Ctx &c, int k, bool bootstrap);
template <class T>
pm_status do_solve(Ctx &c, bool bootstrap);   // forward FFTs, Fourier solve, inverse FFTs
void rotate(Ctx &c);                          // the phi ring after a completed step

// compile-time-N FFT passes (pm_fft.cu)
bool fast_fft_supported(int n);
// column-pass shapes: force_* >= 0 selects one, < 0 times the choices and keeps the fastest;
// false (shape 0 kept) when the context's precision and N have no choice
template <class T>
bool fft_tune_shapes(Ctx &c, int force_y, int force_z);
void fast_twiddles(int n, std::vector<double> &re_im);

}  // namespace pm

// the opaque context of the C ABI
struct pm_ctx {
    pm::Ctx c;
};
