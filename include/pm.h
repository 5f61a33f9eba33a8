/*
 * pm.h -- C ABI of libpm, a single-GPU (sm_103a) implementation of one full
 * relativistic particle-mesh step of gevolution 2.0 (arxiv 2607.17929):
 * cloud-in-cell projection of the particles' stress-energy, FFT solves of
 * the scalar (phi, chi), vector (B_i) and tensor (h_ij) metric
 * perturbations, and the relativistic kick and drift of every particle.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Units: comoving box length L = 1, c = 1, conformal time tau in units of
 *   L/c, critical density today = 1, so 4 pi G = 3/2 H0^2 with
 *   H0 = box_mpch / 2997.92458.  Particle mass m = omega_m / n_part, and
 *   "momentum" means the canonical momentum per unit mass u_i = q_i / m.
 * Mesh: vertex-centred N^3 mesh, row-major [z][y][x] with x fastest (the
 *   "fast" direction of the paper's rod decomposition, Sec. 2, Fig. 1).
 * Particle arrays passed in or out: [n_part][3] doubles in (x, y, z) order;
 *   positions in box units, wrapped into [0, 1).  Rows are in particle-id
 *   order; the id of a particle is its row in the pm_set_particles arrays.
 * Pointers: any pointer argument may be host memory (pageable or pinned) or
 *   device memory of the context's device; the library detects which with
 *   cudaPointerGetAttributes.  Pointers are borrowed for the duration of the
 *   call only; the library owns all of its device memory.
 * Streams: all device work is enqueued on cfg->stream (NULL = the legacy
 *   default stream).  Calls that write host memory synchronise the stream
 *   before returning; every other call returns once its work is enqueued.
 * Errors: every call returns a pm_status and never aborts.  The message of
 *   the last error is kept per context (pm_last_error).  A CUDA error
 *   reported by the runtime poisons the context: later calls return
 *   PM_ERR_STATE.  Thread safety: one context must not be used by two host
 *   threads at once; distinct contexts are independent.
 */
#ifndef PM_H
#define PM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PM_OK = 0,
    PM_ERR_INVALID_ARG = 1,      /* NULL pointer, bad id, value out of range */
    PM_ERR_UNSUPPORTED_SIZE = 2, /* n_mesh not of the form 2^a 3^b with a >= 3 in [8, 1024] */
    PM_ERR_OOM = 3,              /* device allocation failed (nothing leaked) */
    PM_ERR_CUDA = 4,             /* CUDA runtime error; the context is poisoned */
    PM_ERR_TIMEOUT = 5,          /* a bounded device wait ran out */
    PM_ERR_STATE = 6             /* call out of order, poisoned context, schedule exhausted */
} pm_status;

typedef enum {
    PM_FP64 = 0,  /* positions cell + f64 offset, f64 momenta, f64 fields and FFTs */
    PM_MIXED = 1  /* int32 cell + f32 offset, f32 momenta, f32 fields and FFTs;
                     f64 background, compensated per-cell deposit sums, f64 k=0 mode */
} pm_precision;

/* flags */
#define PM_NEWTONIAN 1u /* Newtonian limit (Sec. 3.2): project mass only, Poisson equation
                           Lap phi = 4 pi G a^-1 (rho - omega_m), chi = B = h = 0,
                           du/dtau = -a grad phi, dx/dtau = u/a */
#define PM_FULL_HC 2u   /* full Hamiltonian constraint, Eq. fullHc: the terms that are not linear
                           in phi, psi join the phi source as R -= Nl, with
                           Nl = (e^{2phi}-1) Lap phi - 1/2 e^{2phi} |grad phi|^2
                              + 3/2 [(Hc-phi')^2 e^{-2psi} - Hc^2 + 2 Hc phi' + 2 Hc^2 psi]
                           evaluated once on phi_{n-1}, psi_{n-1} = phi_{n-1} - chi_{n-1} and
                           phi' = (phi_{n-1} - phi_{n-2}) / dtau_{n-2} (the predictor of Sec. 3.1,
                           no corrector iterations); 7-point Lap, centred grad */
#define PM_B_SPACESPACE 4u /* B_i from the spin-1 part of Eq. spacespace instead of the momentum
                           constraint: (d_tau + 2 Hc) B_j = W_j with
                           W_j = -i (delta_jl - kt_j kt_l / kt^2) kt_i Sig_il / kt^2, integrated
                           as a_n^2 B_n = a_{n-1}^2 B_{n-1} + dtau_{n-1} a_n^2 W_n.  Step 0 takes B
                           from the momentum constraint to start the integration; after it the
                           T0i sources F are neither written nor transformed (6 forward FFTs
                           instead of 9), so pm_get_field of F_x..F_z keeps step 0's values.
                           Both variants are ignored with PM_NEWTONIAN. */

typedef struct pm_config {
    int32_t n_mesh;    /* N: 2^a 3^b, a >= 3, 8 <= N <= 1024 */
    int32_t n_steps;   /* length of the time-step schedule (>= 1) */
    int64_t n_part;    /* number of particles, 1 <= n_part < 2^31 */
    double box_mpch;   /* comoving box side in Mpc/h (> 0) */
    double omega_m;    /* matter density today, flat LCDM with Omega_L = 1 - omega_m */
    double z_init;     /* redshift of the first step */
    double z_final;    /* redshift after the last step (< z_init) */
    int32_t precision; /* pm_precision */
    uint32_t flags;    /* 0 or PM_NEWTONIAN | PM_FULL_HC | PM_B_SPACESPACE */
    void *stream;      /* cudaStream_t to enqueue on; NULL = default stream */
} pm_config;

typedef struct pm_ctx pm_ctx;

/* Field ids for pm_get_field.  The potentials are those of the latest solve
 * (after pm_solve or pm_step: phi_n, chi_n, B_n of step n).  The sources are
 * those assembled by the latest pm_project (configuration space):
 *   R     = 4piG a^-2 (S00 - a omega_m) - 3Hc/dtau_{n-1} phi_{n-1} - 3Hc^2 chi_{n-1}
 *   F_i   = 4piG a^-2 S0i - phi' d_i psi
 *   Sig_ij = 16piG a^-2 TF(S_ij) - 2 TF[2 d_i phi d_j phi - (d_i phi + d_i psi)(d_j phi + d_j psi)]
 * (Sig is trace-free; Sig_zz = -Sig_xx - Sig_yy is not stored). */
enum {
    PM_FIELD_PHI = 0, PM_FIELD_CHI = 1, PM_FIELD_BX = 2, PM_FIELD_BY = 3, PM_FIELD_BZ = 4,
    PM_FIELD_R = 5, PM_FIELD_FX = 6, PM_FIELD_FY = 7, PM_FIELD_FZ = 8,
    PM_FIELD_SXX = 9, PM_FIELD_SXY = 10, PM_FIELD_SXZ = 11, PM_FIELD_SYY = 12, PM_FIELD_SYZ = 13
};

/* Tensor state ids for pm_get_tensor: helicity amplitudes and their tau derivatives. */
enum { PM_TENSOR_HPLUS = 0, PM_TENSOR_HCROSS = 1, PM_TENSOR_DHPLUS = 2, PM_TENSOR_DHCROSS = 3 };

/* Stage ids for pm_get_timings: mean milliseconds per step, from CUDA events
 * recorded on cfg->stream around each kernel of every step.  Stages and
 * kernels: projection (deposit + source assembly), forward FFT (x, y, z
 * passes), Fourier solve, inverse FFT (z, y, x passes), gather + kick + drift,
 * counting sort (scan, scatter), and the whole step. */
enum { PM_T_PROJECT = 0, PM_T_FFT_FWD = 1, PM_T_SOLVE = 2, PM_T_FFT_INV = 3, PM_T_UPDATE = 4,
       PM_T_SORT = 5, PM_T_STEP = 6, PM_T_FFT_FWD_X = 7, PM_T_FFT_FWD_Y = 8, PM_T_FFT_FWD_Z = 9,
       PM_T_FFT_INV_Z = 10, PM_T_FFT_INV_Y = 11, PM_T_FFT_INV_X = 12, PM_T_SCAN = 13,
       PM_T_SCATTER = 14, PM_T_COUNT = 15 };

/* Create a context: validates cfg, computes the FP64 background schedule
 * (Sec. 3.1: Hc = d ln a / d tau, flat LCDM; steps uniform in ln a from
 * z_init to z_final, tau by 64-point Gauss-Legendre, half-step a by Newton)
 * and allocates every device buffer on the current device.
 * On success *out owns the context; free it with pm_destroy.
 * Errors: INVALID_ARG, UNSUPPORTED_SIZE, OOM, CUDA. */
pm_status pm_init(const pm_config *cfg, pm_ctx **out);

/* Release all device and host memory of ctx (NULL is ignored). */
void pm_destroy(pm_ctx *ctx);

/* Message of the last failed call on ctx ("" if none).  Valid until the next call. */
const char *pm_last_error(const pm_ctx *ctx);

/* Load the particle state at step 0: pos, mom [n_part][3] f64 (host or
 * device).  pos is wrapped into [0,1); the momenta u are those at half a
 * step before the first step (staggered leap-frog, Sec. 3.1).  Sorts the
 * particles by cell and runs the quasi-static bootstrap solve that gives
 * phi_{-1} (phi = chi = 0 in the projection weights, no d/dtau term).
 * Errors: INVALID_ARG (NULL, NaN/Inf in the input), CUDA, STATE. */
pm_status pm_set_particles(pm_ctx *ctx, const double *pos, const double *mom);

/* Projection of step n (Eqs. matterstress to first order in phi, psi):
 * CIC deposit of S00, S0i, TF(S_ij) from the cell-sorted particles with
 * phi_{n-1}, chi_{n-1} interpolated at the particles, and assembly of the
 * sources R, F_i, Sig_ij of Eqs. NewtonHc, momentumcontraint, spacespace
 * with the quadratic terms from the previous step (Sec. 3.1, predictor with
 * zero iterations).  Errors: STATE (no particles, schedule exhausted), CUDA. */
pm_status pm_project(pm_ctx *ctx);

/* Field solve of step n: forward r2c FFTs of the sources, Fourier-space
 * solutions phi_n, chi_n, B_n and one implicit-midpoint step of the tensor
 * modes (h'' + 2Hc h' + k^2 h = TT source), inverse c2r FFTs.
 * Errors: STATE (pm_project not called for this step), CUDA. */
pm_status pm_solve(pm_ctx *ctx);

/* Particle update of step n (Eqs. kick, drift expanded to first order in
 * phi, psi, B, h neglected): CIC gather of the centred-difference gradients,
 * kick u_{n+1/2} = u_{n-1/2} + dtau_kick K, drift x_{n+1} = x_n + dtau_n V,
 * periodic wrap, then a counting sort of the particles by cell.
 * Advances the step index.  Errors: STATE (pm_solve not called), CUDA. */
pm_status pm_update(pm_ctx *ctx);

/* pm_project + pm_solve + pm_update.  With pm_step_graph(ctx, 1) the step's
 * launches are captured into one CUDA graph on a stream of the context and
 * the graph is launched on the context's stream (two executable graphs
 * alternate and are updated in place); called while the caller captures the
 * context's stream, the step is issued as plain launches into that capture.
 * Errors: as the three calls, CUDA (capture, instantiation, launch). */
pm_status pm_step(pm_ctx *ctx);

/* Graph-captured pm_step on (1) or off (0, the default).  Graph steps run
 * the same kernels in the same order as plain steps (the results differ only
 * through the order of particles inside a cell, which the counting sort
 * leaves open) and record no per-kernel timings (pm_get_timings reports the
 * plain steps only).  Errors: INVALID_ARG. */
pm_status pm_step_graph(pm_ctx *ctx, int32_t on);

/* Replace the particle state between steps without touching the fields,
 * the step index or the tensor state: pos, mom [n_part][3] f64 (host or
 * device) as in pm_set_particles; ids are reassigned to the row order.
 * Used to feed a running simulation from outside (e.g. host buffers every
 * step).  Errors: INVALID_ARG (NULL, NaN/Inf), STATE (no particles yet or
 * mid-step), CUDA. */
pm_status pm_put_particles(pm_ctx *ctx, const double *pos, const double *mom);

/* Current particle state in id order: pos [n_part][3] (box units, [0,1)),
 * mom [n_part][3] (u at half a step before the next step).  Either pointer
 * may be NULL to skip it.  Errors: INVALID_ARG, STATE, CUDA. */
pm_status pm_get_particles(pm_ctx *ctx, double *pos, double *mom);

/* Particle state in the mixed form's own precision (28 bytes a particle
 * instead of the 48 of two f64 triples), for I/O across the CPU-GPU link: the
 * cell index c = i + N (j + N k) of the vertex-centred mesh, the offsets
 * f in [0, 1) inside the cell (position x = (i + f_x) / N, ...) and the
 * momentum per unit mass u, as the mixed step stores them (the paper's
 * mixed-precision positions are cell plus offset; its Sec. 3.1 momentum). */
typedef struct {
    int32_t cell;
    float f[3];
    float u[3];
} pm_packed_particle;

/* pm_put_particles / pm_set_particles / pm_get_particles with n_part packed
 * records (host, pinned host or device memory; pinned and device memory are
 * read and written by the kernels in place).  Mixed-precision contexts only.
 * The records are taken as they are: no rounding, ids are the record order.
 * Errors: INVALID_ARG (NULL, an FP64 context, a cell outside [0, N^3), an
 * offset outside [0, 1), a non-finite offset or momentum), STATE (put: no
 * particles yet or mid-step), CUDA. */
pm_status pm_set_particles_packed(pm_ctx *ctx, const pm_packed_particle *p);
pm_status pm_put_particles_packed(pm_ctx *ctx, const pm_packed_particle *p);
pm_status pm_get_particles_packed(pm_ctx *ctx, pm_packed_particle *p);

/* Overlapped forms of pm_put_particles_packed / pm_get_particles_packed for a
 * loop that feeds every step from the host and reads every result back:
 * both return at once.  The records travel by copy engine on two streams of
 * the context, so an upload and a download run beside the steps on the
 * context's stream and beside each other.  put: the n_part records of p go to
 * a device staging buffer (after the previous put's records left it), and in
 * stream order with the steps they are checked, become the particle state
 * and are sorted by cell.  get: in stream order, the state in id order goes
 * to a second staging buffer (after the previous get's download left it),
 * then downloads into p.  p should be pinned host memory (pageable memory
 * makes the copies synchronous); a put's p must stay unchanged and a get's p
 * unread until pm_io_wait returns.  A bad record (as for
 * pm_put_particles_packed) is neutralised on the device and reported by
 * pm_io_wait, after which the context has no particles.  Staging takes 2 x 28
 * bytes a particle, allocated on first use.  Mixed contexts only.  Errors:
 * INVALID_ARG (NULL, FP64 context), STATE (no particles yet or mid-step), OOM,
 * CUDA. */
pm_status pm_put_particles_packed_async(pm_ctx *ctx, const pm_packed_particle *p);
pm_status pm_get_particles_packed_async(pm_ctx *ctx, pm_packed_particle *p);

/* Wait for the context's stream and both I/O streams; report a bad record of
 * a put since the previous wait (INVALID_ARG; the context then has no
 * particles).  Errors: INVALID_ARG, CUDA. */
pm_status pm_io_wait(pm_ctx *ctx);

/* One N^3 real field as f64 (see PM_FIELD_*), [z][y][x].  Errors: INVALID_ARG, STATE, CUDA. */
pm_status pm_get_field(pm_ctx *ctx, int field_id, double *dst);

/* One tensor-state array as interleaved complex f64 on the half spectrum
 * [kz][ky][kx], kx in [0, N/2], N*N*(N/2+1) complex values, in unnormalised
 * DFT units (sum_x f(x) e^{-i k.x}).  Polarisations: e1 perpendicular to k
 * from the axis with the smallest |n_i| (ties to the lowest axis),
 * e2 = khat x e1, e+ = (e1 e1 - e2 e2)/sqrt2, ex = (e1 e2 + e2 e1)/sqrt2. */
pm_status pm_get_tensor(pm_ctx *ctx, int which, double *dst);

/* Power spectrum of the CIC mass-density contrast delta = rho/omega_m - 1 of
 * the current particles: P(k_b) = mean |delta_k|^2 / N^6 over modes with
 * round(|n|) = b, for 1 <= b < nbins; bin 0 is left empty.  Host outputs
 * k[nbins] (mean |k| = 2 pi |n|), pk[nbins], nmodes[nbins].  Overwrites the
 * stored sources.  Errors: INVALID_ARG, STATE, CUDA. */
pm_status pm_power_spectrum(pm_ctx *ctx, int nbins, double *k, double *pk, int64_t *nmodes);

/* pm_power_spectrum without any device allocation.  The paper has no
 * counterpart; this exists for callers that cannot call cudaMalloc where they
 * want the diagnostic (code running under an allocator that forbids further
 * allocation, or an application whose device memory is entirely handed to its
 * own sub-allocator).  It needs no context.
 * d_pos: n_part x 3 f64 positions in box units, DEVICE memory of the current
 * device (host pointers are rejected with INVALID_ARG).  Computes the CIC
 * mass-density contrast on an n_mesh^3 mesh (mass omega_m / n_part per
 * particle) and the same binned P(k) as pm_power_spectrum into the HOST arrays
 * k, pk, nmodes [nbins]; enqueued on `stream` (NULL = default) and synchronised.
 * Limits: n_mesh of the form 2^a 3^b with a >= 3 and 8 <= n_mesh <= 64, and
 * 2 <= nbins <= 512; larger sizes return PM_ERR_UNSUPPORTED_SIZE.
 * Memory: all scratch (density, spectrum, bins, twiddle tables, about 4.3 MiB)
 * is one file-scope __device__ array that every GPU loading the library holds
 * until the process exits.  The first call on each device looks up the array's
 * device address (cudaGetSymbolAddress).  Every call ends by copying the bins to
 * the host and synchronising `stream`, so it cannot be recorded into a CUDA
 * graph: inside a stream capture it fails with PM_ERR_CUDA.  Every call uses the
 * same array, so calls that overlap on the GPU (on different streams or host
 * threads) race and must be serialised by the caller.  Device memory of another
 * GPU than the current one is rejected with INVALID_ARG.
 * Errors: INVALID_ARG, UNSUPPORTED_SIZE, CUDA. */
pm_status pm_power_spectrum_noalloc(const double *d_pos, int64_t n_part, int32_t n_mesh, double omega_m,
                                    int32_t nbins, double *k, double *pk, int64_t *nmodes, void *stream);

/* Step index (number of completed steps), a at that step, conformal time
 * since z_init.  Any pointer may be NULL. */
pm_status pm_get_time(pm_ctx *ctx, int32_t *step, double *a, double *tau);

/* Schedule arrays: a_n[n_steps+1], dtau[n_steps], a_half[n_steps] (host). */
pm_status pm_get_schedule(pm_ctx *ctx, double *a_n, double *dtau, double *a_half);

/* Mean stage timings in ms per step (see PM_T_*) over the steps completed
 * since the previous call (at most the last 64), n <= PM_T_COUNT; stages
 * without steps read 0.  Synchronises the stream, then starts a new window.
 * *launches (may be NULL) receives the number of library kernels launched
 * in that window. */
pm_status pm_get_timings(pm_ctx *ctx, double *ms, int n, int64_t *launches);

/* Shapes of the y and z column passes of the FFT.  Mixed-precision contexts
 * with N = 64, 128, 256 or 512 have three shapes per pass (points per thread,
 * lines per block):
 *   y pass: 0 = (32, 8), 1 = (16, 8), 2 = (8, 8);
 *   z pass: 0 = (16, 16), 1 = (8, 16), 2 = (16, 8).
 * Shape 0 of each pass is the default.  force_y / force_z in 0..2 select a
 * shape; -2 keeps the current one; -1 times the three shapes of that pass on
 * the context's own spectrum buffers (the 9 forward and 5 inverse line
 * transforms of a step; these buffers hold nothing between steps, they are
 * cleared first) and keeps the fastest.  Every shape computes the same transform in the same arithmetic
 * order.  *y_shape / *z_shape (may be NULL) receive the shapes in use.
 * Contexts without a choice (FP64, other N) keep shape 0 and return PM_OK.
 * Errors: INVALID_ARG (force_* outside -2..2), STATE, CUDA. */
pm_status pm_fft_shapes(pm_ctx *ctx, int32_t force_y, int32_t force_z, int32_t *y_shape, int32_t *z_shape);

/* Shape of the projection's shared-memory bins (Sec. 2.1, the particle-mesh
 * projection): the number of particle records one 8^3 vertex tile stages at
 * a time.  Shape 0: 960 records (FP32) / 640 (FP64), the default; shape 1:
 * 768 / 512.  Fewer records per chunk suit early, nearly uniform loads, more
 * suit clustered late loads (more tiles then fit in one chunk).  Both shapes
 * compute the same sums (only the order of additions inside a cell may
 * differ).  force 0 or 1 selects a shape; -2 keeps the current one; -1 times
 * the deposit of the context's current state with both shapes and keeps the
 * faster one (the context must hold particles and be between steps; the
 * trial deposits write into internal scratch, so the fields pm_get_field
 * returns do not change).  *shape (may be NULL) receives the shape in use.
 * Errors: INVALID_ARG (force outside -2..1), STATE, CUDA. */
pm_status pm_deposit_shape(pm_ctx *ctx, int32_t force, int32_t *shape);

/* Checkpoint: write / read the full state (config, step, particles,
 * phi_{n-1}, chi_{n-1}, phi_{n-2}, tensor state) to / from a host file.
 * pm_load requires a context created with the same config.
 * Errors: INVALID_ARG (bad path, config mismatch, corrupt file), STATE, CUDA. */
pm_status pm_save(pm_ctx *ctx, const char *path);
pm_status pm_load(pm_ctx *ctx, const char *path);

/* ------------------------------------------------------------------------
 * Batched ensemble of independent boxes (each its own n_mesh, n_part,
 * box_mpch and seed; all with the same n_steps, stepped in lockstep).  The
 * paper runs one box per job; stepping many boxes together keeps the GPU
 * busy when single boxes are small.  Each box is a full pm_ctx; an ensemble
 * step issues every box's pm_step on one of K streams and, with use_graph,
 * captures the whole step into one CUDA graph launched on the ensemble's own
 * stream.  The ensemble owns its streams (cfg.stream is ignored).
 * ------------------------------------------------------------------------ */
typedef struct pm_ensemble pm_ensemble;

/* Create nbox contexts from cfgs[nbox].  Errors: INVALID_ARG (n_steps differ),
 * UNSUPPORTED_SIZE, OOM, CUDA (the partially built ensemble is released). */
pm_status pm_ensemble_init(const pm_config *cfgs, int32_t nbox, pm_ensemble **out);
void pm_ensemble_destroy(pm_ensemble *e);
const char *pm_ensemble_last_error(const pm_ensemble *e);

/* The context of box `box`, for the single-box getters (pm_get_particles,
 * pm_get_field, pm_power_spectrum, ...).  Do not destroy it. */
pm_status pm_ensemble_box(pm_ensemble *e, int32_t box, pm_ctx **ctx);

/* pm_set_particles for one box; synchronises. */
pm_status pm_ensemble_set_particles(pm_ensemble *e, int32_t box, const double *pos, const double *mom);

/* One step of every box.  use_graph != 0 captures the step into a CUDA graph
 * (one launch); the first step after pm_ensemble_init or set_particles should
 * run with use_graph = 0 so that kernel attributes are set outside capture.
 * Asynchronous on the ensemble stream; pm_ensemble_sync waits for it. */
pm_status pm_ensemble_step(pm_ensemble *e, int32_t use_graph);
pm_status pm_ensemble_sync(pm_ensemble *e);

/* The ensemble's own stream (a cudaStream_t), on which every ensemble step is
 * launched and completes; callers may record events on it or make their
 * streams wait on it.  Owned by the ensemble. */
pm_status pm_ensemble_stream(pm_ensemble *e, void **stream);

/* Use n_streams streams (1 .. 32) from the next step on.  With more than one,
 * the boxes of the largest mesh run in order on the first stream and the
 * smaller boxes round-robin on the others. */
pm_status pm_ensemble_set_streams(pm_ensemble *e, int32_t n_streams);

/* Batched particle kernels (1) or per-box steps (0, the default).  Batched:
 * one projection launch and one gather + kick + drift launch each cover every
 * box of a precision, as a work list of (box, tile) items (a CTA finds its box
 * in a prefix table of the boxes' tile counts and reads that box's parameters
 * from the launch's parameter block); the transforms, Fourier solves and
 * sorts of the boxes run on the ensemble's streams in between.  Errors:
 * INVALID_ARG. */
pm_status pm_ensemble_set_batched(pm_ensemble *e, int32_t batched);

/* Current stream count and batched flag (either pointer may be NULL). */
pm_status pm_ensemble_get_mode(pm_ensemble *e, int32_t *n_streams, int32_t *batched);

/* Autotuner: first the FFT column-pass shapes and the projection's bin shape
 * of every distinct mesh size and precision (pm_fft_shapes and
 * pm_deposit_shape with -1 on the first box of that size, the choice copied
 * to the others; no box advances), then for each candidate number of streams
 * (1, 2, 4, 8, at most nbox), per-box and batched, one untimed and two timed
 * graph-captured ensemble steps, keeping the fastest; *n_streams receives the
 * stream count (pm_ensemble_get_mode reports the batched flag).  Each trial
 * advances every box by three steps. */
pm_status pm_ensemble_tune(pm_ensemble *e, int32_t *n_streams);

/* ------------------------------------------------------------------------
 * Learned sub-mesh force correction.  The paper has no learned component:
 * this is an optional addition to the Newtonian-mode step.  A 3^3 periodic
 * convolutional network (2 -> 16 -> 16 -> 16 -> 3 channels, ReLU between
 * layers, BF16 weights and activations, FP32 accumulation) maps
 *   x0 = delta = R / kappa,  x1 = phi N^2 / kappa,   kappa = 4piG Omega_m / a,
 * of a solved context to y (3 channels), and the next pm_update kicks every
 * particle with the extra force c = (kappa / N) y interpolated by CIC:
 *   u += dtau_kick * a_n * c(x_p)           (Newtonian mode).
 * Trained on targets y* = (R_2(F_2N) - F_N) N / kappa: the full-weighting
 * restriction of the force -grad phi of the same particles on a mesh twice
 * as fine, minus the force on the context's mesh (centred differences).
 *
 * Layouts (device memory): activations BF16 [cell][16] (cell = (z N + y) N + x,
 * channels beyond the used ones zero); targets and outputs FP32 [cell][8]
 * (channels 0..2 used); parameters FP32, per layer W [27][16 c_out][16 c_in]
 * with d = 9 (dz+1) + 3 (dy+1) + (dx+1), then b [16], padded entries zero
 * (pm_net_param_count() floats in all).  N must be a multiple of 8.
 * ------------------------------------------------------------------------ */
typedef struct pm_net pm_net;

enum { PM_NET_INPUT = 0, PM_NET_OUTPUT = 1, PM_NET_GRAD = 2 };

int64_t pm_net_param_count(void);

/* Network with buffers for an n_mesh^3 mesh, weights He-initialised from `seed`
 * (SplitMix64 + Box-Muller; last layer scaled by 0.1), biases zero.
 * Errors: UNSUPPORTED_SIZE (n_mesh not a multiple of 8 in [8, 1024]), OOM. */
pm_status pm_net_create(int32_t n_mesh, uint64_t seed, void *stream, pm_net **out);
void pm_net_destroy(pm_net *net);
const char *pm_net_last_error(const pm_net *net);

/* FP32 parameters in or out (host or device pointer); set also resets Adam. */
pm_status pm_net_set_params(pm_net *net, const float *params);
pm_status pm_net_get_params(pm_net *net, float *params);

/* Device address of an internal buffer: PM_NET_INPUT (BF16 [cell][16]),
 * PM_NET_OUTPUT (FP32 [cell][8]), PM_NET_GRAD (FP32 parameter gradient,
 * same layout as the parameters; accumulated by pm_net_backward, cleared by
 * pm_net_adam).  Owned by the network. */
pm_status pm_net_buffer(pm_net *net, int32_t which, void **ptr);

/* Normalisation (default 1, 1, 1): the inputs become s_delta x0 and s_phi x1,
 * the targets s_target y*, and the applied correction (kappa / N) y / s_target. */
pm_status pm_net_set_scales(pm_net *net, double s_delta, double s_phi, double s_target);
/* Inputs x0, x1 from a context after pm_solve (Newtonian mode, same n_mesh). */
pm_status pm_net_features(pm_net *net, pm_ctx *ctx);
/* Training target (FP32 [cell][8], device) from a solved context and a
 * solved context of the same particles on a mesh twice as fine, solved at
 * the same scale factor (same box, Omega_m, particle count and precision). */
pm_status pm_net_target(pm_net *net, pm_ctx *coarse, pm_ctx *fine, float *target);
/* Forward pass: input buffer -> output buffer. */
pm_status pm_net_forward(pm_net *net);
/* Forward, MSE loss against `target` (mean over cells and the 3 channels;
 * *loss receives it if non-NULL, which synchronises) and backward into the
 * gradient buffer. */
pm_status pm_net_backward(pm_net *net, const float *target, double *loss);
/* One Adam step (beta 0.9, 0.999, eps 1e-8) with learning rate lr. */
pm_status pm_net_adam(pm_net *net, float lr);
pm_status pm_net_train_step(pm_net *net, const float *target, float lr, double *loss);
/* Features + forward on a solved context, and attach the output as the
 * context's force correction for the following pm_update. */
pm_status pm_net_apply(pm_net *net, pm_ctx *ctx);
/* Attach (or with NULL detach) a force correction FP32 [cell][8] in force
 * units; every later pm_update kicks it in (factor a_n in the Newtonian mode,
 * E = sqrt(a_n^2 + u^2) otherwise).  Not owned by the context. */
pm_status pm_set_correction(pm_ctx *ctx, const float *corr);

/* The layer kernels on caller buffers (device pointers, stream as above):
 * y = act(conv(x, w) + bias) with x BF16 [n^3][16], w BF16 [27][16][16]
 * ([d][c_out][c_in]), bias FP32 [16] or NULL; c_out = 16 writes BF16
 * [n^3][16] (relu 0/1), c_out = 8 writes FP32 [n^3][8] (relu 0) from the first
 * 8 output channels of w.  The input gradient of a layer is this convolution
 * with w'[26 - d][c_in][c_out] = w[d][c_out][c_in].  Meshes with n % 16 == 0
 * run on the tcgen05 tensor cores (FP32 accumulate in tensor memory), others
 * on mma.sync; both accumulate in FP32 over the 27 offsets in order.
 * Errors: UNSUPPORTED_SIZE (n not a multiple of 8 in 8..1024), INVALID_ARG,
 * CUDA (launch); a device-side wait that runs out is reported by
 * pm_conv3d_check. */
pm_status pm_conv3d_forward(int32_t n, const void *x, const void *w, const float *bias, int32_t c_out, int32_t relu,
                            void *y, void *stream);
/* Synchronise `stream` and report whether a bounded device wait of the
 * tensor-core convolution (meshes with n % 16 == 0, in pm_conv3d_forward and
 * in the network calls) ran out since the previous check: PM_ERR_TIMEOUT
 * (the count is then cleared; the affected outputs hold NaN), else PM_OK.
 * The count is per device.  After a timeout a CTA issues no further work and
 * waits once more, bounded, for the MMAs it committed before it frees its
 * tensor memory.  If that second wait also runs out, the convolutions are
 * poisoned for the rest of the process: this call and every later
 * pm_conv3d_forward, pm_net_forward and pm_net_backward return PM_ERR_STATE.
 * Only the timeout in which no MMA was issued is exercised by the tests (it
 * leaves the calls usable).  Errors: CUDA. */
pm_status pm_conv3d_check(void *stream);
/* dw[d][c_out][c_in] += sum over cells of g[cell][c_out] x[cell + d][c_in]
 * (x, g BF16 [n^3][16]; dw FP32 [27][16][16], accumulated with atomics). */
pm_status pm_conv3d_backward_weight(int32_t n, const void *x, const void *g, float *dw, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* PM_H */
