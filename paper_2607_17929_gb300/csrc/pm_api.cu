// C ABI of libpm: context lifecycle, background schedule, step driver,
// host/device I/O and checkpoints.  See include/pm.h for the contract.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "pm_internal.cuh"


namespace pm {

namespace {

// ---------------------------------------------------------------------------
// Background (FP64, host).  Hc(a) = a H0 sqrt(Om a^-3 + OL) (Sec. 3.1: Hc is
// d ln a / d tau).  tau between two scale factors by 64-point Gauss-Legendre
// (nodes by Newton iteration on P_64), a at a given tau offset by Newton.
// ---------------------------------------------------------------------------
struct Background {
    double om, h0;
    double x[64], w[64];

    Background(double omega_m, double hubble0) : om(omega_m), h0(hubble0)
    {
        const int n = 64;
        for (int i = 0; i < n; i++) {
            double t = std::cos(M_PI * (i + 0.75) / (n + 0.5));
            double dpn = 1.0;
            for (int it = 0; it < 100; it++) {
                double pm1 = 1.0, pn = t;
                for (int k = 2; k <= n; k++) {
                    double pk = ((2 * k - 1) * t * pn - (k - 1) * pm1) / k;
                    pm1 = pn;
                    pn = pk;
                }
                dpn = n * (t * pn - pm1) / (t * t - 1.0);
                double step = pn / dpn;
                t -= step;
                if (std::fabs(step) < 1e-16) break;
            }
            double pm1 = 1.0, pn = t;
            for (int k = 2; k <= n; k++) {
                double pk = ((2 * k - 1) * t * pn - (k - 1) * pm1) / k;
                pm1 = pn;
                pn = pk;
            }
            dpn = n * (t * pn - pm1) / (t * t - 1.0);
            x[i] = t;
            w[i] = 2.0 / ((1.0 - t * t) * dpn * dpn);
        }
    }
    double hc(double a) const { return a * h0 * std::sqrt(om / (a * a * a) + (1.0 - om)); }
    double dtda(double a) const { return 1.0 / (a * hc(a)); }
    double tau(double a0, double a1) const
    {
        const double c = 0.5 * (a0 + a1), r = 0.5 * (a1 - a0);
        double s = 0.0;
        for (int i = 0; i < 64; i++) s += w[i] * dtda(c + r * x[i]);
        return r * s;
    }
    double a_at(double a0, double dt) const
    {
        double a = a0 * std::exp(dt * hc(a0));
        for (int it = 0; it < 60; it++) {
            double d = (tau(a0, a) - dt) / dtda(a);
            a -= d;
            if (std::fabs(d) <= 1e-17 * a) break;
        }
        return a;
    }
};

bool valid_n(int n)
{
    if (n < 8 || n > 1024 || n % 8) return false;
    int m = n;
    while (m % 2 == 0) m /= 2;
    while (m % 3 == 0) m /= 3;
    return m == 1;
}

pm_status fail(Ctx &c, pm_status st, const std::string &msg)
{
    c.err = msg;
    return st;
}

pm_status cuda_fail(Ctx &c, cudaError_t e, const char *where)
{
    c.err = std::string(where) + ": " + cudaGetErrorString(e);
    c.poisoned = true;
    return PM_ERR_CUDA;
}

#define CK(call)                                                          \
    do {                                                                  \
        cudaError_t e_ = (call);                                          \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, #call);            \
    } while (0)

#define CKL(where)                                                        \
    do {                                                                  \
        cudaError_t e_ = cudaGetLastError();                              \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, where);            \
    } while (0)

bool is_device_ptr(const void *p)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// An address the kernels can use for p: p itself for device memory, the mapped device address for
// pinned host memory (page-locked by cudaHostAlloc or cudaHostRegister: the kernels then read or
// write it across the CPU-GPU link, with no staging copy), NULL for pageable host memory.
template <class P> P *kernel_ptr(P *p)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return p;
    if (a.type == cudaMemoryTypeHost && a.devicePointer) return static_cast<P *>(a.devicePointer);
    return nullptr;
}

}  // namespace

StepScalars scalars(const Ctx &c, int k, bool bootstrap)
{
    const Background bg(c.cfg.omega_m, c.h0);
    StepScalars s{};
    const int ns = c.cfg.n_steps;
    const int kk = k < ns ? k : ns - 1;
    s.a = c.a_n[k];
    s.hc = bg.hc(s.a);
    const double dprev = k >= 1 ? c.dtau[k - 1] : c.dtau[0];
    const double dprev2 = k >= 2 ? c.dtau[k - 2] : c.dtau[0];
    s.newtonian = c.newtonian;
    s.bootstrap = bootstrap;
    s.c_phi_dt = (c.newtonian || bootstrap) ? 0.0 : 3.0 * s.hc / dprev;
    s.c_phi_h2 = c.newtonian ? 0.0 : 3.0 * s.hc * s.hc;
    s.inv_dtau_prev2 = 1.0 / dprev2;
    s.dtau_prev = dprev;
    s.full_hc = c.full_hc && !bootstrap && !c.newtonian;
    s.b_space = c.b_space;
    s.b_seed = (k == 0);
    s.b_decay = k >= 1 ? (c.a_n[k - 1] / s.a) * (c.a_n[k - 1] / s.a) : 1.0;
    s.dtau = c.dtau[kk];
    s.dtau_kick = 0.5 * (dprev + c.dtau[kk]);
    s.a_half = c.a_half[kk];
    s.hc_half = bg.hc(s.a_half);
    s.four_pi_g = c.four_pi_g;
    s.mass = c.mass;
    s.omega_m = c.cfg.omega_m;
    return s;
}

template <class T> void **src_ptrs(Ctx &c, void **p)
{
    for (int i = 0; i < 9; i++) p[i] = reinterpret_cast<T *>(c.src) + (size_t)i * c.nc;
    return p;
}
template <class T> void **spec_ptrs(Ctx &c, void **p)
{
    using C = typename Cplx<T>::type;
    for (int i = 0; i < 9; i++) p[i] = reinterpret_cast<C *>(c.spec) + (size_t)i * c.nh;
    return p;
}

namespace {

template <class T> pm_status do_project(Ctx &c, bool bootstrap)
{
    StepScalars s = scalars(c, c.step, bootstrap);
    launch_project<T>(c, s);
    CKL("project");
    return PM_OK;
}

}  // namespace

template <class T> pm_status do_solve(Ctx &c, bool bootstrap)
{
    StepScalars s = scalars(c, c.step, bootstrap);
    const bool full = !(c.newtonian || bootstrap);
    void *sp[9], *sr[9];
    spec_ptrs<T>(c, sp);
    src_ptrs<T>(c, sr);
    int nf = full ? 9 : 1;
    void *fin[9], *fout[9];
    for (int i = 0; i < 9; i++) {
        fin[i] = sr[i];
        fout[i] = sp[i];
    }
    if (full && s.b_space && !s.b_seed) {
        // B from Eq. spacespace: the T0i sources F are not needed, transform R and Sig only
        for (int i = 1; i < 6; i++) {
            fin[i] = sr[i + 3];
            fout[i] = sp[i + 3];
        }
        nf = 6;
    }
    fft_forward<T>(c, nf, fin, fout);
    CKL("fft_forward");
    launch_solve<T>(c, s);
    CKL("solve");
    c.mark(EV_SOLVE);
    // phi_n, B_x, B_y, B_z, chi_n from spectra 0..4
    void *outs[5] = {c.phi[c.iphi_new], reinterpret_cast<T *>(c.B), reinterpret_cast<T *>(c.B) + c.nc,
                     reinterpret_cast<T *>(c.B) + 2 * c.nc, c.chi};
    fft_inverse<T>(c, full ? 5 : 1, sp, outs);
    CKL("fft_inverse");
    if (!full) {
        CK(cudaMemsetAsync(c.chi, 0, sizeof(T) * c.nc, c.stream));
        CK(cudaMemsetAsync(c.B, 0, sizeof(T) * 3 * c.nc, c.stream));
    }
    return PM_OK;
}

template pm_status do_solve<float>(Ctx &, bool);
template pm_status do_solve<double>(Ctx &, bool);

namespace {

template <class T> pm_status do_update(Ctx &c)
{
    StepScalars s = scalars(c, c.step, false);
    launch_corr_kick<T>(c, s);
    CKL("corr_kick");
    launch_kick_drift<T>(c, s);
    CKL("kick_drift");
    c.mark(EV_KICK);
    launch_sort<T>(c);
    CKL("sort");
    return PM_OK;
}

}  // namespace

// rotate the phi ring after step n: phi_{n-1} -> phi_{n-2}, phi_n -> phi_{n-1}
void rotate(Ctx &c)
{
    int old2 = c.iphi_prev2;
    c.iphi_prev2 = c.iphi_prev;
    c.iphi_prev = c.iphi_new;
    c.iphi_new = old2;
}

namespace {

template <class T>
pm_status set_particles_t(Ctx &c, const double *pos, const double *mom, bool bootstrap,
                          const pm_packed_particle *packed = nullptr)
{
    if (bootstrap) {
        c.have_particles = false;
        c.stage = 0;
    }
    CK(cudaMemsetAsync(c.count, 0, sizeof(int32_t) * c.nc, c.stream));
    const double *kpos = kernel_ptr(pos), *kmom = kernel_ptr(mom);
    int *dflag = reinterpret_cast<int *>(c.dscal + 4);
    CK(cudaMemsetAsync(dflag, 0, sizeof(int), c.stream));
    if constexpr (sizeof(T) == 4) {
        if (packed) {
            const pm_packed_particle *kp = kernel_ptr(packed);
            if (kp) {
                launch_load_packed(c, kp, 0, c.np, dflag);   // device or pinned host records, read in place
                CKL("load_packed");
            } else {
                auto *st = reinterpret_cast<pm_packed_particle *>(c.stage_buf);
                const int64_t chunk = c.stage_elems * (int64_t)sizeof(double) / (int64_t)sizeof(pm_packed_particle);
                for (int64_t f = 0; f < c.np; f += chunk) {
                    const int64_t n = std::min(chunk, c.np - f);
                    CK(cudaMemcpyAsync(st, packed + f, sizeof(pm_packed_particle) * n, cudaMemcpyHostToDevice,
                                       c.stream));
                    launch_load_packed(c, st, f, n, dflag);
                    CKL("load_packed");
                }
            }
        }
    }
    if (packed) {
        // loaded above
    } else if (kpos && kmom) {
        // device or pinned host arrays: one pass reads them, checks them and builds the records
        launch_load_particles<T>(c, kpos, kmom, 0, c.np, dflag);
        CKL("load");
    } else {
        double *st = reinterpret_cast<double *>(c.stage_buf);
        const int64_t chunk = c.stage_elems / 6;
        for (int64_t f = 0; f < c.np; f += chunk) {
            const int64_t n = std::min(chunk, c.np - f);
            CK(cudaMemcpyAsync(st, pos + 3 * f, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, c.stream));
            CK(cudaMemcpyAsync(st + 3 * chunk, mom + 3 * f, sizeof(double) * 3 * n, cudaMemcpyHostToDevice,
                               c.stream));
            launch_load_particles<T>(c, st, st + 3 * chunk, f, n, dflag);
            CKL("load");
        }
    }
    int hflag = 0;
    CK(cudaMemcpyAsync(&hflag, dflag, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
    CK(cudaStreamSynchronize(c.stream));
    if (hflag) {
        if (!bootstrap) c.have_particles = false;  // the previous state was overwritten
        return fail(c, PM_ERR_INVALID_ARG, packed ? "packed record with a cell out of range, an offset outside [0, 1) "
                                                    "or a non-finite value"
                                                  : "non-finite position or momentum");
    }
    launch_sort<T>(c);
    CKL("sort");
    if (!bootstrap) return PM_OK;
    // bootstrap: phi_{-1} = chi_{-1} = 0 in the weights, quasi-static solve
    CK(cudaMemsetAsync(c.phi[c.iphi_prev], 0, sizeof(T) * c.nc, c.stream));
    CK(cudaMemsetAsync(c.chi, 0, sizeof(T) * c.nc, c.stream));
    CK(cudaMemsetAsync(c.tens, 0, sizeof(typename Cplx<T>::type) * 4 * c.nh, c.stream));
    if (c.bstate) CK(cudaMemsetAsync(c.bstate, 0, sizeof(typename Cplx<T>::type) * 3 * c.nh, c.stream));
    CK(cudaMemsetAsync(c.dscal, 0, sizeof(double) * 8, c.stream));
    c.step = 0;
    pm_status st = do_project<T>(c, true);
    if (st) return st;
    st = do_solve<T>(c, true);
    if (st) return st;
    // phi_{-1} becomes both phi_{n-1} and phi_{n-2} of step 0; chi_{-1} = 0
    rotate(c);
    CK(cudaMemcpyAsync(c.phi[c.iphi_prev2], c.phi[c.iphi_prev], sizeof(T) * c.nc, cudaMemcpyDeviceToDevice,
                       c.stream));
    CK(cudaMemcpyAsync(c.dscal + 1 + c.iphi_prev2, c.dscal + 1 + c.iphi_prev, sizeof(double),
                       cudaMemcpyDeviceToDevice, c.stream));
    CK(cudaMemsetAsync(c.chi, 0, sizeof(T) * c.nc, c.stream));
    c.have_particles = true;
    c.stage = 0;
    return PM_OK;
}

pm_status get_packed_t(Ctx &c, pm_packed_particle *out)
{
    launch_store_particles_scatter<float>(c, nullptr, nullptr);   // records in id order
    CKL("unpermute");
    pm_packed_particle *kp = kernel_ptr(out);
    if (kp) {
        launch_store_packed(c, kp, 0, c.np);
        CKL("store_packed");
        if (!is_device_ptr(out)) CK(cudaStreamSynchronize(c.stream));
        return PM_OK;
    }
    auto *st = reinterpret_cast<pm_packed_particle *>(c.stage_buf);
    const int64_t chunk = c.stage_elems * (int64_t)sizeof(double) / (int64_t)sizeof(pm_packed_particle);
    for (int64_t f = 0; f < c.np; f += chunk) {
        const int64_t n = std::min(chunk, c.np - f);
        launch_store_packed(c, st, f, n);
        CKL("store_packed");
        CK(cudaMemcpyAsync(out + f, st, sizeof(pm_packed_particle) * n, cudaMemcpyDeviceToHost, c.stream));
        CK(cudaStreamSynchronize(c.stream));
    }
    return PM_OK;
}

template <class T> pm_status get_particles_t(Ctx &c, double *pos, double *mom)
{
    launch_store_particles_scatter<T>(c, pos, mom);
    CKL("unpermute");
    double *kpos = pos ? kernel_ptr(pos) : nullptr, *kmom = mom ? kernel_ptr(mom) : nullptr;
    if ((!pos || kpos) && (!mom || kmom)) {
        // device or pinned host arrays: the kernel writes them directly
        launch_store_particles<T>(c, kpos, kmom, 0, c.np);
        CKL("store");
        if (!is_device_ptr(pos ? (const void *)pos : (const void *)mom)) CK(cudaStreamSynchronize(c.stream));
        return PM_OK;
    }
    double *st = reinterpret_cast<double *>(c.stage_buf);
    const int64_t chunk = c.stage_elems / 6;
    for (int64_t f = 0; f < c.np; f += chunk) {
        const int64_t n = std::min(chunk, c.np - f);
        launch_store_particles<T>(c, pos ? st : nullptr, mom ? st + 3 * chunk : nullptr, f, n);
        CKL("store");
        if (pos) CK(cudaMemcpyAsync(pos + 3 * f, st, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, c.stream));
        if (mom)
            CK(cudaMemcpyAsync(mom + 3 * f, st + 3 * chunk, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost,
                               c.stream));
        CK(cudaStreamSynchronize(c.stream));
    }
    return PM_OK;
}

// copy n values of type T at d_src (device) into dst (host or device) as f64
template <class T> pm_status export_f64(Ctx &c, const void *d_src, double *dst, int64_t n)
{
    if (is_device_ptr(dst)) {
        launch_to_f64<T>(c, d_src, dst, n);
        CKL("to_f64");
        return PM_OK;
    }
    double *st = reinterpret_cast<double *>(c.stage_buf);
    for (int64_t f = 0; f < n; f += c.stage_elems) {
        const int64_t m = std::min(c.stage_elems, n - f);
        launch_to_f64<T>(c, reinterpret_cast<const T *>(d_src) + f, st, m);
        CKL("to_f64");
        CK(cudaMemcpyAsync(dst + f, st, sizeof(double) * m, cudaMemcpyDeviceToHost, c.stream));
        CK(cudaStreamSynchronize(c.stream));
    }
    return PM_OK;
}

template <class T> pm_status get_field_t(Ctx &c, int id, double *dst)
{
    const void *src = nullptr;
    if (id == PM_FIELD_PHI) src = c.phi[c.stage == 2 ? c.iphi_new : c.iphi_prev];
    else if (id == PM_FIELD_CHI) src = c.chi;
    else if (id >= PM_FIELD_BX && id <= PM_FIELD_BZ) src = reinterpret_cast<T *>(c.B) + (id - PM_FIELD_BX) * c.nc;
    else src = reinterpret_cast<T *>(c.src) + (id - PM_FIELD_R) * c.nc;
    return export_f64<T>(c, src, dst, c.nc);
}

template <class T> pm_status get_tensor_t(Ctx &c, int which, double *dst)
{
    using C = typename Cplx<T>::type;
    return export_f64<T>(c, reinterpret_cast<C *>(c.tens) + (size_t)which * c.nh, dst, 2 * c.nh);
}

template <class T> pm_status power_t(Ctx &c, int nbins, double *k, double *pk, int64_t *nm)
{
    void *sr[9], *sp[9];
    src_ptrs<T>(c, sr);
    spec_ptrs<T>(c, sp);
    launch_density<T>(c, sr[0]);
    CKL("density");
    fft_forward<T>(c, 1, sr, sp);
    CKL("fft");
    double *acc = reinterpret_cast<double *>(c.stage_buf);
    CK(cudaMemsetAsync(acc, 0, sizeof(double) * 3 * nbins, c.stream));
    launch_pk_bin<T>(c, sp[0], nbins, acc);
    CKL("pk_bin");
    std::vector<double> h(3 * nbins);
    CK(cudaMemcpyAsync(h.data(), acc, sizeof(double) * 3 * nbins, cudaMemcpyDeviceToHost, c.stream));
    CK(cudaStreamSynchronize(c.stream));
    for (int b = 0; b < nbins; b++) {
        const double cnt = h[2 * nbins + b];
        pk[b] = cnt > 0 ? h[b] / cnt : 0.0;
        k[b] = cnt > 0 ? h[nbins + b] / cnt : 0.0;
        nm[b] = (int64_t)std::llround(cnt);
    }
    return PM_OK;
}

// ---------------------------------------------------------------------------
// checkpoint format: header | particles (native records, sorted) | phi ring (3)
// | chi | tensor state | f64 scalars.  All device data copied through the host.
// ---------------------------------------------------------------------------
struct CkptHeader {
    char magic[8];
    int32_t version;
    int32_t n_mesh, n_steps, precision;
    uint32_t flags;
    int64_t n_part;
    double box, om, zi, zf;
    int32_t step, cur, ip2, ip1, ipn;
    int32_t pad;
    uint64_t payload_sum;
};

uint64_t fnv1a(const unsigned char *p, size_t n, uint64_t h)
{
    for (size_t i = 0; i < n; i++) {
        h ^= p[i];
        h *= 1099511628211ull;
    }
    return h;
}

struct Blob {
    void *dev;
    size_t bytes;
};

std::vector<Blob> state_blobs(Ctx &c)
{
    const size_t ts = c.mixed ? 4 : 8;
    const size_t ps = c.mixed ? sizeof(Particle<float>) : sizeof(Particle<double>);
    std::vector<Blob> b;
    b.push_back({c.part[c.cur], ps * (size_t)c.np});
    for (int i = 0; i < 3; i++) b.push_back({c.phi[i], ts * (size_t)c.nc});
    b.push_back({c.chi, ts * (size_t)c.nc});
    b.push_back({c.tens, 2 * ts * 4 * (size_t)c.nh});
    if (c.bstate) b.push_back({c.bstate, 2 * ts * 3 * (size_t)c.nh});
    b.push_back({c.dscal, sizeof(double) * 8});
    return b;
}

pm_status save_impl(Ctx &c, const char *path)
{
    FILE *f = std::fopen(path, "wb");
    if (!f) return fail(c, PM_ERR_INVALID_ARG, std::string("pm_save: cannot open ") + path);
    CkptHeader h{};
    std::memcpy(h.magic, "PMCKPT1", 8);
    h.version = 1;
    h.n_mesh = c.cfg.n_mesh;
    h.n_steps = c.cfg.n_steps;
    h.precision = c.cfg.precision;
    h.flags = c.cfg.flags;
    h.n_part = c.np;
    h.box = c.cfg.box_mpch;
    h.om = c.cfg.omega_m;
    h.zi = c.cfg.z_init;
    h.zf = c.cfg.z_final;
    h.step = c.step;
    h.cur = 0;
    h.ip2 = c.iphi_prev2;
    h.ip1 = c.iphi_prev;
    h.ipn = c.iphi_new;
    std::fwrite(&h, sizeof(h), 1, f);
    uint64_t sum = 1469598103934665603ull;
    std::vector<unsigned char> host;
    bool ok = true;
    for (const Blob &b : state_blobs(c)) {
        host.resize(b.bytes);
        cudaError_t e = cudaMemcpyAsync(host.data(), b.dev, b.bytes, cudaMemcpyDeviceToHost, c.stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
        if (e != cudaSuccess) {
            std::fclose(f);
            return cuda_fail(c, e, "pm_save");
        }
        sum = fnv1a(host.data(), b.bytes, sum);
        ok = ok && std::fwrite(host.data(), 1, b.bytes, f) == b.bytes;
    }
    h.payload_sum = sum;
    std::fseek(f, 0, SEEK_SET);
    ok = ok && std::fwrite(&h, sizeof(h), 1, f) == 1;
    ok = (std::fclose(f) == 0) && ok;
    if (!ok) return fail(c, PM_ERR_INVALID_ARG, "pm_save: write failed");
    return PM_OK;
}

template <class T> pm_status load_impl(Ctx &c, const char *path)
{
    FILE *f = std::fopen(path, "rb");
    if (!f) return fail(c, PM_ERR_INVALID_ARG, std::string("pm_load: cannot open ") + path);
    CkptHeader h{};
    if (std::fread(&h, sizeof(h), 1, f) != 1 || std::memcmp(h.magic, "PMCKPT1", 8) != 0 || h.version != 1) {
        std::fclose(f);
        return fail(c, PM_ERR_INVALID_ARG, "pm_load: not a checkpoint");
    }
    if (h.n_mesh != c.cfg.n_mesh || h.n_steps != c.cfg.n_steps || h.precision != c.cfg.precision ||
        h.flags != c.cfg.flags || h.n_part != c.np || h.box != c.cfg.box_mpch || h.om != c.cfg.omega_m ||
        h.zi != c.cfg.z_init || h.zf != c.cfg.z_final || h.step < 0 || h.step > c.cfg.n_steps) {
        std::fclose(f);
        return fail(c, PM_ERR_INVALID_ARG, "pm_load: checkpoint config differs from the context");
    }
    uint64_t sum = 1469598103934665603ull;
    std::vector<std::vector<unsigned char>> data;
    for (const Blob &b : state_blobs(c)) {
        data.emplace_back(b.bytes);
        if (std::fread(data.back().data(), 1, b.bytes, f) != b.bytes) {
            std::fclose(f);
            return fail(c, PM_ERR_INVALID_ARG, "pm_load: truncated checkpoint");
        }
        sum = fnv1a(data.back().data(), b.bytes, sum);
    }
    std::fclose(f);
    if (sum != h.payload_sum) return fail(c, PM_ERR_INVALID_ARG, "pm_load: checksum mismatch (corrupt file)");
    c.cur = 0;
    c.iphi_prev2 = h.ip2;
    c.iphi_prev = h.ip1;
    c.iphi_new = h.ipn;
    std::vector<Blob> blobs = state_blobs(c);
    for (size_t i = 0; i < blobs.size(); i++)
        CK(cudaMemcpyAsync(blobs[i].dev, data[i].data(), blobs[i].bytes, cudaMemcpyHostToDevice, c.stream));
    CK(cudaStreamSynchronize(c.stream));
    // the cell index (count / start) is rebuilt by the caller (recount)
    CK(cudaMemsetAsync(c.count, 0, sizeof(int32_t) * c.nc, c.stream));
    c.step = h.step;
    c.stage = 0;
    c.have_particles = true;
    return PM_OK;
}

}  // namespace
}  // namespace pm

using namespace pm;

namespace pm {
template <class T> __global__ void k_count_cells(const Particle<T> *part, int64_t np, int32_t *count)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < np) atomicAdd(&count[part[i].cell], 1);
}
template <class T> pm_status recount(Ctx &c)
{
    k_count_cells<T><<<(unsigned)((c.np + 255) / 256), 256, 0, c.stream>>>(
        reinterpret_cast<const Particle<T> *>(c.part[c.cur]), c.np, c.count);
    CKL("count");
    launch_sort<T>(c);
    CKL("sort");
    return PM_OK;
}
}  // namespace pm

#define PM_DISPATCH(ctx, fn, ...) ((ctx)->c.mixed ? fn<float>(__VA_ARGS__) : fn<double>(__VA_ARGS__))

static pm_status guard(pm_ctx *ctx)
{
    if (!ctx) return PM_ERR_INVALID_ARG;
    if (ctx->c.poisoned) {
        ctx->c.err = "context poisoned by an earlier CUDA error";
        return PM_ERR_STATE;
    }
    cudaSetDevice(ctx->c.device);
    ctx->c.err.clear();
    return PM_OK;
}

// streams, events and staging buffers of the overlapped packed I/O, made on first use
static pm_status io_setup(Ctx &c)
{
    if (c.io_up) return PM_OK;
    const size_t bytes = sizeof(pm_packed_particle) * (size_t)c.np;
    bool ok = cudaMalloc(&c.in_stage, bytes) == cudaSuccess && cudaMalloc(&c.out_stage, bytes) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        if (c.in_stage) cudaFree(c.in_stage);
        c.in_stage = c.out_stage = nullptr;
        return fail(c, PM_ERR_OOM, "particle I/O staging buffers");
    }
    ok = cudaStreamCreateWithFlags(&c.io_up, cudaStreamNonBlocking) == cudaSuccess &&
         cudaStreamCreateWithFlags(&c.io_down, cudaStreamNonBlocking) == cudaSuccess;
    for (cudaEvent_t *e : {&c.ev_in_ready, &c.ev_in_free, &c.ev_out_ready, &c.ev_out_free})
        ok = ok && cudaEventCreateWithFlags(e, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) return cuda_fail(c, cudaGetLastError(), "particle I/O streams");
    return PM_OK;
}

static void io_release(Ctx &c)
{
    if (c.io_up) cudaStreamSynchronize(c.io_up);
    if (c.io_down) cudaStreamSynchronize(c.io_down);
    for (cudaEvent_t e : {c.ev_in_ready, c.ev_in_free, c.ev_out_ready, c.ev_out_free})
        if (e) cudaEventDestroy(e);
    if (c.io_up) cudaStreamDestroy(c.io_up);
    if (c.io_down) cudaStreamDestroy(c.io_down);
    if (c.in_stage) cudaFree(c.in_stage);
    if (c.out_stage) cudaFree(c.out_stage);
}

extern "C" {

pm_status pm_init(const pm_config *cfg, pm_ctx **out)
{
    if (!cfg || !out) return PM_ERR_INVALID_ARG;
    *out = nullptr;
    if (!valid_n(cfg->n_mesh)) return PM_ERR_UNSUPPORTED_SIZE;
    if (cfg->n_steps < 1 || cfg->n_part < 1 || cfg->n_part >= (int64_t)1 << 31 || !(cfg->box_mpch > 0) ||
        !(cfg->omega_m > 0 && cfg->omega_m <= 1) || !(cfg->z_init > cfg->z_final) || !(cfg->z_final > -1) ||
        (cfg->precision != PM_FP64 && cfg->precision != PM_MIXED) || (cfg->flags & ~(PM_NEWTONIAN | PM_FULL_HC | PM_B_SPACESPACE)))
        return PM_ERR_INVALID_ARG;
    pm_ctx *ctx = new (std::nothrow) pm_ctx();
    if (!ctx) return PM_ERR_OOM;
    Ctx &c = ctx->c;
    c.cfg = *cfg;
    c.stream = reinterpret_cast<cudaStream_t>(cfg->stream);
    if (cudaGetDevice(&c.device) != cudaSuccess) {
        cudaGetLastError();
        delete ctx;
        return PM_ERR_CUDA;
    }
    c.N = cfg->n_mesh;
    c.nc = (int64_t)c.N * c.N * c.N;
    c.nh = (int64_t)c.N * c.N * (c.N / 2 + 1);
    c.np = cfg->n_part;
    c.mixed = cfg->precision == PM_MIXED;
    c.newtonian = (cfg->flags & PM_NEWTONIAN) != 0;
    c.full_hc = !c.newtonian && (cfg->flags & PM_FULL_HC) != 0;
    c.b_space = !c.newtonian && (cfg->flags & PM_B_SPACESPACE) != 0;
    c.h0 = cfg->box_mpch / 2997.92458;
    c.four_pi_g = 1.5 * c.h0 * c.h0;
    c.mass = cfg->omega_m / (double)c.np;
    c.plan = make_plan(c.N);
    // schedule
    {
        const Background bg(cfg->omega_m, c.h0);
        const int ns = cfg->n_steps;
        const double ai = 1.0 / (1.0 + cfg->z_init), af = 1.0 / (1.0 + cfg->z_final);
        c.a_n.resize(ns + 1);
        c.dtau.resize(ns);
        c.a_half.resize(ns);
        for (int n = 0; n <= ns; n++) c.a_n[n] = ai * std::pow(af / ai, (double)n / ns);
        for (int n = 0; n < ns; n++) {
            c.dtau[n] = bg.tau(c.a_n[n], c.a_n[n + 1]);
            c.a_half[n] = bg.a_at(c.a_n[n], 0.5 * c.dtau[n]);
        }
    }
    const size_t ts = c.mixed ? 4 : 8;
    const size_t ps = c.mixed ? sizeof(Particle<float>) : sizeof(Particle<double>);
    c.nblocksum = (c.nc + 4095) / 4096;
    c.stage_elems = std::min<int64_t>(std::max<int64_t>(6 * c.np, 2 * c.nh), (int64_t)6 << 22);
    c.stage_elems = std::max<int64_t>(c.stage_elems, 3 * 1024);
    struct A {
        void **p;
        size_t bytes;
    } allocs[] = {
        {&c.part[0], ps * (size_t)c.np},
        {&c.part[1], ps * (size_t)c.np},
        {(void **)&c.count, sizeof(int32_t) * (size_t)c.nc},
        {(void **)&c.start, sizeof(int32_t) * ((size_t)c.nc + 1)},
        {(void **)&c.blocksum, sizeof(int32_t) * (size_t)c.nblocksum},
        {&c.phi[0], ts * (size_t)c.nc},
        {&c.phi[1], ts * (size_t)c.nc},
        {&c.phi[2], ts * (size_t)c.nc},
        {&c.chi, ts * (size_t)c.nc},
        {&c.B, 3 * ts * (size_t)c.nc},
        {&c.src, 9 * ts * (size_t)c.nc},
        {&c.spec, 9 * 2 * ts * (size_t)c.nh},
        {&c.tens, 4 * 2 * ts * (size_t)c.nh},
        {&c.ktab, ts * (size_t)c.N},
        {&c.tw, 2 * ts * (size_t)c.N},
        {&c.tw2, 2 * ts * (size_t)(2 * c.N + 64)},
        {(void **)&c.dscal, sizeof(double) * (8 + 1024)},
        {&c.stage_buf, sizeof(double) * (size_t)c.stage_elems},
    };
    // PM_TEST_FAIL_ALLOC=k (test hook): the k-th device allocation of this call reports failure, to
    // exercise the clean-up path without exhausting the device
    const char *fail_env = std::getenv("PM_TEST_FAIL_ALLOC");
    const int fail_at = fail_env ? std::atoi(fail_env) : 0;
    int nalloc = 0;
    for (const A &a : allocs) {
        if (++nalloc == fail_at || cudaMalloc(a.p, a.bytes) != cudaSuccess) {
            cudaGetLastError();
            pm_destroy(ctx);
            return PM_ERR_OOM;
        }
    }
    if (c.b_space && cudaMalloc(&c.bstate, 3 * 2 * ts * (size_t)c.nh) != cudaSuccess) {
        cudaGetLastError();
        c.bstate = nullptr;
        pm_destroy(ctx);
        return PM_ERR_OOM;
    }
    // tables: ktilde(i) = 2N sin(pi n_i / N), twiddles exp(-2 pi i k / N) (long double on the host)
    {
        std::vector<double> kt(c.N), tw(2 * c.N);
        const long double pi = 3.141592653589793238462643383279502884L;
        for (int i = 0; i < c.N; i++) {
            const int m = i <= c.N / 2 ? i : i - c.N;
            kt[i] = (double)(2.0L * c.N * sinl(pi * m / c.N));
            tw[2 * i] = (double)cosl(2.0L * pi * i / c.N);
            tw[2 * i + 1] = (double)(-sinl(2.0L * pi * i / c.N));
        }
        std::vector<double> tw2;
        fast_twiddles(c.N, tw2);
        if (tw2.size() > 2 * (size_t)(2 * c.N + 64)) tw2.resize(2 * (size_t)(2 * c.N + 64));
        if (c.mixed) {
            std::vector<float> tw2f(tw2.begin(), tw2.end());
            if (!tw2f.empty()) cudaMemcpy(c.tw2, tw2f.data(), sizeof(float) * tw2f.size(), cudaMemcpyHostToDevice);
        } else if (!tw2.empty()) {
            cudaMemcpy(c.tw2, tw2.data(), sizeof(double) * tw2.size(), cudaMemcpyHostToDevice);
        }
        if (c.mixed) {
            std::vector<float> ktf(kt.begin(), kt.end()), twf(tw.begin(), tw.end());
            for (int i = 0; i < c.N; i++) {
                const int m = i <= c.N / 2 ? i : i - c.N;
                ktf[i] = (float)(2.0L * c.N * sinl(pi * m / c.N));
                twf[2 * i] = (float)cosl(2.0L * pi * i / c.N);
                twf[2 * i + 1] = (float)(-sinl(2.0L * pi * i / c.N));
            }
            cudaMemcpy(c.ktab, ktf.data(), sizeof(float) * c.N, cudaMemcpyHostToDevice);
            cudaMemcpy(c.tw, twf.data(), sizeof(float) * 2 * c.N, cudaMemcpyHostToDevice);
        } else {
            cudaMemcpy(c.ktab, kt.data(), sizeof(double) * c.N, cudaMemcpyHostToDevice);
            cudaMemcpy(c.tw, tw.data(), sizeof(double) * 2 * c.N, cudaMemcpyHostToDevice);
        }
    }
    cudaMemset(c.dscal, 0, sizeof(double) * (8 + 1024));
    cudaMemset(c.phi[0], 0, ts * c.nc);
    cudaMemset(c.phi[1], 0, ts * c.nc);
    cudaMemset(c.phi[2], 0, ts * c.nc);
    cudaMemset(c.chi, 0, ts * c.nc);
    cudaMemset(c.B, 0, 3 * ts * c.nc);
    cudaMemset(c.tens, 0, 4 * 2 * ts * c.nh);
    if (c.bstate) cudaMemset(c.bstate, 0, 3 * 2 * ts * c.nh);
    cudaMemset(c.count, 0, sizeof(int32_t) * c.nc);
    for (auto &row : c.evr)
        for (auto &e : row) cudaEventCreate(&e);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        pm_destroy(ctx);
        return PM_ERR_CUDA;
    }
    *out = ctx;
    return PM_OK;
}

void pm_destroy(pm_ctx *ctx)
{
    if (!ctx) return;
    Ctx &c = ctx->c;
    cudaSetDevice(c.device);
    if (c.stream) cudaStreamSynchronize(c.stream);
    else cudaDeviceSynchronize();
    void *ps[] = {c.part[0], c.part[1], c.count, c.start, c.blocksum, c.phi[0], c.phi[1], c.phi[2], c.chi, c.B,
                  c.src, c.spec, c.tens, c.ktab, c.tw, c.tw2, c.dscal, c.stage_buf, c.bstate};
    for (void *p : ps)
        if (p) cudaFree(p);
    for (auto &row : c.evr)
        for (auto &e : row)
            if (e) cudaEventDestroy(e);
    for (cudaGraphExec_t x : c.gexec)
        if (x) cudaGraphExecDestroy(x);
    if (c.gstream) cudaStreamDestroy(c.gstream);
    io_release(c);
    cudaGetLastError();
    delete ctx;
}

const char *pm_last_error(const pm_ctx *ctx)
{
    return ctx ? ctx->c.err.c_str() : "null context";
}

pm_status pm_set_particles(pm_ctx *ctx, const double *pos, const double *mom)
{
    pm_status g = guard(ctx);
    if (g) return g;
    Ctx &c = ctx->c;
    if (!pos || !mom) return fail(c, PM_ERR_INVALID_ARG, "pm_set_particles: NULL array");
    return PM_DISPATCH(ctx, set_particles_t, c, pos, mom, true);
}

pm_status pm_put_particles(pm_ctx *ctx, const double *pos, const double *mom)
{
    pm_status g = guard(ctx);
    if (g) return g;
    Ctx &c = ctx->c;
    if (!pos || !mom) return fail(c, PM_ERR_INVALID_ARG, "pm_put_particles: NULL array");
    if (!c.have_particles || c.stage != 0) return fail(c, PM_ERR_STATE, "pm_put_particles: not between steps");
    return PM_DISPATCH(ctx, set_particles_t, c, pos, mom, false);
}

pm_status pm_set_particles_packed(pm_ctx *ctx, const pm_packed_particle *p)
{
    pm_status g = guard(ctx);
    if (g) return g;
    Ctx &c = ctx->c;
    if (!p) return fail(c, PM_ERR_INVALID_ARG, "pm_set_particles_packed: NULL array");
    if (!c.mixed) return fail(c, PM_ERR_INVALID_ARG, "pm_set_particles_packed: packed records need a mixed context");
    return set_particles_t<float>(c, nullptr, nullptr, true, p);
}

pm_status pm_put_particles_packed(pm_ctx *ctx, const pm_packed_particle *p)
{
    pm_status g = guard(ctx);
    if (g) return g;
    Ctx &c = ctx->c;
    if (!p) return fail(c, PM_ERR_INVALID_ARG, "pm_put_particles_packed: NULL array");
    if (!c.mixed) return fail(c, PM_ERR_INVALID_ARG, "pm_put_particles_packed: packed records need a mixed context");
    if (!c.have_particles || c.stage != 0) return fail(c, PM_ERR_STATE, "pm_put_particles_packed: not between steps");
    return set_particles_t<float>(c, nullptr, nullptr, false, p);
}

pm_status pm_get_particles_packed(pm_ctx *ctx, pm_packed_particle *p)
{
    pm_status g = guard(ctx);
    if (g) return g;
    Ctx &c = ctx->c;
    if (!p) return fail(c, PM_ERR_INVALID_ARG, "pm_get_particles_packed: NULL array");
    if (!c.mixed) return fail(c, PM_ERR_INVALID_ARG, "pm_get_particles_packed: packed records need a mixed context");
    if (!c.have_particles) return fail(c, PM_ERR_STATE, "pm_get_particles_packed: no particles");
    return get_packed_t(c, p);
}

pm_status pm_put_particles_packed_async(pm_ctx *ctx, const pm_packed_particle *p)
{
    pm_status g = guard(ctx);
    if (g) return g;
    Ctx &c = ctx->c;
    if (!p) return fail(c, PM_ERR_INVALID_ARG, "pm_put_particles_packed_async: NULL array");
    if (!c.mixed) return fail(c, PM_ERR_INVALID_ARG, "pm_put_particles_packed_async: packed records need a mixed context");
    if (!c.have_particles || c.stage != 0) return fail(c, PM_ERR_STATE, "pm_put_particles_packed_async: not between steps");
    if ((g = io_setup(c))) return g;
    const size_t bytes = sizeof(pm_packed_particle) * (size_t)c.np;
    // upload (copy engine) once the previous put's records have been read out of the staging buffer
    CK(cudaStreamWaitEvent(c.io_up, c.ev_in_free, 0));
    CK(cudaMemcpyAsync(c.in_stage, p, bytes, cudaMemcpyDefault, c.io_up));
    CK(cudaEventRecord(c.ev_in_ready, c.io_up));
    // then, in stream order with the steps: check the records and sort them by cell straight into the
    // particle buffer, which frees the staging buffer
    CK(cudaStreamWaitEvent(c.stream, c.ev_in_ready, 0));
    CK(cudaMemsetAsync(c.count, 0, sizeof(int32_t) * c.nc, c.stream));
    launch_put_packed_sorted(c, reinterpret_cast<const pm_packed_particle *>(c.in_stage),
                             reinterpret_cast<int *>(c.dscal + 5));
    CKL("put_packed_sorted");
    CK(cudaEventRecord(c.ev_in_free, c.stream));
    return PM_OK;
}

pm_status pm_get_particles_packed_async(pm_ctx *ctx, pm_packed_particle *p)
{
    pm_status g = guard(ctx);
    if (g) return g;
    Ctx &c = ctx->c;
    if (!p) return fail(c, PM_ERR_INVALID_ARG, "pm_get_particles_packed_async: NULL array");
    if (!c.mixed) return fail(c, PM_ERR_INVALID_ARG, "pm_get_particles_packed_async: packed records need a mixed context");
    if (!c.have_particles || c.stage != 0) return fail(c, PM_ERR_STATE, "pm_get_particles_packed_async: not between steps");
    if ((g = io_setup(c))) return g;
    const size_t bytes = sizeof(pm_packed_particle) * (size_t)c.np;
    // in stream order: the state in id order into the output staging buffer, once the previous get's
    // download has read it out
    CK(cudaStreamWaitEvent(c.stream, c.ev_out_free, 0));
    launch_store_particles_scatter<float>(c, nullptr, nullptr);
    CKL("unpermute");
    launch_store_packed(c, reinterpret_cast<pm_packed_particle *>(c.out_stage), 0, c.np);
    CKL("store_packed");
    CK(cudaEventRecord(c.ev_out_ready, c.stream));
    // download (copy engine) beside the following steps
    CK(cudaStreamWaitEvent(c.io_down, c.ev_out_ready, 0));
    CK(cudaMemcpyAsync(p, c.out_stage, bytes, cudaMemcpyDefault, c.io_down));
    CK(cudaEventRecord(c.ev_out_free, c.io_down));
    return PM_OK;
}

pm_status pm_io_wait(pm_ctx *ctx)
{
    pm_status g = guard(ctx);
    if (g) return g;
    Ctx &c = ctx->c;
    if (c.io_up) CK(cudaStreamSynchronize(c.io_up));
    if (c.io_down) CK(cudaStreamSynchronize(c.io_down));
    CK(cudaStreamSynchronize(c.stream));
    int bad = 0;
    int *flag = reinterpret_cast<int *>(c.dscal + 5);
    CK(cudaMemcpy(&bad, flag, sizeof(int), cudaMemcpyDeviceToHost));
    if (!bad) return PM_OK;
    CK(cudaMemset(flag, 0, sizeof(int)));
    c.have_particles = false;
    return fail(c, PM_ERR_INVALID_ARG, "pm_io_wait: a record put since the last wait had a cell out of range, an offset "
                                       "outside [0, 1) or a non-finite value; the particle state is invalid");
}

pm_status pm_project(pm_ctx *ctx)
{
    pm_status g = guard(ctx);
    if (g) return g;
    Ctx &c = ctx->c;
    if (!c.have_particles) return fail(c, PM_ERR_STATE, "pm_project: no particles");
    if (c.step >= c.cfg.n_steps) return fail(c, PM_ERR_STATE, "pm_project: schedule exhausted");
    if (c.stage != 0) return fail(c, PM_ERR_STATE, "pm_project: previous step not finished");
    c.stepc++;
    c.timing_on = true;
    c.mark(EV_START);
    pm_status st = PM_DISPATCH(ctx, do_project, c, false);
    c.mark(EV_PROJECT);
    c.timing_on = false;
    if (st) return st;
    c.stage = 1;
    return PM_OK;
}

pm_status pm_solve(pm_ctx *ctx)
{
    pm_status g = guard(ctx);
    if (g) return g;
    Ctx &c = ctx->c;
    if (c.stage != 1) return fail(c, PM_ERR_STATE, "pm_solve: call pm_project first");
    c.timing_on = true;
    pm_status st = PM_DISPATCH(ctx, do_solve, c, false);
    c.timing_on = false;
    if (st) return st;
    c.stage = 2;
    return PM_OK;
}

pm_status pm_update(pm_ctx *ctx)
{
    pm_status g = guard(ctx);
    if (g) return g;
    Ctx &c = ctx->c;
    if (c.stage != 2) return fail(c, PM_ERR_STATE, "pm_update: call pm_solve first");
    c.timing_on = true;
    pm_status st = PM_DISPATCH(ctx, do_update, c);
    c.mark(EV_END);
    c.timing_on = false;
    if (st) return st;
    if (!c.no_timing) c.window = std::min<int64_t>(c.window + 1, Ctx::RING);
    rotate(c);
    c.step += 1;
    c.stage = 0;
    return PM_OK;
}

static pm_status step_plain(pm_ctx *ctx)
{
    pm_status st = pm_project(ctx);
    if (st) return st;
    st = pm_solve(ctx);
    if (st) return st;
    return pm_update(ctx);
}

// one step captured into a graph on the context's capture stream, then launched on its stream; the
// executable graph of the step before the previous one is updated in place when the topology is unchanged
// (two alternate, so an update never waits for the graph that is still running)
static pm_status step_graph(pm_ctx *ctx)
{
    Ctx &c = ctx->c;
    if (!c.gstream && cudaStreamCreateWithFlags(&c.gstream, cudaStreamNonBlocking) != cudaSuccess) {
        c.gstream = nullptr;
        return cuda_fail(c, cudaGetLastError(), "pm_step: capture stream");
    }
    cudaStream_t user = c.stream;
    cudaError_t ce = cudaStreamBeginCapture(c.gstream, cudaStreamCaptureModeThreadLocal);
    if (ce != cudaSuccess) return cuda_fail(c, ce, "pm_step: cudaStreamBeginCapture");
    c.stream = c.gstream;
    c.no_timing = true;
    const pm_status st = step_plain(ctx);
    c.no_timing = false;
    c.stream = user;
    cudaGraph_t graph = nullptr;
    ce = cudaStreamEndCapture(c.gstream, &graph);
    if (st != PM_OK) {
        // the host state of a failed call is unchanged or the context is poisoned; nothing was launched
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return st;
    }
    if (ce != cudaSuccess || !graph) return cuda_fail(c, ce != cudaSuccess ? ce : cudaErrorUnknown, "pm_step: capture");
    cudaGraphExec_t &x = c.gexec[c.gslot];
    c.gslot ^= 1;
    bool updated = false;
    if (x) {
        cudaGraphExecUpdateResultInfo info{};
        updated = cudaGraphExecUpdate(x, graph, &info) == cudaSuccess;
        if (!updated) cudaGetLastError();
    }
    if (!updated) {
        if (x) cudaGraphExecDestroy(x);
        x = nullptr;
        ce = cudaGraphInstantiate(&x, graph, 0);
        if (ce != cudaSuccess) {
            x = nullptr;
            cudaGraphDestroy(graph);
            return cuda_fail(c, ce, "pm_step: cudaGraphInstantiate");
        }
    }
    cudaGraphDestroy(graph);
    ce = cudaGraphLaunch(x, c.stream);
    return ce == cudaSuccess ? PM_OK : cuda_fail(c, ce, "pm_step: cudaGraphLaunch");
}

pm_status pm_step(pm_ctx *ctx)
{
    pm_status g = guard(ctx);
    if (g) return g;
    // inside a capture by the caller (the ensemble) the step is issued as plain launches
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (ctx->c.graph_step && cudaStreamIsCapturing(ctx->c.stream, &cs) == cudaSuccess &&
        cs == cudaStreamCaptureStatusNone)
        return step_graph(ctx);
    cudaGetLastError();
    return step_plain(ctx);
}

pm_status pm_step_graph(pm_ctx *ctx, int32_t on)
{
    pm_status g = guard(ctx);
    if (g) return g;
    if (on != 0 && on != 1) return fail(ctx->c, PM_ERR_INVALID_ARG, "pm_step_graph: on must be 0 or 1");
    ctx->c.graph_step = on != 0;
    return PM_OK;
}

pm_status pm_get_particles(pm_ctx *ctx, double *pos, double *mom)
{
    pm_status g = guard(ctx);
    if (g) return g;
    Ctx &c = ctx->c;
    if (!c.have_particles) return fail(c, PM_ERR_STATE, "pm_get_particles: no particles");
    if (!pos && !mom) return PM_OK;
    return PM_DISPATCH(ctx, get_particles_t, c, pos, mom);
}

pm_status pm_get_field(pm_ctx *ctx, int field_id, double *dst)
{
    pm_status g = guard(ctx);
    if (g) return g;
    Ctx &c = ctx->c;
    if (!dst || field_id < 0 || field_id > PM_FIELD_SYZ) return fail(c, PM_ERR_INVALID_ARG, "pm_get_field: bad id");
    return PM_DISPATCH(ctx, get_field_t, c, field_id, dst);
}

pm_status pm_get_tensor(pm_ctx *ctx, int which, double *dst)
{
    pm_status g = guard(ctx);
    if (g) return g;
    Ctx &c = ctx->c;
    if (!dst || which < 0 || which > 3) return fail(c, PM_ERR_INVALID_ARG, "pm_get_tensor: bad id");
    return PM_DISPATCH(ctx, get_tensor_t, c, which, dst);
}

pm_status pm_power_spectrum(pm_ctx *ctx, int nbins, double *k, double *pk, int64_t *nmodes)
{
    pm_status g = guard(ctx);
    if (g) return g;
    Ctx &c = ctx->c;
    if (!k || !pk || !nmodes || nbins < 2 || nbins > 2048 || 3 * nbins > c.stage_elems)
        return fail(c, PM_ERR_INVALID_ARG, "pm_power_spectrum: bad arguments");
    if (!c.have_particles) return fail(c, PM_ERR_STATE, "pm_power_spectrum: no particles");
    return PM_DISPATCH(ctx, power_t, c, nbins, k, pk, nmodes);
}

pm_status pm_get_time(pm_ctx *ctx, int32_t *step, double *a, double *tau)
{
    if (!ctx) return PM_ERR_INVALID_ARG;
    Ctx &c = ctx->c;
    if (step) *step = c.step;
    if (a) *a = c.a_n[c.step];
    if (tau) {
        double t = 0.0;
        for (int i = 0; i < c.step; i++) t += c.dtau[i];
        *tau = t;
    }
    return PM_OK;
}

pm_status pm_get_schedule(pm_ctx *ctx, double *a_n, double *dtau, double *a_half)
{
    if (!ctx) return PM_ERR_INVALID_ARG;
    Ctx &c = ctx->c;
    if (a_n) std::memcpy(a_n, c.a_n.data(), sizeof(double) * c.a_n.size());
    if (dtau) std::memcpy(dtau, c.dtau.data(), sizeof(double) * c.dtau.size());
    if (a_half) std::memcpy(a_half, c.a_half.data(), sizeof(double) * c.a_half.size());
    return PM_OK;
}

pm_status pm_fft_shapes(pm_ctx *ctx, int32_t force_y, int32_t force_z, int32_t *y_shape, int32_t *z_shape)
{
    pm_status g = guard(ctx);
    if (g) return g;
    Ctx &c = ctx->c;
    if (force_y < -2 || force_y > 2 || force_z < -2 || force_z > 2)
        return fail(c, PM_ERR_INVALID_ARG, "pm_fft_shapes: shape outside -2..2");
    if (force_y == -2) force_y = c.col_shape[0];
    if (force_z == -2) force_z = c.col_shape[1];
    PM_DISPATCH(ctx, fft_tune_shapes, c, force_y, force_z);
    cudaError_t e = c.stream ? cudaStreamSynchronize(c.stream) : cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(c, e, "pm_fft_shapes");
    if (y_shape) *y_shape = c.col_shape[0];
    if (z_shape) *z_shape = c.col_shape[1];
    return PM_OK;
}

pm_status pm_deposit_shape(pm_ctx *ctx, int32_t force, int32_t *shape)
{
    pm_status g = guard(ctx);
    if (g) return g;
    Ctx &c = ctx->c;
    if (force < -2 || force > 1) return fail(c, PM_ERR_INVALID_ARG, "pm_deposit_shape: shape outside -2..1");
    if (force >= 0) c.dep_shape = force;
    else if (force == -1) {
        if (!c.have_particles || c.stage != 0 || c.step >= c.cfg.n_steps)
            return fail(c, PM_ERR_STATE, "pm_deposit_shape: timing needs particles between steps");
        const StepScalars s = scalars(c, c.step, false);
        if (c.mixed) tune_deposit_shape<float>(c, s);
        else tune_deposit_shape<double>(c, s);
        cudaError_t e = c.stream ? cudaStreamSynchronize(c.stream) : cudaDeviceSynchronize();
        if (e == cudaSuccess) e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(c, e, "pm_deposit_shape");
    }
    if (shape) *shape = c.dep_shape;
    return PM_OK;
}

pm_status pm_get_timings(pm_ctx *ctx, double *ms, int n, int64_t *launches)
{
    pm_status g = guard(ctx);
    if (g) return g;
    Ctx &c = ctx->c;
    if (!ms || n < 0 || n > PM_T_COUNT) return fail(c, PM_ERR_INVALID_ARG, "pm_get_timings: bad arguments");
    cudaError_t e = c.stream ? cudaStreamSynchronize(c.stream) : cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(c, e, "pm_get_timings");
    // stage -> (first event, last event)
    static const int span[PM_T_COUNT][2] = {
        {EV_START, EV_PROJECT}, {EV_PROJECT, EV_FWD_Z}, {EV_FWD_Z, EV_SOLVE}, {EV_SOLVE, EV_INV_X},
        {EV_INV_X, EV_KICK},    {EV_KICK, EV_END},      {EV_START, EV_END},   {EV_PROJECT, EV_FWD_X},
        {EV_FWD_X, EV_FWD_Y},   {EV_FWD_Y, EV_FWD_Z},   {EV_SOLVE, EV_INV_Z}, {EV_INV_Z, EV_INV_Y},
        {EV_INV_Y, EV_INV_X},   {EV_KICK, EV_SCAN},     {EV_SCAN, EV_END}};
    double acc[PM_T_COUNT] = {};
    const int64_t w = c.window;
    for (int64_t k = 0; k < w; k++) {
        const int64_t slot = (c.stepc - k) % Ctx::RING;
        for (int t = 0; t < PM_T_COUNT; t++) {
            float v = 0.f;
            if (cudaEventElapsedTime(&v, c.evr[slot][span[t][0]], c.evr[slot][span[t][1]]) == cudaSuccess)
                acc[t] += v;
        }
    }
    cudaGetLastError();
    for (int t = 0; t < n; t++) ms[t] = w ? acc[t] / (double)w : 0.0;
    if (launches) *launches = c.launches - c.launches_mark;
    c.launches_mark = c.launches;
    c.window = 0;
    return PM_OK;
}

pm_status pm_save(pm_ctx *ctx, const char *path)
{
    pm_status g = guard(ctx);
    if (g) return g;
    Ctx &c = ctx->c;
    if (!path) return fail(c, PM_ERR_INVALID_ARG, "pm_save: NULL path");
    if (!c.have_particles || c.stage != 0) return fail(c, PM_ERR_STATE, "pm_save: state not between steps");
    return save_impl(c, path);
}

pm_status pm_load(pm_ctx *ctx, const char *path)
{
    pm_status g = guard(ctx);
    if (g) return g;
    Ctx &c = ctx->c;
    if (!path) return fail(c, PM_ERR_INVALID_ARG, "pm_load: NULL path");
    pm_status st = c.mixed ? load_impl<float>(c, path) : load_impl<double>(c, path);
    if (st) return st;
    return c.mixed ? recount<float>(c) : recount<double>(c);
}

}  // extern "C"
