// pm_power_spectrum_noalloc: the matter power spectrum of a set of particle
// positions without any device allocation.
//
// Some callers cannot call cudaMalloc at the point where they want a
// diagnostic: code running inside a memory pool or allocator that forbids
// further allocation, an application that has handed all device memory to
// its own sub-allocator, or a latency-critical loop in which an allocation
// (and the implicit synchronisation it may bring) is not acceptable.  For
// them this entry point runs the same CIC density, r2c FFT and binning
// kernels as pm_power_spectrum, but on scratch that lives in one file-scope
// __device__ array of fixed size, reserved when the library is loaded and
// held by every GPU that loads it until the process exits.
#include <mutex>

#include "pm_fft_core.cuh"
#include "pm_internal.cuh"

namespace pm {

namespace {

constexpr int NA_MAX_MESH = 64;
constexpr int NA_MAX_BINS = 512;
constexpr size_t na_round(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t NA_RHO = na_round(sizeof(double) * NA_MAX_MESH * NA_MAX_MESH * NA_MAX_MESH);
constexpr size_t NA_SPEC = na_round(sizeof(double2) * NA_MAX_MESH * NA_MAX_MESH * (NA_MAX_MESH / 2 + 1));
constexpr size_t NA_ACC = na_round(sizeof(double) * 3 * NA_MAX_BINS);
constexpr size_t NA_TW = na_round(sizeof(double2) * NA_MAX_MESH);
constexpr size_t NA_TW2 = na_round(sizeof(double2) * (2 * NA_MAX_MESH + 64));
constexpr size_t NA_BYTES = NA_RHO + NA_SPEC + NA_ACC + NA_TW + NA_TW2;

// The scratch.  In host code this name is only a stand-in for the symbol:
// the device address comes from cudaGetSymbolAddress (once per device).
static __device__ __align__(256) unsigned char g_pk_scratch[NA_BYTES];

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_na_mutex;
void *g_na_addr[NA_MAX_DEVICES] = {};

// twiddles exp(-2 pi i k/n) and the per-stage tables of the compile-time-N passes
__global__ void k_na_twiddles(int n, double2 *tw, double2 *tw2)
{
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        double s, c;
        sincospi(-2.0 * (double)k / (double)n, &s, &c);
        tw[k] = make_double2(c, s);
    }
    const int ns = fftc::nstages(n);
    for (int st = 1; st < ns; st++) {
        const int Ns = fftc::span_before(n, st), R = fftc::radix_at(n, st), off = fftc::tw_offset(n, st);
        for (int e = threadIdx.x; e < Ns * (R - 1); e += blockDim.x) {
            const int k = e / (R - 1), r = e % (R - 1) + 1;
            double s, c;
            sincospi(-2.0 * (double)(r * k) / (double)(Ns * R), &s, &c);
            tw2[off + e] = make_double2(c, s);
        }
    }
}

// CIC mass density rho/omega_m of f64 positions (cell and offset as in pm_set_particles)
__global__ void k_na_density(const double *pos, int64_t np, int n, double q, double *rho)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    int ic[3];
    double f[3];
#pragma unroll
    for (int d = 0; d < 3; d++) {
        double x = pos[3 * i + d];
        x -= floor(x);
        if (x >= 1.0) x = 0.0;
        const double s = x * n, fl = floor(s);
        int c = (int)fl;
        if (c >= n) c -= n;
        if (c < 0) c = 0;
        ic[d] = c;
        f[d] = s - fl;
    }
#pragma unroll
    for (int dz = 0; dz < 2; dz++)
#pragma unroll
        for (int dy = 0; dy < 2; dy++)
#pragma unroll
            for (int dx = 0; dx < 2; dx++) {
                const double w = (dx ? f[0] : 1 - f[0]) * (dy ? f[1] : 1 - f[1]) * (dz ? f[2] : 1 - f[2]);
                const int64_t g = ((int64_t)((ic[2] + dz) % n) * n + (ic[1] + dy) % n) * n + (ic[0] + dx) % n;
                atomicAdd(&rho[g], q * w);
            }
}

__global__ void k_na_contrast(double *rho, int64_t nc)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nc) rho[i] -= 1.0;
}

bool na_valid_mesh(int n)
{
    if (n < 8 || n > NA_MAX_MESH || n % 8) return false;
    int m = n;
    while (m % 2 == 0) m /= 2;
    while (m % 3 == 0) m /= 3;
    return m == 1;
}

}  // namespace
}  // namespace pm

extern "C" pm_status pm_power_spectrum_noalloc(const double *d_pos, int64_t n_part, int32_t n_mesh, double omega_m,
                                                int32_t nbins, double *k, double *pk, int64_t *nmodes, void *stream)
{
    using namespace pm;
    if (!d_pos || !k || !pk || !nmodes || n_part < 1 || n_part >= ((int64_t)1 << 31) || !(omega_m > 0.0) ||
        nbins < 2)
        return PM_ERR_INVALID_ARG;
    if (!na_valid_mesh(n_mesh) || nbins > NA_MAX_BINS) return PM_ERR_UNSUPPORTED_SIZE;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) {
        cudaGetLastError();
        return PM_ERR_CUDA;
    }
    cudaPointerAttributes attr{};
    if (cudaPointerGetAttributes(&attr, d_pos) != cudaSuccess ||
        !(attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged) ||
        (attr.type == cudaMemoryTypeDevice && attr.device != dev)) {
        cudaGetLastError();
        return PM_ERR_INVALID_ARG;
    }
    // set-up, once per device: the device address of the scratch array
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_na_mutex);
        if (!g_na_addr[dev]) {
            void *ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_pk_scratch) != cudaSuccess || !ptr) {
                cudaGetLastError();
                return PM_ERR_CUDA;
            }
            g_na_addr[dev] = ptr;
        }
        base = g_na_addr[dev];
    }
    unsigned char *b = static_cast<unsigned char *>(base);
    double *rho = reinterpret_cast<double *>(b);
    double2 *spec = reinterpret_cast<double2 *>(b + NA_RHO);
    double *acc = reinterpret_cast<double *>(b + NA_RHO + NA_SPEC);
    double2 *tw = reinterpret_cast<double2 *>(b + NA_RHO + NA_SPEC + NA_ACC);
    double2 *tw2 = reinterpret_cast<double2 *>(b + NA_RHO + NA_SPEC + NA_ACC + NA_TW);

    // a context shell pointing at the scratch: no allocation, no timing
    Ctx c;
    c.stream = reinterpret_cast<cudaStream_t>(stream);
    c.device = dev;
    c.N = n_mesh;
    c.nc = (int64_t)n_mesh * n_mesh * n_mesh;
    c.nh = (int64_t)n_mesh * n_mesh * (n_mesh / 2 + 1);
    c.np = n_part;
    c.tw = tw;
    c.tw2 = tw2;
    c.plan = make_plan(n_mesh);

    k_na_twiddles<<<1, 256, 0, c.stream>>>(n_mesh, tw, tw2);
    cudaMemsetAsync(rho, 0, sizeof(double) * c.nc, c.stream);
    const double q = (double)c.nc / (double)n_part;  // N^3 m / omega_m with m = omega_m / n_part
    k_na_density<<<(unsigned)((n_part + 255) / 256), 256, 0, c.stream>>>(d_pos, n_part, n_mesh, q, rho);
    k_na_contrast<<<(unsigned)((c.nc + 255) / 256), 256, 0, c.stream>>>(rho, c.nc);
    const void *in[1] = {rho};
    void *out[1] = {spec};
    fft_forward<double>(c, 1, in, out);
    cudaMemsetAsync(acc, 0, sizeof(double) * 3 * nbins, c.stream);
    launch_pk_bin<double>(c, spec, nbins, acc);
    double h[3 * NA_MAX_BINS];
    cudaError_t e = cudaMemcpyAsync(h, acc, sizeof(double) * 3 * nbins, cudaMemcpyDeviceToHost, c.stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return PM_ERR_CUDA;
    for (int bb = 0; bb < nbins; bb++) {
        const double cnt = h[2 * nbins + bb];
        pk[bb] = cnt > 0 ? h[bb] / cnt : 0.0;
        k[bb] = cnt > 0 ? h[nbins + bb] / cnt : 0.0;
        nmodes[bb] = (int64_t)llround(cnt);
    }
    return PM_OK;
}
