// Particle-mesh kernels: stress-energy projection, gather + kick + drift,
// counting sort by cell, particle I/O.
//
// Projection (Sec. 2.1 "particle-mesh projection", Eqs. matterstress):
// particles are kept sorted by cell.  One CTA owns an 8^3 tile of mesh
// vertices and pulls every particle whose CIC cloud touches the tile (the
// 9^3 cells [x0-1, x0+8)), computes its charges once into shared memory and
// lets each thread accumulate the 9 source components of its own vertex in
// registers.  No global atomics, and every mesh value is written once with
// coalesced stores.  The same kernel assembles the configuration-space
// sources of the field equations from phi_{n-1}, chi_{n-1}, phi_{n-2}.
#include <algorithm>

#include "pm_internal.cuh"

namespace pm {

namespace {

constexpr int TILE = 8;
constexpr int REG = TILE + 1;        // 9 source cells per axis
constexpr int FLD = TILE + 2;        // 10 field vertices per axis
constexpr int NREG = REG * REG * REG;  // 729
constexpr int NFLD = FLD * FLD * FLD;  // 1000
constexpr int DEP_THREADS = TILE * TILE * TILE;  // 512
constexpr int NK0SLOTS = 1024;

// Per-cell accumulator of the T^00 charge, whose cell sums cancel against the
// uniform background in R.  FP64: plain double.  Mixed: float-float with
// Knuth's TwoSum, so a cell sum keeps about 48 significant bits.  The other
// components have no such cancellation and are summed in the field type.
template <class T> struct Acc;
template <> struct Acc<double> {
    double s;
    __device__ __forceinline__ void zero() { s = 0.0; }
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ double hi() const { return s; }
    __device__ __forceinline__ double lo() const { return 0.0; }
};
template <> struct Acc<float> {
    float s, c;
    __device__ __forceinline__ void zero() { s = 0.f; c = 0.f; }
    __device__ __forceinline__ void add(float x)
    {
        float t = __fadd_rn(s, x);
        float bp = __fsub_rn(t, s);
        float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(x, bp));
        s = t;
        c = __fadd_rn(c, e);
    }
    __device__ __forceinline__ float hi() const { return s; }
    __device__ __forceinline__ float lo() const { return c; }
};

// 1 / sqrt(x) and a / b: the hardware approximations (a few ulp) in the mixed form, whose
// FP32 rounding already sets the error; IEEE operations in FP64
__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_t(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float div_t(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double div_t(double a, double b) { return a / b; }

template <class T> __device__ __forceinline__ T mulr(T a, T b);
template <> __device__ __forceinline__ float mulr<float>(float a, float b) { return __fmul_rn(a, b); }
template <> __device__ __forceinline__ double mulr<double>(double a, double b) { return __dmul_rn(a, b); }

__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

template <class T> struct DepParams {
    const Particle<T> *part;
    const int32_t *start;
    const T *phi1;   // phi_{n-1}
    const T *chi1;   // chi_{n-1}
    const T *phi2;   // phi_{n-2}
    Ptrs out;        // R, Fx, Fy, Fz, Sxx, Sxy, Sxz, Syy, Syz
    double *k0slots; // NK0SLOTS partial sums of the k = 0 excess
    int N, nt;
    int full;        // 1: relativistic sources; 0: R only (bootstrap / Newtonian)
    int use_fields;  // phi/chi enter the charges (not in the bootstrap / Newtonian mode)
    int newtonian;
    T a, a2, mass;
    T G;             // 4piG a^-2 N^3 (Newtonian: 4piG a^-1 N^3)
    T rb_hi, rb_lo;  // expected per-vertex charge sum of a uniform load, float-float split
    T c1, c2;        // 3Hc/dtau_{n-1}, 3Hc^2
    T inv_dt2;       // 1/dtau_{n-2}
    T halfN;         // N/2 (centred difference 1/(2 dx))
    int full_hc;     // R -= Nl, the remainder of Eq. fullHc
    int write_f;     // F_i is needed (momentum-constraint B)
    T hc, n2;        // Hc(a_n), N^2 (7-point Laplacian 1/dx^2)
    double inv_g;    // 1 / (4piG a^-2 N^3): Nl's share of the k = 0 sum
};

// e^x - 1 - x without cancellation: its Taylor series through x^9 / 9! for small |x| (truncation below
// 1e-8 relative in FP32 for |x| < 1/2 and below 1e-20 in FP64 for |x| < 1e-2), expm1(x) - x beyond.
template <class T> __device__ __forceinline__ T expm1_minus_x(T x)
{
    constexpr T lim = sizeof(T) == 4 ? T(0.5) : T(1e-2);
    if (fabs(x) >= lim) return expm1(x) - x;
    T s = T(1.0 / 362880.0);
    s = s * x + T(1.0 / 40320.0);
    s = s * x + T(1.0 / 5040.0);
    s = s * x + T(1.0 / 720.0);
    s = s * x + T(1.0 / 120.0);
    s = s * x + T(1.0 / 24.0);
    s = s * x + T(1.0 / 6.0);
    s = s * x + T(0.5);
    return s * x * x;
}

// Nonlinear remainder of Eq. fullHc at one vertex, from phi_{n-1} and chi_{n-1} staged with a halo of 1
// (stride st[d] along axis d) and phi_{n-2}:
//   Nl = (e^{2phi} - 1) Lap phi - 1/2 e^{2phi} |grad phi|^2
//      + 3/2 [Hc^2 (e^x - 1 - x) - 2 Hc phi' (e^x - 1) + phi'^2 e^x],  x = -2 psi,
// the bracket being (Hc - phi')^2 e^{-2psi} - Hc^2 + 2 Hc phi' + 2 Hc^2 psi regrouped so that no term
// of size Hc^2 cancels.
template <class T>
__device__ __forceinline__ T hc_remainder(const T *sphi, const T *schi, int vo, const int (&st)[3], T phi2,
                                          const DepParams<T> &p)
{
    const T ph = sphi[vo];
    T lap = T(-6) * ph, g2 = T(0);
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const T up = sphi[vo + st[d]], dn = sphi[vo - st[d]];
        lap += up + dn;
        const T g = (up - dn) * p.halfN;
        g2 += g * g;
    }
    lap *= p.n2;
    const T psi = ph - schi[vo];
    const T dphi = (ph - phi2) * p.inv_dt2;
    const T x = T(-2) * psi;
    const T em = expm1(x);
    const T e2p = exp(T(2) * ph);
    return expm1(T(2) * ph) * lap - T(0.5) * e2p * g2 +
           T(1.5) * (p.hc * p.hc * expm1_minus_x(x) - T(2) * p.hc * dphi * em + dphi * dphi * (em + T(1)));
}

// Particle records per shared-memory chunk, the deposit's tunable "bin shape" (pm_deposit_shape): shape 0
// (960 FP32) was the fastest of 640-1024 at 512^3 in early steps, shape 1 (768) is a little faster in the
// first, unclustered steps and slower late.  Both keep three CTAs per SM in FP32.
constexpr int NDEPSHAPES = 2;
template <class T, int V> constexpr int dep_cap() { return sizeof(T) == 8 ? (V ? 512 : 640) : (V ? 768 : 960); }

template <class T, int V> size_t dep_smem()
{
    return sizeof(T) * (12 * dep_cap<T, V>() + 2 * NFLD) +
           sizeof(int) * (3 * NREG + 64 + FLD * FLD + FLD);
}

// Per-particle record in shared memory: {fx, fy, fz, q00}, {q0x, q0y, q0z, Txx}, {Txy, Txz, Tyy, Tyz}
// (trace-free T_ij, Tzz implied), read back with three 16-byte (FP32) or six 16-byte (FP64) loads.
template <class T> struct alignas(16) DepRec {
    T f[3], q00, q0[3], txx, txy, txz, tyy, tyz;
};
static_assert(sizeof(DepRec<float>) == 48 && sizeof(DepRec<double>) == 96, "packed record");

// Exclusive scan of v[0..n) (n <= 2 * blockDim) in place; returns the total.
__device__ int block_exclusive_scan(int *v, int n, int *warp_tmp)
{
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    int a = (2 * tid < n) ? v[2 * tid] : 0;
    int b = (2 * tid + 1 < n) ? v[2 * tid + 1] : 0;
    int s = a + b, x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tmp[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int nw = blockDim.x >> 5;
        int w = lane < nw ? warp_tmp[lane] : 0, z = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, z, o);
            if (lane >= o) z += y;
        }
        if (lane < nw) warp_tmp[lane] = z - w;
        if (lane == nw - 1) warp_tmp[32] = z;
    }
    __syncthreads();
    int excl = warp_tmp[wid] + x - s;
    if (2 * tid < n) v[2 * tid] = excl;
    if (2 * tid + 1 < n) v[2 * tid + 1] = excl + a;
    int total = warp_tmp[32];
    __syncthreads();
    return total;
}

// The deposit of one 8^3 vertex tile b of the box described by p (smem: dep_smem of this CAP).
template <class T, int CAP>
__device__ __forceinline__ void deposit_tile(const DepParams<T> &p, const int b)
{
    extern __shared__ __align__(16) unsigned char smem[];
    DepRec<T> *rec = reinterpret_cast<DepRec<T> *>(smem);            // [CAP]
    T *sphi = reinterpret_cast<T *>(rec + CAP);
    T *schi = sphi + NFLD;
    int *scnt = reinterpret_cast<int *>(schi + NFLD);
    int *soff = scnt + NREG;
    int *sgs = soff + NREG;
    int *wtmp = sgs + NREG;                                          // 64 ints
    int *rowb = wtmp + 64;                                           // [FLD*FLD] wrapped (z,y) row bases
    int *xw = rowb + FLD * FLD;                                      // [FLD] wrapped x

    const int N = p.N, nt = p.nt, tid = threadIdx.x;
    const int x0 = (b % nt) * TILE, y0 = ((b / nt) % nt) * TILE, z0 = (b / (nt * nt)) * TILE;
    if (tid < FLD * FLD) {
        const int ry = tid % FLD, rz = tid / FLD;
        rowb[tid] = (wrapi(z0 - 1 + rz, N) * N + wrapi(y0 - 1 + ry, N)) * N;
    }
    if (tid < FLD) xw[tid] = wrapi(x0 - 1 + tid, N);
    __syncthreads();

    // potentials of the previous solve on the 10^3 vertices [x0-1, x0+8]
    constexpr int NIT = (NFLD + DEP_THREADS - 1) / DEP_THREADS;
    constexpr int RIT = (NREG + DEP_THREADS - 1) / DEP_THREADS;
    T a[NIT], c[NIT];
    int gs0[RIT], gs1[RIT];
    if (p.use_fields) {
#pragma unroll
        for (int q = 0; q < NIT; q++) {
            const int i = tid + q * DEP_THREADS;
            if (i < NFLD) {
                const int row = i / FLD, rx = i - row * FLD;
                const int64_t g = (int64_t)rowb[row] + xw[rx];
                a[q] = p.phi1[g];
                c[q] = p.chi1[g];
            }
        }
    }
    // particle ranges of the 9^3 source cells [x0-1, x0+8)
#pragma unroll
    for (int q = 0; q < RIT; q++) {
        const int i = tid + q * DEP_THREADS;
        if (i < NREG) {
            const int row = i / REG, sx = i - row * REG;
            const int sy = row % REG, sz = row / REG;
            const int64_t g = (int64_t)rowb[sy + FLD * sz] + xw[sx];
            gs0[q] = p.start[g];
            gs1[q] = p.start[g + 1];
        }
    }
#pragma unroll
    for (int q = 0; q < NIT; q++) {
        const int i = tid + q * DEP_THREADS;
        if (i < NFLD) {
            sphi[i] = p.use_fields ? a[q] : T(0);
            schi[i] = p.use_fields ? c[q] : T(0);
        }
    }
#pragma unroll
    for (int q = 0; q < RIT; q++) {
        const int i = tid + q * DEP_THREADS;
        if (i < NREG) {
            scnt[i] = gs1[q] - gs0[q];
            soff[i] = gs1[q] - gs0[q];
            sgs[i] = gs0[q];
        }
    }
    __syncthreads();
    const int total = block_exclusive_scan(soff, NREG, wtmp);

    const int ox = tid % TILE, oy = (tid / TILE) % TILE, oz = tid / (TILE * TILE);
    Acc<T> acc00;
    acc00.zero();
    T acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    Acc<T> k0;   // this thread's share of the k = 0 excess (float-float in the mixed form)
    k0.zero();
    const bool full = p.full;

    for (int lo = 0; lo < total; lo += CAP) {
        const int hi = min(total, lo + CAP);
        // source cell of local particle i: largest t with soff[t] <= i
        auto cell_of = [&](int i) {
            int t0 = 0, t1 = NREG - 1;
            while (t0 < t1) {
                int m = (t0 + t1 + 1) >> 1;
                if (soff[m] <= i) t0 = m;
                else t1 = m - 1;
            }
            return t0;
        };
        int tn = lo + tid < hi ? cell_of(lo + tid) : 0;
        for (int i = lo + tid; i < hi; i += DEP_THREADS) {
            const int t = tn;
            if (i + DEP_THREADS < hi) {   // the next particle of this thread: its cell now, its record into L1
                tn = cell_of(i + DEP_THREADS);
                asm volatile("prefetch.global.L1 [%0];" ::"l"(p.part + sgs[tn] + (i + DEP_THREADS - soff[tn])));
            }
            const Particle<T> P = p.part[sgs[t] + (i - soff[t])];
            const int sx = t % REG, sy = (t / REG) % REG, sz = t / (REG * REG);
            DepRec<T> r;
            r.f[0] = P.f[0];
            r.f[1] = P.f[1];
            r.f[2] = P.f[2];
            if (!full && p.newtonian) {
                r.q00 = p.mass;
            } else {
                T ph = 0, ch = 0;
                if (p.use_fields) {
                    const T fx = P.f[0], fy = P.f[1], fz = P.f[2];
                    const T wx[2] = {T(1) - fx, fx}, wy[2] = {T(1) - fy, fy}, wz[2] = {T(1) - fz, fz};
#pragma unroll
                    for (int dz = 0; dz < 2; dz++)
#pragma unroll
                        for (int dy = 0; dy < 2; dy++)
#pragma unroll
                            for (int dx = 0; dx < 2; dx++) {
                                const T w = wx[dx] * wy[dy] * wz[dz];
                                const int v = (sx + dx) + FLD * ((sy + dy) + FLD * (sz + dz));
                                ph += w * sphi[v];
                                ch += w * schi[v];
                            }
                }
                const T ux = P.u[0], uy = P.u[1], uz = P.u[2];
                const T u2 = ux * ux + uy * uy + uz * uz;
                const T e2 = p.a2 + u2;
                const T iE = rsqrt_t(e2);
                // E = a + u^2 / (E + a): the approximate E enters only the small term, so E keeps the
                // accuracy of a (the T^00 charge cancels against the background in R)
                const T dE = div_t(u2, e2 * iE + p.a);
                const T E = p.a + dE;
                const T v2 = u2 * iE * iE;
                const T m = p.mass;
                // T^00 charge and its excess over a particle at rest (k = 0 mode, summed in FP64)
                r.q00 = m * E * (T(1) + T(3) * ph + ph * v2);
                if (sx >= 1 && sy >= 1 && sz >= 1) k0.add(m * (dE + E * (T(3) * ph + ph * v2)));
                if (full) {
                    const T wv = m * (T(1) + T(4) * ph - ch);
                    r.q0[0] = wv * ux;
                    r.q0[1] = wv * uy;
                    r.q0[2] = wv * uz;
                    const T ws = m * (T(1) + T(3) * ph - ph * v2) * iE;
                    const T txx = ws * ux * ux, tyy = ws * uy * uy, tzz = ws * uz * uz;
                    const T tr3 = (txx + tyy + tzz) * T(1.0 / 3.0);
                    r.txx = txx - tr3;
                    r.txy = ws * ux * uy;
                    r.txz = ws * ux * uz;
                    r.tyy = tyy - tr3;
                    r.tyz = ws * uy * uz;
                }
            }
            rec[i - lo] = r;
        }
        __syncthreads();
        // vertex o receives from source cells o - d, d in {0,1}^3, weight (d ? f : 1 - f) per axis.
        // The two x-neighbours (region x = ox and ox + 1) are adjacent in the particle order.
#pragma unroll
        for (int dz = 0; dz < 2; dz++)
#pragma unroll
            for (int dy = 0; dy < 2; dy++) {
                const int ts = ox + REG * ((oy + 1 - dy) + REG * (oz + 1 - dz));  // cell with dx = 1
                const int mid = soff[ts + 1];                                     // first particle with dx = 0
                const int jb = max(soff[ts], lo), je = min(mid + scnt[ts + 1], hi);
                for (int jj = jb; jj < je; jj++) {
                    const DepRec<T> r = rec[jj - lo];
                    const T wyz = (dy ? r.f[1] : T(1) - r.f[1]) * (dz ? r.f[2] : T(1) - r.f[2]);
                    const T w = (jj < mid ? r.f[0] : T(1) - r.f[0]) * wyz;
                    acc00.add(mulr(w, r.q00));
                    if (full) {
                        acc[0] += w * r.q0[0];
                        acc[1] += w * r.q0[1];
                        acc[2] += w * r.q0[2];
                        acc[3] += w * r.txx;
                        acc[4] += w * r.txy;
                        acc[5] += w * r.txz;
                        acc[6] += w * r.tyy;
                        acc[7] += w * r.tyz;
                    }
                }
            }
        __syncthreads();
    }

    const int64_t go = ((int64_t)(z0 + oz) * N + (y0 + oy)) * N + (x0 + ox);
    const int vo = (ox + 1) + FLD * ((oy + 1) + FLD * (oz + 1));
    const int st[3] = {1, FLD, FLD * FLD};
    T nl = T(0);
    if (p.full_hc) {
        nl = hc_remainder<T>(sphi, schi, vo, st, p.phi2[go], p);
        k0.add(-nl * (T)p.inv_g);   // the k = 0 mode carries the mean of -Nl
    }

    // k = 0 excess: warp reduction of the (hi, lo) pairs with TwoSum, one FP64 atomic per warp into a slot
    {
        T hi = k0.hi(), lo = k0.lo();
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const T h2 = __shfl_down_sync(0xffffffffu, hi, o), l2 = __shfl_down_sync(0xffffffffu, lo, o);
            const T t = hi + h2, bp = t - hi;
            lo += l2 + ((hi - (t - bp)) + (h2 - bp));
            hi = t;
        }
        if ((tid & 31) == 0 && !p.newtonian)
            atomicAdd(&p.k0slots[(blockIdx.x * (DEP_THREADS >> 5) + (tid >> 5)) & (NK0SLOTS - 1)],
                      (double)hi + (double)lo);
    }

    // epilogue: assemble the field-equation sources at vertex o
    const T phc = sphi[vo], chc = schi[vo];
    // R: the uniform background a*Omega_m is removed before rounding
    const T dS = (acc00.hi() - p.rb_hi) + (acc00.lo() - p.rb_lo);
    reinterpret_cast<T *>(p.out.p[0])[go] = p.G * dS - p.c1 * phc - p.c2 * chc - nl;
    if (!full) return;
    T gphi[3], gpsi[3];
#pragma unroll
    for (int d = 0; d < 3; d++) {
        const T dp = (sphi[vo + st[d]] - sphi[vo - st[d]]) * p.halfN;
        const T dc = (schi[vo + st[d]] - schi[vo - st[d]]) * p.halfN;
        gphi[d] = dp;
        gpsi[d] = dp - dc;
    }
    const T dphi = (phc - p.phi2[go]) * p.inv_dt2;
    if (p.write_f) {
#pragma unroll
        for (int d = 0; d < 3; d++) reinterpret_cast<T *>(p.out.p[1 + d])[go] = p.G * acc[d] - dphi * gpsi[d];
    }
    T Q[3][3];
#pragma unroll
    for (int i = 0; i < 3; i++)
#pragma unroll
        for (int j = 0; j < 3; j++) Q[i][j] = T(2) * gphi[i] * gphi[j] - (gphi[i] + gpsi[i]) * (gphi[j] + gpsi[j]);
    const T trQ3 = (Q[0][0] + Q[1][1] + Q[2][2]) * T(1.0 / 3.0);
    const T G4 = T(4) * p.G;
    reinterpret_cast<T *>(p.out.p[4])[go] = G4 * acc[3] - T(2) * (Q[0][0] - trQ3);
    reinterpret_cast<T *>(p.out.p[5])[go] = G4 * acc[4] - T(2) * Q[0][1];
    reinterpret_cast<T *>(p.out.p[6])[go] = G4 * acc[5] - T(2) * Q[0][2];
    reinterpret_cast<T *>(p.out.p[7])[go] = G4 * acc[6] - T(2) * (Q[1][1] - trQ3);
    reinterpret_cast<T *>(p.out.p[8])[go] = G4 * acc[7] - T(2) * Q[1][2];
}

template <class T, int V>
__global__ void __launch_bounds__(DEP_THREADS, sizeof(T) == 4 ? 3 : 1) k_project(const __grid_constant__ DepParams<T> p)
{
    deposit_tile<T, dep_cap<T, V>()>(p, blockIdx.x);
}

// Several boxes in one launch (the batched ensemble): CTA j deposits tile j - first[i] of box i, the box whose
// range [first[i], first[i+1]) holds j.  The boxes' parameters travel by value in the kernel's parameter space.
constexpr int MAXBATCH = 48;
template <class T> struct DepBatch {
    int nbox;
    int first[MAXBATCH + 1];
    DepParams<T> box[MAXBATCH];
};
static_assert(sizeof(DepBatch<double>) < 32000, "kernel parameter space");

template <class T, int V>
__global__ void __launch_bounds__(DEP_THREADS, sizeof(T) == 4 ? 3 : 1) k_project_batch(const __grid_constant__ DepBatch<T> q)
{
    int i = 0;
    while (i + 1 < q.nbox && (int)blockIdx.x >= q.first[i + 1]) i++;
    deposit_tile<T, dep_cap<T, V>()>(q.box[i], (int)blockIdx.x - q.first[i]);
}

// Sum the k = 0 slots: dscal[0] = sum over particles of the T^00 excess (block b: box b of a batch).
struct K0Batch {
    double *dscal[MAXBATCH];
};
__device__ void k0_reduce_one(double *dscal);
__global__ void k_k0_reduce(double *dscal) { k0_reduce_one(dscal); }
__global__ void k_k0_reduce_batch(const __grid_constant__ K0Batch q) { k0_reduce_one(q.dscal[blockIdx.x]); }
__device__ void k0_reduce_one(double *dscal)
{
    __shared__ double s[32];
    double v = 0.0;
    for (int i = threadIdx.x; i < NK0SLOTS; i += blockDim.x) v += dscal[8 + i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        v = threadIdx.x < (blockDim.x >> 5) ? s[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) dscal[0] = v;
    }
}

// ---------------------------------------------------------------------------
// Gather + kick + drift (Eqs. kick, drift to first order, Sec. 3.1):
//   du_i/dtau = -E d_i psi - (u^2/E) d_i phi - u_j d_i B_j,  E = sqrt(a_n^2 + u^2)
//   dx^i/dtau = (u_i/E')(1 + 3 phi - chi - phi u'^2/E'^2) + B_i,  E' at a_{n+1/2}
// with mesh gradients (f(x+dx) - f(x-dx)) / (2 dx) interpolated by CIC, i.e. a
// 4x2x2 stencil per direction.  Newtonian mode: du = -a grad phi, dx = u/a.
// The new cell of each particle is counted for the sort.
// ---------------------------------------------------------------------------
template <class T> struct KdParams {
    Particle<T> *part;
    const int32_t *start;
    int32_t *count;
    const T *phi, *chi, *Bx, *By, *Bz;
    int64_t np;
    int N, nt;
    int newtonian;
    T a, a2, a_half2, inv_a_half, dt_kick, dt_drift_N, halfN;
};

constexpr int KT = 8;                     // tile side in cells
constexpr int KV = KT + 3;                // vertices per axis: x0-1 .. x0+9
constexpr int KNV = KV * KV * KV;         // 1331
constexpr int KD_THREADS = 256;

// phi, chi, B_x, B_y of one vertex in one 16-byte (FP32) or two 16-byte (FP64) loads
template <class T> struct alignas(4 * sizeof(T) >= 16 ? 16 : 4 * sizeof(T)) Vtx4 {
    T phi, chi, bx, by;
};

template <class T> size_t kd_smem()
{
    return sizeof(Vtx4<T>) * KNV + sizeof(T) * KNV + sizeof(int) * (KV * KV + KV + 2 * KT * KT + 2 + 33);
}

// Accumulate CIC value and centred-difference gradients of one vertex value s
// at stencil offset (kx, ky, kz) in {0..3}^3 (offset -1 .. +2 from the cell);
// terms whose weight is identically zero are skipped at compile time.
template <int kx, int ky, int kz, class T>
__device__ __forceinline__ void stencil_acc(T s, const T *Wx, const T *Wy, const T *Wz, const T *Gx, const T *Gy,
                                            const T *Gz, T &val, T (&g)[3])
{
    constexpr bool cx = (kx == 1 || kx == 2), cy = (ky == 1 || ky == 2), cz = (kz == 1 || kz == 2);
    if constexpr (cx && cy && cz) val += Wx[kx] * Wy[ky] * Wz[kz] * s;
    if constexpr (cy && cz) g[0] += Gx[kx] * (Wy[ky] * Wz[kz]) * s;
    if constexpr (cx && cz) g[1] += Gy[ky] * (Wx[kx] * Wz[kz]) * s;
    if constexpr (cx && cy) g[2] += Gz[kz] * (Wx[kx] * Wy[ky]) * s;
}

template <int I, class T>
__device__ __forceinline__ void gather_all(const Vtx4<T> *sv, const T *sbz, int vb, bool newtonian, const T *Wx,
                                           const T *Wy, const T *Wz, const T *Gx, const T *Gy, const T *Gz, T (&val)[5],
                                           T (&grd)[5][3])
{
    if constexpr (I < 64) {
        constexpr int kx = I % 4, ky = (I / 4) % 4, kz = I / 16;
        constexpr bool cx = (kx == 1 || kx == 2), cy = (ky == 1 || ky == 2), cz = (kz == 1 || kz == 2);
        if constexpr ((int)!cx + (int)!cy + (int)!cz <= 1) {
            const int v = vb + kx + KV * (ky + KV * kz);
            if (newtonian) {
                stencil_acc<kx, ky, kz>(sv[v].phi, Wx, Wy, Wz, Gx, Gy, Gz, val[0], grd[0]);
            } else {
                const Vtx4<T> a = sv[v];
                const T bz = sbz[v];
                stencil_acc<kx, ky, kz>(a.phi, Wx, Wy, Wz, Gx, Gy, Gz, val[0], grd[0]);
                stencil_acc<kx, ky, kz>(a.chi, Wx, Wy, Wz, Gx, Gy, Gz, val[1], grd[1]);
                stencil_acc<kx, ky, kz>(a.bx, Wx, Wy, Wz, Gx, Gy, Gz, val[2], grd[2]);
                stencil_acc<kx, ky, kz>(a.by, Wx, Wy, Wz, Gx, Gy, Gz, val[3], grd[3]);
                stencil_acc<kx, ky, kz>(bz, Wx, Wy, Wz, Gx, Gy, Gz, val[4], grd[4]);
            }
        }
        gather_all<I + 1>(sv, sbz, vb, newtonian, Wx, Wy, Wz, Gx, Gy, Gz, val, grd);
    }
}

// One CTA per 8^3 tile of cells: phi, chi and B on the 11^3 vertices around
// the tile go to shared memory once; each thread then gathers the CIC value
// and centred-difference gradients for one particle from there.
template <class T>
__device__ __forceinline__ void kick_tile(const KdParams<T> &p, const int b)
{
    extern __shared__ __align__(16) unsigned char smem[];
    Vtx4<T> *sv = reinterpret_cast<Vtx4<T> *>(smem);              // [KNV]
    T *sbz = reinterpret_cast<T *>(sv + KNV);                      // [KNV]
    int *rowb = reinterpret_cast<int *>(sbz + KNV);                // [KV*KV] wrapped (z,y) row bases
    int *xw = rowb + KV * KV;                                      // [KV] wrapped x
    int *roff = xw + KV;                                           // 65 row offsets (+1 pad)
    int *rgs = roff + KT * KT + 2;                                 // 64 global row starts
    int *wtmp = rgs + KT * KT;                                     // 33
    const int N = p.N, nt = p.nt, tid = threadIdx.x;
    const int x0 = (b % nt) * KT, y0 = ((b / nt) % nt) * KT, z0 = (b / (nt * nt)) * KT;

    if (tid < KV * KV) {
        const int ry = tid % KV, rz = tid / KV;
        rowb[tid] = (wrapi(z0 - 1 + rz, N) * N + wrapi(y0 - 1 + ry, N)) * N;
    }
    if (tid < KV) xw[tid] = wrapi(x0 - 1 + tid, N);
    // particle rows of the tile: cells (x0 .. x0+7, y, z) are contiguous
    int cnt = 0;
    if (tid < KT * KT) {
        const int ry = tid % KT, rz = tid / KT;
        const int64_t c0 = ((int64_t)(z0 + rz) * N + (y0 + ry)) * N + x0;
        const int gs = p.start[c0];
        cnt = p.start[c0 + KT] - gs;
        rgs[tid] = gs;
    }
    {
        const int lane = tid & 31, wid = tid >> 5;
        int x = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (wid < 2 && lane == 31) wtmp[wid] = x;
        __syncthreads();
        if (tid < KT * KT) roff[tid] = x - cnt + (wid == 1 ? wtmp[0] : 0);
        if (tid == 0) roff[KT * KT] = wtmp[0] + wtmp[1];
    }
    // fields on the vertex block: every load of this thread's vertices issued before the stores
    if (p.newtonian) {
        for (int i = tid; i < KNV; i += KD_THREADS) {
            const int row = i / KV, rx = i - row * KV;
            Vtx4<T> a;
            a.phi = __ldg(p.phi + (int64_t)rowb[row] + xw[rx]);
            sv[i] = a;
        }
    } else {
        constexpr int KIT = (KNV + KD_THREADS - 1) / KD_THREADS;
        Vtx4<T> va[KIT];
        T vz[KIT];
#pragma unroll
        for (int q = 0; q < KIT; q++) {
            const int i = tid + q * KD_THREADS;
            if (i < KNV) {
                const int row = i / KV, rx = i - row * KV;
                const int64_t g = (int64_t)rowb[row] + xw[rx];
                va[q].phi = __ldg(p.phi + g);
                va[q].chi = __ldg(p.chi + g);
                va[q].bx = __ldg(p.Bx + g);
                va[q].by = __ldg(p.By + g);
                vz[q] = __ldg(p.Bz + g);
            }
        }
#pragma unroll
        for (int q = 0; q < KIT; q++) {
            const int i = tid + q * KD_THREADS;
            if (i < KNV) {
                sv[i] = va[q];
                sbz[i] = vz[q];
            }
        }
    }
    __syncthreads();
    const int total = roff[KT * KT];
    const T hn = p.halfN;
    for (int i = tid; i < total; i += KD_THREADS) {
        int r0 = 0, r1 = KT * KT - 1;
        while (r0 < r1) {
            const int m = (r0 + r1 + 1) >> 1;
            if (roff[m] <= i) r0 = m;
            else r1 = m - 1;
        }
        const int64_t gi = (int64_t)rgs[r0] + (i - roff[r0]);
        Particle<T> P = p.part[gi];
        const int ix = P.cell % N, iy = (P.cell / N) % N, iz = P.cell / (N * N);
        const int vb = (ix - x0) + KV * ((iy - y0) + KV * (iz - z0));  // vertex block index of offset -1
        const T fx = P.f[0], fy = P.f[1], fz = P.f[2];
        const T Wx[4] = {0, T(1) - fx, fx, 0}, Wy[4] = {0, T(1) - fy, fy, 0}, Wz[4] = {0, T(1) - fz, fz, 0};
        const T Gx[4] = {-(T(1) - fx) * hn, -fx * hn, (T(1) - fx) * hn, fx * hn};
        const T Gy[4] = {-(T(1) - fy) * hn, -fy * hn, (T(1) - fy) * hn, fy * hn};
        const T Gz[4] = {-(T(1) - fz) * hn, -fz * hn, (T(1) - fz) * hn, fz * hn};
        T val[5] = {0, 0, 0, 0, 0};
        T grd[5][3] = {};
        gather_all<0>(sv, sbz, vb, p.newtonian, Wx, Wy, Wz, Gx, Gy, Gz, val, grd);
        T u[3] = {P.u[0], P.u[1], P.u[2]};
        T dx[3];
        if (p.newtonian) {
#pragma unroll
            for (int d = 0; d < 3; d++) u[d] -= p.dt_kick * p.a * grd[0][d];
#pragma unroll
            for (int d = 0; d < 3; d++) dx[d] = p.dt_drift_N * u[d] * p.inv_a_half;
        } else {
            const T u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
            const T e2 = p.a2 + u2;
            const T iE = rsqrt_t(e2);
            const T E = e2 * iE;
            const T u2E = u2 * iE;
            T K[3];
#pragma unroll
            for (int d = 0; d < 3; d++) {
                const T dpsi = grd[0][d] - grd[1][d];
                K[d] = -E * dpsi - u2E * grd[0][d] - (u[0] * grd[2][d] + u[1] * grd[3][d] + u[2] * grd[4][d]);
            }
#pragma unroll
            for (int d = 0; d < 3; d++) u[d] += p.dt_kick * K[d];
            const T v2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
            const T iEd = rsqrt_t(p.a_half2 + v2);
            const T fac = (T(1) + T(3) * val[0] - val[1] - val[0] * v2 * iEd * iEd) * iEd;
#pragma unroll
            for (int d = 0; d < 3; d++) dx[d] = p.dt_drift_N * (u[d] * fac + val[2 + d]);
        }
        const T fo[3] = {fx, fy, fz};
        const int io[3] = {ix, iy, iz};
        int inew[3];
#pragma unroll
        for (int d = 0; d < 3; d++) {
            T f = fo[d] + dx[d];
            T fl = floor(f);
            f -= fl;
            // a finite move is far below N cells; anything else (NaN, Inf) keeps the cell
            int carry = (fabs(fl) < (T)N) ? (int)fl : 0;
            if (f >= T(1)) {
                f = T(0);
                carry += 1;
            }
            int c = (io[d] + carry) % N;
            if (c < 0) c += N;
            inew[d] = c;
            P.f[d] = f;
            P.u[d] = u[d];
        }
        P.cell = (inew[2] * N + inew[1]) * N + inew[0];
        p.part[gi] = P;
        atomicAdd(&p.count[P.cell], 1);
    }
}

template <class T>
__global__ void __launch_bounds__(KD_THREADS, sizeof(T) == 4 ? 4 : 1) k_kick_drift(const __grid_constant__ KdParams<T> p)
{
    kick_tile<T>(p, blockIdx.x);
}

template <class T> struct KdBatch {
    int nbox;
    int first[MAXBATCH + 1];
    KdParams<T> box[MAXBATCH];
};
static_assert(sizeof(KdBatch<double>) < 32000, "kernel parameter space");

template <class T>
__global__ void __launch_bounds__(KD_THREADS, sizeof(T) == 4 ? 4 : 1) k_kick_batch(const __grid_constant__ KdBatch<T> q)
{
    int i = 0;
    while (i + 1 < q.nbox && (int)blockIdx.x >= q.first[i + 1]) i++;
    kick_tile<T>(q.box[i], (int)blockIdx.x - q.first[i]);
}

// ---------------------------------------------------------------------------
// Counting sort by cell: exclusive scan of the per-cell counts, then scatter.
// The scan takes two passes over the counts.  A scan tile is SCAN_ROUNDS rounds of one 16-byte
// vector per thread; a round covers 4 * SCAN_T consecutive counts, so each warp load and store is
// 512 contiguous bytes.  The first pass writes each tile's sum.  The second reads its tile again,
// adds up the sums of the tiles before it (32 KB at 512^3, read from L2 in 16-byte vectors) and
// writes the exclusive offsets; the last tile also writes the total.
// ---------------------------------------------------------------------------
constexpr int SCAN_T = 1024, SCAN_ROUNDS = 4;
constexpr int SCAN_TILE = SCAN_T * 4 * SCAN_ROUNDS;

// The four counts at cnt[base .. base + 4), zero past n; base is a multiple of 4 (16-byte aligned).
__device__ __forceinline__ int4 scan_load4(const int32_t *cnt, int64_t n, int64_t base)
{
    int4 q = make_int4(0, 0, 0, 0);
    if (base + 4 <= n) {
        q = *reinterpret_cast<const int4 *>(cnt + base);
    } else {
        if (base < n) q.x = cnt[base];
        if (base + 1 < n) q.y = cnt[base + 1];
        if (base + 2 < n) q.z = cnt[base + 2];
    }
    return q;
}

__global__ void __launch_bounds__(SCAN_T) k_scan_reduce(const int32_t *cnt, int64_t n, int32_t *bsum)
{
    __shared__ int wsum[SCAN_T / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t t0 = (int64_t)blockIdx.x * SCAN_TILE + 4 * (int64_t)threadIdx.x;
    int4 q[SCAN_ROUNDS];
#pragma unroll
    for (int r = 0; r < SCAN_ROUNDS; r++) q[r] = scan_load4(cnt, n, t0 + (int64_t)r * 4 * SCAN_T);
    int s = 0;
#pragma unroll
    for (int r = 0; r < SCAN_ROUNDS; r++) s += q[r].x + q[r].y + q[r].z + q[r].w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) wsum[wid] = s;
    __syncthreads();
    if (wid == 0) {
        int t = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (lane == 0) bsum[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(SCAN_T, 2) k_scan_down(const int32_t *cnt, int64_t n, const int32_t *bsum,
                                                       int32_t *start)
{
    static_assert(SCAN_T == 1024, "32 warps: one lane of warp 0 per warp");
    __shared__ int wex[SCAN_ROUNDS][SCAN_T / 32];   // exclusive offset of each warp in each round
    __shared__ int wpre[SCAN_T / 32];
    __shared__ int tile_end;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int tile = (int)blockIdx.x;
    const int64_t t0 = (int64_t)tile * SCAN_TILE + 4 * (int64_t)threadIdx.x;
    int v[SCAN_ROUNDS], inc[SCAN_ROUNDS];
#pragma unroll
    for (int r = 0; r < SCAN_ROUNDS; r++) {
        const int4 q = scan_load4(cnt, n, t0 + (int64_t)r * 4 * SCAN_T);
        inc[r] = v[r] = q.x + q.y + q.z + q.w;
    }
    // this thread's share of the sums of tiles 0 .. tile-1
    int pre = 0;
    const int nv = tile >> 2;
    for (int i = (int)threadIdx.x; i < nv; i += SCAN_T) {
        const int4 b = reinterpret_cast<const int4 *>(bsum)[i];
        pre += b.x + b.y + b.z + b.w;
    }
    if ((int)threadIdx.x < (tile & 3)) pre += bsum[4 * nv + (int)threadIdx.x];
    // inclusive warp scans of the thread sums of every round, and the warp sum of pre
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
        for (int r = 0; r < SCAN_ROUNDS; r++) {
            const int y = __shfl_up_sync(0xffffffffu, inc[r], o);
            if (lane >= o) inc[r] += y;
        }
        pre += __shfl_xor_sync(0xffffffffu, pre, o);
    }
    if (lane == 31) {
#pragma unroll
        for (int r = 0; r < SCAN_ROUNDS; r++) wex[r][wid] = inc[r];
    }
    if (lane == 0) wpre[wid] = pre;
    __syncthreads();
    if (wid == 0) {
        int w[SCAN_ROUNDS], z[SCAN_ROUNDS];
#pragma unroll
        for (int r = 0; r < SCAN_ROUNDS; r++) z[r] = w[r] = wex[r][lane];
        int p = wpre[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
            for (int r = 0; r < SCAN_ROUNDS; r++) {
                const int y = __shfl_up_sync(0xffffffffu, z[r], o);
                if (lane >= o) z[r] += y;
            }
            p += __shfl_xor_sync(0xffffffffu, p, o);
        }
        // round r starts after the tiles before this one and after rounds 0 .. r-1 of this tile
        int carry = p;
#pragma unroll
        for (int r = 0; r < SCAN_ROUNDS; r++) {
            wex[r][lane] = carry + z[r] - w[r];
            carry += __shfl_sync(0xffffffffu, z[r], 31);
        }
        if (lane == 0) tile_end = carry;
    }
    __syncthreads();
    // the counts again (from L1: this CTA read them above), to keep two CTAs of registers per SM
#pragma unroll
    for (int r = 0; r < SCAN_ROUNDS; r++) {
        const int64_t base = t0 + (int64_t)r * 4 * SCAN_T;
        const int4 q = scan_load4(cnt, n, base);
        const int e = wex[r][wid] + inc[r] - v[r];
        const int4 o = make_int4(e, e + q.x, e + q.x + q.y, e + q.x + q.y + q.z);
        if (base + 4 <= n) {
            *reinterpret_cast<int4 *>(start + base) = o;
        } else {
            if (base < n) start[base] = o.x;
            if (base + 1 < n) start[base + 1] = o.y;
            if (base + 2 < n) start[base + 2] = o.z;
        }
    }
    if (tile == (int)gridDim.x - 1 && threadIdx.x == 0) start[n] = tile_end;
}

template <class T>
__global__ void __launch_bounds__(256) k_scatter(const Particle<T> *in, Particle<T> *out, int64_t np,
                                                 const int32_t *start, int32_t *count)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const Particle<T> P = in[i];
    const int r = atomicSub(&count[P.cell], 1) - 1;
    out[start[P.cell] + r] = P;
}

// ---------------------------------------------------------------------------
// Particle I/O: f64 (x, y, z) rows <-> cell + offset records.
// ---------------------------------------------------------------------------
template <class T>
__global__ void k_load(const double *pos, const double *mom, int64_t first, int64_t cnt, int N,
                       Particle<T> *out, int32_t *count, int *nonfinite)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= cnt) return;
    Particle<T> P{};
    int ic[3];
    bool bad = false;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        double x = pos[3 * k + d];
        const double u = mom[3 * k + d];
        bad |= !isfinite(x) || !isfinite(u);
        if (!isfinite(x)) x = 0.0;   // keeps the cell index valid; the caller rejects the input
        x -= floor(x);
        if (x >= 1.0) x = 0.0;
        double s = x * N;
        double fl = floor(s);
        int c = (int)fl;
        double f = s - fl;
        if (c >= N) c -= N;
        ic[d] = c;
        P.f[d] = (T)f;
        if (P.f[d] >= T(1)) {  // rounding of f to the storage type
            P.f[d] = T(0);
            ic[d] = (c + 1) % N;
        }
        P.u[d] = (T)u;
    }
    if (bad) *nonfinite = 1;
    P.cell = (ic[2] * N + ic[1]) * N + ic[0];
    P.id = (uint32_t)(first + k);
    out[first + k] = P;
    atomicAdd(&count[P.cell], 1);
}

// Packed host records (cell, 3 f32 offsets, 3 f32 momenta; 28 bytes) -> device records, checked.  A block
// takes PK_P records (14336 bytes) and moves them between the caller's array and shared memory with 16-byte
// accesses at consecutive addresses (the array may be pinned host memory read across the CPU-GPU link, where
// narrow accesses waste most of each transfer); vec = 0 (an array not 16-byte aligned) uses 4-byte accesses.
constexpr int PK_P = 512;
constexpr int PK_VEC = PK_P * (int)sizeof(pm_packed_particle) / 16;
static_assert(sizeof(pm_packed_particle) == 28 && PK_P * 28 % 16 == 0, "packed record");

__device__ __forceinline__ void pk_copy(uint4 *dst, const uint4 *src, int bytes, int vec)
{
    const int nv = vec ? bytes / 16 : 0;
    for (int v = threadIdx.x; v < nv; v += blockDim.x) dst[v] = src[v];
    for (int w = nv * 4 + threadIdx.x; w < bytes / 4; w += blockDim.x)
        reinterpret_cast<uint32_t *>(dst)[w] = reinterpret_cast<const uint32_t *>(src)[w];
}

// one packed record as the particle it stands for; a record with a cell outside [0, nc), an offset outside
// [0, 1) or a non-finite momentum is flagged (*bad = 1) and kept at a valid cell and offset
__device__ __forceinline__ Particle<float> unpack_record(const pm_packed_particle &q, uint32_t id, int64_t nc, int *bad)
{
    Particle<float> P;
    P.cell = q.cell;
    P.id = id;
    bool ok = q.cell >= 0 && (int64_t)q.cell < nc;
#pragma unroll
    for (int d = 0; d < 3; d++) {
        P.f[d] = q.f[d];
        P.u[d] = q.u[d];
        ok = ok && q.f[d] >= 0.f && q.f[d] < 1.f && isfinite(q.u[d]);
    }
    if (!ok) {   // keeps the cell index valid; the caller rejects the input
        *bad = 1;
        P.cell = 0;
        P.f[0] = P.f[1] = P.f[2] = 0.f;
    }
    return P;
}

__global__ void __launch_bounds__(256) k_load_packed(const pm_packed_particle *in, int64_t first, int64_t cnt,
                                                     int64_t nc, Particle<float> *out, int32_t *count, int *bad, int vec)
{
    __shared__ uint4 sb[PK_VEC];
    const int64_t base = (int64_t)blockIdx.x * PK_P;
    const int nb = (int)min((int64_t)PK_P, cnt - base);
    pk_copy(sb, reinterpret_cast<const uint4 *>(in + base), nb * 28, vec);
    __syncthreads();
    const pm_packed_particle *sq = reinterpret_cast<const pm_packed_particle *>(sb);
    for (int j = threadIdx.x; j < nb; j += blockDim.x) {
        const Particle<float> P = unpack_record(sq[j], (uint32_t)(first + base + j), nc, bad);
        out[first + base + j] = P;
        atomicAdd(&count[P.cell], 1);
    }
}

// The two passes of a counting sort straight from packed records in device memory: the histogram (with the
// record checks), then, after the scan, each record placed at its cell's slot as a particle.  Against loading
// the records into the particle buffer and sorting that, the particle buffer is written once and not read.
__global__ void __launch_bounds__(256) k_count_packed(const pm_packed_particle *in, int64_t cnt, int64_t nc,
                                                      int32_t *count, int *bad, int vec)
{
    __shared__ uint4 sb[PK_VEC];
    const int64_t base = (int64_t)blockIdx.x * PK_P;
    const int nb = (int)min((int64_t)PK_P, cnt - base);
    pk_copy(sb, reinterpret_cast<const uint4 *>(in + base), nb * 28, vec);
    __syncthreads();
    const pm_packed_particle *sq = reinterpret_cast<const pm_packed_particle *>(sb);
    for (int j = threadIdx.x; j < nb; j += blockDim.x)
        atomicAdd(&count[unpack_record(sq[j], 0u, nc, bad).cell], 1);
}

__global__ void __launch_bounds__(256) k_scatter_packed(const pm_packed_particle *in, int64_t cnt, int64_t nc,
                                                        const int32_t *start, int32_t *count, Particle<float> *out,
                                                        int *bad, int vec)
{
    __shared__ uint4 sb[PK_VEC];
    const int64_t base = (int64_t)blockIdx.x * PK_P;
    const int nb = (int)min((int64_t)PK_P, cnt - base);
    pk_copy(sb, reinterpret_cast<const uint4 *>(in + base), nb * 28, vec);
    __syncthreads();
    const pm_packed_particle *sq = reinterpret_cast<const pm_packed_particle *>(sb);
    for (int j = threadIdx.x; j < nb; j += blockDim.x) {
        const Particle<float> P = unpack_record(sq[j], (uint32_t)(base + j), nc, bad);
        const int r = atomicSub(&count[P.cell], 1) - 1;
        out[start[P.cell] + r] = P;
    }
}

// Device records in id order -> packed records (same staging as the load).
__global__ void __launch_bounds__(256) k_store_packed(const Particle<float> *byid, int64_t first, int64_t cnt,
                                                      pm_packed_particle *out, int vec)
{
    __shared__ uint4 sb[PK_VEC];
    const int64_t base = (int64_t)blockIdx.x * PK_P;
    const int nb = (int)min((int64_t)PK_P, cnt - base);
    pm_packed_particle *sq = reinterpret_cast<pm_packed_particle *>(sb);
    for (int j = threadIdx.x; j < nb; j += blockDim.x) {
        const Particle<float> P = byid[first + base + j];
        pm_packed_particle q;
        q.cell = P.cell;
#pragma unroll
        for (int d = 0; d < 3; d++) {
            q.f[d] = P.f[d];
            q.u[d] = P.u[d];
        }
        sq[j] = q;
    }
    __syncthreads();
    pk_copy(reinterpret_cast<uint4 *>(out + base), sb, nb * 28, vec);
}

template <class T>
__global__ void k_unpermute(const Particle<T> *in, Particle<T> *out, int64_t np)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const Particle<T> P = in[i];
    out[P.id] = P;
}

// Particle records (in id order) -> f64 positions and momenta [k][3].  A block stages 512
// particles in shared memory and writes them with 16-byte stores at consecutive addresses, which
// keeps the writes full-line even when the destination is pinned host memory across the link.
constexpr int ST_P = 512;
template <class T>
__global__ void __launch_bounds__(256) k_store(const Particle<T> *byid, int64_t first, int64_t cnt, int N,
                                               double inv_n, double *pos, double *mom, int vec)
{
    __shared__ double sp[3 * ST_P], su[3 * ST_P];
    const int64_t base = (int64_t)blockIdx.x * ST_P;
    const int nb = (int)min((int64_t)ST_P, cnt - base);
    for (int j = threadIdx.x; j < nb; j += blockDim.x) {
        const Particle<T> P = byid[first + base + j];
        const int ic[3] = {P.cell % N, (P.cell / N) % N, P.cell / (N * N)};
#pragma unroll
        for (int d = 0; d < 3; d++) {
            sp[3 * j + d] = ((double)ic[d] + (double)P.f[d]) * inv_n;
            su[3 * j + d] = (double)P.u[d];
        }
    }
    __syncthreads();
    const int nv = 3 * nb;
    double *dst[2] = {pos ? pos + 3 * base : nullptr, mom ? mom + 3 * base : nullptr};
    const double *src[2] = {sp, su};
#pragma unroll
    for (int a = 0; a < 2; a++) {
        if (!dst[a]) continue;
        if (vec) {
            double2 *o = reinterpret_cast<double2 *>(dst[a]);
            for (int v = threadIdx.x; v < nv / 2; v += blockDim.x) o[v] = make_double2(src[a][2 * v], src[a][2 * v + 1]);
            if ((nv & 1) && threadIdx.x == 0) dst[a][nv - 1] = src[a][nv - 1];
        } else {
            for (int v = threadIdx.x; v < nv; v += blockDim.x) dst[a][v] = src[a][v];
        }
    }
}

// CIC mass density contrast delta = rho/omega_m - 1 (diagnostic, global FP64 atomics).
template <class T>
__global__ void k_density_acc(const Particle<T> *part, int64_t np, int N, double q, double *rho)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    const Particle<T> P = part[i];
    const int ix = P.cell % N, iy = (P.cell / N) % N, iz = P.cell / (N * N);
    const double f[3] = {(double)P.f[0], (double)P.f[1], (double)P.f[2]};
#pragma unroll
    for (int dz = 0; dz < 2; dz++)
#pragma unroll
        for (int dy = 0; dy < 2; dy++)
#pragma unroll
            for (int dx = 0; dx < 2; dx++) {
                const double w = (dx ? f[0] : 1 - f[0]) * (dy ? f[1] : 1 - f[1]) * (dz ? f[2] : 1 - f[2]);
                const int64_t g = ((int64_t)wrapi(iz + dz, N) * N + wrapi(iy + dy, N)) * N + wrapi(ix + dx, N);
                atomicAdd(&rho[g], q * w);
            }
}

template <class T>
__global__ void k_density_fin(const double *rho, int64_t n, T *out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (T)(rho[i] - 1.0);
}

template <class T> __global__ void k_to_f64(const T *s, double *d, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) d[i] = (double)s[i];
}

template <class T> __global__ void k_from_f64(const double *s, T *d, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) d[i] = (T)s[i];
}

__global__ void k_check_finite(const double *d, int64_t n, int *flag)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && !isfinite(d[i])) *flag = 1;
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

template <class T> DepParams<T> dep_params(const Ctx &c, const StepScalars &s)
{
    DepParams<T> p{};
    p.part = reinterpret_cast<const Particle<T> *>(c.part[c.cur]);
    p.start = c.start;
    p.phi1 = reinterpret_cast<const T *>(c.phi[c.iphi_prev]);
    p.chi1 = reinterpret_cast<const T *>(c.chi);
    p.phi2 = reinterpret_cast<const T *>(c.phi[c.iphi_prev2]);
    for (int i = 0; i < 9; i++) p.out.p[i] = reinterpret_cast<T *>(c.src) + (size_t)i * c.nc;
    p.k0slots = c.dscal + 8;
    p.N = c.N;
    p.nt = c.N / TILE;
    p.newtonian = s.newtonian;
    p.full = !(s.newtonian || s.bootstrap);
    p.use_fields = p.full;
    p.a = (T)s.a;
    p.a2 = (T)(s.a * s.a);
    p.mass = (T)s.mass;
    const double n3 = (double)c.nc;
    double rb;
    if (s.newtonian) {
        p.G = (T)(s.four_pi_g / s.a * n3);
        rb = s.omega_m / n3;
    } else {
        p.G = (T)(s.four_pi_g / (s.a * s.a) * n3);
        rb = s.a * s.omega_m / n3;
    }
    p.rb_hi = (T)rb;
    p.rb_lo = (T)(rb - (double)p.rb_hi);
    p.c1 = (T)s.c_phi_dt;
    p.c2 = (T)s.c_phi_h2;
    p.inv_dt2 = (T)s.inv_dtau_prev2;
    p.halfN = (T)(0.5 * c.N);
    p.full_hc = s.full_hc;
    p.write_f = !(s.b_space && !s.b_seed);
    p.hc = (T)s.hc;
    p.n2 = (T)((double)c.N * (double)c.N);
    p.inv_g = 1.0 / (s.four_pi_g / (s.a * s.a) * n3);
    return p;
}

template <class T, int V> void dep_attrs()
{
    static std::atomic<uint64_t> attr{0};
    if (first_on_device(attr)) {
        cudaFuncSetAttribute(k_project<T, V>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dep_smem<T, V>());
        cudaFuncSetAttribute(k_project_batch<T, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)dep_smem<T, V>());
    }
}

template <class T>
void launch_project(Ctx &c, const StepScalars &s)
{
    const DepParams<T> p = dep_params<T>(c, s);
    cudaMemsetAsync(c.dscal + 8, 0, sizeof(double) * NK0SLOTS, c.stream);
    const int ntiles = (c.N / TILE) * (c.N / TILE) * (c.N / TILE);
    if (c.dep_shape == 1) {
        dep_attrs<T, 1>();
        k_project<T, 1><<<ntiles, DEP_THREADS, dep_smem<T, 1>(), c.stream>>>(p);
    } else {
        dep_attrs<T, 0>();
        k_project<T, 0><<<ntiles, DEP_THREADS, dep_smem<T, 0>(), c.stream>>>(p);
    }
    k_k0_reduce<<<1, 1024, 0, c.stream>>>(c.dscal);
    c.launches += 2;
}

// One deposit launch over several boxes of one precision and one deposit shape (batches of MAXBATCH).
template <class T>
void launch_project_batch(Ctx *const *cs, const StepScalars *ss, int n, int shape, cudaStream_t st)
{
    for (int b0 = 0; b0 < n; b0 += MAXBATCH) {
        const int nb = std::min(MAXBATCH, n - b0);
        static DepBatch<T> q;   // host staging of the launch parameters (copied at launch)
        K0Batch kq{};
        q.nbox = nb;
        q.first[0] = 0;
        for (int i = 0; i < nb; i++) {
            Ctx &c = *cs[b0 + i];
            q.box[i] = dep_params<T>(c, ss[b0 + i]);
            q.first[i + 1] = q.first[i] + (c.N / TILE) * (c.N / TILE) * (c.N / TILE);
            kq.dscal[i] = c.dscal;
            cudaMemsetAsync(c.dscal + 8, 0, sizeof(double) * NK0SLOTS, st);
            c.launches += 2;
        }
        if (shape == 1) {
            dep_attrs<T, 1>();
            k_project_batch<T, 1><<<q.first[nb], DEP_THREADS, dep_smem<T, 1>(), st>>>(q);
        } else {
            dep_attrs<T, 0>();
            k_project_batch<T, 0><<<q.first[nb], DEP_THREADS, dep_smem<T, 0>(), st>>>(q);
        }
        k_k0_reduce_batch<<<nb, 1024, 0, st>>>(kq);
    }
}

template <class T> KdParams<T> kd_params(const Ctx &c, const StepScalars &s)
{
    KdParams<T> p{};
    p.part = reinterpret_cast<Particle<T> *>(c.part[c.cur]);
    p.start = c.start;
    p.count = c.count;
    p.nt = c.N / KT;
    const T *B = reinterpret_cast<const T *>(c.B);
    p.phi = reinterpret_cast<const T *>(c.phi[c.iphi_new]);
    p.chi = reinterpret_cast<const T *>(c.chi);
    p.Bx = B;
    p.By = B + c.nc;
    p.Bz = B + 2 * c.nc;
    p.np = c.np;
    p.N = c.N;
    p.newtonian = s.newtonian;
    p.a = (T)s.a;
    p.a2 = (T)(s.a * s.a);
    p.a_half2 = (T)(s.a_half * s.a_half);
    p.inv_a_half = (T)(1.0 / s.a_half);
    p.dt_kick = (T)s.dtau_kick;
    p.dt_drift_N = (T)(s.dtau * c.N);
    p.halfN = (T)(0.5 * c.N);
    return p;
}

template <class T> void kd_attrs()
{
    static std::atomic<uint64_t> attr{0};
    if (first_on_device(attr)) {
        cudaFuncSetAttribute(k_kick_drift<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kd_smem<T>());
        cudaFuncSetAttribute(k_kick_batch<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kd_smem<T>());
    }
}

template <class T>
void launch_kick_drift(Ctx &c, const StepScalars &s)
{
    kd_attrs<T>();
    const KdParams<T> p = kd_params<T>(c, s);
    const int ntiles = (c.N / KT) * (c.N / KT) * (c.N / KT);
    k_kick_drift<T><<<ntiles, KD_THREADS, kd_smem<T>(), c.stream>>>(p);
    c.launches++;
}

// One gather + kick + drift launch over several boxes of one precision (batches of MAXBATCH).
template <class T>
void launch_kick_batch(Ctx *const *cs, const StepScalars *ss, int n, cudaStream_t st)
{
    kd_attrs<T>();
    for (int b0 = 0; b0 < n; b0 += MAXBATCH) {
        const int nb = std::min(MAXBATCH, n - b0);
        static KdBatch<T> q;
        q.nbox = nb;
        q.first[0] = 0;
        for (int i = 0; i < nb; i++) {
            Ctx &c = *cs[b0 + i];
            q.box[i] = kd_params<T>(c, ss[b0 + i]);
            q.first[i + 1] = q.first[i] + (c.N / KT) * (c.N / KT) * (c.N / KT);
            c.launches++;
        }
        k_kick_batch<T><<<q.first[nb], KD_THREADS, kd_smem<T>(), st>>>(q);
    }
}

// Time the deposit of the context's current state with each chunk capacity and keep the fastest.  The trial
// deposits write into the spectrum buffer, which holds nothing between steps (9 half spectra hold more than
// 9 real fields), so the sources the caller can read stay as they were; the k = 0 scalar they also write is
// recomputed by the next projection before the solve reads it.
template <class T>
int tune_deposit_shape(Ctx &c, const StepScalars &s)
{
    void *const src = c.src;
    c.src = c.spec;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int best_v = 0;
    for (int v = 0; v < NDEPSHAPES; v++) {
        c.dep_shape = v;
        launch_project<T>(c, s);   // warm-up (and the first launch of the shape)
        cudaEventRecord(e0, c.stream);
        for (int r = 0; r < 3; r++) launch_project<T>(c, s);
        cudaEventRecord(e1, c.stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            best_v = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c.src = src;
    c.dep_shape = best_v;
    return best_v;
}

void launch_scan(Ctx &c)
{
    const int64_t nb = (c.nc + SCAN_TILE - 1) / SCAN_TILE;
    k_scan_reduce<<<(unsigned)nb, SCAN_T, 0, c.stream>>>(c.count, c.nc, c.blocksum);
    k_scan_down<<<(unsigned)nb, SCAN_T, 0, c.stream>>>(c.count, c.nc, c.blocksum, c.start);
    c.launches += 2;
}

template <class T>
void launch_sort(Ctx &c)
{
    launch_scan(c);
    c.mark(EV_SCAN);
    const int o = 1 - c.cur;
    k_scatter<T><<<nblk(c.np, 256), 256, 0, c.stream>>>(reinterpret_cast<const Particle<T> *>(c.part[c.cur]),
                                                         reinterpret_cast<Particle<T> *>(c.part[o]), c.np,
                                                         c.start, c.count);
    c.launches++;
    c.cur = o;
}

template <class T>
void launch_load_particles(Ctx &c, const double *d_pos, const double *d_mom, int64_t first, int64_t count,
                           int *d_nonfinite)
{
    k_load<T><<<nblk(count, 256), 256, 0, c.stream>>>(d_pos, d_mom, first, count, c.N,
                                                      reinterpret_cast<Particle<T> *>(c.part[c.cur]), c.count,
                                                      d_nonfinite);
}

template <class T>
void launch_store_particles_scatter(Ctx &c, double *, double *)
{
    const int o = 1 - c.cur;
    k_unpermute<T><<<nblk(c.np, 256), 256, 0, c.stream>>>(reinterpret_cast<const Particle<T> *>(c.part[c.cur]),
                                                           reinterpret_cast<Particle<T> *>(c.part[o]), c.np);
}

template <class T>
void launch_store_particles(Ctx &c, double *d_pos, double *d_mom, int64_t first, int64_t count)
{
    const int o = 1 - c.cur;
    // 16-byte stores need 16-byte aligned arrays (the block offsets are multiples of 3 * 512 doubles)
    const int vec = ((reinterpret_cast<uintptr_t>(d_pos) | reinterpret_cast<uintptr_t>(d_mom)) & 15) == 0;
    k_store<T><<<nblk(count, ST_P), 256, 0, c.stream>>>(reinterpret_cast<const Particle<T> *>(c.part[o]), first,
                                                        count, c.N, 1.0 / (double)c.N, d_pos, d_mom, vec);
}

void launch_load_packed(Ctx &c, const pm_packed_particle *in, int64_t first, int64_t count, int *d_bad)
{
    const int vec = (reinterpret_cast<uintptr_t>(in) & 15) == 0;
    k_load_packed<<<nblk(count, PK_P), 256, 0, c.stream>>>(in, first, count, c.nc,
                                                           reinterpret_cast<Particle<float> *>(c.part[c.cur]), c.count,
                                                           d_bad, vec);
}

void launch_put_packed_sorted(Ctx &c, const pm_packed_particle *in, int *d_bad)
{
    const int vec = (reinterpret_cast<uintptr_t>(in) & 15) == 0;
    const unsigned nb = nblk(c.np, PK_P);
    k_count_packed<<<nb, 256, 0, c.stream>>>(in, c.np, c.nc, c.count, d_bad, vec);
    launch_scan(c);
    const int o = 1 - c.cur;
    k_scatter_packed<<<nb, 256, 0, c.stream>>>(in, c.np, c.nc, c.start, c.count,
                                               reinterpret_cast<Particle<float> *>(c.part[o]), d_bad, vec);
    c.launches += 2;
    c.cur = o;
}

void launch_store_packed(Ctx &c, pm_packed_particle *out, int64_t first, int64_t count)
{
    const int vec = (reinterpret_cast<uintptr_t>(out) & 15) == 0;
    k_store_packed<<<nblk(count, PK_P), 256, 0, c.stream>>>(
        reinterpret_cast<const Particle<float> *>(c.part[1 - c.cur]), first, count, out, vec);
}

template <class T>
void launch_density(Ctx &c, void *real_out)
{
    double *rho = reinterpret_cast<double *>(c.spec);  // scratch: nc doubles fit in the spectra block
    cudaMemsetAsync(rho, 0, sizeof(double) * c.nc, c.stream);
    const double q = (double)c.nc / (double)c.np;  // N^3 m / omega_m
    k_density_acc<T><<<nblk(c.np, 256), 256, 0, c.stream>>>(reinterpret_cast<const Particle<T> *>(c.part[c.cur]),
                                                             c.np, c.N, q, rho);
    k_density_fin<T><<<nblk(c.nc, 256), 256, 0, c.stream>>>(rho, c.nc, reinterpret_cast<T *>(real_out));
}

template <class T>
void launch_to_f64(Ctx &c, const void *src, double *dst, int64_t n)
{
    k_to_f64<T><<<nblk(n, 256), 256, 0, c.stream>>>(reinterpret_cast<const T *>(src), dst, n);
}

template <class T>
void launch_from_f64(Ctx &c, const double *src, void *dst, int64_t n)
{
    k_from_f64<T><<<nblk(n, 256), 256, 0, c.stream>>>(src, reinterpret_cast<T *>(dst), n);
}

template <class T>
void launch_check_finite(Ctx &c, const double *d, int64_t n, int *d_flag)
{
    k_check_finite<<<nblk(n, 256), 256, 0, c.stream>>>(d, n, d_flag);
}

#define PM_INST(T)                                                                          \
    template void launch_project<T>(Ctx &, const StepScalars &);                            \
    template void launch_project_batch<T>(Ctx *const *, const StepScalars *, int, int, cudaStream_t); \
    template void launch_kick_batch<T>(Ctx *const *, const StepScalars *, int, cudaStream_t); \
    template int tune_deposit_shape<T>(Ctx &, const StepScalars &);                         \
    template void launch_kick_drift<T>(Ctx &, const StepScalars &);                         \
    template void launch_sort<T>(Ctx &);                                                    \
    template void launch_load_particles<T>(Ctx &, const double *, const double *, int64_t,  \
                                           int64_t, int *);                                 \
    template void launch_store_particles<T>(Ctx &, double *, double *, int64_t, int64_t);   \
    template void launch_store_particles_scatter<T>(Ctx &, double *, double *);             \
    template void launch_density<T>(Ctx &, void *);                                         \
    template void launch_to_f64<T>(Ctx &, const void *, double *, int64_t);                 \
    template void launch_from_f64<T>(Ctx &, const double *, void *, int64_t);               \
    template void launch_check_finite<T>(Ctx &, const double *, int64_t, int *);
PM_INST(double)
PM_INST(float)

}  // namespace pm
