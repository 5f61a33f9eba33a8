// Fourier-space solution of the field equations (Sec. 3.1), one thread per
// mode of the half spectrum [kz][ky][kx], kx in [0, N/2]:
//
//   phi_k = -R_k / (kt^2 + 3Hc/dtau_{n-1} + 3Hc^2)          (Eq. NewtonHc, backward difference)
//   chi_k = -3/(4 kt^4) kt_i kt_j Sig_ij,k                  (scalar part of Eq. spacespace)
//   B_i,k = 4 (delta_ij - kt_i kt_j / kt^2) F_j,k / kt^2    (Eq. momentumcontraint, spin-1 part)
//   h_A   : h'' + 2Hc h' + kt^2 h = e^A_ij Sig_ij, one implicit-midpoint step
//
// or, with B from the spin-1 part of Eq. spacespace ((d_tau + 2Hc) B_j = W_j, d_i -> i kt_i):
//   W_j = -i (delta_jl - kt_j kt_l / kt^2) kt_i Sig_il,k / kt^2
//   B_j,k = (a_{n-1} / a_n)^2 B_j,k(previous step) + dtau_{n-1} W_j      (backward Euler in a^2 B)
//
// with kt_i = 2N sin(pi n_i / N), so kt^2 is the eigenvalue of minus the
// 7-point Laplacian.  The k = 0 mode of phi comes from the FP64 particle sum
// of the projection; chi, B and h vanish at k = 0 and on Nyquist modes.
// Outputs are scaled by 1/N^3 so that the inverse transforms need no
// normalisation.
#include "pm_internal.cuh"

namespace pm {

namespace {

template <class T> struct SolveParams {
    void *spec;        // 9 half spectra: R, Fx, Fy, Fz, Sxx, Sxy, Sxz, Syy, Syz
    void *tens;        // 4 half spectra: h+, hx, h+', hx'
    const T *ktab;     // ktilde per DFT index
    double *dscal;     // [0] particle excess sum, [1 + ring] mean phi per ring slot
    int imean_prev, imean_new;
    int N;
    int64_t nh;
    int full, newtonian, bootstrap;
    double four_pi_g_a2, c1, c2;   // FP64 copies for the k = 0 mode
    T cphi, inv_n3, hc_half, dtau;
    void *bstate;      // 3 half spectra of B_k (unnormalised), B from Eq. spacespace only
    int b_space, b_seed;
    T b_decay, dtau_prev;
};

template <class T>
__global__ void __launch_bounds__(256) k_solve(SolveParams<T> p)
{
    using C = typename Cplx<T>::type;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= p.nh) return;
    const int N = p.N, h = N / 2 + 1;
    const int kx = (int)(e % h);
    const int64_t r = e / h;
    const int ky = (int)(r % N), kz = (int)(r / N);
    const int nv[3] = {kx, ky <= N / 2 ? ky : ky - N, kz <= N / 2 ? kz : kz - N};
    const T kt[3] = {p.ktab[kx], p.ktab[ky], p.ktab[kz]};
    const T k2 = kt[0] * kt[0] + kt[1] * kt[1] + kt[2] * kt[2];
    const bool zero = (kx == 0 && ky == 0 && kz == 0);
    const bool nyq = (2 * kx == N) || (2 * abs(nv[1]) == N) || (2 * abs(nv[2]) == N);
    C *S = reinterpret_cast<C *>(p.spec);
    C *H = reinterpret_cast<C *>(p.tens);
    const int64_t nh = p.nh;
    // every input of this mode, loaded before any output is stored
    const bool fullmode = p.full && !zero && !nyq;
    const bool bint = p.b_space && !p.b_seed;
    C inR, inS[5], inH[4], inF[3];
    if (!zero) inR = S[e];
    if (fullmode) {
#pragma unroll
        for (int c = 0; c < 5; c++) inS[c] = S[(4 + c) * nh + e];
#pragma unroll
        for (int c = 0; c < 4; c++) inH[c] = H[c * nh + e];
        const C *FB = bint ? reinterpret_cast<const C *>(p.bstate) : S + nh;
#pragma unroll
        for (int c = 0; c < 3; c++) inF[c] = FB[c * nh + e];
    }

    // scalar potential phi
    if (zero) {
        double mean_phi = 0.0;
        if (!p.newtonian) {
            double mean_r = p.four_pi_g_a2 * p.dscal[0];
            if (!p.bootstrap) mean_r -= p.c1 * p.dscal[1 + p.imean_prev];
            mean_phi = -mean_r / (p.c1 + p.c2);
        }
        p.dscal[1 + p.imean_new] = mean_phi;
        C v;
        v.x = (T)mean_phi;
        v.y = 0;
        S[0] = v;
    } else {
        C R = inR;
        const T f = -p.inv_n3 / (k2 + p.cphi);
        R.x *= f;
        R.y *= f;
        S[e] = R;
    }
    if (!p.full) return;
    if (zero || nyq) {
        C z;
        z.x = 0;
        z.y = 0;
#pragma unroll
        for (int c = 1; c <= 4; c++) S[c * nh + e] = z;
#pragma unroll
        for (int c = 0; c < 4; c++) H[c * nh + e] = z;
        if (p.b_space) {
            C *BS = reinterpret_cast<C *>(p.bstate);
#pragma unroll
            for (int c = 0; c < 3; c++) BS[c * nh + e] = z;
        }
        return;
    }
    // trace-free Sig as a symmetric matrix (Sig_zz = -Sig_xx - Sig_yy)
    const C sxx = inS[0], sxy = inS[1], sxz = inS[2], syy = inS[3], syz = inS[4];
    C szz;
    szz.x = -sxx.x - syy.x;
    szz.y = -sxx.y - syy.y;
    const C Sm[3][3] = {{sxx, sxy, sxz}, {sxy, syy, syz}, {sxz, syz, szz}};

    // tensor sector: polarisation basis from the axis with the smallest |n_i|
    {
        const T kn = sqrt(k2);
        const T kh[3] = {kt[0] / kn, kt[1] / kn, kt[2] / kn};
        int m = 0;
        if (abs(nv[1]) < abs(nv[m])) m = 1;
        if (abs(nv[2]) < abs(nv[m])) m = 2;
        T e1[3] = {-kh[m] * kh[0], -kh[m] * kh[1], -kh[m] * kh[2]};
        e1[m] += T(1);
        const T l = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
#pragma unroll
        for (int d = 0; d < 3; d++) e1[d] /= l;
        const T e2[3] = {kh[1] * e1[2] - kh[2] * e1[1], kh[2] * e1[0] - kh[0] * e1[2],
                         kh[0] * e1[1] - kh[1] * e1[0]};
        const T is2 = T(0.70710678118654752440084436210484903928);
        C sp, sx;
        sp.x = sp.y = sx.x = sx.y = 0;
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                const T ep = (e1[i] * e1[j] - e2[i] * e2[j]) * is2;
                const T ex = (e1[i] * e2[j] + e2[i] * e1[j]) * is2;
                sp.x += ep * Sm[i][j].x;
                sp.y += ep * Sm[i][j].y;
                sx.x += ex * Sm[i][j].x;
                sx.y += ex * Sm[i][j].y;
            }
        // implicit midpoint: (I - dt/2 A) y' = (I + dt/2 A) y + dt (0, s), A = [[0,1],[-k2,-2Hc]]
        const T dt = p.dtau, hc = p.hc_half;
        const T m12 = -T(0.5) * dt, m21 = T(0.5) * dt * k2, m22 = T(1) + dt * hc;
        const T p12 = T(0.5) * dt, p21 = -T(0.5) * dt * k2, p22 = T(1) - dt * hc;
        const T idet = T(1) / (m22 - m12 * m21);
#pragma unroll
        for (int a = 0; a < 2; a++) {
            const C s = a == 0 ? sp : sx;
            C hh = inH[a], vv = inH[2 + a];
            C r1, r2;
            r1.x = hh.x + p12 * vv.x;
            r1.y = hh.y + p12 * vv.y;
            r2.x = p21 * hh.x + p22 * vv.x + dt * s.x;
            r2.y = p21 * hh.y + p22 * vv.y + dt * s.y;
            hh.x = (m22 * r1.x - m12 * r2.x) * idet;
            hh.y = (m22 * r1.y - m12 * r2.y) * idet;
            vv.x = (-m21 * r1.x + r2.x) * idet;
            vv.y = (-m21 * r1.y + r2.y) * idet;
            H[a * nh + e] = hh;
            H[(2 + a) * nh + e] = vv;
        }
    }
    // scalar slip chi (written over Sxx)
    {
        C kks;
        kks.x = kks.y = 0;
#pragma unroll
        for (int i = 0; i < 3; i++)
#pragma unroll
            for (int j = 0; j < 3; j++) {
                kks.x += kt[i] * kt[j] * Sm[i][j].x;
                kks.y += kt[i] * kt[j] * Sm[i][j].y;
            }
        const T f = -T(0.75) / (k2 * k2) * p.inv_n3;
        C chi;
        chi.x = f * kks.x;
        chi.y = f * kks.y;
        S[4 * nh + e] = chi;
    }
    // frame dragging B (written over F)
    if (p.b_space && !p.b_seed) {
        C *BS = reinterpret_cast<C *>(p.bstate);
        C v[3];
#pragma unroll
        for (int l = 0; l < 3; l++) {
            v[l].x = kt[0] * Sm[0][l].x + kt[1] * Sm[1][l].x + kt[2] * Sm[2][l].x;
            v[l].y = kt[0] * Sm[0][l].y + kt[1] * Sm[1][l].y + kt[2] * Sm[2][l].y;
        }
        C kv;
        kv.x = kt[0] * v[0].x + kt[1] * v[1].x + kt[2] * v[2].x;
        kv.y = kt[0] * v[0].y + kt[1] * v[1].y + kt[2] * v[2].y;
        const T ik2 = T(1) / k2;
        const T w = p.dtau_prev * ik2;
#pragma unroll
        for (int j = 0; j < 3; j++) {
            // dtau W_j = dtau (-i) (v_j - kt_j kv / kt^2) / kt^2
            const T px = v[j].x - kt[j] * kv.x * ik2, py = v[j].y - kt[j] * kv.y * ik2;
            C b = inF[j];
            b.x = p.b_decay * b.x + w * py;
            b.y = p.b_decay * b.y - w * px;
            BS[j * nh + e] = b;
            b.x *= p.inv_n3;
            b.y *= p.inv_n3;
            S[(1 + j) * nh + e] = b;
        }
    } else {
        const C F[3] = {inF[0], inF[1], inF[2]};
        C kF;
        kF.x = kt[0] * F[0].x + kt[1] * F[1].x + kt[2] * F[2].x;
        kF.y = kt[0] * F[0].y + kt[1] * F[1].y + kt[2] * F[2].y;
        const T ik2 = T(1) / k2;
        const T f = T(4) * ik2;
#pragma unroll
        for (int i = 0; i < 3; i++) {
            C b;
            b.x = f * (F[i].x - kt[i] * kF.x * ik2);
            b.y = f * (F[i].y - kt[i] * kF.y * ik2);
            if (p.b_space) reinterpret_cast<C *>(p.bstate)[i * nh + e] = b;  // seeds the integration
            b.x *= p.inv_n3;
            b.y *= p.inv_n3;
            S[(1 + i) * nh + e] = b;
        }
    }
}

// P(k) binning of one half spectrum of delta: modes with 0 < kx < N/2 stand
// for themselves and their conjugate partner.
template <class T>
__global__ void __launch_bounds__(256) k_pk_bin(const typename Cplx<T>::type *d, int N, int64_t nh, int nbins,
                                                 double inv_n6, double *acc)
{
    extern __shared__ double sb[];  // 3 * nbins: pk sum, k sum, count
    for (int i = threadIdx.x; i < 3 * nbins; i += blockDim.x) sb[i] = 0.0;
    __syncthreads();
    const int h = N / 2 + 1;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nh; e += (int64_t)gridDim.x * blockDim.x) {
        const int kx = (int)(e % h);
        const int64_t r = e / h;
        const int ky = (int)(r % N), kz = (int)(r / N);
        const int ny = ky <= N / 2 ? ky : ky - N, nz = kz <= N / 2 ? kz : kz - N;
        const double kn = sqrt((double)(kx * kx + ny * ny + nz * nz));
        const int b = (int)rint(kn);
        if (b < 1 || b >= nbins) continue;
        const double w = (kx > 0 && 2 * kx < N) ? 2.0 : 1.0;
        const double re = (double)d[e].x, im = (double)d[e].y;
        atomicAdd(&sb[b], w * (re * re + im * im) * inv_n6);
        atomicAdd(&sb[nbins + b], w * 6.283185307179586476925286766559 * kn);
        atomicAdd(&sb[2 * nbins + b], w);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 3 * nbins; i += blockDim.x)
        if (sb[i] != 0.0) atomicAdd(&acc[i], sb[i]);
}

}  // namespace

template <class T>
void launch_solve(Ctx &c, const StepScalars &s)
{
    SolveParams<T> p{};
    p.spec = c.spec;
    p.tens = c.tens;
    p.ktab = reinterpret_cast<const T *>(c.ktab);
    p.dscal = c.dscal;
    p.imean_prev = c.iphi_prev;
    p.imean_new = c.iphi_new;
    p.N = c.N;
    p.nh = c.nh;
    p.newtonian = s.newtonian;
    p.bootstrap = s.bootstrap;
    p.full = !(s.newtonian || s.bootstrap);
    p.four_pi_g_a2 = s.four_pi_g / (s.a * s.a);
    p.c1 = s.c_phi_dt;
    p.c2 = s.c_phi_h2;
    p.cphi = (T)(s.c_phi_dt + s.c_phi_h2);
    p.inv_n3 = (T)(1.0 / (double)c.nc);
    p.hc_half = (T)s.hc_half;
    p.dtau = (T)s.dtau;
    p.bstate = c.bstate;
    p.b_space = s.b_space && c.bstate != nullptr;
    p.b_seed = s.b_seed;
    p.b_decay = (T)s.b_decay;
    p.dtau_prev = (T)s.dtau_prev;
    k_solve<T><<<(unsigned)((c.nh + 255) / 256), 256, 0, c.stream>>>(p);
    c.launches++;
}

template <class T>
void launch_pk_bin(Ctx &c, const void *spec_in, int nbins, double *d_acc)
{
    const double inv_n6 = 1.0 / ((double)c.nc * (double)c.nc);
    int blocks = (int)std::min<int64_t>((c.nh + 255) / 256, 4096);
    k_pk_bin<T><<<blocks, 256, sizeof(double) * 3 * nbins, c.stream>>>(
        reinterpret_cast<const typename Cplx<T>::type *>(spec_in), c.N, c.nh, nbins, inv_n6, d_acc);
}

template void launch_solve<double>(Ctx &, const StepScalars &);
template void launch_solve<float>(Ctx &, const StepScalars &);
template void launch_pk_bin<double>(Ctx &, const void *, int, double *);
template void launch_pk_bin<float>(Ctx &, const void *, int, double *);

}  // namespace pm
