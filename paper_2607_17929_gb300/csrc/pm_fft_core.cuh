// Register-resident Stockham FFT core with compile-time length N.
//
// A line of N points is handled by TL = N / P threads, each holding P points
// (P = 8, or 24 when N has a factor 3) in registers through every radix
// stage.  Stage s of radix R (Ns = product of the earlier radices) takes the
// points j = b + r N/R of butterfly b, twiddles them by W_{Ns R}^{r (b mod Ns)},
// applies an R-point DFT and produces j' = (b - b mod Ns) R + b mod Ns + r Ns
// (the Stockham autosort order, Govindaraju et al., SC'08).  Consecutive
// stages exchange points through shared memory; the first stage reads and the
// last stage writes the natural order directly, so callers load and store
// global memory with coalesced accesses and no staging pass.
#pragma once

#include "pm_internal.cuh"

namespace pm {
namespace fftc {

template <class C> __device__ __forceinline__ C mk(decltype(C::x) x, decltype(C::x) y)
{
    C r;
    r.x = x;
    r.y = y;
    return r;
}
template <class C> __device__ __forceinline__ C add(C a, C b) { return mk<C>(a.x + b.x, a.y + b.y); }
template <class C> __device__ __forceinline__ C sub(C a, C b) { return mk<C>(a.x - b.x, a.y - b.y); }
template <class C> __device__ __forceinline__ C mul(C a, C b)
{
    return mk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <class C> __device__ __forceinline__ C scale(C z, decltype(C::x) f) { return mk<C>(z.x * f, z.y * f); }
// z * (s i)
template <int S, class C> __device__ __forceinline__ C mul_si(C z)
{
    return S > 0 ? mk<C>(-z.y, z.x) : mk<C>(z.y, -z.x);
}

template <int R, int S, class C> struct Dft;
template <int S, class C> struct Dft<2, S, C> {
    static __device__ __forceinline__ void run(C *v)
    {
        C a = v[0], b = v[1];
        v[0] = add(a, b);
        v[1] = sub(a, b);
    }
};
template <int S, class C> struct Dft<4, S, C> {
    static __device__ __forceinline__ void run(C *v)
    {
        C t0 = add(v[0], v[2]), t1 = sub(v[0], v[2]);
        C t2 = add(v[1], v[3]), t3 = mul_si<S>(sub(v[1], v[3]));
        v[0] = add(t0, t2);
        v[2] = sub(t0, t2);
        v[1] = add(t1, t3);
        v[3] = sub(t1, t3);
    }
};
template <int S, class C> struct Dft<8, S, C> {
    static __device__ __forceinline__ void run(C *v)
    {
        using T = decltype(C::x);
        const T h = (T)0.70710678118654752440084436210484903928;
        C e[4] = {v[0], v[2], v[4], v[6]};
        C o[4] = {v[1], v[3], v[5], v[7]};
        Dft<4, S, C>::run(e);
        Dft<4, S, C>::run(o);
        const C o1 = scale(add(o[1], mul_si<S>(o[1])), h);
        const C o2 = mul_si<S>(o[2]);
        const C o3 = scale(sub(mul_si<S>(o[3]), o[3]), h);
        v[0] = add(e[0], o[0]);
        v[4] = sub(e[0], o[0]);
        v[1] = add(e[1], o1);
        v[5] = sub(e[1], o1);
        v[2] = add(e[2], o2);
        v[6] = sub(e[2], o2);
        v[3] = add(e[3], o3);
        v[7] = sub(e[3], o3);
    }
};
template <int S, class C> struct Dft<3, S, C> {
    static __device__ __forceinline__ void run(C *v)
    {
        using T = decltype(C::x);
        const T r3 = (T)0.86602540378443864676372317075293618347;
        const C t = add(v[1], v[2]);
        const C d = mul_si<S>(scale(sub(v[1], v[2]), r3));
        const C m = sub(v[0], scale(t, (T)0.5));
        v[0] = add(v[0], t);
        v[1] = add(m, d);
        v[2] = sub(m, d);
    }
};

// ---- compile-time plan: radix 3 stages first, then 8s, then a 4 or 2 -----
__host__ __device__ constexpr int radix_at(int n, int s)
{
    int m = n, st = 0;
    while (m % 3 == 0) {
        if (st == s) return 3;
        m /= 3;
        st++;
    }
    while (m % 8 == 0) {
        if (st == s) return 8;
        m /= 8;
        st++;
    }
    if (m % 4 == 0) {
        if (st == s) return 4;
        m /= 4;
        st++;
    }
    if (m % 2 == 0) {
        if (st == s) return 2;
        m /= 2;
        st++;
    }
    return 0;
}
__host__ __device__ constexpr int nstages(int n)
{
    int s = 0;
    while (radix_at(n, s)) s++;
    return s;
}
__host__ __device__ constexpr int span_before(int n, int s)
{
    int p = 1;
    for (int i = 0; i < s; i++) p *= radix_at(n, i);
    return p;
}
// offset of stage s in the per-stage twiddle table ([k][r-1] per stage, s >= 1)
__host__ __device__ constexpr int tw_offset(int n, int s)
{
    int o = 0;
    for (int i = 1; i < s; i++) o += span_before(n, i) * (radix_at(n, i) - 1);
    return o;
}

// PP = points per thread (0: 8, or 24 when N has a factor 3); every radix must divide it
template <int N, int PP = 0> struct Geo {
    static constexpr int P = PP ? PP : ((N % 3 == 0) ? 24 : 8);
    static constexpr int TL = N / P;
    static constexpr int NS = nstages(N);
    static constexpr int R0 = radix_at(N, 0);
    static constexpr int RL = radix_at(N, NS - 1);
    static constexpr int TWN = tw_offset(N, NS);
    static_assert(N % P == 0, "N must be a multiple of the points per thread");
};

// point index held in register i: input order of the first stage, output order of the last
template <int N, int PP = 0> __device__ __forceinline__ int in_pos(int t, int i)
{
    constexpr int R = Geo<N, PP>::R0;
    return t + Geo<N, PP>::TL * (i / R) + (i % R) * (N / R);
}
template <int N, int PP = 0> __device__ __forceinline__ int out_pos(int t, int i)
{
    constexpr int R = Geo<N, PP>::RL;
    return t + Geo<N, PP>::TL * (i / R) + (i % R) * (N / R);
}

template <class C, int N, int PP, int S, int DIR>
__device__ __forceinline__ void bfly(C (&v)[Geo<N, PP>::P], int t, const C *__restrict__ tw)
{
    constexpr int R = radix_at(N, S), Ns = span_before(N, S), P = Geo<N, PP>::P, TL = Geo<N, PP>::TL;
#pragma unroll
    for (int q = 0; q < P / R; q++) {
        if constexpr (S > 0) {
            const int k = (t + TL * q) % Ns;
            const C *w = tw + tw_offset(N, S) + k * (R - 1);
#pragma unroll
            for (int r = 1; r < R; r++) {
                C x = w[r - 1];
                if (DIR > 0) x.y = -x.y;
                v[q * R + r] = mul(v[q * R + r], x);
            }
        }
        Dft<R, DIR, C>::run(&v[q * R]);
    }
}

// outputs of stage S -> shared memory -> inputs of stage S+1
template <class C, int N, int PP, int S, class Idx>
__device__ __forceinline__ void exchange(C (&v)[Geo<N, PP>::P], int t, C *sm, Idx sidx)
{
    constexpr int R = radix_at(N, S), Ns = span_before(N, S), R2 = radix_at(N, S + 1);
    constexpr int P = Geo<N, PP>::P, TL = Geo<N, PP>::TL;
#pragma unroll
    for (int q = 0; q < P / R; q++) {
        const int b = t + TL * q;
        const int k = b % Ns;
#pragma unroll
        for (int r = 0; r < R; r++) sm[sidx((b - k) * R + k + r * Ns)] = v[q * R + r];
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < P / R2; q++) {
        const int b = t + TL * q;
#pragma unroll
        for (int r = 0; r < R2; r++) v[q * R2 + r] = sm[sidx(b + r * (N / R2))];
    }
    __syncthreads();
}

template <class C, int N, int PP, int S, int DIR, class Idx>
__device__ __forceinline__ void run_from(C (&v)[Geo<N, PP>::P], int t, C *sm, const C *tw, Idx sidx)
{
    bfly<C, N, PP, S, DIR>(v, t, tw);
    if constexpr (S + 1 < Geo<N, PP>::NS) {
        exchange<C, N, PP, S>(v, t, sm, sidx);
        run_from<C, N, PP, S + 1, DIR>(v, t, sm, tw, sidx);
    }
}

// In-register FFT of one line: v holds in_pos order on entry, out_pos order on exit.
// Every thread of the block must call it (it synchronises the block).
template <class C, int N, int DIR, int PP = 0, class Idx>
__device__ __forceinline__ void fft(C (&v)[Geo<N, PP>::P], int t, C *sm, const C *tw, Idx sidx)
{
    run_from<C, N, PP, 0, DIR>(v, t, sm, tw, sidx);
}

// Shared-memory index maps.  Column kernels store [j][line] with the row
// index swizzled by j ^ ((j >> 3) & 1): with 16-word rows (8 FP32 or 4 FP64
// complex lines) consecutive rows and rows 8 apart fall in different bank
// halves, so both the unit-stride reads and the stride-R first-stage writes
// of a warp take the minimum two wavefronts.  Row kernels store [line][j]
// with one pad element every 16 (8-byte complex values: a 16-lane half-warp
// covers exactly the 32 banks both for unit-stride reads and for the
// radix-8 stage writes, which with a pad every 8 elements met 2-way
// conflicts in a third of the row passes' wavefronts).
struct ColIdx {
    int pitch, l;
    __device__ __forceinline__ int operator()(int j) const { return (j ^ ((j >> 3) & 1)) * pitch + l; }
};
template <int N> struct RowIdx {
    int base;
    __device__ __forceinline__ int operator()(int j) const { return base + j + (j >> 4); }
    static constexpr int pitch = N + N / 16;
};

}  // namespace fftc

}  // namespace pm
