// Pencil-staged 3D FFT for the metric solves (Sec. 2.3 transforms a 3D
// field as a sequence of 1D FFTs along x, y and z; here every sequence of
// 1D transforms runs from shared memory on one GPU).
//
// Layout: real fields [z][y][x]; half spectra [kz][ky][kx] with
// kx in [0, N/2].  Forward: x pass (two real rows packed as one complex
// line, r2c split), y pass, z pass.  Inverse: z, y, then x (c2r).  No
// normalisation: the Fourier solve applies 1/N^3.
//
// Each pass loads L lines of N points into shared memory as [j][line]
// (line index fastest, so the strided y and z passes read L contiguous
// complex values per row: 128-byte segments), runs a Stockham autosort
// FFT (Govindaraju et al., SC'08 formulation) with radices 8, 4, 2 and 3
// in registers, and writes the lines back.
#include "pm_fft_core.cuh"
#include "pm_internal.cuh"

namespace pm {

FftPlan make_plan(int n)
{
    FftPlan p{};
    p.n = n;
    int m = n;
    while (m % 3 == 0) { p.radix[p.nst++] = 3; m /= 3; }
    while (m % 8 == 0) { p.radix[p.nst++] = 8; m /= 8; }
    if (m % 4 == 0) { p.radix[p.nst++] = 4; m /= 4; }
    if (m % 2 == 0) { p.radix[p.nst++] = 2; m /= 2; }
    return p;
}

namespace {

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
// z * (s i), s = +-1
template <class C> __device__ __forceinline__ C mul_si(C z, int s)
{
    return s > 0 ? mk<C>(-z.y, z.x) : mk<C>(z.y, -z.x);
}
template <class C> __device__ __forceinline__ C scale(C z, decltype(C::x) f) { return mk<C>(z.x * f, z.y * f); }

// In-register DFTs of size R with exponent sign s (-1 forward, +1 inverse).
template <int R, class C> struct Dft;

template <class C> struct Dft<2, C> {
    static __device__ __forceinline__ void run(C *v, int)
    {
        C a = v[0], b = v[1];
        v[0] = add(a, b);
        v[1] = sub(a, b);
    }
};

template <class C> struct Dft<4, C> {
    static __device__ __forceinline__ void run(C *v, int s)
    {
        C t0 = add(v[0], v[2]), t1 = sub(v[0], v[2]);
        C t2 = add(v[1], v[3]), t3 = mul_si(sub(v[1], v[3]), s);
        v[0] = add(t0, t2);
        v[2] = sub(t0, t2);
        v[1] = add(t1, t3);
        v[3] = sub(t1, t3);
    }
};

template <class C> struct Dft<8, C> {
    static __device__ __forceinline__ void run(C *v, int s)
    {
        using T = decltype(C::x);
        const T h = (T)0.70710678118654752440084436210484903928;
        C e[4] = {v[0], v[2], v[4], v[6]};
        C o[4] = {v[1], v[3], v[5], v[7]};
        Dft<4, C>::run(e, s);
        Dft<4, C>::run(o, s);
        // o_k * W8^k,  W8 = exp(s i pi / 4)
        C o1 = scale(add(o[1], mul_si(o[1], s)), h);
        C o2 = mul_si(o[2], s);
        C o3 = scale(sub(mul_si(o[3], s), o[3]), h);
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

template <class C> struct Dft<3, C> {
    static __device__ __forceinline__ void run(C *v, int s)
    {
        using T = decltype(C::x);
        const T r3 = (T)0.86602540378443864676372317075293618347;
        C t = add(v[1], v[2]);
        C d = mul_si(scale(sub(v[1], v[2]), r3), s);
        C m = sub(v[0], scale(t, (T)0.5));
        v[0] = add(v[0], t);
        v[1] = add(m, d);
        v[2] = sub(m, d);
    }
};

// One Stockham stage over L lines held in shared memory as buf[j * L + line].
template <int R, int MAXB, class C>
__device__ __forceinline__ void stage(C *buf, int n, int L, int Ns, const C *tw, int s)
{
    const int nbl = n / R;
    const int total = nbl * L;
    C v[MAXB][R];
#pragma unroll
    for (int q = 0; q < MAXB; q++) {
        int g = threadIdx.x + q * blockDim.x;
        if (g < total) {
            int l = g % L, b = g / L;
#pragma unroll
            for (int r = 0; r < R; r++) v[q][r] = buf[(b + r * nbl) * L + l];
        }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < MAXB; q++) {
        int g = threadIdx.x + q * blockDim.x;
        if (g < total) {
            int l = g % L, b = g / L;
            int k = b % Ns;
            int step = k * (n / (Ns * R));
#pragma unroll
            for (int r = 1; r < R; r++) {
                C w = tw[r * step];
                if (s > 0) w.y = -w.y;
                v[q][r] = mul(v[q][r], w);
            }
            Dft<R, C>::run(v[q], s);
            int j0 = (b - k) * R + k;
#pragma unroll
            for (int r = 0; r < R; r++) buf[(j0 + r * Ns) * L + l] = v[q][r];
        }
    }
    __syncthreads();
}

// Full N-point transform of L lines.  Requires L * n <= 16 * blockDim.x.
template <class C>
__device__ void fft_lines(C *buf, int L, const FftPlan &plan, const C *tw, int s)
{
    int Ns = 1;
    for (int st = 0; st < plan.nst; st++) {
        int R = plan.radix[st];
        if (R == 8) stage<8, 2>(buf, plan.n, L, Ns, tw, s);
        else if (R == 4) stage<4, 4>(buf, plan.n, L, Ns, tw, s);
        else if (R == 2) stage<2, 8>(buf, plan.n, L, Ns, tw, s);
        else stage<3, 6>(buf, plan.n, L, Ns, tw, s);
        Ns *= R;
    }
}

template <class T> constexpr int fft_block() { return sizeof(T) == 8 ? 256 : 512; }

// Strided column pass (y or z): line g = (batch b, column c), point j at
// data[b * stride_b + j * stride_j + c].
template <class T>
__global__ void __launch_bounds__(fft_block<T>())
k_fft_cols(const __grid_constant__ Ptrs ptrs, const typename Cplx<T>::type *__restrict__ twg, FftPlan plan, int L, int64_t stride_j,
           int64_t ncols, int64_t stride_b, int64_t nlines, int s)
{
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem[];
    const int n = plan.n;
    C *tw = reinterpret_cast<C *>(smem);
    C *buf = tw + n;
    int64_t *lbase = reinterpret_cast<int64_t *>(buf + (size_t)L * n);
    C *data = reinterpret_cast<C *>(ptrs.p[blockIdx.y]);
    for (int i = threadIdx.x; i < n; i += blockDim.x) tw[i] = twg[i];
    const int64_t g0 = (int64_t)blockIdx.x * L;
    for (int l = threadIdx.x; l < L; l += blockDim.x) {
        int64_t g = g0 + l;
        lbase[l] = g < nlines ? (g / ncols) * stride_b + (g % ncols) : -1;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < L * n; e += blockDim.x) {
        int l = e % L, j = e / L;
        int64_t base = lbase[l];
        C v = mk<C>(0, 0);
        if (base >= 0) v = data[base + j * stride_j];
        buf[e] = v;
    }
    __syncthreads();
    fft_lines(buf, L, plan, tw, s);
    for (int e = threadIdx.x; e < L * n; e += blockDim.x) {
        int l = e % L, j = e / L;
        int64_t base = lbase[l];
        if (base >= 0) data[base + j * stride_j] = buf[e];
    }
}

// x pass, forward: real rows 2l, 2l+1 packed as z = a + i b, one complex
// FFT, then A_k = (Z_k + conj Z_{N-k})/2, B_k = -i (Z_k - conj Z_{N-k})/2.
template <class T>
__global__ void __launch_bounds__(fft_block<T>())
k_fft_r2c(const __grid_constant__ Ptrs in, const __grid_constant__ Ptrs out, const typename Cplx<T>::type *__restrict__ twg, FftPlan plan, int L, int64_t npairs)
{
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem[];
    const int n = plan.n, h = n / 2 + 1;
    C *tw = reinterpret_cast<C *>(smem);
    C *buf = tw + n;
    T *bufr = reinterpret_cast<T *>(buf);
    const T *src = reinterpret_cast<const T *>(in.p[blockIdx.y]);
    C *dst = reinterpret_cast<C *>(out.p[blockIdx.y]);
    for (int i = threadIdx.x; i < n; i += blockDim.x) tw[i] = twg[i];
    const int64_t p0 = (int64_t)blockIdx.x * L;
    for (int e = threadIdx.x; e < 2 * L * n; e += blockDim.x) {
        int l2 = e / n, x = e % n;
        int l = l2 >> 1, comp = l2 & 1;
        int64_t pair = p0 + l;
        T v = 0;
        if (pair < npairs) v = src[(2 * pair + comp) * n + x];
        bufr[2 * (x * L + l) + comp] = v;
    }
    __syncthreads();
    fft_lines(buf, L, plan, tw, -1);
    for (int e = threadIdx.x; e < L * h; e += blockDim.x) {
        int l = e / h, k = e % h;
        int64_t pair = p0 + l;
        if (pair >= npairs) continue;
        C zk = buf[k * L + l], zn = buf[((n - k) % n) * L + l];
        const T half = (T)0.5;
        C A = mk<C>(half * (zk.x + zn.x), half * (zk.y - zn.y));
        C B = mk<C>(half * (zk.y + zn.y), -half * (zk.x - zn.x));
        dst[(2 * pair) * h + k] = A;
        dst[(2 * pair + 1) * h + k] = B;
    }
}

// x pass, inverse: half spectra A (row 2l), B (row 2l+1) -> Z = A + i B over
// the full line by Hermitian extension (imaginary parts at k = 0 and N/2
// dropped), inverse FFT, a = Re z, b = Im z.
template <class T>
__global__ void __launch_bounds__(fft_block<T>())
k_fft_c2r(const __grid_constant__ Ptrs in, const __grid_constant__ Ptrs out, const typename Cplx<T>::type *__restrict__ twg, FftPlan plan, int L, int64_t npairs)
{
    using C = typename Cplx<T>::type;
    extern __shared__ __align__(16) unsigned char smem[];
    const int n = plan.n, h = n / 2 + 1;
    C *tw = reinterpret_cast<C *>(smem);
    C *buf = tw + n;
    const T *bufr = reinterpret_cast<const T *>(buf);
    const C *src = reinterpret_cast<const C *>(in.p[blockIdx.y]);
    T *dst = reinterpret_cast<T *>(out.p[blockIdx.y]);
    for (int i = threadIdx.x; i < n; i += blockDim.x) tw[i] = twg[i];
    const int64_t p0 = (int64_t)blockIdx.x * L;
    for (int e = threadIdx.x; e < L * h; e += blockDim.x) {
        int l = e / h, k = e % h;
        int64_t pair = p0 + l;
        C A = mk<C>(0, 0), B = mk<C>(0, 0);
        if (pair < npairs) {
            A = src[(2 * pair) * h + k];
            B = src[(2 * pair + 1) * h + k];
        }
        if (k == 0 || 2 * k == n) {
            A.y = 0;
            B.y = 0;
        }
        buf[k * L + l] = mk<C>(A.x - B.y, A.y + B.x);
        if (k > 0 && 2 * k < n) buf[(n - k) * L + l] = mk<C>(A.x + B.y, B.x - A.y);
    }
    __syncthreads();
    fft_lines(buf, L, plan, tw, +1);
    for (int e = threadIdx.x; e < 2 * L * n; e += blockDim.x) {
        int l2 = e / n, x = e % n;
        int l = l2 >> 1, comp = l2 & 1;
        int64_t pair = p0 + l;
        if (pair < npairs) dst[(2 * pair + comp) * n + x] = bufr[2 * (x * L + l) + comp];
    }
}

template <class T> int lines_per_block(int n) { return (16 * fft_block<T>()) / n; }

template <class T> size_t cols_smem(int n, int L)
{
    return sizeof(typename Cplx<T>::type) * ((size_t)L * n + n) + sizeof(int64_t) * L;
}

template <class T> void set_smem_attrs()
{
    static std::atomic<uint64_t> done{0};
    if (!first_on_device(done)) return;
    const int maxs = 160 * 1024;
    cudaFuncSetAttribute(k_fft_cols<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxs);
    cudaFuncSetAttribute(k_fft_r2c<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxs);
    cudaFuncSetAttribute(k_fft_c2r<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxs);
}

template <class T>
void col_pass(Ctx &c, int nf, const Ptrs &p, int64_t stride_j, int64_t ncols, int64_t stride_b, int64_t nlines,
              int s)
{
    int L = lines_per_block<T>(c.N);
    dim3 grid((unsigned)((nlines + L - 1) / L), nf);
    k_fft_cols<T><<<grid, fft_block<T>(), cols_smem<T>(c.N, L), c.stream>>>(
        p, reinterpret_cast<const typename Cplx<T>::type *>(c.tw), c.plan, L, stride_j, ncols, stride_b, nlines,
        s);
    c.launches++;
}


// ---------------------------------------------------------------------------
// Compile-time-N passes (register-resident radix stages, see pm_fft_core.cuh).
// ---------------------------------------------------------------------------
// Shapes of the FP32 column passes for power-of-two sizes >= 64 (ZP: the z
// pass, whose points are a whole plane apart, else the y pass): points per
// thread, lines per block (the line width sets the contiguous row segment)
// and the threads per SM the register budget must allow.  Shape 0 is the one
// timed best at 512^3; fft_tune_shapes picks among the three per context.
struct ColShape {
    int p, l, tpsm;
};
constexpr int NCOLSHAPES = 3;
constexpr ColShape kColY[NCOLSHAPES] = {{32, 8, 512}, {16, 8, 1024}, {8, 8, 1536}};
constexpr ColShape kColZ[NCOLSHAPES] = {{16, 16, 1024}, {8, 16, 1536}, {16, 8, 1024}};

template <class T, int N, bool ZP = false, int V = 0> struct Lines {
    static constexpr bool tuned = sizeof(T) == 4 && N % 3 != 0 && N >= 64;
    static constexpr ColShape sh = ZP ? kColZ[V] : kColY[V];
    static constexpr int CP = tuned && sh.p != 8 ? sh.p : 0;  // 0: default points per thread
    static constexpr int TL = fftc::Geo<N>::TL;
    static constexpr int TLC = fftc::Geo<N, CP>::TL;
    // lines per block of the column passes: 64-byte row segments by default, >= 128 threads
    static constexpr int col0 = tuned ? sh.l : (sizeof(T) == 4 ? 8 : 4);
    static constexpr int col1 = col0 * TLC < 128 ? 128 / TLC : col0;
    static constexpr int col = col1 * TLC > 1024 ? 1024 / TLC : col1;
    static constexpr int row = TL >= 256 ? 1 : 256 / TL;               // row pairs per block, x passes
    // resident blocks per SM the register allocation must allow
    static constexpr int tpsm = tuned ? sh.tpsm : (fftc::Geo<N>::P == 8 ? (sizeof(T) == 4 ? 1536 : 1024) : 0);
    static constexpr int col_min_blocks = tpsm / (TLC * col) > 0 ? tpsm / (TLC * col) : 1;
};

template <class T, int N, bool ZP, int V> size_t col_fast_smem()
{
    using G = fftc::Geo<N>;
    return sizeof(typename Cplx<T>::type) * (G::TWN + (size_t)N * Lines<T, N, ZP, V>::col);  // TWN does not depend on P
}
template <class T, int N> size_t row_fast_smem()
{
    using G = fftc::Geo<N>;
    return sizeof(typename Cplx<T>::type) * (G::TWN + (size_t)Lines<T, N>::row * fftc::RowIdx<N>::pitch);
}

template <class T, int N, int DIR, bool ZP, int V>
__global__ void __launch_bounds__(Lines<T, N, ZP, V>::TLC * Lines<T, N, ZP, V>::col, Lines<T, N, ZP, V>::col_min_blocks)
k_col_fast(const __grid_constant__ Ptrs ptrs, const typename Cplx<T>::type *__restrict__ twg)
{
    using C = typename Cplx<T>::type;
    constexpr int CP = Lines<T, N, ZP, V>::CP;
    using G = fftc::Geo<N, CP>;
    constexpr int L = Lines<T, N, ZP, V>::col;
    extern __shared__ __align__(16) unsigned char smem[];
    C *tw = reinterpret_cast<C *>(smem);
    C *buf = tw + G::TWN;
    for (int i = threadIdx.x; i < G::TWN; i += blockDim.x) tw[i] = twg[i];
    // strides and line counts are compile-time constants of N and the pass, so every point's address is the
    // thread's base plus an immediate (no per-point address registers, no spills)
    constexpr int H = N / 2 + 1;
    constexpr int SJ = ZP ? N * H : H;          // point stride
    constexpr int NLINES = N * H;               // lines (kz, kx) or (ky, kx)
    const int l = threadIdx.x % L, t = threadIdx.x / L;
    const int g = (int)blockIdx.x * L + l;
    const bool ok = g < NLINES;
    // y: line (kz, kx) starts at kz N H + kx; z: line (ky, kx) at ky H + kx = g
    const int base = ok ? (ZP ? g : (g / H) * (N * H) + g % H) : 0;
    C *data = reinterpret_cast<C *>(ptrs.p[blockIdx.y]) + base + (int64_t)t * SJ;
    C v[G::P];
#pragma unroll
    for (int i = 0; i < G::P; i++)
        v[i] = ok ? data[(int64_t)fftc::in_pos<N, CP>(0, i) * SJ] : fftc::mk<C>(0, 0);
    __syncthreads();
    fftc::fft<C, N, DIR, CP>(v, t, buf, tw, fftc::ColIdx{L, l});
    if (ok) {
#pragma unroll
        for (int i = 0; i < G::P; i++) data[(int64_t)fftc::out_pos<N, CP>(0, i) * SJ] = v[i];
    }
}

template <class T, int N>
__global__ void __launch_bounds__(fftc::Geo<N>::TL * Lines<T, N>::row)
k_r2c_fast(const __grid_constant__ Ptrs in, const __grid_constant__ Ptrs out, const typename Cplx<T>::type *__restrict__ twg, int64_t npairs)
{
    using C = typename Cplx<T>::type;
    using G = fftc::Geo<N>;
    constexpr int L = Lines<T, N>::row, H = N / 2 + 1;
    extern __shared__ __align__(16) unsigned char smem[];
    C *tw = reinterpret_cast<C *>(smem);
    C *buf = tw + G::TWN;
    for (int i = threadIdx.x; i < G::TWN; i += blockDim.x) tw[i] = twg[i];
    const int t = threadIdx.x % G::TL, l = threadIdx.x / G::TL;
    const int64_t pair = (int64_t)blockIdx.x * L + l;
    const bool ok = pair < npairs;
    const T *src = reinterpret_cast<const T *>(in.p[blockIdx.y]);
    C *dst = reinterpret_cast<C *>(out.p[blockIdx.y]);
    const T *ra = src + 2 * pair * N, *rb = ra + N;
    C v[G::P];
#pragma unroll
    for (int i = 0; i < G::P; i++) {
        const int j = fftc::in_pos<N>(t, i);
        v[i] = ok ? fftc::mk<C>(ra[j], rb[j]) : fftc::mk<C>(0, 0);
    }
    __syncthreads();
    const fftc::RowIdx<N> ix{l * fftc::RowIdx<N>::pitch};
    fftc::fft<C, N, -1>(v, t, buf, tw, ix);
#pragma unroll
    for (int i = 0; i < G::P; i++) buf[ix(fftc::out_pos<N>(t, i))] = v[i];
    __syncthreads();
    if (!ok) return;
    C *oa = dst + 2 * pair * H, *ob = oa + H;
    const T half = (T)0.5;
    for (int k = t; k < H; k += G::TL) {
        const C zk = buf[ix(k)], zn = buf[ix((N - k) % N)];
        oa[k] = fftc::mk<C>(half * (zk.x + zn.x), half * (zk.y - zn.y));
        ob[k] = fftc::mk<C>(half * (zk.y + zn.y), -half * (zk.x - zn.x));
    }
}

template <class T, int N>
__global__ void __launch_bounds__(fftc::Geo<N>::TL * Lines<T, N>::row)
k_c2r_fast(const __grid_constant__ Ptrs in, const __grid_constant__ Ptrs out, const typename Cplx<T>::type *__restrict__ twg, int64_t npairs)
{
    using C = typename Cplx<T>::type;
    using G = fftc::Geo<N>;
    constexpr int L = Lines<T, N>::row, H = N / 2 + 1;
    extern __shared__ __align__(16) unsigned char smem[];
    C *tw = reinterpret_cast<C *>(smem);
    C *buf = tw + G::TWN;
    for (int i = threadIdx.x; i < G::TWN; i += blockDim.x) tw[i] = twg[i];
    const int t = threadIdx.x % G::TL, l = threadIdx.x / G::TL;
    const int64_t pair = (int64_t)blockIdx.x * L + l;
    const bool ok = pair < npairs;
    const C *src = reinterpret_cast<const C *>(in.p[blockIdx.y]);
    T *dst = reinterpret_cast<T *>(out.p[blockIdx.y]);
    const fftc::RowIdx<N> ix{l * fftc::RowIdx<N>::pitch};
    const C *ia = src + 2 * pair * H, *ib = ia + H;
    constexpr int NK = (H + G::TL - 1) / G::TL;
    C As[NK], Bs[NK];
#pragma unroll
    for (int q = 0; q < NK; q++) {
        const int k = t + q * G::TL;
        As[q] = (ok && k < H) ? ia[k] : fftc::mk<C>(0, 0);
        Bs[q] = (ok && k < H) ? ib[k] : fftc::mk<C>(0, 0);
    }
#pragma unroll
    for (int q = 0; q < NK; q++) {
        const int k = t + q * G::TL;
        if (k >= H) break;
        C A = As[q], B = Bs[q];
        if (k == 0 || 2 * k == N) {
            A.y = 0;
            B.y = 0;
        }
        buf[ix(k)] = fftc::mk<C>(A.x - B.y, A.y + B.x);
        if (k > 0 && 2 * k < N) buf[ix(N - k)] = fftc::mk<C>(A.x + B.y, B.x - A.y);
    }
    __syncthreads();
    C v[G::P];
#pragma unroll
    for (int i = 0; i < G::P; i++) v[i] = buf[ix(fftc::in_pos<N>(t, i))];
    __syncthreads();
    fftc::fft<C, N, +1>(v, t, buf, tw, ix);
    if (!ok) return;
    T *wa = dst + 2 * pair * N, *wb = wa + N;
#pragma unroll
    for (int i = 0; i < G::P; i++) {
        const int j = fftc::out_pos<N>(t, i);
        wa[j] = v[i].x;
        wb[j] = v[i].y;
    }
}

template <class T, int N> struct FastPasses {
    static void attrs()
    {
        static std::atomic<uint64_t> done{0};
        if (!first_on_device(done)) return;
        auto set = [](auto k, size_t b) { cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b); };
        set_col<0>();
        if constexpr (Lines<T, N>::tuned) {
            set_col<1>();
            set_col<2>();
        }
        set(k_r2c_fast<T, N>, row_fast_smem<T, N>());
        set(k_c2r_fast<T, N>, row_fast_smem<T, N>());
    }
    template <int V> static void set_col()
    {
        auto set = [](auto k, size_t b) { cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b); };
        set(k_col_fast<T, N, -1, false, V>, col_fast_smem<T, N, false, V>());
        set(k_col_fast<T, N, 1, false, V>, col_fast_smem<T, N, false, V>());
        set(k_col_fast<T, N, -1, true, V>, col_fast_smem<T, N, true, V>());
        set(k_col_fast<T, N, 1, true, V>, col_fast_smem<T, N, true, V>());
    }
    template <bool ZP, int V>
    static void cols_t(Ctx &c, int nf, const Ptrs &p, int dir)
    {
        constexpr int64_t nl = (int64_t)N * (N / 2 + 1);   // lines of a y or z pass
        constexpr int L = Lines<T, N, ZP, V>::col;
        constexpr int threads = Lines<T, N, ZP, V>::TLC * L;
        dim3 grid((unsigned)((nl + L - 1) / L), nf);
        const auto *tw = reinterpret_cast<const typename Cplx<T>::type *>(c.tw2);
        const size_t sm = col_fast_smem<T, N, ZP, V>();
        if (dir < 0)
            k_col_fast<T, N, -1, ZP, V><<<grid, threads, sm, c.stream>>>(p, tw);
        else
            k_col_fast<T, N, 1, ZP, V><<<grid, threads, sm, c.stream>>>(p, tw);
        c.launches++;
    }
    template <bool ZP>
    static void cols_v(Ctx &c, int nf, const Ptrs &p, int dir)
    {
        const int v = Lines<T, N>::tuned ? c.col_shape[ZP ? 1 : 0] : 0;
        if constexpr (Lines<T, N>::tuned) {
            if (v == 1) return cols_t<ZP, 1>(c, nf, p, dir);
            if (v == 2) return cols_t<ZP, 2>(c, nf, p, dir);
        }
        cols_t<ZP, 0>(c, nf, p, dir);
    }
    // y pass (ZP false): lines (kz, kx), points a row apart; z pass: lines (ky, kx), points a plane apart
    template <bool ZP> static void cols(Ctx &c, int nf, const Ptrs &p, int dir) { cols_v<ZP>(c, nf, p, dir); }
    static void rows(Ctx &c, int nf, const Ptrs &pi, const Ptrs &po, int dir)
    {
        constexpr int L = Lines<T, N>::row;
        const int64_t npairs = (int64_t)N * N / 2;
        dim3 grid((unsigned)((npairs + L - 1) / L), nf);
        const auto *tw = reinterpret_cast<const typename Cplx<T>::type *>(c.tw2);
        if (dir < 0)
            k_r2c_fast<T, N><<<grid, fftc::Geo<N>::TL * L, row_fast_smem<T, N>(), c.stream>>>(pi, po, tw, npairs);
        else
            k_c2r_fast<T, N><<<grid, fftc::Geo<N>::TL * L, row_fast_smem<T, N>(), c.stream>>>(pi, po, tw, npairs);
        c.launches++;
    }
};

// calls f.template operator()<N>() for the specialised sizes; false otherwise
template <class F> bool with_fast_n(int n, F &&f)
{
    switch (n) {
    case 16: f.template operator()<16>(); return true;
    case 32: f.template operator()<32>(); return true;
    case 64: f.template operator()<64>(); return true;
    case 128: f.template operator()<128>(); return true;
    case 192: f.template operator()<192>(); return true;
    case 256: f.template operator()<256>(); return true;
    case 512: f.template operator()<512>(); return true;
    default: return false;
    }
}

}  // namespace

template <class T>
void fft_forward(Ctx &c, int nf, const void *const *real_in, void *const *spec_out)
{
    set_smem_attrs<T>();
    const int N = c.N;
    const int64_t h = N / 2 + 1;
    Ptrs pi{}, po{};
    for (int i = 0; i < nf; i++) {
        pi.p[i] = const_cast<void *>(real_in[i]);
        po.p[i] = spec_out[i];
    }
    auto fast = [&]<int NN>() {
        using F = FastPasses<T, NN>;
        F::attrs();
        F::rows(c, nf, pi, po, -1);
        c.mark(EV_FWD_X);
        F::template cols<false>(c, nf, po, -1);
        c.mark(EV_FWD_Y);
        F::template cols<true>(c, nf, po, -1);
        c.mark(EV_FWD_Z);
    };
    if (with_fast_n(N, fast)) return;
    // x: real rows -> half-spectrum rows.  L complex lines = L row pairs per block.
    int L = lines_per_block<T>(N);
    int64_t npairs = (int64_t)N * N / 2;
    dim3 grid((unsigned)((npairs + L - 1) / L), nf);
    k_fft_r2c<T><<<grid, fft_block<T>(), cols_smem<T>(N, L), c.stream>>>(
        pi, po, reinterpret_cast<const typename Cplx<T>::type *>(c.tw), c.plan, L, npairs);
    c.launches++;
    c.mark(EV_FWD_X);
    // y: lines (z, kx), points stride h
    col_pass<T>(c, nf, po, h, h, (int64_t)N * h, (int64_t)N * h, -1);
    c.mark(EV_FWD_Y);
    // z: lines (ky, kx), points stride N h
    col_pass<T>(c, nf, po, (int64_t)N * h, (int64_t)N * h, 0, (int64_t)N * h, -1);
    c.mark(EV_FWD_Z);
}

template <class T>
void fft_inverse(Ctx &c, int nf, void *const *spec_in, void *const *real_out)
{
    set_smem_attrs<T>();
    const int N = c.N;
    const int64_t h = N / 2 + 1;
    Ptrs pi{}, po{};
    for (int i = 0; i < nf; i++) {
        pi.p[i] = spec_in[i];
        po.p[i] = real_out[i];
    }
    auto fast = [&]<int NN>() {
        using F = FastPasses<T, NN>;
        F::attrs();
        F::template cols<true>(c, nf, pi, +1);
        c.mark(EV_INV_Z);
        F::template cols<false>(c, nf, pi, +1);
        c.mark(EV_INV_Y);
        F::rows(c, nf, pi, po, +1);
        c.mark(EV_INV_X);
    };
    if (with_fast_n(N, fast)) return;
    col_pass<T>(c, nf, pi, (int64_t)N * h, (int64_t)N * h, 0, (int64_t)N * h, +1);
    c.mark(EV_INV_Z);
    col_pass<T>(c, nf, pi, h, h, (int64_t)N * h, (int64_t)N * h, +1);
    c.mark(EV_INV_Y);
    int L = lines_per_block<T>(N);
    int64_t npairs = (int64_t)N * N / 2;
    dim3 grid((unsigned)((npairs + L - 1) / L), nf);
    k_fft_c2r<T><<<grid, fft_block<T>(), cols_smem<T>(N, L), c.stream>>>(
        pi, po, reinterpret_cast<const typename Cplx<T>::type *>(c.tw), c.plan, L, npairs);
    c.launches++;
    c.mark(EV_INV_X);
}

template <class T>
bool fft_shapes_tunable(const Ctx &c)
{
    bool t = false;
    with_fast_n(c.N, [&]<int NN>() { t = Lines<T, NN>::tuned; });
    return t;
}

// Time the column-pass shapes of one pass on the context's spectra (9 forward and 5 inverse line
// transforms, as in a step) and keep the fastest.  pass 0: y, 1: z.
template <class T>
int tune_col_pass(Ctx &c, int pass)
{
    const int N = c.N;
    Ptrs p{};
    for (int i = 0; i < 9; i++) p.p[i] = reinterpret_cast<typename Cplx<T>::type *>(c.spec) + (size_t)i * c.nh;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    int best_v = 0;
    for (int v = 0; v < NCOLSHAPES; v++) {
        c.col_shape[pass] = v;
        auto run = [&]() {
            with_fast_n(N, [&]<int NN>() {
                using F = FastPasses<T, NN>;
                if (pass == 0) {
                    F::template cols<false>(c, 9, p, -1);
                    F::template cols<false>(c, 5, p, +1);
                } else {
                    F::template cols<true>(c, 9, p, -1);
                    F::template cols<true>(c, 5, p, +1);
                }
            });
        };
        run();   // warm-up (and the first launch of a new shape)
        cudaEventRecord(e0, c.stream);
        for (int r = 0; r < 3; r++) run();
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
    c.col_shape[pass] = best_v;
    return best_v;
}

template <class T>
bool fft_tune_shapes(Ctx &c, int force_y, int force_z)
{
    if (!fft_shapes_tunable<T>(c)) {
        c.col_shape[0] = c.col_shape[1] = 0;
        return false;
    }
    set_smem_attrs<T>();
    with_fast_n(c.N, [&]<int NN>() { FastPasses<T, NN>::attrs(); });
    if (force_y < 0 || force_z < 0) {
        // the spectra hold nothing between steps; clear them so the timed transforms see finite data
        cudaMemsetAsync(c.spec, 0, 9 * 2 * sizeof(T) * (size_t)c.nh, c.stream);
    }
    if (force_y >= 0) c.col_shape[0] = force_y;
    else tune_col_pass<T>(c, 0);
    if (force_z >= 0) c.col_shape[1] = force_z;
    else tune_col_pass<T>(c, 1);
    return true;
}

template bool fft_tune_shapes<float>(Ctx &, int, int);
template bool fft_tune_shapes<double>(Ctx &, int, int);

bool fast_fft_supported(int n)
{
    return with_fast_n(n, []<int NN>() {});
}

void fast_twiddles(int n, std::vector<double> &re_im)
{
    re_im.clear();
    const long double pi = 3.141592653589793238462643383279502884L;
    for (int s = 1; s < fftc::nstages(n); s++) {
        const int Ns = fftc::span_before(n, s), R = fftc::radix_at(n, s);
        for (int k = 0; k < Ns; k++)
            for (int r = 1; r < R; r++) {
                const long double ang = -2.0L * pi * (long double)(r * k) / (long double)(Ns * R);
                re_im.push_back((double)cosl(ang));
                re_im.push_back((double)sinl(ang));
            }
    }
}

template void fft_forward<double>(Ctx &, int, const void *const *, void *const *);
template void fft_forward<float>(Ctx &, int, const void *const *, void *const *);
template void fft_inverse<double>(Ctx &, int, void *const *, void *const *);
template void fft_inverse<float>(Ctx &, int, void *const *, void *const *);

}  // namespace pm
