// Learned sub-mesh force correction: a 3^3 periodic convolutional network
// (2 -> 16 -> 16 -> 16 -> 3 channels, ReLU between layers) that maps the
// density contrast and potential of a PM step to an additive correction of
// the mesh force, its training (MSE, Adam) and the extra kick it gives.
//
// Layout.  Activations and gradients are BF16, channels-last [cell][16]
// (cell = (z N + y) N + x); the network output and the targets are FP32
// [cell][8] (channels 0..2 used).  Weights are BF16 [27][c_out = 16][c_in = 16]
// with the offset index d = 9 (dz + 1) + 3 (dy + 1) + (dx + 1); the first
// layer's inputs and the last layer's outputs are zero-padded to 16, so every
// layer is one 16 x 16 contraction per offset.
//
// Convolution as an implicit GEMM on the tensor cores.  Meshes with n % 16 == 0
// take the tcgen05 kernel (k_conv_tc, below: M 128 x N 16 x K 16 MMAs from shared
// memory into tensor memory, persistent and double-buffered); the first layer
// (2 input channels), the weight gradient and other meshes use mma.sync
// m16n8k16 (BF16 in, FP32 accumulate).  In k_conv one CTA computes an 8^3 tile of cells: the
// 10^3 halo of input cells (32 B each) and the weights sit in shared memory,
// each of the 8 warps owns one z-slice of the tile (64 cells = 4 m16 blocks
// x 2 n8 blocks of output channels), and the K dimension runs over the 27
// offsets x 16 input channels, one k16 step per offset.  Rows of 32 B are
// stored with their two 16-byte halves swapped every 4 cells, so the eight
// row addresses of an ldmatrix phase hit eight different bank groups.
//
// Backward: the input gradient is the same convolution with the offsets
// reversed and the weights transposed; the weight gradient is a second GEMM
// (M = c_out, N = c_in, K = cells) per offset, accumulated by persistent CTAs
// and added to global memory once per CTA.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdlib>
#include <cmath>
#include <vector>

#include "pm_internal.cuh"

namespace pm {
namespace {

constexpr int NL = 4;                       // layers
constexpr int CH = 16;                      // padded channels
constexpr int NOFF = 27;
constexpr int WSZ = NOFF * CH * CH;         // weights of one layer (padded)
constexpr int PSZ = WSZ + CH;               // + bias
constexpr int NPARAM = NL * PSZ;
constexpr int CIN[NL] = {2, 16, 16, 16};
constexpr int COUT[NL] = {16, 16, 16, 3};
constexpr int TT = 8;                       // tile side
constexpr int HT = TT + 2;                  // halo tile side
constexpr int NH = HT * HT * HT;            // 1000 halo cells
constexpr int CONV_THREADS = 256;

__device__ __forceinline__ int wrapn(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// 16-byte chunk q (0: channels 0-7, 1: channels 8-15) of row r in a swizzled [rows][2] uint4 array
__device__ __forceinline__ int swz(int r, int q) { return 2 * r + (q ^ ((r >> 2) & 1)); }

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void ldm_x4(unsigned addr, unsigned (&r)[4])
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}
__device__ __forceinline__ void ldm_x4_t(unsigned addr, unsigned (&r)[4])
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}
// D += A (m16 x k16, row) * B (k16 x n8, col), BF16 inputs, FP32 accumulate
__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], unsigned b0, unsigned b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};\n"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// load the 10^3 halo of an 8^3 tile (BF16 [cell][16], 2 x 16 B per cell) into swizzled shared memory
__device__ __forceinline__ void load_halo(uint4 *sx, const uint4 *x, int n, int x0, int y0, int z0)
{
    for (int i = threadIdx.x; i < 2 * NH; i += blockDim.x) {
        const int h = i >> 1, q = i & 1;
        const int hx = h % HT, hy = (h / HT) % HT, hz = h / (HT * HT);
        const int64_t g = ((int64_t)wrapn(z0 - 1 + hz, n) * n + wrapn(y0 - 1 + hy, n)) * n + wrapn(x0 - 1 + hx, n);
        sx[swz(h, q)] = x[2 * g + q];
    }
}

// y = act(conv(x, w) + b): one 8^3 tile per CTA.  NB = 2 (16 outputs) or 1 (8 outputs).
template <int NB, bool RELU, bool OUTF32>
__global__ void __launch_bounds__(CONV_THREADS, 3)
    k_conv(const uint4 *__restrict__ x, const uint4 *__restrict__ w, const float *__restrict__ bias, void *y, int n)
{
    __shared__ uint4 sx[2 * NH];          // 32000 B
    __shared__ uint4 sw[2 * NOFF * CH];   // 13824 B
    const int nt = n / TT, b = blockIdx.x;
    const int x0 = (b % nt) * TT, y0 = ((b / nt) % nt) * TT, z0 = (b / (nt * nt)) * TT;
    load_halo(sx, x, n, x0, y0, z0);
    for (int i = threadIdx.x; i < 2 * NOFF * CH; i += blockDim.x) sw[swz(i >> 1, i & 1)] = w[i];
    __syncthreads();

    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    float acc[4][NB][4] = {};
    // per-lane row of the A fragments: cell (cx, cy = 2j + r / 8, cz = warp), chunk = lane / 16
    const int r = lane & 15, ach = lane >> 4;
    const int acx = r & 7, acy = r >> 3;
    // per-lane row of the B fragments: output channel co = (lane / 16) * 8 + lane % 8, chunk (lane / 8) % 2
    const int bco = ((lane >> 4) << 3) + (lane & 7), bch = (lane >> 3) & 1;
#pragma unroll 1
    for (int d = 0; d < NOFF; d++) {
        const int dz = d / 9 - 1, dy = (d / 3) % 3 - 1, dx = d % 3 - 1;
        unsigned bf[4];
        ldm_x4(smem_u32(&sw[swz(d * CH + bco, bch)]), bf);
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int h = ((warp + dz + 1) * HT + (2 * j + acy + dy + 1)) * HT + (acx + dx + 1);
            unsigned af[4];
            ldm_x4(smem_u32(&sx[swz(h, ach)]), af);
            mma_bf16(acc[j][0], af, bf[0], bf[1]);
            if (NB == 2) mma_bf16(acc[j][NB - 1], af, bf[2], bf[3]);
        }
    }
    // epilogue: rows g (cy = 2j) and g + 8 (cy = 2j + 1) of each m16 block, channels nb*8 + 2t, +1
#pragma unroll
    for (int j = 0; j < 4; j++)
#pragma unroll
        for (int hf = 0; hf < 2; hf++) {
            const int64_t cell = ((int64_t)(z0 + warp) * n + (y0 + 2 * j + hf)) * n + (x0 + g);
#pragma unroll
            for (int nb = 0; nb < NB; nb++) {
                const int ch = nb * 8 + 2 * t;
                float v0 = acc[j][nb][2 * hf] + (bias ? bias[ch] : 0.f);
                float v1 = acc[j][nb][2 * hf + 1] + (bias ? bias[ch + 1] : 0.f);
                if (RELU) {
                    v0 = fmaxf(v0, 0.f);
                    v1 = fmaxf(v1, 0.f);
                }
                if (OUTF32) {
                    reinterpret_cast<float2 *>(y)[(cell * (NB * 8) + ch) >> 1] = make_float2(v0, v1);
                } else {
                    reinterpret_cast<__nv_bfloat162 *>(y)[(cell * CH + ch) >> 1] = __floats2bfloat162_rn(v0, v1);
                }
            }
        }
}

// ---------------------------------------------------------------------------
// The same convolution on the 5th-generation tensor cores (tcgen05.mma, BF16 in,
// FP32 accumulate in tensor memory), for meshes with n % 16 == 0.  Persistent
// CTAs of 128 threads walk 8 x 16 x 4 tiles of cells.  A tile's 10 x 18 x 6 halo
// sits in shared memory in the canonical K-major layout without swizzle: the two
// 16-byte halves of the 16 input channels in separate regions, x-rows of 16-byte
// cells.  An M = 128 block is one z-plane of the tile (rows m = cx + 8 cy, core
// matrices = x-rows), so the operand for offset d is the halo itself seen from a
// shifted start address: 160 B between core matrices along M, 17280 B between the
// channel halves.  Per tile one thread issues 4 x 27 MMAs (M 128, N 16, K 16)
// into 64 TMEM columns and commits them to an mbarrier.  Two halo buffers and
// two TMEM accumulators form a pipeline: while the tensor core works on tile k,
// cp.async fetches the halo of tile k + 1 and the four warps read tile k - 1 back
// from TMEM (tcgen05.ld), add the bias, apply ReLU and store.  The weights are
// staged once per CTA.  Every wait is bounded.  On a timeout the CTA agrees on the
// failure at its next barrier, issues no further MMAs or halo loads, writes NaN
// outputs, and before freeing its TMEM waits once more (bounded) for every MMA
// batch it committed and has not seen complete; a batch still pending after that
// is counted as an unsafe exit, which poisons the convolution entry points.
// ---------------------------------------------------------------------------
constexpr int TCX = 8, TCY = 16, TCZ = 4;                      // tile (cells)
constexpr int HX = TCX + 2, HY = TCY + 2, HZ = TCZ + 2;        // halo 10 x 18 x 6
constexpr int NHT = HX * HY * HZ;                              // 1080 halo cells
constexpr int TC_THREADS = 128;
constexpr uint32_t HPY = HX * 16, HPZ = HY * HPY, HQ = HZ * HPZ;   // 160, 2880, 17280 bytes
constexpr uint32_t TC_HALO = 2 * HQ;                                // one halo buffer, 34560 bytes
constexpr uint32_t TC_A = 128, TC_B = TC_A + 2 * TC_HALO;          // shared-memory offsets
constexpr uint32_t TC_SMEM = TC_B + NOFF * 512;                     // 83072 bytes
constexpr uint32_t TC_COLS = 128;                                   // 2 accumulators x 4 M blocks x N 16
// kind::f16 instruction descriptor: FP32 D (bit 4), BF16 A (bits 7-9) and B (10-12), both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);

__device__ unsigned int g_conv_tc_timeouts;
__device__ unsigned int g_conv_tc_unsafe;   // CTAs that freed TMEM with an MMA batch possibly in flight

// shared-memory matrix descriptor, no swizzle: start, leading (K) and stride (M/N) byte offsets
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}

// bounded wait for an mbarrier phase: each try suspends the thread for up to ~0.1 ms
__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t parity)
{
    uint32_t done = 0;
    for (int it = 0; it < (1 << 14) && !done; it++)
        asm volatile("{\n\t.reg .pred q;\n\tmbarrier.try_wait.parity.shared::cta.b64 q, [%1], %2, %3;\n\t"
                     "selp.u32 %0, 1, 0, q;\n\t}"
                     : "=r"(done)
                     : "r"(mbar), "r"(parity), "r"(100000u));
    return done != 0;
}

__device__ __forceinline__ void tc_tile_origin(int tile, int n, int &x0, int &y0, int &z0)
{
    const int ntx = n / TCX, nty = n / TCY;
    x0 = (tile % ntx) * TCX;
    y0 = ((tile / ntx) % nty) * TCY;
    z0 = (tile / (ntx * nty)) * TCZ;
}

// cp.async of one tile's halo into buffer `buf`: half q of halo cell (hx, hy, hz) at q HQ + hz HPZ + hy HPY + 16 hx
__device__ __forceinline__ void tc_load_halo(uint32_t buf, const uint4 *x, int n, int tile)
{
    int x0, y0, z0;
    tc_tile_origin(tile, n, x0, y0, z0);
    for (int i = threadIdx.x; i < 2 * NHT; i += TC_THREADS) {
        const int h = i >> 1, q = i & 1;
        const int hx = h % HX, hy = (h / HX) % HY, hz = h / (HX * HY);
        const int64_t g = ((int64_t)wrapn(z0 - 1 + hz, n) * n + wrapn(y0 - 1 + hy, n)) * n + wrapn(x0 - 1 + hx, n);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(buf + q * HQ + hz * HPZ + hy * HPY + 16 * hx),
                     "l"(x + 2 * g + q));
    }
    asm volatile("cp.async.commit_group;");
}

// read the 4 M blocks of accumulator `acc` (TMEM column offset) back, add bias, activate, store.  MASK (BF16
// output only): zero every output channel whose value in mact ([cell][16] BF16) is not positive, the ReLU
// derivative of a layer whose output mact is, and add the stored values to part[channel].
template <bool RELU, bool OUTF32, bool MASK>
__device__ __forceinline__ void tc_epilogue(uint32_t tmem, uint32_t acc, const float *bias, void *y, int n, int tile,
                                            bool ok, const uint4 *mact, float (&part)[16])
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int x0, y0, z0;
    tc_tile_origin(tile, n, x0, y0, z0);
    // TMEM lane 32 warp + lane = M row m = cx + 8 cy of every z-plane block t (columns 16 t .. 16 t + 15)
    const int m = 32 * warp + lane, cx = m & 7, cy = m >> 3;
    uint4 mk[MASK ? TCZ : 1][2];   // the mask cells of all z-planes, loaded before the accumulator is read
    if constexpr (MASK) {
#pragma unroll
        for (int t = 0; t < TCZ; t++) {
            const int64_t cell = ((int64_t)(z0 + t) * n + (y0 + cy)) * n + (x0 + cx);
            mk[t][0] = mact[2 * cell];
            mk[t][1] = mact[2 * cell + 1];
        }
    }
    auto plane = [&](const int t) {
        uint32_t r[16] = {};
        if (ok) {   // warp-uniform: after a timeout the accumulator is not read
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                         "[%16];"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                           "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                           "=r"(r[14]), "=r"(r[15])
                         : "r"(tmem + ((uint32_t)(32 * warp) << 16) + acc + 16 * t));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
        }
        float v[16];
#pragma unroll
        for (int c = 0; c < 16; c++) {
            v[c] = ok ? __uint_as_float(r[c]) + (bias ? bias[c] : 0.f) : __int_as_float(0x7fc00000);
            if (RELU) v[c] = fmaxf(v[c], 0.f);
        }
        const int64_t cell = ((int64_t)(z0 + t) * n + (y0 + cy)) * n + (x0 + cx);
        if (OUTF32) {
            float4 *o = reinterpret_cast<float4 *>(y) + 2 * cell;
            o[0] = make_float4(v[0], v[1], v[2], v[3]);
            o[1] = make_float4(v[4], v[5], v[6], v[7]);
        } else {
            uint4 o[2];
            __nv_bfloat162 *ob = reinterpret_cast<__nv_bfloat162 *>(o);
#pragma unroll
            for (int c = 0; c < 8; c++) ob[c] = __floats2bfloat162_rn(v[2 * c], v[2 * c + 1]);
            if constexpr (MASK) {
                const uint4 m0 = mk[t][0], m1 = mk[t][1];
                const unsigned mw[8] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
                unsigned *ow = reinterpret_cast<unsigned *>(o);
#pragma unroll
                for (int k = 0; k < 8; k++) {
                    const bool lo = __uint_as_float(mw[k] << 16) > 0.f, hi = __uint_as_float(mw[k] & 0xffff0000u) > 0.f;
                    ow[k] &= (lo ? 0x0000ffffu : 0u) | (hi ? 0xffff0000u : 0u);
                    part[2 * k] += __uint_as_float(ow[k] << 16);
                    part[2 * k + 1] += __uint_as_float(ow[k] & 0xffff0000u);
                }
            }
            uint4 *dst = reinterpret_cast<uint4 *>(y) + 2 * cell;
            dst[0] = o[0];
            dst[1] = o[1];
        }
    };
    // unrolled for the BF16 outputs (the mask registers need static indices); the FP32 output layer runs
    // faster rolled
    if constexpr (OUTF32) {
#pragma unroll 1
        for (int t = 0; t < TCZ; t++) plane(t);
    } else {
#pragma unroll
        for (int t = 0; t < TCZ; t++) plane(t);
    }
}

template <bool RELU, bool OUTF32, bool MASK>
__global__ void __launch_bounds__(TC_THREADS)
    k_conv_tc(const uint4 *__restrict__ x, const uint4 *__restrict__ w, const float *__restrict__ bias, void *y, int n,
              int ntiles, int skip_mma, const uint4 *__restrict__ mact, float *db)
{
    extern __shared__ __align__(128) unsigned char smem[];
    float part[16] = {};   // MASK: this thread's sums of the stored values per channel
    const uint32_t sbase = smem_u32(smem);
    const uint32_t mbar0 = sbase, tslot = sbase + 16;   // mbarriers at +0 and +8
    const int tid = threadIdx.x, warp = tid >> 5;
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tslot), "r"(TC_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar0));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbar0 + 8));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    // weights of offset d: half q of output channel co at TC_B + 512 d + 256 q + 16 co (once per CTA)
    for (int i = tid; i < 2 * NOFF * CH; i += TC_THREADS) {
        const int row = i >> 1, q = i & 1;   // row = d * 16 + co
        *reinterpret_cast<uint4 *>(smem + TC_B + 512 * (row >> 4) + 256 * q + 16 * (row & 15)) = w[i];
    }
    const int first = blockIdx.x, step = gridDim.x;
    if (first < ntiles) tc_load_halo(sbase + TC_A, x, n, first);
    uint32_t tmem = 0;
    bool ok = true;
    // MMA batches committed to mbarrier 0 / 1 and the waits on them that completed (all threads count the
    // commits alike, since ok is CTA-uniform where they are issued)
    int iss0 = 0, iss1 = 0, fin0 = 0, fin1 = 0;
    int k = 0;
    for (int tile = first; tile < ntiles; tile += step, k++) {
        const int j = k & 1;
        // 1. this tile's halo (and, the first time, the weights) visible to the tensor core; the CTA agrees
        //    on whether any wait has timed out
        asm volatile("cp.async.wait_group 0;");
        asm volatile("fence.proxy.async.shared::cta;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        ok = __syncthreads_and(ok) != 0;
        asm volatile("tcgen05.fence::after_thread_sync;");
        tmem = *reinterpret_cast<volatile uint32_t *>(smem + 16);
        // 2. MMAs of this tile into accumulator j
        if (ok && !skip_mma) {
            if (j) iss1++;
            else iss0++;
        }
        if (tid == 0 && ok && !skip_mma) {
            // the start-address field is the low bits of a descriptor: shifted operands are the base
            // descriptor plus a compile-time offset / 16
            const uint64_t a0 = tc_desc(sbase + TC_A + j * TC_HALO, HQ, HPY), b0 = tc_desc(sbase + TC_B, 256, 128);
            const uint32_t d0 = tmem + 64 * j;
#pragma unroll
            for (int t = 0; t < TCZ; t++)
#pragma unroll
                for (int d = 0; d < NOFF; d++) {
                    const int dz = d / 9 - 1, dy = (d / 3) % 3 - 1, dx = d % 3 - 1;
                    const uint32_t off = (t + dz + 1) * HPZ + (dy + 1) * HPY + (dx + 1) * 16;
                    const uint64_t ad = a0 + (off >> 4), bd = b0 + 32 * d;
                    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d0 + 16 * t),
                                 "l"(ad), "l"(bd), "r"(TC_IDESC), "r"(d > 0 ? 1u : 0u));
                }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                mbar0 + 8 * j));
        }
        // 3. the previous tile's MMAs: its halo buffer becomes free and its accumulator readable
        if (k > 0 && ok) {
            if (tc_wait(mbar0 + 8 * (1 - j), ((k - 1) >> 1) & 1)) {
                if (j) fin0++;
                else fin1++;
            } else {
                ok = false;
                if ((tid & 31) == 0) atomicAdd(&g_conv_tc_timeouts, 1u);
            }
            ok = __all_sync(0xffffffffu, ok) != 0;   // warp-uniform for the TMEM reads
            asm volatile("tcgen05.fence::after_thread_sync;");
        }
        // 4. the next tile's halo into the free buffer (none after a timeout: the buffer may still be read)
        if (ok && tile + step < ntiles) tc_load_halo(sbase + TC_A + (1 - j) * TC_HALO, x, n, tile + step);
        // 5. the previous tile's results
        if (k > 0) tc_epilogue<RELU, OUTF32, MASK>(tmem, 64 * (1 - j), bias, y, n, tile - step, ok, mact, part);
    }
    if (k > 0) {
        const int last = first + (k - 1) * step, j = (k - 1) & 1;
        if (ok) {
            if (tc_wait(mbar0 + 8 * j, ((k - 1) >> 1) & 1)) {
                if (j) fin1++;
                else fin0++;
            } else {
                ok = false;
                if ((tid & 31) == 0) atomicAdd(&g_conv_tc_timeouts, 1u);
            }
            ok = __all_sync(0xffffffffu, ok) != 0;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        tc_epilogue<RELU, OUTF32, MASK>(tmem, 64 * j, bias, y, n, last, ok, mact, part);
    }
    if constexpr (MASK) {
        // db[c] += the CTA's sum of part[c]
        __shared__ float red[TC_THREADS / 32][16];
#pragma unroll
        for (int c = 0; c < 16; c++)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) part[c] += __shfl_xor_sync(0xffffffffu, part[c], o);
        if ((tid & 31) == 0)
#pragma unroll
            for (int c = 0; c < 16; c++) red[warp][c] = part[c];
        __syncthreads();
        if (tid < 16) {
            float t = 0.f;
            for (int w2 = 0; w2 < TC_THREADS / 32; w2++) t += red[w2][tid];
            atomicAdd(&db[tid], t);
        }
    }
    asm volatile("cp.async.wait_group 0;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    ok = __syncthreads_and(ok) != 0;
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0) {
        if (!ok) {
            // drain: at most one batch per mbarrier is outstanding (a batch is committed only after the wait on
            // the previous batch of the same mbarrier completed); its phase parity is the completed count's.
            // Re-waiting a phase this thread gave up on but that completed since returns at once.
            bool drained = true;
            if (iss0 > fin0) drained = tc_wait(mbar0, fin0 & 1) && drained;
            if (iss1 > fin1) drained = tc_wait(mbar0 + 8, fin1 & 1) && drained;
            if (!drained) atomicAdd(&g_conv_tc_unsafe, 1u);
            __syncwarp();
            asm volatile("tcgen05.fence::after_thread_sync;");
        }
        tmem = *reinterpret_cast<volatile uint32_t *>(smem + 16);
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_COLS));
    }
}

// First layer (2 input channels): the K dimension packs 8 offsets x 2 channels per k16 step, so 27
// offsets take 4 steps instead of 27 (slots of offsets 27..31 carry zero weights).  A fragments
// are built from 4-byte (2-channel) shared-memory loads, B fragments once per thread from the
// weights in global memory.  y = relu(conv(x, w) + b), BF16 [cell][16].
__global__ void __launch_bounds__(CONV_THREADS, 3)
    k_conv_in2(const uint4 *__restrict__ x, const __nv_bfloat16 *__restrict__ w, const float *__restrict__ bias,
               __nv_bfloat16 *y, int n)
{
    __shared__ unsigned sx2[NH];   // channels 0-1 of the 10^3 halo cells
    const int nt = n / TT, b = blockIdx.x;
    const int x0 = (b % nt) * TT, y0 = ((b / nt) % nt) * TT, z0 = (b / (nt * nt)) * TT;
    for (int h = threadIdx.x; h < NH; h += blockDim.x) {
        const int hx = h % HT, hy = (h / HT) % HT, hz = h / (HT * HT);
        const int64_t g = ((int64_t)wrapn(z0 - 1 + hz, n) * n + wrapn(y0 - 1 + hy, n)) * n + wrapn(x0 - 1 + hx, n);
        sx2[h] = reinterpret_cast<const unsigned *>(x)[8 * g];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
    // B fragments: k = 16 s + 2 t (+1) -> offset 8 s + t, channels 0, 1; k + 8 -> offset 8 s + t + 4
    unsigned bf[4][2][2];
#pragma unroll
    for (int s4 = 0; s4 < 4; s4++)
#pragma unroll
        for (int nb = 0; nb < 2; nb++)
#pragma unroll
            for (int hfk = 0; hfk < 2; hfk++) {
                const int oi = 8 * s4 + t + 4 * hfk;
                bf[s4][nb][hfk] = oi < NOFF ? reinterpret_cast<const unsigned *>(w)[((oi * CH) + nb * 8 + g) * CH / 2] : 0u;
            }
    __syncthreads();
    float acc[4][2][4] = {};
#pragma unroll
    for (int s4 = 0; s4 < 4; s4++) {
        int hoff[2];
#pragma unroll
        for (int hfk = 0; hfk < 2; hfk++) {
            const int oi = min(8 * s4 + t + 4 * hfk, NOFF - 1);   // zero-weight slots read any valid cell
            const int dz = oi / 9 - 1, dy = (oi / 3) % 3 - 1, dx = oi % 3 - 1;
            hoff[hfk] = ((warp + dz + 1) * HT + (dy + 1)) * HT + (g + dx + 1);
        }
#pragma unroll
        for (int j = 0; j < 4; j++) {
            unsigned af[4];
            af[0] = sx2[hoff[0] + (2 * j) * HT];       // row g (cy = 2j), k = 16 s + 2t
            af[1] = sx2[hoff[0] + (2 * j + 1) * HT];   // row g + 8 (cy = 2j + 1)
            af[2] = sx2[hoff[1] + (2 * j) * HT];       // row g, k + 8
            af[3] = sx2[hoff[1] + (2 * j + 1) * HT];   // row g + 8, k + 8
#pragma unroll
            for (int nb = 0; nb < 2; nb++) mma_bf16(acc[j][nb], af, bf[s4][nb][0], bf[s4][nb][1]);
        }
    }
#pragma unroll
    for (int j = 0; j < 4; j++)
#pragma unroll
        for (int hf = 0; hf < 2; hf++) {
            const int64_t cell = ((int64_t)(z0 + warp) * n + (y0 + 2 * j + hf)) * n + (x0 + g);
#pragma unroll
            for (int nb = 0; nb < 2; nb++) {
                const int ch = nb * 8 + 2 * t;
                const float v0 = fmaxf(acc[j][nb][2 * hf] + bias[ch], 0.f);
                const float v1 = fmaxf(acc[j][nb][2 * hf + 1] + bias[ch + 1], 0.f);
                reinterpret_cast<__nv_bfloat162 *>(y)[(cell * CH + ch) >> 1] = __floats2bfloat162_rn(v0, v1);
            }
        }
}

// dw[d][co][ci] += sum_cells g[cell][co] x[cell + d][ci]; persistent CTAs over 8^3 tiles.
// Warp w of DW_WARPS owns the offsets d = w, w + DW_WARPS, ...  Two shared-memory buffers,
// each one tile's 10^3 input halo and 8^3 gradient block: cp.async fetches tile k + 1 into one
// while the warps run tile k's MMAs from the other.
constexpr int DW_WARPS = 8;
constexpr int DW_OFFS = (NOFF + DW_WARPS - 1) / DW_WARPS;   // offsets per warp (at most)
constexpr int DW_HALO = 2 * NH;                        // uint4 per buffer: input halo
constexpr int DW_BUF = DW_HALO + 2 * TT * TT * TT;     // + gradient block
constexpr size_t DW_SMEM = 2 * DW_BUF * sizeof(uint4);  // 96768 bytes

__device__ __forceinline__ void cp_async16(void *s, const void *g)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(s)), "l"(g));
}

// one tile's halo of x and gradient block into buffer sb.  Halo cell h = (hz HT + hy) HT + hx keeps its
// 16-byte half q at uint4 2 h + (q ^ bit 2 of hx): the 8 cells of one x-row that an ldmatrix reads then
// fall in distinct banks, and the swizzle of a shifted operand does not change from one k-step to the
// next.  The gradient block uses swz (row = tile cell).
__device__ __forceinline__ int dw_hswz(int h, int hx, int q) { return 2 * h + (q ^ ((hx >> 2) & 1)); }

__device__ __forceinline__ void dw_fetch(uint4 *sb, const uint4 *x, const uint4 *gr, int n, int nt, int tile)
{
    const int x0 = (tile % nt) * TT, y0 = ((tile / nt) % nt) * TT, z0 = (tile / (nt * nt)) * TT;
    for (int i = threadIdx.x; i < 2 * NH; i += blockDim.x) {
        const int h = i >> 1, q = i & 1;
        const int hx = h % HT, hy = (h / HT) % HT, hz = h / (HT * HT);
        const int64_t g = ((int64_t)wrapn(z0 - 1 + hz, n) * n + wrapn(y0 - 1 + hy, n)) * n + wrapn(x0 - 1 + hx, n);
        cp_async16(&sb[dw_hswz(h, hx, q)], &x[2 * g + q]);
    }
    uint4 *sg = sb + DW_HALO;
    for (int i = threadIdx.x; i < 2 * TT * TT * TT; i += blockDim.x) {
        const int m = i >> 1, q = i & 1;
        const int cx = m & 7, cy = (m >> 3) & 7, cz = m >> 6;
        const int64_t gc = ((int64_t)(z0 + cz) * n + (y0 + cy)) * n + (x0 + cx);
        cp_async16(&sg[swz(m, q)], &gr[2 * gc + q]);
    }
    asm volatile("cp.async.commit_group;");
}

__global__ void __launch_bounds__(32 * DW_WARPS, 2)
    k_conv_dw(const uint4 *__restrict__ x, const uint4 *__restrict__ gr, float *dw, int n)
{
    extern __shared__ uint4 dsm[];   // 2 x DW_BUF
    const int nt = n / TT, ntiles = nt * nt * nt;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float acc[DW_OFFS][2][4] = {};
    // ldmatrix.trans lane roles.  G (A operand, rows = cells, chunk = co half): matrix mi = lane / 8
    // covers cells (mi / 2) * 8 + lane % 8 of the k16 step, chunk mi % 2.
    const int ga_cell = ((lane >> 4) << 3) + (lane & 7), ga_ch = (lane >> 3) & 1;
    // X (B operand): cells ((lane / 8) % 2) * 8 + lane % 8, chunk (lane / 16) = n8 block.
    const int xb_cell = (((lane >> 3) & 1) << 3) + (lane & 7), xb_ch = lane >> 4;
    // k-step s covers tile cells 16 s .. 16 s + 15: z = s / 4, y = 2 (s % 4) + k / 8, x = k % 8.  The byte
    // address of every operand row is a per-lane (and per-offset) base plus a multiple of s known at
    // compile time (the swizzle bits do not depend on s): 512 s for G, 3200 (s / 4) + 640 (s % 4) for X.
    const uint32_t ga_off = 16u * swz(ga_cell, ga_ch);
    uint32_t xb_off[DW_OFFS];
#pragma unroll
    for (int o = 0; o < DW_OFFS; o++) {
        const int d = min(warp + DW_WARPS * o, NOFF - 1);
        const int dz = d / 9 - 1, dy = (d / 3) % 3 - 1, dx = d % 3 - 1;
        const int hx = (xb_cell & 7) + dx + 1;
        const int h = ((dz + 1) * HT + (xb_cell >> 3) + dy + 1) * HT + hx;
        xb_off[o] = 16u * dw_hswz(h, hx, xb_ch);
    }
    if ((int)blockIdx.x < ntiles) dw_fetch(dsm, x, gr, n, nt, blockIdx.x);
    int b = 0;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x, b ^= 1) {
        // buffer b ^ 1 was last read before the barrier that ended the previous iteration
        if (tile + (int)gridDim.x < ntiles) {
            dw_fetch(dsm + (b ^ 1) * DW_BUF, x, gr, n, nt, tile + gridDim.x);
            asm volatile("cp.async.wait_group 1;" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;" ::: "memory");
        }
        __syncthreads();
        const uint32_t sx = smem_u32(dsm + b * DW_BUF), sg = sx + 16u * DW_HALO;
#pragma unroll
        for (int s = 0; s < 32; s++) {
            unsigned af[4];
            ldm_x4_t(sg + ga_off + 512u * s, af);
#pragma unroll
            for (int o = 0; o < DW_OFFS; o++) {
                if (warp + DW_WARPS * o < NOFF) {
                    unsigned bf[4];
                    ldm_x4_t(sx + xb_off[o] + 32u * (HT * HT * (s >> 2) + HT * 2 * (s & 3)), bf);
                    // x4.trans matrices: 0 = (cells 0-7, chunk 0), 1 = (cells 8-15, chunk 0),
                    // 2 = (cells 0-7, chunk 1), 3 = (cells 8-15, chunk 1)
                    mma_bf16(acc[o][0], af, bf[0], bf[1]);
                    mma_bf16(acc[o][1], af, bf[2], bf[3]);
                }
            }
        }
        __syncthreads();
    }
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int o = 0; o < DW_OFFS; o++) {
        const int d = warp + DW_WARPS * o;
        if (d >= NOFF) continue;
#pragma unroll
        for (int nb = 0; nb < 2; nb++) {
            float *base = dw + (size_t)d * CH * CH;
            const int ci = nb * 8 + 2 * t;
            atomicAdd(&base[g * CH + ci], acc[o][nb][0]);
            atomicAdd(&base[g * CH + ci + 1], acc[o][nb][1]);
            atomicAdd(&base[(g + 8) * CH + ci], acc[o][nb][2]);
            atomicAdd(&base[(g + 8) * CH + ci + 1], acc[o][nb][3]);
        }
    }
}

// G = g * (y > 0) (mask != 0) or G = g, and db[c] += sum_cells G[cell][c].  16-byte accesses: chunk i of the
// [cell][16] BF16 arrays holds channels 8 (i % 2) .. 8 (i % 2) + 7, and with an even grid stride a thread
// keeps its chunk parity, so it sums a fixed set of 8 channels.
__global__ void k_mask(const uint4 *gin, const uint4 *yact, uint4 *gout, float *db, int64_t ncell, int mask)
{
    __shared__ float sdb[CONV_THREADS / 32][CH];
    float part[8] = {};
    const int64_t total = 2 * ncell;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        uint4 gv = gin[i];
        unsigned *gw = reinterpret_cast<unsigned *>(&gv);
        if (mask) {
            const uint4 yv = yact[i];
            const unsigned *yw = reinterpret_cast<const unsigned *>(&yv);
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const bool lo = __uint_as_float(yw[k] << 16) > 0.f, hi = __uint_as_float(yw[k] & 0xffff0000u) > 0.f;
                gw[k] &= (lo ? 0x0000ffffu : 0u) | (hi ? 0xffff0000u : 0u);
            }
        }
        gout[i] = gv;
#pragma unroll
        for (int k = 0; k < 4; k++) {
            part[2 * k] += __uint_as_float(gw[k] << 16);
            part[2 * k + 1] += __uint_as_float(gw[k] & 0xffff0000u);
        }
    }
    // lanes of equal parity hold the same channels
#pragma unroll
    for (int o = 2; o < 32; o <<= 1)
#pragma unroll
        for (int k = 0; k < 8; k++) part[k] += __shfl_xor_sync(0xffffffffu, part[k], o);
    const int lane = threadIdx.x & 31;
    if (lane < 2)
#pragma unroll
        for (int k = 0; k < 8; k++) sdb[threadIdx.x >> 5][8 * lane + k] = part[k];
    __syncthreads();
    if (threadIdx.x < CH) {
        float t = 0.f;
        for (int w = 0; w < CONV_THREADS / 32; w++) t += sdb[w][threadIdx.x];
        atomicAdd(&db[threadIdx.x], t);
    }
}

// loss = mean over cells and channels 0..2 of (out - tgt)^2; G = 2 (out - tgt) / (3 ncell) as BF16 [cell][16],
// and db[c] += sum over cells of G[cell][c] (c < 3; the other channels of G are zero)
__global__ void k_loss(const float *out, const float *tgt, __nv_bfloat16 *gr, double *loss, float *db, int64_t ncell)
{
    __shared__ double sl[CONV_THREADS / 32];
    __shared__ float sdb[CONV_THREADS / 32][3];
    double part = 0.0;
    float pdb[3] = {0.f, 0.f, 0.f};
    const float sc = 2.f / (3.f * (float)ncell);
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x) {
        __nv_bfloat162 gv[8];
#pragma unroll
        for (int k = 0; k < 8; k++) gv[k] = __floats2bfloat162_rn(0.f, 0.f);
        float d[3];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            d[a] = out[8 * c + a] - tgt[8 * c + a];
            part += (double)d[a] * (double)d[a];
        }
        gv[0] = __floats2bfloat162_rn(sc * d[0], sc * d[1]);
        gv[1] = __floats2bfloat162_rn(sc * d[2], 0.f);
        pdb[0] += __low2float(gv[0]);
        pdb[1] += __high2float(gv[0]);
        pdb[2] += __low2float(gv[1]);
        uint4 *dst = reinterpret_cast<uint4 *>(gr + 16 * c);
        dst[0] = *reinterpret_cast<uint4 *>(&gv[0]);
        dst[1] = *reinterpret_cast<uint4 *>(&gv[4]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        part += __shfl_down_sync(0xffffffffu, part, o);
#pragma unroll
        for (int a = 0; a < 3; a++) pdb[a] += __shfl_down_sync(0xffffffffu, pdb[a], o);
    }
    if ((threadIdx.x & 31) == 0) {
        sl[threadIdx.x >> 5] = part;
#pragma unroll
        for (int a = 0; a < 3; a++) sdb[threadIdx.x >> 5][a] = pdb[a];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < CONV_THREADS / 32; w++) s += sl[w];
        atomicAdd(loss, s / (3.0 * (double)ncell));
    }
    if (threadIdx.x < 3) {
        float t = 0.f;
        for (int w = 0; w < CONV_THREADS / 32; w++) t += sdb[w][threadIdx.x];
        atomicAdd(&db[threadIdx.x], t);
    }
}

// BF16 copies of the FP32 master parameters: forward weights [l][27][co][ci], transposed and
// offset-reversed weights [l][27][ci][co] (input-gradient convolution), FP32 biases
__global__ void k_pack(const float *theta, __nv_bfloat16 *wf, __nv_bfloat16 *wt, float *bias)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NPARAM) return;
    const int l = i / PSZ, e = i % PSZ;
    if (e >= WSZ) {
        bias[l * CH + (e - WSZ)] = theta[i];
        return;
    }
    const int d = e / (CH * CH), co = (e / CH) % CH, ci = e % CH;
    const __nv_bfloat16 v = __float2bfloat16_rn(theta[i]);
    wf[(size_t)l * WSZ + e] = v;
    wt[(size_t)l * WSZ + ((NOFF - 1 - d) * CH + ci) * CH + co] = v;
}

// one Adam step (Kingma & Ba 2015) on every parameter; zeroes the gradient for the next step
__global__ void k_adam(float *theta, float *grad, float *m, float *v, float lr, float b1, float b2, float eps,
                       float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NPARAM) return;
    const float g = grad[i];
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    grad[i] = 0.f;
}

// network inputs from a solved context: channel 0 = s_delta R / kappa, channel 1 = s_phi phi N^2 / kappa
template <class T>
__global__ void k_features(const T *R, const T *phi, double s0, double s1, __nv_bfloat16 *x, int64_t ncell)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    __nv_bfloat162 v[8];
    v[0] = __floats2bfloat162_rn((float)((double)R[c] * s0), (float)((double)phi[c] * s1));
#pragma unroll
    for (int k = 1; k < 8; k++) v[k] = __floats2bfloat162_rn(0.f, 0.f);
    uint4 *dst = reinterpret_cast<uint4 *>(x + 16 * c);
    dst[0] = *reinterpret_cast<uint4 *>(&v[0]);
    dst[1] = *reinterpret_cast<uint4 *>(&v[4]);
}

// target = (restriction of the fine-mesh force - coarse-mesh force) N / kappa, FP32 [cell][8]
template <class T>
__global__ void k_target(const T *phic, const T *phif, int n, double scale, float *tgt)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nc = (int64_t)n * n * n;
    if (c >= nc) return;
    const int x = (int)(c % n), y = (int)((c / n) % n), z = (int)(c / ((int64_t)n * n));
    const int m = 2 * n;
    auto pc = [&](int a, int b, int cc) { return (double)phic[((int64_t)wrapn(cc, n) * n + wrapn(b, n)) * n + wrapn(a, n)]; };
    auto pf = [&](int a, int b, int cc) {
        a = a < 0 ? a + m : (a >= m ? a - m : a);
        b = b < 0 ? b + m : (b >= m ? b - m : b);
        cc = cc < 0 ? cc + m : (cc >= m ? cc - m : cc);
        return (double)phif[((int64_t)cc * m + b) * m + a];
    };
    const double fc[3] = {-(pc(x + 1, y, z) - pc(x - 1, y, z)) * 0.5 * n, -(pc(x, y + 1, z) - pc(x, y - 1, z)) * 0.5 * n,
                          -(pc(x, y, z + 1) - pc(x, y, z - 1)) * 0.5 * n};
    double ff[3] = {0, 0, 0};
    for (int ez = -1; ez <= 1; ez++)
        for (int ey = -1; ey <= 1; ey++)
            for (int ex = -1; ex <= 1; ex++) {
                const double wgt = (ex ? 0.25 : 0.5) * (ey ? 0.25 : 0.5) * (ez ? 0.25 : 0.5);
                const int X = 2 * x + ex, Y = 2 * y + ey, Z = 2 * z + ez;
                ff[0] -= wgt * (pf(X + 1, Y, Z) - pf(X - 1, Y, Z)) * 0.5 * m;
                ff[1] -= wgt * (pf(X, Y + 1, Z) - pf(X, Y - 1, Z)) * 0.5 * m;
                ff[2] -= wgt * (pf(X, Y, Z + 1) - pf(X, Y, Z - 1)) * 0.5 * m;
            }
    float4 *dst = reinterpret_cast<float4 *>(tgt + 8 * c);
    dst[0] = make_float4((float)((ff[0] - fc[0]) * scale), (float)((ff[1] - fc[1]) * scale),
                         (float)((ff[2] - fc[2]) * scale), 0.f);
    dst[1] = make_float4(0.f, 0.f, 0.f, 0.f);
}

}  // namespace

// the extra kick of a force correction c (FP32 [cell][8], channels 0..2 = force units):
// u += dtau_kick * f * c(x_p) with f = a_n (Newtonian) or E = sqrt(a_n^2 + u^2), in the
// context's precision (FP32 in the mixed form: FP64 arithmetic is slow on this part)
template <class T>
__global__ void k_corr_kick(Particle<T> *part, int64_t np, const float *corr, T scale, int n, T a, T dtk,
                            int newtonian)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= np) return;
    Particle<T> P = part[i];
    const int cell = P.cell;
    const int x = cell % n, y = (cell / n) % n, z = cell / (n * n);
    const int xp = x + 1 == n ? 0 : x + 1, yp = y + 1 == n ? 0 : y + 1, zp = z + 1 == n ? 0 : z + 1;
    const T wx[2] = {T(1) - P.f[0], P.f[0]}, wy[2] = {T(1) - P.f[1], P.f[1]}, wz[2] = {T(1) - P.f[2], P.f[2]};
    const int xs[2] = {x, xp}, ys[2] = {y, yp}, zs[2] = {z, zp};
    T cv[3] = {0, 0, 0};
#pragma unroll
    for (int dz = 0; dz < 2; dz++)
#pragma unroll
        for (int dy = 0; dy < 2; dy++) {
            const T wyz = wy[dy] * wz[dz];
            const int64_t row = ((int64_t)zs[dz] * n + ys[dy]) * n;
#pragma unroll
            for (int dx = 0; dx < 2; dx++) {
                const T w = wx[dx] * wyz;
                const float4 c4 = reinterpret_cast<const float4 *>(corr)[2 * (row + xs[dx])];
                cv[0] += w * (T)c4.x;
                cv[1] += w * (T)c4.y;
                cv[2] += w * (T)c4.z;
            }
        }
    T f = a * scale;
    if (!newtonian) f = sqrt(a * a + P.u[0] * P.u[0] + P.u[1] * P.u[1] + P.u[2] * P.u[2]) * scale;
#pragma unroll
    for (int k = 0; k < 3; k++) P.u[k] += dtk * f * cv[k];
    part[i] = P;
}

template <class T> void launch_corr_kick(Ctx &c, const StepScalars &s)
{
    if (!c.corr) return;
    const int64_t nb = (c.np + 255) / 256;
    k_corr_kick<T><<<(unsigned)nb, 256, 0, c.stream>>>(reinterpret_cast<Particle<T> *>(c.part[c.cur]), c.np,
                                                         static_cast<const float *>(c.corr), (T)c.corr_scale, c.N,
                                                         (T)s.a, (T)s.dtau_kick, s.newtonian);
    c.launches++;
}
template void launch_corr_kick<float>(Ctx &, const StepScalars &);
template void launch_corr_kick<double>(Ctx &, const StepScalars &);

}  // namespace pm

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
using namespace pm;

struct pm_net {
    int n = 0;
    int64_t ncell = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    float *theta = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;   // NPARAM each
    __nv_bfloat16 *wf = nullptr, *wt = nullptr;                            // NL * WSZ each
    float *bias = nullptr;                                                 // NL * CH
    __nv_bfloat16 *act[NL] = {};      // act[0] = inputs, act[l] = output of layer l-1 ([cell][16])
    __nv_bfloat16 *g0 = nullptr, *g1 = nullptr;   // gradient ping-pong ([cell][16])
    float *out = nullptr;             // network output [cell][8]
    double *dloss = nullptr;
    int64_t adam_t = 0;
    double s_delta = 1.0, s_phi = 1.0, s_target = 1.0;   // input and target normalisation
};

namespace {

// set once a CTA of the tensor-core convolution had to free its TMEM while an MMA batch it committed may still
// have been running (a wait ran out twice): every later convolution call returns PM_ERR_STATE
std::atomic<bool> g_conv_poisoned{false};

pm_status net_fail(pm_net *e, pm_status st, const char *msg)
{
    e->err = msg;
    return st;
}

unsigned grid_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// the 16-channel convolution: tensor-core (tcgen05) kernel for n % 16 == 0, mma.sync kernel otherwise
template <bool RELU, bool OUTF32, bool MASK = false>
void launch_conv_tc(const uint4 *x, const uint4 *w, const float *b, void *y, int n, cudaStream_t st,
                    const uint4 *mact = nullptr, float *db = nullptr)
{
    static std::atomic<uint64_t> done{0};
    if (first_on_device(done))
        cudaFuncSetAttribute(k_conv_tc<RELU, OUTF32, MASK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
    const int ntiles = (n / TCX) * (n / TCY) * (n / TCZ);
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = std::max(1, std::min(ntiles, 2 * std::max(sms, 1)));   // two resident CTAs per SM
    // PM_TEST_CONV_TIMEOUT=1 (test hook): no MMA is issued, so every bounded wait runs out
    const char *inj = std::getenv("PM_TEST_CONV_TIMEOUT");
    const int skip = inj && std::atoi(inj) != 0;
    k_conv_tc<RELU, OUTF32, MASK><<<grid, TC_THREADS, TC_SMEM, st>>>(x, w, b, y, n, ntiles, skip, mact, db);
}

bool conv_on_tcgen05(int n) { return n % TCY == 0; }

void conv16(const uint4 *x, const uint4 *w, const float *b, void *y, int n, bool relu, bool f32, cudaStream_t st)
{
    if (conv_on_tcgen05(n)) {
        if (f32) launch_conv_tc<false, true>(x, w, b, y, n, st);
        else if (relu) launch_conv_tc<true, false>(x, w, b, y, n, st);
        else launch_conv_tc<false, false>(x, w, b, y, n, st);
        return;
    }
    const int ntiles = (n / TT) * (n / TT) * (n / TT);
    if (f32)
        k_conv<1, false, true><<<ntiles, CONV_THREADS, 0, st>>>(x, w, b, y, n);
    else if (relu)
        k_conv<2, true, false><<<ntiles, CONV_THREADS, 0, st>>>(x, w, b, y, n);
    else
        k_conv<2, false, false><<<ntiles, CONV_THREADS, 0, st>>>(x, w, b, y, n);
}

void conv_launch(pm_net *e, int layer, const __nv_bfloat16 *in, void *out, bool transposed, bool relu, bool f32)
{
    const int n = e->n;
    const uint4 *w = reinterpret_cast<const uint4 *>((transposed ? e->wt : e->wf) + (size_t)layer * WSZ);
    const float *b = transposed ? nullptr : e->bias + layer * CH;
    const uint4 *x = reinterpret_cast<const uint4 *>(in);
    conv16(x, w, b, out, n, relu, f32, e->stream);
}

void net_forward(pm_net *e)
{
    const int ntiles = (e->n / TT) * (e->n / TT) * (e->n / TT);
    k_conv_in2<<<ntiles, CONV_THREADS, 0, e->stream>>>(reinterpret_cast<const uint4 *>(e->act[0]), e->wf, e->bias,
                                                       e->act[1], e->n);
    for (int l = 1; l < NL - 1; l++) conv_launch(e, l, e->act[l], e->act[l + 1], false, true, false);
    conv_launch(e, NL - 1, e->act[NL - 1], e->out, false, false, true);
}

int dw_blocks(int n)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int ntiles = (n / TT) * (n / TT) * (n / TT);
    return std::max(1, std::min(ntiles, 2 * std::max(sms, 1)));
}

void launch_conv_dw(const uint4 *x, const uint4 *g, float *dw, int n, cudaStream_t st)
{
    static std::atomic<uint64_t> done{0};
    if (first_on_device(done)) cudaFuncSetAttribute(k_conv_dw, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)DW_SMEM);
    k_conv_dw<<<dw_blocks(n), 32 * DW_WARPS, DW_SMEM, st>>>(x, g, dw, n);
}

bool valid_net_n(int n) { return n >= 8 && n <= 1024 && n % 8 == 0; }

}  // namespace

extern "C" {

int64_t pm_net_param_count(void) { return NPARAM; }

pm_status pm_net_create(int32_t n_mesh, uint64_t seed, void *stream, pm_net **out)
{
    if (!out) return PM_ERR_INVALID_ARG;
    *out = nullptr;
    if (!valid_net_n(n_mesh)) return PM_ERR_UNSUPPORTED_SIZE;
    pm_net *e = new (std::nothrow) pm_net();
    if (!e) return PM_ERR_OOM;
    e->n = n_mesh;
    e->ncell = (int64_t)n_mesh * n_mesh * n_mesh;
    e->stream = reinterpret_cast<cudaStream_t>(stream);
    const size_t nc = (size_t)e->ncell;
    struct A {
        void **p;
        size_t bytes;
    } allocs[] = {
        {(void **)&e->theta, sizeof(float) * NPARAM},  {(void **)&e->grad, sizeof(float) * NPARAM},
        {(void **)&e->m, sizeof(float) * NPARAM},      {(void **)&e->v, sizeof(float) * NPARAM},
        {(void **)&e->wf, 2 * (size_t)NL * WSZ},      {(void **)&e->wt, 2 * (size_t)NL * WSZ},
        {(void **)&e->bias, sizeof(float) * NL * CH}, {(void **)&e->act[0], 2 * CH * nc},
        {(void **)&e->act[1], 2 * CH * nc},            {(void **)&e->act[2], 2 * CH * nc},
        {(void **)&e->act[3], 2 * CH * nc},            {(void **)&e->g0, 2 * CH * nc},
        {(void **)&e->g1, 2 * CH * nc},                {(void **)&e->out, sizeof(float) * 8 * nc},
        {(void **)&e->dloss, sizeof(double)},
    };
    for (const A &a : allocs)
        if (cudaMalloc(a.p, a.bytes) != cudaSuccess) {
            cudaGetLastError();
            pm_net_destroy(e);
            return PM_ERR_OOM;
        }
    // He-normal initial weights (std sqrt(2 / (27 c_in)), last layer x 0.1), zero biases and padding,
    // from SplitMix64 + Box-Muller on the host
    std::vector<float> th(NPARAM, 0.f);
    uint64_t st = seed;
    auto next = [&]() {
        uint64_t z = (st += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    };
    auto uni = [&]() { return ((double)(next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); };
    for (int l = 0; l < NL; l++) {
        const double sd = std::sqrt(2.0 / (NOFF * CIN[l])) * (l == NL - 1 ? 0.1 : 1.0);
        for (int d = 0; d < NOFF; d++)
            for (int co = 0; co < COUT[l]; co++)
                for (int ci = 0; ci < CIN[l]; ci++) {
                    const double u1 = uni(), u2 = uni();
                    th[(size_t)l * PSZ + (d * CH + co) * CH + ci] =
                        (float)(sd * std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2));
                }
    }
    pm_status s = pm_net_set_params(e, th.data());
    if (s != PM_OK) {
        pm_net_destroy(e);
        return s;
    }
    *out = e;
    return PM_OK;
}

void pm_net_destroy(pm_net *e)
{
    if (!e) return;
    if (e->stream) cudaStreamSynchronize(e->stream);
    else cudaDeviceSynchronize();
    void *ps[] = {e->theta, e->grad, e->m, e->v, e->wf, e->wt, e->bias, e->act[0], e->act[1], e->act[2],
                  e->act[3], e->g0, e->g1, e->out, e->dloss};
    for (void *p : ps)
        if (p) cudaFree(p);
    cudaGetLastError();
    delete e;
}

const char *pm_net_last_error(const pm_net *e) { return e ? e->err.c_str() : "null network"; }

pm_status pm_net_set_params(pm_net *e, const float *params)
{
    if (!e || !params) return PM_ERR_INVALID_ARG;
    cudaError_t ce = cudaMemcpyAsync(e->theta, params, sizeof(float) * NPARAM, cudaMemcpyDefault, e->stream);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(e->grad, 0, sizeof(float) * NPARAM, e->stream);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(e->m, 0, sizeof(float) * NPARAM, e->stream);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(e->v, 0, sizeof(float) * NPARAM, e->stream);
    if (ce != cudaSuccess) return net_fail(e, PM_ERR_CUDA, "pm_net_set_params: copy failed");
    e->adam_t = 0;
    k_pack<<<grid_for(NPARAM, 256), 256, 0, e->stream>>>(e->theta, e->wf, e->wt, e->bias);
    ce = cudaStreamSynchronize(e->stream);
    if (ce == cudaSuccess) ce = cudaGetLastError();
    return ce == cudaSuccess ? PM_OK : net_fail(e, PM_ERR_CUDA, "pm_net_set_params: kernel failed");
}

pm_status pm_net_get_params(pm_net *e, float *params)
{
    if (!e || !params) return PM_ERR_INVALID_ARG;
    cudaError_t ce = cudaMemcpyAsync(params, e->theta, sizeof(float) * NPARAM, cudaMemcpyDefault, e->stream);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(e->stream);
    return ce == cudaSuccess ? PM_OK : net_fail(e, PM_ERR_CUDA, "pm_net_get_params: copy failed");
}

pm_status pm_net_buffer(pm_net *e, int32_t which, void **ptr)
{
    if (!e || !ptr) return PM_ERR_INVALID_ARG;
    switch (which) {
    case PM_NET_INPUT: *ptr = e->act[0]; break;
    case PM_NET_OUTPUT: *ptr = e->out; break;
    case PM_NET_GRAD: *ptr = e->grad; break;
    default: return PM_ERR_INVALID_ARG;
    }
    return PM_OK;
}

pm_status pm_net_forward(pm_net *e)
{
    if (!e) return PM_ERR_INVALID_ARG;
    if (g_conv_poisoned.load()) return net_fail(e, PM_ERR_STATE, "pm_net_forward: convolutions poisoned");
    net_forward(e);
    return cudaGetLastError() == cudaSuccess ? PM_OK : net_fail(e, PM_ERR_CUDA, "pm_net_forward: launch failed");
}

pm_status pm_net_backward(pm_net *e, const float *target, double *loss)
{
    if (!e || !target) return PM_ERR_INVALID_ARG;
    if (g_conv_poisoned.load()) return net_fail(e, PM_ERR_STATE, "pm_net_backward: convolutions poisoned");
    const int64_t nc = e->ncell;
    const int n = e->n;
    net_forward(e);
    cudaMemsetAsync(e->dloss, 0, sizeof(double), e->stream);
    // G = dL/d(network output) and the bias gradient of the last layer (no activation)
    k_loss<<<std::min<int64_t>(grid_for(nc, CONV_THREADS), 4096), CONV_THREADS, 0, e->stream>>>(
        e->out, target, e->g0, e->dloss, e->grad + (size_t)(NL - 1) * PSZ + WSZ, nc);
    const unsigned mblocks = (unsigned)std::min<int64_t>(grid_for(2 * nc, CONV_THREADS), 4096);
    // tensor-core meshes: the input-gradient convolution of layer l applies the ReLU derivative of layer
    // l - 1 and sums that layer's bias gradient in its epilogue; other meshes run k_mask after it
    const bool fused = conv_on_tcgen05(n);
    __nv_bfloat16 *g = e->g0, *h = e->g1;
    for (int l = NL - 1; l >= 0; l--) {
        // g holds dL/d(pre-activation of layer l), or, unfused and l < NL - 1, dL/d(output of layer l)
        if (!fused && l < NL - 1) {
            k_mask<<<mblocks, CONV_THREADS, 0, e->stream>>>(
                reinterpret_cast<const uint4 *>(g), reinterpret_cast<const uint4 *>(e->act[l + 1]),
                reinterpret_cast<uint4 *>(h), e->grad + (size_t)l * PSZ + WSZ, nc, 1);
            std::swap(g, h);
        }
        launch_conv_dw(reinterpret_cast<const uint4 *>(e->act[l]), reinterpret_cast<const uint4 *>(g),
                       e->grad + (size_t)l * PSZ, n, e->stream);
        if (l == 0) break;
        const uint4 *wt = reinterpret_cast<const uint4 *>(e->wt + (size_t)l * WSZ);
        if (fused)
            launch_conv_tc<false, false, true>(reinterpret_cast<const uint4 *>(g), wt, nullptr, h, n, e->stream,
                                               reinterpret_cast<const uint4 *>(e->act[l]),
                                               e->grad + (size_t)(l - 1) * PSZ + WSZ);
        else
            conv_launch(e, l, g, h, true, false, false);   // dL/d(output of layer l - 1)
        std::swap(g, h);
    }
    cudaError_t ce = cudaGetLastError();
    if (ce == cudaSuccess && loss) {
        ce = cudaMemcpyAsync(loss, e->dloss, sizeof(double), cudaMemcpyDeviceToHost, e->stream);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(e->stream);
    }
    return ce == cudaSuccess ? PM_OK : net_fail(e, PM_ERR_CUDA, "pm_net_backward: launch failed");
}

pm_status pm_net_adam(pm_net *e, float lr)
{
    if (!e || !(lr > 0.f)) return PM_ERR_INVALID_ARG;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    e->adam_t++;
    const float c1 = (float)(1.0 - std::pow((double)b1, (double)e->adam_t));
    const float c2 = (float)(1.0 - std::pow((double)b2, (double)e->adam_t));
    k_adam<<<grid_for(NPARAM, 256), 256, 0, e->stream>>>(e->theta, e->grad, e->m, e->v, lr, b1, b2, eps, c1, c2);
    k_pack<<<grid_for(NPARAM, 256), 256, 0, e->stream>>>(e->theta, e->wf, e->wt, e->bias);
    return cudaGetLastError() == cudaSuccess ? PM_OK : net_fail(e, PM_ERR_CUDA, "pm_net_adam: launch failed");
}

pm_status pm_net_train_step(pm_net *e, const float *target, float lr, double *loss)
{
    pm_status s = pm_net_backward(e, target, loss);
    if (s != PM_OK) return s;
    return pm_net_adam(e, lr);
}

static pm_status check_solved(pm_ctx *ctx)
{
    if (!ctx) return PM_ERR_INVALID_ARG;
    const Ctx &c = ctx->c;
    if (!c.newtonian) return PM_ERR_UNSUPPORTED_SIZE;   // the correction is trained on the Newtonian force
    if (c.stage != 2) return PM_ERR_STATE;
    return PM_OK;
}

pm_status pm_net_features(pm_net *e, pm_ctx *ctx)
{
    if (!e) return PM_ERR_INVALID_ARG;
    pm_status s = check_solved(ctx);
    if (s != PM_OK) return net_fail(e, s, "pm_net_features: needs a solved Newtonian context");
    Ctx &c = ctx->c;
    if (c.N != e->n) return net_fail(e, PM_ERR_INVALID_ARG, "pm_net_features: mesh size differs");
    const double a = c.a_n[c.step];
    const double inv_kappa = a / (c.four_pi_g * c.cfg.omega_m);
    const double s0 = e->s_delta * inv_kappa, s1 = e->s_phi * (double)c.N * c.N * inv_kappa;
    const unsigned nb = grid_for(e->ncell, 256);
    if (c.mixed)
        k_features<float><<<nb, 256, 0, e->stream>>>(static_cast<const float *>(c.src),
                                                     static_cast<const float *>(c.phi[c.iphi_new]), s0, s1,
                                                     e->act[0], e->ncell);
    else
        k_features<double><<<nb, 256, 0, e->stream>>>(static_cast<const double *>(c.src),
                                                      static_cast<const double *>(c.phi[c.iphi_new]), s0, s1,
                                                      e->act[0], e->ncell);
    return cudaGetLastError() == cudaSuccess ? PM_OK : net_fail(e, PM_ERR_CUDA, "pm_net_features: launch failed");
}

pm_status pm_net_target(pm_net *e, pm_ctx *coarse, pm_ctx *fine, float *target)
{
    if (!e || !target) return PM_ERR_INVALID_ARG;
    pm_status s = check_solved(coarse);
    if (s == PM_OK) s = check_solved(fine);
    if (s != PM_OK) return net_fail(e, s, "pm_net_target: needs two solved Newtonian contexts");
    Ctx &c = coarse->c, &f = fine->c;
    const double a = c.a_n[c.step], af = f.a_n[f.step];
    if (c.N != e->n || f.N != 2 * c.N || c.mixed != f.mixed || c.np != f.np || c.cfg.box_mpch != f.cfg.box_mpch ||
        c.cfg.omega_m != f.cfg.omega_m || !(std::fabs(a - af) <= 1e-12 * a))
        return net_fail(e, PM_ERR_INVALID_ARG, "pm_net_target: contexts do not pair (fine mesh = 2 x coarse, same a)");
    const double scale = e->s_target * (double)c.N * a / (c.four_pi_g * c.cfg.omega_m);
    const unsigned nb = grid_for(e->ncell, 128);
    if (c.mixed)
        k_target<float><<<nb, 128, 0, e->stream>>>(static_cast<const float *>(c.phi[c.iphi_new]),
                                                   static_cast<const float *>(f.phi[f.iphi_new]), c.N, scale, target);
    else
        k_target<double><<<nb, 128, 0, e->stream>>>(static_cast<const double *>(c.phi[c.iphi_new]),
                                                    static_cast<const double *>(f.phi[f.iphi_new]), c.N, scale, target);
    return cudaGetLastError() == cudaSuccess ? PM_OK : net_fail(e, PM_ERR_CUDA, "pm_net_target: launch failed");
}

pm_status pm_net_apply(pm_net *e, pm_ctx *ctx)
{
    pm_status s = pm_net_features(e, ctx);
    if (s != PM_OK) return s;
    net_forward(e);
    if (cudaGetLastError() != cudaSuccess) return net_fail(e, PM_ERR_CUDA, "pm_net_apply: launch failed");
    // the kick reads the network output in force units: c = (kappa / N) y / s_target, kappa = 4piG Omega_m / a
    Ctx &c = ctx->c;
    const double a = c.a_n[c.step];
    c.corr = e->out;
    c.corr_scale = (float)(c.four_pi_g * c.cfg.omega_m / a / (double)c.N / e->s_target);
    return PM_OK;
}

pm_status pm_net_set_scales(pm_net *e, double s_delta, double s_phi, double s_target)
{
    if (!e || !(s_delta > 0) || !(s_phi >= 0) || !(s_target > 0) || !std::isfinite(s_delta) || !std::isfinite(s_phi) ||
        !std::isfinite(s_target))
        return PM_ERR_INVALID_ARG;
    e->s_delta = s_delta;
    e->s_phi = s_phi;
    e->s_target = s_target;
    return PM_OK;
}

pm_status pm_set_correction(pm_ctx *ctx, const float *corr)
{
    if (!ctx) return PM_ERR_INVALID_ARG;
    ctx->c.corr = const_cast<float *>(corr);
    ctx->c.corr_scale = 1.f;
    return PM_OK;
}

pm_status pm_conv3d_forward(int32_t n, const void *x, const void *w, const float *bias, int32_t c_out, int32_t relu,
                            void *y, void *stream)
{
    if (g_conv_poisoned.load()) return PM_ERR_STATE;
    if (!valid_net_n(n)) return PM_ERR_UNSUPPORTED_SIZE;
    if (!x || !w || !y || (c_out != 8 && c_out != 16) || (c_out == 8 && relu)) return PM_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    conv16(static_cast<const uint4 *>(x), static_cast<const uint4 *>(w), bias, y, n, relu != 0, c_out == 8, st);
    return cudaGetLastError() == cudaSuccess ? PM_OK : PM_ERR_CUDA;
}

pm_status pm_conv3d_check(void *stream)
{
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = st ? cudaStreamSynchronize(st) : cudaDeviceSynchronize();
    unsigned int t = 0, u = 0;
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&t, g_conv_tc_timeouts, sizeof(t));
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&u, g_conv_tc_unsafe, sizeof(u));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return PM_ERR_CUDA;
    }
    if (u != 0) g_conv_poisoned.store(true);   // TMEM was freed with MMAs possibly in flight
    if (t == 0) return g_conv_poisoned.load() ? PM_ERR_STATE : PM_OK;
    const unsigned int zero = 0;
    cudaMemcpyToSymbol(g_conv_tc_timeouts, &zero, sizeof(zero));
    return PM_ERR_TIMEOUT;
}

pm_status pm_conv3d_backward_weight(int32_t n, const void *x, const void *g, float *dw, void *stream)
{
    if (!valid_net_n(n)) return PM_ERR_UNSUPPORTED_SIZE;
    if (!x || !g || !dw) return PM_ERR_INVALID_ARG;
    launch_conv_dw(static_cast<const uint4 *>(x), static_cast<const uint4 *>(g), dw, n,
                   reinterpret_cast<cudaStream_t>(stream));
    return cudaGetLastError() == cudaSuccess ? PM_OK : PM_ERR_CUDA;
}

}  // extern "C"
