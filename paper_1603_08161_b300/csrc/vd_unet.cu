// Learned warm start of the lattice solve: a 3-level 3D U-Net (16 / 32 / 64 channels)
// over the lattice grid, BF16 weights and activations with FP32 accumulation on the
// tensor cores, with its own forward, backward and Adam kernels.
//
// Input (6 channels per node): the previous frame's displacement u / h and the current
// data-term gradient (scaled).  Output (3 channels): the predicted change of u in
// lattice units.  Convolutions are 3x3x3, "same", with bias; ReLU after every
// convolution except the head.  Down-sampling is 2x2x2 average pooling, up-sampling is
// nearest-neighbour x2; skip connections are channel concatenations:
//   e1 = b1(a1(x))          96^3, 16      cat1 = [up(d2), e1]   96^3, 48
//   e2 = b2(a2(pool(e1)))   48^3, 32      cat2 = [up(e3), e2]   48^3, 96
//   e3 = b3(a3(pool(e2)))   24^3, 64      d2 = d2c(c2(cat2))    48^3, 32
//   out = head(d1c(c1(cat1)))  96^3, 3
// Activations are stored channels-last with a one-voxel zero halo and 16 voxels of
// slack after each row, so a 16-voxel tile at any tap offset stays inside its buffer
// (a plain strided 16x16 matrix for the WMMA kernels: wgrad and rows wider than 128).
// The convolutions run on tcgen05 (k_conv3d_tc).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <mma.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <new>
#include <random>
#include <string>
#include <vector>

#include "vd.h"

using namespace nvcuda;
typedef __nv_bfloat16 bf16;

namespace {

constexpr int kLayers = 11;
// Cin, Cout of the layers in parameter order (ReLU after all but the head)
constexpr int kCin[kLayers] = {6, 16, 16, 32, 32, 64, 96, 32, 48, 16, 16};
constexpr int kCout[kLayers] = {16, 16, 32, 32, 64, 64, 32, 32, 16, 16, 3};
enum { A1, B1, A2, B2, A3, B3, C2, D2, C1, D1, HEAD };

int pad16(int c) { return (c + 15) / 16 * 16; }

// A channels-last view: p points at channel c0 of voxel (-1, -1, -1); C is the buffer's
// channel stride, nc the view's channel count.
struct View {
    bf16 *p;
    int D, H, W, C, Wp, nc;
    int c0;  // channel offset of the view in its buffer (p = buffer + c0)
};

__host__ __device__ inline size_t vox(const View &t, int z, int y, int x) {
    return ((size_t)(z + 1) * (t.H + 2) + (y + 1)) * t.Wp + (x + 1);
}

// ------------------------------------------------------------------ kernels

// out[..., 0:cout_real) = act(conv3x3x3(in) + bias): one warp per 16-voxel row tile and
// all NF x 16 output channels.  in.nc and the weights' Cin are multiples of 16.  With
// outf set, the result goes to outf[cout_real * node + co] in FP32 instead (the head).
template <int NF>
__global__ void __launch_bounds__(128) k_conv3d(View in, const bf16 *__restrict__ Wt, const float *__restrict__ bias,
                                                View out, int cout_real, int relu, float *__restrict__ outf) {
    __shared__ __align__(32) float tile[4][16 * 16];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int xt_n = (out.W + 15) / 16;
    const long t = (long)blockIdx.x * 4 + warp;
    if (t >= (long)out.D * out.H * xt_n) return;
    const int xt = (int)(t % xt_n), y = (int)((t / xt_n) % out.H), z = (int)(t / ((long)xt_n * out.H));
    const int x0 = xt * 16;
    const int CoutP = NF * 16;
    wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc[NF];
#pragma unroll
    for (int j = 0; j < NF; j++) wmma::fill_fragment(acc[j], 0.f);
    wmma::fragment<wmma::matrix_a, 16, 16, 16, bf16, wmma::row_major> a;
    wmma::fragment<wmma::matrix_b, 16, 16, 16, bf16, wmma::row_major> b;
    for (int tap = 0; tap < 27; tap++) {
        const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
        const bf16 *A = in.p + vox(in, z + dz, y + dy, x0 + dx) * in.C;
        for (int k0 = 0; k0 < in.nc; k0 += 16) {
            wmma::load_matrix_sync(a, A + k0, in.C);
#pragma unroll
            for (int j = 0; j < NF; j++) {
                wmma::load_matrix_sync(b, Wt + ((size_t)tap * in.nc + k0) * CoutP + 16 * j, CoutP);
                wmma::mma_sync(acc[j], a, b, acc[j]);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < NF; j++) {
        wmma::store_matrix_sync(tile[warp], acc[j], 16, wmma::mem_row_major);
        __syncwarp();
        for (int e = lane; e < 256; e += 32) {
            const int r = e >> 4, co = 16 * j + (e & 15);
            const int x = x0 + r;
            if (x < out.W && co < cout_real) {
                float v = tile[warp][e] + (bias ? bias[co] : 0.f);
                if (relu) v = fmaxf(v, 0.f);
                if (outf) outf[((size_t)(z * out.H + y) * out.W + x) * cout_real + co] = v;
                else out.p[vox(out, z, y, x) * out.C + co] = __float2bfloat16_rn(v);
            }
        }
        __syncwarp();
    }
}

// ------------------------------------------------------------------ tcgen05 convolution
//
// The convolution as an implicit GEMM on the 5th-generation tensor cores: a CTA of 4
// warps owns R = tc_rows(W, H) output rows (z, y0 ..), whole in x.  Output position m = r RW + j
// (row r, column j < RW = W + 2; columns j >= W are computed and dropped) needs, for tap
// (dz, dy, dx), the staged input voxel m + off(tap), off = ((dz+1)(R+2) + 1 + dy) RW + 1 + dx,
// so every tap's A operand (128 positions x 16 channels, K-major) is the staged slab
// read from a shifted start address.  The slab holds the 3 x (R + 2) input rows
// (x from -1 to W, zero outside the volume) of one 16-channel slice as two channel-half
// planes of 16 B per voxel, staged by two TMA box loads: core matrices of 8 voxels x 8
// channels are 128 contiguous bytes (SBO = 128, LBO = the plane stride).  B (N output
// channels x 16 input channels of one tap, K-major) comes pre-packed in the same core
// layout (one bulk copy).  Lane blk of warp 0 issues the 27 taps' MMAs of block blk
// (M = 128, N = 16 NF, K = 16, BF16 in, FP32 accumulators in TMEM, nblk x N columns) per
// input slice and commits them to an mbarrier (a lane issues small MMAs at a limited
// rate, so the blocks' lanes issue side by side); the warps then read their 32 TMEM
// lanes (tcgen05.ld) for the epilogue.
constexpr int kTcMaxW = 128;  // wider rows take the generic WMMA kernel
__device__ __forceinline__ void st8(bf16 *p, const float f[8]);

__host__ __device__ inline int tc_rw(int W) { return W + 2; }
// Output rows per CTA: the count (2..8, at most 4 blocks of 128 positions) that wastes
// the fewest MMA positions on the dropped columns, the unused tail of the last block and
// the rows past H of the last row group (at 96^3 five rows: 490 of 512 positions; two
// rows used 196 of 256).
__host__ __device__ inline int tc_rows(int W, int H) {
    const int rw = tc_rw(W);
    int best = 2;
    long best_cost = -1;
    for (int r = 2; r <= 8; r++) {
        const int nblk = (r * rw + 127) / 128;
        if (nblk > 4) break;
        const long cost = (long)((H + r - 1) / r) * nblk;  // blocks per plane
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best = r;
        }
    }
    return best;
}
__host__ __device__ inline int tc_nblk(int W, int H) { return (tc_rows(W, H) * tc_rw(W) + 127) / 128; }
// staged voxels per plane (the shifted A windows of the last block stay inside)
__host__ __device__ inline int tc_nvp(int W, int H) {
    return (tc_nblk(W, H) * 128 + (2 * (tc_rows(W, H) + 2) + 2) * tc_rw(W) + 2 + 7) / 8 * 8;
}
__host__ __device__ inline int tc_smem_bytes(int W, int H, int NF) {
    return 2 * tc_nvp(W, H) * 16 + 27 * 16 * NF * 32 + 64;
}
__host__ inline int tc_tmem_cols(int W, int H, int NF) {
    int c = 32;
    while (c < tc_nblk(W, H) * 16 * NF) c <<= 1;
    return c;
}

__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    // shared-memory matrix descriptor, no swizzle: start >> 4, LBO >> 4, SBO >> 4, 0b001
    return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

__device__ __forceinline__ bool mbar_wait(uint32_t mb, uint32_t parity) {
    const long long t0 = clock64();
    while (true) {
        uint32_t done;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done)
                     : "r"(mb), "r"(parity)
                     : "memory");
        if (done) return true;
        if (clock64() - t0 > 2000000000LL) return false;
    }
}

template <int NF>
__global__ void __launch_bounds__(128) k_conv3d_tc(const __grid_constant__ CUtensorMap tmap, View in,
                                                   const bf16 *__restrict__ Wtc, const float *__restrict__ bias,
                                                   View out, int cout_real, int relu, float *__restrict__ outf,
                                                   int tmem_cols, int *__restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    __shared__ __align__(8) uint64_t mbar, mbar_ld;
    __shared__ uint32_t tmem_base;
    constexpr int N = 16 * NF;
    const int W = out.W, RW = tc_rw(W), R = tc_rows(W, out.H), nblk = tc_nblk(W, out.H), NVP = tc_nvp(W, out.H);
    bf16 *planes = reinterpret_cast<bf16 *>(smraw);                     // [2][NVP][8]
    bf16 *wsl = reinterpret_cast<bf16 *>(smraw + 2 * NVP * 16);         // [27][N/8][2][8][8]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nyb = (out.H + R - 1) / R;
    const int z = blockIdx.x / nyb, y0 = (blockIdx.x - z * nyb) * R;
    const uint32_t mb = (uint32_t)__cvta_generic_to_shared(&mbar), mbl = (uint32_t)__cvta_generic_to_shared(&mbar_ld);
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mb), "r"(nblk));  // one commit per block's lane
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mbl));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         (uint32_t)__cvta_generic_to_shared(&tmem_base)),
                     "r"(tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    const int nz = 3 * (R + 2) * RW;  // staged voxels holding real rows
    const int kchunks = in.nc / 16;
    // the tail past the real rows is only ever read by dropped positions: zero it once
    for (int i = tid; i < 2 * (NVP - nz); i += 128) {
        const int h = i / (NVP - nz), v = nz + i - h * (NVP - nz);
        *reinterpret_cast<uint4 *>(planes + ((size_t)h * NVP + v) * 8) = make_uint4(0u, 0u, 0u, 0u);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the tail, for the tensor core
    bool ok = true;
    for (int kc = 0; kc < kchunks && ok; kc++) {
        const int k0 = 16 * kc;
        // stage the slice with the tensor memory accelerator: per channel half one box of
        // 8 channels x RW voxels x (R + 2) rows x 3 planes (buffer coordinates: x
        // from the halo column, rows from y0 - 1, planes from z - 1; rows and planes past
        // the buffer read as zero), plus the slice's weights by one bulk copy
        if (tid == 0) {
            const uint32_t wbytes = 27u * N * 32u;
            const uint32_t bytes = 2u * (uint32_t)nz * 16u + wbytes;
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbl), "r"(bytes) : "memory");
#pragma unroll
            for (int h = 0; h < 2; h++)
                asm volatile(
                    "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, "
                    "%4, %5}], [%6];" ::"r"((uint32_t)__cvta_generic_to_shared(planes + (size_t)h * NVP * 8)),
                    "l"(&tmap), "r"(in.c0 + k0 + 8 * h), "r"(0), "r"(y0), "r"(z), "r"(mbl)
                    : "memory");
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                             (uint32_t)__cvta_generic_to_shared(wsl)),
                         "l"(Wtc + (size_t)kc * 27 * N * 16), "r"(wbytes), "r"(mbl)
                         : "memory");
        }
        const bool staged = __syncthreads_and(mbar_wait(mbl, (uint32_t)(kc & 1)));
        if (!staged) {
            if (tid == 0) atomicExch(err, 1);
            ok = false;
            break;
        }
        if (tid < nblk) {  // lane blk: block blk's MMAs
            const int blk = tid;
            const uint32_t a0 = (uint32_t)__cvta_generic_to_shared(planes), b0 = (uint32_t)__cvta_generic_to_shared(wsl);
            // D F32, A and B BF16, both K-major, N >> 3 at bit 17, M >> 4 at bit 24
            const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((128u >> 4) << 24);
            // a shift of the start address by 16 d bytes adds d to a descriptor (its start
            // field holds address / 16; shared addresses stay below 2^18)
            const uint64_t da0 = tc_desc(a0 + (uint32_t)(blk * 128) * 16u, (uint32_t)NVP * 16u, 128);
            const uint64_t db0 = tc_desc(b0, 128, 256);
            for (int tap = 0; tap < 27; tap++) {
                const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
                const int off = ((dz + 1) * (R + 2) + 1 + dy) * RW + 1 + dx;
                const uint32_t acc = (kc > 0 || tap > 0) ? 1u : 0u;
                asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                             "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                                 tmem + (uint32_t)(blk * N)),
                             "l"(da0 + (uint64_t)off), "l"(db0 + (uint64_t)(tap * N * 2)), "r"(idesc), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb)
                         : "memory");
        }
        // the MMAs have read the slice (and written TMEM) before it is staged again; the
        // verdict is the same for every thread (a barrier-wide and)
        ok = __syncthreads_and(mbar_wait(mb, (uint32_t)(kc & 1)));
        if (!ok && tid == 0) atomicExch(err, 1);
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok) {
        for (int blk = 0; blk < nblk; blk++) {
            const int m = blk * 128 + warp * 32 + lane;
            const int r = m / RW, j = m - r * RW, y = y0 + r;
            const bool live = r < R && y < out.H && j < W;
#pragma unroll
            for (int h = 0; h < NF; h++) {
                uint32_t v[16];
                const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(blk * N + 16 * h);
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                    "[%16];\n"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                      "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                      "=r"(v[15])
                    : "r"(ta));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (!live) continue;
                float f[16];
#pragma unroll
                for (int e = 0; e < 16; e++) {
                    const int co = 16 * h + e;
                    float a = __uint_as_float(v[e]) + ((bias && co < cout_real) ? bias[co] : 0.f);
                    f[e] = relu ? fmaxf(a, 0.f) : a;
                }
                if (outf) {
#pragma unroll
                    for (int e = 0; e < 16; e++)
                        if (16 * h + e < cout_real) outf[((size_t)(z * out.H + y) * W + j) * cout_real + 16 * h + e] = f[e];
                } else if (16 * h + 16 <= cout_real) {
                    bf16 *dst = out.p + vox(out, z, y, j) * out.C + 16 * h;
                    st8(dst, f);
                    st8(dst + 8, f + 8);
                } else {
                    for (int e = 0; e < 16 && 16 * h + e < cout_real; e++)
                        out.p[vox(out, z, y, j) * out.C + 16 * h + e] = __float2bfloat16_rn(f[e]);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
}

// The same convolution as a persistent, pipelined kernel, for layers whose packed
// weights (every input slice) fit in shared memory beside at least two slab buffers:
// one CTA per SM walks the (plane, row group) items in grid stride.  Warp 4 (one lane)
// stages the weights once and then, slice after slice, the slab of the next (item, input
// slice) by TMA into the next of `nstage` (2-4) buffers, as soon as the MMAs that read
// it last are done; warp 5 (one lane) issues each slice's 27 x nblk MMAs into one of two
// TMEM accumulators (one per item parity); warps 0-3 read the finished accumulator of an
// item (tcgen05.ld, their 32 lanes each) for the epilogue while the next item's MMAs
// run.  mbarriers: full[b] (slab b staged), empty[b] (the MMAs that read it are done),
// tfull[a] (accumulator a complete), tempty[a] (its epilogue done: 128 arrivals), the
// weights, and a drain for the error path.  Every wait is bounded; a wait that gives up
// sets *err and its role stops, and the others then give up too.
constexpr int kTcpMaxStages = 4;
__host__ __device__ inline int tcp_smem_bytes(int W, int H, int NF, int kchunks, int nstage) {
    return nstage * 2 * tc_nvp(W, H) * 16 + kchunks * 27 * 16 * NF * 32;
}
constexpr int kTcpSmemMax = 225 * 1024;
// the most slab buffers (2..4) that fit, 0 if two do not
__host__ inline int tcp_stages(int W, int H, int NF, int kchunks) {
    for (int ns = kTcpMaxStages; ns >= 2; ns--)
        if (tcp_smem_bytes(W, H, NF, kchunks, ns) <= kTcpSmemMax) return ns;
    return 0;
}
// Partial accumulators per item: tap t goes to partial t % nacc and is issued by its own
// lane (one MMA-issuing thread sustains only about one small MMA per 100 ns); the
// epilogue adds the partials.  The most (<= 4) for which two items' accumulators fit the
// 512 TMEM columns.
constexpr int kTcpMaxAcc = 4;
__host__ inline int tcp_nacc(int W, int H, int NF) {
    int n = kTcpMaxAcc;
    while (n > 1 && 2 * n * tc_nblk(W, H) * 16 * NF > 512) n--;
    return n;
}
// 0 when even one partial per item does not fit (the per-row-group kernel then runs)
__host__ inline int tcp_tmem_cols(int W, int H, int NF) {
    const int need = 2 * tcp_nacc(W, H, NF) * tc_nblk(W, H) * 16 * NF;
    if (need > 512) return 0;
    int c = 32;
    while (c < need) c <<= 1;
    return c;
}

__device__ __forceinline__ void mbar_arrive(uint32_t mb) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mb) : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t mb) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb) : "memory");
}

template <int NF>
__global__ void __launch_bounds__(192, 1) k_conv3d_tcp(const __grid_constant__ CUtensorMap tmap, View in,
                                                       const bf16 *__restrict__ Wtc, const float *__restrict__ bias,
                                                       View out, int cout_real, int relu, float *__restrict__ outf,
                                                       int tmem_cols, int nstage, int nacc, int *__restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smraw[];
    __shared__ __align__(8) uint64_t bar[14];
    __shared__ uint32_t tmem_base;
    constexpr int N = 16 * NF;
    enum { FULL = 0, EMPTY = 4, TFULL = 8, TEMPTY = 10, WBAR = 12, DRAIN = 13 };
    const int W = out.W, RW = tc_rw(W), R = tc_rows(W, out.H), nblk = tc_nblk(W, out.H), NVP = tc_nvp(W, out.H);
    const int kchunks = in.nc / 16;
    const int nyb = (out.H + R - 1) / R, n_items = out.D * nyb;
    bf16 *slab = reinterpret_cast<bf16 *>(smraw);                                // [nstage][2 halves][NVP][8]
    bf16 *wsl = reinterpret_cast<bf16 *>(smraw + 2 * (size_t)nstage * NVP * 16);  // [kchunks][27][N/8][2][8][8]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t bar0 = (uint32_t)__cvta_generic_to_shared(&bar[0]);
    auto ba = [&](int i) { return bar0 + 8u * (uint32_t)i; };
    if (tid == 0) {
        for (int i = 0; i < 14; i++)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(ba(i)),
                         "r"((i == TEMPTY || i == TEMPTY + 1) ? 128 : (i >= EMPTY && i < TEMPTY) || i == DRAIN ? nblk * nacc : 1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         (uint32_t)__cvta_generic_to_shared(&tmem_base)),
                     "r"(tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    const int nz = 3 * (R + 2) * RW;  // staged voxels holding real rows
    // the tails past the real rows are only ever read by dropped positions: zero them once
    for (int i = tid; i < 2 * nstage * (NVP - nz); i += blockDim.x) {
        const int hp = i / (NVP - nz), v = nz + i - hp * (NVP - nz);  // hp: buffer x half
        *reinterpret_cast<uint4 *>(slab + ((size_t)hp * NVP + v) * 8) = make_uint4(0u, 0u, 0u, 0u);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // the tails, for the tensor core
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_base;
    if (warp == 4) {
        // ---- producer: the weights once, then the slabs
        if (lane == 0) {
            bool ok = true;
            const uint32_t wbytes = (uint32_t)kchunks * 27u * N * 32u, sbytes = 2u * (uint32_t)nz * 16u;
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(ba(WBAR)), "r"(wbytes) : "memory");
            asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                             (uint32_t)__cvta_generic_to_shared(wsl)),
                         "l"(Wtc), "r"(wbytes), "r"(ba(WBAR))
                         : "memory");
            int b = 0, u = 0, lb = -1, lu = 0;  // buffer and its use count; the last stage issued
            for (int item = blockIdx.x; item < n_items && ok; item += gridDim.x) {
                const int z = item / nyb, y0 = (item - z * nyb) * R;
                for (int kc = 0; kc < kchunks; kc++) {
                    if (u >= 1 && !mbar_wait(ba(EMPTY + b), (uint32_t)((u - 1) & 1))) {
                        ok = false;
                        break;
                    }
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(ba(FULL + b)), "r"(sbytes)
                                 : "memory");
#pragma unroll
                    for (int h = 0; h < 2; h++)
                        asm volatile(
                            "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, "
                            "{%2, %3, %4, %5}], [%6];" ::"r"(
                                (uint32_t)__cvta_generic_to_shared(slab + ((size_t)(2 * b + h) * NVP) * 8)),
                            "l"(&tmap), "r"(in.c0 + 16 * kc + 8 * h), "r"(0), "r"(y0), "r"(z), "r"(ba(FULL + b))
                            : "memory");
                    lb = b;
                    lu = u;
                    if (++b == nstage) {
                        b = 0;
                        u++;
                    }
                }
            }
            if (!ok) {
                atomicExch(err, 1);
                // the copies in flight land before the CTA leaves (bounded)
                if (lb >= 0) mbar_wait(ba(FULL + lb), (uint32_t)(lu & 1));
            }
        }
    } else if (warp == 5) {
        // ---- MMA issue: every slice of an item into accumulator (item parity); lane
        // pa nblk + blk issues the MMAs of block blk and of the taps of partial pa (one
        // instruction issues the MMAs of all these lanes)
        const int nis = nblk * nacc;
        if (lane < nis) {
            const int my_pa = lane / nblk, my_blk = lane - my_pa * nblk;
            bool ok = mbar_wait(ba(WBAR), 0u);
            const uint32_t a_base = (uint32_t)__cvta_generic_to_shared(slab), b0 = (uint32_t)__cvta_generic_to_shared(wsl);
            // D F32, A and B BF16, both K-major, N >> 3 at bit 17, M >> 4 at bit 24
            const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((128u >> 4) << 24);
            int b = 0, u = 0, i = 0;
            for (int item = blockIdx.x; item < n_items && ok; item += gridDim.x, i++) {
                const int a = i & 1;
                if (i >= 2 && !mbar_wait(ba(TEMPTY + a), (uint32_t)(((i >> 1) + 1) & 1))) {
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                for (int kc = 0; kc < kchunks; kc++) {
                    if (!mbar_wait(ba(FULL + b), (uint32_t)(u & 1))) {
                        ok = false;
                        break;
                    }
                    // descriptors of the slice's first tap; a shift of the start address by
                    // 16 d bytes adds d to a descriptor (its start field holds address / 16,
                    // and every shared address here stays below 2^18)
                    const uint64_t da0 = tc_desc(a_base + (uint32_t)b * 2u * (uint32_t)NVP * 16u, (uint32_t)NVP * 16u, 128);
                    const uint64_t db0 = tc_desc(b0 + (uint32_t)(kc * 27) * N * 32u, 128, 256);
                    for (int j = 0; j * nacc < 27; j++) {
                        const int tap = j * nacc + my_pa;
                        if (tap < 27) {
                            const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
                            const int off = ((dz + 1) * (R + 2) + 1 + dy) * RW + 1 + dx;
                            const uint64_t db = db0 + (uint64_t)(tap * N * 2);
                            const uint64_t da = da0 + (uint64_t)(my_blk * 128 + off);
                            const uint32_t acc = (kc > 0 || j > 0) ? 1u : 0u;
                            asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                                         "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
                                             tmem + (uint32_t)((((a * nacc + my_pa) * nblk) + my_blk) * N)),
                                         "l"(da), "l"(db), "r"(idesc), "r"(acc));
                        }
                    }
                    mma_commit(ba(EMPTY + b));  // the slab is free once these MMAs are done
                    if (++b == nstage) {
                        b = 0;
                        u++;
                    }
                }
                if (!ok) break;
                mma_commit(ba(TFULL + a));  // the accumulator is complete
            }
            if (!ok) {
                atomicExch(err, 1);
                mma_commit(ba(DRAIN));  // every MMA issued is done before TMEM is released
                mbar_wait(ba(DRAIN), 0u);
            }
        }
    } else {
        // ---- epilogue (warps 0-3: TMEM lanes 32 warp .. + 31)
        int i = 0;
        for (int item = blockIdx.x; item < n_items; item += gridDim.x, i++) {
            const int a = i & 1;
            const bool got = __all_sync(0xffffffffu, mbar_wait(ba(TFULL + a), (uint32_t)((i >> 1) & 1)));
            if (!got) {
                if (lane == 0) atomicExch(err, 1);
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int z = item / nyb, y0 = (item - z * nyb) * R;
            for (int blk = 0; blk < nblk; blk++) {
                const int m = blk * 128 + warp * 32 + lane;
                const int r = m / RW, j = m - r * RW, y = y0 + r;
                const bool live = r < R && y < out.H && j < W;
#pragma unroll
                for (int h = 0; h < NF; h++) {
                    float f[16];
#pragma unroll
                    for (int e = 0; e < 16; e++) f[e] = 0.f;
                    for (int pa = 0; pa < nacc; pa++) {  // the sum of the partials
                        uint32_t v[16];
                        const uint32_t ta = tmem + ((uint32_t)(warp * 32) << 16) +
                                            (uint32_t)((((a * nacc + pa) * nblk) + blk) * N + 16 * h);
                        asm volatile(
                            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
                            "%15}, [%16];\n"
                            "tcgen05.wait::ld.sync.aligned;\n"
                            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                              "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                              "=r"(v[14]), "=r"(v[15])
                            : "r"(ta)
                            : "memory");
#pragma unroll
                        for (int e = 0; e < 16; e++) f[e] += __uint_as_float(v[e]);
                    }
                    if (!live) continue;
#pragma unroll
                    for (int e = 0; e < 16; e++) {
                        const int co = 16 * h + e;
                        const float x = f[e] + ((bias && co < cout_real) ? bias[co] : 0.f);
                        f[e] = relu ? fmaxf(x, 0.f) : x;
                    }
                    if (outf) {
#pragma unroll
                        for (int e = 0; e < 16; e++)
                            if (16 * h + e < cout_real)
                                outf[((size_t)(z * out.H + y) * W + j) * cout_real + 16 * h + e] = f[e];
                    } else if (16 * h + 16 <= cout_real) {
                        bf16 *dst = out.p + vox(out, z, y, j) * out.C + 16 * h;
                        st8(dst, f);
                        st8(dst + 8, f + 8);
                    } else {
                        for (int e = 0; e < 16 && 16 * h + e < cout_real; e++)
                            out.p[vox(out, z, y, j) * out.C + 16 * h + e] = __float2bfloat16_rn(f[e]);
                    }
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(ba(TEMPTY + a));
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
}

// dW[tap][ci][co] += sum_v X[v + off(tap)][ci] dY[v][co].  A block (16-channel ci group,
// 16-channel co group, slice) walks row bands (z, y, up to 128 voxels of x) in grid
// stride; per band it stages, with 16-byte loads, the 9 rows (z + dz, y + dy) of X it
// needs (x from one before the band to one past it, 16 ci) and the band of dY (16 co)
// in shared memory, and forms every tap's 16 x 16 x 16 products from there: warp w
// accumulates taps w, w + 8, w + 16, w + 24, each loaded operand serving up to 27 taps.
// At the end the 27 accumulators go to dW by FP32 atomics.  (The tensor-core MMAs of
// the convolutions do not fit here: with 16-96 channels a tap's GEMM is at most 96 wide,
// and one operand descriptor cannot span several taps' different shifts.)
constexpr int kWgTiles = 8;  // 16-voxel tiles per staged band
__global__ void __launch_bounds__(256) k_wgrad(View X, View dY, float *__restrict__ dW, int CoutP, int slices) {
    __shared__ __align__(32) bf16 xs[9][kWgTiles * 16 + 2][16];
    __shared__ __align__(32) bf16 ys[kWgTiles * 16][16];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nco = dY.nc / 16;
    int b = blockIdx.x;
    const int slice = b % slices;
    b /= slices;
    const int cof = b % nco, cif = b / nco;
    const int xt_n = (dY.W + 15) / 16, nxc = (xt_n + kWgTiles - 1) / kWgTiles;
    const long nbands = (long)dY.D * dY.H * nxc;
    wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc[4];
#pragma unroll
    for (int k = 0; k < 4; k++) wmma::fill_fragment(acc[k], 0.f);
    for (long band = slice; band < nbands; band += slices) {
        const int xc = (int)(band % nxc);
        const long zy = band / nxc;
        const int y = (int)(zy % dY.H), z = (int)(zy / dY.H);
        const int t0 = xc * kWgTiles, nt = min(kWgTiles, xt_n - t0), nv = 16 * nt, x0 = 16 * t0;
        __syncthreads();  // the last band's operands are read
        // X: row r = 3 (dz + 1) + dy + 1, voxel x0 - 1 + v (the zero halo and the row slack
        // cover the ends), two 16-byte halves of the 16 ci
        for (int i = threadIdx.x; i < 9 * (nv + 2) * 2; i += blockDim.x) {
            const int h = i & 1, rv = i >> 1, r = rv / (nv + 2), v = rv - r * (nv + 2);
            const int dz = r / 3 - 1, dy = r - 3 * (r / 3) - 1;
            *reinterpret_cast<uint4 *>(&xs[r][v][8 * h]) =
                *reinterpret_cast<const uint4 *>(X.p + vox(X, z + dz, y + dy, x0 - 1 + v) * X.C + 16 * cif + 8 * h);
        }
        for (int i = threadIdx.x; i < nv * 2; i += blockDim.x) {
            const int h = i & 1, v = i >> 1;
            *reinterpret_cast<uint4 *>(&ys[v][8 * h]) =
                *reinterpret_cast<const uint4 *>(dY.p + vox(dY, z, y, x0 + v) * dY.C + 16 * cof + 8 * h);
        }
        __syncthreads();
        for (int t = 0; t < nt; t++) {
            wmma::fragment<wmma::matrix_b, 16, 16, 16, bf16, wmma::row_major> bm;
            wmma::load_matrix_sync(bm, &ys[16 * t][0], 16);
#pragma unroll
            for (int k = 0; k < 4; k++) {
                const int tap = warp + 8 * k;
                if (tap < 27) {
                    const int r = tap / 3, dx = tap % 3 - 1;  // r = 3 (dz + 1) + dy + 1
                    wmma::fragment<wmma::matrix_a, 16, 16, 16, bf16, wmma::col_major> a;
                    wmma::load_matrix_sync(a, &xs[r][16 * t + 1 + dx][0], 16);
                    wmma::mma_sync(acc[k], a, bm, acc[k]);
                }
            }
        }
    }
    __syncthreads();
    float *tl = reinterpret_cast<float *>(&xs[0][0][0]) + 256 * warp;  // the staging area is free now
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const int tap = warp + 8 * k;
        if (tap >= 27) break;
        wmma::store_matrix_sync(tl, acc[k], 16, wmma::mem_row_major);
        __syncwarp();
        for (int e = lane; e < 256; e += 32) {
            const int ci = 16 * cif + (e >> 4), co = 16 * cof + (e & 15);
            const float v = tl[e];
            if (v != 0.f) atomicAdd(&dW[((size_t)tap * X.nc + ci) * CoutP + co], v);
        }
        __syncwarp();
    }
}

// Element-wise passes walk (voxel, 8-channel chunk) items with 16-byte loads and
// stores; views' channel offsets and counts are multiples of 8 (16-byte aligned chunks).
__device__ __forceinline__ void ld8(const bf16 *p, float f[8]) {
    const uint4 v = *reinterpret_cast<const uint4 *>(p);
    const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&v);
#pragma unroll
    for (int k = 0; k < 4; k++) {
        const float2 t = __bfloat1622float2(h[k]);
        f[2 * k] = t.x;
        f[2 * k + 1] = t.y;
    }
}

__device__ __forceinline__ void st8(bf16 *p, const float f[8]) {
    uint4 v;
    __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(&v);
#pragma unroll
    for (int k = 0; k < 4; k++) h[k] = __floats2bfloat162_rn(f[2 * k], f[2 * k + 1]);
    *reinterpret_cast<uint4 *>(p) = v;
}

// item i of a view -> (z, y, x) and the chunk's first channel
struct Item {
    int z, y, x, c;
};
__device__ __forceinline__ Item item(const View &t, int i) {
    const int nq = t.nc >> 3;
    const int v = i / nq;
    Item r;
    r.c = (i - v * nq) << 3;
    r.x = v % t.W;
    const int r2 = v / t.W;
    r.y = r2 % t.H;
    r.z = r2 / t.H;
    return r;
}
__device__ __forceinline__ bf16 *at(const View &t, int z, int y, int x, int c) {
    return t.p + vox(t, z, y, x) * t.C + c;
}
__device__ __forceinline__ int items(const View &t) { return t.D * t.H * t.W * (t.nc >> 3); }

// db[co] += sum_v dY[v][co]: the grid stride is a multiple of the chunks per voxel, so
// each thread keeps one chunk and sums it in registers; warps fold lanes of the same
// chunk, the block folds its warps in shared memory, one atomic per channel per block
__global__ void __launch_bounds__(256) k_bias_grad(View dY, int cout_real, float *__restrict__ db) {
    __shared__ float red[8][64];
    const int n = items(dY), nq = dY.nc >> 3;
    float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const int i0 = blockIdx.x * blockDim.x + threadIdx.x;
    for (int i = i0; i < n; i += gridDim.x * blockDim.x) {
        const Item it = item(dY, i);
        float f[8];
        ld8(at(dY, it.z, it.y, it.x, it.c), f);
#pragma unroll
        for (int k = 0; k < 8; k++) s[k] += f[k];
    }
    // lanes with the same chunk differ by multiples of nq (a power of two <= 8)
#pragma unroll
    for (int k = 0; k < 8; k++)
        for (int o = 16; o >= nq; o >>= 1) s[k] += __shfl_xor_sync(0xffffffffu, s[k], o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane < nq) {
#pragma unroll
        for (int k = 0; k < 8; k++) red[warp][8 * lane + k] = s[k];  // lane = chunk (i0 % nq)
    }
    __syncthreads();
    const int c = threadIdx.x;
    if (c < dY.nc && c < cout_real) {
        float t = 0.f;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += red[w][c];
        if (t != 0.f) atomicAdd(&db[c], t);
    }
}

// g *= (y > 0) over the view's channels
__global__ void k_relu_bwd(View g, View y) {
    const int n = items(g);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const Item it = item(g, i);
        float gv[8], yv[8];
        ld8(at(g, it.z, it.y, it.x, it.c), gv);
        ld8(at(y, it.z, it.y, it.x, it.c), yv);
#pragma unroll
        for (int k = 0; k < 8; k++) gv[k] = yv[k] > 0.f ? gv[k] : 0.f;
        st8(at(g, it.z, it.y, it.x, it.c), gv);
    }
}

// out = 2x2x2 average of in (out has half the size)
__global__ void k_pool(View in, View out) {
    const int n = items(out);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const Item it = item(out, i);
        float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < 8; k++) {
            float f[8];
            ld8(at(in, 2 * it.z + (k >> 2), 2 * it.y + ((k >> 1) & 1), 2 * it.x + (k & 1), it.c), f);
#pragma unroll
            for (int e = 0; e < 8; e++) s[e] += f[e];
        }
#pragma unroll
        for (int e = 0; e < 8; e++) s[e] *= 0.125f;
        st8(at(out, it.z, it.y, it.x, it.c), s);
    }
}

// gradient of the pooling: gin[2v + k] (+)= gout[v] / 8
__global__ void k_pool_bwd(View gout, View gin, int accumulate) {
    const int n = items(gin);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const Item it = item(gin, i);
        float g[8], d[8];
        ld8(at(gout, it.z >> 1, it.y >> 1, it.x >> 1, it.c), g);
        bf16 *dst = at(gin, it.z, it.y, it.x, it.c);
        if (accumulate) ld8(dst, d);
#pragma unroll
        for (int e = 0; e < 8; e++) g[e] = 0.125f * g[e] + (accumulate ? d[e] : 0.f);
        st8(dst, g);
    }
}

// out (twice the size) = nearest-neighbour copy of in
__global__ void k_upsample(View in, View out) {
    const int n = items(out);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const Item it = item(out, i);
        *reinterpret_cast<uint4 *>(at(out, it.z, it.y, it.x, it.c)) =
            *reinterpret_cast<const uint4 *>(at(in, it.z >> 1, it.y >> 1, it.x >> 1, it.c));
    }
}

// gradient of the up-sampling: gin[v] = sum of the 8 gout it was copied to
__global__ void k_upsample_bwd(View gout, View gin) {
    const int n = items(gin);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const Item it = item(gin, i);
        float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < 8; k++) {
            float f[8];
            ld8(at(gout, 2 * it.z + (k >> 2), 2 * it.y + ((k >> 1) & 1), 2 * it.x + (k & 1), it.c), f);
#pragma unroll
            for (int e = 0; e < 8; e++) s[e] += f[e];
        }
        st8(at(gin, it.z, it.y, it.x, it.c), s);
    }
}

// input buffer (16 channels, 6 used, the rest zero) from node-major floats (n x 6)
__global__ void k_pack_input(const float *__restrict__ in6, View x) {
    const int n = x.D * x.H * x.W;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int xx = i % x.W, r = i / x.W;
        const float2 a = *reinterpret_cast<const float2 *>(in6 + 6 * (size_t)i);
        const float2 b = *reinterpret_cast<const float2 *>(in6 + 6 * (size_t)i + 2);
        const float2 c = *reinterpret_cast<const float2 *>(in6 + 6 * (size_t)i + 4);
        const float f[8] = {a.x, a.y, b.x, b.y, c.x, c.y, 0.f, 0.f};
        st8(at(x, r / x.H, r % x.H, xx, 0), f);
    }
}

// loss = sum_i w_i |out_i - target_i|^2 / (3 n) with w_i = 1 + surface_weight at nodes
// whose data-gradient input (channels 3-5) is non-zero, else 1; gout = d loss / d out
__global__ void k_mse(const float *__restrict__ outf, const float *__restrict__ target, const float *__restrict__ in6,
                      float surface_weight, View go, double *loss) {
    const long n = (long)go.D * go.H * go.W;
    const float scale = 2.f / (3.f * (float)n);
    float s = 0.f;
    for (long i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
        const int x = (int)(i % go.W), y = (int)((i / go.W) % go.H), z = (int)(i / ((long)go.W * go.H));
        const bool surf = in6[6 * i + 3] != 0.f || in6[6 * i + 4] != 0.f || in6[6 * i + 5] != 0.f;
        const float w = surf ? 1.f + surface_weight : 1.f;
        for (int c = 0; c < 3; c++) {
            const float d = outf[3 * i + c] - target[3 * i + c];
            s += w * d * d;
            go.p[vox(go, z, y, x) * go.C + c] = __float2bfloat16_rn(scale * w * d);
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0 && s != 0.f) atomicAdd(loss, (double)s / (3.0 * (double)n));
}

// Adam on the FP32 master parameters, then the BF16 forward weights (padded [27][CinP]
// [CoutP]) and the flipped, transposed dgrad weights ([27][CoutP][CinP], tap 26 - t).
struct LayerDev {
    float *w, *b, *gw, *gb, *mw, *vw, *mb, *vb;  // master / grads / moments (unpadded)
    bf16 *wf, *wt;                                // forward and dgrad weights (padded)
    bf16 *wfc, *wtc;                              // the same in the tcgen05 operand layout
    int cin, cout, cinp, coutp;
};

__global__ void k_adam(LayerDev L, float lr, float b1, float b2, float eps, float c1, float c2) {
    const int nw = 27 * L.cin * L.cout;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nw + L.cout; i += gridDim.x * blockDim.x) {
        float *p, *m, *v, g;
        if (i < nw) {
            const int tap = i / (L.cin * L.cout), ci = (i / L.cout) % L.cin, co = i % L.cout;
            g = L.gw[((size_t)tap * L.cinp + ci) * L.coutp + co];
            p = L.w + i;
            m = L.mw + i;
            v = L.vw + i;
        } else {
            g = L.gb[i - nw];
            p = L.b + (i - nw);
            m = L.mb + (i - nw);
            v = L.vb + (i - nw);
        }
        *m = b1 * *m + (1.f - b1) * g;
        *v = b2 * *v + (1.f - b2) * g * g;
        *p -= lr * (*m / c1) / (sqrtf(*v / c2) + eps);
    }
}

__global__ void k_pack_weights(LayerDev L) {
    const int n = 27 * L.cinp * L.coutp;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int tap = i / (L.cinp * L.coutp), ci = (i / L.coutp) % L.cinp, co = i % L.coutp;
        const float w = (ci < L.cin && co < L.cout) ? L.w[((size_t)tap * L.cin + ci) * L.cout + co] : 0.f;
        const bf16 wb = __float2bfloat16_rn(w);
        L.wf[i] = wb;
        L.wt[((size_t)(26 - tap) * L.coutp + co) * L.cinp + ci] = wb;
        // tcgen05 B operands, per 16-channel input slice kc and tap: N x 16, K-major core
        // matrices [N/8][2][8][8]; forward N = Cout (K = Cin), dgrad N = Cin (K = Cout)
        auto tc = [](int kc, int t, int n, int kl, int N) {
            return ((((size_t)kc * 27 + t) * (N / 8) + n / 8) * 2 + kl / 8) * 64 + (n % 8) * 8 + (kl % 8);
        };
        L.wfc[tc(ci / 16, tap, co, ci % 16, L.coutp)] = wb;
        L.wtc[tc(co / 16, 26 - tap, ci, co % 16, L.cinp)] = wb;
    }
}

long nvox(const View &v) { return (long)v.D * v.H * v.W; }

int blocks(long n, int threads = 256) {
    long b = (n + threads - 1) / threads;
    return (int)std::max<long>(1, std::min<long>(b, 148 * 8));
}

}  // namespace

struct vd_unet {
    int D, H, W;
    std::vector<void *> bufs;
    // activations (with halo) and gradients
    View x, e1a, cat1, p1, e2a, cat2, p2, e3a, e3, d2a, d2, d1a, d1, out;
    View gx, ge1a, gcat1, gp1, ge2a, gcat2, gp2, ge3a, ge3, gd2a, gd2, gd1a, gd1, gout;
    LayerDev L[kLayers];
    double *loss = nullptr;
    float *io3 = nullptr;  // FP32 output of the training forward pass
    int *tc_err = nullptr; // set by a tensor-core convolution whose bounded wait gave up
    std::map<const void *, CUtensorMap> tmaps;  // per activation / gradient buffer (TMA)
    int step = 0;
    cudaStream_t st = nullptr;
};

namespace {

template <typename T>
bool ualloc(vd_unet *U, T **p, size_t n) {
    void *q = nullptr;
    if (cudaMalloc(&q, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaMemset(q, 0, std::max<size_t>(n, 1) * sizeof(T));
    U->bufs.push_back(q);
    *p = (T *)q;
    return true;
}

bool make_view(vd_unet *U, View *v, int D, int H, int W, int C) {
    v->D = D;
    v->H = H;
    v->W = W;
    v->C = C;
    v->Wp = W + 18;
    v->nc = C;
    v->c0 = 0;
    const size_t n = (size_t)(D + 2) * (H + 2) * v->Wp * C + 16 * (size_t)C;
    bf16 *p;
    if (!ualloc(U, &p, n)) return false;
    v->p = p;
    return true;
}

View slice(View v, int c0, int nc) {
    v.p += c0;
    v.c0 += c0;
    v.nc = nc;
    return v;
}

void conv(cudaStream_t st, View in, const LayerDev &L, View out, bool relu, bool dgrad, vd_unet *U,
          float *outf = nullptr) {
    int *err = U->tc_err;
    // forward: in (cinp) -> out (coutp slice); dgrad: in = grad of out (coutp) -> grad of in (cinp)
    const bf16 *w = dgrad ? L.wt : L.wf;
    const int nf = (dgrad ? L.cinp : L.coutp) / 16;
    const int creal = dgrad ? L.cinp : L.cout;
    const float *bias = dgrad ? nullptr : L.b;
    const int xt = (out.W + 15) / 16;
    // The persistent, pipelined form for 48 or more output channels (the layers where it
    // measured faster: the 16- and 32-channel layers run at the tensor core's rate for
    // N = 16 or 32 MMAs in either form, and there the per-row-group CTAs of k_conv3d_tc
    // overlap better).
    const int nstage = tcp_stages(out.W, out.H, nf, in.nc / 16);
    if (out.W <= kTcMaxW && (nf == 3 || nf == 4 || nf == 6) && nstage >= 2 && tcp_tmem_cols(out.W, out.H, nf) > 0) {
        static int sms = 0;
        if (!sms && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0) != cudaSuccess) sms = 148;
        const int rows = tc_rows(out.W, out.H), items = out.D * ((out.H + rows - 1) / rows);
        const int nb = std::min(items, sms);
        const int sm = tcp_smem_bytes(out.W, out.H, nf, in.nc / 16, nstage), cols = tcp_tmem_cols(out.W, out.H, nf);
        const int nacc = tcp_nacc(out.W, out.H, nf);
        const bf16 *wtc = dgrad ? L.wtc : L.wfc;
        const CUtensorMap &tm = U->tmaps.at(in.p - in.c0);
        switch (nf) {
            case 3: k_conv3d_tcp<3><<<nb, 192, sm, st>>>(tm, in, wtc, bias, out, creal, relu, outf, cols, nstage, nacc, err); break;
            case 4: k_conv3d_tcp<4><<<nb, 192, sm, st>>>(tm, in, wtc, bias, out, creal, relu, outf, cols, nstage, nacc, err); break;
            default: k_conv3d_tcp<6><<<nb, 192, sm, st>>>(tm, in, wtc, bias, out, creal, relu, outf, cols, nstage, nacc, err); break;
        }
        return;
    }
    if (out.W <= kTcMaxW && (nf == 1 || nf == 2 || nf == 3 || nf == 4 || nf == 6) &&
        tc_smem_bytes(out.W, out.H, nf) <= kTcpSmemMax) {
        const int rows = tc_rows(out.W, out.H), nb = out.D * ((out.H + rows - 1) / rows);
        const int sm = tc_smem_bytes(out.W, out.H, nf), cols = tc_tmem_cols(out.W, out.H, nf);
        const bf16 *wtc = dgrad ? L.wtc : L.wfc;
        const CUtensorMap &tm = U->tmaps.at(in.p - in.c0);
        switch (nf) {
            case 1: k_conv3d_tc<1><<<nb, 128, sm, st>>>(tm, in, wtc, bias, out, creal, relu, outf, cols, err); break;
            case 2: k_conv3d_tc<2><<<nb, 128, sm, st>>>(tm, in, wtc, bias, out, creal, relu, outf, cols, err); break;
            case 3: k_conv3d_tc<3><<<nb, 128, sm, st>>>(tm, in, wtc, bias, out, creal, relu, outf, cols, err); break;
            case 4: k_conv3d_tc<4><<<nb, 128, sm, st>>>(tm, in, wtc, bias, out, creal, relu, outf, cols, err); break;
            default: k_conv3d_tc<6><<<nb, 128, sm, st>>>(tm, in, wtc, bias, out, creal, relu, outf, cols, err); break;
        }
        return;
    }
    const long tiles = (long)out.D * out.H * xt;
    const int nb = (int)((tiles + 3) / 4);
    switch (nf) {
        case 1: k_conv3d<1><<<nb, 128, 0, st>>>(in, w, bias, out, creal, relu, outf); break;
        case 2: k_conv3d<2><<<nb, 128, 0, st>>>(in, w, bias, out, creal, relu, outf); break;
        case 3: k_conv3d<3><<<nb, 128, 0, st>>>(in, w, bias, out, creal, relu, outf); break;
        case 4: k_conv3d<4><<<nb, 128, 0, st>>>(in, w, bias, out, creal, relu, outf); break;
        case 6: k_conv3d<6><<<nb, 128, 0, st>>>(in, w, bias, out, creal, relu, outf); break;
        default: break;
    }
}

void wgrad(cudaStream_t st, View X, View dY, const LayerDev &L) {
    const int nci = X.nc / 16, nco = dY.nc / 16;
    const int xt_n = (dY.W + 15) / 16;
    const long bands = (long)dY.D * dY.H * ((xt_n + kWgTiles - 1) / kWgTiles);
    // about six blocks per SM in all (measured best among 2-16; each block ends with 27 x 256
    // atomics)
    const int slices = (int)std::max<long>(1, std::min<long>(bands, (6 * 148 + nci * nco - 1) / (nci * nco)));
    k_wgrad<<<nci * nco * slices, 256, 0, st>>>(X, dY, L.gw, L.coutp, slices);
    k_bias_grad<<<(int)std::min<long>(2 * 148, (nvox(dY) * dY.nc / 8 + 255) / 256), 256, 0, st>>>(dY, L.cout, L.gb);
}

// the head writes FP32 to outf (node-major, 3 per node)
void forward(vd_unet *U, cudaStream_t st, float *outf) {
    View e1 = slice(U->cat1, 32, 16), e2 = slice(U->cat2, 64, 32);
    conv(st, U->x, U->L[A1], U->e1a, true, false, U);
    conv(st, U->e1a, U->L[B1], e1, true, false, U);
    k_pool<<<blocks(nvox(U->p1) * 2), 256, 0, st>>>(e1, U->p1);
    conv(st, U->p1, U->L[A2], U->e2a, true, false, U);
    conv(st, U->e2a, U->L[B2], e2, true, false, U);
    k_pool<<<blocks(nvox(U->p2) * 4), 256, 0, st>>>(e2, U->p2);
    conv(st, U->p2, U->L[A3], U->e3a, true, false, U);
    conv(st, U->e3a, U->L[B3], U->e3, true, false, U);
    k_upsample<<<blocks(nvox(U->cat2) * 8), 256, 0, st>>>(U->e3, slice(U->cat2, 0, 64));
    conv(st, U->cat2, U->L[C2], U->d2a, true, false, U);
    conv(st, U->d2a, U->L[D2], U->d2, true, false, U);
    k_upsample<<<blocks(nvox(U->cat1) * 4), 256, 0, st>>>(U->d2, slice(U->cat1, 0, 32));
    conv(st, U->cat1, U->L[C1], U->d1a, true, false, U);
    conv(st, U->d1a, U->L[D1], U->d1, true, false, U);
    conv(st, U->d1, U->L[HEAD], U->out, false, false, U, outf);
}

void relu_bwd(cudaStream_t st, View g, View y) {
    k_relu_bwd<<<blocks(nvox(g) * g.nc / 8), 256, 0, st>>>(g, y);
}

// gout must hold d loss / d out; fills every layer's gw, gb
void backward(vd_unet *U, cudaStream_t st) {
    View e1 = slice(U->cat1, 32, 16), e2 = slice(U->cat2, 64, 32);
    View ge1 = slice(U->gcat1, 32, 16), ge2 = slice(U->gcat2, 64, 32);
    for (int l = 0; l < kLayers; l++) {
        cudaMemsetAsync(U->L[l].gw, 0, sizeof(float) * 27 * U->L[l].cinp * U->L[l].coutp, st);
        cudaMemsetAsync(U->L[l].gb, 0, sizeof(float) * U->L[l].cout, st);
    }
    // head (linear) and decoder level 1
    wgrad(st, U->d1, U->gout, U->L[HEAD]);
    conv(st, U->gout, U->L[HEAD], U->gd1, false, true, U);
    relu_bwd(st, U->gd1, U->d1);
    wgrad(st, U->d1a, U->gd1, U->L[D1]);
    conv(st, U->gd1, U->L[D1], U->gd1a, false, true, U);
    relu_bwd(st, U->gd1a, U->d1a);
    wgrad(st, U->cat1, U->gd1a, U->L[C1]);
    conv(st, U->gd1a, U->L[C1], U->gcat1, false, true, U);  // [d up(d2), d e1 (skip)]
    // decoder level 2
    k_upsample_bwd<<<blocks(nvox(U->gd2) * 4), 256, 0, st>>>(slice(U->gcat1, 0, 32), U->gd2);
    relu_bwd(st, U->gd2, U->d2);
    wgrad(st, U->d2a, U->gd2, U->L[D2]);
    conv(st, U->gd2, U->L[D2], U->gd2a, false, true, U);
    relu_bwd(st, U->gd2a, U->d2a);
    wgrad(st, U->cat2, U->gd2a, U->L[C2]);
    conv(st, U->gd2a, U->L[C2], U->gcat2, false, true, U);  // [d up(e3), d e2 (skip)]
    // bottleneck
    k_upsample_bwd<<<blocks(nvox(U->ge3) * 8), 256, 0, st>>>(slice(U->gcat2, 0, 64), U->ge3);
    relu_bwd(st, U->ge3, U->e3);
    wgrad(st, U->e3a, U->ge3, U->L[B3]);
    conv(st, U->ge3, U->L[B3], U->ge3a, false, true, U);
    relu_bwd(st, U->ge3a, U->e3a);
    wgrad(st, U->p2, U->ge3a, U->L[A3]);
    conv(st, U->ge3a, U->L[A3], U->gp2, false, true, U);
    // encoder level 2: d e2 = skip part + pooling part
    k_pool_bwd<<<blocks(nvox(ge2) * 4), 256, 0, st>>>(U->gp2, ge2, 1);
    relu_bwd(st, ge2, e2);
    wgrad(st, U->e2a, ge2, U->L[B2]);
    conv(st, ge2, U->L[B2], U->ge2a, false, true, U);
    relu_bwd(st, U->ge2a, U->e2a);
    wgrad(st, U->p1, U->ge2a, U->L[A2]);
    conv(st, U->ge2a, U->L[A2], U->gp1, false, true, U);
    // encoder level 1
    k_pool_bwd<<<blocks(nvox(ge1) * 2), 256, 0, st>>>(U->gp1, ge1, 1);
    relu_bwd(st, ge1, e1);
    wgrad(st, U->e1a, ge1, U->L[B1]);
    conv(st, ge1, U->L[B1], U->ge1a, false, true, U);
    relu_bwd(st, U->ge1a, U->e1a);
    wgrad(st, U->x, U->ge1a, U->L[A1]);
}

int num_params() {
    int n = 0;
    for (int l = 0; l < kLayers; l++) n += 27 * kCin[l] * kCout[l] + kCout[l];
    return n;
}

}  // namespace

extern "C" {

vd_status vd_unet_create(int nx, int ny, int nz, unsigned long long seed, vd_unet **out) {
    if (!out || nx < 4 || ny < 4 || nz < 4 || nx % 4 || ny % 4 || nz % 4) return VD_ERR_INVALID_ARG;
    *out = nullptr;
    vd_unet *U = new (std::nothrow) vd_unet();
    if (!U) return VD_ERR_OOM;
    U->D = nz;
    U->H = ny;
    U->W = nx;
    const int D = nz, H = ny, W = nx;
    bool ok = true;
    struct {
        View *v, *g;
        int s, c;
    } spec[] = {{&U->x, &U->gx, 1, 16},     {&U->e1a, &U->ge1a, 1, 16}, {&U->cat1, &U->gcat1, 1, 48},
                {&U->p1, &U->gp1, 2, 16},   {&U->e2a, &U->ge2a, 2, 32}, {&U->cat2, &U->gcat2, 2, 96},
                {&U->p2, &U->gp2, 4, 32},   {&U->e3a, &U->ge3a, 4, 64}, {&U->e3, &U->ge3, 4, 64},
                {&U->d2a, &U->gd2a, 2, 32}, {&U->d2, &U->gd2, 2, 32},   {&U->d1a, &U->gd1a, 1, 16},
                {&U->d1, &U->gd1, 1, 16},   {&U->out, &U->gout, 1, 16}};
    for (auto &s : spec) {
        ok = ok && make_view(U, s.v, D / s.s, H / s.s, W / s.s, s.c);
        ok = ok && make_view(U, s.g, D / s.s, H / s.s, W / s.s, s.c);
    }
    // one TMA tensor map per buffer: dims (C, Wp, H + 2, D + 2), box (8 channels, W + 2
    // voxels, tc_rows + 2 rows, 3 planes), zero fill past the buffer
    if (ok) {
        static void *encode = nullptr;
        static std::once_flag once;
        std::call_once(once, [] {
            cudaDriverEntryPointQueryResult q;
            if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &encode, 12000, cudaEnableDefault, &q) !=
                    cudaSuccess ||
                q != cudaDriverEntryPointSuccess)
                encode = nullptr;
        });
        typedef CUresult (*EncodeFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                     const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                     CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
        ok = encode != nullptr;
        for (auto &sp : spec) {
            for (View *v : {sp.v, sp.g}) {
                if (!ok) break;
                CUtensorMap tm;
                const cuuint64_t dims[4] = {(cuuint64_t)v->C, (cuuint64_t)v->Wp, (cuuint64_t)v->H + 2, (cuuint64_t)v->D + 2};
                const cuuint64_t strides[3] = {(cuuint64_t)v->C * 2, (cuuint64_t)v->C * 2 * v->Wp,
                                               (cuuint64_t)v->C * 2 * v->Wp * (v->H + 2)};
                const cuuint32_t box[4] = {8, (cuuint32_t)tc_rw(v->W), (cuuint32_t)tc_rows(v->W, v->H) + 2, 3};
                const cuuint32_t es[4] = {1, 1, 1, 1};
                ok = v->W > kTcMaxW ||
                     ((EncodeFn)encode)(&tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, v->p, dims, strides, box, es,
                                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                                        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
                if (ok && v->W <= kTcMaxW) U->tmaps[v->p] = tm;
            }
        }
    }
    std::mt19937_64 rng(seed);
    for (int l = 0; l < kLayers && ok; l++) {
        LayerDev &L = U->L[l];
        L.cin = kCin[l];
        L.cout = kCout[l];
        L.cinp = pad16(kCin[l]);
        L.coutp = pad16(kCout[l]);
        const size_t nw = 27 * (size_t)L.cin * L.cout, np = 27 * (size_t)L.cinp * L.coutp;
        ok = ok && ualloc(U, &L.w, nw) && ualloc(U, &L.b, L.cout) && ualloc(U, &L.gw, np) &&
             ualloc(U, &L.gb, L.cout) && ualloc(U, &L.mw, nw) && ualloc(U, &L.vw, nw) && ualloc(U, &L.mb, L.cout) &&
             ualloc(U, &L.vb, L.cout) && ualloc(U, &L.wf, np) && ualloc(U, &L.wt, np) && ualloc(U, &L.wfc, np) &&
             ualloc(U, &L.wtc, np);
        if (!ok) break;
        // He initialisation (the head starts small: the first prediction is ~0)
        std::normal_distribution<float> nd(0.f, std::sqrt(2.f / (27.f * L.cin)) * (l == HEAD ? 0.01f : 1.f));
        std::vector<float> w(nw);
        for (auto &v : w) v = nd(rng);
        cudaMemcpy(L.w, w.data(), nw * sizeof(float), cudaMemcpyHostToDevice);
        k_pack_weights<<<blocks((long)np), 256>>>(L);
    }
    ok = ok && ualloc(U, &U->loss, 1) && ualloc(U, &U->io3, (size_t)3 * D * H * W) && ualloc(U, &U->tc_err, 1);
    // the staged convolutions may take more than the default 48 KB of shared memory
#define VD_TC_SMEM(N) \
    ok = ok && cudaFuncSetAttribute(k_conv3d_tc<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                    kTcpSmemMax) == cudaSuccess;
    VD_TC_SMEM(1) VD_TC_SMEM(2) VD_TC_SMEM(3) VD_TC_SMEM(4) VD_TC_SMEM(6)
#undef VD_TC_SMEM
#define VD_TCP_SMEM(N) \
    ok = ok && cudaFuncSetAttribute(k_conv3d_tcp<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcpSmemMax) == cudaSuccess;
    VD_TCP_SMEM(3) VD_TCP_SMEM(4) VD_TCP_SMEM(6)
#undef VD_TCP_SMEM
    if (!ok || cudaStreamCreateWithFlags(&U->st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess) {
        vd_unet_destroy(U);
        return VD_ERR_OOM;
    }
    *out = U;
    return VD_OK;
}

vd_status vd_unet_destroy(vd_unet *U) {
    if (!U) return VD_OK;
    if (U->st) cudaStreamSynchronize(U->st);
    for (void *p : U->bufs) cudaFree(p);
    if (U->st) cudaStreamDestroy(U->st);
    delete U;
    return VD_OK;
}

vd_status vd_unet_num_params(const vd_unet *U, int *n) {
    if (!U || !n) return VD_ERR_INVALID_ARG;
    *n = num_params();
    return VD_OK;
}

static vd_status unet_io(vd_unet *U, void *dst_or_src, int n, int dir, int which) {
    // which 0: parameters, 1: gradients; dir 0: device -> host, 1: host -> device
    if (!U || !dst_or_src || n != num_params()) return VD_ERR_INVALID_ARG;
    float *h = (float *)dst_or_src;
    size_t off = 0;
    for (int l = 0; l < kLayers; l++) {
        LayerDev &L = U->L[l];
        const size_t nw = 27 * (size_t)L.cin * L.cout;
        if (which == 0) {
            if (dir == 0) {
                cudaMemcpy(h + off, L.w, nw * sizeof(float), cudaMemcpyDeviceToHost);
                cudaMemcpy(h + off + nw, L.b, L.cout * sizeof(float), cudaMemcpyDeviceToHost);
            } else {
                cudaMemcpy(L.w, h + off, nw * sizeof(float), cudaMemcpyHostToDevice);
                cudaMemcpy(L.b, h + off + nw, L.cout * sizeof(float), cudaMemcpyHostToDevice);
                k_pack_weights<<<blocks(27L * L.cinp * L.coutp), 256>>>(L);
            }
        } else {
            std::vector<float> g(27 * (size_t)L.cinp * L.coutp);
            cudaMemcpy(g.data(), L.gw, g.size() * sizeof(float), cudaMemcpyDeviceToHost);
            for (int t = 0; t < 27; t++)
                for (int ci = 0; ci < L.cin; ci++)
                    for (int co = 0; co < L.cout; co++)
                        h[off + ((size_t)t * L.cin + ci) * L.cout + co] = g[((size_t)t * L.cinp + ci) * L.coutp + co];
            cudaMemcpy(h + off + nw, L.gb, L.cout * sizeof(float), cudaMemcpyDeviceToHost);
        }
        off += nw + L.cout;
    }
    return cudaDeviceSynchronize() == cudaSuccess ? VD_OK : VD_ERR_CUDA;
}

vd_status vd_unet_get_params(vd_unet *U, float *host, int n) { return unet_io(U, host, n, 0, 0); }
vd_status vd_unet_set_params(vd_unet *U, const float *host, int n) { return unet_io(U, (void *)host, n, 1, 0); }
vd_status vd_unet_get_grads(vd_unet *U, float *host, int n) { return unet_io(U, host, n, 0, 1); }

vd_status vd_unet_forward_async(vd_unet *U, const float *in6, float *out3, void *stream) {
    if (!U || !in6 || !out3) return VD_ERR_INVALID_ARG;
    cudaStream_t st = stream ? (cudaStream_t)stream : U->st;
    const long n = (long)U->D * U->H * U->W;
    k_pack_input<<<blocks(n), 256, 0, st>>>(in6, U->x);
    forward(U, st, out3);
    return cudaGetLastError() == cudaSuccess ? VD_OK : VD_ERR_CUDA;
}

// after a synchronisation: a tensor-core convolution whose bounded wait gave up
static vd_status unet_wait_status(vd_unet *U) {
    int e = 0;
    if (cudaMemcpy(&e, U->tc_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return VD_ERR_CUDA;
    if (!e) return VD_OK;
    cudaMemset(U->tc_err, 0, sizeof(int));
    return VD_ERR_TIMEOUT;
}

vd_status vd_unet_forward(vd_unet *U, const float *in6, float *out3) {
    const vd_status s = vd_unet_forward_async(U, in6, out3, nullptr);
    if (s != VD_OK) return s;
    if (cudaStreamSynchronize(U->st) != cudaSuccess) return VD_ERR_CUDA;
    return unet_wait_status(U);
}

// One Adam step on the mean squared error between network(in6) and target3 (device
// arrays); lr = 0 only computes the loss and the gradients.
vd_status vd_unet_train_step(vd_unet *U, const float *in6, const float *target3, float surface_weight, float lr,
                             double *loss) {
    if (!U || !in6 || !target3 || !(surface_weight >= 0.f)) return VD_ERR_INVALID_ARG;
    cudaStream_t st = U->st;
    const long n = (long)U->D * U->H * U->W;
    k_pack_input<<<blocks(n), 256, 0, st>>>(in6, U->x);
    forward(U, st, U->io3);
    cudaMemsetAsync(U->loss, 0, sizeof(double), st);
    k_mse<<<blocks(n), 256, 0, st>>>(U->io3, target3, in6, surface_weight, U->gout, U->loss);
    backward(U, st);
    if (lr > 0.f) {
        U->step++;
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.f - std::pow(b1, (float)U->step), c2 = 1.f - std::pow(b2, (float)U->step);
        for (int l = 0; l < kLayers; l++) {
            k_adam<<<blocks(27L * U->L[l].cin * U->L[l].cout + U->L[l].cout), 256, 0, st>>>(U->L[l], lr, b1, b2, 1e-8f,
                                                                                              c1, c2);
            k_pack_weights<<<blocks(27L * U->L[l].cinp * U->L[l].coutp), 256, 0, st>>>(U->L[l]);
        }
    }
    double h = 0.0;
    cudaMemcpyAsync(&h, U->loss, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) return VD_ERR_CUDA;
    if (loss) *loss = h;
    return unet_wait_status(U);
}

// Weights file: "VDUNET01", int32 layer count, int32 Cin[], int32 Cout[], int32 parameter
// count, then the FP32 parameters (per layer: weights [27][Cin][Cout], bias [Cout]); all
// little-endian.
static const char kMagic[8] = {'V', 'D', 'U', 'N', 'E', 'T', '0', '1'};

static bool little_endian() {
    const unsigned one = 1;
    unsigned char b;
    memcpy(&b, &one, 1);
    return b == 1;
}

vd_status vd_unet_save(vd_unet *U, const char *path) {
    if (!U || !path || !little_endian()) return VD_ERR_INVALID_ARG;
    const int n = num_params();
    std::vector<float> h(n);
    vd_status s = vd_unet_get_params(U, h.data(), n);
    if (s != VD_OK) return s;
    FILE *f = fopen(path, "wb");
    if (!f) return VD_ERR_INVALID_ARG;
    const int layers = kLayers;
    bool ok = fwrite(kMagic, 1, 8, f) == 8 && fwrite(&layers, 4, 1, f) == 1 && fwrite(kCin, 4, kLayers, f) == kLayers &&
              fwrite(kCout, 4, kLayers, f) == kLayers && fwrite(&n, 4, 1, f) == 1 &&
              fwrite(h.data(), 4, n, f) == (size_t)n;
    ok = (fclose(f) == 0) && ok;
    return ok ? VD_OK : VD_ERR_INVALID_ARG;
}

vd_status vd_unet_load(vd_unet *U, const char *path) {
    if (!U || !path || !little_endian()) return VD_ERR_INVALID_ARG;
    FILE *f = fopen(path, "rb");
    if (!f) return VD_ERR_INVALID_ARG;
    char magic[8];
    int layers = 0, cin[kLayers], cout[kLayers], n = 0;
    bool ok = fread(magic, 1, 8, f) == 8 && !memcmp(magic, kMagic, 8) && fread(&layers, 4, 1, f) == 1 &&
              layers == kLayers && fread(cin, 4, kLayers, f) == kLayers && fread(cout, 4, kLayers, f) == kLayers &&
              !memcmp(cin, kCin, sizeof(cin)) && !memcmp(cout, kCout, sizeof(cout)) && fread(&n, 4, 1, f) == 1 &&
              n == num_params();
    std::vector<float> h(ok ? n : 0);
    ok = ok && fread(h.data(), 4, n, f) == (size_t)n;
    fclose(f);
    if (!ok) return VD_ERR_INVALID_ARG;
    return vd_unet_set_params(U, h.data(), n);
}

// The intermediate tensors in the order of the VD_UNET_T_* ids of include/vd.h.
static View unet_tensor(vd_unet *U, int id) {
    const View e1 = slice(U->cat1, 32, 16), e2 = slice(U->cat2, 64, 32);
    const View ge1 = slice(U->gcat1, 32, 16), ge2 = slice(U->gcat2, 64, 32);
    const View t[] = {U->x,    U->e1a,  e1,     U->p1,   U->e2a,  e2,      U->p2,    U->e3a,  U->e3,  U->cat2,
                      U->d2a,  U->d2,   U->cat1, U->d1a, U->d1,   U->gout, U->gd1,   U->gd1a, U->gcat1, U->gd2,
                      U->gd2a, U->gcat2, U->ge3, U->ge3a, U->gp2, ge2,      U->ge2a, U->gp1,  ge1,     U->ge1a};
    static_assert(sizeof(t) / sizeof(t[0]) == VD_UNET_T_COUNT, "tensor table");
    return t[id];
}

vd_status vd_unet_get_tensor(vd_unet *U, int id, float *host, long long n, int dims[4]) {
    if (!U || id < 0 || id >= VD_UNET_T_COUNT) return VD_ERR_INVALID_ARG;
    const View v = unet_tensor(U, id);
    if (dims) {
        dims[0] = v.D;
        dims[1] = v.H;
        dims[2] = v.W;
        dims[3] = v.nc;
    }
    if (!host) return VD_OK;
    const long long need = (long long)v.D * v.H * v.W * v.nc;
    if (n < need) return VD_ERR_INVALID_ARG;
    // the whole buffer (halo and slack included) once, then the view's voxels on the host
    const bf16 *base = v.p - v.c0;
    const size_t elems = (size_t)(v.D + 2) * (v.H + 2) * v.Wp * v.C + 16 * (size_t)v.C;
    std::vector<uint16_t> raw(elems);
    if (cudaStreamSynchronize(U->st) != cudaSuccess ||
        cudaMemcpy(raw.data(), base, elems * sizeof(uint16_t), cudaMemcpyDeviceToHost) != cudaSuccess)
        return VD_ERR_CUDA;
    size_t k = 0;
    for (int z = 0; z < v.D; z++)
        for (int y = 0; y < v.H; y++)
            for (int x = 0; x < v.W; x++) {
                const size_t o = vox(v, z, y, x) * v.C + v.c0;
                for (int c = 0; c < v.nc; c++) {
                    const uint32_t bits = (uint32_t)raw[o + c] << 16;  // BF16 is the top half of an FP32
                    memcpy(&host[k++], &bits, sizeof(float));
                }
            }
    return VD_OK;
}

vd_status vd_unet_dims(const vd_unet *U, int *nx, int *ny, int *nz) {
    if (!U) return VD_ERR_INVALID_ARG;
    if (nx) *nx = U->W;
    if (ny) *ny = U->H;
    if (nz) *nz = U->D;
    return VD_OK;
}

}  // extern "C"
