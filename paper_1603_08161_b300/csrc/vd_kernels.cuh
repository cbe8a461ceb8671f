// Device code of libvd: the per-frame flip-flop lattice solve of VolumeDeform
// (arXiv 1603.08161, Sec. 4-7) for sm_103a.
//
// Data layout in HBM (per lattice):
//   * node-indexed state u (3 x ld floats, SoA) and R (9 x ld floats, SoA, row-major
//     entry (r, c) at plane 3r + c), ld = nodes rounded up to 32;
//   * slot-indexed solver vectors x, r, p, q, Minv (3 x ld each, SoA): slot = node in
//     all-nodes mode, a compact index into the active set M in surface mode;
//   * source samples sorted by lattice cell (float4 point / normal / fractions, int
//     cell), with a list of occupied cells and their sample ranges; per-sample
//     association record float4 (g', r0') written once per Gauss-Newton iteration;
//   * FP64 scalars (PCG rho / p.Ap per iteration, energies) per iteration slot.
// Every reduction sums in FP32 within a warp and in FP64 across warps and blocks.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace vd {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kThreads = 256;

struct Ctx {
    // lattice
    int nx, ny, nz, nn, ld;
    // n / nx and n / ny as (2n m) >> 32 with m = ceil(2^31 / d), exact while n d < 2^31
    // (set when nn nx and nn ny are below 2^31; 0: integer division)
    unsigned mdx, mdy;
    float ox, oy, oz, h;
    // frame
    int W, H;
    float fx, fy, cx, cy;
    float Rg[9], tg[3];
    // weights / thresholds
    float w_s, w_d, w_r, eps_d, eps_n, eps_v;
    // state (node-indexed)
    float *u, *R;
    // active set
    const int *slot_of_node, *node_of_slot, *nbr;
    const int *n_active;
    // solver vectors (slot-indexed)
    float *x, *r, *p, *q, *minv;
    // frame data
    const float *depth;
    const float4 *nrm;
    // sorted samples
    const float4 *sp, *sn, *frac;
    const int *cell, *perm;
    const int *n_samples;
    const int *occ_cell, *occ_beg, *n_occ;
    float4 *rec;
    int *pix;
    int mixed;  // VD_PREC_MIXED: target normals and per-sample records stored as BF16 x 4
    float *wc;
    // sparse pairs
    const float4 *fh, *ft, *sfrac;
    const int *scell;
    int S;
    // Gauss-Newton early stop: after each iteration a gate compares E_total with
    // *e_target and marks the remaining iterations skipped (NULL: no gates)
    const double *e_target;
    // per block of the sample passes: first and end occupied cell, first and end sample
    const int4 *cell_part;
    // samples whose FP32 association lies near a threshold, re-taken in FP64
    int *refine;
    // coarse level of a hierarchy (Sec. 7.2): node counts and spacing of the finest
    // lattice (same origin); a point belongs to this level only if its cell exists on
    // the finest lattice.  dom_h = 0: no such restriction.
    int dom_n[3];
    float dom_h;
    // cached B^T B of the dense samples (Sec. 7.1): per occupied cell a 24 x 24 block,
    // row / column k * 3 + a (corner k, component a), built once per association;
    // nullptr: the J^T J p of the samples is applied matrix-free
    float *btb;
};

// Per-Gauss-Newton-iteration scalar block (FP64 sums and counters), zeroed at the
// start of every solve.
struct Scal {
    double e_dense, e_sparse, e_reg, pad;
    int stop, cg_done, n_valid, n_refined, n_degenerate, assoc_ran;
    int skip;  // this Gauss-Newton iteration is skipped (the energy target was met)
    int n_refine;  // entries of c.refine written by this iteration's association
    double rho[1];  // rho[0..K], then pq[0..K-1] follow (layout set by the host)
};

__host__ __device__ inline size_t scal_bytes(int K) {
    return (sizeof(Scal) + sizeof(double) * (size_t)(2 * K + 2) + 255) & ~(size_t)255;
}
__device__ __forceinline__ double *scal_rho(Scal *s) { return s->rho; }
__device__ __forceinline__ double *scal_pq(Scal *s, int K) { return s->rho + K + 1; }

// ------------------------------------------------------------------ launch ordering

// Programmatic dependent launch: a kernel of the solve may be scheduled while its
// predecessor drains; it waits here, before touching any memory, until the predecessor
// grid has completed and its writes are visible, then lets its own successor be
// scheduled.  Both are no-ops when the kernel was launched without the attribute.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// ------------------------------------------------------------------ reductions

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

// Block-wide sum of one float per thread, accumulated in FP64 across warps; thread 0
// adds the result to *dst.  Every thread of the block must call it.
// (FP64 work is kept to a 5-level tree in warp 0: B300's FP64 rate is low.)
__device__ __forceinline__ double warp0_tree_f64(const double *part, int lane) {
    double s = lane < (int)(blockDim.x >> 5) ? part[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
    return s;
}

__device__ __forceinline__ void block_add_f64(float v, double *dst) {
    __shared__ double part[32];
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) part[wid] = (double)v;
    __syncthreads();
    if (wid == 0) {
        const double s = warp0_tree_f64(part, lane);
        if (lane == 0 && s != 0.0) atomicAdd(dst, s);
    }
    __syncthreads();
}

__device__ __forceinline__ void block_add_f64d(double v, double *dst) {
    __shared__ double partd[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) partd[wid] = v;
    __syncthreads();
    if (wid == 0) {
        const double s = warp0_tree_f64(partd, lane);
        if (lane == 0 && s != 0.0) atomicAdd(dst, s);
    }
    __syncthreads();
}

__device__ __forceinline__ void block_add_int(int v, int *dst) {
    __shared__ int parti[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) parti[wid] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        int s = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); k++) s += parti[k];
        if (s) atomicAdd(dst, s);
    }
    __syncthreads();
}

// Reduce 32 per-lane values so that lane l ends with the warp-wide sum of value l
// (recursive halving: 31 shuffles for 32 sums).
__device__ __forceinline__ float warp_transpose_sum32(float (&v)[32]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int off = 16; off >= 1; off >>= 1) {
        const bool upper = (lane & off) != 0;
#pragma unroll
        for (int j = 0; j < off; j++) {
            const float send = upper ? v[j] : v[j + off];
            const float keep = upper ? v[j + off] : v[j];
            v[j] = keep + __shfl_xor_sync(FULL, send, off);
        }
    }
    return v[0];
}

// ------------------------------------------------------------------ lattice helpers

__device__ __forceinline__ int corner_node(const Ctx &c, int cell, int k) {
    return cell + (k & 1) + c.nx * (((k >> 1) & 1) + c.ny * ((k >> 2) & 1));
}

template <typename T>
__device__ __forceinline__ T trilinear_weight(const T f[3], int k) {
    const T wx = (k & 1) ? f[0] : T(1) - f[0];
    const T wy = (k & 2) ? f[1] : T(1) - f[1];
    const T wz = (k & 4) ? f[2] : T(1) - f[2];
    return wx * wy * wz;
}

template <bool kAll>
__device__ __forceinline__ int slot_node(const Ctx &c, int s) {
    return kAll ? s : c.node_of_slot[s];
}

template <bool kAll>
__device__ __forceinline__ int node_slot(const Ctx &c, int node) {
    return kAll ? node : c.slot_of_node[node];
}

template <bool kAll>
__device__ __forceinline__ int active_count(const Ctx &c) {
    return kAll ? c.nn : *c.n_active;
}

// 6-neighbourhood of slot s inside M (order -x, +x, -y, +y, -z, +z), -1 where absent.
template <bool kAll>
__device__ __forceinline__ void neighbours(const Ctx &c, int s, int nb[6]) {
    if (kAll) {
        int t, z;
        if (c.mdx) {  // multiply-high instead of two integer divisions
            t = (int)__umulhi(2u * (unsigned)s, c.mdx);
            z = (int)__umulhi(2u * (unsigned)t, c.mdy);
        } else {
            t = s / c.nx;
            z = t / c.ny;
        }
        const int x = s - t * c.nx, y = t - z * c.ny;
        const int pl = c.nx * c.ny;
        nb[0] = x > 0 ? s - 1 : -1;
        nb[1] = x + 1 < c.nx ? s + 1 : -1;
        nb[2] = y > 0 ? s - c.nx : -1;
        nb[3] = y + 1 < c.ny ? s + c.nx : -1;
        nb[4] = z > 0 ? s - pl : -1;
        nb[5] = z + 1 < c.nz ? s + pl : -1;
    } else {
#pragma unroll
        for (int d = 0; d < 6; d++) nb[d] = c.nbr[d * c.ld + s];
    }
}

__device__ __forceinline__ float3 ld3(const float *v, int ld, int i) {
    return make_float3(v[i], v[ld + i], v[2 * ld + i]);
}
__device__ __forceinline__ void st3(float *v, int ld, int i, float3 a) {
    v[i] = a.x;
    v[ld + i] = a.y;
    v[2 * ld + i] = a.z;
}

// BF16 x 4 storage (8 bytes) of a float4, round to nearest even
__device__ __forceinline__ uint2 pack_bf16x4(float4 v) {
    const __nv_bfloat162 lo = __floats2bfloat162_rn(v.x, v.y), hi = __floats2bfloat162_rn(v.z, v.w);
    return make_uint2(*reinterpret_cast<const unsigned *>(&lo), *reinterpret_cast<const unsigned *>(&hi));
}
__device__ __forceinline__ float4 unpack_bf16x4(uint2 u) {
    const float2 lo = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u.x));
    const float2 hi = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&u.y));
    return make_float4(lo.x, lo.y, hi.x, hi.y);
}
// per-sample association record (g', r0') and target normal, in the lattice's precision
__device__ __forceinline__ float4 load_rec(const Ctx &c, int j) {
    return c.mixed ? unpack_bf16x4(reinterpret_cast<const uint2 *>(c.rec)[j]) : c.rec[j];
}
__device__ __forceinline__ void store_rec(const Ctx &c, int j, float4 v) {
    if (c.mixed) reinterpret_cast<uint2 *>(c.rec)[j] = pack_bf16x4(v);
    else c.rec[j] = v;
}
__device__ __forceinline__ float4 load_nrm(const Ctx &c, size_t k) {
    return c.mixed ? unpack_bf16x4(reinterpret_cast<const uint2 *>(c.nrm)[k]) : c.nrm[k];
}

// ------------------------------------------------------------------ frame kernels

// Target normal of every pixel: cross product of the central differences of the
// back-projected depth map V(u, v) = D (u - cx, v - cy) / f (z = D), normalised and
// oriented towards the camera; invalid (w = 0) on the border or next to a hole.
// The differences are rearranged so that no two ~1 m values are subtracted:
//   x(u+1) - x(u-1) = [(D(u+1) - D(u-1)) (u - cx) + D(u+1) + D(u-1)] / fx.
__global__ void k_target_normals(const float *__restrict__ D, float4 *__restrict__ nrm, int W, int H,
                                 float fx, float fy, float cx, float cy, int mixed) {
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    const int v = blockIdx.y * blockDim.y + threadIdx.y;
    if (u >= W || v >= H) return;
    float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
    if (u >= 1 && v >= 1 && u + 1 < W && v + 1 < H) {
        const size_t k = (size_t)v * W + u;
        const float d0 = D[k], dl = D[k - 1], dr = D[k + 1], du = D[k - W], dd = D[k + W];
        if (d0 > 0.f && dl > 0.f && dr > 0.f && du > 0.f && dd > 0.f) {
            const float a = (float)u - cx, b = (float)v - cy;
            const float dh = dr - dl, dv = dd - du;
            const float ex = (dh * a + (dr + dl)) / fx, ey = dh * b / fy, ez = dh;
            const float gx = dv * a / fx, gy = (dv * b + (dd + du)) / fy, gz = dv;
            float n0 = ey * gz - ez * gy, n1 = ez * gx - ex * gz, n2 = ex * gy - ey * gx;
            const float L2 = n0 * n0 + n1 * n1 + n2 * n2;
            if (L2 > 0.f) {
                const float inv = 1.0f / sqrtf(L2);
                n0 *= inv;
                n1 *= inv;
                n2 *= inv;
                if (n0 * (a / fx) + n1 * (b / fy) + n2 > 0.f) {
                    n0 = -n0;
                    n1 = -n1;
                    n2 = -n2;
                }
                out = make_float4(n0, n1, n2, 1.f);
            }
        }
    }
    if (mixed) reinterpret_cast<uint2 *>(nrm)[(size_t)v * W + u] = pack_bf16x4(out);
    else nrm[(size_t)v * W + u] = out;
}

// A depth that is not a positive finite number marks an invalid pixel, as 0 does: such
// entries are set to 0 before any kernel reads the map.
__global__ void k_sanitize_depth(float *__restrict__ D, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float d = D[i];
        if (!(d > 0.f) || !isfinite(d)) D[i] = 0.f;
    }
}

// Cell of each point (lower-corner node, or -1 when the cell is not inside the
// lattice) and its trilinear fractions.  The floor decision is taken in FP64 on
// (p - origin) / h, so it does not depend on FP32 rounding.  With normals given, a
// point whose normal is not finite gets -1 too (it is ignored, like one outside).
__global__ void k_point_cells(const float *__restrict__ pts, int n, Ctx c, int *__restrict__ cell,
                              float4 *__restrict__ frac, const float *__restrict__ nrm = nullptr) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const double o[3] = {(double)c.ox, (double)c.oy, (double)c.oz};
        const int dims[3] = {c.nx, c.ny, c.nz};
        double f[3];
        int ci[3];
        bool ok = true;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const double q = __ddiv_rn(__dsub_rn((double)pts[3 * i + a], o[a]), (double)c.h);
            const double fl = floor(q);
            if (!(fl >= 0.0) || fl > (double)(dims[a] - 2)) ok = false;
            ci[a] = ok ? (int)fl : 0;
            f[a] = q - fl;
        }
        if (nrm && !(isfinite(nrm[3 * i]) && isfinite(nrm[3 * i + 1]) && isfinite(nrm[3 * i + 2]))) ok = false;
        if (c.dom_h > 0.f) {  // gathered from the finest level: its cell must exist there
#pragma unroll
            for (int a = 0; a < 3; a++) {
                const double fl = floor(__ddiv_rn(__dsub_rn((double)pts[3 * i + a], o[a]), (double)c.dom_h));
                if (!(fl >= 0.0) || fl > (double)(c.dom_n[a] - 2)) ok = false;
            }
        }
        cell[i] = ok ? ci[0] + c.nx * (ci[1] + c.ny * ci[2]) : -1;
        frac[i] = make_float4((float)f[0], (float)f[1], (float)f[2], 0.f);
    }
}

__global__ void k_histogram(const int *__restrict__ cell, int n, int *__restrict__ cnt) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if (cell[i] >= 0) atomicAdd(&cnt[cell[i]], 1);
}

// ---- exclusive scan of int arrays (3 passes: 4096-element tiles, tile sums, add)
constexpr int kScanThreads = 1024, kScanPer = 4, kScanTile = kScanThreads * kScanPer;

__device__ __forceinline__ int block_exclusive_scan(int v, int *total) {
    __shared__ int ws[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(FULL, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int s = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(FULL, s, o);
            if (lane >= o) s += y;
        }
        ws[lane] = s;
    }
    __syncthreads();
    const int before = (wid > 0 ? ws[wid - 1] : 0) + x - v;
    if (total) *total = ws[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before;
}

// out[i] = sum_{j < i} in[i] for i < n; tile sums to sums[blockIdx.x]
__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const int *__restrict__ in, int n,
                                                             int *__restrict__ out, int *__restrict__ sums) {
    const int base = blockIdx.x * kScanTile + threadIdx.x * kScanPer;
    int v[kScanPer], s = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; k++) {
        v[k] = (base + k < n) ? in[base + k] : 0;
        s += v[k];
    }
    int total;
    int run = block_exclusive_scan(s, &total);
#pragma unroll
    for (int k = 0; k < kScanPer; k++) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// single block: exclusive scan of the tile sums (at most kScanTile of them); the
// grand total goes to out_total
__global__ void __launch_bounds__(kScanThreads) k_scan_sums(int *__restrict__ sums, int nt, int *__restrict__ out_total) {
    const int base = threadIdx.x * kScanPer;
    int v[kScanPer], s = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; k++) {
        v[k] = (base + k < nt) ? sums[base + k] : 0;
        s += v[k];
    }
    int total;
    int run = block_exclusive_scan(s, &total);
#pragma unroll
    for (int k = 0; k < kScanPer; k++) {
        if (base + k < nt) sums[base + k] = run;
        run += v[k];
    }
    if (threadIdx.x == 0) *out_total = total;
}

__global__ void k_scan_add(int *__restrict__ out, int n, const int *__restrict__ sums) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += sums[i / kScanTile];
}

// Counting-sort scatter: each valid sample takes a slot in its cell's range.
__global__ void k_bin_scatter(const int *__restrict__ cell, int n, const int *__restrict__ start,
                              int *__restrict__ cnt, int *__restrict__ tmp) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int cl = cell[i];
        if (cl < 0) continue;
        const int pos = start[cl] + atomicSub(&cnt[cl], 1) - 1;
        tmp[pos] = i;
    }
}

// Deterministic order inside each cell: rank by original index.
__global__ void k_bin_rank(const int *__restrict__ tmp, const int *__restrict__ cell,
                           const int *__restrict__ start, const int *__restrict__ total,
                           int *__restrict__ order) {
    const int n = *total;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int c0 = tmp[i], cl = cell[c0];
        const int beg = start[cl], end = start[cl + 1];
        int rank = 0;
        for (int j = beg; j < end; j++) rank += tmp[j] < c0;
        order[beg + rank] = c0;
    }
}

// Gather the samples into sorted order; mark the first sample of every cell.
__global__ void k_bin_gather(const int *__restrict__ order, const int *__restrict__ total,
                             const float *__restrict__ pts, const float *__restrict__ nrms,
                             const int *__restrict__ cell, const float4 *__restrict__ frac,
                             float4 *__restrict__ sp, float4 *__restrict__ sn, int *__restrict__ scell,
                             float4 *__restrict__ sfrac, int *__restrict__ perm, int *__restrict__ head) {
    const int n = *total;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int c0 = order[i];
        sp[i] = make_float4(pts[3 * c0], pts[3 * c0 + 1], pts[3 * c0 + 2], 0.f);
        sn[i] = make_float4(nrms[3 * c0], nrms[3 * c0 + 1], nrms[3 * c0 + 2], 0.f);
        scell[i] = cell[c0];
        sfrac[i] = frac[c0];
        perm[i] = c0;
        head[i] = (i == 0 || cell[order[i - 1]] != cell[c0]) ? 1 : 0;
    }
}

__global__ void k_occupied(const int *__restrict__ head, const int *__restrict__ hscan,
                           const int *__restrict__ total, const int *__restrict__ scell,
                           const int *__restrict__ n_occ, int *__restrict__ occ_cell, int *__restrict__ occ_beg) {
    const int n = *total;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if (head[i]) {
            occ_cell[hscan[i]] = scell[i];
            occ_beg[hscan[i]] = i;
        }
    if (blockIdx.x == 0 && threadIdx.x == 0) occ_beg[*n_occ] = n;
}

// ---- active set M (surface mode): corners of occupied cells, then their one-ring
__global__ void k_mark_cells(const int *__restrict__ occ_cell, const int *__restrict__ n_occ,
                             const int *__restrict__ scell, int S, Ctx c, int *__restrict__ mark) {
    const int no = *n_occ;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < no + S; i += gridDim.x * blockDim.x) {
        const int cl = i < no ? occ_cell[i] : scell[i - no];
        if (cl < 0) continue;
#pragma unroll
        for (int k = 0; k < 8; k++) mark[corner_node(c, cl, k)] = 1;
    }
}

__global__ void k_dilate(const int *__restrict__ mark, Ctx c, int *__restrict__ act) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < c.nn; i += gridDim.x * blockDim.x) {
        const int x = i % c.nx, t = i / c.nx, y = t % c.ny, z = t / c.ny, pl = c.nx * c.ny;
        int on = mark[i];
        on |= (x > 0 && mark[i - 1]) | (x + 1 < c.nx && mark[i + 1]);
        on |= (y > 0 && mark[i - c.nx]) | (y + 1 < c.ny && mark[i + c.nx]);
        on |= (z > 0 && mark[i - pl]) | (z + 1 < c.nz && mark[i + pl]);
        act[i] = on ? 1 : 0;
    }
}

// slot_of_node holds the exclusive scan of act on entry; -1 for nodes outside M after.
__global__ void k_compact(const int *__restrict__ act, Ctx c, int *__restrict__ slot_of_node,
                          int *__restrict__ node_of_slot) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < c.nn; i += gridDim.x * blockDim.x) {
        if (act[i]) node_of_slot[slot_of_node[i]] = i;
        else slot_of_node[i] = -1;
    }
}

__global__ void k_neighbour_table(Ctx c, int *__restrict__ nbr) {
    const int N = *c.n_active;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < N; s += gridDim.x * blockDim.x) {
        const int i = c.node_of_slot[s];
        const int x = i % c.nx, t = i / c.nx, y = t % c.ny, z = t / c.ny, pl = c.nx * c.ny;
        const int nd[6] = {x > 0 ? i - 1 : -1, x + 1 < c.nx ? i + 1 : -1, y > 0 ? i - c.nx : -1,
                           y + 1 < c.ny ? i + c.nx : -1, z > 0 ? i - pl : -1, z + 1 < c.nz ? i + pl : -1};
#pragma unroll
        for (int d = 0; d < 6; d++) nbr[d * c.ld + s] = nd[d] >= 0 ? c.slot_of_node[nd[d]] : -1;
    }
}

// Slots touched by the samples' or sparse pairs' J^T J contributions (corners of their
// cells), flagged for the persistent position step (which folds their q per flag).
template <bool kAll>
__global__ void k_mark_surface(const int *__restrict__ occ_cell, const int *__restrict__ n_occ,
                               const int *__restrict__ scell, int S, Ctx c, int *__restrict__ flag) {
    const int no = *n_occ;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < no + S; i += gridDim.x * blockDim.x) {
        const int cl = i < no ? occ_cell[i] : scell[i - no];
        if (cl < 0) continue;
#pragma unroll
        for (int k = 0; k < 8; k++) flag[node_slot<kAll>(c, corner_node(c, cl, k))] = 1;
    }
}


// ------------------------------------------------------------------ association (Sec. 5.1)

template <typename T>
struct V3 {
    T x, y, z;
};

template <typename T>
__device__ __forceinline__ T dot(const V3<T> &a, const V3<T> &b) {
    return a.x * b.x + a.y * b.y + a.z * b.z;
}

template <typename T>
__device__ __forceinline__ V3<T> rot(const float *M, const V3<T> &v) {  // row-major 3x3
    return {T(M[0]) * v.x + T(M[1]) * v.y + T(M[2]) * v.z, T(M[3]) * v.x + T(M[4]) * v.y + T(M[5]) * v.z,
            T(M[6]) * v.x + T(M[7]) * v.y + T(M[8]) * v.z};
}

template <typename T>
__device__ __forceinline__ V3<T> rotT(const float *M, const V3<T> &v) {
    return {T(M[0]) * v.x + T(M[3]) * v.y + T(M[6]) * v.z, T(M[1]) * v.x + T(M[4]) * v.y + T(M[7]) * v.z,
            T(M[2]) * v.x + T(M[5]) * v.y + T(M[8]) * v.z};
}

__device__ __forceinline__ double depth_at(const Ctx &c, int px, int py) {
    return (double)c.depth[(size_t)py * c.W + px];
}

// Target normal in FP64 from the depth map (plain central differences of V, with
// V(d, u, v) = d ((u - c_x) / f_x, (v - c_y) / f_y, 1); rfx, rfy = 1 / f_x, 1 / f_y).
__device__ bool target_normal_f64(const Ctx &c, int px, int py, double rfx, double rfy, V3<double> &n) {
    if (px < 1 || py < 1 || px + 1 >= c.W || py + 1 >= c.H) return false;
    const double d0 = depth_at(c, px, py), dl = depth_at(c, px - 1, py), dr = depth_at(c, px + 1, py);
    const double du = depth_at(c, px, py - 1), dd = depth_at(c, px, py + 1);
    if (!(d0 > 0 && dl > 0 && dr > 0 && du > 0 && dd > 0)) return false;
    const double cx = c.cx, cy = c.cy;
    auto V = [&](double d, int uu, int vv) { return V3<double>{d * ((uu - cx) * rfx), d * ((vv - cy) * rfy), d}; };
    const V3<double> a = V(dr, px + 1, py), b = V(dl, px - 1, py), e = V(dd, px, py + 1), f = V(du, px, py - 1);
    const V3<double> ex{a.x - b.x, a.y - b.y, a.z - b.z}, ey{e.x - f.x, e.y - f.y, e.z - f.z};
    V3<double> m{ex.y * ey.z - ex.z * ey.y, ex.z * ey.x - ex.x * ey.z, ex.x * ey.y - ex.y * ey.x};
    const double L2 = dot(m, m);
    if (!(L2 > 0)) return false;
    const double iL = 1.0 / sqrt(L2);
    m = {m.x * iL, m.y * iL, m.z * iL};
    const V3<double> P = V(d0, px, py);
    if (dot(m, P) > 0) m = {-m.x, -m.y, -m.z};
    n = m;
    return true;
}

// The per-sample record from the target point p^a, target normal n^a and weight w_c:
//   g' = sqrt(w_c) R_g^T n^a,  r0' = sqrt(w_c) n^a . (R_g p^ + t_g - p^a)  (r0' in FP64)
template <typename T>
__device__ __forceinline__ float4 sample_record(const Ctx &c, const float4 p4, const V3<T> &na, const V3<T> &pa,
                                                T sw) {
    const V3<T> gt = rotT<T>(c.Rg, na);
    const V3<double> nad{(double)na.x, (double)na.y, (double)na.z};
    V3<double> q0 = rot<double>(c.Rg, V3<double>{(double)p4.x, (double)p4.y, (double)p4.z});
    q0.x += (double)c.tg[0] - (double)pa.x;
    q0.y += (double)c.tg[1] - (double)pa.y;
    q0.z += (double)c.tg[2] - (double)pa.z;
    const double r0 = (double)sw * dot(nad, q0);
    return make_float4((float)(sw * gt.x), (float)(sw * gt.y), (float)(sw * gt.z), (float)r0);
}

// The association of one sample from its corner sums du = sum alpha_k u_k and
// dn = sum alpha_k R_k n^ (Sec. 5.1): warped point and model normal, nearest pixel,
// target point and normal, Phi_d, Phi_n, Phi_v, w_c and the record.  In FP32, with
// the target normal from the precomputed map; returns true when a decision (pixel,
// range, any Phi < 0) lies within a margin of its threshold that FP32 rounding could
// cross, and the sample is then associated again by associate_finish_f64.
__device__ bool associate_finish_f32(const Ctx &c, const float4 p4, V3<float> du, V3<float> dn, int &pix,
                                     float &w_out, float4 &rec) {
    pix = -1;
    w_out = 0.f;
    rec = make_float4(0.f, 0.f, 0.f, 0.f);
    const V3<float> q{p4.x + du.x, p4.y + du.y, p4.z + du.z};
    V3<float> p = rot<float>(c.Rg, q);
    p.x += c.tg[0];
    p.y += c.tg[1];
    p.z += c.tg[2];
    V3<float> n = rot<float>(c.Rg, dn);
    const float nl = sqrtf(dot(n, n));
    bool near = false;
    if (!(nl > 0.f)) return false;
    n = {n.x / nl, n.y / nl, n.z / nl};
    if (fabs((double)p.z) < 1e-4) near = true;
    if (!(p.z > 0.f)) return near;
    const float uf = c.fx * p.x / p.z + c.cx + 0.5f;
    const float vf = c.fy * p.y / p.z + c.cy + 0.5f;
    const float pxf = floorf(uf), pyf = floorf(vf);
    const float mu = uf - pxf, mv = vf - pyf;
    if (mu < 2e-3f || mu > 1.f - 2e-3f || mv < 2e-3f || mv > 1.f - 2e-3f) near = true;
    if (!(pxf >= 0.f && pxf < (float)c.W && pyf >= 0.f && pyf < (float)c.H)) return near;
    const int px = (int)pxf, py = (int)pyf;
    const size_t k = (size_t)py * c.W + px;
    const float D = c.depth[k];
    if (!(D > 0.f)) return near;
    const float4 m4 = load_nrm(c, k);
    if (m4.w == 0.f) return near;
    const V3<float> na{m4.x, m4.y, m4.z};
    const V3<float> pa{D * ((px - c.cx) / c.fx), D * ((py - c.cy) / c.fy), D};
    const V3<float> dd{p.x - pa.x, p.y - pa.y, p.z - pa.z};
    const float dist = sqrtf(dot(dd, dd));
    const float cn = dot(n, na);
    const float pl = sqrtf(dot(p, p));
    const float cv = -dot(n, p) / pl;
    if (fabsf(dist - c.eps_d) < 1e-5f) near = true;
    // BF16 target normals carry up to ~4e-3 of rounding in n_c . n^a
    if (fabsf((1.f - cn) - c.eps_n) < (c.mixed ? 1e-2f : 1e-4f)) near = true;
    if (fabsf((1.f - cv) - c.eps_v) < 1e-4f) near = true;
    pix = (int)k;
    const float phi_d = 1.f - dist / c.eps_d;
    const float phi_n = 1.f - (1.f - cn) / c.eps_n;
    const float phi_v = 1.f - (1.f - cv) / c.eps_v;
    if (phi_d < 0.f || phi_n < 0.f || phi_v < 0.f) return near;
    const float m = (phi_d + phi_n + phi_v) / 3.f;
    const float w = m * m;
    w_out = w;
    rec = sample_record<float>(c, p4, na, pa, sqrtf(w));
    return near;
}

// The same association in FP64, with the target normal from the depth map in FP64.
// Quotients with a common divisor share one reciprocal (one rounding more than a
// division: the decisions move only for values within a few units in the last place
// of a threshold, where FP64 rounding decides anyway).
__device__ void associate_finish_f64(const Ctx &c, const float4 p4, V3<double> du, V3<double> dn, int &pix,
                                     float &w_out, float4 &rec) {
    pix = -1;
    w_out = 0.f;
    rec = make_float4(0.f, 0.f, 0.f, 0.f);
    const V3<double> q{p4.x + du.x, p4.y + du.y, p4.z + du.z};
    V3<double> p = rot<double>(c.Rg, q);
    p.x += (double)c.tg[0];
    p.y += (double)c.tg[1];
    p.z += (double)c.tg[2];
    V3<double> n = rot<double>(c.Rg, dn);
    const double nl2 = dot(n, n);
    if (!(nl2 > 0.0)) return;
    const double inl = 1.0 / sqrt(nl2);
    n = {n.x * inl, n.y * inl, n.z * inl};
    if (!(p.z > 0.0)) return;
    const double iz = 1.0 / p.z;
    const double uf = (double)c.fx * p.x * iz + (double)c.cx + 0.5;
    const double vf = (double)c.fy * p.y * iz + (double)c.cy + 0.5;
    const double pxf = floor(uf), pyf = floor(vf);
    if (!(pxf >= 0.0 && pxf < (double)c.W && pyf >= 0.0 && pyf < (double)c.H)) return;
    const int px = (int)pxf, py = (int)pyf;
    const size_t k = (size_t)py * c.W + px;
    const float D = c.depth[k];
    if (!(D > 0.f)) return;
    const double rfx = 1.0 / (double)c.fx, rfy = 1.0 / (double)c.fy;
    V3<double> na;
    if (!target_normal_f64(c, px, py, rfx, rfy, na)) return;
    const double Dd = D;
    const V3<double> pa{Dd * ((px - (double)c.cx) * rfx), Dd * ((py - (double)c.cy) * rfy), Dd};
    const V3<double> dd{p.x - pa.x, p.y - pa.y, p.z - pa.z};
    const double dist = sqrt(dot(dd, dd));
    const double cn = dot(n, na);
    const double cv = -dot(n, p) / sqrt(dot(p, p));
    pix = (int)k;
    const double phi_d = 1.0 - dist / (double)c.eps_d;
    const double phi_n = 1.0 - (1.0 - cn) / (double)c.eps_n;
    const double phi_v = 1.0 - (1.0 - cv) / (double)c.eps_v;
    if (phi_d < 0.0 || phi_n < 0.0 || phi_v < 0.0) return;
    const double m = (phi_d + phi_n + phi_v) / 3.0;
    const double w = m * m;
    w_out = (float)w;
    rec = sample_record<double>(c, p4, na, pa, sqrt(w));
}

// FP32 trilinear weights of sample i in its cell (precomputed per frame)
__device__ __forceinline__ void sample_frac_f32(const Ctx &c, int i, float f[3]) {
    const float4 f4 = c.frac[i];
    f[0] = f4.x;
    f[1] = f4.y;
    f[2] = f4.z;
}

// FP64 trilinear weights of sample i in its cell cl, from its position
__device__ __forceinline__ void sample_frac_f64(const Ctx &c, int cl, const float4 p4, double f[3]) {
    const int cx_ = cl % c.nx, t = cl / c.nx, cy_ = t % c.ny, cz_ = t / c.ny;
    f[0] = ((double)p4.x - (double)c.ox) / (double)c.h - cx_;
    f[1] = ((double)p4.y - (double)c.oy) / (double)c.h - cy_;
    f[2] = ((double)p4.z - (double)c.oz) / (double)c.h - cz_;
}

// Association of sorted sample i at the current warp in FP32 (see associate_finish_f32)
__device__ bool associate_sample_f32(const Ctx &c, int i, int &pix, float &w_out, float4 &rec) {
    const int cl = c.cell[i];
    const float4 p4 = c.sp[i], n4 = c.sn[i];
    float f[3];
    sample_frac_f32(c, i, f);
    V3<float> du{0.f, 0.f, 0.f}, dn{0.f, 0.f, 0.f};
    const V3<float> nh{n4.x, n4.y, n4.z};
#pragma unroll
    for (int k = 0; k < 8; k++) {
        const int node = corner_node(c, cl, k);
        const float al = trilinear_weight(f, k);
        du.x += al * c.u[node];
        du.y += al * c.u[c.ld + node];
        du.z += al * c.u[2 * c.ld + node];
        float Rk[9];
#pragma unroll
        for (int e = 0; e < 9; e++) Rk[e] = c.R[e * c.ld + node];
        const V3<float> rn = rot<float>(Rk, nh);
        dn.x += al * rn.x;
        dn.y += al * rn.y;
        dn.z += al * rn.z;
    }
    return associate_finish_f32(c, p4, du, dn, pix, w_out, rec);
}

// Four lanes per sample: lane k of a quad gathers corners k and k + 4 (u and R), the quad
// adds its corner sums by shuffles, and lane 0 finishes the association (a sample's
// 96 gathered values spread over four threads: four times the loads in flight per SM).
template <bool kAll>
__global__ void __launch_bounds__(kThreads) k_associate(Ctx c, Scal *sc) {
    pdl_wait();
    pdl_trigger();
    if (sc->skip) return;
    const int n = *c.n_samples;
    int valid = 0, refined = 0;
    const int q = threadIdx.x & 3;
    const int nq = (gridDim.x * blockDim.x) >> 2;
    // the loop bound is the warp's first sample: uniform in the warp (shuffles)
    const int first = (blockIdx.x * blockDim.x + (threadIdx.x & ~31)) >> 2;
    for (int i0 = first; i0 < n; i0 += nq) {
        const int i = i0 + ((threadIdx.x & 31) >> 2);
        const bool has = i < n;
        V3<float> du{0.f, 0.f, 0.f}, dn{0.f, 0.f, 0.f};
        float4 p4 = make_float4(0.f, 0.f, 0.f, 0.f);
        if (has) {
            const int cl = c.cell[i];
            const float4 n4 = c.sn[i];
            p4 = c.sp[i];
            float f[3];
            sample_frac_f32(c, i, f);
            const V3<float> nh{n4.x, n4.y, n4.z};
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const int k = q + 4 * h;
                const int node = corner_node(c, cl, k);
                const float al = trilinear_weight(f, k);
                du.x += al * c.u[node];
                du.y += al * c.u[c.ld + node];
                du.z += al * c.u[2 * c.ld + node];
                float Rk[9];
#pragma unroll
                for (int e = 0; e < 9; e++) Rk[e] = c.R[e * c.ld + node];
                const V3<float> rn = rot<float>(Rk, nh);
                dn.x += al * rn.x;
                dn.y += al * rn.y;
                dn.z += al * rn.z;
            }
        }
#pragma unroll
        for (int o = 1; o < 4; o <<= 1) {
            du.x += __shfl_xor_sync(FULL, du.x, o);
            du.y += __shfl_xor_sync(FULL, du.y, o);
            du.z += __shfl_xor_sync(FULL, du.z, o);
            dn.x += __shfl_xor_sync(FULL, dn.x, o);
            dn.y += __shfl_xor_sync(FULL, dn.y, o);
            dn.z += __shfl_xor_sync(FULL, dn.z, o);
        }
        if (!has || q != 0) continue;
        int pix;
        float w;
        float4 rec;
        const bool near = associate_finish_f32(c, p4, du, dn, pix, w, rec);
        if (near) {  // re-taken in FP64 by k_associate_refine (and counted there)
            c.refine[atomicAdd(&sc->n_refine, 1)] = i;
            refined++;
            continue;
        }
        c.pix[i] = pix;
        c.wc[i] = w;
        store_rec(c, i, rec);
        valid += w > 0.f;
    }
    block_add_int(valid, &sc->n_valid);
    block_add_int(refined, &sc->n_refined);
    if (blockIdx.x == 0 && threadIdx.x == 0) sc->assoc_ran = 1;
}

// The samples k_associate found near a threshold, associated again in FP64: eight lanes
// per sample gather the corner sums (one corner each, FP64 shuffles), lane 0 finishes.
// A warp takes four consecutive list entries and the warps go to different blocks
// first, so that a short list puts one warp on each SM and no two share an FP64 pipe.
// Block `bid` of `nb` blocks on the list.
template <bool kAll>
__device__ __forceinline__ void associate_refine_block(const Ctx &c, Scal *sc, int bid, int nb) {
    const int n = sc->n_refine;
    int valid = 0;
    const int k = threadIdx.x & 7;
    const int warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int wg = warp * nb + bid;                    // this warp's rank among all warps
    const int per_round = 4 * nwarp * nb;
    for (int g0 = 4 * wg; g0 < n; g0 += per_round) {  // the warp's loop bound is uniform
        const int g = g0 + ((threadIdx.x & 31) >> 3);
        V3<double> du{0.0, 0.0, 0.0}, dn{0.0, 0.0, 0.0};
        int i = -1;
        float4 p4 = make_float4(0.f, 0.f, 0.f, 0.f);
        if (g < n) {
            i = c.refine[g];
            const int cl = c.cell[i];
            const float4 n4 = c.sn[i];
            p4 = c.sp[i];
            double f[3];
            sample_frac_f64(c, cl, p4, f);
            const int node = corner_node(c, cl, k);
            const double al = trilinear_weight(f, k);
            du = {al * (double)c.u[node], al * (double)c.u[c.ld + node], al * (double)c.u[2 * c.ld + node]};
            float Rk[9];
#pragma unroll
            for (int e = 0; e < 9; e++) Rk[e] = c.R[e * c.ld + node];
            const V3<double> rn = rot<double>(Rk, V3<double>{(double)n4.x, (double)n4.y, (double)n4.z});
            dn = {al * rn.x, al * rn.y, al * rn.z};
        }
        // butterfly over the eight corner lanes (FP64: its order moves the sums by rounding only)
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            du.x += __shfl_xor_sync(FULL, du.x, o);
            du.y += __shfl_xor_sync(FULL, du.y, o);
            du.z += __shfl_xor_sync(FULL, du.z, o);
            dn.x += __shfl_xor_sync(FULL, dn.x, o);
            dn.y += __shfl_xor_sync(FULL, dn.y, o);
            dn.z += __shfl_xor_sync(FULL, dn.z, o);
        }
        if (k == 0 && g < n) {
            int pix;
            float w;
            float4 rec;
            associate_finish_f64(c, p4, du, dn, pix, w, rec);
            c.pix[i] = pix;
            c.wc[i] = w;
            store_rec(c, i, rec);
            valid += w > 0.f;
        }
    }
    block_add_int(valid, &sc->n_valid);
}

template <bool kAll>
__global__ void __launch_bounds__(kThreads) k_associate_refine(Ctx c, Scal *sc) {
    pdl_wait();
    pdl_trigger();
    if (sc->skip) return;
    associate_refine_block<kAll>(c, sc, blockIdx.x, gridDim.x);
}

// ------------------------------------------------------------------ per-cell sample passes

enum CellOp { kOpRhs = 0, kOpApply = 1, kOpEnergy = 2 };

// Sample passes over the occupied cells.  A block takes a slice of cells [cb, ce) and
// their (contiguous, cell-sorted) samples in two phases per chunk of blockDim samples:
//   1. one thread per sample: s = g' . sum_k alpha_k v_k over the 8 corners, and the
//      per-sample factor t (kept in shared memory);
//   2. one thread per (cell, corner): sum_j alpha_k(j) g'_j t_j over the cell's samples,
//      then one atomic per component.
// vec is the slot-indexed p (kOpApply) or the node-indexed u (kOpRhs / kOpEnergy).
//   kOpRhs:    t = -w_d (s + r0'):  r_k += alpha_k g' t,  diag_k += alpha_k^2 w_d g'^2
//   kOpApply:  t = w_d s:           q_k += alpha_k g' t,  part += t s      (= p.J^T J p)
//   kOpEnergy: part += (s + r0')^2  (E_dense, phase 1 only)
// kFresh reads vec through L2 (it was written by other CTAs of the same grid).
template <bool kFresh>
__device__ __forceinline__ float ldv(const float *p) {
    return kFresh ? __ldcg(p) : *p;
}

// The vector a sample pass reads: vec[i], or (inside the persistent position step, where
// p is formed on the fly) fma(beta, pold[i], vec[i]) with vec = z.
struct VecView {
    const float *vec;
    const float *pold;  // nullptr: plain vec
    float beta;
};

template <bool kFresh>
__device__ __forceinline__ float ldvv(const VecView &v, size_t i) {
    const float a = ldv<kFresh>(v.vec + i);
    return v.pold ? fmaf(v.beta, ldv<kFresh>(v.pold + i), a) : a;
}

// Where the sample passes of the persistent position step find a node's entries in the
// vectors they read and add to (kMap): at x + lx (y + ny z), plane stride ld -- the layout
// of the published vectors of a padded brick, whose rows of lx slots keep every float4
// group aligned; otherwise (!kMap) at the node's slot with plane stride c.ld.
struct SlotMap {
    int lx;
    unsigned m_nx;  // n / nx as (2n m_nx) >> 32, exact for n nx < 2^31
    size_t ld;
};

template <bool kAll, bool kMap>
__device__ __forceinline__ int map_corner(const Ctx &c, const SlotMap &m, int cell, int k) {
    if constexpr (!kMap) {
        return node_slot<kAll>(c, corner_node(c, cell, k));
    } else {
        const int pc = cell + (m.lx - c.nx) * (int)__umulhi(2u * (unsigned)cell, m.m_nx);
        return pc + (k & 1) + m.lx * (((k >> 1) & 1) + c.ny * ((k >> 2) & 1));
    }
}

template <bool kMap>
__device__ __forceinline__ size_t map_ld(const Ctx &c, const SlotMap &m) {
    return kMap ? m.ld : (size_t)c.ld;
}

// synchronise the threads running a cells_block: the whole block (bar_id 0) or the
// nt threads of named barrier bar_id
__device__ __forceinline__ void sub_sync(int bar_id, int nt) {
    if (bar_id == 0) __syncthreads();
    else asm volatile("bar.sync %0, %1;" ::"r"(bar_id), "r"(nt) : "memory");
}

template <int kOp, bool kAll, bool kFresh>
__device__ __forceinline__ void cells_block(const Ctx &c, const VecView vec, float *dst, float *dst2, int cb, int ce,
                                            float *tsm, int tsm_cap, float &part, int lt, int nt, int bar_id,
                                            int js = 0, int je = 0x7fffffff) {
    // the samples of cells [cb, ce), clipped to [js, je) (a cell may be shared with the
    // neighbouring range: each range adds its own samples' contributions)
    const int sb = max(c.occ_beg[cb], js), se = min(c.occ_beg[ce], je);
    const int items = kOp == kOpEnergy ? 1 : (ce - cb) * 8;
    if (kOp != kOpEnergy && se - sb <= tsm_cap) {
        // all the samples' factors fit in shared memory (tsm_cap of them; a thread forms
        // those of samples lt, lt + nt, ...): phase 1 once, then every round of (cell,
        // corner) items reads the same factors
        for (int j = sb + lt; j < se; j += nt) {
            const int ls = j - sb;
            const int cl = c.cell[j];
            const float4 f4 = c.frac[j], g = load_rec(c, j);
            const float f[3] = {f4.x, f4.y, f4.z};
            float sx = 0.f, sy = 0.f, sz = 0.f;
#pragma unroll
            for (int kk = 0; kk < 8; kk++) {
                const int nd = corner_node(c, cl, kk);
                const int vi = (kOp == kOpApply) ? node_slot<kAll>(c, nd) : nd;
                const float al = trilinear_weight(f, kk);
                sx += al * ldvv<kFresh>(vec, vi);
                sy += al * ldvv<kFresh>(vec, c.ld + vi);
                sz += al * ldvv<kFresh>(vec, 2 * (size_t)c.ld + vi);
            }
            const float sv = g.x * sx + g.y * sy + g.z * sz;
            if (kOp == kOpApply) {
                const float t = c.w_d * sv;
                part += t * sv;
                tsm[ls] = t;
            } else {
                tsm[ls] = -c.w_d * (sv + g.w);
            }
        }
        sub_sync(bar_id, nt);
        for (int item = lt; item < items; item += nt) {
            const int ci = cb + (item >> 3), k = item & 7;
            const int ibeg = max(c.occ_beg[ci], js), iend = min(c.occ_beg[ci + 1], je);
            float ax = 0.f, ay = 0.f, az = 0.f, dx = 0.f, dy = 0.f, dz = 0.f;
            for (int jj = ibeg; jj < iend; jj++) {
                const float4 f4 = c.frac[jj], g = load_rec(c, jj);
                const float f[3] = {f4.x, f4.y, f4.z};
                const float al = trilinear_weight(f, k);
                const float t = al * tsm[jj - sb];
                ax += g.x * t;
                ay += g.y * t;
                az += g.z * t;
                if (kOp == kOpRhs) {
                    const float a2 = al * al * c.w_d;
                    dx += a2 * g.x * g.x;
                    dy += a2 * g.y * g.y;
                    dz += a2 * g.z * g.z;
                }
            }
            const int sl = node_slot<kAll>(c, corner_node(c, c.occ_cell[ci], k));
            if (ax != 0.f) atomicAdd(&dst[sl], ax);
            if (ay != 0.f) atomicAdd(&dst[c.ld + sl], ay);
            if (az != 0.f) atomicAdd(&dst[2 * c.ld + sl], az);
            if (kOp == kOpRhs) {
                if (dx != 0.f) atomicAdd(&dst2[sl], dx);
                if (dy != 0.f) atomicAdd(&dst2[c.ld + sl], dy);
                if (dz != 0.f) atomicAdd(&dst2[2 * c.ld + sl], dz);
            }
        }
        sub_sync(bar_id, nt);  // tsm is free again
        return;
    }
    for (int i0 = 0; i0 < items; i0 += nt) {
        const int item = i0 + lt;
        const bool has = kOp != kOpEnergy && item < items;
        const int ci = cb + (has ? item >> 3 : 0), k = item & 7;
        const int ibeg = has ? max(c.occ_beg[ci], js) : 0, iend = has ? min(c.occ_beg[ci + 1], je) : 0;
        float ax = 0.f, ay = 0.f, az = 0.f, dx = 0.f, dy = 0.f, dz = 0.f;
        for (int j0 = sb; j0 < se; j0 += nt) {
            const int j = j0 + lt;
            if (j < se) {
                const int cl = c.cell[j];
                const float4 f4 = c.frac[j], g = load_rec(c, j);
                const float f[3] = {f4.x, f4.y, f4.z};
                float sx = 0.f, sy = 0.f, sz = 0.f;
#pragma unroll
                for (int kk = 0; kk < 8; kk++) {
                    const int nd = corner_node(c, cl, kk);
                    const int vi = (kOp == kOpApply) ? node_slot<kAll>(c, nd) : nd;
                    const float al = trilinear_weight(f, kk);
                    sx += al * ldvv<kFresh>(vec, vi);
                    sy += al * ldvv<kFresh>(vec, c.ld + vi);
                    sz += al * ldvv<kFresh>(vec, 2 * (size_t)c.ld + vi);
                }
                const float sv = g.x * sx + g.y * sy + g.z * sz;
                if (kOp == kOpApply) {
                    const float t = c.w_d * sv;
                    if (i0 == 0) part += t * sv;
                    tsm[lt] = t;
                } else if (kOp == kOpRhs) {
                    tsm[lt] = -c.w_d * (sv + g.w);
                } else {
                    const float e = sv + g.w;
                    part += e * e;
                }
            }
            if (kOp == kOpEnergy) continue;
            sub_sync(bar_id, nt);
            if (has) {
                const int lo = max(ibeg, j0), hi = min(iend, j0 + nt);
                for (int jj = lo; jj < hi; jj++) {
                    const float4 f4 = c.frac[jj], g = load_rec(c, jj);
                    const float f[3] = {f4.x, f4.y, f4.z};
                    const float al = trilinear_weight(f, k);
                    const float t = al * tsm[jj - j0];
                    ax += g.x * t;
                    ay += g.y * t;
                    az += g.z * t;
                    if (kOp == kOpRhs) {
                        const float a2 = al * al * c.w_d;
                        dx += a2 * g.x * g.x;
                        dy += a2 * g.y * g.y;
                        dz += a2 * g.z * g.z;
                    }
                }
            }
            sub_sync(bar_id, nt);
        }
        if (has) {
            const int sl = node_slot<kAll>(c, corner_node(c, c.occ_cell[ci], k));
            if (ax != 0.f) atomicAdd(&dst[sl], ax);
            if (ay != 0.f) atomicAdd(&dst[c.ld + sl], ay);
            if (az != 0.f) atomicAdd(&dst[2 * c.ld + sl], az);
            if (kOp == kOpRhs) {
                if (dx != 0.f) atomicAdd(&dst2[sl], dx);
                if (dy != 0.f) atomicAdd(&dst2[c.ld + sl], dy);
                if (dz != 0.f) atomicAdd(&dst2[2 * c.ld + sl], dz);
            }
        }
    }
}

// The samples' J^T J p (Eq. 2, kOpApply above) of the sorted samples [js, je), in
// chunks of 32 consecutive samples per warp (lane l takes sample j0 + l): every lane
// forms its sample's t = w_d g.(sum_k alpha_k p_k) and the 24 products alpha_k t g_a
// (corner k, component a, at index 3 k + a); a segmented suffix sum over the lanes of
// the same cell (the samples are sorted by cell, so a cell's lanes are contiguous)
// leaves the sums of each cell's lanes in its first lane, which adds them to dst.
// An equal number of samples per warp, whatever their spread over cells.
// part += t (g.(sum alpha p)) per sample.
template <bool kAll, bool kMap = false>
__device__ __forceinline__ void samples_warp_apply(const Ctx &c, const VecView &vec, float *dst, int js, int je,
                                                   float &part, int lt, int nt, const SlotMap &m = SlotMap{}) {
    const size_t ldm = map_ld<kMap>(c, m);
    const int lane = lt & 31;
    for (int j0 = js + (lt & ~31); j0 < je; j0 += nt) {  // the same trip count in every lane of a warp
        const int j = j0 + lane;
        const bool has = j < je;
        int cl = -1;
        float4 f4 = make_float4(0.f, 0.f, 0.f, 0.f), g = f4;
        if (has) {
            cl = c.cell[j];
            f4 = c.frac[j];
            g = load_rec(c, j);
        }
        const float f[3] = {f4.x, f4.y, f4.z};
        float al[8], sx = 0.f, sy = 0.f, sz = 0.f;
#pragma unroll
        for (int k = 0; k < 8; k++) {
            al[k] = trilinear_weight(f, k);
            if (has) {
                const int vi = map_corner<kAll, kMap>(c, m, cl, k);
                sx += al[k] * ldvv<true>(vec, vi);
                sy += al[k] * ldvv<true>(vec, ldm + vi);
                sz += al[k] * ldvv<true>(vec, 2 * ldm + vi);
            }
        }
        const float sv = g.x * sx + g.y * sy + g.z * sz;
        const float t = has ? c.w_d * sv : 0.f;
        part += t * sv;
        const float tg[3] = {t * g.x, t * g.y, t * g.z};
        float v[24];
#pragma unroll
        for (int k = 0; k < 8; k++)
#pragma unroll
            for (int a = 0; a < 3; a++) v[3 * k + a] = al[k] * tg[a];
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int ko = __shfl_down_sync(FULL, cl, off);
            const bool same = lane + off < 32 && ko == cl;
#pragma unroll
            for (int i = 0; i < 24; i++) {
                const float o = __shfl_down_sync(FULL, v[i], off);
                if (same) v[i] += o;
            }
        }
        const int kp = __shfl_up_sync(FULL, cl, 1);
        if (has && (lane == 0 || kp != cl)) {
#pragma unroll
            for (int k = 0; k < 8; k++) {
                const int sl = map_corner<kAll, kMap>(c, m, cl, k);
#pragma unroll
                for (int a = 0; a < 3; a++)
                    if (v[3 * k + a] != 0.f) atomicAdd(&dst[(size_t)a * ldm + sl], v[3 * k + a]);
            }
        }
    }
}

// Sparse pairs (Eq. 3), one thread per pair; d = R_g (f^ + sum alpha u) + t_g - f in FP64.
//   kOpRhs:    r_k -= w_s alpha_k R_g^T d,  diag_k += w_s alpha_k^2 |R_g col|^2
//   kOpApply:  q_k += w_s alpha_k R_g^T R_g sum alpha p;  part += w_s |R_g sum alpha p|^2
//   kOpEnergy: partd += |d|^2
template <int kOp, bool kAll, bool kFresh, bool kMap = false>
__device__ __forceinline__ void sparse_pairs(const Ctx &c, const VecView vec, float *dst, float *dst2, int t0,
                                             int nthreads, float &part, double &partd, const SlotMap &m = SlotMap{}) {
    static_assert(!kMap || kOp == kOpApply, "the slot map serves the position step only");
    const size_t ldm = map_ld<kMap>(c, m);
    for (int sp = t0; sp < c.S; sp += nthreads) {
        const int cl = c.scell[sp];
        if (cl < 0) continue;
        const float4 f4 = c.sfrac[sp];
        const float f[3] = {f4.x, f4.y, f4.z};
        float al[8];
        int sl[8];
        V3<float> sv{0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < 8; k++) {
            al[k] = trilinear_weight(f, k);
            const int nd = corner_node(c, cl, k);
            sl[k] = map_corner<kAll, kMap>(c, m, cl, k);
            const int vi = (kOp == kOpApply) ? sl[k] : nd;
            sv.x += al[k] * ldvv<kFresh>(vec, vi);
            sv.y += al[k] * ldvv<kFresh>(vec, ldm + vi);
            sv.z += al[k] * ldvv<kFresh>(vec, 2 * ldm + vi);
        }
        if (kOp == kOpApply) {
            const V3<float> t = rot<float>(c.Rg, sv);
            part += c.w_s * dot(t, t);
            const V3<float> back = rotT<float>(c.Rg, t);
#pragma unroll
            for (int k = 0; k < 8; k++) {
                const float a = c.w_s * al[k];
                atomicAdd(&dst[sl[k]], a * back.x);
                atomicAdd(&dst[ldm + sl[k]], a * back.y);
                atomicAdd(&dst[2 * ldm + sl[k]], a * back.z);
            }
        } else {
            const float4 fh = c.fh[sp], ft = c.ft[sp];
            const V3<double> xq{(double)fh.x + sv.x, (double)fh.y + sv.y, (double)fh.z + sv.z};
            V3<double> d = rot<double>(c.Rg, xq);
            d.x += (double)c.tg[0] - (double)ft.x;
            d.y += (double)c.tg[1] - (double)ft.y;
            d.z += (double)c.tg[2] - (double)ft.z;
            if (kOp == kOpEnergy) {
                partd += dot(d, d);
            } else {
                const V3<float> back = rotT<float>(c.Rg, V3<float>{(float)d.x, (float)d.y, (float)d.z});
                const float cn[3] = {c.Rg[0] * c.Rg[0] + c.Rg[3] * c.Rg[3] + c.Rg[6] * c.Rg[6],
                                     c.Rg[1] * c.Rg[1] + c.Rg[4] * c.Rg[4] + c.Rg[7] * c.Rg[7],
                                     c.Rg[2] * c.Rg[2] + c.Rg[5] * c.Rg[5] + c.Rg[8] * c.Rg[8]};
#pragma unroll
                for (int k = 0; k < 8; k++) {
                    const float a = c.w_s * al[k];
                    atomicAdd(&dst[sl[k]], -a * back.x);
                    atomicAdd(&dst[c.ld + sl[k]], -a * back.y);
                    atomicAdd(&dst[2 * c.ld + sl[k]], -a * back.z);
                    const float a2 = a * al[k];
                    atomicAdd(&dst2[sl[k]], a2 * cn[0]);
                    atomicAdd(&dst2[c.ld + sl[k]], a2 * cn[1]);
                    atomicAdd(&dst2[2 * c.ld + sl[k]], a2 * cn[2]);
                }
            }
        }
    }
}

// x += v for four consecutive floats (16-byte aligned) as one vector reduction in L2
__device__ __forceinline__ void red_add_f4(float *x, float4 v) {
    asm volatile("red.relaxed.gpu.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(x), "f"(v.x), "f"(v.y), "f"(v.z),
                 "f"(v.w)
                 : "memory");
}

// ---- cached B^T B (Sec. 7.1: "pre-compute and cache B^T B before the PCG iteration
// commences"), the dense samples' part of J^T J per occupied cell:
//   B_cell[(k, a), (m, b)] = w_d sum_{samples j of the cell} alpha_k(j) g'_a(j) alpha_m(j) g'_b(j)
// (v_j = alpha(j) (x) g'_j, a 24-vector; B_cell = w_d sum_j v_j v_j^T), stored as a full
// row-major 24 x 24 block (576 floats).  The build is balanced by samples: each warp
// takes 64 consecutive sorted samples, reads them 32 at a time (one coalesced load per
// lane), broadcasts each sample's fractions and g' by shuffles, and lane l < 24 sums row
// l of the partial block of every cell the 64 samples overlap (v_j[l] v_j[m] for every
// m); each partial block is added to the (zeroed) block with vector reductions.
constexpr int kBtb = 576;
constexpr int kBtbChunk = 64;  // samples per warp of the build

template <bool kAll>
__global__ void __launch_bounds__(kThreads) k_btb_build(Ctx c, const Scal *sc) {
    pdl_wait();
    pdl_trigger();
    if (sc->skip) return;
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    const int n_occ = *c.n_occ;
    const int ns = n_occ > 0 ? c.occ_beg[n_occ] : 0;
    const int k = lane / 3, a = lane - 3 * (lane / 3);
    for (int j0 = warp * kBtbChunk; j0 < ns; j0 += nw * kBtbChunk) {
        const int jend = min(j0 + kBtbChunk, ns);
        int lo = 0, hi = n_occ;  // the cell holding sample j0: last cell starting at or before it
        while (hi - lo > 1) {
            const int m = (lo + hi) >> 1;
            if (c.occ_beg[m] <= j0) lo = m;
            else hi = m;
        }
        for (int ci = lo; ci < n_occ && c.occ_beg[ci] < jend; ci++) {
            const int cb = max(c.occ_beg[ci], j0), ce = min(c.occ_beg[ci + 1], jend);
            float acc[24];
#pragma unroll
            for (int m = 0; m < 24; m++) acc[m] = 0.f;
            for (int jb = cb; jb < ce; jb += 32) {
                float4 f4 = make_float4(0.f, 0.f, 0.f, 0.f), g = f4;
                if (jb + lane < ce) {
                    f4 = c.frac[jb + lane];
                    g = load_rec(c, jb + lane);
                }
                const int nj = min(32, ce - jb);
#pragma unroll 2
                for (int t = 0; t < nj; t++) {
                    const float f[3] = {__shfl_sync(FULL, f4.x, t), __shfl_sync(FULL, f4.y, t),
                                        __shfl_sync(FULL, f4.z, t)};
                    const float gv[3] = {__shfl_sync(FULL, g.x, t), __shfl_sync(FULL, g.y, t), __shfl_sync(FULL, g.z, t)};
                    const float vl = trilinear_weight(f, k) * (a == 0 ? gv[0] : (a == 1 ? gv[1] : gv[2]));
#pragma unroll
                    for (int kk = 0; kk < 8; kk++) {
                        const float al = vl * trilinear_weight(f, kk);
#pragma unroll
                        for (int b = 0; b < 3; b++) acc[3 * kk + b] = fmaf(al, gv[b], acc[3 * kk + b]);
                    }
                }
            }
            if (lane < 24) {
                float *row = c.btb + (size_t)ci * kBtb + lane * 24;
#pragma unroll
                for (int m4 = 0; m4 < 6; m4++)
                    red_add_f4(row + 4 * m4, make_float4(c.w_d * acc[4 * m4], c.w_d * acc[4 * m4 + 1],
                                                         c.w_d * acc[4 * m4 + 2], c.w_d * acc[4 * m4 + 3]));
            }
        }
    }
}

// q += B_cell p_cell for occupied cell ci, one warp: lane l < 24 gathers p at corner l / 3,
// component l % 3, forms row l of the product (p broadcast by shuffles) and adds it to
// q there; part += p_cell . B_cell p_cell.  Every lane of the warp must call it.
template <bool kAll, bool kFresh, bool kMap = false>
__device__ __forceinline__ void btb_cell_apply(const Ctx &c, const VecView vec, int ci, float *dst, float &part,
                                               const SlotMap &m = SlotMap{}) {
    const int lane = threadIdx.x & 31;
    const bool act = lane < 24;
    const int k = lane / 3, a = lane - 3 * (lane / 3);
    const size_t ldm = map_ld<kMap>(c, m);
    int sl = 0;
    float pl = 0.f;
    if (act) {
        sl = map_corner<kAll, kMap>(c, m, c.occ_cell[ci], k);
        pl = ldvv<kFresh>(vec, (size_t)a * ldm + sl);
    }
    const float4 *B = reinterpret_cast<const float4 *>(c.btb + (size_t)ci * kBtb + (act ? lane : 0) * 24);
    float q = 0.f;
#pragma unroll
    for (int m4 = 0; m4 < 6; m4++) {
        const float4 b = act ? __ldg(B + m4) : make_float4(0.f, 0.f, 0.f, 0.f);
        q = fmaf(b.x, __shfl_sync(FULL, pl, 4 * m4), q);
        q = fmaf(b.y, __shfl_sync(FULL, pl, 4 * m4 + 1), q);
        q = fmaf(b.z, __shfl_sync(FULL, pl, 4 * m4 + 2), q);
        q = fmaf(b.w, __shfl_sync(FULL, pl, 4 * m4 + 3), q);
    }
    if (act) {
        part += pl * q;
        if (q != 0.f) atomicAdd(&dst[(size_t)a * ldm + sl], q);
    }
}

// Streamed apply of the samples' part with the cached blocks (one warp per occupied
// cell) plus the sparse pairs matrix-free, and the partial p.Ap.
template <bool kAll>
__global__ void __launch_bounds__(kThreads) k_cells_btb(Ctx c, Scal *sc, int K, int it) {
    pdl_wait();
    pdl_trigger();
    if (sc->skip) return;
    if (sc->stop || !(scal_rho(sc)[it] > 0.0)) return;
    const VecView vec{c.p, nullptr, 0.f};
    float part = 0.f;
    double partd = 0.0;
    const int n_occ = *c.n_occ;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    for (int ci = warp; ci < n_occ; ci += nw) btb_cell_apply<kAll, false>(c, vec, ci, c.q, part);
    sparse_pairs<kOpApply, kAll, false>(c, vec, c.q, nullptr, blockIdx.x + gridDim.x * threadIdx.x,
                                        gridDim.x * blockDim.x, part, partd);
    block_add_f64(part, scal_pq(sc, K) + it);
}

// Partition of the sorted samples among the nb blocks of the sample passes: block b
// takes samples [b n / nb, (b + 1) n / nb) and the occupied cells that hold them.
__global__ void k_cell_partition(const int *__restrict__ occ_beg, const int *__restrict__ n_occ_p, int nb,
                                 int4 *__restrict__ part) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const int n_occ = *n_occ_p, ns = n_occ > 0 ? occ_beg[n_occ] : 0;
    const int js = (int)(((long long)ns * b) / nb), je = (int)(((long long)ns * (b + 1)) / nb);
    int lo = 0, hi = n_occ;  // first cell whose end is past js
    while (lo < hi) {
        const int m = (lo + hi) >> 1;
        if (occ_beg[m + 1] <= js) lo = m + 1;
        else hi = m;
    }
    const int cb = lo;
    hi = n_occ;  // first cell that starts at or after je
    while (lo < hi) {
        const int m = (lo + hi) >> 1;
        if (occ_beg[m] < je) lo = m + 1;
        else hi = m;
    }
    part[b] = make_int4(cb, je > js ? lo : cb, js, je);
}

template <int kOp, bool kAll>
__global__ void __launch_bounds__(kThreads) k_cells(Ctx c, Scal *sc, int K, int it) {
    pdl_wait();
    pdl_trigger();
    if (sc->skip) return;
    if (kOp == kOpApply) {
        if (sc->stop || !(scal_rho(sc)[it] > 0.0)) return;
    }
    __shared__ float tsm[kThreads];
    const VecView vec{(kOp == kOpApply) ? c.p : c.u, nullptr, 0.f};
    float *dst = (kOp == kOpApply) ? c.q : c.r;
    float part = 0.f;
    double partd = 0.0;
    // an equal share of the sorted samples per block (set up with the frame)
    const int4 cp = c.cell_part[blockIdx.x];
    if (cp.y > cp.x)
        cells_block<kOp, kAll, false>(c, vec, dst, c.minv, cp.x, cp.y, tsm, kThreads, part, threadIdx.x, blockDim.x, 0, cp.z,
                                      cp.w);
    // pairs spread one per block first: one SM issuing all their atomics would be the tail
    sparse_pairs<kOp, kAll, false>(c, vec, dst, c.minv, blockIdx.x + gridDim.x * threadIdx.x,
                                   gridDim.x * blockDim.x, part, partd);
    if (kOp == kOpApply) block_add_f64(part, scal_pq(sc, K) + it);
    if (kOp == kOpEnergy) {
        block_add_f64(part, &sc->e_dense);
        block_add_f64d(partd, &sc->e_sparse);
    }
}

// ------------------------------------------------------------------ node passes

// ARAP part of the right-hand side and the Jacobi diagonal (Eq. 4 with R fixed):
//   b_k = -w_r sum_{j in N_k} [2 (u_k - u_j) - (R_k + R_j - 2I)(t^_k - t^_j)],
//   diag_k = 2 w_r |N_k|.  Written with plain stores (the sample pass adds after).
template <bool kAll>
__device__ __forceinline__ void rhs_nodes_block(const Ctx &c, int bid, int nb) {
    const int N = active_count<kAll>(c);
    for (int s = bid * blockDim.x + threadIdx.x; s < N; s += nb * blockDim.x) {
        const int i = slot_node<kAll>(c, s);
        int nb[6];
        neighbours<kAll>(c, s, nb);
        const float3 ui = ld3(c.u, c.ld, i);
        float bx = 0.f, by = 0.f, bz = 0.f;
        int deg = 0;
#pragma unroll
        for (int d = 0; d < 6; d++) {
            if (nb[d] < 0) continue;
            const int j = slot_node<kAll>(c, nb[d]);
            const int a = d >> 1;
            const float sg = (d & 1) ? c.h : -c.h;  // t^_k - t^_j = -sg e_a
            const float3 uj = ld3(c.u, c.ld, j);
            // column a of R_k + R_j - 2 I
            const float cx = c.R[a * c.ld + i] + c.R[a * c.ld + j] - (a == 0 ? 2.f : 0.f);
            const float cy = c.R[(3 + a) * c.ld + i] + c.R[(3 + a) * c.ld + j] - (a == 1 ? 2.f : 0.f);
            const float cz = c.R[(6 + a) * c.ld + i] + c.R[(6 + a) * c.ld + j] - (a == 2 ? 2.f : 0.f);
            bx -= c.w_r * (2.f * (ui.x - uj.x) + sg * cx);
            by -= c.w_r * (2.f * (ui.y - uj.y) + sg * cy);
            bz -= c.w_r * (2.f * (ui.z - uj.z) + sg * cz);
            deg++;
        }
        st3(c.r, c.ld, s, make_float3(bx, by, bz));
        const float dg = 2.f * c.w_r * (float)deg;
        st3(c.minv, c.ld, s, make_float3(dg, dg, dg));
    }
}

template <bool kAll>
__global__ void __launch_bounds__(kThreads) k_rhs_nodes(Ctx c, const Scal *sc) {
    pdl_wait();
    pdl_trigger();
    if (sc->skip) return;
    rhs_nodes_block<kAll>(c, blockIdx.x, gridDim.x);
}

// k_rhs_nodes with the FP64 re-association of the listed samples in its first `nref`
// blocks: the re-association is a latency-bound tail of a few warps, which the node
// pass (independent of the correspondences) runs beside.
template <bool kAll>
__global__ void __launch_bounds__(kThreads, 4) k_rhs_nodes_refine(Ctx c, Scal *sc, int nref) {
    pdl_wait();
    pdl_trigger();
    if (sc->skip) return;
    if ((int)blockIdx.x < nref) associate_refine_block<kAll>(c, sc, blockIdx.x, nref);
    else rhs_nodes_block<kAll>(c, blockIdx.x - nref, gridDim.x - nref);
}

// PCG vectors are walked as float4 groups of one component plane per blockIdx.y (the
// planes are 128-byte aligned, ld is a multiple of 32).  The pad slots [N, 4 ceil(N/4))
// are zeroed by k_pcg_init, so a group straddling N only ever adds zeros.
__device__ __forceinline__ int groups4(int N) { return (N + 3) >> 2; }

// PCG start (x0 = 0): Minv = 1/diag (0 where diag = 0), r = b, p = z = Minv r, rho0 = r.z
template <bool kAll>
__global__ void __launch_bounds__(kThreads) k_pcg_init(Ctx c, Scal *sc) {
    pdl_wait();
    pdl_trigger();
    if (sc->skip) return;
    const int N = active_count<kAll>(c);
    const size_t off = (size_t)blockIdx.y * c.ld;
    float *__restrict__ minv = c.minv + off;
    float *__restrict__ r = c.r + off;
    float *__restrict__ p = c.p + off;
    float *__restrict__ x = c.x + off;
    float *__restrict__ q = c.q + off;
    float part = 0.f;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < 4 * groups4(N); s += gridDim.x * blockDim.x) {
        if (s >= N) {  // pad slots of the last group
            minv[s] = 0.f;
            r[s] = 0.f;
            p[s] = 0.f;
            x[s] = 0.f;
            q[s] = 0.f;
            continue;
        }
        const float dg = minv[s];
        const float mi = dg > 0.f ? 1.0f / dg : 0.f;
        const float rr = r[s];
        const float z = mi * rr;
        minv[s] = mi;
        p[s] = z;
        x[s] = 0.f;
        part += rr * z;
    }
    block_add_f64(part, &scal_rho(sc)[0]);
}

// all-nodes lattice with nx % 4 == 0: q for the 4 nodes of one row starting at s0
__device__ __forceinline__ float stencil4(const Ctx &c, int s0, float w2) {
    const int x0 = s0 % c.nx, t = s0 / c.nx, y = t % c.ny, z = t / c.ny, pl = c.nx * c.ny;
    float part = 0.f;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const float *__restrict__ P = c.p + (size_t)a * c.ld;
        const float4 pc = *reinterpret_cast<const float4 *>(P + s0);
        // a missing neighbour is replaced by the node itself: its difference is 0
        const float left = x0 > 0 ? P[s0 - 1] : pc.x;
        const float right = x0 + 4 < c.nx ? P[s0 + 4] : pc.w;
        float4 d = make_float4((pc.x - left) + (pc.x - pc.y), (pc.y - pc.x) + (pc.y - pc.z),
                               (pc.z - pc.y) + (pc.z - pc.w), (pc.w - pc.z) + (pc.w - right));
        const int offs[4] = {-c.nx, c.nx, -pl, pl};
        const bool has[4] = {y > 0, y + 1 < c.ny, z > 0, z + 1 < c.nz};
#pragma unroll
        for (int k = 0; k < 4; k++) {
            if (!has[k]) continue;
            const float4 v = *reinterpret_cast<const float4 *>(P + s0 + offs[k]);
            d.x += pc.x - v.x;
            d.y += pc.y - v.y;
            d.z += pc.z - v.z;
            d.w += pc.w - v.w;
        }
        d.x *= w2;
        d.y *= w2;
        d.z *= w2;
        d.w *= w2;
        *reinterpret_cast<float4 *>(c.q + (size_t)a * c.ld + s0) = d;
        part += pc.x * d.x + pc.y * d.y + pc.z * d.z + pc.w * d.w;
    }
    return part;
}

// q = 2 w_r L p (7-point graph Laplacian of M), with the partial p.q.
// kVec4: all-nodes lattice with nx % 4 == 0, one thread per 4 nodes of a row.
template <bool kAll, bool kVec4>
__global__ void __launch_bounds__(kThreads) k_apply_stencil(Ctx c, Scal *sc, int K, int it) {
    pdl_wait();
    pdl_trigger();
    if (it >= 0 && (sc->stop || !(scal_rho(sc)[it] > 0.0))) return;
    const int N = active_count<kAll>(c);
    float part = 0.f;
    const float w2 = 2.f * c.w_r;
    if (kVec4) {
        for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < (N >> 2); g += gridDim.x * blockDim.x)
            part += stencil4(c, 4 * g, w2);
    } else {
        for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < N; s += gridDim.x * blockDim.x) {
            int nb[6];
            neighbours<kAll>(c, s, nb);
            const float3 pi = ld3(c.p, c.ld, s);
            float qx = 0.f, qy = 0.f, qz = 0.f;
#pragma unroll
            for (int d = 0; d < 6; d++) {
                if (nb[d] < 0) continue;
                const float3 pj = ld3(c.p, c.ld, nb[d]);
                qx += pi.x - pj.x;
                qy += pi.y - pj.y;
                qz += pi.z - pj.z;
            }
            qx *= w2;
            qy *= w2;
            qz *= w2;
            st3(c.q, c.ld, s, make_float3(qx, qy, qz));
            part += pi.x * qx + pi.y * qy + pi.z * qz;
        }
    }
    block_add_f64(part, scal_pq(sc, K) + (it >= 0 ? it : 0));
}

// alpha = rho/pq; x += alpha p; r -= alpha q; z = Minv r; partial rho' = r.z.
// One wave of fat threads: each thread takes float4 group g of all three component
// planes, so its 15 vector loads are in flight together.
template <bool kAll>
__global__ void __launch_bounds__(kThreads) k_update_x(Ctx c, Scal *sc, int K, int it) {
    pdl_wait();
    pdl_trigger();
    __shared__ float s_alpha;
    __shared__ int s_go;
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
    if (threadIdx.x == 0) {  // one FP64 division per block
        const double rho = scal_rho(sc)[it], pq = scal_pq(sc, K)[it];
        s_go = !sc->stop && rho > 0.0 && pq > 0.0;
        s_alpha = s_go ? (float)(rho / pq) : 0.f;
        if (!s_go && lead) sc->stop = 1;
    }
    __syncthreads();
    if (!s_go) return;
    const float alpha = s_alpha;
    const int G4 = groups4(active_count<kAll>(c));
    const int ld4 = c.ld >> 2;
    float4 *__restrict__ x = reinterpret_cast<float4 *>(c.x);
    float4 *__restrict__ r = reinterpret_cast<float4 *>(c.r);
    const float4 *__restrict__ p = reinterpret_cast<const float4 *>(c.p);
    const float4 *__restrict__ q = reinterpret_cast<const float4 *>(c.q);
    const float4 *__restrict__ m = reinterpret_cast<const float4 *>(c.minv);
    float part = 0.f;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G4; g += gridDim.x * blockDim.x) {
        float4 xv[3], pv[3], rv[3], qv[3], mv[3];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const int k = a * ld4 + g;
            xv[a] = x[k];
            pv[a] = p[k];
            rv[a] = r[k];
            qv[a] = q[k];
            mv[a] = m[k];
        }
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const int k = a * ld4 + g;
            const float4 xn = make_float4(fmaf(alpha, pv[a].x, xv[a].x), fmaf(alpha, pv[a].y, xv[a].y),
                                          fmaf(alpha, pv[a].z, xv[a].z), fmaf(alpha, pv[a].w, xv[a].w));
            const float4 rn = make_float4(fmaf(-alpha, qv[a].x, rv[a].x), fmaf(-alpha, qv[a].y, rv[a].y),
                                          fmaf(-alpha, qv[a].z, rv[a].z), fmaf(-alpha, qv[a].w, rv[a].w));
            x[k] = xn;
            r[k] = rn;
            part += rn.x * (mv[a].x * rn.x) + rn.y * (mv[a].y * rn.y) + rn.z * (mv[a].z * rn.z) +
                    rn.w * (mv[a].w * rn.w);
        }
    }
    if (lead) sc->cg_done = it + 1;
    block_add_f64(part, &scal_rho(sc)[it + 1]);
}

// beta = rho'/rho; p = Minv r + beta p (stop once rho' <= tol^2 rho0)
template <bool kAll>
__global__ void __launch_bounds__(kThreads) k_update_p(Ctx c, Scal *sc, int it, double tol2) {
    pdl_wait();
    pdl_trigger();
    __shared__ float s_beta;
    __shared__ int s_go;
    if (threadIdx.x == 0) {  // one FP64 division per block
        const double rho1 = scal_rho(sc)[it + 1], rho = scal_rho(sc)[it];
        s_go = !sc->stop && !(rho1 <= tol2 * scal_rho(sc)[0]);
        s_beta = s_go ? (float)(rho1 / rho) : 0.f;
        if (!sc->stop && !s_go && blockIdx.x == 0) sc->stop = 1;
    }
    __syncthreads();
    if (!s_go) return;
    const float beta = s_beta;
    const int G4 = groups4(active_count<kAll>(c));
    const int ld4 = c.ld >> 2;
    float4 *__restrict__ p = reinterpret_cast<float4 *>(c.p);
    const float4 *__restrict__ r = reinterpret_cast<const float4 *>(c.r);
    const float4 *__restrict__ m = reinterpret_cast<const float4 *>(c.minv);
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < G4; g += gridDim.x * blockDim.x) {
        float4 pv[3], rv[3], mv[3];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const int k = a * ld4 + g;
            pv[a] = p[k];
            rv[a] = r[k];
            mv[a] = m[k];
        }
#pragma unroll
        for (int a = 0; a < 3; a++)
            p[a * ld4 + g] = make_float4(fmaf(beta, pv[a].x, mv[a].x * rv[a].x), fmaf(beta, pv[a].y, mv[a].y * rv[a].y),
                                         fmaf(beta, pv[a].z, mv[a].z * rv[a].z), fmaf(beta, pv[a].w, mv[a].w * rv[a].w));
    }
}

template <bool kAll>
__global__ void __launch_bounds__(kThreads) k_add_increment(Ctx c, const Scal *sc) {
    pdl_wait();
    pdl_trigger();
    if (sc->skip) return;
    const int N = active_count<kAll>(c);
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < N; s += gridDim.x * blockDim.x) {
        const int i = slot_node<kAll>(c, s);
#pragma unroll
        for (int a = 0; a < 3; a++) c.u[a * c.ld + i] += c.x[a * c.ld + s];
    }
}

// ------------------------------------------------------------------ persistent PCG (Sec. 7.1 position step)

// One cooperative launch runs a whole position step.  Each CTA owns `chunk` slots (a
// brick of full x-rows of an all-nodes lattice, else a contiguous range, a multiple of 4)
// and keeps p, r and q of its slots in shared memory for all K iterations (x accumulates
// in global memory, L2-resident); z and p are published to global memory (read through
// L2 by the CTAs whose stencil or samples need them), and the samples' J^T J p
// contributions go to a global buffer with atomics that the owners fold in and clear.
// Two grid barriers per iteration (after p.Ap, after r.z).  The reductions are
// deterministic: every CTA writes its FP64 partial to a per-iteration row and every CTA
// sums the row in CTA order.  A barrier that waits longer than about a second sets the
// error flag and the whole grid returns.
// 768 threads leave 80 registers to a thread (1024 would leave 64, and spill); the
// stencil gets 512 of them, the samples 256 (a CTA's share of the samples of a 96^3
// frame, about 250, fits one chunk of the sample pass)
constexpr int kPcgThreads = 768;
constexpr int kPcgMaxGroups = 2;  // float4 groups per thread: chunk <= 4 * 2 * 768
constexpr int kPcgStencil = 512;                          // threads on the stencil in phase A
constexpr int kPcgSample = kPcgThreads - kPcgStencil;      // threads on the samples in phase A
constexpr int kPcgStencilGroups = kPcgMaxGroups * kPcgThreads / kPcgStencil;  // per stencil thread
static_assert(kPcgStencilGroups * kPcgStencil == kPcgMaxGroups * kPcgThreads, "the stencil threads cover the chunk");
// Tensor memory of the persistent position step: warp w reads and writes TMEM lanes
// 32 (w % 4) .. + 31 (one lane per thread), columns 64 (w / 4) .. + 63: r of its
// kPcgMaxGroups groups of phase B (12 columns each, component a at + 4 a), then, for a
// stencil thread, x of its kPcgStencilGroups groups of A1
constexpr int kPcgTmemCols = 512;
constexpr int kPcgTmemX = 12 * kPcgMaxGroups;
static_assert(64 * (kPcgThreads / 128) <= kPcgTmemCols && kPcgTmemX + 12 * kPcgStencilGroups <= 64, "TMEM slices");

// 12 consecutive TMEM columns of this thread's lane to / from three float4 (tcgen05.ld
// and its wait in one statement, so that no register is read before the data arrive;
// warp-collective: every lane of the warp executes it)
__device__ __forceinline__ void tmem_ld12(uint32_t ta, float4 (&v)[3]) {
    uint32_t r[12];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%12];\n"
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%8,%9,%10,%11}, [%13];\n"
        "tcgen05.wait::ld.sync.aligned;\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11])
        : "r"(ta), "r"(ta + 8)
        : "memory");
#pragma unroll
    for (int a = 0; a < 3; a++)
        v[a] = make_float4(__uint_as_float(r[4 * a]), __uint_as_float(r[4 * a + 1]), __uint_as_float(r[4 * a + 2]),
                           __uint_as_float(r[4 * a + 3]));
}
__device__ __forceinline__ void tmem_st12(uint32_t ta, const float4 (&v)[3]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%2,%3,%4,%5,%6,%7,%8,%9};\n"
        "tcgen05.st.sync.aligned.32x32b.x4.b32 [%1], {%10,%11,%12,%13};\n" ::"r"(ta),
        "r"(ta + 8), "r"(__float_as_uint(v[0].x)), "r"(__float_as_uint(v[0].y)), "r"(__float_as_uint(v[0].z)),
        "r"(__float_as_uint(v[0].w)), "r"(__float_as_uint(v[1].x)), "r"(__float_as_uint(v[1].y)),
        "r"(__float_as_uint(v[1].z)), "r"(__float_as_uint(v[1].w)), "r"(__float_as_uint(v[2].x)),
        "r"(__float_as_uint(v[2].y)), "r"(__float_as_uint(v[2].z)), "r"(__float_as_uint(v[2].w))
        : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
constexpr long long kBarrierCycles = 2000000000LL;

struct PcgAux {
    double *part;      // rows 0..K: r.z partials, rows K+1..2K: p.Ap partials, G entries each
    unsigned long long *words;  // one word per grid barrier (2K + 1), zeroed before the launch
    int extra;         // arrivals awaited beyond G: 0, or 1 to make the first wait run out
                       // (failure injection for tests, vd_test_stall_barrier)
    int *err;          // set when a barrier wait gives up
    const int *flag;   // per slot: 1 if a sample or a sparse pair touches it (0 past N)
    float *pbuf[2];    // p of even / odd iterations, published for the other CTAs
    int chunk;         // slots per CTA
    int by, bz;        // > 0: each CTA owns a brick of by x bz full x-rows (all-nodes
                       // lattice); 0: a contiguous slot range
    int lx;            // a brick's local row length: nx, or nx rounded up to a multiple of
                       // 4 for a padded brick (the bricks at the far y / z faces may then
                       // also hold fewer rows than by x bz)
    // n / lx and n / by as (2n m) >> 32 with m = ceil(2^31 / d), exact for n d < 2^31
    // (the local slot and row indices of a brick): no integer division in the loops
    unsigned m_nx, m_by;
    // a padded brick with unaligned rows (nx % 4 != 0): z, q and (in pbuf) p published at
    // x + lx (y + ny z), plane stride ldp; m_nx0: the multiply-high constant of nx
    float *zpad, *qpad;
    long long ldp;
    unsigned m_nx0;
};

__device__ __forceinline__ int fast_div(int n, unsigned m) { return (int)__umulhi(2u * (unsigned)n, m); }

constexpr int kPcgMaxRows = 128;  // x-rows of one brick (bounds the plan's search)
constexpr int kPcgMaxCtas = 255;  // the arrival count of a barrier word has 8 bits


// The scalar work around the grid barriers is done with integer operations on the bits
// of the FP64 values (this GPU's FP64 pipe is narrow, and a chain of FP64 operations in
// one thread sits on the critical path of every barrier).

// round(|v| 2^k) with the sign of v (halves away from zero), for a finite v and
// k <= 1012; false when it would reach 2^39 in magnitude (or v is not finite)
__device__ __forceinline__ bool fixed_of(double v, int k, long long &out) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int E = (int)((b >> 52) & 0x7ff);
    if (E == 0x7ff) return false;
    if (E == 0) {  // zero or subnormal: below 2^-1022 2^1012, rounds to 0
        out = 0;
        return true;
    }
    const unsigned long long m = (b & 0xfffffffffffffull) | (1ull << 52);  // |v| = m 2^(E - 1075)
    const int sh = E - 1075 + k;                                           // |v| 2^k = m 2^sh
    if (sh >= -13) return false;                                           // m 2^sh >= 2^39
    const unsigned long long a = sh < -63 ? 0ull : (m + (1ull << (-sh - 1))) >> (-sh);
    if (a >= (1ull << 39)) return false;
    out = (b >> 63) ? -(long long)a : (long long)a;
    return true;
}

// fx 2^-k as an FP64 value (exact for |fx| < 2^53; the exponent must stay normal)
__device__ __forceinline__ double double_of_fixed(long long fx, int k) {
    if (fx == 0) return 0.0;
    const unsigned long long sgn = fx < 0 ? (1ull << 63) : 0ull;
    const unsigned long long a = fx < 0 ? (unsigned long long)(-fx) : (unsigned long long)fx;
    const int lz = __clzll((long long)a);
    const unsigned long long m = lz >= 11 ? a << (lz - 11) : a >> (11 - lz);  // leading 1 at bit 52
    const long long E = 1023 + (63 - lz) - k;
    return __longlong_as_double((long long)(sgn | ((unsigned long long)E << 52) | (m & 0xfffffffffffffull)));
}

// The FP32 quotient n / d of two FP64 values, from their signs, exponents and leading
// 24 bits (rounded) and one FP32 division: within 3 2^-24 of the exact quotient,
// relative (two roundings of the operands and one of the division).  Zero, subnormal or
// non-finite operands, and quotients outside the normal FP32 range, take the FP64
// division instead.
__device__ __forceinline__ float f32_quot(double n, double d) {
    const unsigned long long bn = (unsigned long long)__double_as_longlong(n),
                             bd = (unsigned long long)__double_as_longlong(d);
    const int en = (int)((bn >> 52) & 0x7ff), ed = (int)((bd >> 52) & 0x7ff);
    if (en == 0 || ed == 0 || en == 0x7ff || ed == 0x7ff) return (float)(n / d);
    // the leading bits as FP32 values in [1, 2] (a carry of the rounding gives 2)
    auto lead = [](unsigned long long b) {
        return __uint_as_float((unsigned)(0x3f800000u + (((b & 0xfffffffffffffull) + (1ull << 28)) >> 29)) |
                               (unsigned)((b >> 63) << 31));
    };
    const float q = lead(bn) / lead(bd);  // |q| in [0.5, 2]
    const int eq = (int)((__float_as_uint(q) >> 23) & 0xff) + (en - ed);
    if (eq < 1 || eq > 254) return (float)(n / d);
    return __uint_as_float((__float_as_uint(q) & 0x807fffffu) | ((unsigned)eq << 23));
}

struct NoPost {
    __device__ void operator()(double) const {}
};
struct NoWork {
    __device__ void operator()() const {}
};

// v > 0 and finite, from its bits
__device__ __forceinline__ bool pos_finite(double v) {
    const long long b = __double_as_longlong(v);
    return b > 0 && (b >> 52) < 0x7ff;
}
// a <= b for finite a, b >= 0, from their bits (the bit patterns of non-negative
// doubles are ordered as the values)
__device__ __forceinline__ bool le_nonneg(double a, double b) { return __double_as_longlong(a) <= __double_as_longlong(b); }

// Grid barrier that also reduces, over the G CTAs that share `word` (a whole grid, or
// one group of it: `bid` is the CTA's index in that group).  Each barrier of a launch
// has its own 64-bit word (zeroed before the launch).  Thread 0 of each CTA writes the
// CTA's FP64 partial to `row` and, with a release atom (which publishes every write of
// the CTA: the __syncthreads before it orders them before thread 0's), adds to the
// word 1 (bits 0-7 count the arrivals) plus, when a reference magnitude ref > 0 is given (the previous value of the
// same sum: the same in every CTA), the partial in fixed point, round(part 2^(32 - e))
// with ref = m 2^e, in bits 16-63 -- or 256 (bits 8-15) if it is not below 2^39.  Then it
// polls the word (acquire) until the count is G, for at most kBarrierCycles.  Integer
// addition is associative, so the final word does not depend on the order of arrival.
// When no partial overflowed and the fixed-point sum is at least 2^28 (ref / 16; the
// rounding of at most 160 partials, 80 units, is then below 3e-7 of it, the precision of
// the FP32 partials themselves) that sum is the result, read with the barrier word;
// otherwise every CTA sums `row` itself, in the same order in every CTA.  Either way all
// CTAs get the same `sum`.  kSynced: the caller has synchronised the CTA since its last
// write that other CTAs read (block_sum does).  The thread kLead (lane 0 of its warp; it
// holds `part` and `ref`) arrives and waits; post(sum) runs in it before the CTA's last
// __syncthreads here, so what it stores in shared memory is visible to every thread on
// return.  The other threads run during() while it waits (work that needs neither the
// sum nor other CTAs' data).  The scale 2^e of ref is taken for 2^-960 <= ref < 2^961
// (the row path otherwise).
template <bool kSynced = false, unsigned kLead = 0, typename Post = NoPost, typename During = NoWork>
__device__ __forceinline__ bool grid_reduce(int *err, unsigned G, unsigned arrivals, double *row, unsigned long long *word,
                                            double part, double ref, double &sum, unsigned bid, Post post = Post(),
                                            During during = During()) {
    static_assert(kLead % 32 == 0, "the lead thread is lane 0 of its warp");
    __shared__ int s_ok, s_fast;
    __shared__ double s_sum;
    if (!kSynced) __syncthreads();
    if (threadIdx.x != kLead) {
        during();
    } else {
        row[bid] = part;  // ordered before the arrival by the release of the atom below
        unsigned long long inc = 1;
        const long long rb = __double_as_longlong(ref);
        const int e = (int)((rb >> 52) & 0x7ff) - 1023;  // ref = m 2^e, 1 <= m < 2
        const bool fixed = rb > 0 && e >= -960 && e <= 960;  // positive, normal, finite
        if (fixed) {
            long long fxp;
            if (fixed_of(part, 32 - e, fxp)) inc += (unsigned long long)fxp << 16;
            else inc += 256ull;
        }
        unsigned long long old;
        asm volatile("atom.add.release.gpu.global.u64 %0, [%1], %2;" : "=l"(old) : "l"(word), "l"(inc) : "memory");
        int good = 1;
        unsigned long long w = old + inc;
        const long long t0 = clock64();
        while ((w & 0xFFull) != arrivals) {
            asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(w) : "l"(word) : "memory");
            if ((w & 0xFFull) == arrivals) break;
            if (*(volatile int *)err) {
                good = 0;
                break;
            }
            if (clock64() - t0 > kBarrierCycles) {
                atomicExch(err, 1);
                good = 0;
                break;
            }
        }
        const long long fx = (long long)w >> 16;
        const int fast = good && fixed && ((w >> 8) & 0xFFull) == 0 && (fx >= (1ll << 28) || fx <= -(1ll << 28));
        if (fast) {
            s_sum = double_of_fixed(fx, 32 - e);
            post(s_sum);
        }
        s_fast = fast;
        // a complete count means that no CTA gave up on this barrier (one that gave up on
        // an earlier one never arrives here): no second look at the error word
        s_ok = good;
    }
    __syncthreads();
    if (!s_fast) {  // the same decision in every CTA
        if ((threadIdx.x >> 5) == (kLead >> 5)) {
            const unsigned lane = threadIdx.x & 31u;
            double v[5];
#pragma unroll
            for (int k = 0; k < 5; k++) {  // all loads in flight before the first add
                const unsigned b = lane + 32u * k;
                v[k] = b < G ? __ldcg(row + b) : 0.0;
            }
            double t = (((v[0] + v[1]) + v[2]) + v[3]) + v[4];
            for (unsigned b = lane + 160u; b < G; b += 32) t += __ldcg(row + b);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(FULL, t, o);
            if (threadIdx.x == kLead) {
                s_sum = t;
                post(t);
            }
        }
        __syncthreads();
    }
    sum = s_sum;
    return s_ok != 0;
}

// Test support: `rounds` reductions over the grid, round k summing the partials
// parts[k * G + b] (one per CTA) with grid_reduce, the previous round's sum as the scale
// of the fixed-point path (as the position step does); out[2 k] gets the barrier's
// result, out[2 k + 1] the FP64 sum of the row in CTA order.  words: `rounds` zeroed
// barrier words; rows: rounds x G doubles.
__global__ void k_test_grid_reduce(const double *__restrict__ parts, int rounds, double *rows,
                                   unsigned long long *words, int *err, double *out) {
    const unsigned G = gridDim.x;
    double ref = 0.0, sum = 0.0;
    for (int k = 0; k < rounds; k++) {
        const double mine = parts[(size_t)k * G + blockIdx.x];
        if (!grid_reduce(err, G, G, rows + (size_t)k * G, words + k, mine, ref, sum, blockIdx.x)) return;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            double t = 0.0;
            for (unsigned b = 0; b < G; b++) t += __ldcg(rows + (size_t)k * G + b);
            out[2 * k] = sum;
            out[2 * k + 1] = t;
        }
        ref = sum;
    }
}

// FP64 block sum of one float per thread; valid in thread 0
__device__ __forceinline__ double block_total(float v, double *red) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[wid] = (double)v;
    __syncthreads();
    double s = 0.0;
    if (wid == 0) s = warp0_tree_f64(red, lane);
    return s;
}

// The same sum (FP32 warp sums, FP64 across the warps) for callers in which a
// __syncthreads separates consecutive calls: no barrier before the warp sums are staged,
// and one conversion to FP64 per warp sum in warp kWarp only.  Valid in its lane 0.
template <int kWarp = 0>
__device__ __forceinline__ double block_sum(float v, float *redf) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) redf[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (wid == kWarp) {
        s = lane < (int)(blockDim.x >> 5) ? (double)redf[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(FULL, s, o);
    }
    return s;
}

__device__ __forceinline__ float4 f4add(float4 a, float4 b) { return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w); }


// Tensor memory of a persistent position-step CTA: all kPcgTmemCols columns (one CTA per
// SM), allocated by warp 0; returns the base address
__device__ __forceinline__ uint32_t pcg_tmem_alloc(uint32_t *slot) {
    if (threadIdx.x < 32) {  // one SM per CTA: the columns are free
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         (uint32_t)__cvta_generic_to_shared(slot)),
                     "r"(kPcgTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    return *slot;
}
__device__ __forceinline__ void pcg_tmem_free(uint32_t tmem) {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x < 32) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kPcgTmemCols));
}

// One position step (Sec. 7.1) of one lattice by a group of G co-resident CTAs, this one
// being number bid of the group; tmem: the CTA's tensor memory (kPcgTmemCols columns).
// Returns with the CTA synchronised (its shared and tensor memory free for reuse).
// kPad: 0, a brick that tiles the lattice with 16-byte-aligned rows; otherwise a padded
// brick (rows of ax.lx slots in shared memory, nx of them real; ragged bricks at the far
// faces; the padding elements stay zero and take no part in the stencil or the sums):
// 1 where nx % 4 == 0 (global rows still 16-byte aligned), 2 where not (global vectors
// then read and written element by element).
template <bool kAll, bool kVec4, int kPad = 0>
__device__ __forceinline__ void pcg_persistent_body(const Ctx &c, Scal *sc, const PcgAux &ax, int K, double tol2,
                                                    int apply, const unsigned bid, const unsigned G,
                                                    const uint32_t tmem) {
    // Two grid barriers per iteration.  Phase A forms p = z + beta p_old itself (own
    // slots in shared memory; a remote neighbour's from its published z and p_old), so
    // no barrier is needed after the p update:
    //   A: the p update (own), q = 2 w_r L p (stencil warps) | samples' J^T J p (other
    //      warps)
    //   -- barrier + sum p.Ap --
    //   B: r -= alpha q, z = Minv r (published), r.z
    //   -- barrier + sum r.z; meanwhile x += alpha p (stencil warps) --
    // The first thread of the sample warps (kLead) arrives at the barriers and waits, so
    // that the stencil warps are free to update x during the second wait.
    // p, z / q and Minv of own slots live in shared memory, r and x in tensor memory
    // (each thread keeps the r of the groups it updates in phase B and the x of those it
    // updates in A1).  Global buffers: c.minv (the diagonal on entry, Minv on return),
    // c.r (z, published; holds b on entry), ax.pbuf (p of even / odd iterations), c.q
    // (the samples' contributions), c.x (result, written at the end).
    extern __shared__ float4 sm4[];
    __shared__ float redf[32];
    __shared__ int s_js, s_je, s_go;
    // per own float4 group: 1 if another CTA reads its p and z (a brick-face row, a slot
    // that a sample or a sparse pair touches, or any slot of a contiguous range)
    __shared__ unsigned s_pub[kPcgMaxGroups * kPcgThreads / 32];
    // per own float4 group: 1 if a sample or a sparse pair touches one of its slots (its
    // J^T J p contributions arrive in c.q)
    __shared__ unsigned s_touch[kPcgMaxGroups * kPcgThreads / 32];
    __shared__ float s_ab;
    float *sm = reinterpret_cast<float *>(sm4);
    const int chunk = ax.chunk;
    float *__restrict__ P = sm;               // p of own slots
    float *__restrict__ Q = sm + 3 * chunk;   // z between phases B and A, q within A..B
    float *__restrict__ M = sm + 6 * chunk;   // Minv of own slots
    // the published and accumulated vectors (z, p, the samples' q): at the node's slot, or
    // for a padded brick with unaligned rows (kPad == 2) in ax.zpad, ax.pbuf and ax.qpad at
    // x + lx (y + ny z) (plane stride ax.ldp), where every group is one aligned float4
    float *__restrict__ Zg = kPad == 2 ? ax.zpad : c.r;
    float *__restrict__ Qg = kPad == 2 ? ax.qpad : c.q;
    if (sc->skip) return;  // the same flag for every CTA: none reaches a barrier
    const int N = active_count<kAll>(c);
    const int N4 = 4 * groups4(N);
    // own slots: a brick of full x-rows (local index l = x + lx (row), row = yl + by zl)
    // or the contiguous range [s_beg, s_end) (local index l = slot - s_beg)
    static_assert(!kPad || (kAll && kVec4), "padded bricks are all-nodes bricks");
    const bool brick = kVec4 && ax.by > 0;
    const int nx = c.nx, plane = c.nx * c.ny;
    const int lx = kPad ? ax.lx : nx;
    const int nby = brick ? (c.ny + ax.by - 1) / ax.by : 1;
    const int y0 = brick ? (int)(bid % nby) * ax.by : 0, z0 = brick ? (int)(bid / nby) * ax.bz : 0;
    // rows of the brick that exist (fewer than by x bz in a ragged brick)
    const int byA = kPad ? min(ax.by, c.ny - y0) : ax.by, bzA = kPad ? min(ax.bz, c.nz - z0) : ax.bz;
    const int s_beg = brick ? 0 : bid * chunk;
    const int s_end = brick ? 0 : min(s_beg + chunk, N4);
    const int ng = brick ? chunk >> 2 : (s_end > s_beg ? (s_end - s_beg) >> 2 : 0);
    auto gslot = [&](int l) -> int {
        if (!brick) return s_beg + l;
        const int r = fast_div(l, ax.m_nx), rz = fast_div(r, ax.m_by);
        return (l - r * lx) + nx * (y0 + (r - rz * ax.by)) + plane * (z0 + rz);
    };
    // real elements of the group at local index l: 4, or (padded brick) 0 in a row past
    // the lattice and min(4, nx - x) at the end of a row
    auto gvalid = [&](int l) -> int {
        if (!kPad) return 4;
        const int r = fast_div(l, ax.m_nx), rz = fast_div(r, ax.m_by);
        if (r - rz * ax.by >= byA || rz >= bzA) return 0;
        return min(4, nx - (l - r * lx));
    };
    // a group of a global vector at slot s: one 16-byte access (nv is then 0 or 4), or
    // element by element where the rows are not 16-byte aligned (kPad == 2; elements past
    // nv read as zero and are not written)
    auto gld = [&](const float *p, int nv) -> float4 {
        if constexpr (kPad == 2) {
            float v[4];
#pragma unroll
            for (int e = 0; e < 4; e++) v[e] = e < nv ? __ldcg(p + e) : 0.f;
            return make_float4(v[0], v[1], v[2], v[3]);
        } else {
            return nv > 0 ? __ldcg(reinterpret_cast<const float4 *>(p)) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
    };
    auto gst = [&](float *p, int nv, float4 v) {
        if constexpr (kPad == 2) {
            const float a4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int e = 0; e < 4; e++)
                if (e < nv) p[e] = a4[e];
        } else {
            if (nv > 0) *reinterpret_cast<float4 *>(p) = v;
        }
    };
    const int tid = threadIdx.x;
    const float w2 = 2.f * c.w_r;
    const size_t ld = c.ld;
    const size_t ldg = kPad == 2 ? (size_t)ax.ldp : ld;
    const int pln = kPad == 2 ? lx * c.ny : plane;  // z stride of that layout
    auto pslot = [&](int l) -> int {  // a group's slot in that layout
        if constexpr (kPad != 2) {
            return gslot(l);
        } else {
            const int r = fast_div(l, ax.m_nx), rz = fast_div(r, ax.m_by);
            return (l - r * lx) + lx * (y0 + (r - rz * ax.by)) + pln * (z0 + rz);
        }
    };
    auto pld = [&](const float *p, int nv) -> float4 {
        if constexpr (kPad == 2) return nv > 0 ? __ldcg(reinterpret_cast<const float4 *>(p)) : make_float4(0.f, 0.f, 0.f, 0.f);
        else return gld(p, nv);
    };
    auto pst = [&](float *p, int nv, float4 v) {
        if constexpr (kPad == 2) {
            if (nv > 0) *reinterpret_cast<float4 *>(p) = v;
        } else {
            gst(p, nv, v);
        }
    };

    constexpr unsigned kLead = kPcgStencil;
    constexpr int kLeadWarp = kPcgStencil / 32;
    const uint32_t t_r = tmem + ((uint32_t)(32 * ((tid >> 5) & 3)) << 16) + 64u * (uint32_t)(tid >> 7);
    const uint32_t t_x = t_r + kPcgTmemX;
    if (tid == 0) {  // an equal share of the sorted samples
        const int n_occ = *c.n_occ, ns = n_occ > 0 ? c.occ_beg[n_occ] : 0;
        s_js = (int)(((long long)ns * bid) / G);
        s_je = (int)(((long long)ns * (bid + 1)) / G);
    }
    // ---- init: Minv = 1/diag, r = b, z = Minv r, p_old = 0, x = 0; rho0 = r.z
    float part = 0.f;
    bool pub[kPcgMaxGroups], touch[kPcgMaxGroups];
#pragma unroll
    for (int kk = 0; kk < kPcgMaxGroups; kk++) {
        const int gl = tid + kk * kPcgThreads;
        pub[kk] = touch[kk] = false;
        float4 r3[3];
#pragma unroll
        for (int a = 0; a < 3; a++) r3[a] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (gl < ng) {
            const int l = 4 * gl, s = gslot(l), sp = pslot(l), nv = gvalid(l);
            pub[kk] = true;
            if (brick) {
                const int r = fast_div(l, ax.m_nx), zl = fast_div(r, ax.m_by), yl = r - zl * ax.by;
                pub[kk] = nv > 0 && (yl == 0 || yl == byA - 1 || zl == 0 || zl == bzA - 1);
            }
#pragma unroll
            for (int a = 0; a < 3; a++) {
                const float4 dg = gld(c.minv + a * ld + s, nv);
                const float4 rb = gld(c.r + a * ld + s, nv);
                const float dv[4] = {dg.x, dg.y, dg.z, dg.w}, rv[4] = {rb.x, rb.y, rb.z, rb.w};
                float mi[4], rr[4], z[4];
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    const bool in = kPad ? e < nv : s + e < N;
                    mi[e] = (in && dv[e] > 0.f) ? 1.0f / dv[e] : 0.f;
                    rr[e] = in ? rv[e] : 0.f;
                    z[e] = mi[e] * rr[e];
                    part += rr[e] * z[e];
                }
                const float4 z4 = make_float4(z[0], z[1], z[2], z[3]), zero = make_float4(0.f, 0.f, 0.f, 0.f);
                const float4 mi4 = make_float4(mi[0], mi[1], mi[2], mi[3]);
                gst(c.minv + a * ld + s, nv, mi4);
                *reinterpret_cast<float4 *>(M + a * chunk + l) = mi4;
                r3[a] = make_float4(rr[0], rr[1], rr[2], rr[3]);
                *reinterpret_cast<float4 *>(Q + a * chunk + l) = z4;
                *reinterpret_cast<float4 *>(P + a * chunk + l) = zero;
                pst(Zg + a * ldg + sp, nv, z4);
                pst(ax.pbuf[1] + a * ldg + sp, nv, zero);
            }
            int4 fl;
            if (kPad == 2) {
                fl = make_int4(nv > 0 ? __ldcg(ax.flag + s) : 0, nv > 1 ? __ldcg(ax.flag + s + 1) : 0,
                               nv > 2 ? __ldcg(ax.flag + s + 2) : 0, nv > 3 ? __ldcg(ax.flag + s + 3) : 0);
            } else {
                fl = __ldcg(reinterpret_cast<const int4 *>(ax.flag + s));
            }
            if (fl.x | fl.y | fl.z | fl.w) {  // the samples' contributions arrive here by atomics
#pragma unroll
                for (int a = 0; a < 3; a++) pst(Qg + a * ldg + sp, nv, make_float4(0.f, 0.f, 0.f, 0.f));
                pub[kk] = touch[kk] = true;
            }
        }
        tmem_st12(t_r + 12 * kk, r3);
    }
    if (tid < kPcgStencil) {  // x = 0 (whole warps)
        float4 z3[3];
#pragma unroll
        for (int a = 0; a < 3; a++) z3[a] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int k = 0; k < kPcgStencilGroups; k++) tmem_st12(t_x + 12 * k, z3);
    }
    tmem_wait_st();
#pragma unroll
    for (int kk = 0; kk < kPcgMaxGroups; kk++) {
        const unsigned m = __ballot_sync(FULL, pub[kk]), t = __ballot_sync(FULL, touch[kk]);
        if ((tid & 31) == 0) {
            s_pub[(tid + kk * kPcgThreads) >> 5] = m;
            s_touch[(tid + kk * kPcgThreads) >> 5] = t;
        }
    }
    auto published = [&](int gl) -> bool { return (s_pub[gl >> 5] >> (gl & 31)) & 1u; };
    auto touched_group = [&](int gl) -> bool { return (s_touch[gl >> 5] >> (gl & 31)) & 1u; };
    // The FP64 scalars (rho, the previous p.Ap, tol^2 rho0) live in thread kLead, which takes
    // every decision after a barrier and hands the others alpha or beta (s_ab) and whether
    // to go on (s_go), through the barrier's last __syncthreads.
    double sum = 0.0, rho = 0.0, pq_prev = 0.0, thr = 0.0;
    const unsigned arrivals = G + ax.extra;
    bool ok = grid_reduce<true, kLead>(ax.err, G, arrivals, ax.part, ax.words, block_sum<kLeadWarp>(part, redf), 0.0,
                                       sum, bid,
                                [&](double r0) {
                                    rho = r0;
                                    thr = tol2 * r0;  // the convergence threshold on rho
                                    s_go = pos_finite(r0);
                                    if (bid == 0) scal_rho(sc)[0] = r0;
                                });
    float beta = 0.f;
    int done = 0;
    int stop = !ok || !s_go;
    for (int it = 0; it < K && !stop; it++) {
        // (a select, not an index into the parameter: no local copy of it)
        const float *__restrict__ pold = (it & 1) ? ax.pbuf[0] : ax.pbuf[1];
        float *__restrict__ pnew = (it & 1) ? ax.pbuf[1] : ax.pbuf[0];
        part = 0.f;
        if (tid < kPcgStencil) {
            // ---- A1: p = z + beta p_old for own slots
#pragma unroll 1
            for (int gl = tid; gl < ng; gl += kPcgStencil) {
                const int l = 4 * gl, sp = pslot(l);
                const bool pg = published(gl);
                const int nv = pg ? gvalid(l) : 0;
#pragma unroll
                for (int a = 0; a < 3; a++) {
                    const float4 pv = *reinterpret_cast<const float4 *>(P + a * chunk + l);
                    const float4 zv = *reinterpret_cast<const float4 *>(Q + a * chunk + l);
                    const float4 pn = make_float4(fmaf(beta, pv.x, zv.x), fmaf(beta, pv.y, zv.y),
                                                  fmaf(beta, pv.z, zv.z), fmaf(beta, pv.w, zv.w));
                    *reinterpret_cast<float4 *>(P + a * chunk + l) = pn;
                    if (pg) pst(pnew + a * ldg + sp, nv, pn);
                }
            }
            sub_sync(2, kPcgStencil);
            // ---- A2: q = 2 w_r L p into Q
#pragma unroll 1
            for (int gl = tid; gl < ng; gl += kPcgStencil) {
                const int l = 4 * gl;
                if (kVec4) {
                    int x0, y, z, s0;
                    bool own[4];
                    int loff[4];
                    // s0, offs: the group and its neighbours' offsets in the published layout
                    const int offs[4] = {-lx, lx, -pln, pln};
                    int nv = 4;
                    if (brick) {
                        const int r = fast_div(l, ax.m_nx), zl = fast_div(r, ax.m_by), yl = r - zl * ax.by;
                        x0 = l - r * lx;
                        y = y0 + yl;
                        z = z0 + zl;
                        s0 = x0 + lx * y + pln * z;
                        own[0] = yl > 0;
                        own[1] = yl + 1 < byA;
                        own[2] = zl > 0;
                        own[3] = zl + 1 < bzA;
                        loff[0] = -lx;
                        loff[1] = lx;
                        loff[2] = -ax.by * lx;
                        loff[3] = ax.by * lx;
                        if (kPad) {
                            nv = (yl < byA && zl < bzA) ? min(4, nx - x0) : 0;
                            if (nv <= 0) {  // padding: q = 0
#pragma unroll
                                for (int a = 0; a < 3; a++)
                                    *reinterpret_cast<float4 *>(Q + a * chunk + l) = make_float4(0.f, 0.f, 0.f, 0.f);
                                continue;
                            }
                        }
                    } else {
                        s0 = s_beg + l;
                        x0 = s0 % nx;
                        const int t = s0 / nx;
                        y = t % c.ny;
                        z = t / c.ny;
#pragma unroll
                        for (int k = 0; k < 4; k++) {
                            own[k] = s0 + offs[k] >= s_beg && s0 + offs[k] < s_end;
                            loff[k] = offs[k];
                        }
                    }
                    const bool has[4] = {y > 0, y + 1 < c.ny, z > 0, z + 1 < c.nz};
                    float4 q3[3];  // stored after the three are formed (no store between the loads)
#pragma unroll
                    for (int a = 0; a < 3; a++) {
                        const float *Pa = P + a * chunk;
                        const float *Za = Zg + a * ldg, *Oa = pold + a * ldg;
                        const float4 pc = *reinterpret_cast<const float4 *>(Pa + l);
                        float left = pc.x, right = pc.w;
                        if (x0 > 0)
                            left = (brick || s0 - 1 >= s_beg)
                                       ? Pa[l - 1]
                                       : fmaf(beta, __ldcg(Oa + s0 - 1), __ldcg(Za + s0 - 1));
                        if (x0 + 4 < nx)
                            right = (brick || s0 + 4 < s_end)
                                        ? Pa[l + 4]
                                        : fmaf(beta, __ldcg(Oa + s0 + 4), __ldcg(Za + s0 + 4));
                        float4 d;
                        if (kPad && nv < 4) {  // the end of a row: no edges to the padding
                            const float pv[4] = {pc.x, pc.y, pc.z, pc.w};
                            float dd[4];
#pragma unroll
                            for (int e = 0; e < 4; e++) {
                                const float lf = e == 0 ? left : pv[e - 1];
                                const float rt = (e < 3 && e + 1 < nv) ? pv[e + 1] : pv[e];
                                dd[e] = e < nv ? (pv[e] - lf) + (pv[e] - rt) : 0.f;
                            }
                            d = make_float4(dd[0], dd[1], dd[2], dd[3]);
                        } else {
                            d = make_float4((pc.x - left) + (pc.x - pc.y), (pc.y - pc.x) + (pc.y - pc.z),
                                            (pc.z - pc.y) + (pc.z - pc.w), (pc.w - pc.z) + (pc.w - right));
                        }
#pragma unroll
                        for (int k = 0; k < 4; k++) {
                            if (!has[k]) continue;
                            const int sj = s0 + offs[k];
                            float4 v;
                            if (own[k]) {
                                v = *reinterpret_cast<const float4 *>(Pa + l + loff[k]);
                            } else {
                                const float4 zz = pld(Za + sj, nv);
                                const float4 oo = pld(Oa + sj, nv);
                                v = make_float4(fmaf(beta, oo.x, zz.x), fmaf(beta, oo.y, zz.y), fmaf(beta, oo.z, zz.z),
                                                fmaf(beta, oo.w, zz.w));
                            }
                            d.x += pc.x - v.x;
                            d.y += pc.y - v.y;
                            d.z += pc.z - v.z;
                            d.w += pc.w - v.w;
                        }
                        d = make_float4(w2 * d.x, w2 * d.y, w2 * d.z, w2 * d.w);
                        q3[a] = d;
                        part += pc.x * d.x + pc.y * d.y + pc.z * d.z + pc.w * d.w;
                    }
#pragma unroll
                    for (int a = 0; a < 3; a++) *reinterpret_cast<float4 *>(Q + a * chunk + l) = q3[a];
                } else {
#pragma unroll
                    for (int e = 0; e < 4; e++) {
                        const int si = s_beg + l + e;  // never a brick here
                        float q3[3] = {0.f, 0.f, 0.f};
                        if (si < N) {
                            int nb[6];
                            neighbours<kAll>(c, si, nb);
                            float pi[3];
#pragma unroll
                            for (int a = 0; a < 3; a++) pi[a] = P[a * chunk + l + e];
#pragma unroll
                            for (int d = 0; d < 6; d++) {
                                const int sj = nb[d];
                                if (sj < 0) continue;
                                const bool own = sj >= s_beg && sj < s_end;
#pragma unroll
                                for (int a = 0; a < 3; a++) {
                                    const float pj = own ? P[a * chunk + (sj - s_beg)]
                                                         : fmaf(beta, __ldcg(pold + a * ldg + sj), __ldcg(Zg + a * ldg + sj));
                                    q3[a] += pi[a] - pj;
                                }
                            }
#pragma unroll
                            for (int a = 0; a < 3; a++) {
                                q3[a] *= w2;
                                part += pi[a] * q3[a];
                            }
                        }
#pragma unroll
                        for (int a = 0; a < 3; a++) Q[a * chunk + l + e] = q3[a];
                    }
                }
            }
        } else {
            // ---- A: the samples' J^T J p into Qg (atomics), p formed from z and p_old
            const int lt = tid - kPcgStencil;
            const VecView pv{Zg, pold, beta};
            if (c.btb) {  // cached B^T B: an equal share of the occupied cells, a warp per cell
                const int n_occ = *c.n_occ;
                const int cb = (int)(((long long)n_occ * bid) / G);
                const int ce = (int)(((long long)n_occ * (bid + 1)) / G);
                for (int ci = cb + (lt >> 5); ci < ce; ci += kPcgSample >> 5)
                    if constexpr (kPad == 2) btb_cell_apply<kAll, true, true>(c, pv, ci, Qg, part, SlotMap{lx, ax.m_nx0, ldg});
                    else btb_cell_apply<kAll, true>(c, pv, ci, Qg, part);
            } else {
                if constexpr (kPad == 2)
                    samples_warp_apply<kAll, true>(c, pv, Qg, s_js, s_je, part, lt, kPcgSample, SlotMap{lx, ax.m_nx0, ldg});
                else
                    samples_warp_apply<kAll>(c, pv, Qg, s_js, s_je, part, lt, kPcgSample);
            }
            // the pairs go to the last warps, which hold the fewest cells
            double pd = 0.0;
            if constexpr (kPad == 2)
                sparse_pairs<kOpApply, kAll, true, true>(c, pv, Qg, nullptr, bid + G * (kPcgSample - 1 - lt),
                                                         G * kPcgSample, part, pd, SlotMap{lx, ax.m_nx0, ldg});
            else
                sparse_pairs<kOpApply, kAll, true>(c, pv, Qg, nullptr, bid + G * (kPcgSample - 1 - lt), G * kPcgSample,
                                                   part, pd);
        }
        ok = grid_reduce<true, kLead>(ax.err, G, arrivals, ax.part + (size_t)(K + 1 + it) * G, ax.words + 1 + 2 * it,
                                      block_sum<kLeadWarp>(part, redf), pq_prev, sum, bid, [&](double pq) {
                                   pq_prev = pq;
                                   s_go = pos_finite(pq);
                                   if (s_go) s_ab = f32_quot(rho, pq);  // alpha
                                   if (bid == 0) scal_pq(sc, K)[it] = pq;
                               });
        if (!ok || !s_go) {
            stop = 1;
            break;
        }
        const float alpha = s_ab;
        // ---- B: r -= alpha q; z = Minv r (Q and published); rho' = r.z
        part = 0.f;
#pragma unroll
        for (int kk = 0; kk < kPcgMaxGroups; kk++) {
            const int gl = tid + kk * kPcgThreads;
            float4 r3[3];
            tmem_ld12(t_r + 12 * kk, r3);  // whole warps
            if (gl < ng) {
                const int l = 4 * gl, sp = pslot(l), nv = gvalid(l);
                // the samples' contributions where they arrive (the group's one global
                // round trip), Minv from shared memory
                const bool touched = touched_group(gl), pg = published(gl);
                float4 qg[3], mv[3];
#pragma unroll
                for (int a = 0; a < 3; a++) {
                    qg[a] = touched ? pld(Qg + a * ldg + sp, nv) : make_float4(0.f, 0.f, 0.f, 0.f);
                    mv[a] = *reinterpret_cast<const float4 *>(M + a * chunk + l);
                }
#pragma unroll
                for (int a = 0; a < 3; a++) {
                    float4 qv = *reinterpret_cast<const float4 *>(Q + a * chunk + l);
                    if (touched) {  // fold in (and clear) the samples' contributions
                        qv = f4add(qv, qg[a]);
                        pst(Qg + a * ldg + sp, nv, make_float4(0.f, 0.f, 0.f, 0.f));
                    }
                    const float4 rv = r3[a];
                    const float4 &mvv = mv[a];
                    const float4 rn = make_float4(fmaf(-alpha, qv.x, rv.x), fmaf(-alpha, qv.y, rv.y),
                                                  fmaf(-alpha, qv.z, rv.z), fmaf(-alpha, qv.w, rv.w));
                    const float4 zn = make_float4(mvv.x * rn.x, mvv.y * rn.y, mvv.z * rn.z, mvv.w * rn.w);
                    r3[a] = rn;
                    *reinterpret_cast<float4 *>(Q + a * chunk + l) = zn;
                    if (pg) pst(Zg + a * ldg + sp, nv, zn);
                    part += rn.x * zn.x + rn.y * zn.y + rn.z * zn.z + rn.w * zn.w;
                }
            }
            tmem_st12(t_r + 12 * kk, r3);
        }
        tmem_wait_st();
        done = it + 1;
        // x += alpha p (x in tensor memory; p is this iteration's until the next A1), by
        // the stencil warps while kLead waits
        auto x_step = [&]() {
            if (tid >= kPcgStencil || alpha == 0.f) return;
#pragma unroll 1
            for (int k = 0; k < kPcgStencilGroups; k++) {  // whole warps (tensor memory)
                const int gl = tid + k * kPcgStencil;
                float4 x3[3];
                tmem_ld12(t_x + 12 * k, x3);
                if (gl < ng) {
                    const int l = 4 * gl;
#pragma unroll
                    for (int a = 0; a < 3; a++) {
                        const float4 pv = *reinterpret_cast<const float4 *>(P + a * chunk + l);
                        x3[a] = make_float4(fmaf(alpha, pv.x, x3[a].x), fmaf(alpha, pv.y, x3[a].y),
                                            fmaf(alpha, pv.z, x3[a].z), fmaf(alpha, pv.w, x3[a].w));
                    }
                }
                tmem_st12(t_x + 12 * k, x3);
            }
            tmem_wait_st();
        };
        ok = grid_reduce<true, kLead>(ax.err, G, arrivals, ax.part + (size_t)(it + 1) * G, ax.words + 2 + 2 * it,
                                      block_sum<kLeadWarp>(part, redf), rho, sum, bid,
                                      [&](double rho1) {
                                          if (bid == 0) scal_rho(sc)[it + 1] = rho1;
                                          // go on unless converged (rho1 = r.Minv r >= 0);
                                          // a next step needs rho1 > 0
                                          s_go = pos_finite(rho1) && !le_nonneg(rho1, thr);
                                          if (s_go) s_ab = f32_quot(rho1, rho);  // beta
                                          rho = rho1;
                                      },
                                      x_step);
        if (!ok || !s_go) {
            stop = 1;
            break;
        }
        beta = s_ab;
    }
    // ---- x (every step added during its second barrier) to c.x; u += x when the step is
    // applied
    if (tid < kPcgStencil) {
#pragma unroll 1
        for (int k = 0; k < kPcgStencilGroups; k++) {
            const int gl = tid + k * kPcgStencil;
            float4 x3[3];
            tmem_ld12(t_x + 12 * k, x3);  // whole warps
            if (gl >= ng) continue;
            const int l = 4 * gl, s = gslot(l), nv = gvalid(l);
#pragma unroll
            for (int a = 0; a < 3; a++) {
                const float4 x4 = x3[a];
                gst(c.x + a * ld + s, nv, x4);
                if (apply) {
                    const float xv[4] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
                    for (int e = 0; e < 4; e++)
                        if (kPad ? e < nv : s + e < N) c.u[a * ld + slot_node<kAll>(c, s + e)] += xv[e];
                }
            }
        }
    }
    if (bid == 0 && tid == 0) {
        sc->cg_done = done;
        sc->stop = stop;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

template <bool kAll, bool kVec4, int kPad = 0>
__global__ void __launch_bounds__(kPcgThreads, 1) k_pcg_persistent(Ctx c, Scal *sc, PcgAux ax, int K, double tol2,
                                                                   int apply) {
    __shared__ uint32_t s_tmem;
    if (sc->skip) return;  // the same flag for every CTA: none reaches a barrier
    const uint32_t tmem = pcg_tmem_alloc(&s_tmem);
    pcg_persistent_body<kAll, kVec4, kPad>(c, sc, ax, K, tol2, apply, blockIdx.x, gridDim.x, tmem);
    pcg_tmem_free(tmem);
}

// ------------------------------------------------------------------ position steps of a batch in waves
//
// The position steps (Sec. 7.1) of many lattices in one cooperative launch of one CTA per
// SM, each lattice's vectors in shared and tensor memory exactly as in k_pcg_persistent.
// A lattice takes a group of G CTAs (the fewest whose slots fit in shared memory); the
// groups are packed into waves of at most gridDim.x CTAs.  CTA b runs, wave after wave,
// the step of the group it belongs to in that wave (plan[w * gridDim.x + b] = {item,
// index in the group}, item -1: none) and then moves on: a group waits only for its own
// CTAs (its own barrier words and partial rows), never for a wave to end, and every CTA
// of a later group is resident, so each group completes.  The items are a kernel
// parameter (constant memory): the step reads its lattice's fields there as
// k_pcg_persistent reads its own, without holding them in registers.
struct PcgWaveItem {
    Ctx c;
    PcgAux ax;
    Scal *sc;   // the lattice's scalar block of this Gauss-Newton iteration
    int G;      // CTAs of the lattice's group
    int pad;
};
constexpr int kWaveMaxItems = 56;  // lattices per launch (kernel parameters are limited to 32 KB)
struct PcgWaveArgs {
    PcgWaveItem it[kWaveMaxItems];
};
static_assert(sizeof(PcgWaveArgs) + 64 <= 32764, "the items fit in the kernel parameters");

template <bool kAll, bool kVec4, int kPad = 0>
__global__ void __launch_bounds__(kPcgThreads, 1) k_pcg_wave(const __grid_constant__ PcgWaveArgs args,
                                                              const int2 *__restrict__ plan, int waves, int K,
                                                              double tol2, int apply) {
    __shared__ uint32_t s_tmem;
    const uint32_t tmem = pcg_tmem_alloc(&s_tmem);
    for (int w = 0; w < waves; w++) {
        const int2 a = plan[(size_t)w * gridDim.x + blockIdx.x];
        if (a.x < 0) continue;
        const PcgWaveItem &it = args.it[a.x];
        pcg_persistent_body<kAll, kVec4, kPad>(it.c, it.sc, it.ax, K, tol2, apply, (unsigned)a.y, (unsigned)it.G, tmem);
        // every thread is done with this step's shared and tensor memory
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    pcg_tmem_free(tmem);
}

// ------------------------------------------------------------------ batched position step (config 4)
//
// One cooperative launch runs the position step (Sec. 7.1) of every lattice of a batch.
// The CTAs form one group per lattice (first CTA g0, G CTAs); each group runs the PCG
// recurrence of k_pcg_persistent on its own lattice, with its own barrier words and FP64
// partial rows, and never waits on another group.  The vectors stay in global memory (a
// batch holds millions of nodes, more than the SMs' shared memory): each CTA owns a
// contiguous range of the lattice's slots (a multiple of 4) and an equal share of its
// sorted samples.  Per iteration:
//   A: p = z + beta p_old for own slots (published), q_s = 2 w_r L p into qs (the
//      neighbours' p formed from their published z and p_old, so no barrier is needed
//      for p), the samples' and sparse pairs' J^T J p into the lattice's q by atomics,
//      partial p.Ap -- group barrier + sum --
//   B: x += alpha p, r -= alpha (q_s + q) (q cleared for the next iteration), z = Minv r
//      (published), partial r.z -- group barrier + sum.
struct PcgBatchItem {
    Ctx c;                      // the lattice (slot-indexed vectors, samples, pairs)
    Scal *sc;                   // this Gauss-Newton iteration's scalar block
    double *part;               // (2K + 2) rows of G partials
    unsigned long long *words;  // 2K + 1 barrier words, zeroed before the launch
    float *z, *qs, *pbuf1;      // published z, stencil q, p of odd iterations (3 ld each)
    int *err;                   // the lattice's error word (set when a barrier wait gives up)
    int g0, G, chunk, pad;
    // n / nx and n / ny as (2 n m) >> 32 with m = ceil(2^31 / d), exact for n d < 2^31
    // (a slot over nx, then that quotient over ny)
    unsigned m_nx, m_ny;
};
constexpr int kBatchTsm = 8192;  // samples per CTA whose factors the sample phase keeps

template <bool kAll>
__device__ __forceinline__ float batch_p(const PcgBatchItem &B, const float *pold, float beta, size_t i) {
    return fmaf(beta, __ldcg(pold + i), __ldcg(B.z + i));
}

template <bool kAll>
__device__ void pcg_batch_body(const PcgBatchItem &B, unsigned bid, int K, double tol2, int apply, double *red,
                               float *tsm, int *s_rng, float *s_ab) {
    const Ctx &c = B.c;
    int *err = B.err;
    Scal *sc = B.sc;
    if (sc->skip) return;  // the same flag in every CTA of the group
    const unsigned G = B.G;
    const int N = active_count<kAll>(c);
    const int N4 = 4 * groups4(N);
    const int s_beg = (int)bid * B.chunk, s_end = min(s_beg + B.chunk, N4);
    const int ng = s_end > s_beg ? (s_end - s_beg) >> 2 : 0;
    const size_t ld = c.ld;
    const int tid = threadIdx.x, nt = blockDim.x;
    const float w2 = 2.f * c.w_r;
    const bool vec4 = kAll && (c.nx % 4 == 0);
    if (tid == 0) {  // an equal share of the sorted samples and the occupied cells holding them
        const int n_occ = *c.n_occ, ns = n_occ > 0 ? c.occ_beg[n_occ] : 0;
        const int js = (int)(((long long)ns * bid) / G), je = (int)(((long long)ns * (bid + 1)) / G);
        int lo = 0, hi = n_occ;
        while (lo < hi) {
            const int m = (lo + hi) >> 1;
            if (c.occ_beg[m + 1] <= js) lo = m + 1;
            else hi = m;
        }
        s_rng[0] = lo;
        hi = n_occ;
        while (lo < hi) {
            const int m = (lo + hi) >> 1;
            if (c.occ_beg[m] < je) lo = m + 1;
            else hi = m;
        }
        s_rng[1] = je > js ? lo : s_rng[0];
        s_rng[2] = js;
        s_rng[3] = je;
    }
    // ---- init: Minv = 1/diag, z = Minv r, p_old = 0, x = 0, q = 0; rho0 = r.z
    float part = 0.f;
    for (int gl = tid; gl < ng; gl += nt) {
        const int s = s_beg + 4 * gl;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const size_t o = a * ld + s;
            const float4 dg = *reinterpret_cast<const float4 *>(c.minv + o);
            const float4 rb = *reinterpret_cast<const float4 *>(c.r + o);
            const float dv[4] = {dg.x, dg.y, dg.z, dg.w}, rv[4] = {rb.x, rb.y, rb.z, rb.w};
            float mi[4], rr[4], z[4];
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const bool in = s + e < N;
                mi[e] = (in && dv[e] > 0.f) ? 1.0f / dv[e] : 0.f;
                rr[e] = in ? rv[e] : 0.f;
                z[e] = mi[e] * rr[e];
                part += rr[e] * z[e];
            }
            const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
            *reinterpret_cast<float4 *>(c.minv + o) = make_float4(mi[0], mi[1], mi[2], mi[3]);
            *reinterpret_cast<float4 *>(c.r + o) = make_float4(rr[0], rr[1], rr[2], rr[3]);
            *reinterpret_cast<float4 *>(B.z + o) = make_float4(z[0], z[1], z[2], z[3]);
            *reinterpret_cast<float4 *>(B.pbuf1 + o) = zero;
            *reinterpret_cast<float4 *>(c.x + o) = zero;
            *reinterpret_cast<float4 *>(c.q + o) = zero;
        }
    }
    double sum = 0.0;
    bool ok = grid_reduce(err, G, G, B.part, B.words, block_total(part, red), 0.0, sum, bid);
    const double rho0 = ok ? sum : 0.0;
    double rho = rho0, pq_prev = 0.0;
    float beta = 0.f;
    if (bid == 0 && tid == 0) scal_rho(sc)[0] = rho0;
    int done = 0, stop = !ok;
    const int cb = s_rng[0], ce = s_rng[1], js = s_rng[2], je = s_rng[3];
    for (int it = 0; it < K && !stop; it++) {
        if (!(rho > 0.0)) {
            stop = 1;
            break;
        }
        const float *__restrict__ pold = (it & 1) ? c.p : B.pbuf1;
        float *__restrict__ pnew = (it & 1) ? B.pbuf1 : c.p;
        part = 0.f;
        // ---- A1 + A2: own p (published) and the stencil q_s = 2 w_r L p
        for (int gl = tid; gl < ng; gl += nt) {
            const int s0 = s_beg + 4 * gl;
            if (vec4) {
                const int x0 = s0 % c.nx, t = s0 / c.nx, y = t % c.ny, z = t / c.ny, pl = c.nx * c.ny;
                const int offs[4] = {-c.nx, c.nx, -pl, pl};
                const bool has[4] = {y > 0, y + 1 < c.ny, z > 0, z + 1 < c.nz};
#pragma unroll
                for (int a = 0; a < 3; a++) {
                    const size_t o = a * ld;
                    const float4 zz = __ldcg(reinterpret_cast<const float4 *>(B.z + o + s0));
                    const float4 oo = __ldcg(reinterpret_cast<const float4 *>(pold + o + s0));
                    const float4 pc = make_float4(fmaf(beta, oo.x, zz.x), fmaf(beta, oo.y, zz.y), fmaf(beta, oo.z, zz.z),
                                                  fmaf(beta, oo.w, zz.w));
                    *reinterpret_cast<float4 *>(pnew + o + s0) = pc;
                    const float left = x0 > 0 ? batch_p<kAll>(B, pold, beta, o + s0 - 1) : pc.x;
                    const float right = x0 + 4 < c.nx ? batch_p<kAll>(B, pold, beta, o + s0 + 4) : pc.w;
                    float4 d = make_float4((pc.x - left) + (pc.x - pc.y), (pc.y - pc.x) + (pc.y - pc.z),
                                           (pc.z - pc.y) + (pc.z - pc.w), (pc.w - pc.z) + (pc.w - right));
#pragma unroll
                    for (int k = 0; k < 4; k++) {
                        if (!has[k]) continue;
                        const float4 z4 = __ldcg(reinterpret_cast<const float4 *>(B.z + o + s0 + offs[k]));
                        const float4 o4 = __ldcg(reinterpret_cast<const float4 *>(pold + o + s0 + offs[k]));
                        d.x += pc.x - fmaf(beta, o4.x, z4.x);
                        d.y += pc.y - fmaf(beta, o4.y, z4.y);
                        d.z += pc.z - fmaf(beta, o4.z, z4.z);
                        d.w += pc.w - fmaf(beta, o4.w, z4.w);
                    }
                    d = make_float4(w2 * d.x, w2 * d.y, w2 * d.z, w2 * d.w);
                    *reinterpret_cast<float4 *>(B.qs + o + s0) = d;
                    part += pc.x * d.x + pc.y * d.y + pc.z * d.z + pc.w * d.w;
                }
            } else {  // A1 only here: the stencil follows once every own p is published
#pragma unroll
                for (int a = 0; a < 3; a++) {
                    const size_t o = a * ld + s0;
                    const float4 zz = __ldcg(reinterpret_cast<const float4 *>(B.z + o));
                    const float4 oo = __ldcg(reinterpret_cast<const float4 *>(pold + o));
                    *reinterpret_cast<float4 *>(pnew + o) = make_float4(fmaf(beta, oo.x, zz.x), fmaf(beta, oo.y, zz.y),
                                                                        fmaf(beta, oo.z, zz.z), fmaf(beta, oo.w, zz.w));
                }
            }
        }
        if (!vec4) {
            // A2 slot by slot (coalesced across the threads): a neighbour in this CTA's range
            // reads the p just published (visible to the block after the barrier), another
            // CTA's is formed from its z and p_old
            __syncthreads();
            for (int si = s_beg + tid; si < s_end; si += nt) {
                float pi[3], q3[3] = {0.f, 0.f, 0.f};
#pragma unroll
                for (int a = 0; a < 3; a++) pi[a] = pnew[a * ld + si];
                if (si < N) {
                    int nb[6];
                    if (kAll) {
                        const int x = (int)(__umulhi(2u * (unsigned)si, B.m_nx));  // si / nx
                        const int xr = si - x * c.nx;
                        const int pl = c.nx * c.ny;
                        const int zq = (int)(__umulhi(2u * (unsigned)x, B.m_ny));  // (si / nx) / ny
                        const int yq = x - zq * c.ny;
                        nb[0] = xr > 0 ? si - 1 : -1;
                        nb[1] = xr + 1 < c.nx ? si + 1 : -1;
                        nb[2] = yq > 0 ? si - c.nx : -1;
                        nb[3] = yq + 1 < c.ny ? si + c.nx : -1;
                        nb[4] = zq > 0 ? si - pl : -1;
                        nb[5] = zq + 1 < c.nz ? si + pl : -1;
                    } else {
                        neighbours<kAll>(c, si, nb);
                    }
#pragma unroll
                    for (int d = 0; d < 6; d++) {
                        const int sj = nb[d];
                        if (sj < 0) continue;
                        const bool own = sj >= s_beg && sj < s_end;
#pragma unroll
                        for (int a = 0; a < 3; a++)
                            q3[a] += pi[a] - (own ? pnew[a * ld + sj] : batch_p<kAll>(B, pold, beta, a * ld + sj));
                    }
#pragma unroll
                    for (int a = 0; a < 3; a++) {
                        q3[a] *= w2;
                        part += pi[a] * q3[a];
                    }
                }
#pragma unroll
                for (int a = 0; a < 3; a++) B.qs[a * ld + si] = q3[a];
            }
        }
        // ---- A3: the samples' and sparse pairs' J^T J p (p formed from z and p_old): the
        // cached blocks (an equal share of the occupied cells, a warp per cell) where the
        // lattice has them, else the samples themselves
        const VecView pv{B.z, pold, beta};
        if (c.btb) {
            const int n_occ = *c.n_occ;
            const int cb2 = (int)(((long long)n_occ * bid) / G), ce2 = (int)(((long long)n_occ * (bid + 1)) / G);
            for (int ci = cb2 + (tid >> 5); ci < ce2; ci += nt >> 5) btb_cell_apply<kAll, true>(c, pv, ci, c.q, part);
        } else if (ce > cb) {
            cells_block<kOpApply, kAll, true>(c, pv, c.q, nullptr, cb, ce, tsm, kBatchTsm, part, tid, nt, 0, js, je);
        }
        double pd = 0.0;
        sparse_pairs<kOpApply, kAll, true>(c, pv, c.q, nullptr, bid + G * tid, G * nt, part, pd);
        ok = grid_reduce(err, G, G, B.part + (size_t)(K + 1 + it) * G, B.words + 1 + 2 * it, block_total(part, red),
                         pq_prev, sum, bid);
        if (!ok) {
            stop = 1;
            break;
        }
        const double pq = sum;
        pq_prev = pq;
        if (!(pq > 0.0)) {
            stop = 1;
            break;
        }
        if (tid == 0) {
            *s_ab = (float)(rho / pq);
            if (bid == 0) scal_pq(sc, K)[it] = pq;
        }
        __syncthreads();
        const float alpha = *s_ab;
        // ---- B: x += alpha p, r -= alpha (q_s + q), q = 0, z = Minv r (published); r.z
        part = 0.f;
        for (int gl = tid; gl < ng; gl += nt) {
            const int s = s_beg + 4 * gl;
#pragma unroll
            for (int a = 0; a < 3; a++) {
                const size_t o = a * ld + s;
                const float4 pv4 = *reinterpret_cast<const float4 *>(pnew + o);
                const float4 q1 = *reinterpret_cast<const float4 *>(B.qs + o);
                const float4 q2 = __ldcg(reinterpret_cast<const float4 *>(c.q + o));
                const float4 rv = *reinterpret_cast<const float4 *>(c.r + o);
                const float4 mv = *reinterpret_cast<const float4 *>(c.minv + o);
                const float4 xv = *reinterpret_cast<const float4 *>(c.x + o);
                *reinterpret_cast<float4 *>(c.q + o) = make_float4(0.f, 0.f, 0.f, 0.f);
                const float4 qv = f4add(q1, q2);
                *reinterpret_cast<float4 *>(c.x + o) = make_float4(fmaf(alpha, pv4.x, xv.x), fmaf(alpha, pv4.y, xv.y),
                                                                   fmaf(alpha, pv4.z, xv.z), fmaf(alpha, pv4.w, xv.w));
                const float4 rn = make_float4(fmaf(-alpha, qv.x, rv.x), fmaf(-alpha, qv.y, rv.y),
                                              fmaf(-alpha, qv.z, rv.z), fmaf(-alpha, qv.w, rv.w));
                const float4 zn = make_float4(mv.x * rn.x, mv.y * rn.y, mv.z * rn.z, mv.w * rn.w);
                *reinterpret_cast<float4 *>(c.r + o) = rn;
                *reinterpret_cast<float4 *>(B.z + o) = zn;
                part += rn.x * zn.x + rn.y * zn.y + rn.z * zn.z + rn.w * zn.w;
            }
        }
        done = it + 1;
        ok = grid_reduce(err, G, G, B.part + (size_t)(it + 1) * G, B.words + 2 + 2 * it, block_total(part, red), rho, sum,
                         bid);
        if (!ok) {
            stop = 1;
            break;
        }
        const double rho1 = sum;
        if (bid == 0 && tid == 0) scal_rho(sc)[it + 1] = rho1;
        if (rho1 <= tol2 * rho0) {
            stop = 1;
            break;
        }
        if (tid == 0) *s_ab = (float)(rho1 / rho);
        __syncthreads();
        beta = *s_ab;
        rho = rho1;
    }
    // ---- u += x when the step is applied
    if (apply)
        for (int gl = tid; gl < ng; gl += nt) {
            const int s = s_beg + 4 * gl;
#pragma unroll
            for (int a = 0; a < 3; a++)
#pragma unroll
                for (int e = 0; e < 4; e++)
                    if (s + e < N) c.u[a * ld + slot_node<kAll>(c, s + e)] += c.x[a * ld + s + e];
        }
    if (bid == 0 && tid == 0) {
        sc->cg_done = done;
        sc->stop = stop;
    }
}

template <int kThreadsB>
__global__ void __launch_bounds__(kThreadsB) k_pcg_batch(const PcgBatchItem *__restrict__ items, int n_items, int K,
                                                          double tol2, int apply) {
    __shared__ PcgBatchItem s_it;
    __shared__ double red[32];
    __shared__ float tsm[kBatchTsm];
    __shared__ int s_rng[4];
    __shared__ float s_ab;
    if (threadIdx.x == 0) {  // the CTA's group: the last item whose first CTA is at or before this one
        int lo = 0, hi = n_items;
        while (hi - lo > 1) {
            const int m = (lo + hi) >> 1;
            if (items[m].g0 <= (int)blockIdx.x) lo = m;
            else hi = m;
        }
        s_it = items[lo];
    }
    __syncthreads();
    const unsigned bid = blockIdx.x - (unsigned)s_it.g0;
    if (s_it.c.slot_of_node) pcg_batch_body<false>(s_it, bid, K, tol2, apply, red, tsm, s_rng, &s_ab);
    else pcg_batch_body<true>(s_it, bid, K, tol2, apply, red, tsm, s_rng, &s_ab);
}

// ------------------------------------------------------------------ rotation step (Sec. 7.1)

// Largest-eigenvalue eigenvector of a symmetric 4x4 matrix by cyclic Jacobi
// rotations (Golub & Van Loan, Sec. 8.5); returns lambda_1 - lambda_2.
template <typename T>
__device__ __forceinline__ T sym4_top_eigvec(T a[4][4], T q[4]) {
    const T one = T(1), zero = T(0);
    T v[4][4];
#pragma unroll
    for (int r = 0; r < 4; r++)
#pragma unroll
        for (int s = 0; s < 4; s++) v[r][s] = r == s ? one : zero;
#pragma unroll 1
    for (int sweep = 0; sweep < 8; sweep++) {
        T off = zero, dia = zero;
#pragma unroll
        for (int r = 0; r < 4; r++) {
            dia += a[r][r] * a[r][r];
#pragma unroll
            for (int s = r + 1; s < 4; s++) off += a[r][s] * a[r][s];
        }
        if (off <= (sizeof(T) == 4 ? T(1e-12) : T(1e-28)) * dia) break;  // near the rounding floor
#pragma unroll
        for (int pp = 0; pp < 3; pp++)
#pragma unroll
            for (int qq = pp + 1; qq < 4; qq++) {
                const T apq = a[pp][qq];
                if (apq == zero) continue;
                const T th = (a[qq][qq] - a[pp][pp]) / (T(2) * apq);
                const T t = (th >= zero ? one : -one) / (fabs(th) + sqrt(th * th + one));
                const T cs = one / sqrt(t * t + one), sn = t * cs;
                // A <- J^T A J with J the rotation in the (pp, qq) plane
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const T akp = a[k][pp], akq = a[k][qq];
                    a[k][pp] = cs * akp - sn * akq;
                    a[k][qq] = sn * akp + cs * akq;
                }
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const T apk = a[pp][k], aqk = a[qq][k];
                    a[pp][k] = cs * apk - sn * aqk;
                    a[qq][k] = sn * apk + cs * aqk;
                }
#pragma unroll
                for (int k = 0; k < 4; k++) {
                    const T vkp = v[k][pp], vkq = v[k][qq];
                    v[k][pp] = cs * vkp - sn * vkq;
                    v[k][qq] = sn * vkp + cs * vkq;
                }
            }
    }
    // top eigenpair without dynamic register indexing
    T l1 = a[0][0], l2 = T(-3.4e38);
#pragma unroll
    for (int r = 0; r < 4; r++) q[r] = v[r][0];
#pragma unroll
    for (int k = 1; k < 4; k++) {
        const T lk = a[k][k];
        if (lk > l1) {
            l2 = l1;
            l1 = lk;
#pragma unroll
            for (int r = 0; r < 4; r++) q[r] = v[r][k];
        } else if (lk > l2) {
            l2 = lk;
        }
    }
    return l1 - l2;
}

// unit quaternion (w, x, y, z) of a rotation matrix (Shepperd 1978: divide by the
// largest of the four diagonal combinations)
__device__ __forceinline__ void mat_to_quat(const float R[9], float q[4]) {
    const float tr = R[0] + R[4] + R[8];
    if (tr >= R[0] && tr >= R[4] && tr >= R[8]) {
        const float w = 0.5f * sqrtf(fmaxf(1.f + tr, 0.f)), s = 0.25f / w;
        q[0] = w; q[1] = (R[7] - R[5]) * s; q[2] = (R[2] - R[6]) * s; q[3] = (R[3] - R[1]) * s;
    } else if (R[0] >= R[4] && R[0] >= R[8]) {
        const float x = 0.5f * sqrtf(fmaxf(1.f + R[0] - R[4] - R[8], 0.f)), s = 0.25f / x;
        q[0] = (R[7] - R[5]) * s; q[1] = x; q[2] = (R[1] + R[3]) * s; q[3] = (R[2] + R[6]) * s;
    } else if (R[4] >= R[8]) {
        const float y = 0.5f * sqrtf(fmaxf(1.f + R[4] - R[0] - R[8], 0.f)), s = 0.25f / y;
        q[0] = (R[2] - R[6]) * s; q[1] = (R[1] + R[3]) * s; q[2] = y; q[3] = (R[5] + R[7]) * s;
    } else {
        const float z = 0.5f * sqrtf(fmaxf(1.f + R[8] - R[0] - R[4], 0.f)), s = 0.25f / z;
        q[0] = (R[3] - R[1]) * s; q[1] = (R[2] + R[6]) * s; q[2] = (R[5] + R[7]) * s; q[3] = z;
    }
}

// Per node: A_i = sum_{j in N_i} (t_i - t_j)(t^_i - t^_j)^T (scaled by 1/h^2), and
// R_i = argmax_R tr(R^T A_i) through the unit quaternion of Horn's 4x4 matrix
// (Horn 1987, closed-form absolute orientation).  Nodes whose neighbours span fewer
// than two axes, or whose top eigenvalue is (numerically) double, keep R_i.
// Warm start: with the previous rotation R0 (orthonormal), argmax_R tr(R^T A) =
// R0 argmax_D tr(D^T R0^T A), and the top eigenvector of Horn's matrix of R0^T A is near
// the identity quaternion when the rotation changed little, so a Rayleigh-quotient
// iteration from the identity converges in one or two steps (cyclic Jacobi is the
// fallback); R = R0 D is formed from the product of unit quaternions, which keeps it
// orthonormal.  k_fit_rotations (below the eigen-solvers) also accumulates E_reg
// (Eq. 4) with the new rotations (kFit = false: E_reg only).
// Top eigenvector of a symmetric 4x4 matrix by Rayleigh-quotient iteration from q
// (cubic convergence near an eigenvector), with a certificate: true only if
// M = (mu - delta) I - N + 2 delta q q^T is positive definite (Cholesky), which holds
// exactly when mu = q^T N q is the largest eigenvalue and every other one lies below
// mu - delta.  On false the caller falls back to the Jacobi solve.
// The iteration stops once |N q - mu q| <= 1e-6 max|N| (FP32 rounding level), after at
// most three steps; if it has not got there by then (a warm start far from the answer)
// the result is not used.  The certificate's gap is raised to 1e5 |N q - mu q| when that
// exceeds `delta`: the eigenvector's angular error is at most the residual over the gap
// (Davis-Kahan), so an accepted q is within 1e-5 rad of the top eigenvector.
// Each step solves (N - mu I) y = q through the Schur complement of
// the leading entry: writing N - mu I = [[m, b^T], [b, C]] (C the trailing 3x3 block),
//   S = m det C - b^T adj(C) b  (= det(N - mu I)),  y0' = q0 det C - b^T adj(C) q_r,
//   y  ~  (y0' det C,  S adj(C) q_r - y0' adj(C) b)
// (the solution times det C * S; the sign and the scale drop out in the normalisation).
// The step needs neither division nor pivoting, only C nonsingular: by interlacing
// that holds while the top eigenvector keeps a component along the first axis, as it
// does for the rotation increments of the warm-started fit; otherwise the step yields
// no usable direction and the certificate fails.
__device__ __forceinline__ bool sym4_top_rqi(const float N[4][4], float q[4], float delta, float scale) {
    const float tol2 = 1e-12f * scale * scale;
    float mu = 0.f, res2 = 0.f;
#pragma unroll 1
    for (int it = 0;; it++) {
        float Nq[4];
#pragma unroll
        for (int r = 0; r < 4; r++) Nq[r] = N[r][0] * q[0] + N[r][1] * q[1] + N[r][2] * q[2] + N[r][3] * q[3];
        mu = q[0] * Nq[0] + q[1] * Nq[1] + q[2] * Nq[2] + q[3] * Nq[3];
        res2 = 0.f;
#pragma unroll
        for (int r = 0; r < 4; r++) res2 += (Nq[r] - mu * q[r]) * (Nq[r] - mu * q[r]);
        if (res2 <= tol2 || it == 3) break;
        const float m = N[0][0] - mu, b1 = N[1][0], b2 = N[2][0], b3 = N[3][0];
        const float c11 = N[1][1] - mu, c12 = N[1][2], c13 = N[1][3];
        const float c22 = N[2][2] - mu, c23 = N[2][3], c33 = N[3][3] - mu;
        // adj(C) (symmetric) and det C
        const float a11 = c22 * c33 - c23 * c23, a12 = c13 * c23 - c12 * c33, a13 = c12 * c23 - c13 * c22;
        const float a22 = c11 * c33 - c13 * c13, a23 = c12 * c13 - c11 * c23, a33 = c11 * c22 - c12 * c12;
        const float dC = c11 * a11 + c12 * a12 + c13 * a13;
        const float zb1 = a11 * b1 + a12 * b2 + a13 * b3, zb2 = a12 * b1 + a22 * b2 + a23 * b3,
                    zb3 = a13 * b1 + a23 * b2 + a33 * b3;
        const float zq1 = a11 * q[1] + a12 * q[2] + a13 * q[3], zq2 = a12 * q[1] + a22 * q[2] + a23 * q[3],
                    zq3 = a13 * q[1] + a23 * q[2] + a33 * q[3];
        const float S = m * dC - (b1 * zb1 + b2 * zb2 + b3 * zb3);
        const float y0 = q[0] * dC - (b1 * zq1 + b2 * zq2 + b3 * zq3);
        const float y[4] = {y0 * dC, S * zq1 - y0 * zb1, S * zq2 - y0 * zb2, S * zq3 - y0 * zb3};
        const float n2 = y[0] * y[0] + y[1] * y[1] + y[2] * y[2] + y[3] * y[3];
        if (!(n2 > 1e-30f) || !isfinite(n2)) break;
        const float sc = rsqrtf(n2);
#pragma unroll
        for (int r = 0; r < 4; r++) q[r] = y[r] * sc;
    }
    if (!(res2 <= tol2)) return false;  // not converged in three steps
    delta = fmaxf(delta, 1e5f * sqrtf(res2));
    // certificate: Cholesky of M (all pivots > 0), reciprocal square roots of the pivots
    float L[4][4], rl[4];
#pragma unroll
    for (int r = 0; r < 4; r++)
#pragma unroll
        for (int k = 0; k <= r; k++) {
            float mm = 2.f * delta * q[r] * q[k] - N[r][k] + (r == k ? mu - delta : 0.f);
#pragma unroll
            for (int j = 0; j < k; j++) mm -= L[r][j] * L[k][j];
            if (r == k) {
                if (!(mm > 0.f)) return false;
                rl[r] = rsqrtf(mm);
                L[r][r] = mm * rl[r];
            } else {
                L[r][k] = mm * rl[k];
            }
        }
    return true;
}

// The Jacobi fallback of the rotation step in FP32 (when the Rayleigh-quotient
// iteration is not certified; rare), out of line so that its registers do not count
// against the fast path's occupancy; returns lambda_1 - lambda_2.
__device__ __noinline__ float horn_top_eigvec_f32(const float (&Nm)[4][4], float qv[4]) {
    float a[4][4];
#pragma unroll
    for (int r = 0; r < 4; r++)
#pragma unroll
        for (int k = 0; k < 4; k++) a[r][k] = Nm[r][k];
    return sym4_top_eigvec<float>(a, qv);
}

// The near-tie redo of the rotation step in FP64 (rare), kept out of line so that its
// registers do not count against the FP32 path's occupancy.
__device__ __noinline__ double horn_top_eigvec_f64(float Sxx, float Sxy, float Sxz, float Syx, float Syy, float Syz,
                                                   float Szx, float Szy, float Szz, float qv[4]) {
    double Nd[4][4] = {{(double)Sxx + Syy + Szz, (double)Syz - Szy, (double)Szx - Sxz, (double)Sxy - Syx},
                       {(double)Syz - Szy, (double)Sxx - Syy - Szz, (double)Sxy + Syx, (double)Szx + Sxz},
                       {(double)Szx - Sxz, (double)Sxy + Syx, -(double)Sxx + Syy - Szz, (double)Syz + Szy},
                       {(double)Sxy - Syx, (double)Szx + Sxz, (double)Syz + Szy, -(double)Sxx - Syy + Szz}};
    double qd[4];
    const double gd = sym4_top_eigvec<double>(Nd, qd);
#pragma unroll
    for (int r = 0; r < 4; r++) qv[r] = (float)qd[r];
    return gd;
}

// The rotation step of one node from A = sum_j (t_i - t_j)(t^_i - t^_j)^T / h^2 (three
// columns, one per axis; at least two axes present): Horn's quaternion warm-started at
// the previous rotation Ri, as described above.  Returns true where the node keeps Ri (no
// certified unique fit); Ri holds the new rotation otherwise.
__device__ __forceinline__ bool fit_node_rotation(const float (&A)[3][3], float (&Ri)[9]) {
    // previous rotation usable as a warm start if orthonormal
    float orth = 0.f;
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const float d = Ri[r] * Ri[k] + Ri[3 + r] * Ri[3 + k] + Ri[6 + r] * Ri[6 + k] - (r == k ? 1.f : 0.f);
            orth = fmaxf(orth, fabsf(d));
        }
    const bool warm = orth < 1e-3f;
    float B[3][3];
#pragma unroll
    for (int r = 0; r < 3; r++)
#pragma unroll
        for (int k = 0; k < 3; k++)
            B[r][k] = warm ? Ri[r] * A[0][k] + Ri[3 + r] * A[1][k] + Ri[6 + r] * A[2][k] : A[r][k];
    // Horn's matrix from S = B^T (S_ab = sum_j e_a d_b)
    const float Sxx = B[0][0], Sxy = B[1][0], Sxz = B[2][0];
    const float Syx = B[0][1], Syy = B[1][1], Syz = B[2][1];
    const float Szx = B[0][2], Szy = B[1][2], Szz = B[2][2];
    float Nm[4][4] = {{Sxx + Syy + Szz, Syz - Szy, Szx - Sxz, Sxy - Syx},
                      {Syz - Szy, Sxx - Syy - Szz, Sxy + Syx, Szx + Sxz},
                      {Szx - Sxz, Sxy + Syx, -Sxx + Syy - Szz, Syz + Szy},
                      {Sxy - Syx, Szx + Sxz, Syz + Szy, -Sxx - Syy + Szz}};
    float scale = 0.f;
#pragma unroll
    for (int r = 0; r < 4; r++)
#pragma unroll
        for (int k = 0; k < 4; k++) scale = fmaxf(scale, fabsf(Nm[r][k]));
    // fast path: Rayleigh-quotient iteration from the identity (the previous
    // rotation when warm), certified unique with a gap above 1e-4 of the scale;
    // otherwise cyclic Jacobi, and FP64 for a near-singular block
    float qv[4] = {1.f, 0.f, 0.f, 0.f};
    bool unique = sym4_top_rqi(Nm, qv, 1e-4f * scale, scale);
    if (!unique) {
        // the out-of-line solvers get copies, so that the fast path's matrix and
        // vector never have their address taken (they stay in registers)
        float Nf[4][4], qf[4];
#pragma unroll
        for (int r = 0; r < 4; r++) {
            qf[r] = qv[r];
#pragma unroll
            for (int k = 0; k < 4; k++) Nf[r][k] = Nm[r][k];
        }
        const float gap = horn_top_eigvec_f32(Nf, qf);
        unique = gap > 1e-5f * scale;
        if (gap < 1e-4f * scale) {
            // near-singular block (the rotation's sensitivity exceeds 1e4): polar
            // decomposition again in FP64
            const double gd = horn_top_eigvec_f64(Sxx, Sxy, Sxz, Syx, Syy, Syz, Szx, Szy, Szz, qf);
            unique = gd > 1e-12 * (double)scale;
        }
#pragma unroll
        for (int r = 0; r < 4; r++) qv[r] = qf[r];
    }
    if (!unique) return true;
    float w = qv[0], x = qv[1], y = qv[2], z = qv[3];
    if (warm) {  // q = q(R0) * q(D)
        float q0[4];
        mat_to_quat(Ri, q0);
        const float w2 = q0[0] * w - q0[1] * x - q0[2] * y - q0[3] * z;
        const float x2 = q0[0] * x + q0[1] * w + q0[2] * z - q0[3] * y;
        const float y2 = q0[0] * y - q0[1] * z + q0[2] * w + q0[3] * x;
        const float z2 = q0[0] * z + q0[1] * y - q0[2] * x + q0[3] * w;
        w = w2;
        x = x2;
        y = y2;
        z = z2;
    }
    const float inv = 1.f / (w * w + x * x + y * y + z * z);
    Ri[0] = (w * w + x * x - y * y - z * z) * inv;
    Ri[1] = 2.f * (x * y - w * z) * inv;
    Ri[2] = 2.f * (x * z + w * y) * inv;
    Ri[3] = 2.f * (x * y + w * z) * inv;
    Ri[4] = (w * w - x * x + y * y - z * z) * inv;
    Ri[5] = 2.f * (y * z - w * x) * inv;
    Ri[6] = 2.f * (x * z - w * y) * inv;
    Ri[7] = 2.f * (y * z + w * x) * inv;
    Ri[8] = (w * w - x * x - y * y + z * z) * inv;
    return false;
}

template <bool kAll, bool kFit>
__global__ void __launch_bounds__(kThreads, 2) k_fit_rotations(Ctx c, Scal *sc) {
    pdl_wait();
    pdl_trigger();
    if (sc->skip) return;
    const int N = active_count<kAll>(c);
    float part = 0.f;
    int degenerate = 0;
    const float ih = 1.f / c.h;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < N; s += gridDim.x * blockDim.x) {
        const int i = slot_node<kAll>(c, s);
        int nb[6], nj[6];
        neighbours<kAll>(c, s, nb);
        const float3 ui = ld3(c.u, c.ld, i);
        float A[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
        int axes = 0;
#pragma unroll
        for (int d = 0; d < 6; d++) {
            nj[d] = nb[d] >= 0 ? slot_node<kAll>(c, nb[d]) : -1;
            if (nj[d] < 0) continue;
            const int a = d >> 1;
            axes |= 1 << a;
            const float3 uj = ld3(c.u, c.ld, nj[d]);
            // column a of A/h^2: e_a + (u_j - u_i)/h for +a, e_a + (u_i - u_j)/h for -a
            const float sg = (d & 1) ? ih : -ih;
            A[0][a] += (a == 0 ? 1.f : 0.f) + sg * (uj.x - ui.x);
            A[1][a] += (a == 1 ? 1.f : 0.f) + sg * (uj.y - ui.y);
            A[2][a] += (a == 2 ? 1.f : 0.f) + sg * (uj.z - ui.z);
        }
        float Ri[9];
#pragma unroll
        for (int e = 0; e < 9; e++) Ri[e] = c.R[e * c.ld + i];
        const bool two_axes = __popc(axes) >= 2;
        bool keep = !two_axes;
        if (kFit && two_axes) {
            keep = fit_node_rotation(A, Ri);
            if (!keep) {
#pragma unroll
                for (int e = 0; e < 9; e++) c.R[e * c.ld + i] = Ri[e];
            }
        }
        degenerate += kFit && keep;
        // E_reg terms of the directed edges i -> j: (u_i - u_j) - (R_i - I)(t^_i - t^_j)
#pragma unroll
        for (int d = 0; d < 6; d++) {
            if (nj[d] < 0) continue;
            const int a = d >> 1;
            const float sg = (d & 1) ? c.h : -c.h;  // t^_i - t^_j = -sg e_a
            const float ex = sg * (Ri[a] - (a == 0 ? 1.f : 0.f));
            const float ey = sg * (Ri[3 + a] - (a == 1 ? 1.f : 0.f));
            const float ez = sg * (Ri[6 + a] - (a == 2 ? 1.f : 0.f));
            const float3 uj = ld3(c.u, c.ld, nj[d]);  // reloaded (L1): not kept live through the fit
            const float rx = (ui.x - uj.x) + ex, ry = (ui.y - uj.y) + ey, rz = (ui.z - uj.z) + ez;
            part += rx * rx + ry * ry + rz * rz;
        }
    }
    block_add_f64(part, &sc->e_reg);
    block_add_int(degenerate, &sc->n_degenerate);
}

// The rotation step and E_reg of an all-nodes lattice, node data staged in shared
// memory.  Each CTA takes batches of kFitTile consecutive nodes (one per thread); for the
// batch it copies, by cp.async (no registers held while the copies fly), u of the batch's
// own row segment with one node on either side and of the four segments kFitTile long at
// -nx, +nx, -nx ny and +nx ny, and R of the batch's nodes, the next batch's copies in
// flight while the current one is fitted (two stages).  The per-node arithmetic is that
// of k_fit_rotations, so the rotations are the same to the bit; only the order in which
// the E_reg terms are summed differs.
constexpr int kFitTile = 128;                    // nodes per batch (threads per CTA)
constexpr int kFitSeg = kFitTile + 2;            // the batch's own row segment, one node each side
constexpr int kFitU = kFitSeg + 4 * kFitTile;    // staged u values per component
struct FitStage {
    float u[3][kFitU];   // [0, kFitSeg): nodes s0 - 1 ..; then the -nx, +nx, -plane, +plane segments
    float R[9][kFitTile];
};

__device__ __forceinline__ void cp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((unsigned)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// the copies of the batch starting at node s0 (only nodes inside [0, N) are copied)
__device__ __forceinline__ void fit_stage_issue(const Ctx &c, FitStage &S, int s0, int N) {
    const int t = threadIdx.x, pl = c.nx * c.ny;
    const int offs[4] = {-c.nx, c.nx, -pl, pl};
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const float *ua = c.u + (size_t)a * c.ld;
        for (int e = t; e < kFitSeg; e += kFitTile) {
            const int j = s0 - 1 + e;
            if (j >= 0 && j < N) cp_async4(&S.u[a][e], ua + j);
        }
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const int j = s0 + offs[k] + t;
            if (j >= 0 && j < N) cp_async4(&S.u[a][kFitSeg + k * kFitTile + t], ua + j);
        }
    }
    if (s0 + t < N) {
#pragma unroll
        for (int e = 0; e < 9; e++) cp_async4(&S.R[e][t], c.R + (size_t)e * c.ld + s0 + t);
    }
}

template <bool kFit>
__global__ void __launch_bounds__(kFitTile, 4) k_fit_rotations_staged(Ctx c, Scal *sc) {
    __shared__ FitStage S[2];
    pdl_wait();
    pdl_trigger();
    if (sc->skip) return;
    const int N = c.nn, nbatch = (N + kFitTile - 1) / kFitTile;
    const int t = threadIdx.x;
    float part = 0.f;
    int degenerate = 0;
    const float ih = 1.f / c.h;
    int b = blockIdx.x;
    if (b < nbatch) fit_stage_issue(c, S[0], b * kFitTile, N);
    cp_async_commit();
    for (int k = 0; b < nbatch; k++, b += gridDim.x) {
        if (b + (int)gridDim.x < nbatch) fit_stage_issue(c, S[(k + 1) & 1], (b + gridDim.x) * kFitTile, N);
        cp_async_commit();
        cp_async_wait_prev();  // this thread's copies of batch b have landed
        __syncthreads();       // and every thread's
        const FitStage &B = S[k & 1];
        const int i = b * kFitTile + t;
        if (i < N) {
            int nb[6];
            neighbours<true>(c, i, nb);
            // the stage positions of the node and of its neighbours -x, +x, -y, +y, -z, +z
            auto at = [&](int d) -> int { return d < 2 ? t + 2 * d : kFitSeg + (d - 2) * kFitTile + t; };
            const float3 ui = make_float3(B.u[0][t + 1], B.u[1][t + 1], B.u[2][t + 1]);
            float A[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
            int axes = 0;
#pragma unroll
            for (int d = 0; d < 6; d++) {
                if (nb[d] < 0) continue;
                const int a = d >> 1, q = at(d);
                axes |= 1 << a;
                const float3 uj = make_float3(B.u[0][q], B.u[1][q], B.u[2][q]);
                // column a of A/h^2: e_a + (u_j - u_i)/h for +a, e_a + (u_i - u_j)/h for -a
                const float sg = (d & 1) ? ih : -ih;
                A[0][a] += (a == 0 ? 1.f : 0.f) + sg * (uj.x - ui.x);
                A[1][a] += (a == 1 ? 1.f : 0.f) + sg * (uj.y - ui.y);
                A[2][a] += (a == 2 ? 1.f : 0.f) + sg * (uj.z - ui.z);
            }
            float Ri[9];
#pragma unroll
            for (int e = 0; e < 9; e++) Ri[e] = B.R[e][t];
            const bool two_axes = __popc(axes) >= 2;
            bool keep = !two_axes;
            if (kFit && two_axes) {
                keep = fit_node_rotation(A, Ri);
                if (!keep) {
#pragma unroll
                    for (int e = 0; e < 9; e++) c.R[(size_t)e * c.ld + i] = Ri[e];
                }
            }
            degenerate += kFit && keep;
            // E_reg terms of the directed edges i -> j: (u_i - u_j) - (R_i - I)(t^_i - t^_j)
#pragma unroll
            for (int d = 0; d < 6; d++) {
                if (nb[d] < 0) continue;
                const int a = d >> 1, q = at(d);
                const float sg = (d & 1) ? c.h : -c.h;  // t^_i - t^_j = -sg e_a
                const float ex = sg * (Ri[a] - (a == 0 ? 1.f : 0.f));
                const float ey = sg * (Ri[3 + a] - (a == 1 ? 1.f : 0.f));
                const float ez = sg * (Ri[6 + a] - (a == 2 ? 1.f : 0.f));
                const float rx = (ui.x - B.u[0][q]) + ex, ry = (ui.y - B.u[1][q]) + ey, rz = (ui.z - B.u[2][q]) + ez;
                part += rx * rx + ry * ry + rz * rz;
            }
        }
        __syncthreads();  // the stage is refilled by the next batch but one
    }
    block_add_f64(part, &sc->e_reg);
    block_add_int(degenerate, &sc->n_degenerate);
}

// ------------------------------------------------------------------ hierarchy (Sec. 7.2)

// Start state of a coarse level c from the next finer level f: coarse node X takes u and
// R of finer node 2X.  Along an axis where 2X is one past the finer lattice's last node
// (n - 1 odd), u is extrapolated linearly from the last two finer nodes, 2 u(n-1) -
// u(n-2) (per axis, so affine fields are reproduced), and R is the nearest finer node's.
// u_start (3 planes of c.ld) keeps the start displacement for the prolongation.
__global__ void k_restrict_state(Ctx f, Ctx c, float *__restrict__ u_start) {
    for (int I = blockIdx.x * blockDim.x + threadIdx.x; I < c.nn; I += gridDim.x * blockDim.x) {
        const int X = I % c.nx, t = I / c.nx, Y = t % c.ny, Z = t / c.ny;
        const int xyz[3] = {X, Y, Z}, fd[3] = {f.nx, f.ny, f.nz};
        int p0[3];
        bool ext[3];
#pragma unroll
        for (int a = 0; a < 3; a++) {
            ext[a] = 2 * xyz[a] >= fd[a];
            p0[a] = ext[a] ? fd[a] - 1 : 2 * xyz[a];
        }
        float ax = 0.f, ay = 0.f, az = 0.f;
        for (int k = 0; k < 8; k++) {
            const int kx = k & 1, ky = (k >> 1) & 1, kz = (k >> 2) & 1;
            if ((kx && !ext[0]) || (ky && !ext[1]) || (kz && !ext[2])) continue;
            const float w = (kx ? -1.f : (ext[0] ? 2.f : 1.f)) * (ky ? -1.f : (ext[1] ? 2.f : 1.f)) *
                            (kz ? -1.f : (ext[2] ? 2.f : 1.f));
            const int i = (p0[0] - kx) + f.nx * ((p0[1] - ky) + f.ny * (p0[2] - kz));
            ax += w * f.u[i];
            ay += w * f.u[f.ld + i];
            az += w * f.u[2 * f.ld + i];
        }
        c.u[I] = u_start[I] = ax;
        c.u[c.ld + I] = u_start[c.ld + I] = ay;
        c.u[2 * c.ld + I] = u_start[2 * c.ld + I] = az;
        const int i0 = p0[0] + f.nx * (p0[1] + f.ny * p0[2]);
#pragma unroll
        for (int e = 0; e < 9; e++) c.R[e * c.ld + I] = f.R[e * f.ld + i0];
    }
}

// Jump start of the finer level f from the coarse solution: every finer node adds the
// coarse displacement increment (u - u_start) interpolated trilinearly at its canonical
// position, coarse coordinates (x/2, y/2, z/2) (weights 0, 1/2 or 1: exact in FP32).
__global__ void k_prolongate(Ctx c, const float *__restrict__ u_start, Ctx f) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < f.nn; i += gridDim.x * blockDim.x) {
        const int x = i % f.nx, t = i / f.nx, y = t % f.ny, z = t / f.ny;
        const int X0 = min(x >> 1, c.nx - 2), Y0 = min(y >> 1, c.ny - 2), Z0 = min(z >> 1, c.nz - 2);
        const float fr[3] = {0.5f * x - X0, 0.5f * y - Y0, 0.5f * z - Z0};
        const int cell = X0 + c.nx * (Y0 + c.ny * Z0);
        float ax = 0.f, ay = 0.f, az = 0.f;
#pragma unroll
        for (int k = 0; k < 8; k++) {
            const float al = trilinear_weight(fr, k);
            if (al == 0.f) continue;
            const int nd = corner_node(c, cell, k);
            ax += al * (c.u[nd] - u_start[nd]);
            ay += al * (c.u[c.ld + nd] - u_start[c.ld + nd]);
            az += al * (c.u[2 * c.ld + nd] - u_start[2 * c.ld + nd]);
        }
        f.u[i] += ax;
        f.u[f.ld + i] += ay;
        f.u[2 * f.ld + i] += az;
    }
}

// ------------------------------------------------------------------ global rigid pose (Sec. 6)
//
// Dense projective ICP on the global pose (R_g, t_g) with the lattice warp fixed: each
// step associates every sample projectively at the current pose (Sec. 5.1, the same
// FP32 decisions re-taken in FP64 near a threshold as the solve's association), then
// solves the 6 x 6 normal equations of sum_c w_c (n^a . (R_g q_c + t_g - p^a))^2, q_c =
// p^_c + sum_k alpha_k u_k, over the perturbation R_g <- exp([omega]x) R_g, t_g <- t_g +
// tau, whose Jacobian row is J = ((R_g q_c) x n^a, n^a).
constexpr int kIcpMaxSteps = 64;

struct IcpState {
    double pose[12];                  // R_g (row-major), t_g in FP64 between steps
    double sums[28];                  // upper triangle of A (21, row by row), b (6), E
    double e_hist[kIcpMaxSteps];      // E before each step
    int n_refine, steps, status;      // status 1: A not positive definite (pose kept)
    int pad;
};

__device__ __forceinline__ Ctx with_pose(const Ctx &c, const IcpState *st) {
    Ctx cl = c;
#pragma unroll
    for (int a = 0; a < 9; a++) cl.Rg[a] = (float)st->pose[a];
#pragma unroll
    for (int a = 0; a < 3; a++) cl.tg[a] = (float)st->pose[9 + a];
    return cl;
}

// the 28 sums of sample i associated to pixel k with weight w (FP32 values)
__device__ __forceinline__ void icp_terms(const Ctx &cl, int i, int k, float w, float acc[28]) {
    const int cl_ = cl.cell[i];
    float f[3];
    sample_frac_f32(cl, i, f);
    const float4 p4 = cl.sp[i];
    V3<float> q{p4.x, p4.y, p4.z};
#pragma unroll
    for (int kk = 0; kk < 8; kk++) {
        const int node = corner_node(cl, cl_, kk);
        const float al = trilinear_weight(f, kk);
        q.x += al * cl.u[node];
        q.y += al * cl.u[cl.ld + node];
        q.z += al * cl.u[2 * cl.ld + node];
    }
    const V3<float> Rq = rot<float>(cl.Rg, q);
    const int px = k % cl.W, py = k / cl.W;
    const float D = cl.depth[k];
    const float4 m4 = load_nrm(cl, (size_t)k);
    const V3<float> na{m4.x, m4.y, m4.z};
    const V3<float> pa{D * ((px - cl.cx) / cl.fx), D * ((py - cl.cy) / cl.fy), D};
    const V3<float> d{Rq.x + cl.tg[0] - pa.x, Rq.y + cl.tg[1] - pa.y, Rq.z + cl.tg[2] - pa.z};
    const float r = dot(na, d);
    const float J[6] = {Rq.y * na.z - Rq.z * na.y, Rq.z * na.x - Rq.x * na.z, Rq.x * na.y - Rq.y * na.x,
                        na.x, na.y, na.z};
    int e = 0;
#pragma unroll
    for (int a = 0; a < 6; a++)
#pragma unroll
        for (int b = a; b < 6; b++) acc[e++] += w * J[a] * J[b];
#pragma unroll
    for (int a = 0; a < 6; a++) acc[21 + a] += w * J[a] * r;
    acc[27] += w * r * r;
}

// block sum of the 28 per-thread sums (FP32 within a warp, FP64 across warps), added to
// st->sums by the block's first 28 threads
__device__ __forceinline__ void icp_block_add(float acc[28], IcpState *st) {
    __shared__ float wsum[32][28];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int e = 0; e < 28; e++) {
        float v = acc[e];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
        if (lane == 0) wsum[wid][e] = v;
    }
    __syncthreads();
    if (threadIdx.x < 28) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += (double)wsum[w][threadIdx.x];
        if (t != 0.0) atomicAdd(&st->sums[threadIdx.x], t);
    }
}

template <bool kAll>
__global__ void __launch_bounds__(kThreads) k_icp_assoc(Ctx c, IcpState *st) {
    if (st->status) return;
    const Ctx cl = with_pose(c, st);
    const int n = *c.n_samples;
    float acc[28];
#pragma unroll
    for (int e = 0; e < 28; e++) acc[e] = 0.f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int pix;
        float w;
        float4 rec;
        if (associate_sample_f32(cl, i, pix, w, rec)) {  // near a threshold: FP64 in k_icp_refine
            c.refine[atomicAdd(&st->n_refine, 1)] = i;
            continue;
        }
        if (w > 0.f) icp_terms(cl, i, pix, w, acc);
    }
    icp_block_add(acc, st);
}

// the listed samples associated again in FP64 (eight lanes per sample, as the solve's)
template <bool kAll>
__global__ void __launch_bounds__(kThreads) k_icp_refine(Ctx c, IcpState *st) {
    if (st->status) return;
    const Ctx cl = with_pose(c, st);
    const int n = st->n_refine;
    const int k = threadIdx.x & 7;
    const int warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int wg = warp * gridDim.x + blockIdx.x;
    const int per_round = 4 * nwarp * gridDim.x;
    float acc[28];
#pragma unroll
    for (int e = 0; e < 28; e++) acc[e] = 0.f;
    for (int g0 = 4 * wg; g0 < n; g0 += per_round) {
        const int g = g0 + ((threadIdx.x & 31) >> 3);
        V3<double> du{0.0, 0.0, 0.0}, dn{0.0, 0.0, 0.0};
        int i = -1;
        float4 p4 = make_float4(0.f, 0.f, 0.f, 0.f);
        if (g < n) {
            i = c.refine[g];
            const int cell = cl.cell[i];
            const float4 n4 = cl.sn[i];
            p4 = cl.sp[i];
            double f[3];
            sample_frac_f64(cl, cell, p4, f);
            const int node = corner_node(cl, cell, k);
            const double al = trilinear_weight(f, k);
            du = {al * (double)cl.u[node], al * (double)cl.u[cl.ld + node], al * (double)cl.u[2 * cl.ld + node]};
            float Rk[9];
#pragma unroll
            for (int e = 0; e < 9; e++) Rk[e] = cl.R[e * cl.ld + node];
            const V3<double> rn = rot<double>(Rk, V3<double>{(double)n4.x, (double)n4.y, (double)n4.z});
            dn = {al * rn.x, al * rn.y, al * rn.z};
        }
#pragma unroll
        for (int o = 1; o < 8; o <<= 1) {
            du.x += __shfl_xor_sync(FULL, du.x, o);
            du.y += __shfl_xor_sync(FULL, du.y, o);
            du.z += __shfl_xor_sync(FULL, du.z, o);
            dn.x += __shfl_xor_sync(FULL, dn.x, o);
            dn.y += __shfl_xor_sync(FULL, dn.y, o);
            dn.z += __shfl_xor_sync(FULL, dn.z, o);
        }
        if (k == 0 && g < n) {
            int pix;
            float w;
            float4 rec;
            associate_finish_f64(cl, p4, du, dn, pix, w, rec);
            if (w > 0.f) icp_terms(cl, i, pix, w, acc);
        }
    }
    icp_block_add(acc, st);
}

// one thread: A xi = -b by Cholesky (FP64), then R_g <- exp([omega]x) R_g (Rodrigues),
// t_g <- t_g + tau; the sums are cleared for the next step
__global__ void k_icp_step(IcpState *st) {
    if (threadIdx.x != 0 || st->status) return;
    double A[6][6], b[6], L[6][6] = {}, y[6], xi[6];
    int e = 0;
    for (int a = 0; a < 6; a++)
        for (int c2 = a; c2 < 6; c2++) A[a][c2] = A[c2][a] = st->sums[e++];
    for (int a = 0; a < 6; a++) b[a] = st->sums[21 + a];
    if (st->steps < kIcpMaxSteps) st->e_hist[st->steps] = st->sums[27];
    for (int k = 0; k < 28; k++) st->sums[k] = 0.0;
    st->n_refine = 0;
    for (int j = 0; j < 6; j++) {
        double sj = A[j][j];
        for (int k = 0; k < j; k++) sj -= L[j][k] * L[j][k];
        if (!(sj > 0.0)) {
            st->status = 1;
            return;
        }
        L[j][j] = sqrt(sj);
        for (int i = j + 1; i < 6; i++) {
            double t = A[i][j];
            for (int k = 0; k < j; k++) t -= L[i][k] * L[j][k];
            L[i][j] = t / L[j][j];
        }
    }
    for (int i = 0; i < 6; i++) {
        double t = -b[i];
        for (int k = 0; k < i; k++) t -= L[i][k] * y[k];
        y[i] = t / L[i][i];
    }
    for (int i = 5; i >= 0; i--) {
        double t = y[i];
        for (int k = i + 1; k < 6; k++) t -= L[k][i] * xi[k];
        xi[i] = t / L[i][i];
    }
    const double th = sqrt(xi[0] * xi[0] + xi[1] * xi[1] + xi[2] * xi[2]);
    const double K[9] = {0.0, -xi[2], xi[1], xi[2], 0.0, -xi[0], -xi[1], xi[0], 0.0};
    const double s1 = th > 0.0 ? sin(th) / th : 1.0, s2 = th > 0.0 ? (1.0 - cos(th)) / (th * th) : 0.5;
    double E3[9], Rn[9];
    for (int r = 0; r < 3; r++)
        for (int q = 0; q < 3; q++) {
            const double KK = K[3 * r] * K[q] + K[3 * r + 1] * K[3 + q] + K[3 * r + 2] * K[6 + q];
            E3[3 * r + q] = (r == q ? 1.0 : 0.0) + s1 * K[3 * r + q] + s2 * KK;
        }
    for (int r = 0; r < 3; r++)
        for (int q = 0; q < 3; q++)
            Rn[3 * r + q] = E3[3 * r] * st->pose[q] + E3[3 * r + 1] * st->pose[3 + q] + E3[3 * r + 2] * st->pose[6 + q];
    for (int k = 0; k < 9; k++) st->pose[k] = Rn[k];
    for (int a = 0; a < 3; a++) st->pose[9 + a] += xi[3 + a];
    st->steps++;
}

// ------------------------------------------------------------------ layout helpers

// AoS full-lattice (n x 3) -> slot SoA vector; entries outside M are dropped
template <bool kAll>
__global__ void k_gather_slots(const float *__restrict__ src, Ctx c, float *__restrict__ dst) {
    const int N = active_count<kAll>(c);
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < N; s += gridDim.x * blockDim.x) {
        const int i = slot_node<kAll>(c, s);
#pragma unroll
        for (int a = 0; a < 3; a++) dst[a * c.ld + s] = src[3 * (size_t)i + a];
    }
}

// slot SoA vector -> AoS full lattice (0 outside M)
template <bool kAll>
__global__ void k_scatter_slots(const float *__restrict__ src, Ctx c, float *__restrict__ dst) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < c.nn; i += gridDim.x * blockDim.x) {
        const int s = node_slot<kAll>(c, i);
#pragma unroll
        for (int a = 0; a < 3; a++) dst[3 * (size_t)i + a] = s >= 0 ? src[a * c.ld + s] : 0.f;
    }
}

// SoA (planes x ld) <-> AoS (n x planes)
__global__ void k_soa_to_aos(const float *__restrict__ src, int planes, int n, int ld, float *__restrict__ dst) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        for (int a = 0; a < planes; a++) dst[(size_t)planes * i + a] = src[(size_t)a * ld + i];
}

__global__ void k_aos_to_soa(const float *__restrict__ src, int planes, int n, int ld, float *__restrict__ dst) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        for (int a = 0; a < planes; a++) dst[(size_t)a * ld + i] = src[(size_t)planes * i + a];
}

__global__ void k_reset_warp(float *__restrict__ u, float *__restrict__ R, int n, int ld) {
    pdl_wait();
    pdl_trigger();
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
#pragma unroll
        for (int a = 0; a < 3; a++) u[a * ld + i] = 0.f;
#pragma unroll
        for (int e = 0; e < 9; e++) R[e * ld + i] = (e % 4 == 0) ? 1.f : 0.f;
    }
}

// association results back into the caller's sample order
__global__ void k_clear_association(int n_src, int *__restrict__ pix, float *__restrict__ w, float *__restrict__ r) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_src; i += gridDim.x * blockDim.x) {
        pix[i] = -1;
        w[i] = 0.f;
        r[i] = 0.f;
    }
}

template <bool kAll>
__global__ void k_unsort_association(Ctx c, int *__restrict__ pix, float *__restrict__ w, float *__restrict__ r) {
    const int n = *c.n_samples;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int o = c.perm[i];
        pix[o] = c.pix[i];
        w[o] = c.wc[i];
        float res = 0.f;
        const float4 g = load_rec(c, i);
        if (c.wc[i] > 0.f) {
            const float4 f4 = c.frac[i];
            const float f[3] = {f4.x, f4.y, f4.z};
            float sx = 0.f, sy = 0.f, sz = 0.f;
            for (int k = 0; k < 8; k++) {
                const int nd = corner_node(c, c.cell[i], k);
                const float al = trilinear_weight(f, k);
                sx += al * c.u[nd];
                sy += al * c.u[c.ld + nd];
                sz += al * c.u[2 * c.ld + nd];
            }
            res = sqrtf(c.w_d) * (g.x * sx + g.y * sy + g.z * sz + g.w);
        }
        r[o] = res;
    }
}

__global__ void k_pack_float4(const float *__restrict__ src, int n, float4 *__restrict__ dst) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        dst[i] = make_float4(src[3 * i], src[3 * i + 1], src[3 * i + 2], 0.f);
}

__global__ void k_store_f64(double *dst, double v) { *dst = v; }

// Gauss-Newton early stop: iteration g+1 (slot `next`) is skipped once iteration g was
// skipped or ended with E_total <= *c.e_target.  The PCG kernels also honour `stop`.
__global__ void k_gn_gate(Ctx c, const Scal *prev, Scal *next) {
    pdl_wait();
    pdl_trigger();
    if (threadIdx.x || blockIdx.x) return;
    const double e = (double)c.w_s * prev->e_sparse + (double)c.w_d * prev->e_dense + (double)c.w_r * prev->e_reg;
    if (prev->skip || e <= *c.e_target) {
        next->skip = 1;
        next->stop = 1;
    }
}

__global__ void k_finish_report(Scal *sc_base, size_t stride, int G, Ctx c, double *out, const int *err) {
    pdl_wait();
    pdl_trigger();
    // out: e_total, e_dense, e_sparse, e_reg, then ints as doubles: gn_done, cg_done,
    // n_valid, n_degenerate, n_refined, finite
    if (threadIdx.x || blockIdx.x) return;
    Scal *last = sc_base;
    int nv = 0, nr = 0, done = 0;
    for (int g = 0; g < G; g++) {
        Scal *s = (Scal *)((char *)sc_base + stride * (size_t)g);
        if (s->skip) break;
        last = s;
        done++;
        if (s->assoc_ran) {
            nv = s->n_valid;
            nr = s->n_refined;
        }
    }
    const double ed = last->e_dense, es = last->e_sparse, er = last->e_reg;
    const double et = (double)c.w_s * es + (double)c.w_d * ed + (double)c.w_r * er;
    out[0] = et;
    out[1] = ed;
    out[2] = es;
    out[3] = er;
    out[4] = done;
    out[5] = last->cg_done;
    out[6] = nv;
    out[7] = last->n_degenerate;
    out[8] = nr;
    out[9] = isfinite(et) ? 1.0 : 0.0;
    out[10] = *err ? 1.0 : 0.0;  // a grid barrier of the persistent position step gave up
}


// ------------------------------------------------------------------ learned warm start

// Network input at every active node i (node-major, 6 floats; the caller zeroes the
// rest): the displacement in lattice units u_i / h, and the data-term gradient of the
// current frame at the current warp, b_i = -(J_data^T r)_i (Eq. 2-3 with w_r = 0, as
// left in c.r by the right-hand side pass run with w_r = 0), scaled per component by
// 1 / (h (diag_i + 2 w_r |N_i|)): one Jacobi step of the full system, in lattice units.
template <bool kAll>
__global__ void k_warm_features(Ctx c, float w_reg, float *__restrict__ in6) {
    const int N = active_count<kAll>(c);
    const float ih = 1.f / c.h;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < N; s += gridDim.x * blockDim.x) {
        const int i = slot_node<kAll>(c, s);
        int nb[6];
        neighbours<kAll>(c, s, nb);
        int deg = 0;
#pragma unroll
        for (int d = 0; d < 6; d++) deg += nb[d] >= 0;
        const float reg = 2.f * w_reg * (float)deg;
        const float3 u = ld3(c.u, c.ld, i);
        const float3 b = ld3(c.r, c.ld, s), dg = ld3(c.minv, c.ld, s);
        const float dx = dg.x + reg, dy = dg.y + reg, dz = dg.z + reg;
        float *o = in6 + 6 * (size_t)i;
        o[0] = u.x * ih;
        o[1] = u.y * ih;
        o[2] = u.z * ih;
        o[3] = dx > 0.f ? b.x * ih / dx : 0.f;
        o[4] = dy > 0.f ? b.y * ih / dy : 0.f;
        o[5] = dz > 0.f ? b.z * ih / dz : 0.f;
    }
}

// Candidate start: back up u and R of the active nodes, then u_i += h * pred_i.
template <bool kAll>
__global__ void k_warm_apply(Ctx c, const float *__restrict__ pred3, float *__restrict__ bak) {
    const int N = active_count<kAll>(c);
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < N; s += gridDim.x * blockDim.x) {
        const int i = slot_node<kAll>(c, s);
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const float v = c.u[a * (size_t)c.ld + i];
            bak[a * (size_t)c.ld + i] = v;
            c.u[a * (size_t)c.ld + i] = v + c.h * pred3[3 * (size_t)i + a];
        }
#pragma unroll
        for (int a = 0; a < 9; a++) bak[(3 + a) * (size_t)c.ld + i] = c.R[a * (size_t)c.ld + i];
    }
}

// Keep the candidate only if its energy is finite and below the current warp's; else
// restore u and R.  out: E of the current warp, E of the candidate, 1 if kept.
template <bool kAll>
__global__ void k_warm_select(Ctx c, const Scal *cur, const Scal *cand, const float *__restrict__ bak,
                              double *__restrict__ out) {
    const double e0 = (double)c.w_s * cur->e_sparse + (double)c.w_d * cur->e_dense + (double)c.w_r * cur->e_reg;
    const double e1 = (double)c.w_s * cand->e_sparse + (double)c.w_d * cand->e_dense + (double)c.w_r * cand->e_reg;
    const bool keep = isfinite(e1) && e1 < e0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        out[0] = e0;
        out[1] = e1;
        out[2] = keep ? 1.0 : 0.0;
    }
    if (keep) return;
    const int N = active_count<kAll>(c);
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < N; s += gridDim.x * blockDim.x) {
        const int i = slot_node<kAll>(c, s);
#pragma unroll
        for (int a = 0; a < 3; a++) c.u[a * (size_t)c.ld + i] = bak[a * (size_t)c.ld + i];
#pragma unroll
        for (int a = 0; a < 9; a++) c.R[a * (size_t)c.ld + i] = bak[(3 + a) * (size_t)c.ld + i];
    }
}

}  // namespace vd
