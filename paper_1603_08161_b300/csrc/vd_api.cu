// libvd host side: the C ABI of include/vd.h, device buffers of a lattice, the
// per-frame preprocessing (target normals, sample binning, active set), and the
// flip-flop schedule of Sec. 7.1 captured once into a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "vd.h"
#include "vd_kernels.cuh"
#include "vd_render.cuh"

using namespace vd;

namespace {

constexpr int kSMs = 148;

int blocks_for(long n, int threads = kThreads, int per_sm = 8) {
    long b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    return (int)std::min<long>(b, (long)kSMs * per_sm);
}

int round_pow2(int n) {
    int p = 32;
    while (p < n) p <<= 1;
    return p;
}

struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
};

}  // namespace

struct vd_lattice {
    Ctx c{};
    int all = 1;
    int precision = VD_PREC_FP32;
    cudaStream_t stream = nullptr;   // caller's (or own) stream: where work is ordered
    cudaStream_t cap = nullptr;      // private stream used for graph capture
    // asynchronous read of the warp (vd_get_warp_async): a readback buffer (12 x nn
    // floats), the stream that copies it out, and its events (ready to copy, copied)
    float *rb = nullptr;
    cudaStream_t rb_st = nullptr;
    cudaEvent_t rb_ready = nullptr, rb_done = nullptr;
    bool own_stream = false;
    std::string err;

    std::vector<DevBuf> bufs;        // everything allocated, freed at destroy
    // lattice state and solver vectors
    float *u = nullptr, *R = nullptr, *vecs = nullptr;
    int *slot_of_node = nullptr, *node_of_slot = nullptr, *nbr = nullptr, *mark = nullptr, *act = nullptr;
    int *counts = nullptr;           // [0] n_active, [1] n_occ, [2..] spare
    int *cnt = nullptr, *start = nullptr, *scan_sums = nullptr;
    float *staging = nullptr;        // n x 9 floats for warp transfers
    // frame
    int W = 0, H = 0, cap_px = 0;
    float *depth = nullptr;
    float4 *nrm = nullptr;
    int n_src = 0, cap_src = 0;
    float *pts_in = nullptr, *nrm_in = nullptr, *res_f = nullptr;
    int *cell_in = nullptr, *tmp = nullptr, *order = nullptr, *head = nullptr, *hscan = nullptr;
    int *scell = nullptr, *perm = nullptr, *pix = nullptr, *refine = nullptr, *occ_cell = nullptr, *occ_beg = nullptr, *res_i = nullptr;
    float4 *frac_in = nullptr, *sp = nullptr, *sn = nullptr, *sfrac = nullptr, *rec = nullptr;
    float *wc = nullptr;
    int4 *cell_part = nullptr;       // per block of the sample passes (kSMs x 8 entries)
    // sparse pairs
    int S = 0, cap_S = 0;
    float *sp_in = nullptr;
    float4 *fh = nullptr, *ft = nullptr, *sfr = nullptr;
    int *scell_s = nullptr;
    // scalars and report
    char *scal = nullptr;
    size_t scal_stride = 0;
    int scal_slots = 0;
    double *rep_dev = nullptr, *rep_host = nullptr;
    // host-side sizes of the current frame (for grid sizing)
    int n_active_h = 0, n_samples_h = 0, n_occ_h = 0;
    bool have_frame = false;
    long frame_gen = 0;              // counts vd_set_frame / vd_set_correspondences calls
    // graph
    cudaGraphExec_t gexec = nullptr;
    vd_solve_params gparams{};
    Ctx gctx{};
    int gkey_caps[6] = {0, 0, 0, 0, 0, 0};
    long gen = 0, ggen = -1;         // buffer generation (pointers changed)
    int stall_extra = 0;             // vd_test_stall_barrier: arrivals awaited beyond the grid
    int launches_solve = 0, launches_frame = 0;
    int counting = 0;
    bool solve_pending = false;
    // profiling
    int prof_class = -1;
    std::vector<cudaEvent_t> ev;
    int ev_used = 0;
    double prof_ms = 0.0;
    int prof_launches = 0;
    bool use_pdl = true;             // chain solve kernels with programmatic dependent launch
    // persistent position step
    int *surf_flag = nullptr;        // per slot: touched by a sample or a sparse pair
    double *pcg_part = nullptr;
    int pcg_part_rows = 0;
    unsigned *pcg_bar = nullptr;     // [2] error flag of the persistent position step
    int num_sms = 148;
    bool coop = false;               // device supports cooperative launches
    bool use_persistent = true;      // may be cleared if the graph cannot hold the launch
    bool in_batch = false;           // being captured into a batch graph: streamed PCG
    bool use_brick = true;           // persistent step: brick partition where one fits
    // Gauss-Newton early stop: the energy target lives in rep_dev[15]
    bool gated = false;
    // learned warm start: features (6 nn), prediction (3 nn), backup of u and R (12 ld)
    float *warm = nullptr;
    // persistent batched position step: published z and stencil q (6 ld), lazily allocated
    float *batch_vecs = nullptr;
    // published vectors of a padded brick with unaligned rows (z, p even / odd, q; 3
    // planes of pad_ldp floats each), allocated with such a plan
    float *pad_vecs = nullptr;
    size_t pad_ldp = 0;
    // global pose estimation (dense projective ICP): device state, lazily allocated
    IcpState *icp = nullptr;
    // cached B^T B of the dense samples (per occupied cell, 24 x 24), VD_APPLY_*
    int apply_mode = VD_APPLY_MATRIX_FREE;
    float *btb = nullptr;
    int cap_occ = 0;
};

namespace {

vd_status fail(vd_lattice *L, vd_status s, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (L) L->err = buf;
    return s;
}

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) return fail(L, VD_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

#define CKL()                                                                                   \
    do {                                                                                        \
        cudaError_t e_ = cudaGetLastError();                                                    \
        if (e_ != cudaSuccess) return fail(L, VD_ERR_CUDA, "launch: %s", cudaGetErrorString(e_)); \
    } while (0)

template <typename T>
vd_status dalloc(vd_lattice *L, T **p, size_t count) {
    void *q = nullptr;
    size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    bytes = (bytes + 255) & ~(size_t)255;
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(L, VD_ERR_OOM, "cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
    }
    L->bufs.push_back({q, bytes});
    *p = (T *)q;
    L->gen++;
    return VD_OK;
}

template <typename T>
void dfree(vd_lattice *L, T *&p) {
    if (!p) return;
    for (size_t k = 0; k < L->bufs.size(); k++)
        if (L->bufs[k].ptr == (void *)p) {
            cudaFree(p);
            L->bufs.erase(L->bufs.begin() + k);
            break;
        }
    p = nullptr;
    L->gen++;
}

#define TRY(x)                       \
    do {                             \
        vd_status s_ = (x);          \
        if (s_ != VD_OK) return s_;  \
    } while (0)

// copy `bytes` from a caller pointer (host or device) into device memory
vd_status upload(vd_lattice *L, void *dst, const void *src, size_t bytes, int mem) {
    if (!bytes) return VD_OK;
    CK(cudaMemcpyAsync(dst, src, bytes, mem == VD_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                       L->stream));
    return VD_OK;
}

vd_status download(vd_lattice *L, void *dst, const void *src, size_t bytes, int mem) {
    if (!bytes) return VD_OK;
    CK(cudaMemcpyAsync(dst, src, bytes, mem == VD_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                       L->stream));
    return VD_OK;
}

void scan_launch(const int *in, int n, int *out, int *out_total, int *sums, cudaStream_t st) {
    const int nt = (n + kScanTile - 1) / kScanTile;
    k_scan_tiles<<<std::max(nt, 1), kScanThreads, 0, st>>>(in, n, out, sums);
    k_scan_sums<<<1, kScanThreads, 0, st>>>(sums, std::max(nt, 1), out_total);
    if (n > 0) k_scan_add<<<(n + 255) / 256, 256, 0, st>>>(out, n, sums);
}


// ------------------------------------------------------------------ capacities

vd_status ensure_frame_caps(vd_lattice *L, int W, int H, int n_src) {
    if (W * H > L->cap_px) {
        dfree(L, L->depth);
        dfree(L, L->nrm);
        L->cap_px = W * H;
        TRY(dalloc(L, &L->depth, (size_t)L->cap_px));
        TRY(dalloc(L, &L->nrm, (size_t)L->cap_px));
    }
    if (n_src > L->cap_src || L->cap_src == 0) {  // the first frame allocates even for n_src = 0
        float **fs[] = {&L->pts_in, &L->nrm_in, &L->res_f};
        for (auto f : fs) dfree(L, *f);
        int **is[] = {&L->cell_in, &L->tmp, &L->order, &L->head, &L->hscan, &L->scell, &L->perm, &L->pix, &L->refine,
                      &L->occ_cell, &L->occ_beg, &L->res_i};
        for (auto i : is) dfree(L, *i);
        float4 **f4[] = {&L->frac_in, &L->sp, &L->sn, &L->sfrac, &L->rec};
        for (auto f : f4) dfree(L, *f);
        dfree(L, L->wc);
        dfree(L, L->scan_sums);
        int cap = std::max(n_src, 1024);
        cap = (int)std::min<long>((long)cap + cap / 4, 0x7fffffffL);
        L->cap_src = cap;
        TRY(dalloc(L, &L->pts_in, (size_t)cap * 3));
        TRY(dalloc(L, &L->nrm_in, (size_t)cap * 3));
        TRY(dalloc(L, &L->res_f, (size_t)cap * 2));
        TRY(dalloc(L, &L->cell_in, (size_t)cap));
        TRY(dalloc(L, &L->tmp, (size_t)cap));
        TRY(dalloc(L, &L->order, (size_t)cap));
        TRY(dalloc(L, &L->head, (size_t)cap));
        TRY(dalloc(L, &L->hscan, (size_t)cap + 1));
        TRY(dalloc(L, &L->scell, (size_t)cap));
        TRY(dalloc(L, &L->perm, (size_t)cap));
        TRY(dalloc(L, &L->pix, (size_t)cap));
        TRY(dalloc(L, &L->refine, (size_t)cap));
        TRY(dalloc(L, &L->occ_cell, (size_t)cap));
        TRY(dalloc(L, &L->occ_beg, (size_t)cap + 1));
        TRY(dalloc(L, &L->res_i, (size_t)cap));
        TRY(dalloc(L, &L->frac_in, (size_t)cap));
        TRY(dalloc(L, &L->sp, (size_t)cap));
        TRY(dalloc(L, &L->sn, (size_t)cap));
        TRY(dalloc(L, &L->sfrac, (size_t)cap));
        TRY(dalloc(L, &L->rec, (size_t)cap));
        TRY(dalloc(L, &L->wc, (size_t)cap));
    }
    if (!L->scan_sums) TRY(dalloc(L, &L->scan_sums, (size_t)kScanTile));
    return VD_OK;
}

vd_status ensure_scal(vd_lattice *L, int G, int K) {
    if (2 * K + 2 > L->pcg_part_rows) {
        dfree(L, L->pcg_part);
        L->pcg_part_rows = 2 * K + 2;
        // the rows of partials, then one barrier word per row
        TRY(dalloc(L, &L->pcg_part, (size_t)L->pcg_part_rows * (L->num_sms + 1)));
    }
    const size_t stride = scal_bytes(K);
    if (L->scal && stride == L->scal_stride && G <= L->scal_slots) return VD_OK;
    dfree(L, L->scal);
    const int slots = std::max(G, 1);
    TRY(dalloc(L, &L->scal, stride * (size_t)slots));
    L->scal_stride = stride;
    L->scal_slots = slots;
    return VD_OK;
}

Scal *slot(vd_lattice *L, int g) { return (Scal *)(L->scal + L->scal_stride * (size_t)g); }

// samples per occupied cell from which VD_APPLY_AUTO takes the cached blocks: a block
// is 576 multiply-adds and 2,304 bytes per cell and iteration, the matrix-free apply of
// one sample about 48 multiply-adds, 28 bytes and 8 corner gathers
constexpr int kAutoSamplesPerCell = 32;

bool use_cached(const vd_lattice *L) {
    if (L->apply_mode == VD_APPLY_CACHED) return L->n_occ_h > 0;
    if (L->apply_mode == VD_APPLY_AUTO)
        return L->n_occ_h > 0 && (long)L->n_samples_h >= (long)kAutoSamplesPerCell * L->n_occ_h;
    return false;
}

void refresh_ctx(vd_lattice *L) {
    Ctx &c = L->c;
    c.u = L->u;
    c.R = L->R;
    c.x = L->vecs;
    c.r = L->vecs + 3 * (size_t)c.ld;
    c.p = L->vecs + 6 * (size_t)c.ld;
    c.q = L->vecs + 9 * (size_t)c.ld;
    c.minv = L->vecs + 12 * (size_t)c.ld;
    c.slot_of_node = L->slot_of_node;
    c.node_of_slot = L->node_of_slot;
    c.nbr = L->nbr;
    c.n_active = L->counts;
    c.depth = L->depth;
    c.nrm = L->nrm;
    c.sp = L->sp;
    c.sn = L->sn;
    c.frac = L->sfrac;
    c.cell = L->scell;
    c.perm = L->perm;
    c.n_samples = L->start ? L->start + c.nn : nullptr;
    c.occ_cell = L->occ_cell;
    c.occ_beg = L->occ_beg;
    c.n_occ = L->counts + 1;
    c.rec = L->rec;
    c.pix = L->pix;
    c.refine = L->refine;
    c.wc = L->wc;
    c.fh = L->fh;
    c.ft = L->ft;
    c.sfrac = L->sfr;
    c.scell = L->scell_s;
    c.S = L->S;
    c.e_target = L->gated ? L->rep_dev + 15 : nullptr;
    c.cell_part = L->cell_part;
    c.btb = (use_cached(L) && L->cap_occ >= L->n_occ_h) ? L->btb : nullptr;
}

// room for the cached blocks of the current frame's occupied cells (when they are used)
vd_status ensure_btb(vd_lattice *L) {
    if (L->apply_mode == VD_APPLY_MATRIX_FREE || L->n_occ_h <= L->cap_occ) return VD_OK;
    dfree(L, L->btb);
    L->cap_occ = 0;
    const int cap = L->n_occ_h + L->n_occ_h / 4 + 64;
    TRY(dalloc(L, &L->btb, (size_t)cap * kBtb));
    L->cap_occ = cap;
    return VD_OK;
}

void set_params_ctx(Ctx &c, const vd_solve_params *p) {
    c.w_s = p->w_sparse;
    c.w_d = p->w_dense;
    c.w_r = p->w_reg;
    c.eps_d = p->eps_d;
    c.eps_n = p->eps_n;
    c.eps_v = p->eps_v;
}

vd_status check_params(vd_lattice *L, const vd_solve_params *p) {
    if (!p) return fail(L, VD_ERR_INVALID_ARG, "params is NULL");
    if (p->gn_iters < 1 || p->gn_iters > 1000 || p->cg_iters < 0 || p->cg_iters > 100000)
        return fail(L, VD_ERR_INVALID_ARG, "gn_iters must be in [1, 1000], cg_iters in [0, 100000]");
    if (!(p->eps_d > 0) || !(p->eps_n > 0) || !(p->eps_v > 0))
        return fail(L, VD_ERR_INVALID_ARG, "eps_d, eps_n, eps_v must be > 0");
    if (!(p->w_sparse >= 0) || !(p->w_dense >= 0) || !(p->w_reg >= 0))
        return fail(L, VD_ERR_INVALID_ARG, "weights must be >= 0");
    if (!(p->cg_tol >= 0)) return fail(L, VD_ERR_INVALID_ARG, "cg_tol must be >= 0");
    return VD_OK;
}

// ------------------------------------------------------------------ launch plumbing

struct Grid {
    int node;    // blocks over active slots
    int node4;   // blocks over float4 groups of slots
    int samp, cells;
    int refine;  // blocks of the FP64 re-association (a grid-stride loop over the list)
    int btb;     // blocks of the cached-B^T B apply (one warp per occupied cell)
    int btb_build;  // blocks of its build (one warp per 64 samples)
    bool vec4;   // all-nodes lattice with nx % 4 == 0: float4 stencil
    int assoc;   // blocks of the FP32 association (four lanes per sample)
    int fit;     // blocks of the staged rotation step (all-nodes lattices; kFitTile threads)
};

Grid grids(vd_lattice *L) {
    Grid g;
    const int nact = L->all ? L->c.nn : round_pow2(std::max(L->n_active_h, 1));
    g.node = blocks_for(nact);
    g.node4 = blocks_for((nact + 3) / 4, kThreads, 8);
    g.samp = blocks_for(round_pow2(std::max(L->n_samples_h, 1)));
    // about 128 samples per block (a power of two of them, so the grid, and the
    // captured graph, stay the same for frames of similar size)
    g.cells = (int)std::min<long>(std::max<long>(round_pow2(std::max(L->n_samples_h, 1)) / 128, 1), (long)kSMs * 8);
    g.refine = std::min(g.samp, kSMs);
    g.btb = (int)std::min<long>(std::max<long>((round_pow2(std::max(L->n_occ_h, 1)) + 7) / 8, 1), (long)kSMs * 8);
    g.btb_build = (int)std::min<long>(
        std::max<long>((round_pow2(std::max(L->n_samples_h, 1)) + 8 * kBtbChunk - 1) / (8 * kBtbChunk), 1),
        (long)kSMs * 8);
    g.vec4 = L->all && (L->c.nx % 4 == 0);
    g.assoc = blocks_for(4L * round_pow2(std::max(L->n_samples_h, 1)));
    g.fit = blocks_for(L->c.nn, kFitTile, 4);
    return g;
}

// the rotation step (Sec. 7.1) and E_reg on stream st: node data staged in shared memory
// on an all-nodes lattice
template <bool kAll, bool kFit>
void launch_fit_rotations(const Ctx &c, Scal *sc, const Grid &gr, cudaStream_t st) {
    if (kAll) k_fit_rotations_staged<kFit><<<gr.fit, kFitTile, 0, st>>>(c, sc);
    else k_fit_rotations<kAll, kFit><<<gr.node, kThreads, 0, st>>>(c, sc);
}

// Launches the kernels of a schedule on one stream.  Consecutive kernels are chained
// with programmatic dependent launch (every solve kernel starts with pdl_wait), and a
// launch of the kernel class selected for profiling is bracketed by CUDA events (which
// break the chain around it).
struct Launcher {
    vd_lattice *L;
    cudaStream_t st;
    bool chain = false;
    template <typename... KArgs, typename... Args>
    void go(int kc, void (*kern)(KArgs...), dim3 grid, dim3 block, Args... args) {
        const bool prof = L->prof_class == kc && L->ev_used + 2 <= (int)L->ev.size();
        if (prof) {
            cudaEventRecordWithFlags(L->ev[L->ev_used], st, cudaEventRecordExternal);
            chain = false;
        }
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = grid;
        cfg.blockDim = block;
        cfg.dynamicSmemBytes = 0;
        cfg.stream = st;
        cudaLaunchAttribute at[1];
        if (chain && L->use_pdl) {
            at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
            at[0].val.programmaticStreamSerializationAllowed = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
        }
        cudaLaunchKernelEx(&cfg, kern, args...);
        chain = true;
        L->counting++;
        if (prof) {
            cudaEventRecordWithFlags(L->ev[L->ev_used + 1], st, cudaEventRecordExternal);
            L->ev_used += 2;
            chain = false;
        }
    }
    void other() { chain = false; }  // a memset or copy was enqueued
};

template <bool kAll>
void enqueue_rhs(Launcher &Lc, const Ctx &c, Scal *sc, const Grid &gr, int K) {
    Lc.go(VD_KC_RHS, k_rhs_nodes<kAll>, gr.node, kThreads, c, (const Scal *)sc);
    Lc.go(VD_KC_RHS, k_cells<kOpRhs, kAll>, gr.cells, kThreads, c, sc, K, 0);
}

template <bool kAll>
void enqueue_apply(Launcher &Lc, const Ctx &c, Scal *sc, const Grid &gr, int K, int it) {
    if (gr.vec4) Lc.go(VD_KC_APPLY_STENCIL, k_apply_stencil<kAll, true>, gr.node4, kThreads, c, sc, K, it);
    else Lc.go(VD_KC_APPLY_STENCIL, k_apply_stencil<kAll, false>, gr.node, kThreads, c, sc, K, it);
    if (c.btb) Lc.go(VD_KC_APPLY_SAMPLES, k_cells_btb<kAll>, gr.btb, kThreads, c, sc, K, it);
    else Lc.go(VD_KC_APPLY_SAMPLES, k_cells<kOpApply, kAll>, gr.cells, kThreads, c, sc, K, it);
}

// the cached blocks from this association's records (when the lattice uses them)
template <bool kAll>
void enqueue_btb(Launcher &Lc, const Ctx &c, Scal *sc, const Grid &gr, int n_occ) {
    if (!c.btb) return;
    cudaMemsetAsync(c.btb, 0, sizeof(float) * kBtb * (size_t)std::max(n_occ, 1), Lc.st);
    Lc.other();
    Lc.go(VD_KC_RHS, k_btb_build<kAll>, gr.btb_build, kThreads, c, (const Scal *)sc);
}

// PCG position step: init, then K x (apply, x/r update, p update)
template <bool kAll>
void enqueue_pcg(Launcher &Lc, const Ctx &c, Scal *sc, const Grid &gr, int K, double tol2) {
    Lc.go(VD_KC_RHS, k_pcg_init<kAll>, dim3(gr.node, 3), kThreads, c, sc);
    for (int it = 0; it < K; it++) {
        enqueue_apply<kAll>(Lc, c, sc, gr, K, it);
        Lc.go(VD_KC_UPDATE_X, k_update_x<kAll>, gr.node4, kThreads, c, sc, K, it);
        Lc.go(VD_KC_UPDATE_P, k_update_p<kAll>, gr.node4, kThreads, c, sc, it, tol2);
    }
}

// 9 floats per slot in shared memory (p, z / q and Minv; r and x are in tensor memory),
// and at most kPcgMaxGroups float4 groups per thread
constexpr int kPcgMaxChunk = 4 * kPcgMaxGroups * kPcgThreads;
constexpr int kPcgSmemPerSlot = 36;

// A brick plan for the persistent position step of an all-nodes lattice: bricks of by x
// bz x-rows, each row held as lx = nx rounded up to a multiple of 4 slots in shared
// memory; G = ceil(ny / by) ceil(nz / bz) CTAs of chunk = by bz lx slots.  Exact (the
// unpadded kernel form): nx % 4 == 0 and the bricks tile the lattice; otherwise a padded
// brick (k_pcg_persistent<.., true>).
struct BrickPlan {
    int by = 0, bz = 0, lx = 0, G = 0, chunk = 0;
    bool exact = false;
};

// The cost of a brick: its rows plus the neighbour rows it reads from other CTAs
// (through L2), times lx; the padded form 10% dearer.  few == false: the cheapest brick
// with G <= gmax; few == true: the least SM time (G x cost) with gmin <= G <= gmax.
// by = 0 when none fits.
BrickPlan brick_search(const vd_lattice *L, long gmin, long gmax, bool few) {
    BrickPlan best;
    const Ctx &c = L->c;
    if (!L->all || !L->use_brick) return best;
    const int lx = 4 * ((c.nx + 3) / 4);
    gmax = std::min<long>(gmax, kPcgMaxCtas);
    long best_key = -1;
    for (int y = 1; y <= c.ny; y++)
        for (int z = 1; z <= c.nz && (long)y * z <= kPcgMaxRows && (long)y * z * lx <= kPcgMaxChunk; z++) {
            const long G = (long)((c.ny + y - 1) / y) * ((c.nz + z - 1) / z);
            if (G > gmax || G < gmin) continue;
            const bool exact = c.nx % 4 == 0 && c.ny % y == 0 && c.nz % z == 0;
            const long rows = (long)y * z;
            const long faces = (y < c.ny ? 2L * z : 0) + (z < c.nz ? 2L * y : 0);
            long cost = (rows + faces) * lx;
            if (!exact) cost += cost / 10;
            const long key = few ? G * cost : cost;
            if (best_key < 0 || key < best_key) {
                best_key = key;
                best = BrickPlan{y, z, lx, (int)G, (int)(rows * lx), exact};
            }
        }
    return best;
}

// The persistent position step's partition: bricks (b.by > 0), or contiguous slot ranges
// of `chunk` slots (b.by == 0)
struct PcgPlan {
    int G = 0, chunk = 0;
    BrickPlan b;
};

// The kernel form of a plan (the kPad of k_pcg_persistent): 0 exact bricks or contiguous
// ranges, 1 padded bricks with 16-byte-aligned rows (nx % 4 == 0), 2 padded bricks with
// unaligned rows (their published vectors in the lattice's pad_vecs)
int pcg_kpad(const vd_lattice *L, const PcgPlan &pl) {
    if (!pl.b.by || pl.b.exact) return 0;
    return L->c.nx % 4 ? 2 : 1;
}

// plane stride of the padded published vectors of plan pl
size_t pad_ld(const vd_lattice *L, const PcgPlan &pl) {
    return (((size_t)pl.b.lx * L->c.ny * L->c.nz) + 31) & ~(size_t)31;
}

// Whether the position step runs as one persistent cooperative kernel, with how many
// CTAs and how many slots per CTA: bricks where the cheapest one within the SM count holds
// at most 1.25x the slots of an even split (a padded brick: at most 2x, and only where an
// even split is 2,048 slots or more -- on smaller lattices the contiguous ranges measured
// faster), else contiguous ranges over all SMs.  A padded plan with unaligned rows needs
// the lattice's padded vectors, which ensure_pad allocates outside any capture: until
// then (want == false) the step is streamed instead.
bool persistent_plan(vd_lattice *L, int *G, int *chunk, PcgPlan *out = nullptr, bool want = false) {
    if (!L->use_persistent || !L->coop || L->in_batch) return false;
    PcgPlan pl;
    const int N = L->all ? L->c.nn : L->n_active_h;
    const long even = ((long)std::max(N, 1) + L->num_sms - 1) / L->num_sms;
    const BrickPlan b = brick_search(L, 1, L->num_sms, false);
    if (b.by && (b.exact ? 4L * b.chunk <= 5 * even : (long)b.chunk <= 2 * even && even >= 2048)) {
        pl.G = b.G;
        pl.chunk = b.chunk;
        pl.b = b;
    } else {
        const int N4 = 4 * ((std::max(N, 1) + 3) / 4);
        // all SMs take part even for a small active set: the samples' share of each
        // iteration is spread over the CTAs, and a barrier costs the same for any count
        int ch = (N4 + L->num_sms - 1) / L->num_sms;
        ch = std::max(4 * ((ch + 3) / 4), 4);
        if (ch > kPcgMaxChunk) return false;
        pl.chunk = ch;
        pl.G = (N4 + ch - 1) / ch;
        if (pl.G > std::min(L->num_sms, kPcgMaxCtas)) return false;
    }
    if (!want && pcg_kpad(L, pl) == 2 && !(L->pad_vecs && L->pad_ldp == pad_ld(L, pl))) return false;
    *G = pl.G;
    *chunk = pl.chunk;
    if (out) *out = pl;
    return true;
}

unsigned magic_of(int d) { return d > 0 ? (unsigned)(((1ull << 31) + (unsigned long long)d - 1) / (unsigned long long)d) : 0u; }


// the published vectors of kernel form 2 (allocated, and zeroed once, outside any capture)
vd_status ensure_pad(vd_lattice *L, const PcgPlan &pl, int kpad) {
    if (kpad != 2) return VD_OK;
    const size_t ldp = pad_ld(L, pl);
    if (L->pad_vecs && L->pad_ldp == ldp) return VD_OK;
    dfree(L, L->pad_vecs);
    L->pad_ldp = 0;
    TRY(dalloc(L, &L->pad_vecs, 12 * ldp));
    if (cudaMemsetAsync(L->pad_vecs, 0, sizeof(float) * 12 * ldp, L->stream) != cudaSuccess ||
        cudaStreamSynchronize(L->stream) != cudaSuccess)
        return fail(L, VD_ERR_CUDA, "zeroing the padded vectors");
    L->pad_ldp = ldp;
    return VD_OK;
}

// the aux block of a persistent position step on plan pl in kernel form kpad
PcgAux pcg_aux(const vd_lattice *L, double *part, unsigned long long *words, int extra, const PcgPlan &pl, int kpad) {
    const int lx = pl.b.by ? pl.b.lx : L->c.nx;
    PcgAux ax{part,     words,   extra,   (int *)(L->pcg_bar + 2), L->surf_flag, {L->c.p, L->vecs + 15 * (size_t)L->c.ld},
              pl.chunk, pl.b.by, pl.b.bz, lx,      magic_of(lx), magic_of(pl.b.by), nullptr, nullptr, 0,
              magic_of(L->c.nx)};
    if (kpad == 2) {
        float *v = L->pad_vecs;
        const size_t ldp = L->pad_ldp;
        ax.zpad = v;
        ax.pbuf[0] = v + 3 * ldp;
        ax.pbuf[1] = v + 6 * ldp;
        ax.qpad = v + 9 * ldp;
        ax.ldp = (long long)ldp;
    }
    return ax;
}

template <bool kAll>
void launch_persistent(vd_lattice *L, Launcher &Lc, Scal *sc, int K, double tol2, int apply) {
    int G = 0, chunk = 0;
    PcgPlan pl;
    if (!persistent_plan(L, &G, &chunk, &pl)) return;
    unsigned long long *words = reinterpret_cast<unsigned long long *>(L->pcg_part + (size_t)L->pcg_part_rows * L->num_sms);
    const int kpad = pcg_kpad(L, pl);
    const PcgAux ax = pcg_aux(L, L->pcg_part, words, L->stall_extra, pl, kpad);
    const bool prof = L->prof_class == VD_KC_PCG && L->ev_used + 2 <= (int)L->ev.size();
    cudaMemsetAsync(L->pcg_bar, 0, 4 * sizeof(unsigned), Lc.st);
    cudaMemsetAsync(words, 0, sizeof(unsigned long long) * (size_t)(2 * K + 1), Lc.st);
    Lc.other();
    if (prof) cudaEventRecordWithFlags(L->ev[L->ev_used], Lc.st, cudaEventRecordExternal);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(G);
    cfg.blockDim = dim3(kPcgThreads);
    cfg.dynamicSmemBytes = (size_t)kPcgSmemPerSlot * chunk;
    cfg.stream = Lc.st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const Ctx c = L->c;
    if (kAll && kpad == 1)
        cudaLaunchKernelEx(&cfg, k_pcg_persistent<true, true, 1>, c, sc, ax, K, tol2, apply);
    else if (kAll && kpad == 2)
        cudaLaunchKernelEx(&cfg, k_pcg_persistent<true, true, 2>, c, sc, ax, K, tol2, apply);
    else if (kAll && (pl.b.by || c.nx % 4 == 0)) cudaLaunchKernelEx(&cfg, k_pcg_persistent<kAll, true>, c, sc, ax, K, tol2, apply);
    else cudaLaunchKernelEx(&cfg, k_pcg_persistent<kAll, false>, c, sc, ax, K, tol2, apply);
    L->counting++;
    if (prof) {
        cudaEventRecordWithFlags(L->ev[L->ev_used + 1], Lc.st, cudaEventRecordExternal);
        L->ev_used += 2;
    }
    Lc.other();
}

// the stages of Gauss-Newton iteration g before its position step: association (unless
// frozen), right-hand side and diagonal, the cached blocks
template <bool kAll>
void enqueue_gn_pre(Launcher &Lc, vd_lattice *L, const vd_solve_params *P, int g) {
    const Grid gr = grids(L);
    const Ctx c = L->c;
    Scal *sc = slot(L, g);
    const int K = P->cg_iters;
    if (!(P->fixed_association && g > 0)) {
        Lc.go(VD_KC_ASSOCIATE, k_associate<kAll>, gr.assoc, kThreads, c, sc);
        // the FP64 re-association runs in the first blocks of the right-hand side's node pass
        Lc.go(VD_KC_RHS, k_rhs_nodes_refine<kAll>, gr.refine + gr.node, kThreads, c, sc, gr.refine);
        Lc.go(VD_KC_RHS, k_cells<kOpRhs, kAll>, gr.cells, kThreads, c, sc, K, 0);
        enqueue_btb<kAll>(Lc, c, sc, gr, L->n_occ_h);
    } else {
        enqueue_rhs<kAll>(Lc, c, sc, gr, K);  // the records, and so the cached blocks, are unchanged
    }
}

// the stages after the position step: rotation fit, energies, the energy-target gate
template <bool kAll>
void enqueue_gn_post(Launcher &Lc, vd_lattice *L, const vd_solve_params *P, int g) {
    const Grid gr = grids(L);
    const Ctx c = L->c;
    Scal *sc = slot(L, g);
    const int K = P->cg_iters;
    if (kAll) Lc.go(VD_KC_ROTATION, k_fit_rotations_staged<true>, gr.fit, kFitTile, c, sc);
    else Lc.go(VD_KC_ROTATION, k_fit_rotations<kAll, true>, gr.node, kThreads, c, sc);
    // the energies after the update (this iteration's correspondences): for the report
    // after the last iteration, and after every one when the energy target gates the next
    if (c.e_target || g + 1 == P->gn_iters) Lc.go(VD_KC_ENERGY, k_cells<kOpEnergy, kAll>, gr.cells, kThreads, c, sc, K, 0);
    if (c.e_target && g + 1 < P->gn_iters) Lc.go(-1, k_gn_gate, 1, 32, c, (const Scal *)sc, slot(L, g + 1));
}

template <bool kAll>
void enqueue_gn(Launcher &Lc, vd_lattice *L, const vd_solve_params *P, int g) {
    enqueue_gn_pre<kAll>(Lc, L, P, g);
    const Grid gr = grids(L);
    const Ctx c = L->c;
    Scal *sc = slot(L, g);
    const int K = P->cg_iters;
    int G = 0, chunk = 0;
    if (persistent_plan(L, &G, &chunk)) {
        launch_persistent<kAll>(L, Lc, sc, K, P->cg_tol * P->cg_tol, 1);
    } else {
        enqueue_pcg<kAll>(Lc, c, sc, gr, K, P->cg_tol * P->cg_tol);
        Lc.go(VD_KC_ROTATION, k_add_increment<kAll>, gr.node, kThreads, c, (const Scal *)sc);
    }
    enqueue_gn_post<kAll>(Lc, L, P, g);
}

// the start and the end of a solve: scalar blocks zeroed, the warp reset for VD_INIT_ZERO;
// the report
void enqueue_solve_begin(Launcher &Lc, vd_lattice *L, const vd_solve_params *P, cudaStream_t st) {
    cudaMemsetAsync(L->scal, 0, L->scal_stride * (size_t)P->gn_iters, st);
    Lc.other();
    if (P->init == VD_INIT_ZERO)
        Lc.go(-1, k_reset_warp, blocks_for(L->c.nn), kThreads, L->u, L->R, L->c.nn, L->c.ld);
}

void enqueue_solve_end(Launcher &Lc, vd_lattice *L, const vd_solve_params *P, cudaStream_t st) {
    Lc.go(-1, k_finish_report, 1, 32, (Scal *)L->scal, L->scal_stride, P->gn_iters, L->c, L->rep_dev,
          (const int *)(L->pcg_bar + 2));
    cudaMemcpyAsync(L->rep_host, L->rep_dev, 11 * sizeof(double), cudaMemcpyDeviceToHost, st);
}

void enqueue_solve(vd_lattice *L, const vd_solve_params *P, cudaStream_t st) {
    Launcher Lc{L, st};
    enqueue_solve_begin(Lc, L, P, st);
    for (int g = 0; g < P->gn_iters; g++) {
        if (L->all) enqueue_gn<true>(Lc, L, P, g);
        else enqueue_gn<false>(Lc, L, P, g);
    }
    enqueue_solve_end(Lc, L, P, st);
}

// upper bound on the launches of one kernel class in a solve (sizes the event pool)
int class_launches_per_solve(const vd_solve_params *P, int kc) {
    if (kc < 0) return 0;
    return std::max(P->cg_iters, 3) * P->gn_iters + 8;
}

vd_status build_graph(vd_lattice *L, const vd_solve_params *P) {
    const Grid gr = grids(L);
    int pG = 0, pch = 0;
    PcgPlan pl;
    if (persistent_plan(L, &pG, &pch, &pl, true)) TRY(ensure_pad(L, pl, pcg_kpad(L, pl)));
    persistent_plan(L, &pG, &pch, &pl);
    const int pby = pl.b.by, pbz = pl.b.bz;
    const int caps[6] = {gr.node, gr.samp, gr.cells, L->S * 65536 + pch, pby * 65536 + pbz,
                         gr.btb * 65536 + (L->c.btb ? L->n_occ_h : 0)};
    const bool same = L->gexec && L->ggen == L->gen && !memcmp(&L->gparams, P, sizeof(*P)) &&
                      !memcmp(L->gkey_caps, caps, sizeof(caps)) && !memcmp(&L->gctx, &L->c, sizeof(Ctx));
    if (same) return VD_OK;
    if (L->gexec) {
        cudaGraphExecDestroy(L->gexec);
        L->gexec = nullptr;
    }
    // profiling events for the selected class
    const int need = L->prof_class >= 0 ? 2 * class_launches_per_solve(P, L->prof_class) : 0;
    while ((int)L->ev.size() < need) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        L->ev.push_back(e);
    }
    L->ev_used = 0;
    L->counting = 0;
    cudaError_t e = cudaSuccess;
    for (int attempt = 0; attempt < 2; attempt++) {
        L->ev_used = 0;
        L->counting = 0;
        CK(cudaStreamBeginCapture(L->cap, cudaStreamCaptureModeThreadLocal));
        enqueue_solve(L, P, L->cap);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(L->cap, &graph);
        if (e == cudaSuccess) {
            e = cudaGraphInstantiate(&L->gexec, graph, 0);
            cudaGraphDestroy(graph);
        }
        if (e == cudaSuccess) break;
        cudaGetLastError();
        if (!L->use_persistent) break;
        L->use_persistent = false;  // the graph could not hold the cooperative launch: stream the PCG
    }
    if (e != cudaSuccess) return fail(L, VD_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
    L->launches_solve = L->counting;
    L->gparams = *P;
    L->gctx = L->c;
    memcpy(L->gkey_caps, caps, sizeof(caps));
    L->ggen = L->gen;
    return VD_OK;
}

vd_status collect_profile(vd_lattice *L) {
    for (int k = 0; k + 1 < L->ev_used; k += 2) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, L->ev[k], L->ev[k + 1]));
        L->prof_ms += ms;
        L->prof_launches++;
    }
    return VD_OK;
}

vd_status read_report(vd_lattice *L, vd_solve_report *out) {
    const double *r = L->rep_host;
    vd_status st = VD_OK;
    if (r[9] == 0.0) st = fail(L, VD_ERR_NUMERIC, "non-finite energy after the solve");
    if (r[10] != 0.0) st = fail(L, VD_ERR_TIMEOUT, "a grid barrier of the persistent position step timed out");
    if (out) {
        out->e_total = r[0];
        out->e_dense = r[1];
        out->e_sparse = r[2];
        out->e_reg = r[3];
        out->gn_done = (int)r[4];
        out->cg_done = (int)r[5];
        out->n_valid_corr = (int)r[6];
        out->n_degenerate_rot = (int)r[7];
        out->n_refined = (int)r[8];
        out->status = st;
    }
    return st;
}

vd_status frame_surface_flags(vd_lattice *L) {
    refresh_ctx(L);
    const Ctx c = L->c;
    cudaStream_t st = L->stream;
    CK(cudaMemsetAsync(L->surf_flag, 0, sizeof(int) * (size_t)c.ld, st));
    const int nb = blocks_for(std::max(L->cap_src, 1) + L->S);
    if (L->all) k_mark_surface<true><<<nb, kThreads, 0, st>>>(L->occ_cell, L->counts + 1, L->scell_s, L->S, c, L->surf_flag);
    else k_mark_surface<false><<<nb, kThreads, 0, st>>>(L->occ_cell, L->counts + 1, L->scell_s, L->S, c, L->surf_flag);
    CKL();
    return VD_OK;
}

vd_status frame_active_set(vd_lattice *L) {
    const Ctx c = L->c;
    cudaStream_t st = L->stream;
    if (L->all) return frame_surface_flags(L);
    CK(cudaMemsetAsync(L->mark, 0, sizeof(int) * (size_t)c.nn, st));
    k_mark_cells<<<blocks_for(std::max(L->cap_src, 1) + L->S), kThreads, 0, st>>>(L->occ_cell, L->counts + 1,
                                                                                   L->scell_s, L->S, c, L->mark);
    k_dilate<<<blocks_for(c.nn), kThreads, 0, st>>>(L->mark, c, L->act);
    scan_launch(L->act, c.nn, L->slot_of_node, L->counts, L->scan_sums, st);
    k_compact<<<blocks_for(c.nn), kThreads, 0, st>>>(L->act, c, L->slot_of_node, L->node_of_slot);
    k_neighbour_table<<<blocks_for(c.nn), kThreads, 0, st>>>(c, L->nbr);
    CKL();
    return frame_surface_flags(L);
}

vd_status sync_sizes(vd_lattice *L) {
    int h[2] = {0, 0};
    CK(cudaMemcpyAsync(h, L->counts, 2 * sizeof(int), cudaMemcpyDeviceToHost, L->stream));
    int ns = 0;
    if (L->start) CK(cudaMemcpyAsync(&ns, L->start + L->c.nn, sizeof(int), cudaMemcpyDeviceToHost, L->stream));
    CK(cudaStreamSynchronize(L->stream));
    L->n_active_h = L->all ? L->c.nn : h[0];
    L->n_occ_h = h[1];
    L->n_samples_h = ns;
    return VD_OK;
}

vd_status step_prepare(vd_lattice *L, const vd_solve_params *P, int K) {
    if (!L) return VD_ERR_INVALID_ARG;
    TRY(check_params(L, P));
    if (!L->have_frame) return fail(L, VD_ERR_STATE, "no frame");
    TRY(ensure_scal(L, 1, K));
    set_params_ctx(L->c, P);
    refresh_ctx(L);
    return VD_OK;
}

template <bool kAll>
void rhs_launch(vd_lattice *L, cudaStream_t st) {
    Launcher Lc{L, st};
    enqueue_rhs<kAll>(Lc, L->c, slot(L, 0), grids(L), 1);
}

}  // namespace

// ====================================================================== C ABI

extern "C" {

vd_status vd_create_lattice(const vd_lattice_desc *d, vd_lattice **out) {
    if (!d || !out) return VD_ERR_INVALID_ARG;
    *out = nullptr;
    if (d->nx < 2 || d->ny < 2 || d->nz < 2 || !(d->spacing > 0.f)) return VD_ERR_INVALID_ARG;
    if (d->active_mode != VD_ACTIVE_SURFACE && d->active_mode != VD_ACTIVE_ALL) return VD_ERR_INVALID_ARG;
    if (d->precision != VD_PREC_FP32 && d->precision != VD_PREC_MIXED) return VD_ERR_INVALID_ARG;
    const long nn = (long)d->nx * d->ny * d->nz;
    if (nn > (long)kScanTile * kScanTile) return VD_ERR_INVALID_ARG;  // scan limit: 16.7M nodes
    vd_lattice *L = new (std::nothrow) vd_lattice();
    if (!L) return VD_ERR_OOM;
    Ctx &c = L->c;
    c.nx = d->nx;
    c.ny = d->ny;
    c.nz = d->nz;
    c.nn = (int)nn;
    c.ld = (int)((nn + 31) / 32 * 32);
    if (nn * d->nx < (1L << 31) && nn * d->ny < (1L << 31)) {
        c.mdx = (unsigned)(((1ull << 31) + (unsigned long long)d->nx - 1) / (unsigned long long)d->nx);
        c.mdy = (unsigned)(((1ull << 31) + (unsigned long long)d->ny - 1) / (unsigned long long)d->ny);
    }
    c.ox = d->origin[0];
    c.oy = d->origin[1];
    c.oz = d->origin[2];
    c.h = d->spacing;
    for (int a = 0; a < 9; a++) c.Rg[a] = (a % 4 == 0) ? 1.f : 0.f;
    L->all = d->active_mode == VD_ACTIVE_ALL;
    L->precision = d->precision;
    c.mixed = d->precision == VD_PREC_MIXED;
    if (const char *e = getenv("VD_PDL")) L->use_pdl = atoi(e) != 0;
    vd_status s = VD_OK;
    auto bail = [&](vd_status st) {
        vd_destroy_lattice(L);
        return st;
    };
    if (d->cuda_stream) {
        L->stream = (cudaStream_t)d->cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&L->stream, cudaStreamNonBlocking) != cudaSuccess) return bail(VD_ERR_CUDA);
        L->own_stream = true;
    }
    if (cudaStreamCreateWithFlags(&L->cap, cudaStreamNonBlocking) != cudaSuccess) return bail(VD_ERR_CUDA);
    const size_t ld = c.ld;
    if ((s = dalloc(L, &L->u, 3 * ld)) || (s = dalloc(L, &L->R, 9 * ld)) || (s = dalloc(L, &L->vecs, 18 * ld)) ||
        (s = dalloc(L, &L->counts, 8)) || (s = dalloc(L, &L->cnt, ld)) || (s = dalloc(L, &L->start, ld + 1)) ||
        (s = dalloc(L, &L->staging, 9 * ld)) || (s = dalloc(L, &L->rep_dev, 16)))
        return bail(s);
    if ((s = dalloc(L, &L->surf_flag, ld)) || (s = dalloc(L, &L->pcg_bar, 4)) ||
        (s = dalloc(L, &L->cell_part, (size_t)kSMs * 8)))
        return bail(s);
    {
        int dev = 0, coop = 0, sms = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess) {
            L->coop = coop != 0;
            L->num_sms = sms;
        }
        const int bytes = kPcgSmemPerSlot * kPcgMaxChunk;
        if (cudaFuncSetAttribute(k_pcg_persistent<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) ||
            cudaFuncSetAttribute(k_pcg_persistent<true, true, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) ||
            cudaFuncSetAttribute(k_pcg_persistent<true, true, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) ||
            cudaFuncSetAttribute(k_pcg_persistent<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) ||
            cudaFuncSetAttribute(k_pcg_persistent<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes)) {
            cudaGetLastError();
            L->coop = false;
        }
        int occ = 0;
        if (L->coop && (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pcg_persistent<true, true>, kPcgThreads,
                                                                       bytes) != cudaSuccess || occ < 1)) {
            cudaGetLastError();
            L->coop = false;
        }
        if (const char *e = getenv("VD_PERSISTENT")) L->use_persistent = atoi(e) != 0;
        if (const char *e = getenv("VD_BRICK")) L->use_brick = atoi(e) != 0;
    }
    if (!L->all) {
        if ((s = dalloc(L, &L->slot_of_node, ld + 1)) || (s = dalloc(L, &L->node_of_slot, ld)) ||
            (s = dalloc(L, &L->nbr, 6 * ld)) || (s = dalloc(L, &L->mark, ld)) || (s = dalloc(L, &L->act, ld)))
            return bail(s);
    }
    if (cudaMallocHost(&L->rep_host, 16 * sizeof(double)) != cudaSuccess) return bail(VD_ERR_OOM);
    memset(L->rep_host, 0, 16 * sizeof(double));
    refresh_ctx(L);
    k_reset_warp<<<blocks_for(c.nn), kThreads, 0, L->stream>>>(L->u, L->R, c.nn, c.ld);
    if (cudaMemsetAsync(L->vecs, 0, sizeof(float) * 18 * ld, L->stream) != cudaSuccess ||
        cudaMemsetAsync(L->counts, 0, 8 * sizeof(int), L->stream) != cudaSuccess ||
        cudaMemsetAsync(L->pcg_bar, 0, 4 * sizeof(unsigned), L->stream) != cudaSuccess ||
        cudaMemsetAsync(L->start, 0, sizeof(int) * (ld + 1), L->stream) != cudaSuccess ||
        cudaStreamSynchronize(L->stream) != cudaSuccess)
        return bail(VD_ERR_CUDA);
    *out = L;
    return VD_OK;
}

vd_status vd_destroy_lattice(vd_lattice *L) {
    if (!L) return VD_OK;
    if (L->stream) cudaStreamSynchronize(L->stream);
    if (L->rb_st) cudaStreamSynchronize(L->rb_st);
    if (L->gexec) cudaGraphExecDestroy(L->gexec);
    for (auto &b : L->bufs) cudaFree(b.ptr);
    for (auto e : L->ev) cudaEventDestroy(e);
    if (L->rep_host) cudaFreeHost(L->rep_host);
    if (L->cap) cudaStreamDestroy(L->cap);
    if (L->rb_st) {
        cudaStreamSynchronize(L->rb_st);
        cudaStreamDestroy(L->rb_st);
    }
    if (L->rb_ready) cudaEventDestroy(L->rb_ready);
    if (L->rb_done) cudaEventDestroy(L->rb_done);
    if (L->own_stream && L->stream) cudaStreamDestroy(L->stream);
    delete L;
    return VD_OK;
}

const char *vd_last_error(const vd_lattice *L) { return L ? L->err.c_str() : "null lattice"; }

vd_status vd_set_correspondences(vd_lattice *L, const float *canon, const float *target, int S, int mem) {
    if (!L) return VD_ERR_INVALID_ARG;
    if (S < 0 || (S > 0 && (!canon || !target))) return fail(L, VD_ERR_INVALID_ARG, "bad correspondences");
    if (S > L->cap_S) {
        dfree(L, L->sp_in);
        dfree(L, L->fh);
        dfree(L, L->ft);
        dfree(L, L->sfr);
        dfree(L, L->scell_s);
        L->cap_S = std::max(S, 64);
        TRY(dalloc(L, &L->sp_in, (size_t)L->cap_S * 6));
        TRY(dalloc(L, &L->fh, (size_t)L->cap_S));
        TRY(dalloc(L, &L->ft, (size_t)L->cap_S));
        TRY(dalloc(L, &L->sfr, (size_t)L->cap_S));
        TRY(dalloc(L, &L->scell_s, (size_t)L->cap_S));
    }
    L->S = S;
    L->frame_gen++;
    refresh_ctx(L);
    if (S > 0) {
        TRY(upload(L, L->sp_in, canon, sizeof(float) * 3 * S, mem));
        TRY(upload(L, L->sp_in + 3 * (size_t)S, target, sizeof(float) * 3 * S, mem));
        k_point_cells<<<blocks_for(S), kThreads, 0, L->stream>>>(L->sp_in, S, L->c, L->scell_s, L->sfr);
        k_pack_float4<<<blocks_for(S), kThreads, 0, L->stream>>>(L->sp_in, S, L->fh);
        k_pack_float4<<<blocks_for(S), kThreads, 0, L->stream>>>(L->sp_in + 3 * (size_t)S, S, L->ft);
        CKL();
    }
    if (L->have_frame) TRY(frame_active_set(L));
    TRY(sync_sizes(L));
    return VD_OK;
}

vd_status vd_set_frame(vd_lattice *L, const float *depth, int W, int H, const float K[4], const float pose[12],
                       const float *src_pts, const float *src_nrm, int n_src, int mem) {
    if (!L) return VD_ERR_INVALID_ARG;
    if (W < 3 || H < 3 || !depth || !K) return fail(L, VD_ERR_INVALID_ARG, "depth map must be at least 3x3");
    if (n_src < 0 || (n_src > 0 && (!src_pts || !src_nrm))) return fail(L, VD_ERR_INVALID_ARG, "bad samples");
    if (!(K[0] > 0) || !(K[1] > 0)) return fail(L, VD_ERR_INVALID_ARG, "focal lengths must be > 0");
    if ((long)W * H > (long)kScanTile * kScanTile || n_src > kScanTile * kScanTile)
        return fail(L, VD_ERR_INVALID_ARG, "frame too large");
    TRY(ensure_frame_caps(L, W, H, n_src));
    Ctx &c = L->c;
    L->W = W;
    L->H = H;
    c.W = W;
    c.H = H;
    c.fx = K[0];
    c.fy = K[1];
    c.cx = K[2];
    c.cy = K[3];
    for (int a = 0; a < 9; a++) c.Rg[a] = pose ? pose[a] : ((a % 4 == 0) ? 1.f : 0.f);
    for (int a = 0; a < 3; a++) c.tg[a] = pose ? pose[9 + a] : 0.f;
    L->n_src = n_src;
    L->frame_gen++;
    refresh_ctx(L);
    cudaStream_t st = L->stream;
    L->counting = 0;
    TRY(upload(L, L->depth, depth, sizeof(float) * (size_t)W * H, mem));
    TRY(upload(L, L->pts_in, src_pts, sizeof(float) * 3 * (size_t)n_src, mem));
    TRY(upload(L, L->nrm_in, src_nrm, sizeof(float) * 3 * (size_t)n_src, mem));
    k_sanitize_depth<<<blocks_for((long)W * H), kThreads, 0, st>>>(L->depth, W * H);
    dim3 b2(32, 8), g2((W + 31) / 32, (H + 7) / 8);
    k_target_normals<<<g2, b2, 0, st>>>(L->depth, L->nrm, W, H, c.fx, c.fy, c.cx, c.cy, c.mixed);
    // bin the samples by cell (counting sort with a deterministic order inside a cell)
    CK(cudaMemsetAsync(L->cnt, 0, sizeof(int) * (size_t)c.nn, st));
    CK(cudaMemsetAsync(L->head, 0, sizeof(int) * (size_t)L->cap_src, st));
    const int nb = blocks_for(std::max(n_src, 1));
    k_point_cells<<<nb, kThreads, 0, st>>>(L->pts_in, n_src, c, L->cell_in, L->frac_in, L->nrm_in);
    k_histogram<<<nb, kThreads, 0, st>>>(L->cell_in, n_src, L->cnt);
    scan_launch(L->cnt, c.nn, L->start, L->start + c.nn, L->scan_sums, st);
    k_bin_scatter<<<nb, kThreads, 0, st>>>(L->cell_in, n_src, L->start, L->cnt, L->tmp);
    k_bin_rank<<<nb, kThreads, 0, st>>>(L->tmp, L->cell_in, L->start, L->start + c.nn, L->order);
    k_bin_gather<<<nb, kThreads, 0, st>>>(L->order, L->start + c.nn, L->pts_in, L->nrm_in, L->cell_in, L->frac_in,
                                          L->sp, L->sn, L->scell, L->sfrac, L->perm, L->head);
    scan_launch(L->head, std::max(n_src, 1), L->hscan, L->counts + 1, L->scan_sums, st);
    k_occupied<<<nb, kThreads, 0, st>>>(L->head, L->hscan, L->start + c.nn, L->scell, L->counts + 1, L->occ_cell,
                                        L->occ_beg);
    CKL();
    L->have_frame = true;
    TRY(frame_active_set(L));
    TRY(sync_sizes(L));
    TRY(ensure_btb(L));
    refresh_ctx(L);
    const int nbc = grids(L).cells;
    k_cell_partition<<<(nbc + kThreads - 1) / kThreads, kThreads, 0, st>>>(L->occ_beg, L->counts + 1, nbc,
                                                                          L->cell_part);
    CKL();
    L->launches_frame = 14 + 2 + (L->all ? 0 : 7);
    return VD_OK;
}

vd_status vd_solve_async(vd_lattice *L, const vd_solve_params *P) {
    if (!L) return VD_ERR_INVALID_ARG;
    TRY(check_params(L, P));
    if (!L->have_frame) return fail(L, VD_ERR_STATE, "vd_solve before vd_set_frame");
    TRY(ensure_scal(L, P->gn_iters, P->cg_iters));
    set_params_ctx(L->c, P);
    refresh_ctx(L);
    TRY(build_graph(L, P));
    CK(cudaGraphLaunch(L->gexec, L->stream));
    L->solve_pending = true;
    return VD_OK;
}

vd_status vd_get_report(vd_lattice *L, vd_solve_report *out) {
    if (!L) return VD_ERR_INVALID_ARG;
    CK(cudaStreamSynchronize(L->stream));
    if (L->solve_pending && L->prof_class >= 0) TRY(collect_profile(L));
    L->solve_pending = false;
    return read_report(L, out);
}

vd_status vd_solve(vd_lattice *L, const vd_solve_params *P, vd_solve_report *out) {
    TRY(vd_solve_async(L, P));
    return vd_get_report(L, out);
}

vd_status vd_get_warp(const vd_lattice *Lc, float *disp, float *rot, int mem) {
    vd_lattice *L = const_cast<vd_lattice *>(Lc);
    if (!L) return VD_ERR_INVALID_ARG;
    const Ctx &c = L->c;
    cudaStream_t st = L->stream;
    if (disp) {
        k_soa_to_aos<<<blocks_for(c.nn), kThreads, 0, st>>>(L->u, 3, c.nn, c.ld, L->staging);
        CKL();
        TRY(download(L, disp, L->staging, sizeof(float) * 3 * (size_t)c.nn, mem));
        CK(cudaStreamSynchronize(st));
    }
    if (rot) {
        k_soa_to_aos<<<blocks_for(c.nn), kThreads, 0, st>>>(L->R, 9, c.nn, c.ld, L->staging);
        CKL();
        TRY(download(L, rot, L->staging, sizeof(float) * 9 * (size_t)c.nn, mem));
        CK(cudaStreamSynchronize(st));
    }
    return VD_OK;
}

vd_status vd_get_warp_async(vd_lattice *L, float *disp, float *rot, int mem) {
    if (!L) return VD_ERR_INVALID_ARG;
    if (mem != VD_MEM_HOST && mem != VD_MEM_DEVICE) return fail(L, VD_ERR_INVALID_ARG, "bad memory kind");
    const Ctx &c = L->c;
    if (!L->rb) {
        TRY(dalloc(L, &L->rb, 12 * (size_t)c.nn));
        if (cudaStreamCreateWithFlags(&L->rb_st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&L->rb_ready, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&L->rb_done, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return fail(L, VD_ERR_CUDA, "readback stream");
        }
    }
    cudaStream_t st = L->stream;
    // the previous copy is done with the readback buffer before it is written again
    CK(cudaStreamWaitEvent(st, L->rb_done, 0));
    if (disp) k_soa_to_aos<<<blocks_for(c.nn), kThreads, 0, st>>>(L->u, 3, c.nn, c.ld, L->rb);
    if (rot) k_soa_to_aos<<<blocks_for(c.nn), kThreads, 0, st>>>(L->R, 9, c.nn, c.ld, L->rb + 3 * (size_t)c.nn);
    CKL();
    CK(cudaEventRecord(L->rb_ready, st));
    CK(cudaStreamWaitEvent(L->rb_st, L->rb_ready, 0));
    const cudaMemcpyKind kind = mem == VD_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (disp) CK(cudaMemcpyAsync(disp, L->rb, sizeof(float) * 3 * (size_t)c.nn, kind, L->rb_st));
    if (rot) CK(cudaMemcpyAsync(rot, L->rb + 3 * (size_t)c.nn, sizeof(float) * 9 * (size_t)c.nn, kind, L->rb_st));
    CK(cudaEventRecord(L->rb_done, L->rb_st));
    return VD_OK;
}

vd_status vd_get_warp_wait(vd_lattice *L) {
    if (!L) return VD_ERR_INVALID_ARG;
    if (L->rb_done) CK(cudaEventSynchronize(L->rb_done));
    return VD_OK;
}

vd_status vd_set_warp(vd_lattice *L, const float *disp, const float *rot, int mem) {
    if (!L) return VD_ERR_INVALID_ARG;
    const Ctx &c = L->c;
    cudaStream_t st = L->stream;
    k_reset_warp<<<blocks_for(c.nn), kThreads, 0, st>>>(L->u, L->R, c.nn, c.ld);
    if (disp) {
        TRY(upload(L, L->staging, disp, sizeof(float) * 3 * (size_t)c.nn, mem));
        k_aos_to_soa<<<blocks_for(c.nn), kThreads, 0, st>>>(L->staging, 3, c.nn, c.ld, L->u);
    }
    if (rot) {  // same staging buffer: the copies and conversions are ordered on one stream
        TRY(upload(L, L->staging, rot, sizeof(float) * 9 * (size_t)c.nn, mem));
        k_aos_to_soa<<<blocks_for(c.nn), kThreads, 0, st>>>(L->staging, 9, c.nn, c.ld, L->R);
    }
    CKL();
    CK(cudaStreamSynchronize(st));
    return VD_OK;
}

vd_status vd_num_active(const vd_lattice *L, int *n) {
    if (!L || !n) return VD_ERR_INVALID_ARG;
    *n = L->all ? L->c.nn : (L->have_frame ? L->n_active_h : 0);
    return VD_OK;
}

vd_status vd_get_active(const vd_lattice *Lc, unsigned char *mask, int mem) {
    vd_lattice *L = const_cast<vd_lattice *>(Lc);
    if (!L || !mask) return VD_ERR_INVALID_ARG;
    const int nn = L->c.nn;
    std::vector<unsigned char> h(nn, 1);
    if (!L->all) {
        std::vector<int> s(nn);
        if (L->have_frame) {
            CK(cudaMemcpyAsync(s.data(), L->slot_of_node, sizeof(int) * nn, cudaMemcpyDeviceToHost, L->stream));
            CK(cudaStreamSynchronize(L->stream));
            for (int i = 0; i < nn; i++) h[i] = s[i] >= 0;
        } else {
            std::fill(h.begin(), h.end(), 0);
        }
    }
    if (mem == VD_MEM_DEVICE) {
        CK(cudaMemcpyAsync(mask, h.data(), nn, cudaMemcpyHostToDevice, L->stream));
        CK(cudaStreamSynchronize(L->stream));
    } else {
        memcpy(mask, h.data(), nn);
    }
    return VD_OK;
}

vd_status vd_get_target_normals(const vd_lattice *Lc, float *nrm, int mem) {
    vd_lattice *L = const_cast<vd_lattice *>(Lc);
    if (!L || !nrm) return VD_ERR_INVALID_ARG;
    if (!L->have_frame) return fail(L, VD_ERR_STATE, "no frame");
    const int n = L->W * L->H;
    std::vector<float4> h(n);
    CK(cudaMemcpyAsync(h.data(), L->nrm, sizeof(float4) * n, cudaMemcpyDeviceToHost, L->stream));
    CK(cudaStreamSynchronize(L->stream));
    std::vector<float> o(3 * (size_t)n);
    for (int i = 0; i < n; i++) {
        o[3 * i] = h[i].x;
        o[3 * i + 1] = h[i].y;
        o[3 * i + 2] = h[i].z;
    }
    if (mem == VD_MEM_DEVICE) {
        CK(cudaMemcpyAsync(nrm, o.data(), sizeof(float) * 3 * n, cudaMemcpyHostToDevice, L->stream));
        CK(cudaStreamSynchronize(L->stream));
    } else {
        memcpy(nrm, o.data(), sizeof(float) * 3 * n);
    }
    return VD_OK;
}

// ---- step API (eager launches on the lattice stream; scalar slot 0)

vd_status vd_step_associate(vd_lattice *L, const vd_solve_params *P) {
    TRY(step_prepare(L, P, std::max(P ? P->cg_iters : 0, 1)));
    const Grid gr = grids(L);
    CK(cudaMemsetAsync(L->scal, 0, L->scal_stride, L->stream));
    if (L->all) {
        k_associate<true><<<gr.assoc, kThreads, 0, L->stream>>>(L->c, slot(L, 0));
        k_associate_refine<true><<<gr.refine, kThreads, 0, L->stream>>>(L->c, slot(L, 0));
    } else {
        k_associate<false><<<gr.assoc, kThreads, 0, L->stream>>>(L->c, slot(L, 0));
        k_associate_refine<false><<<gr.refine, kThreads, 0, L->stream>>>(L->c, slot(L, 0));
    }
    CKL();
    CK(cudaStreamSynchronize(L->stream));
    return VD_OK;
}

vd_status vd_get_association(vd_lattice *L, const vd_solve_params *P, int *pix, float *w, float *r, int mem) {
    TRY(step_prepare(L, P, std::max(P ? P->cg_iters : 0, 1)));
    const int n = L->n_src;
    int *dp = L->res_i;
    float *dw = L->res_f, *dr = L->res_f + L->cap_src;
    k_clear_association<<<blocks_for(std::max(n, 1)), kThreads, 0, L->stream>>>(n, dp, dw, dr);
    if (L->all) k_unsort_association<true><<<blocks_for(std::max(n, 1)), kThreads, 0, L->stream>>>(L->c, dp, dw, dr);
    else k_unsort_association<false><<<blocks_for(std::max(n, 1)), kThreads, 0, L->stream>>>(L->c, dp, dw, dr);
    CKL();
    if (pix) TRY(download(L, pix, dp, sizeof(int) * n, mem));
    if (w) TRY(download(L, w, dw, sizeof(float) * n, mem));
    if (r) TRY(download(L, r, dr, sizeof(float) * n, mem));
    CK(cudaStreamSynchronize(L->stream));
    return VD_OK;
}

vd_status vd_step_rhs(vd_lattice *L, const vd_solve_params *P, float *b, float *diag, int mem) {
    TRY(step_prepare(L, P, 1));
    cudaStream_t st = L->stream;
    if (L->all) rhs_launch<true>(L, st);
    else rhs_launch<false>(L, st);
    const Ctx &c = L->c;
    float *out[2] = {b, diag};
    const float *src[2] = {c.r, c.minv};
    for (int k = 0; k < 2; k++) {
        if (!out[k]) continue;
        if (L->all) k_scatter_slots<true><<<blocks_for(c.nn), kThreads, 0, st>>>(src[k], c, L->staging);
        else k_scatter_slots<false><<<blocks_for(c.nn), kThreads, 0, st>>>(src[k], c, L->staging);
        CKL();
        TRY(download(L, out[k], L->staging, sizeof(float) * 3 * (size_t)c.nn, mem));
        CK(cudaStreamSynchronize(st));
    }
    CKL();
    CK(cudaStreamSynchronize(st));
    return VD_OK;
}

vd_status vd_step_apply(vd_lattice *L, const vd_solve_params *P, const float *p, float *Ap, double *pAp, int mem) {
    TRY(step_prepare(L, P, 1));
    if (!p || !Ap) return fail(L, VD_ERR_INVALID_ARG, "p and Ap are required");
    cudaStream_t st = L->stream;
    const Ctx &c = L->c;
    const Grid gr = grids(L);
    TRY(upload(L, L->staging, p, sizeof(float) * 3 * (size_t)c.nn, mem));
    CK(cudaMemsetAsync(L->scal, 0, L->scal_stride, st));
    Scal *sc = slot(L, 0);
    // the gates of the apply kernels read rho[0] > 0
    const double one = 1.0;
    CK(cudaMemcpyAsync((char *)sc + offsetof(Scal, rho), &one, sizeof(double), cudaMemcpyHostToDevice, st));
    Launcher Lc{L, st};
    if (L->all) {
        k_gather_slots<true><<<blocks_for(c.nn), kThreads, 0, st>>>(L->staging, c, c.p);
        enqueue_btb<true>(Lc, c, sc, gr, L->n_occ_h);
        enqueue_apply<true>(Lc, c, sc, gr, 1, 0);
        k_scatter_slots<true><<<blocks_for(c.nn), kThreads, 0, st>>>(c.q, c, L->staging);
    } else {
        k_gather_slots<false><<<blocks_for(c.nn), kThreads, 0, st>>>(L->staging, c, c.p);
        enqueue_btb<false>(Lc, c, sc, gr, L->n_occ_h);
        enqueue_apply<false>(Lc, c, sc, gr, 1, 0);
        k_scatter_slots<false><<<blocks_for(c.nn), kThreads, 0, st>>>(c.q, c, L->staging);
    }
    CKL();
    TRY(download(L, Ap, L->staging, sizeof(float) * 3 * (size_t)c.nn, mem));
    double h[4];
    CK(cudaMemcpyAsync(h, (char *)sc + offsetof(Scal, rho), 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (pAp) *pAp = h[2];  // pq[0] sits after rho[0..K] with K = 1
    return VD_OK;
}

vd_status vd_step_pcg(vd_lattice *L, const vd_solve_params *P, float *delta, int *iters, int apply, int mem) {
    TRY(step_prepare(L, P, std::max(P ? P->cg_iters : 0, 1)));
    cudaStream_t st = L->stream;
    const Ctx &c = L->c;
    const Grid gr = grids(L);
    const int K = P->cg_iters;
    TRY(ensure_scal(L, 1, K));
    Scal *sc = slot(L, 0);
    CK(cudaMemsetAsync(L->scal, 0, L->scal_stride, st));
    const double tol2 = P->cg_tol * P->cg_tol;
    Launcher Lc{L, st};
    int pG = 0, pch = 0;
    PcgPlan ppl;
    if (persistent_plan(L, &pG, &pch, &ppl, true)) TRY(ensure_pad(L, ppl, pcg_kpad(L, ppl)));
    if (persistent_plan(L, &pG, &pch, &ppl)) {
        if (L->all) {
            enqueue_rhs<true>(Lc, c, sc, gr, K);
            enqueue_btb<true>(Lc, c, sc, gr, L->n_occ_h);
            launch_persistent<true>(L, Lc, sc, K, tol2, apply);
            if (delta) k_scatter_slots<true><<<blocks_for(c.nn), kThreads, 0, st>>>(c.x, c, L->staging);
        } else {
            enqueue_rhs<false>(Lc, c, sc, gr, K);
            enqueue_btb<false>(Lc, c, sc, gr, L->n_occ_h);
            launch_persistent<false>(L, Lc, sc, K, tol2, apply);
            if (delta) k_scatter_slots<false><<<blocks_for(c.nn), kThreads, 0, st>>>(c.x, c, L->staging);
        }
    } else if (L->all) {
        enqueue_rhs<true>(Lc, c, sc, gr, K);
        enqueue_btb<true>(Lc, c, sc, gr, L->n_occ_h);
        enqueue_pcg<true>(Lc, c, sc, gr, K, tol2);
        Lc.other();
        if (delta) k_scatter_slots<true><<<blocks_for(c.nn), kThreads, 0, st>>>(c.x, c, L->staging);
        if (apply) k_add_increment<true><<<gr.node, kThreads, 0, st>>>(c, sc);
    } else {
        enqueue_rhs<false>(Lc, c, sc, gr, K);
        enqueue_btb<false>(Lc, c, sc, gr, L->n_occ_h);
        enqueue_pcg<false>(Lc, c, sc, gr, K, tol2);
        if (delta) k_scatter_slots<false><<<blocks_for(c.nn), kThreads, 0, st>>>(c.x, c, L->staging);
        if (apply) k_add_increment<false><<<gr.node, kThreads, 0, st>>>(c, sc);
    }
    CKL();
    if (delta) TRY(download(L, delta, L->staging, sizeof(float) * 3 * (size_t)c.nn, mem));
    int done = 0;
    CK(cudaMemcpyAsync(&done, (char *)sc + offsetof(Scal, cg_done), sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (iters) *iters = done;
    return VD_OK;
}

vd_status vd_step_fit_rotations(vd_lattice *L, int *n_degenerate) {
    if (!L) return VD_ERR_INVALID_ARG;
    if (!L->have_frame && !L->all) return fail(L, VD_ERR_STATE, "no frame");
    TRY(ensure_scal(L, 1, 1));
    refresh_ctx(L);
    cudaStream_t st = L->stream;
    const Grid gr = grids(L);
    CK(cudaMemsetAsync(L->scal, 0, L->scal_stride, st));
    if (L->all) launch_fit_rotations<true, true>(L->c, slot(L, 0), gr, st);
    else launch_fit_rotations<false, true>(L->c, slot(L, 0), gr, st);
    CKL();
    int d = 0;
    CK(cudaMemcpyAsync(&d, (char *)slot(L, 0) + offsetof(Scal, n_degenerate), sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (n_degenerate) *n_degenerate = d;
    return VD_OK;
}

vd_status vd_step_energy(vd_lattice *L, const vd_solve_params *P, double out[4]) {
    TRY(step_prepare(L, P, 1));
    if (!out) return fail(L, VD_ERR_INVALID_ARG, "out is NULL");
    cudaStream_t st = L->stream;
    const Grid gr = grids(L);
    Scal *sc = slot(L, 0);
    CK(cudaMemsetAsync(L->scal, 0, L->scal_stride, st));
    if (L->all) {
        launch_fit_rotations<true, false>(L->c, sc, gr, st);
        k_cells<kOpEnergy, true><<<gr.cells, kThreads, 0, st>>>(L->c, sc, 1, 0);
    } else {
        k_fit_rotations<false, false><<<gr.node, kThreads, 0, st>>>(L->c, sc);
        k_cells<kOpEnergy, false><<<gr.cells, kThreads, 0, st>>>(L->c, sc, 1, 0);
    }
    CKL();
    double h[3];
    CK(cudaMemcpyAsync(h, sc, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    out[1] = h[0];
    out[2] = h[1];
    out[3] = h[2];
    out[0] = (double)P->w_sparse * h[1] + (double)P->w_dense * h[0] + (double)P->w_reg * h[2];
    return VD_OK;
}

vd_status vd_estimate_pose(vd_lattice *L, const vd_solve_params *P, int iters, float pose_out[12], int *steps,
                           double *e_hist) {
    if (!L) return VD_ERR_INVALID_ARG;
    TRY(check_params(L, P));
    if (iters < 0 || iters > kIcpMaxSteps) return fail(L, VD_ERR_INVALID_ARG, "iters must be in [0, %d]", kIcpMaxSteps);
    if (!L->have_frame) return fail(L, VD_ERR_STATE, "vd_estimate_pose before vd_set_frame");
    if (!L->icp) {
        void *q = nullptr;
        if (cudaMalloc(&q, sizeof(IcpState)) != cudaSuccess) {
            cudaGetLastError();
            return fail(L, VD_ERR_OOM, "cudaMalloc of the pose state failed");
        }
        L->bufs.push_back({q, sizeof(IcpState)});
        L->icp = (IcpState *)q;
    }
    set_params_ctx(L->c, P);
    refresh_ctx(L);
    IcpState h{};
    for (int a = 0; a < 9; a++) h.pose[a] = L->c.Rg[a];
    for (int a = 0; a < 3; a++) h.pose[9 + a] = L->c.tg[a];
    cudaStream_t st = L->stream;
    CK(cudaMemcpyAsync(L->icp, &h, sizeof(IcpState), cudaMemcpyHostToDevice, st));
    const Grid gr = grids(L);
    for (int it = 0; it < iters; it++) {
        if (L->all) {
            k_icp_assoc<true><<<gr.samp, kThreads, 0, st>>>(L->c, L->icp);
            k_icp_refine<true><<<gr.refine, kThreads, 0, st>>>(L->c, L->icp);
        } else {
            k_icp_assoc<false><<<gr.samp, kThreads, 0, st>>>(L->c, L->icp);
            k_icp_refine<false><<<gr.refine, kThreads, 0, st>>>(L->c, L->icp);
        }
        k_icp_step<<<1, 32, 0, st>>>(L->icp);
    }
    CKL();
    CK(cudaMemcpyAsync(&h, L->icp, sizeof(IcpState), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    for (int a = 0; a < 9; a++) L->c.Rg[a] = (float)h.pose[a];
    for (int a = 0; a < 3; a++) L->c.tg[a] = (float)h.pose[9 + a];
    if (pose_out)
        for (int a = 0; a < 12; a++) pose_out[a] = (float)h.pose[a];
    if (steps) *steps = h.steps;
    if (e_hist)
        for (int k = 0; k < h.steps; k++) e_hist[k] = h.e_hist[k];
    return VD_OK;
}

vd_status vd_set_apply_mode(vd_lattice *L, int mode) {
    if (!L) return VD_ERR_INVALID_ARG;
    if (mode != VD_APPLY_MATRIX_FREE && mode != VD_APPLY_CACHED && mode != VD_APPLY_AUTO)
        return fail(L, VD_ERR_INVALID_ARG, "unknown apply mode %d", mode);
    L->apply_mode = mode;
    if (L->have_frame) TRY(ensure_btb(L));
    refresh_ctx(L);
    return VD_OK;
}

vd_status vd_get_apply_mode(const vd_lattice *L, int *mode, int *cached_now) {
    if (!L) return VD_ERR_INVALID_ARG;
    if (mode) *mode = L->apply_mode;
    if (cached_now) *cached_now = use_cached(L) ? 1 : 0;
    return VD_OK;
}

vd_status vd_tune_apply(vd_lattice *L, const vd_solve_params *P, int *mode_out, float ms_out[2]) {
    if (!L) return VD_ERR_INVALID_ARG;
    TRY(check_params(L, P));
    if (!L->have_frame) return fail(L, VD_ERR_STATE, "vd_tune_apply before vd_set_frame");
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float ms[2] = {0.f, 0.f};
    const int modes[2] = {VD_APPLY_MATRIX_FREE, VD_APPLY_CACHED};
    vd_status st = VD_OK;
    for (int k = 0; k < 2 && st == VD_OK; k++) {
        st = vd_set_apply_mode(L, modes[k]);
        for (int rep = 0; rep < 3 && st == VD_OK; rep++) {  // the first replay warms up
            if (rep == 1) cudaEventRecord(e0, L->stream);
            st = vd_solve_async(L, P);
        }
        cudaEventRecord(e1, L->stream);
        if (st == VD_OK && cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms[k], e0, e1);
        ms[k] *= 0.5f;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != VD_OK) return st;
    const int best = ms[1] < ms[0] ? VD_APPLY_CACHED : VD_APPLY_MATRIX_FREE;
    TRY(vd_set_apply_mode(L, best));
    if (mode_out) *mode_out = best;
    if (ms_out) {
        ms_out[0] = ms[0];
        ms_out[1] = ms[1];
    }
    return VD_OK;
}

vd_status vd_profile_select(vd_lattice *L, int kc) {
    if (!L || kc < -1 || kc >= VD_KC_COUNT) return VD_ERR_INVALID_ARG;
    if (kc != L->prof_class) {
        L->prof_class = kc;
        L->ggen = -1;  // force a re-capture
    }
    L->prof_ms = 0.0;
    L->prof_launches = 0;
    return VD_OK;
}

vd_status vd_profile_read(vd_lattice *L, double *total_ms, int *launches) {
    if (!L) return VD_ERR_INVALID_ARG;
    if (total_ms) *total_ms = L->prof_ms;
    if (launches) *launches = L->prof_launches;
    L->prof_ms = 0.0;
    L->prof_launches = 0;
    return VD_OK;
}

vd_status vd_launch_counts(vd_lattice *L, const vd_solve_params *P, int *per_solve, int *per_frame) {
    if (!L || !P) return VD_ERR_INVALID_ARG;
    TRY(check_params(L, P));
    const int G = P->gn_iters, K = P->cg_iters;
    const int assoc = P->fixed_association ? 1 : G;
    int pG = 0, pch = 0;
    const int per_gn = persistent_plan(L, &pG, &pch) ? 2 + 1 + 2 : 3 + 4 * K + 3;
    const int n = assoc * (use_cached(L) ? 2 : 1) + G * per_gn + 1 + (P->init == VD_INIT_ZERO ? 1 : 0);
    if (per_solve) *per_solve = n;
    if (per_frame) *per_frame = L->launches_frame;
    return VD_OK;
}

vd_status vd_pcg_plan(vd_lattice *L, int *ctas, int *chunk, int *by, int *bz, int *padded) {
    if (!L) return VD_ERR_INVALID_ARG;
    int G = 0, ch = 0;
    PcgPlan pl;
    if (!persistent_plan(L, &G, &ch, &pl)) pl = PcgPlan{};
    if (ctas) *ctas = pl.G;
    if (chunk) *chunk = pl.chunk;
    if (by) *by = pl.b.by;
    if (bz) *bz = pl.b.bz;
    if (padded) *padded = pl.b.by && !pl.b.exact ? 1 : 0;
    return VD_OK;
}

}  // extern "C"

// ====================================================================== batched solve
//
// A batch captures the solve schedules of many lattices into one CUDA graph: each
// lattice's schedule is a branch on one of P capture streams, so the small lattices'
// kernels run concurrently with the large ones'.  The position steps are streamed
// (several cooperative persistent kernels cannot be co-resident at once).  vd_batch_tune
// times candidate stream counts and branch orders on the batch itself and keeps the
// fastest.

struct vd_batch {
    std::vector<vd_lattice *> L;
    cudaStream_t cap = nullptr;
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr, t0 = nullptr, t1 = nullptr;
    cudaGraphExec_t gexec = nullptr;
    std::vector<char> key;
    vd_solve_params gparams{};
    int streams = 0;           // concurrent branches (0: not tuned, use min(count, 8))
    bool largest_first = true;
    long coop_min = 0x7fffffffL;  // lattices of at least this many active nodes run their
                                  // persistent position step, one after another, before
                                  // the concurrent branches of the others
    bool pending = false;
    int launches = 0;
    std::string err;
    // persistent position step over every lattice (one cooperative launch per Gauss-Newton
    // iteration): threads per CTA, CTAs per SM, weight of a sample against a node in the
    // split of the CTAs among the lattices
    bool persistent = false;
    // position steps in waves of the shared-memory persistent step (k_pcg_wave, one
    // cooperative launch per Gauss-Newton iteration); overrides `persistent`
    bool waves = false;
    int wave_share = 1 << 20;        // samples per CTA that size a lattice's group (at most)
    int pthreads = 512, pctas = 1;
    float sample_weight = 2.f;
    std::vector<void *> pbufs;       // items, barrier words, partial rows
    PcgBatchItem *items = nullptr;
    unsigned long long *words = nullptr;
    double *part = nullptr;
    size_t cap_items = 0, cap_words = 0, cap_part = 0;
    std::vector<int> groups;         // CTAs per lattice of the last persistent build
    int2 *wplan = nullptr;           // wave form: the CTAs' plan of every launch set
    size_t cap_wplan = 0;
    int n_waves = 0;
};

namespace {

vd_status bfail(vd_batch *B, vd_status s, const char *msg) {
    B->err = msg;
    return s;
}

long active_nodes(const vd_lattice *L) { return L->all ? L->c.nn : L->n_active_h; }

std::vector<char> batch_key(vd_batch *B, const vd_solve_params *P, int streams, bool largest, long coop_min) {
    std::vector<char> k;
    auto put = [&](const void *p, size_t n) { k.insert(k.end(), (const char *)p, (const char *)p + n); };
    put(P, sizeof(*P));
    put(&streams, sizeof(streams));
    put(&largest, sizeof(largest));
    put(&coop_min, sizeof(coop_min));
    put(&B->persistent, sizeof(B->persistent));
    put(&B->waves, sizeof(B->waves));
    put(&B->wave_share, sizeof(B->wave_share));
    put(&B->pthreads, sizeof(B->pthreads));
    put(&B->pctas, sizeof(B->pctas));
    put(&B->sample_weight, sizeof(B->sample_weight));
    for (vd_lattice *L : B->L) {
        put(&L->gen, sizeof(L->gen));
        put(&L->c, sizeof(Ctx));
        const Grid g = grids(L);
        put(&g, sizeof(g));
    }
    return k;
}

std::vector<int> batch_order(vd_batch *B, bool largest) {
    std::vector<int> o(B->L.size());
    for (size_t i = 0; i < o.size(); i++) o[i] = (int)i;
    if (largest) {
        std::stable_sort(o.begin(), o.end(),
                         [&](int a, int b) { return active_nodes(B->L[a]) > active_nodes(B->L[b]); });
    }
    return o;
}

vd_status batch_build_persistent(vd_batch *B, const vd_solve_params *P, int streams, bool largest);
vd_status batch_build_waves(vd_batch *B, const vd_solve_params *P, int streams, bool largest);

vd_status batch_build(vd_batch *B, const vd_solve_params *P, int streams, bool largest, long coop_min) {
    std::vector<char> key = batch_key(B, P, streams, largest, coop_min);
    if (B->gexec && key == B->key) return VD_OK;
    if (B->waves || B->persistent) {
        vd_status s = B->waves ? batch_build_waves(B, P, streams, largest) : batch_build_persistent(B, P, streams, largest);
        if (s == VD_OK) {
            B->key = key;
            B->gparams = *P;
        }
        return s;
    }
    if (B->gexec) {
        cudaGraphExecDestroy(B->gexec);
        B->gexec = nullptr;
    }
    while ((int)B->side.size() < streams) {
        cudaStream_t st;
        cudaEvent_t ev;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return bfail(B, VD_ERR_CUDA, "stream");
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return bfail(B, VD_ERR_CUDA, "event");
        B->side.push_back(st);
        B->join.push_back(ev);
    }
    for (vd_lattice *L : B->L) {
        vd_status s = ensure_scal(L, P->gn_iters, P->cg_iters);
        if (s != VD_OK) return bfail(B, s, L->err.c_str());
        set_params_ctx(L->c, P);
        refresh_ctx(L);
        int pG = 0, pch = 0;
        PcgPlan pl;
        if (active_nodes(L) >= coop_min && persistent_plan(L, &pG, &pch, &pl, true)) {
            s = ensure_pad(L, pl, pcg_kpad(L, pl));  // a run-ahead lattice's padded vectors
            if (s != VD_OK) return bfail(B, s, L->err.c_str());
        }
    }
    const std::vector<int> order = batch_order(B, largest);
    if (cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return bfail(B, VD_ERR_CUDA, "begin capture");
    int launches = 0;
    // the large lattices first, one after another on the capture stream: each one's
    // persistent position step has the whole GPU (its CTAs must all be resident)
    for (int idx : order) {
        vd_lattice *L = B->L[idx];
        if (active_nodes(L) < coop_min) continue;
        const int saved = L->prof_class;
        L->prof_class = -1;
        L->counting = 0;
        enqueue_solve(L, P, B->cap);
        launches += L->counting;
        L->prof_class = saved;
    }
    cudaEventRecord(B->fork, B->cap);
    for (int p = 0; p < streams; p++) cudaStreamWaitEvent(B->side[p], B->fork, 0);
    int k = 0;
    for (int idx : order) {
        vd_lattice *L = B->L[idx];
        if (active_nodes(L) >= coop_min) continue;
        const int saved = L->prof_class;
        L->prof_class = -1;
        L->in_batch = true;
        L->counting = 0;
        enqueue_solve(L, P, B->side[k++ % streams]);
        launches += L->counting;
        L->in_batch = false;
        L->prof_class = saved;
    }
    for (int p = 0; p < streams; p++) {
        cudaEventRecord(B->join[p], B->side[p]);
        cudaStreamWaitEvent(B->cap, B->join[p], 0);
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(B->cap, &graph);
    if (e == cudaSuccess) {
        e = cudaGraphInstantiate(&B->gexec, graph, 0);
        cudaGraphDestroy(graph);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return bfail(B, VD_ERR_CUDA, cudaGetErrorString(e));
    }
    B->key = key;
    B->gparams = *P;
    B->launches = launches;
    return VD_OK;
}

template <typename T>
vd_status bgrow(vd_batch *B, T **p, size_t *cap, size_t need) {
    if (need <= *cap && *p) return VD_OK;
    for (size_t k = 0; k < B->pbufs.size(); k++)
        if (B->pbufs[k] == (void *)*p) {
            cudaFree(*p);
            B->pbufs.erase(B->pbufs.begin() + k);
            break;
        }
    *p = nullptr;
    *cap = 0;
    void *q = nullptr;
    if (cudaMalloc(&q, std::max<size_t>(need, 1) * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return bfail(B, VD_ERR_OOM, "batch buffers");
    }
    B->pbufs.push_back(q);
    *p = (T *)q;
    *cap = need;
    return VD_OK;
}

int batch_threads_ok(int t) { return t == 256 || t == 512; }

int batch_occupancy(int threads) {
    int occ = 0;
    cudaError_t e = threads == 256
                        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pcg_batch<256>, 256, 0)
                        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_pcg_batch<512>, 512, 0);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return occ;
}

// Capture a batch graph whose position steps run as cooperative launches: the lattices'
// stages before the first position step as branches on `streams` capture streams, then
// per Gauss-Newton iteration gi the launches that steps(gi) enqueues on the capture stream
// (it returns their count), then the stages after it as branches again.
template <typename Steps>
vd_status batch_capture(vd_batch *B, const vd_solve_params *P, int streams, bool largest, Steps steps) {
    const int GN = P->gn_iters;
    while ((int)B->side.size() < streams) {
        cudaStream_t st;
        cudaEvent_t ev;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return bfail(B, VD_ERR_CUDA, "stream");
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return bfail(B, VD_ERR_CUDA, "event");
        B->side.push_back(st);
        B->join.push_back(ev);
    }
    if (B->gexec) {
        cudaGraphExecDestroy(B->gexec);
        B->gexec = nullptr;
    }
    const std::vector<int> order = batch_order(B, largest);
    if (cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return bfail(B, VD_ERR_CUDA, "begin capture");
    int launches = 0;
    auto fork = [&]() {
        cudaEventRecord(B->fork, B->cap);
        for (int p = 0; p < streams; p++) cudaStreamWaitEvent(B->side[p], B->fork, 0);
    };
    auto joinall = [&]() {
        for (int p = 0; p < streams; p++) {
            cudaEventRecord(B->join[p], B->side[p]);
            cudaStreamWaitEvent(B->cap, B->join[p], 0);
        }
    };
    // the lattices' segments: before the first position step, and between position steps
    auto segment = [&](int gi) {  // gi < 0: start + pre(0); else post(gi) + pre(gi + 1) or end
        fork();
        int k = 0;
        for (int idx : order) {
            vd_lattice *L = B->L[idx];
            cudaStream_t st = B->side[k++ % streams];
            const int saved = L->prof_class;
            L->prof_class = -1;
            L->counting = 0;
            Launcher Lc{L, st};
            if (gi < 0) {
                enqueue_solve_begin(Lc, L, P, st);
                cudaMemsetAsync(L->pcg_bar, 0, 4 * sizeof(unsigned), st);
                Lc.other();
            } else if (L->all) {
                enqueue_gn_post<true>(Lc, L, P, gi);
            } else {
                enqueue_gn_post<false>(Lc, L, P, gi);
            }
            const int nxt = gi + 1;
            if (nxt < GN) {
                if (L->all) enqueue_gn_pre<true>(Lc, L, P, nxt);
                else enqueue_gn_pre<false>(Lc, L, P, nxt);
            } else {
                enqueue_solve_end(Lc, L, P, st);
            }
            launches += L->counting;
            L->prof_class = saved;
        }
        joinall();
    };
    segment(-1);
    for (int gi = 0; gi < GN; gi++) {
        launches += steps(gi);
        segment(gi);
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(B->cap, &graph);
    if (e == cudaSuccess) {
        e = cudaGraphInstantiate(&B->gexec, graph, 0);
        cudaGraphDestroy(graph);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return bfail(B, VD_ERR_CUDA, cudaGetErrorString(e));
    }
    B->launches = launches;
    return VD_OK;
}

// One graph per batch: for every Gauss-Newton iteration, the lattices' stages before the
// position step as branches on `streams` capture streams, then one cooperative launch of
// k_pcg_batch for all position steps, then the stages after it as branches again.  The
// CTAs (SMs x CTAs per SM) are split among the lattices in proportion to (active nodes +
// sample_weight x samples), at least one each.
vd_status batch_build_persistent(vd_batch *B, const vd_solve_params *P, int streams, bool largest) {
    const int n = (int)B->L.size();
    // a solve of the previous graph may still read the items and buffers rewritten below
    if (cudaStreamSynchronize(B->L[0]->stream) != cudaSuccess) return bfail(B, VD_ERR_CUDA, "synchronize");
    const int K = P->cg_iters, GN = P->gn_iters;
    const int occ = batch_occupancy(B->pthreads);
    const int sms = B->L[0]->num_sms;
    if (!B->L[0]->coop || occ < B->pctas || n > sms * B->pctas)
        return bfail(B, VD_ERR_INVALID_ARG, "the persistent batch does not fit on the device with these settings");
    const int T = sms * B->pctas;
    std::vector<double> w(n);
    double W = 0.0;
    for (int i = 0; i < n; i++) {
        vd_lattice *L = B->L[i];
        vd_status s = ensure_scal(L, GN, K);
        if (s == VD_OK && !L->batch_vecs) s = dalloc(L, &L->batch_vecs, 6 * (size_t)L->c.ld);
        if (s != VD_OK) return bfail(B, s, L->err.c_str());
        set_params_ctx(L->c, P);
        refresh_ctx(L);
        const long N = active_nodes(L);
        w[i] = (double)(4 * ((N + 3) / 4)) + (double)B->sample_weight * L->n_samples_h;
        W += w[i];
    }
    // CTAs per lattice: at least one, the rest by the largest remainders; no more than
    // 255 (the arrival count of a barrier word) or one per float4 group
    std::vector<int> g(n, 1);
    std::vector<std::pair<double, int>> rem;
    int used = n;
    for (int i = 0; i < n; i++) {
        const double want = T * w[i] / std::max(W, 1.0);
        const int extra = std::max(0, (int)want - 1);
        g[i] += extra;
        used += extra;
        rem.push_back({want - (int)want, i});
    }
    std::sort(rem.begin(), rem.end(), [](const std::pair<double, int> &a, const std::pair<double, int> &b) {
        return a.first > b.first;
    });
    for (size_t k = 0; used < T && k < rem.size(); k++, used++) g[rem[k].second]++;
    while (used > T) {  // forced minimums overshot: take CTAs back from the largest groups
        int big = (int)(std::max_element(g.begin(), g.end()) - g.begin());
        if (g[big] <= 1) break;
        g[big]--;
        used--;
    }
    long words_need = 0, part_need = 0;
    std::vector<long> woff(n), poff(n);
    std::vector<int> chunk(n), g0(n);
    int start = 0;
    for (int i = 0; i < n; i++) {
        vd_lattice *L = B->L[i];
        const long N = active_nodes(L), G4 = (N + 3) / 4;
        g[i] = (int)std::max<long>(1, std::min<long>(std::min<long>(g[i], 255), G4));
        chunk[i] = (int)(4 * ((G4 + g[i] - 1) / g[i]));
        g0[i] = start;
        start += g[i];
        woff[i] = words_need;
        words_need += 2 * K + 1;
        poff[i] = part_need;
        part_need += (long)(2 * K + 2) * g[i];
    }
    const int grid = start;
    vd_status s = bgrow(B, &B->items, &B->cap_items, (size_t)GN * n);
    if (s == VD_OK) s = bgrow(B, &B->words, &B->cap_words, (size_t)words_need);
    if (s == VD_OK) s = bgrow(B, &B->part, &B->cap_part, (size_t)part_need);
    if (s != VD_OK) return s;
    std::vector<PcgBatchItem> items((size_t)GN * n);
    for (int gi = 0; gi < GN; gi++)
        for (int i = 0; i < n; i++) {
            vd_lattice *L = B->L[i];
            PcgBatchItem &it = items[(size_t)gi * n + i];
            it.c = L->c;
            it.sc = slot(L, gi);
            it.part = B->part + poff[i];
            it.words = B->words + woff[i];
            it.z = L->batch_vecs;
            it.qs = L->batch_vecs + 3 * (size_t)L->c.ld;
            it.pbuf1 = L->vecs + 15 * (size_t)L->c.ld;
            it.err = (int *)(L->pcg_bar + 2);
            it.g0 = g0[i];
            it.G = g[i];
            it.chunk = chunk[i];
            const unsigned long long two31 = 1ull << 31;
            it.m_nx = (unsigned)((two31 + (unsigned long long)L->c.nx - 1) / (unsigned long long)L->c.nx);
            it.m_ny = (unsigned)((two31 + (unsigned long long)L->c.ny - 1) / (unsigned long long)L->c.ny);
        }
    if (cudaMemcpy(B->items, items.data(), sizeof(PcgBatchItem) * items.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return bfail(B, VD_ERR_CUDA, "item upload");
    B->groups = g;
    B->n_waves = 0;
    const double tol2 = P->cg_tol * P->cg_tol;
    return batch_capture(B, P, streams, largest, [&](int gi) {
        cudaMemsetAsync(B->words, 0, sizeof(unsigned long long) * (size_t)words_need, B->cap);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(B->pthreads);
        cfg.stream = B->cap;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeCooperative;
        at[0].val.cooperative = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        const PcgBatchItem *its = B->items + (size_t)gi * n;
        if (B->pthreads == 256) cudaLaunchKernelEx(&cfg, k_pcg_batch<256>, its, n, K, tol2, 1);
        else cudaLaunchKernelEx(&cfg, k_pcg_batch<512>, its, n, K, tol2, 1);
        return 1;
    });
}

// Position-step plan of one lattice inside a wave: the fewest CTAs that hold at most
// `share` of the lattice's samples each (a CTA's sample warps take a share of them beside
// its stencil; as far as the SMs allow) and whose slots fit in shared memory: bricks for
// an all-nodes lattice, contiguous ranges for a surface set.  G = 0 when none fits.
PcgPlan wave_plan(const vd_lattice *L, int cap, int share) {
    PcgPlan w;
    const long N = std::max(active_nodes(L), 1L), N4 = 4 * ((N + 3) / 4);
    const long g_samples = ((long)L->n_samples_h + share - 1) / share;
    if (L->all) {
        BrickPlan b = brick_search(L, std::min<long>(g_samples, cap), cap, true);
        if (!b.by) b = brick_search(L, 1, cap, true);
        if (!b.by) return w;
        w.G = b.G;
        w.chunk = b.chunk;
        w.b = b;
        return w;
    }
    const long g_nodes = (N4 + kPcgMaxChunk - 1) / kPcgMaxChunk;
    const long gmin = std::max(g_nodes, std::min(g_samples, std::min<long>(cap, N4 / 4)));
    w.chunk = 4 * (int)(((N4 + gmin - 1) / gmin + 3) / 4);
    w.G = (int)((N4 + w.chunk - 1) / w.chunk);
    return w;
}

// One graph per batch whose position steps run in waves: per Gauss-Newton iteration one
// cooperative launch of k_pcg_wave (one CTA per SM) per launch set, in which every
// lattice's group runs the shared-memory persistent step of vd_solve.  A launch set holds
// up to kWaveMaxItems lattices of one kernel form: the all-nodes lattices (bricks; the
// padded form unless every one of them tiles exactly) and the surface-set lattices
// (contiguous ranges); its groups
// are packed into waves of at most one CTA per SM, largest first, each into the first
// wave with room (first fit decreasing).  The other stages run as per-lattice branches
// between these launches.
vd_status batch_build_waves(vd_batch *B, const vd_solve_params *P, int streams, bool largest) {
    const int n = (int)B->L.size();
    if (cudaStreamSynchronize(B->L[0]->stream) != cudaSuccess) return bfail(B, VD_ERR_CUDA, "synchronize");
    const int K = P->cg_iters, GN = P->gn_iters;
    const int T = B->L[0]->num_sms;
    if (!B->L[0]->coop) return bfail(B, VD_ERR_INVALID_ARG, "the wave form needs cooperative launches");
    // the lattices' plans; launch sets by kernel form: all nodes in the most general brick
    // form any of them needs -- 2 exact, 3 padded with 16-byte-aligned rows, 4 padded
    // rows (nx % 4 != 0) -- and 0 for the surface sets
    std::vector<PcgPlan> wp(n);
    int all_form = 2;
    for (int i = 0; i < n; i++) {
        vd_lattice *L = B->L[i];
        vd_status s = ensure_scal(L, GN, K);
        if (s != VD_OK) return bfail(B, s, L->err.c_str());
        set_params_ctx(L->c, P);
        refresh_ctx(L);
        wp[i] = wave_plan(L, T, B->wave_share);
        if (!wp[i].G || wp[i].G > T || wp[i].G > kPcgMaxCtas)
            return bfail(B, VD_ERR_INVALID_ARG, "a lattice of the batch is too large for the wave form");
        if (L->all && !wp[i].b.exact) all_form = std::max(all_form, L->c.nx % 4 ? 4 : 3);
    }
    struct Set {
        int form;
        std::vector<int> lat;
        int waves = 0, grid = 0, max_chunk = 4;
        size_t plan_off = 0;
    };
    std::vector<Set> sets;
    for (int form : {4, 3, 2, 0})
        for (int i = 0; i < n; i++) {
            const int f = B->L[i]->all ? all_form : 0;
            if (f != form) continue;
            if (sets.empty() || sets.back().form != form || (int)sets.back().lat.size() == kWaveMaxItems)
                sets.push_back(Set{form, {}});
            sets.back().lat.push_back(i);
        }
    // the kernel form of a set (kPad), and the padded vectors its lattices need
    auto set_kpad = [](int form) { return form == 4 ? 2 : form == 3 ? 1 : 0; };
    for (const Set &S : sets)
        for (int i : S.lat) {
            vd_status s = ensure_pad(B->L[i], wp[i], set_kpad(S.form));
            if (s != VD_OK) return bfail(B, s, B->L[i]->err.c_str());
        }
    // per set, first fit decreasing: the wave of each lattice's group and its first CTA
    std::vector<int2> plan;
    std::vector<int> place_wave(n), place_first(n), item_of(n);
    for (Set &S : sets) {
        std::vector<int> order = S.lat;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return wp[a].G > wp[b].G; });
        std::vector<int> fill;
        for (int i : order) {
            size_t w = 0;
            while (w < fill.size() && fill[w] + wp[i].G > T) w++;
            if (w == fill.size()) fill.push_back(0);
            place_wave[i] = (int)w;
            place_first[i] = fill[w];
            fill[w] += wp[i].G;
            S.grid = std::max(S.grid, fill[w]);
            S.max_chunk = std::max(S.max_chunk, wp[i].chunk);
        }
        S.waves = (int)fill.size();
        S.plan_off = plan.size();
        plan.resize(plan.size() + (size_t)S.waves * S.grid, make_int2(-1, 0));
        for (size_t k = 0; k < S.lat.size(); k++) {
            const int i = S.lat[k];
            item_of[i] = (int)k;
            for (int b = 0; b < wp[i].G; b++)
                plan[S.plan_off + (size_t)place_wave[i] * S.grid + place_first[i] + b] = make_int2((int)k, b);
        }
    }
    const long words_need = (long)n * (2 * K + 1);
    vd_status s = bgrow(B, &B->wplan, &B->cap_wplan, plan.size());
    if (s == VD_OK) s = bgrow(B, &B->words, &B->cap_words, (size_t)words_need);
    if (s != VD_OK) return s;
    if (cudaMemcpy(B->wplan, plan.data(), sizeof(int2) * plan.size(), cudaMemcpyHostToDevice) != cudaSuccess)
        return bfail(B, VD_ERR_CUDA, "plan upload");
    // the items of every (Gauss-Newton iteration, set): kernel parameters of its launch
    std::vector<PcgWaveArgs> args((size_t)GN * sets.size());
    for (int gi = 0; gi < GN; gi++)
        for (size_t si = 0; si < sets.size(); si++) {
            PcgWaveArgs &A = args[(size_t)gi * sets.size() + si];
            memset(&A, 0, sizeof(A));
            for (int i : sets[si].lat) {
                vd_lattice *L = B->L[i];
                PcgWaveItem &it = A.it[item_of[i]];
                it.c = L->c;
                it.ax = pcg_aux(L, L->pcg_part, B->words + (size_t)i * (2 * K + 1), 0, wp[i], set_kpad(sets[si].form));
                it.sc = slot(L, gi);
                it.G = wp[i].G;
            }
        }
    const int bytes = kPcgSmemPerSlot * kPcgMaxChunk;
    for (auto f : {k_pcg_wave<true, true, 2>, k_pcg_wave<true, true, 1>, k_pcg_wave<true, true, 0>,
                   k_pcg_wave<false, false, 0>}) {
        int occ = 0;
        if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, f, kPcgThreads, bytes) != cudaSuccess || occ < 1) {
            cudaGetLastError();
            return bfail(B, VD_ERR_INVALID_ARG, "the wave kernel does not fit on an SM");
        }
    }
    B->groups.assign(n, 0);
    B->n_waves = 0;
    for (int i = 0; i < n; i++) B->groups[i] = wp[i].G;
    for (const Set &S : sets) B->n_waves += S.waves;
    const double tol2 = P->cg_tol * P->cg_tol;
    return batch_capture(B, P, streams, largest, [&](int gi) {
        cudaMemsetAsync(B->words, 0, sizeof(unsigned long long) * (size_t)words_need, B->cap);
        for (size_t si = 0; si < sets.size(); si++) {
            const Set &S = sets[si];
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(S.grid);
            cfg.blockDim = dim3(kPcgThreads);
            cfg.dynamicSmemBytes = (size_t)kPcgSmemPerSlot * S.max_chunk;
            cfg.stream = B->cap;
            cudaLaunchAttribute at[1];
            at[0].id = cudaLaunchAttributeCooperative;
            at[0].val.cooperative = 1;
            cfg.attrs = at;
            cfg.numAttrs = 1;
            const PcgWaveArgs &A = args[(size_t)gi * sets.size() + si];
            const int2 *pl = B->wplan + S.plan_off;
            if (S.form == 4) cudaLaunchKernelEx(&cfg, k_pcg_wave<true, true, 2>, A, pl, S.waves, K, tol2, 1);
            else if (S.form == 3) cudaLaunchKernelEx(&cfg, k_pcg_wave<true, true, 1>, A, pl, S.waves, K, tol2, 1);
            else if (S.form == 2) cudaLaunchKernelEx(&cfg, k_pcg_wave<true, true, 0>, A, pl, S.waves, K, tol2, 1);
            else cudaLaunchKernelEx(&cfg, k_pcg_wave<false, false, 0>, A, pl, S.waves, K, tol2, 1);
        }
        return (int)sets.size();
    });
}

}  // namespace

extern "C" {

vd_status vd_batch_create(vd_lattice *const *ls, int count, vd_batch **out) {
    if (!ls || !out || count < 1) return VD_ERR_INVALID_ARG;
    *out = nullptr;
    for (int i = 0; i < count; i++)
        if (!ls[i]) return VD_ERR_INVALID_ARG;
    vd_batch *B = new (std::nothrow) vd_batch();
    if (!B) return VD_ERR_OOM;
    B->L.assign(ls, ls + count);
    if (cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreate(&B->t0) != cudaSuccess || cudaEventCreate(&B->t1) != cudaSuccess) {
        vd_batch_destroy(B);
        return VD_ERR_CUDA;
    }
    *out = B;
    return VD_OK;
}

vd_status vd_batch_destroy(vd_batch *B) {
    if (!B) return VD_OK;
    if (B->gexec) cudaGraphExecDestroy(B->gexec);
    for (auto st : B->side) cudaStreamDestroy(st);
    for (auto ev : B->join) cudaEventDestroy(ev);
    if (B->fork) cudaEventDestroy(B->fork);
    if (B->t0) cudaEventDestroy(B->t0);
    if (B->t1) cudaEventDestroy(B->t1);
    if (B->cap) cudaStreamDestroy(B->cap);
    for (void *p : B->pbufs) cudaFree(p);
    delete B;
    return VD_OK;
}

const char *vd_batch_last_error(const vd_batch *B) { return B ? B->err.c_str() : "null batch"; }

vd_status vd_batch_solve_async(vd_batch *B, const vd_solve_params *P) {
    if (!B) return VD_ERR_INVALID_ARG;
    for (vd_lattice *L : B->L) {
        vd_status s = check_params(L, P);
        if (s != VD_OK) return bfail(B, s, L->err.c_str());
        if (!L->have_frame) return bfail(B, VD_ERR_STATE, "a lattice of the batch has no frame");
    }
    const int streams = B->streams > 0 ? B->streams : std::min<int>((int)B->L.size(), 8);
    vd_status s = batch_build(B, P, streams, B->largest_first, B->coop_min);
    if (s != VD_OK) return s;
    cudaStream_t main = B->L[0]->stream;
    if (cudaGraphLaunch(B->gexec, main) != cudaSuccess) return bfail(B, VD_ERR_CUDA, "graph launch");
    B->pending = true;
    return VD_OK;
}

vd_status vd_batch_get_reports(vd_batch *B, vd_solve_report *out) {
    if (!B) return VD_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(B->L[0]->stream) != cudaSuccess) return bfail(B, VD_ERR_CUDA, "synchronize");
    B->pending = false;
    vd_status worst = VD_OK;
    for (size_t i = 0; i < B->L.size(); i++) {
        vd_status s = read_report(B->L[i], out ? out + i : nullptr);
        if (s != VD_OK && worst == VD_OK) worst = s;
    }
    return worst;
}

vd_status vd_batch_solve(vd_batch *B, const vd_solve_params *P, vd_solve_report *out) {
    vd_status s = vd_batch_solve_async(B, P);
    if (s != VD_OK) return s;
    return vd_batch_get_reports(B, out);
}

vd_status vd_batch_tune(vd_batch *B, const vd_solve_params *P, int *streams_out, float *ms_out) {
    if (!B) return VD_ERR_INVALID_ARG;
    const int n = (int)B->L.size();
    const int cand[] = {1, 2, 4, 8, 16, 32, 64};
    float best = 3.4e38f;
    int best_s = 1;
    bool best_l = true;
    cudaStream_t main = B->L[0]->stream;
    // build one candidate and time two replays (after one that warms the caches)
    auto time_build = [&](int st, bool lf, long cm, float *out) -> vd_status {
        vd_status s = batch_build(B, P, st, lf, cm);
        if (s != VD_OK) return s;
        float ms = 0.f;
        for (int rep = 0; rep < 3; rep++) {
            cudaEventRecord(B->t0, main);
            if (cudaGraphLaunch(B->gexec, main) != cudaSuccess) return bfail(B, VD_ERR_CUDA, "graph launch");
            cudaEventRecord(B->t1, main);
            if (cudaEventSynchronize(B->t1) != cudaSuccess) return bfail(B, VD_ERR_CUDA, "synchronize");
            float m = 0.f;
            cudaEventElapsedTime(&m, B->t0, B->t1);
            if (rep > 0) ms += m;
        }
        *out = ms;
        return VD_OK;
    };
    for (int lf = 1; lf >= 0; lf--)
        for (int ci = 0; ci < 7; ci++) {
            const int st = cand[ci];
            if (st > n && st != cand[0]) break;
            float ms = 0.f;
            vd_status s = time_build(st, lf != 0, 0x7fffffffL, &ms);
            if (s != VD_OK) return s;
            if (ms < best) {
                best = ms;
                best_s = st;
                best_l = lf != 0;
            }
        }
    // then which lattices run their persistent position step ahead of the branches
    long best_c = 0x7fffffffL;
    for (long cm : {1L << 19, 1L << 17, 1L << 15, 1L << 13}) {
        bool any = false;
        for (vd_lattice *L : B->L) any = any || active_nodes(L) >= cm;
        if (!any) continue;
        float ms = 0.f;
        vd_status s = time_build(best_s, best_l, cm, &ms);
        if (s != VD_OK) return s;
        if (ms < best) {
            best = ms;
            best_c = cm;
        }
    }
    // then the waves of the shared-memory position step, with the branches of the other
    // stages
    bool best_p = false, best_v = false;
    int best_t = B->pthreads, best_k = B->pctas;
    float best_w = B->sample_weight;
    int best_share = B->wave_share;
    if (B->L[0]->coop) {
        bool fits = true;
        for (int share : {1 << 20, 4096, 1024})
            for (int st : {8, 16}) {
                if (!fits || (st > n && st != 8)) continue;
                B->waves = true;
                B->persistent = false;
                B->wave_share = share;
                float ms = 0.f;
                vd_status s = time_build(st, best_l, 0x7fffffffL, &ms);
                B->waves = false;
                if (s != VD_OK) {  // a lattice too large for the waves
                    B->err.clear();
                    fits = false;
                    continue;
                }
                if (ms < best) {
                    best = ms;
                    best_v = true;
                    best_s = st;
                    best_share = share;
                    best_c = 0x7fffffffL;
                }
            }
    }
    B->wave_share = best_share;
    // then the persistent position step over every lattice with its vectors in global
    // memory: threads per CTA, CTAs per SM, the sample weight of the CTA split, and the
    // branches of the other stages
    if (B->L[0]->coop) {
        for (int th : {256, 512}) {
            const int occ = batch_occupancy(th);
            for (int k : {1, 2, 4}) {
                if (k > occ || n > B->L[0]->num_sms * k) continue;
                for (float sw : {1.f, 4.f})
                    for (int st : {8, 16}) {
                        if (st > n && st != 8) continue;
                        B->persistent = true;
                        B->pthreads = th;
                        B->pctas = k;
                        B->sample_weight = sw;
                        float ms = 0.f;
                        vd_status s = time_build(st, best_l, 0x7fffffffL, &ms);
                        if (s != VD_OK) {
                            B->err.clear();
                            continue;
                        }
                        if (ms < best) {
                            best = ms;
                            best_p = true;
                            best_v = false;
                            best_t = th;
                            best_k = k;
                            best_w = sw;
                            best_s = st;
                            best_c = 0x7fffffffL;
                        }
                    }
            }
        }
    }
    B->persistent = best_p;
    B->waves = best_v;
    B->pthreads = best_t;
    B->pctas = best_k;
    B->sample_weight = best_w;
    B->streams = best_s;
    B->largest_first = best_l;
    B->coop_min = best_c;
    if (streams_out) *streams_out = best_s;
    if (ms_out) *ms_out = best / 2.f;
    return VD_OK;
}

vd_status vd_batch_set_plan(vd_batch *B, int streams, int largest_first, long long run_ahead_nodes) {
    if (!B || streams < 1 || streams > 64 || run_ahead_nodes < 0) return VD_ERR_INVALID_ARG;
    B->streams = streams;
    B->largest_first = largest_first != 0;
    B->coop_min = run_ahead_nodes > 0x7fffffffLL ? 0x7fffffffL : (long)run_ahead_nodes;
    return VD_OK;
}

vd_status vd_batch_set_persistent(vd_batch *B, int on, int threads, int ctas_per_sm, float sample_weight) {
    if (!B || !batch_threads_ok(threads) || ctas_per_sm < 1 || ctas_per_sm > 8 || !(sample_weight >= 0.f))
        return VD_ERR_INVALID_ARG;
    if (on < 0 || on > VD_BATCH_WAVES) return VD_ERR_INVALID_ARG;
    B->persistent = on == VD_BATCH_GLOBAL;
    B->waves = on == VD_BATCH_WAVES;
    B->pthreads = threads;
    B->pctas = ctas_per_sm;
    B->sample_weight = sample_weight;
    return VD_OK;
}

vd_status vd_batch_set_wave_share(vd_batch *B, int samples_per_cta) {
    if (!B || samples_per_cta < 32) return VD_ERR_INVALID_ARG;
    B->wave_share = samples_per_cta;
    return VD_OK;
}

vd_status vd_batch_get_plan(const vd_batch *B, int *persistent, int *threads, int *ctas_per_sm, float *sample_weight,
                            int *streams) {
    if (!B) return VD_ERR_INVALID_ARG;
    if (persistent) *persistent = B->waves ? VD_BATCH_WAVES : B->persistent ? VD_BATCH_GLOBAL : VD_BATCH_BRANCHES;
    if (threads) *threads = B->pthreads;
    if (ctas_per_sm) *ctas_per_sm = B->pctas;
    if (sample_weight) *sample_weight = B->sample_weight;
    if (streams) *streams = B->streams > 0 ? B->streams : std::min<int>((int)B->L.size(), 8);
    return VD_OK;
}

vd_status vd_batch_launch_count(const vd_batch *B, int *launches) {
    if (!B || !launches) return VD_ERR_INVALID_ARG;
    *launches = B->launches;
    return VD_OK;
}

vd_status vd_batch_get_groups(const vd_batch *B, int *ctas, int *waves) {
    if (!B) return VD_ERR_INVALID_ARG;
    if (ctas)
        for (size_t i = 0; i < B->L.size(); i++) ctas[i] = i < B->groups.size() ? B->groups[i] : 0;
    if (waves) *waves = B->n_waves;
    return VD_OK;
}

vd_status vd_solve_batch(vd_lattice *const *ls, int count, const vd_solve_params *P, vd_solve_report *out) {
    vd_batch *B = nullptr;
    vd_status s = vd_batch_create(ls, count, &B);
    if (s != VD_OK) return s;
    s = vd_batch_solve(B, P, out);
    vd_batch_destroy(B);
    return s;
}

}  // extern "C"

// ====================================================================== allocation-free rotation step
//
// vd_fit_rotations_noalloc runs the rotation step on caller-owned device arrays without
// allocating anything.  Its scratch -- the structure-of-arrays copies of u and R that the
// kernel reads, and the block of FP64 sums and counters -- is one file-scope device array
// of fixed size, present on every device that loads this library for the life of the
// process.  Host code must not use the array's name as an address: the address is
// obtained once per device with cudaGetSymbolAddress and passed to the kernels.

namespace {

constexpr int kNoAllocLd = VD_NOALLOC_MAX_NODES;                   // plane stride of the SoA copies
constexpr size_t kNoAllocStateBytes = sizeof(float) * 12 * (size_t)kNoAllocLd;  // u (3) + R (9) planes
constexpr size_t kNoAllocBytes = kNoAllocStateBytes + 256;          // + one scalar block (K = 1)
static_assert(kNoAllocLd % 32 == 0, "plane stride must keep 128-byte alignment");
constexpr int kNoAllocMaxDevices = 64;

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

namespace {

void *g_noalloc_addr[kNoAllocMaxDevices] = {nullptr};
std::mutex g_noalloc_mutex;

// Device address of the scratch array on the current device (looked up once per device).
cudaError_t noalloc_scratch(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" vd_status vd_fit_rotations_noalloc(int nx, int ny, int nz, float spacing, const float *disp,
                                              const float *rot_in, float *rot_out, double *e_reg,
                                              int *n_degenerate, void *cuda_stream) {
    if (nx < 2 || ny < 2 || nz < 2 || !(spacing > 0.f) || !disp || !rot_in || !rot_out) return VD_ERR_INVALID_ARG;
    // each factor is bounded before the product is formed, so the product cannot overflow
    if (nx > VD_NOALLOC_MAX_NODES || ny > VD_NOALLOC_MAX_NODES || nz > VD_NOALLOC_MAX_NODES) return VD_ERR_INVALID_ARG;
    const long long nn = (long long)nx * ny * nz;
    if (nn > VD_NOALLOC_MAX_NODES) return VD_ERR_INVALID_ARG;
    // an error left pending by the caller's earlier work is not ours to consume: refuse
    // before enqueueing anything and leave it for the caller to read
    if (cudaPeekAtLastError() != cudaSuccess) return VD_ERR_CUDA;
    void *base = nullptr;
    if (noalloc_scratch(&base) != cudaSuccess) {
        cudaGetLastError();
        return VD_ERR_CUDA;
    }
    cudaStream_t st = (cudaStream_t)cuda_stream;
    Ctx c{};
    c.nx = nx;
    c.ny = ny;
    c.nz = nz;
    c.nn = (int)nn;
    c.ld = kNoAllocLd;
    c.h = spacing;
    c.u = (float *)base;
    c.R = c.u + 3 * (size_t)kNoAllocLd;
    Scal *sc = (Scal *)((char *)base + kNoAllocStateBytes);
    // the sums and counters accumulate with atomics: clear what the last call left
    if (cudaMemsetAsync(sc, 0, scal_bytes(1), st) != cudaSuccess) return VD_ERR_CUDA;
    // no error was pending on entry, so each check below sees only this call's launch
    const int nb = blocks_for(nn);
    k_aos_to_soa<<<nb, kThreads, 0, st>>>(disp, 3, c.nn, c.ld, c.u);
    if (cudaGetLastError() != cudaSuccess) return VD_ERR_CUDA;
    k_aos_to_soa<<<nb, kThreads, 0, st>>>(rot_in, 9, c.nn, c.ld, c.R);
    if (cudaGetLastError() != cudaSuccess) return VD_ERR_CUDA;
    k_fit_rotations<true, true><<<nb, kThreads, 0, st>>>(c, sc);
    if (cudaGetLastError() != cudaSuccess) return VD_ERR_CUDA;
    k_soa_to_aos<<<nb, kThreads, 0, st>>>(c.R, 9, c.nn, c.ld, rot_out);
    if (cudaGetLastError() != cudaSuccess) return VD_ERR_CUDA;
    if (e_reg && cudaMemcpyAsync(e_reg, &sc->e_reg, sizeof(double), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return VD_ERR_CUDA;
    if (n_degenerate &&
        cudaMemcpyAsync(n_degenerate, &sc->n_degenerate, sizeof(int), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return VD_ERR_CUDA;
    return VD_OK;
}

// ------------------------------------------------------------------ early stop and learned warm start

namespace {

vd_status warm_prepare(vd_lattice *L, const vd_solve_params *P) {
    TRY(check_params(L, P));
    if (!L->have_frame) return fail(L, VD_ERR_STATE, "no frame");
    // two scalar slots, keeping the solve's slot layout when it already has them
    if (!L->scal || L->scal_slots < 2) TRY(ensure_scal(L, std::max(2, P->gn_iters), std::max(1, P->cg_iters)));
    if (!L->warm) TRY(dalloc(L, &L->warm, 9 * (size_t)L->c.nn + 12 * (size_t)L->c.ld));
    set_params_ctx(L->c, P);
    refresh_ctx(L);
    return VD_OK;
}

// E_total at the current warp (slot 0), then the data-term right-hand side (w_r = 0)
// and the features
template <bool kAll>
void warm_features_enqueue(vd_lattice *L, float *in6) {
    cudaStream_t st = L->stream;
    const Grid gr = grids(L);
    const Ctx c = L->c;
    Scal *s0 = slot(L, 0);
    cudaMemsetAsync(L->scal, 0, 2 * L->scal_stride, st);
    k_associate<kAll><<<gr.assoc, kThreads, 0, st>>>(c, s0);
    k_associate_refine<kAll><<<gr.refine, kThreads, 0, st>>>(c, s0);
    launch_fit_rotations<kAll, false>(c, s0, gr, st);
    k_cells<kOpEnergy, kAll><<<gr.cells, kThreads, 0, st>>>(c, s0, 1, 0);
    Ctx cd = c;
    cd.w_r = 0.f;
    k_rhs_nodes<kAll><<<gr.node, kThreads, 0, st>>>(cd, s0);
    k_cells<kOpRhs, kAll><<<gr.cells, kThreads, 0, st>>>(cd, s0, 1, 0);
    if (!kAll) cudaMemsetAsync(in6, 0, sizeof(float) * 6 * (size_t)c.nn, st);
    k_warm_features<kAll><<<gr.node, kThreads, 0, st>>>(c, c.w_r, in6);
}

// candidate u + h pred, rotations refitted (slot 1 gets its E_reg), association and
// energy at the candidate, then keep or restore
template <bool kAll>
void warm_select_enqueue(vd_lattice *L, const float *pred) {
    cudaStream_t st = L->stream;
    const Grid gr = grids(L);
    const Ctx c = L->c;
    Scal *s0 = slot(L, 0), *s1 = slot(L, 1);
    float *bak = L->warm + 9 * (size_t)c.nn;
    k_warm_apply<kAll><<<gr.node, kThreads, 0, st>>>(c, pred, bak);
    launch_fit_rotations<kAll, true>(c, s1, gr, st);
    k_associate<kAll><<<gr.assoc, kThreads, 0, st>>>(c, s1);
    k_associate_refine<kAll><<<gr.refine, kThreads, 0, st>>>(c, s1);
    k_cells<kOpEnergy, kAll><<<gr.cells, kThreads, 0, st>>>(c, s1, 1, 0);
    k_warm_select<kAll><<<gr.node, kThreads, 0, st>>>(c, s0, s1, bak, L->rep_dev + 11);
}

}  // namespace

extern "C" {

vd_status vd_test_stall_barrier(vd_lattice *L, int on) {
    if (!L) return VD_ERR_INVALID_ARG;
    L->stall_extra = on ? 1 : 0;
    L->ggen = -1;  // the flag is a launch argument of the captured graph: re-capture
    return VD_OK;
}

vd_status vd_test_grid_reduce(const double *parts, int G, int rounds, double *out) {
    if (!parts || !out || G < 1 || G > 148 || rounds < 1 || rounds > 4096) return VD_ERR_INVALID_ARG;
    int dev = 0, coop = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) || !coop || G > sms) {
        cudaGetLastError();
        return VD_ERR_INVALID_ARG;
    }
    const size_t np = (size_t)rounds * G;
    double *d_parts = nullptr, *d_rows = nullptr, *d_out = nullptr;
    unsigned long long *d_words = nullptr;
    int *d_err = nullptr;
    vd_status st = VD_OK;
    if (cudaMalloc(&d_parts, np * sizeof(double)) || cudaMalloc(&d_rows, np * sizeof(double)) ||
        cudaMalloc(&d_out, 2 * (size_t)rounds * sizeof(double)) ||
        cudaMalloc(&d_words, (size_t)rounds * sizeof(unsigned long long)) || cudaMalloc(&d_err, sizeof(int))) {
        st = VD_ERR_OOM;
    } else if (cudaMemcpy(d_parts, parts, np * sizeof(double), cudaMemcpyHostToDevice) ||
               cudaMemset(d_words, 0, (size_t)rounds * sizeof(unsigned long long)) ||
               cudaMemset(d_err, 0, sizeof(int)) || cudaMemset(d_out, 0, 2 * (size_t)rounds * sizeof(double))) {
        st = VD_ERR_CUDA;
    } else {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(G);
        cfg.blockDim = dim3(64);
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeCooperative;
        at[0].val.cooperative = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        int herr = 0;
        if (cudaLaunchKernelEx(&cfg, k_test_grid_reduce, (const double *)d_parts, rounds, d_rows, d_words, d_err,
                               d_out) != cudaSuccess ||
            cudaDeviceSynchronize() != cudaSuccess ||
            cudaMemcpy(out, d_out, 2 * (size_t)rounds * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
            st = VD_ERR_CUDA;
        else if (herr)
            st = VD_ERR_TIMEOUT;
    }
    cudaGetLastError();
    cudaFree(d_parts);
    cudaFree(d_rows);
    cudaFree(d_out);
    cudaFree(d_words);
    cudaFree(d_err);
    return st;
}

vd_status vd_set_energy_target(vd_lattice *L, double e_target) {
    if (!L) return VD_ERR_INVALID_ARG;
    if (!(e_target >= 0.0)) {
        L->gated = false;
        return VD_OK;
    }
    // by value through a kernel argument: ordered on the stream, no host buffer to keep
    k_store_f64<<<1, 1, 0, L->stream>>>(L->rep_dev + 15, e_target);
    CKL();
    L->gated = true;
    return VD_OK;
}

vd_status vd_warm_features(vd_lattice *L, const vd_solve_params *P, float *in6, int mem) {
    if (!L) return VD_ERR_INVALID_ARG;
    if (!in6) return fail(L, VD_ERR_INVALID_ARG, "in6 is NULL");
    TRY(warm_prepare(L, P));
    if (L->all) warm_features_enqueue<true>(L, L->warm);
    else warm_features_enqueue<false>(L, L->warm);
    CKL();
    TRY(download(L, in6, L->warm, sizeof(float) * 6 * (size_t)L->c.nn, mem));
    CK(cudaStreamSynchronize(L->stream));
    return VD_OK;
}

vd_status vd_warm_start(vd_lattice *L, vd_unet *net, const vd_solve_params *P, vd_warm_report *out) {
    if (!L) return VD_ERR_INVALID_ARG;
    if (!net) return fail(L, VD_ERR_INVALID_ARG, "net is NULL");
    int nx = 0, ny = 0, nz = 0;
    TRY(vd_unet_dims(net, &nx, &ny, &nz));
    if (nx != L->c.nx || ny != L->c.ny || nz != L->c.nz)
        return fail(L, VD_ERR_INVALID_ARG, "network grid %dx%dx%d != lattice %dx%dx%d", nx, ny, nz, L->c.nx, L->c.ny,
                    L->c.nz);
    TRY(warm_prepare(L, P));
    float *in6 = L->warm, *pred = L->warm + 6 * (size_t)L->c.nn;
    if (L->all) warm_features_enqueue<true>(L, in6);
    else warm_features_enqueue<false>(L, in6);
    CKL();
    if (vd_unet_forward_async(net, in6, pred, L->stream) != VD_OK) return fail(L, VD_ERR_CUDA, "network launch failed");
    if (L->all) warm_select_enqueue<true>(L, pred);
    else warm_select_enqueue<false>(L, pred);
    CKL();
    CK(cudaMemcpyAsync(L->rep_host + 11, L->rep_dev + 11, 3 * sizeof(double), cudaMemcpyDeviceToHost, L->stream));
    if (out) return vd_get_warm_report(L, out);
    return VD_OK;
}

vd_status vd_get_warm_report(vd_lattice *L, vd_warm_report *out) {
    if (!L || !out) return VD_ERR_INVALID_ARG;
    CK(cudaStreamSynchronize(L->stream));
    out->e_start = L->rep_host[11];
    out->e_predicted = L->rep_host[12];
    out->used_prediction = L->rep_host[13] != 0.0;
    out->status = VD_OK;
    return VD_OK;
}

}  // extern "C"

// ====================================================================== hierarchy (Sec. 7.2)
//
// A hierarchy owns levels - 1 coarse lattices nested on a caller's lattice (level 0):
// level l has (n_{l-1} // 2 + 1) nodes per axis at spacing 2^l h, the same origin, and
// the same active-set mode, precision and stream.  Their frames are copied from level
// 0's own device buffers whenever level 0 got a new frame or new pairs; their binning
// keeps only the constraints whose cell exists on level 0 (the constraints of each
// parent voxel gathered from its children, expressed trilinearly in the coarse nodes).
// A solve enqueues, on level 0's stream: restriction of the state to every coarse level,
// then from the coarsest up its captured flip-flop graph, the prolongation of its
// increment to the next finer level and a rotation step there; then level 0's graph.

struct vd_hierarchy {
    std::vector<vd_lattice *> L;     // L[0] is the caller's; the others are owned
    std::vector<float *> u_start;    // per coarse level, 3 planes of its ld
    Scal *scal = nullptr;            // sums of the rotation steps after prolongation
    long synced_gen = -1;
    bool pending = false;
    std::string err;
};

namespace {

vd_status hfail(vd_hierarchy *H, vd_status s, const std::string &msg) {
    H->err = msg;
    return s;
}

// copy level 0's current frame and pairs into every coarse level
vd_status hierarchy_sync(vd_hierarchy *H) {
    vd_lattice *F = H->L[0];
    if (H->synced_gen == F->frame_gen) return VD_OK;
    const Ctx &c = F->c;
    const float K[4] = {c.fx, c.fy, c.cx, c.cy};
    float pose[12];
    for (int a = 0; a < 9; a++) pose[a] = c.Rg[a];
    for (int a = 0; a < 3; a++) pose[9 + a] = c.tg[a];
    for (size_t l = 1; l < H->L.size(); l++) {
        vd_lattice *Lc = H->L[l];
        vd_status s = vd_set_correspondences(Lc, F->sp_in, F->sp_in + 3 * (size_t)F->S, F->S, VD_MEM_DEVICE);
        if (s == VD_OK)
            s = vd_set_frame(Lc, F->depth, F->W, F->H, K, pose, F->pts_in, F->nrm_in, F->n_src, VD_MEM_DEVICE);
        if (s != VD_OK) return hfail(H, s, "level " + std::to_string(l) + ": " + Lc->err);
    }
    H->synced_gen = F->frame_gen;
    return VD_OK;
}

}  // namespace

extern "C" {

vd_status vd_hierarchy_create(vd_lattice *fine, int levels, vd_hierarchy **out) {
    if (!fine || !out || levels < 1 || levels > 8) return VD_ERR_INVALID_ARG;
    *out = nullptr;
    vd_hierarchy *H = new (std::nothrow) vd_hierarchy();
    if (!H) return VD_ERR_OOM;
    H->L.push_back(fine);
    H->u_start.push_back(nullptr);
    const Ctx &f = fine->c;
    int dims[3] = {f.nx, f.ny, f.nz};
    float h = f.h;
    for (int l = 1; l < levels; l++) {
        for (int a = 0; a < 3; a++) dims[a] = dims[a] / 2 + 1;
        h *= 2.f;
        vd_lattice_desc d{};
        d.nx = dims[0];
        d.ny = dims[1];
        d.nz = dims[2];
        d.origin[0] = f.ox;
        d.origin[1] = f.oy;
        d.origin[2] = f.oz;
        d.spacing = h;
        d.active_mode = fine->all ? VD_ACTIVE_ALL : VD_ACTIVE_SURFACE;
        d.precision = fine->precision;
        d.cuda_stream = fine->stream;
        vd_lattice *Lc = nullptr;
        vd_status s = vd_create_lattice(&d, &Lc);
        if (s != VD_OK) {
            vd_hierarchy_destroy(H);
            return s;
        }
        Lc->apply_mode = VD_APPLY_AUTO;  // many samples per coarse cell: the cached blocks pay
        Lc->c.dom_n[0] = f.nx;
        Lc->c.dom_n[1] = f.ny;
        Lc->c.dom_n[2] = f.nz;
        Lc->c.dom_h = f.h;
        H->L.push_back(Lc);
        float *us = nullptr;
        if (cudaMalloc(&us, sizeof(float) * 3 * (size_t)Lc->c.ld) != cudaSuccess) {
            cudaGetLastError();
            H->u_start.push_back(nullptr);
            vd_hierarchy_destroy(H);
            return VD_ERR_OOM;
        }
        H->u_start.push_back(us);
    }
    if (cudaMalloc(&H->scal, scal_bytes(1)) != cudaSuccess) {
        cudaGetLastError();
        H->scal = nullptr;
        vd_hierarchy_destroy(H);
        return VD_ERR_OOM;
    }
    *out = H;
    return VD_OK;
}

vd_status vd_hierarchy_destroy(vd_hierarchy *H) {
    if (!H) return VD_OK;
    if (!H->L.empty() && H->L[0]->stream) cudaStreamSynchronize(H->L[0]->stream);
    for (size_t l = 1; l < H->L.size(); l++) vd_destroy_lattice(H->L[l]);
    for (float *p : H->u_start)
        if (p) cudaFree(p);
    if (H->scal) cudaFree(H->scal);
    delete H;
    return VD_OK;
}

vd_status vd_hierarchy_level(vd_hierarchy *H, int level, vd_lattice **out) {
    if (!H || !out || level < 0 || level >= (int)H->L.size()) return VD_ERR_INVALID_ARG;
    *out = H->L[level];
    return VD_OK;
}

const char *vd_hierarchy_last_error(const vd_hierarchy *H) { return H ? H->err.c_str() : "null hierarchy"; }

vd_status vd_hierarchy_solve_async(vd_hierarchy *H, const vd_solve_params *params) {
    if (!H || !params) return VD_ERR_INVALID_ARG;
    const int levels = (int)H->L.size();
    vd_lattice *F = H->L[0];
    for (int l = 0; l < levels; l++) {
        vd_status s = check_params(F, &params[l]);
        if (s != VD_OK) return hfail(H, s, "level schedule " + std::to_string(l) + ": " + F->err);
    }
    if (!F->have_frame) return hfail(H, VD_ERR_STATE, "the finest lattice has no frame");
    vd_status s = hierarchy_sync(H);
    if (s != VD_OK) return s;
    cudaStream_t st = F->stream;
    if (params[levels - 1].init == VD_INIT_ZERO)
        k_reset_warp<<<blocks_for(F->c.nn), kThreads, 0, st>>>(F->u, F->R, F->c.nn, F->c.ld);
    for (int l = 1; l < levels; l++) {
        refresh_ctx(H->L[l]);
        k_restrict_state<<<blocks_for(H->L[l]->c.nn), kThreads, 0, st>>>(H->L[l - 1]->c, H->L[l]->c, H->u_start[l]);
    }
    if (cudaGetLastError() != cudaSuccess) return hfail(H, VD_ERR_CUDA, "restriction launch failed");
    for (int l = levels - 1; l >= 0; l--) {
        vd_lattice *Ll = H->L[l];
        vd_solve_params P = params[levels - 1 - l];
        P.init = VD_INIT_PREV;
        s = vd_solve_async(Ll, &P);
        if (s != VD_OK) return hfail(H, s, "level " + std::to_string(l) + ": " + Ll->err);
        if (l == 0) break;
        vd_lattice *Lf = H->L[l - 1];
        refresh_ctx(Lf);
        k_prolongate<<<blocks_for(Lf->c.nn), kThreads, 0, st>>>(Ll->c, H->u_start[l], Lf->c);
        cudaMemsetAsync(H->scal, 0, scal_bytes(1), st);
        const Grid gr = grids(Lf);
        if (Lf->all) launch_fit_rotations<true, true>(Lf->c, H->scal, gr, st);
        else launch_fit_rotations<false, true>(Lf->c, H->scal, gr, st);
        if (cudaGetLastError() != cudaSuccess) return hfail(H, VD_ERR_CUDA, "prolongation launch failed");
    }
    H->pending = true;
    return VD_OK;
}

vd_status vd_hierarchy_get_reports(vd_hierarchy *H, vd_solve_report *out) {
    if (!H) return VD_ERR_INVALID_ARG;
    const int levels = (int)H->L.size();
    vd_status worst = VD_OK;
    for (int l = levels - 1; l >= 0; l--) {  // out[] coarsest first, like the schedule
        vd_status s = vd_get_report(H->L[l], out ? out + (levels - 1 - l) : nullptr);
        if (s != VD_OK && worst == VD_OK) worst = hfail(H, s, H->L[l]->err);
    }
    H->pending = false;
    return worst;
}

vd_status vd_hierarchy_solve(vd_hierarchy *H, const vd_solve_params *params, vd_solve_report *out) {
    vd_status s = vd_hierarchy_solve_async(H, params);
    if (s != VD_OK) return s;
    return vd_hierarchy_get_reports(H, out);
}

}  // extern "C"

// ====================================================================== source samples (Sec. 4, 5.1)

struct vd_renderer {
    int max_tri = 0, W = 0, H = 0;
    float *tri = nullptr, *nrm = nullptr, *posed = nullptr, *pose_dev = nullptr;
    int *table = nullptr;
    float *grid = nullptr;           // device copy of a host SDF grid
    size_t cap_grid = 0;
    int *cnt = nullptr, *off = nullptr, *sums = nullptr, *total = nullptr;
    long cap_cells = 0;
    unsigned long long *zbuf = nullptr;
    int *flag = nullptr, *poff = nullptr;
    float *stage = nullptr;          // W H x 7: points, normals, pixel index (host outputs)
    int n_tri = 0;
    cudaStream_t st = nullptr;
    std::vector<void *> bufs;
    std::string err;
};

namespace {

template <typename T>
bool ralloc(vd_renderer *R, T **p, size_t count) {
    void *q = nullptr;
    if (cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    R->bufs.push_back(q);
    *p = (T *)q;
    return true;
}

void rfree(vd_renderer *R, void *p) {
    if (!p) return;
    for (size_t k = 0; k < R->bufs.size(); k++)
        if (R->bufs[k] == p) {
            cudaFree(p);
            R->bufs.erase(R->bufs.begin() + k);
            return;
        }
}

vd_status rfail(vd_renderer *R, vd_status s, const char *msg) {
    R->err = msg;
    return s;
}

}  // namespace

extern "C" {

vd_status vd_renderer_create(int max_triangles, int W, int H, vd_renderer **out) {
    if (!out || max_triangles < 1 || W < 1 || H < 1 || (long)W * H > (long)kScanTile * kScanTile ||
        (long)max_triangles * 9 > 0x7fffffffL)
        return VD_ERR_INVALID_ARG;
    *out = nullptr;
    vd_renderer *R = new (std::nothrow) vd_renderer();
    if (!R) return VD_ERR_OOM;
    R->max_tri = max_triangles;
    R->W = W;
    R->H = H;
    const size_t np = (size_t)W * H;
    const bool ok = ralloc(R, &R->tri, 9 * (size_t)max_triangles) && ralloc(R, &R->nrm, 9 * (size_t)max_triangles) &&
                    ralloc(R, &R->posed, 9 * (size_t)max_triangles) && ralloc(R, &R->pose_dev, 12) &&
                    ralloc(R, &R->table, 256 * kMcRow) && ralloc(R, &R->sums, kScanTile) && ralloc(R, &R->total, 2) &&
                    ralloc(R, &R->zbuf, np) && ralloc(R, &R->flag, np) && ralloc(R, &R->poff, np + 1) &&
                    ralloc(R, &R->stage, 7 * np);
    if (!ok || cudaStreamCreateWithFlags(&R->st, cudaStreamNonBlocking) != cudaSuccess) {
        vd_renderer_destroy(R);
        return VD_ERR_OOM;
    }
    const McTable T = mc_make_table();
    if (cudaMemcpy(R->table, T.t, sizeof(T.t), cudaMemcpyHostToDevice) != cudaSuccess) {
        vd_renderer_destroy(R);
        return VD_ERR_CUDA;
    }
    *out = R;
    return VD_OK;
}

int vd_mc_case(int cs, int *edges) {
    if (cs < 0 || cs > 255) return -1;
    static const McTable T = mc_make_table();
    const int n = T.t[cs][0];
    if (edges)
        for (int i = 0; i < 3 * n; i++) edges[i] = T.t[cs][1 + i];
    return n;
}

vd_status vd_renderer_destroy(vd_renderer *R) {
    if (!R) return VD_OK;
    if (R->st) cudaStreamSynchronize(R->st);
    for (void *p : R->bufs) cudaFree(p);
    if (R->st) cudaStreamDestroy(R->st);
    delete R;
    return VD_OK;
}

const char *vd_renderer_last_error(const vd_renderer *R) { return R ? R->err.c_str() : "null renderer"; }

vd_status vd_marching_cubes(vd_renderer *R, const float *sdf, int sx, int sy, int sz, const float origin[3],
                            float spacing, float iso, int mem, int *n_triangles) {
    if (!R) return VD_ERR_INVALID_ARG;
    if (!sdf || !origin || sx < 2 || sy < 2 || sz < 2 || !(spacing > 0.f))
        return rfail(R, VD_ERR_INVALID_ARG, "bad grid");
    const long ncell = (long)(sx - 1) * (sy - 1) * (sz - 1);
    if ((long)sx * sy * sz > (long)kScanTile * kScanTile) return rfail(R, VD_ERR_INVALID_ARG, "grid too large");
    cudaStream_t st = R->st;
    const float *g = sdf;
    if (mem != VD_MEM_DEVICE) {
        const size_t n = (size_t)sx * sy * sz;
        if (n > R->cap_grid) {
            rfree(R, R->grid);
            R->grid = nullptr;
            R->cap_grid = 0;
            if (!ralloc(R, &R->grid, n)) return rfail(R, VD_ERR_OOM, "grid allocation failed");
            R->cap_grid = n;
        }
        if (cudaMemcpyAsync(R->grid, sdf, n * sizeof(float), cudaMemcpyHostToDevice, st) != cudaSuccess)
            return rfail(R, VD_ERR_CUDA, "grid upload failed");
        g = R->grid;
    }
    if (ncell > R->cap_cells) {
        rfree(R, R->cnt);
        rfree(R, R->off);
        R->cnt = R->off = nullptr;
        R->cap_cells = 0;
        if (!ralloc(R, &R->cnt, (size_t)ncell) || !ralloc(R, &R->off, (size_t)ncell + 1))
            return rfail(R, VD_ERR_OOM, "cell buffers");
        R->cap_cells = ncell;
    }
    const Grid3 G{g, sx, sy, sz, origin[0], origin[1], origin[2], spacing, iso};
    const int nb = blocks_for(ncell);
    k_mc_count<<<nb, kThreads, 0, st>>>(G, R->table, R->cnt);
    scan_launch(R->cnt, (int)ncell, R->off, R->total, R->sums, st);
    k_mc_emit<<<nb, kThreads, 0, st>>>(G, R->table, R->off, R->max_tri, R->tri, R->nrm);
    int total = 0;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&total, R->total, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return rfail(R, VD_ERR_CUDA, "marching cubes launch failed");
    if (n_triangles) *n_triangles = total;
    R->n_tri = std::min(total, R->max_tri);
    if (total > R->max_tri) return rfail(R, VD_ERR_INVALID_ARG, "more triangles than max_triangles");
    return VD_OK;
}

vd_status vd_get_mesh(vd_renderer *R, float *tri, float *nrm, int mem) {
    if (!R) return VD_ERR_INVALID_ARG;
    const cudaMemcpyKind kind = mem == VD_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const size_t bytes = sizeof(float) * 9 * (size_t)R->n_tri;
    if ((tri && cudaMemcpyAsync(tri, R->tri, bytes, kind, R->st) != cudaSuccess) ||
        (nrm && cudaMemcpyAsync(nrm, R->nrm, bytes, kind, R->st) != cudaSuccess) ||
        cudaStreamSynchronize(R->st) != cudaSuccess)
        return rfail(R, VD_ERR_CUDA, "mesh download failed");
    return VD_OK;
}

vd_status vd_render_samples(vd_renderer *R, const vd_lattice *lat, const float K[4], const float pose[12],
                            int stride, float *pts, float *nrm, int *pix, int cap, int *count, int mem) {
    if (!R) return VD_ERR_INVALID_ARG;
    if (!K || stride < 1 || cap < 0 || (cap > 0 && (!pts || !nrm)) || !(K[0] > 0.f) || !(K[1] > 0.f))
        return rfail(R, VD_ERR_INVALID_ARG, "bad arguments");
    cudaStream_t st = lat ? lat->stream : R->st;
    if (lat && cudaStreamSynchronize(R->st) != cudaSuccess) return rfail(R, VD_ERR_CUDA, "synchronize");
    float ph[12];
    for (int a = 0; a < 12; a++) ph[a] = pose ? pose[a] : ((a < 9 && a % 4 == 0) ? 1.f : 0.f);
    if (cudaMemcpyAsync(R->pose_dev, ph, sizeof(ph), cudaMemcpyHostToDevice, st) != cudaSuccess)
        return rfail(R, VD_ERR_CUDA, "pose upload failed");
    Ctx c{};
    if (lat) c = lat->c;
    const int np = R->W * R->H;
    const Cam cam{R->W, R->H, K[0], K[1], K[2], K[3]};
    k_mesh_deform<<<blocks_for(3L * R->n_tri), kThreads, 0, st>>>(c, lat ? 1 : 0, R->tri, 3 * R->n_tri, R->pose_dev,
                                                                   R->posed);
    k_zbuf_clear<<<blocks_for(np), kThreads, 0, st>>>(R->zbuf, np);
    k_raster<<<blocks_for(R->n_tri, 128), 128, 0, st>>>(R->posed, R->n_tri, cam, R->zbuf);
    k_zbuf_flags<<<blocks_for(np), kThreads, 0, st>>>(R->zbuf, cam, stride, R->flag);
    scan_launch(R->flag, np, R->poff, R->total + 1, R->sums, st);
    const bool dev = mem == VD_MEM_DEVICE;
    float *op = dev ? pts : R->stage, *on = dev ? nrm : R->stage + 3 * (size_t)np;
    int *opix = dev ? pix : (pix ? reinterpret_cast<int *>(R->stage + 6 * (size_t)np) : nullptr);
    const int wcap = dev ? cap : std::min(cap, np);
    k_resolve<<<blocks_for(np), kThreads, 0, st>>>(R->zbuf, R->flag, R->poff, R->posed, R->tri, R->nrm, cam, wcap,
                                                   op, on, opix);
    int total = 0;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&total, R->total + 1, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return rfail(R, VD_ERR_CUDA, "rasterisation launch failed");
    if (count) *count = total;
    if (!dev) {
        const size_t n = (size_t)std::min(total, wcap);
        if ((n && cudaMemcpy(pts, R->stage, 3 * n * sizeof(float), cudaMemcpyDeviceToHost) != cudaSuccess) ||
            (n && cudaMemcpy(nrm, R->stage + 3 * (size_t)np, 3 * n * sizeof(float), cudaMemcpyDeviceToHost) !=
                      cudaSuccess) ||
            (n && pix && cudaMemcpy(pix, R->stage + 6 * (size_t)np, n * sizeof(int), cudaMemcpyDeviceToHost) !=
                             cudaSuccess))
            return rfail(R, VD_ERR_CUDA, "sample download failed");
    }
    return VD_OK;
}

}  // extern "C"
