/*
 * FP64 CPU oracle for the VolumeDeform lattice solve (arXiv 1603.08161).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's CPU
 * baseline load this library; the product path never does.  It shares no code, header,
 * table or helper with the CUDA implementation.
 *
 * Everything is computed in double precision, plainly and slowly, in the order the
 * paper states it:
 *   - space deformation S(x) = R [sum_i alpha_i(x) t_i] + t, trilinear alpha  (Sec. 4)
 *   - projective association with Phi_r(x) = 1 - x/eps_r and
 *     w_c = ((Phi_d + Phi_n + Phi_v)/3)^2, pruned if any Phi < 0          (Sec. 5.1)
 *   - E_total = w_s E_sparse + w_d E_dense + w_r E_reg                     (Eq. 1)
 *   - point-to-plane E_dense (Eq. 2), feature E_sparse (Eq. 3), ARAP E_reg (Eq. 4)
 *   - flip-flop: positions with rotations fixed, then rotations with positions
 *     fixed (Sec. 7.1); positions by preconditioned CG on the normal equations
 *     (L + B^T B) t = b, rotations by Procrustes/SVD per grid point (Sec. 7.1)
 *
 * The Gauss-Newton system is built from an explicitly assembled sparse Jacobian J
 * (one row per dense residual, three per sparse pair, three per directed lattice
 * edge), applied as J^T (J p).  The rotation step uses a one-sided (Hestenes) Jacobi
 * SVD of the 3x3 cross-covariance (Golub & Van Loan, Matrix Computations, 4th ed.,
 * Sec. 8.6.3).
 *
 * Readings of points the paper leaves open (all documented with the build):
 *   - unknowns are displacements u_i = t_i - t^_i; node i = x + nx (y + ny z);
 *     t^_i = origin + h (x, y, z);
 *   - one-ring N_i = 6-neighbourhood restricted to M; both directions of an edge
 *     are kept (i->j uses R_i, j->i uses R_j);
 *   - M = corners of cells holding a sample or a sparse point, dilated by the
 *     6-neighbourhood (surface mode), or every node (all mode);
 *   - nearest pixel = floor(x + 0.5); target normal by central differences of the
 *     back-projected depth, oriented towards the camera; v = unit vector from the
 *     point to the camera centre; model normal n_c = normalise(R sum_k alpha_k R_k n^_c);
 *   - PCG: x0 = 0 on the increment, scalar Jacobi preconditioner (1/diag, 0 where the
 *     diagonal is 0), exactly K iterations unless p.Ap <= 0, rho = 0 or
 *     rho' <= tol^2 rho0;
 *   - a depth that is not a positive finite number marks an invalid pixel; a sample
 *     with a non-finite position or normal, or outside the lattice, is ignored;
 *   - a rotation is kept unchanged (and counted) when its neighbours span fewer than
 *     two lattice axes, when sigma_2 <= 1e-12 sigma_1, or when det < 0 and
 *     sigma_2 - sigma_3 <= 1e-12 sigma_1 (the best rotation is then not unique).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define VDO_ACTIVE_SURFACE 0
#define VDO_ACTIVE_ALL 1

typedef struct {
    int nrows, cap_rows;
    long nnz, cap_nnz;
    long *row_ptr;       /* nrows + 1 */
    int *col;
    double *val;
    double *res;         /* residual of each row */
} csr_t;

typedef struct vdo_ctx {
    /* lattice (Sec. 4) */
    int nx, ny, nz, nn;
    double o[3], h;
    int active_mode;
    /* coarse level of a hierarchy (Sec. 7.2): the finest lattice's node counts and
       spacing (same origin); a constraint belongs to this level only if its cell exists
       on the finest lattice.  dom_h = 0: no such restriction. */
    int dom_n[3];
    double dom_h;
    /* frame */
    int W, H;
    double fx, fy, cx, cy;
    double Rg[9], tg[3];
    double *depth;                       /* H*W */
    double *V, *Nm;                      /* H*W*3 target vertex / normal maps */
    unsigned char *nvalid;               /* H*W */
    int C;
    double *sp, *sn;                     /* C*3 canonical samples / normals */
    int *cell_c;                         /* C: lower-corner node of the cell or -1 */
    double *frac_c;                      /* C*3 */
    int S;
    double *fh, *ft;                     /* S*3 canonical / observed feature points */
    int *cell_s;
    double *frac_s;
    /* active set M */
    unsigned char *inM;                  /* nn */
    int *slot;                           /* nn: unknown index or -1 */
    int N;
    /* state: displacement and rotation of every node */
    double *u;                           /* nn*3 */
    double *R;                           /* nn*9, row-major */
    /* association (Sec. 5.1) */
    int *pix;                            /* C: py*W+px or -1 */
    double *wc;                          /* C */
    double *pa, *na;                     /* C*3 target point and normal */
    int n_valid;
    int have_assoc;
    /* weights and thresholds */
    double w_s, w_d, w_r, eps_d, eps_n, eps_v;
    /* Jacobian */
    csr_t J;
    int have_J;
} vdo_ctx;

/* ------------------------------------------------------------------ helpers */

static void *xcalloc(size_t n, size_t sz) { return calloc(n ? n : 1, sz); }

static int node_id(const vdo_ctx *c, int x, int y, int z) { return x + c->nx * (y + c->ny * z); }

static void node_xyz(const vdo_ctx *c, int i, int *x, int *y, int *z)
{
    *x = i % c->nx;
    *y = (i / c->nx) % c->ny;
    *z = i / (c->nx * c->ny);
}

static void node_pos(const vdo_ctx *c, int i, double p[3])       /* t^_i */
{
    int x, y, z;
    node_xyz(c, i, &x, &y, &z);
    p[0] = c->o[0] + c->h * x;
    p[1] = c->o[1] + c->h * y;
    p[2] = c->o[2] + c->h * z;
}

static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static void matvec3(const double *M, const double *v, double *out)  /* row-major M v */
{
    for (int r = 0; r < 3; r++) out[r] = M[3 * r] * v[0] + M[3 * r + 1] * v[1] + M[3 * r + 2] * v[2];
}

static void cross3(const double *a, const double *b, double *o)
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

/* 6-neighbourhood offsets: -x, +x, -y, +y, -z, +z */
static const int NB_D[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};

static int neighbour(const vdo_ctx *c, int i, int k)   /* node index or -1 */
{
    int x, y, z;
    node_xyz(c, i, &x, &y, &z);
    x += NB_D[k][0];
    y += NB_D[k][1];
    z += NB_D[k][2];
    if (x < 0 || y < 0 || z < 0 || x >= c->nx || y >= c->ny || z >= c->nz) return -1;
    return node_id(c, x, y, z);
}

/* Cell of a point and its trilinear fractions (Sec. 4).  The cell is named by its
 * lower corner node; points whose cell would need a node outside the lattice get -1. */
static int locate(const vdo_ctx *c, const double p[3], double frac[3])
{
    int ci[3];
    int dims[3] = {c->nx, c->ny, c->nz};
    if (c->dom_h > 0)   /* gathered from the finest level: its cell must exist there */
        for (int a = 0; a < 3; a++) {
            double fl = floor((p[a] - c->o[a]) / c->dom_h);
            if (!(fl >= 0.0) || fl > (double)(c->dom_n[a] - 2)) return -1;
        }
    for (int a = 0; a < 3; a++) {
        double q = (p[a] - c->o[a]) / c->h;
        double fl = floor(q);
        if (!(fl >= 0.0) || fl > (double)(dims[a] - 2)) return -1;
        ci[a] = (int)fl;
        frac[a] = q - fl;
    }
    return node_id(c, ci[0], ci[1], ci[2]);
}

/* the 8 corners k = (dx, dy, dz) of a cell and their weights alpha_k */
static void corners(const vdo_ctx *c, int cell, const double f[3], int node[8], double alpha[8])
{
    for (int k = 0; k < 8; k++) {
        int dx = k & 1, dy = (k >> 1) & 1, dz = (k >> 2) & 1;
        node[k] = cell + dx + c->nx * (dy + c->ny * dz);
        alpha[k] = (dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) * (dz ? f[2] : 1.0 - f[2]);
    }
}

/* S(x) = R_g [sum_k alpha_k t_k] + t_g with t_k = t^_k + u_k (Sec. 4) */
static void deform(const vdo_ctx *c, int cell, const double f[3], double out[3])
{
    int nd[8];
    double al[8], acc[3] = {0, 0, 0}, tk[3];
    corners(c, cell, f, nd, al);
    for (int k = 0; k < 8; k++) {
        node_pos(c, nd[k], tk);
        for (int a = 0; a < 3; a++) acc[a] += al[k] * (tk[a] + c->u[3 * nd[k] + a]);
    }
    matvec3(c->Rg, acc, out);
    for (int a = 0; a < 3; a++) out[a] += c->tg[a];
}

/* ------------------------------------------------------------------ lifetime */

vdo_ctx *vdo_create(int nx, int ny, int nz, const float origin[3], float h, int active_mode)
{
    if (nx < 2 || ny < 2 || nz < 2 || !(h > 0.0f)) return NULL;
    vdo_ctx *c = (vdo_ctx *)xcalloc(1, sizeof(vdo_ctx));
    c->nx = nx; c->ny = ny; c->nz = nz;
    c->nn = nx * ny * nz;
    for (int a = 0; a < 3; a++) c->o[a] = (double)origin[a];
    c->h = (double)h;
    c->active_mode = active_mode;
    c->u = (double *)xcalloc((size_t)c->nn * 3, sizeof(double));
    c->R = (double *)xcalloc((size_t)c->nn * 9, sizeof(double));
    for (int i = 0; i < c->nn; i++) c->R[9 * i] = c->R[9 * i + 4] = c->R[9 * i + 8] = 1.0;
    c->inM = (unsigned char *)xcalloc((size_t)c->nn, 1);
    c->slot = (int *)xcalloc((size_t)c->nn, sizeof(int));
    for (int a = 0; a < 9; a++) c->Rg[a] = (a % 4 == 0) ? 1.0 : 0.0;
    c->w_s = 10.0; c->w_d = 1.0; c->w_r = 1.0;
    c->eps_d = 0.05; c->eps_n = 0.5; c->eps_v = 0.8;
    return c;
}

static void free_frame(vdo_ctx *c)
{
    free(c->depth); free(c->V); free(c->Nm); free(c->nvalid);
    free(c->sp); free(c->sn); free(c->cell_c); free(c->frac_c);
    free(c->pix); free(c->wc); free(c->pa); free(c->na);
    c->depth = c->V = c->Nm = c->sp = c->sn = c->frac_c = c->wc = c->pa = c->na = NULL;
    c->nvalid = NULL; c->cell_c = c->pix = NULL;
}

static void free_J(csr_t *J)
{
    free(J->row_ptr); free(J->col); free(J->val); free(J->res);
    memset(J, 0, sizeof(*J));
}

void vdo_destroy(vdo_ctx *c)
{
    if (!c) return;
    free_frame(c);
    free(c->fh); free(c->ft); free(c->cell_s); free(c->frac_s);
    free(c->u); free(c->R); free(c->inM); free(c->slot);
    free_J(&c->J);
    free(c);
}

void vdo_set_params(vdo_ctx *c, double w_s, double w_d, double w_r,
                    double eps_d, double eps_n, double eps_v)
{
    c->w_s = w_s; c->w_d = w_d; c->w_r = w_r;
    c->eps_d = eps_d; c->eps_n = eps_n; c->eps_v = eps_v;
    c->have_assoc = 0;
    c->have_J = 0;
}

/* ------------------------------------------------------------------ active set */

static void build_active(vdo_ctx *c)
{
    memset(c->inM, 0, (size_t)c->nn);
    if (c->active_mode == VDO_ACTIVE_ALL) {
        memset(c->inM, 1, (size_t)c->nn);
    } else {
        /* corners of every cell that holds a sample or a sparse point ... */
        unsigned char *mark = (unsigned char *)xcalloc((size_t)c->nn, 1);
        int nd[8];
        double al[8];
        for (int s = 0; s < c->C; s++)
            if (c->cell_c[s] >= 0) {
                corners(c, c->cell_c[s], c->frac_c + 3 * s, nd, al);
                for (int k = 0; k < 8; k++) mark[nd[k]] = 1;
            }
        for (int s = 0; s < c->S; s++)
            if (c->cell_s[s] >= 0) {
                corners(c, c->cell_s[s], c->frac_s + 3 * s, nd, al);
                for (int k = 0; k < 8; k++) mark[nd[k]] = 1;
            }
        /* ... plus their one-ring (Sec. 6: "the isosurface plus its one-ring") */
        for (int i = 0; i < c->nn; i++) {
            int on = mark[i];
            for (int k = 0; k < 6 && !on; k++) {
                int j = neighbour(c, i, k);
                if (j >= 0 && mark[j]) on = 1;
            }
            c->inM[i] = (unsigned char)on;
        }
        free(mark);
    }
    c->N = 0;
    for (int i = 0; i < c->nn; i++) c->slot[i] = c->inM[i] ? c->N++ : -1;
}

/* ------------------------------------------------------------------ frame input */

int vdo_set_frame(vdo_ctx *c, const float *depth, int W, int H, const float K[4], const float *pose,
                  const float *src_p, const float *src_n, int C)
{
    if (W < 0 || H < 0 || C < 0) return 1;
    free_frame(c);
    c->W = W; c->H = H;
    c->fx = K[0]; c->fy = K[1]; c->cx = K[2]; c->cy = K[3];
    for (int a = 0; a < 9; a++) c->Rg[a] = pose ? (double)pose[a] : ((a % 4 == 0) ? 1.0 : 0.0);
    for (int a = 0; a < 3; a++) c->tg[a] = pose ? (double)pose[9 + a] : 0.0;
    size_t np = (size_t)W * H;
    c->depth = (double *)xcalloc(np, sizeof(double));
    /* a depth that is not a positive finite number marks an invalid pixel, as 0 does */
    for (size_t k = 0; k < np; k++) {
        double d = (double)depth[k];
        c->depth[k] = (isfinite(d) && d > 0.0) ? d : 0.0;
    }

    /* target vertex map V and normal map (central differences, facing the camera) */
    c->V = (double *)xcalloc(np * 3, sizeof(double));
    c->Nm = (double *)xcalloc(np * 3, sizeof(double));
    c->nvalid = (unsigned char *)xcalloc(np, 1);
    for (int v = 0; v < H; v++)
        for (int uu = 0; uu < W; uu++) {
            double d = c->depth[(size_t)v * W + uu];
            double *P = c->V + 3 * ((size_t)v * W + uu);
            P[0] = d * ((uu - c->cx) / c->fx);
            P[1] = d * ((v - c->cy) / c->fy);
            P[2] = d;
        }
    for (int v = 1; v + 1 < H; v++)
        for (int uu = 1; uu + 1 < W; uu++) {
            size_t k = (size_t)v * W + uu;
            if (c->depth[k] <= 0 || c->depth[k - 1] <= 0 || c->depth[k + 1] <= 0 ||
                c->depth[k - W] <= 0 || c->depth[k + W] <= 0)
                continue;
            double dx[3], dy[3], n[3];
            for (int a = 0; a < 3; a++) {
                dx[a] = c->V[3 * (k + 1) + a] - c->V[3 * (k - 1) + a];
                dy[a] = c->V[3 * (k + W) + a] - c->V[3 * (k - W) + a];
            }
            cross3(dx, dy, n);
            double L = sqrt(dot3(n, n));
            if (!(L > 0)) continue;
            for (int a = 0; a < 3; a++) n[a] /= L;
            if (dot3(n, c->V + 3 * k) > 0)
                for (int a = 0; a < 3; a++) n[a] = -n[a];
            for (int a = 0; a < 3; a++) c->Nm[3 * k + a] = n[a];
            c->nvalid[k] = 1;
        }

    c->C = C;
    c->sp = (double *)xcalloc((size_t)C * 3, sizeof(double));
    c->sn = (double *)xcalloc((size_t)C * 3, sizeof(double));
    c->cell_c = (int *)xcalloc((size_t)C, sizeof(int));
    c->frac_c = (double *)xcalloc((size_t)C * 3, sizeof(double));
    c->pix = (int *)xcalloc((size_t)C, sizeof(int));
    c->wc = (double *)xcalloc((size_t)C, sizeof(double));
    c->pa = (double *)xcalloc((size_t)C * 3, sizeof(double));
    c->na = (double *)xcalloc((size_t)C * 3, sizeof(double));
    for (int s = 0; s < C; s++) {
        for (int a = 0; a < 3; a++) {
            c->sp[3 * s + a] = src_p[3 * s + a];
            c->sn[3 * s + a] = src_n[3 * s + a];
        }
        c->cell_c[s] = locate(c, c->sp + 3 * s, c->frac_c + 3 * s);
        /* a sample whose normal is not finite is ignored, like one outside the lattice
           (a non-finite position already fails locate) */
        if (!isfinite(c->sn[3 * s]) || !isfinite(c->sn[3 * s + 1]) || !isfinite(c->sn[3 * s + 2]))
            c->cell_c[s] = -1;
    }
    if (!c->fh) c->S = 0;
    build_active(c);
    c->have_assoc = 0;
    c->have_J = 0;
    return 0;
}

int vdo_set_correspondences(vdo_ctx *c, const float *canon, const float *target, int S)
{
    if (S < 0) return 1;
    free(c->fh); free(c->ft); free(c->cell_s); free(c->frac_s);
    c->S = S;
    c->fh = (double *)xcalloc((size_t)S * 3, sizeof(double));
    c->ft = (double *)xcalloc((size_t)S * 3, sizeof(double));
    c->cell_s = (int *)xcalloc((size_t)S, sizeof(int));
    c->frac_s = (double *)xcalloc((size_t)S * 3, sizeof(double));
    for (int s = 0; s < S; s++) {
        for (int a = 0; a < 3; a++) {
            c->fh[3 * s + a] = canon[3 * s + a];
            c->ft[3 * s + a] = target[3 * s + a];
        }
        c->cell_s[s] = locate(c, c->fh + 3 * s, c->frac_s + 3 * s);
    }
    if (c->cell_c || c->C == 0) build_active(c);
    c->have_J = 0;
    return 0;
}

/* ------------------------------------------------------------------ state access */

void vdo_set_warp(vdo_ctx *c, const double *u, const double *R)
{
    if (u) memcpy(c->u, u, sizeof(double) * 3 * (size_t)c->nn);
    else memset(c->u, 0, sizeof(double) * 3 * (size_t)c->nn);
    if (R) memcpy(c->R, R, sizeof(double) * 9 * (size_t)c->nn);
    else {
        memset(c->R, 0, sizeof(double) * 9 * (size_t)c->nn);
        for (int i = 0; i < c->nn; i++) c->R[9 * i] = c->R[9 * i + 4] = c->R[9 * i + 8] = 1.0;
    }
    c->have_J = 0;
}

void vdo_get_warp(const vdo_ctx *c, double *u, double *R)
{
    if (u) memcpy(u, c->u, sizeof(double) * 3 * (size_t)c->nn);
    if (R) memcpy(R, c->R, sizeof(double) * 9 * (size_t)c->nn);
}

int vdo_num_active(const vdo_ctx *c) { return c->N; }

void vdo_get_active(const vdo_ctx *c, unsigned char *mask) { memcpy(mask, c->inM, (size_t)c->nn); }

void vdo_target_maps(const vdo_ctx *c, double *V, double *Nm, unsigned char *valid)
{
    size_t np = (size_t)c->W * c->H;
    if (V) memcpy(V, c->V, sizeof(double) * 3 * np);
    if (Nm) memcpy(Nm, c->Nm, sizeof(double) * 3 * np);
    if (valid) memcpy(valid, c->nvalid, np);
}

void vdo_sample_cells(const vdo_ctx *c, int *cell, double *frac)
{
    if (cell) memcpy(cell, c->cell_c, sizeof(int) * (size_t)c->C);
    if (frac) memcpy(frac, c->frac_c, sizeof(double) * 3 * (size_t)c->C);
}

/* ------------------------------------------------------------------ association */

/* Projective association of every sample at the current warp (Sec. 5.1).  Returns
 * the number of samples with w_c > 0. */
int vdo_associate(vdo_ctx *c)
{
    int nvalid = 0;
    for (int s = 0; s < c->C; s++) {
        c->pix[s] = -1;
        c->wc[s] = 0.0;
        for (int a = 0; a < 3; a++) c->pa[3 * s + a] = c->na[3 * s + a] = 0.0;
        int cell = c->cell_c[s];
        if (cell < 0) continue;
        double p[3], n[3], acc[3] = {0, 0, 0}, rn[3];
        deform(c, cell, c->frac_c + 3 * s, p);
        /* model normal: R_g sum_k alpha_k R_k n^_c, normalised */
        int nd[8];
        double al[8];
        corners(c, cell, c->frac_c + 3 * s, nd, al);
        for (int k = 0; k < 8; k++) {
            matvec3(c->R + 9 * nd[k], c->sn + 3 * s, rn);
            for (int a = 0; a < 3; a++) acc[a] += al[k] * rn[a];
        }
        matvec3(c->Rg, acc, n);
        double nl = sqrt(dot3(n, n));
        if (!(nl > 0)) continue;
        for (int a = 0; a < 3; a++) n[a] /= nl;
        if (!(p[2] > 0)) continue;
        double uf = c->fx * p[0] / p[2] + c->cx;
        double vf = c->fy * p[1] / p[2] + c->cy;
        double px = floor(uf + 0.5), py = floor(vf + 0.5);
        if (!(px >= 0 && px < c->W && py >= 0 && py < c->H)) continue;
        size_t k = (size_t)py * c->W + (size_t)px;
        if (!(c->depth[k] > 0) || !c->nvalid[k]) continue;
        const double *pa = c->V + 3 * k, *na = c->Nm + 3 * k;
        double diff[3] = {p[0] - pa[0], p[1] - pa[1], p[2] - pa[2]};
        double pl = sqrt(dot3(p, p));
        double view[3] = {-p[0] / pl, -p[1] / pl, -p[2] / pl};
        double phi_d = 1.0 - sqrt(dot3(diff, diff)) / c->eps_d;
        double phi_n = 1.0 - (1.0 - dot3(n, na)) / c->eps_n;
        double phi_v = 1.0 - (1.0 - dot3(n, view)) / c->eps_v;
        c->pix[s] = (int)k;
        for (int a = 0; a < 3; a++) {
            c->pa[3 * s + a] = pa[a];
            c->na[3 * s + a] = na[a];
        }
        if (phi_d < 0 || phi_n < 0 || phi_v < 0) continue;
        double m = (phi_d + phi_n + phi_v) / 3.0;
        c->wc[s] = m * m;
        nvalid++;
    }
    c->n_valid = nvalid;
    c->have_assoc = 1;
    c->have_J = 0;
    return nvalid;
}

void vdo_get_association(const vdo_ctx *c, int *pix, double *w, double *r)
{
    for (int s = 0; s < c->C; s++) {
        if (pix) pix[s] = c->pix[s];
        if (w) w[s] = c->wc[s];
        if (r) {
            r[s] = 0.0;
            if (c->wc[s] > 0) {
                double p[3];
                deform(c, c->cell_c[s], c->frac_c + 3 * s, p);
                double d[3] = {p[0] - c->pa[3 * s], p[1] - c->pa[3 * s + 1], p[2] - c->pa[3 * s + 2]};
                r[s] = sqrt(c->w_d * c->wc[s]) * dot3(d, c->na + 3 * s);
            }
        }
    }
}

/* ------------------------------------------------------------------ energy (Eq. 1-4) */

void vdo_energy(const vdo_ctx *c, double out[4])
{
    double ed = 0, es = 0, er = 0;
    for (int s = 0; s < c->C && c->have_assoc; s++) {
        if (!(c->wc[s] > 0)) continue;
        double p[3];
        deform(c, c->cell_c[s], c->frac_c + 3 * s, p);
        double d[3] = {p[0] - c->pa[3 * s], p[1] - c->pa[3 * s + 1], p[2] - c->pa[3 * s + 2]};
        double e = dot3(d, c->na + 3 * s);
        ed += c->wc[s] * e * e;                                          /* Eq. 2 */
    }
    for (int s = 0; s < c->S; s++) {
        if (c->cell_s[s] < 0) continue;
        double p[3];
        deform(c, c->cell_s[s], c->frac_s + 3 * s, p);
        for (int a = 0; a < 3; a++) es += (p[a] - c->ft[3 * s + a]) * (p[a] - c->ft[3 * s + a]);  /* Eq. 3 */
    }
    for (int i = 0; i < c->nn; i++) {                                    /* Eq. 4 */
        if (!c->inM[i]) continue;
        double ti[3], hi[3];
        node_pos(c, i, hi);
        for (int a = 0; a < 3; a++) ti[a] = hi[a] + c->u[3 * i + a];
        for (int k = 0; k < 6; k++) {
            int j = neighbour(c, i, k);
            if (j < 0 || !c->inM[j]) continue;
            double tj[3], hj[3], e[3], Re[3];
            node_pos(c, j, hj);
            for (int a = 0; a < 3; a++) {
                tj[a] = hj[a] + c->u[3 * j + a];
                e[a] = hi[a] - hj[a];
            }
            matvec3(c->R + 9 * i, e, Re);
            for (int a = 0; a < 3; a++) {
                double q = (ti[a] - tj[a]) - Re[a];
                er += q * q;
            }
        }
    }
    out[1] = ed;
    out[2] = es;
    out[3] = er;
    out[0] = c->w_s * es + c->w_d * ed + c->w_r * er;                   /* Eq. 1 */
}

/* ------------------------------------------------------------------ Jacobian */

static void J_reserve(csr_t *J, int rows, long nnz)
{
    if (rows + 1 > J->cap_rows) {
        J->cap_rows = 2 * (rows + 1) + 16;
        J->row_ptr = (long *)realloc(J->row_ptr, sizeof(long) * (size_t)J->cap_rows);
        J->res = (double *)realloc(J->res, sizeof(double) * (size_t)J->cap_rows);
    }
    if (nnz > J->cap_nnz) {
        J->cap_nnz = 2 * nnz + 64;
        J->col = (int *)realloc(J->col, sizeof(int) * (size_t)J->cap_nnz);
        J->val = (double *)realloc(J->val, sizeof(double) * (size_t)J->cap_nnz);
    }
}

static void J_begin_row(csr_t *J, double res)
{
    J_reserve(J, J->nrows + 1, J->nnz);
    J->row_ptr[J->nrows] = J->nnz;
    J->res[J->nrows] = res;
}

static void J_entry(csr_t *J, int col, double v)
{
    J_reserve(J, J->nrows + 1, J->nnz + 1);
    J->col[J->nnz] = col;
    J->val[J->nnz] = v;
    J->nnz++;
}

static void J_end_row(csr_t *J)
{
    J->nrows++;
    J_reserve(J, J->nrows + 1, J->nnz);
    J->row_ptr[J->nrows] = J->nnz;
}

/* Residual vector r and Jacobian J of E_total w.r.t. the displacements of M at the
 * current warp, with association and rotations held fixed (Sec. 7.1, position step). */
static void build_J(vdo_ctx *c)
{
    csr_t *J = &c->J;
    J->nrows = 0;
    J->nnz = 0;
    J_reserve(J, 1, 0);
    J->row_ptr[0] = 0;
    int nd[8];
    double al[8];
    /* dense point-to-plane rows (Eq. 2): sqrt(w_d w_c) n^a . (S(p^c) - p^a) */
    for (int s = 0; s < c->C; s++) {
        if (!(c->wc[s] > 0)) continue;
        double p[3], g[3], sw = sqrt(c->w_d * c->wc[s]);
        deform(c, c->cell_c[s], c->frac_c + 3 * s, p);
        double d[3] = {p[0] - c->pa[3 * s], p[1] - c->pa[3 * s + 1], p[2] - c->pa[3 * s + 2]};
        const double *na = c->na + 3 * s;
        for (int a = 0; a < 3; a++)                                  /* R_g^T n^a */
            g[a] = c->Rg[a] * na[0] + c->Rg[3 + a] * na[1] + c->Rg[6 + a] * na[2];
        J_begin_row(J, sw * dot3(d, na));
        corners(c, c->cell_c[s], c->frac_c + 3 * s, nd, al);
        for (int k = 0; k < 8; k++)
            for (int a = 0; a < 3; a++) J_entry(J, 3 * c->slot[nd[k]] + a, sw * al[k] * g[a]);
        J_end_row(J);
    }
    /* sparse feature rows (Eq. 3): sqrt(w_s) (S(f^s) - f_s) */
    double sws = sqrt(c->w_s);
    for (int s = 0; s < c->S; s++) {
        if (c->cell_s[s] < 0) continue;
        double p[3];
        deform(c, c->cell_s[s], c->frac_s + 3 * s, p);
        corners(c, c->cell_s[s], c->frac_s + 3 * s, nd, al);
        for (int e = 0; e < 3; e++) {
            J_begin_row(J, sws * (p[e] - c->ft[3 * s + e]));
            for (int k = 0; k < 8; k++)
                for (int a = 0; a < 3; a++) J_entry(J, 3 * c->slot[nd[k]] + a, sws * al[k] * c->Rg[3 * e + a]);
            J_end_row(J);
        }
    }
    /* ARAP rows (Eq. 4), one triple per directed edge i -> j inside M */
    double swr = sqrt(c->w_r);
    for (int i = 0; i < c->nn; i++) {
        if (!c->inM[i]) continue;
        double hi[3];
        node_pos(c, i, hi);
        for (int k = 0; k < 6; k++) {
            int j = neighbour(c, i, k);
            if (j < 0 || !c->inM[j]) continue;
            double hj[3], e[3], Re[3];
            node_pos(c, j, hj);
            for (int a = 0; a < 3; a++) e[a] = hi[a] - hj[a];
            matvec3(c->R + 9 * i, e, Re);
            for (int a = 0; a < 3; a++) {
                double q = (hi[a] + c->u[3 * i + a]) - (hj[a] + c->u[3 * j + a]) - Re[a];
                J_begin_row(J, swr * q);
                J_entry(J, 3 * c->slot[i] + a, swr);
                J_entry(J, 3 * c->slot[j] + a, -swr);
                J_end_row(J);
            }
        }
    }
    c->have_J = 1;
}

static void ensure_J(vdo_ctx *c)
{
    if (!c->have_assoc) vdo_associate(c);
    if (!c->have_J) build_J(c);
}

/* y = J^T (J x) on the unknowns (length 3N) */
static void apply_JtJ(const csr_t *J, const double *x, double *y, int n3, double *tmp)
{
    for (int r = 0; r < J->nrows; r++) {
        double acc = 0;
        for (long k = J->row_ptr[r]; k < J->row_ptr[r + 1]; k++) acc += J->val[k] * x[J->col[k]];
        tmp[r] = acc;
    }
    memset(y, 0, sizeof(double) * (size_t)n3);
    for (int r = 0; r < J->nrows; r++)
        for (long k = J->row_ptr[r]; k < J->row_ptr[r + 1]; k++) y[J->col[k]] += J->val[k] * tmp[r];
}

static void scatter_nodes(const vdo_ctx *c, const double *xs, double *full)   /* 3N -> 3nn */
{
    memset(full, 0, sizeof(double) * 3 * (size_t)c->nn);
    for (int i = 0; i < c->nn; i++)
        if (c->slot[i] >= 0)
            for (int a = 0; a < 3; a++) full[3 * i + a] = xs[3 * c->slot[i] + a];
}

static void gather_nodes(const vdo_ctx *c, const double *full, double *xs)    /* 3nn -> 3N */
{
    for (int i = 0; i < c->nn; i++)
        if (c->slot[i] >= 0)
            for (int a = 0; a < 3; a++) xs[3 * c->slot[i] + a] = full[3 * i + a];
}

/* b = -J^T r and the diagonal of J^T J, as full-lattice arrays (0 outside M) */
void vdo_rhs(vdo_ctx *c, double *b, double *diag)
{
    ensure_J(c);
    int n3 = 3 * c->N;
    double *bs = (double *)xcalloc((size_t)n3, sizeof(double));
    double *ds = (double *)xcalloc((size_t)n3, sizeof(double));
    const csr_t *J = &c->J;
    for (int r = 0; r < J->nrows; r++)
        for (long k = J->row_ptr[r]; k < J->row_ptr[r + 1]; k++) {
            bs[J->col[k]] -= J->val[k] * J->res[r];
            ds[J->col[k]] += J->val[k] * J->val[k];
        }
    if (b) scatter_nodes(c, bs, b);
    if (diag) scatter_nodes(c, ds, diag);
    free(bs);
    free(ds);
}

void vdo_apply(vdo_ctx *c, const double *p, double *Ap)
{
    ensure_J(c);
    int n3 = 3 * c->N;
    double *ps = (double *)xcalloc((size_t)n3, sizeof(double));
    double *qs = (double *)xcalloc((size_t)n3, sizeof(double));
    double *tmp = (double *)xcalloc((size_t)c->J.nrows, sizeof(double));
    gather_nodes(c, p, ps);
    apply_JtJ(&c->J, ps, qs, n3, tmp);
    scatter_nodes(c, qs, Ap);
    free(ps); free(qs); free(tmp);
}

/* Jacobi-preconditioned CG on J^T J delta = -J^T r, x0 = 0 (Sec. 7.1).  Writes the
 * increment for every node (0 outside M); returns the number of iterations done.
 * rho_hist (optional, K+1 entries) receives r.z before each iteration. */
int vdo_pcg(vdo_ctx *c, int K, double tol, double *delta, double *rho_hist)
{
    ensure_J(c);
    int n3 = 3 * c->N;
    const csr_t *J = &c->J;
    double *x = (double *)xcalloc((size_t)n3, sizeof(double));
    double *r = (double *)xcalloc((size_t)n3, sizeof(double));
    double *z = (double *)xcalloc((size_t)n3, sizeof(double));
    double *p = (double *)xcalloc((size_t)n3, sizeof(double));
    double *q = (double *)xcalloc((size_t)n3, sizeof(double));
    double *Minv = (double *)xcalloc((size_t)n3, sizeof(double));
    double *tmp = (double *)xcalloc((size_t)J->nrows, sizeof(double));
    for (int rr = 0; rr < J->nrows; rr++)
        for (long k = J->row_ptr[rr]; k < J->row_ptr[rr + 1]; k++) {
            r[J->col[k]] -= J->val[k] * J->res[rr];         /* b = -J^T r */
            Minv[J->col[k]] += J->val[k] * J->val[k];       /* diag(J^T J) */
        }
    for (int k = 0; k < n3; k++) Minv[k] = Minv[k] > 0 ? 1.0 / Minv[k] : 0.0;
    double rho = 0;
    for (int k = 0; k < n3; k++) {
        z[k] = Minv[k] * r[k];
        p[k] = z[k];
        rho += r[k] * z[k];
    }
    double rho0 = rho;
    int it = 0;
    for (; it < K; it++) {
        if (rho_hist) rho_hist[it] = rho;
        if (!(rho > 0)) break;
        apply_JtJ(J, p, q, n3, tmp);
        double pq = 0;
        for (int k = 0; k < n3; k++) pq += p[k] * q[k];
        if (!(pq > 0)) break;
        double alpha = rho / pq;
        double rho1 = 0;
        for (int k = 0; k < n3; k++) {
            x[k] += alpha * p[k];
            r[k] -= alpha * q[k];
            z[k] = Minv[k] * r[k];
            rho1 += r[k] * z[k];
        }
        if (rho1 <= tol * tol * rho0) {
            rho = rho1;
            it++;
            break;
        }
        double beta = rho1 / rho;
        for (int k = 0; k < n3; k++) p[k] = z[k] + beta * p[k];
        rho = rho1;
    }
    if (rho_hist) rho_hist[it] = rho;
    scatter_nodes(c, x, delta);
    free(x); free(r); free(z); free(p); free(q); free(Minv); free(tmp);
    return it;
}

/* Exact solution of J^T J delta = -J^T r by dense Cholesky (tiny lattices only).
 * Returns 0 on success, 1 if the matrix is not positive definite. */
int vdo_cholesky(vdo_ctx *c, double *delta)
{
    ensure_J(c);
    int n = 3 * c->N;
    const csr_t *J = &c->J;
    double *A = (double *)xcalloc((size_t)n * n, sizeof(double));
    double *b = (double *)xcalloc((size_t)n, sizeof(double));
    for (int r = 0; r < J->nrows; r++)
        for (long k = J->row_ptr[r]; k < J->row_ptr[r + 1]; k++) {
            b[J->col[k]] -= J->val[k] * J->res[r];
            for (long m = J->row_ptr[r]; m < J->row_ptr[r + 1]; m++)
                A[(size_t)J->col[k] * n + J->col[m]] += J->val[k] * J->val[m];
        }
    int bad = 0;
    for (int j = 0; j < n && !bad; j++) {                 /* A = L L^T, L in the lower half */
        double s = A[(size_t)j * n + j];
        for (int k = 0; k < j; k++) s -= A[(size_t)j * n + k] * A[(size_t)j * n + k];
        if (!(s > 0)) { bad = 1; break; }
        double Ljj = sqrt(s);
        A[(size_t)j * n + j] = Ljj;
        for (int i = j + 1; i < n; i++) {
            double t = A[(size_t)i * n + j];
            for (int k = 0; k < j; k++) t -= A[(size_t)i * n + k] * A[(size_t)j * n + k];
            A[(size_t)i * n + j] = t / Ljj;
        }
    }
    if (!bad) {
        for (int i = 0; i < n; i++) {                      /* L y = b */
            double t = b[i];
            for (int k = 0; k < i; k++) t -= A[(size_t)i * n + k] * b[k];
            b[i] = t / A[(size_t)i * n + i];
        }
        for (int i = n - 1; i >= 0; i--) {                 /* L^T x = y */
            double t = b[i];
            for (int k = i + 1; k < n; k++) t -= A[(size_t)k * n + i] * b[k];
            b[i] = t / A[(size_t)i * n + i];
        }
        scatter_nodes(c, b, delta);
    }
    free(A);
    free(b);
    return bad;
}

void vdo_add_increment(vdo_ctx *c, const double *delta)
{
    for (int i = 0; i < c->nn; i++)
        if (c->inM[i])
            for (int a = 0; a < 3; a++) c->u[3 * i + a] += delta[3 * i + a];
    c->have_J = 0;
}

/* ------------------------------------------------------------------ rotation step */

/* One-sided Jacobi SVD of a 3x3 matrix A = U diag(s) V^T, s descending. */
void vdo_svd3(const double *A, double *U, double *s, double *V)
{
    double B[9];
    memcpy(B, A, sizeof(B));
    for (int k = 0; k < 9; k++) V[k] = (k % 4 == 0) ? 1.0 : 0.0;
    static const int P[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    for (int sweep = 0; sweep < 64; sweep++) {
        int rotated = 0;
        for (int m = 0; m < 3; m++) {
            int p = P[m][0], q = P[m][1];
            double al = 0, be = 0, ga = 0;
            for (int r = 0; r < 3; r++) {
                al += B[3 * r + p] * B[3 * r + p];
                be += B[3 * r + q] * B[3 * r + q];
                ga += B[3 * r + p] * B[3 * r + q];
            }
            if (ga == 0.0 || fabs(ga) <= 1e-15 * sqrt(al * be)) continue;
            rotated = 1;
            double zeta = (be - al) / (2.0 * ga);
            double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
            for (int r = 0; r < 3; r++) {
                double bp = B[3 * r + p], bq = B[3 * r + q];
                B[3 * r + p] = cs * bp - sn * bq;
                B[3 * r + q] = sn * bp + cs * bq;
                double vp = V[3 * r + p], vq = V[3 * r + q];
                V[3 * r + p] = cs * vp - sn * vq;
                V[3 * r + q] = sn * vp + cs * vq;
            }
        }
        if (!rotated) break;
    }
    double sig[3];
    for (int k = 0; k < 3; k++)
        sig[k] = sqrt(B[k] * B[k] + B[3 + k] * B[3 + k] + B[6 + k] * B[6 + k]);
    int ord[3] = {0, 1, 2};
    for (int a = 0; a < 3; a++)                 /* sort columns by singular value */
        for (int b2 = a + 1; b2 < 3; b2++)
            if (sig[ord[b2]] > sig[ord[a]]) { int t = ord[a]; ord[a] = ord[b2]; ord[b2] = t; }
    double Vs[9];
    memcpy(Vs, V, sizeof(Vs));
    for (int k = 0; k < 3; k++) {
        int o = ord[k];
        s[k] = sig[o];
        for (int r = 0; r < 3; r++) {
            V[3 * r + k] = Vs[3 * r + o];
            U[3 * r + k] = sig[o] > 0 ? B[3 * r + o] / sig[o] : 0.0;
        }
    }
    /* complete U where a singular value vanished */
    if (!(s[1] > 0)) {
        double e[3] = {1, 0, 0};
        double u0[3] = {U[0], U[3], U[6]};
        if (fabs(u0[0]) > 0.9) { e[0] = 0; e[1] = 1; }
        double w[3];
        cross3(u0, e, w);
        double L = sqrt(dot3(w, w));
        for (int r = 0; r < 3; r++) U[3 * r + 1] = w[r] / L;
    }
    if (!(s[2] > 0)) {
        double u0[3] = {U[0], U[3], U[6]}, u1[3] = {U[1], U[4], U[7]}, w[3];
        cross3(u0, u1, w);
        for (int r = 0; r < 3; r++) U[3 * r + 2] = w[r];
    }
}

static double det3(const double *M)
{
    return M[0] * (M[4] * M[8] - M[5] * M[7]) - M[1] * (M[3] * M[8] - M[5] * M[6]) +
           M[2] * (M[3] * M[7] - M[4] * M[6]);
}

/* Best rotation argmax_R tr(R^T A) = U diag(1, 1, det(U V^T)) V^T.  Returns 0, or 1
 * when it is not unique (rank <= 1, or a reflection with sigma_2 = sigma_3). */
int vdo_procrustes(const double *A, double *R)
{
    double U[9], s[3], V[9];
    vdo_svd3(A, U, s, V);
    double d = det3(U) * det3(V) < 0 ? -1.0 : 1.0;
    if (!(s[0] > 0) || s[1] <= 1e-12 * s[0]) return 1;
    if (d < 0 && s[1] - s[2] <= 1e-12 * s[0]) return 1;
    for (int r = 0; r < 3; r++)
        for (int q = 0; q < 3; q++)
            R[3 * r + q] = U[3 * r] * V[3 * q] + U[3 * r + 1] * V[3 * q + 1] + d * U[3 * r + 2] * V[3 * q + 2];
    return 0;
}

/* Rotation step of the flip-flop (Sec. 7.1): per node of M, the cross-covariance
 * A_i = sum_{j in N_i} (t_i - t_j)(t^_i - t^_j)^T and its Procrustes rotation.
 * Returns the number of nodes whose rotation was left unchanged. */
int vdo_fit_rotations(vdo_ctx *c)
{
    int degenerate = 0;
    double *Rn = (double *)xcalloc((size_t)c->nn * 9, sizeof(double));
    memcpy(Rn, c->R, sizeof(double) * 9 * (size_t)c->nn);
    for (int i = 0; i < c->nn; i++) {
        if (!c->inM[i]) continue;
        double A[9] = {0}, hi[3];
        int axes[3] = {0, 0, 0};
        node_pos(c, i, hi);
        for (int k = 0; k < 6; k++) {
            int j = neighbour(c, i, k);
            if (j < 0 || !c->inM[j]) continue;
            axes[k / 2] = 1;
            double hj[3], d[3], e[3];
            node_pos(c, j, hj);
            for (int a = 0; a < 3; a++) {
                d[a] = (hi[a] + c->u[3 * i + a]) - (hj[a] + c->u[3 * j + a]);
                e[a] = hi[a] - hj[a];
            }
            for (int r = 0; r < 3; r++)
                for (int q = 0; q < 3; q++) A[3 * r + q] += d[r] * e[q];
        }
        if (axes[0] + axes[1] + axes[2] < 2 || vdo_procrustes(A, Rn + 9 * i)) {
            degenerate++;
            memcpy(Rn + 9 * i, c->R + 9 * i, sizeof(double) * 9);
        }
    }
    memcpy(c->R, Rn, sizeof(double) * 9 * (size_t)c->nn);
    free(Rn);
    c->have_J = 0;
    return degenerate;
}

/* ------------------------------------------------------------------ flip-flop driver */

/* Full per-frame solve: for each Gauss-Newton iteration, associate (unless frozen
 * after the first), solve the position step by PCG (or Cholesky), add the increment,
 * fit rotations, and record E (Eq. 1) under that iteration's association.
 * e_hist receives 4 doubles per iteration (total, dense, sparse, reg); cg_hist the
 * CG iterations of each; stats[0] = valid correspondences of the last association,
 * stats[1] = degenerate rotations of the last step.  Returns iterations done. */
int vdo_solve(vdo_ctx *c, int gn_iters, int cg_iters, double cg_tol, int fixed_assoc,
              int use_cholesky, double *e_hist, int *cg_hist, int *stats)
{
    double *delta = (double *)xcalloc((size_t)c->nn * 3, sizeof(double));
    int g = 0, deg = 0;
    for (; g < gn_iters; g++) {
        if (!(fixed_assoc && g > 0 && c->have_assoc)) vdo_associate(c);
        int it = 0;
        if (use_cholesky) {
            if (vdo_cholesky(c, delta)) break;
        } else {
            it = vdo_pcg(c, cg_iters, cg_tol, delta, NULL);
        }
        vdo_add_increment(c, delta);
        deg = vdo_fit_rotations(c);
        if (e_hist) vdo_energy(c, e_hist + 4 * g);
        if (cg_hist) cg_hist[g] = it;
    }
    if (stats) {
        stats[0] = c->n_valid;
        stats[1] = deg;
    }
    free(delta);
    return g;
}

/* ------------------------------------------------------------------ hierarchy (Sec. 7.2) */

/* Mark c as a coarse level of a hierarchy whose finest lattice has n0 nodes per axis and
 * spacing h0 (same origin): only constraints whose cell exists on the finest lattice are
 * gathered.  Call before vdo_set_frame / vdo_set_correspondences. */
void vdo_set_domain(vdo_ctx *c, int nx0, int ny0, int nz0, float h0)
{
    c->dom_n[0] = nx0; c->dom_n[1] = ny0; c->dom_n[2] = nz0;
    c->dom_h = (double)h0;
}

/* Start state of a coarse level: every coarse node takes the displacement and rotation
 * of the finer node it coincides with (node 2X of the finer level).  A coarse node one
 * spacing past the end of the finer lattice along an axis (n - 1 odd) has no such node:
 * its displacement is extrapolated linearly along that axis from the last two finer
 * nodes, 2 u(n - 1) - u(n - 2) (per axis, so affine fields are reproduced exactly), and
 * it takes the rotation of the finer lattice's nearest node. */
void vdo_restrict_state(const vdo_ctx *fine, vdo_ctx *coarse)
{
    int fd[3] = {fine->nx, fine->ny, fine->nz};
    for (int I = 0; I < coarse->nn; I++) {
        int XYZ[3], pos[3][2], npt[3];
        double wt[3][2];
        node_xyz(coarse, I, &XYZ[0], &XYZ[1], &XYZ[2]);
        for (int a = 0; a < 3; a++) {
            if (2 * XYZ[a] < fd[a]) {
                npt[a] = 1;
                pos[a][0] = 2 * XYZ[a];
                wt[a][0] = 1.0;
            } else {
                npt[a] = 2;
                pos[a][0] = fd[a] - 1;
                wt[a][0] = 2.0;
                pos[a][1] = fd[a] - 2;
                wt[a][1] = -1.0;
            }
        }
        double acc[3] = {0, 0, 0};
        for (int kx = 0; kx < npt[0]; kx++)
            for (int ky = 0; ky < npt[1]; ky++)
                for (int kz = 0; kz < npt[2]; kz++) {
                    int i = node_id(fine, pos[0][kx], pos[1][ky], pos[2][kz]);
                    double w = wt[0][kx] * wt[1][ky] * wt[2][kz];
                    for (int a = 0; a < 3; a++) acc[a] += w * fine->u[3 * i + a];
                }
        memcpy(coarse->u + 3 * I, acc, 3 * sizeof(double));
        int i0 = node_id(fine, pos[0][0], pos[1][0], pos[2][0]);
        memcpy(coarse->R + 9 * I, fine->R + 9 * i0, 9 * sizeof(double));
    }
    coarse->have_J = 0;
}

/* Jump start of the finer level from the coarse solution: every finer node i adds the
 * coarse level's displacement increment (u - u_start) interpolated trilinearly at its
 * canonical position, which lies at coarse coordinates (x/2, y/2, z/2). */
void vdo_prolongate(const vdo_ctx *coarse, const double *u_start, vdo_ctx *fine)
{
    int cd[3] = {coarse->nx, coarse->ny, coarse->nz};
    for (int i = 0; i < fine->nn; i++) {
        int xyz[3], ci[3];
        double f[3], al[8], acc[3] = {0, 0, 0};
        int nd[8];
        node_xyz(fine, i, &xyz[0], &xyz[1], &xyz[2]);
        for (int a = 0; a < 3; a++) {
            ci[a] = xyz[a] / 2 < cd[a] - 2 ? xyz[a] / 2 : cd[a] - 2;
            f[a] = 0.5 * xyz[a] - ci[a];
        }
        corners(coarse, node_id(coarse, ci[0], ci[1], ci[2]), f, nd, al);
        for (int k = 0; k < 8; k++)
            for (int a = 0; a < 3; a++) acc[a] += al[k] * (coarse->u[3 * nd[k] + a] - u_start[3 * nd[k] + a]);
        for (int a = 0; a < 3; a++) fine->u[3 * i + a] += acc[a];
    }
    fine->have_J = 0;
}

/* ------------------------------------------------------------------ global rigid pose (Sec. 6) */

void vdo_set_pose(vdo_ctx *c, const double *pose)
{
    for (int a = 0; a < 9; a++) c->Rg[a] = pose[a];
    for (int a = 0; a < 3; a++) c->tg[a] = pose[9 + a];
    c->have_J = 0;
}

void vdo_get_pose(const vdo_ctx *c, double *pose)
{
    for (int a = 0; a < 9; a++) pose[a] = c->Rg[a];
    for (int a = 0; a < 3; a++) pose[9 + a] = c->tg[a];
}

/* Normal equations of dense projective ICP for the global pose at the current pose and
 * association: over the samples with w_c > 0, with q = sum_k alpha_k t_k (the lattice
 * warp of the sample, before the pose), p = R_g q + t_g, residual r = n^a . (p - p^a)
 * and its derivative J = ((R_g q) x n^a, n^a) for the pose perturbed as
 * R_g <- exp([omega]x) R_g, t_g <- t_g + tau:
 *   A = sum w_c J J^T (6 x 6, row-major), b = sum w_c J r, E = sum w_c r^2.
 * Returns the number of samples used. */
int vdo_icp_system(const vdo_ctx *c, double A[36], double b[6], double *E)
{
    int n = 0;
    memset(A, 0, 36 * sizeof(double));
    memset(b, 0, 6 * sizeof(double));
    *E = 0.0;
    int nd[8];
    double al[8];
    for (int s = 0; s < c->C; s++) {
        if (!(c->wc[s] > 0)) continue;
        double q[3] = {0, 0, 0}, tk[3], Rq[3];
        corners(c, c->cell_c[s], c->frac_c + 3 * s, nd, al);
        for (int k = 0; k < 8; k++) {
            node_pos(c, nd[k], tk);
            for (int a = 0; a < 3; a++) q[a] += al[k] * (tk[a] + c->u[3 * nd[k] + a]);
        }
        matvec3(c->Rg, q, Rq);
        const double *pa = c->pa + 3 * s, *na = c->na + 3 * s;
        double d[3] = {Rq[0] + c->tg[0] - pa[0], Rq[1] + c->tg[1] - pa[1], Rq[2] + c->tg[2] - pa[2]};
        double r = dot3(na, d), J[6];
        cross3(Rq, na, J);
        for (int a = 0; a < 3; a++) J[3 + a] = na[a];
        for (int i = 0; i < 6; i++) {
            b[i] += c->wc[s] * J[i] * r;
            for (int j = 0; j < 6; j++) A[6 * i + j] += c->wc[s] * J[i] * J[j];
        }
        *E += c->wc[s] * r * r;
        n++;
    }
    return n;
}

/* Dense projective ICP (Sec. 6): `iters` Gauss-Newton steps on the pose, each after a
 * projective association at the current pose (Sec. 5.1); the step solves A xi = -b by
 * Cholesky and applies R_g <- exp([omega]x) R_g (Rodrigues), t_g <- t_g + tau.  Stops
 * early when A is not positive definite.  Returns the steps taken; e_hist (iters
 * entries, may be NULL) gets E before each step. */
int vdo_icp(vdo_ctx *c, int iters, double *e_hist)
{
    int it = 0;
    for (; it < iters; it++) {
        vdo_associate(c);
        double A[36], b[6], E;
        vdo_icp_system(c, A, b, &E);
        if (e_hist) e_hist[it] = E;
        double L[36] = {0}, y[6], xi[6];
        int bad = 0;
        for (int j = 0; j < 6 && !bad; j++) {
            double sj = A[6 * j + j];
            for (int k = 0; k < j; k++) sj -= L[6 * j + k] * L[6 * j + k];
            if (!(sj > 0)) { bad = 1; break; }
            L[6 * j + j] = sqrt(sj);
            for (int i = j + 1; i < 6; i++) {
                double t = A[6 * i + j];
                for (int k = 0; k < j; k++) t -= L[6 * i + k] * L[6 * j + k];
                L[6 * i + j] = t / L[6 * j + j];
            }
        }
        if (bad) break;
        for (int i = 0; i < 6; i++) {               /* L y = -b */
            double t = -b[i];
            for (int k = 0; k < i; k++) t -= L[6 * i + k] * y[k];
            y[i] = t / L[6 * i + i];
        }
        for (int i = 5; i >= 0; i--) {              /* L^T xi = y */
            double t = y[i];
            for (int k = i + 1; k < 6; k++) t -= L[6 * k + i] * xi[k];
            xi[i] = t / L[6 * i + i];
        }
        double th = sqrt(dot3(xi, xi)), E3[9], Rn[9];
        double K[9] = {0, -xi[2], xi[1], xi[2], 0, -xi[0], -xi[1], xi[0], 0};
        double s1 = th > 0 ? sin(th) / th : 1.0, s2 = th > 0 ? (1.0 - cos(th)) / (th * th) : 0.5;
        for (int r = 0; r < 3; r++)
            for (int q = 0; q < 3; q++) {
                double KK = K[3 * r] * K[q] + K[3 * r + 1] * K[3 + q] + K[3 * r + 2] * K[6 + q];
                E3[3 * r + q] = (r == q ? 1.0 : 0.0) + s1 * K[3 * r + q] + s2 * KK;
            }
        for (int r = 0; r < 3; r++)
            for (int q = 0; q < 3; q++)
                Rn[3 * r + q] = E3[3 * r] * c->Rg[q] + E3[3 * r + 1] * c->Rg[3 + q] + E3[3 * r + 2] * c->Rg[6 + q];
        memcpy(c->Rg, Rn, sizeof(Rn));
        for (int a = 0; a < 3; a++) c->tg[a] += xi[3 + a];
        c->have_J = 0;
    }
    return it;
}

/* ------------------------------------------------------------------ source samples (Sec. 4, 5.1) */

/* Marching cubes case table, generated from the rule (the paper's Sec. 4 extracts the
 * canonical isosurface by data-parallel marching cubes; no table is printed there):
 *   corner k of a cell sits at (k & 1, (k >> 1) & 1, (k >> 2) & 1) and is inside when its
 *   value is below the iso value; edge e joins corners (a, b), a < b:
 *     x-edges 0..3 = (0,1) (2,3) (4,5) (6,7), y-edges 4..7 = (0,2) (1,3) (4,6) (5,7),
 *     z-edges 8..11 = (0,4) (1,5) (2,6) (3,7);
 *   on each face, walking its corners counter-clockwise as seen from outside the cell,
 *   an edge crossed from outside to inside starts a segment that ends at the next
 *   crossed edge of the walk (so diagonal inside corners of a face are separated, the
 *   same way from both cells that share the face);
 *   every crossed edge starts one segment and ends one, so the segments form loops; a
 *   loop is started at its lowest edge, loops are taken in the order of their lowest
 *   edge, and each is cut into the fan (v0, v_i, v_i+1).  The loops wind counter-
 *   clockwise seen from outside the surface (the side above the iso value). */
static int mc_tab[256][31];   /* [0] = triangles, then 3 edges per triangle */
static int mc_ready = 0;

static void mc_build(void)
{
    static const int E[12][2] = {{0, 1}, {2, 3}, {4, 5}, {6, 7}, {0, 2}, {1, 3}, {4, 6}, {5, 7},
                                 {0, 4}, {1, 5}, {2, 6}, {3, 7}};
    int cyc[6][4];
    for (int A = 0; A < 3; A++) {
        int B = (A + 1) % 3, C = (A + 2) % 3;
        for (int sgn = 0; sgn < 2; sgn++) {
            int q[4][2] = {{0, 0}, {1, 0}, {1, 1}, {0, 1}};   /* (B, C) counter-clockwise about +A */
            for (int i = 0; i < 4; i++) {
                int j = sgn ? i : (4 - i) % 4;                  /* outward -A: walk backwards */
                int k = (sgn << A) | (q[j][0] << B) | (q[j][1] << C);
                cyc[2 * A + sgn][i] = k;
            }
        }
    }
    for (int cs = 0; cs < 256; cs++) {
        int next[12];
        for (int e = 0; e < 12; e++) next[e] = -1;
        for (int f = 0; f < 6; f++) {
            int ce[4], kind[4];          /* edge of each cycle step, +1 entry, -1 exit, 0 none */
            for (int i = 0; i < 4; i++) {
                int a = cyc[f][i], b = cyc[f][(i + 1) % 4];
                int lo = a < b ? a : b, hi = a < b ? b : a;
                for (int e = 0; e < 12; e++)
                    if (E[e][0] == lo && E[e][1] == hi) ce[i] = e;
                int ina = (cs >> a) & 1, inb = (cs >> b) & 1;
                kind[i] = ina == inb ? 0 : (inb ? 1 : -1);
            }
            for (int i = 0; i < 4; i++) {
                if (kind[i] != 1) continue;
                for (int d = 1; d < 4; d++)
                    if (kind[(i + d) % 4] != 0) { next[ce[i]] = ce[(i + d) % 4]; break; }
            }
        }
        int used[12] = {0}, nt = 0;
        for (int e0 = 0; e0 < 12; e0++) {
            if (next[e0] < 0 || used[e0]) continue;
            int loop[12], m = 0, e = e0;
            do { loop[m++] = e; used[e] = 1; e = next[e]; } while (e != e0 && m < 12);
            for (int i = 1; i + 1 < m; i++) {
                mc_tab[cs][1 + 3 * nt] = loop[0];
                mc_tab[cs][2 + 3 * nt] = loop[i];
                mc_tab[cs][3 + 3 * nt] = loop[i + 1];
                nt++;
            }
        }
        mc_tab[cs][0] = nt;
    }
    mc_ready = 1;
}

int vdo_mc_case(int cs, int *edges)
{
    if (!mc_ready) mc_build();
    for (int i = 0; i < 3 * mc_tab[cs][0]; i++) edges[i] = mc_tab[cs][1 + i];
    return mc_tab[cs][0];
}

static double grid_at(const float *g, int sx, int sy, int x, int y, int z)
{
    return (double)g[(size_t)x + (size_t)sx * ((size_t)y + (size_t)sy * z)];
}

/* SDF gradient at grid point (x, y, z): central differences, one-sided at the border */
static void grid_grad(const float *g, int sx, int sy, int sz, double hs, int x, int y, int z, double out[3])
{
    int n[3] = {sx, sy, sz}, p[3] = {x, y, z};
    for (int a = 0; a < 3; a++) {
        int lo[3] = {x, y, z}, hi[3] = {x, y, z};
        lo[a] = p[a] > 0 ? p[a] - 1 : p[a];
        hi[a] = p[a] + 1 < n[a] ? p[a] + 1 : p[a];
        double d = grid_at(g, sx, sy, hi[0], hi[1], hi[2]) - grid_at(g, sx, sy, lo[0], lo[1], lo[2]);
        out[a] = d / ((hi[a] - lo[a]) * hs);
    }
}

/* Marching cubes over a (sx, sy, sz) grid of values g (x fastest) at origin o, spacing hs:
 * the triangles in cell order (cell x fastest), in the table's order within a cell.  A
 * vertex on edge (a, b) sits at p_a + t (p_b - p_a), t = (iso - g_a) / (g_b - g_a); its
 * normal is the SDF gradient interpolated the same way, normalised.  Writes up to cap
 * triangles (9 position and 9 normal doubles each; either may be NULL) and returns the
 * number of triangles of the whole surface. */
long vdo_marching_cubes(const float *g, int sx, int sy, int sz, const double o[3], double hs, double iso,
                        double *tri, double *nrm, long cap)
{
    if (!mc_ready) mc_build();
    static const int E[12][2] = {{0, 1}, {2, 3}, {4, 5}, {6, 7}, {0, 2}, {1, 3}, {4, 6}, {5, 7},
                                 {0, 4}, {1, 5}, {2, 6}, {3, 7}};
    long n = 0;
    for (int z = 0; z + 1 < sz; z++)
        for (int y = 0; y + 1 < sy; y++)
            for (int x = 0; x + 1 < sx; x++) {
                double v[8];
                int cs = 0;
                for (int k = 0; k < 8; k++) {
                    v[k] = grid_at(g, sx, sy, x + (k & 1), y + ((k >> 1) & 1), z + ((k >> 2) & 1));
                    if (v[k] < iso) cs |= 1 << k;
                }
                for (int t = 0; t < mc_tab[cs][0]; t++, n++) {
                    if (n >= cap) continue;
                    for (int j = 0; j < 3; j++) {
                        int e = mc_tab[cs][1 + 3 * t + j], a = E[e][0], b = E[e][1];
                        double w = (iso - v[a]) / (v[b] - v[a]);
                        int pa[3] = {x + (a & 1), y + ((a >> 1) & 1), z + ((a >> 2) & 1)};
                        int pb[3] = {x + (b & 1), y + ((b >> 1) & 1), z + ((b >> 2) & 1)};
                        double ga[3], gb[3], nn[3], L = 0;
                        grid_grad(g, sx, sy, sz, hs, pa[0], pa[1], pa[2], ga);
                        grid_grad(g, sx, sy, sz, hs, pb[0], pb[1], pb[2], gb);
                        for (int c = 0; c < 3; c++) {
                            double qa = o[c] + hs * pa[c], qb = o[c] + hs * pb[c];
                            if (tri) tri[9 * n + 3 * j + c] = qa + w * (qb - qa);
                            nn[c] = ga[c] + w * (gb[c] - ga[c]);
                            L += nn[c] * nn[c];
                        }
                        L = sqrt(L);
                        if (nrm)
                            for (int c = 0; c < 3; c++) nrm[9 * n + 3 * j + c] = L > 0 ? nn[c] / L : 0.0;
                    }
                }
            }
    return n;
}

/* Rasterise the deformed mesh (Sec. 5.1: "rasterize the resulting mesh to obtain sample
 * points S(p^_c)").  Each vertex p^ is deformed by the lattice warp and the pose,
 * S(p^) = R_g (p^ + sum alpha_k u_k) + t_g (u = 0 outside the lattice), and projected,
 * (f_x X / Z + c_x, f_y Y / Z + c_y), pixel centres at integer coordinates.  A pixel is
 * covered by a triangle (all vertices with Z > 1e-3, non-zero screen area) when its
 * centre has all three barycentric coordinates >= 0; among the covering triangles the
 * one with the smallest depth Z = 1 / sum(lambda_i / Z_i) wins, ties to the lower
 * triangle index.  Its sample is the perspective-correct interpolation of the canonical
 * vertices, b_i = (lambda_i / Z_i) / sum_j (lambda_j / Z_j): p^ = sum b_i p^_i, n^ =
 * normalise(sum b_i n^_i).  Writes per pixel (H x W): winning triangle (-1 if none),
 * depth, canonical point and normal (any may be NULL), and the pixel's margin (the
 * smallest screen distance, in pixels, from its centre to an edge of the winner, or
 * to the depth of a runner-up scaled by f_x / Z: small values mark decisions that
 * rounding may take either way).  Returns the number of covered pixels. */
long vdo_render_samples(const vdo_ctx *c, const double *tri, const double *nrm, long ntri, int W, int H,
                        const double K[4], const double pose[12], int *win, double *depth, double *cp,
                        double *cn, double *margin)
{
    size_t np = (size_t)W * H;
    int *best = (int *)xcalloc(np, sizeof(int));
    double *bz = (double *)xcalloc(np, sizeof(double));
    double *second = (double *)xcalloc(np, sizeof(double));
    double *emin = (double *)xcalloc(np, sizeof(double));
    double *bw = (double *)xcalloc(np * 3, sizeof(double));
    for (size_t k = 0; k < np; k++) { best[k] = -1; bz[k] = 1e300; second[k] = 1e300; }
    double *P = (double *)xcalloc((size_t)ntri * 9, sizeof(double));
    for (long t = 0; t < ntri; t++)
        for (int j = 0; j < 3; j++) {
            const double *q = tri + 9 * t + 3 * j;
            double f[3], acc[3] = {q[0], q[1], q[2]}, out[3];
            int cell = locate(c, q, f);
            if (cell >= 0) {
                int nd[8];
                double al[8];
                corners(c, cell, f, nd, al);
                for (int k = 0; k < 8; k++)
                    for (int a = 0; a < 3; a++) acc[a] += al[k] * c->u[3 * nd[k] + a];
            }
            matvec3(pose, acc, out);
            for (int a = 0; a < 3; a++) P[9 * t + 3 * j + a] = out[a] + pose[9 + a];
        }
    for (long t = 0; t < ntri; t++) {
        double X[3], Y[3], Z[3];
        int ok = 1;
        for (int j = 0; j < 3; j++) {
            Z[j] = P[9 * t + 3 * j + 2];
            if (!(Z[j] > 1e-3)) ok = 0;
            X[j] = K[0] * P[9 * t + 3 * j] / Z[j] + K[2];
            Y[j] = K[1] * P[9 * t + 3 * j + 1] / Z[j] + K[3];
        }
        if (!ok) continue;
        double area = (X[1] - X[0]) * (Y[2] - Y[0]) - (X[2] - X[0]) * (Y[1] - Y[0]);
        if (area == 0.0) continue;
        double xmin = fmin(X[0], fmin(X[1], X[2])), xmax = fmax(X[0], fmax(X[1], X[2]));
        double ymin = fmin(Y[0], fmin(Y[1], Y[2])), ymax = fmax(Y[0], fmax(Y[1], Y[2]));
        int u0 = (int)ceil(xmin), u1 = (int)floor(xmax), v0 = (int)ceil(ymin), v1 = (int)floor(ymax);
        if (u0 < 0) u0 = 0;
        if (v0 < 0) v0 = 0;
        if (u1 > W - 1) u1 = W - 1;
        if (v1 > H - 1) v1 = H - 1;
        for (int v = v0; v <= v1; v++)
            for (int u = u0; u <= u1; u++) {
                double l[3], el[3];
                for (int j = 0; j < 3; j++) {
                    int a = (j + 1) % 3, b = (j + 2) % 3;
                    double e = (X[b] - X[a]) * (v - Y[a]) - (Y[b] - Y[a]) * (u - X[a]);
                    l[j] = e / area;
                    double len = sqrt((X[b] - X[a]) * (X[b] - X[a]) + (Y[b] - Y[a]) * (Y[b] - Y[a]));
                    el[j] = len > 0 ? fabs(e) / len : 0.0;
                }
                if (l[0] < 0 || l[1] < 0 || l[2] < 0) continue;
                double s = l[0] / Z[0] + l[1] / Z[1] + l[2] / Z[2], zz = 1.0 / s;
                size_t k = (size_t)v * W + u;
                if (zz < bz[k] || (zz == bz[k] && t < best[k])) {
                    second[k] = bz[k];
                    bz[k] = zz;
                    best[k] = (int)t;
                    emin[k] = fmin(el[0], fmin(el[1], el[2]));
                    for (int j = 0; j < 3; j++) bw[3 * k + j] = (l[j] / Z[j]) / s;
                } else if (zz < second[k]) {
                    second[k] = zz;
                }
            }
    }
    long cnt = 0;
    for (size_t k = 0; k < np; k++) {
        if (win) win[k] = best[k];
        if (depth) depth[k] = best[k] >= 0 ? bz[k] : 0.0;
        if (margin) margin[k] = best[k] >= 0 ? fmin(emin[k], second[k] < 1e299 ? (second[k] - bz[k]) * K[0] / bz[k] : 1e300) : 0.0;
        if (best[k] < 0) {
            if (cp) cp[3 * k] = cp[3 * k + 1] = cp[3 * k + 2] = 0.0;
            if (cn) cn[3 * k] = cn[3 * k + 1] = cn[3 * k + 2] = 0.0;
            continue;
        }
        cnt++;
        long t = best[k];
        double q[3] = {0, 0, 0}, m[3] = {0, 0, 0}, L = 0;
        for (int j = 0; j < 3; j++)
            for (int a = 0; a < 3; a++) {
                q[a] += bw[3 * k + j] * tri[9 * t + 3 * j + a];
                m[a] += bw[3 * k + j] * nrm[9 * t + 3 * j + a];
            }
        for (int a = 0; a < 3; a++) L += m[a] * m[a];
        L = sqrt(L);
        for (int a = 0; a < 3; a++) {
            if (cp) cp[3 * k + a] = q[a];
            if (cn) cn[3 * k + a] = L > 0 ? m[a] / L : 0.0;
        }
    }
    free(best); free(bz); free(second); free(emin); free(bw); free(P);
    return cnt;
}
