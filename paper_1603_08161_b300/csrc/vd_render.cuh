// Source samples on the GPU (Sec. 4 and 5.1): data-parallel marching cubes of a signed
// distance grid with prefix-sum compaction, deformation of the mesh vertices by the
// lattice warp and the global pose, and a z-buffer rasteriser whose covered pixels give
// the canonical sample points p^_c and normals n^_c of the frame.
//
// Included by vd_api.cu after the lattice type and the scan helpers (one translation
// unit holds every kernel of the library's solve path).
#pragma once

namespace vd {

// ------------------------------------------------------------------ marching cubes table
//
// The case table is generated on the host from the rule (no table is printed in the
// paper, and none is copied here):
//   * corner k of a cell is at (k & 1, (k >> 1) & 1, (k >> 2) & 1) and is inside when
//     its value is below the iso value;
//   * the edge parallel to axis A whose lower corner has the other two coordinates
//     (b, c) (in increasing axis order) is edge 4 A + b + 2 c;
//   * on each face, walking its corners counter-clockwise as seen from outside the
//     cell, an edge crossed from outside to inside opens a segment that closes at the
//     next crossed edge of the walk;
//   * the segments form loops (every crossed edge opens one and closes one); each loop
//     starts at its lowest edge, loops are taken in the order of their lowest edges, and
//     a loop v0 v1 ... v(m-1) gives the triangles (v0, v_i, v_i+1).
constexpr int kMcMaxTri = 10;             // at most 12 crossed edges: 12 - 2 triangles
constexpr int kMcRow = 1 + 3 * kMcMaxTri; // count, then three edges per triangle

struct McTable {
    int t[256][kMcRow];
};

inline McTable mc_make_table() {
    McTable T{};
    auto edge_id = [](int a, int b) {      // corners a < b differing in one bit
        const int d = a ^ b, A = d == 1 ? 0 : (d == 2 ? 1 : 2);
        int rest = 0, sh = 0;
        for (int ax = 0; ax < 3; ax++)
            if (ax != A) rest |= ((a >> ax) & 1) << sh++;
        return 4 * A + rest;
    };
    for (int cs = 0; cs < 256; cs++) {
        int closes[12];
        for (int e = 0; e < 12; e++) closes[e] = -1;
        for (int A = 0; A < 3; A++) {
            const int B = (A + 1) % 3, C = (A + 2) % 3;
            for (int side = 0; side < 2; side++) {
                // counter-clockwise about the outward normal: +A for side 1, -A for side 0
                static const int ccw[4][2] = {{0, 0}, {1, 0}, {1, 1}, {0, 1}};
                int corner[4];
                for (int i = 0; i < 4; i++) {
                    const int *q = ccw[side ? i : (4 - i) & 3];
                    corner[i] = (side << A) | (q[0] << B) | (q[1] << C);
                }
                int e[4], opens[4], crossed[4];
                for (int i = 0; i < 4; i++) {
                    const int a = corner[i], b = corner[(i + 1) & 3];
                    e[i] = edge_id(a < b ? a : b, a < b ? b : a);
                    const bool ia = (cs >> a) & 1, ib = (cs >> b) & 1;
                    crossed[i] = ia != ib;
                    opens[i] = crossed[i] && ib;  // outside -> inside along the walk
                }
                for (int i = 0; i < 4; i++) {
                    if (!opens[i]) continue;
                    int j = (i + 1) & 3;
                    while (!crossed[j]) j = (j + 1) & 3;
                    closes[e[i]] = e[j];
                }
            }
        }
        bool seen[12] = {};
        int nt = 0;
        for (int e0 = 0; e0 < 12; e0++) {
            if (closes[e0] < 0 || seen[e0]) continue;
            std::vector<int> loop;
            for (int e = e0; !seen[e]; e = closes[e]) {
                seen[e] = true;
                loop.push_back(e);
            }
            for (size_t i = 1; i + 1 < loop.size(); i++) {
                T.t[cs][1 + 3 * nt] = loop[0];
                T.t[cs][2 + 3 * nt] = (int)loop[i];
                T.t[cs][3 + 3 * nt] = (int)loop[i + 1];
                nt++;
            }
        }
        T.t[cs][0] = nt;
    }
    return T;
}

// ------------------------------------------------------------------ kernels

struct Grid3 {
    const float *g;  // values, x fastest
    int sx, sy, sz;
    float ox, oy, oz, hs, iso;
};

__device__ __forceinline__ float g_at(const Grid3 &G, int x, int y, int z) {
    return G.g[(size_t)x + (size_t)G.sx * ((size_t)y + (size_t)G.sy * z)];
}

__device__ __forceinline__ int mc_case_of(const Grid3 &G, int x, int y, int z, float v[8]) {
    int cs = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) {
        v[k] = g_at(G, x + (k & 1), y + ((k >> 1) & 1), z + ((k >> 2) & 1));
        if (v[k] < G.iso) cs |= 1 << k;
    }
    return cs;
}

// triangles of every cell (cell x fastest)
__global__ void k_mc_count(Grid3 G, const int *__restrict__ tab, int *__restrict__ cnt) {
    const int cx = G.sx - 1, cy = G.sy - 1, ncell = cx * cy * (G.sz - 1);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ncell; i += gridDim.x * blockDim.x) {
        const int x = i % cx, t = i / cx, y = t % cy, z = t / cy;
        float v[8];
        cnt[i] = tab[kMcRow * mc_case_of(G, x, y, z, v)];
    }
}

// SDF gradient at a grid point: central differences, one-sided at the border
__device__ __forceinline__ void g_grad(const Grid3 &G, int x, int y, int z, float out[3]) {
    const int p[3] = {x, y, z}, n[3] = {G.sx, G.sy, G.sz};
#pragma unroll
    for (int a = 0; a < 3; a++) {
        int lo[3] = {x, y, z}, hi[3] = {x, y, z};
        lo[a] = p[a] > 0 ? p[a] - 1 : p[a];
        hi[a] = p[a] + 1 < n[a] ? p[a] + 1 : p[a];
        out[a] = (g_at(G, hi[0], hi[1], hi[2]) - g_at(G, lo[0], lo[1], lo[2])) / ((float)(hi[a] - lo[a]) * G.hs);
    }
}

// the cells' triangles at their offsets: vertex at p_a + t (p_b - p_a), t = (iso - g_a) /
// (g_b - g_a) along the edge from its lower corner, normal = the gradient interpolated
// the same way, normalised; nothing past `cap`
__global__ void k_mc_emit(Grid3 G, const int *__restrict__ tab, const int *__restrict__ off, int cap,
                          float *__restrict__ tri, float *__restrict__ nrm) {
    const int cx = G.sx - 1, cy = G.sy - 1, ncell = cx * cy * (G.sz - 1);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ncell; i += gridDim.x * blockDim.x) {
        const int x = i % cx, t = i / cx, y = t % cy, z = t / cy;
        float v[8];
        const int *row = tab + kMcRow * mc_case_of(G, x, y, z, v);
        for (int k = 0; k < row[0]; k++) {
            const int o = off[i] + k;
            if (o >= cap) break;
#pragma unroll
            for (int j = 0; j < 3; j++) {
                const int e = row[1 + 3 * k + j], A = e >> 2, rest = e & 3;
                // lower corner: bit A clear, the other two bits from `rest` in axis order
                const int B = A == 0 ? 1 : 0, C = A == 2 ? 1 : 2;
                const int ca = (((rest & 1) << B) | (((rest >> 1) & 1) << C)), cb = ca | (1 << A);
                const int pa[3] = {x + (ca & 1), y + ((ca >> 1) & 1), z + ((ca >> 2) & 1)};
                const int pb[3] = {x + (cb & 1), y + ((cb >> 1) & 1), z + ((cb >> 2) & 1)};
                const float w = (G.iso - v[ca]) / (v[cb] - v[ca]);
                float ga[3], gb[3], nn[3];
                g_grad(G, pa[0], pa[1], pa[2], ga);
                g_grad(G, pb[0], pb[1], pb[2], gb);
                const float org[3] = {G.ox, G.oy, G.oz};
                float L2 = 0.f;
#pragma unroll
                for (int a = 0; a < 3; a++) {
                    const float qa = org[a] + G.hs * pa[a], qb = org[a] + G.hs * pb[a];
                    tri[9 * (size_t)o + 3 * j + a] = qa + w * (qb - qa);
                    nn[a] = ga[a] + w * (gb[a] - ga[a]);
                    L2 += nn[a] * nn[a];
                }
                const float iL = L2 > 0.f ? rsqrtf(L2) : 0.f;
#pragma unroll
                for (int a = 0; a < 3; a++) nrm[9 * (size_t)o + 3 * j + a] = nn[a] * iL;
            }
        }
    }
}

// S(p^) = R_g (p^ + sum alpha_k u_k) + t_g for every vertex (u = 0 outside the lattice;
// the cell decision in FP64 as for the samples); c = nullptr-free lattice context, or
// has_lat = 0 for the identity warp
__global__ void k_mesh_deform(Ctx c, int has_lat, const float *__restrict__ tri, int nv, const float *__restrict__ pose,
                              float *__restrict__ out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += gridDim.x * blockDim.x) {
        float q[3] = {tri[3 * i], tri[3 * i + 1], tri[3 * i + 2]};
        if (has_lat) {
            const double o[3] = {(double)c.ox, (double)c.oy, (double)c.oz};
            const int dims[3] = {c.nx, c.ny, c.nz};
            float f[3];
            int ci[3];
            bool ok = true;
#pragma unroll
            for (int a = 0; a < 3; a++) {
                const double s = __ddiv_rn(__dsub_rn((double)q[a], o[a]), (double)c.h);
                const double fl = floor(s);
                if (!(fl >= 0.0) || fl > (double)(dims[a] - 2)) ok = false;
                ci[a] = ok ? (int)fl : 0;
                f[a] = (float)(s - fl);
            }
            if (ok) {
                const int cell = ci[0] + c.nx * (ci[1] + c.ny * ci[2]);
                float du[3] = {0.f, 0.f, 0.f};
#pragma unroll
                for (int k = 0; k < 8; k++) {
                    const int nd = corner_node(c, cell, k);
                    const float al = trilinear_weight(f, k);
#pragma unroll
                    for (int a = 0; a < 3; a++) du[a] += al * c.u[a * c.ld + nd];
                }
#pragma unroll
                for (int a = 0; a < 3; a++) q[a] += du[a];
            }
        }
#pragma unroll
        for (int r = 0; r < 3; r++)
            out[3 * i + r] = pose[3 * r] * q[0] + pose[3 * r + 1] * q[1] + pose[3 * r + 2] * q[2] + pose[9 + r];
    }
}

__global__ void k_zbuf_clear(unsigned long long *__restrict__ z, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) z[i] = ~0ull;
}

struct Cam {
    int W, H;
    float fx, fy, cx, cy;
};

// screen position of a camera-frame point
__device__ __forceinline__ void project(const Cam &k, const float *P, float &X, float &Y) {
    X = k.fx * P[0] / P[2] + k.cx;
    Y = k.fy * P[1] / P[2] + k.cy;
}

// barycentric coordinates of pixel centre (u, v) in a screen triangle; false when the
// area is 0
__device__ __forceinline__ bool bary(const float X[3], const float Y[3], float u, float v, float l[3]) {
    const float area = (X[1] - X[0]) * (Y[2] - Y[0]) - (X[2] - X[0]) * (Y[1] - Y[0]);
    if (area == 0.f) return false;
#pragma unroll
    for (int j = 0; j < 3; j++) {
        const int a = (j + 1) % 3, b = (j + 2) % 3;
        l[j] = ((X[b] - X[a]) * (v - Y[a]) - (Y[b] - Y[a]) * (u - X[a])) / area;
    }
    return true;
}

// one thread per triangle: every pixel centre with all barycentric coordinates >= 0
// takes min(depth, triangle) in the 64-bit z-buffer (depth bits above the index: a
// positive float orders like its bit pattern); triangles with a vertex at Z <= 1e-3
// are skipped
__global__ void k_raster(const float *__restrict__ P, int ntri, Cam k, unsigned long long *__restrict__ zbuf) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < ntri; t += gridDim.x * blockDim.x) {
        const float *p = P + 9 * (size_t)t;
        if (!(p[2] > 1e-3f && p[5] > 1e-3f && p[8] > 1e-3f)) continue;
        float X[3], Y[3];
#pragma unroll
        for (int j = 0; j < 3; j++) project(k, p + 3 * j, X[j], Y[j]);
        const int u0 = max(0, (int)ceilf(fminf(X[0], fminf(X[1], X[2]))));
        const int u1 = min(k.W - 1, (int)floorf(fmaxf(X[0], fmaxf(X[1], X[2]))));
        const int v0 = max(0, (int)ceilf(fminf(Y[0], fminf(Y[1], Y[2]))));
        const int v1 = min(k.H - 1, (int)floorf(fmaxf(Y[0], fmaxf(Y[1], Y[2]))));
        for (int v = v0; v <= v1; v++)
            for (int u = u0; u <= u1; u++) {
                float l[3];
                if (!bary(X, Y, (float)u, (float)v, l) || l[0] < 0.f || l[1] < 0.f || l[2] < 0.f) continue;
                const float zz = 1.f / (l[0] / p[2] + l[1] / p[5] + l[2] / p[8]);
                const unsigned long long key = ((unsigned long long)__float_as_uint(zz) << 32) | (unsigned)t;
                atomicMin(&zbuf[(size_t)v * k.W + u], key);
            }
    }
}

// per sampled pixel (every stride-th in x and y): 1 if a triangle won it
__global__ void k_zbuf_flags(const unsigned long long *__restrict__ zbuf, Cam k, int stride, int *__restrict__ flag) {
    const int n = k.W * k.H;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const int u = i % k.W, v = i / k.W;
        flag[i] = (u % stride == 0 && v % stride == 0 && zbuf[i] != ~0ull) ? 1 : 0;
    }
}

// the winners' canonical points and normals (perspective-correct interpolation of the
// canonical vertices, b_i = (lambda_i / Z_i) / sum_j lambda_j / Z_j), compacted in pixel
// order at the scanned offsets (nothing past `cap`)
__global__ void k_resolve(const unsigned long long *__restrict__ zbuf, const int *__restrict__ flag,
                          const int *__restrict__ off, const float *__restrict__ P, const float *__restrict__ tri,
                          const float *__restrict__ nrm, Cam k, int cap, float *__restrict__ out_p,
                          float *__restrict__ out_n, int *__restrict__ out_pix) {
    const int n = k.W * k.H;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        if (!flag[i]) continue;
        const int o = off[i];
        if (o >= cap) continue;
        const int t = (int)(zbuf[i] & 0xffffffffull);
        const float *p = P + 9 * (size_t)t;
        float X[3], Y[3], l[3];
#pragma unroll
        for (int j = 0; j < 3; j++) project(k, p + 3 * j, X[j], Y[j]);
        bary(X, Y, (float)(i % k.W), (float)(i / k.W), l);
        float w[3], s = 0.f;
#pragma unroll
        for (int j = 0; j < 3; j++) {
            w[j] = l[j] / p[3 * j + 2];
            s += w[j];
        }
        float q[3] = {0.f, 0.f, 0.f}, m[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int j = 0; j < 3; j++) {
            const float b = w[j] / s;
#pragma unroll
            for (int a = 0; a < 3; a++) {
                q[a] += b * tri[9 * (size_t)t + 3 * j + a];
                m[a] += b * nrm[9 * (size_t)t + 3 * j + a];
            }
        }
        const float L2 = m[0] * m[0] + m[1] * m[1] + m[2] * m[2], iL = L2 > 0.f ? rsqrtf(L2) : 0.f;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            out_p[3 * (size_t)o + a] = q[a];
            out_n[3 * (size_t)o + a] = m[a] * iL;
        }
        if (out_pix) out_pix[o] = i;
    }
}

}  // namespace vd
