// Near field of the Nystrom discretisation (Sec. 6.1.1, 6.1.2): structure,
// float64 quadrature weights, coefficient combination and the correction SpMV.
//
// For a target i and a near patch P (the target's own patch or any patch
// whose centroid is closer than near_factor * radius, Sec. 6.1.2) the library
// stores three coefficient-independent weight sets, for k in P:
//
//   W_lb[ik]  = int_P (q^2 - H_i q)/pi          l_k(u,v) J~(u,v) du dv,  q = n.r/|r|^2
//   W_g[c,ik] = int_P r_c / (2 pi |r|^2)        l_k(u,v) J~(u,v) du dv   (c = x, y, z)
//   W_k[ik]   = int_P log|r| / (2 pi)           l_k(u,v) J~(u,v) du dv
//
// with r = x_i - y~(u,v), y~ and J~ the tensor interpolants of the patch's
// node positions and |y_u x y_v|, and l_k the tensor Lagrange basis.  Since
// a(x') enters R and K only as 1/a(x') and a(x_i), grad a(x_i) only as
// factors, the remainder weight of Thm. parametrix is
//   W^R_ik = a_i W_lb[ik] + grad_a_i . W_g[:, ik]   (multiplying sigma_k / a_k),
// so pm_surface_set_coeff only recombines.
//
// Self patch (eq. radial_int): polar coordinates about the target's reference
// point; theta panels from the host plan (adaptive on int L^2, capped width);
// four radial Gauss panels [0,L/8], [L/8,L/4], [L/4,L/2], [L/2,L], the first
// with product-log weights for the log|r| kernel.  The normal in q is that of
// the interpolated patch at the target, and x - y~ is formed from node
// offsets so it keeps its precision as y~ -> x.
// Near patches: quadtree subdivision of [-1,1]^2, splitting a square while the
// target lies within 2*eta*(corner radius) of its centre image, 16 x 16 Gauss
// rule on each leaf (a geometric a-priori criterion standing in for the
// adaptive error test of Sec. 6.1.2).
#include "pm_green.cuh"
#include "pm_internal.cuh"

#include <algorithm>
#include <cstring>
#include <cmath>
#include <vector>

namespace {

__constant__ QuadTables cT;

constexpr int kQThreads = 128;
constexpr int kMaxLeaves = 512;
constexpr int kMaxLevel = 1024;   // squares per BFS level

// Lagrange basis l_a(u) = lambda_a prod_{b != a} (u - t_b), by prefix/suffix
// products (no division; exact at the nodes).
__device__ __forceinline__ void lagrange(double u, int p, double* out) {
    double d[PM_MAX_P];
    for (int b = 0; b < p; ++b) d[b] = u - cT.t[b];
    double pre = 1.0;
    for (int a = 0; a < p; ++a) {
        out[a] = pre;
        pre *= d[a];
    }
    double suf = 1.0;
    for (int a = p - 1; a >= 0; --a) {
        out[a] *= suf * cT.bary[a];
        suf *= d[a];
    }
}

// y~(u, v) for one patch from its node positions X (global layout).
__device__ void interp_pos(const double* X, int p, double u, double v, double* y) {
    double lu[PM_MAX_P], lv[PM_MAX_P];
    lagrange(u, p, lu);
    lagrange(v, p, lv);
    double y0 = 0, y1 = 0, y2 = 0;
    for (int a = 0; a < p; ++a) {
        double z0 = 0, z1 = 0, z2 = 0;
        for (int b = 0; b < p; ++b) {
            const double* xp = X + 3 * (a * p + b);
            z0 += xp[0] * lv[b];
            z1 += xp[1] * lv[b];
            z2 += xp[2] * lv[b];
        }
        y0 += lu[a] * z0;
        y1 += lu[a] * z1;
        y2 += lu[a] * z2;
    }
    y[0] = y0; y[1] = y1; y[2] = y2;
}

// ------------------------------------------------------------------ patch data
__global__ void k_patch_geom(const double* __restrict__ x, int npatch, int p,
                             double* __restrict__ centroid, double* __restrict__ radius) {
    int P = blockIdx.x * blockDim.x + threadIdx.x;
    if (P >= npatch) return;
    const double* X = x + (size_t)3 * P * p * p;
    const double cu[4] = {1, -1, -1, 1}, cv[4] = {1, 1, -1, -1};
    double c[4][3];
    for (int k = 0; k < 4; ++k) interp_pos(X, p, cu[k], cv[k], c[k]);
    double m[3];
    for (int d = 0; d < 3; ++d) m[d] = 0.25 * (c[0][d] + c[1][d] + c[2][d] + c[3][d]);
    double r = 0;
    for (int k = 0; k < 4; ++k) {
        double dx = c[k][0] - m[0], dy = c[k][1] - m[1], dz = c[k][2] - m[2];
        r = fmax(r, sqrt(dx * dx + dy * dy + dz * dz));
    }
    for (int d = 0; d < 3; ++d) centroid[3 * P + d] = m[d];
    radius[P] = r;
}

// Unit normal of the interpolated patch at each node (spectral derivatives).
__global__ void k_node_normals(const double* __restrict__ x, int N, int p,
                               double* __restrict__ nn) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const int pp = p * p, P = k / pp, loc = k - P * pp, i0 = loc / p, j0 = loc % p;
    const double* X = x + (size_t)3 * P * pp;
    double yu[3] = {0, 0, 0}, yv[3] = {0, 0, 0};
    for (int m = 0; m < p; ++m) {
        const double du = cT.Dm[i0 * p + m], dv = cT.Dm[j0 * p + m];
        for (int c = 0; c < 3; ++c) {
            yu[c] += du * X[3 * (m * p + j0) + c];
            yv[c] += dv * X[3 * (i0 * p + m) + c];
        }
    }
    double c0 = yu[1] * yv[2] - yu[2] * yv[1];
    double c1 = yu[2] * yv[0] - yu[0] * yv[2];
    double c2 = yu[0] * yv[1] - yu[1] * yv[0];
    double inv = 1.0 / sqrt(c0 * c0 + c1 * c1 + c2 * c2);
    nn[3 * k] = c0 * inv;
    nn[3 * k + 1] = c1 * inv;
    nn[3 * k + 2] = c2 * inv;
}

__device__ __forceinline__ bool is_near(const double* xi, const double* cen, double rad,
                                        double factor) {
    double dx = xi[0] - cen[0], dy = xi[1] - cen[1], dz = xi[2] - cen[2];
    return sqrt(dx * dx + dy * dy + dz * dz) < factor * rad;
}

__global__ void k_near_count(const double* __restrict__ x, const double* __restrict__ centroid,
                             const double* __restrict__ radius, int N, int npatch, int pp,
                             double factor, int* __restrict__ count) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int own = i / pp;
    int c = 1;
    for (int P = 0; P < npatch; ++P)
        if (P != own && is_near(x + 3 * i, centroid + 3 * P, radius[P], factor)) ++c;
    count[i] = c;
}

__global__ void k_near_fill(const double* __restrict__ x, const double* __restrict__ centroid,
                            const double* __restrict__ radius, int N, int npatch, int pp,
                            double factor, const int* __restrict__ row_ptr,
                            int* __restrict__ blk_patch, int* __restrict__ blk_row) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int own = i / pp;
    int b = row_ptr[i];
    const int end = row_ptr[i + 1];
    blk_patch[b] = own;
    blk_row[b] = i;
    ++b;
    for (int P = 0; P < npatch && b < end; ++P)
        if (P != own && is_near(x + 3 * i, centroid + 3 * P, radius[P], factor)) {
            blk_patch[b] = P;
            blk_row[b] = i;
            ++b;
        }
}

// ------------------------------------------------------------------ self quadrature
// One block per target; shared memory (doubles): D [3*pp], Jn [pp],
// lu [128*p], lv [128*p], f [5*128].
__global__ void __launch_bounds__(kQThreads)
k_self_quad(int N, int p, const double* __restrict__ x, const double* __restrict__ J,
            const double* __restrict__ nn, const double* __restrict__ H,
            const int* __restrict__ th_off, const double* __restrict__ th_ang,
            const double* __restrict__ th_w, const double* __restrict__ th_L,
            const int* __restrict__ row_ptr, int nblk, double* __restrict__ W_lb,
            double* __restrict__ W_g, double* __restrict__ W_k) {
    extern __shared__ double sm[];
    const int pp = p * p;
    double* sD = sm;                       // [3][pp]
    double* sJ = sD + 3 * pp;              // [pp]
    double* sLu = sJ + pp;                 // [128][p]
    double* sLv = sLu + kQThreads * p;     // [128][p]
    double* sF = sLv + kQThreads * p;      // [5][128]
    const int i = blockIdx.x;
    const int tid = threadIdx.x;
    const int P = i / pp, loc = i - P * pp;
    const double u0 = cT.t[loc / p], v0 = cT.t[loc % p];
    const double xi0 = x[3 * i], xi1 = x[3 * i + 1], xi2 = x[3 * i + 2];
    for (int k = tid; k < pp; k += kQThreads) {
        const size_t gk = (size_t)P * pp + k;
        sD[k] = x[3 * gk] - xi0;
        sD[pp + k] = x[3 * gk + 1] - xi1;
        sD[2 * pp + k] = x[3 * gk + 2] - xi2;
        sJ[k] = J[gk];
    }
    const double n0 = nn[3 * i], n1 = nn[3 * i + 1], n2 = nn[3 * i + 2];
    const double Hi = H[i];
    const int t0 = th_off[loc], t1 = th_off[loc + 1];
    const int npts = (t1 - t0) * (PM_RADIAL_PANELS * PM_GL16);
    const double lo_f[4] = {0.0, 0.125, 0.25, 0.5};
    const double hi_f[4] = {0.125, 0.25, 0.5, 1.0};
    double acc_lb = 0, acc_g0 = 0, acc_g1 = 0, acc_g2 = 0, acc_k = 0;
    const int a_own = tid / p, b_own = tid - (tid / p) * p;
    __syncthreads();
    for (int base = 0; base < npts; base += kQThreads) {
        const int q = base + tid;
        double* lu = sLu + tid * p;
        double* lv = sLv + tid * p;
        double f_lb = 0, f_g0 = 0, f_g1 = 0, f_g2 = 0, f_k = 0;
        if (q < npts) {
            const int kth = t0 + q / (PM_RADIAL_PANELS * PM_GL16);
            const int rj = q % (PM_RADIAL_PANELS * PM_GL16);
            const int panel = rj / PM_GL16, node = rj % PM_GL16;
            const double L = th_L[kth];
            const double h = (hi_f[panel] - lo_f[panel]) * L;
            const double r = lo_f[panel] * L + 0.5 * h * (cT.g16t[node] + 1.0);
            const double wr = 0.5 * h * cT.g16w[node];
            double sn, cs;
            sincos(th_ang[kth], &sn, &cs);
            const double u = u0 + r * cs, v = v0 + r * sn;
            lagrange(u, p, lu);
            lagrange(v, p, lv);
            double d0 = 0, d1 = 0, d2 = 0, jj = 0;
            for (int a = 0; a < p; ++a) {
                double z0 = 0, z1 = 0, z2 = 0, zj = 0;
                for (int b = 0; b < p; ++b) {
                    const double l = lv[b];
                    const int k = a * p + b;
                    z0 += sD[k] * l;
                    z1 += sD[pp + k] * l;
                    z2 += sD[2 * pp + k] * l;
                    zj += sJ[k] * l;
                }
                d0 += lu[a] * z0;
                d1 += lu[a] * z1;
                d2 += lu[a] * z2;
                jj += lu[a] * zj;
            }
            // r_vec = x_i - y~ = -(sum of offsets)
            const double rx = -d0, ry = -d1, rz = -d2;
            const double r2 = rx * rx + ry * ry + rz * rz;
            const double inv = 1.0 / r2;
            const double qq = (n0 * rx + n1 * ry + n2 * rz) * inv;
            const double base_w = th_w[kth] * wr * r * jj;
            f_lb = base_w * (qq * qq - Hi * qq) * (1.0 / M_PI);
            const double gfac = base_w * inv * (0.5 / M_PI);
            f_g0 = gfac * rx;
            f_g1 = gfac * ry;
            f_g2 = gfac * rz;
            double lg = 0.5 * log(r2);
            if (panel == 0) lg += cT.logE[node];
            f_k = base_w * lg * (0.5 / M_PI);
        } else {
            for (int a = 0; a < p; ++a) { lu[a] = 0.0; lv[a] = 0.0; }
        }
        sF[tid] = f_lb;
        sF[kQThreads + tid] = f_g0;
        sF[2 * kQThreads + tid] = f_g1;
        sF[3 * kQThreads + tid] = f_g2;
        sF[4 * kQThreads + tid] = f_k;
        __syncthreads();
        if (tid < pp) {
            const int lim = min(kQThreads, npts - base);
            for (int qq = 0; qq < lim; ++qq) {
                const double c = sLu[qq * p + a_own] * sLv[qq * p + b_own];
                acc_lb += sF[qq] * c;
                acc_g0 += sF[kQThreads + qq] * c;
                acc_g1 += sF[2 * kQThreads + qq] * c;
                acc_g2 += sF[3 * kQThreads + qq] * c;
                acc_k += sF[4 * kQThreads + qq] * c;
            }
        }
        __syncthreads();
    }
    if (tid < pp) {
        const size_t b0 = (size_t)row_ptr[i];   // own patch is the row's first block
        W_lb[b0 * pp + tid] = acc_lb;
        W_g[(0 * (size_t)nblk + b0) * pp + tid] = acc_g0;
        W_g[(1 * (size_t)nblk + b0) * pp + tid] = acc_g1;
        W_g[(2 * (size_t)nblk + b0) * pp + tid] = acc_g2;
        W_k[b0 * pp + tid] = acc_k;
    }
}

// ------------------------------------------------------------------ near quadrature
// One block per (target, non-self near patch).  Square codes: level (4 bits),
// iu (12 bits), iv (12 bits); square = [-1 + 2 iu/2^l, -1 + 2 (iu+1)/2^l] x (same for v).
__device__ __forceinline__ int sq_code(int lev, int iu, int iv) { return (lev << 24) | (iu << 12) | iv; }
__device__ __forceinline__ void sq_box(int code, double& u0, double& u1, double& v0, double& v1) {
    const int lev = code >> 24, iu = (code >> 12) & 0xfff, iv = code & 0xfff;
    const double h = 2.0 / (double)(1 << lev);
    u0 = -1.0 + iu * h;
    u1 = u0 + h;
    v0 = -1.0 + iv * h;
    v1 = v0 + h;
}

// Breadth-first quadtree subdivision of [-1,1]^2 for the target (xi0, xi1, xi2)
// against the patch with node positions X: a square splits while the target
// lies within 2 eta (corner radius) of its centre image, up to max_depth levels.
// The leaves end in S.sorted in code order (deterministic); returns their count.
// Called by all threads of the block; a leaf or level overflow sets *err.
struct NearBfs {
    int cur[kMaxLevel], next[kMaxLevel], leaf[kMaxLeaves], sorted[kMaxLeaves];
    int nCur, nNext, nLeaf, overflow;
};

__device__ int near_leaves(const double* X, int p, double xi0, double xi1, double xi2,
                           double eta, int max_depth, int max_leaves, NearBfs& S, int* err) {
    const int tid = threadIdx.x;
    if (tid == 0) {
        S.cur[0] = sq_code(0, 0, 0);
        S.nCur = 1;
        S.nLeaf = 0;
        S.overflow = 0;
    }
    __syncthreads();
    const int leaf_cap = min(max_leaves, kMaxLeaves);
    for (int lev = 0; lev <= max_depth; ++lev) {
        if (tid == 0) S.nNext = 0;
        __syncthreads();
        for (int q = tid; q < S.nCur; q += blockDim.x) {
            const int code = S.cur[q];
            double u0, u1, v0, v1;
            sq_box(code, u0, u1, v0, v1);
            const double us[5] = {u0, u1, u1, u0, 0.5 * (u0 + u1)};
            const double vs[5] = {v0, v0, v1, v1, 0.5 * (v0 + v1)};
            double y[5][3];
            for (int k = 0; k < 5; ++k) interp_pos(X, p, us[k], vs[k], y[k]);
            double size = 0;
            for (int k = 0; k < 4; ++k) {
                const double dx = y[k][0] - y[4][0], dy = y[k][1] - y[4][1], dz = y[k][2] - y[4][2];
                size = fmax(size, sqrt(dx * dx + dy * dy + dz * dz));
            }
            const double dx = xi0 - y[4][0], dy = xi1 - y[4][1], dz = xi2 - y[4][2];
            const double dist = sqrt(dx * dx + dy * dy + dz * dz);
            const bool split = (lev < max_depth) && (dist < 2.0 * eta * size);
            if (split) {
                const int slot = atomicAdd(&S.nNext, 4);
                if (slot + 4 <= kMaxLevel) {
                    const int l1 = lev + 1, iu = (code >> 12) & 0xfff, iv = code & 0xfff;
                    S.next[slot] = sq_code(l1, 2 * iu, 2 * iv);
                    S.next[slot + 1] = sq_code(l1, 2 * iu + 1, 2 * iv);
                    S.next[slot + 2] = sq_code(l1, 2 * iu, 2 * iv + 1);
                    S.next[slot + 3] = sq_code(l1, 2 * iu + 1, 2 * iv + 1);
                } else {
                    S.overflow = 1;
                }
            } else {
                const int slot = atomicAdd(&S.nLeaf, 1);
                if (slot < leaf_cap) S.leaf[slot] = code; else S.overflow = 1;
            }
        }
        __syncthreads();
        const int nn_ = min(S.nNext, kMaxLevel);
        for (int q = tid; q < nn_; q += blockDim.x) S.cur[q] = S.next[q];
        __syncthreads();
        if (tid == 0) S.nCur = nn_;
        __syncthreads();
        if (S.nCur == 0) break;
    }
    const int nleaves = min(S.nLeaf, leaf_cap);
    if (S.overflow && tid == 0) atomicExch(err, PM_DEV_LEAF_OVERFLOW);
    // deterministic leaf order: rank sort by code
    for (int q = tid; q < nleaves; q += blockDim.x) {
        const int c = S.leaf[q];
        int rank = 0;
        for (int t = 0; t < nleaves; ++t) rank += (S.leaf[t] < c);
        S.sorted[rank] = c;
    }
    __syncthreads();
    return nleaves;
}

__global__ void __launch_bounds__(kQThreads)
k_near_quad(int p, int nblk, const double* __restrict__ x, const double* __restrict__ J,
            const double* __restrict__ n, const double* __restrict__ H,
            const int* __restrict__ blk_row, const int* __restrict__ blk_patch,
            const int* __restrict__ row_ptr, double eta, int max_depth, int max_leaves,
            double* __restrict__ W_lb, double* __restrict__ W_g, double* __restrict__ W_k,
            int* __restrict__ err) {
    const int b = blockIdx.x;
    const int i = blk_row[b];
    if (b == row_ptr[i]) return;   // the self block is done by k_self_quad
    const int P = blk_patch[b];
    const int pp = p * p;
    const int tid = threadIdx.x;
    __shared__ double sD[3 * PM_MAX_P * PM_MAX_P];
    __shared__ double sJ[PM_MAX_P * PM_MAX_P];
    __shared__ double sLu[PM_GL16 * PM_MAX_P], sLv[PM_GL16 * PM_MAX_P];
    __shared__ double sZ[4 * PM_MAX_P * PM_GL16];     // [4][a][r]
    __shared__ double sF[5 * PM_GL16 * PM_GL16];      // [5][q*16 + r]
    __shared__ NearBfs bfs;
    const double* X = x + (size_t)3 * P * pp;
    const double xi0 = x[3 * i], xi1 = x[3 * i + 1], xi2 = x[3 * i + 2];
    for (int k = tid; k < pp; k += kQThreads) {
        const size_t gk = (size_t)P * pp + k;
        sD[k] = x[3 * gk] - xi0;
        sD[pp + k] = x[3 * gk + 1] - xi1;
        sD[2 * pp + k] = x[3 * gk + 2] - xi2;
        sJ[k] = J[gk];
    }
    const int nleaves = near_leaves(X, p, xi0, xi1, xi2, eta, max_depth, max_leaves, bfs, err);
    const int a_own = tid / p, b_own = tid - (tid / p) * p;
    double acc[5] = {0, 0, 0, 0, 0};
    const double n0 = n[3 * i], n1 = n[3 * i + 1], n2 = n[3 * i + 2];
    const double Hi = H[i];
    for (int L = 0; L < nleaves; ++L) {
        double u0, u1, v0, v1;
        sq_box(bfs.sorted[L], u0, u1, v0, v1);
        const double hu = 0.5 * (u1 - u0), hv = 0.5 * (v1 - v0);
        if (tid < PM_GL16) lagrange(u0 + hu * (cT.g16t[tid] + 1.0), p, sLu + tid * p);
        else if (tid < 2 * PM_GL16)
            lagrange(v0 + hv * (cT.g16t[tid - PM_GL16] + 1.0), p, sLv + (tid - PM_GL16) * p);
        __syncthreads();
        // Z[c][a][r] = sum_b D_c[a][b] l_b(v_r)  (c = 3: J)
        for (int e = tid; e < 4 * p * PM_GL16; e += kQThreads) {
            const int c = e / (p * PM_GL16), rem = e - c * p * PM_GL16;
            const int a = rem / PM_GL16, r = rem - a * PM_GL16;
            const double* src = (c < 3) ? (sD + c * pp) : sJ;
            double z = 0;
            for (int bb = 0; bb < p; ++bb) z += src[a * p + bb] * sLv[r * p + bb];
            sZ[(c * p + a) * PM_GL16 + r] = z;
        }
        __syncthreads();
        for (int e = tid; e < PM_GL16 * PM_GL16; e += kQThreads) {
            const int qn = e / PM_GL16, r = e - qn * PM_GL16;
            double d0 = 0, d1 = 0, d2 = 0, jj = 0;
            for (int a = 0; a < p; ++a) {
                const double l = sLu[qn * p + a];
                d0 += l * sZ[(0 * p + a) * PM_GL16 + r];
                d1 += l * sZ[(1 * p + a) * PM_GL16 + r];
                d2 += l * sZ[(2 * p + a) * PM_GL16 + r];
                jj += l * sZ[(3 * p + a) * PM_GL16 + r];
            }
            const double rx = -d0, ry = -d1, rz = -d2;
            const double r2 = rx * rx + ry * ry + rz * rz;
            const double inv = 1.0 / r2;
            const double qq = (n0 * rx + n1 * ry + n2 * rz) * inv;
            const double wgt = hu * cT.g16w[qn] * hv * cT.g16w[r] * jj;
            sF[e] = wgt * (qq * qq - Hi * qq) * (1.0 / M_PI);
            const double gfac = wgt * inv * (0.5 / M_PI);
            sF[256 + e] = gfac * rx;
            sF[512 + e] = gfac * ry;
            sF[768 + e] = gfac * rz;
            sF[1024 + e] = wgt * 0.25 / M_PI * log(r2);
        }
        __syncthreads();
        // T[k][a][r] = sum_q F[k][q][r] l_a(u_q)  (reuse sZ region is too small; use a loop)
        if (tid < pp) {
            for (int r = 0; r < PM_GL16; ++r) {
                double t5[5] = {0, 0, 0, 0, 0};
                for (int qn = 0; qn < PM_GL16; ++qn) {
                    const double l = sLu[qn * p + a_own];
                    const int e = qn * PM_GL16 + r;
                    t5[0] += sF[e] * l;
                    t5[1] += sF[256 + e] * l;
                    t5[2] += sF[512 + e] * l;
                    t5[3] += sF[768 + e] * l;
                    t5[4] += sF[1024 + e] * l;
                }
                const double lb = sLv[r * p + b_own];
                for (int k = 0; k < 5; ++k) acc[k] += t5[k] * lb;
            }
        }
        __syncthreads();
    }
    if (tid < pp) {
        const size_t o = (size_t)b * pp + tid;
        W_lb[o] = acc[0];
        W_g[0 * (size_t)nblk * pp + o] = acc[1];
        W_g[1 * (size_t)nblk * pp + o] = acc[2];
        W_g[2 * (size_t)nblk * pp + o] = acc[3];
        W_k[o] = acc[4];
    }
}

// ------------------------------------------------------------------ coefficient combination
__global__ void k_combine(int nblk, int pp, int ppad, const int* __restrict__ blk_row,
                          const int* __restrict__ blk_patch, const double* __restrict__ x,
                          const double* __restrict__ n, const double* __restrict__ H,
                          const double* __restrict__ w, const double* __restrict__ a,
                          const double* __restrict__ g, const double* __restrict__ W_lb,
                          const double* __restrict__ W_g, const double* __restrict__ W_k,
                          double* __restrict__ cR64, double* __restrict__ cK64,
                          float* __restrict__ cR32, float* __restrict__ cK32) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)nblk * ppad) return;
    const int b = (int)(e / ppad), k = (int)(e - (size_t)b * ppad);
    if (k >= pp) {
        cR32[e] = 0.f;
        cK32[e] = 0.f;
        return;
    }
    const int i = blk_row[b], P = blk_patch[b];
    const int j = P * pp + k;
    const size_t o = (size_t)b * pp + k;
    const size_t nv = (size_t)nblk * pp;
    const double ai = a[i];
    const double WR = ai * W_lb[o] + g[3 * i] * W_g[o] + g[3 * i + 1] * W_g[nv + o] +
                      g[3 * i + 2] * W_g[2 * nv + o];
    double cr, ck;
    if (j == i) {
        cr = WR / ai;
        ck = W_k[o] / ai;
    } else {
        const double aj = a[j];
        const double rx = x[3 * i] - x[3 * j], ry = x[3 * i + 1] - x[3 * j + 1],
                     rz = x[3 * i + 2] - x[3 * j + 2];
        const double r2 = rx * rx + ry * ry + rz * rz;
        const double q = (n[3 * i] * rx + n[3 * i + 1] * ry + n[3 * i + 2] * rz) / r2;
        const double Rij = (ai / aj) * (q * q - H[i] * q) / M_PI +
                           (g[3 * i] * rx + g[3 * i + 1] * ry + g[3 * i + 2] * rz) /
                               (2.0 * M_PI * aj * r2);
        const double Kij = log(r2) / (4.0 * M_PI * aj);
        cr = WR / aj - w[j] * Rij;
        ck = W_k[o] / aj - w[j] * Kij;
    }
    cR64[o] = cr;
    cK64[o] = ck;
    cR32[e] = (float)cr;
    cK32[e] = (float)ck;
}

// ------------------------------------------------------------------ c != 0 quadrature
// Weights of a(y) R and a(y) K for real c (eq. explicit_remainder with
// a(y) G = g(r; k(y)), pm_green.cuh), complex as (re, im):
//   W^R_ik = int a(y) R(x_i, y) l_k J~ du dv,  W^K_ik = int g(|x_i - y|; k(y)) l_k J~ du dv.
// The kernels depend on the source through k(y)^2 = q(y) = c(y)/a(y), which is
// interpolated on the patch from its nodes with the tensor Lagrange basis, so
// these weights hold the coefficients and are built per coefficient field.
// Self patch: the polar rule of k_self_quad, with dyadic radial panels
// [0, L 2^-12], [L 2^-12, L 2^-11], ..., [L/2, L] in place of the product-log
// panel: here g = log(r) A(r) + B(r) with A = J0(kr) or I0(kr) not constant, and
// R has r log r terms (Thm. remainder); each graded panel sees an analytic
// integrand, and the innermost one carries O(L^2 2^-24 log) of the integral.
constexpr int kSelfLevelsC = 12;
constexpr int kSelfPanelsC = kSelfLevelsC + 1;

__global__ void __launch_bounds__(kQThreads)
k_self_quad_c(int N, int p, const double* __restrict__ x, const double* __restrict__ J,
              const double* __restrict__ nn, const double* __restrict__ H,
              const double* __restrict__ a, const double* __restrict__ g,
              const double2* __restrict__ c, const double2* __restrict__ qn,
              const int* __restrict__ th_off, const double* __restrict__ th_ang,
              const double* __restrict__ th_w, const double* __restrict__ th_L,
              const int* __restrict__ row_ptr, double2* __restrict__ WR,
              double2* __restrict__ WK) {
    extern __shared__ double sm[];
    const int pp = p * p;
    double* sD = sm;                       // [3][pp]
    double* sJ = sD + 3 * pp;              // [pp]
    double* sQ = sJ + pp;                  // [2][pp]: q = c/a, re and im
    double* sLu = sQ + 2 * pp;             // [128][p]
    double* sLv = sLu + kQThreads * p;     // [128][p]
    double* sF = sLv + kQThreads * p;      // [4][128]
    const int i = blockIdx.x;
    const int tid = threadIdx.x;
    const int P = i / pp, loc = i - P * pp;
    const double u0 = cT.t[loc / p], v0 = cT.t[loc % p];
    const double xi0 = x[3 * i], xi1 = x[3 * i + 1], xi2 = x[3 * i + 2];
    for (int k = tid; k < pp; k += kQThreads) {
        const size_t gk = (size_t)P * pp + k;
        sD[k] = x[3 * gk] - xi0;
        sD[pp + k] = x[3 * gk + 1] - xi1;
        sD[2 * pp + k] = x[3 * gk + 2] - xi2;
        sJ[k] = J[gk];
        sQ[k] = qn[gk].x;
        sQ[pp + k] = qn[gk].y;
    }
    const double n0 = nn[3 * i], n1 = nn[3 * i + 1], n2 = nn[3 * i + 2];
    const double Hi = H[i], ai = a[i];
    const pm_green::cplx_d ci = {c[i].x, c[i].y};
    const double g0 = g[3 * i], g1 = g[3 * i + 1], g2 = g[3 * i + 2];
    const int t0 = th_off[loc], t1 = th_off[loc + 1];
    const int npts = (t1 - t0) * (kSelfPanelsC * PM_GL16);
    double acc[4] = {0, 0, 0, 0};
    const int a_own = tid / p, b_own = tid - (tid / p) * p;
    __syncthreads();
    for (int base = 0; base < npts; base += kQThreads) {
        const int q = base + tid;
        double* lu = sLu + tid * p;
        double* lv = sLv + tid * p;
        double f[4] = {0, 0, 0, 0};
        if (q < npts) {
            const int kth = t0 + q / (kSelfPanelsC * PM_GL16);
            const int rj = q % (kSelfPanelsC * PM_GL16);
            const int panel = rj / PM_GL16, node = rj % PM_GL16;
            const double L = th_L[kth];
            const double lo = panel == 0 ? 0.0 : ldexp(L, panel - kSelfPanelsC);
            const double h = ldexp(L, panel - kSelfLevelsC) - lo;
            const double r = lo + 0.5 * h * (cT.g16t[node] + 1.0);
            const double wr = 0.5 * h * cT.g16w[node];
            double sn, cs;
            sincos(th_ang[kth], &sn, &cs);
            lagrange(u0 + r * cs, p, lu);
            lagrange(v0 + r * sn, p, lv);
            double d0 = 0, d1 = 0, d2 = 0, jj = 0, qr = 0, qi = 0;
            for (int aa = 0; aa < p; ++aa) {
                double z0 = 0, z1 = 0, z2 = 0, zj = 0, zr = 0, zi = 0;
                for (int bb = 0; bb < p; ++bb) {
                    const double l = lv[bb];
                    const int k = aa * p + bb;
                    z0 += sD[k] * l;
                    z1 += sD[pp + k] * l;
                    z2 += sD[2 * pp + k] * l;
                    zj += sJ[k] * l;
                    zr += sQ[k] * l;
                    zi += sQ[pp + k] * l;
                }
                d0 += lu[aa] * z0;
                d1 += lu[aa] * z1;
                d2 += lu[aa] * z2;
                jj += lu[aa] * zj;
                qr += lu[aa] * zr;
                qi += lu[aa] * zi;
            }
            double out[4];
            pm_green::pair_rk_cz(-d0, -d1, -d2, n0, n1, n2, Hi, ai, g0, g1, g2, ci,
                                 pm_green::cplx_d{qr, qi}, cT.g16t, cT.g16w, out);
            const double bw = th_w[kth] * wr * r * jj;
            for (int k = 0; k < 4; ++k) f[k] = bw * out[k];
        } else {
            for (int aa = 0; aa < p; ++aa) { lu[aa] = 0.0; lv[aa] = 0.0; }
        }
        for (int k = 0; k < 4; ++k) sF[k * kQThreads + tid] = f[k];
        __syncthreads();
        if (tid < pp) {
            const int lim = min(kQThreads, npts - base);
            for (int e = 0; e < lim; ++e) {
                const double cc = sLu[e * p + a_own] * sLv[e * p + b_own];
                for (int k = 0; k < 4; ++k) acc[k] += sF[k * kQThreads + e] * cc;
            }
        }
        __syncthreads();
    }
    if (tid < pp) {
        const size_t o = (size_t)row_ptr[i] * pp + tid;     // own patch: the row's first block
        WR[o] = make_double2(acc[0], acc[1]);
        WK[o] = make_double2(acc[2], acc[3]);
    }
}

// Near, non-self patches: the subdivision of k_near_quad, 16 x 16 Gauss points
// per leaf, the target's given normal.
__global__ void __launch_bounds__(kQThreads)
k_near_quad_c(int p, const double* __restrict__ x, const double* __restrict__ J,
              const double* __restrict__ n, const double* __restrict__ H,
              const double* __restrict__ a, const double* __restrict__ g,
              const double2* __restrict__ c, const double2* __restrict__ qn,
              const int* __restrict__ blk_row, const int* __restrict__ blk_patch,
              const int* __restrict__ row_ptr, double eta, int max_depth, int max_leaves,
              double2* __restrict__ WR, double2* __restrict__ WK, int* __restrict__ err) {
    const int b = blockIdx.x;
    const int i = blk_row[b];
    if (b == row_ptr[i]) return;   // the self block is done by k_self_quad_c
    const int P = blk_patch[b];
    const int pp = p * p;
    const int tid = threadIdx.x;
    // sized for the largest order a surface accepts (p <= PM_MAX_P_API)
    __shared__ double sD[3 * PM_MAX_P_API * PM_MAX_P_API];
    __shared__ double sJ[PM_MAX_P_API * PM_MAX_P_API];
    __shared__ double sQ[2 * PM_MAX_P_API * PM_MAX_P_API];   // q = c/a: re, im
    __shared__ double sLu[PM_GL16 * PM_MAX_P_API], sLv[PM_GL16 * PM_MAX_P_API];
    __shared__ double sZ[6 * PM_MAX_P_API * PM_GL16];        // [6][a][r]
    __shared__ double sF[4 * PM_GL16 * PM_GL16];      // [4][q*16 + r]
    __shared__ NearBfs bfs;
    const double* X = x + (size_t)3 * P * pp;
    const double xi0 = x[3 * i], xi1 = x[3 * i + 1], xi2 = x[3 * i + 2];
    for (int k = tid; k < pp; k += kQThreads) {
        const size_t gk = (size_t)P * pp + k;
        sD[k] = x[3 * gk] - xi0;
        sD[pp + k] = x[3 * gk + 1] - xi1;
        sD[2 * pp + k] = x[3 * gk + 2] - xi2;
        sJ[k] = J[gk];
        sQ[k] = qn[gk].x;
        sQ[pp + k] = qn[gk].y;
    }
    const int nleaves = near_leaves(X, p, xi0, xi1, xi2, eta, max_depth, max_leaves, bfs, err);
    const int a_own = tid / p, b_own = tid - (tid / p) * p;
    double acc[4] = {0, 0, 0, 0};
    const double n0 = n[3 * i], n1 = n[3 * i + 1], n2 = n[3 * i + 2];
    const double Hi = H[i], ai = a[i];
    const pm_green::cplx_d ci = {c[i].x, c[i].y};
    const double g0 = g[3 * i], g1 = g[3 * i + 1], g2 = g[3 * i + 2];
    constexpr int kQ2 = PM_GL16 * PM_GL16;
    for (int L = 0; L < nleaves; ++L) {
        double u0, u1, v0, v1;
        sq_box(bfs.sorted[L], u0, u1, v0, v1);
        const double hu = 0.5 * (u1 - u0), hv = 0.5 * (v1 - v0);
        if (tid < PM_GL16) lagrange(u0 + hu * (cT.g16t[tid] + 1.0), p, sLu + tid * p);
        else if (tid < 2 * PM_GL16)
            lagrange(v0 + hv * (cT.g16t[tid - PM_GL16] + 1.0), p, sLv + (tid - PM_GL16) * p);
        __syncthreads();
        // Z[f][a][r] = sum_b F_f[a][b] l_b(v_r) for F = D (3 components), J, q (re, im)
        for (int e = tid; e < 6 * p * PM_GL16; e += kQThreads) {
            const int cf = e / (p * PM_GL16), rem = e - cf * p * PM_GL16;
            const int aa = rem / PM_GL16, r = rem - aa * PM_GL16;
            const double* src = (cf < 3) ? (sD + cf * pp) : (cf == 3 ? sJ : sQ + (cf - 4) * pp);
            double z = 0;
            for (int bb = 0; bb < p; ++bb) z += src[aa * p + bb] * sLv[r * p + bb];
            sZ[(cf * p + aa) * PM_GL16 + r] = z;
        }
        __syncthreads();
        for (int e = tid; e < kQ2; e += kQThreads) {
            const int qn_ = e / PM_GL16, r = e - qn_ * PM_GL16;
            double v5[6] = {0, 0, 0, 0, 0, 0};
            for (int aa = 0; aa < p; ++aa) {
                const double l = sLu[qn_ * p + aa];
                for (int cf = 0; cf < 6; ++cf) v5[cf] += l * sZ[(cf * p + aa) * PM_GL16 + r];
            }
            double out[4];
            pm_green::pair_rk_cz(-v5[0], -v5[1], -v5[2], n0, n1, n2, Hi, ai, g0, g1, g2, ci,
                                 pm_green::cplx_d{v5[4], v5[5]}, cT.g16t, cT.g16w, out);
            const double wgt = hu * cT.g16w[qn_] * hv * cT.g16w[r] * v5[3];
            for (int k = 0; k < 4; ++k) sF[k * kQ2 + e] = wgt * out[k];
        }
        __syncthreads();
        if (tid < pp) {
            for (int r = 0; r < PM_GL16; ++r) {
                double t4[4] = {0, 0, 0, 0};
                for (int qn_ = 0; qn_ < PM_GL16; ++qn_) {
                    const double l = sLu[qn_ * p + a_own];
                    const int e = qn_ * PM_GL16 + r;
                    for (int k = 0; k < 4; ++k) t4[k] += sF[k * kQ2 + e] * l;
                }
                const double lb = sLv[r * p + b_own];
                for (int k = 0; k < 4; ++k) acc[k] += t4[k] * lb;
            }
        }
        __syncthreads();
    }
    if (tid < pp) {
        const size_t o = (size_t)b * pp + tid;
        WR[o] = make_double2(acc[0], acc[1]);
        WK[o] = make_double2(acc[2], acc[3]);
    }
}

// Corrections in place: C = (W - w_j a(y)G(x_i, x_j)) / a_j off the diagonal (the
// smooth rule's term of the node), C_ii = W_ii / a_i; they multiply sigma_j.
__global__ void k_combine_c(int nblk, int pp, const int* __restrict__ blk_row,
                            const int* __restrict__ blk_patch, const double* __restrict__ x,
                            const double* __restrict__ n, const double* __restrict__ H,
                            const double* __restrict__ w, const double* __restrict__ a,
                            const double* __restrict__ g, const double2* __restrict__ c,
                            const double2* __restrict__ qn, double2* __restrict__ CR,
                            double2* __restrict__ CK) {
    const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)nblk * pp) return;
    const int b = (int)(e / pp), k = (int)(e - (size_t)b * pp);
    const int i = blk_row[b], j = blk_patch[b] * pp + k;
    double2 wr = CR[e], wk = CK[e];
    const double inv_a = 1.0 / a[j];
    if (j != i) {
        double out[4];
        pm_green::pair_rk_cz(x[3 * i] - x[3 * j], x[3 * i + 1] - x[3 * j + 1],
                             x[3 * i + 2] - x[3 * j + 2], n[3 * i], n[3 * i + 1], n[3 * i + 2],
                             H[i], a[i], g[3 * i], g[3 * i + 1], g[3 * i + 2],
                             pm_green::cplx_d{c[i].x, c[i].y}, pm_green::cplx_d{qn[j].x, qn[j].y},
                             cT.g16t, cT.g16w, out);
        wr.x -= w[j] * out[0];
        wr.y -= w[j] * out[1];
        wk.x -= w[j] * out[2];
        wk.y -= w[j] * out[3];
    }
    CR[e] = make_double2(wr.x * inv_a, wr.y * inv_a);
    CK[e] = make_double2(wk.x * inv_a, wk.y * inv_a);
}

// ------------------------------------------------------------------ correction SpMV
// L lanes per target row: out_i = sum_s partial[s][i] + sum_b C[b, :] .
// sigma[patch_b].  L = 32 (a warp per row) while all rows fit in one wave of
// warps; beyond that L = 8, so that every warp keeps the load chains of four
// rows in flight (the kernel is bound by load latency, not bandwidth).  float32 path: the row's blocks are contiguous, so the row's
// lanes walk the flat list of float4 values (four loads in flight per lane);
// the split partials (hi, lo) and the lane sums are combined with TwoSum in
// float32.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bp = s - a;
    e = (a - (s - bp)) + (b - bp);
}

// All of a row's loads are issued before any of them is consumed: the lane's
// partial slices (up to 4 per lane), then U float4 correction values and the U
// matching float4 pieces of sigma (their patch index from blk_patch), so that a
// lane keeps about 2U + 4 independent loads in flight; with L = 8 and U = 8 one
// pass covers a row of up to 4 near patches of 8 x 8 nodes.
template <int L, int U>
__global__ void __launch_bounds__(256)
k_near_apply32(int N, int ppad, const int* __restrict__ row_ptr,
               const int* __restrict__ blk_patch, const float* __restrict__ vals,
               const float* __restrict__ sig32, const float2* __restrict__ partial,
               int nsplit, int use_near, double* __restrict__ out,
               const int* __restrict__ skip) {
    if (skip && *skip) return;
    const int gt = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = gt / L;               // row of this lane group
    const int hl = threadIdx.x % L;     // lane within the group
    const bool row_ok = i < N;
    float2 pv[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int sp = hl + k * L;
        pv[k] = (row_ok && sp < nsplit) ? __ldg(partial + (size_t)sp * N + i) : make_float2(0.f, 0.f);
    }
    float acc = 0.f;
    if (use_near && row_ok) {
        const int q4 = ppad >> 2;
        const int rb = row_ptr[i];
        const int total = (row_ptr[i + 1] - rb) * q4;
        const float4* v4 = reinterpret_cast<const float4*>(vals) + (size_t)rb * q4;
        const float4* s4 = reinterpret_cast<const float4*>(sig32);
        for (int e0 = 0; e0 < total; e0 += U * L) {
            float4 v[U], x[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int e = e0 + u * L + hl;
                if (e < total) {
                    const int b = e / q4;
                    v[u] = __ldg(v4 + e);
                    x[u] = __ldg(s4 + (size_t)__ldg(blk_patch + rb + b) * q4 + (e - b * q4));
                } else {
                    v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                    x[u] = v[u];
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
                acc = fmaf(v[u].x, x[u].x, fmaf(v[u].y, x[u].y, fmaf(v[u].z, x[u].z, fmaf(v[u].w, x[u].w, acc))));
        }
    }
    float hi = 0.f, lo = 0.f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float s, e;
        two_sum(hi, pv[k].x, s, e);
        hi = s;
        lo += e + pv[k].y;
    }
    if (row_ok)
        for (int sp = hl + 4 * L; sp < nsplit; sp += L) {
            const float2 v = partial[(size_t)sp * N + i];
            float s, e;
            two_sum(hi, v.x, s, e);
            hi = s;
            lo += e + v.y;
        }
    {
        float s, e;
        two_sum(hi, acc, s, e);
        hi = s;
        lo += e;
    }
    // reduce within the lane group (xor offsets < L stay inside it)
    for (int o = L / 2; o > 0; o >>= 1) {
        const float h2 = __shfl_xor_sync(0xffffffffu, hi, o);
        const float l2 = __shfl_xor_sync(0xffffffffu, lo, o);
        float s, e;
        two_sum(hi, h2, s, e);
        hi = s;
        lo += e + l2;
    }
    if (row_ok && hl == 0) out[i] = (double)hi + (double)lo;
}

// Float-float partial slices summed per row, one thread a row (the slices of a row are
// N entries apart, so consecutive threads read consecutive entries of every slice).
// Runs of 32 slices are added in float-float with the accurate double-word addition
// (two TwoSums and two renormalisations, relative error below 3 * 2^-48 an addition);
// the run sums are added in float64, 1/32 of the float64 operations of a float64
// summation of every slice.  For the many slices of the symmetric sums and of the
// stored symmetric matrix (one per 128-node tile).
__global__ void k_sum_slices_ff(int N, int nsplit, const float2* __restrict__ partial,
                                double* __restrict__ out, const int* __restrict__ skip) {
    if (skip && *skip) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double acc = 0.0;
    for (int s0 = 0; s0 < nsplit; s0 += 32) {
        const int s1 = min(s0 + 32, nsplit);
        float hi = 0.f, lo = 0.f;
#pragma unroll 8
        for (int sp = s0; sp < s1; ++sp) {
            const float2 v = partial[(size_t)sp * N + i];
            float sh, eh, sl, el;
            two_sum(hi, v.x, sh, eh);
            two_sum(lo, v.y, sl, el);
            eh += sl;
            hi = sh + eh;                 // fast two-sum: |sh| >= |eh|
            eh -= hi - sh;
            eh += el;
            lo = eh;
            sh = hi + lo;
            lo -= sh - hi;
            hi = sh;
        }
        acc += (double)hi + (double)lo;
    }
    out[i] = acc;
}

// add_out != 0: the row starts from out[i] (the slices already summed there)
__global__ void k_near_apply64(int N, int pp, const int* __restrict__ row_ptr,
                               const int* __restrict__ blk_patch, const double* __restrict__ vals,
                               const double* __restrict__ sigma, const double* __restrict__ partial,
                               int nsplit, int partial_ff, int use_near, int add_out,
                               double* __restrict__ out, const int* __restrict__ skip) {
    if (skip && *skip) return;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= N) return;
    const int i = warp;
    double acc = (add_out && lane == 0) ? out[i] : 0.0;
    for (int sp = lane; sp < nsplit; sp += 32) {
        if (partial_ff) {
            const float2 v = reinterpret_cast<const float2*>(partial)[(size_t)sp * N + i];
            acc += (double)v.x + (double)v.y;
        } else {
            acc += partial[(size_t)sp * N + i];
        }
    }
    if (use_near) {
        for (int b = row_ptr[i]; b < row_ptr[i + 1]; ++b) {
            const double* v = vals + (size_t)b * pp;
            const double* sg = sigma + (size_t)blk_patch[b] * pp;
            for (int k = lane; k < pp; k += 32) acc += v[k] * sg[k];
        }
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) out[i] = acc;
}

// Smallest squared distance between a target and the other nodes of its near
// patches (every node closer than a patch radius lies in one), as the bits of a
// positive float, which order like the floats themselves.
__global__ void k_near_min_dist(const double* __restrict__ x, const int* __restrict__ blk_row,
                                const int* __restrict__ blk_patch, int pp,
                                unsigned int* __restrict__ out) {
    const int b = blockIdx.x;
    const int i = blk_row[b], P = blk_patch[b];
    double m = 1e300;
    for (int k = threadIdx.x; k < pp; k += blockDim.x) {
        const int j = P * pp + k;
        if (j == i) continue;
        const double dx = x[3 * i] - x[3 * j], dy = x[3 * i + 1] - x[3 * j + 1],
                     dz = x[3 * i + 2] - x[3 * j + 2];
        m = fmin(m, dx * dx + dy * dy + dz * dz);
    }
    for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m < 1e300)
        atomicMin(out, __float_as_uint((float)m));
}

// Largest squared distance of a node from the mean of its tile of `tile`
// consecutive nodes (one block per tile, float bits as above).
__global__ void k_tile_radius(const double* __restrict__ x, int N, int tile,
                              unsigned int* __restrict__ out) {
    __shared__ double red[3][32];
    const int t0 = blockIdx.x * tile, t1 = min(t0 + tile, N);
    double c[3] = {0.0, 0.0, 0.0};
    for (int i = t0 + threadIdx.x; i < t1; i += blockDim.x)
        for (int d = 0; d < 3; ++d) c[d] += x[3 * i + d];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int d = 0; d < 3; ++d) {
        for (int o = 16; o > 0; o >>= 1) c[d] += __shfl_xor_sync(0xffffffffu, c[d], o);
        if (lane == 0) red[d][wid] = c[d];
    }
    __syncthreads();
    for (int d = 0; d < 3; ++d) {
        c[d] = 0.0;
        for (int w = 0; w < nw; ++w) c[d] += red[d][w];
        c[d] /= (double)(t1 - t0);
    }
    double m = 0.0;
    for (int i = t0 + threadIdx.x; i < t1; i += blockDim.x) {
        const double dx = x[3 * i] - c[0], dy = x[3 * i + 1] - c[1], dz = x[3 * i + 2] - c[2];
        m = fmax(m, dx * dx + dy * dy + dz * dz);
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) atomicMax(out, __float_as_uint((float)m));
}


// ------------------------------------------------------------------ boundary-value systems
// Surface-integral weights at an edge node x_e of an open surface (Sec. 5): for a patch P
// near x_e, W_k = int_P G(x, y) l_k J~ du dv with G = nu_e . (x - y) / (2 pi |x - y|^2)
// (K'_Gamma, Sec. 5.2, Thm. NeumannBCsrep; log_kernel = 0) or G = log|x - y| / (2 pi)
// (K_Gamma on gamma, Sec. 5.3, Thm. Dirhclet_enforce; log_kernel = 1); the density
// sigma / a is interpolated, as for the surface operators.  One block per (edge node,
// patch) pair.  own != 0: x_e lies on an edge of P at reference point (u0, v0); the
// rule is polar about the patch's own point x = y~(u0, v0) over the directions that
// enter the square, theta cut at the corner directions and at most pi/32 wide (next to
// a corner direction the ray length L varies fast; pi/16 panels left 1e-10 errors in
// the weights of an edge node 1/16 of a patch from a corner),
// 16-point Gauss in theta and on each radial panel: [0, L/4], [L/4, L] for the
// gradient kernel (after the polar Jacobian its integrand is smooth), dyadic panels
// [2^-(k+1), 2^-k] L, k < 18, and [0, 2^-18 L] for the log kernel (rho log rho).
// own == 0: the quadtree near rule about x = x_e as in k_near_quad.
constexpr int kBvpPts = 128;          // quadrature points per pass of the polar rule
constexpr int kBvpLogLevels = 18;     // dyadic radial panels of the log-kernel polar rule

__device__ double bvp_ray(double u0, double v0, double ct, double st) {
    double L = 1e300;
    if (ct > 1e-15) L = fmin(L, (1.0 - u0) / ct);
    if (ct < -1e-15) L = fmin(L, (-1.0 - u0) / ct);
    if (st > 1e-15) L = fmin(L, (1.0 - v0) / st);
    if (st < -1e-15) L = fmin(L, (-1.0 - v0) / st);
    return L;
}

__global__ void __launch_bounds__(kQThreads)
k_bvp_kp_quad(int p, const double* __restrict__ x, const double* __restrict__ J,
              const int* __restrict__ blk_edge, const int* __restrict__ blk_patch,
              const int* __restrict__ blk_own, const double* __restrict__ xe,
              const double* __restrict__ nue, const double* __restrict__ uv, int log_kernel,
              double eta, int max_depth, int max_leaves, double* __restrict__ W,
              int* __restrict__ err) {
    const int blk = blockIdx.x;
    const int e = blk_edge[blk], P = blk_patch[blk];
    const int pp = p * p, tid = threadIdx.x;
    __shared__ double sD[3 * PM_MAX_P * PM_MAX_P];
    __shared__ double sJ[PM_MAX_P * PM_MAX_P];
    // polar rule: basis values of the pass's points; quadtree: basis values at the
    // leaf's 16 Gauss abscissae in u and v, then the Z partial sums
    __shared__ double sBuf[2 * kBvpPts * PM_MAX_P_API];
    __shared__ double sF[PM_GL16 * PM_GL16];
    __shared__ double sX[3];
    __shared__ double sCut[8];
    __shared__ int sNcut;
    __shared__ NearBfs bfs;
    const double* X = x + (size_t)3 * P * pp;
    const double n0 = nue[3 * e], n1 = nue[3 * e + 1], n2 = nue[3 * e + 2];
    const bool own = blk_own[blk] != 0;
    const double u0 = uv[2 * e], v0 = uv[2 * e + 1];
    if (tid == 0) {
        if (own) {
            double y[3];
            interp_pos(X, p, u0, v0, y);
            sX[0] = y[0]; sX[1] = y[1]; sX[2] = y[2];
        } else {
            sX[0] = xe[3 * e]; sX[1] = xe[3 * e + 1]; sX[2] = xe[3 * e + 2];
        }
    }
    __syncthreads();
    for (int k = tid; k < pp; k += kQThreads) {
        const size_t gk = (size_t)P * pp + k;
        sD[k] = x[3 * gk] - sX[0];
        sD[pp + k] = x[3 * gk + 1] - sX[1];
        sD[2 * pp + k] = x[3 * gk + 2] - sX[2];
        sJ[k] = J[gk];
    }
    __syncthreads();
    const int a_own = tid / p, b_own = tid - (tid / p) * p;
    double acc = 0.0;
    double* sLu = sBuf;
    double* sLv = sBuf + kBvpPts * p;
    if (own) {
        // angular range of the directions entering [-1,1]^2 from the edge point
        if (tid == 0) {
            double lo, hi;
            if (fabs(u0 + 1.0) < 1e-12) { lo = -0.5 * M_PI; hi = 0.5 * M_PI; }
            else if (fabs(u0 - 1.0) < 1e-12) { lo = 0.5 * M_PI; hi = 1.5 * M_PI; }
            else if (fabs(v0 + 1.0) < 1e-12) { lo = 0.0; hi = M_PI; }
            else { lo = M_PI; hi = 2.0 * M_PI; }
            int nc = 0;
            sCut[nc++] = lo;
            const double cu[4] = {1.0, -1.0, -1.0, 1.0}, cv[4] = {1.0, 1.0, -1.0, -1.0};
            for (int c = 0; c < 4; ++c) {
                const double th = atan2(cv[c] - v0, cu[c] - u0);
                for (int k = -1; k <= 2; ++k) {
                    const double tt = th + 2.0 * M_PI * k;
                    if (tt > lo + 1e-12 && tt < hi - 1e-12 && nc < 7) sCut[nc++] = tt;
                }
            }
            sCut[nc++] = hi;
            for (int i = 1; i < nc; ++i)          // insertion sort
                for (int j = i; j > 0 && sCut[j] < sCut[j - 1]; --j) {
                    const double t = sCut[j]; sCut[j] = sCut[j - 1]; sCut[j - 1] = t;
                }
            sNcut = nc;
        }
        __syncthreads();
        const int nc = sNcut;
        for (int seg = 0; seg + 1 < nc; ++seg) {
            const double A = sCut[seg], B = sCut[seg + 1];
            const int nsub = max(1, (int)ceil((B - A) / (M_PI / 32.0) - 1e-9));
            for (int sub = 0; sub < nsub; ++sub) {
                const double s0 = A + (B - A) * sub / nsub, s1 = A + (B - A) * (sub + 1) / nsub;
                const double hs = 0.5 * (s1 - s0);
                const int nrp = log_kernel ? kBvpLogLevels + 1 : 2;
                for (int rp = 0; rp < nrp; ++rp) {
                    for (int half = 0; half < 2; ++half) {
                        // point tid: theta node 8 half + tid / 16, radial node tid % 16
                        {
                            const int qt = 8 * half + tid / PM_GL16, qr = tid % PM_GL16;
                            const double th = s0 + hs * (cT.g16t[qt] + 1.0);
                            const double ct = cos(th), st = sin(th);
                            const double L = bvp_ray(u0, v0, ct, st);
                            double r0, r1;
                            if (log_kernel) {
                                r0 = rp == 0 ? 0.0 : L * ldexp(1.0, rp - 1 - kBvpLogLevels);
                                r1 = L * ldexp(1.0, rp - kBvpLogLevels);
                            } else {
                                r0 = rp == 0 ? 0.0 : 0.25 * L;
                                r1 = rp == 0 ? 0.25 * L : L;
                            }
                            const double hr = 0.5 * (r1 - r0);
                            const double rho = r0 + hr * (cT.g16t[qr] + 1.0);
                            const double u = u0 + rho * ct, v = v0 + rho * st;
                            double* lu = sLu + tid * p;
                            double* lv = sLv + tid * p;
                            lagrange(u, p, lu);
                            lagrange(v, p, lv);
                            double d0 = 0, d1 = 0, d2 = 0, jj = 0;
                            for (int a = 0; a < p; ++a) {
                                double z0 = 0, z1 = 0, z2 = 0, zj = 0;
                                for (int b = 0; b < p; ++b) {
                                    const double l = lv[b];
                                    z0 += sD[a * p + b] * l;
                                    z1 += sD[pp + a * p + b] * l;
                                    z2 += sD[2 * pp + a * p + b] * l;
                                    zj += sJ[a * p + b] * l;
                                }
                                d0 += lu[a] * z0; d1 += lu[a] * z1; d2 += lu[a] * z2; jj += lu[a] * zj;
                            }
                            // r = x - y = -(y - x)
                            const double r2 = d0 * d0 + d1 * d1 + d2 * d2;
                            const double nr = -(n0 * d0 + n1 * d1 + n2 * d2);
                            const double wgt = hs * cT.g16w[qt] * hr * cT.g16w[qr] * rho * jj;
                            sF[tid] = !(r2 > 0.0) ? 0.0
                                      : log_kernel ? wgt * log(r2) * (0.25 / M_PI)
                                                   : wgt * nr / r2 * (0.5 / M_PI);
                        }
                        __syncthreads();
                        if (tid < pp)
                            for (int q = 0; q < kBvpPts; ++q)
                                acc += sF[q] * sLu[q * p + a_own] * sLv[q * p + b_own];
                        __syncthreads();
                    }
                }
            }
        }
    } else {
        double* sLu16 = sBuf;
        double* sLv16 = sBuf + PM_GL16 * p;
        double* sZ = sBuf + 2 * PM_GL16 * p;             // [4][a][r]
        double* sG = sF;
        const int nleaves = near_leaves(X, p, sX[0], sX[1], sX[2], eta, max_depth, max_leaves, bfs,
                                        err);
        for (int Lf = 0; Lf < nleaves; ++Lf) {
            double uu0, uu1, vv0, vv1;
            sq_box(bfs.sorted[Lf], uu0, uu1, vv0, vv1);
            const double hu = 0.5 * (uu1 - uu0), hv = 0.5 * (vv1 - vv0);
            if (tid < PM_GL16) lagrange(uu0 + hu * (cT.g16t[tid] + 1.0), p, sLu16 + tid * p);
            else if (tid < 2 * PM_GL16)
                lagrange(vv0 + hv * (cT.g16t[tid - PM_GL16] + 1.0), p, sLv16 + (tid - PM_GL16) * p);
            __syncthreads();
            for (int q = tid; q < 4 * p * PM_GL16; q += kQThreads) {
                const int c = q / (p * PM_GL16), rem = q - c * p * PM_GL16;
                const int a = rem / PM_GL16, r = rem - a * PM_GL16;
                const double* src = (c < 3) ? (sD + c * pp) : sJ;
                double z = 0;
                for (int bb = 0; bb < p; ++bb) z += src[a * p + bb] * sLv16[r * p + bb];
                sZ[(c * p + a) * PM_GL16 + r] = z;
            }
            __syncthreads();
            for (int q = tid; q < PM_GL16 * PM_GL16; q += kQThreads) {
                const int qn = q / PM_GL16, r = q - qn * PM_GL16;
                double d0 = 0, d1 = 0, d2 = 0, jj = 0;
                for (int a = 0; a < p; ++a) {
                    const double l = sLu16[qn * p + a];
                    d0 += l * sZ[(0 * p + a) * PM_GL16 + r];
                    d1 += l * sZ[(1 * p + a) * PM_GL16 + r];
                    d2 += l * sZ[(2 * p + a) * PM_GL16 + r];
                    jj += l * sZ[(3 * p + a) * PM_GL16 + r];
                }
                const double r2 = d0 * d0 + d1 * d1 + d2 * d2;
                const double nr = -(n0 * d0 + n1 * d1 + n2 * d2);
                const double wgt = hu * cT.g16w[qn] * hv * cT.g16w[r] * jj;
                sG[q] = log_kernel ? wgt * log(r2) * (0.25 / M_PI) : wgt * nr / r2 * (0.5 / M_PI);
            }
            __syncthreads();
            if (tid < pp)
                for (int r = 0; r < PM_GL16; ++r) {
                    double t = 0;
                    for (int qn = 0; qn < PM_GL16; ++qn) t += sG[qn * PM_GL16 + r] * sLu16[qn * p + a_own];
                    acc += t * sLv16[r * p + b_own];
                }
            __syncthreads();
        }
    }
    if (tid < pp) W[(size_t)blk * pp + tid] = acc;
}
}  // namespace

// The quadrature tables live in one __constant__ copy per device, written here
// for the surface's order p: builds are serialised (several host threads may
// create surfaces at once, e.g. the server's workers).
static std::mutex g_near_build_mu;

pm_status pm_near_build(pm_surface* s, const QuadTables& T) {
    std::lock_guard<std::mutex> build_lock(g_near_build_mu);
    const int N = s->N, npatch = s->npatch, p = s->p, pp = s->pp;
    PM_CUDA_TRY(cudaMemcpyToSymbol(cT, &T, sizeof(QuadTables)));
    PM_TRY(pm_dmalloc(&s->centroid, 3 * (size_t)npatch));
    PM_TRY(pm_dmalloc(&s->radius, npatch));
    PM_TRY(pm_dmalloc(&s->npatch_n, 3 * (size_t)N));
    k_patch_geom<<<pm_ceil_div(npatch, 128), 128>>>(s->x, npatch, p, s->centroid, s->radius);
    k_node_normals<<<pm_ceil_div(N, 128), 128>>>(s->x, N, p, s->npatch_n);
    PM_CUDA_TRY(cudaGetLastError());
    PM_TRY(pm_near_structure(s));
    const size_t smem = sizeof(double) * (4 * (size_t)pp + 2 * (size_t)kQThreads * p + 5 * kQThreads);
    if (smem > 48 * 1024)
        PM_CUDA_TRY(cudaFuncSetAttribute(k_self_quad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem));
    k_self_quad<<<N, kQThreads, smem>>>(N, p, s->x, s->J, s->npatch_n, s->H, s->th_off,
                                        s->th_ang, s->th_w, s->th_L, s->row_ptr, s->nblk,
                                        s->W_lb, s->W_g, s->W_k);
    PM_CUDA_TRY(cudaGetLastError());
    k_near_quad<<<s->nblk, kQThreads>>>(p, s->nblk, s->x, s->J, s->n, s->H, s->blk_row,
                                        s->blk_patch, s->row_ptr, s->opts.near_eta,
                                        std::min(s->opts.near_max_depth, 12),
                                        s->opts.near_max_leaves, s->W_lb, s->W_g, s->W_k,
                                        s->dev_err);
    PM_CUDA_TRY(cudaGetLastError());
    PM_CUDA_TRY(cudaDeviceSynchronize());
    int herr = 0;
    PM_CUDA_TRY(cudaMemcpy(&herr, s->dev_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (herr != PM_DEV_OK) {
        pm_set_error("near-field quadrature: device check %d failed (leaf budget exceeded)", herr);
        return PM_ERR_INTERNAL;
    }
    return PM_OK;
}

// The near-field structure from the patch centroids and radii: per target its
// own patch first, then every patch within near_factor radii (CSR over blocks),
// each patch's union of its rows' near patches, the compactness test of the
// float32 parametrix sum's centred form, and the coefficient-free weight sets.
pm_status pm_near_structure(pm_surface* s) {
    const int N = s->N, npatch = s->npatch, pp = s->pp;
    PM_TRY(pm_dmalloc(&s->row_ptr, (size_t)N + 1));
    PM_TRY(pm_dmalloc(&s->dev_err, 1));
    PM_CUDA_TRY(cudaMemset(s->dev_err, 0, sizeof(int)));
    int* count = nullptr;
    PM_TRY(pm_dmalloc(&count, N));
    k_near_count<<<pm_ceil_div(N, 128), 128>>>(s->x, s->centroid, s->radius, N, npatch, pp,
                                                s->opts.near_factor, count);
    PM_CUDA_TRY(cudaGetLastError());
    std::vector<int> hc(N), hr(N + 1);
    cudaError_t e = cudaMemcpy(hc.data(), count, sizeof(int) * N, cudaMemcpyDeviceToHost);
    cudaFree(count);
    if (e != cudaSuccess) {
        pm_set_error("near count copy: %s", cudaGetErrorString(e));
        return PM_ERR_CUDA;
    }
    hr[0] = 0;
    for (int i = 0; i < N; ++i) {
        if (hc[i] < 1 || hc[i] > npatch) {
            pm_set_error("near list count %d out of range at row %d", hc[i], i);
            return PM_ERR_INTERNAL;
        }
        hr[i + 1] = hr[i] + hc[i];
    }
    s->nblk = hr[N];
    PM_CUDA_TRY(cudaMemcpy(s->row_ptr, hr.data(), sizeof(int) * (N + 1), cudaMemcpyHostToDevice));
    PM_TRY(pm_dmalloc(&s->blk_patch, s->nblk));
    PM_TRY(pm_dmalloc(&s->blk_row, s->nblk));
    k_near_fill<<<pm_ceil_div(N, 128), 128>>>(s->x, s->centroid, s->radius, N, npatch, pp,
                                               s->opts.near_factor, s->row_ptr, s->blk_patch,
                                               s->blk_row);
    PM_CUDA_TRY(cudaGetLastError());
    // near-patch unions of every patch (the multi-instance solve's patch-blocked
    // near field, pm_batch.cu k_mnear32_patch)
    {
        std::vector<int> bp(s->nblk);
        PM_CUDA_TRY(cudaMemcpy(bp.data(), s->blk_patch, sizeof(int) * s->nblk,
                               cudaMemcpyDeviceToHost));
        std::vector<int> ptr(npatch + 1, 0), list, bu(s->nblk, 0), un;
        int umax = 0;
        for (int P = 0; P < npatch; ++P) {
            un.assign(bp.begin() + hr[P * pp], bp.begin() + hr[(P + 1) * pp]);
            std::sort(un.begin(), un.end());
            un.erase(std::unique(un.begin(), un.end()), un.end());
            for (int b = hr[P * pp]; b < hr[(P + 1) * pp]; ++b)
                bu[b] = (int)(std::lower_bound(un.begin(), un.end(), bp[b]) - un.begin());
            list.insert(list.end(), un.begin(), un.end());
            ptr[P + 1] = (int)list.size();
            umax = std::max(umax, (int)un.size());
        }
        PM_TRY(pm_dmalloc(&s->nu_ptr, ptr.size()));
        PM_TRY(pm_dmalloc(&s->nu_list, std::max<size_t>(1, list.size())));
        PM_TRY(pm_dmalloc(&s->nu_blk, std::max<size_t>(1, bu.size())));
        PM_CUDA_TRY(cudaMemcpy(s->nu_ptr, ptr.data(), sizeof(int) * ptr.size(), cudaMemcpyHostToDevice));
        PM_CUDA_TRY(cudaMemcpy(s->nu_list, list.data(), sizeof(int) * list.size(), cudaMemcpyHostToDevice));
        PM_CUDA_TRY(cudaMemcpy(s->nu_blk, bu.data(), sizeof(int) * bu.size(), cudaMemcpyHostToDevice));
        s->nu_max = umax;
    }
    // Is the centred form of the float32 parametrix sum safe here (pm_direct.cu)?
    // Every tile of 512 consecutive nodes must be compact: R^2 <= 0.03 |Gamma| and
    // R^2 <= r_min^2 / (80 eps), eps = 2^-24, r_min the smallest node distance.
    {
        unsigned int* mm = nullptr;
        PM_TRY(pm_dmalloc(&mm, 2));
        const unsigned int init[2] = {0x7f7fffffu, 0u};      // FLT_MAX, +0
        cudaError_t ce = cudaMemcpy(mm, init, sizeof(init), cudaMemcpyHostToDevice);
        if (ce == cudaSuccess) {
            k_near_min_dist<<<s->nblk, 64>>>(s->x, s->blk_row, s->blk_patch, pp, mm);
            k_tile_radius<<<pm_ceil_div(N, 512), 256>>>(s->x, N, 512, mm + 1);
            ce = cudaGetLastError();
        }
        unsigned int got[2] = {0u, 0u};
        if (ce == cudaSuccess) ce = cudaMemcpy(got, mm, sizeof(got), cudaMemcpyDeviceToHost);
        cudaFree(mm);
        if (ce != cudaSuccess) {
            pm_set_error("near build (tile radii): %s", cudaGetErrorString(ce));
            return PM_ERR_CUDA;
        }
        float rmin2 = 0.f, tile2 = 0.f;
        std::memcpy(&rmin2, &got[0], sizeof(float));
        std::memcpy(&tile2, &got[1], sizeof(float));
        double area = 0.0;
        for (double v : s->h_w) area += v;
        const double eps = std::ldexp(1.0, -24);
        s->k32_centred = (N > 1 && tile2 <= 0.03 * area && (double)tile2 * 80.0 * eps <= rmin2) ? 1 : 0;
    }
    const size_t nv = (size_t)s->nblk * pp;
    PM_TRY(pm_dmalloc(&s->W_lb, nv));
    PM_TRY(pm_dmalloc(&s->W_g, 3 * nv));
    PM_TRY(pm_dmalloc(&s->W_k, nv));
    return PM_OK;
}

pm_status pm_near_combine_coeff(pm_surface* s, cudaStream_t st) {
    const size_t ne = (size_t)s->nblk * s->ppad;
    k_combine<<<pm_ceil_div((long long)ne, 256), 256, 0, st>>>(
        s->nblk, s->pp, s->ppad, s->blk_row, s->blk_patch, s->x, s->n, s->H, s->w, s->a, s->g,
        s->W_lb, s->W_g, s->W_k, s->cR64, s->cK64, s->cR32, s->cK32);
    PM_CUDA_TRY(cudaGetLastError());
    return PM_OK;
}

pm_status pm_near_apply(pm_surface* s, int which_K, const double* sigma, double* out,
                        int use_near, int nsplit, pm_precision prec, cudaStream_t st) {
    const int N = s->N;
    const int threads = 256;
    const int blocks = pm_ceil_div((long long)N * 32, threads);       // float64: warp per row
    // float32: a lane group per row, a warp while the rows fit in one wave of warps
    const bool one_wave = (long long)N * 32 <= (long long)s->ctx->num_sms * 2048;
    if (prec == PM_PREC_FF && nsplit > 32) {
        // many float-float slices: summed coalesced first, then the corrections added
        k_sum_slices_ff<<<pm_ceil_div(N, 256), 256, 0, st>>>(
            N, nsplit, reinterpret_cast<const float2*>(s->partial), out, s->skip_flag);
        k_near_apply64<<<blocks, threads, 0, st>>>(N, s->pp, s->row_ptr, s->blk_patch,
                                                   which_K ? s->cK64 : s->cR64, sigma, s->partial,
                                                   0, 1, use_near, 1, out, s->skip_flag);
        s->launch_total++;
    } else if (prec == PM_PREC_FP64 || prec == PM_PREC_FF)
        k_near_apply64<<<blocks, threads, 0, st>>>(N, s->pp, s->row_ptr, s->blk_patch,
                                                   which_K ? s->cK64 : s->cR64, sigma,
                                                   s->partial, nsplit, prec == PM_PREC_FF ? 1 : 0,
                                                   use_near, 0, out,
                                                   s->skip_flag);
    else
        (one_wave ? k_near_apply32<32, 4> : k_near_apply32<8, 4>)
            <<<pm_ceil_div((long long)N * (one_wave ? 32 : 8), threads), threads, 0, st>>>(
                N, s->ppad, s->row_ptr, s->blk_patch, which_K ? s->cK32 : s->cR32, s->sig32,
                reinterpret_cast<const float2*>(s->partial), nsplit, use_near, out, s->skip_flag);
    PM_CUDA_TRY(cudaGetLastError());
    return PM_OK;
}

// Complex corrections of the c != 0 operators (weights with the coefficients,
// then minus the smooth rule's node terms), into s->cRc, s->cKc.
pm_status pm_near_build_c(pm_surface* s) {
    std::lock_guard<std::mutex> build_lock(g_near_build_mu);
    const int N = s->N, p = s->p, pp = s->pp;
    QuadTables T;
    pm_build_tables(p, &T);
    PM_CUDA_TRY(cudaMemcpyToSymbol(cT, &T, sizeof(QuadTables)));
    PM_CUDA_TRY(pm_green::upload_cheb_k01());
    PM_CUDA_TRY(cudaMemset(s->dev_err, 0, sizeof(int)));
    const size_t smem = sizeof(double) * (6 * (size_t)pp + 2 * (size_t)kQThreads * p + 4 * kQThreads);
    if (smem > 48 * 1024)
        PM_CUDA_TRY(cudaFuncSetAttribute(k_self_quad_c, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem));
    k_self_quad_c<<<N, kQThreads, smem>>>(N, p, s->x, s->J, s->npatch_n, s->H, s->a, s->g, s->cc,
                                          s->qn, s->th_off, s->th_ang, s->th_w, s->th_L,
                                          s->row_ptr, s->cRc, s->cKc);
    PM_CUDA_TRY(cudaGetLastError());
    k_near_quad_c<<<s->nblk, kQThreads>>>(p, s->x, s->J, s->n, s->H, s->a, s->g, s->cc, s->qn,
                                          s->blk_row, s->blk_patch, s->row_ptr, s->opts.near_eta,
                                          std::min(s->opts.near_max_depth, 12),
                                          s->opts.near_max_leaves, s->cRc, s->cKc, s->dev_err);
    PM_CUDA_TRY(cudaGetLastError());
    const size_t ne = (size_t)s->nblk * pp;
    k_combine_c<<<pm_ceil_div((long long)ne, 256), 256>>>(s->nblk, pp, s->blk_row, s->blk_patch,
                                                          s->x, s->n, s->H, s->w, s->a, s->g,
                                                          s->cc, s->qn, s->cRc, s->cKc);
    PM_CUDA_TRY(cudaGetLastError());
    PM_CUDA_TRY(cudaDeviceSynchronize());
    int herr = 0;
    PM_CUDA_TRY(cudaMemcpy(&herr, s->dev_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (herr != PM_DEV_OK) {
        pm_set_error("c != 0 near-field quadrature: device check %d failed (leaf budget exceeded)", herr);
        return PM_ERR_INTERNAL;
    }
    return PM_OK;
}

// Surface-integral weights at the edge nodes of a boundary-value system (pm_bvp.cu):
// K'_Gamma (log_kernel = 0) or K_Gamma (log_kernel = 1); one block per (edge node,
// patch) pair of the device lists; W [nb][p*p].
pm_status pm_bvp_kp_weights(pm_surface* s, int nb, const int* blk_edge, const int* blk_patch,
                            const int* blk_own, const double* xe, const double* nue,
                            const double* uv, int log_kernel, double* W) {
    std::lock_guard<std::mutex> build_lock(g_near_build_mu);
    if (nb == 0) return PM_OK;
    QuadTables T;
    pm_build_tables(s->p, &T);
    PM_CUDA_TRY(cudaMemcpyToSymbol(cT, &T, sizeof(QuadTables)));
    PM_CUDA_TRY(cudaMemset(s->dev_err, 0, sizeof(int)));
    k_bvp_kp_quad<<<nb, kQThreads>>>(s->p, s->x, s->J, blk_edge, blk_patch, blk_own, xe, nue, uv,
                                     log_kernel, s->opts.near_eta, std::min(s->opts.near_max_depth, 12),
                                     s->opts.near_max_leaves, W, s->dev_err);
    PM_CUDA_TRY(cudaGetLastError());
    PM_CUDA_TRY(cudaDeviceSynchronize());
    int herr = 0;
    PM_CUDA_TRY(cudaMemcpy(&herr, s->dev_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (herr != PM_DEV_OK) {
        pm_set_error("edge-node quadrature: device check %d failed (leaf budget exceeded)", herr);
        return PM_ERR_INTERNAL;
    }
    return PM_OK;
}
