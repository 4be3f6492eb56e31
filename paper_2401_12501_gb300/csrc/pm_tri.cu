// Triangle patches (Sec. 6.1): surfaces whose patches are curved triangles over
// the reference simplex T0 = {u, v >= 0, u + v <= 1}, sampled at the nodes of an
// order-p rule (the paper's Vioreanu-Rokhlin nodes, or any unisolvent set of
// p (p + 1) / 2 points the caller gives).
//
// Only the near field depends on the patch shape.  The interpolant of node data
// on a patch is sum_k f_k l_k(u, v), with l_k the Lagrange basis of the nodes in
// the polynomials of total degree <= p - 1, written through the Koornwinder
// basis K_n (Sec. 6.1.2): l_k = sum_n U[n][k] K_n, U the inverse of
// V[j][n] = K_n(u_j, v_j).  It gives the patch geometry from the node positions
// (y~), the surface element from the nodal |y_u x y_v| (J~) and the density, as
// the tensor Lagrange basis does on quadrilaterals, and the quadrature rules
// write the same coefficient-free weight sets W_lb, W_g, W_k (pm_nearfield.cu),
// so coefficients, smooth sums, FMM, solves, batches and the server are shared.
//
//   self patch (Sec. 6.1.1, eq. radial_int): polar coordinates about the
//     target's node; theta split at the directions of T0's three vertices,
//     panels adaptive on int L^2 and capped in width (host plan); the radial
//     panels and product-log weights of the quadrilateral rule; the curvature
//     terms use the interpolated patch's unit normal at the target;
//   near patches (Sec. 6.1.2): midpoint subdivision of T0 into four triangles
//     while the target lies within 2 eta of a sub-triangle's size from its
//     centroid image, a 16 x 16 collapsed Gauss rule on each leaf.
//
// K_{m,k}(u, v) = A_m(u, v) B_k^{(2m+1)}(2v - 1), m + k <= p - 1, with
// A_m = P_m((2u + v - 1)/(1 - v)) (1 - v)^m computed without the division by the
// homogeneous recurrence (m + 1) A_{m+1} = (2m + 1) a A_m - m b^2 A_{m-1}
// (a = 2u + v - 1, b = 1 - v) and B_k^{(alpha)} the Jacobi polynomials
// P_k^{(alpha, 0)} by their three-term recurrence; unnormalised (U absorbs the
// scale), in the order m = 0..n, k = 0..n - m.
#include "pm_internal.cuh"

#include <algorithm>
#include <cmath>
#include <functional>
#include <mutex>
#include <vector>

namespace {

// ------------------------------------------------------------------ the basis (host and device)
// Forward-mode derivative: a value and its derivative along one direction, so that
// the recurrences below give d K / du and d K / dv exactly (to rounding).
struct Dual {
    double v, d;
    __host__ __device__ Dual(double x = 0.0, double dx = 0.0) : v(x), d(dx) {}
};
__host__ __device__ inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
__host__ __device__ inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
__host__ __device__ inline Dual operator*(Dual a, Dual b) {
    return Dual(a.v * b.v, a.d * b.v + a.v * b.d);
}
__host__ __device__ inline Dual operator+(Dual a, double b) { return Dual(a.v + b, a.d); }
__host__ __device__ inline Dual operator-(Dual a, double b) { return Dual(a.v - b, a.d); }
__host__ __device__ inline Dual operator-(double a, Dual b) { return Dual(a - b.v, -b.d); }
__host__ __device__ inline Dual operator*(double a, Dual b) { return Dual(a * b.v, a * b.d); }
__host__ __device__ inline Dual operator*(Dual a, double b) { return Dual(a.v * b, a.d * b); }
__host__ __device__ inline Dual operator/(Dual a, double b) { return Dual(a.v / b, a.d / b); }

template <typename T>
__host__ __device__ inline void koornwinder(int n, T u, T v, T* out) {
    const T a = 2.0 * u + v - 1.0, b = 1.0 - v, t = 2.0 * v - 1.0;
    T A[PM_TRI_MAX_P];
    A[0] = 1.0;
    if (n >= 1) A[1] = a;
    for (int m = 1; m < n; ++m)
        A[m + 1] = ((2.0 * m + 1.0) * a * A[m] - (double)m * b * b * A[m - 1]) / (m + 1.0);
    int pos = 0;
    for (int m = 0; m <= n; ++m) {
        const double al = 2.0 * m + 1.0;
        T b0 = 1.0, b1 = ((al + 2.0) * t + al) * 0.5;
        for (int k = 0; k <= n - m; ++k) {
            T bk;
            if (k == 0) {
                bk = b0;
            } else if (k == 1) {
                bk = b1;
            } else {
                // P_{j+1} from P_j, P_{j-1} with j = k - 1 (beta = 0)
                const double j = k - 1.0;
                const double c2 = 2.0 * j + al;
                bk = ((c2 + 1.0) * ((c2 + 2.0) * c2 * t + al * al) * b1 -
                      2.0 * j * (j + al) * (c2 + 2.0) * b0) /
                     (2.0 * (j + 1.0) * (j + al + 1.0) * c2);
                b0 = b1;
                b1 = bk;
            }
            out[pos++] = A[m] * bk;
        }
    }
}

double ray_length_tri(double u0, double v0, double th) {
    const double c = std::cos(th), s = std::sin(th);
    double L = INFINITY;
    if (c < 0) L = std::min(L, -u0 / c);
    if (s < 0) L = std::min(L, -v0 / s);
    if (c + s > 0) L = std::min(L, (1.0 - u0 - v0) / (c + s));
    return L;
}

// ------------------------------------------------------------------ device side
struct TriConst {
    int p, n, nt;
    double U[PM_TRI_MAX_NT * PM_TRI_MAX_NT];
    double g16t[PM_GL16], g16w[PM_GL16], logE[PM_GL16];
};
__constant__ TriConst cTri;

constexpr int kTT = 128;            // threads (quadrature points per chunk) of the kernels
constexpr int kTriMaxLevel = 1024;  // sub-triangles per BFS level
constexpr int kTriMaxLeaves = 512;

// l_k(u, v) for all nodes
__device__ inline void tri_basis(double u, double v, double* l) {
    double K[PM_TRI_MAX_NT];
    koornwinder<double>(cTri.n, u, v, K);
    const int nt = cTri.nt;
    for (int k = 0; k < nt; ++k) {
        double acc = 0.0;
        for (int m = 0; m < nt; ++m) acc += K[m] * cTri.U[m * nt + k];
        l[k] = acc;
    }
}

__device__ inline void tri_pos(const double* X, double u, double v, double* y) {
    double l[PM_TRI_MAX_NT];
    tri_basis(u, v, l);
    double y0 = 0, y1 = 0, y2 = 0;
    for (int k = 0; k < cTri.nt; ++k) {
        y0 += l[k] * X[3 * k];
        y1 += l[k] * X[3 * k + 1];
        y2 += l[k] * X[3 * k + 2];
    }
    y[0] = y0; y[1] = y1; y[2] = y2;
}

// centroid and radius from the images of T0's vertices (Sec. 6.1.2 near test)
__global__ void k_patch_geom_tri(const double* __restrict__ x, int npatch,
                                 double* __restrict__ centroid, double* __restrict__ radius) {
    const int P = blockIdx.x * blockDim.x + threadIdx.x;
    if (P >= npatch) return;
    const double* X = x + (size_t)3 * P * cTri.nt;
    const double cu[3] = {0.0, 1.0, 0.0}, cv[3] = {0.0, 0.0, 1.0};
    double c[3][3];
    for (int k = 0; k < 3; ++k) tri_pos(X, cu[k], cv[k], c[k]);
    double m[3];
    for (int d = 0; d < 3; ++d) m[d] = (c[0][d] + c[1][d] + c[2][d]) / 3.0;
    double r = 0;
    for (int k = 0; k < 3; ++k) {
        const double dx = c[k][0] - m[0], dy = c[k][1] - m[1], dz = c[k][2] - m[2];
        r = fmax(r, sqrt(dx * dx + dy * dy + dz * dz));
    }
    for (int d = 0; d < 3; ++d) centroid[3 * P + d] = m[d];
    radius[P] = r;
}

// unit normal of the interpolated patch at each node, from the derivative matrices
__global__ void k_node_normals_tri(const double* __restrict__ x, int N, int nt,
                                   const double* __restrict__ Du, const double* __restrict__ Dv,
                                   double* __restrict__ nn) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const int P = k / nt, j = k - P * nt;
    const double* X = x + (size_t)3 * P * nt;
    double yu[3] = {0, 0, 0}, yv[3] = {0, 0, 0};
    for (int m = 0; m < nt; ++m) {
        const double du = Du[j * nt + m], dv = Dv[j * nt + m];
        for (int c = 0; c < 3; ++c) {
            yu[c] += du * X[3 * m + c];
            yv[c] += dv * X[3 * m + c];
        }
    }
    const double c0 = yu[1] * yv[2] - yu[2] * yv[1];
    const double c1 = yu[2] * yv[0] - yu[0] * yv[2];
    const double c2 = yu[0] * yv[1] - yu[1] * yv[0];
    const double inv = 1.0 / sqrt(c0 * c0 + c1 * c1 + c2 * c2);
    nn[3 * k] = c0 * inv;
    nn[3 * k + 1] = c1 * inv;
    nn[3 * k + 2] = c2 * inv;
}

// One chunk of up to kTT quadrature points: each thread has put its point's basis
// into sL[tid][.] and its five integrand values into sF[.][tid]; threads k < nt add
// sum_q F[.][q] l_k(q) to their accumulators.
__device__ inline void tri_accumulate(const double* sL, const double* sF, int lim, int nt,
                                      double* acc) {
    const int tid = threadIdx.x;
    if (tid < nt) {
        for (int q = 0; q < lim; ++q) {
            const double l = sL[q * nt + tid];
            for (int c = 0; c < 5; ++c) acc[c] += sF[c * kTT + q] * l;
        }
    }
}

// The five coefficient-free integrands (pm_nearfield.cu) at one point, r = x - y~.
__device__ inline void tri_integrands(double rx, double ry, double rz, double n0, double n1,
                                      double n2, double Hi, double wgt, double logc, double* f) {
    const double r2 = rx * rx + ry * ry + rz * rz;
    const double inv = 1.0 / r2;
    const double qq = (n0 * rx + n1 * ry + n2 * rz) * inv;
    f[0] = wgt * (qq * qq - Hi * qq) * (1.0 / M_PI);
    const double gfac = wgt * inv * (0.5 / M_PI);
    f[1] = gfac * rx;
    f[2] = gfac * ry;
    f[3] = gfac * rz;
    f[4] = wgt * (0.5 * log(r2) + logc) * (0.5 / M_PI);
}

// Self patch.  The polar points depend only on the target's node position in its
// patch, so one block takes kTriG targets at the same position in consecutive
// patches: each point's basis values (the costly part: nt^2 products with U) are
// computed once for all of them, then each target's offsets and element give its
// integrands.  The (target, node) accumulators are spread over the block's threads;
// every target's sum runs over the points in the same order as with one target a
// block.  Dynamic shared memory (doubles): basis [kTT][nt], integrands
// [kTriG][5][kTT], offsets [kTriG][3][nt], elements [kTriG][nt].
constexpr int kTriG = 8;
constexpr int kTriAccPerThread = (kTriG * PM_TRI_MAX_NT + kTT - 1) / kTT;

__global__ void __launch_bounds__(kTT)
k_self_quad_tri(int npatch, const double* __restrict__ x, const double* __restrict__ J,
                const double* __restrict__ nn, const double* __restrict__ H,
                const double* __restrict__ ref_u, const double* __restrict__ ref_v,
                const int* __restrict__ th_off, const double* __restrict__ th_ang,
                const double* __restrict__ th_w, const double* __restrict__ th_L,
                const int* __restrict__ row_ptr, int nblk, double* __restrict__ W_lb,
                double* __restrict__ W_g, double* __restrict__ W_k) {
    extern __shared__ double sm[];
    const int nt = cTri.nt;
    const int loc = blockIdx.y, tid = threadIdx.x;   // x: patch groups (no 65,535 cap)
    const int P0 = blockIdx.x * kTriG;
    const int G = min(kTriG, npatch - P0);
    double* sL = sm;                                   // [kTT][nt]
    double* sF = sL + kTT * nt;                        // [kTriG][5][kTT]
    double* sD = sF + kTriG * 5 * kTT;                 // [kTriG][3][nt]
    double* sJ = sD + kTriG * 3 * nt;                  // [kTriG][nt]
    for (int e = tid; e < G * nt; e += kTT) {
        const int g = e / nt, k = e - (e / nt) * nt;
        const size_t i = (size_t)(P0 + g) * nt + loc, gk = (size_t)(P0 + g) * nt + k;
        sD[(g * 3 + 0) * nt + k] = x[3 * gk] - x[3 * i];
        sD[(g * 3 + 1) * nt + k] = x[3 * gk + 1] - x[3 * i + 1];
        sD[(g * 3 + 2) * nt + k] = x[3 * gk + 2] - x[3 * i + 2];
        sJ[g * nt + k] = J[gk];
    }
    const double u0 = ref_u[loc], v0 = ref_v[loc];
    const int t0 = th_off[loc], t1 = th_off[loc + 1];
    const int npts = (t1 - t0) * (PM_RADIAL_PANELS * PM_GL16);
    const double lo_f[4] = {0.0, 0.125, 0.25, 0.5};
    const double hi_f[4] = {0.125, 0.25, 0.5, 1.0};
    double acc[kTriAccPerThread][5];
    for (int m = 0; m < kTriAccPerThread; ++m)
        for (int c = 0; c < 5; ++c) acc[m][c] = 0.0;
    __syncthreads();
    for (int base = 0; base < npts; base += kTT) {
        const int q = base + tid;
        double* l = sL + tid * nt;
        if (q < npts) {
            const int kth = t0 + q / (PM_RADIAL_PANELS * PM_GL16);
            const int rj = q % (PM_RADIAL_PANELS * PM_GL16);
            const int panel = rj / PM_GL16, node = rj % PM_GL16;
            const double L = th_L[kth];
            const double h = (hi_f[panel] - lo_f[panel]) * L;
            const double r = lo_f[panel] * L + 0.5 * h * (cTri.g16t[node] + 1.0);
            const double wr = 0.5 * h * cTri.g16w[node];
            double sn, cs;
            sincos(th_ang[kth], &sn, &cs);
            tri_basis(u0 + r * cs, v0 + r * sn, l);
            const double wpt = th_w[kth] * wr * r;
            const double logc = panel == 0 ? cTri.logE[node] : 0.0;
            for (int g = 0; g < kTriG; ++g) {
                double f[5] = {0, 0, 0, 0, 0};
                if (g < G) {
                    const double* D = sD + g * 3 * nt;
                    const double* Jg = sJ + g * nt;
                    double d0 = 0, d1 = 0, d2 = 0, jj = 0;
                    for (int k = 0; k < nt; ++k) {
                        d0 += l[k] * D[k];
                        d1 += l[k] * D[nt + k];
                        d2 += l[k] * D[2 * nt + k];
                        jj += l[k] * Jg[k];
                    }
                    const size_t i = (size_t)(P0 + g) * nt + loc;
                    tri_integrands(-d0, -d1, -d2, nn[3 * i], nn[3 * i + 1], nn[3 * i + 2], H[i],
                                   wpt * jj, logc, f);
                }
                for (int c = 0; c < 5; ++c) sF[(g * 5 + c) * kTT + tid] = f[c];
            }
        } else {
            for (int k = 0; k < nt; ++k) l[k] = 0.0;
            for (int g = 0; g < kTriG; ++g)
                for (int c = 0; c < 5; ++c) sF[(g * 5 + c) * kTT + tid] = 0.0;
        }
        __syncthreads();
        const int lim = min(kTT, npts - base);
        for (int m = 0; m < kTriAccPerThread; ++m) {
            const int pr = tid + m * kTT;
            if (pr >= G * nt) break;
            const int g = pr / nt, k = pr - (pr / nt) * nt;
            for (int e = 0; e < lim; ++e) {
                const double lv = sL[e * nt + k];
                for (int c = 0; c < 5; ++c) acc[m][c] += sF[(g * 5 + c) * kTT + e] * lv;
            }
        }
        __syncthreads();
    }
    for (int m = 0; m < kTriAccPerThread; ++m) {
        const int pr = tid + m * kTT;
        if (pr >= G * nt) break;
        const int g = pr / nt, k = pr - (pr / nt) * nt;
        const size_t i = (size_t)(P0 + g) * nt + loc;
        const size_t b0 = (size_t)row_ptr[i];          // own patch: the row's first block
        W_lb[b0 * nt + k] = acc[m][0];
        W_g[(0 * (size_t)nblk + b0) * nt + k] = acc[m][1];
        W_g[(1 * (size_t)nblk + b0) * nt + k] = acc[m][2];
        W_g[(2 * (size_t)nblk + b0) * nt + k] = acc[m][3];
        W_k[b0 * nt + k] = acc[m][4];
    }
}

// Sub-triangle codes: level (4 bits) << 24 | child path (2 bits a level, first
// level in the high bits).  Children of (A, B, C): (A, AB, CA), (AB, B, BC),
// (CA, BC, C), (BC, CA, AB).
__device__ inline void tri_box(int code, double* tu, double* tv) {
    const int lev = code >> 24;
    double au = 0, av = 0, bu = 1, bv = 0, cu = 0, cv = 1;
    for (int l = 0; l < lev; ++l) {
        const int ch = (code >> (2 * (lev - 1 - l))) & 3;
        const double abu = 0.5 * (au + bu), abv = 0.5 * (av + bv);
        const double bcu = 0.5 * (bu + cu), bcv = 0.5 * (bv + cv);
        const double cau = 0.5 * (cu + au), cav = 0.5 * (cv + av);
        if (ch == 0) { bu = abu; bv = abv; cu = cau; cv = cav; }
        else if (ch == 1) { au = abu; av = abv; cu = bcu; cv = bcv; }
        else if (ch == 2) { au = cau; av = cav; bu = bcu; bv = bcv; }
        else { au = bcu; av = bcv; bu = cau; bv = cav; cu = abu; cv = abv; }
    }
    tu[0] = au; tv[0] = av; tu[1] = bu; tv[1] = bv; tu[2] = cu; tv[2] = cv;
}

// Shared memory of k_near_quad_tri: the subdivision's work lists are dead once the
// leaves are sorted, so they share storage with the points' basis values.
struct TriNearShared {
    double D[3 * PM_TRI_MAX_NT], J[PM_TRI_MAX_NT], X[3 * PM_TRI_MAX_NT];
    double F[5 * kTT];
    int sorted[kTriMaxLeaves];
    int nCur, nNext, nLeaf, overflow;
    union {
        double L[kTT * PM_TRI_MAX_NT];
        struct {
            int cur[kTriMaxLevel], next[kTriMaxLevel], leaf[kTriMaxLeaves];
        } bfs;
    } u;
};

// Near, non-self patches: one block per (target, patch) block.
__global__ void __launch_bounds__(kTT)
k_near_quad_tri(int nblk, const double* __restrict__ x, const double* __restrict__ J,
                const double* __restrict__ n, const double* __restrict__ H,
                const int* __restrict__ blk_row, const int* __restrict__ blk_patch,
                const int* __restrict__ row_ptr, double eta, int max_depth, int max_leaves,
                double* __restrict__ W_lb, double* __restrict__ W_g, double* __restrict__ W_k,
                int* __restrict__ err) {
    const int b = blockIdx.x;
    const int i = blk_row[b];
    if (b == row_ptr[i]) return;   // the self block is done by k_self_quad_tri
    const int nt = cTri.nt;
    const int P = blk_patch[b];
    const int tid = threadIdx.x;
    __shared__ TriNearShared S;
    double* sD = S.D;
    double* sJ = S.J;
    double* sX = S.X;
    double* sF = S.F;
    double* sL = S.u.L;
    const double xi0 = x[3 * i], xi1 = x[3 * i + 1], xi2 = x[3 * i + 2];
    for (int k = tid; k < nt; k += kTT) {
        const size_t gk = (size_t)P * nt + k;
        sX[3 * k] = x[3 * gk];
        sX[3 * k + 1] = x[3 * gk + 1];
        sX[3 * k + 2] = x[3 * gk + 2];
        sD[k] = x[3 * gk] - xi0;
        sD[nt + k] = x[3 * gk + 1] - xi1;
        sD[2 * nt + k] = x[3 * gk + 2] - xi2;
        sJ[k] = J[gk];
    }
    if (tid == 0) {
        S.u.bfs.cur[0] = 0;            // level 0: T0 itself
        S.nCur = 1;
        S.nLeaf = 0;
        S.overflow = 0;
    }
    __syncthreads();
    const int leaf_cap = min(max_leaves, kTriMaxLeaves);
    for (int lev = 0; lev <= max_depth; ++lev) {
        if (tid == 0) S.nNext = 0;
        __syncthreads();
        for (int q = tid; q < S.nCur; q += kTT) {
            const int code = S.u.bfs.cur[q];
            double tu[3], tv[3], y[4][3];
            tri_box(code, tu, tv);
            for (int k = 0; k < 3; ++k) tri_pos(sX, tu[k], tv[k], y[k]);
            tri_pos(sX, (tu[0] + tu[1] + tu[2]) / 3.0, (tv[0] + tv[1] + tv[2]) / 3.0, y[3]);
            double size = 0;
            for (int k = 0; k < 3; ++k) {
                const double dx = y[k][0] - y[3][0], dy = y[k][1] - y[3][1], dz = y[k][2] - y[3][2];
                size = fmax(size, sqrt(dx * dx + dy * dy + dz * dz));
            }
            const double dx = xi0 - y[3][0], dy = xi1 - y[3][1], dz = xi2 - y[3][2];
            const double dist = sqrt(dx * dx + dy * dy + dz * dz);
            if (lev < max_depth && dist < 2.0 * eta * size) {
                const int slot = atomicAdd(&S.nNext, 4);
                if (slot + 4 <= kTriMaxLevel) {
                    const int l1 = lev + 1, path = code & 0xffffff;
                    for (int c = 0; c < 4; ++c) S.u.bfs.next[slot + c] = (l1 << 24) | (path << 2) | c;
                } else {
                    S.overflow = 1;
                }
            } else {
                const int slot = atomicAdd(&S.nLeaf, 1);
                if (slot < leaf_cap) S.u.bfs.leaf[slot] = code; else S.overflow = 1;
            }
        }
        __syncthreads();
        const int nn_ = min(S.nNext, kTriMaxLevel);
        for (int q = tid; q < nn_; q += kTT) S.u.bfs.cur[q] = S.u.bfs.next[q];
        __syncthreads();
        if (tid == 0) S.nCur = nn_;
        __syncthreads();
        if (S.nCur == 0) break;
    }
    const int nleaves = min(S.nLeaf, leaf_cap);
    if (S.overflow && tid == 0) atomicExch(err, PM_DEV_LEAF_OVERFLOW);
    for (int q = tid; q < nleaves; q += kTT) {
        const int c = S.u.bfs.leaf[q];
        int rank = 0;
        for (int t = 0; t < nleaves; ++t) rank += (S.u.bfs.leaf[t] < c);
        S.sorted[rank] = c;
    }
    __syncthreads();     // the work lists are dead from here: S.u holds basis values
    const double n0 = n[3 * i], n1 = n[3 * i + 1], n2 = n[3 * i + 2];
    const double Hi = H[i];
    double acc[5] = {0, 0, 0, 0, 0};
    const int npts = nleaves * PM_GL16 * PM_GL16;
    for (int base = 0; base < npts; base += kTT) {
        const int q = base + tid;
        double* l = sL + tid * nt;
        double f[5] = {0, 0, 0, 0, 0};
        if (q < npts) {
            const int leaf = q / (PM_GL16 * PM_GL16), e = q - leaf * PM_GL16 * PM_GL16;
            const int is = e / PM_GL16, it = e - is * PM_GL16;
            double tu[3], tv[3];
            tri_box(S.sorted[leaf], tu, tv);
            // collapsed Gauss point of T0 (u' = s (1 - t), v' = t), mapped affinely
            const double s = 0.5 * (cTri.g16t[is] + 1.0), t = 0.5 * (cTri.g16t[it] + 1.0);
            const double up = s * (1.0 - t), vp = t;
            const double wq = 0.25 * cTri.g16w[is] * cTri.g16w[it] * (1.0 - t);
            const double e1u = tu[1] - tu[0], e1v = tv[1] - tv[0];
            const double e2u = tu[2] - tu[0], e2v = tv[2] - tv[0];
            const double det = fabs(e1u * e2v - e2u * e1v);
            tri_basis(tu[0] + up * e1u + vp * e2u, tv[0] + up * e1v + vp * e2v, l);
            double d0 = 0, d1 = 0, d2 = 0, jj = 0;
            for (int k = 0; k < nt; ++k) {
                d0 += l[k] * sD[k];
                d1 += l[k] * sD[nt + k];
                d2 += l[k] * sD[2 * nt + k];
                jj += l[k] * sJ[k];
            }
            tri_integrands(-d0, -d1, -d2, n0, n1, n2, Hi, wq * det * jj, 0.0, f);
        } else {
            for (int k = 0; k < nt; ++k) l[k] = 0.0;
        }
        for (int c = 0; c < 5; ++c) sF[c * kTT + tid] = f[c];
        __syncthreads();
        tri_accumulate(sL, sF, min(kTT, npts - base), nt, acc);
        __syncthreads();
    }
    if (tid < nt) {
        const size_t o = (size_t)b * nt + tid;
        W_lb[o] = acc[0];
        W_g[0 * (size_t)nblk * nt + o] = acc[1];
        W_g[1 * (size_t)nblk * nt + o] = acc[2];
        W_g[2 * (size_t)nblk * nt + o] = acc[3];
        W_k[o] = acc[4];
    }
}

std::mutex g_tri_build_mu;   // cTri holds one surface's tables during its build

}  // namespace

// ------------------------------------------------------------------ host
pm_status pm_tri_tables(int p, const double* ref, PmTriTables* T) {
    if (p < 2 || p > PM_TRI_MAX_P || !ref) {
        pm_set_error("triangle rule: need 2 <= p <= %d and the reference nodes", PM_TRI_MAX_P);
        return PM_ERR_INVALID_ARG;
    }
    const int n = p - 1, nt = p * (p + 1) / 2;
    T->p = p;
    T->nt = nt;
    T->u.resize(nt);
    T->v.resize(nt);
    T->w.resize(nt);
    for (int j = 0; j < nt; ++j) {
        const double u = ref[3 * j], v = ref[3 * j + 1], w = ref[3 * j + 2];
        if (!(u > 0.0 && v > 0.0 && u + v < 1.0) || !(w > 0.0) || !std::isfinite(w)) {
            pm_set_error("triangle rule: node %d (%g, %g) is not inside T0 or its weight %g "
                         "is not positive", j, u, v, w);
            return PM_ERR_INVALID_ARG;
        }
        T->u[j] = u;
        T->v[j] = v;
        T->w[j] = w;
    }
    // V[j][m] = K_m(u_j, v_j); U = V^-1 by Gauss-Jordan elimination with partial pivoting
    std::vector<double> A((size_t)nt * 2 * nt, 0.0);
    std::vector<double> K(nt);
    for (int j = 0; j < nt; ++j) {
        koornwinder<double>(n, T->u[j], T->v[j], K.data());
        for (int m = 0; m < nt; ++m) A[(size_t)j * 2 * nt + m] = K[m];
        A[(size_t)j * 2 * nt + nt + j] = 1.0;
    }
    double vmax = 0.0;
    for (int j = 0; j < nt; ++j)
        for (int m = 0; m < nt; ++m) vmax = std::max(vmax, std::fabs(A[(size_t)j * 2 * nt + m]));
    for (int c = 0; c < nt; ++c) {
        int piv = c;
        for (int r = c + 1; r < nt; ++r)
            if (std::fabs(A[(size_t)r * 2 * nt + c]) > std::fabs(A[(size_t)piv * 2 * nt + c])) piv = r;
        if (!(std::fabs(A[(size_t)piv * 2 * nt + c]) > 1e-12 * vmax)) {
            pm_set_error("triangle rule: the %d nodes are not unisolvent for degree %d", nt, n);
            return PM_ERR_INVALID_ARG;
        }
        if (piv != c)
            for (int k = 0; k < 2 * nt; ++k)
                std::swap(A[(size_t)piv * 2 * nt + k], A[(size_t)c * 2 * nt + k]);
        const double d = A[(size_t)c * 2 * nt + c];
        for (int k = 0; k < 2 * nt; ++k) A[(size_t)c * 2 * nt + k] /= d;
        for (int r = 0; r < nt; ++r) {
            if (r == c) continue;
            const double f = A[(size_t)r * 2 * nt + c];
            if (f == 0.0) continue;
            for (int k = 0; k < 2 * nt; ++k) A[(size_t)r * 2 * nt + k] -= f * A[(size_t)c * 2 * nt + k];
        }
    }
    // the right half holds V^-1 = U with U[m][k] in row m
    T->U.resize((size_t)nt * nt);
    for (int m = 0; m < nt; ++m)
        for (int k = 0; k < nt; ++k) T->U[(size_t)m * nt + k] = A[(size_t)m * 2 * nt + nt + k];
    // d l_k / du, d l_k / dv at the nodes: the recurrences in forward-mode derivatives
    std::vector<Dual> Kd(nt);
    T->Du.assign((size_t)nt * nt, 0.0);
    T->Dv.assign((size_t)nt * nt, 0.0);
    for (int j = 0; j < nt; ++j) {
        for (int dir = 0; dir < 2; ++dir) {
            koornwinder<Dual>(n, Dual(T->u[j], dir == 0 ? 1.0 : 0.0),
                              Dual(T->v[j], dir == 1 ? 1.0 : 0.0), Kd.data());
            std::vector<double>& D = dir == 0 ? T->Du : T->Dv;
            for (int k = 0; k < nt; ++k) {
                double acc = 0.0;
                for (int m = 0; m < nt; ++m) acc += Kd[m].d * T->U[(size_t)m * nt + k];
                D[(size_t)j * nt + k] = acc;
            }
        }
    }
    return PM_OK;
}

// Self-rule theta plan on T0 (Sec. 6.1.1): for each node, the angle split at the
// directions of the three vertices, panels bisected until int L^2 agrees with its
// halves to tol, then cut to at most max_width; 16 Gauss points each, with the ray
// length L(theta) to T0's boundary.
void pm_tri_theta_plan(const PmTriTables& T, const QuadTables& Q, double tol, double max_width,
                       std::vector<int>& off, std::vector<double>& ang, std::vector<double>& wts,
                       std::vector<double>& len) {
    off.assign(1, 0);
    ang.clear();
    wts.clear();
    len.clear();
    for (int loc = 0; loc < T.nt; ++loc) {
        const double u0 = T.u[loc], v0 = T.v[loc];
        auto l2 = [&](double a, double b) {
            double hh = 0.5 * (b - a), acc = 0.0;
            for (int q = 0; q < PM_GL16; ++q) {
                const double L = ray_length_tri(u0, v0, a + hh * (Q.g16t[q] + 1.0));
                acc += hh * Q.g16w[q] * L * L;
            }
            return acc;
        };
        const double cu[3] = {0.0, 1.0, 0.0}, cv[3] = {0.0, 0.0, 1.0};
        double ca[3];
        for (int k = 0; k < 3; ++k) {
            const double a = std::atan2(cv[k] - v0, cu[k] - u0);
            ca[k] = a < 0 ? a + 2 * M_PI : a;
        }
        std::sort(ca, ca + 3);
        std::vector<std::pair<double, double>> panels;
        std::function<void(double, double, double, int)> split = [&](double a, double b,
                                                                      double whole, int depth) {
            const double m = 0.5 * (a + b);
            const double l = l2(a, m), r = l2(m, b);
            if (depth >= 50 || std::fabs(whole - l - r) <= tol) {
                panels.emplace_back(a, b);
                return;
            }
            split(a, m, l, depth + 1);
            split(m, b, r, depth + 1);
        };
        for (int k = 0; k < 3; ++k) {
            const double a = ca[k], b = (k < 2) ? ca[k + 1] : ca[0] + 2 * M_PI;
            split(a, b, l2(a, b), 0);
        }
        for (auto& pb : panels) {
            const int ns = std::max(1, (int)std::ceil((pb.second - pb.first) / max_width));
            const double wdt = (pb.second - pb.first) / ns;
            for (int k = 0; k < ns; ++k) {
                const double a = pb.first + k * wdt, hh = 0.5 * wdt;
                for (int q = 0; q < PM_GL16; ++q) {
                    const double th = a + hh * (Q.g16t[q] + 1.0);
                    ang.push_back(th);
                    wts.push_back(hh * Q.g16w[q]);
                    len.push_back(ray_length_tri(u0, v0, th));
                }
            }
        }
        off.push_back((int)ang.size());
    }
}

// grad_G a at the nodes from the interpolant of a: a_u, a_v by the derivative
// matrices, then grad_G a = [y_u y_v] g^-1 [a_u; a_v] with the given tangents.
void pm_tri_gradient(const pm_surface* s, const double* a, double* grad) {
    const PmTriTables& T = *s->tri;
    const int nt = T.nt;
    for (int k = 0; k < s->N; ++k) {
        const int P = k / nt, j = k - P * nt;
        double au = 0.0, av = 0.0;
        for (int m = 0; m < nt; ++m) {
            au += T.Du[(size_t)j * nt + m] * a[(size_t)P * nt + m];
            av += T.Dv[(size_t)j * nt + m] * a[(size_t)P * nt + m];
        }
        const double* tu = &s->h_tg[6 * (size_t)k];
        const double* tv = tu + 3;
        const double E = tu[0] * tu[0] + tu[1] * tu[1] + tu[2] * tu[2];
        const double F = tu[0] * tv[0] + tu[1] * tv[1] + tu[2] * tv[2];
        const double G = tv[0] * tv[0] + tv[1] * tv[1] + tv[2] * tv[2];
        const double det = E * G - F * F;
        const double cu = (G * au - F * av) / det, cv = (-F * au + E * av) / det;
        for (int c = 0; c < 3; ++c) grad[3 * (size_t)k + c] = cu * tu[c] + cv * tv[c];
    }
}

// Geometry, structure and weight sets of a triangle-patch surface.
pm_status pm_near_build_tri(pm_surface* s, const QuadTables& Q) {
    std::lock_guard<std::mutex> build_lock(g_tri_build_mu);
    const PmTriTables& T = *s->tri;
    const int N = s->N, npatch = s->npatch, nt = T.nt;
    TriConst C{};
    C.p = T.p;
    C.n = T.p - 1;
    C.nt = nt;
    for (int k = 0; k < nt * nt; ++k) C.U[k] = T.U[k];
    for (int q = 0; q < PM_GL16; ++q) {
        C.g16t[q] = Q.g16t[q];
        C.g16w[q] = Q.g16w[q];
        C.logE[q] = Q.logE[q];
    }
    PM_CUDA_TRY(cudaMemcpyToSymbol(cTri, &C, sizeof(TriConst)));
    double *du = nullptr, *dv = nullptr, *ru = nullptr, *rv = nullptr;
    auto free_tmp = [&]() { pm_dfree(du); pm_dfree(dv); pm_dfree(ru); pm_dfree(rv); };
    pm_status st = PM_OK;
    do {
        if ((st = pm_dmalloc(&du, (size_t)nt * nt)) != PM_OK) break;
        if ((st = pm_dmalloc(&dv, (size_t)nt * nt)) != PM_OK) break;
        if ((st = pm_dmalloc(&ru, nt)) != PM_OK) break;
        if ((st = pm_dmalloc(&rv, nt)) != PM_OK) break;
        if ((st = pm_dmalloc(&s->centroid, 3 * (size_t)npatch)) != PM_OK) break;
        if ((st = pm_dmalloc(&s->radius, npatch)) != PM_OK) break;
        if ((st = pm_dmalloc(&s->npatch_n, 3 * (size_t)N)) != PM_OK) break;
        cudaError_t ce = cudaMemcpy(du, T.Du.data(), sizeof(double) * nt * nt, cudaMemcpyHostToDevice);
        if (ce == cudaSuccess) ce = cudaMemcpy(dv, T.Dv.data(), sizeof(double) * nt * nt, cudaMemcpyHostToDevice);
        if (ce == cudaSuccess) ce = cudaMemcpy(ru, T.u.data(), sizeof(double) * nt, cudaMemcpyHostToDevice);
        if (ce == cudaSuccess) ce = cudaMemcpy(rv, T.v.data(), sizeof(double) * nt, cudaMemcpyHostToDevice);
        if (ce != cudaSuccess) {
            pm_set_error("triangle tables: %s", cudaGetErrorString(ce));
            st = PM_ERR_CUDA;
            break;
        }
        k_patch_geom_tri<<<pm_ceil_div(npatch, 128), 128>>>(s->x, npatch, s->centroid, s->radius);
        k_node_normals_tri<<<pm_ceil_div(N, 128), 128>>>(s->x, N, nt, du, dv, s->npatch_n);
        ce = cudaGetLastError();
        if (ce != cudaSuccess) {
            pm_set_error("triangle geometry: %s", cudaGetErrorString(ce));
            st = PM_ERR_CUDA;
            break;
        }
        if ((st = pm_near_structure(s)) != PM_OK) break;
        const size_t smem = sizeof(double) * ((size_t)kTT * nt + (size_t)kTriG * 5 * kTT +
                                              (size_t)kTriG * 4 * nt);
        ce = cudaFuncSetAttribute(k_self_quad_tri, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem);
        if (ce != cudaSuccess) {
            pm_set_error("triangle self rule: %s", cudaGetErrorString(ce));
            st = PM_ERR_CUDA;
            break;
        }
        k_self_quad_tri<<<dim3(pm_ceil_div(npatch, kTriG), nt), kTT, smem>>>(
            npatch, s->x, s->J, s->npatch_n, s->H, ru, rv, s->th_off, s->th_ang, s->th_w,
            s->th_L, s->row_ptr, s->nblk, s->W_lb, s->W_g, s->W_k);
        k_near_quad_tri<<<s->nblk, kTT>>>(s->nblk, s->x, s->J, s->n, s->H, s->blk_row,
                                          s->blk_patch, s->row_ptr, s->opts.near_eta,
                                          std::min(s->opts.near_max_depth, 12),
                                          s->opts.near_max_leaves, s->W_lb, s->W_g, s->W_k,
                                          s->dev_err);
        ce = cudaGetLastError();
        if (ce == cudaSuccess) ce = cudaDeviceSynchronize();
        if (ce != cudaSuccess) {
            pm_set_error("triangle quadrature: %s", cudaGetErrorString(ce));
            st = PM_ERR_CUDA;
            break;
        }
        int herr = 0;
        ce = cudaMemcpy(&herr, s->dev_err, sizeof(int), cudaMemcpyDeviceToHost);
        if (ce != cudaSuccess || herr != PM_DEV_OK) {
            pm_set_error("triangle near-field quadrature: device check %d failed (leaf budget)", herr);
            st = PM_ERR_INTERNAL;
            break;
        }
    } while (false);
    free_tmp();
    return st;
}

extern "C" pm_status pm_selftest_tri_basis(int p, const double* ref, int npts, const double* u,
                                           const double* v, double* l, double* Du, double* Dv) {
    if (!ref || npts < 0 || (npts > 0 && (!u || !v || !l)) || !Du || !Dv) {
        pm_set_error("pm_selftest_tri_basis: NULL argument or npts < 0");
        return PM_ERR_INVALID_ARG;
    }
    PmTriTables T;
    PM_TRY(pm_tri_tables(p, ref, &T));
    const int nt = T.nt;
    std::vector<double> K(nt);
    for (int q = 0; q < npts; ++q) {
        koornwinder<double>(p - 1, u[q], v[q], K.data());
        for (int k = 0; k < nt; ++k) {
            double acc = 0.0;
            for (int m = 0; m < nt; ++m) acc += K[m] * T.U[(size_t)m * nt + k];
            l[(size_t)q * nt + k] = acc;
        }
    }
    std::copy(T.Du.begin(), T.Du.end(), Du);
    std::copy(T.Dv.begin(), T.Dv.end(), Dv);
    return PM_OK;
}
