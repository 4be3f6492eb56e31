// Chebyshev kernel-interpolation FMM for the smooth remainder and parametrix
// sums on large surfaces (the fast far-field apply of Sec. 6.2, in the
// interpolation form rather than the paper's IFMM).
//
// The smooth remainder sum factors into nine translation-invariant kernels of
// r = x - y with target-only coefficients:
//   y_i = sum_{a,b} n'_a n'_b phi_ab(x_i) + sum_a m_a psi_a(x_i),
//   phi_ab(x) = sum_j s_j r_a r_b / |r|^4,   psi_a(x) = sum_j s_j r_a / |r|^2,
// with n' = sqrt(a_i/pi) n_i and m = -(a_i H_i/pi) n_i + grad a_i /(2 pi)
// (eq. explicit_remainder, c = 0); the parametrix sum is the single kernel
// log|r| / (2 pi) (eq. diff_param).
//
// Tree: a uniform-depth octree over the occupied boxes (all leaves on one
// level, so only U lists at the leaves and V lists per level are needed); the
// depth is chosen on the host by a cost model (pair counts of the direct near
// field against node-pair counts of the far field).  Each box carries an
// n x n x n tensor grid of Chebyshev points (first kind); expansions are the
// values at those points:
//   P2M  M_B[m] = sum_{j in B} s_j S_m(y_j)             (S_m: tensor Lagrange basis)
//   M2M  M_P[m] = sum_children sum_k S^P_m(y^C_k) M_C[k]
//   M2L  L_T[c][l] += sum_{S in V(T)} sum_m kernel_c(x^T_l - y^S_m) M_S[m]
//        (evaluated directly between the two boxes' Chebyshev points)
//   L2L  L_C[c][k] += sum_l S^P_l(x^C_k) L_P[c][l]
//   L2P  phi_c(x_i) = sum_l S_l(x_i) L_B[c][l], then the target combination
//   P2P  leaf targets against the sources of the 27 adjacent leaves, exact kernel,
//        one block per (leaf, neighbour); every term goes to its own partial slice
//        (27 neighbours + the far field), which the near-field kernel adds.
// Everything is float32 except the host-side tree; the near-field correction
// (CSR) is added by the regular correction kernel.
#include "pm_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <type_traits>
#include <unordered_map>
#include <vector>

namespace {

constexpr int kFmmN = 8;                       // Chebyshev points per dimension
constexpr int kFmmN3 = kFmmN * kFmmN * kFmmN;  // 512
constexpr int kThreads = 512;                  // one thread per expansion point
constexpr int kMaxLeafPts = 4096;

struct FmmConst {
    float cheb[kFmmN];          // Chebyshev points of the first kind on [-1, 1]
    float bary[kFmmN];          // barycentric weights
    float T[2][kFmmN][kFmmN];   // T[o][m][k] = l_m((t_k + (2o - 1)) / 2): child point k in parent coords
};
__constant__ FmmConst cF;

__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float v) {
    const float s = hi + v;
    const float bp = s - hi;
    lo += (hi - (s - bp)) + (v - bp);
    hi = s;
}

// 1-D Lagrange basis at the Chebyshev points (product form, exact at the points)
__device__ __forceinline__ void cheb_basis(float u, float* out) {
    float d[kFmmN];
#pragma unroll
    for (int b = 0; b < kFmmN; ++b) d[b] = u - cF.cheb[b];
    float pre = 1.f;
#pragma unroll
    for (int a = 0; a < kFmmN; ++a) {
        out[a] = pre;
        pre *= d[a];
    }
    float suf = 1.f;
#pragma unroll
    for (int a = kFmmN - 1; a >= 0; --a) {
        out[a] *= suf * cF.bary[a];
        suf *= d[a];
    }
}

struct DevTree {
    int N, nlev, depth, nbox_total;
    float3 origin;
    float L0;
    const int* perm;          // sorted position -> original node
    const int* lev_off;       // [depth+2] first box index of each level
    const int3* box_ijk;      // [nbox] integer coordinates at its level
    const int* box_first;     // [nbox+1 per leaf] point ranges (leaves only; index by leaf id)
    const int* parent;        // [nbox]
    const int* child_off;     // [nbox+1] CSR of children
    const int* child;         // children box ids
    const int* v_off;         // [nbox+1] CSR of V lists
    const int* v_list;
    const int* u_off;         // [nleaf+1] CSR of U lists (leaf ids)
    const int* u_list;
    const int* p2p_order;     // P2P blocks (leaf, target chunk, e), largest first
    const int* leaf_chunks;   // L2P blocks (leaf << 5 | chunk of 128 targets)
};

__device__ __forceinline__ float3 box_center(const DevTree& t, int lev, int3 ijk) {
    const float h = t.L0 / (float)(1 << lev);
    return make_float3(t.origin.x + (ijk.x + 0.5f) * h, t.origin.y + (ijk.y + 0.5f) * h,
                       t.origin.z + (ijk.z + 0.5f) * h);
}

// gather sorted sources: (x, y, z, s) in leaf order
__global__ void k_fmm_gather(const float4* __restrict__ src, const int* __restrict__ perm, int N,
                             float4* __restrict__ sorted, const int* __restrict__ skip) {
    if (skip && *skip) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) sorted[i] = src[perm[i]];
}

// P2M: one block per leaf.  M[m1][m2][m3] = sum_j s_j l_m1(x_j) l_m2(y_j) l_m3(z_j):
// thread (g, m1, m2) of the 512 accumulates the 8 values m3 over the points of
// group g (every 8th point of each staged batch); the 8 groups' partial sums are
// added in group order at the end.
constexpr int kP2MBatch = 256;
__global__ void __launch_bounds__(kThreads)
k_fmm_p2m(DevTree t, const float4* __restrict__ pts, float* __restrict__ M,
          const int* __restrict__ skip) {
    if (skip && *skip) return;
    static_assert(kThreads == 8 * kFmmN * kFmmN, "8 point groups x (m1, m2)");
    const int leaf = blockIdx.x;
    const int box = t.lev_off[t.depth] + leaf;
    const int p0 = t.box_first[leaf], p1 = t.box_first[leaf + 1];
    const float h = t.L0 / (float)(1 << t.depth);
    const float3 c = box_center(t, t.depth, t.box_ijk[box]);
    const float sc = 2.f / h;
    __shared__ __align__(16) float sB[kP2MBatch][3 * kFmmN];   // s_j l(x_j) | l(y_j) | l(z_j); reused for the reduction
    const int g = threadIdx.x >> 6, m1 = (threadIdx.x >> 3) & 7, m2 = threadIdx.x & 7;
    float acc[kFmmN];
#pragma unroll
    for (int k = 0; k < kFmmN; ++k) acc[k] = 0.f;
    for (int base = p0; base < p1; base += kP2MBatch) {
        const int cnt = min(kP2MBatch, p1 - base);
        __syncthreads();
        if (threadIdx.x < cnt) {
            const float4 q = pts[base + threadIdx.x];
            float l[kFmmN];
            cheb_basis((q.x - c.x) * sc, l);
#pragma unroll
            for (int a = 0; a < kFmmN; ++a) sB[threadIdx.x][a] = q.w * l[a];
            cheb_basis((q.y - c.y) * sc, l);
#pragma unroll
            for (int a = 0; a < kFmmN; ++a) sB[threadIdx.x][kFmmN + a] = l[a];
            cheb_basis((q.z - c.z) * sc, l);
#pragma unroll
            for (int a = 0; a < kFmmN; ++a) sB[threadIdx.x][2 * kFmmN + a] = l[a];
        }
        __syncthreads();
        for (int j = g; j < cnt; j += 8) {
            const float w = sB[j][m1] * sB[j][kFmmN + m2];
            const float4 z0 = *reinterpret_cast<const float4*>(&sB[j][2 * kFmmN]);
            const float4 z1 = *reinterpret_cast<const float4*>(&sB[j][2 * kFmmN + 4]);
            acc[0] = fmaf(w, z0.x, acc[0]); acc[1] = fmaf(w, z0.y, acc[1]);
            acc[2] = fmaf(w, z0.z, acc[2]); acc[3] = fmaf(w, z0.w, acc[3]);
            acc[4] = fmaf(w, z1.x, acc[4]); acc[5] = fmaf(w, z1.y, acc[5]);
            acc[6] = fmaf(w, z1.z, acc[6]); acc[7] = fmaf(w, z1.w, acc[7]);
        }
    }
    // reduce the 8 groups in order: red[g][m], m = (m1 * 8 + m2) * 8 + m3
    __syncthreads();
    float* red = &sB[0][0];
    static_assert(kP2MBatch * 3 * kFmmN >= 8 * kFmmN3, "reduction buffer");
#pragma unroll
    for (int k = 0; k < kFmmN; ++k) red[g * kFmmN3 + ((m1 * kFmmN + m2) * kFmmN + k)] = acc[k];
    __syncthreads();
    const int m = threadIdx.x;
    float v = 0.f;
#pragma unroll
    for (int q = 0; q < 8; ++q) v += red[q * kFmmN3 + m];
    M[(size_t)box * kFmmN3 + m] = v;
}

// The transfer between a parent box and its child o = (ox, oy, oz) is the tensor
// product T[ox] x T[oy] x T[oz] of 8 x 8 matrices (T[o][m][k] = l_m of child
// point k in parent coordinates), applied as three 1-D passes in shared memory
// (3 x 8 instead of 512 multiply-adds per value).  Thread (i1, i2, i3) of the
// 512 computes one value per pass.
//   UP   (M2M, contract child points k):   out[m] = sum_k  prod_a T[o_a][m_a][k_a] in[k]
//   DOWN (L2L, contract parent basis m):   out[k] = sum_m  prod_a T[o_a][m_a][k_a] in[m]
template <bool UP>
__device__ __forceinline__ float transfer3(const float (*sT)[kFmmN][kFmmN], int ox, int oy, int oz,
                                           float* s0, float* s1, int i1, int i2, int i3) {
    // s0 holds the input; returns this thread's output value; s0 and s1 are overwritten
    const int k = (i1 * kFmmN + i2) * kFmmN + i3;
    float v = 0.f;
#pragma unroll
    for (int j = 0; j < kFmmN; ++j)
        v = fmaf(UP ? sT[oz][i3][j] : sT[oz][j][i3], s0[(i1 * kFmmN + i2) * kFmmN + j], v);
    s1[k] = v;
    __syncthreads();
    v = 0.f;
#pragma unroll
    for (int j = 0; j < kFmmN; ++j)
        v = fmaf(UP ? sT[oy][i2][j] : sT[oy][j][i2], s1[(i1 * kFmmN + j) * kFmmN + i3], v);
    s0[k] = v;
    __syncthreads();
    v = 0.f;
#pragma unroll
    for (int j = 0; j < kFmmN; ++j)
        v = fmaf(UP ? sT[ox][i1][j] : sT[ox][j][i1], s0[(j * kFmmN + i2) * kFmmN + i3], v);
    return v;
}

__device__ __forceinline__ void load_transfer(float (*sT)[kFmmN][kFmmN]) {
    for (int e = threadIdx.x; e < 2 * kFmmN * kFmmN; e += blockDim.x)
        (&sT[0][0][0])[e] = (&cF.T[0][0][0])[e];
}

// M2M for the boxes of one level: M_P = sum_children T(child) M_child
__global__ void __launch_bounds__(kThreads)
k_fmm_m2m(DevTree t, int lev, float* __restrict__ M, const int* __restrict__ skip) {
    if (skip && *skip) return;
    static_assert(kThreads == kFmmN3, "one thread per expansion point");
    const int box = t.lev_off[lev] + blockIdx.x;
    const int m = threadIdx.x;
    __shared__ float sT[2][kFmmN][kFmmN];
    __shared__ float s0[kFmmN3], s1[kFmmN3];
    load_transfer(sT);
    const int m1 = m / (kFmmN * kFmmN), m2 = (m / kFmmN) % kFmmN, m3 = m % kFmmN;
    const int3 pijk = t.box_ijk[box];
    float acc = 0.f;
    for (int e = t.child_off[box]; e < t.child_off[box + 1]; ++e) {
        const int ch = t.child[e];
        const int3 cijk = t.box_ijk[ch];
        const int ox = cijk.x - 2 * pijk.x, oy = cijk.y - 2 * pijk.y, oz = cijk.z - 2 * pijk.z;
        __syncthreads();
        s0[m] = M[(size_t)ch * kFmmN3 + m];
        __syncthreads();
        acc += transfer3<true>(sT, ox, oy, oz, s0, s1, m1, m2, m3);
    }
    M[(size_t)box * kFmmN3 + m] = acc;
}

// M2L: one block per target box (any level >= 2), thread per target Chebyshev point;
// direct evaluation between the target box's points and each V-list box's points.
template <bool KERNEL_K>
__global__ void __launch_bounds__(kThreads)
k_fmm_m2l(DevTree t, int box0, const float* __restrict__ M, float* __restrict__ Lc,
          const int* __restrict__ skip) {
    if (skip && *skip) return;
    const int box = box0 + blockIdx.x;
    int lev = 0;
    while (lev + 1 <= t.depth && t.lev_off[lev + 1] <= box) ++lev;
    const float h = t.L0 / (float)(1 << lev);
    const float3 c = box_center(t, lev, t.box_ijk[box]);
    const int l = threadIdx.x;
    const int l1 = l / (kFmmN * kFmmN), l2 = (l / kFmmN) % kFmmN, l3 = l % kFmmN;
    const float tx = c.x + 0.5f * h * cF.cheb[l1 % kFmmN];
    const float ty = c.y + 0.5f * h * cF.cheb[l2 % kFmmN];
    const float tz = c.z + 0.5f * h * cF.cheb[l3 % kFmmN];
    __shared__ float4 sP[kFmmN3];
    constexpr int C = KERNEL_K ? 1 : 9;
    float acc[C];
#pragma unroll
    for (int q = 0; q < C; ++q) acc[q] = 0.f;
    for (int e = t.v_off[box]; e < t.v_off[box + 1]; ++e) {
        const int sb = t.v_list[e];
        const float3 sc = box_center(t, lev, t.box_ijk[sb]);
        __syncthreads();
        if (l < kFmmN3) {
            const int k1 = l / (kFmmN * kFmmN), k2 = (l / kFmmN) % kFmmN, k3 = l % kFmmN;
            sP[l] = make_float4(sc.x + 0.5f * h * cF.cheb[k1], sc.y + 0.5f * h * cF.cheb[k2],
                                sc.z + 0.5f * h * cF.cheb[k3], M[(size_t)sb * kFmmN3 + l]);
        }
        __syncthreads();
#pragma unroll 2
        for (int k = 0; k < kFmmN3; ++k) {
            const float4 s = sP[k];
            const float dx = tx - s.x, dy = ty - s.y, dz = tz - s.z;
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            if (KERNEL_K) {
                acc[0] = fmaf(s.w, lg2_approx(r2), acc[0]);
            } else {
                const float inv = rcp_approx(r2);
                const float ax = dx * inv, ay = dy * inv, az = dz * inv;
                const float sx = s.w * ax, sy = s.w * ay, sz = s.w * az;
                acc[0] = fmaf(sx, dx * inv, acc[0]);   // xx: r_x r_x / r^4
                acc[1] = fmaf(sx, ay, acc[1]);         // xy
                acc[2] = fmaf(sx, az, acc[2]);         // xz
                acc[3] = fmaf(sy, ay, acc[3]);         // yy
                acc[4] = fmaf(sy, az, acc[4]);         // yz
                acc[5] = fmaf(sz, az, acc[5]);         // zz
                acc[6] += sx;                          // x: r_x / r^2
                acc[7] += sy;
                acc[8] += sz;
            }
        }
    }
    if (l < kFmmN3)
#pragma unroll
        for (int q = 0; q < C; ++q) Lc[((size_t)box * C + q) * kFmmN3 + l] = acc[q];
}

// L2L for the boxes of one level (children receive their parent's local expansion)
template <int C>
__global__ void __launch_bounds__(kThreads)
k_fmm_l2l(DevTree t, int lev, float* __restrict__ Lc, const int* __restrict__ skip) {
    if (skip && *skip) return;
    const int box = t.lev_off[lev] + blockIdx.x;
    const int par = t.parent[box];
    const int k = threadIdx.x;
    const int3 cijk = t.box_ijk[box], pijk = t.box_ijk[par];
    const int ox = cijk.x - 2 * pijk.x, oy = cijk.y - 2 * pijk.y, oz = cijk.z - 2 * pijk.z;
    __shared__ float sT[2][kFmmN][kFmmN];
    __shared__ float s0[kFmmN3], s1[kFmmN3];
    load_transfer(sT);
    const int k1 = k / (kFmmN * kFmmN), k2 = (k / kFmmN) % kFmmN, k3 = k % kFmmN;
    for (int q = 0; q < C; ++q) {
        __syncthreads();
        s0[k] = Lc[((size_t)par * C + q) * kFmmN3 + k];
        __syncthreads();
        Lc[((size_t)box * C + q) * kFmmN3 + k] += transfer3<false>(sT, ox, oy, oz, s0, s1, k1, k2, k3);
    }
}

// P2P for one (leaf, U-list neighbour, target chunk) triple, decoded from
// p2p_order[blockIdx.x]: the exact kernel between up to 128 of the leaf's
// targets and the sources of the e-th leaf of its U list (the leaf itself
// included), written as (hi, lo) to partial slice e of each target (zeros when
// the leaf has fewer than e + 1 neighbours).  Splitting the near field by
// neighbour and by target chunk bounds every block's work by 128 x (leaf size)
// pairs; the blocks run largest first.
constexpr int kP2PThreads = 128;               // one target per thread, one chunk per block
constexpr int kP2PStage = 512;                 // sources staged in shared memory per pass
constexpr int kUMax = 27;                      // U list: the 3 x 3 x 3 leaves around a leaf
constexpr int kP2PMaxChunks = 32;              // kMaxLeafPts / kP2PThreads
static_assert(kMaxLeafPts <= kP2PThreads * kP2PMaxChunks, "chunk field of the P2P block code");

__host__ __device__ __forceinline__ int p2p_code(int leaf, int chunk, int e) {
    return (leaf << 10) | (chunk << 5) | e;
}

template <bool KERNEL_K>
__global__ void __launch_bounds__(kP2PThreads)
k_fmm_p2p(DevTree t, const float4* __restrict__ pts, const float4* __restrict__ tgt, float eps2,
          float2* __restrict__ out, const int* __restrict__ skip) {
    if (skip && *skip) return;
    const int code = t.p2p_order[blockIdx.x];
    const int leaf = code >> 10, chunk = (code >> 5) & 31, e = code & 31;
    const int p1 = t.box_first[leaf + 1];
    const int i = t.box_first[leaf] + chunk * kP2PThreads + threadIdx.x;
    const bool active = i < p1;
    const int ne = t.u_off[leaf + 1] - t.u_off[leaf];
    float2* slice = out + (size_t)e * t.N;
    if (e >= ne) {
        if (active) slice[t.perm[i]] = make_float2(0.f, 0.f);
        return;
    }
    const int ul = t.u_list[t.u_off[leaf] + e];
    const int q0 = t.box_first[ul], q1 = t.box_first[ul + 1];
    __shared__ float4 sP[kP2PStage];
    float4 X = make_float4(0.f, 0.f, 0.f, 0.f), NN = X, MM = X;
    int orig = 0;
    if (active) {
        orig = t.perm[i];
        X = tgt[orig];
        NN = tgt[t.N + orig];
        MM = tgt[2 * t.N + orig];
    }
    float hi = 0.f, lo = 0.f;
    for (int qb = q0; qb < q1; qb += kP2PStage) {
        const int cnt = min(kP2PStage, q1 - qb);
        __syncthreads();
        for (int j = threadIdx.x; j < cnt; j += kP2PThreads) sP[j] = pts[qb + j];
        __syncthreads();
        float part = 0.f;
        if (active) {
            for (int j = 0; j < cnt; ++j) {
                const float4 s = sP[j];
                const float dx = X.x - s.x, dy = X.y - s.y, dz = X.z - s.z;
                if (KERNEL_K) {
                    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    const float lg = (qb + j == i) ? 0.f : lg2_approx(r2);
                    part = fmaf(s.w, lg, part);
                } else {
                    const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
                    const float inv = rcp_approx(r2);
                    const float nr = fmaf(NN.x, dx, fmaf(NN.y, dy, NN.z * dz));
                    const float mr = fmaf(MM.x, dx, fmaf(MM.y, dy, MM.z * dz));
                    part = fmaf(s.w, fmaf(nr, nr * inv, mr) * inv, part);
                }
            }
        }
        two_sum_acc(hi, lo, KERNEL_K ? part * (float)(M_LN2 / (4.0 * M_PI)) : part);
    }
    if (active) slice[orig] = make_float2(hi, lo);
}

// L2P for one (leaf, chunk of 128 targets) = leaf_chunks[blockIdx.x]:
// phi_c(x) = sum_l S_l(x) L[c][l] and the target combination, written to
// partial slice kUMax of each target.
constexpr int kL2PThreads = 128;
static_assert(kMaxLeafPts <= kL2PThreads * 32, "chunk field of the L2P block code");
template <bool KERNEL_K>
__global__ void __launch_bounds__(kL2PThreads)
k_fmm_l2p(DevTree t, const float4* __restrict__ tgt, const float* __restrict__ Lc,
          float2* __restrict__ out, const int* __restrict__ skip) {
    if (skip && *skip) return;
    const int code = t.leaf_chunks[blockIdx.x];
    const int leaf = code >> 5, chunk = code & 31;
    const int box = t.lev_off[t.depth] + leaf;
    const int p1 = t.box_first[leaf + 1];
    const int i = t.box_first[leaf] + chunk * kL2PThreads + threadIdx.x;
    const float h = t.L0 / (float)(1 << t.depth);
    const float3 c = box_center(t, t.depth, t.box_ijk[box]);
    const float sc = 2.f / h;
    constexpr int C = KERNEL_K ? 1 : 9;
    __shared__ __align__(16) float sLoc[C * kFmmN3];
    const float4* src = reinterpret_cast<const float4*>(Lc + (size_t)box * C * kFmmN3);
    for (int q = threadIdx.x; q < C * kFmmN3 / 4; q += kL2PThreads)
        reinterpret_cast<float4*>(sLoc)[q] = src[q];
    __syncthreads();
    if (i >= p1) return;
    float2* slice = out + (size_t)kUMax * t.N;
    const int orig = t.perm[i];
    const float4 X = tgt[orig], NN = tgt[t.N + orig], MM = tgt[2 * t.N + orig];
    float bx[kFmmN], by[kFmmN], bz[kFmmN];
    cheb_basis((X.x - c.x) * sc, bx);
    cheb_basis((X.y - c.y) * sc, by);
    cheb_basis((X.z - c.z) * sc, bz);
    float phi[C];
#pragma unroll
    for (int q = 0; q < C; ++q) phi[q] = 0.f;
    for (int l1 = 0; l1 < kFmmN; ++l1) {
        float b1 = bx[0];   // bx[l1] without a runtime-indexed array
#pragma unroll
        for (int k = 1; k < kFmmN; ++k) b1 = (k == l1) ? bx[k] : b1;
#pragma unroll
        for (int l2 = 0; l2 < kFmmN; ++l2) {
            const float w12 = b1 * by[l2];
            float w[kFmmN];
#pragma unroll
            for (int l3 = 0; l3 < kFmmN; ++l3) w[l3] = w12 * bz[l3];
#pragma unroll
            for (int q = 0; q < C; ++q) {
                const float4* row =
                    reinterpret_cast<const float4*>(sLoc + q * kFmmN3 + (l1 * kFmmN + l2) * kFmmN);
                const float4 a0 = row[0], a1 = row[1];
                float v = phi[q];
                v = fmaf(w[0], a0.x, v); v = fmaf(w[1], a0.y, v); v = fmaf(w[2], a0.z, v);
                v = fmaf(w[3], a0.w, v); v = fmaf(w[4], a1.x, v); v = fmaf(w[5], a1.y, v);
                v = fmaf(w[6], a1.z, v); v = fmaf(w[7], a1.w, v);
                phi[q] = v;
            }
        }
    }
    float far;
    if (KERNEL_K) {
        far = phi[0] * (float)(M_LN2 / (4.0 * M_PI));
    } else {
        far = NN.x * NN.x * phi[0] + NN.y * NN.y * phi[3] + NN.z * NN.z * phi[5] +
              2.f * (NN.x * NN.y * phi[1] + NN.x * NN.z * phi[2] + NN.y * NN.z * phi[4]) +
              MM.x * phi[6] + MM.y * phi[7] + MM.z * phi[8];
    }
    slice[orig] = make_float2(far, 0.f);
}

// ---------------------------------------------------------------- M2L as GEMMs
// The M2L operator between two boxes of one level depends only on their offset
// d = ijk_T - ijk_S (a V-list offset: max |d_i| in {2, 3}, 316 of them) and on
// the box size h, through  r = h (d + (t_l - t_m) / 2)  between target point l
// and source point m.  The kernels are homogeneous: r_a r_b / r^4 and r_a / r^2
// scale as h^-2 and h^-1, lg2 r^2 = lg2 u^2 + 2 lg2 h.  So one unit-box operator
// per offset serves every level.
//
// The offsets fall into 16 classes under the 48 signed axis permutations g of
// the cube, (g v)_a = s_a v_{pi(a)}: every d is g d_c for a canonical d_c with
// d_c,x >= d_c,y >= d_c,z >= 0.  The Chebyshev grid is closed under g (the
// points are symmetric about 0), so with the point map g.l (axis a of g.l is
// axis pi(a) of l, mirrored k -> n-1-k where s_a < 0) one has
// r(d, g.l', g.m') = g r(d_c, l', m'), hence
//   sum_m phi_ab(r(d, l, m)) M[m] = s_a s_b  [A_{d_c} Mt]_{pi(a) pi(b)} (g^-1 . l),
//   Mt[m'] = M[g.m'],
// and likewise s_a [.]_{pi(a)} for r_a / r^2; the log kernel is invariant.
// Only the 16 canonical operators are stored (rows c * 512 + l for kernel c and
// target point l, columns m, column-major).  The multipoles of all V-list pairs
// of one class are gathered, permuted into the canonical frame, as the columns
// of B; one GEMM per class forms C = A_c B; each target box sums its V-list
// columns of C, mapped back through g and scaled for its level.
//
// The GEMM runs on the float16 tensor cores (tcgen05, pm_tcgemm.cu) with
// float32 accumulation.  Each float32 operand x, scaled by a power of two into
// the upper float16 range, is split as x0 + x1 (x0 = fp16(x), x1 = fp16(x - x0):
// 22 significand bits, |x - x0 - x1| <= 2^-22 |x|), and the three products
// a1 b0 + a0 b1 + a0 b0 are one GEMM over K = 3 x 512 with A' = [a1 a0 a0] and
// B' = [b0; b1; b0]: the small products first, so that they are accumulated
// before the large one.  The dropped product a1 b1 is below 2^-22 |a||b|.
// Scales: the operators are stored times 2^12 (their entries are below 6 in
// magnitude, so the parts stay normal float16 down to 2^-15 of the largest
// entry); each gathered multipole column is scaled by 2^e so that its largest
// value lies in [2^14, 2^15), and the scatter multiplies the column by
// 2^-(e + 12).  Powers of two: the scaling itself is exact.
constexpr int kNClass = 16;
constexpr int kSplitK = 3 * kFmmN3;
constexpr float kOpScale = 4096.f;   // 2^12
constexpr int kOpScaleExp = 12;

__host__ __device__ __forceinline__ int3 canonical_offset(int c) {
    // enumeration of d_c = (i, j, k), i in {2, 3}, i >= j >= k >= 0
    int n = 0;
    for (int i = 2; i <= 3; ++i)
        for (int j = 0; j <= i; ++j)
            for (int k = 0; k <= j; ++k) {
                if (n == c) return make_int3(i, j, k);
                ++n;
            }
    return make_int3(0, 0, 0);
}

// symmetry code: bits 0-1 pi(0), 2-3 pi(1), 4-5 pi(2), bit 6 + a set where s_a = -1
__device__ __forceinline__ int sym_pi(int g, int a) { return (g >> (2 * a)) & 3; }
__device__ __forceinline__ bool sym_neg(int g, int a) { return (g >> (6 + a)) & 1; }

// g.m: axis a of the result is axis pi(a) of m, mirrored where s_a < 0
__device__ __forceinline__ int sym_apply(int g, int m) {
    const int mi[3] = {m / (kFmmN * kFmmN), (m / kFmmN) % kFmmN, m % kFmmN};
    int o[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int v = mi[sym_pi(g, a)];
        o[a] = sym_neg(g, a) ? kFmmN - 1 - v : v;
    }
    return (o[0] * kFmmN + o[1]) * kFmmN + o[2];
}

// g^-1.l: axis pi(a) of the result is axis a of l, mirrored where s_a < 0
__device__ __forceinline__ int sym_apply_inv(int g, int l) {
    const int li[3] = {l / (kFmmN * kFmmN), (l / kFmmN) % kFmmN, l % kFmmN};
    int o[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const int v = sym_neg(g, a) ? kFmmN - 1 - li[a] : li[a];
        o[sym_pi(g, a)] = v;
    }
    return (o[0] * kFmmN + o[1]) * kFmmN + o[2];
}

__global__ void k_fmm_build_op(int which_K, float* __restrict__ A) {
    const int rows = which_K ? kFmmN3 : 9 * kFmmN3;
    const int o = blockIdx.y;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)rows * kFmmN3) return;
    const int row = (int)(e % rows), m = (int)(e / rows);
    const int c = row / kFmmN3, l = row % kFmmN3;
    const int l1 = l / (kFmmN * kFmmN), l2 = (l / kFmmN) % kFmmN, l3 = l % kFmmN;
    const int m1 = m / (kFmmN * kFmmN), m2 = (m / kFmmN) % kFmmN, m3 = m % kFmmN;
    const int3 d = canonical_offset(o);
    auto cheb = [](int k) { return cos(M_PI * (2 * k + 1) / (2.0 * kFmmN)); };
    const double ux = d.x + 0.5 * (cheb(l1) - cheb(m1));
    const double uy = d.y + 0.5 * (cheb(l2) - cheb(m2));
    const double uz = d.z + 0.5 * (cheb(l3) - cheb(m3));
    const double r2 = ux * ux + uy * uy + uz * uz;
    double v;
    if (which_K) {
        v = log2(r2);
    } else {
        const double u[3] = {ux, uy, uz};
        const int pa[6] = {0, 0, 0, 1, 1, 2}, pb[6] = {0, 1, 2, 1, 2, 2};
        v = (c < 6) ? u[pa[c]] * u[pb[c]] / (r2 * r2) : u[c - 6] / r2;
    }
    A[(size_t)o * rows * kFmmN3 + e] = (float)v;
}

// A'[o][row][kk] (K-major): part a1 for kk < 512, a0 otherwise, of 2^12 A[o][row][kk % 512]
// (A column-major [m][rows])
__global__ void k_fmm_split_op(int rows, const float* __restrict__ A, __half* __restrict__ As) {
    const int o = blockIdx.y;
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)rows * kSplitK) return;
    const int row = (int)(e / kSplitK), kk = (int)(e % kSplitK);
    const float a = A[((size_t)o * kFmmN3 + kk % kFmmN3) * rows + row] * kOpScale;
    const __half a0 = __float2half_rn(a);
    As[(size_t)o * rows * kSplitK + e] = kk < kFmmN3 ? __float2half_rn(a - __half2float(a0)) : a0;
}

// B'[vcol[e]][:] = split multipole of the e-th V-list source in its class's
// frame, scaled by 2^s (s: the column's largest |value| into [2^14, 2^15)):
// B'[vcol[e]][kk] = part (b0, b1, b0)[kk / 512] of 2^s M_S[g.(kk % 512)];
// colscale[vcol[e]] = 2^-(s + 12) undoes both scales (one block per V-list entry)
__global__ void __launch_bounds__(kThreads)
k_fmm_m2l_gather(const int* __restrict__ v_list, const int* __restrict__ vcol,
                 const int* __restrict__ vsym, const float* __restrict__ M,
                 __half* __restrict__ B, float* __restrict__ colscale,
                 const int* __restrict__ skip) {
    if (skip && *skip) return;
    static_assert(kThreads == kFmmN3, "one thread per expansion point");
    __shared__ float sm[kFmmN3];
    __shared__ float smax[kThreads / 32];
    const int e = blockIdx.x;
    const int m = threadIdx.x;
    const float v = M[(size_t)v_list[e] * kFmmN3 + m];
    sm[m] = v;
    float mx = fabsf(v);
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((m & 31) == 0) smax[m >> 5] = mx;
    __syncthreads();
    mx = smax[0];
#pragma unroll
    for (int w = 1; w < kThreads / 32; ++w) mx = fmaxf(mx, smax[w]);
    int ex = 0;
    if (mx > 0.f && mx <= 3.0e38f) {
        int E;
        frexpf(mx, &E);   // mx = f 2^E, f in [0.5, 1)
        ex = min(100, max(-100, 15 - E));
    }
    const float x = ldexpf(sm[sym_apply(vsym[e], m)], ex);
    const __half x0 = __float2half_rn(x);
    const __half x1 = __float2half_rn(x - __half2float(x0));
    __half* col = B + (size_t)vcol[e] * kSplitK;
    col[m] = x0;
    col[kFmmN3 + m] = x1;
    col[2 * kFmmN3 + m] = x0;
    if (m == 0) colscale[vcol[e]] = ldexpf(1.f, -(ex + kOpScaleExp));
}

// sum of a box's multipole values (the log kernel's level term), fixed order
__global__ void __launch_bounds__(kThreads)
k_fmm_msum(int box0, const float* __restrict__ M, float* __restrict__ msum,
           const int* __restrict__ skip) {
    if (skip && *skip) return;
    const int box = box0 + blockIdx.x;
    __shared__ float sh[kThreads / 32];
    float v = (threadIdx.x < kFmmN3) ? M[(size_t)box * kFmmN3 + threadIdx.x] : 0.f;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < kThreads / 32; ++w) t += sh[w];
        msum[box] = t;
    }
}

// L_T[c][l] = sum over V(T) of scale_c(h) times the entry of C's column vcol[e]
// that g maps to (c, l) (+ 2 lg2(h) msum_S for the log kernel); one block per
// (target box of level >= 2, kernel c).  Warp w takes the V-list entries
// e0 + w, e0 + w + 16, ... (each lane 16 of the 512 points; the permuted reads
// of one 2 KB column component go through L1), and the 16 warps' partial sums
// are added in warp order.
constexpr int kScatWarps = kThreads / 32;
constexpr int kScatPerLane = kFmmN3 / 32;

template <bool KERNEL_K>
__global__ void __launch_bounds__(kThreads)
k_fmm_m2l_scatter(DevTree t, int box0, const float* __restrict__ Cm, const int* __restrict__ vcol,
                  const int* __restrict__ vsym, const float* __restrict__ colscale,
                  const float* __restrict__ msum, float* __restrict__ Lc,
                  const int* __restrict__ skip) {
    if (skip && *skip) return;
    static_assert(kThreads == kFmmN3, "one thread per expansion point in the final sum");
    constexpr int C = KERNEL_K ? 1 : 9;
    constexpr int rows = C * kFmmN3;
    __shared__ float red[kScatWarps][kFmmN3];
    const int box = box0 + blockIdx.x, q = blockIdx.y;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int lev = 0;
    while (lev + 1 <= t.depth && t.lev_off[lev + 1] <= box) ++lev;
    const float h = t.L0 / (float)(1 << lev);
    const int e0 = t.v_off[box], e1 = t.v_off[box + 1];
    // kernel q reads kernel (pi(a), pi(b)) of the canonical frame, sign s_a s_b
    // (q < 6: the pair (a, b) = (pa[q], pb[q])), or pi(a), sign s_a (q = 6 + a)
    const int qa = q < 6 ? (q < 3 ? 0 : (q < 5 ? 1 : 2)) : q - 6;
    const int qb = q < 6 ? (q < 3 ? q : (q < 5 ? q - 2 : 2)) : -1;
    float acc[kScatPerLane];
#pragma unroll
    for (int k = 0; k < kScatPerLane; ++k) acc[k] = 0.f;
    for (int e = e0 + warp; e < e1; e += kScatWarps) {
        const int g = vsym[e];
        int qc = 0;
        bool neg = false;
        if (!KERNEL_K) {
            if (qb >= 0) {
                const int x = sym_pi(g, qa), y = sym_pi(g, qb);
                const int lo = min(x, y), hi = max(x, y);
                qc = lo == 0 ? hi : (lo == 1 ? 2 + hi : 5);
                neg = sym_neg(g, qa) != sym_neg(g, qb);
            } else {
                qc = 6 + sym_pi(g, qa);
                neg = sym_neg(g, qa);
            }
        }
        const int ce = vcol[e];
        const float* col = Cm + (size_t)ce * rows + qc * kFmmN3;
        const float cs = __ldg(colscale + ce);
        const float sc = neg ? -cs : cs;
#pragma unroll
        for (int k = 0; k < kScatPerLane; ++k)
            acc[k] = fmaf(__ldg(col + sym_apply_inv(g, lane + 32 * k)), sc, acc[k]);
    }
#pragma unroll
    for (int k = 0; k < kScatPerLane; ++k) red[warp][lane + 32 * k] = acc[k];
    __syncthreads();
    const int l = threadIdx.x;
    float v = 0.f;
#pragma unroll
    for (int w = 0; w < kScatWarps; ++w) v += red[w][l];
    if (KERNEL_K) {
        const float lh = 2.f * log2f(h);
        float ms = 0.f;
        for (int e = e0; e < e1; ++e) ms += msum[t.v_list[e]];
        Lc[(size_t)box * kFmmN3 + l] = v + lh * ms;
    } else {
        const float scale = q < 6 ? 1.f / (h * h) : 1.f / h;
        Lc[((size_t)box * C + q) * kFmmN3 + l] = v * scale;
    }
}

}  // namespace

// ============================================================================ host tree
struct PmFmmTree {
    int depth = 0, nbox = 0, nleaf = 0;
    float3 origin{};
    float L0 = 0.f;
    std::vector<int> lev_off;
    // device arrays
    int *perm = nullptr, *lev_off_d = nullptr, *box_first = nullptr, *parent = nullptr;
    int *child_off = nullptr, *child = nullptr, *v_off = nullptr, *v_list = nullptr;
    int *u_off = nullptr, *u_list = nullptr, *p2p_order = nullptr, *leaf_chunks = nullptr;
    int3* box_ijk = nullptr;
    float4* sorted = nullptr;
    float* M = nullptr;
    float* Lc = nullptr;     // [nbox][9][512]
    long long p2p_pairs = 0, m2l_pairs = 0;
    // M2L as GEMMs: V-list entry -> column (class start + rank within the class)
    // and the symmetry g that maps its offset to the class's canonical offset
    int nv = 0, np2p = 0, nchunks = 0;
    std::vector<int> cls_start;   // [kNClass + 1]
    int *vcol = nullptr, *vsym = nullptr;
    __half* Bm = nullptr;          // [nv][1536] split multipoles (K-major B')
    float *Cm = nullptr, *msum = nullptr, *colscale = nullptr;
    PmTcGemm gemm[2];              // tensor-core M2L plans: remainder (0), parametrix (1)
    bool gemm_ready[2] = {false, false};
    // the far field (P2M, M2M, M2L, L2L) runs on `far` (highest stream priority)
    // beside the adjacent-leaf P2P on the caller's stream: fork after the source
    // gather, join before L2P
    cudaStream_t far = nullptr;
    int far_prio = 0;              // also set on each far-field launch (kept by graph capture)
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    ~PmFmmTree() {
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        if (far) cudaStreamDestroy(far);
        pm_tcgemm_free(&gemm[0]);
        pm_tcgemm_free(&gemm[1]);
        pm_dfree(vcol); pm_dfree(vsym); pm_dfree(Bm); pm_dfree(Cm); pm_dfree(msum);
        pm_dfree(colscale);
        pm_dfree(perm); pm_dfree(lev_off_d); pm_dfree(box_first); pm_dfree(parent);
        pm_dfree(child_off); pm_dfree(child); pm_dfree(v_off); pm_dfree(v_list);
        pm_dfree(u_off); pm_dfree(u_list); pm_dfree(p2p_order); pm_dfree(leaf_chunks); pm_dfree(box_ijk); pm_dfree(sorted); pm_dfree(M);
        pm_dfree(Lc);
    }
};

void pm_fmm_free(pm_surface* s) {
    delete s->fmm;
    s->fmm = nullptr;
}

// Device bytes the FMM of a surface would allocate on its first apply: the tree
// (sorted sources, multipoles, locals, the gathered M2L columns B (float16) and
// results C (float32), lists), modelled as 3 KB per node + 64 MB, and the
// context's unit-box M2L operators (float16, both kernel families) if they do
// not exist yet.  The torus of 98,304 nodes allocates ~0.25 GB of tree.
size_t pm_fmm_need_bytes(const pm_surface* s) {
    size_t need = 0;
    if (!s->fmm) need += 3072 * (size_t)s->N + ((size_t)64 << 20);
    if (!s->ctx->fmm_opR) need += (size_t)kNClass * 9 * kFmmN3 * kSplitK * sizeof(__half);
    if (!s->ctx->fmm_opK) need += (size_t)kNClass * kFmmN3 * kSplitK * sizeof(__half);
    return need;
}

pm_status pm_fmm_check(pm_surface* s) {
    if (!s->fmm) return PM_OK;
    for (int k = 0; k < 2; ++k)
        if (s->fmm->gemm_ready[k]) PM_TRY(pm_tcgemm_check(&s->fmm->gemm[k]));
    return PM_OK;
}

namespace {

struct Key {
    int x, y, z;
    bool operator==(const Key& o) const { return x == o.x && y == o.y && z == o.z; }
};
struct KeyHash {
    size_t operator()(const Key& k) const {
        return ((size_t)(unsigned)k.x * 73856093u) ^ ((size_t)(unsigned)k.y * 19349663u) ^
               ((size_t)(unsigned)k.z * 83492791u);
    }
};

// Class of a V-list offset d (max |d_i| in {2, 3}) and the symmetry code g with
// d = g d_c (see the M2L section); -1 when d is not a V-list offset.  Axes are
// ranked by |d_a| (descending, ties by axis) to give pi; s_a is the sign of d_a.
int offset_class(int3 d, int* sym) {
    const int ad[3] = {std::abs(d.x), std::abs(d.y), std::abs(d.z)};
    if (std::max({ad[0], ad[1], ad[2]}) < 2 || std::max({ad[0], ad[1], ad[2]}) > 3) return -1;
    int order[3] = {0, 1, 2};
    std::stable_sort(order, order + 3, [&](int a, int b) { return ad[a] > ad[b]; });
    int pi[3];
    for (int k = 0; k < 3; ++k) pi[order[k]] = k;
    const int dv[3] = {d.x, d.y, d.z};
    int g = 0;
    for (int a = 0; a < 3; ++a) {
        g |= pi[a] << (2 * a);
        if (dv[a] < 0) g |= 1 << (6 + a);
    }
    *sym = g;
    const int3 dc = make_int3(ad[order[0]], ad[order[1]], ad[order[2]]);
    for (int c = 0; c < kNClass; ++c) {
        const int3 o = canonical_offset(c);
        if (o.x == dc.x && o.y == dc.y && o.z == dc.z) return c;
    }
    return -1;
}

long long morton(int x, int y, int z) {
    long long m = 0;
    for (int b = 0; b < 20; ++b) {
        m |= (long long)((x >> b) & 1) << (3 * b + 2);
        m |= (long long)((y >> b) & 1) << (3 * b + 1);
        m |= (long long)((z >> b) & 1) << (3 * b);
    }
    return m;
}

// Occupied boxes and interaction counts of a uniform tree of the given depth.
struct LevelBoxes {
    std::vector<Key> keys;
    std::unordered_map<Key, int, KeyHash> index;
};

void build_levels(const std::vector<double>& x, int N, double ox, double oy, double oz,
                  double L0, int depth, std::vector<LevelBoxes>& lv) {
    lv.assign(depth + 1, LevelBoxes());
    const int nb = 1 << depth;
    std::vector<long long> codes;
    for (int i = 0; i < N; ++i) {
        int ix = std::min(nb - 1, std::max(0, (int)std::floor((x[3 * i] - ox) / L0 * nb)));
        int iy = std::min(nb - 1, std::max(0, (int)std::floor((x[3 * i + 1] - oy) / L0 * nb)));
        int iz = std::min(nb - 1, std::max(0, (int)std::floor((x[3 * i + 2] - oz) / L0 * nb)));
        codes.push_back(morton(ix, iy, iz));
        for (int l = depth; l >= 0; --l) {
            Key k{ix >> (depth - l), iy >> (depth - l), iz >> (depth - l)};
            auto& L = lv[l];
            if (L.index.find(k) == L.index.end()) {
                L.index[k] = (int)L.keys.size();
                L.keys.push_back(k);
            }
        }
    }
    // order the boxes of each level by Morton code
    for (int l = 0; l <= depth; ++l) {
        auto& L = lv[l];
        std::sort(L.keys.begin(), L.keys.end(), [](const Key& a, const Key& b) {
            return morton(a.x, a.y, a.z) < morton(b.x, b.y, b.z);
        });
        L.index.clear();
        for (int b = 0; b < (int)L.keys.size(); ++b) L.index[L.keys[b]] = b;
    }
}

}  // namespace

static pm_status fmm_build_tree(pm_surface* s) {
    const int N = s->N;
    const std::vector<double>& x = s->h_x;
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int i = 0; i < N; ++i)
        for (int c = 0; c < 3; ++c) {
            lo[c] = std::min(lo[c], x[3 * i + c]);
            hi[c] = std::max(hi[c], x[3 * i + c]);
        }
    double L0 = 0;
    for (int c = 0; c < 3; ++c) L0 = std::max(L0, hi[c] - lo[c]);
    L0 *= 1.0001;
    const double ox = 0.5 * (lo[0] + hi[0]) - 0.5 * L0, oy = 0.5 * (lo[1] + hi[1]) - 0.5 * L0,
                 oz = 0.5 * (lo[2] + hi[2]) - 0.5 * L0;
    // choose the depth by a cost model calibrated on GB300 with these kernels:
    // about 4 ns per adjacent-leaf pair (P2P) and 1 ns per far-field Chebyshev node pair
    int best_depth = 2;
    double best_cost = 1e300;
    std::vector<LevelBoxes> best_lv;
    const int forced = s->opts.fmm_depth;
    for (int depth = 2; depth <= 8; ++depth) {
        if (forced >= 2 && depth != forced) continue;
        std::vector<LevelBoxes> lv;
        build_levels(x, N, ox, oy, oz, L0, depth, lv);
        // leaf occupancies
        const int nb = 1 << depth;
        std::vector<int> occ(lv[depth].keys.size(), 0);
        for (int i = 0; i < N; ++i) {
            int ix = std::min(nb - 1, std::max(0, (int)std::floor((x[3 * i] - ox) / L0 * nb)));
            int iy = std::min(nb - 1, std::max(0, (int)std::floor((x[3 * i + 1] - oy) / L0 * nb)));
            int iz = std::min(nb - 1, std::max(0, (int)std::floor((x[3 * i + 2] - oz) / L0 * nb)));
            occ[lv[depth].index[Key{ix, iy, iz}]]++;
        }
        int maxocc = *std::max_element(occ.begin(), occ.end());
        double p2p = 0, m2l = 0;
        for (size_t b = 0; b < lv[depth].keys.size(); ++b) {
            const Key k = lv[depth].keys[b];
            for (int dx = -1; dx <= 1; ++dx)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dz = -1; dz <= 1; ++dz) {
                        auto it = lv[depth].index.find(Key{k.x + dx, k.y + dy, k.z + dz});
                        if (it != lv[depth].index.end()) p2p += (double)occ[b] * occ[it->second];
                    }
        }
        for (int l = 2; l <= depth; ++l)
            for (const Key& k : lv[l].keys) {
                const Key p{k.x >> 1, k.y >> 1, k.z >> 1};
                for (int dx = -1; dx <= 1; ++dx)
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dz = -1; dz <= 1; ++dz) {
                            if (lv[l - 1].index.find(Key{p.x + dx, p.y + dy, p.z + dz}) ==
                                lv[l - 1].index.end())
                                continue;
                            for (int c = 0; c < 8; ++c) {
                                Key q{2 * (p.x + dx) + (c >> 2), 2 * (p.y + dy) + ((c >> 1) & 1),
                                      2 * (p.z + dz) + (c & 1)};
                                if (std::max({std::abs(q.x - k.x), std::abs(q.y - k.y),
                                              std::abs(q.z - k.z)}) <= 1)
                                    continue;
                                if (lv[l].index.count(q)) m2l += 1;
                            }
                        }
            }
        const double cost = p2p * 4.0 + m2l * kFmmN3 * (double)kFmmN3 * 1.0;
        if (maxocc <= kMaxLeafPts && cost < best_cost) {
            best_cost = cost;
            best_depth = depth;
            best_lv = lv;
            s->fmm_stats[0] = p2p;
            s->fmm_stats[1] = m2l;
        }
        if (forced < 2 && cost > 4 * best_cost) break;
    }
    if (best_lv.empty()) {
        pm_set_error("pm_fmm_build: no tree depth keeps leaves below %d points", kMaxLeafPts);
        return PM_ERR_INVALID_ARG;
    }
    const int depth = best_depth;
    std::vector<LevelBoxes>& lv = best_lv;
    PmFmmTree* T = new PmFmmTree();
    s->fmm = T;
    {
        int lo = 0, hi = 0;
        PM_CUDA_TRY(cudaDeviceGetStreamPriorityRange(&lo, &hi));
        PM_CUDA_TRY(cudaStreamCreateWithPriority(&T->far, cudaStreamNonBlocking, hi));
        T->far_prio = hi;
        PM_CUDA_TRY(cudaEventCreateWithFlags(&T->ev_fork, cudaEventDisableTiming));
        PM_CUDA_TRY(cudaEventCreateWithFlags(&T->ev_join, cudaEventDisableTiming));
    }
    T->depth = depth;
    T->L0 = (float)L0;
    T->origin = make_float3((float)ox, (float)oy, (float)oz);
    T->lev_off.assign(depth + 2, 0);
    for (int l = 0; l <= depth; ++l) T->lev_off[l + 1] = T->lev_off[l] + (int)lv[l].keys.size();
    T->nbox = T->lev_off[depth + 1];
    T->nleaf = (int)lv[depth].keys.size();
    std::vector<int3> ijk(T->nbox);
    std::vector<int> parent(T->nbox, -1), child_off(T->nbox + 1, 0), child;
    std::vector<std::vector<int>> kids(T->nbox);
    for (int l = 0; l <= depth; ++l)
        for (size_t b = 0; b < lv[l].keys.size(); ++b) {
            const Key k = lv[l].keys[b];
            const int id = T->lev_off[l] + (int)b;
            ijk[id] = make_int3(k.x, k.y, k.z);
            if (l > 0) {
                const int pid = T->lev_off[l - 1] + lv[l - 1].index[Key{k.x >> 1, k.y >> 1, k.z >> 1}];
                parent[id] = pid;
                kids[pid].push_back(id);
            }
        }
    for (int b = 0; b < T->nbox; ++b) {
        child_off[b + 1] = child_off[b] + (int)kids[b].size();
        child.insert(child.end(), kids[b].begin(), kids[b].end());
    }
    // V lists (levels >= 2)
    std::vector<int> v_off(T->nbox + 1, 0), v_list;
    for (int l = 0; l <= depth; ++l)
        for (size_t b = 0; b < lv[l].keys.size(); ++b) {
            const int id = T->lev_off[l] + (int)b;
            if (l >= 2) {
                const Key k = lv[l].keys[b];
                const Key p{k.x >> 1, k.y >> 1, k.z >> 1};
                std::vector<int> vl;
                for (int dx = -1; dx <= 1; ++dx)
                    for (int dy = -1; dy <= 1; ++dy)
                        for (int dz = -1; dz <= 1; ++dz) {
                            if (!lv[l - 1].index.count(Key{p.x + dx, p.y + dy, p.z + dz})) continue;
                            for (int c = 0; c < 8; ++c) {
                                Key q{2 * (p.x + dx) + (c >> 2), 2 * (p.y + dy) + ((c >> 1) & 1),
                                      2 * (p.z + dz) + (c & 1)};
                                if (std::max({std::abs(q.x - k.x), std::abs(q.y - k.y),
                                              std::abs(q.z - k.z)}) <= 1)
                                    continue;
                                auto it = lv[l].index.find(q);
                                if (it != lv[l].index.end()) vl.push_back(T->lev_off[l] + it->second);
                            }
                        }
                std::sort(vl.begin(), vl.end());
                v_list.insert(v_list.end(), vl.begin(), vl.end());
            }
            v_off[id + 1] = (int)v_list.size();
        }
    // points sorted by leaf (Morton order of leaves), U lists
    const int nb = 1 << depth;
    std::vector<int> leaf_of(N);
    std::vector<int> cnt(T->nleaf, 0);
    for (int i = 0; i < N; ++i) {
        int ix = std::min(nb - 1, std::max(0, (int)std::floor((x[3 * i] - ox) / L0 * nb)));
        int iy = std::min(nb - 1, std::max(0, (int)std::floor((x[3 * i + 1] - oy) / L0 * nb)));
        int iz = std::min(nb - 1, std::max(0, (int)std::floor((x[3 * i + 2] - oz) / L0 * nb)));
        leaf_of[i] = lv[depth].index[Key{ix, iy, iz}];
        cnt[leaf_of[i]]++;
    }
    std::vector<int> first(T->nleaf + 1, 0);
    for (int b = 0; b < T->nleaf; ++b) first[b + 1] = first[b] + cnt[b];
    std::vector<int> fill(first.begin(), first.end() - 1), perm(N);
    for (int i = 0; i < N; ++i) perm[fill[leaf_of[i]]++] = i;
    std::vector<int> u_off(T->nleaf + 1, 0), u_list;
    for (int b = 0; b < T->nleaf; ++b) {
        const Key k = lv[depth].keys[b];
        for (int dx = -1; dx <= 1; ++dx)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dz = -1; dz <= 1; ++dz) {
                    auto it = lv[depth].index.find(Key{k.x + dx, k.y + dy, k.z + dz});
                    if (it != lv[depth].index.end()) u_list.push_back(it->second);
                }
        u_off[b + 1] = (int)u_list.size();
    }
    // P2P blocks: (leaf, neighbour, chunk of 128 targets), by decreasing pair
    // count; the blocks that only clear a slice (e beyond the leaf's U list) go last
    std::vector<int> p2p_order;
    {
        std::vector<long long> work;
        for (int b = 0; b < T->nleaf; ++b) {
            const int ne = u_off[b + 1] - u_off[b];
            const int nch = (cnt[b] + kP2PThreads - 1) / kP2PThreads;
            if (nch > kP2PMaxChunks) {
                pm_set_error("pm_fmm_build: leaf with %d points exceeds the P2P chunk range", cnt[b]);
                return PM_ERR_INTERNAL;
            }
            for (int ch = 0; ch < nch; ++ch)
                for (int e = 0; e < kUMax; ++e) {
                    const long long nt = std::min(kP2PThreads, cnt[b] - ch * kP2PThreads);
                    p2p_order.push_back(p2p_code(b, ch, e));
                    work.push_back(e < ne ? nt * cnt[u_list[u_off[b] + e]] : -1);
                }
        }
        std::vector<int> idx(p2p_order.size());
        for (size_t k = 0; k < idx.size(); ++k) idx[k] = (int)k;
        std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return work[x] > work[y]; });
        std::vector<int> sorted(idx.size());
        for (size_t k = 0; k < idx.size(); ++k) sorted[k] = p2p_order[idx[k]];
        p2p_order.swap(sorted);
        T->np2p = (int)p2p_order.size();
    }
    std::vector<int> leaf_chunks;
    for (int b = 0; b < T->nleaf; ++b)
        for (int ch = 0; ch * kL2PThreads < cnt[b]; ++ch) leaf_chunks.push_back((b << 5) | ch);
    T->nchunks = (int)leaf_chunks.size();
    T->p2p_pairs = (long long)s->fmm_stats[0];
    T->m2l_pairs = (long long)s->fmm_stats[1];
    s->fmm_stats[2] = depth;
    s->fmm_stats[3] = T->nbox;
    // device copies
    auto up = [&](auto** d, const auto& h) -> pm_status {
        using E = typename std::remove_reference<decltype(h[0])>::type;
        PM_TRY(pm_dmalloc(d, std::max<size_t>(1, h.size())));
        if (!h.empty())
            PM_CUDA_TRY(cudaMemcpy(*d, h.data(), sizeof(E) * h.size(), cudaMemcpyHostToDevice));
        return PM_OK;
    };
    PM_TRY(up(&T->perm, perm));
    PM_TRY(up(&T->lev_off_d, T->lev_off));
    PM_TRY(up(&T->box_first, first));
    PM_TRY(up(&T->parent, parent));
    PM_TRY(up(&T->child_off, child_off));
    PM_TRY(up(&T->child, child));
    PM_TRY(up(&T->v_off, v_off));
    PM_TRY(up(&T->v_list, v_list));
    PM_TRY(up(&T->u_off, u_off));
    PM_TRY(up(&T->u_list, u_list));
    PM_TRY(up(&T->p2p_order, p2p_order));
    PM_TRY(up(&T->leaf_chunks, leaf_chunks));
    PM_TRY(up(&T->box_ijk, ijk));
    // M2L columns: group the V-list entries by offset class
    {
        const size_t nv = v_list.size();
        std::vector<int> cls(nv), rank(nv), vsym(nv), cnt(kNClass, 0);
        for (int b = 0; b < T->nbox; ++b)
            for (int e = v_off[b]; e < v_off[b + 1]; ++e) {
                const int3 dt = ijk[b], ds = ijk[v_list[e]];
                const int c = offset_class(make_int3(dt.x - ds.x, dt.y - ds.y, dt.z - ds.z), &vsym[e]);
                if (c < 0) {
                    pm_set_error("pm_fmm_build: V-list offset outside the interaction range");
                    return PM_ERR_INTERNAL;
                }
                cls[e] = c;
                rank[e] = cnt[c]++;
            }
        T->cls_start.assign(kNClass + 1, 0);
        for (int c = 0; c < kNClass; ++c) T->cls_start[c + 1] = T->cls_start[c] + cnt[c];
        std::vector<int> vcol(nv);
        for (size_t e = 0; e < nv; ++e) vcol[e] = T->cls_start[cls[e]] + rank[e];
        T->nv = (int)nv;
        PM_TRY(up(&T->vcol, vcol));
        PM_TRY(up(&T->vsym, vsym));
    }
    PM_TRY(pm_dmalloc(&T->sorted, N));
    PM_TRY(pm_dmalloc(&T->M, (size_t)T->nbox * kFmmN3));
    PM_TRY(pm_dmalloc(&T->Lc, (size_t)T->nbox * 9 * kFmmN3));
    // interpolation constants
    FmmConst F;
    std::memset(&F, 0, sizeof(F));
    double cheb[kFmmN], bary[kFmmN];
    for (int k = 0; k < kFmmN; ++k) cheb[k] = std::cos(M_PI * (2 * k + 1) / (2.0 * kFmmN));
    for (int a = 0; a < kFmmN; ++a) {
        double prod = 1.0;
        for (int b = 0; b < kFmmN; ++b)
            if (b != a) prod *= cheb[a] - cheb[b];
        bary[a] = 1.0 / prod;
        F.cheb[a] = (float)cheb[a];
        F.bary[a] = (float)bary[a];
    }
    for (int o = 0; o < 2; ++o)
        for (int m = 0; m < kFmmN; ++m)
            for (int k = 0; k < kFmmN; ++k) {
                const double u = 0.5 * (cheb[k] + (2 * o - 1));
                double v = bary[m];
                for (int b = 0; b < kFmmN; ++b)
                    if (b != m) v *= u - cheb[b];
                F.T[o][m][k] = (float)v;
            }
    PM_CUDA_TRY(cudaMemcpyToSymbol(cF, &F, sizeof(F)));
    return PM_OK;
}

// A tree whose build failed part way is released, so that no later apply uses it.
pm_status pm_fmm_build(pm_surface* s) {
    if (s->fmm) return PM_OK;
    const pm_status st = fmm_build_tree(s);
    if (st != PM_OK) pm_fmm_free(s);
    return st;
}

namespace {

// Unit-box M2L operators of the context (one set per kernel family), built once.
pm_status ensure_m2l_ops(pm_surface* s, int which_K, __half** out) {
    pm_ctx* c = s->ctx;
    std::lock_guard<std::mutex> lk(c->fmm_mu);
    __half*& A = which_K ? c->fmm_opK : c->fmm_opR;
    if (!A) {
        const int rows = which_K ? kFmmN3 : 9 * kFmmN3;
        float* tmp = nullptr;
        __half* split = nullptr;
        PM_TRY(pm_dmalloc(&tmp, (size_t)kNClass * rows * kFmmN3));
        const pm_status st = pm_dmalloc(&split, (size_t)kNClass * rows * kSplitK);
        if (st != PM_OK) {
            pm_dfree(tmp);
            return st;
        }
        cudaStream_t bs = nullptr;
        cudaError_t ce = cudaStreamCreateWithFlags(&bs, cudaStreamNonBlocking);
        if (ce == cudaSuccess) {
            const dim3 g(pm_ceil_div((long long)rows * kFmmN3, 256), kNClass);
            k_fmm_build_op<<<g, 256, 0, bs>>>(which_K, tmp);
            ce = cudaGetLastError();
        }
        if (ce == cudaSuccess) {
            const dim3 g(pm_ceil_div((long long)rows * kSplitK, 256), kNClass);
            k_fmm_split_op<<<g, 256, 0, bs>>>(rows, tmp, split);
            ce = cudaGetLastError();
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(bs);
        }
        if (bs) cudaStreamDestroy(bs);
        pm_dfree(tmp);
        if (ce != cudaSuccess) {
            pm_dfree(split);
            pm_set_error("FMM M2L operators: %s", cudaGetErrorString(ce));
            return PM_ERR_CUDA;
        }
        A = split;
    }
    *out = A;
    return PM_OK;
}

// The gathered multipole and result matrices of the tree and its GEMM plan for
// one kernel family: tiles of 128 operator rows x 256 V-list columns, class by
// class (each class's columns start at cls_start[c]; the last tile of a class
// is narrower), ordered class, column tile, row tile so that the CTAs working
// at one time share a class's operator in L2.
pm_status ensure_m2l_gemm(pm_surface* s, PmFmmTree* T, int which_K, const __half* A) {
    if (!T->Bm) {
        const size_t cols = (size_t)std::max(1, T->nv);
        PM_TRY(pm_dmalloc(&T->Bm, cols * kSplitK));
        PM_TRY(pm_dmalloc(&T->Cm, cols * 9 * kFmmN3));
        PM_TRY(pm_dmalloc(&T->colscale, cols));
        PM_TRY(pm_dmalloc(&T->msum, (size_t)T->nbox));
    }
    if (!T->gemm_ready[which_K]) {
        const int rows = which_K ? kFmmN3 : 9 * kFmmN3;
        std::vector<int> tiles;
        for (int c = 0; c < kNClass; ++c) {
            const int c0 = T->cls_start[c], nc = T->cls_start[c + 1] - c0;
            for (int n0 = 0; n0 < nc; n0 += 256)
                for (int m0 = 0; m0 < rows; m0 += 128) {
                    tiles.push_back(c * rows + m0);
                    tiles.push_back(c0 + n0);
                    tiles.push_back(std::min(256, nc - n0));
                    tiles.push_back(m0);
                }
        }
        PM_TRY(pm_tcgemm_init(&T->gemm[which_K], A, (long long)kNClass * rows, T->Bm,
                              std::max(1, T->nv), kSplitK, 0, tiles, T->Cm, rows,
                              std::max(1, T->nv)));
        T->gemm_ready[which_K] = true;
    }
    return PM_OK;
}

}  // namespace

extern "C" pm_status pm_selftest_fmm_classes(int* cls, int* sym, int* canon) {
    if (!cls || !sym || !canon) {
        pm_set_error("pm_selftest_fmm_classes: NULL argument");
        return PM_ERR_INVALID_ARG;
    }
    for (int c = 0; c < kNClass; ++c) {
        const int3 o = canonical_offset(c);
        canon[3 * c] = o.x;
        canon[3 * c + 1] = o.y;
        canon[3 * c + 2] = o.z;
    }
    for (int dx = -3; dx <= 3; ++dx)
        for (int dy = -3; dy <= 3; ++dy)
            for (int dz = -3; dz <= 3; ++dz) {
                const int k = ((dx + 3) * 7 + (dy + 3)) * 7 + (dz + 3);
                int g = 0;
                cls[k] = offset_class(make_int3(dx, dy, dz), &g);
                sym[k] = cls[k] >= 0 ? g : 0;
            }
    return PM_OK;
}

// Partial slices the FMM writes per target (U-list neighbours + far field).
int pm_fmm_splits() { return kUMax + 1; }

pm_status pm_fmm_apply(pm_surface* s, int which_K, cudaStream_t st) {
    PM_TRY(pm_fmm_build(s));
    PmFmmTree* T = s->fmm;
    DevTree t;
    t.N = s->N;
    t.depth = T->depth;
    t.nlev = T->depth + 1;
    t.nbox_total = T->nbox;
    t.origin = T->origin;
    t.L0 = T->L0;
    t.perm = T->perm;
    t.lev_off = T->lev_off_d;
    t.box_ijk = T->box_ijk;
    t.box_first = T->box_first;
    t.parent = T->parent;
    t.child_off = T->child_off;
    t.child = T->child;
    t.v_off = T->v_off;
    t.v_list = T->v_list;
    t.u_off = T->u_off;
    t.u_list = T->u_list;
    t.p2p_order = T->p2p_order;
    t.leaf_chunks = T->leaf_chunks;
    const int* skip = s->skip_flag;
    const int depth = T->depth;
    if (s->opts.fmm_tensor_m2l) {       // operators and GEMM plan (host side, before the fork)
        __half* A = nullptr;
        PM_TRY(ensure_m2l_ops(s, which_K, &A));
        PM_TRY(ensure_m2l_gemm(s, T, which_K, A));
    }
    k_fmm_gather<<<pm_ceil_div(s->N, 256), 256, 0, st>>>(s->src32, T->perm, s->N, T->sorted, skip);
    PM_CUDA_TRY(cudaGetLastError());
    // fork: the far field on T->far, the P2P on st (they share only the sorted sources);
    // with the knob fmm_streams = 1 everything stays on st, in the same order
    const bool two = s->fmm_streams != 1;
    cudaStream_t fs = two ? T->far : st;
    const int pr = two ? T->far_prio : 0;
    const dim3 bt(kThreads);
    if (two) {
        PM_CUDA_TRY(cudaEventRecord(T->ev_fork, st));
        PM_CUDA_TRY(cudaStreamWaitEvent(fs, T->ev_fork, 0));
    }
    PM_CUDA_TRY(pm_launch_prio(k_fmm_p2m, dim3(T->nleaf), bt, 0, fs, pr, t,
                               (const float4*)T->sorted, T->M, skip));
    for (int l = depth - 1; l >= 2; --l) {
        const int nb = T->lev_off[l + 1] - T->lev_off[l];
        PM_CUDA_TRY(pm_launch_prio(k_fmm_m2m, dim3(nb), bt, 0, fs, pr, t, l, T->M, skip));
    }
    const int b2 = T->lev_off[2], nm2l = T->nbox - b2;
    if (s->opts.fmm_tensor_m2l) {
        if (which_K && nm2l > 0)
            PM_CUDA_TRY(pm_launch_prio(k_fmm_msum, dim3(nm2l), bt, 0, fs, pr, b2,
                                       (const float*)T->M, T->msum, skip));
        if (T->nv > 0)
            PM_CUDA_TRY(pm_launch_prio(k_fmm_m2l_gather, dim3(T->nv), bt, 0, fs, pr,
                                       (const int*)T->v_list, (const int*)T->vcol,
                                       (const int*)T->vsym, (const float*)T->M, T->Bm,
                                       T->colscale, skip));
        {
            PhaseTimer pt(s, PM_PHASE_FMM_M2L, fs);
            PM_TRY(pm_tcgemm_run(&T->gemm[which_K], s->ctx->num_sms, skip, fs, pr));
        }
        if (which_K)
            PM_CUDA_TRY(pm_launch_prio(k_fmm_m2l_scatter<true>, dim3(nm2l, 1), bt, 0, fs, pr, t,
                                       b2, (const float*)T->Cm, (const int*)T->vcol,
                                       (const int*)T->vsym, (const float*)T->colscale,
                                       (const float*)T->msum, T->Lc, skip));
        else
            PM_CUDA_TRY(pm_launch_prio(k_fmm_m2l_scatter<false>, dim3(nm2l, 9), bt, 0, fs, pr,
                                       t, b2, (const float*)T->Cm, (const int*)T->vcol,
                                       (const int*)T->vsym, (const float*)T->colscale,
                                       (const float*)T->msum, T->Lc, skip));
        s->launch_total += 3 + (which_K ? 1 : 0);
    } else if (which_K) {
        PM_CUDA_TRY(pm_launch_prio(k_fmm_m2l<true>, dim3(nm2l), bt, 0, fs, pr, t, b2,
                                   (const float*)T->M, T->Lc, skip));
    } else {
        PM_CUDA_TRY(pm_launch_prio(k_fmm_m2l<false>, dim3(nm2l), bt, 0, fs, pr, t, b2,
                                   (const float*)T->M, T->Lc, skip));
    }
    for (int l = 3; l <= depth; ++l) {
        const int nb = T->lev_off[l + 1] - T->lev_off[l];
        if (which_K)
            PM_CUDA_TRY(pm_launch_prio(k_fmm_l2l<1>, dim3(nb), bt, 0, fs, pr, t, l, T->Lc, skip));
        else
            PM_CUDA_TRY(pm_launch_prio(k_fmm_l2l<9>, dim3(nb), bt, 0, fs, pr, t, l, T->Lc, skip));
    }
    if (two) PM_CUDA_TRY(cudaEventRecord(T->ev_join, fs));
    float2* out = reinterpret_cast<float2*>(s->partial);
    const int g2 = T->np2p;
    {
        PhaseTimer pt(s, PM_PHASE_FMM_P2P, st);
        if (which_K)
            k_fmm_p2p<true><<<g2, kP2PThreads, 0, st>>>(t, T->sorted, s->tgt32, s->eps2, out, skip);
        else
            k_fmm_p2p<false><<<g2, kP2PThreads, 0, st>>>(t, T->sorted, s->tgt32, s->eps2, out, skip);
    }
    // join: L2P reads the far field's local expansions
    if (two) PM_CUDA_TRY(cudaStreamWaitEvent(st, T->ev_join, 0));
    if (which_K) {
        k_fmm_l2p<true><<<T->nchunks, kL2PThreads, 0, st>>>(t, s->tgt32, T->Lc, out, skip);
    } else {
        k_fmm_l2p<false><<<T->nchunks, kL2PThreads, 0, st>>>(t, s->tgt32, T->Lc, out, skip);
    }
    s->launch_total += 5 + 2 * std::max(0, depth - 2);
    PM_CUDA_TRY(cudaGetLastError());
    return PM_OK;
}
