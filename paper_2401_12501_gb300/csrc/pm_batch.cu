// Batched (multi right-hand side) applies and solves on one surface.
//
// Many right-hand sides on the same surface and coefficient share every
// pair's geometry: for the remainder, r, |r|^2, 1/|r|^2, n'.r and m.r are
// target/source properties, so the pair factor g = (1/|r|^2)((n'.r)^2/|r|^2 + m.r)
// is formed once and each right-hand side adds s_r * g (one FMA per RHS).
// The same holds for the parametrix (one lg2 per pair) and for the float-float
// accurate sums (one float-float product per RHS).
//
// The batched solve runs independent GMRES iterations for all right-hand
// sides in lockstep (one batched apply per Arnoldi step, per-RHS Krylov bases
// and Givens rotations, per-RHS convergence flags); iterative refinement uses
// batched float-float residuals; u = K~ sigma uses the batched float-float
// parametrix sum.
#include "pm_ff.cuh"
#include "pm_internal.cuh"

#include <map>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

namespace {

constexpr int kThreads = 128;
constexpr int kRB = 16;         // right-hand sides per block (float32) unless tuned (8, 16 or 32)
constexpr int kRBff = 16;       // right-hand sides per block (float-float); 8 for batches of <= 8
constexpr int kTile = 256;
constexpr int kStage = 512;

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

// s[r][j] = w_j sigma_r[j] / a_j (float32), sig32[r][patch][k] = sigma_r
__global__ void k_prep32_multi(const double* __restrict__ sigma, long long ld_sigma,
                               const double* __restrict__ wa, float* __restrict__ s, int N,
                               int pp, int ppad, int npatch, float* __restrict__ sig32,
                               const int* __restrict__ skip) {
    if (skip && *skip) return;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (j >= N) return;
    const double v = sigma[r * ld_sigma + j];
    s[(size_t)r * N + j] = (float)(wa[j] * v);
    const int P = j / pp;
    sig32[((size_t)r * npatch + P) * ppad + (j - P * pp)] = (float)v;
}

// float32 smooth sums for a group of RB right-hand sides (blockIdx.z); sources are
// staged kStage (RB <= 16) or kStage / 2 (RB = 32) at a time
template <int RB>
constexpr int multi_stage() { return RB <= 16 ? kStage : kStage / 2; }

template <bool KERNEL_K, int RB>
__global__ void __launch_bounds__(kThreads)
k_direct_multi32(const float4* __restrict__ pos, const float* __restrict__ s, int nrhs,
                 const float4* __restrict__ tgt, int N, int chunk, float eps2,
                 float2* __restrict__ partial, int nsplit, const int* __restrict__ skip) {
    if (skip && *skip) return;
    static_assert(RB % 4 == 0 && RB >= 4 && RB <= 32, "RB right-hand sides in float4 groups");
    constexpr int kSt = multi_stage<RB>();
    __shared__ float4 sP[kSt];
    __shared__ float4 sS[kSt][RB / 4];          // strengths of RB right-hand sides per source
    const int tid = threadIdx.x;
    const int i = blockIdx.x * kThreads + tid;
    const int r0 = blockIdx.z * RB;
    const int nr = min(RB, nrhs - r0);
    const int tbase = blockIdx.x * kThreads, tend = tbase + kThreads;
    float tx = 0, ty = 0, tz = 0, nx = 0, ny = 0, nz = 0, mx = 0, my = 0, mz = 0;
    if (i < N) {
        const float4 a = tgt[i];
        tx = a.x; ty = a.y; tz = a.z;
        if (!KERNEL_K) {
            const float4 b = tgt[N + i], c = tgt[2 * N + i];
            nx = b.x; ny = b.y; nz = b.z;
            mx = c.x; my = c.y; mz = c.z;
        }
    }
    float hi[RB], lo[RB];
#pragma unroll
    for (int q = 0; q < RB; ++q) hi[q] = lo[q] = 0.f;
    const int s0 = blockIdx.y * chunk;
    const int s1 = min(s0 + chunk, N);
    for (int base = s0; base < s1; base += kSt) {
        const int len = min(kSt, s1 - base);
        __syncthreads();
        for (int j = tid; j < len; j += kThreads) {
            sP[j] = pos[base + j];
            float v[RB];
#pragma unroll
            for (int q = 0; q < RB; ++q) v[q] = (q < nr) ? s[(size_t)(r0 + q) * N + base + j] : 0.f;
#pragma unroll
            for (int q = 0; q < RB / 4; ++q)
                sS[j][q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        }
        __syncthreads();
        for (int j0 = 0; j0 < len; j0 += kTile) {
            const int j1 = min(j0 + kTile, len);
            const bool own = KERNEL_K && !(base + j1 <= tbase || base + j0 >= tend);
            float part[RB];
#pragma unroll
            for (int q = 0; q < RB; ++q) part[q] = 0.f;
#pragma unroll 2
            for (int j = j0; j < j1; ++j) {
                const float4 p = sP[j];
                const float dx = tx - p.x, dy = ty - p.y, dz = tz - p.z;
                float gfac;
                if (KERNEL_K) {
                    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
                    gfac = (own && base + j == i) ? 0.f : lg2_approx(r2);
                } else {
                    const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
                    const float inv = rcp_approx(r2);
                    const float nr2 = fmaf(nx, dx, fmaf(ny, dy, nz * dz));
                    const float mr = fmaf(mx, dx, fmaf(my, dy, mz * dz));
                    gfac = inv * fmaf(nr2, nr2 * inv, mr);
                }
#pragma unroll
                for (int q = 0; q < RB / 4; ++q) {
                    const float4 sv = sS[j][q];
                    part[4 * q] = fmaf(sv.x, gfac, part[4 * q]);
                    part[4 * q + 1] = fmaf(sv.y, gfac, part[4 * q + 1]);
                    part[4 * q + 2] = fmaf(sv.z, gfac, part[4 * q + 2]);
                    part[4 * q + 3] = fmaf(sv.w, gfac, part[4 * q + 3]);
                }
            }
#pragma unroll
            for (int q = 0; q < RB; ++q) two_sum_acc(hi[q], lo[q], part[q]);
        }
    }
    if (i < N) {
        const float sc = KERNEL_K ? (float)(M_LN2 / (4.0 * M_PI)) : 1.f;
#pragma unroll
        for (int q = 0; q < RB; ++q)
            if (q < nr)
                partial[((size_t)(r0 + q) * nsplit + blockIdx.y) * N + i] =
                    make_float2(hi[q] * sc, lo[q] * sc);
    }
}

// out_r[i] = sum_s partial[r][s][i] + sum_b C[b,:] . sigma_r[patch_b]   (warp per (row, rhs))
__global__ void __launch_bounds__(256)
k_near_multi32(int N, int ppad, int npatch, const int* __restrict__ row_ptr,
               const int* __restrict__ blk_patch, const float* __restrict__ vals,
               const float* __restrict__ sig32, const float2* __restrict__ partial, int nsplit,
               double* __restrict__ out, long long ld_out, const int* __restrict__ skip) {
    if (skip && *skip) return;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int r = blockIdx.y;
    if (warp >= N) return;
    const int i = warp;
    float hi = 0.f, lo = 0.f;
    for (int sp = lane; sp < nsplit; sp += 32) {
        const float2 v = partial[((size_t)r * nsplit + sp) * N + i];
        two_sum_acc(hi, lo, v.x);
        lo += v.y;
    }
    const int q4 = ppad >> 2;
    const int rb = row_ptr[i];
    const int total = (row_ptr[i + 1] - rb) * q4;
    const float4* v4 = reinterpret_cast<const float4*>(vals) + (size_t)rb * q4;
    const float4* s4 = reinterpret_cast<const float4*>(sig32 + (size_t)r * npatch * ppad);
    float acc = 0.f;
    for (int e = lane; e < total; e += 32) {
        const int b = e / q4;
        const float4 v = __ldg(v4 + e);
        const float4 x = __ldg(s4 + (size_t)blk_patch[rb + b] * q4 + (e - b * q4));
        acc = fmaf(v.x, x.x, fmaf(v.y, x.y, fmaf(v.z, x.z, fmaf(v.w, x.w, acc))));
    }
    two_sum_acc(hi, lo, acc);
    for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_down_sync(0xffffffffu, hi, o);
        const float l2 = __shfl_down_sync(0xffffffffu, lo, o);
        two_sum_acc(hi, lo, h2);
        lo += l2;
    }
    if (lane == 0) out[r * ld_out + i] = (double)hi + (double)lo;
}

// The same sums, one block per (patch, chunk of 32 right-hand sides): the rows of a
// patch share most of their near patches, so the block stages sigma of the union of
// its rows' near patches for its 32 right-hand sides in shared memory ([node][rhs],
// row stride 33 so that both the staging writes and the lane-per-rhs reads avoid bank
// conflicts), and each warp walks its rows' correction blocks with broadcast loads of
// the values, lane = right-hand side.  Each correction value is read once per 32
// right-hand sides instead of once per right-hand side.
constexpr int kPatchRhs = 32;

// R right-hand sides per block (R = 32, or 8 for small batches): lane = sub-row *
// R + rhs, so a warp takes 32 / R rows at a time and no lane idles when the
// batch has only 8 right-hand sides.  Shared memory: [u * ppad + k][R + 1].
template <int R>
__global__ void __launch_bounds__(256)
k_near_multi32_patch(int N, int pp, int ppad, int npatch, const int* __restrict__ row_ptr,
                     const int* __restrict__ blk_u, const int* __restrict__ pu_ptr,
                     const int* __restrict__ pu_list, const float* __restrict__ vals,
                     const float* __restrict__ sig32, const float2* __restrict__ partial,
                     int nsplit, int nrhs, double* __restrict__ out, long long ld_out,
                     const int* __restrict__ skip) {
    if (skip && *skip) return;
    static_assert(32 % R == 0, "R divides the warp");
    constexpr int kSub = 32 / R;                        // rows per warp step
    constexpr int kLd = R + 1;
    extern __shared__ float shs[];
    const int P = blockIdx.x;
    const int r0 = blockIdx.y * R;
    const int nr = min(R, nrhs - r0);
    const int u0 = pu_ptr[P], U = pu_ptr[P + 1] - u0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // stage: index e = ((u * R + rr) * ppad + k): k fastest, contiguous in global memory
    const int total = U * R * ppad;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int k = e % ppad, t = e / ppad;
        const int rr = t % R, u = t / R;
        float v = 0.f;
        if (rr < nr && k < pp)
            v = sig32[(size_t)(r0 + rr) * npatch * ppad + (size_t)pu_list[u0 + u] * ppad + k];
        shs[(u * ppad + k) * kLd + rr] = v;
    }
    __syncthreads();
    const int sub = lane / R, rr = lane - sub * R;
    const int r = r0 + rr;
    const bool act = rr < nr;
    const int q4 = ppad >> 2;
    for (int t0 = warp * kSub; t0 < pp; t0 += (blockDim.x >> 5) * kSub) {
        const int t = t0 + sub;
        const bool row_ok = t < pp;
        const int i = P * pp + (row_ok ? t : 0);
        float hi = 0.f, lo = 0.f;
        if (act && row_ok)
            for (int sp = 0; sp < nsplit; ++sp) {
                const float2 v = partial[((size_t)r * nsplit + sp) * N + i];
                two_sum_acc(hi, lo, v.x);
                lo += v.y;
            }
        float acc = 0.f;
        const int b0 = row_ok ? row_ptr[i] : 0, b1 = row_ok ? row_ptr[i + 1] : 0;
        for (int b = b0; b < b1; ++b) {
            const float4* c4 = reinterpret_cast<const float4*>(vals + (size_t)b * ppad);
            const float* su = shs + blk_u[b] * ppad * kLd + rr;
            for (int k4 = 0; k4 < q4; ++k4) {
                const float4 c = __ldg(c4 + k4);
                const float* sk = su + 4 * k4 * kLd;
                acc = fmaf(c.x, sk[0], fmaf(c.y, sk[kLd], fmaf(c.z, sk[2 * kLd], fmaf(c.w, sk[3 * kLd], acc))));
            }
        }
        two_sum_acc(hi, lo, acc);
        if (act && row_ok) out[r * ld_out + i] = (double)hi + (double)lo;
    }
}

// ------------------------------------------------------------------ float-float batched sums
// (arithmetic and the coordinate split in pm_ff.cuh)
using pmff::ff;
using pmff::ff_add_lazy;
using pmff::ff_log_lazy;
using pmff::ff_mul;
using pmff::ff_mul_lazy;
using pmff::ff_norm;
using pmff::ff_rcp_lazy;
using pmff::ff_sqr_lazy;
using pmff::fast_two_sum;

// float-float strengths: sff[r][j] = (hi, lo) of w_j sigma_r[j] / a_j
__global__ void k_prep_ff_multi(const double* __restrict__ sigma, long long ld_sigma,
                                const double* __restrict__ wa, float2* __restrict__ sff, int N,
                                const int* __restrict__ skip) {
    if (skip && *skip) return;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (j >= N) return;
    const double v = wa[j] * sigma[r * ld_sigma + j];
    const float h = (float)v;
    sff[(size_t)r * N + j] = make_float2(h, (float)(v - (double)h));
}

// src_ff: source coordinates (their .w strengths are not read; sff holds the
// strengths of every right-hand side) -- plain float-float pairs for the
// remainder, the grid split for the parametrix (pm_ffsum.cu)
template <bool KERNEL_K, int RB>
__global__ void __launch_bounds__(kThreads)
k_direct_multi_ff(const float4* __restrict__ src_ff, const float2* __restrict__ sff, int nrhs,
                  const float4* __restrict__ tg, const float4* __restrict__ log_tab, int N,
                  int chunk, float2* __restrict__ partial, int nsplit,
                  const int* __restrict__ skip) {
    if (skip && *skip) return;
    constexpr int kSt = 256;
    __shared__ float4 sh[2 * kSt];
    __shared__ float2 sS[RB][kSt];
    __shared__ float4 stab[128];
    const int tid = threadIdx.x;
    const int i = blockIdx.x * kThreads + tid;
    const int r0 = blockIdx.z * RB;
    const int nr = min(RB, nrhs - r0);
    const int tbase = blockIdx.x * kThreads, tend = tbase + kThreads;
    if (KERNEL_K)
        for (int k = tid; k < 128; k += kThreads) stab[k] = log_tab[k];
    ff X[3], NP[3], MM[3];
    if (KERNEL_K) {
        // src_ff = grid-split coordinates (pm_ffsum.cu); the target's own entry gives X
        const float4 a = (i < N) ? src_ff[2 * (size_t)i] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 b = (i < N) ? src_ff[2 * (size_t)i + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
        X[0] = ff{a.x, b.x}; X[1] = ff{a.y, b.y}; X[2] = ff{a.z, b.z};
    } else {
        float4 v[6];
        for (int q = 0; q < 6; ++q) v[q] = (i < N) ? tg[6 * (size_t)i + q] : make_float4(0.f, 0.f, 0.f, 0.f);
        X[0] = ff{v[0].x, v[1].x}; X[1] = ff{v[0].y, v[1].y}; X[2] = ff{v[0].z, v[1].z};
        NP[0] = ff{v[2].x, v[3].x}; NP[1] = ff{v[2].y, v[3].y}; NP[2] = ff{v[2].z, v[3].z};
        MM[0] = ff{v[4].x, v[5].x}; MM[1] = ff{v[4].y, v[5].y}; MM[2] = ff{v[4].z, v[5].z};
    }
    ff acc[RB];
#pragma unroll
    for (int q = 0; q < RB; ++q) acc[q] = ff{0.f, 0.f};
    const int s0 = blockIdx.y * chunk;
    const int s1 = min(s0 + chunk, N);
    for (int base = s0; base < s1; base += kSt) {
        const int len = min(kSt, s1 - base);
        __syncthreads();
        for (int j = tid; j < 2 * len; j += kThreads) sh[j] = src_ff[2 * (size_t)base + j];
        for (int j = tid; j < len; j += kThreads)
#pragma unroll
            for (int q = 0; q < RB; ++q)
                sS[q][j] = (q < nr) ? sff[(size_t)(r0 + q) * N + base + j] : make_float2(0.f, 0.f);
        __syncthreads();
        const bool own = !(base + len <= tbase || base >= tend);
        for (int j = 0; j < len; ++j) {
            if (own && base + j == i) continue;
            const float4 A = sh[2 * j], B = sh[2 * j + 1];
            const ff dx = KERNEL_K ? pmff::ff_grid_sub(X[0], A.x, B.x) : pmff::ff_sub(X[0], ff{A.x, B.x});
            const ff dy = KERNEL_K ? pmff::ff_grid_sub(X[1], A.y, B.y) : pmff::ff_sub(X[1], ff{A.y, B.y});
            const ff dz = KERNEL_K ? pmff::ff_grid_sub(X[2], A.z, B.z) : pmff::ff_sub(X[2], ff{A.z, B.z});
            const ff r2 = ff_add_lazy(ff_add_lazy(ff_sqr_lazy(dx), ff_sqr_lazy(dy)), ff_sqr_lazy(dz));
            ff gfac;
            if (KERNEL_K) {
                gfac = ff_norm(ff_log_lazy(r2, stab));
            } else {
                const ff inv = ff_rcp_lazy(r2);
                const ff nr2 = ff_norm(ff_add_lazy(ff_add_lazy(ff_mul_lazy(NP[0], dx),
                                                               ff_mul_lazy(NP[1], dy)),
                                                   ff_mul_lazy(NP[2], dz)));
                const ff mr = ff_add_lazy(ff_add_lazy(ff_mul_lazy(MM[0], dx), ff_mul_lazy(MM[1], dy)),
                                          ff_mul_lazy(MM[2], dz));
                const ff inner = ff_norm(ff_add_lazy(ff_mul_lazy(nr2, ff_mul_lazy(nr2, inv)), mr));
                gfac = ff_mul(inv, inner);
            }
#pragma unroll
            for (int q = 0; q < RB; ++q) {
                // s * g in float-float (product and its error), then a lazy
                // float-float accumulation: TwoSum on the high parts, all error
                // terms summed in the low part (renormalised at the end)
                const float2 sv = sS[q][j];
                const float p = sv.x * gfac.h;
                float e = fmaf(sv.x, gfac.h, -p);
                e = fmaf(sv.x, gfac.l, fmaf(sv.y, gfac.h, e));
                const float t = acc[q].h + p;
                const float bp = t - acc[q].h;
                acc[q].l += ((acc[q].h - (t - bp)) + (p - bp)) + e;
                acc[q].h = t;
            }
        }
    }
    if (i < N) {
#pragma unroll
        for (int q = 0; q < RB; ++q) {
            if (q >= nr) continue;
            ff v;
            fast_two_sum(acc[q].h, acc[q].l, v.h, v.l);
            if (KERNEL_K) v = ff_mul(v, ff{(float)(1.0 / (4.0 * M_PI)),
                                           (float)(1.0 / (4.0 * M_PI) - (double)(float)(1.0 / (4.0 * M_PI)))});
            partial[((size_t)(r0 + q) * nsplit + blockIdx.y) * N + i] = make_float2(v.h, v.l);
        }
    }
}

// float64 near field + float-float split partials, warp per (row, rhs)
__global__ void __launch_bounds__(256)
k_near_multi64(int N, int pp, const int* __restrict__ row_ptr, const int* __restrict__ blk_patch,
               const double* __restrict__ vals, const double* __restrict__ sigma,
               long long ld_sigma, const float2* __restrict__ partial, int nsplit,
               double* __restrict__ out, long long ld_out, const int* __restrict__ skip) {
    if (skip && *skip) return;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int r = blockIdx.y;
    if (warp >= N) return;
    const int i = warp;
    double acc = 0.0;
    for (int sp = lane; sp < nsplit; sp += 32) {
        const float2 v = partial[((size_t)r * nsplit + sp) * N + i];
        acc += (double)v.x + (double)v.y;
    }
    const double* sg = sigma + r * ld_sigma;
    for (int b = row_ptr[i]; b < row_ptr[i + 1]; ++b) {
        const double* v = vals + (size_t)b * pp;
        const double* x = sg + (size_t)blk_patch[b] * pp;
        for (int k = lane; k < pp; k += 32) acc += v[k] * x[k];
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (lane == 0) out[r * ld_out + i] = acc;
}

}  // namespace

// ============================================================================ batched apply
struct PmBatchWork {
    int cap = 0;               // right-hand sides the buffers hold
    float* s32 = nullptr;      // [cap][N]
    float* sig32 = nullptr;    // [cap][npatch][ppad]
    float2* sff = nullptr;     // [cap][N]
    float2* part = nullptr;    // [cap][nsplit_max][N]
    int nsplit_max = 0;
    // patch-blocked near field: per patch the union of its rows' near patches, per
    // correction block its index in that union (built once from the CSR)
    int *pu_ptr = nullptr, *pu_list = nullptr, *blk_u = nullptr;
    int umax = 0;
    bool patch_tried = false;
};

void pm_batch_free(pm_surface* s) {
    if (!s->batch) return;
    pm_dfree(s->batch->s32);
    pm_dfree(s->batch->sig32);
    pm_dfree(s->batch->sff);
    pm_dfree(s->batch->part);
    pm_dfree(s->batch->pu_ptr);
    pm_dfree(s->batch->pu_list);
    pm_dfree(s->batch->blk_u);
    delete s->batch;
    s->batch = nullptr;
}

static pm_status batch_ensure(pm_surface* s, int nrhs) {
    const int nsplit_max = 8;
    if (s->batch && s->batch->cap >= nrhs) return PM_OK;
    pm_batch_free(s);
    s->batch = new PmBatchWork();
    PmBatchWork& B = *s->batch;
    B.cap = nrhs;
    B.nsplit_max = nsplit_max;
    PM_TRY(pm_dmalloc(&B.s32, (size_t)nrhs * s->N));
    PM_TRY(pm_dmalloc(&B.sig32, (size_t)nrhs * s->npatch * s->ppad));
    PM_CUDA_TRY(cudaMemset(B.sig32, 0, sizeof(float) * (size_t)nrhs * s->npatch * s->ppad));
    PM_TRY(pm_dmalloc(&B.sff, (size_t)nrhs * s->N));
    PM_TRY(pm_dmalloc(&B.part, (size_t)nrhs * nsplit_max * s->N));
    return PM_OK;
}

// launch shape of the batched float32 sums (tunable): right-hand sides per block
// and blocks aimed at per SM
static int batch_rb(const pm_surface* s) {
    return (s->batch_rb == 8 || s->batch_rb == 32) ? s->batch_rb : kRB;
}
static int batch_bps(const pm_surface* s) {
    return (s->batch_bps >= 1 && s->batch_bps <= 16) ? s->batch_bps : 8;
}

static int batch_splits(const pm_surface* s, int nrhs, int rb, int bps) {
    const int tblocks = pm_ceil_div(s->N, kThreads) * pm_ceil_div(nrhs, rb);
    const int want = bps * s->ctx->num_sms;
    int ns = (want + tblocks / 2) / tblocks;
    return std::max(1, std::min(ns, std::min(8, std::max(1, s->N / 256))));
}

// Near-patch unions of every patch (see k_near_multi32_patch); umax = 0 when the
// largest union's staging would not fit in shared memory (the per-row kernel is used).
static pm_status build_patch_unions(pm_surface* s, PmBatchWork& B) {
    B.patch_tried = true;
    const int N = s->N, np = s->npatch, pp = s->pp;
    std::vector<int> rp(N + 1), bp(s->nblk);
    PM_CUDA_TRY(cudaMemcpy(rp.data(), s->row_ptr, sizeof(int) * (N + 1), cudaMemcpyDeviceToHost));
    PM_CUDA_TRY(cudaMemcpy(bp.data(), s->blk_patch, sizeof(int) * s->nblk, cudaMemcpyDeviceToHost));
    std::vector<int> ptr(np + 1, 0), list, bu(s->nblk, 0);
    int umax = 0;
    for (int P = 0; P < np; ++P) {
        std::vector<int> un;
        for (int i = P * pp; i < (P + 1) * pp; ++i)
            for (int b = rp[i]; b < rp[i + 1]; ++b) un.push_back(bp[b]);
        std::sort(un.begin(), un.end());
        un.erase(std::unique(un.begin(), un.end()), un.end());
        for (int i = P * pp; i < (P + 1) * pp; ++i)
            for (int b = rp[i]; b < rp[i + 1]; ++b)
                bu[b] = (int)(std::lower_bound(un.begin(), un.end(), bp[b]) - un.begin());
        list.insert(list.end(), un.begin(), un.end());
        ptr[P + 1] = (int)list.size();
        umax = std::max(umax, (int)un.size());
    }
    const size_t smem = (size_t)umax * s->ppad * 33 * sizeof(float);
    constexpr int kSmemCap = 200 * 1024;
    if (smem > (size_t)kSmemCap) return PM_OK;         // too large: keep the per-row kernel
    PM_TRY(pm_dmalloc(&B.pu_ptr, ptr.size()));
    PM_TRY(pm_dmalloc(&B.pu_list, std::max<size_t>(1, list.size())));
    PM_TRY(pm_dmalloc(&B.blk_u, std::max<size_t>(1, bu.size())));
    PM_CUDA_TRY(cudaMemcpy(B.pu_ptr, ptr.data(), sizeof(int) * ptr.size(), cudaMemcpyHostToDevice));
    PM_CUDA_TRY(cudaMemcpy(B.pu_list, list.data(), sizeof(int) * list.size(), cudaMemcpyHostToDevice));
    PM_CUDA_TRY(cudaMemcpy(B.blk_u, bu.data(), sizeof(int) * bu.size(), cudaMemcpyHostToDevice));
    // the attribute is process-wide: always the same cap, so that surfaces prepared by
    // different threads never lower it under one another's launches
    PM_CUDA_TRY(cudaFuncSetAttribute(k_near_multi32_patch<kPatchRhs>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap));
    PM_CUDA_TRY(cudaFuncSetAttribute(k_near_multi32_patch<8>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemCap));
    B.umax = umax;
    return PM_OK;
}

// out[r*ld_out + i] = (R~ or K~) sigma_r, r < nrhs; sigma_r at sigma + r*ld_sigma.
pm_status pm_apply_batch(pm_surface* s, int kernel_K, const double* sigma, long long ld_sigma,
                         double* out, long long ld_out, int nrhs, pm_precision prec,
                         cudaStream_t st) {
    if (prec != PM_PREC_FP32 && prec != PM_PREC_FF) {
        pm_set_error("batched apply: precision %d has no multi-RHS form", (int)prec);
        return PM_ERR_INVALID_ARG;
    }
    PM_TRY(batch_ensure(s, nrhs));
    PmBatchWork& B = *s->batch;
    const int N = s->N;
    const int* skip = s->skip_flag;
    dim3 gp(pm_ceil_div(N, 256), nrhs);
    if (prec == PM_PREC_FF) {
        // 8 right-hand sides per block when the batch has no more: the per-RHS
        // float-float work runs over every slot of a block
        const int rbff = nrhs <= 8 ? 8 : kRBff;
        const int ns = batch_splits(s, nrhs, rbff, 8);
        {
            PhaseTimer t(s, PM_PHASE_PREP, st);
            k_prep_ff_multi<<<gp, 256, 0, st>>>(sigma, ld_sigma, s->wa, B.sff, N, skip);
        }
        {
            PhaseTimer t(s, kernel_K ? PM_PHASE_DIRECT64_K : PM_PHASE_DIRECT64, st);
            dim3 g(pm_ceil_div(N, kThreads), ns, pm_ceil_div(nrhs, rbff));
            const int chunk = pm_ceil_div(N, ns);
            const float4* srcv = kernel_K ? s->src_kg : s->src_ff;
            auto launch = [&](auto kern) {
                kern<<<g, kThreads, 0, st>>>(srcv, B.sff, nrhs, s->tgt_ff, s->log_tab, N, chunk,
                                             B.part, ns, skip);
            };
            if (rbff == 8)
                kernel_K ? launch(k_direct_multi_ff<true, 8>) : launch(k_direct_multi_ff<false, 8>);
            else
                kernel_K ? launch(k_direct_multi_ff<true, kRBff>)
                         : launch(k_direct_multi_ff<false, kRBff>);
        }
        PhaseTimer t(s, PM_PHASE_NEAR, st);
        dim3 gn(pm_ceil_div((long long)N * 32, 256), nrhs);
        k_near_multi64<<<gn, 256, 0, st>>>(N, s->pp, s->row_ptr, s->blk_patch,
                                           kernel_K ? s->cK64 : s->cR64, sigma, ld_sigma, B.part,
                                           ns, out, ld_out, skip);
    } else {
        const int rb = batch_rb(s);
        const int ns = batch_splits(s, nrhs, rb, batch_bps(s));
        {
            PhaseTimer t(s, PM_PHASE_PREP, st);
            k_prep32_multi<<<gp, 256, 0, st>>>(sigma, ld_sigma, s->wa, B.s32, N, s->pp, s->ppad,
                                               s->npatch, B.sig32, skip);
        }
        {
            PhaseTimer t(s, kernel_K ? PM_PHASE_DIRECT_K : PM_PHASE_DIRECT_R, st);
            dim3 g(pm_ceil_div(N, kThreads), ns, pm_ceil_div(nrhs, rb));
            const int chunk = pm_ceil_div(N, ns);
            auto launch = [&](auto kern) {
                kern<<<g, kThreads, 0, st>>>(s->src32, B.s32, nrhs, s->tgt32, N, chunk, s->eps2,
                                             B.part, ns, skip);
            };
            if (rb == 8)
                kernel_K ? launch(k_direct_multi32<true, 8>) : launch(k_direct_multi32<false, 8>);
            else if (rb == 32)
                kernel_K ? launch(k_direct_multi32<true, 32>) : launch(k_direct_multi32<false, 32>);
            else
                kernel_K ? launch(k_direct_multi32<true, kRB>) : launch(k_direct_multi32<false, kRB>);
        }
        if (!B.patch_tried) PM_TRY(build_patch_unions(s, B));
        PhaseTimer t(s, PM_PHASE_NEAR, st);
        if (B.umax > 0) {
            // 8 right-hand sides per block for batches of at most 8 (four rows per warp)
            const int rp = nrhs <= 8 ? 8 : kPatchRhs;
            const dim3 gn(s->npatch, pm_ceil_div(nrhs, rp));
            const size_t smem = (size_t)B.umax * s->ppad * (rp + 1) * sizeof(float);
            auto launch = [&](auto kern) {
                kern<<<gn, 256, smem, st>>>(N, s->pp, s->ppad, s->npatch, s->row_ptr, B.blk_u,
                                            B.pu_ptr, B.pu_list, kernel_K ? s->cK32 : s->cR32,
                                            B.sig32, B.part, ns, nrhs, out, ld_out, skip);
            };
            if (rp == 8)
                launch(k_near_multi32_patch<8>);
            else
                launch(k_near_multi32_patch<kPatchRhs>);
        } else {
            dim3 gn(pm_ceil_div((long long)N * 32, 256), nrhs);
            k_near_multi32<<<gn, 256, 0, st>>>(N, s->ppad, s->npatch, s->row_ptr, s->blk_patch,
                                               kernel_K ? s->cK32 : s->cR32, B.sig32, B.part, ns,
                                               out, ld_out, skip);
        }
    }
    s->launch_total += 3;
    PM_CUDA_TRY(cudaGetLastError());
    return PM_OK;
}

// ============================================================================ batched solve
namespace {

constexpr int kRed = 256;

__device__ __forceinline__ double warp_sum_d(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// partial[r][blk][j] = sum over the block's rows of A_r,j[i] * b_r[i]
__global__ void __launch_bounds__(kRed)
k_bdots(const double* __restrict__ A, long long col_stride, long long rhs_stride_A, int ncols,
        const double* __restrict__ b, long long rhs_stride_b, int N,
        double* __restrict__ partial, const int* __restrict__ done) {
    const int r = blockIdx.y;
    if (done && done[r]) return;
    __shared__ double sh[32];
    const double* Ar = A + r * rhs_stride_A;
    const double* br = b + r * rhs_stride_b;
    const int stride = gridDim.x * blockDim.x;
    for (int j = 0; j < ncols; ++j) {
        const double* a = Ar + j * col_stride;
        double acc = 0.0;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) acc += a[i] * br[i];
        acc = warp_sum_d(acc);
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        __syncthreads();
        if (lane == 0) sh[wid] = acc;
        __syncthreads();
        if (threadIdx.x < 32) {
            double t = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
            t = warp_sum_d(t);
            if (threadIdx.x == 0) partial[((size_t)r * gridDim.x + blockIdx.x) * ncols + j] = t;
        }
    }
}

__global__ void k_breduce(const double* __restrict__ partial, int nblk, int ncols,
                          double* __restrict__ out, long long ld_out, const int* __restrict__ done) {
    const int r = blockIdx.y;
    if (done && done[r]) return;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ncols) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += partial[((size_t)r * nblk + b) * ncols + j];
    out[r * ld_out + j] = s;
}

// w_r -= sum_j A_r,j c_r[j]
__global__ void k_bsub(const double* __restrict__ A, long long col_stride, long long rhs_stride_A,
                       int ncols, const double* __restrict__ c, long long ldc,
                       double* __restrict__ w, int N, const int* __restrict__ done) {
    const int r = blockIdx.y;
    if (done && done[r]) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double* Ar = A + r * rhs_stride_A;
    const double* cr = c + r * ldc;
    double acc = w[(size_t)r * N + i];
    for (int j = 0; j < ncols; ++j) acc -= Ar[j * col_stride + i] * cr[j];
    w[(size_t)r * N + i] = acc;
}

__global__ void k_badd_cols(double* __restrict__ h, long long ldh, const double* __restrict__ h2,
                            long long ldh2, int n, const int* __restrict__ done) {
    const int r = blockIdx.y;
    if (done && done[r]) return;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) h[r * ldh + j] += h2[r * ldh2 + j];
}

// out_r = v_r + y_r + wdot_r  (A v with the rank-one term)
__global__ void k_bfinishA(const double* __restrict__ v, long long ldv, const double* __restrict__ y,
                           const double* __restrict__ wdot, long long ldw,
                           double* __restrict__ out, int N, const int* __restrict__ done) {
    const int r = blockIdx.y;
    if (done && done[r]) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    out[(size_t)r * N + i] = v[r * ldv + i] + y[(size_t)r * N + i] + wdot[r * ldw];
}

__global__ void k_bscale_copy(const double* __restrict__ src, long long lds,
                              const double* __restrict__ sc, long long ldsc, int invert,
                              double* __restrict__ dst, long long ldd, int N,
                              const int* __restrict__ done) {
    const int r = blockIdx.y;
    if (done && done[r]) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double s = sc[r * ldsc];
    const double f = invert ? (s != 0.0 ? 1.0 / s : 0.0) : s;
    dst[r * ldd + i] = src[r * lds + i] * f;
}

// scal layout per rhs: [0] w.v  [1] norm^2  [2] 1/|w|  [3] beta  [4] tol_abs
__global__ void k_bcycle_start(int nrhs, const double* __restrict__ nrm2, long long ldn,
                               double* __restrict__ g, int m, double* __restrict__ scal,
                               int* __restrict__ done, int* __restrict__ iters,
                               int* __restrict__ all_done) {
    __shared__ int any_active;
    if (threadIdx.x == 0) any_active = 0;
    __syncthreads();
    for (int r = threadIdx.x; r < nrhs; r += blockDim.x) {
        const double beta = sqrt(nrm2[r * ldn]);
        double* gr = g + (size_t)r * (m + 1);
        for (int k = 0; k <= m; ++k) gr[k] = 0.0;
        gr[0] = beta;
        scal[r * 8 + 3] = beta;
        iters[r] = 0;
        const int d = (beta <= scal[r * 8 + 4] || beta == 0.0) ? 1 : 0;
        done[r] = d;
        if (!d) atomicOr(&any_active, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) *all_done = any_active ? 0 : 1;
}

__global__ void k_brotate(int nrhs, double* __restrict__ H, int ldh, int m, int k,
                          double* __restrict__ cs, double* __restrict__ sn, double* __restrict__ g,
                          double* __restrict__ scal, int* __restrict__ done,
                          int* __restrict__ iters, int* __restrict__ all_done) {
    __shared__ int any_active;
    if (threadIdx.x == 0) any_active = 0;
    __syncthreads();
    for (int r = threadIdx.x; r < nrhs; r += blockDim.x) {
        if (done[r]) continue;
        double* h = H + ((size_t)r * m + k) * ldh;
        double* csr = cs + (size_t)r * m;
        double* snr = sn + (size_t)r * m;
        double* gr = g + (size_t)r * (m + 1);
        const double hn = sqrt(scal[r * 8 + 1]);
        h[k + 1] = hn;
        scal[r * 8 + 2] = (hn > 0.0) ? 1.0 / hn : 0.0;
        for (int j = 0; j < k; ++j) {
            const double t = csr[j] * h[j] + snr[j] * h[j + 1];
            h[j + 1] = -snr[j] * h[j] + csr[j] * h[j + 1];
            h[j] = t;
        }
        const double a = h[k], b = h[k + 1];
        const double den = hypot(a, b);
        const double c = (den > 0.0) ? a / den : 1.0, s_ = (den > 0.0) ? b / den : 0.0;
        csr[k] = c;
        snr[k] = s_;
        h[k] = den;
        h[k + 1] = 0.0;
        gr[k + 1] = -s_ * gr[k];
        gr[k] = c * gr[k];
        iters[r] = k + 1;
        const int d = (fabs(gr[k + 1]) <= scal[r * 8 + 4] || hn <= 1e-300 || !(hn == hn)) ? 1 : 0;
        done[r] = d;
        if (!d) atomicOr(&any_active, 1);
    }
    __syncthreads();
    if (threadIdx.x == 0) *all_done = any_active ? 0 : 1;
}

// per right-hand side: y = H^{-1} g by back substitution and ynorm = |y|_2 (the
// norm of the cycle's correction V y, V orthonormal)
__global__ void k_bbacksolve(int nrhs, const double* __restrict__ H, int ldh, int m,
                             const double* __restrict__ g, const int* __restrict__ iters,
                             double* __restrict__ y, double* __restrict__ ynorm) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrhs) return;
    const int n = iters[r];
    const double* Hr = H + (size_t)r * m * ldh;
    const double* gr = g + (size_t)r * (m + 1);
    double* yr = y + (size_t)r * m;
    double s2 = 0.0;
    for (int i = n - 1; i >= 0; --i) {
        double t = gr[i];
        for (int j = i + 1; j < n; ++j) t -= Hr[(size_t)j * ldh + i] * yr[j];
        const double d = Hr[(size_t)i * ldh + i];
        yr[i] = (d != 0.0) ? t / d : 0.0;
        s2 += yr[i] * yr[i];
    }
    ynorm[r] = sqrt(s2);
}

__global__ void k_badd_combo(const double* __restrict__ V, long long col_stride,
                             long long rhs_stride, const int* __restrict__ iters,
                             const double* __restrict__ y, int m, double* __restrict__ x, int N) {
    const int r = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int n = iters[r];
    const double* Vr = V + r * rhs_stride;
    double acc = x[(size_t)r * N + i];
    for (int j = 0; j < n; ++j) acc += Vr[j * col_stride + i] * y[(size_t)r * m + j];
    x[(size_t)r * N + i] = acc;
}

__global__ void k_bresidual(const double* __restrict__ b, const double* __restrict__ Ax,
                            double* __restrict__ out, int N) {
    const int r = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) out[(size_t)r * N + i] = b[(size_t)r * N + i] - Ax[(size_t)r * N + i];
}

// y -= x (every right-hand side)
__global__ void k_bsubv(double* __restrict__ y, const double* __restrict__ x, int N) {
    const int r = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) y[(size_t)r * N + i] -= x[(size_t)r * N + i];
}

__global__ void k_baxpy(double* __restrict__ y, const double* __restrict__ x, int N) {
    const int r = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) y[(size_t)r * N + i] += x[(size_t)r * N + i];
}

__global__ void k_bshift(double* __restrict__ y, const double* __restrict__ shift, long long lds,
                         double sgn, int N) {
    const int r = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) y[(size_t)r * N + i] += sgn * shift[r * lds];
}

__global__ void k_bmul(const double* __restrict__ w, const double* __restrict__ f,
                       double* __restrict__ out, int N) {
    const int r = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) out[(size_t)r * N + i] = w[i] * f[(size_t)r * N + i];
}

}  // namespace

struct PmBatchSolveWork {
    int nrhs = 0, m = 0, N = 0, nred = 0;
    double *V = nullptr, *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr, *y = nullptr;
    double *part = nullptr, *scal = nullptr, *hcol = nullptr, *dots = nullptr;
    double *w = nullptr, *tmp = nullptr, *r = nullptr, *res = nullptr, *delta = nullptr;
    double *sig = nullptr, *f = nullptr, *u = nullptr;
    int *done = nullptr, *iters = nullptr, *all_done = nullptr;
    double* ynorm = nullptr;          // [nrhs] |y| of the last cycle
    double* pinned = nullptr;
    double* pinned_y = nullptr;       // [nrhs] host copy of ynorm
    int* pinned_i = nullptr;
};

static void bsolve_release(PmBatchSolveWork& W) {
    pm_dfree(W.V); pm_dfree(W.H); pm_dfree(W.cs); pm_dfree(W.sn); pm_dfree(W.g); pm_dfree(W.y);
    pm_dfree(W.part); pm_dfree(W.scal); pm_dfree(W.hcol); pm_dfree(W.dots); pm_dfree(W.w);
    pm_dfree(W.tmp); pm_dfree(W.r); pm_dfree(W.res); pm_dfree(W.delta); pm_dfree(W.sig);
    pm_dfree(W.f); pm_dfree(W.u); pm_dfree(W.done); pm_dfree(W.iters); pm_dfree(W.all_done);
    pm_dfree(W.ynorm);
    if (W.pinned_y) cudaFreeHost(W.pinned_y);
    if (W.pinned) cudaFreeHost(W.pinned);
    if (W.pinned_i) cudaFreeHost(W.pinned_i);
    W.pinned_y = W.pinned = nullptr;
    W.pinned_i = nullptr;
}

void pm_batch_solve_free(pm_surface* s) {
    if (!s->bsolve) return;
    bsolve_release(*s->bsolve);
    delete s->bsolve;
    s->bsolve = nullptr;
}

// buffers of a lockstep solve of nrhs columns of length N (restart m)
static pm_status bsolve_alloc(PmBatchSolveWork& W, int nrhs, int m, int N) {
    W.nrhs = nrhs;
    W.m = m;
    W.N = N;
    W.nred = std::max(1, std::min(pm_ceil_div(N, 2048), 64));
    const size_t RN = (size_t)nrhs * N;
    PM_TRY(pm_dmalloc(&W.V, (size_t)nrhs * (m + 1) * N));
    PM_TRY(pm_dmalloc(&W.H, (size_t)nrhs * m * (m + 2)));
    PM_TRY(pm_dmalloc(&W.cs, (size_t)nrhs * m));
    PM_TRY(pm_dmalloc(&W.sn, (size_t)nrhs * m));
    PM_TRY(pm_dmalloc(&W.g, (size_t)nrhs * (m + 1)));
    PM_TRY(pm_dmalloc(&W.y, (size_t)nrhs * m));
    PM_TRY(pm_dmalloc(&W.part, (size_t)nrhs * W.nred * (m + 2)));
    PM_TRY(pm_dmalloc(&W.scal, (size_t)nrhs * 8));
    PM_TRY(pm_dmalloc(&W.hcol, (size_t)nrhs * (m + 2)));
    PM_TRY(pm_dmalloc(&W.dots, (size_t)nrhs * 8));
    PM_TRY(pm_dmalloc(&W.w, RN));
    PM_TRY(pm_dmalloc(&W.tmp, RN));
    PM_TRY(pm_dmalloc(&W.r, RN));
    PM_TRY(pm_dmalloc(&W.res, RN));
    PM_TRY(pm_dmalloc(&W.delta, RN));
    PM_TRY(pm_dmalloc(&W.sig, RN));
    PM_TRY(pm_dmalloc(&W.f, RN));
    PM_TRY(pm_dmalloc(&W.u, RN));
    PM_TRY(pm_dmalloc(&W.done, nrhs));
    PM_TRY(pm_dmalloc(&W.iters, nrhs));
    PM_TRY(pm_dmalloc(&W.all_done, 1));
    PM_TRY(pm_dmalloc(&W.ynorm, nrhs));
    PM_CUDA_TRY(cudaMallocHost((void**)&W.pinned_y, sizeof(double) * (size_t)nrhs));
    PM_CUDA_TRY(cudaMallocHost((void**)&W.pinned, sizeof(double) * 8 * (size_t)nrhs));
    PM_CUDA_TRY(cudaMallocHost((void**)&W.pinned_i, sizeof(int) * (2 * (size_t)nrhs + 4)));
    return PM_OK;
}

static pm_status bsolve_work(pm_surface* s, int nrhs, PmBatchSolveWork** out) {
    const int m = std::max(2, std::min(s->opts.gmres_restart, 400));
    if (s->bsolve && s->bsolve->nrhs >= nrhs && s->bsolve->m == m) {
        *out = s->bsolve;
        return PM_OK;
    }
    pm_batch_solve_free(s);
    s->bsolve = new PmBatchSolveWork();
    PM_TRY(bsolve_alloc(*s->bsolve, nrhs, m, s->N));
    *out = s->bsolve;
    return PM_OK;
}

namespace {

struct BSolver {
    pm_surface* s;
    PmBatchSolveWork& W;
    int nrhs;
    cudaStream_t st;
    int grid_n;
    pm_precision op = PM_PREC_FF;   // the solve's operator precision

    // precision of true residuals and of the representation (see pm_solve.cu)
    pm_precision residual_prec() const {
        if (s->opts.residual_prec == PM_PREC_FP64) return PM_PREC_FP64;
        if (s->opts.residual_prec == PM_PREC_FP32 && (op == PM_PREC_FP32 || op == PM_PREC_FMM))
            return op;
        return PM_PREC_FF;
    }

    // dst[r*lddst + j] = A_r,j . b_r for j < ncols
    void dots(const double* A, long long col_stride, long long rhs_stride_A, int ncols,
              const double* b, long long rhs_stride_b, double* dst, long long lddst,
              const int* done) {
        k_bdots<<<dim3(W.nred, nrhs), kRed, 0, st>>>(A, col_stride, rhs_stride_A, ncols, b,
                                                      rhs_stride_b, W.N, W.part, done);
        k_breduce<<<dim3(pm_ceil_div(ncols, 64), nrhs), 64, 0, st>>>(W.part, W.nred, ncols, dst,
                                                                       lddst, done);
        s->launch_total += 2;
    }

    // out_r = A v_r (I + R~ + 1 w^T) for all r
    pm_status apply_A(const double* v, long long ldv, double* out, pm_precision prec,
                      const int* done) {
        if (prec == PM_PREC_FP64 || prec == PM_PREC_FMM) {
            // no multi-RHS form: one apply per right-hand side
            for (int r = 0; r < nrhs; ++r)
                PM_TRY(pm_apply_dev(s, 0, 1, 1, v + r * ldv, W.tmp + (size_t)r * W.N, prec, st));
        } else {
            PM_TRY(pm_apply_batch(s, 0, v, ldv, W.tmp, W.N, nrhs, prec, st));
        }
        dots(s->w, 0, 0, 1, v, ldv, W.dots + 0, 8, done);
        k_bfinishA<<<dim3(grid_n, nrhs), 256, 0, st>>>(v, ldv, W.tmp, W.dots + 0, 8, out, W.N, done);
        s->launch_total += 1;
        PM_CUDA_TRY(cudaGetLastError());
        return PM_OK;
    }

    pm_status norms(const double* v, double* host) {   // host[r] = ||v_r||_2
        dots(v, 0, W.N, 1, v, W.N, W.dots + 1, 8, nullptr);
        PM_CUDA_TRY(cudaMemcpyAsync(W.pinned, W.dots, sizeof(double) * 8 * nrhs,
                                    cudaMemcpyDeviceToHost, st));
        PM_CUDA_TRY(cudaStreamSynchronize(st));
        for (int r = 0; r < nrhs; ++r) host[r] = std::sqrt(W.pinned[8 * r + 1]);
        return PM_OK;
    }

    // lockstep restarted GMRES on A d_r = b_r from d = 0 (operator in prec); x += d.
    // dnorm (optional): per right-hand side, bound on |x_new - x_old| (sum of the cycles' |y|)
    pm_status gmres(const double* b, double* x, pm_precision prec, const std::vector<double>& tol_abs,
                    int max_iter, int* iters_used, std::vector<double>* dnorm = nullptr) {
        if (dnorm) dnorm->assign(nrhs, 0.0);
        const int m = W.m, N = W.N;
        const long long ldV = (long long)(m + 1) * N;
        const int ldh = m + 2;
        PM_CUDA_TRY(cudaMemcpyAsync(W.r, b, sizeof(double) * nrhs * N, cudaMemcpyDeviceToDevice, st));
        PM_CUDA_TRY(cudaMemsetAsync(W.delta, 0, sizeof(double) * nrhs * N, st));
        for (int r = 0; r < nrhs; ++r) W.pinned[8 * r + 4] = tol_abs[r];
        // tolerance into scal[r][4]
        for (int r = 0; r < nrhs; ++r)
            PM_CUDA_TRY(cudaMemcpyAsync(W.scal + 8 * r + 4, W.pinned + 8 * r + 4, sizeof(double),
                                        cudaMemcpyHostToDevice, st));
        int total = 0;
        while (total < max_iter) {
            dots(W.r, 0, N, 1, W.r, N, W.scal + 1, 8, nullptr);
            k_bcycle_start<<<1, 256, 0, st>>>(nrhs, W.scal + 1, 8, W.g, m, W.scal, W.done, W.iters,
                                              W.all_done);
            k_bscale_copy<<<dim3(grid_n, nrhs), 256, 0, st>>>(W.r, N, W.scal + 3, 8, 1, W.V, ldV, N,
                                                              W.done);
            s->launch_total += 2;
            const int steps = std::min(m, max_iter - total);
            s->skip_flag = W.all_done;
            const int chunk = (steps <= 8) ? steps : 4;
            for (int k = 0; k < steps; ++k) {
                if (k > 0 && k % chunk == 0) {
                    PM_CUDA_TRY(cudaMemcpyAsync(W.pinned_i, W.all_done, sizeof(int),
                                                cudaMemcpyDeviceToHost, st));
                    PM_CUDA_TRY(cudaStreamSynchronize(st));
                    if (W.pinned_i[0]) break;
                }
                double* vk = W.V + (size_t)k * N;         // column k of rhs 0; rhs stride ldV
                double* vk1 = W.V + (size_t)(k + 1) * N;
                double* hk = W.H + (size_t)k * ldh;         // rhs stride m*ldh
                pm_status stt = apply_A(vk, ldV, W.w, prec, W.done);
                if (stt != PM_OK) { s->skip_flag = nullptr; return stt; }
                dots(W.V, N, ldV, k + 1, W.w, N, hk, (long long)m * ldh, W.done);
                k_bsub<<<dim3(grid_n, nrhs), 256, 0, st>>>(W.V, N, ldV, k + 1, hk, (long long)m * ldh,
                                                           W.w, N, W.done);
                dots(W.V, N, ldV, k + 1, W.w, N, W.hcol, m + 2, W.done);
                k_bsub<<<dim3(grid_n, nrhs), 256, 0, st>>>(W.V, N, ldV, k + 1, W.hcol, m + 2, W.w, N,
                                                           W.done);
                k_badd_cols<<<dim3(pm_ceil_div(k + 1, 64), nrhs), 64, 0, st>>>(
                    hk, (long long)m * ldh, W.hcol, m + 2, k + 1, W.done);
                dots(W.w, 0, N, 1, W.w, N, W.scal + 1, 8, W.done);
                k_brotate<<<1, 256, 0, st>>>(nrhs, W.H, ldh, m, k, W.cs, W.sn, W.g, W.scal, W.done,
                                             W.iters, W.all_done);
                k_bscale_copy<<<dim3(grid_n, nrhs), 256, 0, st>>>(W.w, N, W.scal + 2, 8, 0, vk1, ldV,
                                                                  N, W.done);
                s->launch_total += 5;
            }
            s->skip_flag = nullptr;
            k_bbacksolve<<<pm_ceil_div(nrhs, 64), 64, 0, st>>>(nrhs, W.H, ldh, m, W.g, W.iters, W.y,
                                                                W.ynorm);
            k_badd_combo<<<dim3(grid_n, nrhs), 256, 0, st>>>(W.V, N, ldV, W.iters, W.y, m, W.delta, N);
            s->launch_total += 2;
            PM_CUDA_TRY(cudaMemcpyAsync(W.pinned_i, W.iters, sizeof(int) * nrhs,
                                        cudaMemcpyDeviceToHost, st));
            PM_CUDA_TRY(cudaMemcpyAsync(W.pinned_i + nrhs, W.done, sizeof(int) * nrhs,
                                        cudaMemcpyDeviceToHost, st));
            PM_CUDA_TRY(cudaMemcpyAsync(W.pinned_y, W.ynorm, sizeof(double) * nrhs,
                                        cudaMemcpyDeviceToHost, st));
            PM_CUDA_TRY(cudaStreamSynchronize(st));
            int it = 0, all = 1;
            for (int r = 0; r < nrhs; ++r) {
                it = std::max(it, W.pinned_i[r]);
                all &= W.pinned_i[nrhs + r];
                if (dnorm && W.pinned_i[r] > 0) (*dnorm)[r] += W.pinned_y[r];
            }
            total += it;
            if (all || it == 0) break;
            PM_TRY(apply_A(W.delta, N, W.w, prec, nullptr));
            k_bresidual<<<dim3(grid_n, nrhs), 256, 0, st>>>(b, W.w, W.r, N);
            s->launch_total += 1;
        }
        k_baxpy<<<dim3(grid_n, nrhs), 256, 0, st>>>(x, W.delta, N);
        s->launch_total += 1;
        PM_CUDA_TRY(cudaGetLastError());
        *iters_used = total;
        return PM_OK;
    }

    pm_status true_residual(const double* f, const double* sig, double* res) {
        PM_TRY(apply_A(sig, W.N, W.w, residual_prec(), nullptr));
        k_bresidual<<<dim3(grid_n, nrhs), 256, 0, st>>>(f, W.w, res, W.N);
        s->launch_total += 1;
        return PM_OK;
    }
};

}  // namespace

// Batched solve of nrhs right-hand sides (same surface and coefficient), in lockstep.
// Device bytes a batched solve of nrhs right-hand sides would allocate on top of
// the surface's current batched buffers (bsolve_work and batch_ensure above).
size_t pm_batch_need_bytes(const pm_surface* s, int nrhs) {
    const size_t m = (size_t)std::max(2, std::min(s->opts.gmres_restart, 400));
    const size_t N = (size_t)s->N, R = (size_t)nrhs;
    size_t need = 0;
    if (!(s->bsolve && (size_t)s->bsolve->nrhs >= R && (size_t)s->bsolve->m == m)) {
        const size_t nred = (size_t)std::max(1, std::min(pm_ceil_div(s->N, 2048), 64));
        need += sizeof(double) * (R * (m + 1) * N + R * (m * (m + 2) + 3 * m + 1) +
                                  R * nred * (m + 2) + R * (m + 2 + 16) + 8 * R * N) +
                sizeof(int) * (2 * R + 1);
    }
    if (!(s->batch && s->batch->cap >= nrhs))
        need += R * N * (sizeof(float) + sizeof(float2) + 8 * sizeof(float2)) +
                R * (size_t)s->npatch * s->ppad * sizeof(float);
    return need;
}

pm_status pm_solve_batch(pm_surface* s, const double* f, double* u, int nrhs, double tol,
                         int maxit, pm_precision prec, unsigned flags, double* sigma_out,
                         pm_solve_info* info, cudaStream_t st) {
    const auto t0 = std::chrono::steady_clock::now();
    PmBatchSolveWork* Wp = nullptr;
    PM_TRY(bsolve_work(s, nrhs, &Wp));
    PmBatchSolveWork& W = *Wp;
    const int N = s->N;
    BSolver S{s, W, nrhs, st, pm_ceil_div(N, 256)};
    S.op = prec;
    const bool dev = (flags & PM_SOLVE_DEVICE_PTRS) != 0;
    PM_CUDA_TRY(cudaMemcpyAsync(W.f, f, sizeof(double) * (size_t)nrhs * N,
                                dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    double sw = 0.0;
    for (double v : s->h_w) sw += v;
    // weighted means and norms of every f_r (Thm. LBsolvable)
    k_bmul<<<dim3(S.grid_n, nrhs), 256, 0, st>>>(s->w, W.f, W.tmp, N);
    S.dots(W.tmp, 0, N, 1, W.f, N, W.dots + 5, 8, nullptr);      // sum w f^2
    S.dots(s->w, 0, 0, 1, W.f, N, W.dots + 4, 8, nullptr);       // sum w f
    PM_CUDA_TRY(cudaMemcpyAsync(W.pinned, W.dots, sizeof(double) * 8 * nrhs,
                                cudaMemcpyDeviceToHost, st));
    PM_CUDA_TRY(cudaStreamSynchronize(st));
    std::vector<double> removed(nrhs, 0.0), fnorm(nrhs, 0.0);
    for (int r = 0; r < nrhs; ++r) {
        const double wf = W.pinned[8 * r + 4], wff = W.pinned[8 * r + 5];
        if (wff > 0.0 && std::fabs(wf) > s->opts.mean_tol * std::sqrt(sw * wff) &&
            !(flags & PM_SOLVE_PROJECT_RHS)) {
            pm_set_error("pm_solve: right-hand side %d has weighted mean %.3e; pass "
                         "PM_SOLVE_PROJECT_RHS to subtract it", r, wf / sw);
            return PM_ERR_RHS_NOT_MEAN_ZERO;
        }
        if (flags & PM_SOLVE_PROJECT_RHS) removed[r] = wf / sw;
    }
    if (flags & PM_SOLVE_PROJECT_RHS) {
        k_bshift<<<dim3(S.grid_n, nrhs), 256, 0, st>>>(W.f, W.dots + 4, 8, -1.0 / sw, N);
        s->launch_total += 1;
    }
    PM_TRY(S.norms(W.f, fnorm.data()));
    PM_CUDA_TRY(cudaMemsetAsync(W.sig, 0, sizeof(double) * (size_t)nrhs * N, st));
    int iters = 0, refinements = 0, updated = 0;
    std::vector<double> relres(nrhs, 0.0);
    const bool accurate_inner = (prec == PM_PREC_FP64 || prec == PM_PREC_FF);
    std::vector<double> tabs(nrhs), dn;
    bool have_update = false;
    for (;;) {
        std::vector<double> rn(nrhs);
        // after a correction d: r - A32 d is the true residual to within 0.1 tol |f_r|
        // when kOpRelErr |d_r| <= 0.1 tol |f_r| for every right-hand side (pm_solve.cu)
        bool small = have_update && s->opts.residual_update && !accurate_inner;
        for (int r = 0; small && r < nrhs; ++r) small = kOpRelErr * dn[r] <= 0.1 * tol * fnorm[r];
        if (refinements == 0) {
            PM_CUDA_TRY(cudaMemcpyAsync(W.res, W.f, sizeof(double) * (size_t)nrhs * N,
                                        cudaMemcpyDeviceToDevice, st));
            rn = fnorm;
        } else if (small) {
            PM_TRY(S.apply_A(W.delta, N, W.w, prec, nullptr));
            k_bsubv<<<dim3(S.grid_n, nrhs), 256, 0, st>>>(W.res, W.w, N);
            s->launch_total += 1;
            PM_TRY(S.norms(W.res, rn.data()));
            ++updated;
        } else {
            PM_TRY(S.true_residual(W.f, W.sig, W.res));
            PM_TRY(S.norms(W.res, rn.data()));
        }
        bool all_ok = true;
        for (int r = 0; r < nrhs; ++r) {
            relres[r] = fnorm[r] > 0 ? rn[r] / fnorm[r] : 0.0;
            all_ok &= relres[r] <= tol;
        }
        if (all_ok || refinements >= (accurate_inner ? 2 : s->opts.max_refine) || iters >= maxit)
            break;
        for (int r = 0; r < nrhs; ++r) {
            const double inner = accurate_inner ? 0.5 * tol * fnorm[r] / std::max(rn[r], 1e-300)
                                                : std::max(s->opts.inner_tol,
                                                           0.5 * tol * fnorm[r] / std::max(rn[r], 1e-300));
            tabs[r] = (relres[r] <= tol) ? 1e300 : inner * rn[r];
        }
        int it = 0;
        PM_TRY(S.gmres(W.res, W.sig, prec, tabs, maxit - iters, &it, &dn));
        have_update = true;
        iters += it;
        ++refinements;
        if (it == 0) break;
    }
    pm_status result = PM_OK;
    for (int r = 0; r < nrhs; ++r)
        if (!(relres[r] <= tol)) {
            pm_set_error("pm_solve: right-hand side %d: relative residual %.3e above %.3e", r,
                         relres[r], tol);
            result = PM_ERR_NOT_CONVERGED;
        }
    // u = K~ sigma (accurate), minus its weighted mean
    const pm_precision rp = S.residual_prec();
    if (rp == PM_PREC_FP64 || rp == PM_PREC_FMM) {
        for (int r = 0; r < nrhs; ++r)
            PM_TRY(pm_apply_dev(s, 1, 1, 1, W.sig + (size_t)r * N, W.u + (size_t)r * N, rp, st));
    } else {
        PM_TRY(pm_apply_batch(s, 1, W.sig, N, W.u, N, nrhs, rp, st));
    }
    S.dots(s->w, 0, 0, 1, W.u, N, W.dots + 6, 8, nullptr);
    k_bshift<<<dim3(S.grid_n, nrhs), 256, 0, st>>>(W.u, W.dots + 6, 8, -1.0 / sw, N);
    s->launch_total += 1;
    const cudaMemcpyKind d2h = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    PM_CUDA_TRY(cudaMemcpyAsync(u, W.u, sizeof(double) * (size_t)nrhs * N, d2h, st));
    if (sigma_out)
        PM_CUDA_TRY(cudaMemcpyAsync(sigma_out, W.sig, sizeof(double) * (size_t)nrhs * N, d2h, st));
    PM_CUDA_TRY(cudaStreamSynchronize(st));
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (info)
        for (int r = 0; r < nrhs; ++r) {
            info[r].iterations = iters;
            info[r].refinements = refinements;
            info[r].residual = relres[r];
            info[r].removed_mean = removed[r];
            info[r].seconds = secs;
            info[r].residual_updates = updated;
        }
    return result;
}

// ============================================================================ multi-instance solve
// One lockstep GMRES over the right-hand sides of several operators ("instances",
// surfaces of any size and coefficient).  Column c = (instance k, right-hand side
// r) of every vector has the stride Nmax of the largest instance; rows N_k..Nmax
// of a column are zero and stay zero (the applies write rows < N_k only, and every
// vector kernel maps zeros to zeros), so the batched vector kernels above serve
// instances of uneven size unchanged.  Each Arnoldi step's operator apply is
// three launches for all instances together: the prep of every column, ONE
// persistent launch of the float32 smooth sums over a device work list of
// (instance, 128-target tile, group of RB right-hand sides, source chunk) items,
// and one launch of the near-field corrections with the split reduction (a warp
// per (instance, right-hand side, row)).  A whole GMRES cycle -- every Arnoldi
// step, the Givens updates and the correction -- is one CUDA graph, captured once
// per cycle length and replayed (finished columns skip their work through the
// done flags, a finished batch every launch through all_done).
namespace {

constexpr int kMultiGroupMax = 64;   // instances per geometry in one multi-instance solve

struct MInst {
    const float4* pos;         // float32 source positions of the instance (src32)
    const float4* tgt;         // float32 target factors [3 N] (tgt32)
    const double* wa;          // w / a
    const int* row_ptr;        // near-field CSR
    const int* blk_patch;
    const float* vals;         // float32 remainder corrections (cR32)
    const int* nu_ptr;         // per patch, the union of its rows' near patches
    const int* nu_list;
    const int* nu_blk;         // per correction block, its index in that union
    const float4* fac;         // [N] (grad a/(2 pi), a/pi): remainder factors (k_mfactors)
    const float* facB;         // [N] -a H/pi
    float* s32;                // [nrhs][N] strengths
    float* sig32;              // [nrhs][npatch][ppad] sigma by patch
    float2* part;              // [nrhs][nsplit][N] partial sums
    float eps2;
    int N, npatch, pp, ppad, nrhs, col0, nsplit, chunk;
    long long warp0;           // first near-field warp (instance-major, rhs, row)
};

__global__ void k_mprep32(const double* __restrict__ sigma, long long ld_sigma,
                          const MInst* __restrict__ I, const int* __restrict__ col_inst,
                          const int* __restrict__ skip) {
    if (skip && *skip) return;
    const int c = blockIdx.y;
    const MInst& in = I[col_inst[c]];
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= in.N) return;
    const int r = c - in.col0;
    const double v = sigma[c * ld_sigma + j];
    in.s32[(size_t)r * in.N + j] = (float)(in.wa[j] * v);
    const int P = j / in.pp;
    in.sig32[((size_t)r * in.npatch + P) * in.ppad + (j - P * in.pp)] = (float)v;
}

// Per-instance remainder factors for the shared-geometry sums: with the unit
// normal n and r = x_i - x_j, the remainder pair factor of eq. explicit_remainder
// (c = 0) is  inv (A (n.r)^2 inv + B (n.r) + g.r),  inv = 1/|r|^2, A = a_i/pi,
// B = -a_i H_i/pi, g = grad a_i/(2 pi): only A, B, g depend on the coefficient.
// fac[i] = (g, A), facB[i] = B; nrm[i] = n (float32).
__global__ void k_mfactors(const double* __restrict__ a, const double* __restrict__ H,
                           const double* __restrict__ g, const double* __restrict__ n, int N,
                           float4* __restrict__ fac, float* __restrict__ facB,
                           float4* __restrict__ nrm) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double c2 = 0.5 / M_PI;
    fac[i] = make_float4((float)(c2 * g[3 * i]), (float)(c2 * g[3 * i + 1]),
                         (float)(c2 * g[3 * i + 2]), (float)(a[i] / M_PI));
    facB[i] = (float)(-a[i] * H[i] / M_PI);
    if (nrm) nrm[i] = make_float4((float)n[3 * i], (float)n[3 * i + 1], (float)n[3 * i + 2], 0.f);
}

struct MGroup {                // instances on one geometry (a surface and its clones)
    const float4* pos;         // source positions (float32)
    const float4* tgt;         // target positions [N] (float32)
    const float4* nrm;         // unit normals [N]
    int N, nsplit, chunk, ninst;
    int inst[kMultiGroupMax];  // instance indices, in column order
    float eps2;
};

// persistent float32 remainder sums sharing each pair's geometry across the
// coefficient fields of a geometry: block b takes items b, b + gridDim.x, ...;
// item = (group, target tile, source chunk, block of FB fields x RB right-hand sides).
// Per pair: r, 1/r^2, n.r and (n.r)^2 / r^2 once; per field A, B, g; per right-hand
// side one FMA.
template <int FB, int RB>
__global__ void __launch_bounds__(kThreads)
k_mgeo32(const MGroup* __restrict__ G, const MInst* __restrict__ I,
         const int4* __restrict__ items, int nitems, const int* __restrict__ skip) {
    if (skip && *skip) return;
    static_assert(RB % 4 == 0 && RB >= 4, "RB right-hand sides in float4 groups");
    constexpr int kSt = (FB * RB <= 16) ? kStage : kStage / 2;
    __shared__ float4 sP[kSt];
    __shared__ float4 sS[kSt][FB * RB / 4];
    const int tid = threadIdx.x;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int4 w = items[it];          // (group, tile, split, field block * 4096 + rhs block)
        const MGroup& gr = G[w.x];
        const int N = gr.N;
        const int i = w.y * kThreads + tid;
        const int f0 = (w.w >> 12) * FB, r0 = (w.w & 4095) * RB;
        const int nf = min(FB, gr.ninst - f0);
        int nrr[FB];
        float A[FB], B[FB], gx[FB], gy[FB], gz[FB];
        float tx = 0, ty = 0, tz = 0, nx = 0, ny = 0, nz = 0;
        if (i < N) {
            const float4 a = gr.tgt[i], b = gr.nrm[i];
            tx = a.x; ty = a.y; tz = a.z;
            nx = b.x; ny = b.y; nz = b.z;
        }
#pragma unroll
        for (int f = 0; f < FB; ++f) {
            nrr[f] = 0;
            A[f] = B[f] = gx[f] = gy[f] = gz[f] = 0.f;
            if (f < nf) {
                const int k = gr.inst[f0 + f];
                nrr[f] = max(0, min(RB, I[k].nrhs - r0));
                if (i < N) {
                    const float4 q = I[k].fac[i];                 // (g, A) of field k
                    gx[f] = q.x; gy[f] = q.y; gz[f] = q.z; A[f] = q.w;
                    B[f] = I[k].facB[i];
                }
            }
        }
        float hi[FB * RB], lo[FB * RB];
#pragma unroll
        for (int q = 0; q < FB * RB; ++q) hi[q] = lo[q] = 0.f;
        const int s0 = w.z * gr.chunk;
        const int s1 = min(s0 + gr.chunk, N);
        for (int base = s0; base < s1; base += kSt) {
            const int len = min(kSt, s1 - base);
            __syncthreads();
            for (int j = tid; j < len; j += kThreads) {
                sP[j] = gr.pos[base + j];
#pragma unroll
                for (int f = 0; f < FB; ++f) {
                    float v[RB];
                    const float* sf = (f < nf) ? I[gr.inst[f0 + f]].s32 : nullptr;
#pragma unroll
                    for (int q = 0; q < RB; ++q)
                        v[q] = (q < nrr[f]) ? sf[(size_t)(r0 + q) * N + base + j] : 0.f;
#pragma unroll
                    for (int q = 0; q < RB / 4; ++q)
                        sS[j][f * (RB / 4) + q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                }
            }
            __syncthreads();
            for (int j0 = 0; j0 < len; j0 += kTile) {
                const int j1 = min(j0 + kTile, len);
                float part[FB * RB];
#pragma unroll
                for (int q = 0; q < FB * RB; ++q) part[q] = 0.f;
#pragma unroll 2
                for (int j = j0; j < j1; ++j) {
                    const float4 p = sP[j];
                    const float dx = tx - p.x, dy = ty - p.y, dz = tz - p.z;
                    const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, gr.eps2)));
                    const float inv = rcp_approx(r2);
                    const float nr = fmaf(nx, dx, fmaf(ny, dy, nz * dz));
                    const float t1 = nr * nr * inv;
#pragma unroll
                    for (int f = 0; f < FB; ++f) {
                        if (f >= nf) break;
                        const float gr_ = fmaf(gx[f], dx, fmaf(gy[f], dy, gz[f] * dz));
                        const float gfac = inv * fmaf(A[f], t1, fmaf(B[f], nr, gr_));
#pragma unroll
                        for (int q = 0; q < RB / 4; ++q) {
                            const float4 sv = sS[j][f * (RB / 4) + q];
                            float* pq = part + f * RB + 4 * q;
                            pq[0] = fmaf(sv.x, gfac, pq[0]);
                            pq[1] = fmaf(sv.y, gfac, pq[1]);
                            pq[2] = fmaf(sv.z, gfac, pq[2]);
                            pq[3] = fmaf(sv.w, gfac, pq[3]);
                        }
                    }
                }
#pragma unroll
                for (int q = 0; q < FB * RB; ++q) two_sum_acc(hi[q], lo[q], part[q]);
            }
        }
        if (i < N) {
#pragma unroll
            for (int f = 0; f < FB; ++f) {
                if (f >= nf) break;
                const MInst& in = I[gr.inst[f0 + f]];
#pragma unroll
                for (int q = 0; q < RB; ++q)
                    if (q < nrr[f])
                        in.part[((size_t)(r0 + q) * in.nsplit + w.z) * N + i] =
                            make_float2(hi[f * RB + q], lo[f * RB + q]);
            }
        }
        __syncthreads();                 // the next item restages the shared arrays
    }
}

// out[(col0 + r) * ld_out + i] = sum_s part[r][s][i] + near corrections; a warp per
// (instance, rhs, row), the instance found by bisection on warp0
__global__ void __launch_bounds__(256)
k_mnear32(const MInst* __restrict__ I, int ninst, long long nwarps, double* __restrict__ out,
          long long ld_out, const int* __restrict__ skip) {
    if (skip && *skip) return;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (warp >= nwarps) return;
    int lo_k = 0, hi_k = ninst - 1;
    while (lo_k < hi_k) {
        const int mid = (lo_k + hi_k + 1) >> 1;
        if (I[mid].warp0 <= warp) lo_k = mid; else hi_k = mid - 1;
    }
    const MInst& in = I[lo_k];
    const long long local = warp - in.warp0;
    const int r = (int)(local / in.N), i = (int)(local - (long long)r * in.N);
    float hi = 0.f, lo = 0.f;
    for (int sp = lane; sp < in.nsplit; sp += 32) {
        const float2 v = in.part[((size_t)r * in.nsplit + sp) * in.N + i];
        two_sum_acc(hi, lo, v.x);
        lo += v.y;
    }
    const int q4 = in.ppad >> 2;
    const int rb = in.row_ptr[i];
    const int total = (in.row_ptr[i + 1] - rb) * q4;
    const float4* v4 = reinterpret_cast<const float4*>(in.vals) + (size_t)rb * q4;
    const float4* s4 = reinterpret_cast<const float4*>(in.sig32 + (size_t)r * in.npatch * in.ppad);
    float acc = 0.f;
    for (int e = lane; e < total; e += 32) {
        const int b = e / q4;
        const float4 v = __ldg(v4 + e);
        const float4 x = __ldg(s4 + (size_t)in.blk_patch[rb + b] * q4 + (e - b * q4));
        acc = fmaf(v.x, x.x, fmaf(v.y, x.y, fmaf(v.z, x.z, fmaf(v.w, x.w, acc))));
    }
    two_sum_acc(hi, lo, acc);
    for (int o = 16; o > 0; o >>= 1) {
        const float h2 = __shfl_down_sync(0xffffffffu, hi, o);
        const float l2 = __shfl_down_sync(0xffffffffu, lo, o);
        two_sum_acc(hi, lo, h2);
        lo += l2;
    }
    if (lane == 0) out[(size_t)(in.col0 + r) * ld_out + i] = (double)hi + (double)lo;
}

// The same for surfaces with patch unions: block = (instance, patch, chunk of R
// right-hand sides) from a work list; sigma of the union of the patch rows' near
// patches staged for the R right-hand sides ([node][rhs], stride R + 1), each
// correction value read once per R right-hand sides (lane = sub-row * R + rhs).
template <int R>
__global__ void __launch_bounds__(256)
k_mnear32_patch(const MInst* __restrict__ I, const int4* __restrict__ items,
                double* __restrict__ out, long long ld_out, const int* __restrict__ skip) {
    if (skip && *skip) return;
    static_assert(32 % R == 0, "R divides the warp");
    constexpr int kSub = 32 / R;
    constexpr int kLd = R + 1;
    extern __shared__ float shs[];
    const int4 w = items[blockIdx.x];          // (instance, patch, first rhs, -)
    const MInst& in = I[w.x];
    const int P = w.y, r0 = w.z;
    const int nr = min(R, in.nrhs - r0);
    const int pp = in.pp, ppad = in.ppad, N = in.N;
    const int u0 = in.nu_ptr[P], U = in.nu_ptr[P + 1] - u0;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int total = U * R * ppad;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int k = e % ppad, t = e / ppad;
        const int rr = t % R, u = t / R;
        float v = 0.f;
        if (rr < nr && k < pp)
            v = in.sig32[(size_t)(r0 + rr) * in.npatch * ppad + (size_t)in.nu_list[u0 + u] * ppad + k];
        shs[(u * ppad + k) * kLd + rr] = v;
    }
    __syncthreads();
    const int sub = lane / R, rr = lane - sub * R;
    const int r = r0 + rr;
    const bool act = rr < nr;
    const int q4 = ppad >> 2;
    for (int t0 = warp * kSub; t0 < pp; t0 += (blockDim.x >> 5) * kSub) {
        const int t = t0 + sub;
        const bool row_ok = t < pp;
        const int i = P * pp + (row_ok ? t : 0);
        float hi = 0.f, lo = 0.f;
        if (act && row_ok)
            for (int sp = 0; sp < in.nsplit; ++sp) {
                const float2 v = in.part[((size_t)r * in.nsplit + sp) * N + i];
                two_sum_acc(hi, lo, v.x);
                lo += v.y;
            }
        float acc = 0.f;
        const int b0 = row_ok ? in.row_ptr[i] : 0, b1 = row_ok ? in.row_ptr[i + 1] : 0;
        for (int b = b0; b < b1; ++b) {
            const float4* c4 = reinterpret_cast<const float4*>(in.vals + (size_t)b * ppad);
            const float* su = shs + in.nu_blk[b] * ppad * kLd + rr;
            for (int k4 = 0; k4 < q4; ++k4) {
                const float4 c = __ldg(c4 + k4);
                const float* sk = su + 4 * k4 * kLd;
                acc = fmaf(c.x, sk[0], fmaf(c.y, sk[kLd], fmaf(c.z, sk[2 * kLd], fmaf(c.w, sk[3 * kLd], acc))));
            }
        }
        two_sum_acc(hi, lo, acc);
        if (act && row_ok) out[(size_t)(in.col0 + r) * ld_out + i] = (double)hi + (double)lo;
    }
}

// out_c = v_c + y_c + wdot_c on the column's own rows (A v with the rank-one term)
__global__ void k_mfinishA(const double* __restrict__ v, long long ldv, const double* __restrict__ y,
                           long long ldy, const double* __restrict__ wdot, long long ldw,
                           double* __restrict__ out, long long ldo, const int* __restrict__ col_n,
                           const int* __restrict__ done) {
    const int c = blockIdx.y;
    if (done && done[c]) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= col_n[c]) return;
    out[c * ldo + i] = v[c * ldv + i] + y[c * ldy + i] + wdot[c * ldw];
}

// out_c = w_c * f_c (per-column weights, zero past the column's rows)
__global__ void k_mmul(const double* __restrict__ w, const double* __restrict__ f,
                       double* __restrict__ out, int N) {
    const int c = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) out[(size_t)c * N + i] = w[(size_t)c * N + i] * f[(size_t)c * N + i];
}

// y_c[i] -= shift_c * scale_c on the column's own rows (weighted-mean projection)
__global__ void k_mshift(double* __restrict__ y, long long ldy, const double* __restrict__ shift,
                         long long lds, const double* __restrict__ scale,
                         const int* __restrict__ col_n) {
    const int c = blockIdx.y;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < col_n[c]) y[c * ldy + i] -= shift[c * lds] * scale[c];
}

}  // namespace

// Per-context workspace of the multi-instance solve, rebuilt when the call's
// shape (instances, right-hand sides, restart, tile) changes; its cycle graphs are
// cached per cycle length.
struct PmMultiWork {
    PmBatchSolveWork W;
    std::vector<const pm_surface*> ops;
    std::vector<int> nrhs;
    std::vector<long long> epochs;     // coefficient epochs of the operators at setup
    int ncols = 0, Nmax = 0, m = 0, rb = 0, nitems = 0, grid = 0, ninst = 0;
    long long nwarps = 0;
    int nnear = 0;                 // patch-blocked near-field items (0: per-row kernel)
    size_t near_smem = 0;
    MInst* dI = nullptr;
    MGroup* dG = nullptr;
    int fb = 4;                    // fields per smooth-sum item (1, 2 or 4), 8 right-hand sides each
    int4* items = nullptr;
    int4* near_items = nullptr;
    float4 *fac = nullptr, *nrm = nullptr;
    float* facB = nullptr;
    int *col_inst = nullptr, *col_n = nullptr;
    double *wcol = nullptr, *inv_sw = nullptr;
    float *s32 = nullptr, *sig32 = nullptr;
    float2* part = nullptr;
    cudaStream_t cap = nullptr;
    std::map<int, cudaGraphExec_t> graphs;
    void release() {
        for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
        graphs.clear();
        bsolve_release(W);
        W = PmBatchSolveWork();
        pm_dfree(dI); pm_dfree(dG); pm_dfree(items); pm_dfree(near_items); pm_dfree(col_inst);
        pm_dfree(fac); pm_dfree(nrm); pm_dfree(facB); pm_dfree(col_n); pm_dfree(wcol);
        pm_dfree(inv_sw); pm_dfree(s32); pm_dfree(sig32); pm_dfree(part);
        if (cap) cudaStreamDestroy(cap);
        cap = nullptr;
        ops.clear();
        nrhs.clear();
    }
    ~PmMultiWork() { release(); }
};

void pm_multi_free(pm_ctx* c) {
    delete c->multi;
    c->multi = nullptr;
}

namespace {

constexpr int kMultiNearRhs = 8;            // right-hand sides per near-field block
constexpr int kMultiNearSmemCap = 200 * 1024;

// (Re)build the workspace for this call's shape.
pm_status multi_setup(pm_ctx* ctx, pm_surface* const* ops, int nops, const int* nrhs, int m,
                      PmMultiWork** out) {
    PmMultiWork*& M = ctx->multi;
    const int rb = ops[0]->batch_rb;
    bool same = M && M->m == m && M->rb == rb && (int)M->ops.size() == nops;
    for (int k = 0; same && k < nops; ++k)
        same = M->ops[k] == ops[k] && M->nrhs[k] == nrhs[k] && M->epochs[k] == ops[k]->graph_epoch;
    if (same) {
        *out = M;
        return PM_OK;
    }
    if (!M) M = new PmMultiWork();
    M->release();
    int ncols = 0, Nmax = 0;
    for (int k = 0; k < nops; ++k) {
        ncols += nrhs[k];
        Nmax = std::max(Nmax, ops[k]->N);
    }
    M->ncols = ncols;
    M->Nmax = Nmax;
    M->m = m;
    M->rb = rb;
    M->ninst = nops;
    PM_TRY(bsolve_alloc(M->W, ncols, m, Nmax));
    PmBatchSolveWork& W = M->W;
    // zero padding of every column: the rows past an instance's N stay zero
    const size_t RN = (size_t)ncols * Nmax;
    for (double* p : {W.w, W.tmp, W.r, W.res, W.delta, W.sig, W.f, W.u})
        PM_CUDA_TRY(cudaMemset(p, 0, sizeof(double) * RN));
    PM_CUDA_TRY(cudaMemset(W.V, 0, sizeof(double) * RN * (m + 1)));
    // per-instance float32 buffers, source chunks of about 1,024 sources per item
    // (the persistent kernel balances items of similar size), the work list
    std::vector<MInst> hI(nops);
    std::vector<int4> items;
    std::vector<int> col_inst(ncols), col_n(ncols);
    std::vector<double> wcol(RN, 0.0), inv_sw(ncols);
    size_t n_s32 = 0, n_sig = 0, n_part = 0;
    long long warp0 = 0;
    int c0 = 0;
    for (int k = 0; k < nops; ++k) {
        const pm_surface* s = ops[k];
        MInst& in = hI[k];
        in.N = s->N;
        in.npatch = s->npatch;
        in.pp = s->pp;
        in.ppad = s->ppad;
        in.nrhs = nrhs[k];
        in.col0 = c0;
        in.nsplit = std::max(1, std::min(64, pm_ceil_div(s->N, 1024)));
        in.chunk = pm_ceil_div(s->N, in.nsplit);
        in.eps2 = s->eps2;
        in.warp0 = warp0;
        warp0 += (long long)nrhs[k] * s->N;
        n_s32 += (size_t)nrhs[k] * s->N;
        n_sig += (size_t)nrhs[k] * s->npatch * s->ppad;
        n_part += (size_t)nrhs[k] * in.nsplit * s->N;
        double sw = 0.0;
        for (double v : s->h_w) sw += v;
        for (int r = 0; r < nrhs[k]; ++r) {
            col_inst[c0 + r] = k;
            col_n[c0 + r] = s->N;
            inv_sw[c0 + r] = 1.0 / sw;
            std::copy(s->h_w.begin(), s->h_w.end(), wcol.begin() + (size_t)(c0 + r) * Nmax);
        }
        c0 += nrhs[k];
    }
    PM_TRY(pm_dmalloc(&M->s32, n_s32));
    PM_TRY(pm_dmalloc(&M->sig32, n_sig));
    PM_CUDA_TRY(cudaMemset(M->sig32, 0, sizeof(float) * n_sig));
    PM_TRY(pm_dmalloc(&M->part, n_part));
    size_t o32 = 0, osig = 0, opart = 0;
    for (int k = 0; k < nops; ++k) {
        const pm_surface* s = ops[k];
        MInst& in = hI[k];
        in.pos = s->src32;
        in.tgt = s->tgt32;
        in.wa = s->wa;
        in.row_ptr = s->row_ptr;
        in.blk_patch = s->blk_patch;
        in.vals = s->cR32;
        in.nu_ptr = s->nu_ptr;
        in.nu_list = s->nu_list;
        in.nu_blk = s->nu_blk;
        in.s32 = M->s32 + o32;
        in.sig32 = M->sig32 + osig;
        in.part = M->part + opart;
        o32 += (size_t)in.nrhs * s->N;
        osig += (size_t)in.nrhs * s->npatch * s->ppad;
        opart += (size_t)in.nrhs * in.nsplit * s->N;
    }
    // geometry groups (a surface and its clones share the float64 node array) of at
    // most kMultiGroupMax instances, their normals, every instance's remainder factors
    std::vector<MGroup> hG;
    std::map<const double*, int> open_group;
    PM_TRY(pm_dmalloc(&M->fac, (size_t)nops * Nmax));
    PM_TRY(pm_dmalloc(&M->facB, (size_t)nops * Nmax));
    for (int k = 0; k < nops; ++k) {
        const pm_surface* s = ops[k];
        auto og = open_group.find(s->x);
        if (og == open_group.end() || hG[og->second].ninst == kMultiGroupMax) {
            MGroup g{};
            g.pos = s->src32;
            g.tgt = s->tgt32;
            g.N = s->N;
            g.nsplit = hI[k].nsplit;
            g.chunk = hI[k].chunk;
            g.eps2 = s->eps2;
            g.ninst = 0;
            hG.push_back(g);
            open_group[s->x] = (int)hG.size() - 1;
            og = open_group.find(s->x);
        }
        MGroup& g = hG[og->second];
        g.inst[g.ninst++] = k;
        hI[k].fac = M->fac + (size_t)k * Nmax;
        hI[k].facB = M->facB + (size_t)k * Nmax;
    }
    PM_TRY(pm_dmalloc(&M->nrm, (size_t)hG.size() * Nmax));
    for (size_t gi = 0; gi < hG.size(); ++gi) {
        const pm_surface* s = ops[hG[gi].inst[0]];
        hG[gi].nrm = M->nrm + gi * Nmax;
        for (int q = 0; q < hG[gi].ninst; ++q) {
            const int k = hG[gi].inst[q];
            const pm_surface* sk = ops[k];
            k_mfactors<<<pm_ceil_div(sk->N, 256), 256>>>(sk->a, sk->H, sk->g, sk->n, sk->N,
                                                         const_cast<float4*>(hI[k].fac),
                                                         const_cast<float*>(hI[k].facB),
                                                         q == 0 ? M->nrm + gi * Nmax : nullptr);
        }
        (void)s;
    }
    PM_CUDA_TRY(cudaGetLastError());
    // fields per item (8 right-hand sides each): ops[0]'s batched knob when set
    // (8, 16 or 32 right-hand sides per block -> 1, 2 or 4 fields), else 2 where a
    // geometry carries several fields
    int gmax = 1;
    for (const MGroup& g : hG) gmax = std::max(gmax, g.ninst);
    const int knob = ops[0]->batch_rb;
    M->fb = knob == 32 ? 4 : (knob == 16 ? 2 : (knob == 8 ? 1 : (gmax >= 2 ? 2 : 1)));
    for (int gi = 0; gi < (int)hG.size(); ++gi) {
        const MGroup& g = hG[gi];
        int rmax = 0;
        for (int q = 0; q < g.ninst; ++q) rmax = std::max(rmax, nrhs[g.inst[q]]);
        for (int t = 0; t < pm_ceil_div(g.N, kThreads); ++t)
            for (int y = 0; y < g.nsplit; ++y)
                for (int fb = 0; fb < pm_ceil_div(g.ninst, M->fb); ++fb)
                    for (int rbk = 0; rbk < pm_ceil_div(rmax, 8); ++rbk)
                        items.push_back(make_int4(gi, t, y, fb * 4096 + rbk));
    }
    // largest items first, so the persistent blocks finish together
    std::stable_sort(items.begin(), items.end(), [&](const int4& a, const int4& b) {
        return hG[a.x].chunk > hG[b.x].chunk;
    });
    M->nitems = (int)items.size();
    PM_TRY(pm_dmalloc(&M->dG, hG.size()));
    PM_CUDA_TRY(cudaMemcpy(M->dG, hG.data(), sizeof(MGroup) * hG.size(), cudaMemcpyHostToDevice));
    M->nwarps = warp0;
    // patch-blocked near field when every instance has its patch unions and the
    // largest staging fits in shared memory
    std::vector<int4> nitems_v;
    size_t smem = 0;
    bool unions = true;
    for (int k = 0; k < nops; ++k) {
        const pm_surface* s = ops[k];
        unions &= s->nu_max > 0;
        smem = std::max(smem, (size_t)s->nu_max * s->ppad * (kMultiNearRhs + 1) * sizeof(float));
        for (int P = 0; P < s->npatch; ++P)
            for (int r0 = 0; r0 < nrhs[k]; r0 += kMultiNearRhs) nitems_v.push_back(make_int4(k, P, r0, 0));
    }
    if (unions && smem <= (size_t)kMultiNearSmemCap) {
        PM_TRY(pm_dmalloc(&M->near_items, nitems_v.size()));
        PM_CUDA_TRY(cudaMemcpy(M->near_items, nitems_v.data(), sizeof(int4) * nitems_v.size(),
                               cudaMemcpyHostToDevice));
        M->nnear = (int)nitems_v.size();
        M->near_smem = smem;
        // on the current device, always the same cap (never lowered under another launch)
        PM_CUDA_TRY(cudaFuncSetAttribute(k_mnear32_patch<kMultiNearRhs>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kMultiNearSmemCap));
    }
    PM_TRY(pm_dmalloc(&M->dI, nops));
    PM_TRY(pm_dmalloc(&M->items, items.size()));
    PM_TRY(pm_dmalloc(&M->col_inst, ncols));
    PM_TRY(pm_dmalloc(&M->col_n, ncols));
    PM_TRY(pm_dmalloc(&M->wcol, RN));
    PM_TRY(pm_dmalloc(&M->inv_sw, ncols));
    PM_CUDA_TRY(cudaMemcpy(M->dI, hI.data(), sizeof(MInst) * nops, cudaMemcpyHostToDevice));
    PM_CUDA_TRY(cudaMemcpy(M->items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice));
    PM_CUDA_TRY(cudaMemcpy(M->col_inst, col_inst.data(), sizeof(int) * ncols, cudaMemcpyHostToDevice));
    PM_CUDA_TRY(cudaMemcpy(M->col_n, col_n.data(), sizeof(int) * ncols, cudaMemcpyHostToDevice));
    PM_CUDA_TRY(cudaMemcpy(M->wcol, wcol.data(), sizeof(double) * RN, cudaMemcpyHostToDevice));
    PM_CUDA_TRY(cudaMemcpy(M->inv_sw, inv_sw.data(), sizeof(double) * ncols, cudaMemcpyHostToDevice));
    const int bps = (ops[0]->batch_bps >= 1 && ops[0]->batch_bps <= 16) ? ops[0]->batch_bps : 8;
    M->grid = std::max(1, std::min(M->nitems, bps * ops[0]->ctx->num_sms));
    PM_CUDA_TRY(cudaStreamCreateWithFlags(&M->cap, cudaStreamNonBlocking));
    M->ops.assign(ops, ops + nops);
    M->nrhs.assign(nrhs, nrhs + nops);
    M->epochs.clear();
    for (int k = 0; k < nops; ++k) M->epochs.push_back(ops[k]->graph_epoch);
    PM_CUDA_TRY(cudaDeviceSynchronize());      // factors written on the default stream
    *out = M;
    return PM_OK;
}

struct MSolver {
    PmMultiWork& M;
    PmBatchSolveWork& W;
    pm_surface* const* ops;
    int nops;
    cudaStream_t st;
    int grid_n;
    bool op_residual;              // residuals in the float32 operator itself
    long long launches = 0;

    void dots(const double* A, long long col_stride, long long rhs_stride_A, int ncols_,
              const double* b, long long rhs_stride_b, double* dst, long long lddst,
              const int* done) {
        k_bdots<<<dim3(W.nred, M.ncols), kRed, 0, st>>>(A, col_stride, rhs_stride_A, ncols_, b,
                                                         rhs_stride_b, W.N, W.part, done);
        k_breduce<<<dim3(pm_ceil_div(ncols_, 64), M.ncols), 64, 0, st>>>(W.part, W.nred, ncols_,
                                                                         dst, lddst, done);
        launches += 2;
    }

    // out_c = A v_c for every column; prec FP32 (one multi-instance launch per stage)
    // or FF (the accurate batched apply of each instance on its columns)
    pm_status apply_A(const double* v, long long ldv, double* out, pm_precision prec,
                      const int* done, const int* skip) {
        if (prec == PM_PREC_FP32) {
            k_mprep32<<<dim3(pm_ceil_div(M.Nmax, 256), M.ncols), 256, 0, st>>>(v, ldv, M.dI,
                                                                                  M.col_inst, skip);
            if (M.fb == 4)
                k_mgeo32<4, 8><<<M.grid, kThreads, 0, st>>>(M.dG, M.dI, M.items, M.nitems, skip);
            else if (M.fb == 2)
                k_mgeo32<2, 8><<<M.grid, kThreads, 0, st>>>(M.dG, M.dI, M.items, M.nitems, skip);
            else
                k_mgeo32<1, 8><<<M.grid, kThreads, 0, st>>>(M.dG, M.dI, M.items, M.nitems, skip);
            if (M.nnear > 0)
                k_mnear32_patch<kMultiNearRhs><<<M.nnear, 256, M.near_smem, st>>>(
                    M.dI, M.near_items, W.tmp, W.N, skip);
            else
                k_mnear32<<<(int)((M.nwarps * 32 + 255) / 256), 256, 0, st>>>(M.dI, M.ninst,
                                                                            M.nwarps, W.tmp, W.N,
                                                                            skip);
            launches += 3;
        } else {
            int c0 = 0;
            for (int k = 0; k < nops; ++k) {
                PM_TRY(pm_apply_batch(ops[k], 0, v + (size_t)c0 * ldv, ldv, W.tmp + (size_t)c0 * W.N,
                                      W.N, M.nrhs[k], prec, st));
                c0 += M.nrhs[k];
            }
        }
        dots(M.wcol, 0, W.N, 1, v, ldv, W.dots + 0, 8, done);
        k_mfinishA<<<dim3(grid_n, M.ncols), 256, 0, st>>>(v, ldv, W.tmp, W.N, W.dots + 0, 8, out,
                                                          W.N, M.col_n, done);
        launches += 1;
        PM_CUDA_TRY(cudaGetLastError());
        return PM_OK;
    }

    pm_status norms(const double* v, double* host) {
        dots(v, 0, W.N, 1, v, W.N, W.dots + 1, 8, nullptr);
        PM_CUDA_TRY(cudaMemcpyAsync(W.pinned, W.dots, sizeof(double) * 8 * M.ncols,
                                    cudaMemcpyDeviceToHost, st));
        PM_CUDA_TRY(cudaStreamSynchronize(st));
        for (int c = 0; c < M.ncols; ++c) host[c] = std::sqrt(W.pinned[8 * c + 1]);
        return PM_OK;
    }

    // the launches of one GMRES cycle of `steps` Arnoldi steps (float32 operator)
    pm_status issue_cycle(int steps) {
        const int m = W.m, N = W.N, nc = M.ncols;
        const long long ldV = (long long)(m + 1) * N;
        const int ldh = m + 2;
        dots(W.r, 0, N, 1, W.r, N, W.scal + 1, 8, nullptr);
        k_bcycle_start<<<1, 256, 0, st>>>(nc, W.scal + 1, 8, W.g, m, W.scal, W.done, W.iters,
                                          W.all_done);
        k_bscale_copy<<<dim3(grid_n, nc), 256, 0, st>>>(W.r, N, W.scal + 3, 8, 1, W.V, ldV, N,
                                                        W.done);
        launches += 2;
        for (int k = 0; k < steps; ++k) {
            double* vk = W.V + (size_t)k * N;
            double* vk1 = W.V + (size_t)(k + 1) * N;
            double* hk = W.H + (size_t)k * ldh;
            PM_TRY(apply_A(vk, ldV, W.w, PM_PREC_FP32, W.done, W.all_done));
            dots(W.V, N, ldV, k + 1, W.w, N, hk, (long long)m * ldh, W.done);
            k_bsub<<<dim3(grid_n, nc), 256, 0, st>>>(W.V, N, ldV, k + 1, hk, (long long)m * ldh,
                                                     W.w, N, W.done);
            dots(W.V, N, ldV, k + 1, W.w, N, W.hcol, m + 2, W.done);
            k_bsub<<<dim3(grid_n, nc), 256, 0, st>>>(W.V, N, ldV, k + 1, W.hcol, m + 2, W.w, N,
                                                     W.done);
            k_badd_cols<<<dim3(pm_ceil_div(k + 1, 64), nc), 64, 0, st>>>(
                hk, (long long)m * ldh, W.hcol, m + 2, k + 1, W.done);
            dots(W.w, 0, N, 1, W.w, N, W.scal + 1, 8, W.done);
            k_brotate<<<1, 256, 0, st>>>(nc, W.H, ldh, m, k, W.cs, W.sn, W.g, W.scal, W.done,
                                         W.iters, W.all_done);
            k_bscale_copy<<<dim3(grid_n, nc), 256, 0, st>>>(W.w, N, W.scal + 2, 8, 0, vk1, ldV, N,
                                                            W.done);
            launches += 5;
        }
        k_bbacksolve<<<pm_ceil_div(nc, 64), 64, 0, st>>>(nc, W.H, ldh, m, W.g, W.iters, W.y,
                                                         W.ynorm);
        k_badd_combo<<<dim3(grid_n, nc), 256, 0, st>>>(W.V, N, ldV, W.iters, W.y, m, W.delta, N);
        launches += 2;
        PM_CUDA_TRY(cudaGetLastError());
        return PM_OK;
    }

    // one cycle as a CUDA graph (captured on the workspace's own stream the first
    // time a cycle of this length runs, replayed on st after that)
    pm_status run_cycle(int steps) {
        auto it = M.graphs.find(steps);
        if (it == M.graphs.end()) {
            cudaStream_t user = st;
            st = M.cap;
            PM_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            const long long before = launches;
            const pm_status ps = issue_cycle(steps);
            cudaGraph_t g = nullptr;
            const cudaError_t ce = cudaStreamEndCapture(st, &g);
            st = user;
            launches = before;
            if (ps != PM_OK) {
                if (g) cudaGraphDestroy(g);
                return ps;
            }
            cudaGraphExec_t ex = nullptr;
            cudaError_t ce2 =
                ce == cudaSuccess
                    ? cudaGraphInstantiate(&ex, g, cudaGraphInstantiateFlagUseNodePriority)
                    : ce;
            if (g) cudaGraphDestroy(g);
            if (ce2 != cudaSuccess) {
                cudaGetLastError();
                pm_set_error("multi-instance solve: cycle graph capture: %s", cudaGetErrorString(ce2));
                return PM_ERR_CUDA;
            }
            it = M.graphs.emplace(steps, ex).first;
        }
        PM_CUDA_TRY(cudaGraphLaunch(it->second, st));
        launches += 1;
        return PM_OK;
    }

    // lockstep restarted GMRES on A d_c = b_c from d = 0 (float32 operator); x += d
    pm_status gmres(const double* b, double* x, const std::vector<double>& tol_abs, int max_iter,
                    int* iters_used, std::vector<double>* dnorm) {
        const int nc = M.ncols, N = W.N;
        dnorm->assign(nc, 0.0);
        PM_CUDA_TRY(cudaMemcpyAsync(W.r, b, sizeof(double) * (size_t)nc * N,
                                    cudaMemcpyDeviceToDevice, st));
        PM_CUDA_TRY(cudaMemsetAsync(W.delta, 0, sizeof(double) * (size_t)nc * N, st));
        for (int c = 0; c < nc; ++c) W.pinned[8 * c + 4] = tol_abs[c];
        for (int c = 0; c < nc; ++c)
            PM_CUDA_TRY(cudaMemcpyAsync(W.scal + 8 * c + 4, W.pinned + 8 * c + 4, sizeof(double),
                                        cudaMemcpyHostToDevice, st));
        int total = 0;
        while (total < max_iter) {
            const int steps = std::min(W.m, max_iter - total);
            PM_TRY(run_cycle(steps));
            PM_CUDA_TRY(cudaMemcpyAsync(W.pinned_i, W.iters, sizeof(int) * nc,
                                        cudaMemcpyDeviceToHost, st));
            PM_CUDA_TRY(cudaMemcpyAsync(W.pinned_i + nc, W.done, sizeof(int) * nc,
                                        cudaMemcpyDeviceToHost, st));
            PM_CUDA_TRY(cudaMemcpyAsync(W.pinned_y, W.ynorm, sizeof(double) * nc,
                                        cudaMemcpyDeviceToHost, st));
            PM_CUDA_TRY(cudaStreamSynchronize(st));
            int it = 0, all = 1;
            for (int c = 0; c < nc; ++c) {
                it = std::max(it, W.pinned_i[c]);
                all &= W.pinned_i[nc + c];
                if (W.pinned_i[c] > 0) (*dnorm)[c] += W.pinned_y[c];
            }
            total += it;
            if (all || it == 0) break;
            PM_TRY(apply_A(W.delta, N, W.w, PM_PREC_FP32, nullptr, nullptr));
            k_bresidual<<<dim3(grid_n, nc), 256, 0, st>>>(b, W.w, W.r, N);
            launches += 1;
        }
        k_baxpy<<<dim3(grid_n, nc), 256, 0, st>>>(x, W.delta, N);
        launches += 1;
        PM_CUDA_TRY(cudaGetLastError());
        *iters_used = total;
        return PM_OK;
    }

};

}  // namespace

namespace {

// u_c = K~ sigma_c (float-float) for the columns of several operators.  The
// parametrix sum depends on an operator's coefficient only through the strengths
// w sigma / a, so the columns of operators on one geometry (consecutive instances
// sharing the node array) go through ONE float-float parametrix sum with every
// column's own strengths; each operator then adds its own float64 corrections.
// Other instances use the per-operator batched apply.
pm_status multi_representation_ff(pm_surface* const* ops, int nops, const int* nrhs,
                                  const double* sig, double* out, long long ld, cudaStream_t st) {
    int k = 0, c0 = 0;
    while (k < nops) {
        int k1 = k + 1, cols = nrhs[k];
        while (k1 < nops && ops[k1]->x == ops[k]->x) cols += nrhs[k1++];
        pm_surface* s0 = ops[k];
        if (k1 - k == 1) {
            PM_TRY(pm_apply_batch(s0, 1, sig + (size_t)c0 * ld, ld, out + (size_t)c0 * ld, ld,
                                  nrhs[k], PM_PREC_FF, st));
        } else {
            PM_TRY(batch_ensure(s0, cols));
            PmBatchWork& B = *s0->batch;
            const int N = s0->N;
            const int rbff = cols <= 8 ? 8 : kRBff;
            const int ns = batch_splits(s0, cols, rbff, 8);
            int c = 0;
            for (int q = k; q < k1; ++q) {
                k_prep_ff_multi<<<dim3(pm_ceil_div(N, 256), nrhs[q]), 256, 0, st>>>(
                    sig + (size_t)(c0 + c) * ld, ld, ops[q]->wa, B.sff + (size_t)c * N, N, nullptr);
                c += nrhs[q];
            }
            const dim3 g(pm_ceil_div(N, kThreads), ns, pm_ceil_div(cols, rbff));
            const int chunk = pm_ceil_div(N, ns);
            if (rbff == 8)
                k_direct_multi_ff<true, 8><<<g, kThreads, 0, st>>>(s0->src_kg, B.sff, cols, s0->tgt_ff,
                                                                  s0->log_tab, N, chunk, B.part, ns,
                                                                  nullptr);
            else
                k_direct_multi_ff<true, kRBff><<<g, kThreads, 0, st>>>(s0->src_kg, B.sff, cols,
                                                                      s0->tgt_ff, s0->log_tab, N,
                                                                      chunk, B.part, ns, nullptr);
            c = 0;
            for (int q = k; q < k1; ++q) {
                const dim3 gn(pm_ceil_div((long long)N * 32, 256), nrhs[q]);
                k_near_multi64<<<gn, 256, 0, st>>>(N, ops[q]->pp, ops[q]->row_ptr,
                                                   ops[q]->blk_patch, ops[q]->cK64,
                                                   sig + (size_t)(c0 + c) * ld, ld,
                                                   B.part + (size_t)c * ns * N, ns,
                                                   out + (size_t)(c0 + c) * ld, ld, nullptr);
                c += nrhs[q];
            }
            s0->launch_total += 2 * (k1 - k) + 1;
            PM_CUDA_TRY(cudaGetLastError());
        }
        c0 += cols;
        k = k1;
    }
    return PM_OK;
}

}  // namespace

extern "C" pm_status pm_solve_multi(pm_surface* const* ops, int nops, const int* nrhs,
                                    const double* const* f, double* const* u, double tol,
                                    int maxit, pm_precision prec, unsigned flags,
                                    pm_solve_info* info, void* stream) {
    const auto t0 = std::chrono::steady_clock::now();
    if (!ops || nops < 1 || !nrhs || !f || !u || !(tol > 0) || maxit < 1) {
        pm_set_error("pm_solve_multi: NULL argument, nops < 1, tol <= 0 or maxit < 1");
        return PM_ERR_INVALID_ARG;
    }
    if (prec != PM_PREC_FP32) {
        pm_set_error("pm_solve_multi: precision %d: the multi-instance solve applies the float32 "
                     "operators (PM_PREC_FP32)", (int)prec);
        return PM_ERR_INVALID_ARG;
    }
    for (int k = 0; k < nops; ++k) {
        if (!ops[k] || !f[k] || !u[k] || nrhs[k] < 1) {
            pm_set_error("pm_solve_multi: instance %d: NULL operator or array, or nrhs < 1", k);
            return PM_ERR_INVALID_ARG;
        }
        if (!ops[k]->has_coeff) {
            pm_set_error("pm_solve_multi: instance %d has no coefficient", k);
            return PM_ERR_NO_COEFF;
        }
        if (ops[k]->has_c) {
            pm_set_error("pm_solve_multi: instance %d has c != 0 (pm_solve_c solves it)", k);
            return PM_ERR_INVALID_ARG;
        }
        if (ops[k]->ctx != ops[0]->ctx) {
            pm_set_error("pm_solve_multi: instance %d belongs to another context", k);
            return PM_ERR_INVALID_ARG;
        }
        for (int j = 0; j < k; ++j)
            if (ops[j] == ops[k]) {
                pm_set_error("pm_solve_multi: operator of instance %d repeats instance %d "
                             "(give it more right-hand sides instead)", k, j);
                return PM_ERR_INVALID_ARG;
            }
    }
    pm_ctx* ctx = ops[0]->ctx;
    std::lock_guard<std::mutex> lock(ctx->multi_mu);
    PM_CUDA_TRY(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    const int m = std::max(2, std::min(ops[0]->opts.gmres_restart, 400));
    PmMultiWork* Mp = nullptr;
    PM_TRY(multi_setup(ctx, ops, nops, nrhs, m, &Mp));
    PmMultiWork& M = *Mp;
    PmBatchSolveWork& W = M.W;
    const int nc = M.ncols, N = W.N;
    MSolver S{M, W, ops, nops, st, pm_ceil_div(N, 256),
              ops[0]->opts.residual_prec == PM_PREC_FP32};
    const bool dev = (flags & PM_SOLVE_DEVICE_PTRS) != 0;
    const cudaMemcpyKind h2d = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const cudaMemcpyKind d2h = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    {
        int c0 = 0;
        for (int k = 0; k < nops; ++k) {
            const size_t Nk = ops[k]->N;
            for (int r = 0; r < nrhs[k]; ++r)
                PM_CUDA_TRY(cudaMemcpyAsync(W.f + (size_t)(c0 + r) * N, f[k] + r * Nk,
                                            sizeof(double) * Nk, h2d, st));
            c0 += nrhs[k];
        }
    }
    // mean-zero check of every f (Thm. LBsolvable): sum w f and sum w f^2 per column
    k_mmul<<<dim3(S.grid_n, nc), 256, 0, st>>>(M.wcol, W.f, W.tmp, N);   // w f per column
    S.dots(M.wcol, 0, N, 1, W.f, N, W.dots + 4, 8, nullptr);           // sum w f
    S.dots(W.tmp, 0, N, 1, W.f, N, W.dots + 5, 8, nullptr);            // sum w f^2
    S.launches += 1;
    PM_CUDA_TRY(cudaMemcpyAsync(W.pinned, W.dots, sizeof(double) * 8 * nc, cudaMemcpyDeviceToHost, st));
    PM_CUDA_TRY(cudaStreamSynchronize(st));
    std::vector<double> removed(nc, 0.0), fnorm(nc, 0.0), sw(nc, 0.0);
    {
        int c0 = 0;
        for (int k = 0; k < nops; ++k) {
            double s = 0.0;
            for (double v : ops[k]->h_w) s += v;
            for (int r = 0; r < nrhs[k]; ++r) sw[c0 + r] = s;
            c0 += nrhs[k];
        }
    }
    std::vector<double> shift(nc, 0.0);
    for (int c = 0; c < nc; ++c) {
        const double wf = W.pinned[8 * c + 4];
        if (W.pinned[8 * c + 5] > 0.0 &&
            std::fabs(wf) > ops[0]->opts.mean_tol * std::sqrt(sw[c] * W.pinned[8 * c + 5]) &&
            !(flags & PM_SOLVE_PROJECT_RHS)) {
            pm_set_error("pm_solve_multi: right-hand side %d has weighted mean %.3e; pass "
                         "PM_SOLVE_PROJECT_RHS to subtract it", c, wf / sw[c]);
            return PM_ERR_RHS_NOT_MEAN_ZERO;
        }
        if (flags & PM_SOLVE_PROJECT_RHS) removed[c] = wf / sw[c];
    }
    if (flags & PM_SOLVE_PROJECT_RHS) {
        k_mshift<<<dim3(S.grid_n, nc), 256, 0, st>>>(W.f, N, W.dots + 4, 8, M.inv_sw, M.col_n);
        S.launches += 1;
    }
    PM_TRY(S.norms(W.f, fnorm.data()));
    PM_CUDA_TRY(cudaMemsetAsync(W.sig, 0, sizeof(double) * (size_t)nc * N, st));
    int iters = 0, refinements = 0, updated = 0;
    std::vector<double> relres(nc, 0.0), tabs(nc), dn;
    bool have_update = false;
    for (;;) {
        std::vector<double> rn(nc);
        if (refinements == 0) {
            PM_CUDA_TRY(cudaMemcpyAsync(W.res, W.f, sizeof(double) * (size_t)nc * N,
                                        cudaMemcpyDeviceToDevice, st));
            rn = fnorm;
        } else {
            // per instance: r - A32 d when every one of its columns' corrections is small
            // (within 0.1 tol |f| of the true residual, see pm_solve.cu), else f - A sigma
            // recomputed in float-float for that instance's columns only
            std::vector<int> exact(nops, 0);
            bool any_exact = false;
            int c0 = 0;
            for (int k = 0; k < nops; ++k) {
                bool small = S.op_residual || (have_update && ops[0]->opts.residual_update);
                for (int r = 0; small && r < nrhs[k]; ++r)
                    small = kOpRelErr * dn[c0 + r] <= 0.1 * tol * fnorm[c0 + r];
                exact[k] = !small;
                any_exact |= !small;
                c0 += nrhs[k];
            }
            PM_TRY(S.apply_A(W.delta, N, W.w, PM_PREC_FP32, nullptr, nullptr));
            k_bsubv<<<dim3(S.grid_n, nc), 256, 0, st>>>(W.res, W.w, N);
            S.launches += 1;
            if (any_exact) {
                c0 = 0;
                for (int k = 0; k < nops; ++k) {
                    if (exact[k])
                        PM_TRY(pm_apply_batch(ops[k], 0, W.sig + (size_t)c0 * N, N,
                                              W.tmp + (size_t)c0 * N, N, nrhs[k], PM_PREC_FF, st));
                    c0 += nrhs[k];
                }
                S.dots(M.wcol, 0, N, 1, W.sig, N, W.dots + 0, 8, nullptr);
                c0 = 0;
                for (int k = 0; k < nops; ++k) {
                    if (exact[k]) {
                        // res = f - (sigma + R~ sigma + (w . sigma) 1) on these columns
                        k_mfinishA<<<dim3(S.grid_n, nrhs[k]), 256, 0, st>>>(
                            W.sig + (size_t)c0 * N, N, W.tmp + (size_t)c0 * N, N, W.dots + 8 * c0, 8,
                            W.w + (size_t)c0 * N, N, M.col_n + c0, nullptr);
                        k_bresidual<<<dim3(S.grid_n, nrhs[k]), 256, 0, st>>>(
                            W.f + (size_t)c0 * N, W.w + (size_t)c0 * N, W.res + (size_t)c0 * N, N);
                        S.launches += 2;
                    } else {
                        updated += 1;
                    }
                    c0 += nrhs[k];
                }
            } else {
                updated += nops;
            }
            PM_TRY(S.norms(W.res, rn.data()));
        }
        bool all_ok = true;
        for (int c = 0; c < nc; ++c) {
            relres[c] = fnorm[c] > 0 ? rn[c] / fnorm[c] : 0.0;
            all_ok &= relres[c] <= tol;
        }
        if (all_ok || refinements >= ops[0]->opts.max_refine || iters >= maxit) break;
        for (int c = 0; c < nc; ++c) {
            const double inner = S.op_residual ? 0.5 * tol * fnorm[c] / std::max(rn[c], 1e-300)
                                               : std::max(ops[0]->opts.inner_tol,
                                                          0.5 * tol * fnorm[c] / std::max(rn[c], 1e-300));
            tabs[c] = (relres[c] <= tol) ? 1e300 : inner * rn[c];
        }
        int it = 0;
        PM_TRY(S.gmres(W.res, W.sig, tabs, maxit - iters, &it, &dn));
        have_update = true;
        iters += it;
        ++refinements;
        if (it == 0) break;
    }
    pm_status result = PM_OK;
    for (int c = 0; c < nc; ++c)
        if (!(relres[c] <= tol)) {
            pm_set_error("pm_solve_multi: column %d: relative residual %.3e above %.3e", c,
                         relres[c], tol);
            result = PM_ERR_NOT_CONVERGED;
        }
    // u = K~ sigma (float-float, or the float32 operator), minus its weighted mean
    if (S.op_residual) {
        int c0 = 0;
        for (int k = 0; k < nops; ++k) {
            PM_TRY(pm_apply_batch(ops[k], 1, W.sig + (size_t)c0 * N, N, W.u + (size_t)c0 * N, N,
                                  nrhs[k], PM_PREC_FP32, st));
            c0 += nrhs[k];
        }
    } else {
        PM_TRY(multi_representation_ff(ops, nops, nrhs, W.sig, W.u, N, st));
    }
    S.dots(M.wcol, 0, N, 1, W.u, N, W.dots + 6, 8, nullptr);
    k_mshift<<<dim3(S.grid_n, nc), 256, 0, st>>>(W.u, N, W.dots + 6, 8, M.inv_sw, M.col_n);
    {
        int c0 = 0;
        for (int k = 0; k < nops; ++k) {
            const size_t Nk = ops[k]->N;
            for (int r = 0; r < nrhs[k]; ++r)
                PM_CUDA_TRY(cudaMemcpyAsync(u[k] + r * Nk, W.u + (size_t)(c0 + r) * N,
                                            sizeof(double) * Nk, d2h, st));
            c0 += nrhs[k];
        }
    }
    PM_CUDA_TRY(cudaStreamSynchronize(st));
    ops[0]->launch_total += S.launches;
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (info)
        for (int c = 0; c < nc; ++c) {
            info[c].iterations = iters;
            info[c].refinements = refinements;
            info[c].residual = relres[c];
            info[c].removed_mean = removed[c];
            info[c].seconds = secs;
            info[c].residual_updates = updated;
        }
    return result;
}
