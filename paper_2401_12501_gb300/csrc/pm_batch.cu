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

void pm_batch_solve_free(pm_surface* s) {
    if (!s->bsolve) return;
    PmBatchSolveWork& W = *s->bsolve;
    pm_dfree(W.V); pm_dfree(W.H); pm_dfree(W.cs); pm_dfree(W.sn); pm_dfree(W.g); pm_dfree(W.y);
    pm_dfree(W.part); pm_dfree(W.scal); pm_dfree(W.hcol); pm_dfree(W.dots); pm_dfree(W.w);
    pm_dfree(W.tmp); pm_dfree(W.r); pm_dfree(W.res); pm_dfree(W.delta); pm_dfree(W.sig);
    pm_dfree(W.f); pm_dfree(W.u); pm_dfree(W.done); pm_dfree(W.iters); pm_dfree(W.all_done);
    pm_dfree(W.ynorm);
    if (W.pinned_y) cudaFreeHost(W.pinned_y);
    if (W.pinned) cudaFreeHost(W.pinned);
    if (W.pinned_i) cudaFreeHost(W.pinned_i);
    delete s->bsolve;
    s->bsolve = nullptr;
}

static pm_status bsolve_work(pm_surface* s, int nrhs, PmBatchSolveWork** out) {
    const int m = std::max(2, std::min(s->opts.gmres_restart, 400));
    if (s->bsolve && s->bsolve->nrhs >= nrhs && s->bsolve->m == m) {
        *out = s->bsolve;
        return PM_OK;
    }
    pm_batch_solve_free(s);
    s->bsolve = new PmBatchSolveWork();
    PmBatchSolveWork& W = *s->bsolve;
    const int N = s->N;
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
    *out = &W;
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
