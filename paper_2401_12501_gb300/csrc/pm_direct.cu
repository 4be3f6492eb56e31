// Smooth-rule N-body sums of the remainder and the parametrix (Sec. 6.1.3).
//
// For every target i (its own node included among the sources, excluded from
// the sum) with source strengths s_j = w_j sigma_j / a_j:
//
//   R part:  y_i = sum_{j != i} s_j [ (a_i/pi) q^2 - (a_i H_i/pi) q + g_i.r/(2 pi r^2) ],
//            q = n_i.r / r^2,  r = x_i - x_j        (Thm. parametrix, eq. explicit_remainder)
//   K part:  u_i = sum_{j != i} s_j log|r| / (2 pi) = (ln 2 / (4 pi)) sum s_j log2(r^2)
//                                                    (eq. diff_param)
//
// The R term is evaluated in the factorised form
//   s * inv * ( (n'.r)(n'.r) inv + m.r ),   inv = 1/r^2,
//   n' = sqrt(a_i/pi) n_i,  m = -(a_i H_i/pi) n_i + g_i/(2 pi),
// i.e. 16 float32 instructions and one MUFU reciprocal per pair.  The j == i
// pair needs no branch: r^2 is formed as r.r + eps2 with eps2 far below any
// inter-node distance, so the self pair has n'.r = m.r = 0 and contributes 0.
//
// float32 path: each thread keeps two targets in registers; sources (x,y,z,s)
// are staged through shared memory in tiles of 256 and broadcast to the warp.
// Each tile's partial sum is added to a (hi, lo) pair with TwoSum, so the
// rounding error grows with the tile length, not with N.  Sources are split
// over gridDim.y; each split writes hi + lo as a float64 partial that the
// near-field kernel adds (pm_nearfield.cu).
#include "pm_internal.cuh"

#include <algorithm>
#include <cmath>
#include <mutex>

namespace {

constexpr int kThreads = 128;
constexpr int kTile = 256;              // sources per compensation tile

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

// Knuth's TwoSum: hi + lo += v with the rounding error of the addition kept.
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float v) {
    float s = hi + v;
    float bp = s - hi;
    float err = (hi - (s - bp)) + (v - bp);
    hi = s;
    lo += err;
}

__global__ void k_prep32(const double* __restrict__ sigma, const double* __restrict__ wa,
                         float4* __restrict__ src, float* __restrict__ sig32, int N, int pp,
                         int ppad, const int* __restrict__ skip) {
    if (skip && *skip) return;
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    double sg = sigma[j];
    src[j].w = (float)(wa[j] * sg);
    int P = j / pp;
    sig32[(size_t)P * ppad + (j - P * pp)] = (float)sg;
}

__global__ void k_prep64(const double* __restrict__ sigma, const double* __restrict__ wa,
                         pm_d4* __restrict__ src, int N, const int* __restrict__ skip) {
    if (skip && *skip) return;
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    src[j].w = wa[j] * sigma[j];
}

__global__ void k_pack(const double* __restrict__ x, const double* __restrict__ n,
                       const double* __restrict__ H, const double* __restrict__ a,
                       const double* __restrict__ g, const double* __restrict__ w,
                       float4* __restrict__ tgt, float4* __restrict__ src32,
                       pm_d4* __restrict__ src64, double* __restrict__ wa, int N, int Npad,
                       double far) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= Npad) return;
    if (i >= N) {
        // padding sources: zero strength, far from every target (finite kernels)
        src32[i] = make_float4((float)far, (float)far, (float)far, 0.f);
        src64[i] = pm_d4{far, far, far, 0.0};
        return;
    }
    const double xi = x[3 * i], yi = x[3 * i + 1], zi = x[3 * i + 2];
    const double nx = n[3 * i], ny = n[3 * i + 1], nz = n[3 * i + 2];
    const double ai = a[i];
    const double c1 = sqrt(ai / M_PI);
    const double cH = -ai * H[i] / M_PI;
    const double c2 = 0.5 / M_PI;
    tgt[i] = make_float4((float)xi, (float)yi, (float)zi, 0.f);
    tgt[N + i] = make_float4((float)(c1 * nx), (float)(c1 * ny), (float)(c1 * nz), 0.f);
    tgt[2 * N + i] = make_float4((float)(cH * nx + c2 * g[3 * i]), (float)(cH * ny + c2 * g[3 * i + 1]),
                                 (float)(cH * nz + c2 * g[3 * i + 2]), 0.f);
    src32[i] = make_float4((float)xi, (float)yi, (float)zi, 0.f);
    src64[i] = pm_d4{xi, yi, zi, 0.0};
    wa[i] = w[i] / ai;
}

// ------------------------------------------------------------------ float32 remainder sum
// Block = 128 threads x TPT targets; blockIdx.y selects a source chunk of any
// length (the chunks split N evenly, so every block has the same work).  The
// chunk is staged through shared memory in stages of kStage sources; every
// kTile sources the tile partial is folded into (hi, lo) with TwoSum.
constexpr int kStage = 1024;

template <int TPT>
__global__ void __launch_bounds__(kThreads)
k_direct_R32(const float4* __restrict__ src, const float4* __restrict__ tgt, int N, int chunk,
             float eps2, float2* __restrict__ partial, const int* __restrict__ skip) {
    if (skip && *skip) return;
    __shared__ float4 sh[kStage];
    const int tid = threadIdx.x;
    const int tbase = blockIdx.x * kThreads * TPT;
    float tx[TPT], ty[TPT], tz[TPT], nx[TPT], ny[TPT], nz[TPT], mx[TPT], my[TPT], mz[TPT],
        hi[TPT], lo[TPT];
#pragma unroll
    for (int t = 0; t < TPT; ++t) {
        const int i = tbase + t * kThreads + tid;
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a, c = a;
        if (i < N) {
            a = tgt[i];
            b = tgt[N + i];
            c = tgt[2 * N + i];
        }
        tx[t] = a.x; ty[t] = a.y; tz[t] = a.z;
        nx[t] = b.x; ny[t] = b.y; nz[t] = b.z;
        mx[t] = c.x; my[t] = c.y; mz[t] = c.z;
        hi[t] = 0.f; lo[t] = 0.f;
    }
    const int s0 = blockIdx.y * chunk;
    const int s1 = min(s0 + chunk, N);
    for (int base = s0; base < s1; base += kStage) {
        const int len = min(kStage, s1 - base);
        __syncthreads();
        for (int j = tid; j < len; j += kThreads) sh[j] = src[base + j];
        __syncthreads();
        for (int j0 = 0; j0 < len; j0 += kTile) {
            const int j1 = min(j0 + kTile, len);
            float part[TPT];
#pragma unroll
            for (int t = 0; t < TPT; ++t) part[t] = 0.f;
#pragma unroll 4
            for (int j = j0; j < j1; ++j) {
                const float4 s = sh[j];
#pragma unroll
                for (int t = 0; t < TPT; ++t) {
                    const float dx = tx[t] - s.x, dy = ty[t] - s.y, dz = tz[t] - s.z;
                    const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
                    const float inv = rcp_approx(r2);
                    const float nr = fmaf(nx[t], dx, fmaf(ny[t], dy, nz[t] * dz));
                    const float mr = fmaf(mx[t], dx, fmaf(my[t], dy, mz[t] * dz));
                    const float inner = fmaf(nr, nr * inv, mr);
                    // inv * inner first: the self pair (r = 0, inner = 0) then adds an
                    // exact zero whatever the strength, where s.w * inv could overflow
                    part[t] = fmaf(s.w, inv * inner, part[t]);
                }
            }
#pragma unroll
            for (int t = 0; t < TPT; ++t) two_sum_acc(hi[t], lo[t], part[t]);
        }
    }
#pragma unroll
    for (int t = 0; t < TPT; ++t) {
        const int i = tbase + t * kThreads + tid;
        if (i < N) partial[(size_t)blockIdx.y * N + i] = make_float2(hi[t], lo[t]);
    }
}

// ------------------------------------------------------------------ float32 parametrix sum
// CENTRED: r^2 about a centre c of the block's targets (their mean).  With
// a = x_i - c and b = x_j - c, r^2 = |a|^2 + |b|^2 - 2 a.b; sources are staged as
// (-2b, s) and |b|^2, so a pair costs one add and three FMAs for r^2 (instead of
// three subtractions, a multiply and two FMAs), one MUFU lg2 and one FMA: about
// 6.5 issue slots a pair at 4 targets per thread, which leaves the MUFU rate
// (16 lg2 per clock per SM) as the bound.  Rounding: the cancellation costs up
// to ~8 eps R^2 in r^2 for a target tile of radius R, so a pair's log error is
// ~12 eps R^2 / r^2; summed with weights w_j ~ dA over the surface that is
// ~12 eps R^2 |sigma| int dA / r^2 ~ 75 eps R^2 log(R/h) |sigma| for node spacing h,
// against a sum of order |sigma| |Gamma|.  The surface takes this form only when
// every tile of 512 consecutive nodes has R^2 <= 0.03 |Gamma| (a relative error
// below ~1e-6 by that bound) and R^2 <= r_min^2 / (80 eps) for the smallest
// distance r_min between two nodes (r^2 stays positive and within 10 %); other
// surfaces (patches in scattered order) take the plain form, CENTRED = false.
// The self pair (in the centred form r^2 is a rounding residue, possibly
// negative) is replaced by zero by index before it is used.
template <int TPT, bool CENTRED>
__global__ void __launch_bounds__(kThreads)
k_direct_K32(const float4* __restrict__ src, const float4* __restrict__ tgt, int N, int chunk,
             float2* __restrict__ partial, const int* __restrict__ skip) {
    if (skip && *skip) return;
    __shared__ float4 sh[kStage];
    __shared__ float sb2[CENTRED ? kStage : 1];
    __shared__ float red[3][kThreads / 32];
    const int tid = threadIdx.x;
    const int tbase = blockIdx.x * kThreads * TPT;
    const int tend = tbase + kThreads * TPT;
    float tx[TPT], ty[TPT], tz[TPT], ta2[TPT], hi[TPT], lo[TPT];
    float cx = 0.f, cy = 0.f, cz = 0.f;
#pragma unroll
    for (int t = 0; t < TPT; ++t) {
        const int i = tbase + t * kThreads + tid;
        float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < N) {
            a = tgt[i];
            cx += a.x; cy += a.y; cz += a.z;
        }
        tx[t] = a.x; ty[t] = a.y; tz[t] = a.z;
        hi[t] = 0.f; lo[t] = 0.f;
    }
    if (CENTRED) {
        // centre: the mean of the block's targets (padding rows excluded)
        for (int o = 16; o > 0; o >>= 1) {
            cx += __shfl_xor_sync(0xffffffffu, cx, o);
            cy += __shfl_xor_sync(0xffffffffu, cy, o);
            cz += __shfl_xor_sync(0xffffffffu, cz, o);
        }
        if ((tid & 31) == 0) {
            red[0][tid >> 5] = cx;
            red[1][tid >> 5] = cy;
            red[2][tid >> 5] = cz;
        }
        __syncthreads();
        cx = cy = cz = 0.f;
#pragma unroll
        for (int w = 0; w < kThreads / 32; ++w) {
            cx += red[0][w];
            cy += red[1][w];
            cz += red[2][w];
        }
        const float inv_n = 1.0f / (float)min(kThreads * TPT, N - tbase);
        cx *= inv_n; cy *= inv_n; cz *= inv_n;
#pragma unroll
        for (int t = 0; t < TPT; ++t) {
            tx[t] -= cx; ty[t] -= cy; tz[t] -= cz;
            ta2[t] = fmaf(tx[t], tx[t], fmaf(ty[t], ty[t], tz[t] * tz[t]));
        }
    }
    // r^2 of target t and the staged source (s, b2)
    auto pair_r2 = [&](int t, const float4& s, float b2) -> float {
        if (CENTRED) return fmaf(tx[t], s.x, fmaf(ty[t], s.y, fmaf(tz[t], s.z, ta2[t] + b2)));
        const float dx = tx[t] - s.x, dy = ty[t] - s.y, dz = tz[t] - s.z;
        return fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    };
    const int s0 = blockIdx.y * chunk;
    const int s1 = min(s0 + chunk, N);
    for (int base = s0; base < s1; base += kStage) {
        const int len = min(kStage, s1 - base);
        __syncthreads();
        for (int j = tid; j < len; j += kThreads) {
            const float4 v = src[base + j];
            if (CENTRED) {
                const float bx = v.x - cx, by = v.y - cy, bz = v.z - cz;
                sh[j] = make_float4(-2.f * bx, -2.f * by, -2.f * bz, v.w);
                sb2[j] = fmaf(bx, bx, fmaf(by, by, bz * bz));
            } else {
                sh[j] = v;
            }
        }
        __syncthreads();
        for (int j0 = 0; j0 < len; j0 += kTile) {
            const int j1 = min(j0 + kTile, len);
            float part[TPT];
#pragma unroll
            for (int t = 0; t < TPT; ++t) part[t] = 0.f;
            // does this tile hold one of the block's own targets (j == i)?
            if (base + j1 <= tbase || base + j0 >= tend) {
#pragma unroll 4
                for (int j = j0; j < j1; ++j) {
                    const float4 s = sh[j];
                    const float b2 = CENTRED ? sb2[j] : 0.f;
#pragma unroll
                    for (int t = 0; t < TPT; ++t)
                        part[t] = fmaf(s.w, lg2_approx(pair_r2(t, s, b2)), part[t]);
                }
            } else {
                for (int j = j0; j < j1; ++j) {
                    const float4 s = sh[j];
                    const float b2 = CENTRED ? sb2[j] : 0.f;
#pragma unroll
                    for (int t = 0; t < TPT; ++t) {
                        const float r2 = pair_r2(t, s, b2);
                        const float l = (base + j == tbase + t * kThreads + tid) ? 0.f : lg2_approx(r2);
                        part[t] = fmaf(s.w, l, part[t]);
                    }
                }
            }
#pragma unroll
            for (int t = 0; t < TPT; ++t) two_sum_acc(hi[t], lo[t], part[t]);
        }
    }
    const float scale = (float)(M_LN2 / (4.0 * M_PI));
#pragma unroll
    for (int t = 0; t < TPT; ++t) {
        const int i = tbase + t * kThreads + tid;
        // scaling (hi, lo) by a float keeps the pair's relative accuracy
        if (i < N) partial[(size_t)blockIdx.y * N + i] = make_float2(hi[t] * scale, lo[t] * scale);
    }
}

// ------------------------------------------------------------------ float64 sums
constexpr int kTile64 = 128;

__global__ void __launch_bounds__(kThreads)
k_direct_64(const pm_d4* __restrict__ src, const double* __restrict__ x,
            const double* __restrict__ n, const double* __restrict__ H,
            const double* __restrict__ a, const double* __restrict__ g, int N, int Npad,
            int chunk, int kernel_K, double* __restrict__ partial, const int* __restrict__ skip) {
    if (skip && *skip) return;
    __shared__ pm_d4 sh[kTile64];
    const int tid = threadIdx.x;
    const int i = blockIdx.x * kThreads + tid;
    double tx = 0, ty = 0, tz = 0, nx = 0, ny = 0, nz = 0, mx = 0, my = 0, mz = 0;
    if (i < N) {
        tx = x[3 * i]; ty = x[3 * i + 1]; tz = x[3 * i + 2];
        const double c1 = sqrt(a[i] / M_PI), cH = -a[i] * H[i] / M_PI, c2 = 0.5 / M_PI;
        nx = c1 * n[3 * i]; ny = c1 * n[3 * i + 1]; nz = c1 * n[3 * i + 2];
        mx = cH * n[3 * i] + c2 * g[3 * i];
        my = cH * n[3 * i + 1] + c2 * g[3 * i + 1];
        mz = cH * n[3 * i + 2] + c2 * g[3 * i + 2];
    }
    double acc = 0.0;
    const int s0 = blockIdx.y * chunk;
    const int s1 = min(s0 + chunk, Npad);
    for (int base = s0; base < s1; base += kTile64) {
        __syncthreads();
        sh[tid] = src[base + tid];
        __syncthreads();
        for (int jj = 0; jj < kTile64; ++jj) {
            const int j = base + jj;
            const pm_d4 s = sh[jj];
            const double dx = tx - s.x, dy = ty - s.y, dz = tz - s.z;
            const double r2 = dx * dx + dy * dy + dz * dz;
            double term;
            if (kernel_K) {
                term = s.w * log(r2);
            } else {
                const double inv = 1.0 / r2;
                const double nr = nx * dx + ny * dy + nz * dz;
                const double mr = mx * dx + my * dy + mz * dz;
                term = s.w * inv * (nr * nr * inv + mr);
            }
            acc += (j == i || j >= N) ? 0.0 : term;
        }
    }
    if (i < N) partial[(size_t)blockIdx.y * N + i] = kernel_K ? acc / (4.0 * M_PI) : acc;
}

}  // namespace

// Targets per thread of the float32 sums: the knob when set, else 2 for the
// remainder (bound by its FP32 datapath, more targets only add registers) and
// 4 for the parametrix (bound by the MUFU rate, more targets per staged source
// take shared-memory reads off the issue slots the lg2s share).
static int direct_tpt(const pm_surface* s, int which_K) {
    const int t = s->opts.direct_tpt;
    return (t == 1 || t == 2 || t == 4) ? t : (which_K ? 4 : 2);
}

int pm_direct_splits(const pm_surface* s, pm_precision prec, int which_K) {
    const int per_block = (prec == PM_PREC_FP64) ? kThreads : kThreads * direct_tpt(s, which_K);
    const int tblocks = pm_ceil_div(s->N, per_block);
    int bps = s->opts.direct_blocks_per_sm;
    if (bps < 1 || bps > 16) bps = 12;
    const int want = bps * s->ctx->num_sms;
    int ns = (want + tblocks / 2) / tblocks;            // nearest split count
    ns = std::max(1, std::min(ns, std::min(s->max_split, std::max(1, s->N / 64))));
    return ns;
}

pm_status pm_pack_targets(pm_surface* s, cudaStream_t st) {
    const int N = s->N;
    const double far = 1e3 * (1.0 + s->scale) + 1e3 * s->h_far;
    k_pack<<<pm_ceil_div(s->Npad, 256), 256, 0, st>>>(s->x, s->n, s->H, s->a, s->g, s->w,
                                                       s->tgt32, s->src32, s->src64, s->wa, N,
                                                       s->Npad, far);
    PM_CUDA_TRY(cudaGetLastError());
    return PM_OK;
}

pm_status pm_prep_sources(pm_surface* s, const double* sigma, pm_precision prec,
                          cudaStream_t st) {
    const int N = s->N;
    if (prec == PM_PREC_FP64)
        k_prep64<<<pm_ceil_div(N, 256), 256, 0, st>>>(sigma, s->wa, s->src64, N, s->skip_flag);
    else
        k_prep32<<<pm_ceil_div(N, 256), 256, 0, st>>>(sigma, s->wa, s->src32, s->sig32, N,
                                                       s->pp, s->ppad, s->skip_flag);
    PM_CUDA_TRY(cudaGetLastError());
    return PM_OK;
}

pm_status pm_direct_sum(pm_surface* s, int which_K, pm_precision prec, int nsplit,
                        cudaStream_t st) {
    const int N = s->N;
    if (prec == PM_PREC_FP64) {
        const int chunk = pm_ceil_div(pm_ceil_div(s->Npad, nsplit), kTile64) * kTile64;
        dim3 grid(pm_ceil_div(N, kThreads), nsplit);
        k_direct_64<<<grid, kThreads, 0, st>>>(s->src64, s->x, s->n, s->H, s->a, s->g, N,
                                               s->Npad, chunk, which_K, s->partial,
                                               s->skip_flag);
    } else {
        const int tpt = direct_tpt(s, which_K);
        const int chunk = pm_ceil_div(N, nsplit);
        dim3 grid(pm_ceil_div(N, kThreads * tpt), nsplit);
        float2* part = reinterpret_cast<float2*>(s->partial);
#define PM_LAUNCH(T)                                                                        \
        if (which_K)                                                                        \
            (s->k32_centred ? k_direct_K32<T, true> : k_direct_K32<T, false>)               \
                <<<grid, kThreads, 0, st>>>(s->src32, s->tgt32, N, chunk, part, s->skip_flag); \
        else                                                                                \
            k_direct_R32<T><<<grid, kThreads, 0, st>>>(s->src32, s->tgt32, N, chunk,        \
                                                       s->eps2, part, s->skip_flag);
        if (tpt == 1) { PM_LAUNCH(1) } else if (tpt == 4) { PM_LAUNCH(4) } else { PM_LAUNCH(2) }
#undef PM_LAUNCH
    }
    PM_CUDA_TRY(cudaGetLastError());
    return PM_OK;
}

// ============================================================================ no-allocation variant
// Smooth remainder sum for callers that must not allocate device memory:
// everything the computation needs beyond the caller's inputs and output
// (packed float32 sources and targets, per-split partial sums) lives in one
// file-scope device array.  See pm_smooth_remainder_f32_noalloc in
// include/parametrix.h for the contract.
namespace {

constexpr int kNoAllocMaxN = 32768;
constexpr int kNoAllocSplits = 8;
constexpr size_t kNoAllocSrcBytes = sizeof(float4) * kNoAllocMaxN;
constexpr size_t kNoAllocTgtBytes = sizeof(float4) * 3 * kNoAllocMaxN;
constexpr size_t kNoAllocPartBytes = sizeof(float2) * kNoAllocSplits * kNoAllocMaxN;
constexpr size_t kNoAllocBytes = kNoAllocSrcBytes + kNoAllocTgtBytes + kNoAllocPartBytes;  // 4 MiB

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of g_noalloc_scratch per device, looked up once with that device current.
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[kNoAllocMaxDevices] = {};

__global__ void k_noalloc_pack(int N, const float* __restrict__ x, const float* __restrict__ n,
                               const float* __restrict__ H, const float* __restrict__ a,
                               const float* __restrict__ g, const float* __restrict__ s,
                               float4* __restrict__ src, float4* __restrict__ tgt) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float c1 = sqrtf(a[i] / (float)M_PI);
    const float cH = -a[i] * H[i] / (float)M_PI;
    const float c2 = 0.5f / (float)M_PI;
    tgt[i] = make_float4(x[3 * i], x[3 * i + 1], x[3 * i + 2], 0.f);
    tgt[N + i] = make_float4(c1 * n[3 * i], c1 * n[3 * i + 1], c1 * n[3 * i + 2], 0.f);
    tgt[2 * N + i] = make_float4(cH * n[3 * i] + c2 * g[3 * i], cH * n[3 * i + 1] + c2 * g[3 * i + 1],
                                 cH * n[3 * i + 2] + c2 * g[3 * i + 2], 0.f);
    src[i] = make_float4(x[3 * i], x[3 * i + 1], x[3 * i + 2], s[i]);
}

__global__ void k_noalloc_reduce(int N, int nsplit, const float2* __restrict__ partial,
                                 double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    float hi = 0.f, lo = 0.f;
    for (int sp = 0; sp < nsplit; ++sp) {
        const float2 v = partial[(size_t)sp * N + i];
        two_sum_acc(hi, lo, v.x);
        lo += v.y;
    }
    out[i] = (double)hi + (double)lo;
}

}  // namespace

extern "C" pm_status pm_smooth_remainder_f32_noalloc(int N, const float* x, const float* n,
                                                     const float* H, const float* a,
                                                     const float* grad_a, const float* s,
                                                     double* out, void* stream) {
    if (N < 1 || N > kNoAllocMaxN) {
        pm_set_error("pm_smooth_remainder_f32_noalloc: N = %d outside 1..%d (the size of the "
                     "library's static scratch)", N, kNoAllocMaxN);
        return PM_ERR_INVALID_ARG;
    }
    if (!x || !n || !H || !a || !grad_a || !s || !out) {
        pm_set_error("pm_smooth_remainder_f32_noalloc: NULL argument");
        return PM_ERR_INVALID_ARG;
    }
    int dev = 0;
    PM_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices) {
        pm_set_error("pm_smooth_remainder_f32_noalloc: device %d beyond %d", dev, kNoAllocMaxDevices);
        return PM_ERR_INVALID_ARG;
    }
    // the scratch's device address in the current context: looked up again on every
    // call made outside stream capture (cudaGetSymbolAddress allocates nothing), so a
    // context reset or another context on the device cannot leave a stale address;
    // during capture the address of the last uncaptured call on this device is used
    cudaStream_t st = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
        cudaGetLastError();
        cap = cudaStreamCaptureStatusActive;            // unknown: do not query the symbol
    }
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (cap == cudaStreamCaptureStatusNone) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                pm_set_error("pm_smooth_remainder_f32_noalloc: cudaGetSymbolAddress: %s",
                             cudaGetErrorString(e));
                return PM_ERR_CUDA;
            }
            g_noalloc_ptr[dev] = p;
        } else if (!g_noalloc_ptr[dev]) {
            pm_set_error("pm_smooth_remainder_f32_noalloc: the first call on device %d was made "
                         "during stream capture; make one call outside capture first", dev);
            return PM_ERR_INVALID_ARG;
        }
        base = g_noalloc_ptr[dev];
    }
    unsigned char* b = static_cast<unsigned char*>(base);
    float4* src = reinterpret_cast<float4*>(b);
    float4* tgt = reinterpret_cast<float4*>(b + kNoAllocSrcBytes);
    float2* part = reinterpret_cast<float2*>(b + kNoAllocSrcBytes + kNoAllocTgtBytes);
    // every (split, target < N) partial and every packed entry < N is written
    // before it is read, so nothing in the scratch needs clearing between calls
    int dev_sms = 0;
    PM_CUDA_TRY(cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, dev));
    const int tblocks = pm_ceil_div(N, kThreads * 2);
    int nsplit = (12 * dev_sms + tblocks / 2) / tblocks;
    nsplit = std::max(1, std::min(nsplit, std::min(kNoAllocSplits, std::max(1, N / 64))));
    const int chunk = pm_ceil_div(N, nsplit);
    k_noalloc_pack<<<pm_ceil_div(N, 256), 256, 0, st>>>(N, x, n, H, a, grad_a, s, src, tgt);
    dim3 grid(tblocks, nsplit);
    // self-pair guard: the j == i term is exactly zero (n'.r = m.r = 0, and the kernel
    // forms (1/r^2) * 0 before multiplying by the strength) while r^2 = 1e-30 keeps
    // 1/r^2 finite; 1e-30 is far below the squared distance of any two distinct nodes
    const float eps2 = 1e-30f;
    k_direct_R32<2><<<grid, kThreads, 0, st>>>(src, tgt, N, chunk, eps2, part, nullptr);
    k_noalloc_reduce<<<pm_ceil_div(N, 256), 256, 0, st>>>(N, nsplit, part, out);
    PM_CUDA_TRY(cudaGetLastError());
    return PM_OK;
}
