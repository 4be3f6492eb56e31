// Float-float (FP32-pair) smooth sums: float64-class accuracy on the FP32 pipe.
//
// GB300 executes float64 at a small fraction of its float32 rate, so the
// accurate remainder and parametrix sums used for true residuals and for the
// representation u = K~ sigma are evaluated in float-float arithmetic: every
// quantity is an unevaluated sum hi + lo of two floats (about 48 significant
// bits).  The primitives are the error-free transformations TwoSum (Knuth)
// and TwoProduct via FMA, composed into the usual double-word add, multiply
// and reciprocal (one Newton step from the hardware reciprocal).
//
// The natural logarithm of a float-float number follows Tang's table-driven
// method ("Table-driven implementation of the logarithm function in IEEE
// floating-point arithmetic", ACM TOMS 16, 1990): x = 2^e m, m in [1, 2);
// m = c_k (1 + t) with c_k = 1 + (k + 1/2)/128 taken from the top seven
// mantissa bits, so |t| <= 2^-8; ln x = e ln 2 + ln c_k + ln(1 + t), with
// ln(1 + t) = t - t^2/2 + t^3 (1/3 - t/4 + t^2/5 - t^3/6) (truncation below
// 2^-56).  The table of ln c_k and 1/c_k is computed on the host in float64.
//
// Kernels mirror the float32 ones (pm_direct.cu): 128 threads, one target
// per thread, sources staged in shared memory, source chunks over gridDim.y,
// (hi, lo) partials combined by the float64 near-field kernel.  The self
// pair is excluded explicitly in the tile that holds the block's targets.
#include "pm_internal.cuh"

#include <algorithm>
#include <cmath>

namespace {

constexpr int kThreads = 128;
constexpr int kStage = 512;        // sources per shared-memory stage (2 float4 each)
constexpr int kLogTable = 128;

struct ff {
    float h, l;
};

__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    e = b - (s - a);
}

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
    const float p = a.h * b.h;
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    ff r;
    fast_two_sum(p, e, r.h, r.l);
    return r;
}

// Unnormalised variants: the low word may exceed half an ulp of the high word.
// Products of such pairs keep float-float accuracy only while the low word
// stays within a few ulps of the high word, so every sum that can cancel
// (differences, dot products, the bracket of the remainder term) is
// renormalised before it is multiplied; sums of positive terms (r^2) and the
// reciprocal and logarithm, whose low words stay small, are not.
__device__ __forceinline__ ff ff_mul_lazy(ff a, ff b) {
    const float p = a.h * b.h;
    float e = fmaf(a.h, b.h, -p);
    e = fmaf(a.h, b.l, e);
    e = fmaf(a.l, b.h, e);
    return ff{p, e};
}
__device__ __forceinline__ ff ff_sqr_lazy(ff a) {
    const float p = a.h * a.h;
    float e = fmaf(a.h, a.h, -p);
    e = fmaf(2.f * a.h, a.l, e);
    return ff{p, e};
}
__device__ __forceinline__ ff ff_add_lazy(ff a, ff b) {
    float s, e;
    two_sum(a.h, b.h, s, e);
    return ff{s, e + (a.l + b.l)};
}
__device__ __forceinline__ ff ff_norm(ff a) {
    ff r;
    fast_two_sum(a.h, a.l, r.h, r.l);
    return r;
}

// a - b, normalised: where the high words cancel the low word would otherwise
// be as large as the high word, and products with it would lose the l^2 term
__device__ __forceinline__ ff ff_sub(ff a, ff b) {
    float s, e;
    two_sum(a.h, -b.h, s, e);
    return ff_norm(ff{s, e + (a.l - b.l)});
}

// 1/a: y = rcp(a.h) and one Newton step y + y (1 - a y), the residual 1 - a y
// formed with the exact product a.h y = p + ep; returned unnormalised as (y, y res)
__device__ __forceinline__ ff ff_rcp_lazy(ff a) {
    const float y = rcp_approx(a.h);
    const float p = a.h * y;
    const float ep = fmaf(a.h, y, -p);
    const float res = ((1.f - p) - ep) - a.l * y;
    return ff{y, y * res};
}

// ln(x) for x = hi + lo > 0 (Tang's table method, see the file header):
// tab[k] = (1/c_k hi, 1/c_k lo, ln c_k hi, ln c_k lo).  The parts e ln 2,
// ln c_k, t and -t^2/2 + t^3 (...) are summed with error-free high words and
// plain low words; the result is left unnormalised.
__device__ __forceinline__ ff ff_log_lazy(ff x, const float4* __restrict__ tab) {
    int e;
    const float mh = frexpf(x.h, &e);
    const float sc = ldexpf(1.f, -e + 1);
    ff m{mh * 2.f, x.l * sc};
    e -= 1;
    const int k = (int)((m.h - 1.f) * (float)kLogTable);
    const float4 T = tab[min(max(k, 0), kLogTable - 1)];
    const ff p = ff_mul(m, ff{T.x, T.y});
    float th, tl;
    fast_two_sum(p.h - 1.f, p.l, th, tl);
    const ff t{th, tl};
    const ff t2 = ff_sqr_lazy(t);
    const float tf = t.h;
    const float poly = fmaf(fmaf(fmaf(-1.f / 6.f, tf, 0.2f), tf, -0.25f), tf, 1.f / 3.f);
    const float cubic = tf * tf * tf * poly;
    const float L2H = 0.693147182464599609375f;
    const float L2L = -1.904654323148236e-09f;
    const float ef = (float)e;
    const float eh = L2H * ef;
    const ff el{eh, fmaf(L2H, ef, -eh) + L2L * ef};    // e ln 2; the FMA recovers L2H e exactly
    ff r = ff_add_lazy(el, ff{T.z, T.w});
    r = ff_add_lazy(r, t);
    r = ff_add_lazy(r, ff{-0.5f * t2.h, fmaf(-0.5f, t2.l, cubic)});
    return r;
}

__device__ __forceinline__ ff ff_from_double(double v) {
    const float h = (float)v;
    return ff{h, (float)(v - (double)h)};
}

// -------------------------------------------------------------------- packing
// sources: src_ff[2j] = (xh, yh, zh, s_h), src_ff[2j+1] = (xl, yl, zl, s_l)
// targets: tg_ff[6i + 0..5] = x (hi, lo), n' (hi, lo), m (hi, lo), each (.x, .y, .z)
__global__ void k_pack_ff(const double* __restrict__ x, const double* __restrict__ n,
                          const double* __restrict__ H, const double* __restrict__ a,
                          const double* __restrict__ g, float4* __restrict__ src,
                          float4* __restrict__ tg, int N) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    ff c[3][3];
    const double c1 = sqrt(a[i] / M_PI), cH = -a[i] * H[i] / M_PI, c2 = 0.5 / M_PI;
    for (int d = 0; d < 3; ++d) {
        c[0][d] = ff_from_double(x[3 * i + d]);
        c[1][d] = ff_from_double(c1 * n[3 * i + d]);
        c[2][d] = ff_from_double(cH * n[3 * i + d] + c2 * g[3 * i + d]);
    }
    for (int q = 0; q < 3; ++q) {
        tg[6 * (size_t)i + 2 * q] = make_float4(c[q][0].h, c[q][1].h, c[q][2].h, 0.f);
        tg[6 * (size_t)i + 2 * q + 1] = make_float4(c[q][0].l, c[q][1].l, c[q][2].l, 0.f);
    }
    src[2 * (size_t)i] = make_float4(c[0][0].h, c[0][1].h, c[0][2].h, 0.f);
    src[2 * (size_t)i + 1] = make_float4(c[0][0].l, c[0][1].l, c[0][2].l, 0.f);
}

__global__ void k_prep_ff(const double* __restrict__ sigma, const double* __restrict__ wa,
                          float4* __restrict__ src, int N, const int* __restrict__ skip) {
    if (skip && *skip) return;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const ff s = ff_from_double(wa[j] * sigma[j]);
    src[2 * (size_t)j].w = s.h;
    src[2 * (size_t)j + 1].w = s.l;
}

// -------------------------------------------------------------------- sums
template <bool KERNEL_K>
__global__ void __launch_bounds__(kThreads)
k_direct_ff(const float4* __restrict__ src, const float4* __restrict__ tg,
            const float4* __restrict__ log_tab, int N, int chunk, float2* __restrict__ partial,
            const int* __restrict__ skip) {
    if (skip && *skip) return;
    __shared__ float4 sh[2 * kStage];
    __shared__ float4 stab[kLogTable];
    const int tid = threadIdx.x;
    const int i = blockIdx.x * kThreads + tid;
    const int tbase = blockIdx.x * kThreads, tend = tbase + kThreads;
    if (KERNEL_K)
        for (int k = tid; k < kLogTable; k += kThreads) stab[k] = log_tab[k];
    ff X[3], NP[3], MM[3];
    {
        float4 v[6];
        for (int q = 0; q < 6; ++q) v[q] = (i < N) ? tg[6 * (size_t)i + q] : make_float4(0.f, 0.f, 0.f, 0.f);
        X[0] = ff{v[0].x, v[1].x}; X[1] = ff{v[0].y, v[1].y}; X[2] = ff{v[0].z, v[1].z};
        NP[0] = ff{v[2].x, v[3].x}; NP[1] = ff{v[2].y, v[3].y}; NP[2] = ff{v[2].z, v[3].z};
        MM[0] = ff{v[4].x, v[5].x}; MM[1] = ff{v[4].y, v[5].y}; MM[2] = ff{v[4].z, v[5].z};
    }
    ff acc{0.f, 0.f};
    const int s0 = blockIdx.y * chunk;
    const int s1 = min(s0 + chunk, N);
    for (int base = s0; base < s1; base += kStage) {
        const int len = min(kStage, s1 - base);
        __syncthreads();
        for (int j = tid; j < 2 * len; j += kThreads) sh[j] = src[2 * (size_t)base + j];
        __syncthreads();
        const bool own = !(base + len <= tbase || base >= tend);
        for (int j = 0; j < len; ++j) {
            const float4 A = sh[2 * j], B = sh[2 * j + 1];
            if (own && base + j == i) continue;
            const ff dx = ff_sub(X[0], ff{A.x, B.x});
            const ff dy = ff_sub(X[1], ff{A.y, B.y});
            const ff dz = ff_sub(X[2], ff{A.z, B.z});
            const ff r2 = ff_add_lazy(ff_add_lazy(ff_sqr_lazy(dx), ff_sqr_lazy(dy)), ff_sqr_lazy(dz));
            const ff s{A.w, B.w};
            ff term;
            if (KERNEL_K) {
                term = ff_mul_lazy(s, ff_log_lazy(r2, stab));
            } else {
                const ff inv = ff_rcp_lazy(r2);
                const ff nr = ff_norm(ff_add_lazy(ff_add_lazy(ff_mul_lazy(NP[0], dx),
                                                              ff_mul_lazy(NP[1], dy)),
                                                  ff_mul_lazy(NP[2], dz)));
                const ff mr = ff_add_lazy(ff_add_lazy(ff_mul_lazy(MM[0], dx), ff_mul_lazy(MM[1], dy)),
                                          ff_mul_lazy(MM[2], dz));
                const ff q = ff_mul_lazy(nr, inv);
                const ff inner = ff_norm(ff_add_lazy(ff_mul_lazy(nr, q), mr));
                term = ff_mul_lazy(ff_mul_lazy(s, inv), inner);
            }
            // lazy accumulation: TwoSum on the high words, error terms in the low word
            const float t = acc.h + term.h;
            const float bp = t - acc.h;
            acc.l += ((acc.h - (t - bp)) + (term.h - bp)) + term.l;
            acc.h = t;
        }
    }
    if (i < N) {
        acc = ff_norm(acc);
        if (KERNEL_K) acc = ff_mul(acc, ff_from_double(1.0 / (4.0 * M_PI)));
        partial[(size_t)blockIdx.y * N + i] = make_float2(acc.h, acc.l);
    }
}

__global__ void k_fflog_test(const float* __restrict__ xh, const float* __restrict__ xl,
                             const float4* __restrict__ tab, int n, double* __restrict__ out) {
    __shared__ float4 stab[kLogTable];
    for (int k = threadIdx.x; k < kLogTable; k += blockDim.x) stab[k] = tab[k];
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const ff r = ff_norm(ff_log_lazy(ff{xh[i], xl[i]}, stab));
    out[i] = (double)r.h + (double)r.l;
}

}  // namespace

pm_status pm_ff_setup(pm_surface* s) {
    if (!s->log_tab) {
        float4 tab[kLogTable];
        for (int k = 0; k < kLogTable; ++k) {
            const double c = 1.0 + (k + 0.5) / kLogTable;
            const double ic = 1.0 / c, lc = std::log(c);
            const float ich = (float)ic, lch = (float)lc;
            tab[k] = make_float4(ich, (float)(ic - ich), lch, (float)(lc - lch));
        }
        PM_TRY(pm_dmalloc(&s->log_tab, kLogTable));
        PM_CUDA_TRY(cudaMemcpy(s->log_tab, tab, sizeof(tab), cudaMemcpyHostToDevice));
    }
    if (!s->src_ff) {
        PM_TRY(pm_dmalloc(&s->src_ff, 2 * (size_t)s->N));
        PM_TRY(pm_dmalloc(&s->tgt_ff, 6 * (size_t)s->N));
    }
    return PM_OK;
}

pm_status pm_pack_ff(pm_surface* s, cudaStream_t st) {
    PM_TRY(pm_ff_setup(s));
    k_pack_ff<<<pm_ceil_div(s->N, 256), 256, 0, st>>>(s->x, s->n, s->H, s->a, s->g, s->src_ff,
                                                       s->tgt_ff, s->N);
    PM_CUDA_TRY(cudaGetLastError());
    return PM_OK;
}

pm_status pm_prep_ff(pm_surface* s, const double* sigma, cudaStream_t st) {
    k_prep_ff<<<pm_ceil_div(s->N, 256), 256, 0, st>>>(sigma, s->wa, s->src_ff, s->N,
                                                       s->skip_flag);
    PM_CUDA_TRY(cudaGetLastError());
    return PM_OK;
}

int pm_ff_splits(const pm_surface* s) {
    const int tblocks = pm_ceil_div(s->N, kThreads);
    const int want = 8 * s->ctx->num_sms;
    int ns = (want + tblocks / 2) / tblocks;
    return std::max(1, std::min(ns, std::min(s->max_split, std::max(1, s->N / 64))));
}

pm_status pm_direct_ff(pm_surface* s, int which_K, int nsplit, cudaStream_t st) {
    const int N = s->N;
    const int chunk = pm_ceil_div(N, nsplit);
    dim3 grid(pm_ceil_div(N, kThreads), nsplit);
    float2* part = reinterpret_cast<float2*>(s->partial);
    if (which_K)
        k_direct_ff<true><<<grid, kThreads, 0, st>>>(s->src_ff, s->tgt_ff, s->log_tab, N, chunk,
                                                     part, s->skip_flag);
    else
        k_direct_ff<false><<<grid, kThreads, 0, st>>>(s->src_ff, s->tgt_ff, s->log_tab, N, chunk,
                                                      part, s->skip_flag);
    PM_CUDA_TRY(cudaGetLastError());
    return PM_OK;
}

extern "C" pm_status pm_selftest_fflog(pm_surface* s, const float* xh, const float* xl, int n,
                                       double* out) {
    if (!s || !xh || !xl || !out || n < 1) {
        pm_set_error("pm_selftest_fflog: NULL argument or n < 1");
        return PM_ERR_INVALID_ARG;
    }
    PM_CUDA_TRY(cudaSetDevice(s->ctx->device));
    PM_TRY(pm_ff_setup(s));
    float *dh = nullptr, *dl = nullptr;
    double* dout = nullptr;
    PM_TRY(pm_dmalloc(&dh, n));
    PM_TRY(pm_dmalloc(&dl, n));
    PM_TRY(pm_dmalloc(&dout, n));
    cudaMemcpy(dh, xh, sizeof(float) * n, cudaMemcpyHostToDevice);
    cudaMemcpy(dl, xl, sizeof(float) * n, cudaMemcpyHostToDevice);
    k_fflog_test<<<pm_ceil_div(n, 256), 256>>>(dh, dl, s->log_tab, n, dout);
    cudaError_t e = cudaMemcpy(out, dout, sizeof(double) * n, cudaMemcpyDeviceToHost);
    cudaFree(dh);
    cudaFree(dl);
    cudaFree(dout);
    if (e != cudaSuccess) {
        pm_set_error("pm_selftest_fflog: %s", cudaGetErrorString(e));
        return PM_ERR_CUDA;
    }
    return PM_OK;
}
