// Float-float (FP32-pair) smooth sums: float64-class accuracy on the FP32 pipe.
//
// GB300 executes float64 at a small fraction of its float32 rate, so the
// accurate remainder and parametrix sums used for true residuals and for the
// representation u = K~ sigma are evaluated in float-float arithmetic (every
// quantity an unevaluated sum hi + lo of two floats, about 48 significant
// bits; the arithmetic, the logarithm and the coordinate split are in
// pm_ff.cuh).  The table of ln c_k and 1/c_k for the logarithm is computed on
// the host in float64.
//
// Kernels mirror the float32 ones (pm_direct.cu): 128 threads, one target
// per thread, sources staged in shared memory, source chunks over gridDim.y,
// (hi, lo) partials combined by the float64 near-field kernel.  The self
// pair is excluded explicitly in the tile that holds the block's targets.
#include "pm_ff.cuh"
#include "pm_internal.cuh"

#include <algorithm>
#include <cmath>

namespace {

using namespace pmff;

constexpr int kThreads = 128;
constexpr int kStage = 512;        // sources per shared-memory stage (2 float4 each)

// -------------------------------------------------------------------- packing
// sources: src_ff[2j] = (xh, yh, zh, s_h), src_ff[2j+1] = (xl, yl, zl, s_l)
// targets: tg_ff[6i + 0..5] = x (hi, lo), n' (hi, lo), m (hi, lo), each (.x, .y, .z)
// parametrix sums: src_kg[2j], src_kg[2j+1] as src_ff with the coordinates
// split on the grid (pm_ff.cuh); targets read their coordinates from it too.
// The remainder sums keep plain float-float coordinates: its n' . r of nearby
// points cancels to O(r^2), where the grid split's absolute error would show.
__global__ void k_pack_ff(const double* __restrict__ x, const double* __restrict__ n,
                          const double* __restrict__ H, const double* __restrict__ a,
                          const double* __restrict__ g, double grid, float4* __restrict__ src,
                          float4* __restrict__ tg, float4* __restrict__ src_kg, int N) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    ff c[3][3], xg[3];
    const double c1 = sqrt(a[i] / M_PI), cH = -a[i] * H[i] / M_PI, c2 = 0.5 / M_PI;
    for (int d = 0; d < 3; ++d) {
        c[0][d] = ff_from_double(x[3 * i + d]);
        c[1][d] = ff_from_double(c1 * n[3 * i + d]);
        c[2][d] = ff_from_double(cH * n[3 * i + d] + c2 * g[3 * i + d]);
        xg[d] = ff_grid_split(x[3 * i + d], grid);
    }
    for (int q = 0; q < 3; ++q) {
        tg[6 * (size_t)i + 2 * q] = make_float4(c[q][0].h, c[q][1].h, c[q][2].h, 0.f);
        tg[6 * (size_t)i + 2 * q + 1] = make_float4(c[q][0].l, c[q][1].l, c[q][2].l, 0.f);
    }
    src[2 * (size_t)i] = make_float4(c[0][0].h, c[0][1].h, c[0][2].h, 0.f);
    src[2 * (size_t)i + 1] = make_float4(c[0][0].l, c[0][1].l, c[0][2].l, 0.f);
    src_kg[2 * (size_t)i] = make_float4(xg[0].h, xg[1].h, xg[2].h, 0.f);
    src_kg[2 * (size_t)i + 1] = make_float4(xg[0].l, xg[1].l, xg[2].l, 0.f);
}

__global__ void k_prep_ff(const double* __restrict__ sigma, const double* __restrict__ wa,
                          float4* __restrict__ src, float4* __restrict__ src_kg, int N,
                          const int* __restrict__ skip) {
    if (skip && *skip) return;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const ff s = ff_from_double(wa[j] * sigma[j]);
    src[2 * (size_t)j].w = s.h;
    src[2 * (size_t)j + 1].w = s.l;
    src_kg[2 * (size_t)j].w = s.h;
    src_kg[2 * (size_t)j + 1].w = s.l;
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
    if (KERNEL_K) {
        // src = grid-split coordinates; the target's own entry gives X
        const float4 a = (i < N) ? src[2 * (size_t)i] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 b = (i < N) ? src[2 * (size_t)i + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
        X[0] = ff{a.x, b.x}; X[1] = ff{a.y, b.y}; X[2] = ff{a.z, b.z};
    } else {
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
            const ff dx = KERNEL_K ? ff_grid_sub(X[0], A.x, B.x) : ff_sub(X[0], ff{A.x, B.x});
            const ff dy = KERNEL_K ? ff_grid_sub(X[1], A.y, B.y) : ff_sub(X[1], ff{A.y, B.y});
            const ff dz = KERNEL_K ? ff_grid_sub(X[2], A.z, B.z) : ff_sub(X[2], ff{A.z, B.z});
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
        PM_TRY(pm_dmalloc(&s->src_kg, 2 * (size_t)s->N));
    }
    return PM_OK;
}

// Grid of the coordinate split: 2^(E - 22) with 2^E >= max |x| (pm_ff.cuh), so a
// high word has at most 23 significant bits and two of them differ exactly.
double pm_ff_grid(const pm_surface* s) {
    int E = 0;
    const double f = std::frexp(std::max(s->h_far, 1e-300), &E);
    if (f == 0.5) E -= 1;                     // max |x| a power of two: 2^E = max |x|
    return std::ldexp(1.0, E - 22);
}

pm_status pm_pack_ff(pm_surface* s, cudaStream_t st) {
    PM_TRY(pm_ff_setup(s));
    k_pack_ff<<<pm_ceil_div(s->N, 256), 256, 0, st>>>(s->x, s->n, s->H, s->a, s->g,
                                                       pm_ff_grid(s), s->src_ff, s->tgt_ff, s->src_kg,
                                                       s->N);
    PM_CUDA_TRY(cudaGetLastError());
    return PM_OK;
}

pm_status pm_prep_ff(pm_surface* s, const double* sigma, cudaStream_t st) {
    k_prep_ff<<<pm_ceil_div(s->N, 256), 256, 0, st>>>(sigma, s->wa, s->src_ff, s->src_kg, s->N,
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
        k_direct_ff<true><<<grid, kThreads, 0, st>>>(s->src_kg, s->tgt_ff, s->log_tab, N, chunk,
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
