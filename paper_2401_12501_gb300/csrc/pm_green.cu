// Host entry point of the c != 0 Green's function evaluators (pm_green.cuh):
// lets the host-side tests compare the library's own g, g', g'' with an
// independent evaluation before any device kernel uses them.

#include "pm_internal.cuh"
#include "pm_green.cuh"

#include <cmath>

extern "C" pm_status pm_selftest_green(const double* r, int n, double q, double* out) {
    if (!r || !out || n < 0 || !std::isfinite(q) || q == 0.0) {
        pm_set_error("pm_selftest_green: NULL array, negative n, or q not finite and non-zero");
        return PM_ERR_INVALID_ARG;
    }
    for (int i = 0; i < n; ++i)
        if (!(r[i] > 0.0) || !std::isfinite(r[i])) {
            pm_set_error("pm_selftest_green: r must be finite and positive");
            return PM_ERR_INVALID_ARG;
        }
    for (int i = 0; i < n; ++i) pm_green::green_scaled(r[i], q, out + 6 * i);
    return PM_OK;
}

extern "C" pm_status pm_selftest_green_c(const double* r, int n, double q_re, double q_im,
                                         double* out) {
    if (!r || !out || n < 0 || !std::isfinite(q_re) || !std::isfinite(q_im) ||
        (q_re == 0.0 && q_im == 0.0)) {
        pm_set_error("pm_selftest_green_c: NULL array, negative n, or q not finite and non-zero");
        return PM_ERR_INVALID_ARG;
    }
    for (int i = 0; i < n; ++i)
        if (!(r[i] > 0.0) || !std::isfinite(r[i])) {
            pm_set_error("pm_selftest_green_c: r must be finite and positive");
            return PM_ERR_INVALID_ARG;
        }
    QuadTables T;
    pm_build_tables(2, &T);
    for (int i = 0; i < n; ++i) {
        if (q_im == 0.0)
            pm_green::green_scaled(r[i], q_re, out + 6 * i);
        else
            pm_green::green_scaled_cz(r[i], pm_green::cplx_d{q_re, q_im}, T.g16t, T.g16w, out + 6 * i);
    }
    return PM_OK;
}

extern "C" pm_status pm_selftest_green_f32(const float* r, int n, float q, float* out) {
    if (!r || !out || n < 0 || !std::isfinite(q) || q == 0.0f) {
        pm_set_error("pm_selftest_green_f32: NULL array, negative n, or q not finite and non-zero");
        return PM_ERR_INVALID_ARG;
    }
    for (int i = 0; i < n; ++i)
        if (!(r[i] > 0.0f) || !std::isfinite(r[i])) {
            pm_set_error("pm_selftest_green_f32: r must be finite and positive");
            return PM_ERR_INVALID_ARG;
        }
    for (int i = 0; i < n; ++i) pm_green::green_scaled_f32(r[i], q, out + 6 * i);
    return PM_OK;
}

extern "C" pm_status pm_selftest_smooth_c_f32(int N, const float* x, const float* n,
                                              const float* H, const float* a, const float* gb,
                                              const float* c, const float* s, double* out) {
    if (N < 0 || !x || !n || !H || !a || !gb || !c || !s || !out) {
        pm_set_error("pm_selftest_smooth_c_f32: NULL array or negative N");
        return PM_ERR_INVALID_ARG;
    }
    for (int i = 0; i < N; ++i)
        if (!(a[i] > 0.0f) || !std::isfinite(c[i]) || c[i] == 0.0f) {
            pm_set_error("pm_selftest_smooth_c_f32: a must be positive and c finite and non-zero");
            return PM_ERR_INVALID_ARG;
        }
    for (int i = 0; i < N; ++i) {
        double sum[4] = {0.0, 0.0, 0.0, 0.0};
        for (int j = 0; j < N; ++j) {
            if (j == i) continue;
            float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            pm_green::pair_rk_c_f32(x[3 * i] - x[3 * j], x[3 * i + 1] - x[3 * j + 1],
                                    x[3 * i + 2] - x[3 * j + 2], n[3 * i], n[3 * i + 1],
                                    n[3 * i + 2], H[i], a[i], gb[3 * i], gb[3 * i + 1],
                                    gb[3 * i + 2], c[i], c[j] / a[j], s[2 * j], s[2 * j + 1],
                                    acc);
            for (int m = 0; m < 4; ++m) sum[m] += acc[m];
        }
        for (int m = 0; m < 4; ++m) out[4 * i + m] = sum[m];
    }
    return PM_OK;
}

// ------------------------------------------------------------------ device smooth sums, c != 0
// One thread per target; sources (x, y, z, q = c/a) and s = w sigma / a staged
// through shared memory in stages of kCStage; every kCTile sources the partial
// is folded into a (hi, lo) pair with TwoSum, as in the c = 0 float32 sums.  The
// self pair j = i is skipped by index (the Hankel kernels have no removable
// value at r = 0).  Threads past N compute on a dummy target and write nothing.
namespace {

constexpr int kCThreads = 128;
constexpr int kCStage = 512;
constexpr int kCTile = 128;

__device__ __forceinline__ void two_sum_c(float& hi, float& lo, float v) {
    const float t = hi + v;
    const float bp = t - hi;
    lo += (hi - (t - bp)) + (v - bp);
    hi = t;
}

__global__ void __launch_bounds__(kCThreads)
k_smooth_c32(int N, const float* __restrict__ x, const float* __restrict__ n,
             const float* __restrict__ H, const float* __restrict__ a,
             const float* __restrict__ gb, const float* __restrict__ c,
             const float* __restrict__ s, double* __restrict__ out) {
    __shared__ float4 sp[kCStage];
    __shared__ float2 ss[kCStage];
    const int i = blockIdx.x * kCThreads + threadIdx.x;
    const bool live = i < N;
    float tx = 0.f, ty = 0.f, tz = 0.f, nx = 0.f, ny = 0.f, nz = 0.f, Hi = 0.f, ai = 1.f,
          gx = 0.f, gy = 0.f, gz = 0.f, ci = 0.f;
    if (live) {
        tx = x[3 * i]; ty = x[3 * i + 1]; tz = x[3 * i + 2];
        nx = n[3 * i]; ny = n[3 * i + 1]; nz = n[3 * i + 2];
        Hi = H[i]; ai = a[i]; ci = c[i];
        gx = gb[3 * i]; gy = gb[3 * i + 1]; gz = gb[3 * i + 2];
    }
    float hi[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};
    for (int base = 0; base < N; base += kCStage) {
        const int len = min(kCStage, N - base);
        __syncthreads();
        for (int j = threadIdx.x; j < len; j += kCThreads) {
            const int g = base + j;
            sp[j] = make_float4(x[3 * g], x[3 * g + 1], x[3 * g + 2], c[g] / a[g]);
            ss[j] = make_float2(s[2 * g], s[2 * g + 1]);
        }
        __syncthreads();
        for (int j0 = 0; j0 < len; j0 += kCTile) {
            const int j1 = min(j0 + kCTile, len);
            float part[4] = {0.f, 0.f, 0.f, 0.f};
            for (int j = j0; j < j1; ++j) {
                if (base + j == i) continue;
                const float4 p = sp[j];
                const float2 w = ss[j];
                pm_green::pair_rk_c_f32(tx - p.x, ty - p.y, tz - p.z, nx, ny, nz, Hi, ai, gx,
                                        gy, gz, ci, p.w, w.x, w.y, part);
            }
#pragma unroll
            for (int m = 0; m < 4; ++m) two_sum_c(hi[m], lo[m], part[m]);
        }
    }
    if (live) {
#pragma unroll
        for (int m = 0; m < 4; ++m) out[4 * (size_t)i + m] = (double)hi[m] + (double)lo[m];
    }
}

constexpr int kSmoothCMaxN = 1 << 26;

}  // namespace

extern "C" pm_status pm_smooth_c_f32(int N, const float* x, const float* n, const float* H,
                                     const float* a, const float* gb, const float* c,
                                     const float* s, double* out, void* stream) {
    if (N < 1 || N > kSmoothCMaxN) {
        pm_set_error("pm_smooth_c_f32: N = %d outside 1..%d", N, kSmoothCMaxN);
        return PM_ERR_INVALID_ARG;
    }
    if (!x || !n || !H || !a || !gb || !c || !s || !out) {
        pm_set_error("pm_smooth_c_f32: NULL argument");
        return PM_ERR_INVALID_ARG;
    }
    const int grid = (N + kCThreads - 1) / kCThreads;
    k_smooth_c32<<<grid, kCThreads, 0, (cudaStream_t)stream>>>(N, x, n, H, a, gb, c, s, out);
    PM_CUDA_TRY(cudaGetLastError());
    return PM_OK;
}
