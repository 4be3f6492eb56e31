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
