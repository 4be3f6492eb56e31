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
