// Device-resident solve of the second-kind system (Sec. 3, Thm. second_kind).
#include "pm_internal.cuh"

pm_status pm_solve_impl(pm_surface* s, const double* f, double* u, double tol, int maxit,
                        pm_precision prec, unsigned flags, double* sigma_out,
                        pm_solve_info* info, cudaStream_t st) {
    (void)s; (void)f; (void)u; (void)tol; (void)maxit; (void)prec; (void)flags;
    (void)sigma_out; (void)info; (void)st;
    pm_set_error("pm_solve: not available in this build");
    return PM_ERR_INTERNAL;
}
