// Device-resident solve of the second-kind system (Sec. 3, Thm. second_kind).
//
//   A sigma = sigma + R~ sigma + (sum_j w_j sigma_j) 1     (rank-one null-space removal, Sec. 3)
//   u = K~ sigma - (sum w K~ sigma)/(sum w)               (eq. representation, mean-zero u)
//
// Mixed precision with iterative refinement: the true residual r = f - A sigma
// is formed with float64 applies; each correction A delta = r is solved by
// restarted GMRES (Saad and Schultz) whose operator applies run in the
// requested precision (float32 smooth sums and near field) while the Krylov
// basis, the Arnoldi orthogonalisation (classical Gram-Schmidt, applied twice),
// the Hessenberg Givens rotations and the least-squares update stay float64.
//
// No host round-trip per Arnoldi step: every kernel of a cycle takes a device
// "done" flag that the rotation kernel sets once the residual estimate meets
// the tolerance (or the Arnoldi vector vanishes); later kernels of the cycle
// return immediately.  The host synchronises once per cycle.
#include "pm_internal.cuh"

#include <chrono>
#include <cmath>
#include <vector>

namespace {

constexpr int kRedThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Block-wide sum; result valid in thread 0.
__device__ double block_sum(double v, double* sh) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double t = 0.0;
    if (wid == 0) {
        t = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
        t = warp_sum(t);
    }
    return t;
}

// partial[blk * ncols + j] = sum_{i in block's rows} A_j[i] * b[i], A_j = A + j*lda
__global__ void __launch_bounds__(kRedThreads)
k_multidot(const double* __restrict__ A, long long lda, int ncols, const double* __restrict__ b,
           int N, double* __restrict__ partial, const int* __restrict__ done) {
    if (done && *done) return;
    __shared__ double sh[32];
    const int stride = gridDim.x * blockDim.x;
    for (int j = 0; j < ncols; ++j) {
        const double* a = A + j * lda;
        double acc = 0.0;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) acc += a[i] * b[i];
        acc = block_sum(acc, sh);
        if (threadIdx.x == 0) partial[blockIdx.x * ncols + j] = acc;
    }
}

// out[j] = (accumulate ? out[j] : 0) + sign * sum_blk partial[blk * ncols + j]  (fixed order)
__global__ void k_reduce_cols(const double* __restrict__ partial, int nblk, int ncols,
                              double* __restrict__ out, const int* __restrict__ done) {
    if (done && *done) return;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ncols) return;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += partial[b * ncols + j];
    out[j] = s;
}

// w -= sum_j A_j * c[j]
__global__ void k_sub_combo(const double* __restrict__ A, long long lda, int ncols,
                            const double* __restrict__ c, double* __restrict__ w, int N,
                            const int* __restrict__ done) {
    if (done && *done) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double acc = w[i];
    for (int j = 0; j < ncols; ++j) acc -= A[j * lda + i] * c[j];
    w[i] = acc;
}

// out = v + y + scal[0] (the rank-one term sum_j w_j v_j)
__global__ void k_apply_A_finish(const double* __restrict__ v, const double* __restrict__ y,
                                 const double* __restrict__ wdot, double* __restrict__ out, int N,
                                 const int* __restrict__ done) {
    if (done && *done) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    out[i] = v[i] + y[i] + *wdot;
}

// r = b - Ax
__global__ void k_residual_from(const double* __restrict__ b, const double* __restrict__ Ax,
                                double* __restrict__ r, int N) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) r[i] = b[i] - Ax[i];
}

// h[j] += h2[j], j < n
__global__ void k_add_cols(double* __restrict__ h, const double* __restrict__ h2, int n,
                           const int* __restrict__ done) {
    if (done && *done) return;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) h[j] += h2[j];
}

__global__ void k_scale_copy(const double* __restrict__ src, const double* __restrict__ s,
                             int invert, double* __restrict__ dst, int N,
                             const int* __restrict__ done) {
    if (done && *done) return;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double f = invert ? 1.0 / *s : *s;
    dst[i] = src[i] * f;
}

__global__ void k_mul(const double* __restrict__ a, const double* __restrict__ b,
                      double* __restrict__ out, int N) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) out[i] = a[i] * b[i];
}

__global__ void k_axpy(double* __restrict__ y, const double* __restrict__ x, double a, int N) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) y[i] += a * x[i];
}

__global__ void k_add_shift(double* __restrict__ y, const double* __restrict__ shift, double sgn,
                            int N) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) y[i] += sgn * *shift;
}

// Start of a cycle: beta = sqrt(nrm2), g = (beta, 0, ...), v0 = r / beta.
__global__ void k_cycle_start(const double* __restrict__ nrm2, double* __restrict__ g, int m,
                              double* __restrict__ scal, double tol_abs, int* __restrict__ done,
                              int* __restrict__ iters) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const double beta = sqrt(*nrm2);
    for (int k = 0; k <= m; ++k) g[k] = 0.0;
    g[0] = beta;
    scal[3] = beta;
    *iters = 0;
    *done = (beta <= tol_abs || beta == 0.0) ? 1 : 0;
}

// Arnoldi step k finished its orthogonalisation: column h[0..k] and the
// squared norm of the new vector are in place.  Apply the previous Givens
// rotations, form the new one, update g, test convergence.
__global__ void k_arnoldi_rotate(double* __restrict__ H, int ldh, int k, double* __restrict__ cs,
                                 double* __restrict__ sn, double* __restrict__ g,
                                 const double* __restrict__ nrm2, double* __restrict__ scal,
                                 double tol_abs, int* __restrict__ done, int* __restrict__ iters) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (*done) return;
    double* h = H + (size_t)k * ldh;    // column k, entries 0..k+1
    const double hn = sqrt(*nrm2);
    h[k + 1] = hn;
    scal[2] = (hn > 0.0) ? 1.0 / hn : 0.0;
    for (int j = 0; j < k; ++j) {
        const double t = cs[j] * h[j] + sn[j] * h[j + 1];
        h[j + 1] = -sn[j] * h[j] + cs[j] * h[j + 1];
        h[j] = t;
    }
    const double a = h[k], b = h[k + 1];
    const double den = hypot(a, b);
    const double c = (den > 0.0) ? a / den : 1.0, s_ = (den > 0.0) ? b / den : 0.0;
    cs[k] = c;
    sn[k] = s_;
    h[k] = den;
    h[k + 1] = 0.0;
    g[k + 1] = -s_ * g[k];
    g[k] = c * g[k];
    *iters = k + 1;
    // breakdown (hn tiny) means the Krylov space is invariant: the LS solution is exact
    if (fabs(g[k + 1]) <= tol_abs || hn <= 1e-300 || !(hn == hn)) *done = 1;
}

// y = H(0:n,0:n)^{-1} g(0:n) by back substitution, n = *iters
__global__ void k_backsolve(const double* __restrict__ H, int ldh, const double* __restrict__ g,
                            const int* __restrict__ iters, double* __restrict__ y) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int n = *iters;
    for (int i = n - 1; i >= 0; --i) {
        double t = g[i];
        for (int j = i + 1; j < n; ++j) t -= H[(size_t)j * ldh + i] * y[j];
        const double d = H[(size_t)i * ldh + i];
        y[i] = (d != 0.0) ? t / d : 0.0;
    }
}

// x += sum_{j < *iters} V_j y_j
__global__ void k_add_combo(const double* __restrict__ V, long long ldv,
                            const int* __restrict__ iters, const double* __restrict__ y,
                            double* __restrict__ x, int N) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int n = *iters;
    double acc = x[i];
    for (int j = 0; j < n; ++j) acc += V[j * ldv + i] * y[j];
    x[i] = acc;
}

struct Work {
    int N = 0, m = 0, nred = 0;
    double *V = nullptr, *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr, *y = nullptr;
    double *part = nullptr, *scal = nullptr, *hcol = nullptr;
    double *w = nullptr, *tmp = nullptr, *r = nullptr, *res = nullptr, *delta = nullptr;
    double *sig = nullptr, *f = nullptr, *u = nullptr;
    int *done = nullptr, *iters = nullptr;
    double* pinned = nullptr;   // host-pinned scalars read back per cycle
    int* pinned_i = nullptr;
};

}  // namespace

struct PmSolveWork : Work {};

void pm_solve_free(pm_surface* s) {
    if (!s->solve_work) return;
    Work& W = *s->solve_work;
    pm_dfree(W.V); pm_dfree(W.H); pm_dfree(W.cs); pm_dfree(W.sn); pm_dfree(W.g); pm_dfree(W.y);
    pm_dfree(W.part); pm_dfree(W.scal); pm_dfree(W.hcol); pm_dfree(W.w); pm_dfree(W.tmp);
    pm_dfree(W.r); pm_dfree(W.res); pm_dfree(W.delta); pm_dfree(W.sig); pm_dfree(W.f);
    pm_dfree(W.u); pm_dfree(W.done); pm_dfree(W.iters);
    if (W.pinned) cudaFreeHost(W.pinned);
    if (W.pinned_i) cudaFreeHost(W.pinned_i);
    delete s->solve_work;
    s->solve_work = nullptr;
}

namespace {

pm_status get_work(pm_surface* s, Work** out) {
    const int m = std::max(2, std::min(s->opts.gmres_restart, 400));
    if (s->solve_work && s->solve_work->m == m) {
        *out = s->solve_work;
        return PM_OK;
    }
    pm_solve_free(s);
    s->solve_work = new PmSolveWork();
    Work& W = *s->solve_work;
    const int N = s->N;
    W.N = N;
    W.m = m;
    W.nred = std::max(1, std::min(pm_ceil_div(N, 1024), 2 * s->ctx->num_sms));
    PM_TRY(pm_dmalloc(&W.V, (size_t)(m + 1) * N));
    PM_TRY(pm_dmalloc(&W.H, (size_t)m * (m + 2)));
    PM_TRY(pm_dmalloc(&W.cs, m));
    PM_TRY(pm_dmalloc(&W.sn, m));
    PM_TRY(pm_dmalloc(&W.g, m + 1));
    PM_TRY(pm_dmalloc(&W.y, m));
    PM_TRY(pm_dmalloc(&W.part, (size_t)W.nred * (m + 2)));
    PM_TRY(pm_dmalloc(&W.scal, 8));
    PM_TRY(pm_dmalloc(&W.hcol, m + 2));
    PM_TRY(pm_dmalloc(&W.w, N));
    PM_TRY(pm_dmalloc(&W.tmp, N));
    PM_TRY(pm_dmalloc(&W.r, N));
    PM_TRY(pm_dmalloc(&W.res, N));
    PM_TRY(pm_dmalloc(&W.delta, N));
    PM_TRY(pm_dmalloc(&W.sig, N));
    PM_TRY(pm_dmalloc(&W.f, N));
    PM_TRY(pm_dmalloc(&W.u, N));
    PM_TRY(pm_dmalloc(&W.done, 1));
    PM_TRY(pm_dmalloc(&W.iters, 1));
    PM_CUDA_TRY(cudaMallocHost((void**)&W.pinned, 8 * sizeof(double)));
    PM_CUDA_TRY(cudaMallocHost((void**)&W.pinned_i, 4 * sizeof(int)));
    *out = &W;
    return PM_OK;
}

struct Solver {
    pm_surface* s;
    Work& W;
    cudaStream_t st;
    int grid_n;

    pm_precision residual_prec() const {
        return s->opts.residual_prec == PM_PREC_FP64 ? PM_PREC_FP64 : PM_PREC_FF;
    }

    // dst[0..ncols) = columns(A) . b (deterministic two-pass reduction)
    pm_status dots(const double* A, long long lda, int ncols, const double* b, double* dst,
                   const int* done) {
        k_multidot<<<W.nred, kRedThreads, 0, st>>>(A, lda, ncols, b, W.N, W.part, done);
        s->launch_total++;
        k_reduce_cols<<<pm_ceil_div(ncols, 64), 64, 0, st>>>(W.part, W.nred, ncols, dst, done);
        s->launch_total++;
        PM_CUDA_TRY(cudaGetLastError());
        return PM_OK;
    }

    // out = A v = v + R~ v + (w . v) 1 in the given precision
    pm_status apply_A(const double* v, double* out, pm_precision prec, const int* done) {
        PM_TRY(pm_apply_dev(s, 0, 1, 1, v, W.tmp, prec, st));
        PM_TRY(dots(s->w, 0, 1, v, W.scal + 0, done));
        k_apply_A_finish<<<grid_n, 256, 0, st>>>(v, W.tmp, W.scal + 0, out, W.N, done);
        s->launch_total++;
        PM_CUDA_TRY(cudaGetLastError());
        return PM_OK;
    }

    pm_status read_scalar(const double* d, double* h) {
        PM_CUDA_TRY(cudaMemcpyAsync(W.pinned, d, sizeof(double), cudaMemcpyDeviceToHost, st));
        PM_CUDA_TRY(cudaStreamSynchronize(st));
        *h = W.pinned[0];
        return PM_OK;
    }

    pm_status norm2(const double* v, double* h) {
        PM_TRY(dots(v, 0, 1, v, W.scal + 1, nullptr));
        double t = 0;
        PM_TRY(read_scalar(W.scal + 1, &t));
        *h = std::sqrt(t);
        return PM_OK;
    }

    // Restarted GMRES(m) for A d = b from d = 0 with the operator in `prec`,
    // stopping when the residual estimate is below tol_abs; x += d.
    pm_status gmres(const double* b, double* x, pm_precision prec, double tol_abs, int max_iter,
                    int* iters_used) {
        const int m = W.m;
        const long long ldv = W.N;
        int total = 0;
        PM_CUDA_TRY(cudaMemcpyAsync(W.r, b, sizeof(double) * W.N, cudaMemcpyDeviceToDevice, st));
        PM_CUDA_TRY(cudaMemsetAsync(W.delta, 0, sizeof(double) * W.N, st));
        while (total < max_iter) {
            PM_TRY(dots(W.r, 0, 1, W.r, W.scal + 1, nullptr));
            k_cycle_start<<<1, 1, 0, st>>>(W.scal + 1, W.g, m, W.scal, tol_abs, W.done, W.iters);
            s->launch_total++;
            k_scale_copy<<<grid_n, 256, 0, st>>>(W.r, W.scal + 3, 1, W.V, W.N, W.done);
            s->launch_total++;
            const int steps = std::min(m, max_iter - total);
            s->skip_flag = W.done;
            // launch the cycle in chunks; between chunks read the done flag so a
            // converged cycle stops launching (kernels after convergence no-op)
            const int chunk = (steps <= 8) ? steps : 4;
            for (int k = 0; k < steps; ++k) {
                if (k > 0 && k % chunk == 0) {
                    cudaError_t ce = cudaMemcpyAsync(W.pinned_i + 2, W.done, sizeof(int),
                                                     cudaMemcpyDeviceToHost, st);
                    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
                    if (ce != cudaSuccess) {
                        s->skip_flag = nullptr;
                        pm_set_error("gmres: %s", cudaGetErrorString(ce));
                        return PM_ERR_CUDA;
                    }
                    if (W.pinned_i[2]) break;
                }
                double* vk = W.V + (size_t)k * ldv;
                double* vk1 = W.V + (size_t)(k + 1) * ldv;
                double* hk = W.H + (size_t)k * (m + 2);
                pm_status stt = apply_A(vk, W.w, prec, W.done);
                if (stt != PM_OK) { s->skip_flag = nullptr; return stt; }
                // classical Gram-Schmidt, applied twice
                dots(W.V, ldv, k + 1, W.w, hk, W.done);
                k_sub_combo<<<grid_n, 256, 0, st>>>(W.V, ldv, k + 1, hk, W.w, W.N, W.done);
                s->launch_total++;
                dots(W.V, ldv, k + 1, W.w, W.hcol, W.done);
                k_sub_combo<<<grid_n, 256, 0, st>>>(W.V, ldv, k + 1, W.hcol, W.w, W.N, W.done);
                s->launch_total++;
                k_add_cols<<<pm_ceil_div(k + 1, 64), 64, 0, st>>>(hk, W.hcol, k + 1, W.done);
                s->launch_total++;
                dots(W.w, 0, 1, W.w, W.scal + 1, W.done);
                k_arnoldi_rotate<<<1, 1, 0, st>>>(W.H, m + 2, k, W.cs, W.sn, W.g, W.scal + 1,
                                                  W.scal, tol_abs, W.done, W.iters);
                s->launch_total++;
                k_scale_copy<<<grid_n, 256, 0, st>>>(W.w, W.scal + 2, 0, vk1, W.N, W.done);
                s->launch_total++;
            }
            s->skip_flag = nullptr;
            PM_CUDA_TRY(cudaGetLastError());
            k_backsolve<<<1, 1, 0, st>>>(W.H, m + 2, W.g, W.iters, W.y);
            s->launch_total++;
            k_add_combo<<<grid_n, 256, 0, st>>>(W.V, ldv, W.iters, W.y, W.delta, W.N);
            s->launch_total++;
            PM_CUDA_TRY(cudaMemcpyAsync(W.pinned_i, W.iters, sizeof(int), cudaMemcpyDeviceToHost, st));
            PM_CUDA_TRY(cudaMemcpyAsync(W.pinned_i + 1, W.done, sizeof(int), cudaMemcpyDeviceToHost, st));
            PM_CUDA_TRY(cudaStreamSynchronize(st));
            const int it = W.pinned_i[0];
            const int converged = W.pinned_i[1];
            total += it;
            if (converged || it == 0) break;
            // cycle exhausted: restart from the residual of the operator in use
            PM_TRY(apply_A(W.delta, W.w, prec, nullptr));
            k_residual_from<<<grid_n, 256, 0, st>>>(b, W.w, W.r, W.N);
            s->launch_total++;
        }
        k_axpy<<<grid_n, 256, 0, st>>>(x, W.delta, 1.0, W.N);
        s->launch_total++;
        PM_CUDA_TRY(cudaGetLastError());
        *iters_used = total;
        return PM_OK;
    }

    // res = f - A sigma in the residual precision (float-float or float64)
    pm_status true_residual(const double* f, const double* sig, double* res) {
        PM_TRY(apply_A(sig, W.w, residual_prec(), nullptr));
        k_residual_from<<<grid_n, 256, 0, st>>>(f, W.w, res, W.N);
        s->launch_total++;
        PM_CUDA_TRY(cudaGetLastError());
        return PM_OK;
    }
};

}  // namespace

pm_status pm_solve_impl(pm_surface* s, const double* f, double* u, double tol, int maxit,
                        pm_precision prec, unsigned flags, double* sigma_out,
                        pm_solve_info* info, cudaStream_t st) {
    const auto t0 = std::chrono::steady_clock::now();
    Work* Wp = nullptr;
    PM_TRY(get_work(s, &Wp));
    Work& W = *Wp;
    const int N = s->N;
    const bool dev = (flags & PM_SOLVE_DEVICE_PTRS) != 0;
    Solver S{s, W, st, pm_ceil_div(N, 256)};
    const cudaMemcpyKind h2d = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const cudaMemcpyKind d2h = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    PM_CUDA_TRY(cudaMemcpyAsync(W.f, f, sizeof(double) * N, h2d, st));

    // mean-zero check of f (Thm. LBsolvable): |sum w f| / (sqrt(sum w) ||f||_w)
    double sw = 0.0;
    for (double v : s->h_w) sw += v;
    k_mul<<<S.grid_n, 256, 0, st>>>(s->w, W.f, W.tmp, N);
    s->launch_total++;
    PM_TRY(S.dots(W.tmp, 0, 1, W.f, W.scal + 5, nullptr));      // sum w f^2
    PM_TRY(S.dots(s->w, 0, 1, W.f, W.scal + 4, nullptr));       // sum w f
    PM_CUDA_TRY(cudaMemcpyAsync(W.pinned, W.scal + 4, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    PM_CUDA_TRY(cudaStreamSynchronize(st));
    const double wf = W.pinned[0], wff = W.pinned[1];
    double removed = 0.0;
    if (wff > 0.0 && std::fabs(wf) > s->opts.mean_tol * std::sqrt(sw * wff)) {
        if (!(flags & PM_SOLVE_PROJECT_RHS)) {
            pm_set_error("pm_solve: f has weighted mean %.3e (relative %.3e > %.1e); pass "
                         "PM_SOLVE_PROJECT_RHS to subtract it", wf / sw,
                         std::fabs(wf) / std::sqrt(sw * wff), s->opts.mean_tol);
            return PM_ERR_RHS_NOT_MEAN_ZERO;
        }
    }
    if (flags & PM_SOLVE_PROJECT_RHS) {
        removed = wf / sw;
        k_add_shift<<<S.grid_n, 256, 0, st>>>(W.f, W.scal + 4, -1.0 / sw, N);
        s->launch_total++;
    }
    double fnorm = 0.0;
    PM_TRY(S.norm2(W.f, &fnorm));
    PM_CUDA_TRY(cudaMemsetAsync(W.sig, 0, sizeof(double) * N, st));
    int iters = 0, refinements = 0;
    double relres = 0.0;
    pm_status result = PM_OK;
    if (fnorm > 0.0) {
        if (prec == PM_PREC_FP64 || prec == PM_PREC_FF) {
            // one GMRES with accurate applies to the target, confirmed by the true residual
            PM_TRY(S.gmres(W.f, W.sig, prec, tol * fnorm, maxit, &iters));
            PM_TRY(S.true_residual(W.f, W.sig, W.res));
            double rn = 0;
            PM_TRY(S.norm2(W.res, &rn));
            relres = rn / fnorm;
            refinements = 1;
        } else {
            // iterative refinement: accurate residual, float32-operator GMRES correction
            for (;;) {
                double rn = 0;
                if (refinements == 0) {
                    // sigma = 0: the residual is f itself
                    PM_CUDA_TRY(cudaMemcpyAsync(W.res, W.f, sizeof(double) * N,
                                                cudaMemcpyDeviceToDevice, st));
                    rn = fnorm;
                } else {
                    PM_TRY(S.true_residual(W.f, W.sig, W.res));
                    PM_TRY(S.norm2(W.res, &rn));
                }
                relres = rn / fnorm;
                if (relres <= tol || refinements >= s->opts.max_refine || iters >= maxit) break;
                int it = 0;
                const double inner = std::max(s->opts.inner_tol, 0.5 * tol * fnorm / rn);
                PM_TRY(S.gmres(W.res, W.sig, prec, inner * rn, maxit - iters, &it));
                iters += it;
                ++refinements;
                if (it == 0) break;
            }
        }
        if (!(relres <= tol)) {
            pm_set_error("pm_solve: relative residual %.3e above %.3e after %d iterations, %d refinements",
                         relres, tol, iters, refinements);
            result = PM_ERR_NOT_CONVERGED;
        }
    }
    // u = K~ sigma (accurate), then subtract its weighted mean (eq. representation)
    PM_TRY(pm_apply_dev(s, 1, 1, 1, W.sig, W.u, S.residual_prec(), st));
    PM_TRY(S.dots(s->w, 0, 1, W.u, W.scal + 6, nullptr));
    k_add_shift<<<S.grid_n, 256, 0, st>>>(W.u, W.scal + 6, -1.0 / sw, N);
    s->launch_total++;
    PM_CUDA_TRY(cudaGetLastError());
    PM_CUDA_TRY(cudaMemcpyAsync(u, W.u, sizeof(double) * N, d2h, st));
    if (sigma_out)
        PM_CUDA_TRY(cudaMemcpyAsync(sigma_out, W.sig, sizeof(double) * N, d2h, st));
    PM_CUDA_TRY(cudaStreamSynchronize(st));
    if (info) {
        info->iterations = iters;
        info->refinements = refinements;
        info->residual = relres;
        info->removed_mean = removed;
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return result;
}
