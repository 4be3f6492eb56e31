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
// "done" flag that the rotation sets once the residual estimate meets the
// tolerance (or the Arnoldi vector vanishes); later kernels of the cycle
// return immediately.  The host reads the flag every few steps.
//
// One Arnoldi step is the operator apply (float32 sums + near field) and four
// fused kernels over blocks of 256 rows: (1) finish A v and form this block's
// partial dots V_j . w; (2) reduce them, subtract, partial dots again (the
// second Gram-Schmidt pass); (3) reduce, subtract, partial |w|^2; (4) reduce,
// Givens update, v_{k+1} = w/|w| together with the float32 source strengths
// of the next apply and the partial of sum_j w_j v_j for its rank-one term.
// Every block reduces the previous kernel's per-block partials itself, in a
// fixed order, so all blocks hold bit-identical sums and the result does not
// depend on scheduling.
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

// Arnoldi step k finished its orthogonalisation: column h[0..k] is in place and
// hn = |w| is the norm of the new vector.  Apply the previous Givens rotations,
// form the new one, update g, test convergence.  One thread.
__device__ void givens_update(double* __restrict__ H, int ldh, int k, double* __restrict__ cs,
                              double* __restrict__ sn, double* __restrict__ g, double hn,
                              double tol_abs, int* __restrict__ done, int* __restrict__ iters) {
    double* h = H + (size_t)k * ldh;    // column k, entries 0..k+1
    h[k + 1] = hn;
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

// ---------------------------------------------------------------- fused Arnoldi step
constexpr int kArnThreads = 256;    // rows per block
constexpr int kArnMaxCols = 408;    // >= restart + 1

// The flag read once per block, so that every thread of a block takes the same path.
__device__ __forceinline__ bool block_done(const int* __restrict__ done) {
    __shared__ int sd;
    if (threadIdx.x == 0) sd = done ? *reinterpret_cast<const volatile int*>(done) : 0;
    __syncthreads();
    return sd != 0;
}

// out_sh[j] = sum over blocks b of part[b * ld + j], j < n: a warp per column,
// lanes over blocks, fixed order (identical in every block).
__device__ void reduce_cols_sh(const double* __restrict__ part, int nblk, int ld, int n,
                               double* out_sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j = wid; j < n; j += nw) {
        double t = 0.0;
        for (int b = lane; b < nblk; b += 32) t += part[(size_t)b * ld + j];
        t = warp_sum(t);
        if (lane == 0) out_sh[j] = t;
    }
    __syncthreads();
}

// part_row[j] = sum over the block's rows r0 + t of V_j[r0 + t] w_sh[t], j < ncols
__device__ void col_dots_sh(const double* __restrict__ V, long long ldv, int ncols,
                            const double* w_sh, int r0, int nr, double* __restrict__ part_row) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (int j = wid; j < ncols; j += nw) {
        const double* a = V + (size_t)j * ldv + r0;
        double t = 0.0;
        for (int q = lane; q < nr; q += 32) t += a[q] * w_sh[q];
        t = warp_sum(t);
        if (lane == 0) part_row[j] = t;
    }
}

// v_i = r_i * inv, with the float32 strengths of the next apply (src32 != NULL)
// and this block's partial of sum_i wq_i v_i.
__device__ void scale_prep_wdot(const double* __restrict__ r, double inv, double* __restrict__ v,
                                const double* __restrict__ wq, const double* __restrict__ wa,
                                float4* __restrict__ src32, float* __restrict__ sig32, int pp,
                                int ppad, double* __restrict__ pw_row, int N, double* red) {
    const int i = blockIdx.x * kArnThreads + threadIdx.x;
    double t = 0.0;
    if (i < N) {
        const double vi = r[i] * inv;
        v[i] = vi;
        if (src32) {
            src32[i].w = (float)(wa[i] * vi);
            const int P = i / pp;
            sig32[(size_t)P * ppad + (i - P * pp)] = (float)vi;
        }
        t = wq[i] * vi;
    }
    t = block_sum(t, red);
    if (threadIdx.x == 0) pw_row[0] = t;
}

// This block's partial of r . r.
__global__ void __launch_bounds__(kArnThreads)
k_sq_partial(const double* __restrict__ r, int N, double* __restrict__ pout, int ld) {
    __shared__ double red[32];
    const int i = blockIdx.x * kArnThreads + threadIdx.x;
    const double v = (i < N) ? r[i] : 0.0;
    const double t = block_sum(v * v, red);
    if (threadIdx.x == 0) pout[(size_t)blockIdx.x * ld] = t;
}

// Step index of the fused kernels: the device counter (graph-driven cycles,
// where one captured step serves every k) or the launch argument.
__device__ __forceinline__ int step_index(int k_arg, const int* __restrict__ k_dev) {
    return k_dev ? *k_dev : k_arg;
}

// Cycle start: beta = |r|, g = (beta, 0, ...), v0 = r / beta (+ prep, wq . v0 partials).
// par = (tol_abs, steps).  use_cond: also sets the graph's loop condition.
__global__ void __launch_bounds__(kArnThreads)
k_arn_start(const double* __restrict__ pin, int nblk, int ld, double* __restrict__ g, int m,
            double* __restrict__ scal, const double* __restrict__ par, int* __restrict__ done,
            int* __restrict__ iters, const double* __restrict__ r, double* __restrict__ v0,
            const double* __restrict__ wq, const double* __restrict__ wa,
            float4* __restrict__ src32, float* __restrict__ sig32, int pp, int ppad,
            double* __restrict__ pw, int N, int use_cond, cudaGraphConditionalHandle cond) {
    __shared__ double red[32];
    reduce_cols_sh(pin, nblk, ld, 1, red);
    const double beta = sqrt(red[0]);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        for (int k = 0; k <= m; ++k) g[k] = 0.0;
        g[0] = beta;
        scal[3] = beta;
        *iters = 0;
        const int d = (beta <= par[0] || beta == 0.0) ? 1 : 0;
        *done = d;
        if (use_cond) cudaGraphSetConditional(cond, (!d && par[1] >= 1.0) ? 1u : 0u);
    }
    __syncthreads();
    scale_prep_wdot(r, beta > 0.0 ? 1.0 / beta : 0.0, v0, wq, wa, src32, sig32, pp, ppad,
                    pw + (size_t)blockIdx.x * ld, N, red);
}

// (1) w = v_k + y + sum_j wq_j v_k,j (A v_k with the rank-one term); partial dots V_j . w, j <= k.
__global__ void __launch_bounds__(kArnThreads)
k_arn_first(const double* __restrict__ y, const double* __restrict__ pw, int nblk, int ld,
            const double* __restrict__ V, long long ldv, int k_arg, const int* __restrict__ k_dev,
            double* __restrict__ w, double* __restrict__ pout, int N,
            const int* __restrict__ done) {
    __shared__ double red[32];
    __shared__ double w_sh[kArnThreads];
    if (block_done(done)) return;
    const int k = step_index(k_arg, k_dev);
    const double* v = V + (size_t)k * ldv;
    reduce_cols_sh(pw, nblk, ld, 1, red);
    const int r0 = blockIdx.x * kArnThreads, i = r0 + threadIdx.x;
    double wi = 0.0;
    if (i < N) {
        wi = v[i] + y[i] + red[0];
        w[i] = wi;
    }
    w_sh[threadIdx.x] = wi;
    __syncthreads();
    col_dots_sh(V, ldv, k + 1, w_sh, r0, min(kArnThreads, N - r0), pout + (size_t)blockIdx.x * ld);
}

// (2) h1 = sum of the partial dots; block 0 stores it as Hessenberg column k;
// w -= V h1; then this block's partial dots V_j . w (j <= k) and w . w (column
// k + 1), all from the same w.
__global__ void __launch_bounds__(kArnThreads)
k_arn_pass(const double* __restrict__ pin, int nblk, int ld, const double* __restrict__ V,
           long long ldv, double* __restrict__ H, int ldh, int k_arg,
           const int* __restrict__ k_dev, double* __restrict__ w, double* __restrict__ pout,
           int N, const int* __restrict__ done) {
    __shared__ double h_sh[kArnMaxCols];
    __shared__ double w_sh[kArnThreads];
    __shared__ double red[32];
    if (block_done(done)) return;
    const int k = step_index(k_arg, k_dev);
    const int ncols = k + 1;
    double* hk = H + (size_t)k * ldh;
    reduce_cols_sh(pin, nblk, ld, ncols, h_sh);
    if (blockIdx.x == 0)
        for (int j = threadIdx.x; j < ncols; j += blockDim.x) hk[j] = h_sh[j];
    const int r0 = blockIdx.x * kArnThreads, i = r0 + threadIdx.x;
    double wi = 0.0;
    if (i < N) {
        wi = w[i];
        for (int j = 0; j < ncols; ++j) wi -= V[(size_t)j * ldv + i] * h_sh[j];
        w[i] = wi;
    }
    w_sh[threadIdx.x] = wi;
    const double t = block_sum(wi * wi, red);     // synchronises the block (w_sh complete)
    if (threadIdx.x == 0) pout[(size_t)blockIdx.x * ld + ncols] = t;
    col_dots_sh(V, ldv, ncols, w_sh, r0, min(kArnThreads, N - r0),
                pout + (size_t)blockIdx.x * ld);
}

// (3) Second Gram-Schmidt correction and normalisation in one kernel: h2 and
// |w1|^2 from the partials of (2) (w1 = w after the first correction); block 0
// adds h2 to Hessenberg column k; w2 = w1 - V h2; |w2| = sqrt(|w1|^2 - |h2|^2)
// (V orthonormal, so no further reduction is needed; h2 is of rounding size
// against w1, so the difference does not cancel); v_{k+1} = w2 / |w2| with the
// next apply's prep and wq . v_{k+1} partials.  givens: block 0 also applies
// the Givens update (may set done); otherwise k_arn_advance does it with the
// |w2| left in *hn_out.
__global__ void __launch_bounds__(kArnThreads)
k_arn_finish(const double* __restrict__ pin, int nblk, int ld, const double* __restrict__ Vr,
             long long ldv, double* __restrict__ H, int ldh, int k_arg,
             const int* __restrict__ k_dev, int givens, double* __restrict__ cs,
             double* __restrict__ sn, double* __restrict__ g, const double* __restrict__ par,
             int* __restrict__ done, int* __restrict__ iters, double* __restrict__ w,
             double* __restrict__ hn_out, double* __restrict__ V, const double* __restrict__ wq,
             const double* __restrict__ wa, float4* __restrict__ src32,
             float* __restrict__ sig32, int pp, int ppad, double* __restrict__ pw, int N) {
    __shared__ double h_sh[kArnMaxCols + 1];
    __shared__ double red[32];
    if (block_done(done)) return;
    const int k = step_index(k_arg, k_dev);
    const int ncols = k + 1;
    reduce_cols_sh(pin, nblk, ld, ncols + 1, h_sh);
    double s2 = 0.0;
    for (int j = 0; j < ncols; ++j) s2 += h_sh[j] * h_sh[j];
    const double hn2 = h_sh[ncols] - s2;
    const double hn = hn2 > 0.0 ? sqrt(hn2) : 0.0;
    if (blockIdx.x == 0) {
        double* hk = H + (size_t)k * ldh;
        for (int j = threadIdx.x; j < ncols; j += blockDim.x) hk[j] += h_sh[j];
        __syncthreads();
        if (threadIdx.x == 0) {
            *hn_out = hn;
            if (givens) givens_update(H, ldh, k, cs, sn, g, hn, par[0], done, iters);
        }
    }
    const int i = blockIdx.x * kArnThreads + threadIdx.x;
    if (i < N) {
        double wi = w[i];
        for (int j = 0; j < ncols; ++j) wi -= Vr[(size_t)j * ldv + i] * h_sh[j];
        w[i] = wi;
    }
    scale_prep_wdot(w, hn > 0.0 ? 1.0 / hn : 0.0, V + (size_t)(k + 1) * ldv, wq, wa, src32,
                    sig32, pp, ppad, pw + (size_t)blockIdx.x * ld, N, red);
}

// Graph-driven cycles: the Givens update of step k = *iters with the |w2| that
// k_arn_finish left in *hn_in, then the loop condition:
// continue while not converged and fewer than par[1] steps were taken.  The
// condition is written on every path, so the loop always ends: at the latest
// after par[1] <= restart steps, since *iters grows by one per step.
__global__ void k_arn_advance(const double* __restrict__ hn_in, double* __restrict__ H, int ldh,
                              double* __restrict__ cs, double* __restrict__ sn,
                              double* __restrict__ g, const double* __restrict__ par,
                              int* __restrict__ done, int* __restrict__ iters,
                              cudaGraphConditionalHandle cond) {
    const bool was_done = block_done(done);
    if (threadIdx.x != 0) return;
    if (was_done) {
        cudaGraphSetConditional(cond, 0u);
        return;
    }
    const int k = *iters;
    givens_update(H, ldh, k, cs, sn, g, *hn_in, par[0], done, iters);
    cudaGraphSetConditional(cond, (!*done && (double)(k + 1) < par[1]) ? 1u : 0u);
}

// y = H(0:n,0:n)^{-1} g(0:n) by back substitution, n = *iters; ynorm = |y|_2,
// which is the norm of the cycle's correction V y (orthonormal V)
__global__ void k_backsolve(const double* __restrict__ H, int ldh, const double* __restrict__ g,
                            const int* __restrict__ iters, double* __restrict__ y,
                            double* __restrict__ ynorm) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int n = *iters;
    double s2 = 0.0;
    for (int i = n - 1; i >= 0; --i) {
        double t = g[i];
        for (int j = i + 1; j < n; ++j) t -= H[(size_t)j * ldh + i] * y[j];
        const double d = H[(size_t)i * ldh + i];
        y[i] = (d != 0.0) ? t / d : 0.0;
        s2 += y[i] * y[i];
    }
    *ynorm = sqrt(s2);
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
    int N = 0, m = 0, nred = 0, narn = 0;
    double *V = nullptr, *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr, *y = nullptr;
    double *part = nullptr, *scal = nullptr, *hcol = nullptr;
    double *pa = nullptr, *pb = nullptr;      // per-block partials of the fused Arnoldi kernels
    double* pc = nullptr;                     // per-block partials of wq . v (rank-one term)
    double* hn = nullptr;                     // |w2| of the last step (graph-driven Givens)
    double *w = nullptr, *tmp = nullptr, *r = nullptr, *res = nullptr, *delta = nullptr;
    double *sig = nullptr, *f = nullptr, *u = nullptr;
    int *done = nullptr, *iters = nullptr;
    double* par = nullptr;          // device (tol_abs, steps) of the current cycle
    double* pinned = nullptr;       // host-pinned scalars read back per cycle
    double* pinned_par = nullptr;   // host-pinned staging of par
    int* pinned_i = nullptr;
    // one GMRES cycle as a CUDA graph: prologue, a device-driven while loop over
    // Arnoldi steps, epilogue (FP32 / FMM operators, profiling off)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap_stream = nullptr, body_stream = nullptr;
    pm_precision graph_prec = PM_PREC_FP64;
    long long graph_epoch = -1;
    long long failed_epoch = -1;
    pm_precision failed_prec = PM_PREC_FP64;
    int body_launches = 0;          // kernels per loop iteration
};

}  // namespace

struct PmSolveWork : Work {};

void pm_solve_free(pm_surface* s) {
    if (!s->solve_work) return;
    Work& W = *s->solve_work;
    pm_dfree(W.V); pm_dfree(W.H); pm_dfree(W.cs); pm_dfree(W.sn); pm_dfree(W.g); pm_dfree(W.y);
    pm_dfree(W.part); pm_dfree(W.scal); pm_dfree(W.hcol); pm_dfree(W.w); pm_dfree(W.tmp);
    pm_dfree(W.r); pm_dfree(W.res); pm_dfree(W.delta); pm_dfree(W.sig); pm_dfree(W.f);
    pm_dfree(W.u); pm_dfree(W.done); pm_dfree(W.iters); pm_dfree(W.pa); pm_dfree(W.pb); pm_dfree(W.pc); pm_dfree(W.hn);
    pm_dfree(W.par);
    if (W.exec) cudaGraphExecDestroy(W.exec);
    if (W.graph) cudaGraphDestroy(W.graph);
    if (W.cap_stream) cudaStreamDestroy(W.cap_stream);
    if (W.body_stream) cudaStreamDestroy(W.body_stream);
    if (W.pinned_par) cudaFreeHost(W.pinned_par);
    if (W.pinned) cudaFreeHost(W.pinned);
    if (W.pinned_i) cudaFreeHost(W.pinned_i);
    delete s->solve_work;
    s->solve_work = nullptr;
}

namespace {

pm_status alloc_work(pm_surface* s, int m);

// The Krylov workspace for the current restart length; a failed allocation frees
// whatever was allocated, so no partly built workspace is ever reused.
pm_status get_work(pm_surface* s, Work** out) {
    const int m = std::max(2, std::min(s->opts.gmres_restart, 400));
    if (s->solve_work && s->solve_work->m == m) {
        *out = s->solve_work;
        return PM_OK;
    }
    const pm_status st = alloc_work(s, m);
    if (st != PM_OK) {
        pm_solve_free(s);
        return st;
    }
    *out = s->solve_work;
    return PM_OK;
}

pm_status alloc_work(pm_surface* s, int m) {
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
    W.narn = pm_ceil_div(N, kArnThreads);
    PM_TRY(pm_dmalloc(&W.pa, (size_t)W.narn * (m + 2)));
    PM_TRY(pm_dmalloc(&W.pb, (size_t)W.narn * (m + 2)));
    PM_TRY(pm_dmalloc(&W.pc, (size_t)W.narn * (m + 2)));
    PM_TRY(pm_dmalloc(&W.hn, 1));
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
    PM_TRY(pm_dmalloc(&W.par, 2));
    PM_CUDA_TRY(cudaMallocHost((void**)&W.pinned, 8 * sizeof(double)));
    PM_CUDA_TRY(cudaMallocHost((void**)&W.pinned_par, 2 * sizeof(double)));
    PM_CUDA_TRY(cudaMallocHost((void**)&W.pinned_i, 4 * sizeof(int)));
    return PM_OK;
}

struct Solver {
    pm_surface* s;
    Work& W;
    cudaStream_t st;
    int grid_n;
    pm_precision op = PM_PREC_FF;   // the solve's operator precision

    // precision of true residuals and of the representation: float64 or float-float,
    // or (opts.residual_prec = PM_PREC_FP32) the float32 / FMM operator itself
    pm_precision residual_prec() const {
        if (s->opts.residual_prec == PM_PREC_FP64) return PM_PREC_FP64;
        if (s->opts.residual_prec == PM_PREC_FP32 && (op == PM_PREC_FP32 || op == PM_PREC_FMM))
            return op;
        return PM_PREC_FF;
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

    void drop_graph() {
        if (W.exec) cudaGraphExecDestroy(W.exec);
        if (W.graph) cudaGraphDestroy(W.graph);
        W.exec = nullptr;
        W.graph = nullptr;
    }

    // Capture one GMRES cycle: [|r|^2 partials, start] -> while (cond) { apply,
    // first, pass, pass, normalize, advance } -> [back substitution, x update].
    // Every kernel reads the step index and the cycle parameters from device
    // memory, so one instantiated graph serves every cycle of every solve.
    pm_status capture_graph(pm_precision prec) {
        const int m = W.m, nb = W.narn, ld = m + 2, N = W.N;
        const long long ldv = N;
        float4* src32 = s->src32;
        if (!W.cap_stream)
            PM_CUDA_TRY(cudaStreamCreateWithFlags(&W.cap_stream, cudaStreamNonBlocking));
        if (!W.body_stream)
            PM_CUDA_TRY(cudaStreamCreateWithFlags(&W.body_stream, cudaStreamNonBlocking));
        cudaStream_t cs = W.cap_stream, bs = W.body_stream;
        PM_CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
        cudaGraph_t g = nullptr;
        cudaStreamCaptureStatus cst;
        cudaError_t ce = cudaStreamGetCaptureInfo(cs, &cst, nullptr, &g, nullptr, nullptr, nullptr);
        cudaGraphConditionalHandle cond = 0;
        if (ce == cudaSuccess) ce = cudaGraphConditionalHandleCreate(&cond, g, 0, cudaGraphCondAssignDefault);
        if (ce == cudaSuccess) {
            k_sq_partial<<<nb, kArnThreads, 0, cs>>>(W.r, N, W.pa, ld);
            k_arn_start<<<nb, kArnThreads, 0, cs>>>(W.pa, nb, ld, W.g, m, W.scal, W.par, W.done,
                                                    W.iters, W.r, W.V, s->w, s->wa, src32, s->sig32,
                                                    s->pp, s->ppad, W.pc, N, 1, cond);
            ce = cudaGetLastError();
        }
        const cudaGraphNode_t* deps = nullptr;
        size_t ndeps = 0;
        if (ce == cudaSuccess)
            ce = cudaStreamGetCaptureInfo(cs, &cst, nullptr, nullptr, &deps, nullptr, &ndeps);
        cudaGraphNodeParams cp = {};
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = cond;
        cp.conditional.type = cudaGraphCondTypeWhile;
        cp.conditional.size = 1;
        cudaGraphNode_t cnode = nullptr;
        if (ce == cudaSuccess) ce = cudaGraphAddNode(&cnode, g, deps, nullptr, ndeps, &cp);
        if (ce == cudaSuccess)
            ce = cudaStreamUpdateCaptureDependencies(cs, &cnode, nullptr, 1,
                                                     cudaStreamSetCaptureDependencies);
        if (ce == cudaSuccess) {
            cudaGraph_t body = cp.conditional.phGraph_out[0];
            ce = cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0,
                                               cudaStreamCaptureModeThreadLocal);
            if (ce == cudaSuccess) {
                const long long before = s->launch_total;
                s->skip_flag = W.done;
                const pm_status stt = pm_apply_dev(s, 0, 1, 1, W.V, W.tmp, prec, bs, 1);
                s->skip_flag = nullptr;
                W.body_launches = (int)(s->launch_total - before) + 4;
                s->launch_total = before;
                k_arn_first<<<nb, kArnThreads, 0, bs>>>(W.tmp, W.pc, nb, ld, W.V, ldv, 0, W.iters,
                                                        W.w, W.pa, N, W.done);
                k_arn_pass<<<nb, kArnThreads, 0, bs>>>(W.pa, nb, ld, W.V, ldv, W.H, m + 2, 0,
                                                       W.iters, W.w, W.pb, N, W.done);
                k_arn_finish<<<nb, kArnThreads, 0, bs>>>(
                    W.pb, nb, ld, W.V, ldv, W.H, m + 2, 0, W.iters, 0, W.cs, W.sn, W.g, W.par,
                    W.done, W.iters, W.w, W.hn, W.V, s->w, s->wa, src32, s->sig32, s->pp, s->ppad,
                    W.pc, N);
                k_arn_advance<<<1, 32, 0, bs>>>(W.hn, W.H, m + 2, W.cs, W.sn, W.g, W.par,
                                                W.done, W.iters, cond);
                ce = cudaGetLastError();
                cudaGraph_t body_out = nullptr;
                const cudaError_t ce2 = cudaStreamEndCapture(bs, &body_out);
                if (ce == cudaSuccess) ce = ce2;
                if (ce == cudaSuccess && stt != PM_OK) ce = cudaErrorUnknown;
            }
        }
        if (ce == cudaSuccess) {
            k_backsolve<<<1, 1, 0, cs>>>(W.H, m + 2, W.g, W.iters, W.y, W.scal + 7);
            k_add_combo<<<pm_ceil_div(N, 256), 256, 0, cs>>>(W.V, ldv, W.iters, W.y, W.delta, N);
            ce = cudaGetLastError();
        }
        cudaGraph_t out = nullptr;
        const cudaError_t ce3 = cudaStreamEndCapture(cs, &out);
        if (ce == cudaSuccess) ce = ce3;
        // per-node priorities: the FMM's far-field kernels keep their stream's priority
        if (ce == cudaSuccess)
            ce = cudaGraphInstantiate(&W.exec, out, cudaGraphInstantiateFlagUseNodePriority);
        if (ce != cudaSuccess) {
            if (out) cudaGraphDestroy(out);
            W.exec = nullptr;
            cudaGetLastError();
            pm_set_error("gmres graph capture: %s", cudaGetErrorString(ce));
            return PM_ERR_CUDA;
        }
        W.graph = out;
        return PM_OK;
    }

    // The cycle graph for this operator precision, (re)built when the surface's
    // buffers or launch shapes changed.  A capture that fails is not retried for
    // the same state; the cycle then runs as host-issued launches.
    bool ensure_graph(pm_precision prec) {
        if (W.exec && W.graph_prec == prec && W.graph_epoch == s->graph_epoch) return true;
        if (W.failed_epoch == s->graph_epoch && W.failed_prec == prec) return false;
        drop_graph();
        // one un-captured apply creates whatever the apply allocates lazily
        if (pm_apply_dev(s, 0, 1, 1, W.V, W.tmp, prec, st, 0) != PM_OK ||
            cudaStreamSynchronize(st) != cudaSuccess || capture_graph(prec) != PM_OK) {
            drop_graph();
            W.failed_epoch = s->graph_epoch;
            W.failed_prec = prec;
            return false;
        }
        W.graph_prec = prec;
        W.graph_epoch = s->graph_epoch;
        return true;
    }

    // Enqueue one GMRES cycle for A d = W.r from d = W.delta's current value plus the
    // cycle's correction (W.delta += V y), with the operator in `prec`: at most `steps`
    // Arnoldi steps, stopping once the residual estimate is below tol_abs.  No host
    // synchronisation, except the done-flag reads of the host-issued form (profiling on).
    // Afterwards W.iters, W.done and W.scal[7] = |y| describe the cycle.
    pm_status launch_cycle(pm_precision prec, double tol_abs, int steps) {
        const int m = W.m;
        const long long ldv = W.N;
        // the float32 strengths of each basis vector are written by the kernel
        // that forms it (FP32 / FMM operators)
        const bool fuse_prep = prec == PM_PREC_FP32 || prec == PM_PREC_FMM;
        const bool graph = fuse_prep && !s->profiling && ensure_graph(prec);
        float4* src32 = fuse_prep ? s->src32 : nullptr;
        const int nb = W.narn, ld = m + 2;
        W.pinned_par[0] = tol_abs;
        W.pinned_par[1] = (double)steps;
        PM_CUDA_TRY(cudaMemcpyAsync(W.par, W.pinned_par, 2 * sizeof(double),
                                    cudaMemcpyHostToDevice, st));
        if (graph) {
            PM_CUDA_TRY(cudaGraphLaunch(W.exec, st));
            s->launch_total += 4;                  // plus body_launches per step, counted on readback
            return PM_OK;
        }
        k_sq_partial<<<nb, kArnThreads, 0, st>>>(W.r, W.N, W.pa, ld);
        k_arn_start<<<nb, kArnThreads, 0, st>>>(W.pa, nb, ld, W.g, m, W.scal, W.par, W.done,
                                                W.iters, W.r, W.V, s->w, s->wa, src32,
                                                s->sig32, s->pp, s->ppad, W.pc, W.N, 0, 0);
        s->launch_total += 2;
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
            // W.tmp = R~ v_k (sources already prepared when fuse_prep)
            pm_status stt = pm_apply_dev(s, 0, 1, 1, W.V + (size_t)k * ldv, W.tmp, prec, st,
                                         fuse_prep ? 1 : 0);
            if (stt != PM_OK) { s->skip_flag = nullptr; return stt; }
            // partials: first -> pa, pass -> pb, finish -> pc (each kernel reduces the
            // previous one's buffer in every block, so it never writes the one it reads)
            k_arn_first<<<nb, kArnThreads, 0, st>>>(W.tmp, W.pc, nb, ld, W.V, ldv, k, nullptr,
                                                    W.w, W.pa, W.N, W.done);
            k_arn_pass<<<nb, kArnThreads, 0, st>>>(W.pa, nb, ld, W.V, ldv, W.H, m + 2, k, nullptr,
                                                   W.w, W.pb, W.N, W.done);
            k_arn_finish<<<nb, kArnThreads, 0, st>>>(
                W.pb, nb, ld, W.V, ldv, W.H, m + 2, k, nullptr, 1, W.cs, W.sn, W.g, W.par, W.done,
                W.iters, W.w, W.hn, W.V, s->w, s->wa, src32, s->sig32, s->pp, s->ppad, W.pc, W.N);
            s->launch_total += 3;
        }
        s->skip_flag = nullptr;
        PM_CUDA_TRY(cudaGetLastError());
        k_backsolve<<<1, 1, 0, st>>>(W.H, m + 2, W.g, W.iters, W.y, W.scal + 7);
        k_add_combo<<<grid_n, 256, 0, st>>>(W.V, ldv, W.iters, W.y, W.delta, W.N);
        s->launch_total += 2;
        PM_CUDA_TRY(cudaGetLastError());
        return PM_OK;
    }

    // Enqueue the copies of the cycle's outcome (iterations, done flag, |y|) to the host.
    pm_status enqueue_cycle_readback() {
        PM_CUDA_TRY(cudaMemcpyAsync(W.pinned_i, W.iters, sizeof(int), cudaMemcpyDeviceToHost, st));
        PM_CUDA_TRY(cudaMemcpyAsync(W.pinned_i + 1, W.done, sizeof(int), cudaMemcpyDeviceToHost, st));
        PM_CUDA_TRY(cudaMemcpyAsync(W.pinned + 7, W.scal + 7, sizeof(double),
                                    cudaMemcpyDeviceToHost, st));
        return PM_OK;
    }

    // After the synchronisation: iterations of the cycle (launch accounting of the graph form).
    int cycle_iterations(pm_precision prec) {
        const int it = W.pinned_i[0];
        const bool fuse_prep = prec == PM_PREC_FP32 || prec == PM_PREC_FMM;
        if (fuse_prep && !s->profiling && W.exec) s->launch_total += (long long)it * W.body_launches;
        return it;
    }

    // Restarted GMRES(m) for A d = b from d = 0 with the operator in `prec`,
    // stopping when the residual estimate is below tol_abs; x += d.
    pm_status gmres(const double* b, double* x, pm_precision prec, double tol_abs, int max_iter,
                    int* iters_used, double* dnorm = nullptr) {
        double dn = 0.0;                    // bound on |x_new - x_old|: sum of the cycles' |y|
        int total = 0;
        PM_CUDA_TRY(cudaMemcpyAsync(W.r, b, sizeof(double) * W.N, cudaMemcpyDeviceToDevice, st));
        PM_CUDA_TRY(cudaMemsetAsync(W.delta, 0, sizeof(double) * W.N, st));
        while (total < max_iter) {
            PM_TRY(launch_cycle(prec, tol_abs, std::min(W.m, max_iter - total)));
            PM_TRY(enqueue_cycle_readback());
            PM_CUDA_TRY(cudaStreamSynchronize(st));
            const int it = cycle_iterations(prec);
            const int converged = W.pinned_i[1];
            if (it > 0) dn += W.pinned[7];
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
        if (dnorm) *dnorm = dn;
        return PM_OK;
    }

    // Enqueue u = K~ sigma in the residual precision minus its weighted mean (eq.
    // representation), with 1/sw the reciprocal of sum w.
    pm_status enqueue_representation(double inv_sw) {
        PM_TRY(pm_apply_dev(s, 1, 1, 1, W.sig, W.u, residual_prec(), st));
        PM_TRY(dots(s->w, 0, 1, W.u, W.scal + 6, nullptr));
        k_add_shift<<<grid_n, 256, 0, st>>>(W.u, W.scal + 6, -inv_sw, W.N);
        s->launch_total++;
        PM_CUDA_TRY(cudaGetLastError());
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

// Device bytes a solve of nrhs right-hand sides would allocate on top of what
// the surface already holds (its Krylov workspaces are kept between solves and
// only grow): the single-RHS workspace of get_work, or the batched solver's and
// batched apply's buffers (pm_batch.cu), plus the FMM tree and the context's M2L
// operators when FMM applies are used and not yet built.  An a-priori model of
// the allocations above, not a measurement.
size_t pm_solve_need_bytes(const pm_surface* s, int nrhs, pm_precision prec) {
    const size_t m = (size_t)std::max(2, std::min(s->opts.gmres_restart, 400));
    const size_t N = (size_t)s->N;
    size_t need = 0;
    if (nrhs <= 1) {
        const bool held = s->solve_work && (size_t)s->solve_work->m == m;
        if (!held) {
            const size_t nred = (size_t)std::max(1, std::min(pm_ceil_div(s->N, 1024),
                                                             2 * s->ctx->num_sms));
            const size_t narn = (size_t)pm_ceil_div(s->N, kArnThreads);
            need += sizeof(double) * ((m + 1) * N + m * (m + 2) + 4 * m + 8 * N +
                                      (nred + 3 * narn + 2) * (m + 2) + 64);
        }
    } else {
        need += pm_batch_need_bytes(s, nrhs);
    }
    if (prec == PM_PREC_FMM) need += pm_fmm_need_bytes(s);
    return need;
}

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
    S.op = prec;
    const cudaMemcpyKind h2d = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const cudaMemcpyKind d2h = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    PM_CUDA_TRY(cudaMemcpyAsync(W.f, f, sizeof(double) * N, h2d, st));

    // mean-zero check of f (Thm. LBsolvable): |sum w f| / (sqrt(sum w) ||f||_w), and |f|
    double sw = 0.0;
    for (double v : s->h_w) sw += v;
    k_mul<<<S.grid_n, 256, 0, st>>>(s->w, W.f, W.tmp, N);
    s->launch_total++;
    PM_TRY(S.dots(W.tmp, 0, 1, W.f, W.scal + 5, nullptr));      // sum w f^2
    PM_TRY(S.dots(s->w, 0, 1, W.f, W.scal + 4, nullptr));       // sum w f
    PM_TRY(S.dots(W.f, 0, 1, W.f, W.scal + 1, nullptr));        // sum f^2
    PM_CUDA_TRY(cudaMemcpyAsync(W.pinned, W.scal + 4, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    PM_CUDA_TRY(cudaMemcpyAsync(W.pinned + 2, W.scal + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
    PM_CUDA_TRY(cudaStreamSynchronize(st));
    const double wf = W.pinned[0], wff = W.pinned[1];
    double fnorm = std::sqrt(W.pinned[2]);
    double removed = 0.0;
    const bool nonzero_mean = wff > 0.0 && std::fabs(wf) > s->opts.mean_tol * std::sqrt(sw * wff);
    if (nonzero_mean && !(flags & PM_SOLVE_PROJECT_RHS)) {
        pm_set_error("pm_solve: f has weighted mean %.3e (relative %.3e > %.1e); pass "
                     "PM_SOLVE_PROJECT_RHS to subtract it", wf / sw,
                     std::fabs(wf) / std::sqrt(sw * wff), s->opts.mean_tol);
        return PM_ERR_RHS_NOT_MEAN_ZERO;
    }
    if (flags & PM_SOLVE_PROJECT_RHS) {
        removed = wf / sw;
        k_add_shift<<<S.grid_n, 256, 0, st>>>(W.f, W.scal + 4, -1.0 / sw, N);
        s->launch_total++;
        PM_TRY(S.norm2(W.f, &fnorm));
    }
    // starting density: the caller's (warm start) or zero
    const bool guess = (flags & PM_SOLVE_INITIAL_GUESS) != 0 && sigma_out;
    if (guess)
        PM_CUDA_TRY(cudaMemcpyAsync(W.sig, sigma_out, sizeof(double) * N, h2d, st));
    else
        PM_CUDA_TRY(cudaMemsetAsync(W.sig, 0, sizeof(double) * N, st));
    int iters = 0, refinements = 0, updated = 0;
    double relres = 0.0;
    bool u_current = false;            // W.u holds the representation of the current sigma
    pm_status result = PM_OK;
    if (fnorm > 0.0) {
        if (prec == PM_PREC_FP64 || prec == PM_PREC_FF) {
            // one GMRES with accurate applies to the target (on the residual of the
            // starting density), confirmed by the true residual
            if (guess) {
                PM_TRY(S.true_residual(W.f, W.sig, W.res));
                double r0 = 0.0;
                PM_TRY(S.norm2(W.res, &r0));
                if (r0 > tol * fnorm) PM_TRY(S.gmres(W.res, W.sig, prec, tol * fnorm, maxit, &iters));
            } else {
                PM_TRY(S.gmres(W.f, W.sig, prec, tol * fnorm, maxit, &iters));
            }
            PM_TRY(S.true_residual(W.f, W.sig, W.res));
            double rn = 0;
            PM_TRY(S.norm2(W.res, &rn));
            relres = rn / fnorm;
            refinements = 1;
        } else {
            // Iterative refinement: one float32-operator GMRES cycle per refinement on
            // the current residual, whose outcome is read with the next residual in one
            // synchronisation.  After a correction d the residual is f - A(sigma + d) =
            // r - A d.  It is recomputed in the residual precision after the first
            // correction (d = sigma is O(|f|)); later it is taken as r - A32 d when the
            // float32 operator's error on d, at most kOpRelErr |d| (|d| = |y|, orthonormal
            // basis), stays below a tenth of the tolerance -- then it is the true residual
            // to within 0.1 tol |f| (opts.residual_update) -- and recomputed otherwise.
            // A cycle that stops before convergence (restart length or iteration budget)
            // ends its refinement; the next one starts from the accurate residual.  When
            // the cycle's target is below the overall tolerance the representation u is
            // enqueued before the synchronisation too.
            double rn = fnorm;
            if (guess) {
                PM_TRY(S.true_residual(W.f, W.sig, W.res));
                PM_TRY(S.norm2(W.res, &rn));
            } else {
                PM_CUDA_TRY(cudaMemcpyAsync(W.res, W.f, sizeof(double) * N,
                                            cudaMemcpyDeviceToDevice, st));
            }
            for (;;) {
                relres = rn / fnorm;
                if (relres <= tol || refinements >= s->opts.max_refine || iters >= maxit) break;
                const double inner = std::max(s->opts.inner_tol, 0.5 * tol * fnorm / rn);
                const double tol_abs = inner * rn;
                PM_CUDA_TRY(cudaMemcpyAsync(W.r, W.res, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
                PM_CUDA_TRY(cudaMemsetAsync(W.delta, 0, sizeof(double) * N, st));
                PM_TRY(S.launch_cycle(prec, tol_abs, std::min(W.m, maxit - iters)));
                k_axpy<<<S.grid_n, 256, 0, st>>>(W.sig, W.delta, 1.0, N);
                s->launch_total++;
                const bool predict_update = s->opts.residual_update && refinements >= 1;
                if (predict_update) {
                    PM_TRY(S.apply_A(W.delta, W.w, prec, nullptr));
                    k_axpy<<<S.grid_n, 256, 0, st>>>(W.res, W.w, -1.0, N);
                    s->launch_total++;
                } else {
                    PM_TRY(S.true_residual(W.f, W.sig, W.res));
                }
                PM_TRY(S.dots(W.res, 0, 1, W.res, W.scal + 1, nullptr));
                const bool predict_final = tol_abs <= tol * fnorm;
                if (predict_final) PM_TRY(S.enqueue_representation(1.0 / sw));
                PM_TRY(S.enqueue_cycle_readback());
                PM_CUDA_TRY(cudaMemcpyAsync(W.pinned + 1, W.scal + 1, sizeof(double),
                                            cudaMemcpyDeviceToHost, st));
                PM_CUDA_TRY(cudaStreamSynchronize(st));
                const int it = S.cycle_iterations(prec);
                const double dnorm = W.pinned[7];
                rn = std::sqrt(W.pinned[1]);
                iters += it;
                ++refinements;
                u_current = predict_final;
                if (predict_update) {
                    if (kOpRelErr * dnorm > 0.1 * tol * fnorm) {
                        // the correction was not small: recompute the true residual
                        PM_TRY(S.true_residual(W.f, W.sig, W.res));
                        PM_TRY(S.norm2(W.res, &rn));
                    } else {
                        ++updated;
                    }
                }
                if (it == 0) {
                    relres = rn / fnorm;
                    break;
                }
            }
        }
        if (!(relres <= tol)) {
            pm_set_error("pm_solve: relative residual %.3e above %.3e after %d iterations, %d refinements",
                         relres, tol, iters, refinements);
            result = PM_ERR_NOT_CONVERGED;
        }
    }
    // u = K~ sigma (accurate), then subtract its weighted mean (eq. representation)
    if (!u_current) PM_TRY(S.enqueue_representation(1.0 / sw));
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
        info->residual_updates = updated;
    }
    return result;
}
