// div_G(a grad_G u) + c u = f for c != 0, real or complex (Sec. 4.2, Thm. second_kind):
// the Helmholtz (c/a > 0) and modified-Helmholtz (c/a < 0) parametrices of
// eq. diff_param, their remainder eq. explicit_remainder, the second-kind
// equation sigma + R~ sigma = f and the representation u = K~ sigma.  With
// c != 0 there is no null space: no rank-one term and no mean projection.
//
// Everything is complex (the Helmholtz kernel is -(i/4) H0(kr); the modified one
// -K0(kappa r)/(2 pi) is real, but one path serves both signs, a c whose sign
// changes over the surface and complex c, whose kernels take K0, K1 at complex
// argument, pm_green.cuh).  Arithmetic is float64 throughout:
//   - smooth sums: one thread per target, sources staged through shared memory,
//     split over gridDim.y, g, g', g'' from pm_green.cuh at every pair;
//   - near field: complex corrections from pm_nearfield.cu (pm_near_build_c);
//   - GMRES(m) with classical Gram-Schmidt applied twice; the Krylov vectors and
//     the orthogonalisation stay on the device, the (m+1) x m Hessenberg matrix and
//     its Givens rotations on the host (a few hundred bytes per step).
#include "pm_green.cuh"
#include "pm_internal.cuh"

#include <chrono>
#include <cmath>
#include <complex>
#include <vector>

namespace {

using cplx = std::complex<double>;
constexpr int kHT = 128;        // threads (targets) per block of the smooth sums
__constant__ double cHG16[2 * PM_GL16];   // 16-point Gauss-Legendre nodes, weights (complex q)
constexpr int kRT = 256;        // threads of the vector kernels

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// s_j = w_j sigma_j / a_j
__global__ void k_prep_c(const double2* __restrict__ sigma, const double* __restrict__ wa,
                         double2* __restrict__ sv, int N) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < N) sv[j] = make_double2(wa[j] * sigma[j].x, wa[j] * sigma[j].y);
}

// partial[y][i] = sum over the split's sources j != i of s_j a(y_j) G(x_i, x_j),
// G = R (WHICH = 0) or K (WHICH = 1).
template <int WHICH>
__global__ void __launch_bounds__(kHT)
k_direct_c64(const double* __restrict__ x, const double* __restrict__ n,
             const double* __restrict__ H, const double* __restrict__ a,
             const double* __restrict__ g, const double2* __restrict__ c,
             const double2* __restrict__ qn, const double2* __restrict__ sv, int N, int chunk,
             double2* __restrict__ partial) {
    __shared__ double4 sx[kHT];          // source x, y, z, Re q
    __shared__ double sqi[kHT];          // source Im q
    __shared__ double2 ss[kHT];          // source strength
    const int tid = threadIdx.x;
    const int i = blockIdx.x * kHT + tid;
    double xi[3] = {0, 0, 0}, ni[3] = {0, 0, 1}, gi[3] = {0, 0, 0}, Hi = 0, ai = 1;
    pm_green::cplx_d ci = {0.0, 0.0};
    if (i < N) {
        for (int d = 0; d < 3; ++d) {
            xi[d] = x[3 * i + d];
            ni[d] = n[3 * i + d];
            gi[d] = g[3 * i + d];
        }
        Hi = H[i];
        ai = a[i];
        ci = {c[i].x, c[i].y};
    }
    double are = 0.0, aim = 0.0;
    const int s0 = blockIdx.y * chunk;
    const int s1 = min(s0 + chunk, N);
    for (int base = s0; base < s1; base += kHT) {
        __syncthreads();
        const int j = base + tid;
        if (j < s1) {
            sx[tid] = make_double4(x[3 * j], x[3 * j + 1], x[3 * j + 2], qn[j].x);
            sqi[tid] = qn[j].y;
            ss[tid] = sv[j];
        }
        __syncthreads();
        const int len = min(kHT, s1 - base);
        if (i < N) {
            for (int jj = 0; jj < len; ++jj) {
                if (base + jj == i) continue;
                const double4 y = sx[jj];
                double out[4];
                pm_green::pair_rk_cz(xi[0] - y.x, xi[1] - y.y, xi[2] - y.z, ni[0], ni[1], ni[2],
                                     Hi, ai, gi[0], gi[1], gi[2], ci,
                                     pm_green::cplx_d{y.w, sqi[jj]}, cHG16, cHG16 + PM_GL16, out);
                const double2 kv = WHICH ? make_double2(out[2], out[3])
                                         : make_double2(out[0], out[1]);
                const double2 t = cmul(kv, ss[jj]);
                are += t.x;
                aim += t.y;
            }
        }
    }
    if (i < N) partial[(size_t)blockIdx.y * N + i] = make_double2(are, aim);
}

// out_i = sum_s partial[s][i] + sum_{b in row i} sum_k C[b][k] sigma[patch_b][k] (warp per row)
__global__ void k_near_apply_c64(int N, int pp, const int* __restrict__ row_ptr,
                                 const int* __restrict__ blk_patch, const double2* __restrict__ C,
                                 const double2* __restrict__ sigma,
                                 const double2* __restrict__ partial, int nsplit,
                                 double2* __restrict__ out) {
    const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (i >= N) return;
    double re = 0.0, im = 0.0;
    for (int sp = lane; sp < nsplit; sp += 32) {
        const double2 v = partial[(size_t)sp * N + i];
        re += v.x;
        im += v.y;
    }
    for (int b = row_ptr[i]; b < row_ptr[i + 1]; ++b) {
        const double2* cv = C + (size_t)b * pp;
        const double2* sg = sigma + (size_t)blk_patch[b] * pp;
        for (int k = lane; k < pp; k += 32) {
            const double2 t = cmul(cv[k], sg[k]);
            re += t.x;
            im += t.y;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_down_sync(0xffffffffu, re, o);
        im += __shfl_down_sync(0xffffffffu, im, o);
    }
    if (lane == 0) out[i] = make_double2(re, im);
}

// ------------------------------------------------------------------ Krylov kernels
// partial[blk * ncols + j] = sum over the block's rows of conj(V_j[i]) w[i]
__global__ void __launch_bounds__(kRT)
k_cdots(const double2* __restrict__ V, long long ldv, int ncols, const double2* __restrict__ w,
        int N, double2* __restrict__ partial) {
    __shared__ double2 sh[kRT / 32];
    const int stride = gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int j = 0; j < ncols; ++j) {
        const double2* v = V + j * ldv;
        double re = 0.0, im = 0.0;
        for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += stride) {
            const double2 a = v[i], b = w[i];
            re += a.x * b.x + a.y * b.y;
            im += a.x * b.y - a.y * b.x;
        }
        for (int o = 16; o > 0; o >>= 1) {
            re += __shfl_down_sync(0xffffffffu, re, o);
            im += __shfl_down_sync(0xffffffffu, im, o);
        }
        __syncthreads();
        if (lane == 0) sh[wid] = make_double2(re, im);
        __syncthreads();
        if (threadIdx.x == 0) {
            double2 t = make_double2(0.0, 0.0);
            for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
                t.x += sh[k].x;
                t.y += sh[k].y;
            }
            partial[blockIdx.x * ncols + j] = t;
        }
    }
}

// out[j] = sum_blk partial[blk * ncols + j] (fixed order)
__global__ void k_creduce(const double2* __restrict__ partial, int nblk, int ncols,
                          double2* __restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= ncols) return;
    double2 s = make_double2(0.0, 0.0);
    for (int b = 0; b < nblk; ++b) {
        s.x += partial[b * ncols + j].x;
        s.y += partial[b * ncols + j].y;
    }
    out[j] = s;
}

// w -= sum_{j < ncols} V_j h_j
__global__ void k_cupdate(const double2* __restrict__ V, long long ldv, int ncols,
                          const double2* __restrict__ h, double2* __restrict__ w, int N) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double2 acc = w[i];
    for (int j = 0; j < ncols; ++j) {
        const double2 t = cmul(V[j * ldv + i], h[j]);
        acc.x -= t.x;
        acc.y -= t.y;
    }
    w[i] = acc;
}

// out = s * v
__global__ void k_cscale(const double2* __restrict__ v, double s, double2* __restrict__ out, int N) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) out[i] = make_double2(s * v[i].x, s * v[i].y);
}

// out = alpha * u + beta * v (real alpha, beta)
__global__ void k_cadd(const double2* __restrict__ u, double alpha, const double2* __restrict__ v,
                       double beta, double2* __restrict__ out, int N) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N)
        out[i] = make_double2(alpha * u[i].x + beta * v[i].x, alpha * u[i].y + beta * v[i].y);
}

// x += sum_{j < n} V_j y_j
__global__ void k_ccombo(const double2* __restrict__ V, long long ldv, int n,
                         const double2* __restrict__ y, double2* __restrict__ x, int N) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double2 acc = x[i];
    for (int j = 0; j < n; ++j) {
        const double2 t = cmul(V[j * ldv + i], y[j]);
        acc.x += t.x;
        acc.y += t.y;
    }
    x[i] = acc;
}

}  // namespace

struct PmHelmWork {
    int N = 0, m = 0, nred = 0;
    double2 *V = nullptr, *w = nullptr, *tmp = nullptr, *x = nullptr, *f = nullptr;
    double2 *r = nullptr, *u = nullptr, *sv = nullptr, *io = nullptr;
    double2 *part = nullptr, *h = nullptr, *y = nullptr;
    double2* pinned = nullptr;          // host-pinned [2 (m + 2) + 1]
};

void pm_helm_free(pm_surface* s) {
    pm_dfree(s->cc); pm_dfree(s->qn); pm_dfree(s->cRc); pm_dfree(s->cKc);
    if (!s->helm) return;
    PmHelmWork& W = *s->helm;
    pm_dfree(W.V); pm_dfree(W.w); pm_dfree(W.tmp); pm_dfree(W.x); pm_dfree(W.f); pm_dfree(W.r);
    pm_dfree(W.u); pm_dfree(W.sv); pm_dfree(W.io); pm_dfree(W.part); pm_dfree(W.h); pm_dfree(W.y);
    if (W.pinned) cudaFreeHost(W.pinned);
    delete s->helm;
    s->helm = nullptr;
}

namespace {

pm_status helm_work_alloc(pm_surface* s, int m);

// Work buffers: the apply's (strengths, staging) always, the Krylov basis when
// m > 0 (reallocated when the restart length changes).  A failed allocation frees
// the work, so a partly allocated one is never reused.
pm_status helm_work(pm_surface* s, int m, PmHelmWork** out) {
    const pm_status st = helm_work_alloc(s, m);
    if (st != PM_OK) {
        if (s->helm) {
            PmHelmWork& W = *s->helm;
            pm_dfree(W.V); pm_dfree(W.w); pm_dfree(W.tmp); pm_dfree(W.x); pm_dfree(W.f);
            pm_dfree(W.r); pm_dfree(W.u); pm_dfree(W.sv); pm_dfree(W.io); pm_dfree(W.part);
            pm_dfree(W.h); pm_dfree(W.y);
            if (W.pinned) cudaFreeHost(W.pinned);
            delete s->helm;
            s->helm = nullptr;
        }
        return st;
    }
    *out = s->helm;
    return PM_OK;
}

pm_status helm_work_alloc(pm_surface* s, int m) {
    if (!s->helm) s->helm = new PmHelmWork();
    PmHelmWork& W = *s->helm;
    const int N = s->N;
    if (!W.sv) {
        W.N = N;
        PM_TRY(pm_dmalloc(&W.sv, N));
        PM_TRY(pm_dmalloc(&W.io, 2 * (size_t)N));
    }
    if (m > 0 && W.m != m) {
        pm_dfree(W.V); pm_dfree(W.w); pm_dfree(W.tmp); pm_dfree(W.x); pm_dfree(W.f);
        pm_dfree(W.r); pm_dfree(W.u); pm_dfree(W.part); pm_dfree(W.h); pm_dfree(W.y);
        if (W.pinned) cudaFreeHost(W.pinned);
        W.pinned = nullptr;
        W.m = m;
        W.nred = std::max(1, std::min(pm_ceil_div(N, 4 * kRT), 2 * s->ctx->num_sms));
        PM_TRY(pm_dmalloc(&W.V, (size_t)(m + 1) * N));
        PM_TRY(pm_dmalloc(&W.w, N));
        PM_TRY(pm_dmalloc(&W.tmp, N));
        PM_TRY(pm_dmalloc(&W.x, N));
        PM_TRY(pm_dmalloc(&W.f, N));
        PM_TRY(pm_dmalloc(&W.r, N));
        PM_TRY(pm_dmalloc(&W.u, N));
        PM_TRY(pm_dmalloc(&W.part, (size_t)W.nred * (m + 2)));
        PM_TRY(pm_dmalloc(&W.h, 2 * (size_t)(m + 2) + 1));
        PM_TRY(pm_dmalloc(&W.y, m + 1));
        PM_CUDA_TRY(cudaMallocHost((void**)&W.pinned, sizeof(double2) * (2 * (size_t)(m + 2) + 1)));
    }
    return PM_OK;
}

// out = R~ sigma (which_K = 0) or K~ sigma (1), complex device vectors
pm_status helm_apply(pm_surface* s, int which_K, const double2* sigma, double2* out,
                     cudaStream_t st) {
    PmHelmWork* W = nullptr;
    PM_TRY(helm_work(s, 0, &W));
    const int N = s->N;
    {
        PhaseTimer t(s, PM_PHASE_PREP, st);
        k_prep_c<<<pm_ceil_div(N, kRT), kRT, 0, st>>>(sigma, s->wa, W->sv, N);
    }
    // source splits: about four blocks per SM, at least 64 sources a split
    const int tblocks = pm_ceil_div(N, kHT);
    int nsplit = pm_ceil_div(4 * s->ctx->num_sms, tblocks);
    nsplit = std::max(1, std::min(nsplit, std::min(s->max_split / 2, std::max(1, N / 64))));
    const int chunk = pm_ceil_div(N, nsplit);
    dim3 grid(tblocks, nsplit);
    double2* part = reinterpret_cast<double2*>(s->partial);
    {
        // the float64 phases of the c = 0 sums time the c != 0 sums too
        PhaseTimer t(s, which_K ? PM_PHASE_DIRECT64_K : PM_PHASE_DIRECT64, st);
        if (which_K)
            k_direct_c64<1><<<grid, kHT, 0, st>>>(s->x, s->n, s->H, s->a, s->g, s->cc, s->qn,
                                                  W->sv, N, chunk, part);
        else
            k_direct_c64<0><<<grid, kHT, 0, st>>>(s->x, s->n, s->H, s->a, s->g, s->cc, s->qn,
                                                  W->sv, N, chunk, part);
    }
    PhaseTimer t(s, PM_PHASE_NEAR, st);
    k_near_apply_c64<<<pm_ceil_div((long long)N * 32, kRT), kRT, 0, st>>>(
        N, s->pp, s->row_ptr, s->blk_patch, which_K ? s->cKc : s->cRc, sigma, part, nsplit, out);
    PM_CUDA_TRY(cudaGetLastError());
    s->launch_total += 3;
    return PM_OK;
}

struct HelmSolver {
    pm_surface* s;
    PmHelmWork& W;
    cudaStream_t st;
    int grid;

    // dst[0..ncols) = V_j^H b on the device
    pm_status dots(const double2* V, long long ldv, int ncols, const double2* b, double2* dst) {
        k_cdots<<<W.nred, kRT, 0, st>>>(V, ldv, ncols, b, W.N, W.part);
        k_creduce<<<pm_ceil_div(ncols, 64), 64, 0, st>>>(W.part, W.nred, ncols, dst);
        PM_CUDA_TRY(cudaGetLastError());
        return PM_OK;
    }

    pm_status norm(const double2* v, double* out) {
        PM_TRY(dots(v, 0, 1, v, W.h));
        PM_CUDA_TRY(cudaMemcpyAsync(W.pinned, W.h, sizeof(double2), cudaMemcpyDeviceToHost, st));
        PM_CUDA_TRY(cudaStreamSynchronize(st));
        *out = std::sqrt(std::max(0.0, W.pinned[0].x));
        return PM_OK;
    }

    // out = (I + R~) v
    pm_status apply_A(const double2* v, double2* out) {
        PM_TRY(helm_apply(s, 0, v, W.tmp, st));
        k_cadd<<<grid, kRT, 0, st>>>(v, 1.0, W.tmp, 1.0, out, W.N);
        PM_CUDA_TRY(cudaGetLastError());
        return PM_OK;
    }

    // r = f - (I + R~) x
    pm_status residual() {
        PM_TRY(apply_A(W.x, W.w));
        k_cadd<<<grid, kRT, 0, st>>>(W.f, 1.0, W.w, -1.0, W.r, W.N);
        PM_CUDA_TRY(cudaGetLastError());
        return PM_OK;
    }
};

}  // namespace

extern "C" pm_status pm_surface_set_coeff_c(pm_surface* s, const double* a, const double* grad_a,
                                            const double* c) {
    if (!s || !a || !c) {
        pm_set_error("pm_surface_set_coeff_c: NULL argument");
        return PM_ERR_INVALID_ARG;
    }
    if (s->tri) {
        pm_set_error("pm_surface_set_coeff_c: c != 0 is built for quadrilateral patches only");
        return PM_ERR_INVALID_ARG;
    }
    const int N = s->N;
    bool any = false;
    for (int k = 0; k < N; ++k) {
        if (!std::isfinite(c[2 * k]) || !std::isfinite(c[2 * k + 1])) {
            pm_set_error("pm_surface_set_coeff_c: c[%d] = %g%+gi is not finite", k, c[2 * k],
                         c[2 * k + 1]);
            return PM_ERR_INVALID_ARG;
        }
        any = any || c[2 * k] != 0.0 || c[2 * k + 1] != 0.0;
    }
    // a and grad_a are checked, copied and packed by the c = 0 path, which also
    // leaves c = 0 surfaces exactly as pm_surface_set_coeff does
    PM_TRY(pm_surface_set_coeff(s, a, grad_a));
    if (!any) return PM_OK;
    pm_ffmat_free(s);                          // the real float-float sums do not apply to c != 0
    std::vector<double> q(2 * (size_t)N);
    for (int k = 0; k < N; ++k) {
        q[2 * k] = c[2 * k] / a[k];
        q[2 * k + 1] = c[2 * k + 1] / a[k];
    }
    if (!s->cc) {
        PM_TRY(pm_dmalloc(&s->cc, N));
        PM_TRY(pm_dmalloc(&s->qn, N));
        PM_TRY(pm_dmalloc(&s->cRc, (size_t)s->nblk * s->pp));
        PM_TRY(pm_dmalloc(&s->cKc, (size_t)s->nblk * s->pp));
    }
    PM_CUDA_TRY(cudaMemcpy(s->cc, c, sizeof(double2) * N, cudaMemcpyHostToDevice));
    PM_CUDA_TRY(cudaMemcpy(s->qn, q.data(), sizeof(double2) * N, cudaMemcpyHostToDevice));
    {
        QuadTables T;
        pm_build_tables(2, &T);
        double g16[2 * PM_GL16];
        for (int k = 0; k < PM_GL16; ++k) {
            g16[k] = T.g16t[k];
            g16[PM_GL16 + k] = T.g16w[k];
        }
        PM_CUDA_TRY(cudaMemcpyToSymbol(cHG16, g16, sizeof(g16)));
        PM_CUDA_TRY(pm_green::upload_cheb_k01());
    }
    PM_TRY(pm_near_build_c(s));
    s->has_c = 1;
    s->graph_epoch++;
    s->coeff_epoch++;
    return PM_OK;
}

extern "C" pm_status pm_apply_c(pm_surface* s, int which_K, const double* sigma, double* out,
                                int on_device, void* stream) {
    if (!s || !sigma || !out || (which_K != 0 && which_K != 1)) {
        pm_set_error("pm_apply_c: NULL argument or which_K not 0 / 1");
        return PM_ERR_INVALID_ARG;
    }
    if (!s->has_c) {
        pm_set_error("pm_apply_c: the surface has no c != 0 (call pm_surface_set_coeff_c)");
        return PM_ERR_NO_COEFF;
    }
    PM_CUDA_TRY(cudaSetDevice(s->ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    PmHelmWork* W = nullptr;
    PM_TRY(helm_work(s, 0, &W));
    const size_t bytes = sizeof(double2) * s->N;
    if (on_device) {
        PM_TRY(helm_apply(s, which_K, reinterpret_cast<const double2*>(sigma),
                          reinterpret_cast<double2*>(out), st));
        return PM_OK;
    }
    PM_CUDA_TRY(cudaMemcpyAsync(W->io, sigma, bytes, cudaMemcpyHostToDevice, st));
    PM_TRY(helm_apply(s, which_K, W->io, W->io + s->N, st));
    PM_CUDA_TRY(cudaMemcpyAsync(out, W->io + s->N, bytes, cudaMemcpyDeviceToHost, st));
    PM_CUDA_TRY(cudaStreamSynchronize(st));
    return PM_OK;
}

extern "C" pm_status pm_solve_c(pm_surface* s, const double* f, double* u, double tol, int maxit,
                                double* sigma_out, pm_solve_info* info) {
    const auto t0 = std::chrono::steady_clock::now();
    if (!s || !f || !u || !(tol > 0) || maxit < 1) {
        pm_set_error("pm_solve_c: NULL argument, tol <= 0 or maxit < 1");
        return PM_ERR_INVALID_ARG;
    }
    if (!s->has_c) {
        pm_set_error("pm_solve_c: the surface has no c != 0 (call pm_surface_set_coeff_c)");
        return PM_ERR_NO_COEFF;
    }
    PM_CUDA_TRY(cudaSetDevice(s->ctx->device));
    const int m = std::max(2, std::min(s->opts.gmres_restart, 400));
    PmHelmWork* Wp = nullptr;
    PM_TRY(helm_work(s, m, &Wp));
    PmHelmWork& W = *Wp;
    const int N = s->N;
    cudaStream_t st = 0;
    HelmSolver S{s, W, st, pm_ceil_div(N, kRT)};
    const size_t bytes = sizeof(double2) * N;
    PM_CUDA_TRY(cudaMemcpyAsync(W.f, f, bytes, cudaMemcpyHostToDevice, st));
    PM_CUDA_TRY(cudaMemsetAsync(W.x, 0, bytes, st));
    double fnorm = 0.0;
    PM_TRY(S.norm(W.f, &fnorm));
    int iters = 0, cycles = 0;
    double relres = 0.0;
    pm_status result = PM_OK;
    if (fnorm > 0.0) {
        PM_CUDA_TRY(cudaMemcpyAsync(W.r, W.f, bytes, cudaMemcpyDeviceToDevice, st));
        std::vector<cplx> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
        const long long ldv = N;
        for (;;) {
            double beta = 0.0;
            PM_TRY(S.norm(W.r, &beta));
            relres = beta / fnorm;
            if (relres <= tol || iters >= maxit) break;
            // one cycle of GMRES(m) on A d = r, x += d
            k_cscale<<<S.grid, kRT, 0, st>>>(W.r, 1.0 / beta, W.V, N);
            std::fill(g.begin(), g.end(), cplx(0.0));
            g[0] = beta;
            int k = 0;
            for (; k < m && iters < maxit; ++k) {
                double2* vk = W.V + (size_t)k * ldv;
                PM_TRY(S.apply_A(vk, W.w));
                // classical Gram-Schmidt, twice: h = V^H w, w -= V h; h2 = V^H w, w -= V h2
                PM_TRY(S.dots(W.V, ldv, k + 1, W.w, W.h));
                k_cupdate<<<S.grid, kRT, 0, st>>>(W.V, ldv, k + 1, W.h, W.w, N);
                PM_TRY(S.dots(W.V, ldv, k + 1, W.w, W.h + (m + 2)));
                k_cupdate<<<S.grid, kRT, 0, st>>>(W.V, ldv, k + 1, W.h + (m + 2), W.w, N);
                PM_TRY(S.dots(W.w, 0, 1, W.w, W.h + 2 * (m + 2)));
                PM_CUDA_TRY(cudaMemcpyAsync(W.pinned, W.h, sizeof(double2) * (2 * (size_t)(m + 2) + 1),
                                            cudaMemcpyDeviceToHost, st));
                PM_CUDA_TRY(cudaStreamSynchronize(st));
                const double hn = std::sqrt(std::max(0.0, W.pinned[2 * (m + 2)].x));
                cplx* col = &H[(size_t)k * (m + 1)];
                for (int j = 0; j <= k; ++j)
                    col[j] = cplx(W.pinned[j].x + W.pinned[m + 2 + j].x,
                                  W.pinned[j].y + W.pinned[m + 2 + j].y);
                col[k + 1] = hn;
                ++iters;
                if (hn > 0.0)
                    k_cscale<<<S.grid, kRT, 0, st>>>(W.w, 1.0 / hn, W.V + (size_t)(k + 1) * ldv, N);
                // the earlier rotations, then a new one that zeroes col[k + 1]:
                // [c s; -conj(s) c] [a; b] = [rho; 0], c = |a|/t, s = (a/|a|) conj(b)/t
                for (int j = 0; j < k; ++j) {
                    const cplx t = cs[j] * col[j] + sn[j] * col[j + 1];
                    col[j + 1] = -std::conj(sn[j]) * col[j] + cs[j] * col[j + 1];
                    col[j] = t;
                }
                const cplx av = col[k], bv = col[k + 1];
                const double t = std::sqrt(std::norm(av) + std::norm(bv));
                if (t == 0.0) {
                    cs[k] = 1.0;
                    sn[k] = 0.0;
                } else if (std::abs(av) == 0.0) {
                    cs[k] = 0.0;
                    sn[k] = std::conj(bv) / t;
                } else {
                    const cplx ph = av / std::abs(av);
                    cs[k] = std::abs(av) / t;
                    sn[k] = ph * std::conj(bv) / t;
                }
                col[k] = cs[k] * av + sn[k] * bv;
                col[k + 1] = 0.0;
                g[k + 1] = -std::conj(sn[k]) * g[k];
                g[k] = cs[k] * g[k];
                if (std::abs(g[k + 1]) <= tol * fnorm || hn == 0.0) {
                    ++k;
                    break;
                }
            }
            // y = H(0:k, 0:k)^-1 g(0:k), x += V y
            for (int i = k - 1; i >= 0; --i) {
                cplx t = g[i];
                for (int j = i + 1; j < k; ++j) t -= H[(size_t)j * (m + 1) + i] * y[j];
                const cplx d = H[(size_t)i * (m + 1) + i];
                y[i] = (std::abs(d) > 0.0) ? t / d : cplx(0.0);
            }
            for (int i = 0; i < k; ++i) W.pinned[i] = make_double2(y[i].real(), y[i].imag());
            PM_CUDA_TRY(cudaMemcpyAsync(W.y, W.pinned, sizeof(double2) * k, cudaMemcpyHostToDevice, st));
            k_ccombo<<<S.grid, kRT, 0, st>>>(W.V, ldv, k, W.y, W.x, N);
            PM_CUDA_TRY(cudaGetLastError());
            ++cycles;
            PM_TRY(S.residual());            // the true residual of the new x
            if (k == 0) {
                PM_TRY(S.norm(W.r, &beta));
                relres = beta / fnorm;
                break;
            }
        }
        if (!(relres <= tol)) {
            pm_set_error("pm_solve_c: relative residual %.3e above %.3e after %d iterations",
                         relres, tol, iters);
            result = PM_ERR_NOT_CONVERGED;
        }
    }
    // u = K~ sigma (eq. representation; no projection for c != 0)
    PM_TRY(helm_apply(s, 1, W.x, W.u, st));
    PM_CUDA_TRY(cudaMemcpyAsync(u, W.u, bytes, cudaMemcpyDeviceToHost, st));
    if (sigma_out) PM_CUDA_TRY(cudaMemcpyAsync(sigma_out, W.x, bytes, cudaMemcpyDeviceToHost, st));
    PM_CUDA_TRY(cudaStreamSynchronize(st));
    if (info) {
        info->iterations = iters;
        info->refinements = cycles;
        info->residual = relres;
        info->removed_mean = 0.0;
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        info->residual_updates = 0;
    }
    return result;
}
