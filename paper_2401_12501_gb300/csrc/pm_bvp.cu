// Boundary-value systems on an open surface: Neumann (Sec. 5.2, eq. NeuBVPsystem) and,
// for a constant coefficient, Dirichlet (Sec. 5.3, eq. DirBVPsystem).
//
// Gamma is a surface built from an open surface's patches (pm_surface_create +
// pm_surface_set_coeff); its boundary gamma is a union of closed curves given at
// edge nodes t_k = 2 pi (k + 1/2) / M of a periodic parameter and at F M oversampled
// points t_j = 2 pi j / (F M).  Unknowns sigma [N] and mu [Me]:
//
//   sigma + R~_Gamma sigma + R_gamma mu                          = f        (surface rows)
//   -mu / (2a) + K'_Gamma sigma + K'_gamma mu + (sum_k w_k mu_k)  = f_gamma  (edge rows)
//   u = K~_Gamma sigma + K_gamma mu                               (eq. BC_rep)
//
// with K = log r / (2 pi a(x')), R of eq. explicit_remainder (c = 0), K' = nu . grad_x K
// at edge nodes (nu the binormal).  The rank-one term removes the one-dimensional null
// space (constants solve the homogeneous Neumann problem); any multiple of it gives the
// same u up to a constant for consistent data.
//
// Dirichlet, a constant (the paper proves T_gamma compact for constant a only):
//
//   sigma + R~_Gamma sigma + T_gamma mu                 = f        (surface rows)
//   +mu / (2a) + K~_Gamma sigma + N_gamma mu            = f_gamma  (edge rows: the trace)
//   u = K~_Gamma sigma + N_gamma mu
//
// N_gamma the double layer nu(x') . grad_x' K, T_gamma = nu(x') . grad_x' R; the trace of
// the double layer from inside is +mu/(2a) plus its value on gamma (the paper prints
// -mu/(2a); Gauss's lemma fixes the sign), and the edge row carries K_Gamma[sigma], as
// the trace theorem states (the printed system writes N_Gamma there).  K~_Gamma at the
// edge nodes: smooth rule plus corrections (polar rule with dyadic radial panels on the
// edge patch, quadtree near rule on the others); N_gamma on gamma: trapezoid rule, its
// diagonal the limit -nu . gamma'' / (4 pi a |gamma'|^2); T_gamma and N_gamma off gamma:
// the oversampled trapezoid rule.
//
// Discretisation (Sec. 6.1.4 with the surface rules of Sec. 6.1):
// * R~_Gamma, K~_Gamma: the surface's float64 applies (smooth sums + near corrections).
// * R_gamma, K_gamma: trapezoid rule on the oversampled points, mu carried there by the
//   trigonometric interpolant (degree < M/2 and the symmetric Nyquist term), the paper's
//   Fourier oversampling; a(x') at the oversampled points.
// * K'_gamma: trapezoid rule on the edge nodes, the diagonal entry the limit of the smooth
//   kernel along the curve, nu . (x - y) / |x - y|^2 -> -nu . gamma'' / (2 |gamma'|^2).
// * K'_Gamma: the smooth rule over all surface nodes plus corrections on the patches near
//   each edge node (pm_nearfield.cu k_bvp_kp_quad: polar rule about the edge point on its
//   own patch, the quadtree near rule on the others).
// Everything runs in float64; the solver is restarted GMRES with classical Gram-Schmidt
// and one reorthogonalisation, the Hessenberg system on the host.
#include "pm_internal.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <vector>

pm_status pm_bvp_kp_weights(pm_surface* s, int nb, const int* blk_edge, const int* blk_patch,
                            const int* blk_own, const double* xe, const double* nue,
                            const double* uv, int log_kernel, double* W);

struct pm_bvp {
    pm_surface* s = nullptr;
    int kind = 0;                        // 0 Neumann, 1 Dirichlet
    long long coeff_epoch = 0;           // the surface's coefficient epoch at creation
    int N = 0, Me = 0, Fo = 0, ncurves = 0;
    std::vector<int> M, F, off, offo;
    std::vector<double> h_we;
    double *xe = nullptr, *nue = nullptr, *we = nullptr, *ae = nullptr, *uv = nullptr;
    double *xo = nullptr, *wo = nullptr, *ao = nullptr, *nuo = nullptr;
    double *interp = nullptr;            // per curve [F M][M], curve blocks concatenated
    int *interp_off = nullptr;           // [ncurves + 1] offsets into interp
    int *curve_of = nullptr;             // [Fo] curve of an oversampled point
    double *Kpg = nullptr;               // [Me][Me] K'_gamma (Neumann) or N_gamma (Dirichlet), weighted
    int *kp_ptr = nullptr, *kp_patch = nullptr;
    double *kp_C = nullptr;              // [nblk][pp] K'_Gamma (K_Gamma) corrections
    int kp_nblk = 0;
    double *mu_o = nullptr;              // [Fo]
    double *part = nullptr;              // dot partials
    cudaStream_t st = nullptr;
};

namespace {

constexpr int kT = 256;
constexpr int kDotBlocks = 128;
constexpr int kTile = 256;

// mu_o[j] = sum_k I_c[j][k] mu[off_c + k] for the curve c of oversampled point j
__global__ void k_bvp_interp(const double* __restrict__ I, const int* __restrict__ ioff,
                             const int* __restrict__ curve_of, const int* __restrict__ offo,
                             const int* __restrict__ off, const int* __restrict__ Mc,
                             const double* __restrict__ mu, double* __restrict__ mu_o, int Fo) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= Fo) return;
    const int c = curve_of[j];
    const int m = Mc[c], jl = j - offo[c];
    const double* row = I + ioff[c] + (size_t)jl * m;
    const double* mc = mu + off[c];
    double s = 0.0;
    for (int k = 0; k < m; ++k) s += row[k] * mc[k];
    mu_o[j] = s;
}

// out[i] += sum_j wo_j mu_o_j G(x_i, xo_j) with r = x_i - xo_j: KIND 0 the remainder
// R / a(x') (target n, H, a, grad a), 1 the parametrix log r / (2 pi a(x')), 2 T =
// nu' . grad' R for constant a (the a's cancel), 3 the double layer
// -nu' . r / (2 pi a r^2)
enum { kEdgeR = 0, kEdgeK = 1, kEdgeT = 2, kEdgeN = 3 };
template <int KIND>
__global__ void __launch_bounds__(kT)
k_bvp_edge_to_surface(int N, const double* __restrict__ x, const double* __restrict__ n,
                      const double* __restrict__ H, const double* __restrict__ a,
                      const double* __restrict__ g, int Fo, const double* __restrict__ xo,
                      const double* __restrict__ wo, const double* __restrict__ ao,
                      const double* __restrict__ nuo, const double* __restrict__ mu_o,
                      double* __restrict__ out) {
    constexpr bool WHICH_K = KIND == kEdgeK || KIND == kEdgeN;
    __shared__ double sx[kTile], sy[kTile], sz[kTile], ss[kTile];
    __shared__ double su[KIND >= kEdgeT ? kTile : 1], sv[KIND >= kEdgeT ? kTile : 1],
        sw[KIND >= kEdgeT ? kTile : 1];
    const int i = blockIdx.x * kT + threadIdx.x;
    double xi0 = 0, xi1 = 0, xi2 = 0, n0 = 0, n1 = 0, n2 = 0, Hi = 0, ai = 0, g0 = 0, g1 = 0, g2 = 0;
    if (i < N) {
        xi0 = x[3 * i]; xi1 = x[3 * i + 1]; xi2 = x[3 * i + 2];
        if (KIND == kEdgeR || KIND == kEdgeT) {
            n0 = n[3 * i]; n1 = n[3 * i + 1]; n2 = n[3 * i + 2];
            Hi = H[i]; ai = a[i];
            g0 = g[3 * i]; g1 = g[3 * i + 1]; g2 = g[3 * i + 2];
        }
    }
    double acc = 0.0;
    for (int base = 0; base < Fo; base += kTile) {
        __syncthreads();
        const int j = base + threadIdx.x;
        if (j < Fo) {
            sx[threadIdx.x] = xo[3 * j];
            sy[threadIdx.x] = xo[3 * j + 1];
            sz[threadIdx.x] = xo[3 * j + 2];
            ss[threadIdx.x] = KIND == kEdgeT ? wo[j] * mu_o[j] : wo[j] * mu_o[j] / ao[j];
            if (KIND >= kEdgeT) {
                su[threadIdx.x] = nuo[3 * j];
                sv[threadIdx.x] = nuo[3 * j + 1];
                sw[threadIdx.x] = nuo[3 * j + 2];
            }
        }
        __syncthreads();
        const int cnt = min(kTile, Fo - base);
        if (i < N)
            for (int q = 0; q < cnt; ++q) {
                const double r0 = xi0 - sx[q], r1 = xi1 - sy[q], r2 = xi2 - sz[q];
                const double rr = r0 * r0 + r1 * r1 + r2 * r2;
                if (KIND == kEdgeK) {
                    acc += ss[q] * log(rr);
                } else if (KIND == kEdgeR) {
                    const double inv = 1.0 / rr;
                    const double qn = (n0 * r0 + n1 * r1 + n2 * r2) * inv;
                    acc += ss[q] * (ai * (qn * qn - Hi * qn) * (1.0 / M_PI) +
                                    (g0 * r0 + g1 * r1 + g2 * r2) * inv * (0.5 / M_PI));
                } else if (KIND == kEdgeN) {
                    acc -= ss[q] * (su[q] * r0 + sv[q] * r1 + sw[q] * r2) / rr;
                } else {
                    // -(1/pi) [2 (n.r)(n.nu')/r^4 - 4 (n.r)^2 (r.nu')/r^6 - H (n.nu')/r^2
                    //          + 2 H (n.r)(r.nu')/r^4]
                    const double inv = 1.0 / rr;
                    const double nr = n0 * r0 + n1 * r1 + n2 * r2;
                    const double nnu = n0 * su[q] + n1 * sv[q] + n2 * sw[q];
                    const double rnu = r0 * su[q] + r1 * sv[q] + r2 * sw[q];
                    acc -= ss[q] * inv * (2.0 * nr * nnu * inv - 4.0 * nr * nr * rnu * inv * inv -
                                          Hi * nnu + 2.0 * Hi * nr * rnu * inv);
                }
            }
    }
    if (i < N)
        out[i] += KIND == kEdgeK ? acc * (0.25 / M_PI)
                  : KIND == kEdgeN ? acc * (0.5 / M_PI)
                  : KIND == kEdgeT ? acc * (1.0 / M_PI) : acc;
}

__device__ double block_sum(double v, double* red) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) red[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
    return t;
}

// edge rows: one block per edge node e; Neumann (dirichlet = 0): K'_Gamma sigma +
// K'_gamma mu - mu/(2a) + sum w mu; Dirichlet: K_Gamma sigma + N_gamma mu + mu/(2a)
__global__ void __launch_bounds__(kT)
k_bvp_edge_row(int dirichlet, int N, int Me, int pp, const double* __restrict__ x,
               const double* __restrict__ wa,
               const double* __restrict__ xe, const double* __restrict__ nue,
               const double* __restrict__ ae, const double* __restrict__ we,
               const int* __restrict__ kp_ptr, const int* __restrict__ kp_patch,
               const double* __restrict__ kp_C, const double* __restrict__ Kpg,
               const double* __restrict__ sigma, const double* __restrict__ mu,
               double* __restrict__ out) {
    __shared__ double red[kT / 32];
    const int e = blockIdx.x;
    const double x0 = xe[3 * e], x1 = xe[3 * e + 1], x2 = xe[3 * e + 2];
    const double n0 = nue[3 * e], n1 = nue[3 * e + 1], n2 = nue[3 * e + 2];
    double acc = 0.0;
    for (int j = threadIdx.x; j < N; j += kT) {
        const double r0 = x0 - x[3 * j], r1 = x1 - x[3 * j + 1], r2 = x2 - x[3 * j + 2];
        const double rr = r0 * r0 + r1 * r1 + r2 * r2;
        acc += wa[j] * sigma[j] * (dirichlet ? 0.5 * log(rr) : (n0 * r0 + n1 * r1 + n2 * r2) / rr);
    }
    acc *= 0.5 / M_PI;
    for (int b = kp_ptr[e]; b < kp_ptr[e + 1]; ++b) {
        const double* C = kp_C + (size_t)b * pp;
        const double* sg = sigma + (size_t)kp_patch[b] * pp;
        for (int k = threadIdx.x; k < pp; k += kT) acc += C[k] * sg[k];
    }
    for (int k = threadIdx.x; k < Me; k += kT)
        acc += (Kpg[(size_t)e * Me + k] + (dirichlet ? 0.0 : we[k])) * mu[k];
    const double t = block_sum(acc, red);
    if (threadIdx.x == 0) out[e] = t + (dirichlet ? 0.5 : -0.5) * mu[e] / ae[e];
}

// C[b][k] = W[b][k] / a_k - w_k G(x_e, x_k) / a_k with G = nu_e . (x_e - x_k) / (2 pi |.|^2)
// (Neumann) or log|x_e - x_k| / (2 pi) (Dirichlet)
__global__ void k_bvp_combine(int dirichlet, int nblk, int pp, const int* __restrict__ blk_edge,
                              const int* __restrict__ blk_patch, const double* __restrict__ x,
                              const double* __restrict__ a, const double* __restrict__ w,
                              const double* __restrict__ xe, const double* __restrict__ nue,
                              double* __restrict__ C) {
    const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= (size_t)nblk * pp) return;
    const int b = (int)(q / pp), k = (int)(q - (size_t)b * pp);
    const int e = blk_edge[b];
    const size_t j = (size_t)blk_patch[b] * pp + k;
    const double r0 = xe[3 * e] - x[3 * j], r1 = xe[3 * e + 1] - x[3 * j + 1],
                 r2 = xe[3 * e + 2] - x[3 * j + 2];
    const double rr = r0 * r0 + r1 * r1 + r2 * r2;
    const double G = dirichlet ? 0.5 * log(rr)
                               : (nue[3 * e] * r0 + nue[3 * e + 1] * r1 + nue[3 * e + 2] * r2) / rr;
    const double smooth = w[j] * G * (0.5 / M_PI) / a[j];
    C[q] = C[q] / a[j] - smooth;
}

__global__ void k_bvp_axpy(int n, double alpha, const double* __restrict__ xv, double* __restrict__ y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] += alpha * xv[i];
}

// partial[j][b] = sum over block b's share of V[j] . w, j < nv
__global__ void k_bvp_dots(int n, int nv, const double* __restrict__ V, const double* __restrict__ w,
                           double* __restrict__ partial) {
    __shared__ double red[kT / 32];
    const int j = blockIdx.y;
    const double* v = V + (size_t)j * n;
    double acc = 0.0;
    for (int i = blockIdx.x * kT + threadIdx.x; i < n; i += gridDim.x * kT) acc += v[i] * w[i];
    const double t = block_sum(acc, red);
    if (threadIdx.x == 0) partial[(size_t)j * gridDim.x + blockIdx.x] = t;
}

// w -= sum_j h_j V[j]
__global__ void k_bvp_sub(int n, int nv, const double* __restrict__ V, const double* __restrict__ h,
                          double* __restrict__ w) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int j = 0; j < nv; ++j) s += h[j] * V[(size_t)j * n + i];
    w[i] -= s;
}

__global__ void k_bvp_scale(int n, double a, const double* __restrict__ xv, double* __restrict__ y) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = a * xv[i];
}

pm_status dots(pm_bvp* b, const double* V, int nv, const double* w, int n, std::vector<double>& out) {
    dim3 grid(kDotBlocks, nv);
    k_bvp_dots<<<grid, kT, 0, b->st>>>(n, nv, V, w, b->part);
    PM_CUDA_TRY(cudaGetLastError());
    std::vector<double> h((size_t)nv * kDotBlocks);
    PM_CUDA_TRY(cudaMemcpyAsync(h.data(), b->part, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, b->st));
    PM_CUDA_TRY(cudaStreamSynchronize(b->st));
    out.assign(nv, 0.0);
    for (int j = 0; j < nv; ++j)
        for (int k = 0; k < kDotBlocks; ++k) out[j] += h[(size_t)j * kDotBlocks + k];
    return PM_OK;
}

// the system's operator on z = [sigma; mu] (device), out = [surface rows; edge rows]
pm_status apply_sys(pm_bvp* b, const double* z, double* out) {
    pm_surface* s = b->s;
    const int N = b->N;
    cudaStream_t st = b->st;
    PM_TRY(pm_apply_dev(s, 0, 1, 1, z, out, PM_PREC_FP64, st));
    k_bvp_axpy<<<pm_ceil_div(N, kT), kT, 0, st>>>(N, 1.0, z, out);
    if (b->Me > 0) {
        k_bvp_interp<<<pm_ceil_div(b->Fo, kT), kT, 0, st>>>(
            b->interp, b->interp_off, b->curve_of, b->interp_off + b->ncurves + 1,
            b->interp_off + 2 * (b->ncurves + 1), b->interp_off + 3 * (b->ncurves + 1), z + N,
            b->mu_o, b->Fo);
        if (b->kind)
            k_bvp_edge_to_surface<kEdgeT><<<pm_ceil_div(N, kT), kT, 0, st>>>(
                N, s->x, s->n, s->H, s->a, s->g, b->Fo, b->xo, b->wo, b->ao, b->nuo, b->mu_o, out);
        else
            k_bvp_edge_to_surface<kEdgeR><<<pm_ceil_div(N, kT), kT, 0, st>>>(
                N, s->x, s->n, s->H, s->a, s->g, b->Fo, b->xo, b->wo, b->ao, b->nuo, b->mu_o, out);
        k_bvp_edge_row<<<b->Me, kT, 0, st>>>(b->kind, N, b->Me, s->pp, s->x, s->wa, b->xe, b->nue, b->ae,
                                             b->we, b->kp_ptr, b->kp_patch, b->kp_C, b->Kpg, z,
                                             z + N, out + N);
    }
    PM_CUDA_TRY(cudaGetLastError());
    return PM_OK;
}

pm_status represent(pm_bvp* b, const double* z, double* u) {
    pm_surface* s = b->s;
    const int N = b->N;
    cudaStream_t st = b->st;
    PM_TRY(pm_apply_dev(s, 1, 1, 1, z, u, PM_PREC_FP64, st));
    if (b->Me > 0) {
        k_bvp_interp<<<pm_ceil_div(b->Fo, kT), kT, 0, st>>>(
            b->interp, b->interp_off, b->curve_of, b->interp_off + b->ncurves + 1,
            b->interp_off + 2 * (b->ncurves + 1), b->interp_off + 3 * (b->ncurves + 1), z + N,
            b->mu_o, b->Fo);
        if (b->kind)
            k_bvp_edge_to_surface<kEdgeN><<<pm_ceil_div(N, kT), kT, 0, st>>>(
                N, s->x, s->n, s->H, s->a, s->g, b->Fo, b->xo, b->wo, b->ao, b->nuo, b->mu_o, u);
        else
            k_bvp_edge_to_surface<kEdgeK><<<pm_ceil_div(N, kT), kT, 0, st>>>(
                N, s->x, s->n, s->H, s->a, s->g, b->Fo, b->xo, b->wo, b->ao, b->nuo, b->mu_o, u);
    }
    PM_CUDA_TRY(cudaGetLastError());
    return PM_OK;
}

void free_bvp(pm_bvp* b) {
    if (!b) return;
    if (b->s) cudaSetDevice(b->s->ctx->device);
    pm_dfree(b->xe); pm_dfree(b->nue); pm_dfree(b->we); pm_dfree(b->ae); pm_dfree(b->uv);
    pm_dfree(b->xo); pm_dfree(b->wo); pm_dfree(b->ao); pm_dfree(b->nuo); pm_dfree(b->interp);
    pm_dfree(b->interp_off);
    pm_dfree(b->curve_of); pm_dfree(b->Kpg); pm_dfree(b->kp_ptr); pm_dfree(b->kp_patch);
    pm_dfree(b->kp_C); pm_dfree(b->mu_o); pm_dfree(b->part);
    delete b;
}

template <typename T>
pm_status upload(T** d, const T* h, size_t n) {
    PM_TRY(pm_dmalloc(d, n));
    if (n) PM_CUDA_TRY(cudaMemcpy(*d, h, sizeof(T) * n, cudaMemcpyHostToDevice));
    return PM_OK;
}

pm_status create_impl(pm_bvp* b, const double* edge_x, const double* edge_d1,
                      const double* edge_d2, const double* edge_nu, const double* edge_a,
                      const int* edge_patch, const double* edge_uv, const double* over_x,
                      const double* over_nu, const double* over_speed, const double* over_a) {
    pm_surface* s = b->s;
    const int Me = b->Me, Fo = b->Fo, pp = s->pp;
    // trapezoid weights, K'_gamma (host, dense), interpolation matrices
    b->h_we.resize(Me);
    std::vector<double> wo(Fo), Kpg((size_t)Me * Me), I;
    std::vector<int> ioff(4 * (b->ncurves + 1), 0), curve_of(Fo);
    for (int c = 0; c < b->ncurves; ++c) {
        const int m = b->M[c], f = b->F[c];
        for (int k = 0; k < m; ++k) {
            const int e = b->off[c] + k;
            const double* d1 = edge_d1 + 3 * e;
            b->h_we[e] = (2.0 * M_PI / m) * std::sqrt(d1[0] * d1[0] + d1[1] * d1[1] + d1[2] * d1[2]);
        }
        for (int j = 0; j < f * m; ++j) {
            wo[b->offo[c] + j] = (2.0 * M_PI / (f * m)) * over_speed[b->offo[c] + j];
            curve_of[b->offo[c] + j] = c;
        }
        ioff[c] = (int)I.size();
        const int nyq = (m % 2 == 0) ? m / 2 : 0;
        for (int j = 0; j < f * m; ++j) {
            const double tj = 2.0 * M_PI * j / (f * m);
            for (int k = 0; k < m; ++k) {
                const double d = tj - 2.0 * M_PI * (k + 0.5) / m;
                double v = 1.0;
                for (int q = 1; q <= (m - 1) / 2; ++q) v += 2.0 * std::cos(q * d);
                if (nyq) v += std::cos(nyq * d);
                I.push_back(v / m);
            }
        }
    }
    const int nc1 = b->ncurves + 1;
    ioff[b->ncurves] = (int)I.size();
    for (int c = 0; c < nc1; ++c) {
        ioff[nc1 + c] = c < b->ncurves ? b->offo[c] : Fo;
        ioff[2 * nc1 + c] = c < b->ncurves ? b->off[c] : Me;
        ioff[3 * nc1 + c] = c < b->ncurves ? b->M[c] : 0;
    }
    for (int e = 0; e < Me; ++e) {
        const double* xe_ = edge_x + 3 * e;
        const double* ne = edge_nu + 3 * e;
        for (int k = 0; k < Me; ++k) {
            double v;
            if (k == e) {
                const double* d1 = edge_d1 + 3 * e;
                const double* d2 = edge_d2 + 3 * e;
                const double sp2 = d1[0] * d1[0] + d1[1] * d1[1] + d1[2] * d1[2];
                v = -(ne[0] * d2[0] + ne[1] * d2[1] + ne[2] * d2[2]) / (2.0 * sp2);
            } else {
                const double r0 = xe_[0] - edge_x[3 * k], r1 = xe_[1] - edge_x[3 * k + 1],
                             r2 = xe_[2] - edge_x[3 * k + 2];
                // Neumann: nu(x_e) . r;  Dirichlet (double layer): -nu(x_k) . r
                const double* nn = b->kind ? edge_nu + 3 * k : ne;
                const double sg = b->kind ? -1.0 : 1.0;
                v = sg * (nn[0] * r0 + nn[1] * r1 + nn[2] * r2) / (r0 * r0 + r1 * r1 + r2 * r2);
            }
            Kpg[(size_t)e * Me + k] = b->h_we[k] * v / (2.0 * M_PI * edge_a[k]);
        }
    }
    // near patches of each edge node: its own patch first, then every patch within
    // near_factor radii of the node
    std::vector<double> cen(3 * (size_t)s->npatch), rad(s->npatch);
    PM_CUDA_TRY(cudaMemcpy(cen.data(), s->centroid, sizeof(double) * cen.size(), cudaMemcpyDeviceToHost));
    PM_CUDA_TRY(cudaMemcpy(rad.data(), s->radius, sizeof(double) * rad.size(), cudaMemcpyDeviceToHost));
    std::vector<int> kp_ptr(Me + 1, 0), kp_patch, blk_edge, blk_own;
    for (int e = 0; e < Me; ++e) {
        const int own = edge_patch[e];
        kp_patch.push_back(own);
        blk_edge.push_back(e);
        blk_own.push_back(1);
        for (int P = 0; P < s->npatch; ++P) {
            if (P == own) continue;
            const double d0 = edge_x[3 * e] - cen[3 * P], d1 = edge_x[3 * e + 1] - cen[3 * P + 1],
                         d2 = edge_x[3 * e + 2] - cen[3 * P + 2];
            if (std::sqrt(d0 * d0 + d1 * d1 + d2 * d2) < s->opts.near_factor * rad[P]) {
                kp_patch.push_back(P);
                blk_edge.push_back(e);
                blk_own.push_back(0);
            }
        }
        kp_ptr[e + 1] = (int)kp_patch.size();
    }
    b->kp_nblk = (int)kp_patch.size();
    int *d_be = nullptr, *d_own = nullptr;
    PM_TRY(upload(&b->xe, edge_x, 3 * (size_t)Me));
    PM_TRY(upload(&b->nue, edge_nu, 3 * (size_t)Me));
    PM_TRY(upload(&b->we, b->h_we.data(), (size_t)Me));
    PM_TRY(upload(&b->ae, edge_a, (size_t)Me));
    PM_TRY(upload(&b->uv, edge_uv, 2 * (size_t)Me));
    PM_TRY(upload(&b->xo, over_x, 3 * (size_t)Fo));
    PM_TRY(upload(&b->wo, wo.data(), (size_t)Fo));
    PM_TRY(upload(&b->ao, over_a, (size_t)Fo));
    PM_TRY(upload(&b->nuo, over_nu, 3 * (size_t)Fo));
    PM_TRY(upload(&b->interp, I.data(), I.size()));
    PM_TRY(upload(&b->interp_off, ioff.data(), ioff.size()));
    PM_TRY(upload(&b->curve_of, curve_of.data(), curve_of.size()));
    PM_TRY(upload(&b->Kpg, Kpg.data(), Kpg.size()));
    PM_TRY(upload(&b->kp_ptr, kp_ptr.data(), kp_ptr.size()));
    PM_TRY(upload(&b->kp_patch, kp_patch.data(), kp_patch.size()));
    PM_TRY(pm_dmalloc(&b->kp_C, (size_t)b->kp_nblk * pp));
    PM_TRY(pm_dmalloc(&b->mu_o, (size_t)std::max(Fo, 1)));
    PM_TRY(pm_dmalloc(&b->part, (size_t)kDotBlocks * 128));
    pm_status stt = upload(&d_be, blk_edge.data(), blk_edge.size());
    if (stt == PM_OK) stt = upload(&d_own, blk_own.data(), blk_own.size());
    if (stt == PM_OK)
        stt = pm_bvp_kp_weights(s, b->kp_nblk, d_be, b->kp_patch, d_own, b->xe, b->nue, b->uv,
                                b->kind, b->kp_C);
    if (stt == PM_OK && b->kp_nblk > 0) {
        k_bvp_combine<<<pm_ceil_div((long long)b->kp_nblk * pp, kT), kT>>>(
            b->kind, b->kp_nblk, pp, d_be, b->kp_patch, s->x, s->a, s->w, b->xe, b->nue, b->kp_C);
        if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
            pm_set_error("pm_bvp_create: correction kernel failed");
            stt = PM_ERR_CUDA;
        }
    }
    pm_dfree(d_be);
    pm_dfree(d_own);
    return stt;
}

}  // namespace

extern "C" pm_status pm_bvp_create(pm_surface* s, int kind, int ncurves, const int* M,
                                   const int* F, const double* edge_x, const double* edge_d1,
                                   const double* edge_d2, const double* edge_nu,
                                   const double* edge_a, const int* edge_patch,
                                   const double* edge_uv, const double* over_x,
                                   const double* over_nu, const double* over_speed,
                                   const double* over_a, pm_bvp** out) {
    if (!out) { pm_set_error("pm_bvp_create: out is NULL"); return PM_ERR_INVALID_ARG; }
    *out = nullptr;
    if (!s || ncurves < 0 || (ncurves > 0 && (!M || !F || !edge_x || !edge_d1 || !edge_d2 ||
                                              !edge_nu || !edge_a || !edge_patch || !edge_uv ||
                                              !over_x || !over_nu || !over_speed || !over_a))) {
        pm_set_error("pm_bvp_create: NULL argument");
        return PM_ERR_INVALID_ARG;
    }
    if (kind != PM_BVP_NEUMANN && kind != PM_BVP_DIRICHLET) {
        pm_set_error("pm_bvp_create: kind %d is neither PM_BVP_NEUMANN nor PM_BVP_DIRICHLET", kind);
        return PM_ERR_INVALID_ARG;
    }
    if (!s->has_coeff) { pm_set_error("pm_bvp_create: call pm_surface_set_coeff first"); return PM_ERR_NO_COEFF; }
    if (s->has_c || s->tri) {
        pm_set_error("pm_bvp_create: built for quadrilateral patches with c = 0");
        return PM_ERR_INVALID_ARG;
    }
    PM_CUDA_TRY(cudaSetDevice(s->ctx->device));
    pm_bvp* b = new pm_bvp();
    b->s = s;
    b->kind = kind == PM_BVP_DIRICHLET ? 1 : 0;
    b->coeff_epoch = s->coeff_epoch;
    b->N = s->N;
    b->ncurves = ncurves;
    for (int c = 0; c < ncurves; ++c) {
        if (M[c] < 2 || F[c] < 1 || (long long)M[c] * F[c] > (1 << 24)) {
            pm_set_error("pm_bvp_create: curve %d has M = %d, F = %d (need M >= 2, F >= 1)", c, M[c], F[c]);
            delete b;
            return PM_ERR_INVALID_ARG;
        }
        b->M.push_back(M[c]);
        b->F.push_back(F[c]);
        b->off.push_back(b->Me);
        b->offo.push_back(b->Fo);
        b->Me += M[c];
        b->Fo += M[c] * F[c];
    }
    long long interp_entries = 0;        // the interpolation matrices: F M x M per curve
    for (int c = 0; c < ncurves; ++c) interp_entries += (long long)F[c] * M[c] * M[c];
    if (b->Me > 4096 || interp_entries > (1LL << 26)) {
        pm_set_error("pm_bvp_create: %d edge nodes (at most 4096), %lld interpolation entries "
                     "sum F M^2 (at most 2^26)", b->Me, interp_entries);
        delete b;
        return PM_ERR_INVALID_ARG;
    }
    for (int e = 0; e < b->Me; ++e) {
        const double u0 = edge_uv[2 * e], v0 = edge_uv[2 * e + 1];
        const bool on_edge = std::fabs(std::fabs(u0) - 1.0) < 1e-12 || std::fabs(std::fabs(v0) - 1.0) < 1e-12;
        if (edge_patch[e] < 0 || edge_patch[e] >= s->npatch || !on_edge || std::fabs(u0) > 1.0 ||
            std::fabs(v0) > 1.0 || !(edge_a[e] > 0.0)) {
            pm_set_error("pm_bvp_create: edge node %d: patch %d, (u, v) = (%g, %g), a = %g (the node "
                         "must lie on an edge of its patch, a > 0)", e, edge_patch[e], u0, v0, edge_a[e]);
            delete b;
            return PM_ERR_INVALID_ARG;
        }
    }
    if (b->kind) {
        // Dirichlet: a constant over the surface, the edge nodes and the oversampled points
        std::vector<double> ah(s->N), gh(3 * (size_t)s->N);
        cudaError_t ce = cudaMemcpy(ah.data(), s->a, sizeof(double) * s->N, cudaMemcpyDeviceToHost);
        if (ce == cudaSuccess)
            ce = cudaMemcpy(gh.data(), s->g, sizeof(double) * gh.size(), cudaMemcpyDeviceToHost);
        if (ce != cudaSuccess) {
            pm_set_error("pm_bvp_create: %s", cudaGetErrorString(ce));
            delete b;
            return PM_ERR_CUDA;
        }
        const double a0 = ah[0];
        bool ok = true;
        for (double v : ah) ok = ok && std::fabs(v - a0) <= 1e-14 * a0;
        for (double v : gh) ok = ok && v == 0.0;
        for (int e = 0; e < b->Me; ++e) ok = ok && std::fabs(edge_a[e] - a0) <= 1e-14 * a0;
        for (int j = 0; j < b->Fo; ++j) ok = ok && std::fabs(over_a[j] - a0) <= 1e-14 * a0;
        if (!ok) {
            pm_set_error("pm_bvp_create: the Dirichlet system needs a constant coefficient "
                         "(on the surface, the edge nodes and the oversampled points)");
            delete b;
            return PM_ERR_INVALID_ARG;
        }
    }
    const pm_status st = create_impl(b, edge_x, edge_d1, edge_d2, edge_nu, edge_a, edge_patch,
                                     edge_uv, over_x, over_nu, over_speed, over_a);
    if (st != PM_OK) {
        free_bvp(b);
        return st;
    }
    *out = b;
    return PM_OK;
}

extern "C" void pm_bvp_destroy(pm_bvp* b) { free_bvp(b); }

extern "C" pm_status pm_bvp_apply(pm_bvp* b, const double* sigma, const double* mu, double* out_s,
                                  double* out_e) {
    if (!b || !sigma || !out_s || (b->Me > 0 && (!mu || !out_e))) {
        pm_set_error("pm_bvp_apply: NULL argument");
        return PM_ERR_INVALID_ARG;
    }
    if (b->coeff_epoch != b->s->coeff_epoch) {
        pm_set_error("pm_bvp_apply: the surface's coefficient changed after pm_bvp_create");
        return PM_ERR_INVALID_ARG;
    }
    PM_CUDA_TRY(cudaSetDevice(b->s->ctx->device));
    const size_t n = (size_t)b->N + b->Me;
    double *z = nullptr, *y = nullptr;
    PM_TRY(pm_dmalloc(&z, n));
    pm_status st = pm_dmalloc(&y, n);
    if (st == PM_OK) {
        cudaError_t e = cudaMemcpy(z, sigma, sizeof(double) * b->N, cudaMemcpyHostToDevice);
        if (e == cudaSuccess && b->Me)
            e = cudaMemcpy(z + b->N, mu, sizeof(double) * b->Me, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            pm_set_error("pm_bvp_apply: %s", cudaGetErrorString(e));
            st = PM_ERR_CUDA;
        }
    }
    if (st == PM_OK) st = apply_sys(b, z, y);
    if (st == PM_OK) {
        cudaError_t e = cudaMemcpy(out_s, y, sizeof(double) * b->N, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && b->Me) e = cudaMemcpy(out_e, y + b->N, sizeof(double) * b->Me, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) { pm_set_error("pm_bvp_apply: %s", cudaGetErrorString(e)); st = PM_ERR_CUDA; }
    }
    pm_dfree(z);
    pm_dfree(y);
    return st;
}

extern "C" pm_status pm_bvp_solve(pm_bvp* b, const double* f, const double* f_gamma, double tol,
                                  int maxit, double* u, double* sigma_out, double* mu_out,
                                  pm_solve_info* info) {
    if (!b || !f || !u || (b->Me > 0 && !f_gamma) || !(tol > 0.0) || maxit < 1) {
        pm_set_error("pm_bvp_solve: NULL argument, tol <= 0 or maxit < 1");
        return PM_ERR_INVALID_ARG;
    }
    if (b->coeff_epoch != b->s->coeff_epoch) {
        pm_set_error("pm_bvp_solve: the surface's coefficient changed after pm_bvp_create");
        return PM_ERR_INVALID_ARG;
    }
    PM_CUDA_TRY(cudaSetDevice(b->s->ctx->device));
    const int n = b->N + b->Me;
    const int m = std::max(2, std::min(b->s->opts.gmres_restart, 120));
    double *V = nullptr, *w = nullptr, *rhs = nullptr, *x = nullptr, *hd = nullptr, *ud = nullptr;
    pm_status st = pm_dmalloc(&V, (size_t)(m + 1) * n);
    if (st == PM_OK) st = pm_dmalloc(&w, (size_t)n);
    if (st == PM_OK) st = pm_dmalloc(&rhs, (size_t)n);
    if (st == PM_OK) st = pm_dmalloc(&x, (size_t)n);
    if (st == PM_OK) st = pm_dmalloc(&hd, (size_t)m + 1);
    if (st == PM_OK) st = pm_dmalloc(&ud, (size_t)b->N);
    auto cleanup = [&]() {
        pm_dfree(V); pm_dfree(w); pm_dfree(rhs); pm_dfree(x); pm_dfree(hd); pm_dfree(ud);
    };
    if (st != PM_OK) { cleanup(); return st; }
    const auto t0 = std::chrono::steady_clock::now();
    {
        cudaError_t e = cudaMemcpy(rhs, f, sizeof(double) * b->N, cudaMemcpyHostToDevice);
        if (e == cudaSuccess && b->Me)
            e = cudaMemcpy(rhs + b->N, f_gamma, sizeof(double) * b->Me, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemset(x, 0, sizeof(double) * n);
        if (e != cudaSuccess) {
            pm_set_error("pm_bvp_solve: %s", cudaGetErrorString(e));
            cleanup();
            return PM_ERR_CUDA;
        }
    }
    const int grid = pm_ceil_div(n, kT);
    std::vector<double> d;
    st = dots(b, rhs, 1, rhs, n, d);
    if (st != PM_OK) { cleanup(); return st; }
    const double bnorm = std::sqrt(d[0]);
    int iters = 0;
    double relres = bnorm > 0 ? 1.0 : 0.0;
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
    while (st == PM_OK && bnorm > 0 && relres > tol && iters < maxit) {
        // r = b - A x
        st = apply_sys(b, x, w);
        if (st != PM_OK) break;
        k_bvp_scale<<<grid, kT, 0, b->st>>>(n, -1.0, w, w);
        k_bvp_axpy<<<grid, kT, 0, b->st>>>(n, 1.0, rhs, w);
        if ((st = dots(b, w, 1, w, n, d)) != PM_OK) break;
        const double beta = std::sqrt(d[0]);
        relres = beta / bnorm;
        if (relres <= tol) break;
        k_bvp_scale<<<grid, kT, 0, b->st>>>(n, 1.0 / beta, w, V);
        std::fill(g.begin(), g.end(), 0.0);
        g[0] = beta;
        int k = 0;
        for (; k < m && iters < maxit; ++k, ++iters) {
            double* vk1 = V + (size_t)(k + 1) * n;
            if ((st = apply_sys(b, V + (size_t)k * n, vk1)) != PM_OK) break;
            // classical Gram-Schmidt with one reorthogonalisation
            std::vector<double> h(k + 1, 0.0);
            for (int pass = 0; pass < 2 && st == PM_OK; ++pass) {
                if ((st = dots(b, V, k + 1, vk1, n, d)) != PM_OK) break;
                for (int j = 0; j <= k; ++j) h[j] += d[j];
                cudaMemcpyAsync(hd, d.data(), sizeof(double) * (k + 1), cudaMemcpyHostToDevice, b->st);
                k_bvp_sub<<<grid, kT, 0, b->st>>>(n, k + 1, V, hd, vk1);
            }
            if (st != PM_OK) break;
            if ((st = dots(b, vk1, 1, vk1, n, d)) != PM_OK) break;
            const double hn = std::sqrt(d[0]);
            for (int j = 0; j <= k; ++j) H[(size_t)j * m + k] = h[j];
            H[(size_t)(k + 1) * m + k] = hn;
            if (hn > 0) k_bvp_scale<<<grid, kT, 0, b->st>>>(n, 1.0 / hn, vk1, vk1);
            // Givens rotations
            for (int j = 0; j < k; ++j) {
                const double a0 = H[(size_t)j * m + k], a1 = H[(size_t)(j + 1) * m + k];
                H[(size_t)j * m + k] = cs[j] * a0 + sn[j] * a1;
                H[(size_t)(j + 1) * m + k] = -sn[j] * a0 + cs[j] * a1;
            }
            const double a0 = H[(size_t)k * m + k], a1 = H[(size_t)(k + 1) * m + k];
            const double rr = std::hypot(a0, a1);
            cs[k] = rr > 0 ? a0 / rr : 1.0;
            sn[k] = rr > 0 ? a1 / rr : 0.0;
            H[(size_t)k * m + k] = rr;
            H[(size_t)(k + 1) * m + k] = 0.0;
            g[k + 1] = -sn[k] * g[k];
            g[k] = cs[k] * g[k];
            relres = std::fabs(g[k + 1]) / bnorm;
            if (relres <= tol || hn == 0.0) { ++k; ++iters; break; }
        }
        if (st != PM_OK) break;
        // x += V y, H y = g (upper triangular k x k)
        for (int i = k - 1; i >= 0; --i) {
            double t = g[i];
            for (int j = i + 1; j < k; ++j) t -= H[(size_t)i * m + j] * y[j];
            y[i] = t / H[(size_t)i * m + i];
        }
        for (int j = 0; j < k; ++j) k_bvp_axpy<<<grid, kT, 0, b->st>>>(n, y[j], V + (size_t)j * n, x);
        if (relres <= tol) {
            // the true residual confirms the estimate
            if ((st = apply_sys(b, x, w)) != PM_OK) break;
            k_bvp_scale<<<grid, kT, 0, b->st>>>(n, -1.0, w, w);
            k_bvp_axpy<<<grid, kT, 0, b->st>>>(n, 1.0, rhs, w);
            if ((st = dots(b, w, 1, w, n, d)) != PM_OK) break;
            relres = std::sqrt(d[0]) / bnorm;
        }
    }
    if (st == PM_OK) st = represent(b, x, ud);
    if (st == PM_OK) {
        cudaError_t e = cudaMemcpy(u, ud, sizeof(double) * b->N, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && sigma_out) e = cudaMemcpy(sigma_out, x, sizeof(double) * b->N, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && mu_out && b->Me)
            e = cudaMemcpy(mu_out, x + b->N, sizeof(double) * b->Me, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) { pm_set_error("pm_bvp_solve: %s", cudaGetErrorString(e)); st = PM_ERR_CUDA; }
    }
    if (st == PM_OK && !(relres <= tol)) {
        pm_set_error("pm_bvp_solve: relative residual %.3e above %.3e after %d iterations", relres, tol, iters);
        st = PM_ERR_NOT_CONVERGED;
    }
    if (info) {
        info->iterations = iters;
        info->refinements = 0;
        info->residual = relres;
        info->removed_mean = 0.0;
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        info->residual_updates = 0;
    }
    cleanup();
    return st;
}
