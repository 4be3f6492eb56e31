// C-ABI entry points, host-side quadrature tables and surface management.
//
// Contents:
//   - error reporting (thread-local message), options, contexts;
//   - Gauss-Legendre rules by Newton iteration on the three-term Legendre
//     recurrence, barycentric weights and the spectral differentiation matrix
//     of the tensor Lagrange interpolant on a patch (Sec. 6.1.1 remark);
//   - the self-rule theta plan: per reference node (u0, v0), theta panels that
//     split at the corner directions and are refined until int L(theta)^2 is
//     integrated to a tolerance (Sec. 6.1.1), then capped in width;
//   - pm_surface_create / set_coeff / apply_* / get_near.
#include "pm_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdlib>
#include <cstring>
#include <functional>

static thread_local std::string g_last_error;

void pm_set_error(const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
}

extern "C" const char* pm_last_error(void) { return g_last_error.c_str(); }

extern "C" const char* pm_status_str(pm_status st) {
    switch (st) {
        case PM_OK: return "ok";
        case PM_ERR_INVALID_ARG: return "invalid argument";
        case PM_ERR_OOM: return "out of memory";
        case PM_ERR_CUDA: return "CUDA error";
        case PM_ERR_NOT_CONVERGED: return "not converged";
        case PM_ERR_BREAKDOWN: return "Krylov breakdown";
        case PM_ERR_RHS_NOT_MEAN_ZERO: return "right-hand side is not mean zero";
        case PM_ERR_TIMEOUT: return "device wait timed out";
        case PM_ERR_INTERNAL: return "internal error";
        case PM_ERR_NO_COEFF: return "no coefficient set";
    }
    return "unknown status";
}

extern "C" void pm_default_opts(pm_opts* o) {
    if (!o) return;
    o->near_factor = 1.5;
    o->theta_tol = 1e-14;
    o->theta_max_width = 0.0;          // automatic: pi/16, or pi/24 for p = 11 (surface create)
    o->near_eta = 1.0;
    o->near_max_depth = 12;
    o->near_max_leaves = 512;
    o->gmres_restart = 50;
    o->max_refine = 8;
    o->inner_tol = 1e-6;
    o->mean_tol = 1e-8;
    o->residual_prec = PM_PREC_FF;
    o->fmm_depth = 0;
    o->batch_rhs = 1;
    o->direct_tpt = 0;
    o->direct_blocks_per_sm = 0;
    o->direct_symmetric = 1;
    o->residual_update = 1;
    o->fmm_tensor_m2l = 1;
}

// ----------------------------------------------------------------------------- tables
// Gauss-Legendre nodes (ascending) and weights by Newton's method on P_n.
static void gauss_legendre(int n, double* t, double* w) {
    for (int k = 0; k < n; ++k) {
        double x = std::cos(M_PI * (k + 0.75) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = x;
            for (int j = 2; j <= n; ++j) {
                double p2 = ((2.0 * j - 1.0) * x * p1 - (j - 1.0) * p0) / j;
                p0 = p1;
                p1 = p2;
            }
            double pn = (n == 1) ? x : p1;
            double pnm1 = (n == 1) ? 1.0 : p0;
            dp = n * (x * pn - pnm1) / (x * x - 1.0);
            double dx = pn / dp;
            x -= dx;
            if (std::fabs(dx) < 1e-16) break;
        }
        // recompute the derivative at the converged node
        double p0 = 1.0, p1 = x;
        for (int j = 2; j <= n; ++j) {
            double p2 = ((2.0 * j - 1.0) * x * p1 - (j - 1.0) * p0) / j;
            p0 = p1;
            p1 = p2;
        }
        double pn = (n == 1) ? x : p1, pnm1 = (n == 1) ? 1.0 : p0;
        dp = n * (x * pn - pnm1) / (x * x - 1.0);
        t[n - 1 - k] = x;   // cos is decreasing in k: store ascending
        w[n - 1 - k] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
}

static double legendre_p(int n, double x) {
    if (n == 0) return 1.0;
    double p0 = 1.0, p1 = x;
    for (int j = 2; j <= n; ++j) {
        double p2 = ((2.0 * j - 1.0) * x * p1 - (j - 1.0) * p0) / j;
        p0 = p1;
        p1 = p2;
    }
    return p1;
}

void pm_build_tables(int p, QuadTables* T) {
    std::memset(T, 0, sizeof(*T));
    T->p = p;
    gauss_legendre(p, T->t, T->wt);
    for (int a = 0; a < p; ++a) {
        double prod = 1.0;
        for (int b = 0; b < p; ++b)
            if (b != a) prod *= (T->t[a] - T->t[b]);
        T->bary[a] = 1.0 / prod;
    }
    // spectral differentiation: l_a'(t_i) = (lambda_a/lambda_i)/(t_i - t_a), diagonal by row sum
    for (int i = 0; i < p; ++i) {
        double diag = 0.0;
        for (int a = 0; a < p; ++a) {
            if (a == i) continue;
            double v = (T->bary[a] / T->bary[i]) / (T->t[i] - T->t[a]);
            T->Dm[i * p + a] = v;
            diag -= v;
        }
        T->Dm[i * p + i] = diag;
    }
    // l_a(+-1) by the barycentric formula
    for (int sgn = -1; sgn <= 1; sgn += 2) {
        double den = 0.0;
        for (int a = 0; a < p; ++a) den += T->bary[a] / (sgn - T->t[a]);
        for (int a = 0; a < p; ++a) {
            double v = (T->bary[a] / (sgn - T->t[a])) / den;
            if (sgn < 0) T->Lm[a] = v; else T->Lp[a] = v;
        }
    }
    gauss_legendre(PM_GL16, T->g16t, T->g16w);
    // Product-log correction for a panel [0, h] with 16 Gauss nodes r_q = h(1+t_q)/2:
    // int_0^h log(r) f(r) dr ~= sum_q (h/2) w_q (B_q + log h) f(r_q), where
    // B_q = sum_{n<16} (2n+1) P_n(t_q) M_n and M_n = int_0^1 log(s) P_n(2s-1) ds
    // (M_0 = -1, M_n = (-1)^(n+1) / (n (n+1))).  Relative to the plain rule,
    // which uses log(r_q), the extra term per node is (h/2) w_q E_q with
    // E_q = B_q - log((1 + t_q)/2).
    for (int q = 0; q < PM_GL16; ++q) {
        double B = 0.0;
        for (int nn = 0; nn < PM_GL16; ++nn) {
            double M = (nn == 0) ? -1.0 : ((nn % 2) ? 1.0 : -1.0) / (nn * (nn + 1.0));
            B += (2.0 * nn + 1.0) * legendre_p(nn, T->g16t[q]) * M;
        }
        T->logE[q] = B - std::log(0.5 * (1.0 + T->g16t[q]));
    }
}

// ----------------------------------------------------------------------------- theta plan
static double ray_length(double u0, double v0, double th) {
    double c = std::cos(th), s = std::sin(th);
    double L = INFINITY;
    if (c > 0) L = std::min(L, (1.0 - u0) / c);
    if (c < 0) L = std::min(L, (-1.0 - u0) / c);
    if (s > 0) L = std::min(L, (1.0 - v0) / s);
    if (s < 0) L = std::min(L, (-1.0 - v0) / s);
    return L;
}

void pm_theta_plan(const QuadTables& T, double tol, double max_width, std::vector<int>& off,
                   std::vector<double>& ang, std::vector<double>& wts,
                   std::vector<double>& len) {
    const int p = T.p;
    off.assign(1, 0);
    ang.clear();
    wts.clear();
    len.clear();
    for (int loc = 0; loc < p * p; ++loc) {
        const double u0 = T.t[loc / p], v0 = T.t[loc % p];
        auto l2 = [&](double a, double b) {
            double h = 0.5 * (b - a), acc = 0.0;
            for (int q = 0; q < PM_GL16; ++q) {
                double L = ray_length(u0, v0, a + h * (T.g16t[q] + 1.0));
                acc += h * T.g16w[q] * L * L;
            }
            return acc;
        };
        double cu[4] = {1, -1, -1, 1}, cv[4] = {1, 1, -1, -1}, ca[4];
        for (int k = 0; k < 4; ++k) {
            double a = std::atan2(cv[k] - v0, cu[k] - u0);
            ca[k] = a < 0 ? a + 2 * M_PI : a;
        }
        std::sort(ca, ca + 4);
        std::vector<std::pair<double, double>> panels;
        std::function<void(double, double, double, int)> split = [&](double a, double b,
                                                                      double whole, int depth) {
            double m = 0.5 * (a + b);
            double l = l2(a, m), r = l2(m, b);
            if (depth >= 50 || std::fabs(whole - l - r) <= tol) {
                panels.emplace_back(a, b);
                return;
            }
            split(a, m, l, depth + 1);
            split(m, b, r, depth + 1);
        };
        for (int k = 0; k < 4; ++k) {
            double a = ca[k], b = (k < 3) ? ca[k + 1] : ca[0] + 2 * M_PI;
            split(a, b, l2(a, b), 0);
        }
        for (auto& pb : panels) {
            int ns = std::max(1, (int)std::ceil((pb.second - pb.first) / max_width));
            double wdt = (pb.second - pb.first) / ns;
            for (int k = 0; k < ns; ++k) {
                double a = pb.first + k * wdt, h = 0.5 * wdt;
                for (int q = 0; q < PM_GL16; ++q) {
                    double th = a + h * (T.g16t[q] + 1.0);
                    ang.push_back(th);
                    wts.push_back(h * T.g16w[q]);
                    len.push_back(ray_length(u0, v0, th));
                }
            }
        }
        off.push_back((int)ang.size());
    }
}

// ----------------------------------------------------------------------------- contexts
extern "C" pm_status pm_ctx_create(int device, pm_ctx** out) {
    if (!out) { pm_set_error("pm_ctx_create: out is NULL"); return PM_ERR_INVALID_ARG; }
    *out = nullptr;
    int ndev = 0;
    PM_CUDA_TRY(cudaGetDeviceCount(&ndev));
    if (device < 0 || device >= ndev) {
        pm_set_error("pm_ctx_create: device %d out of range (%d devices)", device, ndev);
        return PM_ERR_INVALID_ARG;
    }
    PM_CUDA_TRY(cudaSetDevice(device));
    pm_ctx* c = new pm_ctx();
    c->device = device;
    cudaError_t e = cudaGetDeviceProperties(&c->prop, device);
    if (e != cudaSuccess) {
        delete c;
        pm_set_error("cudaGetDeviceProperties: %s", cudaGetErrorString(e));
        return PM_ERR_CUDA;
    }
    c->num_sms = c->prop.multiProcessorCount;
    *out = c;
    return PM_OK;
}

extern "C" void pm_ctx_destroy(pm_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    pm_dfree(c->fmm_opR);
    pm_dfree(c->fmm_opK);
    pm_multi_free(c);
    delete c;
}

// ----------------------------------------------------------------------------- surfaces
// Buffers a surface shares with its clones: built once, read-only afterwards.
#define PM_SHARED_FIELDS(X)                                                          \
    X(x) X(n) X(H) X(w) X(J) X(npatch_n) X(centroid) X(radius) X(row_ptr) X(blk_patch) \
    X(blk_row) X(W_lb) X(W_g) X(W_k) X(dev_err) X(th_off) X(th_ang) X(th_w) X(th_L)   \
    X(nu_ptr) X(nu_list) X(nu_blk)

PmSharedBuffers::~PmSharedBuffers() {
    cudaSetDevice(device);
    for (void* p : ptrs)
        if (p) cudaFree(p);
}

static void share_buffers(pm_surface* s) {
    auto sb = std::make_shared<PmSharedBuffers>();
    sb->device = s->ctx->device;
#define PM_X(f) sb->ptrs.push_back((void*)s->f);
    PM_SHARED_FIELDS(PM_X)
#undef PM_X
    s->shared = sb;
}

size_t pm_free_hbm_bytes() {
    if (const char* fake = std::getenv("PM_FAKE_HBM_BYTES")) return (size_t)std::strtoull(fake, nullptr, 10);
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return 0;
    return fr;
}

static void free_surface(pm_surface* s) {
    if (!s) return;
    if (s->ctx) cudaSetDevice(s->ctx->device);
    if (s->shared) {
        // the shared buffers go with the last surface that holds them
#define PM_X(f) s->f = nullptr;
        PM_SHARED_FIELDS(PM_X)
#undef PM_X
        s->shared.reset();
    }
    pm_solve_free(s);
    pm_fmm_free(s);
    pm_batch_free(s);
    pm_batch_solve_free(s);
    pm_helm_free(s);
    pm_ffmat_free(s);
    pm_dfree(s->x); pm_dfree(s->n); pm_dfree(s->H); pm_dfree(s->w); pm_dfree(s->J);
    pm_dfree(s->npatch_n); pm_dfree(s->centroid); pm_dfree(s->radius);
    pm_dfree(s->row_ptr); pm_dfree(s->blk_patch); pm_dfree(s->blk_row);
    pm_dfree(s->W_lb); pm_dfree(s->W_g); pm_dfree(s->W_k); pm_dfree(s->dev_err);
    pm_dfree(s->nu_ptr); pm_dfree(s->nu_list); pm_dfree(s->nu_blk);
    pm_dfree(s->th_off); pm_dfree(s->th_ang); pm_dfree(s->th_w); pm_dfree(s->th_L);
    pm_dfree(s->a); pm_dfree(s->g); pm_dfree(s->wa); pm_dfree(s->src32); pm_dfree(s->tgt32);
    pm_dfree(s->src64); pm_dfree(s->cR64); pm_dfree(s->cK64); pm_dfree(s->cR32);
    pm_dfree(s->cK32); pm_dfree(s->partial); pm_dfree(s->sig32);
    pm_dfree(s->src_ff); pm_dfree(s->tgt_ff); pm_dfree(s->src_kg); pm_dfree(s->log_tab);
    pm_dfree(s->dbuf_in); pm_dfree(s->dbuf_out);
    for (auto& ev : s->prof_events) {
        cudaEventDestroy(ev.second.first);
        cudaEventDestroy(ev.second.second);
    }
    delete s;
}

extern "C" void pm_surface_destroy(pm_surface* s) { free_surface(s); }

// Device bytes a new operator of npatch patches of order p would hold (model of
// the allocations of pm_surface_create + pm_surface_set_coeff, or of a clone +
// set_coeff): geometry and packed source/target arrays, the smooth sums' partial
// slices, the near-field CSR and coefficient-free weights with about 6 near patch
// blocks per node (the test surfaces have 3.9-4.9), and the coefficient-dependent
// corrections.  A clone holds only the per-coefficient part.
size_t pm_operator_need_bytes(int npatch, int p, int clone) {
    const size_t pp = (size_t)p * p, ppad = (pp + 3) / 4 * 4;
    const size_t N = (size_t)npatch * pp, Npad = (N + 255) / 256 * 256;
    const size_t nblk = 6 * N;
    const size_t nt = (N + 127) / 128;
    const size_t split = std::max<size_t>(32, nt * N * sizeof(float2) <= (size_t)kSymPartialCap ? nt : 0);
    const size_t per_coeff =
        sizeof(double) * (5 * N + nblk * pp * 2 + split * N) + sizeof(float) * (nblk * ppad * 2) +
        sizeof(float) * (size_t)npatch * ppad + Npad * (sizeof(float4) + sizeof(pm_d4)) +
        sizeof(float4) * (3 * N + 2 * N + 6 * N + 2 * N + 128);
    const size_t shared = sizeof(double) * (11 * N + 4 * (size_t)npatch + nblk * pp * 5) +
                          sizeof(int) * (N + 1 + 2 * nblk) + ((size_t)1 << 20);
    return clone ? per_coeff : per_coeff + shared;
}

// per-surface scratch of the smooth sums (a clone allocates its own)
static pm_status alloc_scratch(pm_surface* s) {
    const size_t N = s->N;
    s->max_split = std::max(32, pm_sym_tiles(s));     // one slice per tile for the symmetric sums
    PM_TRY(pm_dmalloc(&s->partial, (size_t)s->max_split * N));
    PM_TRY(pm_dmalloc(&s->sig32, (size_t)s->npatch * s->ppad));
    PM_CUDA_TRY(cudaMemset(s->sig32, 0, sizeof(float) * (size_t)s->npatch * s->ppad));
    PM_TRY(pm_dmalloc(&s->src32, s->Npad));
    PM_TRY(pm_dmalloc(&s->src64, s->Npad));
    PM_CUDA_TRY(cudaMemset(s->src32, 0, sizeof(float4) * s->Npad));
    PM_CUDA_TRY(cudaMemset(s->src64, 0, sizeof(pm_d4) * s->Npad));
    PM_TRY(pm_dmalloc(&s->tgt32, 3 * N));
    PM_CUDA_TRY(cudaDeviceSynchronize());
    return PM_OK;
}

static bool all_finite(const double* v, size_t n) {
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

// Quadrilateral patches (tri_ref == NULL: tensor Gauss-Legendre nodes of order p) or
// triangle patches (tri_ref: the rule's nt = p (p + 1) / 2 reference nodes and weights).
static pm_status create_impl(pm_ctx* ctx, int npatch, int p, const double* tri_ref,
                             const double* nodes, const double* normals, const double* tangents,
                             const double* curvature, const double* weights, const pm_opts* opts,
                             pm_surface** out) {
    const char* who = tri_ref ? "pm_surface_create_tri" : "pm_surface_create";
    if (!out) { pm_set_error("%s: out is NULL", who); return PM_ERR_INVALID_ARG; }
    *out = nullptr;
    if (!ctx || !nodes || !normals || !tangents || !curvature || !weights) {
        pm_set_error("%s: NULL argument", who);
        return PM_ERR_INVALID_ARG;
    }
    const int pmax = tri_ref ? PM_TRI_MAX_P : PM_MAX_P_API;
    const int pp = tri_ref ? p * (p + 1) / 2 : p * p;
    if (p < 2 || p > pmax || npatch < 1 || (long long)npatch * pp > (1LL << 26)) {
        pm_set_error("%s: need 2 <= p <= %d, npatch >= 1, N <= 2^26 (p=%d, npatch=%d)", who,
                     pmax, p, npatch);
        return PM_ERR_INVALID_ARG;
    }
    std::shared_ptr<PmTriTables> tri;
    if (tri_ref) {
        tri = std::make_shared<PmTriTables>();
        PM_TRY(pm_tri_tables(p, tri_ref, tri.get()));
    }
    const int N = npatch * pp;
    if (!all_finite(nodes, 3 * (size_t)N) || !all_finite(normals, 3 * (size_t)N) ||
        !all_finite(tangents, 6 * (size_t)N) || !all_finite(curvature, N) ||
        !all_finite(weights, N)) {
        pm_set_error("pm_surface_create: non-finite input");
        return PM_ERR_INVALID_ARG;
    }
    QuadTables T;
    pm_build_tables(p, &T);
    // |y_u x y_v| and consistency of the weights with the tensor Gauss rule
    std::vector<double> J(N);
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int k = 0; k < N; ++k) {
        const double* tu = tangents + 6 * (size_t)k;
        const double* tv = tu + 3;
        double c0 = tu[1] * tv[2] - tu[2] * tv[1];
        double c1 = tu[2] * tv[0] - tu[0] * tv[2];
        double c2 = tu[0] * tv[1] - tu[1] * tv[0];
        J[k] = std::sqrt(c0 * c0 + c1 * c1 + c2 * c2);
        int loc = k % pp;
        double wk = (tri ? tri->w[loc] : T.wt[loc / p] * T.wt[loc % p]) * J[k];
        if (!(J[k] > 0) || std::fabs(wk - weights[k]) > 1e-8 * std::fabs(wk)) {
            pm_set_error("%s: weight %d (%g) is not the rule's weight times |y_u x y_v| (%g)",
                         who, k, weights[k], wk);
            return PM_ERR_INVALID_ARG;
        }
        double nn = 0;
        for (int c = 0; c < 3; ++c) nn += normals[3 * (size_t)k + c] * normals[3 * (size_t)k + c];
        if (std::fabs(nn - 1.0) > 1e-8) {
            pm_set_error("%s: normal %d is not a unit vector", who, k);
            return PM_ERR_INVALID_ARG;
        }
        for (int c = 0; c < 3; ++c) {
            lo[c] = std::min(lo[c], nodes[3 * (size_t)k + c]);
            hi[c] = std::max(hi[c], nodes[3 * (size_t)k + c]);
        }
    }
    PM_CUDA_TRY(cudaSetDevice(ctx->device));
    pm_surface* s = new pm_surface();
    s->ctx = ctx;
    if (opts) s->opts = *opts; else pm_default_opts(&s->opts);
    s->npatch = npatch;
    s->p = p;
    s->pp = pp;
    s->tri = tri;
    s->ppad = (pp + 3) & ~3;
    s->N = N;
    s->Npad = pm_ceil_div(N, 256) * 256;
    s->scale = std::sqrt((hi[0] - lo[0]) * (hi[0] - lo[0]) + (hi[1] - lo[1]) * (hi[1] - lo[1]) +
                         (hi[2] - lo[2]) * (hi[2] - lo[2]));
    if (!(s->scale > 0)) s->scale = 1.0;
    // r^2 guard of the float32 remainder sum: exact zero for j == i, invisible otherwise
    s->eps2 = (float)((1e-10 * s->scale) * (1e-10 * s->scale));
    s->h_x.assign(nodes, nodes + 3 * (size_t)N);
    s->h_w.assign(weights, weights + N);
    s->h_tg.assign(tangents, tangents + 6 * (size_t)N);
    for (double v : s->h_x) s->h_far = std::max(s->h_far, std::fabs(v));

    pm_status st = PM_OK;
#define PM_STEP(expr) do { st = (expr); if (st != PM_OK) { free_surface(s); return st; } } while (0)
#define PM_CSTEP(expr) do { cudaError_t e_ = (expr); if (e_ != cudaSuccess) { \
        pm_set_error("%s: %s", #expr, cudaGetErrorString(e_)); free_surface(s); \
        return e_ == cudaErrorMemoryAllocation ? PM_ERR_OOM : PM_ERR_CUDA; } } while (0)
    PM_STEP(pm_dmalloc(&s->x, 3 * (size_t)N));
    PM_STEP(pm_dmalloc(&s->n, 3 * (size_t)N));
    PM_STEP(pm_dmalloc(&s->H, N));
    PM_STEP(pm_dmalloc(&s->w, N));
    PM_STEP(pm_dmalloc(&s->J, N));
    PM_CSTEP(cudaMemcpy(s->x, nodes, 3 * sizeof(double) * N, cudaMemcpyHostToDevice));
    PM_CSTEP(cudaMemcpy(s->n, normals, 3 * sizeof(double) * N, cudaMemcpyHostToDevice));
    PM_CSTEP(cudaMemcpy(s->H, curvature, sizeof(double) * N, cudaMemcpyHostToDevice));
    PM_CSTEP(cudaMemcpy(s->w, weights, sizeof(double) * N, cudaMemcpyHostToDevice));
    PM_CSTEP(cudaMemcpy(s->J, J.data(), sizeof(double) * N, cudaMemcpyHostToDevice));

    // self-rule theta plan (geometry of the reference square only)
    std::vector<int> off;
    std::vector<double> ang, wts, len;
    // Largest theta panel: the self-rule integrand carries the degree p - 1 Lagrange
    // basis along each ray; pi/16 panels integrate it to ~1e-13 up to p = 10, p = 11
    // needs pi/24 (pi/16 leaves ~5e-7 in the self weights).
    // On triangles the basis varies along a ray over a shorter length with a sharper
    // turn at the vertices: pi/24 as for the highest quad orders.
    const double theta_w = s->opts.theta_max_width > 0.0 ? s->opts.theta_max_width
                                                         : (p >= 11 || tri ? M_PI / 24 : M_PI / 16);
    if (tri)
        pm_tri_theta_plan(*tri, T, s->opts.theta_tol, theta_w, off, ang, wts, len);
    else
        pm_theta_plan(T, s->opts.theta_tol, theta_w, off, ang, wts, len);
    s->nth_total = (int)ang.size();
    PM_STEP(pm_dmalloc(&s->th_off, off.size()));
    PM_STEP(pm_dmalloc(&s->th_ang, ang.size()));
    PM_STEP(pm_dmalloc(&s->th_w, wts.size()));
    PM_STEP(pm_dmalloc(&s->th_L, len.size()));
    PM_CSTEP(cudaMemcpy(s->th_off, off.data(), sizeof(int) * off.size(), cudaMemcpyHostToDevice));
    PM_CSTEP(cudaMemcpy(s->th_ang, ang.data(), sizeof(double) * ang.size(), cudaMemcpyHostToDevice));
    PM_CSTEP(cudaMemcpy(s->th_w, wts.data(), sizeof(double) * wts.size(), cudaMemcpyHostToDevice));
    PM_CSTEP(cudaMemcpy(s->th_L, len.data(), sizeof(double) * len.size(), cudaMemcpyHostToDevice));

    PM_STEP(tri ? pm_near_build_tri(s, T) : pm_near_build(s, T));
    PM_STEP(alloc_scratch(s));
#undef PM_STEP
#undef PM_CSTEP
    share_buffers(s);
    *out = s;
    return PM_OK;
}

extern "C" pm_status pm_surface_create(pm_ctx* ctx, int npatch, int p, const double* nodes,
                                       const double* normals, const double* tangents,
                                       const double* curvature, const double* weights,
                                       const pm_opts* opts, pm_surface** out) {
    return create_impl(ctx, npatch, p, nullptr, nodes, normals, tangents, curvature, weights,
                       opts, out);
}

extern "C" pm_status pm_surface_create_tri(pm_ctx* ctx, int npatch, int p, const double* ref,
                                           const double* nodes, const double* normals,
                                           const double* tangents, const double* curvature,
                                           const double* weights, const pm_opts* opts,
                                           pm_surface** out) {
    if (!ref) {
        if (out) *out = nullptr;
        pm_set_error("pm_surface_create_tri: NULL reference nodes");
        return PM_ERR_INVALID_ARG;
    }
    return create_impl(ctx, npatch, p, ref, nodes, normals, tangents, curvature, weights, opts,
                       out);
}

extern "C" pm_status pm_surface_clone(const pm_surface* src, pm_surface** out) {
    if (!out) { pm_set_error("pm_surface_clone: out is NULL"); return PM_ERR_INVALID_ARG; }
    *out = nullptr;
    if (!src || !src->shared) {
        pm_set_error("pm_surface_clone: NULL or unbuilt source surface");
        return PM_ERR_INVALID_ARG;
    }
    PM_CUDA_TRY(cudaSetDevice(src->ctx->device));
    pm_surface* s = new pm_surface();
    s->ctx = src->ctx;
    s->opts = src->opts;
    s->npatch = src->npatch;
    s->p = src->p;
    s->pp = src->pp;
    s->ppad = src->ppad;
    s->N = src->N;
    s->Npad = src->Npad;
    s->scale = src->scale;
    s->h_far = src->h_far;
    s->eps2 = src->eps2;
    s->k32_centred = src->k32_centred;
    s->tri = src->tri;
    s->h_x = src->h_x;
    s->h_w = src->h_w;
    s->h_tg = src->h_tg;
    s->nblk = src->nblk;
    s->nu_max = src->nu_max;
    s->nth_total = src->nth_total;
    s->batch_rb = src->batch_rb;
    s->batch_bps = src->batch_bps;
    s->fmm_streams = src->fmm_streams;
#define PM_X(f) s->f = src->f;
    PM_SHARED_FIELDS(PM_X)
#undef PM_X
    s->shared = src->shared;
    const pm_status st = alloc_scratch(s);
    if (st != PM_OK) {
        free_surface(s);
        return st;
    }
    *out = s;
    return PM_OK;
}

extern "C" pm_status pm_surface_tune(pm_surface* s, int direct_tpt, int direct_blocks_per_sm) {
    if (!s || !(direct_tpt == 0 || direct_tpt == 1 || direct_tpt == 2 || direct_tpt == 4) ||
        direct_blocks_per_sm < 0 || direct_blocks_per_sm > 16) {
        pm_set_error("pm_surface_tune: NULL surface or knob out of range");
        return PM_ERR_INVALID_ARG;
    }
    s->opts.direct_tpt = direct_tpt;
    s->opts.direct_blocks_per_sm = direct_blocks_per_sm;
    s->graph_epoch++;
    return PM_OK;
}

extern "C" pm_status pm_surface_fmm_stats(pm_surface* s, double stats[4]) {
    if (!s || !stats) { pm_set_error("pm_surface_fmm_stats: NULL argument"); return PM_ERR_INVALID_ARG; }
    PM_CUDA_TRY(cudaSetDevice(s->ctx->device));
    PM_TRY(pm_fmm_build(s));
    for (int k = 0; k < 4; ++k) stats[k] = s->fmm_stats[k];
    return PM_OK;
}

extern "C" pm_status pm_surface_info(const pm_surface* s, int* N, int* nblocks) {
    if (!s) { pm_set_error("pm_surface_info: NULL surface"); return PM_ERR_INVALID_ARG; }
    if (N) *N = s->N;
    if (nblocks) *nblocks = s->nblk;
    return PM_OK;
}

extern "C" pm_status pm_surface_set_coeff(pm_surface* s, const double* a, const double* grad_a) {
    if (!s || !a) { pm_set_error("pm_surface_set_coeff: NULL argument"); return PM_ERR_INVALID_ARG; }
    const int N = s->N;
    for (int k = 0; k < N; ++k)
        if (!std::isfinite(a[k]) || !(a[k] > 0)) {
            pm_set_error("pm_surface_set_coeff: a[%d] = %g is not finite and positive", k, a[k]);
            return PM_ERR_INVALID_ARG;
        }
    if (grad_a && !all_finite(grad_a, 3 * (size_t)N)) {
        pm_set_error("pm_surface_set_coeff: non-finite grad_a");
        return PM_ERR_INVALID_ARG;
    }
    PM_CUDA_TRY(cudaSetDevice(s->ctx->device));
    if (!s->a) {
        PM_TRY(pm_dmalloc(&s->a, N));
        PM_TRY(pm_dmalloc(&s->g, 3 * (size_t)N));
        PM_TRY(pm_dmalloc(&s->wa, N));
        PM_TRY(pm_dmalloc(&s->cR64, (size_t)s->nblk * s->pp));
        PM_TRY(pm_dmalloc(&s->cK64, (size_t)s->nblk * s->pp));
        PM_TRY(pm_dmalloc(&s->cR32, (size_t)s->nblk * s->ppad));
        PM_TRY(pm_dmalloc(&s->cK32, (size_t)s->nblk * s->ppad));
    }
    PM_CUDA_TRY(cudaMemcpy(s->a, a, sizeof(double) * N, cudaMemcpyHostToDevice));
    cudaStream_t st = 0;
    if (grad_a) {
        PM_CUDA_TRY(cudaMemcpy(s->g, grad_a, 3 * sizeof(double) * N, cudaMemcpyHostToDevice));
    } else {
        std::vector<double> gh(3 * (size_t)N);
        if (s->tri) {
            pm_tri_gradient(s, a, gh.data());
        } else {
            QuadTables T;
            pm_build_tables(s->p, &T);
            pm_patch_gradient(s, T, a, gh.data());
        }
        PM_CUDA_TRY(cudaMemcpy(s->g, gh.data(), 3 * sizeof(double) * N, cudaMemcpyHostToDevice));
    }
    PM_TRY(pm_pack_targets(s, st));
    PM_TRY(pm_pack_ff(s, st));
    PM_TRY(pm_near_combine_coeff(s, st));
    PM_TRY(pm_ffmat_refresh(s, st));
    PM_CUDA_TRY(cudaStreamSynchronize(st));
    s->has_coeff = true;
    s->has_c = 0;
    s->graph_epoch++;
    s->coeff_epoch++;
    return PM_OK;
}

// grad_G a at the nodes from the tensor interpolant of a (eq. gradg):
// grad_G a = [y_u y_v] g^{-1} [a_u; a_v], with a_u, a_v by spectral
// differentiation along the patch lines and y_u, y_v the given tangents.
void pm_patch_gradient(const pm_surface* s, const QuadTables& T, const double* a,
                       double* grad) {
    const int p = s->p, pp = s->pp;
    for (int k = 0; k < s->N; ++k) {
        const int P = k / pp, loc = k - P * pp, i0 = loc / p, j0 = loc % p;
        double au = 0.0, av = 0.0;
        for (int m = 0; m < p; ++m) {
            au += T.Dm[i0 * p + m] * a[P * pp + m * p + j0];
            av += T.Dm[j0 * p + m] * a[P * pp + i0 * p + m];
        }
        const double* tu = &s->h_tg[6 * (size_t)k];
        const double* tv = tu + 3;
        const double E = tu[0] * tu[0] + tu[1] * tu[1] + tu[2] * tu[2];
        const double F = tu[0] * tv[0] + tu[1] * tv[1] + tu[2] * tv[2];
        const double G = tv[0] * tv[0] + tv[1] * tv[1] + tv[2] * tv[2];
        const double det = E * G - F * F;
        const double cu = (G * au - F * av) / det, cv = (-F * au + E * av) / det;
        for (int c = 0; c < 3; ++c) grad[3 * (size_t)k + c] = cu * tu[c] + cv * tv[c];
    }
}

pm_status pm_ensure_scratch(pm_surface* s, size_t n) {
    if (s->dbuf_n >= n) return PM_OK;
    pm_dfree(s->dbuf_in);
    pm_dfree(s->dbuf_out);
    s->dbuf_n = 0;
    PM_TRY(pm_dmalloc(&s->dbuf_in, n));
    PM_TRY(pm_dmalloc(&s->dbuf_out, n));
    s->dbuf_n = n;
    return PM_OK;
}

// One right-hand side, device pointers.  kernel_K selects K instead of R.
// prepped != 0: the float32 source strengths (src32.w, sig32) for sigma were
// already written by the caller's kernel (fused Arnoldi step), skip the prep.
pm_status pm_apply_dev(pm_surface* s, int kernel_K, int smooth, int near, const double* sigma,
                       double* out, pm_precision prec, cudaStream_t st, int prepped) {
    int nsplit = 0;
    prepped = prepped && (prec == PM_PREC_FP32 || prec == PM_PREC_FMM);
    if ((smooth || near) && !prepped) {
        PhaseTimer t(s, PM_PHASE_PREP, st);
        if (prec == PM_PREC_FF && pm_ffmat_has(s, kernel_K)) {
            PM_TRY(pm_ffmat_prep(s, sigma, st));
        } else if (prec == PM_PREC_FF) {
            PM_TRY(pm_prep_ff(s, sigma, st));
        } else {
            PM_TRY(pm_prep_sources(s, sigma, prec == PM_PREC_FMM ? PM_PREC_FP32 : prec, st));
        }
    }
    if (smooth) {
        PhaseTimer t(s, prec == PM_PREC_FP64 || prec == PM_PREC_FF
                            ? (kernel_K ? PM_PHASE_DIRECT64_K : PM_PHASE_DIRECT64)
                            : (kernel_K ? PM_PHASE_DIRECT_K : PM_PHASE_DIRECT_R), st);
        const int nt = pm_sym_tiles(s);
        if (prec == PM_PREC_FF && pm_ffmat_has(s, kernel_K)) {
            PM_TRY(pm_ffmat_apply(s, kernel_K, &nsplit, st));
        } else if (prec == PM_PREC_FF && nt > 0) {
            nsplit = nt;
            PM_TRY(pm_sym_ff(s, kernel_K, st));
        } else if (prec == PM_PREC_FF) {
            nsplit = pm_ff_splits(s);
            PM_TRY(pm_direct_ff(s, kernel_K, nsplit, st));
        } else if (prec == PM_PREC_FMM) {
            nsplit = pm_fmm_splits();
            PM_TRY(pm_fmm_apply(s, kernel_K, st));
        } else {
            nsplit = pm_direct_splits(s, prec, kernel_K);
            PM_TRY(pm_direct_sum(s, kernel_K, prec, nsplit, st));
        }
    }
    PhaseTimer t(s, PM_PHASE_NEAR, st);
    s->launch_total += ((smooth || near) && !prepped) + (smooth && prec != PM_PREC_FMM) + 1;
    return pm_near_apply(s, kernel_K, sigma, out, near, nsplit,
                         prec == PM_PREC_FMM ? PM_PREC_FP32 : prec, st);
}

static pm_status apply_impl(pm_surface* s, int kernel_K, int smooth, int near,
                            const double* sigma, double* out, int nrhs, pm_precision prec,
                            int on_device, void* stream) {
    if (!s || !sigma || !out || nrhs < 1) {
        pm_set_error("apply: NULL argument or nrhs < 1");
        return PM_ERR_INVALID_ARG;
    }
    if (prec != PM_PREC_FP64 && prec != PM_PREC_FP32 && prec != PM_PREC_FF &&
        prec != PM_PREC_FMM) {
        pm_set_error("apply: precision %d is not available for this operator", (int)prec);
        return PM_ERR_INVALID_ARG;
    }
    if (!s->has_coeff) { pm_set_error("apply: call pm_surface_set_coeff first"); return PM_ERR_NO_COEFF; }
    if (s->has_c) {
        pm_set_error("apply: the surface has c != 0 (pm_surface_set_coeff_c): use pm_apply_c");
        return PM_ERR_INVALID_ARG;
    }
    PM_CUDA_TRY(cudaSetDevice(s->ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    const size_t N = s->N;
    const bool batched = nrhs > 1 && smooth && near && s->opts.batch_rhs &&
                         (prec == PM_PREC_FP32 || prec == PM_PREC_FF);
    if (on_device) {
        if (batched) {
            PM_TRY(pm_apply_batch(s, kernel_K, sigma, (long long)N, out, (long long)N, nrhs, prec, st));
        } else {
            for (int r = 0; r < nrhs; ++r)
                PM_TRY(pm_apply_dev(s, kernel_K, smooth, near, sigma + r * N, out + r * N, prec, st));
        }
        PM_CUDA_TRY(cudaGetLastError());
        return PM_OK;
    }
    if (batched) {
        PM_TRY(pm_ensure_scratch(s, N * (size_t)nrhs));
        PM_CUDA_TRY(cudaMemcpyAsync(s->dbuf_in, sigma, N * nrhs * sizeof(double),
                                    cudaMemcpyHostToDevice, st));
        PM_TRY(pm_apply_batch(s, kernel_K, s->dbuf_in, (long long)N, s->dbuf_out, (long long)N,
                              nrhs, prec, st));
        PM_CUDA_TRY(cudaMemcpyAsync(out, s->dbuf_out, N * nrhs * sizeof(double),
                                    cudaMemcpyDeviceToHost, st));
        PM_CUDA_TRY(cudaStreamSynchronize(st));
        return PM_OK;
    }
    PM_TRY(pm_ensure_scratch(s, N));
    for (int r = 0; r < nrhs; ++r) {
        PM_CUDA_TRY(cudaMemcpyAsync(s->dbuf_in, sigma + r * N, N * sizeof(double),
                                    cudaMemcpyHostToDevice, st));
        PM_TRY(pm_apply_dev(s, kernel_K, smooth, near, s->dbuf_in, s->dbuf_out, prec, st));
        PM_CUDA_TRY(cudaMemcpyAsync(out + r * N, s->dbuf_out, N * sizeof(double),
                                    cudaMemcpyDeviceToHost, st));
    }
    PM_CUDA_TRY(cudaStreamSynchronize(st));
    return PM_OK;
}

// With -DPM_BOUNDS_CHECK every apply is bracketed by pm_surface_check and a finite
// scan of its result (PM_ERR_INTERNAL on a failure, with the check's message).
static pm_status apply_common(pm_surface* s, int kernel_K, int smooth, int near,
                              const double* sigma, double* out, int nrhs, pm_precision prec,
                              int on_device, void* stream) {
#ifdef PM_BOUNDS_CHECK
    if (s && s->row_ptr) PM_TRY(pm_surface_check(s));
#endif
    PM_TRY(apply_impl(s, kernel_K, smooth, near, sigma, out, nrhs, prec, on_device, stream));
#ifdef PM_BOUNDS_CHECK
    const size_t n = (size_t)s->N * nrhs;
    if (on_device) {
        PM_TRY(pm_check_finite(out, n, (cudaStream_t)stream, "apply result"));
    } else {
        for (size_t k = 0; k < n; ++k)
            if (!std::isfinite(out[k])) {
                pm_set_error("apply result: non-finite value at %zu", k);
                return PM_ERR_INTERNAL;
            }
    }
#endif
    return PM_OK;
}

extern "C" pm_status pm_apply_R(pm_surface* s, const double* sigma, double* out, int nrhs,
                                pm_precision prec, int on_device, void* stream) {
    return apply_common(s, 0, 1, 1, sigma, out, nrhs, prec, on_device, stream);
}

extern "C" pm_status pm_apply_K(pm_surface* s, const double* sigma, double* out, int nrhs,
                                pm_precision prec, int on_device, void* stream) {
    return apply_common(s, 1, 1, 1, sigma, out, nrhs, prec, on_device, stream);
}

extern "C" pm_status pm_apply_part(pm_surface* s, int part, const double* sigma, double* out,
                                   int nrhs, pm_precision prec, int on_device, void* stream) {
    switch (part) {
        case PM_PART_SMOOTH_R: return apply_common(s, 0, 1, 0, sigma, out, nrhs, prec, on_device, stream);
        case PM_PART_SMOOTH_K: return apply_common(s, 1, 1, 0, sigma, out, nrhs, prec, on_device, stream);
        case PM_PART_NEAR_R: return apply_common(s, 0, 0, 1, sigma, out, nrhs, prec, on_device, stream);
        case PM_PART_NEAR_K: return apply_common(s, 1, 0, 1, sigma, out, nrhs, prec, on_device, stream);
    }
    pm_set_error("pm_apply_part: unknown part %d", part);
    return PM_ERR_INVALID_ARG;
}

extern "C" pm_status pm_surface_get_near(const pm_surface* s, int* row_ptr, int* blk_patch,
                                         double* corr_R, double* corr_K) {
    if (!s) { pm_set_error("pm_surface_get_near: NULL surface"); return PM_ERR_INVALID_ARG; }
    PM_CUDA_TRY(cudaSetDevice(s->ctx->device));
    if ((corr_R || corr_K) && !s->has_coeff) {
        pm_set_error("pm_surface_get_near: corrections need pm_surface_set_coeff");
        return PM_ERR_NO_COEFF;
    }
    if (row_ptr)
        PM_CUDA_TRY(cudaMemcpy(row_ptr, s->row_ptr, sizeof(int) * (s->N + 1), cudaMemcpyDeviceToHost));
    if (blk_patch)
        PM_CUDA_TRY(cudaMemcpy(blk_patch, s->blk_patch, sizeof(int) * s->nblk, cudaMemcpyDeviceToHost));
    size_t nv = (size_t)s->nblk * s->pp;
    if (corr_R) PM_CUDA_TRY(cudaMemcpy(corr_R, s->cR64, sizeof(double) * nv, cudaMemcpyDeviceToHost));
    if (corr_K) PM_CUDA_TRY(cudaMemcpy(corr_K, s->cK64, sizeof(double) * nv, cudaMemcpyDeviceToHost));
    return PM_OK;
}

extern "C" pm_status pm_profile_enable(pm_surface* s, int enable) {
    if (!s) { pm_set_error("pm_profile_enable: NULL surface"); return PM_ERR_INVALID_ARG; }
    s->profiling = enable != 0;
    return PM_OK;
}

extern "C" pm_status pm_profile_read(pm_surface* s, int phase, double* ms, int* launches,
                                     int reset) {
    if (!s || phase < 0 || phase > PM_PHASE_COUNT) {
        pm_set_error("pm_profile_read: NULL surface or bad phase");
        return PM_ERR_INVALID_ARG;
    }
    if (phase == PM_PHASE_COUNT) {
        if (ms) *ms = 0.0;
        if (launches) *launches = (int)std::min<long long>(s->launch_total, 2147483647LL);
        if (reset) s->launch_total = 0;
        return PM_OK;
    }
    PM_CUDA_TRY(cudaSetDevice(s->ctx->device));
    for (auto& ev : s->prof_events) {
        float t = 0.f;
        PM_CUDA_TRY(cudaEventSynchronize(ev.second.second));
        PM_CUDA_TRY(cudaEventElapsedTime(&t, ev.second.first, ev.second.second));
        s->prof_ms[ev.first] += t;
        s->prof_n[ev.first] += 1;
        cudaEventDestroy(ev.second.first);
        cudaEventDestroy(ev.second.second);
    }
    s->prof_events.clear();
    if (ms) *ms = s->prof_ms[phase];
    if (launches) *launches = s->prof_n[phase];
    if (reset) {
        for (int k = 0; k < PM_PHASE_COUNT; ++k) {
            s->prof_ms[k] = 0;
            s->prof_n[k] = 0;
        }
        s->launch_total = 0;
    }
    return PM_OK;
}

extern "C" pm_status pm_solve(pm_surface* s, const double* f, double* u, int nrhs, double tol,
                              int maxit, pm_precision prec, unsigned flags, double* sigma_out,
                              pm_solve_info* info, void* stream) {
    if (!s || !f || !u || nrhs < 1 || !(tol > 0) || maxit < 1) {
        pm_set_error("pm_solve: NULL argument, nrhs < 1, tol <= 0 or maxit < 1");
        return PM_ERR_INVALID_ARG;
    }
    if (prec != PM_PREC_FP64 && prec != PM_PREC_FP32 && prec != PM_PREC_FF &&
        prec != PM_PREC_FMM) {
        pm_set_error("pm_solve: precision %d is not available", (int)prec);
        return PM_ERR_INVALID_ARG;
    }
    if (!s->has_coeff) { pm_set_error("pm_solve: call pm_surface_set_coeff first"); return PM_ERR_NO_COEFF; }
    if (s->has_c) {
        pm_set_error("pm_solve: the surface has c != 0 (pm_surface_set_coeff_c): use pm_solve_c");
        return PM_ERR_INVALID_ARG;
    }
    if ((flags & PM_SOLVE_INITIAL_GUESS) && !sigma_out) {
        pm_set_error("pm_solve: PM_SOLVE_INITIAL_GUESS needs sigma_out (the starting sigma)");
        return PM_ERR_INVALID_ARG;
    }
    PM_CUDA_TRY(cudaSetDevice(s->ctx->device));
    const size_t N = s->N;
    if (nrhs > 1 && s->opts.batch_rhs && !(flags & PM_SOLVE_INITIAL_GUESS))
        return pm_solve_batch(s, f, u, nrhs, tol, maxit, prec, flags, sigma_out, info,
                              (cudaStream_t)stream);
    pm_status worst = PM_OK;
    for (int r = 0; r < nrhs; ++r) {
        pm_status st = pm_solve_impl(s, f + r * N, u + r * N, tol, maxit, prec, flags,
                                     sigma_out ? sigma_out + r * N : nullptr,
                                     info ? info + r : nullptr, (cudaStream_t)stream);
        if (st != PM_OK && st != PM_ERR_NOT_CONVERGED) return st;
        if (st != PM_OK) worst = st;
    }
    return worst;
}
