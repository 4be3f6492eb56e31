// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <string>
#include <memory>
#include <mutex>
#include <utility>
#include <vector>

#include "../../include/parametrix.h"

// ----------------------------------------------------------------------------- errors
void pm_set_error(const char* fmt, ...);

#define PM_CUDA_TRY(expr)                                                          \
    do {                                                                           \
        cudaError_t e_ = (expr);                                                   \
        if (e_ != cudaSuccess) {                                                   \
            pm_set_error("%s:%d: %s: %s", __FILE__, __LINE__, #expr,               \
                         cudaGetErrorString(e_));                                  \
            return e_ == cudaErrorMemoryAllocation ? PM_ERR_OOM : PM_ERR_CUDA;     \
        }                                                                          \
    } while (0)

#define PM_TRY(expr)                                                               \
    do {                                                                           \
        pm_status s_ = (expr);                                                     \
        if (s_ != PM_OK) return s_;                                                \
    } while (0)

// Kernel launch with a scheduling priority (cudaLaunchAttributePriority): the
// attribute travels with the launch into a captured graph, where stream
// priorities alone are not kept.
template <typename... KArgs, typename... Args>
static inline cudaError_t pm_launch_prio(void (*kernel)(KArgs...), dim3 grid, dim3 block,
                                         size_t smem, cudaStream_t st, int prio,
                                         Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributePriority;
    at[0].val.priority = prio;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Device-side error word: kernels record a failed check here (no trap).
enum : int {
    PM_DEV_OK = 0,
    PM_DEV_LEAF_OVERFLOW = 1,   // near rule exceeded its leaf budget
    PM_DEV_BAD_INDEX = 2,       // an index check failed
    PM_DEV_NONFINITE = 3,       // a non-finite quadrature value
    PM_DEV_TIMEOUT = 4,         // a bounded wait (mbarrier, flag) ran out
};

// (x, y, z, s) in float64, 32-byte aligned for one 256-bit access
struct alignas(32) pm_d4 {
    double x, y, z, w;
};

// ----------------------------------------------------------------------------- constants
constexpr int PM_MAX_P = 16;
constexpr int PM_MAX_P_API = 11;     // quadrature kernels give one basis entry per thread (p*p <= 128)
constexpr int PM_GL16 = 16;          // points per quadrature panel
constexpr int PM_TRI_MAX_P = 8;      // triangle patches: order p <= 8, p (p + 1) / 2 <= 36 nodes
constexpr int PM_TRI_MAX_NT = 36;
constexpr int PM_RADIAL_PANELS = 4;  // self rule: [0,L/8],[L/8,L/4],[L/4,L/2],[L/2,L]

// Host-computed tables for the quadrature kernels (constant memory).
struct QuadTables {
    double t[PM_MAX_P];            // p-point Gauss-Legendre nodes (ascending)
    double wt[PM_MAX_P];           // p-point Gauss-Legendre weights
    double bary[PM_MAX_P];         // barycentric weights of the nodes
    double Dm[PM_MAX_P * PM_MAX_P];// Dm[i*p + a] = l_a'(t_i) (spectral differentiation)
    double Lm[PM_MAX_P];           // l_a(-1)
    double Lp[PM_MAX_P];           // l_a(+1)
    double g16t[PM_GL16];          // 16-point Gauss-Legendre nodes on [-1,1]
    double g16w[PM_GL16];          // and weights
    double logE[PM_GL16];          // product-log correction of the first radial panel
    int p;
};

// ----------------------------------------------------------------------------- handles
struct pm_ctx {
    int device = 0;
    int num_sms = 0;
    cudaDeviceProp prop{};
    // FMM M2L operators for unit boxes, one per offset class, shared by all
    // surfaces of the context; built on first use (pm_fmm.cu)
    std::mutex fmm_mu;
    // M2L operators per canonical offset, K-major [rows][1536] in float16: the
    // float32 operator times 2^12, split in two float16 parts (a0, a1), as K
    // blocks a1 a0 a0 (pm_fmm.cu)
    __half* fmm_opR = nullptr;   // rows = 9 * 512
    __half* fmm_opK = nullptr;   // rows = 512
    // multi-instance lockstep solve (pm_batch.cu): workspace of the last call's shape
    std::mutex multi_mu;
    struct PmMultiWork* multi = nullptr;
};
void pm_multi_free(pm_ctx* c);

// Device buffers fixed once a surface is built (geometry, near-field CSR and
// quadrature weights, self-rule plan): shared by a surface and its clones
// (pm_surface_clone) and freed with the last of them.
struct PmSharedBuffers {
    int device = 0;
    std::vector<void*> ptrs;
    ~PmSharedBuffers();
};

struct PmSolveWork;
struct PmFmmTree;
struct PmBatchWork;
struct PmBatchSolveWork;
struct PmHelmWork;

// Triangle patches (pm_tri.cu): the reference nodes (u, v) and weights w of the
// surface's rule on T0, U = V^-1 with V[j][n] = K_n(u_j, v_j) (Koornwinder basis,
// the library's ordering) so that l_k = sum_n K_n U[n * nt + k], and the
// derivative matrices Du[j * nt + k] = d l_k / du at node j (Dv likewise).
struct PmTriTables {
    int p = 0, nt = 0;
    std::vector<double> u, v, w, U, Du, Dv;
};

struct pm_surface {
    pm_ctx* ctx = nullptr;
    pm_opts opts{};
    int npatch = 0, p = 0, pp = 0, ppad = 0, N = 0, Npad = 0;
    double scale = 1.0;           // bounding-box diagonal (for the self-pair guard)
    double h_far = 0.0;           // largest |coordinate| (placement of padding sources)
    float eps2 = 0.f;             // r^2 guard of the float32 R sum
    int k32_centred = 0;          // float32 parametrix sum in the centred form (pm_direct.cu)

    // float64 geometry (device)
    double* x = nullptr;          // [N*3]
    double* n = nullptr;          // [N*3]
    double* H = nullptr;          // [N]
    double* w = nullptr;          // [N]
    double* J = nullptr;          // [N] |y_u x y_v|
    double* npatch_n = nullptr;   // [N*3] normal of the interpolated patch at each node
    double* centroid = nullptr;   // [npatch*3]
    double* radius = nullptr;     // [npatch]
    std::vector<double> h_x, h_w, h_tg; // host copies used for the spectral gradient

    // near field (CSR over (target, patch) blocks)
    int nblk = 0;
    int* row_ptr = nullptr;       // [N+1]
    int* blk_patch = nullptr;     // [nblk]
    int* blk_row = nullptr;       // [nblk]
    double* W_lb = nullptr;       // [nblk*pp] int (q^2 - H q)/pi l_k J~
    double* W_g = nullptr;        // [3*nblk*pp] int r/(2 pi r^2) l_k J~ (component-major)
    double* W_k = nullptr;        // [nblk*pp] int log|r|/(2 pi) l_k J~
    int* dev_err = nullptr;       // device error word
    // per patch, the union of its rows' near patches (multi-instance near field):
    // nu_list[nu_ptr[P] .. nu_ptr[P+1]) ascending; nu_blk[b] = index of blk_patch[b]
    // in its row's patch union; nu_max = the largest union (0: not built)
    int* nu_ptr = nullptr;        // [npatch+1]
    int* nu_list = nullptr;
    int* nu_blk = nullptr;        // [nblk]
    int nu_max = 0;

    // self-rule plan: theta nodes per local node
    int* th_off = nullptr;        // [pp+1]
    double* th_ang = nullptr;     // [nth]
    double* th_w = nullptr;       // [nth]
    double* th_L = nullptr;       // [nth]
    int nth_total = 0;

    // coefficient-dependent data
    bool has_coeff = false;
    double* a = nullptr;          // [N]
    double* g = nullptr;          // [N*3]
    double* wa = nullptr;         // [N] w/a
    float4* src32 = nullptr;      // [Npad] (x, y, z, s)
    float4* tgt32 = nullptr;      // [3*N] (x,y,z,0), (sqrt(a/pi) n, 0), (m, 0)
    pm_d4* src64 = nullptr;     // [Npad] (x, y, z, s)
    float4* src_ff = nullptr;     // [2N] float-float sources
    float4* tgt_ff = nullptr;     // [6N] float-float targets
    float4* src_kg = nullptr;     // [2N] grid-split coordinates + strengths (parametrix sums)
    float4* log_tab = nullptr;    // [128] table of the float-float logarithm
    double* cR64 = nullptr;       // [nblk*pp]
    double* cK64 = nullptr;       // [nblk*pp]
    float* cR32 = nullptr;        // [nblk*ppad]
    float* cK32 = nullptr;        // [nblk*ppad]

    // c != 0 (pm_surface_set_coeff_c, pm_helm.cu): c at the nodes, q = c/a (complex,
    // (re, im)), complex corrections of a(y) R and a(y) K (with the coefficients), work
    int has_c = 0;
    double2* cc = nullptr;        // [N] c
    double2* qn = nullptr;        // [N] c/a
    double2* cRc = nullptr;       // [nblk*pp]
    double2* cKc = nullptr;       // [nblk*pp]
    PmHelmWork* helm = nullptr;

    // stored float-float smooth-sum matrices (pm_ffmat.cu, pm_surface_store_ff): the
    // remainder and parametrix entries (6-byte format, row or symmetric tile layout)
    // and the float-float strengths of the apply; null when not stored
    unsigned char* ffm_R = nullptr;
    unsigned char* ffm_K = nullptr;
    float2* ffm_s = nullptr;      // [ffm_ld]
    int* ffm_err = nullptr;       // device error word of the stored-matrix GEMVs (PM_DEV_TIMEOUT)
    long long ffm_ld = 0;
    int ffm_symK = 0;             // tiles of 128 per side when ffm_K holds the symmetric
                                  // tile-pair layout (upper triangle only), else 0

    // per-phase timing (events recorded around launches while enabled)
    bool profiling = false;
    long long graph_epoch = 0;    // bumped when buffers or launch shapes captured in graphs change
    long long coeff_epoch = 0;    // bumped by every coefficient change (set_coeff, set_coeff_c)
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> prof_events;
    double prof_ms[PM_PHASE_COUNT] = {};
    int prof_n[PM_PHASE_COUNT] = {};
    long long launch_total = 0;   // kernels launched for this surface since the last reset

    // solve workspace (pm_solve.cu) and the device flag that lets the apply
    // kernels of a finished Krylov cycle return at once
    PmSolveWork* solve_work = nullptr;
    PmFmmTree* fmm = nullptr;
    PmBatchWork* batch = nullptr;
    PmBatchSolveWork* bsolve = nullptr;
    double fmm_stats[4] = {0, 0, 0, 0};
    const int* skip_flag = nullptr;

    // owner of the buffers listed in PM_SHARED_FIELDS (pm_api.cu) once the surface is built
    std::shared_ptr<PmSharedBuffers> shared;

    // triangle patches (pm_surface_create_tri); null for quadrilateral patches
    std::shared_ptr<const PmTriTables> tri;

    // launch-shape knobs beyond pm_opts (pm_surface_set_knobs / pm_surface_autotune)
    int batch_rb = 0;             // right-hand sides per block of the batched float32 sums (0 = 16)
    int batch_bps = 0;            // blocks aimed at per SM by the batched float32 sums (0 = 8)
    int fmm_streams = 0;          // FMM applies: 1 = one stream, 2 (0) = far field beside the P2P

    // scratch
    double* partial = nullptr;    // [max_split*N]
    int max_split = 0;
    float* sig32 = nullptr;       // [npatch*ppad]
    double* dbuf_in = nullptr;    // [N] host-pointer staging
    double* dbuf_out = nullptr;   // [N]
    size_t dbuf_n = 0;
};

// ----------------------------------------------------------------------------- modules
// quadrature setup (host)
void pm_build_tables(int p, QuadTables* T);
void pm_theta_plan(const QuadTables& T, double tol, double max_width,
                   std::vector<int>& off, std::vector<double>& ang,
                   std::vector<double>& wts, std::vector<double>& len);

// near field (pm_nearfield.cu)
pm_status pm_near_build(pm_surface* s, const QuadTables& T);
pm_status pm_near_combine_coeff(pm_surface* s, cudaStream_t st);
pm_status pm_near_apply(pm_surface* s, int which_K, const double* sigma, double* out,
                        int add_partials, int nsplit, pm_precision prec, cudaStream_t st);
void pm_patch_gradient(const pm_surface* s, const QuadTables& T, const double* a,
                       double* grad);

// smooth sums (pm_direct.cu)
int pm_direct_splits(const pm_surface* s, pm_precision prec, int which_K);
pm_status pm_prep_sources(pm_surface* s, const double* sigma, pm_precision prec,
                          cudaStream_t st);
pm_status pm_direct_sum(pm_surface* s, int which_K, pm_precision prec, int nsplit,
                        cudaStream_t st);
pm_status pm_pack_targets(pm_surface* s, cudaStream_t st);

// float-float sums (pm_ffsum.cu)
pm_status pm_ff_setup(pm_surface* s);
pm_status pm_pack_ff(pm_surface* s, cudaStream_t st);
pm_status pm_prep_ff(pm_surface* s, const double* sigma, cudaStream_t st);
int pm_ff_splits(const pm_surface* s);
pm_status pm_direct_ff(pm_surface* s, int which_K, int nsplit, cudaStream_t st);

// stored float-float matrices (pm_ffmat.cu)
size_t pm_ffmat_bytes(const pm_surface* s, int which);
void pm_ffmat_free(pm_surface* s);
bool pm_ffmat_has(const pm_surface* s, int which_K);
pm_status pm_ffmat_refresh(pm_surface* s, cudaStream_t st);
pm_status pm_ffmat_prep(pm_surface* s, const double* sigma, cudaStream_t st);
pm_status pm_ffmat_apply(pm_surface* s, int which_K, int* nsplit, cudaStream_t st);

// free device memory now (cudaMemGetInfo), or the value of the environment variable
// PM_FAKE_HBM_BYTES when set (a host-side stand-in for a full device) (pm_api.cu)
size_t pm_free_hbm_bytes();

// Chebyshev FMM (pm_fmm.cu)
pm_status pm_fmm_build(pm_surface* s);
int pm_fmm_splits();
pm_status pm_fmm_apply(pm_surface* s, int which_K, cudaStream_t st);
void pm_fmm_free(pm_surface* s);
pm_status pm_fmm_check(pm_surface* s);
size_t pm_fmm_need_bytes(const pm_surface* s);       // first-apply allocation model   // reads the tensor-core M2L error words (synchronises)

// tensor-core GEMM (pm_tcgemm.cu): C[(bcol0 + j) * ldc + crow0 + r] =
// sum_k A[arow0 + r][k] B[bcol0 + j][k] for r < 128, j < ncols over a list of
// tiles (arow0, bcol0, ncols <= 256, crow0); A, B 16-bit K-major, C float32.
struct PmTcGemm {
    alignas(64) unsigned char mapA[128];   // CUtensorMap of A (box 64 x 128)
    alignas(64) unsigned char mapB[128];   // CUtensorMap of B (box 64 x 256)
    int* tiles = nullptr;                  // [4 * ntiles] device
    int* err = nullptr;                    // device error word (PM_DEV_TIMEOUT)
    int ntiles = 0, nkb = 0, bf16 = 0;
    float* C = nullptr;
    long long ldc = 0;
};
pm_status pm_tcgemm_init(PmTcGemm* g, const void* A, long long a_rows, const void* B,
                         long long b_rows, int K, int bf16, const std::vector<int>& tiles,
                         float* C, long long ldc, long long c_cols);
pm_status pm_tcgemm_run(const PmTcGemm* g, int num_sms, const int* skip, cudaStream_t st,
                        int prio = 0);
pm_status pm_tcgemm_check(const PmTcGemm* g);
void pm_tcgemm_free(PmTcGemm* g);

// near-field CSR structure, patch unions and weight-set allocation after the
// patch geometry (centroid, radius, npatch_n) is in place (pm_nearfield.cu)
pm_status pm_near_structure(pm_surface* s);

// consistency checks (pm_check.cu): a finite scan of a device array
pm_status pm_check_finite(const double* v, size_t n, cudaStream_t st, const char* what);
extern "C" pm_status pm_surface_check(pm_surface* s);

// triangle patches (pm_tri.cu)
pm_status pm_tri_tables(int p, const double* ref_uvw, PmTriTables* T);
void pm_tri_theta_plan(const PmTriTables& T, const QuadTables& Q, double tol, double max_width,
                       std::vector<int>& off, std::vector<double>& ang, std::vector<double>& wts,
                       std::vector<double>& len);
pm_status pm_near_build_tri(pm_surface* s, const QuadTables& Q);
void pm_tri_gradient(const pm_surface* s, const double* a, double* grad);

// c != 0 (pm_nearfield.cu: near field; pm_helm.cu: sums, solve)
pm_status pm_near_build_c(pm_surface* s);
void pm_helm_free(pm_surface* s);

// batched applies and solves (pm_batch.cu)
pm_status pm_apply_batch(pm_surface* s, int kernel_K, const double* sigma, long long ld_sigma,
                         double* out, long long ld_out, int nrhs, pm_precision prec,
                         cudaStream_t st);
pm_status pm_solve_batch(pm_surface* s, const double* f, double* u, int nrhs, double tol,
                         int maxit, pm_precision prec, unsigned flags, double* sigma_out,
                         pm_solve_info* info, cudaStream_t st);
void pm_batch_free(pm_surface* s);
void pm_batch_solve_free(pm_surface* s);
size_t pm_batch_need_bytes(const pm_surface* s, int nrhs);

// solve (pm_solve.cu)
pm_status pm_solve_impl(pm_surface* s, const double* f, double* u, double tol, int maxit,
                        pm_precision prec, unsigned flags, double* sigma_out,
                        pm_solve_info* info, cudaStream_t st);

void pm_solve_free(pm_surface* s);
// device bytes a solve of nrhs right-hand sides would newly allocate (model)
size_t pm_solve_need_bytes(const pm_surface* s, int nrhs, pm_precision prec);

// Bound on the relative error of a float32 (or FMM) operator apply against the
// float64 operator, |(A32 - A) v| <= kOpRelErr |v|: measured errors are below
// 7e-6 (float32 direct sums and FMM, relative to |A v|, |A| = O(1) for the
// second-kind operator); the bound keeps a margin.  Used to decide when a
// refinement residual may be updated with a float32 apply (pm_solve.cu, pm_batch.cu).
constexpr double kOpRelErr = 1e-5;

// symmetric tile-pair float-float sums (pm_symsum.cu); partial slices capped at this size
constexpr double kSymPartialCap = 1024.0 * 1024.0 * 1024.0;
int pm_sym_tiles(const pm_surface* s);

// Tile pair (a, b), a <= b, of block p in the row-major upper triangle of the
// nt x nt tile grid: row a holds nt - a blocks and S(a) = a nt - a (a - 1) / 2
// blocks precede it.  The floating-point estimate is corrected by at most a
// step or two; the loops are bounded by nt.  (Symmetric float-float sums and the
// stored symmetric parametrix matrix.)
__device__ __forceinline__ void pm_tile_pair(int p, int nt, int& a, int& b) {
    const double B = 2.0 * nt + 1.0;
    int x = (int)((B - sqrt(fmax(B * B - 8.0 * (double)p, 0.0))) * 0.5);
    x = max(0, min(x, nt - 1));
    auto S = [nt](int r) { return (long long)r * nt - (long long)r * (r - 1) / 2; };
    for (int it = 0; it < nt && x > 0 && S(x) > p; ++it) --x;
    for (int it = 0; it < nt && x + 1 < nt && S(x + 1) <= p; ++it) ++x;
    a = x;
    b = x + (int)(p - S(x));
}
pm_status pm_sym_ff(pm_surface* s, int which_K, cudaStream_t st);
double pm_ff_grid(const pm_surface* s);

// apply helpers (pm_api.cu)
pm_status pm_apply_dev(pm_surface* s, int part_mask_K, int smooth, int near,
                       const double* sigma, double* out, pm_precision prec,
                       cudaStream_t st, int prepped = 0);
pm_status pm_ensure_scratch(pm_surface* s, size_t n);
size_t pm_operator_need_bytes(int npatch, int p, int clone);   // device bytes of a new operator (model)

// Records an event pair around the launches in its scope when profiling is on.
struct PhaseTimer {
    pm_surface* s;
    int phase;
    cudaStream_t st;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    PhaseTimer(pm_surface* s_, int phase_, cudaStream_t st_) : s(s_), phase(phase_), st(st_) {
        if (s->profiling && cudaEventCreate(&e0) == cudaSuccess &&
            cudaEventCreate(&e1) == cudaSuccess)
            cudaEventRecord(e0, st);
    }
    ~PhaseTimer() {
        if (e1) {
            cudaEventRecord(e1, st);
            s->prof_events.push_back({phase, {e0, e1}});
        } else if (e0) {
            cudaEventDestroy(e0);
        }
    }
};

template <typename T>
static inline pm_status pm_dmalloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
    if (e != cudaSuccess) {
        pm_set_error("cudaMalloc of %zu bytes failed: %s", count * sizeof(T),
                     cudaGetErrorString(e));
        *p = nullptr;
        return e == cudaErrorMemoryAllocation ? PM_ERR_OOM : PM_ERR_CUDA;
    }
    return PM_OK;
}

template <typename T>
static inline void pm_dfree(T*& p) {
    if (p) cudaFree((void*)p);
    p = nullptr;
}

static inline int pm_ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }
