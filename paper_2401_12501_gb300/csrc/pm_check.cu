// Consistency checks of a surface's device data (the library's stand-in for a
// memory checker, which this pool does not offer): every index the apply
// kernels follow is verified against the array it addresses, and the stored
// geometry, weights and corrections are scanned for non-finite values.  A
// failed check records (code, index) in a device word by compare-and-swap (the
// first failure wins) and the kernel carries on; nothing traps.  With
// -DPM_BOUNDS_CHECK the library also runs the check before, and a finite scan of
// the result after, every apply.
#include "pm_internal.cuh"

#include <cmath>

namespace {

enum CheckCode {
    CK_OK = 0,
    CK_ROW_PTR = 1,        // row_ptr not 0 at 0, not increasing, or not nblk at N
    CK_OWN_FIRST = 2,      // a row's first block is not its own patch
    CK_BLK_PATCH = 3,      // blk_patch outside [0, npatch)
    CK_BLK_ROW = 4,        // blk_row disagrees with row_ptr
    CK_UNION = 5,          // patch unions (multi-instance near field) inconsistent
    CK_THETA = 6,          // self-rule theta plan offsets or ray lengths invalid
    CK_NONFINITE = 7,      // a stored float64 value is NaN or Inf
    CK_NONFINITE32 = 8,    // a stored float32 value is NaN or Inf
};

__device__ inline void fail(int* word, int code, int index) {
    if (atomicCAS(word, 0, code) == 0) word[1] = index;
}

__global__ void k_check_rows(int N, int pp, int npatch, int nblk, const int* __restrict__ row_ptr,
                             const int* __restrict__ blk_patch, const int* __restrict__ blk_row,
                             int* __restrict__ word) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > N) return;
    if (i == 0 && row_ptr[0] != 0) fail(word, CK_ROW_PTR, 0);
    if (i == N) {
        if (row_ptr[N] != nblk) fail(word, CK_ROW_PTR, N);
        return;
    }
    const int b0 = row_ptr[i], b1 = row_ptr[i + 1];
    if (!(b0 >= 0 && b0 < b1 && b1 <= nblk)) {
        fail(word, CK_ROW_PTR, i);
        return;
    }
    if (blk_patch[b0] != i / pp) fail(word, CK_OWN_FIRST, i);
    for (int b = b0; b < b1; ++b) {
        const int P = blk_patch[b];
        if (P < 0 || P >= npatch) fail(word, CK_BLK_PATCH, b);
        if (blk_row[b] != i) fail(word, CK_BLK_ROW, b);
    }
}

// per patch: the union list of its rows' near patches holds valid patches, and
// every block of those rows points inside the union
__global__ void k_check_unions(int npatch, int pp, const int* __restrict__ row_ptr,
                               const int* __restrict__ nu_ptr, const int* __restrict__ nu_list,
                               const int* __restrict__ nu_blk, const int* __restrict__ blk_patch,
                               int* __restrict__ word) {
    const int P = blockIdx.x * blockDim.x + threadIdx.x;
    if (P >= npatch) return;
    const int u0 = nu_ptr[P], u1 = nu_ptr[P + 1];
    if (!(u0 >= 0 && u1 > u0)) {
        fail(word, CK_UNION, P);
        return;
    }
    for (int k = u0; k < u1; ++k)
        if (nu_list[k] < 0 || nu_list[k] >= npatch) fail(word, CK_UNION, P);
    for (int b = row_ptr[P * pp]; b < row_ptr[(P + 1) * pp]; ++b) {
        const int u = nu_blk[b];
        if (u < 0 || u >= u1 - u0 || nu_list[u0 + u] != blk_patch[b]) fail(word, CK_UNION, P);
    }
}

__global__ void k_check_theta(int pp, int nth, const int* __restrict__ off,
                              const double* __restrict__ L, int* __restrict__ word) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < pp && !(off[k] >= 0 && off[k] < off[k + 1] && off[k + 1] <= nth)) fail(word, CK_THETA, k);
    if (k < nth && !(L[k] > 0.0 && isfinite(L[k]))) fail(word, CK_THETA, k);
}

__global__ void k_check_finite(const double* __restrict__ v, size_t n, int* __restrict__ word) {
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (size_t)gridDim.x * blockDim.x)
        if (!isfinite(v[k])) fail(word, CK_NONFINITE, (int)(k < 0x7fffffff ? k : 0x7fffffff));
}

__global__ void k_check_finite32(const float* __restrict__ v, size_t n, int* __restrict__ word) {
    for (size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (size_t)gridDim.x * blockDim.x)
        if (!isfinite(v[k])) fail(word, CK_NONFINITE32, (int)(k < 0x7fffffff ? k : 0x7fffffff));
}

const char* code_name(int c) {
    switch (c) {
        case CK_ROW_PTR: return "near-field row pointers";
        case CK_OWN_FIRST: return "own patch not first in its row";
        case CK_BLK_PATCH: return "near-field block patch index";
        case CK_BLK_ROW: return "near-field block row index";
        case CK_UNION: return "patch near-field unions";
        case CK_THETA: return "self-rule theta plan";
        case CK_NONFINITE: return "non-finite float64 data";
        case CK_NONFINITE32: return "non-finite float32 data";
        default: return "unknown";
    }
}

}  // namespace

pm_status pm_check_finite(const double* v, size_t n, cudaStream_t st, const char* what) {
    int* word = nullptr;
    PM_TRY(pm_dmalloc(&word, 2));
    int h[2] = {0, 0};
    cudaError_t ce = cudaMemsetAsync(word, 0, 2 * sizeof(int), st);
    if (ce == cudaSuccess && n > 0) {
        k_check_finite<<<(int)std::min<size_t>(1024, (n + 255) / 256), 256, 0, st>>>(v, n, word);
        ce = cudaGetLastError();
    }
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(h, word, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    cudaFree(word);
    if (ce != cudaSuccess) {
        pm_set_error("finite check: %s", cudaGetErrorString(ce));
        return PM_ERR_CUDA;
    }
    if (h[0] != CK_OK) {
        pm_set_error("%s: non-finite value at %d", what, h[1]);
        return PM_ERR_INTERNAL;
    }
    return PM_OK;
}

extern "C" pm_status pm_surface_check(pm_surface* s) {
    if (!s || !s->row_ptr) {
        pm_set_error("pm_surface_check: NULL or unbuilt surface");
        return PM_ERR_INVALID_ARG;
    }
    PM_CUDA_TRY(cudaSetDevice(s->ctx->device));
    int* word = nullptr;
    PM_TRY(pm_dmalloc(&word, 2));
    const int N = s->N, pp = s->pp, nblk = s->nblk;
    cudaError_t ce = cudaMemset(word, 0, 2 * sizeof(int));
    auto finite = [&](const double* v, size_t n) {
        if (v && n && ce == cudaSuccess)
            k_check_finite<<<(int)std::min<size_t>(1024, (n + 255) / 256), 256>>>(v, n, word);
    };
    auto finite32 = [&](const float* v, size_t n) {
        if (v && n && ce == cudaSuccess)
            k_check_finite32<<<(int)std::min<size_t>(1024, (n + 255) / 256), 256>>>(v, n, word);
    };
    if (ce == cudaSuccess) {
        k_check_rows<<<pm_ceil_div(N + 1, 256), 256>>>(N, pp, s->npatch, nblk, s->row_ptr,
                                                        s->blk_patch, s->blk_row, word);
        ce = cudaDeviceSynchronize();
    }
    int h[2] = {0, 0};
    if (ce == cudaSuccess) ce = cudaMemcpy(h, word, sizeof(h), cudaMemcpyDeviceToHost);
    // the structure checks below follow row_ptr: only once it is sound
    if (ce == cudaSuccess && h[0] == CK_OK) {
        if (s->nu_ptr)
            k_check_unions<<<pm_ceil_div(s->npatch, 128), 128>>>(s->npatch, pp, s->row_ptr, s->nu_ptr,
                                                                s->nu_list, s->nu_blk, s->blk_patch,
                                                                word);
        if (s->th_off)
            k_check_theta<<<pm_ceil_div(std::max(pp, s->nth_total), 256), 256>>>(
                pp, s->nth_total, s->th_off, s->th_L, word);
        const size_t nv = (size_t)nblk * pp;
        finite(s->x, 3 * (size_t)N);
        finite(s->n, 3 * (size_t)N);
        finite(s->H, N);
        finite(s->w, N);
        finite(s->J, N);
        finite(s->W_lb, nv);
        finite(s->W_g, 3 * nv);
        finite(s->W_k, nv);
        if (s->has_coeff) {
            finite(s->a, N);
            finite(s->g, 3 * (size_t)N);
            finite(s->wa, N);
            finite(s->cR64, nv);
            finite(s->cK64, nv);
            finite32(s->cR32, (size_t)nblk * s->ppad);
            finite32(s->cK32, (size_t)nblk * s->ppad);
        }
        if (s->has_c) {
            finite(reinterpret_cast<const double*>(s->cRc), 2 * nv);
            finite(reinterpret_cast<const double*>(s->cKc), 2 * nv);
        }
        if (ce == cudaSuccess) ce = cudaGetLastError();
        if (ce == cudaSuccess) ce = cudaDeviceSynchronize();
        if (ce == cudaSuccess) ce = cudaMemcpy(h, word, sizeof(h), cudaMemcpyDeviceToHost);
    }
    cudaFree(word);
    if (ce != cudaSuccess) {
        pm_set_error("pm_surface_check: %s", cudaGetErrorString(ce));
        return PM_ERR_CUDA;
    }
    if (h[0] != CK_OK) {
        pm_set_error("pm_surface_check: %s (check %d) at index %d", code_name(h[0]), h[0], h[1]);
        return PM_ERR_INTERNAL;
    }
    if (s->ffm_err) {
        int fe = 0;
        PM_CUDA_TRY(cudaMemcpy(&fe, s->ffm_err, sizeof(int), cudaMemcpyDeviceToHost));
        if (fe != PM_DEV_OK) {
            pm_set_error("pm_surface_check: a stored-matrix GEMV's bulk copy did not arrive in time");
            return PM_ERR_TIMEOUT;
        }
    }
    return PM_OK;
}
