// Launch-shape knobs and the autotuner: every candidate shape of a surface's
// remainder apply is timed with CUDA events and the fastest is kept.  The knobs
// change float32 summation order and launch geometry only; the quadrature and
// the operator are untouched.
#include "pm_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

namespace {

// smooth fixed density for timing: sigma_r[i] = sin(0.37 i + r) + 0.5 cos(0.011 i)
__global__ void k_tune_fill(double* __restrict__ sigma, int N, int nrhs) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (long long)N * nrhs) return;
    const int i = (int)(e % N), r = (int)(e / N);
    sigma[e] = sin(0.37 * i + r) + 0.5 * cos(0.011 * i);
}

bool knobs_valid(const pm_knobs& k) {
    return (k.direct_tpt == 0 || k.direct_tpt == 1 || k.direct_tpt == 2 || k.direct_tpt == 4) &&
           k.direct_blocks_per_sm >= 0 && k.direct_blocks_per_sm <= 16 &&
           (k.batch_rhs_per_block == 0 || k.batch_rhs_per_block == 8 ||
            k.batch_rhs_per_block == 16 || k.batch_rhs_per_block == 32) &&
           k.batch_blocks_per_sm >= 0 && k.batch_blocks_per_sm <= 16 &&
           (k.fmm_depth == 0 || (k.fmm_depth >= 2 && k.fmm_depth <= 8)) &&
           k.fmm_streams >= 0 && k.fmm_streams <= 2;
}

pm_knobs knobs_of(const pm_surface* s) {
    pm_knobs k;
    k.direct_tpt = s->opts.direct_tpt;
    k.direct_blocks_per_sm = s->opts.direct_blocks_per_sm;
    k.batch_rhs_per_block = s->batch_rb;
    k.batch_blocks_per_sm = s->batch_bps;
    k.fmm_depth = s->opts.fmm_depth;
    k.fmm_streams = s->fmm_streams;
    return k;
}

void apply_knobs(pm_surface* s, const pm_knobs& k) {
    if (k.fmm_depth != s->opts.fmm_depth) pm_fmm_free(s);
    s->opts.direct_tpt = k.direct_tpt;
    s->opts.direct_blocks_per_sm = k.direct_blocks_per_sm;
    s->batch_rb = k.batch_rhs_per_block;
    s->batch_bps = k.batch_blocks_per_sm;
    s->opts.fmm_depth = k.fmm_depth;
    s->fmm_streams = k.fmm_streams;
    s->graph_epoch++;      // captured solve graphs hold launch shapes
}

struct TuneBuffers {
    double* sigma = nullptr;
    double* out = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~TuneBuffers() {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (st) cudaStreamDestroy(st);
        pm_dfree(sigma);
        pm_dfree(out);
    }
};

pm_status one_apply(pm_surface* s, int nrhs, pm_precision prec, TuneBuffers& B) {
    if (nrhs > 1)
        return pm_apply_batch(s, 0, B.sigma, s->N, B.out, s->N, nrhs, prec, B.st);
    return pm_apply_dev(s, 0, 1, 1, B.sigma, B.out, prec, B.st);
}

// median time of reps applies with knobs k (after one warm-up apply)
pm_status time_knobs(pm_surface* s, const pm_knobs& k, int nrhs, pm_precision prec, int reps,
                     TuneBuffers& B, double* ms) {
    apply_knobs(s, k);
    PM_TRY(one_apply(s, nrhs, prec, B));
    PM_CUDA_TRY(cudaStreamSynchronize(B.st));
    std::vector<double> t(reps);
    for (int r = 0; r < reps; ++r) {
        PM_CUDA_TRY(cudaEventRecord(B.e0, B.st));
        PM_TRY(one_apply(s, nrhs, prec, B));
        PM_CUDA_TRY(cudaEventRecord(B.e1, B.st));
        PM_CUDA_TRY(cudaEventSynchronize(B.e1));
        float f = 0.f;
        PM_CUDA_TRY(cudaEventElapsedTime(&f, B.e0, B.e1));
        t[r] = f;
    }
    std::sort(t.begin(), t.end());
    *ms = t[reps / 2];
    return PM_OK;
}

}  // namespace

extern "C" pm_status pm_surface_set_knobs(pm_surface* s, const pm_knobs* k) {
    if (!s || !k || !knobs_valid(*k)) {
        pm_set_error("pm_surface_set_knobs: NULL argument or knob out of range");
        return PM_ERR_INVALID_ARG;
    }
    PM_CUDA_TRY(cudaSetDevice(s->ctx->device));
    PM_CUDA_TRY(cudaDeviceSynchronize());   // no apply of this surface may be in flight
    apply_knobs(s, *k);
    return PM_OK;
}

extern "C" pm_status pm_surface_get_knobs(const pm_surface* s, pm_knobs* k) {
    if (!s || !k) {
        pm_set_error("pm_surface_get_knobs: NULL argument");
        return PM_ERR_INVALID_ARG;
    }
    *k = knobs_of(s);
    return PM_OK;
}

extern "C" pm_status pm_ctx_info(const pm_ctx* ctx, char* name, int len, int* num_sms) {
    if (!ctx || (name && len < 1)) {
        pm_set_error("pm_ctx_info: NULL context or len < 1");
        return PM_ERR_INVALID_ARG;
    }
    if (name) {
        std::strncpy(name, ctx->prop.name, (size_t)len - 1);
        name[len - 1] = '\0';
    }
    if (num_sms) *num_sms = ctx->num_sms;
    return PM_OK;
}

extern "C" pm_status pm_surface_autotune(pm_surface* s, int nrhs, pm_precision prec, int reps,
                                         pm_tune_result* out) {
    if (!s || !out || nrhs < 1 || reps < 1 || reps > 100 ||
        !(prec == PM_PREC_FP32 || (prec == PM_PREC_FMM && nrhs == 1))) {
        pm_set_error("pm_surface_autotune: NULL argument, nrhs < 1, reps outside 1..100, or a "
                     "precision other than float32 (any nrhs) / FMM (nrhs = 1)");
        return PM_ERR_INVALID_ARG;
    }
    if (!s->has_coeff) {
        pm_set_error("pm_surface_autotune: call pm_surface_set_coeff first");
        return PM_ERR_NO_COEFF;
    }
    if (s->has_c) {
        pm_set_error("pm_surface_autotune: the surface has c != 0");
        return PM_ERR_INVALID_ARG;
    }
    PM_CUDA_TRY(cudaSetDevice(s->ctx->device));
    PM_CUDA_TRY(cudaDeviceSynchronize());
    const pm_knobs orig = knobs_of(s);
    TuneBuffers B;
    const size_t n = (size_t)s->N * nrhs;
    PM_TRY(pm_dmalloc(&B.sigma, n));
    PM_TRY(pm_dmalloc(&B.out, n));
    PM_CUDA_TRY(cudaStreamCreateWithFlags(&B.st, cudaStreamNonBlocking));
    PM_CUDA_TRY(cudaEventCreate(&B.e0));
    PM_CUDA_TRY(cudaEventCreate(&B.e1));
    k_tune_fill<<<pm_ceil_div((long long)n, 256), 256, 0, B.st>>>(B.sigma, s->N, nrhs);
    PM_CUDA_TRY(cudaGetLastError());

    // candidates: the built-in choice first (its time is default_ms)
    std::vector<pm_knobs> cand;
    pm_knobs base = orig;
    if (prec == PM_PREC_FMM) {
        base.fmm_depth = 0;
        cand.push_back(base);
    } else if (nrhs == 1) {
        base.direct_tpt = 0;
        base.direct_blocks_per_sm = 0;
        cand.push_back(base);
        for (int tpt : {1, 2, 4})
            for (int bps : {4, 8, 12, 16}) {
                pm_knobs k = base;
                k.direct_tpt = tpt;
                k.direct_blocks_per_sm = bps;
                cand.push_back(k);
            }
    } else {
        base.batch_rhs_per_block = 0;
        base.batch_blocks_per_sm = 0;
        cand.push_back(base);
        for (int rb : {8, 16, 32})
            for (int bps : {4, 8, 12, 16}) {
                pm_knobs k = base;
                k.batch_rhs_per_block = rb;
                k.batch_blocks_per_sm = bps;
                cand.push_back(k);
            }
    }
    int timed = 0;
    double best_ms = 0.0, default_ms = 0.0;
    pm_knobs best = base;
    auto fail = [&](pm_status st) {
        cudaStreamSynchronize(B.st);
        apply_knobs(s, orig);
        return st;
    };
    for (size_t c = 0; c < cand.size(); ++c) {
        double ms = 0.0;
        const pm_status st = time_knobs(s, cand[c], nrhs, prec, reps, B, &ms);
        if (st != PM_OK) {
            // a neighbouring FMM depth may be infeasible (leaves above the P2P limit)
            // or too large for the device: skip it; anything else is an error
            if (prec == PM_PREC_FMM && c > 0 && (st == PM_ERR_INVALID_ARG || st == PM_ERR_OOM)) {
                cudaGetLastError();
                continue;
            }
            return fail(st);
        }
        ++timed;
        if (c == 0) {
            default_ms = ms;
            best_ms = ms;
            best = cand[c];
            if (prec == PM_PREC_FMM) {
                // the cost model's depth is now known: add its neighbours
                const int d0 = (int)s->fmm_stats[2];
                for (int d : {d0 - 1, d0 + 1})
                    if (d >= 2 && d <= 8) {
                        pm_knobs k = base;
                        k.fmm_depth = d;
                        cand.push_back(k);
                    }
            }
            continue;
        }
        if (ms < best_ms) {
            best_ms = ms;
            best = cand[c];
        }
    }
    apply_knobs(s, best);
    out->best = best;
    out->best_ms = best_ms;
    out->default_ms = default_ms;
    out->candidates = timed;
    return PM_OK;
}
