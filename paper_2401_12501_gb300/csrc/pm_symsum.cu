// Symmetric tile-pair float-float smooth sums: each unordered pair of nodes once.
//
// The float-float smooth sums y_i = sum_{j != i} s_j G(x_i, x_j) of the
// remainder and the parametrix share their pair geometry between (i, j) and (j, i): the offset
// r = x_i - x_j changes sign, r^2, 1/r^2 and log r^2 do not.  The parametrix
// kernel is symmetric (G_ji = G_ij); the remainder is not (its normal and
// coefficient factors belong to the target), but its reversed term needs only
// the source's factors, r -> -r:  G_ji = (n'_j . r)^2 / r^4 - (m_j . r) / r^2.
//
// Nodes are cut into tiles of 128.  Block (a, b), a <= b, runs tile a's 128
// targets (one per thread) against tile b's 128 sources (staged in shared
// memory, with their own normal and coefficient factors for the remainder):
//   - each thread sums its row s_j G_ij over the tile (row sum of target i);
//   - each warp sums s_i G_ji over its 32 targets for every source j, with
//     column sums that rotate across the lanes (see k_sym_ff), and the four
//     warps' values are combined in a fixed order (column sum of target j);
//   - the diagonal block a = b evaluates its ordered pairs one way only.
// Block (a, b) writes the row sums of tile a into partial slice b and the
// column sums of tile b into slice a; every (slice, row) is written exactly
// once, and the near-field kernel adds the nt slices of each row (the same
// layout as the one-sided sums' source splits).  All reductions have a fixed
// order: results are bit-reproducible.
//
// Padding: rows past N are targets at (-F, 0, 0), sources past N have zero
// strength at (+F, 0, 0), F outside the surface's bounding cube, so no padded
// pair coincides.  Kernels are launched for the surface's own tile count.
//
// The float32 remainder sum stays one-sided (pm_direct.cu): at ~18 instructions
// a pair, the three distinct shared-memory reads per pair of this schedule
// would bound it by shared-memory bandwidth, above what the shared geometry saves.
#include "pm_ff.cuh"
#include "pm_internal.cuh"

#include <algorithm>
#include <cmath>

namespace {

using namespace pmff;

constexpr int kT = 128;           // tile = block size
constexpr int kW = kT / 32;       // warps per block

// ------------------------------------------------------------- float-float sums
// Remainder (KERNEL_K = false): src = src_ff (float-float coordinates, strength
// in .w), tg = tgt_ff (x, n', m pairs).  Parametrix (KERNEL_K = true): src =
// src_kg (grid-split coordinates and strengths; the target's coordinates are
// its own entry), tg unused.
//
// Schedule: the 128 sources are taken in four sub-tiles of 32; at step k of a
// sub-tile, lane l evaluates source (l + k) mod 32 of it, so the 32 lanes work
// on 32 different sources (conflict-free shared reads) and each lane carries
// the column sum of the source it just evaluated.  After the step the column
// sums rotate down one lane (lane l takes lane l + 1's), so lane l next holds
// the column of the source it evaluates next; after 32 steps each column sum
// has visited all 32 targets of the warp and sits on lane (its source mod 32).
// Rotation costs two shuffles per step instead of a per-source warp reduction.
template <bool KERNEL_K>
struct SymCtx {
    const float4 *sA, *sB, *sNh, *sNl, *sMh, *sMl, *stab;
    const ff *X, *NP, *MM;
    ff si;
};

// The pair loop of one block; DIAG: tile against itself, rows only, the self
// pair evaluated at a unit offset with zero strength (exactly zero).
template <bool KERNEL_K, bool DIAG>
__device__ __forceinline__ void sym_loop(const SymCtx<KERNEL_K>& C, int lane, int tid, ff& acc,
                                         ff* colv) {
    const int src_lane_next = (lane + 1) & 31;
    const ff X0 = C.X[0], X1 = C.X[1], X2 = C.X[2];
#pragma unroll
    for (int c = 0; c < kW; ++c) {
        ff cacc{0.f, 0.f};                         // column sum of the source evaluated next
#pragma unroll 2
        for (int k = 0; k < 32; ++k) {
            const int q = c * 32 + ((lane + k) & 31);
            const float4 A = C.sA[q], B = C.sB[q];
            const ff dx = KERNEL_K ? ff_grid_sub(X0, A.x, B.x) : ff_sub(X0, ff{A.x, B.x});
            const ff dy = KERNEL_K ? ff_grid_sub(X1, A.y, B.y) : ff_sub(X1, ff{A.y, B.y});
            const ff dz = KERNEL_K ? ff_grid_sub(X2, A.z, B.z) : ff_sub(X2, ff{A.z, B.z});
            ff r2 = ff_add_lazy(ff_add_lazy(ff_sqr_lazy(dx), ff_sqr_lazy(dy)), ff_sqr_lazy(dz));
            ff sj{A.w, B.w};
            if (DIAG && q == tid) {
                r2 = ff{1.f, 0.f};
                sj = ff{0.f, 0.f};
            }
            ff row, col{0.f, 0.f};
            if (KERNEL_K) {
                const ff L = ff_norm(ff_log_lazy(r2, C.stab));
                row = ff_mul_lazy(sj, L);
                if (!DIAG) col = ff_mul_lazy(C.si, L);
            } else {
                const ff inv = ff_rcp_lazy(r2);
                const ff nr = ff_norm(ff_add_lazy(ff_add_lazy(ff_mul_lazy(C.NP[0], dx),
                                                              ff_mul_lazy(C.NP[1], dy)),
                                                  ff_mul_lazy(C.NP[2], dz)));
                const ff mr = ff_add_lazy(ff_add_lazy(ff_mul_lazy(C.MM[0], dx),
                                                      ff_mul_lazy(C.MM[1], dy)),
                                          ff_mul_lazy(C.MM[2], dz));
                const ff inner = ff_norm(ff_add_lazy(ff_mul_lazy(nr, ff_mul_lazy(nr, inv)), mr));
                row = ff_mul_lazy(ff_mul_lazy(sj, inv), inner);
                if (!DIAG) {
                    const float4 nh = C.sNh[q], nl = C.sNl[q], mh = C.sMh[q], ml = C.sMl[q];
                    const ff nrj = ff_norm(ff_add_lazy(
                        ff_add_lazy(ff_mul_lazy(ff{nh.x, nl.x}, dx), ff_mul_lazy(ff{nh.y, nl.y}, dy)),
                        ff_mul_lazy(ff{nh.z, nl.z}, dz)));
                    const ff mrj = ff_add_lazy(
                        ff_add_lazy(ff_mul_lazy(ff{mh.x, ml.x}, dx), ff_mul_lazy(ff{mh.y, ml.y}, dy)),
                        ff_mul_lazy(ff{mh.z, ml.z}, dz));
                    // reversed pair: r -> -r, so (n'_j . r)^2 is unchanged and m_j . r flips
                    const ff innerj = ff_norm(ff_add_lazy(ff_mul_lazy(nrj, ff_mul_lazy(nrj, inv)),
                                                          ff{-mrj.h, -mrj.l}));
                    col = ff_mul_lazy(ff_mul_lazy(C.si, inv), innerj);
                }
            }
            // row: TwoSum on the high words, error terms in the low word
            const float t = acc.h + row.h;
            const float bp = t - acc.h;
            acc.l += ((acc.h - (t - bp)) + (row.h - bp)) + row.l;
            acc.h = t;
            if (!DIAG) {
                cacc = ff_add_lazy(cacc, col);
                cacc = ff{__shfl_sync(0xffffffffu, cacc.h, src_lane_next),
                          __shfl_sync(0xffffffffu, cacc.l, src_lane_next)};
            }
        }
        colv[c] = cacc;                            // column c * 32 + lane of this warp's targets
    }
}

// 7 blocks of 128 threads per SM: the register cap (72) keeps 28 warps resident
// against 24 at the unconstrained 80 registers, at the cost of 16 bytes of spill in
// the remainder form; measured on the 98,304-node torus, 44.1 -> 41.1 ms (remainder),
// 17.6 ms unchanged (parametrix); 8 blocks (64 registers, 76-byte spills) gave 43.6 ms.
template <bool KERNEL_K>
__global__ void __launch_bounds__(kT, 7)
k_sym_ff(const float4* __restrict__ src, const float4* __restrict__ tg,
         const float4* __restrict__ log_tab, int N, int nt, float far_h, float far_l,
         float2* __restrict__ partial, const int* __restrict__ skip) {
    if (skip && *skip) return;
    constexpr int kNS = KERNEL_K ? 1 : kT;
    __shared__ float4 sA[kT], sB[kT];                 // source (hi, s_h), (lo, s_l)
    __shared__ float4 sNh[kNS], sNl[kNS], sMh[kNS], sMl[kNS];   // source n', m (remainder)
    __shared__ float4 stab[KERNEL_K ? kLogTable : 1];
    __shared__ float2 csh[kW][kT];
    int a, b;
    pm_tile_pair(blockIdx.x, nt, a, b);
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int i = a * kT + tid;
    const int j = b * kT + tid;
    if (KERNEL_K)
        for (int k = tid; k < kLogTable; k += kT) stab[k] = log_tab[k];
    // stage tile b's sources (padding: zero strength at +F)
    if (j < N) {
        sA[tid] = src[2 * (size_t)j];
        sB[tid] = src[2 * (size_t)j + 1];
        if (!KERNEL_K) {
            sNh[tid] = tg[6 * (size_t)j + 2];
            sNl[tid] = tg[6 * (size_t)j + 3];
            sMh[tid] = tg[6 * (size_t)j + 4];
            sMl[tid] = tg[6 * (size_t)j + 5];
        }
    } else {
        sA[tid] = make_float4(far_h, 0.f, 0.f, 0.f);
        sB[tid] = make_float4(far_l, 0.f, 0.f, 0.f);
        if (!KERNEL_K) sNh[tid] = sNl[tid] = sMh[tid] = sMl[tid] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    // this thread's target (padding: at -F) and its strength as a source
    ff X[3], NP[3], MM[3], si{0.f, 0.f};
    if (i < N) {
        const float4 p0 = src[2 * (size_t)i], p1 = src[2 * (size_t)i + 1];
        si = ff{p0.w, p1.w};
        if (KERNEL_K) {
            X[0] = ff{p0.x, p1.x}; X[1] = ff{p0.y, p1.y}; X[2] = ff{p0.z, p1.z};
        } else {
            float4 v[6];
            for (int q = 0; q < 6; ++q) v[q] = tg[6 * (size_t)i + q];
            X[0] = ff{v[0].x, v[1].x}; X[1] = ff{v[0].y, v[1].y}; X[2] = ff{v[0].z, v[1].z};
            NP[0] = ff{v[2].x, v[3].x}; NP[1] = ff{v[2].y, v[3].y}; NP[2] = ff{v[2].z, v[3].z};
            MM[0] = ff{v[4].x, v[5].x}; MM[1] = ff{v[4].y, v[5].y}; MM[2] = ff{v[4].z, v[5].z};
        }
    } else {
        X[0] = ff{-far_h, -far_l}; X[1] = ff{0.f, 0.f}; X[2] = ff{0.f, 0.f};
        for (int d = 0; d < 3; ++d) NP[d] = MM[d] = ff{0.f, 0.f};
    }
    __syncthreads();
    const bool diag = (a == b);
    ff acc{0.f, 0.f};
    ff colv[kW];
    const SymCtx<KERNEL_K> C{sA, sB, sNh, sNl, sMh, sMl, stab, X, NP, MM, si};
    if (diag)
        sym_loop<KERNEL_K, true>(C, lane, tid, acc, colv);
    else
        sym_loop<KERNEL_K, false>(C, lane, tid, acc, colv);
    const float scale_h = KERNEL_K ? (float)(1.0 / (4.0 * M_PI)) : 1.f;
    const float scale_l = KERNEL_K ? (float)(1.0 / (4.0 * M_PI) - (double)(float)(1.0 / (4.0 * M_PI))) : 0.f;
    if (i < N) {
        ff v = ff_norm(acc);
        if (KERNEL_K) v = ff_mul(v, ff{scale_h, scale_l});
        partial[(size_t)b * N + i] = make_float2(v.h, v.l);
    }
    if (diag) return;
#pragma unroll
    for (int c = 0; c < kW; ++c) csh[wid][c * 32 + lane] = make_float2(colv[c].h, colv[c].l);
    __syncthreads();
    if (j < N) {
        ff v{csh[0][tid].x, csh[0][tid].y};
#pragma unroll
        for (int w = 1; w < kW; ++w) v = ff_add_lazy(v, ff{csh[w][tid].x, csh[w][tid].y});
        v = ff_norm(v);
        if (KERNEL_K) v = ff_mul(v, ff{scale_h, scale_l});
        partial[(size_t)a * N + j] = make_float2(v.h, v.l);
    }
}

}  // namespace

// Tile count of the symmetric sums, or 0 when the surface uses the one-sided
// kernels (option off, too few nodes, or partial slices above the memory cap).
int pm_sym_tiles(const pm_surface* s) {
    if (!s->opts.direct_symmetric || s->N < 2 * kT) return 0;
    const int nt = pm_ceil_div(s->N, kT);
    if ((double)nt * s->N * sizeof(float2) > kSymPartialCap) return 0;
    return nt;
}

// Padding offset F = 2^(E + 1), twice the half-width 2^E >= max |x| of the
// coordinate grid (pm_ff_grid): every real point is at least 2^E away, and
// differences to it stay exact on the grid.
static double sym_far(const pm_surface* s) { return pm_ff_grid(s) * 8388608.0; }

pm_status pm_sym_ff(pm_surface* s, int which_K, cudaStream_t st) {
    const int nt = pm_sym_tiles(s);
    const int nblocks = nt * (nt + 1) / 2;
    float2* part = reinterpret_cast<float2*>(s->partial);
    const double F = sym_far(s);
    const float fh = (float)F, fl = 0.f;
    if (which_K)
        k_sym_ff<true><<<nblocks, kT, 0, st>>>(s->src_kg, s->tgt_ff, s->log_tab, s->N, nt, fh, fl,
                                               part, s->skip_flag);
    else
        k_sym_ff<false><<<nblocks, kT, 0, st>>>(s->src_ff, s->tgt_ff, s->log_tab, s->N, nt, fh,
                                                fl, part, s->skip_flag);
    PM_CUDA_TRY(cudaGetLastError());
    return PM_OK;
}
