// Stored float-float smooth-sum matrices: the accurate applies as a streaming GEMV.
//
// The refinement residual f - A sigma and the representation u = K~ sigma need the
// smooth sums y_i = sum_{j != i} s_j G(x_i, x_j) to float64-class accuracy, with
// s_j = w_j sigma_j / a_j (Sec. 6.1; the smooth rule of the Nystrom discretisation).
// Evaluated pair by pair in float-float (pm_symsum.cu) they cost ~140 FP32
// instructions per ordered pair of the remainder and ~65 of the parametrix, issue-
// bound.  Their matrices G_ij depend on the operator but not on sigma, so when HBM
// holds them they are evaluated once, in the same float-float arithmetic, and kept;
// every later float-float apply is then one pass over the matrix, bound by HBM
// bandwidth.  The paper's method stores its operators too (compressed, in its
// interpolative FMM); here the stored form is dense.
//
// Entries: remainder G_ij = (n'_i . r)^2 / r^4 + (m_i . r) / r^2 with r = x_i - x_j
// (eq. explicit_remainder, c = 0, the target's coefficient factors n' and m of the
// packed float-float targets); parametrix G_ij = log(r^2) / (4 pi) (eq. diff_param,
// 1/a_j in s_j).  G_ii = 0 and padding entries are 0.  The remainder matrix depends
// on the coefficient a and is re-evaluated by set_coeff; the parametrix matrix
// depends on the geometry only.
//
// Entry format, 6 bytes: the float-float value h + l (|l| <= ulp(h) / 2 <= 2^-24 |h|)
// as the float h and the 16-bit code u = q + 2^15 of the integer q = round(l / (h 2^-39)),
// |q| <= 2^15 - 1, so that h + q h 2^-39 is the value to within 2^-40 |h| (relative
// 9.1e-13 per entry, against ~2^-46 of the float-float evaluation).  q becomes a float
// through the significand of 2^23 + u (one byte permutation).  A matrix is two planes,
// the floats and the 16-bit codes, 4 + 2 bytes an entry instead of the 8 of a float pair.
//
// Row layout (the remainder; the parametrix where the symmetric layout is not used):
// [N][ld] per plane, ld = N rounded up to 128.  GEMV: a block takes 32 rows (4 per
// warp) and one column segment; lane l takes column quads l, l + 32, ... of the
// segment, loads 16 + 8 bytes (four entries) of each of its 4 rows and the four
// columns' float-float strengths, and accumulates each row in float-float (TwoProduct
// by FMA, TwoSum on the high words, the error terms summed in the low word).  The
// warp's 32 partial sums of a row are added in a fixed butterfly order; segment k
// writes partial slice k, which the float64 near-field kernel adds with the
// corrections.  Results are bit-reproducible.
//
// Symmetric layout (the parametrix on surfaces that use the symmetric tile-pair sums,
// pm_symsum.cu): only the upper triangle of 128 x 128 tiles is stored, half the
// bytes, and one pass over a tile (a, b), a < b, gives both the row sums of tile a
// against tile b's strengths and the column sums of tile b against tile a's, with the
// same block schedule and partial-slice layout as those sums: a block's four warps
// take 32 rows each; at step k of a 32-column sub-tile lane l reads the entry of its
// row and column (l + k) mod 32, adds it times that column's strength to its row sum
// and times its own row's strength to the column sum it carries, and the column sums
// rotate one lane per step.  Entries are stored in the order the lanes read them (four
// steps per load, a warp's loads contiguous).
#include "pm_ff.cuh"
#include "pm_internal.cuh"

#include <algorithm>
#include <cmath>

namespace {

using namespace pmff;

constexpr int kBuildRows = 8;        // rows per build block, one per warp
constexpr int kBuildStage = 512;     // source columns staged in shared memory per step
constexpr int kGemvWarps = 8;
constexpr int kGemvRowsPerWarp = 4;
constexpr int kGemvRows = kGemvWarps * kGemvRowsPerWarp;
constexpr int kLd = 128;             // row layout: ld is a multiple of this
constexpr int kST = 128;             // symmetric layout: tile side (= the symmetric sums' tile)
constexpr size_t kTileHiBytes = (size_t)kST * kST * sizeof(float);
constexpr size_t kTileBytes = (size_t)kST * kST * 6;

// ------------------------------------------------------------------ entry format
// 16-bit code u = q + 2^15 of the low word (see the file header)
__device__ __forceinline__ unsigned ff_code(ff e) {
    const float sc = e.h * 0x1p-39f;
    const float r = sc != 0.f ? e.l / sc : 0.f;
    return (unsigned)((int)fmaxf(-32767.f, fminf(32767.f, rintf(r))) + 32768);
}

// 2^23 + u as a float, for the code in the low (SEL_HIGH = false) or high half of w
template <bool SEL_HIGH>
__device__ __forceinline__ float code_float(unsigned w) {
    return __uint_as_float(__byte_perm(w, 0x4B000000u, SEL_HIGH ? 0x7632u : 0x7610u));
}

// q 2^-39 from 2^23 + u, exactly: (2^23 + u) 2^-39 - (2^23 + 2^15) 2^-39
constexpr float kCodeScale = 0x1p-39f;
constexpr float kCodeBias = -(0x1p-16f + 0x1p-24f);

// low word of the entry with high word h and code word f = 2^23 + u
__device__ __forceinline__ float ff_lo(float h, float f) {
    return fmaf(f, kCodeScale, kCodeBias) * h;
}

__device__ __forceinline__ unsigned code_pack(unsigned lo, unsigned hi) { return lo | (hi << 16); }

// ------------------------------------------------------------- bulk copies (TMA)
constexpr unsigned long long kBulkWaitNs = 2000000000ull;   // give up on a copy after 2 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void bar_init(uint32_t bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void bar_expect(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool bar_test(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred P;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, P;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}
// bounded wait for the phase with the given parity; false (and *err set) after 2 s
__device__ bool bar_wait(uint32_t bar, uint32_t parity, int* err) {
    if (bar_test(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (uint32_t it = 1;; ++it) {
        if (bar_test(bar, parity)) return true;
        if ((it & 63) == 0 && global_ns() - t0 > kBulkWaitNs) {
            atomicExch(err, PM_DEV_TIMEOUT);
            return false;
        }
    }
}
// global -> shared bulk copy (16-byte aligned addresses, size a multiple of 16)
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(dst), "l"(reinterpret_cast<unsigned long long>(src)), "r"(bytes), "r"(bar)
        : "memory");
}

// --------------------------------------------------------------------- build
// Remainder (KERNEL_K = false): src = src_ff (plain float-float coordinates),
// tg = tgt_ff (x, n', m pairs of the target).  Parametrix (KERNEL_K = true):
// src = src_kg (grid-split coordinates; the target reads its own entry).
// The per-pair arithmetic is that of the float-float sums (pm_ffsum.cu) without
// the strength factor.
template <bool KERNEL_K>
__device__ __forceinline__ ff pair_entry(const ff* X, const ff* NP, const ff* MM, float4 A,
                                         float4 B, const float4* stab, ff scale) {
    const ff dx = KERNEL_K ? ff_grid_sub(X[0], A.x, B.x) : ff_sub(X[0], ff{A.x, B.x});
    const ff dy = KERNEL_K ? ff_grid_sub(X[1], A.y, B.y) : ff_sub(X[1], ff{A.y, B.y});
    const ff dz = KERNEL_K ? ff_grid_sub(X[2], A.z, B.z) : ff_sub(X[2], ff{A.z, B.z});
    const ff r2 = ff_add_lazy(ff_add_lazy(ff_sqr_lazy(dx), ff_sqr_lazy(dy)), ff_sqr_lazy(dz));
    if (KERNEL_K) return ff_mul(ff_norm(ff_log_lazy(r2, stab)), scale);
    const ff inv = ff_rcp_lazy(r2);
    const ff nr = ff_norm(ff_add_lazy(ff_add_lazy(ff_mul_lazy(NP[0], dx), ff_mul_lazy(NP[1], dy)),
                                      ff_mul_lazy(NP[2], dz)));
    const ff mr = ff_add_lazy(ff_add_lazy(ff_mul_lazy(MM[0], dx), ff_mul_lazy(MM[1], dy)),
                              ff_mul_lazy(MM[2], dz));
    const ff inner = ff_norm(ff_add_lazy(ff_mul_lazy(nr, ff_mul_lazy(nr, inv)), mr));
    return ff_mul(inv, inner);
}

// row layout: planes Mh [N][ld] (float) and Mq [N][ld] (16-bit codes)
template <bool KERNEL_K>
__global__ void __launch_bounds__(kBuildRows * 32)
k_ffmat_build(const float4* __restrict__ src, const float4* __restrict__ tg,
              const float4* __restrict__ log_tab, int N, int ld, float* __restrict__ Mh,
              unsigned short* __restrict__ Mq) {
    __shared__ float4 sA[kBuildStage], sB[kBuildStage];
    __shared__ float4 stab[KERNEL_K ? kLogTable : 1];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (KERNEL_K)
        for (int k = tid; k < kLogTable; k += blockDim.x) stab[k] = log_tab[k];
    const int i = blockIdx.x * kBuildRows + warp;
    const bool row_ok = i < N;
    const int ii = row_ok ? i : 0;
    ff X[3], NP[3], MM[3];
    if (KERNEL_K) {
        const float4 a = src[2 * (size_t)ii], b = src[2 * (size_t)ii + 1];
        X[0] = ff{a.x, b.x}; X[1] = ff{a.y, b.y}; X[2] = ff{a.z, b.z};
    } else {
        float4 v[6];
        for (int q = 0; q < 6; ++q) v[q] = tg[6 * (size_t)ii + q];
        X[0] = ff{v[0].x, v[1].x}; X[1] = ff{v[0].y, v[1].y}; X[2] = ff{v[0].z, v[1].z};
        NP[0] = ff{v[2].x, v[3].x}; NP[1] = ff{v[2].y, v[3].y}; NP[2] = ff{v[2].z, v[3].z};
        MM[0] = ff{v[4].x, v[5].x}; MM[1] = ff{v[4].y, v[5].y}; MM[2] = ff{v[4].z, v[5].z};
    }
    const ff scale = KERNEL_K ? ff_from_double(1.0 / (4.0 * M_PI)) : ff{1.f, 0.f};
    float* rowh = Mh + (size_t)ii * ld;
    unsigned short* rowq = Mq + (size_t)ii * ld;
    for (int base = 0; base < ld; base += kBuildStage) {
        __syncthreads();
        for (int k = tid; k < kBuildStage; k += blockDim.x) {
            const int j = base + k;
            if (j < N) {
                sA[k] = src[2 * (size_t)j];
                sB[k] = src[2 * (size_t)j + 1];
            } else {
                sA[k] = sB[k] = make_float4(0.f, 0.f, 0.f, 0.f);
            }
        }
        __syncthreads();
        if (!row_ok) continue;
        const int kend = min(kBuildStage, ld - base);
        for (int k = lane; k < kend; k += 32) {
            const int j = base + k;
            ff e{0.f, 0.f};
            if (j < N && j != i) e = pair_entry<KERNEL_K>(X, NP, MM, sA[k], sB[k], stab, scale);
            __stcs(rowh + j, e.h);
            rowq[j] = (unsigned short)ff_code(e);
        }
    }
}

// Symmetric parametrix layout, block per tile pair (a, b) of pm_tile_pair: warp w,
// sub-tile c, step k = 4 kq + t, lane l hold the entry of row a 128 + 32 w + l and
// column b 128 + 32 c + ((l + k) mod 32); its float is element t of float4
// (((w 4 + c) 8 + kq) 32 + l) of the tile's float plane, its code element t of the
// same-numbered 8-byte group of the code plane that follows.
__global__ void __launch_bounds__(kST)
k_ffmat_symK_build(const float4* __restrict__ src, const float4* __restrict__ log_tab, int N,
                   int nt, unsigned char* __restrict__ T) {
    __shared__ float4 sA[kST], sB[kST];
    __shared__ float4 stab[kLogTable];
    int a, b;
    pm_tile_pair(blockIdx.x, nt, a, b);
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    for (int k = tid; k < kLogTable; k += kST) stab[k] = log_tab[k];
    const int i = a * kST + tid, j = b * kST + tid;
    if (j < N) {
        sA[tid] = src[2 * (size_t)j];
        sB[tid] = src[2 * (size_t)j + 1];
    } else {
        sA[tid] = sB[tid] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    ff X[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    if (i < N) {
        const float4 p0 = src[2 * (size_t)i], p1 = src[2 * (size_t)i + 1];
        X[0] = ff{p0.x, p1.x}; X[1] = ff{p0.y, p1.y}; X[2] = ff{p0.z, p1.z};
    }
    __syncthreads();
    const ff scale = ff_from_double(1.0 / (4.0 * M_PI));
    unsigned char* tile = T + (size_t)blockIdx.x * kTileBytes;
    float4* oh = reinterpret_cast<float4*>(tile) + (size_t)w * (4 * 8 * 32) + lane;
    uint2* oq = reinterpret_cast<uint2*>(tile + kTileHiBytes) + (size_t)w * (4 * 8 * 32) + lane;
    for (int c = 0; c < 4; ++c) {
        for (int kq = 0; kq < 8; ++kq) {
            float h[4];
            unsigned q[4];
            for (int t = 0; t < 4; ++t) {
                const int col = c * 32 + ((lane + 4 * kq + t) & 31);
                const int jj = b * kST + col;
                ff e{0.f, 0.f};
                if (i < N && jj < N && jj != i)
                    e = pair_entry<true>(X, nullptr, nullptr, sA[col], sB[col], stab, scale);
                h[t] = e.h;
                q[t] = ff_code(e);
            }
            const int o = (c * 8 + kq) * 32;
            __stcs(oh + o, make_float4(h[0], h[1], h[2], h[3]));
            __stcs(oq + o, make_uint2(code_pack(q[0], q[1]), code_pack(q[2], q[3])));
        }
    }
}

// s_j = w_j sigma_j / a_j in float-float, [ld] (the padding entries stay zero)
__global__ void k_ffmat_prep(const double* __restrict__ sigma, const double* __restrict__ wa,
                             float2* __restrict__ sv, int N, const int* __restrict__ skip) {
    if (skip && *skip) return;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    const ff s = ff_from_double(wa[j] * sigma[j]);
    sv[j] = make_float2(s.h, s.l);
}

// ---------------------------------------------------------------------- GEMV
// (S, E) += (mh + ml)(sh + sl): TwoProduct of the high words by FMA, the cross
// terms into its error, TwoSum of the high words, every error term into E.
__device__ __forceinline__ void ff_mac(float& S, float& E, float mh, float ml, float sh, float sl) {
    const float p = mh * sh;
    float e = fmaf(mh, sh, -p);
    e = fmaf(mh, sl, e);
    e = fmaf(ml, sh, e);
    const float t = S + p;
    const float bp = t - S;
    E += ((S - (t - bp)) + (p - bp)) + e;
    S = t;
}

// four entries (floats h, codes w) of one row against four columns' strengths
// sa = (s0 hi, lo, s1 hi, lo), sb = (s2, s3)
__device__ __forceinline__ void ff_mac4(float& S, float& E, float4 h, uint2 w, float4 sa,
                                        float4 sb) {
    ff_mac(S, E, h.x, ff_lo(h.x, code_float<false>(w.x)), sa.x, sa.y);
    ff_mac(S, E, h.y, ff_lo(h.y, code_float<true>(w.x)), sa.z, sa.w);
    ff_mac(S, E, h.z, ff_lo(h.z, code_float<false>(w.y)), sb.x, sb.y);
    ff_mac(S, E, h.w, ff_lo(h.w, code_float<true>(w.y)), sb.z, sb.w);
}

__global__ void __launch_bounds__(kGemvWarps * 32)
k_ffmat_gemv(const float4* __restrict__ Mh, const uint2* __restrict__ Mq, long long ldq,
             const float4* __restrict__ sv, int N, int cs, int ld, float2* __restrict__ partial,
             const int* __restrict__ skip) {
    if (skip && *skip) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int r0 = (blockIdx.x * kGemvWarps + warp) * kGemvRowsPerWarp;
    if (r0 >= N) return;                                  // whole warp
    const int nr = min(kGemvRowsPerWarp, N - r0);
    const int q0 = (blockIdx.y * cs) >> 2, q1 = min(blockIdx.y * cs + cs, ld) >> 2;   // column quads
    const float4* Hr[kGemvRowsPerWarp];
    const uint2* Qr[kGemvRowsPerWarp];
#pragma unroll
    for (int r = 0; r < kGemvRowsPerWarp; ++r) {
        const size_t row = (size_t)(r0 + min(r, nr - 1)) * ldq;
        Hr[r] = Mh + row;
        Qr[r] = Mq + row;
    }
    float S[kGemvRowsPerWarp], E[kGemvRowsPerWarp];
#pragma unroll
    for (int r = 0; r < kGemvRowsPerWarp; ++r) S[r] = E[r] = 0.f;
#pragma unroll 2
    for (int q = q0 + lane; q < q1; q += 32) {
        const float4 sa = __ldg(sv + 2 * q), sb = __ldg(sv + 2 * q + 1);
        float4 h[kGemvRowsPerWarp];
        uint2 w[kGemvRowsPerWarp];
#pragma unroll
        for (int r = 0; r < kGemvRowsPerWarp; ++r) {
            h[r] = __ldcs(Hr[r] + q);
            w[r] = __ldcs(Qr[r] + q);
        }
#pragma unroll
        for (int r = 0; r < kGemvRowsPerWarp; ++r) ff_mac4(S[r], E[r], h[r], w[r], sa, sb);
    }
    // butterfly over the lanes in float-float: every lane ends with the row sum
#pragma unroll
    for (int r = 0; r < kGemvRowsPerWarp; ++r) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float S2 = __shfl_xor_sync(0xffffffffu, S[r], o);
            const float E2 = __shfl_xor_sync(0xffffffffu, E[r], o);
            float t, e;
            two_sum(S[r], S2, t, e);
            E[r] = (E[r] + E2) + e;
            S[r] = t;
        }
    }
    float2* out = partial + (size_t)blockIdx.y * N + r0;
#pragma unroll
    for (int r = 0; r < kGemvRowsPerWarp; ++r)
        if (lane == r && r < nr) {
            const ff v = ff_norm(ff{S[r], E[r]});
            out[r] = make_float2(v.h, v.l);
        }
}

// Packed float-float multiply-add on two independent chains (S.x, E.x), (S.y, E.y):
// ff_mac on each, one f32x2 instruction per step of both.
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

__device__ __forceinline__ void ff_mac2(float2& S, float2& E, float2 h, float2 l, float2 sh,
                                        float2 sl) {
    const float2 p = __fmul2_rn(h, sh);
    float2 e = __ffma2_rn(h, sh, neg2(p));
    e = __ffma2_rn(h, sl, e);
    e = __ffma2_rn(l, sh, e);
    const float2 t = __fadd2_rn(S, p);
    const float2 bp = __fadd2_rn(t, neg2(S));
    const float2 d1 = __fadd2_rn(S, neg2(__fadd2_rn(t, neg2(bp))));
    const float2 d2 = __fadd2_rn(p, neg2(bp));
    E = __fadd2_rn(E, __fadd2_rn(__fadd2_rn(d1, d2), e));
    S = t;
}

// (S, E) of one chain += (S2, E2) of another, in float-float
__device__ __forceinline__ void ff_join(float& S, float& E, float S2, float E2) {
    float t, d;
    two_sum(S, S2, t, d);
    E = (E + E2) + d;
    S = t;
}

// Symmetric parametrix GEMV over the stored upper-triangle tiles (layout above):
// block (a, b) writes the row sums of tile a into partial slice b and, for a < b,
// the column sums of tile b into slice a (the four warps' values added in warp
// order), so every (slice, row) is written once, as by the symmetric sums.  A lane
// takes two steps k, k + 1 at a time in packed f32x2 arithmetic: its row sum as two
// chains (even and odd steps), and two column sums, for columns (l + k) and
// (l + k + 1) mod 32, that rotate by two lanes per double step; after the 32 steps of
// a sub-tile lane l holds column l's even chain and column l + 1's odd chain.  The
// strengths of a sub-tile's 32 columns sit twice in a row in shared memory (and once
// more shifted by one), so that the pair of a double step is one aligned 8-byte load.
// Each warp streams its four 32-column sub-tiles (4 KB of floats and 2 KB of codes each,
// contiguous in the layout) through a two-stage shared-memory ring filled by bulk copies
// (TMA), so the loads of the next sub-tile are in flight while one is consumed; lane 0
// issues them, every wait is bounded (2 s, then *err = PM_DEV_TIMEOUT and the warp stops).
constexpr int kChunkHi = 8 * 32 * 16;               // floats of one (warp, sub-tile): 4 KB
constexpr int kChunkQ = 8 * 32 * 8;                 // codes: 2 KB
constexpr int kStageBytes = kChunkHi + kChunkQ;
constexpr int kSymDynSmem = 4 * 2 * kStageBytes;    // 4 warps x 2 stages = 48 KB

__global__ void __launch_bounds__(kST, 4)
k_ffmat_symK_gemv(const unsigned char* __restrict__ T, const float2* __restrict__ sv, int N,
                  int nt, float2* __restrict__ partial, const int* __restrict__ skip,
                  int* __restrict__ err) {
    if (skip && *skip) return;
    extern __shared__ __align__(128) unsigned char ring[];
    __shared__ __align__(8) unsigned long long bars[8];     // [warp][stage]
    // Dh[c][i] = hi of column c 32 + (i mod 32); Ph[c][i] = Dh[c][i + 1] (likewise lo)
    __shared__ __align__(16) float Dh[4][64], Dl[4][64], Ph[4][64], Pl[4][64];
    int a, b;
    pm_tile_pair(blockIdx.x, nt, a, b);
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int i = a * kST + tid, j = b * kST + tid;
    const unsigned char* tile = T + (size_t)blockIdx.x * kTileBytes;
    const unsigned char* gh = tile + (size_t)w * 4 * kChunkHi;               // warp's floats
    const unsigned char* gq = tile + kTileHiBytes + (size_t)w * 4 * kChunkQ; // warp's codes
    unsigned char* wring = ring + w * 2 * kStageBytes;
    const uint32_t bar0 = smem_u32(&bars[2 * w]), bar1 = smem_u32(&bars[2 * w + 1]);
    int issued[2] = {1, 1}, waited[2] = {0, 0};       // copy phases per stage (warp-uniform)
    if (lane == 0) {
        bar_init(bar0);
        bar_init(bar1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int c = 0; c < 2; ++c) {
            const uint32_t bar = c ? bar1 : bar0;
            bar_expect(bar, kStageBytes);
            bulk_load(smem_u32(wring + c * kStageBytes), gh + c * kChunkHi, kChunkHi, bar);
            bulk_load(smem_u32(wring + c * kStageBytes + kChunkHi), gq + c * kChunkQ, kChunkQ, bar);
        }
    }
    {
        const float2 sj = j < N ? sv[j] : make_float2(0.f, 0.f);   // column tid = 32 w + lane
        const int pm = (lane + 31) & 31;
        Dh[w][lane] = Dh[w][lane + 32] = sj.x;
        Dl[w][lane] = Dl[w][lane + 32] = sj.y;
        Ph[w][pm] = Ph[w][pm + 32] = sj.x;
        Pl[w][pm] = Pl[w][pm + 32] = sj.y;
    }
    const float2 si = i < N ? sv[i] : make_float2(0.f, 0.f);
    __syncthreads();
    const bool diag = (a == b);
    bool ok = true;
    const int nxt2 = (lane + 2) & 31, prv = (lane + 31) & 31;
    const bool odd = lane & 1;
    const float2 SIH = make_float2(si.x, si.x), SIL = make_float2(si.y, si.y);
    const float2 CSC = make_float2(kCodeScale, kCodeScale), CBI = make_float2(kCodeBias, kCodeBias);
    float2 RS = make_float2(0.f, 0.f), RE = make_float2(0.f, 0.f);
    float cS[4], cE[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const float2* ph = reinterpret_cast<const float2*>(odd ? &Ph[c][lane - 1] : &Dh[c][lane]);
        const float2* pl = reinterpret_cast<const float2*>(odd ? &Pl[c][lane - 1] : &Dl[c][lane]);
        float2 CS = make_float2(0.f, 0.f), CE = make_float2(0.f, 0.f);
        const int stage = c & 1;
        if (ok) {
            ok = bar_wait(stage ? bar1 : bar0, c >> 1, err);
            ok = __all_sync(0xffffffffu, ok);
            if (ok) ++waited[stage];
        }
        const float4* th = reinterpret_cast<const float4*>(wring + stage * kStageBytes) + lane;
        const uint2* tq = reinterpret_cast<const uint2*>(wring + stage * kStageBytes + kChunkHi) + lane;
#pragma unroll 4
        for (int kq = 0; kq < 8 && ok; ++kq) {
            const int o = kq * 32;
            const float4 h4 = th[o];
            const uint2 w2 = tq[o];
            const float2 H0 = make_float2(h4.x, h4.y), H1 = make_float2(h4.z, h4.w);
            const float2 F0 = make_float2(code_float<false>(w2.x), code_float<true>(w2.x));
            const float2 F1 = make_float2(code_float<false>(w2.y), code_float<true>(w2.y));
            const float2 L0 = __fmul2_rn(__ffma2_rn(F0, CSC, CBI), H0);
            const float2 L1 = __fmul2_rn(__ffma2_rn(F1, CSC, CBI), H1);
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const float2 H = half ? H1 : H0, L = half ? L1 : L0;
                const int d = 2 * kq + half;
                ff_mac2(RS, RE, H, L, ph[d], pl[d]);
                if (!diag) {
                    ff_mac2(CS, CE, H, L, SIH, SIL);
                    CS.x = __shfl_sync(0xffffffffu, CS.x, nxt2);
                    CS.y = __shfl_sync(0xffffffffu, CS.y, nxt2);
                    CE.x = __shfl_sync(0xffffffffu, CE.x, nxt2);
                    CE.y = __shfl_sync(0xffffffffu, CE.y, nxt2);
                }
            }
        }
        // the stage is consumed: refill it with sub-tile c + 2
        __syncwarp();
        if (ok && c + 2 < 4) {
            if (lane == 0) {
                const uint32_t bar = stage ? bar1 : bar0;
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                bar_expect(bar, kStageBytes);
                bulk_load(smem_u32(wring + stage * kStageBytes), gh + (c + 2) * kChunkHi, kChunkHi,
                          bar);
                bulk_load(smem_u32(wring + stage * kStageBytes + kChunkHi), gq + (c + 2) * kChunkQ,
                          kChunkQ, bar);
            }
            ++issued[stage];
        }
        // column lane: its even chain here, its odd chain on the previous lane
        float s = CS.x, e = CE.x;
        ff_join(s, e, __shfl_sync(0xffffffffu, CS.y, prv), __shfl_sync(0xffffffffu, CE.y, prv));
        cS[c] = s;
        cE[c] = e;
    }
    if (!ok) {
        // a copy did not arrive in time (*err is set; the results are not valid): wait
        // once more, bounded, for the copies still in flight into this warp's ring
        // before the ring is reused or the block's shared memory released
        for (int st2 = 0; st2 < 2; ++st2)
            for (int ph = waited[st2]; ph < issued[st2]; ++ph)
                if (!bar_wait(st2 ? bar1 : bar0, ph & 1, err)) break;
    }
    if (ok && i < N) {
        float s = RS.x, e = RE.x;
        ff_join(s, e, RS.y, RE.y);
        const ff v = ff_norm(ff{s, e});
        partial[(size_t)b * N + i] = make_float2(v.h, v.l);
    }
    if (diag) return;                              // block-uniform
    // the column sums of the four warps, in the ring once every warp is done with it
    __syncthreads();
    float2 (*csh)[kST] = reinterpret_cast<float2 (*)[kST]>(ring);
#pragma unroll
    for (int c = 0; c < 4; ++c) csh[w][c * 32 + lane] = make_float2(cS[c], cE[c]);
    __syncthreads();
    if (j < N) {
        float t = csh[0][tid].x, e = csh[0][tid].y;
#pragma unroll
        for (int q = 1; q < 4; ++q) ff_join(t, e, csh[q][tid].x, csh[q][tid].y);
        const ff v = ff_norm(ff{t, e});
        partial[(size_t)a * N + j] = make_float2(v.h, v.l);
    }
}

// Column segments of the row-layout GEMV: about four waves of blocks, at most the
// surface's partial slices, segments a multiple of 128 columns.
void gemv_shape(const pm_surface* s, int* nseg, int* cs) {
    const int rowblocks = pm_ceil_div(s->N, kGemvRows);
    const int want = 16 * s->ctx->num_sms;
    const int ld = (int)s->ffm_ld;
    int S = std::max(1, std::min(pm_ceil_div(want, rowblocks), std::min(s->max_split, ld / kLd)));
    int c = pm_ceil_div(pm_ceil_div(ld, S), kLd) * kLd;
    *cs = c;
    *nseg = pm_ceil_div(ld, c);
}

// planes of a row-layout matrix: the floats, then the codes
float* plane_h(unsigned char* M) { return reinterpret_cast<float*>(M); }
unsigned short* plane_q(unsigned char* M, const pm_surface* s) {
    return reinterpret_cast<unsigned short*>(M + (size_t)s->N * s->ffm_ld * sizeof(float));
}

pm_status build_one(pm_surface* s, int which_K, cudaStream_t st) {
    unsigned char* M = which_K ? s->ffm_K : s->ffm_R;
    const int ld = (int)s->ffm_ld;
    if (which_K && s->ffm_symK) {
        const int nt = s->ffm_symK;
        k_ffmat_symK_build<<<nt * (nt + 1) / 2, kST, 0, st>>>(s->src_kg, s->log_tab, s->N, nt, M);
        PM_CUDA_TRY(cudaGetLastError());
        return PM_OK;
    }
    const int blocks = pm_ceil_div(s->N, kBuildRows);
    if (which_K)
        k_ffmat_build<true><<<blocks, kBuildRows * 32, 0, st>>>(s->src_kg, s->tgt_ff, s->log_tab,
                                                                s->N, ld, plane_h(M), plane_q(M, s));
    else
        k_ffmat_build<false><<<blocks, kBuildRows * 32, 0, st>>>(s->src_ff, s->tgt_ff, s->log_tab,
                                                                 s->N, ld, plane_h(M), plane_q(M, s));
    PM_CUDA_TRY(cudaGetLastError());
    return PM_OK;
}

long long row_ld(int N) { return (long long)pm_ceil_div(N, kLd) * kLd; }

// bytes of the stored parametrix matrix: the symmetric tile layout when the surface
// uses the symmetric sums, else the row layout
size_t k_bytes(const pm_surface* s, int* nt_sym) {
    const int nt = pm_sym_tiles(s);
    *nt_sym = nt;
    if (nt > 0) return (size_t)nt * (nt + 1) / 2 * kTileBytes;
    return (size_t)s->N * (size_t)row_ld(s->N) * 6;
}

}  // namespace

size_t pm_ffmat_bytes(const pm_surface* s, int which) {
    const size_t ld = (size_t)row_ld(s->N);
    int nt = 0;
    size_t b = ld * sizeof(float2);
    if (which & 1) b += (size_t)s->N * ld * 6;
    if (which & 2) b += k_bytes(s, &nt);
    return b;
}

void pm_ffmat_free(pm_surface* s) {
    pm_dfree(s->ffm_R);
    pm_dfree(s->ffm_K);
    pm_dfree(s->ffm_s);
    pm_dfree(s->ffm_err);
    s->ffm_ld = 0;
    s->ffm_symK = 0;
}

bool pm_ffmat_has(const pm_surface* s, int which_K) {
    return which_K ? s->ffm_K != nullptr : s->ffm_R != nullptr;
}

// Re-evaluates the stored remainder matrix after a coefficient change (the
// packed float-float targets hold the new n' and m).
pm_status pm_ffmat_refresh(pm_surface* s, cudaStream_t st) {
    if (s->ffm_R) PM_TRY(build_one(s, 0, st));
    return PM_OK;
}

pm_status pm_ffmat_prep(pm_surface* s, const double* sigma, cudaStream_t st) {
    k_ffmat_prep<<<pm_ceil_div(s->N, 256), 256, 0, st>>>(sigma, s->wa, s->ffm_s, s->N,
                                                         s->skip_flag);
    PM_CUDA_TRY(cudaGetLastError());
    return PM_OK;
}

pm_status pm_ffmat_apply(pm_surface* s, int which_K, int* nsplit, cudaStream_t st) {
    if (which_K && s->ffm_symK) {
        const int nt = s->ffm_symK;
        // the dynamic shared-memory limit was raised on this device by pm_surface_store_ff
        k_ffmat_symK_gemv<<<nt * (nt + 1) / 2, kST, kSymDynSmem, st>>>(
            s->ffm_K, s->ffm_s, s->N, nt, reinterpret_cast<float2*>(s->partial), s->skip_flag,
            s->ffm_err);
        PM_CUDA_TRY(cudaGetLastError());
        *nsplit = nt;
        return PM_OK;
    }
    int nseg = 0, cs = 0;
    gemv_shape(s, &nseg, &cs);
    unsigned char* M = which_K ? s->ffm_K : s->ffm_R;
    dim3 grid(pm_ceil_div(s->N, kGemvRows), nseg);
    k_ffmat_gemv<<<grid, kGemvWarps * 32, 0, st>>>(
        reinterpret_cast<const float4*>(plane_h(M)), reinterpret_cast<const uint2*>(plane_q(M, s)),
        s->ffm_ld / 4, reinterpret_cast<const float4*>(s->ffm_s), s->N, cs, (int)s->ffm_ld,
        reinterpret_cast<float2*>(s->partial), s->skip_flag);
    PM_CUDA_TRY(cudaGetLastError());
    *nsplit = nseg;
    return PM_OK;
}

extern "C" pm_status pm_surface_store_ff(pm_surface* s, int which) {
    if (!s || which < 0 || which > 3) {
        pm_set_error("pm_surface_store_ff: NULL surface or which outside 0..3");
        return PM_ERR_INVALID_ARG;
    }
    PM_CUDA_TRY(cudaSetDevice(s->ctx->device));
    PM_CUDA_TRY(cudaDeviceSynchronize());
    if (which == 0) {
        pm_ffmat_free(s);
        s->graph_epoch++;
        return PM_OK;
    }
    if (!s->has_coeff) {
        pm_set_error("pm_surface_store_ff: call pm_surface_set_coeff first");
        return PM_ERR_NO_COEFF;
    }
    if (s->has_c) {
        pm_set_error("pm_surface_store_ff: the surface has c != 0 (its sums are complex float64)");
        return PM_ERR_INVALID_ARG;
    }
    pm_ffmat_free(s);
    s->graph_epoch++;
    const size_t need = pm_ffmat_bytes(s, which);
    const size_t fr = pm_free_hbm_bytes();
    size_t total = 0, fr_real = 0;
    cudaMemGetInfo(&fr_real, &total);
    const size_t margin = std::max<size_t>(1ull << 30, total / 50);
    if (need + margin > fr) {
        pm_set_error("pm_surface_store_ff: %.2f GB needed, %.2f GB free (less a %.2f GB margin)",
                     need / 1e9, fr / 1e9, margin / 1e9);
        return PM_ERR_OOM;
    }
    s->ffm_ld = row_ld(s->N);
    int nt_sym = 0;
    const size_t bytesK = k_bytes(s, &nt_sym);
    pm_status st = pm_dmalloc(&s->ffm_s, (size_t)s->ffm_ld);
    if (st == PM_OK && (which & 1)) st = pm_dmalloc(&s->ffm_R, (size_t)s->N * s->ffm_ld * 6);
    if (st == PM_OK && (which & 2)) {
        st = pm_dmalloc(&s->ffm_K, bytesK);
        s->ffm_symK = nt_sym;
    }
    // the symmetric GEMV's shared-memory ring is above the default 48 KB: raise the
    // function's limit on this device (set here, outside any stream capture)
    if (st == PM_OK && s->ffm_symK &&
        cudaFuncSetAttribute(k_ffmat_symK_gemv, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kSymDynSmem) != cudaSuccess) {
        pm_set_error("pm_surface_store_ff: cudaFuncSetAttribute failed");
        st = PM_ERR_CUDA;
    }
    if (st == PM_OK) st = pm_dmalloc(&s->ffm_err, 1);
    if (st == PM_OK && cudaMemset(s->ffm_err, 0, sizeof(int)) != cudaSuccess) {
        pm_set_error("pm_surface_store_ff: cudaMemset failed");
        st = PM_ERR_CUDA;
    }
    if (st == PM_OK && cudaMemset(s->ffm_s, 0, sizeof(float2) * s->ffm_ld) != cudaSuccess) {
        pm_set_error("pm_surface_store_ff: cudaMemset failed");
        st = PM_ERR_CUDA;
    }
    if (st == PM_OK && s->ffm_R) st = build_one(s, 0, 0);
    if (st == PM_OK && s->ffm_K) st = build_one(s, 1, 0);
    if (st == PM_OK) {
        const cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) {
            pm_set_error("pm_surface_store_ff: %s", cudaGetErrorString(e));
            st = PM_ERR_CUDA;
        }
    }
    if (st != PM_OK) pm_ffmat_free(s);
    return st;
}

extern "C" int pm_surface_stored_ff(const pm_surface* s) {
    if (!s) return 0;
    return (s->ffm_R ? 1 : 0) | (s->ffm_K ? 2 : 0);
}
