// Tensor-core GEMM for sm_103a: tcgen05.mma with the accumulator in tensor
// memory (TMEM), operand tiles staged in shared memory by TMA, one persistent
// CTA per SM.  It serves the FMM's M2L (Sec. 6.2: the far-field apply is one
// dense operator product per offset class), where
//
//   C[col * ldc + crow0 + r] = sum_k A[arow0 + r][k] * B[bcol0 + j][k],   r < 128, j < ncols
//
// for every tile (arow0, bcol0, ncols, crow0) of a host-built list.  A and B
// are 16-bit (float16 or bfloat16, both the same type), K-major (each row's K
// values contiguous); C is float32.
//
// Per CTA (192 threads, one CTA per SM):
//   warp 0      TMA producer: for each tile and 64-wide K block, one 128 x 64 tile
//               of A and one 256 x 64 tile of B into a 4-stage ring (48 KB a stage,
//               128-byte swizzle), completion signalled on the stage's "full" mbarrier;
//   warp 1      allocates 512 TMEM columns (two 128 x 256 float32 accumulators) and
//               one lane issues the MMAs: 4 x (M=128, N<=256, K=16) per K block,
//               tcgen05.commit frees the stage ("empty") and, after the last K
//               block, hands the accumulator to the epilogue ("tmem full");
//   warps 2..5  epilogue: tcgen05.ld of 32 columns at a time (each warp reads the
//               32 TMEM lanes of its quarter, warp % 4), float32 stores of the
//               tile's valid columns (a warp writes 128 contiguous bytes per
//               column), then release the accumulator ("tmem empty").
// The two accumulators let the epilogue of one tile overlap the MMAs of the next.
//
// Every wait is bounded: after kWaitNs the waiting thread records
// PM_DEV_TIMEOUT in the error word, raises a CTA-wide abort flag that ends the
// other roles' waits, and all roles leave their loops.  Before the CTA exits the
// producer waits (bounded) for its copies in flight, the MMA lane waits for its
// MMAs to finish, and warp 1 frees the TMEM.
#include "pm_internal.cuh"

#include <cuda.h>

#include <algorithm>
#include <cstring>

namespace {

constexpr int kM = 128, kN = 256, kBK = 64;  // tile M x N, K block (64 x 2 B = one 128-byte swizzle row)
constexpr int kStages = 4;
constexpr int kThreads = 192;
constexpr int kStageA = kM * kBK * 2;      // 16 KB
constexpr int kStageB = kN * kBK * 2;      // 32 KB
constexpr int kTmemCols = 2 * kN;          // two accumulators
constexpr int kBarBytes = 256;
constexpr int kSmemBytes = kStages * (kStageA + kStageB) + kBarBytes + 1024;  // + alignment slack
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s
static_assert(kSmemBytes <= 227 * 1024, "shared memory per CTA");

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long gtimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait until the phase of parity `parity` of the barrier has completed.  Gives
// up (false) when the CTA's abort flag is raised, or after kWaitNs, in which
// case it records the timeout and raises the flag itself.
__device__ __noinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag,
                                       int* err, bool honour_abort) {
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = gtimer();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 63) == 0) {
            if (honour_abort && *abort_flag) return false;
            if (gtimer() - t0 > kWaitNs) {
                *abort_flag = 1;
                atomicExch(err, PM_DEV_TIMEOUT);
                return false;
            }
        }
    }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, uint32_t bar,
                                            int c0, int c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(dst),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(bar), "r"(c0), "r"(c1)
        : "memory");
}

// Shared-memory matrix descriptor of a K-major tile written by TMA with the
// 128-byte swizzle: rows of 128 bytes, 8-row core groups 1024 bytes apart
// (stride byte offset), leading byte offset unused for this layout, descriptor
// version 1 (bits 46-48), swizzle mode 2 = 128 B (bits 61-63).
__device__ __forceinline__ unsigned long long sw128_desc(uint32_t saddr) {
    unsigned long long d = 0;
    d |= (unsigned long long)((saddr & 0x3FFFFu) >> 4);
    d |= (unsigned long long)1 << 16;
    d |= (unsigned long long)(1024 >> 4) << 32;
    d |= (unsigned long long)1 << 46;
    d |= (unsigned long long)2 << 61;
    return d;
}

// Instruction descriptor of kind::f16: float32 accumulator (bits 4-5 = 1), A and
// B format (bits 7-9, 10-12: 0 = float16, 1 = bfloat16), both K-major (bits 15,
// 16 = 0), N / 8 in bits 17-22, M / 16 in bits 24-28.
__device__ __forceinline__ uint32_t f16_idesc(int bf16, int n) {
    const uint32_t fmt = bf16 ? 1u : 0u;
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(kM >> 4) << 24);
}

__device__ __forceinline__ void umma_f16(uint32_t d_tmem, unsigned long long adesc,
                                         unsigned long long bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
        : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
        "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
        "%28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__global__ void __launch_bounds__(kThreads, 1)
k_tc_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
          const int4* __restrict__ tiles, int ntiles, int nkb, int bf16, float* __restrict__ C,
          long long ldc, int* __restrict__ err, const int* __restrict__ skip) {
    if (skip && *skip) return;
    extern __shared__ unsigned char smem_raw[];
    const uint32_t raw = smem_u32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;  // swizzled tiles need 1024-byte alignment
    const uint32_t sA0 = base;
    const uint32_t sB0 = base + kStages * kStageA;
    const uint32_t bars = sB0 + kStages * kStageB;
    unsigned char* bar_ptr = smem_raw + (bars - raw);
    // barrier layout: full[kStages], empty[kStages], tfull[2], tempty[2], done
    auto full = [&](int s) { return bars + 8u * s; };
    auto empty = [&](int s) { return bars + 8u * (kStages + s); };
    auto tfull = [&](int a) { return bars + 8u * (2 * kStages + a); };
    auto tempty = [&](int a) { return bars + 8u * (2 * kStages + 2 + a); };
    const uint32_t done = bars + 8u * (2 * kStages + 4);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar_ptr + 8 * (2 * kStages + 5));
    volatile int* abort_flag = reinterpret_cast<volatile int*>(bar_ptr + 8 * (2 * kStages + 5) + 4);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(full(s), 1);
            mbar_init(empty(s), 1);
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init(tfull(a), 1);
            mbar_init(tempty(a), 4);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile(
            "tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                smem_u32(tmem_slot)),
            "r"(kTmemCols)
            : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // ------------------------------------------------------------ TMA producer
        int stage = 0;
        uint32_t phase = 0, issued = 0, last_phase = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
            const int4 tl = tiles[t];
            bool ok = true;
            for (int kb = 0; kb < nkb; ++kb) {
                if (!mbar_wait(empty(stage), phase ^ 1u, abort_flag, err, true)) {
                    ok = false;
                    break;
                }
                mbar_expect_tx(full(stage), kStageA + kStageB);
                tma_load_2d(sA0 + stage * kStageA, &tmA, full(stage), kb * kBK, tl.x);
                tma_load_2d(sB0 + stage * kStageB, &tmB, full(stage), kb * kBK, tl.y);
                issued |= 1u << stage;
                last_phase = (last_phase & ~(1u << stage)) | (phase << stage);
                if (++stage == kStages) {
                    stage = 0;
                    phase ^= 1u;
                }
            }
            if (!ok) break;
        }
        // copies in flight must land before the CTA's shared memory goes away
        for (int s = 0; s < kStages; ++s)
            if (issued & (1u << s)) mbar_wait(full(s), (last_phase >> s) & 1u, abort_flag, err, false);
    } else if (warp == 1 && lane == 0) {
        // ------------------------------------------------------------ MMA issuer
        int stage = 0, it = 0;
        uint32_t phase = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
            const int4 tl = tiles[t];
            const int acc = it & 1;
            const uint32_t aph = (uint32_t)(it >> 1) & 1u;
            if (!mbar_wait(tempty(acc), aph ^ 1u, abort_flag, err, true)) break;
            tc_fence_after();
            const int n = (min(tl.z, kN) + 15) & ~15;
            const uint32_t idesc = f16_idesc(bf16, n);
            const uint32_t d = tmem + (uint32_t)(acc * kN);
            bool ok = true;
            for (int kb = 0; kb < nkb; ++kb) {
                if (!mbar_wait(full(stage), phase, abort_flag, err, true)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const unsigned long long ad = sw128_desc(sA0 + stage * kStageA);
                const unsigned long long bd = sw128_desc(sB0 + stage * kStageB);
#pragma unroll
                for (int k = 0; k < kBK / 16; ++k)  // 16 elements = 32 bytes along the swizzled row
                    umma_f16(d, ad + (unsigned long long)(2 * k), bd + (unsigned long long)(2 * k),
                             idesc, (kb | k) != 0);
                umma_commit(empty(stage));
                if (++stage == kStages) {
                    stage = 0;
                    phase ^= 1u;
                }
            }
            if (!ok) break;
            umma_commit(tfull(acc));
        }
        // every MMA of this thread must finish before the TMEM is freed
        umma_commit(done);
        mbar_wait(done, 0u, abort_flag, err, false);
    } else if (warp >= 2) {
        // ------------------------------------------------------------ epilogue
        const int q = warp & 3;  // TMEM lane quarter this warp may read
        int it = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
            const int4 tl = tiles[t];
            const int acc = it & 1;
            const uint32_t aph = (uint32_t)(it >> 1) & 1u;
            int ok = 1;
            if (lane == 0) ok = mbar_wait(tfull(acc), aph, abort_flag, err, true) ? 1 : 0;
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            tc_fence_after();
            const int nv = min(tl.z, kN);
            float* cp = C + (size_t)tl.y * (size_t)ldc + (size_t)(tl.w + q * 32 + lane);
            for (int c0 = 0; c0 < nv; c0 += 32) {
                uint32_t r[32];
                tmem_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(acc * kN + c0), r);
                const int m = min(32, nv - c0);
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (j < m) cp[(size_t)(c0 + j) * (size_t)ldc] = __uint_as_float(r[j]);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(tempty(acc));
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(kTmemCols)
                     : "memory");
    }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

pm_status encode_fn(EncodeTiledFn* out) {
    static EncodeTiledFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    if (!fn) {
        pm_set_error("tensor-core GEMM: cuTensorMapEncodeTiled is not available from the driver");
        return PM_ERR_CUDA;
    }
    *out = fn;
    return PM_OK;
}

// 2-D K-major tensor map of rows x K 16-bit values, box (64, box_rows), 128-byte swizzle
pm_status make_map(CUtensorMap* map, const void* ptr, long long rows, int K, int box_rows,
                   int bf16) {
    EncodeTiledFn fn = nullptr;
    PM_TRY(encode_fn(&fn));
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)K * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r =
        fn(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2,
           const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
        pm_set_error("tensor-core GEMM: cuTensorMapEncodeTiled failed (%d)", (int)r);
        return PM_ERR_CUDA;
    }
    return PM_OK;
}

}  // namespace

static_assert(sizeof(CUtensorMap) == sizeof(PmTcGemm::mapA), "tensor map storage");

pm_status pm_tcgemm_init(PmTcGemm* g, const void* A, long long a_rows, const void* B,
                         long long b_rows, int K, int bf16, const std::vector<int>& tiles,
                         float* C, long long ldc, long long c_cols) {
    pm_tcgemm_free(g);
    if (!A || !B || !C || K <= 0 || K % kBK != 0 || a_rows <= 0 || b_rows <= 0 ||
        tiles.size() % 4 != 0 || ldc <= 0) {
        pm_set_error("tensor-core GEMM: bad shape (K = %d must be a positive multiple of %d)", K,
                     kBK);
        return PM_ERR_INVALID_ARG;
    }
    if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) & 15u) {
        pm_set_error("tensor-core GEMM: operands must be 16-byte aligned");
        return PM_ERR_INVALID_ARG;
    }
    const int nt = (int)(tiles.size() / 4);
    // every tile must stay inside A (all 128 rows), start inside B, and write
    // inside C (rows crow0 .. crow0 + 127 < ldc, columns bcol0 .. bcol0 + ncols - 1 < c_cols)
    for (int t = 0; t < nt; ++t) {
        const long long ar = tiles[4 * t], bc = tiles[4 * t + 1], nc = tiles[4 * t + 2],
                        cr = tiles[4 * t + 3];
        if (ar < 0 || ar + kM > a_rows || bc < 0 || bc >= b_rows || nc <= 0 || nc > kN ||
            bc + nc > c_cols || cr < 0 || cr + kM > ldc) {
            pm_set_error("tensor-core GEMM: tile %d (%lld, %lld, %lld, %lld) out of range", t, ar,
                         bc, nc, cr);
            return PM_ERR_INVALID_ARG;
        }
    }
    PM_TRY(make_map(reinterpret_cast<CUtensorMap*>(g->mapA), A, a_rows, K, kM, bf16));
    PM_TRY(make_map(reinterpret_cast<CUtensorMap*>(g->mapB), B, b_rows, K, kN, bf16));
    if (nt > 0) {
        PM_TRY(pm_dmalloc(&g->tiles, tiles.size()));
        PM_CUDA_TRY(cudaMemcpy(g->tiles, tiles.data(), tiles.size() * sizeof(int),
                               cudaMemcpyHostToDevice));
    }
    PM_TRY(pm_dmalloc(&g->err, 1));
    PM_CUDA_TRY(cudaMemset(g->err, 0, sizeof(int)));
    // the shared-memory limit of the kernel, on the current device (always the same
    // value, so that setting it again never lowers it under another thread's launch)
    PM_CUDA_TRY(cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     kSmemBytes));
    g->ntiles = nt;
    g->nkb = K / kBK;
    g->bf16 = bf16;
    g->C = C;
    g->ldc = ldc;
    return PM_OK;
}

pm_status pm_tcgemm_run(const PmTcGemm* g, int num_sms, const int* skip, cudaStream_t st,
                        int prio) {
    if (g->ntiles == 0) return PM_OK;
    const int grid = std::max(1, std::min(g->ntiles, num_sms));
    const CUtensorMap mA = *reinterpret_cast<const CUtensorMap*>(g->mapA);
    const CUtensorMap mB = *reinterpret_cast<const CUtensorMap*>(g->mapB);
    PM_CUDA_TRY(pm_launch_prio(k_tc_gemm, dim3(grid), dim3(kThreads), kSmemBytes, st, prio, mA,
                               mB, reinterpret_cast<const int4*>(g->tiles), g->ntiles, g->nkb,
                               g->bf16, g->C, (long long)g->ldc, g->err, skip));
    return PM_OK;
}

pm_status pm_tcgemm_check(const PmTcGemm* g) {
    if (!g->err) return PM_OK;
    int h = 0;
    PM_CUDA_TRY(cudaMemcpy(&h, g->err, sizeof(int), cudaMemcpyDeviceToHost));
    if (h != 0) {
        pm_set_error("tensor-core GEMM: a bounded wait ran out (device code %d)", h);
        return PM_ERR_TIMEOUT;
    }
    return PM_OK;
}

void pm_tcgemm_free(PmTcGemm* g) {
    pm_dfree(g->tiles);
    pm_dfree(g->err);
    g->ntiles = 0;
}

// C = A B^T on caller's host arrays (float16 or bfloat16 bits), the tiles of
// one plain product: rows a multiple of 128, K a multiple of 64, any ncols.
// reps > 0: the product is then run reps more times and *ms receives the mean
// device time of one launch (CUDA events).
extern "C" pm_status pm_selftest_tc_gemm(pm_ctx* ctx, const unsigned short* A,
                                         const unsigned short* B, float* C, int rows, int K,
                                         int ncols, int bf16, int reps, double* ms) {
    if (reps > 0 && !ms) {
        pm_set_error("pm_selftest_tc_gemm: reps > 0 needs ms");
        return PM_ERR_INVALID_ARG;
    }
    if (!ctx || !A || !B || !C || rows <= 0 || rows % kM != 0 || K <= 0 || K % kBK != 0 ||
        ncols <= 0) {
        pm_set_error("pm_selftest_tc_gemm: rows must be a positive multiple of %d, K of %d", kM,
                     kBK);
        return PM_ERR_INVALID_ARG;
    }
    PM_CUDA_TRY(cudaSetDevice(ctx->device));
    std::vector<int> tiles;
    for (int n0 = 0; n0 < ncols; n0 += kN)
        for (int m0 = 0; m0 < rows; m0 += kM) {
            tiles.push_back(m0);
            tiles.push_back(n0);
            tiles.push_back(std::min(kN, ncols - n0));
            tiles.push_back(m0);
        }
    unsigned short *dA = nullptr, *dB = nullptr;
    float* dC = nullptr;
    PmTcGemm g;
    pm_status st = pm_dmalloc(&dA, (size_t)rows * K);
    if (st == PM_OK) st = pm_dmalloc(&dB, (size_t)ncols * K);
    if (st == PM_OK) st = pm_dmalloc(&dC, (size_t)ncols * rows);
    cudaError_t ce = cudaSuccess;
    if (st == PM_OK) {
        ce = cudaMemcpy(dA, A, (size_t)rows * K * 2, cudaMemcpyHostToDevice);
        if (ce == cudaSuccess) ce = cudaMemcpy(dB, B, (size_t)ncols * K * 2, cudaMemcpyHostToDevice);
        if (ce == cudaSuccess) ce = cudaMemset(dC, 0, (size_t)ncols * rows * sizeof(float));
        if (ce != cudaSuccess) {
            pm_set_error("pm_selftest_tc_gemm: %s", cudaGetErrorString(ce));
            st = PM_ERR_CUDA;
        }
    }
    if (st == PM_OK) st = pm_tcgemm_init(&g, dA, rows, dB, ncols, K, bf16, tiles, dC, rows, ncols);
    if (st == PM_OK) st = pm_tcgemm_run(&g, ctx->num_sms, nullptr, nullptr);
    if (st == PM_OK) {
        ce = cudaDeviceSynchronize();
        if (ce != cudaSuccess) {
            pm_set_error("pm_selftest_tc_gemm: %s", cudaGetErrorString(ce));
            st = PM_ERR_CUDA;
        }
    }
    if (st == PM_OK) st = pm_tcgemm_check(&g);
    if (st == PM_OK && reps > 0) {
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        ce = cudaEventCreate(&e0);
        if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
        if (ce == cudaSuccess) ce = cudaEventRecord(e0, nullptr);
        for (int r = 0; r < reps && ce == cudaSuccess && st == PM_OK; ++r)
            st = pm_tcgemm_run(&g, ctx->num_sms, nullptr, nullptr);
        if (ce == cudaSuccess) ce = cudaEventRecord(e1, nullptr);
        if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
        float t = 0.f;
        if (ce == cudaSuccess) ce = cudaEventElapsedTime(&t, e0, e1);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (ce != cudaSuccess && st == PM_OK) {
            pm_set_error("pm_selftest_tc_gemm: %s", cudaGetErrorString(ce));
            st = PM_ERR_CUDA;
        }
        if (st == PM_OK) st = pm_tcgemm_check(&g);
        *ms = (double)t / reps;
    }
    if (st == PM_OK) {
        ce = cudaMemcpy(C, dC, (size_t)ncols * rows * sizeof(float), cudaMemcpyDeviceToHost);
        if (ce != cudaSuccess) {
            pm_set_error("pm_selftest_tc_gemm: %s", cudaGetErrorString(ce));
            st = PM_ERR_CUDA;
        }
    }
    pm_tcgemm_free(&g);
    pm_dfree(dA);
    pm_dfree(dB);
    pm_dfree(dC);
    return st;
}
