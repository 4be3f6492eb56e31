"""The library's tcgen05 tensor-core GEMM (the product that carries the FMM's
M2L, Sec. 6.2) against float64 products of the same 16-bit operands.

Small-integer operands make every product and partial sum exact in float32, so
the GEMM must reproduce the integer product bit for bit: a wrong shared-memory
descriptor, swizzle, K step or TMEM lane mapping moves values between rows,
columns or K positions and fails that check.  Random operands then bound the
float32 accumulation error; the shapes cover ragged column tiles (MMA widths
that are not 256) and several row tiles."""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2401_12501_gb300 as pm
    c = pm.Context(0)
    yield c
    c.close()


def _bits(x, bf16):
    """16-bit patterns of x (round to nearest even) and their float64 values."""
    if bf16:
        u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
        r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)
        vals = (r.astype(np.uint32) << 16).view(np.float32).astype(np.float64)
        return r, vals
    h = np.asarray(x, dtype=np.float16)
    return h.view(np.uint16), h.astype(np.float64)


@pytest.mark.parametrize("rows,K,ncols,bf16", [
    (128, 64, 16, 0), (128, 64, 1, 0), (256, 128, 300, 0), (384, 192, 513, 1),
    (512, 1536, 257, 0), (4608, 1536, 700, 0)])
def test_tc_gemm_exact_on_integers(ctx, rows, K, ncols, bf16):
    rng = np.random.default_rng(rows * 7 + K * 3 + ncols)
    A, Av = _bits(rng.integers(-2, 3, (rows, K)).astype(np.float32), bf16)
    B, Bv = _bits(rng.integers(-2, 3, (ncols, K)).astype(np.float32), bf16)
    C, _ = ctx.selftest_tc_gemm(A, B, bf16=bf16)
    ref = Bv @ Av.T
    assert C.shape == (ncols, rows)
    assert np.array_equal(C.astype(np.float64), ref), np.argwhere(C != ref)[:8]


@pytest.mark.parametrize("rows,K,ncols,bf16", [(256, 1536, 300, 0), (512, 1536, 200, 1)])
def test_tc_gemm_float32_accumulation(ctx, rows, K, ncols, bf16):
    """Random operands: every product of two 16-bit values is exact in float32, so
    the only error is the float32 accumulation, at most K 2^-23 of sum |a||b| per
    entry even with truncating additions; the typical error is far smaller."""
    rng = np.random.default_rng(5 + bf16)
    A, Av = _bits(rng.standard_normal((rows, K)), bf16)
    B, Bv = _bits(rng.standard_normal((ncols, K)), bf16)
    C, _ = ctx.selftest_tc_gemm(A, B, bf16=bf16)
    ref = Bv @ Av.T
    bound = np.abs(Bv) @ np.abs(Av).T
    err = np.abs(C - ref)
    assert np.all(err <= K * 2.0 ** -23 * bound)
    assert np.linalg.norm(err) <= 1e-6 * np.linalg.norm(bound)


def test_tc_gemm_rejects_bad_shapes(ctx):
    import paper_2401_12501_gb300 as pm
    A = np.zeros((100, 64), np.uint16)
    B = np.zeros((8, 64), np.uint16)
    with pytest.raises(pm.PmError) as e:
        ctx.selftest_tc_gemm(A, B)
    assert e.value.status == 1
    with pytest.raises(pm.PmError):
        ctx.selftest_tc_gemm(np.zeros((128, 40), np.uint16), np.zeros((8, 40), np.uint16))


def test_tc_gemm_timing_repeats_give_same_product(ctx):
    """The timed repetitions run the same product (the result after them equals the
    first launch's, bit for bit) and report a positive time."""
    rng = np.random.default_rng(9)
    A, _ = _bits(rng.standard_normal((4608, 1536)), 0)
    B, _ = _bits(rng.standard_normal((712, 1536)), 0)
    C0, _ = ctx.selftest_tc_gemm(A, B)
    C1, ms = ctx.selftest_tc_gemm(A, B, reps=10)
    assert ms > 0
    assert np.array_equal(C0, C1)
    flops = 2.0 * 4608 * 1536 * 712
    print(f"tcgen05 GEMM 4608 x 712 x 1536 (float16): {ms * 1e3:.1f} us, "
          f"{flops / ms / 1e9:.0f} TFLOP/s")
