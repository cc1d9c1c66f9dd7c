"""The tensor-core building blocks (shared-memory descriptors, tcgen05 MMA
into tensor memory, mbarrier completion, tensor-memory loads) against a host
product: small-integer bfloat16 operands make every sum exact, so the check
is exact whatever the accumulation order."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def probes():
    from paper_1112_0065_gb300 import probes

    probes.load()
    return probes


def _bf16_bits(x):
    return (np.asarray(x, dtype=np.float32).view(np.uint32) >> 16).astype(np.uint16)


@pytest.mark.parametrize("n,k", [(16, 16), (32, 64), (64, 144), (64, 256), (256, 32), (48, 96)])
def test_tc_gemm_exact(probes, n, k):
    rng = np.random.default_rng(n * 1000 + k)
    a = rng.integers(-3, 4, size=(128, k)).astype(np.float32)
    b = rng.integers(-3, 4, size=(n, k)).astype(np.float32)
    d = probes.tc_gemm(_bf16_bits(a), _bf16_bits(b))
    np.testing.assert_array_equal(d, a @ b.T)


def test_tc_gemm_layout_is_not_symmetric(probes):
    """Distinct row / column patterns catch a transposed operand or swapped
    descriptor offsets."""
    k, n = 64, 32
    a = np.zeros((128, k), np.float32)
    b = np.zeros((n, k), np.float32)
    a[np.arange(128), np.arange(128) % k] = np.arange(128) % 7 + 1
    b[np.arange(n), (3 * np.arange(n)) % k] = 1
    d = probes.tc_gemm(_bf16_bits(a), _bf16_bits(b))
    np.testing.assert_array_equal(d, a @ b.T)


def test_packed_fma_matches_fmaf(probes):
    """Packed two-wide float FMAs round each half like fmaf (the fixed-order
    classifier relies on it)."""
    r = probes.fp_rates()
    assert r["ffma2_mismatches"] == 0
    assert r["ffma"] > 1.0 and r["ffma2"] > 1.0


def test_bounded_wait_gives_up_and_frees_tensor_memory(probes):
    """A tensor-core wait on an mbarrier phase that nothing completes gives up
    after its poll limit in every warp, the kernel frees its tensor memory and
    returns, and the GPU context stays usable (a following tensor-core GEMM
    is still exact)."""
    st, flags, msg = probes.wait_giveup(2000)
    assert st == -5 and flags == 0xF, (st, flags, msg)
    assert "gave up" in msg
    a = np.ones((128, 16), np.float32)
    b = np.ones((16, 16), np.float32)
    np.testing.assert_array_equal(probes.tc_gemm(_bf16_bits(a), _bf16_bits(b)), a @ b.T)
