"""The allocation-free product (copse_poly_mul_noalloc) against the pooled one
(copse_poly_mul), through the C ABI.

Callers that cannot allocate device memory when they need a product -- serving
loops that forbid allocation after start-up, or programs whose GPU memory is
already reserved by another allocator -- use the allocation-free entry point,
whose scratch is a fixed device array shared by all calls.  Two calls in a
row with different inputs check that nothing left in that array from one call
leaks into the next.  Results are exact residues, so they must be equal."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
K = pytest.importorskip("paper_2104_09583_gb300.copse")

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _rand_res(rng, primes, N):
    return np.stack([rng.integers(0, q, size=N, dtype=np.uint64) for q in primes])


@pytest.mark.parametrize("log_n,bits,n_primes,n_res", [(10, 50, 8, 8), (14, 55, 16, 16)])
def test_noalloc_product_equals_pooled_product(log_n, bits, n_primes, n_res):
    ctx = K.copse_ctx_create(log_n, bits, n_primes, 3)
    try:
        primes = K.copse_ctx_primes(ctx)[:n_res]
        N = 1 << log_n
        rng = np.random.default_rng(log_n)
        for call in range(2):
            a = torch.from_numpy(_rand_res(rng, primes, N).view(np.int64)).cuda()
            b = torch.from_numpy(_rand_res(rng, primes, N).view(np.int64)).cuda()
            want = torch.empty_like(a)
            got = torch.full_like(a, -1)
            K.copse_poly_mul(ctx, a.data_ptr(), b.data_ptr(), want.data_ptr(), n_res)
            K.copse_poly_mul_noalloc(ctx, a.data_ptr(), b.data_ptr(), got.data_ptr(), n_res)
            torch.cuda.synchronize()
            assert torch.equal(got, want), f"call {call}: allocation-free product differs"
    finally:
        K.copse_ctx_destroy(ctx)


def test_noalloc_rejects_sizes_above_its_scratch():
    ctx = K.copse_ctx_create(14, 55, 17, 3)
    try:
        a = torch.zeros(17 << 14, dtype=torch.int64, device="cuda")
        with pytest.raises(K.CopseError) as e:
            K.copse_poly_mul_noalloc(ctx, a.data_ptr(), a.data_ptr(), a.data_ptr(), 17)
        assert e.value.name == "EINVAL" and "scratch" in str(e.value)
    finally:
        K.copse_ctx_destroy(ctx)
