"""The persistent work-list kernel (copse_worklist_run): chained elementwise
ciphertext operations in one resident launch equal the same operations done
one by one (additions and subtractions coefficient by coefficient, tensors
against the oracle's), and a list whose wait cannot end returns ETIMEOUT
after its limit while the context stays usable."""
import numpy as np
import pytest

from oracle import bgv as B

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
K = pytest.importorskip("paper_2104_09583_gb300.copse")

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

LOGN, BITS, L = 10, 50, 6


@pytest.fixture(scope="module")
def setup():
    ctx = K.copse_ctx_create(LOGN, BITS, L, 3)
    P = B.Params(logN=LOGN, L=L, bits=BITS, dnum=3)
    q = np.asarray(P.primes[:L], dtype=np.uint64)
    rng = np.random.default_rng(11)
    cts = np.stack([np.stack([rng.integers(0, q[r], size=P.N, dtype=np.uint64) for r in range(L)])[None].repeat(2, 0)
                    for _ in range(3)])
    cts[:, 1] = np.stack([np.stack([rng.integers(0, q[r], size=P.N, dtype=np.uint64) for r in range(L)])
                          for _ in range(3)])
    buf = K.copse_ctbuf_import(ctx, cts)
    yield ctx, P, q, cts, buf
    K.copse_ctbuf_destroy(buf)
    K.copse_ctx_destroy(ctx)


def test_chained_items_equal_separate_ops(setup):
    ctx, P, q, cts, buf = setup
    qq = q[None, :, None]
    a, b, c = (cts[i].astype(object) for i in range(3))
    # items 0..4: a + b, a - b, (a + b) + c, ((a + b) + c) - (a - b), tensor a x b
    items = [("add", 0, 1, -1), ("sub", 0, 1, -1), ("add", 3, 2, -1), ("sub", 5, 4, -1), ("tensor", 0, 1, -1)]
    out = K.copse_worklist_run(ctx, buf, items)
    try:
        got = [K.copse_ctbuf_export(ctx, out, i, P.N) for i in range(len(items))]
    finally:
        K.copse_ctbuf_destroy(out)
    ab = (a + b) % qq.astype(object)
    amb = (a - b) % qq.astype(object)
    abc = (ab + c) % qq.astype(object)
    want = [ab, amb, abc, (abc - amb) % qq.astype(object)]
    for i, w in enumerate(want):
        assert np.array_equal(got[i], np.asarray(w, dtype=np.uint64)), f"item {i}"
    assert np.array_equal(got[4], B.Bgv(P).tensor(cts[0], cts[1]))


def test_long_chain_over_many_tiles(setup):
    ctx, P, q, cts, buf = setup
    # 200 items: x_0 = a + b, x_i = x_{i-1} + c: the last is a + b + 199 c
    items = [("add", 0, 1, -1)] + [("add", 3 + i - 1, 2, -1) for i in range(1, 200)]
    out = K.copse_worklist_run(ctx, buf, items)
    try:
        last = K.copse_ctbuf_export(ctx, out, 199, P.N)
    finally:
        K.copse_ctbuf_destroy(out)
    qq = q[None, :, None].astype(object)
    want = (cts[0].astype(object) + cts[1].astype(object) + 199 * cts[2].astype(object)) % qq
    assert np.array_equal(last, np.asarray(want, dtype=np.uint64))


def test_wait_that_cannot_end_times_out(setup):
    ctx, P, q, cts, buf = setup
    # item 1 waits for itself: nothing ever completes it, so its wait runs into the limit
    with pytest.raises(K.CopseError) as e:
        K.copse_worklist_run(ctx, buf, [("add", 0, 1, -1), ("add", 0, 2, 1)], timeout_ms=200)
    assert e.value.name == "ETIMEOUT"
    # the context is still usable
    out = K.copse_worklist_run(ctx, buf, [("sub", 1, 1, -1)])
    try:
        assert not K.copse_ctbuf_export(ctx, out, 0, P.N).any()
    finally:
        K.copse_ctbuf_destroy(out)
