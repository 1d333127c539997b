"""The oracle's C loops run on several host threads (OpenMP), each thread computing
whole, independent residues or coefficients, so every result must be the same on
one thread as on all of them: keys, encryption, products, rotations, diagonal
products and key switching, bit for bit."""
import numpy as np

from oracle import bgv as B


def _run():
    logN, k = 8, 3
    g = B.galois_rot(logN, k)
    P = B.Params(logN=logN, L=6, bits=50, dnum=3)
    bgv = B.Bgv(P)
    keys = bgv.keygen(4242, [g])
    rng = np.random.default_rng(1)
    a = bgv.encrypt_slots(keys.pk, rng.integers(0, 2, P.N), 5, 0)
    b = bgv.encrypt_slots(keys.pk, rng.integers(0, 2, P.N), 5, 1)
    prod = bgv.mul(a, b, keys.rlk)
    rot = bgv.rotate(a, g, keys.gk[g])
    one = B.encode(P, np.ones(P.N, dtype=np.int64))
    (mm,) = bgv.matmul(a, [1, g], [None, keys.gk[g]], [[one, one]])
    drop = bgv.relin_drop(bgv.tensor(a, b), keys.rlk)
    return [keys.pk, keys.rlk, keys.gk[g], a, b, prod, rot, mm, drop]


def test_results_do_not_depend_on_the_thread_count():
    n = B.oracle_threads()
    try:
        B.set_oracle_threads(1)
        one = _run()
        B.set_oracle_threads(max(n, 4))
        many = _run()
    finally:
        B.set_oracle_threads(n)
    for x, y in zip(one, many):
        assert np.array_equal(x, y)
