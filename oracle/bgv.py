"""Python face of the CPU oracle's BGV layer (``bgv_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; the product library never imports it.

The paper runs its vectorised primitives on BGV (Section 5, "COPSE Runtime";
the operation list of Section 6: Encrypt, Rotate, Add, Multiply, Constant
Add).  The concrete scheme -- ring, keys, hybrid key switching, modulus
switching -- is this oracle's canonical reading, stated in ``bgv_oracle.c``.
Ciphertexts are numpy ``uint64`` arrays of shape ``(ncomp, level, N)`` holding
coefficient residues in ``[0, q_i)``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bgv_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "libcopse_oracle.so")
MAXP = 64
T_DEFAULT = 65537

u64p = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle's C core with gcc (plain -O2, portable C11)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


class _Params(C.Structure):
    _fields_ = [
        ("logN", C.c_int32), ("N", C.c_int32), ("t", C.c_uint64),
        ("L", C.c_int32), ("alpha", C.c_int32), ("ndig", C.c_int32), ("pad", C.c_int32),
        ("primes", C.c_uint64 * MAXP),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        P = C.POINTER(_Params)
        sig = {
            "or_is_prime": (C.c_int, [C.c_uint64]),
            "or_threads": (C.c_int, []),
            "or_set_threads": (C.c_int, [C.c_int]),
            "or_find_primes": (C.c_int, [C.c_int, C.c_uint64, C.c_int, C.c_int, u64p]),
            "or_root_2n": (C.c_uint64, [C.c_uint64, C.c_int]),
            "or_mulmod": (C.c_uint64, [C.c_uint64, C.c_uint64, C.c_uint64]),
            "or_powmod": (C.c_uint64, [C.c_uint64, C.c_uint64, C.c_uint64]),
            "or_ntt_fwd": (None, [u64p, C.c_int, C.c_uint64, C.c_uint64]),
            "or_ntt_inv": (None, [u64p, C.c_int, C.c_uint64, C.c_uint64]),
            "or_eval_direct": (None, [u64p, C.c_int, C.c_uint64, C.c_uint64, u64p]),
            "or_negacyclic_schoolbook": (None, [u64p, u64p, C.c_int, C.c_uint64, u64p]),
            "or_negacyclic_mul": (None, [u64p, u64p, C.c_int, C.c_uint64, u64p]),
            "or_slot_exponents": (None, [C.c_int, u64p]),
            "or_encode": (None, [u64p, C.c_int, C.c_uint64, u64p]),
            "or_decode": (None, [u64p, C.c_int, C.c_uint64, u64p]),
            "or_word": (C.c_uint64, [C.c_uint64, C.c_uint64, C.c_uint64]),
            "or_sample_ternary": (None, [C.c_uint64, C.c_uint64, C.c_int, i64p]),
            "or_sample_cbd": (None, [C.c_uint64, C.c_uint64, C.c_int, i64p]),
            "or_automorphism": (None, [u64p, C.c_int, C.c_uint64, C.c_uint64, u64p]),
            "or_keygen_secret": (None, [P, C.c_uint64, i64p]),
            "or_keygen_public": (None, [P, C.c_uint64, i64p, u64p]),
            "or_keygen_switch": (None, [P, C.c_uint64, C.c_uint64, i64p, u64p, u64p]),
            "or_encrypt": (None, [P, u64p, i64p, C.c_uint64, C.c_uint64, u64p]),
            "or_decrypt_raw": (None, [P, i64p, u64p, C.c_int, u64p]),
            "or_decrypt": (None, [P, i64p, u64p, C.c_int, u64p]),
            "or_modswitch": (None, [P, u64p, C.c_int, C.c_int, u64p]),
            "or_keyswitch": (None, [P, u64p, C.c_int, u64p, u64p]),
            "or_tensor": (None, [P, u64p, u64p, C.c_int, u64p]),
            "or_relin": (None, [P, u64p, C.c_int, u64p, u64p]),
            "or_rotate": (None, [P, u64p, C.c_int, C.c_uint64, u64p, u64p]),
            "or_mul_plain": (None, [P, u64p, C.c_int, C.c_int, i64p, u64p]),
            "or_add_plain": (None, [P, u64p, C.c_int, i64p]),
            "or_add": (None, [P, u64p, u64p, C.c_int, C.c_int, C.c_int, u64p]),
            "or_matmul": (None, [P, u64p, C.c_int, C.c_int, u64p, C.POINTER(C.c_void_p), C.c_int, i64p,
                                 np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS"), u64p]),
            "or_rotsum": (None, [P, C.POINTER(C.c_void_p), C.c_int, C.c_int, u64p, C.POINTER(C.c_void_p), u64p]),
            "or_encrypt_sk": (None, [P, i64p, i64p, C.c_uint64, C.c_uint64, C.c_int, u64p]),
            "or_relin_drop": (None, [P, u64p, C.c_int, u64p, u64p]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def oracle_threads() -> int:
    """Threads the oracle's C loops use (OpenMP; OMP_NUM_THREADS, default all host cores)."""
    return int(lib().or_threads())


def set_oracle_threads(n: int) -> int:
    """Run the oracle's C loops on n threads from now on (results do not depend on it);
    returns the count in force."""
    return int(lib().or_set_threads(int(n)))


# ---------------------------------------------------------------------------
# Randomness streams (the counter-based SplitMix64 layout both sides follow).
# word(seed, stream, idx) is output number stream * 2^40 + idx + 1, so every
# stream id stays below 2^24 (the product never wraps past 2^64 and no two
# streams share words): secret 1, public key 2-3, relinearisation key from 16,
# rotation keys from 0x10000 (64 per odd Galois element, < 0x410000),
# encryptions from 0x500000, encrypted-model ciphertexts from 0x800000.
# ---------------------------------------------------------------------------
STREAM_SECRET = 1
STREAM_PK_A = 2
STREAM_PK_E = 3
STREAM_RELIN = 16


def stream_galois(g: int) -> int:
    """Stream base of the switching key for Galois element g."""
    return 0x10000 + 64 * g


def stream_encrypt(index: int) -> int:
    """Stream base (u, e0, e1) of the index-th encryption under one seed."""
    assert 0 <= index < 0x100000
    return 0x500000 + 3 * index


def stream_model(index: int) -> int:
    """Stream base (a, e) of the index-th secret-key encryption of an encrypted model."""
    assert 0 <= index < 0x400000
    return 0x800000 + 2 * index


# ---------------------------------------------------------------------------
# Parameters
# ---------------------------------------------------------------------------
@dataclass
class Params:
    """BGV parameters: ring degree 2^logN, plaintext modulus t, L ciphertext
    primes and alpha = ceil(L/dnum) special primes, all = 1 mod 2N*t and below
    2^bits, taken in decreasing order (ciphertext primes first)."""

    logN: int
    L: int
    bits: int
    dnum: int = 3
    t: int = T_DEFAULT
    primes: list = field(default_factory=list)

    def __post_init__(self):
        self.N = 1 << self.logN
        self.alpha = -(-self.L // self.dnum)
        self.ndig = -(-self.L // self.alpha)
        if not self.primes:
            out = np.zeros(self.L + self.alpha, dtype=np.uint64)
            got = lib().or_find_primes(self.logN, self.t, self.bits, self.L + self.alpha, out)
            if got != self.L + self.alpha:
                raise ValueError("not enough primes of this size")
            self.primes = [int(x) for x in out]
        self._c = _Params()
        self._c.logN, self._c.N, self._c.t = self.logN, self.N, self.t
        self._c.L, self._c.alpha, self._c.ndig = self.L, self.alpha, self.ndig
        for i, p in enumerate(self.primes):
            self._c.primes[i] = p

    @property
    def c(self):
        return C.byref(self._c)

    @property
    def q(self):
        return self.primes[: self.L]

    @property
    def special(self):
        return self.primes[self.L:]


def galois_rot(logN: int, k: int) -> int:
    """Galois element of a left rotation by k slots within each row: 3^k mod 2N."""
    return pow(3, k, 2 << logN)


# ---------------------------------------------------------------------------
# Plaintext encoding (slots mod t)
# ---------------------------------------------------------------------------
def encode(P: Params, slots) -> np.ndarray:
    """Slot vector (length N, values mod t) -> centred coefficients int64."""
    s = np.ascontiguousarray(np.asarray(slots, dtype=np.int64) % P.t, dtype=np.uint64)
    out = np.zeros(P.N, dtype=np.uint64)
    lib().or_encode(s, P.logN, P.t, out)
    c = out.astype(np.int64)
    c[c > (P.t - 1) // 2] -= P.t
    return c


def decode(P: Params, coeffs) -> np.ndarray:
    """Coefficients mod t -> slot vector (uint64 in [0,t))."""
    c = np.ascontiguousarray(np.asarray(coeffs, dtype=np.int64) % P.t, dtype=np.uint64)
    out = np.zeros(P.N, dtype=np.uint64)
    lib().or_decode(c, P.logN, P.t, out)
    return out


# ---------------------------------------------------------------------------
# Keys and ciphertext operations
# ---------------------------------------------------------------------------
def residues_of(P: Params, v: np.ndarray, gidx) -> np.ndarray:
    """Residues of an integer polynomial v for global prime indices gidx."""
    out = np.zeros((len(gidx), P.N), dtype=np.uint64)
    for r, g in enumerate(gidx):
        out[r] = (v.astype(object) % P.primes[g]).astype(np.uint64)
    return out


@dataclass
class Keys:
    sk: np.ndarray                 # ternary int64[N]
    pk: np.ndarray                 # [2][L][N]
    rlk: np.ndarray                # [ndig][2][L+alpha][N]
    gk: dict                       # Galois element -> [ndig][2][L+alpha][N]


class Bgv:
    def __init__(self, P: Params):
        self.P = P
        self.L = lib()

    # -- keys -------------------------------------------------------------
    def keygen(self, seed: int, galois=()) -> Keys:
        P = self.P
        s = np.zeros(P.N, dtype=np.int64)
        self.L.or_keygen_secret(P.c, seed, s)
        pk = np.zeros((2, P.L, P.N), dtype=np.uint64)
        self.L.or_keygen_public(P.c, seed, s, pk)
        allp = list(range(P.L + P.alpha))
        s_res = np.stack([(s % P.primes[g]).astype(np.uint64) for g in allp])
        s2 = np.zeros_like(s_res)
        for g in allp:
            self.L.or_negacyclic_mul(np.ascontiguousarray(s_res[g]), np.ascontiguousarray(s_res[g]),
                                     P.logN, P.primes[g], s2[g])
        rlk = self._switch_key(seed, STREAM_RELIN, s, s2)
        gk = {}
        for g in sorted(set(galois)):
            gk[g] = self.galois_key(seed, s, g)
        return Keys(s, pk, rlk, gk)

    def galois_key(self, seed: int, s: np.ndarray, g: int) -> np.ndarray:
        P = self.P
        allp = list(range(P.L + P.alpha))
        sg = np.zeros((len(allp), P.N), dtype=np.uint64)
        for gi in allp:
            sr = np.ascontiguousarray((s % P.primes[gi]).astype(np.uint64))
            self.L.or_automorphism(sr, P.logN, P.primes[gi], g, sg[gi])
        return self._switch_key(seed, stream_galois(g), s, sg)

    def _switch_key(self, seed, sb, s, s_from):
        P = self.P
        ksk = np.zeros((P.ndig, 2, P.L + P.alpha, P.N), dtype=np.uint64)
        self.L.or_keygen_switch(P.c, seed, sb, s, np.ascontiguousarray(s_from), ksk)
        return ksk

    # -- encryption -------------------------------------------------------
    def encrypt(self, pk, m_centred, seed: int, index: int) -> np.ndarray:
        P = self.P
        ct = np.zeros((2, P.L, P.N), dtype=np.uint64)
        self.L.or_encrypt(P.c, pk, np.ascontiguousarray(m_centred, dtype=np.int64), seed,
                          stream_encrypt(index), ct)
        return ct

    def encrypt_sk(self, sk, m_centred, seed: int, index: int, ell: int) -> np.ndarray:
        """Secret-key encryption at level ell with a seeded mask (see or_encrypt_sk)."""
        P = self.P
        ct = np.zeros((2, ell, P.N), dtype=np.uint64)
        self.L.or_encrypt_sk(P.c, np.ascontiguousarray(sk, dtype=np.int64),
                             np.ascontiguousarray(m_centred, dtype=np.int64), seed, stream_model(index), ell, ct)
        return ct

    def encrypt_slots(self, pk, slots, seed: int, index: int) -> np.ndarray:
        return self.encrypt(pk, encode(self.P, slots), seed, index)

    def decrypt(self, sk, ct) -> np.ndarray:
        """Plaintext coefficients in [0, t) (modswitch to level 1, then [c0+c1 s]_q0 mod t)."""
        ct = np.ascontiguousarray(ct)
        m = np.zeros(self.P.N, dtype=np.uint64)
        self.L.or_decrypt(self.P.c, sk, ct, ct.shape[1], m)
        return m

    def decrypt_slots(self, sk, ct) -> np.ndarray:
        return decode(self.P, self.decrypt(sk, ct))

    def decrypt_raw(self, sk, ct) -> np.ndarray:
        ct = np.ascontiguousarray(ct)
        x = np.zeros((ct.shape[1], self.P.N), dtype=np.uint64)
        self.L.or_decrypt_raw(self.P.c, sk, ct, ct.shape[1], x)
        return x

    def noise_bits(self, sk, ct) -> float:
        """log2 of the infinity norm of [c0 + c1*s]_Q (CRT over the ct's primes,
        exact integers), i.e. plaintext plus t*noise."""
        x = self.decrypt_raw(sk, ct)
        ell = ct.shape[1]
        qs = self.P.primes[:ell]
        Q = 1
        for q in qs:
            Q *= q
        acc = [0] * self.P.N
        for r, q in enumerate(qs):
            Qh = Q // q
            f = Qh * pow(Qh % q, -1, q)
            xr = x[r].tolist()
            for j in range(self.P.N):
                acc[j] += xr[j] * f
        mx = 0
        for j in range(self.P.N):
            v = acc[j] % Q
            if v > Q // 2:
                v = Q - v
            mx = max(mx, v)
        return float(np.log2(float(mx))) if mx else 0.0

    def budget_bits(self, sk, ct) -> float:
        """Remaining headroom: log2(q_0/2) - log2|[c0+c1 s]_Q| after the decryption-path modswitches."""
        cur = np.ascontiguousarray(ct)
        while cur.shape[1] > 1:
            cur = self.modswitch(cur)
        return float(np.log2(self.P.primes[0] / 2)) - self.noise_bits(sk, cur)

    # -- arithmetic -------------------------------------------------------
    def modswitch(self, ct) -> np.ndarray:
        ct = np.ascontiguousarray(ct)
        nc, ell, N = ct.shape
        out = np.zeros((nc, ell - 1, N), dtype=np.uint64)
        self.L.or_modswitch(self.P.c, ct, nc, ell, out)
        return out

    def to_level(self, ct, ell: int) -> np.ndarray:
        while ct.shape[1] > ell:
            ct = self.modswitch(ct)
        return ct

    def align(self, a, b):
        ell = min(a.shape[1], b.shape[1])
        return self.to_level(a, ell), self.to_level(b, ell)

    def add(self, a, b) -> np.ndarray:
        a, b = self.align(a, b)
        out = np.zeros_like(a)
        self.L.or_add(self.P.c, np.ascontiguousarray(a), np.ascontiguousarray(b), a.shape[0], a.shape[1], 0, out)
        return out

    def sub(self, a, b) -> np.ndarray:
        a, b = self.align(a, b)
        out = np.zeros_like(a)
        self.L.or_add(self.P.c, np.ascontiguousarray(a), np.ascontiguousarray(b), a.shape[0], a.shape[1], 1, out)
        return out

    def add_plain(self, ct, m_centred) -> np.ndarray:
        out = np.ascontiguousarray(ct).copy()
        self.L.or_add_plain(self.P.c, out, out.shape[1], np.ascontiguousarray(m_centred, dtype=np.int64))
        return out

    def mul_plain(self, ct, m_centred) -> np.ndarray:
        ct = np.ascontiguousarray(ct)
        out = np.zeros_like(ct)
        self.L.or_mul_plain(self.P.c, ct, ct.shape[0], ct.shape[1],
                            np.ascontiguousarray(m_centred, dtype=np.int64), out)
        return out

    def tensor(self, a, b) -> np.ndarray:
        a, b = self.align(a, b)
        out = np.zeros((3, a.shape[1], self.P.N), dtype=np.uint64)
        self.L.or_tensor(self.P.c, np.ascontiguousarray(a), np.ascontiguousarray(b), a.shape[1], out)
        return out

    def relin(self, ct3, rlk) -> np.ndarray:
        ell = ct3.shape[1]
        out = np.zeros((2, ell, self.P.N), dtype=np.uint64)
        self.L.or_relin(self.P.c, np.ascontiguousarray(ct3), ell, rlk, out)
        return out

    def keyswitch(self, x, ksk) -> np.ndarray:
        x = np.ascontiguousarray(x)
        ell = x.shape[0]
        out = np.zeros((2, ell, self.P.N), dtype=np.uint64)
        self.L.or_keyswitch(self.P.c, x, ell, ksk, out)
        return out

    def rotate(self, ct, g: int, gk) -> np.ndarray:
        ct = np.ascontiguousarray(ct)
        ell = ct.shape[1]
        out = np.zeros((2, ell, self.P.N), dtype=np.uint64)
        self.L.or_rotate(self.P.c, ct, ell, g, gk, out)
        return out

    def matmul(self, ct, galois, gks, pts) -> list:
        """Sums of plaintext-times-rotation products sharing the rotations of ct, with one
        modulus-down step per sum (see or_matmul).  galois[k]: Galois element of rotation k
        (1 = none), gks[k]: its key (None for 1); pts[a][k]: centred plaintext coefficients
        or None for a zero diagonal.  Returns one 2-component ciphertext per accumulator."""
        P = self.P
        ct = np.ascontiguousarray(ct)
        ell = ct.shape[1]
        nrot, nacc = len(galois), len(pts)
        g = np.ascontiguousarray(galois, dtype=np.uint64)
        keys = (C.c_void_p * max(nrot, 1))(*[None if k is None else k.ctypes.data for k in gks])
        m = np.zeros((nacc, nrot, P.N), dtype=np.int64)
        present = np.zeros(nacc * nrot, dtype=np.int32)
        for a in range(nacc):
            for k in range(nrot):
                if pts[a][k] is not None:
                    m[a, k] = pts[a][k]
                    present[a * nrot + k] = 1
        out = np.zeros((nacc, 2, ell, P.N), dtype=np.uint64)
        self.L.or_matmul(P.c, ct, ell, nrot, g, keys, nacc, m, present, out)
        return [out[a] for a in range(nacc)]

    def rotsum(self, cts, galois, gks) -> np.ndarray:
        """sum_k rot_{galois[k]}(cts[k]) with one modulus-down step for the sum (see
        or_rotsum); galois[k] = 1 adds cts[k] unrotated (gks[k] then None)."""
        P = self.P
        cts = [np.ascontiguousarray(c) for c in cts]
        ell = cts[0].shape[1]
        assert all(c.shape == (2, ell, P.N) for c in cts)
        n = len(cts)
        g = np.ascontiguousarray(galois, dtype=np.uint64)
        ptrs = (C.c_void_p * n)(*[c.ctypes.data for c in cts])
        keys = (C.c_void_p * n)(*[None if k is None else k.ctypes.data for k in gks])
        out = np.zeros((2, ell, P.N), dtype=np.uint64)
        self.L.or_rotsum(P.c, ptrs, ell, n, g, keys, out)
        return out

    def relin_drop(self, ct3, rlk) -> np.ndarray:
        """Relinearise and drop one prime in one ModDown over P q_{ell-1} (see or_relin_drop)."""
        ell = ct3.shape[1]
        out = np.zeros((2, ell - 1, self.P.N), dtype=np.uint64)
        self.L.or_relin_drop(self.P.c, np.ascontiguousarray(ct3), ell, rlk, out)
        return out

    def mul(self, a, b, rlk) -> np.ndarray:
        """ct x ct: tensor, then relinearise and drop one prime (the canonical policy) in one
        ModDown over P q_{ell-1}."""
        return self.relin_drop(self.tensor(a, b), rlk)
