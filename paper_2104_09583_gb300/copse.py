"""Thin Python binding of the C ABI in ``include/copse.h`` (ctypes).

Argument marshalling only: every step of the secure-inference path runs in
the CUDA library.  Functions keep the C names; handles are opaque
``ctypes.c_void_p`` values that the caller releases with the matching
``*_destroy``.  A nonzero status raises ``CopseError`` with the library's
message.  If the shared library has not been built the import fails loudly;
there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

from .build_lib import LIB as _LIB_PATH

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "copse.h")

if not os.path.exists(_LIB_PATH):
    raise ImportError(f"CUDA library {_LIB_PATH} is not built; run __graft_entry__.build()")

_lib = C.CDLL(_LIB_PATH)

STATUS = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "EPARSE", -4: "ECUDA", -5: "ENOKEY", -6: "ELEVEL", -7: "EFIT"}


class CopseError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code
        self.name = STATUS.get(code, str(code))


class copse_params(C.Structure):
    _fields_ = [("log_n", C.c_uint32), ("prime_bits", C.c_uint32), ("n_primes", C.c_uint32), ("dnum", C.c_uint32)]


class copse_model_info(C.Structure):
    _fields_ = [(n, C.c_uint32) for n in (
        "n_features", "precision", "K", "q", "b", "n_leaves", "depth", "n_trees", "n_classes", "block",
        "n_rot_reshuffle", "n_rot_level", "levels_used", "n_out", "n_segments", "block_branches",
        "block_leaves")]


vp = C.c_void_p
pvp = C.POINTER(C.c_void_p)
u64p = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
u8p = np.ctypeslib.ndpointer(dtype=np.uint8, flags="C_CONTIGUOUS")

_SIG = {
    "copse_last_error": (C.c_char_p, []),
    "copse_ctx_create": (C.c_int, [C.POINTER(copse_params), C.c_int, pvp]),
    "copse_ctx_destroy": (None, [vp]),
    "copse_ctx_primes": (C.c_int, [vp, u64p, C.c_size_t, C.POINTER(C.c_size_t)]),
    "copse_compile_forest": (C.c_int, [C.c_char_p, C.c_size_t, C.c_uint32, C.c_uint32, C.c_uint32, pvp]),
    "copse_model_destroy": (None, [vp]),
    "copse_model_info_get": (C.c_int, [vp, C.POINTER(copse_model_info)]),
    "copse_model_export": (C.c_int, [vp, vp, vp, vp, vp, vp, vp]),
    "copse_model_rotations": (C.c_int, [vp, vp, vp]),
    "copse_model_set_bsgs": (C.c_int, [vp, C.c_uint32, C.c_uint32]),
    "copse_ctx_set_ntt_cluster_max": (C.c_int, [vp, C.c_uint32]),
    "copse_ctx_set_ntt_fused_max": (C.c_int, [vp, C.c_uint32]),
    "copse_tune_fused": (C.c_int, [vp, vp, u32p, C.c_size_t, C.c_size_t, C.c_int, C.POINTER(C.c_float),
                                   C.POINTER(C.c_uint32)]),
    "copse_model_set_encrypted": (C.c_int, [vp, C.c_int]),
    "copse_model_set_fused": (C.c_int, [vp, C.c_int]),
    "copse_model_is_fused": (C.c_int, [vp]),
    "copse_model_set_shuffle": (C.c_int, [vp, vp, C.c_size_t, vp]),
    "copse_model_codebook": (C.c_int, [vp, u32p]),
    "copse_model_is_encrypted": (C.c_int, [vp]),
    "copse_encrypt_model": (C.c_int, [vp, vp, vp, C.c_uint64]),
    "copse_encmodel_export": (C.c_int, [vp, vp, C.c_size_t, u64p, C.c_size_t]),
    "copse_tune_ntt": (C.c_int, [vp, u32p, C.c_size_t, C.c_int, C.POINTER(C.c_float), C.POINTER(C.c_float),
                                 C.POINTER(C.c_uint32)]),
    "copse_tune_bsgs": (C.c_int, [vp, vp, u32p, C.c_size_t, u32p, C.c_size_t, C.c_size_t, C.c_int,
                                  C.POINTER(C.c_float), C.POINTER(C.c_float)]),
    "copse_tune_dnum": (C.c_int, [vp, C.c_int, vp, u32p, C.c_size_t, C.c_size_t, C.c_int,
                                  C.POINTER(C.c_float), C.POINTER(C.c_uint32)]),
    "copse_model_get_bsgs": (C.c_int, [vp, C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]),
    "copse_classify_plain": (C.c_int, [vp, u32p, C.c_size_t, u8p]),
    "copse_keygen": (C.c_int, [vp, C.c_uint64, C.POINTER(C.c_void_p), C.c_size_t, pvp, pvp]),
    "copse_keys_destroy": (None, [vp]),
    "copse_evk_destroy": (None, [vp]),
    "copse_keys_export_secret": (C.c_int, [vp, i64p]),
    "copse_evk_export": (C.c_int, [vp, C.c_uint64, u64p, C.c_size_t]),
    "copse_encrypt_features": (C.c_int, [vp, vp, vp, vp, C.c_size_t, C.c_int, C.c_uint64, pvp, vp]),
    "copse_infer": (C.c_int, [vp, vp, vp, vp, pvp, vp]),
    "copse_infer_timed": (C.c_int, [vp, vp, vp, vp, pvp, vp, C.POINTER(C.c_float)]),
    "copse_decrypt_labels": (C.c_int, [vp, vp, vp, vp, vp, C.c_size_t, C.c_int, vp]),
    "copse_decrypt_slots": (C.c_int, [vp, vp, vp, C.c_size_t, u64p]),
    "copse_ctbuf_count": (C.c_size_t, [vp]),
    "copse_ctbuf_shape": (C.c_int, [vp, C.c_size_t, C.POINTER(C.c_uint32), C.POINTER(C.c_uint32)]),
    "copse_ctbuf_export": (C.c_int, [vp, vp, C.c_size_t, u64p, C.c_size_t]),
    "copse_ctbuf_import": (C.c_int, [vp, u64p, C.c_size_t, C.c_uint32, pvp]),
    "copse_ctbuf_destroy": (None, [vp]),
    "copse_ct_mul": (C.c_int, [vp, vp, vp, C.c_size_t, vp, C.c_size_t, pvp, vp]),
    "copse_ct_rotate": (C.c_int, [vp, vp, vp, C.c_size_t, C.c_uint32, pvp, vp]),
    "copse_ct_modswitch": (C.c_int, [vp, vp, C.c_size_t, pvp, vp]),
    "copse_ct_mul_plain": (C.c_int, [vp, vp, C.c_size_t, u64p, vp, pvp, vp]),
    "copse_ntt": (C.c_int, [vp, vp, C.c_size_t, C.c_uint32, C.c_int, vp]),
    "copse_poly_mul": (C.c_int, [vp, vp, vp, vp, C.c_uint32, vp]),
    "copse_stats_enable": (C.c_int, [C.c_int]),
    "copse_stats_reset": (C.c_int, []),
    "copse_stats_get": (C.c_int, [C.c_char_p, C.POINTER(C.c_uint64), C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "copse_stats_names": (C.c_int, [C.c_char_p, C.c_size_t]),
    "copse_stats_get_ops": (C.c_int, [C.c_char_p, C.POINTER(C.c_double)]),
    "copse_measure_int_peak": (C.c_int, [vp, C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_float)]),
    "copse_ctx_device_status": (C.c_int, [vp, C.POINTER(C.c_int)]),
}
for _n, (_r, _a) in _SIG.items():
    _f = getattr(_lib, _n)
    _f.restype = _r
    _f.argtypes = _a


def declared_functions():
    """Names of the functions include/copse.h declares."""
    with open(HEADER) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(copse_[a-z0-9_]+)\s*\(", text)))


def library():
    return _lib


def _check(st):
    if st != 0:
        raise CopseError(st, _lib.copse_last_error().decode())


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


# ---------------------------------------------------------------- context
def copse_ctx_create(log_n, prime_bits, n_primes, dnum=3, device=0):
    p = copse_params(log_n, prime_bits, n_primes, dnum)
    h = C.c_void_p()
    _check(_lib.copse_ctx_create(C.byref(p), device, C.byref(h)))
    return h


def copse_ctx_destroy(ctx):
    _lib.copse_ctx_destroy(ctx)


COPSE_DEV_MAC_WAIT = 1


def copse_ctx_device_status(ctx):
    """The context's device status bits (COPSE_DEV_*), read after all queued work and then
    cleared; 0 when no kernel's bounded wait ran out."""
    st = C.c_int(0)
    rc = _lib.copse_ctx_device_status(ctx, C.byref(st))
    if rc not in (0, -9):  # COPSE_ETIMEOUT: the bits say which wait
        _check(rc)
    return st.value


def copse_ctx_primes(ctx):
    n = C.c_size_t()
    buf = np.zeros(128, dtype=np.uint64)
    _check(_lib.copse_ctx_primes(ctx, buf, buf.size, C.byref(n)))
    return [int(x) for x in buf[: n.value]]


# ---------------------------------------------------------------- models
def copse_compile_forest(text, precision, n_features=0, log_n=14):
    b = text.encode()
    h = C.c_void_p()
    _check(_lib.copse_compile_forest(b, len(b), precision, n_features, log_n, C.byref(h)))
    return h


def copse_model_destroy(m):
    _lib.copse_model_destroy(m)


def copse_model_info_get(m):
    info = copse_model_info()
    _check(_lib.copse_model_info_get(m, C.byref(info)))
    return {n: getattr(info, n) for n, _ in copse_model_info._fields_}


def copse_model_export(m):
    i = copse_model_info_get(m)
    q, b, L, d = i["q"], i["b"], i["n_leaves"], i["depth"]
    thr = np.zeros(q, np.uint32)
    sb = np.zeros(q, np.int32)
    R = np.zeros(b * q, np.uint8)
    lvl = np.zeros(max(d * L * b, 1), np.uint8)
    mask = np.zeros(max(d * L, 1), np.uint8)
    bl = np.zeros(b, np.uint32)
    _check(_lib.copse_model_export(m, _ptr(thr), _ptr(sb), _ptr(R), _ptr(lvl), _ptr(mask), _ptr(bl)))
    return {"thr_slot": thr, "slot_branch": sb, "R": R.reshape(b, q), "lvl": lvl[: d * L * b].reshape(d, L, b),
            "mask": mask[: d * L].reshape(d, L), "br_level": bl}


def copse_model_rotations(m):
    i = copse_model_info_get(m)
    a = np.zeros(max(i["n_rot_reshuffle"], 1), np.uint32)
    b = np.zeros(max(i["n_rot_level"], 1), np.uint32)
    _check(_lib.copse_model_rotations(m, _ptr(a), _ptr(b)))
    return a[: i["n_rot_reshuffle"]].tolist(), b[: i["n_rot_level"]].tolist()


def copse_model_set_bsgs(m, g_reshuffle, g_level):
    _check(_lib.copse_model_set_bsgs(m, g_reshuffle, g_level))


def copse_model_set_shuffle(m, src=None, codebook=None):
    """src[j]: leaf of output slot j (-1 = padding); codebook[j]: its class; None turns it off."""
    if src is None:
        _check(_lib.copse_model_set_shuffle(m, None, 0, None))
        return
    a = np.ascontiguousarray(src, dtype=np.int32)
    b = np.ascontiguousarray(codebook, dtype=np.uint32)
    _check(_lib.copse_model_set_shuffle(m, a.ctypes.data_as(C.c_void_p), a.size, b.ctypes.data_as(C.c_void_p)))


def copse_model_codebook(m):
    i = copse_model_info_get(m)
    out = np.zeros(max(i["n_out"], 1), np.uint32)
    _check(_lib.copse_model_codebook(m, out))
    return out[: i["n_out"]]


def copse_model_set_encrypted(m, on=True):
    _check(_lib.copse_model_set_encrypted(m, 1 if on else 0))


def copse_model_set_fused(m, on=True):
    _check(_lib.copse_model_set_fused(m, 1 if on else 0))


def copse_model_is_fused(m):
    return bool(_lib.copse_model_is_fused(m))


def copse_encrypt_model(ctx, keys, m, seed):
    _check(_lib.copse_encrypt_model(ctx, keys, m, seed))


def copse_encmodel_export(ctx, m, index, level, N):
    """model ciphertext `index` in coefficient form, [2][level][N]"""
    out = np.zeros(2 * level * N, dtype=np.uint64)
    _check(_lib.copse_encmodel_export(ctx, m, index, out, out.size))
    return out.reshape(2, level, N)


def copse_model_get_bsgs(m):
    a, b = C.c_uint32(), C.c_uint32()
    _check(_lib.copse_model_get_bsgs(m, C.byref(a), C.byref(b)))
    return a.value, b.value


def copse_tune_ntt(ctx, sizes=(4, 8, 16, 32, 64, 128, 256), reps=5):
    """-> (max_cluster, {size: (cluster ms, tiled ms)}); the context takes the cluster
    NTT for batches up to max_cluster residue polynomials."""
    sz = np.ascontiguousarray(sizes, dtype=np.uint32)
    mc = (C.c_float * len(sizes))()
    mt = (C.c_float * len(sizes))()
    lim = C.c_uint32()
    _check(_lib.copse_tune_ntt(ctx, sz, len(sizes), reps, mc, mt, C.byref(lim)))
    return lim.value, {int(x): (float(mc[i]), float(mt[i])) for i, x in enumerate(sizes)}


def copse_ctx_set_ntt_cluster_max(ctx, max_cluster):
    _check(_lib.copse_ctx_set_ntt_cluster_max(ctx, max_cluster))


def copse_ctx_set_ntt_fused_max(ctx, max_fused):
    _check(_lib.copse_ctx_set_ntt_fused_max(ctx, max_fused))


def copse_tune_fused(ctx, model, cands=(64, 128, 256, 512, 1 << 30), n_queries=1, reps=3):
    """-> (best, {candidate: ms per inference}); the fused-transform crossover is left set."""
    c = np.ascontiguousarray(cands, dtype=np.uint32)
    ms = (C.c_float * len(cands))()
    best = C.c_uint32()
    _check(_lib.copse_tune_fused(ctx, model, c, len(cands), n_queries, reps, ms, C.byref(best)))
    return best.value, {int(x): float(ms[i]) for i, x in enumerate(cands)}


def copse_tune_bsgs(ctx, model, g_r, g_l, n_queries=1, reps=3):
    """-> ({g_r: reshuffle ms}, {g_l: level ms}); the best plan is left set on the model."""
    a = np.ascontiguousarray(g_r, dtype=np.uint32) if len(g_r) else np.zeros(1, np.uint32)
    b = np.ascontiguousarray(g_l, dtype=np.uint32) if len(g_l) else np.zeros(1, np.uint32)
    ma = (C.c_float * max(len(g_r), 1))()
    mb = (C.c_float * max(len(g_l), 1))()
    _check(_lib.copse_tune_bsgs(ctx, model, a, len(g_r), b, len(g_l), n_queries, reps, ma, mb))
    return ({int(g): float(ma[i]) for i, g in enumerate(g_r)}, {int(g): float(mb[i]) for i, g in enumerate(g_l)})


def copse_tune_dnum(log_n, prime_bits, n_primes, model, dnums, n_queries=1, reps=3, device=0):
    """-> (best dnum, {dnum: ms per inference})."""
    p = copse_params(log_n, prime_bits, n_primes, 1)
    d = np.ascontiguousarray(dnums, dtype=np.uint32)
    ms = (C.c_float * len(dnums))()
    best = C.c_uint32()
    _check(_lib.copse_tune_dnum(C.byref(p), device, model, d, len(dnums), n_queries, reps, ms, C.byref(best)))
    return best.value, {int(x): float(ms[i]) for i, x in enumerate(dnums)}


def copse_classify_plain(m, feats):
    feats = np.ascontiguousarray(feats, dtype=np.uint32)
    i = copse_model_info_get(m)
    n = feats.shape[0]
    out = np.zeros(max(n * i["n_leaves"], 1), np.uint8)
    _check(_lib.copse_classify_plain(m, feats.reshape(-1) if n else np.zeros(1, np.uint32), n, out))
    return out[: n * i["n_leaves"]].reshape(n, i["n_leaves"])


# ---------------------------------------------------------------- keys
def copse_keygen(ctx, seed, models):
    arr = (C.c_void_p * max(len(models), 1))(*[m.value for m in models])
    k, e = C.c_void_p(), C.c_void_p()
    _check(_lib.copse_keygen(ctx, seed, arr, len(models), C.byref(k), C.byref(e)))
    return k, e


def copse_keys_destroy(k):
    _lib.copse_keys_destroy(k)


def copse_evk_destroy(e):
    _lib.copse_evk_destroy(e)


def copse_keys_export_secret(k, n):
    s = np.zeros(n, np.int64)
    _check(_lib.copse_keys_export_secret(k, s))
    return s


def copse_evk_export(e, galois, words):
    out = np.zeros(words, np.uint64)
    _check(_lib.copse_evk_export(e, galois, out, words))
    return out


# ---------------------------------------------------------------- data
def copse_encrypt_features(ctx, keys, model, feats, seed, stream=None, on_device=False, n_queries=None):
    """feats: host numpy [n, n_features] (on_device=False) or a device pointer (int) with n_queries."""
    h = C.c_void_p()
    if on_device:
        _check(_lib.copse_encrypt_features(ctx, keys, model, C.c_void_p(feats), n_queries, 1, seed, C.byref(h),
                                           C.c_void_p(stream)))
    else:
        f = np.ascontiguousarray(feats, dtype=np.uint32)
        _check(_lib.copse_encrypt_features(ctx, keys, model, _ptr(f), f.shape[0], 0, seed, C.byref(h),
                                           C.c_void_p(stream)))
    return h


def copse_infer(ctx, evk, model, feats, stream=None):
    h = C.c_void_p()
    _check(_lib.copse_infer(ctx, evk, model, feats, C.byref(h), C.c_void_p(stream)))
    return h


STAGES = ("comparison", "reshuffle", "levels", "aggregation")


def copse_infer_timed(ctx, evk, model, feats, stream=None):
    """copse_infer with device time per stage of Algorithm 1; returns
    (result buffer, {stage: ms})."""
    h = C.c_void_p()
    ms = (C.c_float * 4)()
    _check(_lib.copse_infer_timed(ctx, evk, model, feats, C.byref(h), C.c_void_p(stream), ms))
    return h, dict(zip(STAGES, (float(v) for v in ms)))


def copse_decrypt_labels(ctx, keys, model, result, n_queries, stream=None, out_device_ptr=None, out=None):
    """Leaf bits [n_queries, n_out]: into device memory at out_device_ptr (async), else into the
    host array `out` (e.g. pinned memory; uint8, at least n_queries * n_out) or a new array."""
    if out_device_ptr is not None:
        _check(_lib.copse_decrypt_labels(ctx, keys, model, result, C.c_void_p(out_device_ptr), n_queries, 1,
                                         C.c_void_p(stream)))
        return None
    L = copse_model_info_get(model)["n_out"]
    if out is None:
        out = np.zeros(max(n_queries * L, 1), np.uint8)
    out = out.reshape(-1)
    _check(_lib.copse_decrypt_labels(ctx, keys, model, result, _ptr(out), n_queries, 0, C.c_void_p(stream)))
    return out[: n_queries * L].reshape(n_queries, L)


def copse_decrypt_slots(ctx, keys, buf, index, n):
    out = np.zeros(n, np.uint64)
    _check(_lib.copse_decrypt_slots(ctx, keys, buf, index, out))
    return out


# ---------------------------------------------------------------- buffers
def copse_ctbuf_count(b):
    return _lib.copse_ctbuf_count(b)


def copse_ctbuf_shape(b, i):
    lv, nc = C.c_uint32(), C.c_uint32()
    _check(_lib.copse_ctbuf_shape(b, i, C.byref(lv), C.byref(nc)))
    return lv.value, nc.value


def copse_ctbuf_export(ctx, b, i, N):
    lv, nc = copse_ctbuf_shape(b, i)
    out = np.zeros(nc * lv * N, np.uint64)
    _check(_lib.copse_ctbuf_export(ctx, b, i, out, out.size))
    return out.reshape(nc, lv, N)


def copse_ctbuf_import(ctx, cts):
    """cts: numpy [n_ct, 2, level, N] coefficient residues."""
    a = np.ascontiguousarray(cts, dtype=np.uint64)
    h = C.c_void_p()
    _check(_lib.copse_ctbuf_import(ctx, a.reshape(-1), a.shape[0], a.shape[2], C.byref(h)))
    return h


def copse_ctbuf_destroy(b):
    _lib.copse_ctbuf_destroy(b)


# ---------------------------------------------------------------- ring ops
def copse_ct_mul(ctx, evk, a, ia, b, ib, stream=None):
    h = C.c_void_p()
    _check(_lib.copse_ct_mul(ctx, evk, a, ia, b, ib, C.byref(h), C.c_void_p(stream)))
    return h


def copse_ct_rotate(ctx, evk, a, ia, k, stream=None):
    h = C.c_void_p()
    _check(_lib.copse_ct_rotate(ctx, evk, a, ia, k, C.byref(h), C.c_void_p(stream)))
    return h


def copse_ct_modswitch(ctx, a, ia, stream=None):
    h = C.c_void_p()
    _check(_lib.copse_ct_modswitch(ctx, a, ia, C.byref(h), C.c_void_p(stream)))
    return h


def copse_ct_mul_plain(ctx, a, ia, mul_slots, add_slots=None, stream=None):
    h = C.c_void_p()
    m = np.ascontiguousarray(mul_slots, dtype=np.uint64)
    ad = None if add_slots is None else np.ascontiguousarray(add_slots, dtype=np.uint64)
    _check(_lib.copse_ct_mul_plain(ctx, a, ia, m, _ptr(ad), C.byref(h), C.c_void_p(stream)))
    return h


def copse_ntt(ctx, data_ptr, n_polys, n_res, inverse=False, stream=None):
    _check(_lib.copse_ntt(ctx, C.c_void_p(data_ptr), n_polys, n_res, 1 if inverse else 0, C.c_void_p(stream)))


def copse_poly_mul(ctx, a_ptr, b_ptr, c_ptr, n_res, stream=None):
    _check(_lib.copse_poly_mul(ctx, C.c_void_p(a_ptr), C.c_void_p(b_ptr), C.c_void_p(c_ptr), n_res,
                               C.c_void_p(stream)))


# ---------------------------------------------------------------- kernel timing
def copse_stats_enable(on=True):
    _check(_lib.copse_stats_enable(1 if on else 0))


def copse_stats_reset():
    _check(_lib.copse_stats_reset())


def copse_stats_get(name=None):
    n, ms, by = C.c_uint64(), C.c_double(), C.c_double()
    _check(_lib.copse_stats_get(name.encode() if name else None, C.byref(n), C.byref(ms), C.byref(by)))
    return {"launches": n.value, "ms": ms.value, "bytes": by.value}


def copse_stats_get_ops(name=None):
    v = C.c_double()
    _check(_lib.copse_stats_get_ops(name.encode() if name else None, C.byref(v)))
    return v.value


class copse_wl_item(C.Structure):
    _fields_ = [("kind", C.c_uint32), ("a", C.c_uint32), ("b", C.c_uint32), ("dep", C.c_int32)]


WL_KINDS = {"add": 0, "sub": 1, "tensor": 3}
_lib.copse_worklist_run.restype = C.c_int
_lib.copse_worklist_run.argtypes = [vp, vp, C.POINTER(copse_wl_item), C.c_size_t, C.c_int, pvp, vp]


def copse_worklist_run(ctx, inbuf, items, timeout_ms=1000, stream=None):
    """items: (kind, a, b, dep) with kind in WL_KINDS; returns the buffer of the items' results."""
    arr = (copse_wl_item * max(1, len(items)))(*[copse_wl_item(WL_KINDS[k], a, b, d) for k, a, b, d in items])
    h = C.c_void_p()
    _check(_lib.copse_worklist_run(ctx, inbuf, arr, len(items), timeout_ms, C.byref(h), C.c_void_p(stream)))
    return h


INT_PEAK_KINDS = {"mac": 0, "butterfly": 1, "barrett": 2}


def copse_measure_int_peak(ctx, kind, reps=5):
    """Measured device rate of one kind of modular arithmetic ("mac", "butterfly",
    "barrett"): (operations per second, best run in ms)."""
    ops, ms = C.c_double(), C.c_float()
    _check(_lib.copse_measure_int_peak(ctx, INT_PEAK_KINDS[kind], reps, C.byref(ops), C.byref(ms)))
    return ops.value, ms.value


def copse_stats_names():
    buf = C.create_string_buffer(4096)
    _check(_lib.copse_stats_names(buf, 4096))
    return [x for x in buf.value.decode().split("\n") if x]


def copse_stats_all():
    return {n: copse_stats_get(n) for n in copse_stats_names()}


# ---------------------------------------------------------------- allocation-free product
_lib.copse_poly_mul_noalloc.restype = C.c_int
_lib.copse_poly_mul_noalloc.argtypes = [vp, vp, vp, vp, C.c_uint32, vp]


def copse_poly_mul_noalloc(ctx, a_ptr, b_ptr, c_ptr, n_res, stream=None):
    """copse_poly_mul without any allocation (fixed device scratch; see include/copse.h)."""
    _check(_lib.copse_poly_mul_noalloc(ctx, C.c_void_p(a_ptr), C.c_void_p(b_ptr), C.c_void_p(c_ptr), n_res,
                                       C.c_void_p(stream)))


# ---------------------------------------------------------------- sessions (CUDA graphs)
_lib.copse_session_create.restype = C.c_int
_lib.copse_session_create.argtypes = [vp, vp, vp, vp, C.c_size_t, pvp]
_lib.copse_session_run.restype = C.c_int
_lib.copse_session_run.argtypes = [vp, vp, C.c_int, C.c_uint64, vp, C.c_int, vp]
_lib.copse_session_destroy.restype = None
_lib.copse_session_destroy.argtypes = [vp]


def copse_session_create(ctx, keys, evk, model, n_queries):
    h = C.c_void_p()
    _check(_lib.copse_session_create(ctx, keys, evk, model, n_queries, C.byref(h)))
    return h


def copse_session_run(session, feats, seed, out=None, stream=None, feats_ptr=None, out_ptr=None):
    """feats: host numpy [n, n_features] or feats_ptr (device); result into `out` (host numpy
    uint8 [n, n_leaves], returned) or out_ptr (device, async)."""
    if feats_ptr is not None:
        fp, fd = C.c_void_p(feats_ptr), 1
    else:
        f = np.ascontiguousarray(feats, dtype=np.uint32)
        fp, fd = _ptr(f), 0
    if out_ptr is not None:
        _check(_lib.copse_session_run(session, fp, fd, seed, C.c_void_p(out_ptr), 1, C.c_void_p(stream)))
        return None
    _check(_lib.copse_session_run(session, fp, fd, seed, _ptr(out), 0, C.c_void_p(stream)))
    return out


def copse_session_destroy(session):
    _lib.copse_session_destroy(session)


_lib.copse_session_create_batch.restype = C.c_int
_lib.copse_session_create_batch.argtypes = [vp, vp, vp, C.c_size_t, C.POINTER(C.c_void_p),
                                            C.POINTER(C.c_size_t), pvp]


def copse_session_create_batch(ctx, keys, evk, models, n_queries):
    """One graph over several (model, n_queries) items; see include/copse.h."""
    n = len(models)
    ms = (C.c_void_p * n)(*[m.value for m in models])
    qs = (C.c_size_t * n)(*n_queries)
    h = C.c_void_p()
    _check(_lib.copse_session_create_batch(ctx, keys, evk, n, ms, qs, C.byref(h)))
    return h


# ---------------------------------------------------------------- serving
STATUS.update({-8: "EADMIT", -9: "ETIMEOUT"})
_lib.copse_server_create.restype = C.c_int
_lib.copse_server_create.argtypes = [vp, vp, vp, C.POINTER(C.c_void_p), C.c_size_t, C.c_size_t, pvp]
_lib.copse_server_submit.restype = C.c_int
_lib.copse_server_submit.argtypes = [vp, C.c_uint32, u32p, C.POINTER(C.c_uint64)]
_lib.copse_server_poll.restype = C.c_int
_lib.copse_server_poll.argtypes = [vp, C.c_uint64, u8p, C.c_int, C.POINTER(C.c_double)]
_lib.copse_server_pending.restype = C.c_int
_lib.copse_server_pending.argtypes = [vp, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]
_lib.copse_server_destroy.restype = None
_lib.copse_server_destroy.argtypes = [vp]
_lib.copse_server_memory.restype = C.c_int
_lib.copse_server_memory.argtypes = [vp, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t), C.POINTER(C.c_size_t),
                                     C.POINTER(C.c_uint32)]
_lib.copse_server_set_memory_floor.restype = C.c_int
_lib.copse_server_set_memory_floor.argtypes = [vp, C.c_size_t]


def copse_server_create(ctx, keys, evk, models, max_pending=0):
    arr = (C.c_void_p * len(models))(*[m.value for m in models])
    h = C.c_void_p()
    _check(_lib.copse_server_create(ctx, keys, evk, arr, len(models), max_pending, C.byref(h)))
    return h


def copse_server_submit(server, model_id, feats):
    t = C.c_uint64()
    _check(_lib.copse_server_submit(server, model_id, np.ascontiguousarray(feats, dtype=np.uint32), C.byref(t)))
    return t.value


def copse_server_poll(server, ticket, n_leaves, timeout_ms=10000):
    """(bits, latency_ms) or raises CopseError(ETIMEOUT)."""
    out = np.zeros(n_leaves, dtype=np.uint8)
    lat = C.c_double()
    _check(_lib.copse_server_poll(server, ticket, out, timeout_ms, C.byref(lat)))
    return out, lat.value


def copse_server_memory(server):
    """(reserved bytes, largest launch bytes, admission floor bytes, concurrent launches)."""
    a, b, c, n = C.c_size_t(), C.c_size_t(), C.c_size_t(), C.c_uint32()
    _check(_lib.copse_server_memory(server, C.byref(a), C.byref(b), C.byref(c), C.byref(n)))
    return a.value, b.value, c.value, n.value


def copse_server_set_memory_floor(server, floor):
    _check(_lib.copse_server_set_memory_floor(server, floor))


def copse_server_pending(server):
    a, b = C.c_size_t(), C.c_size_t()
    _check(_lib.copse_server_pending(server, C.byref(a), C.byref(b)))
    return a.value, b.value


def copse_server_destroy(server):
    _lib.copse_server_destroy(server)
