"""Thin Python binding of the C ABI in include/hetal.h (argument marshalling
only: every computation runs in the CUDA library).

Functions keep the C names; handles are returned as ctypes pointers and
released with the matching *_free / *_destroy call.  Failures raise
HetalError with the library's status code and message.  Importing this
module never falls back to anything: if libhetal_gb300.so is missing the
first call raises.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libhetal_gb300.so")

OK = 0
MAX_MODULI = 128   # HETAL_MAX_MODULI_ABI
ERR_INVALID_ARG, ERR_SHAPE, ERR_LEVEL, ERR_MISSING_KEY = -1, -2, -3, -4
ERR_OOM, ERR_CUDA, ERR_SCALE, ERR_TIMEOUT, ERR_RECORDING, ERR_CANCELLED = -5, -6, -7, -8, -9, -10
TILE_NONE, TILE_VERT, TILE_HORIZ = 0, 1, 2
FLAG_HOIST, FLAG_LAZY_RELIN, FLAG_RADIX_SUM, FLAG_SHARED_ROT = 1, 2, 4, 8
PT_COLMASK, PT_ABT_DIAG, PT_DMASK, PT_ATB_DIAG, PT_SM_COEF, PT_SM_CONST, PT_DMASK_C = 1, 2, 3, 4, 5, 6, 7


class HetalError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("hetal status %d: %s" % (code, msg))
        self.code = code


class hetal_params(ctypes.Structure):
    _fields_ = [("log_n", ctypes.c_int), ("q0_bits", ctypes.c_int), ("n_rescale", ctypes.c_int),
                ("rescale_bits", ctypes.c_int), ("n_special", ctypes.c_int), ("special_bits", ctypes.c_int),
                ("alpha", ctypes.c_int), ("hamming_weight", ctypes.c_int), ("scale", ctypes.c_double),
                ("n_upper", ctypes.c_int), ("upper_bits", ctypes.c_int)]


class hetal_mat_desc(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int), ("n", ctypes.c_int), ("rows", ctypes.c_int), ("cols", ctypes.c_int),
                ("s0", ctypes.c_int), ("s1", ctypes.c_int), ("level", ctypes.c_int), ("scale", ctypes.c_double)]


class hetal_counters(ctypes.Structure):
    _fields_ = [("cmult", ctypes.c_longlong), ("mult", ctypes.c_longlong), ("rot", ctypes.c_longlong),
                ("conj", ctypes.c_longlong), ("keyswitch", ctypes.c_longlong), ("modup_digits", ctypes.c_longlong),
                ("ntt_limbs", ctypes.c_longlong), ("rescale", ctypes.c_longlong), ("modmul", ctypes.c_double)]


_lib = None
VP = ctypes.c_void_p
PVP = ctypes.POINTER(ctypes.c_void_p)
U64P = ctypes.POINTER(ctypes.c_uint64)
I64P = ctypes.POINTER(ctypes.c_int64)
DP = ctypes.POINTER(ctypes.c_double)
I32P = ctypes.POINTER(ctypes.c_int32)

_SIGS = {
    "hetal_ctx_create": [ctypes.POINTER(hetal_params), ctypes.c_int, VP, PVP],
    "hetal_ctx_destroy": [VP],
    "hetal_last_error": [VP],
    "hetal_ctx_moduli": [VP, U64P, ctypes.c_int],
    "hetal_ctx_info": [VP, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)],
    "hetal_ctx_sync": [VP],
    "hetal_ctx_set_batch_bytes": [VP, ctypes.c_size_t],
    "hetal_ctx_set_row_group": [VP, ctypes.c_int],
    "hetal_counters_get": [VP, ctypes.POINTER(hetal_counters)],
    "hetal_counters_reset": [VP],
    "hetal_keygen": [VP, ctypes.c_uint64, PVP],
    "hetal_sk_export": [VP, I64P],
    "hetal_sk_free": [VP],
    "hetal_evk_create": [VP, VP, ctypes.c_uint64, I32P, ctypes.c_size_t, ctypes.c_int, ctypes.c_int, PVP],
    "hetal_evk_export": [VP, VP, ctypes.c_int, ctypes.c_int32, U64P],
    "hetal_evk_free": [VP],
    "hetal_encrypt": [VP, VP, ctypes.c_uint64, ctypes.c_uint64, DP, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                      ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, PVP],
    "hetal_encrypt_int": [VP, VP, ctypes.c_uint64, ctypes.c_uint64, I64P, ctypes.POINTER(hetal_mat_desc), PVP],
    "hetal_decrypt": [VP, VP, VP, DP],
    "hetal_encode": [VP, DP, DP, ctypes.c_int, ctypes.c_double, I64P],
    "hetal_mat_desc_get": [VP, ctypes.POINTER(hetal_mat_desc)],
    "hetal_mat_export": [VP, VP, U64P],
    "hetal_mat_import": [VP, U64P, ctypes.POINTER(hetal_mat_desc), PVP],
    "hetal_mat_export_dev": [VP, VP, VP],
    "hetal_mat_import_dev": [VP, VP, ctypes.POINTER(hetal_mat_desc), PVP],
    "hetal_mat_drop": [VP, VP, ctypes.c_int, PVP],
    "hetal_mat_slice": [VP, VP, ctypes.c_int, ctypes.c_int, PVP],
    "hetal_mat_stack": [VP, PVP, ctypes.c_int, ctypes.POINTER(hetal_mat_desc), PVP],
    "hetal_mat_free": [VP],
    "hetal_ptset_create": [PVP],
    "hetal_ptset_put": [VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, I64P, ctypes.c_int],
    "hetal_ptset_free": [VP],
    "hetal_rotate": [VP, VP, VP, ctypes.c_int32, PVP],
    "hetal_rotate_hoisted": [VP, VP, VP, I32P, ctypes.c_size_t, PVP],
    "hetal_rotate_sum": [VP, VP, VP, I32P, ctypes.c_size_t, PVP],
    "hetal_conj": [VP, VP, VP, PVP],
    "hetal_mult": [VP, VP, VP, VP, PVP],
    "hetal_cmult": [VP, VP, DP, DP, PVP],
    "hetal_add": [VP, VP, VP, PVP],
    "hetal_mul_const": [VP, VP, ctypes.c_double, ctypes.c_double, PVP],
    "hetal_mul_int": [VP, VP, ctypes.c_int64, PVP],
    "hetal_mat_set_scale": [VP, VP, ctypes.c_double, PVP],
    "hetal_mod_raise": [VP, VP, ctypes.c_int, PVP],
    "hetal_plain_create": [VP, I64P, ctypes.c_int, ctypes.c_double, PVP],
    "hetal_plain_free": [VP],
    "hetal_cmult_plain": [VP, VP, VP, ctypes.c_double, PVP],
    "hetal_add_plain": [VP, VP, VP, PVP],
    "hetal_cmult_plain_sum": [VP, PVP, PVP, ctypes.c_int, ctypes.c_double, PVP],
    "hetal_mul_i": [VP, VP, PVP],
    "hetal_mult_scaled": [VP, VP, VP, VP, ctypes.c_double, PVP],
    "hetal_cmult_int": [VP, VP, I64P, ctypes.c_double, PVP],
    "hetal_add_plain_int": [VP, VP, I64P, PVP],
    "hetal_sub": [VP, VP, VP, PVP],
    "hetal_rescale": [VP, VP, PVP],
    "hetal_diag_abt": [VP, VP, VP, VP, ctypes.c_int, ctypes.c_double, VP, ctypes.c_int, PVP],
    "hetal_diag_atb": [VP, VP, VP, VP, ctypes.c_int, ctypes.c_double, VP, ctypes.c_int, PVP],
    "hetal_softmax_approx": [VP, VP, VP, DP, DP, ctypes.c_double, VP, PVP],
    "hetal_rotation_amounts": [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, I32P, ctypes.c_size_t],
    "hetal_ntt_forward": [VP, VP, ctypes.c_int, ctypes.c_int],
    "hetal_ntt_inverse": [VP, VP, ctypes.c_int, ctypes.c_int],
    "hetal_ntt_root": [VP, ctypes.c_int, U64P],
    "hetal_ntt32_moduli": [VP, ctypes.c_int, ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint32)],
    "hetal_ntt32_forward": [VP, VP, ctypes.c_int, ctypes.c_int],
    "hetal_probe_butterfly32_rate": [VP, ctypes.c_int, DP],
    "hetal_profile_kernel": [VP, ctypes.c_char_p],
    "hetal_profile_read": [VP, ctypes.POINTER(ctypes.c_longlong), DP, DP, DP],
    "hetal_launch_count": [VP, ctypes.POINTER(ctypes.c_longlong)],
    "hetal_alloc_count": [VP, ctypes.POINTER(ctypes.c_longlong)],
    "hetal_profile_summary": [VP, ctypes.c_char_p, ctypes.c_size_t],
    "hetal_rescale_noalloc": [VP, VP, VP, ctypes.c_int, ctypes.c_int],
    "hetal_run_pairs": [VP, VP, VP, ctypes.c_size_t, ctypes.c_int, ctypes.c_int, PVP, PVP],
    "hetal_run_pairs_batched": [VP, VP, VP, ctypes.c_size_t, ctypes.c_int, PVP, PVP],
    "hetal_tile_choose": [VP, VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int)],
    "hetal_plan_choose": [VP, VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                          ctypes.POINTER(ctypes.c_int)],
    "hetal_server_create": [VP, ctypes.c_int, ctypes.c_size_t, PVP],
    "hetal_server_destroy": [VP],
    "hetal_server_add_client": [VP, VP, ctypes.POINTER(ctypes.c_int)],
    "hetal_server_submit": [VP, VP, ctypes.POINTER(ctypes.c_uint64)],
    "hetal_server_wait": [VP, ctypes.c_uint64, PVP, DP, DP],
    "hetal_server_cancel": [VP, ctypes.c_uint64],
    "hetal_server_stats": [VP, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_size_t),
                           ctypes.POINTER(ctypes.c_size_t)],
    "hetal_probe_butterfly_rate": [VP, ctypes.c_int, DP],
    "hetal_probe_mac_rate": [VP, ctypes.c_int, DP],
    "hetal_graph_begin": [VP],
    "hetal_graph_end": [VP, PVP],
    "hetal_graph_launch": [VP, VP],
    "hetal_graph_kernels": [VP, ctypes.POINTER(ctypes.c_longlong)],
    "hetal_graph_free": [VP],
}
_VOID = {"hetal_ctx_destroy", "hetal_sk_free", "hetal_evk_free", "hetal_mat_free", "hetal_ptset_free",
         "hetal_plain_free",
         "hetal_server_destroy", "hetal_graph_free"}


def declared_symbols():
    """Names declared in include/hetal.h (parsed from the header text)."""
    import re
    hdr = os.path.join(_HERE, "..", "include", "hetal.h")
    with open(hdr) as f:
        txt = f.read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char \*)\s*(hetal_\w+)\s*\(", txt, re.M)))


def lib():
    """Load libhetal_gb300.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise HetalError(ERR_INVALID_ARG, "libhetal_gb300.so is not built (run __graft_entry__.build())")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = None if name in _VOID else (ctypes.c_char_p if name == "hetal_last_error" else ctypes.c_int)
        _lib = L
    return _lib


def _check(ctx, st):
    if st < 0:
        msg = lib().hetal_last_error(ctx)
        raise HetalError(st, msg.decode() if msg else "")
    return st


def _p(a, t):
    return a.ctypes.data_as(t)


def _out():
    return ctypes.c_void_p()


# ---- context ---------------------------------------------------------------------
def hetal_ctx_create(log_n, q0_bits, n_rescale, rescale_bits, n_special, special_bits, alpha,
                     hamming_weight=192, scale=2.0 ** 40, device=0, stream=None, n_upper=0, upper_bits=0):
    prm = hetal_params(log_n, q0_bits, n_rescale, rescale_bits, n_special, special_bits, alpha,
                       hamming_weight, scale, n_upper, upper_bits)
    out = _out()
    _check(None, lib().hetal_ctx_create(ctypes.byref(prm), device, stream, ctypes.byref(out)))
    return out


def hetal_ctx_destroy(ctx):
    lib().hetal_ctx_destroy(ctx)


def hetal_last_error(ctx):
    m = lib().hetal_last_error(ctx)
    return m.decode() if m else ""


def hetal_ctx_moduli(ctx):
    buf = np.zeros(MAX_MODULI, dtype=np.uint64)
    n = _check(ctx, lib().hetal_ctx_moduli(ctx, _p(buf, U64P), MAX_MODULI))
    return [int(x) for x in buf[:n]]


def hetal_ctx_info(ctx):
    n, l, k = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(ctx, lib().hetal_ctx_info(ctx, ctypes.byref(n), ctypes.byref(l), ctypes.byref(k)))
    return n.value, l.value, k.value


def hetal_ctx_sync(ctx):
    _check(ctx, lib().hetal_ctx_sync(ctx))


def hetal_ctx_set_batch_bytes(ctx, nbytes):
    _check(ctx, lib().hetal_ctx_set_batch_bytes(ctx, int(nbytes)))


def hetal_ctx_set_row_group(ctx, polys):
    _check(ctx, lib().hetal_ctx_set_row_group(ctx, int(polys)))


def hetal_counters_get(ctx):
    c = hetal_counters()
    _check(ctx, lib().hetal_counters_get(ctx, ctypes.byref(c)))
    return {k: getattr(c, k) for k, _ in hetal_counters._fields_}


def hetal_counters_reset(ctx):
    _check(ctx, lib().hetal_counters_reset(ctx))


# ---- keys ------------------------------------------------------------------------
def hetal_keygen(ctx, seed):
    out = _out()
    _check(ctx, lib().hetal_keygen(ctx, seed, ctypes.byref(out)))
    return out


def hetal_sk_export(ctx, sk):
    n = hetal_ctx_info(ctx)[0]
    out = np.zeros(n, dtype=np.int64)
    _check(ctx, lib().hetal_sk_export(sk, _p(out, I64P)))
    return out


def hetal_sk_free(sk):
    lib().hetal_sk_free(sk)


def hetal_evk_create(ctx, sk, seed, rot_steps, with_conj=True, with_relin=True):
    steps = np.ascontiguousarray(list(rot_steps), dtype=np.int32)
    out = _out()
    _check(ctx, lib().hetal_evk_create(ctx, sk, seed, _p(steps, I32P), len(steps), int(with_conj),
                                       int(with_relin), ctypes.byref(out)))
    return out


def hetal_evk_export(ctx, evk, kind, step, dnum, n_moduli):
    n = hetal_ctx_info(ctx)[0]
    out = np.zeros((dnum, 2, n_moduli, n), dtype=np.uint64)
    _check(ctx, lib().hetal_evk_export(ctx, evk, kind, step, _p(out, U64P)))
    return out


def hetal_evk_free(evk):
    lib().hetal_evk_free(evk)


# ---- matrices ----------------------------------------------------------------------
def hetal_encrypt(ctx, sk, seed, nonce, M, s0, s1, tiling=TILE_NONE, tile_c=0, level=0, scale=2.0 ** 40):
    M = np.ascontiguousarray(M, dtype=np.float64)
    out = _out()
    _check(ctx, lib().hetal_encrypt(ctx, sk, seed, nonce, _p(M, DP), M.shape[0], M.shape[1], s0, s1, tiling,
                                    tile_c, level, scale, ctypes.byref(out)))
    return out


def make_desc(m, n, rows, cols, s0, s1, level, scale):
    return hetal_mat_desc(m, n, rows, cols, s0, s1, level, scale)


def hetal_encrypt_int(ctx, sk, seed, nonce, pts, desc):
    pts = np.ascontiguousarray(pts, dtype=np.int64)
    out = _out()
    _check(ctx, lib().hetal_encrypt_int(ctx, sk, seed, nonce, _p(pts, I64P), ctypes.byref(desc),
                                        ctypes.byref(out)))
    return out


def hetal_mat_desc_get(mat):
    d = hetal_mat_desc()
    _check(None, lib().hetal_mat_desc_get(mat, ctypes.byref(d)))
    return d


def hetal_decrypt(ctx, sk, mat):
    d = hetal_mat_desc_get(mat)
    out = np.zeros((d.m * d.s0, d.n * d.s1), dtype=np.float64)
    _check(ctx, lib().hetal_decrypt(ctx, sk, mat, _p(out, DP)))
    return out


def hetal_encode(ctx, re, im, scale):
    re = np.ascontiguousarray(np.atleast_2d(re), dtype=np.float64)
    imp = None
    if im is not None:
        im = np.ascontiguousarray(np.atleast_2d(im), dtype=np.float64)
        imp = _p(im, DP)
    n = hetal_ctx_info(ctx)[0]
    out = np.zeros((re.shape[0], n), dtype=np.int64)
    _check(ctx, lib().hetal_encode(ctx, _p(re, DP), imp, re.shape[0], scale, _p(out, I64P)))
    return out


def hetal_mat_export(ctx, mat, out=None):
    """Coefficient residues [ct][2][level+1][N]; into `out` (C-contiguous uint64, e.g. a view of
    pinned memory, which a recorded export needs) when given."""
    d = hetal_mat_desc_get(mat)
    n = hetal_ctx_info(ctx)[0]
    shape = (d.m * d.n, 2, d.level + 1, n)
    if out is None:
        out = np.zeros(shape, dtype=np.uint64)
    elif out.dtype != np.uint64 or not out.flags.c_contiguous or out.size != int(np.prod(shape)):
        raise ValueError("export buffer must be C-contiguous uint64 with %d words" % int(np.prod(shape)))
    _check(ctx, lib().hetal_mat_export(ctx, mat, _p(out, U64P)))
    return out.reshape(shape)


def hetal_mat_import(ctx, residues, desc):
    residues = np.ascontiguousarray(residues, dtype=np.uint64)
    out = _out()
    _check(ctx, lib().hetal_mat_import(ctx, _p(residues, U64P), ctypes.byref(desc), ctypes.byref(out)))
    return out


def hetal_mat_export_dev(ctx, mat, dev_ptr):
    _check(ctx, lib().hetal_mat_export_dev(ctx, mat, ctypes.c_void_p(dev_ptr)))


def hetal_mat_import_dev(ctx, dev_ptr, desc):
    out = _out()
    _check(ctx, lib().hetal_mat_import_dev(ctx, ctypes.c_void_p(dev_ptr), ctypes.byref(desc), ctypes.byref(out)))
    return out


def hetal_mat_drop(ctx, mat, level):
    out = _out()
    _check(ctx, lib().hetal_mat_drop(ctx, mat, level, ctypes.byref(out)))
    return out


def hetal_mat_slice(ctx, mat, first, count):
    out = _out()
    _check(ctx, lib().hetal_mat_slice(ctx, mat, int(first), int(count), ctypes.byref(out)))
    return out


def hetal_mat_stack(ctx, mats, desc):
    """One matrix holding the blocks of `mats` in order, with desc's block grid and shape."""
    arr = (VP * len(mats))(*[m.value if isinstance(m, VP) else m for m in mats])
    out = _out()
    _check(ctx, lib().hetal_mat_stack(ctx, arr, len(mats), ctypes.byref(desc), ctypes.byref(out)))
    return out


def hetal_mat_free(mat):
    lib().hetal_mat_free(mat)


# ---- plaintext sets ----------------------------------------------------------------
def hetal_ptset_create():
    out = _out()
    _check(None, lib().hetal_ptset_create(ctypes.byref(out)))
    return out


def hetal_ptset_put(ptset, kind, index, level, coeffs):
    coeffs = np.ascontiguousarray(coeffs, dtype=np.int64)
    _check(None, lib().hetal_ptset_put(ptset, kind, index, level, _p(coeffs, I64P), coeffs.size))


def hetal_ptset_free(ptset):
    lib().hetal_ptset_free(ptset)


# ---- server-side operations ------------------------------------------------------------
def hetal_rotate(ctx, evk, mat, step):
    out = _out()
    _check(ctx, lib().hetal_rotate(ctx, evk, mat, step, ctypes.byref(out)))
    return out


def hetal_rotate_sum(ctx, evk, mat, steps):
    st = np.ascontiguousarray(list(steps), dtype=np.int32)
    out = _out()
    _check(ctx, lib().hetal_rotate_sum(ctx, evk, mat, _p(st, I32P), len(st), ctypes.byref(out)))
    return out


def hetal_rotate_hoisted(ctx, evk, mat, steps):
    st = np.ascontiguousarray(list(steps), dtype=np.int32)
    outs = (ctypes.c_void_p * len(st))()
    _check(ctx, lib().hetal_rotate_hoisted(ctx, evk, mat, _p(st, I32P), len(st), outs))
    return [ctypes.c_void_p(o) for o in outs]


def hetal_conj(ctx, evk, mat):
    out = _out()
    _check(ctx, lib().hetal_conj(ctx, evk, mat, ctypes.byref(out)))
    return out


def hetal_mult(ctx, evk, a, b):
    out = _out()
    _check(ctx, lib().hetal_mult(ctx, evk, a, b, ctypes.byref(out)))
    return out


def hetal_cmult(ctx, a, re, im=None):
    re = np.ascontiguousarray(re, dtype=np.float64)
    imp = None
    if im is not None:
        im = np.ascontiguousarray(im, dtype=np.float64)
        imp = _p(im, DP)
    out = _out()
    _check(ctx, lib().hetal_cmult(ctx, a, _p(re, DP), imp, ctypes.byref(out)))
    return out


def hetal_mul_const(ctx, a, value, out_scale):
    out = _out()
    _check(ctx, lib().hetal_mul_const(ctx, a, float(value), float(out_scale), ctypes.byref(out)))
    return out


def hetal_mat_set_scale(ctx, a, scale):
    out = _out()
    _check(ctx, lib().hetal_mat_set_scale(ctx, a, float(scale), ctypes.byref(out)))
    return out


def hetal_mod_raise(ctx, a, level):
    out = _out()
    _check(ctx, lib().hetal_mod_raise(ctx, a, int(level), ctypes.byref(out)))
    return out


def hetal_mul_i(ctx, a):
    out = _out()
    _check(ctx, lib().hetal_mul_i(ctx, a, ctypes.byref(out)))
    return out


def hetal_mul_int(ctx, a, t):
    out = _out()
    _check(ctx, lib().hetal_mul_int(ctx, a, int(t), ctypes.byref(out)))
    return out


def hetal_mult_scaled(ctx, evk, a, b, target_scale):
    out = _out()
    _check(ctx, lib().hetal_mult_scaled(ctx, evk, a, b, float(target_scale), ctypes.byref(out)))
    return out


def _plain_arg(ctx, pt):
    pt = np.ascontiguousarray(pt, dtype=np.int64)
    if pt.shape != (hetal_ctx_info(ctx)[0],):
        raise ValueError("a plaintext holds N coefficients")
    return pt


def hetal_cmult_int(ctx, a, pt, out_scale):
    pt = _plain_arg(ctx, pt)
    out = _out()
    _check(ctx, lib().hetal_cmult_int(ctx, a, _p(pt, I64P), float(out_scale), ctypes.byref(out)))
    return out


def hetal_add_plain_int(ctx, a, pt):
    pt = _plain_arg(ctx, pt)
    out = _out()
    _check(ctx, lib().hetal_add_plain_int(ctx, a, _p(pt, I64P), ctypes.byref(out)))
    return out


def hetal_plain_create(ctx, pt, level, scale):
    pt = _plain_arg(ctx, pt)
    out = _out()
    _check(ctx, lib().hetal_plain_create(ctx, _p(pt, I64P), int(level), float(scale), ctypes.byref(out)))
    return out


def hetal_plain_free(pt):
    lib().hetal_plain_free(pt)


def hetal_cmult_plain(ctx, a, pt, out_scale):
    out = _out()
    _check(ctx, lib().hetal_cmult_plain(ctx, a, pt, float(out_scale), ctypes.byref(out)))
    return out


def hetal_cmult_plain_sum(ctx, mats, plains, out_scale):
    """sum_i mats[i] (.) plains[i] (device plaintexts), one rescale; see include/hetal.h."""
    n = len(mats)
    if n != len(plains) or n == 0:
        raise ValueError("one plaintext per matrix")
    ma = (ctypes.c_void_p * n)(*[m.value if isinstance(m, ctypes.c_void_p) else m for m in mats])
    pa = (ctypes.c_void_p * n)(*[p.value if isinstance(p, ctypes.c_void_p) else p for p in plains])
    out = _out()
    _check(ctx, lib().hetal_cmult_plain_sum(ctx, ma, pa, n, float(out_scale), ctypes.byref(out)))
    return out


def hetal_add_plain(ctx, a, pt):
    out = _out()
    _check(ctx, lib().hetal_add_plain(ctx, a, pt, ctypes.byref(out)))
    return out


def hetal_add(ctx, a, b):
    out = _out()
    _check(ctx, lib().hetal_add(ctx, a, b, ctypes.byref(out)))
    return out


def hetal_sub(ctx, a, b):
    out = _out()
    _check(ctx, lib().hetal_sub(ctx, a, b, ctypes.byref(out)))
    return out


def hetal_rescale(ctx, a):
    out = _out()
    _check(ctx, lib().hetal_rescale(ctx, a, ctypes.byref(out)))
    return out


def hetal_diag_abt(ctx, evk, a, bbar, c, t, ptset=None, flags=0):
    out = _out()
    _check(ctx, lib().hetal_diag_abt(ctx, evk, a, bbar, c, t, ptset, flags, ctypes.byref(out)))
    return out


def hetal_diag_atb(ctx, evk, a_under, b, c, t, ptset=None, flags=0):
    out = _out()
    _check(ctx, lib().hetal_diag_atb(ctx, evk, a_under, b, c, t, ptset, flags, ctypes.byref(out)))
    return out


def hetal_softmax_approx(ctx, evk, mat, coeffs16, valid, target_scale, ptset=None):
    co = np.ascontiguousarray(coeffs16, dtype=np.float64)
    va = np.ascontiguousarray(valid, dtype=np.float64)
    out = _out()
    _check(ctx, lib().hetal_softmax_approx(ctx, evk, mat, _p(co, DP), _p(va, DP), target_scale, ptset,
                                           ctypes.byref(out)))
    return out


def hetal_rotation_amounts(s0, s1, c, flags=0):
    """Left-rotation amounts whose keys DiagABT / DiagATB use (ascending)."""
    n = lib().hetal_rotation_amounts(s0, s1, c, flags, None, 0)
    if n < 0:
        raise HetalError(n, "invalid block shape or class count")
    buf = np.zeros(max(n, 1), dtype=np.int32)
    lib().hetal_rotation_amounts(s0, s1, c, flags, _p(buf, I32P), n)
    return [int(x) for x in buf[:n]]


def hetal_ntt_forward(ctx, dev_ptr, n_polys, n_limbs):
    _check(ctx, lib().hetal_ntt_forward(ctx, ctypes.c_void_p(dev_ptr), n_polys, n_limbs))


def hetal_ntt_inverse(ctx, dev_ptr, n_polys, n_limbs):
    _check(ctx, lib().hetal_ntt_inverse(ctx, ctypes.c_void_p(dev_ptr), n_polys, n_limbs))


def hetal_ntt_root(ctx, limb):
    out = ctypes.c_uint64()
    _check(ctx, lib().hetal_ntt_root(ctx, limb, ctypes.byref(out)))
    return out.value


def hetal_ntt32_moduli(ctx, n_limbs):
    """(primes, 2N-th roots) of the 32-bit transform's first n_limbs limbs."""
    m = np.zeros(n_limbs, dtype=np.uint32)
    r = np.zeros(n_limbs, dtype=np.uint32)
    _check(ctx, lib().hetal_ntt32_moduli(ctx, n_limbs, m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                         r.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))))
    return [int(x) for x in m], [int(x) for x in r]


def hetal_ntt32_forward(ctx, dev_ptr, n_polys, n_limbs):
    _check(ctx, lib().hetal_ntt32_forward(ctx, dev_ptr, n_polys, n_limbs))


def hetal_probe_butterfly32_rate(ctx, iters=20000):
    r = ctypes.c_double()
    _check(ctx, lib().hetal_probe_butterfly32_rate(ctx, iters, ctypes.byref(r)))
    return r.value


def hetal_profile_kernel(ctx, name):
    _check(ctx, lib().hetal_profile_kernel(ctx, name.encode() if name else None))


def hetal_profile_read(ctx):
    n = ctypes.c_longlong()
    ms, mm, by = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(ctx, lib().hetal_profile_read(ctx, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(mm), ctypes.byref(by)))
    return {"launches": n.value, "ms": ms.value, "modmul": mm.value, "bytes": by.value}


def hetal_rescale_noalloc(ctx, dev_in, dev_out, n_ct, level):
    """Rescale on caller-owned NTT-domain device buffers without any device allocation."""
    _check(ctx, lib().hetal_rescale_noalloc(ctx, ctypes.c_void_p(dev_in), ctypes.c_void_p(dev_out), n_ct, level))


class hetal_pair_job(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("wbar", ctypes.c_void_p), ("a_under", ctypes.c_void_p),
                ("b", ctypes.c_void_p), ("c", ctypes.c_int), ("t_abt", ctypes.c_double), ("t_atb", ctypes.c_double),
                ("flags", ctypes.c_int)]


def _pair_jobs(jobs):
    n = len(jobs)
    return (hetal_pair_job * n)(*[hetal_pair_job(j["x"].value, j["wbar"].value, j["a_under"].value, j["b"].value,
                                                 j["c"], j["t_abt"], j["t_atb"], j.get("flags", -1)) for j in jobs])


def hetal_run_pairs(ctx, evk, jobs, workers=1, flags=0):
    """jobs: list of dicts with keys x, wbar, a_under, b (matrix handles), c, t_abt, t_atb and
    optionally flags (per instance).  Returns (list of DiagABT outputs, list of DiagATB outputs)."""
    n = len(jobs)
    arr = _pair_jobs(jobs)
    oa, ob = (ctypes.c_void_p * n)(), (ctypes.c_void_p * n)()
    _check(ctx, lib().hetal_run_pairs(ctx, evk, arr, n, workers, flags, oa, ob))
    return [ctypes.c_void_p(v) for v in oa], [ctypes.c_void_p(v) for v in ob]


def hetal_run_pairs_batched(ctx, evk, jobs, flags=0):
    """The same instances batched across instances (same bits as hetal_run_pairs)."""
    n = len(jobs)
    arr = _pair_jobs(jobs)
    oa, ob = (ctypes.c_void_p * n)(), (ctypes.c_void_p * n)()
    _check(ctx, lib().hetal_run_pairs_batched(ctx, evk, arr, n, flags, oa, ob))
    return [ctypes.c_void_p(v) for v in oa], [ctypes.c_void_p(v) for v in ob]


class hetal_request(ctypes.Structure):
    _fields_ = [("client", ctypes.c_int), ("kind", ctypes.c_int), ("a", ctypes.c_void_p), ("b", ctypes.c_void_p),
                ("c", ctypes.c_int), ("t", ctypes.c_double), ("flags", ctypes.c_int)]


def hetal_server_create(ctx, slots, budget_bytes):
    out = _out()
    _check(ctx, lib().hetal_server_create(ctx, slots, budget_bytes, ctypes.byref(out)))
    return out


def hetal_server_destroy(srv):
    lib().hetal_server_destroy(srv)


def hetal_server_add_client(ctx, srv, evk):
    cid = ctypes.c_int()
    _check(ctx, lib().hetal_server_add_client(srv, evk, ctypes.byref(cid)))
    return cid.value


def hetal_server_submit(ctx, srv, client, kind, a, b, c, t, flags=0):
    req = hetal_request(client, kind, a.value, b.value, c, t, flags)
    ticket = ctypes.c_uint64()
    _check(ctx, lib().hetal_server_submit(srv, ctypes.byref(req), ctypes.byref(ticket)))
    return ticket.value


def hetal_server_wait(ctx, srv, ticket):
    out = _out()
    q, r = ctypes.c_double(), ctypes.c_double()
    _check(ctx, lib().hetal_server_wait(srv, ticket, ctypes.byref(out), ctypes.byref(q), ctypes.byref(r)))
    return out, q.value, r.value


def hetal_server_cancel(ctx, srv, ticket):
    _check(ctx, lib().hetal_server_cancel(srv, ticket))


def hetal_server_stats(srv):
    n, res, peak = ctypes.c_longlong(), ctypes.c_size_t(), ctypes.c_size_t()
    _check(None, lib().hetal_server_stats(srv, ctypes.byref(n), ctypes.byref(res), ctypes.byref(peak)))
    return {"completed": n.value, "resident_bytes": res.value, "peak_inflight_bytes": peak.value}


def hetal_tile_choose(ctx, evk, a, b, c):
    out = ctypes.c_int()
    _check(ctx, lib().hetal_tile_choose(ctx, evk, a, b, c, ctypes.byref(out)))
    return out.value


def hetal_plan_choose(ctx, evk, a, b, c):
    """(s0, flags) for an a x b instance with c classes."""
    s0, fl = ctypes.c_int(), ctypes.c_int()
    _check(ctx, lib().hetal_plan_choose(ctx, evk, a, b, c, ctypes.byref(s0), ctypes.byref(fl)))
    return s0.value, fl.value


def hetal_profile_summary(ctx):
    buf = ctypes.create_string_buffer(1 << 16)
    _check(ctx, lib().hetal_profile_summary(ctx, buf, len(buf)))
    out = {}
    for ln in buf.value.decode().splitlines():
        name, n, ms, mm, by = ln.split("\t")
        out[name] = {"launches": int(n), "ms": float(ms), "modmul": float(mm), "bytes": float(by)}
    return out


def hetal_alloc_count(ctx):
    n = ctypes.c_longlong()
    _check(ctx, lib().hetal_alloc_count(ctx, ctypes.byref(n)))
    return n.value


def hetal_launch_count(ctx):
    n = ctypes.c_longlong()
    _check(ctx, lib().hetal_launch_count(ctx, ctypes.byref(n)))
    return n.value


def hetal_probe_butterfly_rate(ctx, iters=20000):
    out = ctypes.c_double()
    _check(ctx, lib().hetal_probe_butterfly_rate(ctx, iters, ctypes.byref(out)))
    return out.value


def hetal_graph_begin(ctx):
    """Open a recording: the calls that follow on ctx are captured into a CUDA graph."""
    _check(ctx, lib().hetal_graph_begin(ctx))


def hetal_graph_end(ctx):
    """Close the recording, instantiate the graph and launch it once; returns the graph."""
    out = _out()
    _check(ctx, lib().hetal_graph_end(ctx, ctypes.byref(out)))
    return out


def hetal_graph_launch(ctx, graph):
    _check(ctx, lib().hetal_graph_launch(ctx, graph))


def hetal_graph_kernels(graph):
    n = ctypes.c_longlong()
    _check(None, lib().hetal_graph_kernels(graph, ctypes.byref(n)))
    return n.value


def hetal_graph_free(graph):
    lib().hetal_graph_free(graph)


def hetal_probe_mac_rate(ctx, iters=20000):
    out = ctypes.c_double()
    _check(ctx, lib().hetal_probe_mac_rate(ctx, iters, ctypes.byref(out)))
    return out.value
