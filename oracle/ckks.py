"""Plain RNS-CKKS oracle (Python side): parameters, FP64 canonical-embedding
encode/decode, keys, and ciphertext operations that call the plain-C ring
arithmetic in hetal_oracle.c.

TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
CPU-baseline leg of the benchmark may import this module; the product path
never does.  It shares no code with the CUDA library.

CKKS as the paper uses it (Sec. 2.2): s = N/2 complex slots, slot-wise add,
Mult (ciphertext product), CMult (plaintext product, which consumes a level
even for a constant), Lrot (left rotation of the slot vector), Conj, and
multiplication by sqrt(-1) without depth (Sec. 4.2.2).  The RNS variant,
hybrid key switching and samplers are the standard ones; each bit-fixing
choice is stated in hetal_oracle.c.
"""
import ctypes

import numpy as np

from . import build as _build

_LIB = None
u64p = ctypes.POINTER(ctypes.c_uint64)
i64p = ctypes.POINTER(ctypes.c_int64)


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        c_int, c_u64, vp = ctypes.c_int, ctypes.c_uint64, ctypes.c_void_p
        sig = {
            "orc_set_threads": (c_int, [c_int]),
            "orc_get_threads": (c_int, []),
            "orc_mulmod": (c_u64, [c_u64, c_u64, c_u64]),
            "orc_powmod": (c_u64, [c_u64, c_u64, c_u64]),
            "orc_is_prime": (c_int, [c_u64]),
            "orc_gen_primes": (c_int, [c_u64, c_int, c_int, u64p]),
            "orc_find_psi": (c_u64, [c_u64, c_u64]),
            "orc_ntt_fwd": (None, [u64p, c_int, c_u64, c_u64]),
            "orc_ntt_inv": (None, [u64p, c_int, c_u64, c_u64]),
            "orc_polymul_schoolbook": (None, [u64p, u64p, u64p, c_int, c_u64]),
            "orc_polymul": (None, [u64p, u64p, u64p, c_int, c_u64, c_u64]),
            "orc_philox4x64": (None, [u64p, u64p, u64p]),
            "orc_sample_uniform": (None, [c_u64, c_u64, c_int, c_u64, c_u64, u64p]),
            "orc_sample_cbd": (None, [c_u64, c_u64, c_int, i64p]),
            "orc_sample_secret": (None, [c_u64, c_u64, c_int, c_int, i64p]),
            "orc_params_size": (c_int, []),
            "orc_params_init": (None, [vp, c_int, c_int, c_int, c_int, u64p]),
            "orc_dnum": (c_int, [vp, c_int]),
            "orc_automorphism": (None, [u64p, u64p, c_int, c_u64, c_u64]),
            "orc_automorphism_signed": (None, [i64p, i64p, c_int, c_u64]),
            "orc_square_signed": (None, [i64p, i64p, c_int]),
            "orc_modup": (None, [vp, c_int, c_int, u64p, u64p]),
            "orc_moddown": (None, [vp, c_int, u64p, u64p]),
            "orc_kip": (None, [vp, c_int, c_int, u64p, u64p, u64p, u64p]),
            "orc_keyswitch": (None, [vp, c_int, u64p, u64p, u64p, u64p]),
            "orc_stream_secret": (c_u64, []),
            "orc_stream_key_a": (c_u64, [c_u64, c_u64]),
            "orc_stream_key_e": (c_u64, [c_u64, c_u64]),
            "orc_stream_enc_a": (c_u64, [c_u64]),
            "orc_stream_enc_e": (c_u64, [c_u64]),
            "orc_gen_switch_key": (None, [vp, c_u64, c_u64, i64p, i64p, u64p]),
            "orc_encrypt": (None, [vp, c_u64, c_u64, i64p, i64p, c_int, u64p]),
            "orc_decrypt": (None, [vp, i64p, u64p, c_int, u64p]),
            "orc_ct_add": (None, [vp, u64p, u64p, c_int, u64p]),
            "orc_ct_sub": (None, [vp, u64p, u64p, c_int, u64p]),
            "orc_ct_add_plain": (None, [vp, u64p, i64p, c_int, u64p]),
            "orc_ct_drop": (None, [vp, u64p, c_int, c_int, u64p]),
            "orc_ct_mul_i": (None, [vp, u64p, c_int, u64p]),
            "orc_rescale": (None, [vp, u64p, c_int, u64p]),
            "orc_ct_mul_plain": (None, [vp, u64p, i64p, c_int, u64p]),
            "orc_tensor": (None, [vp, u64p, u64p, c_int, u64p, u64p, u64p]),
            "orc_relin": (None, [vp, u64p, u64p, u64p, u64p, c_int, u64p]),
            "orc_automorph_ct": (None, [vp, u64p, c_int, c_u64, u64p, u64p]),
            "orc_automorph_hoisted": (None, [vp, u64p, c_int, c_int, u64p,
                                             ctypes.POINTER(u64p), u64p]),
            "orc_rot_sum": (None, [vp, u64p, c_int, c_int, u64p, ctypes.POINTER(u64p), u64p]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


def set_threads(n):
    """Threads the ring arithmetic splits independent limbs over (0 = every online
    processor, 1 = sequential); results do not depend on it.  Returns the count in use."""
    lib().orc_set_threads(int(n))
    return lib().orc_get_threads()


def threads():
    return lib().orc_get_threads()


def P(a):
    """ctypes pointer to a contiguous uint64 / int64 numpy array."""
    if a.dtype == np.uint64:
        return a.ctypes.data_as(u64p)
    if a.dtype == np.int64:
        return a.ctypes.data_as(i64p)
    raise TypeError(a.dtype)


def u64(a):
    return np.ascontiguousarray(a, dtype=np.uint64)


def i64(a):
    return np.ascontiguousarray(a, dtype=np.int64)


# --------------------------------------------------------------------------
# Parameters
# --------------------------------------------------------------------------
def gen_primes(step, bits, count):
    """The `count` largest primes below 2^bits that are 1 mod step, descending."""
    out = np.zeros(count, dtype=np.uint64)
    got = lib().orc_gen_primes(step, bits, count, P(out))
    return [int(x) for x in out[:got]]


PRIME_STEP = 1 << 32


def prime_chain(log_n, q0_bits, n_rescale, rescale_bits, n_special, special_bits, n_upper=0, upper_bits=0):
    """q_0 (the largest prime < 2^q0_bits that is 1 mod 2^32), then the
    n_rescale largest such primes below 2^rescale_bits, then (the levels above
    them) the n_upper largest below 2^upper_bits, then the n_special largest
    below 2^special_bits, each list descending and skipping primes already taken.  1 mod 2^32 implies 1 mod 2N (N <= 2^16), which the
    negacyclic NTT needs; the paper fixes neither the primes nor their form."""
    assert 2 << log_n <= PRIME_STEP
    taken = []

    def take(bits, count):
        cand = gen_primes(PRIME_STEP, bits, count + len(taken))
        got = [p for p in cand if p not in taken][:count]
        if len(got) != count:
            raise ValueError("not enough primes")
        taken.extend(got)
        return got

    q0 = take(q0_bits, 1)
    qs = take(rescale_bits, n_rescale)
    up = take(upper_bits, n_upper) if n_upper else []
    ps = take(special_bits, n_special)
    return q0 + qs + up, ps


class Params:
    """RNS-CKKS parameters: ring degree N = 2^log_n, ciphertext primes
    q_0..q_{L-1} (top level L-1), special primes p_0..p_{K-1}, digit size
    alpha, secret Hamming weight h, default scale delta."""

    def __init__(self, log_n, q0_bits, n_rescale, rescale_bits, n_special, special_bits,
                 alpha, h=192, log_delta=40, n_upper=0, upper_bits=0):
        self.log_n = log_n
        self.N = 1 << log_n
        self.slots = self.N // 2
        self.q, self.p = prime_chain(log_n, q0_bits, n_rescale, rescale_bits, n_special, special_bits,
                                     n_upper, upper_bits)
        self.L = len(self.q)
        self.K = len(self.p)
        if self.L + self.K > 128:   # orc_params holds at most 128 moduli
            raise ValueError("at most 128 moduli")
        self.alpha = alpha
        self.h = min(h, self.N // 2)
        self.delta = float(2 ** log_delta)
        self.moduli = self.q + self.p
        self.top = self.L - 1
        self._c = ctypes.create_string_buffer(lib().orc_params_size())
        mods = u64(self.moduli)
        lib().orc_params_init(self._c, self.N, self.L, self.K, alpha, P(mods))

    @property
    def c(self):
        return self._c

    def dnum(self, lv):
        return (lv + 1 + self.alpha - 1) // self.alpha

    def dnum_full(self):
        return (self.L + self.alpha - 1) // self.alpha

    def galois_rot(self, r):
        """X -> X^{5^r mod 2N}: left rotation of the slot vector by r."""
        return pow(5, r % self.slots, 2 * self.N)

    def galois_conj(self):
        return 2 * self.N - 1


# The two parameter sets the encrypted-matmul workloads use.
def params_n13():
    """N=2^13: q_0 ~ 2^60, three rescale primes ~ 2^40, one special prime ~ 2^61, scale 2^40."""
    return Params(13, 60, 3, 40, 1, 61, alpha=1, log_delta=40)


def params_n16():
    """N=2^16: q_0 ~ 2^60, eleven rescale primes ~ 2^50, two special primes ~ 2^61, scale 2^50."""
    return Params(16, 60, 11, 50, 2, 61, alpha=2, log_delta=50)


# --------------------------------------------------------------------------
# Canonical-embedding encode / decode (FP64).  Slot j sits at the root
# zeta^{5^j}, zeta = exp(i*pi/N); so X -> X^{5^r} rotates the slots left by r
# and X -> X^{-1} conjugates them.
# --------------------------------------------------------------------------
def _slot_exponents(N):
    s = N // 2
    g = np.empty(s, dtype=np.int64)
    e = 1
    for j in range(s):
        g[j] = e
        e = (e * 5) % (2 * N)
    return g


_GCACHE = {}


def slot_exponents(N):
    if N not in _GCACHE:
        _GCACHE[N] = _slot_exponents(N)
    return _GCACHE[N]


def round_half_away(x):
    return np.sign(x) * np.floor(np.abs(x) + 0.5)


def encode(z, scale, N):
    """Integer coefficients of round(scale * sigma^{-1}(z)) for z in C^{N/2}.

    sigma^{-1}: m_k = (1/N) sum_{e odd} w_e zeta^{-e k}, with w at 5^j equal to z_j
    and w at -5^j equal to conj(z_j); that sum is an N-point DFT after the
    substitution e = 2u+1 (library FFT)."""
    z = np.asarray(z, dtype=np.complex128)
    g = slot_exponents(N)
    v = np.zeros(N, dtype=np.complex128)
    v[(g - 1) // 2] = z
    v[(2 * N - g - 1) // 2] = np.conj(z)
    V = np.fft.fft(v)
    k = np.arange(N)
    m = (np.exp(-1j * np.pi * k / N) * V).real / N
    r = round_half_away(m * scale)
    if np.max(np.abs(r)) >= 2.0 ** 62:
        raise OverflowError("encoded plaintext exceeds 2^62")
    return r.astype(np.int64)


def encode_direct(z, scale, N):
    """Same as encode() by the O(N^2) definition (small N only; the pin for encode)."""
    z = np.asarray(z, dtype=np.complex128)
    g = slot_exponents(N)
    k = np.arange(N)
    acc = np.zeros(N)
    for j in range(N // 2):
        acc += 2.0 * (z[j] * np.exp(-1j * np.pi * g[j] * k / N)).real
    return round_half_away(acc / N * scale).astype(np.int64)


def decode_real_coeffs(m, scale, N):
    """Slots of a real-coefficient polynomial m (float array): z_j = m(zeta^{5^j}) / scale."""
    m = np.asarray(m, dtype=np.float64)
    k = np.arange(N)
    w = m * np.exp(1j * np.pi * k / N)
    vals = np.fft.ifft(w) * N           # m(zeta^{2u+1}) at index u
    g = slot_exponents(N)
    return vals[(g - 1) // 2] / scale


def crt_centered(residues, moduli):
    """Exact CRT of per-limb residues to centred Python integers (floats returned)."""
    Q = 1
    for q in moduli:
        Q *= q
    n = residues.shape[1]
    terms = []
    for i, q in enumerate(moduli):
        Qi = Q // q
        ci = (Qi * pow(Qi % q, -1, q)) % Q
        terms.append(ci)
    out = np.empty(n, dtype=np.float64)
    half = Q // 2
    cols = [residues[i].tolist() for i in range(len(moduli))]
    for x in range(n):
        v = 0
        for i in range(len(moduli)):
            v += cols[i][x] * terms[i]
        v %= Q
        if v > half:
            v -= Q
        out[x] = float(v)
    return out


# --------------------------------------------------------------------------
# Ciphertexts and keys
# --------------------------------------------------------------------------
class Ct:
    """A ciphertext at level lv: data[c, i, x] (c in {0,1}, limb i in [0, lv]),
    coefficient domain; scale is the factor its message carries."""
    __slots__ = ("data", "lv", "scale")

    def __init__(self, data, lv, scale):
        self.data = data
        self.lv = lv
        self.scale = scale

    def copy(self):
        return Ct(self.data.copy(), self.lv, self.scale)


KID_RELIN = 0
KID_CONJ = 1


def kid_rot(r):
    return 2 + r


class Oracle:
    """RNS-CKKS on the plain-C ring arithmetic, with op counters.

    seed fixes the secret key and every switching key (Philox streams, see
    hetal_oracle.c).  hoist: rotations asked for through rot_many() share one
    ModUp of the source (hoisted key switching)."""

    def __init__(self, params, seed):
        self.p = params
        self.seed = seed
        N = params.N
        L = lib()
        self.sk = np.zeros(N, dtype=np.int64)
        L.orc_sample_secret(seed, L.orc_stream_secret(), N, params.h, P(self.sk))
        self.keys = {}
        self.counts = {}

    # -- counters ---------------------------------------------------------
    def count(self, name, k=1):
        self.counts[name] = self.counts.get(name, 0) + k

    # -- keys -------------------------------------------------------------
    def switch_key(self, kid, s_from):
        p = self.p
        key = np.zeros((p.dnum_full(), 2, p.L + p.K, p.N), dtype=np.uint64)
        lib().orc_gen_switch_key(p.c, self.seed, kid, P(self.sk), P(i64(s_from)), P(key))
        return key

    def key(self, kid):
        if kid not in self.keys:
            p = self.p
            if kid == KID_RELIN:
                s2 = np.zeros(p.N, dtype=np.int64)
                lib().orc_square_signed(P(self.sk), P(s2), p.N)
                s_from = s2
            else:
                g = p.galois_conj() if kid == KID_CONJ else p.galois_rot(kid - 2)
                s_from = np.zeros(p.N, dtype=np.int64)
                lib().orc_automorphism_signed(P(self.sk), P(s_from), p.N, g)
            self.keys[kid] = self.switch_key(kid, s_from)
        return self.keys[kid]

    # -- encrypt / decrypt -----------------------------------------------
    def encrypt_int(self, m, lv, scale, nonce):
        p = self.p
        ct = np.zeros((2, lv + 1, p.N), dtype=np.uint64)
        lib().orc_encrypt(p.c, self.seed, nonce, P(self.sk), P(i64(m)), lv, P(ct))
        return Ct(ct, lv, scale)

    def decrypt_int(self, ct):
        """Centred integer message polynomial (as floats) of a ciphertext."""
        p = self.p
        out = np.zeros((ct.lv + 1, p.N), dtype=np.uint64)
        lib().orc_decrypt(p.c, P(self.sk), P(ct.data), ct.lv, P(out))
        return crt_centered(out, p.q[:ct.lv + 1])

    def decrypt_slots(self, ct):
        return decode_real_coeffs(self.decrypt_int(ct), ct.scale, self.p.N)

    # -- level / scale helpers -------------------------------------------
    def drop(self, a, lv):
        if lv == a.lv:
            return a
        assert lv < a.lv
        out = np.zeros((2, lv + 1, self.p.N), dtype=np.uint64)
        lib().orc_ct_drop(self.p.c, P(a.data), a.lv, lv, P(out))
        return Ct(out, lv, a.scale)

    def _align(self, a, b):
        lv = min(a.lv, b.lv)
        return self.drop(a, lv), self.drop(b, lv)

    @staticmethod
    def _check_scale(a, b):
        if abs(a.scale / b.scale - 1.0) > 1e-9:
            raise ValueError("scale mismatch %r vs %r" % (a.scale, b.scale))

    # -- slot-wise operations --------------------------------------------
    def add(self, a, b):
        a, b = self._align(a, b)
        self._check_scale(a, b)
        out = np.zeros_like(a.data)
        lib().orc_ct_add(self.p.c, P(a.data), P(b.data), a.lv, P(out))
        return Ct(out, a.lv, a.scale)

    def sub(self, a, b):
        a, b = self._align(a, b)
        self._check_scale(a, b)
        out = np.zeros_like(a.data)
        lib().orc_ct_sub(self.p.c, P(a.data), P(b.data), a.lv, P(out))
        return Ct(out, a.lv, a.scale)

    def mul_i(self, a):
        out = np.zeros_like(a.data)
        lib().orc_ct_mul_i(self.p.c, P(a.data), a.lv, P(out))
        return Ct(out, a.lv, a.scale)

    def rescale(self, a):
        assert a.lv >= 1
        out = np.zeros((2, a.lv, self.p.N), dtype=np.uint64)
        lib().orc_rescale(self.p.c, P(a.data), a.lv, P(out))
        return Ct(out, a.lv - 1, a.scale / self.p.q[a.lv])

    def mul_plain_int(self, a, m, pt_scale):
        """(c0*m, c1*m) then rescale by q_lv; the result carries scale*pt_scale/q_lv."""
        out = np.zeros_like(a.data)
        lib().orc_ct_mul_plain(self.p.c, P(a.data), P(i64(m)), a.lv, P(out))
        r = self.rescale(Ct(out, a.lv, a.scale * pt_scale))
        return r

    def mul_plain_sum(self, cts, ms, out_scale):
        """sum_i (c0_i m_i, c1_i m_i) over ciphertexts at one level, then one rescale by
        q_lv; the result is given out_scale (the plaintexts were encoded for it)."""
        lv = cts[0].lv
        acc = None
        for ct, m in zip(cts, ms):
            assert ct.lv == lv
            prod = np.zeros_like(ct.data)
            lib().orc_ct_mul_plain(self.p.c, P(ct.data), P(i64(m)), lv, P(prod))
            if acc is None:
                acc = prod
            else:
                nxt = np.zeros_like(acc)
                lib().orc_ct_add(self.p.c, P(acc), P(prod), lv, P(nxt))
                acc = nxt
        r = self.rescale(Ct(acc, lv, cts[0].scale))
        return Ct(r.data, r.lv, out_scale)

    def mul_const(self, a, value, out_scale):
        """CMult by the constant `value` landing on exactly out_scale: the integer constant
        polynomial round(value * out_scale * q_lv / scale(a)) (half away from zero), then the
        rescale by q_lv."""
        q = float(self.p.q[a.lv])
        v = value * out_scale * q / a.scale
        m = np.zeros(self.p.N, dtype=np.int64)
        m[0] = int(round_half_away(v))
        r = self.mul_plain_int(a, m, float(m[0]) / value if value else q)
        return Ct(r.data, r.lv, out_scale)

    def mod_raise(self, a, lv):
        """A level-0 ciphertext as one at level lv (bootstrapping's first step): each
        residue c mod q_0, centred (c if c <= (q_0 - 1) / 2, else c - q_0), reduced
        modulo q_0..q_lv.  It decrypts to t = Delta m + e + q_0 I over the integers; it is
        read at scale q_0, so its slots are sigma(t) / q_0."""
        assert a.lv == 0 and 0 < lv < self.p.L
        q0 = int(self.p.q[0])
        c = a.data[:, 0, :].astype(np.int64)
        v = np.where(c > (q0 - 1) // 2, c - q0, c)
        out = np.zeros((2, lv + 1, self.p.N), dtype=np.uint64)
        for i in range(lv + 1):
            out[:, i, :] = (v % int(self.p.q[i])).astype(np.uint64)
        return Ct(out, lv, float(q0))

    def mul_int(self, a, t):
        """t * (c0, c1) for a nonzero integer t: the message times t, same level and scale."""
        t = int(t)
        assert t != 0 and abs(t) < 2 ** 63
        m = np.zeros(self.p.N, dtype=np.int64)
        m[0] = t
        out = np.zeros_like(a.data)
        lib().orc_ct_mul_plain(self.p.c, P(a.data), P(m), a.lv, P(out))
        return Ct(out, a.lv, a.scale)

    def mult_scaled(self, a, b, target):
        """Mult whose result carries (about) the scale `target`: at the common level lv, the
        integer t = round(target * q_lv / (scale(a) * scale(b))) (half away from zero) multiplies
        a before the tensor product, relinearisation and rescale, which leave
        scale(a) * t * scale(b) / q_lv = target * (1 + e), |e| <= 1 / (2 t)."""
        a, b = self._align(a, b)
        q = float(self.p.q[a.lv])
        v = target * q / (a.scale * b.scale)
        if not (1.0 <= v < 4.0e18):
            raise ValueError("scaled product: the integer factor must lie in [1, 2^62)")
        t = int(round_half_away(v))
        at = self.mul_int(a, t)
        at.scale = a.scale * t
        d, lv, sc = self.tensor(at, b)
        return self.rescale(self.relin(d, lv, sc))

    def mul_plain2_int(self, a, ma, b, mb, pt_scale):
        """(a (.) ma + b (.) mb) then one rescale by q_lv; a and b at one level and scale."""
        assert a.lv == b.lv and abs(a.scale / b.scale - 1) < 1e-9
        ta, tb = np.zeros_like(a.data), np.zeros_like(b.data)
        lib().orc_ct_mul_plain(self.p.c, P(a.data), P(i64(ma)), a.lv, P(ta))
        lib().orc_ct_mul_plain(self.p.c, P(b.data), P(i64(mb)), b.lv, P(tb))
        out = np.zeros_like(a.data)
        lib().orc_ct_add(self.p.c, P(ta), P(tb), a.lv, P(out))
        return self.rescale(Ct(out, a.lv, a.scale * pt_scale))

    def add_plain_int(self, a, m):
        out = np.zeros_like(a.data)
        lib().orc_ct_add_plain(self.p.c, P(a.data), P(i64(m)), a.lv, P(out))
        return Ct(out, a.lv, a.scale)

    def tensor(self, a, b):
        a, b = self._align(a, b)
        n, lv = self.p.N, a.lv
        d = [np.zeros((lv + 1, n), dtype=np.uint64) for _ in range(3)]
        lib().orc_tensor(self.p.c, P(a.data), P(b.data), lv, P(d[0]), P(d[1]), P(d[2]))
        return d, lv, a.scale * b.scale

    def relin(self, d, lv, scale):
        out = np.zeros((2, lv + 1, self.p.N), dtype=np.uint64)
        lib().orc_relin(self.p.c, P(d[0]), P(d[1]), P(d[2]), P(self.key(KID_RELIN)), lv, P(out))
        return Ct(out, lv, scale)

    def automorph(self, a, g, kid):
        out = np.zeros_like(a.data)
        lib().orc_automorph_ct(self.p.c, P(a.data), a.lv, g, P(self.key(kid)), P(out))
        return Ct(out, a.lv, a.scale)

    def automorph_hoisted(self, a, gs, kids):
        n_g = len(gs)
        outs = np.zeros((n_g,) + a.data.shape, dtype=np.uint64)
        keys = [self.key(k) for k in kids]
        arr = (u64p * n_g)(*[P(k) for k in keys])
        gsa = u64(gs)
        lib().orc_automorph_hoisted(self.p.c, P(a.data), a.lv, n_g, P(gsa), arr, P(outs))
        return [Ct(outs[i], a.lv, a.scale) for i in range(n_g)]

    def rot_sum(self, a, rs):
        """a + sum of Lrot(a, r) for r in rs (nonzero, each with its key), one ModUp and one ModDown."""
        gs = u64([self.p.galois_rot(r % self.p.slots) for r in rs])
        keys = [self.key(kid_rot(r % self.p.slots)) for r in rs]
        arr = (u64p * len(rs))(*[P(k) for k in keys])
        out = np.zeros_like(a.data)
        lib().orc_rot_sum(self.p.c, P(a.data), a.lv, len(rs), P(gs), arr, P(out))
        return Ct(out, a.lv, a.scale)

    def rot_raw(self, a, r):
        r %= self.p.slots
        if r == 0:
            return a
        return self.automorph(a, self.p.galois_rot(r), kid_rot(r))

    def conj_raw(self, a):
        return self.automorph(a, self.p.galois_conj(), KID_CONJ)
