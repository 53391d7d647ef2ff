"""Seeded synthetic inputs for the encrypted-matmul workloads (no CKKS or
matrix-product arithmetic here; the same generators feed the CUDA library,
the tests and the benchmark).

The paper fine-tunes on features from pre-trained encoders (ViT-Base,
MPNet-Base: 768-dim, Sec. 5.2) with batch sizes 512-2048 (App. C.2); the
datasets are not used here.  Stand-ins:
  * features X ~ N(0, 1) / sqrt(dim), rows = batch size;
  * labels uniform over `classes`, one-hot Y zero-padded to c = 2^ceil(log2);
  * weights W: the first `classes` rows ~ N(0, 0.01^2), padded rows zero;
  * the matrix-product benchmark shapes of Table "tab:matmul_comp" use
    U(-1, 1) entries.
"""
import numpy as np


# Parameter sets (the argument lists of hetal_ctx_create / oracle Params).
#  log_n, q0_bits, n_rescale, rescale_bits, n_special, special_bits, alpha, log2 scale
PARAMS_N13 = dict(log_n=13, q0_bits=60, n_rescale=3, rescale_bits=40, n_special=1, special_bits=61, alpha=1,
                  log_scale=40)
PARAMS_N16 = dict(log_n=16, q0_bits=60, n_rescale=11, rescale_bits=50, n_special=2, special_bits=61, alpha=2,
                  log_scale=50)
# N = 2^13 with enough levels for DiagATB's two branches and the softmax stand-in
PARAMS_N13_DEEP = dict(log_n=13, q0_bits=60, n_rescale=6, rescale_bits=40, n_special=2, special_bits=61, alpha=2,
                       log_scale=40)
# Two NAG iterations and the validation logits without bootstrapping: 28 levels.  At N = 2^16
# the modulus is about 2^1520 (60 + 28 x 50 bits, plus 2 special primes), near the paper's
# log q ~ 1555 (Sec. 5.1); the N = 2^13 set runs the same circuit small for the oracle.
PARAMS_N16_NAG = dict(log_n=16, q0_bits=60, n_rescale=28, rescale_bits=50, n_special=2, special_bits=61, alpha=2,
                      log_scale=50)
# (45-bit rescale primes: there are too few primes 1 + k 2^32 near 2^40 for 28 levels)
PARAMS_N13_NAG = dict(log_n=13, q0_bits=60, n_rescale=28, rescale_bits=45, n_special=2, special_bits=61, alpha=2,
                      log_scale=45)


# Algorithm ASoftmax (App. A) on ciphertexts without bootstrapping: 74 levels for
# c' = 2, 89 for c' = 4, 119 for c' = 8 or 16, on 60-bit primes with scale 2^40
# (each product re-aims at the scale through an integer factor ~2^20), digits of 4
# primes and 4 special primes.  The modulus is far above what N = 2^16 secures
# (~2^7200 against the paper's 2^1555): these sets stand in for the levels
# bootstrapping would refresh between the algorithm's stages.
PARAMS_N13_SMX2 = dict(log_n=13, q0_bits=60, n_rescale=74, rescale_bits=60, n_special=4, special_bits=61, alpha=4,
                       log_scale=40)
PARAMS_N12_SMX4 = dict(log_n=12, q0_bits=60, n_rescale=89, rescale_bits=60, n_special=4, special_bits=61, alpha=4,
                       log_scale=40)
PARAMS_N16_SMX16 = dict(log_n=16, q0_bits=60, n_rescale=119, rescale_bits=60, n_special=4, special_bits=61, alpha=4,
                        log_scale=40)
# the same with the precise inverse of the extension (4 more levels: 128 moduli)
PARAMS_N16_SMX16P = dict(PARAMS_N16_SMX16, n_rescale=123)


def pad_pow2(x, lo=2):
    v = lo
    while v < x:
        v *= 2
    return v


def uniform_matrix(rows, cols, seed, lo=-1.0, hi=1.0):
    return np.random.default_rng(seed).uniform(lo, hi, (rows, cols))


def features(rows, dim, seed):
    return np.random.default_rng(seed).standard_normal((rows, dim)) / np.sqrt(dim)


def labels(rows, classes, seed):
    return np.random.default_rng(seed).integers(0, classes, rows)


def one_hot(lab, c):
    Y = np.zeros((len(lab), c))
    Y[np.arange(len(lab)), lab] = 1.0
    return Y


def weights(classes, dim, c, seed, std=0.01):
    W = np.zeros((c, dim))
    W[:classes] = np.random.default_rng(seed).standard_normal((classes, dim)) * std
    return W


def sigmoid_cheb15(R=8.0):
    """Power-basis coefficients (in y) of the degree-15 Chebyshev interpolant of
    y -> 1 / (1 + exp(-R y)) on [-1, 1] at the 16 Chebyshev nodes; the even
    coefficients beyond the constant are zero by symmetry and set so."""
    from numpy.polynomial import chebyshev as C
    k = np.arange(16)
    nodes = np.cos((2 * k + 1) * np.pi / 32)
    cc = C.chebfit(nodes, 1.0 / (1.0 + np.exp(-R * nodes)), 15)
    pc = C.cheb2poly(cc)
    pc[2::2] = 0.0
    pc[0] = 0.5
    return pc


def valid_mask(rows, classes, c, s0, s1):
    """0/1 slot vector of one s0 x s1 block: entry (i, j) is 1 when i < rows and
    (j mod c) < classes (the real entries of a horizontally tiled a x c matrix)."""
    i = np.arange(s0)[:, None]
    j = np.arange(s1)[None, :]
    return (((i < rows) & ((j % c) < classes)).astype(np.float64)).reshape(-1)


def batched_instances(n=64, seed=3, rows=(256, 4096), classes=(2, 100), dims=(384, 768, 1024), scale_rows=1):
    """Independent DiagABT + DiagATB instances of uneven size: a ~ U{rows}, classes ~ U{classes}
    (c = next power of two >= 2), b uniform over dims; X ~ N(0,1)/sqrt(b) (a x b), W (c x b) with
    the first `classes` rows ~ N(0, 0.01^2), A ~ U(-0.5, 0.5) (a x classes) as the DiagATB left operand."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        a = int(rng.integers(rows[0], rows[1] + 1)) // scale_rows
        k = int(rng.integers(classes[0], classes[1] + 1))
        b = int(rng.choice(dims))
        c = pad_pow2(k)
        X = rng.standard_normal((a, b)) / np.sqrt(b)
        W = np.zeros((c, b))
        W[:k] = rng.standard_normal((k, b)) * 0.01
        A = rng.uniform(-0.5, 0.5, (a, k))
        out.append(dict(a=a, b=b, classes=k, c=c, X=X, W=W, A=A))
    return out


def training_step(rows=1024, dim=768, classes=10, seed=2):
    """Inputs of one encrypted softmax-regression step: X (rows x dim), one-hot
    Y (rows x c), W (c x dim), c = classes padded to a power of two >= 16."""
    c = max(16, pad_pow2(classes))
    X = features(rows, dim, seed)
    Y = one_hot(labels(rows, classes, seed + 1), c)
    W = weights(classes, dim, c, seed + 2)
    return X, Y, W, c


def classification_split(n_batches, rows=1024, dim=768, classes=10, seed=11, separation=1.0):
    """Seeded synthetic stand-in for extracted features with learnable labels (Sec. 5.2 uses
    768-dimensional ViT / MPNet features): each class has a mean with entries ~ N(0, 1/dim)
    (norm about 1); a row is `separation` times its class's mean plus N(0, 1/dim) noise.
    Returns n_batches training batches [(X, labels)] and one validation set (X, labels), rows
    each."""
    rng = np.random.default_rng(seed)
    means = rng.standard_normal((classes, dim)) / np.sqrt(dim)

    def draw():
        lab = rng.integers(0, classes, rows)
        return separation * means[lab] + rng.standard_normal((rows, dim)) / np.sqrt(dim), lab
    return [draw() for _ in range(n_batches)], draw()
