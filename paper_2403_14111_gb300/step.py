"""One encrypted softmax-regression training step through the C ABI (Protocol 1, step
3(a)), the NAG loop around it (step 3, Sec. 2.1), and the loop for any number of
iterations with W and V refreshed by bootstrapping (Sec. 2.2).  The step:

    logits/8 = DiagABT(<X>, <W-bar>, t = 1/8)          (Sec. 4.2.2)
    P        = p15(logits/8) (.) valid                  (degree-15 softmax stand-in)
    D        = P - <Y>
    G        = DiagATB(<D>, <X> at level(D)+1, t = lr/batch)   (Sec. 4.2.3, PRotUp branch)

train_step_asoftmax is the same step with the paper's softmax (Algorithm ASoftmax,
refreshed between its stages); refresh_packed bootstraps W and V together;
nag_train_boot runs NAG iterations on one batch, train_epochs Protocol 1's epochs over
mini-batches with the validation logits sent to a client (ValidationClient) that stops the
training.  Every operation is one C-ABI call; this module only sequences the calls.
"""
import math

import numpy as np

from . import hetal as H


def step_rotations(s0, s1, c, flags=0):
    """Rotation amounts DiagABT and DiagATB need for block shape s0 x s1, c classes and flags."""
    return H.hetal_rotation_amounts(s0, s1, c, flags)


def train_step(ctx, evk, X, Wbar, Y, coeffs, valid, c, lr_over_n, target_scale, flags=0, pts=(None, None, None)):
    """Returns (G, intermediates); the caller frees G (and the intermediates)."""
    logits = H.hetal_diag_abt(ctx, evk, X, Wbar, c, 1.0 / 8.0, pts[0], flags)
    P = H.hetal_softmax_approx(ctx, evk, logits, coeffs, valid, target_scale, pts[1])
    D = H.hetal_sub(ctx, P, Y)
    lvl = H.hetal_mat_desc_get(D).level
    Xl = H.hetal_mat_drop(ctx, X, lvl + 1)
    G = H.hetal_diag_atb(ctx, evk, D, Xl, c, lr_over_n, pts[2], flags)
    return G, (logits, P, D, Xl)


def nag_gammas(steps):
    """gamma_1 .. gamma_steps of NAG (Sec. 2.1): gamma_t = (1 - lambda_t) / lambda_{t+1},
    lambda_0 = 0, lambda_{t+1} = (1 + sqrt(1 + 4 lambda_t^2)) / 2."""
    lam = [0.0]
    for _ in range(steps + 1):
        lam.append((1.0 + (1.0 + 4.0 * lam[-1] ** 2) ** 0.5) / 2.0)
    return [(1.0 - lam[t]) / lam[t + 1] for t in range(1, steps + 1)]


def nag_train(ctx, evk, X, Wbar, Y, coeffs, valid, c, lr_over_n, target_scale, steps, Xval, flags=0,
              pts=(None, None, None, None)):
    """Protocol 1, step 3 with NAG (Sec. 2.1): `steps` updates
        W_{t+1} = V_t - (alpha/N) (P - Y)^T X,  P from the logits X V_t^T,
        V_{t+1} = W_{t+1} + gamma_t (W_t - W_{t+1}),  V_1 = W_1,
    each gradient moved to V's scale by a constant product by 1 (additions need equal
    scales); then the validation logits DiagABT(X_val, W, t = 1) with the last W (step 3(b)).
    Returns (W, V, logits); the caller frees them (Wbar itself is not freed)."""
    W = V = Wbar
    owned = []
    for gamma in nag_gammas(steps):
        G, inter = train_step(ctx, evk, X, V, Y, coeffs, valid, c, lr_over_n, target_scale, flags, pts[:3])
        for h in inter:
            H.hetal_mat_free(h)
        Gs = H.hetal_mul_const(ctx, G, 1.0, H.hetal_mat_desc_get(V).scale)
        H.hetal_mat_free(G)
        Wn = H.hetal_sub(ctx, V, Gs)
        H.hetal_mat_free(Gs)
        d = H.hetal_sub(ctx, W, Wn)
        gd = H.hetal_mul_const(ctx, d, gamma, H.hetal_mat_desc_get(Wn).scale)
        H.hetal_mat_free(d)
        Vn = H.hetal_add(ctx, Wn, gd)
        H.hetal_mat_free(gd)
        for h in owned:
            H.hetal_mat_free(h)
        W, V, owned = Wn, Vn, [Wn, Vn]
    logits = H.hetal_diag_abt(ctx, evk, Xval, W, c, 1.0, pts[3], flags)
    return W, V, logits


def replicate_stages(w):
    """Rotate-and-sum stages that copy one window of P slots to all w windows of a
    ciphertext (w a power of two): log2 w in stages of at most 3 bits, [(radix, stride in
    windows)]; a stage adds the radix - 1 right rotations by stride, 2 stride, ... windows."""
    e = int(round(math.log2(w)))
    if w < 1 or 1 << e != w:
        raise ValueError("the window count must be a power of two")
    stages, stride = [], 1
    while e > 0:
        b = min(3, e)
        stages.append((1 << b, stride))
        stride <<= b
        e -= b
    return stages


def replicate_rotations(P, w):
    """Rotation amounts (negative: right rotations) of the packed refresh's replication."""
    return sorted({-(j * stride * P) for radix, stride in replicate_stages(w) for j in range(1, radix)})


def train_boot_rotations(s0, s1, c, flags=0, boot_prm=None):
    """Every rotation nag_train_boot uses: the training step's, bootstrapping's and the
    packed refresh's (W-bar's rows repeat every c rows: windows of P = c s1 slots)."""
    from . import bootstrap as B
    N = 2 * s0 * s1
    return sorted(set(step_rotations(s0, s1, c, flags)) | set(B.rotations(N, boot_prm))
                  | set(replicate_rotations(c * s1, s0 // c)))


def _window(k, P, slots):
    v = np.zeros(slots)
    v[k * P:(k + 1) * P] = 1.0
    return v


def refresh_packed(ctx, evk, mats, P, w, target_scale, boot_prm=None, delta_w=2.0 ** 55, boot_pts=None,
                   boot_cache=None, bound=1.0):
    """Bootstrapping (Sec. 2.2) of matrices whose blocks' slots repeat with period P (w = slots
    / P periods; a vertically tiled W-bar has P = c s1, w = s0 / c), w blocks per
    bootstrapping instead of one:
      pack:    window t of the t-th block of a group of w (blocks in order over all matrices)
               into one ciphertext: one plaintext-product sum of window masks (one level),
               landing on target_scale;
      refresh: that ciphertext bootstrapped (bootstrap.bootstrap);
      unpack:  each block keeps its window (a window-mask product landing on exactly
               target_scale, one level), the blocks of each matrix are stacked again and every
               window is copied to all w windows by rotate-and-sum stages (replicate_stages).
    The matrices (blocks at one level >= 1 and one scale) come back as new handles with the
    same block grids, at bootstrapping's output level minus one and exactly target_scale.
    With bound (a power of two, |entries| <= bound) the pack masks are 1 / bound, so that
    bootstrapping sees messages in [-1, 1], and the bootstrapped ciphertext is read at its
    scale / bound; the plaintexts of bound 2^e != 1 are named "pack_e<e>" and "unpack_e<e>"."""
    from .circuit import Circuit
    C = Circuit(ctx, evk, delta_w, pts=boot_pts, cache=boot_cache)
    try:
        return _refresh_packed(C, mats, P, w, target_scale, boot_prm, delta_w, boot_pts, boot_cache, bound)
    finally:
        C.close()


def _refresh_packed(C, mats, P, w, target_scale, boot_prm, delta_w, boot_pts, boot_cache, bound):
    from . import bootstrap as B
    ctx, evk, slots = C.ctx, C.evk, C.slots
    e = int(math.ceil(math.log2(bound)))
    bound = 2.0 ** e
    names = ("pack", "unpack") if e == 0 else ("pack_e%d" % e, "unpack_e%d" % e)
    descs = [H.hetal_mat_desc_get(M) for M in mats]
    where = [(mi, j) for mi, d in enumerate(descs) for j in range(d.m * d.n)]
    pieces = [[None] * (d.m * d.n) for d in descs]
    outs = []
    try:
        for k0 in range(0, len(where), w):
            group = where[k0:k0 + w]
            sl = [C.wrap(H.hetal_mat_slice(ctx, mats[mi], j, 1)) for mi, j in group]
            packed = C.cmult_scaled_sum([(x, _window(t, P, slots) / bound, names[0], t) for t, x in enumerate(sl)],
                                        target_scale)
            del sl
            p0 = C.wrap(H.hetal_mat_drop(ctx, packed.h, 0))
            del packed
            r = C.wrap(B.bootstrap(ctx, evk, p0.h, p0.scale, delta_w, boot_prm, pts=boot_pts, cache=boot_cache))
            del p0
            if e:
                r = C.read_at(r, r.scale / bound)
            for t, (mi, j) in enumerate(group):
                pieces[mi][j] = C.cmult_scaled(r, _window(t, P, slots), names[1], t, target_scale).detach()
            del r
        for mi, d in enumerate(descs):
            M = H.hetal_mat_stack(ctx, pieces[mi], H.make_desc(d.m, d.n, d.rows, d.cols, d.s0, d.s1, 0, 0.0))
            for h in pieces[mi]:
                H.hetal_mat_free(h)
            pieces[mi] = []
            try:
                for radix, stride in replicate_stages(w):
                    M2 = H.hetal_rotate_sum(ctx, evk, M, [-(j * stride * P) for j in range(1, radix)])
                    H.hetal_mat_free(M)
                    M = M2
            except BaseException:
                H.hetal_mat_free(M)
                raise
            outs.append(M)
        return outs
    except BaseException:
        for h in outs:
            H.hetal_mat_free(h)
        raise
    finally:
        for row in pieces:
            for h in row:
                if h is not None:
                    H.hetal_mat_free(h)


def train_step_asoftmax(ctx, evk, X, Wbar, Y, c_real, c, valid, lr_over_n, target_scale, sm_delta, flags=0,
                        pts=(None, None, None), sm_prm=None, sm_pts=None, refresh=None, cache=None):
    """Protocol 1, step 3(a) with the paper's softmax (Algorithm ASoftmax, asoftmax.py) in place
    of the degree-15 stand-in, on a chain whose softmax runs on refreshes (refresh: a
    bootstrap.Refresher):
      logits = DiagABT(X, W-bar, t = 1), moved to the softmax's scale sm_delta (a constant
               product, one level);
      P      = ASoftmax(logits) over the c_real classes, refreshed if it has fewer than 6
               levels left, times the valid mask (rows and classes of the batch) landing on
               exactly sm_delta (one level);
      D      = P - Y (Y at sm_delta);
      G      = DiagATB(D, X at level(D) + 1, lr/N), then times the integer 2^k and read at
               2^k its scale, about target_scale (DiagATB leaves D's scale).
    evk holds the step's rotations, asoftmax.rotations(c_real, s1), bootstrapping's and the
    conjugation key.  sm_pts / cache: the softmax's plaintexts by name, device plaintexts
    reused across calls (circuit.Circuit).  Returns (G, intermediates) like train_step."""
    from . import asoftmax as A
    from .circuit import Circuit
    d = H.hetal_mat_desc_get(X)
    inter = []
    try:
        logits = H.hetal_diag_abt(ctx, evk, X, Wbar, c, 1.0, pts[0], flags)
        inter.append(logits)
        inter.append(H.hetal_mul_const(ctx, logits, 1.0, sm_delta))
        inter.append(A.asoftmax(ctx, evk, inter[-1], c_real, d.s0, d.s1, sm_delta, sm_prm, pts=sm_pts, cache=cache,
                                refresh=refresh))
        C = Circuit(ctx, evk, sm_delta, sm_pts, cache=cache, refresh=refresh)
        try:
            inter.append(_valid_output(C, inter[-1], valid, sm_delta))
        finally:
            C.close()
        D = H.hetal_sub(ctx, inter[-1], Y)
        inter.append(D)
        Xl = H.hetal_mat_drop(ctx, X, H.hetal_mat_desc_get(D).level + 1)
        inter.append(Xl)
        G = H.hetal_diag_atb(ctx, evk, D, Xl, c, lr_over_n, pts[2], flags)
        g = H.hetal_mat_desc_get(G)
        k = int(round(math.log2(target_scale / g.scale)))
        try:
            G2 = H.hetal_mul_int(ctx, G, 1 << k)
        finally:
            H.hetal_mat_free(G)
        try:
            return H.hetal_mat_set_scale(ctx, G2, g.scale * 2.0 ** k), tuple(inter)
        finally:
            H.hetal_mat_free(G2)
    except BaseException:
        for h in inter:
            H.hetal_mat_free(h)
        raise


def _valid_output(C, P, valid, sm_delta):
    Pk = C.keep(C.adopt(P), 5, 2.0)
    return C.cmult_scaled(Pk, valid, "valid", 0, sm_delta).detach()


def nag_train_boot(ctx, evk, X, Wbar, Y, coeffs, valid, c, lr_over_n, target_scale, steps, Xval, flags=0,
                   pts=(None, None, None, None), boot_prm=None, delta_w=2.0 ** 55, boot_pts=None,
                   boot_cache=None, on_iteration=None, grad=None):
    """nag_train for any number of iterations, W and V refreshed by bootstrapping after every
    update.  The update is written
        W_{t+1} = V_t - G,
        V_{t+1} = W_{t+1} + gamma (W_t - W_{t+1}) = (1 - gamma) V_t + gamma W_t - (1 - gamma) G,
    every term moved to target_scale by a constant product, so that W_{t+1} and V_{t+1} end
    one level above 0, at the same level and scale; both are then refreshed together by
    refresh_packed (W-bar's rows repeat every c rows), back to the level Wbar starts at (the
    training primes' top minus one, where X sits too, and Y eight levels below).  Wbar is at
    target_scale; evk holds train_boot_rotations and the conjugation key.  on_iteration(t), if
    given, is called after each iteration (e.g. to time it).  grad(V), if given, replaces the
    stand-in step (train_step) and returns (G at about target_scale, intermediates), e.g.
    train_step_asoftmax.  Returns (W, V, logits); the caller frees them (Wbar itself is not
    freed)."""
    S = target_scale
    d = H.hetal_mat_desc_get(Wbar)
    if d.scale != S:
        raise ValueError("W-bar must be at the target scale")
    P, w = c * d.s1, d.s0 // c
    W = V = Wbar
    owned = []
    for t, gamma in enumerate(nag_gammas(steps)):
        if grad is None:
            G, inter = train_step(ctx, evk, X, V, Y, coeffs, valid, c, lr_over_n, S, flags, pts[:3])
        else:
            G, inter = grad(V)
        for h in inter:
            H.hetal_mat_free(h)
        try:
            Wr, Vr = nag_update_refresh(ctx, evk, W, V, G, gamma, S, P, w, boot_prm, delta_w, boot_pts, boot_cache)
        finally:
            H.hetal_mat_free(G)
        for h in owned:
            H.hetal_mat_free(h)
        W, V, owned = Wr, Vr, [Wr, Vr]
        if on_iteration is not None:
            on_iteration(t)
    logits = H.hetal_diag_abt(ctx, evk, Xval, W, c, 1.0, pts[3], flags)
    return W, V, logits


def nag_update_refresh(ctx, evk, W, V, G, gamma, target_scale, P, w, boot_prm=None, delta_w=2.0 ** 55,
                       boot_pts=None, boot_cache=None, bound=1.0):
    """One NAG update (Sec. 2.1) from the gradient G (at about target_scale):
        W_{t+1} = V_t - G,  V_{t+1} = (1 - gamma) V_t + gamma W_t - (1 - gamma) G,
    every term moved to target_scale by a constant product, then W_{t+1} and V_{t+1} refreshed
    together (refresh_packed, windows of P slots, w per ciphertext, `bound` on their entries).
    Returns new handles (W_{t+1}, V_{t+1}); W, V and G are left as they are."""
    S = target_scale
    tmp = []
    try:
        tmp.append(H.hetal_mul_const(ctx, G, 1.0, S))
        tmp.append(H.hetal_sub(ctx, V, tmp[0]))                                      # W_{t+1}
        tmp += [H.hetal_mul_const(ctx, V, 1.0 - gamma, S), H.hetal_mul_const(ctx, W, gamma, S)]
        tmp.append(H.hetal_add(ctx, tmp[2], tmp[3]))
        tmp.append(H.hetal_mul_const(ctx, G, 1.0 - gamma, S))
        tmp.append(H.hetal_sub(ctx, tmp[4], tmp[5]))                                 # V_{t+1}
        return tuple(refresh_packed(ctx, evk, [tmp[1], tmp[6]], P, w, S, boot_prm, delta_w, boot_pts, boot_cache,
                                    bound))
    finally:
        for h in tmp:
            H.hetal_mat_free(h)


class ValidationClient:
    """The client's side of Protocol 1, step 3(c)-(d): it decrypts the validation logits with its
    secret key, computes the cross-entropy loss of the softmax over the c_real classes against
    its labels, and answers (stop, improved): improved when the loss is below every earlier
    epoch's, stop once it has not improved for `patience` epochs in a row.  The losses are kept
    in `losses`."""

    def __init__(self, ctx, sk, labels, c_real, patience=3):
        self.ctx, self.sk = ctx, sk
        self.labels = np.asarray(labels, dtype=np.int64)
        self.c_real, self.patience = c_real, patience
        self.best, self.bad, self.losses = math.inf, 0, []

    def loss(self, logits):
        z = logits[:, :self.c_real]
        z = z - z.max(axis=1, keepdims=True)
        logp = z - np.log(np.exp(z).sum(axis=1, keepdims=True))
        return float(-logp[np.arange(len(self.labels)), self.labels].mean())

    def __call__(self, logits_handle):
        L = H.hetal_decrypt(self.ctx, self.sk, logits_handle)[:len(self.labels)]
        loss = self.loss(L)
        self.losses.append(loss)
        improved = loss < self.best
        if improved:
            self.best, self.bad = loss, 0
        else:
            self.bad += 1
        return self.bad >= self.patience, improved


def train_epochs(ctx, evk, Wbar, grads, Xval, c, target_scale, max_epochs, client, flags=0, pts_val=None,
                 boot_prm=None, delta_w=2.0 ** 55, boot_pts=None, boot_cache=None, on_update=None, w_bound=1.0):
    """Protocol 1, step 3: for each epoch, one NAG update per mini-batch in order
    (nag_update_refresh; grads[b](V) returns batch b's gradient at about target_scale and its
    intermediates, e.g. a closure of train_step or train_step_asoftmax over (X_b, Y_b)), with
    gamma_t running on across batches and epochs; after each epoch the validation logits
    DiagABT(X_val, W, t = 1) go to client(logits) -> (stop, improved) (the client decrypts
    them: ValidationClient); the W of an improved epoch becomes the best weight W*.  Stops
    after max_epochs or when the client says so.  on_update(epoch, b), if given, is called
    after every update; w_bound bounds the entries of W and V for their refreshes.  Returns
    (W*, epochs run); the caller frees W* (Wbar is not freed)."""
    S = target_scale
    d = H.hetal_mat_desc_get(Wbar)
    if d.scale != S:
        raise ValueError("W-bar must be at the target scale")
    P, w = c * d.s1, d.s0 // c
    gammas = nag_gammas(max_epochs * len(grads))
    W = V = Wbar
    owned, best, t, epochs = [], None, 0, 0
    try:
        for epoch in range(max_epochs):
            for b, grad in enumerate(grads):
                G, inter = grad(V)
                for h in inter:
                    H.hetal_mat_free(h)
                try:
                    Wr, Vr = nag_update_refresh(ctx, evk, W, V, G, gammas[t], S, P, w, boot_prm, delta_w, boot_pts,
                                                boot_cache, w_bound)
                finally:
                    H.hetal_mat_free(G)
                for h in owned:
                    H.hetal_mat_free(h)
                W, V, owned, t = Wr, Vr, [Wr, Vr], t + 1
                if on_update is not None:
                    on_update(epoch, b)
            epochs = epoch + 1
            logits = H.hetal_diag_abt(ctx, evk, Xval, W, c, 1.0, pts_val, flags)
            try:
                stop, improved = client(logits)
            finally:
                H.hetal_mat_free(logits)
            if improved:
                if best is not None:
                    H.hetal_mat_free(best)
                best = H.hetal_mat_drop(ctx, W, H.hetal_mat_desc_get(W).level)   # a copy of W
            if stop:
                break
        if best is None:
            best = H.hetal_mat_drop(ctx, W, H.hetal_mat_desc_get(W).level)
        return best, epochs
    except BaseException:
        if best is not None:
            H.hetal_mat_free(best)
        raise
    finally:
        for h in owned:
            H.hetal_mat_free(h)
