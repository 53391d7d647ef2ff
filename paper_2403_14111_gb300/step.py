"""One encrypted softmax-regression training step through the C ABI (Protocol 1, step
3(a)), the NAG loop around it (step 3, Sec. 2.1), and the loop for any number of
iterations with W and V refreshed by bootstrapping (Sec. 2.2).  The step:

    logits/8 = DiagABT(<X>, <W-bar>, t = 1/8)          (Sec. 4.2.2)
    P        = p15(logits/8) (.) valid                  (degree-15 softmax stand-in)
    D        = P - <Y>
    G        = DiagATB(<D>, <X> at level(D)+1, t = lr/batch)   (Sec. 4.2.3, PRotUp branch)

Every operation is one C-ABI call; this module only sequences the calls.
"""
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


def refresh(ctx, evk, M, target_scale, boot_prm=None, delta_w=2.0 ** 55, boot_pts=None, boot_cache=None):
    """A matrix back to the training levels by bootstrapping (Sec. 2.2), on a chain whose
    upper primes hold exactly the bootstrapping: dropped to level 0, bootstrapped (read at
    its message's scale), then a constant product by 1 that lands on exactly target_scale
    (one level), so that every iteration starts from the same levels and scales.  Returns a
    new handle; M is kept."""
    from . import bootstrap as B
    M0 = H.hetal_mat_drop(ctx, M, 0)
    try:
        out = B.bootstrap(ctx, evk, M0, H.hetal_mat_desc_get(M0).scale, delta_w, boot_prm, pts=boot_pts,
                          cache=boot_cache)
    finally:
        H.hetal_mat_free(M0)
    try:
        return H.hetal_mul_const(ctx, out, 1.0, target_scale)
    finally:
        H.hetal_mat_free(out)


def nag_train_boot(ctx, evk, X, Wbar, Y, coeffs, valid, c, lr_over_n, target_scale, steps, Xval, flags=0,
                   pts=(None, None, None, None), boot_prm=None, delta_w=2.0 ** 55, boot_pts=None,
                   boot_cache=None, on_iteration=None):
    """nag_train for any number of iterations: after every update W and V are refreshed by
    bootstrapping (refresh) back to the level Wbar starts at (the training primes' top minus
    one, where X sits too, and Y eight levels below).  evk holds the training step's
    rotations, bootstrapping's (bootstrap.rotations) and the conjugation key.  on_iteration(t), if given, is called after each iteration (e.g.
    to time it).  Returns (W, V, logits); the caller frees them (Wbar itself is not freed)."""
    W = V = Wbar
    owned = []
    for t, gamma in enumerate(nag_gammas(steps)):
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
        Wr = refresh(ctx, evk, Wn, target_scale, boot_prm, delta_w, boot_pts, boot_cache)
        Vr = refresh(ctx, evk, Vn, target_scale, boot_prm, delta_w, boot_pts, boot_cache)
        H.hetal_mat_free(Wn)
        H.hetal_mat_free(Vn)
        W, V, owned = Wr, Vr, [Wr, Vr]
        if on_iteration is not None:
            on_iteration(t)
    logits = H.hetal_diag_abt(ctx, evk, Xval, W, c, 1.0, pts[3], flags)
    return W, V, logits
