"""One encrypted softmax-regression training step through the C ABI
(Protocol 1, step 3(a), without the NAG update):

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
