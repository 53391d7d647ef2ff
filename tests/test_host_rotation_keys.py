"""Host logic without a GPU: the rotation amounts the library asks keys for
(hetal_rotation_amounts) are exactly the rotations that DiagABT and both
branches of DiagATB perform, for every algorithm variant.  The amounts actually
used are collected from the oracle's FP64 slot simulator running the algorithms."""
import numpy as np
import pytest

import paper_2403_14111_gb300.hetal as H
from oracle import matmul as mm

SLOTS = 32768


class RecordingSlotOps(mm.SlotOps):
    """The slot simulator, noting every left-rotation amount (mod the slot count)."""

    def __init__(self, *a, **k):
        super().__init__(*a, **k)
        self.used = set()

    def rot(self, a, r):
        if r % self.s:
            self.used.add(r % self.s)
        return super().rot(a, r)

    def rot_many(self, a, rs):
        self.used |= {r % self.s for r in rs if r % self.s}
        return super().rot_many(a, rs)

    def rot_sum(self, a, rs):
        self.used |= {r % self.s for r in rs if r % self.s}
        return super().rot_sum(a, rs)


def _sim_mat(M, s0, s1, lv):
    return mm.EncMat([[mm.SV(b.astype(np.complex128), lv) for b in row] for row in mm.block_split(M, s0, s1)],
                     M.shape[0], M.shape[1], s0, s1)


def used_amounts(a, b, c, s0, flags):
    s1 = SLOTS // s0
    rng = np.random.default_rng(0)
    kw = dict(hoist=bool(flags & H.FLAG_HOIST), lazy_relin=bool(flags & H.FLAG_LAZY_RELIN),
              radix_sum=bool(flags & H.FLAG_RADIX_SUM), shared_rot=bool(flags & H.FLAG_SHARED_ROT))
    used = set()
    ops = RecordingSlotOps(SLOTS, **kw)
    A, W = rng.uniform(-1, 1, (a, b)), rng.uniform(-1, 1, (c, b))
    mm.diag_abt(ops, _sim_mat(A, s0, s1, 12), _sim_mat(mm.tile_vertical(W, c, s0), s0, s1, 12), c, 1.0)
    used |= ops.used
    P = rng.uniform(-1, 1, (a, c))
    for lvA in (12, 11):   # RotLeft branch, PRotUp branch
        ops = RecordingSlotOps(SLOTS, **kw)
        mm.diag_atb(ops, _sim_mat(mm.tile_horizontal(P, c, s1), s0, s1, lvA), _sim_mat(A, s0, s1, 12), c, 1.0)
        used |= ops.used
    return used


FLAGS = [0, H.FLAG_HOIST | H.FLAG_LAZY_RELIN, H.FLAG_RADIX_SUM, H.FLAG_SHARED_ROT,
         H.FLAG_HOIST | H.FLAG_LAZY_RELIN | H.FLAG_RADIX_SUM | H.FLAG_SHARED_ROT]


@pytest.mark.parametrize("flags", FLAGS)
@pytest.mark.parametrize("a,b,c,s0", [(300, 100, 8, 128), (1024, 64, 16, 1024), (64, 96, 4, 64)])
def test_rotation_keys_are_the_algorithms_rotations(a, b, c, s0, flags):
    s1 = SLOTS // s0
    keys = set(H.hetal_rotation_amounts(s0, s1, c, flags))
    assert all(0 < r < SLOTS for r in keys)
    used = used_amounts(a, b, c, s0, flags)
    missing, unused = sorted(used - keys), sorted(keys - used)
    assert not missing, "no key for rotations %s" % missing[:8]
    assert not unused, "keys no algorithm uses: %s" % unused[:8]


def test_rotation_amounts_rejects_bad_shapes():
    assert H.lib().hetal_rotation_amounts(128, 32, 3, 0, None, 0) == H.ERR_SHAPE      # c not a power of two
    assert H.lib().hetal_rotation_amounts(128, 32, 64, 0, None, 0) == H.ERR_SHAPE     # c > s1
    assert H.lib().hetal_rotation_amounts(96, 32, 4, 0, None, 0) == H.ERR_SHAPE       # s0 not a power of two
