"""Packed active-cell layout on the GPU (enzo_pack_active / enzo_unpack_active):
on a ragged batch (1-cell axes, patches of one to several fill tiles, with and
without the periodic flag) the
packed arrays hold each patch's active cells x fastest in its block, with the
gas energy when asked; unpacking writes exactly the active cells back and
leaves the ghost zones untouched.  Pure data movement: bit-exact."""
import numpy as np
import pytest
import torch

import paper_1307_2265_gb300 as ez
from gpu_helpers import active, white_patch

pytestmark = pytest.mark.gpu
SIZES = [(1, 1, 1), (7, 1, 3), (16, 9, 5), (33, 20, 17), (1, 40, 2), (64, 8, 8)]


def _batch(seed=0, flags=0):
    patches = [white_patch(n, seed + i) for i, n in enumerate(SIZES)]
    ges = [np.random.default_rng(50 + i).normal(size=U[0].shape) for i, U in enumerate(patches)]
    offs = np.concatenate([[0], np.cumsum([U[0].size for U in patches])[:-1]])
    table = ez.patch_table([(n[0], n[1], n[2]) for n in SIZES], offs, [0.1] * 3, flags=flags)
    flat = [np.concatenate([U[f].ravel() for U in patches]) for f in range(5)]
    b = ez.PatchBatch(table, flat, ge=np.concatenate([g.ravel() for g in ges]))
    return b, patches, ges


@pytest.mark.parametrize("flags", [0, ez.PATCH_PERIODIC])
@pytest.mark.parametrize("with_ge", [False, True])
def test_pack_then_unpack_round_trip(with_ge, flags):
    b, patches, ges = _batch(flags=flags)
    act_off_h = ez.active_offsets(b.table)
    cells = int(sum(np.prod(n) for n in SIZES))
    act_off = torch.from_numpy(act_off_h).to(b.device)
    packed = [torch.full((cells,), np.nan, dtype=torch.float64, device=b.device) for _ in range(5)]
    pge = torch.full((cells,), np.nan, dtype=torch.float64, device=b.device) if with_ge else None
    ez.pack_active(b, packed, act_off, pge)
    torch.cuda.synchronize()
    got = [p.cpu().numpy() for p in packed]
    for i, U in enumerate(patches):
        o, c = act_off_h[i], int(np.prod(SIZES[i]))
        for f in range(5):
            assert np.array_equal(got[f][o:o + c], active(U[f]).ravel()), (i, f)
        if with_ge:
            assert np.array_equal(pge.cpu().numpy()[o:o + c], active(ges[i]).ravel()), i
    # unpack into a batch whose cells hold a sentinel: the active cells come
    # back, the ghosts keep the sentinel
    for u in b.U:
        u.fill_(-7.0)
    b.ge.fill_(-7.0)
    ez.unpack_active(b, packed, act_off, pge)
    torch.cuda.synchronize()
    for i, U in enumerate(patches):
        views = [f.cpu().numpy() for f in b.patch_fields(i)] + [b.patch_ge(i).cpu().numpy()]
        for f in range(6):
            want = (ges[i] if f == 5 else U[f]) if (f < 5 or with_ge) else None
            a = views[f]
            ghost = np.ones(a.shape, dtype=bool)
            ghost[3:-3, 3:-3, 3:-3] = False
            assert np.all(a[ghost] == -7.0), (i, f)
            if want is None:
                assert np.all(active(a) == -7.0), (i, f)
            else:
                assert np.array_equal(active(a), active(want)), (i, f)


def test_pack_needs_five_packed_arrays():
    b, _, _ = _batch()
    act_off = torch.zeros(len(SIZES), dtype=torch.int64, device=b.device)
    packed = [torch.zeros(1, dtype=torch.float64, device=b.device) for _ in range(4)]
    with pytest.raises(ValueError):
        ez.pack_active(b, packed, act_off)
