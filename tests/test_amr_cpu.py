"""Host logic of the hierarchy rebuild, no GPU: the library's Berger-Rigoutsos
clustering (host C++) returns the oracle's boxes, in the oracle's order, on
seeded flag patterns; the plans for general layouts agree with the
tensor-tiling plans where both apply; flux-correction parts at a concave
corner of the refined region come in separate waves in the oracle's order."""
import numpy as np
import pytest

from oracle import amr
from paper_1307_2265_gb300 import hierarchy as gh
from paper_1307_2265_gb300 import synth


def _pattern(seed):
    rng = np.random.default_rng(seed)
    shape = (int(rng.integers(1, 14)), int(rng.integers(1, 22)), int(rng.integers(1, 30)))
    F = np.zeros(shape, np.uint8)
    for _ in range(int(rng.integers(0, 6))):
        c = [int(rng.integers(0, s)) for s in shape]
        r = [int(rng.integers(1, 5)) for _ in shape]
        F[max(0, c[0] - r[0]):c[0] + r[0], max(0, c[1] - r[1]):c[1] + r[1], max(0, c[2] - r[2]):c[2] + r[2]] = 1
    F |= (rng.random(shape) < float(rng.choice([0.0, 0.005, 0.03]))).astype(np.uint8)
    return F


@pytest.mark.parametrize("seed", range(40))
def test_native_clustering_equals_the_oracle(seed):
    F = _pattern(seed)
    for eff, small, buf, mar in ((0.3, 64, 1, 0), (0.7, 8, 0, 1), (0.9, 1, 2, 0), (0.3, 8, 1, 3)):
        want = amr.cluster(F, efficiency=eff, small_cells=small, buffer=buf, margin=mar)
        got = gh.cluster_flags(F, efficiency=eff, small_cells=small, buffer=buf, margin=mar)
        assert got == [(tuple(lo), tuple(hi)) for lo, hi in want]


def test_native_clustering_grows_its_output_array():
    F = np.zeros((1, 1, 200), np.uint8)
    F[0, 0, ::4] = 1                                   # 50 isolated flags
    got = gh.cluster_flags(F, efficiency=1.0, small_cells=1, buffer=0)
    assert got == [(tuple(lo), tuple(hi)) for lo, hi in amr.cluster(F, efficiency=1.0, small_cells=1, buffer=0)]
    assert len(got) == 50


def test_general_plans_match_the_tensor_plans_on_static_layouts():
    layout = synth.hierarchy_layout(16, [(4, 12), (6, 10)], [4, 8], seed=2)
    for l in (1, 2):
        n, o = layout[l]["n"], layout[l]["origin"]
        a = gh.sibling_boxes(n, o)
        b = gh.sibling_boxes_general(n, o)
        assert sorted(map(bytes, a)) == sorted(map(bytes, b))
        a = gh.interp_boxes(n, o)
        b = gh.interp_boxes_general(n, o)
        assert sorted(map(bytes, a)) == sorted(map(bytes, b))
        fine = {"n": n, "origin": o}
        coarse = {"n": layout[l - 1]["n"], "origin": layout[l - 1]["origin"]}
        fc = gh.correction_faces(fine, coarse)
        parts, wave = gh.correction_parts(fine, coarse)
        assert np.array_equal(fc, parts) and not wave.any()


def test_correction_parts_order_concave_corners_in_waves():
    """An L of two fine patches over one coarse patch: the coarse cell in the
    inner corner lies outside a face of each, so the two parts touching it go
    to successive waves, the lower fine patch index first; a fine face whose
    outside spans two coarse patches is split into two parts."""
    coarse = {"n": np.array([[8, 8, 8], [8, 8, 8]]), "origin": np.array([[0, 0, 0], [8, 0, 0]])}
    # fine patches (in fine cells): A over coarse [2,4)x[2,6)x[2,4), B over [4,6)x[2,4)x[2,4)
    fine = {"n": np.array([[4, 8, 4], [4, 4, 4]]), "origin": np.array([[4, 4, 4], [8, 4, 4]])}
    parts, wave = gh.correction_parts(fine, coarse)
    corner = np.array([4, 4, 2])                    # outside A's +x face and B's +y face (coarse cell)
    touching = []
    for k, p in enumerate(parts):
        i, d, side = p["fine"], p["dir"], p["side"]
        fo, fn = fine["origin"][i] // 2, fine["n"][i] // 2
        a1 = 1 if d == 0 else 0
        a2 = 1 if d == 2 else 2
        lo, hi = fo.copy(), fo + fn
        lo[d] = fo[d] - 1 if side == 0 else fo[d] + fn[d]
        hi[d] = lo[d] + 1
        lo[a1], hi[a1] = fo[a1] + p["lo"][0], fo[a1] + p["hi"][0]
        lo[a2], hi[a2] = fo[a2] + p["lo"][1], fo[a2] + p["hi"][1]
        if np.all((lo <= corner) & (corner < hi)):
            touching.append(k)
    assert len(touching) == 2
    k0, k1 = touching
    assert parts[k0]["fine"] == 0 and parts[k1]["fine"] == 1
    assert wave[k1] > wave[k0]
    # B's +x face (coarse x = 6) lies in coarse patch 0 (x < 8); make a face cross two
    fine2 = {"n": np.array([[4, 4, 4]]), "origin": np.array([[10, 4, 4]])}     # coarse [5,7): +x face at 7
    coarse2 = {"n": np.array([[7, 8, 8], [9, 8, 8]]), "origin": np.array([[0, 0, 0], [7, 0, 0]])}
    p2, _ = gh.correction_parts(fine2, coarse2)
    xs = p2[(p2["dir"] == 0) & (p2["side"] == 1)]
    assert len(xs) == 1 and xs[0]["target"] == 1
    fine3 = {"n": np.array([[4, 8, 4]]), "origin": np.array([[4, 4, 4]])}       # coarse y in [2, 6)
    coarse3 = {"n": np.array([[8, 4, 8], [8, 4, 8]]), "origin": np.array([[0, 0, 0], [0, 4, 0]])}
    p3, _ = gh.correction_parts(fine3, coarse3)
    xs = p3[(p3["dir"] == 0) & (p3["side"] == 0)]
    assert sorted(xs["target"]) == [0, 1]                     # split at coarse y = 4
    assert sorted((int(a[0]), int(b[0])) for a, b in zip(xs["lo"], xs["hi"])) == [(0, 2), (2, 4)]


def test_register_sizes_count_components_per_face():
    """Flux-register sizes: every face bounding an active cell along each axis
    (all-face register) and the two end faces of each pencil (boundary
    register), times the components per face (5, or 6 with the gas energy)."""
    n = np.array([(3, 4, 5), (1, 1, 1), (16, 8, 2)])
    for nc in (5, 6):
        a, b = gh.register_sizes(n, nc)
        for i, (nx, ny, nz) in enumerate(n):
            assert a[i] == nc * ((nx + 1) * ny * nz + nx * (ny + 1) * nz + nx * ny * (nz + 1))
            assert b[i] == nc * 2 * (ny * nz + nx * nz + nx * ny)


def test_active_offsets_are_consecutive_blocks():
    import paper_1307_2265_gb300 as ez
    sizes = [(3, 4, 5), (1, 1, 1), (16, 8, 2)]
    t = ez.patch_table(sizes, [0, 1000, 2000], [0.1] * 3)
    assert list(ez.active_offsets(t)) == [0, 60, 61]


def test_hierarchy_driver_rejects_bad_layouts_before_any_cuda_call():
    import ctypes
    L = gh._lib()

    def create(levels, nf=5, dx=1.0 / 16):
        keep, lays = [], []
        for n, o, p in levels:
            n = np.ascontiguousarray(np.asarray(n, dtype=np.int32).reshape(-1, 3))
            o = np.ascontiguousarray(np.asarray(o, dtype=np.int32).reshape(-1, 3))
            p = np.ascontiguousarray(np.asarray(p, dtype=np.int32).reshape(-1))
            keep += [n, o, p]
            lays.append(gh._LevelLayout(len(n), n.ctypes.data, o.ctypes.data, p.ctypes.data))
        arr = (gh._LevelLayout * len(lays))(*lays)
        h = ctypes.c_void_p()
        return L.enzo_hierarchy_create(arr, len(lays), dx, nf, None, None, None, ctypes.byref(h))

    root = ([[16, 16, 16]], [[0, 0, 0]], [-1])
    assert create([root, ([[8, 8, 8]], [[12, 12, 12]], [1])]) == -1      # parent out of range
    assert create([root, ([[8, 8, 7]], [[12, 12, 12]], [0])]) == -1      # odd size below the root
    assert create([root, ([[8, 8, 8]], [[12, 12, 13]], [0])]) == -1      # odd origin
    assert create([([[16, 16, 16]], [[0, 0, 0]], [0])]) == -1             # a root with a parent
    assert create([root], nf=7) == -1
    assert create([([[8, 16, 16], [8, 16, 16]], [[0, 0, 0], [8, 0, 0]], [-1, -1])]) == -1   # a root of two grids
    assert create([root], dx=0.0) == -1
    # level 1 must stay 3 root cells inside a periodic root (no ghosts to interpolate from)
    assert create([root, ([[8, 8, 8]], [[2, 12, 12]], [0])]) == -3
    assert L.enzo_hierarchy_destroy(None) == -1


def _brute_plans(n, origin):
    """Level plans by their definitions, every patch against every other."""
    n, origin = np.asarray(n, dtype=np.int64), np.asarray(origin, dtype=np.int64)
    lo, hi = origin, origin + n
    sib, itp = [], []
    for a in range(len(n)):
        for b in range(len(n)):
            if b == a:
                continue
            blo, bhi = np.maximum(lo[a] - 3, lo[b]), np.minimum(hi[a] + 3, hi[b])
            if np.all(blo < bhi):
                sib.append((a, b, tuple(blo), tuple(bhi)))
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    if dx == dy == dz == 0:
                        continue
                    d = np.array([dx, dy, dz])
                    rlo = np.where(d < 0, lo[a] - 3, np.where(d > 0, hi[a], lo[a]))
                    rhi = np.where(d < 0, lo[a], np.where(d > 0, hi[a] + 3, hi[a]))
                    if not any(np.all((lo[b] <= rlo) & (rhi <= hi[b])) for b in range(len(n))):
                        itp.append((a, a, tuple(rlo), tuple(rhi)))
    return sib, itp


def _random_disjoint_layout(rng, count, extent=48):
    """Disjoint boxes of even sizes at even origins (a rebuilt level's shape)."""
    boxes = []
    occ = np.zeros((extent,) * 3, dtype=bool)
    tries = 0
    while len(boxes) < count and tries < 2000:
        tries += 1
        size = 2 * rng.integers(1, 5, size=3)
        o = 2 * rng.integers(0, (extent - size) // 2 + 1, size=3)
        sl = tuple(slice(int(o[d]), int(o[d] + size[d])) for d in range(3))
        if occ[sl[2], sl[1], sl[0]].any():
            continue
        occ[sl[2], sl[1], sl[0]] = True
        boxes.append((size, o))
    return np.array([b[0] for b in boxes]), np.array([b[1] for b in boxes])


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_native_level_plans_equal_their_definition_on_random_layouts(seed):
    """The library's bucket-indexed plans against every pair of patches: the
    same sibling copy boxes in the same (dst, src) order, the same regions to
    interpolate in the same (patch, direction) order."""
    rng = np.random.default_rng(seed)
    n, o = _random_disjoint_layout(rng, 40)
    want_sib, want_itp = _brute_plans(n, o)
    got_sib, got_itp = gh._level_plans(n, o)
    as_t = lambda t: [(int(r["dst"]), int(r["src"]), tuple(int(v) for v in r["lo"]), tuple(int(v) for v in r["hi"]))
                      for r in t]
    assert as_t(got_sib) == want_sib
    assert as_t(got_itp) == want_itp
    assert len(want_sib) > 0 and len(want_itp) > 0


def _brute_parts(fn, fo, cn, co):
    """Flux-correction parts and waves by their definition (every pair)."""
    fn, fo, cn, co = (np.asarray(a, dtype=np.int64) for a in (fn, fo, cn, co))
    flo, fhi = fo // 2, (fo + fn) // 2
    parts, cells = [], []
    for i in range(len(fn)):
        for d in range(3):
            a1, a2 = (1 if d == 0 else 0), (1 if d == 2 else 2)
            for side in (0, 1):
                X = (fo[i, d] + (fn[i, d] if side else 0)) // 2
                olo, ohi = flo[i].copy(), fhi[i].copy()
                olo[d], ohi[d] = (X - 1, X) if side == 0 else (X, X + 1)
                vol = int(np.prod(ohi - olo))
                cov = sum(int(np.prod(np.clip(np.minimum(ohi, fhi[j]) - np.maximum(olo, flo[j]), 0, None)))
                          for j in range(len(fn)))
                if cov >= vol:
                    continue
                for t in range(len(cn)):
                    tlo, thi = np.maximum(olo, co[t]), np.minimum(ohi, co[t] + cn[t])
                    if np.all(tlo < thi):
                        parts.append((i, d, side, t, (int(tlo[a1] - flo[i, a1]), int(tlo[a2] - flo[i, a2])),
                                      (int(thi[a1] - flo[i, a1]), int(thi[a2] - flo[i, a2]))))
                        cells.append((t, tlo, thi))
    wave = []
    for k in range(len(parts)):
        w = 0
        for q in range(k):
            if cells[q][0] == cells[k][0] and np.all(np.maximum(cells[k][1], cells[q][1]) <
                                                     np.minimum(cells[k][2], cells[q][2])):
                w = max(w, wave[q] + 1)
        wave.append(w)
    return parts, wave


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_native_correction_parts_equal_their_definition_on_random_layouts(seed):
    rng = np.random.default_rng(10 + seed)
    # coarse level: the 24^3 domain cut into slabs along x and y
    cx = sorted(set([0, 24] + list(rng.integers(4, 20, size=2))))
    cy = sorted(set([0, 24] + list(rng.integers(4, 20, size=1))))
    cn, co = [], []
    for x0, x1 in zip(cx[:-1], cx[1:]):
        for y0, y1 in zip(cy[:-1], cy[1:]):
            cn.append((x1 - x0, y1 - y0, 24))
            co.append((x0, y0, 0))
    fn, fo = _random_disjoint_layout(rng, 25, extent=48)
    want_parts, want_wave = _brute_parts(fn, fo, cn, co)
    parts, wave = gh.correction_parts({"n": fn, "origin": fo}, {"n": np.array(cn), "origin": np.array(co)})
    got = [(int(p["fine"]), int(p["dir"]), int(p["side"]), int(p["target"]), tuple(int(v) for v in p["lo"]),
            tuple(int(v) for v in p["hi"])) for p in parts]
    assert got == want_parts
    assert list(wave) == want_wave
    assert len(got) > 0
