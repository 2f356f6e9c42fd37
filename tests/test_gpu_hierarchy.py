"""GPU parity of the static hierarchy (ghost fill from parents and siblings,
flux registers, flux correction, projection, subcycled W-cycle) against the
FP64 reference in oracle/hierarchy.py, and conservation of the composite grid."""
import numpy as np
import pytest

import oracle
import paper_1307_2265_gb300 as ez
from oracle import hierarchy as H
from paper_1307_2265_gb300 import hierarchy as gh
from paper_1307_2265_gb300 import synth

pytestmark = pytest.mark.gpu


def _setup(seed=0):
    layout = synth.hierarchy_layout(16, [(4, 12), (6, 10)], [4, 8], seed=seed)
    fields = synth.hierarchy_fields(layout, config=5)
    return layout, fields


def test_fp64_root_steps_match_oracle_bitwise():
    layout, fields = _setup(1)
    ref = H.make_levels(layout, fields, 1.0 / 16)
    hier = gh.Hierarchy(layout, fields, 1.0 / 16)
    P = oracle.Params()
    params = ez.Params(precision=ez.FP64)
    for _ in range(2):
        log_o, log_g = [], []
        H.root_step(ref, P, log=log_o)
        hier.root_step(params, log=log_g)
        assert log_g == log_o
    hier.stream.synchronize()
    for l, L in enumerate(ref):
        for i, p in enumerate(L["patches"]):
            g = hier.patch_fields(l, i)
            for a, b in zip(g, p["U"]):
                assert np.array_equal(H._active(a), H._active(b)), (l, i)


def _composite(hier):
    levels = []
    for l, lev in enumerate(hier.levels):
        patches = []
        for i in range(len(lev["n"])):
            patches.append({"n": tuple(int(v) for v in lev["n"][i]),
                            "origin": tuple(int(v) for v in lev["origin"][i]),
                            "parent": int(lev["table"]["level"][i] * 0 + (-1 if l == 0 else 0)),
                            "U": hier.patch_fields(l, i)})
        levels.append({"patches": patches, "dx": lev["dx"]})
    return levels


@pytest.mark.parametrize("precision", [ez.FP64, ez.FP32])
def test_composite_conservation_gpu(precision):
    layout, fields = _setup(2)
    hier = gh.Hierarchy(layout, fields, 1.0 / 16)

    def totals():
        lv = []
        for l, lev in enumerate(hier.levels):
            lv.append({"patches": [{"n": tuple(int(v) for v in lev["n"][i]),
                                    "origin": tuple(int(v) for v in lev["origin"][i]),
                                    "parent": int(layout[l]["parent"][i]),
                                    "U": hier.patch_fields(l, i)} for i in range(len(lev["n"]))],
                       "dx": lev["dx"]})
        t = H.composite_totals(lv)
        for L in lv:
            for p in L["patches"]:
                p["U"] = [np.abs(f) for f in p["U"]]
        return t, H.composite_totals(lv)

    t0, _ = totals()
    for _ in range(2):
        hier.root_step(ez.Params(precision=precision))
    hier.stream.synchronize()
    t1, scale = totals()
    assert np.all(np.abs(t1 - t0) <= 1e-13 * scale), (t1 - t0) / scale


def _l1_by_level(a_levels, b_levels):
    """Per level, per field: sum |a - b| / sum |b| over the active cells."""
    out = []
    for A, B in zip(a_levels, b_levels):
        num, den = np.zeros(5), np.zeros(5)
        for pa, pb in zip(A, B):
            for f in range(5):
                num[f] += np.sum(np.abs(H._active(pa[f]) - H._active(pb[f])))
                den[f] += np.sum(np.abs(H._active(pb[f])))
        out.append(num / den)
    return np.array(out)


@pytest.fixture(scope="module")
def fp64_reference():
    """Two FP64 oracle runs of two root steps: the reference, and one whose
    initial fields carry 2^-24 relative noise (the flow's own sensitivity to
    rounding-sized changes, the chaotic floor of the FP32 rule)."""
    layout, fields = _setup(3)
    P = oracle.Params()
    ref = H.make_levels(layout, fields, 1.0 / 16)
    rng = np.random.default_rng(9)
    noisy = [[[f * (1.0 + 2.0 ** -24 * rng.standard_normal(f.shape)) for f in U] for U in lev] for lev in fields]
    pert = H.make_levels(layout, noisy, 1.0 / 16)
    logs = []
    for _ in range(2):
        log = []
        H.root_step(ref, P, log=log)
        H.root_step(pert, P)
        logs.append(log)
    r = [[p["U"] for p in L["patches"]] for L in ref]
    q = [[p["U"] for p in L["patches"]] for L in pert]
    return layout, fields, r, logs, _l1_by_level(q, r)


@pytest.mark.parametrize("learned", [False, True])
def test_fp32_root_steps_close_to_oracle(fp64_reference, learned):
    """The FP32 path (plain, or with the learned guess at every interface) over
    two subcycled root steps of a white-noise hierarchy: the same substeps as
    the FP64 oracle, and a per-level, per-field L1 relative error within
    max(4 x chaotic floor, 2e-6), the FP32 parity rule of the single-grid tests."""
    layout, fields, ref, logs, floor = fp64_reference
    hier = gh.Hierarchy(layout, fields, 1.0 / 16)
    net = ez.MLP(seed=2)
    params = (ez.Params(precision=ez.FP32, guess=ez.GUESS_MLP, mlp=net.blob, mlp_gate=-1.0) if learned
              else ez.Params(precision=ez.FP32))
    for log_o in logs:
        log_g = []
        hier.root_step(params, log=log_g)
        assert [l for l, _ in log_g] == [l for l, _ in log_o]
        assert np.allclose([d for _, d in log_g], [d for _, d in log_o], rtol=1e-5)
    hier.stream.synchronize()
    got = [[hier.patch_fields(l, i) for i in range(len(L))] for l, L in enumerate(ref)]
    err = _l1_by_level(got, ref)
    bound = np.maximum(4.0 * floor, 2e-6)
    print(f"\nFP32{' learned' if learned else ''} hierarchy L1 by level:\n{err}\nchaotic floor:\n{floor}")
    assert np.all(err <= bound), (err, floor)
    st = sum(np.array(list(lev["batch"].read_status().values())) for lev in hier.levels)
    assert st[7] == 0                                   # no NaN anywhere


def test_full_size_hierarchy_keeps_a_uniform_moving_state():
    """The bench's hierarchy (256^3 root, 29 491 patches on three refined
    levels) with a uniform state moving obliquely: one subcycled FP32 root step
    with the learned guess (ghost interpolation, sibling copies, sweeps, flux
    correction and projection) keeps it to FP32 rounding of the increments."""
    import torch
    root = 256
    layout = synth.hierarchy_layout(root, [(root // 8, 7 * root // 8), (root // 4, 3 * root // 4),
                                           (3 * root // 8, 5 * root // 8)], list(range(16, 33, 2)), seed=0)
    g = 5.0 / 3.0
    state = synth.prims_to_conserved(np.ones(1), np.full(1, 0.3), np.full(1, -0.2), np.full(1, 0.1), np.ones(1), g)
    fields = []
    for L in layout:
        lev = []
        for n in L["n"]:
            shape = (int(n[2]) + 6, int(n[1]) + 6, int(n[0]) + 6)
            lev.append([np.full(shape, float(v[0])) for v in state])
        fields.append(lev)
    hier = gh.Hierarchy(layout, fields, 1.0 / root)
    net = ez.MLP(seed=4)
    log = []
    hier.root_step(ez.Params(gamma=g, precision=ez.FP32, guess=ez.GUESS_MLP, mlp=net.blob, mlp_gate=-1.0), log=log)
    hier.stream.synchronize()
    assert [sum(1 for l, _ in log if l == k) for k in range(4)][0] == 1
    for lev in hier.levels:
        for u, v in zip(lev["batch"].U, state):
            dev = float(torch.max(torch.abs(u - float(v[0]))))
            assert dev <= 1e-6 * max(1.0, abs(float(v[0]))), dev


def _uncovered_masks(hier):
    """Per level, a device bool mask over the flat field storage: active cells
    that no finer patch covers (the composite grid)."""
    import torch
    out = []
    for l, lev in enumerate(hier.levels):
        table = lev["table"]
        m = np.zeros(int(lev["batch"].field_len), dtype=bool)
        kids = {}
        if l + 1 < len(hier.levels):
            fine = hier.levels[l + 1]
            for j, p in enumerate(fine["parent"]):
                kids.setdefault(int(p), []).append(j)
        for i in range(len(lev["n"])):
            nx, ny, nz = (int(v) for v in lev["n"][i])
            blk = np.zeros((nz + 6, ny + 6, nx + 6), dtype=bool)
            blk[3:-3, 3:-3, 3:-3] = True
            for j in kids.get(i, []):
                fo = hier.levels[l + 1]["origin"][j] // 2 - lev["origin"][i] + 3
                fn = hier.levels[l + 1]["n"][j] // 2
                blk[fo[2]:fo[2] + fn[2], fo[1]:fo[1] + fn[1], fo[0]:fo[0] + fn[0]] = False
            off = int(table["off"][i])
            m[off:off + blk.size] = blk.ravel()
        out.append(torch.from_numpy(m).to(lev["batch"].device))
    return out


def _device_totals(hier, masks):
    import torch
    t = np.zeros(5)
    s = np.zeros(5)
    for lev, m in zip(hier.levels, masks):
        vol = lev["dx"] ** 3
        for f, u in enumerate(lev["batch"].U):
            t[f] += vol * float(torch.sum(u[m]))
            s[f] += vol * float(torch.sum(torch.abs(u[m])))
    return t, s


def test_full_size_hierarchy_conserves_the_composite_totals():
    """The bench's hierarchy (256^3 root, 29 491 patches on three refined
    levels) with its white-noise state: one subcycled FP32 root step with the
    learned guess keeps mass, momentum and energy of the composite grid to
    1e-13 of the summed magnitudes (flux correction cancels each coarse
    increment at a fine face exactly; the sums run on the device in FP64)."""
    root = 256
    layout = synth.hierarchy_layout(root, [(root // 8, 7 * root // 8), (root // 4, 3 * root // 4),
                                           (3 * root // 8, 5 * root // 8)], list(range(16, 33, 2)), seed=0)
    fields = synth.hierarchy_fields(layout, config=5)
    hier = gh.Hierarchy(layout, fields, 1.0 / root)
    del fields
    masks = _uncovered_masks(hier)
    t0, scale = _device_totals(hier, masks)
    net = ez.MLP(seed=4)
    log = []
    hier.root_step(ez.Params(precision=ez.FP32, guess=ez.GUESS_MLP, mlp=net.blob), log=log)
    hier.stream.synchronize()
    assert [sum(1 for l, _ in log if l == k) for k in range(4)][0] == 1 and len(log) > 4
    t1, _ = _device_totals(hier, masks)
    assert np.all(np.abs(t1 - t0) <= 1e-13 * scale), (t1 - t0) / scale
    st = sum(np.array(list(lev["batch"].read_status().values())) for lev in hier.levels)
    assert st[7] == 0                                   # no NaN anywhere


def test_c_caller_runs_the_w_cycle_on_its_own():
    """The driver's C entry points as a C caller uses them: device memory from
    cudaMalloc (no allocator), the active cells loaded with enzo_unpack_active
    (ghost zones start at zero: the W-cycle fills them before any read), two
    FP32 root steps.  The step log and every active cell equal those of the
    Python wrapper, which uploads whole ghost-zoned patches."""
    import ctypes
    import torch
    layout, fields = _setup(3)
    params = ez.Params(precision=ez.FP32)
    hier = gh.Hierarchy(layout, fields, 1.0 / 16)
    L = gh._lib()
    keep, lays = [], []
    for Lv in layout:
        n = np.ascontiguousarray(np.asarray(Lv["n"], dtype=np.int32).reshape(-1, 3))
        o = np.ascontiguousarray(np.asarray(Lv["origin"], dtype=np.int32).reshape(-1, 3))
        par = np.ascontiguousarray(np.asarray(Lv["parent"], dtype=np.int32).reshape(-1))
        keep += [n, o, par]
        lays.append(gh._LevelLayout(len(n), n.ctypes.data, o.ctypes.data, par.ctypes.data))
    arr = (gh._LevelLayout * len(lays))(*lays)
    stream = torch.cuda.Stream()
    h = ctypes.c_void_p()
    assert L.enzo_hierarchy_create(arr, len(lays), 1.0 / 16, 5, None, stream.cuda_stream, None,
                                   ctypes.byref(h)) == 0
    try:
        def level(l):
            info = gh._LevelInfo()
            assert L.enzo_hierarchy_level(h, l, ctypes.byref(info)) == 0
            table = gh._host_array(info.table, ez.PATCH_DTYPE, int(info.batch.npatch))
            return info, torch.from_numpy(ez.active_offsets(table)).cuda()

        for l, Lv in enumerate(layout):
            info, act = level(l)
            packed = [torch.from_numpy(np.concatenate([H._active(np.asarray(fields[l][i][f])).ravel()
                                                       for i in range(len(fields[l]))])).cuda() for f in range(5)]
            torch.cuda.synchronize()
            ptrs = (ctypes.c_void_p * 5)(*[t.data_ptr() for t in packed])
            assert L.enzo_unpack_active(ctypes.byref(info.batch), ptrs, None, act.data_ptr()) == 0
        p, c = params.c(), ez.Params(precision=ez.FP32).c()
        for _ in range(2):
            log_w = []
            hier.root_step(params, log=log_w)
            dt0 = ctypes.c_double(0.0)
            assert L.enzo_hierarchy_root_step(h, ctypes.byref(p), ctypes.byref(c), None, ctypes.byref(dt0)) == 0
            lv, dts, cnt = (ctypes.c_int32 * 256)(), (ctypes.c_double * 256)(), ctypes.c_int32(0)
            assert L.enzo_hierarchy_take_log(h, lv, dts, 256, ctypes.byref(cnt)) == 0
            assert [(int(lv[k]), float(dts[k])) for k in range(cnt.value)] == log_w
        hier.stream.synchronize()
        for l in range(len(layout)):
            info, act = level(l)
            cells = int(info.cells)
            out = [torch.empty(cells, dtype=torch.float64, device="cuda") for _ in range(5)]
            ptrs = (ctypes.c_void_p * 5)(*[t.data_ptr() for t in out])
            assert L.enzo_pack_active(ctypes.byref(info.batch), ptrs, None, act.data_ptr()) == 0
            stream.synchronize()
            want = [np.concatenate([H._active(hier.patch_fields(l, i)[f]).ravel()
                                    for i in range(len(layout[l]["n"]))]) for f in range(5)]
            for f in range(5):
                assert np.array_equal(out[f].cpu().numpy(), want[f]), (l, f)
        cu = ctypes.c_int64(0)
        assert L.enzo_hierarchy_timing(h, -1, None, ctypes.byref(cu)) == 0
        assert cu.value == hier.cell_updates
    finally:
        assert L.enzo_hierarchy_destroy(h) == 0
