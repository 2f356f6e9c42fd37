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
