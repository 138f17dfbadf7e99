"""The autotuner (ed_autotune, ed_autotune_index): every candidate variant is
one of the product paths the parity tests check against the oracle; here the
tuned product must equal the forced variant bit for bit, stay within the
single-precision bar of the default product, be no slower than the default,
and the choice must reach the tuning file and later basis builds."""
import os

import numpy as np
import pytest

import ed_inputs as ei
from gpu_util import gpu

pytestmark = pytest.mark.gpu

POLICY = {1: "rowwise", 2: "term_parallel"}


@pytest.fixture
def clean_tuning():
    torch, ed = gpu()
    ed.tune_reset()
    yield
    ed.tune_reset()
    ed.kernel_policy("auto")
    ed.force_all_rotations(False)


@pytest.mark.parametrize("nvec,dt", [(1, "float32"), (8, "float32"), (1, "float64")])
def test_autotune_product(clean_tuning, tmp_path, nvec, dt):
    torch, ed = gpu()
    os.environ["ED_TUNE_FILE"] = str(tmp_path / "tune.txt")
    try:
        w = ei.workload("ring32")
        O = ed.operator_create(32, w["op"]["sites"], w["op"]["coeff"], w["op"]["local"])
        B = ed.basis_build(32, 16, +1, w["perms"], w["chars"])
        st, _ = ed.basis_states(B)
        x = ei.x_by_state_torch_chunked(3, st, nvec, False, dtype=getattr(torch, dt))
        y_def, y_tuned, y_forced = torch.empty_like(x), torch.empty_like(x), torch.empty_like(x)
        ed.matvec(O, B, x, y_def, nvec)
        r = ed.autotune(O, B, x, torch.empty_like(x), nvec)
        assert r["variants_timed"] >= 2 and r["ms_best"] <= r["ms_default"]
        ed.matvec(O, B, x, y_tuned, nvec)
        # the same variant forced through the test hooks gives the same bits
        if r["kernel"] in POLICY:
            ed.kernel_policy(POLICY[r["kernel"]])
        ed.force_all_rotations(r["search"] == 0)
        ed.matvec(O, B, x, y_forced, nvec)
        assert torch.equal(y_tuned, y_forced)
        tol = 2e-6 if dt == "float32" else 1e-13
        assert float((y_tuned - y_def).abs().max()) <= tol * float(y_def.abs().max())
        lines = (tmp_path / "tune.txt").read_text().split("\n")
        assert any(l.startswith("P ") and f" 32 128 1 22 {nvec} " in l for l in lines), lines
    finally:
        del os.environ["ED_TUNE_FILE"]


def test_autotune_index_reaches_later_builds(clean_tuning):
    torch, ed = gpu()
    w = ei.workload("ring32")
    O = ed.operator_create(32, w["op"]["sites"], w["op"]["coeff"], w["op"]["local"])
    r = ed.autotune_index(O, 32, 16, +1, w["perms"], w["chars"], 1, ed.ED_F32)
    assert r["index"] in (1, 2) and r["ms_best"] > 0
    B = ed.basis_build(32, 16, +1, w["perms"], w["chars"])
    assert ed.basis_bucket(B)[0] == (r["index"] == 2)
    assert ed.basis_hash(B)[0] == (r["index"] == 1)
