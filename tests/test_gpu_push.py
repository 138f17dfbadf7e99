"""The transposed (push) form of the product -- every term of H|r> added to y
at the index of its representative with an atomic add, the paper's distributed
product on one GPU -- kept as an ablation of the pull form.  Checked against
the oracle with the pull form's bars (fp64 1e-12, fp32 2e-6 of max|y|); its
results are not bit-reproducible (the order of the atomic adds varies), which
is measured here, not asserted away."""
import numpy as np
import pytest

import ed_inputs as ei
import oracle
from gpu_util import gpu, rel_err, to_torch
from test_gpu_parity import SECTORS, make

pytestmark = pytest.mark.gpu

EXCHANGE = [s for s in SECTORS if not s[0].startswith("ring10_noU1_xx")]


@pytest.mark.parametrize("case", EXCHANGE, ids=[s[0] for s in EXCHANGE])
def test_push_matches_oracle(case):
    torch, ed = gpu()
    S = make(case)
    if S["dim"] == 0:
        pytest.skip("empty sector")
    cplx = not ed.basis_is_real(S["B"])
    x = ei.x_by_index(17, S["dim"], 1, cplx)
    want = oracle.matvec(S["G"], S["H"], S["st"], S["nm"], x)[:, 0]
    for dt, tol in (((np.complex128 if cplx else np.float64), 1e-12), ((np.complex64 if cplx else np.float32), 2e-6)):
        xt = to_torch(x[:, 0], dt)
        yt = torch.full_like(xt, float("nan"))
        ed.matvec_push(S["O"], S["B"], xt, yt)
        got = yt.cpu().numpy().astype(np.complex128)
        assert rel_err(got, want if cplx else want.real) < tol


def test_push_full_size_ring32_against_pull():
    """N=32 ring: push and pull agree to rounding; repeated pushes agree to
    rounding (bitwise equality is not guaranteed and not required)."""
    torch, ed = gpu()
    w = ei.workload("ring32")
    B = ed.basis_build(32, 16, +1, w["perms"], w["chars"])
    O = ed.operator_create(32, w["op"]["sites"], w["op"]["coeff"], w["op"]["local"])
    st, _ = ed.basis_states(B)
    for dt, tol in ((torch.float64, 1e-13), (torch.float32, 2e-6)):
        x = ei.x_by_state_torch(3, st, 1, False, dtype=dt).reshape(-1).contiguous()
        y_pull, y_a, y_b = torch.empty_like(x), torch.empty_like(x), torch.empty_like(x)
        ed.matvec(O, B, x, y_pull, 1)
        ed.matvec_push(O, B, x, y_a)
        ed.matvec_push(O, B, x, y_b)
        scale = float(y_pull.abs().max())
        assert float((y_a - y_pull).abs().max()) <= tol * scale
        assert float((y_a - y_b).abs().max()) <= tol * scale


def test_push_rejects_general_two_site_terms():
    torch, ed = gpu()
    case = [s for s in SECTORS if s[0].startswith("ring10_noU1_xx")][0]
    S = make(case, with_oracle=False)
    x = torch.ones(S["dim"], dtype=torch.float64, device="cuda")
    with pytest.raises(ed.EDError):
        ed.matvec_push(S["O"], S["B"], x, torch.empty_like(x))
