"""ed_matvec_multi (many sectors, one launch) against ed_matvec sector by
sector: results must be bit-identical (same arithmetic in the same order)."""
import numpy as np
import pytest

import ed_inputs as ei
from gpu_util import gpu

pytestmark = pytest.mark.gpu


def xxz_sectors(n):
    out = []
    for sz in range(3):
        for k in range(n):
            for z in ((1, -1) if sz == 0 else (0,)):
                p, c = ei.ring_group(n, k)
                out.append((n // 2 + sz, z, p, c))
    return out


@pytest.mark.parametrize("nvec", [1, 3, 8])
@pytest.mark.parametrize("dt", ["complex128", "complex64"])
def test_multi_equals_single(nvec, dt):
    torch, ed = gpu()
    n = 14
    op = ei.xxz_ring(n, 1.0, 1.5)
    O = ed.operator_create(n, op["sites"], op["coeff"], op["local"])
    dtype = getattr(torch, dt)
    items, bases = [], []
    for n_up, z, p, c in xxz_sectors(n):
        B = ed.basis_build(n, n_up, z, p, c)
        d = ed.basis_size(B)
        st, _ = ed.basis_states(B)
        x = ei.x_by_state_torch(7, st, nvec, True, dtype=dtype).contiguous() if d else \
            torch.zeros((0, nvec), dtype=dtype, device="cuda")
        items.append((B, x, torch.full_like(x, float("nan"))))
        bases.append(B)
    ed.matvec_multi(O, items, nvec)
    for B, x, y in items:
        if x.numel() == 0:
            continue
        y1 = torch.empty_like(x)
        ed.matvec(O, B, x, y1, nvec)
        assert torch.equal(y, y1)


def test_multi_real_and_generic_search():
    torch, ed = gpu()
    n = 12
    op = ei.heisenberg_ring(n)
    O = ed.operator_create(n, op["sites"], op["coeff"], op["local"])
    for generic in (False, True):
        ed.force_generic(generic)
        try:
            items = []
            for k in (0, 6):          # real characters only: momenta 0 and pi
                for par in (1, -1):
                    for z in (1, -1):
                        p, c = ei.ring_group(n, k, par)
                        B = ed.basis_build(n, n // 2, z, p, c)
                        st, _ = ed.basis_states(B)
                        x = ei.x_by_state_torch(3, st, 1, False, dtype=torch.float64).contiguous()
                        items.append((B, x, torch.empty_like(x)))
            ed.matvec_multi(O, items, 1)
            for B, x, y in items:
                y1 = torch.empty_like(x)
                ed.matvec(O, B, x, y1, 1)
                assert torch.equal(y, y1)
        finally:
            ed.force_generic(False)


def test_multi_rejects_mixed_groups():
    torch, ed = gpu()
    op = ei.heisenberg_ring(8)
    O = ed.operator_create(8, op["sites"], op["coeff"], op["local"])
    p1, c1 = ei.ring_group(8, 0)
    p2, c2 = ei.ring_group(8, 0, +1)
    B1 = ed.basis_build(8, 4, 0, p1, c1)
    B2 = ed.basis_build(8, 4, 0, p2, c2)
    x1 = torch.zeros(ed.basis_size(B1), dtype=torch.float64, device="cuda")
    x2 = torch.zeros(ed.basis_size(B2), dtype=torch.float64, device="cuda")
    with pytest.raises(ed.EDError) as e:
        ed.matvec_multi(O, [(B1, x1, torch.empty_like(x1)), (B2, x2, torch.empty_like(x2))])
    assert e.value.status == 1


@pytest.mark.parametrize("nvec,dt", [(1, "complex64"), (8, "complex128")])
def test_injected_stall_times_out_and_the_context_survives(nvec, dt):
    """Failure detection of the batched launch: with a stall injected (every
    block first waits on a gate word that nothing opens) the bounded wait runs
    out, ed_stream_status reports ED_ERR_TIMEOUT, the outputs are untouched,
    and the next launch on the same context computes the right products."""
    torch, ed = gpu()
    n = 12
    op = ei.xxz_ring(n, 1.0, 1.5)
    O = ed.operator_create(n, op["sites"], op["coeff"], op["local"])
    dtype = getattr(torch, dt)
    items = []
    for n_up, z, p, c in xxz_sectors(n)[:9]:
        B = ed.basis_build(n, n_up, z, p, c)
        st, _ = ed.basis_states(B)
        x = ei.x_by_state_torch(5, st, nvec, True, dtype=dtype).contiguous()
        items.append((B, x, torch.full_like(x, 7.0)))
    assert ed.stream_status() == 0
    ed.inject_stall(True)
    try:
        ed.matvec_multi(O, items, nvec)
        assert ed.stream_status() == 10  # ED_ERR_TIMEOUT
    finally:
        ed.inject_stall(False)
    for _, _, y in items:
        assert bool((y == 7.0).all())
    assert ed.stream_status() == 0
    ed.matvec_multi(O, items, nvec)
    assert ed.stream_status() == 0
    for B, x, y in items:
        y1 = torch.empty_like(x)
        ed.matvec(O, B, x, y1, nvec)
        assert torch.equal(y, y1)
