"""The workloads other than the timed one, at their full sizes,
as parity cases: basis dimensions against the character formula (and, for the
N=40 ring, against the paper's Table 2), sampled representatives checked one by
one by the oracle, and sampled rows of y = Hx (x keyed by the state) against the
oracle's row evaluation.

Bars as in test_gpu_parity: bit-exact integers, fp64/complex128 within 1e-12 of
max|y| on the sampled rows, fp32/complex64 within 2e-6."""
import math

import numpy as np
import pytest

import ed_inputs as ei
import oracle
from gpu_util import gpu, rel_err

pytestmark = pytest.mark.gpu

F64_TOL = 1e-12
F32_TOL = 2e-6


def sampled_rows_check(B, O, G, H, seed, nvec, cplx, n_rows=120, rng_seed=0):
    """Sampled rows of y = Hx against the oracle; x keyed by state, generated on
    the device from the GPU basis; only the sampled rows come back to the host."""
    torch, ed = gpu()
    st_t, nm_t = ed.basis_states(B)
    dim = st_t.numel()
    rng = np.random.default_rng(rng_seed)
    idx = np.unique(np.concatenate([[0, dim - 1], rng.integers(0, dim, n_rows)]))
    idx_t = torch.from_numpy(idx).cuda()
    st = st_t[idx_t].cpu().numpy().view(np.uint64)
    nm = nm_t[idx_t].cpu().numpy().view(np.uint16)
    # sampled representatives are representatives with the stored norm
    for s_, n_ in list(zip(st, nm))[:40]:
        rep, _, norm, _ = oracle.state_info(G, int(s_))
        assert rep == int(s_) and norm == int(n_)
    want, _ = oracle.rows_statex(G, H, st, seed, nvec, cplx)
    for dt, tol in ((torch.complex128 if cplx else torch.float64, F64_TOL),
                    (torch.complex64 if cplx else torch.float32, F32_TOL)):
        xt = ei.x_by_state_torch_chunked(seed, st_t, nvec, cplx, dtype=dt)
        yt = torch.empty_like(xt)
        ed.matvec(O, B, xt, yt, nvec)
        got = yt[idx_t].cpu().numpy().astype(np.complex128)
        assert rel_err(got, want if cplx else want.real) < tol
        del xt, yt
        torch.cuda.empty_cache()


def test_ring40_config():
    """Heisenberg ring N=40, Sz=0, k=0, p=+1, z=+1: 861 725 794 representatives
    (the paper's Table 2), 64-bit words, factored search."""
    torch, ed = gpu()
    w = ei.workload("ring40")
    B = ed.basis_build(40, 20, +1, w["perms"], w["chars"])
    assert ed.basis_size(B) == 861725794
    assert ed.basis_factored(B)[0]
    assert ed.basis_bucket(B)[0]  # the bucketed index (chosen for large sectors)
    O = ed.operator_create(40, w["op"]["sites"], w["op"]["coeff"], w["op"]["local"])
    G = oracle.Group(40, w["perms"], w["chars"], +1)
    st_t, _ = ed.basis_states(B)
    assert bool((st_t[1:] > st_t[:-1]).all())
    del st_t
    sampled_rows_check(B, O, G, oracle.Operator(w["op"]), 31, 1, False, n_rows=60)
    # the launch configuration of the benchmark's block product: 8 interleaved
    # vectors, fp32 (and fp64)
    sampled_rows_check(B, O, G, oracle.Operator(w["op"]), 32, 8, False, n_rows=40, rng_seed=1)


def test_ring42_config():
    """Heisenberg ring N=42, Sz=0, k=0, p=+1, z=+1: 3 204 236 779 representatives
    (the paper's Table 2), built in full on one GPU (64-bit words, bucketed
    index, indices beyond 2^31); sampled rows of y = Hx in fp64 (row-per-lane
    kernel) and fp32 (term-parallel kernel) against the oracle."""
    torch, ed = gpu()
    torch.cuda.empty_cache()  # the basis and its index take ~125 GB outside torch's cache
    w = ei.workload("ring42")
    B = ed.basis_build(42, 21, +1, w["perms"], w["chars"])
    assert ed.basis_size(B) == 3204236779
    assert ed.basis_factored(B)[0]
    assert ed.basis_bucket(B)[0] and not ed.basis_hash(B)[0]
    O = ed.operator_create(42, w["op"]["sites"], w["op"]["coeff"], w["op"]["local"])
    G = oracle.Group(42, w["perms"], w["chars"], +1)
    st_t, _ = ed.basis_states(B)
    for lo in range(0, st_t.numel() - 1, 1 << 28):  # ascending, checked in slices
        sl = st_t[lo:lo + (1 << 28) + 1]
        assert bool((sl[1:] > sl[:-1]).all())
    del sl
    # lookups beyond index 2^31
    q = st_t[[0, (1 << 31) + 12345, 3204236778]].contiguous()
    assert ed.basis_index(B, q).cpu().tolist() == [0, (1 << 31) + 12345, 3204236778]
    sampled_rows_check(B, O, G, oracle.Operator(w["op"]), 43, 1, False, n_rows=40)


def test_ring36_bucketed_equals_hash_index():
    """Heisenberg ring N=36 (63 068 876 representatives): the products through
    the bucketed index equal those through the hash index bit for bit (both
    lookups are exact and the summation order is the same), for the
    term-parallel kernel (fp32), the row-per-lane kernel (fp64) and block
    vectors (fp32, nvec = 8)."""
    torch, ed = gpu()
    w = ei.workload("ring36")
    O = ed.operator_create(36, w["op"]["sites"], w["op"]["coeff"], w["op"]["local"])
    bases = {}
    try:
        for pol in ("hash", "bucket"):
            ed.index_policy(pol)
            bases[pol] = ed.basis_build(36, 18, +1, w["perms"], w["chars"])
    finally:
        ed.index_policy("auto")
    assert ed.basis_hash(bases["hash"])[0] and ed.basis_bucket(bases["bucket"])[0]
    assert ed.basis_size(bases["hash"]) == ed.basis_size(bases["bucket"]) == 63068876
    st, _ = ed.basis_states(bases["hash"])
    for dt, nvec in ((torch.float32, 1), (torch.float64, 1), (torch.float32, 8)):
        x = ei.x_by_state_torch_chunked(7, st, nvec, False, dtype=dt)
        ys = []
        for pol in ("hash", "bucket"):
            y = torch.empty_like(x)
            ed.matvec(O, bases[pol], x, y, nvec)
            ys.append(y)
        assert torch.equal(ys[0], ys[1])
        del x, ys
        torch.cuda.empty_cache()


def test_table2_n44_count_on_gpu():
    """The paper's Table 2 for 44 spins (11 955 836 258, beyond 2^32), counted
    on the GPU by the enumeration's count pass (2.1e12 states visited)."""
    torch, ed = gpu()
    p, c = ei.ring_group(44, 0, +1)
    assert ed.basis_count(44, 22, +1, p, c) == 11955836258


def test_torus6x6_config():
    """6x6 J1-J2 (J2 = 0.5), Sz=0, momentum (pi/3, 0), z=+1, translations only:
    complex characters, minimiser tracked, 64-bit words."""
    torch, ed = gpu()
    w = ei.workload("torus6x6")
    B = ed.basis_build(36, 18, +1, w["perms"], w["chars"])
    G = oracle.Group(36, w["perms"], w["chars"], +1)
    dim = ed.basis_size(B)
    assert dim == oracle.sector_dim(G, 18) == 126039218
    assert not ed.basis_is_real(B)
    O = ed.operator_create(36, w["op"]["sites"], w["op"]["coeff"], w["op"]["local"])
    sampled_rows_check(B, O, G, oracle.Operator(w["op"]), 37, 1, True, n_rows=60)


def test_xxz28_all_sectors():
    """XXZ ring N=28 (Jxy=1, Delta=1.5): all 140 sectors (Sz = 0..3 x 28 momenta,
    z = +-1 at Sz = 0); the dimensions of each Sz resolve the U(1) sector; block
    vectors nvec=8 checked on sampled rows of a few sectors."""
    torch, ed = gpu()
    op = ei.xxz_ring(28, 1.0, 1.5)
    O = ed.operator_create(28, op["sites"], op["coeff"], op["local"])
    H = oracle.Operator(op)
    sectors = ei.xxz28_sectors()
    assert len(sectors) == 140
    totals = {}
    dims = []
    for s in sectors:
        B = ed.basis_build(28, s["n_up"], s["spin_inversion"], s["perms"], s["chars"])
        d = ed.basis_size(B)
        dims.append(d)
        totals[s["n_up"]] = totals.get(s["n_up"], 0) + d
        del B
    for n_up, tot in totals.items():
        assert tot == math.comb(28, n_up)
    assert min(dims) >= 100000 and max(dims) <= 1400000
    # all 140 sectors in one launch, nvec = 8, against the sector-by-sector product
    items = []
    for s in sectors:
        B = ed.basis_build(28, s["n_up"], s["spin_inversion"], s["perms"], s["chars"])
        st, _ = ed.basis_states(B)
        x = ei.x_by_state_torch(5, st, 8, True, dtype=torch.complex64).contiguous()
        items.append((B, x, torch.empty_like(x)))
    ed.matvec_multi(O, items, 8)
    for B, x, y in items[::7]:
        y1 = torch.empty_like(x)
        ed.matvec(O, B, x, y1, 8)
        assert torch.equal(y, y1)
    del items
    torch.cuda.empty_cache()
    # one vector in single precision: the batched term-parallel launch (tiles
    # from the work queue), the same bits as ed_matvec
    items = []
    for s in sectors[::5]:
        B = ed.basis_build(28, s["n_up"], s["spin_inversion"], s["perms"], s["chars"])
        st, _ = ed.basis_states(B)
        x = ei.x_by_state_torch(6, st, 1, True, dtype=torch.complex64).reshape(-1).contiguous()
        items.append((B, x, torch.empty_like(x)))
    ed.matvec_multi(O, items, 1)
    for B, x, y in items:
        y1 = torch.empty_like(x)
        ed.matvec(O, B, x, y1, 1)
        assert torch.equal(y, y1)
    del items
    torch.cuda.empty_cache()
    for k in (0, 33, 77, 139):  # Sz=0 z=+1 k=0; a complex Sz=0 sector; Sz=1 and Sz=3 sectors
        s = sectors[k]
        B = ed.basis_build(28, s["n_up"], s["spin_inversion"], s["perms"], s["chars"])
        G = oracle.Group(28, s["perms"], s["chars"], s["spin_inversion"])
        assert ed.basis_size(B) == oracle.sector_dim(G, s["n_up"])
        cplx = not ed.basis_is_real(B)
        sampled_rows_check(B, O, G, H, 41 + k, 8, cplx, n_rows=40, rng_seed=k)


def test_table2_n42_count_on_gpu():
    """The paper's Table 2 for 42 spins (3 204 236 779), counted on the GPU by the
    enumeration's count pass (5.4e11 states visited)."""
    torch, ed = gpu()
    p, c = ei.ring_group(42, 0, +1)
    assert ed.basis_count(42, 21, +1, p, c) == 3204236779
