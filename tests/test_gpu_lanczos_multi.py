"""ed_lanczos_multi (the Lanczos recurrence batched over many sectors, steps
replayed from a CUDA graph) against the oracle and against ed_lanczos.

Pins: every sector's energy against the oracle's dense spectrum of that sector
(small rings); the lowest Ritz value after m steps against the oracle's plain
Lanczos run for the same m (m = 1 is the Rayleigh quotient of the start
vector), which covers the steps taken outside the captured graph and the odd
remainder; the full 140-sector XXZ configuration against ed_lanczos sector by
sector.  Bars: 1e-10 on fp64-mode energies, 1e-9 in the fp32-matvec mode on
the small sectors (measured error up to 1.6e-10 there); Ritz values of short runs
within 1e-12 relative (the same recurrence in a different summation order)."""
import numpy as np
import pytest

import ed_inputs as ei
import oracle
from gpu_util import gpu

pytestmark = pytest.mark.gpu


def xxz_sectors(n, max_sz):
    out = []
    for sz in range(max_sz + 1):
        for k in range(n):
            for z in ((1, -1) if sz == 0 else (0,)):
                p, c = ei.ring_group(n, k)
                out.append((n // 2 + sz, z, p, c))
    return out


def start_vectors(ed, torch, bases, cplx, seed=11):
    xs = []
    for B in bases:
        st, _ = ed.basis_states(B)
        xs.append(ei.x_by_state_torch(seed, st, 1, cplx,
                                      dtype=torch.complex128 if cplx else torch.float64)
                  .reshape(-1).contiguous())
    return xs


@pytest.mark.parametrize("recompute", [False, True], ids=["kept", "two_pass"])
@pytest.mark.parametrize("mode", ["f64", "f32_matvec"])
def test_xxz14_all_sectors_against_dense_spectra(mode, recompute):
    """XXZ ring N=14 (Delta = 1.5), Sz = 0..2, all momenta, z = +-1 at Sz = 0:
    56 complex sectors of dimension 118..217 in one call; sectors smaller than
    the step count end on an invariant subspace."""
    torch, ed = gpu()
    n = 14
    op = ei.xxz_ring(n, 1.0, 1.5)
    O = ed.operator_create(n, op["sites"], op["coeff"], op["local"])
    H = oracle.Operator(op)
    secs = xxz_sectors(n, 2)
    bases = [ed.basis_build(n, nu, z, p, c) for nu, z, p, c in secs]
    assert all(ed.basis_size(B) > 0 for B in bases)
    xs = start_vectors(ed, torch, bases, True)
    vs = [torch.empty_like(x) for x in xs]
    m = (ed.ED_LANCZOS_F64 if mode == "f64" else ed.ED_LANCZOS_F32_MATVEC) | \
        (ed.ED_LANCZOS_RECOMPUTE if recompute else 0)
    res = ed.lanczos_multi(O, list(zip(bases, xs, vs)), 90, m)
    # fp32-matvec mode: six fp64 refinement steps from the fp32 Ritz vector
    # leave residuals up to 2e-5 on these sectors (measured), which bounds the
    # energy error near residual^2 / gap ~ 2e-10
    res_tol = 1e-6 if mode == "f64" else 1e-4
    e_tol = 1e-10 if mode == "f64" else 1e-9
    for (nu, z, p, c), B, x, v, r in zip(secs, bases, xs, vs, res):
        G = oracle.Group(n, p, c, z)
        st, nm = oracle.enumerate_basis(G, nu)
        e_dense = np.linalg.eigvalsh(oracle.dense_matrix(G, H, st, nm))[0]
        assert abs(r.e0 - e_dense) < e_tol, (nu, z, r.e0, e_dense)
        assert r.residual < res_tol
        assert abs(float(v.norm()) - 1.0) < 1e-12
        hv = torch.empty_like(v)
        ed.matvec(O, B, v, hv, 1)
        assert float((hv - r.e0 * v).norm()) < res_tol
    # the same energies as the single-sector solver
    for B, x, r in list(zip(bases, xs, res))[::9]:
        r1 = ed.lanczos(O, B, x, 90, m)
        assert abs(r1.e0 - r.e0) < e_tol


@pytest.mark.parametrize("recompute", [False, True], ids=["kept", "two_pass"])
@pytest.mark.parametrize("steps", [1, 2, 3, 4, 5, 8])
def test_short_runs_match_oracle_lanczos(steps, recompute):
    """Real sectors of the Heisenberg ring N=12 (k = 0, pi; reflection +-1;
    z = +-1): the lowest Ritz value after `steps` steps equals the oracle's
    plain Lanczos on the dense sector matrix from the same start vector."""
    torch, ed = gpu()
    n = 12
    op = ei.heisenberg_ring(n)
    O = ed.operator_create(n, op["sites"], op["coeff"], op["local"])
    H = oracle.Operator(op)
    secs = [(k, par, z) for k in (0, 6) for par in (1, -1) for z in (1, -1)]
    bases, gs = [], []
    for k, par, z in secs:
        p, c = ei.ring_group(n, k, par)
        bases.append(ed.basis_build(n, n // 2, z, p, c))
        gs.append(oracle.Group(n, p, c, z))
    keep = [i for i, B in enumerate(bases) if ed.basis_size(B) > steps]
    bases = [bases[i] for i in keep]
    gs = [gs[i] for i in keep]
    xs = start_vectors(ed, torch, bases, False, seed=3)
    flags = ed.ED_LANCZOS_RECOMPUTE if recompute else 0
    res = ed.lanczos_multi(O, [(B, x, None) for B, x in zip(bases, xs)], steps,
                           ed.ED_LANCZOS_F64 | flags)
    for G, r in zip(gs, res):
        st, nm = oracle.enumerate_basis(G, n // 2)
        Hd = oracle.dense_matrix(G, H, st, nm).real
        x0 = ei.x_by_state(3, st)[:, 0]
        _, _, ritz = oracle.lanczos(lambda v: Hd @ v, x0, steps)
        assert abs(r.ritz - ritz) <= 1e-12 * abs(ritz), (steps, r.ritz, ritz)
        assert r.matvecs == (2 * steps + 1 if recompute else steps + 1)
        if steps == 1:
            assert abs(r.e0 - float(x0 @ Hd @ x0) / float(x0 @ x0)) <= 1e-12 * abs(r.e0)


def test_argument_errors():
    torch, ed = gpu()
    n = 8
    op = ei.heisenberg_ring(n)
    O = ed.operator_create(n, op["sites"], op["coeff"], op["local"])
    p1, c1 = ei.ring_group(n, 1)     # complex characters
    B1 = ed.basis_build(n, 4, 0, p1, c1)
    st, _ = ed.basis_states(B1)
    x = ei.x_by_state_torch(1, st, 1, False, dtype=torch.float64).reshape(-1).contiguous()
    with pytest.raises(ed.EDError):  # real vectors for a complex sector
        ed.lanczos_multi(O, [(B1, x, None)], 5)
    B0 = ed.basis_build(n, 0, 0, p1, c1)   # n_up = 0 at k != 0: empty sector
    assert ed.basis_size(B0) == 0
    xe = torch.zeros(1, dtype=torch.complex128, device="cuda")
    xc = x.to(torch.complex128)
    with pytest.raises(ed.EDError):
        ed.lanczos_multi(O, [(B1, xc, None), (B0, xe, None)], 5)
    B2 = ed.basis_build(n, 4, 0, *ei.ring_group(n, 0, +1))  # other permutation list
    st2, _ = ed.basis_states(B2)
    x2 = ei.x_by_state_torch(1, st2, 1, True, dtype=torch.complex128).reshape(-1).contiguous()
    with pytest.raises(ed.EDError):
        ed.lanczos_multi(O, [(B1, xc, None), (B2, x2, None)], 5)


def test_xxz28_config_all_140_sectors():
    """XXZ ring N=28 (Delta = 1.5), all 140 sectors (129 454 695 rows) in one
    batched fp32-matvec solve; a sample of sectors against ed_lanczos."""
    torch, ed = gpu()
    op = ei.xxz_ring(28, 1.0, 1.5)
    O = ed.operator_create(28, op["sites"], op["coeff"], op["local"])
    secs = ei.xxz28_sectors()
    bases = [ed.basis_build(28, s["n_up"], s["spin_inversion"], s["perms"], s["chars"]) for s in secs]
    xs = start_vectors(ed, torch, bases, True, seed=5)
    steps = 100
    res = ed.lanczos_multi(O, [(B, x, None) for B, x in zip(bases, xs)], steps,
                           ed.ED_LANCZOS_F32_MATVEC)
    assert all(np.isfinite(r.e0) for r in res)
    for k in (0, 1, 33, 77, 139):
        r1 = ed.lanczos(O, bases[k], xs[k], steps, ed.ED_LANCZOS_F32_MATVEC)
        assert abs(r1.e0 - res[k].e0) < 1e-8 * abs(r1.e0), (k, r1.e0, res[k].e0)
    # the Sz = 0 ground state lies below every Sz > 0 sector's (antiferromagnet)
    e_by_sz = {}
    for s, r in zip(secs, res):
        e_by_sz[s["n_up"]] = min(e_by_sz.get(s["n_up"], np.inf), r.e0)
    assert e_by_sz[14] < e_by_sz[15] < e_by_sz[16] < e_by_sz[17]
