"""ed_lanczos_block (block Lanczos on nvec vectors, products of the interleaved
block) against the oracle's dense spectra and against the single-vector fp64
solver.

Bars: with fp64 block products the lowest nvec Ritz values equal the lowest
dense eigenvalues of the sector to 1e-10; with fp32 block products (fp64
recurrence, fp64 refinement) the refined ground energy is within 1e-10 of the
dense value, and of the fp64 single-vector Lanczos at N = 32 (the |dE0| target);
the returned vector is an eigenvector to the reported residual."""
import numpy as np
import pytest

import ed_inputs as ei
import oracle
from gpu_util import build_pair, gpu, to_torch
from pins import bethe_e0

pytestmark = pytest.mark.gpu


def dense_spectrum(S):
    return np.linalg.eigvalsh(oracle.dense_matrix(S["G"], S["H"], S["st"], S["nm"]).real)


def start_block(dim, nvec, seed=3):
    return to_torch(ei.x_by_index(seed, dim, nvec), np.float64)


@pytest.mark.parametrize("nvec,steps", [(2, 60), (4, 30), (8, 20), (16, 15)])
def test_ring16_block_eigenvalues_match_dense(nvec, steps):
    torch, ed = gpu()
    w = ei.workload("ring16")
    S = build_pair(16, 8, +1, w["perms"], w["chars"], w["op"])
    ev = dense_spectrum(S)
    x0 = start_block(S["dim"], nvec)
    # reorthogonalised: the lowest nvec Ritz values are the lowest nvec
    # eigenvalues (no spurious copies)
    eigs, r = ed.lanczos_block(S["O"], S["B"], x0, nvec, steps, ed.ED_LANCZOS_F64 | ed.ED_LANCZOS_REORTH,
                               n_eig=nvec)
    assert r.steps == steps
    assert np.max(np.abs(np.array(eigs) - ev[:nvec])) < 1e-10, (eigs, ev[:nvec])
    assert abs(r.e0 - ev[0]) < 1e-10
    # plain recurrence: the lowest eigenvalue all the same
    eigs, r = ed.lanczos_block(S["O"], S["B"], x0, nvec, steps, ed.ED_LANCZOS_F64, n_eig=1)
    assert abs(eigs[0] - ev[0]) < 1e-10 and abs(r.e0 - ev[0]) < 1e-10
    assert abs(ev[0] - bethe_e0(16)) < 1e-10


@pytest.mark.parametrize("nvec,steps", [(2, 5), (4, 3), (8, 3), (16, 2)])
def test_unconverged_ritz_values_equal_the_block_krylov_definition(nvec, steps):
    """After a few steps, far from convergence, the Ritz values of the block
    tridiagonal matrix equal the oracle's Rayleigh-Ritz values of the block
    Krylov space span{X0, H X0, ..., H^(steps-1) X0}: the recurrence (block
    Gram and update, Cholesky QR, the coupling blocks) is checked entry by
    entry through the whole spectrum of T, not only its converged end."""
    torch, ed = gpu()
    for name, p, c, op, z in (("ring16", *ei.ring_group(16, 0, +1), ei.heisenberg_ring(16), +1),
                              ("torus4x4", *ei.torus_group(4, 4, 0, 0), ei.j1j2_torus(4, 4, 1.0, 0.5), +1)):
        S = build_pair(16, 8, z, p, c, op)
        if not ed.basis_is_real(S["B"]):
            continue
        M = oracle.sparse_matrix(S["G"], S["H"], S["st"], S["nm"]).real
        x0 = start_block(S["dim"], nvec, seed=11)
        want = oracle.block_krylov_ritz(lambda V: M @ V, x0.cpu().numpy(), steps)
        k = nvec * steps
        eigs, _ = ed.lanczos_block(S["O"], S["B"], x0, nvec, steps, ed.ED_LANCZOS_F64 | ed.ED_LANCZOS_VALUES_ONLY,
                                   n_eig=k)
        assert len(want) == k
        assert np.max(np.abs(np.array(eigs) - want)) < 1e-9 * np.max(np.abs(want)), (name, eigs, want)


@pytest.mark.parametrize("nvec", [4, 8])
def test_ring16_block_f32_products_refined(nvec):
    torch, ed = gpu()
    w = ei.workload("ring16")
    S = build_pair(16, 8, +1, w["perms"], w["chars"], w["op"])
    ev = dense_spectrum(S)
    x0 = start_block(S["dim"], nvec)
    v = torch.empty(S["dim"], dtype=torch.float64, device="cuda")
    eigs, r = ed.lanczos_block(S["O"], S["B"], x0, nvec, 20, ed.ED_LANCZOS_F32_MATVEC, n_eig=nvec, vec_out=v)
    assert abs(r.e0 - ev[0]) < 1e-10
    assert abs(eigs[0] - ev[0]) < 1e-5      # unrefined: fp32 products
    assert r.residual < 1e-6
    hv = torch.empty_like(v)
    ed.matvec(S["O"], S["B"], v, hv, 1)
    assert abs(float(v.norm()) - 1.0) < 1e-12
    assert float((hv - r.e0 * v).norm()) < 2 * r.residual + 1e-12


def test_torus4x4_real_sector_block():
    """4x4 J1-J2 torus, momentum (0, 0), z = +1 (real characters): the lowest
    eight Ritz values of reorthogonalised fp64 block Lanczos (40 steps, 320 of
    441 dimensions) against the dense spectrum."""
    torch, ed = gpu()
    p, c = ei.torus_group(4, 4, 0, 0)
    S = build_pair(16, 8, +1, p, c, ei.j1j2_torus(4, 4, 1.0, 0.5))
    ev = dense_spectrum(S)
    assert S["dim"] > 200
    x0 = start_block(S["dim"], 8, seed=11)
    eigs, r = ed.lanczos_block(S["O"], S["B"], x0, 8, 40, ed.ED_LANCZOS_F64 | ed.ED_LANCZOS_REORTH, n_eig=8)
    assert np.max(np.abs(np.array(eigs) - ev[:8])) < 1e-10, (eigs, ev[:8])
    assert abs(r.e0 - ev[0]) < 1e-10


def test_block_space_exhausted_stops_early():
    """A sector smaller than the block Krylov space: the recurrence stops when
    the space stops growing, and the eigenvalues found are exact."""
    torch, ed = gpu()
    p, c = ei.ring_group(10, 0, +1)
    S = build_pair(10, 5, +1, p, c, ei.heisenberg_ring(10))
    ev = dense_spectrum(S)
    x0 = start_block(S["dim"], 2)
    eigs, r = ed.lanczos_block(S["O"], S["B"], x0, 2, 40, ed.ED_LANCZOS_F64, n_eig=2)
    assert r.steps * 2 <= S["dim"] + 2 and r.steps < 40
    assert abs(r.e0 - ev[0]) < 1e-10


def test_ring32_block_f32_dE0_against_f64_plain():
    """Heisenberg ring N=32 (4 707 969 rows): fp32 block products (nvec = 8)
    with fp64 recurrence and refinement against the fp64 single-vector
    Lanczos (|dE0| < 1e-10) and the Bethe ansatz."""
    torch, ed = gpu()
    w = ei.workload("ring32")
    S = build_pair(32, 16, +1, w["perms"], w["chars"], w["op"], with_oracle=False)
    x1 = to_torch(ei.x_by_index(0, S["dim"])[:, 0], np.float64)
    r64 = ed.lanczos(S["O"], S["B"], x1, 100, ed.ED_LANCZOS_F64)
    x0 = start_block(S["dim"], 8, seed=0)
    _, rb = ed.lanczos_block(S["O"], S["B"], x0, 8, 40, ed.ED_LANCZOS_F32_MATVEC)
    assert abs(rb.e0 - r64.e0) < 1e-10, (rb.e0, r64.e0)
    assert abs(rb.e0 - bethe_e0(32)) < 1e-10
    assert rb.residual < 1e-6


def test_block_argument_errors():
    torch, ed = gpu()
    w = ei.workload("ring16")
    S = build_pair(16, 8, +1, w["perms"], w["chars"], w["op"], with_oracle=False)
    x0 = start_block(S["dim"], 4)
    with pytest.raises(ed.EDError) as e:
        ed.lanczos_block(S["O"], S["B"], x0, 3, 5)
    assert e.value.status == 1
    p, c = ei.ring_group(12, 5)
    C = build_pair(12, 6, +1, p, c, ei.xxz_ring(12, 1.0, 1.5), with_oracle=False)
    with pytest.raises(ed.EDError) as e:
        ed.lanczos_block(C["O"], C["B"], start_block(C["dim"], 4), 4, 5)
    assert e.value.status == 9


def test_values_only_modes():
    """ED_LANCZOS_VALUES_ONLY: the Ritz values of the main run alone (no Ritz
    vector, no refinement) -- equal to the dense lowest eigenvalue once
    converged, with a small residual estimate; a vector output is refused."""
    torch, ed = gpu()
    w = ei.workload("ring16")
    S = build_pair(16, 8, +1, w["perms"], w["chars"], w["op"])
    ev = dense_spectrum(S)
    x1 = to_torch(ei.x_by_index(0, S["dim"])[:, 0], np.float64)
    r = ed.lanczos(S["O"], S["B"], x1, 60, ed.ED_LANCZOS_F64 | ed.ED_LANCZOS_VALUES_ONLY)
    assert abs(r.e0 - ev[0]) < 1e-10 and r.residual < 1e-6 and r.matvecs == 60
    x0 = start_block(S["dim"], 8)
    eigs, rb = ed.lanczos_block(S["O"], S["B"], x0, 8, 20, ed.ED_LANCZOS_F64 | ed.ED_LANCZOS_VALUES_ONLY, n_eig=1)
    assert abs(rb.e0 - ev[0]) < 1e-10 and rb.e0 == eigs[0] and rb.matvecs == 20 and rb.residual < 1e-6
    with pytest.raises(ed.EDError) as e:
        ed.lanczos_block(S["O"], S["B"], x0, 8, 5, ed.ED_LANCZOS_F64 | ed.ED_LANCZOS_VALUES_ONLY,
                         vec_out=torch.empty(S["dim"], dtype=torch.float64, device="cuda"))
    assert e.value.status == 1
