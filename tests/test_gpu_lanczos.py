"""ed_lanczos on the GPU against the oracle's dense spectrum (small sectors) and
against the Bethe ansatz (Heisenberg rings at the benchmark sizes).

Bars: fp64 Lanczos ground energy within 1e-10 of the reference; the fp32-matvec
mode (fp64 recurrence, fp64 refinement) within 1e-10 of the fp64 mode, which
is the |dE0| target; residuals reported by the library are small."""
import numpy as np
import pytest

import ed_inputs as ei
import oracle
from gpu_util import build_pair, gpu, to_torch
from pins import bethe_e0

pytestmark = pytest.mark.gpu


def lanczos_pair(S, steps, cplx, flags=0):
    torch, ed = gpu()
    x0 = ei.x_by_index(0, S["dim"], 1, cplx)[:, 0]
    xt = to_torch(x0, np.complex128 if cplx else np.float64)
    r64 = ed.lanczos(S["O"], S["B"], xt, steps, ed.ED_LANCZOS_F64 | flags)
    r32 = ed.lanczos(S["O"], S["B"], xt, steps, ed.ED_LANCZOS_F32_MATVEC | flags)
    return r64, r32


def test_ring16_lanczos_matches_dense_spectrum():
    w = ei.workload("ring16")
    S = build_pair(16, 8, +1, w["perms"], w["chars"], w["op"])
    e_dense = np.linalg.eigvalsh(oracle.dense_matrix(S["G"], S["H"], S["st"], S["nm"]).real)[0]
    r64, r32 = lanczos_pair(S, 50, False)
    assert abs(r64.e0 - e_dense) < 1e-10
    assert abs(r32.e0 - e_dense) < 1e-10
    assert abs(r64.e0 - r32.e0) < 1e-10
    assert r64.residual < 1e-6 and r32.residual < 1e-6
    assert abs(e_dense - bethe_e0(16)) < 1e-10


def test_two_pass_ritz_vector_is_identical():
    torch, ed = gpu()
    w = ei.workload("ring16")
    S = build_pair(16, 8, +1, w["perms"], w["chars"], w["op"], with_oracle=False)
    x0 = to_torch(ei.x_by_index(0, S["dim"])[:, 0], np.float64)
    v1 = torch.empty_like(x0)
    v2 = torch.empty_like(x0)
    r1 = ed.lanczos(S["O"], S["B"], x0, 40, ed.ED_LANCZOS_F64, vec_out=v1)
    r2 = ed.lanczos(S["O"], S["B"], x0, 40, ed.ED_LANCZOS_F64 | ed.ED_LANCZOS_RECOMPUTE, vec_out=v2)
    assert r1.e0 == r2.e0
    assert torch.allclose(v1, v2, atol=1e-14, rtol=0)
    # the returned vector is an eigenvector: |H v - e0 v| small
    hv = torch.empty_like(v1)
    ed.matvec(S["O"], S["B"], v1, hv, 1)
    assert float((hv - r1.e0 * v1).norm()) < 1e-6


def test_two_pass_refinement_is_identical():
    """fp32-matvec mode: with RECOMPUTE both the main Ritz vector and the
    fp64 refinement's come from second passes (the layout used when their
    vectors do not fit beside a sector of billions of states); energy and
    vector equal those from stored vectors."""
    torch, ed = gpu()
    w = ei.workload("ring16")
    S = build_pair(16, 8, +1, w["perms"], w["chars"], w["op"], with_oracle=False)
    x0 = to_torch(ei.x_by_index(0, S["dim"])[:, 0], np.float64)
    v1 = torch.empty_like(x0)
    v2 = torch.empty_like(x0)
    r1 = ed.lanczos(S["O"], S["B"], x0, 40, ed.ED_LANCZOS_F32_MATVEC, vec_out=v1)
    r2 = ed.lanczos(S["O"], S["B"], x0, 40, ed.ED_LANCZOS_F32_MATVEC | ed.ED_LANCZOS_RECOMPUTE, vec_out=v2)
    assert r1.e0 == r2.e0 and r1.residual == r2.residual
    assert torch.equal(v1, v2)
    assert r2.matvecs == r1.matvecs + 40 + 6
    assert abs(r2.e0 - bethe_e0(16)) < 1e-10


def test_complex_sector_lanczos():
    p, c = ei.torus_group(4, 4, 1, 0)
    op = ei.j1j2_torus(4, 4, 1.0, 0.5)
    S = build_pair(16, 8, +1, p, c, op)
    e_dense = np.linalg.eigvalsh(oracle.dense_matrix(S["G"], S["H"], S["st"], S["nm"]))[0]
    r64, r32 = lanczos_pair(S, 80, True)
    assert abs(r64.e0 - e_dense) < 1e-10
    assert abs(r32.e0 - e_dense) < 1e-10


def test_invariant_subspace_stops_early():
    # a 3-dimensional sector: Lanczos must stop after 3 steps, not divide by zero
    p, c = ei.ring_group(6, 0, +1)
    S = build_pair(6, 3, +1, p, c, ei.heisenberg_ring(6))
    e_dense = np.linalg.eigvalsh(oracle.dense_matrix(S["G"], S["H"], S["st"], S["nm"]).real)[0]
    r64, r32 = lanczos_pair(S, 20, False)
    assert r64.steps <= S["dim"]
    assert abs(r64.e0 - e_dense) < 1e-12 and abs(r32.e0 - e_dense) < 1e-10


def test_ring32_fp32_matvec_lanczos_reaches_fp64():
    w = ei.workload("ring32")
    S = build_pair(32, 16, +1, w["perms"], w["chars"], w["op"], with_oracle=False)
    r64, r32 = lanczos_pair(S, 100, False)
    e_bethe = bethe_e0(32)
    assert abs(r64.e0 - e_bethe) < 1e-9
    assert abs(r32.e0 - e_bethe) < 1e-9
    assert abs(r64.e0 - r32.e0) < 1e-10


def test_push_mode_lanczos():
    """ED_LANCZOS_PUSH (transposed products with atomic adds): the same energy
    as the dense spectrum within the bar; refused where a recomputed pass
    would be needed."""
    torch, ed = gpu()
    w = ei.workload("ring16")
    S = build_pair(16, 8, +1, w["perms"], w["chars"], w["op"])
    e_dense = np.linalg.eigvalsh(oracle.dense_matrix(S["G"], S["H"], S["st"], S["nm"]).real)[0]
    x0 = to_torch(ei.x_by_index(0, S["dim"])[:, 0], np.float64)
    for mode in (ed.ED_LANCZOS_F64, ed.ED_LANCZOS_F32_MATVEC):
        r = ed.lanczos(S["O"], S["B"], x0, 50, mode | ed.ED_LANCZOS_PUSH)
        assert abs(r.e0 - e_dense) < 1e-10
        assert r.residual < 1e-6
    with pytest.raises(ed.EDError):
        ed.lanczos(S["O"], S["B"], x0, 50, ed.ED_LANCZOS_F64 | ed.ED_LANCZOS_PUSH | ed.ED_LANCZOS_RECOMPUTE)


def _heisenberg12_real_sectors(ed):
    n = 12
    op = ei.heisenberg_ring(n)
    out = []
    for k in (0, 6):
        for par in (1, -1):
            p, c = ei.ring_group(n, k, par)
            out.append(build_pair(n, n // 2, +1, p, c, op))
    return out


@pytest.mark.parametrize("reorth", [False, True], ids=["plain", "reorth"])
@pytest.mark.parametrize("steps", [3, 6, 10])
def test_eigs_short_runs_match_oracle(steps, reorth):
    """The lowest Ritz values after `steps` steps against the eigenvalues of the
    oracle's tridiagonal matrix from the same start vector (plain recurrence, or
    classical Gram-Schmidt twice against all earlier vectors)."""
    from scipy.linalg import eigh_tridiagonal
    torch, ed = gpu()
    flags = ed.ED_LANCZOS_F64 | (ed.ED_LANCZOS_REORTH if reorth else 0)
    for S in _heisenberg12_real_sectors(ed):
        if S["dim"] <= steps:
            continue
        Hd = oracle.dense_matrix(S["G"], S["H"], S["st"], S["nm"]).real
        x0 = ei.x_by_state(3, S["st"])[:, 0]
        a, b, _ = oracle.lanczos(lambda v: Hd @ v, x0, steps, reorth=reorth)
        want = eigh_tridiagonal(a, b, eigvals_only=True)
        n_eig = min(3, steps)
        eigs, r = ed.lanczos_eigs(S["O"], S["B"], to_torch(x0, np.float64), steps, n_eig, flags)
        for g, e in zip(eigs, want[:n_eig]):
            assert abs(g - e) <= 1e-12 * max(1.0, abs(e)), (steps, reorth, eigs, want[:n_eig])


def test_eigs_low_spectrum_with_reorthogonalisation():
    """ring N=16 sector (dimension 257), 120 steps with full reorthogonalisation:
    the five lowest Ritz values are the five lowest eigenvalues of the dense
    sector matrix (fp64 within 1e-9; fp32 products within 2e-6 relative)."""
    torch, ed = gpu()
    w = ei.workload("ring16")
    S = build_pair(16, 8, +1, w["perms"], w["chars"], w["op"])
    ev = np.linalg.eigvalsh(oracle.dense_matrix(S["G"], S["H"], S["st"], S["nm"]).real)
    x0 = to_torch(ei.x_by_index(0, S["dim"])[:, 0], np.float64)
    eigs, r = ed.lanczos_eigs(S["O"], S["B"], x0, 120, 5, ed.ED_LANCZOS_F64 | ed.ED_LANCZOS_REORTH)
    assert np.max(np.abs(np.array(eigs) - ev[:5])) < 1e-9
    assert abs(r.e0 - ev[0]) < 1e-10
    eigs32, r32 = ed.lanczos_eigs(S["O"], S["B"], x0, 120, 5, ed.ED_LANCZOS_F32_MATVEC | ed.ED_LANCZOS_REORTH)
    assert np.max(np.abs(np.array(eigs32) - ev[:5]) / np.abs(ev[:5])) < 2e-6
    assert abs(r32.e0 - ev[0]) < 1e-10
    # beyond the Krylov space (29 states, 28 distinct eigenvalues: a single start
    # vector spans 28 dimensions): the 28 distinct eigenvalues, then NaN
    small = build_pair(12, 6, +1, *ei.ring_group(12, 6, -1), ei.heisenberg_ring(12))
    ev_s = np.linalg.eigvalsh(oracle.dense_matrix(small["G"], small["H"], small["st"], small["nm"]).real)
    distinct = [ev_s[0]]
    for e in ev_s[1:]:
        if e - distinct[-1] > 1e-8:
            distinct.append(e)
    xs = to_torch(ei.x_by_index(1, small["dim"])[:, 0], np.float64)
    e_s, r_s = ed.lanczos_eigs(small["O"], small["B"], xs, 40, 40, ed.ED_LANCZOS_F64 | ed.ED_LANCZOS_REORTH)
    nd = len(distinct)
    assert small["dim"] == 29 and nd == 28 and r_s.steps == nd
    assert np.max(np.abs(np.array(e_s[:nd]) - np.array(distinct))) < 1e-9
    assert np.all(np.isnan(e_s[nd:]))
    with pytest.raises(ed.EDError):
        ed.lanczos_eigs(S["O"], S["B"], x0, 20, 21)
    # residual check: 5 steps cannot reach 1e-10; 120 steps reach 1e-6
    with pytest.raises(ed.EDError) as err:
        ed.lanczos_eigs(S["O"], S["B"], x0, 5, 1, tol=1e-10)
    assert err.value.status == 8  # ED_ERR_NOT_CONVERGED
    ed.lanczos_eigs(S["O"], S["B"], x0, 120, 1, ed.ED_LANCZOS_F64 | ed.ED_LANCZOS_REORTH, tol=1e-6)
    with pytest.raises(ed.EDError):
        ed.lanczos_eigs(S["O"], S["B"], x0, 20, 2,
                        ed.ED_LANCZOS_F64 | ed.ED_LANCZOS_REORTH | ed.ED_LANCZOS_RECOMPUTE)


def test_cached_workspace_memory_is_reused_and_released():
    """Work arrays come from the library's pool: a second identical solve gives
    the same bits, and the cached memory can be handed back."""
    torch, ed = gpu()
    w = ei.workload("ring16")
    S = build_pair(16, 8, +1, w["perms"], w["chars"], w["op"], with_oracle=False)
    x0 = to_torch(ei.x_by_index(0, S["dim"])[:, 0], np.float64)
    r1 = ed.lanczos(S["O"], S["B"], x0, 40, ed.ED_LANCZOS_F32_MATVEC)
    r2 = ed.lanczos(S["O"], S["B"], x0, 40, ed.ED_LANCZOS_F32_MATVEC)
    assert r1.e0 == r2.e0 and r1.residual == r2.residual
    ed.release_cached_memory()
    r3 = ed.lanczos(S["O"], S["B"], x0, 40, ed.ED_LANCZOS_F32_MATVEC)
    assert r3.e0 == r1.e0


@pytest.mark.parametrize("mode_name", ["f64", "f32", "f64_recompute", "f32_recompute", "values_only"])
@pytest.mark.parametrize("steps", [1, 2, 40, 41])
def test_graph_replayed_steps_equal_eager_steps(mode_name, steps):
    """Steps replayed from a CUDA graph (device step index, ring buffers
    copied into the Krylov store) give the eager launches' results bit for
    bit: energy, residual, Ritz values and vector."""
    torch, ed = gpu()
    w = ei.workload("ring16")
    S = build_pair(16, 8, +1, w["perms"], w["chars"], w["op"], with_oracle=False)
    x0 = to_torch(ei.x_by_index(3, S["dim"])[:, 0], np.float64)
    mode = {"f64": ed.ED_LANCZOS_F64, "f32": ed.ED_LANCZOS_F32_MATVEC,
            "f64_recompute": ed.ED_LANCZOS_F64 | ed.ED_LANCZOS_RECOMPUTE,
            "f32_recompute": ed.ED_LANCZOS_F32_MATVEC | ed.ED_LANCZOS_RECOMPUTE,
            "values_only": ed.ED_LANCZOS_F64 | ed.ED_LANCZOS_VALUES_ONLY}[mode_name]
    out = {}
    old = ed.lanczos_graph(0)
    try:
        for policy in (0, 1):
            ed.lanczos_graph(policy)
            v = None if mode_name == "values_only" else torch.empty_like(x0)
            n_eig = min(3, steps)
            eigs, r = ed.lanczos_eigs(S["O"], S["B"], x0, steps, n_eig, mode, vec_out=v)
            out[policy] = (eigs, r.e0, r.residual, r.ritz, r.matvecs, v)
    finally:
        ed.lanczos_graph(old)
    e, g = out[0], out[1]
    assert e[0] == g[0] and e[1] == g[1] and e[2] == g[2] and e[3] == g[3] and e[4] == g[4]
    if e[5] is not None:
        assert torch.equal(e[5], g[5])


def test_graph_replayed_complex_sector():
    torch, ed = gpu()
    p, c = ei.torus_group(4, 4, 1, 0)
    op = ei.j1j2_torus(4, 4, 1.0, 0.5)
    S = build_pair(16, 8, +1, p, c, op, with_oracle=False)
    x0 = to_torch(ei.x_by_index(0, S["dim"], 1, True)[:, 0], np.complex128)
    res = []
    old = ed.lanczos_graph(0)
    try:
        for policy in (0, 1):
            ed.lanczos_graph(policy)
            v = torch.empty_like(x0)
            r = ed.lanczos(S["O"], S["B"], x0, 37, ed.ED_LANCZOS_F32_MATVEC, vec_out=v)
            res.append((r.e0, r.residual, v))
    finally:
        ed.lanczos_graph(old)
    assert res[0][0] == res[1][0] and res[0][1] == res[1][1]
    assert torch.equal(res[0][2], res[1][2])
