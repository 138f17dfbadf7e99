"""Pins of the CPU oracle against things other than itself: the paper's printed
numbers, textbook constructions written independently here (Kronecker-product
Hamiltonians, explicit symmetry projectors), closed forms (singlet, 4-ring,
Bethe ansatz), invariants (Hermiticity, Sz conservation, union of sector
spectra) and brute force."""
import math

import numpy as np
import pytest

import ed_inputs as ei
import oracle
from conftest import read_golden


from pins import act_all, bethe_e0, kron_hamiltonian, projected_basis


def ring_sector(n, n_up, k=0, parity=None, z=0, op=None):
    p, c = ei.ring_group(n, k, parity)
    G = oracle.Group(n, p, c, z)
    st, nm = oracle.enumerate_basis(G, n_up)
    H = oracle.Operator(op if op is not None else ei.heisenberg_ring(n))
    return G, H, st, nm


# ----------------------------------------------------------------------------
# the paper's printed numbers
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("row", read_golden("table2_dims.txt"))
def test_table2_dimensions(row):
    n, dim = int(row[0]), int(row[1])
    p, c = ei.ring_group(n, 0, parity=+1)
    assert oracle.sector_dim(oracle.Group(n, p, c, +1), n // 2) == dim


def test_fig1_four_spins():
    want = {r[0]: int(r[1]) for r in read_golden("fig1_four_spins.txt")}
    pt, ct = ei.trivial_group(4)
    st, _ = oracle.enumerate_basis(oracle.Group(4, pt, ct), -1)
    assert len(st) == want["full"]
    p, c = ei.ring_group(4, 0)
    st, _ = oracle.enumerate_basis(oracle.Group(4, p, c), -1)
    assert len(st) == want["translations"]
    # the six translation classes of Fig. 1: 0000, 0001, 0011, 0101, 0111, 1111
    assert list(st) == [0b0000, 0b0001, 0b0011, 0b0101, 0b0111, 0b1111]
    st, _ = oracle.enumerate_basis(oracle.Group(4, pt, ct), 2)
    assert len(st) == want["u1_weight2"] == math.comb(4, 2)


# ----------------------------------------------------------------------------
# enumeration vs the character formula vs brute force
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("n", [4, 6, 8, 10, 12])
def test_enumeration_matches_character_formula_and_irrep_sum(n):
    for n_up in range(0, n + 1):
        total = 0
        zs = (1, -1) if 2 * n_up == n else (0,)
        for k in range(n):
            for z in zs:
                p, c = ei.ring_group(n, k)
                G = oracle.Group(n, p, c, z)
                st, nm = oracle.enumerate_basis(G, n_up)
                assert len(st) == oracle.sector_dim(G, n_up)
                assert np.all(np.diff(st.astype(np.int64)) > 0)
                assert all(bin(int(s)).count("1") == n_up for s in st)
                total += len(st)
        # the one-dimensional irreps of an abelian group resolve the whole space
        assert total == math.comb(n, n_up)


def test_norms_are_stabilizer_orders_brute_force():
    n = 10
    p, c = ei.ring_group(n, 0, parity=+1)
    G = oracle.Group(n, p, c, +1)
    st, nm = oracle.enumerate_basis(G, 5)
    elems = [(q, 0) for q in p] + [(q, 1) for q in p]
    for s, m in zip(st, nm):
        stab = sum(act_all(n, q, f, [int(s)])[0] == int(s) for q, f in elems)
        assert m == stab
        orbit = {int(act_all(n, q, f, [int(s)])[0]) for q, f in elems}
        assert min(orbit) == int(s)
        assert len(orbit) * stab == len(elems)  # orbit-stabilizer


def test_norm_zero_states_are_excluded():
    # k = pi on a 4-ring.  0000 is fixed by every translation and chi(T) = -1,
    # so its character sum over the stabilizer vanishes: norm 0, not in the
    # basis.  0101 is fixed by T^0 and T^2 only, chi(T^2) = +1: norm 2.
    p, c = ei.ring_group(4, 2)
    G = oracle.Group(4, p, c)
    st, nm = oracle.enumerate_basis(G, -1)
    assert 0 not in set(int(s) for s in st)
    rep, chi, norm, ssum = oracle.state_info(G, 0)
    assert norm == 0 and abs(ssum) < 1e-12
    rep, chi, norm, ssum = oracle.state_info(G, 0b0101)
    assert norm == 2 and abs(ssum - 2) < 1e-12


# ----------------------------------------------------------------------------
# the matrix elements against an explicit projector construction
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("case", [
    dict(n=8, n_up=4, k=0, parity=+1, z=+1),
    dict(n=8, n_up=4, k=4, parity=-1, z=+1),
    dict(n=8, n_up=4, k=4, parity=+1, z=-1),
    dict(n=8, n_up=3, k=3, parity=None, z=0),
    dict(n=10, n_up=5, k=1, parity=None, z=+1),
    dict(n=9, n_up=4, k=2, parity=None, z=0),
])
def test_sector_matrix_equals_projected_full_hamiltonian(case):
    n = case["n"]
    p, c = ei.ring_group(n, case["k"], case["parity"])
    rng = np.random.default_rng(7)
    # a Hermitian, translation- and reflection-invariant operator with complex
    # off-diagonal entries would break reflection; use Heisenberg + XXZ mix
    op = ei.heisenberg_ring(n)
    op2 = ei.xxz_ring(n, 0.7, 1.9)
    for key in ("sites", "coeff", "local"):
        op[key] = np.concatenate([op[key], op2[key]])
    G = oracle.Group(n, p, c, case["z"])
    st, nm = oracle.enumerate_basis(G, case["n_up"])
    reps, V = projected_basis(n, case["n_up"], p, c, case["z"])
    assert len(reps) > 0 and np.array_equal(st, reps)
    np.testing.assert_allclose(V.conj().T @ V, np.eye(len(reps)), atol=1e-12)
    Hs = V.conj().T @ kron_hamiltonian(n, op) @ V
    Ho = oracle.dense_matrix(G, oracle.Operator(op), st, nm)
    np.testing.assert_allclose(Ho, Hs, atol=1e-12, rtol=0)


def test_torus_complex_sector_matrix_equals_projection():
    # 3x2 torus, momentum (2pi/3, pi), J1-J2: complex characters, two generators
    p, c = ei.torus_group(3, 2, 1, 1)
    op = ei.j1j2_torus(3, 2, 1.0, 0.5)
    G = oracle.Group(6, p, c, +1)
    st, nm = oracle.enumerate_basis(G, 3)
    reps, V = projected_basis(6, 3, p, c, +1)
    assert np.array_equal(st, reps)
    Hs = V.conj().T @ kron_hamiltonian(6, op) @ V
    Ho = oracle.dense_matrix(G, oracle.Operator(op), st, nm)
    np.testing.assert_allclose(Ho, Hs, atol=1e-12, rtol=0)


def test_full_space_matches_kron_with_random_hermitian_terms():
    n = 6
    rng = np.random.default_rng(3)
    bonds, locs = [], []
    for _ in range(7):
        i, j = rng.choice(n, 2, replace=False)
        a = rng.normal(size=(4, 4)) + 1j * rng.normal(size=(4, 4))
        locs.append(a + a.conj().T)
        bonds.append((i, j))
    op = ei.make_operator(bonds, rng.normal(size=len(bonds)), np.zeros((len(bonds), 4, 4)))
    op["local"][:, :, 0] = np.array([l.real.reshape(16) for l in locs])
    op["local"][:, :, 1] = np.array([l.imag.reshape(16) for l in locs])
    pt, ct = ei.trivial_group(n)
    G = oracle.Group(n, pt, ct)
    st, nm = oracle.enumerate_basis(G, -1)
    assert np.array_equal(st, np.arange(2 ** n, dtype=np.uint64)) and np.all(nm == 1)
    Ho = oracle.dense_matrix(G, oracle.Operator(op), st, nm)
    np.testing.assert_allclose(Ho, kron_hamiltonian(n, op), atol=1e-12, rtol=0)


# ----------------------------------------------------------------------------
# spectra
# ----------------------------------------------------------------------------
def test_union_of_sector_spectra_is_full_spectrum():
    n = 10
    full = np.linalg.eigvalsh(kron_hamiltonian(n, ei.heisenberg_ring(n)))
    parts = []
    for n_up in range(n + 1):
        zs = (1, -1) if 2 * n_up == n else (0,)
        for k in range(n):
            for z in zs:
                G, H, st, nm = ring_sector(n, n_up, k, None, z)
                if len(st):
                    M = oracle.dense_matrix(G, H, st, nm)
                    assert np.abs(M - M.conj().T).max() < 1e-13
                    parts.append(np.linalg.eigvalsh(M))
    union = np.sort(np.concatenate(parts))
    assert len(union) == 2 ** n
    np.testing.assert_allclose(union, full, atol=1e-11)


def test_reflection_sectors_resolve_momentum_sector():
    n, n_up = 12, 6
    for k in (0, 6):
        G, H, st, nm = ring_sector(n, n_up, k, None, 0)
        want = np.linalg.eigvalsh(oracle.dense_matrix(G, H, st, nm))
        got = []
        for par in (+1, -1):
            Gp, Hp, sp_, np_ = ring_sector(n, n_up, k, par, 0)
            if len(sp_):
                got.append(np.linalg.eigvalsh(oracle.dense_matrix(Gp, Hp, sp_, np_)))
        np.testing.assert_allclose(np.sort(np.concatenate(got)), want, atol=1e-11)


def test_two_site_singlet():
    op = ei.make_operator([(0, 1)], [1.0], ei.heisenberg_local())
    pt, ct = ei.trivial_group(2)
    G = oracle.Group(2, pt, ct)
    st, nm = oracle.enumerate_basis(G, -1)
    ev = np.linalg.eigvalsh(oracle.dense_matrix(G, oracle.Operator(op), st, nm))
    np.testing.assert_allclose(ev, [-0.75, 0.25, 0.25, 0.25], atol=1e-15)


def test_four_site_ring_ground_state():
    G, H, st, nm = ring_sector(4, 2, 0, +1, +1)
    ev = np.linalg.eigvalsh(oracle.dense_matrix(G, H, st, nm))
    assert abs(ev[0] + 2.0) < 1e-14


def test_bethe_solver_closed_forms():
    assert abs(bethe_e0(2) + 1.5) < 1e-14          # 2 S0.S1 on the 2-ring
    assert abs(bethe_e0(4) + 2.0) < 1e-12           # the 4-ring
    # thermodynamic limit 1/4 - ln 2 (Hulthen) with the known -pi^2/(12 n^2)
    # leading finite-size correction to the energy per site
    n = 1000
    e = bethe_e0(n) / n
    assert abs(e - (0.25 - math.log(2)) + math.pi ** 2 / (12 * n * n)) < 1e-8


@pytest.mark.parametrize("n", [8, 12, 16, 20])
def test_ground_state_sector_matches_bethe_ansatz(n):
    import scipy.sparse.linalg as sla
    G, H, st, nm = ring_sector(n, n // 2, 0, +1, +1)
    M = oracle.sparse_matrix(G, H, st, nm)
    if M.shape[0] < 400:
        e0 = np.linalg.eigvalsh(M.toarray())[0]
    else:
        e0 = sla.eigsh(M, k=1, which="SA", tol=1e-14)[0][0]
    assert abs(e0 - bethe_e0(n)) < 1e-10


@pytest.mark.parametrize("n", [10, 14, 18])
def test_ground_state_of_2_mod_4_rings_lies_at_momentum_pi(n):
    """For n = 2 mod 4 the ground state is at momentum pi with reflection +1
    and spin inversion -1 (the 2-site singlet is odd under the swap): that
    sector reaches the Bethe ansatz energy, the k = 0, z = +1 sector of the
    same dimension does not."""
    import scipy.sparse.linalg as sla

    def lowest(k, p, z):
        G, H, st, nm = ring_sector(n, n // 2, k, p, z)
        M = oracle.sparse_matrix(G, H, st, nm)
        if M.shape[0] < 400:
            return len(st), np.linalg.eigvalsh(M.toarray())[0]
        return len(st), sla.eigsh(M, k=1, which="SA", tol=1e-14)[0][0]

    d_pi, e_pi = lowest(n // 2, +1, -1)
    d_0, e_0 = lowest(0, +1, +1)
    assert d_pi == d_0
    assert abs(e_pi - bethe_e0(n)) < 1e-10
    assert e_0 > bethe_e0(n) + 0.1


def test_block_krylov_ritz_full_space_is_the_spectrum():
    """Once the block Krylov space fills the whole space its Ritz values are
    the eigenvalues (random symmetric matrix, blocks of 4 and of 1)."""
    rng = np.random.default_rng(5)
    A = rng.standard_normal((40, 40))
    A = A + A.T
    ev = np.linalg.eigvalsh(A)
    for p, m in ((4, 10), (1, 40), (8, 6)):
        X0 = rng.standard_normal((40, p))
        r = oracle.block_krylov_ritz(lambda V: A @ V, X0, m)
        assert len(r) == 40
        assert np.max(np.abs(r - ev)) < 1e-10 * np.max(np.abs(ev))


def test_block_krylov_ritz_of_one_vector_is_lanczos():
    """Block size 1: the Ritz values equal those of the oracle's plain
    Lanczos (with full reorthogonalisation) after the same number of steps,
    and the lowest one decreases with the steps towards the lowest eigenvalue
    without passing it."""
    from scipy.linalg import eigh_tridiagonal
    G, H, st, nm = ring_sector(12, 6, 0, +1, +1)
    M = oracle.sparse_matrix(G, H, st, nm).real
    x0 = np.random.default_rng(3).standard_normal(len(st))
    lam0 = np.linalg.eigvalsh(M.toarray())[0]
    prev = np.inf
    for m in (3, 6, 9):
        a, b, _ = oracle.lanczos(lambda v: M @ v, x0, m, reorth=True)
        want = eigh_tridiagonal(a, b[: len(a) - 1], eigvals_only=True)
        got = oracle.block_krylov_ritz(lambda V: M @ V, x0[:, None], m)
        assert np.max(np.abs(got - want)) < 1e-10
        assert lam0 - 1e-12 <= got[0] <= prev
        prev = got[0]


def test_hermiticity_and_sz_conservation():
    # complex sector: <u, H v> = <H u, v>
    p, c = ei.ring_group(12, 5)
    G = oracle.Group(12, p, c)
    st, nm = oracle.enumerate_basis(G, 5)
    H = oracle.Operator(ei.xxz_ring(12, 1.0, 1.5))
    rng = np.random.default_rng(0)
    u = rng.normal(size=len(st)) + 1j * rng.normal(size=len(st))
    v = rng.normal(size=len(st)) + 1j * rng.normal(size=len(st))
    lhs = np.vdot(u, oracle.matvec(G, H, st, nm, v))
    rhs = np.vdot(oracle.matvec(G, H, st, nm, u), v)
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)
    # Sz conservation on the full space: H commutes with the popcount operator
    pt, ct = ei.trivial_group(8)
    Gt = oracle.Group(8, pt, ct)
    st, nm = oracle.enumerate_basis(Gt, -1)
    M = oracle.dense_matrix(Gt, oracle.Operator(ei.heisenberg_ring(8)), st, nm)
    Sz = np.diag([bin(int(s)).count("1") for s in st])
    assert np.abs(M @ Sz - Sz @ M).max() == 0.0


def test_oracle_lanczos_matches_dense():
    G, H, st, nm = ring_sector(16, 8, 0, +1, +1)
    M = oracle.dense_matrix(G, H, st, nm).real
    x0 = ei.x_by_index(0, len(st))[:, 0]
    _, _, e0 = oracle.lanczos(lambda v: M @ v, x0, 50)
    assert abs(e0 - np.linalg.eigvalsh(M)[0]) < 1e-10


def test_oracle_reorthogonalised_lanczos_spans_the_spectrum():
    """With full reorthogonalisation and as many steps as the Krylov space has
    dimensions, the tridiagonal matrix carries every distinct eigenvalue the
    start vector touches: for a 29-state sector with one degenerate pair, the
    28 distinct eigenvalues of the dense matrix; the plain recurrence after
    many more steps repeats converged values (ghosts) instead."""
    from scipy.linalg import eigh_tridiagonal
    G, H, st, nm = ring_sector(12, 6, 6, -1, +1)
    M = oracle.dense_matrix(G, H, st, nm).real
    ev = np.linalg.eigvalsh(M)
    distinct = [ev[0]]
    for e in ev[1:]:
        if e - distinct[-1] > 1e-8:
            distinct.append(e)
    assert len(st) == 29 and len(distinct) == 28
    x0 = ei.x_by_index(1, len(st))[:, 0]
    a, b, e0 = oracle.lanczos(lambda v: M @ v, x0, 28, reorth=True)
    ritz = eigh_tridiagonal(a, b, eigvals_only=True)
    assert np.max(np.abs(ritz - np.array(distinct))) < 1e-10
    a, b, _ = oracle.lanczos(lambda v: M @ v, x0, 80)
    plain = eigh_tridiagonal(a, b, eigvals_only=True)
    assert abs(plain[0] - ev[0]) < 1e-10 and len(plain) > 28  # extra copies of converged values


# ----------------------------------------------------------------------------
# rows evaluated from states alone (used at sizes where no basis is enumerated)
# ----------------------------------------------------------------------------
@pytest.mark.parametrize("cplx,nvec", [(False, 1), (True, 3)])
def test_state_keyed_rows_match_indexed_matvec(cplx, nvec):
    n, k = 12, (2 if cplx else 0)
    p, c = ei.ring_group(n, k)
    G = oracle.Group(n, p, c, +1)
    st, nm = oracle.enumerate_basis(G, 6)
    H = oracle.Operator(ei.heisenberg_ring(n))
    x = ei.x_by_state(11, st, nvec, cplx)
    y = oracle.matvec(G, H, st, nm, x)
    y2, nnz = oracle.rows_statex(G, H, st, 11, nvec, cplx)
    np.testing.assert_allclose(y2, y, atol=1e-13, rtol=0)
    # nnz = distinct stored elements: off-diagonal terms + one diagonal
    r, cc, _ = oracle.coo(G, H, st, nm)
    offd = np.bincount(r[r != cc], minlength=len(st))
    np.testing.assert_array_equal(nnz, offd + 1)


def test_enumerate_slice_partitions_the_sector():
    n, n_up = 14, 7
    p, c = ei.ring_group(n, 0, +1)
    G = oracle.Group(n, p, c, +1)
    st, _ = oracle.enumerate_basis(G, n_up)
    done, kept = oracle.enumerate_slice(G, n_up, (1 << n_up) - 1, math.comb(n, n_up))
    assert done == math.comb(n, n_up) and kept == len(st)


def test_input_generator_properties():
    x = ei.x_by_index(0, 1 << 16)[:, 0]
    assert x.min() >= -1 and x.max() < 1
    assert abs(x.mean()) < 0.01 and abs(x.var() - 1 / 3) < 0.01
    # the mixer is a bijection (distinct inputs give distinct outputs)
    h = ei.hash64_01(np.arange(1 << 16, dtype=np.uint64))
    assert len(np.unique(h)) == 1 << 16


def test_device_generator_matches_numpy_generator():
    import torch
    st = np.random.default_rng(4).integers(0, 1 << 62, 5000).astype(np.uint64)
    st[:3] = [0, (1 << 40) - 1, (1 << 63) + 12345]
    for cplx, nvec in ((False, 1), (True, 3)):
        want = ei.x_by_state(9, st, nvec, cplx)
        got = ei.x_by_state_torch(9, torch.from_numpy(st.view(np.int64)), nvec, cplx).numpy()
        assert np.array_equal(got, want)
        got_c = ei.x_by_state_torch_chunked(9, torch.from_numpy(st.view(np.int64)), nvec, cplx,
                                            chunk=777).numpy()
        assert np.array_equal(got_c, want)
