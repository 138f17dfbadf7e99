"""GPU path (through the C ABI) against the oracle, element by element.

Bars: basis states, orbit norms and indices bit-exact; fp64 / complex128
matvec within 1e-12 of the oracle, relative to the largest |y| (each element is
a sum of a few dozen products of O(1) numbers, so the only difference is the
summation order: a few ulps); fp32 / complex64 within 2e-6 relative (single
precision coefficients and accumulation over the row's terms)."""
import math

import numpy as np
import pytest

import ed_inputs as ei
import oracle
from gpu_util import build_pair, elem_rel_err, gpu, gpu_basis_numpy, rel_err, to_torch

pytestmark = pytest.mark.gpu

F64_TOL = 1e-12
F32_TOL = 2e-6

def xx_ring(n):
    """J Sx_i Sx_{i+1} (no U(1) symmetry: couples |00> <-> |11> as well)."""
    h = np.zeros((4, 4))
    h[0, 3] = h[3, 0] = h[1, 2] = h[2, 1] = 0.25
    return ei.make_operator([(i, (i + 1) % n) for i in range(n)], [1.0] * n, h)


def dm_ring(n, d):
    """Heisenberg ring plus a uniform Dzyaloshinskii-Moriya coupling
    d (Sx_i Sy_j - Sy_i Sx_j): exchange-only, with imaginary matrix entries."""
    op = ei.heisenberg_ring(n)
    op["local"][:, 4 * 2 + 1, 1] = 0.5 * d   # h[2][1] = +i d/2 (row-major 4x4)
    op["local"][:, 4 * 1 + 2, 1] = -0.5 * d  # h[1][2] = -i d/2
    return op


def affine_group(n, a, sign=1.0):
    """Site maps i -> u*i + b mod n, u in {1, a} (a*a = 1 mod n): translations
    times one non-reflection automorphism of the ring, so that the factored
    search has a coset applied by a Benes network; chi = sign on the second
    coset (momentum 0)."""
    perms, chars = [], []
    for u in (1, a):
        for b in range(n):
            perms.append([(u * i + b) % n for i in range(n)])
            chars.append([1.0 if u == 1 else sign, 0.0])
    return np.asarray(perms, np.int32), np.asarray(chars)


def affine_heisenberg(n, a):
    """Heisenberg bonds at distances 1 and a (the affine map exchanges them)."""
    bonds = [(i, (i + 1) % n) for i in range(n)] + [(i, (i + a) % n) for i in range(n)]
    return ei.make_operator(bonds, [1.0] * len(bonds), ei.heisenberg_local())


SECTORS = [
    # name, n, n_up, z, group builder, operator
    ("ring16_k0_p+_z+", 16, 8, +1, lambda: ei.ring_group(16, 0, +1), lambda: ei.heisenberg_ring(16)),
    ("ring12_k0_z-", 12, 6, -1, lambda: ei.ring_group(12, 0), lambda: ei.heisenberg_ring(12)),
    ("ring12_k6_p-_z+", 12, 6, +1, lambda: ei.ring_group(12, 6, -1), lambda: ei.heisenberg_ring(12)),
    ("ring12_k5_z+", 12, 6, +1, lambda: ei.ring_group(12, 5), lambda: ei.xxz_ring(12, 1.0, 1.5)),
    ("ring13_k3", 13, 5, 0, lambda: ei.ring_group(13, 3), lambda: ei.xxz_ring(13, 1.0, 1.5)),
    ("ring10_noU1_k0_z+", 10, -1, +1, lambda: ei.ring_group(10, 0), lambda: ei.heisenberg_ring(10)),
    ("ring20_k0_p-_z-", 20, 10, -1, lambda: ei.ring_group(20, 0, -1), lambda: ei.heisenberg_ring(20)),
    ("torus4x4_k12_z-", 16, 8, -1, lambda: ei.torus_group(4, 4, 1, 2), lambda: ei.j1j2_torus(4, 4, 1.0, 0.5)),
    ("torus3x4_k10", 12, 5, 0, lambda: ei.torus_group(3, 4, 1, 0), lambda: ei.j1j2_torus(3, 4, 1.0, 0.5)),
    ("trivial10", 10, 5, 0, lambda: ei.trivial_group(10), lambda: ei.heisenberg_ring(10)),
    ("ring34_nup3_k1", 34, 3, 0, lambda: ei.ring_group(34, 1), lambda: ei.heisenberg_ring(34)),
    ("ring40_nup2_k0_p+", 40, 2, 0, lambda: ei.ring_group(40, 0, +1), lambda: ei.heisenberg_ring(40)),
    ("ring36_k0_nup4_z", 36, 4, 0, lambda: ei.ring_group(36, 0), lambda: ei.xxz_ring(36, 1.0, 1.5)),
    ("ring8_nup0", 8, 0, 0, lambda: ei.ring_group(8, 0), lambda: ei.heisenberg_ring(8)),
    ("ring8_nup8", 8, 8, 0, lambda: ei.ring_group(8, 0), lambda: ei.heisenberg_ring(8)),
    ("ring8_empty", 8, 4, -1, lambda: ei.ring_group(8, 4, -1), lambda: ei.heisenberg_ring(8)),
    ("ring10_noU1_xx_z-", 10, -1, -1, lambda: ei.ring_group(10, 0, +1), lambda: xx_ring(10)),
    ("ring11_dm_k2", 11, 5, 0, lambda: ei.ring_group(11, 2), lambda: dm_ring(11, 0.3)),
    ("ring32_nup4_k3", 32, 4, 0, lambda: ei.ring_group(32, 3), lambda: ei.heisenberg_ring(32)),
    ("ring33_nup3_k0_p-", 33, 3, 0, lambda: ei.ring_group(33, 0, -1), lambda: ei.xxz_ring(33, 1.0, 1.5)),
    ("ring64_nup2_k0_p+", 64, 2, 0, lambda: ei.ring_group(64, 0, +1), lambda: ei.heisenberg_ring(64)),
    ("affine16_a7_z+", 16, 8, +1, lambda: affine_group(16, 7, -1.0), lambda: affine_heisenberg(16, 7)),
]


def make(case, with_oracle=True):
    name, n, n_up, z, grp, opf = case
    p, c = grp()
    return build_pair(n, n_up, z, p, c, opf(), with_oracle)


@pytest.fixture(params=["factored", "all_rotations", "generic", "prefix", "rowwise", "term_parallel",
                        "bucket"], autouse=True)
def search_mode(request):
    """Run every parity test six times: factored (rotation x coset) group
    search with the hash index, pruned to the tops of the longest runs where
    the rotations step by one site; the same search visiting every rotation;
    generic Benes search over every element with the hash index; factored
    search with the prefix-table binary search (the row-per-lane kernel);
    factored search and hash index with the row-per-lane kernel forced; and
    with the term-parallel kernel forced in both precisions and for real
    8-vector blocks (by default it serves single vectors of exchange-only
    operators in single precision, and in double above 32 sites); and with
    the bucketed index (one 32-byte bucket per lookup) built for every sector
    whose key fits its entry."""
    torch, ed = gpu()
    ed.index_policy("bucket" if request.param == "bucket" else "hash")
    ed.force_generic(request.param == "generic")
    ed.force_all_rotations(request.param == "all_rotations")
    ed.force_prefix_search(request.param == "prefix")
    ed.kernel_policy(request.param if request.param in ("rowwise", "term_parallel") else "auto")
    yield request.param
    ed.index_policy("auto")
    ed.force_generic(False)
    ed.force_all_rotations(False)
    ed.force_prefix_search(False)
    ed.kernel_policy("auto")


@pytest.mark.parametrize("case", SECTORS, ids=[s[0] for s in SECTORS])
def test_basis_bit_exact(case, search_mode):
    S = make(case)
    torch, ed = gpu()
    fact, L, d, nc = ed.basis_factored(S["B"])
    if case[0].startswith(("ring", "torus")) and search_mode == "factored":
        assert fact and nc * L == len(case[4]()[0])
    has_hash, hbits, hmax, wide = ed.basis_hash(S["B"])
    has_bkt, bbits, n_stash = ed.basis_bucket(S["B"])
    assert (has_hash or has_bkt) == (S["dim"] > 0) and not (has_hash and has_bkt)
    if has_hash:
        assert (2 << hbits) >= S["dim"] and hmax <= 16
    if has_bkt:
        assert search_mode == "bucket" and 1.8 * (1 << bbits) >= S["dim"] and n_stash <= S["dim"]
    st, nm = gpu_basis_numpy(S["B"])
    assert S["dim"] == len(S["st"]) == oracle.sector_dim(S["G"], case[2])
    assert np.array_equal(st, S["st"])
    assert np.array_equal(nm, S["nm"])


@pytest.mark.parametrize("case", SECTORS, ids=[s[0] for s in SECTORS])
def test_index_bit_exact(case):
    torch, ed = gpu()
    S = make(case)
    st = S["st"]
    n = case[1]
    rng = np.random.default_rng(5)
    # every basis state, plus random states (mostly absent) and edge values
    extra = rng.integers(0, 1 << min(n, 62), size=2000, dtype=np.int64).astype(np.uint64)
    q = np.concatenate([st, extra, np.array([0, (1 << n) - 1], np.uint64)])
    got = ed.basis_index(S["B"], to_torch(q.view(np.int64), np.int64)).cpu().numpy()
    pos = np.searchsorted(st, q)
    want = np.where((pos < len(st)) & (st[np.minimum(pos, max(len(st) - 1, 0))] == q), pos, -1) \
        if len(st) else np.full(len(q), -1)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("case", SECTORS, ids=[s[0] for s in SECTORS])
@pytest.mark.parametrize("nvec", [1, 3, 8])
def test_matvec_f64_parity(case, nvec):
    torch, ed = gpu()
    S = make(case)
    if S["dim"] == 0:
        pytest.skip("empty sector")
    cplx = not ed.basis_is_real(S["B"])
    x = ei.x_by_index(17, S["dim"], nvec, cplx)
    want = oracle.matvec(S["G"], S["H"], S["st"], S["nm"], x)
    dt = np.complex128 if cplx else np.float64
    xt = to_torch(x, dt)
    yt = torch.empty_like(xt)
    ed.matvec(S["O"], S["B"], xt, yt, nvec)
    got = yt.cpu().numpy()
    assert rel_err(got, want if cplx else want.real) < F64_TOL
    # element-wise, where a relative error is meaningful
    assert elem_rel_err(got, want if cplx else want.real, 1e-3) < 1e-9
    # determinism: a second product is bit-identical
    y2 = torch.empty_like(xt)
    ed.matvec(S["O"], S["B"], xt, y2, nvec)
    assert torch.equal(yt, y2)


@pytest.mark.parametrize("case", SECTORS[:9], ids=[s[0] for s in SECTORS[:9]])
@pytest.mark.parametrize("nvec", [1, 8, 16])
def test_matvec_f32_error_bounded(case, nvec):
    torch, ed = gpu()
    S = make(case)
    cplx = not ed.basis_is_real(S["B"])
    x = ei.x_by_index(3, S["dim"], nvec, cplx)
    want = oracle.matvec(S["G"], S["H"], S["st"], S["nm"], x)
    dt = np.complex64 if cplx else np.float32
    xt = to_torch(x, dt)
    yt = torch.empty_like(xt)
    ed.matvec(S["O"], S["B"], xt, yt, nvec)
    err = rel_err(yt.cpu().numpy().astype(np.complex128), want if cplx else want.real)
    assert err < F32_TOL, err


@pytest.mark.parametrize("name", ["ring16_k0_p+_z+", "ring20_k0_p-_z-", "ring40_nup2_k0_p+"])
def test_term_parallel_block_columns_equal_single_products(name, search_mode):
    """The term-parallel kernel on a real block of 8 vectors sums every
    column in the order of its single-vector form: columns equal the
    term-parallel single products bit for bit, in fp64 and fp32."""
    if search_mode != "term_parallel":
        pytest.skip("runs once, with the term-parallel kernel forced")
    torch, ed = gpu()
    case = [c for c in SECTORS if c[0] == name][0]
    S = make(case, with_oracle=False)
    for np_dt in (np.float64, np.float32):
        x = to_torch(ei.x_by_index(23, S["dim"], 8, False).real, np_dt)
        y = torch.empty_like(x)
        ed.matvec(S["O"], S["B"], x, y, 8)
        for v in range(8):
            xv = x[:, v].contiguous()
            yv = torch.empty_like(xv)
            ed.matvec(S["O"], S["B"], xv, yv, 1)
            assert torch.equal(yv, y[:, v])


def test_matvec_nvec_columns_equal_single_products(search_mode):
    """Block products equal the single products of the row-per-lane kernel bit
    for bit (same per-row summation order), and those of the term-parallel
    kernel to rounding."""
    torch, ed = gpu()
    S = make(SECTORS[7], with_oracle=False)
    x = ei.x_by_index(9, S["dim"], 5, True)
    xt = to_torch(x, np.complex128)
    yt = torch.empty_like(xt)
    ed.matvec(S["O"], S["B"], xt, yt, 5)
    for v in range(5):
        xv = xt[:, v].contiguous()
        yv = torch.empty_like(xv)
        ed.kernel_policy("rowwise")
        try:
            ed.matvec(S["O"], S["B"], xv, yv, 1)
        finally:
            ed.kernel_policy(search_mode if search_mode in ("rowwise", "term_parallel") else "auto")
        assert torch.equal(yv, yt[:, v])
        ed.matvec(S["O"], S["B"], xv, yv, 1)
        assert float((yv - yt[:, v]).abs().max()) <= 1e-13 * float(yt[:, v].abs().max())


@pytest.mark.parametrize("case", SECTORS, ids=[s[0] for s in SECTORS])
def test_term_parallel_matches_rowwise(case, search_mode):
    """The term-parallel kernel (one vector) against the row-per-lane kernel:
    fp64 to 1e-13 of max|y| (summation order only), fp32 to 1e-6."""
    if search_mode != "factored":
        pytest.skip("compared once")
    torch, ed = gpu()
    S = make(case, with_oracle=False)
    if S["dim"] == 0:
        pytest.skip("empty sector")
    cplx = not ed.basis_is_real(S["B"])
    for dt, tol in (((np.complex128 if cplx else np.float64), 1e-13), ((np.complex64 if cplx else np.float32), 1e-6)):
        xt = to_torch(ei.x_by_index(29, S["dim"], 1, cplx)[:, 0], dt)
        y_tp, y_rw = torch.empty_like(xt), torch.empty_like(xt)
        ed.kernel_policy("term_parallel")
        try:
            ed.matvec(S["O"], S["B"], xt, y_tp, 1)
            ed.kernel_policy("rowwise")
            ed.matvec(S["O"], S["B"], xt, y_rw, 1)
        finally:
            ed.kernel_policy("auto")
        scale = float(y_rw.abs().max())
        assert float((y_tp - y_rw).abs().max()) <= tol * max(scale, 1e-300)


def test_argument_errors():
    torch, ed = gpu()
    S = make(SECTORS[0], with_oracle=False)
    x = torch.zeros(S["dim"], dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(ed.EDError) as e:
        ed.matvec(S["O"], S["B"], x, y, 17)
    assert e.value.status == 1
    with pytest.raises(ed.EDError):
        ed.matvec(S["O"], S["B"], x, x, 1)                  # aliasing
    xs = torch.zeros(S["dim"] + 1, dtype=torch.float64, device="cuda")[1:]
    with pytest.raises(ed.EDError):
        ed.matvec(S["O"], S["B"], xs, y, 1)                 # misaligned
    # complex sector with a real dtype
    C = make(SECTORS[3], with_oracle=False)
    xr = torch.zeros(C["dim"], dtype=torch.float64, device="cuda")
    with pytest.raises(ed.EDError):
        ed.matvec(C["O"], C["B"], xr, torch.zeros_like(xr), 1)
    # operator that breaks the lattice symmetry
    op = ei.heisenberg_ring(16)
    op["coeff"][0, 0] = 2.0
    O2 = ed.operator_create(16, op["sites"], op["coeff"], op["local"])
    with pytest.raises(ed.EDError) as e:
        ed.matvec(O2, S["B"], x, y, 1)
    assert e.value.status == 4
    # operator on a different number of sites
    O3 = ed.operator_create(12, ei.heisenberg_ring(12)["sites"], ei.heisenberg_ring(12)["coeff"],
                            ei.heisenberg_ring(12)["local"])
    with pytest.raises(ed.EDError):
        ed.matvec(O3, S["B"], x, y, 1)
    # group errors
    p, c = ei.ring_group(8, 1)
    with pytest.raises(ed.EDError) as e:
        ed.basis_build(8, 4, 0, p[:4], c[:4])
    assert e.value.status == 2


# ----------------------------------------------------------------------------
# the full-size ring N=32 sector (k=0, p=+1, z=+1): counts against the
# character formula, sampled elements against the oracle one by one
# ----------------------------------------------------------------------------
@pytest.fixture(scope="module")
def ring32():
    w = ei.workload("ring32")
    S = build_pair(32, 16, +1, w["perms"], w["chars"], w["op"], with_oracle=False)
    S["G"] = oracle.Group(32, w["perms"], w["chars"], +1)
    S["H"] = oracle.Operator(w["op"])
    return S


def test_ring32_basis(ring32):
    S = ring32
    assert S["dim"] == oracle.sector_dim(S["G"], 16) == 4707969
    st, nm = gpu_basis_numpy(S["B"])
    assert np.all(np.diff(st.astype(np.int64)) > 0)
    assert all(bin(int(s)).count("1") == 16 for s in st[:: len(st) // 500])
    rng = np.random.default_rng(1)
    idx = np.concatenate([[0, len(st) - 1], rng.integers(0, len(st), 300)])
    for i in idx:
        rep, chi, norm, _ = oracle.state_info(S["G"], int(st[i]))
        assert rep == int(st[i]) and norm == int(nm[i]) and norm > 0
    # random states of the right popcount: in the basis iff the oracle says so
    torch, ed = gpu()
    cand = []
    while len(cand) < 300:
        bits = rng.choice(32, 16, replace=False)
        cand.append(sum(1 << int(b) for b in bits))
    q = np.array(cand, np.uint64)
    got = ed.basis_index(S["B"], to_torch(q.view(np.int64), np.int64)).cpu().numpy()
    for s, j in zip(cand, got):
        rep, _, norm, _ = oracle.state_info(S["G"], s)
        assert (j >= 0) == (rep == s and norm > 0)
        if j >= 0:
            assert int(st[j]) == s


def test_ring32_matvec_sampled_rows(ring32):
    torch, ed = gpu()
    S = ring32
    st, _ = gpu_basis_numpy(S["B"])
    x = ei.x_by_state(23, st)
    xt = to_torch(x, np.float64)
    yt = torch.empty_like(xt)
    ed.matvec(S["O"], S["B"], xt, yt, 1)
    y = yt.cpu().numpy()[:, 0]
    rng = np.random.default_rng(2)
    idx = np.concatenate([[0, len(st) - 1], rng.integers(0, len(st), 400)])
    want, _ = oracle.rows_statex(S["G"], S["H"], st[idx], 23)
    assert rel_err(y[idx], want[:, 0].real) < F64_TOL
    # fp32 on the same rows
    xf = to_torch(x, np.float32)
    yf = torch.empty_like(xf)
    ed.matvec(S["O"], S["B"], xf, yf, 1)
    assert rel_err(yf.cpu().numpy()[idx, 0].astype(np.float64), want[:, 0].real) < F32_TOL


def test_stream_status_clean_after_work():
    torch, ed = gpu()
    S = make(SECTORS[0], with_oracle=False)
    x = torch.ones(S["dim"], dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    ed.matvec(S["O"], S["B"], x, y, 1)
    assert ed.stream_status() == 0


@pytest.mark.parametrize("case", SECTORS[:9], ids=[s[0] for s in SECTORS[:9]])
def test_nnz_count_matches_oracle(case):
    torch, ed = gpu()
    S = make(case)
    # off-diagonal terms whose representative has nonzero norm, plus one
    # diagonal entry per row (the oracle's per-row count)
    _, nnz = oracle.rows_statex(S["G"], S["H"], S["st"], 0)
    assert ed.count_nnz(S["O"], S["B"]) == int(nnz.sum())
