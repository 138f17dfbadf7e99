"""Host-side checks of the C-ABI library that need no GPU: it loads, exports
every entry point include/ed.h declares, validates groups and operators before
any CUDA call, and its Benes routing realises the permutations it is given."""
import ctypes
import os
import re

import numpy as np
import pytest

import ed_inputs as ei

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2308_16712_gb300 import build
    if not os.path.exists(build.LIB):
        build.build()
    from paper_2308_16712_gb300 import ed
    return ed._lib


def header_functions():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names += re.findall(r"\b(ed_[a-z0-9_]+)\s*\(", txt)
    return sorted(set(names))


def test_library_exports_every_declared_function(lib):
    names = header_functions()
    assert "ed_matvec" in names and "ed_basis_build" in names and "ed_lanczos" in names
    for n in names:
        assert hasattr(lib, n), n


def test_status_strings(lib):
    from paper_2308_16712_gb300 import ed
    for code in range(10):
        assert ed.status_string(code) != "unknown status"


# ----------------------------------------------------------------------------
# Benes routing
# ----------------------------------------------------------------------------
def apply_masks(x, masks, log2w):
    w = 1 << log2w
    full = (1 << w) - 1
    for i, m in enumerate(masks):
        d = 1 << (log2w - 1 - i) if i < log2w else 1 << (i - log2w + 1)
        t = ((x >> d) ^ x) & int(m)
        x = (x ^ t ^ (t << d)) & full
    return x


def permute_bits(x, perm):
    out = 0
    for i, p in enumerate(perm):
        if (x >> i) & 1:
            out |= 1 << int(p)
    return out


@pytest.mark.parametrize("log2w,n", [(5, 32), (5, 17), (6, 64), (6, 40), (6, 36), (5, 2), (6, 1)])
def test_benes_masks_realise_permutations(lib, log2w, n):
    rng = np.random.default_rng(log2w * 100 + n)
    masks = np.zeros(16, np.uint64)
    for trial in range(40):
        perm = np.ascontiguousarray(rng.permutation(n).astype(np.int32))
        k = lib.edx_benes_masks(log2w, n, perm.ctypes.data_as(ctypes.c_void_p),
                                masks.ctypes.data_as(ctypes.c_void_p))
        assert k == 2 * log2w - 1
        for _ in range(20):
            x = int(rng.integers(0, 1 << min(n, 63))) | (int(rng.integers(0, 2)) << (n - 1))
            assert apply_masks(x, masks[:k], log2w) == permute_bits(x, perm)


def test_benes_masks_lattice_groups(lib):
    masks = np.zeros(16, np.uint64)
    for perms, n in [(ei.ring_group(32, 0, +1)[0], 32), (ei.torus_group(6, 6)[0], 36),
                     (ei.ring_group(40, 0, +1)[0], 40)]:
        log2w = 5 if n <= 32 else 6
        rng = np.random.default_rng(n)
        for p in perms:
            p = np.ascontiguousarray(p.astype(np.int32))
            k = lib.edx_benes_masks(log2w, n, p.ctypes.data_as(ctypes.c_void_p),
                                    masks.ctypes.data_as(ctypes.c_void_p))
            for _ in range(5):
                x = int(rng.integers(0, 1 << n))
                assert apply_masks(x, masks[:k], log2w) == permute_bits(x, p)


# ----------------------------------------------------------------------------
# group validation (ED_ERR_NOT_A_GROUP = 2, ED_ERR_BAD_CHARACTER = 3)
# ----------------------------------------------------------------------------
def validate(lib, perms, chars):
    perms = np.ascontiguousarray(np.asarray(perms, np.int32))
    chars = np.ascontiguousarray(np.asarray(chars, np.float64).reshape(-1, 2))
    return lib.edx_validate_group(perms.shape[1], perms.shape[0],
                                  perms.ctypes.data_as(ctypes.c_void_p),
                                  chars.ctypes.data_as(ctypes.c_void_p))


def test_group_validation(lib):
    p, c = ei.ring_group(8, 3)
    assert validate(lib, p, c) == 0
    p, c = ei.ring_group(8, 0, -1)
    assert validate(lib, p, c) == 0
    p, c = ei.torus_group(4, 3, 1, 2)
    assert validate(lib, p, c) == 0
    p, c = ei.ring_group(8, 1)
    assert validate(lib, p[1:], c[1:]) == 2                       # no identity
    assert validate(lib, p[:5], c[:5]) == 2                       # not closed
    assert validate(lib, np.concatenate([p, p[:1]]), np.concatenate([c, c[:1]])) == 2  # repeat
    bad = p.copy()
    bad[2, 0] = bad[2, 1]
    assert validate(lib, bad, c) == 2                             # not a permutation
    c2 = c.copy()
    c2[3] *= 1.5
    assert validate(lib, p, c2) == 3                              # |chi| != 1
    c3 = c.copy()
    c3[3] = [1.0, 0.0]
    assert validate(lib, p, c3) == 3                              # not a homomorphism
    # a dihedral group with a momentum other than 0 or pi has no 1-d character
    p4, c4 = ei.ring_group(8, 0, +1)
    ph = np.exp(-2j * np.pi * 1 * np.arange(8) / 8)
    chi = np.concatenate([ph, ph])
    assert validate(lib, p4, np.stack([chi.real, chi.imag], 1)) == 3


# ----------------------------------------------------------------------------
# operator symmetry check
# ----------------------------------------------------------------------------
def commutes(lib, n, op, perms, z):
    args = [np.ascontiguousarray(op[k]) for k in ("coeff", "sites", "local")]
    perms = np.ascontiguousarray(np.asarray(perms, np.int32))
    return lib.edx_terms_commute(n, len(op["sites"]), *[a.ctypes.data_as(ctypes.c_void_p) for a in args],
                                 perms.shape[0], perms.ctypes.data_as(ctypes.c_void_p), z)


def test_operator_symmetry_check(lib):
    p, _ = ei.ring_group(12, 0, +1)
    assert commutes(lib, 12, ei.heisenberg_ring(12), p, +1) == 1
    assert commutes(lib, 12, ei.xxz_ring(12, 1.0, 1.5), p, -1) == 1
    op = ei.heisenberg_ring(12)
    op["coeff"][3, 0] = 1.1                                       # breaks translations
    assert commutes(lib, 12, op, p, 0) == 0
    # reversed bond orientation describes the same operator
    op = ei.heisenberg_ring(12)
    op["sites"] = np.ascontiguousarray(op["sites"][:, ::-1])
    assert commutes(lib, 12, op, p, +1) == 1
    pt, _ = ei.torus_group(6, 6)
    assert commutes(lib, 36, ei.j1j2_torus(6, 6, 1.0, 0.5), pt, +1) == 1
    # an Sz_i Sx_j coupling is translation invariant but odd under spin inversion
    loc = np.zeros((4, 4))
    sz = np.diag([-0.5, 0.5])
    sx = np.array([[0, 0.5], [0.5, 0]])
    loc[:] = np.kron(sz, sx)
    op = ei.make_operator([(i, (i + 1) % 12) for i in range(12)], [1.0] * 12, loc)
    pr, _ = ei.ring_group(12, 0)
    assert commutes(lib, 12, op, pr, 0) == 1
    assert commutes(lib, 12, op, pr, +1) == 0


def test_argument_errors_before_any_launch(lib):
    from paper_2308_16712_gb300 import ed
    P = ctypes.c_void_p
    out = P()
    p, c = ei.ring_group(8, 0)
    pp = np.ascontiguousarray(p)
    cc = np.ascontiguousarray(c)
    call = lambda n, nup, z, ne: lib.ed_basis_build(n, nup, z, ne, pp.ctypes.data_as(P),
                                                    cc.ctypes.data_as(P), None, ctypes.byref(out))
    assert call(0, 0, 0, 8) == 1
    assert call(65, 0, 0, 8) == 1
    assert call(8, 9, 0, 8) == 1
    assert call(8, 3, 1, 8) == 1            # spin inversion outside Sz = 0
    assert call(8, 4, 2, 8) == 1
    assert call(8, 4, 0, 7) == 2            # truncated group is not closed
    assert lib.ed_matvec(None, None, None, None, 1, 0, None) == 1
    assert lib.ed_basis_size(None, None) == 1
    assert lib.ed_lanczos(None, None, None, 10, 0, None, None, None, None) == 1
    # invalid operator terms: a site out of range, a repeated site
    sites = np.ascontiguousarray(np.array([[0, 8]], np.int32))
    loc = np.ascontiguousarray(np.zeros((1, 16, 2)))
    co = np.ascontiguousarray(np.ones((1, 2)))
    assert lib.ed_operator_create(8, 1, co.ctypes.data_as(P), sites.ctypes.data_as(P),
                                  loc.ctypes.data_as(P), ctypes.byref(out)) == 1
    sites[0] = [3, 3]
    assert lib.ed_operator_create(8, 1, co.ctypes.data_as(P), sites.ctypes.data_as(P),
                                  loc.ctypes.data_as(P), ctypes.byref(out)) == 1


def test_noalloc_count_rejects_sectors_beyond_its_bound(lib):
    """The allocation-free count has a fixed scratch: at most 2^18 chunks of at
    most 2^24 states.  A larger sector (C(64, 32) = 1.8e18 states) returns
    ED_ERR_UNSUPPORTED before any CUDA call (this host has no GPU), and so does
    C(46, 23) = 8.2e12 > 2^42; the group validation still comes first."""
    P = ctypes.c_void_p
    dim = ctypes.c_uint64(0)
    for n in (64, 46):
        p, c = ei.ring_group(n, 0, +1)
        pp, cc = np.ascontiguousarray(p), np.ascontiguousarray(c)
        st = lib.ed_basis_count_noalloc(n, n // 2, 1, len(p), pp.ctypes.data_as(P), cc.ctypes.data_as(P),
                                        None, ctypes.byref(dim))
        assert st == 9, (n, st)
    p, c = ei.ring_group(64, 0, +1)
    pp, cc = np.ascontiguousarray(p[:5]), np.ascontiguousarray(c[:5])  # not a group
    assert lib.ed_basis_count_noalloc(64, 32, 1, 5, pp.ctypes.data_as(P), cc.ctypes.data_as(P), None,
                                      ctypes.byref(dim)) == 2


# ----------------------------------------------------------------------------
# factored form of lattice groups (rotation subgroup x coset representatives)
# ----------------------------------------------------------------------------
def factorize(lib, perms):
    perms = np.ascontiguousarray(np.asarray(perms, np.int32))
    L, d = ctypes.c_int(), ctypes.c_int()
    kinds = np.zeros(len(perms), np.uint8)
    nc = lib.edx_factorize(perms.shape[1], perms.shape[0], perms.ctypes.data_as(ctypes.c_void_p),
                           ctypes.byref(L), ctypes.byref(d), kinds.ctypes.data_as(ctypes.c_void_p))
    return nc, L.value, d.value, list(kinds[:max(nc, 0)])


def test_factorization_of_lattice_groups(lib):
    assert factorize(lib, ei.ring_group(32, 0, +1)[0]) == (2, 32, 1, [0, 1])
    assert factorize(lib, ei.ring_group(40, 0, +1)[0]) == (2, 40, 1, [0, 1])
    assert factorize(lib, ei.ring_group(28, 3)[0]) == (1, 28, 1, [0])
    nc, L, d, kinds = factorize(lib, ei.torus_group(6, 6)[0])
    assert (nc, L, d) == (6, 6, 6) and kinds[0] == 0 and all(k == 2 for k in kinds[1:])
    assert factorize(lib, ei.trivial_group(10)[0])[0] == 0
    # the factored elements cover the group exactly once (checked through the
    # rotation closure: cosets x L = |G|)
    for p in (ei.ring_group(12, 0, -1)[0], ei.torus_group(3, 4)[0], ei.torus_group(4, 4)[0]):
        nc, L, d, _ = factorize(lib, p)
        assert nc * L == len(p)


def families(lib, n, op):
    args = [np.ascontiguousarray(op[k]) for k in ("coeff", "sites", "local")]
    return lib.edx_operator_families(n, len(op["sites"]), *[a.ctypes.data_as(ctypes.c_void_p) for a in args])


def test_operator_rotation_families(lib):
    # a ring: one family (offset 1, every site); the 6x6 J1-J2 torus: nearest
    # bonds at offsets 1 and 31 (row wrap) and 6, next-nearest at 7, 1, 31, 25
    assert families(lib, 32, ei.heisenberg_ring(32)) == 1
    assert families(lib, 36, ei.j1j2_torus(6, 6, 1.0, 0.5)) == 7
    # a repeated bond opens a second family of the same kind
    op = ei.heisenberg_ring(8)
    for k in ("sites", "coeff", "local"):
        op[k] = np.concatenate([op[k], op[k][:1]])
    assert families(lib, 8, op) == 2
