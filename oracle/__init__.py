"""Plain CPU oracle for the symmetry-adapted spin-1/2 ED hot path.

TEST INFRASTRUCTURE ONLY: tests/, the smoke check and the benchmark's
cpu_baseline / reference legs may use it; the product path never does.  It
shares no code with the CUDA path (the only common import is ``ed_inputs``,
which generates problems and random inputs and holds none of the method's
arithmetic).

Layers:

* ``ed_oracle.c`` (plain C, fp64/complex128): group action bit by bit,
  brute-force representative and orbit norm, ascending enumeration of the
  U(1) sector, the pull-form matrix elements and y = Hx (Sec. "Matrix-vector
  product"), rows evaluated from states alone.
* this module: ctypes marshalling, spin-inversion expansion of the group,
  the character-formula sector dimension, the sector matrix as a scipy sparse
  matrix, dense diagonalisation (numpy ``eigvalsh``) and a plain fp64 Lanczos
  whose tridiagonal problem is solved by ``scipy.linalg.eigh_tridiagonal``;
  the Ritz values of a block Krylov space by Rayleigh-Ritz (the definition
  block Lanczos computes).

Functions without an independent pin are marked "parity unpinned" in their
docstring.  (At present every function has at least one pin in
tests/test_oracle_pins.py.)
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from collections import defaultdict

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ed_oracle.c")
_LIB = os.path.join(_HERE, "libedoracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile ed_oracle.c with the host C compiler (plain -O2, no vectorisation
    flags, portable to x86-64 and aarch64)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i64, i32, u64 = ctypes.c_int64, ctypes.c_int, ctypes.c_uint64
        L.orc_apply.restype = u64
        L.orc_apply.argtypes = [i32, P, i32, u64]
        L.orc_state_info.restype = i32
        L.orc_state_info.argtypes = [i32, i32, P, P, P, u64, P, P, P, P]
        L.orc_enumerate.restype = i64
        L.orc_enumerate.argtypes = [i32, i32, i32, P, P, P, P, P, i64]
        L.orc_enumerate_slice.restype = i64
        L.orc_enumerate_slice.argtypes = [i32, i32, i32, P, P, P, u64, i64, P]
        L.orc_matvec.restype = i32
        L.orc_matvec.argtypes = [i32, i32, P, P, P, i32, P, P, P, P, P, i64, i32, P, P]
        L.orc_coo.restype = i64
        L.orc_coo.argtypes = [i32, i32, P, P, P, i32, P, P, P, P, P, i64, P, P, P, i64]
        L.orc_rows_statex.restype = i32
        L.orc_rows_statex.argtypes = [i32, i32, P, P, P, i32, P, P, P, P, i64, u64, i32, i32, P, P]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


class Group:
    """The symmetry group with spin inversion expanded.

    Every user element g = (perm, chi) appears once unflipped and, when
    spin_inversion = z != 0, once more flipped with character chi(g) * z
    (the full group is the direct product of the lattice group and {1, F}).
    """

    def __init__(self, n_sites: int, perms, chars, spin_inversion: int = 0):
        perms = np.ascontiguousarray(np.asarray(perms, dtype=np.int32).reshape(-1, n_sites))
        chars = np.asarray(chars, dtype=np.float64).reshape(-1, 2)
        chi = chars[:, 0] + 1j * chars[:, 1]
        if spin_inversion:
            perms = np.concatenate([perms, perms])
            flips = np.concatenate([np.zeros(len(chi), np.uint8), np.ones(len(chi), np.uint8)])
            chi = np.concatenate([chi, chi * spin_inversion])
        else:
            flips = np.zeros(len(chi), np.uint8)
        self.n = n_sites
        self.perm = np.ascontiguousarray(perms)
        self.flip = np.ascontiguousarray(flips)
        self.chi = np.ascontiguousarray(np.stack([chi.real, chi.imag], axis=1))
        self.order = len(flips)

    def args(self):
        return (self.n, self.order, _p(self.perm), _p(self.flip), _p(self.chi))


class Operator:
    def __init__(self, op: dict):
        self.sites = np.ascontiguousarray(np.asarray(op["sites"], dtype=np.int32).reshape(-1, 2))
        self.coeff = np.ascontiguousarray(np.asarray(op["coeff"], dtype=np.float64).reshape(-1, 2))
        self.local = np.ascontiguousarray(np.asarray(op["local"], dtype=np.float64).reshape(-1, 16, 2))
        self.n_terms = len(self.sites)

    def args(self):
        return (self.n_terms, _p(self.coeff), _p(self.sites), _p(self.local))


def apply(n: int, perm, flip: int, s: int) -> int:
    perm = np.ascontiguousarray(np.asarray(perm, dtype=np.int32))
    return int(lib().orc_apply(n, _p(perm), int(flip), int(s)))


def state_info(G: Group, s: int):
    """(rep, chi(g*) complex, norm, stabilizer character sum complex)."""
    rep = np.zeros(1, np.uint64)
    chs = np.zeros(2)
    nrm = np.zeros(1, np.int32)
    ss = np.zeros(2)
    rc = lib().orc_state_info(*G.args(), int(s), _p(rep), _p(chs), _p(nrm), _p(ss))
    if rc != 0:
        raise RuntimeError("argmins with different characters at nonzero norm")
    return int(rep[0]), complex(chs[0], chs[1]), int(nrm[0]), complex(ss[0], ss[1])


def enumerate_basis(G: Group, n_up: int):
    """Ascending representatives with nonzero norm and their integer norms
    (Sec. "States enumeration" filter, done by brute force)."""
    L = lib()
    cnt = L.orc_enumerate(*G.args()[:1], n_up, *G.args()[1:], None, None, 0)
    if cnt < 0:
        raise ValueError("bad enumeration arguments")
    states = np.zeros(max(cnt, 1), np.uint64)
    norms = np.zeros(max(cnt, 1), np.uint16)
    got = L.orc_enumerate(G.n, n_up, G.order, _p(G.perm), _p(G.flip), _p(G.chi),
                          _p(states), _p(norms), cnt)
    assert got == cnt
    return states[:cnt], norms[:cnt]


def enumerate_slice(G: Group, n_up: int, first_state: int, count: int):
    """Filter `count` consecutive states of popcount n_up from first_state;
    returns (states visited, representatives kept)."""
    kept = np.zeros(1, np.int64)
    done = lib().orc_enumerate_slice(G.n, n_up, G.order, _p(G.perm), _p(G.flip), _p(G.chi),
                                     int(first_state), int(count), _p(kept))
    if done < 0:
        raise ValueError("first_state has the wrong popcount")
    return int(done), int(kept[0])


def matvec(G: Group, H: Operator, states, norms, x):
    """y = H x over the basis (complex128; x may be real). x shape (dim,) or (dim, nvec)."""
    x = np.asarray(x)
    squeeze = x.ndim == 1
    xv = x.reshape(len(states), -1)
    nvec = xv.shape[1]
    xc = np.ascontiguousarray(xv.astype(np.complex128)).view(np.float64)
    y = np.zeros((len(states), nvec), np.complex128)
    st = np.ascontiguousarray(states, dtype=np.uint64)
    nm = np.ascontiguousarray(norms, dtype=np.uint16)
    rc = lib().orc_matvec(*G.args(), *H.args(), _p(st), _p(nm), len(st), nvec, _p(xc),
                          _p(y.view(np.float64)))
    if rc != 0:
        raise RuntimeError(f"oracle matvec failed ({rc})")
    return y[:, 0] if squeeze else y


def coo(G: Group, H: Operator, states, norms):
    """Sector matrix entries (rows, cols, complex vals), duplicates not merged."""
    L = lib()
    st = np.ascontiguousarray(states, dtype=np.uint64)
    nm = np.ascontiguousarray(norms, dtype=np.uint16)
    total = L.orc_coo(*G.args(), *H.args(), _p(st), _p(nm), len(st), None, None, None, 0)
    if total < 0:
        raise RuntimeError(f"oracle coo failed ({total})")
    r = np.zeros(max(total, 1), np.int64)
    c = np.zeros(max(total, 1), np.int64)
    v = np.zeros(max(total, 1), np.complex128)
    got = L.orc_coo(*G.args(), *H.args(), _p(st), _p(nm), len(st), _p(r), _p(c),
                    _p(v.view(np.float64)), total)
    assert got == total
    return r[:total], c[:total], v[:total]


def sparse_matrix(G: Group, H: Operator, states, norms):
    import scipy.sparse as sp
    r, c, v = coo(G, H, states, norms)
    d = len(states)
    return sp.coo_matrix((v, (r, c)), shape=(d, d)).tocsr()


def dense_matrix(G: Group, H: Operator, states, norms):
    return sparse_matrix(G, H, states, norms).toarray()


def rows_statex(G: Group, H: Operator, row_states, seed: int, nvec: int = 1,
                complex_: bool = False):
    """y(r) for representative row states r with x keyed by the state (the
    ``ed_inputs.x_by_state`` vector).  Returns (y [rows, nvec] complex, nnz per row)."""
    rs = np.ascontiguousarray(np.asarray(row_states, dtype=np.uint64))
    y = np.zeros((len(rs), nvec), np.complex128)
    nnz = np.zeros(len(rs), np.int32)
    rc = lib().orc_rows_statex(*G.args(), *H.args(), _p(rs), len(rs), int(seed), nvec,
                               int(complex_), _p(y.view(np.float64)), _p(nnz))
    if rc != 0:
        raise RuntimeError(f"oracle rows failed ({rc})")
    return y, nnz


# ----------------------------------------------------------------------------
# sector dimension by the character (projection) formula
# ----------------------------------------------------------------------------
def _cycles(perm):
    n = len(perm)
    seen = [False] * n
    out = []
    for i in range(n):
        if not seen[i]:
            length, j = 0, i
            while not seen[j]:
                seen[j] = True
                j = int(perm[j])
                length += 1
            out.append(length)
    return out


def _fixed_count(perm, flip: int, n_up: int) -> int:
    """Number of states with popcount n_up (any, if n_up < 0) fixed by g."""
    cyc = _cycles(perm)
    n = len(perm)
    if flip:
        # s fixed by "permute then complement": bits alternate along each cycle,
        # so every cycle must be even and contributes exactly half its sites up.
        if any(c % 2 for c in cyc):
            return 0
        if n_up >= 0 and 2 * n_up != n:
            return 0
        return 2 ** len(cyc)
    if n_up < 0:
        return 2 ** len(cyc)
    # coefficient of t^n_up in prod_c (1 + t^c): a cycle is all-up or all-down
    poly = [1] + [0] * n_up
    for c in cyc:
        for k in range(n_up, c - 1, -1):
            poly[k] += poly[k - c]
    return poly[n_up]


def sector_dim(G: Group, n_up: int) -> int:
    """D = |G|^-1 sum_g conj(chi(g)) fix(g): the trace of the sector projector
    restricted to the U(1) sector (exact for one-dimensional characters)."""
    by_chi = defaultdict(int)
    for g in range(G.order):
        f = _fixed_count(G.perm[g], int(G.flip[g]), n_up)
        if f:
            key = (round(G.chi[g, 0], 12), round(G.chi[g, 1], 12))
            by_chi[key] += f
    if all(abs(im) < 1e-12 and abs(abs(re) - 1) < 1e-12 for re, im in by_chi):
        total = sum(int(round(re)) * f for (re, _), f in by_chi.items())
        assert total % G.order == 0, "character sum not divisible by |G|"
        return total // G.order
    total = math.fsum(re * f for (re, _), f in by_chi.items())
    d = total / G.order
    assert abs(d - round(d)) < 1e-6 * max(1.0, abs(d)), d
    return int(round(d))


# ----------------------------------------------------------------------------
# eigenvalues
# ----------------------------------------------------------------------------
def lanczos(apply_h, v0, steps: int, reorth: bool = False):
    """Plain fp64 Lanczos: v_0 = v0/|v0|; w = H v_j - alpha_j v_j - beta_j v_{j-1};
    beta_{j+1} = |w|.  Returns (alphas, betas, lowest Ritz value).  With
    ``reorth`` every w is re-orthogonalised against all earlier v (modified
    Gram-Schmidt -- each coefficient taken from the already updated w -- in
    two passes)."""
    from scipy.linalg import eigh_tridiagonal
    v = v0 / np.linalg.norm(v0)
    vprev = np.zeros_like(v)
    alphas, betas = [], []
    beta = 0.0
    basis = [v]
    for _ in range(steps):
        w = apply_h(v)
        alpha = np.vdot(v, w).real
        w = w - alpha * v - beta * vprev
        if reorth:
            for _ in range(2):
                for u in basis:
                    w = w - np.vdot(u, w) * u
        alphas.append(alpha)
        beta = np.linalg.norm(w)
        if beta == 0.0:
            break
        betas.append(beta)
        vprev, v = v, w / beta
        if reorth:
            basis.append(v)
    a = np.array(alphas)
    b = np.array(betas[: len(alphas) - 1])
    e0 = eigh_tridiagonal(a, b, eigvals_only=True)[0]
    return a, b, float(e0)


def block_krylov_ritz(apply_h, X0, m: int, rank_tol: float = 1e-12):
    """Ritz values, ascending, of the block Krylov space
    K_m(H, X0) = span{X0, H X0, ..., H^(m-1) X0}: the eigenvalues of Q^T H Q
    for an orthonormal basis Q of the space (Rayleigh-Ritz).  These are the
    values block Lanczos with m steps produces in exact arithmetic (Krylov
    methods consume products, Background).  apply_h maps an (n, k) array to
    H times it; H real symmetric.

    Q is built block by block: the newest block times H, orthogonalised
    against every earlier block (block Gram-Schmidt, twice), then numpy's
    Householder QR; directions whose R diagonal falls below rank_tol of the
    block's size before the projections are dropped (the space stops
    growing)."""
    blocks = []
    V = np.array(X0, dtype=np.float64, copy=True)
    for _ in range(m):
        scale = max(float(np.abs(V).max()) if V.size else 0.0, 1e-300)  # before the projections
        for _pass in range(2):
            for Bk in blocks:
                V = V - Bk @ (Bk.T @ V)
        Qj, R = np.linalg.qr(V)
        d = np.abs(np.diag(R))
        keep = d > rank_tol * scale * np.sqrt(V.shape[0])
        Qj = Qj[:, keep]
        if Qj.shape[1] == 0:
            break
        blocks.append(Qj)
        V = apply_h(Qj)
    Q = np.hstack(blocks)
    T = Q.T @ apply_h(Q)
    return np.linalg.eigvalsh(0.5 * (T + T.T))
