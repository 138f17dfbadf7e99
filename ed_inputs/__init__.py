"""Seeded, synthetic workload generators shared by the oracle side and the CUDA side.

This module describes *problems*, not how to solve them: lattice symmetry groups
(site permutations plus one-dimensional characters), two-spin Hamiltonian term
lists, and the random input vectors x.  It contains none of the method's
arithmetic (no representative search, no orbit norms, no matrix elements), so
both the oracle and the GPU path may import it without sharing any of the
computation they are compared on.

Conventions (the encoding the whole project uses):

* site i <-> bit i of a uint64 state (LSB = site 0), bit value 1 = spin up;
* a permutation is an int32 row ``perm`` with "site i goes to site perm[i]";
* a character is a complex number per group element, given as (re, im);
* a two-spin term is (coefficient c, sites (i, j), local 4x4 matrix h) acting on
  |s_i s_j> with row/column index 2*s_i + s_j.

The random vector uses the 64-bit mixing function printed in the paper's
"Hashed distribution" subsection (there it maps basis states to locales; here it
is the counter-based generator):  u = (hash64_01(seed + c * 0x9E3779B97F4A7C15)
>> 11) * 2**-53 and x = 2u - 1, for counter c.  Real vectors use c = i*nvec + v;
complex vectors use 2c for the real part and 2c + 1 for the imaginary part.
"""
from __future__ import annotations

import math

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


# ----------------------------------------------------------------------------
# counter-based random numbers
# ----------------------------------------------------------------------------
def hash64_01(x):
    """The paper's 64-bit mixer (Sec. "Hashed distribution"), vectorised, mod 2**64."""
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        x = (x ^ (x >> np.uint64(30))) * _M1
        x = (x ^ (x >> np.uint64(27))) * _M2
        x = x ^ (x >> np.uint64(31))
    return x


def uniform_pm1(seed: int, counters) -> np.ndarray:
    """Uniform numbers in [-1, 1) from 64-bit counters (fp64)."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        h = hash64_01(np.uint64(seed) + c * GOLDEN)
    u = (h >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return 2.0 * u - 1.0


def x_by_index(seed: int, dim: int, nvec: int = 1, complex_: bool = False,
               chunk: int = 1 << 24) -> np.ndarray:
    """x[i, v] keyed by the basis index i; shape (dim, nvec) (interleaved rows)."""
    dtype = np.complex128 if complex_ else np.float64
    out = np.empty((dim, nvec), dtype=dtype)
    for lo in range(0, dim, chunk):
        hi = min(dim, lo + chunk)
        c = (np.arange(lo, hi, dtype=np.uint64)[:, None] * np.uint64(nvec)
             + np.arange(nvec, dtype=np.uint64)[None, :])
        if complex_:
            out[lo:hi] = uniform_pm1(seed, 2 * c) + 1j * uniform_pm1(seed, 2 * c + 1)
        else:
            out[lo:hi] = uniform_pm1(seed, c)
    return out


def x_by_state(seed: int, states, nvec: int = 1, complex_: bool = False) -> np.ndarray:
    """x keyed by the basis *state* instead of its index; shape (len(states), nvec).

    Used at sizes where the oracle cannot enumerate the basis: a row of y = Hx
    can then be evaluated from states alone.
    """
    s = np.asarray(states, dtype=np.uint64)
    c = s[:, None] * np.uint64(nvec) + np.arange(nvec, dtype=np.uint64)[None, :]
    if complex_:
        return uniform_pm1(seed, 2 * c) + 1j * uniform_pm1(seed, 2 * c + 1)
    return uniform_pm1(seed, c)


def _hash64_torch(x):
    """hash64_01 on an int64 torch tensor holding uint64 bit patterns (logical
    shifts done as arithmetic shift + mask; multiplication wraps mod 2**64)."""
    import torch
    def srl(v, k):
        return (v >> k) & ((1 << (64 - k)) - 1)
    m1 = torch.tensor(np.int64(np.uint64(0xBF58476D1CE4E5B9).view(np.int64)), device=x.device)
    m2 = torch.tensor(np.int64(np.uint64(0x94D049BB133111EB).view(np.int64)), device=x.device)
    x = (x ^ srl(x, 30)) * m1
    x = (x ^ srl(x, 27)) * m2
    return x ^ srl(x, 31)


def x_by_state_torch(seed: int, states, nvec: int = 1, complex_: bool = False, dtype=None):
    """Device version of ``x_by_state`` for a torch int64 tensor of states (same
    numbers, computed where the states live)."""
    import torch
    golden = torch.tensor(np.int64(GOLDEN.view(np.int64)), device=states.device)
    seed_t = torch.tensor(np.int64(np.uint64(seed).view(np.int64)), device=states.device)
    c = states.reshape(-1, 1) * nvec + torch.arange(nvec, device=states.device).reshape(1, -1)

    def unif(cnt):
        h = _hash64_torch(seed_t + cnt * golden)
        u = ((h >> 11) & ((1 << 53) - 1)).to(torch.float64) * (2.0 ** -53)
        return 2.0 * u - 1.0

    if complex_:
        out = torch.complex(unif(2 * c), unif(2 * c + 1))
    else:
        out = unif(c)
    return out if dtype is None else out.to(dtype)


def x_by_state_torch_chunked(seed: int, states, nvec: int = 1, complex_: bool = False, dtype=None,
                             chunk: int = 1 << 26):
    """``x_by_state_torch`` computed ``chunk`` states at a time into one output
    (the same numbers; bounded temporaries for bases of billions of states)."""
    import torch
    if dtype is None:
        dtype = torch.complex128 if complex_ else torch.float64
    n = states.numel()
    out = torch.empty((n, nvec), dtype=dtype, device=states.device)
    for i in range(0, n, chunk):
        out[i:i + chunk] = x_by_state_torch(seed, states[i:i + chunk], nvec, complex_, dtype=dtype)
    return out


# ----------------------------------------------------------------------------
# symmetry groups (site permutations + characters)
# ----------------------------------------------------------------------------
def _chars(phases) -> np.ndarray:
    ph = np.asarray(phases, dtype=np.float64)
    return np.stack([np.cos(ph), np.sin(ph)], axis=1)


def ring_group(n: int, k: int = 0, parity=None):
    """Translations T^a (site i -> i + a mod n) of an n-site ring, optionally with
    the reflection R (site i -> -i mod n).

    k is the momentum index (momentum 2*pi*k/n); chi(T^a) = exp(-i 2 pi k a / n).
    With ``parity`` (+1 or -1) the group is dihedral, chi(T^a R) = chi(T^a) * parity;
    it is a one-dimensional representation only for k = 0 or k = n/2.
    Returns (perms int32 [G, n], chars float64 [G, 2]).
    """
    perms, phases, signs = [], [], []
    q = 2.0 * math.pi * k / n
    for a in range(n):
        perms.append([(i + a) % n for i in range(n)])
        phases.append(-q * a)
        signs.append(1.0)
    if parity is not None:
        if (2 * k) % n != 0:
            raise ValueError("reflection parity needs momentum 0 or pi")
        for a in range(n):
            perms.append([(a - i) % n for i in range(n)])
            phases.append(-q * a)
            signs.append(float(parity))
    ch = _chars(phases) * np.asarray(signs)[:, None]
    return np.asarray(perms, dtype=np.int32), ch


def torus_group(lx: int, ly: int, kx: int = 0, ky: int = 0):
    """Translations of an lx x ly periodic square lattice, site = x + lx*y.

    chi(Tx^a Ty^b) = exp(-i (2 pi kx a / lx + 2 pi ky b / ly)).
    """
    perms, phases = [], []
    for b in range(ly):
        for a in range(lx):
            p = []
            for y in range(ly):
                for x in range(lx):
                    p.append(((x + a) % lx) + lx * ((y + b) % ly))
            perms.append(p)
            phases.append(-(2.0 * math.pi * kx * a / lx + 2.0 * math.pi * ky * b / ly))
    return np.asarray(perms, dtype=np.int32), _chars(phases)


def trivial_group(n: int):
    """The one-element group (no lattice symmetry)."""
    return np.arange(n, dtype=np.int32)[None, :], np.array([[1.0, 0.0]])


# ----------------------------------------------------------------------------
# two-spin Hamiltonians
# ----------------------------------------------------------------------------
def heisenberg_local() -> np.ndarray:
    """S_i . S_j (S = sigma/2) on |s_i s_j>, index 2*s_i + s_j, as a real 4x4."""
    h = np.zeros((4, 4))
    h[0, 0] = h[3, 3] = 0.25
    h[1, 1] = h[2, 2] = -0.25
    h[1, 2] = h[2, 1] = 0.5
    return h


def xxz_local(jxy: float, delta: float) -> np.ndarray:
    """jxy (Sx Sx + Sy Sy) + delta * jxy * Sz Sz on |s_i s_j>."""
    h = np.zeros((4, 4))
    h[0, 0] = h[3, 3] = 0.25 * delta * jxy
    h[1, 1] = h[2, 2] = -0.25 * delta * jxy
    h[1, 2] = h[2, 1] = 0.5 * jxy
    return h


def make_operator(bonds, coeffs, local) -> dict:
    """Pack a term list: sites int32 [T, 2], coeff float64 [T, 2] (re, im),
    local float64 [T, 16, 2] (4x4 complex, row-major)."""
    bonds = np.asarray(bonds, dtype=np.int32).reshape(-1, 2)
    t = len(bonds)
    c = np.zeros((t, 2))
    c[:, 0] = np.asarray(coeffs, dtype=np.float64).reshape(-1)
    loc = np.zeros((t, 16, 2))
    loc[:, :, 0] = np.asarray(local, dtype=np.float64).reshape(-1, 16) if np.ndim(local) == 3 \
        else np.broadcast_to(np.asarray(local, dtype=np.float64).reshape(16), (t, 16))
    return {"sites": bonds, "coeff": c, "local": loc}


def heisenberg_ring(n: int, j: float = 1.0) -> dict:
    bonds = [(i, (i + 1) % n) for i in range(n)]
    return make_operator(bonds, [j] * n, heisenberg_local())


def xxz_ring(n: int, jxy: float = 1.0, delta: float = 1.0) -> dict:
    bonds = [(i, (i + 1) % n) for i in range(n)]
    return make_operator(bonds, [1.0] * n, xxz_local(jxy, delta))


def j1j2_torus(lx: int, ly: int, j1: float = 1.0, j2: float = 0.5) -> dict:
    """Nearest bonds (x,y)-(x+1,y), (x,y)-(x,y+1); next-nearest (x,y)-(x+1,y+1),
    (x,y)-(x+1,y-1); each bond once, site = x + lx*y."""
    s = lambda x, y: (x % lx) + lx * (y % ly)
    bonds, cs = [], []
    for y in range(ly):
        for x in range(lx):
            bonds += [(s(x, y), s(x + 1, y)), (s(x, y), s(x, y + 1))]
            cs += [j1, j1]
    for y in range(ly):
        for x in range(lx):
            bonds += [(s(x, y), s(x + 1, y + 1)), (s(x, y), s(x + 1, y - 1))]
            cs += [j2, j2]
    return make_operator(bonds, cs, heisenberg_local())


# ----------------------------------------------------------------------------
# the named workloads, at their full sizes
# ----------------------------------------------------------------------------
def workload(name: str) -> dict:
    """Problem definitions: n_sites, n_up, spin inversion, group, operator."""
    if name == "ring16":
        p, c = ring_group(16, 0, parity=+1)
        return dict(name=name, n_sites=16, n_up=8, spin_inversion=+1, perms=p, chars=c,
                    op=heisenberg_ring(16), complex_=False, lanczos_steps=50)
    if name == "ring32":
        p, c = ring_group(32, 0, parity=+1)
        return dict(name=name, n_sites=32, n_up=16, spin_inversion=+1, perms=p, chars=c,
                    op=heisenberg_ring(32), complex_=False, lanczos_steps=100)
    if name == "ring36":
        p, c = ring_group(36, 0, parity=+1)
        return dict(name=name, n_sites=36, n_up=18, spin_inversion=+1, perms=p, chars=c,
                    op=heisenberg_ring(36), complex_=False, lanczos_steps=150)
    if name == "ring40":
        p, c = ring_group(40, 0, parity=+1)
        return dict(name=name, n_sites=40, n_up=20, spin_inversion=+1, perms=p, chars=c,
                    op=heisenberg_ring(40), complex_=False, lanczos_steps=150)
    if name == "ring42":
        p, c = ring_group(42, 0, parity=+1)
        return dict(name=name, n_sites=42, n_up=21, spin_inversion=+1, perms=p, chars=c,
                    op=heisenberg_ring(42), complex_=False, lanczos_steps=150)
    if name == "ring42_pi":
        # for n = 2 mod 4 the ground state lies at momentum pi, reflection +1,
        # spin inversion -1 (a sector of the same dimension as k = 0, z = +1)
        p, c = ring_group(42, 21, parity=+1)
        return dict(name=name, n_sites=42, n_up=21, spin_inversion=-1, perms=p, chars=c,
                    op=heisenberg_ring(42), complex_=False, lanczos_steps=150)
    if name == "torus6x6":
        p, c = torus_group(6, 6, 1, 0)
        return dict(name=name, n_sites=36, n_up=18, spin_inversion=+1, perms=p, chars=c,
                    op=j1j2_torus(6, 6, 1.0, 0.5), complex_=True, lanczos_steps=100)
    if name == "xxz28_k0":
        p, c = ring_group(28, 0)
        return dict(name=name, n_sites=28, n_up=14, spin_inversion=+1, perms=p, chars=c,
                    op=xxz_ring(28, 1.0, 1.5), complex_=False, lanczos_steps=100)
    if name == "xxz28_k5":
        p, c = ring_group(28, 5)
        return dict(name=name, n_sites=28, n_up=14, spin_inversion=+1, perms=p, chars=c,
                    op=xxz_ring(28, 1.0, 1.5), complex_=True, lanczos_steps=100)
    raise KeyError(name)


def xxz28_sectors():
    """The 140 sectors of the XXZ ring N=28 (Jxy=1, Delta=1.5): Sz in {0,1,2,3}
    (n_up = 14..17) x 28 momenta, and spin inversion +-1 at Sz = 0."""
    out = []
    for sz in range(4):
        for k in range(28):
            zs = (+1, -1) if sz == 0 else (0,)
            for z in zs:
                p, c = ring_group(28, k)
                out.append(dict(n_sites=28, n_up=14 + sz, spin_inversion=z, perms=p, chars=c,
                                k=k, complex_=(2 * k) % 28 != 0))
    return out
