"""Independent constructions the oracle (and the GPU path) are pinned to:
Kronecker-product Hamiltonians, explicit symmetry projectors, and the Bethe
ansatz energy of the Heisenberg ring.  numpy only; no oracle code."""
import numpy as np


def kron_hamiltonian(n, op):
    """Full 2^n matrix from Kronecker products of single-site matrices.
    State index s has bit k = site k (site n-1 is the most significant factor)."""
    def emb(a, site):
        return np.kron(np.kron(np.eye(2 ** (n - 1 - site)), a), np.eye(2 ** site))
    E = lambda a, c: np.outer(np.eye(2)[a], np.eye(2)[c])
    H = np.zeros((2 ** n, 2 ** n), complex)
    for t in range(len(op["sites"])):
        i, j = op["sites"][t]
        c = op["coeff"][t, 0] + 1j * op["coeff"][t, 1]
        h = (op["local"][t, :, 0] + 1j * op["local"][t, :, 1]).reshape(4, 4)
        for a in range(2):
            for b in range(2):
                for cc in range(2):
                    for d in range(2):
                        v = h[2 * a + b, 2 * cc + d]
                        if v != 0:
                            H += c * v * emb(E(a, cc), i) @ emb(E(b, d), j)
    return H


def act_all(n, perm, flip, states):
    """g.s for an array of states, vectorised (bit perm[i] of g.s = bit i of s)."""
    s = np.asarray(states, dtype=np.int64)
    out = np.zeros_like(s)
    for i in range(n):
        out |= ((s >> i) & 1) << int(perm[i])
    if flip:
        out ^= (1 << n) - 1
    return out


def projected_basis(n, n_up, perms, chars, z):
    """Explicit symmetry-adapted vectors |r^> = P|r> / |P|r>| with
    P = |G|^-1 sum_g conj(chi(g)) U_g, for every orbit minimum r with P|r> != 0.
    Returns (reps ascending, V with columns |r^> in the full 2^n space)."""
    elems = [(p, 0, complex(c[0], c[1])) for p, c in zip(perms, chars)]
    if z:
        elems += [(p, 1, complex(c[0], c[1]) * z) for p, c in zip(perms, chars)]
    allst = np.arange(2 ** n)
    pc = np.array([bin(s).count("1") for s in allst])
    sector = allst[pc == n_up] if n_up >= 0 else allst
    images = np.stack([act_all(n, p, f, sector) for p, f, _ in elems])
    orbit_min = images.min(axis=0)
    reps, cols = [], []
    for s, m in zip(sector, orbit_min):
        if s != m:
            continue
        v = np.zeros(2 ** n, complex)
        for p, f, ch in elems:
            v[act_all(n, p, f, [s])[0]] += np.conj(ch)
        v /= len(elems)
        nv = np.linalg.norm(v)
        if nv > 1e-9:
            reps.append(s)
            cols.append(v / nv)
    V = np.array(cols).T if cols else np.zeros((2 ** n, 0), complex)
    return np.array(reps, dtype=np.uint64), V


def bethe_e0(n, iters=20000, tol=1e-15):
    """Ground-state energy of the n-site periodic Heisenberg ring, J = 1, from
    the Bethe ansatz (n even, M = n/2 magnons, quantum numbers
    I_j = -(M-1)/2 .. (M-1)/2):  n atan(2 l_j) = pi I_j + sum_k atan(l_j - l_k),
    E = n/4 - sum_j 2/(4 l_j^2 + 1)."""
    m = n // 2
    I = np.arange(m) - (m - 1) / 2.0
    lam = 0.5 * np.tan(np.pi * I / n)
    for _ in range(iters):
        s = np.arctan(lam[:, None] - lam[None, :]).sum(axis=1)
        new = 0.5 * np.tan((np.pi * I + s) / n)
        if np.max(np.abs(new - lam)) < tol:
            lam = new
            break
        lam = 0.5 * lam + 0.5 * new
    return n / 4.0 - np.sum(2.0 / (4.0 * lam ** 2 + 1.0))


