"""Helpers shared by the GPU parity tests: build a sector on the GPU through the
C ABI and the same sector in the oracle, from one problem description."""
import numpy as np

import ed_inputs as ei
import oracle


def gpu():
    import torch
    from paper_2308_16712_gb300 import ed
    return torch, ed


def build_pair(n, n_up, z, perms, chars, op, with_oracle=True):
    torch, ed = gpu()
    B = ed.basis_build(n, n_up, z, perms, chars)
    O = ed.operator_create(n, op["sites"], op["coeff"], op["local"])
    out = {"B": B, "O": O, "dim": ed.basis_size(B)}
    if with_oracle:
        G = oracle.Group(n, perms, chars, z)
        st, nm = oracle.enumerate_basis(G, n_up)
        out.update(G=G, H=oracle.Operator(op), st=st, nm=nm)
    return out


def gpu_basis_numpy(B):
    torch, ed = gpu()
    st, nm = ed.basis_states(B)
    return st.cpu().numpy().view(np.uint64), nm.cpu().numpy().view(np.uint16)


def to_torch(a, dtype):
    torch, _ = gpu()
    return torch.from_numpy(np.ascontiguousarray(a).astype(dtype)).cuda()


def elem_rel_err(got, want, floor=1e-3):
    """Largest element-wise relative error over the elements whose magnitude is
    at least `floor` times the largest (where a relative error is meaningful)."""
    got = np.asarray(got)
    want = np.asarray(want)
    if not want.size:
        return 0.0
    big = np.abs(want) >= floor * np.abs(want).max()
    return float((np.abs(got - want)[big] / np.abs(want)[big]).max()) if big.any() else 0.0


def rel_err(got, want):
    got = np.asarray(got)
    want = np.asarray(want)
    scale = max(np.abs(want).max(), 1e-300) if want.size else 1.0
    return float(np.abs(got - want).max() / scale) if want.size else 0.0
