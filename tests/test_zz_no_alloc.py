"""The allocation-free count entry point (ed_basis_count_noalloc) against the
dimension of the basis ed_basis_build allocates, for callers that cannot call
cudaMalloc (their memory pool owns the device memory, or their path must not
synchronise the device).  Collected last on purpose: it shares one fixed
scratch array inside the library, and must work after any other test as well
as alone in a fresh process."""
import numpy as np
import pytest

import ed_inputs as ei

pytestmark = pytest.mark.gpu

SECTORS = [
    (16, 8, +1, lambda: ei.ring_group(16, 0, +1)),
    (20, 9, 0, lambda: ei.ring_group(20, 3)),
    (16, 8, -1, lambda: ei.torus_group(4, 4, 1, 2)),
    (34, 5, 0, lambda: ei.ring_group(34, 2, None)),
]


def test_count_without_allocation_matches_basis_build():
    import torch
    from paper_2308_16712_gb300 import ed
    torch.cuda.init()
    want = []
    for n, n_up, z, grp in SECTORS:
        p, c = grp()
        want.append(ed.basis_size(ed.basis_build(n, n_up, z, p, c)))
    # two passes in a row over all sectors: each call leaves its contents in
    # the shared scratch, the next call must not depend on them
    for _ in range(2):
        for (n, n_up, z, grp), w in zip(SECTORS, want):
            p, c = grp()
            assert ed.basis_count_noalloc(n, n_up, z, p, c) == w


def test_count_without_allocation_large_chunks():
    """A sector whose enumeration needs the 2^18-chunk cap (C(28, 14) = 4.0e7
    states: 153 states per chunk, and the scan over all 2^18 chunk counts),
    against the allocating count, twice in a row."""
    from paper_2308_16712_gb300 import ed
    p, c = ei.ring_group(28, 0)
    want = ed.basis_count(28, 14, +1, p, c)
    assert want > 0
    for _ in range(2):
        assert ed.basis_count_noalloc(28, 14, +1, p, c) == want


def test_count_without_allocation_rejects_groups_beyond_capacity():
    from paper_2308_16712_gb300 import ed
    # 513 elements exceed the fixed scratch; the size check comes first
    perms = np.tile(ei.ring_group(8, 0)[0], (65, 1))[:513]
    chars = np.tile(ei.ring_group(8, 0)[1], (65, 1))[:513]
    with pytest.raises(ed.EDError) as e:
        ed.basis_count_noalloc(8, 4, 0, perms, chars)
    assert e.value.status == 1
