"""The host-side transposed-entry map of a symmetric sampling pattern
(solver.mirror_map), against its definition entry by entry."""
import numpy as np
import pytest

import pf_synthetic as syn

pytest.importorskip("torch")


@pytest.mark.parametrize("n,rate,seed", [(1, 1.0, 0), (7, 0.5, 1), (120, 0.3, 5), (500, 0.02, 9)])
def test_mirror_map_sends_each_entry_to_its_transpose(n, rate, seed):
    from paper_1904_10585_gb300 import solver as S
    inst = syn.completion_instance(max(n, 2), 1, rate, 1, seed=seed)
    rp, ci = inst.omega.rowptr, inst.omega.colind
    nn = len(rp) - 1
    m = S.mirror_map(rp, ci)
    rows = np.repeat(np.arange(nn), np.diff(rp))
    assert m.dtype == np.int32 and m.shape == ci.shape
    assert np.array_equal(np.sort(m), np.arange(len(ci)))      # a permutation
    assert np.array_equal(ci[m], rows)                         # (i, j) -> column i ...
    assert np.array_equal(rows[m], ci)                         # ... in row j
    assert np.array_equal(m[m], np.arange(len(ci)))            # an involution
    diag = rows == ci
    assert np.array_equal(m[diag], np.nonzero(diag)[0])        # diagonal entries are fixed
