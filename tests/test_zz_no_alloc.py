"""Handle-free SVD entry point without allocation (sctm_svd_noalloc) against
the handle's sctm_svd: two calls in a row on each path give the same
decomposition (same kernel, different scratch).  This file sorts after every
other test file, so a run that stops at the first failure has run all the
others before it, and the entry point is exercised after them in the same
process."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_2502_10298_gb300 as S  # noqa: E402


@pytest.mark.parametrize("m,n", [(40, 40), (300, 256), (1024, 1024)])
def test_noalloc_svd_matches_handle_svd(m, n):
    rng = np.random.default_rng(m * 7 + n)
    h = S.sctm_create(1, 1, 2, 2, 4, workspace_bytes=1 << 30)
    try:
        for call in range(2):
            M = torch.tensor(rng.standard_normal((m, n)) * np.logspace(0, -5, n)[None, :], device="cuda")
            U0, S0, V0 = S.sctm_svd(h, M)
            U1, S1, V1 = S.sctm_svd_noalloc(M)
            torch.cuda.synchronize()
            for a, b in ((S0, S1), (U0, U1), (V0, V1)):
                assert torch.allclose(a, b, rtol=0, atol=1e-13 * float(S0[0])), call
            rec = (U1 * S1[None, :]) @ V1.T
            assert float((rec - M).abs().max()) < 1e-12 * float(S1[0])
    finally:
        S.sctm_destroy(h)


def test_noalloc_rejects_sizes_beyond_the_maximum():
    M = torch.zeros((2048, 1024), dtype=torch.float64, device="cuda")   # (m + n) n = 3 * 2^20 > 2^21
    with pytest.raises(S.SctmError):
        S.sctm_svd_noalloc(M)
