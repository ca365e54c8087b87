"""The allocation-free block Gram (mhde_block_gram_noalloc) against the
regular entry point (mhde_block_gram, caller-provided scratch).

Callers that cannot allocate device memory (hosts that own the device's
memory pool, latency-critical loops) use the no-alloc variant; its results
must match the regular path.  Kept in its own file, collected last, so that a
run stopping at the first failure has run every other test first.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2108_05110_gb300 as P  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n_rows,ld,r,k", [(148739, 20, 20, 5), (5003, 64, 61, 3), (700, 4, 3, 1)])
def test_noalloc_gram_matches_regular_entry_point_twice(n_rows, ld, r, k):
    rng = np.random.default_rng(7 + n_rows)
    G_out = torch.empty((k, r, r), dtype=torch.float64, device="cuda")
    for call in range(2):                          # two calls in a row share the fixed scratch
        V = torch.from_numpy(rng.standard_normal((k, n_rows, ld))).cuda()
        W = torch.from_numpy(rng.standard_normal((n_rows, ld))).cuda()
        ref = P.block_gram(V, W, k, r)
        got = P.block_gram_noalloc(V, W, k, r, G=G_out)
        torch.cuda.synchronize()
        Vn, Wn = V.cpu().numpy(), W.cpu().numpy()
        for i in range(k):
            scale = np.abs(Vn[i][:, :r]).T @ np.abs(Wn[:, :r])
            assert np.all(np.abs(got[i].cpu().numpy() - ref[i].cpu().numpy()) <= 1e-13 * scale)


def test_noalloc_gram_rejects_sizes_beyond_its_scratch():
    V = torch.zeros((70, 64, 64), dtype=torch.float64, device="cuda")
    W = torch.zeros((64, 64), dtype=torch.float64, device="cuda")
    with pytest.raises(P.MhdeError) as e:
        P.block_gram_noalloc(V, W, 70, 64)        # 70 * 64 * 64 partials per chunk > 262144
    assert e.value.code == -6
