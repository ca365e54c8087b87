"""The FP32 block Gram G_i = V_i^T W of the block Krylov iteration (Section
1: all J right-hand sides solved together with block linear solvers) on the
tensor cores (tcgen05, TF32 on split operands) and on the CUDA cores,
through the C ABI, against an FP64 numpy reference of the same FP32 inputs.
Sizes span the benchmark's (148,739 rows, 20 columns, 16 and 31 blocks),
the channel workload's (52-wide rows, 50 columns, block groups), narrow
blocks, ragged row counts and a single block."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2108_05110_gb300 as P  # noqa: E402

pytestmark = pytest.mark.gpu

CASES = [(148739, 20, 20, 16), (148739, 20, 20, 31), (177747, 52, 50, 16), (5003, 24, 23, 3), (700, 4, 3, 1),
         (1000, 64, 64, 2), (129, 8, 5, 7), (40000, 32, 17, 12)]


def _data(n_rows, ld, k, seed, scale=1.0):
    rng = np.random.default_rng(seed)
    V = (rng.standard_normal((k, n_rows, ld)) * scale / np.sqrt(n_rows)).astype(np.float32)
    W = (rng.standard_normal((n_rows, ld)) * scale).astype(np.float32)
    return V, W


@pytest.mark.parametrize("n_rows,ld,r,k", CASES)
@pytest.mark.parametrize("tensor_cores", [True, False])
def test_f32_gram_matches_fp64_reference(n_rows, ld, r, k, tensor_cores):
    V, W = _data(n_rows, ld, k, seed=n_rows + 7 * k)
    Vd, Wd = torch.from_numpy(V).cuda(), torch.from_numpy(W).cuda()
    G = P.block_gram_f32(Vd, Wd, k, r, tensor_cores=tensor_cores).cpu().numpy()
    V64, W64 = V.astype(np.float64)[:, :, :r], W.astype(np.float64)[:, :r]
    for i in range(k):
        ref = V64[i].T @ W64
        bound = np.abs(V64[i]).T @ np.abs(W64)
        # relative to the sum of |terms|: the split products (about 2^-21 each)
        # plus FP32 accumulation over one CTA's rows (at most ~1000 here;
        # random-walk growth, 4 sigma), the CTAs being summed in FP64
        tol = 1e-6 + 2.5e-7 * np.sqrt(min(n_rows, 1000))
        assert np.all(np.abs(G[i] - ref) <= tol * bound + 1e-30), (i, np.abs(G[i] - ref).max(), bound.max())


def test_tensor_core_gram_splits_operands_to_fp32_accuracy():
    """Inputs near 1 with small perturbations: TF32 inputs alone (10 mantissa
    bits) would shift every product by ~2^-11 relative, always the same way;
    the split keeps the error at the level of FP32 accumulation, far below."""
    n_rows, ld, r, k = 20000, 20, 20, 4
    rng = np.random.default_rng(11)
    V = (1.0 + 1e-3 * rng.standard_normal((k, n_rows, ld))).astype(np.float32)
    W = (1.0 + 1e-3 * rng.standard_normal((n_rows, ld))).astype(np.float32)
    G = P.block_gram_f32(torch.from_numpy(V).cuda(), torch.from_numpy(W).cuda(), k, r).cpu().numpy()
    ref = np.einsum("krp,rq->kpq", V.astype(np.float64), W.astype(np.float64))

    def tf32(x):                                   # keep sign, exponent and 10 mantissa bits
        return (x.view(np.uint32) & np.uint32(0xFFFFE000)).view(np.float32).astype(np.float64)
    plain = np.einsum("krp,rq->kpq", tf32(V), tf32(W))
    rel = np.abs(G - ref).max() / np.abs(ref).max()
    rel_plain = np.abs(plain - ref).max() / np.abs(ref).max()
    assert rel_plain > 1e-4 and rel <= 2e-5 and rel <= 0.05 * rel_plain, (rel, rel_plain)


def test_tensor_core_gram_rejects_sizes_outside_its_range():
    V = torch.zeros((1, 64, 68), dtype=torch.float32, device="cuda")
    W = torch.zeros((64, 68), dtype=torch.float32, device="cuda")
    with pytest.raises(P.MhdeError) as e:
        P.block_gram_f32(V, W, 1, 66, tensor_cores=True)
    assert e.value.code == -1
