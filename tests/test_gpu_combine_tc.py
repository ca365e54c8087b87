"""The FP32 block combination of the block Krylov iteration (Section 1:
block linear solvers; the new basis block W - sum_i V_i H_i T and the
solution update sum_i Z_i Y_i), out = alpha in + sum_i V_i C_i, on the
tensor cores (tcgen05, TF32 on split operands) and on the CUDA cores,
through the C ABI, against an FP64 numpy reference of the same FP32 inputs;
including the in-place forms the solver uses (out aliasing in, and out
aliasing one of the blocks)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2108_05110_gb300 as P  # noqa: E402

pytestmark = pytest.mark.gpu

# n_rows, ldv, r_in, r_out, ldo, kblocks
CASES = [(148739, 20, 20, 20, 20, 16), (148739, 20, 20, 20, 20, 31), (177747, 52, 50, 50, 52, 16),
         (5003, 24, 23, 17, 20, 3), (129, 8, 5, 7, 8, 2), (700, 4, 3, 3, 4, 1), (1000, 64, 60, 40, 40, 2),
         (40000, 20, 20, 20, 20, 1), (400000, 20, 20, 20, 20, 5)]


def _tol(nterms):
    """Relative to sum |terms|: the split products (about 2^-21 each) plus
    FP32 accumulation of nterms products (random-walk growth, 4 sigma)."""
    return 1e-6 + 2.5e-7 * np.sqrt(nterms)


def _reference(V, Cf, r_in, r_out, ldo, inp, alpha):
    acc = np.einsum("krp,kpq->rq", V[:, :, :r_in].astype(np.float64), Cf.astype(np.float64))
    mag = np.einsum("krp,kpq->rq", np.abs(V[:, :, :r_in]).astype(np.float64), np.abs(Cf).astype(np.float64))
    out = np.zeros((V.shape[1], ldo))
    out[:, :r_out] = acc
    bound = np.zeros_like(out)
    bound[:, :r_out] = mag
    if inp is not None:
        out[:, :r_out] += alpha * inp[:, :r_out].astype(np.float64)
        bound[:, :r_out] += abs(alpha) * np.abs(inp[:, :r_out])
    return out, bound


@pytest.mark.parametrize("n_rows,ldv,r_in,r_out,ldo,k", CASES)
@pytest.mark.parametrize("tensor_cores", [True, False])
def test_f32_combine_matches_fp64_reference(n_rows, ldv, r_in, r_out, ldo, k, tensor_cores):
    rng = np.random.default_rng(n_rows + 3 * k)
    V = (rng.standard_normal((k, n_rows, ldv)) / np.sqrt(n_rows)).astype(np.float32)
    Cf = rng.standard_normal((k, r_in, r_out)).astype(np.float32)
    inp = rng.standard_normal((n_rows, ldo)).astype(np.float32)
    for alpha, use_in in ((0.0, False), (1.0, True), (-0.5, True)):
        out = torch.full((n_rows, ldo), float("nan"), dtype=torch.float32, device="cuda")
        P.block_combine_f32(out, torch.from_numpy(V).cuda(), torch.from_numpy(Cf).cuda(), r_in, r_out,
                            in_=torch.from_numpy(inp).cuda() if use_in else None, alpha=alpha,
                            tensor_cores=tensor_cores)
        got = out.cpu().numpy().astype(np.float64)
        want, bound = _reference(V, Cf, r_in, r_out, ldo, inp if use_in else None, alpha)
        assert np.all(np.abs(got - want) <= _tol(k * r_in) * bound + 1e-30), (alpha, np.abs(got - want).max())


@pytest.mark.parametrize("tensor_cores", [True, False])
def test_f32_combine_in_place_forms(tensor_cores):
    """out = in (W += sum_i V_i C_i) and out = the last block (V_k := sum_i V_i C_i
    over blocks 0..k), as the block Gram-Schmidt step writes them."""
    n_rows, ld, r, k = 30011, 20, 20, 6
    rng = np.random.default_rng(5)
    V = (rng.standard_normal((k, n_rows, ld)) / np.sqrt(n_rows)).astype(np.float32)
    Cf = rng.standard_normal((k, r, r)).astype(np.float32)
    Vd = torch.from_numpy(V).cuda()
    # out aliases in
    W = torch.from_numpy(V[-1].copy()).cuda()
    P.block_combine_f32(W, Vd[:-1], torch.from_numpy(Cf[:-1]).cuda(), r, r, in_=W, alpha=1.0,
                        v_stride=n_rows * ld, tensor_cores=tensor_cores)
    want, bound = _reference(V[:-1], Cf[:-1], r, r, ld, V[-1], 1.0)
    assert np.all(np.abs(W.cpu().numpy() - want) <= _tol(k * r) * bound + 1e-30)
    # out aliases the last block
    Vd2 = torch.from_numpy(V.copy()).cuda()
    P.block_combine_f32(Vd2[-1], Vd2, torch.from_numpy(Cf).cuda(), r, r, v_stride=n_rows * ld,
                        tensor_cores=tensor_cores)
    want, bound = _reference(V, Cf, r, r, ld, None, 0.0)
    assert np.all(np.abs(Vd2[-1].cpu().numpy() - want) <= _tol(k * r) * bound + 1e-30)
