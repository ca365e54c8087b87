"""CPU checks of the library's host-side small dense routines against numpy:
the block least-squares update of the block GMRES iteration and the Cholesky
QR factors of a new Krylov block."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("sd") / "small_dense_check")
    src = [os.path.join(ROOT, "tests", "cpp", "small_dense_check.cpp"),
           os.path.join(ROOT, "paper_2108_05110_gb300", "csrc", "fe_host.cpp")]
    subprocess.run(["g++", "-O2", "-std=c++17", "-I/usr/local/cuda/include", *src, "-o", exe], check=True)
    return exe


@pytest.mark.parametrize("r,J,m", [(1, 1, 6), (3, 5, 4), (4, 4, 7), (20, 20, 6)])
def test_block_least_squares_matches_numpy_lstsq(checker, r, J, m):
    """BlockLS: Householder QR of the block Hessenberg matrix, one block column
    at a time.  After every column the residual norms of
    min || E_1 S0 - Hbar_k Y || must equal numpy's, and the final Y must match
    numpy.linalg.lstsq on the assembled ((m+1) r) x (m r) problem."""
    rng = np.random.default_rng(11 + r + J + m)
    S0 = rng.standard_normal((r, J))
    blocks = [rng.standard_normal(((k + 2) * r, r)) for k in range(m)]
    text = f"L {r} {J} {m}\n" + " ".join(repr(float(v)) for v in S0.ravel()) + "\n"
    text += "".join(" ".join(repr(float(v)) for v in b.ravel()) + "\n" for b in blocks)
    out = subprocess.run([checker], input=text, capture_output=True, text=True, check=True).stdout.split()
    Hbar = np.zeros(((m + 1) * r, m * r))
    for k, b in enumerate(blocks):
        Hbar[:(k + 2) * r, k * r:(k + 1) * r] = b
    B = np.zeros(((m + 1) * r, J))
    B[:r] = S0
    pos = 0
    for k in range(m):
        ok = int(out[pos]); pos += 1
        res = np.array([float(v) for v in out[pos:pos + J]]); pos += J
        H = Hbar[:(k + 2) * r, :(k + 1) * r]
        Y = np.linalg.lstsq(H, B[:(k + 2) * r], rcond=None)[0]
        want = np.linalg.norm(B[:(k + 2) * r] - H @ Y, axis=0)
        assert ok == 1
        assert np.allclose(res, want, rtol=1e-9, atol=1e-12 * np.linalg.norm(S0))
    Y = np.array([float(v) for v in out[pos:pos + m * r * J]]).reshape(m * r, J)
    Yref = np.linalg.lstsq(Hbar, B, rcond=None)[0]
    assert np.allclose(Y, Yref, rtol=1e-8, atol=1e-10 * np.abs(Yref).max())


@pytest.mark.parametrize("r,rk", [(4, 2), (6, 1), (20, 13)])
def test_block_least_squares_with_a_rank_deficient_last_block(checker, r, rk):
    """The block column a GMRES cycle adds when its new Krylov block turns out
    numerically rank-deficient: only rk of the r rows of its subdiagonal
    factor S are nonzero (the significant directions of the SVQB factor), and
    the cycle ends there.  BlockLS must give the least-squares residuals of
    exactly that matrix, as numpy does, and they differ from those of the
    matrix whose whole S block is zero: keeping the rk rows changes the
    correction that the cycle returns."""
    J, m = r, 3
    rng = np.random.default_rng(7 + r + rk)
    S0 = rng.standard_normal((r, J))
    blocks = [rng.standard_normal(((k + 2) * r, r)) for k in range(m)]
    last = blocks[-1]
    last[(m) * r + rk:, :] = 0.0                     # rows rk..r-1 of the last S block
    text = f"L {r} {J} {m}\n" + " ".join(repr(float(v)) for v in S0.ravel()) + "\n"
    text += "".join(" ".join(repr(float(v)) for v in b.ravel()) + "\n" for b in blocks)
    out = subprocess.run([checker], input=text, capture_output=True, text=True, check=True).stdout.split()
    Hbar = np.zeros(((m + 1) * r, m * r))
    for k, b in enumerate(blocks):
        Hbar[:(k + 2) * r, k * r:(k + 1) * r] = b
    B = np.zeros(((m + 1) * r, J))
    B[:r] = S0
    pos = (1 + J) * (m - 1)
    assert int(out[pos]) == 1
    res = np.array([float(v) for v in out[pos + 1:pos + 1 + J]])
    Y = np.linalg.lstsq(Hbar, B, rcond=None)[0]
    want = np.linalg.norm(B - Hbar @ Y, axis=0)
    assert np.allclose(res, want, rtol=1e-9, atol=1e-12 * np.linalg.norm(S0))
    dropped = Hbar.copy()
    dropped[m * r:, (m - 1) * r:] = 0.0
    Yd = np.linalg.lstsq(dropped, B, rcond=None)[0]
    true_resid_of_dropped = np.linalg.norm(B - Hbar @ Yd, axis=0)
    assert np.all(true_resid_of_dropped >= want - 1e-12) and np.any(true_resid_of_dropped > want * (1 + 1e-6))


def _cholqr(exe, G, thresh):
    r = G.shape[0]
    text = f"Q {r} {thresh!r}\n" + " ".join(repr(float(v)) for v in G.ravel()) + "\n"
    out = subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout.split()
    if int(out[0]) == 0:
        return None
    vals = np.array([float(v) for v in out[1:1 + 2 * r * r]])
    return vals[:r * r].reshape(r, r), vals[r * r:].reshape(r, r)


@pytest.mark.parametrize("r", [1, 4, 20])
def test_cholesky_qr_factors_orthonormalise_the_block(checker, r):
    """A full-rank block W (n x r): with G = W^T W, W T has orthonormal columns,
    (W T) S = W, S is numpy's upper-triangular Cholesky factor (unique with a
    positive diagonal) and T = S^{-1}."""
    rng = np.random.default_rng(5 + r)
    W = rng.standard_normal((400, r)) @ (np.eye(r) + 0.5 * np.triu(rng.standard_normal((r, r)), 1))
    G = W.T @ W
    res = _cholqr(checker, G, 1e-9)
    assert res is not None
    T, S = res
    Q = W @ T
    assert np.allclose(Q.T @ Q, np.eye(r), atol=1e-10)
    assert np.allclose(Q @ S, W, atol=1e-10 * np.abs(W).max())
    assert np.allclose(S, np.linalg.cholesky(G).T, rtol=1e-12, atol=1e-12 * np.abs(S).max())
    assert np.allclose(T @ S, np.eye(r), atol=1e-11)
    assert np.allclose(np.tril(S, -1), 0.0) and np.allclose(np.tril(T, -1), 0.0)


def test_cholesky_qr_declines_a_nearly_rank_deficient_block(checker):
    """Eigenvalues spread over 1e-8 of the largest: with thresh = 1e-9 full
    rank cannot be certified (the eigen form must decide what to drop), and an
    indefinite or zero matrix is refused outright."""
    rng = np.random.default_rng(3)
    U = np.linalg.qr(rng.standard_normal((6, 6)))[0]
    G = U @ np.diag([1.0, 0.5, 0.1, 1e-3, 1e-6, 1e-8]) @ U.T
    assert _cholqr(checker, G, 1e-9) is None
    assert _cholqr(checker, G, 1e-14) is not None          # a looser threshold accepts it
    assert _cholqr(checker, np.zeros((3, 3)), 1e-9) is None
    assert _cholqr(checker, np.diag([1.0, -1.0, 1.0]), 1e-9) is None
