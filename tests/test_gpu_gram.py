"""Gram matrices of the Cholesky-QR stabilisation through the C ABI
(sldqmc_gram_batch_dev) against an extended-precision host sum.

The mixed-precision modes compute W = X X^T for N >= 128 on the BF16 tensor
cores by error-free digit splitting (exact accumulation in chunks of K <= 384,
so N = 400 and N = 1024 take two and three chunks; N = 1296 walks two groups
of row strips, 8 and 3, the last with a partial column of tiles); the result
must be as accurate as FP64 itself.  Inputs are seeded Gaussian rows with power-of-two row scales
2^-20 .. 2^20 (the grading of X's columns in the stabilised chain), rows
whose entries span nine decades, and a zero row.  The error measure is
|W_ij - W_ij,ref| / sqrt(W_ii W_jj) over the upper triangle."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    from paper_1612_03804_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _rows(seed, B, N):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((B, N, N))
    X *= np.ldexp(1.0, rng.integers(-20, 21, size=(B, N, 1)))
    X[:, 3, ::7] *= 1e-9
    X[:, 5, :] = 0.0
    return X


def _err(W, X):
    Xl = X.astype(np.longdouble)
    worst = 0.0
    for b in range(X.shape[0]):
        ref = Xl[b] @ Xl[b].T
        d = np.sqrt(np.outer(np.diag(ref), np.diag(ref)).astype(np.float64))
        iu = np.triu_indices(X.shape[1])
        den = d[iu]
        num = np.abs((W[b].astype(np.longdouble) - ref)[iu]).astype(np.float64)
        ok = den > 0
        worst = max(worst, float(np.max(num[ok] / den[ok])))
        assert np.all(W[b][iu][~ok] == 0.0)
    return worst


@pytest.mark.parametrize("prec,L1,L2,tensor", [("3xtf32", 12, 12, True), ("bf16x3", 16, 16, True),
                                               ("3xtf32", 16, 24, True), ("3xtf32", 20, 20, True),
                                               ("bf16x3", 32, 32, True), ("3xtf32", 36, 36, True),
                                               ("fp64", 16, 16, False)])
def test_gram_against_extended_precision(prec, L1, L2, tensor):
    import torch
    from paper_1612_03804_gb300 import sldqmc
    N = L1 * L2
    B = 3 if N <= 400 else (2 if N <= 1024 else 1)
    X = _rows(17 + N, B, N)
    with sldqmc.Context(L1, L2, mu=-0.5, xi=1.0, beta=1.0, dtau=0.1, n_wrap=5, prec=prec, max_batch=B) as ctx:
        dX = torch.from_numpy(X).cuda()
        dW = torch.zeros_like(dX)
        ctx.profile(True)
        ctx.gram_batch_dev(dX, dW)
        prof = ctx.profile_read()
        ctx.profile(False)
        ctx.sync()
        W = dW.cpu().numpy()
    assert (prof["gemm_oz"]["launches"] > 0) == tensor
    assert (prof["gemm_f64"]["launches"] > 0) == (not tensor)
    err = _err(W, X)
    print(f"{prec} N={N} {'tensor-core' if tensor else 'FP64'} Gram: max err / sqrt(WiiWjj) {err:.2e}")
    assert err <= (4e-16 if tensor else N * 2.0 ** -52)
