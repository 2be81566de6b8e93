"""Tensor-core (tcgen05) BF16 GEMMs of the MLP against an FP64 reference of the same op.

Inputs are BF16 (exact in FP64), so the reference is exact; the kernel accumulates in FP32.
Bound per element: |C - C_ref| <= 1e-5 * sum_k |A_ik B_jk| (FP32 accumulation over K), plus
one BF16 rounding of the result for the BF16 epilogues.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from scipy.special import erf  # noqa: E402


@pytest.fixture(scope="module")
def lc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2402_18858_gb300 import build, chem
    build.build()
    chem.lib()
    return chem


def _bf16(rng, shape, scale=1.0):
    return torch.as_tensor(rng.standard_normal(shape) * scale, dtype=torch.float32).to(torch.bfloat16)


def _gelu(x):
    return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))


def _dgelu(x):
    return 0.5 * (1.0 + erf(x / math.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / math.sqrt(2 * math.pi)


# long-K shapes with at least 256 rows run on CTA pairs (tiles 256 x 128/160/224/256), the others
# on single CTAs
SHAPES = [(128, 32, 64), (257, 160, 200), (1000, 1600, 64), (513, 400, 800), (4096, 32, 400), (130, 800, 1600),
          (600, 1000, 520), (300, 128, 304), (700, 800, 1600)]


@pytest.mark.parametrize("M,N,K", SHAPES)
@pytest.mark.parametrize("epi", [0, 1, 2, 3])
def test_gemm_epilogues(lc, M, N, K, epi):
    rng = np.random.default_rng(M * 7 + N * 3 + K + epi)
    A = _bf16(rng, (M, K))
    B = _bf16(rng, (N, K), 1.0 / math.sqrt(K))
    bias = torch.as_tensor(rng.standard_normal(N) * 0.1, dtype=torch.float32)
    z = _bf16(rng, (M, N))
    Ad, Bd, bd, zd = A.cuda(), B.cuda(), bias.cuda(), z.cuda()
    out = torch.empty((M, N), dtype=torch.bfloat16 if epi in (0, 2) else torch.float32, device="cuda")
    err = lc.chem_selftest_gemm(epi, Ad, Bd, out, bias=bd if epi in (0, 1) else None, z=zd if epi == 2 else None)
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    a, b = A.double().numpy(), B.double().numpy()
    acc = a @ b.T
    bound = 1e-5 * (np.abs(a) @ np.abs(b).T) + 1e-30
    got = out.double().cpu().numpy()
    if epi == 3:
        assert (np.abs(got - acc) <= bound).all()
    elif epi == 1:
        ref = acc + bias.double().numpy()[None, :]
        assert (np.abs(got - ref) <= bound + 1e-7 * np.abs(ref)).all()
    else:
        if epi == 0:
            pre = acc + bias.double().numpy()[None, :]
            ref = _gelu(pre)
            slope = np.abs(_dgelu(pre))
        else:
            zz = z.double().numpy()
            ref = acc * _dgelu(zz)
            slope = np.abs(_dgelu(zz))
        tol = slope * bound + 2.0 ** -8 * np.abs(ref) + 1e-6 * np.abs(ref).max()
        assert (np.abs(got - ref) <= tol).all(), np.abs(got - ref).max()
