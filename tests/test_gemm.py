"""The batched max-plus GEMM kernel (Eq. 2) through tn_maxplus_gemm against the
oracle's product written from the definition.  float32 sums are single
roundings and max is exact, so results must be bit-identical to numpy in
float32; int32 is exact."""
import numpy as np
import pytest

from oracle import semiring as S
from paper_2008_06888_gb300 import binding as B

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2008_06888_gb300 import build
    build.build()


SHAPES = [(1, 1, 1, 1), (2, 5, 7, 3), (1, 128, 128, 16), (3, 130, 67, 33), (1, 257, 129, 80),
          (4, 64, 300, 17), (1, 1, 500, 257), (2, 256, 384, 48)]


@pytest.mark.parametrize("dtype", ["float32", "int32"])
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("trans", [(False, False), (True, False), (False, True), (True, True)])
def test_maxplus_gemm_matches_definition(dtype, shape, trans):
    import torch
    bt, M, N, K = shape
    ta, tb = trans
    rng = np.random.default_rng(bt * 1000 + M * 7 + N * 3 + K)
    if dtype == "float32":
        A = rng.standard_normal((bt, M, K)).astype(np.float32)
        Bm = rng.standard_normal((bt, K, N)).astype(np.float32)
    else:
        A = rng.integers(-50, 50, (bt, M, K)).astype(np.int32)
        Bm = rng.integers(-50, 50, (bt, K, N)).astype(np.int32)
    ref = np.stack([S.maxplus_matmul(A[i], Bm[i]) for i in range(bt)]).astype(A.dtype)
    Ad = torch.tensor(np.ascontiguousarray(A.transpose(0, 2, 1)) if ta else A, device="cuda")
    Bd = torch.tensor(np.ascontiguousarray(Bm.transpose(0, 2, 1)) if tb else Bm, device="cuda")
    Cd = torch.empty((bt, M, N), dtype=Ad.dtype, device="cuda")
    B.tn_maxplus_gemm(Ad, Bd, Cd, transA=ta, transB=tb)
    torch.cuda.synchronize()
    assert np.array_equal(Cd.cpu().numpy(), ref)
