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
          (4, 64, 300, 17), (1, 1, 500, 257), (2, 256, 384, 48),
          # a few outputs over a long K: the split-K form (reduction to the root)
          (1, 1, 1, 1 << 16), (2, 2, 3, 1 << 15), (1, 4, 4, 20001)]


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


@pytest.mark.parametrize("tile", ["0 2", "0 8", "1 2", "1 8"])
def test_every_tile_candidate_is_bit_identical(tile, monkeypatch):
    """The autotuner's candidates (16- or 4-byte staging x 2 or 8 blocks per SM)
    compute each output as the max of the same single-rounding sums."""
    import torch
    rng = np.random.default_rng(7)
    A = rng.standard_normal((2, 256, 96)).astype(np.float32)
    Bm = rng.standard_normal((2, 96, 384)).astype(np.float32)
    ref = np.stack([S.maxplus_matmul(A[i], Bm[i]) for i in range(2)]).astype(np.float32)
    Ad, Bd = torch.tensor(A, device="cuda"), torch.tensor(Bm, device="cuda")
    Cd = torch.empty((2, 256, 384), dtype=torch.float32, device="cuda")
    monkeypatch.setenv("TN_GEMM_TILE", tile)
    B.tn_maxplus_gemm(Ad, Bd, Cd)
    torch.cuda.synchronize()
    assert np.array_equal(Cd.cpu().numpy(), ref)


def test_autotuner_records_its_choice(tmp_path):
    """A shape class is timed once; its choice lands in TN_AUTOTUNE_CACHE."""
    import subprocess
    import sys
    cache = tmp_path / "tiles.txt"
    code = (
        "import torch, numpy as np\n"
        "from paper_2008_06888_gb300 import binding as B\n"
        "A = torch.randn(1, 384, 128, device='cuda'); Bm = torch.randn(1, 128, 256, device='cuda')\n"
        "C = torch.empty(1, 384, 256, device='cuda')\n"
        "B.tn_maxplus_gemm(A, Bm, C); torch.cuda.synchronize()\n"
        "ref = (A[0][:, :, None] + Bm[0][None]).amax(1)\n"
        "assert torch.equal(C[0], ref)\n")
    env = dict(__import__("os").environ, TN_AUTOTUNE_CACHE=str(cache))
    env.pop("TN_NO_AUTOTUNE", None)
    subprocess.run([sys.executable, "-c", code], check=True, env=env, timeout=300,
                   cwd=__import__("os").path.dirname(__import__("os").path.dirname(__file__)))
    lines = cache.read_text().splitlines()
    assert len(lines) == 1 and "m384 n256 k128" in lines[0]
    variant, per_sm = map(int, lines[0].split("|")[1].split())
    assert variant in (0, 1) and per_sm in (2, 8)
