"""The tensor-core GEMM tile of the FP32 transform solvers (three TF32
products per K step on tcgen05, FP32 accumulation in tensor memory) against
an FP64 product of the same FP32 inputs."""
import numpy as np
import pytest

from paper_2303_10783_gb300 import cases, solid

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("transposed", [False, True], ids=["k-adjacent", "row-adjacent"])
@pytest.mark.parametrize("n,k", [(128, 128), (48, 50), (256, 96), (16, 8), (96, 200), (112, 37)])
def test_tensor_core_tile_matches_fp64_product(lib, n, k, transposed):
    import torch
    rng = np.random.default_rng(1000 + 7 * n + k)
    a = rng.standard_normal((128, k)).astype(np.float32)
    b = rng.standard_normal((n, k)).astype(np.float32)
    # a cosine-matrix-like operand as well: rows of very different size
    a[:8] *= 1e3
    ref = a.astype(np.float64) @ b.astype(np.float64).T
    scale = np.abs(a).astype(np.float64) @ np.abs(b).astype(np.float64).T
    c = solid.Case(cases.cavity_2d(8, 8))
    if transposed:
        ta, tb = torch.from_numpy(np.ascontiguousarray(a.T)).cuda(), torch.from_numpy(np.ascontiguousarray(b.T)).cuda()
    else:
        ta, tb = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    td = torch.full((128, n), float("nan"), dtype=torch.float32, device="cuda")
    c.tc_selftest(ta.data_ptr(), tb.data_ptr(), td.data_ptr(), n, k, transposed)
    assert c.sync() == solid.SS_OK
    d = td.cpu().numpy().astype(np.float64)
    c.close()
    err = np.abs(d - ref) / scale
    # FP32 products and sums: a few 2^-24 per term; plain TF32 would leave ~2^-11
    assert np.all(np.isfinite(d))
    assert err.max() < 2e-6, err.max()


def test_tensor_core_selftest_rejects_bad_shapes(lib):
    c = solid.Case(cases.cavity_2d(8, 8))
    for n, k in ((8, 16), (17, 16), (272, 16), (32, 0), (32, 5000)):
        assert lib.ss_tc_selftest(c.h, 1, 1, 1, n, k, 0) == solid.SS_EINVAL
    c.close()
