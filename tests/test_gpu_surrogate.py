"""The learned surrogate source on the tensor cores (tcgen05): forward values
against the FP64 oracle network evaluated with the same BF16 weights and
BF16 hidden activations. Remaining differences: FP32 accumulation order and
the FP32 SiLU, which can move an activation across a BF16 rounding boundary
(one BF16 ulp = 2^-8 relative); bound used: 1e-2 of the output scale."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2603_00538_gb300 as sft  # noqa: E402

DEV = torch.device("cuda:0")


def _as_gpu_params(orc, p64):
    """The parameters the GPU network computes with: FP32 everywhere, BF16
    for the three 256x256 weight matrices."""
    p = p64.astype(np.float32).astype(np.float64)
    parts = orc.mlp_split(p)
    for i in (2, 4, 6):
        parts[i][...] = np.vectorize(orc.bf16_round)(parts[i])
    return p


@pytest.mark.parametrize("n", [1, 128, 1037])
def test_forward_matches_oracle(orc, n):
    p64 = W.mlp_init(7)
    net = sft.sft_mlp_create(p64.astype(np.float32))
    X = np.random.default_rng(n).random((n, 3)).astype(np.float32)
    y = sft.sft_mlp_forward(net, X)
    ref = orc.mlp_forward(_as_gpu_params(orc, p64), X.astype(np.float64), act_bf16=True)
    scale = max(np.abs(ref).max(), 1e-3)
    err = np.abs(y - ref).max() / scale
    print(f"n={n} max rel err {err:.2e}")
    assert err < 1e-2


def test_forward_device_pointers_and_params_roundtrip(orc):
    p64 = W.mlp_init(8)
    p32 = p64.astype(np.float32)
    net = sft.sft_mlp_create(torch.as_tensor(p32).to(DEV))
    assert np.array_equal(sft.sft_mlp_params(net), p32)
    X = torch.rand((4096, 3), device=DEV, dtype=torch.float32)
    out = torch.zeros(4096, device=DEV, dtype=torch.float32)
    sft.sft_mlp_forward(net, X, out=out)
    torch.cuda.synchronize()
    ref = orc.mlp_forward(_as_gpu_params(orc, p64), X.cpu().numpy().astype(np.float64), act_bf16=True)
    assert np.abs(out.cpu().numpy() - ref).max() / np.abs(ref).max() < 1e-2
