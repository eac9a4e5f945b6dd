"""Tensor-core kernels of the learned denoiser against plain float64 references."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N,K", [(128, 64, 64), (300, 48, 96), (1000, 256, 208), (77, 16, 16)])
def test_tcgen05_gemm_matches_float64(sde_gpu, M, N, K):
    import torch
    g = torch.Generator().manual_seed(M * 7 + N)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16)
    ref = A.double() @ B.double().T
    D = sde_gpu.gemm_bf16(A.cuda(), B.cuda()).cpu().double()
    err = (D - ref).abs().max().item()
    assert err <= 1e-4 * ref.abs().max().item() + 1e-4, err


def _torch_conv_ref(x, w, bias=None):
    """Plain PyTorch CPU float64 reference: x [n,D,H,W,C] channels-last, w [Cout,27,Cin]."""
    import torch
    import torch.nn.functional as F
    Cout, _, Cin = w.shape
    wt = w.double().reshape(Cout, 3, 3, 3, Cin).permute(0, 4, 1, 2, 3)
    y = F.conv3d(x.double().permute(0, 4, 1, 2, 3), wt, None if bias is None else bias.double(), padding=1)
    return y.permute(0, 2, 3, 4, 1)


@pytest.mark.parametrize("Cin,Cout,shape", [(16, 32, (4, 8, 8)), (32, 64, (3, 8, 16)), (96, 32, (2, 8, 8)),
                                            (192, 64, (2, 4, 16)), (64, 128, (4, 4, 8))])
def test_conv3d_forward_dgrad_wgrad_match_torch(sde_gpu, Cin, Cout, shape):
    import torch
    g = torch.Generator().manual_seed(Cin * 1000 + Cout)
    n = 2
    D, H, W = shape
    x = torch.randn(n, D, H, W, Cin, generator=g).to(torch.bfloat16)
    w = (0.2 * torch.randn(Cout, 27, Cin, generator=g)).to(torch.bfloat16)
    b = torch.randn(Cout, generator=g).float()
    ref = _torch_conv_ref(x, w, b)
    S = sde_gpu
    y = S.conv3d(x.cuda(), w.cuda(), b.cuda(), fp32=True)
    S.denoise_status()
    assert (y.cpu().double() - ref).abs().max().item() <= 1e-5 * ref.abs().max().item() + 1e-5
    yr = S.conv3d(x.cuda(), w.cuda(), b.cuda(), relu=True)  # BF16 output with ReLU
    S.denoise_status()
    assert (yr.cpu().double() - ref.clamp(min=0)).abs().max().item() <= 1e-2 * ref.abs().max().item()
    # gradients by autograd in float64
    xr = x.double().permute(0, 4, 1, 2, 3).clone().requires_grad_(True)
    wt = w.double().reshape(Cout, 3, 3, 3, Cin).permute(0, 4, 1, 2, 3).clone().requires_grad_(True)
    yt = torch.nn.functional.conv3d(xr, wt, padding=1)
    dy = torch.randn(yt.shape, generator=g, dtype=torch.float64).to(torch.bfloat16)
    yt.backward(dy.double())
    dx_ref = xr.grad.permute(0, 2, 3, 4, 1)
    dw_ref = wt.grad.permute(0, 2, 3, 4, 1).reshape(Cout, 27, Cin)
    dy_cl = dy.permute(0, 2, 3, 4, 1).contiguous().cuda()
    if Cin <= 256:
        wd = S.conv3d_flip_weights(w.cuda())
        dx = S.conv3d(dy_cl, wd, fp32=True)
        S.denoise_status()
        assert (dx.cpu().double() - dx_ref).abs().max().item() <= 1e-5 * dx_ref.abs().max().item() + 1e-5
    if Cout <= 128:
        dw = torch.zeros(Cout, 27, Cin, dtype=torch.float32, device="cuda")
        S.conv3d_wgrad(x.cuda(), dy_cl, dw)
        S.denoise_status()
        assert (dw.cpu().double() - dw_ref).abs().max().item() <= 1e-4 * dw_ref.abs().max().item() + 1e-4
