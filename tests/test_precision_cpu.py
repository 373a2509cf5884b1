"""The bf16 split storage of D (BF16_SPLIT mode), checked on the CPU with torch's
round-to-nearest-even conversions (the same rounding the library's conversion kernel uses):
hi = bf16(d) and lo = bf16(d - hi) reproduce an FP32 d to 2^-16 relative (bf16 keeps 8
significant bits, so rounding to it errs by at most 2^-8 relative, and lo carries the next 8
bits of d - hi), hi alone to 2^-8, and d - hi is exact in FP32."""
import numpy as np
import torch


def _split(d):
    hi = d.bfloat16()
    lo = (d - hi.float()).bfloat16()
    return hi, lo


def test_hi_lo_reproduce_fp32_to_2_pow_minus_17():
    g = torch.Generator().manual_seed(0)
    d = (torch.randn(1 << 16, generator=g) * torch.exp(torch.randn(1 << 16, generator=g) * 4)).float()
    hi, lo = _split(d)
    dd = d.double()
    rel_hi = ((hi.double() - dd).abs() / dd.abs()).max().item()
    rel_hl = ((hi.double() + lo.double() - dd).abs() / dd.abs()).max().item()
    assert rel_hi <= 2.0 ** -8
    assert rel_hl <= 2.0 ** -16
    # d - hi is exactly representable in FP32 (hi has 8 significant bits, d has 24)
    assert torch.equal((d.double() - hi.double()).float().double(), d.double() - hi.double())


def test_split_of_special_values():
    d = torch.tensor([0.0, -0.0, 1.0, -1.0, 2.0 ** -126, 3.0e38, 1.0 + 2.0 ** -23], dtype=torch.float32)
    hi, lo = _split(d)
    back = hi.double() + lo.double()
    assert np.all(np.abs(back.numpy() - d.double().numpy()) <= 2.0 ** -16 * np.abs(d.double().numpy()))
