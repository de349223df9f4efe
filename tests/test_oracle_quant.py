"""Pins of the oracle's reduced-precision roundings (CPU only).

The oracle writes its roundings from the bit layouts; these tests pin them to
hand-checkable values of the formats (ties to even, largest finite value,
subnormals) and to an independent library conversion (PyTorch's own
FP32 -> BF16 and FP32 -> float8_e4m3fn casts) on many random values.
"""
import numpy as np
import pytest
import torch

from oracle import quant as Q


def test_bf16_known_values():
    one = 1.0
    cases = {
        one: one,
        one + 2 ** -8: one,                      # halfway, ties to even (down)
        one + 3 * 2 ** -8: one + 2 ** -6,        # halfway, ties to even (up)
        one + 2 ** -8 + 2 ** -20: one + 2 ** -7,  # just above halfway
        -(one + 2 ** -7): -(one + 2 ** -7),     # representable
        3.4e38: float("inf"),                    # above (2 - 2^-8) 2^127: rounds to inf
        0.0: 0.0,
    }
    x = np.array(list(cases.keys()), np.float32)
    got = Q.bf16_rn(x)
    assert np.array_equal(got, np.array(list(cases.values()), np.float32))
    assert np.isnan(Q.bf16_rn(np.array([np.nan], np.float32))).all()


def test_bf16_matches_torch_cast():
    g = torch.Generator().manual_seed(0)
    x = torch.randn(200000, generator=g) * torch.exp2(torch.randint(-30, 30, (200000,), generator=g).float())
    got = Q.bf16_rn(x.numpy())
    want = x.to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(got, want)


def test_split_properties():
    g = torch.Generator().manual_seed(1)
    x = (torch.randn(100000, generator=g) * 10).numpy()
    hi, lo = Q.split_bf16(x)
    # hi and lo are BF16 values: their low 16 bits are zero
    assert not (hi.view(np.uint32) & 0xFFFF).any()
    assert not (lo.view(np.uint32) & 0xFFFF).any()
    # hi + lo is within 2^-16 |x| of x (two 8-bit significands, nearest rounding)
    err = np.abs(x.astype(np.float64) - hi.astype(np.float64) - lo.astype(np.float64))
    assert (err <= 2.0 ** -16 * np.abs(x.astype(np.float64))).all()
    # |lo| is at most half an ulp of hi
    assert (np.abs(lo) <= 2.0 ** -8 * np.abs(hi) + 1e-45).all()
    # values already in BF16 split into (x, 0)
    b = Q.bf16_rn(x)
    hb, lb = Q.split_bf16(b)
    assert np.array_equal(hb, b) and not lb.any()


def test_e4m3_known_values():
    cases = {
        448.0: 448.0, 1000.0: 448.0, -1e9: -448.0, 464.0: 448.0,  # saturate / tie to even
        1.0: 1.0, 1.0625: 1.0, 1.1875: 1.25, 1.125: 1.125,         # 3 fraction bits
        2.0 ** -9: 2.0 ** -9,                                        # smallest subnormal
        2.0 ** -10: 0.0,                                             # halfway to 0: even
        3 * 2.0 ** -10: 2.0 ** -8,                                   # halfway 1 -> 2 (even)
        2.0 ** -6: 2.0 ** -6, 0.0: 0.0, 240.0: 240.0, 250.0: 256.0,
    }
    x = np.array(list(cases.keys()), np.float32)
    assert np.array_equal(Q.e4m3_rn_sat(x), np.array(list(cases.values()), np.float32))


def test_e4m3_matches_torch_cast_in_range():
    if not hasattr(torch, "float8_e4m3fn"):
        pytest.skip("no float8 in this torch")
    g = torch.Generator().manual_seed(2)
    x = torch.randn(200000, generator=g) * torch.exp2(torch.randint(-12, 9, (200000,), generator=g).float())
    x = x.clamp(-448, 448)
    got = Q.e4m3_rn_sat(x.numpy())
    want = x.to(torch.float8_e4m3fn).to(torch.float32).numpy()
    assert np.array_equal(got, want)


def test_block_quant():
    g = torch.Generator().manual_seed(3)
    X = (torch.randn(300, 200, generator=g) * 5).numpy()
    X[:128, :128] = 0.0  # an all-zero block gets scale 1
    codes, s = Q.fp8_block_quant(X)
    assert s.shape == (3, 2) and s[0, 0] == 1.0
    for bi in range(3):
        for bj in range(2):
            blk = X[bi * 128:(bi + 1) * 128, bj * 128:(bj + 1) * 128]
            cb = codes[bi * 128:(bi + 1) * 128, bj * 128:(bj + 1) * 128]
            if np.abs(blk).max() > 0:
                # the largest element maps to the largest code
                assert np.abs(cb).max() == 448.0
                # normal-range codes carry 3 fraction bits: rel. error <= 2^-4
                rec = cb.astype(np.float64) * s[bi, bj]
                big = np.abs(cb) >= 2.0 ** -6
                rel = np.abs(rec - blk)[big] / np.abs(blk)[big]
                assert rel.max() <= 2.0 ** -4 * (1 + 1e-6)


def test_split3_properties():
    g = torch.Generator().manual_seed(4)
    # magnitudes over 2^-100 .. 2^100 (far from BF16's subnormal range)
    x = (torch.randn(200000, generator=g) *
         torch.exp2(torch.randint(-100, 100, (200000,), generator=g).float())).numpy()
    hi, mid, lo = Q.split3_bf16(x)
    for t in (hi, mid, lo):
        assert not (t.view(np.uint32) & 0xFFFF).any()  # BF16 values
    # the three parts carry x exactly: 8 + 8 + 8 significant bits with
    # nearest rounding cover FP32's 24
    total = hi.astype(np.float64) + mid.astype(np.float64) + lo.astype(np.float64)
    assert np.array_equal(total, x.astype(np.float64))
    # hi is the BF16 rounding of x (PyTorch's cast), mid is at most half an
    # ulp of hi, lo at most half an ulp of mid
    assert np.array_equal(hi, torch.from_numpy(x).to(torch.bfloat16).float().numpy())
    assert (np.abs(mid) <= 2.0 ** -8 * np.abs(hi)).all()
    assert (np.abs(lo) <= 2.0 ** -8 * np.abs(mid)).all()
    # the first two parts are the two-term split
    h2, l2 = Q.split_bf16(x)
    assert np.array_equal(h2, hi) and np.array_equal(l2, mid)
    # values with at most 8 (16) significant bits need one (two) parts
    b = Q.bf16_rn(x)
    hb, mb, lb = Q.split3_bf16(b)
    assert np.array_equal(hb, b) and not mb.any() and not lb.any()
    c = (x.view(np.uint32) & np.uint32(0xFFFFFF00)).view(np.float32)  # 16 bits
    hc, mc, lc = Q.split3_bf16(c)
    assert not lc.any() and np.array_equal(hc.astype(np.float64) + mc, c.astype(np.float64))
