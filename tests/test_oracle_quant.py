"""Pins for the oracle's reduced-precision stores: the format definitions checked against
torch's independent conversions and against hand-worked values."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")


def test_bf16_matches_torch_round_to_nearest_even():
    x = (np.random.default_rng(1).standard_normal((300, 40)) * 100).astype(np.float32)
    want = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(oracle.quantize_bf16(x), want)


def test_bf16_hand_values():
    # 1.0 = 0x3F80; 1 + 2^-8 is the tie between 0x3F80 and 0x3F81 -> even 0x3F80;
    # 1 + 3*2^-8 ties between 0x3F81 and 0x3F82 -> even 0x3F82; 255 is exact (8-bit mantissa).
    x = np.array([[1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, 255.0, -2.0]], np.float32)
    assert oracle.quantize_bf16(x).tolist() == [[0x3F80, 0x3F80, 0x3F82, 0x437F, 0xC000]]
    np.testing.assert_array_equal(oracle.decode("bf16", oracle.quantize_bf16(x)), [[1.0, 1.0, 1 + 2 ** -6, 255.0, -2.0]])


def test_fp8_matches_torch_e4m3fn_in_range():
    x = (np.random.default_rng(2).standard_normal((400, 48)) * 7).astype(np.float32)
    codes, scales = oracle.quantize_fp8(x)
    want = torch.from_numpy(x / scales[:, None]).to(torch.float8_e4m3fn).view(torch.uint8).numpy()
    assert np.array_equal(codes, want)
    np.testing.assert_allclose(scales, np.abs(x).max(1) / np.float32(448), rtol=0)


def test_fp8_hand_values_and_scale():
    # row max 448 -> s = 1. Codes: 448 = 1.75 * 2^8 -> e=15, m=6 -> 0x7E; 1.0 -> e=7 -> 0x38;
    # 2^-9 (smallest subnormal) -> 0x01; 3 * 2^-10 (tie between 2^-9 and 2^-8) -> even 2^-8 = 0x02;
    # 17 lies between 16 and 18 (spacing 2) -> tie -> even mantissa 16 = 0x58; -0.5 -> 0xB0.
    x = np.array([[448.0, 1.0, 2 ** -9, 3 * 2 ** -10, 17.0, -0.5]], np.float32)
    codes, scales = oracle.quantize_fp8(x)
    assert scales.tolist() == [1.0]
    assert codes.tolist() == [[0x7E, 0x38, 0x01, 0x02, 0x58, 0xB0]]
    np.testing.assert_array_equal(oracle.decode("fp8", codes, scales), [[448, 1, 2 ** -9, 2 ** -8, 16, -0.5]])
    # all-zero row -> scale 1, zero codes
    c0, s0 = oracle.quantize_fp8(np.zeros((1, 4), np.float32))
    assert s0.tolist() == [1.0] and c0.tolist() == [[0, 0, 0, 0]]


def test_fp8_relative_error_bound():
    # Normal E4M3 values carry 3 mantissa bits: |x - s*c| <= 2^-4 |x| above the subnormal range.
    x = (np.random.default_rng(3).random((100, 64)) + 0.5).astype(np.float32)
    codes, scales = oracle.quantize_fp8(x)
    dec = oracle.decode("fp8", codes, scales)
    assert np.all(np.abs(dec - x) <= 2 ** -4 * np.abs(x) + 1e-12)
