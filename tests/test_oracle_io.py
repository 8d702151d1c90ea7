"""Pins of the oracle's pixel-format helpers (the 16-bit and interleaved
inputs of Sec. 4.1): 16-bit and 8-bit codes agree where they name the same
value (65535 = 255 * 257), hand-written interleaved images decode to the
expected planes, 8-bit codes survive a decode/encode round trip, and the
identity transform maps 16-bit codes to round(v / 257) in 8 bits."""
import numpy as np
import pytest

import oracle
import svdlut_inputs as si


def test_u16_endpoints_and_agreement_with_u8():
    ends = oracle.u16_to_unit(np.array([0, 65535], dtype=np.uint16))
    assert ends[0] == 0.0 and ends[1] == 1.0
    v8 = np.arange(256, dtype=np.uint16)
    # 257 v / 65535 and v / 255 are the same rational, correctly rounded twice
    assert np.array_equal(oracle.u16_to_unit(v8 * 257), oracle.u8_to_unit(v8.astype(np.uint8)))
    all16 = oracle.u16_to_unit(np.arange(65536, dtype=np.uint16))
    assert np.all(np.diff(all16) > 0)


def test_interleaved_decode_of_a_hand_written_image():
    # 1 x 2 image, pixels (r, g, b) = (10, 20, 30) and (40, 50, 60)
    v = np.array([[[10, 20, 30], [40, 50, 60]]], dtype=np.uint8)
    x = oracle.decode(v, "u8_hwc")
    assert x.shape == (3, 1, 2)
    assert np.array_equal(x[0, 0], np.array([10, 40]) / 255.0)
    assert np.array_equal(x[1, 0], np.array([20, 50]) / 255.0)
    assert np.array_equal(x[2, 0], np.array([30, 60]) / 255.0)
    w = np.array([[[1000, 2000, 3000], [65535, 0, 7]]], dtype=np.uint16)
    x16 = oracle.decode(w, "u16_hwc")
    assert np.array_equal(x16[:, 0, 1], np.array([65535, 0, 7]) / 65535.0)
    assert np.array_equal(x16[:, 0, 0], np.array([1000, 2000, 3000]) / 65535.0)


def test_u8_round_trip_and_layouts():
    rng = np.random.default_rng(3)
    v = rng.integers(0, 256, (2, 3, 5, 7), dtype=np.uint8)
    assert np.array_equal(oracle.encode(oracle.decode(v, "u8"), "u8"), v)
    hwc = np.ascontiguousarray(np.moveaxis(v, 1, -1))
    assert np.array_equal(oracle.encode(oracle.decode(hwc, "u8_hwc"), "u8_hwc"), hwc)
    assert np.array_equal(oracle.decode(hwc, "u8_hwc"), oracle.decode(v, "u8"))


def test_identity_transform_16_to_8_bits():
    d = si.Dims(33, 8, 2, 5, 4, 9)
    p = si.identity_params(d)
    rng = np.random.default_rng(4)
    v = rng.integers(0, 65536, (3, 6, 11), dtype=np.uint16)
    v[:, 0, :4] = [[0, 128, 129, 65535]] * 3  # round(128 / 257) = 0, round(129 / 257) = 1
    y = oracle.forward_io(d, p, v, "u16", "u8")
    want = ((2 * v.astype(np.int64) + 257) // 514).astype(np.uint8)  # round(v / 257): no ties for integers
    assert np.array_equal(y, want)
    yh = oracle.forward_io(d, p, np.ascontiguousarray(np.moveaxis(v, 0, -1)), "u16_hwc", "u8_hwc")
    assert np.array_equal(yh, np.moveaxis(want, 0, -1))


def test_unknown_formats_are_rejected():
    with pytest.raises(ValueError):
        oracle.decode(np.zeros(3), "f16")
    with pytest.raises(ValueError):
        oracle.encode(np.zeros((3, 1, 1)), "u16")
