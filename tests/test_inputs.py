"""CPU pins of the seeded input module: the counter-based generator Philox4x32-10 against the
known-answer vectors published with it, and the statistics of the uniforms built from it."""
import torch

from paper_1806_03095_gb300 import inputs


def test_philox4x32_10_known_answers():
    cases = [
        ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
        ((0xFFFFFFFF,) * 4, (0xFFFFFFFF, 0xFFFFFFFF), (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
        ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
         (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
    ]
    for ctr, key, want in cases:
        got = inputs.philox4x32([[c] for c in ctr], key)
        assert tuple(int(w[0]) for w in got) == want


def test_philox_uniform_range_and_moments():
    u = inputs.philox_uniform(200001, 1806)
    assert u.dtype == torch.float64 and u.numel() == 200001
    assert float(u.min()) >= 0.0 and float(u.max()) < 1.0
    assert abs(float(u.mean()) - 0.5) < 3e-3
    assert abs(float(u.var()) - 1.0 / 12.0) < 2e-3
    # the 53-bit mantissa is filled: values are integer multiples of 2^-53, not of 2^-32
    k = u * 2.0 ** 53
    assert torch.equal(k, torch.round(k)) and bool(((k % 2 ** 21) != 0).any())
    # a different seed gives different numbers; the same seed the same
    assert not torch.equal(u[:100], inputs.philox_uniform(100, 1807))
    assert torch.equal(u[:100], inputs.philox_uniform(100, 1806))
