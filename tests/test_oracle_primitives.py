"""Pins of the oracle's primitives: Philox4x64-10 against numpy's independent
implementation, log2 by the atanh series against the C library's log2."""
import math

import numpy as np
import pytest


def _numpy_block(ctr, key):
    """numpy.random.Philox increments its 256-bit counter before producing a
    block, so load counter - 1 and read four raw words."""
    c = sum(int(v) << (64 * i) for i, v in enumerate(ctr))
    c = (c - 1) % (1 << 256)
    bg = np.random.Philox(key=int(key[0]) | (int(key[1]) << 64))
    st = bg.state
    st["state"]["counter"] = np.array([(c >> (64 * i)) & ((1 << 64) - 1) for i in range(4)],
                                      dtype=np.uint64)
    st["buffer_pos"] = 4
    bg.state = st
    return bg.random_raw(4)


@pytest.mark.parametrize("ctr,key", [
    ((0, 0, 0, 0), (0, 0)),
    ((1, 0, 0, 0), (0, 0)),
    ((5, 17, 200, 3), (0, 0)),
    ((0, 255, 199, 3), (12345, 0)),
    ((2**64 - 1, 2**64 - 1, 2**64 - 1, 2**64 - 1), (2**64 - 1, 2**64 - 1)),
    ((0x243F6A8885A308D3, 0x13198A2E03707344, 0xA4093822299F31D0, 0x082EFA98EC4E6C89),
     (0x452821E638D01377, 0xBE5466CF34E90C6C)),
])
def test_philox_matches_numpy(oracle, ctr, key):
    ours = oracle.philox4x64_10(ctr, key)
    ref = _numpy_block(ctr, key)
    assert [int(x) for x in ours] == [int(x) for x in ref]


def test_draw32_layout(oracle):
    """Draw d = half (d&1) of 64-bit word (d>>1)&3 of block d>>3."""
    seed, slot, gen, tag = 99, 7, 3, 3
    for blk in range(3):
        words = oracle.philox4x64_10((blk, slot, gen, tag), (seed, 0))
        for w in range(4):
            lo = int(words[w]) & 0xFFFFFFFF
            hi = int(words[w]) >> 32
            d = blk * 8 + 2 * w
            assert oracle.draw32(seed, slot, gen, tag, d) == lo
            assert oracle.draw32(seed, slot, gen, tag, d + 1) == hi


def _ulp_err(a, b):
    return abs(a - b) / math.ulp(b) if b != 0 else abs(a)


def test_log2_det_against_libm(oracle):
    rng = np.random.default_rng(0)
    xs = list(1.0 + rng.random(4000) * 4)
    xs += list(10.0 ** rng.uniform(0, 300, 4000))
    xs += [1.0, 2.0, 4.0, 1.5, math.sqrt(2), math.sqrt(0.5) * 2, 1 + 2**-52, 1 + 2**-30,
           2 - 2**-52, 101.0, 7.25, 65.0, 1e308]
    worst = 0.0
    for x in xs:
        got = oracle.log2_det(x)
        ref = math.log2(x)
        if ref == 0:
            assert got == 0
            continue
        worst = max(worst, _ulp_err(got, ref))
    assert worst <= 4.0
    assert oracle.log2_det(1.0) == 0.0
    for e in range(0, 60):
        assert oracle.log2_det(2.0 ** e) == float(e)
    assert oracle.log2_det(math.inf) == math.inf
