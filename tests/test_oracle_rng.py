"""Pins of the oracle's Philox4x32-10 and FNV-1a against their published test vectors."""

import os

from oracle.fnv import chromosome_hash, fnv1a64_bytes, tabu_key
from oracle.philox import WordStream, philox4x32_10, uniform

from conftest import GOLDEN


def read_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def test_philox_known_answers():
    rows = read_rows("philox4x32_10_kat.txt")
    assert len(rows) == 3
    for r in rows:
        v = [int(t, 16) for t in r]
        assert philox4x32_10(v[0:4], v[4:6]) == tuple(v[6:10])


def test_fnv1a64_known_answers():
    rows = read_rows("fnv1a64_kat.txt")
    assert len(rows) == 3
    for text, hexval in rows:
        assert fnv1a64_bytes(text.strip('"').encode()) == int(hexval, 16)


def test_chromosome_hash_is_order_sensitive_and_le_int32():
    assert chromosome_hash([1, 2]) != chromosome_hash([2, 1])
    assert chromosome_hash([0x61]) == fnv1a64_bytes(b"a\0\0\0")
    assert tabu_key(0) != 0 and tabu_key(5) == 5


def test_word_stream_consumes_blocks_in_order():
    s = WordStream(0x1234567890ABCDEF, 3, 7, 1)
    words = [s.next() for _ in range(9)]
    key = (0x90ABCDEF, 0x12345678)
    b0 = philox4x32_10((3, 7, 1, 0), key)
    b1 = philox4x32_10((3, 7, 1, 1), key)
    b2 = philox4x32_10((3, 7, 1, 2), key)
    assert words == list(b0) + list(b1) + [b2[0]]


def test_uniform_multiply_high():
    assert uniform(10, 0) == 0
    assert uniform(10, 0xFFFFFFFF) == 9
    assert uniform(1, 0xFFFFFFFF) == 0
    assert uniform(3, 0x80000000) == 1
