"""64-bit FNV-1a over a column sequence.

EBIC keeps "hashes" of evaluated individuals in a tabu list (Sec. 2.3, "EBIC" paragraph) but the
paper does not name the hash.  Reading: FNV-1a (Fowler, Noll, Vo), 64-bit variant, applied to the
column indices in chromosome order, each as four little-endian bytes of an int32.  It is order
sensitive, so a sequence and its reverse are different individuals, as the trend definition
requires.  The tabu-table key is the hash with the value 0 mapped to a fixed non-zero constant
(0 marks an empty slot in the device table); both sides apply the same map.

Test infrastructure only (see the package docstring).
"""

FNV64_OFFSET = 0xCBF29CE484222325
FNV64_PRIME = 0x100000001B3
MASK64 = 0xFFFFFFFFFFFFFFFF
ZERO_KEY_SUBSTITUTE = 0x9E3779B97F4A7C15


def fnv1a64_bytes(data):
    h = FNV64_OFFSET
    for byte in data:
        h ^= byte
        h = (h * FNV64_PRIME) & MASK64
    return h


def chromosome_hash(cols):
    """FNV-1a 64 of the int32 little-endian encoding of the column sequence."""
    data = bytearray()
    for c in cols:
        data += int(c).to_bytes(4, "little", signed=True)
    return fnv1a64_bytes(bytes(data))


def tabu_key(h):
    return ZERO_KEY_SUBSTITUTE if h == 0 else h
