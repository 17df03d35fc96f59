"""Philox4x32-10 and the per-(generation, slot, attempt) word stream.

The generator is written from its definition in Salmon, Moraes, Dror and Shaw, "Parallel random
numbers: as easy as 1, 2, 3" (SC'11): a 4x32-bit counter and a 2x32-bit key; each of the ten
rounds multiplies counter words 0 and 2 by two fixed odd multipliers, splits each 64-bit product
into high and low halves, and mixes them with words 1 and 3 and the round key; the key is bumped
by the two Weyl constants between rounds.

EBIC.jl draws random numbers for initialisation, selection and mutation (Sec. 2.4, steps 1 and 5)
but does not name a generator.  Reading: Philox4x32-10 keyed by the run seed, with the counter
(generation, slot, attempt, block); the words of a stream are consumed in order x0..x3 of block 0,
then block 1, and so on.  A uniform integer in [0, n) is the high word of the 64-bit product w*n.

Test infrastructure only (see the package docstring).
"""

MASK32 = 0xFFFFFFFF
MUL0 = 0xD2511F53
MUL1 = 0xCD9E8D57
WEYL0 = 0x9E3779B9
WEYL1 = 0xBB67AE85
ROUNDS = 10


def philox4x32_10(counter, key):
    """One Philox4x32-10 block: counter (4 ints < 2**32), key (2 ints < 2**32) -> 4 words."""
    x0, x1, x2, x3 = (int(v) & MASK32 for v in counter)
    k0, k1 = (int(v) & MASK32 for v in key)
    for r in range(ROUNDS):
        if r:
            k0 = (k0 + WEYL0) & MASK32
            k1 = (k1 + WEYL1) & MASK32
        p0 = MUL0 * x0
        p1 = MUL1 * x2
        hi0, lo0 = p0 >> 32, p0 & MASK32
        hi1, lo1 = p1 >> 32, p1 & MASK32
        x0, x1, x2, x3 = hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0
    return (x0, x1, x2, x3)


def seed_key(seed):
    """The 64-bit run seed as the two key words (low word first)."""
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return (seed & MASK32, seed >> 32)


def uniform(n, word):
    """Uniform integer in [0, n) from one 32-bit word (multiply-high; its small bias is part of
    the specification and is the same on every implementation)."""
    return (int(word) * int(n)) >> 32


class WordStream:
    """Sequential 32-bit words of the stream (generation g, slot s, attempt a)."""

    def __init__(self, seed, g, s, a):
        self.key = seed_key(seed)
        self.ctr = [int(g) & MASK32, int(s) & MASK32, int(a) & MASK32, 0]
        self.buf = []
        self.used = 0

    def next(self):
        if not self.buf:
            self.buf = list(philox4x32_10(self.ctr, self.key))
            self.ctr[3] = (self.ctr[3] + 1) & MASK32
        self.used += 1
        return self.buf.pop(0)

    def below(self, n):
        return uniform(n, self.next())
