"""SplitMix64 counter-based generator (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014; constants as published there).

Pure Python integers, so the stream is identical on every host and every
architecture.  Used only to draw synthetic inputs; it does none of the
integration arithmetic.
"""

_MASK = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15


class SplitMix64:
    """Sequential SplitMix64 stream starting from an integer seed."""

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + _GOLDEN) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1): the top 53 bits times 2**-53 (exact)."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi] (inclusive), by multiply-shift on 64 bits."""
        span = hi - lo + 1
        if span <= 0:
            raise ValueError("empty range")
        return lo + ((self.next_u64() * span) >> 64)

    def choice(self, seq):
        return seq[self.randint(0, len(seq) - 1)]

    def shuffle(self, lst):
        """In-place Fisher-Yates shuffle."""
        for i in range(len(lst) - 1, 0, -1):
            j = self.randint(0, i)
            lst[i], lst[j] = lst[j], lst[i]
        return lst
