"""SplitMix64 counter-style generator used for every seeded synthetic input.

SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014; finaliser constants as published by Vigna) adds the
golden-ratio increment to a 64-bit state and passes the state through a
three-step xor-shift/multiply mixer.  It is used here only to draw circuit
structure, angles, noise positions and rates; none of the noisy-simulation
arithmetic lives in this package.
"""

MASK64 = (1 << 64) - 1
GOLDEN_GAMMA = 0x9E3779B97F4A7C15
MIX1 = 0xBF58476D1CE4E5B9
MIX2 = 0x94D049BB133111EB


class SplitMix64:
    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + GOLDEN_GAMMA) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * MIX1) & MASK64
        z = ((z ^ (z >> 27)) * MIX2) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Float in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def uniform_range(self, lo: float, hi: float) -> float:
        return lo + (hi - lo) * self.uniform()

    def log_uniform(self, lo: float, hi: float) -> float:
        import math
        return math.exp(self.uniform_range(math.log(lo), math.log(hi)))

    def randbelow(self, m: int) -> int:
        """Unbiased integer in [0, m) by rejection on the top bits."""
        if m <= 0:
            raise ValueError("m must be positive")
        if m == 1:
            return 0
        bits = (m - 1).bit_length()
        while True:
            r = self.next_u64() >> (64 - bits)
            if r < m:
                return r

    def randint(self, lo: int, hi: int) -> int:
        """Integer in [lo, hi] inclusive."""
        return lo + self.randbelow(hi - lo + 1)

    def choice_distinct(self, m: int, k: int) -> list:
        """k distinct integers from [0, m), by a partial Fisher-Yates shuffle."""
        if k > m:
            raise ValueError("cannot draw more distinct values than the range holds")
        pool = list(range(m))
        for i in range(k):
            j = i + self.randbelow(m - i)
            pool[i], pool[j] = pool[j], pool[i]
        return pool[:k]

    def shuffle(self, xs: list) -> None:
        for i in range(len(xs) - 1, 0, -1):
            j = self.randbelow(i + 1)
            xs[i], xs[j] = xs[j], xs[i]
