"""SplitMix64 pseudo-random generator (Steele, Lea and Flood, OOPSLA 2014).

Plain Python integers, so the stream is bit-identical on every machine and
every numpy version.  Used only to draw graphs and angles.
"""

_MASK = (1 << 64) - 1


class SplitMix64:
    """64-bit SplitMix generator: state += golden gamma, then a mix function."""

    GAMMA = 0x9E3779B97F4A7C15

    def __init__(self, seed: int):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + self.GAMMA) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def randbelow(self, k: int) -> int:
        """Integer in [0, k) by the multiply-high map of a 64-bit draw."""
        if k <= 0:
            raise ValueError("randbelow needs k > 0")
        return (self.next_u64() * k) >> 64

    def shuffle(self, items: list) -> None:
        """In-place Fisher-Yates shuffle."""
        for i in range(len(items) - 1, 0, -1):
            j = self.randbelow(i + 1)
            items[i], items[j] = items[j], items[i]
