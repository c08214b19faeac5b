"""SplitMix64 (Steele, Lea & Flood 2014): a counter-based 64-bit generator.

Every random number of the synthetic workloads is drawn here, on the host,
and handed to both the CUDA path and the oracle as input.
"""

_MASK = (1 << 64) - 1


class SplitMix64:
    def __init__(self, seed: int = 0):
        self.state = seed & _MASK

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def symmetric(self, half_width: float) -> float:
        """Uniform double in [-half_width, half_width)."""
        return (2.0 * self.uniform() - 1.0) * half_width
