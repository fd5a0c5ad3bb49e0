"""SplitMix64 counter-based uniform draws for random row selection.

The paper samples rows from a distribution (Sec. III-A for RK, the greedy
rule of Sec. IV-A for GRK) but names no generator.  Both the oracle and the
CUDA library implement, independently, the SplitMix64 generator of Steele,
Lea and Flood ("Fast splittable pseudorandom number generators", OOPSLA
2014): the state advances by the golden-ratio increment and each output is
the state passed through the 64-bit finaliser below.

Stream for (seed, instance, rhs): key = mix(seed + (instance * 2**32 + rhs + 1) * GOLDEN);
draw t (0-based) = mix(key + (t + 1) * GOLDEN) >> 11, scaled by 2**-53 into [0, 1).
"""
MASK = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15


def mix(z: int) -> int:
    z &= MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def splitmix64_sequence(state: int, n: int):
    """The plain sequential generator: n outputs starting from ``state``."""
    out = []
    for _ in range(n):
        state = (state + GOLDEN) & MASK
        out.append(mix(state))
    return out


def stream_key(seed: int, instance: int, rhs: int) -> int:
    return mix((seed + ((instance << 32) + rhs + 1) * GOLDEN) & MASK)


def uniform(seed: int, instance: int, rhs: int, t: int) -> float:
    key = stream_key(seed, instance, rhs)
    z = mix((key + (t + 1) * GOLDEN) & MASK)
    return (z >> 11) * (1.0 / 9007199254740992.0)
