"""Random draws of Algorithm 1 -- TEST INFRASTRUCTURE ONLY (part of the oracle).

Algorithm 1 draws a random shift s from {-c*delta+1, ..., 0} for every k and a
Uniform(0,1) for every window j, but the paper fixes no generator.  Both the
oracle and the CUDA library therefore implement, separately, one
counter-based generator from its published definition: SplitMix64 (Steele,
Lea & Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014).

SplitMix64 with state S returns mix(S + n*G) as its n-th output (n = 1, 2, ...),
where G = 0x9E3779B97F4A7C15 and
    mix(z) = z ^ (z >> 31) after z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9,
                                    z = (z ^ (z >> 27)) * 0x94D049BB133111EB
(all arithmetic mod 2^64).

Draw layout (the reading this library takes):
    base_k   = output k+1 of SplitMix64 seeded with `seed`
    draw(k,n) = output n+1 of SplitMix64 seeded with base_k
    shift    s_k = -(draw(k, 0) mod c*delta)
    keep     U_{k,j} = (draw(k, j) >> 11) * 2^-53, window j kept iff U < q_j
"""
MASK = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15


def mix(z: int) -> int:
    z &= MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
    return z ^ (z >> 31)


def splitmix64_output(seed: int, n: int) -> int:
    """n-th output (n >= 1) of SplitMix64 seeded with `seed`."""
    return mix((seed + n * GOLDEN) & MASK)


def draw(seed: int, k: int, n: int) -> int:
    base = splitmix64_output(seed & MASK, k + 1)
    return splitmix64_output(base, n + 1)


def shift(seed: int, k: int, cdelta: int) -> int:
    """Shift s in {-cdelta+1, ..., 0} for the k-th repetition."""
    return -(draw(seed, k, 0) % cdelta)


def uniform(seed: int, k: int, j: int) -> float:
    """Uniform(0,1) draw for window j (j >= 1) of repetition k: a multiple of 2^-53."""
    return (draw(seed, k, j) >> 11) * (2.0 ** -53)
