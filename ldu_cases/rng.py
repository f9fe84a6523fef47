"""Counter-based random numbers for the synthetic inputs.

SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) written in its counter form: output k of a stream
with base state s is mix(s + (k + 1) * GOLDEN), so any slice of a stream can
be produced without generating what comes before it.  Uniform doubles take
the top 53 bits; normals use the Box-Muller transform (Box and Muller 1958).

This module holds no arithmetic of the solver; it only draws inputs.
"""
import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# one stream per purpose, so that changing one input leaves the others alone
TAGS = {
    "rhs": 1,
    "diffusivity": 2,
    "perm": 3,
    "aP": 4,
    "flux": 5,
    "sides": 6,
    "ref_diffusivity": 7,
    "probe": 8,
    "piso-flux": 9,
    "piso-dflux": 10,
}


def mix64(z):
    """The SplitMix64 finaliser on a uint64 array (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64).copy()
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
    return z


def stream_base(seed, tag, sub=0):
    """Base state of the stream for (seed, purpose tag, sub-stream index)."""
    t = TAGS[tag] if isinstance(tag, str) else int(tag)
    with np.errstate(over="ignore"):
        s = np.array([np.uint64(seed)], dtype=np.uint64)
        s = mix64(s + GOLDEN * np.uint64(t + 1))
        s = mix64(s ^ (np.uint64(sub) * _M2 + np.uint64(0x632BE59BD9B4E019)))
    return s[0]


def raw(base, count, start=0):
    """Outputs start .. start+count-1 of the SplitMix64 stream with state `base`."""
    k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(np.uint64(base) + k * GOLDEN)


def uniform01(base, count, start=0):
    """Doubles in [0, 1): (x >> 11) * 2^-53."""
    return (raw(base, count, start) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform(base, count, lo, hi, start=0):
    return lo + (hi - lo) * uniform01(base, count, start)


def normal(base, count, start=0):
    """Standard normals by Box-Muller; draw pair j uses outputs 2j and 2j+1."""
    m = (count + 1) // 2
    u1 = uniform01(base, 2 * m, 2 * start)
    a = 1.0 - u1[0::2]            # in (0, 1], keeps the log finite
    b = u1[1::2]
    rad = np.sqrt(-2.0 * np.log(a))
    z = np.empty(2 * m)
    z[0::2] = rad * np.cos(2.0 * np.pi * b)
    z[1::2] = rad * np.sin(2.0 * np.pi * b)
    return z[:count]


def permutation(base, count):
    """A random permutation: the stable argsort of one random key per item."""
    return np.argsort(raw(base, count), kind="stable").astype(np.int64)


def integers(base, count, lo, hi_inclusive, start=0):
    """Integers uniform in [lo, hi] by multiply-shift of the top 53 bits."""
    span = hi_inclusive - lo + 1
    u = uniform01(base, count, start)
    return lo + np.minimum((u * span).astype(np.int64), span - 1)
