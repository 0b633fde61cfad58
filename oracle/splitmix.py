"""Counter-based SplitMix64 streams (oracle side).

Published definition: Steele, Lea, Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014 (the ``mix64`` finaliser with constants
0xbf58476d1ce4e5b9 / 0x94d049bb133111eb and the golden gamma
0x9e3779b97f4a7c15).  The FD method draws random numbers in three places --
the on-site disorder of the Anderson matrices, the random start block of FD
(Sec. 2: FD starts from random search vectors) and the Lanczos start vector
(Sec. 2: the inclusion interval comes from a short Lanczos run) -- and these draws happen
inside the library, so each side implements this generator on its own:

    key(seed, stream) = mix64(seed XOR mix64(stream))
    x_i               = mix64(key + (i + 1) * GAMMA)        (mod 2^64)
    uniform u_i       = (x_i >> 11) * 2^-53                  in [0, 1)
    normal-like g_e   = (sum_{t<12} (x_{12 e + t} >> 11)) * 2^-53 - 6

The Irwin-Hall sum is taken in integer arithmetic (12 * 2^53 < 2^57) and
converted once, so its value does not depend on the order of additions.

Stream identifiers (fixed constants of this project):
    1 disorder, 2 start block, 3 Lanczos start vector, 4 KPM random vectors,
    5 instance size L, 6 instance disorder W, 7 road-graph tree, 8 road-graph extra edges.
"""
import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
M1 = np.uint64(0xBF58476D1CE4E5B9)
M2 = np.uint64(0x94D049BB133111EB)

STREAM_DISORDER = 1
STREAM_START = 2
STREAM_LANCZOS = 3
STREAM_KPM = 4
STREAM_INST_L = 5
STREAM_INST_W = 6
STREAM_ROAD_TREE = 7
STREAM_ROAD_EXTRA = 8


def mix64(z):
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * M1
        z = (z ^ (z >> np.uint64(27))) * M2
        return z ^ (z >> np.uint64(31))


def key(seed, stream):
    return mix64(np.uint64(seed) ^ mix64(np.uint64(stream)))


def raw(seed, stream, counters):
    """x_i for the given integer counters (array-like of int)."""
    c = np.asarray(counters, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(key(seed, stream) + (c + np.uint64(1)) * GAMMA)


def uniform(seed, stream, counters):
    x = raw(seed, stream, counters)
    return (x >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def irwin_hall(seed, stream, counters):
    """Normal-like draw g_e for each counter e (mean 0, variance 1)."""
    e = np.asarray(counters, dtype=np.uint64)
    base = e[..., None] * np.uint64(12) + np.arange(12, dtype=np.uint64)
    s = (raw(seed, stream, base) >> np.uint64(11)).sum(axis=-1, dtype=np.uint64)
    return s.astype(np.float64) * 2.0 ** -53 - 6.0
