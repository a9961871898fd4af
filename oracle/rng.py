"""Counter-based SplitMix64 streams (oracle side; test infrastructure only).

The paper draws its random quantities "uniformly at random" (Procedure OsGen, Sec. 6;
the random permutation of Sec. 4.1) without naming a generator, so the generator is a
choice of this project.  It is defined from the published SplitMix64 (Steele, Lea &
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014):

    state_{i+1} = state_i + 0x9E3779B97F4A7C15           (mod 2^64)
    output_i    = mix64(state_{i+1})
    mix64(z)    = z ^= z >> 30; z *= 0xBF58476D1CE4E5B9;
                  z ^= z >> 27; z *= 0x94D049BB133111EB; z ^= z >> 31

so the i-th output (0-based) of a generator started at state s0 is
``mix64(s0 + (i + 1) * gamma)`` and can be computed for any i independently.

A named stream ``tag`` of a seed starts at the ``tag``-th output of the generator
seeded with ``seed``; ``draw(seed, tag, i)`` is the i-th output of that stream.
A uniform double in [0, 1) is ``(u >> 11) * 2^-53``.

The CUDA side implements the same definition independently.
"""

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Stream tags.  Each random quantity of the generator draws from its own stream.
TAG_SIGMA = 1     # keys whose ranks assign the singular values to indices
TAG_PERM = 2      # keys whose argsort is the row permutation P (P1 = P2 = P, Sec. 4.1)
TAG_SUPPORT = 3   # keys whose s smallest select the support S of x* (OsGen, Sec. 6)
TAG_XVAL = 4      # magnitudes of the nonzeros of x*
TAG_XSIGN = 5     # signs of the nonzeros of x*
TAG_GOFF = 6      # subgradient entries g_i off the support (IGen, Sec. 3.1)
TAG_NROW = 7      # IGen2: row indices of the columns of N
TAG_NVAL = 8      # IGen2: values of the columns of N
TAG_XI = 9        # IGen2: the scalars xi (Sec. 3.2)


def mix64(z):
    """SplitMix64 (Steele, Lea & Flood 2014) finaliser applied elementwise to a uint64 array (wraps mod 2^64)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def splitmix_output(state0, index):
    """The ``index``-th output (0-based) of SplitMix64 (Steele, Lea & Flood 2014) started at
    ``state0``: the state advances by the golden-ratio increment, then the finaliser."""
    idx = np.asarray(index, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = np.uint64(state0) + (idx + np.uint64(1)) * GAMMA
    return mix64(state)


def stream_key(seed, tag):
    """Starting state of stream ``tag`` of ``seed`` (one stream per quantity the paper draws at
    random without naming a generator: keys of Sec. 4.1 and 6, magnitudes, signs)."""
    return np.uint64(splitmix_output(np.uint64(seed), np.array([tag], dtype=np.uint64))[0])


def draws(seed, tag, count, start=0):
    """Outputs ``start .. start+count-1`` of stream ``tag`` of ``seed`` (uint64 array)."""
    idx = np.arange(start, start + count, dtype=np.uint64)
    return splitmix_output(stream_key(seed, tag), idx)


def unit_uniform(u):
    """Map uint64 draws to doubles in [0, 1) with 53 random bits (the uniform draws of
    Sec. 3-6)."""
    u = np.asarray(u, dtype=np.uint64)
    return (u >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
