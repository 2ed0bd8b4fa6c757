"""Counter-based Gaussian draws for the oracle (test infrastructure only).

The method samples two Gaussian matrices: G in Algorithm 1 (turned into the
orthogonal Q) and the test matrix of the truncated randomized SVD in
Algorithm 2 (and of the optional attribute reduction, Section 3.2.1). The
CUDA library draws them on the device from a seed; this module draws the
same numbers on the host from the published definition of the generator, so
neither side hands its random matrix to the other.

Generator: Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, "Parallel
random numbers: as easy as 1, 2, 3", SC'11): a 128-bit counter, a 64-bit key,
multipliers 0xD2511F53 / 0xCD9E8D57, Weyl key increments 0x9E3779B9 /
0xBB67AE85.

Mapping to Gaussians (a convention of this project, shared by contract with
the CUDA side): entry e (row-major) of a matrix drawn on ``stream`` uses the
counter (b mod 2^32, b >> 32, stream, 0) with b = e // 4 and the key
(seed mod 2^32, seed >> 32). The four output words give two Box-Muller
pairs: u = (x + 0.5) / 2^32, z_even = sqrt(-2 ln u_a) cos(2 pi u_b),
z_odd = sqrt(-2 ln u_a) sin(2 pi u_b), for (a, b) = (0, 1) and (2, 3);
entry e takes z[e mod 4], computed in float64.
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint32(0x9E3779B9)
W1 = np.uint32(0xBB67AE85)
MASK = np.uint64(0xFFFFFFFF)

# stream ids of the random matrices the method draws
STREAM_G = 1        # Algorithm 1: G (d x d) -> Q
STREAM_OMEGA_R = 2  # Algorithm 2: randomized SVD test matrix of R
STREAM_OMEGA_X = 3  # Section 3.2.1: randomized SVD test matrix of X_U


def philox4x32_10(ctr: np.ndarray, key: np.ndarray) -> np.ndarray:
    """Vectorised Philox4x32-10. ctr: uint32 [..., 4]; key: uint32 [..., 2] (broadcast)."""
    c = [np.asarray(ctr[..., i], dtype=np.uint32) for i in range(4)]
    k0 = np.asarray(key[..., 0], dtype=np.uint32)
    k1 = np.asarray(key[..., 1], dtype=np.uint32)
    with np.errstate(over="ignore"):
        for rnd in range(10):
            if rnd:
                k0 = (k0 + W0).astype(np.uint32)
                k1 = (k1 + W1).astype(np.uint32)
            p0 = M0 * c[0].astype(np.uint64)
            p1 = M1 * c[2].astype(np.uint64)
            hi0 = (p0 >> np.uint64(32)).astype(np.uint32)
            lo0 = (p0 & MASK).astype(np.uint32)
            hi1 = (p1 >> np.uint64(32)).astype(np.uint32)
            lo1 = (p1 & MASK).astype(np.uint32)
            c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return np.stack(c, axis=-1)


def gaussian_matrix(seed: int, stream: int, rows: int, cols: int) -> np.ndarray:
    """rows x cols standard-normal float64 matrix under the mapping in the module docstring."""
    n = rows * cols
    nb = (n + 3) // 4
    b = np.arange(nb, dtype=np.uint64)
    ctr = np.zeros((nb, 4), dtype=np.uint32)
    ctr[:, 0] = (b & MASK).astype(np.uint32)
    ctr[:, 1] = (b >> np.uint64(32)).astype(np.uint32)
    ctr[:, 2] = np.uint32(stream)
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint32)
    x = philox4x32_10(ctr, key).astype(np.float64)
    u = (x + 0.5) * 2.0 ** -32
    out = np.empty((nb, 4), dtype=np.float64)
    for a in (0, 2):
        rad = np.sqrt(-2.0 * np.log(u[:, a]))
        ang = 2.0 * np.pi * u[:, a + 1]
        out[:, a] = rad * np.cos(ang)
        out[:, a + 1] = rad * np.sin(ang)
    return out.reshape(-1)[:n].reshape(rows, cols)
