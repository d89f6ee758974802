"""Philox4x32-10 counter-based generator and Box-Muller normals (oracle, test infrastructure).

The paper's preconditioner draws a standard normal test matrix Omega (§2.2).  Both this
oracle and the CUDA path generate it with the same published counter-based generator,
Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
1, 2, 3", SC'11), written here from that definition:

  round:  (c0, c1, c2, c3), (k0, k1) ->
          (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0))
          with M0 = 0xD2511F53, M1 = 0xCD9E8D57 (32 x 32 -> 64-bit products);
  key schedule: after each round k0 += 0x9E3779B9, k1 += 0xBB67AE85 (mod 2^32).

Normals: u = (bits + 0.5) 2^-32 in (0, 1); Box-Muller on the pairs (r0, r1), (r2, r3):
sqrt(-2 ln u_a) cos(2 pi u_b), sqrt(-2 ln u_a) sin(2 pi u_b).

Omega layout: element e = j * s + c of the row-major n x s matrix is normal number (e mod 4)
of the Philox block with counter (e div 4, stream, 0, 0) and key (seed lo, seed hi).

Pinned by the published known-answer vectors (tests/golden/philox4x32_10_kat.txt).
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint32(0x9E3779B9)
W1 = np.uint32(0xBB67AE85)
MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr, key):
    """ctr: uint32 array (..., 4); key: uint32 array (..., 2). Returns uint32 (..., 4)."""
    c = np.array(ctr, dtype=np.uint32, copy=True)
    k = np.array(key, dtype=np.uint32, copy=True)
    c = np.broadcast_to(c, np.broadcast_shapes(c.shape, k.shape[:-1] + (4,))).copy()
    k = np.broadcast_to(k, c.shape[:-1] + (2,)).copy()
    with np.errstate(over="ignore"):
        for r in range(10):
            p0 = M0 * c[..., 0].astype(np.uint64)
            p1 = M1 * c[..., 2].astype(np.uint64)
            hi0 = (p0 >> np.uint64(32)).astype(np.uint32)
            lo0 = (p0 & MASK).astype(np.uint32)
            hi1 = (p1 >> np.uint64(32)).astype(np.uint32)
            lo1 = (p1 & MASK).astype(np.uint32)
            c = np.stack([hi1 ^ c[..., 1] ^ k[..., 0], lo1, hi0 ^ c[..., 3] ^ k[..., 1], lo0],
                         axis=-1)
            if r < 9:
                k = np.stack([k[..., 0] + W0, k[..., 1] + W1], axis=-1)
    return c


def box_muller(bits4):
    """uint32 (..., 4) -> float64 (..., 4) standard normals."""
    u = (bits4.astype(np.float64) + 0.5) * 2.0 ** -32
    ra = np.sqrt(-2.0 * np.log(u[..., 0]))
    rb = np.sqrt(-2.0 * np.log(u[..., 2]))
    ta = 2.0 * np.pi * u[..., 1]
    tb = 2.0 * np.pi * u[..., 3]
    return np.stack([ra * np.cos(ta), ra * np.sin(ta), rb * np.cos(tb), rb * np.sin(tb)], axis=-1)


def omega(n, s, seed, stream=0):
    """Row-major n x s standard-normal test matrix with the layout described above."""
    total = n * s
    nblk = (total + 3) // 4
    ctr = np.zeros((nblk, 4), dtype=np.uint32)
    ctr[:, 0] = np.arange(nblk, dtype=np.uint64).astype(np.uint32)
    ctr[:, 1] = np.uint32(stream)
    key = np.array([seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF], dtype=np.uint32)
    g = box_muller(philox4x32_10(ctr, key)).reshape(-1)[:total]
    return g.reshape(n, s)
