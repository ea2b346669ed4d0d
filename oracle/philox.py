"""Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11), pure Python.

ORACLE / TEST INFRASTRUCTURE ONLY: imported by tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py, never by the product path.

Algorithm 2 step 3 (and Algorithm 1 step 2) re-draws the dual initial guess at random when
(r_0, rt_0) = 0.  The random numbers are part of the method's input, so the CPU oracle and
the CUDA library each implement this one published generator and draw identical bits.

Definition used (the paper's Philox4x32 with 10 rounds):
  round:  (hi0, lo0) = mulhilo32(0xD2511F53, c0); (hi1, lo1) = mulhilo32(0xCD9E8D57, c2)
          c <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0)
  key schedule between rounds: k0 += 0x9E3779B9, k1 += 0xBB67AE85 (mod 2^32).
Mapping to doubles (a choice of this project): element e of a vector drawn with 64-bit
seed s uses counter (e mod 2^32, e >> 32, 0, 0) and key (s mod 2^32, s >> 32); the top
53 bits of (w1 << 32 | w0) give u in [0, 1); the value is 2u - 1 in [-1, 1).  For complex
vectors the imaginary part uses (w3 << 32 | w2) the same way.
"""
from __future__ import annotations

import numpy as np

M0 = 0xD2511F53
M1 = 0xCD9E8D57
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    """One Philox4x32-10 block: ctr is 4 uint32, key is 2 uint32; returns 4 uint32."""
    c0, c1, c2, c3 = (int(v) & MASK for v in ctr)
    k0, k1 = (int(v) & MASK for v in key)
    for r in range(10):
        if r:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = M0 * c0
        p1 = M1 * c2
        hi0, lo0 = p0 >> 32, p0 & MASK
        hi1, lo1 = p1 >> 32, p1 & MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & MASK, lo1, (hi0 ^ c3 ^ k1) & MASK, lo0
    return c0, c1, c2, c3


def philox_vector(n, seed, complex_=False):
    """Vector of n values in [-1, 1) (complex: both parts), drawn as documented above.

    Vectorised over elements with numpy uint64 arithmetic (products of two 32-bit values
    fit in 64 bits exactly).
    """
    e = np.arange(n, dtype=np.uint64)
    c0 = e & np.uint64(MASK)
    c1 = e >> np.uint64(32)
    c2 = np.zeros(n, dtype=np.uint64)
    c3 = np.zeros(n, dtype=np.uint64)
    k0 = np.uint64(seed & MASK)
    k1 = np.uint64((seed >> 32) & MASK)
    m = np.uint64(MASK)
    for r in range(10):
        if r:
            k0 = np.uint64((int(k0) + W0) & MASK)
            k1 = np.uint64((int(k1) + W1) & MASK)
        p0 = np.uint64(M0) * c0
        p1 = np.uint64(M1) * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & m
        hi1, lo1 = p1 >> np.uint64(32), p1 & m
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & m, lo1, (hi0 ^ c3 ^ k1) & m, lo0
    two53 = float(2 ** 53)
    re = ((c1 << np.uint64(32)) | c0) >> np.uint64(11)
    out = 2.0 * (re.astype(np.float64) / two53) - 1.0
    if complex_:
        im = ((c3 << np.uint64(32)) | c2) >> np.uint64(11)
        out = out + 1j * (2.0 * (im.astype(np.float64) / two53) - 1.0)
    return out
